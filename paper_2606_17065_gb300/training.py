"""Training through the differentiable Jaeckel operator (Section 3.2; SPX appendix
"Differentiable IV inside the loss"; NaN-poisoning diagnostic).

A pricer emits prices P_hat, the operator maps them to implied volatilities
sigma_hat = JaeckelIV(P_hat) (``ImpliedVol``: CUDA LBR forward, gated IFT
backward), and an IV-space loss trains the pricer.  The pricer here is one
small MLP per synthetic SVI surface, batched over surfaces; its prices are
mapped into the open no-arbitrage interval (intrinsic, upper bound) by a
sigmoid so that every quote stays invertible.
"""
from __future__ import annotations

import math
import time

import torch

from . import api
from .workloads import SVIBatch


class SurfacePricer(torch.nn.Module):
    """One MLP 2 -> width x depth -> 1 (SiLU, FP32) per surface, weights batched over surfaces."""

    def __init__(self, n_surfaces: int, width: int = 128, depth: int = 4, seed: int = 0):
        super().__init__()
        g = torch.Generator().manual_seed(seed)
        dims = [2] + [width] * depth + [1]
        self.W = torch.nn.ParameterList()
        self.b = torch.nn.ParameterList()
        for fan_in, fan_out in zip(dims[:-1], dims[1:]):
            bound = 1.0 / math.sqrt(fan_in)
            self.W.append(torch.nn.Parameter((torch.rand(n_surfaces, fan_in, fan_out, generator=g) * 2 - 1) * bound))
            self.b.append(torch.nn.Parameter((torch.rand(n_surfaces, 1, fan_out, generator=g) * 2 - 1) * bound))

    def forward(self, X):  # X: [S, Q, 2] -> [S, Q]
        h = X
        for i, (W, b) in enumerate(zip(self.W, self.b)):
            h = torch.baddbmm(b, h, W)
            if i < len(self.W) - 1:
                h = torch.nn.functional.silu(h)
        return h.squeeze(-1)


def padded(batch: SVIBatch, device):
    """Quotes laid out [surface, slot] (padding repeats the surface's first quote, masked out)."""
    S, Q = batch.n_surfaces, batch.max_quotes
    idx = torch.zeros(S, Q, dtype=torch.long)
    mask = torch.zeros(S, Q, dtype=torch.bool)
    surf = torch.from_numpy(batch.surface).long()
    slot = torch.from_numpy(batch.slot).long()
    idx[surf, slot] = torch.arange(batch.n)
    mask[surf, slot] = True
    # quotes are grouped by surface: the first quote of surface j sits at searchsorted(surface, j)
    first = torch.searchsorted(surf.contiguous(), torch.arange(S))
    idx = torch.where(mask, idx, first[:, None].expand(S, Q))
    flat = idx.reshape(-1)
    t = lambda a: torch.from_numpy(a)[flat].to(device)  # noqa: E731
    F, K, T, sig = t(batch.F), t(batch.K), t(batch.T), t(batch.sigma_star)
    flag = torch.from_numpy(batch.flag)[flat].to(device)
    k = torch.from_numpy(batch.k)[flat].to(device)
    X = torch.stack([k / 0.3, torch.sqrt(T)], dim=-1).float().reshape(S, Q, 2)
    return X, F, K, T, flag, sig, mask.reshape(-1).to(device)


def train_iv_loss(batch: SVIBatch, steps: int = 100, lr: float = 1e-3, tau: float = 1e-6, gate: str = "smooth",
                  device=None, seed: int = 0):
    """Adam on the IV-space loss sum (sigma_hat - sigma*)^2 through ``ImpliedVol``.

    Returns a dict with the loss per step, the number of steps with a
    non-finite gradient, the fraction of quotes inside G_tau, and the time.
    """
    device = device or torch.device("cuda", torch.cuda.current_device())
    X, F, K, T, flag, sig_star, mask = padded(batch, device)
    call = flag > 0
    intrinsic = torch.where(call, (F - K).clamp_min(0), (K - F).clamp_min(0))
    upper = torch.where(call, F, K)
    model = SurfacePricer(batch.n_surfaces, seed=seed).to(device)
    opt = torch.optim.Adam(model.parameters(), lr=lr)
    losses, bad_steps, kept = [], 0, []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        o = model(X).reshape(-1).double()
        P_hat = intrinsic + (upper - intrinsic) * torch.sigmoid(o)
        sig_hat = api.ImpliedVol.apply(P_hat, F, K, T, flag, tau, gate)
        err = torch.where(mask, sig_hat - sig_star, torch.zeros_like(sig_hat))
        loss = (err * err).sum()
        opt.zero_grad(set_to_none=True)
        loss.backward()
        finite = all(bool(torch.isfinite(p.grad).all()) for p in model.parameters())
        bad_steps += 0 if finite else 1
        opt.step()
        losses.append(float(loss.detach()))
        with torch.no_grad():
            _, V = api.black_price(F, K, T, sig_hat.detach().nan_to_num(0.0), flag)
            kept.append(float(((V.abs() > tau) & mask).sum() / mask.sum()))
    torch.cuda.synchronize()
    return {"loss": losses, "nan_grad_steps": bad_steps, "iv_gate_kept": kept,
            "seconds": time.perf_counter() - t0, "quotes": int(mask.sum()), "rows": int(mask.numel())}


def per_quote_round_trip(batch, steps: int = 20, lr: float = 1e-2, gated: bool = True, tau: float = 1e-6,
                         device=None):
    """The NaN-poisoning diagnostic: one softplus parameter per quote, sigma_hat = softplus(theta),
    P_hat = Black(sigma_hat), sigma_rt = JaeckelIV(P_hat), loss = mean(w (sigma_rt - sigma*)^2).

    naive (gated=False): the operator's documented NaN branch off G_1e-14 and
    no weight, as in the paper's negative control; gated: smooth gate w_tau on
    the operator's backward and on the residual.  Returns the fraction of
    finite parameters and the loss after each step.
    """
    device = device or torch.device("cuda", torch.cuda.current_device())
    t = lambda a: torch.from_numpy(a).to(device)  # noqa: E731
    F, K, T, flag, sig_star = t(batch.F), t(batch.K), t(batch.T), t(batch.flag), t(batch.sigma_star)
    theta = torch.full_like(sig_star, math.log(math.expm1(0.3)), requires_grad=True)  # softplus^-1(0.3)
    opt = torch.optim.Adam([theta], lr=lr)
    finite_frac, losses = [], []
    for _ in range(steps):
        sig_hat = torch.nn.functional.softplus(theta)
        P_hat = api.BlackPrice.apply(sig_hat, F, K, T, flag)
        if gated:
            sig_rt = api.ImpliedVol.apply(P_hat, F, K, T, flag, tau, "smooth")
            with torch.no_grad():
                _, V = api.black_price(F, K, T, sig_hat.detach(), flag)
                w = V * V / (V * V + tau * tau)
            loss = (w * (sig_rt - sig_star) ** 2).mean()
        else:
            sig_rt = api.ImpliedVol.apply(P_hat, F, K, T, flag, 1e-14, "nan")
            loss = ((sig_rt - sig_star) ** 2).mean()
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        finite_frac.append(float(torch.isfinite(theta).float().mean()))
        losses.append(float(loss.detach()))
    return {"finite_frac": finite_frac, "loss": losses}


def operator_pairs(n: int, seed: int = 4, device=None):
    """Training pairs generated by the operator itself: quotes of the body distribution priced by
    ``black_price`` and inverted by ``iv`` (the sigma the library returns is the target)."""
    from . import workloads
    device = device or torch.device("cuda", torch.cuda.current_device())
    b = workloads.body_batch(n, seed=seed)
    t = lambda a: torch.from_numpy(a).to(device)  # noqa: E731
    F, K, T, flag = t(b.F), t(b.K), t(b.T), t(b.flag)
    P, _ = api.black_price(F, K, T, t(b.sigma_star), flag, vega=False)
    sig, _ = api.iv(F, K, T, P, flag, status=False)
    return F, K, T, P, flag, sig


def train_learned_guess(n_rows: int = 16 * 1024 * 1024, steps: int = 4000, batch: int = 65536, lr: float = 3e-3,
                        seed: int = 4, device=None, log_every: int = 250):
    """Train the MLP seed of PIVOT_MODE_LEARNED with the library's kernels (pivot_mlp_grad,
    pivot_mlp_adam) on ``n_rows`` operator-generated pairs; cosine-decayed Adam on random
    mini-batches.  Returns (trainer, history of (step, mean squared error), seconds)."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    F, K, T, P, flag, sig = operator_pairs(n_rows, seed=seed, device=device)
    trainer = api.MlpTrainer(device, seed=seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    history = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for step in range(steps):
        idx = torch.randint(0, F.numel(), (batch,), device=device, generator=gen)
        trainer.grad(F[idx], K[idx], T[idx], P[idx], flag[idx], sig[idx])
        if step % log_every == 0 or step == steps - 1:
            _, _, loss_sum, rows, _ = trainer.fields()
            history.append((step, loss_sum / max(rows, 1.0)))
        lr_t = 0.5 * lr * (1.0 + math.cos(math.pi * step / steps))
        trainer.adam(lr_t)
    torch.cuda.synchronize()
    return trainer, history, time.perf_counter() - t0
