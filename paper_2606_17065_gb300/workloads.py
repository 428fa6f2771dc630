"""Seeded synthetic option batches (input generators only).

This module draws the random inputs of each workload and nothing else: it
holds none of the method's arithmetic (no Black price, no inversion, no
adjoint).  Both the CUDA path (bench, tests) and the CPU oracle (tests) take
their inputs from here, so the two always see identical rows.

The prices P of the synthetic rows are *not* produced here: they come from a
Black-76 price evaluated by the caller (the oracle in tests, the library's
``black_price`` in the benchmark), exactly as the paper builds its synthetic
batches from a known sigma* (Section 4.1, "Gradient correctness").  The only
prices set here are the boundary quotes of the stress workload, which the
workload defines directly as a relative offset from the intrinsic value or
from the upper bound.

Layout: structure of arrays, float64 F, K, T, sigma_star and int8 flag
(+1 call, -1 put); r = 0 (forward measure), so P is the undiscounted price.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

#: rows in the plain FP64 workload of 4,096 options (ln(K/F) ~ U[-1, 1])
SMALL_N = 4096
#: rows in the 16M-option stress workload (ln(K/F) ~ U[-6, 6])
STRESS_N = 16 * 1024 * 1024
#: rows in the 64M-option mixed-precision / learned-guess workloads
LARGE_N = 64 * 1024 * 1024


@dataclass
class Batch:
    F: np.ndarray
    K: np.ndarray
    T: np.ndarray
    sigma_star: np.ndarray
    flag: np.ndarray
    #: price fixed by the workload itself (boundary quotes), NaN elsewhere
    P_fixed: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.F.shape[0])

    def subset(self, idx) -> "Batch":
        return Batch(self.F[idx], self.K[idx], self.T[idx], self.sigma_star[idx], self.flag[idx],
                     None if self.P_fixed is None else self.P_fixed[idx])


def _flags(rng, n):
    return np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)


def body_batch(n: int = SMALL_N, seed: int = 1) -> Batch:
    """F = 100, ln(K/F) ~ U[-1,1], T ~ U[1/365, 3], sigma* ~ U[0.05, 1], calls/puts 50/50.

    The paper's canonical synthetic grid (Section 4.1, Table 1: 1e5 synthetic
    options; IV band [0.05, 1.0] of Section 2) with 4,096 rows; the same
    distribution at 64M rows is the mixed-precision workload.
    """
    rng = np.random.default_rng(seed)
    F = np.full(n, 100.0)
    k = rng.uniform(-1.0, 1.0, n)
    K = F * np.exp(k)
    T = rng.uniform(1.0 / 365.0, 3.0, n)
    sig = rng.uniform(0.05, 1.0, n)
    return Batch(F, K, T, sig, _flags(rng, n))


def stress_batch(n: int = STRESS_N, seed: int = 2, boundary_frac: float = 0.05) -> Batch:
    """ln(K/F) ~ U[-6,6], s = sigma sqrt(T) log-uniform on [1e-4, 3], T ~ U[1/365, 3].

    A fraction ``boundary_frac`` of quotes sits within 1e-12 relative of a
    bound of the no-arbitrage interval: half are in-the-money quotes at
    P = intrinsic * (1 + u 1e-12), half at P = U (1 - u 1e-12) with U = F for
    calls and K for puts, u ~ U(0, 1].  The paper's low-vega stress chain
    (Section 4 appendix, "NaN-poisoning diagnostic": deep wings, expiries down
    to 1e-8 years) motivates the ranges.
    """
    rng = np.random.default_rng(seed)
    F = np.full(n, 100.0)
    k = rng.uniform(-6.0, 6.0, n)
    K = F * np.exp(k)
    T = rng.uniform(1.0 / 365.0, 3.0, n)
    s = np.exp(rng.uniform(np.log(1e-4), np.log(3.0), n))
    sig = s / np.sqrt(T)
    flag = _flags(rng, n)
    P_fixed = np.full(n, np.nan)
    nb = int(round(boundary_frac * n))
    if nb:
        idx = rng.choice(n, size=nb, replace=False)
        u = 1.0 - rng.random(nb)  # (0, 1]
        near_intrinsic = np.arange(nb) < nb // 2
        i1, u1 = idx[near_intrinsic], u[near_intrinsic]
        # in the money: a call when F > K, a put otherwise
        flag[i1] = np.where(F[i1] > K[i1], 1, -1).astype(np.int8)
        itm = np.where(flag[i1] > 0, F[i1] - K[i1], K[i1] - F[i1])
        P_fixed[i1] = itm * (1.0 + u1 * 1e-12)
        i2, u2 = idx[~near_intrinsic], u[~near_intrinsic]
        upper = np.where(flag[i2] > 0, F[i2], K[i2])
        P_fixed[i2] = upper * (1.0 - u2 * 1e-12)
    return Batch(F, K, T, sig, flag, P_fixed)


def merge_prices(batch: Batch, P_model: np.ndarray) -> np.ndarray:
    """Prices of the batch: the workload's fixed boundary quotes where set, else ``P_model``."""
    if batch.P_fixed is None:
        return P_model
    return np.where(np.isnan(batch.P_fixed), P_model, batch.P_fixed)


def sample_indices(n: int, m: int, seed: int = 12345) -> np.ndarray:
    """Deterministic sorted sample of m distinct row indices out of n."""
    rng = np.random.default_rng(seed)
    m = min(m, n)
    return np.sort(rng.choice(n, size=m, replace=False))


@dataclass
class SVIBatch:
    """Ragged quotes on synthetic SVI surfaces (flat arrays, one entry per quote)."""
    surface: np.ndarray  # int32 surface index of each quote
    slot: np.ndarray     # int32 position of the quote within its surface
    k: np.ndarray        # ln(K/F)
    F: np.ndarray
    K: np.ndarray
    T: np.ndarray
    flag: np.ndarray
    sigma_star: np.ndarray
    n_surfaces: int
    max_quotes: int

    @property
    def n(self) -> int:
        return int(self.F.shape[0])


SVI_MATURITIES = (1 / 12, 1 / 6, 1 / 4, 1 / 2, 3 / 4, 1.0, 1.5, 2.0)


def svi_batch(n_surfaces: int = 1024, seed: int = 5, min_quotes: int = 50, max_quotes: int = 400) -> SVIBatch:
    """Synthetic raw-SVI surfaces (the parameterisation the paper cites in its appendix on IV as the
    working coordinate): a ~ U[.01,.05], b ~ U[.05,.3], rho ~ U[-.8,.2], m ~ U[-.1,.1],
    s ~ U[.05,.3]; 50-400 quotes per surface over 8 maturities, k = ln(K/F) ~ U[-0.3, 0.3], F = 100.
    w(k) = a + b (rho (k - m) + sqrt((k - m)^2 + s^2)) is read as annualised variance, sigma = sqrt(w).
    """
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.01, 0.05, n_surfaces)
    b = rng.uniform(0.05, 0.3, n_surfaces)
    rho = rng.uniform(-0.8, 0.2, n_surfaces)
    m = rng.uniform(-0.1, 0.1, n_surfaces)
    s = rng.uniform(0.05, 0.3, n_surfaces)
    nq = rng.integers(min_quotes, max_quotes + 1, n_surfaces)
    surface = np.repeat(np.arange(n_surfaces, dtype=np.int32), nq)
    slot = np.concatenate([np.arange(q, dtype=np.int32) for q in nq])
    n = surface.shape[0]
    k = rng.uniform(-0.3, 0.3, n)
    T = np.asarray(SVI_MATURITIES)[rng.integers(0, len(SVI_MATURITIES), n)]
    km = k - m[surface]
    w = a[surface] + b[surface] * (rho[surface] * km + np.sqrt(km * km + s[surface] ** 2))
    F = np.full(n, 100.0)
    return SVIBatch(surface, slot, k, F, F * np.exp(k), T, _flags(rng, n), np.sqrt(w), n_surfaces, int(nq.max()))


def low_vega_chain(n: int = 65536, seed: int = 31) -> Batch:
    """The paper's low-vega stress chain (appendix, NaN-poisoning diagnostic): deep wings,
    T log-uniform on [1e-8, 10^-0.5] years, |ln(K/F)| <= 2.5, out-of-the-money quotes, F = 100,
    sigma* ~ U[0.05, 1] (the paper does not give its sigma range)."""
    rng = np.random.default_rng(seed)
    F = np.full(n, 100.0)
    k = rng.uniform(-2.5, 2.5, n)
    T = np.exp(rng.uniform(np.log(1e-8), np.log(10 ** -0.5), n))
    sig = rng.uniform(0.05, 1.0, n)
    flag = np.where(k > 0, 1, -1).astype(np.int8)
    return Batch(F, F * np.exp(k), T, sig, flag)


@dataclass
class BSBatch:
    """Rows of the Black-Scholes interface: xi = (S, K, tau, r, q) and the flag (Section 2)."""
    S: np.ndarray
    K: np.ndarray
    T: np.ndarray
    r: np.ndarray
    q: np.ndarray
    sigma_star: np.ndarray
    flag: np.ndarray

    @property
    def n(self) -> int:
        return int(self.S.shape[0])

    def subset(self, idx) -> "BSBatch":
        return BSBatch(*(getattr(self, f)[idx] for f in ("S", "K", "T", "r", "q", "sigma_star", "flag")))


def bs_batch(n: int = SMALL_N, seed: int = 6, wide: bool = False) -> BSBatch:
    """S = 100, ln(K/S) ~ U[-1,1] (U[-6,6] with ``wide``), T ~ U[1/365, 3], sigma* ~ U[0.05, 1]
    (s = sigma sqrt(T) log-uniform on [1e-4, 3] with ``wide``), r ~ U[-0.01, 0.08],
    q ~ U[0, 0.05], calls/puts 50/50.

    The spot-coordinate form of the canonical grid: rates and dividend yields of listed
    equity-index options, negative rates included (Section 2, the tuple xi).  The
    discounted prices V come from a Black-Scholes price evaluated by the caller.
    """
    rng = np.random.default_rng(seed)
    S = np.full(n, 100.0)
    K = S * np.exp(rng.uniform(-6.0, 6.0, n) if wide else rng.uniform(-1.0, 1.0, n))
    T = rng.uniform(1.0 / 365.0, 3.0, n)
    if wide:
        sig = 10.0 ** rng.uniform(-4.0, np.log10(3.0), n) / np.sqrt(T)
    else:
        sig = rng.uniform(0.05, 1.0, n)
    r = rng.uniform(-0.01, 0.08, n)
    q = rng.uniform(0.0, 0.05, n)
    return BSBatch(S, K, T, r, q, sig, _flags(rng, n))
