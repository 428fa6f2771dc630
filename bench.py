"""Benchmark: IV inversions/s, forward + backward, on the 16M-option stress batch.

One step = one pivot_iv_forward_backward call over the whole batch (every row
of the hot path: normalise, LBR boundary, rational guess, Householder(3)
steps, sigma, gated IFT adjoint), inputs resident in HBM.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--rows R]

--impl reference times the CPU oracle (the reference arm of this build) on a
bounded sample of the same workload.  --rows runs a smaller batch of the same
distribution (profiling only; the default is the full workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2606_17065_gb300 import workloads  # noqa: E402

METRIC = "IV inversions/s fwd+bwd on 1 GB300 (plain FP64, <=1e-13 rel err)"
UNIT = "inversions/s"
TAU = 1e-6
GATE = "nan"
WORKLOAD = ("stress-16M: ln(K/F)~U[-6,6], sigma*sqrt(T) log-uniform [1e-4,3], T~U[1/365,3], "
            "5% quotes within 1e-12 rel of intrinsic/upper bound, float64 SoA, fwd+bwd gate=nan tau=1e-6")

# Bytes per row moved by one fused forward+backward: F, K, T, P (4 x 8) + flag (1)
# in; sigma (8) + status (1) + dP, dF, dK, dT (4 x 8) out.
BYTES_PER_ROW = 33 + 41
# FP64 FLOPs per row of the fused kernel on this workload, counted by ncu
# (smsp__sass_thread_inst_executed_op_{dadd,dmul}_pred_on + 2 x ..._dfma_pred_on
# over one launch of 4,194,304 stress rows, divided by the rows), see
# profiles/k_iv_binned_fwdbwd_stress.md.  Counts scale with the rows: every
# launch of the same distribution does the same work per row on average.
FLOPS_PER_ROW = 235.1
# dram__bytes_read.sum + dram__bytes_write.sum per row of the current kernel (one launch of
# 4,194,304 stress rows, profiles/k_iv_binned_fwdbwd_stress.md).
TRAFFIC_PER_ROW = 125.6
# Executed FLOPs per row of the other measured forms, counted by ncu the same way on one launch
# of 4,194,304 rows of each workload (python bench.py --case <name> --rows 4194304; FP32 from
# smsp__sass_thread_inst_executed_op_{fadd,fmul}_pred_on + 2 x ..._ffma_pred_on), see
# profiles/flops_per_row_all_forms.md.
FLOPS = {
    # case: (FP64 FLOP / row, FP32 FLOP / row)
    "stress": (FLOPS_PER_ROW, 72.6),
    "stress-mixed": (93.0, 232.0),
    "body": (502.0, 124.4),
    "body-mixed": (214.2, 508.9),
    "body-learned": (213.5, 1589.0),
    "bs-wide": (320.5, 86.2),
    "bs-wide-mixed": (155.6, 272.1),
}
# MLP inference of the learned seed, 2 -> 64 -> 64 -> 64 -> 1: 2 (2 64 + 64 64 + 64 64 + 64) FLOP
# per seeded row on the BF16 tensor cores (algorithmic count)
MLP_FLOPS_PER_ROW = 2 * (2 * 64 + 64 * 64 + 64 * 64 + 64)
# FP64 peak derived from unit counts and clocks: 152 SMs x 2 DFMA lanes/clk x 2 FLOP
# (= 1.25 TFLOP/s nominal at 2.07 GHz), scaled by the SM clock seen under load; FP32:
# 128 FFMA lanes/clk/SM.
SMS = 152
FP64_FLOP_PER_CLK_PER_SM = 4.0
FP32_FLOP_PER_CLK_PER_SM = 256.0
HBM_PEAK_FALLBACK = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rows", type=int, default=workloads.STRESS_N)
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="target wall time of the CPU oracle sample")
    ap.add_argument("--case", default=None, choices=sorted(FLOPS),
                    help="time one form on --rows rows of its workload only (profiling captures)")
    ap.add_argument("--probe", action="store_true", help="only the unit throughput probes (profiling captures)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        load = [v for v in sm if smax and v > 0.3 * smax] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    rank, world = 0, 1
    if args.gpus > 1 or "WORLD_SIZE" in os.environ:
        import torch.distributed as dist
        world = int(os.environ.get("WORLD_SIZE", args.gpus))
        rank = int(os.environ.get("RANK", 0))
        if world > 1:
            import torch
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend=backend)
    return rank, world


def shard_seed(rank: int) -> int:
    """Each rank draws its own independent rows (weak scaling): seed 2 + rank."""
    return 2 + rank


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_rate(target_seconds: float, seed: int = 2, threads: int | None = None):
    """Forward+backward rows/s of the CPU oracle on a bounded sample of the stress workload."""
    import oracle
    threads = threads or oracle.max_threads()
    pilot = workloads.stress_batch(4096, seed=seed + 1000)
    P, _ = oracle.black_price(pilot.F, pilot.K, pilot.T, pilot.sigma_star, pilot.flag, nthreads=threads)
    P = workloads.merge_prices(pilot, P)
    t0 = time.perf_counter()
    sig, _ = oracle.implied_vol(pilot.F, pilot.K, pilot.T, P, pilot.flag, nthreads=threads)
    oracle.iv_grad(pilot.F, pilot.K, pilot.T, pilot.flag, sig, None, TAU, 1, nthreads=threads)
    rate = pilot.n / max(time.perf_counter() - t0, 1e-6)
    n = int(min(max(rate * target_seconds, 4096), 4_000_000))
    b = workloads.stress_batch(n, seed=seed + 2000)
    P, _ = oracle.black_price(b.F, b.K, b.T, b.sigma_star, b.flag, nthreads=threads)
    P = workloads.merge_prices(b, P)
    t0 = time.perf_counter()
    sig, _ = oracle.implied_vol(b.F, b.K, b.T, P, b.flag, nthreads=threads)
    oracle.iv_grad(b.F, b.K, b.T, b.flag, sig, None, TAU, 1, nthreads=threads)
    dt = time.perf_counter() - t0
    return n / dt, threads, n, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    per_step, threads, n, dt = [], None, None, 0.0
    if args.warmup > 0:
        oracle_rate(min(1.0, args.cpu_seconds / 4))
    for _ in range(max(args.steps, 1)):
        r, threads, n, d = oracle_rate(args.cpu_seconds / max(args.steps, 1))
        per_step.append(r)
        dt += d
    value = statistics.median(per_step)
    sample = f"{n} rows of the stress workload per step (seeded), fwd+bwd, oracle with OpenMP"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "rows_per_step": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def time_variant(fn, n, stream, reps):
    """Mean ms per call of fn (after 2 untimed calls) on `stream`, and its rate."""
    import torch
    for _ in range(2):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms}


def unit_peaks(dev, stream, sm_mhz):
    """Measured throughput of the FP64 and FP32 fma pipes and of MUFU (pivot_probe_units): a
    pilot launch sizes each probe to ~25 ms, then the best of 3 timed launches (CUDA events)."""
    import torch

    import paper_2606_17065_gb300 as pv
    out = {}
    for unit, iters0 in (("fp64_fma", 64), ("fp32_fma", 4096), ("mufu_ex2", 512), ("mufu_tanh", 512)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def timed(iters):
            torch.cuda.synchronize()
            e0.record(stream)
            ops = pv.api.probe_units(unit, iters, device=dev)
            e1.record(stream)
            torch.cuda.synchronize()
            return ops, e0.elapsed_time(e1)

        timed(iters0)
        ops, ms = timed(iters0)
        iters = max(int(iters0 * 25.0 / max(ms, 1e-3)), 1)
        best = 0.0
        for _ in range(3):
            ops, ms = timed(iters)
            best = max(best, ops / (ms * 1e-3))
        rec = {"lane_ops_per_s": best, "per_sm_per_clk": best / (SMS * sm_mhz * 1e6), "iters": iters}
        if unit.endswith("fma"):
            rec["flop_per_s"] = 2 * best
        out[unit] = rec
    return out


def stream_probe(F, K, T, P, flag, outs, stream, reps):
    """HBM rate of the 74-byte rows with 64-bit and with 128-bit accesses (pivot_probe_stream)."""
    import paper_2606_17065_gb300 as pv
    n = F.numel()
    res = {}
    for width in (1, 2):
        r = time_variant(lambda: pv.api.probe_stream(width, F, K, T, P, flag, outs), n, stream, reps)
        res[f"width{width}"] = {"gb_per_s": BYTES_PER_ROW * n / (r["ms_per_step"] * 1e-3) / 1e9,
                                "ms": r["ms_per_step"]}
    return res


def variant_roofline(case, rows, ms, peaks, sm_mhz, tensor_rows=0):
    """Roofline of one timed form: the time its executed FP64 work needs at the FP64 peak, plus
    its FP32 work at the FP32 peak (and MLP work at the BF16 tensor peak), against the measured
    time.  Peaks derived from unit counts x the sampled clock; measured ones (unit probes) beside."""
    f64, f32 = FLOPS.get(case, (None, None))
    if f64 is None:
        return {"case": case, "flops_per_row": None, "note": "FLOPs per row not yet counted by ncu on this kernel"}
    p64 = SMS * FP64_FLOP_PER_CLK_PER_SM * sm_mhz * 1e6
    p32 = SMS * FP32_FLOP_PER_CLK_PER_SM * sm_mhz * 1e6
    ptc = measured_peaks().get("bf16_tflops_sustained", 1728.1) * 1e12
    t = f64 * rows / p64 + (f32 or 0.0) * rows / p32 + MLP_FLOPS_PER_ROW * tensor_rows / ptc
    rec = {"case": case, "bound": "alu", "flops_per_row": {"fp64": f64, "fp32": f32},
           "achieved_fp64_tflops": f64 * rows / (ms * 1e-3) / 1e12, "peak_fp64_tflops": p64 / 1e12,
           "frac": t / (ms * 1e-3)}
    if peaks:
        m64 = peaks["fp64_fma"]["flop_per_s"]
        m32 = peaks["fp32_fma"]["flop_per_s"]
        tm = f64 * rows / m64 + (f32 or 0.0) * rows / m32 + MLP_FLOPS_PER_ROW * tensor_rows / ptc
        rec["frac_of_measured_units"] = tm / (ms * 1e-3)
    if tensor_rows:
        rec["mlp_rows"] = tensor_rows
        rec["mlp_flops_per_seeded_row"] = MLP_FLOPS_PER_ROW
    return rec


BIN_NAMES = {
    0: ["lower", "mid-low", "mid-high", "upper", "mid-low near money", "mid-high near money",
        "lower beta<1e-100", "lower near money"],
    1: ["float lower", "float mid-low", "float mid-high", "float upper", "fp64 lower", "fp64 mid-low",
        "fp64 mid-high", "fp64 upper", "float deep lower (ln beta)", "float mid-low near money",
        "float mid-high near money", "float lower near money"],
    2: ["mlp lower", "mlp b-beta", "mlp upper", "deep lower (ln beta)", "mlp lower near money",
        "mlp b-beta near money"],
}


def counters_summary(c, mode):
    """The per-launch counters (include/pivot.h) as fractions of the rows."""
    c = [int(v) for v in c.tolist()]
    rows = sum(c[0:6])
    solved = max(c[0], 1)
    names = BIN_NAMES[mode]
    return {"rows": rows, "status_frac": {str(k): c[k] / max(rows, 1) for k in range(6)},
            "bins_frac_of_solved": {names[k]: c[6 + k] / solved for k in range(len(names))},
            "rejected_accelerated_frac_of_solved": c[18] / solved}


def oracle_reference(F, K, T, P, flag, threads=None):
    """The CPU oracle's sigma, status and conditioning kappa_P = P/(sigma V) on given rows."""
    import oracle
    threads = threads or oracle.max_threads()
    t0 = time.perf_counter()
    ref, st_ref = oracle.implied_vol(F, K, T, P, flag, nthreads=threads)
    secs = time.perf_counter() - t0
    _, V = oracle.black_price(F, K, T, np.where(np.isfinite(ref), ref, 1.0), flag, nthreads=threads)
    with np.errstate(divide="ignore", invalid="ignore"):
        kp = P / (ref * V)
    return {"ref": ref, "st": st_ref, "kp": kp, "seconds": secs, "threads": threads}


def oracle_error(sig_gpu, st_gpu, R):
    """sigma of a form against the oracle reference R (oracle_reference): status agreement, and
    the max relative error on the parity domain (status 0, kappa_P <= 100) and elsewhere."""
    ref, st_ref = R["ref"], R["st"]
    ok = st_ref == 0
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = np.abs(sig_gpu - ref) / ref
    dom = ok & (R["kp"] <= 100)
    return {"rows": int(ref.size), "status_equal": bool(np.array_equal(st_gpu, st_ref)),
            "parity_domain_rows": int(dom.sum()),
            "max_rel_sigma_parity_domain": float(rel[dom].max()) if dom.any() else None,
            "rows_ge_1e-13_parity_domain": int((rel[dom] >= 1e-13).sum()),
            "max_rel_sigma_off_domain": float(rel[ok & ~dom].max()) if (ok & ~dom).any() else None,
            "oracle_seconds": R["seconds"], "oracle_threads": R["threads"]}


def body_variants(dev, stream, steps, peaks, sm_mhz, oracle_rows=1 << 20):
    """The 64M-option body batch (ln K/F ~ U[-1,1], sigma* ~ U[0.05,1]; configurations 3 and 4):
    plain FP64, the mixed form and the learned seed, fwd+bwd, same launch configuration.  Beside
    each timing: its roofline, the launch's counters, and sigma against the CPU oracle on a
    deterministic 1M-row subsample plus every row where the form and the GPU's FP64 path differ
    by 1e-13 or more on the parity domain."""
    import ctypes

    import torch

    import paper_2606_17065_gb300 as pv
    from paper_2606_17065_gb300 import _native
    b = workloads.body_batch(workloads.LARGE_N, seed=3)
    n = b.n
    F, K, T = (torch.from_numpy(a).to(dev) for a in (b.F, b.K, b.T))
    flag = torch.from_numpy(b.flag).to(dev)
    P, _ = pv.black_price(F, K, T, torch.from_numpy(b.sigma_star).to(dev), flag, vega=False)
    sig = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.uint8, device=dev)
    g = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(4)]
    lib = _native.lib()
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    opts = _native.PivotOpts()

    # the learned seed: trained first by the library's kernels on 16M operator-generated pairs
    from paper_2606_17065_gb300 import training
    trainer, hist, train_s = training.train_learned_guess(n_rows=workloads.STRESS_N, steps=12000, batch=32768,
                                                          lr=3e-3, seed=4, device=dev)

    def run(mode, counters=None):
        opts.mode, opts.householder = mode, 0
        opts.mlp = trainer.weights_ptr() if mode == 2 else None
        opts.fallback = 0.0
        opts.counters = None if counters is None else counters.data_ptr()
        rc = lib.pivot_iv_forward_backward(n, p(F), p(K), p(T), p(P), p(flag), None, TAU, pv.GATES[GATE], p(sig),
                                           p(st), *[p(x) for x in g], ctypes.byref(opts),
                                           ctypes.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise RuntimeError(_native.error_string(rc))

    forms = {"plain_fp64": (0, "body"), "mixed": (1, "body-mixed"), "learned": (2, "body-learned")}
    res = {name: time_variant(lambda m=mode: run(m), n, stream, steps) for name, (mode, _) in forms.items()}
    res["learned"]["training"] = {"pairs": workloads.STRESS_N, "adam_steps": 12000, "batch": 32768,
                                  "seconds": train_s, "final_mse_ln_s": hist[-1][1]}
    # counters of one launch of each form, then its roofline (the learned form's MLP runs on the
    # rows it seeds: all solved rows less those sent straight to the fallback)
    for name, (mode, case) in forms.items():
        c = pv.new_counters(dev)
        run(mode, c)
        cs = counters_summary(c.cpu(), mode)
        res[name]["counters"] = cs
        mlp_rows = int(sum(int(v) for v in c[6:12].cpu().tolist())) if mode == 2 else 0
        res[name]["roofline"] = variant_roofline(case, n, res[name]["ms_per_step"], peaks, sm_mhz, mlp_rows)
    res["learned"]["fallback_frac_of_solved"] = res["learned"]["counters"]["rejected_accelerated_frac_of_solved"]

    # sigma against the oracle: a deterministic subsample of 1M rows, and the rows the GPU's
    # FP64 path flags (the form differs from it by >= 1e-13 on the parity domain)
    run(0)
    s64, st64 = sig.clone(), st.clone()
    ok = st64 == 0
    _, V = pv.black_price(F, K, T, torch.where(ok, s64, torch.ones_like(s64)), flag)
    dom = ok & (P <= 100 * s64 * V)
    idx = workloads.sample_indices(n, oracle_rows, seed=13)
    tidx = torch.from_numpy(idx).to(dev)
    P_np = P.cpu().numpy()
    R = oracle_reference(b.F[idx], b.K[idx], b.T[idx], P_np[idx], b.flag[idx])
    for name, (mode, _) in forms.items():
        run(mode)
        rec = res[name]
        rec["oracle_error_1M_sample"] = oracle_error(sig[tidx].cpu().numpy(), st[tidx].cpu().numpy(), R)
        if mode:
            rel = torch.zeros_like(s64)
            rel[dom] = (sig[dom] - s64[dom]).abs() / s64[dom]
            rec["max_rel_sigma_vs_fp64_on_parity_domain"] = float(rel.max())
            flagged = torch.nonzero(rel >= 1e-13).flatten()[:100000]
            rec["fp64_recheck_flagged_rows"] = int(torch.count_nonzero(rel >= 1e-13))
            if flagged.numel():
                fidx = flagged.cpu().numpy()
                Rf = oracle_reference(b.F[fidx], b.K[fidx], b.T[fidx], P_np[fidx], b.flag[fidx])
                rec["oracle_error_flagged_rows"] = oracle_error(sig[flagged].cpu().numpy(),
                                                                st[flagged].cpu().numpy(), Rf)
    # what the network gains over LBR's rational seed: relative error of each seed against the
    # FP64 root on the first 1M rows
    m = 1 << 20
    s_root = s64[:m] * T[:m].sqrt()
    errs = {}
    for seed_mode, kw in (("rational", {"mode": "fp64"}), ("mlp", {"mode": "learned", "mlp": trainer})):
        s0 = pv.iv_guess(F[:m], K[:m], T[:m], P[:m], flag[:m], **kw)
        good = ok[:m] & torch.isfinite(s0) & (s_root > 0)
        e = ((s0[good] / s_root[good]) - 1).abs().float()
        errs[seed_mode] = {f"q{int(q * 1000) / 10:g}": float(torch.quantile(e[: 1 << 20], q))
                           for q in (0.5, 0.9, 0.99, 0.999)}
    res["learned"]["seed_rel_error_vs_root"] = errs
    del F, K, T, flag, P, sig, st, g, s64, st64, V, dom, trainer
    torch.cuda.empty_cache()
    out = {"workload": "body-64M: F=100, ln(K/F)~U[-1,1], T~U[1/365,3], sigma*~U[0.05,1], fwd+bwd", "rows": n}
    out.update(res)
    out["mixed_speedup"] = res["plain_fp64"]["ms_per_step"] / res["mixed"]["ms_per_step"]
    out["learned_speedup"] = res["plain_fp64"]["ms_per_step"] / res["learned"]["ms_per_step"]
    return out


def svi_variant(dev, n_surfaces=1024, steps=100):
    """Configuration 5: Adam through ImpliedVol on 1,024 synthetic SVI surfaces (ragged 50-400
    quotes over 8 maturities), one MLP pricer 2 -> 128 x 4 -> 1 (FP32) per surface, loss
    sum (sigma_hat - sigma*)^2, 100 steps at lr 1e-3, smooth gate tau = 1e-6."""
    from paper_2606_17065_gb300 import training
    batch = workloads.svi_batch(n_surfaces, seed=5)
    # untimed warm-up: the first steps load torch's CUDA kernels (seconds on a fresh machine)
    training.train_iv_loss(batch, steps=3, lr=1e-3, tau=1e-6, gate="smooth", device=dev)
    out = training.train_iv_loss(batch, steps=steps, lr=1e-3, tau=1e-6, gate="smooth", device=dev)
    L = out["loss"]
    return {"workload": f"svi-{n_surfaces}: ragged 50-400 quotes over 8 maturities, MLP 2->128x4->1 per surface, "
                        f"{steps} Adam steps lr 1e-3, loss sum (sigma_hat - sigma*)^2, smooth gate tau 1e-6",
            "surfaces": n_surfaces, "quotes": out["quotes"], "padded_rows": out["rows"], "steps": steps,
            "ms_per_step": 1e3 * out["seconds"] / steps,
            "loss": {"step0": L[0], "step50": L[min(50, steps - 1)], "step100": L[-1]},
            "loss_ratio_first_last": L[0] / L[-1] if L[-1] > 0 else None,
            "nan_grad_steps": out["nan_grad_steps"],
            "iv_gate_kept": {"first": out["iv_gate_kept"][0], "last": out["iv_gate_kept"][-1],
                             "min": min(out["iv_gate_kept"])}}


def bs_variants(dev, stream, steps, peaks, sm_mhz):
    """The Black-Scholes interface on xi = (S, K, tau, r, q): fused fwd+bwd on a 16M-row batch
    of the wide distribution (ln(K/S) ~ U[-6,6], s log-uniform on [1e-4, 3], r ~ U[-0.01, 0.08],
    q ~ U[0, 0.05]), and the streaming label loop: 64 batches of 65,536 quotes copied from
    pinned host memory, inverted (forward only) and copied back, on two alternating streams."""
    import ctypes

    import torch

    import paper_2606_17065_gb300 as pv
    from paper_2606_17065_gb300 import _native
    b = workloads.bs_batch(workloads.STRESS_N, seed=7, wide=True)
    n = b.n
    S, K, T, r, q, s0 = (torch.from_numpy(a).to(dev) for a in (b.S, b.K, b.T, b.r, b.q, b.sigma_star))
    flag = torch.from_numpy(b.flag).to(dev)
    V, _ = pv.bs_price(S, K, T, r, q, s0, flag, vega=False)
    sig = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.uint8, device=dev)
    g = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(6)]
    lib = _native.lib()
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    opts = _native.PivotOpts()

    def run(mode, backward=True, strm=stream, m=n, ins=None, out=None, counters=None):
        opts.mode, opts.householder = mode, 0
        opts.counters = None if counters is None else counters.data_ptr()
        a = ins or (S, K, T, r, q, V, flag)
        if backward:
            rc = lib.pivot_bs_iv_forward_backward(m, *[p(x) for x in a], None, TAU, pv.GATES[GATE], p(sig), p(st),
                                                  *[p(x) for x in g], ctypes.byref(opts),
                                                  ctypes.c_void_p(strm.cuda_stream))
        else:
            rc = lib.pivot_bs_iv_forward(m, *[p(x) for x in a], p(out if out is not None else sig), None,
                                         ctypes.byref(opts), ctypes.c_void_p(strm.cuda_stream))
        if rc != 0:
            raise RuntimeError(_native.error_string(rc))

    plain = time_variant(lambda: run(0), n, stream, steps)
    mixed = time_variant(lambda: run(1), n, stream, steps)
    fwd = time_variant(lambda: run(0, backward=False), n, stream, steps)
    for rec, mode, case in ((plain, 0, "bs-wide"), (mixed, 1, "bs-wide-mixed")):
        c = pv.new_counters(dev)
        run(mode, counters=c)
        rec["counters"] = counters_summary(c.cpu(), mode)
        rec["roofline"] = variant_roofline(case, n, rec["ms_per_step"], peaks, sm_mhz)

    # streaming label generation from host memory
    nb, m = 64, 65536
    host = [torch.from_numpy(np.ascontiguousarray(a[:nb * m])).pin_memory()
            for a in (b.S, b.K, b.T, b.r, b.q)]
    host.append(V[:nb * m].cpu().pin_memory())
    host.append(torch.from_numpy(b.flag[:nb * m]).pin_memory())
    labels = torch.empty(nb * m, dtype=torch.float64).pin_memory()
    streams = [torch.cuda.Stream(dev) for _ in range(2)]
    bufs = [[torch.empty(m, dtype=h.dtype, device=dev) for h in host] + [torch.empty(m, dtype=torch.float64,
                                                                                    device=dev)]
            for _ in range(2)]

    def pipeline():
        for j in range(nb):
            k = j % 2
            with torch.cuda.stream(streams[k]):
                for d, h in zip(bufs[k][:7], host):
                    d.copy_(h[j * m:(j + 1) * m], non_blocking=True)
                run(0, backward=False, strm=streams[k], m=m, ins=bufs[k][:7], out=bufs[k][7])
                labels[j * m:(j + 1) * m].copy_(bufs[k][7], non_blocking=True)
        for s_ in streams:
            s_.synchronize()

    for _ in range(2):
        pipeline()
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        pipeline()
    wall = (time.perf_counter() - t0) / reps
    ok = bool(torch.isfinite(labels[:1024]).any())
    label_rate = {"value": nb * m / wall, "unit": "labels/s", "ms_per_loop": wall * 1e3, "batches": nb,
                  "batch_rows": m, "h2d_bytes_per_loop": nb * m * 49, "d2h_bytes_per_loop": nb * m * 8,
                  "labels_finite": ok}
    del S, K, T, r, q, s0, flag, V, sig, st, g, bufs
    torch.cuda.empty_cache()
    return {"workload": "bs-wide-16M: S=100, ln(K/S)~U[-6,6], sigma*sqrt(T) log-uniform [1e-4,3], T~U[1/365,3], "
                        "r~U[-0.01,0.08], q~U[0,0.05], fwd+bwd in (V,S,K,tau,r,q)",
            "rows": n, "plain_fp64": plain, "mixed": mixed, "forward_only": fwd,
            "label_pipeline": label_rate}


def run_ours(args, rank, world):
    import torch

    import paper_2606_17065_gb300 as pv

    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    # inputs: this rank's own shard of independent rows (weak scaling)
    b = workloads.stress_batch(args.rows, seed=shard_seed(rank))
    n = b.n
    F = torch.from_numpy(b.F).to(dev)
    K = torch.from_numpy(b.K).to(dev)
    T = torch.from_numpy(b.T).to(dev)
    flag = torch.from_numpy(b.flag).to(dev)
    P, _ = pv.black_price(F, K, T, torch.from_numpy(b.sigma_star).to(dev), flag, vega=False)
    fixed = torch.from_numpy(b.P_fixed).to(dev)
    P = torch.where(torch.isnan(fixed), P, fixed).contiguous()
    del fixed
    outs = dict(sigma=torch.empty(n, dtype=torch.float64, device=dev),
                status=torch.empty(n, dtype=torch.uint8, device=dev),
                grads=[torch.empty(n, dtype=torch.float64, device=dev) for _ in range(4)])

    import ctypes
    from paper_2606_17065_gb300 import _native
    lib = _native.lib()
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    sptr = ctypes.c_void_p(stream.cuda_stream)
    opts = _native.PivotOpts()
    opts.mode, opts.householder = 0, 0

    def step(mode=0, counters=None):
        opts.mode = mode
        opts.counters = None if counters is None else counters.data_ptr()
        rc = lib.pivot_iv_forward_backward(n, p(F), p(K), p(T), p(P), p(flag), None, TAU, pv.GATES[GATE],
                                           p(outs["sigma"]), p(outs["status"]), *[p(g) for g in outs["grads"]],
                                           ctypes.byref(opts), sptr)
        if rc != 0:
            raise RuntimeError(f"pivot_iv_forward_backward failed: {_native.error_string(rc)}")

    def step_fwd():
        opts.mode = 0
        opts.counters = None
        rc = lib.pivot_iv_forward(n, p(F), p(K), p(T), p(P), p(flag), p(outs["sigma"]), p(outs["status"]),
                                  ctypes.byref(opts), sptr)
        if rc != 0:
            raise RuntimeError(f"pivot_iv_forward failed: {_native.error_string(rc)}")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K fused steps, CUDA events on the launching stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(local) as clocks:
        barrier(world)
        torch.cuda.synchronize()
        ev[0].record(stream)
        for i in range(args.steps):
            step()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
    per_launch = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms = max_over_ranks(total_ms, world)
    ms_per_step = total_ms / args.steps
    value = n * world / (ms_per_step * 1e-3)
    clk = clocks.summary()

    # ---- measured unit rates (FP64 / FP32 fma, MUFU) and the HBM rate of the path's 74-byte rows
    sm_mhz = clk["sm_mhz"] or 2070.0
    peaks = unit_peaks(dev, stream, sm_mhz)
    peaks["row_stream"] = stream_probe(F, K, T, P, flag, [outs["sigma"], outs["status"], *outs["grads"]], stream,
                                       max(args.steps // 2, 4))

    # ---- the mixed-precision form on the same batch (float seed, FP64 final step)
    mixed = time_variant(lambda: step(mode=1), n, stream, max(args.steps // 2, 2))
    mixed["roofline"] = variant_roofline("stress-mixed", n, mixed["ms_per_step"], peaks, sm_mhz)
    counts = {}
    for mode in (0, 1):
        c = pv.new_counters(dev)
        step(mode=mode, counters=c)
        counts[mode] = counters_summary(c.cpu(), mode)
    mixed["counters"] = counts[1]

    # ---- sigma of the plain and mixed forms against the CPU oracle on a deterministic 1M-row
    # subsample of this batch (outside every timed region)
    oracle_err = None
    if rank == 0 and world == 1 and args.rows == workloads.STRESS_N:
        idx = workloads.sample_indices(n, 1 << 20, seed=14)
        tidx = torch.from_numpy(idx).to(dev)
        P_np = P.cpu().numpy()
        R = oracle_reference(b.F[idx], b.K[idx], b.T[idx], P_np[idx], b.flag[idx])
        oracle_err = {}
        for name, mode in (("plain_fp64", 0), ("mixed", 1)):
            step(mode=mode)
            oracle_err[name] = oracle_error(outs["sigma"][tidx].cpu().numpy(), outs["status"][tidx].cpu().numpy(), R)
        mixed["oracle_error_1M_sample"] = oracle_err["mixed"]

    # ---- forward-only throughput (same inputs), for context
    for _ in range(2):
        step_fwd()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(max(args.steps // 2, 1)):
        step_fwd()
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / max(args.steps // 2, 1)

    # ---- end to end through the public API with pinned host buffers: inputs and the caller's
    # outputs in pinned host memory, allocated once as a serving loop would (a first pinning of
    # ~0.7 GB of outputs costs ~50 ms once and is not part of the steady state)
    hF, hK, hT, hP = (t.cpu().pin_memory() for t in (F, K, T, P))
    hflag = flag.cpu().pin_memory()
    hout = [torch.empty(n, dtype=d).pin_memory() for d in (torch.float64, torch.uint8) + (torch.float64,) * 4]
    for _ in range(3):
        pv.iv_forward_backward(hF, hK, hT, hP, hflag, tau=TAU, gate=GATE, out=hout)
    torch.cuda.synchronize()
    e2e_steps = max(min(args.steps, 10), 1)
    e2e_calls = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        res = pv.iv_forward_backward(hF, hK, hT, hP, hflag, tau=TAU, gate=GATE, out=hout)
        float(res[0][0])  # results are on the host
        e2e_calls.append(time.perf_counter() - t0)
    # the median call: a host shared with other jobs can stall one call's copies (one run saw a
    # mean 1.6x its median); the mean, min and max are reported beside it
    e2e_s = max_over_ranks(float(np.median(e2e_calls)), world)
    e2e_mean_s = max_over_ranks(float(np.mean(e2e_calls)), world)
    h2d = n * 33
    d2h = n * (8 + 1 + 4 * 8)

    # ---- roofline of the fused kernel
    mean_ms = statistics.mean(per_launch)
    fp64_peak = SMS * FP64_FLOP_PER_CLK_PER_SM * sm_mhz * 1e6
    if FLOPS_PER_ROW is not None:
        achieved = FLOPS_PER_ROW * n / (mean_ms * 1e-3)
        roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak,
                "traffic": None if TRAFFIC_PER_ROW is None else TRAFFIC_PER_ROW * n,
                "flops_per_row": FLOPS_PER_ROW,
                "peak_source": f"152 SMs x 4 FP64 FLOP/clk (1.25 TFLOP/s nominal at 2.07 GHz) at {sm_mhz:.0f} MHz"}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": fp64_peak / 1e12, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "flops_per_row": None, "peak_source": "FP64 FLOPs per row not yet counted by ncu"}
    if FLOPS_PER_ROW is not None:
        m64 = peaks["fp64_fma"]["flop_per_s"]
        roof["peak_measured"] = m64 / 1e12
        roof["frac_of_measured_peak"] = FLOPS_PER_ROW * n / (mean_ms * 1e-3) / m64
        roof["peak_measured_source"] = "pivot_probe_units FP64 fma chains on every SM, best of 3 launches"
    roof["counters"] = counts[0]
    hbm_peak = measured_peaks().get("hbm_gbs", HBM_PEAK_FALLBACK)
    roof["hbm"] = {"achieved": BYTES_PER_ROW * n / (mean_ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                   "frac": BYTES_PER_ROW * n / (mean_ms * 1e-3) / 1e9 / hbm_peak}

    full = args.rows == workloads.STRESS_N
    body = body_variants(dev, stream, max(args.steps // 4, 2), peaks, sm_mhz) if full else None
    bsv = bs_variants(dev, stream, max(args.steps // 4, 2), peaks, sm_mhz) if full else None
    svi = svi_variant(dev) if full else None

    # configuration 1: 4,096 rows, one launch (launch- and latency-bound, not a throughput line)
    small = workloads.body_batch(workloads.SMALL_N, seed=1)
    sF, sK, sT = (torch.from_numpy(a).to(dev) for a in (small.F, small.K, small.T))
    sflag = torch.from_numpy(small.flag).to(dev)
    sP, _ = pv.black_price(sF, sK, sT, torch.from_numpy(small.sigma_star).to(dev), sflag, vega=False)
    sout = [torch.empty(small.n, dtype=torch.float64, device=dev) for _ in range(5)]
    sst = torch.empty(small.n, dtype=torch.uint8, device=dev)

    def small_step():
        rc = lib.pivot_iv_forward_backward(small.n, p(sF), p(sK), p(sT), p(sP), p(sflag), None, TAU,
                                           pv.GATES[GATE], p(sout[0]), p(sst), *[p(g) for g in sout[1:]],
                                           ctypes.byref(opts), sptr)
        if rc != 0:
            raise RuntimeError(_native.error_string(rc))

    opts.mode = 0
    small_line = time_variant(small_step, small.n, stream, 50)
    small_line["note"] = "4,096 body rows per launch: launch- and latency-bound"

    cpu = None
    if rank == 0 and world == 1:
        r, threads, m, dt = oracle_rate(args.cpu_seconds)
        r1, _, m1, dt1 = oracle_rate(max(args.cpu_seconds / 4, 0.5), threads=1)
        cpu = {"value": r, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{m} seeded rows of the same stress workload, fwd+bwd, {dt:.1f} s wall",
               "cpu_model": cpu_model(),
               "single_thread": {"value": r1, "unit": UNIT, "sample": f"{m1} rows, {dt1:.1f} s wall"}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "rows_per_gpu": n, "parallelism": f"replicas x{world}",
                           "l2": "inputs 553 MB per step > 129 MB L2: no flush"},
                "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
                "e2e": {"value": n * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "calls": len(e2e_calls), "statistic": "median call",
                        "value_mean": n * world / e2e_mean_s,
                        "ms_per_call_min_max": [1e3 * min(e2e_calls), 1e3 * max(e2e_calls)]},
                "gpu_launches": args.steps,
                "roofline": roof,
                "forward_only": {"value": n * world / (fwd_ms * 1e-3), "unit": UNIT, "ms_per_step": fwd_ms},
                "oracle_error_1M_sample": None if oracle_err is None else oracle_err["plain_fp64"],
                "measured_units": peaks,
                "variants": {"mixed_same_workload": mixed,
                             "mixed_speedup_same_workload": ms_per_step / mixed["ms_per_step"],
                             "config1_4096": small_line,
                             "body_64M": body,
                             "black_scholes_16M": bsv,
                             "svi_iv_loss": svi},
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)


def run_case(args):
    """One form on --rows rows of its workload: --warmup untimed and --steps timed launches of its
    fused forward+backward, then one launch with counters.  Used for profiling captures of a
    single kernel on a small batch; prints one JSON line (not a headline measurement)."""
    import ctypes

    import torch

    import paper_2606_17065_gb300 as pv
    from paper_2606_17065_gb300 import _native
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    mode = 1 if args.case.endswith("mixed") else 2 if args.case.endswith("learned") else 0
    n = args.rows
    trainer = None
    if mode == 2:
        from paper_2606_17065_gb300 import training
        trainer, _, _ = training.train_learned_guess(n_rows=workloads.STRESS_N, steps=12000, batch=32768, lr=3e-3,
                                                     seed=4, device=dev)
    if args.case.startswith("bs"):
        b = workloads.bs_batch(n, seed=7, wide=True)
        ins = [t(a) for a in (b.S, b.K, b.T, b.r, b.q)]
        V, _ = pv.bs_price(*ins, t(b.sigma_star), t(b.flag), vega=False)
        ins += [V, t(b.flag)]
        ngrad = 6
        fn = "pivot_bs_iv_forward_backward"
    else:
        b = (workloads.stress_batch(n, seed=2) if args.case.startswith("stress")
             else workloads.body_batch(n, seed=3))
        ins = [t(a) for a in (b.F, b.K, b.T)]
        flag = t(b.flag)
        P, _ = pv.black_price(*ins, t(b.sigma_star), flag, vega=False)
        if getattr(b, "P_fixed", None) is not None:
            fixed = t(b.P_fixed)
            P = torch.where(torch.isnan(fixed), P, fixed).contiguous()
        ins += [P, flag]
        ngrad = 4
        fn = "pivot_iv_forward_backward"
    sig = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.uint8, device=dev)
    g = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(ngrad)]
    opts = _native.PivotOpts()
    opts.mode, opts.householder = mode, 0
    opts.mlp = trainer.weights_ptr() if trainer is not None else None
    p = lambda x: ctypes.c_void_p(x.data_ptr())  # noqa: E731
    lib = _native.lib()

    def run(counters=None):
        opts.counters = None if counters is None else counters.data_ptr()
        rc = getattr(lib, fn)(n, *[p(x) for x in ins], None, TAU, pv.GATES[GATE], p(sig), p(st), *[p(x) for x in g],
                              ctypes.byref(opts), ctypes.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise RuntimeError(_native.error_string(rc))

    for _ in range(args.warmup):
        run()
    r = time_variant(run, n, stream, max(args.steps, 1)) if args.steps > 0 else {}
    c = pv.new_counters(dev)
    run(c)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "rows": n, "timing": r, "counters": counters_summary(c.cpu(), mode),
                      "note": "profiling case, not a headline measurement"}), flush=True)


def main():
    args = parse()
    if args.case is not None:
        run_case(args)
        return
    if args.probe:
        import torch
        dev = torch.device("cuda", 0)
        with ClockSampler(0) as clocks:
            peaks = unit_peaks(dev, torch.cuda.current_stream(dev), 2070.0)
        print(json.dumps({"probe": peaks, "clocks": clocks.summary(),
                          "note": "per_sm_per_clk at 2,070 MHz; see clocks for the sampled SM clock"}), flush=True)
        return
    rank, world = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
