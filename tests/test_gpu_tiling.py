"""Carried partial warps in the binned kernels.

The binned kernels consume each region bin of a tile in whole warps and carry the bin's last,
partial warp (rows, LBR nodes and global indices) into the block's next tile; the block's last
tile takes every row.  A row's arithmetic depends only on its own inputs and its bin, never on
the tile it is solved in, so one launch with many tiles per block must give, bit for bit, what
launches of at most one tile per block (batches of 65,536 rows, where nothing is carried) give on
the same rows.  The multi-tile launch is also held to the oracle on a sample of its rows.
Black-76 and Black-Scholes forms, FP64 and mixed.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2606_17065_gb300 as pv  # noqa: E402
from paper_2606_17065_gb300 import workloads  # noqa: E402

from gpu_helpers import DEV, assert_grad_parity, assert_sigma_parity, oracle_inputs, to_dev, to_np  # noqa: E402
from test_gpu_bs import check_sigma  # noqa: E402

pytestmark = pytest.mark.gpu

ROWS = 3_000_000 + 123  # ~6 tiles per resident block, and a ragged tail
CHUNK = 65_536          # at most one tile per resident block: nothing carried


def bits(t):
    return t.contiguous().view(torch.int64) if t.dtype == torch.float64 else t


def assert_same_bits(a, b, where):
    for k, (x, y) in enumerate(zip(a, b)):
        assert torch.equal(bits(x), bits(y)), f"{where}: output {k} differs on {int((bits(x) != bits(y)).sum())} rows"


def chunked(fn, arrays, n):
    parts = [fn(*[a[lo:lo + CHUNK] for a in arrays]) for lo in range(0, n, CHUNK)]
    return [torch.cat([p[k] for p in parts]) for k in range(len(parts[0]))]


@pytest.fixture(scope="module")
def stress_rows():
    b = workloads.stress_batch(ROWS, seed=31)
    F, K, T, flag = to_dev(b.F), to_dev(b.K), to_dev(b.T), to_dev(b.flag)
    P, _ = pv.black_price(F, K, T, to_dev(b.sigma_star), flag, vega=False)
    fixed = torch.from_numpy(b.P_fixed).to(DEV)
    P = torch.where(torch.isnan(fixed), P, fixed)
    # sampled rows priced by the oracle, so that the oracle check takes only the oracle's inputs
    idx = workloads.sample_indices(b.n, 3000, seed=32)
    sb = b.subset(idx)
    P_s = oracle_inputs(sb)
    P[torch.from_numpy(idx).to(DEV)] = torch.from_numpy(P_s).to(DEV)
    return b, (F, K, T, P.contiguous(), flag), idx, sb, P_s


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_black76_carry_is_invisible(stress_rows, mode):
    b, (F, K, T, P, flag), idx, sb, P_s = stress_rows

    def run(F, K, T, P, flag):
        return pv.iv_forward_backward(F, K, T, P, flag, tau=1e-6, gate="nan", mode=mode)

    whole = run(F, K, T, P, flag)
    parts = chunked(run, (F, K, T, P, flag), b.n)
    torch.cuda.synchronize()
    assert_same_bits(whole, parts, f"{mode} one launch vs 65,536-row launches")
    # the multi-tile launch against the oracle on the sampled rows
    sel = torch.from_numpy(idx).to(DEV)
    sig, st = to_np(whole[0][sel]), to_np(whole[1][sel])
    ref, st_ref = oracle.implied_vol(sb.F, sb.K, sb.T, P_s, sb.flag, nthreads=0)
    dom = assert_sigma_parity(sb.F, sb.K, sb.T, P_s, sb.flag, sig, st, ref, st_ref, where=f"{mode} sample")
    want = oracle.iv_grad(sb.F, sb.K, sb.T, sb.flag, ref, None, 1e-6, 1, nthreads=0)
    assert_grad_parity([to_np(g[sel]) for g in whole[2:]], want, dom, where=f"{mode} sample")


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_black_scholes_carry_is_invisible(mode):
    n = ROWS // 2
    b = workloads.bs_batch(n, seed=33, wide=True)
    d = [to_dev(a) for a in (b.S, b.K, b.T, b.r, b.q, b.sigma_star)]
    fl = to_dev(b.flag)
    V, _ = pv.bs_price(*d, fl, vega=False)
    idx = workloads.sample_indices(n, 3000, seed=34)
    sb = b.subset(idx)
    V_s, _ = oracle.bs_price(sb.S, sb.K, sb.T, sb.r, sb.q, sb.sigma_star, sb.flag, nthreads=0)
    V[torch.from_numpy(idx).to(DEV)] = torch.from_numpy(V_s).to(DEV)
    V = V.contiguous()

    def run(S, K, T, r, q, V, flag):
        return pv.bs_iv_forward_backward(S, K, T, r, q, V, flag, tau=1e-6, gate="nan", mode=mode)

    args = (*d[:5], V, fl)
    whole = run(*args)
    parts = chunked(run, args, n)
    torch.cuda.synchronize()
    assert_same_bits(whole, parts, f"Black-Scholes {mode} one launch vs 65,536-row launches")
    sel = torch.from_numpy(idx).to(DEV)
    ref, st_ref = oracle.bs_implied_vol(sb.S, sb.K, sb.T, sb.r, sb.q, V_s, sb.flag, nthreads=0)
    check_sigma(sb, V_s, to_np(whole[0][sel]), to_np(whole[1][sel]), ref, st_ref, f"Black-Scholes {mode} sample")


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_sparse_solves_fill_tiles_from_many_chunks(mode):
    """A batch where 1 row in 200 needs a solve and the rest sit at their intrinsic value
    (status 4): a tile then draws on its full 32 chunks (8,192 rows) for ~40 solves, so the
    chunk cap, tiles with fewer rows than a warp in a bin, the carry and the last-tile flush all
    run.  One launch matches 65,536-row launches bit for bit, every status matches the oracle,
    and sigma and the gradients of the solved rows match it on the parity domain."""
    n = 1_000_000 + 77
    b = workloads.body_batch(n, seed=35)
    rng = np.random.default_rng(36)
    solved = np.sort(rng.choice(n, n // 200, replace=False))
    itm = np.where(b.flag > 0, np.maximum(b.F - b.K, 0.0), np.maximum(b.K - b.F, 0.0))
    P = itm.copy()
    sb = b.subset(solved)
    P_s = oracle_inputs(sb)
    P[solved] = P_s
    args = [to_dev(a) for a in (b.F, b.K, b.T, P, b.flag)]

    def run(F, K, T, P, flag):
        return pv.iv_forward_backward(F, K, T, P, flag, tau=1e-6, gate="nan", mode=mode)

    whole = run(*args)
    parts = chunked(run, args, n)
    torch.cuda.synchronize()
    assert_same_bits(whole, parts, f"sparse {mode} one launch vs 65,536-row launches")
    st = to_np(whole[1])
    want_st = np.full(n, 4, dtype=st.dtype)
    _, st_ref_all = oracle.implied_vol(b.F, b.K, b.T, P, b.flag, nthreads=0)
    assert np.array_equal(st, st_ref_all), f"sparse {mode}: status mismatch on {np.sum(st != st_ref_all)} rows"
    assert np.count_nonzero(st == want_st) >= n - len(solved)
    sel = torch.from_numpy(solved).to(DEV)
    ref, st_ref = oracle.implied_vol(sb.F, sb.K, sb.T, P_s, sb.flag, nthreads=0)
    dom = assert_sigma_parity(sb.F, sb.K, sb.T, P_s, sb.flag, to_np(whole[0][sel]), to_np(whole[1][sel]), ref, st_ref,
                              where=f"sparse {mode}")
    want = oracle.iv_grad(sb.F, sb.K, sb.T, sb.flag, ref, None, 1e-6, 1, nthreads=0)
    assert_grad_parity([to_np(g[sel]) for g in whole[2:]], want, dom, where=f"sparse {mode}")


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_small_batch_chunks_match_full_chunks(mode):
    """Batches too small for a 256-row chunk per resident block run a separate kernel
    instantiation with 32- to 224-row chunks.  Rows are solved independently of their chunk and
    tile, so each small batch gives, bit for bit, what the same rows give inside a large batch
    run with full chunks; the sizes cover several chunk sizes and ragged ends."""
    n_big = 400_000
    b = workloads.stress_batch(n_big, seed=37)
    big = [to_dev(a) for a in (b.F, b.K, b.T, oracle_inputs(b), b.flag)]

    def run(F, K, T, P, flag):
        return pv.iv_forward_backward(F, K, T, P, flag, tau=1e-6, gate="nan", mode=mode)

    whole = run(*big)
    fwd_whole = pv.iv(*big, mode=mode)
    for n in (1, 33, 4_096, 9_001, 40_000, 77_823):
        sub = [t[:n].contiguous() for t in big]
        part = run(*sub)
        fwd = pv.iv(*sub, mode=mode)
        torch.cuda.synchronize()
        assert_same_bits(part, [w[:n] for w in whole], f"{mode} {n} rows vs the same rows in {n_big}")
        assert_same_bits(fwd, [w[:n] for w in fwd_whole], f"{mode} forward {n} rows vs the same rows in {n_big}")


def test_small_black_scholes_batch_matches_full_chunks():
    """The same for the Black-Scholes form (its own kernel instantiations)."""
    n_big = 400_000
    b = workloads.bs_batch(n_big, seed=38, wide=True)
    d = [to_dev(a) for a in (b.S, b.K, b.T, b.r, b.q, b.sigma_star)]
    fl = to_dev(b.flag)
    V, _ = pv.bs_price(*d, fl, vega=False)
    args = (*d[:5], V.contiguous(), fl)
    whole = pv.bs_iv_forward_backward(*args, tau=1e-6, gate="nan")
    for n in (57, 9_001, 77_823):
        part = pv.bs_iv_forward_backward(*[t[:n].contiguous() for t in args], tau=1e-6, gate="nan")
        torch.cuda.synchronize()
        assert_same_bits(part, [w[:n] for w in whole], f"Black-Scholes {n} rows vs the same rows in {n_big}")
