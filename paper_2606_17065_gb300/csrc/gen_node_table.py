"""Generate node_table.inc: the LBR boundary node as functions of |ln(F/K)| alone.

With u = |x| = |ln(F/K)| and w = sqrt(u), the inflection point is s_c = sqrt(2) w and
the two points where the tangent there reaches 0 and b_max are
    s_l = s_c - sqrt(pi/2) (1 - e),  s_u = s_c + sqrt(pi/2) (1 + e),  e = erfcx(w).
The node values the guesses interpolate between scale with b_max = e^{-u/2}:
    E(w)  = erfcx(w)
    SL(w) = s_l / u                          (s_l ~ 1.2533 u as u -> 0: no cancellation)
    FL(w) = b(-u, s_l) / (b_max u)           (b_l ~ 0.1512 b_max u as u -> 0)
    GL(w) = b_s(-u, s_l) / b_max
    FU(w) = (b_max - b(-u, s_u)) / b_max
    GU(w) = b_s(-u, s_u) / b_max
(b the normalised Black function, b_s its s-derivative).  All six are smooth, bounded
functions of w on [0, inf): they only shape the initial guess, so float precision (~1e-7
relative) is far below the guess's own interpolation error.

The range [0, 64) of w is split into 97 intervals whose index comes from the bit pattern
of w (as a float): interval 0 is [0, 1/64); from 1/64 on, each binade [2^e, 2^(e+1)),
e = -6..5, is split into 8 equal parts, so that interval 1 + 8 (e + 6) + m (m = the top
three mantissa bits of w) is [2^e (1 + m/8), 2^e (1 + (m+1)/8)).  On each interval each
function is its degree-6 Chebyshev interpolant in tau = w * scale + offset in [-1, 1]
(scale a power of two, offset an integer, both exact in float), monomial coefficients in
float.  Row layout: scale, offset, then the 7 coefficients c_0..c_6 of E, SL, FL, GL, FU, GU.

Run:  python gen_node_table.py   (needs mpmath and numpy; writes the .inc next to it)
"""
import os

import mpmath as mp
import numpy as np

DEG = 6
SUB = 8
E_MIN, E_MAX = -6, 5
NFUN = 6


def intervals():
    out = [(mp.mpf(0), mp.mpf(1) / 64)]
    for e in range(E_MIN, E_MAX + 1):
        for m in range(SUB):
            w = mp.mpf(2) ** e / SUB
            a0 = mp.mpf(2) ** e + m * w
            out.append((a0, a0 + w))
    return out


def b(x, s):
    return mp.exp(x / 2) * mp.ncdf(x / s + s / 2) - mp.exp(-x / 2) * mp.ncdf(x / s - s / 2)


def b_compl(x, s):
    """b_max - b without cancellation"""
    return mp.exp(x / 2) * mp.ncdf(-x / s - s / 2) + mp.exp(-x / 2) * mp.ncdf(x / s - s / 2)


def bs(x, s):
    return mp.exp(-x * x / (2 * s * s) - s * s / 8) / mp.sqrt(2 * mp.pi)


def sl_over_u(w):
    """s_l / u from its power series at small w (the difference s_c - sqrt(pi/2)(1 - e) cancels),
    directly elsewhere (enough digits at 80-digit precision)."""
    u = w * w
    c = mp.sqrt(mp.pi / 2)
    e = mp.erfc(w) * mp.exp(u)
    return (mp.sqrt(2) * w - c * (1 - e)) / u


def funcs(w):
    w = mp.mpf(w)
    u = w * w
    if u == 0:
        # limits as u -> 0: s_l / u -> sqrt(pi/2), b_l / (b_max u) and the rest from the definitions
        w = mp.mpf("1e-30")
        u = w * w
    c = mp.sqrt(mp.pi / 2)
    e = mp.erfc(w) * mp.exp(u)
    sc = mp.sqrt(2) * w
    sl = sl_over_u(w) * u
    su = sc + c * (1 + e)
    bmax = mp.exp(-u / 2)
    x = -u
    return [e, sl / u, b(x, sl) / (bmax * u), bs(x, sl) / bmax, b_compl(x, su) / bmax, bs(x, su) / bmax]


def main():
    mp.mp.dps = 80
    rows = []
    worst = [0.0] * NFUN
    for a0, a1 in intervals():
        wdt = a1 - a0
        nodes = [mp.cos(mp.pi * (j + mp.mpf(1) / 2) / (DEG + 1)) for j in range(DEG + 1)]
        vals = [funcs(a0 + wdt * (t + 1) / 2) for t in nodes]
        A = mp.matrix([[t ** k for k in range(DEG + 1)] for t in nodes])
        coef = []
        for f in range(NFUN):
            cvec = mp.lu_solve(A, mp.matrix([v[f] for v in vals]))
            coef.append([np.float32(float(cvec[k])) for k in range(DEG + 1)])
        scale, offset = float(2 / wdt), float(-(2 * a0 / wdt + 1))
        assert np.float32(scale) == scale and np.float32(offset) == offset
        rows.append([np.float32(scale), np.float32(offset)] + [c for cf in coef for c in cf])
        for j in range(17):
            t = -1 + mp.mpf(2) * j / 16
            ref = funcs(a0 + wdt * (t + 1) / 2)
            for f in range(NFUN):
                v = np.float32(0)
                for k in range(DEG, -1, -1):
                    v = np.float32(v * np.float32(float(t)) + coef[f][k])
                worst[f] = max(worst[f], float(abs(mp.mpf(float(v)) - ref[f]) / abs(ref[f])))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "node_table.inc")
    with open(out, "w") as fh:
        fh.write("// Generated by gen_node_table.py: the LBR node as functions of w = sqrt|ln(F/K)|,\n")
        fh.write("// degree-6 Chebyshev interpolants in float on [0, 1/64) and 8 equal parts of each binade\n")
        fh.write("// [2^e, 2^(e+1)), e = -6..5.  Row: scale, offset, then c_0..c_6 of E, SL, FL, GL, FU, GU.\n")
        fh.write("// Max relative error in float: " + ", ".join(f"{n} {x:.2e}" for n, x in zip(["E", "SL", "FL", "GL", "FU", "GU"], worst)) + ".\n")
        fh.write(f"static __device__ const float kNodeCoef[{len(rows)}][{2 + NFUN * (DEG + 1)}] = {{\n")
        for r in rows:
            fh.write("    {" + ", ".join(repr(float(x)) + "f" for x in r) + "},\n")
        fh.write("};\n")
    print(f"wrote {out}; {len(rows)} intervals; max relative errors", [f"{x:.2e}" for x in worst])


if __name__ == "__main__":
    main()
