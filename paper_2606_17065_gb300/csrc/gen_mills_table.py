"""Generate mills_table.inc: piecewise polynomial coefficients of the Mills ratio
M(w) = Y(-w) = Phi(-w) / phi(w) = sqrt(pi/2) erfcx(w / sqrt 2), w >= 0.

Y(z) = Phi(z)/phi(z) is the ratio through which the solver writes the normalised
Black function and its adjoint; every evaluation on the hot path is at z <= 0, i.e.
M(w) with w = -z >= 0, so the table is indexed by w itself and returns M(w) with no
scaling of argument or result.

The range [0, 128) is split into 177 intervals whose index comes from the bit
pattern of w alone: interval 0 is [0, 1/16); from 1/16 on, each binade
[2^e, 2^(e+1)), e = -4..6, is split into 16 equal parts, so that interval
1 + 16 (e + 4) + m (m = the top four mantissa bits of w) is
[2^e (1 + m/16), 2^e (1 + (m+1)/16)).  The widths grow with w, as M flattens
(it behaves like 1/w far out), and the index needs no floating-point instruction.

On each interval M is replaced by its degree-9 Chebyshev interpolant (the
polynomial through M at the 10 Chebyshev points of the interval), written in the
monomial basis of tau = w * scale + offset in [-1, 1]; scale = 2 / width is a
power of two and offset = -(2 w_0 / width + 1) an integer, so tau is formed by
one fma.  M is analytic on Re w > -infinity and close to 1/w for large w, so
Chebyshev interpolation converges geometrically on intervals of a fixed relative
width; at degree 9 the rounded coefficients reproduce M to about 1 ulp (checked
below against 60-digit mpmath).  From 128 on the device code uses the asymptotic
series M(w) ~ (1/w) sum_n (-1)^n (2n-1)!! / w^(2n).

Each row holds c_0..c_9, scale, offset (12 doubles, 96 bytes).

Run:  python gen_mills_table.py   (needs mpmath; writes the .inc next to it)
"""
import os

import mpmath as mp

DEG = 9
SUB = 16              # parts per binade
E_MIN, E_MAX = -4, 6  # binades [2^e, 2^(e+1)) covered by the split


def intervals():
    out = [(mp.mpf(0), mp.mpf(1) / 16)]
    for e in range(E_MIN, E_MAX + 1):
        for m in range(SUB):
            w = mp.mpf(2) ** e / SUB
            a0 = mp.mpf(2) ** e + m * w
            out.append((a0, a0 + w))
    return out


def mills(w):
    """Phi(-w) / phi(w) from the normal tail and density (no cancellation for w >= 0)."""
    return mp.ncdf(-w) / mp.npdf(w)


def interval_coefficients(a0, w):
    nodes = [mp.cos(mp.pi * (j + mp.mpf(1) / 2) / (DEG + 1)) for j in range(DEG + 1)]
    vals = [mills(a0 + w * (t + 1) / 2) for t in nodes]
    A = mp.matrix([[t ** k for k in range(DEG + 1)] for t in nodes])
    c = mp.lu_solve(A, mp.matrix(vals))
    return [c[k] for k in range(DEG + 1)]


def main():
    mp.mp.dps = 60
    rows = []
    worst = 0.0
    for a0, a1 in intervals():
        w = a1 - a0
        cd = [float(x) for x in interval_coefficients(a0, w)]
        scale, offset = float(2 / w), float(-(2 * a0 / w + 1))
        assert scale == 2 / w and offset == -(2 * a0 / w + 1)  # both exact in double
        rows.append(cd + [scale, offset])
        for j in range(33):
            t = -1 + mp.mpf(2) * j / 32
            v = 0.0
            for k in range(DEG, -1, -1):
                v = v * float(t) + cd[k]
            ref = mills(a0 + w * (t + 1) / 2)
            worst = max(worst, float(abs(v - ref) / ref))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mills_table.inc")
    with open(out, "w") as fh:
        fh.write("// Generated by gen_mills_table.py: degree-9 Chebyshev interpolants of the Mills ratio\n")
        fh.write("// M(w) = Phi(-w)/phi(w) on [0, 1/16) and on 16 equal parts of each binade [2^e, 2^(e+1)),\n")
        fh.write("// e = -4..6.  Row: monomial coefficients c_0..c_9 in tau = w * scale + offset, then scale, offset.\n")
        fh.write(f"// Max relative error in double: {worst:.3e}.\n")
        fh.write(f"static __device__ const double kMillsCoef[{len(rows)}][{DEG + 3}] = {{\n")
        for cd in rows:
            fh.write("    {" + ", ".join(repr(x) for x in cd) + "},\n")
        fh.write("};\n")
    print(f"wrote {out}; {len(rows)} intervals; max relative error {worst:.3e}")


if __name__ == "__main__":
    main()
