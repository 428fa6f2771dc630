"""Generate erfcx_table.inc: piecewise polynomial coefficients of erfcx(a) = exp(a^2) erfc(a).

On [0, 16) the function is split into 128 intervals of width 1/8.  On each
interval it is replaced by its degree-9 Chebyshev interpolant (the polynomial
through erfcx at the 10 Chebyshev points of the interval), written in the
monomial basis of tau = 16 (a - a_i) - 1 in [-1, 1].  erfcx is entire, so
Chebyshev interpolation converges geometrically; at degree 9 the rounded
coefficients reproduce erfcx to about 1 ulp (checked below against 60-digit
mpmath).  Beyond 16 the device code uses the asymptotic series instead.

Run:  python gen_erfcx_table.py   (needs mpmath; writes the .inc next to it)
"""
import os

import mpmath as mp

WIDTH = mp.mpf(1) / 8
N_INT = 128
DEG = 9


def erfcx(a):
    return mp.erfc(a) * mp.exp(a * a)


def interval_coefficients(i):
    a0 = i * WIDTH
    nodes = [mp.cos(mp.pi * (j + mp.mpf(1) / 2) / (DEG + 1)) for j in range(DEG + 1)]
    vals = [erfcx(a0 + WIDTH * (t + 1) / 2) for t in nodes]
    A = mp.matrix([[t ** k for k in range(DEG + 1)] for t in nodes])
    c = mp.lu_solve(A, mp.matrix(vals))
    return [c[k] for k in range(DEG + 1)]


def main():
    mp.mp.dps = 60
    rows = []
    worst = 0.0
    for i in range(N_INT):
        c = interval_coefficients(i)
        cd = [float(x) for x in c]
        rows.append(cd)
        for j in range(33):
            t = -1 + mp.mpf(2) * j / 32
            v = 0.0
            for k in range(DEG, -1, -1):
                v = v * float(t) + cd[k]
            ref = erfcx(i * WIDTH + WIDTH * (t + 1) / 2)
            worst = max(worst, float(abs(v - ref) / ref))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "erfcx_table.inc")
    with open(out, "w") as fh:
        fh.write("// Generated by gen_erfcx_table.py: degree-9 Chebyshev interpolants of\n")
        fh.write("// erfcx(a) on [i/8, (i+1)/8), i = 0..127, monomial coefficients in\n")
        fh.write(f"// tau = 16 (a - i/8) - 1.  Max relative error in double: {worst:.3e}.\n")
        fh.write(f"static __device__ const double kErfcxCoef[{N_INT}][{DEG + 1}] = {{\n")
        for cd in rows:
            fh.write("    {" + ", ".join(repr(x) for x in cd) + "},\n")
        fh.write("};\n")
    print(f"wrote {out}; max relative error {worst:.3e}")


if __name__ == "__main__":
    main()
