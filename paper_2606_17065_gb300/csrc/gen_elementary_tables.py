"""Generate elementary_tables.inc: the tables of the table-driven FP64 logarithm and
exponential in pivot_device.cuh (P. T. P. Tang's method: ACM TOMS 15(2), 1989, for exp;
16(4), 1990, for log), written for this library.

log: v = 2^e m, m in [1, 2), c_j = 1 + j/1024 with j = round(1024 (m - 1)) in [0, 1024];
     ln v = e ln 2 + ln c_j + ln(1 + f), f = (m - c_j)/c_j, |f| <= 1/2048.
     Tables: 1/c_j, and ln c_j split as hi + lo with hi a multiple of 2^-43, so that
     e ln2_hi + ln c_j hi is exact for every exponent e.
exp: v = (128 n' + k) ln2/128 + r, |r| <= ln2/256; e^v = 2^n' 2^(k/128) e^r.
     Tables: 2^(k/128) as hi + lo (k = 0..127).
Constants (ln 2 split for both reductions) are printed alongside.

Run:  python gen_elementary_tables.py   (needs mpmath; writes the .inc next to it)
"""
import os

import mpmath as mp

LOG_N = 1024  # log table: c_j = 1 + j/LOG_N, j = 0..LOG_N


def split43(v):
    """v = hi + lo with hi a multiple of 2^-43 (|v| < 1): hi has at most ~43 significant bits."""
    hi = mp.floor(v * mp.mpf(2) ** 43) / mp.mpf(2) ** 43
    return float(hi), float(v - hi)


def main():
    mp.mp.dps = 50
    inv_c, lnc_hi, lnc_lo = [], [], []
    for j in range(LOG_N + 1):
        c = 1 + mp.mpf(j) / LOG_N
        inv_c.append(float(1 / c))
        hi, lo = split43(mp.log(c))
        lnc_hi.append(hi)
        lnc_lo.append(lo)
    ln2_hi, ln2_lo = split43(mp.log(2))
    # exp reduction by ln2/128: the high part with 35 significant bits (|n| < 2^18 keeps n * hi exact)
    l = mp.log(2) / 128
    l_hi = mp.floor(l * mp.mpf(2) ** 42) / mp.mpf(2) ** 42
    exp_hi, exp_lo = [], []
    for k in range(128):
        t = mp.mpf(2) ** (mp.mpf(k) / 128)
        exp_hi.append(float(t))
        exp_lo.append(float(t - mp.mpf(float(t))))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "elementary_tables.inc")
    with open(out, "w") as fh:
        fh.write("// Generated by gen_elementary_tables.py: tables of the table-driven FP64 log and exp.\n")
        fh.write(f"static constexpr double kLn2Hi = {ln2_hi!r};\n")
        fh.write(f"static constexpr double kLn2Lo = {ln2_lo!r};\n")
        fh.write(f"static constexpr double kLn2By128Hi = {float(l_hi)!r};\n")
        fh.write(f"static constexpr double kLn2By128Lo = {float(l - l_hi)!r};\n")
        fh.write(f"static constexpr double k128ByLn2 = {float(128 / mp.log(2))!r};\n")
        fh.write(f"static __device__ const double kLogInvC[{LOG_N + 1}] = {{\n")
        fh.write("".join(f"    {v!r},\n" for v in inv_c))
        fh.write(f"}};\nstatic __device__ const double kLogCHi[{LOG_N + 1}] = {{\n")
        fh.write("".join(f"    {v!r},\n" for v in lnc_hi))
        fh.write(f"}};\nstatic __device__ const double kLogCLo[{LOG_N + 1}] = {{\n")
        fh.write("".join(f"    {v!r},\n" for v in lnc_lo))
        fh.write("};\nstatic __device__ const double kExp2Hi[128] = {\n")
        fh.write("".join(f"    {v!r},\n" for v in exp_hi))
        fh.write("};\nstatic __device__ const double kExp2Lo[128] = {\n")
        fh.write("".join(f"    {v!r},\n" for v in exp_lo))
        fh.write("};\n")
    print(f"wrote {out}")


if __name__ == "__main__":
    main()
