"""Write mathfn_tables.h: the tables of the library's FP64 log and exp.

The functions follow P. T. P. Tang's table-driven method ("Table-driven
implementation of the exponential function in IEEE floating-point
arithmetic", ACM TOMS 15, 1989; "... of the logarithm function", ACM TOMS 16,
1990).  The tables hold, for j = 0..127,
    c_j = RN(1 / (1 + (j + 1/2) / 128)),   -ln(c_j) = L_hi[j] + L_lo[j],
and, for j = 0..31,
    2^(j/32) = S_hi[j] + S_lo[j],
each value computed with 60 significant digits (mpmath) and split into the
nearest double and the nearest double of the remainder.

Usage: python gen_mathfn_tables.py  (rewrites mathfn_tables.h beside it)
"""
import os

import mpmath

mpmath.mp.dps = 60
HERE = os.path.dirname(os.path.abspath(__file__))


def split(v):
    hi = float(v)
    lo = float(v - mpmath.mpf(hi))
    return hi, lo


def fmt(x):
    return float.hex(x)


def main():
    c, lhi, llo = [], [], []
    for j in range(128):
        cj = float(1 / (1 + (mpmath.mpf(j) + mpmath.mpf(0.5)) / 128))
        h, l = split(-mpmath.log(mpmath.mpf(cj)))
        c.append(cj)
        lhi.append(h)
        llo.append(l)
    shi, slo = [], []
    for j in range(32):
        h, l = split(mpmath.power(2, mpmath.mpf(j) / 32))
        shi.append(h)
        slo.append(l)
    ln2 = mpmath.log(2)
    # ln 2 to 42 significant bits (k ln2_hi is exact for |k| < 2^11)
    m, e = mpmath.frexp(ln2)
    ln2_hi = float(mpmath.ldexp(mpmath.floor(mpmath.ldexp(m, 42)), e - 42))
    ln2_lo = float(ln2 - mpmath.mpf(ln2_hi))
    # ln2/32 with 36 significant bits (n L1 is exact for |n| < 2^17)
    l32 = ln2 / 32
    m, e = mpmath.frexp(l32)
    l1 = float(mpmath.ldexp(mpmath.floor(mpmath.ldexp(m, 36)), e - 36))
    l2 = float(l32 - mpmath.mpf(l1))
    inv = float(32 / ln2)
    lines = ["// Generated by gen_mathfn_tables.py -- do not edit.",
             "// Tables of Tang's table-driven FP64 log and exp (see mathfn.cuh).",
             "#pragma once", ""]

    def arr(name, vals):
        lines.append(f"static __device__ const double {name}[{len(vals)}] = {{")
        for i in range(0, len(vals), 4):
            lines.append("    " + ", ".join(fmt(v) for v in vals[i:i + 4]) + ",")
        lines.append("};")

    arr("NSFR_LOG_C", c)
    arr("NSFR_LOG_LHI", lhi)
    arr("NSFR_LOG_LLO", llo)
    arr("NSFR_EXP_SHI", shi)
    arr("NSFR_EXP_SLO", slo)
    lines += ["",
              f"#define NSFR_LN2_HI {fmt(ln2_hi)}",
              f"#define NSFR_LN2_LO {fmt(ln2_lo)}",
              f"#define NSFR_EXP_INV_L {fmt(inv)}  // 32 / ln 2",
              f"#define NSFR_EXP_L1 {fmt(l1)}      // ln 2 / 32, 36 bits",
              f"#define NSFR_EXP_L2 {fmt(l2)}      // ln 2 / 32 - L1", ""]
    with open(os.path.join(HERE, "mathfn_tables.h"), "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
