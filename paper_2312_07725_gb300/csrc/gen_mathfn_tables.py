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

The float-float versions (mathfn_ff.cuh) use float tables of the same kind:
    cf_j = RN_float(1 / (1 + (j + 1/2) / 128)),  -ln(cf_j) = FL_hi[j] + FL_lo[j]  (j < 128),
    2^(j/64) = FS_hi[j] + FS_lo[j]  (j < 64),
each pair the nearest float and the nearest float of the remainder, and ln 2
and ln 2 / 64 cut into pieces short enough that k times a piece is exact.

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


def f32(v):
    """Nearest binary32 value of v (as a Python float)."""
    import struct
    return struct.unpack("f", struct.pack("f", float(v)))[0]


def split_f(v):
    hi = f32(v)
    lo = f32(v - mpmath.mpf(hi))
    return hi, lo


def chop(v, bits):
    """v truncated to `bits` significant bits."""
    m, e = mpmath.frexp(v)
    return float(mpmath.ldexp(mpmath.floor(mpmath.ldexp(m, bits)), e - bits))


def fmtf(x):
    return float.hex(x) + "f"


def main(path=None):
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

    # float tables of the float-float functions
    cf, flh, fll = [], [], []
    for j in range(128):
        cj = f32(1 / (1 + (mpmath.mpf(j) + mpmath.mpf(0.5)) / 128))
        h, l = split_f(-mpmath.log(mpmath.mpf(cj)))
        cf.append(cj)
        flh.append(h)
        fll.append(l)
    fsh, fsl = [], []
    for j in range(64):
        h, l = split_f(mpmath.power(2, mpmath.mpf(j) / 64))
        fsh.append(h)
        fsl.append(l)
    # ln 2 = A + B + C, A and B with 15 significant bits (k A, k B exact for |k| < 2^9)
    fa = chop(ln2, 15)
    fb = chop(ln2 - mpmath.mpf(fa), 15)
    fc = f32(ln2 - mpmath.mpf(fa) - mpmath.mpf(fb))
    # ln 2 / 64 = L1 + L2 + L3, L1 with 11 significant bits (n L1 exact for |n| < 2^13)
    l64 = ln2 / 64
    g1 = chop(l64, 11)
    g2 = f32(l64 - mpmath.mpf(g1))
    g3 = f32(l64 - mpmath.mpf(g1) - mpmath.mpf(g2))
    inv64 = f32(64 / ln2)

    def arrf(name, vals):
        lines.append(f"static __device__ const float {name}[{len(vals)}] = {{")
        for i in range(0, len(vals), 4):
            lines.append("    " + ", ".join(fmtf(v) for v in vals[i:i + 4]) + ",")
        lines.append("};")

    arr("NSFR_LOG_C", c)
    arr("NSFR_LOG_LHI", lhi)
    arr("NSFR_LOG_LLO", llo)
    arr("NSFR_EXP_SHI", shi)
    arr("NSFR_EXP_SLO", slo)
    arrf("NSFR_FLOG_C", cf)
    arrf("NSFR_FLOG_LHI", flh)
    arrf("NSFR_FLOG_LLO", fll)
    arrf("NSFR_FEXP_SHI", fsh)
    arrf("NSFR_FEXP_SLO", fsl)
    lines += ["",
              f"#define NSFR_FLN2_A {fmtf(fa)}  // ln 2 = A + B + C, A and B 15 bits",
              f"#define NSFR_FLN2_B {fmtf(fb)}",
              f"#define NSFR_FLN2_C {fmtf(fc)}",
              f"#define NSFR_FEXP_INV_L {fmtf(inv64)}  // 64 / ln 2",
              f"#define NSFR_FEXP_L1 {fmtf(g1)}  // ln 2 / 64 = L1 + L2 + L3, L1 11 bits",
              f"#define NSFR_FEXP_L2 {fmtf(g2)}",
              f"#define NSFR_FEXP_L3 {fmtf(g3)}"]
    lines += ["",
              f"#define NSFR_LN2_HI {fmt(ln2_hi)}",
              f"#define NSFR_LN2_LO {fmt(ln2_lo)}",
              f"#define NSFR_EXP_INV_L {fmt(inv)}  // 32 / ln 2",
              f"#define NSFR_EXP_L1 {fmt(l1)}      // ln 2 / 32, 36 bits",
              f"#define NSFR_EXP_L2 {fmt(l2)}      // ln 2 / 32 - L1", ""]
    with open(path or os.path.join(HERE, "mathfn_tables.h"), "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
