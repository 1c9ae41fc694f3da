"""The committed tables of the library's table-driven log and exp
(csrc/mathfn_tables.h) are what csrc/gen_mathfn_tables.py writes, and satisfy
the defining relations of Tang's method (checked here in 60-digit arithmetic)."""
import importlib.util
import os
import re

import pytest

mpmath = pytest.importorskip("mpmath")

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2312_07725_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_mathfn_tables", os.path.join(CSRC, "gen_mathfn_tables.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _array(text, name):
    body = re.search(name + r"\[\d+\] = \{(.*?)\};", text, re.S).group(1)
    return [float.fromhex(v.strip().rstrip("f")) for v in body.split(",") if v.strip()]


def test_header_is_the_generator_output(tmp_path):
    out = tmp_path / "mathfn_tables.h"
    _gen().main(str(out))
    assert out.read_text() == open(os.path.join(CSRC, "mathfn_tables.h")).read()


def test_tables_satisfy_their_definitions():
    mpmath.mp.dps = 60
    text = open(os.path.join(CSRC, "mathfn_tables.h")).read()
    c, lhi, llo = (_array(text, n) for n in ("NSFR_LOG_C", "NSFR_LOG_LHI", "NSFR_LOG_LLO"))
    for j in range(128):
        # c_j in [1/2, 1) within half an ulp (2^-54) of 1/(1 + (j + 1/2)/128); -ln c_j split
        # into two doubles
        exact = 1 / (1 + (mpmath.mpf(j) + mpmath.mpf("0.5")) / 128)
        assert 0.5 <= c[j] < 1.0 and abs(mpmath.mpf(c[j]) - exact) <= mpmath.mpf(2) ** -54
        err = mpmath.mpf(lhi[j]) + mpmath.mpf(llo[j]) + mpmath.log(mpmath.mpf(c[j]))
        assert abs(err) <= mpmath.mpf(2) ** -100
    shi, slo = _array(text, "NSFR_EXP_SHI"), _array(text, "NSFR_EXP_SLO")
    for j in range(32):
        err = mpmath.mpf(shi[j]) + mpmath.mpf(slo[j]) - mpmath.power(2, mpmath.mpf(j) / 32)
        assert abs(err) <= mpmath.mpf(2) ** -100
