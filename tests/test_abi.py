"""CPU-side checks of the C ABI: the library loads and exports every declared symbol,
and argument validation needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "nsfr.h")).read()
    return sorted(set(re.findall(r"\b(nsfr_[a-z_]+)\s*\(", text)))


def test_header_and_binding_agree():
    from paper_2312_07725_gb300 import nsfr
    assert declared_symbols() == sorted(nsfr.EXPORTS)


def test_header_and_binding_agree_on_enums_and_kernel_ids():
    """The binding's tables are the header's: nsfr_profile_read writes
    NSFR_NKERNELS values into the buffer the binding sizes from KERNELS."""
    from paper_2312_07725_gb300 import nsfr
    text = open(os.path.join(ROOT, "include", "nsfr.h")).read()
    assert int(re.search(r"#define NSFR_NKERNELS (\d+)", text).group(1)) == len(nsfr.KERNELS)
    enums = dict((k, int(v)) for k, v in re.findall(r"\b(NSFR_[A-Z0-9_]+) = (-?\d+)", text))
    assert nsfr.FACE_FLUX == {"ec": enums["NSFR_FACE_EC"], "ec_roe": enums["NSFR_FACE_EC_ROE"],
                              "ec_es": enums["NSFR_FACE_EC_ES"]}
    assert nsfr.PRECISION == {"fp64": enums["NSFR_FP64"], "fp32_bulk": enums["NSFR_FP32_BULK"],
                              "fp32_bulk_ff": enums["NSFR_FP32_BULK_FF"]}
    assert nsfr.NODES == {"gl": enums["NSFR_NODES_GL"], "lgl": enums["NSFR_NODES_LGL"]}
    assert nsfr.VOL_FLUX == {"chandrashekar": enums["NSFR_FLUX_CHANDRASHEKAR"], "ranocha": enums["NSFR_FLUX_RANOCHA"]}
    assert nsfr.SOURCES == {"none": enums["NSFR_SOURCE_NONE"], "manufactured": enums["NSFR_SOURCE_MANUFACTURED"]}
    assert {v: k for k, v in nsfr.STATUS.items()} == {k: v for k, v in enums.items() if k.startswith("NSFR_OK")
                                                      or k.startswith("NSFR_ERR")}
    assert nsfr.MATH_FN == {k[len("NSFR_FN_"):].lower(): v for k, v in enums.items() if k.startswith("NSFR_FN_")}


def test_library_exports_every_declared_symbol():
    from paper_2312_07725_gb300 import nsfr
    if not os.path.exists(nsfr.LIB_PATH):
        from paper_2312_07725_gb300 import build
        build.build()
    lib = ctypes.CDLL(nsfr.LIB_PATH)
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_setup_rejects_bad_arguments_without_touching_a_gpu():
    from paper_2312_07725_gb300 import nsfr
    lib = nsfr.lib()
    h = ctypes.c_void_p()
    buf = (ctypes.c_double * 24)()
    # p out of range, zero elements, p_geo > p, gamma <= 1, negative c, unknown flux, unknown node set
    bad = [(1, 1, 1, 1, 9, 0.0, 0, 1.4, 0, 0), (0, 1, 1, 1, 1, 0.0, 0, 1.4, 0, 0),
           (1, 1, 1, 3, 2, 0.0, 0, 1.4, 0, 0), (1, 1, 1, 1, 1, 0.0, 0, 1.0, 0, 0),
           (1, 1, 1, 1, 1, -1.0, 0, 1.4, 0, 0), (1, 1, 1, 1, 1, 0.0, 7, 1.4, 0, 0),
           (1, 1, 1, 1, 1, 0.0, 0, 1.4, 0, 2)]
    for nx, ny, nz, pg, p, c, ff, g, prec, nodes in bad:
        st = lib.nsfr_setup(ctypes.cast(buf, ctypes.c_void_p), nx, ny, nz, pg, p, c, 0, ff, g, prec, nodes,
                            ctypes.byref(h))
        assert st == -1
        assert not h.value
    assert lib.nsfr_setup(None, 1, 1, 1, 1, 1, 0.0, 0, 0, 1.4, 0, 0, ctypes.byref(h)) == -1
    # unknown volume flux; Ranocha's pressure terms with an FP32-bulk precision
    for vf, prec in ((2, 0), (-1, 0), (1, 1), (1, 2)):
        st = lib.nsfr_setup(ctypes.cast(buf, ctypes.c_void_p), 1, 1, 1, 1, 1, 0.0, vf, 0, 1.4, prec, 0,
                            ctypes.byref(h))
        assert st == -1 and not h.value
    assert lib.nsfr_residual(None, None, None, None) == -1
    assert lib.nsfr_last_error(None) == b"NULL context"
    lib.nsfr_destroy(None)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2312_07725_gb300 import nsfr
    with pytest.raises(ImportError):
        nsfr.load_library(str(tmp_path / "libnsfr.so"))
