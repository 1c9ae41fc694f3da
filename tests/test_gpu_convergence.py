"""Order of accuracy of the full GPU scheme (FP64): the exact density wave on the warped
unit cube, Roe-dissipated face flux, RK4 to t = 0.1 -- the L2 error of rho converges at
p + 1 (the paper's Fig. OOA claim), for c = 0 and c = c_HU.  (c_HU enters the asymptotic
range one refinement later than c = 0, hence the levels.)"""
import json
import os

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
C_HU = {int(k): v for k, v in json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                                           "c_values.json")))["c_hu"].items()}


@pytest.mark.parametrize("p,levels", [(2, (8, 16, 32)), (3, (8, 16)), (4, (8, 16))])
@pytest.mark.parametrize("c_kind", ["dg", "hu"])
def test_order_p_plus_one(p, levels, c_kind):
    from paper_2312_07725_gb300.experiments import convergence
    r = convergence(p, levels, c=0.0 if c_kind == "dg" else C_HU[p])
    print(json.dumps(r))
    assert r["orders"][-1] > p + 1 - 0.35, r
