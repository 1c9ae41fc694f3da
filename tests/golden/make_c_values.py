"""Write tests/golden/c_values.json: the ESFR parameter c_HU for p = 1..7.

c_HU is the value for which the GL mass matrix plus c K equals the
Lobatto-integrated mass matrix (the paper's description of c_HU, Sec.
"Maximum CFL").  Computed by the oracle only; the benchmark reads this file as
its positive-c stand-in (the paper does not print c_+).
"""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle.operators1d import c_hu  # noqa: E402

out = {"_source": "tests/golden/make_c_values.py (oracle.operators1d.c_hu)",
       "c_hu": {str(p): c_hu(p) for p in range(1, 8)}}
path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c_values.json")
with open(path, "w") as f:
    json.dump(out, f, indent=1)
print(path)
