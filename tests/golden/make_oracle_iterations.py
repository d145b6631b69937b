"""Write oracle_iterations_32c8.json: the oracle's own shifted-CG solve of the 32^3 x 8 workload.

Runs only oracle/ (and the shared seeded input generator): the FP64 shifted CG for the 16-pole
Zolotarev approximation of x^{-1/2} on [4m^2, 16 + 4m^2], m = 0.02, to 1e-10, and records the
iteration count and the FP64 true residual of every shift.  tests/test_oracle_cpp.py checks the
C++ oracle's own full-size solve against this record (same iteration count, same residuals to
rounding).

    python tests/golden/make_oracle_iterations.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import rational, solvers, staggered  # noqa: E402
from paper_1710_09178_gb300 import inputs  # noqa: E402

dims, mass, npoles, tol = (32, 32, 32, 8), 0.02, 16, 1e-10
U = inputs.gauge_field(dims, seed=5)
b = inputs.gaussian_vector(dims, 6)
lo, hi = 4 * mass * mass, 16 + 4 * mass * mass
c0, res, poles, err = rational.zolotarev_inv_sqrt(npoles, lo, hi)
t0 = time.time()
xs, info = solvers.multishift_cg(lambda v: staggered.A_apply(U, v, mass, dims, poles.min()), b, poles, tol=tol)
dt = time.time() - t0
tr = solvers.true_residuals(lambda v, s: staggered.A_apply(U, v, mass, dims, s), b, xs, poles)
out = {"workload": "32^3x8", "mass": mass, "poles": npoles, "tol": tol, "gauge_seed": 5, "source_seed": 6,
       "iterations": int(info["iterations"]), "true_residuals": [float(t) for t in tr],
       "approximation_error": float(err), "oracle_seconds": round(dt, 1)}
with open(os.path.join(HERE, "oracle_iterations_32c8.json"), "w") as f:
    json.dump(out, f, indent=1)
print(json.dumps(out))
