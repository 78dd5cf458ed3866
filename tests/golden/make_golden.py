"""Write the stored expected values of the GPU parity tests.

Calls only the FP64 oracle (oracle/) and the seeded input generators; run from
the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import bloch_oracle as O  # noqa: E402
from paper_2106_12487_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def bands(name, n_k=None, method="lanczos", tol=1e-12):
    p = synth.workload(name, n_k)
    med = O.Medium.from_problem(p)
    t0 = time.time()
    res = O.solve_bands(med, p.k_list, p.n_bands, tol_lin=tol, tol_eig=tol, method=method)
    out = {
        "workload": name,
        "source": "oracle/bloch_oracle.py solve_bands (method=%s, tol_lin=tol_eig=%g)" % (method, tol),
        "grid": list(p.grid), "n_bands": p.n_bands,
        "k_list": p.k_list.tolist(),
        "omega": res.omega.tolist(),
        "oracle_cg_iters": int(res.cg_iters.sum()),
        "oracle_solves": int(res.solves.sum()),
        "eigenpairs": int(res.omega.size),
        "oracle_seconds": time.time() - t0,
    }
    with open(os.path.join(HERE, f"{name}_bands.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, "done in", out["oracle_seconds"], "s")


if __name__ == "__main__":
    bands("rve16_g8")
