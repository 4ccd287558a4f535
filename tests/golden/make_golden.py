"""Write the stored expected values under tests/golden/.

Calls only the CPU oracle and the seeded input generators, never the CUDA
path.  Run from the repository root: ``python tests/golden/make_golden.py``.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2104_03293_gb300 import instances as I  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def config1_record():
    inst, g, b = I.config1()
    cmin, cmax, arg, cnt = oracle.ground(inst)
    E, P = oracle.expect(inst, g, b)
    val, dg, db = oracle.adjoint(inst, g, b, 0)
    return {
        "source": "CPU oracle (complex128, gate by gate): Eq. (QAOA_state) with H_C of Eq. (HC), "
                  "readout of Sec. III.B.1; 3-regular MaxCut stand-in for the paper's instances",
        "n": inst.n, "edges": inst.edges.tolist(), "J": inst.J.tolist(), "h": inst.h.tolist(),
        "gamma": g.tolist(), "beta": b.tolist(),
        "cmin": cmin, "cmax": cmax, "argmin": arg, "ground_count": cnt,
        "E": E, "P_ground": P, "dE_dgamma": dg.tolist(), "dE_dbeta": db.tolist(),
    }


if __name__ == "__main__":
    rec = config1_record()
    with open(os.path.join(HERE, "config1_maxcut3r_n12_p2.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print("wrote", rec["E"], rec["P_ground"])
