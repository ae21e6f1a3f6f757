"""Write spheres27_64_ceff.json: the effective stiffness of the 64^3 27-sphere workload (seeded,
contrast 100) computed by the CPU oracle alone (element-by-element assembly, PCG of Algorithm 1
with the FFT form of the preconditioner, tol 1e-11 per load case).  Takes several minutes.

    python tests/golden/make_spheres27_ceff.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import XFEM  # noqa: E402


def main():
    w = synth.make_workload("spheres27")
    t0 = time.time()
    o = XFEM(w["L"], w["n"], lame_minus=w["lame_minus"], lame_plus=w["lame_plus"])
    Cs, Ce, _ = o.effective_stiffness(solver="pcg", tol=1e-11, green="fft")
    out = {"workload": "spheres27 (64^3, 27 spheres, vf 20 %, contrast 100, seed 2)",
           "source": "oracle/xfem.py XFEM.effective_stiffness(solver='pcg', tol=1e-11, green='fft')",
           "n_enriched": int(o.nX), "n_cut_tets": int(len(o.cut_list)),
           "C_stress": Cs.tolist(), "C_energy": Ce.tolist(),
           "seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, "spheres27_64_ceff.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("n_enriched", "n_cut_tets", "seconds")}))


if __name__ == "__main__":
    main()
