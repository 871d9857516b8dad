"""Write c2_oracle_reference.json: what the CPU oracle (and only the oracle)
computes on the 64^3 high-contrast diffusion workload, seed 0: the top
eigenvalues of eq. gevpsvd per subdomain, n_C, and the PCG iteration count
to 1e-8 with the two-level preconditioner.

Run from the repository root:  python tests/golden/make_c2_reference.py
(about twenty minutes on eight cores)."""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from asm_inputs import config  # noqa: E402


def main():
    p = config("c2", seed=0)
    A = p.csr()
    t0 = time.time()
    st = O.setup(A, p.part, p.N, 1, p.nev)
    t1 = time.time()
    res = O.solve(st, p.b)
    t2 = time.time()
    vals = [[float(v) for v in loc.values] for loc in st.locals]
    out = {
        "workload": "3D 7-point diffusion 64^3, contrast 1e6 channels/inclusions at 10%, 512 boxes of 8^3, "
                    "overlap 1, nev 16, seed 0 (asm_inputs.config('c2'))",
        "source": "oracle/asm_oracle.py, FP64 dense local eigensolves",
        "n_C": int(st.n_C),
        "pcg_iterations_two_level": int(res.iterations),
        "pcg_final_relres": float(res.final_relres),
        "oracle_setup_s_8core": t1 - t0,
        "oracle_solve_s_8core": t2 - t1,
        "eigenvalues": vals,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_oracle_reference.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(json.dumps({k: v for k, v in out.items() if k != "eigenvalues"}, indent=1))


if __name__ == "__main__":
    main()
