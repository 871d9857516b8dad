"""Write c3_oracle_reference.json and c4_oracle_reference.json: what the CPU
oracle (and only the oracle) computes on the full-size elasticity workload
(Q1 hexahedra on 32^3 elements, 256 subdomains, overlap 1, nev 24; PCG) and
the convection-diffusion workload (upwind FD on 512^2, 1024 subdomains,
overlap 2, nev 16, general method; FGMRES(30)), seed 0: the kept local
values of every subdomain (eigenvalues of eq. gevpsvd, or singular values of
D_i Pi_i), n_C and the Krylov iteration count to 1e-8.

Run from the repository root:  python tests/golden/make_config_reference.py [c3|c4]
(several minutes each)."""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from asm_inputs import config  # noqa: E402

WORKLOADS = {
    "c3": "3D linear elasticity, Q1 hexahedra on 32^3 elements (3 dofs/node, face x = 0 clamped), "
          "lognormal Young's modulus, 256 coordinate boxes, overlap 1, nev 24, seed 0 (asm_inputs.config('c3'))",
    "c4": "2D upwind convection-diffusion 512^2, rotating field, Peclet 1e3, 1024 boxes of 16^2, overlap 2, "
          "nev 16, general method, seed 0 (asm_inputs.config('c4'))",
}


def main(name: str):
    p = config(name, seed=0)
    A = p.csr()
    t0 = time.time()
    st = O.setup(A, p.part, p.N, p.delta, p.nev, spd=p.spd)
    t1 = time.time()
    res = O.solve(st, p.b)
    t2 = time.time()
    out = {
        "workload": WORKLOADS[name],
        "source": "oracle/asm_oracle.py, FP64 dense local eigensolves / SVDs",
        "method": "PCG" if p.spd else "FGMRES(30)",
        "n_C": int(st.Z.shape[1]),
        "iterations": int(res.iterations),
        "final_relres": float(res.final_relres),
        "oracle_setup_s": t1 - t0,
        "oracle_solve_s": t2 - t1,
        "values": [[float(v) for v in loc.values] for loc in st.locals],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_oracle_reference.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(json.dumps({k: v for k, v in out.items() if k != "values"}, indent=1))


if __name__ == "__main__":
    for n in (sys.argv[1:] or ["c3", "c4"]):
        main(n)
