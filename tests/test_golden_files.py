"""The stored oracle references of the full-size workloads (tests/golden/*.json,
written by tests/golden/make_config_reference.py and make_c2_reference.py)
are what the oracle computes: a fresh oracle run on sampled subdomains gives
the stored local values, and the stored counts add up to the stored n_C."""
import json
import os

import numpy as np
import pytest

import oracle as O
from asm_inputs import config

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, f"{name}_oracle_reference.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("name,samples", [("c3", [0, 101, 255]), ("c4", [0, 517, 1023])])
def test_stored_values_are_the_oracles(name, samples):
    ref = _load(name)
    p = config(name, seed=0)
    A = p.csr()
    assert len(ref["values"]) == p.N
    assert sum(len(v) for v in ref["values"]) == ref["n_C"]
    assert ref["final_relres"] <= 1e-8 and ref["iterations"] > 0
    ovs = O.overlap(A, p.part, p.N, p.delta)
    for i in samples:
        Aii = O.local_matrix(A, ovs[i])
        if p.spd:
            vals = O.gevp_svd(Aii, ovs[i])[0]
        else:
            vals = O.svd_dpi(Aii, ovs[i])[0]
        k = len(ref["values"][i])
        assert k == O.select_count(np.asarray(vals), p.nev)
        np.testing.assert_allclose(ref["values"][i], vals[:k], rtol=1e-12, atol=0)
