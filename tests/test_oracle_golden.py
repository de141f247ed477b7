"""The oracle against its stored outputs (tests/golden/, written by
tests/golden/make_golden.py from the oracle alone)."""
import json
import os

import numpy as np
import pytest

from oracle import oracle
from paper_2604_20384_gb300.inputs import make_workload

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _c(lst):
    a = np.array(lst, dtype=float)
    return a[:, 0] + 1j * a[:, 1]


@pytest.mark.parametrize("name", ["n6_L3_Ns16_seed0", "n6_L3_Ns16_seed0_near0.1"])
def test_oracle_matches_golden(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        doc = json.load(f)
    w = make_workload(**doc["workload"])
    phi = oracle.reference_states(w.n, w.n_layers, w.Uref, w.psi1q)
    o = oracle.evaluate(w.n, w.n_layers, w.G, w.V, w.psi1q, phi, threads=1)
    assert abs(o["loss"] - doc["loss"]) < 1e-14
    for key in ("T", "Omega", "grad", "hvp", "grad_r", "hvp_r"):
        assert np.max(np.abs(o[key].ravel() - _c(doc[key]))) < 1e-14, key
