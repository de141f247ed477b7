"""Writes the stored expected values under tests/golden/ from the FP64 oracle.

It calls only oracle/ (and the seeded input generator). The paper prints no
worked numeric example, so these fixtures are oracle outputs on seeded
synthetic circuits: the smallest benchmark shape (n = 6, L = 3, N_s = 16) and
its near-solution variant. They anchor the oracle against regressions; its
correctness is pinned by tests/test_oracle_pins.py.

Usage: python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle  # noqa: E402
from paper_2604_20384_gb300.inputs import make_workload  # noqa: E402

CASES = [
    ("n6_L3_Ns16_seed0", dict(n=6, n_layers=3, n_samples=16, seed=0)),
    ("n6_L3_Ns16_seed0_near0.1", dict(n=6, n_layers=3, n_samples=16, seed=0, near_solution=0.1)),
]


def cplx_list(a):
    return [[float(z.real), float(z.imag)] for z in a.ravel()]


def main():
    for name, kw in CASES:
        w = make_workload(**kw)
        phi = oracle.reference_states(w.n, w.n_layers, w.Uref, w.psi1q)
        o = oracle.evaluate(w.n, w.n_layers, w.G, w.V, w.psi1q, phi, threads=1)
        doc = dict(workload=kw, source="oracle/oracle.c via tests/golden/make_golden.py",
                   loss=o["loss"], T=cplx_list(o["T"]), Omega=cplx_list(o["Omega"]),
                   grad=cplx_list(o["grad"]), hvp=cplx_list(o["hvp"]),
                   grad_r=cplx_list(o["grad_r"]), hvp_r=cplx_list(o["hvp_r"]))
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(doc, f, indent=0)
        print("wrote", name)


if __name__ == "__main__":
    main()
