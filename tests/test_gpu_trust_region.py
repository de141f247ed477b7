"""Riemannian trust-region steps (Sec. 4; Absil et al. 2008, Algorithms 10
and 11) driven by the library's Riemannian gradients and HVPs on the GPU,
against the same driver fed by the FP64 oracle."""
import numpy as np
import pytest

from common import rel
from oracle import oracle
from paper_2604_20384_gb300 import native
from paper_2604_20384_gb300 import trust_region as tr
from paper_2604_20384_gb300.inputs import make_workload

pytestmark = pytest.mark.gpu


class OracleProblem:
    def __init__(self, w):
        self.w = w
        self.phi = oracle.reference_states(w.n, w.n_layers, w.Uref, w.psi1q)

    def loss_grad(self, G):
        o = oracle.evaluate(self.w.n, self.w.n_layers, G, None, self.w.psi1q, self.phi)
        return o["loss"], o["grad_r"]

    def hvp(self, G, V):
        o = oracle.evaluate(self.w.n, self.w.n_layers, G, V, self.w.psi1q, self.phi)
        return o["loss"], o["grad_r"], o["hvp_r"]


def test_trust_region_on_gpu_matches_oracle_and_converges():
    w = make_workload(10, 6, 16, seed=11, near_solution=0.05)
    po = OracleProblem(w)
    lo, go = po.loss_grad(w.G)
    with native.Context(w.n, w.n_layers, w.psi1q, w.Uref, riemannian=True) as ctx:
        lg, gg = ctx.loss_grad(w.G)
        assert rel(gg, go) < 1e-5
        # three truncated-CG iterations inside a wide radius (positive
        # curvature along them here): the same Krylov steps from both sources
        # of HVPs
        ro = tr.truncated_cg(po, w.G, tr.project(w.G, go), 10.0, kappa=0.0, max_iter=3)
        rg = tr.truncated_cg(ctx, w.G, tr.project(w.G, gg), 10.0, kappa=0.0, max_iter=3)
        assert ro.stop == rg.stop == "max iterations" and ro.iterations == rg.iterations == 3
        assert rel(rg.eta, ro.eta) < 1e-4 and rel(rg.Heta, ro.Heta) < 1e-4
        st = tr.trust_region(ctx, w.G, steps=8)
    h0 = st.history[0]
    assert st.loss < 1e-4 * h0["loss"], (st.loss, h0["loss"])
    assert tr.norm(st.grad) < 1e-2 * h0["grad_norm"]
    losses = [h["loss"] for h in st.history] + [st.loss]
    for i, h in enumerate(st.history):
        if h["accepted"]:
            assert losses[i + 1] < losses[i]
    assert np.allclose(np.conj(np.swapaxes(st.G, -1, -2)) @ st.G, np.eye(4), atol=1e-12)
