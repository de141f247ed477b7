"""Riemannian trust-region driver (Absil et al. 2008, Algorithms 10 and 11, as
used in Sec. 4) on a tiny problem, with the FP64 oracle as the source of
Riemannian gradients and HVPs (CPU)."""
import numpy as np

from common import rel
from oracle import oracle
from paper_2604_20384_gb300 import trust_region as tr
from paper_2604_20384_gb300.inputs import make_workload, random_direction


class OracleProblem:
    def __init__(self, w):
        self.w = w
        self.phi = oracle.reference_states(w.n, w.n_layers, w.Uref, w.psi1q)
        self.hvps = 0

    def loss_grad(self, G):
        o = oracle.evaluate(self.w.n, self.w.n_layers, G, None, self.w.psi1q, self.phi)
        return o["loss"], o["grad_r"]

    def hvp(self, G, V):
        self.hvps += 1
        o = oracle.evaluate(self.w.n, self.w.n_layers, G, V, self.w.psi1q, self.phi)
        return o["loss"], o["grad_r"], o["hvp_r"]


def test_retraction_and_projection():
    w = make_workload(4, 3, 2, seed=1)
    X = random_direction(w.K, w.G, seed=2)
    xi = tr.project(w.G, X)
    R = tr.retract(w.G, 1e-3 * xi)
    eye = np.eye(4)
    assert np.allclose(np.conj(np.swapaxes(R, -1, -2)) @ R, eye, atol=1e-13)       # unitary
    # R(t xi) = G + t xi + O(t^2): halving t quarters the remainder
    e1 = tr.norm(tr.retract(w.G, 1e-3 * xi) - w.G - 1e-3 * xi)
    e2 = tr.norm(tr.retract(w.G, 5e-4 * xi) - w.G - 5e-4 * xi)
    assert 3.5 < e1 / e2 < 4.5, e1 / e2
    assert rel(tr.project(w.G, xi), xi) < 1e-13                                    # tangent
    assert rel(tr.project(w.G, tr.project(w.G, X)), tr.project(w.G, X)) < 1e-13  # idempotent


def test_truncated_cg_model_decrease_and_radius():
    w = make_workload(4, 3, 6, seed=3, near_solution=0.3)
    p = OracleProblem(w)
    loss, g = p.loss_grad(w.G)
    g = tr.project(w.G, g)
    for delta in (1e-3, 1e-1, 10.0):
        res = tr.truncated_cg(p, w.G, g, delta)
        assert tr.norm(res.eta) <= delta * (1 + 1e-12)
        m = tr.inner(g, res.eta) + 0.5 * tr.inner(res.eta, res.Heta)
        assert m < 0                                                 # the model decreases
        Hd = p.hvp(w.G, res.eta)[2]                                  # Heta kept by linearity
        assert rel(tr.project(w.G, Hd), res.Heta) < 1e-9
        # at least the Cauchy decrease along -g (Algorithm 11 starts there)
        gg = tr.inner(g, g)
        Hg = tr.inner(g, tr.project(w.G, p.hvp(w.G, g)[2]))
        t = delta / np.sqrt(gg) if Hg <= 0 else min(gg / Hg, delta / np.sqrt(gg))
        cauchy = -t * gg + 0.5 * t * t * Hg
        assert m <= cauchy + 1e-12 * abs(cauchy)


def test_trust_region_converges_near_the_solution():
    # Near G = U_ref (a global minimum, cost 0) the iteration must decrease the
    # cost monotonically on accepted steps and drive the Riemannian gradient
    # down by orders of magnitude within a few steps.
    w = make_workload(5, 3, 8, seed=7, near_solution=0.2)
    p = OracleProblem(w)
    st = tr.trust_region(p, w.G, steps=12)
    losses = [h["loss"] for h in st.history] + [st.loss]
    acc = [h["accepted"] for h in st.history]
    for i, a in enumerate(acc):
        if a:
            assert losses[i + 1] < losses[i]
    assert st.loss < 1e-3 * st.history[0]["loss"]
    assert tr.norm(st.grad) < 1e-3 * st.history[0]["grad_norm"]
    assert np.allclose(np.conj(np.swapaxes(st.G, -1, -2)) @ st.G, np.eye(4), atol=1e-12)
