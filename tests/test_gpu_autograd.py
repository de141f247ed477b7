"""The torch.autograd layer (differentiation form): loss backward = adjoint
sweep, jvp of the gradient = tangent sweep (forward-over-reverse HVP),
checked against the FP64 oracle and against central finite differences of
the loss computed by the library itself (Eq. grad-real, Eq. FoR)."""
import numpy as np
import pytest

from common import rel
from oracle import oracle
from paper_2604_20384_gb300.inputs import make_workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to("cuda:0")


def test_autograd_loss_grad_and_hvp_match_oracle():
    from paper_2604_20384_gb300 import autograd as hsa

    w = make_workload(11, 7, 12, seed=3)
    phi = oracle.reference_states(11, 7, w.Uref, w.psi1q)
    o = oracle.evaluate(11, 7, w.G, w.V, w.psi1q, phi)
    cost = hsa.HSCost(11, 7, w.psi1q, w.Uref, window=9)
    G = _t(w.G).requires_grad_(True)
    L = hsa.loss(G, cost)
    L.backward()
    assert abs((1 - L.item()) - (1 - o["loss"])) <= 1e-5 * (1 - o["loss"])
    assert rel(G.grad.cpu().numpy(), o["grad"]) < 1e-5
    g, hv = hsa.hvp(_t(w.G), _t(w.V), cost)
    assert rel(g.cpu().numpy(), o["grad"]) < 1e-5
    assert rel(hv.cpu().numpy(), o["hvp"]) < 1e-5
    # reverse mode through the gradient: d/dG Re<W, grad C> = H[W]
    G2 = _t(w.G).requires_grad_(True)
    gr = hsa.grad(G2, cost)
    Wt = _t(w.V)
    torch.real(torch.sum(Wt.conj() * gr)).backward()
    assert rel(G2.grad.cpu().numpy(), o["hvp"]) < 1e-5
    cost.close()


def test_differentiation_form_n26_checkpointed_against_finite_differences():
    # n = 26, L = 24 (K = 300), N_s = 8, complex64, forward checkpoints every
    # 2 window passes (about 5 layers) with the others recomputed; gradient
    # against central differences (h = 1e-3) of the library's own loss on 16
    # random gate entries (real and imaginary directions). Near-solution gates
    # keep the overlaps O(1) so that the differences are well conditioned in
    # complex64.
    from paper_2604_20384_gb300 import autograd as hsa

    w = make_workload(26, 24, 8, seed=0, near_solution=0.1)
    cost = hsa.HSCost(26, 24, w.psi1q, w.Uref, checkpoint_stride=2)
    info = cost.ctx.plan_info()
    assert info["checkpoint_stride"] == 2 and info["passes"] > 4
    G = _t(w.G).requires_grad_(True)
    L = hsa.loss(G, cost)
    L.backward()
    grad = G.grad.cpu().numpy()
    rng = np.random.default_rng(7)
    h = 1e-3
    errs = []
    for _ in range(16):
        k, i, j = int(rng.integers(w.K)), int(rng.integers(4)), int(rng.integers(4))
        for direction in (1.0, 1j):
            E = np.zeros_like(w.G)
            E[k, i, j] = h * direction
            lp = hsa.loss(_t(w.G + E), cost).item()
            lm = hsa.loss(_t(w.G - E), cost).item()
            fd = (lp - lm) / (2 * h)
            an = grad[k, i, j].real if direction == 1.0 else grad[k, i, j].imag
            errs.append(abs(fd - an) / max(np.abs(grad).max(), 1e-12))
    assert max(errs) < 1e-3, max(errs)
    # the HVP of the same configuration equals the directional derivative of
    # the gradient (Richardson-free central difference, loose bound)
    g0, hv = hsa.hvp(_t(w.G), _t(w.V), cost)
    eps = 1e-3
    gp = hsa.grad(_t(w.G + eps * w.V), cost)
    gm = hsa.grad(_t(w.G - eps * w.V), cost)
    fd = ((gp - gm) / (2 * eps)).cpu().numpy()
    assert rel(hv.cpu().numpy(), fd) < 1e-2
    cost.close()
