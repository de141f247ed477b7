"""Host logic of the torch.autograd layer, with a stand-in cost on the CPU:
the quadratic C(G) = Re<G, A G> (A Hermitian, acting on the flattened gates),
whose gradient in PyTorch's convention is 2 A G and whose Hessian applied to
V is 2 A V. Checks that forward-over-reverse returns those, that the primal
and the jvp of hvp() come from a single loss/gradient/HVP call, and that the
reverse-mode and plain-gradient paths still make their own calls."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2604_20384_gb300 import autograd as hsa  # noqa: E402


class QuadraticCost:
    def __init__(self, K, seed=0):
        rng = np.random.default_rng(seed)
        m = 16 * K
        X = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
        self.A = torch.from_numpy((X + X.conj().T) / 2)
        self.K = K
        self.calls = {"loss_grad": 0, "loss_grad_hvp": 0}
        self._fused_tangent = None
        self._fused_hv = None

    def _apply(self, X):
        return (self.A @ X.reshape(-1)).reshape(self.K, 4, 4)

    def loss_grad(self, G):
        self.calls["loss_grad"] += 1
        G = G.detach()
        AG = self._apply(G)
        return torch.real(torch.vdot(G.reshape(-1), AG.reshape(-1))), 2 * AG

    def loss_grad_hvp(self, G, V):
        self.calls["loss_grad_hvp"] += 1
        loss, grad = self.loss_grad(G)
        self.calls["loss_grad"] -= 1
        return loss, grad, 2 * self._apply(V.detach())


def _rand(K, seed):
    rng = np.random.default_rng(seed)
    return torch.from_numpy(rng.standard_normal((K, 4, 4)) + 1j * rng.standard_normal((K, 4, 4)))


def test_forward_over_reverse_uses_one_sweep():
    K = 3
    cost = QuadraticCost(K)
    G, V = _rand(K, 1), _rand(K, 2)
    g, hv = hsa.hvp(G, V, cost)
    assert cost.calls == {"loss_grad": 0, "loss_grad_hvp": 1}
    assert torch.allclose(g, 2 * cost._apply(G))
    assert torch.allclose(hv, 2 * cost._apply(V))
    assert cost._fused_tangent is None and cost._fused_hv is None
    # a second call with another direction gives that direction's product
    V2 = _rand(K, 3)
    _, hv2 = hsa.hvp(G, V2, cost)
    assert torch.allclose(hv2, 2 * cost._apply(V2))
    assert cost.calls == {"loss_grad": 0, "loss_grad_hvp": 2}


def test_loss_backward_and_gradient_reverse_mode():
    K = 2
    cost = QuadraticCost(K, seed=4)
    G = _rand(K, 5).requires_grad_(True)
    hsa.loss(G, cost).backward()
    assert cost.calls == {"loss_grad": 1, "loss_grad_hvp": 0}
    assert torch.allclose(G.grad, 2 * cost._apply(G.detach()))
    # reverse mode through the gradient: d/dG Re<W, grad C> = H[W] (self-adjoint)
    G2 = _rand(K, 5).requires_grad_(True)
    W = _rand(K, 6)
    torch.real(torch.sum(W.conj() * hsa.grad(G2, cost))).backward()
    assert torch.allclose(G2.grad, 2 * cost._apply(W))
    assert cost.calls == {"loss_grad": 2, "loss_grad_hvp": 1}


def test_jvp_of_plain_gradient_computes_its_own_product():
    # a dual tensor built outside hvp(): no tangent was announced, so the
    # forward takes the adjoint sweep and the jvp its own tangent sweep
    import torch.autograd.forward_ad as fwAD

    K = 2
    cost = QuadraticCost(K, seed=7)
    G, V = _rand(K, 8), _rand(K, 9)
    with fwAD.dual_level():
        out = hsa.grad(fwAD.make_dual(G, V), cost)
        _, t = fwAD.unpack_dual(out)
    assert cost.calls == {"loss_grad": 1, "loss_grad_hvp": 1}
    assert torch.allclose(t, 2 * cost._apply(V))
