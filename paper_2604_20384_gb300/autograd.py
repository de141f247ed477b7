"""PyTorch integration: the sampled Hilbert-Schmidt cost as differentiable
functions of the gate tensor G (complex128, shape (K, 4, 4), on the GPU).

* ``HSLoss.apply(G, cost)`` returns C(G) (Eq. costHS); its backward is the
  adjoint sweep: grad_out * grad C, where grad C = dC/dRe + i dC/dIm
  (Eq. grad-real), which is PyTorch's gradient convention for a real loss of
  complex inputs.
* ``HSGrad.apply(G, cost)`` returns grad C(G). Its forward-mode derivative
  (``jvp``) along V is the Hessian-vector product D(grad C)[V] computed by the
  tangent sweep (forward-over-reverse, Eq. FoR); its backward applied to W
  returns H[W] as well (the Hessian is self-adjoint for Re<., .>).
* ``hvp(G, V, cost)`` is the forward-mode derivative of ``HSGrad`` along V
  (dual tensors of ``torch.autograd.forward_ad``). Since the tangent is
  known before the primal is evaluated, the primal and its jvp come from one
  tangent sweep (which returns the gradient as well) instead of an adjoint
  sweep followed by a tangent sweep.

All arithmetic runs in libhvp; tensors are passed as device pointers and the
work is ordered against PyTorch's current stream with stream waits.
"""
from __future__ import annotations

import torch

from . import native


class HSCost:
    """A loss/gradient/HVP problem (brickwall shape, samples, reference) bound
    to one GPU. Keyword arguments are those of :class:`native.Context`."""

    def __init__(self, n: int, n_layers: int, psi1q, ref, device: int = 0, **kw):
        self.device = torch.device("cuda", device)
        self.stream = torch.cuda.Stream(device=self.device)
        self.ctx = native.Context(n, n_layers, psi1q, ref, device=device, stream=self.stream.cuda_stream, **kw)
        self.K = self.ctx.K
        self._fused_tangent = None   # set by hvp(): the tangent of the next HSGrad
        self._fused_hv = None        # (tangent, H[tangent]) left by that HSGrad forward

    def _run(self, G: torch.Tensor, V: torch.Tensor | None, want_hvp: bool):
        if G.dtype != torch.complex128 or G.shape != (self.K, 4, 4) or G.device != self.device:
            raise ValueError(f"G must be complex128 of shape ({self.K}, 4, 4) on {self.device}")
        cur = torch.cuda.current_stream(self.device)
        G = G.detach().contiguous()
        Vc = None if V is None else V.detach().to(torch.complex128).contiguous()
        loss = torch.empty(1, dtype=torch.float64, device=self.device)
        grad = torch.empty(self.K, 4, 4, dtype=torch.complex128, device=self.device)
        hv = torch.empty(self.K, 4, 4, dtype=torch.complex128, device=self.device) if want_hvp else None
        self.stream.wait_stream(cur)
        for t in (G, Vc, loss, grad, hv):
            if t is not None:
                t.record_stream(self.stream)
        self.ctx.hvp_dev(G.data_ptr(), None if Vc is None else Vc.data_ptr(), loss.data_ptr(), grad.data_ptr(),
                         None if hv is None else hv.data_ptr())
        cur.wait_stream(self.stream)
        return loss.reshape(()).clone(), grad, hv

    def loss_grad(self, G: torch.Tensor):
        loss, grad, _ = self._run(G, None, False)
        return loss, grad

    def loss_grad_hvp(self, G: torch.Tensor, V: torch.Tensor):
        return self._run(G, V, True)

    def close(self):
        self.ctx.close()


class HSLoss(torch.autograd.Function):
    """C(G); backward = grad_out * grad C (the adjoint sweep of Alg. 1)."""

    @staticmethod
    def forward(G, cost):
        loss, grad = cost.loss_grad(G)
        return loss, grad

    @staticmethod
    def setup_context(ctx, inputs, output):
        ctx.save_for_backward(output[1])
        ctx.mark_non_differentiable(output[1])

    @staticmethod
    def backward(ctx, gout, _ggrad):
        (grad,) = ctx.saved_tensors
        return gout * grad, None


class HSGrad(torch.autograd.Function):
    """grad C(G); jvp along V = H[V] (tangent sweep); backward of W = H[W]."""

    @staticmethod
    def forward(G, cost):
        V = cost._fused_tangent
        if V is None:
            return cost.loss_grad(G)[1]
        _, grad, hv = cost.loss_grad_hvp(G, V)
        cost._fused_hv = (V, hv)
        return grad

    @staticmethod
    def setup_context(ctx, inputs, output):
        G, cost = inputs
        ctx.cost = cost
        ctx.save_for_backward(G)
        ctx.save_for_forward(G)

    @staticmethod
    def jvp(ctx, V, _dcost):
        stash, ctx.cost._fused_hv = ctx.cost._fused_hv, None
        if stash is not None and stash[0].data_ptr() == V.data_ptr() and stash[0].shape == V.shape:
            return stash[1]
        (G,) = ctx.saved_tensors
        return ctx.cost.loss_grad_hvp(G, V)[2]

    @staticmethod
    def backward(ctx, W):
        (G,) = ctx.saved_tensors
        return ctx.cost.loss_grad_hvp(G, W)[2], None


def loss(G: torch.Tensor, cost: HSCost) -> torch.Tensor:
    """Differentiable C(G)."""
    return HSLoss.apply(G, cost)[0]


def grad(G: torch.Tensor, cost: HSCost) -> torch.Tensor:
    """grad C(G), differentiable in forward mode (jvp = HVP)."""
    return HSGrad.apply(G, cost)


def hvp(G: torch.Tensor, V: torch.Tensor, cost: HSCost):
    """(grad C(G), H C(G)[V]) by forward-over-reverse: the forward-mode
    derivative of grad C along V."""
    import torch.autograd.forward_ad as fwAD

    T = V.detach().to(G.dtype).contiguous()
    with fwAD.dual_level():
        cost._fused_tangent = T
        try:
            out = HSGrad.apply(fwAD.make_dual(G.detach(), T), cost)
        finally:
            cost._fused_tangent = None
            cost._fused_hv = None
        primal, tangent = fwAD.unpack_dual(out)
    return primal, tangent
