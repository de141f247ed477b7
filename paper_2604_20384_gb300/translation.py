"""Translation-invariant brickwalls (App. E, Alg. 3): every gate of layer l
is the same layer gate G_l, and the direction is layer-wise constant too.

The library does the work on the device (flag HVP_TRANSLATION): it expands
the layer gates to every gate of their layer and sums the per-gate
derivative blocks over each layer in FP64 (the chain rule through the tying
map). This module only builds such a context and marshals (L, 4, 4) arrays.
"""
from __future__ import annotations

from . import native


class TranslationInvariant:
    """Loss, gradient and HVP with respect to the L layer gates of a
    brickwall; keyword arguments as for :class:`native.Context`."""

    def __init__(self, n: int, n_layers: int, psi1q, ref, **kw):
        self.ctx = native.Context(n, n_layers, psi1q, ref, translation=True, **kw)
        self.n, self.L = n, n_layers

    def loss_grad(self, Gl):
        return self.ctx.loss_grad(Gl)

    def hvp(self, Gl, Vl):
        return self.ctx.hvp(Gl, Vl)

    def hvp_dev(self, Gl_ptr: int, Vl_ptr: int | None, loss_ptr: int | None, grad_ptr: int | None,
                hvp_ptr: int | None):
        self.ctx.hvp_dev(Gl_ptr, Vl_ptr, loss_ptr, grad_ptr, hvp_ptr)

    def close(self):
        self.ctx.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
