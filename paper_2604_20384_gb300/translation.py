"""Translation-invariant brickwalls (App. E, Alg. 3): every gate of layer l
is the same layer gate G_l, and the direction is layer-wise constant too.

By the chain rule the derivatives with respect to a layer gate are the sums of
the per-gate derivatives over the gates of that layer (App. E), for the
gradient and the HVP alike; the Riemannian forms are linear in those sums for
a fixed G_l, so they sum the same way. This wrapper expands layer gates to
the per-gate arrays of a context and sums the results back per layer.
"""
from __future__ import annotations

import numpy as np


def layer_of_gates(n: int, n_layers: int) -> np.ndarray:
    """Layer index (0-based) of every gate in the brickwall order."""
    out = []
    for layer in range(n_layers):
        out += [layer] * ((n - layer % 2) // 2)
    return np.array(out, dtype=np.int64)


def expand(layer_gates, n: int, n_layers: int) -> np.ndarray:
    """(L, 4, 4) layer gates -> (K, 4, 4) per-gate array."""
    return np.asarray(layer_gates, dtype=np.complex128)[layer_of_gates(n, n_layers)]


def contract(per_gate, n: int, n_layers: int) -> np.ndarray:
    """(K, 4, 4) per-gate derivatives -> (L, 4, 4) sums over each layer."""
    out = np.zeros((n_layers, 4, 4), dtype=np.complex128)
    np.add.at(out, layer_of_gates(n, n_layers), np.asarray(per_gate))
    return out


class TranslationInvariant:
    """Loss, gradient and HVP with respect to layer gates, on top of a
    :class:`paper_2604_20384_gb300.native.Context` for the same brickwall."""

    def __init__(self, ctx):
        self.ctx = ctx
        self.n, self.L = ctx.n, ctx.n_layers

    def loss_grad(self, Gl):
        loss, g = self.ctx.loss_grad(expand(Gl, self.n, self.L))
        return loss, contract(g, self.n, self.L)

    def hvp(self, Gl, Vl):
        loss, g, h = self.ctx.hvp(expand(Gl, self.n, self.L), expand(Vl, self.n, self.L))
        return loss, contract(g, self.n, self.L), contract(h, self.n, self.L)
