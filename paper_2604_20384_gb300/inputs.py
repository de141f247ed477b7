"""Seeded synthetic workloads for the brickwall HVP problem.

This module only draws random inputs; it holds none of the method's
arithmetic (no state sweeps, no environments, no derivatives). It is the one
module that both the CUDA path's tests and the FP64 oracle consume, so that
both sides see identical inputs.

Problem statement (Sec. 3.1 and Sec. 4.1, Eq. costHS): a brickwall circuit of
two-qubit unitaries G^[k] on n qubits, a reference brickwall U_ref of the same
shape, N_s Haar-random single-qubit product input states psi_s and a
direction V (one 4x4 complex matrix per gate).

Layout conventions (the paper is silent on them; the same conventions are
written out independently in the oracle and in the CUDA library):
  * qubit 0 is the most significant bit of an amplitude index;
  * layer l (1-based) has offset (l-1) mod 2 and gates on qubits (i, i+1) for
    i = offset, offset+2, ... with i+1 <= n-1 (open boundary);
  * gates are ordered layer-major, then by first qubit ascending;
  * a gate's 4x4 matrix is indexed by 2*b_i + b_{i+1}.

Draw order with numpy PCG64(seed): (1) K Haar gates G; (2) K Haar gates of
U_ref; (3) N_s*n single-qubit states; (4) K complex Gaussian matrices A that
give V_k = G_k (A_k - A_k^dagger)/2. A near-solution variant draws (5) K more
Gaussian matrices B and replaces G_k by U_ref,k exp(eps (B_k - B_k^dagger)/2).
"""
from __future__ import annotations

import dataclasses

import numpy as np


def num_gates(n: int, n_layers: int) -> int:
    """Number of two-qubit gates of an open-boundary brickwall."""
    if n < 2 or n_layers < 1:
        raise ValueError("need n >= 2 and n_layers >= 1")
    return sum((n - ((layer - 1) % 2)) // 2 for layer in range(1, n_layers + 1))


def haar_unitary(rng: np.random.Generator, dim: int) -> np.ndarray:
    """Haar-random U(dim): QR of a complex Ginibre matrix with the phase fix
    of Mezzadri (2007)."""
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def haar_qubit_state(rng: np.random.Generator) -> np.ndarray:
    """Haar-random single-qubit pure state (normalised complex Gaussian)."""
    v = rng.standard_normal(2) + 1j * rng.standard_normal(2)
    return v / np.linalg.norm(v)


def _skew(a: np.ndarray) -> np.ndarray:
    return 0.5 * (a - a.conj().T)


def _expm_skew(x: np.ndarray) -> np.ndarray:
    """exp(X) for skew-Hermitian X through the eigendecomposition of the
    Hermitian matrix -iX."""
    w, u = np.linalg.eigh(-1j * x)
    return (u * np.exp(1j * w)[None, :]) @ u.conj().T


@dataclasses.dataclass
class Workload:
    """One synthetic problem instance. Complex arrays are complex128."""
    n: int
    n_layers: int
    n_samples: int
    G: np.ndarray        # (K, 4, 4)
    Uref: np.ndarray     # (K, 4, 4)
    psi1q: np.ndarray    # (N_s, n, 2)
    V: np.ndarray        # (K, 4, 4)
    seed: int

    @property
    def K(self) -> int:
        return self.G.shape[0]


def make_workload(n: int, n_layers: int, n_samples: int, seed: int = 0,
                  near_solution: float | None = None) -> Workload:
    """Draw a workload in the fixed order described in the module docstring.

    near_solution=eps replaces G_k by U_ref,k exp(eps X_k) with a fresh
    skew-Hermitian X_k, so that the overlaps are O(1) as late in an
    optimisation (Sec. 3.3 and Sec. 4.2 start from circuits close to U_ref).
    """
    K = num_gates(n, n_layers)
    rng = np.random.Generator(np.random.PCG64(seed))
    G = np.stack([haar_unitary(rng, 4) for _ in range(K)])
    Uref = np.stack([haar_unitary(rng, 4) for _ in range(K)])
    psi1q = np.stack([np.stack([haar_qubit_state(rng) for _ in range(n)])
                      for _ in range(n_samples)]) if n_samples > 0 else np.zeros((0, n, 2), complex)
    A = rng.standard_normal((K, 4, 4)) + 1j * rng.standard_normal((K, 4, 4))
    if near_solution is not None:
        B = rng.standard_normal((K, 4, 4)) + 1j * rng.standard_normal((K, 4, 4))
        G = np.stack([Uref[k] @ _expm_skew(near_solution * _skew(B[k])) for k in range(K)])
    V = np.stack([G[k] @ _skew(A[k]) for k in range(K)])
    return Workload(n=n, n_layers=n_layers, n_samples=n_samples, G=G, Uref=Uref,
                    psi1q=psi1q, V=V, seed=seed)


def random_direction(K: int, G: np.ndarray, seed: int) -> np.ndarray:
    """An extra tangent direction G_k (A_k - A_k^dagger)/2 from its own seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    A = rng.standard_normal((K, 4, 4)) + 1j * rng.standard_normal((K, 4, 4))
    return np.stack([G[k] @ _skew(A[k]) for k in range(K)])


# The five workload shapes of the benchmark plan: a tiny FP64 case, a
# precision-comparison case, the headline HVP workload, a batch of uneven
# circuits and a large differentiation case.
WORKLOADS = {
    "n6_L3_Ns16": dict(n=6, n_layers=3, n_samples=16),
    "n12_L8_Ns256": dict(n=12, n_layers=8, n_samples=256),
    "n20_L16_Ns64": dict(n=20, n_layers=16, n_samples=64),
    "n26_L24_Ns8": dict(n=26, n_layers=24, n_samples=8),
}


def uneven_batch_shapes(n_circuits: int = 64, seed: int = 0):
    """Shapes of the uneven batch: n ~ U{8..16}, L ~ U{4..20}, N_s
    log-uniform in [32, 512] (rounded). Returns a list of (n, L, N_s, seed)."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000003))
    shapes = []
    for c in range(n_circuits):
        n = int(rng.integers(8, 17))
        L = int(rng.integers(4, 21))
        ns = int(round(float(np.exp(rng.uniform(np.log(32.0), np.log(512.0))))))
        shapes.append((n, L, ns, seed * 1000 + c))
    return shapes


def make_uneven_batch(n_circuits: int = 64, seed: int = 0):
    return [make_workload(n, L, ns, s) for (n, L, ns, s) in uneven_batch_shapes(n_circuits, seed)]


def as_interleaved(a: np.ndarray) -> np.ndarray:
    """C-contiguous float64 view (re, im interleaved) of a complex array."""
    return np.ascontiguousarray(a, dtype=np.complex128).view(np.float64)
