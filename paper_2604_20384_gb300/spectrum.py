"""Dense Riemannian Hessian of the sampled cost from Hessian-vector products
(App. G): with the tangent basis E_(k,a,b) = i G_k (P_a (x) P_b) / 2 (Pauli
matrices P in {I, X, Y, Z}, the other gates zero), which is orthonormal for
the metric Re Tr(A^dag B) when G_k is unitary, the matrix entries are
H_ij = Re <E_i, H_R[E_j]>, one Riemannian HVP per column (16 K columns). The
matrix is symmetric (self-adjointness of H_R) and its eigenvalues are real.
"""
from __future__ import annotations

import numpy as np

_P = [np.eye(2, dtype=complex), np.array([[0, 1], [1, 0]], dtype=complex),
      np.array([[0, -1j], [1j, 0]], dtype=complex), np.array([[1, 0], [0, -1]], dtype=complex)]


def tangent_basis(G) -> np.ndarray:
    """(16 K, K, 4, 4): direction j has one nonzero gate block."""
    G = np.asarray(G, dtype=np.complex128)
    K = G.shape[0]
    B = np.zeros((16 * K, K, 4, 4), dtype=np.complex128)
    for k in range(K):
        for a in range(4):
            for b in range(4):
                B[16 * k + 4 * a + b, k] = 0.5j * G[k] @ np.kron(_P[a], _P[b])
    return B


def riemannian_hessian(hvp_fn, G, hvp_multi_fn=None, chunk: int = 64) -> np.ndarray:
    """Dense (16K x 16K) matrix in the Pauli tangent basis. hvp_fn(G, V)
    returns the Riemannian HVP H_R[V] as a (K, 4, 4) array (for example a
    context created with riemannian=True: lambda G, V: ctx.hvp(G, V)[2]).
    With hvp_multi_fn(G, Vs) -> (n_dir, K, 4, 4) (e.g. a context with
    riemannian=True and multi_dir=True: lambda G, Vs: ctx.hvp_multi(G, Vs)[2])
    the columns are evaluated `chunk` directions per call, which the library
    sends through its sweeps in pairs."""
    B = tangent_basis(G)
    n = B.shape[0]
    Bf = B.reshape(n, -1)
    H = np.zeros((n, n))
    if hvp_multi_fn is not None:
        for j0 in range(0, n, chunk):
            cols = np.asarray(hvp_multi_fn(G, B[j0:j0 + chunk])).reshape(-1, Bf.shape[1])
            H[:, j0:j0 + cols.shape[0]] = np.real(Bf.conj() @ cols.T)
        return H
    for j in range(n):
        col = np.asarray(hvp_fn(G, B[j])).reshape(-1)
        H[:, j] = np.real(Bf.conj() @ col)
    return H


def spectrum(H: np.ndarray) -> np.ndarray:
    """Eigenvalues of the symmetrised matrix, ascending."""
    return np.linalg.eigvalsh(0.5 * (H + H.T))
