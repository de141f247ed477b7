"""Dense brute-force evaluation for tiny n (test infrastructure only).

It shares nothing with oracle.c: it builds the full 2^n x 2^n brickwall
unitary from Kronecker products of layer operators and obtains every
derivative by substitution, using only that the overlap
T = phi^dagger G_K ... G_1 psi is linear in each gate (Sec. 2.2):
  * dT/dG_k[i][j]  = T with G_k replaced by the elementary matrix e_ij
                     (Eq. environment);
  * D(dT/dG_k)[V]  = sum over k' != k of T with G_k <- e_ij and G_k' <- V_k'
                     (the derivative of a multilinear function);
  * Omega = D T[V] = sum_k T with G_k <- V_k (Eq. Omega).
Loss and derivatives of C = 1 - mean|T|^2 then follow from the chain rule in
Wirtinger form (App. A): grad C = -(2/N_s) sum T conj(dT/dG), and its
directional derivative along V.
"""
from __future__ import annotations

import numpy as np


def layer_gate_indices(n: int, n_layers: int):
    """[(layer, first_qubit, k)] in the brickwall order, written out here
    independently of every other implementation."""
    out, k = [], 0
    for layer in range(n_layers):
        i = layer % 2
        while i + 1 <= n - 1:
            out.append((layer, i, k))
            k += 1
            i += 2
    return out


def circuit_matrix(n: int, n_layers: int, gates) -> np.ndarray:
    """Dense matrix G_K ... G_1 of a brickwall whose k-th gate is gates[k]."""
    idx = layer_gate_indices(n, n_layers)
    U = np.eye(1 << n, dtype=complex)
    for layer in range(n_layers):
        factors, q = [], 0
        members = {i: k for (lay, i, k) in idx if lay == layer}
        while q < n:
            if q in members:
                factors.append(np.asarray(gates[members[q]], dtype=complex))
                q += 2
            else:
                factors.append(np.eye(2, dtype=complex))
                q += 1
        L = factors[0]
        for f in factors[1:]:
            L = np.kron(L, f)
        U = L @ U
    return U


def product_state(psi1q_s: np.ndarray) -> np.ndarray:
    v = np.array([1.0 + 0j])
    for q in range(psi1q_s.shape[0]):
        v = np.kron(v, psi1q_s[q])
    return v


def evaluate(n: int, n_layers: int, G, V, psi1q, Uref) -> dict:
    """Brute-force loss, T, Omega, E, DE, gradient and HVP of C."""
    G = np.asarray(G, complex)
    V = np.asarray(V, complex)
    K = G.shape[0]
    ns = psi1q.shape[0]
    psis = np.stack([product_state(psi1q[s]) for s in range(ns)])          # (ns, d)
    phis = psis @ circuit_matrix(n, n_layers, Uref).T                        # phi_s = U_ref psi_s

    def overlaps(gates):
        M = circuit_matrix(n, n_layers, gates)
        return np.einsum("sd,de,se->s", phis.conj(), M, psis)

    T = overlaps(list(G))
    E = np.zeros((ns, K, 4, 4), complex)
    DE = np.zeros((ns, K, 4, 4), complex)
    for k in range(K):
        for i in range(4):
            for j in range(4):
                e = np.zeros((4, 4), complex)
                e[i, j] = 1.0
                gates = list(G)
                gates[k] = e
                E[:, k, i, j] = overlaps(gates)
                acc = np.zeros(ns, complex)
                for kp in range(K):
                    if kp == k:
                        continue
                    g2 = list(gates)
                    g2[kp] = V[kp]
                    acc += overlaps(g2)
                DE[:, k, i, j] = acc
    Omega = np.zeros(ns, complex)
    for k in range(K):
        gates = list(G)
        gates[k] = V[k]
        Omega += overlaps(gates)
    loss = 1.0 - np.mean(np.abs(T) ** 2)
    grad = -(2.0 / ns) * np.einsum("s,skij->kij", T, E.conj())
    hvp = -(2.0 / ns) * (np.einsum("s,skij->kij", Omega, E.conj())
                         + np.einsum("s,skij->kij", T, DE.conj()))
    loss_f = 1.0 - np.mean(T.real)                       # Frobenius cost (Eq. Frobenius)
    grad_f = -(1.0 / ns) * E.conj().sum(axis=0)
    hvp_f = -(1.0 / ns) * DE.conj().sum(axis=0)
    return dict(loss=loss, T=T, Omega=Omega, E=E, DE=DE, grad=grad, hvp=hvp, phi=phis, psi=psis,
                loss_f=loss_f, grad_f=grad_f, hvp_f=hvp_f)
