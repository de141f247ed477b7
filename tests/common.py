"""Shared helpers of the test suite (no method arithmetic beyond what a test
states as the property it checks)."""
from __future__ import annotations

import numpy as np

from oracle import oracle
from paper_2604_20384_gb300.inputs import make_workload


def rel(a, b) -> float:
    """||a - b||_F / ||b||_F (absolute when b == 0)."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b.ravel())
    d = np.linalg.norm((a - b).ravel())
    return float(d / nb) if nb > 0 else float(d)


def re_inner(a, b) -> float:
    """Re <A, B> = Re Tr(A^dagger B) summed over gates (the metric of App. F)."""
    return float(np.real(np.vdot(np.asarray(a).ravel(), np.asarray(b).ravel())))


def oracle_case(n, L, ns, seed=0, near_solution=None, threads=None, **kw):
    w = make_workload(n, L, ns, seed, near_solution=near_solution)
    phi = oracle.reference_states(n, L, w.Uref, w.psi1q)
    out = oracle.evaluate(n, L, w.G, w.V, w.psi1q, phi, threads=threads, **kw)
    return w, phi, out


def loss_at(w, phi, G, threads=None):
    return oracle.evaluate(w.n, w.n_layers, G, None, w.psi1q, phi, threads=threads)["loss"]


def grad_at(w, phi, G, threads=None):
    return oracle.evaluate(w.n, w.n_layers, G, None, w.psi1q, phi, threads=threads)["grad"]


def expm_skew(x):
    w, u = np.linalg.eigh(-1j * x)
    return (u * np.exp(1j * w)[None, :]) @ u.conj().T
