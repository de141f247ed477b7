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


def _phi_chunk(args):
    n, L, uref, psi1q = args
    return oracle.reference_states(n, L, uref, psi1q)


def oracle_parallel(w, G=None, V=None):
    """Oracle on every sample of workload w using the host's cores: reference
    states in a spawned process pool (chunks of samples), then one evaluation
    with a thread per core."""
    import multiprocessing as mp
    import os

    cores = os.cpu_count() or 1
    step = max(1, -(-w.n_samples // cores))
    chunks = [w.psi1q[i:i + step] for i in range(0, w.n_samples, step)]
    if len(chunks) > 1:
        with mp.get_context("spawn").Pool(min(cores, len(chunks))) as pool:
            parts = pool.map(_phi_chunk, [(w.n, w.n_layers, w.Uref, c) for c in chunks])
        phi = np.concatenate(parts)
    else:
        phi = oracle.reference_states(w.n, w.n_layers, w.Uref, w.psi1q)
    o = oracle.evaluate(w.n, w.n_layers, w.G if G is None else G, w.V if V is None else V, w.psi1q, phi,
                        threads=cores, ckpt_stride=max(1, int(round(w.K ** 0.5))))
    return phi, o


_HEADLINE = {}


def headline_oracle():
    """The benchmark workload (n = 20, L = 16, N_s = 64, seed 0) and the oracle
    on all of its samples: reference states in a spawned process pool (chunks
    of samples), then one oracle evaluation with a thread per host core and
    forward checkpoints every 12 gates. Cached for the test session (about a
    minute on 16 cores)."""
    if "o" not in _HEADLINE:
        w = make_workload(20, 16, 64, seed=0)
        phi, o = oracle_parallel(w)
        _HEADLINE.update(w=w, phi=phi, o=o)
    return _HEADLINE["w"], _HEADLINE["phi"], _HEADLINE["o"]


def layer_of_gates(n: int, n_layers: int) -> np.ndarray:
    """Layer index (0-based) of every gate in the brickwall order (the
    convention of the library's header)."""
    out = []
    for layer in range(n_layers):
        out += [layer] * ((n - layer % 2) // 2)
    return np.array(out, dtype=np.int64)


def expand(layer_gates, n: int, n_layers: int) -> np.ndarray:
    """(L, 4, 4) layer gates -> (K, 4, 4), every gate of a layer the layer's."""
    return np.asarray(layer_gates, dtype=np.complex128)[layer_of_gates(n, n_layers)]


def contract(per_gate, n: int, n_layers: int) -> np.ndarray:
    """(K, 4, 4) per-gate blocks -> (L, 4, 4) sums over each layer."""
    out = np.zeros((n_layers, 4, 4), dtype=np.complex128)
    np.add.at(out, layer_of_gates(n, n_layers), np.asarray(per_gate))
    return out
