"""ctypes front end of the FP64 oracle in oracle.c (test infrastructure only).

Every quantity follows arXiv 2604.20384: Alg. 1 (with the pre-update
backward order of Eq. overlap-hvp), Alg. 2, Eq. costHS and App. F. See the
header of oracle.c for the readings of the paper that it takes.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_layout.argtypes = [ctypes.c_int, ctypes.c_int, _ip]
        lib.oracle_layout.restype = ctypes.c_int
        lib.oracle_reference_states.argtypes = [ctypes.c_int] * 3 + [_dp] * 3
        lib.oracle_reference_states.restype = ctypes.c_int
        lib.oracle_hvp.argtypes = ([ctypes.c_int] * 3 + [_dp] * 4 + [ctypes.c_int] * 2 + [_dp] * 16)
        lib.oracle_hvp.restype = ctypes.c_int
        lib.oracle_project.argtypes = [ctypes.c_int, _dp, _dp, _dp]
        lib.oracle_project.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def layout(n: int, n_layers: int) -> np.ndarray:
    """First qubit i of every gate (i, i+1), in the oracle's own layout code."""
    lib = _load()
    K = lib.oracle_layout(n, n_layers, None)
    fq = np.zeros(K, dtype=np.int32)
    lib.oracle_layout(n, n_layers, fq.ctypes.data_as(_ip))
    return fq


def reference_states(n: int, n_layers: int, uref: np.ndarray, psi1q: np.ndarray) -> np.ndarray:
    """phi_s = U_ref psi_s as an (N_s, 2^n) complex128 array."""
    lib = _load()
    uref, psi1q = _c128(uref), _c128(psi1q)
    ns = psi1q.shape[0]
    phi = np.zeros((ns, 1 << n), dtype=np.complex128)
    rc = lib.oracle_reference_states(n, n_layers, ns, _ptr(uref.view(np.float64)),
                                     _ptr(psi1q.view(np.float64)), _ptr(phi.view(np.float64)))
    if rc != 0:
        raise RuntimeError(f"oracle_reference_states failed: {rc}")
    return phi


def evaluate(n: int, n_layers: int, G: np.ndarray, V: np.ndarray | None, psi1q: np.ndarray,
             phi: np.ndarray, threads: int | None = None, ckpt_stride: int = 1,
             want_env: bool = False, want_cuts: bool = False) -> dict:
    """Loss, gradient, HVP (V given) and their Riemannian forms.

    Returns a dict with loss, T, Omega, Omega_fwd (N_s), grad, hvp, grad_r,
    hvp_r (K,4,4), the Frobenius-cost forms loss_f, grad_f, hvp_f, grad_fr,
    hvp_fr, and optionally E, DE (N_s,K,4,4) and cuts (N_s,K+1).
    """
    lib = _load()
    G = _c128(G)
    K = G.shape[0]
    psi1q, phi = _c128(psi1q), _c128(phi)
    ns = psi1q.shape[0]
    if threads is None:
        threads = min(ns, os.cpu_count() or 1)
    Vc = None if V is None else _c128(V)
    out = dict(loss=np.zeros(1), T=np.zeros(ns, complex), Omega=np.zeros(ns, complex),
               Omega_fwd=np.zeros(ns, complex), grad=np.zeros((K, 4, 4), complex),
               hvp=np.zeros((K, 4, 4), complex), grad_r=np.zeros((K, 4, 4), complex),
               hvp_r=np.zeros((K, 4, 4), complex), loss_f=np.zeros(1),
               grad_f=np.zeros((K, 4, 4), complex), hvp_f=np.zeros((K, 4, 4), complex),
               grad_fr=np.zeros((K, 4, 4), complex), hvp_fr=np.zeros((K, 4, 4), complex))
    E = np.zeros((ns, K, 4, 4), complex) if want_env else None
    DE = np.zeros((ns, K, 4, 4), complex) if want_env else None
    cuts = np.zeros((ns, K + 1), complex) if want_cuts else None

    def f(a):
        return None if a is None else _ptr(a.view(np.float64))

    rc = lib.oracle_hvp(n, n_layers, ns, f(G), f(Vc), f(psi1q), f(phi), ckpt_stride, threads,
                        _ptr(out["loss"]), f(out["T"]), f(out["Omega"]), f(out["Omega_fwd"]),
                        f(E), f(DE), f(out["grad"]), f(out["hvp"]), f(out["grad_r"]),
                        f(out["hvp_r"]), f(cuts), _ptr(out["loss_f"]), f(out["grad_f"]), f(out["hvp_f"]),
                        f(out["grad_fr"]), f(out["hvp_fr"]))
    if rc != 0:
        raise RuntimeError(f"oracle_hvp failed: {rc}")
    out["loss"] = float(out["loss"][0])
    out["loss_f"] = float(out["loss_f"][0])
    if want_env:
        out["E"], out["DE"] = E, DE
    if want_cuts:
        out["cuts"] = cuts
    if V is None:
        for key in ("hvp", "hvp_r", "Omega", "Omega_fwd", "hvp_f", "hvp_fr"):
            out.pop(key)
    return out


def project(G: np.ndarray, X: np.ndarray) -> np.ndarray:
    """P_G(X) = X/2 - G X^dagger G/2 gate-wise (App. F, Eq. projec)."""
    lib = _load()
    G, X = _c128(G), _c128(X)
    out = np.zeros_like(G)
    lib.oracle_project(G.shape[0], _ptr(G.view(np.float64)), _ptr(X.view(np.float64)),
                       _ptr(out.view(np.float64)))
    return out
