"""ctypes binding of libhvp (include/hvp.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module converts
numpy arrays and torch tensors to the pointers and sizes of the C ABI. There
is no CPU fallback: if libhvp.so is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhvp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "hvp.h")

HVP_OK, HVP_EINVAL, HVP_ENOMEM, HVP_ECUDA, HVP_ETIMEOUT, HVP_ENONFINITE = 0, -1, -2, -3, -4, -5
HVP_C64, HVP_C128 = 0, 1
HVP_RIEMANNIAN, HVP_PHI_GIVEN, HVP_UNFUSED, HVP_NO_GRAPH, HVP_AUTOTUNE, HVP_FROBENIUS = 1, 2, 4, 8, 16, 32
HVP_RECOMPUTE, HVP_MULTI_DIR, HVP_TENSOR, HVP_TRANSLATION = 64, 128, 256, 512
KINDS = {0: "prep", 1: "pass_fwd", 2: "pass_turnaround", 3: "pass_bwd", 4: "gate_init", 5: "gate_fwd",
         6: "gate_load_phi", 7: "gate_bwd", 8: "post", 9: "block_fwd", 10: "block_bwd"}
OUT = dict(T=1, Omega=2, grad_e=3, hvp_e=4, grad_r=5, hvp_r=6, loss=7, env=8)
ERRORS = {HVP_EINVAL: "EINVAL", HVP_ENOMEM: "ENOMEM", HVP_ECUDA: "ECUDA", HVP_ETIMEOUT: "ETIMEOUT",
          HVP_ENONFINITE: "ENONFINITE"}


class HVPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class HVPConfig(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("n_layers", ctypes.c_int), ("n_samples", ctypes.c_int),
                ("precision", ctypes.c_int), ("flags", ctypes.c_int), ("checkpoint_stride", ctypes.c_int),
                ("window", ctypes.c_int), ("threads", ctypes.c_int), ("variant", ctypes.c_int),
                ("device", ctypes.c_int), ("stream", ctypes.c_void_p)]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def load() -> ctypes.CDLL:
    """Loads libhvp.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    lib.hvp_batch_wait_test.argtypes = [vp, ctypes.c_int, ctypes.c_longlong]
    lib.hvp_batch_wait_test.restype = ctypes.c_int
    lib.hvp_cache_wait_test.argtypes = [vp, ctypes.c_int, ctypes.c_longlong]
    lib.hvp_cache_wait_test.restype = ctypes.c_int
    lib.hvp_num_gates.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.hvp_num_gates.restype = ctypes.c_int
    lib.hvp_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(HVPConfig), _dp, _dp]
    lib.hvp_init.restype = ctypes.c_int
    lib.hvp_loss_grad.argtypes = [vp, _dp, _dp, _dp]
    lib.hvp_loss_grad.restype = ctypes.c_int
    lib.hvp_hvp.argtypes = [vp, _dp, _dp, _dp, _dp, _dp]
    lib.hvp_hvp.restype = ctypes.c_int
    lib.hvp_hvp_dev.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.hvp_hvp_dev.restype = ctypes.c_int
    lib.hvp_hvp_multi.argtypes = [vp, _dp, ctypes.c_int, _dp, _dp, _dp, _dp]
    lib.hvp_hvp_multi.restype = ctypes.c_int
    lib.hvp_hvp_multi_dev.argtypes = [vp, vp, ctypes.c_int, vp, vp, vp, vp]
    lib.hvp_hvp_multi_dev.restype = ctypes.c_int
    lib.hvp_get.argtypes = [vp, ctypes.c_int, _dp]
    lib.hvp_get.restype = ctypes.c_int
    lib.hvp_plan_info.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    lib.hvp_plan_info.restype = ctypes.c_int
    lib.hvp_plan_brickwall.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_int)]
    lib.hvp_plan_brickwall.restype = ctypes.c_int
    lib.hvp_plan_blocks.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]
    lib.hvp_plan_blocks.restype = ctypes.c_int
    lib.hvp_profile.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                ctypes.POINTER(ctypes.c_int), _dp, _dp]
    lib.hvp_profile.restype = ctypes.c_int
    lib.hvp_hvp_noalloc.argtypes = [ctypes.c_int] * 3 + [vp] * 8
    lib.hvp_hvp_noalloc.restype = ctypes.c_int
    lib.hvp_init_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(HVPConfig),
                                   ctypes.POINTER(_dp), ctypes.POINTER(_dp)]
    lib.hvp_init_batch.restype = ctypes.c_int
    lib.hvp_free.argtypes = [vp]
    lib.hvp_free.restype = None
    lib.hvp_last_error.argtypes = [vp]
    lib.hvp_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def header_functions() -> list[str]:
    """Names of the functions include/hvp.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hvp_[a-z_0-9]+)\s*\(", text)))


def num_gates(n: int, n_layers: int) -> int:
    return load().hvp_num_gates(n, n_layers)


def plan_brickwall(n: int, n_layers: int, window: int = 12, low_bits: int = 4):
    """(number of passes, pass index of every gate) of the window-pass plan."""
    lib = load()
    K = lib.hvp_num_gates(n, n_layers)
    arr = (ctypes.c_int * max(K, 1))()
    P = lib.hvp_plan_brickwall(n, n_layers, window, low_bits, arr)
    if P < 0:
        raise HVPError(P, "hvp_plan_brickwall failed")
    return P, np.array(arr[:K], dtype=np.int64)


def plan_blocks(n: int, n_layers: int):
    """(block of every gate, first qubit of every block) of the fused-block
    plan of the HVP_TENSOR schedule."""
    lib = load()
    K = lib.hvp_num_gates(n, n_layers)
    bog = (ctypes.c_int * max(K, 1))()
    bq = (ctypes.c_int * max(K, 1))()
    nb = lib.hvp_plan_blocks(n, n_layers, bog, bq)
    if nb < 0:
        raise HVPError(nb, "hvp_plan_blocks failed")
    return np.array(bog[:K], dtype=np.int64), np.array(bq[:nb], dtype=np.int64)


def hvp_noalloc(n: int, n_layers: int, n_samples: int, psi1q_ptr: int, phi_ptr: int, G_ptr: int,
                V_ptr: int | None, loss_ptr: int | None, grad_ptr: int | None, hvp_ptr: int | None,
                stream: int | None = None) -> None:
    """Loss, gradient and HVP on device pointers without any device allocation
    (hvp_hvp_noalloc): for callers whose device memory is owned by someone
    else, e.g. a framework allocator holding the whole device pool, or that
    run under a strict device-memory budget. Work space is a fixed 16 MiB
    static device array shared by all calls on a device, so calls must not
    overlap on the GPU. The call is synchronous (it waits for its stream)."""
    lib = load()
    rc = lib.hvp_hvp_noalloc(n, n_layers, n_samples, psi1q_ptr, phi_ptr, G_ptr, V_ptr, loss_ptr, grad_ptr,
                             hvp_ptr, stream)
    if rc != HVP_OK:
        raise HVPError(rc, lib.hvp_last_error(None).decode())


def _f64(a, shape_last=None):
    a = np.ascontiguousarray(a)
    if np.iscomplexobj(a):
        a = np.ascontiguousarray(a, dtype=np.complex128).view(np.float64)
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(_dp)


class Context:
    """One loss/gradient/HVP problem on one GPU (hvp_init ... hvp_free).

    psi1q: (N_s, n, 2) complex; ref: U_ref gates (K, 4, 4) complex, or the
    reference states (N_s, 2^n) with phi_given=True.
    """

    def __init__(self, n: int, n_layers: int, psi1q, ref, *, precision: str = "c64",
                 riemannian: bool = False, phi_given: bool = False, unfused: bool = False,
                 graphs: bool = True, checkpoint_stride: int = 0, window: int = 0, threads: int = 0,
                 variant: int = 0, autotune: bool = False, frobenius: bool = False, recompute: bool = False,
                 multi_dir: bool = False, tensor: bool = False, translation: bool = False, device: int = 0,
                 stream: int | None = None):
        self._lib = load()
        psi1q = np.asarray(psi1q)
        self.n, self.n_layers, self.n_samples = n, n_layers, int(psi1q.shape[0])
        self.K = self._lib.hvp_num_gates(n, n_layers)
        # blocks per call the caller passes and receives: layers (HVP_TRANSLATION) or gates
        self.blocks = n_layers if translation else self.K
        flags = ((HVP_RIEMANNIAN if riemannian else 0) | (HVP_PHI_GIVEN if phi_given else 0)
                 | (HVP_UNFUSED if unfused else 0) | (0 if graphs else HVP_NO_GRAPH)
                 | (HVP_AUTOTUNE if autotune else 0) | (HVP_FROBENIUS if frobenius else 0)
                 | (HVP_RECOMPUTE if recompute else 0) | (HVP_MULTI_DIR if multi_dir else 0)
                 | (HVP_TENSOR if tensor else 0) | (HVP_TRANSLATION if translation else 0))
        cfg = HVPConfig(n, n_layers, self.n_samples, HVP_C128 if precision == "c128" else HVP_C64, flags,
                        checkpoint_stride, window, threads, variant, device, stream)
        self._psi = _f64(psi1q)
        self._ref = _f64(ref)
        h = ctypes.c_void_p()
        rc = self._lib.hvp_init(ctypes.byref(h), ctypes.byref(cfg), _ptr(self._psi), _ptr(self._ref))
        if rc != HVP_OK:
            raise HVPError(rc, self._lib.hvp_last_error(None).decode())
        self._h = h
        self.riemannian = riemannian
        self.frobenius = frobenius

    def _check(self, rc):
        if rc != HVP_OK:
            raise HVPError(rc, self._lib.hvp_last_error(self._h).decode())

    def loss_grad(self, G):
        G = _f64(G)
        loss = np.zeros(1)
        grad = np.zeros(32 * self.blocks)
        self._check(self._lib.hvp_loss_grad(self._h, _ptr(G), _ptr(loss), _ptr(grad)))
        return float(loss[0]), grad.view(np.complex128).reshape(self.blocks, 4, 4)

    def hvp(self, G, V):
        G, V = _f64(G), _f64(V)
        loss = np.zeros(1)
        grad = np.zeros(32 * self.blocks)
        hv = np.zeros(32 * self.blocks)
        self._check(self._lib.hvp_hvp(self._h, _ptr(G), _ptr(V), _ptr(loss), _ptr(grad), _ptr(hv)))
        return (float(loss[0]), grad.view(np.complex128).reshape(self.blocks, 4, 4),
                hv.view(np.complex128).reshape(self.blocks, 4, 4))

    def hvp_multi(self, G, Vs):
        """(loss, grad, [HVP along each direction]) at the same gates
        (hvp_hvp_multi); Vs: (n_dir, K, 4, 4)."""
        G = _f64(G)
        Vs = np.asarray(Vs)
        nd = int(Vs.shape[0])
        V = _f64(Vs)
        loss = np.zeros(1)
        grad = np.zeros(32 * self.blocks)
        hv = np.zeros(32 * self.blocks * nd)
        self._check(self._lib.hvp_hvp_multi(self._h, _ptr(G), nd, _ptr(V), _ptr(loss), _ptr(grad), _ptr(hv)))
        return (float(loss[0]), grad.view(np.complex128).reshape(self.blocks, 4, 4),
                hv.view(np.complex128).reshape(nd, self.blocks, 4, 4))

    def hvp_multi_dev(self, G_ptr: int, n_dir: int, V_ptr: int, loss_ptr: int | None, grad_ptr: int | None,
                      hvp_ptr: int | None):
        """Stream-ordered hvp_hvp_multi_dev on device pointers."""
        self._check(self._lib.hvp_hvp_multi_dev(self._h, G_ptr, n_dir, V_ptr, loss_ptr, grad_ptr, hvp_ptr))

    def hvp_dev(self, G_ptr: int, V_ptr: int | None, loss_ptr: int | None, grad_ptr: int | None,
                hvp_ptr: int | None):
        """Stream-ordered call on device pointers (torch tensors' data_ptr())."""
        self._check(self._lib.hvp_hvp_dev(self._h, G_ptr, V_ptr, loss_ptr, grad_ptr, hvp_ptr))

    def profile(self, G_ptr: int, V_ptr: int | None, max_launches: int = 4096):
        """Per-launch device times (ms), kinds, algorithmic flops and bytes of one
        evaluation, each launch bracketed by CUDA events on the context's stream."""
        ms = (ctypes.c_float * max_launches)()
        kind = (ctypes.c_int * max_launches)()
        fl = np.zeros(max_launches)
        by = np.zeros(max_launches)
        n = self._lib.hvp_profile(self._h, G_ptr, V_ptr, max_launches, ms, kind, _ptr(fl), _ptr(by))
        if n < 0:
            self._check(n)
        n = min(n, max_launches)
        return dict(ms=np.array(ms[:n]), kind=np.array(kind[:n]), flops=fl[:n], bytes=by[:n])

    def get(self, what: str):
        sizes = dict(T=2 * self.n_samples, Omega=2 * self.n_samples, loss=1,
                     env=64 * self.K * self.n_samples)
        m = sizes.get(what, 32 * self.blocks)
        out = np.zeros(m)
        self._check(self._lib.hvp_get(self._h, OUT[what], _ptr(out)))
        if what == "loss":
            return float(out[0])
        c = out.view(np.complex128)
        if what in ("T", "Omega"):
            return c
        if what == "env":
            e = c.reshape(self.n_samples, self.K, 2, 4, 4)
            return e[:, :, 0], e[:, :, 1]
        return c.reshape(self.blocks, 4, 4)

    def plan_info(self) -> dict:
        info = (ctypes.c_longlong * 10)()
        self._check(self._lib.hvp_plan_info(self._h, info))
        keys = ["K", "passes", "window", "checkpoint_stride", "launches_per_hvp", "device_mib",
                "tiles_per_cta", "ctas_per_sample", "threads", "variant"]
        return dict(zip(keys, list(info)))

    def cache_wait_test(self, extra_bytes: int, spin_limit: int = 0):
        """hvp_cache_wait_test: extra_bytes=16 makes the forward-cache copy waits
        of the next calls run out after spin_limit polls."""
        self._check(self._lib.hvp_cache_wait_test(self._h, extra_bytes, spin_limit))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hvp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class BatchContext(Context):
    """Many independent circuits evaluated together (hvp_init_batch).

    circuits: list of (n, n_layers, psi1q, ref) tuples. Gates, directions and
    derivatives are lists of per-circuit (K_c, 4, 4) arrays; the loss is one
    value per circuit.
    """

    def __init__(self, circuits, *, riemannian: bool = False, phi_given: bool = False, graphs: bool = True,
                 frobenius: bool = False, window: int = 0, autotune: bool = False, device: int = 0,
                 stream: int | None = None):
        self._lib = load()
        nc = len(circuits)
        flags = ((HVP_RIEMANNIAN if riemannian else 0) | (HVP_PHI_GIVEN if phi_given else 0)
                 | (0 if graphs else HVP_NO_GRAPH) | (HVP_FROBENIUS if frobenius else 0)
                 | (HVP_AUTOTUNE if autotune else 0))
        cfgs = (HVPConfig * nc)()
        self._keep = []
        psis = (_dp * nc)()
        refs = (_dp * nc)()
        self.Ks, self.ns = [], []
        for c, (n, L, psi1q, ref) in enumerate(circuits):
            psi1q = np.asarray(psi1q)
            cfgs[c] = HVPConfig(n, L, int(psi1q.shape[0]), HVP_C64, flags, 0, window, 0, 0, device, stream)
            a, r = _f64(psi1q), _f64(ref)
            self._keep += [a, r]
            psis[c] = _ptr(a)
            refs[c] = _ptr(r)
            self.Ks.append(self._lib.hvp_num_gates(n, L))
            self.ns.append(int(psi1q.shape[0]))
        h = ctypes.c_void_p()
        rc = self._lib.hvp_init_batch(ctypes.byref(h), nc, cfgs, psis, refs)
        if rc != HVP_OK:
            raise HVPError(rc, self._lib.hvp_last_error(None).decode())
        self._h = h
        self.riemannian = riemannian
        self.frobenius = frobenius
        self.K = sum(self.Ks)
        self.blocks = self.K
        self.n_samples = sum(self.ns)
        self.n_circuits = nc

    def wait_test(self, dep_bias: int, spin_limit: int = 20000000):
        """hvp_batch_wait_test: dep_bias=1 makes the next calls' chain waits run out."""
        self._check(self._lib.hvp_batch_wait_test(self._h, dep_bias, spin_limit))

    def _split(self, flat):
        out, o = [], 0
        for k in self.Ks:
            out.append(flat[o:o + k])
            o += k
        return out

    def loss_grad(self, Gs):
        G = _f64(np.concatenate([np.asarray(g, dtype=np.complex128) for g in Gs]))
        loss = np.zeros(self.n_circuits)
        grad = np.zeros(32 * self.K)
        self._check(self._lib.hvp_loss_grad(self._h, _ptr(G), _ptr(loss), _ptr(grad)))
        return loss, self._split(grad.view(np.complex128).reshape(self.K, 4, 4))

    def hvp(self, Gs, Vs):
        G = _f64(np.concatenate([np.asarray(g, dtype=np.complex128) for g in Gs]))
        V = _f64(np.concatenate([np.asarray(v, dtype=np.complex128) for v in Vs]))
        loss = np.zeros(self.n_circuits)
        grad = np.zeros(32 * self.K)
        hv = np.zeros(32 * self.K)
        self._check(self._lib.hvp_hvp(self._h, _ptr(G), _ptr(V), _ptr(loss), _ptr(grad), _ptr(hv)))
        return (loss, self._split(grad.view(np.complex128).reshape(self.K, 4, 4)),
                self._split(hv.view(np.complex128).reshape(self.K, 4, 4)))

    def get(self, what: str):
        if what == "loss":
            out = np.zeros(self.n_circuits)
            self._check(self._lib.hvp_get(self._h, OUT[what], _ptr(out)))
            return out
        if what in ("T", "Omega"):
            out = np.zeros(2 * self.n_samples)
            self._check(self._lib.hvp_get(self._h, OUT[what], _ptr(out)))
            c = out.view(np.complex128)
            res, o = [], 0
            for ns in self.ns:
                res.append(c[o:o + ns])
                o += ns
            return res
        out = np.zeros(32 * self.K)
        self._check(self._lib.hvp_get(self._h, OUT[what], _ptr(out)))
        return self._split(out.view(np.complex128).reshape(self.K, 4, 4))

    def plan_info(self) -> dict:
        info = (ctypes.c_longlong * 10)()
        self._check(self._lib.hvp_plan_info(self._h, info))
        keys = ["K", "items", "window", "checkpoint_stride", "launches_per_hvp", "device_mib", "ctas",
                "circuits", "threads", "variant"]
        return dict(zip(keys, list(info)))
