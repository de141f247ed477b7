"""Allocation failures during context creation (failure injection on the
host): with HVP_DEVICE_ALLOC_CAP_MB set below what a context needs, hvp_init
and hvp_init_batch return HVP_ENOMEM with a message, release every byte they
had allocated (free device memory is unchanged), and a context created after
the cap is lifted works. (Free memory is compared only around the failed
creation: a successful one may load kernel code for the first time.)"""
import os

import numpy as np
import pytest

from common import rel
from oracle import oracle
from paper_2604_20384_gb300 import native
from paper_2604_20384_gb300.inputs import make_workload

pytestmark = pytest.mark.gpu


def _free_bytes(torch):
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info(0)[0]


@pytest.mark.parametrize("cap_mb,kw", [(1, {}), (40, {}), (40, {"recompute": True}), (200, {"tensor": True}),
                                       (2, {"unfused": True, "precision": "c128"})])
def test_context_allocation_failure_is_reported_and_leaks_nothing(cap_mb, kw):
    torch = pytest.importorskip("torch")
    w = make_workload(16, 6, 16, seed=4)
    native.load()
    torch.cuda.init()
    with native.Context(6, 3, make_workload(6, 3, 2).psi1q, make_workload(6, 3, 2).Uref):
        pass                                   # the CUDA context and the library's static state exist
    before = _free_bytes(torch)
    os.environ["HVP_DEVICE_ALLOC_CAP_MB"] = str(cap_mb)
    try:
        with pytest.raises(native.HVPError) as e:
            native.Context(16, 6, w.psi1q, w.Uref, **kw)
        assert e.value.code == native.HVP_ENOMEM
        assert "HVP_DEVICE_ALLOC_CAP_MB" in str(e.value)
    finally:
        del os.environ["HVP_DEVICE_ALLOC_CAP_MB"]
    assert _free_bytes(torch) == before
    phi = oracle.reference_states(16, 6, w.Uref, w.psi1q)
    o = oracle.evaluate(16, 6, w.G, w.V, w.psi1q, phi)
    with native.Context(16, 6, w.psi1q, w.Uref, **kw) as ctx:
        loss, grad, hvp = ctx.hvp(w.G, w.V)
    tol = 1e-11 if kw.get("precision") == "c128" else 1e-5
    assert rel(grad, o["grad"]) < tol and rel(hvp, o["hvp"]) < tol


def test_batch_allocation_failure_is_reported_and_leaks_nothing():
    torch = pytest.importorskip("torch")
    ws = [make_workload(n, L, ns, seed=60 + i) for i, (n, L, ns) in enumerate([(9, 4, 8), (14, 6, 5), (16, 5, 3)])]
    circuits = [(x.n, x.n_layers, x.psi1q, x.Uref) for x in ws]
    with native.BatchContext(circuits):
        pass
    before = _free_bytes(torch)
    os.environ["HVP_DEVICE_ALLOC_CAP_MB"] = "1"
    try:
        with pytest.raises(native.HVPError) as e:
            native.BatchContext(circuits)
        assert e.value.code == native.HVP_ENOMEM
    finally:
        del os.environ["HVP_DEVICE_ALLOC_CAP_MB"]
    assert _free_bytes(torch) == before
    with native.BatchContext(circuits) as b:
        loss, grads, hvps = b.hvp([x.G for x in ws], [x.V for x in ws])
    for i, x in enumerate(ws):
        phi = oracle.reference_states(x.n, x.n_layers, x.Uref, x.psi1q)
        o = oracle.evaluate(x.n, x.n_layers, x.G, x.V, x.psi1q, phi)
        assert rel(hvps[i], o["hvp"]) < 1e-5
