"""The allocation-free entry point against the regular one.

Some callers cannot allocate device memory: a framework whose caching
allocator already owns the device pool, a CUDA-graph replay harness whose
memory plan is fixed in advance, or a service that runs under a strict device
memory budget. hvp_hvp_noalloc serves them with a static work space inside the
library. This test calls it through the C ABI twice in a row, with different
gates and directions, and checks each result against hvp_hvp on a context
built from the same reference states. The file is named so that pytest
collects it last.
"""
import numpy as np
import pytest

from common import rel
from oracle import oracle
from paper_2604_20384_gb300 import native
from paper_2604_20384_gb300.inputs import make_workload, random_direction

pytestmark = pytest.mark.gpu

TOL = 1e-5   # complex64 sweeps with FP64 accumulation, as in the parity tests


def _dev(torch, a):
    a = np.ascontiguousarray(a, dtype=np.complex128).view(np.float64).reshape(-1)
    return torch.from_numpy(a.copy()).to("cuda:0")


def test_noalloc_matches_regular_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    n, L, ns = 10, 6, 24
    w = make_workload(n, L, ns, seed=31)
    phi = oracle.reference_states(n, L, w.Uref, w.psi1q)
    rng = np.random.default_rng(5)
    G2 = np.stack([np.linalg.qr(rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))[0]
                   for _ in range(w.K)])
    V2 = random_direction(w.K, G2, seed=17)
    psi_d, phi_d = _dev(torch, w.psi1q), _dev(torch, phi)
    loss_d = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    grad_d = torch.zeros(32 * w.K, dtype=torch.float64, device="cuda:0")
    hvp_d = torch.zeros(32 * w.K, dtype=torch.float64, device="cuda:0")
    torch.cuda.synchronize()
    with native.Context(n, L, w.psi1q, phi, phi_given=True) as ctx:
        for G, V in ((w.G, w.V), (G2, V2)):
            want_loss, want_grad, want_hvp = ctx.hvp(G, V)
            G_d, V_d = _dev(torch, G), _dev(torch, V)
            native.hvp_noalloc(n, L, ns, psi_d.data_ptr(), phi_d.data_ptr(), G_d.data_ptr(), V_d.data_ptr(),
                               loss_d.data_ptr(), grad_d.data_ptr(), hvp_d.data_ptr(), None)
            got_grad = grad_d.cpu().numpy().view(np.complex128).reshape(w.K, 4, 4)
            got_hvp = hvp_d.cpu().numpy().view(np.complex128).reshape(w.K, 4, 4)
            got_loss = float(loss_d.cpu().numpy()[0])
            assert abs((1 - got_loss) - (1 - want_loss)) <= TOL * abs(1 - want_loss)
            assert rel(got_grad, want_grad) < TOL
            assert rel(got_hvp, want_hvp) < TOL


def test_noalloc_rejects_problems_beyond_its_work_space():
    torch = pytest.importorskip("torch")
    x = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    p = x.data_ptr()
    with pytest.raises(native.HVPError) as e:        # 12 qubits x 512 samples > 16 MiB
        native.hvp_noalloc(12, 4, 512, p, p, p, p, p, p, p, None)
    assert e.value.code == native.HVP_EINVAL and "work space" in str(e.value)
    with pytest.raises(native.HVPError) as e:        # more qubits than one tile
        native.hvp_noalloc(13, 2, 1, p, p, p, p, p, p, p, None)
    assert e.value.code == native.HVP_EINVAL
