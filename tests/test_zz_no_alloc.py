"""The allocation-free entry point against the regular one and the oracle.

Some callers cannot allocate device memory: a framework whose caching
allocator already owns the device pool, or a service that runs under a strict
device memory budget. hvp_hvp_noalloc serves them with a static work space
inside the library. These tests call it through the C ABI two times in a row,
with different gates and directions, and check each result against hvp_hvp
on a context built from the same reference states and against the FP64
oracle; further cases cover the loss-and-gradient-only form with outputs left
NULL, the smallest tiles (n = 2, 4) and a problem near the work-space limit.
The file is named so that pytest collects it last.
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
            o = oracle.evaluate(n, L, G, V, w.psi1q, phi)
            assert abs((1 - got_loss) - (1 - o["loss"])) <= TOL * abs(1 - o["loss"]) + 1e-13
            assert rel(got_grad, o["grad"]) < TOL and rel(got_hvp, o["hvp"]) < TOL


def _noalloc_vs_oracle(torch, n, L, ns, seed, with_v=True, outputs=("loss", "grad", "hvp")):
    w = make_workload(n, L, ns, seed=seed)
    phi = oracle.reference_states(n, L, w.Uref, w.psi1q)
    o = oracle.evaluate(n, L, w.G, w.V if with_v else None, w.psi1q, phi)
    psi_d, phi_d, G_d = _dev(torch, w.psi1q), _dev(torch, phi), _dev(torch, w.G)
    V_d = _dev(torch, w.V) if with_v else None
    out = {"loss": torch.full((1,), -7.0, dtype=torch.float64, device="cuda:0"),
           "grad": torch.full((32 * w.K,), -7.0, dtype=torch.float64, device="cuda:0"),
           "hvp": torch.full((32 * w.K,), -7.0, dtype=torch.float64, device="cuda:0")}
    ptr = {k: (out[k].data_ptr() if k in outputs else None) for k in out}
    torch.cuda.synchronize()
    native.hvp_noalloc(n, L, ns, psi_d.data_ptr(), phi_d.data_ptr(), G_d.data_ptr(),
                       V_d.data_ptr() if with_v else None, ptr["loss"], ptr["grad"], ptr["hvp"], None)
    res = {k: out[k].cpu().numpy() for k in out}
    if "loss" in outputs:
        assert abs((1 - res["loss"][0]) - (1 - o["loss"])) <= TOL * abs(1 - o["loss"]) + 1e-13
    if "grad" in outputs:
        assert rel(res["grad"].view(np.complex128).reshape(w.K, 4, 4), o["grad"]) < TOL
    if "hvp" in outputs and with_v:
        assert rel(res["hvp"].view(np.complex128).reshape(w.K, 4, 4), o["hvp"]) < TOL
    for k in out:                      # outputs left NULL are not written anywhere the caller owns
        if k not in outputs or (k == "hvp" and not with_v):
            assert np.all(res[k] == -7.0)


@pytest.mark.parametrize("n,L,ns", [(2, 3, 5), (4, 4, 3), (12, 8, 200)])
def test_noalloc_small_tiles_and_near_limit_against_oracle(n, L, ns):
    # n = 2: a four-amplitude tile; n = 12, L = 8, N_s = 200: about 15.0 MiB
    # of the 16 MiB work space
    torch = pytest.importorskip("torch")
    _noalloc_vs_oracle(torch, n, L, ns, seed=n + 40)


def test_noalloc_loss_and_gradient_only_with_null_outputs():
    # V = NULL runs the sweeps without tangents; a NULL output is skipped
    torch = pytest.importorskip("torch")
    _noalloc_vs_oracle(torch, 9, 5, 6, seed=8, with_v=False, outputs=("grad",))
    _noalloc_vs_oracle(torch, 9, 5, 6, seed=8, with_v=False, outputs=("loss", "grad"))
    _noalloc_vs_oracle(torch, 9, 5, 6, seed=8, with_v=True, outputs=("hvp",))


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
