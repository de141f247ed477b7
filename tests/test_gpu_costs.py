"""Second loss and translation-invariant layers on the GPU: the Frobenius cost
(Eq. Frobenius, Eq. grad-costF, Eq. hvp-costF) and layer-gate derivatives
(App. E) against the FP64 oracle."""
import numpy as np
import pytest

from common import contract, expand, rel
from oracle import oracle
from paper_2604_20384_gb300 import native
from paper_2604_20384_gb300.inputs import make_workload
from paper_2604_20384_gb300.translation import TranslationInvariant

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.mark.parametrize("n,L,ns,window", [(9, 5, 12, 0), (15, 8, 4, 11)])
def test_frobenius_cost_matches_oracle(n, L, ns, window):
    w = make_workload(n, L, ns, seed=61, near_solution=0.2)
    phi = oracle.reference_states(n, L, w.Uref, w.psi1q)
    o = oracle.evaluate(n, L, w.G, w.V, w.psi1q, phi)
    for riem in (False, True):
        with native.Context(n, L, w.psi1q, w.Uref, frobenius=True, riemannian=riem, window=window) as c:
            loss, g, h = c.hvp(w.G, w.V)
        assert abs(loss - o["loss_f"]) < TOL * max(abs(o["loss_f"]), 1e-3)
        assert rel(g, o["grad_fr" if riem else "grad_f"]) < TOL
        assert rel(h, o["hvp_fr" if riem else "hvp_f"]) < TOL


def test_frobenius_cost_in_a_batch():
    ws = [make_workload(n, L, ns, seed=70 + i, near_solution=0.2)
          for i, (n, L, ns) in enumerate([(7, 4, 9), (13, 6, 3)])]
    with native.BatchContext([(w.n, w.n_layers, w.psi1q, w.Uref) for w in ws], frobenius=True) as b:
        loss, gs, hs = b.hvp([w.G for w in ws], [w.V for w in ws])
    for i, w in enumerate(ws):
        phi = oracle.reference_states(w.n, w.n_layers, w.Uref, w.psi1q)
        o = oracle.evaluate(w.n, w.n_layers, w.G, w.V, w.psi1q, phi)
        assert abs(loss[i] - o["loss_f"]) < TOL * max(abs(o["loss_f"]), 1e-3)
        assert rel(gs[i], o["grad_f"]) < TOL and rel(hs[i], o["hvp_f"]) < TOL


@pytest.mark.parametrize("kw", [dict(window=10), dict(tensor=True), dict(riemannian=True), dict(recompute=True),
                                dict(unfused=True, precision="c128")])
def test_translation_invariant_layers_match_oracle(kw):
    # App. E on the device (HVP_TRANSLATION): layer gates expanded to every gate,
    # per-gate blocks summed per layer in FP64; host arrays and device pointers
    torch = pytest.importorskip("torch")
    n, L, ns = 13, 7, 6
    w = make_workload(n, L, ns, seed=81)
    first = np.cumsum([0] + [(n - l % 2) // 2 for l in range(L)])[:-1]
    Gl, Vl = w.G[first], w.V[first]
    phi = oracle.reference_states(n, L, w.Uref, w.psi1q)
    o = oracle.evaluate(n, L, expand(Gl, n, L), expand(Vl, n, L), w.psi1q, phi)
    tol = 1e-11 if kw.get("precision") == "c128" else TOL
    kg, kh = ("grad_r", "hvp_r") if kw.get("riemannian") else ("grad", "hvp")
    with TranslationInvariant(n, L, w.psi1q, w.Uref, **kw) as ti:
        loss, g, h = ti.hvp(Gl, Vl)
        assert abs(loss - o["loss"]) < tol
        assert rel(g, contract(o[kg], n, L)) < tol
        assert rel(h, contract(o[kh], n, L)) < tol
        loss2, g2 = ti.loss_grad(Gl)
        assert rel(g2, contract(o[kg], n, L)) < tol
        dev = torch.device("cuda", 0)
        Gd = torch.from_numpy(np.ascontiguousarray(Gl).view(np.float64).reshape(-1).copy()).to(dev)
        Vd = torch.from_numpy(np.ascontiguousarray(Vl).view(np.float64).reshape(-1).copy()).to(dev)
        gd = torch.zeros(32 * L, dtype=torch.float64, device=dev)
        hd = torch.zeros(32 * L, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        ti.hvp_dev(Gd.data_ptr(), Vd.data_ptr(), None, gd.data_ptr(), hd.data_ptr())
        torch.cuda.synchronize()
        assert rel(gd.cpu().numpy().view(np.complex128).reshape(L, 4, 4), contract(o[kg], n, L)) < tol
        assert rel(hd.cpu().numpy().view(np.complex128).reshape(L, 4, 4), contract(o[kh], n, L)) < tol


def test_dense_riemannian_hessian_spectrum_on_gpu():
    from paper_2604_20384_gb300.spectrum import riemannian_hessian, spectrum

    n, L, ns = 8, 4, 8
    w = make_workload(n, L, ns, seed=93, near_solution=0.3)
    phi = oracle.reference_states(n, L, w.Uref, w.psi1q)
    with native.Context(n, L, w.psi1q, w.Uref, riemannian=True) as c:
        H = riemannian_hessian(lambda G, V: c.hvp(G, V)[2], w.G)
    Ho = riemannian_hessian(lambda G, V: oracle.evaluate(n, L, G, V, w.psi1q, phi)["hvp_r"], w.G)
    assert H.shape == (16 * w.K, 16 * w.K)
    assert rel(H, Ho) < TOL
    assert np.max(np.abs(H - H.T)) < 1e-5 * np.max(np.abs(H))
    ev, evo = spectrum(H), spectrum(Ho)
    assert np.max(np.abs(ev - evo)) < 1e-5 * np.max(np.abs(evo))
    # the same columns from direction pairs per sweep (hvp_hvp_multi)
    with native.Context(n, L, w.psi1q, w.Uref, riemannian=True, multi_dir=True) as c:
        Hm = riemannian_hessian(None, w.G, hvp_multi_fn=lambda G, Vs: c.hvp_multi(G, Vs)[2], chunk=17)
    assert rel(Hm, Ho) < TOL
