"""Host-side checks of the C ABI (no GPU): the library loads, exports every
function that include/hvp.h declares, validates arguments before touching
CUDA, and its window-pass planner produces valid plans."""
import ctypes

import numpy as np
import pytest

from paper_2604_20384_gb300 import native
from paper_2604_20384_gb300.inputs import num_gates


def test_library_exports_every_declared_function():
    lib = native.load()
    names = native.header_functions()
    assert {"hvp_init", "hvp_loss_grad", "hvp_hvp", "hvp_free"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("n,L", [(2, 1), (3, 2), (6, 3), (12, 8), (20, 16), (26, 24), (9, 7)])
def test_num_gates_matches_independent_count(n, L):
    assert native.num_gates(n, L) == num_gates(n, L)


def test_num_gates_rejects_bad_shapes():
    assert native.num_gates(1, 3) == -1
    assert native.num_gates(5, 0) == -1


def _deps(n, L):
    fq = []
    for layer in range(L):
        i = layer % 2
        while i + 1 <= n - 1:
            fq.append(i)
            i += 2
    last = [-1] * n
    deps = []
    for k, i in enumerate(fq):
        deps.append([p for p in (last[i], last[i + 1]) if p >= 0])
        last[i] = last[i + 1] = k
    return deps


@pytest.mark.parametrize("n,L,w", [(20, 16, 12), (20, 16, 11), (20, 16, 10), (26, 24, 12), (13, 20, 12),
                                   (16, 20, 12), (14, 8, 11), (12, 8, 12), (6, 3, 12), (30, 5, 12),
                                   (17, 33, 8)])
def test_plan_respects_circuit_order(n, L, w):
    P, pog = native.plan_brickwall(n, L, w, 4)
    K = num_gates(n, L)
    assert len(pog) == K and P >= 1
    assert pog.min() == 0 and pog.max() <= P - 1
    for g, ds in enumerate(_deps(n, L)):
        for d in ds:
            assert pog[d] <= pog[g]
    if n <= w:
        assert P == 1


def test_plan_pass_counts_of_benchmark_shapes():
    # The headline brickwall (n = 20, L = 16, K = 152) fits in 4 window passes
    # of 12 qubits (the planner's search over window positions; a fixed
    # zig-zag of evenly spaced windows needs 5) and 6 passes of 11 qubits;
    # no pass exceeds the 64-gate shared-memory budget.
    for w, P_expected in ((12, 4), (11, 6)):
        P, pog = native.plan_brickwall(20, 16, w, 4)
        assert P == P_expected
        assert np.bincount(pog).max() <= 64
    assert native.plan_brickwall(12, 8, 12, 4)[0] == 1


@pytest.mark.parametrize("n,L", [(20, 16), (5, 7), (6, 3), (12, 8), (26, 24), (13, 11), (30, 5), (9, 1)])
def test_block_plan_covers_gates_in_circuit_order(n, L):
    # Fused-block plan of the tensor-core schedule: every gate in exactly one
    # block, both of its qubits inside the block's five qubits [a, a + 5), and
    # no gate in an earlier block than a gate it depends on (within a block the
    # gates run in circuit order, which respects every dependency).
    bog, bq = native.plan_blocks(n, L)
    K = num_gates(n, L)
    fq = [i for layer in range(1, L + 1) for i in range((layer - 1) % 2, n - 1, 2)]
    assert len(bog) == K and bog.min() == 0 and bog.max() == len(bq) - 1
    assert np.all((bq >= 0) & (bq + 5 <= n))
    for k in range(K):
        a = bq[bog[k]]
        assert a <= fq[k] and fq[k] + 1 <= a + 4
    for g, ds in enumerate(_deps(n, L)):
        for d in ds:
            assert bog[d] <= bog[g]


def test_block_plan_of_benchmark_shape():
    # n = 20, L = 16: 152 gates in 26 blocks of five qubits (about six gates
    # per dense 32 x 32 block); fewer than five qubits cannot form a block.
    bog, bq = native.plan_blocks(20, 16)
    assert len(bq) == 26
    assert native.load().hvp_plan_blocks(4, 3, None, None) == -1


def test_plan_rejects_bad_arguments():
    lib = native.load()
    assert lib.hvp_plan_brickwall(1, 3, 12, 4, None) < 0
    assert lib.hvp_plan_brickwall(20, 3, 40, 4, None) < 0
    assert lib.hvp_plan_brickwall(20, 3, 12, 12, None) < 0


def test_init_validates_arguments_before_cuda():
    lib = native.load()
    psi = np.zeros(4 * 6 * 2)
    ref = np.zeros(32 * 8)
    h = ctypes.c_void_p()
    cfg = native.HVPConfig(1, 3, 2, 0, 0, 0, 0, 0, 0, 0, None)          # n < 2
    assert lib.hvp_init(ctypes.byref(h), ctypes.byref(cfg), native._ptr(psi), native._ptr(ref)) == native.HVP_EINVAL
    assert not h.value
    assert b"n = 1" in lib.hvp_last_error(None)
    cfg = native.HVPConfig(6, 3, 2, 7, 0, 0, 0, 0, 0, 0, None)          # bad precision
    assert lib.hvp_init(ctypes.byref(h), ctypes.byref(cfg), native._ptr(psi), native._ptr(ref)) == native.HVP_EINVAL
    cfg = native.HVPConfig(6, 3, 2, 0, 1 << 10, 0, 0, 0, 0, 0, None)    # unknown flag
    assert lib.hvp_init(ctypes.byref(h), ctypes.byref(cfg), native._ptr(psi), native._ptr(ref)) == native.HVP_EINVAL
    cfg = native.HVPConfig(6, 3, 2, 0, 0, 0, 0, 192, 0, 0, None)        # unsupported thread count
    assert lib.hvp_init(ctypes.byref(h), ctypes.byref(cfg), native._ptr(psi), native._ptr(ref)) == native.HVP_EINVAL
    cfg = native.HVPConfig(6, 3, 2, 0, 0, 0, 0, 128, 2, 0, None)        # 128 threads: scalar arithmetic only
    assert lib.hvp_init(ctypes.byref(h), ctypes.byref(cfg), native._ptr(psi), native._ptr(ref)) == native.HVP_EINVAL
    assert b"128 threads" in lib.hvp_last_error(None)
    cfg = native.HVPConfig(6, 3, 65536, 0, 0, 0, 0, 0, 0, 0, None)      # one grid row per sample: at most 65535
    assert lib.hvp_init(ctypes.byref(h), ctypes.byref(cfg), native._ptr(psi), native._ptr(ref)) == native.HVP_EINVAL
    assert b"n_samples = 65536" in lib.hvp_last_error(None)
    cfg = native.HVPConfig(6, 3, 2, 0, 0, 0, 0, 0, 0, 0, None)
    assert lib.hvp_init(ctypes.byref(h), ctypes.byref(cfg), None, native._ptr(ref)) == native.HVP_EINVAL
    bad = psi.copy()
    bad[3] = np.nan
    assert lib.hvp_init(ctypes.byref(h), ctypes.byref(cfg), native._ptr(bad), native._ptr(ref)) == native.HVP_ENONFINITE
    lib.hvp_free(None)   # NULL is ignored
    assert lib.hvp_loss_grad(None, None, None, None) == native.HVP_EINVAL
