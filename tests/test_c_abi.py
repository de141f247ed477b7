"""The C ABI used from plain C (tests/c_abi_demo.c): compiled with gcc against
include/hvp.h and linked to libhvp.so, with no Python or PyTorch in the
process. The CPU test runs the calls that need no GPU; the GPU test runs a
whole loss/gradient/HVP evaluation and compares it with the FP64 oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from common import rel
from oracle import oracle
from paper_2604_20384_gb300 import native
from paper_2604_20384_gb300.inputs import make_workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIBDIR = os.path.join(ROOT, "paper_2604_20384_gb300")


@pytest.fixture(scope="module")
def demo(tmp_path_factory):
    native.load()                                   # libhvp.so must exist (no fallback)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path_factory.mktemp("cabi") / "c_abi_demo")
    subprocess.run([cc, "-O1", "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_demo.c"), "-L", LIBDIR, "-lhvp",
                    "-Wl,-rpath," + LIBDIR, "-o", exe], check=True)
    return exe


def test_c_caller_without_gpu(demo):
    r = subprocess.run([demo, "cpu"], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "num_gates 20 16 = 152" in r.stdout
    assert "rc = -1 ctx_null = 1" in r.stdout


@pytest.mark.gpu
def test_c_caller_matches_oracle(demo, tmp_path):
    w = make_workload(9, 5, 6, seed=77)
    src = tmp_path / "in.bin"
    dst = tmp_path / "out.bin"
    np.concatenate([w.psi1q.view(np.float64).ravel(), w.Uref.view(np.float64).ravel(),
                    w.G.view(np.float64).ravel(), w.V.view(np.float64).ravel()]).astype("<f8").tofile(src)
    r = subprocess.run([demo, "gpu", "9", "5", "6", str(src), str(dst)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    out = np.fromfile(dst, dtype="<f8")
    K = w.K
    loss = out[0]
    grad = out[1:1 + 32 * K].view(np.complex128).reshape(K, 4, 4)
    hvp = out[1 + 32 * K:].view(np.complex128).reshape(K, 4, 4)
    phi = oracle.reference_states(9, 5, w.Uref, w.psi1q)
    o = oracle.evaluate(9, 5, w.G, w.V, w.psi1q, phi)
    assert abs((1 - loss) - (1 - o["loss"])) <= 1e-5 * (1 - o["loss"]) + 1e-13
    assert rel(grad, o["grad"]) < 1e-5
    assert rel(hvp, o["hvp"]) < 1e-5
