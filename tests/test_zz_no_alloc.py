"""Allocation-free Gram entry point (pou_gram_noalloc).

Some callers of this library cannot call cudaMalloc: a host that hands the
library a fixed device-memory budget, or a loop that must not allocate (and so
must not synchronise the device) once it has started.  pou_gram_noalloc gives
them the Gram matrix S = dV * A^T A without a caller workspace; its partial
sums live in the library's fixed static device buffer, which every call
shares and which keeps the previous call's contents.

Each case checks the result against dV * A^T A formed in FP64 by NumPy from
the same block, on two calls in a row, within the tolerances of the Gram
tests.  The 512-orbital FP32 case uses more splits than fit the buffer, so the
capped split count is exercised; the fresh-process case makes the
allocation-free call the first library call of a process, so the one-time
address lookup runs there.

The file name sorts last so that a run that stops at the first failure has
run every other test before this one; the tests do not depend on that order.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _ref_and_scale(Ar, dV):
    ref = dV * (Ar @ Ar.T)
    d = np.sum(Ar * Ar, 1)
    return ref, dV * np.sqrt(np.outer(d, d))


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("N,ng", [(1, 37), (7, 5000), (100, 50000), (128, 4099), (512, 200000)])
def test_gram_noalloc_matches_numpy_twice(dt, N, ng):
    assert torch.cuda.is_available()
    from paper_1510_07230_gb300 import pou
    rng = np.random.default_rng(N * 13 + ng)
    tdt = torch.float64 if dt == "f64" else torch.float32
    A = torch.as_tensor(rng.standard_normal((N, ng)), dtype=tdt, device="cuda")
    dV = 0.37
    Ar = A.double().cpu().numpy()
    ref, scale = _ref_and_scale(Ar, dV)
    tol = 1e-13 if dt == "f64" else 2e-6
    for _ in range(2):
        S = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
        pou.gram_noalloc(A, dV, S)
        torch.cuda.synchronize()
        got = S.cpu().numpy()
        assert np.max(np.abs(got - ref) / scale) < tol
        assert np.array_equal(got, got.T)
        # the next call sees other contents in A: the buffer must not leak the old sums
        A.mul_(-0.5)
        Ar = Ar * -0.5
        ref, scale = _ref_and_scale(Ar, dV)


FRESH = r"""
import sys
sys.path.insert(0, %(root)r)
import numpy as np
import torch
from paper_1510_07230_gb300 import pou
torch.cuda.set_device(0)
rng = np.random.default_rng(5)
for dt, tol in ((torch.float32, 2e-6), (torch.float64, 1e-13)):
    A = torch.as_tensor(rng.standard_normal((64, 30000)), dtype=dt, device="cuda")
    S = torch.full((64, 64), float("nan"), dtype=torch.float64, device="cuda")
    pou.gram_noalloc(A, 0.5, S)
    torch.cuda.synchronize()
    Ar = A.double().cpu().numpy()
    ref = 0.5 * (Ar @ Ar.T)
    d = np.sum(Ar * Ar, 1)
    err = np.max(np.abs(S.cpu().numpy() - ref) / (0.5 * np.sqrt(np.outer(d, d))))
    assert err < tol, err
print("ok")
"""


def test_gram_noalloc_first_call_of_a_process():
    """The allocation-free call made before any other library call of a
    fresh process (where the buffer's device address is looked up)."""
    r = subprocess.run([sys.executable, "-c", FRESH % {"root": ROOT}], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().endswith("ok")


def test_gram_noalloc_rejects_too_many_orbitals():
    from paper_1510_07230_gb300 import pou
    N = pou.MAX_N + 1
    A = torch.zeros((N, 64), dtype=torch.float32, device="cuda")
    S = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    with pytest.raises(pou.PouError) as ei:
        pou.gram_noalloc(A, 1.0, S)
    assert ei.value.status == pou.EINVAL
