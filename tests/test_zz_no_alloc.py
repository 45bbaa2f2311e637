"""Allocation-free Gram entry point (pou_gram_noalloc) against pou_gram.

For callers that cannot allocate device memory (stream capture, real-time
loops, fixed memory budgets), pou_gram_noalloc keeps its partial sums in the
library's static device buffer.  Its result must equal pou_gram's within the
tolerance of the Gram tests, on two calls in a row (the buffer keeps the
previous call's contents).  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("N,ng", [(1, 37), (7, 5000), (100, 50000), (128, 4099)])
def test_gram_noalloc_matches_gram_twice(dt, N, ng):
    assert torch.cuda.is_available()
    from paper_1510_07230_gb300 import pou
    rng = np.random.default_rng(N * 13 + ng)
    tdt = torch.float64 if dt == "f64" else torch.float32
    A = torch.as_tensor(rng.standard_normal((N, ng)), dtype=tdt, device="cuda")
    code = pou.DT_F64 if dt == "f64" else pou.DT_F32
    ws = torch.empty(pou.gram_workspace_bytes(code, ng, N) // 8 + 1, dtype=torch.float64, device="cuda")
    dV = 0.37
    S_ref = torch.empty((N, N), dtype=torch.float64, device="cuda")
    pou.gram(A, dV, S_ref, ws)
    Ar = A.double().cpu().numpy()
    scale = dV * np.sqrt(np.outer(np.sum(Ar * Ar, 1), np.sum(Ar * Ar, 1)))
    tol = 1e-13 if dt == "f64" else 2e-6
    ref = S_ref.cpu().numpy()
    for _ in range(2):
        S = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
        pou.gram_noalloc(A, dV, S)
        torch.cuda.synchronize()
        got = S.cpu().numpy()
        assert np.max(np.abs(got - ref) / scale) < tol
        assert np.allclose(got, got.T, rtol=0, atol=0)


def test_gram_noalloc_rejects_too_many_orbitals():
    from paper_1510_07230_gb300 import pou
    N = pou.MAX_N + 1
    A = torch.zeros((N, 64), dtype=torch.float32, device="cuda")
    S = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    with pytest.raises(pou.PouError) as ei:
        pou.gram_noalloc(A, 1.0, S)
    assert ei.value.status == pou.EINVAL
