"""The C-ABI library loads without a GPU and exports what include/pou.h declares."""
import ctypes as C
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1510_07230_gb300", "libpou.so")


@pytest.fixture(scope="module")
def pou():
    if not os.path.exists(LIB):
        from paper_1510_07230_gb300 import build
        build.build()
    from paper_1510_07230_gb300 import pou as P
    return P


def test_every_declared_function_is_exported(pou):
    names = pou.header_functions()
    assert len(names) >= 25
    missing = [n for n, ok in pou.library_exports(names).items() if not ok]
    assert not missing, missing


def test_exported_symbols_with_nm(pou):
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for n in pou.header_functions():
        assert n in exported, n


def test_config_default_is_the_papers_constants(pou):
    cfg = pou.Config()
    pou._lib.pou_config_default(C.byref(cfg))
    assert cfg.rho1 == 1e-4 and cfg.delta == 0.1 and cfg.eta == 0.85
    assert cfg.n_org == 1 and cfg.n_diag == 0 and cfg.bb_variant == 3
    assert cfg.max_backtrack == 10 and cfg.stencil_order == 2


@pytest.mark.parametrize("field,value", [
    ("N", 0), ("N", 129), ("N", 513), ("stencil_order", 3), ("precision", 7), ("bb_variant", 0),
    ("delta", 1.5), ("eta", -0.1), ("n_org", 0), ("n_diag", -1), ("tau_min", 0.0), ("direction", 2),
])
def test_invalid_configs_rejected_before_touching_the_device(pou, field, value):
    cfg = pou.make_config(16, 8.0, 4)
    setattr(cfg, field, value)
    ctx = C.c_void_p()
    assert pou._lib.pou_create(C.byref(cfg), C.byref(ctx)) == pou.EINVAL
    assert not ctx.value


@pytest.mark.parametrize("precision,n_diag,ok", [(1, 0, True), (2, 0, True), (0, 0, False), (1, 10, False),
                                                 (2, 10, False)])
def test_more_than_128_orbitals_in_the_fp32_forms_only(pou, precision, n_diag, ok):
    """N > 128 is accepted by the FP32 forms (split or single TF32 Gram)
    without the subspace diagonalisation; the validation decides before any
    device call (without a GPU an accepted configuration fails later, at the
    device)."""
    cfg = pou.make_config((16, 16, 18), (6.0, 6.0, 7.0), 512)
    cfg.precision = precision
    cfg.n_diag = n_diag
    ctx = C.c_void_p()
    st = pou._lib.pou_create(C.byref(cfg), C.byref(ctx))
    if ok:
        assert st != pou.EINVAL
        if ctx.value:
            pou._lib.pou_destroy(ctx)
    else:
        assert st == pou.EINVAL and not ctx.value


def test_invalid_grid_rejected(pou):
    for n in [(7, 8, 8), (16, 1, 16), (0, 8, 8)]:  # 7 is not 2^a 3^b 5^c
        cfg = pou.make_config(n, 8.0, 2)
        ctx = C.c_void_p()
        assert pou._lib.pou_create(C.byref(cfg), C.byref(ctx)) == pou.EINVAL


def test_null_arguments(pou):
    assert pou._lib.pou_create(None, None) == pou.EINVAL
    assert pou._lib.pou_iterate(None, 1, 0.0, 0.0, None) == pou.EINVAL
    pou._lib.pou_destroy(None)
    assert pou._lib.pou_launch_count(None) == 0


def test_workspace_sizes(pou):
    assert pou.gram_workspace_bytes(pou.DT_F64, 4096, 100) > 0
    assert pou.hartree_workspace_bytes((8, 6, 10)) == 8 * 6 * 10 * 16


def test_product_path_does_not_import_the_oracle():
    code = ("import sys; import paper_1510_07230_gb300.pou, paper_1510_07230_gb300.autograd; "
            "print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT)
    assert r.stdout.strip() == "False", r.stderr


def test_standalone_ops_refuse_host_tensors(pou):
    """The stand-alone operations take device memory: host tensors are refused
    before the library is called (and the library refuses host pointers)."""
    torch = pytest.importorskip("torch")
    A = torch.zeros((4, 64), dtype=torch.float32)
    S = torch.zeros((4, 4), dtype=torch.float64)
    with pytest.raises(ValueError):
        pou.gram(A, 1.0, S, torch.zeros(1024, dtype=torch.float64))
    with pytest.raises(ValueError):
        pou.gram_noalloc(A, 1.0, S)
    with pytest.raises(ValueError):
        pou.cholinv(S, torch.zeros_like(S), torch.zeros(1, dtype=torch.int32))
    with pytest.raises(ValueError):
        pou.rotate(A, S, torch.zeros_like(A))
    with pytest.raises(ValueError):
        pou.hartree((4, 4, 4), (1.0, 1.0, 1.0), torch.zeros(64, dtype=torch.float64),
                    torch.zeros(64, dtype=torch.float64), torch.zeros(4096, dtype=torch.float64))


def test_backward_refuses_mismatched_output(pou):
    """U and dE/dU share one dtype code and one on_device flag in the call:
    the binding refuses an output of another dtype before the library runs."""
    s = pou.Solver.__new__(pou.Solver)  # no context: the check comes first
    s.M = 0
    s._ctx = None
    with pytest.raises(TypeError):
        pou.Solver.backward(s, np.zeros((2, 8)), 1.0, np.zeros((2, 8), dtype=np.float32))


def test_every_boundary_function_is_documented():
    """Each function of the C-ABI header has a comment block right above its
    declaration (what it computes, with its section or equation, arguments,
    layout, ownership and errors)."""
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "pou.h")).read()
    lines = hdr.splitlines()
    missing = []
    for i, ln in enumerate(lines):
        m = re.match(r"^(?:pou_status|void|const char\*|size_t|long long)\s+(pou_\w+)\(", ln)
        if not m:
            continue
        # declarations written together (no blank line between them) share
        # one comment; a blank line ends the group
        j = i - 1
        while j >= 0 and lines[j].strip() and not lines[j].rstrip().endswith("*/"):
            j -= 1
        if j < 0 or not lines[j].strip():
            missing.append(m.group(1))
    assert not missing, missing


def test_product_package_does_not_import_the_oracle():
    """The oracle is test infrastructure: nothing in the library package
    imports it (no CPU fallback through it)."""
    pkg = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1510_07230_gb300")
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(root, f)).read()
                assert "pou_oracle" not in text and "import oracle" not in text and "from oracle" not in text, f
