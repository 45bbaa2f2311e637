"""ctypes binding of libpou.so (include/pou.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels.  Arrays may be
NumPy arrays (host memory) or torch tensors (host or CUDA memory); device
tensors are passed by pointer and used on the context's stream.  If the
library is missing this module raises at import: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpou.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pou.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_1510_07230_gb300.build`")
_lib = C.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ENOTSPD, ENAN, ENOCONV = range(7)
STATUS_NAMES = {0: "POU_OK", 1: "POU_EINVAL", 2: "POU_ENOMEM", 3: "POU_ECUDA", 4: "POU_ENOTSPD",
                5: "POU_ENAN", 6: "POU_ENOCONV"}
FP64, FP32, FP32_TF32 = 0, 1, 2  # FP32 = TF32x3 split products; FP32_TF32 = single-product TF32 Gram
OPT_PAR, OPTM_QR = 0, 1  # config direction: per-orbital sigma_ii (the paper's method) or full Sigma
TAU_SHARED, TAU_PER_ORBITAL = 0, 1  # config tau_mode
STEEPEST_DESCENT, CONJUGATE_GRADIENT = 0, 1  # config solver
DT_F64, DT_F32 = 0, 1
MAX_N = 512       # FP32 form
MAX_N_FP64 = 128  # FP64 form, subspace diagonalisation


class PouError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("L", C.c_double * 3), ("stencil_order", C.c_int), ("N", C.c_int),
                ("precision", C.c_int), ("hartree", C.c_int), ("exchange", C.c_int),
                ("bb_variant", C.c_int), ("rho1", C.c_double), ("delta", C.c_double),
                ("eta", C.c_double), ("max_backtrack", C.c_int), ("tau0", C.c_double),
                ("tau_min", C.c_double), ("tau_max", C.c_double), ("n_org", C.c_int),
                ("n_diag", C.c_int), ("stream", C.c_void_p), ("direction", C.c_int),
                ("tau_mode", C.c_int), ("solver", C.c_int)]


class EnergyTerms(C.Structure):
    _fields_ = [("kinetic", C.c_double), ("external", C.c_double), ("hartree", C.c_double),
                ("exchange", C.c_double), ("total", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Report(C.Structure):
    _fields_ = [("iterations", C.c_int), ("passes", C.c_int), ("backtracks", C.c_int), ("forced", C.c_int),
                ("total_iterations", C.c_int), ("converged", C.c_int), ("energy", C.c_double),
                ("tau", C.c_double), ("df_mean3", C.c_double), ("grad_norm", C.c_double),
                ("gram_offdiag", C.c_double), ("second_passes", C.c_int), ("diagonalisations", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_D = C.c_double
_I = C.c_int
_PD = C.POINTER(C.c_double)
_SIG = {
    "pou_config_default": (None, [C.POINTER(Config)]),
    "pou_create": (_I, [C.POINTER(Config), C.POINTER(_P)]),
    "pou_destroy": (None, [_P]),
    "pou_last_error": (C.c_char_p, [_P]),
    "pou_set_vext": (_I, [_P, _P, _I]),
    "pou_set_atoms": (_I, [_P, _I, _P, _P, _D]),
    "pou_set_orbitals": (_I, [_P, _P, _I, _I]),
    "pou_set_projectors": (_I, [_P, _I, _P, _P, _P]),
    "pou_iterate": (_I, [_P, _I, _D, _D, C.POINTER(Report)]),
    "pou_energy": (_I, [_P, C.POINTER(EnergyTerms)]),
    "pou_get_orbitals": (_I, [_P, _P, _I, _I]),
    "pou_get_density": (_I, [_P, _P, _I]),
    "pou_get_potential": (_I, [_P, _P, _I]),
    "pou_gradient_norm": (_I, [_P, _PD]),
    "pou_evaluate": (_I, [_P, _P, _I, _I, C.POINTER(EnergyTerms)]),
    "pou_backward": (_I, [_P, _P, _I, _I, _D, _P, _P, _P]),
    "pou_get_history": (_I, [_P, _P, _P, _I, C.POINTER(C.c_int)]),
    "pou_get_state": (_I, [_P, _P, C.POINTER(C.c_size_t)]),
    "pou_set_state": (_I, [_P, _P, C.c_size_t]),
    "pou_synchronize": (_I, [_P]),
    "pou_selftest_wait_timeout": (_I, [_D, C.POINTER(C.c_int)]),
    "pou_launch_count": (C.c_longlong, [_P]),
    "pou_set_profiling": (_I, [_P, _I]),
    "pou_get_profile": (_I, [_P, _I, _P, _P, _P, C.POINTER(C.c_int)]),
    "pou_gram_workspace_bytes": (C.c_size_t, [_I, C.c_longlong, _I]),
    "pou_gram": (_I, [_I, C.c_longlong, _I, _P, _D, _P, _P, C.c_size_t, _P]),
    "pou_gram_noalloc": (_I, [_I, C.c_longlong, _I, _P, _D, _P, _P]),
    "pou_cholinv": (_I, [_I, _P, _P, _P, _P]),
    "pou_rotate": (_I, [_I, C.c_longlong, _I, _P, _P, _P, _P, _P]),
    "pou_hartree_workspace_bytes": (C.c_size_t, [C.POINTER(C.c_int)]),
    "pou_hartree": (_I, [C.POINTER(C.c_int), C.POINTER(C.c_double), _P, _P, _P, C.c_size_t, _P]),
}
for _name, (_res, _args) in _SIG.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def header_functions() -> list:
    """Names of the functions include/pou.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pou_[a-z0-9_]+)\s*\(", txt)))


def library_exports(names) -> dict:
    return {n: hasattr(_lib, n) for n in names}


# ------------------------------------------------------------------ arrays
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, keep=None):
    """(pointer, dtype code, on_device) of a contiguous float32/float64 array.

    A non-contiguous NumPy input is copied when ``keep`` (a list that holds
    the copy alive for the call) is given; outputs must be contiguous.
    """
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        import torch
        if x.dtype == torch.float64:
            dt = DT_F64
        elif x.dtype == torch.float32:
            dt = DT_F32
        else:
            raise TypeError("orbital tensors must be float32 or float64")
        return C.c_void_p(x.data_ptr()), dt, 1 if x.is_cuda else 0
    a = np.asarray(x)
    if not a.flags["C_CONTIGUOUS"]:
        if keep is None:
            raise ValueError("array must be C-contiguous")
        a = np.ascontiguousarray(a)
        keep.append(a)
    if a.dtype == np.float64:
        dt = DT_F64
    elif a.dtype == np.float32:
        dt = DT_F32
    else:
        raise TypeError("arrays must be float32 or float64")
    return C.c_void_p(a.ctypes.data), dt, 0


def _fptr(x):
    """Pointer / on_device of a float64 field (numpy or torch)."""
    p, dt, dev = _ptr(x)
    if dt != DT_F64:
        raise TypeError("fields are float64")
    return p, dev


def make_config(n, L, N, order=2, precision=FP64, hartree=1, exchange=1, stream=None, **kw) -> Config:
    cfg = Config()
    _lib.pou_config_default(C.byref(cfg))
    n = (n, n, n) if np.isscalar(n) else tuple(n)
    L = (L, L, L) if np.isscalar(L) else tuple(L)
    for a in range(3):
        cfg.n[a] = int(n[a])
        cfg.L[a] = float(L[a])
    cfg.N = int(N)
    cfg.stencil_order = int(order)
    cfg.precision = int(precision)
    cfg.hartree = int(hartree)
    cfg.exchange = int(exchange)
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    if stream is not None:
        cfg.stream = C.c_void_p(int(stream))
    return cfg


class Solver:
    """One solver context (pou_ctx) on the current CUDA device."""

    def __init__(self, n, L, N, order=2, precision=FP64, hartree=1, exchange=1, stream=None, **kw):
        self.cfg = make_config(n, L, N, order, precision, hartree, exchange, stream, **kw)
        self._ctx = C.c_void_p()
        st = _lib.pou_create(C.byref(self.cfg), C.byref(self._ctx))
        if st != OK:
            raise PouError(st, "pou_create failed (configuration or device memory)")
        self.n = tuple(self.cfg.n)
        self.N = int(N)
        self.precision = precision
        self.M = 0

    # -- helpers
    def _check(self, st):
        if st != OK:
            raise PouError(st, (_lib.pou_last_error(self._ctx) or b"").decode())
        return st

    @property
    def shape(self):
        nx, ny, nz = self.n
        return (self.N, nz, ny, nx)

    @property
    def grid_shape(self):
        nx, ny, nz = self.n
        return (nz, ny, nx)

    def close(self):
        if self._ctx:
            _lib.pou_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- problem statement
    def set_vext(self, vext):
        p, dev = _fptr(vext)
        self._check(_lib.pou_set_vext(self._ctx, p, dev))

    def set_atoms(self, R, Z, width=0.8):
        R = np.ascontiguousarray(R, dtype=np.float64)
        Z = np.ascontiguousarray(Z, dtype=np.float64)
        self.M = len(Z)
        self._check(_lib.pou_set_atoms(self._ctx, self.M, R.ctypes.data, Z.ctypes.data, float(width)))

    def set_projectors(self, centres, widths, amps):
        """Nonlocal projectors (pou_set_projectors); an empty set removes them."""
        c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(widths, dtype=np.float64).ravel()
        a = np.ascontiguousarray(amps, dtype=np.float64).ravel()
        if not (len(c) == len(w) == len(a)):
            raise ValueError("centres, widths and amps need one entry per projector")
        P = len(w)
        self._check(_lib.pou_set_projectors(self._ctx, P, c.ctypes.data if P else None,
                                            w.ctypes.data if P else None, a.ctypes.data if P else None))

    def set_orbitals(self, U):
        keep = []
        p, dt, dev = _ptr(U, keep)
        self._check(_lib.pou_set_orbitals(self._ctx, p, dt, dev))

    def iterate(self, max_iter, e_tol=0.0, grad_tol=0.0, check=True):
        rep = Report()
        st = _lib.pou_iterate(self._ctx, int(max_iter), float(e_tol), float(grad_tol), C.byref(rep))
        if check and st not in (OK, ENOCONV):
            self._check(st)
        out = rep.as_dict()
        out["status"] = st
        return out

    def energy(self):
        t = EnergyTerms()
        self._check(_lib.pou_energy(self._ctx, C.byref(t)))
        return t.as_dict()

    def get_orbitals(self, out=None, dtype=np.float64):
        if out is None:
            out = np.empty(self.shape, dtype=dtype)
        p, dt, dev = _ptr(out)
        self._check(_lib.pou_get_orbitals(self._ctx, p, dt, dev))
        return out

    def get_density(self, out=None):
        if out is None:
            out = np.empty(self.grid_shape)
        p, dev = _fptr(out)
        self._check(_lib.pou_get_density(self._ctx, p, dev))
        return out

    def get_potential(self, out=None):
        if out is None:
            out = np.empty(self.grid_shape)
        p, dev = _fptr(out)
        self._check(_lib.pou_get_potential(self._ctx, p, dev))
        return out

    def gradient_norm(self):
        v = C.c_double()
        self._check(_lib.pou_gradient_norm(self._ctx, C.byref(v)))
        return v.value

    def evaluate(self, U):
        keep = []
        p, dt, dev = _ptr(U, keep)
        t = EnergyTerms()
        self._check(_lib.pou_evaluate(self._ctx, p, dt, dev, C.byref(t)))
        return t.as_dict()

    def backward(self, U=None, g=1.0, dEdU=None, atoms=False):
        """dE/dU (into dEdU if given) and, with atoms=True, (dE/dR, dE/dZ)."""
        keep = []
        if U is not None:
            p, dt, dev = _ptr(U, keep)
        else:
            p, dt, dev = C.c_void_p(), DT_F64, 0
        gp = C.c_void_p()
        if dEdU is not None:
            gp, gdt, gdev = _ptr(dEdU)
            if U is None:
                dt, dev = gdt, gdev
            elif (gdt, gdev) != (dt, dev):
                # one dtype and one on_device flag describe both arrays in the call
                raise TypeError("dEdU must have the dtype and the device of U")
        dR = np.zeros((self.M, 3)) if atoms else None
        dZ = np.zeros(self.M) if atoms else None
        self._check(_lib.pou_backward(self._ctx, p, dt, dev, float(g), gp,
                                      dR.ctypes.data if atoms else None,
                                      dZ.ctypes.data if atoms else None))
        return dEdU, dR, dZ

    def history(self, max_entries=16384):
        E = np.empty(max_entries)
        tau = np.empty(max_entries)
        cnt = C.c_int()
        self._check(_lib.pou_get_history(self._ctx, E.ctypes.data, tau.ctypes.data, max_entries, C.byref(cnt)))
        return E[:cnt.value].copy(), tau[:cnt.value].copy()

    def get_state(self) -> bytes:
        size = C.c_size_t()
        self._check(_lib.pou_get_state(self._ctx, None, C.byref(size)))
        buf = (C.c_char * size.value)()
        self._check(_lib.pou_get_state(self._ctx, buf, C.byref(size)))
        return bytes(buf)

    def set_state(self, blob: bytes):
        self._check(_lib.pou_set_state(self._ctx, blob, len(blob)))

    def synchronize(self):
        self._check(_lib.pou_synchronize(self._ctx))

    def launch_count(self) -> int:
        return int(_lib.pou_launch_count(self._ctx))

    def set_profiling(self, enable: bool):
        self._check(_lib.pou_set_profiling(self._ctx, 1 if enable else 0))

    def profile(self, max_entries=64) -> dict:
        """{kernel name: (launches, total ms)} since profiling was enabled."""
        names = C.create_string_buffer(32 * max_entries)
        launches = (C.c_longlong * max_entries)()
        ms = (C.c_double * max_entries)()
        cnt = C.c_int()
        self._check(_lib.pou_get_profile(self._ctx, max_entries, names, launches, ms, C.byref(cnt)))
        out = {}
        for i in range(cnt.value):
            nm = names.raw[32 * i:32 * i + 32].split(b"\0", 1)[0].decode()
            out[nm] = (int(launches[i]), float(ms[i]))
        return out


# ------------------------------------------------------------ stand-alone ops
def _dev(x, what, dtype=None, numel=None):
    """Device pointer of a contiguous CUDA tensor, checked before the call
    (the library also refuses host pointers where it expects device memory)."""
    if not _is_torch(x) or not x.is_cuda:
        raise ValueError(f"{what}: a CUDA tensor is required")
    if not x.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")
    if dtype is not None and x.dtype != dtype:
        raise TypeError(f"{what}: dtype {x.dtype}, expected {dtype}")
    if numel is not None and x.numel() < numel:
        raise ValueError(f"{what}: {x.numel()} elements, need {numel}")
    return C.c_void_p(x.data_ptr())


def _stream_ptr(stream):
    return C.c_void_p(int(stream)) if stream is not None else C.c_void_p()


def gram(A, dV, S, workspace, stream=None):
    """S = dV A^T A for a device block A [N][Ng] (torch tensors on CUDA)."""
    import torch
    _dev(A, "A")
    N = A.shape[0]
    ng = A.numel() // N
    p, dt, _ = _ptr(A)
    sp = _dev(S, "S", torch.float64, N * N)
    wp = _dev(workspace, "workspace")
    st = _lib.pou_gram(dt, ng, N, p, float(dV), sp, wp, workspace.numel() * workspace.element_size(),
                       _stream_ptr(stream))
    if st != OK:
        raise PouError(st, "pou_gram")


def gram_noalloc(A, dV, S, stream=None):
    """S = dV A^T A like gram(), with no workspace: the library's fixed device buffer."""
    import torch
    _dev(A, "A")
    N = A.shape[0]
    ng = A.numel() // N
    p, dt, _ = _ptr(A)
    st = _lib.pou_gram_noalloc(dt, ng, N, p, float(dV), _dev(S, "S", torch.float64, N * N), _stream_ptr(stream))
    if st != OK:
        raise PouError(st, "pou_gram_noalloc")


def gram_workspace_bytes(dtype_code, ng, N):
    return int(_lib.pou_gram_workspace_bytes(dtype_code, ng, N))


def cholinv(S, Rinv, info, stream=None):
    import torch
    N = S.shape[0]
    st = _lib.pou_cholinv(N, _dev(S, "S", torch.float64, N * N), _dev(Rinv, "Rinv", torch.float64, N * N),
                          _dev(info, "info", torch.int32, 1), _stream_ptr(stream))
    if st != OK:
        raise PouError(st, "pou_cholinv")


def rotate(A, Rinv, B, rho=None, stream=None):
    import torch
    _dev(A, "A")
    N = A.shape[0]
    ng = A.numel() // N
    p, dt, _ = _ptr(A)
    bp = _dev(B, "B", A.dtype, A.numel())
    rp = _dev(rho, "rho", torch.float64, ng) if rho is not None else None
    st = _lib.pou_rotate(dt, ng, N, p, _dev(Rinv, "Rinv", torch.float64, N * N), bp, rp, _stream_ptr(stream))
    if st != OK:
        raise PouError(st, "pou_rotate")


def hartree_workspace_bytes(n):
    arr = (C.c_int * 3)(*n)
    return int(_lib.pou_hartree_workspace_bytes(arr))


def hartree(n, L, rho, vh, workspace, stream=None):
    import torch
    narr = (C.c_int * 3)(*n)
    Larr = (C.c_double * 3)(*L)
    ng = int(n[0]) * int(n[1]) * int(n[2])
    st = _lib.pou_hartree(narr, Larr, _dev(rho, "rho", torch.float64, ng), _dev(vh, "vh", torch.float64, ng),
                          _dev(workspace, "workspace"), workspace.numel() * workspace.element_size(),
                          _stream_ptr(stream))
    if st != OK:
        raise PouError(st, "pou_hartree")


def selftest_wait_timeout(limit_s=0.05) -> bool:
    """Run the bounded barrier wait on a barrier nothing arrives at
    (pou_selftest_wait_timeout); True when it gave up as designed."""
    t = C.c_int(0)
    st = _lib.pou_selftest_wait_timeout(float(limit_s), C.byref(t))
    if st != OK:
        raise PouError(st, "pou_selftest_wait_timeout")
    return bool(t.value)
