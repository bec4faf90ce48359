"""GB300 block PLHR: interior eigenpairs of Hermitian problems (Vecharynski &
Knyazev, arXiv 1408.0042) on one GPU.

This module is a thin ctypes binding of libplhr.so (C ABI in include/plhr.h):
it only marshals arguments.  Every step of the solver runs in the library's
CUDA kernels; there is no CPU fallback, and importing an entry point without a
built library raises.  PyTorch supplies device memory and streams.

    import paper_1408_0042_gb300 as plhr
    A = plhr.Operator.laplacian((128, 128, 128), h=1/129)
    T = plhr.AVMG(A, sigma, levels=4, nu=2)
    lam, V, info = plhr.solve(A, sigma, k=10, T=T, tol=1e-8)
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libplhr.so")

PLHR_OK, PLHR_ENOTCONV, PLHR_EINVAL, PLHR_EBREAKDOWN, PLHR_ENAN, PLHR_ENOMEM, PLHR_ECUDA = range(7)
LAP5_2D, LAP7_3D, HAM7_BLOCH, Q1_STIFF27, Q1_MASS27 = 1, 2, 3, 4, 5
BC_DIRICHLET, BC_PERIODIC = 0, 1
PRECISION_F64, PRECISION_MIXED = 0, 1
GRAM_F64, GRAM_F32, GRAM_DW, GRAM_F32_TC = 0, 1, 2, 3


class StencilDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dims", ctypes.c_int64 * 3), ("h", ctypes.c_double),
                ("scale", ctypes.c_double), ("bc", ctypes.c_int), ("bloch_k", ctypes.c_double * 3),
                ("field", ctypes.c_void_p)]


class MGOpts(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("nu", ctypes.c_int), ("delta", ctypes.c_double),
                ("transfer", ctypes.c_int), ("coarse", ctypes.c_int), ("indefinite", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [("maxit", ctypes.c_int), ("precision", ctypes.c_int), ("real_arithmetic", ctypes.c_int),
                ("s_vectors", ctypes.c_int), ("soft_lock", ctypes.c_int),
                ("v_init", ctypes.c_void_p), ("ld_init", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("history", ctypes.c_void_p), ("history_cap", ctypes.c_int), ("guard", ctypes.c_int),
                ("switch_tol", ctypes.c_double), ("extraction", ctypes.c_int), ("tensor_cores", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("max_rel_residual", ctypes.c_double), ("setup_seconds", ctypes.c_double),
                ("solve_seconds", ctypes.c_double), ("history_len", ctypes.c_int),
                ("mixed_iterations", ctypes.c_int)]


# name -> (restype, argtypes); every symbol declared in include/plhr.h
_SIGS = {
    "plhr_op_stencil": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(StencilDesc)]),
    "plhr_op_size": (ctypes.c_int64, [ctypes.c_void_p]),
    "plhr_op_hamiltonian": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_void_p]),
    "plhr_eigval_grad": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "plhr_prec_tpa": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_double,
                                     ctypes.c_double]),
    "plhr_prec_tpa_energy": (ctypes.c_double, [ctypes.c_void_p]),
    "plhr_prec_diag": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_void_p, ctypes.c_int]),
    "plhr_prec_callback": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "plhr_op_csr": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int]),
    "plhr_eigvec_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p,
                                           ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                           ctypes.c_void_p]),
    "plhr_op_destroy": (None, [ctypes.c_void_p]),
    "plhr_op_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "plhr_op_apply_c128": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "plhr_op_apply_pair": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_void_p]),
    "plhr_mg_opts_default": (None, [ctypes.POINTER(MGOpts)]),
    "plhr_prec_avmg": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_double,
                                      ctypes.POINTER(MGOpts)]),
    "plhr_prec_destroy": (None, [ctypes.c_void_p]),
    "plhr_prec_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "plhr_profile_work": (None, [ctypes.c_void_p]),
    "plhr_profile_bytes": (None, [ctypes.c_void_p]),
    "plhr_gram": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "plhr_prec_apply_dw": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "plhr_prec_apply_f32": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "plhr_options_default": (None, [ctypes.POINTER(Options)]),
    "plhr_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(Options),
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(Info),
                                  ctypes.c_void_p]),
    "plhr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "plhr_kernel_launches": (ctypes.c_longlong, []),
    "plhr_profile_enable": (None, [ctypes.c_int]),
    "plhr_profile_read": (None, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "plhr_last_error": (ctypes.c_char_p, []),
    "plhr_tharm_extract": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 11
                           + [ctypes.c_void_p]),
    "plhr_tharm_extract_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 11),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libplhr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libplhr.so is not built (%s); run `python -m paper_1408_0042_gb300.build`" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PlhrError(RuntimeError):
    def __init__(self, status, where):
        lib = load_library()
        msg = "%s: %s (%s)" % (where, lib.plhr_status_string(status).decode(), lib.plhr_last_error().decode())
        super().__init__(msg)
        self.status = status


def _check(status, where):
    if status != PLHR_OK:
        raise PlhrError(status, where)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_block(X, n, name):
    import torch
    if not isinstance(X, torch.Tensor) or not X.is_cuda or X.dtype != torch.float64 or X.dim() != 2:
        raise ValueError("%s must be a 2-D float64 CUDA tensor" % name)
    if X.shape[0] != n:
        raise ValueError("%s has %d rows, operator has %d" % (name, X.shape[0], n))
    if X.stride(1) != 1 or (X.shape[0] > 1 and X.stride(0) < X.shape[1]):
        raise ValueError("%s must be row-major with unit column stride" % name)


class Operator:
    """A stencil operator (Dirichlet FD Laplacian, 5-point in 2D, 7-point in 3D)."""

    def __init__(self, handle, dims, h, scale):
        self._h = handle
        self.dims = tuple(dims)
        self.h = h
        self.scale = scale

    @classmethod
    def _stencil(cls, kind, dims, h, scale=1.0, bc=BC_DIRICHLET, bloch_k=(0.0, 0.0, 0.0), field=None):
        lib = load_library()
        d = StencilDesc()
        d.kind = kind
        d.dims[:] = list(dims) + [1] * (3 - len(dims))
        d.h = h
        d.scale = scale
        d.bc = bc
        d.bloch_k[:] = [float(v) for v in bloch_k]
        d.field = field.data_ptr() if field is not None else None
        out = ctypes.c_void_p()
        _check(lib.plhr_op_stencil(ctypes.byref(out), ctypes.byref(d)), "plhr_op_stencil")
        op = cls(out, tuple(dims), h, scale)
        op._field = field
        return op

    @classmethod
    def laplacian(cls, dims, h, scale=1.0, periodic=False):
        """Negative FD Laplacian (5-point 2D, 7-point 3D), Dirichlet or periodic."""
        if len(dims) not in (2, 3):
            raise ValueError("dims must have 2 or 3 entries")
        return cls._stencil(LAP5_2D if len(dims) == 2 else LAP7_3D, dims, h, scale,
                            BC_PERIODIC if periodic else BC_DIRICHLET)

    @staticmethod
    def _device_field(v, count, name):
        import torch
        if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == torch.float64):
            raise ValueError("%s must be a float64 CUDA tensor" % name)
        v = v.contiguous().reshape(-1)
        if v.numel() != count:
            raise ValueError("%s has %d values, %d expected" % (name, v.numel(), count))
        return v

    @classmethod
    def q1_stiffness(cls, elems, coeff=None, scale=1.0):
        """Trilinear FE stiffness of -div(c grad u) on the unit cube with elems =
        (Ex, Ey, Ez) elements per axis (an int: the same on every axis), h =
        1/Ex, interior nodes x fastest; coeff: float64 CUDA tensor of the element
        coefficients (x fastest) or None (c = 1)."""
        E = (elems,) * 3 if isinstance(elems, int) else tuple(elems)
        f = None if coeff is None else cls._device_field(coeff, int(np.prod(E)), "coeff")
        return cls._stencil(Q1_STIFF27, tuple(e - 1 for e in E), 1.0 / E[0], scale, field=f)

    @classmethod
    def q1_mass(cls, elems, scale=1.0):
        """Trilinear FE mass matrix on the mesh of q1_stiffness(elems)."""
        E = (elems,) * 3 if isinstance(elems, int) else tuple(elems)
        return cls._stencil(Q1_MASS27, tuple(e - 1 for e in E), 1.0 / E[0], scale)

    @classmethod
    def bloch(cls, dims, h, potential, kappa):
        """Bloch Hamiltonian -1/2 Lap_kappa + diag(V) on a periodic 3D grid
        (complex for kappa != 0: apply_c128)."""
        f = cls._device_field(potential, int(np.prod(dims)), "potential")
        return cls._stencil(HAM7_BLOCH, dims, h, 0.5, BC_PERIODIC, kappa, f)

    @classmethod
    def csr(cls, A):
        """A general sparse symmetric operator from a scipy sparse matrix (or
        anything with .tocsr()); the arrays are copied to the device."""
        lib = load_library()
        A = A.tocsr()
        n = A.shape[0]
        if A.shape != (n, n):
            raise ValueError("A must be square")
        rowptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
        col = np.ascontiguousarray(A.indices, dtype=np.int32)
        val = np.ascontiguousarray(A.data, dtype=np.float64)
        out = ctypes.c_void_p()
        _check(lib.plhr_op_csr(ctypes.byref(out), n, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data, 0),
               "plhr_op_csr")
        return cls(out, (n,), 1.0, 1.0)

    @classmethod
    def hamiltonian(cls, dims, h, potential, periodic=True):
        """H = -1/2 Lap + diag(V) (periodic or Dirichlet) with V a float64 CUDA
        tensor of prod(dims) values, x fastest; the operator keeps a reference."""
        import torch
        lib = load_library()
        if not (isinstance(potential, torch.Tensor) and potential.is_cuda and potential.dtype == torch.float64):
            raise ValueError("potential must be a float64 CUDA tensor")
        pot = potential.contiguous().reshape(-1)
        if pot.numel() != int(np.prod(dims)):
            raise ValueError("potential has %d values for a grid of %d" % (pot.numel(), int(np.prod(dims))))
        d3 = (ctypes.c_int64 * 3)(*(list(dims) + [1] * (3 - len(dims))))
        out = ctypes.c_void_p()
        _check(lib.plhr_op_hamiltonian(ctypes.byref(out), len(dims), d3, h, 1 if periodic else 0,
                                       ctypes.c_void_p(pot.data_ptr())), "plhr_op_hamiltonian")
        op = cls(out, tuple(dims), h, 0.5)
        op._potential = pot
        return op

    @property
    def n(self):
        return int(load_library().plhr_op_size(self._h))

    def apply(self, X, out=None, stream=None):
        import torch
        _check_block(X, self.n, "X")
        if out is None:
            out = torch.empty_like(X)
        _check_block(out, self.n, "out")
        _check(load_library().plhr_op_apply(self._h, X.shape[1], ctypes.c_void_p(X.data_ptr()), X.stride(0),
                                            ctypes.c_void_p(out.data_ptr()), out.stride(0), _stream_ptr(stream)),
               "plhr_op_apply")
        return out

    def apply_c128(self, X, out=None, stream=None):
        """Y = op X for a complex128 CUDA block (n x ncols, row-major)."""
        import torch
        if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.complex128 and X.dim() == 2
                and X.shape[0] == self.n and X.stride(1) == 1):
            raise ValueError("X must be a row-major complex128 CUDA block with n rows")
        if out is None:
            out = torch.empty_like(X)
        _check(load_library().plhr_op_apply_c128(self._h, X.shape[1], ctypes.c_void_p(X.data_ptr()), X.stride(0),
                                                 ctypes.c_void_p(out.data_ptr()), out.stride(0),
                                                 _stream_ptr(stream)), "plhr_op_apply_c128")
        return out

    def apply_pair(self, B, X, stream=None):
        """(A X, B X) in one pass for the Q1 stiffness/mass pair of a mesh."""
        import torch
        _check_block(X, self.n, "X")
        AX = torch.empty_like(X)
        BX = torch.empty_like(X)
        _check(load_library().plhr_op_apply_pair(self._h, B._h, X.shape[1], ctypes.c_void_p(X.data_ptr()),
                                                 X.stride(0), ctypes.c_void_p(AX.data_ptr()), AX.stride(0),
                                                 ctypes.c_void_p(BX.data_ptr()), BX.stride(0), _stream_ptr(stream)),
               "plhr_op_apply_pair")
        return AX, BX

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.plhr_op_destroy(self._h)
            self._h = None


class AVMG:
    """Absolute-value multigrid preconditioner T ~ |L - sigma I|^{-1} (Alg. 4);
    indefinite=True gives INV-MG (Alg. 5), T ~ (L - sigma I)^{-1}."""

    def __init__(self, A: Operator, sigma: float, levels: int = 1, nu: int = 2,
                 delta: float = 2 * math.pi / 10, transfer: int = 0, coarse: int = 0, indefinite: bool = False):
        lib = load_library()
        o = MGOpts()
        lib.plhr_mg_opts_default(ctypes.byref(o))
        o.levels, o.nu, o.delta, o.transfer, o.coarse = levels, nu, delta, transfer, coarse
        o.indefinite = 1 if indefinite else 0
        out = ctypes.c_void_p()
        _check(lib.plhr_prec_avmg(ctypes.byref(out), A._h, sigma, ctypes.byref(o)), "plhr_prec_avmg")
        self._h = out
        self.n = A.n
        self.sigma = sigma

    def apply(self, R, out=None, stream=None):
        import torch
        _check_block(R, self.n, "R")
        if out is None:
            out = torch.empty_like(R)
        _check_block(out, self.n, "out")
        _check(load_library().plhr_prec_apply(self._h, R.shape[1], ctypes.c_void_p(R.data_ptr()), R.stride(0),
                                              ctypes.c_void_p(out.data_ptr()), out.stride(0), _stream_ptr(stream)),
               "plhr_prec_apply")
        return out

    def apply_dw(self, R, out=None, stream=None):
        """The same V-cycle in double-word arithmetic on float64 CUDA blocks."""
        import torch
        _check_block(R, self.n, "R")
        if out is None:
            out = torch.empty_like(R)
        _check_block(out, self.n, "out")
        _check(load_library().plhr_prec_apply_dw(self._h, R.shape[1], ctypes.c_void_p(R.data_ptr()), R.stride(0),
                                                 ctypes.c_void_p(out.data_ptr()), out.stride(0), _stream_ptr(stream)),
               "plhr_prec_apply_dw")
        return out

    def apply_f32(self, R, out=None, stream=None):
        """The same V-cycle in FP32 (the form the mixed-precision solve uses)
        on a float32 CUDA block."""
        import torch
        if R.dtype != torch.float32 or not R.is_cuda or R.dim() != 2 or R.shape[0] != self.n or R.stride(1) != 1:
            raise ValueError("R must be a row-major float32 CUDA block with n rows")
        if out is None:
            out = torch.empty_like(R)
        _check(load_library().plhr_prec_apply_f32(self._h, R.shape[1], ctypes.c_void_p(R.data_ptr()), R.stride(0),
                                                  ctypes.c_void_p(out.data_ptr()), out.stride(0),
                                                  _stream_ptr(stream)), "plhr_prec_apply_f32")
        return out

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.plhr_prec_destroy(self._h)
            self._h = None


class _PrecBase:
    def apply(self, R, out=None, stream=None):
        import torch
        _check_block(R, self.n, "R")
        if out is None:
            out = torch.empty_like(R)
        _check_block(out, self.n, "out")
        _check(load_library().plhr_prec_apply(self._h, R.shape[1], ctypes.c_void_p(R.data_ptr()), R.stride(0),
                                              ctypes.c_void_p(out.data_ptr()), out.stride(0), _stream_ptr(stream)),
               "plhr_prec_apply")
        return out

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.plhr_prec_destroy(self._h)
            self._h = None


class DiagPrec(_PrecBase):
    """T = diag(d) for positive d (numpy array or CUDA tensor, copied)."""

    def __init__(self, d):
        import torch
        lib = load_library()
        out = ctypes.c_void_p()
        if isinstance(d, torch.Tensor) and d.is_cuda:
            dd = d.detach().to(torch.float64).contiguous()
            _check(lib.plhr_prec_diag(ctypes.byref(out), dd.numel(), ctypes.c_void_p(dd.data_ptr()), 1),
                   "plhr_prec_diag")
            self.n = dd.numel()
        else:
            dh = np.ascontiguousarray(np.asarray(d, dtype=np.float64).ravel())
            _check(lib.plhr_prec_diag(ctypes.byref(out), dh.size, dh.ctypes.data, 0), "plhr_prec_diag")
            self.n = dh.size
        self._h = out


_APPLY_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                             ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p)


class _DeviceView:
    """A CUDA array interface over a raw row-major float64 device block."""

    def __init__(self, ptr, rows, cols, ld):
        self.__cuda_array_interface__ = {"shape": (rows, cols), "typestr": "<f8", "data": (ptr, False),
                                         "strides": (8 * ld, 8), "version": 2, "stream": None}


class CallbackPrec(_PrecBase):
    """A preconditioner given as a Python function fn(R, W) that writes T R
    into W (n x c float64 CUDA tensors viewing the library's buffers) on the
    current stream; T must be symmetric positive definite and fixed."""

    def __init__(self, n, fn):
        import torch
        lib = load_library()

        def tramp(ctx, ncols, R, ldr, W, ldw, stream):
            try:
                r = torch.as_tensor(_DeviceView(R, n, ncols, ldr), device="cuda")
                w = torch.as_tensor(_DeviceView(W, n, ncols, ldw), device="cuda")
                fn(r, w)
                return PLHR_OK
            except Exception:   # reported to the library as an invalid-argument failure
                return PLHR_EINVAL

        self._fn = _APPLY_FN(tramp)
        out = ctypes.c_void_p()
        _check(lib.plhr_prec_callback(ctypes.byref(out), n, ctypes.cast(self._fn, ctypes.c_void_p), None),
               "plhr_prec_callback")
        self._h = out
        self.n = n


class TPA:
    """Teter-Payne-Allan preconditioner (Section 5.3) on the grid of A:
    T = S diag(K(mu / energy)) S^T over the grid's kinetic modes; energy <= 0
    takes sigma - min(potential) (or the mean kinetic energy)."""

    def __init__(self, A: Operator, sigma: float, energy: float = 0.0):
        lib = load_library()
        out = ctypes.c_void_p()
        _check(lib.plhr_prec_tpa(ctypes.byref(out), A._h, sigma, energy), "plhr_prec_tpa")
        self._h = out
        self.n = A.n
        self.sigma = sigma
        self.energy = lib.plhr_prec_tpa_energy(out)

    def apply(self, R, out=None, stream=None):
        import torch
        _check_block(R, self.n, "R")
        if out is None:
            out = torch.empty_like(R)
        _check_block(out, self.n, "out")
        _check(load_library().plhr_prec_apply(self._h, R.shape[1], ctypes.c_void_p(R.data_ptr()), R.stride(0),
                                              ctypes.c_void_p(out.data_ptr()), out.stride(0), _stream_ptr(stream)),
               "plhr_prec_apply")
        return out

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.plhr_prec_destroy(self._h)
            self._h = None


def tharm_extract(Gzz, Guq, Gqz, colscale, kp, nv, stream=None, clocks=False):
    """Device T-harmonic extraction step (see include/plhr.h) on torch CUDA
    float64 m x m Grams.  Returns dict with Cp (m x kp), Cvv (nv x kp), tags,
    partner, xi (units x 2), status, and optional stage clocks."""
    import torch
    lib = load_library()
    m = Gzz.shape[0]
    dev = Gzz.device
    Cp = torch.zeros((m, kp), dtype=torch.float64, device=dev)
    Cvv = torch.zeros((nv, kp), dtype=torch.float64, device=dev)
    tags = torch.zeros(kp, dtype=torch.int32, device=dev)
    partner = torch.zeros(kp, dtype=torch.int32, device=dev)
    xi = torch.zeros(2 * kp, dtype=torch.float64, device=dev)
    status = torch.zeros(3, dtype=torch.int32, device=dev)
    clk = torch.zeros(16, dtype=torch.int64, device=dev) if clocks else None
    args = [Gzz, Guq, Gqz, colscale, Cp, Cvv, tags, partner, xi, status]
    ptrs = [ctypes.c_void_p(t.contiguous().data_ptr()) for t in args]
    _check(lib.plhr_tharm_extract(m, kp, nv, *ptrs, ctypes.c_void_p(clk.data_ptr()) if clk is not None else None,
                                  _stream_ptr(stream)), "plhr_tharm_extract")
    torch.cuda.synchronize()
    st = status.cpu().numpy()
    out = {"Cp": Cp.cpu().numpy(), "Cvv": Cvv.cpu().numpy(), "tags": tags.cpu().numpy(),
           "partner": partner.cpu().numpy(), "xi": xi.cpu().numpy()[: 2 * int(st[2])].reshape(-1, 2),
           "status": int(st[0]), "kept": int(st[1]), "units": int(st[2])}
    if clk is not None:
        out["clocks"] = clk.cpu().numpy()
    return out


PHASES = ("stencil", "preconditioner", "gram", "update", "dense", "residual", "preconditioner_f32", "gram_f32",
          "update_f32")


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load_library().plhr_kernel_launches())


def profile_enable(on: bool = True) -> None:
    load_library().plhr_profile_enable(1 if on else 0)


def profile_read(reset: bool = False) -> dict:
    """Accumulated CUDA-event time (ms) and calls per solver phase."""
    ms = (ctypes.c_double * len(PHASES))()
    calls = (ctypes.c_longlong * len(PHASES))()
    work = (ctypes.c_double * len(PHASES))()
    nbytes = (ctypes.c_double * len(PHASES))()
    lib = load_library()
    lib.plhr_profile_work(work)
    lib.plhr_profile_bytes(nbytes)
    lib.plhr_profile_read(ms, calls, 1 if reset else 0)
    return {name: {"ms": ms[i], "calls": calls[i], "work": work[i], "bytes": nbytes[i]}
            for i, name in enumerate(PHASES)}


def gram(form, Z, AZ, Q=None, sigma=0.0, colscale=None, stream=None):
    """The three projected Grams [Z^T Z, U^T Q, Q^T Z] (U = AZ - sigma Z,
    columns scaled by colscale) in one of the library's arithmetic forms
    (GRAM_F64 / GRAM_DW on float64 blocks, GRAM_F32 / GRAM_F32_TC on float32
    blocks).  Z, AZ, Q: a CUDA tensor (n x m) or a list of up to 4 column
    blocks.  Returns a (3, m, m) float64 CUDA tensor."""
    import torch
    lib = load_library()
    zs = list(Z) if isinstance(Z, (list, tuple)) else [Z]
    az = list(AZ) if isinstance(AZ, (list, tuple)) else [AZ]
    qs = None if Q is None else (list(Q) if isinstance(Q, (list, tuple)) else [Q])
    nb = len(zs)
    dt = torch.float64 if form in (GRAM_F64, GRAM_DW) else torch.float32
    n = zs[0].shape[0]
    for X in zs + az + (qs or []):
        if not X.is_cuda or X.dtype != dt or X.dim() != 2 or X.shape[0] != n or X.stride(1) != 1:
            raise ValueError("gram blocks must be row-major %s CUDA tensors with n rows" % dt)
    m = sum(X.shape[1] for X in zs)
    dev = zs[0].device
    if colscale is None:
        colscale = torch.ones(m, dtype=torch.float64, device=dev)
    out = torch.empty((3, m, m), dtype=torch.float64, device=dev)
    ncols = (ctypes.c_int * nb)(*[X.shape[1] for X in zs])
    P = lambda L: (ctypes.c_void_p * nb)(*[X.data_ptr() for X in L])
    LD = lambda L: (ctypes.c_int64 * nb)(*[X.stride(0) for X in L])
    _check(lib.plhr_gram(form, n, nb, ncols, P(zs), LD(zs), P(az), LD(az), P(qs) if qs else None,
                         LD(qs) if qs else None, sigma, ctypes.c_void_p(colscale.data_ptr()),
                         ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "plhr_gram")
    return out


def solve(A: Operator, sigma: float, k: int, T: AVMG | None = None, tol: float = 1e-8, maxit: int = 1000,
          v_init=None, seed: int = 20140801, history: bool = False, precision: int = PRECISION_F64,
          stream=None, raise_on_notconv: bool = False, guard: int = 1, switch_tol: float = 1e-6,
          extraction: str = "tharm", s_vectors: bool = True, B: Operator | None = None,
          tensor_cores: bool = True):
    """k eigenpairs of A v = lambda v nearest sigma with k + guard block
    columns (B: the generalized problem A v = lambda B v, FP64 form).
    extraction "tharm" (T-harmonic, default) or "harm" (harmonic:
    T = I in the Petrov-Galerkin condition); s_vectors False drops the S block
    (trial space [V W P]); extraction "refined" is the single-vector
    method with the refinement of Eq. rRR (k = 1, guard = 0).  Returns
    (eigvals (numpy, k), eigvecs (torch n x k
    float64, CUDA), info dict)."""
    import torch
    lib = load_library()
    n = A.n
    kp = k + guard
    opt = Options()
    lib.plhr_options_default(ctypes.byref(opt))
    opt.maxit = maxit
    opt.precision = precision
    opt.seed = seed
    opt.guard = guard
    opt.switch_tol = switch_tol
    if extraction not in ("tharm", "harm", "refined"):
        raise ValueError("extraction must be 'tharm', 'harm' or 'refined'")
    opt.extraction = {"tharm": 0, "harm": 1, "refined": 2}[extraction]
    opt.s_vectors = 1 if s_vectors else 0
    opt.tensor_cores = 1 if tensor_cores else 0
    if v_init is not None:
        _check_block(v_init, n, "v_init")
        if v_init.shape[1] < kp:
            raise ValueError("v_init needs k + guard columns")
        opt.v_init = v_init.data_ptr()
        opt.ld_init = v_init.stride(0)
    hist = None
    rl = 2 * kp + 3
    if history:
        hist = np.zeros((maxit + 2) * rl, dtype=np.float64)
        opt.history = hist.ctypes.data
        opt.history_cap = maxit + 2
    vals = np.zeros(k, dtype=np.float64)
    vecs = torch.empty((n, k), dtype=torch.float64, device="cuda")
    info = Info()
    st = lib.plhr_solve(A._h, B._h if B is not None else None, sigma, k, T._h if T is not None else None, tol, ctypes.byref(opt),
                        vals.ctypes.data, ctypes.c_void_p(vecs.data_ptr()), k, ctypes.byref(info),
                        _stream_ptr(stream))
    if st not in (PLHR_OK, PLHR_ENOTCONV) or (raise_on_notconv and st == PLHR_ENOTCONV):
        raise PlhrError(st, "plhr_solve")
    out = {"status": st, "iterations": info.iterations, "converged": bool(info.converged),
           "max_rel_residual": info.max_rel_residual, "setup_seconds": info.setup_seconds,
           "solve_seconds": info.solve_seconds, "mixed_iterations": info.mixed_iterations}
    if hist is not None:
        rec = hist[: info.history_len * rl].reshape(info.history_len, rl)
        out["history"] = [{"it": int(r[0]), "lam": r[1:1 + k].copy(), "rel": r[1 + kp:1 + kp + k].copy(),
                           "lam_all": r[1:1 + kp].copy(), "rel_all": r[1 + kp:1 + 2 * kp].copy(),
                           "kept": int(r[1 + 2 * kp]), "m": int(r[2 + 2 * kp])} for r in rec]
    return vals, vecs, out


def eigval_grad(vecs, weights, stream=None):
    """g = sum_k w_k v_k^2 (device): the gradient of sum_k w_k lambda_k with
    respect to the potential of a Hamiltonian, for B-orthonormal eigenvectors
    vecs (n x k float64 CUDA)."""
    import torch
    if vecs.dtype != torch.float64 or not vecs.is_cuda or vecs.dim() != 2 or vecs.stride(1) != 1:
        raise ValueError("vecs must be a row-major float64 CUDA block")
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).ravel())
    if w.size != vecs.shape[1]:
        raise ValueError("one weight per eigenvector")
    g = torch.empty(vecs.shape[0], dtype=torch.float64, device=vecs.device)
    _check(load_library().plhr_eigval_grad(vecs.shape[0], vecs.shape[1], ctypes.c_void_p(vecs.data_ptr()),
                                           vecs.stride(0), w.ctypes.data, ctypes.c_void_p(g.data_ptr()),
                                           _stream_ptr(stream)), "plhr_eigval_grad")
    return g


def eigvec_adjoint(op, lam, vecs, G, tol=1e-12, maxit=None, T=None, stream=None, return_iterations=False):
    """dL/dV (device, n) of a loss L on the orthonormal eigenvectors vecs
    (n x k float64 CUDA, eigenvalues lam) of a Hamiltonian operator, given
    G = dL/dvecs (n x k float64 CUDA): first-order perturbation theory with
    the component outside the block from MINRES on P (H - lam_c) P,
    preconditioned by P T P when T (TPA or AV-MG) is given."""
    import torch
    for name, t in (("vecs", vecs), ("G", G)):
        if t.dtype != torch.float64 or not t.is_cuda or t.dim() != 2 or t.stride(1) != 1:
            raise ValueError(name + " must be a row-major float64 CUDA block")
    if G.shape != vecs.shape:
        raise ValueError("G must have the shape of vecs")
    lam = np.ascontiguousarray(np.asarray(lam, dtype=np.float64).ravel())
    if lam.size != vecs.shape[1]:
        raise ValueError("one eigenvalue per eigenvector")
    n = vecs.shape[0]
    if maxit is None:
        maxit = max(1000, min(20000, 2 * n))
    g = torch.empty(n, dtype=torch.float64, device=vecs.device)
    its = ctypes.c_int(0)
    _check(load_library().plhr_eigvec_adjoint(op._h, T._h if T is not None else None, vecs.shape[1], lam.ctypes.data,
                                              ctypes.c_void_p(vecs.data_ptr()),
                                              vecs.stride(0), ctypes.c_void_p(G.data_ptr()), G.stride(0), tol,
                                              int(maxit), ctypes.c_void_p(g.data_ptr()), ctypes.byref(its),
                                              _stream_ptr(stream)), "plhr_eigvec_adjoint")
    return (g, its.value) if return_iterations else g


def _hamiltonian_eig_class():
    import torch

    class HamiltonianEig(torch.autograd.Function):
        """lambda (k, float64 CUDA) = the k eigenvalues nearest sigma of
        H(V) = -1/2 Lap + diag(V); backward gives dL/dV = sum_k (dL/dlambda_k)
        v_k^2 on the device (Hellmann-Feynman)."""

        @staticmethod
        def forward(ctx, V, dims, h, periodic, sigma, k, tol, maxit, guard, T):
            op = Operator.hamiltonian(dims, h, V.detach().reshape(-1).contiguous(), periodic)
            lam, vecs, info = solve(op, sigma, k, T=T, tol=tol, maxit=maxit, guard=guard, raise_on_notconv=True)
            ctx.save_for_backward(vecs)
            ctx.vshape = V.shape
            return torch.from_numpy(lam).to(V.device)

        @staticmethod
        def backward(ctx, glam):
            (vecs,) = ctx.saved_tensors
            g = eigval_grad(vecs, glam.detach().cpu().numpy())
            return (g.reshape(ctx.vshape),) + (None,) * 9

    return HamiltonianEig


def _hamiltonian_eigh_class():
    import torch

    class HamiltonianEigh(torch.autograd.Function):
        """(lambda, vecs): the k eigenpairs nearest sigma of H(V) = -1/2 Lap +
        diag(V); backward gives dL/dV = sum_k (dL/dlambda_k) v_k^2 plus the
        eigenvector adjoint term of dL/dvecs, both on the device."""

        @staticmethod
        def forward(ctx, V, dims, h, periodic, sigma, k, tol, maxit, guard, prec, energy, adj_tol):
            Vf = V.detach().reshape(-1).contiguous()
            op = Operator.hamiltonian(dims, h, Vf, periodic)
            T = TPA(op, sigma, energy) if prec == "tpa" else None
            lam, vecs, info = solve(op, sigma, k, T=T, tol=tol, maxit=maxit, guard=guard, raise_on_notconv=True)
            ctx.save_for_backward(Vf, vecs)
            ctx.lam = lam
            ctx.meta = (V.shape, tuple(dims), h, periodic, sigma, prec, energy, adj_tol)
            return torch.from_numpy(lam).to(V.device), vecs

        @staticmethod
        def backward(ctx, glam, gvecs):
            Vf, vecs = ctx.saved_tensors
            vshape, dims, h, periodic, sigma, prec, energy, adj_tol = ctx.meta
            g = torch.zeros(Vf.shape[0], dtype=torch.float64, device=Vf.device)
            if glam is not None:
                g += eigval_grad(vecs, glam.detach().cpu().numpy())
            if gvecs is not None:
                op = Operator.hamiltonian(dims, h, Vf, periodic)
                T = TPA(op, sigma, energy) if prec == "tpa" else None
                g += eigvec_adjoint(op, ctx.lam, vecs, gvecs.detach().contiguous(), tol=adj_tol, T=T)
            return (g.reshape(vshape),) + (None,) * 11

    return HamiltonianEigh


def hamiltonian_eigh(V, dims, h, sigma, k, periodic=True, tol=1e-10, maxit=5000, guard=2, prec=None, energy=0.0,
                     adj_tol=1e-12):
    """Differentiable k eigenpairs (lambda, vecs) nearest sigma of
    H(V) = -1/2 Lap + diag(V); prec="tpa" preconditions the forward solve and
    the adjoint MINRES with the Teter-Payne-Allan T (energy <= 0: default).
    Losses on vecs should not depend on the sign of each eigenvector
    (densities, |v|^2 weights), which the solver does not fix."""
    if prec not in (None, "tpa"):
        raise ValueError("prec must be None or 'tpa'")
    return _hamiltonian_eigh_class().apply(V, tuple(dims), h, periodic, sigma, k, tol, maxit, guard, prec, energy,
                                           adj_tol)


def hamiltonian_eigvals(V, dims, h, sigma, k, periodic=True, tol=1e-10, maxit=5000, guard=2, T=None):
    """Differentiable k eigenvalues nearest sigma of H(V) = -1/2 Lap + diag(V)
    (V: float64 CUDA tensor with prod(dims) values, requires_grad allowed)."""
    return _hamiltonian_eig_class().apply(V, tuple(dims), h, periodic, sigma, k, tol, maxit, guard, T)
