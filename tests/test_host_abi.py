"""Host logic of the C ABI, without a GPU: status strings, option defaults,
operator descriptors and sizes, and the argument checks that return
PLHR_EINVAL before any device work (every call here fails validation or
touches no device memory, so no kernel is launched)."""
import ctypes
import math
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def p():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1408_0042_gb300 import build
    build.build()
    import paper_1408_0042_gb300 as plhr
    try:
        plhr.load_library()
    except OSError as e:          # CUDA runtime library missing on this host
        pytest.skip("cannot load libplhr.so here: %s" % e)
    return plhr


def _err(p):
    return p.load_library().plhr_last_error().decode()


def test_status_strings_cover_every_code(p):
    lib = p.load_library()
    texts = [lib.plhr_status_string(s).decode() for s in range(7)]
    assert texts[p.PLHR_OK] == "ok"
    assert len(set(texts)) == 7 and all(texts)
    assert lib.plhr_status_string(99).decode() == "unknown status"


def test_option_defaults(p):
    lib = p.load_library()
    o = p.Options()
    lib.plhr_options_default(ctypes.byref(o))
    assert (o.maxit, o.precision, o.real_arithmetic, o.s_vectors, o.soft_lock) == (1000, p.PRECISION_F64, 1, 1, 1)
    assert (o.guard, o.extraction, o.seed) == (1, 0, 20140801)
    assert o.switch_tol == 1e-6 and not o.v_init and not o.history
    g = p.MGOpts()
    lib.plhr_mg_opts_default(ctypes.byref(g))
    assert (g.levels, g.nu, g.transfer, g.coarse) == (1, 2, 0, 0)
    assert g.delta == pytest.approx(2 * math.pi / 10, rel=1e-15)


def _stencil(p, kind, dims, h=0.1, scale=1.0):
    lib = p.load_library()
    d = p.StencilDesc()
    d.kind = kind
    for i, v in enumerate(dims):
        d.dims[i] = v
    d.h = h
    d.scale = scale
    op = ctypes.c_void_p()
    st = lib.plhr_op_stencil(ctypes.byref(op), ctypes.byref(d))
    return st, op


def test_stencil_descriptors_and_sizes(p):
    lib = p.load_library()
    st, op = _stencil(p, p.LAP7_3D, (6, 5, 4))
    assert st == p.PLHR_OK and lib.plhr_op_size(op) == 120
    lib.plhr_op_destroy(op)
    st, op = _stencil(p, p.LAP5_2D, (7, 3, 1))
    assert st == p.PLHR_OK and lib.plhr_op_size(op) == 21
    lib.plhr_op_destroy(op)
    assert lib.plhr_op_size(None) == 0
    lib.plhr_op_destroy(None)


@pytest.mark.parametrize("kind,dims,h,scale,msg", [
    (7, (4, 4, 4), 0.1, 1.0, "unknown kind"),
    (2, (0, 4, 4), 0.1, 1.0, "bad dims"),
    (2, (4, 4, 4), 0.0, 1.0, "bad dims"),
    (2, (4, 4, 4), 0.1, -1.0, "scale must be positive"),
    (6, (4, 4, 4), 0.1, 1.0, "unknown kind"),
    (1, (4, 4, 2), 0.1, 1.0, "dims[2] == 1"),
])
def test_stencil_rejects_bad_descriptors(p, kind, dims, h, scale, msg):
    st, op = _stencil(p, kind, dims, h, scale)
    assert st == p.PLHR_EINVAL and not op.value
    assert msg in _err(p)


def test_new_stencil_kinds_descriptors(p):
    """Q1 stiffness / mass (interior nodes per axis), the Bloch Hamiltonian
    (needs its potential), periodic Laplacian, and the argument checks of
    the complex and paired products (no device work is enqueued)."""
    lib = p.load_library()
    for kind in (p.Q1_STIFF27, p.Q1_MASS27):
        st, op = _stencil(p, kind, (7, 5, 6), h=1.0 / 8)
        assert st == p.PLHR_OK and lib.plhr_op_size(op) == 210
        lib.plhr_op_destroy(op)
    st, op = _stencil(p, p.HAM7_BLOCH, (6, 6, 6), h=1.0)
    assert st == p.PLHR_EINVAL and "potential" in _err(p)
    d = p.StencilDesc()
    d.kind = p.LAP7_3D
    d.dims[:] = [4, 4, 4]
    d.h, d.scale, d.bc = 0.1, 1.0, 5
    op = ctypes.c_void_p()
    assert lib.plhr_op_stencil(ctypes.byref(op), ctypes.byref(d)) == p.PLHR_EINVAL
    assert "boundary condition" in _err(p)
    d.bc = p.BC_PERIODIC
    assert lib.plhr_op_stencil(ctypes.byref(op), ctypes.byref(d)) == p.PLHR_OK
    # a Bloch operator with kappa != 0 is complex: the real product refuses it
    buf = (ctypes.c_double * 512)()
    ptr = ctypes.cast(buf, ctypes.c_void_p)
    db = p.StencilDesc()
    db.kind = p.HAM7_BLOCH
    db.dims[:] = [4, 4, 4]
    db.h, db.scale = 1.0, 1.0
    db.bloch_k[:] = [0.1, 0.0, 0.0]
    db.field = ptr.value
    ob = ctypes.c_void_p()
    assert lib.plhr_op_stencil(ctypes.byref(ob), ctypes.byref(db)) == p.PLHR_OK
    assert lib.plhr_op_apply(ob, 1, ptr, 1, ptr, 1, None) == p.PLHR_EINVAL
    assert "complex" in _err(p)
    assert lib.plhr_op_apply_c128(ob, 2, ptr, 1, ptr, 2, None) == p.PLHR_EINVAL      # ldx < ncols
    assert lib.plhr_op_apply_c128(ob, 0, None, 0, None, 0, None) == p.PLHR_OK
    st, q = _stencil(p, p.Q1_MASS27, (3, 3, 3), h=0.25)
    assert lib.plhr_op_apply_pair(op, q, 1, ptr, 1, ptr, 1, ptr, 1, None) == p.PLHR_EINVAL   # sizes differ
    assert lib.plhr_op_apply_pair(ob, op, 1, ptr, 1, ptr, 1, ptr, 1, None) == p.PLHR_EINVAL  # complex
    for o in (op, ob, q):
        lib.plhr_op_destroy(o)


def test_stencil_rejects_null_arguments(p):
    lib = p.load_library()
    assert lib.plhr_op_stencil(None, None) == p.PLHR_EINVAL
    assert "null argument" in _err(p)


def test_hamiltonian_descriptor(p):
    lib = p.load_library()
    dims = (ctypes.c_int64 * 3)(8, 6, 4)
    op = ctypes.c_void_p()
    # the potential pointer is only stored here (it is read by the products)
    assert lib.plhr_op_hamiltonian(ctypes.byref(op), 3, dims, 1.0, 1, None) == p.PLHR_OK
    assert lib.plhr_op_size(op) == 192
    lib.plhr_op_destroy(op)
    assert lib.plhr_op_hamiltonian(ctypes.byref(op), 2, dims, 1.0, 0, None) == p.PLHR_OK
    assert lib.plhr_op_size(op) == 48
    lib.plhr_op_destroy(op)
    for d, h in ((4, 1.0), (1, 1.0), (3, 0.0), (3, float("nan"))):
        assert lib.plhr_op_hamiltonian(ctypes.byref(op), d, dims, h, 1, None) == p.PLHR_EINVAL
    bad = (ctypes.c_int64 * 3)(8, 0, 4)
    assert lib.plhr_op_hamiltonian(ctypes.byref(op), 3, bad, 1.0, 1, None) == p.PLHR_EINVAL
    assert "bad dims" in _err(p)


def test_operator_apply_checks_before_any_product(p):
    lib = p.load_library()
    st, op = _stencil(p, p.LAP7_3D, (4, 4, 4))
    buf = (ctypes.c_double * 64)()
    ptr = ctypes.cast(buf, ctypes.c_void_p)
    assert lib.plhr_op_apply(op, 2, ptr, 1, ptr, 2, None) == p.PLHR_EINVAL      # ldx < ncols
    assert lib.plhr_op_apply(op, 2, None, 2, ptr, 2, None) == p.PLHR_EINVAL     # X missing
    assert lib.plhr_op_apply(op, -1, ptr, 2, ptr, 2, None) == p.PLHR_EINVAL
    assert lib.plhr_op_apply(None, 1, ptr, 1, ptr, 1, None) == p.PLHR_EINVAL
    assert lib.plhr_op_apply(op, 0, None, 0, None, 0, None) == p.PLHR_OK         # nothing to do
    lib.plhr_op_destroy(op)


def test_avmg_option_and_grid_checks(p):
    lib = p.load_library()
    st, lap = _stencil(p, p.LAP7_3D, (12, 12, 12))
    T = ctypes.c_void_p()
    g = p.MGOpts()
    lib.plhr_mg_opts_default(ctypes.byref(g))
    for field, value in (("levels", 0), ("nu", 0), ("delta", 0.0), ("transfer", 2), ("coarse", 3)):
        h = p.MGOpts.from_buffer_copy(g)
        setattr(h, field, value)
        assert lib.plhr_prec_avmg(ctypes.byref(T), lap, 100.0, ctypes.byref(h)) == p.PLHR_EINVAL
        assert "bad options" in _err(p)
    assert lib.plhr_prec_avmg(ctypes.byref(T), lap, float("inf"), None) == p.PLHR_EINVAL
    h = p.MGOpts.from_buffer_copy(g)
    h.levels = 4                       # 12 is not divisible by 2^3
    assert lib.plhr_prec_avmg(ctypes.byref(T), lap, 100.0, ctypes.byref(h)) == p.PLHR_EINVAL
    assert "divisible" in _err(p)
    dims = (ctypes.c_int64 * 3)(8, 8, 8)
    ham = ctypes.c_void_p()
    lib.plhr_op_hamiltonian(ctypes.byref(ham), 3, dims, 1.0, 1, None)
    assert lib.plhr_prec_avmg(ctypes.byref(T), ham, 1.0, None) == p.PLHR_EINVAL
    assert "Dirichlet Laplacian" in _err(p)
    lib.plhr_op_destroy(ham)
    lib.plhr_op_destroy(lap)


def _solve(p, A, k, tol=1e-8, sigma=100.0, B=None, ldv=None, **opts):
    lib = p.load_library()
    o = p.Options()
    lib.plhr_options_default(ctypes.byref(o))
    for kk, v in opts.items():
        setattr(o, kk, v)
    ev = (ctypes.c_double * 64)()
    vecs = (ctypes.c_double * 64)()     # never reached: every call below fails validation
    info = p.Info()
    return lib.plhr_solve(A, B, sigma, k, None, tol, ctypes.byref(o), ctypes.cast(ev, ctypes.c_void_p),
                          ctypes.cast(vecs, ctypes.c_void_p), k if ldv is None else ldv, ctypes.byref(info), None)


def test_solve_rejects_invalid_problems_before_device_work(p):
    lib = p.load_library()
    st, A = _stencil(p, p.LAP7_3D, (8, 8, 8))
    st, A2 = _stencil(p, p.LAP7_3D, (4, 4, 4))
    st, tiny = _stencil(p, p.LAP5_2D, (2, 2, 1))
    E = p.PLHR_EINVAL
    assert _solve(p, None, 2) == E
    assert _solve(p, A, 0) == E                                     # k < 1
    assert _solve(p, A, 4, ldv=3) == E                              # ldv < k
    assert _solve(p, A, 2, tol=0.0) == E
    assert _solve(p, A, 2, sigma=float("nan")) == E
    assert _solve(p, A, 2, maxit=-1) == E
    assert "invalid argument" in _err(p)
    assert _solve(p, A, 2, B=A2) == E                               # B of another size
    assert _solve(p, A, 2, B=A, precision=p.PRECISION_MIXED) == E   # B != I only in FP64
    assert "B must have the size of A" in _err(p)
    assert _solve(p, A, 2, real_arithmetic=0) == E
    assert _solve(p, A, 2, extraction=2) == E
    assert _solve(p, A, 2, precision=7) == E
    assert _solve(p, A, 2, extraction=1, precision=p.PRECISION_MIXED) == E
    assert _solve(p, A, 2, s_vectors=0, precision=p.PRECISION_MIXED) == E
    assert _solve(p, A, 2, guard=-1) == E
    assert _solve(p, A, 14, guard=3) == E                           # 4 (k + guard) > 64
    assert "too large" in _err(p)
    assert _solve(p, tiny, 1) == E                                  # n = 4 < m = 8
    assert "too small" in _err(p)
    dims = (ctypes.c_int64 * 3)(8, 8, 8)
    ham = ctypes.c_void_p()
    lib.plhr_op_hamiltonian(ctypes.byref(ham), 3, dims, 1.0, 1, None)
    assert _solve(p, ham, 2, precision=p.PRECISION_MIXED) == E      # mixed form: plain Laplacian only
    assert "mixed-precision form" in _err(p)
    for op in (A, A2, tiny, ham):
        lib.plhr_op_destroy(op)
