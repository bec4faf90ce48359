"""GPU checks of the general operator and preconditioner entries of the C
ABI: CSR operators, the diagonal preconditioner and the callback
preconditioner, against scipy / dense LAPACK references and against the
built-in stencil operators they reproduce."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as wl
from oracle import operators as oops

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plhr():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1408_0042_gb300 as p
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return p


def _random_sym(n, density, seed):
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, format="csr")
    return ((M + M.T) * 0.5 + sp.diags(rng.uniform(2.0, 4.0, n))).tocsr()


@pytest.mark.parametrize("n,nc,ldpad", [(1, 1, 0), (37, 3, 2), (500, 5, 0), (4096, 8, 3)])
def test_csr_apply_matches_scipy(plhr, n, nc, ldpad):
    A = _random_sym(n, min(1.0, 8.0 / n), 70 + n)
    op = plhr.Operator.csr(A)
    assert op.n == n
    X = wl.uniform_block(n, nc + ldpad, 71)
    Xt = torch.from_numpy(X).cuda()[:, :nc]
    Y = op.apply(Xt).cpu().numpy()
    ref = A @ X[:, :nc]
    assert np.abs(Y - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max())


def test_csr_structure_checked_on_host(plhr):
    lib = plhr.load_library()
    import ctypes
    out = ctypes.c_void_p()
    rowptr = np.array([0, 1, 3], dtype=np.int64)
    bad_col = np.array([0, 1, 2], dtype=np.int32)        # column 2 in a 2 x 2 matrix
    val = np.ones(3)
    assert lib.plhr_op_csr(ctypes.byref(out), 2, rowptr.ctypes.data, bad_col.ctypes.data, val.ctypes.data, 0) == \
        plhr.PLHR_EINVAL
    bad_rp = np.array([0, 2, 1], dtype=np.int64)
    col = np.array([0, 1, 1], dtype=np.int32)
    assert lib.plhr_op_csr(ctypes.byref(out), 2, bad_rp.ctypes.data, col.ctypes.data, val.ctypes.data, 0) == \
        plhr.PLHR_EINVAL


def test_csr_hamiltonian_solve_equals_stencil_solve(plhr):
    p = wl.hamiltonian_small(8, 4, k=4)
    H = oops.hamiltonian(p["dims"], 1.0, p["V"])
    lam = np.linalg.eigvalsh(H.toarray())
    sigma = 0.5 * (lam[24] + lam[25])
    near = np.sort(np.argsort(np.abs(lam - sigma))[:4])
    opc = plhr.Operator.csr(H)
    ops_ = plhr.Operator.hamiltonian(p["dims"], 1.0, torch.from_numpy(p["V"]).cuda())
    ev_c, vec_c, info_c = plhr.solve(opc, sigma, 4, tol=1e-11, maxit=6000, guard=2)
    ev_s, vec_s, info_s = plhr.solve(ops_, sigma, 4, tol=1e-11, maxit=6000, guard=2)
    assert info_c["converged"] and info_s["converged"]
    assert np.allclose(np.sort(ev_c), lam[near], rtol=1e-11)
    assert np.allclose(np.sort(ev_s), np.sort(ev_c), rtol=1e-11)
    # eigenvector adjoint through the CSR operator equals the stencil one
    m = wl.uniform_block(H.shape[0], 1, 72).ravel() ** 2
    for op, ev, vec in ((opc, ev_c, vec_c), (ops_, ev_s, vec_s)):
        G = (2.0 * torch.from_numpy(m).cuda()[:, None] * vec).contiguous()
        g = plhr.eigvec_adjoint(op, ev, vec, G, tol=1e-13)
        if op is opc:
            g_c = g.cpu().numpy()
        else:
            assert np.abs(g.cpu().numpy() - g_c).max() <= 1e-8 * np.abs(g_c).max()


def test_fe_stiffness_csr_with_diagonal_preconditioner(plhr):
    """Q1 stiffness of the 2D FE problem (B = I here) as CSR, Jacobi-type
    diagonal T = diag(1 / |a_ii - sigma|... floored), against dense eigh."""
    A, _ = oops.q1_fe_2d(24)
    lam = np.linalg.eigvalsh(A.toarray())
    sigma = 0.5 * (lam[40] + lam[41])
    k = 4
    near = np.sort(np.argsort(np.abs(lam - sigma))[:k])
    op = plhr.Operator.csr(A)
    d = 1.0 / np.maximum(np.abs(A.diagonal() - sigma), 1e-3 * np.abs(A.diagonal()).max())
    T = plhr.DiagPrec(d)
    ev, vecs, info = plhr.solve(op, sigma, k, T=T, tol=1e-10, maxit=6000, guard=2)
    assert info["converged"], info
    assert np.allclose(np.sort(ev), lam[near], rtol=1e-10)
    V = vecs.cpu().numpy()
    assert np.abs(V.T @ V - np.eye(k)).max() <= 1e-12
    R = A @ V - V * ev[None, :]
    assert np.linalg.norm(R, axis=0).max() <= 1e-10 * max(1.0, np.abs(ev).max()) * 1.01


def test_callback_preconditioner_reproduces_diagonal(plhr):
    A, _ = oops.q1_fe_2d(24)
    lam = np.linalg.eigvalsh(A.toarray())
    sigma = 0.5 * (lam[40] + lam[41])
    op = plhr.Operator.csr(A)
    d = 1.0 / np.maximum(np.abs(A.diagonal() - sigma), 1e-3 * np.abs(A.diagonal()).max())
    dt = torch.from_numpy(d).cuda()
    calls = []

    def fn(R, W):
        calls.append(R.shape[1])
        W.copy_(dt[:, None] * R)

    Tc = plhr.CallbackPrec(A.shape[0], fn)
    Td = plhr.DiagPrec(torch.from_numpy(d).cuda())
    X = torch.from_numpy(wl.uniform_block(A.shape[0], 3, 73)).cuda()
    assert torch.equal(Tc.apply(X), Td.apply(X))
    ev_c, _, info_c = plhr.solve(op, sigma, 4, T=Tc, tol=1e-10, maxit=6000, guard=2)
    ev_d, _, info_d = plhr.solve(op, sigma, 4, T=Td, tol=1e-10, maxit=6000, guard=2)
    assert info_c["iterations"] == info_d["iterations"]
    assert np.array_equal(ev_c, ev_d)
    assert len(calls) > info_c["iterations"]

    def bad(R, W):
        raise RuntimeError("planted failure")

    Tb = plhr.CallbackPrec(A.shape[0], bad)
    with pytest.raises(plhr.PlhrError):
        plhr.solve(op, sigma, 4, T=Tb, tol=1e-10, maxit=50, guard=2)


def test_diagonal_preconditioner_rejects_nonpositive(plhr):
    with pytest.raises(plhr.PlhrError):
        plhr.DiagPrec(np.array([1.0, 0.0, 2.0]))
    with pytest.raises(plhr.PlhrError):
        plhr.DiagPrec(np.array([1.0, np.nan]))
    with pytest.raises(plhr.PlhrError):
        plhr.TPA(plhr.Operator.csr(sp.identity(8, format="csr")), 0.5)
