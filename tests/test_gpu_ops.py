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


# ---------------------------------------------------------------- generalized problem A v = lambda B v

def _fe_pencil(elems):
    A, Bm = oops.q1_fe_2d(elems)
    import scipy.linalg as sl
    lam, Y = sl.eigh(A.toarray(), Bm.toarray())
    return A, Bm, lam, Y


@pytest.mark.parametrize("prec", ["none", "diag"])
def test_generalized_fe_matches_dense_and_is_b_orthonormal(plhr, prec):
    """Q1 stiffness A and mass B (Section 5.1) as CSR operators: the k pairs
    nearest sigma of A v = lambda B v against LAPACK's generalized eigh, with
    B-orthonormal vectors and residuals recomputed on the CPU."""
    A, Bm, lam, Y = _fe_pencil(20)
    sigma = 0.5 * (lam[30] + lam[31])
    k = 4
    near = np.sort(np.argsort(np.abs(lam - sigma))[:k])
    opA, opB = plhr.Operator.csr(A), plhr.Operator.csr(Bm)
    T = None
    if prec == "diag":
        T = plhr.DiagPrec(1.0 / np.abs(A.diagonal() - sigma * Bm.diagonal()))
    ev, vecs, info = plhr.solve(opA, sigma, k, T=T, B=opB, tol=1e-10, maxit=8000, guard=2)
    assert info["converged"], info
    assert np.allclose(np.sort(ev), lam[near], rtol=1e-10)
    V = vecs.cpu().numpy()
    assert np.abs(V.T @ (Bm @ V) - np.eye(k)).max() <= 1e-11
    R = A @ V - (Bm @ V) * ev[None, :]
    rel = np.linalg.norm(R, axis=0) / (np.maximum(np.abs(ev), 1.0) * np.linalg.norm(Bm @ V, axis=0))
    assert np.all(rel <= 1e-10 * 1.0001), rel


def test_generalized_tracks_oracle(plhr):
    """Per-iteration Ritz values of the generalized T-harmonic iteration equal
    the oracle's (Algorithm 3 with B) for the first iterations, on the same
    start block, with the exact shifted-inverse preconditioner of the oracle's
    pin perturbed to stay generic."""
    from oracle import plhr as oplhr
    A, Bm, lam, Y = _fe_pencil(12)
    Ad, Bd = A.toarray(), Bm.toarray()
    n = Ad.shape[0]
    sigma = 0.5 * (lam[15] + lam[16])
    k, guard = 3, 1
    # T = |A - sigma B|^{-1} (symmetric, from the eigendecomposition of A - sigma B) + 0.1 I / ||...||
    w, Q = np.linalg.eigh(Ad - sigma * Bd)
    Tm = (Q / np.abs(w)[None, :]) @ Q.T
    Tm = Tm + 0.05 * np.abs(Tm).max() * np.eye(n)
    Tt = torch.from_numpy(Tm).cuda()

    def fn(R, Wout):
        Wout.copy_(Tt @ R)

    Tc = plhr.CallbackPrec(n, fn)
    V0 = wl.uniform_block(n, k + guard, 81)
    ev, vecs, info = plhr.solve(plhr.Operator.csr(A), sigma, k, T=Tc, B=plhr.Operator.csr(Bm), tol=1e-10,
                                maxit=300, guard=guard, v_init=torch.from_numpy(V0).cuda(), history=True)
    ref = oplhr.bplhr(A, Bm, lambda Xb: Tm @ Xb, sigma, k, V0, tol=1e-10, maxit=8)
    for a, b in list(zip(info["history"], ref.history))[:6]:
        assert np.allclose(a["lam"], b["lam"][:k], rtol=1e-9), (a["it"], a["lam"], b["lam"])


def test_generalized_fe_50x50_reproduces_printed_eigenvalues(plhr):
    """The paper's Section 5.1 FE problem (50 x 50 elements, n = 2401): the
    eigenvalues nearest the shifts 497 and 980 are the printed lambda_31 and
    lambda_66 (tests/golden/fe_q1_50x50.json, 4 decimals)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "fe_q1_50x50.json")) as f:
        gold = json.load(f)
    A, Bm = oops.q1_fe_2d(gold["elements_per_side"])
    opA, opB = plhr.Operator.csr(A), plhr.Operator.csr(Bm)
    for shift, key in ((497.0, "31"), (980.0, "66")):
        ev, vecs, info = plhr.solve(opA, shift, 1, B=opB, tol=1e-10, maxit=20000, guard=3)
        assert info["converged"], info
        assert abs(ev[0] - gold["eigenvalues_1based"][key]) <= 0.5e-4 * 1.0001, (key, ev[0])


def test_generalized_rejected_in_mixed_form(plhr):
    A, Bm = oops.q1_fe_2d(8)
    with pytest.raises(plhr.PlhrError):
        plhr.solve(plhr.Operator.csr(A), 100.0, 2, B=plhr.Operator.csr(Bm), precision=plhr.PRECISION_MIXED)
