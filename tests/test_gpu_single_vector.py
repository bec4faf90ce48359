"""The single-vector methods on the GPU, through the C ABI: Algorithm 1
(k = 1, no guard column: the T-harmonic extraction on [v w s p]) and the
refinement extraction of Section 3.3 (Eq. rRR, extraction = 2), against the
oracle's per-iteration values, the closed form, LAPACK for a generalized
pencil, and CPU-recomputed residuals."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import avmg as oavmg
from oracle import operators as oops
from oracle import plhr as oplhr

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


def _near_start(A, sigma, eps, seed):
    ev, U = np.linalg.eigh(A.toarray())
    j = int(np.argmin(np.abs(ev - sigma)))
    return U[:, j] + eps * np.random.default_rng(seed).standard_normal(A.shape[0]), ev[j]


@pytest.mark.parametrize("levels", [1, 2])
def test_plmr_tracks_oracle_and_converges(plhr, levels):
    w = wl.lap2d_small(16, k=4, gap_index=20)
    A, _ = oops.model_operator(w)
    v0, target = _near_start(A, w.sigma, 1e-2, 3)
    op = plhr.Operator.laplacian(w.dims, w.h)
    T = plhr.AVMG(op, w.sigma, levels=levels)
    lam, V, info = plhr.solve(op, w.sigma, 1, T=T, tol=1e-10, maxit=300, guard=0, extraction="refined",
                              v_init=torch.from_numpy(v0[:, None].copy()).cuda(), history=True)
    assert info["converged"], info
    ref = oplhr.plmr(A, None, oavmg.AVMG(w.dims, w.h, w.sigma, levels), v0, tol=1e-10, maxit=300)
    for a, b in list(zip(info["history"], ref.history))[:8]:
        assert a["lam"][0] == pytest.approx(b["lam"][0], rel=1e-9), (a["it"], a["lam"], b["lam"])
    assert lam[0] == pytest.approx(target, rel=1e-10)
    v = V.cpu().numpy()[:, 0]
    r = A @ v - lam[0] * v
    assert np.linalg.norm(r) / (max(abs(lam[0]), 1.0) * np.linalg.norm(v)) <= 1e-10 * 1.0001
    assert abs(v @ v - 1.0) <= 1e-12


def test_plmr_generalized_q1_pencil(plhr):
    """Refinement on A v = lambda B v with the Q1 stencils (E = 8, coefficient
    cubes), diagonal T, from a start near a LAPACK eigenvector."""
    E = 8
    c = wl.q1_coefficient(E, 2, wl.SEED_BASE + 4)
    A, Bm = oops.q1_fe_3d(E, c)
    lam, Y = sla.eigh(A.toarray(), Bm.toarray())
    j = 40
    v0 = Y[:, j] + 1e-3 * np.random.default_rng(5).standard_normal(A.shape[0]) * np.abs(Y[:, j]).max()
    opA = plhr.Operator.q1_stiffness(E, torch.from_numpy(c).cuda())
    opB = plhr.Operator.q1_mass(E)
    T = plhr.DiagPrec(1.0 / np.abs(A.diagonal() - lam[j] * Bm.diagonal()))
    ev, V, info = plhr.solve(opA, lam[j], 1, T=T, B=opB, tol=1e-10, maxit=2000, guard=0, extraction="refined",
                             v_init=torch.from_numpy(v0[:, None].copy()).cuda())
    assert info["converged"], info
    assert ev[0] == pytest.approx(lam[j], rel=1e-10)
    v = V.cpu().numpy()[:, 0]
    assert abs(v @ (Bm @ v) - 1.0) <= 1e-11


def test_single_vector_plhr_tracks_oracle(plhr):
    """Algorithm 1 = the block iteration with one column (k = 1, guard 0):
    the GPU's Ritz values follow the oracle's and reach the closed-form
    eigenvalue nearest sigma."""
    w = wl.lap2d_small(32, k=4, gap_index=60)
    A, _ = oops.model_operator(w)
    v0 = wl.start_block(A.shape[0], 1, 32)
    op = plhr.Operator.laplacian(w.dims, w.h)
    T = plhr.AVMG(op, w.sigma, levels=3, transfer=1, coarse=1)
    lam, V, info = plhr.solve(op, w.sigma, 1, T=T, tol=1e-10, maxit=500, guard=0,
                              v_init=torch.from_numpy(v0).cuda(), history=True)
    assert info["converged"], info
    To = oavmg.AVMG(w.dims, w.h, w.sigma, 3, 2, transfer="linear", coarse="fine_spectrum")
    ref = oplhr.bplhr(A, None, To, w.sigma, 1, v0, tol=1e-10, maxit=500)
    for a, b in list(zip(info["history"], ref.history))[:6]:
        assert a["lam"][0] == pytest.approx(b["lam"][0], rel=1e-9)
    cf = wl.lap_closed_form(w.dims, w.h)
    assert lam[0] == pytest.approx(cf[np.argmin(np.abs(cf - w.sigma))], rel=1e-10)


def test_refined_extraction_argument_checks(plhr):
    w = wl.lap2d_small(16, k=4, gap_index=20)
    op = plhr.Operator.laplacian(w.dims, w.h)
    with pytest.raises(plhr.PlhrError):
        plhr.solve(op, w.sigma, 2, guard=0, extraction="refined")          # k must be 1
    with pytest.raises(plhr.PlhrError):
        plhr.solve(op, w.sigma, 1, guard=1, extraction="refined")          # no guard column
