"""Pins of the oracle's single-vector methods: Algorithm 1 (PLHR with one
vector, the T-harmonic extraction on the 4-dimensional trial space
[v w s p]) and the refinement extraction of Section 3.3 (Eq. rRR, the
preconditioned locally minimal residual method).  CPU only."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import avmg, operators, plhr


def _sqrtm_spd(M):
    w, Q = np.linalg.eigh(0.5 * (M + M.T))
    return (Q * np.sqrt(w)[None, :]) @ Q.T


@pytest.mark.parametrize("generalized", [False, True])
def test_refined_coefficients_minimise_the_t_norm_residual(generalized):
    """Eq. rRR by a different route: with T^{1/2} and B^{1/2} from dense
    eigendecompositions, the minimiser of ||T^{1/2} X y|| / ||B^{1/2} Z y|| is
    the right singular vector of the smallest singular value of
    T^{1/2} X N^{-1} (N from the QR of B^{1/2} Z), mapped back by N^{-1}."""
    rng = np.random.default_rng(11)
    if generalized:
        A, Bm = operators.q1_fe_2d(9)
        A, Bm = A.toarray(), Bm.toarray()
    else:
        A = operators.laplacian_dirichlet((8, 8), 1 / 9).toarray()
        Bm = np.eye(64)
    n = A.shape[0]
    M = rng.standard_normal((n, n))
    Tm = M @ M.T / n + np.eye(n)
    Z = rng.standard_normal((n, 4))
    lam_t = 310.0
    y = plhr.refined_coefficients(Z, A @ Z, Bm @ Z, lam_t, lambda X: Tm @ X)
    y = y[:, 0]
    X = A @ Z - lam_t * (Bm @ Z)
    Qb, N = np.linalg.qr(_sqrtm_spd(Bm) @ Z)
    _, sv, Vh = np.linalg.svd(_sqrtm_spd(Tm) @ X @ np.linalg.inv(N))
    yref = np.linalg.solve(N, Vh[-1])
    cos = abs(y @ (Z.T @ Bm @ Z) @ yref) / np.sqrt((y @ Z.T @ Bm @ Z @ y) * (yref @ Z.T @ Bm @ Z @ yref))
    assert cos == pytest.approx(1.0, abs=1e-10)
    # the minimum value is the smallest singular value
    val = np.sqrt((X @ y) @ Tm @ (X @ y) / ((Z @ y) @ Bm @ (Z @ y)))
    assert val == pytest.approx(sv[-1], rel=1e-10)


@pytest.mark.parametrize("eps", [1e-3, 1e-2])
def test_plmr_converges_from_a_close_start(eps):
    """Started near an eigenvector, PLMR converges to that eigenpair (the
    closed-form value) with the exact absolute-value preconditioner and with
    a two-level V-cycle."""
    w = wl.lap2d_small(16, k=4, gap_index=20)
    A, _ = operators.model_operator(w)
    ev, U = np.linalg.eigh(A.toarray())
    j = int(np.argmin(np.abs(ev - w.sigma)))
    v0 = U[:, j] + eps * np.random.default_rng(1).standard_normal(A.shape[0])
    lam = wl.lap_closed_form(w.dims, w.h)
    target = lam[np.argmin(np.abs(lam - ev[j]))]
    for levels in (1, 2):
        T = avmg.AVMG(w.dims, w.h, w.sigma, levels)
        r = plhr.plmr(A, None, T, v0, tol=1e-10, maxit=200)
        assert r.converged
        assert r.eigvals[0] == pytest.approx(target, rel=1e-10)
        assert r.residuals[0] <= 1e-10


def test_single_vector_plhr_is_algorithm_1():
    """bplhr with one column: T = I, B = I gives real xi, so real arithmetic
    (Algorithm 3 with k' = 1) equals complex arithmetic (Algorithm 1) step by
    step; with AV-MG it converges to the closed-form eigenvalue nearest sigma."""
    w = wl.lap2d_small(12, k=3, gap_index=12)
    A, _ = operators.model_operator(w)
    v0 = wl.start_block(A.shape[0], 1, 31)
    hr = plhr.bplhr(A, None, None, w.sigma, 1, v0, tol=1e-14, maxit=10).history
    hc = plhr.bplhr(A, None, None, w.sigma, 1, v0.astype(np.complex128), tol=1e-14, maxit=10, real=False).history
    for a, b in zip(hr, hc):
        assert np.allclose(a["lam"], b["lam"], rtol=1e-9)
    w2 = wl.lap2d_small(32, k=4, gap_index=60)
    A2, _ = operators.model_operator(w2)
    T = avmg.AVMG(w2.dims, w2.h, w2.sigma, 3, 2, transfer="linear", coarse="fine_spectrum")
    r = plhr.bplhr(A2, None, T, w2.sigma, 1, wl.start_block(A2.shape[0], 1, 32), tol=1e-10, maxit=500)
    assert r.converged
    lam = wl.lap_closed_form(w2.dims, w2.h)
    assert r.eigvals[0] == pytest.approx(lam[np.argmin(np.abs(lam - w2.sigma))], rel=1e-10)
