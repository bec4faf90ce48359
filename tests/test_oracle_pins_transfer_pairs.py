"""Pins of the oracle parts that the 128^3 workload depends on: the trilinear
cell-centred transfers, the "fine spectrum" coarsest operator, the V-cycle
built from them (Appendix A, Algorithm 4), and the conjugate-pair branch of
Algorithm 3 (Section 4.1, Eq. lambda_complex and the real block
V' = [V_0 V_R v~_R V_I]).  Each expected value comes from a construction that
shares no code with the oracle function it checks: brute-force loops over the
definition, LAPACK eigensolves of independently built matrices, or complex
arithmetic on the complex Ritz vectors.  CPU only."""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import avmg, operators, plhr


# ---------------------------------------------------------------- trilinear transfers

def _centre_weights_1d(N):
    """Brute force from the definition of cell-centred linear interpolation:
    fine cell i has its centre at (i + 1/2) h, coarse cell I at (2I + 1) h
    (h the fine width).  The interpolated value is the linear interpolant of
    the two coarse centres that bracket the fine centre; a coarse cell beyond
    the wall contributes zero."""
    Nc = N // 2
    W = np.zeros((N, Nc))
    for i in range(N):
        x = i + 0.5
        # coarse centres X_I = 2I + 1 that bracket x
        lo = math.floor((x - 1.0) / 2.0)
        for I in (lo, lo + 1):
            if 0 <= I < Nc:
                W[i, I] += 1.0 - abs(x - (2 * I + 1)) / 2.0
    return W


def _brute_restriction(dims):
    """R[(I,J,K), (i,j,k)] = prod_axes w(i, I) / 2^d from loops over the grids
    (x fastest in both orderings)."""
    ws = [_centre_weights_1d(N) for N in dims]
    cd = [N // 2 for N in dims]
    nf, nc = int(np.prod(dims)), int(np.prod(cd))
    R = np.zeros((nc, nf))
    for fi in itertools.product(*[range(N) for N in reversed(dims)]):
        f = fi[::-1]                      # (x, y, z)
        fidx = 0
        for a in reversed(range(len(dims))):
            fidx = fidx * dims[a] + f[a]
        for ci in itertools.product(*[range(N) for N in reversed(cd)]):
            c = ci[::-1]
            wgt = 1.0
            for a in range(len(dims)):
                wgt *= ws[a][f[a], c[a]]
            if wgt:
                cidx = 0
                for a in reversed(range(len(dims))):
                    cidx = cidx * cd[a] + c[a]
                R[cidx, fidx] += wgt / 2 ** len(dims)
    return R


@pytest.mark.parametrize("Nc", [2, 3, 6])
def test_linear_prolongation_weights_and_linear_reproduction(Nc):
    P = avmg.linear_prolongation_1d(Nc).toarray()
    assert np.array_equal(P, _centre_weights_1d(2 * Nc))
    # a field linear in the cell centres is reproduced on interior fine cells
    X = 2.0 * np.arange(Nc) + 1.0            # coarse centres (fine-width units)
    x = np.arange(2 * Nc) + 0.5              # fine centres
    a, b = 0.37, -1.9
    pf = P @ (a + b * X)
    assert np.allclose(pf[1:-1], (a + b * x)[1:-1], rtol=0, atol=1e-14)
    # next to a wall the missing coarse neighbour is zero: 3/4 of the nearest
    assert pf[0] == pytest.approx(0.75 * (a + b * X[0]), abs=1e-15)
    assert pf[-1] == pytest.approx(0.75 * (a + b * X[-1]), abs=1e-15)
    # row sums 1 inside, 3/4 at the walls; column sums 2 inside, 7/4 at the walls
    rs = P.sum(axis=1)
    assert np.allclose(rs[1:-1], 1.0) and np.allclose(rs[[0, -1]], 0.75)
    cs = P.sum(axis=0)
    if Nc > 2:
        assert np.allclose(cs[1:-1], 2.0)
    assert np.allclose(cs[[0, -1]], 1.75)


@pytest.mark.parametrize("dims", [(4, 6), (4, 6, 8), (6, 4, 2)])
def test_linear_restriction_equals_brute_force(dims):
    R = avmg.restriction(dims, "linear").toarray()
    assert np.allclose(R, _brute_restriction(dims), rtol=0, atol=1e-15)
    d = len(dims)
    nf = int(np.prod(dims))
    # R = P^T / 2^d: (2^d R x, y) = (x, P y) with P from the brute-force weights
    Pb = 2 ** d * _brute_restriction(dims).T
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(nf), rng.standard_normal(R.shape[0])
    assert abs(2 ** d * (R @ x) @ y - x @ (Pb @ y)) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)
    # R 1 = 1 on coarse cells away from every wall, (7/8) per wall-adjacent axis
    r1 = R @ np.ones(nf)
    cd = [N // 2 for N in dims]
    for ci in itertools.product(*[range(N) for N in reversed(cd)]):
        c = ci[::-1]
        cidx = 0
        for a in reversed(range(d)):
            cidx = cidx * cd[a] + c[a]
        expect = 1.0
        for a in range(d):
            if cd[a] == 1:
                expect *= 0.75            # both neighbours missing: (3/4 + 3/4) / 2
            elif c[a] in (0, cd[a] - 1):
                expect *= 7.0 / 8.0
        assert r1[cidx] == pytest.approx(expect, abs=1e-14)


# ---------------------------------------------------------------- fine-spectrum coarsest operator

def _cell_centred_dirichlet_1d(N0):
    """Second difference on N0 cells with the wall half a cell beyond the end
    centres (ghost value -u): tridiag(-1, 2, -1) with 3 in the corners.  Its
    eigenvectors are the cell-centred sine modes."""
    M = 2.0 * np.eye(N0) - np.eye(N0, k=1) - np.eye(N0, k=-1)
    M[0, 0] = M[-1, -1] = 3.0
    return M


@pytest.mark.parametrize("coarse,fine", [((4,), (16,)), ((4, 3), (16, 12)), ((2, 3, 4), (8, 12, 16))])
def test_fine_spectrum_operator_eigenpairs(coarse, fine):
    """Eigenvectors = the cell-centred sine modes (from LAPACK on the
    cell-centred Dirichlet matrix, distinct eigenvalues so unique up to sign);
    eigenvalue of mode m = the m-th smallest eigenvalue of the FINE 1D
    Laplacian (from LAPACK on the fine second difference), summed over axes."""
    h = 1.0 / (max(fine) + 1)
    L0 = avmg.fine_spectrum_operator(coarse, fine, h)
    assert np.abs(L0 - L0.T).max() <= 1e-12 * np.abs(L0).max()
    vecs, vals = [], []
    for N0, N in zip(coarse, fine):               # x, y, z
        _, S = np.linalg.eigh(_cell_centred_dirichlet_1d(N0))   # ascending = mode 1 .. N0
        vecs.append(S)
        mu_fine = np.linalg.eigvalsh(operators.second_difference_1d(N, h).toarray())
        vals.append(mu_fine[:N0])
    for modes in itertools.product(*[range(N0) for N0 in coarse]):
        u = vecs[-1][:, modes[-1]]
        for a in reversed(range(len(coarse) - 1)):
            u = np.kron(u, vecs[a][:, modes[a]])
        lam = sum(vals[a][modes[a]] for a in range(len(coarse)))
        assert np.allclose(L0 @ u, lam * u, rtol=0, atol=1e-9 * lam)
    # the modes are sin((p + 1/2) m pi / N0): check the LAPACK vectors are them
    for S, N0 in zip(vecs, coarse):
        for m in range(1, N0 + 1):
            s = np.sin((np.arange(N0) + 0.5) * m * np.pi / N0)
            s /= np.linalg.norm(s)
            assert abs(abs(s @ S[:, m - 1]) - 1.0) <= 1e-12


# ---------------------------------------------------------------- V-cycle with these options

def _dense(op, n):
    return np.column_stack([op(e) for e in np.eye(n)])


def _coarse_absinv(coarse_dims, fine_dims, h, sigma):
    """|L_0 - sigma I|^{-1} built from the independent eigenpairs above."""
    vecs, vals = [], []
    for N0, N in zip(coarse_dims, fine_dims):
        _, S = np.linalg.eigh(_cell_centred_dirichlet_1d(N0))
        vecs.append(S)
        vals.append(np.linalg.eigvalsh(operators.second_difference_1d(N, h).toarray())[:N0])
    S3 = vecs[-1]
    lam = vals[-1]
    for a in reversed(range(len(coarse_dims) - 1)):
        S3 = np.kron(S3, vecs[a])
        lam = (lam[:, None] + vals[a][None, :]).ravel()
    return S3 @ np.diag(1.0 / np.abs(lam - sigma)) @ S3.T


@pytest.mark.parametrize("sigma", [60.0, 700.0])
def test_two_level_vcycle_linear_fine_spectrum_algebraic_form(sigma):
    """Two-grid Algorithm 4 with the trilinear transfers and the fine-spectrum
    coarsest operator equals T = B^{-1}(I - E^{2nu}) + E^nu P T_c R E^nu,
    E = I - omega B, with P and R from the brute-force weights and T_c from
    the independent eigenpairs."""
    dims, h, nu = (4, 4, 6), 1.0 / 7.0, 2
    T = avmg.AVMG(dims, h, sigma, levels=2, nu=nu, transfer="linear", coarse="fine_spectrum")
    n = int(np.prod(dims))
    Td = _dense(T, n)
    fine = T.levels[1]
    B = _dense(fine.apply_B, n)
    om = 1.0 / fine.beta
    E = np.eye(n) - om * B
    En = np.linalg.matrix_power(E, nu)
    R = _brute_restriction(dims)
    P = 8.0 * R.T
    Tc = _coarse_absinv(tuple(N // 2 for N in dims), dims, h, sigma)
    ref = np.linalg.solve(B, np.eye(n) - En @ En) + En @ P @ Tc @ R @ En
    assert np.allclose(Td, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("levels,sigma", [(3, 60.0), (3, 700.0), (3, 1500.0)])
def test_vcycle_linear_fine_spectrum_symmetric_positive_definite(levels, sigma):
    dims, h = (8, 8, 8), 1.0 / 9.0
    T = avmg.AVMG(dims, h, sigma, levels=levels, transfer="linear", coarse="fine_spectrum")
    Td = _dense(T, 512)
    assert np.abs(Td - Td.T).max() <= 1e-12 * np.abs(Td).max()
    assert np.linalg.eigvalsh(0.5 * (Td + Td.T)).min() > 0


def test_fine_spectrum_single_level_is_exact_absolute_inverse():
    """levels = 1 with the fine-spectrum option: the coarsest grid is the fine
    grid, whose vertex-centred sine modes are not the cell-centred ones, but
    the eigenvalues must be the fine Laplacian's own: the spectrum of T^{-1}
    equals |lambda_i - sigma| over the closed-form FD spectrum."""
    dims, h, sigma = (4, 6), 1.0 / 7.0, 300.0
    T = avmg.AVMG(dims, h, sigma, levels=1, transfer="linear", coarse="fine_spectrum")
    Td = _dense(T, 24)
    ev = np.sort(1.0 / np.linalg.eigvalsh(0.5 * (Td + Td.T)))
    mu = [np.array([4.0 / h**2 * math.sin(m * math.pi / (2 * (N + 1))) ** 2 for m in range(1, N + 1)])
          for N in dims]
    ref = np.sort(np.abs((mu[0][None, :] + mu[1][:, None]).ravel() - sigma))
    assert np.allclose(ev, ref, rtol=1e-11)


# ---------------------------------------------------------------- conjugate pairs (Alg. 3)

def _pair_problem(seed=6, n=400, m=20, kp=5):
    """A projected T-harmonic problem whose kp smallest |xi| contain a
    complex conjugate pair (seed 6 of this recipe does)."""
    rng = np.random.default_rng(seed)
    A = operators.laplacian_dirichlet((20, 20), 1 / 21).toarray()
    M = rng.standard_normal((n, n))
    T = np.linalg.inv(A + 50.0 * np.eye(n))
    T = 0.5 * (T + T.T) + 1e-4 * (M @ M.T) / n
    sigma = 300.0
    Zh, _ = np.linalg.qr(rng.standard_normal((n, m)))
    U = A @ Zh - sigma * Zh
    Q = T @ U
    GL, GR = U.T @ Q, Q.T @ Zh
    return A, Zh, 0.5 * (GL + GL.T), GR, kp


def test_pair_rayleigh_quotient_is_complex_rayleigh_quotient():
    """Eq. lambda_complex: the value given to both columns of a pair equals
    v^* A v / v^* v for the complex Ritz vector v = v_R + i v_I."""
    A, Zh, GL, GR, kp = _pair_problem()
    xi, Y = plhr.tharmonic_extract(GL, GR)
    Yp, tags, chosen = plhr.select_real(xi, Y, kp)
    kinds = [t[0] for t in tags]
    assert "pairR" in kinds and "pairI" in kinds
    V = Zh @ Yp
    lam, b = plhr.rayleigh_quotients(V, A @ V, V, tags)
    jr, ji = kinds.index("pairR"), kinds.index("pairI")
    v = V[:, jr] + 1j * V[:, ji]
    rq = np.vdot(v, A @ v) / np.vdot(v, v)
    assert abs(rq.imag) <= 1e-12 * abs(rq)
    assert lam[jr] == pytest.approx(rq.real, rel=1e-13)
    assert lam[ji] == lam[jr]
    # not the mean of the two real quotients (the parts have unequal norms)
    own = [V[:, j] @ A @ V[:, j] / (V[:, j] @ V[:, j]) for j in (jr, ji)]
    assert abs(0.5 * (own[0] + own[1]) - rq.real) > 1e-8 * abs(rq)
    # real columns keep their own quotient
    for j, kd in enumerate(kinds):
        if kd == "real":
            assert lam[j] == pytest.approx(V[:, j] @ A @ V[:, j] / (V[:, j] @ V[:, j]), rel=1e-13)


def test_pair_columns_span_the_complex_ritz_vectors():
    """Section 4.1: the real block V' = [V_0 V_R V_I] spans, over C, the same
    space as the complex T-harmonic Ritz vectors Z y of the selected xi, and
    the pair's columns are the real and imaginary parts of Z y times a unit
    complex factor."""
    A, Zh, GL, GR, kp = _pair_problem()
    xi, Y = plhr.tharmonic_extract(GL, GR)
    Yp, tags, chosen = plhr.select_real(xi, Y, kp)
    V = Zh @ Yp
    Vc = Zh @ Y[:, chosen]
    q1, _ = np.linalg.qr(V.astype(np.complex128))
    q2, _ = np.linalg.qr(Vc)
    sv = np.linalg.svd(q1.conj().T @ q2, compute_uv=False)
    assert np.allclose(sv, 1.0, atol=1e-10)
    kinds = [t[0] for t in tags]
    jr, ji = kinds.index("pairR"), kinds.index("pairI")
    v = V[:, jr] + 1j * V[:, ji]
    ipos = [i for i in chosen if np.imag(xi[i]) > 0][0]
    w = Zh @ Y[:, ipos]
    assert abs(abs(np.vdot(v, w)) - np.linalg.norm(v) * np.linalg.norm(w)) <= 1e-12 * np.linalg.norm(v) * np.linalg.norm(w)
    # the Ritz vector's own eigen-equation in the projected pencil: G_L y = xi G_R y
    y = Y[:, ipos]
    assert np.linalg.norm(GL @ y - xi[ipos] * (GR @ y)) <= 1e-10 * np.linalg.norm(GL) * np.linalg.norm(y)


def test_solver_with_pairs_mid_solve_matches_closed_form_and_dense():
    """A 2D AV-MG case (trilinear transfers, fine-spectrum coarsest operator,
    3 levels) on which the extraction selects conjugate pairs in many
    iterations: Algorithm 3 still converges to the closed-form eigenvalues and
    to the same pairs as a dense solve, and the returned block is orthonormal."""
    w = wl.lap2d_small(32, k=4, gap_index=60)
    A, _ = operators.model_operator(w)
    T = avmg.AVMG(w.dims, w.h, w.sigma, 3, 2, transfer="linear", coarse="fine_spectrum")
    r = plhr.bplhr(A, None, T, w.sigma, w.k, w.v0(), tol=1e-10, maxit=500)
    assert r.converged
    npair = sum(1 for h in r.history if "pairR" in h.get("tags", ()))
    assert npair >= 5
    lam = wl.lap_closed_form(w.dims, w.h)
    ref = lam[np.lexsort((lam, np.abs(lam - w.sigma)))][: w.k]
    assert np.allclose(np.sort(r.eigvals), np.sort(ref), rtol=1e-10)
    ev = sla.eigh(A.toarray(), eigvals_only=True)
    ref2 = ev[np.lexsort((ev, np.abs(ev - w.sigma)))][: w.k]
    assert np.allclose(np.sort(r.eigvals), np.sort(ref2), rtol=1e-10)
    assert np.abs(r.eigvecs.T @ r.eigvecs - np.eye(w.k)).max() <= 1e-12


# ---------------------------------------------------------------- INV-MG (Algorithm 5)

def test_inv_mg_single_level_is_exact_inverse():
    """levels = 1: T = (L - sigma I)^{-1}, signed: on an analytic sine mode
    T u = u / (lambda - sigma)."""
    dims, h, sigma = (6, 5, 4), 1.0 / 7.0, 300.0
    T = avmg.AVMG(dims, h, sigma, levels=1, indefinite=True)
    signs = set()
    for modes in [(1, 1, 1), (2, 3, 1), (6, 5, 4), (3, 2, 2)]:
        vecs = [np.sin(np.arange(1, N + 1) * m * np.pi / (N + 1)) for N, m in zip(dims, modes)]
        u = vecs[2]
        for v in (vecs[1], vecs[0]):
            u = np.kron(u, v)
        lam = sum((2.0 - 2.0 * math.cos(m * math.pi / (N + 1))) / h**2 for N, m in zip(dims, modes))
        assert np.allclose(T(u), u / (lam - sigma), rtol=1e-10, atol=1e-14)
        signs.add(np.sign(lam - sigma))
    assert signs == {-1.0, 1.0}


@pytest.mark.parametrize("sigma", [60.0, 700.0])
def test_inv_mg_two_level_algebraic_form(sigma):
    """Two-grid Algorithm 5: T = S^{-1}(I - E^{2nu}) + E^nu P T_c R E^nu with
    S = L - sigma I, E = I - S / beta, beta the Gershgorin bound of |S|, P and
    R from the brute-force trilinear weights, T_c = (L_0 - sigma I)^{-1} from
    the independent eigenpairs (fine-spectrum coarse operator)."""
    dims, h, nu = (4, 4, 6), 1.0 / 7.0, 2
    T = avmg.AVMG(dims, h, sigma, levels=2, nu=nu, transfer="linear", coarse="fine_spectrum", indefinite=True)
    n = int(np.prod(dims))
    Td = _dense(T, n)
    S = operators.laplacian_dirichlet(dims, h).toarray() - sigma * np.eye(n)
    beta = max(sigma, 12.0 / h**2 - sigma)
    E = np.eye(n) - S / beta
    En = np.linalg.matrix_power(E, nu)
    R = _brute_restriction(dims)
    P = 8.0 * R.T
    cd = tuple(N // 2 for N in dims)
    vecs, vals = [], []
    for N0, N in zip(cd, dims):
        _, Sv = np.linalg.eigh(_cell_centred_dirichlet_1d(N0))
        vecs.append(Sv)
        vals.append(np.linalg.eigvalsh(operators.second_difference_1d(N, h).toarray())[:N0])
    S3, lam = vecs[-1], vals[-1]
    for a in reversed(range(len(cd) - 1)):
        S3 = np.kron(S3, vecs[a])
        lam = (lam[:, None] + vals[a][None, :]).ravel()
    Tc = S3 @ np.diag(1.0 / (lam - sigma)) @ S3.T
    ref = np.linalg.solve(S, np.eye(n) - En @ En) + En @ P @ Tc @ R @ En
    assert np.allclose(Td, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    # symmetric; indefinite when sigma lies inside the spectrum of L (max 12/h^2 = 588)
    assert np.abs(Td - Td.T).max() <= 1e-12 * np.abs(Td).max()
    ev = np.linalg.eigvalsh(0.5 * (Td + Td.T))
    if sigma < 12.0 / h**2:
        assert ev.min() < 0 < ev.max()


def test_bplhr_harmonic_with_inv_mg_matches_closed_form():
    """The paper's "BPLHR, Indef., harm." combination (Table tab:laplace10):
    harmonic extraction (T = I in the Petrov-Galerkin condition) with the
    indefinite INV-MG T converges to the closed-form eigenvalues."""
    w = wl.lap2d_small(32, k=4, gap_index=60)
    A, _ = operators.model_operator(w)
    T = avmg.AVMG(w.dims, w.h, w.sigma, 3, 2, transfer="linear", coarse="fine_spectrum", indefinite=True)
    r = plhr.bplhr(A, None, T, w.sigma, w.k, w.v0(), tol=1e-9, maxit=1500, extraction="harm")
    assert r.converged
    lam = wl.lap_closed_form(w.dims, w.h)
    ref = lam[np.lexsort((lam, np.abs(lam - w.sigma)))][: w.k]
    assert np.allclose(np.sort(r.eigvals), np.sort(ref), rtol=1e-9)
