"""GPU parity: the CUDA path through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

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


def _padded(X, extra=3):
    """Copy of X (n x c) in a row-major buffer with leading dimension c + extra."""
    n, c = X.shape
    buf = torch.full((n, c + extra), float("nan"), dtype=torch.float64, device="cuda")
    buf[:, :c] = torch.from_numpy(X).cuda()
    return buf[:, :c]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("dims,nc", [((5, 7), 1), ((6, 5, 4), 3), ((33, 17, 9), 5), ((32, 32, 32), 11)])
def test_stencil_apply_matches_oracle(plhr, dims, nc):
    h = 1.0 / (max(dims) + 1)
    A = plhr.Operator.laplacian(dims, h)
    X = wl.uniform_block(A.n, nc, 123)
    Y = A.apply(_padded(X)).cpu().numpy()
    ref = oops.laplacian_dirichlet(dims, h) @ X
    assert _rel(Y, ref) <= 1e-14


@pytest.mark.parametrize("levels,sigma,transfer,coarse", [
    (1, 300.0, 0, 0), (2, 120.0, 0, 0), (3, 900.0, 0, 0), (3, 900.0, 1, 0), (3, 900.0, 1, 1),
    (3, 2500.0, 1, 1), (2, 60.0, 0, 1)])
def test_avmg_matches_oracle(plhr, levels, sigma, transfer, coarse):
    dims, h = (16, 16, 16), 1.0 / 17.0
    A = plhr.Operator.laplacian(dims, h)
    T = plhr.AVMG(A, sigma, levels=levels, nu=2, transfer=transfer, coarse=coarse)
    R = wl.uniform_block(A.n, 3, 7)
    W = T.apply(_padded(R)).cpu().numpy()
    ref = oavmg.AVMG(dims, h, sigma, levels, nu=2, transfer=["constant", "linear"][transfer],
                     coarse=["rediscretised", "fine_spectrum"][coarse])(R)
    assert _rel(W, ref) <= 1e-12


def test_avmg_2d_matches_oracle(plhr):
    dims, h, sigma = (32, 24), 1.0 / 33.0, 700.0
    A = plhr.Operator.laplacian(dims, h)
    T = plhr.AVMG(A, sigma, levels=3, nu=2)
    R = wl.uniform_block(A.n, 2, 8)
    W = T.apply(_padded(R)).cpu().numpy()
    ref = oavmg.AVMG(dims, h, sigma, 3, nu=2)(R)
    assert _rel(W, ref) <= 1e-12


def _independent_residuals(workload, lam, V):
    A, _ = oops.model_operator(workload)
    R = A @ V - V * lam[None, :]
    return np.linalg.norm(R, axis=0) / (np.maximum(np.abs(lam), 1.0) * np.linalg.norm(V, axis=0))


def _run_pair(plhr, w, maxit, track):
    A = plhr.Operator.laplacian(w.dims, w.h)
    T = None
    if w.prec == "avmg":
        T = plhr.AVMG(A, w.sigma, levels=w.mg_levels, nu=w.mg_nu,
                      transfer=1 if w.extra.get("transfer") == "linear" else 0,
                      coarse=1 if w.extra.get("coarse") == "fine_spectrum" else 0)
    v0 = torch.from_numpy(w.v0()).cuda()
    lam, V, info = plhr.solve(A, w.sigma, w.k, T=T, tol=w.tol, maxit=maxit, v_init=v0, history=True)
    ref = oplhr.solve_workload(w, maxit=maxit)
    return lam, V.cpu().numpy(), info, ref


@pytest.mark.parametrize("case", ["lap2d_T_identity", "lap3d_avmg"])
def test_solve_tracks_oracle_and_closed_form(plhr, case):
    if case == "lap2d_T_identity":
        w = wl.lap2d_small(16, k=4, gap_index=20)
        maxit = 2000
    else:
        w = wl.lap3d_small(16, levels=3, k=4, gap_index=40)
        maxit = 600
    lam, V, info, ref = _run_pair(plhr, w, maxit, True)
    assert info["converged"] and ref.converged
    # per-iteration Ritz values follow the oracle until rounding separates them
    hg, ho = info["history"], ref.history
    for a, b in list(zip(hg, ho))[:8]:
        assert np.allclose(a["lam"], b["lam"][: w.k], rtol=1e-9), (a["it"], a["lam"], b["lam"])
    # final eigenvalues: closed form and oracle
    cf = wl.lap_closed_form(w.dims, w.h)
    want = cf[np.lexsort((cf, np.abs(cf - w.sigma)))][: w.k]
    assert np.allclose(np.sort(lam), np.sort(want), rtol=1e-10)
    assert np.allclose(np.sort(lam), np.sort(ref.eigvals), rtol=1e-10)
    # residuals recomputed independently, B-orthonormality of the returned block
    res = _independent_residuals(w, lam, V)
    assert np.all(res <= w.tol * 1.0001), res
    assert np.abs(V.T @ V - np.eye(w.k)).max() <= 1e-12
    # subspace of the returned vectors equals the oracle's (angle)
    Q1, _ = np.linalg.qr(V)
    Q2, _ = np.linalg.qr(ref.eigvecs)
    s = np.linalg.svd(Q1.T @ Q2, compute_uv=False)
    assert np.sqrt(max(0.0, 1.0 - s.min() ** 2)) <= 1e-7


def test_lap2d_32x32_full(plhr):
    w = wl.lap2d_32x32_k4()
    A = plhr.Operator.laplacian(w.dims, w.h)
    v0 = torch.from_numpy(w.v0()).cuda()
    lam, V, info = plhr.solve(A, w.sigma, w.k, T=None, tol=w.tol, maxit=w.maxit, v_init=v0, guard=w.guard)
    assert info["converged"], info
    cf = wl.lap_closed_form(w.dims, w.h)
    want = cf[np.lexsort((cf, np.abs(cf - w.sigma)))][: w.k]
    assert np.allclose(np.sort(lam), np.sort(want), rtol=1e-10)
    res = _independent_residuals(w, lam, V.cpu().numpy())
    assert np.all(res <= w.tol * 1.0001)


def _extract_problem(seed, n=400, nv=5, nrest=15, generalized=False, complexish=False):
    """Realistic projected problem: Laplacian A, SPD preconditioner T, a trial
    basis Z = [V, rest] with uneven column scales."""
    rng = np.random.default_rng(seed)
    A = oops.laplacian_dirichlet((20, 20), 1 / 21).toarray()
    M = rng.standard_normal((n, n))
    T = np.linalg.inv(np.abs(np.linalg.eigvalsh(A)).max() * np.eye(n) * 0 + A + 50.0 * np.eye(n))
    T = 0.5 * (T + T.T) + 1e-4 * (M @ M.T) / n
    sigma = 300.0
    m = nv + nrest
    Z = rng.standard_normal((n, m)) * 10.0 ** rng.uniform(-3, 1, m)[None, :]
    cs = 10.0 ** rng.uniform(-1, 1, m)
    Zs = Z * cs[None, :]
    U = A @ Zs - sigma * Zs
    Q = T @ U
    return A, T, sigma, Z, cs, Zs, Zs.T @ Zs, U.T @ Q, Q.T @ Zs, nv


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_tharm_extract_matches_lapack(plhr, seed):
    """Device extraction (Cholesky basis, Hessenberg/Francis QR, selection)
    against LAPACK on the same projected pencil: selected xi values and the
    spans of the extracted blocks agree; the extracted vectors satisfy the
    T-harmonic Petrov-Galerkin condition (Eq. orth_gen)."""
    A, T, sigma, Z, cs, Zs, Gzz, Guq, Gqz, nv = _extract_problem(seed)
    kp = nv
    t = lambda X: torch.from_numpy(np.ascontiguousarray(X)).cuda()
    out = plhr.tharm_extract(t(Gzz), t(Guq), t(Gqz), t(cs), kp, nv, clocks=True)
    assert out["status"] == 0, out
    # reference: orthonormal basis, LAPACK eig through the oracle's routines
    Q0, R0 = np.linalg.qr(Zs)
    Zh = Q0
    U = A @ Zh - sigma * Zh
    GL = U.T @ T @ U
    GR = (T @ U).T @ Zh
    xi, Y = oplhr.tharmonic_extract(0.5 * (GL + GL.T), GR)
    Yp, tags, chosen = oplhr.select_real(xi, Y, kp)
    order, partner = oplhr.order_real_spectrum(xi)
    ref_units = []
    for i in order:
        if partner[i] < 0 or np.imag(xi[i]) > 0:
            ref_units.append(xi[i])
    got = out["xi"][:, 0] + 1j * out["xi"][:, 1]
    assert np.allclose(got, np.array(ref_units[: len(got)]), rtol=1e-9, atol=1e-12)
    # device coefficients on raw Z: V_new = Z_V C_VV + Z C_P
    Vd = Z[:, :nv] @ out["Cvv"] + Z @ out["Cp"]
    Vr = Zh @ Yp
    q1, _ = np.linalg.qr(Vd)
    q2, _ = np.linalg.qr(Vr)
    sv = np.linalg.svd(q1.T @ q2, compute_uv=False)
    assert sv.min() >= 1 - 1e-9
    # B-norm of the columns before RQ normalisation: unit for real columns
    nrm = np.linalg.norm(Vd, axis=0)
    for j, tg in enumerate(out["tags"]):
        if tg == 0:
            assert abs(nrm[j] - 1.0) <= 1e-9


def test_lap3d_128cube_full(plhr):
    """128^3 Laplacian, k = 10 nearest sigma, 4-level AV-MG: eigenvalues equal
    the closed-form ones, residuals (recomputed on the CPU) meet tol."""
    w = wl.lap3d_128cube_k10()
    A = plhr.Operator.laplacian(w.dims, w.h)
    T = plhr.AVMG(A, w.sigma, levels=w.mg_levels, nu=w.mg_nu, transfer=1, coarse=1)
    v0 = torch.from_numpy(w.v0()).cuda()
    lam, V, info = plhr.solve(A, w.sigma, w.k, T=T, tol=w.tol, maxit=w.maxit, v_init=v0, guard=w.guard)
    assert info["converged"], info
    cf = wl.lap_closed_form(w.dims, w.h)
    want = cf[np.lexsort((cf, np.abs(cf - w.sigma)))][: w.k]
    assert np.allclose(np.sort(lam), np.sort(want), rtol=1e-10)
    Vn = V.cpu().numpy()
    res = _independent_residuals(w, lam, Vn)
    assert np.all(res <= w.tol * 1.0001), res
    assert np.abs(Vn.T @ Vn - np.eye(w.k)).max() <= 1e-12


@pytest.mark.parametrize("variant", [{"extraction": "harm"}, {"s_vectors": False},
                                     {"extraction": "harm", "s_vectors": False}])
def test_ablation_variants_track_oracle(plhr, variant):
    """The ablations of Section 5.1 (harmonic instead of T-harmonic extraction;
    no S block) follow the oracle's iteration with the same options; the
    harmonic variant converges to eigenpairs of the closed form (the variants
    without S stall, as the oracle's pin shows)."""
    w = wl.lap3d_small(16, levels=3, k=4, gap_index=40)
    A = plhr.Operator.laplacian(w.dims, w.h)
    T = plhr.AVMG(A, w.sigma, levels=w.mg_levels, nu=w.mg_nu,
                  transfer=1 if w.extra.get("transfer") == "linear" else 0,
                  coarse=1 if w.extra.get("coarse") == "fine_spectrum" else 0)
    v0 = torch.from_numpy(w.v0()).cuda()
    stalls = variant.get("s_vectors", True) is False
    maxit = 12 if stalls else 1500
    lam, V, info = plhr.solve(A, w.sigma, w.k, T=T, tol=w.tol, maxit=maxit, v_init=v0, history=True, **variant)
    ref = oplhr.solve_workload(w, maxit=8, **variant)     # the first iterations, for tracking
    for a, b in list(zip(info["history"], ref.history))[:6]:
        assert np.allclose(a["lam"], b["lam"][: w.k], rtol=1e-9), (a["it"], a["lam"], b["lam"])
    if stalls:
        return
    assert info["converged"]
    # every returned pair is an eigenpair of the closed form (the harmonic
    # extraction is the less robust one: with one guard column it may settle
    # on a farther eigenvalue of a degenerate cluster's neighbourhood)
    cf = wl.lap_closed_form(w.dims, w.h)
    for x in lam:
        assert np.min(np.abs(cf - x)) <= 1e-10 * abs(x)
    res = _independent_residuals(w, lam, V.cpu().numpy())
    assert np.all(res <= w.tol * 1.0001), res


def test_ablation_variants_rejected_in_mixed_form(plhr):
    A = plhr.Operator.laplacian((16, 16), 1.0 / 17)
    for kw in ({"extraction": "harm"}, {"s_vectors": False}):
        with pytest.raises(plhr.PlhrError):
            plhr.solve(A, 500.0, 2, precision=plhr.PRECISION_MIXED, **kw)
