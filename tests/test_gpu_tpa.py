"""GPU parity of the Teter-Payne-Allan preconditioner (Section 5.3) against
the oracle's FFT form, and its use in block PLHR and in the preconditioned
eigenvector adjoint on Hamiltonians.  The GPU transforms run in double-word
arithmetic (~2^-48 per operation over six passes of up to 64 terms), hence
1e-12 relative for the apply."""
import numpy as np
import pytest

import workloads as wl
from oracle import grad as og
from oracle import operators as oops
from oracle import spectral as osp

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


@pytest.mark.parametrize("dims,periodic,nc,energy", [((8, 6, 4), True, 3, 1.7), ((7, 6), True, 2, 0.9),
                                                     ((9, 5, 3), True, 4, 2.5), ((16, 12, 10), True, 5, 3.0),
                                                     ((64, 64, 64), True, 8, 2.2)])
def test_tpa_apply_matches_oracle_hamiltonian(plhr, dims, periodic, nc, energy):
    n = int(np.prod(dims))
    V = wl.uniform_block(n, 1, 61).ravel() * 2.0
    op = plhr.Operator.hamiltonian(dims, 0.8, torch.from_numpy(V).cuda(), periodic=periodic)
    T = plhr.TPA(op, 0.0, energy=energy)
    assert T.energy == energy
    X = wl.uniform_block(n, nc, 62)
    Y = T.apply(torch.from_numpy(X).cuda()).cpu().numpy()
    ref = osp.TPA(dims, 0.8, energy, periodic=periodic)(X)
    assert np.abs(Y - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dims", [(6, 5, 4), (10, 8)])
def test_tpa_apply_matches_oracle_dirichlet_laplacian(plhr, dims):
    """On the Dirichlet Laplacian (stencil scale 1) the modes are sines."""
    n = int(np.prod(dims))
    h = 1.0 / (dims[0] + 1)
    op = plhr.Operator.laplacian(dims, h)
    T = plhr.TPA(op, 0.0, energy=400.0)
    X = wl.uniform_block(n, 3, 63)
    Y = T.apply(torch.from_numpy(X).cuda()).cpu().numpy()
    ref = osp.TPA(dims, h, 400.0, periodic=False, scale=1.0)(X)
    assert np.abs(Y - ref).max() <= 1e-12 * np.abs(ref).max()


def test_tpa_default_energy_and_leading_dimension(plhr):
    p = wl.hamiltonian_small(8, 4)
    Vt = torch.from_numpy(p["V"]).cuda()
    op = plhr.Operator.hamiltonian(p["dims"], 1.0, Vt)
    sigma = -0.5
    T = plhr.TPA(op, sigma)
    assert T.energy == pytest.approx(osp.default_energy(sigma, p["V"], p["dims"], 1.0), rel=1e-15)
    T2 = plhr.TPA(op, p["V"].min() - 1.0)          # sigma below the potential: mean kinetic energy
    assert T2.energy == pytest.approx(3.0, rel=1e-15)
    X = torch.from_numpy(wl.uniform_block(512, 6, 64)).cuda()
    out = torch.zeros(512, 9, dtype=torch.float64, device="cuda")
    T.apply(X[:, :4], out=out[:, 2:6])            # strided input and output
    ref = osp.TPA(p["dims"], 1.0, T.energy)(X[:, :4].cpu().numpy())
    assert np.abs(out[:, 2:6].cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    assert float(out[:, :2].abs().max()) == 0.0 and float(out[:, 6:].abs().max()) == 0.0


def test_tpa_rejected_by_mixed_and_low_precision_forms(plhr):
    p = wl.hamiltonian_small(8, 4)
    op = plhr.Operator.hamiltonian(p["dims"], 1.0, torch.from_numpy(p["V"]).cuda())
    T = plhr.TPA(op, -0.5)
    with pytest.raises(plhr.PlhrError):
        T2 = plhr.TPA(op, -0.5)
        plhr.AVMG.apply_f32(T2, torch.zeros(512, 2, dtype=torch.float32, device="cuda"))
    A = plhr.Operator.laplacian((16, 16), 1.0 / 17)
    TL = plhr.TPA(A, 500.0)
    with pytest.raises(plhr.PlhrError):
        plhr.solve(A, 500.0, 2, T=TL, precision=plhr.PRECISION_MIXED)
    assert T.n == 512


def _hproblem(N=8, nwells=4, k=4, index=24):
    p = wl.hamiltonian_small(N, nwells, k=k)
    lam, Y = np.linalg.eigh(oops.hamiltonian(p["dims"], 1.0, p["V"]).toarray())
    best = None
    for i in range(index - 6, index + 6):
        sig = 0.5 * (lam[i] + lam[i + 1])
        d = np.abs(lam - sig)
        o = np.argsort(d)
        near = np.sort(o[:k])
        gaps = np.diff(lam[near[0] - 1:near[-1] + 2])
        score = min(gaps.min(), d[o[k]] - d[o[k - 1]])
        if best is None or score > best[0]:
            best = (score, sig, near)
    return p, best[1], lam, Y, best[2]


def test_solve_with_tpa_matches_dense_and_takes_fewer_iterations(plhr):
    p, sigma, lam, Y, near = _hproblem()
    op = plhr.Operator.hamiltonian(p["dims"], 1.0, torch.from_numpy(p["V"]).cuda())
    T = plhr.TPA(op, sigma)
    ev, vecs, info = plhr.solve(op, sigma, 4, T=T, tol=1e-11, maxit=6000, guard=2)
    assert info["converged"], info
    assert np.allclose(np.sort(ev), lam[near], rtol=1e-11)
    ev0, _, info0 = plhr.solve(op, sigma, 4, tol=1e-11, maxit=6000, guard=2)
    assert info0["converged"]
    assert info["iterations"] < info0["iterations"], (info["iterations"], info0["iterations"])


def test_preconditioned_adjoint_matches_dense_reference(plhr):
    p, sigma, lam, Y, near = _hproblem()
    op = plhr.Operator.hamiltonian(p["dims"], 1.0, torch.from_numpy(p["V"]).cuda())
    T = plhr.TPA(op, sigma)
    ev, vecs, info = plhr.solve(op, sigma, 4, T=T, tol=1e-12, maxit=6000, guard=2)
    assert info["converged"]
    m = wl.uniform_block(p["V"].size, 1, 65).ravel() ** 2 + 0.1
    G = 2.0 * m[:, None] * vecs.cpu().numpy()
    g1, it1 = plhr.eigvec_adjoint(op, ev, vecs, torch.from_numpy(G).cuda(), tol=1e-13, T=T, return_iterations=True)
    g0, it0 = plhr.eigvec_adjoint(op, ev, vecs, torch.from_numpy(G).cuda(), tol=1e-13, return_iterations=True)
    H = oops.hamiltonian(p["dims"], 1.0, p["V"]).toarray()
    ref, _, _ = og.eigvec_grad(H, list(near), 2.0 * m[:, None] * Y[:, near])
    for g in (g1, g0):
        assert np.abs(g.cpu().numpy() - ref).max() <= 1e-8 * np.abs(ref).max()
    assert it1 < it0, (it1, it0)


def test_eigh_autograd_with_tpa_32cube_matches_finite_differences(plhr):
    """32^3 periodic Hamiltonian (no dense reference at this size): the
    gradient of sum_k w_k lambda_k + sum_k |m (.) v_k|^2 through the
    TPA-preconditioned forward solve and adjoint against central differences
    of the same loss at sampled grid points."""
    p = wl.hamiltonian_small(32, 12, k=4)
    V = p["V"]
    import scipy.sparse.linalg as sla
    lam = np.sort(sla.eigsh(oops.hamiltonian(p["dims"], 1.0, V), k=30, which="SA", tol=1e-12)[0])
    # a shift whose 4 nearest eigenvalues are well inside a window with clean gaps
    best = None
    for i in range(2, 24):
        sig = 0.5 * (lam[i + 1] + lam[i + 2])
        d = np.abs(lam - sig)
        o = np.argsort(d)
        score = min(np.diff(lam[i - 1:i + 5]).min(), d[o[4]] - d[o[3]])
        if best is None or score > best[0]:
            best = (score, sig)
    sigma = best[1]
    w = np.array([0.7, 1.3, 0.9, 1.1])
    mask = (wl.uniform_block(V.size, 1, 66).ravel() >= 0).astype(np.float64)
    mt = torch.from_numpy(mask).cuda()
    wt = torch.from_numpy(w).cuda()

    def loss_of(Vn, grad=False):
        Vt = torch.from_numpy(Vn).cuda().requires_grad_(grad)
        ev, vecs = plhr.hamiltonian_eigh(Vt, p["dims"], 1.0, sigma, 4, tol=1e-12, maxit=4000, guard=2,
                                         prec="tpa")
        o = torch.argsort(ev.detach())
        L = (wt * ev[o]).sum() + ((mt[:, None] * vecs) ** 2).sum()
        if grad:
            L.backward()
            return float(L), Vt.grad.cpu().numpy()
        return float(L)

    L0, g = loss_of(V, grad=True)
    eps = 1e-4 * np.abs(V).max()
    rng = np.random.default_rng(12)
    for i in rng.choice(V.size, 4, replace=False):
        e = np.zeros_like(V); e[i] = eps
        fd = (loss_of(V + e) - loss_of(V - e)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-4 * abs(g[i]) + 1e-6 * np.abs(g).max(), (i, fd, g[i])
