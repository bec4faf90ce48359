"""GPU parity of the 27-point trilinear (Q1) finite-element stencils (Section
5.1's elements in 3D: stiffness of -div(c grad) with a coefficient per element,
and the mass matrix) and of the complex Bloch Hamiltonian stencil (Section
5.3), through the C ABI, against the oracle's element-by-element assembly,
its Kronecker form and its Bloch operator; and the generalized problem
A v = lambda B v solved with the Q1 stencils (both products in one pass)
against LAPACK and against the same pencil given as CSR."""
import numpy as np
import pytest
import scipy.linalg as sla
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


def _coeff(E, seed):
    rng = np.random.default_rng(seed)
    return np.where(rng.uniform(size=E**3) < 0.5, 10.0, 1.0) * rng.uniform(0.5, 1.5, E**3)


# E = 8 (n = 343), E = 5 (n = 64: every node near a wall), E = 13 (n = 1728)
@pytest.mark.parametrize("E,nc,ldpad", [(8, 4, 0), (5, 3, 2), (13, 9, 1)])
def test_q1_stencils_match_element_assembly(plhr, E, nc, ldpad):
    c = _coeff(E, 40 + E)
    A, Bm = oops.q1_fe_3d(E, c)
    n = A.shape[0]
    opA = plhr.Operator.q1_stiffness(E, torch.from_numpy(c).cuda())
    opB = plhr.Operator.q1_mass(E)
    assert opA.n == n and opB.n == n
    X = wl.uniform_block(n, nc + ldpad, 41)
    Xt = torch.from_numpy(X).cuda()[:, :nc]
    ra, rb = A @ X[:, :nc], Bm @ X[:, :nc]
    ya = opA.apply(Xt).cpu().numpy()
    yb = opB.apply(Xt).cpu().numpy()
    assert np.abs(ya - ra).max() <= 1e-14 * np.abs(ra).max()
    assert np.abs(yb - rb).max() <= 1e-14 * np.abs(rb).max()
    pa, pb = opA.apply_pair(opB, Xt)
    assert np.abs(pa.cpu().numpy() - ra).max() <= 1e-14 * np.abs(ra).max()
    assert np.abs(pb.cpu().numpy() - rb).max() <= 1e-14 * np.abs(rb).max()


def test_q1_box_mesh_matches_kronecker_form(plhr):
    """Unequal node counts per axis (6 x 4 x 5 interior nodes, h = 0.1,
    c = 1): the products equal K (x) M (x) M + M (x) K (x) M + M (x) M (x) K
    and M (x) M (x) M built from the 1D linear-element matrices."""
    dims, h = (6, 4, 5), 0.1
    K1 = [oops.q1_1d(N, h) for N in dims]           # (K, M) per axis, x first
    kz, mz = K1[2]
    ky, my = K1[1]
    kx, mx = K1[0]
    A = (sp.kron(kz, sp.kron(my, mx)) + sp.kron(mz, sp.kron(ky, mx)) + sp.kron(mz, sp.kron(my, kx))).tocsr()
    Bm = sp.kron(mz, sp.kron(my, mx)).tocsr()
    opA = plhr.Operator._stencil(plhr.Q1_STIFF27, dims, h)
    opB = plhr.Operator._stencil(plhr.Q1_MASS27, dims, h)
    X = wl.uniform_block(A.shape[0], 3, 42)
    Xt = torch.from_numpy(X).cuda()
    assert np.abs(opA.apply(Xt).cpu().numpy() - A @ X).max() <= 1e-14 * np.abs(A @ X).max()
    assert np.abs(opB.apply(Xt).cpu().numpy() - Bm @ X).max() <= 1e-14 * np.abs(Bm @ X).max()


@pytest.mark.parametrize("dims,nc", [((6, 6, 6), 3), ((5, 4, 3), 2), ((7, 1, 4), 1)])
def test_bloch_stencil_matches_oracle(plhr, dims, nc):
    rng = np.random.default_rng(sum(dims))
    n = int(np.prod(dims))
    V = rng.uniform(-4.0, -1.0, n)
    kappa = [rng.uniform(-np.pi / N, np.pi / N) for N in dims]
    H = oops.bloch_hamiltonian(dims, 1.0, V, kappa)
    op = plhr.Operator.bloch(dims, 1.0, torch.from_numpy(V).cuda(), kappa)
    X = wl.start_block(n, nc, 43, complex_=True)
    Y = op.apply_c128(torch.from_numpy(X).cuda()).cpu().numpy()
    ref = H @ X
    assert np.abs(Y - ref).max() <= 1e-13 * np.abs(ref).max()
    # kappa = 0: the real periodic Hamiltonian; real and complex products agree
    op0 = plhr.Operator.bloch(dims, 1.0, torch.from_numpy(V).cuda(), (0.0, 0.0, 0.0))
    Xr = wl.uniform_block(n, nc, 44)
    yr = op0.apply(torch.from_numpy(Xr).cuda()).cpu().numpy()
    assert np.abs(yr - oops.hamiltonian(dims, 1.0, V) @ Xr).max() <= 1e-13 * np.abs(yr).max()


def test_real_operator_on_complex_blocks(plhr):
    dims, h = (6, 5, 4), 0.1
    op = plhr.Operator.laplacian(dims, h)
    X = wl.start_block(120, 3, 45, complex_=True)
    Y = op.apply_c128(torch.from_numpy(X).cuda()).cpu().numpy()
    ref = oops.laplacian_dirichlet(dims, h) @ X
    assert np.abs(Y - ref).max() <= 1e-13 * np.abs(ref).max()


def test_generalized_q1_stencil_solve(plhr):
    """A v = lambda B v with the Q1 stencils (E = 8, coefficient in {1, 10}
    on 2^3-element cubes; the solver forms A X and B X in one pass): the k
    pairs nearest sigma equal LAPACK's, the vectors are B-orthonormal, and the
    per-iteration Ritz values equal those of the same pencil given as CSR."""
    E = 8
    c = wl.q1_coefficient(E, 2, wl.SEED_BASE + 4)
    A, Bm = oops.q1_fe_3d(E, c)
    lam = sla.eigh(A.toarray(), Bm.toarray(), eigvals_only=True)
    sigma = 0.5 * (lam[40] + lam[41])
    k, guard = 4, 2
    near = np.sort(lam[np.argsort(np.abs(lam - sigma))[:k]])
    opA = plhr.Operator.q1_stiffness(E, torch.from_numpy(c).cuda())
    opB = plhr.Operator.q1_mass(E)
    d = 1.0 / np.abs(A.diagonal() - sigma * Bm.diagonal())
    T = plhr.DiagPrec(d)
    v0 = torch.from_numpy(wl.uniform_block(A.shape[0], k + guard, 46)).cuda()
    ev, vecs, info = plhr.solve(opA, sigma, k, T=T, B=opB, tol=1e-10, maxit=6000, guard=guard, v_init=v0,
                                history=True)
    assert info["converged"], info
    assert np.allclose(np.sort(ev), near, rtol=1e-10)
    V = vecs.cpu().numpy()
    assert np.abs(V.T @ (Bm @ V) - np.eye(k)).max() <= 1e-11
    ev2, _, info2 = plhr.solve(plhr.Operator.csr(A), sigma, k, T=T, B=plhr.Operator.csr(Bm), tol=1e-10,
                               maxit=6000, guard=guard, v_init=v0, history=True)
    for a, b in list(zip(info["history"], info2["history"]))[:20]:
        assert np.allclose(a["lam"], b["lam"], rtol=1e-9)
