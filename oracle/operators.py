"""Model operators of the paper, assembled from their definitions (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Grid ordering: a grid with axis sizes (nx, ny[, nz]) is flattened with x
fastest, i.e. index = (z*ny + y)*nx + x.  Kronecker products are therefore
written with the slowest axis first.

* Finite-difference Laplacian (Section 5.2: "standard 5-point FD
  discretization"; the 3D 7-point analogue): the 1D second difference
  (-u[j-1] + 2u[j] - u[j+1]) / h^2 with homogeneous Dirichlet ends, combined as
  a Kronecker sum over the axes.
* Real-space Hamiltonian H = -1/2 Lap + diag(V) (the role of the Hamiltonians
  of Section 5.3 in the synthetic differentiation workload): the same
  Kronecker sum with the 1D second difference closed periodically
  (u[-1] = u[N-1], u[N] = u[0]) or with Dirichlet ends, times 1/2, plus the
  potential on the diagonal.
* Bloch Hamiltonian H_kappa = -1/2 Lap_kappa + diag(V) on a periodic grid
  (the complex Hermitian Hamiltonians of Section 5.3 at a crystal momentum
  kappa): the periodic second difference with the phase e^{+-i kappa_d h} on
  every link along axis d, (2u[j] - e^{i kappa h} u[j+1] - e^{-i kappa h}
  u[j-1]) / h^2, so that a plane wave e^{i theta j} has the eigenvalue
  (2 - 2 cos(theta + kappa h)) / h^2; kappa = 0 is the real periodic case.
* Bilinear (Q1) finite elements (Section 5.1: "standard bilinear finite
  elements", stiffness A and mass B): on a tensor mesh the Q1 element matrices
  factor into 1D linear-element matrices, so A = K (x) M + M (x) K and
  B = M (x) M with K = tridiag(-1, 2, -1)/h and M = tridiag(1, 4, 1) h/6 on
  the interior nodes.
* Trilinear (Q1) finite elements in 3D with a coefficient c per element
  (the generalized pencil of -div(c grad u) = lambda u): assembled element by
  element from the 8 x 8 element matrices c_e (k (x) m (x) m + m (x) k (x) m
  + m (x) m (x) k) and m (x) m (x) m of the 1D linear element (k = [[1, -1],
  [-1, 1]] / h, m = [[2, 1], [1, 2]] h / 6), then restricted to the interior
  nodes (homogeneous Dirichlet).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def second_difference_1d(N: int, h: float) -> sp.csr_matrix:
    """(-u[j-1] + 2u[j] - u[j+1]) / h^2 on N interior points, Dirichlet ends."""
    main = np.full(N, 2.0)
    off = np.full(N - 1, -1.0)
    return (sp.diags([off, main, off], [-1, 0, 1], format="csr") / h**2).tocsr()


def kron_sum(mats_slow_to_fast):
    """Kronecker sum  sum_d I (x) .. (x) M_d (x) .. (x) I  (first matrix = slowest axis)."""
    sizes = [m.shape[0] for m in mats_slow_to_fast]
    total = None
    for d, m in enumerate(mats_slow_to_fast):
        left = int(np.prod(sizes[:d])) if d > 0 else 1
        right = int(np.prod(sizes[d + 1:])) if d + 1 < len(sizes) else 1
        term = sp.kron(sp.kron(sp.identity(left, format="csr"), m, format="csr"),
                       sp.identity(right, format="csr"), format="csr")
        total = term if total is None else total + term
    return total.tocsr()


def laplacian_dirichlet(dims, h: float) -> sp.csr_matrix:
    """Negative FD Laplacian, Dirichlet, on a grid with axis sizes dims = (nx, ny[, nz])."""
    mats = [second_difference_1d(N, h) for N in reversed(dims)]  # slowest axis first
    return kron_sum(mats)


def second_difference_periodic_1d(N: int, h: float) -> sp.csr_matrix:
    """(-u[j-1] + 2u[j] - u[j+1]) / h^2 on N points of a periodic line."""
    D = sp.lil_matrix((N, N))
    for j in range(N):
        D[j, j] += 2.0
        D[j, (j - 1) % N] -= 1.0
        D[j, (j + 1) % N] -= 1.0
    return (D.tocsr() / h**2).tocsr()


def hamiltonian(dims, h: float, V, periodic: bool = True) -> sp.csr_matrix:
    """H = -1/2 Lap + diag(V) on the grid dims = (nx, ny[, nz]); V flattened x fastest."""
    one_d = second_difference_periodic_1d if periodic else second_difference_1d
    lap = kron_sum([one_d(N, h) for N in reversed(dims)])
    return (0.5 * lap + sp.diags(np.asarray(V, dtype=np.float64).ravel(), 0)).tocsr()


def second_difference_bloch_1d(N: int, h: float, kappa: float) -> sp.csr_matrix:
    """(2u[j] - e^{i kappa h} u[j+1] - e^{-i kappa h} u[j-1]) / h^2 on N points
    of a periodic line (Hermitian; the phase sits on every link)."""
    ph = np.exp(1j * kappa * h)
    D = sp.lil_matrix((N, N), dtype=np.complex128)
    for j in range(N):
        D[j, j] += 2.0
        D[j, (j + 1) % N] -= ph
        D[j, (j - 1) % N] -= np.conj(ph)
    return (D.tocsr() / h**2).tocsr()


def bloch_hamiltonian(dims, h: float, V, kappa) -> sp.csr_matrix:
    """H = -1/2 Lap_kappa + diag(V) on the periodic grid dims = (nx, ny[, nz])
    at crystal momentum kappa = (kappa_x, kappa_y[, kappa_z]); V flattened x
    fastest; complex Hermitian."""
    kap = [float(k) for k in kappa]
    assert len(kap) == len(dims)
    mats = [second_difference_bloch_1d(N, h, k) for N, k in zip(reversed(dims), reversed(kap))]
    lap = kron_sum(mats)
    return (0.5 * lap + sp.diags(np.asarray(V, dtype=np.float64).ravel().astype(np.complex128), 0)).tocsr()


def q1_1d(N: int, h: float):
    """1D linear-element stiffness and mass on N interior nodes of a uniform mesh."""
    K = sp.diags([np.full(N - 1, -1.0), np.full(N, 2.0), np.full(N - 1, -1.0)],
                 [-1, 0, 1], format="csr") / h
    M = sp.diags([np.full(N - 1, 1.0), np.full(N, 4.0), np.full(N - 1, 1.0)],
                 [-1, 0, 1], format="csr") * (h / 6.0)
    return K.tocsr(), M.tocsr()


def q1_fe_2d(elems: int):
    """Stiffness A and mass B of bilinear elements for -Laplace on the unit square
    with `elems` elements per side, homogeneous Dirichlet (Section 5.1)."""
    h = 1.0 / elems
    K, M = q1_1d(elems - 1, h)
    A = (sp.kron(K, M) + sp.kron(M, K)).tocsr()
    B = sp.kron(M, M).tocsr()
    return A, B


def q1_fe_3d(elems: int, coeff=None):
    """Stiffness A (of -div(c grad)) and mass B of trilinear elements on the
    unit cube with `elems` elements per side, homogeneous Dirichlet; coeff is
    None (c = 1) or an array of elems^3 element values, x fastest.  Assembled
    element by element (interior nodes, x fastest)."""
    E = int(elems)
    h = 1.0 / E
    k1 = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    m1 = np.array([[2.0, 1.0], [1.0, 2.0]]) * (h / 6.0)
    # local node (a, b, c) -> a + 2 b + 4 c: Kronecker products slowest axis first
    Ke = np.kron(m1, np.kron(m1, k1)) + np.kron(m1, np.kron(k1, m1)) + np.kron(k1, np.kron(m1, m1))
    Me = np.kron(m1, np.kron(m1, m1))
    c = np.ones(E**3) if coeff is None else np.asarray(coeff, dtype=np.float64).ravel()
    assert c.size == E**3
    ex, ey, ez = np.meshgrid(np.arange(E), np.arange(E), np.arange(E), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    elem = (ez * E + ey) * E + ex
    nn = E + 1
    local = np.array([[a, b, cc] for cc in (0, 1) for b in (0, 1) for a in (0, 1)])   # a fastest
    gnode = np.stack([((ez + cc) * nn + (ey + b)) * nn + (ex + a) for a, b, cc in local], axis=1)
    rows = np.repeat(gnode, 8, axis=1).ravel()
    cols = np.tile(gnode, (1, 8)).ravel()
    A = sp.coo_matrix(((c[elem][:, None] * Ke.ravel()[None, :]).ravel(), (rows, cols)),
                      shape=(nn**3, nn**3)).tocsr()
    B = sp.coo_matrix((np.tile(Me.ravel(), E**3), (rows, cols)), shape=(nn**3, nn**3)).tocsr()
    g = np.arange(nn)
    inner = (g > 0) & (g < E)
    mask = (inner[None, None, :] & inner[None, :, None] & inner[:, None, None]).ravel()   # [z][y][x]
    idx = np.nonzero(mask)[0]
    return A[idx][:, idx].tocsr(), B[idx][:, idx].tocsr()


def model_operator(workload):
    """(A, B) of a workload description; B is None for the standard problem."""
    if workload.kind in ("lap2d", "lap3d"):
        return laplacian_dirichlet(workload.dims, workload.h), None
    raise ValueError("unknown operator kind %r" % workload.kind)
