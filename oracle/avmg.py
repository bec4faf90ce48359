"""Absolute-value multigrid preconditioner T ~ |L - sigma I|^{-1} (Appendix A,
Algorithm 4, "AV-MG"), FP64, for the Dirichlet FD Laplacian.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Algorithm 4 fixes the structure of the V-cycle: per level a choice of B_l
(the Laplacian L_l when sqrt(sigma) h_l < delta, otherwise a polynomial
p_m(L_l - sigma I_l)), nu Richardson pre-smoothing steps from zero with
smoother M_l, restriction of r_l - B_l w_l, recursion (exact
|L_0 - sigma I_0|^{-1} on the coarsest grid), prolongation of the coarse
correction, and nu post-smoothing steps with M_l^{-*}.  The paper leaves the
parameters to its reference [Ve.Kn:13]; the readings taken here are:

* delta = 2 pi / 10 (ten points per wavelength);
* m = 2, p_2(x) = (x^2 + c_l^2) / (2 c_l) with c_l = max(|a_l|, |b_l|) / 2,
  where [a_l, b_l] is the Gershgorin interval of L_l - sigma I_l
  (p_2 >= c_l / 2 > 0, so B_l is positive definite);
* M_l = beta_l I with beta_l an upper bound of the spectrum of B_l: the
  Gershgorin bound of L_l when B_l = L_l, and p_2 evaluated at the ends of the
  Gershgorin interval of L_l - sigma I_l otherwise (M_l is symmetric, so the
  post-smoother M_l^{-*} equals the pre-smoother);
* cell-centred coarsening by two per axis with P = 2^d R^T: either
  transfer="constant" (restriction averages the 2^d children of a coarse
  cell, prolongation copies the coarse value to them) or transfer="linear"
  (prolongation interpolates with the 1D weights 3/4 and 1/4 from the two
  nearest coarse cells, zero beyond the boundary, tensor product over axes);
* the level Laplacians are rediscretised with h_{l-1} = 2 h_l; the coarsest
  operator L_0 is either that rediscretised Laplacian (coarse="rediscretised")
  or (coarse="fine_spectrum") the operator whose eigenvectors are the
  cell-centred sine modes sin((p + 1/2) m pi / N_0) of the coarse grid and
  whose eigenvalues are those the finest-grid Laplacian has for the same mode
  numbers m (so |L_0 - sigma I|^{-1} resonates where the fine operator does);
* the garbled "|L_l - I_l|^{-1}" of the algorithm's output line is read as
  |L_l - sigma I_l|^{-1}.

INV-MG (Appendix A, Algorithm 5, indefinite=True): the same V-cycle with
B_l = L_l - sigma I_l on every level and the exact (L_0 - sigma I_0)^{-1} on
the coarsest grid (an indefinite T ~ (L - sigma I)^{-1}); the smoother is
Richardson with 1/beta_l, beta_l = max(|a_l|, |b_l|) over the Gershgorin
interval [a_l, b_l] of L_l - sigma I_l (the paper takes the smoothers and
transfers of Algorithm 4).  The algorithm's recursion into "AV-MG" and its
"(L_l - I_l)^{-1}" are read as INV-MG and (L_l - sigma I_l)^{-1}.

Pins (tests/test_oracle_pins.py, tests/test_oracle_pins_transfer_pairs.py):
one level is exactly |L - sigma I|^{-1} on the analytic modes; the spectrum of
p_2; the transfer identities of both transfers (the trilinear weights against
a brute-force construction from the cell centres, reproduction of linear
fields, R 1 = 1 away from the walls); the fine-spectrum coarsest operator's
eigenpairs against LAPACK on independently built matrices; a two-grid cycle
equals its closed algebraic form for both option pairs; the cycle is
symmetric positive definite for both option pairs.  Parity unpinned with respect to the paper's own multigrid: the
parameter readings above replace a reference that is not available, so no
printed number of the paper checks them.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .operators import laplacian_dirichlet

DELTA = 2.0 * math.pi / 10.0


def aggregation_1d(N: int) -> sp.csr_matrix:
    """(N/2) x N averaging of cell pairs (2I, 2I+1) -> I."""
    if N % 2:
        raise ValueError("cell-centred coarsening needs an even axis size, got %d" % N)
    Nc = N // 2
    rows = np.repeat(np.arange(Nc), 2)
    cols = np.arange(N)
    return sp.csr_matrix((np.full(N, 0.5), (rows, cols)), shape=(Nc, N))


def linear_prolongation_1d(Nc: int) -> sp.csr_matrix:
    """(2 Nc) x Nc cell-centred linear interpolation: fine 2I gets 3/4 of
    coarse I and 1/4 of coarse I-1, fine 2I+1 gets 3/4 of I and 1/4 of I+1
    (coarse cells outside the grid are zero)."""
    P = sp.lil_matrix((2 * Nc, Nc))
    for I in range(Nc):
        P[2 * I, I] = 0.75
        P[2 * I + 1, I] = 0.75
        if I > 0:
            P[2 * I, I - 1] = 0.25
        if I < Nc - 1:
            P[2 * I + 1, I + 1] = 0.25
    return P.tocsr()


def restriction(dims, transfer: str = "constant") -> sp.csr_matrix:
    """R = P^T / 2^d for the cell-centred prolongation P (Kronecker product of
    the 1D operators over the axes)."""
    R = None
    for N in reversed(dims):  # slowest axis first
        if transfer == "constant":
            r1 = aggregation_1d(N)
        elif transfer == "linear":
            if N % 2:
                raise ValueError("cell-centred coarsening needs an even axis size, got %d" % N)
            r1 = (linear_prolongation_1d(N // 2).T / 2.0).tocsr()
        else:
            raise ValueError("unknown transfer %r" % transfer)
        R = r1 if R is None else sp.kron(R, r1, format="csr")
    return R.tocsr()


class Level:
    def __init__(self, dims, h, sigma, indefinite=False):
        self.dims = tuple(dims)
        self.h = h
        self.d = len(dims)
        self.L = laplacian_dirichlet(dims, h)
        self.n = self.L.shape[0]
        # Gershgorin interval of L_l - sigma I: diagonal 2d/h^2, off-diagonal sum 2d/h^2
        a = -sigma
        b = 4.0 * self.d / h**2 - sigma
        self.use_poly = not (math.sqrt(max(sigma, 0.0)) * h < DELTA)
        self.sigma = sigma
        self.indefinite = indefinite
        if indefinite:
            self.use_poly = False
            self.c = None
            self.beta = max(abs(a), abs(b))
        elif self.use_poly:
            self.c = 0.5 * max(abs(a), abs(b))
            self.beta = (max(a * a, b * b) + self.c**2) / (2.0 * self.c)
        else:
            self.c = None
            self.beta = 4.0 * self.d / h**2

    def apply_B(self, x):
        """B_l x: the Laplacian, or p_2(L_l - sigma I) x (INV-MG: L_l - sigma I)."""
        if self.indefinite:
            return self.L @ x - self.sigma * x
        if not self.use_poly:
            return self.L @ x
        y = self.L @ x - self.sigma * x
        y2 = self.L @ y - self.sigma * y
        return (y2 + self.c**2 * x) / (2.0 * self.c)


def fine_spectrum_operator(coarse_dims, fine_dims, h):
    """Dense coarse operator with the cell-centred sine modes as eigenvectors
    and the fine-grid Laplacian's eigenvalues (2 - 2 cos(m pi/(N+1)))/h^2 of
    the same mode numbers, as a Kronecker sum over the axes."""
    mats = []
    for N0, N in zip(reversed(coarse_dims), reversed(fine_dims)):  # slowest axis first
        p = np.arange(N0) + 0.5
        m = np.arange(1, N0 + 1)
        S = np.sin(np.outer(p, m) * np.pi / N0)
        S /= np.linalg.norm(S, axis=0)[None, :]
        mu = (2.0 - 2.0 * np.cos(m * np.pi / (N + 1))) / h**2
        mats.append(sp.csr_matrix((S * mu[None, :]) @ S.T))
    from .operators import kron_sum
    return kron_sum(mats).toarray()


class AVMG:
    """V-cycle T r of Algorithm 4 with `levels` grids (levels = 1: exact
    |L - sigma I|^{-1} on the given grid)."""

    def __init__(self, dims, h, sigma, levels, nu=2, transfer="constant", coarse="rediscretised",
                 indefinite=False):
        if levels < 1:
            raise ValueError("levels >= 1")
        self.indefinite = indefinite
        self.transfer = transfer
        self.coarse = coarse
        self.sigma = sigma
        self.nu = nu
        self.levels = []  # index 0 = coarsest
        dl, hl = list(dims), h
        grids = []
        for _ in range(levels):
            grids.append((tuple(dl), hl))
            if len(grids) < levels:
                dl = [N // 2 for N in dl]
                hl = 2.0 * hl
        for dims_l, h_l in reversed(grids):
            self.levels.append(Level(dims_l, h_l, sigma, indefinite))
        self.R = [None] + [restriction(self.levels[l].dims, transfer) for l in range(1, levels)]
        # coarsest: |L_0 - sigma I|^{-1} from a dense symmetric eigendecomposition
        if coarse == "rediscretised":
            L0 = self.levels[0].L.toarray()
        elif coarse == "fine_spectrum":
            L0 = fine_spectrum_operator(self.levels[0].dims, dims, h)
        else:
            raise ValueError("unknown coarse operator %r" % coarse)
        lam, Q = np.linalg.eigh(L0 - sigma * np.eye(L0.shape[0]))
        self.coarse_eigs = lam
        self.coarse_inv = (Q / (lam if indefinite else np.abs(lam))[None, :]) @ Q.T

    @property
    def n(self):
        return self.levels[-1].n

    def coarse_solve(self, r):
        return self.coarse_inv @ r

    def _cycle(self, l, r):
        if l == 0:
            return self.coarse_solve(r)
        lev = self.levels[l]
        omega = 1.0 / lev.beta
        d = lev.d
        # step 2: pre-smoothing from w = 0
        w = np.zeros_like(r)
        for _ in range(self.nu):
            w = w + omega * (r - lev.apply_B(w))
        # step 3: coarse grid correction
        rc = self.R[l] @ (r - lev.apply_B(w))
        wc = self._cycle(l - 1, rc)
        w = w + (2.0 ** d) * (self.R[l].T @ wc)   # P = 2^d R^T
        # step 4: post-smoothing (M^{-*} = M^{-1} = omega I)
        for _ in range(self.nu):
            w = w + omega * (r - lev.apply_B(w))
        return w

    def __call__(self, r):
        r = np.asarray(r)
        one = r.ndim == 1
        if one:
            r = r[:, None]
        if np.iscomplexobj(r):
            w = self._cycle(len(self.levels) - 1, r.real) + 1j * self._cycle(len(self.levels) - 1, r.imag)
        else:
            w = self._cycle(len(self.levels) - 1, r)
        return w[:, 0] if one else w


def preconditioner(workload):
    """T of a workload description (None means T = I)."""
    if workload.prec == "none":
        return None
    if workload.prec == "avmg":
        return AVMG(workload.dims, workload.h, workload.sigma, workload.mg_levels, workload.mg_nu,
                    transfer=workload.extra.get("transfer", "constant"),
                    coarse=workload.extra.get("coarse", "rediscretised"))
    raise ValueError("unknown preconditioner %r" % workload.prec)
