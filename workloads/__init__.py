"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the eigensolver: it only describes the
workloads (grid sizes, mesh widths, shifts, block sizes, multigrid depth) and
draws the seeded starting blocks.  Both the oracle and the GPU path receive
the same arrays from here.

Starting block V0 (the paper recommends a random initial guess, Section 3.2):
element (i, j) of an n x kc block is the (i*kc + j + 1)-th output of the
SplitMix64 generator (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) started from ``seed``; the 64-bit
output x is mapped to (x >> 11) * 2**-53 - 0.5, uniform in [-0.5, 0.5).
The C library implements the same published generator for the case where the
caller passes no starting block.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_BASE = 20140801


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start+1 .. start+count of SplitMix64 seeded with ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_block(n: int, kc: int, seed: int, start: int = 0) -> np.ndarray:
    """n x kc float64 block, entries uniform in [-0.5, 0.5) (row-major draw order)."""
    x = splitmix64(seed, n * kc, start)
    u = (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) - 0.5
    return u.reshape(n, kc)


def start_block(n: int, kc: int, seed: int, complex_: bool = False) -> np.ndarray:
    """Seeded starting block V0 (n x kc).  Complex blocks draw the imaginary
    part from the outputs that follow the real part's n*kc outputs."""
    re = uniform_block(n, kc, seed)
    if not complex_:
        return re
    im = uniform_block(n, kc, seed, start=n * kc)
    return re + 1j * im


@dataclass
class Workload:
    """One seeded eigenproblem: operator description + solver parameters."""
    name: str
    kind: str                 # "lap2d" (5-point) or "lap3d" (7-point), Dirichlet
    dims: tuple               # grid points per axis, x fastest: (nx, ny[, nz])
    h: float                  # mesh width
    sigma: float              # target shift
    k: int                    # wanted eigenpairs
    tol: float                # relative residual tolerance
    prec: str = "none"        # "none" (T = I) or "avmg"
    mg_levels: int = 1
    mg_nu: int = 2
    maxit: int = 1000
    guard: int = 1            # block columns beyond k (real arithmetic)
    seed: int = SEED_BASE
    real: bool = True
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(np.prod(self.dims))

    @property
    def kprime(self) -> int:
        # real arithmetic runs guard extra columns (at least one, so that a
        # conjugate pair is never cut at the k-th position)
        return self.k + self.guard if self.real else self.k

    def v0(self) -> np.ndarray:
        return start_block(self.n, self.kprime, self.seed, complex_=not self.real)


def lap_closed_form(dims, h) -> np.ndarray:
    """Sorted eigenvalues of the Dirichlet finite-difference Laplacian on a
    tensor grid: sum over axes of (4/h^2) sin^2(i pi / (2(N+1))), i = 1..N.
    Used only to place shifts (midpoints of gaps); tests pin the operators
    against it independently."""
    mus = [4.0 / h**2 * np.sin(np.arange(1, N + 1) * np.pi / (2.0 * (N + 1))) ** 2 for N in dims]
    tot = mus[0]
    for m in mus[1:]:
        tot = (tot[:, None] + m[None, :]).ravel()
    return np.sort(tot)


def _mid_gap(dims, h, lo_index: int) -> float:
    lam = lap_closed_form(dims, h)
    return 0.5 * (lam[lo_index] + lam[lo_index + 1])


def lap2d_32x32_k4() -> Workload:
    """2D 5-point Laplacian, 32x32 Dirichlet interior grid, h = 1/33, B = I,
    sigma midway between the 100th and 101st eigenvalues, k = 4, T = I."""
    dims, h = (32, 32), 1.0 / 33.0
    return Workload(name="lap2d_32x32_k4", kind="lap2d", dims=dims, h=h,
                    sigma=_mid_gap(dims, h, 99), k=4, tol=1e-8, prec="none", maxit=20000,
                    guard=2, seed=SEED_BASE + 1)


# 3D 7-point Laplacian, 128^3 interior, h = 1/129: the shift is the midpoint of
# the eigenvalues 1064.0220711725 (mode (6,6,6)) and 1073.1201516674 (modes
# (3,6,8) and permutations); 471 eigenvalues lie below it and the 10 nearest
# form complete multiplets (3 + 1 + 6), the 11th is 12.18 away.
def lap3d_128cube_k10() -> Workload:
    dims, h = (128, 128, 128), 1.0 / 129.0
    sigma = 0.5 * (_lap3_mode((6, 6, 6), h) + _lap3_mode((3, 6, 8), h))
    return Workload(name="lap3d_128cube_k10", kind="lap3d", dims=dims, h=h,
                    sigma=sigma, k=10, tol=1e-8, prec="avmg", mg_levels=4,
                    mg_nu=2, guard=6, seed=SEED_BASE + 2,
                    extra={"transfer": "linear", "coarse": "fine_spectrum"})


def _lap3_mode(mode, h) -> float:
    return sum(4.0 / h**2 * math.sin(i * math.pi * h / 2.0) ** 2 for i in mode)


def lap3d_small(N: int = 32, levels: int = 3, k: int = 4, gap_index: int | None = None,
                seed: int = SEED_BASE + 12) -> Workload:
    """Reduced 3D Laplacian with the same structure as the 128^3 problem, for
    parity runs the oracle finishes in seconds.  The shift sits in the widest
    gap around the requested index such that the k nearest eigenvalues are
    complete multiplets."""
    h = 1.0 / (N + 1)
    lam = lap_closed_form((N, N, N), h)
    target = gap_index if gap_index is not None else 60
    sigma = _clean_shift(lam, target, k)
    return Workload(name=f"lap3d_{N}cube_k{k}", kind="lap3d", dims=(N, N, N), h=h,
                    sigma=sigma, k=k, tol=1e-8, prec="avmg", mg_levels=levels,
                    mg_nu=2, seed=seed)


def lap2d_small(N: int = 16, k: int = 4, gap_index: int = 20, prec: str = "none",
                levels: int = 1, seed: int = SEED_BASE + 11) -> Workload:
    h = 1.0 / (N + 1)
    lam = lap_closed_form((N, N), h)
    sigma = _clean_shift(lam, gap_index, k)
    return Workload(name=f"lap2d_{N}sq_k{k}", kind="lap2d", dims=(N, N), h=h,
                    sigma=sigma, k=k, tol=1e-8, prec=prec, mg_levels=levels,
                    mg_nu=2, seed=seed)


def _clean_shift(lam: np.ndarray, target: int, k: int) -> float:
    """Midpoint of a gap near index ``target`` such that the k eigenvalues
    nearest the midpoint do not split a multiplet (ties within 1e-9 relative)."""
    best = None
    for lo in range(max(0, target - 40), min(len(lam) - 1, target + 40)):
        if lam[lo + 1] - lam[lo] <= 1e-9 * lam[lo + 1]:
            continue
        s = 0.5 * (lam[lo] + lam[lo + 1])
        d = np.sort(np.abs(lam - s))
        if d[k] - d[k - 1] > 1e-6 * s:  # k-th and (k+1)-th distances differ
            score = (d[k] - d[k - 1]) / s
            if best is None or score > best[0]:
                best = (score, s)
    if best is None:
        raise ValueError("no clean shift near index %d" % target)
    return float(best[1])


WORKLOADS = {"lap2d_32x32_k4": lap2d_32x32_k4, "lap3d_128cube_k10": lap3d_128cube_k10}


def gaussian_potential(dims, nwells: int, seed: int, depth=(-4.0, -1.0), width=(0.5, 1.5)) -> np.ndarray:
    """Seeded potential on a periodic grid with unit spacing (x fastest):
    V(x) = sum_j d_j exp(-|x - c_j|^2 / (2 w_j^2)) with minimum-image
    distances, centres uniform in the box, depths d_j and widths w_j uniform in
    the given ranges (grid units).  The well draws come from one SplitMix64
    stream: per well (c_x, c_y[, c_z], d, w)."""
    dims = tuple(dims)
    nd = len(dims)
    u = uniform_block(nwells, nd + 2, seed) + 0.5          # uniform [0, 1)
    axes = [np.arange(N, dtype=np.float64) for N in dims]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]   # x fastest when raveled
    V = np.zeros(grids[0].shape)
    for j in range(nwells):
        r2 = np.zeros_like(V)
        for a, N in enumerate(dims):
            c = u[j, a] * N
            dx = np.abs(grids[a] - c)
            dx = np.minimum(dx, N - dx)
            r2 += dx * dx
        d = depth[0] + (depth[1] - depth[0]) * u[j, nd]
        w = width[0] + (width[1] - width[0]) * u[j, nd + 1]
        V += d * np.exp(-r2 / (2.0 * w * w))
    return V.ravel()


def hamiltonian_small(N: int = 10, nwells: int = 6, k: int = 4, seed: int = SEED_BASE + 5, dim: int = 3):
    """Differentiation test problem: H(V) = -1/2 Lap + V on an N^dim periodic
    grid (h = 1) with a seeded Gaussian-well potential (the structure of the
    64^3, 32-well workload at a size a dense eigensolver finishes quickly)."""
    dims = (N,) * dim
    return {"dims": dims, "h": 1.0, "V": gaussian_potential(dims, nwells, seed), "k": k, "seed": seed}


def bloch_small(N: int = 6, nwells: int = 3, seed: int = SEED_BASE + 3, dim: int = 3):
    """Complex Hermitian test problem of the Bloch-Hamiltonian workload at a
    size a dense eigensolver finishes quickly: a seeded Gaussian-well
    potential on an N^dim periodic grid (h = 1) and a crystal momentum kappa
    uniform in the supercell zone [-pi/N, pi/N)^dim (drawn after the wells)."""
    dims = (N,) * dim
    V = gaussian_potential(dims, nwells, seed)
    u = uniform_block(dim, 1, seed, start=nwells * (dim + 2)).ravel()     # [-0.5, 0.5)
    kappa = tuple(2.0 * np.pi / N * float(x) for x in u)
    return {"dims": dims, "h": 1.0, "V": V, "kappa": kappa, "seed": seed}


def bloch_96cube():
    """96^3 periodic Bloch Hamiltonian: 64 seeded Gaussian wells (depth
    U(-4, -1), width U(0.5, 1.5) grid units, centres uniform) and kappa uniform
    in [-pi/96, pi/96)^3 (h = 1).  The shift is the midpoint of the 31st and
    32nd eigenvalues of the assembled operator, k = 16."""
    return bloch_small(96, 64, SEED_BASE + 3, 3)


def q1_coefficient(elems: int, block: int, seed: int) -> np.ndarray:
    """Element coefficients c in {1, 10} (x fastest): constant on cubes of
    block^3 elements, each cube 10 with probability 1/2 (one SplitMix64 draw
    per cube, cubes in x-fastest order)."""
    nb = elems // block
    assert nb * block == elems
    u = uniform_block(nb**3, 1, seed).ravel()
    cb = np.where(u >= 0.0, 10.0, 1.0).reshape(nb, nb, nb)         # [z][y][x] cubes
    e = np.arange(elems) // block
    return cb[e[:, None, None], e[None, :, None], e[None, None, :]].ravel()


def q1_fe_64cube():
    """64^3 trilinear elements on the unit cube (interior 63^3 nodes),
    coefficient c in {1, 10} on 8^3-element cubes; k = 8 pairs near spectral
    index 300 of the pencil (stiffness, mass)."""
    return {"elems": 64, "coeff": q1_coefficient(64, 8, SEED_BASE + 4), "k": 8}


def ham64_potential():
    """64^3 periodic grid, 32 seeded Gaussian wells (h = 1)."""
    dims = (64, 64, 64)
    return dims, gaussian_potential(dims, 32, SEED_BASE + 5)


# Shift of the 64^3 differentiation workload: the 8 eigenvalues nearest it are
# lambda_6 .. lambda_13 of H (about -1.4972 .. -1.3181; smallest gap inside the
# block 4.8e-3; the 9th is 1.62 times farther than the 8th).  Written by
# workloads/select_shift_ham64.py from a Lanczos solve of the oracle's operator.
HAM64_SIGMA = -1.4076
HAM64_K = 8
# the 8 eigenvalues nearest HAM64_SIGMA from the same Lanczos solve (tol 1e-10)
HAM64_LAMBDA_REF = (-1.4972095727, -1.4646666705, -1.3947918710, -1.3900142734, -1.3677701223, -1.3384194736,
                    -1.3285495681, -1.3180617417)


def ham64_k8_grad():
    """Differentiation workload on the 64^3 Hamiltonian: potential, shift,
    block size, eigenvalue weights w ~ U(0.5, 1.5) and a density mask
    m ~ Bernoulli(1/2) for the loss sum_k w_k lambda_k + sum_k |m (.) v_k|^2."""
    dims, V = ham64_potential()
    n = int(np.prod(dims))
    w = 0.5 + (uniform_block(HAM64_K, 1, SEED_BASE + 51).ravel() + 0.5)
    mask = (uniform_block(n, 1, SEED_BASE + 52).ravel() >= 0.0).astype(np.float64)
    return {"dims": dims, "h": 1.0, "V": V, "sigma": HAM64_SIGMA, "k": HAM64_K, "w": w, "mask": mask,
            "seed": SEED_BASE + 5}
