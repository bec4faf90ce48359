"""Block PLHR, plain FP64 CPU oracle (Section 4, Algorithm 2 = complex
arithmetic, Algorithm 3 = real arithmetic).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The iteration follows the paper's steps in order:

1. V <- V0, B-normalise the columns, Lambda <- diag(V* A V), P <- [] (Alg. 2/3
   steps 1-2).
2. Until the k wanted pairs converge:
   a. preconditioned residuals W <- T(AV - BV Lambda) (step 4);
   b. s-vectors S <- T(AW - BW Lambda) (step 5);
   c. Z <- [V, W, S, P]; B-orthonormalise blockwise: V-hat, then W against
      V-hat, S against [V-hat W-hat], P against [V-hat W-hat S-hat] (step 6 and
      the paragraph after Alg. 2);
   d. solve the T-harmonic projected problem (Eq. THarm_evp)
          Z*(A - sB)T(A - sB)Z y = xi Z*(A - sB)TBZ y,
      through its shift-invert form (Eq. THarm_evp_sinv): with the Hermitian
      positive definite left matrix G_L = L L*, the eigenpairs (tau, z) of
      L^{-1} G_R L^{-*} give y = L^{-*} z and xi = 1/tau (step 7);
   e. real arithmetic: sort by |xi| with every complex xi followed by its
      conjugate, take k eigenvectors, split complex pairs into real and
      imaginary parts, keep only the real part of a pair cut at the k-th
      position (Alg. 3 steps 7-10);
   f. P <- W-hat Y_W + S-hat Y_S + P-hat Y_P, V <- V-hat Y_V + P (steps 8-9 /
      11-12), with the stored images AZ, BZ and T(A - sB)Z updated by the same
      coefficients (storage paragraph after Alg. 2: 2 products with A and B and
      4 applications of T per iteration);
   g. Rayleigh quotients: one per real column, the pair value of
      Eq. lambda_complex for (v_R, v_I), the own value of the cut column; then
      B-normalise V (Alg. 3 steps 13-14).
3. Standard Rayleigh-Ritz with respect to V (step 12 / 16).

plmr() is the single-vector method with the refinement extraction of Eq. rRR
(Section 3.3); bplhr with one column (k = 1, V0 of one column) is Algorithm 1
(in real arithmetic a conjugate pair at the selection keeps its real part,
Algorithm 3 with k' = k).

Readings where the paper is silent (each also listed in the design notes):
* convergence: relative residual ||Av - lam Bv|| / (max(|lam|, 1) ||Bv||) of
  the k pairs nearest sigma (ties broken by the smaller eigenvalue);
* soft locking: columns whose relative residual is below tol contribute no
  W and S columns in that iteration; the mask is recomputed every iteration
  because the extraction mixes the columns;
* blockwise B-orthonormalisation: projection against the earlier blocks done
  twice, then Cholesky QR twice; a column whose Cholesky pivot squared falls
  below 1e-12 times its squared B-norm before projection is dropped;
* xi ordering ties: ascending |xi|, then ascending Re(xi);
* a complex y is rotated by a unit complex factor so that its real and
  imaginary parts are orthogonal with the real part the longer one, and has
  unit 2-norm (this fixes the cut column's real part independently of the
  basis used for Z).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

DROP_TOL = 1e-12


def _adj(X):
    return X.conj().T


def _bmul(B, X):
    return X if B is None else B @ X


def _tmul(T, X):
    return X.copy() if T is None else T(X)


def _cdot(X, Y):
    """Column-wise real part of x_j^* y_j."""
    return np.real(np.sum(np.conj(X) * Y, axis=0))


@dataclass
class Result:
    eigvals: np.ndarray
    eigvecs: np.ndarray
    residuals: np.ndarray       # final relative residuals (explicit A V, B V)
    converged: bool
    iterations: int
    history: list = field(default_factory=list)


def chol_drop(G, norm0sq, drop_tol=DROP_TOL):
    """Cholesky G = R* R of a Hermitian PSD Gram with column dropping: column j
    is dropped when its pivot squared is below drop_tol * norm0sq[j].  Returns
    (R restricted to the kept columns, kept index list)."""
    m = G.shape[0]
    keep = []
    R = np.zeros_like(G)
    for j in range(m):
        # pivot of column j against the kept columns before it
        s = G[j, j]
        for i in keep:
            s = s - np.conj(R[i, j]) * R[i, j]
        s = np.real(s)
        if s <= drop_tol * norm0sq[j] or not np.isfinite(s):
            continue
        d = np.sqrt(s)
        R[j, j] = d
        for jj in range(j + 1, m):
            t = G[j, jj]
            for i in keep:
                t = t - np.conj(R[i, j]) * R[i, jj]
            R[j, jj] = t / d
        keep.append(j)
    Rk = R[np.ix_(keep, keep)]
    return Rk, keep


def _apply_rinv(mats, R):
    """X R^{-1} for each X in mats (R upper triangular)."""
    # Y R = X  <=>  R^T Y^T = X^T (plain transpose, also for complex R)
    return [sla.solve_triangular(R, X.T, trans="T", lower=False).T for X in mats]


def orthonormalize_block(block, basis, drop_tol=DROP_TOL):
    """B-orthonormalise one block (X, AX, BX, QX) against the B-orthonormal
    blocks in `basis` (projection twice), then Cholesky QR twice with column
    dropping.  Returns the new block (possibly with fewer columns)."""
    X, AX, BX, QX = [M.copy() for M in block]
    norm0sq = _cdot(X, BX)
    for _ in range(2):
        for (Zb, AZb, BZb, QZb) in basis:
            C = _adj(BZb) @ X          # = Zb^* B X  (B Hermitian)
            X -= Zb @ C
            AX -= AZb @ C
            BX -= BZb @ C
            QX -= QZb @ C
    G = _adj(X) @ BX
    G = 0.5 * (G + _adj(G))
    R, keep = chol_drop(G, norm0sq, drop_tol)
    X, AX, BX, QX = [M[:, keep] for M in (X, AX, BX, QX)]
    if len(keep) == 0:
        return X, AX, BX, QX
    X, AX, BX, QX = _apply_rinv((X, AX, BX, QX), R)
    G = _adj(X) @ BX
    G = 0.5 * (G + _adj(G))
    R2 = np.linalg.cholesky(G).conj().T
    X, AX, BX, QX = _apply_rinv((X, AX, BX, QX), R2)
    return X, AX, BX, QX


def rotate_principal(y):
    """Unit-modulus rotation of complex y making Re(y) orthogonal to Im(y)
    with ||Re(y)|| >= ||Im(y)||; returns the rotated y scaled to unit norm."""
    a, b = np.real(y), np.imag(y)
    aa, bb, ab = a @ a, b @ b, a @ b
    phi = 0.5 * np.arctan2(-2.0 * ab, aa - bb)
    y = y * np.exp(1j * phi)
    return y / np.linalg.norm(y)


def order_real_spectrum(xi):
    """Indices of xi sorted by |xi| with each complex xi (Im > 0) followed by
    its conjugate.  Returns (order, partner) where partner[i] is the index of
    the conjugate of eigenvalue i, or -1 for a real eigenvalue."""
    m = len(xi)
    partner = -np.ones(m, dtype=int)
    units = []
    used = np.zeros(m, dtype=bool)
    for i in range(m):
        if used[i]:
            continue
        if np.imag(xi[i]) == 0.0:
            units.append((abs(xi[i]), np.real(xi[i]), [i]))
            used[i] = True
            continue
        # conjugate partner: LAPACK returns exact conjugates for a real matrix
        cand = [j for j in range(m) if not used[j] and j != i and xi[j] == np.conj(xi[i])]
        if not cand:
            cand = [j for j in range(m) if not used[j] and j != i and np.imag(xi[j]) * np.imag(xi[i]) < 0]
            cand.sort(key=lambda j: abs(xi[j] - np.conj(xi[i])))
        j = cand[0]
        pos, neg = (i, j) if np.imag(xi[i]) > 0 else (j, i)
        partner[pos], partner[neg] = neg, pos
        used[i] = used[j] = True
        units.append((abs(xi[pos]), np.real(xi[pos]), [pos, neg]))
    units.sort(key=lambda u: (u[0], u[1]))
    order = [i for u in units for i in u[2]]
    return np.array(order, dtype=int), partner


def tharmonic_extract(GL, GR):
    """All eigenpairs (xi, y) of GL y = xi GR y with GL Hermitian positive
    definite, via tau = 1/xi: with GL = L L*, C = L^{-1} GR L^{-*} has
    eigenpairs (tau, z) and y = L^{-*} z (Eq. THarm_evp_sinv).  y has unit
    2-norm; xi = inf where tau = 0."""
    L = np.linalg.cholesky(GL)
    C = sla.solve_triangular(L, GR, lower=True)
    C = _adj(sla.solve_triangular(L, _adj(C), lower=True))
    tau, Zc = np.linalg.eig(C)
    Y = sla.solve_triangular(_adj(L), Zc, lower=False)
    Y = Y / np.linalg.norm(Y, axis=0)[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        xi = np.where(tau == 0, np.inf, 1.0 / np.where(tau == 0, 1.0, tau))
    return xi, Y


def select_real(xi, Y, kp):
    """Alg. 3 steps 7-10: real coefficient block Y' = [Y0 YR y~R YI] for the
    kp eigenvalues of smallest |xi|.  Returns (Yp, groups) where groups lists,
    per column of Yp, a tag: ('real',), ('pairR', p), ('cut',), ('pairI', p)."""
    order, partner = order_real_spectrum(xi)
    chosen = list(order[:kp])
    chosen_set = set(chosen)
    Y0, YR, YI, cut = [], [], [], None
    for i in chosen:
        if partner[i] < 0:
            Y0.append(np.real(Y[:, i]))
        elif np.imag(xi[i]) > 0:
            y = rotate_principal(Y[:, i])
            if partner[i] in chosen_set:
                YR.append(np.real(y))
                YI.append(np.imag(y))
            else:
                cut = np.real(y)
    cols = Y0 + YR + ([cut] if cut is not None else []) + YI
    tags = ([("real",)] * len(Y0) + [("pairR", p) for p in range(len(YR))]
            + ([("cut",)] if cut is not None else []) + [("pairI", p) for p in range(len(YI))])
    return np.array(cols).T, tags, np.array(chosen)


def select_complex(xi, Y, k):
    order = sorted(range(len(xi)), key=lambda i: (abs(xi[i]), np.real(xi[i]), np.imag(xi[i])))
    chosen = order[:k]
    return Y[:, chosen], [("real",)] * k, np.array(chosen)


def rayleigh_quotients(V, AV, BV, tags):
    """Alg. 3 step 13: RQ per real column; Eq. lambda_complex for a pair."""
    a = _cdot(V, AV)
    b = _cdot(V, BV)
    lam = a / b
    R_idx = [j for j, t in enumerate(tags) if t[0] == "pairR"]
    I_idx = [j for j, t in enumerate(tags) if t[0] == "pairI"]
    for jr, ji in zip(R_idx, I_idx):
        pl = (a[jr] + a[ji]) / (b[jr] + b[ji])
        lam[jr] = lam[ji] = pl
    return lam, b


def wanted_order(lam, sigma):
    """Column order by distance to sigma, ties by the smaller value."""
    return np.lexsort((lam, np.abs(lam - sigma)))


def relative_residuals(R, lam, BV):
    return np.linalg.norm(R, axis=0) / (np.maximum(np.abs(lam), 1.0) * np.linalg.norm(BV, axis=0))


def bplhr(A, B, T, sigma, k, V0, tol=1e-8, maxit=1000, real=None, s_vectors=True,
          lock=True, plain=False, extraction="tharm", callback=None):
    """Block PLHR for the k eigenpairs of A v = lam B v nearest sigma.

    A, B: sparse/dense Hermitian matrices (B = None means I), T: callable
    Hermitian positive definite preconditioner on n x c blocks (None means I),
    V0: n x k' starting block (k' = k + 1 in real arithmetic, else k).
    plain=True recomputes AZ, BZ and T(A - sigma B)Z explicitly each iteration
    instead of carrying them by linear updates (a self-check on small n).
    extraction='harm' replaces the T-harmonic test space by the standard
    harmonic one (T = I in the Petrov-Galerkin condition, Section 5.1)."""
    if real is None:
        real = not (np.iscomplexobj(V0) or np.iscomplexobj(A if not hasattr(A, "dtype") else np.zeros(1, A.dtype)))
    V = np.array(V0, dtype=np.float64 if real else np.complex128, copy=True)
    n, kp = V.shape
    if kp < k:
        raise ValueError("V0 has fewer columns than k")
    AV = A @ V
    BV = _bmul(B, V)
    b = _cdot(V, BV)
    s = np.sqrt(b)
    V, AV, BV = V / s, AV / s, BV / s
    lam = _cdot(V, AV)
    QV = _tmul(T, AV - sigma * BV)
    P = AP = BP = QP = None
    history = []
    converged = False
    it = 0
    for it in range(maxit + 1):
        if plain:
            AV = A @ V
            BV = _bmul(B, V)
            QV = _tmul(T, AV - sigma * BV)
            if P is not None:
                AP = A @ P
                BP = _bmul(B, P)
                QP = _tmul(T, AP - sigma * BP)
        R = AV - BV * lam[None, :]
        rel = relative_residuals(R, lam, BV)
        order = wanted_order(lam, sigma)
        want = order[:k]
        rec = {"it": it, "lam": lam[order].copy(), "rel": rel[order].copy()}
        history.append(rec)
        if callback is not None:
            callback(rec)
        if np.all(rel[want] <= tol):
            # the returned pairs come from the final standard Rayleigh-Ritz step:
            # accept only if they meet tol, else carry on from the rotated block
            fin = final_rayleigh_ritz(A, B, V, sigma, k)
            if np.all(fin[2] <= tol):
                converged = True
                break
            C = fin[3]
            V, AV, BV, QV = V @ C, AV @ C, BV @ C, QV @ C
            lam = fin[4]
            R = AV - BV * lam[None, :]
            rel = relative_residuals(R, lam, BV)
        if it == maxit:
            break
        act = ~(rel <= tol) if lock else np.ones(kp, dtype=bool)
        lam_a = lam[act]
        W = _tmul(T, R[:, act])
        AW = A @ W
        BW = _bmul(B, W)
        QW = _tmul(T, AW - sigma * BW)
        blocks = [(V, AV, BV, QV), (W, AW, BW, QW)]
        if s_vectors:
            S = _tmul(T, AW - BW * lam_a[None, :])
            AS = A @ S
            BS = _bmul(B, S)
            QS = _tmul(T, AS - sigma * BS)
            blocks.append((S, AS, BS, QS))
        if P is not None:
            blocks.append((P, AP, BP, QP))
        basis = []
        sizes = []
        for blk in blocks:
            ob = orthonormalize_block(blk, basis)
            sizes.append(ob[0].shape[1])
            if ob[0].shape[1] > 0:
                basis.append(ob)
        Zh = np.hstack([b_[0] for b_ in basis])
        AZh = np.hstack([b_[1] for b_ in basis])
        BZh = np.hstack([b_[2] for b_ in basis])
        QZh = np.hstack([b_[3] for b_ in basis])
        U = AZh - sigma * BZh
        if extraction == "tharm":
            GL = _adj(U) @ QZh
            GR = _adj(QZh) @ BZh
        else:
            GL = _adj(U) @ U
            GR = _adj(U) @ BZh
        GL = 0.5 * (GL + _adj(GL))
        xi, Y = tharmonic_extract(GL, GR)
        if real:
            Yp, tags, _ = select_real(xi, Y, kp)
        else:
            Yp, tags, _ = select_complex(xi, Y, kp)
        rec["tags"] = [t[0] for t in tags]
        nv = sizes[0]
        Yv, Yr = Yp[:nv], Yp[nv:]
        P = Zh[:, nv:] @ Yr
        AP = AZh[:, nv:] @ Yr
        BP = BZh[:, nv:] @ Yr
        QP = QZh[:, nv:] @ Yr
        V = Zh[:, :nv] @ Yv + P
        AV = AZh[:, :nv] @ Yv + AP
        BV = BZh[:, :nv] @ Yv + BP
        QV = QZh[:, :nv] @ Yv + QP
        lam, bnorm = rayleigh_quotients(V, AV, BV, tags)
        s = np.sqrt(bnorm)
        V, AV, BV, QV = V / s, AV / s, BV / s, QV / s
    theta, V, res, _, _ = final_rayleigh_ritz(A, B, V, sigma, k)
    return Result(eigvals=theta, eigvecs=V, residuals=res, converged=converged,
                  iterations=it, history=history)


def refined_coefficients(Zh, AZh, BZh, lam_t, T):
    """Eq. rRR on the basis Zh (images AZh, BZh; BZh = Zh for B = I): the
    coefficient vector y of v = Zh y minimising ||(A - lam_t B) v||_T / ||v||_B,
    i.e. the eigenvector of X* T X y = theta^2 Zh* B Zh y, X = (A - lam_t B) Zh,
    for the smallest theta^2."""
    X = AZh - lam_t * BZh
    TX = _tmul(T, X)
    G = _adj(X) @ TX
    G = 0.5 * (G + _adj(G))
    Gz = _adj(Zh) @ BZh
    theta2, Y = sla.eigh(G, 0.5 * (Gz + _adj(Gz)))
    return Y[:, [0]]                       # smallest theta^2 (eigh sorts ascending)


def plmr(A, B, T, v0, tol=1e-8, maxit=1000, callback=None):
    """Preconditioned locally minimal residual method (Section 3.3, "Possible
    variations"): the single-vector trial space of Algorithm 1,
    Z = [v, w, s, p] with w = T(Av - lam Bv) and s = T(Aw - lam Bw), and the
    refinement extraction of Eq. rRR in place of the T-harmonic one: the new
    v minimises ||(A - lam~ B) v||_T over the unit B-norm vectors of span(Z),
    lam~ the current Rayleigh quotient, i.e. v = Z y with y the eigenvector of
        Z*(A - lam~ B) T (A - lam~ B) Z y = theta^2 Z*BZ y
    for the smallest theta^2; p = the w, s, p part of Z y (as in Algorithm 1
    steps 6-7).  Z is B-orthonormalised blockwise first (as in bplhr).  Real
    or complex v0 (n x 1 or n).  Returns a Result with the final eigenpair
    (no final Rayleigh-Ritz: the block has one column)."""
    v = np.array(v0, dtype=np.complex128 if np.iscomplexobj(v0) else np.float64, copy=True).reshape(-1, 1)
    Av, Bv = A @ v, _bmul(B, v)
    nb = np.sqrt(_cdot(v, Bv))
    v, Av, Bv = v / nb, Av / nb, Bv / nb
    lam = _cdot(v, Av)
    P = AP = BP = None
    history = []
    converged = False
    it = 0
    for it in range(maxit + 1):
        R = Av - Bv * lam[None, :]
        rel = relative_residuals(R, lam, Bv)
        rec = {"it": it, "lam": lam.copy(), "rel": rel.copy()}
        history.append(rec)
        if callback is not None:
            callback(rec)
        if rel[0] <= tol:
            converged = True
            break
        if it == maxit:
            break
        W = _tmul(T, R)
        AW, BW = A @ W, _bmul(B, W)
        S = _tmul(T, AW - BW * lam[None, :])
        AS, BS = A @ S, _bmul(B, S)
        # blockwise B-orthonormal basis of [v w s p] with the A and B images
        # (the T images are formed below for the fixed lam~)
        blocks = [(v, Av, Bv, Bv), (W, AW, BW, BW), (S, AS, BS, BS)]
        if P is not None:
            blocks.append((P, AP, BP, BP))
        basis, sizes = [], []
        for blk in blocks:
            ob = orthonormalize_block(blk, basis)
            sizes.append(ob[0].shape[1])
            if ob[0].shape[1] > 0:
                basis.append(ob)
        Zh = np.hstack([b_[0] for b_ in basis])
        AZh = np.hstack([b_[1] for b_ in basis])
        BZh = np.hstack([b_[2] for b_ in basis])
        y = refined_coefficients(Zh, AZh, BZh, lam[0], T)
        nv = sizes[0]
        P = Zh[:, nv:] @ y[nv:]
        AP, BP = AZh[:, nv:] @ y[nv:], BZh[:, nv:] @ y[nv:]
        v = Zh[:, :nv] @ y[:nv] + P
        Av = AZh[:, :nv] @ y[:nv] + AP
        Bv = BZh[:, :nv] @ y[:nv] + BP
        nb = np.sqrt(_cdot(v, Bv))
        v, Av, Bv, P, AP, BP = v / nb, Av / nb, Bv / nb, P / nb, AP / nb, BP / nb
        lam = _cdot(v, Av)
    # explicit products for the reported residual
    AVx, BVx = A @ v, _bmul(B, v)
    res = relative_residuals(AVx - BVx * lam[None, :], lam, BVx)
    return Result(eigvals=lam, eigvecs=v, residuals=res, converged=converged, iterations=it, history=history)


def final_rayleigh_ritz(A, B, V, sigma, k):
    """Standard Rayleigh-Ritz with respect to V (Alg. 2 step 12, Alg. 3 step 16):
    V*AV c = theta V*BV c.  Returns (theta of the k nearest sigma, their Ritz
    vectors, their relative residuals from explicit products with A and B,
    the full coefficient matrix C, all Ritz values) ."""
    AVx = A @ V
    BVx = _bmul(B, V)
    GA = _adj(V) @ AVx
    GB = _adj(V) @ BVx
    GA = 0.5 * (GA + _adj(GA))
    GB = 0.5 * (GB + _adj(GB))
    theta_all, C = sla.eigh(GA, GB)
    order = wanted_order(theta_all, sigma)
    C = C[:, order]
    theta_all = theta_all[order]
    Vk = V @ C[:, :k]
    theta = theta_all[:k]
    AVk = A @ Vk
    BVk = _bmul(B, Vk)
    res = relative_residuals(AVk - BVk * theta[None, :], theta, BVk)
    return theta, Vk, res, C, theta_all


def solve_workload(workload, maxit=None, **kw):
    """Convenience: build A, B, T of a workload description and run bplhr."""
    from .operators import model_operator
    from .avmg import preconditioner
    A, B = model_operator(workload)
    T = preconditioner(workload)
    return bplhr(A, B, T, workload.sigma, workload.k, workload.v0(), tol=workload.tol,
                 maxit=workload.maxit if maxit is None else maxit, real=workload.real, **kw)
