// Single-vector iteration with the refinement extraction (Section 3.3,
// "Possible variations", Eq. rRR): the preconditioned locally minimal
// residual method.  The trial space is Algorithm 1's Z = [v, w, s, p] with
// w = T(Av - lam Bv), s = T(Aw - lam Bw); the new v minimises
// ||(A - lam B) v||_T over the unit B-norm vectors of span(Z), lam the current
// Rayleigh quotient:
//     X = (A - lam B) Z,   X^T T X y = theta^2 Z^T B Z y,   smallest theta^2,
//     p <- Z[w s p] y[w s p],   v <- y_v v + p,   v <- v / ||v||_B.
// The T images need no extra preconditioner applications for v and w:
// T (A - lam B) v = w and T (A - lam B) w = s; two more give T X for s and p.
// Every step runs in the library's kernels (stencil/CSR products, the
// preconditioner, the multi-Gram pass, the coefficient update); the 4 x 4
// symmetric-definite problem is solved on the device by one warp.
#include <chrono>
#include <cmath>
#include <vector>

#include "blockops.h"
#include "plhr_internal.h"

namespace plhr {
plhr_status prec_reserve(plhr_prec* T, int nc, int64_t extra_doubles);

namespace {

constexpr int kM = 4;

double wall_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// dots = [v.Av, v.v | v.Bv, ..] -> lam = v.Av / v.Bv, scale = 1 / sqrt(v.Bv)
__global__ void k_plmr_rq(const double* __restrict__ da, const double* __restrict__ db, double* __restrict__ sc) {
    if (threadIdx.x != 0) return;
    const double a = da[0], b = db ? db[0] : da[1];
    sc[0] = a / b;
    sc[1] = 1.0 / sqrt(b);
}

// x_i *= scale for the listed vectors (null entries skipped)
struct Six {
    double* p[6];
};
__global__ void k_plmr_scale(int64_t n, const double* __restrict__ sc, Six v) {
    const double f = sc[1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int j = 0; j < 6; ++j)
            if (v.p[j]) v.p[j][i] *= f;
}

// The refined extraction on the m x m Grams (m <= 4), one thread:
// Gzz = Z^T B Z, G = X^T T X.  With D = diag(Gzz)^{-1/2}, the Cholesky of
// D Gzz D with column dropping (pivot^2 < 1e-12: the column is numerically in
// the span of the earlier ones), C = L^{-1} D G D L^{-T} and its eigenvectors
// by cyclic Jacobi; y = D L^{-T} z for the smallest eigenvalue.  Out:
// Cp (m) = y with the v entry zeroed, Cvv (1) = y_v, st = [ok, kept columns].
__global__ void k_plmr_extract(int m, const double* __restrict__ Gzz, const double* __restrict__ G,
                               double* __restrict__ Cp, double* __restrict__ Cvv, int* __restrict__ st) {
    if (threadIdx.x != 0) return;
    double d[kM], S[kM][kM], K[kM][kM], L[kM][kM];
    int keep[kM], nk = 0;
    for (int i = 0; i < m; ++i) d[i] = Gzz[i * m + i] > 0.0 ? 1.0 / sqrt(Gzz[i * m + i]) : 0.0;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            S[i][j] = d[i] * Gzz[i * m + j] * d[j];
            K[i][j] = 0.5 * d[i] * (G[i * m + j] + G[j * m + i]) * d[j];
        }
    // Cholesky of S on the kept columns (lower L, row = kept index)
    for (int j = 0; j < m; ++j) {
        if (d[j] == 0.0) continue;
        double row[kM];
        for (int q = 0; q < nk; ++q) {
            double t = S[j][keep[q]];
            for (int r = 0; r < q; ++r) t -= row[r] * L[q][r];
            row[q] = t / L[q][q];
        }
        double pv = S[j][j];
        for (int q = 0; q < nk; ++q) pv -= row[q] * row[q];
        if (!(pv > 1e-12)) continue;
        for (int q = 0; q < nk; ++q) L[nk][q] = row[q];
        L[nk][nk] = sqrt(pv);
        for (int q = nk + 1; q < kM; ++q) L[nk][q] = 0.0;
        keep[nk++] = j;
    }
    if (nk == 0) {
        st[0] = 0;
        st[1] = 0;
        return;
    }
    // C = L^{-1} Kk L^{-T}, Kk = K on the kept columns
    double M1[kM][kM], C[kM][kM];
    for (int c = 0; c < nk; ++c)          // M1 = L^{-1} Kk (forward substitution per column)
        for (int i = 0; i < nk; ++i) {
            double t = K[keep[i]][keep[c]];
            for (int q = 0; q < i; ++q) t -= L[i][q] * M1[q][c];
            M1[i][c] = t / L[i][i];
        }
    for (int r = 0; r < nk; ++r)          // C = M1 L^{-T}: C L^T = M1, row by row
        for (int i = 0; i < nk; ++i) {
            double t = M1[r][i];
            for (int q = 0; q < i; ++q) t -= C[r][q] * L[i][q];
            C[r][i] = t / L[i][i];
        }
    for (int i = 0; i < nk; ++i)
        for (int j = i + 1; j < nk; ++j) C[i][j] = C[j][i] = 0.5 * (C[i][j] + C[j][i]);
    // cyclic Jacobi: C = Q diag Q^T
    double Q[kM][kM];
    for (int i = 0; i < nk; ++i)
        for (int j = 0; j < nk; ++j) Q[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < nk; ++i)
            for (int j = 0; j < nk; ++j) {
                tot += C[i][j] * C[i][j];
                if (i != j) off += C[i][j] * C[i][j];
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < nk; ++p)
            for (int q = p + 1; q < nk; ++q) {
                if (C[p][q] == 0.0) continue;
                const double th = (C[q][q] - C[p][p]) / (2.0 * C[p][q]);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int r = 0; r < nk; ++r) {   // columns p, q
                    const double a = C[r][p], b = C[r][q];
                    C[r][p] = c * a - sn * b;
                    C[r][q] = sn * a + c * b;
                }
                for (int r = 0; r < nk; ++r) {   // rows p, q
                    const double a = C[p][r], b = C[q][r];
                    C[p][r] = c * a - sn * b;
                    C[q][r] = sn * a + c * b;
                }
                for (int r = 0; r < nk; ++r) {
                    const double a = Q[r][p], b = Q[r][q];
                    Q[r][p] = c * a - sn * b;
                    Q[r][q] = sn * a + c * b;
                }
            }
    }
    int best = 0;
    for (int i = 1; i < nk; ++i)
        if (C[i][i] < C[best][best]) best = i;
    // y_kept = L^{-T} z (back substitution), y = D y_full
    double yk[kM];
    for (int i = nk - 1; i >= 0; --i) {
        double t = Q[i][best];
        for (int q = i + 1; q < nk; ++q) t -= L[q][i] * yk[q];
        yk[i] = t / L[i][i];
    }
    double y[kM] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < nk; ++i) y[keep[i]] = yk[i] * d[keep[i]];
    Cvv[0] = y[0];
    Cp[0] = 0.0;
    for (int i = 1; i < m; ++i) Cp[i] = y[i];
    st[0] = 1;
    st[1] = nk;
}

}  // namespace

plhr_status plmr_solve(const plhr_op* A, const plhr_op* B, plhr_prec* T, double tol, const plhr_options& opt,
                       double* eigvals, double* eigvecs, int64_t ldv, plhr_info* info, cudaStream_t s,
                       double t_start) {
    const Grid& g = A->g;
    const int64_t n = g.n();
    const bool hasB = B != nullptr;
    if (n < kM) {
        set_error("plhr_solve: n too small");
        return PLHR_EINVAL;
    }
    // ---------------------------------------------------------------- workspace
    enum { V, AV, BV, P, AP, BP, R, W, AW, BW, XW, S, AS, BS, XS, TXS, XP, TXP, NV };
    double* big = nullptr;
    const int64_t parts = (int64_t)reduce_blocks() * 3 * kM * kM + (int64_t)residual_blocks(1) * 2 + 64;
    const int64_t small = 3 * kM * kM + 2 * kM + 64;
    if (cudaMallocAsync(&big, sizeof(double) * ((int64_t)NV * n + parts + small), s) != cudaSuccess) {
        set_error("plhr_solve: device allocation failed");
        return PLHR_ENOMEM;
    }
    int* dst = nullptr;
    if (cudaMallocAsync(&dst, sizeof(int) * 4, s) != cudaSuccess) {
        cudaFreeAsync(big, s);
        set_error("plhr_solve: device allocation failed");
        return PLHR_ENOMEM;
    }
    struct Free {
        double* a; int* b; cudaStream_t s;
        ~Free() { cudaStreamSynchronize(s); cudaFree(a); cudaFree(b); }
    } fr{big, dst, s};
    double* vec[NV];
    for (int i = 0; i < NV; ++i) vec[i] = big + (int64_t)i * n;
    double* part = big + (int64_t)NV * n;
    double* sm = part + parts;
    double* grams = sm;                    // [Z^T B Z | X^T T X | ..]
    double* Cp = grams + 3 * kM * kM;
    double* Cvv = Cp + kM;
    double* sc = Cvv + kM;                 // [lam, scale]
    double* dots = sc + 2;                 // 4 x 2
    double* ones = dots + 8;               // kM
    double* Bv = hasB ? vec[BV] : vec[V];
    double* Bw = hasB ? vec[BW] : vec[W];
    double* Bs = hasB ? vec[BS] : vec[S];
    double* Bp = hasB ? vec[BP] : vec[P];
    {
        const double one4[kM] = {1.0, 1.0, 1.0, 1.0};
        PLHR_TRY_CUDA(cudaMemcpyAsync(ones, one4, sizeof(one4), cudaMemcpyHostToDevice, s));
        PLHR_TRY_CUDA(cudaStreamSynchronize(s));
    }

    // A x (and B x); o = A x - lam B x when o is given (lam on the device)
    auto prod = [&](const double* x, double* ax, double* bx, double* o) -> plhr_status {
        if (!hasB) {
            PLHR_TRY_CUDA(lap_apply_shifts(g, 1, x, 1, ax, 1, o, 1, sc, nullptr, 0, 0.0, s));
            return PLHR_OK;
        }
        if (q1_same_mesh(g, B->g)) {
            PLHR_TRY_CUDA(q1_pair(g, B->g, 1, x, 1, ax, 1, bx, 1, s));
        } else {
            PLHR_TRY_CUDA(lap_axpby(g, 1, x, 1, ax, 1, 1.0, 0.0, s));
            PLHR_TRY_CUDA(lap_axpby(B->g, 1, x, 1, bx, 1, 1.0, 0.0, s));
        }
        if (o) PLHR_TRY_CUDA(shift_combine(n, 1, ax, 1, bx, 1, sc, o, 1, 0.0, nullptr, 0, s));
        return PLHR_OK;
    };
    auto applyT = [&](const double* r, double* w) -> plhr_status {
        if (!T) {
            PLHR_TRY_CUDA(cudaMemcpyAsync(w, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            return PLHR_OK;
        }
        PhaseScope ps(PH_VCYCLE, s, (double)n);
        PLHR_TRY(prec_apply64(T, 1, r, 1, w, T->work, s));
        return PLHR_OK;
    };
    // lam, scale from the current v; then v and its images scaled to ||v||_B = 1
    auto normalise = [&](bool with_p) -> plhr_status {
        PLHR_TRY_CUDA(column_dots(n, 1, vec[V], 1, vec[AV], 1, part, dots, s));
        if (hasB) PLHR_TRY_CUDA(column_dots(n, 1, vec[V], 1, vec[BV], 1, part, dots + 2, s));
        k_plmr_rq<<<1, 32, 0, s>>>(dots, hasB ? dots + 2 : nullptr, sc);
        count_launches(1);
        PLHR_TRY_CUDA(cudaGetLastError());
        Six six{{vec[V], vec[AV], hasB ? vec[BV] : nullptr, with_p ? vec[P] : nullptr, with_p ? vec[AP] : nullptr,
                 with_p && hasB ? vec[BP] : nullptr}};
        k_plmr_scale<<<grid_size_for(n, 256, sm_count() * 8), 256, 0, s>>>(n, sc, six);
        count_launches(1);
        PLHR_TRY_CUDA(cudaGetLastError());
        return PLHR_OK;
    };

    // ---------------------------------------------------------------- start
    if (opt.v_init)
        PLHR_TRY_CUDA(cudaMemcpy2DAsync(vec[V], sizeof(double), opt.v_init, sizeof(double) * opt.ld_init,
                                        sizeof(double), n, cudaMemcpyDeviceToDevice, s));
    else
        PLHR_TRY_CUDA(seeded_block(n, 1, opt.seed, vec[V], 1, s));
    if (T) PLHR_TRY(prec_reserve(T, 1, 0));
    PLHR_TRY(prod(vec[V], vec[AV], vec[BV], nullptr));
    PLHR_TRY(normalise(false));
    bool have_p = false;
    const double t1 = wall_s();
    plhr_status result = PLHR_ENOTCONV;
    int it = 0, hist = 0;
    double h[4], lam = 0.0, rel = INFINITY;
    for (it = 0; it <= opt.maxit; ++it) {
        // residual r = A v - lam B v and its relative norm
        PLHR_TRY_CUDA(shift_combine(n, 1, vec[AV], 1, Bv, 1, sc, vec[R], 1, 0.0, nullptr, 0, s));
        PLHR_TRY_CUDA(column_dots(n, 1, vec[R], 1, vec[R], 1, part, dots + 4, s));
        PLHR_TRY_CUDA(column_dots(n, 1, Bv, 1, Bv, 1, part, dots + 6, s));
        PLHR_TRY_CUDA(cudaMemcpyAsync(h, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
        PLHR_TRY_CUDA(cudaMemcpyAsync(h + 1, dots + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
        PLHR_TRY_CUDA(cudaMemcpyAsync(h + 2, dots + 6, sizeof(double), cudaMemcpyDeviceToHost, s));
        PLHR_TRY_CUDA(cudaStreamSynchronize(s));
        lam = h[0];
        rel = std::sqrt(h[1]) / (std::fmax(std::fabs(lam), 1.0) * std::sqrt(h[2]));
        if (!std::isfinite(rel)) {
            set_error("plhr_solve: NaN/Inf at iteration %d", it);
            result = PLHR_ENAN;
            break;
        }
        if (opt.history && hist < opt.history_cap) {
            double* rec = opt.history + (size_t)hist * 5;
            rec[0] = it; rec[1] = lam; rec[2] = rel; rec[3] = have_p ? 4 : 3; rec[4] = have_p ? 4 : 3;
            ++hist;
        }
        if (rel <= tol) {
            result = PLHR_OK;
            break;
        }
        if (it == opt.maxit) break;
        // w = T r; s = T(A w - lam B w); X = (A - lam B) [v w s p], T X = [w, s, T xs, T xp]
        PLHR_TRY(applyT(vec[R], vec[W]));
        PLHR_TRY(prod(vec[W], vec[AW], vec[BW], vec[XW]));
        PLHR_TRY(applyT(vec[XW], vec[S]));
        PLHR_TRY(prod(vec[S], vec[AS], vec[BS], vec[XS]));
        PLHR_TRY(applyT(vec[XS], vec[TXS]));
        if (have_p) {
            PLHR_TRY_CUDA(shift_combine(n, 1, vec[AP], 1, Bp, 1, sc, vec[XP], 1, 0.0, nullptr, 0, s));
            PLHR_TRY(applyT(vec[XP], vec[TXP]));
        }
        const int nb = have_p ? 4 : 3;
        Blk<const double> zb[4] = {{vec[V], 1, 1}, {vec[W], 1, 1}, {vec[S], 1, 1}, {vec[P], 1, 1}};
        Blk<const double> xb[4] = {{vec[R], 1, 1}, {vec[XW], 1, 1}, {vec[XS], 1, 1}, {vec[XP], 1, 1}};
        Blk<const double> tb[4] = {{vec[W], 1, 1}, {vec[S], 1, 1}, {vec[TXS], 1, 1}, {vec[TXP], 1, 1}};
        Blk<const double> bb[4] = {{Bv, 1, 1}, {Bw, 1, 1}, {Bs, 1, 1}, {Bp, 1, 1}};
        {
            PhaseScope ps(PH_GRAM, s, 2.0 * n * 3 * nb * nb, 8.0 * n * nb * (hasB ? 4 : 3));
            // U = X - 0 B Z = X: grams = [Z^T B Z | X^T T X | (T X)^T B Z]
            PLHR_TRY_CUDA(multi_gram_b(n, nb, zb, xb, tb, hasB ? bb : nullptr, 0.0, ones, part, grams, s));
        }
        {
            PhaseScope ps(PH_DENSE, s);
            k_plmr_extract<<<1, 32, 0, s>>>(nb, grams, grams + nb * nb, Cp, Cvv, dst);
            count_launches(1);
            PLHR_TRY_CUDA(cudaGetLastError());
        }
        {
            PhaseScope ps(PH_UPDATE, s, 2.0 * n * nb, 8.0 * n * (nb + 2));
            // p = Z Cp (the v entry of Cp is zero), v = v Cvv + p
            PLHR_TRY_CUDA(block_update(n, nb, zb, 1, Cp, Cvv, vec[V], 1, vec[P], 1, nullptr, 0, nullptr, nullptr, s));
        }
        have_p = true;
        PLHR_TRY(prod(vec[V], vec[AV], vec[BV], nullptr));
        PLHR_TRY(prod(vec[P], vec[AP], vec[BP], nullptr));
        PLHR_TRY(normalise(true));
    }
    const double t2 = wall_s();
    // explicit products for the reported residual (v B-normalised, lam its quotient)
    eigvals[0] = lam;
    PLHR_TRY_CUDA(cudaMemcpy2DAsync(eigvecs, sizeof(double) * ldv, vec[V], sizeof(double), sizeof(double), n,
                                    cudaMemcpyDeviceToDevice, s));
    PLHR_TRY_CUDA(cudaStreamSynchronize(s));
    if (info) {
        info->iterations = it;
        info->converged = result == PLHR_OK;
        info->max_rel_residual = rel;
        info->setup_seconds = t1 - t_start;
        info->solve_seconds = t2 - t1;
        info->history_len = hist;
        info->mixed_iterations = 0;
    }
    return result;
}

}  // namespace plhr
