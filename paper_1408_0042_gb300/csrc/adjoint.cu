// Eigenvector adjoint for the differentiation extension: for H(V) = -1/2 Lap +
// diag(V) with B-orthonormal eigenvectors v_1..v_k (eigenvalues lambda) and
// the gradients g_k = dL/dv_k of a loss L, first-order perturbation theory
// gives
//     dL/dV = sum_k v_k (.) b_k,
//     b_k = sum_{j != k} v_j (v_j^T g_k) / (lambda_k - lambda_j) - a_k,
// where the in-block sum is explicit and a_k solves (H - lambda_k) a_k =
// P g_k on the orthogonal complement of the block (P = I - V V^T).  The k
// shifted systems are solved together by MINRES (Paige & Saunders 1975; the
// short recurrence for symmetric indefinite systems) on the projected
// operator P (H - lambda_k) P, one set of recurrence scalars per column, with
// the optional symmetric positive definite preconditioner P T P (PMINRES,
// the solver the paper's Section 2 discusses for these singular consistent
// systems); the host reads the two inner products of each step.
#include <cmath>
#include <cstring>
#include <vector>

#include "blockops.h"
#include "plhr_internal.h"

namespace plhr {
namespace {

constexpr int kMaxK = 16;
constexpr int kCrossRows = 32;

struct Coef {
    double a[kMaxK];
};

// partial[block][j][c] = sum over the block's rows of V[i][j] X[i][c]
__global__ void __launch_bounds__(256) k_cross(int64_t n, int k, const double* __restrict__ V, int64_t ldv,
                                               const double* __restrict__ X, int64_t ldx,
                                               double* __restrict__ partial) {
    __shared__ double sv[kCrossRows][kMaxK], sx[kCrossRows][kMaxK];
    const int t = threadIdx.x;
    const int j = t / kMaxK, c = t % kMaxK;
    double acc = 0.0;
    const int64_t nchunks = (n + kCrossRows - 1) / kCrossRows;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t r0 = ch * kCrossRows;
        __syncthreads();
        for (int e = t; e < kCrossRows * k; e += blockDim.x) {
            const int r = e / k, q = e - r * k;
            const int64_t row = r0 + r;
            sv[r][q] = row < n ? V[row * ldv + q] : 0.0;
            sx[r][q] = row < n ? X[row * ldx + q] : 0.0;
        }
        __syncthreads();
        if (j < k && c < k)
            for (int r = 0; r < kCrossRows; ++r) acc = fma(sv[r][j], sx[r][c], acc);
    }
    if (j < k && c < k) partial[(int64_t)blockIdx.x * k * k + j * k + c] = acc;
}

__global__ void k_sum(int nb, int width, const double* __restrict__ partial, double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= width) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[(int64_t)b * width + j];
    out[j] = s;
}

// X[i][c] += alpha * sum_j V[i][j] G[j][c]   (G: k x k on the device)
__global__ void __launch_bounds__(256) k_add_vg(int64_t n, int k, const double* __restrict__ V, int64_t ldv,
                                                const double* __restrict__ G, double alpha, double* __restrict__ X,
                                                int64_t ldx) {
    const int64_t total = n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k;
        const int c = (int)(e - i * k);
        double s = 0.0;
        for (int j = 0; j < k; ++j) s = fma(V[i * ldv + j], G[j * k + c], s);
        X[i * ldx + c] += alpha * s;
    }
}

// out = a .* x + b .* y + c .* z  per column (coefficient vectors of length k;
// y, z may be null)
__global__ void __launch_bounds__(256) k_lin3(int64_t n, int k, Coef a, const double* __restrict__ x, Coef b,
                                              const double* __restrict__ y, Coef c, const double* __restrict__ z,
                                              double* __restrict__ out) {
    const int64_t total = n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e % k);
        double s = a.a[q] * x[e];
        if (y) s = fma(b.a[q], y[e], s);
        if (z) s = fma(c.a[q], z[e], s);
        out[e] = s;
    }
}

// out[i] = sum_c V[i][c] B[i][c]
__global__ void __launch_bounds__(256) k_rowdot(int64_t n, int k, const double* __restrict__ V, int64_t ldv,
                                                const double* __restrict__ B, double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < k; ++c) s = fma(V[i * ldv + c], B[i * k + c], s);
        out[i] = s;
    }
}

int nblocks(int64_t work) { return grid_size_for(work, 256, sm_count() * 8); }

}  // namespace
}  // namespace plhr

using namespace plhr;

namespace plhr {
plhr_status prec_reserve(plhr_prec* T, int nc, int64_t extra_doubles);
}

extern "C" plhr_status plhr_eigvec_adjoint(const plhr_op* A, plhr_prec* T, int k, const double* lam, const double* V,
                                           int64_t ldv, const double* G, int64_t ldg, double tol, int maxit,
                                           double* grad, int* iterations, void* stream) {
    clear_error();
    if (!A || k < 1 || k > kMaxK || !lam || !V || !G || !grad || ldv < k || ldg < k || !(tol > 0) || maxit < 1) {
        set_error("plhr_eigvec_adjoint: invalid argument (1 <= k <= %d)", kMaxK);
        return PLHR_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = A->g.n();
    const int64_t nk = n * k;
    if (T) {
        if (prec_size(T) != n) {
            set_error("plhr_eigvec_adjoint: preconditioner size does not match A");
            return PLHR_EINVAL;
        }
        PLHR_TRY(prec_reserve(T, k, 0));
    }
    const int cross_blocks = sm_count() * 2;
    const int res_blocks = residual_blocks(k);
    // device workspace: 9 n x k blocks, the k x k cross matrix and partials
    double* ws = nullptr;
    const int64_t need = 9 * nk + k * k + (int64_t)cross_blocks * k * k + (int64_t)res_blocks * 2 * k + 4 * kMaxK;
    if (cudaMallocAsync(&ws, sizeof(double) * need, s) != cudaSuccess) {
        set_error("plhr_eigvec_adjoint: device allocation failed");
        return PLHR_ENOMEM;
    }
    struct Free {
        double* p;
        cudaStream_t s;
        ~Free() { cudaStreamSynchronize(s); cudaFree(p); }
    } fr{ws, s};
    double* q = ws;
    double *x = q; q += nk;
    double *v = q; q += nk;
    double *y = q; q += nk;
    double *r1 = q; q += nk;
    double *r2 = q; q += nk;
    double *w = q; q += nk;
    double *w1 = q; q += nk;
    double *w2 = q; q += nk;
    double *bb = q; q += nk;
    double *Gc = q; q += k * k;
    double *cpart = q; q += (int64_t)cross_blocks * k * k;
    double *rpart = q; q += (int64_t)res_blocks * 2 * k;
    double *dots = q; q += 2 * kMaxK;
    double *dlam = q; q += kMaxK;
    PLHR_TRY_CUDA(cudaMemcpyAsync(dlam, lam, sizeof(double) * k, cudaMemcpyHostToDevice, s));

    // X <- X - V (V^T X)  (X dense n x k)
    auto project = [&](double* X) -> plhr_status {
        k_cross<<<cross_blocks, 256, 0, s>>>(n, k, V, ldv, X, k, cpart);
        k_sum<<<(k * k + 127) / 128, 128, 0, s>>>(cross_blocks, k * k, cpart, Gc);
        k_add_vg<<<nblocks(nk), 256, 0, s>>>(n, k, V, ldv, Gc, -1.0, X, k);
        count_launches(3);
        PLHR_TRY_CUDA(cudaGetLastError());
        return PLHR_OK;
    };
    auto coldots = [&](const double* X, const double* Y, double* host) -> plhr_status {
        PLHR_TRY_CUDA(column_dots(n, k, X, k, Y, k, rpart, dots, s));
        PLHR_TRY_CUDA(cudaMemcpyAsync(host, dots, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, s));
        PLHR_TRY_CUDA(cudaStreamSynchronize(s));
        return PLHR_OK;
    };
    Coef one{}, zero{};
    for (int c = 0; c < kMaxK; ++c) { one.a[c] = 1.0; zero.a[c] = 0.0; }
    // Y = P T X (or P X = X without T; X is in the complement already)
    auto precond = [&](const double* X, double* Y) -> plhr_status {
        if (!T) {
            PLHR_TRY_CUDA(cudaMemcpyAsync(Y, X, sizeof(double) * nk, cudaMemcpyDeviceToDevice, s));
            return PLHR_OK;
        }
        PLHR_TRY(prec_apply64(T, k, X, k, Y, T->work, s));
        return project(Y);
    };

    // in-block part of b: V C with C[j][c] = (v_j^T g_c) / (lambda_c - lambda_j), j != c
    PLHR_TRY_CUDA(cudaMemcpy2DAsync(r1, sizeof(double) * k, G, sizeof(double) * ldg, sizeof(double) * k, n,
                                    cudaMemcpyDeviceToDevice, s));
    k_cross<<<cross_blocks, 256, 0, s>>>(n, k, V, ldv, r1, k, cpart);
    k_sum<<<(k * k + 127) / 128, 128, 0, s>>>(cross_blocks, k * k, cpart, Gc);
    count_launches(2);
    std::vector<double> hg(k * k), hc(k * k, 0.0);
    PLHR_TRY_CUDA(cudaMemcpyAsync(hg.data(), Gc, sizeof(double) * k * k, cudaMemcpyDeviceToHost, s));
    PLHR_TRY_CUDA(cudaStreamSynchronize(s));
    const double lscale = std::fmax(1.0, std::fabs(lam[0]));
    for (int j = 0; j < k; ++j)
        for (int c = 0; c < k; ++c) {
            const double d = lam[c] - lam[j];
            // a (numerically) repeated eigenvalue has no well-defined eigenvector
            // derivative inside its eigenspace: that term is left out
            if (j != c && std::fabs(d) > 1e-12 * lscale) hc[j * k + c] = hg[j * k + c] / d;
        }
    PLHR_TRY_CUDA(cudaMemcpyAsync(Gc, hc.data(), sizeof(double) * k * k, cudaMemcpyHostToDevice, s));
    PLHR_TRY_CUDA(cudaMemsetAsync(bb, 0, sizeof(double) * nk, s));
    k_add_vg<<<nblocks(nk), 256, 0, s>>>(n, k, V, ldv, Gc, 1.0, bb, k);
    count_launches(1);
    PLHR_TRY_CUDA(cudaGetLastError());

    // MINRES on P (H - lambda_c) P a = P g_c (unpreconditioned), all columns at once
    std::vector<double> hd(2 * k), gnorm(k);
    PLHR_TRY(coldots(r1, r1, hd.data()));
    for (int c = 0; c < k; ++c) gnorm[c] = std::sqrt(std::fmax(hd[c], 0.0));
    PLHR_TRY(project(r1));                                   // r1 = P g
    PLHR_TRY(coldots(r1, r1, hd.data()));
    std::vector<double> pnorm(k);
    for (int c = 0; c < k; ++c) pnorm[c] = std::sqrt(std::fmax(hd[c], 0.0));
    PLHR_TRY_CUDA(cudaMemcpyAsync(r2, r1, sizeof(double) * nk, cudaMemcpyDeviceToDevice, s));
    PLHR_TRY(precond(r1, y));                                // y = P T r1
    PLHR_TRY_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * nk, s));
    PLHR_TRY_CUDA(cudaMemsetAsync(w, 0, sizeof(double) * nk, s));
    PLHR_TRY_CUDA(cudaMemsetAsync(w2, 0, sizeof(double) * nk, s));
    PLHR_TRY(coldots(r1, y, hd.data()));
    std::vector<double> beta1(k), beta(k), oldb(k, 0.0), dbar(k, 0.0), epsln(k, 0.0), phibar(k), cs(k, -1.0),
        sn(k, 0.0), alfa(k);
    // a column whose projected right-hand side is at rounding level of g_c
    // (g_c inside the block's span) has a_c = 0
    bool all_zero = true;
    std::vector<bool> done(k, false);
    for (int c = 0; c < k; ++c) {
        beta1[c] = std::sqrt(std::fmax(hd[c], 0.0));
        beta[c] = beta1[c];
        phibar[c] = beta1[c];
        done[c] = !(pnorm[c] > 1e-14 * gnorm[c]) || !(beta1[c] > 0.0);
        if (!done[c]) all_zero = false;
    }
    int itn = 0;
    bool converged = all_zero, finite = true;
    while (!converged && itn < maxit) {
        ++itn;
        // converged columns are frozen: every coefficient of theirs is zero, so
        // their v, y, w stay zero and x keeps its value
        Coef inv{}, c1{}, c2{};
        for (int c = 0; c < k; ++c) inv.a[c] = (!done[c] && beta[c] > 0.0) ? 1.0 / beta[c] : 0.0;
        k_lin3<<<nblocks(nk), 256, 0, s>>>(n, k, inv, y, zero, nullptr, zero, nullptr, v);   // v = y / beta
        count_launches(1);
        // y = P (H - lambda) v  (v is in the complement)
        PLHR_TRY_CUDA(lap_apply_shifts(A->g, k, v, k, nullptr, 0, y, k, dlam, nullptr, 0, 0.0, s));
        PLHR_TRY(project(y));
        if (itn >= 2) {
            for (int c = 0; c < k; ++c) c1.a[c] = (!done[c] && oldb[c] > 0.0) ? -beta[c] / oldb[c] : 0.0;
            k_lin3<<<nblocks(nk), 256, 0, s>>>(n, k, one, y, c1, r1, zero, nullptr, y);
            count_launches(1);
        }
        PLHR_TRY(coldots(v, y, hd.data()));
        for (int c = 0; c < k; ++c) {
            alfa[c] = hd[c];
            c2.a[c] = (!done[c] && beta[c] > 0.0) ? -alfa[c] / beta[c] : 0.0;
        }
        k_lin3<<<nblocks(nk), 256, 0, s>>>(n, k, one, y, c2, r2, zero, nullptr, y);
        count_launches(1);
        std::swap(r1, r2);                                    // r1 <- r2, r2 <- y
        std::swap(r2, y);
        PLHR_TRY(precond(r2, y));                             // y = P T r2
        PLHR_TRY(coldots(r2, y, hd.data()));
        Coef dn{}, dc{}, ph{};
        converged = true;
        for (int c = 0; c < k; ++c) {
            if (done[c]) {
                dn.a[c] = 0.0; dc.a[c] = 0.0; ph.a[c] = 0.0; inv.a[c] = 0.0;
                continue;
            }
            if (!std::isfinite(hd[c]) || !std::isfinite(alfa[c])) finite = false;
            oldb[c] = beta[c];
            beta[c] = std::sqrt(std::fmax(hd[c], 0.0));
            const double oldeps = epsln[c];
            const double delta = cs[c] * dbar[c] + sn[c] * alfa[c];
            const double gbar = sn[c] * dbar[c] - cs[c] * alfa[c];
            epsln[c] = sn[c] * beta[c];
            dbar[c] = -cs[c] * beta[c];
            double gamma = std::sqrt(gbar * gbar + beta[c] * beta[c]);
            gamma = std::fmax(gamma, 1e-300);
            cs[c] = gbar / gamma;
            sn[c] = beta[c] / gamma;
            const double phi = cs[c] * phibar[c];
            phibar[c] = sn[c] * phibar[c];
            // w <- (v - oldeps w1 - delta w2) / gamma with w1 <- w2, w2 <- w
            dn.a[c] = -oldeps / gamma;
            dc.a[c] = -delta / gamma;
            ph.a[c] = phi;
            inv.a[c] = 1.0 / gamma;
            if (phibar[c] <= tol * beta1[c]) done[c] = true;
        }
        for (int c = 0; c < k; ++c) converged = converged && done[c];
        std::swap(w1, w2);     // w1 <- old w2
        std::swap(w2, w);      // w2 <- old w; w (old w1 storage) is overwritten next
        k_lin3<<<nblocks(nk), 256, 0, s>>>(n, k, inv, v, dn, w1, dc, w2, w);
        k_lin3<<<nblocks(nk), 256, 0, s>>>(n, k, one, x, ph, w, zero, nullptr, x);
        count_launches(2);
        PLHR_TRY_CUDA(cudaGetLastError());
        if (!finite) {
            if (iterations) *iterations = itn;
            set_error("plhr_eigvec_adjoint: NaN or Inf in MINRES at iteration %d", itn);
            return PLHR_ENAN;
        }
    }
    // b = in-block part - a; grad = sum_c V(:,c) .* b(:,c)
    Coef mone{};
    for (int c = 0; c < kMaxK; ++c) mone.a[c] = -1.0;
    k_lin3<<<nblocks(nk), 256, 0, s>>>(n, k, one, bb, mone, x, zero, nullptr, bb);
    k_rowdot<<<nblocks(n), 256, 0, s>>>(n, k, V, ldv, bb, grad);
    count_launches(2);
    PLHR_TRY_CUDA(cudaGetLastError());
    if (iterations) *iterations = itn;
    if (!converged) {
        set_error("plhr_eigvec_adjoint: MINRES did not reach tol in %d iterations", maxit);
        return PLHR_ENOTCONV;
    }
    return PLHR_OK;
}
