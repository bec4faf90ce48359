// Teter-Payne-Allan preconditioner (Section 5.3: a positive diagonal matrix
// in the plane-wave basis) on a tensor grid, FP64:
//     T = S diag(K(mu / E)) S^T,
//     K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4),
// with S = Sx (x) Sy (x) Sz the orthonormal eigenvectors of the grid's kinetic
// operator -1/2 Lap_h (real Fourier modes on a periodic axis, sine modes on a
// Dirichlet axis), mu = mu_x + mu_y + mu_z their kinetic energies and E one
// fixed reference energy.  T is symmetric positive definite and commutes with
// -1/2 Lap_h.
//
// Application: the FP64 block is split once into double-word values (hi + lo
// FP32 pairs, ~48-bit significands); three forward passes (one per axis, each
// a dense N_a x N_a product along that axis with the double-word matrix in
// shared memory, double-word multiply-adds on the FP32 pipes), the factor
// (a precomputed per-mode table) fused into the last of them, and three
// inverse passes, the last one writing FP64.  GB300 issues FP64 at 1/64 of
// the FP32 rate, so a double-word multiply-add (13 FP32 instructions) costs
// about a fifth of an FP64 one.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dword.h"
#include "plhr_internal.h"

namespace plhr {
namespace {

constexpr int kT = 256;
constexpr int kMaxAxis = 144;   // N_a^2 doubles of shared memory per pass

struct AxisPass {
    int64_t nx, ny, nz;   // grid
    int axis;             // 0 x, 1 y, 2 z
    int N;                // size along the axis
    int64_t stride;       // point stride along the axis
    int nc;
};

double tpa(double x) {
    const double num = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x));
    const double x2 = x * x;
    return num / (num + 16.0 * x2 * x2);
}

// x (double-word, dense [point][nc]) = r (FP64, leading dimension ldr)
__global__ void __launch_bounds__(kT) k_split(int64_t total, int nc, const double* __restrict__ r, int64_t ldr,
                                              dw* __restrict__ x) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t pt;
        int cc;
        split_index(e, nc, pt, cc);
        x[e] = dw_from_double_fast(r[pt * ldr + cc]);
    }
}

// first point of line l along the axis (lines of axis x: (y, z) rows; of
// axis y: (x, z) with x fastest; of axis z: (x, y) with x fastest, so that
// consecutive lines are neighbours in memory)
__device__ __forceinline__ int64_t line_base(const AxisPass& a, int64_t l) {
    if (a.axis == 0) return l * a.nx;
    if (a.axis == 1) return (l / a.nx) * a.nx * a.ny + l % a.nx;
    return l;
}

constexpr int kQ = 4;   // outputs along the axis per thread (register block)

// out[.., q, ..] = sum_j M[j][q] in[.., j, ..] along one axis (M = S for the
// forward transform, S^T for the inverse; in dense [point][nc]), for tiles of
// TL lines: the CTA stages the tile's N x TL x nc inputs in shared memory
// once, and each thread forms kQ outputs of one (line, column) from them.
// SCALE: times the factor K of the output's mode (last forward pass); OUT64:
// FP64 output with leading dimension ldo, else double-word dense
template <bool SCALE, bool OUT64>
__global__ void __launch_bounds__(kT) k_axis(AxisPass a, int TL, const dw* __restrict__ M,
                                             const dw* __restrict__ in, void* __restrict__ out, int64_t ldo,
                                             const dw* __restrict__ K) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = a.N, nc = a.nc;
    dw* sm = reinterpret_cast<dw*>(smraw);   // [N][N]
    dw* tile = sm + N * N;                   // [N][TL][nc]
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) sm[i] = M[i];
    const int64_t L = a.nx * a.ny * a.nz / N;
    const int nqg = (N + kQ - 1) / kQ;
    for (int64_t l0 = (int64_t)blockIdx.x * TL; l0 < L; l0 += (int64_t)gridDim.x * TL) {
        const int nl = (int)(L - l0 < TL ? L - l0 : TL);
        __syncthreads();   // the previous tile is consumed (and M is staged)
        const int tot = N * nl * nc;
        for (int t = threadIdx.x; t < tot; t += blockDim.x) {
            const int c = t % nc, r = t / nc, o = r % nl, j = r / nl;
            tile[(j * TL + o) * nc + c] = in[(line_base(a, l0 + o) + (int64_t)j * a.stride) * nc + c];
        }
        __syncthreads();
        const int items = nqg * nl * nc;
        for (int t = threadIdx.x; t < items; t += blockDim.x) {
            const int c = t % nc, r = t / nc, o = r % nl, qg = r / nl;
            const int q0 = qg * kQ;
            float hi[kQ], lo[kQ];
#pragma unroll
            for (int u = 0; u < kQ; ++u) { hi[u] = 0.0f; lo[u] = 0.0f; }
            if (q0 + kQ <= N) {
                for (int j = 0; j < N; ++j) {
                    const dw x = tile[(j * TL + o) * nc + c];
                    const dw* mr = sm + j * N + q0;
#pragma unroll
                    for (int u = 0; u < kQ; ++u) dw_fma_acc(hi[u], lo[u], mr[u], x);
                }
            } else {
                for (int j = 0; j < N; ++j) {
                    const dw x = tile[(j * TL + o) * nc + c];
#pragma unroll
                    for (int u = 0; u < kQ; ++u)
                        if (q0 + u < N) dw_fma_acc(hi[u], lo[u], sm[j * N + q0 + u], x);
                }
            }
            const int64_t base = line_base(a, l0 + o);
#pragma unroll
            for (int u = 0; u < kQ; ++u) {
                if (q0 + u >= N) break;
                const int64_t pt = base + (int64_t)(q0 + u) * a.stride;
                dw v = dw_fast_two_sum(hi[u], lo[u]);
                if (SCALE) v = dw_mul(v, K[pt]);
                if (OUT64) static_cast<double*>(out)[pt * ldo + c] = dw_to_double_fast(v);
                else static_cast<dw*>(out)[pt * nc + c] = v;
            }
        }
    }
}

// shared memory of one k_axis launch and its tile height (lines per CTA)
constexpr int kAxisShm = 200 * 1024;
int tile_lines(int N, int nc) {
    const int64_t room = (int64_t)kAxisShm - (int64_t)sizeof(dw) * N * N;
    int64_t tl = room / ((int64_t)sizeof(dw) * N * nc);
    if (tl > 8) tl = 8;
    return (int)(tl < 1 ? 1 : tl);
}

int nblk(int64_t total) { return grid_size_for(total, kT, sm_count() * 8); }

// orthonormal eigenvectors S[p][m] and eigenvalues mu (times 1/2 scale of the
// kinetic operator folded in by the caller) of the 1D second difference
void axis_basis(int64_t N, bool periodic, std::vector<double>& S, std::vector<double>& mu) {
    S.assign(N * N, 0.0);
    mu.assign(N, 0.0);
    if (!periodic) {
        for (int64_t m = 0; m < N; ++m) {
            const double th = (m + 1) * M_PI / (N + 1);
            mu[m] = 2.0 - 2.0 * std::cos(th);
            for (int64_t p = 0; p < N; ++p) S[p * N + m] = std::sqrt(2.0 / (N + 1)) * std::sin((p + 1) * th);
        }
        return;
    }
    // real Fourier modes: constant; cos and sin of frequency f = 1 .. (N-1)/2;
    // the alternating mode when N is even
    int64_t col = 0;
    for (int64_t p = 0; p < N; ++p) S[p * N + col] = 1.0 / std::sqrt((double)N);
    mu[col++] = 0.0;
    for (int64_t f = 1; 2 * f < N; ++f) {
        const double th = 2.0 * M_PI * f / N;
        for (int64_t p = 0; p < N; ++p) {
            S[p * N + col] = std::sqrt(2.0 / N) * std::cos(th * p);
            S[p * N + col + 1] = std::sqrt(2.0 / N) * std::sin(th * p);
        }
        mu[col] = mu[col + 1] = 2.0 - 2.0 * std::cos(th);
        col += 2;
    }
    if (N % 2 == 0) {
        for (int64_t p = 0; p < N; ++p) S[p * N + col] = (p % 2 ? -1.0 : 1.0) / std::sqrt((double)N);
        mu[col++] = 4.0;
    }
}

}  // namespace

int64_t spectral_workspace_doubles(const SpecPrec& P, int nc) { return 2 * P.n() * nc; }

cudaError_t spectral_apply(const SpecPrec& P, int nc, const double* r, int64_t ldr, double* w, double* work,
                           cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    const int64_t n = P.n();
    dw* t0 = reinterpret_cast<dw*>(work);
    dw* t1 = t0 + n * nc;
    const int64_t Ns[3] = {P.nx, P.ny, P.nz};
    const int64_t strides[3] = {1, P.nx, P.nx * P.ny};
    const int64_t total = n * nc;
    const dw* K = reinterpret_cast<const dw*>(P.d_K);
    auto pass = [&](int axis, bool inverse, bool scale, const dw* in, void* out, bool out64) {
        AxisPass a{P.nx, P.ny, P.nz, axis, (int)Ns[axis], strides[axis], nc};
        const int N = (int)Ns[axis];
        // one line of nc columns and the matrix must fit the shared memory
        if ((int64_t)sizeof(dw) * ((int64_t)N * N + (int64_t)N * nc) > kAxisShm) return cudaErrorInvalidValue;
        const int TL = tile_lines(N, nc);
        const size_t shm = sizeof(dw) * ((size_t)N * N + (size_t)N * TL * nc);
        const int64_t lines = n / N;
        const int blocks = (int)std::min<int64_t>((lines + TL - 1) / TL, (int64_t)sm_count() * 16);
        const dw* M = reinterpret_cast<const dw*>(inverse ? P.d_St[axis] : P.d_S[axis]);
        if (scale)
            k_axis<true, false><<<blocks, kT, shm, s>>>(a, TL, M, in, out, 0, K);
        else if (out64)
            k_axis<false, true><<<blocks, kT, shm, s>>>(a, TL, M, in, out, nc, nullptr);
        else
            k_axis<false, false><<<blocks, kT, shm, s>>>(a, TL, M, in, out, 0, nullptr);
        count_launches(1);
        return cudaGetLastError();
    };
    k_split<<<nblk(total), kT, 0, s>>>(total, nc, r, ldr, t0);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // forward x, y (, z) with the factor on the last forward pass; inverse in
    // reverse order; the inverse x pass writes the FP64 result (dense, ld nc)
    if ((e = pass(0, false, false, t0, t1, false)) != cudaSuccess) return e;
    if (P.d == 3) {
        if ((e = pass(1, false, false, t1, t0, false)) != cudaSuccess) return e;
        if ((e = pass(2, false, true, t0, t1, false)) != cudaSuccess) return e;
        if ((e = pass(2, true, false, t1, t0, false)) != cudaSuccess) return e;
        if ((e = pass(1, true, false, t0, t1, false)) != cudaSuccess) return e;
    } else {
        if ((e = pass(1, false, true, t1, t0, false)) != cudaSuccess) return e;
        if ((e = pass(1, true, false, t0, t1, false)) != cudaSuccess) return e;
    }
    return pass(0, true, false, t1, w, true);
}

}  // namespace plhr

using namespace plhr;

extern "C" plhr_status plhr_prec_tpa(plhr_prec** out, const plhr_op* A, double sigma, double energy) {
    clear_error();
    if (!out || !A || !std::isfinite(sigma) || !std::isfinite(energy)) {
        set_error("plhr_prec_tpa: invalid argument");
        return PLHR_EINVAL;
    }
    const Grid& g = A->g;
    if (g.csr) {
        set_error("plhr_prec_tpa: A must be a stencil or Hamiltonian operator (not CSR)");
        return PLHR_EINVAL;
    }
    const int64_t Ns[3] = {g.nx, g.ny, g.d == 3 ? g.nz : 1};
    for (int a = 0; a < g.d; ++a)
        if (Ns[a] > kMaxAxis) {
            set_error("plhr_prec_tpa: axis size %lld exceeds %d", (long long)Ns[a], kMaxAxis);
            return PLHR_EINVAL;
        }
    if (!(energy > 0)) {
        // sigma - min V, or the mean kinetic energy of the grid's modes d / h^2
        double vmin = 0.0;
        if (g.pot) {
            std::vector<double> hv(g.n());
            if (cudaMemcpy(hv.data(), g.pot, sizeof(double) * g.n(), cudaMemcpyDeviceToHost) != cudaSuccess) {
                set_error("plhr_prec_tpa: reading the potential failed");
                return PLHR_ECUDA;
            }
            vmin = hv[0];
            for (double v : hv) vmin = std::fmin(vmin, v);
        }
        energy = sigma - vmin;
        if (!(energy > 0)) energy = g.d * 2.0 * g.inv_h2();   // d / h^2 for the scale 1/2
    }
    plhr_prec* T = new plhr_prec;
    T->kind = PREC_TPA;
    SpecPrec& P = T->sp;
    P.d = g.d;
    P.nx = Ns[0]; P.ny = Ns[1]; P.nz = Ns[2];
    P.energy = energy;
    // double-word (hi, lo) pairs of FP64 values
    auto pairs = [](const std::vector<double>& v) {
        std::vector<float> w(2 * v.size());
        for (size_t i = 0; i < v.size(); ++i) {
            w[2 * i] = (float)v[i];
            w[2 * i + 1] = (float)(v[i] - (double)w[2 * i]);
        }
        return w;
    };
    auto upload = [&](float** dst, const std::vector<float>& src) {
        return cudaMalloc(dst, sizeof(float) * src.size()) == cudaSuccess &&
               cudaMemcpy(*dst, src.data(), sizeof(float) * src.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    };
    std::vector<double> mus[3];
    for (int a = 0; a < 3; ++a) mus[a].assign(1, 0.0);
    for (int a = 0; a < g.d; ++a) {
        const int64_t N = Ns[a];
        std::vector<double> S;
        axis_basis(N, g.periodic != 0, S, mus[a]);
        for (auto& v : mus[a]) v *= g.inv_h2();     // scale / h^2: the kinetic operator's eigenvalues
        std::vector<double> St(N * N);
        for (int64_t p = 0; p < N; ++p)
            for (int64_t m = 0; m < N; ++m) St[m * N + p] = S[p * N + m];
        if (!upload(&P.d_S[a], pairs(S)) || !upload(&P.d_St[a], pairs(St))) {
            set_error("plhr_prec_tpa: device allocation or upload failed");
            plhr_prec_destroy(T);
            return PLHR_ENOMEM;
        }
    }
    // the factor per 3D mode, x fastest
    std::vector<double> Kf(P.n());
    for (int64_t iz = 0; iz < P.nz; ++iz)
        for (int64_t iy = 0; iy < P.ny; ++iy)
            for (int64_t ix = 0; ix < P.nx; ++ix)
                Kf[(iz * P.ny + iy) * P.nx + ix] =
                    tpa((mus[0][ix] + mus[1][iy] + (g.d == 3 ? mus[2][iz] : 0.0)) / energy);
    if (!upload(&P.d_K, pairs(Kf))) {
        set_error("plhr_prec_tpa: device allocation or upload failed");
        plhr_prec_destroy(T);
        return PLHR_ENOMEM;
    }
    const int shm = kAxisShm;   // the launches size their tiles to fit
    if (cudaFuncSetAttribute(k_axis<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm) != cudaSuccess ||
        cudaFuncSetAttribute(k_axis<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm) != cudaSuccess ||
        cudaFuncSetAttribute(k_axis<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm) != cudaSuccess) {
        set_error("plhr_prec_tpa: shared-memory attribute failed");
        plhr_prec_destroy(T);
        return PLHR_ECUDA;
    }
    *out = T;
    return PLHR_OK;
}

extern "C" double plhr_prec_tpa_energy(const plhr_prec* T) {
    return (T && T->kind == PREC_TPA) ? T->sp.energy : 0.0;
}
