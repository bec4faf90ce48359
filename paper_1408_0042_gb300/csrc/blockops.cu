// Tall-skinny block kernels of the PLHR sweep (FP64 path):
//  - residual R = s_j (A v_j - lambda_j v_j) with column norms (Alg. 2/3 step 4
//    input, convergence test);
//  - the multi-Gram pass over Z = [V W S P], AZ and Q = T(A - sigma B)Z that
//    yields Z*Z, U*Q (U = AZ - sigma Z) and Q*Z (B-orthonormalisation Gram and
//    the two matrices of the T-harmonic problem, Eq. THarm_evp);
//  - the coefficient update V <- Z C_V, P <- Z C_P applied to Z, AZ and Q
//    (Alg. 2 steps 8-9, Alg. 3 steps 11-12) with the column dot products that
//    give the new Rayleigh quotients (Alg. 3 step 13).
// Column reductions write one partial per CTA; a fixed-order second pass sums
// them, so results are bitwise reproducible run to run.
#include "blockops.h"

namespace plhr {
namespace {

constexpr int kThreads = 256;

// ------------------------------------------------------------------ residual
// The grid is a multiple of kp CTAs of kThreads threads, so the grid stride is
// a multiple of kp and every thread keeps one column: per-thread sums are then
// combined in thread order (deterministic).
__global__ void __launch_bounds__(kThreads) k_residual(int64_t n, int kp, const double* __restrict__ V,
                                                       int64_t ldv, const double* __restrict__ AV,
                                                       int64_t ldav, const double* __restrict__ lam,
                                                       const double* __restrict__ sc,
                                                       double* __restrict__ R, int64_t ldr,
                                                       double* __restrict__ partial) {
    // partial layout: [gridDim.x][2*kp]: sum r^2, sum (s v)^2
    __shared__ double srr[kThreads], sbb[kThreads];
    const int64_t total = n * kp;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = (int)(e0 % kp);
    const double s = sc[c], l = lam[c];
    double rr = 0.0, bb = 0.0;
    const int64_t drow = stride / kp;   // the stride is a multiple of kp: the column stays c
    int64_t row = e0 / kp;
    for (int64_t e = e0; e < total; e += stride, row += drow) {
        double v = V[row * ldv + c];
        double r = s * (AV[row * ldav + c] - l * v);
        R[row * ldr + c] = r;
        rr = fma(r, r, rr);
        bb = fma(s * v, s * v, bb);
    }
    srr[threadIdx.x] = rr;
    sbb[threadIdx.x] = bb;
    __syncthreads();
    const int cbase = (int)(((int64_t)blockIdx.x * blockDim.x) % kp);
    for (int j = threadIdx.x; j < kp; j += blockDim.x) {
        // threads t with (cbase + t) % kp == j, in increasing t
        int t0 = (j - cbase) % kp;
        if (t0 < 0) t0 += kp;
        double a = 0.0, b2 = 0.0;
        for (int t = t0; t < kThreads; t += kp) { a += srr[t]; b2 += sbb[t]; }
        partial[(int64_t)blockIdx.x * 2 * kp + j] = a;
        partial[(int64_t)blockIdx.x * 2 * kp + kp + j] = b2;
    }
}

// fixed-order sum of per-CTA partials: out[j] = sum_b partial[b * width + j]
// (one thread per output; launch with sum_blocks(width) CTAs of 128)
__global__ void k_sum_partials(int nblocks, int width, const double* __restrict__ partial,
                               double* __restrict__ out) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < width; j += gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < nblocks; ++b) t += partial[(int64_t)b * width + j];
        out[j] = t;
    }
}

// ------------------------------------------------------------------ Gram
constexpr int kGramRows = 16;       // rows staged per pass
constexpr int kGramThreads = 256;

struct FamPtrs {
    const double* p[4];
    int64_t ld[4];
    int nc[4];
    int off[4];
};

__device__ __forceinline__ void stage_rows(double* dst, int m, int64_t row0, int nrows, const FamPtrs& F,
                                           int nb) {
    // dst[r * m + col] for r < nrows
    for (int b = 0; b < nb; ++b) {
        int nc = F.nc[b];
        if (nc == 0) continue;
        int tot = nrows * nc;
        for (int t = threadIdx.x; t < tot; t += blockDim.x) {
            int r = t / nc, c = t - r * nc;
            dst[r * m + F.off[b] + c] = F.p[b][(row0 + r) * F.ld[b] + c];
        }
    }
}

// Gram tile bookkeeping: 4x4 register tiles over three m x m outputs.
//   g = 0: Z^T BZ and g = 1: U^T Q (upper tiles only, mirrored: both are
//   symmetric, U^T Q = U^T T U), g = 2: Q^T BZ, with U = AZ - sigma BZ;
//   without a BZ family (B = I) BZ is Z
__global__ void __launch_bounds__(kGramThreads) k_gram(int64_t n, int m, int nb, FamPtrs Z, FamPtrs AZ, FamPtrs Q,
                                                       FamPtrs BZ, int has_b, int q_from_u, double sigma,
                                                       const double* __restrict__ csc,
                                                       double* __restrict__ partial) {
    extern __shared__ double sh[];
    double* sz = sh;                         // [rows][m]
    double* su = sz + kGramRows * m;         // [rows][m]
    double* sq = su + kGramRows * m;         // [rows][m]
    double* sb = has_b ? sq + kGramRows * m : sz;   // [rows][m], B Z
    const int T = (m + 3) / 4;
    const int nt0 = T * (T + 1) / 2, nt1 = T * T;
    const int ntiles = 2 * nt0 + nt1;
    constexpr int kMaxTilesPerThread = 4;
    double acc[kMaxTilesPerThread][16];
    int tg[kMaxTilesPerThread], ti[kMaxTilesPerThread], tj[kMaxTilesPerThread];
    int my = 0;
    for (int t = threadIdx.x; t < ntiles && my < kMaxTilesPerThread; t += blockDim.x, ++my) {
        if (t < 2 * nt0) {
            // upper triangle tile enumeration (outputs 0 and 1)
            const int g = t < nt0 ? 0 : 1;
            int r = 0, rem = t - g * nt0;
            while (rem >= T - r) { rem -= T - r; ++r; }
            tg[my] = g; ti[my] = r; tj[my] = r + rem;
        } else {
            int u = t - 2 * nt0;
            tg[my] = 2; ti[my] = u / T; tj[my] = u % T;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[my][q] = 0.0;
    }
    const int64_t nchunks = (n + kGramRows - 1) / kGramRows;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        int64_t row0 = ch * kGramRows;
        int nrows = (int)((n - row0) < kGramRows ? (n - row0) : kGramRows);
        stage_rows(sz, m, row0, nrows, Z, nb);
        stage_rows(su, m, row0, nrows, AZ, nb);
        if (!q_from_u) stage_rows(sq, m, row0, nrows, Q, nb);
        if (has_b) stage_rows(sb, m, row0, nrows, BZ, nb);
        __syncthreads();
        // u = (az - sigma bz) * scale, z, bz, q scaled by the column scales
        // (q = u when T = I)
        for (int t = threadIdx.x; t < nrows * m; t += blockDim.x) {
            int c = t % m;
            double s = csc[c];
            double z = sz[t] * s;
            sz[t] = z;
            double bz = z;
            if (has_b) {
                bz = sb[t] * s;
                sb[t] = bz;
            }
            double u = su[t] * s - sigma * bz;
            su[t] = u;
            sq[t] = q_from_u ? u : sq[t] * s;
        }
        for (int t = nrows * m + threadIdx.x; t < kGramRows * m; t += blockDim.x) {
            sz[t] = 0.0; su[t] = 0.0; sq[t] = 0.0;
            if (has_b) sb[t] = 0.0;
        }
        __syncthreads();
        for (int q = 0; q < my; ++q) {
            const double* A = tg[q] == 0 ? sz : (tg[q] == 1 ? su : sq);
            const double* B = tg[q] == 0 ? sb : (tg[q] == 1 ? sq : sb);
            int i0 = ti[q] * 4, j0 = tj[q] * 4;
            for (int r = 0; r < kGramRows; ++r) {
                double a[4], b[4];
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    a[x] = (i0 + x < m) ? A[r * m + i0 + x] : 0.0;
                    b[x] = (j0 + x < m) ? B[r * m + j0 + x] : 0.0;
                }
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[q][x * 4 + y] = fma(a[x], b[y], acc[q][x * 4 + y]);
            }
        }
        __syncthreads();
    }
    // write partial: [block][3][m][m]
    double* out = partial + (int64_t)blockIdx.x * 3 * m * m;
    for (int q = 0; q < my; ++q) {
        int i0 = ti[q] * 4, j0 = tj[q] * 4;
        double* G = out + (int64_t)tg[q] * m * m;
        for (int x = 0; x < 4; ++x)
            for (int y = 0; y < 4; ++y) {
                int i = i0 + x, j = j0 + y;
                if (i < m && j < m) {
                    G[i * m + j] = acc[q][x * 4 + y];
                    if (tg[q] <= 1) G[j * m + i] = acc[q][x * 4 + y];
                }
            }
    }
}

// ------------------------------------------------------------------ update
constexpr int kUpdRows = 32;

// new P = Zraw C_P (m x kp), new V = V C_VV (kp x kp) + new P, for one family,
// in place: every output row depends only on the same input row, and a chunk
// is fully staged before any of its rows is written.
// dotV (optional): the matching block of the new V (already updated); the
// kernel then accumulates, per column, sum_i out_ij * dotV_ij and
// sum_i dotV_ij^2 in fixed row order into partial[block][2*kp].
__global__ void __launch_bounds__(kThreads) k_update(int64_t n, int m, int kp, int nb, FamPtrs F,
                                                     const double* __restrict__ Cp,
                                                     const double* __restrict__ Cvv,
                                                     double* __restrict__ Vout, int64_t ldvo,
                                                     double* __restrict__ Pout, int64_t ldpo,
                                                     const double* __restrict__ dotV, int64_t lddv,
                                                     double* __restrict__ partial) {
    extern __shared__ double sh[];
    double* sc = sh;                        // C_P [m][kp]
    double* sv = sc + m * kp;               // C_VV [kp][kp]
    double* srow = sv + kp * kp;            // [kUpdRows][m]
    double* sout = srow + kUpdRows * m;     // [kUpdRows][kp] new V-part values
    double* sd = sout + kUpdRows * kp;      // [kUpdRows][kp] dotV values
    for (int t = threadIdx.x; t < m * kp; t += blockDim.x) sc[t] = Cp[t];
    for (int t = threadIdx.x; t < kp * kp; t += blockDim.x) sv[t] = Cvv[t];
    double acc_a = 0.0, acc_b = 0.0;        // owned by threads j < kp
    const int64_t nchunks = (n + kUpdRows - 1) / kUpdRows;
    __syncthreads();
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        int64_t row0 = ch * kUpdRows;
        int nrows = (int)((n - row0) < kUpdRows ? (n - row0) : kUpdRows);
        stage_rows(srow, m, row0, nrows, F, nb);
        if (dotV)
            for (int t = threadIdx.x; t < nrows * kp; t += blockDim.x) {
                int r = t / kp, j = t - r * kp;
                sd[t] = dotV[(row0 + r) * lddv + j];
            }
        __syncthreads();
        for (int t = threadIdx.x; t < nrows * kp; t += blockDim.x) {
            int r = t / kp, j = t - r * kp;
            const double* z = srow + r * m;
            double p = 0.0;
            for (int i = 0; i < m; ++i) p = fma(z[i], sc[i * kp + j], p);
            double v = p;
            for (int i = 0; i < kp; ++i) v = fma(z[i], sv[i * kp + j], v);
            int64_t row = row0 + r;
            Pout[row * ldpo + j] = p;
            Vout[row * ldvo + j] = v;
            sout[t] = v;
        }
        __syncthreads();
        if (dotV && threadIdx.x < kp) {
            int j = threadIdx.x;
            for (int r = 0; r < nrows; ++r) {
                double d = sd[r * kp + j];
                acc_a = fma(sout[r * kp + j], d, acc_a);
                acc_b = fma(d, d, acc_b);
            }
        }
        __syncthreads();
    }
    if (dotV && threadIdx.x < kp) {
        partial[(int64_t)blockIdx.x * 2 * kp + threadIdx.x] = acc_a;
        partial[(int64_t)blockIdx.x * 2 * kp + kp + threadIdx.x] = acc_b;
    }
}

FamPtrs fam_of(const Blk<const double>* b, int nb) {
    FamPtrs F{};
    int off = 0;
    for (int i = 0; i < 4; ++i) {
        if (i < nb) {
            F.p[i] = b[i].p; F.ld[i] = b[i].ld; F.nc[i] = b[i].nc; F.off[i] = off; off += b[i].nc;
        } else {
            F.p[i] = nullptr; F.ld[i] = 0; F.nc[i] = 0; F.off[i] = off;
        }
    }
    return F;
}

}  // namespace

int reduce_blocks() { return sm_count() * 2; }

int residual_blocks(int kp) {
    int g = (sm_count() * 2 + kp - 1) / kp;
    return g * kp;
}

cudaError_t residual_norms(int64_t n, int kp, const double* V, int64_t ldv, const double* AV, int64_t ldav,
                           const double* lam, const double* sc, double* R, int64_t ldr, double* partial,
                           double* out, cudaStream_t s) {
    int blocks = residual_blocks(kp);
    k_residual<<<blocks, kThreads, 0, s>>>(n, kp, V, ldv, AV, ldav, lam, sc, R, ldr, partial);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_partials<<<(2 * kp + 127) / 128, 128, 0, s>>>(blocks, 2 * kp, partial, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t multi_gram(int64_t n, int nb, const Blk<const double>* Z, const Blk<const double>* AZ,
                       const Blk<const double>* Q, double sigma, const double* colscale, double* partial,
                       double* out, cudaStream_t s) {
    return multi_gram_b(n, nb, Z, AZ, Q, nullptr, sigma, colscale, partial, out, s);
}

cudaError_t multi_gram_b(int64_t n, int nb, const Blk<const double>* Z, const Blk<const double>* AZ,
                         const Blk<const double>* Q, const Blk<const double>* BZ, double sigma,
                         const double* colscale, double* partial, double* out, cudaStream_t s) {
    FamPtrs FZ = fam_of(Z, nb), FA = fam_of(AZ, nb), FQ = fam_of(Q ? Q : AZ, nb), FB = fam_of(BZ ? BZ : Z, nb);
    int m = 0;
    for (int i = 0; i < nb; ++i) m += Z[i].nc;
    int blocks = reduce_blocks();
    size_t shm = sizeof(double) * (BZ ? 4 : 3) * kGramRows * m;
    k_gram<<<blocks, kGramThreads, shm, s>>>(n, m, nb, FZ, FA, FQ, FB, BZ ? 1 : 0, Q ? 0 : 1, sigma, colscale,
                                             partial);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_partials<<<(3 * m * m + 127) / 128, 128, 0, s>>>(blocks, 3 * m * m, partial, out);
    count_launches(1);
    return cudaGetLastError();
}

int gram_max_m() {
    // 4 tiles per thread * 256 threads >= ntiles(m) = T(T+1) + T^2, T = ceil(m/4)
    return 64;
}

cudaError_t block_update(int64_t n, int nb, const Blk<const double>* F, int kp, const double* Cp,
                         const double* Cvv, double* Vout, int64_t ldvo, double* Pout, int64_t ldpo,
                         const double* dotV, int64_t lddv, double* partial, double* out, cudaStream_t s) {
    FamPtrs FF = fam_of(F, nb);
    int m = 0;
    for (int i = 0; i < nb; ++i) m += F[i].nc;
    int blocks = reduce_blocks();
    size_t shm = sizeof(double) * (m * kp + kp * kp + kUpdRows * m + 2 * kUpdRows * kp);
    k_update<<<blocks, kThreads, shm, s>>>(n, m, kp, nb, FF, Cp, Cvv, Vout, ldvo, Pout, ldpo, dotV, lddv,
                                           partial);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (dotV) {
        k_sum_partials<<<1, 128, 0, s>>>(blocks, 2 * kp, partial, out);
        count_launches(1);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace plhr

namespace plhr {
namespace {

constexpr int kRows = 32;

// Y = X C, rows staged through shared memory (in place allowed).
__global__ void __launch_bounds__(256) k_times_small(int64_t n, const double* __restrict__ X, int64_t ldx, int kx,
                                                     const double* __restrict__ C, int ky, double* Y, int64_t ldy) {
    extern __shared__ double sh[];
    double* sc = sh;               // kx * ky
    double* sr = sc + kx * ky;     // kRows * kx
    for (int t = threadIdx.x; t < kx * ky; t += blockDim.x) sc[t] = C[t];
    const int64_t nch = (n + kRows - 1) / kRows;
    __syncthreads();
    for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        int64_t row0 = ch * kRows;
        int nr = (int)((n - row0) < kRows ? (n - row0) : kRows);
        for (int t = threadIdx.x; t < nr * kx; t += blockDim.x) {
            int r = t / kx, c = t - r * kx;
            sr[t] = X[(row0 + r) * ldx + c];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nr * ky; t += blockDim.x) {
            int r = t / ky, j = t - r * ky;
            double s = 0.0;
            for (int i = 0; i < kx; ++i) s = fma(sr[r * kx + i], sc[i * ky + j], s);
            Y[(row0 + r) * ldy + j] = s;
        }
        __syncthreads();
    }
}

__global__ void k_gather(int64_t n, const double* __restrict__ X, int64_t ldx, const int* __restrict__ idx, int nc,
                         double* __restrict__ Y, int64_t ldy) {
    int64_t total = n * nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r;
        int j;
        split_index(e, nc, r, j);
        Y[r * ldy + j] = X[r * ldx + idx[j]];
    }
}

__device__ __forceinline__ uint64_t splitmix_out(uint64_t seed, uint64_t i) {
    uint64_t z = seed + i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_seeded(int64_t n, int kc, uint64_t seed, double* X, int64_t ldx) {
    int64_t total = n * kc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r;
        int j;
        split_index(e, kc, r, j);
        uint64_t x = splitmix_out(seed, (uint64_t)e + 1);
        X[r * ldx + j] = (double)(x >> 11) * 0x1.0p-53 - 0.5;
    }
}

}  // namespace

cudaError_t block_times_small(int64_t n, const double* X, int64_t ldx, int kx, const double* C, int ky, double* Y,
                              int64_t ldy, cudaStream_t s) {
    if (n == 0 || ky == 0) return cudaSuccess;
    size_t shm = sizeof(double) * (kx * ky + kRows * kx);
    k_times_small<<<reduce_blocks(), 256, shm, s>>>(n, X, ldx, kx, C, ky, Y, ldy);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t gather_columns(int64_t n, const double* X, int64_t ldx, const int* idx, int nc, double* Y, int64_t ldy,
                           cudaStream_t s) {
    if (n == 0 || nc == 0) return cudaSuccess;
    k_gather<<<grid_size_for(n * nc, 256, sm_count() * 16), 256, 0, s>>>(n, X, ldx, idx, nc, Y, ldy);
    count_launches(1);
    return cudaGetLastError();
}

namespace {
__global__ void __launch_bounds__(256) k_shift_combine(int64_t n, int nc, const double* __restrict__ AX, int64_t ldax,
                                                       const double* __restrict__ BX, int64_t ldbx,
                                                       const double* __restrict__ lam, double* __restrict__ o1,
                                                       int64_t ld1, double sig, double* __restrict__ o2,
                                                       int64_t ld2) {
    const int64_t total = n * nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i;
        int c;
        split_index(e, nc, i, c);
        const double a = AX[i * ldax + c], b = BX[i * ldbx + c];
        if (o1) o1[i * ld1 + c] = a - lam[c] * b;
        if (o2) o2[i * ld2 + c] = a - sig * b;
    }
}
}  // namespace

cudaError_t shift_combine(int64_t n, int nc, const double* AX, int64_t ldax, const double* BX, int64_t ldbx,
                          const double* lam, double* o1, int64_t ld1, double sig, double* o2, int64_t ld2,
                          cudaStream_t s) {
    const int64_t total = n * nc;
    if (total == 0) return cudaSuccess;
    k_shift_combine<<<grid_size_for(total, 256, sm_count() * 16), 256, 0, s>>>(n, nc, AX, ldax, BX, ldbx, lam, o1,
                                                                                ld1, sig, o2, ld2);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t seeded_block(int64_t n, int kc, uint64_t seed, double* X, int64_t ldx, cudaStream_t s) {
    if (n == 0 || kc == 0) return cudaSuccess;
    k_seeded<<<grid_size_for(n * kc, 256, sm_count() * 16), 256, 0, s>>>(n, kc, seed, X, ldx);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plhr

namespace plhr {
namespace {

// out[j] = sum_i X_ij Y_ij, out[kc + j] = sum_i X_ij^2 (fixed column per thread,
// grid a multiple of kc CTAs; deterministic order as in k_residual)
__global__ void __launch_bounds__(256) k_coldots(int64_t n, int kc, const double* __restrict__ X, int64_t ldx,
                                                 const double* __restrict__ Y, int64_t ldy,
                                                 double* __restrict__ partial) {
    __shared__ double sa[256], sb[256];
    const int64_t total = n * kc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = (int)(e0 % kc);
    double a = 0.0, b = 0.0;
    const int64_t drow = stride / kc;   // the stride is a multiple of kc: the column stays c
    int64_t row = e0 / kc;
    for (int64_t e = e0; e < total; e += stride, row += drow) {
        double x = X[row * ldx + c];
        a = fma(x, Y[row * ldy + c], a);
        b = fma(x, x, b);
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    const int cbase = (int)(((int64_t)blockIdx.x * blockDim.x) % kc);
    for (int j = threadIdx.x; j < kc; j += blockDim.x) {
        int t0 = (j - cbase) % kc;
        if (t0 < 0) t0 += kc;
        double s1 = 0.0, s2 = 0.0;
        for (int t = t0; t < 256; t += kc) { s1 += sa[t]; s2 += sb[t]; }
        partial[(int64_t)blockIdx.x * 2 * kc + j] = s1;
        partial[(int64_t)blockIdx.x * 2 * kc + kc + j] = s2;
    }
}

}  // namespace

cudaError_t column_dots(int64_t n, int kc, const double* X, int64_t ldx, const double* Y, int64_t ldy,
                        double* partial, double* out, cudaStream_t s) {
    int blocks = residual_blocks(kc);
    k_coldots<<<blocks, 256, 0, s>>>(n, kc, X, ldx, Y, ldy, partial);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_partials<<<1, 128, 0, s>>>(blocks, 2 * kc, partial, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plhr
