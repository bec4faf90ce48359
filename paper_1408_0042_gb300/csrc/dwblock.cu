// Double-word forms of the multi-Gram and the coefficient update on FP64
// blocks, for the FP64 phase of the mixed-precision solve.  The inputs are
// split once into double-word values (hi = the leading 24 bits, lo = the
// rest rounded to FP32: ~48-bit significands, dw_split_trunc); products are
// formed with the FMA exact product of the high
// parts plus the FP32 cross terms, and sums are accumulated with TwoSum on the
// high part, so every result carries ~2^-46 relative error of the sum of
// |terms| - FP64-class accuracy for the projected problem at a fraction of the
// FP64 pipe's cost on GB300.  Results and partial sums are FP64; the per-CTA
// partials are summed in FP64 in a fixed order (deterministic).
#include "blockops.h"
#include "dword.h"

namespace plhr {
namespace {

constexpr int kDwRows = 32;
constexpr int kDwThreads = 768;

struct FamD {
    const double* p[4];
    int64_t ld[4];
    int nc[4];
    int off[4];
};

FamD fam_d(const Blk<const double>* b, int nb) {
    FamD F{};
    int off = 0;
    for (int i = 0; i < 4; ++i) {
        if (i < nb) {
            F.p[i] = b[i].p; F.ld[i] = b[i].ld; F.nc[i] = b[i].nc; F.off[i] = off;
            off += b[i].nc;
        } else {
            F.p[i] = nullptr; F.ld[i] = 0; F.nc[i] = 0; F.off[i] = off;
        }
    }
    return F;
}


// Start the copies of rows row0 .. row0 + kDwRows - 1 (those below n) of the
// Z, AZ and (unless q_from_u) Q families into the FP64 row buffers rz, ra, rq
// ([row][mp], column off[b] + c for column c of block b)
__device__ void fetch_dw(double* rz, double* ra, double* rq, int mp, int64_t n, int64_t row0, const FamD& Z,
                         const FamD& AZ, const FamD& Q, int nb, int q_from_u) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        if (b >= nb) break;
        const int nc = Z.nc[b];
        if (nc == 0) continue;
        const int tot = kDwRows * nc;
        for (int t = threadIdx.x; t < tot; t += blockDim.x) {
            const int r = t / nc, c = t - r * nc;
            const int64_t row = row0 + r;
            if (row >= n) continue;
            const int at = r * mp + Z.off[b] + c;
            cp_async8(rz + at, Z.p[b] + row * Z.ld[b] + c);
            cp_async8(ra + at, AZ.p[b] + row * AZ.ld[b] + c);
            if (!q_from_u) cp_async8(rq + at, Q.p[b] + row * Q.ld[b] + c);
        }
    }
}

// Stage the fetched rows as double-word [row][mp] tiles of z = Z, u = AZ -
// sigma Z, q = Q (q = u when q_from_u); U is formed by one FP64 FMA before the
// split, rows at or past n are zero (the column scales are applied to the
// finished Grams)
__device__ void stage_dw(dw* sz, dw* su, dw* sq, const double* rz, const double* ra, const double* rq, int m,
                         int mp, int64_t n, int64_t row0, int q_from_u, double sigma) {
    const int tot = kDwRows * m;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        const int r = t / m, col = t - r * m;
        const int at = r * mp + col;
        dw z = dw_make(0.0f), u = z, q = z;
        if (row0 + r < n) {
            const double zd = rz[at];
            const double ud = fma(-sigma, zd, ra[at]);
            z = dw_split_trunc(zd);
            u = dw_split_trunc(ud);
            q = q_from_u ? u : dw_split_trunc(rq[at]);
        }
        sz[at] = z;
        su[at] = u;
        sq[at] = q;
    }
}

// 768 threads: thread t owns tile t of gram_tile (outputs g = 0: Z^T Z and
// 1: U^T Q written for ti <= tj and mirrored; 2: Q^T Z); at most 528 tiles
// (mp <= 64), every thread fetches and stages.  The rows of the next chunk
// are copied asynchronously while the current one is multiplied.
__global__ void __launch_bounds__(kDwThreads, 1) k_gram_dw(int64_t n, int m, int mp, int nb, FamD Z, FamD AZ, FamD Q,
                                                           int q_from_u, double sigma,
                                                           double* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char raw[];
    dw* sz = reinterpret_cast<dw*>(raw);
    dw* su = sz + kDwRows * mp;
    dw* sq = su + kDwRows * mp;
    double* rz = reinterpret_cast<double*>(sq + kDwRows * mp);
    double* ra = rz + kDwRows * mp;
    double* rq = ra + kDwRows * mp;
    const int T = mp / 4;
    int g, ti, tj;
    const bool act = gram_tile(threadIdx.x, T, g, ti, tj);
    const dw* A = g == 0 ? sz : (g == 1 ? su : sq);
    const dw* B = g == 1 ? sq : sz;
    float hi[16], lo[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) { hi[e] = 0.0f; lo[e] = 0.0f; }
    for (int t = threadIdx.x; t < kDwRows * mp; t += blockDim.x) {
        if (t % mp >= m) { sz[t] = dw_make(0.0f); su[t] = dw_make(0.0f); sq[t] = dw_make(0.0f); }
    }
    const int64_t nchunks = (n + kDwRows - 1) / kDwRows;
    if ((int64_t)blockIdx.x < nchunks) fetch_dw(rz, ra, rq, mp, n, (int64_t)blockIdx.x * kDwRows, Z, AZ, Q, nb, q_from_u);
    cp_async_commit();
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();          // rows of chunk ch landed; the previous chunk's products are done
        stage_dw(sz, su, sq, rz, ra, rq, m, mp, n, ch * kDwRows, q_from_u, sigma);
        __syncthreads();          // tiles staged; the row buffers are free
        if (ch + gridDim.x < nchunks)
            fetch_dw(rz, ra, rq, mp, n, (ch + gridDim.x) * kDwRows, Z, AZ, Q, nb, q_from_u);
        cp_async_commit();
        if (act) {
#pragma unroll 2
            for (int r = 0; r < kDwRows; ++r) {
                const float4* ap = reinterpret_cast<const float4*>(A + r * mp + 4 * ti);
                const float4* bp = reinterpret_cast<const float4*>(B + r * mp + 4 * tj);
                const float4 a01 = ap[0], a23 = ap[1], b01 = bp[0], b23 = bp[1];
                const dw av[4] = {{a01.x, a01.y}, {a01.z, a01.w}, {a23.x, a23.y}, {a23.z, a23.w}};
                const dw bv[4] = {{b01.x, b01.y}, {b01.z, b01.w}, {b23.x, b23.y}, {b23.z, b23.w}};
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) dw_fma_acc(hi[x * 4 + y], lo[x * 4 + y], av[x], bv[y]);
            }
        }
    }
    cp_async_wait_all();
    if (!act) return;
    double* out = partial + (int64_t)blockIdx.x * 3 * m * m + (int64_t)g * m * m;
    for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y) {
            const int i = 4 * ti + x, j = 4 * tj + y;
            if (i < m && j < m) {
                const double v = (double)hi[x * 4 + y] + (double)lo[x * 4 + y];
                out[i * m + j] = v;
                if (g <= 1) out[j * m + i] = v;
            }
        }
}

// out = D (sum of the per-CTA partials) D for each of the three m x m Grams
// (D = diag(csc), the column scales)
__global__ void k_sum_wide_dw(int nblocks, int m, const double* __restrict__ csc, const double* __restrict__ partial,
                              double* __restrict__ out) {
    const int width = 3 * m * m;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= width) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partial[(int64_t)b * width + j];
    const int idx = j % (m * m);
    out[j] = t * (csc[idx / m] * csc[idx % m]);
}

// Pout = F C_P, Vout = F_0 C_VV + F C_P in double-word arithmetic on FP64
// blocks (in place allowed: every output row depends only on the same input
// row and a chunk is staged before any of its rows is written)
constexpr int kDwUpRows = 32;
// Thread t owns column j = t % kp of rows r = t / kp and r + kDwUpRows / 2 of
// each chunk (kp <= 16, so 16 kp <= 256 threads): the two rows share the
// coefficient loads and give each thread two independent sums.  Every output
// is summed over i in the same order as with one output per thread.
__global__ void __launch_bounds__(256) k_update_dw(int64_t n, int m, int kp, int nb, FamD F,
                                                   const double* __restrict__ Cp, const double* __restrict__ Cvv,
                                                   double* __restrict__ Vout, int64_t ldvo, double* __restrict__ Pout,
                                                   int64_t ldpo) {
    extern __shared__ __align__(16) unsigned char raw[];
    dw* cp = reinterpret_cast<dw*>(raw);      // [m][kp]
    dw* cv = cp + m * kp;                     // [kp][kp]
    dw* zr = cv + kp * kp;                    // [rows][m]
    for (int t = threadIdx.x; t < m * kp; t += blockDim.x) cp[t] = dw_from_double(Cp[t]);
    for (int t = threadIdx.x; t < kp * kp; t += blockDim.x) cv[t] = dw_from_double(Cvv[t]);
    constexpr int kHalf = kDwUpRows / 2;
    const int r0 = threadIdx.x / kp, j = threadIdx.x - r0 * kp;
    const bool own = r0 < kHalf;
    const int64_t nchunks = (n + kDwUpRows - 1) / kDwUpRows;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t row0 = ch * kDwUpRows;
        const int nrows = (int)((n - row0) < kDwUpRows ? (n - row0) : kDwUpRows);
        __syncthreads();
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if (b >= nb) break;
            const int nc = F.nc[b];
            for (int t = threadIdx.x; t < nrows * nc; t += blockDim.x) {
                const int r = t / nc, c = t - r * nc;
                zr[r * m + F.off[b] + c] = dw_split_trunc(F.p[b][(row0 + r) * F.ld[b] + c]);
            }
        }
        __syncthreads();
        if (!own || r0 >= nrows) continue;
        const bool two = r0 + kHalf < nrows;
        const dw* z0 = zr + r0 * m;
        const dw* z1 = zr + (two ? r0 + kHalf : r0) * m;
        float ph0 = 0.0f, pl0 = 0.0f, ph1 = 0.0f, pl1 = 0.0f;
        for (int i = 0; i < m; ++i) {
            const dw c = cp[i * kp + j];
            dw_fma_acc(ph0, pl0, z0[i], c);
            dw_fma_acc(ph1, pl1, z1[i], c);
        }
        float vh0 = ph0, vl0 = pl0, vh1 = ph1, vl1 = pl1;
        for (int i = 0; i < kp; ++i) {
            const dw c = cv[i * kp + j];
            dw_fma_acc(vh0, vl0, z0[i], c);
            dw_fma_acc(vh1, vl1, z1[i], c);
        }
        const int64_t row = row0 + r0;
        Pout[row * ldpo + j] = dw_to_double_fast(dw{ph0, pl0});
        Vout[row * ldvo + j] = dw_to_double_fast(dw{vh0, vl0});
        if (two) {
            Pout[(row + kHalf) * ldpo + j] = dw_to_double_fast(dw{ph1, pl1});
            Vout[(row + kHalf) * ldvo + j] = dw_to_double_fast(dw{vh1, vl1});
        }
    }
}

}  // namespace

cudaError_t multi_gram_dw(int64_t n, int nb, const Blk<const double>* Z, const Blk<const double>* AZ,
                          const Blk<const double>* Q, double sigma, const double* colscale, double* partial,
                          double* out, cudaStream_t s) {
    FamD FZ = fam_d(Z, nb), FA = fam_d(AZ, nb), FQ = fam_d(Q ? Q : AZ, nb);
    int m = 0;
    for (int i = 0; i < nb; ++i) m += Z[i].nc;
    const int mp = (m + 3) / 4 * 4;
    if (mp > 64) return cudaErrorInvalidValue;
    const int blocks = sm_count();
    const size_t shm = (sizeof(dw) + sizeof(double)) * 3 * kDwRows * mp;
    // above the 48 KB default: raise the limit on the current device (every
    // call, so that each device a process uses gets it)
    {
        cudaError_t e = cudaFuncSetAttribute(k_gram_dw, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)((sizeof(dw) + sizeof(double)) * 3 * kDwRows * 64));
        if (e != cudaSuccess) return e;
    }
    k_gram_dw<<<blocks, kDwThreads, shm, s>>>(n, m, mp, nb, FZ, FA, FQ, Q ? 0 : 1, sigma, partial);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int width = 3 * m * m;
    k_sum_wide_dw<<<(width + 127) / 128, 128, 0, s>>>(blocks, m, colscale, partial, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t block_update_dw(int64_t n, int nb, const Blk<const double>* F, int kp, const double* Cp, const double* Cvv,
                            double* Vout, int64_t ldvo, double* Pout, int64_t ldpo, cudaStream_t s) {
    FamD FF = fam_d(F, nb);
    int m = 0;
    for (int i = 0; i < nb; ++i) m += F[i].nc;
    const size_t shm = sizeof(dw) * (m * kp + kp * kp + kDwUpRows * m);
    k_update_dw<<<sm_count() * 4, 256, shm, s>>>(n, m, kp, nb, FF, Cp, Cvv, Vout, ldvo, Pout, ldpo);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plhr
