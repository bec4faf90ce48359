// Tall-skinny kernels of the mixed-precision iteration.  The block V and its
// image A V stay FP64 (the residual A v - lambda v of a vector near
// convergence needs them); W, S, P, their images and the T-harmonic images Q
// are FP32.  The Grams of the trial basis take FP32 products of values that
// were formed in full precision and then rounded (the V columns, U_V =
// (A V - sigma V) s), sum 32 rows at a time in FP32 registers and fold each
// 32-row sum into a per-thread double-FP32 (hi, lo) accumulator with TwoSum,
// so the accumulation error does not grow with n.  The per-CTA partials are
// summed in FP64 in a fixed order (deterministic).
#include "blockops.h"
#include "dword.h"
#include "mixed.h"

namespace plhr {
namespace {

constexpr int kMxRows = 64;         // rows per staged chunk (folded every 32 rows)
constexpr int kMxThreads = 256;

struct FamMx {
    const void* p[4];
    int64_t ld[4];
    int nc[4];
    int off[4];
    int f64[4];
    int is_u[4];
};

FamMx fam_mx(const BlkMx* b, int nb) {
    FamMx F{};
    int off = 0;
    for (int i = 0; i < 4; ++i) {
        if (i < nb) {
            F.p[i] = b[i].p; F.ld[i] = b[i].ld; F.nc[i] = b[i].nc; F.off[i] = off; F.f64[i] = b[i].f64;
            F.is_u[i] = b[i].is_u;
            off += b[i].nc;
        } else {
            F.p[i] = nullptr; F.ld[i] = 0; F.nc[i] = 0; F.off[i] = off; F.f64[i] = 0; F.is_u[i] = 0;
        }
    }
    return F;
}

__device__ __forceinline__ double ldv(const FamMx& F, int b, int64_t row, int c) {
    return F.f64[b] ? static_cast<const double*>(F.p[b])[row * F.ld[b] + c]
                    : (double)static_cast<const float*>(F.p[b])[row * F.ld[b] + c];
}
__device__ __forceinline__ float ldf(const FamMx& F, int b, int64_t row, int c) {
    return F.f64[b] ? f64_to_f32_rn(static_cast<const double*>(F.p[b])[row * F.ld[b] + c])
                    : static_cast<const float*>(F.p[b])[row * F.ld[b] + c];
}

// Start the copies of rows row0 .. row0 + kMxRows - 1 (those below n) of the
// Z, AZ and (with has_q) Q families into the row buffers rz, ra, rq: one
// 8-byte slot per element ([row][mp], column off[b] + c), an FP32 element in
// the slot's first 4 bytes
__device__ __forceinline__ void fetch_el(double* dst, const FamMx& F, int b, int64_t row, int c) {
    if (F.f64[b]) cp_async8(dst, static_cast<const double*>(F.p[b]) + row * F.ld[b] + c);
    else cp_async4(dst, static_cast<const float*>(F.p[b]) + row * F.ld[b] + c);
}
__device__ void fetch_mx(double* rz, double* ra, double* rq, int mp, int64_t n, int64_t row0, const FamMx& Z,
                         const FamMx& AZ, const FamMx& Q, int nb, int has_q) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        if (b >= nb) break;
        const int nc = Z.nc[b];
        if (nc == 0) continue;
        const int tot = kMxRows * nc;
        for (int t = threadIdx.x; t < tot; t += blockDim.x) {
            const int r = t / nc, c = t - r * nc;
            const int64_t row = row0 + r;
            if (row >= n) continue;
            const int at = r * mp + Z.off[b] + c;
            fetch_el(rz + at, Z, b, row, c);
            fetch_el(ra + at, AZ, b, row, c);
            if (has_q) fetch_el(rq + at, Q, b, row, c);
        }
    }
}

// a fetched element as FP64 / rounded to FP32
__device__ __forceinline__ double rdv(const FamMx& F, int b, const double* slot) {
    return F.f64[b] ? *slot : (double)*reinterpret_cast<const float*>(slot);
}
__device__ __forceinline__ float rdf(const FamMx& F, int b, const double* slot) {
    return F.f64[b] ? f64_to_f32_rn(*slot) : *reinterpret_cast<const float*>(slot);
}

// Stage the fetched rows of z = Z s, u = (AZ - sigma Z) s (u = AZ s for a
// block flagged is_u, which already holds AZ - sigma Z) and q = Q s (q = u
// when Q is absent) as [row][mp] FP32 tiles; FP64 blocks are combined in FP64
// and rounded once; rows at or past n are zero.
__device__ void stage_mx(float* sz, float* su, float* sq, const double* rz, const double* ra, const double* rq,
                         int mp, int64_t n, int64_t row0, const FamMx& Z, const FamMx& AZ, const FamMx& Q, int nb,
                         int has_q, double sigma, const double* __restrict__ csc,
                         const float* __restrict__ cscf, float sigf) {
    // static block indices: the family descriptors stay in registers / the
    // parameter space instead of a local copy
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        if (b >= nb) break;
        const int nc = Z.nc[b];
        if (nc == 0) continue;
        const int tot = kMxRows * nc;
        const bool wide = Z.f64[b] || AZ.f64[b];
        const bool isu = AZ.is_u[b];
        for (int t = threadIdx.x; t < tot; t += blockDim.x) {
            const int r = t / nc, c = t - r * nc;
            const int64_t row = row0 + r;
            const int col = Z.off[b] + c;
            const int at = r * mp + col;
            float z = 0.0f, u = 0.0f, q = 0.0f;
            if (row < n) {
                const float sf = cscf[col];
                if (wide) {
                    const double s = csc[col];
                    const double zd = rdv(Z, b, rz + at) * s;
                    const double ud = isu ? rdv(AZ, b, ra + at) * s : rdv(AZ, b, ra + at) * s - sigma * zd;
                    z = (float)zd;
                    u = (float)ud;
                } else {
                    z = rdf(Z, b, rz + at) * sf;
                    u = isu ? rdf(AZ, b, ra + at) * sf : rdf(AZ, b, ra + at) * sf - sigf * z;
                }
                q = has_q ? rdf(Q, b, rq + at) * sf : u;
            }
            sz[at] = z;
            su[at] = u;
            sq[at] = q;
        }
    }
}

__device__ __forceinline__ void outer4(float* acc, const float4& a, const float4& b) {
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x * 4 + y] = fmaf(av[x], bv[y], acc[x * 4 + y]);
}

// hi + lo += acc (TwoSum on hi, lo collects the rounding errors)
__device__ __forceinline__ void fold(float* hi, float* lo, const float* acc) {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const dw t = dw_two_sum(hi[e], acc[e]);
        hi[e] = t.hi;
        lo[e] = __fadd_rn(lo[e], t.lo);
    }
}

__device__ __forceinline__ void put_tile(double* G, int m, int i0, int j0, const float* hi, const float* lo,
                                         bool mirror) {
    for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y) {
            const int i = i0 + x, j = j0 + y;
            if (i < m && j < m) {
                const double v = (double)hi[x * 4 + y] + (double)lo[x * 4 + y];
                G[i * m + j] = v;
                if (mirror) G[j * m + i] = v;
            }
        }
}

// 768 threads: thread t owns tile t of gram_tile (outputs g = 0: Z^T Z and
// 1: U^T Q written for ti <= tj and mirrored; 2: Q^T Z); at most 528 tiles
// (mp <= 64).  One tile per thread keeps ~70 registers, and all 24 warps
// stage, which hides the latency of the staging loads.
constexpr int kGramMxThreads = 768;
__global__ void __launch_bounds__(kGramMxThreads, 1) k_gram_mx(int64_t n, int m, int mp, int nb, FamMx Z, FamMx AZ,
                                                               FamMx Q, int has_q, double sigma,
                                                               const double* __restrict__ csc,
                                                               double* __restrict__ partial) {
    extern __shared__ __align__(16) double shmd[];
    double* rz = shmd;                      // [rows][mp] fetched rows (8-byte slots)
    double* ra = rz + kMxRows * mp;
    double* rq = ra + kMxRows * mp;
    float* sz = reinterpret_cast<float*>(rq + kMxRows * mp);
    float* su = sz + kMxRows * mp;
    float* sq = su + kMxRows * mp;
    float* cscf = sq + kMxRows * mp;        // [mp] FP32 column scales
    for (int t = threadIdx.x; t < m; t += blockDim.x) cscf[t] = (float)csc[t];
    const float sigf = (float)sigma;
    const int T = mp / 4;
    int g, ti, tj;
    const bool act = gram_tile(threadIdx.x, T, g, ti, tj);
    // operands of this output: A^T B with A, B in {z, u, q}
    const float* A = g == 0 ? sz : (g == 1 ? su : sq);
    const float* B = g == 1 ? sq : sz;
    float hi[16], lo[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) { hi[e] = 0.0f; lo[e] = 0.0f; }
    // zero the padding columns once (staging never writes them)
    for (int t = threadIdx.x; t < kMxRows * mp; t += blockDim.x) {
        if (t % mp >= m) { sz[t] = 0.0f; su[t] = 0.0f; sq[t] = 0.0f; }
    }
    const int64_t nchunks = (n + kMxRows - 1) / kMxRows;
    if ((int64_t)blockIdx.x < nchunks) fetch_mx(rz, ra, rq, mp, n, (int64_t)blockIdx.x * kMxRows, Z, AZ, Q, nb, has_q);
    cp_async_commit();
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();          // rows of chunk ch landed; the previous chunk's products are done
        stage_mx(sz, su, sq, rz, ra, rq, mp, n, ch * kMxRows, Z, AZ, Q, nb, has_q, sigma, csc, cscf, sigf);
        __syncthreads();          // tiles staged; the row buffers are free
        if (ch + gridDim.x < nchunks) fetch_mx(rz, ra, rq, mp, n, (ch + gridDim.x) * kMxRows, Z, AZ, Q, nb, has_q);
        cp_async_commit();
        if (act) {
            float acc[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) acc[e] = 0.0f;
            for (int half = 0; half < kMxRows; half += 32) {
#pragma unroll 4
                for (int r = half; r < half + 32; ++r) {
                    const float4 a = *reinterpret_cast<const float4*>(A + r * mp + 4 * ti);
                    const float4 b = *reinterpret_cast<const float4*>(B + r * mp + 4 * tj);
                    outer4(acc, a, b);
                }
                fold(hi, lo, acc);
#pragma unroll
                for (int e = 0; e < 16; ++e) acc[e] = 0.0f;
            }
        }
    }
    cp_async_wait_all();
    if (!act) return;
    double* out = partial + (int64_t)blockIdx.x * 3 * m * m + (int64_t)g * m * m;
    put_tile(out, m, 4 * ti, 4 * tj, hi, lo, g <= 1);
}

// out[j] = sum_b partial[b * width + j], fixed order, many CTAs
__global__ void k_sum_wide(int nblocks, int width, const double* __restrict__ partial, double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= width) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partial[(int64_t)b * width + j];
    out[j] = t;
}

// ------------------------------------------------------------------ update
constexpr int kUpRows = 32;

// Family F = [F_0 .. F_{nb-1}] (m columns): Pout = F C_P, Vout = F_0 C_VV + F C_P.
// With an FP64 F_0 and an FP64 Vout, the F_0 part of Vout is summed in
// double-word arithmetic (V keeps ~48-bit accuracy: A amplifies rounding noise
// in V by ||A|| / lambda, and FP64 FMAs would make the kernel FP64-pipe
// bound), accumulated as in the double-word update (exact products of the
// high parts, TwoSum on the high sum); all other sums are FP32.  Every output
// row depends only on the same input row and a chunk is staged before any of
// its rows is written (in place allowed: Vout may be F_0, Pout may be
// F_{nb-1}).
//
// Shared memory (byte offsets rounded up to 16): csw [kp][kp] and zw
// [rows][kp] double-word, then cpt [kp][cs] (C_P transposed, rows padded
// with zeros to mp = m rounded up to 4, row stride cs = mp + 4 so that the
// 16-byte loads of consecutive columns j fall in different banks), csf
// [kp][kp], zf [rows][mp] (the staged rows, zero past m): a row segment and
// a coefficient segment of 4 consecutive i are one 16-byte load each.
struct UpMxLayout {
    int mp, cs;
    size_t zw, cpt, csf, zf, bytes;
};
__host__ __device__ inline size_t up16(size_t b) { return (b + 15) & ~(size_t)15; }
__host__ __device__ inline UpMxLayout up_mx_layout(int m, int kp) {
    UpMxLayout L;
    L.mp = (m + 3) / 4 * 4;
    L.cs = L.mp + 4;
    L.zw = sizeof(dw) * kp * kp;
    L.cpt = up16(L.zw + sizeof(dw) * kUpRows * kp);
    L.csf = up16(L.cpt + sizeof(float) * kp * L.cs);
    L.zf = up16(L.csf + sizeof(float) * kp * kp);
    L.bytes = L.zf + sizeof(float) * kUpRows * L.mp;
    return L;
}

__global__ void __launch_bounds__(256) k_update_mx(int64_t n, int m, int kp, int nb, FamMx F,
                                                   const double* __restrict__ Cp, const double* __restrict__ Cvv,
                                                   void* __restrict__ Vout, int vo64, int64_t ldvo,
                                                   void* __restrict__ Pout, int po64, int64_t ldpo) {
    extern __shared__ __align__(16) unsigned char raw[];
    const UpMxLayout L = up_mx_layout(m, kp);
    const int mp = L.mp;
    dw* csw = reinterpret_cast<dw*>(raw);                    // [kp][kp]  C_VV + C_P (V rows), double-word
    dw* zw = reinterpret_cast<dw*>(raw + L.zw);              // [rows][kp] V rows, double-word
    float* cpt = reinterpret_cast<float*>(raw + L.cpt);      // [kp][cs] C_P transposed
    float* csf = reinterpret_cast<float*>(raw + L.csf);      // [kp][kp]
    float* zf = reinterpret_cast<float*>(raw + L.zf);        // [rows][mp]
    const bool v64 = F.f64[0] && vo64;
    const int cs = L.cs;
    for (int t = threadIdx.x; t < kp * cs; t += blockDim.x) {
        const int jj = t / cs, i = t - jj * cs;
        cpt[t] = i < m ? (float)Cp[i * kp + jj] : 0.0f;
    }
    for (int t = threadIdx.x; t < kp * kp; t += blockDim.x) {
        const double v = Cvv[t] + Cp[t];     // V rows of C_P are the first kp rows
        csw[t] = dw_from_double(v);
        csf[t] = (float)v;
    }
    for (int t = threadIdx.x; t < kUpRows * (mp - m); t += blockDim.x) {
        const int r = t / (mp - m), i = m + t - r * (mp - m);
        zf[r * mp + i] = 0.0f;
    }
    // thread t owns column j = t % kp of rows t / kp and t / kp + kUpRows / 2
    // (kp <= 16): two independent sums sharing the coefficient loads, each
    // summed in the same order as with one output per thread
    constexpr int kHalfUp = kUpRows / 2;
    const int r0 = threadIdx.x / kp, j = threadIdx.x - r0 * kp;
    const bool own = r0 < kHalfUp;
    const float* cj = cpt + j * cs;
    const int64_t nchunks = (n + kUpRows - 1) / kUpRows;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t row0 = ch * kUpRows;
        const int nrows = (int)((n - row0) < kUpRows ? (n - row0) : kUpRows);
        __syncthreads();
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if (b >= nb) break;
            const int nc = F.nc[b];
            for (int t = threadIdx.x; t < nrows * nc; t += blockDim.x) {
                const int r = t / nc, c = t - r * nc;
                const int64_t row = row0 + r;
                if (b == 0 && v64) {
                    const dw v = dw_from_double_fast(ldv(F, 0, row, c));
                    zw[r * kp + c] = v;
                    zf[r * mp + c] = v.hi;
                } else {
                    zf[r * mp + F.off[b] + c] = ldf(F, b, row, c);
                }
            }
        }
        __syncthreads();
        if (!own || r0 >= nrows) continue;
        // rows ra = r0 and rb = r0 + kUpRows / 2 (rb = ra, not stored, past nrows)
        const bool two = r0 + kHalfUp < nrows;
        const int ra = r0, rb = two ? r0 + kHalfUp : r0;
        const float* za = zf + ra * mp;
        const float* zb = zf + rb * mp;
        float resta = 0.0f, restb = 0.0f, pva = 0.0f, pvb = 0.0f;
        // i = kp .. m - 1 (then zeros to mp), in order
        int i = kp;
        for (; i < mp && (i & 3); ++i) {
            const float c = cj[i];
            resta = fmaf(za[i], c, resta);
            restb = fmaf(zb[i], c, restb);
        }
        for (; i < mp; i += 4) {
            const float4 c4 = *reinterpret_cast<const float4*>(cj + i);
            const float4 a4 = *reinterpret_cast<const float4*>(za + i);
            const float4 b4 = *reinterpret_cast<const float4*>(zb + i);
            resta = fmaf(a4.x, c4.x, resta); restb = fmaf(b4.x, c4.x, restb);
            resta = fmaf(a4.y, c4.y, resta); restb = fmaf(b4.y, c4.y, restb);
            resta = fmaf(a4.z, c4.z, resta); restb = fmaf(b4.z, c4.z, restb);
            resta = fmaf(a4.w, c4.w, resta); restb = fmaf(b4.w, c4.w, restb);
        }
        for (int q = 0; q < kp; ++q) {
            const float c = cj[q];
            pva = fmaf(za[q], c, pva);
            pvb = fmaf(zb[q], c, pvb);
        }
        const int64_t rowa = row0 + ra, rowb = row0 + rb;
        const float pa = pva + resta, pb = pvb + restb;
        if (po64) {
            static_cast<double*>(Pout)[rowa * ldpo + j] = f32_to_f64_bits(pa);
            if (two) static_cast<double*>(Pout)[rowb * ldpo + j] = f32_to_f64_bits(pb);
        } else {
            static_cast<float*>(Pout)[rowa * ldpo + j] = pa;
            if (two) static_cast<float*>(Pout)[rowb * ldpo + j] = pb;
        }
        if (v64) {
            const dw* zra = zw + ra * kp;
            const dw* zrb = zw + rb * kp;
            float vha = resta, vla = 0.0f, vhb = restb, vlb = 0.0f;
            for (int q = 0; q < kp; ++q) {
                const dw c = csw[q * kp + j];
                dw_fma_acc(vha, vla, zra[q], c);
                dw_fma_acc(vhb, vlb, zrb[q], c);
            }
            static_cast<double*>(Vout)[rowa * ldvo + j] = dw_to_double_fast(dw{vha, vla});
            if (two) static_cast<double*>(Vout)[rowb * ldvo + j] = dw_to_double_fast(dw{vhb, vlb});
        } else {
            float va = 0.0f, vb = 0.0f;
            for (int q = 0; q < kp; ++q) {
                const float c = csf[q * kp + j];
                va = fmaf(za[q], c, va);
                vb = fmaf(zb[q], c, vb);
            }
            va += resta;
            vb += restb;
            if (vo64) {
                static_cast<double*>(Vout)[rowa * ldvo + j] = f32_to_f64_bits(va);
                if (two) static_cast<double*>(Vout)[rowb * ldvo + j] = f32_to_f64_bits(vb);
            } else {
                static_cast<float*>(Vout)[rowa * ldvo + j] = va;
                if (two) static_cast<float*>(Vout)[rowb * ldvo + j] = vb;
            }
        }
    }
}

// V32 = V, U32 = A V - sigma V (formed in FP64, then rounded), X3 = A V - sigma V
// in FP64 (optional); n x kp blocks with leading dimension kp
__global__ void k_prepare_v(int64_t n, int kp, const double* __restrict__ V, const double* __restrict__ AV,
                            double sigma, float* __restrict__ V32, float* __restrict__ U32,
                            double* __restrict__ X3) {
    const int64_t total = n * kp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const double v = V[e];
        const double u = fma(-sigma, v, AV[e]);
        V32[e] = f64_to_f32_rn(v);
        U32[e] = f64_to_f32_rn(u);
        if (X3) X3[e] = u;
    }
}

// ------------------------------------------------------------------ FP32 stencil
constexpr int kSt = 256;

struct Ln {
    int nx, ny, nz, nc;
    float ih2;
};

// ax = L x; o1 = ax - lam_c x (optional); o2 = ax - sig x (optional); one
// thread per element, a CTA covers 256 elements of one x-line
template <bool D3>
__global__ void __launch_bounds__(kSt) k_lap32(Ln g, const float* __restrict__ x, int64_t ldx, float* __restrict__ ax,
                                               int64_t ldax, float* __restrict__ o1, int64_t ld1,
                                               const double* __restrict__ lam, float* __restrict__ o2, int64_t ld2,
                                               float sig) {
    const int t = blockIdx.x * kSt + threadIdx.x;
    if (t >= g.nx * g.nc) return;
    const int ix = t / g.nc, c = t - ix * g.nc;
    const int iy = blockIdx.y, iz = blockIdx.z;
    const int64_t row = ((int64_t)iz * g.ny + iy) * g.nx + ix;
    const float* xp = x + row * ldx + c;
    const int64_t sy = ldx * g.nx, sz = sy * g.ny;
    // sum of the differences x_c - x_nb (exact for a smooth field; missing
    // neighbours are zero), not 2d x_c - sum x_nb, which cancels
    const float xv = xp[0];
    float s = ((ix > 0 ? xv - xp[-ldx] : xv) + (ix < g.nx - 1 ? xv - xp[ldx] : xv)) +
              ((iy > 0 ? xv - xp[-sy] : xv) + (iy < g.ny - 1 ? xv - xp[sy] : xv));
    if (D3) s += (iz > 0 ? xv - xp[-sz] : xv) + (iz < g.nz - 1 ? xv - xp[sz] : xv);
    const float a = g.ih2 * s;
    if (ax) ax[row * ldax + c] = a;
    if (o1) o1[row * ld1 + c] = a - (float)lam[c] * xv;
    if (o2) o2[row * ld2 + c] = a - sig * xv;
}

// the same with four consecutive columns per thread (16-byte loads and
// stores; nc, the leading dimensions and the base addresses multiples of 4
// floats): a CTA covers 1024 elements of one x-line
template <bool D3>
__global__ void __launch_bounds__(kSt) k_lap32v(Ln g, const float* __restrict__ x, int64_t ldx, float* __restrict__ ax,
                                                int64_t ldax, float* __restrict__ o1, int64_t ld1,
                                                const double* __restrict__ lam, float* __restrict__ o2, int64_t ld2,
                                                float sig) {
    const int nq = g.nc >> 2;
    const int t = blockIdx.x * kSt + threadIdx.x;
    if (t >= g.nx * nq) return;
    const int ix = t / nq, c = (t - ix * nq) * 4;
    const int iy = blockIdx.y, iz = blockIdx.z;
    const int64_t row = ((int64_t)iz * g.ny + iy) * g.nx + ix;
    const float* xp = x + row * ldx + c;
    const int64_t sy = ldx * g.nx, sz = sy * g.ny;
    const float4 xv = *reinterpret_cast<const float4*>(xp);
    float4 s = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    // differences x_c - x_nb per direction, summed in the order of k_lap32
    auto diff = [&](bool in, int64_t off) -> float4 {
        if (!in) return xv;
        const float4 nb = *reinterpret_cast<const float4*>(xp + off);
        return make_float4(xv.x - nb.x, xv.y - nb.y, xv.z - nb.z, xv.w - nb.w);
    };
    const float4 a0 = diff(ix > 0, -ldx), a1 = diff(ix < g.nx - 1, ldx);
    const float4 b0 = diff(iy > 0, -sy), b1 = diff(iy < g.ny - 1, sy);
    s.x = (a0.x + a1.x) + (b0.x + b1.x);
    s.y = (a0.y + a1.y) + (b0.y + b1.y);
    s.z = (a0.z + a1.z) + (b0.z + b1.z);
    s.w = (a0.w + a1.w) + (b0.w + b1.w);
    if (D3) {
        const float4 c0 = diff(iz > 0, -sz), c1 = diff(iz < g.nz - 1, sz);
        s.x += c0.x + c1.x;
        s.y += c0.y + c1.y;
        s.z += c0.z + c1.z;
        s.w += c0.w + c1.w;
    }
    const float4 a = make_float4(g.ih2 * s.x, g.ih2 * s.y, g.ih2 * s.z, g.ih2 * s.w);
    if (ax) *reinterpret_cast<float4*>(ax + row * ldax + c) = a;
    if (o1) {
        const float l0 = (float)lam[c], l1 = (float)lam[c + 1], l2 = (float)lam[c + 2], l3 = (float)lam[c + 3];
        *reinterpret_cast<float4*>(o1 + row * ld1 + c) =
            make_float4(a.x - l0 * xv.x, a.y - l1 * xv.y, a.z - l2 * xv.z, a.w - l3 * xv.w);
    }
    if (o2)
        *reinterpret_cast<float4*>(o2 + row * ld2 + c) =
            make_float4(a.x - sig * xv.x, a.y - sig * xv.y, a.z - sig * xv.z, a.w - sig * xv.w);
}

// Y (FP64, ldy) = X (FP32, ldx), n x nc
__global__ void k_widen(int64_t n, int nc, const float* __restrict__ X, int64_t ldx, double* __restrict__ Y,
                        int64_t ldy) {
    const int64_t total = n * nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r;
        int c;
        split_index(e, nc, r, c);
        Y[r * ldy + c] = f32_to_f64_bits(X[r * ldx + c]);
    }
}

// Y (FP32, ldy) = X (FP64, ldx), n x nc
__global__ void k_narrow(int64_t n, int nc, const double* __restrict__ X, int64_t ldx, float* __restrict__ Y,
                         int64_t ldy) {
    const int64_t total = n * nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r;
        int c;
        split_index(e, nc, r, c);
        Y[r * ldy + c] = f64_to_f32_rn(X[r * ldx + c]);
    }
}

}  // namespace

int gram_mx_blocks() { return sm_count(); }

cudaError_t multi_gram_mx(int64_t n, int nb, const BlkMx* Z, const BlkMx* AZ, const BlkMx* Q, double sigma,
                          const double* colscale, double* partial, double* out, cudaStream_t s) {
    FamMx FZ = fam_mx(Z, nb), FA = fam_mx(AZ, nb), FQ = fam_mx(Q ? Q : AZ, nb);
    int m = 0;
    for (int i = 0; i < nb; ++i) m += Z[i].nc;
    const int mp = (m + 3) / 4 * 4;
    if (mp > 64) return cudaErrorInvalidValue;
    const int blocks = gram_mx_blocks();
    const size_t shm = sizeof(double) * 3 * kMxRows * mp + sizeof(float) * (3 * kMxRows * mp + mp);
    // above the 48 KB default: raise the kernel's limit to the largest size on
    // the current device (every call, so that each device a process uses gets it)
    {
        cudaError_t e = cudaFuncSetAttribute(k_gram_mx, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(double) * 3 * kMxRows * 64 +
                                                   sizeof(float) * (3 * kMxRows * 64 + 64)));
        if (e != cudaSuccess) return e;
    }
    k_gram_mx<<<blocks, kGramMxThreads, shm, s>>>(n, m, mp, nb, FZ, FA, FQ, Q ? 1 : 0, sigma, colscale, partial);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int width = 3 * m * m;
    k_sum_wide<<<(width + 127) / 128, 128, 0, s>>>(blocks, width, partial, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t block_update_mx(int64_t n, int nb, const BlkMx* F, int kp, const double* Cp, const double* Cvv,
                            void* Vout, int vo64, int64_t ldvo, void* Pout, int po64, int64_t ldpo, cudaStream_t s) {
    FamMx FF = fam_mx(F, nb);
    int m = 0;
    for (int i = 0; i < nb; ++i) m += F[i].nc;
    const size_t shm = up_mx_layout(m, kp).bytes;
    k_update_mx<<<sm_count() * 4, 256, shm, s>>>(n, m, kp, nb, FF, Cp, Cvv, Vout, vo64, ldvo, Pout, po64, ldpo);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t prepare_v_mx(int64_t n, int kp, const double* V, const double* AV, double sigma, float* V32, float* U32,
                         double* X3, cudaStream_t s) {
    k_prepare_v<<<grid_size_for(n * kp, 256, sm_count() * 8), 256, 0, s>>>(n, kp, V, AV, sigma, V32, U32, X3);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t lap32_apply_shifts(const Grid& g, int nc, const float* x, int64_t ldx, float* ax, int64_t ldax, float* o1,
                               int64_t ld1, const double* lam, float* o2, int64_t ld2, double sig, cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    Ln L{(int)g.nx, (int)g.ny, (int)g.nz, nc, (float)g.inv_h2()};
    auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const bool vec = nc % 4 == 0 && ldx % 4 == 0 && a16(x) && (!ax || (ldax % 4 == 0 && a16(ax))) &&
                     (!o1 || (ld1 % 4 == 0 && a16(o1))) && (!o2 || (ld2 % 4 == 0 && a16(o2)));
    if (vec) {
        dim3 gv((unsigned)((g.nx * (nc / 4) + kSt - 1) / kSt), (unsigned)g.ny, (unsigned)g.nz);
        if (g.d == 3) k_lap32v<true><<<gv, kSt, 0, s>>>(L, x, ldx, ax, ldax, o1, ld1, lam, o2, ld2, (float)sig);
        else k_lap32v<false><<<gv, kSt, 0, s>>>(L, x, ldx, ax, ldax, o1, ld1, lam, o2, ld2, (float)sig);
        count_launches(1);
        return cudaGetLastError();
    }
    dim3 gr((unsigned)((g.nx * nc + kSt - 1) / kSt), (unsigned)g.ny, (unsigned)g.nz);
    if (g.d == 3) k_lap32<true><<<gr, kSt, 0, s>>>(L, x, ldx, ax, ldax, o1, ld1, lam, o2, ld2, (float)sig);
    else k_lap32<false><<<gr, kSt, 0, s>>>(L, x, ldx, ax, ldax, o1, ld1, lam, o2, ld2, (float)sig);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t widen_block(int64_t n, int nc, const float* X, int64_t ldx, double* Y, int64_t ldy, cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    k_widen<<<grid_size_for(n * nc, 256, sm_count() * 8), 256, 0, s>>>(n, nc, X, ldx, Y, ldy);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t narrow_block(int64_t n, int nc, const double* X, int64_t ldx, float* Y, int64_t ldy, cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    k_narrow<<<grid_size_for(n * nc, 256, sm_count() * 8), 256, 0, s>>>(n, nc, X, ldx, Y, ldy);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plhr
