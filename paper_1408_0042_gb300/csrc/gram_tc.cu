// The three projected Grams of the FP32 form on the tensor cores (tcgen05).
//
// One pass over the trial basis Z (m <= 64 columns), its image A Z and the
// T-harmonic images Q gives, with U = A Z - sigma Z and every column scaled
// by colscale,
//     Z^T Z,   U^T Q,   Q^T Z          (Eq. THarm_evp: G_L = U^T T U = U^T Q,
//                                       G_R = (T U)^T Z = Q^T Z for B = I)
// as FP64 m x m matrices.  The contraction runs over the n grid points.
//
// Split-precision compensation.  Each FP32 operand value x is split into
// three BF16 slices x = x0 + x1 + x2 (+ about 2^-24 |x|), and a product
// a b is formed from the six slice products of total order <= 2,
//     a0 b0 + a0 b1 + a1 b0 + a0 b2 + a1 b1 + a2 b0,
// each exact (8-bit x 8-bit significands), so a product carries about the
// FP32 rounding of its inputs (the dropped terms are below 2^-24 |a b|).
// The sums are what the tensor core rounds (each MMA adds its products to
// the FP32 accumulator with at most about one unit of the accumulator's last
// place), so the leading products a0 b0 and the five corrections (2^-8 and
// smaller) accumulate separately in tensor memory: the leading sum is read
// back after every chunk of 32 points (two MMA additions, no more rounding
// than the FP32 pipes' 32-row sums), the corrections after every 128 points;
// both are folded into a per-thread double-FP32 (hi, lo) sum with TwoSum, so
// the accumulation error does not grow with n.
//
// Tiles.  A chunk of 32 grid points is staged in shared memory as one
// K-major operand panel of 192 rows (U columns 0..63, Z columns 64..127, Q
// columns 128..191; padding columns and points past n are zero), per slice.
// One 128 x 128 x 16 MMA with A = panel rows 0..127 ([U; Z]) and B = panel
// rows 64..191 ([Z; Q]) yields
//     D = [ U^T Z  U^T Q ]
//         [ Z^T Z  Z^T Q ]
// so all three Grams come from one accumulator (U^T Z is not needed).
//
// Pipeline (one CTA of 512 threads per SM, chunks strided over the CTAs):
// the raw FP32 rows of the next four chunks are in flight into a ring of
// shared-memory row buffers (cp.async) while the current chunk is converted
// and the tensor cores multiply the one before; two panels alternate between
// conversion and MMA; two TMEM accumulators alternate by groups of four
// chunks (128 points), one read back while the other accumulates.  Thread 0
// issues the MMAs, 12 warps copy, all 16 convert, 12 read back.
#include "blockops.h"
#include "dword.h"
#include "mixed.h"
#include "tc.h"

namespace plhr {
namespace {

constexpr int kTcK = 32;                                   // grid points per chunk
constexpr int kGroup = 4;                                  // chunks per accumulator group (128 points)
constexpr int kRawBufs = 5;                                // raw row buffers: chunks in flight
constexpr int kTcThreads = 512;
constexpr int kPanelRows = 192;                            // U | Z | Q
constexpr int kCoreBytes = 128;                            // 8 rows x 16 bytes
constexpr uint32_t kLBO = kPanelRows / 8 * kCoreBytes;     // next core matrix along K
constexpr uint32_t kSBO = kCoreBytes;                      // next 8-row group along M / N
constexpr int kSliceBytes = kPanelRows * kTcK * 2;         // one BF16 slice of a panel
constexpr int kBufBytes = 3 * kSliceBytes;                 // three slices
constexpr int kOperandBytes = 2 * kBufBytes;               // two panels
constexpr int kRawStride = 192;                            // raw row: Z (64) | AZ (64) | Q (64) floats
constexpr int kRawBytes = kTcK * kRawStride * 4;           // one chunk of raw FP32 rows
constexpr int kMetaBytes = 4096;
constexpr int kSmemBytes = kOperandBytes + kRawBufs * kRawBytes + kMetaBytes;
// tensor memory: leading-product accumulators for even / odd chunks (columns
// 0, 128), correction accumulators for even / odd groups (256, 384)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kIdesc = tc::idesc_bf16_f32(128, 128);
constexpr long long kWaitCycles = 4LL << 30;               // about 2 s at 2 GHz

// slice pairs (a, b) of the six products of order <= 2:
// (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
__device__ __forceinline__ constexpr int slice_a(int p) { return p == 2 || p == 4 ? 1 : (p == 5 ? 2 : 0); }
__device__ __forceinline__ constexpr int slice_b(int p) { return p == 1 || p == 4 ? 1 : (p == 3 ? 2 : 0); }

struct ColTc {
    const float* z[64];   // element (i, j): z[j][i * ld[j]]
    const float* a[64];
    const float* q[64];
    int64_t ldz[64], lda[64], ldq[64];
    int is_u[64];
    int quad[3][16];      // columns 4q .. 4q + 3 of the family contiguous and 16-byte aligned in every row
};

// The column table in shared memory: indexing the kernel-parameter copy with
// a per-thread column serialises every access of a warp (one distinct
// constant-bank address per lane), shared memory serves it in one pass.
struct ColSh {
    const float* p[3][64];    // Z, AZ, Q
    int64_t ld[3][64];
    int is_u[64];
    int quad[3][16];
};

static_assert(512 + sizeof(ColSh) <= (size_t)kMetaBytes, "column table fits the meta area");

// TwoSum fold of 16 values into (hi, lo)
__device__ __forceinline__ void fold16(float* hi, float* lo, const float* v) {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const dw t = dw_two_sum(hi[e], v[e]);
        hi[e] = t.hi;
        lo[e] = __fadd_rn(lo[e], t.lo);
    }
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Start the asynchronous copies of the raw rows row0 .. row0 + 31 (those
// below n) of the Z, AZ and (with has_q) Q families into raw[row][192]:
// element (r, j) of family f at raw[r * 192 + 64 f + j].  Thread t < 384
// copies the column quad 4q .. 4q + 3 of family f for 4 rows (consecutive
// threads take consecutive quads, so a warp reads contiguous 256-byte row
// segments): one 16-byte copy per row when the quad is contiguous and aligned
// in memory, else one 4-byte copy per element.
__device__ __forceinline__ void fetch_tc(float* raw, int64_t n, int64_t row0, int m, const ColSh& C, int has_q) {
    const int t = threadIdx.x;
    if (t >= 3 * 16 * (kTcK / 4)) return;
    const int f = t / (16 * (kTcK / 4)), rem = t - f * (16 * (kTcK / 4));
    const int qd = rem & 15, part = rem >> 4;
    const int j0 = 4 * qd;
    if (j0 >= m || (f == 2 && !has_q)) return;
    const int64_t r0 = row0 + part * 4;
    const int cnt = (int)(n - r0 < 4 ? n - r0 : 4);
    float* dst = raw + part * 4 * kRawStride + 64 * f + j0;
    if (C.quad[f][qd]) {
        const int64_t ld = C.ld[f][j0];
        const float* src = C.p[f][j0] + r0 * ld;
        for (int r = 0; r < cnt; ++r, src += ld, dst += kRawStride) cp_async16(dst, src);
        return;
    }
    for (int j = j0; j < j0 + 4 && j < m; ++j) {
        const int64_t ld = C.ld[f][j];
        const float* src = C.p[f][j] + r0 * ld;
        float* d = dst + (j - j0);
        for (int r = 0; r < cnt; ++r, src += ld, d += kRawStride) cp_async4(d, src);
    }
}

// Convert the chunk of grid points row0 .. row0 + 31 (raw rows in shared
// memory) into the panel at buf.  Task t: panel row mr (column j of U, Z or
// Q) and half hf of core-matrix column ki (4 consecutive grid points): 4
// values, three 8-byte slice stores.  1536 tasks: three per thread, so the
// barrier after the staging waits for no thread with more work than the rest.
static_assert(kPanelRows * (kTcK / 4) % kTcThreads == 0, "staging tasks divide evenly");
__device__ __forceinline__ void stage_tc(unsigned char* buf, const float* raw, int64_t n, int64_t row0, int m,
                                         const ColSh& C, int has_q, float sigf, const float* cscf) {
    for (int t = threadIdx.x; t < kPanelRows * (kTcK / 4); t += kTcThreads) {
        const int mr = t % kPanelRows, kq = t / kPanelRows;
        const int ki = kq >> 1, hf = kq & 1;
        const int part = mr >> 6, j = mr & 63;
        float x[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) x[r] = 0.0f;
        if (j < m) {
            const float sf = cscf[j];
            const bool isu = C.is_u[j] != 0;
            const float* rr = raw + (4 * kq) * kRawStride;
#pragma unroll
            for (int r = 0; r < 4; ++r, rr += kRawStride) {
                if (row0 + 4 * kq + r >= n) break;
                if (part == 1) {
                    x[r] = rr[j] * sf;
                } else if (part == 2 && has_q) {
                    x[r] = rr[128 + j] * sf;
                } else {
                    const float z = rr[j] * sf, a = rr[64 + j] * sf;
                    x[r] = isu ? a : a - sigf * z;
                }
            }
        }
        __nv_bfloat16 s0[4], s1[4], s2[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) tc::split3(x[r], s0[r], s1[r], s2[r]);
        const int off = (ki * (kPanelRows / 8) + (mr >> 3)) * kCoreBytes + (mr & 7) * 16 + 8 * hf;
        *reinterpret_cast<uint2*>(buf + off) = make_uint2(pack2(s0[0], s0[1]), pack2(s0[2], s0[3]));
        *reinterpret_cast<uint2*>(buf + kSliceBytes + off) = make_uint2(pack2(s1[0], s1[1]), pack2(s1[2], s1[3]));
        *reinterpret_cast<uint2*>(buf + 2 * kSliceBytes + off) = make_uint2(pack2(s2[0], s2[1]), pack2(s2[2], s2[3]));
    }
}

__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(int64_t n, int m, const __grid_constant__ ColTc C,
                                                           int has_q, float sigf, const double* __restrict__ csc,
                                                           double* __restrict__ partial, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    float* raw = reinterpret_cast<float*>(smem + kOperandBytes);
    unsigned char* meta = smem + kOperandBytes + kRawBufs * kRawBytes;
    // [0..1] panels, [2..3] correction accumulators, [4..5] leading accumulators
    uint64_t* bars = reinterpret_cast<uint64_t*>(meta);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(meta + 64);
    float* cscf = reinterpret_cast<float*>(meta + 128);        // [64]
    ColSh& cols = *reinterpret_cast<ColSh*>(meta + 512);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < 64) {
        cscf[tid] = tid < m ? (float)csc[tid] : 0.0f;
        cols.p[0][tid] = C.z[tid];
        cols.p[1][tid] = C.a[tid];
        cols.p[2][tid] = C.q[tid];
        cols.ld[0][tid] = C.ldz[tid];
        cols.ld[1][tid] = C.lda[tid];
        cols.ld[2][tid] = C.ldq[tid];
        cols.is_u[tid] = C.is_u[tid];
    }
    if (tid < 48) cols.quad[tid / 16][tid % 16] = C.quad[tid / 16][tid % 16];
    if (tid == 0) {
        for (int i = 0; i < 6; ++i) tc::mbar_init(&bars[i], 1);
        tc::mbar_init_fence();
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    // read-back role: lane quarter q (TMEM lanes = panel rows 32q ..), column
    // quarter cq (accumulator columns 32cq ..); the U^T Z quadrant is skipped
    const int q = warp & 3, cq = warp >> 2;
    const bool useful = q >= 2 || cq >= 2;
    float hi[32], lo[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) { hi[e] = 0.0f; lo[e] = 0.0f; }

    const int64_t nchunks = (n + kTcK - 1) / kTcK;
    const int nloc = (int64_t)blockIdx.x < nchunks ? (int)((nchunks - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const int ngroups = (nloc + kGroup - 1) / kGroup;
    bool ok = true;
    int drained = 0, issued = 0;   // correction groups read back / chunks whose MMAs were issued

    // read back the accumulator at TMEM column col0 once the barrier's phase
    // with the given parity has completed, and fold it into (hi, lo)
    auto drain_acc = [&](uint64_t* bar, uint32_t parity, uint32_t col0) -> bool {
        const bool w = tc::mbar_wait(bar, parity, kWaitCycles);
        if (__syncthreads_or(!w)) return false;
        tc::fence_after_sync();
        if (useful) {
            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + col0 + (uint32_t)(32 * cq);
            float v[16];
            tc::tmem_ld16(ta, v);
            tc::tmem_ld_wait();
            fold16(hi, lo, v);
            tc::tmem_ld16(ta + 16, v);
            tc::tmem_ld_wait();
            fold16(hi + 16, lo + 16, v);
        }
        tc::fence_before_sync();
        return true;
    };
    // corrections of group g; leading products of chunk i
    auto drain = [&](int g) -> bool {
        return drain_acc(&bars[2 + (g & 1)], (uint32_t)((g >> 1) & 1), 256u + 128u * (uint32_t)(g & 1));
    };
    auto drain_main = [&](int i) -> bool {
        return drain_acc(&bars[4 + (i & 1)], (uint32_t)((i >> 1) & 1), 128u * (uint32_t)(i & 1));
    };

    // prologue: the copies of the first kRawBufs - 1 chunks, one commit group each
    for (int i = 0; i < kRawBufs - 1; ++i) {
        if (i < nloc) fetch_tc(raw + i * (kRawBytes / 4), n, ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * kTcK,
                               m, cols, has_q);
        cp_async_commit();
    }
    for (int i = 0; i < nloc; ++i) {
        const int64_t row0 = ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * kTcK;
        const int b = i & 1;
        unsigned char* buf = smem + b * kBufBytes;
        // this thread's raw rows of chunk i (the groups complete in order and one
        // is committed per chunk); the barrier below shows every thread's rows
        cp_async_wait_group<kRawBufs - 2>();
        bool w = true;
        if (i >= 2)            // the MMAs that read this panel two chunks ago have completed
            w = tc::mbar_wait(&bars[b], (uint32_t)(((i >> 1) - 1) & 1), kWaitCycles);
        if (__syncthreads_or(!w)) { ok = false; break; }
        stage_tc(buf, raw + (i % kRawBufs) * (kRawBytes / 4), n, row0, m, cols, has_q, sigf, cscf);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        // the raw buffer of chunk i - 1 is free: start the copies of chunk i + kRawBufs - 1 into it
        {
            const int inext = i + kRawBufs - 1;
            if (inext < nloc)
                fetch_tc(raw + (inext % kRawBufs) * (kRawBytes / 4), n,
                         ((int64_t)blockIdx.x + (int64_t)inext * gridDim.x) * kTcK, m, cols, has_q);
            cp_async_commit();
        }
        const int g = i / kGroup, a = g & 1;
        const bool group_start = i % kGroup == 0;
        const bool group_end = (i + 1) % kGroup == 0 || i == nloc - 1;
        if (tid == 0) {
            const uint32_t dmain = tmem + 128u * (uint32_t)(i & 1);
            const uint32_t dcorr = tmem + 256u + 128u * (uint32_t)a;
            const uint32_t sb = tc::smem_u32(buf);
#pragma unroll
            for (int s = 0; s < kTcK / 16; ++s) {
                const uint32_t kofs = (uint32_t)(2 * s) * kLBO;
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    const uint64_t ad = tc::smem_desc(sb + slice_a(p) * kSliceBytes + kofs, kLBO, kSBO);
                    const uint64_t bd = tc::smem_desc(sb + slice_b(p) * kSliceBytes + kofs + 8 * kCoreBytes, kLBO, kSBO);
                    if (p == 0) tc::mma_bf16(dmain, ad, bd, kIdesc, s ? 1u : 0u);
                    else tc::mma_bf16(dcorr, ad, bd, kIdesc, (!group_start || s || p > 1) ? 1u : 0u);
                }
            }
            tc::mma_commit(&bars[b]);
            tc::mma_commit(&bars[4 + (i & 1)]);
            if (group_end) tc::mma_commit(&bars[2 + a]);
        }
        ++issued;
        // the leading products of the previous chunk (their accumulator is next
        // written by chunk i + 1)
        if (i >= 1 && !drain_main(i - 1)) { ok = false; break; }
        // after the last chunk of group g, the corrections of group g - 1 (their
        // accumulator is next written by group g + 1)
        if (group_end && g >= 1 && drained == g - 1) {
            if (!drain(drained)) { ok = false; break; }
            ++drained;
        }
    }
    if (ok && nloc > 0 && !drain_main(nloc - 1)) ok = false;
    while (ok && drained < ngroups) {
        if (!drain(drained)) { ok = false; break; }
        ++drained;
    }
    cp_async_wait_all();
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        // let the MMAs already issued finish (bounded) before the TMEM is freed:
        // the last chunk's commit tracks every MMA issued before it
        if (issued > 0) {
            const int il = issued - 1;
            tc::mbar_wait(&bars[4 + (il & 1)], (uint32_t)((il >> 1) & 1), kWaitCycles);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
    if (!ok || !useful) return;
    double* out = partial + (int64_t)blockIdx.x * 3 * m * m;
    const int r = 32 * q + lane;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        const int c = 32 * cq + t;
        const double v = (double)hi[t] + (double)lo[t];
        if (r < 64) {                       // U column r against Q column c - 64
            const int i = r, j = c - 64;
            if (i < m && j < m) out[(int64_t)m * m + i * m + j] = v;
        } else if (c < 64) {                // Z column r - 64 against Z column c
            const int i = r - 64, j = c;
            if (i < m && j < m) out[i * m + j] = v;
        } else {                            // Z column r - 64 against Q column c - 64
            const int i = r - 64, j = c - 64;
            if (i < m && j < m) out[2 * (int64_t)m * m + j * m + i] = v;
        }
    }
}

// out[j] = sum_b partial[b * width + j], fixed order
__global__ void k_sum_tc(int nblocks, int width, const double* __restrict__ partial, double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= width) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partial[(int64_t)b * width + j];
    out[j] = t;
}

}  // namespace

int gram_tc_blocks() { return sm_count(); }

cudaError_t multi_gram_tc(int64_t n, int nb, const BlkMx* Z, const BlkMx* AZ, const BlkMx* Q, double sigma,
                          const double* colscale, double* partial, double* out, int* err, cudaStream_t s) {
    ColTc C{};
    int m = 0;
    for (int b = 0; b < nb; ++b) {
        if (Z[b].f64 || AZ[b].f64 || (Q && Q[b].f64)) return cudaErrorInvalidValue;   // FP32 families only
        for (int c = 0; c < Z[b].nc; ++c) {
            if (m >= 64) return cudaErrorInvalidValue;
            C.z[m] = static_cast<const float*>(Z[b].p) + c;
            C.a[m] = static_cast<const float*>(AZ[b].p) + c;
            C.q[m] = Q ? static_cast<const float*>(Q[b].p) + c : nullptr;
            C.ldz[m] = Z[b].ld;
            C.lda[m] = AZ[b].ld;
            C.ldq[m] = Q ? Q[b].ld : 0;
            C.is_u[m] = AZ[b].is_u;
            ++m;
        }
    }
    if (m == 0) return cudaSuccess;
    // column quads that one 16-byte copy per row can fetch: same block (the
    // pointers consecutive, the same leading dimension), aligned base, leading
    // dimension a multiple of 4 floats
    {
        const float* const* ptr[3] = {C.z, C.a, C.q};
        const int64_t* ldv[3] = {C.ldz, C.lda, C.ldq};
        for (int f = 0; f < 3; ++f)
            for (int q = 0; q < 16; ++q) {
                const int j0 = 4 * q;
                bool ok = j0 + 3 < m && ptr[f][j0] != nullptr;
                for (int c = 1; ok && c < 4; ++c)
                    ok = ptr[f][j0 + c] == ptr[f][j0] + c && ldv[f][j0 + c] == ldv[f][j0];
                ok = ok && (reinterpret_cast<uintptr_t>(ptr[f][j0]) & 15) == 0 && ldv[f][j0] % 4 == 0;
                C.quad[f][q] = ok ? 1 : 0;
            }
    }
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t nchunks = (n + kTcK - 1) / kTcK;
    int grid = gram_tc_blocks();
    if (nchunks < grid) grid = (int)(nchunks > 0 ? nchunks : 1);
    k_gram_tc<<<grid, kTcThreads, kSmemBytes, s>>>(n, m, C, Q ? 1 : 0, (float)sigma, colscale, partial, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int width = 3 * m * m;
    k_sum_tc<<<(width + 255) / 256, 256, 0, s>>>(grid, width, partial, out);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace plhr
