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
// each exact in the tensor core's FP32 accumulation (8-bit x 8-bit
// significands), so a product carries about the FP32 rounding of its inputs
// (the dropped terms are below 2^-24 |a b|).  The FP32 accumulator in tensor
// memory sums 128 grid points; every 128 points it is read back and folded
// into a per-thread double-FP32 (hi, lo) sum with TwoSum, so the accumulation
// error does not grow with n (as in the FP32-pipe Gram of the same form).
//
// Tiles.  A chunk of 64 grid points is staged in shared memory as one
// K-major operand panel of 192 rows (U columns 0..63, Z columns 64..127, Q
// columns 128..191; padding columns and points past n are zero), per slice.
// One 128 x 128 x 16 MMA with A = panel rows 0..127 ([U; Z]) and B = panel
// rows 64..191 ([Z; Q]) yields
//     D = [ U^T Z  U^T Q ]
//         [ Z^T Z  Z^T Q ]
// so all three Grams come from one accumulator (U^T Z is not needed).  Two
// panels alternate so that the MMAs of one chunk run while the next chunk is
// converted; two TMEM accumulators alternate so that one is read back while
// the other accumulates.  One CTA of 512 threads per SM; thread 0 issues the
// MMAs, all 16 warps stage, 12 warps read back.
#include "blockops.h"
#include "dword.h"
#include "mixed.h"
#include "tc.h"

namespace plhr {
namespace {

constexpr int kTcK = 64;                                   // grid points per chunk
constexpr int kTcThreads = 512;
constexpr int kPanelRows = 192;                            // U | Z | Q
constexpr int kCoreBytes = 128;                            // 8 rows x 16 bytes
constexpr uint32_t kLBO = kPanelRows / 8 * kCoreBytes;     // next core matrix along K
constexpr uint32_t kSBO = kCoreBytes;                      // next 8-row group along M / N
constexpr int kSliceBytes = kPanelRows * kTcK * 2;         // one BF16 slice of a panel
constexpr int kBufBytes = 3 * kSliceBytes;                 // three slices
constexpr int kOperandBytes = 2 * kBufBytes;               // two panels
// shared memory kept past the panels: the descriptors address the panels
// only, but the allocation also covers the span the same descriptors would
// reach with the two byte offsets exchanged
constexpr int kGuardBytes = 48 * 1024;
constexpr int kMetaBytes = 4096;
constexpr int kSmemBytes = kOperandBytes + kGuardBytes + kMetaBytes;
constexpr uint32_t kTmemCols = 256;                        // two 128-column FP32 accumulators
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
};

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

// Convert the chunk of grid points row0 .. row0 + 63 into the panel at buf.
// Task t: panel row mr (column j of U, Z or Q) and core-matrix column ki
// (8 consecutive grid points): 8 values, three 16-byte slice stores.
__device__ __forceinline__ void stage_tc(unsigned char* buf, int64_t n, int64_t row0, int m, const ColTc& C,
                                         int has_q, float sigf, const float* cscf) {
    for (int t = threadIdx.x; t < kPanelRows * (kTcK / 8); t += kTcThreads) {
        const int mr = t % kPanelRows, ki = t / kPanelRows;
        const int part = mr >> 6, j = mr & 63;
        float x[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) x[r] = 0.0f;
        if (j < m) {
            const float sf = cscf[j];
            const int64_t r0 = row0 + 8 * ki;
            const bool needa = part == 0 || (part == 2 && !has_q);
            const bool isu = C.is_u[j] != 0;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int64_t row = r0 + r;
                if (row < n) {
                    float v;
                    if (part == 2 && has_q) {
                        v = C.q[j][row * C.ldq[j]] * sf;
                    } else {
                        const float z = C.z[j][row * C.ldz[j]] * sf;
                        if (needa) {
                            const float a = C.a[j][row * C.lda[j]] * sf;
                            v = isu ? a : a - sigf * z;
                        } else {
                            v = z;
                        }
                    }
                    x[r] = v;
                }
            }
        }
        __nv_bfloat16 s0[8], s1[8], s2[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) tc::split3(x[r], s0[r], s1[r], s2[r]);
        const int off = (ki * (kPanelRows / 8) + (mr >> 3)) * kCoreBytes + (mr & 7) * 16;
        *reinterpret_cast<uint4*>(buf + off) =
            make_uint4(pack2(s0[0], s0[1]), pack2(s0[2], s0[3]), pack2(s0[4], s0[5]), pack2(s0[6], s0[7]));
        *reinterpret_cast<uint4*>(buf + kSliceBytes + off) =
            make_uint4(pack2(s1[0], s1[1]), pack2(s1[2], s1[3]), pack2(s1[4], s1[5]), pack2(s1[6], s1[7]));
        *reinterpret_cast<uint4*>(buf + 2 * kSliceBytes + off) =
            make_uint4(pack2(s2[0], s2[1]), pack2(s2[2], s2[3]), pack2(s2[4], s2[5]), pack2(s2[6], s2[7]));
    }
}

__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(int64_t n, int m, const __grid_constant__ ColTc C,
                                                           int has_q, float sigf, const double* __restrict__ csc,
                                                           double* __restrict__ partial, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* meta = smem + kOperandBytes + kGuardBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(meta);        // [0..1] panels, [2..3] accumulators
    uint32_t* tslot = reinterpret_cast<uint32_t*>(meta + 64);
    float* cscf = reinterpret_cast<float*>(meta + 128);        // [64]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < 64) cscf[tid] = tid < m ? (float)csc[tid] : 0.0f;
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) tc::mbar_init(&bars[i], 1);
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
    const int ngroups = (nloc + 1) / 2;
    bool ok = true;
    int drained = 0, committed = 0;   // groups read back / whose accumulator commit was issued

    auto drain = [&](int g) -> bool {
        const int a = g & 1;
        const bool w = tc::mbar_wait(&bars[2 + a], (uint32_t)((g >> 1) & 1), kWaitCycles);
        if (__syncthreads_or(!w)) return false;
        tc::fence_after_sync();
        if (useful) {
            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * 128 + 32 * cq);
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

    for (int i = 0; i < nloc; ++i) {
        const int64_t row0 = ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * kTcK;
        const int b = i & 1;
        unsigned char* buf = smem + b * kBufBytes;
        if (i >= 2) {   // the MMAs that read this panel two chunks ago have completed
            const bool w = tc::mbar_wait(&bars[b], (uint32_t)(((i >> 1) - 1) & 1), kWaitCycles);
            if (__syncthreads_or(!w)) { ok = false; break; }
        }
        stage_tc(buf, n, row0, m, C, has_q, sigf, cscf);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        const int g = i >> 1, a = g & 1;
        const bool group_end = (i & 1) || i == nloc - 1;
        if (tid == 0) {
            const uint32_t d = tmem + (uint32_t)(a * 128);
            const uint32_t sb = tc::smem_u32(buf);
#pragma unroll
            for (int s = 0; s < kTcK / 16; ++s) {
                const uint32_t kofs = (uint32_t)(2 * s) * kLBO;
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    const uint64_t ad = tc::smem_desc(sb + slice_a(p) * kSliceBytes + kofs, kLBO, kSBO);
                    const uint64_t bd = tc::smem_desc(sb + slice_b(p) * kSliceBytes + kofs + 8 * kCoreBytes, kLBO, kSBO);
                    tc::mma_bf16(d, ad, bd, kIdesc, ((i & 1) | s | p) ? 1u : 0u);
                }
            }
            tc::mma_commit(&bars[b]);
            if (group_end) tc::mma_commit(&bars[2 + a]);
        }
        if (group_end) ++committed;
        if ((i & 1) && i >= 3) {
            if (!drain(drained)) { ok = false; break; }
            ++drained;
        }
    }
    while (ok && drained < ngroups) {
        if (!drain(drained)) { ok = false; break; }
        ++drained;
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        // let the MMAs already issued finish (bounded) before the TMEM is freed
        if (committed > 0) {
            const int gl = committed - 1;
            tc::mbar_wait(&bars[2 + (gl & 1)], (uint32_t)((gl >> 1) & 1), kWaitCycles);
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
