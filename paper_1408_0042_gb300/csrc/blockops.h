// Tall-skinny block kernels (residual, multi-Gram, coefficient update).
#pragma once

#include "plhr_internal.h"

namespace plhr {

int reduce_blocks();

// Asynchronous global -> shared copies of one 8- or 4-byte element (both
// addresses aligned to the size); wait_all waits for this thread's copies, a
// barrier after it makes every thread's copies visible.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
// 16 bytes (both addresses 16-byte aligned), bypassing L1
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// wait until at most N of this thread's most recent commit groups are pending
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// The 4x4 register tiles of the three m x m Gram outputs (T = ceil(m / 4)
// tiles per side), numbered compactly: t < T(T+1)/2 are the upper tiles
// ti <= tj of output 0 (Z^T Z) in row order, the next T(T+1)/2 the upper
// tiles of output 1 (U^T Q, symmetric in exact arithmetic: U^T T U, or U^T U
// without T, so its upper triangle is mirrored like output 0's), then the T^2
// tiles of output 2 in row order.  Returns false for t past the last tile.
// Numbering only the tiles that exist keeps the idle lanes of a warp at the
// end of the list, so fewer warps issue when m < 64.
__host__ __device__ __forceinline__ bool gram_tile(int t, int T, int& g, int& ti, int& tj) {
    const int nt0 = T * (T + 1) / 2, nt2 = T * T;
    g = 0; ti = 0; tj = 0;
    if (t < 2 * nt0) {
        g = t < nt0 ? 0 : 1;
        int r = 0, rem = t - g * nt0;
        while (rem >= T - r) { rem -= T - r; ++r; }
        ti = r; tj = r + rem;
        return true;
    }
    if (t >= 2 * nt0 + nt2) return false;
    const int u = t - 2 * nt0;
    g = 2;
    ti = u / T; tj = u % T;
    return true;
}
int residual_blocks(int kp);
int gram_max_m();

// R = sc_j (AV_j - lam_j V_j); out[0:kp] = sum R^2, out[kp:2kp] = sum (sc V)^2.
// partial: residual_blocks(kp) * 2 * kp doubles.
cudaError_t residual_norms(int64_t n, int kp, const double* V, int64_t ldv, const double* AV, int64_t ldav,
                           const double* lam, const double* sc, double* R, int64_t ldr, double* partial,
                           double* out, cudaStream_t s);

// Over nb blocks per family (Z, AZ, Q), columns scaled by colscale:
// out = [Z^T Z | U^T Q | Q^T Z] (3 m x m, row-major), U = AZ - sigma Z.
// Q == nullptr means Q = U (preconditioner T = I).
// partial: reduce_blocks() * 3 * m * m doubles.
cudaError_t multi_gram(int64_t n, int nb, const Blk<const double>* Z, const Blk<const double>* AZ,
                       const Blk<const double>* Q, double sigma, const double* colscale, double* partial,
                       double* out, cudaStream_t s);

// The same with a B Z family (generalized problem): out = [Z^T BZ | U^T Q |
// Q^T BZ], U = AZ - sigma BZ; BZ == nullptr is B = I (multi_gram).  The
// partial buffer is the same.
cudaError_t multi_gram_b(int64_t n, int nb, const Blk<const double>* Z, const Blk<const double>* AZ,
                         const Blk<const double>* Q, const Blk<const double>* BZ, double sigma,
                         const double* colscale, double* partial, double* out, cudaStream_t s);

// o1 = AX - BX diag(lam) and o2 = AX - sig BX (each optional), n x nc
cudaError_t shift_combine(int64_t n, int nc, const double* AX, int64_t ldax, const double* BX, int64_t ldbx,
                          const double* lam, double* o1, int64_t ld1, double sig, double* o2, int64_t ld2,
                          cudaStream_t s);

// Family F = [F_0 .. F_{nb-1}] (m columns): Pout = F C_P, Vout = F_0 C_VV + F C_P
// (in place allowed: Vout may be F_0, Pout may be F_{nb-1}).  When dotV is
// given, out[0:kp] = sum Vout .* dotV, out[kp:2kp] = sum dotV .^ 2.
cudaError_t block_update(int64_t n, int nb, const Blk<const double>* F, int kp, const double* Cp,
                         const double* Cvv, double* Vout, int64_t ldvo, double* Pout, int64_t ldpo,
                         const double* dotV, int64_t lddv, double* partial, double* out, cudaStream_t s);

// Y = X C for X n x kx (ldx), C kx x ky (row-major); in place allowed when
// ky <= kx and Y == X (rows are staged).
cudaError_t block_times_small(int64_t n, const double* X, int64_t ldx, int kx, const double* C, int ky, double* Y,
                              int64_t ldy, cudaStream_t s);

// Gather columns: Y[:, j] = X[:, idx[j]] for j < nc (device idx).
cudaError_t gather_columns(int64_t n, const double* X, int64_t ldx, const int* idx, int nc, double* Y, int64_t ldy,
                           cudaStream_t s);

// out[j] = sum_i X_ij Y_ij, out[kc + j] = sum_i X_ij^2 (partial: residual_blocks(kc) * 2 kc)
cudaError_t column_dots(int64_t n, int kc, const double* X, int64_t ldx, const double* Y, int64_t ldy,
                        double* partial, double* out, cudaStream_t s);

// Double-word forms of multi_gram and block_update (same arguments and
// results; inputs rounded once to hi + lo FP32 pairs, products and sums in
// double-word arithmetic on the FP32 pipes; partial: sm_count() * 3 m^2).
cudaError_t multi_gram_dw(int64_t n, int nb, const Blk<const double>* Z, const Blk<const double>* AZ,
                          const Blk<const double>* Q, double sigma, const double* colscale, double* partial,
                          double* out, cudaStream_t s);
cudaError_t block_update_dw(int64_t n, int nb, const Blk<const double>* F, int kp, const double* Cp, const double* Cvv,
                            double* Vout, int64_t ldvo, double* Pout, int64_t ldpo, cudaStream_t s);

// Seeded starting block: element (i, j) = (SplitMix64 output i*kc + j + 1 >> 11) * 2^-53 - 0.5.
cudaError_t seeded_block(int64_t n, int kc, uint64_t seed, double* X, int64_t ldx, cudaStream_t s);

}  // namespace plhr
