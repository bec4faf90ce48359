// Kernels of the mixed-precision iteration (FP64 V and A V, FP32 everything
// else); see mixed.cu.
#pragma once

#include "plhr_internal.h"

namespace plhr {

// A block of a family whose element type is FP64 (f64 = 1) or FP32.
struct BlkMx {
    const void* p = nullptr;
    int64_t ld = 0;
    int nc = 0;
    int f64 = 0;
    int is_u = 0;    // in the AZ family: the block already holds AZ - sigma Z
};

int gram_mx_blocks();

// out = [Z^T Z | U^T Q | Q^T Z] (3 m x m, FP64, row-major), U = (AZ - sigma Z),
// all columns scaled by colscale; Q == nullptr: Q = U.  FP32 products.
// partial: gram_mx_blocks() * 3 m^2 doubles.  m <= 64.
cudaError_t multi_gram_mx(int64_t n, int nb, const BlkMx* Z, const BlkMx* AZ, const BlkMx* Q, double sigma,
                          const double* colscale, double* partial, double* out, cudaStream_t s);

// The same three Grams on the tensor cores (gram_tc.cu): FP32 families only,
// each value split into three BF16 slices, FP32 accumulation in tensor
// memory folded into double-FP32 every 128 rows.  partial: gram_tc_blocks()
// * 3 m^2 doubles; *err (device) is set to 1 when a completion wait times
// out (the outputs are then invalid).  m <= 64.
int gram_tc_blocks();
cudaError_t multi_gram_tc(int64_t n, int nb, const BlkMx* Z, const BlkMx* AZ, const BlkMx* Q, double sigma,
                          const double* colscale, double* partial, double* out, int* err, cudaStream_t s);

// Pout = F C_P, Vout = F_0 C_VV + F C_P (types by the flags; in place allowed).
cudaError_t block_update_mx(int64_t n, int nb, const BlkMx* F, int kp, const double* Cp, const double* Cvv,
                            void* Vout, int vo64, int64_t ldvo, void* Pout, int po64, int64_t ldpo, cudaStream_t s);

// V32 = V, U32 = A V - sigma V (FP64, then rounded), X3 = A V - sigma V (FP64,
// optional); dense n x kp blocks
cudaError_t prepare_v_mx(int64_t n, int kp, const double* V, const double* AV, double sigma, float* V32, float* U32,
                         double* X3, cudaStream_t s);

// FP32 stencil: ax = L x; o1 = ax - lam_c x; o2 = ax - sig x (each optional)
cudaError_t lap32_apply_shifts(const Grid& g, int nc, const float* x, int64_t ldx, float* ax, int64_t ldax, float* o1,
                               int64_t ld1, const double* lam, float* o2, int64_t ld2, double sig, cudaStream_t s);

cudaError_t widen_block(int64_t n, int nc, const float* X, int64_t ldx, double* Y, int64_t ldy, cudaStream_t s);
cudaError_t narrow_block(int64_t n, int nc, const double* X, int64_t ldx, float* Y, int64_t ldy, cudaStream_t s);

}  // namespace plhr
