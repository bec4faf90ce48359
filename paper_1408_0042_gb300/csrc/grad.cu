// Gradient of eigenvalues with respect to a diagonal potential (the
// differentiation extension on top of the eigensolver): for H(V) = -1/2 Lap +
// diag(V) and B-orthonormal (here B = I) eigenvectors v_k, first-order
// perturbation theory (Hellmann-Feynman) gives d lambda_k / d V_i = v_k(i)^2,
// so the gradient of L = sum_k w_k lambda_k is g_i = sum_k w_k v_k(i)^2.
#include "plhr_internal.h"

namespace plhr {
namespace {

constexpr int kMaxGradK = 64;
struct Weights {
    double w[kMaxGradK];
};

__global__ void __launch_bounds__(256) k_eigval_grad(int64_t n, int k, const double* __restrict__ V, int64_t ldv,
                                                     Weights wt, double* __restrict__ g) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double* row = V + i * ldv;
        double s = 0.0;
        for (int j = 0; j < k; ++j) s = fma(wt.w[j] * row[j], row[j], s);
        g[i] = s;
    }
}

}  // namespace
}  // namespace plhr

using namespace plhr;

extern "C" plhr_status plhr_eigval_grad(int64_t n, int k, const double* V, int64_t ldv, const double* weights,
                                        double* g, void* stream) {
    clear_error();
    if (n < 1 || k < 1 || k > kMaxGradK || ldv < k || !V || !weights || !g) {
        set_error("plhr_eigval_grad: invalid argument (1 <= k <= %d, ldv >= k)", kMaxGradK);
        return PLHR_EINVAL;
    }
    Weights wt{};
    for (int j = 0; j < k; ++j) wt.w[j] = weights[j];
    k_eigval_grad<<<grid_size_for(n, 256, sm_count() * 8), 256, 0, (cudaStream_t)stream>>>(n, k, V, ldv, wt, g);
    count_launches(1);
    PLHR_TRY_CUDA(cudaGetLastError());
    return PLHR_OK;
}
