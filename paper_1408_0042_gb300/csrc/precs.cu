// Preconditioners other than AV-MG and TPA: a positive diagonal T = diag(d)
// (the form the paper's Section 5.3 preconditioner takes in its own basis)
// and a caller-supplied T applied through a callback; plus the FP64
// dispatcher over every kind.
#include <cmath>
#include <vector>

#include "plhr_internal.h"

namespace plhr {
namespace {

__global__ void __launch_bounds__(256) k_diag(int64_t n, int nc, const double* __restrict__ d,
                                              const double* __restrict__ r, int64_t ldr, double* __restrict__ w,
                                              int64_t ldw) {
    const int64_t total = n * nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i;
        int c;
        split_index(e, nc, i, c);
        w[i * ldw + c] = d[i] * r[i * ldr + c];
    }
}

}  // namespace

plhr_status prec_apply64(const plhr_prec* T, int nc, const double* r, int64_t ldr, double* w, double* work,
                         cudaStream_t s) {
    if (nc <= 0) return PLHR_OK;
    switch (T->kind) {
        case PREC_TPA:
            PLHR_TRY_CUDA(spectral_apply(T->sp, nc, r, ldr, w, work, s));
            return PLHR_OK;
        case PREC_DIAG:
            k_diag<<<grid_size_for(T->n_user * nc, 256, sm_count() * 16), 256, 0, s>>>(T->n_user, nc, T->diag, r, ldr,
                                                                                       w, nc);
            count_launches(1);
            PLHR_TRY_CUDA(cudaGetLastError());
            return PLHR_OK;
        case PREC_CALLBACK: {
            const plhr_status st = T->fn(T->ctx, nc, r, ldr, w, nc, (void*)s);
            if (st != PLHR_OK) {
                set_error("preconditioner callback returned status %d", (int)st);
                return st;
            }
            return PLHR_OK;
        }
        default:
            PLHR_TRY_CUDA(mg_vcycle(T->H, nc, r, ldr, w, nc, work, s));
            return PLHR_OK;
    }
}

}  // namespace plhr

using namespace plhr;

extern "C" plhr_status plhr_prec_diag(plhr_prec** out, int64_t n, const double* d, int is_device) {
    clear_error();
    if (!out || n < 1 || !d) {
        set_error("plhr_prec_diag: invalid argument");
        return PLHR_EINVAL;
    }
    std::vector<double> h(n);
    if (cudaMemcpy(h.data(), d, sizeof(double) * n, is_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost) !=
        cudaSuccess) {
        set_error("plhr_prec_diag: reading d failed");
        return PLHR_EINVAL;
    }
    for (int64_t i = 0; i < n; ++i)
        if (!(h[i] > 0) || !std::isfinite(h[i])) {
            set_error("plhr_prec_diag: d[%lld] is not positive and finite", (long long)i);
            return PLHR_EINVAL;
        }
    plhr_prec* T = new plhr_prec;
    T->kind = PREC_DIAG;
    T->n_user = n;
    if (cudaMalloc(&T->diag, sizeof(double) * n) != cudaSuccess ||
        cudaMemcpy(T->diag, h.data(), sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("plhr_prec_diag: device allocation or upload failed");
        plhr_prec_destroy(T);
        return PLHR_ENOMEM;
    }
    *out = T;
    return PLHR_OK;
}

extern "C" plhr_status plhr_prec_callback(plhr_prec** out, int64_t n, plhr_apply_fn fn, void* ctx) {
    clear_error();
    if (!out || n < 1 || !fn) {
        set_error("plhr_prec_callback: invalid argument");
        return PLHR_EINVAL;
    }
    plhr_prec* T = new plhr_prec;
    T->kind = PREC_CALLBACK;
    T->n_user = n;
    T->fn = fn;
    T->ctx = ctx;
    *out = T;
    return PLHR_OK;
}
