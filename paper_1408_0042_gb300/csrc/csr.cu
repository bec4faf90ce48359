// A general sparse symmetric operator in CSR form (FP64): the products the
// solver needs, y = alpha A x + beta x and A x with the fused shifted outputs
// A x - x diag(lam) and A x - sigma x, one thread per (row, column) element.
#include <algorithm>
#include <vector>

#include "plhr_internal.h"

namespace plhr {
namespace {

__device__ __forceinline__ double row_dot(const CsrData& A, int64_t row, const double* __restrict__ x, int64_t ldx,
                                          int c) {
    double a = 0.0;
    for (int64_t p = A.rowptr[row]; p < A.rowptr[row + 1]; ++p) a = fma(A.val[p], x[(int64_t)A.col[p] * ldx + c], a);
    return a;
}

__global__ void __launch_bounds__(256) k_csr_axpby(CsrData A, int nc, const double* __restrict__ x, int64_t ldx,
                                                   double* __restrict__ y, int64_t ldy, double alpha, double beta) {
    const int64_t total = A.n * nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t row;
        int c;
        split_index(e, nc, row, c);
        double v = alpha * row_dot(A, row, x, ldx, c);
        if (beta != 0.0) v = fma(beta, x[row * ldx + c], v);
        y[row * ldy + c] = v;
    }
}

__global__ void __launch_bounds__(256) k_csr_shifts(CsrData A, int nc, const double* __restrict__ x, int64_t ldx,
                                                    double* __restrict__ ax, int64_t ldax, double* __restrict__ o1,
                                                    int64_t ld1, const double* __restrict__ lam,
                                                    double* __restrict__ o2, int64_t ld2, double sig) {
    const int64_t total = A.n * nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t row;
        int c;
        split_index(e, nc, row, c);
        const double a = row_dot(A, row, x, ldx, c);
        const double xv = x[row * ldx + c];
        if (ax) ax[row * ldax + c] = a;
        if (o1) o1[row * ld1 + c] = a - lam[c] * xv;
        if (o2) o2[row * ld2 + c] = a - sig * xv;
    }
}

int nblk(int64_t total) { return grid_size_for(total, 256, sm_count() * 16); }

}  // namespace

cudaError_t csr_axpby(const CsrData& A, int nc, const double* x, int64_t ldx, double* y, int64_t ldy, double alpha,
                      double beta, cudaStream_t s) {
    const int64_t total = A.n * nc;
    if (total == 0) return cudaSuccess;
    k_csr_axpby<<<nblk(total), 256, 0, s>>>(A, nc, x, ldx, y, ldy, alpha, beta);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t csr_apply_shifts(const CsrData& A, int nc, const double* x, int64_t ldx, double* ax, int64_t ldax,
                             double* o1, int64_t ld1, const double* lam, double* o2, int64_t ld2, double sig,
                             cudaStream_t s) {
    const int64_t total = A.n * nc;
    if (total == 0) return cudaSuccess;
    k_csr_shifts<<<nblk(total), 256, 0, s>>>(A, nc, x, ldx, ax, ldax, o1, ld1, lam, o2, ld2, sig);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plhr

using namespace plhr;

extern "C" plhr_status plhr_op_csr(plhr_op** out, int64_t n, const int64_t* rowptr, const int32_t* col,
                                   const double* val, int is_device) {
    clear_error();
    if (!out || n < 1 || n > INT32_MAX || !rowptr || !col || !val) {
        set_error("plhr_op_csr: invalid argument");
        return PLHR_EINVAL;
    }
    // the structure is checked on the host, so that no kernel reads out of range
    std::vector<int64_t> rp(n + 1);
    const cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    if (cudaMemcpy(rp.data(), rowptr, sizeof(int64_t) * (n + 1), kind) != cudaSuccess) {
        set_error("plhr_op_csr: reading rowptr failed");
        return PLHR_EINVAL;
    }
    if (rp[0] != 0) {
        set_error("plhr_op_csr: rowptr[0] != 0");
        return PLHR_EINVAL;
    }
    for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) {
            set_error("plhr_op_csr: rowptr decreases at row %lld", (long long)i);
            return PLHR_EINVAL;
        }
    const int64_t nnz = rp[n];
    std::vector<int32_t> cl(nnz);
    std::vector<double> vl(nnz);
    if (nnz > 0 && (cudaMemcpy(cl.data(), col, sizeof(int32_t) * nnz, kind) != cudaSuccess ||
                    cudaMemcpy(vl.data(), val, sizeof(double) * nnz, kind) != cudaSuccess)) {
        set_error("plhr_op_csr: reading col/val failed");
        return PLHR_EINVAL;
    }
    for (int64_t p = 0; p < nnz; ++p)
        if (cl[p] < 0 || cl[p] >= n) {
            set_error("plhr_op_csr: column index %d out of range at entry %lld", cl[p], (long long)p);
            return PLHR_EINVAL;
        }
    plhr_op* op = new plhr_op;
    op->kind = OP_KIND_CSR;
    op->csr.n = n;
    op->csr.nnz = nnz;
    if (cudaMalloc(&op->csr.rowptr, sizeof(int64_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&op->csr.col, sizeof(int32_t) * std::max<int64_t>(nnz, 1)) != cudaSuccess ||
        cudaMalloc(&op->csr.val, sizeof(double) * std::max<int64_t>(nnz, 1)) != cudaSuccess) {
        plhr_op_destroy(op);
        set_error("plhr_op_csr: device allocation failed");
        return PLHR_ENOMEM;
    }
    if (cudaMemcpy(op->csr.rowptr, rp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        (nnz > 0 && (cudaMemcpy(op->csr.col, cl.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice) != cudaSuccess ||
                     cudaMemcpy(op->csr.val, vl.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice) != cudaSuccess))) {
        plhr_op_destroy(op);
        set_error("plhr_op_csr: upload failed");
        return PLHR_ECUDA;
    }
    op->g.d = 1;
    op->g.nx = n;
    op->g.ny = op->g.nz = 1;
    op->g.csr = &op->csr;
    *out = op;
    return PLHR_OK;
}
