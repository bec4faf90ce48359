// C ABI: the projected-Gram pass in each of its arithmetic forms, on caller
// blocks (the solver's own Gram step, exposed so that each form can be
// checked element by element against plain products).
#include <algorithm>
#include <vector>

#include "blockops.h"
#include "mixed.h"
#include "plhr_internal.h"

using namespace plhr;

extern "C" {

plhr_status plhr_gram(int form, int64_t n, int nb, const int* ncols, const void* const* Z, const int64_t* ldz,
                      const void* const* AZ, const int64_t* ldaz, const void* const* Q, const int64_t* ldq,
                      double sigma, const double* colscale, double* out, void* stream) {
    clear_error();
    if (form < PLHR_GRAM_F64 || form > PLHR_GRAM_F32_TC) {
        set_error("plhr_gram: unknown form %d", form);
        return PLHR_EINVAL;
    }
    if (n < 0 || nb < 1 || nb > 4 || !ncols || !Z || !ldz || !AZ || !ldaz || !colscale || !out ||
        (Q && !ldq)) {
        set_error("plhr_gram: bad arguments");
        return PLHR_EINVAL;
    }
    int m = 0;
    for (int b = 0; b < nb; ++b) {
        if (ncols[b] < 0 || (ncols[b] > 0 && (!Z[b] || !AZ[b] || (Q && !Q[b]))) || ldz[b] < ncols[b] ||
            ldaz[b] < ncols[b] || (Q && ldq[b] < ncols[b])) {
            set_error("plhr_gram: bad block %d", b);
            return PLHR_EINVAL;
        }
        m += ncols[b];
    }
    if (m < 1 || m > 64) {
        set_error("plhr_gram: the trial basis needs 1..64 columns (got %d)", m);
        return PLHR_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = std::max(std::max(reduce_blocks(), gram_mx_blocks()), std::max(gram_tc_blocks(), sm_count()));
    double* partial = nullptr;
    int* err = nullptr;
    PLHR_TRY_CUDA(cudaMallocAsync(&partial, sizeof(double) * (size_t)blocks * 3 * m * m, s));
    struct Free {
        void* p; void* q; cudaStream_t s;
        ~Free() { cudaStreamSynchronize(s); if (p) cudaFree(p); if (q) cudaFree(q); }
    } fr{partial, nullptr, s};
    PLHR_TRY_CUDA(cudaMallocAsync(&err, sizeof(int), s));
    fr.q = err;
    PLHR_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    if (form == PLHR_GRAM_F64 || form == PLHR_GRAM_DW) {
        std::vector<Blk<const double>> zb(nb), ab(nb), qb(nb);
        for (int b = 0; b < nb; ++b) {
            zb[b] = {static_cast<const double*>(Z[b]), ldz[b], ncols[b]};
            ab[b] = {static_cast<const double*>(AZ[b]), ldaz[b], ncols[b]};
            if (Q) qb[b] = {static_cast<const double*>(Q[b]), ldq[b], ncols[b]};
        }
        if (form == PLHR_GRAM_F64)
            PLHR_TRY_CUDA(multi_gram(n, nb, zb.data(), ab.data(), Q ? qb.data() : nullptr, sigma, colscale, partial,
                                     out, s));
        else
            PLHR_TRY_CUDA(multi_gram_dw(n, nb, zb.data(), ab.data(), Q ? qb.data() : nullptr, sigma, colscale,
                                        partial, out, s));
    } else {
        std::vector<BlkMx> zb(nb), ab(nb), qb(nb);
        for (int b = 0; b < nb; ++b) {
            zb[b] = {Z[b], ldz[b], ncols[b], 0, 0};
            ab[b] = {AZ[b], ldaz[b], ncols[b], 0, 0};
            if (Q) qb[b] = {Q[b], ldq[b], ncols[b], 0, 0};
        }
        if (form == PLHR_GRAM_F32)
            PLHR_TRY_CUDA(multi_gram_mx(n, nb, zb.data(), ab.data(), Q ? qb.data() : nullptr, sigma, colscale,
                                        partial, out, s));
        else
            PLHR_TRY_CUDA(multi_gram_tc(n, nb, zb.data(), ab.data(), Q ? qb.data() : nullptr, sigma, colscale,
                                        partial, out, err, s));
    }
    int herr = 0;
    PLHR_TRY_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PLHR_TRY_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("plhr_gram: a tensor-core completion wait timed out");
        return PLHR_ECUDA;
    }
    return PLHR_OK;
}

}  // extern "C"
