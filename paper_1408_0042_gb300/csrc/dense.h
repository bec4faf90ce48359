// Small dense FP64 device stages of the PLHR iteration (single warp / CTA).
#pragma once

#include "plhr_internal.h"

namespace plhr {

constexpr int kDenseMaxM = 64;        // largest trial-basis size m = 4 k'
constexpr int kDenseOK = 0;
constexpr int kDenseBreakdown = 1;    // G_L not positive definite
constexpr int kDenseNoConv = 2;       // Hessenberg QR did not converge
constexpr int kDenseRankLoss = 3;     // fewer than k' independent columns

struct DenseArgs {
    int m;               // trial basis size
    int kp;              // columns to extract (k')
    int nv;              // size of the V block (first nv columns of Z)
    const double* Gzz;   // m x m   (Z D)^T (Z D), D = diag(colscale)
    const double* Guq;   // m x m   (U D)^T (Q D)
    const double* Gqz;   // m x m   (Q D)^T (Z D)
    const double* colscale;  // m
    double* work;        // dense_work_doubles()
    double* Cp;          // out: m x kp
    double* Cvv;         // out: nv x kp (rows of the V block)
    int* tags;           // out: kp  (0 real, 1 pair real part, 2 cut column, 3 pair imaginary part)
    int* tag_partner;    // out: kp
    double* xi;          // out: 2 * kp  (re, im) of the selected xi, per unit
    int* out_int;        // out: [status, kept columns, selected units]
    long long* clk;      // optional: clock64() at stage boundaries (16 entries)
};

size_t dense_smem_bytes();
size_t dense_work_doubles();
cudaError_t dense_extract(const DenseArgs& a, cudaStream_t s);

// Convergence status from the residual column sums.
struct StatusArgs {
    int kp, k;
    double sigma, tol;
    const double* sums;   // [2 kp]: sum r^2, sum (Bv)^2
    const double* lam;    // kp
    double* lam_act;      // out: lam of the active columns
    int* active;          // out: kp active column list
    double* rel;          // out: kp relative residuals
    int* order;           // out: kp column order by |lam - sigma|
    int* hstat;           // out (device): [converged, n_active, nan]
};
cudaError_t dense_status(const StatusArgs& a, cudaStream_t s);

// Rayleigh quotients after the update (Alg. 3 step 13, Eq. lambda_complex)
// and the column scales that B-normalise V (step 14).
cudaError_t dense_rq(int kp, const double* dots, const int* tags, const int* partner, double* lam, double* scale,
                     cudaStream_t s);

// Standard Rayleigh-Ritz (Alg. 2 step 12): G_A c = theta G_B c for kp x kp
// Grams; C (kp x kp, columns ordered by |theta - sigma|, ties by theta) and theta.
// rowscale (kp, optional): C rows are multiplied by it (Ritz coefficients on
// the stored, unscaled columns).
cudaError_t dense_rr(int kp, const double* GA, const double* GB, double sigma, const double* rowscale, double* C,
                     double* theta, int* ok, cudaStream_t s);

}  // namespace plhr
