// Small dense FP64 stage of one PLHR iteration, run by a single warp on the
// device (no host round trip).  Input: the raw Grams of the trial basis
// Z = [V W S P] (Z*Z, U*Q with U = AZ - sigma Z, Q*Z, Q = T U) and the column
// scales of Z.  Steps:
//  1. B-orthonormalisation of Z (Alg. 2 step 6) done implicitly: with the
//     column-scaled Gram D Z*Z D = R^T R (Cholesky, columns whose pivot^2 falls
//     below 1e-12 are dropped), Z-hat = Z D R^{-1} is B-orthonormal and spans
//     [V], [V W], [V W S], [V W S P] blockwise, as the paper's blockwise
//     procedure does.
//  2. Projected T-harmonic problem (Eq. THarm_evp) in the Z-hat basis:
//     G_L = sym(R^-T D U*Q D R^-1), G_R = R^-T D Q*Z D R^-1; through tau = 1/xi
//     (Eq. THarm_evp_sinv): G_L = L L^T, C = L^-1 G_R L^-T, eigenpairs (tau, z)
//     of C, y = L^-T z.
//  3. Eigenvalues of C: Householder reduction to Hessenberg form and the
//     Francis double-shift QR iteration with Schur vectors (Golub & Van Loan,
//     "Matrix Computations", Sec. 7.4-7.5); eigenvectors of the quasi-triangular
//     Schur factor by back substitution.
//  4. Order by |xi| with each complex xi followed by its conjugate, select k'
//     (Alg. 3 steps 7-10), rotate complex y so Re(y) is orthogonal to Im(y)
//     and the longer of the two, build the real Y' = [Y0 YR yR~ YI].
//  5. Coefficients on the raw basis: P_new = Z C_P, V_new = V C_VV + P_new.
#include "dense.h"

#include <cfloat>
#include <mutex>

namespace plhr {
namespace {

constexpr int MAXM = kDenseMaxM;

struct cplx {
    double re, im;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    // Smith's algorithm
    if (fabs(b.re) >= fabs(b.im)) {
        double r = b.im / b.re, d = b.re + b.im * r;
        return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    } else {
        double r = b.re / b.im, d = b.im + b.re * r;
        return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
    }
}

__device__ __forceinline__ void wsync() { __syncwarp(); }

// ---------------------------------------------------------------- Cholesky with drop
// A (n x n, ld) symmetric, overwritten: upper triangle holds R for kept
// columns.  keep[j] = 1 if kept.  Returns number kept.  Pivot test relative
// to the original diagonal (1 after scaling).
__device__ int chol_drop(double* A, int n, int ld, int* keep, double tol) {
    const int lane = threadIdx.x;
    int nk = 0;
    for (int j = 0; j < n; ++j) {
        double p = A[j * ld + j];
        bool ok = (p > tol) && isfinite(p);
        wsync();
        if (lane == 0) keep[j] = ok ? 1 : 0;
        if (ok) {
            double r = sqrt(p);
            for (int l = j + 1 + lane; l < n; l += 32) A[j * ld + l] /= r;
            wsync();
            if (lane == 0) A[j * ld + j] = r;
            // trailing update of the upper triangle
            for (int idx = lane; idx < (n - j - 1) * (n - j - 1); idx += 32) {
                int a = j + 1 + idx / (n - j - 1), b = j + 1 + idx % (n - j - 1);
                if (b >= a) A[a * ld + b] -= A[j * ld + a] * A[j * ld + b];
            }
            ++nk;
        } else {
            // drop: row/column j take no further part
            for (int l = lane; l < n; l += 32) { A[j * ld + l] = 0.0; }
        }
        wsync();
    }
    return nk;
}

// X <- R^-T X R^-1 for upper triangular R (n x n) and square X (n x n); in place.
__device__ void congruence_rinv(const double* R, int ldr, double* X, int ldx, int n) {
    const int lane = threadIdx.x;
    // solve R^T Y = X  (forward substitution down the rows), one column per lane
    for (int c = lane; c < n; c += 32) {
        for (int i = 0; i < n; ++i) {
            double s = X[i * ldx + c];
            for (int l = 0; l < i; ++l) s -= R[l * ldr + i] * X[l * ldx + c];
            X[i * ldx + c] = s / R[i * ldr + i];
        }
    }
    wsync();
    // solve Z R = Y  row by row: z_j = (y_j - sum_{l<j} z_l R_lj) / R_jj
    for (int r = lane; r < n; r += 32) {
        for (int j = 0; j < n; ++j) {
            double s = X[r * ldx + j];
            for (int l = 0; l < j; ++l) s -= X[r * ldx + l] * R[l * ldr + j];
            X[r * ldx + j] = s / R[j * ldr + j];
        }
    }
    wsync();
}

// plain Cholesky A = L L^T (lower stored in A's lower triangle); false on failure
__device__ bool chol_lower(double* A, int n, int ld) {
    const int lane = threadIdx.x;
    bool ok = true;
    for (int j = 0; j < n; ++j) {
        double p = A[j * ld + j];
        if (!(p > 0.0) || !isfinite(p)) { ok = false; break; }
        double r = sqrt(p);
        wsync();
        for (int l = j + 1 + lane; l < n; l += 32) A[l * ld + j] /= r;
        wsync();
        if (lane == 0) A[j * ld + j] = r;
        for (int idx = lane; idx < (n - j - 1) * (n - j - 1); idx += 32) {
            int a = j + 1 + idx / (n - j - 1), b = j + 1 + idx % (n - j - 1);
            if (b <= a) A[a * ld + b] -= A[a * ld + j] * A[b * ld + j];
        }
        wsync();
    }
    wsync();
    return ok;
}

// ---------------------------------------------------------------- Hessenberg + QR
// Householder reduction of H (n x n) to upper Hessenberg; Z accumulates.
__device__ void hessenberg(double* H, double* Z, int n, int ld, double* v) {
    const int lane = threadIdx.x;
    for (int i = lane; i < n * n; i += 32) Z[(i / n) * ld + i % n] = (i / n == i % n) ? 1.0 : 0.0;
    wsync();
    for (int k = 0; k < n - 2; ++k) {
        // x = H[k+1:n, k]
        double ss = 0.0;
        for (int i = k + 1 + lane; i < n; i += 32) ss += H[i * ld + k] * H[i * ld + k];
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        double alpha = sqrt(ss);
        double x0 = H[(k + 1) * ld + k];
        if (alpha == 0.0) continue;
        if (x0 > 0) alpha = -alpha;
        // v = x - alpha e1, normalised so that P = I - 2 v v^T / (v^T v)
        for (int i = k + 1 + lane; i < n; i += 32) v[i] = H[i * ld + k];
        wsync();
        if (lane == 0) v[k + 1] = x0 - alpha;
        wsync();
        double vv = ss - x0 * x0 + (x0 - alpha) * (x0 - alpha);
        if (vv == 0.0) continue;
        double beta = 2.0 / vv;
        // H = P H : rows k+1..n-1, all columns
        for (int c = lane; c < n; c += 32) {
            double s = 0.0;
            for (int i = k + 1; i < n; ++i) s += v[i] * H[i * ld + c];
            s *= beta;
            for (int i = k + 1; i < n; ++i) H[i * ld + c] -= s * v[i];
        }
        wsync();
        // H = H P : all rows, columns k+1..n-1
        for (int r = lane; r < n; r += 32) {
            double s = 0.0;
            for (int i = k + 1; i < n; ++i) s += H[r * ld + i] * v[i];
            s *= beta;
            for (int i = k + 1; i < n; ++i) H[r * ld + i] -= s * v[i];
        }
        // Z = Z P
        for (int r = lane; r < n; r += 32) {
            double s = 0.0;
            for (int i = k + 1; i < n; ++i) s += Z[r * ld + i] * v[i];
            s *= beta;
            for (int i = k + 1; i < n; ++i) Z[r * ld + i] -= s * v[i];
        }
        wsync();
        for (int i = k + 2 + lane; i < n; i += 32) H[i * ld + k] = 0.0;
        wsync();
    }
}

// Apply the reflector I - tau u u^T (u[0] = 1, length nr = 2 or 3) to rows
// k..k+nr-1 of H (columns c0..n-1) and columns k..k+nr-1 (rows 0..r1) of H and Z.
__device__ void apply_refl(double* H, double* Z, int n, int ld, int k, int nr, double u1, double u2, double tau,
                           int c0, int r1) {
    const int lane = threadIdx.x;
    for (int c = c0 + lane; c < n; c += 32) {
        double s = H[k * ld + c] + u1 * H[(k + 1) * ld + c] + (nr == 3 ? u2 * H[(k + 2) * ld + c] : 0.0);
        s *= tau;
        H[k * ld + c] -= s;
        H[(k + 1) * ld + c] -= s * u1;
        if (nr == 3) H[(k + 2) * ld + c] -= s * u2;
    }
    wsync();
    for (int r = lane; r <= r1; r += 32) {
        double s = H[r * ld + k] + u1 * H[r * ld + k + 1] + (nr == 3 ? u2 * H[r * ld + k + 2] : 0.0);
        s *= tau;
        H[r * ld + k] -= s;
        H[r * ld + k + 1] -= s * u1;
        if (nr == 3) H[r * ld + k + 2] -= s * u2;
    }
    for (int r = lane; r < n; r += 32) {
        double s = Z[r * ld + k] + u1 * Z[r * ld + k + 1] + (nr == 3 ? u2 * Z[r * ld + k + 2] : 0.0);
        s *= tau;
        Z[r * ld + k] -= s;
        Z[r * ld + k + 1] -= s * u1;
        if (nr == 3) Z[r * ld + k + 2] -= s * u2;
    }
    wsync();
}

// Householder vector for (x, y[, z]): returns u1, u2, tau with
// (I - tau u u^T) (x, y, z)^T = (beta, 0, 0)^T, u = (1, u1, u2).
__device__ __forceinline__ void house3(double x, double y, double z, int nr, double& u1, double& u2, double& tau) {
    double nrm = sqrt(x * x + y * y + (nr == 3 ? z * z : 0.0));
    if (nrm == 0.0 || (y == 0.0 && (nr == 2 || z == 0.0))) {
        u1 = 0.0; u2 = 0.0; tau = 0.0;
        return;
    }
    double beta = x > 0 ? -nrm : nrm;
    double v0 = x - beta;
    u1 = y / v0;
    u2 = nr == 3 ? z / v0 : 0.0;
    tau = (beta - x) / beta;
}

// Givens rotation making the 2x2 block at (p, p+1) upper triangular when its
// eigenvalues are real; applied to H rows/cols and Z columns.
__device__ void split_real_2x2(double* H, double* Z, int n, int ld, int p) {
    const int lane = threadIdx.x;
    double a = H[p * ld + p], b = H[p * ld + p + 1], c = H[(p + 1) * ld + p], d = H[(p + 1) * ld + p + 1];
    double hf = 0.5 * (a - d);
    double disc = hf * hf + b * c;
    if (disc < 0.0) return;
    double sq = sqrt(disc);
    // eigenvalue mu with eigenvector (b, mu - a) or (mu - d, c)
    double mu = 0.5 * (a + d) + (hf >= 0 ? sq : -sq);
    double x1, x2;
    if (fabs(b) + fabs(mu - a) >= fabs(mu - d) + fabs(c)) { x1 = b; x2 = mu - a; }
    else { x1 = mu - d; x2 = c; }
    double r = hypot(x1, x2);
    if (r == 0.0) return;
    double cs = x1 / r, sn = x2 / r;
    // G = [cs -sn; sn cs] with first column the eigenvector: H <- G^T H G
    wsync();
    for (int col = p + lane; col < n; col += 32) {
        double h1 = H[p * ld + col], h2 = H[(p + 1) * ld + col];
        H[p * ld + col] = cs * h1 + sn * h2;
        H[(p + 1) * ld + col] = -sn * h1 + cs * h2;
    }
    wsync();
    for (int row = lane; row <= p + 1; row += 32) {
        double h1 = H[row * ld + p], h2 = H[row * ld + p + 1];
        H[row * ld + p] = cs * h1 + sn * h2;
        H[row * ld + p + 1] = -sn * h1 + cs * h2;
    }
    for (int row = lane; row < n; row += 32) {
        double z1 = Z[row * ld + p], z2 = Z[row * ld + p + 1];
        Z[row * ld + p] = cs * z1 + sn * z2;
        Z[row * ld + p + 1] = -sn * z1 + cs * z2;
    }
    wsync();
    if (lane == 0) H[(p + 1) * ld + p] = 0.0;
    wsync();
}

// Francis double-shift QR on Hessenberg H (n x n) -> real Schur form, Z updated.
// Returns false if an eigenvalue fails to converge.
__device__ bool francis_qr(double* H, double* Z, int n, int ld) {
    const int lane = threadIdx.x;
    const double eps = DBL_EPSILON;
    double anorm = 0.0;
    for (int i = lane; i < n * n; i += 32) {
        int r = i / n, c = i % n;
        if (c >= r - 1) anorm = fmax(anorm, fabs(H[r * ld + c]));
    }
    for (int o = 16; o > 0; o >>= 1) anorm = fmax(anorm, __shfl_xor_sync(0xffffffffu, anorm, o));
    if (anorm == 0.0) anorm = 1.0;
    int hi = n - 1;
    int its = 0, total_its = 0;
    while (hi >= 0) {
        // locate the lowest negligible subdiagonal in [1, hi]
        int l = hi;
        while (l > 0) {
            double s = fabs(H[(l - 1) * ld + l - 1]) + fabs(H[l * ld + l]);
            if (s == 0.0) s = anorm;
            if (fabs(H[l * ld + l - 1]) <= eps * s) break;
            --l;
        }
        wsync();
        if (l > 0 && lane == 0) H[l * ld + l - 1] = 0.0;
        wsync();
        if (l == hi) {
            --hi;
            its = 0;
            continue;
        }
        if (l == hi - 1) {
            split_real_2x2(H, Z, n, ld, hi - 1);
            hi -= 2;
            its = 0;
            continue;
        }
        if (its >= 40) {
            // Stalled window: a (near-)defective cluster of numerically equal
            // eigenvalues converges only linearly.  Deflate at the smallest
            // subdiagonal when it is below 1e-7 ||H||: this moves eigenvalues by
            // about that much, and only a basis of the cluster is needed.
            int jm = l + 1;
            double vm = fabs(H[(l + 1) * ld + l]);
            for (int j = l + 2; j <= hi; ++j) {
                double v = fabs(H[j * ld + j - 1]);
                if (v < vm) { vm = v; jm = j; }
            }
            if (vm <= 1e-7 * anorm) {
                wsync();
                if (lane == 0) H[jm * ld + jm - 1] = 0.0;
                wsync();
                its = 0;
                continue;
            }
        }
        if (++total_its > 100 * n) return false;
        ++its;
        double s, t;
        if (its % 10 == 0) {
            // exceptional shift
            double w = fabs(H[hi * ld + hi - 1]) + fabs(H[(hi - 1) * ld + hi - 2]);
            s = 1.5 * w;
            t = w * w;
        } else {
            double a = H[(hi - 1) * ld + hi - 1], b = H[(hi - 1) * ld + hi], c = H[hi * ld + hi - 1],
                   d = H[hi * ld + hi];
            s = a + d;
            t = a * d - b * c;
        }
        // first column of (H - s1 I)(H - s2 I) at rows l, l+1, l+2
        double h00 = H[l * ld + l], h01 = H[l * ld + l + 1], h10 = H[(l + 1) * ld + l],
               h11 = H[(l + 1) * ld + l + 1], h21 = H[(l + 2) * ld + l + 1];
        double x = h00 * h00 + h01 * h10 - s * h00 + t;
        double y = h10 * (h00 + h11 - s);
        double z = h10 * h21;
        for (int k = l; k <= hi - 1; ++k) {
            int nr = (k < hi - 1) ? 3 : 2;
            double u1, u2, tau;
            house3(x, y, z, nr, u1, u2, tau);
            if (tau != 0.0) {
                int c0 = k > l ? k - 1 : l;
                int r1 = (k + 3 < hi) ? k + 3 : hi;
                apply_refl(H, Z, n, ld, k, nr, u1, u2, tau, c0, r1);
                // rows above the active block, for the full Schur form
                (void)r1;
            }
            if (k > l && lane == 0) {
                H[(k + 1) * ld + k - 1] = 0.0;
                if (nr == 3) H[(k + 2) * ld + k - 1] = 0.0;
            }
            wsync();
            if (k < hi - 1) {
                x = H[(k + 1) * ld + k];
                y = H[(k + 2) * ld + k];
                z = (k < hi - 2) ? H[(k + 3) * ld + k] : 0.0;
            }
            wsync();
        }
    }
    return true;
}

// ---------------------------------------------------------------- eigenvectors
// Eigenvector x (complex, length n) of quasi-triangular T for eigenvalue lam at
// diagonal position p (p = first row of a 2x2 block for a complex lam).
// Sequential; executed by one lane.
__device__ void schur_eigvec(const double* T, int n, int ld, int p, bool block2, cplx lam, cplx* x,
                             double smallnum) {
    for (int i = 0; i < n; ++i) x[i] = {0.0, 0.0};
    int top;
    if (!block2) {
        x[p] = {1.0, 0.0};
        top = p - 1;
    } else {
        // (T_pp - lam) x_p + T_p,p+1 x_p+1 = 0
        x[p] = {T[p * ld + p + 1], 0.0};
        x[p + 1] = csub(lam, cplx{T[p * ld + p], 0.0});
        top = p - 1;
    }
    int i = top;
    while (i >= 0) {
        bool two = (i > 0) && (T[i * ld + i - 1] != 0.0);
        if (!two) {
            cplx s = {0.0, 0.0};
            for (int l = i + 1; l < n; ++l) s = cadd(s, cmul(cplx{T[i * ld + l], 0.0}, x[l]));
            cplx d = csub(cplx{T[i * ld + i], 0.0}, lam);
            if (fabs(d.re) + fabs(d.im) < smallnum) d = {smallnum, 0.0};
            x[i] = cdiv(cplx{-s.re, -s.im}, d);
            i -= 1;
        } else {
            // 2x2 diagonal block at rows (i-1, i)
            int a = i - 1;
            cplx s1 = {0.0, 0.0}, s2 = {0.0, 0.0};
            for (int l = i + 1; l < n; ++l) {
                s1 = cadd(s1, cmul(cplx{T[a * ld + l], 0.0}, x[l]));
                s2 = cadd(s2, cmul(cplx{T[i * ld + l], 0.0}, x[l]));
            }
            cplx m11 = csub(cplx{T[a * ld + a], 0.0}, lam), m12 = {T[a * ld + i], 0.0};
            cplx m21 = {T[i * ld + a], 0.0}, m22 = csub(cplx{T[i * ld + i], 0.0}, lam);
            cplx det = csub(cmul(m11, m22), cmul(m12, m21));
            if (fabs(det.re) + fabs(det.im) < smallnum) det = {smallnum, 0.0};
            cplx r1 = {-s1.re, -s1.im}, r2 = {-s2.re, -s2.im};
            x[a] = cdiv(csub(cmul(m22, r1), cmul(m12, r2)), det);
            x[i] = cdiv(csub(cmul(m11, r2), cmul(m21, r1)), det);
            i -= 2;
        }
        // rescale to avoid overflow
        double mx = 0.0;
        for (int l = i + 1; l < n; ++l) mx = fmax(mx, fabs(x[l].re) + fabs(x[l].im));
        if (mx > 1e100) {
            for (int l = 0; l < n; ++l) { x[l].re /= mx; x[l].im /= mx; }
        }
    }
}

// ---------------------------------------------------------------- the kernel
// Shared-memory matrices use a row stride of MAXM + 1 doubles so that
// column-wise accesses by the lanes of the warp fall in distinct banks.
constexpr int LDS = MAXM + 1;
struct Smem {
    double H[MAXM * LDS];
    double Z[MAXM * LDS];
    double A[MAXM * LDS];    // scaled Z*Z -> R
    double B[MAXM * LDS];    // G_L -> L
    double v[MAXM];
    double t[MAXM];          // column scale of the raw basis
    int keep[MAXM];
    int kidx[MAXM];          // kept -> raw index
    double eig_re[MAXM], eig_im[MAXM];
    int eig_pos[MAXM];       // diagonal position in T
    int eig_blk[MAXM];       // 1 if from a 2x2 block
    int order[MAXM];
    int partner[MAXM];
    cplx x[16 * MAXM];       // eigenvector workspace, one per selected unit
};

__global__ void __launch_bounds__(32) k_extract(DenseArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    const int lane = threadIdx.x;
    const int m = a.m, kp = a.kp;
    const int ld = LDS;
    double* G = a.work;  // global scratch: [3][m][m] of scaled, compacted matrices
#define STAMP(i) do { if (a.clk && lane == 0) a.clk[i] = clock64(); } while (0)
    STAMP(0);
    // ---- 1. scaling and Cholesky with drop of the B-Gram.  The implicit
    // basis Z D R^{-1} amplifies Gram rounding by cond(R)^2; if G_L then fails
    // to be positive definite, the pass is repeated with a stricter drop
    // threshold (fewer, better conditioned columns).
    // The Grams are of the scaled columns Z diag(colscale); t normalises them.
    const double drop_tols[3] = {1e-12, 1e-9, 1e-6};
    int attempt = 0;
    int nk = 0, nvk = 0;
retry:
    for (int i = lane; i < m; i += 32) {
        double g = a.Gzz[i * m + i];
        S.t[i] = (g > 0.0 && isfinite(g)) ? 1.0 / sqrt(g) : 0.0;
    }
    wsync();
    for (int i = lane; i < m * m; i += 32) {
        int r = i / m, c = i % m;
        S.A[r * ld + c] = a.Gzz[i] * S.t[r] * S.t[c];
    }
    wsync();
    nk = chol_drop(S.A, m, ld, S.keep, drop_tols[attempt]);
    if (lane == 0) {
        int q = 0;
        for (int j = 0; j < m; ++j)
            if (S.keep[j] && S.t[j] != 0.0) S.kidx[q++] = j;
        nk = q;
        a.out_int[1] = nk;
    }
    nk = __shfl_sync(0xffffffffu, nk, 0);
    wsync();
    // kept count in the V block
    nvk = 0;
    for (int q = 0; q < nk; ++q) nvk += (S.kidx[q] < a.nv) ? 1 : 0;
    // columns of V may be dropped (nearly parallel Ritz vectors of a converged
    // cluster); the selection needs k' kept columns overall
    if (nvk < 1 || nk < kp) {
        if (lane == 0) a.out_int[0] = kDenseRankLoss;
        return;
    }
    // compact R (upper) into H temporarily -> keep in A compacted
    for (int i = lane; i < nk * nk; i += 32) {
        int r = i / nk, c = i % nk;
        S.H[r * ld + c] = (c >= r) ? S.A[S.kidx[r] * ld + S.kidx[c]] : 0.0;
    }
    wsync();
    for (int i = lane; i < nk * nk; i += 32) S.A[(i / nk) * ld + i % nk] = S.H[(i / nk) * ld + i % nk];
    wsync();
    STAMP(1);
    // ---- 2. projected G_L, G_R in the orthonormal basis
    double* GL = G;               // nk x nk, ld nk (global scratch)
    double* GR = G + m * m;
    for (int i = lane; i < nk * nk; i += 32) {
        int r = i / nk, c = i % nk;
        int rr = S.kidx[r], cc = S.kidx[c];
        double uq = a.Guq[rr * m + cc], qu = a.Guq[cc * m + rr];
        S.B[r * ld + c] = 0.5 * (uq + qu) * S.t[rr] * S.t[cc];      // G_L = sym(U^T Q)
        S.H[r * ld + c] = a.Gqz[rr * m + cc] * S.t[rr] * S.t[cc];   // G_R[r][c] = q_r . z_c
    }
    wsync();
    congruence_rinv(S.A, ld, S.B, ld, nk);
    congruence_rinv(S.A, ld, S.H, ld, nk);
    // symmetrise G_L exactly
    for (int i = lane; i < nk * nk; i += 32) {
        int r = i / nk, c = i % nk;
        if (c > r) {
            double s = 0.5 * (S.B[r * ld + c] + S.B[c * ld + r]);
            S.B[r * ld + c] = s;
            S.B[c * ld + r] = s;
        }
    }
    wsync();
    for (int i = lane; i < nk * nk; i += 32) { GL[i] = S.B[(i / nk) * ld + i % nk]; GR[i] = S.H[(i / nk) * ld + i % nk]; }
    wsync();
    // ---- Cholesky G_L = L L^T
    bool ok = chol_lower(S.B, nk, ld);
    if (!ok) {
        if (attempt < 2) {
            ++attempt;
            wsync();
            goto retry;
        }
        if (lane == 0) a.out_int[0] = kDenseBreakdown;
        return;
    }
    STAMP(2);
    // C = L^-1 G_R L^-T : solve L Y = G_R (columns), then C L^T = Y (rows)
    for (int c = lane; c < nk; c += 32) {
        for (int i = 0; i < nk; ++i) {
            double s = S.H[i * ld + c];
            for (int l = 0; l < i; ++l) s -= S.B[i * ld + l] * S.H[l * ld + c];
            S.H[i * ld + c] = s / S.B[i * ld + i];
        }
    }
    wsync();
    for (int r = lane; r < nk; r += 32) {
        for (int j = 0; j < nk; ++j) {
            double s = S.H[r * ld + j];
            for (int l = 0; l < j; ++l) s -= S.H[r * ld + l] * S.B[j * ld + l];
            S.H[r * ld + j] = s / S.B[j * ld + j];
        }
    }
    wsync();
    STAMP(3);
    // ---- 3. eigenvalues of C
    hessenberg(S.H, S.Z, nk, ld, S.v);
    STAMP(4);
    ok = francis_qr(S.H, S.Z, nk, ld);
    STAMP(5);
    if (!ok) {
        if (lane == 0) a.out_int[0] = kDenseNoConv;
        return;
    }
    // eigenvalue list from the quasi-triangular T = H
    if (lane == 0) {
        int q = 0;
        int i = 0;
        while (i < nk) {
            if (i + 1 < nk && S.H[(i + 1) * ld + i] != 0.0) {
                double aa = S.H[i * ld + i], bb = S.H[i * ld + i + 1], cc = S.H[(i + 1) * ld + i],
                       dd = S.H[(i + 1) * ld + i + 1];
                double hf = 0.5 * (aa - dd);
                double disc = hf * hf + bb * cc;
                double re = 0.5 * (aa + dd), im = sqrt(fmax(-disc, 0.0));
                // tau = re +- i im;  xi = 1/tau.  Record the member with Im(xi) > 0,
                // i.e. Im(tau) < 0, first.
                S.eig_re[q] = re; S.eig_im[q] = -im; S.eig_pos[q] = i; S.eig_blk[q] = 1; ++q;
                S.eig_re[q] = re; S.eig_im[q] = im; S.eig_pos[q] = i; S.eig_blk[q] = 1; ++q;
                i += 2;
            } else {
                S.eig_re[q] = S.H[i * ld + i]; S.eig_im[q] = 0.0; S.eig_pos[q] = i; S.eig_blk[q] = 0; ++q;
                i += 1;
            }
        }
        // ---- 4. ordering: units (real eigenvalue or conjugate pair) by (|xi|, Re xi)
        // xi = 1/tau = conj(tau) / |tau|^2
        int nu = 0;
        int unit_first[MAXM];
        double key_abs[MAXM], key_re[MAXM];
        for (int e = 0; e < nk; ++e) {
            if (S.eig_blk[e] && S.eig_im[e] > 0.0) continue;   // second member of a pair
            double re = S.eig_re[e], im = S.eig_im[e];
            double m2 = re * re + im * im;
            double xr = m2 > 0.0 ? re / m2 : INFINITY, xim = m2 > 0.0 ? -im / m2 : 0.0;
            key_abs[nu] = m2 > 0.0 ? hypot(xr, xim) : INFINITY;
            key_re[nu] = xr;
            unit_first[nu] = e;
            ++nu;
        }
        // insertion sort (stable)
        for (int i2 = 1; i2 < nu; ++i2) {
            double ka = key_abs[i2], kr = key_re[i2];
            int uf = unit_first[i2];
            int j = i2 - 1;
            while (j >= 0 && (key_abs[j] > ka || (key_abs[j] == ka && key_re[j] > kr))) {
                key_abs[j + 1] = key_abs[j]; key_re[j + 1] = key_re[j]; unit_first[j + 1] = unit_first[j];
                --j;
            }
            key_abs[j + 1] = ka; key_re[j + 1] = kr; unit_first[j + 1] = uf;
        }
        // expand to the first kp eigenvalues; record the selection
        int sel = 0;
        int nsel_units = 0;
        for (int u = 0; u < nu && sel < kp; ++u) {
            int e = unit_first[u];
            S.order[nsel_units] = e;
            S.partner[nsel_units] = S.eig_blk[e] ? ((kp - sel >= 2) ? 2 : 1) : 0;  // 0 real, 2 full pair, 1 cut pair
            sel += S.eig_blk[e] ? 2 : 1;
            ++nsel_units;
        }
        a.out_int[2] = nsel_units;
    }
    wsync();
    int nsel_units = a.out_int[2];
    __syncwarp();
    nsel_units = __shfl_sync(0xffffffffu, nsel_units, 0);
    // ---- eigenvectors of C for the selected units (z = Z x), then y = L^-T z
    // Store complex y (kept basis) into global scratch Y: [unit][nk] re, im
    double* Yre = G + 2 * m * m;
    double* Yim = Yre + MAXM * MAXM;
    double anorm = 0.0;
    for (int i = lane; i < nk * nk; i += 32) anorm = fmax(anorm, fabs(S.H[(i / nk) * ld + i % nk]));
    for (int o = 16; o > 0; o >>= 1) anorm = fmax(anorm, __shfl_xor_sync(0xffffffffu, anorm, o));
    const double smallnum = DBL_EPSILON * (anorm > 0 ? anorm : 1.0);
    STAMP(6);
    // one selected unit per lane: eigenvector x of the quasi-triangular T
    // (back substitution), z = Z x, y = L^{-T} z, normalise, rotate pairs
    for (int u = lane; u < nsel_units; u += 32) {
        int e = S.order[u];
        cplx* x = S.x + u * MAXM;
        cplx lam = {S.eig_re[e], S.eig_im[e]};
        schur_eigvec(S.H, nk, ld, S.eig_pos[e], S.eig_blk[e] != 0, lam, x, smallnum);
        double* yr = Yre + u * MAXM;
        double* yi = Yim + u * MAXM;
        for (int r = 0; r < nk; ++r) {
            double zr = 0.0, zi = 0.0;
            for (int l = 0; l < nk; ++l) {
                zr += S.Z[r * ld + l] * x[l].re;
                zi += S.Z[r * ld + l] * x[l].im;
            }
            yr[r] = zr;
            yi[r] = zi;
        }
        for (int i = nk - 1; i >= 0; --i) {
            double sr = yr[i], si = yi[i];
            for (int l = i + 1; l < nk; ++l) {
                sr -= S.B[l * ld + i] * yr[l];
                si -= S.B[l * ld + i] * yi[l];
            }
            yr[i] = sr / S.B[i * ld + i];
            yi[i] = si / S.B[i * ld + i];
        }
        double aa = 0.0, bb = 0.0, ab = 0.0;
        for (int i = 0; i < nk; ++i) {
            aa += yr[i] * yr[i]; bb += yi[i] * yi[i]; ab += yr[i] * yi[i];
        }
        double c = 1.0, sn = 0.0;
        if (S.eig_blk[e]) {
            double phi = 0.5 * atan2(-2.0 * ab, aa - bb);
            c = cos(phi); sn = sin(phi);
        }
        double nrm = sqrt(aa + bb);
        for (int i = 0; i < nk; ++i) {
            double r = yr[i], im = yi[i];
            yr[i] = (r * c - im * sn) / nrm;
            yi[i] = (r * sn + im * c) / nrm;
        }
    }
    wsync();
    STAMP(7);
    // ---- Y' = [Y0 YR yR~ YI] columns, in kept basis; tags
    // column order: real units, then full pairs' real parts, then the cut
    // column, then full pairs' imaginary parts
    double* Yp = Yim + MAXM * MAXM;  // [kp][nk]
    if (lane == 0) {
        int col = 0;
        int npair = 0;
        for (int u = 0; u < nsel_units; ++u) if (S.partner[u] == 2) ++npair;
        int nreal = 0;
        for (int u = 0; u < nsel_units; ++u) if (S.partner[u] == 0) ++nreal;
        int pr = 0;
        bool has_cut = false;
        for (int u = 0; u < nsel_units; ++u) if (S.partner[u] == 1) has_cut = true;
        for (int u = 0; u < nsel_units; ++u) {
            int kind = S.partner[u];
            if (kind == 0) {
                for (int i = 0; i < nk; ++i) Yp[col * MAXM + i] = Yre[u * MAXM + i];
                a.tags[col] = 0; a.tag_partner[col] = -1;
                ++col;
            }
        }
        int base_R = nreal, base_cut = nreal + npair, base_I = nreal + npair + (has_cut ? 1 : 0);
        for (int u = 0; u < nsel_units; ++u) {
            int kind = S.partner[u];
            if (kind == 2) {
                int cr = base_R + pr, ci = base_I + pr;
                for (int i = 0; i < nk; ++i) {
                    Yp[cr * MAXM + i] = Yre[u * MAXM + i];
                    Yp[ci * MAXM + i] = Yim[u * MAXM + i];
                }
                a.tags[cr] = 1; a.tag_partner[cr] = ci;
                a.tags[ci] = 3; a.tag_partner[ci] = cr;
                ++pr;
            } else if (kind == 1) {
                for (int i = 0; i < nk; ++i) Yp[base_cut * MAXM + i] = Yre[u * MAXM + i];
                a.tags[base_cut] = 2; a.tag_partner[base_cut] = -1;
            }
        }
        // diagnostic xi of the selected columns
        for (int u = 0; u < nsel_units; ++u) {
            int e = S.order[u];
            double re = S.eig_re[e], im = S.eig_im[e], m2 = re * re + im * im;
            a.xi[2 * u] = re / m2;
            a.xi[2 * u + 1] = -im / m2;
        }
    }
    wsync();
    // ---- 5. raw coefficients.  Z-hat = Z diag(colscale t) R^{-1}; R^{-1} is
    // upper triangular and the V columns come first, so
    //   P_new = Z-hat[:, rest] Y'_rest = Z diag(colscale t) R^{-1} [0; Y'_rest]
    //   V_new - P_new = Z-hat[:, V] Y'_V = Z_V diag(colscale t) R_VV^{-1} Y'_V
    double* Wr = Yp + MAXM * MAXM;   // [kp][nk]: R^{-1} [0; Y'_rest]
    double* Wv = Wr + MAXM * MAXM;   // [kp][nk]: R_VV^{-1} Y'_V (rows < nvk)
    for (int j = lane; j < kp; j += 32) {
        for (int i = nk - 1; i >= 0; --i) {
            double s = (i >= nvk) ? Yp[j * MAXM + i] : 0.0;
            for (int l = i + 1; l < nk; ++l) s -= S.A[i * ld + l] * Wr[j * MAXM + l];
            Wr[j * MAXM + i] = s / S.A[i * ld + i];
        }
        for (int i = nvk - 1; i >= 0; --i) {
            double s = Yp[j * MAXM + i];
            for (int l = i + 1; l < nvk; ++l) s -= S.A[i * ld + l] * Wv[j * MAXM + l];
            Wv[j * MAXM + i] = s / S.A[i * ld + i];
        }
    }
    wsync();
    for (int i = lane; i < m * kp; i += 32) a.Cp[i] = 0.0;
    for (int i = lane; i < a.nv * kp; i += 32) a.Cvv[i] = 0.0;
    wsync();
    for (int i = lane; i < nk * kp; i += 32) {
        int q = i / kp, j = i % kp;
        int raw = S.kidx[q];
        double tr = S.t[raw] * a.colscale[raw];
        a.Cp[raw * kp + j] = tr * Wr[j * MAXM + q];
        if (q < nvk) a.Cvv[raw * kp + j] = tr * Wv[j * MAXM + q];
    }
    wsync();
    STAMP(8);
    if (lane == 0) a.out_int[0] = kDenseOK;
#undef STAMP
}

}  // namespace

size_t dense_smem_bytes() { return sizeof(Smem); }

size_t dense_work_doubles() { return 2 * (size_t)MAXM * MAXM + 6 * (size_t)MAXM * MAXM; }

cudaError_t dense_extract(const DenseArgs& a, cudaStream_t s) {
    size_t shm = sizeof(Smem);
    cudaError_t e = cudaFuncSetAttribute(k_extract, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) return e;
    k_extract<<<1, 32, shm, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plhr

// ======================================================================
// Convergence status, Rayleigh quotients, final Rayleigh-Ritz.
namespace plhr {
namespace {

// relative residual ||r|| / (max(|lam|, 1) ||Bv||); order by |lam - sigma|
// (ties: smaller lam first); converged when the k nearest meet tol; a column
// is active (contributes W and S) when its residual is above tol.
__global__ void k_status(StatusArgs a) {
    if (threadIdx.x != 0) return;
    const int kp = a.kp;
    int nan = 0;
    for (int j = 0; j < kp; ++j) {
        double rn = sqrt(a.sums[j]), bn = sqrt(a.sums[kp + j]);
        double l = a.lam[j];
        double rel = rn / (fmax(fabs(l), 1.0) * bn);
        if (!isfinite(rel)) { nan = 1; rel = INFINITY; }
        a.rel[j] = rel;
        a.order[j] = j;
    }
    for (int i = 1; i < kp; ++i) {
        int o = a.order[i];
        double d = fabs(a.lam[o] - a.sigma), l = a.lam[o];
        int j = i - 1;
        while (j >= 0) {
            int p = a.order[j];
            double dp = fabs(a.lam[p] - a.sigma);
            if (dp > d || (dp == d && a.lam[p] > l)) { a.order[j + 1] = p; --j; }
            else break;
        }
        a.order[j + 1] = o;
    }
    int conv = 1;
    for (int q = 0; q < a.k; ++q)
        if (!(a.rel[a.order[q]] <= a.tol)) conv = 0;
    int na = 0;
    for (int j = 0; j < kp; ++j)
        if (!(a.rel[j] <= a.tol)) { a.lam_act[na] = a.lam[j]; a.active[na++] = j; }
    a.hstat[0] = conv;
    a.hstat[1] = na;
    a.hstat[2] = nan;
}

__global__ void k_rq(int kp, const double* dots, const int* tags, const int* partner, double* lam, double* scale) {
    if (threadIdx.x != 0) return;
    for (int j = 0; j < kp; ++j) {
        double aa = dots[j], bb = dots[kp + j];
        double l = aa / bb;
        if (tags[j] == 1 || tags[j] == 3) {
            int p = partner[j];
            l = (aa + dots[p]) / (bb + dots[kp + p]);
        }
        lam[j] = l;
        scale[j] = 1.0 / sqrt(bb);
    }
}

// one warp: Cholesky of GB, M = L^-1 GA L^-T, cyclic Jacobi (Golub & Van Loan
// Sec. 8.5), C = L^-T W, sort by |theta - sigma|.
__global__ void __launch_bounds__(32) k_rr(int n, const double* GA, const double* GB, double sigma,
                                           const double* rowscale, double* C, double* theta, int* ok_out) {
    __shared__ double L[32 * 33], M[32 * 33], W[32 * 33];
    __shared__ double th[32];
    __shared__ int ord[32];
    const int lane = threadIdx.x;
    const int ld = 33;
    for (int i = lane; i < n * n; i += 32) {
        int r = i / n, c = i % n;
        L[r * ld + c] = 0.5 * (GB[r * n + c] + GB[c * n + r]);
        M[r * ld + c] = 0.5 * (GA[r * n + c] + GA[c * n + r]);
    }
    __syncwarp();
    if (!chol_lower(L, n, ld)) {
        if (lane == 0) *ok_out = 0;
        return;
    }
    // M <- L^-1 M L^-T
    for (int c = lane; c < n; c += 32)
        for (int i = 0; i < n; ++i) {
            double s = M[i * ld + c];
            for (int l = 0; l < i; ++l) s -= L[i * ld + l] * M[l * ld + c];
            M[i * ld + c] = s / L[i * ld + i];
        }
    __syncwarp();
    for (int r = lane; r < n; r += 32)
        for (int j = 0; j < n; ++j) {
            double s = M[r * ld + j];
            for (int l = 0; l < j; ++l) s -= M[r * ld + l] * L[j * ld + l];
            M[r * ld + j] = s / L[j * ld + j];
        }
    __syncwarp();
    for (int i = lane; i < n * n; i += 32) {
        int r = i / n, c = i % n;
        if (c > r) { double s = 0.5 * (M[r * ld + c] + M[c * ld + r]); M[r * ld + c] = s; M[c * ld + r] = s; }
        W[r * ld + c] = (r == c) ? 1.0 : 0.0;
    }
    __syncwarp();
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = lane; i < n * n; i += 32) {
            int r = i / n, c = i % n;
            double v = M[r * ld + c] * M[r * ld + c];
            tot += v;
            if (r != c) off += v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = M[p * ld + q];
                if (apq == 0.0) continue;
                double app = M[p * ld + p], aqq = M[q * ld + q];
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                __syncwarp();
                // rows p, q of M
                for (int j = lane; j < n; j += 32) {
                    double mp = M[p * ld + j], mq = M[q * ld + j];
                    M[p * ld + j] = c * mp - s * mq;
                    M[q * ld + j] = s * mp + c * mq;
                }
                __syncwarp();
                for (int j = lane; j < n; j += 32) {
                    double mp = M[j * ld + p], mq = M[j * ld + q];
                    M[j * ld + p] = c * mp - s * mq;
                    M[j * ld + q] = s * mp + c * mq;
                    double wp = W[j * ld + p], wq = W[j * ld + q];
                    W[j * ld + p] = c * wp - s * wq;
                    W[j * ld + q] = s * wp + c * wq;
                }
                __syncwarp();
            }
    }
    if (lane == 0) {
        for (int j = 0; j < n; ++j) { th[j] = M[j * ld + j]; ord[j] = j; }
        for (int i = 1; i < n; ++i) {
            int o = ord[i];
            double d = fabs(th[o] - sigma), l = th[o];
            int j = i - 1;
            while (j >= 0) {
                int p = ord[j];
                double dp = fabs(th[p] - sigma);
                if (dp > d || (dp == d && th[p] > l)) { ord[j + 1] = p; --j; }
                else break;
            }
            ord[j + 1] = o;
        }
    }
    __syncwarp();
    // C = L^-T W (back substitution per column), columns reordered
    for (int jj = lane; jj < n; jj += 32) {
        int j = ord[jj];
        double x[32];
        for (int i = n - 1; i >= 0; --i) {
            double s = W[i * ld + j];
            for (int l = i + 1; l < n; ++l) s -= L[l * ld + i] * x[l];
            x[i] = s / L[i * ld + i];
        }
        for (int i = 0; i < n; ++i) C[i * n + jj] = x[i] * (rowscale ? rowscale[i] : 1.0);
        theta[jj] = th[j];
    }
    if (lane == 0) *ok_out = 1;
}

}  // namespace

cudaError_t dense_status(const StatusArgs& a, cudaStream_t s) {
    k_status<<<1, 32, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t dense_rq(int kp, const double* dots, const int* tags, const int* partner, double* lam, double* scale,
                     cudaStream_t s) {
    k_rq<<<1, 32, 0, s>>>(kp, dots, tags, partner, lam, scale);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t dense_rr(int kp, const double* GA, const double* GB, double sigma, const double* rowscale, double* C,
                     double* theta, int* ok, cudaStream_t s) {
    if (kp > 32) return cudaErrorInvalidValue;
    k_rr<<<1, 32, 0, s>>>(kp, GA, GB, sigma, rowscale, C, theta, ok);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plhr

extern "C" plhr_status plhr_tharm_extract(int m, int kp, int nv, const double* Gzz, const double* Guq,
                                          const double* Gqz, const double* colscale, double* Cp, double* Cvv,
                                          int* tags, int* partner, double* xi, int* status, long long* clk,
                                          void* stream) {
    using namespace plhr;
    clear_error();
    if (m < 1 || m > kDenseMaxM || kp < 1 || kp > 16 || kp > m || nv < 1 || nv > m || !Gzz || !Guq || !Gqz ||
        !colscale || !Cp || !Cvv || !tags || !partner || !xi || !status) {
        set_error("plhr_tharm_extract: invalid argument");
        return PLHR_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    double* work = nullptr;
    PLHR_TRY_CUDA(cudaMallocAsync(&work, sizeof(double) * dense_work_doubles(), s));
    DenseArgs a;
    a.m = m; a.kp = kp; a.nv = nv; a.Gzz = Gzz; a.Guq = Guq; a.Gqz = Gqz; a.colscale = colscale; a.work = work;
    a.Cp = Cp; a.Cvv = Cvv; a.tags = tags; a.tag_partner = partner; a.xi = xi; a.out_int = status; a.clk = clk;
    cudaError_t e = dense_extract(a, s);
    cudaFreeAsync(work, s);
    PLHR_TRY_CUDA(e);
    return PLHR_OK;
}

// ======================================================================
// Allocation-free variant of plhr_tharm_extract.
//
// Some callers cannot allocate device memory at the moment they need the
// projected eigensolve: an application that has handed the whole device to
// its own pooled allocator or arena, a service with a fixed memory budget
// that forbids allocation after start-up, or code running from a host
// callback where an allocation could block on the allocator.  For them this
// entry point takes its scratch from a fixed array compiled into the library
// instead of calling the CUDA allocator.
namespace {

// Scratch of the projected eigensolve for the largest supported basis
// (m = 64): 8 * 64 * 64 doubles = 256 KiB.  Every GPU that loads the library
// holds this array until the process exits.
constexpr size_t kNoAllocScratchDoubles = 8 * (size_t)plhr::kDenseMaxM * plhr::kDenseMaxM;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

plhr_status noalloc_scratch(double** out) {
    int dev = 0;
    PLHR_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        plhr::set_error("plhr_tharm_extract_noalloc: device ordinal %d out of range", dev);
        return PLHR_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        // host code sees only a stand-in for g_noalloc_scratch; its device
        // address comes from the runtime, with this device current
        PLHR_TRY_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return PLHR_OK;
}

}  // namespace

extern "C" plhr_status plhr_tharm_extract_noalloc(int m, int kp, int nv, const double* Gzz, const double* Guq,
                                                  const double* Gqz, const double* colscale, double* Cp,
                                                  double* Cvv, int* tags, int* partner, double* xi, int* status,
                                                  void* stream) {
    using namespace plhr;
    clear_error();
    if (m > kDenseMaxM) {
        set_error("plhr_tharm_extract_noalloc: m = %d exceeds the maximum %d of the built-in scratch", m,
                  kDenseMaxM);
        return PLHR_EINVAL;
    }
    if (m < 1 || kp < 1 || kp > 16 || kp > m || nv < 1 || nv > m || !Gzz || !Guq || !Gqz || !colscale || !Cp ||
        !Cvv || !tags || !partner || !xi || !status) {
        set_error("plhr_tharm_extract_noalloc: invalid argument");
        return PLHR_EINVAL;
    }
    if (dense_work_doubles() > kNoAllocScratchDoubles) {
        set_error("plhr_tharm_extract_noalloc: built-in scratch too small");
        return PLHR_EINVAL;
    }
    double* work = nullptr;
    PLHR_TRY(noalloc_scratch(&work));
    DenseArgs a;
    a.m = m; a.kp = kp; a.nv = nv; a.Gzz = Gzz; a.Guq = Guq; a.Gqz = Gqz; a.colscale = colscale; a.work = work;
    a.Cp = Cp; a.Cvv = Cvv; a.tags = tags; a.tag_partner = partner; a.xi = xi; a.out_int = status; a.clk = nullptr;
    PLHR_TRY_CUDA(dense_extract(a, (cudaStream_t)stream));
    return PLHR_OK;
}
