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
#include "dword.h"

#include <cfloat>
#include <mutex>

namespace plhr {
namespace {

constexpr int MAXM = kDenseMaxM;
constexpr int LDS = MAXM + 1;     // shared row stride: column accesses hit distinct banks
constexpr int NT = 128;           // threads of the extraction CTA

__device__ __forceinline__ void wsync() { __syncwarp(); }
__device__ __forceinline__ void bsync() { __syncthreads(); }

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------- warp Cholesky (final Rayleigh-Ritz)
// plain Cholesky A = L L^T by one warp (lower stored in A's lower triangle)
__device__ bool chol_lower(double* A, int n, int ld) {
    const int lane = threadIdx.x & 31;
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

// ---------------------------------------------------------------- block-wide dense kernels
// Cholesky with column dropping of a symmetric n x n (upper triangle used):
// A = R^T R on the kept columns; column j is dropped when its pivot is below
// tol (the matrix is column-normalised, so the test is relative).
__device__ int bchol_drop(double* A, int n, int* keep, double tol) {
    const int tid = threadIdx.x;
    int nk = 0;
    for (int j = 0; j < n; ++j) {
        double p = A[j * LDS + j];
        bool ok = (p > tol) && isfinite(p);
        bsync();
        if (tid == 0) keep[j] = ok ? 1 : 0;
        if (ok) {
            double r = sqrt(p);
            for (int l = j + 1 + tid; l < n; l += NT) A[j * LDS + l] /= r;
            bsync();
            if (tid == 0) A[j * LDS + j] = r;
            const int w = n - j - 1;
            for (int idx = tid; idx < w * w; idx += NT) {
                int a = j + 1 + idx / w, b = j + 1 + idx % w;
                if (b >= a) A[a * LDS + b] -= A[j * LDS + a] * A[j * LDS + b];
            }
            ++nk;
        } else {
            for (int l = tid; l < n; l += NT) A[j * LDS + l] = 0.0;
        }
        bsync();
    }
    return nk;
}

// Column (row) index of this thread in the one-column-per-thread FP64 loops:
// 16 lanes of each of the four warps, one warp per SM sub-partition, so that
// all four FP64 pipes work (a warp instruction occupies the pipe for the same
// time whatever its active lanes).  Lanes 16..31 take the same index of a
// second matrix (spread_second).  Every index is handled by one thread, in
// the same order as with one thread per index.
static_assert(NT == 128 && MAXM <= 64, "four warps of 16 lanes cover the columns");
__device__ __forceinline__ int spread_index() { return (threadIdx.x >> 5) * 16 + (threadIdx.x & 15); }
__device__ __forceinline__ bool spread_second() { return (threadIdx.x & 16) != 0; }

// X1 <- R^{-T} X1 R^{-1} and X2 <- R^{-T} X2 R^{-1} (X2 optional) for upper
// triangular R (all n x n, stride LDS)
__device__ void bcongruence2(const double* R, double* X1, double* X2, int n) {
    const int c = spread_index();
    double* X = spread_second() ? X2 : X1;
    if (X != nullptr && c < n) {
        for (int i = 0; i < n; ++i) {
            double s = X[i * LDS + c];
            for (int l = 0; l < i; ++l) s -= R[l * LDS + i] * X[l * LDS + c];
            X[i * LDS + c] = s / R[i * LDS + i];
        }
    }
    bsync();
    if (X != nullptr && c < n) {
        const int r = c;
        for (int j = 0; j < n; ++j) {
            double s = X[r * LDS + j];
            for (int l = 0; l < j; ++l) s -= X[r * LDS + l] * R[l * LDS + j];
            X[r * LDS + j] = s / R[j * LDS + j];
        }
    }
    bsync();
}

// A = L L^T (lower triangle), block-wide; false when not positive definite
__device__ bool bchol_lower(double* A, int n, int* flag) {
    const int tid = threadIdx.x;
    for (int j = 0; j < n; ++j) {
        double p = A[j * LDS + j];
        bool ok = (p > 0.0) && isfinite(p);
        if (!ok) { bsync(); return false; }
        double r = sqrt(p);
        bsync();
        for (int l = j + 1 + tid; l < n; l += NT) A[l * LDS + j] /= r;
        bsync();
        if (tid == 0) A[j * LDS + j] = r;
        const int w = n - j - 1;
        for (int idx = tid; idx < w * w; idx += NT) {
            int a = j + 1 + idx / w, b = j + 1 + idx % w;
            if (b <= a) A[a * LDS + b] -= A[a * LDS + j] * A[b * LDS + j];
        }
        bsync();
    }
    (void)flag;
    return true;
}

// Householder reduction of H (n x n) to upper Hessenberg form.  The reflector
// of step k, I - beta_k v v^T with v = (0,..,0, v_{k+1}, .., v_{n-1}), is kept
// in row k of Vh and beta[k] (beta = 0: identity).
//
// The reduction runs in double-word arithmetic on H scaled by a power of two
// to unit norm: its transformations are orthogonal, so it is as accurate as
// the double-word QR iteration that follows it, and the FP64 form (one
// dependent FP64 chain per column, each warp instruction holding the FP64 pipe
// for 64 cycles) cost about a million cycles at n = 64.  Every column and row
// belongs to a pair of threads that split its sum over i by parity (lazily
// normalised double-word sums, combined by one shuffle).  v and beta describe
// the same reflector at any scale, so only H is scaled back; H, Vh and beta
// are FP64 again on return.
__device__ void bhessenberg(double* Hd, double* Vhd, double* betad, int n, double* red) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const dw zero = dw_make(0.0f);
    double an = 0.0;
    for (int i = tid; i < n * n; i += NT) an = fmax(an, fabs(Hd[(i / n) * LDS + i % n]));
    an = warp_max(an);
    if (lane == 0) red[warp] = an;
    bsync();
    for (int w = 0; w < NT / 32; ++w) an = fmax(an, red[w]);
    bsync();
    const int ex = an > 0.0 ? ilogb(an) : 0;
    const double down = ldexp(1.0, -ex), up = ldexp(1.0, ex);
    dw* H = reinterpret_cast<dw*>(Hd);
    dw* V = reinterpret_cast<dw*>(Vhd);
    dw* B = reinterpret_cast<dw*>(betad);
    for (int i = tid; i < n * n; i += NT) {
        const int r = i / n, c = i % n;
        H[r * LDS + c] = dw_from_double_fast(Hd[r * LDS + c] * down);
    }
    bsync();
    float* redf = reinterpret_cast<float*>(red);
    const int own = tid >> 1, half = tid & 1;
    for (int k = 0; k < n - 2; ++k) {
        // ||x||^2 for x = H[k+1:n, k]  (warp 0)
        if (warp == 0) {
            dwacc acc = {0.0f, 0.0f};
            for (int i = k + 1 + lane; i < n; i += 32) {
                const dw x = H[i * LDS + k];
                dwacc_add_mul(acc, x, x);
            }
            dw ss = dwacc_result(acc);
            for (int o = 16; o > 0; o >>= 1)
                ss = dw_add(ss, dw{__shfl_xor_sync(0xffffffffu, ss.hi, o), __shfl_xor_sync(0xffffffffu, ss.lo, o)});
            if (lane == 0) { redf[0] = ss.hi; redf[1] = ss.lo; }
        }
        bsync();
        const dw ss = {redf[0], redf[1]};
        const dw x0 = H[(k + 1) * LDS + k];
        dw alpha = dw_sqrt(ss);
        if (x0.hi > 0.0f) alpha = dw_neg(alpha);
        // v_{k+1} = x0 - alpha, v^T v = 2 (ss - x0 alpha) (alpha^2 = ss, no
        // cancellation: -x0 alpha >= 0), beta = 2 / v^T v
        const dw den = dw_sub(ss, dw_mul(x0, alpha));
        const bool skip = dw_is_zero(alpha) || !(den.hi > 0.0f);
        const dw b = skip ? zero : dw_div(dw_make(1.0f), den);
        for (int i = tid; i < n; i += NT)
            V[k * LDS + i] = (i <= k || skip) ? zero : (i == k + 1 ? dw_sub(x0, alpha) : H[i * LDS + k]);
        if (tid == 0) B[k] = b;
        bsync();
        if (!skip) {
            const dw* v = V + k * LDS;
            // H <- (I - b v v^T) H : column c = own (columns below k are zero in rows > k)
            {
                const int c = own;
                const bool act = c < n && c >= k;
                dwacc acc = {0.0f, 0.0f};
                if (act)
                    for (int i = k + 1 + half; i < n; i += 2) dwacc_add_mul(acc, v[i], H[i * LDS + c]);
                dw sv = dwacc_result(acc);
                sv = dw_add(sv, dw{__shfl_xor_sync(0xffffffffu, sv.hi, 1), __shfl_xor_sync(0xffffffffu, sv.lo, 1)});
                sv = dw_mul(sv, b);
                if (act)
                    for (int i = k + 1 + half; i < n; i += 2) H[i * LDS + c] = dw_sub(H[i * LDS + c], dw_mul(sv, v[i]));
            }
            bsync();
            // H <- H (I - b v v^T) : row r = own
            {
                const int r = own;
                const bool act = r < n;
                dwacc acc = {0.0f, 0.0f};
                if (act)
                    for (int i = k + 1 + half; i < n; i += 2) dwacc_add_mul(acc, H[r * LDS + i], v[i]);
                dw sv = dwacc_result(acc);
                sv = dw_add(sv, dw{__shfl_xor_sync(0xffffffffu, sv.hi, 1), __shfl_xor_sync(0xffffffffu, sv.lo, 1)});
                sv = dw_mul(sv, b);
                if (act)
                    for (int i = k + 1 + half; i < n; i += 2) H[r * LDS + i] = dw_sub(H[r * LDS + i], dw_mul(sv, v[i]));
            }
            bsync();
            for (int i = k + 2 + tid; i < n; i += NT) H[i * LDS + k] = zero;
        }
        bsync();
    }
    // back to FP64 (each entry converted in place by the thread that reads it)
    for (int i = tid; i < n * n; i += NT) {
        const int r = i / n, c = i % n;
        Hd[r * LDS + c] = dw_to_double(H[r * LDS + c]) * up;
    }
    for (int i = tid; i < (n - 2) * n; i += NT) {
        const int r = i / n, c = i % n;
        Vhd[r * LDS + c] = dw_to_double(V[r * LDS + c]);
    }
    for (int i = tid; i < n - 2; i += NT) betad[i] = dw_to_double(B[i]);
    bsync();
}

// ---------------------------------------------------------------- eigenvalues (one warp)
// Householder vector for (x, y[, z]) in double-word arithmetic: u = (1, u1, u2)
// and tau with (I - tau u u^T)(x, y, z)^T = (beta, 0, 0)^T.
__device__ __forceinline__ void house3(dw x, dw y, dw z, int nr, dw& u1, dw& u2, dw& tau) {
    const dw zero = dw_make(0.0f);
    if (dw_is_zero(y) && (nr == 2 || dw_is_zero(z))) {
        u1 = zero; u2 = zero; tau = zero;
        return;
    }
    // u and tau do not depend on the scale of (x, y, z): bring the largest to
    // about 1 by a power of two (exact) so that the squares stay inside FP32's
    // exponent range
    {
        const float mx = fmaxf(fabsf(x.hi), fmaxf(fabsf(y.hi), nr == 3 ? fabsf(z.hi) : 0.0f));
        const float sc = pow2_inverse_of(mx);
        x = dw_mul_pow2(x, sc);
        y = dw_mul_pow2(y, sc);
        z = dw_mul_pow2(z, sc);
    }
    dw ss = dw_add(dw_mul(x, x), dw_mul(y, y));
    if (nr == 3) ss = dw_add(ss, dw_mul(z, z));
    dw nrm = dw_sqrt(ss);
    if (dw_is_zero(nrm)) {
        u1 = zero; u2 = zero; tau = zero;
        return;
    }
    dw beta = x.hi > 0.0f ? dw_neg(nrm) : nrm;
    dw v0 = dw_sub(x, beta);
    dw rv = dw_div(dw_make(1.0f), v0);
    u1 = dw_mul(y, rv);
    u2 = nr == 3 ? dw_mul(z, rv) : zero;
    tau = dw_div(dw_neg(v0), beta);   // (beta - x) / beta
}

// Francis double-shift QR (Golub & Van Loan Sec. 7.5) on the upper Hessenberg
// H, eigenvalues only: every transformation is applied to the active window
// rows/columns l..hi alone (no Schur vectors, no full Schur form), which is
// all the eigenvalues need.  Deflated 1x1 and 2x2 diagonal blocks remain.
// kFrancisThreads threads (two warps, on two sub-partitions): in a bulge step
// each thread updates one column (left reflection) and then one row (right
// reflection), so a step costs one short double-word chain per side instead of
// two per lane in one warp; the reflector itself is formed redundantly by
// every thread.  The iteration runs in double-word arithmetic on H scaled by a
// power of two to unit norm (H is converted in place: a double and a
// double-word value take the same 8 bytes) and is converted back at the end.
// Every entry is updated by the same operations in the same order as with
// one warp, so the result does not depend on the thread count.  Returns false
// if the iteration does not converge; sweeps (optional) gets the number of QR
// sweeps and of bulge steps.
constexpr int kFrancisThreads = 64;
static_assert(kFrancisThreads >= MAXM, "one column / row per thread");

__device__ __noinline__ bool francis_eigenvalues(double* Hd, int n, long long* sweeps) {
    __shared__ double red[kFrancisThreads / 32];
    const int t = threadIdx.x;
    double anorm = 0.0;
    for (int i = t; i < n * n; i += kFrancisThreads) {
        int r = i / n, c = i % n;
        if (c >= r - 1) anorm = fmax(anorm, fabs(Hd[r * LDS + c]));
    }
    anorm = warp_max(anorm);
    if ((t & 31) == 0) red[t >> 5] = anorm;
    __syncthreads();
    for (int w = 0; w < kFrancisThreads / 32; ++w) anorm = fmax(anorm, red[w]);
    const int ex = anorm > 0.0 ? ilogb(anorm) : 0;
    const double down = ldexp(1.0, -ex), up = ldexp(1.0, ex);
    dw* H = reinterpret_cast<dw*>(Hd);
    for (int i = t; i < n * n; i += kFrancisThreads) {
        int r = i / n, c = i % n;
        double v = (c >= r - 1) ? Hd[r * LDS + c] * down : 0.0;
        H[r * LDS + c] = dw_from_double(v);
    }
    __syncthreads();
    // negligible subdiagonal: relative to the neighbouring diagonal, or to
    // ||H|| (= 1 to 2 after scaling; normwise backward stable).  Only the
    // eigenvalues of largest modulus are used, and they keep full relative
    // accuracy; the normwise test lets the many eigenvalues near zero deflate
    // quickly.  eps is a few units of the double-word precision.
    const float eps = 0x1p-46f;
    const float hnorm = 1.0f;
    const dw zero = dw_make(0.0f);
    bool ok = true;
    int hi = n - 1;
    int its = 0, total_its = 0, total_steps = 0;
    while (hi >= 0) {
        int l = hi;
        while (l > 0) {
            float s = fabsf(H[(l - 1) * LDS + l - 1].hi) + fabsf(H[l * LDS + l].hi);
            if (s < hnorm) s = hnorm;
            if (fabsf(H[l * LDS + l - 1].hi) <= eps * s) break;
            --l;
        }
        __syncthreads();
        if (l > 0 && t == 0) H[l * LDS + l - 1] = zero;
        __syncthreads();
        if (l >= hi - 1) {          // 1x1 or 2x2 block converged
            hi = l - 1;
            its = 0;
            continue;
        }
        if (its >= 40) {
            // a stalled window holds a (near-)defective cluster of numerically
            // equal eigenvalues, which converges only linearly; deflate at the
            // smallest subdiagonal when it is below 1e-7 ||H|| (the eigenvalues
            // move by about that much; only a basis of the cluster is needed)
            int jm = l + 1;
            float vm = fabsf(H[(l + 1) * LDS + l].hi);
            for (int j = l + 2; j <= hi; ++j) {
                float v = fabsf(H[j * LDS + j - 1].hi);
                if (v < vm) { vm = v; jm = j; }
            }
            if (vm <= 1e-7f * hnorm) {
                __syncthreads();
                if (t == 0) H[jm * LDS + jm - 1] = zero;
                __syncthreads();
                its = 0;
                continue;
            }
        }
        if (++total_its > 100 * n) { ok = false; break; }
        ++its;
        total_steps += hi - l;
        dw s, tt;
        if (its % 10 == 0) {
            dw w = dw_add(dw_make(fabsf(H[hi * LDS + hi - 1].hi)), dw_make(fabsf(H[(hi - 1) * LDS + hi - 2].hi)));
            s = dw_mul_f(w, 1.5f);
            tt = dw_mul(w, w);
        } else {
            dw a = H[(hi - 1) * LDS + hi - 1], b = H[(hi - 1) * LDS + hi], c = H[hi * LDS + hi - 1],
               d = H[hi * LDS + hi];
            s = dw_add(a, d);
            tt = dw_sub(dw_mul(a, d), dw_mul(b, c));
        }
        dw h00 = H[l * LDS + l], h01 = H[l * LDS + l + 1], h10 = H[(l + 1) * LDS + l],
           h11 = H[(l + 1) * LDS + l + 1], h21 = H[(l + 2) * LDS + l + 1];
        // first column of (H - s1 I)(H - s2 I)
        dw x = dw_add(dw_add(dw_mul(h00, dw_sub(h00, s)), dw_mul(h01, h10)), tt);
        dw y = dw_mul(h10, dw_sub(dw_add(h00, h11), s));
        dw z = dw_mul(h10, h21);
        // every thread has read the shift and the first bulge column before
        // any thread writes
        __syncthreads();
        for (int k = l; k <= hi - 1; ++k) {
            const int nr = (k < hi - 1) ? 3 : 2;
            dw u1, u2, tau;
            house3(x, y, z, nr, u1, u2, tau);
            if (!dw_is_zero(tau)) {
                // left: rows k..k+2, column c0 + t
                const int c0 = k > l ? k - 1 : l;
                {
                    const int ca = c0 + t;
                    if (ca <= hi) {
                        const dw a0 = H[k * LDS + ca], a1 = H[(k + 1) * LDS + ca];
                        const dw a2 = nr == 3 ? H[(k + 2) * LDS + ca] : zero;
                        const dw sa = dw_mul(dw_add(dw_add(a0, dw_mul(u1, a1)), dw_mul(u2, a2)), tau);
                        H[k * LDS + ca] = dw_sub(a0, sa);
                        H[(k + 1) * LDS + ca] = dw_sub(a1, dw_mul(sa, u1));
                        if (nr == 3) H[(k + 2) * LDS + ca] = dw_sub(a2, dw_mul(sa, u2));
                    }
                }
                __syncthreads();
                // right: columns k..k+2, row l + t (rows l..min(k+3, hi))
                const int r1 = (k + 3 < hi) ? k + 3 : hi;
                {
                    const int ra = l + t;
                    if (ra <= r1) {
                        const dw a0 = H[ra * LDS + k], a1 = H[ra * LDS + k + 1];
                        const dw a2 = nr == 3 ? H[ra * LDS + k + 2] : zero;
                        const dw sa = dw_mul(dw_add(dw_add(a0, dw_mul(u1, a1)), dw_mul(u2, a2)), tau);
                        H[ra * LDS + k] = dw_sub(a0, sa);
                        H[ra * LDS + k + 1] = dw_sub(a1, dw_mul(sa, u1));
                        if (nr == 3) H[ra * LDS + k + 2] = dw_sub(a2, dw_mul(sa, u2));
                    }
                }
                __syncthreads();
            }
            if (k > l && t == 0) {
                H[(k + 1) * LDS + k - 1] = zero;
                if (nr == 3) H[(k + 2) * LDS + k - 1] = zero;
            }
            __syncthreads();
            if (k < hi - 1) {
                x = H[(k + 1) * LDS + k];
                y = H[(k + 2) * LDS + k];
                z = (k < hi - 2) ? H[(k + 3) * LDS + k] : zero;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    for (int i = t; i < n * n; i += kFrancisThreads) {
        int r = i / n, c = i % n;
        dw v = H[r * LDS + c];
        Hd[r * LDS + c] = (c >= r - 1) ? dw_to_double(v) * up : 0.0;
    }
    if (sweeps && t == 0) { sweeps[0] = total_its; sweeps[1] = total_steps; }
    __syncthreads();
    return ok;
}

// ---------------------------------------------------------------- eigenvectors (one warp each)
// Complex double-word arithmetic for the per-unit eigenvector work: each
// step of a triangular factorisation or solve is a short serial chain, and
// on GB300 an FP64 warp instruction holds the FP64 pipe for 64 cycles, so
// the chains run several times faster on the FP32 pipes in double-word form
// (~48-bit significands, the accuracy of the QR iteration that supplies the
// shifts).  The operands are scaled by a power of two to unit norm first so
// that they stay inside FP32's exponent range.
struct cdw {
    dw re, im;
};
__device__ __forceinline__ cdw cdw_mul(cdw a, cdw b) {
    return {dw_sub(dw_mul(a.re, b.re), dw_mul(a.im, b.im)), dw_add(dw_mul(a.re, b.im), dw_mul(a.im, b.re))};
}
__device__ __forceinline__ cdw cdw_sub(cdw a, cdw b) { return {dw_sub(a.re, b.re), dw_sub(a.im, b.im)}; }
__device__ __forceinline__ float cdw_abs1(cdw a) { return fabsf(a.re.hi) + fabsf(a.im.hi); }
// 1 / b, the denominator scaled by a power of two first (no under- or overflow)
__device__ __forceinline__ cdw cdw_recip(cdw b) {
    const float sc = pow2_inverse_of(fmaxf(fabsf(b.re.hi), fabsf(b.im.hi)));
    const dw r = dw_mul_pow2(b.re, sc), i = dw_mul_pow2(b.im, sc);
    const dw den = dw_add(dw_mul(r, r), dw_mul(i, i));
    const dw inv = dw_div(dw_make(1.0f), den);
    return {dw_mul_pow2(dw_mul(r, inv), sc), dw_mul_pow2(dw_neg(dw_mul(i, inv)), sc)};
}

// Inverse iteration on the Hessenberg H0 (FP64, scaled here by `down`, a power
// of two) for the eigenvalue lam (same scale): (H0 - lam I) is factored once
// by Gaussian elimination with adjacent-row pivoting (keeps the Hessenberg
// structure; multipliers, swaps, the packed upper factor U and the
// reciprocals of its pivots kept), then two solves starting from b = 1, each
// normalised to max |x_i| = 1.  Column-oriented back substitution: one
// reciprocal multiply on the critical path per step, the updates in parallel.

__device__ void inverse_iteration_dw(const double* H0, int n, double down, cdw lam, cdw* x, cdw* U, cdw* mult,
                                     cdw* rpiv, int* swp, cdw* cur, cdw* nxt, float tiny) {
    const int lane = threadIdx.x & 31;
    const cdw zero = {dw_make(0.0f), dw_make(0.0f)};
    auto hs = [&](int r, int c) -> cdw {
        dw v = dw_from_double(H0[r * LDS + c] * down);
        cdw e = {v, dw_make(0.0f)};
        if (r == c) e = cdw_sub(e, lam);
        return e;
    };
    for (int j = lane; j < n; j += 32) cur[j] = hs(0, j);
    wsync();
    for (int k = 0; k < n - 1; ++k) {
        for (int j = k + lane; j < n; j += 32) nxt[j] = (j >= k) ? hs(k + 1, j) : zero;
        wsync();
        const bool swap = cdw_abs1(nxt[k]) > cdw_abs1(cur[k]);
        wsync();
        if (swap) {
            for (int j = k + lane; j < n; j += 32) { const cdw t2 = cur[j]; cur[j] = nxt[j]; nxt[j] = t2; }
        }
        wsync();
        cdw piv = cur[k];
        if (cdw_abs1(piv) < tiny) piv = {dw_make(tiny), dw_make(0.0f)};
        const cdw rp = cdw_recip(piv);
        const cdw f = cdw_mul(nxt[k], rp);
        cdw* urow = U + (k * n - (k * (k - 1)) / 2);   // row k holds columns k..n-1
        for (int j = k + lane; j < n; j += 32) {
            urow[j - k] = (j == k) ? piv : cur[j];
            if (j > k) nxt[j] = cdw_sub(nxt[j], cdw_mul(f, cur[j]));
        }
        if (lane == 0) { mult[k] = f; rpiv[k] = rp; swp[k] = swap ? 1 : 0; }
        wsync();
        for (int j = k + 1 + lane; j < n; j += 32) cur[j] = nxt[j];
        wsync();
    }
    {
        cdw piv = cur[n - 1];
        if (cdw_abs1(piv) < tiny) piv = {dw_make(tiny), dw_make(0.0f)};
        if (lane == 0) {
            U[(n - 1) * n - ((n - 1) * (n - 2)) / 2] = piv;
            rpiv[n - 1] = cdw_recip(piv);
        }
    }
    for (int i = lane; i < n; i += 32) x[i] = {dw_make(1.0f), dw_make(0.0f)};
    wsync();
    for (int iter = 0; iter < 2; ++iter) {
        // forward: the recorded row swaps and eliminations applied to b = x
        if (lane == 0) {
            for (int k = 0; k < n - 1; ++k) {
                if (swp[k]) { const cdw t2 = x[k]; x[k] = x[k + 1]; x[k + 1] = t2; }
                x[k + 1] = cdw_sub(x[k + 1], cdw_mul(mult[k], x[k]));
            }
        }
        wsync();
        // backward: x_i = b_i / U_ii, then b_j -= U_ji x_i for j < i
        for (int i = n - 1; i >= 0; --i) {
            const cdw xi_ = cdw_mul(x[i], rpiv[i]);
            wsync();
            for (int j = lane; j < i; j += 32) {
                const cdw u = U[j * n - (j * (j - 1)) / 2 + (i - j)];
                x[j] = cdw_sub(x[j], cdw_mul(u, xi_));
            }
            if (lane == 0) x[i] = xi_;
            wsync();
        }
        // normalise to max |x_i| = 1 (scale by a power of two, then exactly)
        float mx = 0.0f;
        for (int j = lane; j < n; j += 32) mx = fmaxf(mx, cdw_abs1(x[j]));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float sc = (mx > 0.0f && isfinite(mx)) ? pow2_inverse_of(mx) : 1.0f;
        for (int j = lane; j < n; j += 32) x[j] = {dw_mul_pow2(x[j].re, sc), dw_mul_pow2(x[j].im, sc)};
        wsync();
    }
}

__device__ __forceinline__ dw warp_sum_dw(dw v) {
    for (int o = 16; o > 0; o >>= 1) {
        const dw t = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = dw_add(v, t);
    }
    return v;
}

// ---------------------------------------------------------------- the kernel
struct Smem {
    double H[MAXM * LDS];     // C, then its Hessenberg form, then the quasi-triangular result
    double H0[MAXM * LDS];    // Hessenberg form of C (kept for inverse iteration)
    double Vh[MAXM * LDS];    // Householder vectors of the Hessenberg reduction
    double A[MAXM * LDS];     // column-normalised B-Gram -> R
    double B[MAXM * LDS];     // G_L -> L
    double beta[MAXM];
    double t[MAXM];           // column normalisation of the (scaled) basis
    double red[NT];
    int keep[MAXM];
    int kidx[MAXM];           // kept -> raw index
    double eig_re[MAXM], eig_im[MAXM];
    int order[MAXM];          // selected units: eigenvalue index
    int kind[MAXM];           // 0 real, 2 full pair, 1 cut pair
    int nclose[MAXM];         // earlier selected units in the same numerical cluster
    int ints[8];
};

// words of the shared-memory state saved to global memory between the launches
constexpr int kStateWords = (int)(sizeof(Smem) / sizeof(int));
static_assert(sizeof(Smem) % sizeof(int) == 0, "state copy granularity");
// Yre, Yim, Yp (MAXM^2 each), then the saved state; a selected unit (at most
// MAXKP) keeps its packed complex LU factor (MAXM (MAXM+1) / 2) in shared memory
constexpr int MAXKP = 16;
constexpr size_t kLuComplex = (size_t)MAXM * (MAXM + 1) / 2;
constexpr size_t kWorkMainDoubles = 3 * (size_t)MAXM * MAXM;
constexpr size_t kDenseWorkDoubles = kWorkMainDoubles + (sizeof(Smem) + sizeof(double) - 1) / sizeof(double);

__device__ __forceinline__ Smem* state_of(const DenseArgs& a) {
    return reinterpret_cast<Smem*>(a.work + kWorkMainDoubles);
}

// X <- L^{-1} X L^{-T} for the n x n block X (stride LDS, FP64 in and out)
// and the lower triangular L (FP64), in double-word arithmetic; Lw (n x LDS
// double-word) and rinv (n double-word values) are scratch.  Block-wide.
__device__ void dense_csolve_dw(double* Xd, const double* L, double* Lwd, double* rinvd, int n) {
    const int tid = threadIdx.x, lane = tid & 31;
    dw* X = reinterpret_cast<dw*>(Xd);
    dw* Lw = reinterpret_cast<dw*>(Lwd);
    dw* rinv = reinterpret_cast<dw*>(rinvd);
    for (int i = tid; i < n * n; i += NT) {
        const int r = i / n, c = i % n;
        X[r * LDS + c] = dw_from_double_fast(Xd[r * LDS + c]);
        if (c <= r) Lw[r * LDS + c] = dw_from_double_fast(L[r * LDS + c]);
    }
    bsync();
    for (int i = tid; i < n; i += NT) rinv[i] = dw_div(dw_make(1.0f), Lw[i * LDS + i]);
    bsync();
    const int own = tid >> 1, half = tid & 1;
    const bool act = own < n;
    // columns: X[i][c] = (X[i][c] - sum_{l<i} L[i][l] X[l][c]) / L[i][i]
    for (int i = 0; i < n; ++i) {
        dwacc acc = {0.0f, 0.0f};
        if (act)
            for (int l = half; l < i; l += 2) dwacc_add_mul(acc, Lw[i * LDS + l], X[l * LDS + own]);
        dw sv = dwacc_result(acc);
        sv = dw_add(sv, dw{__shfl_xor_sync(0xffffffffu, sv.hi, 1), __shfl_xor_sync(0xffffffffu, sv.lo, 1)});
        if (act && half == 0) X[i * LDS + own] = dw_mul(dw_sub(X[i * LDS + own], sv), rinv[i]);
        __syncwarp();
    }
    bsync();
    // rows: X[r][j] = (X[r][j] - sum_{l<j} X[r][l] L[j][l]) / L[j][j]
    for (int j = 0; j < n; ++j) {
        dwacc acc = {0.0f, 0.0f};
        if (act)
            for (int l = half; l < j; l += 2) dwacc_add_mul(acc, X[own * LDS + l], Lw[j * LDS + l]);
        dw sv = dwacc_result(acc);
        sv = dw_add(sv, dw{__shfl_xor_sync(0xffffffffu, sv.hi, 1), __shfl_xor_sync(0xffffffffu, sv.lo, 1)});
        if (act && half == 0) X[own * LDS + j] = dw_mul(dw_sub(X[own * LDS + j], sv), rinv[j]);
        __syncwarp();
    }
    bsync();
    for (int i = tid; i < n * n; i += NT) {
        const int r = i / n, c = i % n;
        Xd[r * LDS + c] = dw_to_double(X[r * LDS + c]);
    }
    (void)lane;
}

// The dense stage runs as five launches: phase 0 of k_extract (up to the
// Hessenberg form, state saved to global scratch), k_francis (two warps: the
// eigenvalues), phase 1 (selection, state saved), k_eigvec (one CTA per
// selected unit, in parallel), phase 2 (orthogonalisation, Y', coefficients).
// The eigenvalue iteration measured 2x slower per bulge step when run inside
// the large kernel than as its own launch on the same data and code, and the
// eigenvectors ran four rounds on four warps of one SM.
__global__ void __launch_bounds__(NT) k_extract(DenseArgs a, int phase) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = a.m, kp = a.kp;
    int* gst = reinterpret_cast<int*>(state_of(a));
    int* sst = reinterpret_cast<int*>(&S);
    int nk = 0, nvk = 0;
    // global scratch: complex eigenvector coefficients per selected unit and Y'
    double* Yre = a.work;                          // [unit][MAXM]
    double* Yim = Yre + MAXM * MAXM;               // [unit][MAXM]
    double* Yp = Yim + MAXM * MAXM;                // [col][MAXM]
    double* Wr = Yre;                              // reused after Y' is assembled
    double* Wv = Yim;
#define STAMP(i) do { if (a.clk && tid == 0) a.clk[i] = clock64(); } while (0)
  if (phase == 0) {
    STAMP(0);
    // ---- 1. B-orthonormalisation of Z, implicitly: Cholesky with column
    // dropping of the column-normalised Gram (the Grams are of Z diag(colscale)).
    // The basis Z D R^{-1} amplifies Gram rounding by cond(R)^2; if G_L then is
    // not numerically positive definite the pass is repeated with a stricter
    // drop threshold.
    for (int i = tid; i < m; i += NT) {
        double g = a.Gzz[i * m + i];
        S.t[i] = (g > 0.0 && isfinite(g)) ? 1.0 / sqrt(g) : 0.0;
    }
    bsync();
    const double drop_tols[3] = {1e-12, 1e-9, 1e-6};
    bool ok = false;
    for (int attempt = 0; attempt < 3 && !ok; ++attempt) {
        for (int i = tid; i < m * m; i += NT) {
            int r = i / m, c = i % m;
            S.A[r * LDS + c] = a.Gzz[i] * S.t[r] * S.t[c];
        }
        bsync();
        bchol_drop(S.A, m, S.keep, drop_tols[attempt]);
        STAMP(11);
        if (tid == 0) {
            int q = 0, qv = 0;
            for (int j = 0; j < m; ++j)
                if (S.keep[j] && S.t[j] != 0.0) {
                    S.kidx[q++] = j;
                    if (j < a.nv) ++qv;
                }
            S.ints[0] = q;
            S.ints[1] = qv;
        }
        bsync();
        nk = S.ints[0];
        nvk = S.ints[1];
        if (nvk < 1 || nk < kp) break;
        // compact R (upper) in place through H
        for (int i = tid; i < nk * nk; i += NT) {
            int r = i / nk, c = i % nk;
            S.H[r * LDS + c] = (c >= r) ? S.A[S.kidx[r] * LDS + S.kidx[c]] : 0.0;
        }
        bsync();
        for (int i = tid; i < nk * nk; i += NT) S.A[(i / nk) * LDS + i % nk] = S.H[(i / nk) * LDS + i % nk];
        bsync();
        // G_L = sym(U^T Q), G_R[r][c] = q_r . z_c, on the kept, normalised columns
        for (int i = tid; i < nk * nk; i += NT) {
            int r = i / nk, c = i % nk;
            int rr = S.kidx[r], cc = S.kidx[c];
            S.B[r * LDS + c] = 0.5 * (a.Guq[rr * m + cc] + a.Guq[cc * m + rr]) * S.t[rr] * S.t[cc];
            S.H[r * LDS + c] = a.Gqz[rr * m + cc] * S.t[rr] * S.t[cc];
        }
        bsync();
        // ---- 2. the pencil in the B-orthonormal basis, via tau = 1/xi
        STAMP(12);
        bcongruence2(S.A, S.B, S.H, nk);
        STAMP(13);
        for (int i = tid; i < nk * nk; i += NT) {
            int r = i / nk, c = i % nk;
            if (c > r) {
                double sv = 0.5 * (S.B[r * LDS + c] + S.B[c * LDS + r]);
                S.B[r * LDS + c] = sv;
                S.B[c * LDS + r] = sv;
            }
        }
        bsync();
        ok = bchol_lower(S.B, nk, nullptr);
    }
    STAMP(1);
    if (nvk < 1 || nk < kp) {
        if (tid == 0) { a.out_int[0] = kDenseRankLoss; a.out_int[1] = nk; a.out_int[2] = 0; state_of(a)->ints[6] = 1; }
        return;
    }
    if (!ok) {
        if (tid == 0) { a.out_int[0] = kDenseBreakdown; a.out_int[1] = nk; a.out_int[2] = 0; state_of(a)->ints[6] = 1; }
        return;
    }
    // C = L^{-1} G_R L^{-T}: L Y = G_R by columns, then C L^T = Y by rows, in
    // double-word arithmetic (L is the Cholesky factor of the SPD G_L in the
    // B-orthonormal basis; its condition is the square root of G_L's, so the
    // solves lose little; in FP64 each dependent chain held a warp's FP64 pipe
    // for 64 cycles per step).  A pair of threads owns a column (then a row)
    // and splits each inner sum by parity; L (double-word) goes into the
    // H0 array, free until the Hessenberg form is copied there, the
    // reciprocals of its diagonal into red.
    dense_csolve_dw(S.H, S.B, S.H0, S.red, nk);
    bsync();
    STAMP(2);
    // ---- 3. eigenvalues of C: Hessenberg form, then Francis QR on a copy
    bhessenberg(S.H, S.Vh, S.beta, nk, S.red);
    STAMP(14);
    for (int i = tid; i < nk * LDS; i += NT) S.H0[i] = S.H[i];
    if (tid == 0) S.ints[6] = 0;
    bsync();
    for (int i = tid; i < kStateWords; i += NT) gst[i] = sst[i];
    return;
  }
    // ---- phases 1, 2: reload the state (the eigenvalues are in S.H, S.ints[2])
    for (int i = tid; i < kStateWords; i += NT) sst[i] = gst[i];
    bsync();
    if (S.ints[6]) return;            // an earlier phase stopped (status already written)
    nk = S.ints[0];
    nvk = S.ints[1];
  if (phase == 1) {
    if (!S.ints[2]) {
        if (tid == 0) { a.out_int[0] = kDenseNoConv; a.out_int[1] = nk; a.out_int[2] = 0; state_of(a)->ints[6] = 1; }
        return;
    }
    // ---- 4. order by |xi| (xi = 1/tau), conjugate pairs adjacent, select k'
    if (tid == 0) {
        int q = 0, i = 0;
        while (i < nk) {
            if (i + 1 < nk && S.H[(i + 1) * LDS + i] != 0.0) {
                double aa = S.H[i * LDS + i], bb = S.H[i * LDS + i + 1], cc = S.H[(i + 1) * LDS + i],
                       dd = S.H[(i + 1) * LDS + i + 1];
                double hf = 0.5 * (aa - dd), disc = hf * hf + bb * cc;
                if (disc >= 0.0) {   // deflated block with two real eigenvalues
                    double sq = sqrt(disc);
                    S.eig_re[q] = 0.5 * (aa + dd) + sq; S.eig_im[q] = 0.0; ++q;
                    S.eig_re[q] = 0.5 * (aa + dd) - sq; S.eig_im[q] = 0.0; ++q;
                } else {
                    // tau = re -+ i im: the member with Im(tau) < 0 has Im(xi) > 0
                    S.eig_re[q] = 0.5 * (aa + dd); S.eig_im[q] = -sqrt(-disc); ++q;
                    S.eig_re[q] = 0.5 * (aa + dd); S.eig_im[q] = sqrt(-disc); ++q;
                }
                i += 2;
            } else {
                S.eig_re[q] = S.H[i * LDS + i]; S.eig_im[q] = 0.0; ++q;
                i += 1;
            }
        }
        // units: real eigenvalues and conjugate pairs (represented by Im(tau) < 0)
        int nu = 0;
        int unit_e[MAXM];
        double key_abs[MAXM], key_re[MAXM];
        for (int e = 0; e < nk; ++e) {
            if (S.eig_im[e] > 0.0) continue;
            double re = S.eig_re[e], im = S.eig_im[e], m2 = re * re + im * im;
            double xr = m2 > 0.0 ? re / m2 : INFINITY, xim = m2 > 0.0 ? -im / m2 : 0.0;
            key_abs[nu] = m2 > 0.0 ? hypot(xr, xim) : INFINITY;
            key_re[nu] = xr;
            unit_e[nu] = e;
            ++nu;
        }
        for (int i2 = 1; i2 < nu; ++i2) {
            double ka = key_abs[i2], kr = key_re[i2];
            int ue = unit_e[i2];
            int j = i2 - 1;
            while (j >= 0 && (key_abs[j] > ka || (key_abs[j] == ka && key_re[j] > kr))) {
                key_abs[j + 1] = key_abs[j]; key_re[j + 1] = key_re[j]; unit_e[j + 1] = unit_e[j];
                --j;
            }
            key_abs[j + 1] = ka; key_re[j + 1] = kr; unit_e[j + 1] = ue;
        }
        int sel = 0, ns = 0;
        for (int u = 0; u < nu && sel < kp; ++u) {
            int e = unit_e[u];
            bool pair = S.eig_im[e] != 0.0;
            S.order[ns] = e;
            S.kind[ns] = pair ? ((kp - sel >= 2) ? 2 : 1) : 0;
            sel += pair ? 2 : 1;
            ++ns;
        }
        // numerical clusters among the selected: later members get a shifted
        // inverse iteration and are orthogonalised against earlier ones
        for (int u = 0; u < ns; ++u) {
            int c = 0;
            double re = S.eig_re[S.order[u]], im = S.eig_im[S.order[u]];
            double mag = fmax(fabs(re) + fabs(im), 1e-300);
            for (int v = 0; v < u; ++v) {
                double d = fabs(S.eig_re[S.order[v]] - re) + fabs(S.eig_im[S.order[v]] - im);
                if (d <= 1e-8 * mag) ++c;
            }
            S.nclose[u] = c;
        }
        S.ints[3] = ns;
        for (int u = 0; u < ns; ++u) {
            int e = S.order[u];
            double re = S.eig_re[e], im = S.eig_im[e], m2 = re * re + im * im;
            a.xi[2 * u] = re / m2;
            a.xi[2 * u + 1] = -im / m2;
        }
    }
    bsync();
    for (int i = tid; i < kStateWords; i += NT) gst[i] = sst[i];   // selection saved for k_eigvec
    return;
  }
    const int nsel = S.ints[3];
    STAMP(5);
    // ---- 5. (k_eigvec) eigenvectors of the selected units are in Yre, Yim
    bsync();
    STAMP(6);
    // ---- cluster orthogonalisation, pair rotation, unit norm (warp 0, in the
    // orthonormal basis: plain complex inner products)
    if (warp == 0) {
        for (int u = 0; u < nsel; ++u) {
            double* yr = Yre + u * MAXM;
            double* yi = Yim + u * MAXM;
            // two passes of modified Gram-Schmidt against the earlier members
            // of the cluster (the second restores the orthogonality the first
            // loses when most of y lies in their span)
            for (int pass = 0; pass < 2 && S.nclose[u] > 0; ++pass) {
                const int e = S.order[u];
                const double re = S.eig_re[e], im = S.eig_im[e];
                const double mag = fmax(fabs(re) + fabs(im), 1e-300);
                for (int v = 0; v < u; ++v) {
                    const int f = S.order[v];
                    if (fabs(S.eig_re[f] - re) + fabs(S.eig_im[f] - im) > 1e-8 * mag) continue;
                    const double* vr = Yre + v * MAXM;
                    const double* vi = Yim + v * MAXM;
                    // y -= v (v^H y) / (v^H v)
                    double pr = 0.0, pi = 0.0, vv = 0.0;
                    for (int i = lane; i < nk; i += 32) {
                        pr += vr[i] * yr[i] + vi[i] * yi[i];
                        pi += vr[i] * yi[i] - vi[i] * yr[i];
                        vv += vr[i] * vr[i] + vi[i] * vi[i];
                    }
                    pr = warp_sum(pr); pi = warp_sum(pi); vv = warp_sum(vv);
                    pr /= vv; pi /= vv;
                    for (int i = lane; i < nk; i += 32) {
                        double ar = vr[i] * pr - vi[i] * pi, ai = vr[i] * pi + vi[i] * pr;
                        yr[i] -= ar;
                        yi[i] -= ai;
                    }
                    __threadfence_block();
                    wsync();
                }
            }
            double aa = 0.0, bb = 0.0, ab = 0.0;
            for (int i = lane; i < nk; i += 32) { aa += yr[i] * yr[i]; bb += yi[i] * yi[i]; ab += yr[i] * yi[i]; }
            aa = warp_sum(aa); bb = warp_sum(bb); ab = warp_sum(ab);
            double c = 1.0, sn = 0.0;
            if (S.kind[u] != 0) {
                double phi = 0.5 * atan2(-2.0 * ab, aa - bb);
                c = cos(phi); sn = sin(phi);
            }
            double nrm = sqrt(aa + bb);
            if (!(nrm > 0.0)) nrm = 1.0;
            for (int i = lane; i < nk; i += 32) {
                double r = yr[i], im2 = yi[i];
                yr[i] = (r * c - im2 * sn) / nrm;
                yi[i] = (r * sn + im2 * c) / nrm;
            }
            __threadfence_block();
            wsync();
        }
    }
    bsync();
    // ---- Y' = [Y0 YR yR~ YI] (kept basis), column tags: thread 0 assigns the
    // columns of each unit (keep: real part, nclose: imaginary part or -1;
    // both free after the cluster step), then every thread copies entries
    if (tid == 0) {
        int nreal = 0, npair = 0;
        bool has_cut = false;
        for (int u = 0; u < nsel; ++u) {
            if (S.kind[u] == 0) ++nreal;
            else if (S.kind[u] == 2) ++npair;
            else has_cut = true;
        }
        int col = 0, pr = 0;
        const int base_R = nreal, base_cut = nreal + npair, base_I = nreal + npair + (has_cut ? 1 : 0);
        for (int u = 0; u < nsel; ++u) {
            if (S.kind[u] == 0) {
                S.keep[u] = col; S.nclose[u] = -1;
                a.tags[col] = 0; a.tag_partner[col] = -1;
                ++col;
            } else if (S.kind[u] == 2) {
                const int cr = base_R + pr, ci = base_I + pr;
                S.keep[u] = cr; S.nclose[u] = ci;
                a.tags[cr] = 1; a.tag_partner[cr] = ci;
                a.tags[ci] = 3; a.tag_partner[ci] = cr;
                ++pr;
            } else {
                S.keep[u] = base_cut; S.nclose[u] = -1;
                a.tags[base_cut] = 2; a.tag_partner[base_cut] = -1;
            }
        }
    }
    bsync();
    for (int idx = tid; idx < nsel * nk; idx += NT) {
        const int u = idx / nk, i = idx - u * nk;
        Yp[S.keep[u] * MAXM + i] = Yre[u * MAXM + i];
        if (S.nclose[u] >= 0) Yp[S.nclose[u] * MAXM + i] = Yim[u * MAXM + i];
    }
    __threadfence_block();
    bsync();
    STAMP(7);
    // ---- 6. raw coefficients.  Z-hat = Z diag(colscale t) R^{-1}; R^{-1} is
    // upper triangular with the V columns first, so
    //   P_new = Z-hat[:, rest] Y'_rest = Z diag(colscale t) R^{-1} [0; Y'_rest]
    //   V_new - P_new = Z-hat[:, V] Y'_V = Z_V diag(colscale t) R_VV^{-1} Y'_V
    // Four lanes per solve split each inner sum (l mod 4) and combine it by two
    // shuffles: column j = 4 warp + (g & 3) of lane group g = lane / 4, groups
    // 0..3 solve for Wr and 4..7 for Wv, all in one instruction stream (an
    // FP64 warp instruction costs the same whatever its active lanes, so a
    // quarter of the terms per lane is a quarter of the time); the diagonal's
    // reciprocals are formed once, in parallel.
    static_assert(MAXKP <= 16, "four warps of four columns");
    for (int i = tid; i < nk; i += NT) S.red[i] = 1.0 / S.A[i * LDS + i];
    bsync();
    {
        const int g4 = lane & 3, grp = lane >> 2;
        const int j = warp * 4 + (grp & 3);
        const bool isv = grp >= 4;
        double* W = isv ? Wv : Wr;
        const int lim = isv ? nvk : nk;
        for (int i = nk - 1; i >= 0; --i) {
            const bool act = j < kp && i < lim;
            double part = 0.0;
            if (act)
                for (int l = i + 1 + g4; l < lim; l += 4) part = fma(-S.A[i * LDS + l], W[j * MAXM + l], part);
            part += __shfl_xor_sync(0xffffffffu, part, 1);
            part += __shfl_xor_sync(0xffffffffu, part, 2);
            if (act && g4 == 0) {
                const double y = (isv || i >= nvk) ? Yp[j * MAXM + i] : 0.0;
                W[j * MAXM + i] = (y + part) * S.red[i];
            }
            __syncwarp();
        }
    }
    for (int i = tid; i < m * kp; i += NT) a.Cp[i] = 0.0;
    for (int i = tid; i < a.nv * kp; i += NT) a.Cvv[i] = 0.0;
    __threadfence_block();
    bsync();
    for (int i = tid; i < nk * kp; i += NT) {
        const int q = i / kp, j = i % kp;
        const int raw = S.kidx[q];
        const double tr = S.t[raw] * a.colscale[raw];
        a.Cp[raw * kp + j] = tr * Wr[j * MAXM + q];
        if (q < nvk) a.Cvv[raw * kp + j] = tr * Wv[j * MAXM + q];
    }
    STAMP(8);
    if (tid == 0) {
        a.out_int[0] = kDenseOK;
        a.out_int[1] = nk;
        a.out_int[2] = nsel;
    }
#undef STAMP
}

// Eigenvector of one selected unit (CTA u, one warp): inverse iteration on the
// saved Hessenberg form H0, back to C's basis with the Householder reflectors,
// then y = L^{-T} z in the orthonormal basis, into Yre[u], Yim[u].  The units
// run as separate CTAs on separate SMs (the FP64 work of one unit is serial).
// shared memory of k_eigvec: H0, the Cholesky factor L of G_L and the
// Householder vectors (MAXM x LDS each), the reflector coefficients, then the
// double-word working set: the packed LU factor of the inverse iteration,
// its multipliers, pivot reciprocals and row swaps, the vector and two work
// rows, and the result y (re, im)
struct EigvecDw {
    cdw U[kLuComplex];
    cdw mult[MAXM], rpiv[MAXM], x[MAXM], cur[MAXM], nxt[MAXM];
    dw yr[MAXM], yi[MAXM];
    int swp[MAXM];
};
constexpr size_t kEigvecShmDoubles = 3 * (size_t)MAXM * LDS + MAXM + (sizeof(EigvecDw) + 7) / 8;

__global__ void __launch_bounds__(32) k_eigvec(DenseArgs a) {
    extern __shared__ __align__(16) double sh0[];
    double* sL = sh0 + MAXM * LDS;
    double* sV = sL + MAXM * LDS;
    double* sbeta = sV + MAXM * LDS;
    EigvecDw* E = reinterpret_cast<EigvecDw*>(sbeta + MAXM);
    const Smem* G = state_of(a);
    if (G->ints[6]) return;
    const int u = blockIdx.x;
    const int nsel = G->ints[3], nk = G->ints[0];
    if (u >= nsel) return;
    const int lane = threadIdx.x;
    double hn = 0.0, ln = 0.0;
    for (int i = lane; i < nk * LDS; i += 32) {
        const double v = G->H0[i];
        sh0[i] = v;
        sL[i] = G->B[i];
        sV[i] = G->Vh[i];
        if (i % LDS < nk) {
            hn = fmax(hn, fabs(v));
            ln = fmax(ln, fabs(G->B[i]));
        }
    }
    for (int i = lane; i < nk; i += 32) sbeta[i] = G->beta[i];
    hn = warp_max(hn);
    ln = warp_max(ln);
    __syncwarp();
    // H0 and lam scaled by a power of two to unit norm
    const double down = ldexp(1.0, -(hn > 0.0 ? ilogb(hn) : 0));
    const int e = G->order[u];
    double lre = G->eig_re[e], lim = G->eig_im[e];
    if (G->nclose[u] > 0) { lre *= 1.0 + 1e-10 * G->nclose[u]; lim *= 1.0 + 1e-10 * G->nclose[u]; }
    const cdw lam = {dw_from_double(lre * down), dw_from_double(lim * down)};
    const float tiny = 0x1p-46f;   // a few units of the double-word precision of the unit-norm matrix
    inverse_iteration_dw(sh0, nk, down, lam, E->x, E->U, E->mult, E->rpiv, E->swp, E->cur, E->nxt, tiny);
    // z = Q x with Q = H_0 H_1 ... (reflectors applied last-first)
    for (int k = nk - 3; k >= 0; --k) {
        const double bk = sbeta[k];
        if (bk == 0.0) continue;
        const double* v = sV + k * LDS;
        dw sr = dw_make(0.0f), si = dw_make(0.0f);
        for (int i = k + 1 + lane; i < nk; i += 32) {
            const dw vi = dw_from_double(v[i]);
            sr = dw_add(sr, dw_mul(vi, E->x[i].re));
            si = dw_add(si, dw_mul(vi, E->x[i].im));
        }
        const dw b = dw_from_double(bk);
        sr = dw_mul(warp_sum_dw(sr), b);
        si = dw_mul(warp_sum_dw(si), b);
        __syncwarp();
        for (int i = k + 1 + lane; i < nk; i += 32) {
            const dw vi = dw_from_double(v[i]);
            E->x[i].re = dw_sub(E->x[i].re, dw_mul(sr, vi));
            E->x[i].im = dw_sub(E->x[i].im, dw_mul(si, vi));
        }
        __syncwarp();
    }
    // y = L^{-T} z: column-oriented back substitution with the lower factor L
    // (scaled to unit norm; y then carries the inverse scale, undone below)
    const double ld = ldexp(1.0, -(ln > 0.0 ? ilogb(ln) : 0));
    for (int i = lane; i < nk; i += 32) { E->yr[i] = E->x[i].re; E->yi[i] = E->x[i].im; }
    __syncwarp();
    for (int i = nk - 1; i >= 0; --i) {
        const dw rl = dw_div(dw_make(1.0f), dw_from_double(sL[i * LDS + i] * ld));
        const dw yr = dw_mul(E->yr[i], rl), yi = dw_mul(E->yi[i], rl);
        __syncwarp();
        for (int j = lane; j < i; j += 32) {
            const dw l = dw_from_double(sL[i * LDS + j] * ld);
            E->yr[j] = dw_sub(E->yr[j], dw_mul(l, yr));
            E->yi[j] = dw_sub(E->yi[j], dw_mul(l, yi));
        }
        if (lane == 0) { E->yr[i] = yr; E->yi[i] = yi; }
        __syncwarp();
    }
    double* yr = a.work + (size_t)u * MAXM;
    double* yi = a.work + (size_t)MAXM * MAXM + (size_t)u * MAXM;
    for (int i = lane; i < nk; i += 32) {
        yr[i] = dw_to_double(E->yr[i]) * ld;
        yi[i] = dw_to_double(E->yi[i]) * ld;
    }
}

// Eigenvalues of the saved Hessenberg form (two warps; see k_extract).  The
// stage clocks 3 and 4 and the sweep counts come from this launch.
__global__ void __launch_bounds__(kFrancisThreads) k_francis(DenseArgs a) {
    extern __shared__ __align__(16) double shh[];
    Smem* G = state_of(a);
    if (G->ints[6]) return;
    const int nk = G->ints[0];
    const int t = threadIdx.x;
    for (int i = t; i < nk * LDS; i += kFrancisThreads) shh[i] = G->H[i];
    __syncthreads();
    if (a.clk && t == 0) a.clk[3] = clock64();
    const bool conv = francis_eigenvalues(shh, nk, a.clk ? a.clk + 9 : nullptr);
    if (a.clk && t == 0) a.clk[4] = clock64();
    for (int i = t; i < nk * LDS; i += kFrancisThreads) G->H[i] = shh[i];
    if (t == 0) G->ints[2] = conv ? 1 : 0;
}

}  // namespace

size_t dense_smem_bytes() { return sizeof(Smem); }

// Yre, Yim, Yp (3 MAXM^2) and the shared-memory state passed between the
// launches.
size_t dense_work_doubles() { return kDenseWorkDoubles; }
static_assert(kWorkMainDoubles >= 3 * (size_t)MAXM * MAXM, "dense scratch layout");

cudaError_t dense_extract(const DenseArgs& a, cudaStream_t s) {
    size_t shm = sizeof(Smem);
    cudaError_t e = cudaFuncSetAttribute(k_extract, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) return e;
    const size_t shf = sizeof(double) * MAXM * LDS;
    e = cudaFuncSetAttribute(k_francis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shf);
    if (e != cudaSuccess) return e;
    const size_t she = sizeof(double) * kEigvecShmDoubles;
    e = cudaFuncSetAttribute(k_eigvec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)she);
    if (e != cudaSuccess) return e;
    k_extract<<<1, NT, shm, s>>>(a, 0);
    k_francis<<<1, kFrancisThreads, shf, s>>>(a);
    k_extract<<<1, NT, shm, s>>>(a, 1);
    k_eigvec<<<a.kp, 32, she, s>>>(a);
    k_extract<<<1, NT, shm, s>>>(a, 2);
    count_launches(5);
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
// (m = 64): three 64 x 64 arrays and the saved state, about 263 KiB.  Every
// GPU that loads the library holds this array until the process exits.
constexpr size_t kNoAllocScratchDoubles = plhr::kDenseWorkDoubles;
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
