// Absolute-value multigrid V-cycle (Appendix A, Algorithm 4) on blocks of
// vectors [grid point][column], FP64.
//
// Per smoothing level l (finest first):
//   step 2  pre-smoothing  w <- w + omega_l (r - B_l w), nu times from w = 0
//   step 3  r_c = R (r - B_l w), w_c = AV-MG(r_c) (or the exact coarsest
//           solve), w <- w + P w_c
//   step 4  post-smoothing, nu times (M_l = omega_l^{-1} I is symmetric, so
//           M_l^{-*} = M_l^{-1})
// B_l is the level Laplacian L_l or p_2(L_l - sigma I) = ((L_l - sigma)^2 +
// c_l^2)/(2 c_l).  Transfers are cell-centred: the restriction is R = P^T / 2^d
// for the prolongation P (piecewise constant, or the tensor product of the 1D
// weights 3/4, 1/4 to the two nearest coarse cells).  The coarsest solve
// applies |L_0 - sigma I|^{-1} = S diag(1 / |mu - sigma|) S^T with a separable
// orthonormal basis S = Sx (x) Sy (x) Sz and per-axis eigenvalues mu.
//
// INV-MG (Appendix A, Algorithm 5; H.indefinite): the same cycle with
// B_l = L_l - sigma I_l on every level (the shift enters the sweeps and the
// residual) and the signed coarsest solve S diag(1 / (mu - sigma)) S^T.
#include "plhr_internal.h"

namespace plhr {
namespace {

constexpr int kT = 256;

struct G3 {
    int64_t nx, ny, nz;
};

__device__ __forceinline__ void unflat(int64_t row, const G3& g, int64_t& ix, int64_t& iy, int64_t& iz) {
    if ((uint64_t)row <= 0xffffffffull) {   // 32-bit divisions (the grid fits: nx, ny < 2^32)
        const unsigned r = (unsigned)row, nx = (unsigned)g.nx, ny = (unsigned)g.ny;
        const unsigned t = r / nx;
        ix = r - t * nx;
        const unsigned z = t / ny;
        iy = t - z * ny;
        iz = z;
        return;
    }
    ix = row % g.nx;
    int64_t t = row / g.nx;
    iy = t % g.ny;
    iz = t / g.ny;
}

// 2d/h^2 u - sum of neighbours / h^2 (scaled by ih2), zero outside the grid
template <bool D3>
__device__ __forceinline__ double lap_pt(const double* __restrict__ xp, int64_t ld, int64_t ix, int64_t iy,
                                         int64_t iz, const G3& g) {
    double s = (D3 ? 6.0 : 4.0) * xp[0];
    if (ix > 0) s -= xp[-ld];
    if (ix < g.nx - 1) s -= xp[ld];
    if (iy > 0) s -= xp[-ld * g.nx];
    if (iy < g.ny - 1) s -= xp[ld * g.nx];
    if (D3) {
        if (iz > 0) s -= xp[-ld * g.nx * g.ny];
        if (iz < g.nz - 1) s -= xp[ld * g.nx * g.ny];
    }
    return s;
}

#define GRID_LOOP(total)                                                                 \
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (total);        \
         e += (int64_t)gridDim.x * blockDim.x)

// w_out = w_in + om * (r - (ih2 * L - shift) w_in)    (w_in may be null: w_out = om r);
// SHIFT = false is the AV-MG sweep (shift 0, the expression without the shift term)
template <bool D3, bool SHIFT>
__global__ void __launch_bounds__(kT) k_rich_lap(G3 g, int nc, double ih2, double shift, double om,
                                                 const double* __restrict__ win, const double* __restrict__ r,
                                                 int64_t ldr, double* __restrict__ wout, int64_t total) {
    GRID_LOOP(total) {
        int64_t row;
        int c;
        split_index(e, nc, row, c);
        double rv = r[row * ldr + c];
        double v;
        if (win) {
            int64_t ix, iy, iz;
            unflat(row, g, ix, iy, iz);
            const double* wp = win + row * nc + c;
            if (SHIFT) v = wp[0] + om * (rv - (ih2 * lap_pt<D3>(wp, nc, ix, iy, iz, g) - shift * wp[0]));
            else v = wp[0] + om * (rv - ih2 * lap_pt<D3>(wp, nc, ix, iy, iz, g));
        } else {
            v = om * rv;
        }
        wout[row * nc + c] = v;
    }
}

// t = ih2 * L x - sig * x
template <bool D3>
__global__ void __launch_bounds__(kT) k_shifted(G3 g, int nc, double ih2, double sig, const double* __restrict__ x,
                                                double* __restrict__ t, int64_t total) {
    GRID_LOOP(total) {
        int64_t row;
        int c;
        split_index(e, nc, row, c);
        int64_t ix, iy, iz;
        unflat(row, g, ix, iy, iz);
        const double* xp = x + row * nc + c;
        t[row * nc + c] = ih2 * lap_pt<D3>(xp, nc, ix, iy, iz, g) - sig * xp[0];
    }
}

// B w for the polynomial level from t = (L - sig) w:  ((L - sig) t + c^2 w) / (2c)
// mode 0: w_out = w + om (r - Bw);  mode 1: w_out = r - Bw (residual)
template <bool D3>
__global__ void __launch_bounds__(kT) k_poly_step(G3 g, int nc, double ih2, double sig, double cpar, double om,
                                                  int mode, const double* __restrict__ w,
                                                  const double* __restrict__ t, const double* __restrict__ r,
                                                  int64_t ldr, double* __restrict__ out, int64_t total) {
    GRID_LOOP(total) {
        int64_t row;
        int c;
        split_index(e, nc, row, c);
        int64_t ix, iy, iz;
        unflat(row, g, ix, iy, iz);
        const double* tp = t + row * nc + c;
        double tt = ih2 * lap_pt<D3>(tp, nc, ix, iy, iz, g) - sig * tp[0];
        double wv = w[row * nc + c];
        double bw = (tt + cpar * cpar * wv) / (2.0 * cpar);
        double res = r[row * ldr + c] - bw;
        out[row * nc + c] = mode == 0 ? wv + om * res : res;
    }
}

// res = r - (ih2 * L - shift) w  (SHIFT = false: r - ih2 * L w)
template <bool D3, bool SHIFT>
__global__ void __launch_bounds__(kT) k_resid_lap(G3 g, int nc, double ih2, double shift, const double* __restrict__ w,
                                                  const double* __restrict__ r, int64_t ldr,
                                                  double* __restrict__ out, int64_t total) {
    GRID_LOOP(total) {
        int64_t row;
        int c;
        split_index(e, nc, row, c);
        int64_t ix, iy, iz;
        unflat(row, g, ix, iy, iz);
        if (SHIFT)
            out[row * nc + c] = r[row * ldr + c] - (ih2 * lap_pt<D3>(w + row * nc + c, nc, ix, iy, iz, g) -
                                                    shift * w[row * nc + c]);
        else
            out[row * nc + c] = r[row * ldr + c] - ih2 * lap_pt<D3>(w + row * nc + c, nc, ix, iy, iz, g);
    }
}

// 1D cell-centred prolongation weights from coarse cells to fine point f:
// constant: f -> (f/2, 1);  linear: f -> (f/2, 3/4) and (f/2 -+ 1, 1/4)
__device__ __forceinline__ int pw1(int lin, int64_t f, int64_t nc_axis, int64_t* idx, double* wt) {
    int64_t I = f >> 1;
    idx[0] = I;
    if (!lin) {
        wt[0] = 1.0;
        return 1;
    }
    wt[0] = 0.75;
    int64_t J = (f & 1) ? I + 1 : I - 1;
    if (J < 0 || J >= nc_axis) return 1;
    idx[1] = J;
    wt[1] = 0.25;
    return 2;
}

// w_fine += P w_coarse
template <bool D3>
__global__ void __launch_bounds__(kT) k_prolong_add(G3 gf, G3 gc, int nc, int lin, const double* __restrict__ wc,
                                                    double* __restrict__ wf, int64_t total) {
    GRID_LOOP(total) {
        int64_t row;
        int c;
        split_index(e, nc, row, c);
        int64_t ix, iy, iz;
        unflat(row, gf, ix, iy, iz);
        int64_t xi[2], yi[2], zi[2];
        double xw[2], yw[2], zw[2];
        int nxw = pw1(lin, ix, gc.nx, xi, xw);
        int nyw = pw1(lin, iy, gc.ny, yi, yw);
        int nzw = D3 ? pw1(lin, iz, gc.nz, zi, zw) : 1;
        if (!D3) { zi[0] = 0; zw[0] = 1.0; }
        double s = 0.0;
        for (int a = 0; a < nzw; ++a)
            for (int b = 0; b < nyw; ++b)
                for (int q = 0; q < nxw; ++q)
                    s += zw[a] * yw[b] * xw[q] * wc[((zi[a] * gc.ny + yi[b]) * gc.nx + xi[q]) * nc + c];
        wf[row * nc + c] += s;
    }
}

// 1D restriction taps R = P^T / 2 per axis: coarse I gathers fine 2I, 2I+1
// (weight 1/2 each, constant) or additionally 2I-1, 2I+2 (linear: 3/8, 3/8,
// 1/8, 1/8).
__device__ __forceinline__ int rw1(int lin, int64_t I, int64_t nf_axis, int64_t* idx, double* wt) {
    if (!lin) {
        idx[0] = 2 * I; wt[0] = 0.5;
        idx[1] = 2 * I + 1; wt[1] = 0.5;
        return 2;
    }
    int n = 0;
    idx[n] = 2 * I; wt[n++] = 0.375;
    idx[n] = 2 * I + 1; wt[n++] = 0.375;
    if (2 * I - 1 >= 0) { idx[n] = 2 * I - 1; wt[n++] = 0.125; }
    if (2 * I + 2 < nf_axis) { idx[n] = 2 * I + 2; wt[n++] = 0.125; }
    return n;
}

template <bool D3>
__global__ void __launch_bounds__(kT) k_restrict(G3 gf, G3 gc, int nc, int lin, const double* __restrict__ f,
                                                 double* __restrict__ rc, int64_t total) {
    GRID_LOOP(total) {
        int64_t row;
        int c;
        split_index(e, nc, row, c);
        int64_t ix, iy, iz;
        unflat(row, gc, ix, iy, iz);
        int64_t xi[4], yi[4], zi[4];
        double xw[4], yw[4], zw[4];
        int nxw = rw1(lin, ix, gf.nx, xi, xw);
        int nyw = rw1(lin, iy, gf.ny, yi, yw);
        int nzw = D3 ? rw1(lin, iz, gf.nz, zi, zw) : 1;
        if (!D3) { zi[0] = 0; zw[0] = 1.0; }
        double s = 0.0;
        for (int a = 0; a < nzw; ++a)
            for (int b = 0; b < nyw; ++b)
                for (int q = 0; q < nxw; ++q)
                    s += zw[a] * yw[b] * xw[q] * f[((zi[a] * gf.ny + yi[b]) * gf.nx + xi[q]) * nc + c];
        rc[row * nc + c] = s;
    }
}

// Coarsest solve, one CTA per column: out = S diag(1/|mu_i + mu_j + mu_k - sig|) S^T in
// (signed: 1 / (mu - sig)); the two work vectors of the column live in shared
// memory, or in global scratch (gwork, 2 n0 doubles per column) when the
// coarsest grid is too large for it
// (S[point][mode] per axis, orthonormal).
// coarsest level: 1024 threads per column (each output is still one thread's
// sum in a fixed order); the transforms of one column are latency-bound
constexpr int kTC = 1024;
__global__ void __launch_bounds__(kTC) k_coarse_sep(int d, int64_t nx, int64_t ny, int64_t nz, int nc,
                                                   const double* __restrict__ Sx, const double* __restrict__ Sy,
                                                   const double* __restrict__ Sz, const double* __restrict__ mx,
                                                   const double* __restrict__ my, const double* __restrict__ mz,
                                                   double sig, int signed_inv, const double* __restrict__ in,
                                                   int64_t ldi, double* __restrict__ out, int64_t ldo,
                                                   double* __restrict__ gwork) {
    extern __shared__ double sh[];
    const int64_t n0 = nx * ny * nz;
    const int c = blockIdx.x;
    double* a = gwork ? gwork + (int64_t)c * 2 * n0 : sh;
    double* b = a + n0;
    for (int64_t i = threadIdx.x; i < n0; i += blockDim.x) a[i] = in[i * ldi + c];
    __syncthreads();
    // forward: coefficient(mode) = sum_point S[point][mode] x[point], axis by axis
    // x axis
    for (int64_t i = threadIdx.x; i < n0; i += blockDim.x) {
        int64_t m = i % nx, rest = i / nx;
        double s = 0.0;
        for (int64_t p = 0; p < nx; ++p) s += Sx[p * nx + m] * a[rest * nx + p];
        b[i] = s;
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n0; i += blockDim.x) {
        int64_t x = i % nx, m = (i / nx) % ny, z = i / (nx * ny);
        double s = 0.0;
        for (int64_t p = 0; p < ny; ++p) s += Sy[p * ny + m] * b[(z * ny + p) * nx + x];
        a[i] = s;
    }
    __syncthreads();
    if (d == 3) {
        for (int64_t i = threadIdx.x; i < n0; i += blockDim.x) {
            int64_t xy = i % (nx * ny), m = i / (nx * ny);
            double s = 0.0;
            for (int64_t p = 0; p < nz; ++p) s += Sz[p * nz + m] * a[p * nx * ny + xy];
            b[i] = s;
        }
        __syncthreads();
    } else {
        for (int64_t i = threadIdx.x; i < n0; i += blockDim.x) b[i] = a[i];
        __syncthreads();
    }
    // scale
    for (int64_t i = threadIdx.x; i < n0; i += blockDim.x) {
        int64_t ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
        double mu = mx[ix] + my[iy] + (d == 3 ? mz[iz] : 0.0);
        b[i] = b[i] / (signed_inv ? mu - sig : fabs(mu - sig));
    }
    __syncthreads();
    // inverse: x[point] = sum_mode S[point][mode] coef[mode]
    if (d == 3) {
        for (int64_t i = threadIdx.x; i < n0; i += blockDim.x) {
            int64_t xy = i % (nx * ny), p = i / (nx * ny);
            double s = 0.0;
            for (int64_t m = 0; m < nz; ++m) s += Sz[p * nz + m] * b[m * nx * ny + xy];
            a[i] = s;
        }
        __syncthreads();
    } else {
        for (int64_t i = threadIdx.x; i < n0; i += blockDim.x) a[i] = b[i];
        __syncthreads();
    }
    for (int64_t i = threadIdx.x; i < n0; i += blockDim.x) {
        int64_t x = i % nx, p = (i / nx) % ny, z = i / (nx * ny);
        double s = 0.0;
        for (int64_t m = 0; m < ny; ++m) s += Sy[p * ny + m] * a[(z * ny + m) * nx + x];
        b[i] = s;
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n0; i += blockDim.x) {
        int64_t p = i % nx, rest = i / nx;
        double s = 0.0;
        for (int64_t m = 0; m < nx; ++m) s += Sx[p * nx + m] * b[rest * nx + m];
        out[i * ldo + c] = s;
    }
}

G3 g3(const Grid& g) { return G3{g.nx, g.ny, g.nz}; }

int nblk(int64_t total) { return grid_size_for(total, kT, sm_count() * 16); }

struct LevelBufs {
    double* cw;    // coarsest level only: global scratch of a large coarsest solve
    double* w0;    // ping
    double* w1;    // pong
    double* tmp;   // residual / polynomial intermediate
    double* rc;    // restricted residual for the next coarser level
    double* wc;    // coarse correction from the next coarser level
};

cudaError_t rich_sweep(const MGLevel& L, double sigma, int nc, const double* win, const double* r, int64_t ldr,
                       double* tmp, double* wout, cudaStream_t s) {
    const Grid& g = L.g;
    int64_t total = g.n() * nc;
    G3 G = g3(g);
    bool d3 = g.d == 3;
    const double shift = L.shifted ? sigma : 0.0;
    if (!L.poly || win == nullptr) {
        const double* wi = L.poly ? nullptr : win;
        if (L.shifted) {
            if (d3) k_rich_lap<true, true><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), shift, L.omega, wi, r, ldr, wout, total);
            else k_rich_lap<false, true><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), shift, L.omega, wi, r, ldr, wout, total);
        } else {
            if (d3) k_rich_lap<true, false><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), 0.0, L.omega, wi, r, ldr, wout, total);
            else k_rich_lap<false, false><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), 0.0, L.omega, wi, r, ldr, wout, total);
        }
        count_launches(1);
        return cudaGetLastError();
    }
    if (d3) k_shifted<true><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), sigma, win, tmp, total);
    else k_shifted<false><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), sigma, win, tmp, total);
    count_launches(1);
    if (d3) k_poly_step<true><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), sigma, L.c, L.omega, 0, win, tmp, r, ldr, wout, total);
    else k_poly_step<false><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), sigma, L.c, L.omega, 0, win, tmp, r, ldr, wout, total);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t level_residual(const MGLevel& L, double sigma, int nc, const double* w, const double* r, int64_t ldr,
                           double* tmp, double* out, cudaStream_t s) {
    const Grid& g = L.g;
    int64_t total = g.n() * nc;
    G3 G = g3(g);
    bool d3 = g.d == 3;
    if (!L.poly) {
        if (L.shifted) {
            if (d3) k_resid_lap<true, true><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), sigma, w, r, ldr, out, total);
            else k_resid_lap<false, true><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), sigma, w, r, ldr, out, total);
        } else {
            if (d3) k_resid_lap<true, false><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), 0.0, w, r, ldr, out, total);
            else k_resid_lap<false, false><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), 0.0, w, r, ldr, out, total);
        }
        count_launches(1);
        return cudaGetLastError();
    }
    if (d3) k_shifted<true><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), sigma, w, tmp, total);
    else k_shifted<false><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), sigma, w, tmp, total);
    count_launches(1);
    if (d3) k_poly_step<true><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), sigma, L.c, L.omega, 1, w, tmp, r, ldr, out, total);
    else k_poly_step<false><<<nblk(total), kT, 0, s>>>(G, nc, g.inv_h2(), sigma, L.c, L.omega, 1, w, tmp, r, ldr, out, total);
    count_launches(1);
    return cudaGetLastError();
}

// largest coarsest grid whose two work vectors are staged in shared memory
constexpr int64_t kCoarseShmPoints = kMaxSmemCoarse;

cudaError_t coarse_solve(const MGHierarchy& H, int nc, const double* in, int64_t ldi, double* out, int64_t ldo,
                         double* gwork, cudaStream_t s) {
    const Grid& g = H.lev[0].g;
    int64_t n0 = g.n();
    const bool global = n0 > kCoarseShmPoints;
    size_t shm = global ? 0 : sizeof(double) * 2 * n0;
    if (shm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_coarse_sep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e != cudaSuccess) return e;
    }
    k_coarse_sep<<<nc, kTC, shm, s>>>(g.d, g.nx, g.ny, g.nz, nc, H.d_basis[0], H.d_basis[1],
                                     g.d == 3 ? H.d_basis[2] : H.d_basis[1], H.d_mu[0], H.d_mu[1],
                                     g.d == 3 ? H.d_mu[2] : H.d_mu[1], H.sigma, H.indefinite, in, ldi, out, ldo,
                                     global ? gwork : nullptr);
    count_launches(1);
    return cudaGetLastError();
}

// Recursive V-cycle on level l; r has leading dimension ldr (level nc otherwise);
// the result is written to out with leading dimension nc.
cudaError_t vcycle(const MGHierarchy& H, int l, int nc, const double* r, int64_t ldr, double* out,
                   std::vector<LevelBufs>& B, cudaStream_t s) {
    if (l == 0) return coarse_solve(H, nc, r, ldr, out, nc, B[0].cw, s);
    const MGLevel& L = H.lev[l];
    const MGLevel& Lc = H.lev[l - 1];
    LevelBufs& b = B[l];
    cudaError_t e;
    // pre-smoothing from zero
    double* cur = b.w0;
    double* nxt = b.w1;
    e = rich_sweep(L, H.sigma, nc, nullptr, r, ldr, b.tmp, cur, s);
    if (e != cudaSuccess) return e;
    for (int i = 1; i < H.nu; ++i) {
        e = rich_sweep(L, H.sigma, nc, cur, r, ldr, b.tmp, nxt, s);
        if (e != cudaSuccess) return e;
        double* t = cur; cur = nxt; nxt = t;
    }
    // coarse-grid correction
    e = level_residual(L, H.sigma, nc, cur, r, ldr, b.tmp, nxt, s);
    if (e != cudaSuccess) return e;
    int64_t totc = Lc.g.n() * nc;
    if (L.g.d == 3) k_restrict<true><<<nblk(totc), kT, 0, s>>>(g3(L.g), g3(Lc.g), nc, H.linear, nxt, b.rc, totc);
    else k_restrict<false><<<nblk(totc), kT, 0, s>>>(g3(L.g), g3(Lc.g), nc, H.linear, nxt, b.rc, totc);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = vcycle(H, l - 1, nc, b.rc, nc, b.wc, B, s);
    if (e != cudaSuccess) return e;
    int64_t tot = L.g.n() * nc;
    if (L.g.d == 3) k_prolong_add<true><<<nblk(tot), kT, 0, s>>>(g3(L.g), g3(Lc.g), nc, H.linear, b.wc, cur, tot);
    else k_prolong_add<false><<<nblk(tot), kT, 0, s>>>(g3(L.g), g3(Lc.g), nc, H.linear, b.wc, cur, tot);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // post-smoothing; the last step writes to out
    for (int i = 0; i < H.nu; ++i) {
        double* dst = (i == H.nu - 1) ? out : nxt;
        e = rich_sweep(L, H.sigma, nc, cur, r, ldr, b.tmp, dst, s);
        if (e != cudaSuccess) return e;
        nxt = cur;
        cur = dst;
    }
    return cudaSuccess;
}

}  // namespace

int64_t mg_workspace_doubles(const MGHierarchy& H, int nc) {
    int64_t tot = 0;
    for (size_t l = 1; l < H.lev.size(); ++l) {
        tot += 3 * H.lev[l].g.n() * nc;            // w0, w1, tmp
        tot += 2 * H.lev[l - 1].g.n() * nc;        // rc, wc
    }
    if (H.lev[0].g.n() > kCoarseShmPoints) tot += 2 * H.lev[0].g.n() * nc;   // large coarsest solve
    return tot;
}

cudaError_t mg_vcycle(const MGHierarchy& H, int nc, const double* r, int64_t ldr, double* w, int64_t ldw,
                      double* work, cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    const int top = (int)H.lev.size() - 1;
    std::vector<LevelBufs> B(H.lev.size());
    double* p = work;
    B[0].cw = nullptr;
    for (int l = 1; l <= top; ++l) {
        int64_t nf = H.lev[l].g.n() * nc, ncc = H.lev[l - 1].g.n() * nc;
        B[l].w0 = p; p += nf;
        B[l].w1 = p; p += nf;
        B[l].tmp = p; p += nf;
        B[l].rc = p; p += ncc;
        B[l].wc = p; p += ncc;
    }
    if (H.lev[0].g.n() > kCoarseShmPoints) B[0].cw = p;
    // the kernels use leading dimension nc for level buffers; the caller's
    // output must be dense (ldw == nc) or is staged through the ping buffer
    if (ldw == nc) return vcycle(H, top, nc, r, ldr, w, B, s);
    return cudaErrorInvalidValue;
}

}  // namespace plhr
