// Double-word form of the absolute-value multigrid V-cycle (Appendix A,
// Algorithm 4): the same cycle as the FP64 and FP32 ones, with level buffers
// stored as double-word values (hi + lo FP32 pairs, ~48 bits) and all
// arithmetic in double-word operations on the FP32 pipes.  It serves the FP64
// phase of the mixed-precision solve: accurate enough that T acts as a fixed
// linear operator down to ~1e-13 (an FP32 V-cycle's rounding, ~1e-6 of its
// output, stalls the T-harmonic iteration near 1e-6), and several times
// faster than FP64 arithmetic, which is bound by GB300's FP64 pipe.
// The FP64 right-hand side is converted once; the result is converted back.
#include "dword.h"
#include "plhr_internal.h"

namespace plhr {
namespace {

constexpr int kT = 256;

struct Ld {
    int nx, ny, nz, nc;
    dw ih2;
};

struct Pos {
    int ix, iy, iz, c;
    int64_t row;
};

// one element (grid point, column) per thread; a CTA covers 256 elements of
// one x-line; ix = floor(t / nc) through a float reciprocal (t < 2^13, nc <= 32)
__device__ __forceinline__ bool pos_of(const Ld& g, Pos& p) {
    const int t = blockIdx.x * kT + threadIdx.x;
    if (t >= g.nx * g.nc) return false;
    p.ix = (int)(((float)t + 0.5f) / (float)g.nc);
    p.c = t - p.ix * g.nc;
    p.iy = blockIdx.y;
    p.iz = blockIdx.z;
    p.row = ((int64_t)p.iz * g.ny + p.iy) * g.nx + p.ix;
    return true;
}

// L x at p (leading dimension nc), zero outside: 2d x_c - sum of the
// neighbours, summed lazily (48 bits leave ample room for the cancellation);
// xc receives x
template <bool D3>
__device__ __forceinline__ dw lapd(dw& xc, const dw* __restrict__ xp, const Ld& g, const Pos& p) {
    const int ld = g.nc, sy = ld * g.nx, sz = sy * g.ny;
    xc = xp[0];
    dwacc s = {0.0f, 0.0f};
    if (p.ix > 0) dwacc_sub(s, xp[-ld]);
    if (p.ix < g.nx - 1) dwacc_sub(s, xp[ld]);
    if (p.iy > 0) dwacc_sub(s, xp[-sy]);
    if (p.iy < g.ny - 1) dwacc_sub(s, xp[sy]);
    if (D3) {
        if (p.iz > 0) dwacc_sub(s, xp[-sz]);
        if (p.iz < g.nz - 1) dwacc_sub(s, xp[sz]);
    }
    dwacc_add_mul_f(s, xc, D3 ? 6.0f : 4.0f);
    return dwacc_result(s);
}

// w = 2 om r - om^2 L r  (first two sweeps from w = 0, B = L); om2x = 2 om,
// om2ih2 = om^2 / h^2
template <bool D3>
__global__ void __launch_bounds__(kT) k_rich2(Ld g, dw om2x, dw om2ih2, const dw* __restrict__ r, dw* __restrict__ w) {
    Pos p;
    if (!pos_of(g, p)) return;
    dw rc;
    const dw l = lapd<D3>(rc, r + p.row * g.nc + p.c, g, p);
    dwacc a = {0.0f, 0.0f};
    dwacc_add_mul(a, om2x, rc);
    dwacc_add_mul(a, dw_neg(om2ih2), l);
    w[p.row * g.nc + p.c] = dwacc_result(a);
}

// w = om r
__global__ void __launch_bounds__(kT) k_scale(Ld g, dw om, const dw* __restrict__ r, dw* __restrict__ w) {
    Pos p;
    if (!pos_of(g, p)) return;
    const int64_t e = p.row * g.nc + p.c;
    w[e] = dw_mul(om, r[e]);
}

// wout = win + om (r - L win) = win + om r - (om / h^2) L' win; omih2 = om / h^2
template <bool D3>
__global__ void __launch_bounds__(kT) k_rich(Ld g, dw om, dw omih2, const dw* __restrict__ win,
                                             const dw* __restrict__ r, dw* __restrict__ wout) {
    Pos p;
    if (!pos_of(g, p)) return;
    const int64_t e = p.row * g.nc + p.c;
    dw wc;
    const dw l = lapd<D3>(wc, win + e, g, p);
    dwacc a = dwacc_of(wc);
    dwacc_add_mul(a, om, r[e]);
    dwacc_add_mul(a, dw_neg(omih2), l);
    wout[e] = dwacc_result(a);
}

// t = L x - sig x
template <bool D3>
__global__ void __launch_bounds__(kT) k_shifted(Ld g, dw sig, const dw* __restrict__ x, dw* __restrict__ t) {
    Pos p;
    if (!pos_of(g, p)) return;
    const int64_t e = p.row * g.nc + p.c;
    dw xc;
    const dw l = lapd<D3>(xc, x + e, g, p);
    dwacc a = {0.0f, 0.0f};
    dwacc_add_mul(a, g.ih2, l);
    dwacc_add_mul(a, dw_neg(sig), xc);
    t[e] = dwacc_result(a);
}

// B w = ((L - sig) t + c^2 w) / (2c), t = (L - sig) w;
// mode 0: out = w + om (r - B w);  mode 1: out = r - B w
template <bool D3>
__global__ void __launch_bounds__(kT) k_poly(Ld g, dw sig, dw c2, dw inv2c, dw om, int mode,
                                             const dw* __restrict__ w, const dw* __restrict__ t,
                                             const dw* __restrict__ r, dw* __restrict__ out) {
    Pos p;
    if (!pos_of(g, p)) return;
    const int64_t e = p.row * g.nc + p.c;
    dw tc;
    const dw l = lapd<D3>(tc, t + e, g, p);
    const dw tt = dw_sub(dw_mul(g.ih2, l), dw_mul(sig, tc));
    const dw wv = w[e];
    const dw bw = dw_mul(dw_add(tt, dw_mul(c2, wv)), inv2c);
    const dw res = dw_sub(r[e], bw);
    out[e] = mode == 0 ? dw_add(wv, dw_mul(om, res)) : res;
}

// out = r - L w
template <bool D3>
__global__ void __launch_bounds__(kT) k_resid(Ld g, const dw* __restrict__ w, const dw* __restrict__ r,
                                              dw* __restrict__ out) {
    Pos p;
    if (!pos_of(g, p)) return;
    const int64_t e = p.row * g.nc + p.c;
    dw wc;
    const dw l = lapd<D3>(wc, w + e, g, p);
    dwacc a = dwacc_of(r[e]);
    dwacc_add_mul(a, dw_neg(g.ih2), l);
    out[e] = dwacc_result(a);
}

// 1D cell-centred prolongation weights (constant: 1; linear: 3/4 and 1/4) and
// restriction taps R = P^T / 2 (1/2, 1/2; linear: 3/8, 3/8, 1/8, 1/8): all
// exact in FP32, as are their products
__device__ __forceinline__ int pw(int lin, int f, int ncx, int* idx, float* wt) {
    const int I = f >> 1;
    idx[0] = I;
    if (!lin) {
        wt[0] = 1.0f;
        return 1;
    }
    wt[0] = 0.75f;
    const int J = (f & 1) ? I + 1 : I - 1;
    if (J < 0 || J >= ncx) return 1;
    idx[1] = J;
    wt[1] = 0.25f;
    return 2;
}

__device__ __forceinline__ int rw(int lin, int I, int nfx, int* idx, float* wt) {
    if (!lin) {
        idx[0] = 2 * I; wt[0] = 0.5f;
        idx[1] = 2 * I + 1; wt[1] = 0.5f;
        return 2;
    }
    int n = 0;
    idx[n] = 2 * I; wt[n++] = 0.375f;
    idx[n] = 2 * I + 1; wt[n++] = 0.375f;
    if (2 * I - 1 >= 0) { idx[n] = 2 * I - 1; wt[n++] = 0.125f; }
    if (2 * I + 2 < nfx) { idx[n] = 2 * I + 2; wt[n++] = 0.125f; }
    return n;
}

// wf += P wc   (over the fine level)
template <bool D3>
__global__ void __launch_bounds__(kT) k_prolong_add(Ld gf, Ld gc, int lin, const dw* __restrict__ wc,
                                                    dw* __restrict__ wf) {
    Pos p;
    if (!pos_of(gf, p)) return;
    int xi[2], yi[2], zi[2];
    float xw[2], yw[2], zw[2];
    const int nxw = pw(lin, p.ix, gc.nx, xi, xw);
    const int nyw = pw(lin, p.iy, gc.ny, yi, yw);
    int nzw = 1;
    zi[0] = 0; zw[0] = 1.0f;
    if (D3) nzw = pw(lin, p.iz, gc.nz, zi, zw);
    const int64_t e = p.row * gf.nc + p.c;
    dwacc acc = dwacc_of(wf[e]);
    for (int a = 0; a < nzw; ++a)
        for (int b = 0; b < nyw; ++b) {
            const dw* line = wc + ((int64_t)zi[a] * gc.ny + yi[b]) * gc.nx * gc.nc + p.c;
            for (int q = 0; q < nxw; ++q) dwacc_add_mul_f(acc, line[(int64_t)xi[q] * gc.nc], zw[a] * yw[b] * xw[q]);
        }
    wf[e] = dwacc_result(acc);
}

// rc = R f   (over the coarse level)
template <bool D3>
__global__ void __launch_bounds__(kT) k_restrict(Ld gf, Ld gc, int lin, const dw* __restrict__ f,
                                                 dw* __restrict__ rc) {
    Pos p;
    if (!pos_of(gc, p)) return;
    int xi[4], yi[4], zi[4];
    float xw[4], yw[4], zw[4];
    const int nxw = rw(lin, p.ix, gf.nx, xi, xw);
    const int nyw = rw(lin, p.iy, gf.ny, yi, yw);
    int nzw = 1;
    zi[0] = 0; zw[0] = 1.0f;
    if (D3) nzw = rw(lin, p.iz, gf.nz, zi, zw);
    dwacc acc = {0.0f, 0.0f};
    for (int a = 0; a < nzw; ++a)
        for (int b = 0; b < nyw; ++b) {
            const dw* line = f + ((int64_t)zi[a] * gf.ny + yi[b]) * gf.nx * gf.nc + p.c;
            for (int q = 0; q < nxw; ++q) dwacc_add_mul_f(acc, line[(int64_t)xi[q] * gf.nc], zw[a] * yw[b] * xw[q]);
        }
    rc[p.row * gc.nc + p.c] = dwacc_result(acc);
}

// The transfers one grid line per CTA, separably.  Prolongation (one fine
// x-line): the y-z interpolation of the coarse values under the line, once
// per coarse x (up to 4 taps), then the x interpolation (2 taps), 4 instead
// of 8 double-word multiply-adds per fine value.  Restriction (one coarse
// x-line): the y-z sums of the fine values, once per fine x (up to 16 taps),
// then the x taps (up to 4), 36 instead of 64 per coarse value.  The partial
// line is kept in shared memory.
template <bool D3>
__global__ void __launch_bounds__(kT) k_prolong_line(Ld gf, Ld gc, int lin, const dw* __restrict__ wc,
                                                     dw* __restrict__ wf) {
    extern __shared__ dw ush[];   // [coarse x][column]
    const int iy = blockIdx.x, iz = blockIdx.y;
    int yi[2], zi[2];
    float yw[2], zw[2];
    const int nyw = pw(lin, iy, gc.ny, yi, yw);
    int nzw = 1;
    zi[0] = 0; zw[0] = 1.0f;
    if (D3) nzw = pw(lin, iz, gc.nz, zi, zw);
    const int nc = gf.nc, nu = gc.nx * nc;
    for (int t = threadIdx.x; t < nu; t += blockDim.x) {
        const int X = t / nc, c = t - X * nc;
        dwacc acc = {0.0f, 0.0f};
        for (int a = 0; a < nzw; ++a)
            for (int b = 0; b < nyw; ++b)
                dwacc_add_mul_f(acc, wc[(((int64_t)zi[a] * gc.ny + yi[b]) * gc.nx + X) * nc + c], zw[a] * yw[b]);
        ush[t] = dwacc_result(acc);
    }
    __syncthreads();
    const int nf = gf.nx * nc;
    const int64_t row0 = ((int64_t)iz * gf.ny + iy) * gf.nx;
    for (int t = threadIdx.x; t < nf; t += blockDim.x) {
        const int x = t / nc, c = t - x * nc;
        int xi[2];
        float xw[2];
        const int nxw = pw(lin, x, gc.nx, xi, xw);
        const int64_t e = (row0 + x) * nc + c;
        dwacc acc = dwacc_of(wf[e]);
        for (int q = 0; q < nxw; ++q) dwacc_add_mul_f(acc, ush[xi[q] * nc + c], xw[q]);
        wf[e] = dwacc_result(acc);
    }
}

template <bool D3>
__global__ void __launch_bounds__(kT) k_restrict_line(Ld gf, Ld gc, int lin, const dw* __restrict__ f,
                                                      dw* __restrict__ rc) {
    extern __shared__ dw tsh[];   // [fine x][column]
    const int J = blockIdx.x, K = blockIdx.y;
    int yi[4], zi[4];
    float yw[4], zw[4];
    const int nyw = rw(lin, J, gf.ny, yi, yw);
    int nzw = 1;
    zi[0] = 0; zw[0] = 1.0f;
    if (D3) nzw = rw(lin, K, gf.nz, zi, zw);
    const int nc = gf.nc, nt = gf.nx * nc;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const int x = t / nc, c = t - x * nc;
        dwacc acc = {0.0f, 0.0f};
        for (int a = 0; a < nzw; ++a)
            for (int b = 0; b < nyw; ++b)
                dwacc_add_mul_f(acc, f[(((int64_t)zi[a] * gf.ny + yi[b]) * gf.nx + x) * nc + c], zw[a] * yw[b]);
        tsh[t] = dwacc_result(acc);
    }
    __syncthreads();
    const int no = gc.nx * nc;
    const int64_t row0 = ((int64_t)K * gc.ny + J) * gc.nx;
    for (int t = threadIdx.x; t < no; t += blockDim.x) {
        const int X = t / nc, c = t - X * nc;
        int xi[4];
        float xw[4];
        const int nxw = rw(lin, X, gf.nx, xi, xw);
        dwacc acc = {0.0f, 0.0f};
        for (int q = 0; q < nxw; ++q) dwacc_add_mul_f(acc, tsh[xi[q] * nc + c], xw[q]);
        rc[(row0 + X) * nc + c] = dwacc_result(acc);
    }
}

// the line kernels keep one x-line of all columns in shared memory
constexpr size_t kLineSmemMax = 48 * 1024;

// coarsest solve, one CTA of 1024 threads per column:
// out = S diag(1/|mu_i + mu_j + mu_k - sig|) S^T in.  Each output is still one
// thread's sum in a fixed order; the transforms of one column are latency-bound.
constexpr int kTC = 1024;
__global__ void __launch_bounds__(kTC) k_coarse_sep(int d, int nx, int ny, int nz, int nc, const dw* __restrict__ Sx,
                                                   const dw* __restrict__ Sy, const dw* __restrict__ Sz,
                                                   const dw* __restrict__ mx, const dw* __restrict__ my,
                                                   const dw* __restrict__ mz, dw sig, const dw* __restrict__ in,
                                                   dw* __restrict__ out) {
    extern __shared__ dw shd[];
    const int n0 = nx * ny * nz;
    dw* a = shd;
    dw* b = shd + n0;
    const int c = blockIdx.x;
    const dw zero = dw_make(0.0f);
    for (int i = threadIdx.x; i < n0; i += blockDim.x) a[i] = in[(int64_t)i * nc + c];
    __syncthreads();
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const int m = i % nx, rest = i / nx;
        dw s = zero;
        for (int q = 0; q < nx; ++q) s = dw_add(s, dw_mul(Sx[q * nx + m], a[rest * nx + q]));
        b[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const int x = i % nx, m = (i / nx) % ny, z = i / (nx * ny);
        dw s = zero;
        for (int q = 0; q < ny; ++q) s = dw_add(s, dw_mul(Sy[q * ny + m], b[(z * ny + q) * nx + x]));
        a[i] = s;
    }
    __syncthreads();
    if (d == 3) {
        for (int i = threadIdx.x; i < n0; i += blockDim.x) {
            const int xy = i % (nx * ny), m = i / (nx * ny);
            dw s = zero;
            for (int q = 0; q < nz; ++q) s = dw_add(s, dw_mul(Sz[q * nz + m], a[q * nx * ny + xy]));
            b[i] = s;
        }
    } else {
        for (int i = threadIdx.x; i < n0; i += blockDim.x) b[i] = a[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const int ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
        dw mu = dw_add(mx[ix], my[iy]);
        if (d == 3) mu = dw_add(mu, mz[iz]);
        dw den = dw_sub(mu, sig);
        if (den.hi < 0.0f) den = dw_neg(den);
        b[i] = dw_div(b[i], den);
    }
    __syncthreads();
    if (d == 3) {
        for (int i = threadIdx.x; i < n0; i += blockDim.x) {
            const int xy = i % (nx * ny), q = i / (nx * ny);
            dw s = zero;
            for (int m = 0; m < nz; ++m) s = dw_add(s, dw_mul(Sz[q * nz + m], b[m * nx * ny + xy]));
            a[i] = s;
        }
    } else {
        for (int i = threadIdx.x; i < n0; i += blockDim.x) a[i] = b[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const int x = i % nx, q = (i / nx) % ny, z = i / (nx * ny);
        dw s = zero;
        for (int m = 0; m < ny; ++m) s = dw_add(s, dw_mul(Sy[q * ny + m], a[(z * ny + m) * nx + x]));
        b[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const int q = i % nx, rest = i / nx;
        dw s = zero;
        for (int m = 0; m < nx; ++m) s = dw_add(s, dw_mul(Sx[q * nx + m], b[rest * nx + m]));
        out[(int64_t)i * nc + c] = s;
    }
}

// dense double-word copy of an FP64 block (leading dimension ld) and back
__global__ void k_to_dw(int64_t n, int nc, const double* __restrict__ x, int64_t ldx, dw* __restrict__ y) {
    const int64_t total = n * nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t row;
        int cc;
        split_index(e, nc, row, cc);
        y[e] = dw_split_trunc(x[row * ldx + cc]);
    }
}
__global__ void k_from_dw(int64_t n, int nc, const dw* __restrict__ x, double* __restrict__ y, int64_t ldy) {
    const int64_t total = n * nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t row;
        int cc;
        split_index(e, nc, row, cc);
        y[row * ldy + cc] = dw_to_double_fast(x[e]);
    }
}

dw dw_host(double c) {
    const float hi = (float)c;
    return dw{hi, (float)(c - (double)hi)};
}
Ld ld_of(const Grid& g, int nc) { return Ld{(int)g.nx, (int)g.ny, (int)g.nz, nc, dw_host(g.inv_h2())}; }
dim3 grid_of(const Grid& g, int nc) { return dim3((unsigned)((g.nx * nc + kT - 1) / kT), (unsigned)g.ny, (unsigned)g.nz); }

struct Bufs {
    dw *w0, *w1, *tmp, *rc, *wc;
};

#define PLHR_LD(K, GR, ...)                                                        \
    do {                                                                           \
        if (d3) K<true><<<GR, kT, 0, s>>>(__VA_ARGS__);                            \
        else K<false><<<GR, kT, 0, s>>>(__VA_ARGS__);                              \
        count_launches(1);                                                         \
    } while (0)

void sweep(const MGLevel& L, dw sig, int nc, const dw* win, const dw* r, dw* tmp, dw* wout, cudaStream_t s) {
    const Ld g = ld_of(L.g, nc);
    const dim3 gr = grid_of(L.g, nc);
    const bool d3 = L.g.d == 3;
    if (!L.poly) {
        PLHR_LD(k_rich, gr, g, dw_host(L.omega), dw_host(L.omega * L.g.inv_h2()), win, r, wout);
        return;
    }
    PLHR_LD(k_shifted, gr, g, sig, win, tmp);
    PLHR_LD(k_poly, gr, g, sig, dw_host(L.c * L.c), dw_host(0.5 / L.c), dw_host(L.omega), 0, win, tmp, r, wout);
}

cudaError_t vcycle(const MGHierarchy& H, int l, int nc, const dw* r, dw* out, const std::vector<Bufs>& B,
                   cudaStream_t s) {
    if (l == 0) {
        const Grid& g0 = H.lev[0].g;
        const size_t shm = sizeof(dw) * 2 * g0.n();
        if (shm > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_coarse_sep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            if (e != cudaSuccess) return e;
        }
        const dw* b[3] = {reinterpret_cast<const dw*>(H.w_basis[0]), reinterpret_cast<const dw*>(H.w_basis[1]),
                          reinterpret_cast<const dw*>(H.w_basis[g0.d == 3 ? 2 : 1])};
        const dw* mu[3] = {reinterpret_cast<const dw*>(H.w_mu[0]), reinterpret_cast<const dw*>(H.w_mu[1]),
                           reinterpret_cast<const dw*>(H.w_mu[g0.d == 3 ? 2 : 1])};
        k_coarse_sep<<<nc, kTC, shm, s>>>(g0.d, (int)g0.nx, (int)g0.ny, (int)g0.nz, nc, b[0], b[1], b[2], mu[0], mu[1],
                                        mu[2], dw_host(H.sigma), r, out);
        count_launches(1);
        return cudaGetLastError();
    }
    const MGLevel& L = H.lev[l];
    const MGLevel& Lc = H.lev[l - 1];
    const Bufs& bf = B[l];
    const Ld g = ld_of(L.g, nc), gc = ld_of(Lc.g, nc);
    const dim3 gr = grid_of(L.g, nc), grc = grid_of(Lc.g, nc);
    const bool d3 = L.g.d == 3;
    const dw sig = dw_host(H.sigma), om = dw_host(L.omega);
    dw* cur = bf.w0;
    dw* nxt = bf.w1;
    int done;
    if (!L.poly && H.nu >= 2) {
        PLHR_LD(k_rich2, gr, g, dw_host(2.0 * L.omega), dw_host(L.omega * L.omega * L.g.inv_h2()), r, cur);
        done = 2;
    } else {
        k_scale<<<gr, kT, 0, s>>>(g, om, r, cur);
        count_launches(1);
        done = 1;
    }
    for (int i = done; i < H.nu; ++i) {
        sweep(L, sig, nc, cur, r, bf.tmp, nxt, s);
        dw* t = cur; cur = nxt; nxt = t;
    }
    if (!L.poly) {
        PLHR_LD(k_resid, gr, g, cur, r, nxt);
    } else {
        PLHR_LD(k_shifted, gr, g, sig, cur, bf.tmp);
        PLHR_LD(k_poly, gr, g, sig, dw_host(L.c * L.c), dw_host(0.5 / L.c), om, 1, cur, bf.tmp, r, nxt);
    }
    if (sizeof(dw) * L.g.nx * nc <= kLineSmemMax && Lc.g.ny <= 65535 && Lc.g.nz <= 65535) {
        const dim3 gl((unsigned)Lc.g.ny, (unsigned)Lc.g.nz);
        const size_t sh = sizeof(dw) * L.g.nx * nc;
        if (d3) k_restrict_line<true><<<gl, kT, sh, s>>>(g, gc, H.linear, nxt, bf.rc);
        else k_restrict_line<false><<<gl, kT, sh, s>>>(g, gc, H.linear, nxt, bf.rc);
        count_launches(1);
    } else {
        PLHR_LD(k_restrict, grc, g, gc, H.linear, nxt, bf.rc);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = vcycle(H, l - 1, nc, bf.rc, bf.wc, B, s);
    if (e != cudaSuccess) return e;
    if (sizeof(dw) * Lc.g.nx * nc <= kLineSmemMax && L.g.ny <= 65535 && L.g.nz <= 65535) {
        const dim3 gl((unsigned)L.g.ny, (unsigned)L.g.nz);
        const size_t sh = sizeof(dw) * Lc.g.nx * nc;
        if (d3) k_prolong_line<true><<<gl, kT, sh, s>>>(g, gc, H.linear, bf.wc, cur);
        else k_prolong_line<false><<<gl, kT, sh, s>>>(g, gc, H.linear, bf.wc, cur);
        count_launches(1);
    } else {
        PLHR_LD(k_prolong_add, gr, g, gc, H.linear, bf.wc, cur);
    }
    for (int i = 0; i < H.nu; ++i) {
        dw* dst = (i == H.nu - 1) ? out : nxt;
        sweep(L, sig, nc, cur, r, bf.tmp, dst, s);
        nxt = cur;
        cur = dst;
    }
    return cudaGetLastError();
}
#undef PLHR_LD

}  // namespace

// level buffers plus double-word copies of the right-hand side and the result,
// in units of 8-byte double-word values
int64_t mg_workspace_dw(const MGHierarchy& H, int nc) {
    int64_t tot = 2 * H.lev.back().g.n() * nc;
    for (size_t l = 1; l < H.lev.size(); ++l) tot += 3 * H.lev[l].g.n() * nc + 2 * H.lev[l - 1].g.n() * nc;
    return tot;
}

cudaError_t mg_vcycle_dw(const MGHierarchy& H, int nc, const double* r, int64_t ldr, double* w, int64_t ldw,
                         void* work_v, cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    const int top = (int)H.lev.size() - 1;
    const int64_t n = H.lev.back().g.n();
    dw* work = static_cast<dw*>(work_v);
    std::vector<Bufs> B(H.lev.size());
    dw* p = work;
    for (int l = 1; l <= top; ++l) {
        const int64_t nf = H.lev[l].g.n() * nc, ncc = H.lev[l - 1].g.n() * nc;
        B[l].w0 = p; p += nf;
        B[l].w1 = p; p += nf;
        B[l].tmp = p; p += nf;
        B[l].rc = p; p += ncc;
        B[l].wc = p; p += ncc;
    }
    dw* rdw = p; p += n * nc;
    dw* wdw = p;
    return mg_graphed(H, 2, nc, r, ldr, w, ldw, work_v, s, [&](cudaStream_t st) -> cudaError_t {
        const int blocks = grid_size_for(n * nc, 256, sm_count() * 8);
        k_to_dw<<<blocks, 256, 0, st>>>(n, nc, r, ldr, rdw);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = vcycle(H, top, nc, rdw, wdw, B, st);
        if (e != cudaSuccess) return e;
        k_from_dw<<<blocks, 256, 0, st>>>(n, nc, wdw, w, ldw);
        count_launches(1);
        return cudaGetLastError();
    });
}

}  // namespace plhr
