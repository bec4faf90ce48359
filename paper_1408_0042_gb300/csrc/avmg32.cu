// FP32 form of the absolute-value multigrid V-cycle (Appendix A, Algorithm 4):
// the same cycle as the FP64 one (B_l = L_l or p_2(L_l - sigma I), Richardson
// smoothing with omega_l = 1/beta_l, cell-centred transfers R = P^T / 2^d,
// separable exact coarsest solve), with FP32 storage and arithmetic.  T only
// has to be an approximate HPD operator, and in FP32 every level sweep is
// bound by HBM instead of GB300's FP64 pipe.
//
// Thread layout: one thread per (grid point, column) element of a block
// [point][column]; a CTA covers 256 consecutive elements of one x-line
// (blockIdx.y = y, blockIdx.z = z), so a warp reads 128 contiguous bytes and no
// 64-bit index division is needed.  The two pre-smoothing sweeps from w = 0 on
// an L_l level are fused: w = 2 omega r - omega^2 L r.
#include "plhr_internal.h"

namespace plhr {
namespace {

constexpr int kT = 256;

struct Lv {
    int nx, ny, nz, nc;
    float ih2;
};

struct Pos {
    int ix, iy, iz, c;
    int64_t row;
};

// element position of this thread on level g; false when past the line end
__device__ __forceinline__ bool pos_of(const Lv& g, Pos& p) {
    const int t = blockIdx.x * kT + threadIdx.x;
    if (t >= g.nx * g.nc) return false;
    p.ix = t / g.nc;
    p.c = t - p.ix * g.nc;
    p.iy = blockIdx.y;
    p.iz = blockIdx.z;
    p.row = ((int64_t)p.iz * g.ny + p.iy) * g.nx + p.ix;
    return true;
}

template <typename T>
__device__ __forceinline__ float ld(const T* p) { return (float)*p; }

// (2d x - sum of neighbours) at x (leading dimension ld), zero outside, as
// the sum of the differences x_c - x_nb: for a smooth field each difference is
// exact in FP32 (the operands are within a factor 2 of each other), so the
// result is correct to a few ulps of itself instead of ulps of 2d |x_c|
template <bool D3, typename T>
__device__ __forceinline__ float lap(const T* __restrict__ xp, int64_t ldx, const Lv& g, const Pos& p) {
    const float xc = ld(xp);
    const int64_t sy = ldx * g.nx, sz = sy * g.ny;
    const float dxm = p.ix > 0 ? xc - ld(xp - ldx) : xc;
    const float dxp = p.ix < g.nx - 1 ? xc - ld(xp + ldx) : xc;
    const float dym = p.iy > 0 ? xc - ld(xp - sy) : xc;
    const float dyp = p.iy < g.ny - 1 ? xc - ld(xp + sy) : xc;
    float s = (dxm + dxp) + (dym + dyp);
    if (D3) {
        const float dzm = p.iz > 0 ? xc - ld(xp - sz) : xc;
        const float dzp = p.iz < g.nz - 1 ? xc - ld(xp + sz) : xc;
        s += dzm + dzp;
    }
    return s;
}

// first two Richardson sweeps from w = 0 with B = L:  w = 2 om r - om^2 L r
template <bool D3, typename Tr>
__global__ void __launch_bounds__(kT) k_rich2(Lv g, float om, const Tr* __restrict__ r, int64_t ldr,
                                              float* __restrict__ w) {
    Pos p;
    if (!pos_of(g, p)) return;
    const Tr* rp = r + p.row * ldr + p.c;
    w[p.row * g.nc + p.c] = 2.0f * om * ld(rp) - om * om * g.ih2 * lap<D3>(rp, ldr, g, p);
}

// w = om r (one sweep from zero)
template <typename Tr>
__global__ void __launch_bounds__(kT) k_scale(Lv g, float om, const Tr* __restrict__ r, int64_t ldr,
                                              float* __restrict__ w) {
    Pos p;
    if (!pos_of(g, p)) return;
    w[p.row * g.nc + p.c] = om * ld(r + p.row * ldr + p.c);
}

// wout = win + om (r - L win)
template <bool D3, typename Tr>
__global__ void __launch_bounds__(kT) k_rich(Lv g, float om, const float* __restrict__ win, const Tr* __restrict__ r,
                                             int64_t ldr, float* __restrict__ wout) {
    Pos p;
    if (!pos_of(g, p)) return;
    const float* wp = win + p.row * g.nc + p.c;
    wout[p.row * g.nc + p.c] = wp[0] + om * (ld(r + p.row * ldr + p.c) - g.ih2 * lap<D3>(wp, g.nc, g, p));
}

// t = L x - sig x
template <bool D3>
__global__ void __launch_bounds__(kT) k_shifted(Lv g, float sig, const float* __restrict__ x, float* __restrict__ t) {
    Pos p;
    if (!pos_of(g, p)) return;
    const float* xp = x + p.row * g.nc + p.c;
    t[p.row * g.nc + p.c] = g.ih2 * lap<D3>(xp, g.nc, g, p) - sig * xp[0];
}

// with B w = ((L - sig) t + c^2 w) / (2c), t = (L - sig) w:
// mode 0: out = w + om (r - B w);  mode 1: out = r - B w
template <bool D3, typename Tr>
__global__ void __launch_bounds__(kT) k_poly(Lv g, float sig, float cpar, float om, int mode,
                                             const float* __restrict__ w, const float* __restrict__ t,
                                             const Tr* __restrict__ r, int64_t ldr, float* __restrict__ out) {
    Pos p;
    if (!pos_of(g, p)) return;
    const float* tp = t + p.row * g.nc + p.c;
    const float tt = g.ih2 * lap<D3>(tp, g.nc, g, p) - sig * tp[0];
    const float wv = w[p.row * g.nc + p.c];
    const float res = ld(r + p.row * ldr + p.c) - (tt + cpar * cpar * wv) / (2.0f * cpar);
    out[p.row * g.nc + p.c] = mode == 0 ? wv + om * res : res;
}

// out = r - L w
template <bool D3, typename Tr>
__global__ void __launch_bounds__(kT) k_resid(Lv g, const float* __restrict__ w, const Tr* __restrict__ r, int64_t ldr,
                                              float* __restrict__ out) {
    Pos p;
    if (!pos_of(g, p)) return;
    out[p.row * g.nc + p.c] =
        ld(r + p.row * ldr + p.c) - g.ih2 * lap<D3>(w + p.row * g.nc + p.c, g.nc, g, p);
}

// 1D cell-centred prolongation weights from coarse cells to fine point f:
// constant: f -> (f/2, 1);  linear: f -> (f/2, 3/4) and (f/2 -+ 1, 1/4)
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

// 1D restriction taps R = P^T / 2: coarse I gathers fine 2I, 2I+1 (1/2 each,
// constant) or 2I, 2I+1 (3/8) and 2I-1, 2I+2 (1/8, linear)
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

// wf += P wc   (launched over the fine level)
template <bool D3>
__global__ void __launch_bounds__(kT) k_prolong_add(Lv gf, Lv gc, int lin, const float* __restrict__ wc,
                                                    float* __restrict__ wf) {
    Pos p;
    if (!pos_of(gf, p)) return;
    int xi[2], yi[2], zi[2];
    float xw[2], yw[2], zw[2];
    const int nxw = pw(lin, p.ix, gc.nx, xi, xw);
    const int nyw = pw(lin, p.iy, gc.ny, yi, yw);
    int nzw = 1;
    zi[0] = 0; zw[0] = 1.0f;
    if (D3) nzw = pw(lin, p.iz, gc.nz, zi, zw);
    float s = 0.0f;
    for (int a = 0; a < nzw; ++a)
        for (int b = 0; b < nyw; ++b) {
            const float* line = wc + ((int64_t)zi[a] * gc.ny + yi[b]) * gc.nx * gc.nc + p.c;
            float sl = 0.0f;
            for (int q = 0; q < nxw; ++q) sl += xw[q] * line[(int64_t)xi[q] * gc.nc];
            s += zw[a] * yw[b] * sl;
        }
    wf[p.row * gf.nc + p.c] += s;
}

// rc = R f   (launched over the coarse level)
template <bool D3>
__global__ void __launch_bounds__(kT) k_restrict(Lv gf, Lv gc, int lin, const float* __restrict__ f,
                                                 float* __restrict__ rc) {
    Pos p;
    if (!pos_of(gc, p)) return;
    int xi[4], yi[4], zi[4];
    float xw[4], yw[4], zw[4];
    const int nxw = rw(lin, p.ix, gf.nx, xi, xw);
    const int nyw = rw(lin, p.iy, gf.ny, yi, yw);
    int nzw = 1;
    zi[0] = 0; zw[0] = 1.0f;
    if (D3) nzw = rw(lin, p.iz, gf.nz, zi, zw);
    float s = 0.0f;
    for (int a = 0; a < nzw; ++a)
        for (int b = 0; b < nyw; ++b) {
            const float* line = f + ((int64_t)zi[a] * gf.ny + yi[b]) * gf.nx * gf.nc + p.c;
            float sl = 0.0f;
            for (int q = 0; q < nxw; ++q) sl += xw[q] * line[(int64_t)xi[q] * gf.nc];
            s += zw[a] * yw[b] * sl;
        }
    rc[p.row * gc.nc + p.c] = s;
}

// Coarsest solve, one CTA per column: out = S diag(1/|mu_i + mu_j + mu_k - sig|) S^T in,
// S = Sx (x) Sy (x) Sz, applied one axis at a time through shared memory.
template <typename Tr>
__global__ void __launch_bounds__(kT) k_coarse_sep(int d, int nx, int ny, int nz, int nc, const float* __restrict__ Sx,
                                                   const float* __restrict__ Sy, const float* __restrict__ Sz,
                                                   const float* __restrict__ mx, const float* __restrict__ my,
                                                   const float* __restrict__ mz, float sig,
                                                   const Tr* __restrict__ in, int64_t ldi, float* __restrict__ out) {
    extern __shared__ float shf[];
    const int n0 = nx * ny * nz;
    float* a = shf;
    float* b = shf + n0;
    const int c = blockIdx.x;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) a[i] = ld(in + (int64_t)i * ldi + c);
    __syncthreads();
    // forward transform: coef[mode] = sum_point S[point][mode] x[point], per axis
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const int m = i % nx, rest = i / nx;
        float s = 0.0f;
        for (int q = 0; q < nx; ++q) s += Sx[q * nx + m] * a[rest * nx + q];
        b[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const int x = i % nx, m = (i / nx) % ny, z = i / (nx * ny);
        float s = 0.0f;
        for (int q = 0; q < ny; ++q) s += Sy[q * ny + m] * b[(z * ny + q) * nx + x];
        a[i] = s;
    }
    __syncthreads();
    if (d == 3) {
        for (int i = threadIdx.x; i < n0; i += blockDim.x) {
            const int xy = i % (nx * ny), m = i / (nx * ny);
            float s = 0.0f;
            for (int q = 0; q < nz; ++q) s += Sz[q * nz + m] * a[q * nx * ny + xy];
            b[i] = s;
        }
    } else {
        for (int i = threadIdx.x; i < n0; i += blockDim.x) b[i] = a[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const int ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
        const float mu = mx[ix] + my[iy] + (d == 3 ? mz[iz] : 0.0f);
        b[i] = b[i] / fabsf(mu - sig);
    }
    __syncthreads();
    // inverse transform: x[point] = sum_mode S[point][mode] coef[mode]
    if (d == 3) {
        for (int i = threadIdx.x; i < n0; i += blockDim.x) {
            const int xy = i % (nx * ny), q = i / (nx * ny);
            float s = 0.0f;
            for (int m = 0; m < nz; ++m) s += Sz[q * nz + m] * b[m * nx * ny + xy];
            a[i] = s;
        }
    } else {
        for (int i = threadIdx.x; i < n0; i += blockDim.x) a[i] = b[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const int x = i % nx, q = (i / nx) % ny, z = i / (nx * ny);
        float s = 0.0f;
        for (int m = 0; m < ny; ++m) s += Sy[q * ny + m] * a[(z * ny + m) * nx + x];
        b[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const int q = i % nx, rest = i / nx;
        float s = 0.0f;
        for (int m = 0; m < nx; ++m) s += Sx[q * nx + m] * b[rest * nx + m];
        out[(int64_t)i * nc + c] = s;
    }
}

Lv lv(const Grid& g, int nc) { return Lv{(int)g.nx, (int)g.ny, (int)g.nz, nc, (float)g.inv_h2()}; }
dim3 grid_of(const Grid& g, int nc) { return dim3((unsigned)((g.nx * nc + kT - 1) / kT), (unsigned)g.ny, (unsigned)g.nz); }

struct Bufs {
    float *w0, *w1, *tmp, *rc, *wc;
};

template <typename Tr>
cudaError_t coarse(const MGHierarchy& H, int nc, const Tr* r, int64_t ldr, float* out, cudaStream_t s) {
    const Grid& g = H.lev[0].g;
    const size_t shm = sizeof(float) * 2 * g.n();
    if (shm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_coarse_sep<Tr>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e != cudaSuccess) return e;
    }
    k_coarse_sep<Tr><<<nc, kT, shm, s>>>(g.d, (int)g.nx, (int)g.ny, (int)g.nz, nc, H.f_basis[0], H.f_basis[1],
                                        g.d == 3 ? H.f_basis[2] : H.f_basis[1], H.f_mu[0], H.f_mu[1],
                                        g.d == 3 ? H.f_mu[2] : H.f_mu[1], (float)H.sigma, r, ldr, out);
    count_launches(1);
    return cudaGetLastError();
}

// one smoothing sweep w_out = w_in + om (r - B w_in) on level L
template <typename Tr>
void sweep(const MGLevel& L, float sig, int nc, const float* win, const Tr* r, int64_t ldr, float* tmp, float* wout,
           cudaStream_t s) {
    const Lv g = lv(L.g, nc);
    const dim3 gr = grid_of(L.g, nc);
    const bool d3 = L.g.d == 3;
    if (!L.poly) {
        if (d3) k_rich<true, Tr><<<gr, kT, 0, s>>>(g, (float)L.omega, win, r, ldr, wout);
        else k_rich<false, Tr><<<gr, kT, 0, s>>>(g, (float)L.omega, win, r, ldr, wout);
        count_launches(1);
        return;
    }
    if (d3) k_shifted<true><<<gr, kT, 0, s>>>(g, sig, win, tmp);
    else k_shifted<false><<<gr, kT, 0, s>>>(g, sig, win, tmp);
    if (d3) k_poly<true, Tr><<<gr, kT, 0, s>>>(g, sig, (float)L.c, (float)L.omega, 0, win, tmp, r, ldr, wout);
    else k_poly<false, Tr><<<gr, kT, 0, s>>>(g, sig, (float)L.c, (float)L.omega, 0, win, tmp, r, ldr, wout);
    count_launches(2);
}

template <typename Tr>
cudaError_t vcycle(const MGHierarchy& H, int l, int nc, const Tr* r, int64_t ldr, float* out,
                   const std::vector<Bufs>& B, cudaStream_t s) {
    if (l == 0) return coarse(H, nc, r, ldr, out, s);
    const MGLevel& L = H.lev[l];
    const MGLevel& Lc = H.lev[l - 1];
    const Bufs& b = B[l];
    const Lv g = lv(L.g, nc), gc = lv(Lc.g, nc);
    const dim3 gr = grid_of(L.g, nc), grc = grid_of(Lc.g, nc);
    const bool d3 = L.g.d == 3;
    const float sig = (float)H.sigma, om = (float)L.omega;
    float* cur = b.w0;
    float* nxt = b.w1;
    // pre-smoothing from w = 0
    int done;
    if (!L.poly && H.nu >= 2) {
        if (d3) k_rich2<true, Tr><<<gr, kT, 0, s>>>(g, om, r, ldr, cur);
        else k_rich2<false, Tr><<<gr, kT, 0, s>>>(g, om, r, ldr, cur);
        done = 2;
    } else {
        k_scale<Tr><<<gr, kT, 0, s>>>(g, om, r, ldr, cur);
        done = 1;
    }
    count_launches(1);
    for (int i = done; i < H.nu; ++i) {
        sweep(L, sig, nc, cur, r, ldr, b.tmp, nxt, s);
        float* t = cur; cur = nxt; nxt = t;
    }
    // coarse-grid correction: r_c = R (r - B w)
    if (!L.poly) {
        if (d3) k_resid<true, Tr><<<gr, kT, 0, s>>>(g, cur, r, ldr, nxt);
        else k_resid<false, Tr><<<gr, kT, 0, s>>>(g, cur, r, ldr, nxt);
        count_launches(1);
    } else {
        if (d3) k_shifted<true><<<gr, kT, 0, s>>>(g, sig, cur, b.tmp);
        else k_shifted<false><<<gr, kT, 0, s>>>(g, sig, cur, b.tmp);
        if (d3) k_poly<true, Tr><<<gr, kT, 0, s>>>(g, sig, (float)L.c, om, 1, cur, b.tmp, r, ldr, nxt);
        else k_poly<false, Tr><<<gr, kT, 0, s>>>(g, sig, (float)L.c, om, 1, cur, b.tmp, r, ldr, nxt);
        count_launches(2);
    }
    if (d3) k_restrict<true><<<grc, kT, 0, s>>>(g, gc, H.linear, nxt, b.rc);
    else k_restrict<false><<<grc, kT, 0, s>>>(g, gc, H.linear, nxt, b.rc);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = vcycle<float>(H, l - 1, nc, b.rc, nc, b.wc, B, s);
    if (e != cudaSuccess) return e;
    if (d3) k_prolong_add<true><<<gr, kT, 0, s>>>(g, gc, H.linear, b.wc, cur);
    else k_prolong_add<false><<<gr, kT, 0, s>>>(g, gc, H.linear, b.wc, cur);
    count_launches(1);
    // post-smoothing; the last sweep writes out
    for (int i = 0; i < H.nu; ++i) {
        float* dst = (i == H.nu - 1) ? out : nxt;
        sweep(L, sig, nc, cur, r, ldr, b.tmp, dst, s);
        nxt = cur;
        cur = dst;
    }
    return cudaGetLastError();
}

template <typename Tr>
cudaError_t run(const MGHierarchy& H, int nc, const Tr* r, int64_t ldr, float* w, float* work, cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    const int top = (int)H.lev.size() - 1;
    std::vector<Bufs> B(H.lev.size());
    float* p = work;
    for (int l = 1; l <= top; ++l) {
        const int64_t nf = H.lev[l].g.n() * nc, ncc = H.lev[l - 1].g.n() * nc;
        B[l].w0 = p; p += nf;
        B[l].w1 = p; p += nf;
        B[l].tmp = p; p += nf;
        B[l].rc = p; p += ncc;
        B[l].wc = p; p += ncc;
    }
    return vcycle<Tr>(H, top, nc, r, ldr, w, B, s);
}

}  // namespace

int64_t mg_workspace_floats(const MGHierarchy& H, int nc) {
    int64_t tot = 0;
    for (size_t l = 1; l < H.lev.size(); ++l) tot += 3 * H.lev[l].g.n() * nc + 2 * H.lev[l - 1].g.n() * nc;
    return tot;
}

cudaError_t mg_vcycle_f32(const MGHierarchy& H, int nc, const double* r, int64_t ldr, float* w, float* work,
                          cudaStream_t s) {
    return run<double>(H, nc, r, ldr, w, work, s);
}

cudaError_t mg_vcycle_f32(const MGHierarchy& H, int nc, const float* r, int64_t ldr, float* w, float* work,
                          cudaStream_t s) {
    return run<float>(H, nc, r, ldr, w, work, s);
}

}  // namespace plhr
