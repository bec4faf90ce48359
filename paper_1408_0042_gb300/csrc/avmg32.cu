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
#include "dword.h"
#include "plhr_internal.h"

namespace plhr {
namespace {

constexpr int kT = 256;

struct Lv {
    int nx, ny, nz, nc;
    float ih2;
    int nq;          // column groups per grid point (nc / VW)
    float inv_nq;    // 1 / nq
};

struct Pos {
    int ix, iy, iz, c;
    int64_t row;
};

// Element group of this thread on level g: VW consecutive columns c.. of one
// grid point; false past the line end.  ix = floor(t / nq) through a float
// reciprocal: t < 2^12 and nq <= 32 keep (t + 1/2) / nq at least 1/64 away
// from an integer, far above the rounding error.
template <int VW>
__device__ __forceinline__ bool pos_of(const Lv& g, Pos& p) {
    const int t = blockIdx.x * kT + threadIdx.x;
    if (t >= g.nx * g.nq) return false;
    p.ix = (int)(((float)t + 0.5f) * g.inv_nq);
    p.c = (t - p.ix * g.nq) * VW;
    p.iy = blockIdx.y;
    p.iz = blockIdx.z;
    p.row = ((int64_t)p.iz * g.ny + p.iy) * g.nx + p.ix;
    return true;
}

template <typename T>
__device__ __forceinline__ float ld(const T* p) { return (float)*p; }

// VW consecutive values (16-byte loads and stores when VW = 4)
template <int VW>
__device__ __forceinline__ void vld(float* o, const float* p) {
    if (VW == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else {
#pragma unroll
        for (int q = 0; q < VW; ++q) o[q] = p[q];
    }
}
template <int VW>
__device__ __forceinline__ void vld(float* o, const double* p) {
    if (VW == 4) {
        const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
        o[0] = (float)a.x; o[1] = (float)a.y; o[2] = (float)b.x; o[3] = (float)b.y;
    } else {
#pragma unroll
        for (int q = 0; q < VW; ++q) o[q] = (float)p[q];
    }
}
template <int VW>
__device__ __forceinline__ void vst(float* p, const float* v) {
    if (VW == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int q = 0; q < VW; ++q) p[q] = v[q];
    }
}

// L x at (p, columns c..c+VW) with leading dimension ld, zero outside, as the
// sum of the differences x_c - x_nb: for a smooth field each difference is
// exact in FP32 (the operands are within a factor 2 of each other), so the
// result is correct to a few ulps of itself instead of ulps of 2d |x_c|.
// xc receives x itself.
template <bool D3, int VW, typename T>
__device__ __forceinline__ void lap(float* out, float* xc, const T* __restrict__ xp, int64_t ldx, const Lv& g,
                                    const Pos& p) {
    const int64_t sy = ldx * g.nx, sz = sy * g.ny;
    float nb[VW];
    vld<VW>(xc, xp);
    float s[VW];
#pragma unroll
    for (int q = 0; q < VW; ++q) s[q] = 0.0f;
    auto add_dir = [&](bool in, int64_t off) {
        if (in) {
            vld<VW>(nb, xp + off);
#pragma unroll
            for (int q = 0; q < VW; ++q) s[q] += xc[q] - nb[q];
        } else {
#pragma unroll
            for (int q = 0; q < VW; ++q) s[q] += xc[q];
        }
    };
    float sx[VW];
    add_dir(p.ix > 0, -ldx);
    add_dir(p.ix < g.nx - 1, ldx);
#pragma unroll
    for (int q = 0; q < VW; ++q) { sx[q] = s[q]; s[q] = 0.0f; }
    add_dir(p.iy > 0, -sy);
    add_dir(p.iy < g.ny - 1, sy);
    if (D3) {
        float sxy[VW];
#pragma unroll
        for (int q = 0; q < VW; ++q) { sxy[q] = sx[q] + s[q]; s[q] = 0.0f; }
        add_dir(p.iz > 0, -sz);
        add_dir(p.iz < g.nz - 1, sz);
#pragma unroll
        for (int q = 0; q < VW; ++q) out[q] = sxy[q] + s[q];
    } else {
#pragma unroll
        for (int q = 0; q < VW; ++q) out[q] = sx[q] + s[q];
    }
}

// first two Richardson sweeps from w = 0 with B = L:  w = 2 om r - om^2 L r
template <bool D3, int VW, typename Tr>
__global__ void __launch_bounds__(kT) k_rich2(Lv g, float om, const Tr* __restrict__ r, int64_t ldr,
                                              float* __restrict__ w) {
    Pos p;
    if (!pos_of<VW>(g, p)) return;
    float l[VW], rc[VW], o[VW];
    lap<D3, VW>(l, rc, r + p.row * ldr + p.c, ldr, g, p);
#pragma unroll
    for (int q = 0; q < VW; ++q) o[q] = 2.0f * om * rc[q] - om * om * g.ih2 * l[q];
    vst<VW>(w + p.row * g.nc + p.c, o);
}

// w = om r (one sweep from zero)
template <bool D3, int VW, typename Tr>
__global__ void __launch_bounds__(kT) k_scale(Lv g, float om, const Tr* __restrict__ r, int64_t ldr,
                                              float* __restrict__ w) {
    Pos p;
    if (!pos_of<VW>(g, p)) return;
    float rv[VW];
    vld<VW>(rv, r + p.row * ldr + p.c);
#pragma unroll
    for (int q = 0; q < VW; ++q) rv[q] *= om;
    vst<VW>(w + p.row * g.nc + p.c, rv);
}

// wout = win + om (r - L win)
template <bool D3, int VW, typename Tr>
__global__ void __launch_bounds__(kT) k_rich(Lv g, float om, const float* __restrict__ win, const Tr* __restrict__ r,
                                             int64_t ldr, float* __restrict__ wout) {
    Pos p;
    if (!pos_of<VW>(g, p)) return;
    float l[VW], wc[VW], rv[VW];
    lap<D3, VW>(l, wc, win + p.row * g.nc + p.c, g.nc, g, p);
    vld<VW>(rv, r + p.row * ldr + p.c);
#pragma unroll
    for (int q = 0; q < VW; ++q) wc[q] += om * (rv[q] - g.ih2 * l[q]);
    vst<VW>(wout + p.row * g.nc + p.c, wc);
}

// t = L x - sig x
template <bool D3, int VW, typename Tr>
__global__ void __launch_bounds__(kT) k_shifted(Lv g, float sig, const float* __restrict__ x, float* __restrict__ t) {
    Pos p;
    if (!pos_of<VW>(g, p)) return;
    float l[VW], xc[VW];
    lap<D3, VW>(l, xc, x + p.row * g.nc + p.c, g.nc, g, p);
#pragma unroll
    for (int q = 0; q < VW; ++q) l[q] = g.ih2 * l[q] - sig * xc[q];
    vst<VW>(t + p.row * g.nc + p.c, l);
}

// with B w = ((L - sig) t + c^2 w) / (2c), t = (L - sig) w:
// mode 0: out = w + om (r - B w);  mode 1: out = r - B w
template <bool D3, int VW, typename Tr>
__global__ void __launch_bounds__(kT) k_poly(Lv g, float sig, float cpar, float om, int mode,
                                             const float* __restrict__ w, const float* __restrict__ t,
                                             const Tr* __restrict__ r, int64_t ldr, float* __restrict__ out) {
    Pos p;
    if (!pos_of<VW>(g, p)) return;
    float l[VW], tc[VW], wv[VW], rv[VW];
    lap<D3, VW>(l, tc, t + p.row * g.nc + p.c, g.nc, g, p);
    vld<VW>(wv, w + p.row * g.nc + p.c);
    vld<VW>(rv, r + p.row * ldr + p.c);
#pragma unroll
    for (int q = 0; q < VW; ++q) {
        const float tt = g.ih2 * l[q] - sig * tc[q];
        const float res = rv[q] - (tt + cpar * cpar * wv[q]) / (2.0f * cpar);
        rv[q] = mode == 0 ? wv[q] + om * res : res;
    }
    vst<VW>(out + p.row * g.nc + p.c, rv);
}

// out = r - L w
template <bool D3, int VW, typename Tr>
__global__ void __launch_bounds__(kT) k_resid(Lv g, const float* __restrict__ w, const Tr* __restrict__ r, int64_t ldr,
                                              float* __restrict__ out) {
    Pos p;
    if (!pos_of<VW>(g, p)) return;
    float l[VW], wc[VW], rv[VW];
    lap<D3, VW>(l, wc, w + p.row * g.nc + p.c, g.nc, g, p);
    vld<VW>(rv, r + p.row * ldr + p.c);
#pragma unroll
    for (int q = 0; q < VW; ++q) rv[q] -= g.ih2 * l[q];
    vst<VW>(out + p.row * g.nc + p.c, rv);
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
template <bool D3, int VW, typename Tr>
__global__ void __launch_bounds__(kT) k_prolong_add(Lv gf, Lv gc, int lin, const float* __restrict__ wc,
                                                    float* __restrict__ wf) {
    Pos p;
    if (!pos_of<VW>(gf, p)) return;
    int xi[2], yi[2], zi[2];
    float xw[2], yw[2], zw[2];
    const int nxw = pw(lin, p.ix, gc.nx, xi, xw);
    const int nyw = pw(lin, p.iy, gc.ny, yi, yw);
    int nzw = 1;
    zi[0] = 0; zw[0] = 1.0f;
    if (D3) nzw = pw(lin, p.iz, gc.nz, zi, zw);
    float acc[VW], v[VW];
    vld<VW>(acc, wf + p.row * gf.nc + p.c);
    for (int a = 0; a < nzw; ++a)
        for (int b = 0; b < nyw; ++b) {
            const float* line = wc + ((int64_t)zi[a] * gc.ny + yi[b]) * gc.nx * gc.nc + p.c;
            const float wyz = zw[a] * yw[b];
            for (int q = 0; q < nxw; ++q) {
                vld<VW>(v, line + (int64_t)xi[q] * gc.nc);
                const float wt = wyz * xw[q];
#pragma unroll
                for (int e = 0; e < VW; ++e) acc[e] += wt * v[e];
            }
        }
    vst<VW>(wf + p.row * gf.nc + p.c, acc);
}

// rc = R f   (launched over the coarse level)
template <bool D3, int VW, typename Tr>
__global__ void __launch_bounds__(kT) k_restrict(Lv gf, Lv gc, int lin, const float* __restrict__ f,
                                                 float* __restrict__ rc) {
    Pos p;
    if (!pos_of<VW>(gc, p)) return;
    int xi[4], yi[4], zi[4];
    float xw[4], yw[4], zw[4];
    const int nxw = rw(lin, p.ix, gf.nx, xi, xw);
    const int nyw = rw(lin, p.iy, gf.ny, yi, yw);
    int nzw = 1;
    zi[0] = 0; zw[0] = 1.0f;
    if (D3) nzw = rw(lin, p.iz, gf.nz, zi, zw);
    float acc[VW], v[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) acc[e] = 0.0f;
    for (int a = 0; a < nzw; ++a)
        for (int b = 0; b < nyw; ++b) {
            const float* line = f + ((int64_t)zi[a] * gf.ny + yi[b]) * gf.nx * gf.nc + p.c;
            const float wyz = zw[a] * yw[b];
            for (int q = 0; q < nxw; ++q) {
                vld<VW>(v, line + (int64_t)xi[q] * gf.nc);
                const float wt = wyz * xw[q];
#pragma unroll
                for (int e = 0; e < VW; ++e) acc[e] += wt * v[e];
            }
        }
    vst<VW>(rc + p.row * gc.nc + p.c, acc);
}

// The transfers one grid line per CTA, separably (as in the double-word
// form): the y-z interpolation (prolongation) or y-z sums (restriction) of
// one line of all columns go to shared memory, then the x taps.  VW
// consecutive columns per thread.
template <bool D3, int VW>
__global__ void __launch_bounds__(kT) k_prolong_line(Lv gf, Lv gc, int lin, const float* __restrict__ wc,
                                                     float* __restrict__ wf) {
    extern __shared__ float ush32[];   // [coarse x][column]
    const int iy = blockIdx.x, iz = blockIdx.y;
    int yi[2], zi[2];
    float yw[2], zw[2];
    const int nyw = pw(lin, iy, gc.ny, yi, yw);
    int nzw = 1;
    zi[0] = 0; zw[0] = 1.0f;
    if (D3) nzw = pw(lin, iz, gc.nz, zi, zw);
    const int nc = gf.nc, nq = gf.nq;
    float acc[VW], v[VW];
    for (int t = threadIdx.x; t < gc.nx * nq; t += blockDim.x) {
        const int X = t / nq, c = (t - X * nq) * VW;
#pragma unroll
        for (int e = 0; e < VW; ++e) acc[e] = 0.0f;
        for (int a = 0; a < nzw; ++a)
            for (int b = 0; b < nyw; ++b) {
                vld<VW>(v, wc + (((int64_t)zi[a] * gc.ny + yi[b]) * gc.nx + X) * nc + c);
                const float wt = zw[a] * yw[b];
#pragma unroll
                for (int e = 0; e < VW; ++e) acc[e] += wt * v[e];
            }
        vst<VW>(ush32 + X * nc + c, acc);
    }
    __syncthreads();
    const int64_t row0 = ((int64_t)iz * gf.ny + iy) * gf.nx;
    for (int t = threadIdx.x; t < gf.nx * nq; t += blockDim.x) {
        const int x = t / nq, c = (t - x * nq) * VW;
        int xi[2];
        float xw[2];
        const int nxw = pw(lin, x, gc.nx, xi, xw);
        float* dst = wf + (row0 + x) * nc + c;
        vld<VW>(acc, dst);
        for (int q = 0; q < nxw; ++q) {
            vld<VW>(v, ush32 + xi[q] * nc + c);
#pragma unroll
            for (int e = 0; e < VW; ++e) acc[e] += xw[q] * v[e];
        }
        vst<VW>(dst, acc);
    }
}

template <bool D3, int VW>
__global__ void __launch_bounds__(kT) k_restrict_line(Lv gf, Lv gc, int lin, const float* __restrict__ f,
                                                      float* __restrict__ rc) {
    extern __shared__ float tsh32[];   // [fine x][column]
    const int J = blockIdx.x, K = blockIdx.y;
    int yi[4], zi[4];
    float yw[4], zw[4];
    const int nyw = rw(lin, J, gf.ny, yi, yw);
    int nzw = 1;
    zi[0] = 0; zw[0] = 1.0f;
    if (D3) nzw = rw(lin, K, gf.nz, zi, zw);
    const int nc = gf.nc, nq = gf.nq;
    float acc[VW], v[VW];
    for (int t = threadIdx.x; t < gf.nx * nq; t += blockDim.x) {
        const int x = t / nq, c = (t - x * nq) * VW;
#pragma unroll
        for (int e = 0; e < VW; ++e) acc[e] = 0.0f;
        for (int a = 0; a < nzw; ++a)
            for (int b = 0; b < nyw; ++b) {
                vld<VW>(v, f + (((int64_t)zi[a] * gf.ny + yi[b]) * gf.nx + x) * nc + c);
                const float wt = zw[a] * yw[b];
#pragma unroll
                for (int e = 0; e < VW; ++e) acc[e] += wt * v[e];
            }
        vst<VW>(tsh32 + x * nc + c, acc);
    }
    __syncthreads();
    const int64_t row0 = ((int64_t)K * gc.ny + J) * gc.nx;
    for (int t = threadIdx.x; t < gc.nx * nq; t += blockDim.x) {
        const int X = t / nq, c = (t - X * nq) * VW;
        int xi[4];
        float xw[4];
        const int nxw = rw(lin, X, gf.nx, xi, xw);
#pragma unroll
        for (int e = 0; e < VW; ++e) acc[e] = 0.0f;
        for (int q = 0; q < nxw; ++q) {
            vld<VW>(v, tsh32 + xi[q] * nc + c);
#pragma unroll
            for (int e = 0; e < VW; ++e) acc[e] += xw[q] * v[e];
        }
        vst<VW>(rc + (row0 + X) * nc + c, acc);
    }
}

// the line kernels keep one x-line of all columns in shared memory
constexpr size_t kLineSmemMax = 48 * 1024;

// Coarsest solve, one CTA per column: out = S diag(1/|mu_i + mu_j + mu_k - sig|) S^T in,
// S = Sx (x) Sy (x) Sz, applied one axis at a time through shared memory.
// coarsest level: 1024 threads per column (each output is still one thread's
// sum in a fixed order); the transforms of one column are latency-bound
constexpr int kTC = 1024;
template <typename Tr>
__global__ void __launch_bounds__(kTC) k_coarse_sep(int d, int nx, int ny, int nz, int nc, const float* __restrict__ Sx,
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

Lv lv(const Grid& g, int nc, int vw) {
    const int nq = nc / vw;
    return Lv{(int)g.nx, (int)g.ny, (int)g.nz, nc, (float)g.inv_h2(), nq, 1.0f / (float)nq};
}
dim3 grid_of(const Grid& g, int nc, int vw) {
    return dim3((unsigned)((g.nx * (nc / vw) + kT - 1) / kT), (unsigned)g.ny, (unsigned)g.nz);
}

// launch K<D3, VW, TR> on grid GR for the level of this call
#define PLHR_L4(K, TR, GR, ...)                                                         \
    do {                                                                                   \
        if (d3) {                                                                          \
            if (v4) K<true, 4, TR><<<GR, kT, 0, s>>>(__VA_ARGS__);                       \
            else K<true, 1, TR><<<GR, kT, 0, s>>>(__VA_ARGS__);                          \
        } else {                                                                           \
            if (v4) K<false, 4, TR><<<GR, kT, 0, s>>>(__VA_ARGS__);                      \
            else K<false, 1, TR><<<GR, kT, 0, s>>>(__VA_ARGS__);                         \
        }                                                                                  \
        count_launches(1);                                                                 \
    } while (0)

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
    k_coarse_sep<Tr><<<nc, kTC, shm, s>>>(g.d, (int)g.nx, (int)g.ny, (int)g.nz, nc, H.f_basis[0], H.f_basis[1],
                                        g.d == 3 ? H.f_basis[2] : H.f_basis[1], H.f_mu[0], H.f_mu[1],
                                        g.d == 3 ? H.f_mu[2] : H.f_mu[1], (float)H.sigma, r, ldr, out);
    count_launches(1);
    return cudaGetLastError();
}

// one smoothing sweep w_out = w_in + om (r - B w_in) on level L
template <typename Tr>
void sweep(const MGLevel& L, float sig, int nc, bool v4, const float* win, const Tr* r, int64_t ldr, float* tmp,
           float* wout, cudaStream_t s) {
    const Lv g = lv(L.g, nc, v4 ? 4 : 1);
    const dim3 gr = grid_of(L.g, nc, v4 ? 4 : 1);
    const bool d3 = L.g.d == 3;
    if (!L.poly) {
        PLHR_L4(k_rich, Tr, gr, g, (float)L.omega, win, r, ldr, wout);
        return;
    }
    PLHR_L4(k_shifted, Tr, gr, g, sig, win, tmp);
    PLHR_L4(k_poly, Tr, gr, g, sig, (float)L.c, (float)L.omega, 0, win, tmp, r, ldr, wout);
}

template <typename Tr>
cudaError_t vcycle(const MGHierarchy& H, int l, int nc, bool v4, const Tr* r, int64_t ldr, float* out,
                   const std::vector<Bufs>& B, cudaStream_t s) {
    if (l == 0) return coarse(H, nc, r, ldr, out, s);
    const MGLevel& L = H.lev[l];
    const MGLevel& Lc = H.lev[l - 1];
    const Bufs& b = B[l];
    const int vw = v4 ? 4 : 1;
    const Lv g = lv(L.g, nc, vw), gc = lv(Lc.g, nc, vw);
    const dim3 gr = grid_of(L.g, nc, vw), grc = grid_of(Lc.g, nc, vw);
    const bool d3 = L.g.d == 3;
    const float sig = (float)H.sigma, om = (float)L.omega;
    float* cur = b.w0;
    float* nxt = b.w1;
    // pre-smoothing from w = 0
    int done;
    if (!L.poly && H.nu >= 2) {
        PLHR_L4(k_rich2, Tr, gr, g, om, r, ldr, cur);
        done = 2;
    } else {
        PLHR_L4(k_scale, Tr, gr, g, om, r, ldr, cur);
        done = 1;
    }
    for (int i = done; i < H.nu; ++i) {
        sweep(L, sig, nc, v4, cur, r, ldr, b.tmp, nxt, s);
        float* t = cur; cur = nxt; nxt = t;
    }
    // coarse-grid correction: r_c = R (r - B w)
    if (!L.poly) {
        PLHR_L4(k_resid, Tr, gr, g, cur, r, ldr, nxt);
    } else {
        PLHR_L4(k_shifted, Tr, gr, g, sig, cur, b.tmp);
        PLHR_L4(k_poly, Tr, gr, g, sig, (float)L.c, om, 1, cur, b.tmp, r, ldr, nxt);
    }
    if (sizeof(float) * L.g.nx * nc <= kLineSmemMax && Lc.g.ny <= 65535 && Lc.g.nz <= 65535) {
        const dim3 gl((unsigned)Lc.g.ny, (unsigned)Lc.g.nz);
        const size_t sh = sizeof(float) * L.g.nx * nc;
        if (d3) {
            if (v4) k_restrict_line<true, 4><<<gl, kT, sh, s>>>(g, gc, H.linear, nxt, b.rc);
            else k_restrict_line<true, 1><<<gl, kT, sh, s>>>(g, gc, H.linear, nxt, b.rc);
        } else {
            if (v4) k_restrict_line<false, 4><<<gl, kT, sh, s>>>(g, gc, H.linear, nxt, b.rc);
            else k_restrict_line<false, 1><<<gl, kT, sh, s>>>(g, gc, H.linear, nxt, b.rc);
        }
        count_launches(1);
    } else {
        PLHR_L4(k_restrict, float, grc, g, gc, H.linear, nxt, b.rc);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = vcycle<float>(H, l - 1, nc, v4, b.rc, nc, b.wc, B, s);
    if (e != cudaSuccess) return e;
    if (sizeof(float) * Lc.g.nx * nc <= kLineSmemMax && L.g.ny <= 65535 && L.g.nz <= 65535) {
        const dim3 gl((unsigned)L.g.ny, (unsigned)L.g.nz);
        const size_t sh = sizeof(float) * Lc.g.nx * nc;
        if (d3) {
            if (v4) k_prolong_line<true, 4><<<gl, kT, sh, s>>>(g, gc, H.linear, b.wc, cur);
            else k_prolong_line<true, 1><<<gl, kT, sh, s>>>(g, gc, H.linear, b.wc, cur);
        } else {
            if (v4) k_prolong_line<false, 4><<<gl, kT, sh, s>>>(g, gc, H.linear, b.wc, cur);
            else k_prolong_line<false, 1><<<gl, kT, sh, s>>>(g, gc, H.linear, b.wc, cur);
        }
        count_launches(1);
    } else {
        PLHR_L4(k_prolong_add, float, gr, g, gc, H.linear, b.wc, cur);
    }
    // post-smoothing; the last sweep writes out
    for (int i = 0; i < H.nu; ++i) {
        float* dst = (i == H.nu - 1) ? out : nxt;
        sweep(L, sig, nc, v4, cur, r, ldr, b.tmp, dst, s);
        nxt = cur;
        cur = dst;
    }
    return cudaGetLastError();
}
#undef PLHR_L4

// r32 (n x nc, leading dimension ldo) = r (FP64, leading dimension ldr)
__global__ void k_narrow_rhs(int64_t n, int nc, const double* __restrict__ r, int64_t ldr, float* __restrict__ r32,
                             int64_t ldo) {
    const int64_t total = n * nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t row;
        int cc;
        split_index(e, nc, row, cc);
        r32[row * ldo + cc] = f64_to_f32_rn(r[row * ldr + cc]);
    }
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
    // four columns per thread with 16-byte accesses when every block allows it
    auto al16 = [](const void* q) { return ((uintptr_t)q & 15) == 0; };
    const bool v4 = nc % 4 == 0 && ldr % 4 == 0 && al16(r) && al16(w) && al16(work);
    return vcycle<Tr>(H, top, nc, v4, r, ldr, w, B, s);
}

}  // namespace

int64_t mg_workspace_floats(const MGHierarchy& H, int nc) {
    // level buffers, plus an FP32 copy of an FP64 right-hand side
    int64_t tot = H.lev.back().g.n() * nc;
    for (size_t l = 1; l < H.lev.size(); ++l) tot += 3 * H.lev[l].g.n() * nc + 2 * H.lev[l - 1].g.n() * nc;
    return tot;
}

cudaError_t mg_vcycle_f32(const MGHierarchy& H, int nc, const double* r, int64_t ldr, float* w, float* work,
                          cudaStream_t s) {
    // an FP64 right-hand side is read by four fine-level kernels: round it to
    // FP32 once (one pass) so that every level kernel streams FP32
    if (nc <= 0) return cudaSuccess;
    return mg_graphed(H, 1, nc, r, ldr, w, nc, work, s, [&](cudaStream_t st) -> cudaError_t {
        const int64_t n = H.lev.back().g.n();
        float* r32 = work + (mg_workspace_floats(H, nc) - n * nc);
        k_narrow_rhs<<<grid_size_for(n * nc, 256, sm_count() * 8), 256, 0, st>>>(n, nc, r, ldr, r32, nc);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return run<float>(H, nc, r32, nc, w, work, st);
    });
}

cudaError_t mg_vcycle_f32_pair(const MGHierarchy& H, int nc1, const double* r1, int64_t ldr1, int nc2,
                               const double* r2, int64_t ldr2, float* w, float* work, cudaStream_t s) {
    // both right-hand sides narrowed side by side, then one cycle of
    // nc1 + nc2 columns: the coarse levels cost one cycle instead of two
    const int nc = nc1 + nc2;
    if (nc1 <= 0 || nc2 <= 0) return cudaErrorInvalidValue;
    return mg_graphed(
        H, 3, nc1, r1, ldr1, w, nc, work, s,
        [&](cudaStream_t st) -> cudaError_t {
            const int64_t n = H.lev.back().g.n();
            float* r32 = work + (mg_workspace_floats(H, nc) - n * nc);
            k_narrow_rhs<<<grid_size_for(n * nc1, 256, sm_count() * 8), 256, 0, st>>>(n, nc1, r1, ldr1, r32, nc);
            k_narrow_rhs<<<grid_size_for(n * nc2, 256, sm_count() * 8), 256, 0, st>>>(n, nc2, r2, ldr2, r32 + nc1, nc);
            count_launches(2);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            return run<float>(H, nc, r32, nc, w, work, st);
        },
        r2, ldr2, nc2);
}

cudaError_t mg_vcycle_f32(const MGHierarchy& H, int nc, const float* r, int64_t ldr, float* w, float* work,
                          cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    return mg_graphed(H, 0, nc, r, ldr, w, nc, work, s,
                      [&](cudaStream_t st) -> cudaError_t { return run<float>(H, nc, r, ldr, w, work, st); });
}

}  // namespace plhr
