// Stencil products with the finite-difference Laplacian (Section 5.2: 5-point
// in 2D, 7-point in 3D; Dirichlet, or periodic with a diagonal potential for
// the real-space Hamiltonian -1/2 Lap + V), on blocks of vectors stored row-major
// [grid point][column].  One thread per (grid point, column) pair; a CTA
// covers 256 consecutive elements of one x-line (blockIdx.y = y, blockIdx.z =
// z), so a warp covers 32 consecutive doubles of the block, every neighbour
// access of a warp (x +- 1: +-ld, y +- 1: +-ld*nx, z +- 1: +-ld*nx*ny) is one
// contiguous 256-byte segment, the plane/line reuse is served from L1/L2, and
// no 64-bit index division is needed.  The kernels are bound by GB300's FP64
// pipe, so the FP64 operations per element are kept to seven: five additions
// of the neighbours, one fused 2d x_c - sum, one scaling by 1/h^2.
#include "plhr_internal.h"

namespace plhr {
namespace {

struct Geo {
    int64_t nx, ny, nz, sx, sy, sz;   // sizes and row strides (in rows)
    int periodic;
    const double* pot;                // diagonal term or null
};

// sum over axes of (2 x_c - x_- - x_+); neighbours outside the grid are zero
// (Dirichlet) or wrap around (periodic).  The neighbour sum is formed first,
// then 2d x_c - sum in one fused operation.
template <bool D3>
__device__ __forceinline__ double lap_at(const double* __restrict__ xp, int64_t ld, int ix, int iy, int iz,
                                         const Geo& g) {
    const double xc = xp[0];
    double x0, x1, y0, y1, z0 = 0.0, z1 = 0.0;
    if (!g.periodic) {
        x0 = ix > 0 ? xp[-ld] : 0.0;
        x1 = ix < g.nx - 1 ? xp[ld] : 0.0;
        y0 = iy > 0 ? xp[-ld * g.sy] : 0.0;
        y1 = iy < g.ny - 1 ? xp[ld * g.sy] : 0.0;
        if (D3) {
            z0 = iz > 0 ? xp[-ld * g.sz] : 0.0;
            z1 = iz < g.nz - 1 ? xp[ld * g.sz] : 0.0;
        }
    } else {
        // offsets of the wrapped neighbours (in rows)
        const int64_t xm = ix > 0 ? -1 : g.nx - 1, xq = ix < g.nx - 1 ? 1 : -(g.nx - 1);
        const int64_t ym = iy > 0 ? -g.sy : (g.ny - 1) * g.sy, yq = iy < g.ny - 1 ? g.sy : -(g.ny - 1) * g.sy;
        x0 = xp[ld * xm];
        x1 = xp[ld * xq];
        y0 = xp[ld * ym];
        y1 = xp[ld * yq];
        if (D3) {
            const int64_t zm = iz > 0 ? -g.sz : (g.nz - 1) * g.sz, zq = iz < g.nz - 1 ? g.sz : -(g.nz - 1) * g.sz;
            z0 = xp[ld * zm];
            z1 = xp[ld * zq];
        }
    }
    double nb = (x0 + x1) + (y0 + y1);
    if (D3) nb += z0 + z1;
    return fma(D3 ? 6.0 : 4.0, xc, -nb);
}

// element of this thread: (ix, column c) on the x-line (blockIdx.y, blockIdx.z)
struct El {
    int ix, iy, iz, c;
    int64_t row;
};
__device__ __forceinline__ bool element_of(const Geo& g, int nc, El& e) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int)g.nx * nc) return false;
    e.ix = t / nc;
    e.c = t - e.ix * nc;
    e.iy = blockIdx.y;
    e.iz = blockIdx.z;
    e.row = ((int64_t)e.iz * g.ny + e.iy) * g.nx + e.ix;
    return true;
}

// y = alpha (L + pot) x + beta x; mode (chosen on the host, so that no FP64
// comparison runs per element): 0 alpha = 1, beta = 0; 1 beta = 0; 2 general
template <bool D3>
__global__ void __launch_bounds__(256) k_lap_axpby(Geo g, int nc, double ih2, const double* __restrict__ x,
                                                   int64_t ldx, double* __restrict__ y, int64_t ldy,
                                                   double alpha, double beta, int mode) {
    El e;
    if (!element_of(g, nc, e)) return;
    const double* xp = x + e.row * ldx + e.c;
    double lx = ih2 * lap_at<D3>(xp, ldx, e.ix, e.iy, e.iz, g);
    if (g.pot) lx = fma(g.pot[e.row], xp[0], lx);
    double out = lx;
    if (mode == 1) out = alpha * lx;
    else if (mode == 2) out = fma(alpha, lx, beta * xp[0]);
    y[e.row * ldy + e.c] = out;
}

template <bool D3>
__global__ void __launch_bounds__(256) k_lap_shifts(Geo g, int nc, double ih2, const double* __restrict__ x,
                                                    int64_t ldx, double* __restrict__ ax, int64_t ldax,
                                                    double* __restrict__ o1, int64_t ld1,
                                                    const double* __restrict__ lam,
                                                    double* __restrict__ o2, int64_t ld2, double sig) {
    El e;
    if (!element_of(g, nc, e)) return;
    const double* xp = x + e.row * ldx + e.c;
    double a = ih2 * lap_at<D3>(xp, ldx, e.ix, e.iy, e.iz, g);
    const double xv = xp[0];
    if (g.pot) a = fma(g.pot[e.row], xv, a);
    if (ax) ax[e.row * ldax + e.c] = a;
    if (o1) o1[e.row * ld1 + e.c] = fma(-lam[e.c], xv, a);
    if (o2) o2[e.row * ld2 + e.c] = fma(-sig, xv, a);
}

dim3 grid_of(const Grid& g, int nc) {
    return dim3((unsigned)((g.nx * nc + 255) / 256), (unsigned)g.ny, (unsigned)g.nz);
}
// the launch shape's limits: y and z lines in gridDim.y / z, x-line elements in an int
bool grid_fits(const Grid& g, int nc) {
    return g.ny <= 65535 && g.nz <= 65535 && g.nx * nc <= (int64_t)1 << 30;
}

Geo geo_of(const Grid& g) {
    Geo o;
    o.nx = g.nx; o.ny = g.ny; o.nz = g.nz;
    o.sx = 1; o.sy = g.nx; o.sz = g.nx * g.ny;
    o.periodic = g.periodic;
    o.pot = g.pot;
    return o;
}

}  // namespace

cudaError_t lap_axpby(const Grid& g, int nc, const double* x, int64_t ldx, double* y, int64_t ldy,
                      double alpha, double beta, cudaStream_t s) {
    if (g.csr) return csr_axpby(*g.csr, nc, x, ldx, y, ldy, alpha, beta, s);
    if (g.q1) return q1_axpby(g, nc, x, ldx, y, ldy, alpha, beta, s);
    if (g.n() * nc == 0) return cudaSuccess;
    if (!grid_fits(g, nc)) return cudaErrorInvalidValue;
    Geo G = geo_of(g);
    const int mode = beta != 0.0 ? 2 : (alpha != 1.0 ? 1 : 0);
    if (g.d == 3)
        k_lap_axpby<true><<<grid_of(g, nc), 256, 0, s>>>(G, nc, g.inv_h2(), x, ldx, y, ldy, alpha, beta, mode);
    else
        k_lap_axpby<false><<<grid_of(g, nc), 256, 0, s>>>(G, nc, g.inv_h2(), x, ldx, y, ldy, alpha, beta, mode);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t lap_apply_shifts(const Grid& g, int nc, const double* x, int64_t ldx, double* ax,
                             int64_t ldax, double* o1, int64_t ld1, const double* lam, double* o2,
                             int64_t ld2, double sig, cudaStream_t s) {
    if (g.csr) return csr_apply_shifts(*g.csr, nc, x, ldx, ax, ldax, o1, ld1, lam, o2, ld2, sig, s);
    if (g.q1) return q1_apply_shifts(g, nc, x, ldx, ax, ldax, o1, ld1, lam, o2, ld2, sig, s);
    if (g.n() * nc == 0) return cudaSuccess;
    if (!grid_fits(g, nc)) return cudaErrorInvalidValue;
    Geo G = geo_of(g);
    if (g.d == 3)
        k_lap_shifts<true><<<grid_of(g, nc), 256, 0, s>>>(G, nc, g.inv_h2(), x, ldx, ax, ldax, o1, ld1, lam, o2,
                                                           ld2, sig);
    else
        k_lap_shifts<false><<<grid_of(g, nc), 256, 0, s>>>(G, nc, g.inv_h2(), x, ldx, ax, ldax, o1, ld1, lam,
                                                            o2, ld2, sig);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plhr
