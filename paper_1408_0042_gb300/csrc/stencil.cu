// Stencil products with the Dirichlet finite-difference Laplacian (Section 5.2:
// 5-point in 2D, 7-point in 3D), on blocks of vectors stored row-major
// [grid point][column].  One thread per (grid point, column) pair: a warp
// covers 32 consecutive doubles of the block, so every neighbour access of a
// warp (x +- 1: +-ld, y +- 1: +-ld*nx, z +- 1: +-ld*nx*ny) is one contiguous
// 256-byte segment and the plane/line reuse is served from L1/L2.
#include "plhr_internal.h"

namespace plhr {
namespace {

struct Geo {
    int64_t nx, ny, nz, sx, sy, sz;   // sizes and row strides (in rows)
};

template <bool D3>
__device__ __forceinline__ double lap_at(const double* __restrict__ xp, int64_t ld, int64_t ix,
                                         int64_t iy, int64_t iz, const Geo& g) {
    double xc = xp[0];
    double s = (D3 ? 6.0 : 4.0) * xc;
    if (ix > 0) s -= xp[-ld];
    if (ix < g.nx - 1) s -= xp[ld];
    if (iy > 0) s -= xp[-ld * g.sy];
    if (iy < g.ny - 1) s -= xp[ld * g.sy];
    if (D3) {
        if (iz > 0) s -= xp[-ld * g.sz];
        if (iz < g.nz - 1) s -= xp[ld * g.sz];
    }
    return s;
}

template <bool D3>
__global__ void __launch_bounds__(256) k_lap_axpby(Geo g, int nc, double ih2, const double* __restrict__ x,
                                                   int64_t ldx, double* __restrict__ y, int64_t ldy,
                                                   double alpha, double beta, int64_t total) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = e / nc;
        int c = (int)(e - row * nc);
        int64_t ix = row % g.nx, t = row / g.nx, iy = t % g.ny, iz = t / g.ny;
        const double* xp = x + row * ldx + c;
        double lx = lap_at<D3>(xp, ldx, ix, iy, iz, g);
        y[row * ldy + c] = alpha * ih2 * lx + beta * xp[0];
    }
}

template <bool D3>
__global__ void __launch_bounds__(256) k_lap_shifts(Geo g, int nc, double ih2, const double* __restrict__ x,
                                                    int64_t ldx, double* __restrict__ ax, int64_t ldax,
                                                    double* __restrict__ o1, int64_t ld1,
                                                    const double* __restrict__ lam,
                                                    double* __restrict__ o2, int64_t ld2, double sig,
                                                    int64_t total) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = e / nc;
        int c = (int)(e - row * nc);
        int64_t ix = row % g.nx, t = row / g.nx, iy = t % g.ny, iz = t / g.ny;
        const double* xp = x + row * ldx + c;
        double a = ih2 * lap_at<D3>(xp, ldx, ix, iy, iz, g);
        double xv = xp[0];
        if (ax) ax[row * ldax + c] = a;
        if (o1) o1[row * ld1 + c] = a - lam[c] * xv;
        if (o2) o2[row * ld2 + c] = a - sig * xv;
    }
}

Geo geo_of(const Grid& g) {
    Geo o;
    o.nx = g.nx; o.ny = g.ny; o.nz = g.nz;
    o.sx = 1; o.sy = g.nx; o.sz = g.nx * g.ny;
    return o;
}

}  // namespace

cudaError_t lap_axpby(const Grid& g, int nc, const double* x, int64_t ldx, double* y, int64_t ldy,
                      double alpha, double beta, cudaStream_t s) {
    int64_t total = g.n() * nc;
    if (total == 0) return cudaSuccess;
    int blocks = grid_size_for(total, 256, sm_count() * 16);
    Geo G = geo_of(g);
    if (g.d == 3)
        k_lap_axpby<true><<<blocks, 256, 0, s>>>(G, nc, g.inv_h2(), x, ldx, y, ldy, alpha, beta, total);
    else
        k_lap_axpby<false><<<blocks, 256, 0, s>>>(G, nc, g.inv_h2(), x, ldx, y, ldy, alpha, beta, total);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t lap_apply_shifts(const Grid& g, int nc, const double* x, int64_t ldx, double* ax,
                             int64_t ldax, double* o1, int64_t ld1, const double* lam, double* o2,
                             int64_t ld2, double sig, cudaStream_t s) {
    int64_t total = g.n() * nc;
    if (total == 0) return cudaSuccess;
    int blocks = grid_size_for(total, 256, sm_count() * 16);
    Geo G = geo_of(g);
    if (g.d == 3)
        k_lap_shifts<true><<<blocks, 256, 0, s>>>(G, nc, g.inv_h2(), x, ldx, ax, ldax, o1, ld1, lam, o2,
                                                  ld2, sig, total);
    else
        k_lap_shifts<false><<<blocks, 256, 0, s>>>(G, nc, g.inv_h2(), x, ldx, ax, ldax, o1, ld1, lam,
                                                   o2, ld2, sig, total);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plhr
