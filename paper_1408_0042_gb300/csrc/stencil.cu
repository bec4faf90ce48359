// Stencil products with the finite-difference Laplacian (Section 5.2: 5-point
// in 2D, 7-point in 3D; Dirichlet, or periodic with a diagonal potential for
// the real-space Hamiltonian -1/2 Lap + V), on blocks of vectors stored row-major
// [grid point][column].  One thread per (grid point, column) pair: a warp
// covers 32 consecutive doubles of the block, so every neighbour access of a
// warp (x +- 1: +-ld, y +- 1: +-ld*nx, z +- 1: +-ld*nx*ny) is one contiguous
// 256-byte segment and the plane/line reuse is served from L1/L2.
#include "plhr_internal.h"

namespace plhr {
namespace {

struct Geo {
    int64_t nx, ny, nz, sx, sy, sz;   // sizes and row strides (in rows)
    int periodic;
    const double* pot;                // diagonal term or null
};

// sum over axes of (2 x_c - x_- - x_+); neighbours outside the grid are zero
// (Dirichlet) or wrap around (periodic)
template <bool D3>
__device__ __forceinline__ double lap_at(const double* __restrict__ xp, int64_t ld, int64_t ix,
                                         int64_t iy, int64_t iz, const Geo& g) {
    double xc = xp[0];
    double s = (D3 ? 6.0 : 4.0) * xc;
    if (!g.periodic) {
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
    // periodic: offsets of the wrapped neighbours (in rows)
    const int64_t xm = ix > 0 ? -1 : g.nx - 1, xq = ix < g.nx - 1 ? 1 : -(g.nx - 1);
    const int64_t ym = iy > 0 ? -g.sy : (g.ny - 1) * g.sy, yq = iy < g.ny - 1 ? g.sy : -(g.ny - 1) * g.sy;
    s -= xp[ld * xm] + xp[ld * xq] + xp[ld * ym] + xp[ld * yq];
    if (D3) {
        const int64_t zm = iz > 0 ? -g.sz : (g.nz - 1) * g.sz, zq = iz < g.nz - 1 ? g.sz : -(g.nz - 1) * g.sz;
        s -= xp[ld * zm] + xp[ld * zq];
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
        double lx = ih2 * lap_at<D3>(xp, ldx, ix, iy, iz, g);
        if (g.pot) lx += g.pot[row] * xp[0];
        y[row * ldy + c] = alpha * lx + beta * xp[0];
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
        if (g.pot) a += g.pot[row] * xv;
        if (ax) ax[row * ldax + c] = a;
        if (o1) o1[row * ld1 + c] = a - lam[c] * xv;
        if (o2) o2[row * ld2 + c] = a - sig * xv;
    }
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
    if (g.csr) return csr_apply_shifts(*g.csr, nc, x, ldx, ax, ldax, o1, ld1, lam, o2, ld2, sig, s);
    if (g.q1) return q1_apply_shifts(g, nc, x, ldx, ax, ldax, o1, ld1, lam, o2, ld2, sig, s);
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
