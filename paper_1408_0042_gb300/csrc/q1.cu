// 27-point trilinear (Q1) finite-element stiffness and mass products, and the
// complex Bloch Hamiltonian product, on blocks stored row-major
// [grid point][column].
//
// Q1 (Section 5.1's bilinear elements, in 3D).  The unknowns are the interior
// nodes of a tensor mesh of E_a = n_a + 1 elements per axis with width h;
// interior node i (0-based) sits at mesh point i + 1 and belongs to the cells
// i (as their upper corner) and i + 1 (as their lower corner) along each axis.
// With the 1D linear-element matrices k = [[1, -1], [-1, 1]] / h and
// m = [[2, 1], [1, 2]] h / 6, the element stiffness entry between local
// corners a and b depends only on which axes differ (d_a = [a_a != b_a]):
//     K_e(a, b) = c_e (k(d_x) m(d_y) m(d_z) + m(d_x) k(d_y) m(d_z) + m(d_x) m(d_y) k(d_z)),
//     k(0) = 1/h, k(1) = -1/h, m(0) = 2h/6, m(1) = h/6,
// so a row of the assembled stiffness is the sum over the 8 cells around the
// node of c_e times 8 constant weights on the cell's corners; the mass row is
// the tensor product of the 1D rows [1, 4, 1] h / 6 (coefficient-free).
// Nodes on the boundary carry the homogeneous Dirichlet value 0.  One thread
// per (node, column): the 27 neighbour values are loaded once (x +- 1 at +-ld,
// y +- 1 at +-ld nx, z +- 1 at +-ld nx ny; a warp reads contiguous 256-byte
// segments) and serve both the stiffness and the mass row.
//
// Bloch Hamiltonian (Section 5.3, complex Hermitian): periodic 7-point
// stencil with the phase e^{i kappa_d h} on the link j -> j + e_d and the
// potential on the diagonal, on complex128 blocks (re, im interleaved).
#include "plhr_internal.h"

namespace plhr {
namespace {

struct Q1Geo {
    int64_t nx, ny, nz;   // interior nodes per axis
    double h;
    const double* cell;   // element coefficients ((nx+1)(ny+1)(nz+1), x fastest) or null (c = 1)
};

enum { Q1_AXPBY = 0, Q1_SHIFTS = 1, Q1_PAIR = 2 };

// stiffness weight of a cell corner pair differing along the axes (dx, dy, dz)
__device__ __forceinline__ double kw(int dx, int dy, int dz, double h) {
    const double k0 = 1.0 / h, k1 = -1.0 / h, m0 = h / 3.0, m1 = h / 6.0;
    const double kx = dx ? k1 : k0, ky = dy ? k1 : k0, kz = dz ? k1 : k0;
    const double mx = dx ? m1 : m0, my = dy ? m1 : m0, mz = dz ? m1 : m0;
    return kx * my * mz + mx * ky * mz + mx * my * kz;
}

// Stiffness and mass rows of node (ix, iy, iz) applied to column c.
template <bool NEED_A, bool NEED_B>
__device__ __forceinline__ void q1_rows(const Q1Geo& g, const double* __restrict__ x, int64_t ldx, int64_t row,
                                        int64_t ix, int64_t iy, int64_t iz, int c, double& ya, double& yb) {
    double xv[3][3][3];
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const int64_t qx = ix + dx - 1, qy = iy + dy - 1, qz = iz + dz - 1;
                const bool in = qx >= 0 && qx < g.nx && qy >= 0 && qy < g.ny && qz >= 0 && qz < g.nz;
                const int64_t q = row + (dx - 1) + (int64_t)(dy - 1) * g.nx + (int64_t)(dz - 1) * g.nx * g.ny;
                xv[dz][dy][dx] = in ? x[q * ldx + c] : 0.0;
            }
    ya = 0.0;
    yb = 0.0;
    if (NEED_A) {
        const int64_t ex0 = g.nx + 1, ey0 = g.ny + 1;
#pragma unroll
        for (int sz = 0; sz < 2; ++sz)
#pragma unroll
            for (int sy = 0; sy < 2; ++sy)
#pragma unroll
                for (int sx = 0; sx < 2; ++sx) {
                    // cell (ix + sx, iy + sy, iz + sz); this node is its corner (1 - sx, 1 - sy, 1 - sz)
                    const double ce = g.cell ? g.cell[((iz + sz) * ey0 + (iy + sy)) * ex0 + (ix + sx)] : 1.0;
                    double acc = 0.0;
#pragma unroll
                    for (int bz = 0; bz < 2; ++bz)
#pragma unroll
                        for (int by = 0; by < 2; ++by)
#pragma unroll
                            for (int bx = 0; bx < 2; ++bx)
                                acc += kw(bx != 1 - sx, by != 1 - sy, bz != 1 - sz, g.h) * xv[sz + bz][sy + by][sx + bx];
                    ya += ce * acc;
                }
    }
    if (NEED_B) {
        const double m0 = 4.0 * g.h / 6.0, m1 = g.h / 6.0;
#pragma unroll
        for (int dz = 0; dz < 3; ++dz) {
            const double wz = dz == 1 ? m0 : m1;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                const double wy = dy == 1 ? m0 : m1;
                double t = 0.0;
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) t += (dx == 1 ? m0 : m1) * xv[dz][dy][dx];
                yb += wz * wy * t;
            }
        }
    }
}

// MODE Q1_AXPBY: y = alpha (op x) + beta x (op = stiffness when stiff, else mass)
// MODE Q1_SHIFTS: y = op x, o1 = y - lam_c x, o2 = y - sig x (each optional)
// MODE Q1_PAIR: y = sa (stiffness x), o1 = sb (mass x)
template <int MODE>
__global__ void __launch_bounds__(256) k_q1(Q1Geo g, int nc, int stiff, double sa, double sb,
                                            const double* __restrict__ x, int64_t ldx, double* __restrict__ y,
                                            int64_t ldy, double* __restrict__ o1, int64_t ld1,
                                            const double* __restrict__ lam, double* __restrict__ o2, int64_t ld2,
                                            double alpha, double beta, double sig, int64_t total) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t row;
        int c;
        split_index(e, nc, row, c);
        const int64_t ix = row % g.nx, t = row / g.nx, iy = t % g.ny, iz = t / g.ny;
        double ya, yb;
        if (MODE == Q1_PAIR) {
            q1_rows<true, true>(g, x, ldx, row, ix, iy, iz, c, ya, yb);
            y[row * ldy + c] = sa * ya;
            o1[row * ld1 + c] = sb * yb;
        } else {
            if (stiff) q1_rows<true, false>(g, x, ldx, row, ix, iy, iz, c, ya, yb);
            else q1_rows<false, true>(g, x, ldx, row, ix, iy, iz, c, ya, yb);
            const double a = stiff ? sa * ya : sb * yb;
            const double xc = x[row * ldx + c];
            if (MODE == Q1_AXPBY) {
                y[row * ldy + c] = alpha * a + beta * xc;
            } else {
                if (y) y[row * ldy + c] = a;
                if (o1) o1[row * ld1 + c] = a - lam[c] * xc;
                if (o2) o2[row * ld2 + c] = a - sig * xc;
            }
        }
    }
}

Q1Geo q1geo(const Grid& g) { return {g.nx, g.ny, g.nz, g.h, g.cell}; }

// Bloch Hamiltonian on complex128 blocks: y = 1/2 sum_d (2 x - ph_d x_{+d} - conj(ph_d) x_{-d}) / h^2 + V x
struct BlochGeo {
    int64_t nx, ny, nz;
    double ih2;                 // 1 / h^2
    double cr[3], ci[3];        // e^{i kappa_d h}
    const double* pot;
};

__global__ void __launch_bounds__(256) k_bloch(BlochGeo g, int nc, const double2* __restrict__ x, int64_t ldx,
                                               double2* __restrict__ y, int64_t ldy, int64_t total) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t row;
        int c;
        split_index(e, nc, row, c);
        const int64_t ix = row % g.nx, t = row / g.nx, iy = t % g.ny, iz = t / g.ny;
        const int64_t n[3] = {g.nx, g.ny, g.nz}, i[3] = {ix, iy, iz}, st[3] = {1, g.nx, g.nx * g.ny};
        const double2 xc = x[row * ldx + c];
        double sr = 0.0, si = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int64_t up = i[d] < n[d] - 1 ? st[d] : -(n[d] - 1) * st[d];
            const int64_t dn = i[d] > 0 ? -st[d] : (n[d] - 1) * st[d];
            const double2 xp = x[(row + up) * ldx + c], xm = x[(row + dn) * ldx + c];
            // 2 x - ph x_+ - conj(ph) x_-
            sr += 2.0 * xc.x - (g.cr[d] * xp.x - g.ci[d] * xp.y) - (g.cr[d] * xm.x + g.ci[d] * xm.y);
            si += 2.0 * xc.y - (g.cr[d] * xp.y + g.ci[d] * xp.x) - (g.cr[d] * xm.y - g.ci[d] * xm.x);
        }
        const double v = g.pot ? g.pot[row] : 0.0;
        y[row * ldy + c] = make_double2(0.5 * g.ih2 * sr + v * xc.x, 0.5 * g.ih2 * si + v * xc.y);
    }
}

}  // namespace

cudaError_t q1_axpby(const Grid& g, int nc, const double* x, int64_t ldx, double* y, int64_t ldy, double alpha,
                     double beta, cudaStream_t s) {
    const int64_t total = g.n() * nc;
    if (total == 0) return cudaSuccess;
    const int blocks = grid_size_for(total, 256, sm_count() * 16);
    k_q1<Q1_AXPBY><<<blocks, 256, 0, s>>>(q1geo(g), nc, g.q1 == 1, g.scale, g.scale, x, ldx, y, ldy, nullptr, 0,
                                          nullptr, nullptr, 0, alpha, beta, 0.0, total);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t q1_apply_shifts(const Grid& g, int nc, const double* x, int64_t ldx, double* ax, int64_t ldax,
                            double* o1, int64_t ld1, const double* lam, double* o2, int64_t ld2, double sig,
                            cudaStream_t s) {
    const int64_t total = g.n() * nc;
    if (total == 0) return cudaSuccess;
    const int blocks = grid_size_for(total, 256, sm_count() * 16);
    k_q1<Q1_SHIFTS><<<blocks, 256, 0, s>>>(q1geo(g), nc, g.q1 == 1, g.scale, g.scale, x, ldx, ax, ldax, o1, ld1,
                                           lam, o2, ld2, 1.0, 0.0, sig, total);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t q1_pair(const Grid& A, const Grid& B, int nc, const double* x, int64_t ldx, double* ax, int64_t ldax,
                    double* bx, int64_t ldbx, cudaStream_t s) {
    const int64_t total = A.n() * nc;
    if (total == 0) return cudaSuccess;
    const int blocks = grid_size_for(total, 256, sm_count() * 16);
    k_q1<Q1_PAIR><<<blocks, 256, 0, s>>>(q1geo(A), nc, 1, A.scale, B.scale, x, ldx, ax, ldax, bx, ldbx, nullptr,
                                         nullptr, 0, 1.0, 0.0, 0.0, total);
    count_launches(1);
    return cudaGetLastError();
}

bool q1_same_mesh(const Grid& A, const Grid& B) {
    return A.q1 == 1 && B.q1 == 2 && A.nx == B.nx && A.ny == B.ny && A.nz == B.nz && A.h == B.h;
}

cudaError_t bloch_apply(const Grid& g, int nc, const double* x, int64_t ldx, double* y, int64_t ldy,
                        cudaStream_t s) {
    const int64_t total = g.n() * nc;
    if (total == 0) return cudaSuccess;
    BlochGeo b;
    b.nx = g.nx; b.ny = g.ny; b.nz = g.nz;
    b.ih2 = 1.0 / (g.h * g.h);
    for (int d = 0; d < 3; ++d) {
        b.cr[d] = std::cos(g.kappa[d] * g.h);
        b.ci[d] = std::sin(g.kappa[d] * g.h);
    }
    b.pot = g.pot;
    const int blocks = grid_size_for(total, 256, sm_count() * 16);
    k_bloch<<<blocks, 256, 0, s>>>(b, nc, reinterpret_cast<const double2*>(x), ldx, reinterpret_cast<double2*>(y),
                                   ldy, total);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace plhr
