// Teter-Payne-Allan preconditioner (Section 5.3: a positive diagonal matrix
// in the plane-wave basis) on a tensor grid, FP64:
//     T = S diag(K(mu / E)) S^T,
//     K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4),
// with S = Sx (x) Sy (x) Sz the orthonormal eigenvectors of the grid's kinetic
// operator -1/2 Lap_h (real Fourier modes on a periodic axis, sine modes on a
// Dirichlet axis), mu = mu_x + mu_y + mu_z their kinetic energies and E one
// fixed reference energy.  T is symmetric positive definite and commutes with
// -1/2 Lap_h.
//
// Application: three forward passes (one per axis, each a dense N_a x N_a
// product along that axis with the matrix in shared memory), the factor
// fused into the last of them, and three inverse passes.
#include <cmath>
#include <vector>

#include "plhr_internal.h"

namespace plhr {
namespace {

constexpr int kT = 256;
constexpr int kMaxAxis = 144;   // N_a^2 doubles of shared memory per pass

struct AxisPass {
    int64_t nx, ny, nz;   // grid
    int axis;             // 0 x, 1 y, 2 z
    int N;                // size along the axis
    int64_t stride;       // point stride along the axis
    int nc;
};

__device__ __forceinline__ double tpa(double x) {
    const double num = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x));
    const double x2 = x * x;
    return num / (num + 16.0 * x2 * x2);
}

// out[.., q, ..] = sum_j M[j][q] in[.., j, ..] along one axis (M = S for the
// forward transform, S^T for the inverse); with scale: times K(mu / E) of the
// mode (qx, qy, qz) of the element (used on the last forward pass)
template <bool SCALE>
__global__ void __launch_bounds__(kT) k_axis(AxisPass a, const double* __restrict__ M, const double* __restrict__ in,
                                             int64_t ldi, double* __restrict__ out, int64_t ldo,
                                             const double* __restrict__ mux, const double* __restrict__ muy,
                                             const double* __restrict__ muz, double inv_e) {
    extern __shared__ double sm[];
    const int N = a.N;
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) sm[i] = M[i];
    __syncthreads();
    const int64_t total = a.nx * a.ny * a.nz * a.nc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pt = e / a.nc;
        const int c = (int)(e - pt * a.nc);
        const int64_t ix = pt % a.nx, t = pt / a.nx, iy = t % a.ny, iz = t / a.ny;
        const int q = (int)(a.axis == 0 ? ix : (a.axis == 1 ? iy : iz));
        const int64_t base = pt - (int64_t)q * a.stride;
        double s = 0.0;
        for (int j = 0; j < N; ++j) s = fma(sm[j * N + q], in[(base + j * a.stride) * ldi + c], s);
        if (SCALE) {
            double mu = mux[ix] + muy[iy] + (muz ? muz[iz] : 0.0);
            s *= tpa(mu * inv_e);
        }
        out[pt * ldo + c] = s;
    }
}

int nblk(int64_t total) { return grid_size_for(total, kT, sm_count() * 8); }

// orthonormal eigenvectors S[p][m] and eigenvalues mu (times 1/2 scale of the
// kinetic operator folded in by the caller) of the 1D second difference
void axis_basis(int64_t N, bool periodic, std::vector<double>& S, std::vector<double>& mu) {
    S.assign(N * N, 0.0);
    mu.assign(N, 0.0);
    if (!periodic) {
        for (int64_t m = 0; m < N; ++m) {
            const double th = (m + 1) * M_PI / (N + 1);
            mu[m] = 2.0 - 2.0 * std::cos(th);
            for (int64_t p = 0; p < N; ++p) S[p * N + m] = std::sqrt(2.0 / (N + 1)) * std::sin((p + 1) * th);
        }
        return;
    }
    // real Fourier modes: constant; cos and sin of frequency f = 1 .. (N-1)/2;
    // the alternating mode when N is even
    int64_t col = 0;
    for (int64_t p = 0; p < N; ++p) S[p * N + col] = 1.0 / std::sqrt((double)N);
    mu[col++] = 0.0;
    for (int64_t f = 1; 2 * f < N; ++f) {
        const double th = 2.0 * M_PI * f / N;
        for (int64_t p = 0; p < N; ++p) {
            S[p * N + col] = std::sqrt(2.0 / N) * std::cos(th * p);
            S[p * N + col + 1] = std::sqrt(2.0 / N) * std::sin(th * p);
        }
        mu[col] = mu[col + 1] = 2.0 - 2.0 * std::cos(th);
        col += 2;
    }
    if (N % 2 == 0) {
        for (int64_t p = 0; p < N; ++p) S[p * N + col] = (p % 2 ? -1.0 : 1.0) / std::sqrt((double)N);
        mu[col++] = 4.0;
    }
}

}  // namespace

int64_t spectral_workspace_doubles(const SpecPrec& P, int nc) { return 2 * P.n() * nc; }

cudaError_t spectral_apply(const SpecPrec& P, int nc, const double* r, int64_t ldr, double* w, double* work,
                           cudaStream_t s) {
    if (nc <= 0) return cudaSuccess;
    const int64_t n = P.n();
    double* t0 = work;
    double* t1 = work + n * nc;
    const int64_t Ns[3] = {P.nx, P.ny, P.nz};
    const int64_t strides[3] = {1, P.nx, P.nx * P.ny};
    const int d = P.d;
    const int64_t total = n * nc;
    auto pass = [&](int axis, bool inverse, bool scale, const double* in, int64_t ldi, double* out) {
        AxisPass a{P.nx, P.ny, P.nz, axis, (int)Ns[axis], strides[axis], nc};
        const size_t shm = sizeof(double) * Ns[axis] * Ns[axis];
        const double* M = inverse ? P.d_St[axis] : P.d_S[axis];
        if (scale)
            k_axis<true><<<nblk(total), kT, shm, s>>>(a, M, in, ldi, out, nc, P.d_mu[0], P.d_mu[1],
                                                      d == 3 ? P.d_mu[2] : nullptr, 1.0 / P.energy);
        else
            k_axis<false><<<nblk(total), kT, shm, s>>>(a, M, in, ldi, out, nc, nullptr, nullptr, nullptr, 0.0);
        count_launches(1);
        return cudaGetLastError();
    };
    cudaError_t e;
    // forward: x, y (, z); the factor on the last forward pass
    if ((e = pass(0, false, false, r, ldr, t0)) != cudaSuccess) return e;
    if ((e = pass(1, false, d == 2, t0, nc, t1)) != cudaSuccess) return e;
    const double* f = t1;
    if (d == 3) {
        if ((e = pass(2, false, true, t1, nc, t0)) != cudaSuccess) return e;
        if ((e = pass(2, true, false, t0, nc, t1)) != cudaSuccess) return e;
    }
    if ((e = pass(1, true, false, f, nc, t0)) != cudaSuccess) return e;
    return pass(0, true, false, t0, nc, w);
}

}  // namespace plhr

using namespace plhr;

extern "C" plhr_status plhr_prec_tpa(plhr_prec** out, const plhr_op* A, double sigma, double energy) {
    clear_error();
    if (!out || !A || !std::isfinite(sigma) || !std::isfinite(energy)) {
        set_error("plhr_prec_tpa: invalid argument");
        return PLHR_EINVAL;
    }
    const Grid& g = A->g;
    if (g.csr) {
        set_error("plhr_prec_tpa: A must be a stencil or Hamiltonian operator (not CSR)");
        return PLHR_EINVAL;
    }
    const int64_t Ns[3] = {g.nx, g.ny, g.d == 3 ? g.nz : 1};
    for (int a = 0; a < g.d; ++a)
        if (Ns[a] > kMaxAxis) {
            set_error("plhr_prec_tpa: axis size %lld exceeds %d", (long long)Ns[a], kMaxAxis);
            return PLHR_EINVAL;
        }
    if (!(energy > 0)) {
        // sigma - min V, or the mean kinetic energy of the grid's modes d / h^2
        double vmin = 0.0;
        if (g.pot) {
            std::vector<double> hv(g.n());
            if (cudaMemcpy(hv.data(), g.pot, sizeof(double) * g.n(), cudaMemcpyDeviceToHost) != cudaSuccess) {
                set_error("plhr_prec_tpa: reading the potential failed");
                return PLHR_ECUDA;
            }
            vmin = hv[0];
            for (double v : hv) vmin = std::fmin(vmin, v);
        }
        energy = sigma - vmin;
        if (!(energy > 0)) energy = g.d * 2.0 * g.inv_h2();   // d / h^2 for the scale 1/2
    }
    plhr_prec* T = new plhr_prec;
    T->kind = PREC_TPA;
    SpecPrec& P = T->sp;
    P.d = g.d;
    P.nx = Ns[0]; P.ny = Ns[1]; P.nz = Ns[2];
    P.energy = energy;
    for (int a = 0; a < g.d; ++a) {
        const int64_t N = Ns[a];
        std::vector<double> S, mu;
        axis_basis(N, g.periodic != 0, S, mu);
        for (auto& v : mu) v *= g.inv_h2();     // scale / h^2: the kinetic operator's eigenvalues
        std::vector<double> St(N * N);
        for (int64_t p = 0; p < N; ++p)
            for (int64_t m = 0; m < N; ++m) St[m * N + p] = S[p * N + m];
        if (cudaMalloc(&P.d_S[a], sizeof(double) * N * N) != cudaSuccess ||
            cudaMalloc(&P.d_St[a], sizeof(double) * N * N) != cudaSuccess ||
            cudaMalloc(&P.d_mu[a], sizeof(double) * N) != cudaSuccess) {
            set_error("plhr_prec_tpa: cudaMalloc failed");
            plhr_prec_destroy(T);
            return PLHR_ENOMEM;
        }
        if (cudaMemcpy(P.d_S[a], S.data(), sizeof(double) * N * N, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(P.d_St[a], St.data(), sizeof(double) * N * N, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(P.d_mu[a], mu.data(), sizeof(double) * N, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("plhr_prec_tpa: upload failed");
            plhr_prec_destroy(T);
            return PLHR_ECUDA;
        }
        const int shm = (int)(sizeof(double) * N * N);
        if (shm > 48 * 1024) {
            if (cudaFuncSetAttribute(k_axis<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm) != cudaSuccess ||
                cudaFuncSetAttribute(k_axis<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm) != cudaSuccess) {
                set_error("plhr_prec_tpa: shared-memory attribute failed");
                plhr_prec_destroy(T);
                return PLHR_ECUDA;
            }
        }
    }
    *out = T;
    return PLHR_OK;
}

extern "C" double plhr_prec_tpa_energy(const plhr_prec* T) {
    return (T && T->kind == PREC_TPA) ? T->sp.energy : 0.0;
}
