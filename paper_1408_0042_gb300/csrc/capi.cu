// C ABI: error state, stencil operators, the AV-MG preconditioner object.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "plhr_internal.h"

namespace plhr {

namespace {
thread_local char g_err[512] = {0};
}

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

int sm_count() {
    static int cached = 0;
    if (cached == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            cached = v;
        else
            cached = 132;
    }
    return cached;
}

}  // namespace plhr

using namespace plhr;

extern "C" {

const char* plhr_last_error(void) { return g_err; }

const char* plhr_status_string(plhr_status s) {
    switch (s) {
        case PLHR_OK: return "ok";
        case PLHR_ENOTCONV: return "not converged within maxit";
        case PLHR_EINVAL: return "invalid argument";
        case PLHR_EBREAKDOWN: return "breakdown of the projected problem";
        case PLHR_ENAN: return "NaN or Inf in the iteration";
        case PLHR_ENOMEM: return "device allocation failed";
        case PLHR_ECUDA: return "CUDA error";
    }
    return "unknown status";
}

plhr_status plhr_op_stencil(plhr_op** out, const plhr_stencil_desc* d) {
    clear_error();
    if (!out || !d) { set_error("plhr_op_stencil: null argument"); return PLHR_EINVAL; }
    const int kind = d->kind;
    if (kind < PLHR_STENCIL_LAP5_2D || kind > PLHR_STENCIL_Q1_MASS27) {
        set_error("plhr_op_stencil: unknown kind %d", kind);
        return PLHR_EINVAL;
    }
    if (d->dims[0] < 1 || d->dims[1] < 1 || d->dims[2] < 1 || !(d->h > 0) || !std::isfinite(d->h)) {
        set_error("plhr_op_stencil: bad dims/h");
        return PLHR_EINVAL;
    }
    if (kind != PLHR_STENCIL_HAM7_BLOCH && !(d->scale > 0 && std::isfinite(d->scale))) {
        set_error("plhr_op_stencil: scale must be positive and finite");
        return PLHR_EINVAL;
    }
    if (kind == PLHR_STENCIL_LAP5_2D && d->dims[2] != 1) {
        set_error("plhr_op_stencil: 2D stencil needs dims[2] == 1");
        return PLHR_EINVAL;
    }
    if ((kind == PLHR_STENCIL_LAP5_2D || kind == PLHR_STENCIL_LAP7_3D) && d->bc != PLHR_BC_DIRICHLET &&
        d->bc != PLHR_BC_PERIODIC) {
        set_error("plhr_op_stencil: unknown boundary condition %d", d->bc);
        return PLHR_EINVAL;
    }
    if (kind == PLHR_STENCIL_HAM7_BLOCH) {
        if (!d->field) { set_error("plhr_op_stencil: HAM7_BLOCH needs the potential (field)"); return PLHR_EINVAL; }
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(d->bloch_k[a])) { set_error("plhr_op_stencil: bloch_k not finite"); return PLHR_EINVAL; }
    }
    plhr_op* op = new plhr_op;
    op->kind = kind;
    op->g.d = kind == PLHR_STENCIL_LAP5_2D ? 2 : 3;
    op->g.nx = d->dims[0];
    op->g.ny = d->dims[1];
    op->g.nz = d->dims[2];
    op->g.h = d->h;
    op->g.scale = d->scale;
    switch (kind) {
        case PLHR_STENCIL_LAP5_2D:
        case PLHR_STENCIL_LAP7_3D:
            op->g.periodic = d->bc == PLHR_BC_PERIODIC;
            break;
        case PLHR_STENCIL_HAM7_BLOCH:
            op->g.scale = 0.5;
            op->g.periodic = 1;
            op->g.pot = d->field;
            for (int a = 0; a < 3; ++a) op->g.kappa[a] = d->bloch_k[a];
            break;
        case PLHR_STENCIL_Q1_STIFF27:
            op->g.q1 = 1;
            op->g.cell = d->field;
            break;
        case PLHR_STENCIL_Q1_MASS27:
            op->g.q1 = 2;
            break;
    }
    *out = op;
    return PLHR_OK;
}

plhr_status plhr_op_hamiltonian(plhr_op** out, int d, const int64_t* dims, double h, int periodic,
                                const double* potential) {
    clear_error();
    if (!out || !dims || (d != 2 && d != 3) || !(h > 0)) {
        set_error("plhr_op_hamiltonian: invalid argument");
        return PLHR_EINVAL;
    }
    if (dims[0] < 1 || dims[1] < 1 || (d == 3 && dims[2] < 1)) {
        set_error("plhr_op_hamiltonian: bad dims");
        return PLHR_EINVAL;
    }
    plhr_op* op = new plhr_op;
    op->kind = d == 3 ? PLHR_STENCIL_LAP7_3D : PLHR_STENCIL_LAP5_2D;
    op->g.d = d;
    op->g.nx = dims[0];
    op->g.ny = dims[1];
    op->g.nz = d == 3 ? dims[2] : 1;
    op->g.h = h;
    op->g.scale = 0.5;
    op->g.periodic = periodic ? 1 : 0;
    op->g.pot = potential;
    *out = op;
    return PLHR_OK;
}

int64_t plhr_op_size(const plhr_op* op) { return op ? op->g.n() : 0; }

void plhr_op_destroy(plhr_op* op) {
    if (!op) return;
    if (op->csr.rowptr || op->csr.col || op->csr.val) {
        cudaDeviceSynchronize();   // queued products may still read the arrays
        if (op->csr.rowptr) cudaFree(op->csr.rowptr);
        if (op->csr.col) cudaFree(op->csr.col);
        if (op->csr.val) cudaFree(op->csr.val);
    }
    delete op;
}

plhr_status plhr_op_apply(const plhr_op* op, int ncols, const double* X, int64_t ldx, double* Y, int64_t ldy,
                          void* stream) {
    clear_error();
    if (!op || ncols < 0 || (ncols > 0 && (!X || !Y)) || ldx < ncols || ldy < ncols) {
        set_error("plhr_op_apply: invalid argument");
        return PLHR_EINVAL;
    }
    if (op->g.complex_op()) {
        set_error("plhr_op_apply: a Bloch operator with kappa != 0 is complex (use plhr_op_apply_c128)");
        return PLHR_EINVAL;
    }
    if (ncols == 0) return PLHR_OK;
    PLHR_TRY_CUDA(lap_axpby(op->g, ncols, X, ldx, Y, ldy, 1.0, 0.0, (cudaStream_t)stream));
    return PLHR_OK;
}

plhr_status plhr_op_apply_c128(const plhr_op* op, int ncols, const double* X, int64_t ldx, double* Y, int64_t ldy,
                               void* stream) {
    clear_error();
    if (!op || ncols < 0 || (ncols > 0 && (!X || !Y)) || ldx < ncols || ldy < ncols) {
        set_error("plhr_op_apply_c128: invalid argument");
        return PLHR_EINVAL;
    }
    if (op->g.csr) {
        set_error("plhr_op_apply_c128: stencil operators only");
        return PLHR_EINVAL;
    }
    if (ncols == 0) return PLHR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (op->g.complex_op()) {
        PLHR_TRY_CUDA(bloch_apply(op->g, ncols, X, ldx, Y, ldy, s));
    } else {
        // a real operator acts on the real and imaginary parts alike: the
        // interleaved block is a real block of 2 ncols columns
        PLHR_TRY_CUDA(lap_axpby(op->g, 2 * ncols, X, 2 * ldx, Y, 2 * ldy, 1.0, 0.0, s));
    }
    return PLHR_OK;
}

plhr_status plhr_op_apply_pair(const plhr_op* A, const plhr_op* B, int ncols, const double* X, int64_t ldx,
                               double* AX, int64_t ldax, double* BX, int64_t ldbx, void* stream) {
    clear_error();
    if (!A || !B || ncols < 0 || (ncols > 0 && (!X || !AX || !BX)) || ldx < ncols || ldax < ncols ||
        ldbx < ncols || A->g.n() != B->g.n()) {
        set_error("plhr_op_apply_pair: invalid argument");
        return PLHR_EINVAL;
    }
    if (A->g.complex_op() || B->g.complex_op()) {
        set_error("plhr_op_apply_pair: real operators only");
        return PLHR_EINVAL;
    }
    if (ncols == 0) return PLHR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (q1_same_mesh(A->g, B->g)) {
        PLHR_TRY_CUDA(q1_pair(A->g, B->g, ncols, X, ldx, AX, ldax, BX, ldbx, s));
    } else {
        PLHR_TRY_CUDA(lap_axpby(A->g, ncols, X, ldx, AX, ldax, 1.0, 0.0, s));
        PLHR_TRY_CUDA(lap_axpby(B->g, ncols, X, ldx, BX, ldbx, 1.0, 0.0, s));
    }
    return PLHR_OK;
}

void plhr_mg_opts_default(plhr_mg_opts* o) {
    if (!o) return;
    o->levels = 1;
    o->nu = 2;
    o->delta = 2.0 * M_PI / 10.0;
    o->transfer = 0;
    o->coarse = 0;
    o->indefinite = 0;
}

plhr_status plhr_prec_avmg(plhr_prec** out, const plhr_op* A, double sigma, const plhr_mg_opts* opts) {
    clear_error();
    plhr_mg_opts o;
    plhr_mg_opts_default(&o);
    if (opts) o = *opts;
    if (!out || !A) { set_error("plhr_prec_avmg: null argument"); return PLHR_EINVAL; }
    if (o.levels < 1 || o.nu < 1 || !(o.delta > 0) || (o.transfer != 0 && o.transfer != 1) ||
        (o.coarse != 0 && o.coarse != 1) || (o.indefinite != 0 && o.indefinite != 1) || !std::isfinite(sigma)) {
        set_error("plhr_prec_avmg: bad options");
        return PLHR_EINVAL;
    }
    const Grid& g = A->g;
    if (!g.plain()) {
        // the level operators are rediscretised Dirichlet Laplacians
        set_error("plhr_prec_avmg: A must be a Dirichlet Laplacian (plhr_op_stencil)");
        return PLHR_EINVAL;
    }
    const int64_t f = (int64_t)1 << (o.levels - 1);
    if (g.nx % f || g.ny % f || (g.d == 3 && g.nz % f)) {
        set_error("plhr_prec_avmg: axis sizes must be divisible by 2^(levels-1) = %lld", (long long)f);
        return PLHR_EINVAL;
    }
    plhr_prec* T = new plhr_prec;
    MGHierarchy& H = T->H;
    H.dim = g.d;
    H.nu = o.nu;
    H.linear = o.transfer;
    H.indefinite = o.indefinite;
    H.sigma = sigma;
    H.lev.resize(o.levels);
    for (int l = o.levels - 1, s = 0; l >= 0; --l, ++s) {
        MGLevel& L = H.lev[l];
        int64_t sc = (int64_t)1 << s;
        L.g = g;
        L.g.nx = g.nx / sc;
        L.g.ny = g.ny / sc;
        L.g.nz = g.d == 3 ? g.nz / sc : 1;
        L.g.h = g.h * (double)sc;
        // Gershgorin interval of L_l - sigma I: [-sigma, 4 d scale / h_l^2 - sigma]
        double a = -sigma, b = 4.0 * g.d * L.g.inv_h2() - sigma;
        L.poly = !(std::sqrt(std::fmax(sigma, 0.0)) * L.g.h < o.delta);
        if (o.indefinite) {
            // INV-MG: B_l = L_l - sigma I, Richardson step 1 / max(|a|, |b|)
            L.poly = false;
            L.shifted = true;
            L.c = 0.0;
            L.omega = 1.0 / std::fmax(std::fabs(a), std::fabs(b));
        } else if (L.poly) {
            L.c = 0.5 * std::fmax(std::fabs(a), std::fabs(b));
            double beta = (std::fmax(a * a, b * b) + L.c * L.c) / (2.0 * L.c);
            L.omega = 1.0 / beta;
        } else {
            L.c = 0.0;
            L.omega = 1.0 / (4.0 * g.d * L.g.inv_h2());
        }
    }
    // coarsest separable basis and eigenvalues per axis
    const Grid& g0 = H.lev[0].g;
    int64_t N0[3] = {g0.nx, g0.ny, g0.nz};
    int64_t Nf[3] = {g.nx, g.ny, g.nz};
    for (int ax = 0; ax < g.d; ++ax) {
        int64_t N = N0[ax];
        std::vector<double> S(N * N), mu(N);
        for (int64_t m = 0; m < N; ++m) {
            if (o.coarse == 0) {
                mu[m] = 4.0 * g0.inv_h2() * std::pow(std::sin((m + 1) * M_PI / (2.0 * (N + 1))), 2);
                for (int64_t p = 0; p < N; ++p)
                    S[p * N + m] = std::sqrt(2.0 / (N + 1)) * std::sin((p + 1) * (m + 1) * M_PI / (N + 1));
            } else {
                mu[m] = 4.0 * g.inv_h2() * std::pow(std::sin((m + 1) * M_PI / (2.0 * (Nf[ax] + 1))), 2);
                double nrm = (m == N - 1) ? std::sqrt(1.0 / N) : std::sqrt(2.0 / N);
                for (int64_t p = 0; p < N; ++p) S[p * N + m] = nrm * std::sin((p + 0.5) * (m + 1) * M_PI / N);
            }
        }
        if (cudaMalloc(&H.d_basis[ax], sizeof(double) * N * N) != cudaSuccess ||
            cudaMalloc(&H.d_mu[ax], sizeof(double) * N) != cudaSuccess) {
            set_error("plhr_prec_avmg: cudaMalloc failed");
            plhr_prec_destroy(T);
            return PLHR_ENOMEM;
        }
        if (cudaMemcpy(H.d_basis[ax], S.data(), sizeof(double) * N * N, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(H.d_mu[ax], mu.data(), sizeof(double) * N, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("plhr_prec_avmg: upload failed");
            plhr_prec_destroy(T);
            return PLHR_ECUDA;
        }
        std::vector<float> Sw(2 * N * N), muw(2 * N);
        for (int64_t q = 0; q < N * N; ++q) {
            Sw[2 * q] = (float)S[q];
            Sw[2 * q + 1] = (float)(S[q] - (double)Sw[2 * q]);
        }
        for (int64_t q = 0; q < N; ++q) {
            muw[2 * q] = (float)mu[q];
            muw[2 * q + 1] = (float)(mu[q] - (double)muw[2 * q]);
        }
        if (cudaMalloc(&H.w_basis[ax], sizeof(float) * 2 * N * N) != cudaSuccess ||
            cudaMalloc(&H.w_mu[ax], sizeof(float) * 2 * N) != cudaSuccess ||
            cudaMemcpy(H.w_basis[ax], Sw.data(), sizeof(float) * 2 * N * N, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(H.w_mu[ax], muw.data(), sizeof(float) * 2 * N, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("plhr_prec_avmg: double-word basis upload failed");
            plhr_prec_destroy(T);
            return PLHR_ENOMEM;
        }
        std::vector<float> Sf(S.begin(), S.end()), muf(mu.begin(), mu.end());
        if (cudaMalloc(&H.f_basis[ax], sizeof(float) * N * N) != cudaSuccess ||
            cudaMalloc(&H.f_mu[ax], sizeof(float) * N) != cudaSuccess ||
            cudaMemcpy(H.f_basis[ax], Sf.data(), sizeof(float) * N * N, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(H.f_mu[ax], muf.data(), sizeof(float) * N, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("plhr_prec_avmg: FP32 basis upload failed");
            plhr_prec_destroy(T);
            return PLHR_ENOMEM;
        }
        H.n0[ax] = N;
    }
    // a coarsest grid above kMaxSmemCoarse points is solved with global
    // scratch by the FP64 cycle; the FP32 and double-word cycles (the mixed
    // form) stage it in shared memory and refuse larger grids
    (void)g0;
    *out = T;
    return PLHR_OK;
}

void plhr_prec_destroy(plhr_prec* T) {
    if (!T) return;
    cudaDeviceSynchronize();   // queued V-cycles may still read the hierarchy and workspace
    mg_release_graphs(T->H);
    if (T->H.capture) cudaStreamDestroy(T->H.capture);
    for (int a = 0; a < 3; ++a) {
        if (T->sp.d_S[a]) cudaFree(T->sp.d_S[a]);
        if (T->sp.d_St[a]) cudaFree(T->sp.d_St[a]);
        if (T->H.d_basis[a]) cudaFree(T->H.d_basis[a]);
        if (T->H.d_mu[a]) cudaFree(T->H.d_mu[a]);
        if (T->H.f_basis[a]) cudaFree(T->H.f_basis[a]);
        if (T->H.f_mu[a]) cudaFree(T->H.f_mu[a]);
        if (T->H.w_basis[a]) cudaFree(T->H.w_basis[a]);
        if (T->H.w_mu[a]) cudaFree(T->H.w_mu[a]);
    }
    if (T->diag) cudaFree(T->diag);
    if (T->sp.d_K) cudaFree(T->sp.d_K);
    if (T->work) cudaFree(T->work);
    if (T->work32) cudaFree(T->work32);
    delete T;
}

}  // extern "C"

namespace plhr {
plhr_status prec_reserve(plhr_prec* T, int nc, int64_t extra_doubles) {
    int64_t need = prec_workspace_doubles(T, nc) + extra_doubles;
    if (need <= T->work_doubles) return PLHR_OK;
    if (T->work) {
        cudaDeviceSynchronize();
        mg_release_graphs(T->H);   // they hold the old workspace's addresses
        cudaFree(T->work);
        T->work = nullptr;
        T->work_doubles = 0;
    }
    if (need == 0) return PLHR_OK;
    if (cudaMalloc(&T->work, sizeof(double) * need) != cudaSuccess) {
        set_error("prec workspace: cudaMalloc of %lld doubles failed", (long long)need);
        return PLHR_ENOMEM;
    }
    T->work_doubles = need;
    return PLHR_OK;
}
plhr_status prec_reserve32(plhr_prec* T, int nc, int64_t extra_floats) {
    int64_t need = mg_workspace_floats(T->H, nc) + extra_floats;
    if (need <= T->work_floats) return PLHR_OK;
    if (T->work32) {
        cudaDeviceSynchronize();
        mg_release_graphs(T->H);
        cudaFree(T->work32);
        T->work32 = nullptr;
        T->work_floats = 0;
    }
    if (need == 0) return PLHR_OK;
    if (cudaMalloc(&T->work32, sizeof(float) * need) != cudaSuccess) {
        set_error("prec FP32 workspace: cudaMalloc of %lld floats failed", (long long)need);
        return PLHR_ENOMEM;
    }
    T->work_floats = need;
    return PLHR_OK;
}
plhr_status prec_reserve_dw(plhr_prec* T, int nc) {
    // the double-word V-cycle uses T->work (8-byte entries); it never runs at
    // the same time as the FP64 one
    const int64_t need = mg_workspace_dw(T->H, nc);
    const int64_t have_nc = T->work_doubles;
    if (need <= have_nc) return PLHR_OK;
    return prec_reserve(T, nc, need - mg_workspace_doubles(T->H, nc));
}
}  // namespace plhr

extern "C" plhr_status plhr_prec_apply_dw(plhr_prec* T, int ncols, const double* R, int64_t ldr, double* W,
                                          int64_t ldw, void* stream) {
    clear_error();
    if (!T || ncols < 0 || (ncols > 0 && (!R || !W)) || ldr < ncols || ldw < ncols) {
        set_error("plhr_prec_apply_dw: invalid argument");
        return PLHR_EINVAL;
    }
    if (T->kind != PREC_AVMG || T->H.indefinite || T->H.lev[0].g.n() > kMaxSmemCoarse) {
        set_error("plhr_prec_apply_dw: double-word form exists for AV-MG only");
        return PLHR_EINVAL;
    }
    if (ncols == 0) return PLHR_OK;
    PLHR_TRY(plhr::prec_reserve_dw(T, ncols));
    PLHR_TRY_CUDA(plhr::mg_vcycle_dw(T->H, ncols, R, ldr, W, ldw, T->work, (cudaStream_t)stream));
    return PLHR_OK;
}

extern "C" plhr_status plhr_prec_apply_f32(plhr_prec* T, int ncols, const float* R, int64_t ldr, float* W,
                                           int64_t ldw, void* stream) {
    clear_error();
    if (!T || ncols < 0 || (ncols > 0 && (!R || !W)) || ldr < ncols || ldw < ncols) {
        set_error("plhr_prec_apply_f32: invalid argument");
        return PLHR_EINVAL;
    }
    if (T->kind != PREC_AVMG || T->H.indefinite || T->H.lev[0].g.n() > kMaxSmemCoarse) {
        set_error("plhr_prec_apply_f32: FP32 form exists for AV-MG only");
        return PLHR_EINVAL;
    }
    if (ncols == 0) return PLHR_OK;
    const int64_t n = T->H.lev.back().g.n();
    const int64_t stage = (ldw == ncols) ? 0 : n * ncols;
    PLHR_TRY(prec_reserve32(T, ncols, stage));
    cudaStream_t s = (cudaStream_t)stream;
    float* out = (ldw == ncols) ? W : T->work32 + mg_workspace_floats(T->H, ncols);
    PLHR_TRY_CUDA(mg_vcycle_f32(T->H, ncols, R, ldr, out, T->work32, s));
    if (ldw != ncols)
        PLHR_TRY_CUDA(cudaMemcpy2DAsync(W, sizeof(float) * ldw, out, sizeof(float) * ncols, sizeof(float) * ncols,
                                        n, cudaMemcpyDeviceToDevice, s));
    return PLHR_OK;
}

extern "C" plhr_status plhr_prec_apply(plhr_prec* T, int ncols, const double* R, int64_t ldr, double* W, int64_t ldw,
                                       void* stream) {
    clear_error();
    if (!T || ncols < 0 || (ncols > 0 && (!R || !W)) || ldr < ncols || ldw < ncols) {
        set_error("plhr_prec_apply: invalid argument");
        return PLHR_EINVAL;
    }
    if (ncols == 0) return PLHR_OK;
    const int64_t n = prec_size(T);
    const int64_t stage = (ldw == ncols) ? 0 : n * ncols;
    PLHR_TRY(prec_reserve(T, ncols, stage));
    cudaStream_t s = (cudaStream_t)stream;
    double* out = (ldw == ncols) ? W : T->work + prec_workspace_doubles(T, ncols);
    PLHR_TRY(prec_apply64(T, ncols, R, ldr, out, T->work, s));
    if (ldw != ncols)
        PLHR_TRY_CUDA(cudaMemcpy2DAsync(W, sizeof(double) * ldw, out, sizeof(double) * ncols, sizeof(double) * ncols,
                                        n, cudaMemcpyDeviceToDevice, s));
    return PLHR_OK;
}
