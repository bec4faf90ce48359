// Internal declarations shared by the translation units of libplhr.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <vector>

#include "plhr.h"

namespace plhr {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
void clear_error();

#define PLHR_TRY_CUDA(call)                                                    \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            ::plhr::set_error("%s failed: %s (%s:%d)", #call,                  \
                              cudaGetErrorString(e_), __FILE__, __LINE__);     \
            return PLHR_ECUDA;                                                 \
        }                                                                      \
    } while (0)

#define PLHR_TRY(expr)                                                         \
    do {                                                                       \
        plhr_status s_ = (expr);                                               \
        if (s_ != PLHR_OK) return s_;                                          \
    } while (0)

// Launch check: the kernel launch itself (configuration) failed.
#define PLHR_LAUNCHED() PLHR_TRY_CUDA(cudaGetLastError())

// ---------------------------------------------------------------- grids
enum { OP_KIND_CSR = 100 };   // plhr_op::kind of a CSR operator (stencil kinds are plhr_stencil_kind)

// A general sparse symmetric operator in CSR form (device arrays owned by the
// plhr_op that holds them).
struct CsrData {
    int64_t n = 0, nnz = 0;
    int64_t* rowptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
};

// Tensor grid, x fastest, homogeneous Dirichlet boundary (or periodic), with
// an optional diagonal potential.  With csr set the operator is that sparse
// matrix instead (nx = n, no stencil).
struct Grid {
    int d = 3;            // 2 or 3
    int64_t nx = 1, ny = 1, nz = 1;
    double h = 1.0;
    double scale = 1.0;   // stencil multiplier
    int periodic = 0;     // 1: periodic wrap instead of zero Dirichlet values
    const double* pot = nullptr;   // optional diagonal term (device, n values): A = scale L + diag(pot)
    const CsrData* csr = nullptr;  // general sparse operator instead of the stencil
    int q1 = 0;                    // 1: Q1 stiffness, 2: Q1 mass (27-point finite-element stencils)
    const double* cell = nullptr;  // Q1 stiffness: element coefficients ((nx+1)(ny+1)(nz+1)) or null (1)
    double kappa[3] = {0.0, 0.0, 0.0};   // Bloch phases e^{i kappa_d h} on the links (periodic Hamiltonian)
    int64_t n() const { return nx * ny * nz; }
    double inv_h2() const { return scale / (h * h); }
    bool complex_op() const { return kappa[0] != 0.0 || kappa[1] != 0.0 || kappa[2] != 0.0; }
    // the Dirichlet finite-difference Laplacian
    bool plain() const { return !periodic && pot == nullptr && csr == nullptr && q1 == 0 && !complex_op(); }
};

// A block of row-major vectors: element (i, j) at p[i * ld + j].
template <typename T>
struct Blk {
    T* p = nullptr;
    int64_t ld = 0;
    int nc = 0;
};

inline int grid_size_for(int64_t work, int threads, int max_blocks) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

int sm_count();

// Kernel launches issued by the library (all entry points, process-wide).
void count_launches(int n);

// Optional phase timing with CUDA events on the launching stream.
enum Phase { PH_STENCIL = 0, PH_VCYCLE = 1, PH_GRAM = 2, PH_UPDATE = 3, PH_DENSE = 4, PH_OTHER = 5,
             PH_VCYCLE32 = 6, PH_GRAM32 = 7, PH_UPDATE32 = 8, PH_COUNT = 9 };
struct PhaseScope {
    // work: algorithmic work of the call, in the phase's unit (see plhr_profile_work);
    // bytes: algorithmic HBM bytes of the call (each operand read or written once)
    PhaseScope(int phase, cudaStream_t s, double work = 0.0, double bytes = 0.0);
    ~PhaseScope();
    int phase;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
};
void profile_flush();   // accumulate finished event pairs (synchronises their events)

// ---------------------------------------------------------------- stencil
// y = alpha * L x + beta * x   (L: scaled Dirichlet Laplacian of g)
cudaError_t lap_axpby(const Grid& g, int nc, const double* x, int64_t ldx, double* y,
                      int64_t ldy, double alpha, double beta, cudaStream_t s);
// ax = L x; o1 = ax - x * diag(lam) (optional); o2 = ax - sig * x (optional)
cudaError_t lap_apply_shifts(const Grid& g, int nc, const double* x, int64_t ldx,
                             double* ax, int64_t ldax, double* o1, int64_t ld1,
                             const double* lam, double* o2, int64_t ld2, double sig,
                             cudaStream_t s);

// the same two entry points for a CSR operator (csr.cu)
cudaError_t csr_axpby(const CsrData& A, int nc, const double* x, int64_t ldx, double* y, int64_t ldy, double alpha,
                      double beta, cudaStream_t s);
cudaError_t csr_apply_shifts(const CsrData& A, int nc, const double* x, int64_t ldx, double* ax, int64_t ldax,
                             double* o1, int64_t ld1, const double* lam, double* o2, int64_t ld2, double sig,
                             cudaStream_t s);

// Q1 finite-element stencils (q1.cu): a single operator (stiffness or mass by
// g.q1) as y = alpha op x + beta x or with the shifted outputs; both
// operators of a mesh in one pass (ax = A x, bx = B x)
cudaError_t q1_axpby(const Grid& g, int nc, const double* x, int64_t ldx, double* y, int64_t ldy, double alpha,
                     double beta, cudaStream_t s);
cudaError_t q1_apply_shifts(const Grid& g, int nc, const double* x, int64_t ldx, double* ax, int64_t ldax,
                            double* o1, int64_t ld1, const double* lam, double* o2, int64_t ld2, double sig,
                            cudaStream_t s);
cudaError_t q1_pair(const Grid& A, const Grid& B, int nc, const double* x, int64_t ldx, double* ax, int64_t ldax,
                    double* bx, int64_t ldbx, cudaStream_t s);
bool q1_same_mesh(const Grid& A, const Grid& B);
// Bloch Hamiltonian on complex128 blocks (ld in complex elements)
cudaError_t bloch_apply(const Grid& g, int nc, const double* x, int64_t ldx, double* y, int64_t ldy, cudaStream_t s);

// ---------------------------------------------------------------- multigrid
struct MGLevel {
    Grid g;
    bool poly = false;    // B_l = p_2(L_l - sigma I) instead of L_l
    bool shifted = false; // B_l = L_l - sigma I (INV-MG)
    double c = 0.0;       // p_2 parameter
    double omega = 0.0;   // Richardson step 1 / beta_l
};

struct MGHierarchy {
    int dim = 3;
    int nu = 2;
    int linear = 0;                    // 1: trilinear cell-centred transfers, 0: piecewise constant
    int indefinite = 0;                // 1: INV-MG (Algorithm 5), T ~ (L - sigma I)^{-1}
    double sigma = 0.0;
    std::vector<MGLevel> lev;          // 0 = coarsest
    // coarsest solve: w = S3 diag(1/|mu_i + mu_j + mu_k - sigma|) S3^T r with
    // S3 = Sx (x) Sy (x) Sz (orthonormal 1D bases) and 1D eigenvalues mu
    double* d_basis[3] = {nullptr, nullptr, nullptr};   // N_a x N_a, row-major [point][mode]
    double* d_mu[3] = {nullptr, nullptr, nullptr};
    float* f_basis[3] = {nullptr, nullptr, nullptr};   // FP32 copies for the FP32 V-cycle
    float* f_mu[3] = {nullptr, nullptr, nullptr};
    float* w_basis[3] = {nullptr, nullptr, nullptr};   // double-word (hi, lo) copies for the
    float* w_mu[3] = {nullptr, nullptr, nullptr};      // double-word V-cycle
    int64_t n0[3] = {1, 1, 1};
    // V-cycles captured as CUDA graphs, keyed by their arguments, and replayed
    // instead of issuing their ~35 launches again (mg_graphed)
    struct Graph {
        int kind, nc;
        const void* r;
        int64_t ldr;
        const void* w;
        int64_t ldw;
        const void* work;
        const void* r2;   // second right-hand side (paired cycles), else null
        int64_t ldr2;
        int nc2;
        cudaGraphExec_t exec;
        int launches;
    };
    mutable std::vector<Graph> graphs;
    mutable cudaStream_t capture = nullptr;   // non-default stream the captures run on
};

// Run body (the launches of one V-cycle, issued on the stream it is given)
// on s: the first call with a given (kind, nc, r, ldr, w, ldw, work) captures
// it into a CUDA graph, later calls replay the graph.  Falls back to issuing
// body on s directly when a capture fails or the cache is full.  The launch
// counter counts the graph's kernels on every replay.
cudaError_t mg_graphed(const MGHierarchy& H, int kind, int nc, const void* r, int64_t ldr, const void* w,
                       int64_t ldw, const void* work, cudaStream_t s,
                       const std::function<cudaError_t(cudaStream_t)>& body, const void* r2 = nullptr,
                       int64_t ldr2 = 0, int nc2 = 0);
// Destroy the captured graphs (the hierarchy's buffers or workspace change
// or go away).
void mg_release_graphs(const MGHierarchy& H);

// Largest coarsest grid (points) of the FP32 and double-word V-cycles, whose
// coarsest solve stages the grid in shared memory (the FP64 cycle takes any
// size: above this it works in global scratch).
constexpr int64_t kMaxSmemCoarse = 12288;

cudaError_t mg_vcycle(const MGHierarchy& H, int nc, const double* r, int64_t ldr, double* w,
                      int64_t ldw, double* work, cudaStream_t s);
int64_t mg_workspace_doubles(const MGHierarchy& H, int nc);

// ---------------------------------------------------------------- TPA preconditioner
// T = S diag(K(mu / energy)) S^T with S the separable orthonormal modes of the
// grid's kinetic operator (spectral.cu)
struct SpecPrec {
    int d = 3;
    int64_t nx = 1, ny = 1, nz = 1;
    double energy = 1.0;
    // double-word (hi, lo) FP32 pairs
    float* d_S[3] = {nullptr, nullptr, nullptr};     // N_a x N_a, [point][mode]
    float* d_St[3] = {nullptr, nullptr, nullptr};    // transposes
    float* d_K = nullptr;                            // factor K(mu / energy) per 3D mode (n pairs)
    int64_t n() const { return nx * ny * nz; }
};
cudaError_t spectral_apply(const SpecPrec& P, int nc, const double* r, int64_t ldr, double* w, double* work,
                           cudaStream_t s);
int64_t spectral_workspace_doubles(const SpecPrec& P, int nc);

enum { PREC_AVMG = 0, PREC_TPA = 1, PREC_DIAG = 2, PREC_CALLBACK = 3 };

// FP32 V-cycle (same cycle, FP32 storage and arithmetic); r is FP64 or FP32
// with leading dimension ldr, w is dense (leading dimension nc).
cudaError_t mg_vcycle_f32(const MGHierarchy& H, int nc, const double* r, int64_t ldr, float* w, float* work,
                          cudaStream_t s);
cudaError_t mg_vcycle_f32(const MGHierarchy& H, int nc, const float* r, int64_t ldr, float* w, float* work,
                          cudaStream_t s);
// w (n x (nc1 + nc2), dense) = [T r1 | T r2] in one FP32 cycle of nc1 + nc2
// columns (r1, r2 FP64; work: mg_workspace_floats(H, nc1 + nc2))
cudaError_t mg_vcycle_f32_pair(const MGHierarchy& H, int nc1, const double* r1, int64_t ldr1, int nc2,
                               const double* r2, int64_t ldr2, float* w, float* work, cudaStream_t s);
int64_t mg_workspace_floats(const MGHierarchy& H, int nc);

// Double-word V-cycle (same cycle; hi + lo FP32 pairs, ~48-bit arithmetic on
// the FP32 pipes): w (FP64, ldw) = T r (FP64, ldr); work: mg_workspace_dw(H, nc)
// 8-byte entries.
cudaError_t mg_vcycle_dw(const MGHierarchy& H, int nc, const double* r, int64_t ldr, double* w, int64_t ldw,
                         void* work, cudaStream_t s);
int64_t mg_workspace_dw(const MGHierarchy& H, int nc);

}  // namespace plhr

struct plhr_op {
    int kind;
    plhr::Grid g;
    plhr::CsrData csr;   // owned arrays of a CSR operator (g.csr points here)
};

struct plhr_prec {
    int kind = plhr::PREC_AVMG;
    plhr::MGHierarchy H;          // PREC_AVMG
    plhr::SpecPrec sp;            // PREC_TPA
    double* diag = nullptr;       // PREC_DIAG: positive diagonal (device, owned)
    plhr_apply_fn fn = nullptr;   // PREC_CALLBACK: the caller's T
    void* ctx = nullptr;
    int64_t n_user = 0;           // size for PREC_DIAG / PREC_CALLBACK
    double* work = nullptr;
    int64_t work_doubles = 0;
    float* work32 = nullptr;      // FP32 V-cycle workspace
    int64_t work_floats = 0;
};

namespace plhr {
// FP64 application of either preconditioner kind: w (dense, ld nc) = T r;
// work: prec_workspace_doubles(T, nc) doubles
inline int64_t prec_size(const plhr_prec* T) {
    if (T->kind == PREC_TPA) return T->sp.n();
    if (T->kind == PREC_DIAG || T->kind == PREC_CALLBACK) return T->n_user;
    return T->H.lev.back().g.n();
}
inline int64_t prec_workspace_doubles(const plhr_prec* T, int nc) {
    if (T->kind == PREC_TPA) return spectral_workspace_doubles(T->sp, nc);
    if (T->kind == PREC_DIAG || T->kind == PREC_CALLBACK) return 0;
    return mg_workspace_doubles(T->H, nc);
}
// any kind (precs.cu); sets the error message on failure
plhr_status prec_apply64(const plhr_prec* T, int nc, const double* r, int64_t ldr, double* w, double* work,
                         cudaStream_t s);
}  // namespace plhr

#ifdef __CUDACC__
namespace plhr {
// row = e / nc and col = e - row nc for a flat index e of a row-major n x nc
// block: a 32-bit division while e fits in 32 bits (a 64-bit division is a
// long instruction sequence on the GPU), the 64-bit one past that
__device__ __forceinline__ void split_index(int64_t e, int nc, int64_t& row, int& col) {
    if ((uint64_t)e <= 0xffffffffull) {
        const unsigned q = (unsigned)e / (unsigned)nc;
        row = (int64_t)q;
        col = (int)((unsigned)e - q * (unsigned)nc);
    } else {
        row = e / nc;
        col = (int)(e - row * nc);
    }
}
}  // namespace plhr
#endif
