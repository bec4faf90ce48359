// Block PLHR driver (Algorithm 3, real arithmetic; FP64 and mixed precision).  Every step of
// the iteration runs on the device; the host enqueues kernels and reads one
// small status record per iteration (convergence flags, Ritz values).
//
// Stored state (n rows each, row-major):
//   V, AV, QV      current block and its images A V, T(A - sigma B) V (k' columns,
//                  stored unnormalised; `scale` holds the B-normalising factors
//                  of Alg. 3 step 14, applied wherever V is used)
//   P, AP, QP      conjugate directions and images (k' columns, absent at it 0)
//   W, AW          preconditioned residuals of the active columns (Alg. 3 step 4)
//   SQ = [S | Q_W] s-vectors (step 5) and T(A - sigma B) W, one 2 n_a-wide V-cycle
//   AS, QS         A S and T(A - sigma B) S
// Per iteration: 2 block products with A (W, S) and 4 applications of T
// (W, S, Q_W, Q_S), as in the storage/cost paragraph after Algorithm 2.
//
// Mixed precision (PLHR_PRECISION_MIXED): while the relative residuals of the
// k pairs nearest sigma are above switch_tol the iteration runs in an FP32
// form: W, A W, S, Q_W, A S, Q_S, P, A P and the V-cycles are FP32, V and A V
// stay FP64 (A V explicit every iteration, so the residual is exact for the
// stored V), the Grams take FP32 products with compensated accumulation, the
// projected problem is FP64, the V part of the update is summed in FP64, and
// Q_V, Q_P are recomputed explicitly (2 more V-cycles on k' columns) instead
// of carried.  Then P is widened, its images and Q_V, Q_P are recomputed in
// FP64 and the iteration continues in FP64 to the requested tolerance.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "blockops.h"
#include "dense.h"
#include "mixed.h"
#include "plhr_internal.h"

namespace plhr {
plhr_status prec_reserve(plhr_prec* T, int nc, int64_t extra_doubles);
plhr_status plmr_solve(const plhr_op* A, const plhr_op* B, plhr_prec* T, double tol, const plhr_options& opt,
                       double* eigvals, double* eigvecs, int64_t ldv, plhr_info* info, cudaStream_t s,
                       double t_start);
plhr_status prec_reserve32(plhr_prec* T, int nc, int64_t extra_floats);
plhr_status prec_reserve_dw(plhr_prec* T, int nc);
}

using namespace plhr;

namespace {

struct DevBuf {
    double* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

struct HostStatus {
    int conv, nact, nan;
    int dense[3];
    int rr_ok;
    int pad;
};

// flops of one multi-Gram pass over an n x m trial basis: Z^T Z and U^T Q
// (upper triangles; both symmetric) and Q^T Z
double gram_flops(int64_t n, int m) { return 2.0 * (double)n * ((double)m * (m + 1) + (double)m * m); }

// Algorithmic HBM bytes of one preconditioner application on nc columns of
// eb-byte elements: for AV-MG 14.25 passes per level above the coarsest (the
// fused first two sweeps 2, residual 3, restriction 1 1/8, prolongation with
// correction 2 1/8, two post-sweeps 6); any other T reads r and writes w.
double prec_bytes(const plhr_prec* T, int64_t n, int nc, int eb) {
    if (T->kind != PREC_AVMG) return 2.0 * (double)n * nc * eb;
    double el = 0.0;
    for (size_t l = 1; l < T->H.lev.size(); ++l) el += (double)T->H.lev[l].g.n();
    if (T->H.lev.size() <= 1) el = (double)n;
    return 14.25 * el * nc * eb;
}

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

extern "C" void plhr_options_default(plhr_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->maxit = 1000;
    o->precision = PLHR_PRECISION_F64;
    o->real_arithmetic = 1;
    o->s_vectors = 1;
    o->soft_lock = 1;
    o->seed = 20140801ull;
    o->guard = 1;
    o->switch_tol = 1e-6;
    o->extraction = 0;
    o->tensor_cores = 1;
}

extern "C" plhr_status plhr_solve(const plhr_op* A, const plhr_op* B, double sigma, int k, plhr_prec* T, double tol,
                                  const plhr_options* opt_in, double* eigvals, double* eigvecs, int64_t ldv,
                                  plhr_info* info, void* stream) {
    clear_error();
    const double t0 = now_s();
    plhr_options opt;
    plhr_options_default(&opt);
    if (opt_in) opt = *opt_in;
    if (!A || !eigvals || !eigvecs || k < 1 || ldv < k || !(tol > 0) || !std::isfinite(sigma) || opt.maxit < 0) {
        set_error("plhr_solve: invalid argument");
        return PLHR_EINVAL;
    }
    if (A->g.complex_op() || (B && B->g.complex_op())) {
        set_error("plhr_solve: complex operators (Bloch kappa != 0) are not supported by the real solver");
        return PLHR_EINVAL;
    }
    if (B != nullptr && (B->g.n() != A->g.n() || opt.precision != PLHR_PRECISION_F64)) {
        set_error("plhr_solve: B must have the size of A, and B != I runs in PLHR_PRECISION_F64");
        return PLHR_EINVAL;
    }
    if (!opt.real_arithmetic || (opt.precision != PLHR_PRECISION_F64 && opt.precision != PLHR_PRECISION_MIXED) ||
        opt.extraction < 0 || opt.extraction > 2) {
        set_error("plhr_solve: this build supports real arithmetic, FP64 or mixed precision, extraction 0, 1 or 2");
        return PLHR_EINVAL;
    }
    if (opt.extraction == 2) {
        // the refinement extraction of Eq. rRR: the single-vector method of Section 3.3
        if (k != 1 || opt.guard != 0 || opt.precision != PLHR_PRECISION_F64 ||
            (T && T->kind == PREC_AVMG && T->H.indefinite) || (T && prec_size(T) != A->g.n()) ||
            (opt.v_init && opt.ld_init < 1)) {
            set_error("plhr_solve: extraction 2 (refinement, Eq. rRR) is the single-vector method: k = 1, "
                      "guard = 0, PLHR_PRECISION_F64, a symmetric positive definite T of A's size");
            return PLHR_EINVAL;
        }
        return plmr_solve(A, B, T, tol, opt, eigvals, eigvecs, ldv, info, (cudaStream_t)stream, t0);
    }
    if ((!opt.s_vectors || opt.extraction != 0) && opt.precision != PLHR_PRECISION_F64) {
        set_error("plhr_solve: harmonic extraction and s_vectors = 0 run in PLHR_PRECISION_F64");
        return PLHR_EINVAL;
    }
    const int64_t n = A->g.n();
    if (T && T->kind == PREC_AVMG && T->H.indefinite && (opt.extraction == 0 || opt.precision != PLHR_PRECISION_F64)) {
        set_error("plhr_solve: the INV-MG preconditioner is indefinite: it needs the harmonic extraction "
                  "(extraction = 1) in PLHR_PRECISION_F64");
        return PLHR_EINVAL;
    }
    if (opt.precision == PLHR_PRECISION_MIXED && T && T->kind == PREC_AVMG && T->H.lev[0].g.n() > kMaxSmemCoarse) {
        set_error("plhr_solve: PLHR_PRECISION_MIXED needs a coarsest multigrid grid of at most %lld points",
                  (long long)kMaxSmemCoarse);
        return PLHR_EINVAL;
    }
    if (opt.precision == PLHR_PRECISION_MIXED && (!A->g.plain() || (T && T->kind != PREC_AVMG))) {
        set_error("plhr_solve: the mixed-precision form supports the Dirichlet Laplacian with AV-MG or T = I only");
        return PLHR_EINVAL;
    }
    if (opt.guard < 0) {
        set_error("plhr_solve: guard < 0");
        return PLHR_EINVAL;
    }
    const int kp = k + opt.guard;
    const int mmax = 4 * kp;
    if (mmax > kDenseMaxM || mmax > gram_max_m() || kp > 32) {
        set_error("plhr_solve: k + guard = %d too large (4 (k + guard) must be <= %d)", kp, kDenseMaxM);
        return PLHR_EINVAL;
    }
    if (n < (int64_t)mmax) {
        set_error("plhr_solve: n = %lld too small for k = %d", (long long)n, k);
        return PLHR_EINVAL;
    }
    if (T && prec_size(T) != n) {
        set_error("plhr_solve: preconditioner size does not match A");
        return PLHR_EINVAL;
    }
    if (opt.v_init && opt.ld_init < kp) {
        set_error("plhr_solve: ld_init < k + guard");
        return PLHR_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const Grid& g = A->g;

    // ---------------------------------------------------------------- workspace
    const int64_t nk = n * kp;
    const bool hasB = B != nullptr;
    const int64_t big_doubles = 6 * nk /*V AV QV P AP QP*/ + nk /*R*/ + nk /*Rc*/ + nk /*W*/ + nk /*AW*/ +
                                2 * nk /*SQ*/ + 2 * nk /*X2*/ + nk /*AS*/ + nk /*X3*/ + nk /*QS*/ +
                                (hasB ? 4 * nk /*BV BW BS BP*/ : 0);
    const int m3 = 3 * mmax * mmax;
    const int64_t part_doubles = (int64_t)reduce_blocks() * m3 + (int64_t)residual_blocks(kp) * 2 * kp + 64;
    const int64_t small_doubles = m3 /*grams*/ + (int64_t)dense_work_doubles() + mmax * kp /*Cp*/ + kp * kp /*Cvv*/ +
                                  9 * 64 /*vectors*/ + kp * kp /*Crr*/ + 2 * 64 /*xi*/;
    DevBuf big, part, small;
    if (cudaMallocAsync(&big.p, sizeof(double) * big_doubles, s) != cudaSuccess ||
        cudaMallocAsync(&part.p, sizeof(double) * part_doubles, s) != cudaSuccess ||
        cudaMallocAsync(&small.p, sizeof(double) * small_doubles, s) != cudaSuccess) {
        set_error("plhr_solve: device allocation of %.1f MB failed", 8e-6 * (double)(big_doubles + part_doubles));
        return PLHR_ENOMEM;
    }
    int* ints = nullptr;
    if (cudaMallocAsync(&ints, sizeof(int) * 512, s) != cudaSuccess) {
        set_error("plhr_solve: device allocation failed");
        return PLHR_ENOMEM;
    }
    struct IntFree { int* p; ~IntFree() { if (p) cudaFree(p); } } int_free{ints};
    HostStatus* hs = nullptr;
    if (cudaMallocHost(&hs, sizeof(HostStatus) + sizeof(double) * 4 * 64) != cudaSuccess) {
        set_error("plhr_solve: pinned allocation failed");
        return PLHR_ENOMEM;
    }
    struct HostFree { void* p; ~HostFree() { if (p) cudaFreeHost(p); } } host_free{hs};
    // on every exit, wait for the work queued on the stream before any buffer
    // above (or the FP32 ones below) is released: an error return can happen
    // with kernels of the current iteration still in flight
    struct StreamDrain { cudaStream_t s; ~StreamDrain() { cudaStreamSynchronize(s); } } drain_before_free{s};
    double* h_rel = reinterpret_cast<double*>(hs + 1);
    double* h_lam = h_rel + 64;
    double* h_theta = h_lam + 64;
    int* h_order = reinterpret_cast<int*>(h_theta + 64);

    double* p = big.p;
    auto take = [&](int64_t cnt) { double* r = p; p += cnt; return r; };
    double *V = take(nk), *AV = take(nk), *QV = take(nk), *P = take(nk), *AP = take(nk), *QP = take(nk);
    double *R = take(nk), *Rc = take(nk), *W = take(nk), *AW = take(nk), *SQ = take(2 * nk), *X2 = take(2 * nk);
    double *AS = take(nk), *X3 = take(nk), *QS = take(nk);
    // B images of V, W, S, P (generalized problem A v = lambda B v)
    double *BV = hasB ? take(nk) : nullptr, *BW = hasB ? take(nk) : nullptr, *BS = hasB ? take(nk) : nullptr,
           *BP = hasB ? take(nk) : nullptr;
    // FP32 blocks of the mixed form: W, A W, [S | Q_W], its input, A S, A S - sigma S,
    // Q_S, P, A P, Q_P, Q_V
    bool mx = opt.precision == PLHR_PRECISION_MIXED;
    // FP64 phase of the mixed form: V-cycle, Gram and update in double-word
    // arithmetic on the FP64 blocks (FP64-class accuracy on the FP32 pipes)
    const bool dwf = opt.precision == PLHR_PRECISION_MIXED;
    // thq: T-harmonic images Q = T(A - sigma B)Z are formed (T given and the
    // T-harmonic extraction); sv: the trial space holds the S block
    const bool thq = T && opt.extraction == 0;
    const bool sv = opt.s_vectors != 0;
    int mixed_its = 0;
    int restarts = 0;     // restarts of dependent columns at acceptance
    double best_worst = INFINITY;   // FP32 form: smallest worst residual so far and when
    int best_it = 0;
    struct FloatBuf {
        float* p = nullptr;
        cudaStream_t s = nullptr;
        ~FloatBuf() {
            if (!p) return;
            cudaStreamSynchronize(s);   // destroyed before drain_before_free: wait here too
            cudaFree(p);
        }
    } big32;
    big32.s = s;
    float *W32 = nullptr, *AW32 = nullptr, *SQ32 = nullptr, *X2_32 = nullptr, *AS32 = nullptr, *X3_32 = nullptr,
          *QS32 = nullptr, *P32 = nullptr, *AP32 = nullptr, *QP32 = nullptr, *QV32 = nullptr, *V32 = nullptr,
          *U32 = nullptr, *WQ32 = nullptr, *QSP32 = nullptr;
    if (mx) {
        if (cudaMallocAsync(&big32.p, sizeof(float) * 19 * nk, s) != cudaSuccess) {
            set_error("plhr_solve: device allocation of %.1f MB failed", 4e-6 * 19.0 * (double)nk);
            return PLHR_ENOMEM;
        }
        float* f = big32.p;
        W32 = f; f += nk; AW32 = f; f += nk; SQ32 = f; f += 2 * nk; X2_32 = f; f += 2 * nk; AS32 = f; f += nk;
        X3_32 = f; f += nk; QS32 = f; f += nk; P32 = f; f += nk; AP32 = f; f += nk; QP32 = f; f += nk;
        QV32 = f; f += nk; V32 = f; f += nk; U32 = f; f += nk;
        WQ32 = f; f += 2 * nk;    // [W | Q_V] from one paired V-cycle (leading dimension na + kp)
        QSP32 = f; f += 2 * nk;   // [Q_S | Q_P] likewise
        if (T) PLHR_TRY(prec_reserve32(T, 2 * kp, 0));
        if (T) PLHR_TRY(prec_reserve_dw(T, 2 * kp));
    }
    double* gpart = part.p;
    double* rpart = part.p + (int64_t)reduce_blocks() * m3;
    double* q = small.p;
    double* grams = q; q += m3;
    double* dwork = q; q += dense_work_doubles();
    double* Cp = q; q += mmax * kp;
    double* Cvv = q; q += kp * kp;
    double* sums = q; q += 64;
    double* lam = q; q += 64;
    double* scale = q; q += 64;
    double* colscale = q; q += 64;
    double* rel = q; q += 64;
    double* lam_act = q; q += 64;
    double* dots = q; q += 64;
    double* theta = q; q += 64;
    double* dots2 = q; q += 64;
    double* Crr = q; q += kp * kp;
    double* xi = q; q += 128;
    int* active = ints;
    int* order = ints + 64;
    int* tags = ints + 128;
    int* partner = ints + 192;
    int* dstat = ints + 256;   // [conv, nact, nan, dense0, dense1, dense2, rr_ok, tensor-core wait timeout]
    if (T) PLHR_TRY(prec_reserve(T, 2 * kp, 0));

    // colscale = 1 everywhere (the V part is overwritten every iteration)
    {
        std::vector<double> ones(64, 1.0);
        PLHR_TRY_CUDA(cudaMemcpyAsync(colscale, ones.data(), sizeof(double) * 64, cudaMemcpyHostToDevice, s));
        PLHR_TRY_CUDA(cudaStreamSynchronize(s));
    }

    auto applyT = [&](int nc, const double* r, int64_t ldr, double* w) -> plhr_status {
        // w (ld nc) = T r
        if (nc == 0) return PLHR_OK;
        if (!T) {
            PLHR_TRY_CUDA(cudaMemcpy2DAsync(w, sizeof(double) * nc, r, sizeof(double) * ldr, sizeof(double) * nc, n,
                                            cudaMemcpyDeviceToDevice, s));
            return PLHR_OK;
        }
        PhaseScope ps(PH_VCYCLE, s, (double)n * nc, prec_bytes(T, n, nc, 8));
        if (dwf)   // FP64 phase of the mixed form: double-word V-cycle
            PLHR_TRY_CUDA(mg_vcycle_dw(T->H, nc, r, ldr, w, nc, T->work, s));
        else
            PLHR_TRY(prec_apply64(T, nc, r, ldr, w, T->work, s));
        return PLHR_OK;
    };

    auto applyT32 = [&](int nc, const auto* r, int64_t ldr, float* w) -> plhr_status {
        // w (ld nc, FP32) = T r in the FP32 V-cycle
        if (nc == 0) return PLHR_OK;
        PhaseScope ps(PH_VCYCLE32, s, (double)n * nc, prec_bytes(T, n, nc, 4));
        PLHR_TRY_CUDA(mg_vcycle_f32(T->H, nc, r, ldr, w, T->work32, s));
        return PLHR_OK;
    };
    // w (ld nc1 + nc2) = [T r1 | T r2], one FP32 V-cycle of nc1 + nc2 columns
    auto applyT32_pair = [&](int nc1, const double* r1, int64_t ldr1, int nc2, const double* r2, int64_t ldr2,
                             float* w) -> plhr_status {
        const int nc = nc1 + nc2;
        PhaseScope ps(PH_VCYCLE32, s, (double)n * nc, prec_bytes(T, n, nc, 4));
        PLHR_TRY_CUDA(mg_vcycle_f32_pair(T->H, nc1, r1, ldr1, nc2, r2, ldr2, w, T->work32, s));
        return PLHR_OK;
    };

    // A X with the shifted outputs o1 = AX - BX diag(lam), o2 = AX - sigma BX
    // (each optional); BX = B X is formed when B is given (FP64 forms)
    auto prod = [&](int nc, const double* X, int64_t ldx, double* AX, int64_t ldax, double* BX, int64_t ldbx,
                    double* o1, int64_t ld1, const double* lamv, double* o2, int64_t ld2) -> plhr_status {
        if (!hasB) {
            PLHR_TRY_CUDA(lap_apply_shifts(g, nc, X, ldx, AX, ldax, o1, ld1, lamv, o2, ld2, sigma, s));
            return PLHR_OK;
        }
        if (q1_same_mesh(g, B->g)) {   // both finite-element operators in one pass
            PLHR_TRY_CUDA(q1_pair(g, B->g, nc, X, ldx, AX, ldax, BX, ldbx, s));
        } else {
            PLHR_TRY_CUDA(lap_axpby(g, nc, X, ldx, AX, ldax, 1.0, 0.0, s));
            PLHR_TRY_CUDA(lap_axpby(B->g, nc, X, ldx, BX, ldbx, 1.0, 0.0, s));
        }
        if (o1 || o2) PLHR_TRY_CUDA(shift_combine(n, nc, AX, ldax, BX, ldbx, lamv, o1, ld1, sigma, o2, ld2, s));
        return PLHR_OK;
    };
    // algorithmic bytes of prod on nc columns with `outs` shifted outputs
    auto prod_bytes = [&](int nc, int outs) -> double {
        const double passes = hasB ? 4.0 + (outs ? 2.0 + outs : 0.0) : 2.0 + outs;
        return 8.0 * (double)n * nc * passes;
    };
    // dots = [v.Av (kp) | v.Bv (kp)] for the Rayleigh quotients and scales
    auto rq_dots = [&]() -> plhr_status {
        PLHR_TRY_CUDA(column_dots(n, kp, V, kp, AV, kp, rpart, dots, s));   // v.Av, v.v
        if (hasB) {
            PLHR_TRY_CUDA(column_dots(n, kp, V, kp, BV, kp, rpart, dots2, s));
            PLHR_TRY_CUDA(cudaMemcpyAsync(dots + kp, dots2, sizeof(double) * kp, cudaMemcpyDeviceToDevice, s));
        }
        return PLHR_OK;
    };

    // ---------------------------------------------------------------- start (Alg. 3 steps 1-2)
    if (opt.v_init)
        PLHR_TRY_CUDA(cudaMemcpy2DAsync(V, sizeof(double) * kp, opt.v_init, sizeof(double) * opt.ld_init,
                                        sizeof(double) * kp, n, cudaMemcpyDeviceToDevice, s));
    else
        PLHR_TRY_CUDA(seeded_block(n, kp, opt.seed, V, kp, s));
    // AV, X3 := AV - sigma V, QV = T(AV - sigma V) (with T = I, Q = AZ - sigma Z is
    // formed inside the Gram pass and no Q block is stored)
    PLHR_TRY(prod(kp, V, kp, AV, kp, BV, kp, nullptr, 0, nullptr, X3, kp));
    if (thq) {
        if (mx) PLHR_TRY(applyT32(kp, (const double*)X3, kp, QV32));
        else PLHR_TRY(applyT(kp, X3, kp, QV));
    }
    PLHR_TRY(rq_dots());
    {
        std::vector<int> zeros(64, 0), neg(64, -1);
        PLHR_TRY_CUDA(cudaMemcpyAsync(tags, zeros.data(), sizeof(int) * 64, cudaMemcpyHostToDevice, s));
        PLHR_TRY_CUDA(cudaMemcpyAsync(partner, neg.data(), sizeof(int) * 64, cudaMemcpyHostToDevice, s));
        PLHR_TRY_CUDA(cudaMemsetAsync(dstat + 7, 0, sizeof(int), s));
        PLHR_TRY_CUDA(cudaStreamSynchronize(s));
    }
    PLHR_TRY_CUDA(dense_rq(kp, dots, tags, partner, lam, scale, s));
    int np = 0;

    // images of V and P under A: explicit stencil products after every update
    // (no recursion, so no drift), dots for the Rayleigh quotients of V
    auto refresh_images = [&]() -> plhr_status {
        // V (and B V) and P: read the block, write its image
        PhaseScope ps(PH_STENCIL, s, (double)n * (np ? 2 * kp : kp),
                      (double)n * kp * 2.0 * (8.0 * (hasB ? 2 : 1) + (np ? (mx ? 4.0 : 8.0 * (hasB ? 2 : 1)) : 0.0)));
        if (hasB) PLHR_TRY(prod(kp, V, kp, AV, kp, BV, kp, nullptr, 0, nullptr, nullptr, 0));
        else PLHR_TRY_CUDA(lap_axpby(g, kp, V, kp, AV, kp, 1.0, 0.0, s));
        if (np) {
            if (mx) PLHR_TRY_CUDA(lap32_apply_shifts(g, kp, P32, kp, AP32, kp, nullptr, 0, nullptr, nullptr, 0, 0.0, s));
            else if (hasB) PLHR_TRY(prod(kp, P, kp, AP, kp, BP, kp, nullptr, 0, nullptr, nullptr, 0));
            else PLHR_TRY_CUDA(lap_axpby(g, kp, P, kp, AP, kp, 1.0, 0.0, s));
        }
        PLHR_TRY(rq_dots());
        return PLHR_OK;
    };

    // Columns of V numerically dependent on the columns nearer sigma: Cholesky
    // of the normalised Gram G = D V^T V D (host copy, kp x kp) in the order
    // ord, skipping the columns already marked; a column whose squared
    // distance to the span of the kept ones is below thresh is marked.  An
    // iteration can let two columns drift into one direction of a degenerate
    // eigenspace; the slot they waste leaves a member of another cluster out.
    auto mark_dependent = [&](const double* G, const int* ord, double thresh, std::vector<char>& mark) {
        std::vector<double> L(kp * kp, 0.0);
        std::vector<int> kept;
        bool any = false;
        for (int q2 = 0; q2 < kp; ++q2) {
            const int j = ord[q2];
            if (mark[j]) continue;
            double rest = 1.0;
            for (size_t p = 0; p < kept.size(); ++p) {
                const int i = kept[p];
                double c = G[j * kp + i] / std::sqrt(G[j * kp + j] * G[i * kp + i]);
                for (size_t r = 0; r < p; ++r) c -= L[j * kp + r] * L[i * kp + r];
                L[j * kp + p] = c / L[i * kp + p];
                rest -= L[j * kp + p] * L[j * kp + p];
            }
            if (!(rest > thresh)) {
                mark[j] = 1;
                any = true;
                continue;
            }
            L[j * kp + kept.size()] = std::sqrt(rest);
            kept.push_back(j);
        }
        return any;
    };
    // the marked columns of V restart from seeded random vectors (FP64 forms);
    // A V, the images and the Rayleigh quotients are recomputed
    auto restart_columns = [&](const std::vector<char>& mark, uint64_t salt) -> plhr_status {
        PLHR_TRY_CUDA(seeded_block(n, kp, opt.seed ^ salt, Rc, kp, s));
        for (int j = 0; j < kp; ++j)
            if (mark[j])
                PLHR_TRY_CUDA(cudaMemcpy2DAsync(V + j, sizeof(double) * kp, Rc + j, sizeof(double) * kp,
                                                sizeof(double), n, cudaMemcpyDeviceToDevice, s));
        PLHR_TRY(prod(kp, V, kp, AV, kp, BV, kp, nullptr, 0, nullptr, X3, kp));
        if (thq) PLHR_TRY(applyT(kp, X3, kp, QV));
        std::vector<int> zeros(64, 0), neg(64, -1);
        PLHR_TRY_CUDA(cudaMemcpyAsync(tags, zeros.data(), sizeof(int) * 64, cudaMemcpyHostToDevice, s));
        PLHR_TRY_CUDA(cudaMemcpyAsync(partner, neg.data(), sizeof(int) * 64, cudaMemcpyHostToDevice, s));
        PLHR_TRY(rq_dots());
        PLHR_TRY_CUDA(dense_rq(kp, dots, tags, partner, lam, scale, s));
        PLHR_TRY_CUDA(cudaStreamSynchronize(s));   // the host vectors above
        return PLHR_OK;
    };

    // end of the FP32 form: P to FP64, then A V, A P, T(A V - sigma V) and
    // T(A P - sigma P) explicitly in FP64
    // ord: host column order by distance to sigma (the first k are kept)
    auto switch_to_f64 = [&](const int* ord) -> plhr_status {
        // guard columns (beyond the k nearest sigma) restart from fresh seeded
        // random vectors: the FP32 form can lose a weak direction (a member of a
        // degenerate cluster whose component sat below its rounding level), and
        // random columns contain every eigendirection for the FP64 phase to
        // find; so do columns dependent on the ones nearer sigma
        std::vector<char> restart(kp, 0);
        for (int q2 = k; q2 < kp; ++q2) restart[ord[q2]] = 1;
        {
            Blk<const double> vb[1] = {{V, kp, kp}};
            PLHR_TRY_CUDA(multi_gram(n, 1, vb, vb, vb, 0.0, colscale, gpart, grams, s));
            std::vector<double> G(kp * kp);
            PLHR_TRY_CUDA(cudaMemcpyAsync(G.data(), grams, sizeof(double) * kp * kp, cudaMemcpyDeviceToHost, s));
            PLHR_TRY_CUDA(cudaStreamSynchronize(s));
            mark_dependent(G.data(), ord, 1e-4, restart);
        }
        bool any = false;
        for (int j2 = 0; j2 < kp; ++j2) any = any || restart[j2];
        if (any) {
            PLHR_TRY_CUDA(seeded_block(n, kp, opt.seed ^ 0x5bd1e995ull, Rc, kp, s));
            for (int j2 = 0; j2 < kp; ++j2)
                if (restart[j2])
                    PLHR_TRY_CUDA(cudaMemcpy2DAsync(V + j2, sizeof(double) * kp, Rc + j2, sizeof(double) * kp,
                                                    sizeof(double), n, cudaMemcpyDeviceToDevice, s));
        }
        if (np) {
            PLHR_TRY_CUDA(widen_block(n, kp, P32, kp, P, kp, s));
            // a restarted column drops its search direction too: the old
            // direction would bring the FP32 guard content straight back into
            // the first FP64 projection, ahead of what the random column holds
            for (int j2 = 0; j2 < kp; ++j2)
                if (restart[j2])
                    PLHR_TRY_CUDA(cudaMemset2DAsync(P + j2, sizeof(double) * kp, 0, sizeof(double), n, s));
        }
        PLHR_TRY_CUDA(lap_apply_shifts(g, kp, V, kp, AV, kp, nullptr, 0, nullptr, X3, kp, sigma, s));
        if (T) PLHR_TRY(applyT(kp, X3, kp, QV));
        if (np) {
            PLHR_TRY_CUDA(lap_apply_shifts(g, kp, P, kp, AP, kp, nullptr, 0, nullptr, X3, kp, sigma, s));
            if (T) PLHR_TRY(applyT(kp, X3, kp, QP));
        }
        mx = false;
        if (any) {
            // Rayleigh quotients and scales of the new columns (every column
            // real: the pairing of the last extraction no longer applies)
            std::vector<int> zeros(64, 0), neg(64, -1);
            PLHR_TRY_CUDA(cudaMemcpyAsync(tags, zeros.data(), sizeof(int) * 64, cudaMemcpyHostToDevice, s));
            PLHR_TRY_CUDA(cudaMemcpyAsync(partner, neg.data(), sizeof(int) * 64, cudaMemcpyHostToDevice, s));
            PLHR_TRY_CUDA(column_dots(n, kp, V, kp, AV, kp, rpart, dots, s));
            PLHR_TRY_CUDA(dense_rq(kp, dots, tags, partner, lam, scale, s));
            PLHR_TRY_CUDA(cudaStreamSynchronize(s));   // the host vectors above
        }
        return PLHR_OK;
    };

    const double t1 = now_s();
    plhr_status result = PLHR_ENOTCONV;
    int it = 0;
    int hist = 0;
    int last_m = 0;
    int last_kept = 0;
    for (it = 0; it <= opt.maxit; ++it) {
        // -------------------------------------------- residual, convergence (step 4 input)
        {
            PhaseScope ps(PH_OTHER, s, (double)n * kp, 24.0 * (double)n * kp);
            PLHR_TRY_CUDA(residual_norms(n, kp, hasB ? BV : V, kp, AV, kp, lam, scale, R, kp, rpart, sums, s));
        }
        StatusArgs sa;
        sa.kp = kp; sa.k = k; sa.sigma = sigma; sa.tol = tol;
        sa.sums = sums; sa.lam = lam; sa.lam_act = lam_act; sa.active = active; sa.rel = rel; sa.order = order;
        sa.hstat = dstat;
        PLHR_TRY_CUDA(dense_status(sa, s));
        PLHR_TRY_CUDA(cudaMemcpyAsync(hs, dstat, sizeof(int) * 7, cudaMemcpyDeviceToHost, s));
        PLHR_TRY_CUDA(cudaMemcpyAsync(h_rel, rel, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
        PLHR_TRY_CUDA(cudaMemcpyAsync(h_lam, lam, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
        PLHR_TRY_CUDA(cudaMemcpyAsync(h_order, order, sizeof(int) * kp, cudaMemcpyDeviceToHost, s));
        PLHR_TRY_CUDA(cudaStreamSynchronize(s));
        if (hs->nan) {
            set_error("plhr_solve: NaN/Inf at iteration %d", it);
            result = PLHR_ENAN;
            break;
        }
        if (opt.history && hist < opt.history_cap) {
            double* rec = opt.history + (int64_t)hist * (2 * kp + 3);
            rec[0] = it;
            for (int q2 = 0; q2 < kp; ++q2) {
                rec[1 + q2] = h_lam[h_order[q2]];
                rec[1 + kp + q2] = h_rel[h_order[q2]];
            }
            rec[1 + 2 * kp] = last_kept;
            rec[2 + 2 * kp] = last_m;
            ++hist;
        }
        if (hs->conv) {
            // final standard Rayleigh-Ritz (Alg. 3 step 16) and acceptance on the
            // returned vectors: explicit A V, B V
            PLHR_TRY_CUDA(lap_axpby(g, kp, V, kp, AW, kp, 1.0, 0.0, s));
            if (hasB) PLHR_TRY_CUDA(lap_axpby(B->g, kp, V, kp, X3, kp, 1.0, 0.0, s));
            Blk<const double> zb[1] = {{V, kp, kp}}, ab[1] = {{AW, kp, kp}}, qb[1] = {{V, kp, kp}},
                              bzb[1] = {{X3, kp, kp}};
            PLHR_TRY_CUDA(cudaMemcpyAsync(colscale, scale, sizeof(double) * kp, cudaMemcpyDeviceToDevice, s));
            PLHR_TRY_CUDA(multi_gram_b(n, 1, zb, ab, qb, hasB ? bzb : nullptr, 0.0, colscale, gpart, grams, s));
            // grams: [V^T B V | (AV)^T V | V^T B V] (kp x kp blocks)
            if (!mx && kp > k && restarts < 8) {
                // a column dependent on the ones nearer sigma holds a slot that a
                // missing eigenvector needs: restart it instead of accepting
                std::vector<double> G(kp * kp);
                PLHR_TRY_CUDA(cudaMemcpyAsync(G.data(), grams, sizeof(double) * kp * kp, cudaMemcpyDeviceToHost, s));
                PLHR_TRY_CUDA(cudaStreamSynchronize(s));
                std::vector<char> mark(kp, 0);
                if (mark_dependent(G.data(), h_order, 1e-8, mark)) {
                    ++restarts;
                    PLHR_TRY(restart_columns(mark, 0x2545f4914f6cdd1dull * (uint64_t)(restarts + 1)));
                    continue;
                }
            }
            PLHR_TRY_CUDA(dense_rr(kp, grams + kp * kp, grams, sigma, scale, Crr, theta, dstat + 6, s));
            PLHR_TRY_CUDA(block_times_small(n, V, kp, kp, Crr, kp, Rc, kp, s));   // all Ritz vectors
            PLHR_TRY_CUDA(lap_axpby(g, kp, Rc, kp, AW, kp, 1.0, 0.0, s));
            if (hasB) PLHR_TRY_CUDA(lap_axpby(B->g, kp, Rc, kp, X3, kp, 1.0, 0.0, s));
            {
                std::vector<double> ones(kp, 1.0);
                PLHR_TRY_CUDA(cudaMemcpyAsync(dots, ones.data(), sizeof(double) * kp, cudaMemcpyHostToDevice, s));
            }
            PLHR_TRY_CUDA(residual_norms(n, kp, hasB ? X3 : Rc, kp, AW, kp, theta, dots, R, kp, rpart, sums, s));
            sa.lam = theta;
            PLHR_TRY_CUDA(dense_status(sa, s));
            PLHR_TRY_CUDA(cudaMemcpyAsync(hs, dstat, sizeof(int) * 7, cudaMemcpyDeviceToHost, s));
            PLHR_TRY_CUDA(cudaMemcpyAsync(h_rel, rel, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
            PLHR_TRY_CUDA(cudaMemcpyAsync(h_theta, theta, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
            PLHR_TRY_CUDA(cudaStreamSynchronize(s));
            if (!hs->rr_ok) {
                set_error("plhr_solve: final Rayleigh-Ritz failed");
                result = PLHR_EBREAKDOWN;
                break;
            }
            bool acc = true;
            for (int q2 = 0; q2 < k; ++q2) acc = acc && (h_rel[q2] <= tol);
            if (acc) {
                result = PLHR_OK;
                break;
            }
            // carry on from the rotated block (same span): V <- V C, A V explicit
            PLHR_TRY_CUDA(cudaMemcpyAsync(V, Rc, sizeof(double) * nk, cudaMemcpyDeviceToDevice, s));
            PLHR_TRY_CUDA(cudaMemcpyAsync(AV, AW, sizeof(double) * nk, cudaMemcpyDeviceToDevice, s));
            if (hasB) PLHR_TRY_CUDA(cudaMemcpyAsync(BV, X3, sizeof(double) * nk, cudaMemcpyDeviceToDevice, s));
            if (!mx && thq) PLHR_TRY_CUDA(block_times_small(n, QV, kp, kp, Crr, kp, QV, kp, s));
            PLHR_TRY_CUDA(cudaMemcpyAsync(lam, theta, sizeof(double) * kp, cudaMemcpyDeviceToDevice, s));
            {
                std::vector<double> ones(kp, 1.0);
                PLHR_TRY_CUDA(cudaMemcpyAsync(scale, ones.data(), sizeof(double) * kp, cudaMemcpyHostToDevice, s));
                PLHR_TRY_CUDA(cudaStreamSynchronize(s));
            }
            if (mx) {
                mixed_its = it;
                std::vector<int> ident(kp);
                for (int q2 = 0; q2 < kp; ++q2) ident[q2] = q2;   // the RR sorted the columns
                PLHR_TRY(switch_to_f64(ident.data()));
            }
            continue;
        }
        if (it == opt.maxit) break;
        if (mx) {
            double worst = 0.0;
            for (int q2 = 0; q2 < k; ++q2) worst = std::fmax(worst, h_rel[h_order[q2]]);
            if (worst < best_worst) {
                best_worst = worst;
                best_it = it;
            }
            // leave the FP32 form at switch_tol, or earlier when it stagnates at its
            // rounding floor (no new minimum for 25 iterations below 1e-5)
            if (worst < opt.switch_tol || (best_worst < 1e-5 && it - best_it >= 25)) {
                mixed_its = it;
                PLHR_TRY(switch_to_f64(h_order));
            }
        }
        const int na = hs->nact;
        // -------------------------------------------- W = T(AV - BV Lambda), active columns
        const double* Ract = R;
        int64_t ldra = kp;
        if (na < kp) {
            PLHR_TRY_CUDA(gather_columns(n, R, kp, active, na, Rc, na, s));
            Ract = Rc;
            ldra = na;
        }
        if (mx) {
            // ---------------------------------------- the same step in the FP32 form
            // W = T(AV - V Lambda) and, with T, Q_V = T(A V - sigma V) explicitly:
            // carrying Q_V (and Q_P below) through the update would mix the FP32
            // V-cycle's rounding of different iterations into one image, and the
            // projected pencil (built from Q = T U) would lose consistency below
            // ~1e-5.  Both right-hand sides are ready here, so they share one
            // V-cycle when the 16-byte column groups allow it.
            float* Wp = W32;
            int64_t ldw = na;
            float* QVp = QV32;
            int64_t ldqv = kp;
            // FP32 copies of V and U_V = A V - sigma V (formed in FP64) for the Gram
            PLHR_TRY_CUDA(prepare_v_mx(n, kp, V, AV, sigma, V32, U32, T ? X3 : nullptr, s));
            if (T && na % 4 == 0 && kp % 4 == 0) {
                PLHR_TRY(applyT32_pair(na, Ract, ldra, kp, (const double*)X3, kp, WQ32));
                Wp = WQ32;
                QVp = WQ32 + na;
                ldw = ldqv = na + kp;
            } else if (T) {
                PLHR_TRY(applyT32(na, Ract, ldra, W32));
                PLHR_TRY(applyT32(kp, (const double*)X3, kp, QV32));
            } else {
                PLHR_TRY_CUDA(narrow_block(n, na, Ract, ldra, W32, na, s));
            }
            float* X2in = T ? X2_32 : SQ32;
            {
                PhaseScope ps(PH_STENCIL, s, (double)n * na, 4.0 * n * na * (T ? 4 : 3));
                PLHR_TRY_CUDA(lap32_apply_shifts(g, na, Wp, ldw, AW32, na, X2in, T ? 2 * na : na, lam_act,
                                                 T ? X2in + na : nullptr, 2 * na, sigma, s));
            }
            const float* S32 = SQ32;
            const int64_t lds = T ? 2 * na : na;
            if (T) PLHR_TRY(applyT32(2 * na, (const float*)X2_32, 2 * na, SQ32));
            const float* QW32 = SQ32 + na;
            // Q_S = T(A S - sigma S) and Q_P = T(A P - sigma P) from one V-cycle too
            // when both widths allow it: their inputs go side by side into X2_32
            // (free once the cycle above has read it)
            const bool pair_sp = T && np && na % 4 == 0 && kp % 4 == 0;
            const int64_t ldsp = na + kp;
            float* QSp = QS32;
            float* QPp = QP32;
            int64_t ldqs = na, ldqp = kp;
            {
                PhaseScope ps(PH_STENCIL, s, (double)n * na, 4.0 * n * na * (T ? 3 : 2));
                PLHR_TRY_CUDA(lap32_apply_shifts(g, na, S32, lds, AS32, na, nullptr, 0, nullptr,
                                                 T ? (pair_sp ? X2_32 : X3_32) : nullptr, pair_sp ? ldsp : na, sigma,
                                                 s));
            }
            if (pair_sp) {
                PLHR_TRY_CUDA(lap32_apply_shifts(g, kp, P32, kp, AP32, kp, nullptr, 0, nullptr, X2_32 + na, ldsp,
                                                 sigma, s));
                PLHR_TRY(applyT32(na + kp, (const float*)X2_32, ldsp, QSP32));
                QSp = QSP32;
                QPp = QSP32 + na;
                ldqs = ldqp = ldsp;
            } else {
                if (T) PLHR_TRY(applyT32(na, (const float*)X3_32, na, QS32));
                if (T && np) {
                    PLHR_TRY_CUDA(
                        lap32_apply_shifts(g, kp, P32, kp, AP32, kp, nullptr, 0, nullptr, X3_32, kp, sigma, s));
                    PLHR_TRY(applyT32(kp, (const float*)X3_32, kp, QP32));
                }
            }
            const int nb = np ? 4 : 3;
            const int m = kp + 2 * na + np;
            last_m = m;
            BlkMx zb[4] = {{V32, kp, kp, 0}, {Wp, ldw, na, 0}, {S32, lds, na, 0}, {P32, kp, np, 0}};
            BlkMx ab[4] = {{U32, kp, kp, 0, 1}, {AW32, na, na, 0}, {AS32, na, na, 0}, {AP32, kp, np, 0}};
            BlkMx ub[4] = {{V, kp, kp, 1}, {Wp, ldw, na, 0}, {S32, lds, na, 0}, {P32, kp, np, 0}};
            BlkMx qb[4] = {{QVp, ldqv, kp, 0}, {QW32, 2 * na, na, 0}, {QSp, ldqs, na, 0}, {QPp, ldqp, np, 0}};
            PLHR_TRY_CUDA(cudaMemcpyAsync(colscale, scale, sizeof(double) * kp, cudaMemcpyDeviceToDevice, s));
            DenseArgs da;
            da.m = m; da.kp = kp; da.nv = kp;
            da.Gzz = grams; da.Guq = grams + m * m; da.Gqz = grams + 2 * m * m;
            da.colscale = colscale; da.work = dwork; da.Cp = Cp; da.Cvv = Cvv; da.tags = tags;
            da.tag_partner = partner; da.xi = xi; da.out_int = dstat + 3; da.clk = nullptr;
            {
                PhaseScope ps(PH_GRAM32, s, gram_flops(n, m), 4.0 * n * m * (T ? 3 : 2));
                if (opt.tensor_cores)
                    PLHR_TRY_CUDA(multi_gram_tc(n, nb, zb, ab, T ? qb : nullptr, sigma, colscale, gpart, grams,
                                                dstat + 7, s));
                else
                    PLHR_TRY_CUDA(multi_gram_mx(n, nb, zb, ab, T ? qb : nullptr, sigma, colscale, gpart, grams, s));
            }
            {
                PhaseScope ps(PH_DENSE, s);
                PLHR_TRY_CUDA(dense_extract(da, s));
            }
            PLHR_TRY_CUDA(cudaMemcpyAsync(hs->dense, dstat + 3, sizeof(int) * 3, cudaMemcpyDeviceToHost, s));
            PLHR_TRY_CUDA(cudaMemcpyAsync(&hs->pad, dstat + 7, sizeof(int), cudaMemcpyDeviceToHost, s));
            PLHR_TRY_CUDA(cudaStreamSynchronize(s));
            if (hs->pad) {
                set_error("plhr_solve: a tensor-core completion wait of the Gram timed out at iteration %d", it);
                result = PLHR_ECUDA;
                break;
            }
            if (hs->dense[0] != kDenseOK) {
                // the images are already explicit: leave the FP32 form and redo the
                // step in FP64 (the next pass of the loop, from the same V)
                mixed_its = it;
                PLHR_TRY(switch_to_f64(h_order));
                continue;
            }
            last_kept = hs->dense[1];
            {
                // read V (FP64) and W, S, P (FP32); write V (FP64) and P (FP32)
                PhaseScope ps(PH_UPDATE32, s, 2.0 * n * m * kp, (double)n * (8.0 * kp + 4.0 * (m - kp) + 12.0 * kp));
                PLHR_TRY_CUDA(block_update_mx(n, nb, ub, kp, Cp, Cvv, V, 1, kp, P32, 0, kp, s));
            }
            np = kp;
            PLHR_TRY(refresh_images());
            PLHR_TRY_CUDA(dense_rq(kp, dots, tags, partner, lam, scale, s));
            continue;
        }
        PLHR_TRY(applyT(na, Ract, ldra, W));
        const double* S = SQ;
        int64_t lds = na;
        const double* QW = SQ + na;
        int64_t ldqw = 2 * na;
        if (sv) {
            // ---------------------------------------- S = T(AW - BW Lambda), Q_W = T(AW - sigma BW)
            {
                // read W, write A W (B W) and the shifted outputs
                PhaseScope ps(PH_STENCIL, s, (double)n * na, prod_bytes(na, thq ? 2 : 1));
                if (thq)
                    PLHR_TRY(prod(na, W, na, AW, na, BW, na, X2, 2 * na, lam_act, X2 + na, 2 * na));
                else
                    PLHR_TRY(prod(na, W, na, AW, na, BW, na, T ? X2 : SQ, na, lam_act, nullptr, 0));
            }
            if (thq) {
                PLHR_TRY(applyT(2 * na, X2, 2 * na, SQ));
                lds = 2 * na;
            } else if (T) {
                PLHR_TRY(applyT(na, X2, na, SQ));
            }
            // ---------------------------------------- A S, Q_S = T(AS - sigma BS)
            {
                PhaseScope ps(PH_STENCIL, s, (double)n * na, prod_bytes(na, thq ? 1 : 0));
                PLHR_TRY(prod(na, S, lds, AS, na, BS, na, nullptr, 0, nullptr, thq ? X3 : nullptr, na));
            }
            if (thq) PLHR_TRY(applyT(na, X3, na, QS));
        } else {
            // ---------------------------------------- trial space [V W P]: A W and Q_W only
            {
                PhaseScope ps(PH_STENCIL, s, (double)n * na, prod_bytes(na, thq ? 1 : 0));
                PLHR_TRY(prod(na, W, na, AW, na, BW, na, nullptr, 0, nullptr, thq ? X2 : nullptr, na));
            }
            if (thq) PLHR_TRY(applyT(na, X2, na, SQ));
            QW = SQ;
            ldqw = na;
        }

        // -------------------------------------------- Grams over Z = [V W S P] (or [V W P]), AZ, Q (steps 6-7)
        // Recovery when the projected problem fails: first the carried images
        // T(A - sigma B)V, T(A - sigma B)P are recomputed explicitly (they may
        // have drifted), then the step is taken without the P block (a restart
        // of the search directions, trial space [V W S]).
        int nb = 0, m = 0, np_use = np;
        Blk<const double> zb[4], ab[4], qb[4], bzb[4];
        DenseArgs da;
        PLHR_TRY_CUDA(cudaMemcpyAsync(colscale, scale, sizeof(double) * kp, cudaMemcpyDeviceToDevice, s));
        for (int pass = 0; pass < 3; ++pass) {
            nb = (sv ? 3 : 2) + (np_use ? 1 : 0);
            m = kp + (sv ? 2 : 1) * na + np_use;
            last_m = m;
            zb[0] = {V, kp, kp}; zb[1] = {W, na, na}; zb[2] = {S, lds, na}; zb[3] = {P, kp, np_use};
            ab[0] = {AV, kp, kp}; ab[1] = {AW, na, na}; ab[2] = {AS, na, na}; ab[3] = {AP, kp, np_use};
            qb[0] = {QV, kp, kp}; qb[1] = {QW, ldqw, na}; qb[2] = {QS, na, na}; qb[3] = {QP, kp, np_use};
            bzb[0] = {BV, kp, kp}; bzb[1] = {BW, na, na}; bzb[2] = {BS, na, na}; bzb[3] = {BP, kp, np_use};
            if (!sv) {   // drop the S family: [V W P]
                zb[2] = zb[3];
                ab[2] = ab[3];
                qb[2] = qb[3];
                bzb[2] = bzb[3];
            }
            da.m = m; da.kp = kp; da.nv = kp;
            da.Gzz = grams; da.Guq = grams + m * m; da.Gqz = grams + 2 * m * m;
            da.colscale = colscale; da.work = dwork; da.Cp = Cp; da.Cvv = Cvv; da.tags = tags; da.tag_partner = partner;
            da.xi = xi; da.out_int = dstat + 3; da.clk = nullptr;
            {
                PhaseScope ps(PH_GRAM, s, gram_flops(n, m), 8.0 * n * m * ((thq ? 3 : 2) + (hasB ? 1 : 0)));
                if (dwf)
                    PLHR_TRY_CUDA(multi_gram_dw(n, nb, zb, ab, thq ? qb : nullptr, sigma, colscale, gpart, grams, s));
                else
                    PLHR_TRY_CUDA(multi_gram_b(n, nb, zb, ab, thq ? qb : nullptr, hasB ? bzb : nullptr, sigma, colscale,
                                               gpart, grams, s));
            }
            // ---------------------------------------- projected T-harmonic problem, selection (steps 7-10)
            {
                PhaseScope ps(PH_DENSE, s);
                PLHR_TRY_CUDA(dense_extract(da, s));
            }
            PLHR_TRY_CUDA(cudaMemcpyAsync(hs->dense, dstat + 3, sizeof(int) * 3, cudaMemcpyDeviceToHost, s));
            PLHR_TRY_CUDA(cudaStreamSynchronize(s));
            if (hs->dense[0] == kDenseOK) break;
            if (pass == 0 && thq) {
                PLHR_TRY(prod(kp, V, kp, AV, kp, BV, kp, nullptr, 0, nullptr, X3, kp));
                PLHR_TRY(applyT(kp, X3, kp, QV));
                if (np) {
                    PLHR_TRY(prod(kp, P, kp, AP, kp, BP, kp, nullptr, 0, nullptr, X3, kp));
                    PLHR_TRY(applyT(kp, X3, kp, QP));
                }
                continue;
            }
            if (np_use == 0) break;
            np_use = 0;
        }
        last_kept = hs->dense[1];
        if (hs->dense[0] != kDenseOK) {
            set_error("plhr_solve: projected problem failed at iteration %d (code %d)", it, hs->dense[0]);
            result = PLHR_EBREAKDOWN;
            break;
        }
        // -------------------------------------------- P, V (steps 11-12), images, RQs (13-14)
        {
            PhaseScope ps(PH_UPDATE, s, (thq ? 4.0 : 2.0) * n * m * kp, (thq ? 2.0 : 1.0) * 8.0 * n * (m + 2.0 * kp));
            if (dwf) {
                PLHR_TRY_CUDA(block_update_dw(n, nb, zb, kp, Cp, Cvv, V, kp, P, kp, s));
                if (thq) PLHR_TRY_CUDA(block_update_dw(n, nb, qb, kp, Cp, Cvv, QV, kp, QP, kp, s));
            } else {
                PLHR_TRY_CUDA(block_update(n, nb, zb, kp, Cp, Cvv, V, kp, P, kp, nullptr, 0, nullptr, nullptr, s));
                if (thq) PLHR_TRY_CUDA(block_update(n, nb, qb, kp, Cp, Cvv, QV, kp, QP, kp, nullptr, 0, nullptr, nullptr, s));
            }
        }
        np = kp;
        PLHR_TRY(refresh_images());
        PLHR_TRY_CUDA(dense_rq(kp, dots, tags, partner, lam, scale, s));
    }
    const double t2 = now_s();
    if (result == PLHR_OK || result == PLHR_ENOTCONV) {
        if (result == PLHR_ENOTCONV) {
            // final Rayleigh-Ritz on the current block
            PLHR_TRY_CUDA(lap_axpby(g, kp, V, kp, AW, kp, 1.0, 0.0, s));
            if (hasB) PLHR_TRY_CUDA(lap_axpby(B->g, kp, V, kp, X3, kp, 1.0, 0.0, s));
            Blk<const double> zb[1] = {{V, kp, kp}}, ab[1] = {{AW, kp, kp}}, qb[1] = {{V, kp, kp}},
                              bzb[1] = {{X3, kp, kp}};
            PLHR_TRY_CUDA(cudaMemcpyAsync(colscale, scale, sizeof(double) * kp, cudaMemcpyDeviceToDevice, s));
            PLHR_TRY_CUDA(multi_gram_b(n, 1, zb, ab, qb, hasB ? bzb : nullptr, 0.0, colscale, gpart, grams, s));
            PLHR_TRY_CUDA(dense_rr(kp, grams + kp * kp, grams, sigma, scale, Crr, theta, dstat + 6, s));
            PLHR_TRY_CUDA(block_times_small(n, V, kp, kp, Crr, kp, Rc, kp, s));
            PLHR_TRY_CUDA(lap_axpby(g, kp, Rc, kp, AW, kp, 1.0, 0.0, s));
            if (hasB) PLHR_TRY_CUDA(lap_axpby(B->g, kp, Rc, kp, X3, kp, 1.0, 0.0, s));
            std::vector<double> ones(kp, 1.0);
            PLHR_TRY_CUDA(cudaMemcpyAsync(dots, ones.data(), sizeof(double) * kp, cudaMemcpyHostToDevice, s));
            PLHR_TRY_CUDA(residual_norms(n, kp, hasB ? X3 : Rc, kp, AW, kp, theta, dots, R, kp, rpart, sums, s));
            StatusArgs sa;
            sa.kp = kp; sa.k = k; sa.sigma = sigma; sa.tol = tol;
            sa.sums = sums; sa.lam = theta; sa.lam_act = lam_act; sa.active = active; sa.rel = rel; sa.order = order;
            sa.hstat = dstat;
            PLHR_TRY_CUDA(dense_status(sa, s));
            PLHR_TRY_CUDA(cudaMemcpyAsync(h_rel, rel, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
            PLHR_TRY_CUDA(cudaMemcpyAsync(h_theta, theta, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
            PLHR_TRY_CUDA(cudaStreamSynchronize(s));
        }
        // Rc holds the Ritz vectors ordered by |theta - sigma|: the first k are returned
        PLHR_TRY_CUDA(cudaMemcpy2DAsync(eigvecs, sizeof(double) * ldv, Rc, sizeof(double) * kp, sizeof(double) * k, n,
                                        cudaMemcpyDeviceToDevice, s));
        PLHR_TRY_CUDA(cudaStreamSynchronize(s));
        double mx = 0.0;
        for (int q2 = 0; q2 < k; ++q2) {
            eigvals[q2] = h_theta[q2];
            mx = std::fmax(mx, h_rel[q2]);
        }
        if (info) info->max_rel_residual = mx;
    }
    if (info) {
        info->iterations = it;
        info->converged = result == PLHR_OK ? 1 : 0;
        info->setup_seconds = t1 - t0;
        info->solve_seconds = t2 - t1;
        info->history_len = hist;
        info->mixed_iterations = (opt.precision == PLHR_PRECISION_MIXED) ? (mx ? it : mixed_its) : 0;
    }
    cudaFreeAsync(big.p, s);
    cudaFreeAsync(part.p, s);
    cudaFreeAsync(small.p, s);
    cudaFreeAsync(ints, s);
    if (big32.p) cudaFreeAsync(big32.p, s);
    big32.p = nullptr;
    big.p = part.p = small.p = nullptr;
    int_free.p = nullptr;
    cudaStreamSynchronize(s);
    profile_flush();
    return result;
}
