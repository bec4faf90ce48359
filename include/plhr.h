/*
 * plhr.h - C ABI of the GB300 block PLHR library (libplhr.so).
 *
 * Block PLHR computes the k eigenpairs of the Hermitian problem
 *     A v = lambda B v,   A = A^*,  B = B^* > 0,
 * whose eigenvalues are closest to a real interior shift sigma
 * (Vecharynski & Knyazev, "Preconditioned locally harmonic residual method
 * for computing interior eigenpairs of certain classes of Hermitian
 * matrices", Section 1, Eq. eqn:eigp), using a Hermitian positive definite
 * preconditioner T ~ |A - sigma B|^{-1} (Section 5) and the T-harmonic
 * Rayleigh-Ritz extraction of Algorithm 2 / Algorithm 3 (Section 4).
 *
 * Conventions for every entry point
 *   - Blocks of vectors are n x ncols, row-major, FP64, in device memory:
 *     element (i, j) sits at ptr[i * ld + j], ld >= ncols.  Grid vectors are
 *     flattened with x fastest: i = (z * ny + y) * nx + x.
 *   - The caller owns every pointer it passes; the library never frees or
 *     retains them.  Opaque objects (plhr_op, plhr_prec) are owned by the
 *     library and released with their destroy call.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Entry points
 *     that only enqueue work return before it completes.
 *   - Errors are returned as plhr_status; nothing aborts, traps or prints.
 *     Invalid arguments give PLHR_EINVAL before any work is enqueued; a
 *     failing CUDA call gives PLHR_ECUDA (plhr_last_error() has the text).
 *   - Every entry point needs the CUDA device that holds the pointers to be
 *     current on the calling thread.
 */
#ifndef PLHR_H
#define PLHR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PLHR_OK = 0,
    PLHR_ENOTCONV = 1,   /* maxit reached; outputs hold the best current pairs */
    PLHR_EINVAL = 2,     /* invalid argument (null pointer, size, descriptor) */
    PLHR_EBREAKDOWN = 3, /* projected problem not solvable (G_L not positive definite) */
    PLHR_ENAN = 4,       /* NaN or Inf met in the iteration */
    PLHR_ENOMEM = 5,     /* device workspace allocation failed */
    PLHR_ECUDA = 6       /* CUDA runtime error */
} plhr_status;

/* ------------------------------------------------------------------ operators
 * A model operator given by a stencil on a tensor grid.
 *   LAP5_2D / LAP7_3D: the negative finite-difference Laplacians of Section
 *     5.2 ("standard 5-point FD discretization"; the 7-point 3D analogue):
 *         (L u)_i = scale * sum_axes (2 u_i - u_{i-e} - u_{i+e}) / h^2,
 *     values outside the grid zero (bc = DIRICHLET) or wrapped around
 *     (bc = PERIODIC).
 *   HAM7_BLOCH: the Bloch Hamiltonian H = -1/2 Lap_kappa + diag(V) of the
 *     complex Hermitian problems of Section 5.3 on a periodic 3D grid at
 *     crystal momentum kappa = bloch_k: the link from point j to j + e_d
 *     carries the phase e^{i kappa_d h},
 *         (H u)_j = 1/2 sum_d (2 u_j - e^{i kappa_d h} u_{j+e_d}
 *                   - e^{-i kappa_d h} u_{j-e_d}) / h^2 + V_j u_j
 *     (indices wrap; a plane wave e^{i theta j} has the kinetic eigenvalue
 *     (1 - cos(theta + kappa h)) / h^2 per axis); field = V (device, n
 *     doubles, caller-owned, kept alive while the operator is used); scale
 *     and bc ignored.  Complex blocks: plhr_op_apply_c128; real blocks only
 *     when kappa = 0.
 *   Q1_STIFF27 / Q1_MASS27: the trilinear (Q1) finite-element stiffness of
 *     -div(c grad u) and the mass matrix (Section 5.1's bilinear elements in
 *     3D) on the unit cube with E = dims[a] + 1 elements per axis, h = 1/E,
 *     homogeneous Dirichlet (the unknowns are the dims[0] x dims[1] x dims[2]
 *     interior nodes, x fastest; dims need not be equal, h is taken from the
 *     descriptor); 27-point stencils assembled from the element matrices
 *     c_e (k (x) m (x) m + m (x) k (x) m + m (x) m (x) k) and m (x) m (x) m of
 *     the 1D linear element (k = [[1, -1], [-1, 1]] / h, m = [[2, 1], [1, 2]]
 *     h / 6).  field (STIFF only) = the element coefficients c_e (device,
 *     (dims[0]+1)(dims[1]+1)(dims[2]+1) positive doubles, x fastest,
 *     caller-owned) or NULL for c = 1; scale multiplies the matrix. */
typedef enum {
    PLHR_STENCIL_LAP5_2D = 1,
    PLHR_STENCIL_LAP7_3D = 2,
    PLHR_STENCIL_HAM7_BLOCH = 3,
    PLHR_STENCIL_Q1_STIFF27 = 4,
    PLHR_STENCIL_Q1_MASS27 = 5
} plhr_stencil_kind;

typedef enum { PLHR_BC_DIRICHLET = 0, PLHR_BC_PERIODIC = 1 } plhr_bc;

typedef struct {
    int kind;            /* plhr_stencil_kind */
    int64_t dims[3];     /* grid points (interior nodes) per axis (x, y, z); dims[2] = 1 for 2D */
    double h;            /* mesh width, > 0 */
    double scale;        /* multiplier of the stencil, > 0 (1 for -Laplacian) */
    int bc;              /* plhr_bc (LAP kinds) */
    double bloch_k[3];   /* HAM7_BLOCH: crystal momentum kappa */
    const double* field; /* HAM7_BLOCH: potential V; Q1_STIFF27: element coefficients or NULL */
} plhr_stencil_desc;

typedef struct plhr_op plhr_op;

/* Create a stencil operator.  *out is set only on PLHR_OK. */
plhr_status plhr_op_stencil(plhr_op** out, const plhr_stencil_desc* desc);
/* Number of rows n of the operator (0 for NULL). */
/* Real-space Hamiltonian H = -1/2 Lap_h + diag(V) on a d-dimensional grid
 * (d = 2, 3; dims[2] ignored for d = 2) with mesh width h: the 5/7-point
 * Laplacian above with scale 1/2, neighbours outside the grid zero
 * (periodic = 0) or wrapped around (periodic = 1), and the potential V given
 * as a device array of n doubles (x fastest) that the caller keeps alive and
 * unchanged while the operator is in use.  The role of the Hamiltonians of
 * Section 5.3 in the synthetic differentiation workload.  Supported by
 * plhr_op_apply and by plhr_solve in PLHR_PRECISION_F64. */
plhr_status plhr_op_hamiltonian(plhr_op** out, int d, const int64_t* dims, double h, int periodic,
                                const double* potential);
/* A general sparse symmetric operator A (n x n, FP64) in CSR form: row i
 * holds val[p] at column col[p] for rowptr[i] <= p < rowptr[i+1]
 * (rowptr: n + 1 int64 values starting at 0; col: int32 in [0, n)).  The
 * arrays are host memory, or device memory when is_device != 0; they are
 * copied (the caller may free them afterwards) and the structure is checked
 * on the host (PLHR_EINVAL on a decreasing rowptr or a column out of range).
 * Symmetry is the caller's promise: it is not checked.  Usable by
 * plhr_op_apply, plhr_solve (PLHR_PRECISION_F64) and plhr_eigvec_adjoint;
 * not by AV-MG or TPA (use plhr_prec_diag, plhr_prec_callback or T = NULL). */
plhr_status plhr_op_csr(plhr_op** out, int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                        int is_device);
int64_t plhr_op_size(const plhr_op* op);
void plhr_op_destroy(plhr_op* op);

/* Y = op X for an n x ncols block (ncols >= 0).  X and Y must not overlap.
 * PLHR_EINVAL for a Bloch operator with kappa != 0 (complex). */
plhr_status plhr_op_apply(const plhr_op* op, int ncols, const double* X, int64_t ldx,
                          double* Y, int64_t ldy, void* stream);
/* Y = op X for complex blocks: element (i, j) is the pair (re, im) of doubles
 * at X[2 (i * ldx + j)], X[2 (i * ldx + j) + 1] (complex128 row-major, ld in
 * complex elements).  Any stencil operator (a real one acts on the real and
 * imaginary parts alike); not CSR. */
plhr_status plhr_op_apply_c128(const plhr_op* op, int ncols, const double* X, int64_t ldx,
                               double* Y, int64_t ldy, void* stream);
/* AX = A X and BX = B X in one pass over X, for the Q1 pair (A Q1_STIFF27,
 * B Q1_MASS27 on the same mesh); any other pair of operators of equal size is
 * applied one after the other.  Blocks as for plhr_op_apply. */
plhr_status plhr_op_apply_pair(const plhr_op* A, const plhr_op* B, int ncols, const double* X, int64_t ldx,
                               double* AX, int64_t ldax, double* BX, int64_t ldbx, void* stream);

/* ------------------------------------------------------------- preconditioner
 * T ~ |L - sigma I|^{-1}: the absolute-value multigrid V-cycle of Appendix A,
 * Algorithm 4 ("AV-MG"), for a stencil Laplacian L.  On level l the smoother
 * works with B_l = L_l when sqrt(sigma) h_l < delta, otherwise with the
 * polynomial B_l = p_2(L_l - sigma I_l) = ((L_l - sigma I_l)^2 + c_l^2 I)/(2 c_l);
 * nu Richardson steps w <- w + omega_l (r - B_l w) before and after the
 * coarse-grid correction; cell-centred coarsening by two per axis (average
 * of the 2^d children, piecewise-constant prolongation); the exact
 * |L_0 - sigma I_0|^{-1} on the coarsest grid.  T is symmetric positive
 * definite. */
typedef struct {
    int levels;        /* number of grids, >= 1 (1 = exact |L - sigma I|^{-1}) */
    int nu;            /* smoothing steps before and after, >= 1 */
    double delta;      /* resolution threshold for B_l = L_l (default 2 pi / 10) */
    int transfer;      /* 0: piecewise-constant prolongation / averaging restriction;
                          1: trilinear cell-centred prolongation (1D weights 3/4, 1/4),
                             restriction P^T / 2^d */
    int coarse;        /* coarsest |L_0 - sigma I_0|^{-1}: 0 = L_0 the Laplacian
                          rediscretised with h_0 = 2^(levels-1) h; 1 = L_0 with the
                          cell-centred sine modes as eigenvectors and the fine grid's
                          eigenvalues of the same modes */
    int indefinite;    /* 1: INV-MG of Appendix A, Algorithm 5 instead: the same cycle for
                          (L - sigma I) w = r (B_l = L_l - sigma I_l on every level,
                          Richardson step 1 / max |Gershgorin bound of L_l - sigma I_l|,
                          exact (L_0 - sigma I_0)^{-1} on the coarsest grid), an indefinite
                          T ~ (L - sigma I)^{-1}: usable by plhr_prec_apply and by
                          plhr_solve with the harmonic extraction (extraction = 1, FP64)
                          only, the combination of Section 5.2's Table tab:laplace10;
                          default 0 */
} plhr_mg_opts;

typedef struct plhr_prec plhr_prec;

void plhr_mg_opts_default(plhr_mg_opts* o);
/* Build the hierarchy for the stencil operator A (LAP5_2D or LAP7_3D from
 * plhr_op_stencil, Dirichlet; every axis size divisible by 2^(levels-1);
 * PLHR_EINVAL for a Hamiltonian operator).  opts NULL = defaults. */
plhr_status plhr_prec_avmg(plhr_prec** out, const plhr_op* A, double sigma,
                           const plhr_mg_opts* opts);
/* The Teter-Payne-Allan preconditioner of Section 5.3 (Teter, Payne, Allan,
 * Phys. Rev. B 40, 12255, 1989) on the grid of A: a positive diagonal matrix
 * in the basis of the grid's kinetic modes,
 *     T = S diag(K(mu / energy)) S^T,
 *     K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4),
 * S the orthonormal eigenvectors of A's stencil part (real Fourier modes on
 * a periodic grid, sine modes on a Dirichlet grid), mu their eigenvalues.  T
 * is symmetric positive definite and the same for every column.  energy <= 0
 * selects sigma - min(potential) when positive, else the mean of mu.  Any
 * stencil or Hamiltonian operator whose axis sizes are at most 144 (an
 * application takes 8 (N^2 + N ncols) <= 200 KB for every axis size N, else
 * PLHR_ECUDA with an invalid-value error); the potential is read once here.
 * The transforms run in double-word arithmetic (~1e-12 relative rounding per
 * application): PLHR with this T reaches relative residuals near 1e-11, below
 * which the T-harmonic iteration stalls (use T = NULL for tighter
 * tolerances).  Usable by plhr_solve (PLHR_PRECISION_F64), plhr_prec_apply
 * and plhr_eigvec_adjoint. */
plhr_status plhr_prec_tpa(plhr_prec** out, const plhr_op* A, double sigma, double energy);
/* The reference energy a TPA preconditioner uses (0 for other kinds). */
double plhr_prec_tpa_energy(const plhr_prec* T);
/* T = diag(d) for n positive finite values d (host, or device when
 * is_device != 0; copied, so the caller may free d afterwards).  PLHR_EINVAL
 * when an entry is not positive and finite. */
plhr_status plhr_prec_diag(plhr_prec** out, int64_t n, const double* d, int is_device);
/* A caller-supplied preconditioner: the library calls
 *     fn(ctx, ncols, R, ldr, W, ldw, stream)
 * to form W = T R (device n x ncols blocks, row-major; W dense, ldw == ncols)
 * on the solver's stream and continues only when it returns PLHR_OK (any
 * other status ends the calling solve or apply with that status).  T must be
 * symmetric positive definite and the same operator on every call (the
 * T-harmonic images are carried by linear updates). */
typedef plhr_status (*plhr_apply_fn)(void* ctx, int ncols, const double* R, int64_t ldr, double* W, int64_t ldw,
                                     void* stream);
plhr_status plhr_prec_callback(plhr_prec** out, int64_t n, plhr_apply_fn fn, void* ctx);
void plhr_prec_destroy(plhr_prec* T);
/* W = T R for an n x ncols block.  R and W must not overlap.  Uses device
 * workspace owned by T (grown on demand; calls on one T must not overlap). */
plhr_status plhr_prec_apply(plhr_prec* T, int ncols, const double* R, int64_t ldr,
                            double* W, int64_t ldw, void* stream);
/* The same V-cycle in FP32 storage and arithmetic (the form the mixed-precision
 * solve uses): W = T R for FP32 blocks.  Workspace as for plhr_prec_apply.
 * AV-MG only (PLHR_EINVAL for a TPA preconditioner).  This form and the
 * double-word one below run the cycle as a CUDA graph: the first call with a
 * given (ncols, R, ldr, W, ldw) captures the cycle's launches on a stream T
 * owns (nothing runs during the capture) and launches the graph on `stream`;
 * later calls with the same arguments replay it.  T keeps up to 64 graphs
 * (the oldest is dropped) and releases them when its workspace is
 * reallocated or T is destroyed.  Do not call these two while `stream` is
 * itself being captured into a graph. */
plhr_status plhr_prec_apply_f32(plhr_prec* T, int ncols, const float* R, int64_t ldr,
                                float* W, int64_t ldw, void* stream);
/* The same V-cycle with double-word storage and arithmetic (hi + lo FP32
 * pairs, ~48-bit significands, run on the FP32 pipes) on FP64 blocks: the
 * form the FP64 phase of the mixed-precision solve uses.  Same arguments,
 * workspace and overlap rules as plhr_prec_apply.  AV-MG only. */
plhr_status plhr_prec_apply_dw(plhr_prec* T, int ncols, const double* R, int64_t ldr,
                               double* W, int64_t ldw, void* stream);

/* -------------------------------------------------------------------- solver */
typedef enum {
    PLHR_PRECISION_F64 = 0,   /* every step in FP64 */
    PLHR_PRECISION_MIXED = 1  /* FP32 operator/preconditioner, FP64 projection */
} plhr_precision;

typedef struct {
    int maxit;                 /* iteration cap (default 1000) */
    int precision;             /* plhr_precision */
    int real_arithmetic;       /* 1: Algorithm 3 with k' = k + 1 columns (default) */
    int s_vectors;             /* 1: trial space [V W S P] (default); 0: [V W P] */
    int soft_lock;             /* 1: converged columns add no W, S columns (default) */
    const double* v_init;      /* device n x k' starting block, or NULL (seeded) */
    int64_t ld_init;
    uint64_t seed;             /* SplitMix64 seed used when v_init == NULL */
    double* history;           /* host, history_cap * (2 k' + 3) doubles, or NULL: per
                                  iteration [it, Ritz values (k'), rel. residuals (k'),
                                  trial-basis columns kept, trial-basis size] ordered by
                                  distance to sigma */
    int history_cap;
    int guard;                 /* extra block columns beyond k (real arithmetic: k' = k + guard,
                                  default 1 as the paper suggests: "(at least) by 1"); more guard
                                  columns make it less likely that a wanted pair of a degenerate
                                  cluster is left out; 4 (k + guard) <= 64 */
    double switch_tol;         /* PLHR_PRECISION_MIXED: the iteration runs W, S, P, the Q images,
                                  the operator products on them and the V-cycles in FP32 (V and
                                  A V stay FP64) until the relative residuals of the k pairs
                                  nearest sigma are all below switch_tol (or have stopped
                                  improving for 25 iterations below 1e-5), then continues in
                                  FP64 with the images recomputed explicitly and the columns beyond the
                                  k nearest restarted from seeded random vectors (default 1e-6) */
    int extraction;            /* 0: T-harmonic Rayleigh-Ritz (Section 3.1, default); 1: harmonic
                                  (T = I in the Petrov-Galerkin condition, Section 5.1's
                                  comparison).  extraction 1 and s_vectors 0 (the trial space
                                  [V W P] of the ablation in Section 5.1) run in PLHR_PRECISION_F64;
                                  2: the refinement of Section 3.3 (Eq. rRR): the single-vector
                                  method (k = 1, guard = 0, FP64) whose new v minimises
                                  ||(A - lam B) v||_T over span[v w s p], lam the current Rayleigh
                                  quotient (the preconditioned locally minimal residual method; it
                                  converges to the eigenpair its start vector is close to, not
                                  necessarily the one nearest sigma; sigma is not used) */
    int tensor_cores;          /* PLHR_PRECISION_MIXED: 1 (default) forms the Grams of the FP32
                                  phase on the tensor cores (split-BF16 slices, FP32 accumulation,
                                  PLHR_GRAM_F32_TC of plhr_gram); 0 on the FP32 pipes
                                  (PLHR_GRAM_F32) */
} plhr_options;

typedef struct {
    int iterations;            /* iterations taken */
    int converged;             /* 1 when all k relative residuals <= tol */
    double max_rel_residual;   /* max over the k returned pairs (explicit A V, B V) */
    double setup_seconds;      /* host wall time before the first iteration */
    double solve_seconds;      /* host wall time of the iteration loop */
    int history_len;           /* records written to options.history */
    int mixed_iterations;      /* iterations run in the FP32 form (PLHR_PRECISION_MIXED) */
} plhr_info;

void plhr_options_default(plhr_options* o);

/* Gradient of sum_k w_k lambda_k with respect to the potential of a
 * Hamiltonian: g (device, n) = sum_k w_k V(:,k)^2 for B-orthonormal
 * eigenvectors V (device n x k, leading dimension ldv >= k, as plhr_solve
 * returns them) and host weights w (k values, 1 <= k <= 64): first-order
 * perturbation theory (Hellmann-Feynman), d lambda_k / d V_i = v_k(i)^2. */
plhr_status plhr_eigval_grad(int64_t n, int k, const double* V, int64_t ldv, const double* weights, double* g,
                             void* stream);

/* Gradient with respect to the potential of a loss L on the eigenvectors of
 * a Hamiltonian operator A (plhr_op_hamiltonian; B = I): given k
 * orthonormal eigenvectors V (device n x k, leading dimension ldv >= k, as
 * plhr_solve returns them), their eigenvalues lam (HOST, k values) and
 * G = dL/dV (device n x k, leading dimension ldg >= k), first-order
 * perturbation theory gives
 *     grad (device, n) = sum_c V(:,c) .* b_c,
 *     b_c = sum_{j != c} V(:,j) (V(:,j)^T G(:,c)) / (lam_c - lam_j) - a_c,
 * where a_c solves (A - lam_c I) a_c = P G(:,c) on the orthogonal
 * complement of the block (P = I - V V^T).  The k systems are solved
 * together by MINRES on P (A - lam_c I) P, preconditioned by P T P when T is
 * non-null (T symmetric positive definite: plhr_prec_tpa, or AV-MG for a
 * Laplacian; its workspace grows to k columns), to relative residual tol in
 * the preconditioned norm (at most maxit iterations; the count taken is
 * written to *iterations when non-null).  Pairs with |lam_c - lam_j| <= 1e-12 max(1,
 * |lam_0|) contribute no in-block term (a repeated eigenvalue has no
 * eigenvector derivative inside its eigenspace).  1 <= k <= 16.  The call
 * synchronises the stream (it reads two inner products per iteration) and
 * allocates its own device workspace (9 n x k doubles).  PLHR_EINVAL on bad
 * arguments, PLHR_ENOMEM when the workspace cannot be allocated, PLHR_ENAN
 * on a non-finite inner product, PLHR_ENOTCONV when maxit is reached (grad
 * then holds the result of the last iterate). */
plhr_status plhr_eigvec_adjoint(const plhr_op* A, plhr_prec* T, int k, const double* lam, const double* V,
                                int64_t ldv, const double* G, int64_t ldg, double tol, int maxit, double* grad,
                                int* iterations, void* stream);

/* Compute the k eigenpairs of A v = lambda B v nearest sigma.
 *   A        stencil (plhr_op_stencil), Hamiltonian (plhr_op_hamiltonian) or
 *            CSR (plhr_op_csr); PLHR_PRECISION_MIXED takes the Dirichlet
 *            Laplacian with AV-MG or T = NULL only.
 *   B        NULL = identity; else a symmetric positive definite operator of
 *            A's size (stencil, Hamiltonian or CSR), PLHR_PRECISION_F64 only:
 *            the B images of V, W, S, P are formed explicitly, the Grams are
 *            Z^T B Z, U^T Q and Q^T B Z with U = A Z - sigma B Z, and the
 *            returned vectors are B-orthonormal.
 *   T        NULL = identity (no preconditioning); AV-MG, TPA, diagonal or
 *            callback, symmetric positive definite.
 *   tol      relative residual ||A v - lambda B v|| / (max(|lambda|, 1) ||B v||).
 *   eigvals  host, k doubles, ordered by |lambda - sigma| (ties: smaller first).
 *   eigvecs  device n x k block (ldv >= k), B-orthonormal Ritz vectors.
 * Returns PLHR_OK on convergence, PLHR_ENOTCONV after maxit iterations (the
 * outputs then hold the current approximations).  The call synchronises
 * `stream` once per iteration. */
plhr_status plhr_solve(const plhr_op* A, const plhr_op* B, double sigma, int k,
                       plhr_prec* T, double tol, const plhr_options* opt,
                       double* eigvals, double* eigvecs, int64_t ldv,
                       plhr_info* info, void* stream);

/* ------------------------------------------------- projected problem (device)
 * One extraction step of the T-harmonic Rayleigh-Ritz procedure (Section 3.1,
 * Eq. THarm_evp, solved through Eq. THarm_evp_sinv) with the selection of
 * Algorithm 3 steps 7-10, on device data.  The trial basis is Z D (m columns,
 * D = diag(colscale)), its first nv columns the V block; inputs are the
 * m x m row-major Grams Gzz = (ZD)^T B (ZD), Guq = (UD)^T (QD),
 * Gqz = (QD)^T B (ZD) with U = (A - sigma B) Z and Q = T U.  Z is
 * B-orthonormalised implicitly (Cholesky of the column-normalised Gzz; columns
 * whose pivot^2 < 1e-12 are dropped), the pencil G_L y = xi G_R y is reduced
 * with G_L = L L^T and solved by Hessenberg/Francis QR, the k' = kp
 * eigenvectors of smallest |xi| are selected with conjugate pairs kept
 * together (a pair cut at position kp keeps its real part), and the outputs are
 * coefficients on the raw columns: P_new = Z C_P (Cp, m x kp) and
 * V_new = V C_VV + P_new (Cvv, nv x kp).  tags/partner (kp ints): column kind
 * 0 real, 1 real part of a pair, 2 cut column, 3 imaginary part, and the pair
 * partner column; xi: 2 kp doubles (re, im of each selected unit);
 * status (device, 3 ints): [0 ok / 1 G_L not positive definite / 2 QR did not
 * converge / 3 rank loss, columns kept, units selected]; clk (device, 16 long
 * long, optional): clock64 stamps of the stages in [0..8] (the stage runs as
 * three launches: [0..2] and [5..8] come from the first and last, [3], [4]
 * bracket the QR iteration in the middle one; SM clocks of different launches
 * are not comparable), the number of QR sweeps in [9] and of bulge-chase
 * steps in [10].  m <= 64, kp <= 16. */
plhr_status plhr_tharm_extract(int m, int kp, int nv, const double* Gzz, const double* Guq,
                               const double* Gqz, const double* colscale, double* Cp, double* Cvv,
                               int* tags, int* partner, double* xi, int* status, long long* clk,
                               void* stream);

/* Same computation as plhr_tharm_extract, for callers that cannot allocate
 * device memory when they call it: an application whose allocator owns all of
 * the device memory, a service with a fixed memory budget that forbids
 * allocation after start-up, or code running from a host callback where an
 * allocation could block.  The paper has no counterpart: this is a property
 * of the library, not of the method.
 *   - Scratch comes from a 263 KiB array built into the library (enough for
 *     the largest supported m = 64); every GPU that loads the library keeps it
 *     until the process exits.  m > 64 is rejected with PLHR_EINVAL.
 *   - The call performs no cudaMalloc, cudaFree or other allocation.  Its first
 *     call on a device looks up the array's device address for that device
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture.  The address is kept for the life of the
 *     process: do not call this entry point after cudaDeviceReset on that
 *     device (the array then lives at a new address).
 *   - All calls share the one array, which keeps the last call's contents (the
 *     solver writes every scratch element it reads, so nothing needs clearing).
 *     Calls whose work overlaps on the GPU, e.g. on two streams at once, race
 *     on the array: serialise them.
 * Arguments, outputs and status are those of plhr_tharm_extract (no clk). */
plhr_status plhr_tharm_extract_noalloc(int m, int kp, int nv, const double* Gzz, const double* Guq,
                                       const double* Gqz, const double* colscale, double* Cp, double* Cvv,
                                       int* tags, int* partner, double* xi, int* status, void* stream);

/* ------------------------------------------------------- projected Grams (device)
 * The Gram pass of the solver on caller blocks, in one of its arithmetic
 * forms: with the trial basis Z = [Z_0 .. Z_{nb-1}] (nb <= 4 blocks of
 * ncols[b] columns, m = sum ncols in 1..64), its image AZ (same block shapes)
 * and, when Q is non-NULL, its T-harmonic image Q (Q NULL: Q = U), all columns
 * scaled by colscale (device, m doubles, D = diag(colscale)),
 *     out[0 .. m^2)        = (Z D)^T (Z D)
 *     out[m^2 .. 2 m^2)    = (U D)^T (Q D),   U = AZ - sigma Z
 *     out[2 m^2 .. 3 m^2)  = (Q D)^T (Z D)
 * (row-major m x m, device, FP64): the Grams of Eq. THarm_evp for B = I
 * (G_L = U^T T U = U^T Q, G_R = (T U)^T Z), Algorithm 2 steps 6-7.  The
 * first two are symmetric for Q = T U with T symmetric (and for Q = U): the
 * pass forms their upper triangles and mirrors them (for an input with a
 * non-symmetric U^T Q the lower triangle is the mirror of the upper).  The
 * tensor-core form computes the full U^T Q.  Block b
 * has n rows, element (i, j) at Z[b][i * ldz[b] + j] (host arrays of device
 * pointers and leading dimensions).  Forms:
 *   PLHR_GRAM_F64     FP64 blocks, FP64 products and sums;
 *   PLHR_GRAM_F32     FP32 blocks, FP32 products on the FP32 pipes, sums
 *                     folded into double-FP32 every 32 rows;
 *   PLHR_GRAM_DW      FP64 blocks, double-word (hi + lo FP32) arithmetic;
 *   PLHR_GRAM_F32_TC  FP32 blocks on the tensor cores (tcgen05): each value
 *                     split into three BF16 slices, the six slice products of
 *                     order <= 2 accumulated in FP32 in tensor memory, folded
 *                     into double-FP32 every 128 rows (the form the
 *                     mixed-precision solve uses).
 * Allocates a partial-sum buffer (max(2 x SMs, 152) x 3 m^2 doubles) on the
 * stream, synchronises the stream before returning.  PLHR_EINVAL for bad
 * arguments, PLHR_ECUDA on a CUDA error or a timed-out tensor-core wait. */
enum { PLHR_GRAM_F64 = 0, PLHR_GRAM_F32 = 1, PLHR_GRAM_DW = 2, PLHR_GRAM_F32_TC = 3 };
plhr_status plhr_gram(int form, int64_t n, int nb, const int* ncols, const void* const* Z, const int64_t* ldz,
                      const void* const* AZ, const int64_t* ldaz, const void* const* Q, const int64_t* ldq,
                      double sigma, const double* colscale, double* out, void* stream);

/* ---------------------------------------------------------------- utilities */
const char* plhr_status_string(plhr_status s);
/* Number of CUDA kernels the library has launched in this process. */
long long plhr_kernel_launches(void);
/* Phase timing with CUDA events recorded on the launching stream, around the
 * solver's phases: 0 stencil products, 1 preconditioner applications (FP64),
 * 2 Gram pass (FP64), 3 coefficient updates (FP64), 4 small dense device
 * stages, 5 residual pass, 6 preconditioner applications in FP32, 7 Gram pass
 * of the FP32 form, 8 coefficient update of the FP32 form.  Off by default;
 * enabling adds two events per phase call. */
void plhr_profile_enable(int on);
/* ms[9], calls[9] (either may be NULL): accumulated milliseconds and calls per
 * phase since the last reset; reset != 0 clears the accumulators.  Waits for
 * the recorded events. */
void plhr_profile_read(double* ms, long long* calls, int reset);
/* work[9]: algorithmic work accumulated per phase since the last reset of
 * plhr_profile_read: stencil products and residual pass: grid points x
 * columns; preconditioner phases: finest-level grid points x columns of the
 * V-cycles; Gram phases: flops 2 n (m(m+1) + m^2) (the upper triangles of
 * Z^T Z and U^T Q, which are symmetric, and Q^T Z for an n x m trial basis); update phases: flops 2 n m k' per
 * updated family; dense: 0. */
void plhr_profile_work(double* work);
/* bytes[9]: algorithmic HBM bytes accumulated per phase since the last reset
 * of plhr_profile_read, counting every operand block read once and every
 * result block written once per call (the unit of the roofline of these
 * bandwidth-bound passes): stencil products (1 + outputs) x element size per
 * grid point x column; AV-MG V-cycles 14.25 passes per smoothing level (the
 * fused first two sweeps 2, residual 3, restriction 1 1/8, prolongation with
 * correction 2 1/8, two post-sweeps 6) summed over the levels above the
 * coarsest; Grams the Z, AZ (, BZ) and Q families once (3 n m elements);
 * updates the m input columns once and the V and P outputs once per updated
 * family; residual pass V, AV read and R written; dense: 0. */
void plhr_profile_bytes(double* bytes);
/* Text of the last error recorded on the calling thread ("" if none). */
const char* plhr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PLHR_H */
