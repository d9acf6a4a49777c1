/*
 * rk.h — C ABI of the GB300 recycling Krylov library (librk.so).
 *
 * Solves sequences of nonsymmetric linear systems A x_t = b_t whose matrix A
 * is a 7- or 19-point stencil on a structured 3-D grid (the pressure Poisson
 * systems of eq. 1, Sec. 2.1, stored as bands: "Data Layout", Sec. 2.1) with
 * the Krylov methods of Sec. 2.2-2.4:
 *   RK_GMRES      GMRES(m), Algorithm 1;
 *   RK_RGCROT     rGCROT(m,k) with a recycle space carried across solves,
 *                 Algorithm 3 (recycle update after each cycle by harmonic Ritz
 *                 vectors);
 *   RK_RBICGSTAB  rBiCGStab with one recycle space, Algorithm 4 (k = 0 or no
 *                 recycle space: plain BiCGStab, Algorithm 2);
 *   RK_HYBRID     rGCROT for the first `hybrid_switch` solves of a problem,
 *                 then rBiCGStab with that recycle space frozen (Sec. 2.4).
 * All solvers are right-preconditioned by point Jacobi, M = diag(A)
 * (the preconditioner of Sec. 2.1, restricted to its point-Jacobi sweep).
 *
 * Conventions
 *  - Grid: nx*ny*nz cells, cell index i + nx*(j + ny*k) (x fastest).
 *  - Bands: coef is S (7 or 19) contiguous arrays of N doubles; band s
 *    multiplies the unknown at offset OFF[s]:
 *      0 (0,0,0); 1 (-1,0,0) 2 (1,0,0) 3 (0,-1,0) 4 (0,1,0) 5 (0,0,-1) 6 (0,0,1);
 *      7 (-1,-1,0) 8 (1,-1,0) 9 (-1,1,0) 10 (1,1,0);
 *      11 (-1,0,-1) 12 (1,0,-1) 13 (-1,0,1) 14 (1,0,1);
 *      15 (0,-1,-1) 16 (0,1,-1) 17 (0,-1,1) 18 (0,1,1).
 *    Periodic axes wrap; a band pointing out of a non-periodic face must be
 *    exactly 0 (checked by rk_create_problem).
 *  - The recycle space is stored in x-space: U, C are N x k column-major
 *    (column c at offset c*N) with A U = C and C^T C = I; the R of the QR that forms C
 *    is folded into U. Inside the library U, C and the Arnoldi basis are
 *    stored in FP64 and every projection, orthogonalisation, Gram and
 *    recycle-update product is FP64 arithmetic (precisions RK_FP64 and
 *    RK_MIXED); with RK_DF they are kept as double-float pairs (hi + lo of
 *    two FP32 numbers, about 48 significant bits) and that arithmetic runs in
 *    double-float on the FP32 pipe. A stored space is converted in place when
 *    a solve of the other kind comes (one rounding to double-float). A
 *    recycle space set and read back is bit-exact in FP64 storage and agrees
 *    to about 2^-46 relative in double-float storage.
 *  - Every pointer argument named "device" is CUDA device memory owned by
 *    the caller and only read or written during the call. Host pointers are
 *    named so. All GPU work is ordered on the stream passed to the call; the
 *    call returns after that stream's work for it has completed (it
 *    synchronises on the stream, never on the device).
 *  - Errors: every entry point returns an rk_status; RK_OK = 0. Nothing
 *    throws across the ABI. rk_last_error() gives a thread-local message.
 */
#ifndef RK_H
#define RK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RK_OK = 0,
  RK_E_INVALID = 1,          /* bad argument, stencil band pointing out of a wall, NaN in b */
  RK_E_OOM = 2,              /* the allocator returned NULL */
  RK_E_NOT_CONVERGED = 3,    /* max_matvec reached; x holds the last iterate */
  RK_E_BREAKDOWN = 4,        /* rBiCGStab breakdown persisted through max restarts */
  RK_E_RECYCLE_INVARIANT = 5,/* rk_set_recycle: ||A U - C|| or ||C^T C - I|| too large */
  RK_E_DEVICE_TIMEOUT = 6,   /* a bounded device wait gave up */
  RK_E_CUDA = 7              /* a CUDA runtime call failed */
} rk_status;

typedef enum { RK_GMRES = 0, RK_RGCROT = 1, RK_RBICGSTAB = 2, RK_HYBRID = 3 } rk_mode;
typedef enum { RK_FP64 = 0, RK_MIXED = 1, RK_DF = 2 } rk_precision;

/*
 * The preconditioner M (Sec. 2.1, "Preconditioners").
 * RK_PC_JACOBI: point Jacobi, M = diag(A).
 * RK_PC_SUBDOMAIN: the paper's sub-domain Jacobi preconditioner. The grid is
 * cut into boxes of 16 x 8 x 8 owned cells (the last box along an axis takes
 * the remainder); each box grown by one cell per side (wrapping on periodic
 * axes, cut at non-periodic faces) carries the local problem "A restricted to
 * the grown box" (couplings leaving it dropped), solved inexactly by 5 damped
 * Jacobi sweeps z <- z + omega D^{-1} (r - A_loc z) from z = 0 with
 * omega = 2/3; each box keeps its own cells' values (restricted additive
 * Schwarz), and one damped point-Jacobi sweep z <- z + omega D^{-1} (r - A z)
 * on the whole grid follows. A fixed linear operator, evaluated in FP64 in a
 * fixed order (bands in storage order, one fma each):
 *   s = a_0 z_p; s = fma(a_t, z_nb, s); u = dinv_p (r_p - s); z_p <- fma(omega, u, z_p).
 */
typedef enum { RK_PC_JACOBI = 0, RK_PC_SUBDOMAIN = 1 } rk_preconditioner;

typedef struct {
  int32_t nx, ny, nz;
  uint8_t periodic[3]; /* nonzero: that axis wraps */
  uint8_t reserved;
} rk_grid;

typedef struct {
  double tol;            /* stop when ||b - A x|| <= tol * ||b|| (relative to ||b||) */
  int32_t m;             /* Arnoldi steps per cycle (GMRES, rGCROT, hybrid's rGCROT phase) */
  int32_t k;             /* max recycle dimension (rGCROT, rBiCGStab, hybrid); 0 = none */
  int32_t max_matvec;    /* cap on matrix-vector products in the recurrences (<= 0: 2000) */
  int32_t hybrid_switch; /* RK_HYBRID: solves of this problem run with rGCROT before the switch */
  int32_t mode;          /* rk_mode */
  int32_t precision;     /* rk_precision: RK_FP64 = FP64 storage and arithmetic throughout (the
                            operator, the basis, U and C, the projections, orthogonalisation,
                            Gram, recycle-update products and the Schur iteration of the
                            harmonic Ritz problem); RK_MIXED = the A M^{-1} products of the
                            recurrences with an FP32 copy of the operator (FP32 accumulation),
                            everything else as in RK_FP64, b - A x recomputed in FP64 every
                            cycle / on convergence (residual replacement); RK_DF = those
                            products with a double-float copy of the operator (bands and
                            1/a_pp rounded to ~48 bits once, double-float accumulation in band
                            order) and the basis, U, C, projections and Schur iteration in
                            double-float on the FP32 pipe; residuals, x and the small least
                            squares problems in FP64 */
  int32_t update_recycle;/* rGCROT: 1 = update U, C after every cycle (Algorithm 3), 0 = keep */
  int32_t hybrid_refresh;  /* RK_HYBRID, Sec. 2.4 "intermittent solves with rGCROT": after the
                              switch, every hybrid_refresh-th solve runs rGCROT (updating U, C);
                              0 = never */
  int32_t hybrid_fallback; /* RK_HYBRID, Sec. 2.4 "switch back to rGCROT": an rBiCGStab solve that
                              breaks down or has used hybrid_fallback matrix-vector products
                              without converging is finished by rGCROT from its current iterate
                              (within max_matvec in total), and the hybrid starts a new rGCROT
                              phase: that solve and the next hybrid_switch - 1 use rGCROT;
                              0 = off */
  int32_t precond_side;  /* 0 = right preconditioning (A M^{-1}, every solver); 1 = left for GMRES
                            and rGCROT, as Sec. 2.1 states it: Arnoldi on M^{-1} A, x <- x + V y + U z,
                            recycle pair M^{-1} A U = C; the cycles stop early on their own residual
                            M^{-1}(b - A x) against a target that starts at tol ||M^{-1} b||, and the
                            solve stops on ||b - A x|| <= tol ||b|| (checked after every cycle; when
                            the target is met but the true residual is not, the target is scaled by
                            tol ||b|| / ||b - A x||). rBiCGStab is
                            always right-preconditioned (Sec. 2.1); a stored recycle space is
                            converted (C re-derived from U by CholQR2) when a solve uses the other
                            side. With RK_MIXED the left product is M32^{-1} (A32 v) (FP32 bands,
                            1/a_pp and preconditioner) */
  int32_t precond;       /* rk_preconditioner. RK_PC_SUBDOMAIN: precision RK_FP64 (the operator and
                            the preconditioner in FP64, bit-exact order), RK_DF (the products of
                            the recurrences with the double-float operator and a double-float
                            evaluation of the same preconditioner) or RK_MIXED (those products with
                            the FP32 operator and the same sweeps in FP32: bands, 1/a_pp, r and
                            omega rounded to FP32 once, every step one FP32 rounding in the FP64
                            order); residuals, M^{-1} b and the final M^{-1} x~ in FP64 in every
                            precision; GMRES, rGCROT and the hybrid's rGCROT phase
                            left-preconditioned only (precond_side = 1), rBiCGStab
                            right-preconditioned (x <- x + M^{-1} x~); otherwise RK_E_INVALID */
} rk_solve_params;

typedef struct {
  int32_t status;        /* rk_status of the solve */
  int32_t mode_used;     /* rk_mode actually run (RK_HYBRID resolves to one of the others) */
  int32_t matvecs;       /* matrix-vector products in the recurrences (b - A x excluded) */
  int32_t cycles_or_iters; /* cycles (GMRES, rGCROT) or iterations (rBiCGStab) */
  int32_t restarts;      /* rBiCGStab restarts (true-residual replacement or breakdown) */
  int32_t recycle_dim;   /* recycle dimension after the solve */
  double relres_true;    /* ||b - A x|| / ||b|| of the returned x, recomputed in FP64 */
  double relres_est;     /* last recurrence estimate (|g_{j+1}| or ||r||) / ||b|| */
  double model_bytes;    /* algorithmic HBM bytes of the solve (byte model of the library) */
} rk_solve_info;

typedef void* (*rk_alloc_fn)(size_t bytes, void* user);
typedef void (*rk_free_fn)(void* ptr, void* user);

typedef struct rk_context rk_context;
typedef struct rk_problem rk_problem;

/* Thread-local description of the last error on this thread (never NULL). */
const char* rk_last_error(void);

/* Library version string. */
const char* rk_version(void);

/*
 * Create a context on the current CUDA device. alloc/free draw device memory
 * (e.g. from a framework's caching allocator); both NULL means cudaMalloc /
 * cudaFree. `user` is passed through. *out receives the context.
 */
int rk_context_create(rk_alloc_fn alloc, rk_free_fn free_fn, void* user, rk_context** out);
/* Release the context. Problems created from it stay valid: the context's
 * memory is released when the last of them is destroyed. */
void rk_context_destroy(rk_context* ctx);

/*
 * Create a problem: the banded operator of Sec. 2.1 ("Data Layout").
 * coef: device, S*N doubles (S in {7, 19}); copied into library memory.
 * Fails with RK_E_INVALID if a band points out of a non-periodic face with a
 * nonzero coefficient or a diagonal entry is zero. stream: cudaStream_t.
 */
int rk_create_problem(rk_context* ctx, const rk_grid* grid, int32_t S, const double* coef,
                      void* stream, rk_problem** out);
void rk_problem_destroy(rk_problem* p);

/*
 * Set the recycle space (the forming of C from U in Algorithms 3 and 4).
 * U: device, N x k column-major. C: device N x k or NULL. With C == NULL the
 * library forms C~ = A U and its thin QR C~ = C R and stores
 * U R^{-1}, so that A U = C, C^T C = I. With C given it checks
 * ||A U - C||_F <= 1e-10 ||A||_F ||U||_F and ||C^T C - I||_F <= 1e-10 and
 * returns RK_E_RECYCLE_INVARIANT otherwise. k = 0 clears the space. On any
 * error the problem is left with no recycle space.
 * k must not exceed kmax (the problem's capacity, grown on demand).
 */
int rk_set_recycle(rk_problem* p, const double* U, const double* C, int32_t k, void* stream);

/*
 * Copy the recycle space out. U, C: device, N x capacity column-major (either
 * may be NULL). *k: in = capacity (columns), out = stored dimension.
 * Returns RK_E_INVALID if the capacity is smaller than the dimension.
 * The pair satisfies A U = C after rk_set_recycle and right-preconditioned
 * solves, M^{-1} A U = C after left-preconditioned GMRES / rGCROT solves
 * (precond_side = 1); both with C^T C = I.
 */
int rk_get_recycle(const rk_problem* p, double* U, double* C, int32_t* k, void* stream);

/*
 * Solve A x = b (one time step of a sequence).
 * b: device, N doubles. x: device, N doubles; in: initial guess x0, out: the
 * solution. params: host. info: host (may be NULL). The problem keeps its
 * recycle space (and, for RK_HYBRID, its solve counter) across calls, which
 * is how a sequence carries U, C from one step to the next (Sec. 2.4).
 * ||b|| = 0 returns x = 0 with RK_OK and no matrix-vector products.
 * Returns the solve status (also in info->status).
 */
int rk_solve(rk_problem* p, const double* b, double* x, const rk_solve_params* params,
             rk_solve_info* info, void* stream);

/*
 * Operator application (single products, for tests and callers that compose):
 * precond = 1: y = A (M^{-1} v); 0: y = A v; 4: y = M^{-1} (A v) (left
 * preconditioning: the product, then one rounded multiplication); 2: the FP32 operator of
 * RK_MIXED, y = A32 (M32^{-1} v) with A32, M32^{-1} the coefficients and
 * 1/a_pp rounded to FP32, v rounded to FP32, FP32 accumulation in band order,
 * the result widened to FP64; 3: the double-float operator of RK_DF,
 * y = A_df (M_df^{-1} v) with v rounded to double-float and the result
 * widened to FP64 (exact); 5: y = M^{-1} v and 6: y = M^{-1} (A v) with the
 * sub-domain preconditioner (RK_PC_SUBDOMAIN); 7 and 8: the same with the
 * double-float variant of RK_DF (v rounded to double-float, the result
 * widened to FP64); 9 and 10: y = M32^{-1} v and y = M32^{-1} (A32 v) with
 * the FP32 variant of RK_MIXED; 11: y = d32 .* (A32 v), the FP32 left
 * point-Jacobi product of RK_MIXED; for 5-11 y must not alias v. Other
 * values: RK_E_INVALID. The operator copies of modes 2, 3, 7 and 8 and the
 * workspace of modes 5-8 are made on first use (and freed by
 * rk_problem_release).
 * And r = b - A x. All vectors device, N doubles.
 */
int rk_apply(const rk_problem* p, const double* v, double* y, int32_t precond, void* stream);
int rk_residual(const rk_problem* p, const double* b, const double* x, double* r, void* stream);

/*
 * Block inner products used by the projections (the C and V projections of
 * Algorithm 3, the C projections of Algorithm 4): out[q] = Q_q^T w for the nq columns of Q
 * (device, column-major, leading dimension ld >= N), w device, out device
 * (nq doubles). The reduction order is fixed by N alone (deterministic).
 */
int rk_dots(rk_context* ctx, int64_t n, int32_t nq, const double* Q, int64_t ld, const double* w,
            double* out, void* stream);

/*
 * The fused inner products of one Arnoldi step of GMRES / rGCROT
 * (Algorithms 1 and 3: the projection of the new vector onto [C V_j] and its
 * norm, by classical Gram-Schmidt with the second pass of the previous
 * vector delayed to this step) on their own, with the kernel that solves of
 * the given precision run: out = [Q^T p (nq), Q^T w (nq), p^T p, p^T w,
 * w^T w] (2 nq + 3 doubles) for Q (N x nq, leading dimension ld >= N), p and
 * w (N doubles), all device FP64. precision RK_FP64: the FP64 kernel of the
 * RK_FP64 and RK_MIXED basis on the operands as given; RK_DF: the operands
 * first rounded to double-float, then the double-float kernel. 0 <= nq <=
 * 128, else RK_E_INVALID; RK_E_DEVICE_TIMEOUT if a bounded device wait
 * gave up. Allocates temporary device memory through the context's
 * allocator; synchronises `stream`. The reduction order is fixed by N.
 * A test entry point.
 */
int rk_arnoldi_dots(rk_context* ctx, int64_t n, int32_t nq, const double* Q, int64_t ld, const double* p,
                    const double* w, double* out, int32_t precision, void* stream);

/*
 * The row-tiled product of the recycle updates of Algorithm 3 (C <- W_hat QC,
 * U <- W PU) on its own: out = [A, diag(s) B] P with A (N x na) and B
 * (N x nb) device FP64 column-major (leading dimensions lda, ldb >= N; either
 * part may be empty), s device N doubles or NULL (identity), P device FP64
 * (na + nb) x nc column-major with leading dimension na + nb, out device
 * N x nc FP64 (leading dimension ldo >= N). For engines 0 and 1, A and B
 * are first rounded to double-float, as RK_DF solves store their basis;
 * engine = 1 runs the tensor-core kernel those solves use for
 * 2 <= nc <= 32 and na + nb <= 64
 * (7 BF16 digits per operand, exact FP32 accumulation per digit level on the
 * fifth-generation tensor cores); engine = 0 the double-float kernel on the
 * FP32 pipe; engine = 2 the FP64 fused multiply-add kernel on A and B as
 * given; engine = 3 the tensor-core kernel on A and B as given (the RK_FP64 /
 * RK_MIXED recycle update, 2 <= nc <= 32, na + nb <= 64): each FP64 row of X
 * cut exactly into a 56-bit fixed-point integer against its largest entry
 * (bits below 2^-56 of it truncated) and seven balanced base-256 digits,
 * exact digit products summed per level in FP32 on the tensor cores, the
 * levels combined exactly in integers and rounded once to FP64.
 * RK_E_INVALID for bad arguments or a shape the tensor-core
 * engine does not take; RK_E_DEVICE_TIMEOUT if a bounded device wait gave
 * up. Engines 0, 1 and 3 allocate temporary device memory through the
 * context's allocator (engine 2 allocates nothing); synchronises `stream`. No counterpart in the paper (a test entry point).
 */
int rk_row_gemm(rk_context* ctx, int64_t n, int32_t na, const double* A, int64_t lda, int32_t nb,
                const double* B, int64_t ldb, const double* s, const double* P, int32_t nc, double* out,
                int64_t ldo, int32_t engine, void* stream);

/*
 * Solve n independent problems, one right-hand side each (one time step of
 * n sequences; the batched and serving workloads of the recycling solver).
 * Equivalent to calling rk_solve(problems[i], b[i], x[i], &params[i],
 * &infos[i]) for every i, except that the solves run concurrently: a pool of
 * nthreads host threads (<= 0: min(n, 16)), each driving its own CUDA
 * stream, takes problems from a shared queue, largest N first. With the
 * environment variable RK_BATCHED_BICG=1, the rBiCGStab solves of the batch
 * (also a hybrid's after its switch) with right point Jacobi in RK_FP64 or
 * RK_MIXED instead run their iterations together, one launch per iteration
 * phase over a (problem, block) work list, on the calling thread beside the
 * pool (launch shapes tuned on first use and cached in memory and, when
 * RK_TUNE_CACHE names a file, in that JSON file); the results are the same
 * bit for bit. problems, b, x, params, infos:
 * host arrays of n entries (b[i], x[i] device pointers as in rk_solve). The
 * batch starts after the work already queued on `stream`, and work queued on
 * `stream` afterwards runs after the whole batch; the call returns when every
 * solve has finished (infos valid). A problem may appear only once per batch
 * (RK_E_INVALID otherwise); distinct problems share nothing on the device,
 * so each solve gives exactly the result it gives alone. Returns RK_OK if
 * every solve returned RK_OK, else the status of the first failing one (in
 * batch order); every infos[i].status holds its own status. The paper
 * solves one system at a time; this entry point has no counterpart there.
 */
int rk_solve_batch(rk_problem* const* problems, const double* const* b, double* const* x, int32_t n,
                   const rk_solve_params* params, rk_solve_info* infos, int32_t nthreads, void* stream);

/*
 * Device bytes currently held by a problem (operator copies, basis and
 * recycle storage, workspace), for memory budgets. No counterpart in the
 * paper.
 */
int rk_problem_memory(const rk_problem* p, int64_t* device_bytes);

/*
 * Device bytes the problem will hold during and after a solve with the
 * given parameters: rk_problem_memory plus every buffer that solve would
 * make (basis and recycle storage for capacity max(k, stored dimension) and
 * m, the small buffers, operator copies of RK_MIXED / RK_DF, the
 * preconditioner's workspace, the rBiCGStab vectors), counting the old and
 * new basis once each where a growing capacity copies the recycle space
 * over. A bound for admission under a memory budget, before a problem's
 * first solve. No counterpart in the paper.
 */
int rk_problem_footprint(const rk_problem* p, const rk_solve_params* params, int64_t* device_bytes);

/*
 * Free a problem's basis, recycle and solver workspace, keeping the operator
 * (memory pressure: a serving process evicting an idle problem). The recycle
 * space is dropped: save it first with rk_get_recycle and restore it with
 * rk_set_recycle. The next solve reallocates what it needs. Synchronises
 * `stream` first. No counterpart in the paper.
 */
int rk_problem_release(rk_problem* p, void* stream);

/*
 * Exact spill and restore of the recycle space (U and C as stored, in
 * double-float): an opaque blob of rk_recycle_bytes(p) bytes in device
 * memory (a 32-byte header, then the columns). rk_export_recycle writes it
 * into buf (cap bytes, RK_E_INVALID if smaller); rk_import_recycle makes it
 * the problem's recycle space (the problem must have the same N; RK_E_INVALID
 * otherwise). Unlike rk_get_recycle / rk_set_recycle, whose FP64 copy rounds
 * a double-float pair, the round trip is bit-exact, so a problem spilled
 * from device memory and restored continues with identical iterates.
 * Both synchronise `stream`. No counterpart in the paper.
 */
int rk_recycle_bytes(const rk_problem* p, int64_t* bytes);
int rk_export_recycle(const rk_problem* p, void* buf, int64_t cap, void* stream);
int rk_import_recycle(rk_problem* p, const void* buf, int64_t bytes, void* stream);

/*
 * Opt-in kernel timing of the solves of a problem: CUDA events on the solve's
 * stream around every launch, summed per kernel class ("spmv", "residual",
 * "dots", "update", "gemm_rows", "gram", "small", "bicg", "harmonic_ritz", "subdomain_local", "subdomain_df",
 * "subdomain32") with the class's algorithmic HBM bytes (the library's byte
 * model of each launch) and the FP64 fused multiply-adds of its launches that
 * run on the FP64 pipe (the FP64 basis kernels, the FP64 stencil and the
 * rBiCGStab vector updates; the roofline of kernels bound by that pipe).
 * rk_profile_enable resets the counters; rk_profile_read copies up to cap
 * entries to out (host) and sets *count to the number of classes.
 */
typedef struct {
  char name[16];
  int64_t launches;
  double ms;
  double bytes;
  double fma;
} rk_prof_entry;
int rk_profile_enable(rk_problem* p, int32_t on);
int rk_profile_read(rk_problem* p, rk_prof_entry* out, int32_t cap, int32_t* count);

/*
 * The small problem of Algorithm 3's recycle update on its own (the same device code
 * the solver runs after every cycle). G, F: device, (n+1) x n column-major:
 * the cycle's G = [[I, B], [0, H]] with A W = W_hat G, and
 * F = W_hat^T M W. Selects the harmonic Ritz vectors p of the k smallest
 * |theta| of G^T G p = theta G^T F p (a complex pair counts as two, and is
 * dropped whole if only one of it fits) and returns QC ((n+1) x knew, ld n+1)
 * with orthonormal columns and PU (n x knew, ld n) with G PU = QC and
 * range(PU) = span of the selected vectors; *knew (host) = their number.
 * Then C <- W_hat QC and U <- W PU keep A U = C and C^T C = I.
 * precision: RK_FP64 runs the Hessenberg reduction and the Francis
 * iteration in FP64 (as RK_FP64 and RK_MIXED solves do), RK_DF in
 * double-float on the FP32 pipe (as RK_DF solves do); other values:
 * RK_E_INVALID. The QR of G and everything after the Schur form are FP64.
 * Returns RK_E_BREAKDOWN if the eigen-iteration fails to converge.
 */
int rk_harmonic_ritz(rk_context* ctx, int32_t n, const double* G, const double* F, int32_t k, double* QC,
                     double* PU, int32_t* knew, int32_t precision, void* stream);

/*
 * rk_dots without any device allocation. The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory once
 * they are running — for instance a serving process that reserves its whole
 * memory budget at start-up, or an application whose memory manager forbids
 * cudaMalloc on its critical path (cudaMalloc can synchronise the device and
 * fragment a pool). rk_dots itself draws its reduction scratch from the
 * context's allocator; this variant uses a fixed scratch array compiled into
 * the library instead (304 KiB of per-block partial sums plus a counter, in
 * static device memory that every GPU loading the library holds until the
 * process exits), and calls no cudaMalloc, cudaFree or allocating routine.
 *
 * Same arguments and results as rk_dots (out[q] = Q_q^T w, q < nq, in the
 * same fixed reduction order, so the two agree bit for bit; nq = 0 does
 * nothing, as there), without a context. Limit: nq <= 64 columns (larger nq
 * returns RK_E_INVALID with a message); any n. Like every entry point, the
 * call returns after its work on `stream` has completed (it synchronises
 * that stream). The first call on a device looks up the scratch array's
 * device address (cudaGetSymbolAddress) and clears its counter, which
 * synchronises that device: make the first call on each device before any
 * stream capture. All calls share the one scratch array, whose contents
 * persist from call to call: calls whose kernels overlap on a GPU (other
 * threads or streams) race on it and must be serialised by the caller.
 */
int rk_dots_noalloc(int64_t n, int32_t nq, const double* Q, int64_t ld, const double* w, double* out,
                    void* stream);

/* Number of solves run on this problem (the hybrid's step counter) and its
 * recycle dimension. */
int rk_problem_stats(const rk_problem* p, int32_t* solves, int32_t* recycle_dim, int64_t* n);

/*
 * Start a new time-step sequence on the same operator: the recycle space is
 * dropped (as rk_set_recycle with k = 0) and RK_HYBRID's solve counter
 * restarts, so the next solve is solve 0 of a new rGCROT phase (Sec. 2.4).
 * Buffers, operator copies and captured cycles are kept. Returns RK_E_INVALID
 * for a NULL problem. No counterpart in the paper (its runs are one sequence).
 */
int rk_problem_reset(rk_problem* p);

/*
 * Test hook for the failure path of the bounded device waits: with
 * polls > 0, the bulk-copy producer of the double-float Arnoldi inner
 * products (RK_DF solves) gives up after that many polls of a stage-release
 * barrier, issues no further copies, lets the consumers stop at the first
 * stage it did not issue (so no copy into shared memory is in flight when
 * the block exits) and flags the failure; the solve then returns
 * RK_E_DEVICE_TIMEOUT and the problem stays usable. polls = 0 restores the
 * default limit (2^22 polls). Synchronises `stream`. No counterpart in the
 * paper.
 */
int rk_problem_wait_limit(rk_problem* p, int32_t polls, void* stream);

/*
 * Measure this GPU's FP64 fma issue rate (lane operations per second, one
 * fma = 2 flops): 608 blocks of 256 threads, 8 independent fma chains of
 * 4096 steps per thread, best of three timed launches (CUDA events on
 * `stream`) after one warm-up launch. The denominator of the rooflines of
 * kernels bound by the FP64 pipe. No counterpart in the paper.
 */
int rk_fp64_fma_rate(double* fma_per_s, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RK_H */
