/*
 * ie.h -- C ABI of the GB300 interior eigensolver built on the composite-rule
 * rational filter of Chen & Li, "Interior Eigensolver Based on Rational Filter
 * with Composite Rule" (arXiv 2310.18043).
 *
 * Problem (Sec. 1, Eq. problem): all eigenpairs A x = lambda B x with lambda in
 * the disk D = { |z - center| < radius } of a sparse non-Hermitian pencil (A, B).
 * Filter (Sec. 3.1-3.2, Thm 2): U = R_{c,r,p*q}(B^{-1}A) Y, applied as
 *   inner:  G(V) = sum_{i<=q} w_i K_i^{-1} B V,  K_i = p_i B - A   (Eq. linearsolve2)
 *   outer:  U = sum_{j} c_j (s_j I - G)^{-1} G Y (+ (1/p) G Y, p odd) (Eq. linearsolve1abs)
 * with the q inner factorisations done once (band LU, partial pivoting) and the
 * p outer shifts solved together by multi-shift GMRES (one Krylov space per column).
 *
 * Conventions
 *  - Complex numbers are ie_complex = {double re, im}, layout-identical to C99
 *    double _Complex, CUDA double2 and numpy complex128.
 *  - Blocks (Y, U, X, ...) are column-major n x k with leading dimension ld >= n.
 *  - Pointers named d_* must be device pointers on the handle's device.
 *    Pointers named *_any may be device or host memory (pageable or pinned);
 *    host buffers are staged through the handle's device workspace on the
 *    call's stream. Pointers named h_* must be host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Every function returns an ie_status; nothing is thrown across the ABI.
 *    After IE_ERR_CUDA the handle should be destroyed.
 *  - Calls on one handle must not overlap (the handle owns one workspace).
 */
#ifndef IE_H_
#define IE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } ie_complex;

typedef struct ie_handle_s* ie_handle;   /* opaque, owned by the library */

typedef enum {
  IE_OK = 0,
  IE_ERR_ARG = 1,        /* invalid argument (sizes, NULL pointers, options) */
  IE_ERR_CUDA = 2,       /* a CUDA runtime call or kernel failed */
  IE_ERR_OOM = 3,        /* device allocation failed */
  IE_ERR_SINGULAR = 4,   /* an LU pivot was exactly zero: a pole hit an eigenvalue (Prop. 1 case) */
  IE_ERR_NOCONV = 5,     /* GMRES reached m_max or the driver reached max_outer; outputs still written */
  IE_ERR_BREAKDOWN = 6,  /* reserved: orthogonalisation could not extend a basis */
  IE_ERR_TIMEOUT = 7,    /* a device-side bounded wait gave up (kernel returned early) */
  IE_ERR_SCRATCH_LIMIT = 8 /* ie_apply_G_static: problem larger than its static scratch */
} ie_status;

/* Sparse pencil in DIA form: M[i, i + offsets[d]] = dia[d * n + i] (entries with
 * i + offsets[d] outside [0, n) are ignored). A and B share the offsets.
 * Sec. 1 Eq. (problem). d_A_dia, d_B_dia: device, ndiag * n complex128, read
 * during ie_create and copied (the caller may free them afterwards).
 * h_offsets: host, ndiag entries, |offset| < n. ndiag <= 16. */
typedef struct {
  int64_t n;
  int32_t ndiag;
  const int64_t* h_offsets;
  const ie_complex* d_A_dia;
  const ie_complex* d_B_dia;
} ie_pencil;

/* Solver options (Alg. 1 / Alg. 2 REQUIRE lines; Sec. 6 preamble for defaults). */
typedef struct {
  int32_t k;              /* block width n_col (max columns per filter call), >= 1 */
  int32_t driver;         /* 1 = Alg. 1 (fixed p, subspace iteration); 2 = Alg. 2 (p doubled) */
  int32_t m_max;          /* max GMRES (Arnoldi) steps per column per filter application */
  int32_t max_outer;      /* max outer iterations of the driver */
  double tau_g;           /* ghost tolerance on e_i (Sec. 3.2), default 1e-2 */
  double tau;             /* convergence tolerance on rho_i, default 1e-10 */
  double gmres_tol;       /* per-shift relative GMRES residual, default 1e-12 */
  int32_t sigma_is_center;/* 1: HSRR shift sigma = center (Sec. 6 preamble); 0: use sigma_re/im */
  double sigma_re, sigma_im;
  uint64_t seed;          /* seeds rank-guard replacement vectors and the random Y0 */
  int32_t precision;      /* 0: complex128 band LU and solves. 1: mixed precision -- K_i is
                             assembled in complex64 and factored by the band LU in FP32
                             arithmetic, the triangular solves run in FP32, and each
                             K_i^{-1} b is refined in FP64: x += K~_i^{-1} (b - K_i x) */
  int32_t refine_steps;   /* precision = 1: at most this many FP64 refinement steps per solve
                             (default 8). The steps stop earlier once the measured correction
                             shows the accuracy the call needs is reached (the FP64 floor for
                             ie_apply_G and the first G(Y) of a filter; a relaxed accuracy in
                             the later GMRES steps) or once corrections stop shrinking. */
  int32_t adjoint;        /* 1: also prepare the conjugate-transpose solves K_i^{-H} with the same
                             factors (ie_apply_GH, ie_solve_left): the adjoint pencil in DIA
                             form, a row-major copy of each U factor (q * n * 2*kl entries,
                             complex128 or complex64 as the factors) and a 16 x 24 transform
                             per 8-row panel and pole. Default 0. Not in the paper. */
} ie_opts;

/* Fills defaults: k=16, driver=1, m_max=100, max_outer=10, tau_g=1e-2, tau=1e-10,
 * gmres_tol=1e-12, sigma = center, seed = 0, precision = 0, refine_steps = 8, adjoint = 0. */
void ie_opts_default(ie_opts* opts);

/* Counters and timings of the last ie_solve / ie_filter_apply on a handle. */
typedef struct {
  int32_t outer_iters;     /* outer iterations performed (ie_solve) */
  int32_t n_found;         /* filtered pairs: in D and e_i < tau_g (Sec. 3.2) */
  int32_t p_final;         /* outer order used by the last filter (Alg. 2 doubles it) */
  int32_t gmres_iters_max; /* max Arnoldi steps over the columns, last filter */
  int32_t gmres_iters_min;
  int32_t converged;       /* 1 if the stop test was met */
  int64_t g_columns;       /* columns G was applied to since create; solves = q * this */
  double t_factor_ms;      /* ie_create: assembly + batched band LU */
  double t_filter_ms;      /* total filter time of the last ie_solve (or the last filter call) */
  double t_hsrr_ms;        /* total HSRR time of the last ie_solve */
  double max_rho_found;    /* max rho_i over the filtered pairs */
  int64_t solve_launches;  /* band-solve kernel launches since create */
  double t_solve_ms;       /* their summed device time (CUDA events on the launch stream) */
  double solve_flops;      /* their algorithmic flops: q*k*(8 (n kl + n kv - band corners) + 12 n) */
  double solve_bytes;      /* their algorithmic DRAM bytes (factors once per launch, RHS, y, x) */
  int64_t kernel_launches; /* CUDA kernels launched by this library in this process so far */
  int64_t solve32_launches;/* complex64 band-solve launches (precision = 1) since create */
  double t_solve32_ms;     /* their summed device time */
  double solve32_flops;    /* their algorithmic flops (same count as solve_flops, in FP32) */
  int64_t adj_launches;    /* conjugate-transpose band-solve launches since create (either precision) */
  double t_adj_ms;         /* their summed device time */
  double adj_flops;        /* their algorithmic flops (same count per launch as the forward solve) */
  int64_t refine_solves;   /* precision = 1: FP32 refinement solves (each: q poles x the block) since create */
  double refine_last_corr; /* precision = 1: the last refinement step's largest relative correction
                              max |dx|_inf / |x|_inf over poles and columns (an error estimate) */
  int32_t solve_kernel;    /* band-solve kernel of the last complex128 solve launched in this
                              process: 0 barrier-synchronised, 1 warp-specialised, 2 look-ahead
                              (the launch-shape tuner's choice); -1 none yet */
  int32_t solve32_kernel;  /* the same for the complex64 solves */
} ie_stats;

/* ie_create: computes the inner poles/weights (Eq. pwtp, q points) and the outer
 * shifts/weights (Thm 2, p roots of z^p = -1), assembles K_i = p_i B - A for all
 * q poles into LAPACK band storage (kl = ku = max|offset|, ldab = 3*kl + 1) and
 * factors all of them with partial pivoting in one cooperative launch
 * (set-up steps of Alg. 1). Requires p >= 1, q >= 1, radius > 0, 1 <= opts->k <= n.
 * Returns IE_ERR_SINGULAR if a pivot is exactly zero (the handle is still
 * created and must be destroyed). Synchronises the stream before returning. */
ie_status ie_create(const ie_pencil* pencil, ie_complex center, double radius,
                    int32_t p, int32_t q, const ie_opts* opts, void* stream,
                    ie_handle* out);

ie_status ie_destroy(ie_handle h);

const char* ie_status_str(ie_status s);

/* ie_filter_apply: U = R_{c,r,p*q}(B^{-1}A) Y by the composite rule (Alg. 1 lines
 * 7-9): Ytilde = G(Y); per column multi-shift GMRES from x0 = 0 for all p outer
 * shifts until every shift's relative residual <= gmres_tol (or m_max);
 * U = sum_j c_j (s_j I - G)^{-1} Ytilde (+ (1/p) Ytilde for odd p).
 * Y_any, U_any: n x k, k <= opts.k, ld >= n, device or host. Synchronises the
 * stream (the GMRES loop tests convergence on the host after each step).
 * Returns IE_ERR_NOCONV if a column reached m_max (U is still written). */
ie_status ie_filter_apply(ie_handle h, const ie_complex* Y_any, int64_t ldy, int32_t k,
                          ie_complex* U_any, int64_t ldu, void* stream);

/* ie_apply_G: the inner operator alone, GV = G(V) = sum_i w_i K_i^{-1} B V
 * (Eq. linearsolve2; Alg. 1). V_any, GV_any: n x k (k <= opts.k). */
ie_status ie_apply_G(ie_handle h, const ie_complex* V_any, int64_t ldv, int32_t k,
                     ie_complex* GV_any, int64_t ldgv, void* stream);

/* ie_hsrr: the harmonic Rayleigh-Ritz step HSRR(A, B, U, sigma) (Sec. 2.1,
 * extraction steps of Alg. SIsketch): V = orth(U) (CGS2 with rank guard), W = orth(AV - sigma BV),
 * QZ of (W^*AV, W^*BV), lambda_i = (H_A)_ii/(H_B)_ii, x_i = V P_R V_R(:,i) scaled
 * to unit norm; e_i (Eq. rel-error) and rho_i = ||Ax - lambda Bx|| /
 * ((||A||_1 + |lambda| ||B||_1) ||x||). Outputs in QZ order (no sorting):
 * h_lambda, h_e, h_rho host arrays of k entries (infinite Ritz values are
 * returned as +inf); X_any n x k. Synchronises the stream. */
ie_status ie_hsrr(ie_handle h, const ie_complex* U_any, int64_t ldu, int32_t k,
                  ie_complex* h_lambda, ie_complex* X_any, int64_t ldx,
                  double* h_e, double* h_rho, void* stream);

/* ie_solve: all eigenpairs in D by Alg. 1 (opts.driver = 1) or Alg. 2 (= 2).
 * Y0_any: n x opts.k starting block (orthonormal), or NULL for a seeded random
 * orthonormal block. Outputs, ordered filtered pairs first (each group by
 * |lambda - center| ascending): h_lambda (k, host), X_any (n x k, ldx),
 * h_rho (k, host, nullable), h_e (k, host, nullable); *n_found = number of
 * filtered pairs (Ritz value in D and e_i < tau_g). stats nullable.
 * Returns IE_ERR_NOCONV if max_outer was reached without meeting the stop test. */
ie_status ie_solve(ie_handle h, const ie_complex* Y0_any, int64_t ldy0,
                   ie_complex* h_lambda, ie_complex* X_any, int64_t ldx,
                   double* h_rho, double* h_e, int32_t* n_found, ie_stats* stats,
                   void* stream);

/* ie_spmv: Y = M X with M = A (which = 0) or B (which = 1), n x k blocks
 * (the sparse products of Eq. linearsolve2 and of HSRR). */
ie_status ie_spmv(ie_handle h, int32_t which, const ie_complex* X_any, int64_t ldx, int32_t k,
                  ie_complex* Y_any, int64_t ldy, void* stream);

/* ie_get_coeffs: copies the coefficients to host arrays (any may be NULL):
 * h_poles, h_weights: q inner poles p_i and weights w_i (Eq. pwtp);
 * h_shifts, h_cweights: the n_shift outer shifts s_j and weights c_j (Thm 2;
 * for odd p the sigma = -1 root is left out, n_shift = p - p%2); *odd_coef = 1/p
 * for odd p else 0. Arrays must hold q and p entries. */
ie_status ie_get_coeffs(ie_handle h, ie_complex* h_poles, ie_complex* h_weights,
                        ie_complex* h_shifts, ie_complex* h_cweights, int32_t* n_shift,
                        double* odd_coef);

/* ie_get_factor: copies pole i's band LU (LAPACK zgbtrf layout: column j holds rows j-kv..j+kl
 * at offsets 0..ldab-1 with kv = 2*kl, ldab = 3*kl + 1; U in rows 0..kv, the multipliers of L
 * below) and its 1-based pivot vector (LAPACK ipiv convention) into host arrays h_ab
 * (ldab * n) and h_ipiv (n). *kl, *ldab set. For precision = 1 handles the factors are the
 * complex64 ones (LAPACK cgbtrf semantics, FP32 arithmetic), widened exactly to complex128.
 * Either array may be NULL. */
ie_status ie_get_factor(ie_handle h, int32_t pole, ie_complex* h_ab, int32_t* h_ipiv,
                        int32_t* kl, int32_t* ldab);

/* ie_get_stats: counters of the last call (see ie_stats). */
ie_status ie_get_stats(ie_handle h, ie_stats* out);

/* ie_apply_G_static: the same G(V) as ie_apply_G (same kernels, same results), for callers
 * that must not make the library allocate device memory at call time: a host application
 * whose own allocator owns the device memory budget, or a latency-critical loop that cannot
 * afford the implicit device synchronisation of cudaMalloc/cudaFree. The paper has no
 * counterpart; this is a deployment variant of the inner-operator application.
 * It calls no cudaMalloc, cudaFree or allocating library routine. Its scratch (the B V block
 * and the q per-pole solve buffers) lives in one file-scope device array of
 * IE_STATIC_SCRATCH_BYTES bytes, which every GPU that loads the library keeps until the
 * process exits. Limit: (q + 1) * n * k * 16 <= IE_STATIC_SCRATCH_BYTES, else
 * IE_ERR_SCRATCH_LIMIT (nothing is launched). k may exceed opts.k within that limit.
 * Complex128 handles only (precision = 0; IE_ERR_ARG otherwise). d_V, d_GV: device (or
 * managed) memory of the handle's GPU, n x k, ld >= n; the current device must be the
 * handle's (IE_ERR_ARG otherwise). The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) once for that device; under CUDA's lazy module loading
 * that first call also loads the module that holds the array, which is when the device
 * reserves its IE_STATIC_SCRATCH_BYTES. Make that first call before any stream capture.
 * Every call synchronises its stream before returning (it reads the kernels' status word).
 * All calls in the process share the one array: calls whose work overlaps on the GPU
 * (different streams or threads, any handles) race on it and must be serialised by the
 * caller. Every scratch element a call reads is first written by the same call, so nothing
 * needs clearing between calls. */
#define IE_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
ie_status ie_apply_G_static(ie_handle h, const ie_complex* d_V, int64_t ldv, int32_t k,
                            ie_complex* d_GV, int64_t ldgv, void* stream);

/* ---------------------------------------------------------------------------------------
 * Adjoint pencil, left eigenvectors and eigenvalue sensitivities. The paper computes right
 * eigenpairs only; these entry points carry its method over to the adjoint pencil.
 * A left eigenvector y of (A, B) for lambda (y^H A = lambda y^H B) is a right eigenvector of
 * (A^H, B^H) for conj(lambda). The trapezoidal nodes and weights of the conjugate disk are
 * the conjugates of p_i, w_i (Eq. pwtp; the angles (2i-1) pi / q are closed under negation),
 * and conj(p_i) B^H - A^H = K_i^H, so the adjoint pencil's inner operator reuses the band
 * factors of K_i = P_i^T L_i U_i through K_i^{-H} = P_i^T L_i^{-H} U_i^{-H}.
 * ie_apply_GH and ie_solve_left need a handle created with opts.adjoint = 1 (else
 * IE_ERR_ARG); ie_eig_sensitivity works on any handle. */

/* ie_apply_GH: GV = G_adj(V) = sum_i conj(w_i) K_i^{-H} B^H V, the inner operator
 * (Eq. linearsolve2) of (A^H, B^H) on the disk |z - conj(center)| < radius.
 * V_any, GV_any: n x k (k <= opts.k), column-major. Mixed-precision handles refine each
 * K_i^{-H} b in FP64 like ie_apply_G. */
ie_status ie_apply_GH(ie_handle h, const ie_complex* V_any, int64_t ldv, int32_t k,
                      ie_complex* GV_any, int64_t ldgv, void* stream);

/* ie_solve_left: left eigenvectors for the nl eigenvalues h_lambda[0..nl) of (A, B)
 * (typically the first n_found outputs of ie_solve; 1 <= nl <= opts.k). Runs the handle's
 * driver (opts.driver, same options) on (A^H, B^H) over the conjugate disk, then pairs each
 * requested eigenvalue with the nearest conjugated adjoint eigenvalue (one-to-one).
 * Outputs: Y_any column i (unit 2-norm) is the left vector of h_lambda[i];
 * h_lambda_left[i] (host, nullable) the paired adjoint eigenvalue conjugated back;
 * h_rho_left[i] (host, nullable) its residual rho for (A^H, B^H) (Sec. 3.2 definition).
 * Y0_any: n x opts.k starting block or NULL (seeded random). stats: nullable.
 * Returns IE_ERR_NOCONV if the adjoint driver missed its stop test, or if a requested
 * eigenvalue has no partner within 1e-8 * max(|lambda|, radius) or two requests share one
 * (all outputs are still written). */
ie_status ie_solve_left(ie_handle h, const ie_complex* h_lambda, int32_t nl,
                        const ie_complex* Y0_any, int64_t ldy0, ie_complex* Y_any, int64_t ldy,
                        ie_complex* h_lambda_left, double* h_rho_left, ie_stats* stats,
                        void* stream);

/* ie_eig_sensitivity: first-order sensitivities of nf simple eigenvalues to the diagonal of
 * A, from right vectors X and left vectors Y (column i of each belongs to eigenvalue i):
 *   S[j, i] = d lambda_i / d t_j = alpha * conj(Y[j, i]) * X[j, i] / (Y[:, i]^H B X[:, i])
 * for A_jj(t) = A_jj + alpha t_j (alpha = i for a parameter entering as + i gamma_j), and
 * the vector-Jacobian product of a real loss J(lambda) with h_gbar[i] = dJ/dRe lambda_i +
 * i dJ/dIm lambda_i:  grad[j] = Re sum_i conj(gbar_i) S[j, i].
 * X_any, Y_any: n x nf (1 <= nf <= opts.k). S_any: n x nf (lds >= n) or NULL.
 * h_gbar: host, nf entries, or NULL (then grad_any must be NULL). grad_any: n doubles or NULL.
 * S and grad do not depend on the scaling of X or Y. */
ie_status ie_eig_sensitivity(ie_handle h, const ie_complex* X_any, int64_t ldx,
                             const ie_complex* Y_any, int64_t ldy, int32_t nf, ie_complex alpha,
                             ie_complex* S_any, int64_t lds, const ie_complex* h_gbar,
                             double* grad_any, void* stream);

/* ---------------------------------------------------------------------------------------
 * Batched solves: many independent problems (pencils, or disks of one pencil) at once. The
 * paper notes that disks are independent problems (Sec. 1); small problems leave most of the
 * GPU idle during their sequential Arnoldi steps and host-side tests, so running their drivers
 * concurrently fills it. */
typedef struct {
  ie_handle h;                 /* the problem; every item needs its own handle */
  const ie_complex* Y0_any;    /* n x opts.k starting block, or NULL (seeded random) */
  int64_t ldy0;
  ie_complex* h_lambda;        /* out: opts.k eigenvalues (host), ordered as by ie_solve */
  ie_complex* X_any;           /* out: n x opts.k eigenvectors, leading dimension ldx */
  int64_t ldx;
  double* h_rho;               /* out, nullable: opts.k residuals rho (host) */
  double* h_e;                 /* out, nullable: opts.k errors e (host) */
  void* stream;                /* stream for this item's work; NULL: the library makes a
                                  non-blocking stream for the call and destroys it after */
  int32_t n_found;             /* out */
  int32_t status;              /* out: the item's ie_status */
  ie_stats stats;              /* out */
} ie_batch_item;

/* ie_solve_batch: ie_solve for nb items concurrently. max_workers host threads (0: min(nb, 16))
 * each take the next item, make its handle's device current and run the item's driver
 * (opts.driver of its handle) on the item's stream. Every item's outputs equal those of
 * ie_solve on its handle alone. Returns IE_ERR_ARG for nb < 1, a NULL item field that ie_solve
 * requires, or two items sharing a handle (nothing runs); otherwise IE_OK if every item
 * returned IE_OK, else the first non-OK item status in item order (all items still run).
 * Not in the paper. */
ie_status ie_solve_batch(ie_batch_item* items, int32_t nb, int32_t max_workers);

/* ie_solve_batch_fused: the same results as ie_solve_batch, with every item's driver advancing
 * in lockstep on one stream. Each Arnoldi step applies G (Eq. linearsolve2) to the active
 * columns of every item with one band-solve launch per factor precision for all items
 * together (a problem table on the device: each CTA serves one (item, pole, column group)),
 * then each item's Krylov kernels run, and one stream synchronisation serves every item's
 * convergence test. Mixed-precision items refine in lockstep, each to its own accuracy. An
 * item whose filter is complete runs its HSRR and stop test (Sec. 3.2) and either finishes or
 * starts its next outer iteration (Alg. 1 or Alg. 2, opts.driver of its handle) while the
 * others keep stepping. Every handle must be on the current device; items[i].stream is
 * ignored (stream is used for all). Returns IE_ERR_ARG for nb < 1, a NULL item field that
 * ie_solve requires, two items sharing a handle or a handle on another device (nothing runs);
 * otherwise IE_OK if every item returned IE_OK, else the first non-OK item status in item
 * order. Each item's stats carry its counters (outer iterations, n_found, GMRES steps, solve
 * and refinement counts); its per-phase times (t_filter_ms, t_hsrr_ms) are not measured and
 * read 0, since the phases of all items interleave. Not in the paper (the paper notes disks
 * are independent problems, Sec. 1). */
ie_status ie_solve_batch_fused(ie_batch_item* items, int32_t nb, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* IE_H_ */
