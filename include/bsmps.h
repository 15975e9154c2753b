/*
 * bsmps.h -- C ABI of the GB300 block-sparse MPS eigensolver.
 *
 * The library implements, on one CUDA device, the operations of the low-rank
 * preconditioned inverse iteration for particle-number-conserving matrix
 * product states ("Low-Rank Eigenvalue Solvers for Block-Sparse Matrix
 * Product States"): Hamiltonian MPO construction, MPO x MPS application,
 * block-sparse rank truncation, the exponential-sum preconditioner, inner
 * products and the error-controlled PINVIT step (Alg. 2).
 *
 * Conventions used by every call
 * ------------------------------
 * Sites t = 0..K-1 (the paper numbers them 1..K); bonds b = 0..K, bond b
 * separates sites < b from sites >= b.  With spin = 0 the K = n_orb sites
 * are spinless orbitals (species 0).  With spin = 1 spatial orbital p owns the
 * two sites 2p (species 0, "up") and 2p+1 (species 1, "down"), K = 2 n_orb.
 * Occupying a site adds one particle of its species.  A sector at bond b is the
 * pair (n0, n1) of particles on sites < b; valid sectors are those that can be
 * completed to the target (n_up, n_dn) (Sec. 2.3, the sets K_k).  Sectors of a
 * bond are sorted ascending by (n0, n1).
 *
 * Block layout ("flat layout") of an MPS: sites ascending; within a site the
 * left sectors ascending, then sigma = 0 (unoccupied block, n -> n) and sigma = 1
 * (occupied block, n -> n + e_species); each existing block is a dense
 * rho_left x rho_right matrix stored row-major in float64 (Eq. (blockstructure)).
 *
 * Ownership: the library owns all device memory behind handles.  Host arrays
 * passed in are read during the call only; host arrays passed out are written
 * during the call and owned by the caller.  Every handle returned through an
 * out-pointer is new and is released by the matching *_destroy call.
 *
 * Errors: every call returns a bsmps_status; no call aborts or throws across
 * the ABI.  On failure the out-handles are left untouched and
 * bsmps_last_error(ctx) describes the failure.  CUDA errors map to
 * BSMPS_ERR_CUDA; a device that cannot satisfy an allocation gives
 * BSMPS_ERR_OOM.
 *
 * Streams: all device work of a context is ordered on the stream given to
 * bsmps_ctx_create (NULL: the legacy default stream).  Calls that return host
 * scalars synchronise that stream before returning.
 *
 * Names: every symbol carries the bsmps_ prefix (a plain "truncate" would
 * interpose the POSIX truncate(2) of the C library).
 */
#ifndef BSMPS_H
#define BSMPS_H

#include <stdint.h>

#if defined(__GNUC__)
#define BSMPS_API __attribute__((visibility("default")))
#else
#define BSMPS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bsmps_ctx_s* bsmps_ctx;
typedef struct bsmps_mps_s* bsmps_mps;
typedef struct bsmps_mpo_s* bsmps_mpo;
typedef struct bsmps_mlp_s* bsmps_mlp;
typedef struct bsmps_plan_s* bsmps_plan;

typedef enum {
    BSMPS_OK = 0,
    BSMPS_ERR_INVALID_ARG = 1, /* null handle, negative size, inconsistent arrays */
    BSMPS_ERR_CHARGE = 2,      /* particle numbers / sectors not realisable */
    BSMPS_ERR_OOM = 3,         /* device allocation failed */
    BSMPS_ERR_RANK_CAP = 4,    /* result would exceed a hard capacity */
    BSMPS_ERR_NOT_SPD = 5,     /* preconditioner data violates t_min > 0 */
    BSMPS_ERR_NUMERIC = 6,     /* NaN / Inf detected in a scalar of the step */
    BSMPS_ERR_TIMEOUT = 7,     /* a bounded device wait gave up */
    BSMPS_ERR_CUDA = 8         /* any other CUDA runtime error */
} bsmps_status;

/* Arithmetic of the contraction stage of the zip-up MPO application. */
typedef enum {
    BSMPS_PREC_FP64 = 0,   /* FP64 grouped GEMM on the FP64 units */
    BSMPS_PREC_TF32X3 = 1  /* split precision on the tensor cores: operands split into two TF32
                              parts, three products accumulated in FP32 (relative error of an entry
                              a few 2^-21 of sum_k |a_ik||b_kj|); results stored in FP64 */
} bsmps_precision;

/* Exponential-sum preconditioner data (Sec. 4.2-4.3, Cor. lrprecond).
 * d: the K diagonal coefficients d_i of D = sum_i d_i a_i^* a_i (theta_i of
 * Sec. 7.1.1), host array of length K, read during the calls that take it.
 * [t_min, t_max] must contain the spectrum of D on the sector (t_min > 0).
 * c0 in (0,1) sets h, M^-, M^+ by Eq. (expsumparams); alpha0 is the scaling of
 * Eq. (Sdef).  The library forms S = sum_m S_m with
 * S_m = (x)_i diag(alpha_m^{1/K}, alpha_m^{1/K} exp(-beta_m d_i)),
 * alpha_m = h alpha0 / sqrt(pi) e^{mh/2}, beta_m = e^{mh} / t_min. */
typedef struct {
    int K;
    const double* d;
    double t_min;
    double t_max;
    double c0;
    double alpha0;
} bsmps_precond;

/* Constants of Alg. 2: c (Eq. (specequivA)), delta >= lambda_2/(lambda_2 -
 * lambda_1) (Sec. 5.4), eps_num in (0, 1-c) (Lemma truncr; Sec. 7.1.3 uses
 * (1-c)/2), t_eig in (0,1) (Thm. conv (ii)), tau the eigenvector tolerance of
 * the termination test (Thm. aposterbound).  r_max > 0 caps the ranks of the
 * truncated iterate x^{n+1} (0: no cap).  u_rel: each exactly applied term
 * u_k' = (H_gamma - lambda) S_k' x is compressed once by trunc at
 * u_rel ||u_k'|| before the residual sum (1e-13 keeps the terms exact to
 * working precision; 0 disables). */
typedef struct {
    double c;
    double delta;
    double eps_num;
    double t_eig;
    double tau;
    int r_max;
    double u_rel;
} bsmps_solver_params;

/* State carried between steps: eta_res of the previous step (start with
 * +INFINITY as in Alg. 2), the step counter n, and the number of eta_res passes
 * beyond the first that the previous step needed (start with 0).  The last
 * field only sizes the next step's first batch of candidate tolerances: the
 * passes of the eta_res loop are evaluated several at a time (their truncations
 * share launches), which changes no result.  The last two fields drive the
 * split-precision policy of bsmps_ctx_set_precision (start with 0, 0): the
 * previous step's sum of residual-term norms sum_j ||s_j|| (Sec. 5.3.1), and
 * 1 once the iteration has fallen back to FP64 contractions. */
typedef struct {
    double eta_res;
    int n;
    int last_tries;
    double last_sum_norms;
    int fp64_locked;
} bsmps_solver_state;

/* Scalars reported by one step. */
typedef struct {
    double lambda;        /* lambda(x^n), Eq. (exactrq) */
    double rho;           /* rho^n, Eq. (rhobound) */
    double eta_res;       /* accepted residual tolerance */
    double res_norm;      /* ||res_eta(x^n)|| */
    int eta_tries;        /* passes of the eta_res loop beyond the first */
    double bound;         /* eigenvector bound of Thm. aposterbound (+inf if invalid) */
    double releig_bound;  /* relative eigenvalue bound, Eq. (releigerr) (+inf if invalid) */
    double lambda_star;   /* lower Ritz value of the 2x2 problem (Remark omegamin) */
    double omega;         /* step size: x* is proportional to x - omega r */
    double eta_in;        /* truncation tolerance of the iterate (Sec. 5.3.2) */
    double delta_A;
    int converged;        /* 1 when the termination test of Alg. 2 held */
    int max_rank;         /* largest bond dimension of the returned iterate */
    double flops;         /* algorithmic FP64 flops issued by the step */
    double cap_discarded; /* norm discarded by the r_max cap of the iterate */
    int precision;        /* arithmetic of the step's apply contraction (bsmps_precision) */
} bsmps_step_info;

BSMPS_API const char* bsmps_status_string(bsmps_status s);

/* ---- context ---------------------------------------------------------- */

/* Create a context on CUDA device `device` ordering its work on `stream`
 * (a cudaStream_t, or NULL).  Errors: INVALID_ARG (out NULL), CUDA. */
BSMPS_API bsmps_status bsmps_ctx_create(int device, void* stream, bsmps_ctx* out);
BSMPS_API bsmps_status bsmps_ctx_destroy(bsmps_ctx ctx);
/* Wait for all work of the context. */
BSMPS_API bsmps_status bsmps_ctx_sync(bsmps_ctx ctx);
/* Message of the last failed call on this context ("" if none). */
BSMPS_API const char* bsmps_last_error(bsmps_ctx ctx);
/* Number of kernel launches issued by the context so far. */
BSMPS_API int64_t bsmps_ctx_launch_count(bsmps_ctx ctx);
/* Number of device-memory requests the context's allocator has served so far
 * (from its cache or from the stream-ordered pool). */
BSMPS_API int64_t bsmps_ctx_alloc_count(bsmps_ctx ctx);

/* Kernel profiler.  enable != 0 brackets every launch with CUDA events on the
 * context stream and records its kind and algorithmic flops / bytes (this
 * adds two event records per launch); enable = 0 stops recording.
 * bsmps_ctx_kernel_stats synchronises the stream and returns, for kernel kind
 * `kind` (0 copy, 1 grouped GEMM, 2 QR, 3 SVD, 4 sum of squares, 5 the
 * contraction stage of the zip-up MPO application, 6 the zip-up's own
 * factorisation launches: zeroing, gathers, QR; 7 the tensor-core products
 * of the learned controller's network, FP32 flops), the number
 * of recorded launches, their summed device time in ms and summed
 * algorithmic FP64 flops and bytes; `reset` != 0 clears the records after
 * reading.  Errors: INVALID_ARG (kind out of range), CUDA. */
BSMPS_API bsmps_status bsmps_ctx_profile(bsmps_ctx ctx, int enable);
BSMPS_API bsmps_status bsmps_ctx_kernel_stats(bsmps_ctx ctx, int kind, int reset, int64_t* launches,
                                              double* ms, double* flops, double* bytes);

/* Diagnostic of the bounded grid-wide waits used by the persistent sweep
 * kernels (no counterpart in the paper).  Launches a two-CTA cooperative
 * kernel whose CTAs meet at one grid-wide phase boundary.  skip_cta < 0: both
 * arrive, *timed_out = 0.  skip_cta = 0 or 1: that CTA returns without
 * arriving, the other one gives up after the wait limit (about 1 s), and
 * *timed_out = 1; the context stays usable.  Errors: INVALID_ARG (skip_cta >
 * 1), CUDA. */
BSMPS_API bsmps_status bsmps_check_grid_wait(bsmps_ctx ctx, int skip_cta, int* timed_out);

/* ---- problem set-up (host only, no device needed) ----------------------- */

/* theta[i] = gamma/N + t_ii + sum_{j=k_i+1}^{k_i+N} (v_ijji - v_ijij),
 * k_i = max(0, i - N) (1-based i, j; Sec. 7.1.1): the diagonal coefficients
 * d_i of D = sum_i d_i a_i^* a_i that the preconditioner approximates
 * D^{-1/2} of.  N = n_particles; the spin-orbital integrals are
 * t_{p s, q s'} = h_pq delta_ss' and v_ijkl = 1/2 (il|jk) with matching spins
 * (Eq. (tvdef)).  h: n_orb x n_orb row-major; eri: (pq|rs) chemist order,
 * n_orb^4 row-major; theta: K = n_orb (spin = 0) or 2 n_orb (spin = 1)
 * entries, written.  Errors: INVALID_ARG. */
BSMPS_API bsmps_status bsmps_precond_theta(int n_orb, const double* h, const double* eri, int spin,
                                           int n_particles, double gamma, double* theta);

/* [t_min, t_max] enclosing the spectrum of D on the sector (Sec. 4.3, Cor.
 * lrprecond).  Per species s with n_s particles: when h is given and the
 * one-body diagonal h_pp increases strictly along that species' sites (the
 * orbital basis of the paper's Sec. 7.2, where t_min is D at e_1), the sums of
 * theta over the species' first / last n_s sites; otherwise the sums of the
 * n_s smallest / largest theta (the exact range of the spectrum of D).
 * theta: K entries; h: n_orb x n_orb or NULL.  Errors: INVALID_ARG, CHARGE. */
BSMPS_API bsmps_status bsmps_precond_interval(int n_orb, int spin, const double* theta, const double* h,
                                              int n_up, int n_dn, double* t_min, double* t_max);

/* A rigorous lower bound e_lb of the ground energy, for a shift
 * gamma = margin - e_lb that makes H_gamma = H + gamma I positive definite
 * (Sec. 3.1).  cholesky = 0: the interaction is nonnegative (on-site U >= 0),
 * e_lb is the ground energy of the one-body part.  cholesky = 1: (pq|rs) is
 * positive semidefinite (a sum of products of symmetric Cholesky vectors), and
 * normal ordering gives H >= the one-body operator h_pq - 1/2 sum_r (pr|rq).
 * The ground energy of a one-body operator is the sum of the n_up (and, with
 * spin = 1, n_dn) lowest eigenvalues of its matrix.  eri may be NULL when
 * cholesky = 0.  Errors: INVALID_ARG. */
BSMPS_API bsmps_status bsmps_energy_lower_bound(int n_orb, const double* h, const double* eri, int spin,
                                                int n_up, int n_dn, int cholesky, double* e_lb);

/* alpha_0 of Eq. (Sdef) and the spectral equivalence constant c of Eq.
 * (precondcdef) from c0 (Thm. expsum), t_min and C_lower, C_upper of Eq.
 * (lowerupper).  Errors: INVALID_ARG (c0 outside (0, 1), t_min <= 0, or
 * C_lower, C_upper not positive). */
BSMPS_API bsmps_status bsmps_precond_alpha0(double c0, double t_min, double c_lower, double c_upper,
                                            double* alpha0, double* c);

/* The D occupation strings (occ: D x K bytes, written; row i = determinant
 * i) of smallest one-particle energy sum_{i occupied} t_diag[i], the start
 * e_1, ..., e_D of the subspace iteration (Sec. 7.1.4).  Ties: strings
 * compared from site 0, occupied first (so the first is e_1 when t_diag
 * increases).  The sector is enumerated.  Errors: INVALID_ARG (sector
 * smaller than D), CHARGE, RANK_CAP (more than max_configs strings). */
BSMPS_API bsmps_status bsmps_lowest_determinants(int K, const double* t_diag, int spin, int n_up, int n_dn,
                                                 int D, int64_t max_configs, unsigned char* occ);

/* ---- MPS ----------------------------------------------------------------- */

/* Number of float64 entries of a fresh random iterate of maximal rank r_max
 * (block dims rho = min(left count, right count) if these fit r_max in total,
 * else min(left, right, floor(r_max * left*right / sum left*right)); sectors
 * of dim 0 dropped).  Errors: INVALID_ARG, CHARGE. */
BSMPS_API bsmps_status bsmps_mps_random_size(int n_orb, int spin, int n_up, int n_dn, int r_max,
                                   int64_t* n_values);

/* New iterate.  init = 0: e_1, the rank-one lowest determinant with the first
 * n_up species-0 and n_dn species-1 sites occupied (Sec. 7.1.4); values
 * ignored.  init = 1: blocks of the rule above filled from `values` (host,
 * n_values entries in flat layout, see bsmps_mps_random_size).
 * Errors: INVALID_ARG, CHARGE, OOM, CUDA. */
BSMPS_API bsmps_status bsmps_mps_create(bsmps_ctx ctx, int n_orb, int spin, int n_up, int n_dn,
                              int r_max, int init, const double* values, int64_t n_values,
                              bsmps_mps* out);

/* New iterate with explicit sectors: n_sectors[b] (b = 0..K) sectors per
 * bond, `sectors` the concatenated (n0, n1, dim) int triples per bond,
 * ascending; values in flat layout.  Errors: INVALID_ARG, CHARGE, OOM, CUDA. */
BSMPS_API bsmps_status bsmps_mps_import(bsmps_ctx ctx, int n_orb, int spin, int n_up, int n_dn,
                              const int* n_sectors, const int* sectors,
                              const double* values, int64_t n_values, bsmps_mps* out);

/* Shape queries: K; per-bond sector counts (K+1 ints) and their total; the
 * (n0, n1, dim) triples; the number of float64 entries in flat layout. */
BSMPS_API bsmps_status bsmps_mps_num_sites(bsmps_mps x, int* K);
BSMPS_API bsmps_status bsmps_mps_num_sectors(bsmps_mps x, int* per_bond, int* total);
BSMPS_API bsmps_status bsmps_mps_sectors(bsmps_mps x, int* triples);
BSMPS_API bsmps_status bsmps_mps_size(bsmps_mps x, int64_t* n_values);
/* Copy the blocks to host memory in flat layout (synchronises). */
BSMPS_API bsmps_status bsmps_mps_export(bsmps_mps x, double* values);
/* Overwrite the blocks of x in place from host memory in flat layout (n_values
 * = bsmps_mps_size; synchronises).  The device buffers of x keep their
 * addresses, so a recorded plan that reads x sees the new values at its next
 * launch.  Errors: INVALID_ARG, CUDA. */
BSMPS_API bsmps_status bsmps_mps_write(bsmps_mps x, const double* values, int64_t n_values);
BSMPS_API bsmps_status bsmps_mps_destroy(bsmps_mps x);

/* ---- MPO ----------------------------------------------------------------- */

/* MPO of H_gamma = H + gamma I for the second-quantized Hamiltonian
 * H = sum t_ij a_i^* a_j + sum v_ijkl a_i^* a_j^* a_k a_l (Eq. (hamil)),
 * v_ijkl = 1/2 (il|jk) (Eq. (tvdef), chemist notation), gamma folded into the
 * diagonal as t_ii + gamma/N (Sec. 7.1.1).
 * h: n_orb x n_orb row-major; eri: n_orb^4 row-major (pq|rs), both host.
 * With spin = 1 the spatial integrals are expanded to the interleaved
 * spin-orbitals.  Construction: Jordan--Wigner terms merged by canonical
 * site-local factors and wired as a finite-state MPO (channels: identity,
 * placed-prefix, remaining-suffix, finished; the prefix/suffix choice for
 * half-placed terms switches at bond K/2), ranks within Thm. opranks.
 * compress_tol: canonical terms with |coefficient| <= compress_tol are
 * dropped (0: keep every nonzero term).  Errors: INVALID_ARG, OOM, CUDA. */
BSMPS_API bsmps_status bsmps_mpo_from_integrals(bsmps_ctx ctx, int n_orb, const double* h,
                                      const double* eri, int spin, int n_particles,
                                      double gamma, double compress_tol, bsmps_mpo* out);
/* Bond dims (K+1 ints), per-site entry count, entries (a, b, sigma_out,
 * sigma_in) int quadruples with weights, and channel charges (pairs per
 * channel) of a bond. */
BSMPS_API bsmps_status bsmps_mpo_bond_dims(bsmps_mpo W, int* dims);
BSMPS_API bsmps_status bsmps_mpo_num_entries(bsmps_mpo W, int site, int* n);
BSMPS_API bsmps_status bsmps_mpo_entries(bsmps_mpo W, int site, int* quads, double* w);
BSMPS_API bsmps_status bsmps_mpo_channel_charges(bsmps_mpo W, int bond, int* pairs);
BSMPS_API bsmps_status bsmps_mpo_destroy(bsmps_mpo W);

/* ---- operations (all results are new handles) -------------------------- */

/* y = (H_gamma + shift I) x (Sec. 2.4).  tol = 0 and r_max = 0: exact
 * application, bond basis = MPO channel x x's basis, grouped by sector
 * (channel-major), sectors that no complete path reaches dropped.  Otherwise
 * y = trunc_tol of that result capped at r_max (see bsmps_truncate), computed
 * as the zip-up application of bsmps_apply_zipup followed by the right SVD
 * sweep of the truncation (the zip-up result is already left-orthogonal).
 * flops (may be NULL): algorithmic FP64 flops issued.
 * Errors: INVALID_ARG (mismatched sites/species), OOM, CUDA, TIMEOUT. */
BSMPS_API bsmps_status bsmps_apply_H(bsmps_ctx ctx, bsmps_mpo W, bsmps_mps x, double shift,
                           double tol, int r_max, bsmps_mps* y, double* flops);

/* y = (H_gamma + shift I) x in left-orthogonal form by the zip-up application
 * (Sec. 2.4 fused with the left-to-right QR sweep of Sec. 2.3), never forming
 * the exact cores.  The carry C_t[m] maps y's orthogonalised bond-t basis of
 * sector m to the exact basis (MPO channel a, x's sector m - Delta_a); site t
 * forms every block T(m, s')[:, seg_b] = sum over MPO entries (a, b, s', s)
 * of w C_t[m][:, seg_a] X_t(m - Delta_a, s) in one grouped GEMM (the
 * contraction stage, profiled as kernel kind 5), then per sector m' of bond
 * t+1 stacks the blocks (m, s') -> m' in layout order (m ascending, then s')
 * and takes Q = I, C_{t+1} = stack when the stack has no more rows than
 * columns, else Householder QR with diag(R) >= 0 (Q into y's core t,
 * C_{t+1} = R).  Bond t+1 of y has, per sector, min(stacked rows, exact
 * columns); the last core holds the norm.  D = 1 MPS only.  flops (may be
 * NULL): algorithmic FP64 flops issued.  Errors: INVALID_ARG, OOM, CUDA. */
BSMPS_API bsmps_status bsmps_apply_zipup(bsmps_ctx ctx, bsmps_mpo W, bsmps_mps x, double shift, bsmps_mps* y,
                                         double* flops);

/* The zip-up application of bsmps_apply_zipup for n independent problems
 * y[i] = (H_i + shift[i] I) x[i] (W[i] the operator of x[i]; the problems may
 * differ in operator, sites, particle numbers and ranks), advanced together:
 * site t of every problem that has one shares one grouped-GEMM launch for the
 * contraction and one launch each for the zeroing, gathers, QRs and scatters of
 * the factorisation.  Results equal those of n separate bsmps_apply_zipup
 * calls to rounding (the contraction's kernel split is autotuned per launch
 * size class, so sums may be ordered differently).  W, x, shift: n entries, host
 * arrays; y: n new handles.  flops (may be NULL): algorithmic FP64 flops of the
 * batch.  Errors: INVALID_ARG, OOM, CUDA. */
BSMPS_API bsmps_status bsmps_apply_zipup_batch(bsmps_ctx ctx, int n, const bsmps_mpo* W, const bsmps_mps* x,
                                               const double* shift, bsmps_mps* y, double* flops);

/* The batched zip-up application of bsmps_apply_zipup_batch recorded once as a
 * CUDA graph, for repeated application of the same operators to iterates of
 * fixed structure (the inner loop of a batch of independent solves at fixed
 * ranks).  Recording runs the batch once on the context's stream (which sizes
 * the graph's memory and fixes the contraction autotuner's choices), then
 * captures the same launch sequence into a graph whose buffers live in one
 * device arena and whose task lists live in pinned host memory owned by the
 * plan.  bsmps_plan_launch replays every launch of the batch with one graph
 * launch on the context's stream: it reads the blocks x[i] hold at that point
 * in stream order (update them in place with bsmps_mps_write) and overwrites
 * the plan's outputs.  ctx: a context created with a non-default stream, which
 * must outlive the plan.  W, x: n handles each, which must outlive the plan;
 * shift: n values, read now.
 * y: n new handles to the outputs, whose blocks belong to the plan (valid from
 * the first bsmps_plan_launch until bsmps_plan_destroy; bsmps_mps_destroy on
 * them releases the handle only).  flops (may be NULL): algorithmic FP64 flops
 * of one launch.  The recording runs the zip-up's FP64 or split-precision
 * contraction as the context's precision selects at this call.
 * Errors: INVALID_ARG (null arguments, default stream), OOM, CUDA. */
BSMPS_API bsmps_status bsmps_plan_apply_zipup_batch(bsmps_ctx ctx, int n, const bsmps_mpo* W, const bsmps_mps* x,
                                                    const double* shift, bsmps_plan* plan, bsmps_mps* y,
                                                    double* flops);
/* One replay of the recorded batch on the context's stream (asynchronous;
 * bsmps_ctx_sync or any synchronising call waits for it).  Errors: INVALID_ARG,
 * CUDA. */
BSMPS_API bsmps_status bsmps_plan_launch(bsmps_plan plan);
/* Kernel launches one bsmps_plan_launch replays (also added to the context's
 * bsmps_ctx_launch_count at every launch). */
BSMPS_API int64_t bsmps_plan_launch_count(bsmps_plan plan);
/* Waits for the context's stream, then releases the graph and its memory. */
BSMPS_API bsmps_status bsmps_plan_destroy(bsmps_plan plan);

/* trunc_eps (Sec. 2.2, Eq. (ttsvdquasiopt)): QR sweep left to right (diag R
 * >= 0), then right to left SVD of [X_b(n,0) | X_b(n,1)] per left sector;
 * at every bond the pooled singular values are discarded from the smallest
 * while their squared sum stays <= eps^2/(K-1) (so ||x - y|| <= eps), a cut
 * inside a cluster of relative gap < 1e-10 moves to keep the cluster; then at
 * most r_max (> 0) are kept.  disc_tol / disc_cap (may be NULL): Frobenius
 * norms discarded by the tolerance / by the cap.
 * Errors: INVALID_ARG, OOM, CUDA. */
BSMPS_API bsmps_status bsmps_truncate(bsmps_ctx ctx, bsmps_mps x, double eps, int r_max,
                            bsmps_mps* y, double* disc_tol, double* disc_cap);

/* out = alpha x + beta y by block concatenation (Sec. 2.3).  Errors:
 * INVALID_ARG (different sites / targets), OOM, CUDA. */
BSMPS_API bsmps_status bsmps_add(bsmps_ctx ctx, bsmps_mps x, bsmps_mps y, double alpha, double beta,
                       bsmps_mps* out);

/* out = x with every sigma=0 block of site t scaled by f0[t] and every sigma=1
 * block by f1[t] (f0, f1 host arrays of length K): the action of one
 * rank-one diagonal Kronecker operator (Sec. 4.3). */
BSMPS_API bsmps_status bsmps_scale_sites(bsmps_ctx ctx, bsmps_mps x, const double* f0, const double* f1,
                               bsmps_mps* out);

/* y = S_m x for term = m - M^- in [0, #S), or y = S x = sum_m S_m x
 * (block concatenation of the scaled copies, rank #S times) for term = -1
 * (Sec. 4.3).  n_terms (may be NULL) receives #S = M^+ - M^- + 1.
 * Errors: INVALID_ARG, NOT_SPD (t_min <= 0 or t_max < t_min), OOM, CUDA. */
BSMPS_API bsmps_status bsmps_precondition(bsmps_ctx ctx, const bsmps_precond* p, int term, bsmps_mps x,
                                bsmps_mps* y, int* n_terms);

/* out = <a, O b> in float64 with O = (H_gamma + shift I) given by W, or the
 * identity when W is NULL (left-to-right environment recursion). */
BSMPS_API bsmps_status bsmps_dot(bsmps_ctx ctx, bsmps_mps a, bsmps_mps b, bsmps_mpo W, double shift,
                       double* out);

/* Same result as bsmps_dot, computed without allocating device memory.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc (or any allocating routine) at the time they need an inner
 * product -- for example code running under a device-memory budget enforced by
 * another framework's allocator, or latency-critical loops that must not
 * trigger an allocation.  a, b (and W) are ordinary handles created earlier.
 * All temporaries (environment blocks, intermediate products, kernel task
 * lists) live in one 32 MiB file-scope device array that every device which
 * loads the library holds until the process exits.  The first call on a device
 * resolves the array's device address (cudaGetSymbolAddress with that device
 * current); make that first call before any stream capture.  Contractions
 * whose temporaries do not fit the 32 MiB return BSMPS_ERR_RANK_CAP with the
 * required size in bsmps_last_error.  Every call reuses the same array, so
 * calls that overlap on the GPU (several streams or host threads at once)
 * race and must be serialised by the caller.  Synchronises the context stream.
 * Errors: INVALID_ARG, RANK_CAP, CUDA. */
BSMPS_API bsmps_status bsmps_dot_noalloc(bsmps_ctx ctx, bsmps_mps a, bsmps_mps b, bsmps_mpo W,
                                         double shift, double* out);

/* One pass of the loop body of Alg. 2 on x^n = *x:
 * lambda^n (Eq. (exactrq)), normalisation in the A-norm, the residual
 * res_eta from the terms S_k (H_gamma - lambda) S_k' x (Sec. 5.3.1, eta_res
 * started at min(2 eta_res, 4/5 zeta sum ||s_j||) and multiplied by 4/5 until
 * accepted), rho^n (Eq. (rhobound)), the termination test (Thm.
 * aposterbound), the 2x2 Rayleigh-Ritz step (Remark omegamin) and
 * x^{n+1} = trunc_{eta_in}(x*) (Sec. 5.3.2).
 * *x is replaced by x^{n+1} (or by the normalised x^n when the test holds);
 * the old handle is destroyed by the call.  state is updated in place.
 * Errors: INVALID_ARG, NOT_SPD, NUMERIC, OOM, CUDA. */
BSMPS_API bsmps_status bsmps_eigensolve_step(bsmps_ctx ctx, bsmps_mpo W, const bsmps_precond* p,
                                   const bsmps_solver_params* params,
                                   bsmps_solver_state* state, bsmps_mps* x,
                                   bsmps_step_info* info);

/* ---- FP64 products on the tensor cores ----------------------------------- */

/* C = A B in float64, emulated on the bf16 tensor cores by the Ozaki scheme
 * (Ozaki, Ogita, Oishi, Rump 2012; not part of the paper).
 *   - Scaling: each row of A and each column of B is scaled by a power of two
 *     below which all its entries lie.
 *   - Slices: the scaled values are cut into `slices` (1..8) digits of 7 bits
 *     plus sign, each exact in bf16.
 *   - Products: slice pairs (p, q) with p + q <= slices + 1 are multiplied
 *     exactly (FP32 accumulation of integers below 2^24, 128 values of k at a
 *     time) and summed in float64.
 * Error bound per entry, in units of K 2^{e_i + f_j}:
 * 2^{1 - 7 slices} + sum_{d > slices+1} (2 slices - d + 1) 2^{14 - 7d}
 * + slices 2^{-52}.  With 8 slices this is within a few units of float64
 * rounding relative to max_k |a_ik| max_k |b_kj| K.
 * A (M x K, leading dimension lda), B (K x N, ldb) and C (M x N, ldc) are
 * row-major DEVICE pointers.  The work is ordered on the context stream and the
 * call does not synchronise.  Errors: INVALID_ARG, OOM, CUDA. */
/* C = A B (M x N) on the tensor cores in split precision (BSMPS_PREC_TF32X3):
 * every entry of A and B is split into two TF32 values, the three products
 * A_hi B_hi + A_hi B_lo + A_lo B_hi are accumulated in FP32 in tensor memory
 * (tcgen05.mma kind::tf32, 128 x 64 tiles), and C is stored in FP64.  The error
 * of C_ij is a few units of 2^-21 times sum_k |a_ik| |b_kj| plus the FP32
 * accumulation error.  The paper has no counterpart: this is the contraction
 * kernel of the split-precision MPO application, exposed for testing.  A
 * (M x K, lda), B (K x N, ldb) and C (M x N, ldc) are row-major DEVICE
 * pointers; stream-ordered on the context stream, no synchronisation.  A bounded
 * wait that gives up is reported as TIMEOUT at the context's next
 * synchronising call.  Errors: INVALID_ARG, OOM, CUDA. */
BSMPS_API bsmps_status bsmps_gemm_tf32x3(bsmps_ctx ctx, int M, int N, int K, const double* A, int lda,
                                         const double* B, int ldb, double* C, int ldc);

/* Arithmetic of the contraction stage of the zip-up MPO application
 * (bsmps_apply_zipup, bsmps_apply_H with a tolerance, and the residual terms
 * of bsmps_eigensolve_step): BSMPS_PREC_FP64 (the default) or
 * BSMPS_PREC_TF32X3.  Factorisations, inner products, the Rayleigh quotient and
 * norms stay FP64.  In the eigensolver step the split precision is used only
 * while its error estimate stays below a tenth of the previous step's residual
 * tolerance eta_res (the budget of Lemma truncr); after that the step falls
 * back to FP64 for the rest of the iteration (bsmps_step_info.precision
 * reports the choice).  Errors: INVALID_ARG. */
BSMPS_API bsmps_status bsmps_ctx_set_precision(bsmps_ctx ctx, int precision);

/* Block products of at least 2^min_log2_flops flops with a single untransposed
 * contribution (the large R X and U S X products of sweeps over wide sectors;
 * transposed products stay on the FP64 units) run as
 * bsmps_gemm_ozaki with 8 slices, all such products of one grouped launch
 * together; 0 (the default) keeps every product on the FP64 units.  The
 * emulation's error is relative to row and column maxima, so on graded factors
 * it can move truncation decisions at the level of the truncation tolerance
 * (the iteration stays within its error control, but the trajectory is not the
 * FP64 one).  Errors: INVALID_ARG (negative or above 60). */
BSMPS_API bsmps_status bsmps_ctx_set_gemm_emulation(bsmps_ctx ctx, int min_log2_flops);

/* Truncation SVDs whose triangular factor is k x k with min_k <= k <= 336 start
 * the FP64 one-sided Jacobi from an FP32 one: the FP32 rotations P (orthogonal
 * to about 1e-6), re-orthogonalised in FP64 by Householder QR (Qp), give
 * G Qp, whose FP64 Jacobi converges in a few sweeps; V = Qp V1.  Every
 * quantity the truncation reads (singular values, vectors) is still the
 * result of the FP64 Jacobi, to FP64 rounding.  min_k = 0 turns it off; the
 * default is 48.  Errors: INVALID_ARG (negative). */
BSMPS_API bsmps_status bsmps_ctx_set_jacobi_precond(bsmps_ctx ctx, int min_k);

BSMPS_API bsmps_status bsmps_gemm_ozaki(bsmps_ctx ctx, int M, int N, int K, const double* A, int lda,
                                        const double* B, int ldb, double* C, int ldc, int slices);

/* ---- joint block MPS and the subspace iteration (Alg. 4, Sec. 6) -------- */

/* A joint block MPS holds D vectors x_1..x_D in one MPS whose last bond (the
 * single target sector) has dimension D: the eigenvector-specific core of
 * Sec. 6.2 placed after the last site (position p = K + 1) and absorbed into
 * the last core.  Inner bonds carry the vectors' bases stacked block-diagonally,
 * so their ranks are at most the sums of the individual ranks.  Vector i is
 * column i of the last core's blocks.  A plain MPS is the case D = 1.
 * bsmps_truncate (one tolerance for the whole joint tensor, Frobenius norm
 * over all columns), bsmps_add (columns added, not stacked) and
 * bsmps_scale_sites accept joint MPS; bsmps_dot, bsmps_dot_noalloc and the
 * single-vector solvers require D = 1. */
#define BSMPS_MAX_COLUMNS 16

/* Number of float64 entries of a fresh random joint iterate of D columns: the
 * rule of bsmps_mps_random_size with every right configuration count
 * multiplied by D.  Errors: INVALID_ARG, CHARGE. */
BSMPS_API bsmps_status bsmps_mps_joint_random_size(int n_orb, int spin, int n_up, int n_dn, int r_max, int D,
                                                   int64_t* n_values);

/* New joint iterate of D columns.  init = 0: the unit vectors of the D
 * occupation strings in occ (host, D x K bytes, row i = vector i, entries 0/1,
 * each in the particle sector): vector i owns one basis index on every inner
 * bond (block-diagonal stacking of Sec. 6.2).  init = 1: random, blocks of the
 * rule of bsmps_mps_joint_random_size filled from values (host, flat layout).
 * Errors: INVALID_ARG, CHARGE, OOM, CUDA. */
BSMPS_API bsmps_status bsmps_mps_create_joint(bsmps_ctx ctx, int n_orb, int spin, int n_up, int n_dn, int D,
                                              int init, const unsigned char* occ, int r_max, const double* values,
                                              int64_t n_values, bsmps_mps* out);

/* D of a (joint) MPS. */
BSMPS_API bsmps_status bsmps_mps_num_columns(bsmps_mps x, int* D);

/* out = the D_a x D_b matrix <a_i, O b_j> (row-major, host) with
 * O = H_gamma + shift I given by W, or the identity when W is NULL: one
 * left-to-right environment sweep whose last environment keeps both column
 * indices (Sec. 6.1).  Errors: INVALID_ARG, RANK_CAP (environments too large
 * for the persistent sweep), OOM, CUDA, TIMEOUT. */
BSMPS_API bsmps_status bsmps_gram(bsmps_ctx ctx, bsmps_mps a, bsmps_mps b, bsmps_mpo W, double shift,
                                  double* out);

/* Exact y = (H_gamma + shift I) X + X diag(col_shift) for a joint block MPS X of
 * D columns (col_shift: host, D entries), the operator of Eq. (respara) with
 * shift = 0 and col_shift = -Lambda.  The column term enters on the MPO's
 * identity rail at the last site, so y has the bond dimensions of the exact
 * application (see bsmps_apply_H).  Errors: INVALID_ARG, OOM, CUDA. */
BSMPS_API bsmps_status bsmps_apply_columns(bsmps_ctx ctx, bsmps_mpo W, bsmps_mps x, double shift,
                                           const double* col_shift, bsmps_mps* y);

/* y = X Wm: the D_in x D_out row-major host matrix Wm mixes the columns (the
 * last core's blocks are multiplied by Wm), y has D_out columns (Sec. 6.1).
 * Errors: INVALID_ARG (K = 1), OOM, CUDA. */
BSMPS_API bsmps_status bsmps_mix_columns(bsmps_ctx ctx, bsmps_mps x, const double* Wm, int D_out, bsmps_mps* y);

/* Scalars reported by one step of Alg. 4 (column i = i-th lowest Ritz value). */
typedef struct {
    int D;
    double lambda[BSMPS_MAX_COLUMNS];       /* Lambda^n after the Rayleigh-Ritz step on X^n */
    double rho[BSMPS_MAX_COLUMNS];          /* rho_i^n, Eq. (rhobound) with ||x_i||_A = 1 */
    double res_norm[BSMPS_MAX_COLUMNS];     /* ||r_i^n|| of res_eta(X^n) */
    double lambda_star[BSMPS_MAX_COLUMNS];  /* lowest D Ritz values on span (X^n R^n) */
    double delta_A[BSMPS_MAX_COLUMNS];
    double eta_res;      /* accepted residual tolerance */
    int eta_tries;       /* passes of the eta_res loop beyond the first */
    double bound;        /* eigenvector bound of column 1 (Thm. aposterbound) */
    double releig_bound; /* relative eigenvalue bound of column 1, Eq. (releigerr) */
    double eta_in;       /* truncation tolerance of the iterate */
    int converged;       /* 1 when the termination test of Alg. 4 held */
    int max_rank;        /* largest bond dimension of the returned iterate */
    double flops;        /* algorithmic FP64 flops issued by the step */
    double cap_discarded;
} bsmps_joint_step_info;

/* One pass of the loop body of Alg. 4 on the joint iterate X^n = *x (D
 * columns, 1 <= D <= BSMPS_MAX_COLUMNS): Rayleigh-Ritz on span X^n (lowest
 * generalized eigenpairs of X^T A X, X^T E X; A-orthonormal columns, Lambda^n);
 * residual terms S_k (H_gamma S_k' X - S_k' X Lambda) (Eq. (respara)) summed by
 * res_eta as in Alg. 2 with Frobenius norms of the joint terms, eta_res
 * multiplied by 4/5 while min_i ||r_i|| < (1 + 1/zeta) eta_res; rho_i; the
 * termination test on rho_1; Rayleigh-Ritz on span (X^n R^n) in the basis
 * normalised by the column norms (Sec. 6.1), lowest D pairs;
 * eta_in = (1+c)^{-1/2} min_i Delta_{A,i}; X^{n+1} = trunc_{eta_in}(X*) capped at
 * params->r_max.  Gram matrices use the symmetry of H_gamma and the S_k.
 * *x is replaced (old handle destroyed); state as for bsmps_eigensolve_step.
 * Errors: INVALID_ARG, NOT_SPD, NUMERIC (also a singular subspace basis), OOM,
 * CUDA, TIMEOUT. */
BSMPS_API bsmps_status bsmps_eigensolve_joint_step(bsmps_ctx ctx, bsmps_mpo W, const bsmps_precond* p,
                                                   const bsmps_solver_params* params, bsmps_solver_state* state,
                                                   bsmps_mps* x, bsmps_joint_step_info* info);

/* One outer step of Alg. 3 as reported by bsmps_eigensolve_outer. */
typedef struct {
    int inner_steps;       /* Alg. 2 steps run from y^m */
    int inner_converged;   /* 1 when the inner termination test (bound <= tau_m) held */
    double lambda;         /* lambda(y^+) */
    double rho;            /* rho(y^+), Eq. (rhobound) */
    double releig_bound;   /* Eq. (releigerr) at y^+ */
    double eta_out;        /* eta_m */
    double tau_m;          /* inner tolerance eta_m / (2 (1 + (1 + alpha) kappa)) */
    int max_rank_before;   /* largest bond dimension of y^+ */
    int max_rank_after;    /* largest bond dimension of y^{m+1} (of y^+ at the last step) */
    double flops;          /* algorithmic FP64 flops of the outer step */
} bsmps_outer_record;

/* Outer perturbed inverse iteration (Alg. 3, one eigenvector): with
 * kappa = sqrt((1+c)/(1-c)) sqrt(K-1) (Eq. (kappadef)) and
 * theta = (1+alpha) kappa / (2 (1 + (1+alpha) kappa)) (Thm. quasioptr),
 * eta_0 = 1/(2 theta); outer step m runs Alg. 2 steps from y^m (fresh state,
 * eta_res = +inf) until the eigenvector bound of Thm. aposterbound is at most
 * tau_m = eta_m / (2 (1 + (1+alpha) kappa)) or max_inner steps were taken;
 * it stops when the relative eigenvalue bound of Eq. (releigerr) at the
 * result y^+ is below tau, else y^{m+1} = trunc_{theta eta_m}(y^+) and
 * eta_{m+1} = eta_m / 2.  params as for bsmps_eigensolve_step except that
 * params->tau is ignored (the inner tolerance is tau_m); params->r_max caps the
 * inner iterates only.  alpha > 0 is not fixed by the paper.  *x (y^0) is
 * replaced by the final y^+ (the old handle is destroyed); records (may be
 * NULL) receives up to max_outer records, *n_outer the number of outer steps,
 * *converged 1 when the tau test held.  Errors: INVALID_ARG, NOT_SPD, NUMERIC,
 * OOM, CUDA. */
BSMPS_API bsmps_status bsmps_eigensolve_outer(bsmps_ctx ctx, bsmps_mpo W, const bsmps_precond* p,
                                              const bsmps_solver_params* params, double alpha, double tau,
                                              int max_outer, int max_inner, bsmps_mps* x,
                                              bsmps_outer_record* records, int* n_outer, int* converged);

/* ---- learned preconditioner network ------------------------------------- *
 * A multilayer perceptron (no counterpart in the paper; it serves the learned
 * preconditioner controller that predicts preconditioner parameters from the
 * one-body spectrum and the residual history, with the paper's plain
 * preconditioner as fallback).  Layers l = 0..n_layers-1 map widths[l] to
 * widths[l+1]; hidden layers use ReLU, the last layer is linear.  The forward
 * and backward products use BF16 copies of the weights with FP32 accumulation;
 * the FP32 master parameters are updated by Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8) and re-rounded to BF16 (round to nearest even) after every update.
 * Flat parameter layout: for each layer W (widths[l+1] x widths[l], row-major)
 * then b (widths[l+1]).  Inputs/outputs are host float32 arrays, row-major
 * (batch x width).  Loss: mean over batch and outputs of (y - t)^2. */
BSMPS_API bsmps_status bsmps_mlp_create(bsmps_ctx ctx, int n_layers, const int* widths,
                                        const float* params, int64_t n_params, bsmps_mlp* out);
BSMPS_API bsmps_status bsmps_mlp_num_params(bsmps_mlp net, int64_t* n);
BSMPS_API bsmps_status bsmps_mlp_get_params(bsmps_mlp net, float* params);
BSMPS_API bsmps_status bsmps_mlp_forward(bsmps_mlp net, const float* x, int batch, float* y);
/* loss and (when grad != NULL) the gradient of the loss w.r.t. the flat
 * parameters, evaluated with the BF16 weights. */
BSMPS_API bsmps_status bsmps_mlp_loss_grad(bsmps_mlp net, const float* x, const float* t, int batch,
                                           float* loss, float* grad);
/* one Adam step on a batch; *loss (may be NULL) is the loss before the step. */
BSMPS_API bsmps_status bsmps_mlp_train_step(bsmps_mlp net, const float* x, const float* t, int batch,
                                            float lr, float* loss);
BSMPS_API bsmps_status bsmps_mlp_destroy(bsmps_mlp net);

#ifdef __cplusplus
}
#endif

#endif /* BSMPS_H */
