/*
 * qhfpe.h -- C ABI of the GB300 (sm_103a) library for the multi-state quantum hierarchical
 * Fokker-Planck equation (MS-QHFPE) of Ikeda & Tanimura, J. Chem. Phys. 2017 (arXiv:1706.09590).
 *
 * The library time-steps the hierarchy of electronic-state-resolved Wigner distributions
 * W^(n)_jk(q, p) of Eq. (heom) on a phase-space grid, applies the dipole super-operators of Sec. III
 * and returns the response functions of Eqs. (R1), (R3) and the spectra built from them.
 *
 * Units: hbar = m = omega_0 = 1 (the dimensionless q, p of Sec. III).
 *
 * Conventions shared by every call:
 *   - Grid: x_i = x_min + i*dx with dx = (x_max - x_min)/n, i = 0..n-1 (end point excluded), for both
 *     q (nq points) and p (np points, np a power of two, 8 <= np <= 512).
 *   - Hierarchy: the index set {n in N^(K+1) : |n| <= depth} of Eq. (heom) with K = n_matsubara,
 *     ordered by tier |n| ascending and, inside a tier, lexicographically with n_0 largest first.
 *     qhfpe_hierarchy() returns the list.
 *   - State layout at the ABI ("canonical"): complex128 (re, im interleaved) array
 *     [n_elem][S][S][nq][np], element index, ket state j, bra state k, q row, p column.  One such
 *     array per replica; replica r of a batch starts at r * state_elems(h) complex numbers.
 *   - Potential tables: U_table[j][k][i][t] = U_jk(q_i + s_t) with s_t = (t - np/2) * pi / (np*dp),
 *     t = 0..np (np+1 samples per q row): the surfaces at q +/- r/2 on the grid r conjugate to p,
 *     Eq. (quantum-liouvillian).  Real, symmetric in (j, k).  The caller chooses how U continues
 *     beyond the q box (the kernel samples up to pi/(2 dp) outside it).
 *   - Time: one step is one RK4 step of size dt (classic RK4 = the degree-4 Taylor polynomial of the
 *     propagator for this linear equation, the 4th-order integrator of Sec. III at fixed step).
 *
 * Ownership and streams: the library owns every device buffer it allocates (released by
 * qhfpe_destroy).  Host arrays passed in are copied before the call returns.  Device pointers passed in
 * are read/written in stream order on the handle's stream and are not retained.  Host outputs are
 * complete when the call returns.
 *
 * Errors: every call returns a qhfpe_status; no exception or abort crosses the ABI.  After a CUDA
 * failure or a device-side timeout the handle turns sticky: every later call returns QHFPE_ESTATE
 * until qhfpe_destroy.  qhfpe_last_error() gives a one-line description of the last failure.
 */
#ifndef QHFPE_H
#define QHFPE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QHFPE_OK = 0,
    QHFPE_EINVAL = 1,       /* invalid argument (message in qhfpe_last_error) */
    QHFPE_ENOMEM = 2,       /* device or host allocation failed */
    QHFPE_ECUDA = 3,        /* CUDA runtime error */
    QHFPE_ENUMERIC = 4,     /* NaN or Inf found where finite values are required */
    QHFPE_ETIMEOUT = 5,     /* a device-side wait gave up (reported, never hung) */
    QHFPE_EUNSUPPORTED = 6, /* valid request this build does not implement */
    QHFPE_ESTATE = 7        /* handle unusable after an earlier device failure */
} qhfpe_status;

/* Arithmetic of the propagation. */
typedef enum {
    /* Everything in FP64; potential kernel by shared-memory FFT.  Reference form. */
    QHFPE_FP64 = 0,
    /* State and right-hand side in FP32 (FFT potential kernel in FP32); the zeroth tier's state and
     * its RK4 accumulation kept in FP64; traces and response sums in FP64. */
    QHFPE_MIXED = 1,
    /* As QHFPE_MIXED, but the potential kernel is a DFT-as-GEMM on the tcgen05 tensor cores with
     * split bf16 (hi + lo, three products) operands and FP32 accumulation. */
    QHFPE_MIXED_BF16X3 = 2,
    /* Reserved: the same DFT-as-GEMM with split TF32 operands.  Not built; qhfpe_create returns
     * QHFPE_EUNSUPPORTED.  kind::tf32 runs at half the bf16 tensor rate with twice the operand bytes,
     * so the resident cosine/sine operand tiles (hi and lo, 256 KB at np = 128) no longer fit in
     * shared memory beside the streamed state; the split-bf16 form already meets the mixed forms'
     * 1e-4 accuracy on the responses. */
    QHFPE_MIXED_TF32X3 = 3
} qhfpe_precision;

typedef enum {
    QHFPE_TRUNCATE = 0,   /* W^(n + e_k) = 0 beyond the deepest tier */
    QHFPE_TERMINATOR = 1, /* Eq. (GMFP) at the deepest tier; requires n_matsubara = 0 */
    QHFPE_LEARNED = 2,    /* learned closure, n_matsubara = 0 (see qhfpe_closure_load) */
    QHFPE_LEARNED_STATE = 3 /* state-input learned closure (see qhfpe_closure_state_load): n_matsubara = 0,
                             * QHFPE_FP64, n_states <= 2, np in {32, 64, 128, 256}; classic RK4 */
} qhfpe_closure;

typedef enum {
    QHFPE_LEFT = 1,       /* mu^-> W = mu W  (ket side)   */
    QHFPE_RIGHT = 2,      /* mu^<- W = W mu  (bra side)   */
    QHFPE_COMMUTATOR = 3  /* mu^x W = mu W - W mu          */
} qhfpe_side;

/* Right-hand-side term mask for qhfpe_apply_rhs (test and diagnostics entry point). */
enum {
    QHFPE_TERM_KINETIC = 1,   /* -p dW/dq, 5th-order upwind (Sec. III)                              */
    QHFPE_TERM_POTENTIAL = 2, /* -i [U, W] in Wigner space, Eq. (quantum-liouvillian)                */
    QHFPE_TERM_DAMPING = 4,   /* -(sum_k n_k gamma_k) W + c_delta d2W/dp2, Eq. (heom)                */
    QHFPE_TERM_TIER_UP = 8,   /* sum_k dW^(n+e_k)/dp, or the Eq. (GMFP) terminator                   */
    QHFPE_TERM_TIER_DOWN = 16,/* sum_k n_k gamma_k (r_k p + c_k d/dp) W^(n-e_k), Eq. (heom)          */
    QHFPE_TERM_ALL = 31
};

typedef struct {
    int n_states;            /* S >= 1 (at most 4) */
    int nq, np;              /* nq >= 1; np a power of two in [8, 512] */
    double q_min, q_max, p_min, p_max;
    const double *U_table;   /* host, [S][S][nq][np+1] (see conventions); copied */
    const double *mu;        /* host, [S][S] Condon dipole matrix, real symmetric; copied */
    double eta, gamma, beta; /* Drude coupling zeta (Eq. (Drude-J)), cutoff gamma, inverse temperature */
    int n_matsubara;         /* K: modes k = 0..K (K <= 7) */
    int high_temperature;    /* 1: c_0 = eta/beta, no Matsubara terms, no delta-term (end of Sec. II) */
    int use_cdelta;          /* 1: keep the delta-term c_delta d2/dp2 (low-temperature remainder) */
    int depth;               /* N >= 0 */
    int closure;             /* qhfpe_closure */
    int periodic_q;          /* 0: open q boundary (zero ghost cells); 1: periodic q */
    int precision;           /* qhfpe_precision */
    double dt;               /* RK4 step > 0 */
    int n_replicas;          /* independent propagations held by the handle, >= 1 */
    /* System side of the system-bath coupling, Sec. II: V(q) = q + v_c2 q^2 (0: the linear coupling
     * the paper works with).  With hbar = m = 1 and phi(q) = 1 + 2 v_c2 q the operators of Eq. (heom)
     * become Phi = -phi d/dp, Lambda^(1) = -p phi - (v_c2/2) d2/dp dq, Lambda^(2) = v_c2 phi d/dp
     * (Lambda^(>=3) = 0), and Phi^2 = phi^2 d2/dp2; the |m| = 2 couplings of Eq. (heom) to
     * W^(n - e_k - e_l) enter with their multinomial weights.  d/dq in the mixed derivative: 4th-order
     * central differences (zero ghost cells, or periodic).  Nonzero v_c2 requires closure =
     * QHFPE_TRUNCATE (the Eq. (GMFP) terminator assumes V = q), a fused shape (np in {32, 64, 128, 256},
     * n_states <= 3) and a finite value; EINVAL / EUNSUPPORTED otherwise. */
    double v_c2;
} qhfpe_params;

typedef struct qhfpe qhfpe_t;

/* Validates params, derives the bath coefficients (Eqs. (expansion-of-bath-*) for the Drude J) and
 * the hierarchy, uploads the tables and allocates all device buffers.  All replicas start at zero.
 * stream: a cudaStream_t or NULL for the legacy default stream.  Errors: EINVAL (bad parameter),
 * ENOMEM, ECUDA, EUNSUPPORTED (e.g. a precision this GPU cannot run). */
qhfpe_status qhfpe_create(const qhfpe_params *params, void *stream, qhfpe_t **out);
qhfpe_status qhfpe_destroy(qhfpe_t *h);
const char *qhfpe_last_error(const qhfpe_t *h);

/* Sizes: number of hierarchy elements, modes (K+1) and complex numbers per replica state. */
qhfpe_status qhfpe_sizes(const qhfpe_t *h, int *n_elem, int *n_modes, size_t *state_elems);
/* idx_out: host int[n_elem][n_modes], the multi-indices in storage order. */
qhfpe_status qhfpe_hierarchy(const qhfpe_t *h, int *idx_out);
/* Bath coefficients as used (host arrays of n_modes doubles; cdelta one double). */
qhfpe_status qhfpe_bath_coefficients(const qhfpe_t *h, double *gamma_k, double *r_k, double *c_k, double *cdelta);
/* Upper bound of a stable dt from a Gershgorin-type estimate of the generator's spectral radius and
 * RK4's stability interval on the imaginary axis (2.8). */
qhfpe_status qhfpe_max_stable_dt(const qhfpe_t *h, double *dt_out);

/* Copy a canonical-layout complex128 state into / out of replica `replica` (or every replica when
 * replica = -1 for set_state: the same state is broadcast).  is_device: the pointer is device memory.
 * In the mixed forms the state is rounded to FP32 except the zeroth tier, which stays FP64.
 * set_state checks the values on the device and returns QHFPE_ENUMERIC on NaN/Inf. */
qhfpe_status qhfpe_set_state(qhfpe_t *h, int replica, const double *src, int is_device);
qhfpe_status qhfpe_get_state(qhfpe_t *h, int replica, double *dst, int is_device);
/* The same with a complex64 canonical state (half the bytes; for the mixed forms, whose higher tiers
 * are FP32 anyway): set_state32 widens the values as given (the zeroth tier of the mixed forms becomes
 * their FP64 value), get_state32 rounds each value, including the FP64 zeroth tier, to FP32. */
qhfpe_status qhfpe_set_state32(qhfpe_t *h, int replica, const float *src, int is_device);
qhfpe_status qhfpe_get_state32(qhfpe_t *h, int replica, float *dst, int is_device);
/* Copy replica src onto each of dst[0..n-1] (host int array). */
qhfpe_status qhfpe_fork(qhfpe_t *h, int src, const int *dst, int n);

/* Advance every replica n_steps RK4 steps.  trace_out (host, may be NULL): complex128
 * [n_replicas][n_steps + 1], Tr{mu W^(0)} = sum_jk mu_kj sum_il W^(0)_jk(q_i, p_l) dq dp before the
 * first step and after each step (FP64 sums, Eqs. (R1), (R3)). */
qhfpe_status qhfpe_step(qhfpe_t *h, long n_steps, double *trace_out);

/* ---- Heterogeneous batch ------------------------------------------------------------------------
 * Several handles advanced together: each Horner stage of the RK4 step (Sec. III's 4th-order
 * integrator applied to Eq. (heom)) of every member is ONE launch of the fused stage kernel, whose
 * blocks read their member's description (grid, tables, buffers, dt) from a device table, and whole
 * steps are replayed from captured CUDA graphs.  Members may differ in nq, the q and p ranges, the
 * surfaces, the bath (eta, gamma, beta, Matsubara count, delta-term), the depth, the closure
 * (TRUNCATE or TERMINATOR), periodic_q, dt and n_replicas; they must share np, n_states and the
 * precision (QHFPE_FP64 or QHFPE_MIXED; not the tensor-core form, not the learned closure), and np and
 * n_states must have a fused kernel (np in {32, 64, 128, 256}, n_states <= 3).  Each member's result
 * is that of qhfpe_step on the member alone (the same per-cell arithmetic).
 * members: host array of n distinct handles; the batch keeps the pointers, does not own the handles,
 * and must be destroyed before any of them.  Errors are reported through members[0]
 * (qhfpe_last_error); EINVAL for mismatched or repeated members, EUNSUPPORTED for the forms above. */
typedef struct qhfpe_batch qhfpe_batch_t;
qhfpe_status qhfpe_batch_create(qhfpe_t *const *members, int n, qhfpe_batch_t **out);
/* Advance every replica of every member n_steps RK4 steps (each member with its own dt), on members[0]'s
 * stream after waiting for every member's stream.  trace_out: NULL, or a host array of n pointers, each
 * NULL or a host complex128 [n_replicas][n_steps + 1] array receiving that member's Tr{mu W^(0)} as
 * qhfpe_step does.  The tile height is timed on the first call (QHFPE_TILE_ROWS pins it). */
qhfpe_status qhfpe_batch_step(qhfpe_batch_t *b, long n_steps, double *const *trace_out);
/* Tile height (q rows per block) the batch runs with (0 before the first step). */
qhfpe_status qhfpe_batch_tile_rows(const qhfpe_batch_t *b, int *rows);
qhfpe_status qhfpe_batch_destroy(qhfpe_batch_t *b);

/* Dipole super-operator on every hierarchy element of the listed replicas (replicas = NULL: all),
 * Sec. III (Condon: mu constant, so the p-convolution with mu(p, q) is a product). */
qhfpe_status qhfpe_apply_dipole(qhfpe_t *h, int side, const int *replicas, int n);

/* out (host complex128, canonical layout of one replica) = selected terms of the right-hand side of
 * Eq. (heom) evaluated on replica `replica`, in the handle's arithmetic. */
qhfpe_status qhfpe_apply_rhs(qhfpe_t *h, int replica, int terms, double *out);

/* Tr{mu W^(0)} of every replica now: host complex128 [n_replicas]. */
qhfpe_status qhfpe_trace(qhfpe_t *h, double *out);

/* Coordinate-dependent (non-Condon) dipole, Sec. III: "a non-Condon dipolar interaction can be
 * included"; the dipole super-operators are the p-convolutions
 *   (mu^-> W)_jk = sum_l mu_jl(p, q) * W_lk,   (mu^<- W)_jk = sum_l mu*_lk(p, q) * W_jl,
 *   mu_jk(p, q) = (1 / 2 pi hbar) int dr e^{-i p r / hbar} mu_jk(q + r/2),
 * which on the grid are circulants along p: after an FFT along p, products with mu_jl(q_i + r_m/2) and
 * mu_lk(q_i - r_m/2) at the r-grid modes (Nyquist mode: the symmetric value, as for the potential).
 * The trace Tr{mu W^(0)} weights W_jk(q_i, p) with mu_kj(q_i).  mu_table: host, [S][S][nq][np+1] in the
 * U_table convention (mu_jk(q_i + s_t)), real and symmetric in (j, k); copied.  NULL restores the
 * Condon dipole of qhfpe_params.mu.  Applies to every later dipole application and trace of the handle
 * (qhfpe_apply_dipole, qhfpe_step traces, qhfpe_response, qhfpe_first_order_distribution); the mixed
 * forms apply it to their FP64 zeroth tier in FP64.  Errors: QHFPE_EUNSUPPORTED unless np is 32, 64,
 * 128 or 256 and S <= 3; QHFPE_EINVAL for non-finite or non-symmetric tables. */
qhfpe_status qhfpe_set_dipole_table(qhfpe_t *h, const double *mu_table);

/* Adiabatic-basis wavepacket marginals, Sec. III ("Wavepacket dynamics"): for replica `replica`,
 *   out[a][b][i] = sum_jk V_ja(q_i) V_kb(q_i) dp sum_l W^(0)_jk(q_i, p_l),
 * the coordinate marginal of the zeroth-tier Wigner distribution (the reduced density matrix on its
 * diagonal q = q') in the adiabatic basis.  V(q_i) holds the eigenvectors of the real symmetric
 * diabatic matrix U_jk(q_i) (the U_table column of zero offset, t = np/2), ordered by ascending
 * eigenvalue (a = 0 is the lowest adiabatic surface); each is signed so that its first component of
 * largest magnitude (within 1e-9) is positive.  Because the rotation is local in q it is exact for the
 * coordinate marginal.  out: host complex128 [S][S][nq] (re, im interleaved).  FP64 sums in a fixed
 * order on the device; the mixed forms use their FP64 zeroth tier.  Errors: QHFPE_EINVAL for a bad
 * replica or NULL output. */
qhfpe_status qhfpe_adiabatic_marginals(qhfpe_t *h, int replica, double *out);

/* First-order perturbed Wigner distributions in the frequency domain, Sec. III (W'(omega_1), used for
 * the 1D and 2D correlation spectra; W''(t2, omega_1) = G(t2) i [W'(omega_1) + W'(-omega_1)] follows from
 * two of them):
 *   W'(omega) = i [ mu^-> F(omega) - mu^<- F(-omega) ],
 *   F(omega)  = sum_a w_a e^{i omega t_a} X(t_a),  X(t) = G(t) mu^x W_eq,  t_a = a t1_stride dt,
 * a = 0 .. n_t1 - 1, with the trapezoid weights of the two-dimensional spectrum's t1 sum
 * (w_a = dt1 / 2 at both ends, dt1 inside, all zero when n_t1 = 1).  Every hierarchy tier is returned.
 * The propagation runs in the handle's arithmetic on an internal one-replica batch from the
 * equilibrium state; the sums are FP64.  omega: host [n_omega].  out: host complex128
 * [n_omega][n_elem][S][S][nq][np].  Needs an equilibrium state (QHFPE_EINVAL otherwise); QHFPE_EINVAL
 * for n_t1 < 1, n_omega < 1, t1_stride < 1 with n_t1 > 1, NULL pointers or non-finite omega.
 * Allocates device memory for 4 n_omega + 1 canonical states for the duration of the call. */
qhfpe_status qhfpe_first_order_distribution(qhfpe_t *h, int n_t1, int t1_stride, const double *omega, int n_omega,
                                            double *out);

/* Equilibrium of Sec. III: the ground surface U_00 alone with the full hierarchy, started from the
 * classical Boltzmann distribution exp(-beta (p^2/2 + U_00(q))) normalised to unit trace, propagated
 * n_steps RK4 steps (FP64 always).  The result (ground block of every hierarchy element, all other
 * blocks zero) is kept as the handle's equilibrium state and written to every replica.
 * residual_out (may be NULL): ||L W|| / ||W|| of the final ground problem (2-norm, all elements). */
qhfpe_status qhfpe_equilibrate(qhfpe_t *h, long n_steps, double *residual_out);
/* The same equilibration run until it is stationary, Sec. III ("a sufficiently long time to obtain a
 * true thermal equilibrium state"): the residual ||L W|| / ||W|| of the ground problem is evaluated
 * before the first step and after every check_every steps (one right-hand side and two FP64 norms on
 * the device, two scalars to the host), and the propagation stops at the first check where it is
 * below tol, or when the steps reach t_max / dt (rounded to the nearest step).  steps_taken (may be
 * NULL): the RK4 steps propagated, a multiple of check_every unless t_max ended the run.
 * residual_out (may be NULL): the residual at the stop.  The result is that of qhfpe_equilibrate with
 * n_steps = *steps_taken.  Errors: EINVAL for t_max < 0 or not finite, tol <= 0, check_every < 1. */
qhfpe_status qhfpe_equilibrate_tol(qhfpe_t *h, double t_max, double tol, long check_every, long *steps_taken,
                                   double *residual_out);
/* Provide the equilibrium state directly (canonical layout, one replica). */
qhfpe_status qhfpe_set_equilibrium(qhfpe_t *h, const double *src, int is_device);

/* Response-function schedules (Eqs. (R1), (R3)); all delays are in steps of dt.
 *   QHFPE_LINEAR:     R1(c dt), c = 0..n_t3.  R_out: complex128 [n_t3 + 1].
 *   QHFPE_THIRD_ORDER: R3(c dt, t2[b] dt, a t1_stride dt), a < n_t1, b < n_t2, c <= n_t3.
 *                     R_out: complex128 [n_paths][n_t2][n_t1][n_t3 + 1] with n_paths = 2 when
 *                     split_pathways (first interaction mu^-> then -mu^<-; they add up to mu^x),
 *                     else 1.  Transient absorption is n_t1 = 1.
 * All propagations of one phase are packed as replicas of one batch and run by one captured CUDA
 * graph per phase. */
typedef enum { QHFPE_LINEAR = 0, QHFPE_THIRD_ORDER = 1 } qhfpe_response_kind;
typedef struct {
    int kind;
    int n_t1, t1_stride;
    int n_t2;
    const int *t2_steps;    /* host, ascending, n_t2 entries */
    int n_t3;
    int split_pathways;
} qhfpe_schedule;
qhfpe_status qhfpe_response(qhfpe_t *h, const qhfpe_schedule *sched, double *R_out);

/* Spectra by trapezoid Fourier-Laplace sums in FP64 on the device (host arrays in and out).
 * Absorption, Eq. (I1):  out[w] = omega_w Im sum_c w_c dt e^{i omega_w c dt} R1[c].
 * Two-dimensional, Eqs. (nonreph), (reph): R3 [n_t1][n_t3 + 1] for one waiting time;
 *   nr[w3][w1] = Im sum_a sum_c w_a w_c dt1 dt3 e^{i omega3 t3} e^{+i omega1 t1} R3,
 *   re[w3][w1] = same with e^{-i omega1 t1}; the correlation spectrum, Eq. (I3), is nr + re. */
qhfpe_status qhfpe_spectrum_absorption(qhfpe_t *h, const double *R1, long n_t, double dt,
                                       const double *omega, int n_omega, double *out);
qhfpe_status qhfpe_spectrum_2d(qhfpe_t *h, const double *R3, int n_t1, int n_t3, double dt1, double dt3,
                               const double *omega1, int n_omega1, const double *omega3, int n_omega3,
                               double *nr, double *re);

/* Kernel timing for measurement: when enabled, every launch of the right-hand-side stage kernels
 * (and the separate potential kernel, if the form has one) is bracketed by CUDA events on the
 * handle's stream.  read returns the launch count and total device milliseconds per kernel kind
 * (index 0: stage kernel, 1: potential kernel, 2: trace/auxiliary) and resets the counters. */
qhfpe_status qhfpe_kernel_timing(qhfpe_t *h, int enable);
/* Failure-detection self-test: a one-thread kernel waits on a device flag with the library's bounded
 * wait (%globaltimer limit of limit_ms milliseconds, 1..10000).  release = 1 sets the flag first
 * (returns QHFPE_OK); release = 0 leaves it unset, so the wait gives up and the call returns
 * QHFPE_ETIMEOUT while the handle and the CUDA context stay usable. */
qhfpe_status qhfpe_wait_selftest(qhfpe_t *h, int release, int limit_ms);
/* Tile of the fused right-hand-side kernel (q rows per block) picked by the autotuner for the
 * handle's replicas: timed with CUDA events on the first propagation (0 before it, or when the
 * shape has no fused kernel; candidates 1, 2, 3, 4, 5, 6, 8, 12, 16 rows up to the kernel's
 * shared-memory limit, a power of two, and the q-window form's fixed tile, see qhfpe_stage_form).
 * The environment variable QHFPE_TILE_ROWS, when it holds a height from 1 to that limit, replaces
 * the timing with that tile (the q-window form then serves the shapes it applies to). */
qhfpe_status qhfpe_tile_rows(const qhfpe_t *h, int *rows);
/* Persistent propagation (on = 1), Sec. III protocol on the device: every later run of RK4 steps of
 * the handle -- qhfpe_step and the propagations of qhfpe_response, whose phases pack all delays as
 * replicas -- runs as ONE cooperative launch that stays resident: each Horner stage is a grid-stride
 * loop over the blocks of the fused stage kernel, grid-wide barriers separate the stages, and the
 * FP64 trace Tr{mu W^(0)} is reduced in the same launch after each step (fixed order).  Results equal
 * those of the graph-replayed launches (on = 0, the default) to rounding of the trace sums (the state is
 * the same arithmetic).  It covers the shapes with a fused kernel (np in {32, 64, 128, 256}, n_states
 * <= 3), the FP64 and QHFPE_MIXED forms, the Condon dipole and the TRUNCATE / TERMINATOR closures; other
 * handles keep the graph replay.  Every barrier wait is bounded (2 s): when one gives up the call
 * returns QHFPE_ETIMEOUT and the handle turns sticky.  Kernel timing (qhfpe_kernel_timing) uses the
 * per-stage launches. */
qhfpe_status qhfpe_set_persistent(qhfpe_t *h, int on);
/* Failure-detection self-test of the persistent kernel's grid barrier: four blocks meet at one barrier
 * with the bounded wait (limit_ms, 1..10000); withhold = 1 keeps one block away, so the others give up
 * and the call returns QHFPE_ETIMEOUT while the handle and the CUDA context stay usable. */
qhfpe_status qhfpe_barrier_selftest(qhfpe_t *h, int withhold, int limit_ms);
/* Form of the fused right-hand-side kernel the autotuner picked for the handle's replicas, timed
 * together with the tile heights: 1 the q-window form (FP32 states with np = 128 and one or two
 * states, each warp one electronic pair and four q rows; candidate only where it applies), 0 the
 * general form; -1 before the first propagation or without a fused kernel.  QHFPE_FUSED_WINDOW=0
 * removes the q-window form from the candidates. */
qhfpe_status qhfpe_stage_form(const qhfpe_t *h, int *form);
qhfpe_status qhfpe_kernel_timing_read(qhfpe_t *h, long *launches, double *total_ms, int n_kinds);
/* Measurement aid with no counterpart in the paper: the FP64 fused multiply-add rate of the current
 * device, the denominator of the FP64 form's roofline.  8 blocks of 256 threads per SM each run eight
 * independent chains of 4096 x 8 DFMAs; the best of `repeats` (1..100) launches timed with CUDA events
 * on `stream` (NULL: legacy default stream) gives flops_per_s = 2 x DFMAs / time.  No clock or other
 * device setting is touched: the rate is at whatever clock the device runs.  Allocates and frees a
 * small output buffer.  Errors: EINVAL (bad repeats or NULL output), ECUDA. */
qhfpe_status qhfpe_fp64_fma_rate(void *stream, int repeats, double *flops_per_s);

/* ---- Learned closure (one Drude mode, K = 0) --------------------------------------------------
 * With closure = QHFPE_LEARNED the deepest tier's missing element W^(N+1) is the Eq. (GMFP)
 * terminator's estimate plus a learned local correction
 *   dW^(N+1) = sum_{b=-2..2} c_b(x) W^N(q, p_{l+b}) + c_{5+b}(x) W^(N-1)(q, p_{l+b})  (p periodic),
 * the ten coefficients coming from a perceptron of x = (q/8, p/8, ln eta): three tanh layers of
 * width 256 and a linear output of width 10.  Linear in the state, so the closed hierarchy keeps the
 * linear Green's function of Eqs. (R1), (R3).  Weights (float, row-major, this order):
 * W1[256][3], b1[256], W2[256][256], b2[256], W3[256][256], b3[256], W4[10][256], b4[10].
 * Until weights are loaded the correction is zero: the terminator.  QHFPE_TRUNCATE stays available
 * as the plain truncated hierarchy.
 * Regression statistics, per grid point (nq*np points, row-major [q][p]), 67 doubles: the upper
 * triangle (row-major) of G = sum Re(conj(phi) phi^T), h = sum Re(conj(phi) y), sum |y|^2, the number
 * of samples; phi = the ten patch values of tiers t-1 and t-2, y = tier t minus the terminator's
 * estimate (r_0 p + c_0 d/dp) W^(t-1) (4th-order central d/dp). */
#define QHFPE_CLOSURE_N_IN 3
#define QHFPE_CLOSURE_N_HIDDEN 256
#define QHFPE_CLOSURE_N_OUT 10
#define QHFPE_CLOSURE_N_WEIGHTS 135178
#define QHFPE_CLOSURE_N_STATS 67
/* The network's inputs on a grid (host, [nq*np][3] doubles, row-major [q][p]): (q_i / 8, p_l / 8, ln eta)
 * with the grid convention above; the same values the library's inference uses.  EINVAL for an empty
 * grid, eta <= 0 or a NULL output. */
qhfpe_status qhfpe_closure_inputs(int nq, int np, double q_min, double q_max, double p_min, double p_max, double eta,
                                  double *X);
/* Add the statistics of target tier t (1 <= t <= depth, n_matsubara = 0) over every replica's current
 * state to stats_dev (device, caller-owned, nq*np*67 doubles, accumulated into). */
qhfpe_status qhfpe_closure_collect(qhfpe_t *h, int target_tier, double *stats_dev);
/* Load weights (host, QHFPE_CLOSURE_N_WEIGHTS floats) and evaluate the network on the handle's grid at
 * its eta: bf16 weights and activations with FP32 accumulation in the mixed forms, FP32 in the FP64
 * form.  Requires closure = QHFPE_LEARNED. */
qhfpe_status qhfpe_closure_load(qhfpe_t *h, const float *weights, size_t n);
/* The coefficient table in use (host, [nq][np][10] doubles). */
qhfpe_status qhfpe_closure_coefficients(const qhfpe_t *h, double *out);
/* Training (FP32 kernels on the current device; the call allocates and frees its workspace).
 * X: host [n_points][3] network inputs; stats: host [n_points][67].  The loss is
 *   sum_x [c^T G_x c - 2 c^T h_x + yy_x + ridge (tr G_x / 10) |c|^2] / sum_x n_x
 * (the mean squared closure error over all samples plus a data-scaled ridge on the correction).
 * loss_grad: the loss and its gradient (float[N_WEIGHTS]).  train: n_iters Adam steps (beta1 0.9,
 * beta2 0.999, eps 1e-8) on minibatches of `batch` points drawn without replacement per epoch
 * (seeded), w updated in place; loss_history (may be NULL) gets each minibatch's estimate. */
qhfpe_status qhfpe_closure_loss_grad(const float *w, const double *X, const double *stats, int n_points,
                                     double ridge, double *loss, float *grad);
qhfpe_status qhfpe_closure_train(float *w, const double *X, const double *stats, int n_points, int n_iters,
                                 int batch, double lr, double ridge, unsigned seed, double *loss_history);

/* ---- State-input learned closure (the network reads the state; no counterpart in the paper) ------
 * With closure = QHFPE_LEARNED_STATE the deepest tier (one Drude mode, a chain) keeps the Eq. (GMFP)
 * terminator, d/dp (r_0 p W^(N)) + c_0 d2W^(N)/dp2, and adds d/dp D, where D is the missing element
 * W^(N+1) less the element the terminator stands for, r_0 p W^(N) + c_0 dW^(N)/dp (the derivatives the
 * stencils of the right-hand side: 4th-order central, periodic p).  D is predicted at every grid
 * point (q_i, p_l) by a perceptron of the state itself: inputs
 * (q_i / 8, p_l / 8, ln eta) followed by the 3 x 3 patches (q_{i+a}, p_{l+b}), a, b in {-1, 0, 1} (q: zero
 * outside the grid, or periodic; p periodic), of tiers N and N-1, pair by pair (j, k row-major), patch
 * row-major over (a, b), (re, im) innermost -- 36 S^2 + 3 values; three tanh layers of width 256 and a
 * linear output of 2 S^2 values, D_jk(q_i, p_l) (re, im) pair by pair.  The closed hierarchy is
 * nonlinear in the state, so the step is classic RK4 (four right-hand sides, FP64) and pathway
 * additivity no longer holds exactly.  Inference runs in every right-hand side with bf16 weights and
 * activations and FP32 accumulation.  Until weights are loaded D is zero (the terminator alone).  The
 * equilibrium (qhfpe_equilibrate) uses the Eq. (GMFP) terminator.  Weights (float):
 * W1[256][36 S^2 + 3], b1[256], W2[256][256], b2, W3[256][256], b3, W4[2 S^2][256], b4, then three scales
 * (tier-N inputs, tier-(N-1) inputs, outputs: the network sees the values divided by them) --
 * qhfpe_closure_state_n_weights(S) floats. */
size_t qhfpe_closure_state_n_weights(int n_states);
qhfpe_status qhfpe_closure_state_load(qhfpe_t *h, const float *weights, size_t n);
/* Training samples from the handle's current state (FP64, n_matsubara = 0, any closure): for every
 * replica and grid point, the inputs of the target tier t (1 <= t <= depth; tiers t-1, t-2, unscaled) into
 * X_dev [..][36 S^2 + 3] and the targets into Y_dev [..][2 S^2] (device, floats): the tier-t values less
 * r_0 p W^(t-1) + c_0 dW^(t-1)/dp (4th-order central along the periodic p axis), i.e. the D of a depth
 * t - 1 closure; starting at sample `offset`, at most up to `capacity`; count_out: samples written. */
qhfpe_status qhfpe_closure_state_collect(qhfpe_t *h, int target_tier, float *X_dev, float *Y_dev, long offset,
                                         long capacity, long *count_out);
/* The mean squared error over the n_points samples and all outputs, and its gradient (FP32 kernels),
 * for weights w (the scales are not used: X and Y as given).  grad: qhfpe_closure_state_n_weights(S) - 3
 * floats.  Host arrays. */
qhfpe_status qhfpe_closure_state_loss_grad(int n_states, const float *w, const float *X, const float *Y,
                                           int n_points, double *loss, float *grad);
/* Adam training (beta1 0.9, beta2 0.999, eps 1e-8, minibatches drawn without replacement per epoch,
 * seeded) on the samples scaled by the RMS of the tier-N inputs, of the tier-(N-1) inputs and of the
 * outputs; w (host, qhfpe_closure_state_n_weights(S) floats) updated in place, the three scales written
 * at its end; loss_history (may be NULL) gets each minibatch's mean squared error (scaled values). */
qhfpe_status qhfpe_closure_state_train(int n_states, float *w, const float *X, const float *Y, int n_points,
                                       int n_iters, int batch, double lr, unsigned seed, double *loss_history);

/* ---- Potential term without allocation -----------------------------------------------------
 * No counterpart in the paper: this entry point exists for callers that cannot allocate device
 * memory -- code whose device memory is a fixed budget owned by another allocator (an embedding
 * application or framework that hands out all of the GPU's memory itself), or code that must not
 * synchronise the device, which cudaMalloc/cudaFree may do.  It needs no handle.
 *
 * out_dev = -i [U, W] in Wigner space (the QHFPE_TERM_POTENTIAL part of qhfpe_apply_rhs, FP64) for
 * n_elem hierarchy elements of one state.  W_dev, out_dev: device, canonical complex128 layout
 * [n_elem][S][S][nq][np].  U_table_dev: device, [S][S][nq][np+1] as in qhfpe_params.  p_min, p_max:
 * the p range.  stream: cudaStream_t (NULL: legacy default stream); the call only enqueues work.
 *
 * Scratch: a file-scope device array of QHFPE_STATIC_SCRATCH_BYTES (32 MiB) that every GPU which loads
 * the library holds until the process exits.  Sizes with 7*S*S*nq*np + np doubles above that are
 * rejected with QHFPE_EINVAL (message in qhfpe_last_error(NULL)); larger n_elem is processed in chunks.
 * The first call on a device does a one-time set-up on that device (it looks up the array's device
 * address and raises a kernel attribute), so make the first call before any stream capture.  Every
 * call shares the one array: calls that overlap on the GPU race.  The call performs no cudaMalloc,
 * cudaFree or other allocation. */
#define QHFPE_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
qhfpe_status qhfpe_potential_term_static(int n_states, int nq, int np, double p_min, double p_max,
                                         const double *U_table_dev, int n_elem, const double *W_dev,
                                         double *out_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QHFPE_H */
