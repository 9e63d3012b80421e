// Internal declarations of the QHFPE CUDA library (kernels + host orchestration).
// Nothing here is part of the C ABI; see include/qhfpe.h for that.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <string>
#include <vector>

#define QH_MAX_MODES 8
#define QH_MAX_S 4

// Per hierarchy element: the couplings of Eq. (heom) with the linear-coupling operators of Sec. II.
//   tier-up   : + sum_k dW^(n+e_k)/dp                        (element up[k], or -1)
//   tier-down : + sum_k n_k gamma_k (r_k p + c_k d/dp) W^(n-e_k)   (element dn[k], weights wr, wc)
//   damping   : - (sum_k n_k gamma_k) W
//   terminator: at the deepest tier with the Eq. (GMFP) closure, d/dp (r_0 p W) + c_0 d2W/dp2 replaces
//               the missing tier-up term.
//   nonlinear coupling V(q) = q + c2 q^2 (GridInfo::c2 != 0): the mixed derivative
//               + wmx d2/dp dq W^(n-e_k) (element mx[a]) and the |m| = 2 couplings, terms of
//               phi d/dp W^(n-m) with weight w2 (element d2[a]), where phi = 1 + 2 c2 q
struct ElemInfo {
    int up[QH_MAX_MODES];
    int dn[QH_MAX_MODES];
    double wr[QH_MAX_MODES];
    double wc[QH_MAX_MODES];
    double ngam;
    int n_up, n_dn;
    int terminator;
    int tier;
    int mx[QH_MAX_MODES];
    double wmx[QH_MAX_MODES];
    int d2[QH_MAX_MODES];
    double w2[QH_MAX_MODES];
    int n_mx, n_d2;
};

// Geometry and bath scalars shared by every kernel of one propagator.
struct GridInfo {
    int S, nq, np, log2np;
    int n_elem, n_rep;
    int periodic_q;
    double q_min, p_min, dq, dp;
    double cdelta;     // delta-term coefficient
    double term_r0, term_c0;  // terminator coefficients (r_0, c_0)
    size_t blk;        // nq*np (one re or im plane of one (j,k) block)
    size_t elem_stride;    // S*S*2*blk reals per element
    size_t rep_stride;     // n_elem*elem_stride reals per replica
    size_t tier0_rep_stride;  // S*S*2*blk reals per replica in the FP64 tier-0 buffer
    int max_nb;        // most tier neighbours (up + down) of any element
    double c2;         // nonlinear system-bath coupling V(q) = q + c2 q^2 (0: linear)
};

// Potential-kernel tables in FFT output (bit-reversed) order, pre-scaled by 1/np:
//   D[j][k][i][pos]  = UL_jj(m) - UR_kk(m)          (coefficient of rho_jk)
//   L[j][s][i][pos]  = UL_js(m)  (used for s != j)   R[s][k][i][pos] = UR_sk(m)  (used for s != k)
// with m the r-grid mode sitting at FFT position pos.
template <typename T>
struct PotTables {
    const T *D, *L, *R;
    const T *tw;   // twiddles (cos, sin)(2 pi k / np), k < np/2, interleaved
};

// Tables of the fused stage kernel: same D, L, R as PotTables but in the fused FFT's
// digit-reversed order (fused_fft_frequency), np twiddles e^{2 pi i t/np}, t < np, and lpp: the
// eigenvalues of the periodic 5-point d2/dp2 stencil (without 1/(12 dp^2)) at each FFT position, over np.
template <typename T>
struct FusedTables {
    const T *D, *L, *R;
    const T *tw;
    const T *lpp;
};

// Scalars of one fused stage launch, rounded once on the host: 1/(12 dp), 1/(60 dq), the delta-term and
// terminator coefficients of the 5-point d2/dp2, r_0 and the Horner step h.
template <typename T>
struct StageScalars {
    T inv12dp, fkin, fdelta, fterm, r0, h;
};

// One member of a heterogeneous batch of fused stages (see launch_fused_multi): its grid and tables,
// its Horner buffers, and the number of its first block in the batch launch.
template <typename T>
struct MultiMember {
    GridInfo g;
    const ElemInfo *elems;
    FusedTables<T> tab;
    StageScalars<T> sc[5];  // [k]: stage k = 1..4 (h = dt / k); [0]: the right-hand side alone (h = 0)
    double dt;
    T *y, *vA, *vB;
    double *y0;             // FP64 zeroth tier (mixed form), else nullptr
    long block0;
};

// Device-side trace sink: trace kernel writes slot `counter` of every replica then the counter
// advances; keeps captured graphs independent of the call's output length.
struct TraceSink {
    double *base;   // [n_rep][stride] complex
    long stride;    // complex numbers per replica
    long counter;
    int done;       // blocks of the running reduction that have finished (0 between launches)
};

enum { QH_KIND_STAGE = 0, QH_KIND_POT = 1, QH_KIND_AUX = 2, QH_KINDS = 3 };

// ---- launchers (qhfpe_kernels.cu) -----------------------------------------------------------------
template <typename T>
cudaError_t launch_potential(const GridInfo &g, const PotTables<T> &tab, const T *v, T *P, int rep0, int n_rep,
                             cudaStream_t st);

template <typename T, bool MIXED>
cudaError_t launch_stage(const GridInfo &g, const ElemInfo *elems, const T *v_in, const T *P, const T *y,
                         const double *y0, T *v_out, double *y0_out, double h, int mode, int terms,
                         int rep0, int n_rep, cudaStream_t st);

// partial: device scratch of 2 * n_rep * QH_TRACE_MAX_CHUNKS doubles
#define QH_TRACE_MAX_CHUNKS 64
template <typename T>
// mu_q: non-Condon dipole at the grid points, [nq][S][S] (nullptr: the constant mu_dev)
cudaError_t launch_trace(const GridInfo &g, const T *state, size_t rep_stride, const double *mu_dev,
                         TraceSink *sink, int advance, double *partial, cudaStream_t st,
                         const double *mu_q = nullptr);

cudaError_t launch_advance(TraceSink *sink, cudaStream_t st);
cudaError_t prepare_potential(size_t smem_bytes_fp64);

// ---- fused stage (qhfpe_fused.cu) -------------------------------------------------------------------
bool fused_supported(int np, int S);
int fused_rows_per_tile(int np, int S, int elem_bytes);
size_t fused_smem_bytes(int tq, int np, int S, int elem_bytes);
int fused_fft_frequency(int np, int pos);
// Pg: potential term computed elsewhere (same layout as v_in), or nullptr to compute it in the kernel.
// tq: q rows per block (0: the default heuristic), at most fused_max_rows.
// form: -1 the q-window kernel where it applies (fused_window_applies), 0 always fused_stage_kernel,
// 1 the q-window kernel where it applies (the autotuner's choice).
template <typename T, bool MIXED>
cudaError_t launch_fused(const GridInfo &g, const ElemInfo *elems, const FusedTables<T> &tab, const T *v_in,
                         const T *y, const double *y0, T *v_out, double *y0_out, double h, int mode, int terms,
                         int rep0, int n_rep, cudaStream_t st, const T *Pg = nullptr, int tq = 0, int form = -1);
// The q-window form of the fused stage kernel (FP32, np 128, one or two states, every term with the
// potential in the kernel, lanes of one p sign, at most six tier neighbours, linear coupling), unless
// QHFPE_FUSED_WINDOW=0; its q rows per block.
bool fused_window_applies(const GridInfo &g, int terms, bool have_pg);
int fused_window_rows(int S);
int fused_max_rows(int np, int S, int elem_bytes);
template <typename T>
StageScalars<T> stage_scalars(const GridInfo &g, double h);
// blocks of one fused launch over all replicas at tile height tq
long fused_blocks(const GridInfo &g, int tq);
// Horner stage k (4..1; 0: the right-hand side into vB) of every member of mem (device array, n_mem
// members sharing np and S, block0 ascending from 0, blocks in total) as one launch; nonlinear: some
// member has c2 != 0 (the instantiation with those terms).
template <typename T, bool MIXED>
cudaError_t launch_fused_multi(int np, int S, const MultiMember<T> *mem, int n_mem, int k, int tq, long blocks,
                               bool nonlinear, cudaStream_t st);
// shared-memory limit of the batch instantiation (called by prepare_fused)
template <typename T, bool MIXED>
cudaError_t prepare_fused_multi(int np, int S, size_t smem);
// The single-model stage with the nonlinear coupling's terms compiled in (qhfpe_fused_nl.cu; launch_fused
// takes it when GridInfo::c2 != 0), and its shared-memory limit (called by prepare_fused).
template <typename T, bool MIXED>
cudaError_t launch_fused_nl(const GridInfo &g, const ElemInfo *elems, const FusedTables<T> &tab, const T *v_in,
                            const T *y, const double *y0, T *v_out, double *y0_out, double h, int mode, int terms,
                            int rep0, int n_rep, cudaStream_t st, const T *Pg, int tq);
template <typename T, bool MIXED>
cudaError_t prepare_fused_nl(int np, int S);
// Non-Condon dipole super-operator (side 1: mu^->, 2: mu^<-, 3: mu^x, times scale) on n_elem elements of
// n_rep replicas (reps: device list or nullptr for 0..n_rep-1), in place, through an FFT along p.
// TL, TR: [S][S][nq][np] r-space multipliers mu(q + r/2), mu(q - r/2) / np in the fused FFT's order;
// tw: its np twiddles.  mirror: FP32 copy to update as well (nullptr: none).  np in {32..256}, S <= 3.
template <typename T>
cudaError_t launch_dipole_fft(const GridInfo &g, const T *TL, const T *TR, const T *tw, T *state, size_t rep_stride,
                              int n_elem, const int *reps, int n_rep, int side, double scale, float *mirror,
                              size_t mirror_rep_stride, cudaStream_t st);

// ---- persistent propagation (qhfpe_persistent.cu) ---------------------------------------------------------
// n_steps RK4 steps of the one-member batch `mem` (device, block0 = 0) in one cooperative launch: every
// Horner stage a grid-stride loop over the n_items blocks of a fused stage launch at tile height tq,
// grid barriers between stages (bar_words: two zeroed words, count and generation; *err set to 1 when a
// wait exceeded limit_ns).  trace_out (device, may be nullptr): Tr{mu W^(0)} of every replica after
// each step into slots slot0 .. slot0 + n_steps - 1 of [n_rep][trace_stride] complex, from the FP64
// trace_state (Condon mu), chunk partials in `partial` ([n_rep][n_chunks][2]).  nonlinear: the member has
// c2 != 0 (the instantiation with those terms).
template <typename T, bool MIXED>
cudaError_t launch_persistent(int np, int S, const MultiMember<T> *mem, long n_items, int tq, int n_steps,
                              const double *trace_state, size_t trace_rep_stride, const double *mu, double *partial,
                              int n_chunks, double *trace_out, long trace_stride, long slot0, unsigned *bar_words,
                              int *err, unsigned long long limit_ns, bool nonlinear, cudaStream_t st);
// The barrier alone on four one-warp blocks; withhold = 1 keeps block 0 away, so the others give up.
cudaError_t launch_barrier_selftest(unsigned *bar_words, int *err, unsigned long long limit_ns, int withhold,
                                    cudaStream_t st);
int trace_chunks(int n_rep, size_t blk);

// ---- tensor-core potential term (qhfpe_tc.cu) ----------------------------------------------------------
bool tc_supported(int np, int S);
cudaError_t prepare_tc(int np, int S);
// tD/tL/tR: FP32 potential tables in natural mode order [pair][i][m]; bmat: build_tc_matrices output
cudaError_t launch_potential_tc(const GridInfo &g, const float *v, float *P, const void *bmat, const float *tD,
                                const float *tL, const float *tR, int n_rep, int *err, cudaStream_t st);
void build_tc_matrices(int np, std::vector<uint16_t> &out);
template <typename T, bool MIXED>
cudaError_t prepare_fused(int np, int S);

// ---- learned closure (qhfpe_closure.cu) ---------------------------------------------------------------
template <typename T>
cudaError_t launch_closure_apply(const GridInfo &g, T *state, int e_n, int e_n1, int e_slot, const T *coef, int rep0,
                                 int n_rep, cudaStream_t st);
template <typename T>
cudaError_t launch_closure_collect(const GridInfo &g, const T *state, int e_t, int e_t1, int e_t2, double *stats,
                                   cudaStream_t st);
cudaError_t launch_closure_infer(const GridInfo &g, double eta, const float *w_dev, int bf16, double *out64,
                                 float *out32, cudaStream_t st);

// State-input closure (qhfpe_closure.cu): weights per S; fill the W^(N+1) slot of `state` from tiers
// e_n, e_n1 of replicas rep0 .. rep0 + n_rep - 1; training samples of the tier e_t from e_t1, e_t2.
size_t closure_state_n_weights(int S);
// the fill reads w = the weights followed, at closure_state_prepared_offset(S) floats, by the
// closure_state_prepared_floats(S) that launch_closure_state_prepare writes from them
size_t closure_state_prepared_offset(int S);
size_t closure_state_prepared_floats(int S);
cudaError_t launch_closure_state_prepare(int S, const float *w, float *wt, cudaStream_t st);
template <typename T>
cudaError_t launch_closure_state_fill(const GridInfo &g, T *state, int e_n, int e_n1, int e_slot, const float *w,
                                      double eta, int rep0, int n_rep, cudaStream_t st);
template <typename T>
cudaError_t launch_closure_state_collect(const GridInfo &g, const T *state, int e_t, int e_t1, int e_t2, double eta,
                                         float *X, float *Y, long offset, long capacity, cudaStream_t st);
// classic RK4 combination over n values: first: acc = y + a_acc k; else acc += a_acc k; then v = y + a_v k;
// last: y = acc + a_acc k (v untouched)
cudaError_t launch_rk4_combine(size_t n, double *y, const double *k, double *acc, double *v, double a_acc, double a_v,
                               int first, int last, cudaStream_t st);

// Error text for calls without a handle (failed create, the static-scratch entry point).
void qh_set_free_error(const std::string &msg);

template <typename T>
cudaError_t launch_dipole(const GridInfo &g, T *state, double *y0, const int *reps, int n_reps,
                          const double *mu_dev, int side, double scale, cudaStream_t st);

// canonical layout [elem][j][k][q][p] complex with host element type H (double or float)
template <typename T, typename H = double>
cudaError_t launch_from_canonical(const GridInfo &g, const H *src, T *dst, double *y0_dst, int rep, int n_rep,
                                  cudaStream_t st, int *nonfinite = nullptr);
template <typename T, typename H = double>
cudaError_t launch_to_canonical(const GridInfo &g, const T *src, const double *y0_src, H *dst, int rep,
                                cudaStream_t st);

// Adiabatic-basis coordinate marginals of one replica's zeroth tier (FP64, layout [S][S][re|im][q][p]);
// V: [nq][S][S] eigenvector components; out: [S][S][nq] complex.
cudaError_t launch_marginals(const GridInfo &g, const double *tier0, const double *V, double *out, cudaStream_t st);
// W'(omega) of Sec. III: Fourier-weighted sums of canonical complex states (cs: [2][n_omega] weights of
// this sample) and the dipole combination i [mu^-> (A_c + i A_s) - mu^<- (A_c - i A_s)].
cudaError_t launch_fourier_accumulate(const double *x, size_t n, const double *cs, int n_omega, double *acc_c,
                                      double *acc_s, cudaStream_t st);
// out = (ar + i ai) a + (br + i bi) b for n complex values (canonical states)
cudaError_t launch_complex_combine(const double *a, const double *b, double ar, double ai, double br, double bi,
                                   double *out, size_t n, cudaStream_t st);
cudaError_t launch_first_order_combine(int S, size_t blk, int n_elem, int n_omega, const double *mu,
                                       const double *acc_c, const double *acc_s, double *out, cudaStream_t st);
cudaError_t launch_norm2(const double *x, size_t n, double *out_dev, cudaStream_t st);
// DFMA throughput probe: blocks x 256 threads, each n_iter x 64 DFMAs; out: blocks * 256 doubles
cudaError_t launch_dfma_rate(int blocks, int n_iter, double *out, cudaStream_t st);
cudaError_t launch_wait_flag(const int *flag, unsigned long long limit_ns, int *status, cudaStream_t st);
cudaError_t launch_absorption(const double *R1, long n_t, double dt, const double *omega, int n_omega,
                              double *out, cudaStream_t st);
cudaError_t launch_spectrum2d(const double *R3, int n_t1, int n_t3, double dt1, double dt3, const double *omega1,
                              int n1, const double *omega3, int n3, double *nr, double *re, double *scratch,
                              cudaStream_t st);
