// SIMT kernels of the QHFPE library: right-hand side stages, FFT potential kernel, traces, dipoles,
// layout conversion and spectra.  Templated on the state's real type (double for the FP64 form,
// float for the mixed forms).
//
// State layout on the device ("internal"): [rep][elem][j][k][re|im][q][p] with p fastest, re and im in
// separate planes of nq*np reals.  The mixed forms also keep the zeroth tier in FP64:
// y0[rep][j][k][re|im][q][p].
#include "qhfpe_internal.cuh"

#include <algorithm>
#include <cstdint>
#include <mutex>

namespace {

constexpr int STAGE_THREADS = 256;
constexpr int POT_THREADS = 128;

__device__ __forceinline__ int wrap(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// ---------------------------------------------------------------------------------------------------
// Right-hand side of Eq. (heom) (linear coupling, Sec. II) at one cell, fused with the Horner update of
// the degree-4 Taylor / RK4 step: v_out = base + h * L(v_in).  The potential term comes precomputed in P
// (same layout as v_in).  mode 0: v_out = L(v_in) (diagnostics); 1: Horner stage; 2: final Horner
// stage (mixed forms also write the FP64 zeroth tier).
// ---------------------------------------------------------------------------------------------------
template <typename T, bool MIXED>
__global__ void __launch_bounds__(STAGE_THREADS)
stage_kernel(GridInfo g, const ElemInfo *__restrict__ elems, const T *__restrict__ v_in, const T *__restrict__ P,
             const T *y, const double *y0, T *v_out, double *y0_out, double h, int mode, int terms, int rep0,
             int tiles_per_block)
{
    const int S2 = g.S * g.S;
    const int bid = blockIdx.x / tiles_per_block;
    const int tile = blockIdx.x - bid * tiles_per_block;
    const int cell = tile * STAGE_THREADS + threadIdx.x;
    if (cell >= (int)g.blk) return;
    const int pair = bid % S2;
    const int e = (bid / S2) % g.n_elem;
    const int rep = rep0 + bid / (S2 * g.n_elem);
    const int np = g.np, nq = g.nq;
    const int l = cell & (np - 1);
    const int i = cell >> g.log2np;
    const size_t blk = g.blk;

    const size_t rep_off = (size_t)rep * g.rep_stride;
    const size_t pair_off = (size_t)pair * 2 * blk;
    const T *V = v_in + rep_off + (size_t)e * g.elem_stride + pair_off;

    const T p = (T)(g.p_min + l * g.dp);
    T acc_r = 0, acc_i = 0;

    // -p dW/dq, 5th-order upwind (Sec. III)
    if (terms & 1) {
        T sr = 0, si = 0;
        auto ld = [&](int ii, T c) {
            if (ii < 0 || ii >= nq) {
                if (!g.periodic_q) return;
                ii = ii < 0 ? ii + nq : ii - nq;
            }
            size_t o = (size_t)ii * np + l;
            sr += c * V[o];
            si += c * V[o + blk];
        };
        if (p < (T)0) {
            ld(i + 3, (T)2); ld(i + 2, (T)-15); ld(i + 1, (T)60); ld(i, (T)-20); ld(i - 1, (T)-30); ld(i - 2, (T)3);
        } else {
            ld(i + 2, (T)-3); ld(i + 1, (T)30); ld(i, (T)20); ld(i - 1, (T)-60); ld(i - 2, (T)15); ld(i - 3, (T)-2);
        }
        const T f = -p / (T)(60.0 * g.dq);
        acc_r += f * sr;
        acc_i += f * si;
    }
    // -i [U, W], precomputed by the potential kernel
    if (terms & 2) {
        size_t o = rep_off + (size_t)e * g.elem_stride + pair_off + cell;
        acc_r += P[o];
        acc_i += P[o + blk];
    }

    const ElemInfo &E = elems[e];
    const int lm2 = wrap(l - 2, np), lm1 = wrap(l - 1, np), lp1 = wrap(l + 1, np), lp2 = wrap(l + 2, np);
    const size_t row = (size_t)i * np;
    const T inv12dp = (T)(1.0 / (12.0 * g.dp));

    // damping and delta-term, plus the terminator's c_0 d2/dp2
    T cpp = 0;
    if (terms & 4) {
        const T c = V[row + l], ci = V[row + l + blk];
        acc_r -= (T)E.ngam * c;
        acc_i -= (T)E.ngam * ci;
        cpp += (T)g.cdelta;
    }
    const bool term = (terms & 8) && E.terminator;
    if (term) cpp += (T)g.term_c0;
    if (cpp != (T)0) {
        const T f = cpp * inv12dp / (T)g.dp;
        const T *Vr = V + row, *Vi = V + row + blk;
        acc_r += f * (-Vr[lm2] + (T)16 * Vr[lm1] - (T)30 * Vr[l] + (T)16 * Vr[lp1] - Vr[lp2]);
        acc_i += f * (-Vi[lm2] + (T)16 * Vi[lm1] - (T)30 * Vi[l] + (T)16 * Vi[lp1] - Vi[lp2]);
    }

    // d/dp of G = sum_up W^(n+e_k) + sum_dn n_k gamma_k c_k W^(n-e_k) [+ r_0 p W^n at the terminator],
    // plus p * sum_dn n_k gamma_k r_k W^(n-e_k)
    T g_r[5] = {0, 0, 0, 0, 0}, g_i[5] = {0, 0, 0, 0, 0};
    const int cols[5] = {lm2, lm1, l, lp1, lp2};
    bool have_g = false;
    const T *base_e0 = v_in + rep_off + pair_off;  // element 0 of this replica and pair
    if (terms & 8) {
        for (int a = 0; a < E.n_up; ++a) {
            const T *U = base_e0 + (size_t)E.up[a] * g.elem_stride + row;
            for (int t = 0; t < 5; ++t) {
                if (t == 2) continue;
                g_r[t] += U[cols[t]];
                g_i[t] += U[cols[t] + blk];
            }
            have_g = true;
        }
        if (term) {
            const T r0 = (T)g.term_r0;
            for (int t = 0; t < 5; ++t) {
                if (t == 2) continue;
                const T pc = (T)(g.p_min + cols[t] * g.dp);
                g_r[t] += r0 * pc * V[row + cols[t]];
                g_i[t] += r0 * pc * V[row + cols[t] + blk];
            }
            have_g = true;
        }
    }
    if (terms & 16) {
        T pr = 0, pi = 0;
        for (int a = 0; a < E.n_dn; ++a) {
            const T *D = base_e0 + (size_t)E.dn[a] * g.elem_stride + row;
            const T wc = (T)E.wc[a], wr = (T)E.wr[a];
            for (int t = 0; t < 5; ++t) {
                if (t == 2) continue;
                g_r[t] += wc * D[cols[t]];
                g_i[t] += wc * D[cols[t] + blk];
            }
            pr += wr * D[l];
            pi += wr * D[l + blk];
            have_g = true;
        }
        acc_r += p * pr;
        acc_i += p * pi;
    }
    if (have_g) {
        acc_r += inv12dp * (g_r[0] - (T)8 * g_r[1] + (T)8 * g_r[3] - g_r[4]);
        acc_i += inv12dp * (g_i[0] - (T)8 * g_i[1] + (T)8 * g_i[3] - g_i[4]);
    }

    const size_t o = rep_off + (size_t)e * g.elem_stride + pair_off + cell;
    if (mode == 0) {
        v_out[o] = acc_r;
        v_out[o + blk] = acc_i;
        return;
    }
    if (MIXED && e == 0) {
        const size_t o0 = (size_t)rep * g.tier0_rep_stride + pair_off + cell;
        const double nr = y0[o0] + h * (double)acc_r;
        const double ni = y0[o0 + blk] + h * (double)acc_i;
        v_out[o] = (T)nr;
        v_out[o + blk] = (T)ni;
        if (mode == 2) {
            y0_out[o0] = nr;
            y0_out[o0 + blk] = ni;
        }
        return;
    }
    const T hh = (T)h;
    const T br = y[o], bi = y[o + blk];
    v_out[o] = br + hh * acc_r;
    v_out[o + blk] = bi + hh * acc_i;
}

// ---------------------------------------------------------------------------------------------------
// Potential kernel, Eq. (quantum-liouvillian): for one (replica, element, q row), all S*S blocks.
// In r-space (the density matrix rho(q + r/2, q - r/2), Sec. II) the commutator is local:
//   -i [ sum_s U_js(q + r/2) rho_sk - sum_s rho_js U_sk(q - r/2) ],
// so: forward FFT along p of every block (sign +), the S x S mixing per mode, inverse FFT (sign -).
// Radix-2 Gentleman-Sande forward leaves modes in bit-reversed order; the tables are stored in that
// order and the Cooley-Tukey inverse takes bit-reversed input, so no permutation pass is needed.
// ---------------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void fft_forward_dif(T *re, T *im, int log2N, const T *__restrict__ tw, int lane)
{
    const int N = 1 << log2N;
    for (int s = log2N - 1; s >= 0; --s) {
        const int h = 1 << s;
        for (int b = lane; b < (N >> 1); b += 32) {
            const int grp = b >> s, j = b & (h - 1);
            const int i0 = (grp << (s + 1)) + j, i1 = i0 + h;
            const T ar = re[i0], ai = im[i0], cr = re[i1], ci = im[i1];
            re[i0] = ar + cr;
            im[i0] = ai + ci;
            const T dr = ar - cr, di = ai - ci;
            const int t = j << (log2N - 1 - s);
            const T wr = tw[2 * t], wi = tw[2 * t + 1];
            re[i1] = dr * wr - di * wi;
            im[i1] = dr * wi + di * wr;
        }
        __syncwarp();
    }
}

template <typename T>
__device__ __forceinline__ void fft_inverse_dit(T *re, T *im, int log2N, const T *__restrict__ tw, int lane)
{
    const int N = 1 << log2N;
    for (int s = 0; s < log2N; ++s) {
        const int h = 1 << s;
        for (int b = lane; b < (N >> 1); b += 32) {
            const int grp = b >> s, j = b & (h - 1);
            const int i0 = (grp << (s + 1)) + j, i1 = i0 + h;
            const int t = j << (log2N - 1 - s);
            const T wr = tw[2 * t], wi = -tw[2 * t + 1];
            const T xr = re[i1] * wr - im[i1] * wi;
            const T xi = re[i1] * wi + im[i1] * wr;
            const T ar = re[i0], ai = im[i0];
            re[i1] = ar - xr;
            im[i1] = ai - xi;
            re[i0] = ar + xr;
            im[i0] = ai + xi;
        }
        __syncwarp();
    }
}

template <typename T>
__global__ void __launch_bounds__(POT_THREADS)
pot_kernel(GridInfo g, PotTables<T> tab, const T *__restrict__ v, T *__restrict__ P, int rep0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int S = g.S, S2 = S * S, N = g.np, nq = g.nq;
    T *bin = reinterpret_cast<T *>(smem_raw);  // [S2][2][N]
    T *bout = bin + (size_t)S2 * 2 * N;        // [S2][2][N]
    const int row = blockIdx.x;
    const int i = row % nq;
    const int e = (row / nq) % g.n_elem;
    const int rep = rep0 + row / (nq * g.n_elem);
    const size_t blk = g.blk;
    const size_t ebase = (size_t)rep * g.rep_stride + (size_t)e * g.elem_stride + (size_t)i * N;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

    for (int idx = tid; idx < S2 * 2 * N; idx += blockDim.x) {
        const int pr = idx / (2 * N), c = (idx / N) & 1, l = idx & (N - 1);
        bin[idx] = v[ebase + (size_t)pr * 2 * blk + (size_t)c * blk + l];
    }
    __syncthreads();
    for (int pr = warp; pr < S2; pr += nwarps) fft_forward_dif(bin + pr * 2 * N, bin + pr * 2 * N + N, g.log2np, tab.tw, lane);
    __syncthreads();
    for (int pos = tid; pos < N; pos += blockDim.x) {
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < S; ++k) {
                const size_t trow = (size_t)i * N + pos;
                const T d = tab.D[((size_t)(j * S + k) * nq) * N + trow];
                const T *rjk = bin + (j * S + k) * 2 * N;
                T ar = d * rjk[pos], ai = d * rjk[N + pos];
                for (int s = 0; s < S; ++s) {
                    if (s != j) {
                        const T u = tab.L[((size_t)(j * S + s) * nq) * N + trow];
                        const T *r = bin + (s * S + k) * 2 * N;
                        ar += u * r[pos];
                        ai += u * r[N + pos];
                    }
                    if (s != k) {
                        const T u = tab.R[((size_t)(s * S + k) * nq) * N + trow];
                        const T *r = bin + (j * S + s) * 2 * N;
                        ar -= u * r[pos];
                        ai -= u * r[N + pos];
                    }
                }
                // times -i
                T *o = bout + (j * S + k) * 2 * N;
                o[pos] = ai;
                o[N + pos] = -ar;
            }
    }
    __syncthreads();
    for (int pr = warp; pr < S2; pr += nwarps) fft_inverse_dit(bout + pr * 2 * N, bout + pr * 2 * N + N, g.log2np, tab.tw, lane);
    __syncthreads();
    for (int idx = tid; idx < S2 * 2 * N; idx += blockDim.x) {
        const int pr = idx / (2 * N), c = (idx / N) & 1, l = idx & (N - 1);
        P[ebase + (size_t)pr * 2 * blk + (size_t)c * blk + l] = bout[idx];
    }
}

// ---------------------------------------------------------------------------------------------------
// Tr{mu W^(0)} = sum_jk mu_kj sum_il W^(0)_jk dq dp for every replica, FP64, in a fixed summation
// order (deterministic): pass 1 sums fixed chunks of cells per (replica, chunk) block into partials,
// pass 2 adds each replica's partials in chunk order, writes the sink slot and advances the counter.
// ---------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
trace_partial_kernel(GridInfo g, const T *__restrict__ state, size_t rep_stride, const double *__restrict__ mu,
                     const double *__restrict__ mu_q, double *partial, int n_chunks)
{
    __shared__ double red[2][256];
    // programmatic dependent launch (no-ops for a plain launch): let the next kernel be scheduled, then
    // wait for the stage that wrote the state
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int chunk = blockIdx.x, rep = blockIdx.y;
    const int S = g.S;
    const size_t blk = g.blk;
    const size_t len = (blk + n_chunks - 1) / n_chunks;
    const size_t c0 = (size_t)chunk * len, c1 = c0 + len < blk ? c0 + len : blk;
    const T *W = state + (size_t)rep * rep_stride;
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < S; ++j)
        for (int k = 0; k < S; ++k) {
            const T *b = W + (size_t)(j * S + k) * 2 * blk;
            if (mu_q) {  // non-Condon: the Wigner function of mu(q) is mu_kj(q_i) at every p of row i
                for (size_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
                    const double m = mu_q[(c / g.np) * S * S + k * S + j];
                    sr += m * (double)b[c];
                    si += m * (double)b[c + blk];
                }
                continue;
            }
            const double m = mu[k * S + j];
            if (m == 0.0) continue;
            double ar = 0.0, ai = 0.0;
            for (size_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
                ar += (double)b[c];
                ai += (double)b[c + blk];
            }
            sr += m * ar;
            si += m * ai;
        }
    red[0][threadIdx.x] = sr;
    red[1][threadIdx.x] = si;
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * ((size_t)rep * n_chunks + chunk)] = red[0][0];
        partial[2 * ((size_t)rep * n_chunks + chunk) + 1] = red[1][0];
    }
}

__global__ void trace_finish_kernel(GridInfo g, const double *__restrict__ partial, int n_chunks, TraceSink *sink,
                                    int advance)
{
    // one warp per replica, replicas spread over the blocks: lanes sum strided chunk partials, then a
    // fixed butterfly over the lanes (the same order on every call, so the result is reproducible bit
    // for bit)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the partials are complete
    const long slot = sink->counter;
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    const int n_warps = warps * gridDim.x;
    for (int rep = blockIdx.x * warps + (threadIdx.x >> 5); rep < g.n_rep; rep += n_warps) {
        double sr = 0.0, si = 0.0;
        for (int c = lane; c < n_chunks; c += 32) {
            sr += partial[2 * ((size_t)rep * n_chunks + c)];
            si += partial[2 * ((size_t)rep * n_chunks + c) + 1];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, off);
            si += __shfl_xor_sync(0xffffffffu, si, off);
        }
        if (lane == 0) {
            double *out = sink->base + 2 * ((size_t)rep * sink->stride + slot);
            out[0] = sr * g.dq * g.dp;
            out[1] = si * g.dq * g.dp;
        }
    }
    __syncthreads();
    // the last block to finish advances the slot; every block read it before taking its ticket
    if (threadIdx.x == 0 && atomicAdd(&sink->done, 1) == (int)gridDim.x - 1) {
        sink->done = 0;
        if (advance) sink->counter = slot + 1;
    }
}

__global__ void advance_kernel(TraceSink *sink) { sink->counter += 1; }

// ---------------------------------------------------------------------------------------------------
// Dipole super-operators (Sec. III, Condon): mu^-> W = mu W, mu^<- W = W mu, mu^x = mu^-> - mu^<-, on
// every hierarchy element of the listed replicas, in place; `scale` multiplies the result.
// ---------------------------------------------------------------------------------------------------
template <typename T>
__global__ void dipole_kernel(GridInfo g, T *state, double *y0, const int *__restrict__ reps, int n_reps,
                              const double *__restrict__ mu, int side, double scale)
{
    const size_t blk = g.blk;
    const size_t total = (size_t)n_reps * g.n_elem * blk;
    const int S = g.S;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t cell = idx % blk;
        const int e = (int)((idx / blk) % g.n_elem);
        const int ri = (int)(idx / (blk * g.n_elem));
        const int rep = reps ? reps[ri] : ri;
        const bool t0 = (y0 != nullptr) && e == 0;
        T *W = state + (size_t)rep * g.rep_stride + (size_t)e * g.elem_stride + cell;
        double *W0 = t0 ? y0 + (size_t)rep * g.tier0_rep_stride + cell : nullptr;
        double xr[QH_MAX_S * QH_MAX_S], xi[QH_MAX_S * QH_MAX_S];
        for (int a = 0; a < S * S; ++a) {
            if (t0) {
                xr[a] = W0[(size_t)a * 2 * blk];
                xi[a] = W0[(size_t)a * 2 * blk + blk];
            } else {
                xr[a] = (double)W[(size_t)a * 2 * blk];
                xi[a] = (double)W[(size_t)a * 2 * blk + blk];
            }
        }
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < S; ++k) {
                double lr = 0, li = 0, rr = 0, ri2 = 0;
                for (int l = 0; l < S; ++l) {
                    lr += mu[j * S + l] * xr[l * S + k];
                    li += mu[j * S + l] * xi[l * S + k];
                    rr += xr[j * S + l] * mu[l * S + k];
                    ri2 += xi[j * S + l] * mu[l * S + k];
                }
                double o_r = side == 1 ? lr : (side == 2 ? rr : lr - rr);
                double o_i = side == 1 ? li : (side == 2 ? ri2 : li - ri2);
                o_r *= scale;
                o_i *= scale;
                const size_t a = (size_t)(j * S + k) * 2 * blk;
                W[a] = (T)o_r;
                W[a + blk] = (T)o_i;
                if (t0) {
                    W0[a] = o_r;
                    W0[a + blk] = o_i;
                }
            }
    }
}

// canonical complex128 [elem][j][k][q][p]  <->  internal planar layout of one replica
template <typename T, typename H>
__global__ void from_canonical_kernel(GridInfo g, const H *__restrict__ src, T *dst, double *y0, int rep0,
                                      int *nonfinite)
{
    const size_t blk = g.blk;
    const size_t per = (size_t)g.n_elem * g.S * g.S * blk;
    const int rep = rep0 + blockIdx.y;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < per; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t cell = idx % blk;
        const size_t ep = idx / blk;  // e*S2 + pair
        const double re = (double)src[2 * idx], im = (double)src[2 * idx + 1];
        if (nonfinite && !(isfinite(re) && isfinite(im))) *nonfinite = 1;
        const size_t o = (size_t)rep * g.rep_stride + ep * 2 * blk + cell;
        dst[o] = (T)re;
        dst[o + blk] = (T)im;
        if (y0 && ep < (size_t)(g.S * g.S)) {
            const size_t o0 = (size_t)rep * g.tier0_rep_stride + ep * 2 * blk + cell;
            y0[o0] = re;
            y0[o0 + blk] = im;
        }
    }
}

// N consecutive floats or doubles (N x size a multiple of 16 bytes, 16-byte aligned) through 16-byte accesses
template <typename V, int N> __device__ __forceinline__ void ld16(const V *p, V *out)
{
    static_assert((N * sizeof(V)) % 16 == 0, "16-byte chunks");
#pragma unroll
    for (int c = 0; c < (int)(N * sizeof(V) / 16); ++c) {
        if constexpr (sizeof(V) == 4) {
            const float4 a = reinterpret_cast<const float4 *>(p)[c];
            out[4 * c] = a.x; out[4 * c + 1] = a.y; out[4 * c + 2] = a.z; out[4 * c + 3] = a.w;
        } else {
            const double2 a = reinterpret_cast<const double2 *>(p)[c];
            out[2 * c] = a.x; out[2 * c + 1] = a.y;
        }
    }
}
template <typename V, int N> __device__ __forceinline__ void st16(V *p, const V *in)
{
    static_assert((N * sizeof(V)) % 16 == 0, "16-byte chunks");
#pragma unroll
    for (int c = 0; c < (int)(N * sizeof(V) / 16); ++c) {
        if constexpr (sizeof(V) == 4)
            reinterpret_cast<float4 *>(p)[c] = make_float4(in[4 * c], in[4 * c + 1], in[4 * c + 2], in[4 * c + 3]);
        else
            reinterpret_cast<double2 *>(p)[c] = make_double2(in[2 * c], in[2 * c + 1]);
    }
}

// The same conversions four cells at a time (blk a multiple of 4, the canonical array 16-byte aligned):
// one thread reads four interleaved complex values and writes four values of each plane.
template <typename T, typename H>
__global__ void from_canonical4_kernel(GridInfo g, const H *__restrict__ src, T *dst, double *y0, int rep0,
                                       int *nonfinite)
{
    const size_t blk = g.blk, blk4 = blk / 4;
    const size_t per4 = (size_t)g.n_elem * g.S * g.S * blk4;
    const int rep = rep0 + blockIdx.y;
    bool bad = false;
    for (size_t qd = blockIdx.x * (size_t)blockDim.x + threadIdx.x; qd < per4; qd += (size_t)gridDim.x * blockDim.x) {
        const size_t ep = qd / blk4, cell = (qd - ep * blk4) * 4;
        H v[8];
        ld16<H, 8>(src + 2 * (ep * blk + cell), v);
        double re[4], im[4];
        T tr[4], ti[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            re[j] = (double)v[2 * j];
            im[j] = (double)v[2 * j + 1];
            bad = bad || !(isfinite(re[j]) && isfinite(im[j]));
            tr[j] = (T)re[j];
            ti[j] = (T)im[j];
        }
        const size_t o = (size_t)rep * g.rep_stride + ep * 2 * blk + cell;
        st16<T, 4>(dst + o, tr);
        st16<T, 4>(dst + o + blk, ti);
        if (y0 && ep < (size_t)(g.S * g.S)) {
            const size_t o0 = (size_t)rep * g.tier0_rep_stride + ep * 2 * blk + cell;
            st16<double, 4>(y0 + o0, re);
            st16<double, 4>(y0 + o0 + blk, im);
        }
    }
    if (bad && nonfinite) *nonfinite = 1;
}

template <typename T, typename H>
__global__ void to_canonical4_kernel(GridInfo g, const T *__restrict__ src, const double *__restrict__ y0, H *dst, int rep)
{
    const size_t blk = g.blk, blk4 = blk / 4;
    const size_t per4 = (size_t)g.n_elem * g.S * g.S * blk4;
    for (size_t qd = blockIdx.x * (size_t)blockDim.x + threadIdx.x; qd < per4; qd += (size_t)gridDim.x * blockDim.x) {
        const size_t ep = qd / blk4, cell = (qd - ep * blk4) * 4;
        double re[4], im[4];
        if (y0 && ep < (size_t)(g.S * g.S)) {
            const size_t o0 = (size_t)rep * g.tier0_rep_stride + ep * 2 * blk + cell;
            ld16<double, 4>(y0 + o0, re);
            ld16<double, 4>(y0 + o0 + blk, im);
        } else {
            const size_t o = (size_t)rep * g.rep_stride + ep * 2 * blk + cell;
            T tr[4], ti[4];
            ld16<T, 4>(src + o, tr);
            ld16<T, 4>(src + o + blk, ti);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                re[j] = (double)tr[j];
                im[j] = (double)ti[j];
            }
        }
        H v[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[2 * j] = (H)re[j];
            v[2 * j + 1] = (H)im[j];
        }
        st16<H, 8>(dst + 2 * (ep * blk + cell), v);
    }
}

template <typename T, typename H>
__global__ void to_canonical_kernel(GridInfo g, const T *__restrict__ src, const double *__restrict__ y0,
                                    H *dst, int rep)
{
    const size_t blk = g.blk;
    const size_t per = (size_t)g.n_elem * g.S * g.S * blk;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < per; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t cell = idx % blk;
        const size_t ep = idx / blk;
        double re, im;
        if (y0 && ep < (size_t)(g.S * g.S)) {
            const size_t o0 = (size_t)rep * g.tier0_rep_stride + ep * 2 * blk + cell;
            re = y0[o0];
            im = y0[o0 + blk];
        } else {
            const size_t o = (size_t)rep * g.rep_stride + ep * 2 * blk + cell;
            re = (double)src[o];
            im = (double)src[o + blk];
        }
        dst[2 * idx] = (H)re;
        dst[2 * idx + 1] = (H)im;
    }
}

__global__ void __launch_bounds__(1024) norm2_kernel(const double *__restrict__ x, size_t n, double *out)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) s += x[i] * x[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Eq. (I1) by the trapezoid rule: out[w] = omega Im sum_c wgt_c e^{i omega t_c} R1[c]
__global__ void absorption_kernel(const double *__restrict__ R1, long n_t, double dt, const double *__restrict__ omega,
                                  int n_omega, double *out)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_omega) return;
    const double om = omega[w];
    double acc = 0.0;
    for (long c = 0; c < n_t; ++c) {
        double s, co;
        sincos(om * (c * dt), &s, &co);
        const double wgt = (c == 0 || c == n_t - 1) ? 0.5 * dt : dt;
        acc += wgt * (s * R1[2 * c] + co * R1[2 * c + 1]);
    }
    out[w] = om * acc;
}

// Eqs. (nonreph), (reph): first the t3 transform G[w3][a], then the t1 transforms of both signs.
__global__ void spec2d_t3_kernel(const double *__restrict__ R3, int n_t1, int n_t3, double dt3,
                                 const double *__restrict__ omega3, int n3, double *G)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n3 * n_t1) return;
    const int w = idx / n_t1, a = idx % n_t1;
    const double om = omega3[w];
    const int nt = n_t3 + 1;
    double gr = 0.0, gi = 0.0;
    for (int c = 0; c < nt; ++c) {
        double s, co;
        sincos(om * (c * dt3), &s, &co);
        const double wgt = (c == 0 || c == nt - 1) ? 0.5 * dt3 : dt3;
        const double rr = R3[2 * ((size_t)a * nt + c)], ri = R3[2 * ((size_t)a * nt + c) + 1];
        gr += wgt * (co * rr - s * ri);
        gi += wgt * (s * rr + co * ri);
    }
    G[2 * idx] = gr;
    G[2 * idx + 1] = gi;
}

__global__ void spec2d_t1_kernel(const double *__restrict__ G, int n_t1, double dt1, const double *__restrict__ omega1,
                                 int n1, int n3, double *nr, double *re)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n3 * n1) return;
    const int w3 = idx / n1, w1 = idx % n1;
    const double om = omega1[w1];
    double an = 0.0, ar = 0.0;
    for (int a = 0; a < n_t1; ++a) {
        double s, co;
        sincos(om * (a * dt1), &s, &co);
        const double wgt = (n_t1 == 1) ? 0.0 : ((a == 0 || a == n_t1 - 1) ? 0.5 * dt1 : dt1);
        const double gr = G[2 * ((size_t)w3 * n_t1 + a)], gi = G[2 * ((size_t)w3 * n_t1 + a) + 1];
        // Im[e^{+i om t} G] and Im[e^{-i om t} G]
        an += wgt * (s * gr + co * gi);
        ar += wgt * (-s * gr + co * gi);
    }
    nr[idx] = an;
    re[idx] = ar;
}

// Bounded wait on a device flag (the pattern every device-side wait of the library follows): spin until
// *flag != 0 or `limit_ns` of %globaltimer have passed; status 1 = the flag arrived, 2 = gave up.
__global__ void wait_flag_kernel(const volatile int *flag, unsigned long long limit_ns, int *status)
{
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        if (*flag != 0) {
            *status = 1;
            return;
        }
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) {
            *status = 2;
            return;
        }
        __nanosleep(1000);
    }
}

// FP64 fused multiply-add throughput: every thread runs eight independent dependency chains of
// n_iter x 8 DFMAs (a = a * x + y); one result per thread is stored so nothing is dropped.
__global__ void __launch_bounds__(256) dfma_rate_kernel(double x, double y, int n_iter, double *out)
{
    double a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int it = 0; it < n_iter; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c) a[c] = fma(a[c], x, y);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

__global__ void rk4_combine_kernel(size_t n, double *y, const double *__restrict__ k, double *acc, double *v, double a_acc,
                                   double a_v, int first, int last)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double kv = k[i];
        if (last) {
            y[i] = acc[i] + a_acc * kv;
            continue;
        }
        const double yv = y[i];
        acc[i] = (first ? yv : acc[i]) + a_acc * kv;
        v[i] = yv + a_v * kv;
    }
}

inline int grid_for(size_t n, int threads, int cap = 152 * 32)
{
    size_t b = (n + threads - 1) / threads;
    if (b > (size_t)cap) b = cap;
    return (int)(b ? b : 1);
}

}  // namespace

// ----------------------------------------- launchers ----------------------------------------------
template <typename T>
cudaError_t launch_potential(const GridInfo &g, const PotTables<T> &tab, const T *v, T *P, int rep0, int n_rep,
                             cudaStream_t st)
{
    const size_t smem = (size_t)2 * g.S * g.S * 2 * g.np * sizeof(T);
    const int blocks = n_rep * g.n_elem * g.nq;
    if (blocks <= 0) return cudaSuccess;
    pot_kernel<T><<<blocks, POT_THREADS, smem, st>>>(g, tab, v, P, rep0);
    return cudaGetLastError();
}

template <typename T, bool MIXED>
cudaError_t launch_stage(const GridInfo &g, const ElemInfo *elems, const T *v_in, const T *P, const T *y,
                         const double *y0, T *v_out, double *y0_out, double h, int mode, int terms, int rep0,
                         int n_rep, cudaStream_t st)
{
    const int tiles = (int)((g.blk + STAGE_THREADS - 1) / STAGE_THREADS);
    const long blocks = (long)n_rep * g.n_elem * g.S * g.S * tiles;
    if (blocks <= 0) return cudaSuccess;
    stage_kernel<T, MIXED><<<(unsigned)blocks, STAGE_THREADS, 0, st>>>(g, elems, v_in, P, y, y0, v_out, y0_out, h, mode,
                                                                       terms, rep0, tiles);
    return cudaGetLastError();
}

int trace_chunks(int n_rep, size_t blk)
{
    int c = (int)((304 + n_rep - 1) / n_rep);  // about two blocks per SM in total
    if (c > QH_TRACE_MAX_CHUNKS) c = QH_TRACE_MAX_CHUNKS;
    if ((size_t)c > blk) c = (int)blk;
    return c < 1 ? 1 : c;
}

template <typename T>
cudaError_t launch_trace(const GridInfo &g, const T *state, size_t rep_stride, const double *mu_dev,
                         TraceSink *sink, int advance, double *partial, cudaStream_t st, const double *mu_q)
{
    const int nc = trace_chunks(g.n_rep, g.blk);
    // both launched with programmatic stream serialisation (each waits for its predecessor in-kernel)
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nc, g.n_rep);
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t err = cudaLaunchKernelEx(&cfg, trace_partial_kernel<T>, g, state, rep_stride, mu_dev, mu_q, partial, nc);
    if (err != cudaSuccess) return err;
    const int warps = 8;  // 256 threads, one warp per replica
    int nb = (g.n_rep + warps - 1) / warps;
    if (nb > 304) nb = 304;
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(32 * warps);
    return cudaLaunchKernelEx(&cfg, trace_finish_kernel, g, (const double *)partial, nc, sink, advance);
}

// Raises the dynamic shared-memory limit of the potential kernels; called at set-up, outside any
// stream capture.
// The limit only ever rises (per device), so a later, smaller request cannot undo a larger one.
cudaError_t prepare_potential(size_t smem_bytes_fp64)
{
    static std::mutex mtx;
    static size_t configured[64] = {0};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    std::lock_guard<std::mutex> lock(mtx);
    if (dev >= 0 && dev < 64 && configured[dev] >= smem_bytes_fp64) return cudaSuccess;
    err = cudaFuncSetAttribute(pot_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes_fp64);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(pot_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(smem_bytes_fp64 / 2));
    if (err == cudaSuccess && dev >= 0 && dev < 64) configured[dev] = smem_bytes_fp64;
    return err;
}

cudaError_t launch_advance(TraceSink *sink, cudaStream_t st)
{
    advance_kernel<<<1, 1, 0, st>>>(sink);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dipole(const GridInfo &g, T *state, double *y0, const int *reps, int n_reps,
                          const double *mu_dev, int side, double scale, cudaStream_t st)
{
    const size_t total = (size_t)n_reps * g.n_elem * g.blk;
    dipole_kernel<T><<<grid_for(total, 256), 256, 0, st>>>(g, state, y0, reps, n_reps, mu_dev, side, scale);
    return cudaGetLastError();
}

template <typename T, typename H>
cudaError_t launch_from_canonical(const GridInfo &g, const H *src, T *dst, double *y0_dst, int rep, int n_rep,
                                  cudaStream_t st, int *nonfinite)
{
    const size_t per = (size_t)g.n_elem * g.S * g.S * g.blk;
    if (g.blk % 4 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0) {
        dim3 grid(grid_for(per / 4, 256, 2048), n_rep);
        from_canonical4_kernel<T, H><<<grid, 256, 0, st>>>(g, src, dst, y0_dst, rep, nonfinite);
    } else {
        dim3 grid(grid_for(per, 256, 2048), n_rep);
        from_canonical_kernel<T, H><<<grid, 256, 0, st>>>(g, src, dst, y0_dst, rep, nonfinite);
    }
    return cudaGetLastError();
}

template <typename T, typename H>
cudaError_t launch_to_canonical(const GridInfo &g, const T *src, const double *y0_src, H *dst, int rep,
                                cudaStream_t st)
{
    const size_t per = (size_t)g.n_elem * g.S * g.S * g.blk;
    if (g.blk % 4 == 0 && reinterpret_cast<uintptr_t>(dst) % 16 == 0)
        to_canonical4_kernel<T, H><<<grid_for(per / 4, 256, 2048), 256, 0, st>>>(g, src, y0_src, dst, rep);
    else
        to_canonical_kernel<T, H><<<grid_for(per, 256, 2048), 256, 0, st>>>(g, src, y0_src, dst, rep);
    return cudaGetLastError();
}

cudaError_t launch_wait_flag(const int *flag, unsigned long long limit_ns, int *status, cudaStream_t st)
{
    wait_flag_kernel<<<1, 1, 0, st>>>(flag, limit_ns, status);
    return cudaGetLastError();
}

cudaError_t launch_dfma_rate(int blocks, int n_iter, double *out, cudaStream_t st)
{
    dfma_rate_kernel<<<blocks, 256, 0, st>>>(0.999999, 1e-7, n_iter, out);
    return cudaGetLastError();
}

cudaError_t launch_rk4_combine(size_t n, double *y, const double *k, double *acc, double *v, double a_acc, double a_v,
                               int first, int last, cudaStream_t st)
{
    rk4_combine_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, y, k, acc, v, a_acc, a_v, first, last);
    return cudaGetLastError();
}

cudaError_t launch_norm2(const double *x, size_t n, double *out_dev, cudaStream_t st)
{
    norm2_kernel<<<1, 1024, 0, st>>>(x, n, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_absorption(const double *R1, long n_t, double dt, const double *omega, int n_omega,
                              double *out, cudaStream_t st)
{
    absorption_kernel<<<(n_omega + 127) / 128, 128, 0, st>>>(R1, n_t, dt, omega, n_omega, out);
    return cudaGetLastError();
}

cudaError_t launch_spectrum2d(const double *R3, int n_t1, int n_t3, double dt1, double dt3, const double *omega1,
                              int n1, const double *omega3, int n3, double *nr, double *re, double *scratch,
                              cudaStream_t st)
{
    spec2d_t3_kernel<<<(n3 * n_t1 + 127) / 128, 128, 0, st>>>(R3, n_t1, n_t3, dt3, omega3, n3, scratch);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    spec2d_t1_kernel<<<(n3 * n1 + 127) / 128, 128, 0, st>>>(scratch, n_t1, dt1, omega1, n1, n3, nr, re);
    return cudaGetLastError();
}

// Adiabatic-basis coordinate marginals of the zeroth tier (Sec. III, "Wavepacket dynamics"): one block
// per q row.  Warp w sums the p row of pairs jk = w, w + warps, ... in a fixed order (lanes over p,
// then a butterfly), so the result is reproducible; then S*S threads rotate the S x S marginal with
// the row's eigenvector matrix V[i][j][a].
__global__ void marginal_kernel(GridInfo g, const double *__restrict__ state, const double *__restrict__ V,
                                double *__restrict__ out)
{
    __shared__ double rho[2 * QH_MAX_S * QH_MAX_S];
    const int i = blockIdx.x, S = g.S, np = g.np;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    for (int jk = warp; jk < S * S; jk += n_warps) {
        const double *re = state + (size_t)(2 * jk) * g.blk + (size_t)i * np;
        const double *im = re + g.blk;
        double sr = 0.0, si = 0.0;
        for (int l = lane; l < np; l += 32) {
            sr += re[l];
            si += im[l];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, off);
            si += __shfl_xor_sync(0xffffffffu, si, off);
        }
        if (lane == 0) {
            rho[2 * jk] = sr * g.dp;
            rho[2 * jk + 1] = si * g.dp;
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < S * S) {
        const int a = threadIdx.x / S, b = threadIdx.x % S;
        const double *v = V + (size_t)i * S * S;  // v[j * S + a]: component j of adiabatic state a
        double pr = 0.0, pi = 0.0;
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < S; ++k) {
                const double w = v[j * S + a] * v[k * S + b];
                pr += w * rho[2 * (j * S + k)];
                pi += w * rho[2 * (j * S + k) + 1];
            }
        out[2 * ((size_t)(a * S + b) * g.nq + i)] = pr;
        out[2 * ((size_t)(a * S + b) * g.nq + i) + 1] = pi;
    }
}

cudaError_t launch_marginals(const GridInfo &g, const double *tier0, const double *V, double *out, cudaStream_t st)
{
    marginal_kernel<<<g.nq, 128, 0, st>>>(g, tier0, V, out);
    return cudaGetLastError();
}

// Fourier-weighted accumulation of canonical complex states (W'(omega) of Sec. III): for each of
// n_omega frequencies, acc_c[w] += cs[w] x and acc_s[w] += cs[n_omega + w] x, where cs holds this
// sample's trapezoid weight times dt times cos / sin(omega_w t).
__global__ void fourier_accumulate_kernel(const double *__restrict__ x, size_t n, const double *__restrict__ cs,
                                          int n_omega, double *acc_c, double *acc_s)
{
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const double xr = x[2 * idx], xi = x[2 * idx + 1];
        for (int w = 0; w < n_omega; ++w) {
            const double c = cs[w], s = cs[n_omega + w];
            acc_c[2 * ((size_t)w * n + idx)] += c * xr;
            acc_c[2 * ((size_t)w * n + idx) + 1] += c * xi;
            acc_s[2 * ((size_t)w * n + idx)] += s * xr;
            acc_s[2 * ((size_t)w * n + idx) + 1] += s * xi;
        }
    }
}

// W'(omega) = i [ mu^-> F(omega) - mu^<- F(-omega) ] with F(+-omega) = A_c +- i A_s, per frequency,
// hierarchy element and cell (canonical layout [elem][j][k][cell] complex, cell = q * np + p).
__global__ void first_order_combine_kernel(int S, size_t blk, int n_elem, int n_omega, const double *__restrict__ mu,
                                           const double *__restrict__ acc_c, const double *__restrict__ acc_s,
                                           double *__restrict__ out)
{
    const size_t per_elem = (size_t)S * S * blk, n = (size_t)n_elem * per_elem;
    const size_t total = (size_t)n_omega * n_elem * blk;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t c = t % blk, e = (t / blk) % n_elem, w = t / (blk * n_elem);
        const size_t base = w * n + e * per_elem + c;  // complex index of pair (0, 0)
        double pr[QH_MAX_S * QH_MAX_S], pi[QH_MAX_S * QH_MAX_S], mr[QH_MAX_S * QH_MAX_S], mi[QH_MAX_S * QH_MAX_S];
        for (int jk = 0; jk < S * S; ++jk) {
            const size_t o = 2 * (base + (size_t)jk * blk);
            const double cr = acc_c[o], ci = acc_c[o + 1], sr = acc_s[o], si = acc_s[o + 1];
            pr[jk] = cr - si;  // A_c + i A_s
            pi[jk] = ci + sr;
            mr[jk] = cr + si;  // A_c - i A_s
            mi[jk] = ci - sr;
        }
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < S; ++k) {
                double zr = 0.0, zi = 0.0;
                for (int l = 0; l < S; ++l) {
                    zr += mu[j * S + l] * pr[l * S + k] - mr[j * S + l] * mu[l * S + k];
                    zi += mu[j * S + l] * pi[l * S + k] - mi[j * S + l] * mu[l * S + k];
                }
                const size_t o = 2 * (base + (size_t)(j * S + k) * blk);
                out[o] = -zi;  // times i
                out[o + 1] = zr;
            }
    }
}

// out = (ar + i ai) a + (br + i bi) b over n complex values
__global__ void complex_combine_kernel(const double *__restrict__ a, const double *__restrict__ b, double ar, double ai,
                                       double br, double bi, double *__restrict__ out, size_t n)
{
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const double xr = a[2 * idx], xi = a[2 * idx + 1], yr = b[2 * idx], yi = b[2 * idx + 1];
        out[2 * idx] = ar * xr - ai * xi + br * yr - bi * yi;
        out[2 * idx + 1] = ar * xi + ai * xr + br * yi + bi * yr;
    }
}

cudaError_t launch_complex_combine(const double *a, const double *b, double ar, double ai, double br, double bi,
                                   double *out, size_t n, cudaStream_t st)
{
    const long blocks = (long)std::min<size_t>((n + 255) / 256, 152 * 16);
    complex_combine_kernel<<<(unsigned)std::max(blocks, 1L), 256, 0, st>>>(a, b, ar, ai, br, bi, out, n);
    return cudaGetLastError();
}

cudaError_t launch_fourier_accumulate(const double *x, size_t n, const double *cs, int n_omega, double *acc_c,
                                      double *acc_s, cudaStream_t st)
{
    const long blocks = (long)std::min<size_t>((n + 255) / 256, 152 * 16);
    fourier_accumulate_kernel<<<(unsigned)std::max(blocks, 1L), 256, 0, st>>>(x, n, cs, n_omega, acc_c, acc_s);
    return cudaGetLastError();
}

cudaError_t launch_first_order_combine(int S, size_t blk, int n_elem, int n_omega, const double *mu,
                                       const double *acc_c, const double *acc_s, double *out, cudaStream_t st)
{
    const size_t total = (size_t)n_omega * n_elem * blk;
    const long blocks = (long)std::min<size_t>((total + 255) / 256, 152 * 16);
    first_order_combine_kernel<<<(unsigned)std::max(blocks, 1L), 256, 0, st>>>(S, blk, n_elem, n_omega, mu, acc_c,
                                                                              acc_s, out);
    return cudaGetLastError();
}

// explicit instantiations
template cudaError_t launch_potential<double>(const GridInfo &, const PotTables<double> &, const double *, double *, int, int, cudaStream_t);
template cudaError_t launch_potential<float>(const GridInfo &, const PotTables<float> &, const float *, float *, int, int, cudaStream_t);
template cudaError_t launch_stage<double, false>(const GridInfo &, const ElemInfo *, const double *, const double *, const double *, const double *, double *, double *, double, int, int, int, int, cudaStream_t);
template cudaError_t launch_stage<float, true>(const GridInfo &, const ElemInfo *, const float *, const float *, const float *, const double *, float *, double *, double, int, int, int, int, cudaStream_t);
template cudaError_t launch_trace<double>(const GridInfo &, const double *, size_t, const double *, TraceSink *, int, double *, cudaStream_t, const double *);
template cudaError_t launch_dipole<double>(const GridInfo &, double *, double *, const int *, int, const double *, int, double, cudaStream_t);
template cudaError_t launch_dipole<float>(const GridInfo &, float *, double *, const int *, int, const double *, int, double, cudaStream_t);
template cudaError_t launch_from_canonical<double, double>(const GridInfo &, const double *, double *, double *, int, int, cudaStream_t, int *);
template cudaError_t launch_from_canonical<float, double>(const GridInfo &, const double *, float *, double *, int, int, cudaStream_t, int *);
template cudaError_t launch_from_canonical<double, float>(const GridInfo &, const float *, double *, double *, int, int, cudaStream_t, int *);
template cudaError_t launch_from_canonical<float, float>(const GridInfo &, const float *, float *, double *, int, int, cudaStream_t, int *);
template cudaError_t launch_to_canonical<double, double>(const GridInfo &, const double *, const double *, double *, int, cudaStream_t);
template cudaError_t launch_to_canonical<float, double>(const GridInfo &, const float *, const double *, double *, int, cudaStream_t);
template cudaError_t launch_to_canonical<double, float>(const GridInfo &, const double *, const double *, float *, int, cudaStream_t);
template cudaError_t launch_to_canonical<float, float>(const GridInfo &, const float *, const double *, float *, int, cudaStream_t);
