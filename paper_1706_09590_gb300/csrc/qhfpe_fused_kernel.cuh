// Fused right-hand-side stage: one launch evaluates the whole of Eq. (heom) (linear coupling, Sec. II)
// for a tile of TQ q-rows of one (replica, hierarchy element) -- all S x S electronic blocks, all p --
// and applies the Horner update of the RK4 step.
//
//   phase A  potential term, Eq. (quantum-liouvillian): the tile's p-rows are loaded into shared
//            memory, transformed by a two-pass in-place FFT (radix NP/16, then 16; sign +, digit-reversed
//            output), mixed per r-mode across the S x S blocks with the tables
//            D = UL_jj - UR_kk, L = UL_js, R = UR_sk (pre-scaled by 1/np, stored in the same
//            digit-reversed order), multiplied by -i, and transformed back (sign -, natural order).
//   phase B  one warp per p-row: upwind q-stencil (rows i-3..i+3 through L1/L2), damping and
//            delta-term, tier-up/-down couplings (neighbour elements' rows), terminator, the
//            potential term from shared memory, and out = base + h * L.
//
// Grid order: the hierarchy element varies fastest, then the replica, then the q-tile, so the blocks
// in flight cover all elements of a few q-tiles and the neighbour tiers and q-halos they re-read are
// L2-resident.
#pragma once
// (the fused stage kernel template; included by qhfpe_fused.cu, which instantiates the single-model
// kernel, and by qhfpe_fused_multi.cu, which instantiates the heterogeneous-batch kernel, so that the
// two compile in parallel)
#include "qhfpe.h"
#include "qhfpe_internal.cuh"

namespace {

constexpr int FTHREADS = 128;

template <typename T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename C> __device__ __forceinline__ C cconjmul(C a, C w) { return {a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y}; }
// multiply by s*i, s = +1 or -1
template <int SG, typename C> __device__ __forceinline__ C cmul_si(C a) { return SG > 0 ? C{-a.y, a.x} : C{a.y, -a.x}; }

// a + SG i b and a - SG i b
template <int SG, typename C> __device__ __forceinline__ C cadd_si(C a, C b) { return {a.x - SG * b.y, a.y + SG * b.x}; }
template <int SG, typename C> __device__ __forceinline__ C csub_si(C a, C b) { return {a.x + SG * b.y, a.y - SG * b.x}; }

// ---- packed FP32x2 arithmetic (sm_100 and later) ---------------------------------------------------
// An FP32 complex value occupies a register pair, so one packed instruction adds or subtracts both of
// its parts; the lanes' runs of consecutive p values pair up the same way.  Each component is rounded
// exactly as the scalar instruction would round it.  The FP64 form keeps scalar arithmetic.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// y += a x (a broadcast), y += u x (elementwise), y += x over N values
template <int N> __device__ __forceinline__ void v_axpy(float *y, float a, const float *x)
{
    if constexpr (N % 2 == 0) {
        const float2 a2 = make_float2(a, a);
#pragma unroll
        for (int v = 0; v < N; v += 2) {
            const float2 r = __ffma2_rn(a2, make_float2(x[v], x[v + 1]), make_float2(y[v], y[v + 1]));
            y[v] = r.x;
            y[v + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int v = 0; v < N; ++v) y[v] = fmaf(a, x[v], y[v]);
    }
}
template <int N> __device__ __forceinline__ void v_axpy(double *y, double a, const double *x)
{
#pragma unroll
    for (int v = 0; v < N; ++v) y[v] = fma(a, x[v], y[v]);
}
template <int N> __device__ __forceinline__ void v_fma(float *y, const float *u, const float *x)
{
    if constexpr (N % 2 == 0) {
#pragma unroll
        for (int v = 0; v < N; v += 2) {
            const float2 r = __ffma2_rn(make_float2(u[v], u[v + 1]), make_float2(x[v], x[v + 1]), make_float2(y[v], y[v + 1]));
            y[v] = r.x;
            y[v + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int v = 0; v < N; ++v) y[v] = fmaf(u[v], x[v], y[v]);
    }
}
template <int N> __device__ __forceinline__ void v_fma(double *y, const double *u, const double *x)
{
#pragma unroll
    for (int v = 0; v < N; ++v) y[v] = fma(u[v], x[v], y[v]);
}
template <int N> __device__ __forceinline__ void v_add(float *y, const float *x)
{
    if constexpr (N % 2 == 0) {
#pragma unroll
        for (int v = 0; v < N; v += 2) {
            const float2 r = __fadd2_rn(make_float2(x[v], x[v + 1]), make_float2(y[v], y[v + 1]));
            y[v] = r.x;
            y[v + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int v = 0; v < N; ++v) y[v] += x[v];
    }
}
template <int N> __device__ __forceinline__ void v_add(double *y, const double *x)
{
#pragma unroll
    for (int v = 0; v < N; ++v) y[v] += x[v];
}

// In-register DFTs of length 2, 4, 8 with sign SG (y_u = sum_t x_t e^{SG 2 pi i t u / R}), natural order.
template <int SG, typename C> __device__ __forceinline__ void dft2(C &a, C &b)
{
    C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}
template <int SG, typename C> __device__ __forceinline__ void dft4(C &x0, C &x1, C &x2, C &x3)
{
    const C t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), d = csub(x1, x3);
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd_si<SG>(t1, d);
    x3 = csub_si<SG>(t1, d);
}
template <int SG, typename C> __device__ __forceinline__ void dft8(C *x)
{
    using R = decltype(x[0].x);
    C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    C o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    dft4<SG>(e0, e1, e2, e3);
    dft4<SG>(o0, o1, o2, o3);
    const R h = (R)0.70710678118654752440;
    // w8^u, w8 = e^{SG 2 pi i / 8}
    C w1o = {(o1.x - SG * o1.y) * h, (o1.y + SG * o1.x) * h};    // o1 * (1 + SG i)/sqrt2
    C w3o = {(-o3.x - SG * o3.y) * h, (-o3.y + SG * o3.x) * h};  // o3 * (-1 + SG i)/sqrt2
    x[0] = cadd(e0, o0);
    x[4] = csub(e0, o0);
    x[1] = cadd(e1, w1o);
    x[5] = csub(e1, w1o);
    x[2] = cadd_si<SG>(e2, o2);  // e2 +- o2 * SG i
    x[6] = csub_si<SG>(e2, o2);
    x[3] = cadd(e3, w3o);
    x[7] = csub(e3, w3o);
}
// Length 16 as 4 x 4 (index n = 4 n1 + n2, frequency k = k1 + 4 k2): length-4 DFTs over n1, the
// twiddles w16^(n2 k1), length-4 DFTs over n2.
template <int SG, typename C> __device__ __forceinline__ void dft16(C *x)
{
    using R = decltype(x[0].x);
    const R c1 = (R)0.92387953251128675613;  // cos(pi/8)
    const R s1 = (R)0.38268343236508977173;  // sin(pi/8)
    const R h = (R)0.70710678118654752440;   // cos(pi/4)
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<SG>(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);  // y[n2][k1] at x[4 k1 + n2]
    // w16^m = cos(2 pi m / 16) + SG i sin(2 pi m / 16) for m = n2 k1 in {1, 2, 3, 4, 6, 9}
    auto rot = [](C a, R c, R s) { return C{a.x * c - a.y * s, a.x * s + a.y * c}; };
    x[5] = rot(x[5], c1, SG * s1);    // n2 = 1, k1 = 1
    x[9] = rot(x[9], h, SG * h);      // n2 = 1, k1 = 2
    x[13] = rot(x[13], s1, SG * c1);  // n2 = 1, k1 = 3
    x[6] = rot(x[6], h, SG * h);      // n2 = 2, k1 = 1
    x[10] = cmul_si<SG>(x[10]);       // n2 = 2, k1 = 2
    x[14] = rot(x[14], -h, SG * h);   // n2 = 2, k1 = 3
    x[7] = rot(x[7], s1, SG * c1);    // n2 = 3, k1 = 1
    x[11] = rot(x[11], -h, SG * h);   // n2 = 3, k1 = 2
    x[15] = rot(x[15], -c1, -SG * s1); // n2 = 3, k1 = 3
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<SG>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);  // -> X[k1 + 4 k2] at x[4 k1 + k2]
    C t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = x[4 * k1 + k2];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = t[k];
}
template <int R, int SG, typename C> __device__ __forceinline__ void dft_small(C *x)
{
    if constexpr (R == 2) dft2<SG>(x[0], x[1]);
    else if constexpr (R == 4) dft4<SG>(x[0], x[1], x[2], x[3]);
    else if constexpr (R == 8) dft8<SG>(x);
    else dft16<SG>(x);
}

// Radix sequence (first pass = longest span): a first pass of span NP with stride 16 and a last pass
// of radix 16.  With the padding below, the 16 threads of a half-warp then touch 16 distinct bank
// pairs in both passes.
template <int NP> struct Radices;
template <> struct Radices<32> { static constexpr int n = 2; static constexpr int r[2] = {2, 16}; };
template <> struct Radices<64> { static constexpr int n = 2; static constexpr int r[2] = {4, 16}; };
template <> struct Radices<128> { static constexpr int n = 2; static constexpr int r[2] = {8, 16}; };
template <> struct Radices<256> { static constexpr int n = 2; static constexpr int r[2] = {16, 16}; };

// Shared-memory index with one padding slot per 16 complex values (breaks the power-of-two strides of
// the FFT passes across banks).
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// One DIF pass (forward, sign +) or DIT pass (inverse, sign -) of radix R at sub-length M over
// n_tr transforms of length NP stored contiguously in X.
template <int NP, int R, int M, bool FWD, typename C>
__device__ __forceinline__ void fft_pass(C *X, int n_tr, const C *__restrict__ tw)
{
    constexpr int S = M / R;
    constexpr int PER = NP / R;  // butterflies per transform
    // padded stride between the R inputs of a butterfly: exact when S is a multiple of 16, or when
    // S = 1 and every butterfly starts on a multiple of 16 (M a multiple of 16, R <= 16)
    static_assert(S % 16 == 0 || (S == 1 && M % 16 == 0 && R <= 16), "padding");
    // a thread keeps the same butterfly position (and twiddles) in every transform it visits
    static_assert(FTHREADS % PER == 0, "butterfly positions");
    constexpr int PS = S + S / 16;
    constexpr int PNP = NP + NP / 16;  // padded length of one transform
    const int jl = threadIdx.x % PER;
    const int grp = jl / S, j = jl - grp * S;
    const int off = pad16(grp * M + j);
    C w[R];
    if constexpr (S > 1) {  // the last pass (sub-length R) has only unit twiddles
#pragma unroll
        for (int u = 1; u < R; ++u) w[u] = tw[(j * u) * (NP / M)];
    }
    for (int tr = threadIdx.x / PER; tr < n_tr; tr += FTHREADS / PER) {
        C *xb = X + tr * PNP + off;
        C x[R];
#pragma unroll
        for (int t = 0; t < R; ++t) x[t] = xb[t * PS];
        if (FWD) {
            dft_small<R, +1>(x);
            if constexpr (S > 1) {
#pragma unroll
                for (int u = 1; u < R; ++u) x[u] = cmul(x[u], w[u]);
            }
        } else {
            if constexpr (S > 1) {
#pragma unroll
                for (int u = 1; u < R; ++u) x[u] = cconjmul(x[u], w[u]);
            }
            dft_small<R, -1>(x);
        }
#pragma unroll
        for (int t = 0; t < R; ++t) xb[t * PS] = x[t];
    }
    __syncthreads();
}

template <int NP, bool FWD, typename C>
__device__ __forceinline__ void fft_all(C *X, int n_tr, const C *tw)
{
    using RD = Radices<NP>;
    constexpr int R0 = RD::r[0], R1 = RD::r[1];
    static_assert(R0 * R1 == NP, "radices");
    if (FWD) {
        fft_pass<NP, R0, NP, true>(X, n_tr, tw);
        fft_pass<NP, R1, R1, true>(X, n_tr, tw);
    } else {
        fft_pass<NP, R1, R1, false>(X, n_tr, tw);
        fft_pass<NP, R0, NP, false>(X, n_tr, tw);
    }
}

// VEC consecutive reals through 16-byte vector accesses where the size allows (rows are 16-byte
// aligned); the vector is unpacked member by member so that the destination stays in registers.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

__device__ __forceinline__ void unpack(const float4 &q, float *o) { o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w; }
__device__ __forceinline__ void unpack(const double2 &q, double *o) { o[0] = q.x; o[1] = q.y; }
__device__ __forceinline__ float4 pack(const float *i) { return make_float4(i[0], i[1], i[2], i[3]); }
__device__ __forceinline__ double2 pack(const double *i) { return make_double2(i[0], i[1]); }

template <typename T, int VEC>
__device__ __forceinline__ void ldv(const T *__restrict__ p, T *out)
{
    constexpr int N = 16 / (int)sizeof(T);
    if constexpr (VEC % N == 0) {
#pragma unroll
        for (int c = 0; c < VEC / N; ++c) unpack(reinterpret_cast<const typename Vec16<T>::type *>(p)[c], out + c * N);
    } else if constexpr (sizeof(T) == 4 && VEC == 2) {
        const float2 q = *reinterpret_cast<const float2 *>(p);
        out[0] = q.x;
        out[1] = q.y;
    } else {
#pragma unroll
        for (int v = 0; v < VEC; ++v) out[v] = p[v];
    }
}

template <typename T, int VEC>
__device__ __forceinline__ void stv(T *p, const T *in)
{
    constexpr int N = 16 / (int)sizeof(T);
    if constexpr (VEC % N == 0) {
#pragma unroll
        for (int c = 0; c < VEC / N; ++c) reinterpret_cast<typename Vec16<T>::type *>(p)[c] = pack(in + c * N);
    } else if constexpr (sizeof(T) == 4 && VEC == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(in[0], in[1]);
    } else {
#pragma unroll
        for (int v = 0; v < VEC; ++v) p[v] = in[v];
    }
}

// 128-thread blocks (measured faster than 256: more independent blocks per SM keep phase A and phase B
// of different blocks overlapping, and each barrier stalls four warps).  The kernel waits mostly on L2
// loads, so resident warps count: FP32 with one or two states runs seven blocks per SM (72 registers;
// measured 5 % faster than six at 80), three states six (seven would spill), NP = 256 four (wider rows).
template <typename T, int NP, int S>
struct FusedOcc {
    static constexpr int blocks = sizeof(T) == 4 ? (NP >= 256 ? 4 : (S >= 3 ? 6 : 7)) : 2;
};

// Phase A of the fused stage kernels: the potential term of Eq. (quantum-liouvillian) in place on the
// block's rows * S^2 p-rows in X (padded, complex): forward FFT (sign +, digit-reversed), per r-mode
// mixing across the S x S blocks with the tables D, L, R (pre-scaled by 1/NP) times -i, plus the
// p-diagonal bath terms (f_pp lambda_pp(m) - ngam) / NP (damping, delta-term, terminator d2/dp2, which
// are circulants along p), and the inverse FFT (sign -, natural order).  Called by all threads of the
// block after a barrier that makes X complete; ends with the inverse FFT's barrier.
// c2 != 0 (nonlinear coupling V = q + c2 q^2): the d2/dp2 coefficient of row i is fpp phi(q_i)^2,
// phi = 1 + 2 c2 q (Phi^2 = phi^2 d2/dp2); q_i = q_min + i dq.
template <typename T, int NP, int S>
__device__ __forceinline__ void potential_in_place(typename V2<T>::type *X, const typename V2<T>::type *tw,
                                                   const FusedTables<T> &tab, int nq, int i0, int rows, T fpp,
                                                   T ngam, const T *s_lpp, double c2 = 0.0, double q_min = 0.0,
                                                   double dq = 0.0)
{
    using C = typename V2<T>::type;
    constexpr int S2 = S * S;
    fft_all<NP, true>(X, rows * S2, tw);
    constexpr int MV = S >= 3 ? (NP > FTHREADS ? 2 : 1) : (S == 2 ? 2 : 4);  // modes per thread (vector table loads)
    static_assert(FTHREADS % (NP / MV) == 0, "mixing positions");
    const int pos0 = (threadIdx.x % (NP / MV)) * MV;
    // r-space coefficient of the bath terms diagonal in p (already over NP, like the tables):
    // (f_pp lambda_pp(m) - sum n_k gamma_k) / NP
    T cf[MV];
    {
        const T ng_a = ngam / (T)NP;
#pragma unroll
        for (int v = 0; v < MV; ++v) cf[v] = fpp * s_lpp[pos0 + v] - ng_a;
    }
    for (int r = threadIdx.x / (NP / MV); r < rows; r += FTHREADS / (NP / MV)) {
        const int i = i0 + r;
        if (c2 != 0.0) {  // block-uniform
            const T ph = (T)(1.0 + 2.0 * c2 * (q_min + i * dq));
            const T ng_a = ngam / (T)NP;
#pragma unroll
            for (int v = 0; v < MV; ++v) cf[v] = fpp * ph * ph * s_lpp[pos0 + v] - ng_a;
        }
        C rho[S2][MV];
#pragma unroll
        for (int a = 0; a < S2; ++a)
#pragma unroll
            for (int v = 0; v < MV; ++v) rho[a][v] = X[pad16((r * S2 + a) * NP + pos0 + v)];
#pragma unroll
        for (int j = 0; j < S; ++j)
#pragma unroll
            for (int k = 0; k < S; ++k) {
                T d[MV];
                ldv<T, MV>(tab.D + ((size_t)(j * S + k) * nq + i) * NP + pos0, d);
                C acc[MV];
#pragma unroll
                for (int v = 0; v < MV; ++v) acc[v] = C{d[v] * rho[j * S + k][v].x, d[v] * rho[j * S + k][v].y};
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    if (s != j) {
                        T u[MV];
                        ldv<T, MV>(tab.L + ((size_t)(j * S + s) * nq + i) * NP + pos0, u);
#pragma unroll
                        for (int v = 0; v < MV; ++v) {
                            acc[v].x += u[v] * rho[s * S + k][v].x;
                            acc[v].y += u[v] * rho[s * S + k][v].y;
                        }
                    }
                    if (s != k) {
                        T u[MV];
                        ldv<T, MV>(tab.R + ((size_t)(s * S + k) * nq + i) * NP + pos0, u);
#pragma unroll
                        for (int v = 0; v < MV; ++v) {
                            acc[v].x -= u[v] * rho[j * S + s][v].x;
                            acc[v].y -= u[v] * rho[j * S + s][v].y;
                        }
                    }
                }
#pragma unroll
                for (int v = 0; v < MV; ++v) {  // times -i, plus the p-diagonal bath terms
                    const C w = rho[j * S + k][v];
                    X[pad16((r * S2 + j * S + k) * NP + pos0 + v)] = C{acc[v].y + cf[v] * w.x, cf[v] * w.y - acc[v].x};
                }
            }
    }
    __syncthreads();
    fft_all<NP, false>(X, rows * S2, tw);
}

// MULTI: one Horner stage of several propagators at once (heterogeneous batch: members differ in q
// grid, surfaces, bath, hierarchy depth, closure, dt and replica count, and share NP, S and the
// precision).  Blocks are numbered member by member; a block finds its member (first block numbers
// ascending), copies the member's description into shared memory and does that member's block of stage
// k = 4..1 of the Horner form (k = 0: the right-hand side alone into the second stage buffer, for the
// autotuner).  The other arguments are then taken from the member.
// The block `bid` of a fused stage launch (see fused_stage_kernel below); also called in a loop by the
// persistent kernel (a barrier must separate two calls of one block: shared memory is reused).
// NL: the terms of the nonlinear coupling (GridInfo::c2 != 0) are compiled in; NL = false requires
// c2 = 0 (the linear coupling of every workload but the NEXT-3b one keeps their registers free).
template <typename T, int NP, int S, bool MIXED, bool MULTI, bool NL>
__device__ __forceinline__ void
fused_stage_body(unsigned bid, GridInfo g, const ElemInfo *__restrict__ elems, FusedTables<T> tab, StageScalars<T> sc,
                 const T *__restrict__ v_in, const T *y, const double *y0, T *v_out, double *y0_out, double h, int mode,
                 int terms, int rep0, int n_rep, int tq, const T *__restrict__ Pg, const MultiMember<T> *__restrict__ mem,
                 int n_mem, int k, bool warm = false)
{
    // warm: this block's previous call was for the same member and tile height (the persistent kernel's
    // one-member loop), so the member's description, twiddles, p grid and r-space eigenvalues are still
    // in shared memory
    if constexpr (MULTI) {
        __shared__ MultiMember<T> M;
        __shared__ int s_m;
        if (!warm) {
            if (threadIdx.x == 0) {
                int m = 0;
                while (m + 1 < n_mem && mem[m + 1].block0 <= (long)bid) ++m;
                s_m = m;
            }
            __syncthreads();
            static_assert(sizeof(MultiMember<T>) % sizeof(int) == 0, "member size");
            const int *src = reinterpret_cast<const int *>(mem + s_m);
            int *dst = reinterpret_cast<int *>(&M);
            for (int w = threadIdx.x; w < (int)(sizeof(MultiMember<T>) / sizeof(int)); w += FTHREADS) dst[w] = src[w];
            __syncthreads();
        }
        g = M.g;
        elems = M.elems;
        tab = M.tab;
        sc = M.sc[k];
        v_in = k == 4 || k == 0 ? M.y : (k == 3 ? M.vA : (k == 2 ? M.vB : M.vA));
        y = M.y;
        y0 = M.y0;
        v_out = k == 0 ? M.vB : (k == 1 ? M.y : (k == 4 ? M.vA : (k == 3 ? M.vB : M.vA)));
        y0_out = k == 1 ? M.y0 : nullptr;
        h = k == 0 ? 0.0 : M.dt / k;
        mode = k == 0 ? 0 : (k == 1 ? 2 : 1);
        terms = QHFPE_TERM_ALL;
        rep0 = 0;
        n_rep = M.g.n_rep;
        Pg = nullptr;
        bid -= (unsigned)M.block0;
    }
    using C = typename V2<T>::type;
    constexpr int S2 = S * S;
    // phase B: a lane holds VEC consecutive p values of one row, a row spans LPR lanes, and a warp
    // covers RPW rows (several for NP < 128, so that short rows still fill a warp with 16-byte loads)
    constexpr int VEC = NP >= 128 ? NP / 32 : 4;
    constexpr int LPR = NP / VEC;
    constexpr int RPW = 32 / LPR;
    static_assert(LPR * VEC == NP && RPW * LPR == 32, "lane layout");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *X = reinterpret_cast<C *>(smem_raw);          // [tq * S2][NP], padded (pad16)
    C *tw = X + pad16(tq * S2 * NP) + 1;             // [NP]

    const int nq = g.nq;
    const int e = bid % g.n_elem;
    const int rep = rep0 + (bid / g.n_elem) % n_rep;
    const int tile = bid / (g.n_elem * n_rep);
    const int i0 = tile * tq;
    const int rows = min(tq, nq - i0);
    const size_t blk = g.blk;
    const size_t ebase = (size_t)rep * g.rep_stride + (size_t)e * g.elem_stride;

    __shared__ long long nb_off[3 * QH_MAX_MODES];
    __shared__ T nb_wg[3 * QH_MAX_MODES], nb_wa[3 * QH_MAX_MODES];
    __shared__ long long mx_off[QH_MAX_MODES];  // nonlinear coupling: mixed-derivative neighbours
    __shared__ T mx_w[QH_MAX_MODES];
    __shared__ int s_nmx;
    __shared__ int s_cnt[4];
    __shared__ T s_ngam;
    __shared__ __align__(16) T pgrid[NP];
    __shared__ __align__(16) T s_lpp[NP];
    if (threadIdx.x == 0) {
        const ElemInfo &E = elems[e];
        int n = 0;
        const int n_up = (terms & 8) ? E.n_up : 0;
        for (int a = 0; a < n_up; ++a, ++n) {
            nb_off[n] = (long long)(E.up[a] - e) * (long long)g.elem_stride;
            nb_wg[n] = (T)1;
            nb_wa[n] = (T)0;
        }
        const int n_dn = (terms & 16) ? E.n_dn : 0;
        for (int pass = 0; pass < 2; ++pass) {
            if (NL && pass == 0 && (terms & 16)) {  // |m| = 2 couplings of the nonlinear coupling: G only
                for (int a = 0; a < E.n_d2; ++a, ++n) {
                    nb_off[n] = (long long)(E.d2[a] - e) * (long long)g.elem_stride;
                    nb_wg[n] = (T)E.w2[a];
                    nb_wa[n] = (T)0;
                }
            }
            for (int a = 0; a < n_dn; ++a) {
                if ((E.wr[a] != 0.0) != (pass == 1)) continue;
                nb_off[n] = (long long)(E.dn[a] - e) * (long long)g.elem_stride;
                nb_wg[n] = (T)E.wc[a];
                nb_wa[n] = (T)E.wr[a];
                ++n;
            }
            if (pass == 0) s_cnt[1] = n;
        }
        const int n_mx = NL && (terms & 16) ? E.n_mx : 0;
        for (int a = 0; a < n_mx; ++a) {
            mx_off[a] = (long long)(E.mx[a] - e) * (long long)g.elem_stride;
            mx_w[a] = (T)(E.wmx[a] / (12.0 * g.dq));
        }
        s_nmx = n_mx;
        s_cnt[0] = n_up;
        s_cnt[2] = n;
        s_cnt[3] = (terms & 8) && E.terminator;
        s_ngam = (terms & 4) ? (T)E.ngam : (T)0;
    }
    if (!warm)
        for (int t = threadIdx.x; t < NP; t += FTHREADS) {
            tw[t] = C{tab.tw[2 * t], tab.tw[2 * t + 1]};
            pgrid[t] = (T)(g.p_min + t * g.dp);
            s_lpp[t] = tab.lpp[t];
        }

    // the previous launch on the stream (the stage whose output this one reads) has completed and its
    // writes are visible
    asm volatile("griddepcontrol.wait;" ::: "memory");

    // ---- phase A: potential term -------------------------------------------------------------
    // With the potential term computed here, the p-diagonal parts of the bath terms ride along in
    // r-space: the damping -(sum n_k gamma_k) W and the 5-point d2/dp2 of the delta-term and of the
    // terminator are circulants along p, i.e. products with their eigenvalues after the FFT.
    const bool want_pot = (terms & 2) != 0;
    const bool fold = want_pot && !Pg;
    if (fold) {
        constexpr int LV = 4;  // p values per load
        constexpr int PL = NP / LV;
        static_assert(FTHREADS % PL == 0, "load positions");
        const int l = (threadIdx.x % PL) * LV;
        for (int rp = threadIdx.x / PL; rp < rows * S2; rp += FTHREADS / PL) {
            const int pr = rp % S2, r = rp / S2;
            const T *src = v_in + ebase + (size_t)pr * 2 * blk + (size_t)(i0 + r) * NP + l;
            T re[LV], im[LV];
            ldv<T, LV>(src, re);
            ldv<T, LV>(src + blk, im);
            const int base = (r * S2 + pr) * NP + l;
#pragma unroll
            for (int v = 0; v < LV; ++v) X[pad16(base + v)] = C{re[v], im[v]};
        }
        __syncthreads();
        potential_in_place<T, NP, S>(X, tw, tab, nq, i0, rows,
                                     ((terms & 4) ? sc.fdelta : (T)0) + ((s_cnt[3] != 0) ? sc.fterm : (T)0), s_ngam,
                                     s_lpp, NL ? g.c2 : 0.0, g.q_min, g.dq);
    }

    // ---- phase B: one warp per p-row ------------------------------------------------------------
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_up = s_cnt[0], n_d0 = s_cnt[1], n_nb = s_cnt[2];
    const bool term = s_cnt[3] != 0;
    // (folded into phase A when it ran)
    const T ngam = fold ? (T)0 : s_ngam;
    const T inv12dp = sc.inv12dp;
    const T fkin = sc.fkin;
    const T fpp = fold ? (T)0 : ((terms & 4) ? sc.fdelta : (T)0) + (term ? sc.fterm : (T)0);
    const int lr = lane / LPR;            // this lane's row among the warp's RPW rows
    const int l0 = (lane % LPR) * VEC;    // its first p index
    T pcol[VEC];
    ldv<T, VEC>(pgrid + l0, pcol);
    const bool neg0 = pcol[0] < (T)0;
    const bool uni_warp = __all_sync(0xffffffffu, neg0 == (pcol[VEC - 1] < (T)0));
    const int sh = neg0 ? 1 : 0;
    const bool interior = i0 >= 3 && i0 + rows + 3 <= nq;  // no q-stencil row outside the grid
    T pk[VEC];  // -p / (60 dq)
#pragma unroll
    for (int v = 0; v < VEC; ++v) pk[v] = -(pcol[v] * fkin);

    // work unit: RPW consecutive rows of one pair; lanes past the tile's last row compute a copy of it
    // (their shuffles are needed) and store nothing
    const int n_units = RPW == 1 ? rows * S2 : ((rows + RPW - 1) / RPW) * S2;
    for (int rp = warp; rp < n_units; rp += FTHREADS / 32) {
        int pr, r;
        bool act = true;
        if constexpr (RPW == 1) {
            pr = rp % S2;
            r = rp / S2;
        } else {
            pr = rp % S2;
            const int r_lane = (rp / S2) * RPW + lr;
            act = r_lane < rows;
            r = act ? r_lane : rows - 1;
        }
        const int i = i0 + r;
        const size_t poff = ebase + (size_t)pr * 2 * blk;
        const T *Vre = v_in + poff, *Vim = Vre + blk;
        const size_t o = poff + (size_t)i * NP + l0;
        T ar[VEC], ai[VEC], wr[VEC], wi[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) ar[v] = ai[v] = (T)0;

        if (uni_warp) {
            // the six stencil rows in two batches of three (loads of a batch issued before use); the
            // centre row is among them
            const T cneg[6] = {3, -30, -20, 60, -15, 2};  // p < 0: offsets -2..+3
            const T cpos[6] = {-2, 15, -60, 20, 30, -3};  // p >= 0: offsets -3..+2
            const int tc = neg0 ? 2 : 3;                  // centre row
            T kr[VEC], ki[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) kr[v] = ki[v] = (T)0;
            // interior tiles: the six rows lie inside the grid, at fixed offsets from row i - 3 + sh
            const T *rre = interior ? Vre + (size_t)(i - 3 + sh) * NP + l0 : Vre;
            const T *rim = rre + blk;
#pragma unroll
            for (int t0 = 0; t0 < 6; t0 += 3) {
                T sr[3][VEC], si[3][VEC];
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    if (interior) {
                        ldv<T, VEC>(rre + (t0 + b) * NP, sr[b]);
                        ldv<T, VEC>(rim + (t0 + b) * NP, si[b]);
                        continue;
                    }
                    int ii = i + t0 + b - 3 + sh;
                    bool ok = ii >= 0 && ii < nq;
                    if (!ok && g.periodic_q) {
                        ii = ii < 0 ? ii + nq : ii - nq;
                        ok = true;
                    }
                    if (ok) {
                        ldv<T, VEC>(Vre + (size_t)ii * NP + l0, sr[b]);
                        ldv<T, VEC>(Vim + (size_t)ii * NP + l0, si[b]);
                    } else {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) sr[b][v] = si[b][v] = (T)0;
                    }
                }
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const T c = neg0 ? cneg[t0 + b] : cpos[t0 + b];
                    v_axpy<VEC>(kr, c, sr[b]);
                    v_axpy<VEC>(ki, c, si[b]);
                    if (t0 + b == tc) {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            wr[v] = sr[b][v];
                            wi[v] = si[b][v];
                        }
                    }
                }
            }
            if (terms & 1) {
                v_fma<VEC>(ar, pk, kr);
                v_fma<VEC>(ai, pk, ki);
            }
        } else {
            if (terms & 1) {
                const T cneg[7] = {0, 3, -30, -20, 60, -15, 2};
                const T cpos[7] = {-2, 15, -60, 20, 30, -3, 0};
                T kr[VEC], ki[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) kr[v] = ki[v] = (T)0;
#pragma unroll
                for (int d = -3; d <= 3; ++d) {
                    int ii = i + d;
                    if (ii < 0 || ii >= nq) {
                        if (!g.periodic_q) continue;
                        ii = ii < 0 ? ii + nq : ii - nq;
                    }
                    T rr[VEC], ri[VEC];
                    ldv<T, VEC>(Vre + (size_t)ii * NP + l0, rr);
                    ldv<T, VEC>(Vim + (size_t)ii * NP + l0, ri);
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        const T c = pcol[v] < (T)0 ? cneg[d + 3] : cpos[d + 3];
                        kr[v] += c * rr[v];
                        ki[v] += c * ri[v];
                    }
                }
                v_fma<VEC>(ar, pk, kr);
                v_fma<VEC>(ai, pk, ki);
            }
            ldv<T, VEC>(Vre + (size_t)i * NP + l0, wr);
            ldv<T, VEC>(Vim + (size_t)i * NP + l0, wi);
        }
        if (ngam != (T)0) {
            v_axpy<VEC>(ar, -ngam, wr);
            v_axpy<VEC>(ai, -ngam, wi);
        }
        // G = sum_up W^(n+e_k) + sum_dn wc W^(n-e_k) [+ r_0 p W at the terminator]; d/dp of G below
        T gr[VEC], gi[VEC], hr[VEC], hi[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) gr[v] = gi[v] = hr[v] = hi[v] = (T)0;
        for (int a = 0; a < n_up; ++a) {
            const T *u = v_in + (long long)o + nb_off[a];
            T xr[VEC], xi[VEC];
            ldv<T, VEC>(u, xr);
            ldv<T, VEC>(u + blk, xi);
            v_add<VEC>(gr, xr);
            v_add<VEC>(gi, xi);
        }
        for (int a = n_up; a < n_d0; ++a) {
            const T *u = v_in + (long long)o + nb_off[a];
            T xr[VEC], xi[VEC];
            ldv<T, VEC>(u, xr);
            ldv<T, VEC>(u + blk, xi);
            const T wg = nb_wg[a];
            v_axpy<VEC>(gr, wg, xr);
            v_axpy<VEC>(gi, wg, xi);
        }
        // nonlinear coupling V = q + c2 q^2: phi = 1 + 2 c2 q_i multiplies Phi = -phi d/dp and the
        // p phi part of Lambda^(1); its d2/dp dq part enters G below (block-uniform branches)
        const T phi = NL && g.c2 != 0.0 ? (T)(1.0 + 2.0 * g.c2 * (g.q_min + i * g.dq)) : (T)1;
        if (n_d0 < n_nb) {
            for (int a = n_d0; a < n_nb; ++a) {
                const T *u = v_in + (long long)o + nb_off[a];
                T xr[VEC], xi[VEC];
                ldv<T, VEC>(u, xr);
                ldv<T, VEC>(u + blk, xi);
                const T wg = nb_wg[a], wa = nb_wa[a];
                v_axpy<VEC>(gr, wg, xr);
                v_axpy<VEC>(gi, wg, xi);
                v_axpy<VEC>(hr, wa, xr);
                v_axpy<VEC>(hi, wa, xi);
            }
            if (NL && g.c2 != 0.0) {
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    hr[v] *= phi;
                    hi[v] *= phi;
                }
            }
            v_fma<VEC>(ar, pcol, hr);
            v_fma<VEC>(ai, pcol, hi);
        }
        const int n_mx = NL ? s_nmx : 0;
        if (NL && g.c2 != 0.0) {
            // G' = phi G + sum_a wmx_a d/dq W^(mx_a) (4th-order central in q, rows i-2..i+2), so that
            // d/dp G' = phi dG/dp + wmx d2/dp dq W: the p-stencil below covers both
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                gr[v] *= phi;
                gi[v] *= phi;
            }
            for (int a = 0; a < n_mx; ++a) {
                const T *Ere = v_in + poff + mx_off[a];
                const T w = mx_w[a];
                const T cq[4] = {(T)1, (T)-8, (T)8, (T)-1};
                const int dqo[4] = {-2, -1, 1, 2};
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    int ii = i + dqo[b];
                    if (ii < 0 || ii >= nq) {
                        if (!g.periodic_q) continue;
                        ii = ii < 0 ? ii + nq : ii - nq;
                    }
                    T xr[VEC], xi[VEC];
                    ldv<T, VEC>(Ere + (size_t)ii * NP + l0, xr);
                    ldv<T, VEC>(Ere + blk + (size_t)ii * NP + l0, xi);
                    v_axpy<VEC>(gr, w * cq[b], xr);
                    v_axpy<VEC>(gi, w * cq[b], xi);
                }
            }
        }
        const bool have_g = n_nb > 0 || term || n_mx > 0;
        if (term) {
            T r0p[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) r0p[v] = sc.r0 * pcol[v];
            v_fma<VEC>(gr, r0p, wr);
            v_fma<VEC>(gi, r0p, wi);
        }
        // neighbours along p (periodic) through the warp: ext[k] = value at l0 - 2 + k
        auto stencil = [&](const T *xr, const T *xi, T *er, T *ei) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                er[v + 2] = xr[v];
                ei[v + 2] = xi[v];
            }
            // lanes of one row form a shuffle segment of width LPR; source lanes are relative to it
            static_assert(VEC >= 2, "two p values per lane");
            int left, right;
            if constexpr (LPR == 32) {
                left = (lane + 31) & 31;
                right = (lane + 1) & 31;
            } else {
                const int li = lane % LPR;
                left = (li + LPR - 1) & (LPR - 1);
                right = (li + 1) & (LPR - 1);
            }
            er[0] = __shfl_sync(0xffffffffu, xr[VEC - 2], left, LPR);
            er[1] = __shfl_sync(0xffffffffu, xr[VEC - 1], left, LPR);
            ei[0] = __shfl_sync(0xffffffffu, xi[VEC - 2], left, LPR);
            ei[1] = __shfl_sync(0xffffffffu, xi[VEC - 1], left, LPR);
            er[VEC + 2] = __shfl_sync(0xffffffffu, xr[0], right, LPR);
            er[VEC + 3] = __shfl_sync(0xffffffffu, xr[1], right, LPR);
            ei[VEC + 2] = __shfl_sync(0xffffffffu, xi[0], right, LPR);
            ei[VEC + 3] = __shfl_sync(0xffffffffu, xi[1], right, LPR);
        };
        if (have_g) {  // uniform across the block (same element)
            T er[VEC + 4], ei[VEC + 4];
            stencil(gr, gi, er, ei);
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                ar[v] += inv12dp * (er[v] - (T)8 * er[v + 1] + (T)8 * er[v + 3] - er[v + 4]);
                ai[v] += inv12dp * (ei[v] - (T)8 * ei[v + 1] + (T)8 * ei[v + 3] - ei[v + 4]);
            }
        }
        if (fpp != (T)0) {
            T er[VEC + 4], ei[VEC + 4];
            stencil(wr, wi, er, ei);
            const T f = fpp * phi * phi;
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                ar[v] += f * (-er[v] + (T)16 * er[v + 1] - (T)30 * er[v + 2] + (T)16 * er[v + 3] - er[v + 4]);
                ai[v] += f * (-ei[v] + (T)16 * ei[v + 1] - (T)30 * ei[v + 2] + (T)16 * ei[v + 3] - ei[v + 4]);
            }
        }
        if (want_pot && Pg) {  // potential term computed by another kernel
            T pr_[VEC], pi_[VEC];
            ldv<T, VEC>(Pg + poff + (size_t)i * NP + l0, pr_);
            ldv<T, VEC>(Pg + poff + blk + (size_t)i * NP + l0, pi_);
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                ar[v] += pr_[v];
                ai[v] += pi_[v];
            }
        } else if (want_pot) {
            const int pb = (r * S2 + pr) * NP + l0;
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const C pv = X[pad16(pb + v)];
                ar[v] += pv.x;
                ai[v] += pv.y;
            }
        }
        // ---- update -------------------------------------------------------------------------------
        if (!act) {
        } else if (mode == 0) {
            stv<T, VEC>(v_out + o, ar);
            stv<T, VEC>(v_out + o + blk, ai);
        } else if (MIXED && e == 0) {
            const size_t o0 = (size_t)rep * g.tier0_rep_stride + (size_t)pr * 2 * blk + (size_t)i * NP + l0;
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const double nr = y0[o0 + v] + h * (double)ar[v];
                const double ni = y0[o0 + v + blk] + h * (double)ai[v];
                v_out[o + v] = (T)nr;
                v_out[o + v + blk] = (T)ni;
                if (mode == 2) {
                    y0_out[o0 + v] = nr;
                    y0_out[o0 + v + blk] = ni;
                }
            }
        } else {
            const T hh = sc.h;
            T br[VEC], bi[VEC];
            ldv<T, VEC>(y + o, br);
            ldv<T, VEC>(y + o + blk, bi);
            v_axpy<VEC>(br, hh, ar);
            v_axpy<VEC>(bi, hh, ai);
            stv<T, VEC>(v_out + o, br);
            stv<T, VEC>(v_out + o + blk, bi);
        }
    }
}

template <typename T, int NP, int S, bool MIXED, bool MULTI, bool NL>
__global__ void __launch_bounds__(FTHREADS, FusedOcc<T, NP, S>::blocks - (MULTI && FusedOcc<T, NP, S>::blocks > 2 ? 1 : 0))
fused_stage_kernel(GridInfo g, const ElemInfo *__restrict__ elems, FusedTables<T> tab, StageScalars<T> sc, const T *__restrict__ v_in,
                   const T *y, const double *y0, T *v_out, double *y0_out, double h, int mode, int terms, int rep0,
                   int n_rep, int tq, const T *__restrict__ Pg, const MultiMember<T> *__restrict__ mem, int n_mem, int k)
{
    // Programmatic dependent launch: the next stage may start its blocks (prologue only) once every
    // block of this one has started; the body waits (griddepcontrol.wait) for this grid's completion
    // before touching the state.  Both are no-ops for a plain launch.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    fused_stage_body<T, NP, S, MIXED, MULTI, NL>(blockIdx.x, g, elems, tab, sc, v_in, y, y0, v_out, y0_out, h, mode, terms,
                                             rep0, n_rep, tq, Pg, mem, n_mem, k);
}


// One stage of the single-model kernel at tile height tq_req (0: default), launched with programmatic
// stream serialisation: its blocks may be scheduled while the previous kernel drains (the kernel waits
// for it before reading the state).
template <typename T, int NP, int S, bool MIXED, bool NL>
cudaError_t launch_general_t(const GridInfo &g, const ElemInfo *elems, const FusedTables<T> &tab, const T *v_in,
                             const T *y, const double *y0, T *v_out, double *y0_out, double h, int mode, int terms,
                             int rep0, int n_rep, cudaStream_t st, const T *Pg, int tq_req)
{
    int tq = tq_req > 0 ? tq_req : fused_rows_per_tile(NP, S, sizeof(T));
    const int tmax = fused_max_rows(NP, S, sizeof(T));  // the shared-memory limit set at preparation
    if (tq > tmax) tq = tmax;
    if (tq > g.nq) tq = g.nq;
    const size_t smem = fused_smem_bytes(tq, NP, S, sizeof(T));
    const int tiles = (g.nq + tq - 1) / tq;
    const long blocks = (long)tiles * n_rep * g.n_elem;
    if (blocks <= 0) return cudaSuccess;
    const StageScalars<T> sc = stage_scalars<T>(g, h);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(FTHREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fused_stage_kernel<T, NP, S, MIXED, false, NL>, g, elems, tab, sc, v_in, y, y0,
                              v_out, y0_out, h, mode, terms, rep0, n_rep, tq, Pg, (const MultiMember<T> *)nullptr, 0, 0);
}

template <typename T, int NP, int S, bool MIXED, bool NL>
cudaError_t prepare_general_t()
{
    const size_t smem = fused_smem_bytes(fused_max_rows(NP, S, sizeof(T)), NP, S, sizeof(T));
    return cudaFuncSetAttribute(fused_stage_kernel<T, NP, S, MIXED, false, NL>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace
