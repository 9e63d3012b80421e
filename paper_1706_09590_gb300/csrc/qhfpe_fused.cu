// Fused right-hand-side stage: launchers of the single-model kernel (qhfpe_fused_kernel.cuh) and the
// non-Condon dipole kernel, which shares its FFT.
#include "qhfpe_fused_kernel.cuh"
#include "qhfpe_fused_window.cuh"

#include <cstdlib>
#include <cstring>

namespace {

// Non-Condon dipole super-operators of Sec. III: (mu^-> W)_jk = sum_l mu_jl(p, q) * W_lk and
// (mu^<- W)_jk = sum_l mu*_lk(p, q) * W_jl are p-convolutions with the Fourier transform of
// mu(q + r/2); after an FFT along p they are products with mu_jl(q_i + r_m/2) (TL) and
// mu_lk(q_i - r_m/2) (TR), both tabulated in the FFT's digit-reversed order and pre-scaled by 1/np.
// side 1: mu^->, 2: mu^<-, 3: mu^x; times `scale`.  One block = (replica, element, tile of tq q rows),
// all pairs, in place.  mirror (the mixed forms' FP32 copy of the zeroth tier): also written.
template <typename T, int NP, int S>
__global__ void __launch_bounds__(FTHREADS)
dipole_fft_kernel(GridInfo g, const T *__restrict__ TL, const T *__restrict__ TR, const T *__restrict__ twt, T *state,
                  size_t rep_stride, int n_elem, const int *__restrict__ reps, int n_rep, int side, double scale, int tq,
                  float *mirror, size_t mirror_rep_stride)
{
    using C = typename V2<T>::type;
    constexpr int S2 = S * S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *X = reinterpret_cast<C *>(smem_raw);  // [tq * S2][NP], padded (pad16)
    C *tw = X + pad16(tq * S2 * NP) + 1;     // [NP]
    const int nq = g.nq;
    const int e = blockIdx.x % n_elem;
    const int ri = (blockIdx.x / n_elem) % n_rep;
    const int rep = reps ? reps[ri] : ri;
    const int tile = blockIdx.x / (n_elem * n_rep);
    const int i0 = tile * tq, rows = min(tq, nq - i0);
    const size_t blk = g.blk;
    T *base = state + (size_t)rep * rep_stride + (size_t)e * g.elem_stride;
    for (int t = threadIdx.x; t < NP; t += FTHREADS) tw[t] = C{twt[2 * t], twt[2 * t + 1]};
    for (int idx = threadIdx.x; idx < rows * S2 * NP; idx += FTHREADS) {
        const int l = idx % NP, rp = idx / NP, pr = rp % S2, r = rp / S2;
        const T *src = base + (size_t)pr * 2 * blk + (size_t)(i0 + r) * NP + l;
        X[pad16((r * S2 + pr) * NP + l)] = C{src[0], src[blk]};
    }
    __syncthreads();
    fft_all<NP, true>(X, rows * S2, tw);
    const T cl = (side & 1) ? (T)1 : (T)0;                          // mu^-> part
    const T cr = side == 2 ? (T)1 : (side == 3 ? (T)-1 : (T)0);     // mu^<- part
    const T sc = (T)scale;
    for (int idx = threadIdx.x; idx < rows * NP; idx += FTHREADS) {
        const int pos = idx % NP, r = idx / NP, i = i0 + r;
        C x[S2];
#pragma unroll
        for (int a = 0; a < S2; ++a) x[a] = X[pad16((r * S2 + a) * NP + pos)];
#pragma unroll
        for (int j = 0; j < S; ++j)
#pragma unroll
            for (int k = 0; k < S; ++k) {
                T ar = (T)0, ai = (T)0;
#pragma unroll
                for (int l = 0; l < S; ++l) {
                    const T a = cl * TL[((size_t)(j * S + l) * nq + i) * NP + pos];
                    const T b = cr * TR[((size_t)(l * S + k) * nq + i) * NP + pos];
                    ar += a * x[l * S + k].x + b * x[j * S + l].x;
                    ai += a * x[l * S + k].y + b * x[j * S + l].y;
                }
                X[pad16((r * S2 + j * S + k) * NP + pos)] = C{sc * ar, sc * ai};
            }
    }
    __syncthreads();
    fft_all<NP, false>(X, rows * S2, tw);
    float *mb = mirror ? mirror + (size_t)rep * mirror_rep_stride : nullptr;
    for (int idx = threadIdx.x; idx < rows * S2 * NP; idx += FTHREADS) {
        const int l = idx % NP, rp = idx / NP, pr = rp % S2, r = rp / S2;
        const size_t o = (size_t)pr * 2 * blk + (size_t)(i0 + r) * NP + l;
        const C v = X[pad16((r * S2 + pr) * NP + l)];
        base[o] = v.x;
        base[o + blk] = v.y;
        if (mb) {
            mb[o] = (float)v.x;
            mb[o + blk] = (float)v.y;
        }
    }
}

template <typename T, int NP, int S>
cudaError_t launch_dipole_fft_t(const GridInfo &g, const T *TL, const T *TR, const T *tw, T *state, size_t rep_stride,
                                int n_elem, const int *reps, int n_rep, int side, double scale, float *mirror,
                                size_t mirror_rep_stride, cudaStream_t st)
{
    // the largest tile (q rows, a power of two up to 16) whose shared memory stays within 44 KB
    int tq = 16;
    while (tq > 1 && fused_smem_bytes(tq, NP, S, sizeof(T)) > 44 * 1024) tq /= 2;
    if (tq > g.nq) tq = g.nq;
    const size_t smem = fused_smem_bytes(tq, NP, S, sizeof(T));
    const long blocks = (long)((g.nq + tq - 1) / tq) * n_rep * n_elem;
    if (blocks <= 0) return cudaSuccess;
    dipole_fft_kernel<T, NP, S><<<(unsigned)blocks, FTHREADS, smem, st>>>(g, TL, TR, tw, state, rep_stride, n_elem, reps,
                                                                         n_rep, side, scale, tq, mirror,
                                                                         mirror_rep_stride);
    return cudaGetLastError();
}

// The q-window kernel serves FP32 states with np = 128 and one or two electronic states when the stage
// computes every term with the potential term in the kernel, each lane's four p values share a sign
// (p = 0 on a multiple of four, or off the grid), and no element has more than six tier neighbours.
// QHFPE_FUSED_WINDOW=0 in the environment selects fused_stage_kernel instead.
bool window_enabled()
{
    const char *v = std::getenv("QHFPE_FUSED_WINDOW");
    return !(v && std::strcmp(v, "0") == 0);
}

}  // namespace

int fused_window_rows(int S) { return S == 1 ? WinTile<1>::TQ : WinTile<2>::TQ; }

bool fused_window_applies(const GridInfo &g, int terms, bool have_pg)
{
    const int np = g.np, S = g.S;
    if (np != 128 || S < 1 || S > 2 || have_pg || terms != QHFPE_TERM_ALL || g.max_nb > WIN_MAXNB || g.c2 != 0.0)
        return false;
    for (int c = 0; c < np; c += 4) {
        const bool a = (float)(g.p_min + c * g.dp) < 0.0f, b = (float)(g.p_min + (c + 3) * g.dp) < 0.0f;
        if (a != b) return false;
    }
    return window_enabled();
}

namespace {

template <int S, bool MIXED>
cudaError_t launch_window_t(const GridInfo &g, const ElemInfo *elems, const FusedTables<float> &tab, const float *v_in,
                            const float *y, const double *y0, float *v_out, double *y0_out, double h, int mode,
                            int rep0, int n_rep, cudaStream_t st)
{
    constexpr int NP = 128, TQ = WinTile<S>::TQ;
    const size_t smem = win_kin_offset<NP, S, TQ>() + WIN_KIN_BYTES;
    const long blocks = (long)((g.nq + TQ - 1) / TQ) * n_rep * g.n_elem;
    if (blocks <= 0) return cudaSuccess;
    const StageScalars<float> sc = stage_scalars<float>(g, h);
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
    return cudaLaunchKernelEx(&cfg, fused_window_kernel<NP, S, MIXED>, g, elems, tab, sc, v_in, y, y0, v_out, y0_out, h,
                              mode, rep0, n_rep);
}

template <typename T, int NP, int S, bool MIXED>
cudaError_t launch_fused_t(const GridInfo &g, const ElemInfo *elems, const FusedTables<T> &tab, const T *v_in,
                           const T *y, const double *y0, T *v_out, double *y0_out, double h, int mode, int terms,
                           int rep0, int n_rep, cudaStream_t st, const T *Pg, int tq_req, int form)
{
    if constexpr (sizeof(T) == 4 && NP == 128 && S <= 2) {
        if (form != 0 && fused_window_applies(g, terms, Pg != nullptr))
            return launch_window_t<S, MIXED>(g, elems, tab, v_in, y, y0, v_out, y0_out, h, mode, rep0, n_rep, st);
    }
    if (g.c2 != 0.0)  // the nonlinear coupling's terms: the instantiation of qhfpe_fused_nl.cu
        return launch_fused_nl<T, MIXED>(g, elems, tab, v_in, y, y0, v_out, y0_out, h, mode, terms, rep0, n_rep, st, Pg,
                                         tq_req);
    return launch_general_t<T, NP, S, MIXED, false>(g, elems, tab, v_in, y, y0, v_out, y0_out, h, mode, terms, rep0,
                                                    n_rep, st, Pg, tq_req);
}

template <typename T, int NP, int S, bool MIXED>
cudaError_t prepare_fused_t()
{
    const int tq = fused_max_rows(NP, S, sizeof(T));
    const size_t smem = fused_smem_bytes(tq, NP, S, sizeof(T));
    cudaError_t e = prepare_general_t<T, NP, S, MIXED, false>();
    if (e != cudaSuccess) return e;
    e = prepare_fused_nl<T, MIXED>(NP, S);
    if (e != cudaSuccess) return e;
    if constexpr (sizeof(T) == 4 && NP == 128 && S <= 2) {
        constexpr int TQ = WinTile<S>::TQ;
        e = cudaFuncSetAttribute(fused_window_kernel<NP, S, MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(win_kin_offset<NP, S, TQ>() + WIN_KIN_BYTES));
        if (e != cudaSuccess) return e;
    }
    return prepare_fused_multi<T, MIXED>(NP, S, smem);
}

}  // namespace

template <typename T>
StageScalars<T> stage_scalars(const GridInfo &g, double h)
{
    StageScalars<T> sc;
    sc.inv12dp = (T)(1.0 / (12.0 * g.dp));
    sc.fkin = (T)(1.0 / (60.0 * g.dq));
    sc.fdelta = (T)(g.cdelta / (12.0 * g.dp * g.dp));
    sc.fterm = (T)(g.term_c0 / (12.0 * g.dp * g.dp));
    sc.r0 = (T)g.term_r0;
    sc.h = (T)h;
    return sc;
}

long fused_blocks(const GridInfo &g, int tq)
{
    if (tq > g.nq) tq = g.nq;
    return (long)((g.nq + tq - 1) / tq) * g.n_rep * g.n_elem;
}

int fused_rows_per_tile(int np, int S, int elem_bytes)
{
    // keep the shared-memory tile near 32 KB (FP32) so that several blocks fit per SM
    const int budget = 32 * 1024 * (elem_bytes == 8 ? 2 : 1);
    int tq = budget / (S * S * np * 2 * elem_bytes);
    if (tq < 1) tq = 1;
    if (tq > 16) tq = 16;
    return tq;
}

size_t fused_smem_bytes(int tq, int np, int S, int elem_bytes)
{
    const int n = tq * S * S * np;
    return ((size_t)(n + (n >> 4) + 1) + np) * 2 * elem_bytes;
}

// Largest tile (q rows) the autotuner may pick: at most 16 rows and at most 96 KB of shared memory.
int fused_max_rows(int np, int S, int elem_bytes)
{
    int tq = 16;
    while (tq > 1 && fused_smem_bytes(tq, np, S, elem_bytes) > 96 * 1024) tq /= 2;
    return tq;
}

bool fused_supported(int np, int S) { return (np == 32 || np == 64 || np == 128 || np == 256) && S >= 1 && S <= 3; }

template <typename T, bool MIXED>
cudaError_t launch_fused(const GridInfo &g, const ElemInfo *elems, const FusedTables<T> &tab, const T *v_in,
                         const T *y, const double *y0, T *v_out, double *y0_out, double h, int mode, int terms,
                         int rep0, int n_rep, cudaStream_t st, const T *Pg, int tq, int form)
{
#define QH_CALL(T_, NP_, S_, M_) launch_fused_t<T_, NP_, S_, M_>(g, elems, tab, v_in, y, y0, v_out, y0_out, h, mode, terms, rep0, n_rep, st, Pg, tq, form)
    switch (g.np * 8 + g.S) {
    case 32 * 8 + 1: return QH_CALL(T, 32, 1, MIXED);
    case 32 * 8 + 2: return QH_CALL(T, 32, 2, MIXED);
    case 32 * 8 + 3: return QH_CALL(T, 32, 3, MIXED);
    case 64 * 8 + 1: return QH_CALL(T, 64, 1, MIXED);
    case 64 * 8 + 2: return QH_CALL(T, 64, 2, MIXED);
    case 64 * 8 + 3: return QH_CALL(T, 64, 3, MIXED);
    case 128 * 8 + 1: return QH_CALL(T, 128, 1, MIXED);
    case 128 * 8 + 2: return QH_CALL(T, 128, 2, MIXED);
    case 128 * 8 + 3: return QH_CALL(T, 128, 3, MIXED);
    case 256 * 8 + 1: return QH_CALL(T, 256, 1, MIXED);
    case 256 * 8 + 2: return QH_CALL(T, 256, 2, MIXED);
    case 256 * 8 + 3: return QH_CALL(T, 256, 3, MIXED);
    default: return cudaErrorInvalidValue;
    }
#undef QH_CALL
}

template <typename T, bool MIXED>
cudaError_t prepare_fused(int np, int S)
{
    switch (np * 8 + S) {
    case 32 * 8 + 1: return prepare_fused_t<T, 32, 1, MIXED>();
    case 32 * 8 + 2: return prepare_fused_t<T, 32, 2, MIXED>();
    case 32 * 8 + 3: return prepare_fused_t<T, 32, 3, MIXED>();
    case 64 * 8 + 1: return prepare_fused_t<T, 64, 1, MIXED>();
    case 64 * 8 + 2: return prepare_fused_t<T, 64, 2, MIXED>();
    case 64 * 8 + 3: return prepare_fused_t<T, 64, 3, MIXED>();
    case 128 * 8 + 1: return prepare_fused_t<T, 128, 1, MIXED>();
    case 128 * 8 + 2: return prepare_fused_t<T, 128, 2, MIXED>();
    case 128 * 8 + 3: return prepare_fused_t<T, 128, 3, MIXED>();
    case 256 * 8 + 1: return prepare_fused_t<T, 256, 1, MIXED>();
    case 256 * 8 + 2: return prepare_fused_t<T, 256, 2, MIXED>();
    case 256 * 8 + 3: return prepare_fused_t<T, 256, 3, MIXED>();
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_dipole_fft(const GridInfo &g, const T *TL, const T *TR, const T *tw, T *state, size_t rep_stride,
                              int n_elem, const int *reps, int n_rep, int side, double scale, float *mirror,
                              size_t mirror_rep_stride, cudaStream_t st)
{
#define QH_CALL(NP_, S_) launch_dipole_fft_t<T, NP_, S_>(g, TL, TR, tw, state, rep_stride, n_elem, reps, n_rep, side, scale, mirror, mirror_rep_stride, st)
    switch (g.np * 8 + g.S) {
    case 32 * 8 + 1: return QH_CALL(32, 1);
    case 32 * 8 + 2: return QH_CALL(32, 2);
    case 32 * 8 + 3: return QH_CALL(32, 3);
    case 64 * 8 + 1: return QH_CALL(64, 1);
    case 64 * 8 + 2: return QH_CALL(64, 2);
    case 64 * 8 + 3: return QH_CALL(64, 3);
    case 128 * 8 + 1: return QH_CALL(128, 1);
    case 128 * 8 + 2: return QH_CALL(128, 2);
    case 128 * 8 + 3: return QH_CALL(128, 3);
    case 256 * 8 + 1: return QH_CALL(256, 1);
    case 256 * 8 + 2: return QH_CALL(256, 2);
    case 256 * 8 + 3: return QH_CALL(256, 3);
    default: return cudaErrorInvalidValue;
    }
#undef QH_CALL
}

// Position -> frequency index of the in-place mixed-radix DIF above: the pass with radix R_a at
// sub-length M_a writes its output digit u_a at stride M_a / R_a, and that digit is the frequency's
// a-th mixed-radix digit (weight R_0 ... R_{a-1}).
int fused_fft_frequency(int np, int pos)
{
    int radix[2], n = 2;
    switch (np) {
    case 32: radix[0] = 2; break;
    case 64: radix[0] = 4; break;
    case 128: radix[0] = 8; break;
    case 256: radix[0] = 16; break;
    default: return -1;
    }
    radix[1] = 16;
    int k = 0, weight = 1, span = np;
    for (int a = 0; a < n; ++a) {
        const int stride = span / radix[a];
        const int u = (pos / stride) % radix[a];
        k += u * weight;
        weight *= radix[a];
        span = stride;
    }
    return k;
}

template cudaError_t launch_fused<float, true>(const GridInfo &, const ElemInfo *, const FusedTables<float> &, const float *, const float *, const double *, float *, double *, double, int, int, int, int, cudaStream_t, const float *, int, int);
template cudaError_t launch_fused<double, false>(const GridInfo &, const ElemInfo *, const FusedTables<double> &, const double *, const double *, const double *, double *, double *, double, int, int, int, int, cudaStream_t, const double *, int, int);
template cudaError_t prepare_fused<float, true>(int, int);
template StageScalars<float> stage_scalars<float>(const GridInfo &, double);
template StageScalars<double> stage_scalars<double>(const GridInfo &, double);
template cudaError_t prepare_fused<double, false>(int, int);
template cudaError_t launch_dipole_fft<float>(const GridInfo &, const float *, const float *, const float *, float *, size_t, int, const int *, int, int, double, float *, size_t, cudaStream_t);
template cudaError_t launch_dipole_fft<double>(const GridInfo &, const double *, const double *, const double *, double *, size_t, int, const int *, int, int, double, float *, size_t, cudaStream_t);
