// The single-model fused stage kernel with the terms of the nonlinear system-bath coupling
// V(q) = q + c2 q^2 compiled in (NL = true, qhfpe_fused_kernel.cuh); launch_fused takes it when
// GridInfo::c2 != 0.  Its own translation unit so that the two instantiation sets compile in parallel.
#include "qhfpe_fused_kernel.cuh"

template <typename T, bool MIXED>
cudaError_t launch_fused_nl(const GridInfo &g, const ElemInfo *elems, const FusedTables<T> &tab, const T *v_in,
                            const T *y, const double *y0, T *v_out, double *y0_out, double h, int mode, int terms,
                            int rep0, int n_rep, cudaStream_t st, const T *Pg, int tq)
{
#define QH_CALL(NP_, S_) launch_general_t<T, NP_, S_, MIXED, true>(g, elems, tab, v_in, y, y0, v_out, y0_out, h, mode, terms, rep0, n_rep, st, Pg, tq)
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

template <typename T, bool MIXED>
cudaError_t prepare_fused_nl(int np, int S)
{
#define QH_CALL(NP_, S_) prepare_general_t<T, NP_, S_, MIXED, true>()
    switch (np * 8 + S) {
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

template cudaError_t launch_fused_nl<float, true>(const GridInfo &, const ElemInfo *, const FusedTables<float> &,
                                                  const float *, const float *, const double *, float *, double *,
                                                  double, int, int, int, int, cudaStream_t, const float *, int);
template cudaError_t launch_fused_nl<double, false>(const GridInfo &, const ElemInfo *, const FusedTables<double> &,
                                                    const double *, const double *, const double *, double *, double *,
                                                    double, int, int, int, int, cudaStream_t, const double *, int);
template cudaError_t prepare_fused_nl<float, true>(int, int);
template cudaError_t prepare_fused_nl<double, false>(int, int);
