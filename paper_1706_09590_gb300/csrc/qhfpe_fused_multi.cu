// The linear set of the heterogeneous-batch instantiations (qhfpe_fused_multi.cuh) and the batch
// entry points, which take the nonlinear set of qhfpe_fused_multi_nl.cu when a member has c2 != 0.
#include "qhfpe_fused_multi.cuh"

template <typename T, bool MIXED>
cudaError_t launch_fused_multi_nl(int np, int S, const MultiMember<T> *mem, int n_mem, int k, int tq, long blocks,
                                  cudaStream_t st);
template <typename T, bool MIXED>
cudaError_t prepare_fused_multi_nl(int np, int S, size_t smem);

template <typename T, bool MIXED>
cudaError_t launch_fused_multi(int np, int S, const MultiMember<T> *mem, int n_mem, int k, int tq, long blocks,
                               bool nonlinear, cudaStream_t st)
{
    if (nonlinear) return launch_fused_multi_nl<T, MIXED>(np, S, mem, n_mem, k, tq, blocks, st);
    return launch_fused_multi_set<T, MIXED, false>(np, S, mem, n_mem, k, tq, blocks, st);
}

template <typename T, bool MIXED>
cudaError_t prepare_fused_multi(int np, int S, size_t smem)
{
    cudaError_t e = prepare_fused_multi_set<T, MIXED, false>(np, S, smem);
    if (e != cudaSuccess) return e;
    return prepare_fused_multi_nl<T, MIXED>(np, S, smem);
}

template cudaError_t launch_fused_multi<float, true>(int, int, const MultiMember<float> *, int, int, int, long, bool,
                                                    cudaStream_t);
template cudaError_t launch_fused_multi<double, false>(int, int, const MultiMember<double> *, int, int, int, long, bool,
                                                      cudaStream_t);
template cudaError_t prepare_fused_multi<float, true>(int, int, size_t);
template cudaError_t prepare_fused_multi<double, false>(int, int, size_t);
