// The nonlinear set of the heterogeneous-batch instantiations (qhfpe_fused_multi.cuh: NL = true, the
// terms of the nonlinear system-bath coupling compiled in), taken when a member of the batch has c2 != 0.
#include "qhfpe_fused_multi.cuh"

template <typename T, bool MIXED>
cudaError_t launch_fused_multi_nl(int np, int S, const MultiMember<T> *mem, int n_mem, int k, int tq, long blocks,
                                  cudaStream_t st)
{
    return launch_fused_multi_set<T, MIXED, true>(np, S, mem, n_mem, k, tq, blocks, st);
}

template <typename T, bool MIXED>
cudaError_t prepare_fused_multi_nl(int np, int S, size_t smem)
{
    return prepare_fused_multi_set<T, MIXED, true>(np, S, smem);
}

template cudaError_t launch_fused_multi_nl<float, true>(int, int, const MultiMember<float> *, int, int, int, long,
                                                       cudaStream_t);
template cudaError_t launch_fused_multi_nl<double, false>(int, int, const MultiMember<double> *, int, int, int, long,
                                                         cudaStream_t);
template cudaError_t prepare_fused_multi_nl<float, true>(int, int, size_t);
template cudaError_t prepare_fused_multi_nl<double, false>(int, int, size_t);
