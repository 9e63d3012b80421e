// Heterogeneous-batch instantiation of the fused stage kernel (MULTI = true, qhfpe_fused_kernel.cuh):
// one launch per Horner stage over the members of a batch.  The set with the nonlinear coupling's
// terms (NL = true, taken when a member has c2 != 0) is instantiated in qhfpe_fused_multi_nl.cu, the
// linear set in qhfpe_fused_multi.cu, so that the two compile in parallel.
#pragma once
#include "qhfpe_fused_kernel.cuh"

namespace {

template <typename T, int NP, int S, bool MIXED, bool NL>
cudaError_t launch_fused_multi_t(const MultiMember<T> *mem, int n_mem, int k, int tq, long blocks, cudaStream_t st)
{
    if (blocks <= 0) return cudaSuccess;
    const size_t smem = fused_smem_bytes(tq, NP, S, sizeof(T));
    fused_stage_kernel<T, NP, S, MIXED, true, NL><<<(unsigned)blocks, FTHREADS, smem, st>>>(
        GridInfo{}, nullptr, FusedTables<T>{}, StageScalars<T>{}, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, 0, 0, 0,
        1, tq, nullptr, mem, n_mem, k);
    return cudaGetLastError();
}

template <typename T, int NP, int S, bool MIXED, bool NL>
cudaError_t prepare_fused_multi_t(size_t smem)
{
    return cudaFuncSetAttribute(fused_stage_kernel<T, NP, S, MIXED, true, NL>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// the (np, S) switch over the instantiations of one NL set
template <typename T, bool MIXED, bool NL>
cudaError_t launch_fused_multi_set(int np, int S, const MultiMember<T> *mem, int n_mem, int k, int tq, long blocks,
                                   cudaStream_t st)
{
#define QH_CALL(NP_, S_) launch_fused_multi_t<T, NP_, S_, MIXED, NL>(mem, n_mem, k, tq, blocks, st)
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

template <typename T, bool MIXED, bool NL>
cudaError_t prepare_fused_multi_set(int np, int S, size_t smem)
{
#define QH_CALL(NP_, S_) prepare_fused_multi_t<T, NP_, S_, MIXED, NL>(smem)
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

}  // namespace
