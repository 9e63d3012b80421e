// Persistent, device-resident propagation (kernels; instantiated by qhfpe_persistent.cu, the linear
// set, and qhfpe_persistent_nl.cu, the set with the nonlinear coupling's terms): ONE cooperative launch advances every replica of a
// propagator n_steps RK4 steps (the Horner form of Sec. III's 4th-order integrator applied to Eq. (heom))
// and records Tr{mu W^(0)} after each step (Eqs. (R1), (R3)), instead of one launch per stage.
//
// The grid is as large as the device holds at once; each Horner stage k = 4..1 is a grid-stride loop
// over the blocks of one fused stage launch (fused_stage_body with the propagator described as a
// one-member batch), and a grid-wide barrier separates the stages.  The barrier's wait is bounded by
// %globaltimer: a block that gives up records the failure and returns, so every block returns and the
// host reports QHFPE_ETIMEOUT; the context stays usable.
#pragma once
#include "qhfpe_fused_kernel.cuh"

namespace {

// One grid barrier: arrivals are counted in count; the last block resets the count and opens the next
// generation.  A block reads the generation before it arrives, so it cannot miss the opening.
struct GridBarrier {
    unsigned *count;
    unsigned *gen;
    int *err;                    // 1 after a wait gave up
    unsigned long long limit_ns; // per wait
};

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool grid_barrier(const GridBarrier &b)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = b.gen;
        const unsigned g0 = *gen;
        __threadfence();
        int pass = 1;
        if (atomicAdd(b.count, 1u) == gridDim.x - 1) {
            *b.count = 0;
            __threadfence();
            atomicAdd(b.gen, 1u);
        } else {
            const unsigned long long t0 = globaltimer();
            while (*gen == g0) {
                if (*(volatile int *)b.err || globaltimer() - t0 > b.limit_ns) {
                    atomicExch(b.err, 1);
                    pass = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = pass;
    }
    __syncthreads();
    return ok != 0;
}

// Trace of one step, in the kernel: chunk partials of sum_jk mu_kj sum W^(0)_jk (blocks over (replica,
// chunk) items, fixed-order tree per block), a barrier, then one warp per replica sums its chunks in a
// fixed order and writes slot `slot` of the sink.
struct TraceJob {
    int record;
    const double *state;   // FP64 zeroth tier (mixed forms) or FP64 state
    size_t rep_stride;
    const double *mu;      // [S][S] (Condon)
    double *partial;       // [n_rep][n_chunks][2]
    int n_chunks;
    double *out;           // sink base: [n_rep][stride] complex
    long stride;
    long slot0;            // slot of the first recorded step
};

__device__ bool trace_step(const GridInfo &g, const TraceJob &tj, long slot, const GridBarrier &bar)
{
    __shared__ double red[2][FTHREADS];
    const int S = g.S;
    const size_t blk = g.blk;
    const size_t len = (blk + tj.n_chunks - 1) / tj.n_chunks;
    for (long it = blockIdx.x; it < (long)g.n_rep * tj.n_chunks; it += gridDim.x) {
        const int chunk = (int)(it % tj.n_chunks), rep = (int)(it / tj.n_chunks);
        const size_t c0 = (size_t)chunk * len, c1 = c0 + len < blk ? c0 + len : blk;
        const double *W = tj.state + (size_t)rep * tj.rep_stride;
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < S; ++k) {
                const double m = tj.mu[k * S + j];
                if (m == 0.0) continue;
                const double *b = W + (size_t)(j * S + k) * 2 * blk;
                double ar = 0.0, ai = 0.0;
                for (size_t c = c0 + threadIdx.x; c < c1; c += FTHREADS) {
                    ar += b[c];
                    ai += b[c + blk];
                }
                sr += m * ar;
                si += m * ai;
            }
        __syncthreads();
        red[0][threadIdx.x] = sr;
        red[1][threadIdx.x] = si;
        __syncthreads();
        for (int w = FTHREADS >> 1; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) {
                red[0][threadIdx.x] += red[0][threadIdx.x + w];
                red[1][threadIdx.x] += red[1][threadIdx.x + w];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            tj.partial[2 * ((size_t)rep * tj.n_chunks + chunk)] = red[0][0];
            tj.partial[2 * ((size_t)rep * tj.n_chunks + chunk) + 1] = red[1][0];
        }
    }
    if (!grid_barrier(bar)) return false;
    const int lane = threadIdx.x & 31, warps = FTHREADS >> 5;
    for (int rep = blockIdx.x * warps + (threadIdx.x >> 5); rep < g.n_rep; rep += gridDim.x * warps) {
        double sr = 0.0, si = 0.0;
        for (int c = lane; c < tj.n_chunks; c += 32) {
            sr += tj.partial[2 * ((size_t)rep * tj.n_chunks + c)];
            si += tj.partial[2 * ((size_t)rep * tj.n_chunks + c) + 1];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, off);
            si += __shfl_xor_sync(0xffffffffu, si, off);
        }
        if (lane == 0) {
            double *o = tj.out + 2 * ((size_t)rep * tj.stride + slot);
            o[0] = sr * g.dq * g.dp;
            o[1] = si * g.dq * g.dp;
        }
    }
    return true;
}

// NL: the nonlinear coupling's terms compiled in (the member's c2 != 0).
template <typename T, int NP, int S, bool MIXED, bool NL>
__global__ void __launch_bounds__(FTHREADS, FusedOcc<T, NP, S>::blocks - (FusedOcc<T, NP, S>::blocks > 2 ? 1 : 0))
persistent_steps_kernel(const MultiMember<T> *__restrict__ mem, long n_items, int tq, int n_steps, TraceJob tj,
                        GridBarrier bar)
{
    const GridInfo g = mem->g;
    bool warm = false;  // the member's description and tables stay in shared memory after the first item
    for (int s = 0; s < n_steps; ++s) {
        for (int k = 4; k >= 1; --k) {
            for (long it = blockIdx.x; it < n_items; it += gridDim.x) {
                __syncthreads();  // the previous item's shared memory is free
                fused_stage_body<T, NP, S, MIXED, true, NL>((unsigned)it, GridInfo{}, nullptr, FusedTables<T>{},
                                                           StageScalars<T>{}, nullptr, nullptr, nullptr, nullptr,
                                                           nullptr, 0.0, 0, 0, 0, 1, tq, nullptr, mem, 1, k, warm);
                warm = true;
            }
            if (!grid_barrier(bar)) return;
        }
        if (tj.record && !trace_step(g, tj, tj.slot0 + s, bar)) return;
        // the next step's stage 4 reads y (written by stage 1 above, behind the barrier) and writes vA;
        // the partials are rewritten only after four more barriers
    }
}

// Failure-detection self-test of the barrier: `withhold` = 1 keeps block 0 from arriving, so every other
// block's wait gives up; 0 passes.
__global__ void barrier_selftest_kernel(GridBarrier bar, int withhold)
{
    if (withhold && blockIdx.x == 0) return;
    grid_barrier(bar);
}

template <typename T, int NP, int S, bool MIXED, bool NL>
cudaError_t launch_persistent_t(const MultiMember<T> *mem, long n_items, int tq, int n_steps, const TraceJob &tj,
                                const GridBarrier &bar, cudaStream_t st)
{
    auto kern = persistent_steps_kernel<T, NP, S, MIXED, NL>;
    const size_t smem = fused_smem_bytes(tq, NP, S, sizeof(T));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FTHREADS, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long grid = (long)per_sm * sms;
    if (grid > n_items) grid = n_items;
    if (grid < 1) grid = 1;
    void *args[] = {(void *)&mem, (void *)&n_items, (void *)&tq, (void *)&n_steps, (void *)&tj, (void *)&bar};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)grid), dim3(FTHREADS), args, smem, st);
}


// the (np, S) switch over the persistent kernels of one NL set
template <typename T, bool MIXED, bool NL>
cudaError_t launch_persistent_set(int np, int S, const MultiMember<T> *mem, long n_items, int tq, int n_steps,
                                  const TraceJob &tj, const GridBarrier &bar, cudaStream_t st)
{
#define QH_CALL(NP_, S_) launch_persistent_t<T, NP_, S_, MIXED, NL>(mem, n_items, tq, n_steps, tj, bar, st)
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
