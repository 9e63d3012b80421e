// qhfpe_potential_term_static: the potential term of the right-hand side for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code that must run with a fixed, pre-planned device footprint
// (embedded or real-time loops, memory owned by another allocator), or code that must not synchronise
// the device, which cudaMalloc/cudaFree can do.  The handle-based calls allocate their
// buffers in qhfpe_create; this entry point needs no handle.  It works in a file-scope device array of
// fixed size instead of allocated scratch.
//
// Scratch layout (doubles): [D | L | R tables: 3*S*S*nq*np][twiddles: np][planar input chunk][planar
// output chunk], the chunks holding as many hierarchy elements as fit.  Every call rebuilds the tables
// and overwrites the chunks before reading them, so nothing needs clearing between calls; the array
// keeps the last call's contents.  Calls share the one array: calls that overlap on the GPU (different
// streams, or different host threads) race and give wrong results.
#include "../../include/qhfpe.h"
#include "qhfpe_internal.cuh"

#include <mutex>

namespace {

constexpr size_t kScratchDoubles = QHFPE_STATIC_SCRATCH_BYTES / sizeof(double);

__device__ __align__(256) double g_static_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Potential tables of Eq. (quantum-liouvillian) in r-space, in the bit-reversed order of the FFT
// potential kernel, scaled by 1/np (same content as the tables qhfpe_create builds on the host).
__global__ void static_tables_kernel(const double *__restrict__ U, int S, int nq, int np, int log2np, double *out)
{
    const size_t n = (size_t)S * S * nq * np;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n + np / 2;
         idx += (size_t)gridDim.x * blockDim.x) {
        if (idx >= n) {
            const int t = (int)(idx - n);
            double s, c;
            sincospi(2.0 * t / np, &s, &c);
            out[3 * n + 2 * t] = c;
            out[3 * n + 2 * t + 1] = s;
            continue;
        }
        const int pos = (int)(idx % np);
        const int i = (int)((idx / np) % nq);
        const int k = (int)((idx / ((size_t)np * nq)) % S);
        const int j = (int)(idx / ((size_t)np * nq * S));
        const int kk = (int)(__brev((unsigned)pos) >> (32 - log2np));
        const int m = kk < np / 2 ? kk : kk - np;
        auto T = [&](int a, int b, int t) { return U[(((size_t)a * S + b) * nq + i) * (np + 1) + t]; };
        auto UL = [&](int a, int b) { return m == -np / 2 ? 0.5 * (T(a, b, 0) + T(a, b, np)) : T(a, b, m + np / 2); };
        auto UR = [&](int a, int b) { return m == -np / 2 ? 0.5 * (T(a, b, 0) + T(a, b, np)) : T(a, b, np / 2 - m); };
        out[idx] = (UL(j, j) - UR(k, k)) / np;
        out[n + idx] = UL(j, k) / np;
        out[2 * n + idx] = UR(j, k) / np;
    }
}

// Once per device, with that device current: the device address of the scratch array (the host-side
// symbol is only a stand-in) and the shared-memory limit of the potential kernels.
qhfpe_status static_setup(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        qh_set_free_error(std::string("potential_term_static: cudaGetDevice: ") + cudaGetErrorString(e));
        return QHFPE_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        qh_set_free_error("potential_term_static: device ordinal out of range");
        return QHFPE_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            qh_set_free_error(std::string("potential_term_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return QHFPE_ECUDA;
        }
        e = prepare_potential(200 * 1024);
        if (e != cudaSuccess) {
            qh_set_free_error(std::string("potential_term_static: set-up: ") + cudaGetErrorString(e));
            return QHFPE_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return QHFPE_OK;
}

}  // namespace

extern "C" qhfpe_status qhfpe_potential_term_static(int n_states, int nq, int np, double p_min, double p_max,
                                                     const double *U_table_dev, int n_elem, const double *W_dev,
                                                     double *out_dev, void *stream)
{
    const int S = n_states;
    if (S < 1 || S > QH_MAX_S || nq < 1 || np < 8 || np > 512 || (np & (np - 1)) || n_elem < 1 ||
        !(p_max > p_min) || !U_table_dev || !W_dev || !out_dev) {
        qh_set_free_error("potential_term_static: invalid argument (S in [1,4], np a power of two in [8,512], "
                          "nq >= 1, n_elem >= 1, p_max > p_min, non-NULL pointers)");
        return QHFPE_EINVAL;
    }
    if ((size_t)2 * S * S * 2 * np * sizeof(double) > 200 * 1024) {
        qh_set_free_error("potential_term_static: n_states * np too large for the shared-memory potential kernel");
        return QHFPE_EINVAL;
    }
    const size_t blk = (size_t)nq * np;
    const size_t tables = 3 * (size_t)S * S * blk + np;
    const size_t per_elem = (size_t)S * S * 2 * blk;  // one planar element
    if (tables + 2 * per_elem > kScratchDoubles) {
        qh_set_free_error("potential_term_static: one hierarchy element of this grid needs more than the "
                          "32 MiB static scratch (3*S*S*nq*np + np + 4*S*S*nq*np doubles must fit)");
        return QHFPE_EINVAL;
    }
    double *scratch = nullptr;
    qhfpe_status r = static_setup(&scratch);
    if (r != QHFPE_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    int log2np = 0;
    while ((1 << log2np) < np) ++log2np;

    static_tables_kernel<<<256, 256, 0, st>>>(U_table_dev, S, nq, np, log2np, scratch);
    cudaError_t e = cudaGetLastError();
    const size_t n = (size_t)S * S * blk;
    PotTables<double> tab{scratch, scratch + n, scratch + 2 * n, scratch + 3 * n};
    const int chunk = (int)((kScratchDoubles - tables) / (2 * per_elem));
    double *in = scratch + tables;
    for (int e0 = 0; e0 < n_elem && e == cudaSuccess; e0 += chunk) {
        const int ne = (n_elem - e0 < chunk) ? n_elem - e0 : chunk;
        double *outp = in + (size_t)ne * per_elem;
        GridInfo g{};
        g.S = S;
        g.nq = nq;
        g.np = np;
        g.log2np = log2np;
        g.n_elem = ne;
        g.n_rep = 1;
        g.p_min = p_min;
        g.dp = (p_max - p_min) / np;
        g.blk = blk;
        g.elem_stride = per_elem;
        g.rep_stride = (size_t)ne * per_elem;
        g.tier0_rep_stride = per_elem;
        const size_t off = (size_t)e0 * S * S * blk * 2;  // canonical complex128 offset, in doubles
        e = launch_from_canonical<double>(g, W_dev + off, in, nullptr, 0, 1, st);
        if (e == cudaSuccess) e = launch_potential<double>(g, tab, in, outp, 0, 1, st);
        if (e == cudaSuccess) e = launch_to_canonical<double>(g, outp, nullptr, out_dev + off, 0, st);
    }
    if (e != cudaSuccess) {
        qh_set_free_error(std::string("potential_term_static: ") + cudaGetErrorString(e));
        return QHFPE_ECUDA;
    }
    return QHFPE_OK;
}
