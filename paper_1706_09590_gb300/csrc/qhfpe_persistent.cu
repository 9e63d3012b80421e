// Persistent propagation: the entry points and the linear set of its kernels (qhfpe_persistent.cuh); the
// set with the nonlinear coupling's terms is instantiated in qhfpe_persistent_nl.cu, so that the two
// compile in parallel.
#include "qhfpe_persistent.cuh"

template <typename T, bool MIXED>
cudaError_t launch_persistent_nl(int np, int S, const MultiMember<T> *mem, long n_items, int tq, int n_steps,
                                 const double *trace_state, size_t trace_rep_stride, const double *mu, double *partial,
                                 int n_chunks, double *trace_out, long trace_stride, long slot0, unsigned *bar_words,
                                 int *err, unsigned long long limit_ns, cudaStream_t st);

template <typename T, bool MIXED>
cudaError_t launch_persistent(int np, int S, const MultiMember<T> *mem, long n_items, int tq, int n_steps,
                              const double *trace_state, size_t trace_rep_stride, const double *mu, double *partial,
                              int n_chunks, double *trace_out, long trace_stride, long slot0, unsigned *bar_words,
                              int *err, unsigned long long limit_ns, bool nonlinear, cudaStream_t st)
{
    if (nonlinear)
        return launch_persistent_nl<T, MIXED>(np, S, mem, n_items, tq, n_steps, trace_state, trace_rep_stride, mu,
                                              partial, n_chunks, trace_out, trace_stride, slot0, bar_words, err,
                                              limit_ns, st);
    TraceJob tj{trace_out != nullptr, trace_state, trace_rep_stride, mu, partial, n_chunks, trace_out, trace_stride,
                slot0};
    GridBarrier bar{bar_words, bar_words + 1, err, limit_ns};
    return launch_persistent_set<T, MIXED, false>(np, S, mem, n_items, tq, n_steps, tj, bar, st);
}

cudaError_t launch_barrier_selftest(unsigned *bar_words, int *err, unsigned long long limit_ns, int withhold,
                                    cudaStream_t st)
{
    GridBarrier bar{bar_words, bar_words + 1, err, limit_ns};
    void *args[] = {(void *)&bar, (void *)&withhold};
    return cudaLaunchCooperativeKernel((const void *)barrier_selftest_kernel, dim3(4), dim3(32), args, 0, st);
}

template cudaError_t launch_persistent<float, true>(int, int, const MultiMember<float> *, long, int, int, const double *,
                                                    size_t, const double *, double *, int, double *, long, long,
                                                    unsigned *, int *, unsigned long long, bool, cudaStream_t);
template cudaError_t launch_persistent<double, false>(int, int, const MultiMember<double> *, long, int, int,
                                                      const double *, size_t, const double *, double *, int, double *,
                                                      long, long, unsigned *, int *, unsigned long long, bool,
                                                      cudaStream_t);
