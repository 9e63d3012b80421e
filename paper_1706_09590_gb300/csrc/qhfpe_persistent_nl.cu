// The persistent propagation's kernels with the nonlinear system-bath coupling's terms compiled in
// (qhfpe_persistent.cuh, NL = true), taken when the propagator has c2 != 0.
#include "qhfpe_persistent.cuh"

template <typename T, bool MIXED>
cudaError_t launch_persistent_nl(int np, int S, const MultiMember<T> *mem, long n_items, int tq, int n_steps,
                                 const double *trace_state, size_t trace_rep_stride, const double *mu, double *partial,
                                 int n_chunks, double *trace_out, long trace_stride, long slot0, unsigned *bar_words,
                                 int *err, unsigned long long limit_ns, cudaStream_t st)
{
    TraceJob tj{trace_out != nullptr, trace_state, trace_rep_stride, mu, partial, n_chunks, trace_out, trace_stride,
                slot0};
    GridBarrier bar{bar_words, bar_words + 1, err, limit_ns};
    return launch_persistent_set<T, MIXED, true>(np, S, mem, n_items, tq, n_steps, tj, bar, st);
}

template cudaError_t launch_persistent_nl<float, true>(int, int, const MultiMember<float> *, long, int, int,
                                                       const double *, size_t, const double *, double *, int, double *,
                                                       long, long, unsigned *, int *, unsigned long long, cudaStream_t);
template cudaError_t launch_persistent_nl<double, false>(int, int, const MultiMember<double> *, long, int, int,
                                                         const double *, size_t, const double *, double *, int,
                                                         double *, long, long, unsigned *, int *, unsigned long long,
                                                         cudaStream_t);
