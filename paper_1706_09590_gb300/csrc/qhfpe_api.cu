// C ABI of the QHFPE library (include/qhfpe.h): validation, set-up of the model (bath coefficients,
// hierarchy, potential tables), device buffers, the RK4 step loop with captured CUDA graphs, the
// equilibration and response protocols of Sec. III, and spectra.
#include "../../include/qhfpe.h"
#include "qhfpe_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

namespace {

thread_local std::string g_create_error;  // message of the last failed qhfpe_create on this thread

constexpr double kPi = 3.14159265358979323846;
constexpr int kGraphChunk = 16;

// ------------------------------------------------------------------------------------------------
// Bath coefficients for the Drude spectral density (Eqs. (Drude-J), (bath-response),
// (bath-correlation), (expansion-of-bath-*)).  Psi_B(t) = zeta gamma e^{-gamma t} gives
// gamma_0 = gamma, r_0 = zeta; the poles of coth(beta w/2) J(w) give the correlation terms:
//   c_0 = (zeta gamma / 2) cot(beta gamma / 2),
//   gamma_k = 2 pi k / beta,  c_k = 2 zeta gamma^2 / (beta (gamma_k^2 - gamma^2)),  r_k = 0,
//   c_delta = zeta/beta - c_0 - sum_{k<=K} c_k   (the Matsubara tail folded into a delta function).
// High temperature (end of Sec. II): c_0 = zeta / beta and nothing else.
// ------------------------------------------------------------------------------------------------
struct Bath {
    std::vector<double> gamma, r, c;
    double cdelta = 0.0;
};

Bath drude_coefficients(double eta, double gamma, double beta, int K, bool high_t, bool use_cdelta)
{
    Bath b;
    b.gamma.assign(K + 1, 0.0);
    b.r.assign(K + 1, 0.0);
    b.c.assign(K + 1, 0.0);
    b.gamma[0] = gamma;
    b.r[0] = eta;
    if (high_t) {
        b.c[0] = eta / beta;
        return b;
    }
    b.c[0] = eta * gamma / (2.0 * std::tan(beta * gamma / 2.0));
    double tail = eta / beta - b.c[0];
    for (int k = 1; k <= K; ++k) {
        const double nu = 2.0 * kPi * k / beta;
        b.gamma[k] = nu;
        b.c[k] = 2.0 * eta * gamma * gamma / (beta * (nu * nu - gamma * gamma));
        tail -= b.c[k];
    }
    if (use_cdelta) b.cdelta = tail;
    return b;
}

// Hierarchy {n : |n| <= N} ordered by tier, then lexicographically with n_0 largest first.
std::vector<std::vector<int>> build_hierarchy(int modes, int depth)
{
    std::vector<std::vector<int>> all;
    std::vector<int> cur(modes, 0);
    // odometer over the box [0, depth]^modes, keeping |n| <= depth
    while (true) {
        int s = 0;
        for (int v : cur) s += v;
        if (s <= depth) all.push_back(cur);
        int a = modes - 1;
        while (a >= 0 && cur[a] == depth) cur[a--] = 0;
        if (a < 0) break;
        cur[a] += 1;
    }
    std::stable_sort(all.begin(), all.end(), [](const std::vector<int> &x, const std::vector<int> &y) {
        int sx = 0, sy = 0;
        for (int v : x) sx += v;
        for (int v : y) sy += v;
        if (sx != sy) return sx < sy;
        return x > y;  // lexicographic, n_0 largest first
    });
    return all;
}

unsigned bitrev(unsigned x, int bits)
{
    unsigned r = 0;
    for (int b = 0; b < bits; ++b) r |= ((x >> b) & 1u) << (bits - 1 - b);
    return r;
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};


// Eigenvectors of a real symmetric S x S matrix (S <= QH_MAX_S) by cyclic Jacobi rotations, ordered by
// ascending eigenvalue; each vector is signed so that its first component of largest magnitude (within
// 1e-9) is positive.  v[j * S + a] = component j of eigenvector a.
void sym_eigvec(int S, const double *A, double *v)
{
    double a[QH_MAX_S][QH_MAX_S], e[QH_MAX_S][QH_MAX_S];
    for (int r = 0; r < S; ++r)
        for (int c = 0; c < S; ++c) {
            a[r][c] = 0.5 * (A[r * S + c] + A[c * S + r]);
            e[r][c] = r == c ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < S; ++p)
            for (int q = p + 1; q < S; ++q) off += a[p][q] * a[p][q];
        if (off == 0.0) break;
        for (int p = 0; p < S; ++p)
            for (int q = p + 1; q < S; ++q) {
                if (a[p][q] == 0.0) continue;
                // rotation that zeroes a[p][q]: t = tan(phi) of the smaller root
                const double th = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < S; ++k) {
                    const double kp = a[k][p], kq = a[k][q];
                    a[k][p] = c * kp - sn * kq;
                    a[k][q] = sn * kp + c * kq;
                }
                for (int k = 0; k < S; ++k) {
                    const double pk = a[p][k], qk = a[q][k];
                    a[p][k] = c * pk - sn * qk;
                    a[q][k] = sn * pk + c * qk;
                }
                for (int k = 0; k < S; ++k) {
                    const double kp = e[k][p], kq = e[k][q];
                    e[k][p] = c * kp - sn * kq;
                    e[k][q] = sn * kp + c * kq;
                }
            }
    }
    int order[QH_MAX_S];  // ascending eigenvalue (insertion sort, S <= QH_MAX_S, stable)
    for (int k = 0; k < S; ++k) {
        int m = k;
        while (m > 0 && a[k][k] < a[order[m - 1]][order[m - 1]]) {
            order[m] = order[m - 1];
            --m;
        }
        order[m] = k;
    }
    for (int col = 0; col < S; ++col) {
        const int src = order[col];
        double mx = 0.0;
        for (int r = 0; r < S; ++r) mx = std::max(mx, std::fabs(e[r][src]));
        int lead = 0;
        while (std::fabs(e[lead][src]) < mx - 1e-9) ++lead;
        const double sg = e[lead][src] < 0.0 ? -1.0 : 1.0;
        for (int r = 0; r < S; ++r) v[r * S + col] = sg * e[r][src];
    }
}
}  // namespace

// A model: grid, bath and hierarchy data and the potential tables for one set of surfaces.
struct Model {
    int S = 0, nq = 0, np = 0, log2np = 0, n_modes = 0, n_elem = 0, depth = 0, closure = 0;
    GridInfo g{};
    Bath bath;
    std::vector<std::vector<int>> hier;
    std::vector<ElemInfo> elems_host;
    std::vector<double> mu_host;
    ElemInfo *elems = nullptr;
    double *mu = nullptr;
    double *tab64 = nullptr;   // D | L | R | twiddles, FP64
    float *tab32 = nullptr;    // same in FP32
    size_t tab_n = 0;          // entries of one of D, L, R
    double max_rate = 0.0;     // Gershgorin estimate of the generator's spectral radius
    std::vector<double> adia_host;  // adiabatic eigenvectors of U(q_i): [nq][S][S], v[j][a]
    double *adia = nullptr;
    // non-Condon dipole (qhfpe_set_dipole_table): r-space multipliers mu(q + r/2), mu(q - r/2) in the
    // fused FFT's order (TL | TR, FP64 and FP32) and mu(q_i) at the grid points for the trace
    bool noncondon = false;
    double *dip64 = nullptr;
    float *dip32 = nullptr;
    double *mu_q = nullptr;
    const double *trace_mu_q() const { return noncondon ? mu_q : nullptr; }

    PotTables<double> t64() const
    {
        return {tab64, tab64 + tab_n, tab64 + 2 * tab_n, tab64 + 3 * tab_n};
    }
    PotTables<float> t32() const
    {
        return {tab32, tab32 + tab_n, tab32 + 2 * tab_n, tab32 + 3 * tab_n};
    }
    int closure_slot = -1;      // learned closure: element slot holding W^(N+1) (after the real elements)
    bool closure_state = false; // the slot is predicted from the state (QHFPE_LEARNED_STATE)
    int closure_n = -1, closure_n1 = -1;  // elements of tiers N and N-1 (chain, K = 0)
    double *coef64 = nullptr;   // closure coefficients [nq][np][10] (owned by the handle)
    float *coef32 = nullptr;
    float *tcN = nullptr;       // tensor-core path: FP32 tables in natural mode order (D | L | R)
    void *tcB = nullptr;        // tensor-core path: pre-swizzled bf16 hi/lo cosine and sine tiles
    bool fused = false;         // fused stage kernel available for (np, S)
    double *ftab64 = nullptr;   // its tables (digit-reversed order, np twiddles)
    float *ftab32 = nullptr;
    FusedTables<double> f64() const
    {
        return {ftab64, ftab64 + tab_n, ftab64 + 2 * tab_n, ftab64 + 3 * tab_n, ftab64 + 3 * tab_n + 2 * np};
    }
    FusedTables<float> f32() const
    {
        return {ftab32, ftab32 + tab_n, ftab32 + 2 * tab_n, ftab32 + 3 * tab_n, ftab32 + 3 * tab_n + 2 * np};
    }
    ~Model()
    {
        if (elems) cudaFree(elems);
        if (mu) cudaFree(mu);
        if (tab64) cudaFree(tab64);
        if (tab32) cudaFree(tab32);
        if (ftab64) cudaFree(ftab64);
        if (ftab32) cudaFree(ftab32);
        if (tcN) cudaFree(tcN);
        if (tcB) cudaFree(tcB);
        if (adia) cudaFree(adia);
        if (dip64) cudaFree(dip64);
        if (dip32) cudaFree(dip32);
        if (mu_q) cudaFree(mu_q);
    }
};

struct Timing {
    bool enabled = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    long launches[QH_KINDS] = {0, 0, 0};
    double ms[QH_KINDS] = {0, 0, 0};
    ~Timing()
    {
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// One propagator: a batch of replicas of one model in one arithmetic.
struct Prop {
    Model *m = nullptr;
    GridInfo g{};
    bool mixed = false;
    bool tc = false;        // potential term on the tensor cores (bf16 x3)
    int tq = 0;             // fused stage kernel: q rows per block (autotuned on first use; 0 = not yet)
    int form = -1;          // fused stage kernel form (launch_fused): -1 rule, 0 general, 1 q-window
    double dt = 0.0;
    void *y = nullptr, *vA = nullptr, *vB = nullptr, *P = nullptr;
    double *y0 = nullptr;
    TraceSink *sink = nullptr;
    double *partial = nullptr;  // trace reduction partials [n_rep][QH_TRACE_MAX_CHUNKS][2]
    double *trace_buf = nullptr;
    size_t trace_cap = 0;
    cudaGraphExec_t graphs[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [chunk][trace]
    void *pdesc = nullptr;      // persistent propagation: this propagator as a one-member batch
    int pdesc_tq = 0;           // its tile height
    unsigned *pbar = nullptr;   // barrier words (count, generation) and the give-up flag

    void drop_graphs()
    {
        for (auto &a : graphs)
            for (auto &x : a)
                if (x) {
                    cudaGraphExecDestroy(x);
                    x = nullptr;
                }
    }
    ~Prop()
    {
        for (auto &a : graphs)
            for (auto &x : a)
                if (x) cudaGraphExecDestroy(x);
        for (void *b : {y, vA, vB, P, (void *)y0, (void *)sink, (void *)partial, (void *)trace_buf, pdesc,
                        (void *)pbar})
            if (b) cudaFree(b);
    }
};

struct qhfpe {
    qhfpe_params p{};
    std::vector<double> U, mu;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    bool sticky = false;
    std::unique_ptr<Model> model, ground;
    std::unique_ptr<Prop> main;
    std::map<int, std::unique_ptr<Prop>> batches;  // response phases, keyed by replica count
    double *eq = nullptr;   // canonical FP64 equilibrium of one replica
    bool have_eq = false;
    double *scratch = nullptr;
    size_t scratch_cap = 0;
    int *flag = nullptr;    // device flag for non-finite input checks
    int *tc_err = nullptr;  // device flag: a tensor-core kernel gave up waiting
    double *coef64 = nullptr;  // learned-closure coefficient table [nq][np][10]
    float *coef32 = nullptr;
    float *closure_w = nullptr;
    bool persistent = false;   // qhfpe_set_persistent: whole runs of steps in one cooperative launch
    float *state_w = nullptr;  // state-input closure weights (device), nullptr until loaded
    Timing timing;

    ~qhfpe()
    {
        batches.clear();
        main.reset();
        if (eq) cudaFree(eq);
        if (scratch) cudaFree(scratch);
        if (flag) cudaFree(flag);
        if (tc_err) cudaFree(tc_err);
        model.reset();
        ground.reset();
        if (coef64) cudaFree(coef64);
        if (coef32) cudaFree(coef32);
        if (closure_w) cudaFree(closure_w);
        if (state_w) cudaFree(state_w);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }

    qhfpe_status fail(qhfpe_status s, const std::string &msg)
    {
        err = msg;
        return s;
    }
    qhfpe_status cuda_fail(cudaError_t e, const char *what)
    {
        err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
        sticky = true;
        return QHFPE_ECUDA;
    }
};

#define QH_CK(h, call)                                              \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return (h)->cuda_fail(e_, #call);    \
    } while (0)

namespace {

template <typename T>
cudaError_t dalloc(T **p, size_t n)
{
    return cudaMalloc((void **)p, n * sizeof(T) + 16);
}

// Potential tables (Eq. (quantum-liouvillian) in r-space) for an FFT's output order, pre-scaled by
// 1/np.  freq(pos) gives the frequency index sitting at position pos; n_tw twiddles e^{2 pi i t/np}.
template <typename F>
void build_tables(const Model &M, const double *U, std::vector<double> &out, F freq, int n_tw, bool with_lpp = false)
{
    const int S = M.S, nq = M.nq, N = M.np;
    const size_t n = (size_t)S * S * nq * N;
    out.assign(3 * n + 2 * n_tw + (with_lpp ? N : 0), 0.0);
    auto T = [&](int j, int k, int i, int t) { return U[(((size_t)j * S + k) * nq + i) * (N + 1) + t]; };
    auto UL = [&](int j, int s, int i, int m) {
        return m == -N / 2 ? 0.5 * (T(j, s, i, 0) + T(j, s, i, N)) : T(j, s, i, m + N / 2);
    };
    auto UR = [&](int s, int k, int i, int m) {
        return m == -N / 2 ? 0.5 * (T(s, k, i, 0) + T(s, k, i, N)) : T(s, k, i, N / 2 - m);
    };
    for (int j = 0; j < S; ++j)
        for (int k = 0; k < S; ++k)
            for (int i = 0; i < nq; ++i)
                for (int pos = 0; pos < N; ++pos) {
                    const int kk = freq(pos);
                    const int m = kk < N / 2 ? kk : kk - N;
                    const size_t o = (((size_t)j * S + k) * nq + i) * N + pos;
                    out[o] = (UL(j, j, i, m) - UR(k, k, i, m)) / N;
                    out[n + o] = UL(j, k, i, m) / N;
                    out[2 * n + o] = UR(j, k, i, m) / N;
                }
    for (int t = 0; t < n_tw; ++t) {
        out[3 * n + 2 * t] = std::cos(2.0 * kPi * t / N);
        out[3 * n + 2 * t + 1] = std::sin(2.0 * kPi * t / N);
    }
    // eigenvalues of the periodic 5-point second difference (-1, 16, -30, 16, -1) along p at the mode
    // of each FFT position, divided by N (the inverse transform's normalisation): the delta-term and
    // the terminator's c_0 d2/dp2 act as products in r-space
    if (with_lpp)
        for (int pos = 0; pos < N; ++pos) {
            const double th = 2.0 * kPi * freq(pos) / N;
            out[3 * n + 2 * n_tw + pos] = (-2.0 * std::cos(2.0 * th) + 32.0 * std::cos(th) - 30.0) / N;
        }
}

qhfpe_status build_model(qhfpe *h, Model &M, int S, const double *U, const double *mu, int closure_override = -1)
{
    qhfpe_params p = h->p;
    if (closure_override >= 0) p.closure = closure_override;
    M.S = S;
    M.nq = p.nq;
    M.np = p.np;
    M.log2np = 0;
    while ((1 << M.log2np) < p.np) ++M.log2np;
    M.n_modes = p.n_matsubara + 1;
    M.depth = p.depth;
    M.closure = p.closure;
    M.bath = drude_coefficients(p.eta, p.gamma, p.beta, p.n_matsubara, p.high_temperature != 0, p.use_cdelta != 0);
    M.hier = build_hierarchy(M.n_modes, p.depth);
    M.n_elem = (int)M.hier.size();
    std::map<std::vector<int>, int> index;
    for (int e = 0; e < M.n_elem; ++e) index[M.hier[e]] = e;
    M.elems_host.assign(M.n_elem, ElemInfo{});
    for (int e = 0; e < M.n_elem; ++e) {
        ElemInfo &E = M.elems_host[e];
        const std::vector<int> &n = M.hier[e];
        int tier = 0;
        double ngam = 0.0;
        for (int k = 0; k < M.n_modes; ++k) {
            tier += n[k];
            ngam += n[k] * M.bath.gamma[k];
        }
        E.ngam = ngam;
        E.tier = tier;
        E.terminator = ((p.closure == QHFPE_TERMINATOR || p.closure == QHFPE_LEARNED || p.closure == QHFPE_LEARNED_STATE) &&
                        tier == p.depth) ? 1 : 0;
        for (int k = 0; k < M.n_modes; ++k) {
            std::vector<int> v = n;
            v[k] += 1;
            auto it = index.find(v);
            if (it != index.end()) E.up[E.n_up++] = it->second;
            if (n[k] > 0) {
                v[k] -= 2;
                E.dn[E.n_dn] = index.at(v);
                E.wr[E.n_dn] = n[k] * M.bath.gamma[k] * M.bath.r[k];
                E.wc[E.n_dn] = n[k] * M.bath.gamma[k] * M.bath.c[k];
                E.n_dn++;
            }
        }
        // nonlinear coupling: -r_k Lambda^(1) brings (v_c2/2) d2/dp dq of W^(n - e_k) (weight
        // n_k gamma_k r_k v_c2 / 2), and the |m| = 2 terms bring -(multinomial) gamma^m r^m v_c2 phi
        // d/dp W^(n - m), which joins the tier sum G (differentiated as phi d/dp) with weight
        // -(multinomial) gamma^m r^m v_c2
        E.n_mx = E.n_d2 = 0;
        if (p.v_c2 != 0.0) {
            for (int k = 0; k < M.n_modes; ++k) {
                const double w = n[k] * M.bath.gamma[k] * M.bath.r[k] * 0.5 * p.v_c2;
                if (n[k] > 0 && w != 0.0) {
                    std::vector<int> v = n;
                    v[k] -= 1;
                    E.mx[E.n_mx] = index.at(v);
                    E.wmx[E.n_mx] = w;
                    E.n_mx++;
                }
                for (int l = k; l < M.n_modes; ++l) {
                    const double gr = M.bath.gamma[k] * M.bath.r[k] * M.bath.gamma[l] * M.bath.r[l];
                    const double mult = (k == l) ? 0.5 * n[k] * (n[k] - 1) : (double)n[k] * n[l];
                    if (gr == 0.0 || mult == 0.0) continue;
                    std::vector<int> v = n;
                    v[k] -= 1;
                    v[l] -= 1;
                    if (v[k] < 0 || v[l] < 0 || E.n_d2 >= QH_MAX_MODES) continue;
                    E.d2[E.n_d2] = index.at(v);
                    E.w2[E.n_d2] = -mult * gr * p.v_c2;
                    E.n_d2++;
                }
            }
        }
    }
    if (p.closure == QHFPE_LEARNED || p.closure == QHFPE_LEARNED_STATE) {
        M.closure_state = p.closure == QHFPE_LEARNED_STATE;
        M.closure_slot = M.n_elem;
        for (int e = 0; e < M.n_elem; ++e) {
            ElemInfo &E = M.elems_host[e];
            if (E.tier == p.depth) {
                E.up[E.n_up++] = M.closure_slot;
                M.closure_n = e;
                M.closure_n1 = E.n_dn > 0 ? E.dn[0] : -1;
            }
        }
        M.coef64 = h->coef64;
        M.coef32 = h->coef32;
    }
    GridInfo &g = M.g;
    g.S = S;
    g.nq = p.nq;
    g.np = p.np;
    g.log2np = M.log2np;
    g.n_elem = M.n_elem;
    g.n_rep = 0;
    g.periodic_q = p.periodic_q;
    g.q_min = p.q_min;
    g.p_min = p.p_min;
    g.dq = (p.q_max - p.q_min) / p.nq;
    g.dp = (p.p_max - p.p_min) / p.np;
    g.cdelta = M.bath.cdelta;
    g.term_r0 = M.bath.r[0];
    g.term_c0 = M.bath.c[0];
    g.blk = (size_t)p.nq * p.np;
    g.elem_stride = (size_t)S * S * 2 * g.blk;
    g.rep_stride = (size_t)(M.n_elem + (M.closure_slot >= 0 ? 1 : 0)) * g.elem_stride;
    g.tier0_rep_stride = g.elem_stride;
    g.max_nb = 0;
    for (const ElemInfo &E : M.elems_host) g.max_nb = std::max(g.max_nb, E.n_up + E.n_dn);
    g.c2 = p.v_c2;

    M.mu_host.assign(mu, mu + S * S);
    std::vector<double> tab;
    build_tables(M, U, tab, [&](int pos) { return (int)bitrev((unsigned)pos, M.log2np); }, p.np / 2);
    M.tab_n = (size_t)S * S * p.nq * p.np;
    M.fused = fused_supported(p.np, S);

    // Gershgorin-type bound of the spectral radius (for qhfpe_max_stable_dt)
    double pmax = std::max(std::fabs(p.p_min), std::fabs(p.p_max));
    double kin = 130.0 * pmax / (60.0 * g.dq);
    double pot = 0.0;
    const size_t n = M.tab_n;
    for (int j = 0; j < S; ++j)
        for (int k = 0; k < S; ++k)
            for (int i = 0; i < p.nq; ++i)
                for (int pos = 0; pos < p.np; ++pos) {
                    const size_t row = (size_t)i * p.np + pos;
                    double r = std::fabs(tab[((size_t)(j * S + k) * p.nq) * p.np + row]);
                    for (int s = 0; s < S; ++s) {
                        if (s != j) r += std::fabs(tab[n + ((size_t)(j * S + s) * p.nq) * p.np + row]);
                        if (s != k) r += std::fabs(tab[2 * n + ((size_t)(s * S + k) * p.nq) * p.np + row]);
                    }
                    pot = std::max(pot, r * p.np);
                }
    double bathr = 0.0;
    // nonlinear coupling: Phi = -phi d/dp with |phi| <= phimax on the grid
    const double phimax = 1.0 + 2.0 * std::fabs(p.v_c2) * std::max(std::fabs(p.q_min), std::fabs(p.q_max));
    for (const ElemInfo &E : M.elems_host) {
        double r = E.ngam + (std::fabs(g.cdelta) * phimax * phimax + (E.terminator ? g.term_c0 : 0.0)) * 64.0 /
                                (12.0 * g.dp * g.dp);
        r += E.n_up * 1.5 / g.dp * phimax + (E.terminator ? g.term_r0 * (pmax / g.dp * 1.5 + 1.0) : 0.0);
        for (int a = 0; a < E.n_dn; ++a) r += (std::fabs(E.wr[a]) * pmax + std::fabs(E.wc[a]) * 1.5 / g.dp) * phimax;
        for (int a = 0; a < E.n_mx; ++a) r += std::fabs(E.wmx[a]) * (1.5 / g.dp) * (1.5 / g.dq);
        for (int a = 0; a < E.n_d2; ++a) r += std::fabs(E.w2[a]) * 1.5 / g.dp * phimax;
        bathr = std::max(bathr, r);
    }
    M.max_rate = kin + pot + bathr;

    cudaStream_t st = h->stream;
    QH_CK(h, prepare_potential((size_t)2 * S * S * 2 * p.np * sizeof(double)));
    QH_CK(h, dalloc(&M.elems, M.n_elem));
    QH_CK(h, cudaMemcpyAsync(M.elems, M.elems_host.data(), sizeof(ElemInfo) * M.n_elem, cudaMemcpyHostToDevice, st));
    QH_CK(h, dalloc(&M.mu, S * S));
    QH_CK(h, cudaMemcpyAsync(M.mu, M.mu_host.data(), sizeof(double) * S * S, cudaMemcpyHostToDevice, st));
    // adiabatic basis at each grid point: eigenvectors of the diabatic matrix U_jk(q_i), the table
    // column of zero offset
    M.adia_host.assign((size_t)p.nq * S * S, 0.0);
    for (int i = 0; i < p.nq; ++i) {
        double A[QH_MAX_S * QH_MAX_S];
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < S; ++k) A[j * S + k] = U[(((size_t)j * S + k) * p.nq + i) * (p.np + 1) + p.np / 2];
        sym_eigvec(S, A, M.adia_host.data() + (size_t)i * S * S);
    }
    QH_CK(h, dalloc(&M.adia, M.adia_host.size()));
    QH_CK(h, cudaMemcpyAsync(M.adia, M.adia_host.data(), sizeof(double) * M.adia_host.size(), cudaMemcpyHostToDevice, st));
    QH_CK(h, dalloc(&M.tab64, tab.size()));
    QH_CK(h, cudaMemcpyAsync(M.tab64, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, st));
    std::vector<float> tab32(tab.begin(), tab.end());
    QH_CK(h, dalloc(&M.tab32, tab32.size()));
    QH_CK(h, cudaMemcpyAsync(M.tab32, tab32.data(), sizeof(float) * tab32.size(), cudaMemcpyHostToDevice, st));
    if (M.fused) {
        std::vector<double> ft;
        build_tables(M, U, ft, [&](int pos) { return fused_fft_frequency(p.np, pos); }, p.np, true);
        QH_CK(h, dalloc(&M.ftab64, ft.size()));
        QH_CK(h, cudaMemcpyAsync(M.ftab64, ft.data(), sizeof(double) * ft.size(), cudaMemcpyHostToDevice, st));
        std::vector<float> ft32(ft.begin(), ft.end());
        QH_CK(h, dalloc(&M.ftab32, ft32.size()));
        QH_CK(h, cudaMemcpyAsync(M.ftab32, ft32.data(), sizeof(float) * ft32.size(), cudaMemcpyHostToDevice, st));
        QH_CK(h, (prepare_fused<float, true>(p.np, S)));
        QH_CK(h, (prepare_fused<double, false>(p.np, S)));
    }
    if (p.precision == QHFPE_MIXED_BF16X3 && tc_supported(p.np, S)) {
        std::vector<double> nt;
        build_tables(M, U, nt, [](int pos) { return pos; }, 0);
        std::vector<float> nt32(nt.begin(), nt.begin() + 3 * M.tab_n);
        QH_CK(h, dalloc(&M.tcN, nt32.size()));
        QH_CK(h, cudaMemcpyAsync(M.tcN, nt32.data(), sizeof(float) * nt32.size(), cudaMemcpyHostToDevice, st));
        std::vector<uint16_t> bm;
        build_tc_matrices(p.np, bm);
        QH_CK(h, cudaMalloc(&M.tcB, bm.size() * sizeof(uint16_t)));
        QH_CK(h, cudaMemcpyAsync(M.tcB, bm.data(), bm.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st));
        QH_CK(h, prepare_tc(p.np, S));
    }
    QH_CK(h, cudaStreamSynchronize(st));
    return QHFPE_OK;
}

qhfpe_status make_prop(qhfpe *h, Model *M, int n_rep, bool mixed, double dt, std::unique_ptr<Prop> &out)
{
    std::unique_ptr<Prop> P(new (std::nothrow) Prop());
    if (!P) return h->fail(QHFPE_ENOMEM, "host allocation failed");
    P->m = M;
    P->g = M->g;
    P->g.n_rep = n_rep;
    P->mixed = mixed;
    P->tc = mixed && M->tcB != nullptr;
    P->dt = dt;
    const size_t n = (size_t)n_rep * P->g.rep_stride;
    const size_t es = mixed ? sizeof(float) : sizeof(double);
    for (void **b : {&P->y, &P->vA, &P->vB, &P->P}) {
        cudaError_t e = cudaMalloc(b, n * es + 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return h->fail(QHFPE_ENOMEM, "device allocation of the state buffers failed");
        }
        QH_CK(h, cudaMemsetAsync(*b, 0, n * es, h->stream));
    }
    if (mixed) {
        cudaError_t e = cudaMalloc((void **)&P->y0, (size_t)n_rep * P->g.tier0_rep_stride * sizeof(double) + 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return h->fail(QHFPE_ENOMEM, "device allocation of the tier-0 buffer failed");
        }
        QH_CK(h, cudaMemsetAsync(P->y0, 0, (size_t)n_rep * P->g.tier0_rep_stride * sizeof(double), h->stream));
    }
    QH_CK(h, cudaMalloc((void **)&P->partial, (size_t)n_rep * QH_TRACE_MAX_CHUNKS * 2 * sizeof(double)));
    QH_CK(h, cudaMalloc((void **)&P->sink, sizeof(TraceSink)));
    QH_CK(h, cudaMemsetAsync(P->sink, 0, sizeof(TraceSink), h->stream));
    out = std::move(P);
    return QHFPE_OK;
}

// ---- timing helpers --------------------------------------------------------------------------
cudaEvent_t next_event(qhfpe *h)
{
    Timing &T = h->timing;
    if (T.used == T.pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        T.pool.push_back(e);
    }
    return T.pool[T.used++];
}

struct Bracket {
    qhfpe *h;
    int kind;
    cudaEvent_t a = nullptr, b = nullptr;
    Bracket(qhfpe *h_, int k) : h(h_), kind(k)
    {
        if (h->timing.enabled) {
            a = next_event(h);
            b = next_event(h);
            if (a) cudaEventRecord(a, h->stream);
        }
    }
    ~Bracket()
    {
        if (a && b) {
            cudaEventRecord(b, h->stream);
            h->timing.pending.push_back({kind, {a, b}});
        }
    }
};

// Learned closure: fill the W^(N+1) slot of `in` from its two deepest tiers (no-op otherwise).
template <typename T>
qhfpe_status closure_fill(qhfpe *h, const Prop &P, T *in, int rep0, int n_rep)
{
    const Model &M = *P.m;
    if (M.closure_slot < 0) return QHFPE_OK;
    if (M.closure_state) {  // predicted from the state; zero (truncation) until weights are loaded
        if constexpr (sizeof(T) == 8) {
            if (h->state_w)
                QH_CK(h, launch_closure_state_fill<double>(P.g, in, M.closure_n, M.closure_n1, M.closure_slot,
                                                           h->state_w, h->p.eta, rep0, n_rep, h->stream));
        }
        return QHFPE_OK;
    }
    const T *coef = std::is_same<T, float>::value ? (const T *)M.coef32 : (const T *)M.coef64;
    QH_CK(h, launch_closure_apply<T>(P.g, in, M.closure_n, M.closure_n1, M.closure_slot, coef, rep0, n_rep, h->stream));
    return QHFPE_OK;
}

// ---- one RK4 step: Horner form of the degree-4 Taylor polynomial ---------------------------------
//   v = y;  v = y + (dt/4) L v;  v = y + (dt/3) L v;  v = y + (dt/2) L v;  y = y + dt L v.
template <typename T, bool MIXED>
qhfpe_status step_once(qhfpe *h, Prop &P, bool record)
{
    cudaStream_t st = h->stream;
    T *y = (T *)P.y, *vA = (T *)P.vA, *vB = (T *)P.vB, *Pt = (T *)P.P;
    const Model &M = *P.m;
    for (int k = 4; k >= 1; --k) {
        T *in = (k == 4) ? y : (k == 3 ? vA : (k == 2 ? vB : vA));
        T *out = (k == 1) ? y : (k == 4 ? vA : (k == 3 ? vB : vA));
        if (M.closure_slot >= 0) {
            qhfpe_status r = closure_fill<T>(h, P, in, 0, P.g.n_rep);
            if (r != QHFPE_OK) return r;
        }
        if (MIXED && P.tc) {
            {
                Bracket br(h, QH_KIND_POT);
                QH_CK(h, launch_potential_tc(P.g, (const float *)in, (float *)Pt, M.tcB, M.tcN, M.tcN + M.tab_n,
                                             M.tcN + 2 * M.tab_n, P.g.n_rep, h->tc_err, st));
            }
            Bracket br(h, QH_KIND_STAGE);
            QH_CK(h, (launch_fused<float, true>(P.g, M.elems, M.f32(), (const float *)in, (const float *)y, P.y0,
                                               (float *)out, k == 1 ? P.y0 : nullptr, P.dt / k, k == 1 ? 2 : 1,
                                               QHFPE_TERM_ALL, 0, P.g.n_rep, st, (const float *)Pt, P.tq, P.form)));
            continue;
        }
        if (M.fused) {
            Bracket br(h, QH_KIND_STAGE);
            if (MIXED)
                QH_CK(h, (launch_fused<float, true>(P.g, M.elems, M.f32(), (const float *)in, (const float *)y, P.y0,
                                                   (float *)out, k == 1 ? P.y0 : nullptr, P.dt / k, k == 1 ? 2 : 1,
                                                   QHFPE_TERM_ALL, 0, P.g.n_rep, st, nullptr, P.tq, P.form)));
            else
                QH_CK(h, (launch_fused<double, false>(P.g, M.elems, M.f64(), (const double *)in, (const double *)y,
                                                     nullptr, (double *)out, nullptr, P.dt / k, k == 1 ? 2 : 1,
                                                     QHFPE_TERM_ALL, 0, P.g.n_rep, st, nullptr, P.tq)));
            continue;
        }
        {
            Bracket br(h, QH_KIND_POT);
            if (MIXED) QH_CK(h, launch_potential<float>(P.g, M.t32(), (const float *)in, (float *)Pt, 0, P.g.n_rep, st));
            else QH_CK(h, launch_potential<double>(P.g, M.t64(), (const double *)in, (double *)Pt, 0, P.g.n_rep, st));
        }
        {
            Bracket br(h, QH_KIND_STAGE);
            QH_CK(h, (launch_stage<T, MIXED>(P.g, M.elems, in, Pt, y, P.y0, out, k == 1 ? P.y0 : nullptr, P.dt / k,
                                             k == 1 ? 2 : 1, QHFPE_TERM_ALL, 0, P.g.n_rep, st)));
        }
    }
    if (record) {
        Bracket br(h, QH_KIND_AUX);
        if (MIXED) QH_CK(h, launch_trace<double>(P.g, P.y0, P.g.tier0_rep_stride, M.mu, P.sink, 1, P.partial, st, M.trace_mu_q()));
        else QH_CK(h, launch_trace<double>(P.g, (const double *)P.y, P.g.rep_stride, M.mu, P.sink, 1, P.partial, st, M.trace_mu_q()));
    }
    return QHFPE_OK;
}

// ---- one classic RK4 step (the state-input closure makes the right-hand side nonlinear) ------------
//   k1 = L(y), k2 = L(y + dt/2 k1), k3 = L(y + dt/2 k2), k4 = L(y + dt k3),
//   y <- y + dt/6 (k1 + 2 k2 + 2 k3 + k4); FP64, k in vA, the stage input in vB, the sum in P.
qhfpe_status step_rk4(qhfpe *h, Prop &P, bool record)
{
    cudaStream_t st = h->stream;
    const Model &M = *P.m;
    double *y = (double *)P.y, *K = (double *)P.vA, *V = (double *)P.vB, *A = (double *)P.P;
    const size_t n = (size_t)P.g.n_rep * P.g.rep_stride;
    const double dt = P.dt;
    const double a_acc[4] = {dt / 6, dt / 3, dt / 3, dt / 6}, a_v[4] = {dt / 2, dt / 2, dt, 0.0};
    for (int j = 0; j < 4; ++j) {
        double *in = j == 0 ? y : V;
        qhfpe_status r = closure_fill<double>(h, P, in, 0, P.g.n_rep);
        if (r != QHFPE_OK) return r;
        {
            Bracket br(h, QH_KIND_STAGE);
            QH_CK(h, (launch_fused<double, false>(P.g, M.elems, M.f64(), in, in, nullptr, K, nullptr, 0.0, 0,
                                                  QHFPE_TERM_ALL, 0, P.g.n_rep, st, nullptr, P.tq, P.form)));
        }
        QH_CK(h, launch_rk4_combine(n, y, K, A, V, a_acc[j], a_v[j], j == 0, j == 3, st));
    }
    if (record) {
        Bracket br(h, QH_KIND_AUX);
        QH_CK(h, launch_trace<double>(P.g, (const double *)P.y, P.g.rep_stride, M.mu, P.sink, 1, P.partial, st,
                                      M.trace_mu_q()));
    }
    return QHFPE_OK;
}

qhfpe_status step_dispatch(qhfpe *h, Prop &P, bool record)
{
    if (P.m->closure_state) return step_rk4(h, P, record);
    return P.mixed ? step_once<float, true>(h, P, record) : step_once<double, false>(h, P, record);
}

// Autotuner of the fused stage kernel's tile (q rows per block): each candidate evaluates the full
// right-hand side of every replica (into a stage buffer, which holds no data between steps) a few
// times, timed with CUDA events on the handle's stream; the fastest is kept for this propagator.
// Results do not depend on the tile (every cell is computed by the same arithmetic).
qhfpe_status autotune(qhfpe *h, Prop &P)
{
    const Model &M = *P.m;
    if (P.tq || !M.fused) return QHFPE_OK;
    cudaStream_t st = h->stream;
    const int esize = P.mixed ? 4 : 8;
    const int tmax = std::min(fused_max_rows(P.g.np, P.g.S, esize), P.g.nq);
    // QHFPE_TILE_ROWS pins the tile (1 .. the limit) instead of timing the candidates, e.g. to profile
    // the launch configuration that a timed run chose
    if (const char *env = std::getenv("QHFPE_TILE_ROWS")) {
        const int t = std::atoi(env);
        if (t >= 1 && t <= tmax) {
            P.tq = t;
            return QHFPE_OK;
        }
    }
    cudaEvent_t a, b;
    QH_CK(h, cudaEventCreate(&a));
    QH_CK(h, cudaEventCreate(&b));
    // one right-hand side of every replica into vB with the given form and tile, timed over three launches
    auto time_one = [&](int form, int tq, float *ms) -> qhfpe_status {
        for (int rep = 0; rep < 4; ++rep) {
            if (rep == 1) QH_CK(h, cudaEventRecord(a, st));
            cudaError_t e;
            if (P.mixed)
                e = launch_fused<float, true>(P.g, M.elems, M.f32(), (const float *)P.y, (const float *)P.y, P.y0,
                                              (float *)P.vB, nullptr, 0.0, 0, QHFPE_TERM_ALL, 0, P.g.n_rep, st,
                                              P.tc ? (const float *)P.P : nullptr, tq, form);
            else
                e = launch_fused<double, false>(P.g, M.elems, M.f64(), (const double *)P.y, (const double *)P.y,
                                                nullptr, (double *)P.vB, nullptr, 0.0, 0, QHFPE_TERM_ALL, 0, P.g.n_rep,
                                                st, nullptr, tq, form);
            QH_CK(h, e);
        }
        QH_CK(h, cudaEventRecord(b, st));
        QH_CK(h, cudaEventSynchronize(b));
        QH_CK(h, cudaEventElapsedTime(ms, a, b));
        return QHFPE_OK;
    };
    float best = 1e30f, ms = 0.f;
    int best_tq = 1, best_form = 0;
    // the kernel form: the q-window kernel (fixed tile) where it applies, against the general kernel
    if (P.mixed && !P.tc && fused_window_applies(P.g, QHFPE_TERM_ALL, false)) {
        qhfpe_status r = time_one(1, 0, &ms);
        if (r != QHFPE_OK) return r;
        best = ms;
        best_tq = fused_window_rows(P.g.S);
        best_form = 1;
    }
    // tile heights of the general kernel, between the powers of two as well: the block count (tiles x
    // elements x replicas) against the blocks resident at once decides how full the last wave is
    static const int cand[] = {1, 2, 3, 4, 5, 6, 8, 12, 16};
    for (int tq : cand) {
        if (tq > tmax) break;
        qhfpe_status r = time_one(0, tq, &ms);
        if (r != QHFPE_OK) return r;
        if (ms < best) {
            best = ms;
            best_tq = tq;
            best_form = 0;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    P.tq = best_tq;
    P.form = best_form;
    return QHFPE_OK;
}

__global__ void set_sink_kernel(TraceSink *s, double *base, long stride, long counter)
{
    s->base = base;
    s->stride = stride;
    s->counter = counter;
}

// Persistent propagation (qhfpe_set_persistent) covers the fused shapes with the shared-memory FFT
// potential, linear closures without the learned slot and the Condon trace.
bool persistent_ok(const qhfpe *h, const Prop &P)
{
    const Model &M = *P.m;
    return h->persistent && M.fused && !P.tc && M.closure_slot < 0 && !M.noncondon && !h->timing.enabled;
}

template <typename T>
qhfpe_status persistent_desc(qhfpe *h, Prop &P)
{
    if (P.pdesc) return QHFPE_OK;
    const Model &M = *P.m;
    const int esize = sizeof(T);
    // the general stage kernel's tile: the autotuned one when the general form won, else the default
    int tq = P.form == 0 && P.tq > 0 ? P.tq : fused_rows_per_tile(P.g.np, P.g.S, esize);
    tq = std::min(std::min(tq, fused_max_rows(P.g.np, P.g.S, esize)), P.g.nq);
    MultiMember<T> x;
    std::memset(&x, 0, sizeof(x));
    x.g = P.g;
    x.elems = M.elems;
    if constexpr (sizeof(T) == 4) x.tab = M.f32();
    else x.tab = M.f64();
    x.sc[0] = stage_scalars<T>(P.g, 0.0);
    for (int k = 1; k <= 4; ++k) x.sc[k] = stage_scalars<T>(P.g, P.dt / k);
    x.dt = P.dt;
    x.y = (T *)P.y;
    x.vA = (T *)P.vA;
    x.vB = (T *)P.vB;
    x.y0 = P.mixed ? P.y0 : nullptr;
    x.block0 = 0;
    QH_CK(h, cudaMalloc(&P.pdesc, sizeof(x)));
    QH_CK(h, cudaMemcpy(P.pdesc, &x, sizeof(x), cudaMemcpyHostToDevice));
    QH_CK(h, cudaMalloc((void **)&P.pbar, 4 * sizeof(unsigned)));
    P.pdesc_tq = tq;
    return QHFPE_OK;
}

qhfpe_status run_persistent(qhfpe *h, Prop &P, long n_steps, double *trace_dev, long stride)
{
    cudaStream_t st = h->stream;
    qhfpe_status r = P.mixed ? persistent_desc<float>(h, P) : persistent_desc<double>(h, P);
    if (r != QHFPE_OK) return r;
    const long n_items = fused_blocks(P.g, P.pdesc_tq);
    const int nc = trace_chunks(P.g.n_rep, P.g.blk);
    const unsigned long long limit = 2000000000ull;  // 2 s per barrier wait
    for (long done = 0; done < n_steps;) {
        const int len = (int)std::min<long>(n_steps - done, 1 << 20);
        QH_CK(h, cudaMemsetAsync(P.pbar, 0, 4 * sizeof(unsigned), st));
        int *err = reinterpret_cast<int *>(P.pbar + 2);
        const double *ts = P.mixed ? P.y0 : (const double *)P.y;
        const size_t trs = P.mixed ? P.g.tier0_rep_stride : P.g.rep_stride;
        cudaError_t e;
        if (P.mixed)
            e = launch_persistent<float, true>(P.g.np, P.g.S, (const MultiMember<float> *)P.pdesc, n_items, P.pdesc_tq,
                                               len, ts, trs, P.m->mu, P.partial, nc, trace_dev, stride, 1 + done,
                                               P.pbar, err, limit, P.g.c2 != 0.0, st);
        else
            e = launch_persistent<double, false>(P.g.np, P.g.S, (const MultiMember<double> *)P.pdesc, n_items,
                                                 P.pdesc_tq, len, ts, trs, P.m->mu, P.partial, nc, trace_dev, stride,
                                                 1 + done, P.pbar, err, limit, P.g.c2 != 0.0, st);
        QH_CK(h, e);
        int bad = 0;
        QH_CK(h, cudaMemcpyAsync(&bad, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        QH_CK(h, cudaStreamSynchronize(st));
        if (bad) {
            h->sticky = true;
            return h->fail(QHFPE_ETIMEOUT, "persistent propagation: a grid barrier wait gave up");
        }
        done += len;
    }
    return QHFPE_OK;
}

qhfpe_status run_steps(qhfpe *h, Prop &P, long n_steps, double *trace_dev, long stride)
{
    cudaStream_t st = h->stream;
    if (!P.tq && P.m->fused && n_steps > 0) {
        qhfpe_status r = autotune(h, P);
        if (r != QHFPE_OK) return r;
    }
    const bool record = trace_dev != nullptr;
    if (record) {
        set_sink_kernel<<<1, 1, 0, st>>>(P.sink, trace_dev, stride, 0);
        QH_CK(h, cudaGetLastError());
        if (P.mixed) QH_CK(h, launch_trace<double>(P.g, P.y0, P.g.tier0_rep_stride, P.m->mu, P.sink, 1, P.partial, st, P.m->trace_mu_q()));
        else QH_CK(h, launch_trace<double>(P.g, (const double *)P.y, P.g.rep_stride, P.m->mu, P.sink, 1, P.partial, st, P.m->trace_mu_q()));
    }
    if (n_steps > 0 && persistent_ok(h, P)) return run_persistent(h, P, n_steps, trace_dev, stride);
    if (h->timing.enabled) {
        for (long s = 0; s < n_steps; ++s) {
            qhfpe_status r = step_dispatch(h, P, record);
            if (r != QHFPE_OK) return r;
        }
        return QHFPE_OK;
    }
    long done = 0;
    while (done < n_steps) {
        const int chunk = (n_steps - done >= kGraphChunk) ? 1 : 0;
        const int len = chunk ? kGraphChunk : 1;
        cudaGraphExec_t &ge = P.graphs[chunk][record ? 1 : 0];
        if (!ge) {
            cudaGraph_t graph;
            QH_CK(h, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            qhfpe_status r = QHFPE_OK;
            for (int s = 0; s < len && r == QHFPE_OK; ++s) r = step_dispatch(h, P, record);
            cudaError_t e = cudaStreamEndCapture(st, &graph);
            if (r != QHFPE_OK) return r;
            QH_CK(h, e);
            e = cudaGraphInstantiate(&ge, graph, 0);
            cudaGraphDestroy(graph);
            QH_CK(h, e);
        }
        QH_CK(h, cudaGraphLaunch(ge, st));
        done += len;
    }
    return QHFPE_OK;
}

// After a synchronisation: did a tensor-core kernel give up waiting?
qhfpe_status check_timeout(qhfpe *h)
{
    if (!h->tc_err) return QHFPE_OK;
    int bad = 0;
    QH_CK(h, cudaMemcpy(&bad, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (bad) {
        h->sticky = true;
        return h->fail(QHFPE_ETIMEOUT, "a tensor-core kernel gave up waiting for its MMAs");
    }
    return QHFPE_OK;
}

qhfpe_status ensure_trace(qhfpe *h, Prop &P, size_t n_complex)
{
    if (P.trace_cap >= n_complex) return QHFPE_OK;
    if (P.trace_buf) cudaFree(P.trace_buf);
    P.trace_buf = nullptr;
    P.trace_cap = 0;
    QH_CK(h, cudaMalloc((void **)&P.trace_buf, n_complex * 2 * sizeof(double)));
    P.trace_cap = n_complex;
    return QHFPE_OK;
}

qhfpe_status ensure_scratch(qhfpe *h, size_t bytes)
{
    if (h->scratch_cap >= bytes) return QHFPE_OK;
    if (h->scratch) cudaFree(h->scratch);
    h->scratch = nullptr;
    h->scratch_cap = 0;
    QH_CK(h, cudaMalloc((void **)&h->scratch, bytes));
    h->scratch_cap = bytes;
    return QHFPE_OK;
}

template <typename H>
qhfpe_status set_from_canonical_t(qhfpe *h, Prop &P, const H *src_dev, int rep, int n_rep, int *nonfinite)
{
    if (P.mixed)
        QH_CK(h, (launch_from_canonical<float, H>(P.g, src_dev, (float *)P.y, P.y0, rep, n_rep, h->stream, nonfinite)));
    else
        QH_CK(h, (launch_from_canonical<double, H>(P.g, src_dev, (double *)P.y, nullptr, rep, n_rep, h->stream, nonfinite)));
    return QHFPE_OK;
}

template <typename H>
qhfpe_status get_to_canonical_t(qhfpe *h, Prop &P, const void *src, const double *y0, H *dst_dev, int rep)
{
    if (P.mixed) QH_CK(h, (launch_to_canonical<float, H>(P.g, (const float *)src, y0, dst_dev, rep, h->stream)));
    else QH_CK(h, (launch_to_canonical<double, H>(P.g, (const double *)src, nullptr, dst_dev, rep, h->stream)));
    return QHFPE_OK;
}

qhfpe_status set_from_canonical(qhfpe *h, Prop &P, const double *src_dev, int rep, int n_rep, int *nonfinite = nullptr)
{
    if (P.mixed)
        QH_CK(h, launch_from_canonical<float>(P.g, src_dev, (float *)P.y, P.y0, rep, n_rep, h->stream, nonfinite));
    else
        QH_CK(h, launch_from_canonical<double>(P.g, src_dev, (double *)P.y, nullptr, rep, n_rep, h->stream, nonfinite));
    return QHFPE_OK;
}

qhfpe_status get_to_canonical(qhfpe *h, Prop &P, const void *src, const double *y0, double *dst_dev, int rep)
{
    if (P.mixed) QH_CK(h, launch_to_canonical<float>(P.g, (const float *)src, y0, dst_dev, rep, h->stream));
    else QH_CK(h, launch_to_canonical<double>(P.g, (const double *)src, nullptr, dst_dev, rep, h->stream));
    return QHFPE_OK;
}

qhfpe_status apply_dipole_prop(qhfpe *h, Prop &P, int side, const int *reps_dev, int n, double scale)
{
    const Model &M = *P.m;
    if (M.noncondon) {
        const size_t tn = (size_t)M.S * M.S * M.nq * M.np;
        if (P.mixed) {
            // FP32 pass over every element, then the FP64 zeroth tier (which also rewrites its FP32 copy)
            QH_CK(h, launch_dipole_fft<float>(P.g, M.dip32, M.dip32 + tn, M.ftab32 + 3 * tn, (float *)P.y, P.g.rep_stride,
                                              M.n_elem, reps_dev, n, side, scale, nullptr, 0, h->stream));
            QH_CK(h, launch_dipole_fft<double>(P.g, M.dip64, M.dip64 + tn, M.ftab64 + 3 * tn, P.y0,
                                               P.g.tier0_rep_stride, 1, reps_dev, n, side, scale, (float *)P.y,
                                               P.g.rep_stride, h->stream));
        } else {
            QH_CK(h, launch_dipole_fft<double>(P.g, M.dip64, M.dip64 + tn, M.ftab64 + 3 * tn, (double *)P.y,
                                               P.g.rep_stride, M.n_elem, reps_dev, n, side, scale, nullptr, 0,
                                               h->stream));
        }
        return QHFPE_OK;
    }
    if (P.mixed) QH_CK(h, launch_dipole<float>(P.g, (float *)P.y, P.y0, reps_dev, n, P.m->mu, side, scale, h->stream));
    else QH_CK(h, launch_dipole<double>(P.g, (double *)P.y, nullptr, reps_dev, n, P.m->mu, side, scale, h->stream));
    return QHFPE_OK;
}

// copy replica `src` of A into replica `dst` of B (same model and arithmetic)
qhfpe_status copy_replica(qhfpe *h, Prop &A, int src, Prop &B, int dst)
{
    if (&A == &B && src == dst) return QHFPE_OK;
    const size_t es = A.mixed ? sizeof(float) : sizeof(double);
    QH_CK(h, cudaMemcpyAsync((char *)B.y + (size_t)dst * B.g.rep_stride * es, (char *)A.y + (size_t)src * A.g.rep_stride * es,
                             A.g.rep_stride * es, cudaMemcpyDeviceToDevice, h->stream));
    if (A.mixed)
        QH_CK(h, cudaMemcpyAsync(B.y0 + (size_t)dst * B.g.tier0_rep_stride, A.y0 + (size_t)src * A.g.tier0_rep_stride,
                                 A.g.tier0_rep_stride * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    return QHFPE_OK;
}

bool finite_all(const double *x, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

qhfpe_status check_handle(qhfpe *h)
{
    if (!h) return QHFPE_EINVAL;
    if (h->sticky) return QHFPE_ESTATE;
    return QHFPE_OK;
}

qhfpe_status batch_prop(qhfpe *h, int n_rep, Prop **out)
{
    auto it = h->batches.find(n_rep);
    if (it == h->batches.end()) {
        std::unique_ptr<Prop> P;
        qhfpe_status r = make_prop(h, h->model.get(), n_rep, h->p.precision != QHFPE_FP64, h->p.dt, P);
        if (r != QHFPE_OK) return r;
        it = h->batches.emplace(n_rep, std::move(P)).first;
    }
    *out = it->second.get();
    return QHFPE_OK;
}

}  // namespace

// ================================================================================================
//                                          C ABI
// ================================================================================================
extern "C" {

qhfpe_status qhfpe_create(const qhfpe_params *params, void *stream, qhfpe_t **out)
{
    if (!params || !out) return QHFPE_EINVAL;
    *out = nullptr;
    const qhfpe_params &p = *params;
    std::string &create_err = g_create_error;
    auto bad = [&](const char *m) {
        create_err = m;
        return QHFPE_EINVAL;
    };
    if (p.n_states < 1 || p.n_states > QH_MAX_S) return bad("n_states must be in [1, 4]");
    if (p.nq < 1) return bad("nq must be >= 1");
    if (p.np < 8 || p.np > 512 || (p.np & (p.np - 1))) return bad("np must be a power of two in [8, 512]");
    if (!(p.q_max > p.q_min) || !(p.p_max > p.p_min)) return bad("empty grid range");
    if (!p.U_table || !p.mu) return bad("U_table and mu are required");
    if (!(p.dt > 0.0) || !std::isfinite(p.dt)) return bad("dt must be positive and finite");
    if (p.n_matsubara < 0 || p.n_matsubara + 1 > QH_MAX_MODES) return bad("n_matsubara must be in [0, 7]");
    if (p.high_temperature && p.n_matsubara != 0) return bad("high_temperature requires n_matsubara = 0");
    if (p.depth < 0) return bad("depth must be >= 0");
    if (p.closure == QHFPE_TERMINATOR && p.n_matsubara != 0) return bad("the terminator closure needs n_matsubara = 0");
    if (p.closure == QHFPE_LEARNED && p.n_matsubara != 0) return bad("the learned closure needs n_matsubara = 0");
    if (p.closure != QHFPE_TRUNCATE && p.closure != QHFPE_TERMINATOR && p.closure != QHFPE_LEARNED &&
        p.closure != QHFPE_LEARNED_STATE)
        return bad("unknown closure");
    if (p.closure == QHFPE_LEARNED_STATE &&
        (p.n_matsubara != 0 || p.precision != QHFPE_FP64 || p.n_states > 2 || !fused_supported(p.np, p.n_states)))
        return bad("the state-input closure needs n_matsubara = 0, QHFPE_FP64, n_states <= 2 and np in {32, 64, 128, 256}");
    if (p.precision == QHFPE_MIXED_TF32X3) {
        create_err = "QHFPE_MIXED_TF32X3 is not built (its tf32 operand tiles do not fit in shared memory; "
                     "use QHFPE_MIXED_BF16X3)";
        return QHFPE_EUNSUPPORTED;
    }
    if (p.precision != QHFPE_FP64 && p.precision != QHFPE_MIXED && p.precision != QHFPE_MIXED_BF16X3)
        return bad("unknown precision");
    if (p.precision == QHFPE_MIXED_BF16X3 && !tc_supported(p.np, p.n_states)) {
        create_err = "the bf16x3 tensor-core potential kernel covers np in {64, 128} and n_states <= 2";
        return QHFPE_EUNSUPPORTED;
    }
    if (p.n_replicas < 1) return bad("n_replicas must be >= 1");
    if (!std::isfinite(p.v_c2)) return bad("v_c2 must be finite");
    if (p.v_c2 != 0.0 && p.closure != QHFPE_TRUNCATE)
        return bad("a nonlinear coupling (v_c2 != 0) needs closure = QHFPE_TRUNCATE");
    if (p.v_c2 != 0.0 && !fused_supported(p.np, p.n_states)) {
        create_err = "a nonlinear coupling (v_c2 != 0) needs np in {32, 64, 128, 256} and n_states <= 3";
        return QHFPE_EUNSUPPORTED;
    }
    if (!(p.beta > 0.0) || !(p.gamma > 0.0) || !(p.eta >= 0.0)) return bad("bath parameters out of range");
    if (!p.high_temperature && std::fabs(std::sin(p.beta * p.gamma / 2.0)) < 1e-12)
        return bad("beta*gamma/2 is a multiple of pi (cot diverges)");
    const int S = p.n_states;
    const size_t tn = (size_t)S * S * p.nq * (p.np + 1);
    if (!finite_all(p.U_table, tn) || !finite_all(p.mu, (size_t)S * S)) {
        create_err = "U_table or mu holds NaN/Inf";
        return QHFPE_ENUMERIC;
    }
    for (int j = 0; j < S; ++j)
        for (int k = 0; k < S; ++k)
            if (p.mu[j * S + k] != p.mu[k * S + j]) return bad("mu must be symmetric");
    const size_t smem64 = (size_t)2 * S * S * 2 * p.np * sizeof(double);
    if (smem64 > 200 * 1024) return bad("n_states * np too large for the shared-memory potential kernel");

    std::unique_ptr<qhfpe> h(new (std::nothrow) qhfpe());
    if (!h) return QHFPE_ENOMEM;
    h->p = p;
    h->U.assign(p.U_table, p.U_table + tn);
    h->mu.assign(p.mu, p.mu + S * S);
    h->p.U_table = h->U.data();
    h->p.mu = h->mu.data();
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            create_err = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
            cudaGetLastError();
            return QHFPE_ECUDA;
        }
        h->own_stream = true;
    }
    if (p.closure == QHFPE_LEARNED) {
        const size_t nc = (size_t)p.nq * p.np * QHFPE_CLOSURE_N_OUT;
        cudaError_t e = cudaMalloc((void **)&h->coef64, nc * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->coef32, nc * sizeof(float));
        if (e == cudaSuccess) e = cudaMemsetAsync(h->coef64, 0, nc * sizeof(double), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->coef32, 0, nc * sizeof(float), h->stream);
        if (e != cudaSuccess) {
            create_err = std::string("closure tables: ") + cudaGetErrorString(e);
            cudaGetLastError();
            return QHFPE_ENOMEM;
        }
    }
    h->model.reset(new Model());
    qhfpe_status r = build_model(h.get(), *h->model, S, h->U.data(), h->mu.data());
    if (r != QHFPE_OK) {
        create_err = h->err;
        return r;
    }
    if (h->model->tcB) {
        cudaError_t e = cudaMalloc((void **)&h->tc_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->stream);
        if (e != cudaSuccess) {
            create_err = std::string("create: ") + cudaGetErrorString(e);
            return QHFPE_ECUDA;
        }
    }
    r = make_prop(h.get(), h->model.get(), p.n_replicas, p.precision != QHFPE_FP64, p.dt, h->main);
    if (r != QHFPE_OK) {
        create_err = h->err;
        return r;
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        create_err = std::string("create: ") + cudaGetErrorString(e);
        return QHFPE_ECUDA;
    }
    *out = h.release();
    return QHFPE_OK;
}

qhfpe_status qhfpe_destroy(qhfpe_t *h)
{
    if (!h) return QHFPE_EINVAL;
    if (h->stream) cudaStreamSynchronize(h->stream);
    delete h;
    return QHFPE_OK;
}

const char *qhfpe_last_error(const qhfpe_t *h)
{
    if (!h) return g_create_error.c_str();  // calls without a handle (failed create, static entry point)
    return h->err.c_str();
}

qhfpe_status qhfpe_sizes(const qhfpe_t *h, int *n_elem, int *n_modes, size_t *state_elems)
{
    if (!h) return QHFPE_EINVAL;
    const Model &M = *h->model;
    if (n_elem) *n_elem = M.n_elem;
    if (n_modes) *n_modes = M.n_modes;
    if (state_elems) *state_elems = (size_t)M.n_elem * M.S * M.S * M.g.blk;
    return QHFPE_OK;
}

qhfpe_status qhfpe_hierarchy(const qhfpe_t *h, int *idx_out)
{
    if (!h || !idx_out) return QHFPE_EINVAL;
    const Model &M = *h->model;
    for (int e = 0; e < M.n_elem; ++e)
        for (int k = 0; k < M.n_modes; ++k) idx_out[e * M.n_modes + k] = M.hier[e][k];
    return QHFPE_OK;
}

qhfpe_status qhfpe_bath_coefficients(const qhfpe_t *h, double *gamma_k, double *r_k, double *c_k, double *cdelta)
{
    if (!h) return QHFPE_EINVAL;
    const Model &M = *h->model;
    for (int k = 0; k < M.n_modes; ++k) {
        if (gamma_k) gamma_k[k] = M.bath.gamma[k];
        if (r_k) r_k[k] = M.bath.r[k];
        if (c_k) c_k[k] = M.bath.c[k];
    }
    if (cdelta) *cdelta = M.bath.cdelta;
    return QHFPE_OK;
}

qhfpe_status qhfpe_max_stable_dt(const qhfpe_t *h, double *dt_out)
{
    if (!h || !dt_out) return QHFPE_EINVAL;
    *dt_out = 2.8 / h->model->max_rate;
    return QHFPE_OK;
}

}  // extern "C"

namespace {

template <typename H>
qhfpe_status set_state_t(qhfpe_t *h, int replica, const H *src, int is_device)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    Prop &P = *h->main;
    if (!src || replica < -1 || replica >= P.g.n_rep) return h->fail(QHFPE_EINVAL, "set_state: bad replica or NULL source");
    const size_t n = (size_t)P.g.n_elem * P.g.S * P.g.S * P.g.blk;
    const H *dsrc = src;
    if (!h->flag) QH_CK(h, cudaMalloc((void **)&h->flag, sizeof(int)));
    QH_CK(h, cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    if (!is_device) {
        r = ensure_scratch(h, n * 2 * sizeof(H));
        if (r != QHFPE_OK) return r;
        QH_CK(h, cudaMemcpyAsync(h->scratch, src, n * 2 * sizeof(H), cudaMemcpyHostToDevice, h->stream));
        dsrc = reinterpret_cast<const H *>(h->scratch);
    }
    r = set_from_canonical_t<H>(h, P, dsrc, replica < 0 ? 0 : replica, replica < 0 ? P.g.n_rep : 1, h->flag);
    if (r != QHFPE_OK) return r;
    int bad = 0;
    QH_CK(h, cudaMemcpyAsync(&bad, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    QH_CK(h, cudaStreamSynchronize(h->stream));
    if (bad) return h->fail(QHFPE_ENUMERIC, "set_state: source holds NaN/Inf (the replica now holds it too)");
    return QHFPE_OK;
}

template <typename H>
qhfpe_status get_state_t(qhfpe_t *h, int replica, H *dst, int is_device)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    Prop &P = *h->main;
    if (!dst || replica < 0 || replica >= P.g.n_rep) return h->fail(QHFPE_EINVAL, "get_state: bad replica or NULL destination");
    const size_t n = (size_t)P.g.n_elem * P.g.S * P.g.S * P.g.blk;
    H *ddst = dst;
    if (!is_device) {
        r = ensure_scratch(h, n * 2 * sizeof(H));
        if (r != QHFPE_OK) return r;
        ddst = reinterpret_cast<H *>(h->scratch);
    }
    r = get_to_canonical_t<H>(h, P, P.y, P.y0, ddst, replica);
    if (r != QHFPE_OK) return r;
    if (!is_device) QH_CK(h, cudaMemcpyAsync(dst, ddst, n * 2 * sizeof(H), cudaMemcpyDeviceToHost, h->stream));
    QH_CK(h, cudaStreamSynchronize(h->stream));
    return QHFPE_OK;
}

}  // namespace

extern "C" {

qhfpe_status qhfpe_set_state(qhfpe_t *h, int replica, const double *src, int is_device)
{
    return set_state_t<double>(h, replica, src, is_device);
}

qhfpe_status qhfpe_get_state(qhfpe_t *h, int replica, double *dst, int is_device)
{
    return get_state_t<double>(h, replica, dst, is_device);
}

qhfpe_status qhfpe_set_state32(qhfpe_t *h, int replica, const float *src, int is_device)
{
    return set_state_t<float>(h, replica, src, is_device);
}

qhfpe_status qhfpe_get_state32(qhfpe_t *h, int replica, float *dst, int is_device)
{
    return get_state_t<float>(h, replica, dst, is_device);
}

qhfpe_status qhfpe_fork(qhfpe_t *h, int src, const int *dst, int n)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    Prop &P = *h->main;
    if (src < 0 || src >= P.g.n_rep || (n > 0 && !dst)) return h->fail(QHFPE_EINVAL, "fork: bad replica");
    for (int a = 0; a < n; ++a) {
        if (dst[a] < 0 || dst[a] >= P.g.n_rep) return h->fail(QHFPE_EINVAL, "fork: bad destination replica");
        if (dst[a] == src) continue;
        r = copy_replica(h, P, src, P, dst[a]);
        if (r != QHFPE_OK) return r;
    }
    QH_CK(h, cudaStreamSynchronize(h->stream));
    return QHFPE_OK;
}

qhfpe_status qhfpe_step(qhfpe_t *h, long n_steps, double *trace_out)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    if (n_steps < 0) return h->fail(QHFPE_EINVAL, "step: n_steps < 0");
    Prop &P = *h->main;
    double *tr = nullptr;
    const long stride = n_steps + 1;
    if (trace_out) {
        r = ensure_trace(h, P, (size_t)P.g.n_rep * stride);
        if (r != QHFPE_OK) return r;
        tr = P.trace_buf;
    }
    r = run_steps(h, P, n_steps, tr, stride);
    if (r != QHFPE_OK) return r;
    if (trace_out)
        QH_CK(h, cudaMemcpyAsync(trace_out, tr, (size_t)P.g.n_rep * stride * 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                 h->stream));
    QH_CK(h, cudaStreamSynchronize(h->stream));
    return check_timeout(h);
}

qhfpe_status qhfpe_apply_dipole(qhfpe_t *h, int side, const int *replicas, int n)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    Prop &P = *h->main;
    if (side < 1 || side > 3) return h->fail(QHFPE_EINVAL, "apply_dipole: side must be 1, 2 or 3");
    const int *reps_dev = nullptr;
    int count = P.g.n_rep;
    if (replicas) {
        for (int a = 0; a < n; ++a)
            if (replicas[a] < 0 || replicas[a] >= P.g.n_rep) return h->fail(QHFPE_EINVAL, "apply_dipole: bad replica");
        r = ensure_scratch(h, (size_t)n * sizeof(int) + 16);
        if (r != QHFPE_OK) return r;
        QH_CK(h, cudaMemcpyAsync(h->scratch, replicas, (size_t)n * sizeof(int), cudaMemcpyHostToDevice, h->stream));
        reps_dev = (const int *)h->scratch;
        count = n;
    }
    if (count > 0) {
        r = apply_dipole_prop(h, P, side, reps_dev, count, 1.0);
        if (r != QHFPE_OK) return r;
    }
    QH_CK(h, cudaStreamSynchronize(h->stream));
    return QHFPE_OK;
}

qhfpe_status qhfpe_apply_rhs(qhfpe_t *h, int replica, int terms, double *out)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    Prop &P = *h->main;
    if (!out || replica < 0 || replica >= P.g.n_rep) return h->fail(QHFPE_EINVAL, "apply_rhs: bad replica or NULL output");
    cudaStream_t st = h->stream;
    const Model &M = *P.m;
    r = P.mixed ? closure_fill<float>(h, P, (float *)P.y, replica, 1) : closure_fill<double>(h, P, (double *)P.y, replica, 1);
    if (r != QHFPE_OK) return r;
    if (P.tc) {
        QH_CK(h, launch_potential_tc(P.g, (const float *)P.y, (float *)P.P, M.tcB, M.tcN, M.tcN + M.tab_n,
                                     M.tcN + 2 * M.tab_n, P.g.n_rep, h->tc_err, st));
        QH_CK(h, (launch_fused<float, true>(P.g, M.elems, M.f32(), (const float *)P.y, (const float *)P.y, P.y0,
                                           (float *)P.vA, nullptr, 0.0, 0, terms, replica, 1, st, (const float *)P.P,
                                           P.tq)));
    } else if (M.fused) {
        if (P.mixed)
            QH_CK(h, (launch_fused<float, true>(P.g, M.elems, M.f32(), (const float *)P.y, (const float *)P.y, P.y0,
                                               (float *)P.vA, nullptr, 0.0, 0, terms, replica, 1, st, nullptr, P.tq)));
        else
            QH_CK(h, (launch_fused<double, false>(P.g, M.elems, M.f64(), (const double *)P.y, (const double *)P.y,
                                                 nullptr, (double *)P.vA, nullptr, 0.0, 0, terms, replica, 1, st,
                                                 nullptr, P.tq)));
    } else if (P.mixed) {
        QH_CK(h, launch_potential<float>(P.g, M.t32(), (const float *)P.y, (float *)P.P, replica, 1, st));
        QH_CK(h, (launch_stage<float, true>(P.g, M.elems, (const float *)P.y, (const float *)P.P, (const float *)P.y,
                                            P.y0, (float *)P.vA, nullptr, 0.0, 0, terms, replica, 1, st)));
    } else {
        QH_CK(h, launch_potential<double>(P.g, M.t64(), (const double *)P.y, (double *)P.P, replica, 1, st));
        QH_CK(h, (launch_stage<double, false>(P.g, M.elems, (const double *)P.y, (const double *)P.P,
                                              (const double *)P.y, nullptr, (double *)P.vA, nullptr, 0.0, 0, terms,
                                              replica, 1, st)));
    }
    const size_t n = (size_t)P.g.n_elem * P.g.S * P.g.S * P.g.blk;
    r = ensure_scratch(h, n * 2 * sizeof(double));
    if (r != QHFPE_OK) return r;
    r = get_to_canonical(h, P, P.vA, nullptr, h->scratch, replica);
    if (r != QHFPE_OK) return r;
    QH_CK(h, cudaMemcpyAsync(out, h->scratch, n * 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    QH_CK(h, cudaStreamSynchronize(st));
    return check_timeout(h);
}

qhfpe_status qhfpe_trace(qhfpe_t *h, double *out)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    if (!out) return h->fail(QHFPE_EINVAL, "trace: NULL output");
    Prop &P = *h->main;
    r = ensure_trace(h, P, P.g.n_rep);
    if (r != QHFPE_OK) return r;
    set_sink_kernel<<<1, 1, 0, h->stream>>>(P.sink, P.trace_buf, 1, 0);
    QH_CK(h, cudaGetLastError());
    if (P.mixed) QH_CK(h, launch_trace<double>(P.g, P.y0, P.g.tier0_rep_stride, P.m->mu, P.sink, 0, P.partial, h->stream, P.m->trace_mu_q()));
    else QH_CK(h, launch_trace<double>(P.g, (const double *)P.y, P.g.rep_stride, P.m->mu, P.sink, 0, P.partial, h->stream, P.m->trace_mu_q()));
    QH_CK(h, cudaMemcpyAsync(out, P.trace_buf, (size_t)P.g.n_rep * 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    QH_CK(h, cudaStreamSynchronize(h->stream));
    return QHFPE_OK;
}

qhfpe_status qhfpe_set_dipole_table(qhfpe_t *h, const double *mu_table)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    Model &M = *h->model;
    cudaStream_t st = h->stream;
    const int S = M.S, nq = M.nq, N = M.np;
    if (!mu_table) {
        M.noncondon = false;
    } else {
        if (!fused_supported(N, S) || S > 3)
            return h->fail(QHFPE_EUNSUPPORTED, "set_dipole_table: coordinate-dependent dipoles need np in {32, 64, "
                                               "128, 256} and at most 3 states");
        const size_t nt = (size_t)S * S * nq * (N + 1);
        for (size_t x = 0; x < nt; ++x)
            if (!std::isfinite(mu_table[x])) return h->fail(QHFPE_EINVAL, "set_dipole_table: non-finite entry");
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < S; ++k)
                for (size_t x = 0; x < (size_t)nq * (N + 1); ++x)
                    if (mu_table[((size_t)j * S + k) * nq * (N + 1) + x] != mu_table[((size_t)k * S + j) * nq * (N + 1) + x])
                        return h->fail(QHFPE_EINVAL, "set_dipole_table: the table must be symmetric in (j, k)");
        // multipliers at r-grid mode m (the Nyquist mode takes the symmetric value, as the potential)
        auto T = [&](int a, int b, int i, int t) { return mu_table[(((size_t)a * S + b) * nq + i) * (N + 1) + t]; };
        auto ML = [&](int a, int b, int i, int m) {
            return m == -N / 2 ? 0.5 * (T(a, b, i, 0) + T(a, b, i, N)) : T(a, b, i, m + N / 2);
        };
        auto MR = [&](int a, int b, int i, int m) {
            return m == -N / 2 ? 0.5 * (T(a, b, i, 0) + T(a, b, i, N)) : T(a, b, i, N / 2 - m);
        };
        const size_t tn = (size_t)S * S * nq * N;
        std::vector<double> tab(2 * tn);
        std::vector<float> tab32(2 * tn);
        for (int a = 0; a < S; ++a)
            for (int b = 0; b < S; ++b)
                for (int i = 0; i < nq; ++i)
                    for (int pos = 0; pos < N; ++pos) {
                        const int kk = fused_fft_frequency(N, pos);
                        const int m = kk < N / 2 ? kk : kk - N;
                        const size_t o = (((size_t)a * S + b) * nq + i) * N + pos;
                        tab[o] = ML(a, b, i, m) / N;
                        tab[tn + o] = MR(a, b, i, m) / N;
                    }
        for (size_t x = 0; x < 2 * tn; ++x) tab32[x] = (float)tab[x];
        std::vector<double> muq((size_t)nq * S * S);
        for (int i = 0; i < nq; ++i)
            for (int a = 0; a < S; ++a)
                for (int b = 0; b < S; ++b) muq[((size_t)i * S + a) * S + b] = T(a, b, i, N / 2);
        if (!M.dip64) QH_CK(h, dalloc(&M.dip64, 2 * tn));
        if (!M.dip32) QH_CK(h, dalloc(&M.dip32, 2 * tn));
        if (!M.mu_q) QH_CK(h, dalloc(&M.mu_q, muq.size()));
        QH_CK(h, cudaMemcpyAsync(M.dip64, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        QH_CK(h, cudaMemcpyAsync(M.dip32, tab32.data(), tab32.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        QH_CK(h, cudaMemcpyAsync(M.mu_q, muq.data(), muq.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        QH_CK(h, cudaStreamSynchronize(st));
        M.noncondon = true;
    }
    // captured step graphs hold the trace's dipole arguments: capture them again on next use
    h->main->drop_graphs();
    for (auto &b : h->batches) b.second->drop_graphs();
    return QHFPE_OK;
}

qhfpe_status qhfpe_adiabatic_marginals(qhfpe_t *h, int replica, double *out)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    Prop &P = *h->main;
    if (!out || replica < 0 || replica >= P.g.n_rep)
        return h->fail(QHFPE_EINVAL, "adiabatic_marginals: bad replica or NULL output");
    const size_t n = 2 * (size_t)P.g.S * P.g.S * P.g.nq;
    r = ensure_scratch(h, n * sizeof(double));
    if (r != QHFPE_OK) return r;
    const double *tier0 = P.mixed ? P.y0 + (size_t)replica * P.g.tier0_rep_stride
                                  : (const double *)P.y + (size_t)replica * P.g.rep_stride;
    QH_CK(h, launch_marginals(P.g, tier0, P.m->adia, (double *)h->scratch, h->stream));
    QH_CK(h, cudaMemcpyAsync(out, h->scratch, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    QH_CK(h, cudaStreamSynchronize(h->stream));
    return QHFPE_OK;
}

qhfpe_status qhfpe_first_order_distribution(qhfpe_t *h, int n_t1, int t1_stride, const double *omega, int n_omega,
                                            double *out)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    if (!omega || !out || n_t1 < 1 || n_omega < 1 || t1_stride < 0 || (n_t1 > 1 && t1_stride < 1))
        return h->fail(QHFPE_EINVAL, "first_order_distribution: need n_t1 >= 1, t1_stride >= 1, n_omega >= 1 and "
                                     "non-NULL omega / out");
    for (int w = 0; w < n_omega; ++w)
        if (!std::isfinite(omega[w])) return h->fail(QHFPE_EINVAL, "first_order_distribution: non-finite omega");
    if (!h->have_eq)
        return h->fail(QHFPE_EINVAL, "first_order_distribution: no equilibrium state (call qhfpe_equilibrate or "
                                     "qhfpe_set_equilibrium)");
    cudaStream_t st = h->stream;
    Prop *B;
    if ((r = batch_prop(h, 1, &B)) != QHFPE_OK) return r;
    const Model &M = *B->m;
    const size_t n = (size_t)M.n_elem * M.S * M.S * B->g.blk;  // complex values of one canonical state
    // trapezoid weights over the t1 grid (the convention of the two-dimensional spectrum) times
    // cos / sin(omega t1)
    const double dt1 = (double)t1_stride * h->p.dt;
    std::vector<double> cs((size_t)n_t1 * 2 * n_omega);
    for (int a = 0; a < n_t1; ++a) {
        const double wgt = n_t1 == 1 ? 0.0 : ((a == 0 || a == n_t1 - 1) ? 0.5 * dt1 : dt1);
        for (int w = 0; w < n_omega; ++w) {
            cs[((size_t)a * 2) * n_omega + w] = wgt * std::cos(omega[w] * a * dt1);
            cs[((size_t)a * 2 + 1) * n_omega + w] = wgt * std::sin(omega[w] * a * dt1);
        }
    }
    struct Buf {
        double *p = nullptr;
        ~Buf() { if (p) cudaFree(p); }
    } x, acc_c, acc_s, res, coef;
    QH_CK(h, dalloc(&x.p, 2 * n));
    QH_CK(h, dalloc(&acc_c.p, 2 * n * n_omega));
    QH_CK(h, dalloc(&acc_s.p, 2 * n * n_omega));
    QH_CK(h, dalloc(&res.p, 2 * n * n_omega));
    QH_CK(h, dalloc(&coef.p, cs.size()));
    QH_CK(h, cudaMemcpyAsync(coef.p, cs.data(), cs.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    QH_CK(h, cudaMemsetAsync(acc_c.p, 0, 2 * n * n_omega * sizeof(double), st));
    QH_CK(h, cudaMemsetAsync(acc_s.p, 0, 2 * n * n_omega * sizeof(double), st));
    // X(0) = mu^x W_eq, then X(t1) = G(t1) X(0) sampled every t1_stride steps
    if ((r = set_from_canonical(h, *B, h->eq, 0, 1)) != QHFPE_OK) return r;
    if ((r = apply_dipole_prop(h, *B, QHFPE_COMMUTATOR, nullptr, 1, 1.0)) != QHFPE_OK) return r;
    for (int a = 0; a < n_t1; ++a) {
        if (a > 0 && (r = run_steps(h, *B, t1_stride, nullptr, 0)) != QHFPE_OK) return r;
        if ((r = get_to_canonical(h, *B, B->y, B->y0, x.p, 0)) != QHFPE_OK) return r;
        QH_CK(h, launch_fourier_accumulate(x.p, n, coef.p + (size_t)a * 2 * n_omega, n_omega, acc_c.p, acc_s.p, st));
    }
    if (!M.noncondon) {
        QH_CK(h, launch_first_order_combine(M.S, B->g.blk, M.n_elem, n_omega, M.mu, acc_c.p, acc_s.p, res.p, st));
    } else {
        // coordinate-dependent dipole: mu^-> and mu^<- are p-convolutions, applied through the batch's
        // dipole path to F(omega) = A_c + i A_s and F(-omega) = A_c - i A_s, then W' = i (mu^-> F(omega)
        // - mu^<- F(-omega)); x holds each input, out_w first the left part
        for (int w = 0; w < n_omega; ++w) {
            const double *ac = acc_c.p + 2 * n * w, *as = acc_s.p + 2 * n * w;
            double *out_w = res.p + 2 * n * w;
            QH_CK(h, launch_complex_combine(ac, as, 1.0, 0.0, 0.0, 1.0, x.p, n, st));
            if ((r = set_from_canonical(h, *B, x.p, 0, 1)) != QHFPE_OK) return r;
            if ((r = apply_dipole_prop(h, *B, QHFPE_LEFT, nullptr, 1, 1.0)) != QHFPE_OK) return r;
            if ((r = get_to_canonical(h, *B, B->y, B->y0, out_w, 0)) != QHFPE_OK) return r;
            QH_CK(h, launch_complex_combine(ac, as, 1.0, 0.0, 0.0, -1.0, x.p, n, st));
            if ((r = set_from_canonical(h, *B, x.p, 0, 1)) != QHFPE_OK) return r;
            if ((r = apply_dipole_prop(h, *B, QHFPE_RIGHT, nullptr, 1, 1.0)) != QHFPE_OK) return r;
            if ((r = get_to_canonical(h, *B, B->y, B->y0, x.p, 0)) != QHFPE_OK) return r;
            QH_CK(h, launch_complex_combine(out_w, x.p, 0.0, 1.0, 0.0, -1.0, out_w, n, st));
        }
    }
    QH_CK(h, cudaMemcpyAsync(out, res.p, 2 * n * n_omega * sizeof(double), cudaMemcpyDeviceToHost, st));
    QH_CK(h, cudaStreamSynchronize(st));
    return check_timeout(h);
}

namespace {

// The ground problem of the equilibration (Sec. III): U_00 alone with the full hierarchy, started
// from the classical Boltzmann distribution with unit trace.
qhfpe_status equilibrium_start(qhfpe_t *h, std::unique_ptr<Prop> &GP)
{
    const qhfpe_params &p = h->p;
    const int nq = p.nq, np = p.np, S = p.n_states;
    cudaStream_t st = h->stream;
    qhfpe_status r;
    if (!h->ground) {
        std::vector<double> U00((size_t)nq * (np + 1));
        for (int i = 0; i < nq; ++i)
            for (int t = 0; t <= np; ++t) U00[(size_t)i * (np + 1) + t] = h->U[(size_t)i * (np + 1) + t];
        const double zero = 0.0;
        h->ground.reset(new Model());
        // the state-input closure's network is for n_states pairs: the ground problem is closed by the
        // Eq. (GMFP) terminator
        r = build_model(h, *h->ground, 1, U00.data(), &zero,
                        p.closure == QHFPE_LEARNED_STATE ? (int)QHFPE_TERMINATOR : -1);
        if (r != QHFPE_OK) return r;
    }
    Model &G = *h->ground;
    r = make_prop(h, &G, 1, false, p.dt, GP);
    if (r != QHFPE_OK) return r;
    const size_t blk = (size_t)nq * np;
    const size_t gn = (size_t)G.n_elem * blk;
    std::vector<double> w0(2 * gn, 0.0);
    double norm = 0.0;
    const double dq = (p.q_max - p.q_min) / nq, dp = (p.p_max - p.p_min) / np;
    for (int i = 0; i < nq; ++i)
        for (int l = 0; l < np; ++l) {
            const double pl = p.p_min + l * dp;
            const double v = std::exp(-p.beta * (0.5 * pl * pl + h->U[(size_t)i * (np + 1) + np / 2]));
            w0[2 * ((size_t)i * np + l)] = v;
            norm += v;
        }
    norm *= dq * dp;
    for (size_t c = 0; c < blk; ++c) w0[2 * c] /= norm;
    const size_t full = (size_t)G.n_elem * S * S * blk;
    r = ensure_scratch(h, std::max(gn, full) * 2 * sizeof(double) + 64);
    if (r != QHFPE_OK) return r;
    QH_CK(h, cudaMemcpyAsync(h->scratch, w0.data(), gn * 2 * sizeof(double), cudaMemcpyHostToDevice, st));
    return set_from_canonical(h, *GP, h->scratch, 0, 1);
}

// ||L W|| / ||W|| of the ground problem's current state (2-norm over all elements; the closure slot
// is not part of the state): one right-hand side into vA, two norms, two scalars to the host.
qhfpe_status equilibrium_residual(qhfpe_t *h, Prop &GP, double *res)
{
    Model &G = *h->ground;
    cudaStream_t st = h->stream;
    qhfpe_status r = closure_fill<double>(h, GP, (double *)GP.y, 0, 1);
    if (r != QHFPE_OK) return r;
    if (G.fused) {
        QH_CK(h, (launch_fused<double, false>(GP.g, G.elems, G.f64(), (const double *)GP.y, (const double *)GP.y,
                                              nullptr, (double *)GP.vA, nullptr, 0.0, 0, QHFPE_TERM_ALL, 0, 1, st)));
    } else {
        QH_CK(h, launch_potential<double>(GP.g, G.t64(), (const double *)GP.y, (double *)GP.P, 0, 1, st));
        QH_CK(h, (launch_stage<double, false>(GP.g, G.elems, (const double *)GP.y, (const double *)GP.P,
                                              (const double *)GP.y, nullptr, (double *)GP.vA, nullptr, 0.0, 0,
                                              QHFPE_TERM_ALL, 0, 1, st)));
    }
    const size_t real = (size_t)G.n_elem * GP.g.elem_stride;
    QH_CK(h, launch_norm2((const double *)GP.vA, real, h->scratch, st));
    QH_CK(h, launch_norm2((const double *)GP.y, real, h->scratch + 1, st));
    double nn[2];
    QH_CK(h, cudaMemcpyAsync(nn, h->scratch, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    QH_CK(h, cudaStreamSynchronize(st));
    if (!std::isfinite(nn[0]) || !std::isfinite(nn[1])) return h->fail(QHFPE_ENUMERIC, "equilibrate: state not finite");
    *res = std::sqrt(nn[0] / nn[1]);
    return check_timeout(h);
}

// Embeds the ground problem's state in the 00 block of every element: the handle's equilibrium state,
// also written to every replica.
qhfpe_status equilibrium_embed(qhfpe_t *h, Prop &GP)
{
    const int S = h->p.n_states;
    const Model &G = *h->ground;
    const size_t blk = (size_t)h->p.nq * h->p.np;
    const size_t full = (size_t)G.n_elem * S * S * blk;
    cudaStream_t st = h->stream;
    if (!h->eq) QH_CK(h, cudaMalloc((void **)&h->eq, full * 2 * sizeof(double)));
    QH_CK(h, cudaMemsetAsync(h->eq, 0, full * 2 * sizeof(double), st));
    qhfpe_status r = get_to_canonical(h, GP, GP.y, nullptr, h->scratch, 0);
    if (r != QHFPE_OK) return r;
    QH_CK(h, cudaMemcpy2DAsync(h->eq, (size_t)S * S * blk * 2 * sizeof(double), h->scratch, blk * 2 * sizeof(double),
                               blk * 2 * sizeof(double), G.n_elem, cudaMemcpyDeviceToDevice, st));
    h->have_eq = true;
    r = set_from_canonical(h, *h->main, h->eq, 0, h->main->g.n_rep);
    if (r != QHFPE_OK) return r;
    QH_CK(h, cudaStreamSynchronize(st));
    return QHFPE_OK;
}

}  // namespace

qhfpe_status qhfpe_equilibrate(qhfpe_t *h, long n_steps, double *residual_out)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    if (n_steps < 0) return h->fail(QHFPE_EINVAL, "equilibrate: n_steps < 0");
    std::unique_ptr<Prop> GP;
    if ((r = equilibrium_start(h, GP)) != QHFPE_OK) return r;
    if ((r = run_steps(h, *GP, n_steps, nullptr, 0)) != QHFPE_OK) return r;
    double res = 0.0;
    if ((r = equilibrium_residual(h, *GP, &res)) != QHFPE_OK) return r;
    if (residual_out) *residual_out = res;
    return equilibrium_embed(h, *GP);
}

qhfpe_status qhfpe_equilibrate_tol(qhfpe_t *h, double t_max, double tol, long check_every, long *steps_taken,
                                   double *residual_out)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    if (!(t_max >= 0.0) || !std::isfinite(t_max) || !(tol > 0.0) || check_every < 1)
        return h->fail(QHFPE_EINVAL, "equilibrate_tol: need finite t_max >= 0, tol > 0, check_every >= 1");
    // the last step may end at most half a step past t_max
    const long max_steps = (long)std::floor(t_max / h->p.dt + 0.5);
    std::unique_ptr<Prop> GP;
    if ((r = equilibrium_start(h, GP)) != QHFPE_OK) return r;
    long done = 0;
    double res = 0.0;
    if ((r = equilibrium_residual(h, *GP, &res)) != QHFPE_OK) return r;
    while (res >= tol && done < max_steps) {
        const long n = std::min(check_every, max_steps - done);
        if ((r = run_steps(h, *GP, n, nullptr, 0)) != QHFPE_OK) return r;
        done += n;
        if ((r = equilibrium_residual(h, *GP, &res)) != QHFPE_OK) return r;
    }
    if (steps_taken) *steps_taken = done;
    if (residual_out) *residual_out = res;
    return equilibrium_embed(h, *GP);
}

qhfpe_status qhfpe_set_equilibrium(qhfpe_t *h, const double *src, int is_device)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    if (!src) return h->fail(QHFPE_EINVAL, "set_equilibrium: NULL source");
    const Model &M = *h->model;
    const size_t n = (size_t)M.n_elem * M.S * M.S * M.g.blk;
    if (!is_device && !finite_all(src, 2 * n)) return h->fail(QHFPE_ENUMERIC, "set_equilibrium: NaN/Inf");
    if (!h->eq) QH_CK(h, cudaMalloc((void **)&h->eq, n * 2 * sizeof(double)));
    QH_CK(h, cudaMemcpyAsync(h->eq, src, n * 2 * sizeof(double), is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             h->stream));
    QH_CK(h, cudaStreamSynchronize(h->stream));
    h->have_eq = true;
    return QHFPE_OK;
}

qhfpe_status qhfpe_response(qhfpe_t *h, const qhfpe_schedule *s, double *R_out)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    if (!s || !R_out) return h->fail(QHFPE_EINVAL, "response: NULL schedule or output");
    if (!h->have_eq) return h->fail(QHFPE_EINVAL, "response: no equilibrium state (call qhfpe_equilibrate or qhfpe_set_equilibrium)");
    if (s->n_t3 < 0) return h->fail(QHFPE_EINVAL, "response: n_t3 < 0");
    cudaStream_t st = h->stream;
    const long nt = s->n_t3 + 1;
    if (s->kind == QHFPE_LINEAR) {
        Prop *B;
        r = batch_prop(h, 1, &B);
        if (r != QHFPE_OK) return r;
        r = set_from_canonical(h, *B, h->eq, 0, 1);
        if (r != QHFPE_OK) return r;
        r = apply_dipole_prop(h, *B, QHFPE_COMMUTATOR, nullptr, 1, 1.0);
        if (r != QHFPE_OK) return r;
        r = ensure_trace(h, *B, nt);
        if (r != QHFPE_OK) return r;
        r = run_steps(h, *B, s->n_t3, B->trace_buf, nt);
        if (r != QHFPE_OK) return r;
        std::vector<double> tr(2 * nt);
        QH_CK(h, cudaMemcpyAsync(tr.data(), B->trace_buf, nt * 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        QH_CK(h, cudaStreamSynchronize(st));
        if ((r = check_timeout(h)) != QHFPE_OK) return r;
        for (long c = 0; c < nt; ++c) {  // R1 = i * Tr
            R_out[2 * c] = -tr[2 * c + 1];
            R_out[2 * c + 1] = tr[2 * c];
        }
        return QHFPE_OK;
    }
    if (s->kind != QHFPE_THIRD_ORDER) return h->fail(QHFPE_EINVAL, "response: unknown kind");
    if (s->n_t1 < 1 || s->t1_stride < 0 || s->n_t2 < 1 || !s->t2_steps)
        return h->fail(QHFPE_EINVAL, "response: bad third-order schedule");
    for (int b = 0; b < s->n_t2; ++b)
        if (s->t2_steps[b] < 0 || (b > 0 && s->t2_steps[b] < s->t2_steps[b - 1]))
            return h->fail(QHFPE_EINVAL, "response: t2_steps must be non-negative and ascending");
    const int n_paths = s->split_pathways ? 2 : 1;
    const int n1 = n_paths, n2 = n_paths * s->n_t1, n3 = n2 * s->n_t2;
    Prop *P1, *P2, *P3;
    if ((r = batch_prop(h, n1, &P1)) != QHFPE_OK) return r;
    if ((r = batch_prop(h, n2, &P2)) != QHFPE_OK) return r;
    if ((r = batch_prop(h, n3, &P3)) != QHFPE_OK) return r;
    // Equal replica counts share one cached batch (only when n_t1 = 1 or n_t2 = 1); the snapshot
    // copies then land on their own slots and are skipped.
    // phase 1: first interaction
    r = set_from_canonical(h, *P1, h->eq, 0, n1);
    if (r != QHFPE_OK) return r;
    if (s->split_pathways) {
        int zero = 0, one = 1;
        int *dev = nullptr;
        r = ensure_scratch(h, 2 * sizeof(int) + 16);
        if (r != QHFPE_OK) return r;
        dev = (int *)h->scratch;
        QH_CK(h, cudaMemcpyAsync(dev, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
        QH_CK(h, cudaMemcpyAsync(dev + 1, &one, sizeof(int), cudaMemcpyHostToDevice, st));
        if ((r = apply_dipole_prop(h, *P1, QHFPE_LEFT, dev, 1, 1.0)) != QHFPE_OK) return r;
        if ((r = apply_dipole_prop(h, *P1, QHFPE_RIGHT, dev + 1, 1, -1.0)) != QHFPE_OK) return r;
        QH_CK(h, cudaStreamSynchronize(st));
    } else {
        if ((r = apply_dipole_prop(h, *P1, QHFPE_COMMUTATOR, nullptr, 1, 1.0)) != QHFPE_OK) return r;
    }
    // phase 2: t1 propagation with snapshots
    for (int a = 0; a < s->n_t1; ++a) {
        if (a > 0 && s->t1_stride > 0) {
            if ((r = run_steps(h, *P1, s->t1_stride, nullptr, 0)) != QHFPE_OK) return r;
        }
        for (int pth = 0; pth < n_paths; ++pth)
            if ((r = copy_replica(h, *P1, pth, *P2, pth * s->n_t1 + a)) != QHFPE_OK) return r;
    }
    if ((r = apply_dipole_prop(h, *P2, QHFPE_COMMUTATOR, nullptr, n2, 1.0)) != QHFPE_OK) return r;
    // phase 3: t2 propagation with forks
    int done = 0;
    for (int b = 0; b < s->n_t2; ++b) {
        const int t2 = s->t2_steps[b];
        if (t2 > done) {
            if ((r = run_steps(h, *P2, t2 - done, nullptr, 0)) != QHFPE_OK) return r;
            done = t2;
        }
        for (int pth = 0; pth < n_paths; ++pth)
            for (int a = 0; a < s->n_t1; ++a)
                if ((r = copy_replica(h, *P2, pth * s->n_t1 + a, *P3, (pth * s->n_t2 + b) * s->n_t1 + a)) != QHFPE_OK)
                    return r;
    }
    if ((r = apply_dipole_prop(h, *P3, QHFPE_COMMUTATOR, nullptr, n3, 1.0)) != QHFPE_OK) return r;
    // phase 4: detection, every t3 job of the spectrum in one batch
    if ((r = ensure_trace(h, *P3, (size_t)n3 * nt)) != QHFPE_OK) return r;
    if ((r = run_steps(h, *P3, s->n_t3, P3->trace_buf, nt)) != QHFPE_OK) return r;
    std::vector<double> tr((size_t)n3 * nt * 2);
    QH_CK(h, cudaMemcpyAsync(tr.data(), P3->trace_buf, tr.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    QH_CK(h, cudaStreamSynchronize(st));
    if ((r = check_timeout(h)) != QHFPE_OK) return r;
    for (size_t c = 0; c < (size_t)n3 * nt; ++c) {  // R3 = i^3 Tr = -i Tr
        R_out[2 * c] = tr[2 * c + 1];
        R_out[2 * c + 1] = -tr[2 * c];
    }
    return QHFPE_OK;
}

qhfpe_status qhfpe_spectrum_absorption(qhfpe_t *h, const double *R1, long n_t, double dt, const double *omega,
                                       int n_omega, double *out)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    if (!R1 || !omega || !out || n_t < 1 || n_omega < 1) return h->fail(QHFPE_EINVAL, "spectrum_absorption: bad arguments");
    const size_t bytes = (2 * n_t + 2 * n_omega) * sizeof(double);
    if ((r = ensure_scratch(h, bytes)) != QHFPE_OK) return r;
    double *dR = h->scratch, *dw = dR + 2 * n_t, *dout = dw + n_omega;
    cudaStream_t st = h->stream;
    QH_CK(h, cudaMemcpyAsync(dR, R1, 2 * n_t * sizeof(double), cudaMemcpyHostToDevice, st));
    QH_CK(h, cudaMemcpyAsync(dw, omega, n_omega * sizeof(double), cudaMemcpyHostToDevice, st));
    QH_CK(h, launch_absorption(dR, n_t, dt, dw, n_omega, dout, st));
    QH_CK(h, cudaMemcpyAsync(out, dout, n_omega * sizeof(double), cudaMemcpyDeviceToHost, st));
    QH_CK(h, cudaStreamSynchronize(st));
    return QHFPE_OK;
}

qhfpe_status qhfpe_spectrum_2d(qhfpe_t *h, const double *R3, int n_t1, int n_t3, double dt1, double dt3,
                               const double *omega1, int n_omega1, const double *omega3, int n_omega3, double *nr,
                               double *re)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    if (!R3 || !omega1 || !omega3 || !nr || !re || n_t1 < 1 || n_t3 < 0 || n_omega1 < 1 || n_omega3 < 1)
        return h->fail(QHFPE_EINVAL, "spectrum_2d: bad arguments");
    const size_t nR = (size_t)n_t1 * (n_t3 + 1) * 2;
    const size_t nG = (size_t)n_omega3 * n_t1 * 2;
    const size_t nO = (size_t)n_omega1 * n_omega3;
    const size_t bytes = (nR + nG + n_omega1 + n_omega3 + 2 * nO) * sizeof(double);
    if ((r = ensure_scratch(h, bytes)) != QHFPE_OK) return r;
    double *dR = h->scratch, *dG = dR + nR, *dw1 = dG + nG, *dw3 = dw1 + n_omega1, *dnr = dw3 + n_omega3, *dre = dnr + nO;
    cudaStream_t st = h->stream;
    QH_CK(h, cudaMemcpyAsync(dR, R3, nR * sizeof(double), cudaMemcpyHostToDevice, st));
    QH_CK(h, cudaMemcpyAsync(dw1, omega1, n_omega1 * sizeof(double), cudaMemcpyHostToDevice, st));
    QH_CK(h, cudaMemcpyAsync(dw3, omega3, n_omega3 * sizeof(double), cudaMemcpyHostToDevice, st));
    QH_CK(h, launch_spectrum2d(dR, n_t1, n_t3, dt1, dt3, dw1, n_omega1, dw3, n_omega3, dnr, dre, dG, st));
    QH_CK(h, cudaMemcpyAsync(nr, dnr, nO * sizeof(double), cudaMemcpyDeviceToHost, st));
    QH_CK(h, cudaMemcpyAsync(re, dre, nO * sizeof(double), cudaMemcpyDeviceToHost, st));
    QH_CK(h, cudaStreamSynchronize(st));
    return QHFPE_OK;
}

qhfpe_status qhfpe_wait_selftest(qhfpe_t *h, int release, int limit_ms)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    if (limit_ms < 1 || limit_ms > 10000) return h->fail(QHFPE_EINVAL, "wait_selftest: limit_ms must be in [1, 10000]");
    int *buf = nullptr;
    QH_CK(h, cudaMalloc((void **)&buf, 2 * sizeof(int)));
    int init[2] = {release ? 1 : 0, 0};
    cudaError_t e = cudaMemcpyAsync(buf, init, sizeof(init), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_wait_flag(buf, (unsigned long long)limit_ms * 1000000ull, buf + 1, h->stream);
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, buf + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(buf);
    QH_CK(h, e);
    if (status == 2) return h->fail(QHFPE_ETIMEOUT, "wait_selftest: the device wait gave up (flag never set)");
    return status == 1 ? QHFPE_OK : h->fail(QHFPE_ECUDA, "wait_selftest: no status written");
}

qhfpe_status qhfpe_fp64_fma_rate(void *stream, int repeats, double *flops_per_s)
{
    if (!flops_per_s || repeats < 1 || repeats > 100) {
        qh_set_free_error("fp64_fma_rate: need repeats in [1, 100] and an output");
        return QHFPE_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = 8 * (sms > 0 ? sms : 1), n_iter = 4096;
    double *out = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void **)&out, (size_t)blocks * 256 * sizeof(double));
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = launch_dfma_rate(blocks, 64, out, st);  // warm-up
    float best = 0.0f;
    for (int r = 0; r < repeats && e == cudaSuccess; ++r) {
        e = cudaEventRecord(a, st);
        if (e == cudaSuccess) e = launch_dfma_rate(blocks, n_iter, out, st);
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && (best == 0.0f || ms < best)) best = ms;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (out) cudaFree(out);
    if (e != cudaSuccess || best <= 0.0f) {
        qh_set_free_error(std::string("fp64_fma_rate: ") + cudaGetErrorString(e));
        return QHFPE_ECUDA;
    }
    *flops_per_s = 2.0 * 64.0 * n_iter * (double)blocks * 256.0 / (best * 1e-3);
    return QHFPE_OK;
}

qhfpe_status qhfpe_tile_rows(const qhfpe_t *h, int *rows)
{
    if (!h || !rows) return QHFPE_EINVAL;
    *rows = h->main->tq;
    return QHFPE_OK;
}

qhfpe_status qhfpe_set_persistent(qhfpe_t *h, int on)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    h->persistent = on != 0;
    return QHFPE_OK;
}

qhfpe_status qhfpe_barrier_selftest(qhfpe_t *h, int withhold, int limit_ms)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    if (limit_ms < 1 || limit_ms > 10000) return h->fail(QHFPE_EINVAL, "barrier_selftest: limit_ms must be in [1, 10000]");
    unsigned *buf = nullptr;
    QH_CK(h, cudaMalloc((void **)&buf, 4 * sizeof(unsigned)));
    cudaError_t e = cudaMemsetAsync(buf, 0, 4 * sizeof(unsigned), h->stream);
    if (e == cudaSuccess)
        e = launch_barrier_selftest(buf, reinterpret_cast<int *>(buf + 2), (unsigned long long)limit_ms * 1000000ull,
                                    withhold != 0, h->stream);
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, buf + 2, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(buf);
    QH_CK(h, e);
    if (bad) return h->fail(QHFPE_ETIMEOUT, "barrier_selftest: the grid barrier wait gave up (a block never arrived)");
    return QHFPE_OK;
}

qhfpe_status qhfpe_stage_form(const qhfpe_t *h, int *form)
{
    if (!h || !form) return QHFPE_EINVAL;
    const Prop &P = *h->main;
    if (!P.tq) *form = -1;
    else if (P.form >= 0) *form = P.form;
    else *form = (P.mixed && !P.tc && fused_window_applies(P.g, QHFPE_TERM_ALL, false)) ? 1 : 0;  // pinned tile
    return QHFPE_OK;
}

qhfpe_status qhfpe_kernel_timing(qhfpe_t *h, int enable)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    h->timing.enabled = enable != 0;
    return QHFPE_OK;
}

qhfpe_status qhfpe_kernel_timing_read(qhfpe_t *h, long *launches, double *total_ms, int n_kinds)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    QH_CK(h, cudaStreamSynchronize(h->stream));
    Timing &T = h->timing;
    for (auto &pe : T.pending) {
        float ms = 0.f;
        QH_CK(h, cudaEventElapsedTime(&ms, pe.second.first, pe.second.second));
        T.launches[pe.first] += 1;
        T.ms[pe.first] += ms;
    }
    T.pending.clear();
    T.used = 0;
    for (int k = 0; k < n_kinds && k < QH_KINDS; ++k) {
        if (launches) launches[k] = T.launches[k];
        if (total_ms) total_ms[k] = T.ms[k];
        T.launches[k] = 0;
        T.ms[k] = 0.0;
    }
    return QHFPE_OK;
}

qhfpe_status qhfpe_closure_collect(qhfpe_t *h, int target_tier, double *stats_dev)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    const Model &M = *h->model;
    if (h->p.n_matsubara != 0) return h->fail(QHFPE_EINVAL, "closure_collect: needs n_matsubara = 0");
    if (!stats_dev || target_tier < 1 || target_tier > h->p.depth)
        return h->fail(QHFPE_EINVAL, "closure_collect: target tier must be in [1, depth]");
    // K = 0: element index = tier
    Prop &P = *h->main;
    const int t = target_tier;
    if (P.mixed) QH_CK(h, launch_closure_collect<float>(P.g, (const float *)P.y, t, t - 1, t - 2, stats_dev, h->stream));
    else QH_CK(h, launch_closure_collect<double>(P.g, (const double *)P.y, t, t - 1, t - 2, stats_dev, h->stream));
    (void)M;
    QH_CK(h, cudaStreamSynchronize(h->stream));
    return QHFPE_OK;
}

qhfpe_status qhfpe_closure_load(qhfpe_t *h, const float *weights, size_t n)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    if (h->p.closure != QHFPE_LEARNED) return h->fail(QHFPE_EINVAL, "closure_load: the handle was not created with QHFPE_LEARNED");
    if (!weights || n != QHFPE_CLOSURE_N_WEIGHTS) return h->fail(QHFPE_EINVAL, "closure_load: expected QHFPE_CLOSURE_N_WEIGHTS floats");
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(weights[i])) return h->fail(QHFPE_ENUMERIC, "closure_load: non-finite weight");
    if (!h->closure_w) QH_CK(h, cudaMalloc((void **)&h->closure_w, n * sizeof(float)));
    QH_CK(h, cudaMemcpyAsync(h->closure_w, weights, n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    QH_CK(h, launch_closure_infer(h->model->g, h->p.eta, h->closure_w, h->p.precision != QHFPE_FP64 ? 1 : 0, h->coef64,
                                  h->coef32, h->stream));
    QH_CK(h, cudaStreamSynchronize(h->stream));
    return QHFPE_OK;
}

size_t qhfpe_closure_state_n_weights(int n_states)
{
    return (n_states >= 1 && n_states <= 2) ? closure_state_n_weights(n_states) : 0;
}

qhfpe_status qhfpe_closure_state_load(qhfpe_t *h, const float *weights, size_t n)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    if (h->p.closure != QHFPE_LEARNED_STATE)
        return h->fail(QHFPE_EINVAL, "closure_state_load: the handle was not created with QHFPE_LEARNED_STATE");
    if (!weights || n != closure_state_n_weights(h->p.n_states))
        return h->fail(QHFPE_EINVAL, "closure_state_load: expected qhfpe_closure_state_n_weights(n_states) floats");
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(weights[i])) return h->fail(QHFPE_ENUMERIC, "closure_state_load: non-finite weight");
    for (size_t i = n - 3; i < n; ++i)
        if (!(weights[i] > 0.f)) return h->fail(QHFPE_EINVAL, "closure_state_load: the three scales must be positive");
    const size_t off = closure_state_prepared_offset(h->p.n_states);
    if (!h->state_w)
        QH_CK(h, cudaMalloc((void **)&h->state_w, (off + closure_state_prepared_floats(h->p.n_states)) * sizeof(float)));
    QH_CK(h, cudaMemcpyAsync(h->state_w, weights, n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    QH_CK(h, launch_closure_state_prepare(h->p.n_states, h->state_w, h->state_w + off, h->stream));
    QH_CK(h, cudaStreamSynchronize(h->stream));
    for (auto &kv : h->batches) kv.second->drop_graphs();
    h->main->drop_graphs();
    return QHFPE_OK;
}

qhfpe_status qhfpe_closure_state_collect(qhfpe_t *h, int target_tier, float *X_dev, float *Y_dev, long offset,
                                         long capacity, long *count_out)
{
    qhfpe_status r = check_handle(h);
    if (r != QHFPE_OK) return r;
    const Model &M = *h->model;
    Prop &P = *h->main;
    if (h->p.n_matsubara != 0 || h->p.precision != QHFPE_FP64 || h->p.n_states > 2)
        return h->fail(QHFPE_EINVAL, "closure_state_collect: needs n_matsubara = 0, QHFPE_FP64 and n_states <= 2");
    if (target_tier < 1 || target_tier > h->p.depth || !X_dev || !Y_dev || offset < 0 || capacity < offset)
        return h->fail(QHFPE_EINVAL, "closure_state_collect: invalid argument");
    // chain: the element of tier t is the one with n_0 = t
    auto elem_of = [&](int t) -> int {
        for (int e = 0; e < M.n_elem; ++e)
            if (M.hier[e][0] == t) return e;
        return -1;
    };
    const int et = elem_of(target_tier), et1 = elem_of(target_tier - 1), et2 = target_tier >= 2 ? elem_of(target_tier - 2) : -1;
    QH_CK(h, launch_closure_state_collect<double>(P.g, (const double *)P.y, et, et1, et2, h->p.eta, X_dev, Y_dev, offset,
                                                  capacity, h->stream));
    QH_CK(h, cudaStreamSynchronize(h->stream));
    if (count_out) *count_out = std::min<long>((long)P.g.n_rep * (long)P.g.blk, capacity - offset);
    return QHFPE_OK;
}

qhfpe_status qhfpe_closure_coefficients(const qhfpe_t *h, double *out)
{
    if (!h || !out) return QHFPE_EINVAL;
    if (h->sticky) return QHFPE_ESTATE;
    if (!h->coef64) return QHFPE_EINVAL;
    const size_t nc = (size_t)h->p.nq * h->p.np * QHFPE_CLOSURE_N_OUT;
    if (cudaMemcpy(out, h->coef64, nc * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return QHFPE_ECUDA;
    return QHFPE_OK;
}

}  // extern "C"

// ---- heterogeneous batch ---------------------------------------------------------------------------
// Members are handles sharing np, S and the precision (FP64 or MIXED); every Horner stage of all of
// them is one launch of the fused stage kernel over a device table of member descriptions (the
// members' own buffers, tables and step sizes), and whole steps are replayed from captured graphs.
struct qhfpe_batch {
    std::vector<qhfpe *> mem;
    bool mixed = false;
    int np = 0, S = 0, tq = 0;
    long blocks = 0;
    void *desc = nullptr;  // device MultiMember<float or double>[n]
    cudaGraphExec_t graphs[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [chunk][trace]
    void *pdesc = nullptr;      // persistent propagation: this propagator as a one-member batch
    int pdesc_tq = 0;           // its tile height
    unsigned *pbar = nullptr;   // barrier words (count, generation) and the give-up flag
    ~qhfpe_batch()
    {
        for (auto &a : graphs)
            for (auto &x : a)
                if (x) cudaGraphExecDestroy(x);
        if (desc) cudaFree(desc);
    }
};

namespace {

// descriptions of all members at tile height tq into b->desc (blocking copy); b->blocks set
template <typename T>
qhfpe_status batch_upload(qhfpe_batch *b, int tq)
{
    qhfpe *h0 = b->mem[0];
    std::vector<MultiMember<T>> d(b->mem.size());
    long blocks = 0;
    for (size_t m = 0; m < b->mem.size(); ++m) {
        Prop &P = *b->mem[m]->main;
        const Model &M = *P.m;
        MultiMember<T> &x = d[m];
        std::memset(&x, 0, sizeof(x));
        x.g = P.g;
        x.elems = M.elems;
        if constexpr (sizeof(T) == 4) x.tab = M.f32();
        else x.tab = M.f64();
        x.sc[0] = stage_scalars<T>(P.g, 0.0);
        for (int k = 1; k <= 4; ++k) x.sc[k] = stage_scalars<T>(P.g, P.dt / k);
        x.dt = P.dt;
        x.y = (T *)P.y;
        x.vA = (T *)P.vA;
        x.vB = (T *)P.vB;
        x.y0 = b->mixed ? P.y0 : nullptr;
        x.block0 = blocks;
        blocks += fused_blocks(P.g, tq);
    }
    if (blocks > 0x7fffffffL) return h0->fail(QHFPE_EUNSUPPORTED, "batch: more than 2^31 - 1 blocks per stage");
    if (!b->desc) QH_CK(h0, cudaMalloc(&b->desc, d.size() * sizeof(MultiMember<T>)));
    QH_CK(h0, cudaMemcpy(b->desc, d.data(), d.size() * sizeof(MultiMember<T>), cudaMemcpyHostToDevice));
    b->blocks = blocks;
    return QHFPE_OK;
}

qhfpe_status batch_launch(qhfpe_batch *b, int k, cudaStream_t st)
{
    qhfpe *h0 = b->mem[0];
    const int n = (int)b->mem.size();
    bool nonlinear = false;
    for (qhfpe *m : b->mem) nonlinear = nonlinear || m->main->g.c2 != 0.0;
    if (b->mixed)
        QH_CK(h0, (launch_fused_multi<float, true>(b->np, b->S, (const MultiMember<float> *)b->desc, n, k, b->tq,
                                                   b->blocks, nonlinear, st)));
    else
        QH_CK(h0, (launch_fused_multi<double, false>(b->np, b->S, (const MultiMember<double> *)b->desc, n, k, b->tq,
                                                     b->blocks, nonlinear, st)));
    return QHFPE_OK;
}

// the batch's tile height: every candidate evaluates every member's right-hand side (into its second
// stage buffer, which holds no data between steps) a few times, timed with CUDA events
qhfpe_status batch_autotune(qhfpe_batch *b, cudaStream_t st)
{
    qhfpe *h0 = b->mem[0];
    int tmax = fused_max_rows(b->np, b->S, b->mixed ? 4 : 8), nq_max = 1;
    for (qhfpe *h : b->mem) nq_max = std::max(nq_max, h->main->g.nq);
    tmax = std::min(tmax, nq_max);
    auto upload = [&](int tq) { return b->mixed ? batch_upload<float>(b, tq) : batch_upload<double>(b, tq); };
    if (const char *env = std::getenv("QHFPE_TILE_ROWS")) {
        const int t = std::atoi(env);
        if (t >= 1 && t <= tmax) {
            b->tq = t;
            return upload(t);
        }
    }
    cudaEvent_t e0, e1;
    QH_CK(h0, cudaEventCreate(&e0));
    QH_CK(h0, cudaEventCreate(&e1));
    float best = 1e30f;
    int best_tq = 1;
    static const int cand[] = {1, 2, 3, 4, 5, 6, 8, 12, 16};
    for (int tq : cand) {
        if (tq > tmax) break;
        qhfpe_status r = upload(tq);
        if (r != QHFPE_OK) return r;
        b->tq = tq;
        float ms = 0.f;
        for (int rep = 0; rep < 4; ++rep) {
            if (rep == 1) QH_CK(h0, cudaEventRecord(e0, st));
            r = batch_launch(b, 0, st);
            if (r != QHFPE_OK) return r;
        }
        QH_CK(h0, cudaEventRecord(e1, st));
        QH_CK(h0, cudaEventSynchronize(e1));
        QH_CK(h0, cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            best_tq = tq;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tq = best_tq;
    return upload(best_tq);
}

qhfpe_status batch_step_once(qhfpe_batch *b, bool record, cudaStream_t st)
{
    for (int k = 4; k >= 1; --k) {
        qhfpe_status r = batch_launch(b, k, st);
        if (r != QHFPE_OK) return r;
    }
    if (record)
        for (qhfpe *h : b->mem) {
            Prop &P = *h->main;
            if (b->mixed)
                QH_CK(h, launch_trace<double>(P.g, P.y0, P.g.tier0_rep_stride, P.m->mu, P.sink, 1, P.partial, st,
                                              P.m->trace_mu_q()));
            else
                QH_CK(h, launch_trace<double>(P.g, (const double *)P.y, P.g.rep_stride, P.m->mu, P.sink, 1, P.partial,
                                              st, P.m->trace_mu_q()));
        }
    return QHFPE_OK;
}

}  // namespace

void qh_set_free_error(const std::string &msg) { g_create_error = msg; }


extern "C" {

qhfpe_status qhfpe_batch_create(qhfpe_t *const *members, int n, qhfpe_batch_t **out)
{
    if (!out || !members || n < 1) return QHFPE_EINVAL;
    *out = nullptr;
    qhfpe *h0 = members[0];
    qhfpe_status r = check_handle(h0);
    if (r != QHFPE_OK) return r;
    std::unique_ptr<qhfpe_batch> b(new qhfpe_batch());
    for (int m = 0; m < n; ++m) {
        qhfpe *h = members[m];
        if ((r = check_handle(h)) != QHFPE_OK) return h ? r : h0->fail(QHFPE_EINVAL, "batch_create: NULL member");
        for (int a = 0; a < m; ++a)
            if (members[a] == h) return h0->fail(QHFPE_EINVAL, "batch_create: a handle appears twice");
        const Prop &P = *h->main;
        if (P.tc || h->p.precision == QHFPE_MIXED_BF16X3)
            return h0->fail(QHFPE_EUNSUPPORTED, "batch_create: the tensor-core form is not batched");
        if (P.m->closure_slot >= 0)
            return h0->fail(QHFPE_EUNSUPPORTED, "batch_create: the learned closure is not batched");
        if (!P.m->fused) return h0->fail(QHFPE_EUNSUPPORTED, "batch_create: no fused stage kernel for this np and S");
        if (m == 0) {
            b->mixed = P.mixed;
            b->np = P.g.np;
            b->S = P.g.S;
        } else if (P.mixed != b->mixed || P.g.np != b->np || P.g.S != b->S) {
            return h0->fail(QHFPE_EINVAL, "batch_create: members must share np, the number of states and the precision");
        }
        b->mem.push_back(h);
    }
    *out = b.release();
    return QHFPE_OK;
}

qhfpe_status qhfpe_batch_step(qhfpe_batch_t *b, long n_steps, double *const *trace_out)
{
    if (!b || b->mem.empty()) return QHFPE_EINVAL;
    qhfpe *h0 = b->mem[0];
    qhfpe_status r;
    for (qhfpe *h : b->mem)
        if ((r = check_handle(h)) != QHFPE_OK) return r;
    if (n_steps < 0) return h0->fail(QHFPE_EINVAL, "batch_step: n_steps < 0");
    // every member's earlier work (on its own stream) is complete before the batch touches its buffers
    for (qhfpe *h : b->mem) QH_CK(h, cudaStreamSynchronize(h->stream));
    cudaStream_t st = h0->stream;
    if (!b->tq && n_steps > 0 && (r = batch_autotune(b, st)) != QHFPE_OK) return r;
    const bool record = trace_out != nullptr;
    const long stride = n_steps + 1;
    if (record)
        for (qhfpe *h : b->mem) {
            Prop &P = *h->main;
            if ((r = ensure_trace(h, P, (size_t)P.g.n_rep * stride)) != QHFPE_OK) return r;
            set_sink_kernel<<<1, 1, 0, st>>>(P.sink, P.trace_buf, stride, 0);
            QH_CK(h, cudaGetLastError());
            if (b->mixed)
                QH_CK(h, launch_trace<double>(P.g, P.y0, P.g.tier0_rep_stride, P.m->mu, P.sink, 1, P.partial, st,
                                              P.m->trace_mu_q()));
            else
                QH_CK(h, launch_trace<double>(P.g, (const double *)P.y, P.g.rep_stride, P.m->mu, P.sink, 1, P.partial,
                                              st, P.m->trace_mu_q()));
        }
    long done = 0;
    while (done < n_steps) {
        const int chunk = (n_steps - done >= kGraphChunk) ? 1 : 0;
        const int len = chunk ? kGraphChunk : 1;
        cudaGraphExec_t &ge = b->graphs[chunk][record ? 1 : 0];
        if (!ge) {
            cudaGraph_t graph;
            QH_CK(h0, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            r = QHFPE_OK;
            for (int s = 0; s < len && r == QHFPE_OK; ++s) r = batch_step_once(b, record, st);
            cudaError_t e = cudaStreamEndCapture(st, &graph);
            if (r != QHFPE_OK) return r;
            QH_CK(h0, e);
            e = cudaGraphInstantiate(&ge, graph, 0);
            cudaGraphDestroy(graph);
            QH_CK(h0, e);
        }
        QH_CK(h0, cudaGraphLaunch(ge, st));
        done += len;
    }
    if (record)
        for (size_t m = 0; m < b->mem.size(); ++m) {
            Prop &P = *b->mem[m]->main;
            if (trace_out[m])
                QH_CK(h0, cudaMemcpyAsync(trace_out[m], P.trace_buf, (size_t)P.g.n_rep * stride * 2 * sizeof(double),
                                          cudaMemcpyDeviceToHost, st));
        }
    QH_CK(h0, cudaStreamSynchronize(st));
    return QHFPE_OK;
}

qhfpe_status qhfpe_batch_tile_rows(const qhfpe_batch_t *b, int *rows)
{
    if (!b || !rows) return QHFPE_EINVAL;
    *rows = b->tq;
    return QHFPE_OK;
}

qhfpe_status qhfpe_batch_destroy(qhfpe_batch_t *b)
{
    if (!b) return QHFPE_EINVAL;
    if (!b->mem.empty()) cudaStreamSynchronize(b->mem[0]->stream);
    delete b;
    return QHFPE_OK;
}

}  // extern "C"
