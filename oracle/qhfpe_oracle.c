/*
 * qhfpe_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the multi-state quantum hierarchical Fokker-Planck equation
 * (MS-QHFPE) of Ikeda & Tanimura (2017).  It exists so that the CUDA library can be checked against
 * something written directly from the paper.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it; the product library never does, and the two share no code,
 * headers, tables or constant generators.
 *
 * Every function states the passage it follows.  Readings of points the paper leaves open:
 *   - grid: x_i = x_min + i*dx, dx = (x_max - x_min)/n (end point excluded); r-grid conjugate to p:
 *     dr = 2*pi/(np*dp), r_m = m*dr, m = -np/2 .. np/2-1 (hbar = m = omega_0 = 1, Sec. III);
 *   - the caller tabulates the diabatic surfaces as T_jk[i][t] = U_jk(q_i + (t - np/2)*dr/2),
 *     t = 0..np, so U(q + r_m/2) = T[m + np/2] and U(q - r_m/2) = T[np/2 - m];
 *   - the Nyquist mode m = -np/2 uses the symmetric value (T[0] + T[np])/2 on both sides, so the
 *     commutator of a diagonal block vanishes there and real diagonal blocks stay real;
 *   - bath derivatives along p are 4th-order central differences on the periodic p axis (the
 *     potential kernel is a circulant, i.e. already periodic in p; the wrap keeps the trace exactly
 *     conserved by the population terms);
 *   - the q boundary is open (zero ghost cells) unless periodic_q is set;
 *   - time stepping is classic RK4 (for this linear autonomous equation it equals the degree-4 Taylor
 *     polynomial of the propagator, which is what the 4th-order exponential integrator of Sec. III
 *     amounts to at fixed step);
 *   - Matsubara coefficients and the delta-term are the residues of the Drude correlation function.
 * Parity-relevant derivations are written out beside each function.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double complex cplx;

/* Term mask for oq_rhs: lets the tests isolate each part of Eq. (heom). */
enum {
    OQ_KINETIC = 1,     /* -(p/m) dW/dq,                      Eq. (quantum-liouvillian), K term      */
    OQ_POTENTIAL = 2,   /* -(i/hbar)[U, W] in Wigner space,   Eq. (quantum-liouvillian), U terms     */
    OQ_DAMPING = 4,     /* -(sum_k n_k gamma_k) W + c_delta Phi^2 W,  Eq. (heom) first line           */
    OQ_TIER_UP = 8,     /* -sum_k Phi W^(n+e_k) (or the terminator, Eq. (GMFP)),  Eq. (heom)          */
    OQ_TIER_DOWN = 16,  /* Lambda^(1) and c_k Phi couplings to W^(n-e_k),  Eq. (heom) lines 3-4       */
    OQ_ALL = 31
};

typedef struct {
    int S, nq, np;
    double q_min, q_max, p_min, p_max;
    const double *U_table; /* [S][S][nq][np+1] */
    const double *mu;      /* [S][S] */
    double eta, gamma, beta;
    int n_matsubara;       /* K: modes k = 0..K */
    int high_temperature;  /* Sec. II high-temperature Drude case: c_0 = eta/beta, K = 0 */
    int use_cdelta;
    int depth;             /* N */
    int closure;           /* 0: truncate, 1: terminator of Eq. (GMFP) */
    int periodic_q;
    double dt;
    const double *closure_coef; /* closure 2 (learned): [nq][np][10] coefficients, see oq_rhs */
    double v_c2;           /* system side of the system-bath coupling, V(q) = q + v_c2 q^2 (Sec. II) */
} oq_params;

typedef struct {
    oq_params P;
    double *U;     /* own copy of the table */
    double mu[64];
    int n_modes;
    double gam[32], r[32], c[32], cdelta;
    int n_elem;
    int *idx;      /* [n_elem][n_modes] */
    int *up, *dn;  /* [n_elem][n_modes], -1 when absent */
    double dq, dp, dr;
    double *qv, *pv;
    cplx *AL, *AR; /* circulant kernels [S][S][nq][np], index d = (l - l') mod np */
    double *coef;  /* learned-closure coefficients [nq][np][10] (own copy) or NULL */
} oq_ctx;

/* ------------------------------------------------------------------------------------------------
 * Bath coefficients, Eqs. (bath-correlation), (expansion-of-bath-*), (Drude-J), (psi-Drude).
 * Psi_B(t) = 2 int J(w)/w cos(wt) dw = m*zeta*gamma*exp(-gamma t)  ->  gamma_0 = gamma, r_0 = zeta.
 * C_B(t) for the Drude J(w) by contour integration:
 *   pole w = i*gamma:     c_0 = (zeta*gamma/2) cot(beta*gamma/2)
 *   poles w = i*nu_k:     gamma_k = nu_k = 2 pi k / beta,  c_k = (2 zeta gamma^2/beta)/(nu_k^2 - gamma^2)
 *   remainder as delta:   c_delta = zeta/beta - c_0 - sum_{k=1..K} c_k  (the infinite sum equals zeta/beta)
 * High-temperature case (end of Sec. II): K = 0, c_0 = zeta/beta, no delta term.
 * ---------------------------------------------------------------------------------------------- */
int oq_bath_coefficients(double eta, double gamma, double beta, int K, int high_t, int use_cdelta,
                         double *gam, double *r, double *c, double *cdelta)
{
    if (K < 0) return -1;
    if (high_t && K != 0) return -1;
    gam[0] = gamma;
    r[0] = eta;
    if (high_t) {
        c[0] = eta / beta;
        *cdelta = 0.0;
        return 0;
    }
    c[0] = 0.5 * eta * gamma / tan(0.5 * beta * gamma);
    double sum = c[0];
    for (int k = 1; k <= K; ++k) {
        double nu = 2.0 * M_PI * k / beta;
        gam[k] = nu;
        r[k] = 0.0;
        c[k] = (2.0 * eta * gamma * gamma / beta) / (nu * nu - gamma * gamma);
        sum += c[k];
    }
    *cdelta = use_cdelta ? (eta / beta - sum) : 0.0;
    return 0;
}

/* ------------------------------------------------------------------------------------------------
 * Hierarchy index set {n in N^(K+1) : |n| <= N}, Eq. (heom).  Order: by tier |n| ascending; inside a
 * tier, lexicographic on (n_0, ..., n_K) with n_0 largest first.  Count C(N+K+1, K+1).
 * ---------------------------------------------------------------------------------------------- */
static int count_elements(int modes, int depth)
{
    /* C(depth + modes, modes) */
    double v = 1.0;
    for (int i = 1; i <= modes; ++i) v = v * (depth + i) / i;
    return (int)(v + 0.5);
}

static void enumerate_tier(int modes, int remaining, int pos, int *cur, int *out, int *count)
{
    if (pos == modes - 1) {
        cur[pos] = remaining;
        memcpy(out + (size_t)(*count) * modes, cur, sizeof(int) * modes);
        (*count)++;
        return;
    }
    for (int v = remaining; v >= 0; --v) {
        cur[pos] = v;
        enumerate_tier(modes, remaining - v, pos + 1, cur, out, count);
    }
}

int oq_hierarchy(int modes, int depth, int *idx_out /* may be NULL */)
{
    int total = count_elements(modes, depth);
    if (!idx_out) return total;
    int cur[64];
    int count = 0;
    for (int t = 0; t <= depth; ++t) enumerate_tier(modes, t, 0, cur, idx_out, &count);
    return count;
}

static int find_element(const oq_ctx *C, const int *v)
{
    for (int e = 0; e < C->n_elem; ++e) {
        if (memcmp(C->idx + (size_t)e * C->n_modes, v, sizeof(int) * C->n_modes) == 0) return e;
    }
    return -1;
}

/* ------------------------------------------------------------------------------------------------
 * Context: grid, coefficients, hierarchy, and the circulant potential kernels of
 * Eq. (quantum-liouvillian).  Discretising W(p) = (1/2pi) int dr e^{-ipr} rho(q+r/2, q-r/2) on the
 * p-grid and its conjugate r-grid turns U(p,q) * W into a circulant along p:
 *   (U * W)(p_l) = sum_l' A_L[l - l'] W(p_l'),  A_L[d] = (1/np) sum_m U(q + r_m/2) exp(-2 pi i m d/np)
 * and the right product (rho U) into the same form with U(q - r_m/2).
 * ---------------------------------------------------------------------------------------------- */
static double table_at(const oq_ctx *C, int j, int k, int i, int t)
{
    const oq_params *P = &C->P;
    return C->U[(((size_t)j * P->S + k) * P->nq + i) * (P->np + 1) + t];
}

static double UL_mode(const oq_ctx *C, int j, int s, int i, int m)
{
    int np = C->P.np;
    if (m == -np / 2) return 0.5 * (table_at(C, j, s, i, 0) + table_at(C, j, s, i, np));
    return table_at(C, j, s, i, m + np / 2);
}

static double UR_mode(const oq_ctx *C, int s, int k, int i, int m)
{
    int np = C->P.np;
    if (m == -np / 2) return 0.5 * (table_at(C, s, k, i, 0) + table_at(C, s, k, i, np));
    return table_at(C, s, k, i, np / 2 - m);
}

void oq_destroy(oq_ctx *C)
{
    if (!C) return;
    free(C->U); free(C->idx); free(C->up); free(C->dn);
    free(C->qv); free(C->pv); free(C->AL); free(C->AR); free(C->coef);
    free(C);
}

oq_ctx *oq_create(const oq_params *P)
{
    if (P->S < 1 || P->S > 8 || P->nq < 1 || P->np < 2 || (P->np & 1) || P->depth < 0) return NULL;
    if ((P->closure == 1 || P->closure == 2) && P->n_matsubara != 0) return NULL; /* K = 0 closures only */
    if (P->closure == 2 && !P->closure_coef) return NULL;
    if (P->v_c2 != 0.0 && P->closure != 0) return NULL; /* the Eq. (GMFP) terminator assumes V(q) = q */
    oq_ctx *C = (oq_ctx *)calloc(1, sizeof(oq_ctx));
    C->P = *P;
    int S = P->S, nq = P->nq, np = P->np;
    size_t tsz = (size_t)S * S * nq * (np + 1);
    C->U = (double *)malloc(sizeof(double) * tsz);
    memcpy(C->U, P->U_table, sizeof(double) * tsz);
    for (int a = 0; a < S * S; ++a) C->mu[a] = P->mu ? P->mu[a] : 0.0;
    C->P.U_table = C->U;
    C->P.mu = C->mu;
    if (P->closure == 2) {
        C->coef = (double *)malloc(sizeof(double) * (size_t)nq * np * 10);
        memcpy(C->coef, P->closure_coef, sizeof(double) * (size_t)nq * np * 10);
        C->P.closure_coef = C->coef;
    }

    if (P->n_matsubara < 0 || P->n_matsubara > 30) { oq_destroy(C); return NULL; }
    C->n_modes = P->n_matsubara + 1;
    if (oq_bath_coefficients(P->eta, P->gamma, P->beta, P->n_matsubara, P->high_temperature,
                             P->use_cdelta, C->gam, C->r, C->c, &C->cdelta) != 0) {
        oq_destroy(C);
        return NULL;
    }
    C->n_elem = oq_hierarchy(C->n_modes, P->depth, NULL);
    C->idx = (int *)malloc(sizeof(int) * C->n_elem * C->n_modes);
    oq_hierarchy(C->n_modes, P->depth, C->idx);
    C->up = (int *)malloc(sizeof(int) * C->n_elem * C->n_modes);
    C->dn = (int *)malloc(sizeof(int) * C->n_elem * C->n_modes);
    int v[64];
    for (int e = 0; e < C->n_elem; ++e) {
        for (int k = 0; k < C->n_modes; ++k) {
            memcpy(v, C->idx + (size_t)e * C->n_modes, sizeof(int) * C->n_modes);
            v[k] += 1;
            C->up[e * C->n_modes + k] = find_element(C, v);
            v[k] -= 2;
            C->dn[e * C->n_modes + k] = (v[k] >= 0) ? find_element(C, v) : -1;
        }
    }

    C->dq = (P->q_max - P->q_min) / nq;
    C->dp = (P->p_max - P->p_min) / np;
    C->dr = 2.0 * M_PI / (np * C->dp);
    C->qv = (double *)malloc(sizeof(double) * nq);
    C->pv = (double *)malloc(sizeof(double) * np);
    for (int i = 0; i < nq; ++i) C->qv[i] = P->q_min + i * C->dq;
    for (int l = 0; l < np; ++l) C->pv[l] = P->p_min + l * C->dp;

    size_t ksz = (size_t)S * S * nq * np;
    C->AL = (cplx *)malloc(sizeof(cplx) * ksz);
    C->AR = (cplx *)malloc(sizeof(cplx) * ksz);
#pragma omp parallel for collapse(3) schedule(static)
    for (int j = 0; j < S; ++j)
        for (int s = 0; s < S; ++s)
            for (int i = 0; i < nq; ++i)
                for (int d = 0; d < np; ++d) {
                    cplx aL = 0.0, aR = 0.0;
                    for (int m = -np / 2; m < np / 2; ++m) {
                        /* exp(-2 pi i m d / np), angle reduced exactly modulo np */
                        long md = ((long)m * d) % np;
                        if (md < 0) md += np;
                        double ang = -2.0 * M_PI * (double)md / np;
                        cplx ph = cos(ang) + I * sin(ang);
                        aL += UL_mode(C, j, s, i, m) * ph;
                        aR += UR_mode(C, j, s, i, m) * ph;
                    }
                    size_t o = (((size_t)j * S + s) * nq + i) * np + d;
                    C->AL[o] = aL / np;
                    C->AR[o] = aR / np;
                }
    return C;
}

int oq_n_elements(const oq_ctx *C) { return C->n_elem; }
int oq_n_modes(const oq_ctx *C) { return C->n_modes; }
void oq_get_hierarchy(const oq_ctx *C, int *idx) { memcpy(idx, C->idx, sizeof(int) * C->n_elem * C->n_modes); }
void oq_get_coefficients(const oq_ctx *C, double *gam, double *r, double *c, double *cdelta)
{
    for (int k = 0; k < C->n_modes; ++k) { gam[k] = C->gam[k]; r[k] = C->r[k]; c[k] = C->c[k]; }
    *cdelta = C->cdelta;
}

/* ------------------------------------------------------------------------------------------------
 * Finite differences.
 * dW/dq: 5th-order upwind scheme of Sec. III (stencil chosen by the sign of p), zero ghost cells
 * (or periodic wrap).  d/dp and d^2/dp^2 for the bath terms: 4th-order central, periodic along p.
 * ---------------------------------------------------------------------------------------------- */
static cplx Wq(const oq_ctx *C, const cplx *blk, int i, int l)
{
    int nq = C->P.nq, np = C->P.np;
    if (i < 0 || i >= nq) {
        if (!C->P.periodic_q) return 0.0;
        i = ((i % nq) + nq) % nq;
    }
    return blk[(size_t)i * np + l];
}

static cplx dq_upwind(const oq_ctx *C, const cplx *blk, int i, int l)
{
    double p = C->pv[l];
    cplx s;
    if (p < 0.0) {
        s = 2.0 * Wq(C, blk, i + 3, l) - 15.0 * Wq(C, blk, i + 2, l) + 60.0 * Wq(C, blk, i + 1, l)
          - 20.0 * Wq(C, blk, i, l) - 30.0 * Wq(C, blk, i - 1, l) + 3.0 * Wq(C, blk, i - 2, l);
    } else {
        s = -3.0 * Wq(C, blk, i + 2, l) + 30.0 * Wq(C, blk, i + 1, l) + 20.0 * Wq(C, blk, i, l)
          - 60.0 * Wq(C, blk, i - 1, l) + 15.0 * Wq(C, blk, i - 2, l) - 2.0 * Wq(C, blk, i - 3, l);
    }
    return s / (60.0 * C->dq);
}

/* X at column l of a row, wrapped periodically along p; optionally multiplied by p_l (for d/dp of
 * p*W).  The potential kernel already makes the discrete p axis periodic (it is a circulant), and the
 * wrapped differences keep the trace exactly conserved by the population terms. */
static cplx Xp(const oq_ctx *C, const cplx *row, int l, int times_p)
{
    int np = C->P.np;
    l = ((l % np) + np) % np;
    return times_p ? C->pv[l] * row[l] : row[l];
}

static cplx dp_central(const oq_ctx *C, const cplx *row, int l, int times_p)
{
    return (Xp(C, row, l - 2, times_p) - 8.0 * Xp(C, row, l - 1, times_p)
          + 8.0 * Xp(C, row, l + 1, times_p) - Xp(C, row, l + 2, times_p)) / (12.0 * C->dp);
}

/* Learned closure (K = 0 chain): the correction to the terminator's W^(N+1) at column l of row i, the
 * local linear combination  sum_{b=-2..2} c_b(q_i, p_l) W^N(p_{l+b}) + c_{5+b}(q_i, p_l) W^(N-1)(p_{l+b})
 * (p wrapped periodically; the W^(N-1) part is absent at N = 0). */
static cplx closure_value(const oq_ctx *C, const cplx *rowN, const cplx *rowNm1, int i, int l)
{
    int np = C->P.np;
    l = ((l % np) + np) % np;
    const double *c = C->coef + ((size_t)i * np + l) * 10;
    cplx v = 0.0;
    for (int b = -2; b <= 2; ++b) {
        int lb = ((l + b) % np + np) % np;
        v += c[2 + b] * rowN[lb];
        if (rowNm1) v += c[7 + b] * rowNm1[lb];
    }
    return v;
}

static cplx dp_closure(const oq_ctx *C, const cplx *rowN, const cplx *rowNm1, int i, int l)
{
    return (closure_value(C, rowN, rowNm1, i, l - 2) - 8.0 * closure_value(C, rowN, rowNm1, i, l - 1)
          + 8.0 * closure_value(C, rowN, rowNm1, i, l + 1) - closure_value(C, rowN, rowNm1, i, l + 2)) / (12.0 * C->dp);
}

static cplx dpp_central(const oq_ctx *C, const cplx *row, int l)
{
    return (-Xp(C, row, l - 2, 0) + 16.0 * Xp(C, row, l - 1, 0) - 30.0 * Xp(C, row, l, 0)
            + 16.0 * Xp(C, row, l + 1, 0) - Xp(C, row, l + 2, 0)) / (12.0 * C->dp * C->dp);
}

/* d^2 W/dp dq at (q_i, p_l): 4th-order central differences along q (zero ghost cells, or periodic)
 * and along p (periodic), the q-difference taken first. */
static cplx dq_central(const oq_ctx *C, const cplx *blk, int i, int l)
{
    return (Wq(C, blk, i - 2, l) - 8.0 * Wq(C, blk, i - 1, l) + 8.0 * Wq(C, blk, i + 1, l) - Wq(C, blk, i + 2, l))
           / (12.0 * C->dq);
}

static cplx dpq_central(const oq_ctx *C, const cplx *blk, int i, int l)
{
    int np = C->P.np;
    cplx v[5];
    for (int b = -2; b <= 2; ++b) v[b + 2] = dq_central(C, blk, i, ((l + b) % np + np) % np);
    return (v[0] - 8.0 * v[1] + 8.0 * v[3] - v[4]) / (12.0 * C->dp);
}

/* ------------------------------------------------------------------------------------------------
 * Right-hand side of Eq. (heom) with the linear-coupling operators of Sec. II:
 *   Phi = -d/dp, Psi = q, Lambda^(1) = -p/m, Lambda^(2) = 0  (so only m = e_k survives in the sum,
 *   with binomial weight n_k), giving
 *   dW^n_jk/dt = -p dW^n_jk/dq
 *               - i sum_s [ (U_js * W^n_sk) - (U_sk^* * W^n_js) ]
 *               - (sum_k n_k gamma_k) W^n_jk + c_delta d^2W^n_jk/dp^2
 *               + sum_k dW^(n+e_k)_jk/dp
 *               + sum_k n_k gamma_k ( r_k p W^(n-e_k)_jk + c_k dW^(n-e_k)_jk/dp ).
 * Nonlinear coupling V(q) = q + c2 q^2 (Sec. II keeps V general; with hbar = m = 1).  From the
 * definitions there -- Phi = i (V(p,q) - V*(p,q)) *, Psi = (V(p,q) + V*(p,q))/2 *, K = p d/dq,
 * Lambda^(l) = (Psi^x)^l K with the commutator A^x B = AB - BA -- and r <-> i d/dp under the Wigner
 * transform along p:  V(q + r/2) - V(q - r/2) = r phi(q),  phi(q) = 1 + 2 c2 q, and
 * (V(q + r/2) + V(q - r/2))/2 = V(q) + c2 r^2/4, so
 *   Phi        = -phi(q) d/dp,
 *   Psi        = V(q) - (c2/4) d^2/dp^2,
 *   Lambda^(1) = [Psi, p d/dq] = -p phi(q) - (c2/2) d^2/dp dq,
 *   Lambda^(2) = [Psi, Lambda^(1)] = c2 phi(q) d/dp,   Lambda^(l >= 3) = 0,
 *   Phi^2      = phi(q)^2 d^2/dp^2.
 * In Eq. (heom) the sum over m then keeps |m| = 1 (weight n_k) and |m| = 2 (weight n!/(m!(n-m)!)
 * gamma^m r^m: C(n_k, 2) gamma_k^2 r_k^2 for m = 2 e_k, n_k n_l gamma_k gamma_l r_k r_l for
 * m = e_k + e_l).  c2 = 0 gives back the linear form above exactly.  Closure: truncation only.
 * At the deepest tier with the terminator closure (Eq. (GMFP), K = 0), the missing W^(N+1) in the
 * tier-up term is replaced by r_0 p W^N + c_0 dW^N/dp, i.e. the term becomes
 *   d/dp (r_0 p W^N) + c_0 d^2 W^N/dp^2.
 * With the learned closure (K = 0) it is the terminator's term plus d/dp of closure_value (see there):
 * the network supplies a local correction to Eq. (GMFP).
 * State layout: [n_elem][S][S][nq][np] complex.
 * ---------------------------------------------------------------------------------------------- */
/* One row of the right-hand side above: element e, pair (j, k), q index i, all p; out[np]. */
static void rhs_row(const oq_ctx *C, const cplx *W, int e, int j, int k, int i, cplx *out, int terms)
{
    const oq_params *P = &C->P;
    int S = P->S, nq = P->nq, np = P->np, M = C->n_modes;
    size_t blk = (size_t)nq * np;
    size_t elem = (size_t)S * S * blk;
    const int *n = C->idx + (size_t)e * M;
    int tier = 0;
    double ngam = 0.0;
    for (int a = 0; a < M; ++a) { tier += n[a]; ngam += n[a] * C->gam[a]; }
    const cplx *Wjk = W + e * elem + ((size_t)j * S + k) * blk;
    const cplx *row = Wjk + (size_t)i * np;
    const double c2 = P->v_c2;
    const double phi = 1.0 + 2.0 * c2 * C->qv[i];   /* Phi = -phi d/dp */
    for (int l = 0; l < np; ++l) {
        cplx acc = 0.0;
        if (terms & OQ_KINETIC) acc += -C->pv[l] * dq_upwind(C, Wjk, i, l);
        if (terms & OQ_POTENTIAL) {
            cplx pot = 0.0;
            for (int s = 0; s < S; ++s) {
                const cplx *Wsk = W + e * elem + ((size_t)s * S + k) * blk + (size_t)i * np;
                const cplx *Wjs = W + e * elem + ((size_t)j * S + s) * blk + (size_t)i * np;
                const cplx *aL = C->AL + (((size_t)j * S + s) * nq + i) * np;
                const cplx *aR = C->AR + (((size_t)s * S + k) * nq + i) * np;
                for (int lp = 0; lp < np; ++lp) {
                    int d = ((l - lp) % np + np) % np;
                    pot += aL[d] * Wsk[lp] - aR[d] * Wjs[lp];
                }
            }
            acc += -I * pot;
        }
        if (terms & OQ_DAMPING) {
            acc += -ngam * row[l];
            if (C->cdelta != 0.0) acc += C->cdelta * phi * phi * dpp_central(C, row, l);
        }
        if (terms & OQ_TIER_UP) {
            for (int a = 0; a < M; ++a) {
                int u = C->up[e * M + a];
                if (u >= 0) {
                    const cplx *urow = W + u * elem + ((size_t)j * S + k) * blk + (size_t)i * np;
                    acc += phi * dp_central(C, urow, l, 0);
                } else if (P->closure == 1 && tier == P->depth) {
                    acc += C->r[0] * dp_central(C, row, l, 1) + C->c[0] * dpp_central(C, row, l);
                } else if (P->closure == 2 && tier == P->depth) {
                    int dn = C->dn[e * M + a];
                    const cplx *rowm1 = dn >= 0 ? W + dn * elem + ((size_t)j * S + k) * blk + (size_t)i * np : NULL;
                    acc += C->r[0] * dp_central(C, row, l, 1) + C->c[0] * dpp_central(C, row, l);
                    acc += dp_closure(C, row, rowm1, i, l);
                }
            }
        }
        if (terms & OQ_TIER_DOWN) {
            for (int a = 0; a < M; ++a) {
                int dn = C->dn[e * M + a];
                if (dn < 0) continue;
                const cplx *drow = W + dn * elem + ((size_t)j * S + k) * blk + (size_t)i * np;
                double w = n[a] * C->gam[a];
                acc += w * (C->r[a] * phi * C->pv[l] * drow[l] + C->c[a] * phi * dp_central(C, drow, l, 0));
                if (c2 != 0.0 && C->r[a] != 0.0) {  /* the d^2/dp dq part of -r_k Lambda^(1) */
                    const cplx *dblk = W + dn * elem + ((size_t)j * S + k) * blk;
                    acc += w * C->r[a] * 0.5 * c2 * dpq_central(C, dblk, i, l);
                }
            }
            /* |m| = 2: -(n!/(m!(n-m)!)) gamma^m r^m Lambda^(2) W^(n-m), Lambda^(2) = c2 phi d/dp */
            if (c2 != 0.0) {
                int v[64];
                for (int a = 0; a < M; ++a)
                    for (int b = a; b < M; ++b) {
                        double wgt;
                        if (a == b) wgt = 0.5 * n[a] * (n[a] - 1) * C->gam[a] * C->gam[a] * C->r[a] * C->r[a];
                        else wgt = (double)n[a] * n[b] * C->gam[a] * C->gam[b] * C->r[a] * C->r[b];
                        if (wgt == 0.0) continue;
                        memcpy(v, n, sizeof(int) * M);
                        v[a] -= 1;
                        v[b] -= 1;
                        if (v[a] < 0 || v[b] < 0) continue;
                        int d2 = find_element(C, v);
                        const cplx *drow = W + d2 * elem + ((size_t)j * S + k) * blk + (size_t)i * np;
                        acc += -wgt * c2 * phi * dp_central(C, drow, l, 0);
                    }
            }
        }
        out[l] = acc;
    }
}

void oq_rhs(const oq_ctx *C, const cplx *W, cplx *dW, int terms)
{
    int S = C->P.S, nq = C->P.nq, np = C->P.np;
    size_t blk = (size_t)nq * np;
    size_t elem = (size_t)S * S * blk;
#pragma omp parallel for collapse(4) schedule(static)
    for (int e = 0; e < C->n_elem; ++e)
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < S; ++k)
                for (int i = 0; i < nq; ++i)
                    rhs_row(C, W, e, j, k, i, dW + e * elem + ((size_t)j * S + k) * blk + (size_t)i * np, terms);
}

/* The same right-hand side at n_rows selected rows only (rows[4 r .. 4 r + 3] = e, j, k, i); out is
 * [n_rows][np].  For checking a full-size state at sampled rows without the whole evaluation. */
int oq_rhs_rows(const oq_ctx *C, const cplx *W, const int *rows, int n_rows, cplx *out, int terms)
{
    int S = C->P.S, nq = C->P.nq, np = C->P.np;
    for (int r = 0; r < n_rows; ++r) {
        const int *x = rows + 4 * r;
        if (x[0] < 0 || x[0] >= C->n_elem || x[1] < 0 || x[1] >= S || x[2] < 0 || x[2] >= S || x[3] < 0 || x[3] >= nq)
            return -1;
    }
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < n_rows; ++r) {
        const int *x = rows + 4 * r;
        rhs_row(C, W, x[0], x[1], x[2], x[3], out + (size_t)r * np, terms);
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------------
 * Observables, Eqs. (R1), (R3): Tr{mu X} = sum_jk mu_kj int dq dp X^(0)_jk(p,q) (tier 0 only).
 * ---------------------------------------------------------------------------------------------- */
void oq_trace(const oq_ctx *C, const cplx *W, double *out /* re, im */)
{
    int S = C->P.S;
    size_t blk = (size_t)C->P.nq * C->P.np;
    cplx tr = 0.0;
    for (int j = 0; j < S; ++j)
        for (int k = 0; k < S; ++k) {
            double m = C->mu[k * S + j];
            if (m == 0.0) continue;
            cplx s = 0.0;
            const cplx *b = W + ((size_t)j * S + k) * blk;
            for (size_t x = 0; x < blk; ++x) s += b[x];
            tr += m * s;
        }
    tr *= C->dq * C->dp;
    out[0] = creal(tr);
    out[1] = cimag(tr);
}

/* Classic RK4 (see header comment), n_steps steps in place; trace_out (may be NULL) gets
 * Tr{mu W^(0)} before the first step and after every step: 2*(n_steps+1) doubles. */
void oq_step(const oq_ctx *C, cplx *W, long n_steps, double *trace_out)
{
    size_t n = (size_t)C->n_elem * C->P.S * C->P.S * C->P.nq * C->P.np;
    cplx *k1 = (cplx *)malloc(sizeof(cplx) * n), *k2 = (cplx *)malloc(sizeof(cplx) * n);
    cplx *k3 = (cplx *)malloc(sizeof(cplx) * n), *k4 = (cplx *)malloc(sizeof(cplx) * n);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * n);
    double dt = C->P.dt;
    if (trace_out) oq_trace(C, W, trace_out);
    for (long s = 0; s < n_steps; ++s) {
        oq_rhs(C, W, k1, OQ_ALL);
        for (size_t x = 0; x < n; ++x) tmp[x] = W[x] + 0.5 * dt * k1[x];
        oq_rhs(C, tmp, k2, OQ_ALL);
        for (size_t x = 0; x < n; ++x) tmp[x] = W[x] + 0.5 * dt * k2[x];
        oq_rhs(C, tmp, k3, OQ_ALL);
        for (size_t x = 0; x < n; ++x) tmp[x] = W[x] + dt * k3[x];
        oq_rhs(C, tmp, k4, OQ_ALL);
        for (size_t x = 0; x < n; ++x) W[x] += (dt / 6.0) * (k1[x] + 2.0 * k2[x] + 2.0 * k3[x] + k4[x]);
        if (trace_out) oq_trace(C, W, trace_out + 2 * (s + 1));
    }
    free(k1); free(k2); free(k3); free(k4); free(tmp);
}

/* ------------------------------------------------------------------------------------------------
 * Dipole super-operators (Sec. III, Condon approximation so mu(p,q) is a constant matrix and the
 * convolution with it is a plain product):  side 1: mu^-> W = mu W;  side 2: mu^<- W = W mu;
 * side 3: mu^x W = mu^-> W - mu^<- W.  Applied to every hierarchy element.
 * ---------------------------------------------------------------------------------------------- */
void oq_apply_dipole(const oq_ctx *C, cplx *W, int side)
{
    int S = C->P.S;
    size_t blk = (size_t)C->P.nq * C->P.np;
    size_t elem = (size_t)S * S * blk;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * elem);
    for (int e = 0; e < C->n_elem; ++e) {
        cplx *We = W + e * elem;
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < S; ++k)
                for (size_t x = 0; x < blk; ++x) {
                    cplx acc = 0.0;
                    cplx left = 0.0, right = 0.0;
                    for (int l = 0; l < S; ++l) {
                        left += C->mu[j * S + l] * We[((size_t)l * S + k) * blk + x];
                        right += We[((size_t)j * S + l) * blk + x] * C->mu[l * S + k];
                    }
                    if (side == 1) acc = left;
                    else if (side == 2) acc = right;
                    else acc = left - right;
                    tmp[((size_t)j * S + k) * blk + x] = acc;
                }
        memcpy(We, tmp, sizeof(cplx) * elem);
    }
    free(tmp);
}

/* ------------------------------------------------------------------------------------------------
 * Equilibrium (Sec. III protocol): the ground surface U_00 alone with the full hierarchy is
 * propagated from the classical Boltzmann distribution exp(-beta(p^2/2 + U_00(q))), normalised to
 * unit trace, for n_steps RK4 steps; the result fills the 00 block of every hierarchy element of
 * W_out ([n_elem][S][S][nq][np], other blocks zero).  residual = ||L W|| / ||W|| (2-norm over the
 * whole hierarchy) of the final state.
 * ---------------------------------------------------------------------------------------------- */
void oq_equilibrate(const oq_ctx *C, long n_steps, cplx *W_out, double *residual)
{
    const oq_params *P = &C->P;
    int nq = P->nq, np = P->np, S = P->S;
    oq_params g = *P;
    g.S = 1;
    double *U00 = (double *)malloc(sizeof(double) * nq * (np + 1));
    for (int i = 0; i < nq; ++i)
        for (int t = 0; t <= np; ++t) U00[i * (np + 1) + t] = table_at(C, 0, 0, i, t);
    double mu1 = 0.0;
    g.U_table = U00;
    g.mu = &mu1;
    oq_ctx *G = oq_create(&g);
    size_t blk = (size_t)nq * np;
    size_t n = (size_t)G->n_elem * blk;
    cplx *W = (cplx *)calloc(n, sizeof(cplx));
    double norm = 0.0;
    for (int i = 0; i < nq; ++i)
        for (int l = 0; l < np; ++l) {
            double e = 0.5 * G->pv[l] * G->pv[l] + table_at(G, 0, 0, i, np / 2);
            W[(size_t)i * np + l] = exp(-P->beta * e);
            norm += exp(-P->beta * e);
        }
    norm *= G->dq * G->dp;
    for (size_t x = 0; x < blk; ++x) W[x] /= norm;
    oq_step(G, W, n_steps, NULL);
    cplx *LW = (cplx *)malloc(sizeof(cplx) * n);
    oq_rhs(G, W, LW, OQ_ALL);
    double a = 0.0, b = 0.0;
    for (size_t x = 0; x < n; ++x) {
        a += creal(LW[x] * conj(LW[x]));
        b += creal(W[x] * conj(W[x]));
    }
    if (residual) *residual = sqrt(a / b);
    size_t elem = (size_t)S * S * blk;
    memset(W_out, 0, sizeof(cplx) * elem * C->n_elem);
    for (int e = 0; e < C->n_elem; ++e) memcpy(W_out + e * elem, W + e * blk, sizeof(cplx) * blk);
    free(LW); free(W); free(U00);
    oq_destroy(G);
}

int oq_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
