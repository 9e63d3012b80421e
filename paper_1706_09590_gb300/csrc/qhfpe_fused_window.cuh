// Fused right-hand-side stage, q-window form (FP32 state, np = 128, one or two electronic states): the
// same Horner stage of Eq. (heom) as fused_stage_kernel, organised so that each warp waits on global
// memory a few times per block instead of several times per p-row.
//
// A block is (replica, hierarchy element, tile of TQ q rows) with all S x S blocks; each of its four
// warps owns one unit = (electronic pair, RG = 4 consecutive q rows), a lane holding four consecutive p
// values.
//   1. window  the warp loads the RG + 6 q rows its 5th-order upwind stencil reads (rows outside the grid
//              are zero, or wrap for a periodic q axis) in two batches of five, forms the kinetic term
//              -p dW/dq of its RG rows in registers and writes its own rows into the FFT buffer;
//   2. phase A the potential term (FFT along p, r-space mixing with the p-diagonal bath terms, inverse
//              FFT) in shared memory, as in fused_stage_kernel;
//   3. rows    per q row, the loads of every tier neighbour and of the Horner base y are issued
//              together, then the tier couplings, the p-stencil of the tier-up/down sum (shuffles), the
//              potential term from shared memory and out = y + h L.
// The kinetic term of the unit's rows waits in shared memory (each lane reads back only what it wrote)
// so that no registers are held across phase A.
// Requirements (checked by the launcher): every lane's four p values have one sign, at most six tier
// neighbours per element, the potential term computed here (all terms).
#pragma once
#include "qhfpe_fused_kernel.cuh"

namespace {

constexpr int WIN_RG = 4;       // q rows per warp
constexpr int WIN_MAXNB = 6;    // tier neighbours of an element (at most)
constexpr int WIN_WB = 5;       // window rows loaded per batch
constexpr int WIN_BLOCKS = 5;   // blocks per SM the register budget is set for

template <int S> struct WinTile { static constexpr int TQ = 4 * WIN_RG / (S * S); };

// byte offset of the per-warp kinetic-term buffers: after the FFT buffer and its twiddles
// (fused_smem_bytes), rounded up to 128 bytes; each warp keeps RG rows x 2 planes x 128 floats
template <int NP, int S, int TQ>
__host__ __device__ constexpr size_t win_kin_offset()
{
    return ((((size_t)(TQ * S * S * NP + ((TQ * S * S * NP) >> 4) + 1) + NP) * 2 * sizeof(float) + 127) / 128) * 128;
}
constexpr size_t WIN_KIN_BYTES = (FTHREADS / 32) * WIN_RG * 2 * 128 * sizeof(float);

template <int NP, int S, bool MIXED>
__global__ void __launch_bounds__(FTHREADS, WIN_BLOCKS)
fused_window_kernel(GridInfo g, const ElemInfo *__restrict__ elems, FusedTables<float> tab, StageScalars<float> sc,
                    const float *__restrict__ v_in, const float *y, const double *y0, float *v_out, double *y0_out,
                    double h, int mode, int rep0, int n_rep)
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    using T = float;
    using C = float2;
    constexpr int S2 = S * S;
    constexpr int TQ = WinTile<S>::TQ;
    constexpr int RG = WIN_RG;
    constexpr int VEC = 4;
    static_assert(NP == 32 * VEC, "one p row per warp");
    static_assert(S2 * (TQ / RG) == FTHREADS / 32, "one unit per warp");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *X = reinterpret_cast<C *>(smem_raw);  // [TQ * S2][NP], padded (pad16)
    C *tw = X + pad16(TQ * S2 * NP) + 1;     // [NP]

    const int nq = g.nq;
    const unsigned bid = blockIdx.x;
    const int e = bid % g.n_elem;
    const int rep = rep0 + (bid / g.n_elem) % n_rep;
    const int tile = bid / (g.n_elem * n_rep);
    const int i0 = tile * TQ;
    const int rows = min(TQ, nq - i0);
    const size_t blk = g.blk;
    const size_t ebase = (size_t)rep * g.rep_stride + (size_t)e * g.elem_stride;

    __shared__ long long nb_off[WIN_MAXNB];
    __shared__ T nb_wg[WIN_MAXNB], nb_wa[WIN_MAXNB];
    __shared__ int s_cnt[4];
    __shared__ T s_ngam;
    __shared__ __align__(16) T pgrid[NP];
    __shared__ __align__(16) T s_lpp[NP];
    if (threadIdx.x == 0) {
        const ElemInfo &E = elems[e];
        int n = 0;
        for (int a = 0; a < E.n_up; ++a, ++n) {
            nb_off[n] = (long long)(E.up[a] - e) * (long long)g.elem_stride;
            nb_wg[n] = (T)1;
            nb_wa[n] = (T)0;
        }
        for (int pass = 0; pass < 2; ++pass) {
            for (int a = 0; a < E.n_dn; ++a) {
                if ((E.wr[a] != 0.0) != (pass == 1)) continue;
                nb_off[n] = (long long)(E.dn[a] - e) * (long long)g.elem_stride;
                nb_wg[n] = (T)E.wc[a];
                nb_wa[n] = (T)E.wr[a];
                ++n;
            }
            if (pass == 0) s_cnt[1] = n;
        }
        s_cnt[0] = E.n_up;
        s_cnt[2] = n;
        s_cnt[3] = E.terminator;
        s_ngam = (T)E.ngam;
    }
    for (int t = threadIdx.x; t < NP; t += FTHREADS) {
        tw[t] = C{tab.tw[2 * t], tab.tw[2 * t + 1]};
        pgrid[t] = (T)(g.p_min + t * g.dp);
        s_lpp[t] = tab.lpp[t];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pr = warp % S2;                 // this warp's electronic pair
    const int rg = warp / S2;                 // its row group inside the tile
    const int ia = i0 + rg * RG;              // first q row of the unit
    const int l0 = lane * VEC;
    T pcol[VEC];
    ldv<T, VEC>(pgrid + l0, pcol);
    const bool neg = pcol[0] < (T)0;          // one sign per lane (launcher's requirement)
    // upwind taps at offsets -3..+3 (one end zero): p < 0 reads -2..+3, p >= 0 reads -3..+2
    T ck[7];
    {
        const T cneg[7] = {0, 3, -30, -20, 60, -15, 2};
        const T cpos[7] = {-2, 15, -60, 20, 30, -3, 0};
#pragma unroll
        for (int t = 0; t < 7; ++t) ck[t] = neg ? cneg[t] : cpos[t];
    }
    T pk[VEC];  // -p / (60 dq)
#pragma unroll
    for (int v = 0; v < VEC; ++v) pk[v] = -(pcol[v] * sc.fkin);

    asm volatile("griddepcontrol.wait;" ::: "memory");

    const size_t poff = ebase + (size_t)pr * 2 * blk;
    float *kbuf = reinterpret_cast<float *>(smem_raw + win_kin_offset<NP, S, TQ>()) + (size_t)warp * RG * 2 * NP;

    // ---- 1. window: kinetic term of the unit's rows, own rows into the FFT buffer ------------------
    const T *Vre = v_in + poff, *Vim = Vre + blk;
    T kr[RG][VEC], ki[RG][VEC];
#pragma unroll
    for (int r = 0; r < RG; ++r)
#pragma unroll
        for (int v = 0; v < VEC; ++v) kr[r][v] = ki[r][v] = (T)0;
#pragma unroll
    for (int b0 = 0; b0 < RG + 6; b0 += WIN_WB) {
        constexpr int NB = WIN_WB;
        T wr_[NB][VEC], wi_[NB][VEC];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (b0 + b >= RG + 6) break;
            int ii = ia - 3 + b0 + b;
            bool ok = ii >= 0 && ii < nq;
            if (!ok && g.periodic_q) {
                ii = ii < 0 ? ii + nq : ii - nq;
                ok = ii >= 0 && ii < nq;
            }
            if (ok) {
                ldv<T, VEC>(Vre + (size_t)ii * NP + l0, wr_[b]);
                ldv<T, VEC>(Vim + (size_t)ii * NP + l0, wi_[b]);
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) wr_[b][v] = wi_[b][v] = (T)0;
            }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int t = b0 + b;  // window row: q row ia - 3 + t
            if (t >= RG + 6) break;
#pragma unroll
            for (int r = 0; r < RG; ++r) {
                const int tap = t - r;  // offset tap - 3 from output row r
                if (tap >= 0 && tap < 7) {
                    v_axpy<VEC>(kr[r], ck[tap], wr_[b]);
                    v_axpy<VEC>(ki[r], ck[tap], wi_[b]);
                }
            }
            if (t >= 3 && t < 3 + RG) {  // an own row: into the FFT buffer (rows past the grid are zero)
                const int lr = rg * RG + t - 3;
                C *xb = X + pad16((lr * S2 + pr) * NP + l0);
#pragma unroll
                for (int v = 0; v < VEC; ++v) xb[v] = C{wr_[b][v], wi_[b][v]};
            }
        }
    }
#pragma unroll
    for (int r = 0; r < RG; ++r) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            kr[r][v] *= pk[v];
            ki[r][v] *= pk[v];
        }
        stv<T, VEC>(kbuf + (size_t)(2 * r) * NP + l0, kr[r]);
        stv<T, VEC>(kbuf + (size_t)(2 * r + 1) * NP + l0, ki[r]);
    }

    // ---- 2. phase A: potential term and the p-diagonal bath terms, in place in X ------------------
    __syncthreads();
    potential_in_place<T, NP, S>(X, tw, tab, nq, i0, rows, sc.fdelta + (s_cnt[3] != 0 ? sc.fterm : (T)0), s_ngam,
                                 s_lpp);

    // ---- 3. per q row: tier couplings, p-stencil, update -------------------------------------------
    const int n_up = s_cnt[0], n_d0 = s_cnt[1], n_nb = s_cnt[2];
    const bool term = s_cnt[3] != 0;
    const T inv12dp = sc.inv12dp;
    const bool tier0 = MIXED && e == 0;
#pragma unroll
    for (int r = 0; r < RG; ++r) {
        const int i = ia + r;
        if (i >= nq || i >= i0 + rows) continue;  // warp-uniform
        const size_t o = poff + (size_t)i * NP + l0;
        // the Horner base and the tier neighbours, three at a time, each batch's loads in flight together
        T br[VEC], bi[VEC];
        double b0r[VEC], b0i[VEC];
        const size_t o0 = (size_t)rep * g.tier0_rep_stride + (size_t)pr * 2 * blk + (size_t)i * NP + l0;
        if (mode != 0) {
            if (tier0) {
                ldv<double, VEC>(y0 + o0, b0r);
                ldv<double, VEC>(y0 + o0 + blk, b0i);
            } else {
                ldv<T, VEC>(y + o, br);
                ldv<T, VEC>(y + o + blk, bi);
            }
        }
        T gr[VEC], gi[VEC], hr[VEC], hi[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) gr[v] = gi[v] = hr[v] = hi[v] = (T)0;
#pragma unroll
        for (int a0 = 0; a0 < WIN_MAXNB; a0 += 3) {
            T xr[3][VEC], xi[3][VEC];
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (a0 + b < n_nb) {
                    const T *u = v_in + (long long)o + nb_off[a0 + b];
                    ldv<T, VEC>(u, xr[b]);
                    ldv<T, VEC>(u + blk, xi[b]);
                }
            }
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int a = a0 + b;
                if (a < n_up) {
                    v_add<VEC>(gr, xr[b]);
                    v_add<VEC>(gi, xi[b]);
                } else if (a < n_d0) {
                    v_axpy<VEC>(gr, nb_wg[a], xr[b]);
                    v_axpy<VEC>(gi, nb_wg[a], xi[b]);
                } else if (a < n_nb) {
                    v_axpy<VEC>(gr, nb_wg[a], xr[b]);
                    v_axpy<VEC>(gi, nb_wg[a], xi[b]);
                    v_axpy<VEC>(hr, nb_wa[a], xr[b]);
                    v_axpy<VEC>(hi, nb_wa[a], xi[b]);
                }
            }
        }
        T ar[VEC], ai[VEC];
        ldv<T, VEC>(kbuf + (size_t)(2 * r) * NP + l0, ar);
        ldv<T, VEC>(kbuf + (size_t)(2 * r + 1) * NP + l0, ai);
        if (n_d0 < n_nb) {
            v_fma<VEC>(ar, pcol, hr);
            v_fma<VEC>(ai, pcol, hi);
        }
        if (term) {  // d/dp (r_0 p W) of the Eq. (GMFP) terminator: the centre row again
            T wr[VEC], wi[VEC], r0p[VEC];
            ldv<T, VEC>(Vre + (size_t)i * NP + l0, wr);
            ldv<T, VEC>(Vim + (size_t)i * NP + l0, wi);
#pragma unroll
            for (int v = 0; v < VEC; ++v) r0p[v] = sc.r0 * pcol[v];
            v_fma<VEC>(gr, r0p, wr);
            v_fma<VEC>(gi, r0p, wi);
        }
        if (n_nb > 0 || term) {  // 4th-order central d/dp of G, periodic p, neighbours through the warp
            T er[VEC + 4], ei[VEC + 4];
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                er[v + 2] = gr[v];
                ei[v + 2] = gi[v];
            }
            const int left = (lane + 31) & 31, right = (lane + 1) & 31;
            er[0] = __shfl_sync(0xffffffffu, gr[VEC - 2], left);
            er[1] = __shfl_sync(0xffffffffu, gr[VEC - 1], left);
            ei[0] = __shfl_sync(0xffffffffu, gi[VEC - 2], left);
            ei[1] = __shfl_sync(0xffffffffu, gi[VEC - 1], left);
            er[VEC + 2] = __shfl_sync(0xffffffffu, gr[0], right);
            er[VEC + 3] = __shfl_sync(0xffffffffu, gr[1], right);
            ei[VEC + 2] = __shfl_sync(0xffffffffu, gi[0], right);
            ei[VEC + 3] = __shfl_sync(0xffffffffu, gi[1], right);
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                ar[v] += inv12dp * (er[v] - (T)8 * er[v + 1] + (T)8 * er[v + 3] - er[v + 4]);
                ai[v] += inv12dp * (ei[v] - (T)8 * ei[v + 1] + (T)8 * ei[v + 3] - ei[v + 4]);
            }
        }
        {  // potential term (with the p-diagonal bath terms) from phase A
            const int pb = ((rg * RG + r) * S2 + pr) * NP + l0;
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const C pv = X[pad16(pb + v)];
                ar[v] += pv.x;
                ai[v] += pv.y;
            }
        }
        if (mode == 0) {
            stv<T, VEC>(v_out + o, ar);
            stv<T, VEC>(v_out + o + blk, ai);
        } else if (tier0) {
            const double hd = h;
            T outr[VEC], outi[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                b0r[v] += hd * (double)ar[v];
                b0i[v] += hd * (double)ai[v];
                outr[v] = (T)b0r[v];
                outi[v] = (T)b0i[v];
            }
            stv<T, VEC>(v_out + o, outr);
            stv<T, VEC>(v_out + o + blk, outi);
            if (mode == 2) {
                stv<double, VEC>(y0_out + o0, b0r);
                stv<double, VEC>(y0_out + o0 + blk, b0i);
            }
        } else {
            v_axpy<VEC>(br, sc.h, ar);
            v_axpy<VEC>(bi, sc.h, ai);
            stv<T, VEC>(v_out + o, br);
            stv<T, VEC>(v_out + o + blk, bi);
        }
    }
}

}  // namespace
