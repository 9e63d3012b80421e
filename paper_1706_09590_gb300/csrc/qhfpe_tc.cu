// Potential term of Eq. (quantum-liouvillian) as a DFT-as-GEMM on the tcgen05 tensor cores.
//
// Every (replica, element, q row, electronic pair) row of the state is a length-np complex vector
// along p.  The forward transform (sign +) of a tile of 128 rows is a real GEMM against the cosine and
// sine matrices C[m][l] = cos(2 pi m l/np), S[m][l] = sin(2 pi m l/np):
//     D_re = W_re C - W_im S,   D_im = W_re S + W_im C,
// the S x S r-space mixing with the potential tables (pre-scaled by 1/np, times -i) is applied per row
// in the epilogue (the pairs of one q row sit in neighbouring TMEM lanes), and the inverse transform
// (sign -) is a second GEMM:
//     P_re = Y_re C + Y_im S,   P_im = Y_im C - Y_re S.
// Operands are bf16 split in two (x = hi + lo, hi = bf16(x), lo = bf16(x - hi)); each real product
// takes three MMAs (hi*hi + hi*lo + lo*hi) accumulating in FP32 in tensor memory.  Operands are staged
// in shared memory in the 128-byte-swizzled K-major layout the MMA descriptors expect; C and S (hi/lo)
// are pre-swizzled on the host.
//
// Persistent CTAs (one per SM) of 256 threads loop over 128-row tiles; the cosine/sine operand tiles
// stay in shared memory for the whole kernel.  Tensor memory holds the forward result D (2 np columns)
// and the inverse accumulator P (2 np columns); the inverse runs slice by slice as the epilogue turns
// each 64-mode slice of D into the bf16 operand Y.  The A operand is streamed in sub-slices (one re/im
// plane of one 64-wide K slice: hi and lo tiles, 32 KB) through two buffers, so that the threads load,
// split and store (or mix) the next sub-slice while the tensor core multiplies the current one; each
// sub-slice's MMAs end with a commit to that buffer's barrier, which the threads wait for before they
// refill the buffer.  Warps 4q..4q+3 share TMEM lane quadrant q and split the columns.  Thread 0
// issues the MMAs.  Waits on the MMA-completion barriers are bounded: on timeout the kernel records an
// error, skips the rest of its work, waits (bounded) for MMAs still in flight, and frees its tensor
// memory.
#include "qhfpe_internal.cuh"

#include <cuda_bf16.h>
#include <stdint.h>

#include <cmath>
#include <vector>

namespace {

constexpr int TC_THREADS = 256;
constexpr int TILE_M = 128;
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;  // give up on an MMA barrier after 2 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address (16-byte units)
    d |= (uint64_t)1u << 16;                  // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;        // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1u << 46;                  // descriptor version
    d |= (uint64_t)2u << 61;                  // 128-byte swizzle
    return d;
}

// kind::f16 instruction descriptor: bf16 A and B, FP32 accumulator, both K-major, M x N.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N, bool neg_a)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (neg_a ? (1u << 13) : 0u) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait for the barrier phase `parity` (wall-clock limit); false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity)
{
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (globaltimer_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
}

__device__ __forceinline__ void tmem_load32(uint32_t taddr, float *out)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) out[j] = __uint_as_float(r[j]);
}

// byte offset of element (row, k) (k < 64) in a 128-row x 64 bf16 K-major tile with 128-byte swizzle
__device__ __forceinline__ uint32_t sw128_chunk(int row, int chunk)
{
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

// split 8 floats into bf16 hi/lo and store them as one 16-byte chunk each
__device__ __forceinline__ void split_store8(const float *x, char *hi_tile, char *lo_tile, uint32_t off)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * c]), h1 = __float2bfloat16_rn(x[2 * c + 1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * c] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * c + 1] - __bfloat162float(h1));
        h[c] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        l[c] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    *reinterpret_cast<uint4 *>(hi_tile + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(lo_tile + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// split 4 floats into bf16 hi/lo and store them as 8 bytes each
__device__ __forceinline__ void split_store4(const float *x, char *hi_tile, char *lo_tile, uint32_t off)
{
    uint32_t h[2], l[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * c]), h1 = __float2bfloat16_rn(x[2 * c + 1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * c] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * c + 1] - __bfloat162float(h1));
        h[c] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        l[c] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    *reinterpret_cast<uint2 *>(hi_tile + off) = make_uint2(h[0], h[1]);
    *reinterpret_cast<uint2 *>(lo_tile + off) = make_uint2(l[0], l[1]);
}

template <int NP, int S>
__global__ void __launch_bounds__(TC_THREADS, 1)
pot_tc_kernel(GridInfo g, const float *__restrict__ v, float *__restrict__ P, const uint4 *__restrict__ bmat,
              const float *__restrict__ tD, const float *__restrict__ tL, const float *__restrict__ tR, long total_rows,
              int *err)
{
    constexpr int KA = NP / 64;            // K slices of 64
    constexpr int TILE = TILE_M * 64 * 2;  // bytes of one 128 x 64 bf16 tile (A side) = 16 KB
    constexpr int BT = NP * 64 * 2;        // bytes of one np x 64 bf16 tile (B side)
    constexpr int S2 = S * S;
    // shared memory: B resident for the whole kernel ([slice][C_hi, C_lo, S_hi, S_lo] tiles); two A
    // buffers, each one sub-slice (the hi and lo tiles of one re/im plane of one K slice); one
    // MMA-completion barrier per A buffer; the TMEM address
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    char *Bs = reinterpret_cast<char *>(smem);
    char *A = Bs + (size_t)KA * 4 * BT;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(A + 4 * TILE);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 2);
    long long *rbase_s = reinterpret_cast<long long *>(A + 4 * TILE + 64);  // [TILE_M] row offsets, -1 past the end
    long long *pbase_s = rbase_s + TILE_M;  // the same for the tile whose P rows are being written

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int quad = warp & 3;                  // TMEM lane quadrant of this warp
    const int grp = warp >> 2;                  // column group of this warp in the epilogues
    const int erow = quad * 32 + lane;          // epilogue row (TMEM lane) of this thread
    const uint32_t mbar0 = smem_u32(mbar), mbar1 = smem_u32(mbar + 1);
    if (t == 0) {
        mbar_init(mbar0, 1);
        mbar_init(mbar1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)(4 * NP)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // the cosine / sine operand tiles, once per CTA
    {
        uint4 *dst = reinterpret_cast<uint4 *>(Bs);
        for (int c = t; c < KA * 4 * BT / 16; c += TC_THREADS) dst[c] = bmat[c];
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t d_re = tmem, d_im = tmem + NP, p_re = tmem + 2 * NP, p_im = tmem + 3 * NP;
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    bool ok = true;

    // Buffer b may be overwritten once the MMAs of its last sub-slice have completed: every use ends
    // with one commit to barrier b, and every reuse first waits for that phase (at most one pending).
    // (per-buffer state in scalars, bit b of `pending` and of `phases`, so that nothing is indexed at
    // run time and nothing lands in local memory)
    uint32_t phases = 0u, pending = 0u;
    auto free_buf = [&](int b) {
        if (pending & (1u << b)) {
            if (ok) ok = mbar_wait(b ? mbar1 : mbar0, (phases >> b) & 1u);
            phases ^= 1u << b;
            pending &= ~(1u << b);
        }
    };

    // One sub-slice: 2 real products x 3 bf16 products x 4 k-steps, then a commit to barrier b.
    //   forward  re: D_re += W_re C,   D_im += W_re S        im: D_re -= W_im S,  D_im += W_im C
    //   inverse  re: P_re += Y_re C,   P_im -= Y_re S        im: P_re += Y_im S,  P_im += Y_im C
    auto issue_sub = [&](int slice, bool inverse, int plane, int b, bool first) {
        const uint32_t b0 = smem_u32(Bs + (size_t)slice * 4 * BT);  // C_hi, C_lo, S_hi, S_lo at 0, 1, 2, 3 BT
        const uint32_t a_h = smem_u32(A + (size_t)b * 2 * TILE), a_l = a_h + TILE;
        // product 0 accumulates into the real part, product 1 into the imaginary part; the first uses
        // C (forward re, inverse re) or S, the second the other matrix
        const uint32_t acc0 = inverse ? p_re : d_re, acc1 = inverse ? p_im : d_im;
        const uint32_t m0 = plane == 0 ? b0 : b0 + 2 * BT, m1 = plane == 0 ? b0 + 2 * BT : b0;
        const bool neg0 = !inverse && plane == 1, neg1 = inverse && plane == 0;
        const uint32_t id0 = idesc_bf16(TILE_M, NP, neg0), id1 = idesc_bf16(TILE_M, NP, neg1);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {  // 4 x K = 16 inside the 64-wide slice: +32 bytes
            const uint32_t ko = (uint32_t)ks * 32;
            const uint32_t acc = (first && ks == 0) ? 0u : 1u;
            mma_bf16(acc0, sdesc_sw128(a_h + ko), sdesc_sw128(m0 + ko), id0, acc);
            mma_bf16(acc0, sdesc_sw128(a_h + ko), sdesc_sw128(m0 + BT + ko), id0, 1u);
            mma_bf16(acc0, sdesc_sw128(a_l + ko), sdesc_sw128(m0 + ko), id0, 1u);
            mma_bf16(acc1, sdesc_sw128(a_h + ko), sdesc_sw128(m1 + ko), id1, acc);
            mma_bf16(acc1, sdesc_sw128(a_h + ko), sdesc_sw128(m1 + BT + ko), id1, 1u);
            mma_bf16(acc1, sdesc_sw128(a_l + ko), sdesc_sw128(m1 + ko), id1, 1u);
        }
        mma_commit(b ? mbar1 : mbar0);
    };
    int sub = 0;  // sub-slices issued so far; sub-slice n uses buffer n & 1
    // hand the sub-slice just written to buffer (sub & 1) to the tensor core
    auto submit = [&](int slice, bool inverse, int plane, bool first) {
        const int b = sub & 1;
        fence_async_smem();
        fence_before();
        ok = __syncthreads_and(ok);
        if (ok && t == 0) {
            fence_after();
            issue_sub(slice, inverse, plane, b, first);
        }
        if (ok) pending |= 1u << b;  // (ok is uniform here: nothing was issued otherwise)
        ++sub;
    };

    // Row order: pair fastest (the pairs of one state row sit in neighbouring TMEM lanes for the
    // mixing), then (replica, element), then q, so that the rows of a warp share their q row and read
    // the same few table rows in the mixing.
    const long n_er = total_rows / ((long)g.nq * S2);  // replicas x elements
    auto row_base = [&](long row) -> size_t {           // offset of a row's real plane in v and P
        const int pr = (int)(row % S2);
        const long rest = row / S2;
        const long er = rest % n_er;
        const int i = (int)(rest / n_er);
        const int e = (int)(er % g.n_elem);
        const long rep = er / g.n_elem;
        return (size_t)rep * g.rep_stride + (size_t)e * g.elem_stride + (size_t)pr * 2 * g.blk + (size_t)i * NP;
    };
    const long n_tiles = (total_rows + TILE_M - 1) / TILE_M;
    // Forward operand: warp w loads rows 16w .. 16w + 15 of the tile, two per instruction (lanes 0-15
    // one row, lanes 16-31 the next), four consecutive floats per lane, so that each request covers two
    // 256-byte row segments; two sub-slices in registers.  The first two sub-slices of a tile are
    // requested before the previous tile writes its P rows, so that their latency overlaps that store.
    const int sl = lane & 15;
    float x[2][32];
    // sub-slice j (plane j & 1, K slice j >> 1) of this thread's 8 rows
    auto load = [&](int j, float *xx) {
        const size_t off = (size_t)(j & 1) * g.blk + (size_t)(j >> 1) * 64 + (size_t)sl * 4;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const long long rb = rbase_s[warp * 16 + 2 * u + (lane >> 4)];
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            if (rb >= 0) a = *reinterpret_cast<const float4 *>(v + (size_t)rb + off);
            xx[4 * u] = a.x;
            xx[4 * u + 1] = a.y;
            xx[4 * u + 2] = a.z;
            xx[4 * u + 3] = a.w;
        }
    };
    // (called by all threads together)
    auto begin_tile = [&](long tl) {
        if (t < TILE_M) {
            const long row = tl * TILE_M + t;
            rbase_s[t] = row < total_rows ? (long long)row_base(row) : -1ll;
        }
        __syncthreads();
        load(0, x[0]);
        if (2 * KA > 1) load(1, x[1]);
    };
    if (blockIdx.x < n_tiles) begin_tile(blockIdx.x);
    for (long tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        // ---- forward transform: W rows -> D, sub-slices (slice, plane) ----------------------------
        {
            // two sub-slices in flight: sub-slice j + 2 is loaded while j is split, stored and multiplied
            // (the loop is unrolled, so x[j & 1] is a fixed register set)
#pragma unroll
            for (int j = 0; j < 2 * KA; ++j) {
                const int b = sub & 1;
                free_buf(b);
                char *hi = A + (size_t)b * 2 * TILE;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    split_store4(x[j & 1] + 4 * u, hi, hi + TILE,
                                 sw128_chunk(warp * 16 + 2 * u + (lane >> 4), sl >> 1) + (uint32_t)(sl & 1) * 8u);
                submit(j >> 1, false, j & 1, j == 0);
                if (!ok) break;
                if (j + 2 < 2 * KA) load(j + 2, x[j & 1]);
            }
        }
        // ---- r-space mixing per slice of modes, then that slice of the inverse transform ------------
        {
            const long row = tile * TILE_M + erow;
            const bool valid = row < total_rows;
            int pr = 0, i = 0;
            if (valid) {
                pr = (int)(row % S2);
                i = (int)(row / S2 / n_er);
            }
            const int jj = pr / S, kk = pr % S;
            // this row's 32 table entries of slice s, as 16-byte vectors (zero for rows past the end)
            auto load_tables = [&](int s, float *td, float *tl, float *tr) {
                const int c0 = s * 64 + grp * 32;
                const float4 *pd = reinterpret_cast<const float4 *>(tD + ((size_t)pr * g.nq + i) * NP + c0);
                const float4 *pl = reinterpret_cast<const float4 *>(
                    tL + ((size_t)(jj * S + (S > 1 ? 1 - jj : 0)) * g.nq + i) * NP + c0);
                const float4 *pq = reinterpret_cast<const float4 *>(
                    tR + ((size_t)((S > 1 ? 1 - kk : 0) * S + kk) * g.nq + i) * NP + c0);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 a = valid ? pd[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                    td[4 * q] = a.x; td[4 * q + 1] = a.y; td[4 * q + 2] = a.z; td[4 * q + 3] = a.w;
                    if (S > 1) {
                        const float4 b = valid ? pl[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                        const float4 c = valid ? pq[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                        tl[4 * q] = b.x; tl[4 * q + 1] = b.y; tl[4 * q + 2] = b.z; tl[4 * q + 3] = b.w;
                        tr[4 * q] = c.x; tr[4 * q + 1] = c.y; tr[4 * q + 2] = c.z; tr[4 * q + 3] = c.w;
                    }
                }
            };
            float td[32], tl[32], tr[32];
            load_tables(0, td, tl, tr);  // independent of D: in flight while the forward MMAs finish
            free_buf((sub - 1) & 1);  // the last forward commit: every forward MMA has completed
            ok = __syncthreads_and(ok);
            fence_after();
            for (int s = 0; s < KA && ok; ++s) {
                const int c0 = s * 64 + grp * 32;  // 32 modes of this warp
                float dr[32], di[32];
                tmem_load32(d_re + lane_off + c0, dr);
                tmem_load32(d_im + lane_off + c0, di);
                float y2[2][32];  // Y re, im of this row's 32 modes
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float ar, ai;
                    if (S == 1) {
                        ar = td[j] * dr[j];
                        ai = td[j] * di[j];
                    } else {
                        // pairs of this q row: lane ^ 2 holds (1-j, k), lane ^ 1 holds (j, 1-k)
                        const float sr = __shfl_xor_sync(0xffffffffu, dr[j], 2), si = __shfl_xor_sync(0xffffffffu, di[j], 2);
                        const float br = __shfl_xor_sync(0xffffffffu, dr[j], 1), bi = __shfl_xor_sync(0xffffffffu, di[j], 1);
                        ar = td[j] * dr[j] + tl[j] * sr - tr[j] * br;
                        ai = td[j] * di[j] + tl[j] * si - tr[j] * bi;
                    }
                    y2[0][j] = ai;  // times -i
                    y2[1][j] = -ar;
                }
                // the next slice's tables, in flight while this slice is stored and multiplied
                if (s + 1 < KA) load_tables(s + 1, td, tl, tr);
#pragma unroll
                for (int plane = 0; plane < 2; ++plane) {
                    const int b = sub & 1;
                    free_buf(b);
                    char *hi = A + (size_t)b * 2 * TILE;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        split_store8(y2[plane] + 8 * q, hi, hi + TILE, sw128_chunk(erow, grp * 4 + q));
                    submit(s, true, plane, s == 0 && plane == 0);
                    if (!ok) break;
                }
            }
            free_buf((sub - 1) & 1);  // the last inverse commit: P is complete
            ok = __syncthreads_and(ok);
            fence_after();
            if (ok && tile + gridDim.x < n_tiles) begin_tile(tile + gridDim.x);
            // ---- P rows to global, through shared memory ---------------------------------------------
            // Each pass stages 32 columns of each warp group's half, both planes, of all 128 rows in the
            // (now idle) A buffers, as [group][plane][row][8 chunks of 16 B] with the chunk index XOR-ed
            // by row & 7 (conflict-free both ways); then every warp writes four 128-byte row segments
            // per instruction.
            if (ok) {
                if (grp == 0) pbase_s[erow] = valid ? (long long)row_base(row) : -1ll;
                float *stg = reinterpret_cast<float *>(A);
#pragma unroll
                for (int it = 0; it < NP / 64; ++it) {
                    const int c0 = grp * (NP / 2) + 32 * it;
                    {
                        float pr_[32], pi_[32];
                        tmem_load32(p_re + lane_off + c0, pr_);
                        tmem_load32(p_im + lane_off + c0, pi_);
                        float4 *s_r = reinterpret_cast<float4 *>(stg + ((grp * 2 + 0) * TILE_M + erow) * 32);
                        float4 *s_i = reinterpret_cast<float4 *>(stg + ((grp * 2 + 1) * TILE_M + erow) * 32);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            s_r[q ^ (erow & 7)] = make_float4(pr_[4 * q], pr_[4 * q + 1], pr_[4 * q + 2], pr_[4 * q + 3]);
                            s_i[q ^ (erow & 7)] = make_float4(pi_[4 * q], pi_[4 * q + 1], pi_[4 * q + 2], pi_[4 * q + 3]);
                        }
                    }
                    __syncthreads();
                    const int ch = lane & 7;
#pragma unroll 1
                    for (int u = 0; u < 16; ++u) {
                        const int seg = u * 32 + warp * 4 + (lane >> 3);  // (group, plane, row)
                        const int gg = seg >> 8, pl = (seg >> 7) & 1, r = seg & (TILE_M - 1);
                        const long long rb = pbase_s[r];
                        if (rb >= 0) {
                            const float4 val = reinterpret_cast<const float4 *>(stg + (size_t)seg * 32)[ch ^ (r & 7)];
                            *reinterpret_cast<float4 *>(P + (size_t)rb + (size_t)pl * g.blk + gg * (NP / 2) + 32 * it +
                                                        4 * ch) = val;
                        }
                    }
                    __syncthreads();
                }
            }
        }
        // tensor memory of this tile fully read before the next tile's MMAs overwrite it
        fence_before();
        __syncthreads();
        fence_after();
    }
    if (!ok && t == 0) atomicExch(err, 1);
    // MMAs possibly still in flight after a give-up: wait for them (bounded) before freeing TMEM
    if (pending & 1u) mbar_wait(mbar0, phases & 1u);
    if (pending & 2u) mbar_wait(mbar1, (phases >> 1) & 1u);
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(4 * NP)));
    }
}

template <int NP, int S>
size_t tc_smem_bytes()
{
    // B, 2 A buffers, barriers, row offsets (forward and P), alignment slack
    return (size_t)(NP / 64) * 4 * NP * 64 * 2 + 4 * (size_t)TILE_M * 64 * 2 + 64 + 16 * TILE_M + 1024;
}

template <int NP, int S>
cudaError_t launch_tc_t(const GridInfo &g, const float *v, float *P, const void *bmat, const float *tD,
                        const float *tL, const float *tR, int n_rep, int *err, cudaStream_t st)
{
    const long rows = (long)n_rep * g.n_elem * g.nq * S * S;
    const long tiles = (rows + TILE_M - 1) / TILE_M;
    if (tiles <= 0) return cudaSuccess;
    static int n_sm = 0;
    if (!n_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 148;
    }
    const int blocks = (int)(tiles < n_sm ? tiles : n_sm);  // persistent: one CTA per SM
    pot_tc_kernel<NP, S><<<blocks, TC_THREADS, tc_smem_bytes<NP, S>(), st>>>(
        g, v, P, reinterpret_cast<const uint4 *>(bmat), tD, tL, tR, rows, err);
    return cudaGetLastError();
}

template <int NP, int S>
cudaError_t prepare_tc_t()
{
    return cudaFuncSetAttribute(pot_tc_kernel<NP, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc_smem_bytes<NP, S>());
}

}  // namespace

bool tc_supported(int np, int S) { return (np == 64 || np == 128) && (S == 1 || S == 2); }

cudaError_t prepare_tc(int np, int S)
{
    if (np == 64 && S == 1) return prepare_tc_t<64, 1>();
    if (np == 64 && S == 2) return prepare_tc_t<64, 2>();
    if (np == 128 && S == 1) return prepare_tc_t<128, 1>();
    if (np == 128 && S == 2) return prepare_tc_t<128, 2>();
    return cudaErrorInvalidValue;
}

cudaError_t launch_potential_tc(const GridInfo &g, const float *v, float *P, const void *bmat, const float *tD,
                                const float *tL, const float *tR, int n_rep, int *err, cudaStream_t st)
{
    if (g.np == 64 && g.S == 1) return launch_tc_t<64, 1>(g, v, P, bmat, tD, tL, tR, n_rep, err, st);
    if (g.np == 64 && g.S == 2) return launch_tc_t<64, 2>(g, v, P, bmat, tD, tL, tR, n_rep, err, st);
    if (g.np == 128 && g.S == 1) return launch_tc_t<128, 1>(g, v, P, bmat, tD, tL, tR, n_rep, err, st);
    if (g.np == 128 && g.S == 2) return launch_tc_t<128, 2>(g, v, P, bmat, tD, tL, tR, n_rep, err, st);
    return cudaErrorInvalidValue;
}

// Host: C and S split into bf16 hi/lo, laid out per 64-wide K slice as four pre-swizzled np x 64
// K-major tiles (C_hi, C_lo, S_hi, S_lo), each row m = output mode, K = l.
void build_tc_matrices(int np, std::vector<uint16_t> &out)
{
    const int KA = np / 64;
    const size_t tile = (size_t)np * 64;  // elements
    out.assign((size_t)KA * 4 * tile, 0);
    auto bf16_bits = [](float x) {
        const __nv_bfloat16 b = __float2bfloat16_rn(x);
        return __bfloat16_as_ushort(b);
    };
    auto bf16_val = [](float x) { return __bfloat162float(__float2bfloat16_rn(x)); };
    const double two_pi = 6.283185307179586476925286766559;
    for (int s = 0; s < KA; ++s)
        for (int m = 0; m < np; ++m)
            for (int k = 0; k < 64; ++k) {
                const int l = s * 64 + k;
                const long ml = ((long)m * l) % np;
                const float c = (float)std::cos(two_pi * ml / np), sn = (float)std::sin(two_pi * ml / np);
                const float vals[4] = {bf16_val(c), c - bf16_val(c), bf16_val(sn), sn - bf16_val(sn)};
                // element (row m, k) of a 128-byte swizzled K-major tile
                const int chunk = k / 8, within = k % 8;
                const size_t byte = (size_t)(m >> 3) * 1024 + (m & 7) * 128 + ((chunk ^ (m & 7)) << 4) + within * 2;
                for (int q = 0; q < 4; ++q) out[((size_t)s * 4 + q) * tile + byte / 2] = bf16_bits(vals[q]);
            }
}
