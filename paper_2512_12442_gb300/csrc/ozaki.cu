// FP64-class whitened rows W = K_* L^-T on the BF16 tensor cores by an error-free digit split
// (Ozaki scheme): both operands are written as sums of S slices of signed 6-bit integer digits
// times powers of two,
//   a' = k / sf2 in [0,1]:        a' = sum_s i_s 2^(-6(s+1)),   |i_0| <= 64, |i_s| <= 32,
//   b' = [L^-1]_ji / 2^F_j:       b' = sum_t l_t 2^(-6(t+1)),   per output column j,
// so every digit is exact in BF16 and every product i_s * l_t is exact.  Products of the same
// level d = s + t share one power-of-two weight and are accumulated in one TMEM accumulator;
// over K chunks of at most 1024 the integer sums stay below 2^24, so the FP32 accumulation is
// exact; after each chunk the levels are drained (smallest first) into float-float registers.
// W is written as (hi, lo) float pairs.  Products with s + t < S are kept; S = 7 -> 28 products.
//
// Two kernels.  k_oz_adig writes the A digit slices of a chunk of rows once (BF16, [slice][row]
// [k]), from the float-float separable tables.  k_oz_gemm (M = 128 points, N = 64 columns, K
// blocks of 32 digits with 64-byte rows and 64B swizzle, two stages) is warp-specialised: warp 0
// loads all slices of A and of B for a K block with one 3-D TMA each; warp 1 issues the MMAs;
// warps 2-9 drain the accumulators.  The S level accumulators use S x 64 of the 512 TMEM
// columns, and because B's slices sit next to each other in shared memory, A slice s meets
// B slices 0 .. S-1-s in one MMA of N = (S - s) 64 columns (split at 256) that lands exactly
// on levels s .. S-1: 10 MMAs per K step instead of 28.  Mbarrier waits are bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>

#include <mutex>
#include <vector>

#include "internal.h"

namespace {

constexpr int TM = 128, TN = 64, BKE = 32, BETA = 6;
constexpr uint32_t kSpin = 1u << 22;
constexpr int KCH = 1024 / BKE;    // K blocks per exact accumulation (K <= 1024 keeps sums < 2^24)
constexpr int A_SLICE = TM * 64;   // bytes of one A digit slice per K block
constexpr int B_SLICE = TN * 64;   // bytes of one B digit slice per K block

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, 64-byte swizzle (8-row groups 512 B apart).
__device__ __forceinline__ uint64_t desc_sw64(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;  // 64-byte swizzle
    return d;
}


__device__ __forceinline__ bool wait_bar(uint32_t a, uint32_t par)
{
    for (uint32_t it = 0; it < kSpin; ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(a), "r"(par)
                     : "memory");
        if (done) return true;
    }
    return false;
}

struct FF {
    float h, l;
};
__device__ __forceinline__ FF ff_mul(FF a, FF b)
{
    float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    float s = p + e;
    return {s, e - (s - p)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    float s = a.h + b.h;
    float bv = s - a.h;
    float err = (a.h - (s - bv)) + (b.h - bv);
    err += a.l + b.l;
    float r = s + err;
    return {r, err - (r - s)};
}
__device__ __forceinline__ FF ff_add_f(FF a, float b)
{
    float s = a.h + b;
    float bv = s - a.h;
    float err = (a.h - (s - bv)) + (b - bv) + a.l;
    float r = s + err;
    return {r, err - (r - s)};
}

struct OzParams {
    const float2 *Tu;  // unit (no sf2) float-float SE tables, 3 axes
    int64_t off1, off2, mp, m;
    GridDev g;
    const int64_t *pts;
    int64_t pt_base, count;
    const float *colscale;  // 2^F_j
    float sf2;
    float2 *W;  // rows out_off + r, mp float-float each (or rows at p % row_mod when out_by_point)
    int out_by_point;
    int64_t row_mod;
    int64_t mpt, out_off;
    int *status;
};

// A digit slices of rows [0, count) of the list: out[s][row][k], k < mpt (zero beyond m and for
// rows whose point is off the grid).  a' = k/sf2 from the unit tables in float-float; signed
// 6-bit digits, the low word joining once the high word is consumed.  Thread: 8 consecutive k.
__global__ void k_oz_adig(OzParams prm, __nv_bfloat16 *out)
{
    constexpr int S = 7;
    const int64_t chunks = prm.mpt / 8;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= prm.count * chunks) return;
    const int64_t row = t / chunks, j0 = (t % chunks) * 8;
    int64_t p = prm.pts ? prm.pts[row] : prm.pt_base + row;
    const int64_t nx = prm.g.n[0], ny = prm.g.n[1];
    const bool rv = p >= 0 && p < nx * ny * (int64_t)prm.g.n[2];
    if (!rv) p = 0;
    const int gx = (int)(p % nx), gy = (int)((p / nx) % ny), gz = (int)(p / (nx * ny));
    const float2 *px = prm.Tu + (int64_t)gx * prm.mp, *py = prm.Tu + prm.off1 + (int64_t)gy * prm.mp,
                 *pz = prm.Tu + prm.off2 + (int64_t)gz * prm.mp;
    // table rows are 512-byte aligned and zero from m to mp: two elements per 16-byte load
    float2 tx[8], ty[8], tz[8];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
        const float4 a = *(const float4 *)(px + j0 + e), b = *(const float4 *)(py + j0 + e),
                     c = *(const float4 *)(pz + j0 + e);
        tx[e] = make_float2(a.x, a.y); tx[e + 1] = make_float2(a.z, a.w);
        ty[e] = make_float2(b.x, b.y); ty[e + 1] = make_float2(b.z, b.w);
        tz[e] = make_float2(c.x, c.y); tz[e + 1] = make_float2(c.z, c.w);
    }
    float dig[S][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        FF a = ff_mul(ff_mul(FF{tx[e].x, tx[e].y}, FF{ty[e].x, ty[e].y}), FF{tz[e].x, tz[e].y});
        if (!rv || j0 + e >= prm.m) a = FF{0.f, 0.f};
        float rr = a.h;
#pragma unroll
        for (int d = 0; d < S; ++d) {
            if (d == 3) rr += a.l;
            const float i = rintf(ldexpf(rr, BETA * (d + 1)));
            dig[d][e] = i;
            rr = fmaf(-i, ldexpf(1.0f, -BETA * (d + 1)), rr);
        }
    }
#pragma unroll
    for (int d = 0; d < S; ++d) {
        uint32_t wd[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(dig[d][2 * q]));
            const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(dig[d][2 * q + 1]));
            wd[q] = lo | (hi << 16);
        }
        *(uint4 *)(out + ((int64_t)d * prm.count + row) * prm.mpt + j0) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    }
}

constexpr int G_NTHR = 320;  // warp 0: TMA, warp 1: MMA, warps 2-9: TMEM drain and store

__host__ __device__ constexpr uint32_t idesc_n(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// The pipeline shared by the digit-split GEMMs.  Stage layout: S A slices (TM rows x 64 B) then
// S B slices (TN rows x 64 B) per K block of BKE digits.
template <int S>
struct OzPipe {
    static constexpr int A_ST = S * A_SLICE, B_ST = S * B_SLICE, STAGE = A_ST + B_ST;
    unsigned char *smem;
    uint32_t full0, empty0, done, drained, tmem;
};

// Producer (one thread): K blocks kb0 .. kb0 + nkb - 1 of all A slices (rows arow ..) and all
// B slices (rows brow ..), one 3-D TMA copy each, into a two-stage ring.
template <int S>
__device__ __forceinline__ void oz_produce(const OzPipe<S> &P, const CUtensorMap *mapA, const CUtensorMap *mapB, int kb0,
                                           int nkb, int arow, int brow, bool &ok)
{
    for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb & 1;
        unsigned char *st = P.smem + s * OzPipe<S>::STAGE;
        if (kb >= 2 && !wait_bar(P.empty0 + 8 * s, ((kb >> 1) - 1) & 1)) ok = false;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(P.full0 + 8 * s),
                     "r"((uint32_t)OzPipe<S>::STAGE)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4}], [%5];" ::"r"(su32(st)),
            "l"((uint64_t)mapA), "r"((kb0 + kb) * BKE), "r"(arow), "r"(0), "r"(P.full0 + 8 * s)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4}], [%5];" ::"r"(su32(st + OzPipe<S>::A_ST)),
            "l"((uint64_t)mapB), "r"((kb0 + kb) * BKE), "r"(brow), "r"(0), "r"(P.full0 + 8 * s)
            : "memory");
    }
}

// MMA issue (one thread): A slice sa against B slices 0 .. S-1-sa, contiguous rows of the B
// stage, onto TMEM levels sa .. S-1; `done` after every KCH blocks, then wait for the drain.
template <int S>
__device__ __forceinline__ void oz_issue(const OzPipe<S> &P, int nkb, bool &ok)
{
    for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb & 1;
        unsigned char *st = P.smem + s * OzPipe<S>::STAGE;
        if (!wait_bar(P.full0 + 8 * s, (kb >> 1) & 1)) ok = false;
        if (kb % KCH == 0 && kb > 0 && !wait_bar(P.drained, ((kb / KCH) - 1) & 1)) ok = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ab = su32(st), bb = su32(st + OzPipe<S>::A_ST);
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
#pragma unroll
            for (int sa = 0; sa < S; ++sa) {
                const int nrow = (S - sa) * TN;
#pragma unroll
                for (int p0 = 0; p0 < nrow; p0 += 256) {
                    const int nn = nrow - p0 < 256 ? nrow - p0 : 256;
                    const uint32_t acc = (kb % KCH == 0 && kk == 0 && sa == 0) ? 0u : 1u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                            P.tmem + (uint32_t)(sa * TN + p0)),
                        "l"(desc_sw64(ab + sa * A_SLICE + kk * 32)), "l"(desc_sw64(bb + p0 * 64 + kk * 32)),
                        "r"(idesc_n(nn)), "r"(acc));
                }
            }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(P.empty0 + 8 * s)
                     : "memory");
        if (kb == nkb - 1 || kb % KCH == KCH - 1)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(P.done)
                         : "memory");
    }
}

// Drain (warps 2-9): warp w reads TMEM lanes 32 (w % 4), columns 32 ((w - 2) / 4) of every
// level after each K chunk and adds the exact level sums, smallest first, in float-float.
template <int S>
__device__ __forceinline__ void oz_drain(const OzPipe<S> &P, int nch, int lq, int half, int lane, FF acc[32], bool &ok)
{
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = FF{0.f, 0.f};
    for (int ch = 0; ch < nch; ++ch) {
        if (!wait_bar(P.done, (uint32_t)(ch & 1))) ok = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int lvl = S - 1; lvl >= 0; --lvl) {
            uint32_t rr[32];
            const uint32_t taddr = P.tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(lvl * TN + half * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]),
                  "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]),
                  "=r"(rr[14]), "=r"(rr[15]), "=r"(rr[16]), "=r"(rr[17]), "=r"(rr[18]), "=r"(rr[19]), "=r"(rr[20]),
                  "=r"(rr[21]), "=r"(rr[22]), "=r"(rr[23]), "=r"(rr[24]), "=r"(rr[25]), "=r"(rr[26]), "=r"(rr[27]),
                  "=r"(rr[28]), "=r"(rr[29]), "=r"(rr[30]), "=r"(rr[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const float wgt = ldexpf(1.0f, -BETA * (lvl + 2));
#pragma unroll
            for (int c = 0; c < 32; ++c) acc[c] = ff_add_f(acc[c], __uint_as_float(rr[c]) * wgt);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (ch < nch - 1 && lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(P.drained) : "memory");
    }
}

// Barriers and the 512 TMEM columns of a digit-split GEMM CTA (G_NTHR threads).
template <int S>
__device__ __forceinline__ OzPipe<S> oz_setup(unsigned char *smem_raw, uint32_t *tmem_slot)
{
    OzPipe<S> P;
    P.smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(P.smem + 2 * OzPipe<S>::STAGE);  // full[2], empty[2], done, drained
    P.full0 = su32(&bars[0]);
    P.empty0 = su32(&bars[2]);
    P.done = su32(&bars[4]);
    P.drained = su32(&bars[5]);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        for (int b = 0; b < 5; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bars[b])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(P.drained));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    P.tmem = *tmem_slot;
    return P;
}

__device__ __forceinline__ void oz_teardown(uint32_t tmem, bool ok, int *status)
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (!ok) atomicCAS(status, 0, (int)GPR_ERR_TIMEOUT);
    if ((threadIdx.x >> 5) == 0) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
    }
}

// W rows: kernel-row digits (A, 128 points) x L^-1 digits (B, 64 output columns); B is lower
// triangular, so K stops at the tile's last column.
template <int S>
__global__ void __launch_bounds__(G_NTHR, 1) k_oz_gemm(const __grid_constant__ CUtensorMap mapA,
                                                      const __grid_constant__ CUtensorMap mapB, OzParams prm)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint32_t tmem_slot;
    const OzPipe<S> P = oz_setup<S>(smem_raw, &tmem_slot);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // N tiles fastest: the tiles of one row block run together and share its A digits in L2
    const int64_t row0 = (int64_t)blockIdx.y * TM;
    const int n0 = blockIdx.x * TN;
    const int64_t m = prm.m;
    const int64_t kend = (int64_t)n0 + TN < m ? (int64_t)n0 + TN : m;
    const int nkb = (int)((kend + BKE - 1) / BKE);
    const int nch = (nkb + KCH - 1) / KCH;
    bool ok = true;

    if (warp == 0 && lane == 0) {
        oz_produce<S>(P, &mapA, &mapB, 0, nkb, (int)row0, n0, ok);
    } else if (warp == 1 && lane == 0) {
        oz_issue<S>(P, nkb, ok);
    } else if (warp >= 2) {
        const int lq = warp & 3, half = (warp - 2) >> 2;
        FF acc[32];
        oz_drain<S>(P, nch, lq, half, lane, acc, ok);
        // Stage the 128 x 64 tile in shared memory (the pipeline stages are free: every MMA has
        // completed), 16-byte chunks XOR-swizzled by row, then store whole 512-byte row pieces.
        float4 *tile = (float4 *)P.smem;  // row r, chunk k (columns 2k, 2k+1) at r * 32 + (k ^ (r & 31))
        const int r = lq * 32 + lane;
#pragma unroll
        for (int c = 0; c < 32; c += 2) {
            const int64_t j = n0 + half * 32 + c;
            FF v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float cs = (j + h < prm.mp) ? prm.colscale[j + h] : 0.f;
                v[h] = FF{acc[c + h].h * cs, acc[c + h].l * cs};  // power-of-two scale: exact
                if (prm.sf2 != 1.0f) v[h] = ff_mul(v[h], FF{prm.sf2, 0.f});
            }
            const int k = (half * 32 + c) >> 1;
            tile[r * 32 + (k ^ (r & 31))] = make_float4(v[0].h, v[0].l, v[1].h, v[1].l);
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");  // the 8 drain warps
        const int64_t npts = (int64_t)prm.g.n[0] * prm.g.n[1] * (int64_t)prm.g.n[2];
        for (int rr = 0; rr < 16; ++rr) {
            const int rt = (warp - 2) * 16 + rr;
            const int64_t row = row0 + rt;
            if (row >= prm.count) break;
            const int64_t p = prm.pts ? prm.pts[row] : prm.pt_base + row;
            if (p < 0 || p >= npts) continue;
            const int64_t orow = prm.out_by_point ? p % prm.row_mod : prm.out_off + row;
            if (n0 + 2 * lane < prm.mp)
                *(float4 *)(prm.W + orow * prm.mp + n0 + 2 * lane) = tile[rt * 32 + (lane ^ (rt & 31))];
        }
    }
    oz_teardown(P.tmem, ok, prm.status);
}

// A digits generated in the kernel (no HBM staging): 8 consecutive k of one row, all S slices,
// written in the layout the 64-byte-swizzled 3-D TMA box would give ([slice][row][k], 64-byte rows,
// 16-byte chunk c of row r at chunk c ^ ((r >> 1) & 3)).  Same digits as k_oz_adig.
template <int S>
__device__ __forceinline__ void gen_a_chunk(const OzParams &prm, unsigned char *a_stage, int r, int c, int kb,
                                            const int *gx, const int *gy, const int *gz, const bool *rv)
{
    const int64_t j0 = (int64_t)kb * BKE + c * 8;
    const float2 *px = prm.Tu + (int64_t)gx[r] * prm.mp, *py = prm.Tu + prm.off1 + (int64_t)gy[r] * prm.mp,
                 *pz = prm.Tu + prm.off2 + (int64_t)gz[r] * prm.mp;
    float2 tx[8], ty[8], tz[8];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
        const float4 a = *(const float4 *)(px + j0 + e), b = *(const float4 *)(py + j0 + e),
                     d = *(const float4 *)(pz + j0 + e);
        tx[e] = make_float2(a.x, a.y); tx[e + 1] = make_float2(a.z, a.w);
        ty[e] = make_float2(b.x, b.y); ty[e + 1] = make_float2(b.z, b.w);
        tz[e] = make_float2(d.x, d.y); tz[e + 1] = make_float2(d.z, d.w);
    }
    float dig[S][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        FF a = ff_mul(ff_mul(FF{tx[e].x, tx[e].y}, FF{ty[e].x, ty[e].y}), FF{tz[e].x, tz[e].y});
        if (!rv[r] || j0 + e >= prm.m) a = FF{0.f, 0.f};
        float rr = a.h;
#pragma unroll
        for (int d = 0; d < S; ++d) {
            if (d == 3) rr += a.l;
            const float i = rintf(ldexpf(rr, BETA * (d + 1)));
            dig[d][e] = i;
            rr = fmaf(-i, ldexpf(1.0f, -BETA * (d + 1)), rr);
        }
    }
    const int pc = c ^ ((r >> 1) & 3);
#pragma unroll
    for (int d = 0; d < S; ++d) {
        uint32_t wd[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(dig[d][2 * q]));
            const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(dig[d][2 * q + 1]));
            wd[q] = lo | (hi << 16);
        }
        *(uint4 *)(a_stage + d * A_SLICE + r * 64 + pc * 16) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    }
}

// W rows with the kernel-row digits generated in shared memory by warps 2-9, which also drain the
// accumulators: they fill each stage's A slices (after the MMAs of two blocks earlier freed it),
// and at the end of each K chunk wait for its MMAs, drain and release TMEM.  Warp 0 loads only the
// B slices by TMA; warp 1 issues the MMAs once both halves of a stage are in.
template <int S>
__global__ void __launch_bounds__(G_NTHR, 1) k_oz_gemm_gen(const __grid_constant__ CUtensorMap mapB, OzParams prm)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint32_t tmem_slot;
    __shared__ int gx[TM], gy[TM], gz[TM];
    __shared__ bool rv[TM];
    __shared__ __align__(8) uint64_t fullA[2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row0 = (int64_t)blockIdx.y * TM;
    for (int r = tid; r < TM; r += G_NTHR) {
        const int64_t row = row0 + r;
        bool ok = row < prm.count;
        int64_t p = ok ? (prm.pts ? prm.pts[row] : prm.pt_base + row) : 0;
        const int64_t nx = prm.g.n[0], ny = prm.g.n[1];
        if (p < 0 || p >= nx * ny * (int64_t)prm.g.n[2]) { ok = false; p = 0; }
        gx[r] = (int)(p % nx);
        gy[r] = (int)((p / nx) % ny);
        gz[r] = (int)(p / (nx * ny));
        rv[r] = ok;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 256;" ::"r"(su32(&fullA[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 256;" ::"r"(su32(&fullA[1])));
    }
    const OzPipe<S> P = oz_setup<S>(smem_raw, &tmem_slot);  // its __syncthreads publishes the above
    const int n0 = blockIdx.x * TN;
    const int64_t m = prm.m;
    const int64_t kend = (int64_t)n0 + TN < m ? (int64_t)n0 + TN : m;
    const int nkb = (int)((kend + BKE - 1) / BKE);
    const int nch = (nkb + KCH - 1) / KCH;
    bool ok = true;
    const uint32_t fa0 = su32(&fullA[0]);

    if (warp == 0 && lane == 0) {
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb & 1;
            unsigned char *st = P.smem + s * OzPipe<S>::STAGE;
            if (kb >= 2 && !wait_bar(P.empty0 + 8 * s, ((kb >> 1) - 1) & 1)) ok = false;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(P.full0 + 8 * s),
                         "r"((uint32_t)OzPipe<S>::B_ST)
                         : "memory");
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4}], [%5];" ::"r"(su32(st + OzPipe<S>::A_ST)),
                "l"((uint64_t)&mapB), "r"(kb * BKE), "r"(n0), "r"(0), "r"(P.full0 + 8 * s)
                : "memory");
        }
    } else if (warp == 1 && lane == 0) {
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb & 1;
            unsigned char *st = P.smem + s * OzPipe<S>::STAGE;
            if (!wait_bar(P.full0 + 8 * s, (kb >> 1) & 1)) ok = false;
            if (!wait_bar(fa0 + 8 * s, (kb >> 1) & 1)) ok = false;
            if (kb % KCH == 0 && kb > 0 && !wait_bar(P.drained, ((kb / KCH) - 1) & 1)) ok = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ab = su32(st), bb = su32(st + OzPipe<S>::A_ST);
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
#pragma unroll
                for (int sa = 0; sa < S; ++sa) {
                    const int nrow = (S - sa) * TN;
#pragma unroll
                    for (int p0 = 0; p0 < nrow; p0 += 256) {
                        const int nn = nrow - p0 < 256 ? nrow - p0 : 256;
                        const uint32_t acc = (kb % KCH == 0 && kk == 0 && sa == 0) ? 0u : 1u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                                P.tmem + (uint32_t)(sa * TN + p0)),
                            "l"(desc_sw64(ab + sa * A_SLICE + kk * 32)), "l"(desc_sw64(bb + p0 * 64 + kk * 32)),
                            "r"(idesc_n(nn)), "r"(acc));
                    }
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(P.empty0 + 8 * s)
                         : "memory");
            if (kb == nkb - 1 || kb % KCH == KCH - 1)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(P.done)
                             : "memory");
        }
    } else if (warp >= 2) {
        const int at = tid - 64;  // 0 .. 255
        const int lq = warp & 3, half = (warp - 2) >> 2;
        FF acc[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] = FF{0.f, 0.f};
        for (int ch = 0; ch < nch; ++ch) {
            const int kb1 = (ch + 1) * KCH < nkb ? (ch + 1) * KCH : nkb;
            for (int kb = ch * KCH; kb < kb1; ++kb) {
                const int s = kb & 1;
                unsigned char *st = P.smem + s * OzPipe<S>::STAGE;
                if (kb >= 2 && !wait_bar(P.empty0 + 8 * s, ((kb >> 1) - 1) & 1)) ok = false;
                for (int q = at; q < TM * 4; q += 256) gen_a_chunk<S>(prm, st, q >> 2, q & 3, kb, gx, gy, gz, rv);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(fa0 + 8 * s) : "memory");
            }
            // drain this chunk's level accumulators (smallest first) into float-float
            if (!wait_bar(P.done, (uint32_t)(ch & 1))) ok = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int lvl = S - 1; lvl >= 0; --lvl) {
                uint32_t rr[32];
                const uint32_t taddr = P.tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(lvl * TN + half * 32);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                    "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]),
                      "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]),
                      "=r"(rr[14]), "=r"(rr[15]), "=r"(rr[16]), "=r"(rr[17]), "=r"(rr[18]), "=r"(rr[19]), "=r"(rr[20]),
                      "=r"(rr[21]), "=r"(rr[22]), "=r"(rr[23]), "=r"(rr[24]), "=r"(rr[25]), "=r"(rr[26]), "=r"(rr[27]),
                      "=r"(rr[28]), "=r"(rr[29]), "=r"(rr[30]), "=r"(rr[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                const float wgt = ldexpf(1.0f, -BETA * (lvl + 2));
#pragma unroll
                for (int c = 0; c < 32; ++c) acc[c] = ff_add_f(acc[c], __uint_as_float(rr[c]) * wgt);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (ch < nch - 1 && lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(P.drained) : "memory");
        }
        // the MMAs are complete: stage the tile through shared memory and store whole row pieces
        asm volatile("bar.sync 1, 256;" ::: "memory");  // every drain warp is past its last stage read
        float4 *tile = (float4 *)P.smem;
        const int r = lq * 32 + lane;
#pragma unroll
        for (int c = 0; c < 32; c += 2) {
            const int64_t j = n0 + half * 32 + c;
            FF v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float cs = (j + h < prm.mp) ? prm.colscale[j + h] : 0.f;
                v[h] = FF{acc[c + h].h * cs, acc[c + h].l * cs};
                if (prm.sf2 != 1.0f) v[h] = ff_mul(v[h], FF{prm.sf2, 0.f});
            }
            const int k = (half * 32 + c) >> 1;
            tile[r * 32 + (k ^ (r & 31))] = make_float4(v[0].h, v[0].l, v[1].h, v[1].l);
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");
        const int64_t npts = (int64_t)prm.g.n[0] * prm.g.n[1] * (int64_t)prm.g.n[2];
        for (int rr2 = 0; rr2 < 16; ++rr2) {
            const int rt = (warp - 2) * 16 + rr2;
            const int64_t row = row0 + rt;
            if (row >= prm.count) break;
            const int64_t p = prm.pts ? prm.pts[row] : prm.pt_base + row;
            if (p < 0 || p >= npts) continue;
            const int64_t orow = prm.out_by_point ? p % prm.row_mod : prm.out_off + row;
            if (n0 + 2 * lane < prm.mp)
                *(float4 *)(prm.W + orow * prm.mp + n0 + 2 * lane) = tile[rt * 32 + (lane ^ (rt & 31))];
        }
    }
    oz_teardown(P.tmem, ok, prm.status);
}

// (double)f * 2^sc built from the bit pattern (no FP64 instructions): exact for normal f while
// the result stays normal; zero and subnormal f give 0, a result outside the normal range its
// FP64 evaluation.
__device__ __forceinline__ double f2d_scaled(float f, int sc)
{
    const uint32_t b = __float_as_uint(f);
    const int ef = (int)((b >> 23) & 0xFF);
    if (ef == 0) return 0.0;
    const int ed = ef + 896 + sc;  // FP64 biased exponent
    if (ed <= 0 || ed >= 2047) return ldexp((double)f, sc);
    const unsigned long long db = ((unsigned long long)(b >> 31) << 63) | ((unsigned long long)ed << 52) |
                                  ((unsigned long long)(b & 0x7FFFFF) << 29);
    return __longlong_as_double((long long)db);
}

// General FP64-class product C = A B of FP64 matrices given as digit slices: A rows (M, K-major,
// row r scaled by 2^-ea[r]) and B columns (N rows of K, column j scaled by 2^-eb[j]); C is
// written in FP64, scaled back by 2^(ea + eb) (or added to C).  Split z of the K range
// (kb_per_split blocks) writes its own partial at C + z cstride; with lower_b (B[k][j] = 0 for
// k < j) K starts at the tile's first column instead.
struct OzG {
    int64_t M, N, kblocks, kb_per_split;
    int lower_b, accumulate;  // accumulate: C += A B
    const int *ea, *eb;
    double *C;
    int64_t ldc, cstride;
    int *status;
};

template <int S>
__global__ void __launch_bounds__(G_NTHR, 1) k_oz_dgemm(const __grid_constant__ CUtensorMap mapA,
                                                       const __grid_constant__ CUtensorMap mapB, OzG prm)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint32_t tmem_slot;
    const OzPipe<S> P = oz_setup<S>(smem_raw, &tmem_slot);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row0 = (int64_t)blockIdx.y * TM;
    const int n0 = blockIdx.x * TN;
    int64_t kb0 = prm.lower_b ? n0 / BKE : (int64_t)blockIdx.z * prm.kb_per_split;
    int64_t kb1 = prm.lower_b ? prm.kblocks : kb0 + prm.kb_per_split;
    if (kb1 > prm.kblocks) kb1 = prm.kblocks;
    const int nkb = kb1 > kb0 ? (int)(kb1 - kb0) : 0;
    const int nch = (nkb + KCH - 1) / KCH;
    bool ok = true;

    if (warp == 0 && lane == 0) {
        oz_produce<S>(P, &mapA, &mapB, (int)kb0, nkb, (int)row0, n0, ok);
    } else if (warp == 1 && lane == 0) {
        oz_issue<S>(P, nkb, ok);
    } else if (warp >= 2) {
        const int lq = warp & 3, half = (warp - 2) >> 2;
        FF acc[32];
        oz_drain<S>(P, nch, lq, half, lane, acc, ok);
        // FP64 values staged in shared memory (16-byte chunks XOR-swizzled by row, as in
        // k_oz_gemm), then stored (or added) as whole row pieces
        double2 *tile = (double2 *)P.smem;
        const int r = lq * 32 + lane;
        const int64_t row = row0 + r;
        const int er = row < prm.M ? prm.ea[row] : 0;
#pragma unroll
        for (int c = 0; c < 32; c += 2) {
            const int64_t j = n0 + half * 32 + c;
            const int s0 = er + (j < prm.N ? prm.eb[j] : 0), s1 = er + (j + 1 < prm.N ? prm.eb[j + 1] : 0);
            const int k = (half * 32 + c) >> 1;
            tile[r * 32 + (k ^ (r & 31))] = make_double2(f2d_scaled(acc[c].h, s0) + f2d_scaled(acc[c].l, s0),
                                                         f2d_scaled(acc[c + 1].h, s1) + f2d_scaled(acc[c + 1].l, s1));
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");  // the 8 drain warps
        const int64_t j = n0 + 2 * lane;
        for (int rr = 0; rr < 16; ++rr) {
            const int rt = (warp - 2) * 16 + rr;
            const int64_t orow = row0 + rt;
            if (orow >= prm.M) break;
            const double2 v = tile[rt * 32 + (lane ^ (rt & 31))];
            double *out = prm.C + (int64_t)blockIdx.z * prm.cstride + orow * prm.ldc + j;
            if (j + 1 < prm.N) {
                double2 o = v;
                if (prm.accumulate) {
                    const double2 a = *(const double2 *)out;
                    o = make_double2(a.x + v.x, a.y + v.y);
                }
                *(double2 *)out = o;
            } else if (j < prm.N) {
                out[0] = prm.accumulate ? out[0] + v.x : v.x;
            }
        }
    }
    oz_teardown(P.tmem, ok, prm.status);
}

// Digit slices of b' = [L^-1]_ji / 2^F_j, layout [S][mpt rows j][mpt cols i] (K-major), BF16.
__global__ void k_oz_split_b(const double *Linv, int64_t mb, int64_t m, int64_t mpt, int S, const float *colscale,
                             __nv_bfloat16 *B)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= mpt * mpt) return;
    int64_t j = idx / mpt, i = idx % mpt;
    double v = (j < m && i <= j) ? Linv[j * mb + i] / (double)colscale[j] : 0.0;
    double r = v;
    for (int t = 0; t < S; ++t) {
        double sc = ldexp(1.0, BETA * (t + 1));
        double d = rint(r * sc);
        r -= d / sc;
        B[(int64_t)t * mpt * mpt + idx] = __double2bfloat16(d);
    }
}

// Column scales 2^F_j with max_i |[L^-1]_ji| <= 2^F_j (one warp per column).
__global__ void k_oz_colscale(const double *Linv, int64_t mb, int64_t m, int64_t mpt, float *cs)
{
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    int64_t j = blockIdx.x * (int64_t)(blockDim.x / 32) + warp;
    if (j >= mpt) return;
    double mx = 0.0;
    if (j < m)
        for (int64_t i = lane; i <= j; i += 32) mx = fmax(mx, fabs(Linv[j * mb + i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
        int e = 0;
        if (mx > 0.0) {
            frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1)
        }
        cs[j] = ldexpf(1.0f, e);
    }
}

// Unit float-float SE tables exp(-(x_g - X_jd)^2 / (2 l_d^2)) (no signal variance).
__global__ void k_unit_tables(const double *X, int64_t m, int64_t mp, KernParams kp, GridDev g, float2 *Tu)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t total = (int64_t)(g.n[0] + g.n[1] + g.n[2]) * mp;
    if (idx >= total) return;
    int64_t row = idx / mp, j = idx % mp;
    int d = 0;
    int64_t gi = row;
    if (gi >= g.n[0]) { gi -= g.n[0]; d = 1; if (gi >= g.n[1]) { gi -= g.n[1]; d = 2; } }
    double v = 0.0;
    if (j < m) {
        double x = g.lo[d] + (double)gi * g.h[d];
        double t = (x - X[3 * j + d]) / kp.ell[d];
        v = exp(-0.5 * t * t);
    }
    float h = (float)v;
    Tu[idx] = make_float2(h, (float)(v - (double)h));
}

// stats15 from float-float W rows (warp per listed point).
__constant__ int c_off[13][3] = {{1, -1, -1}, {1, -1, 0}, {1, -1, 1}, {1, 0, -1}, {1, 0, 0}, {1, 0, 1}, {1, 1, -1},
                                 {1, 1, 0},   {1, 1, 1},  {0, 1, -1}, {0, 1, 0},  {0, 1, 1}, {0, 0, 1}};
struct Prior13 {
    double k[13];
};

// Compensated dot product step (Ogita-Rump-Oishi Dot2 with float-float inputs): the product's
// high part is added by an error-free TwoSum, every rounding error goes to one FP32 carry.
__device__ __forceinline__ void dot2_step(float &sh, float &sl, float2 a, float2 b)
{
    float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    float s = sh + p;
    float bv = s - sh;
    sl += ((sh - (s - bv)) + (p - bv)) + e;
    sh = s;
}

__global__ void __launch_bounds__(256, 2) k_stats_ff(GridDev g, const int64_t *pts, int64_t count,
                                                     const int32_t *slot, const float2 *W, int64_t mp, int64_t m,
                                                     const float2 *vyff, double sf2, const __grid_constant__ Prior13 pr,
                                                     double *out15,
                                                     int out_by_point, int64_t row_mod)
{
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    int64_t pos = blockIdx.x * (int64_t)(blockDim.x / 32) + warp;
    if (pos >= count) return;
    int64_t p = pts[pos];
    int64_t nx = g.n[0], ny = g.n[1], nz = g.n[2];
    int ix = (int)(p % nx), iy = (int)((p / nx) % ny), iz = (int)(p / (nx * ny));
    // rows of W: through the slot map, or (slot == nullptr) at the grid index modulo row_mod
    const int64_t self = slot ? (int64_t)slot[p] : (p < row_mod ? p : p % row_mod);
    int32_t nb[13];  // neighbour rows (< 2^31: rows of one call), -1 = off the grid
#pragma unroll
    for (int e = 0; e < 13; ++e) {
        int a = ix + c_off[e][0], b = iy + c_off[e][1], c = iz + c_off[e][2];
        int32_t r = -1;
        if (a >= 0 && b >= 0 && c >= 0 && a < nx && b < ny && c < nz) {
            int64_t q = a + nx * (b + ny * (int64_t)c);
            r = slot ? slot[q] : (int32_t)(q < row_mod ? q : q % row_mod);
        }
        nb[e] = r;
    }
    float sh[15], sl[15];
#pragma unroll
    for (int q = 0; q < 15; ++q) { sh[q] = 0.f; sl[q] = 0.f; }
    // two consecutive float-float elements per lane and load (rows are 512-byte aligned, mp even,
    // and W, vyff are zero from m to mp)
    const float4 *wp = (const float4 *)(W + self * mp);
    const float4 *W4 = (const float4 *)W;
    const float4 *v4 = (const float4 *)vyff;
    const int64_t half_mp = mp / 2, m2 = (m + 1) / 2;
    for (int64_t j = lane; j < m2; j += 32) {
        const float4 a = wp[j], v = v4[j];
        float4 q[13];
#pragma unroll
        for (int e = 0; e < 13; ++e) q[e] = nb[e] >= 0 ? W4[(int64_t)nb[e] * half_mp + j] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 a0 = make_float2(a.x, a.y), a1 = make_float2(a.z, a.w);
        dot2_step(sh[0], sl[0], a0, make_float2(v.x, v.y));
        dot2_step(sh[0], sl[0], a1, make_float2(v.z, v.w));
        dot2_step(sh[1], sl[1], a0, a0);
        dot2_step(sh[1], sl[1], a1, a1);
#pragma unroll
        for (int e = 0; e < 13; ++e) {
            dot2_step(sh[2 + e], sl[2 + e], a0, make_float2(q[e].x, q[e].y));
            dot2_step(sh[2 + e], sl[2 + e], a1, make_float2(q[e].z, q[e].w));
        }
    }
    // Combine the lanes in float-float (FP64 arithmetic runs at 1/64 rate on this part) by a
    // halving exchange: at offset o each lane keeps one half of its values and adds its partner's
    // copy of that half, so 16 values take 8 + 4 + 2 + 1 + 1 exchanges instead of 16 x 5; value
    // q ends in lanes 2q and 2q + 1.
    FF v[16];
#pragma unroll
    for (int q = 0; q < 15; ++q) v[q] = ff_add(FF{sh[q], 0.f}, FF{sl[q], 0.f});
    v[15] = FF{0.f, 0.f};
#pragma unroll
    for (int half = 8, o = 16; half >= 1; half >>= 1, o >>= 1) {
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const FF keep = hi ? v[i + half] : v[i], send = hi ? v[i] : v[i + half];
            const FF t = {__shfl_xor_sync(0xffffffffu, send.h, o), __shfl_xor_sync(0xffffffffu, send.l, o)};
            v[i] = ff_add(keep, t);
        }
    }
    {
        const FF t = {__shfl_xor_sync(0xffffffffu, v[0].h, 1), __shfl_xor_sync(0xffffffffu, v[0].l, 1)};
        v[0] = ff_add(v[0], t);
    }
    uint32_t valid = 0;  // neighbours on the grid, as bits (no runtime index into nb)
#pragma unroll
    for (int e = 0; e < 13; ++e) valid |= (nb[e] >= 0 ? 1u : 0u) << e;
    const int q = lane >> 1;
    if ((lane & 1) == 0 && q < 15) {
        const double dv = (double)v[0].h + (double)v[0].l;
        double *o = out15 + (out_by_point ? p : pos) * 15;
        if (q == 0) o[0] = dv;
        else if (q == 1) o[1] = sf2 - dv;
        else o[q] = (valid >> (q - 2)) & 1u ? pr.k[q - 2] - dv : (double)NAN;
    }
}

__global__ void k_vyff(const double *vy, int64_t mp, float2 *out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= mp) return;
    double v = vy[i];
    float h = (float)v;
    out[i] = make_float2(h, (float)(v - (double)h));
}

// Digits of an FP64 value x with |x| < 2^e: the fixed-point integer q = round(x 2^(42-e))
// (|q| <= 2^42, from the bit pattern) in balanced base 64, q = sum_s d_s 2^(6(6-s)), returned as
// BF16 bit patterns.  Integer work only: |q| is split at bit 18 and each 32-bit half yields three
// digits in [-32, 31] (the carry moving up), the top digit |d_0| <= 64 is what remains; the
// signs follow x.  Zero and subnormal x give 0.
__device__ __forceinline__ void fixed_digits7(double x, int e, uint32_t d[7])
{
    const long long bits = __double_as_longlong(x);
    const int E = (int)((bits >> 52) & 0x7FF);
    unsigned long long q = 0;
    if (E != 0) {
        const unsigned long long mant = (unsigned long long)(bits & 0xFFFFFFFFFFFFFLL) | (1ULL << 52);  // x = mant 2^(E-1075)
        const int rs = 1033 + e - E;  // q = mant 2^-rs, rs >= 11
        if (rs < 63) q = (mant + (1ULL << (rs - 1))) >> rs;
    }
    int lo = (int)(q & 0x3FFFF), hi = (int)(q >> 18), v[7];
#pragma unroll
    for (int t = 6; t >= 4; --t) {
        v[t] = ((lo + 32) & 63) - 32;
        lo = (lo - v[t]) >> 6;
    }
    hi += lo;  // carry out of the low 18 bits (0 or 1)
#pragma unroll
    for (int t = 3; t >= 1; --t) {
        v[t] = ((hi + 32) & 63) - 32;
        hi = (hi - v[t]) >> 6;
    }
    v[0] = hi;
    const int sg = bits < 0 ? -1 : 1;
#pragma unroll
    for (int t = 0; t < 7; ++t) {
        // small integer -> FP32 through the 1.5 * 2^23 magic constant (exact), then its BF16 half
        const float f = __int_as_float(0x4B400000 + sg * v[t]) - 12582912.0f;
        d[t] = __float_as_uint(f) >> 16;
    }
}

// Power-of-two exponent e with |x| < 2^e for every x of a slice whose largest magnitude is mx.
__device__ __forceinline__ int exp_above(double mx)
{
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    return e;
}

// Row digits (K-major as stored): out[s][r][k] for rows r < rows of X (ld ldx, even), k < kv,
// zero to kpad (a multiple of 8); ea[r] the row's exponent.  Warp per row, 8 k per lane.
__global__ void k_oz_rowdig(const double *X, int64_t ldx, int64_t rows, int64_t kv, int64_t kpad, __nv_bfloat16 *out,
                            int *ea)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + warp;
    if (r >= rows) return;
    const double *x = X + r * ldx;
    double mx = 0.0;
    for (int64_t k = lane; k < kv; k += 32) mx = fmax(mx, fabs(x[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = exp_above(mx);
    if (lane == 0) ea[r] = e;
    for (int64_t k0 = (int64_t)lane * 8; k0 < kpad; k0 += 256) {
        double v[8];
        if (k0 + 8 <= kv) {
#pragma unroll
            for (int c = 0; c < 8; c += 2) {
                const double2 p = *(const double2 *)(x + k0 + c);
                v[c] = p.x;
                v[c + 1] = p.y;
            }
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) v[c] = k0 + c < kv ? x[k0 + c] : 0.0;
        }
        uint32_t d[8][7];
#pragma unroll
        for (int c = 0; c < 8; ++c) fixed_digits7(v[c], e, d[c]);
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            uint32_t wd[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) wd[h] = d[2 * h][q] | (d[2 * h + 1][q] << 16);
            *(uint4 *)(out + ((int64_t)q * rows + r) * kpad + k0) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        }
    }
}

// Largest magnitude per column over rows [0, rows) of X (ld ldx), columns < nc: non-negative
// doubles order like their bit patterns, so an integer atomicMax suffices (cmax zeroed first).
__global__ void k_oz_colmax(const double *X, int64_t ldx, int64_t rows, int64_t nc, int64_t rows_per_block,
                            unsigned long long *cmax)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int64_t r0 = blockIdx.y * rows_per_block, r1 = r0 + rows_per_block < rows ? r0 + rows_per_block : rows;
    double mx = 0.0;
    for (int64_t r = r0; r < r1; ++r) mx = fmax(mx, fabs(X[r * ldx + c]));
    atomicMax(cmax + c, (unsigned long long)__double_as_longlong(mx));
}

__global__ void k_oz_colexp(const unsigned long long *cmax, int64_t n, int *e)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c < n) e[c] = exp_above(__longlong_as_double((long long)cmax[c]));
}

// Column digits (the transpose, K-major over rows): out[s][c][r] for columns c < ncpad (zero
// from nc) and rows r < kpad (zero from rows; kpad a multiple of 32), column c scaled by
// 2^-e[c]; with `lower`, X[r][c] = 0 for r < c.  Block: a tile of 64 columns x 32 rows, read
// row by row (coalesced), its digits transposed in shared memory (row pairs as 32-bit words,
// rows padded to 17 words) and written 64 bytes per (slice, column).
__global__ void __launch_bounds__(256) k_oz_coldig(const double *X, int64_t ldx, int64_t rows, int64_t nc,
                                                   int64_t ncpad, int64_t kpad, int lower, const int *e,
                                                   __nv_bfloat16 *out)
{
    __shared__ uint32_t sd[7][64][17];
    const int t = threadIdx.x, cl = t & 63, grp = t >> 6;
    const int64_t c0 = (int64_t)blockIdx.x * 64, r0 = (int64_t)blockIdx.y * 32, c = c0 + cl;
    const int ec = c < nc ? e[c] : 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int rp = grp + 4 * i;  // row pair 0..15
        uint32_t d0[7], d1[7];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t r = r0 + 2 * rp + h;
            const double v = (c < nc && r < rows && !(lower && r < c)) ? X[r * ldx + c] : 0.0;
            fixed_digits7(v, ec, h ? d1 : d0);
        }
#pragma unroll
        for (int q = 0; q < 7; ++q) sd[q][cl][rp] = d0[q] | (d1[q] << 16);
    }
    __syncthreads();
    // 7 x 64 (slice, column) rows of 4 16-byte pieces
    for (int u = t; u < 7 * 64 * 4; u += 256) {
        const int row = u >> 2, k = u & 3, q = row >> 6, cc = row & 63;
        if (c0 + cc >= ncpad) continue;
        const uint32_t *w = &sd[q][cc][4 * k];
        *(uint4 *)(out + ((int64_t)q * ncpad + c0 + cc) * kpad + r0 + 8 * k) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

}  // namespace

struct OzOperands {
    int S = 7;
    int64_t mpt = 0;
    void *B = nullptr;        // S x mpt x mpt BF16 digits
    float *colscale = nullptr;
    float2 *vyff = nullptr;
    CUtensorMap map;
    void *Bc = nullptr;  // S x mpt x mpt BF16 digits of the columns of L^-1 (for X L^-1)
    int *ec = nullptr;   // their exponents
    CUtensorMap mapc;
};

bool oz_supported(const gpr_model *M) { return M->kp.kind == GPR_K_SE; }

static gpr_status oz_prepare_locked(gpr_model *M, cudaStream_t st);

// Lazily built per model; under the model's lock, finished on the stream before it is shared.
gpr_status oz_prepare(gpr_model *M, cudaStream_t st)
{
    std::lock_guard<std::mutex> lock(M->init_mu);
    if (M->oz) return GPR_OK;
    GPR_TRY(oz_prepare_locked(M, st));
    GPR_CUDA_TRY(cudaStreamSynchronize(st));
    return GPR_OK;
}

static gpr_status oz_prepare_locked(gpr_model *M, cudaStream_t st)
{
    if (M->oz) return GPR_OK;
    OzOperands *O = new OzOperands();
    O->mpt = (M->mp + 63) / 64 * 64;
    int64_t mpt = O->mpt, mb = (M->m + 31) / 32 * 32;
    size_t n = (size_t)mpt * mpt;
    cudaError_t e = cudaMalloc(&O->B, n * 2 * (size_t)O->S);
    if (e == cudaSuccess) e = cudaMalloc(&O->colscale, sizeof(float) * mpt);
    if (e == cudaSuccess) e = cudaMalloc(&O->vyff, sizeof(float2) * mpt);
    if (e != cudaSuccess) {
        cudaFree(O->B); cudaFree(O->colscale); cudaFree(O->vyff);
        delete O;
        return e == cudaErrorMemoryAllocation ? GPR_ERR_OOM : GPR_ERR_CUDA;
    }
    GPR_CUDA_TRY(cudaMemsetAsync(O->vyff, 0, sizeof(float2) * mpt, st));
    k_oz_colscale<<<(unsigned)((mpt + 7) / 8), 256, 0, st>>>(M->Linv, mb, M->m, mpt, O->colscale);
    note_launch();
    k_oz_split_b<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M->Linv, mb, M->m, mpt, O->S, O->colscale,
                                                              (__nv_bfloat16 *)O->B);
    note_launch();
    k_vyff<<<(unsigned)((M->mp + 255) / 256), 256, 0, st>>>(M->vy, M->mp, O->vyff);
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    auto enc = encoder();
    if (!enc) { M->oz = O; return GPR_ERR_UNSUPPORTED; }
    cuuint64_t gdim[3] = {(cuuint64_t)mpt, (cuuint64_t)mpt, (cuuint64_t)O->S};
    cuuint64_t gstride[2] = {(cuuint64_t)mpt * 2, (cuuint64_t)mpt * mpt * 2};
    cuuint32_t box[3] = {BKE, TN, (cuuint32_t)O->S};  // all slices of a K block in one copy
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&O->map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, O->B, gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    M->oz = O;
    return r == CUDA_SUCCESS ? GPR_OK : GPR_ERR_UNSUPPORTED;
}

void oz_release(gpr_model *M)
{
    if (!M->oz) return;
    cudaFree(M->oz->B); cudaFree(M->oz->colscale); cudaFree(M->oz->vyff);
    cudaFree(M->oz->Bc); cudaFree(M->oz->ec);
    delete M->oz;
    M->oz = nullptr;
}

gpr_status oz_unit_tables(const gpr_model *M, const GridDev &g, float2 *Tu, cudaStream_t st)
{
    int64_t total = (int64_t)table_elems(M, g);
    k_unit_tables<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(M->X, M->m, M->mp, M->kp, g, Tu);
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

// Device scratch for the A digit slices, shared by host threads (batched workers): a buffer is
// reused only after the stream that last used it has passed its release event.
struct AdigBuf {
    void *p = nullptr;
    size_t bytes = 0;
    bool busy = false;
    cudaEvent_t released = nullptr;
};
std::mutex g_adig_mu;
std::vector<AdigBuf *> g_adig;

gpr_status adig_acquire(size_t bytes, cudaStream_t st, AdigBuf **out)
{
    AdigBuf *b = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_adig_mu);
        for (AdigBuf *c : g_adig)
            if (!c->busy && c->bytes >= bytes) { b = c; break; }
        if (!b)
            for (AdigBuf *c : g_adig)
                if (!c->busy) { b = c; break; }
        if (!b) {
            b = new AdigBuf();
            g_adig.push_back(b);
        }
        b->busy = true;
    }
    if (!b->released) GPR_CUDA_TRY(cudaEventCreateWithFlags(&b->released, cudaEventDisableTiming));
    if (b->bytes < bytes) {
        GPR_CUDA_TRY(cudaEventSynchronize(b->released));
        cudaFree(b->p);
        b->p = nullptr;
        b->bytes = 0;
        cudaError_t e = cudaMalloc(&b->p, bytes);
        if (e != cudaSuccess) {
            std::lock_guard<std::mutex> lock(g_adig_mu);
            b->busy = false;
            return e == cudaErrorMemoryAllocation ? GPR_ERR_OOM : GPR_ERR_CUDA;
        }
        b->bytes = bytes;
    }
    GPR_CUDA_TRY(cudaStreamWaitEvent(st, b->released, 0));
    *out = b;
    return GPR_OK;
}

// Frees the pooled digit buffers no call is using (after their last use has finished).
void adig_free_idle()
{
    std::lock_guard<std::mutex> lock(g_adig_mu);
    std::vector<AdigBuf *> keep;
    for (AdigBuf *b : g_adig) {
        if (b->busy) {
            keep.push_back(b);
            continue;
        }
        if (b->released) {
            cudaEventSynchronize(b->released);
            cudaEventDestroy(b->released);
        }
        cudaFree(b->p);
        delete b;
    }
    g_adig.swap(keep);
}

void adig_release(AdigBuf *b, cudaStream_t st)
{
    cudaEventRecord(b->released, st);
    std::lock_guard<std::mutex> lock(g_adig_mu);
    b->busy = false;
}

// The W rows with the A digits staged in HBM by k_oz_adig first, in row chunks whose digits
// (S x rows x mpt BF16) fit 1.5 GB, and loaded by TMA in k_oz_gemm.
static gpr_status oz_w_staged(const gpr_model *M, const GridDev &g, const float2 *Tu, const int64_t *pts,
                              int64_t pt_base, int64_t count, float2 *W, cudaStream_t st, bool out_by_point,
                              int64_t row_mod)
{
    if (count <= 0) return GPR_OK;
    const OzOperands *O = M->oz;
    if (!O) return GPR_ERR_ARG;
    auto enc = encoder();
    if (!enc) return GPR_ERR_UNSUPPORTED;
    constexpr int S = 7;
    OzParams prm;
    prm.Tu = Tu;
    prm.off1 = (int64_t)g.n[0] * M->mp;
    prm.off2 = prm.off1 + (int64_t)g.n[1] * M->mp;
    prm.mp = M->mp;
    prm.mpt = O->mpt;
    prm.m = M->m;
    prm.g = g;
    prm.colscale = O->colscale;
    prm.sf2 = (float)M->kp.sf2;
    prm.W = W;
    prm.out_by_point = out_by_point ? 1 : 0;
    prm.row_mod = row_mod > 0 ? row_mod : g.npts();
    prm.status = gpr_status_word();
    if (!prm.status) return GPR_ERR_CUDA;
    const size_t per_row = (size_t)O->mpt * 2 * S;
    int64_t chunk = (int64_t)(((size_t)3 << 29) / per_row) / TM * TM;
    if (chunk < TM) chunk = TM;
    if (chunk > count) chunk = count;
    size_t smem = 2 * (size_t)(S * A_SLICE + S * B_SLICE) + 64 + 1024;
    GPR_CUDA_TRY(cudaFuncSetAttribute(k_oz_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    AdigBuf *buf = nullptr;
    GPR_TRY(adig_acquire((size_t)chunk * per_row, st, &buf));
    gpr_status rs = GPR_OK;
    for (int64_t c0 = 0; c0 < count && rs == GPR_OK; c0 += chunk) {
        const int64_t cnt = count - c0 < chunk ? count - c0 : chunk;
        prm.pts = pts ? pts + c0 : nullptr;
        prm.pt_base = pt_base + c0;
        prm.count = cnt;
        prm.out_off = c0;
        const int64_t nthr = cnt * (O->mpt / 8);
        {
            ProfScope ps("oz_adig", st, (double)cnt);
            k_oz_adig<<<(unsigned)((nthr + 255) / 256), 256, 0, st>>>(prm, (__nv_bfloat16 *)buf->p);
        }
        note_launch();
        CUtensorMap mapA;
        cuuint64_t gdim[3] = {(cuuint64_t)O->mpt, (cuuint64_t)cnt, (cuuint64_t)S};
        cuuint64_t gstride[2] = {(cuuint64_t)O->mpt * 2, (cuuint64_t)cnt * O->mpt * 2};
        cuuint32_t box[3] = {BKE, TM, (cuuint32_t)S};
        cuuint32_t estr[3] = {1, 1, 1};
        if (enc(&mapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, buf->p, gdim, gstride, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
            rs = GPR_ERR_UNSUPPORTED;
            break;
        }
        dim3 grid((unsigned)(M->mp / TN), (unsigned)((cnt + TM - 1) / TM));  // row tiles < 65536 per chunk
        {
            ProfScope ps("oz_w", st, (double)cnt);
            k_oz_gemm<S><<<grid, G_NTHR, smem, st>>>(mapA, O->map, prm);
        }
        note_launch();
        if (cudaGetLastError() != cudaSuccess) rs = GPR_ERR_CUDA;
    }
    adig_release(buf, st);
    return rs;
}

// The same rows with the A digits generated inside the GEMM (k_oz_gemm_gen): nothing is staged in
// HBM; launches of <= 65535 row tiles.
static gpr_status oz_w_fused(const gpr_model *M, const GridDev &g, const float2 *Tu, const int64_t *pts,
                             int64_t pt_base, int64_t count, float2 *W, cudaStream_t st, bool out_by_point,
                             int64_t row_mod)
{
    const OzOperands *O = M->oz;
    constexpr int S = 7;
    OzParams prm;
    prm.Tu = Tu;
    prm.off1 = (int64_t)g.n[0] * M->mp;
    prm.off2 = prm.off1 + (int64_t)g.n[1] * M->mp;
    prm.mp = M->mp;
    prm.mpt = O->mpt;
    prm.m = M->m;
    prm.g = g;
    prm.colscale = O->colscale;
    prm.sf2 = (float)M->kp.sf2;
    prm.W = W;
    prm.out_by_point = out_by_point ? 1 : 0;
    prm.row_mod = row_mod > 0 ? row_mod : g.npts();
    prm.status = gpr_status_word();
    if (!prm.status) return GPR_ERR_CUDA;
    size_t smem = 2 * (size_t)(S * A_SLICE + S * B_SLICE) + 64 + 1024;
    GPR_CUDA_TRY(cudaFuncSetAttribute(k_oz_gemm_gen<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t chunk = (int64_t)65535 * TM;
    for (int64_t c0 = 0; c0 < count; c0 += chunk) {
        const int64_t cnt = count - c0 < chunk ? count - c0 : chunk;
        prm.pts = pts ? pts + c0 : nullptr;
        prm.pt_base = pt_base + c0;
        prm.count = cnt;
        prm.out_off = c0;
        dim3 grid((unsigned)(M->mp / TN), (unsigned)((cnt + TM - 1) / TM));
        {
            ProfScope ps("oz_w", st, (double)cnt);
            k_oz_gemm_gen<S><<<grid, G_NTHR, smem, st>>>(O->map, prm);
        }
        note_launch();
        GPR_CUDA_TRY(cudaGetLastError());
    }
    return GPR_OK;
}

// Float-float W rows of the listed points on the tensor cores: row r of the list goes to row r
// of W (count x mp float2), or to row p % row_mod for point p when out_by_point.  Two kernels with
// the same digits and the same MMA order (so the same bits): A digits generated in the GEMM (no
// HBM traffic but the kernel rows' digits, but regenerated by every 64-column tile), or staged in
// HBM once by k_oz_adig; the autotuner keeps the faster per (row count, column tiles) bucket.
gpr_status launch_oz_w(const gpr_model *M, const GridDev &g, const float2 *Tu, const int64_t *pts, int64_t pt_base,
                       int64_t count, float2 *W, cudaStream_t st, bool out_by_point, int64_t row_mod)
{
    if (count <= 0) return GPR_OK;
    if (!M->oz) return GPR_ERR_ARG;
    if (!encoder()) return GPR_ERR_UNSUPPORTED;
    auto run = [&](int c) -> gpr_status {
        return c == 0 ? oz_w_fused(M, g, Tu, pts, pt_base, count, W, st, out_by_point, row_mod)
                      : oz_w_staged(M, g, Tu, pts, pt_base, count, W, st, out_by_point, row_mod);
    };
    // key: the row count's bucket and the number of 64-column tiles (the fused kernel regenerates a
    // row block's digits once per tile, so its cost relative to staging grows with the model size)
    return tune_run("oz_w_kernel", tune_bucket(count) * 256 + M->mp / TN, 2, run, st);
}

gpr_status launch_stats_ff(const gpr_model *M, const GridDev &g, const int64_t *pts, int64_t count, const int32_t *slot,
                           const float2 *W, double *out15, cudaStream_t st, bool out_by_point,
                           int64_t row_mod)
{
    if (count <= 0) return GPR_OK;
    Prior13 pr;
    for (int e = 0; e < 13; ++e) {
        double r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            double t = kOff13[e][d] * g.h[d] / M->kp.ell[d];
            r2 += t * t;
        }
        pr.k[e] = M->kp.sf2 * exp(-0.5 * r2);
    }
    {
        ProfScope ps("stats_ff", st, (double)count);
        k_stats_ff<<<(unsigned)((count + 7) / 8), 256, 0, st>>>(g, pts, count, slot, W, M->mp, M->m, M->oz->vyff,
                                                              M->kp.sf2, pr, out15, out_by_point ? 1 : 0,
                                                              row_mod > 0 ? row_mod : g.npts());
    }
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

// 3-D tensor map over BF16 digit slices [S][rows][kpad], boxes of BKE digits x box_rows x S.
static bool encode_digits(CUtensorMap *map, void *base, int64_t kpad, int64_t rows, int box_rows)
{
    auto enc = encoder();
    if (!enc) return false;
    constexpr int S = 7;
    cuuint64_t gdim[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)S};
    cuuint64_t gstride[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)rows * kpad * 2};
    cuuint32_t box[3] = {BKE, (cuuint32_t)box_rows, (cuuint32_t)S};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static size_t dgemm_smem()
{
    constexpr int S = 7;
    return 2 * (size_t)(S * A_SLICE + S * B_SLICE) + 64 + 1024;
}

// Digits of the columns of L^-1 (lower triangular), built once per model.
gpr_status oz_prepare_cols(gpr_model *M, cudaStream_t st)
{
    GPR_TRY(oz_prepare(M, st));
    std::lock_guard<std::mutex> lock(M->init_mu);
    OzOperands *O = M->oz;
    if (O->Bc) return GPR_OK;
    constexpr int S = 7;
    const int64_t mpt = O->mpt, m = M->m, mb = (m + 31) / 32 * 32;
    void *Bc = nullptr;
    int *ec = nullptr;
    unsigned long long *cmax = nullptr;
    cudaError_t e = cudaMalloc(&Bc, (size_t)S * mpt * mpt * 2);
    if (e == cudaSuccess) e = cudaMalloc(&ec, sizeof(int) * mpt);
    if (e == cudaSuccess) e = cudaMalloc(&cmax, sizeof(unsigned long long) * mpt);
    if (e != cudaSuccess) {
        cudaFree(Bc); cudaFree(ec); cudaFree(cmax);
        return e == cudaErrorMemoryAllocation ? GPR_ERR_OOM : GPR_ERR_CUDA;
    }
    GPR_CUDA_TRY(cudaMemsetAsync(cmax, 0, sizeof(unsigned long long) * mpt, st));
    GPR_CUDA_TRY(cudaMemsetAsync(ec, 0, sizeof(int) * mpt, st));
    k_oz_colmax<<<dim3((unsigned)((m + 255) / 256), (unsigned)((m + 63) / 64)), 256, 0, st>>>(M->Linv, mb, m, m, 64, cmax);
    k_oz_colexp<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(cmax, m, ec);
    k_oz_coldig<<<dim3((unsigned)(mpt / 64), (unsigned)(mpt / 32)), 256, 0, st>>>(M->Linv, mb, m, m, mpt, mpt, 1, ec,
                                                                                (__nv_bfloat16 *)Bc);
    note_launch();
    note_launch();
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    GPR_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(cmax);
    if (!encode_digits(&O->mapc, Bc, mpt, mpt, TN)) {
        cudaFree(Bc); cudaFree(ec);
        return GPR_ERR_UNSUPPORTED;
    }
    O->ec = ec;
    O->Bc = Bc;
    return GPR_OK;
}

// FP64-class C = X L^-1 (X: rows x m FP64, ld ldx; C: rows x m, ld ldc) on the tensor cores.
gpr_status oz_mul_linv(gpr_model *M, const double *X, int64_t rows, int64_t ldx, double *C, int64_t ldc,
                       cudaStream_t st)
{
    if (rows <= 0) return GPR_OK;
    GPR_TRY(oz_prepare_cols(M, st));
    const OzOperands *O = M->oz;
    constexpr int S = 7;
    const int64_t mpt = O->mpt, m = M->m;
    const size_t per_row = (size_t)mpt * 2 * S + sizeof(int);
    int64_t chunk = (int64_t)(((size_t)3 << 29) / per_row) / TM * TM;
    if (chunk < TM) chunk = TM;
    if (chunk > rows) chunk = rows;
    const size_t smem = dgemm_smem();
    GPR_CUDA_TRY(cudaFuncSetAttribute(k_oz_dgemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    AdigBuf *buf = nullptr;
    GPR_TRY(adig_acquire((size_t)chunk * per_row + 256, st, &buf));
    __nv_bfloat16 *dig = (__nv_bfloat16 *)buf->p;
    int *ea = (int *)((char *)buf->p + (size_t)chunk * mpt * 2 * S);
    OzG prm;
    prm.N = m;
    prm.kblocks = (m + BKE - 1) / BKE;
    prm.kb_per_split = prm.kblocks;
    prm.lower_b = 1;
    prm.accumulate = 0;
    prm.ea = ea;
    prm.eb = O->ec;
    prm.ldc = ldc;
    prm.cstride = 0;
    prm.status = gpr_status_word();
    gpr_status rs = prm.status ? GPR_OK : GPR_ERR_CUDA;
    for (int64_t c0 = 0; c0 < rows && rs == GPR_OK; c0 += chunk) {
        const int64_t cnt = rows - c0 < chunk ? rows - c0 : chunk;
        k_oz_rowdig<<<(unsigned)((cnt + 7) / 8), 256, 0, st>>>(X + c0 * ldx, ldx, cnt, m, mpt, dig, ea);
        note_launch();
        CUtensorMap mapA;
        if (!encode_digits(&mapA, dig, mpt, cnt, TM)) { rs = GPR_ERR_UNSUPPORTED; break; }
        prm.M = cnt;
        prm.C = C + c0 * ldc;
        k_oz_dgemm<S><<<dim3((unsigned)(mpt / TN), (unsigned)((cnt + TM - 1) / TM), 1), G_NTHR, smem, st>>>(mapA, O->mapc,
                                                                                                      prm);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) rs = GPR_ERR_CUDA;
    }
    adig_release(buf, st);
    return rs;
}

// FP64-class C = A^T B for A, B: K x nc FP64 (row-major, ld) on the tensor cores, as nsplit
// partial products part[z] (ncp x ncp each, ncp = nc rounded up to 64, zero beyond nc) whose
// sum is C.  K runs in chunks whose digits fit 2 GB, each chunk scaled by its own column
// exponents and added onto the partials in order (deterministic).
gpr_status oz_mul_tn(const double *A, const double *B, int64_t K, int64_t nc, int64_t ld, double *part, int nsplit,
                     cudaStream_t st, int64_t kchunk)
{
    constexpr int S = 7;
    const int64_t ncp = (nc + 63) / 64 * 64;
    if (K <= 0) {
        GPR_CUDA_TRY(cudaMemsetAsync(part, 0, sizeof(double) * (size_t)nsplit * ncp * ncp, st));
        return GPR_OK;
    }
    int64_t kc = kchunk > 0 ? (kchunk + 31) / 32 * 32 : (int64_t)131072 * 512 / ncp / 32 * 32;
    const int64_t kall = (K + 31) / 32 * 32;
    if (kc > kall) kc = kall;
    const size_t dig_bytes = (size_t)S * ncp * kc * 2;
    const size_t bytes = 2 * dig_bytes + 2 * ncp * (sizeof(unsigned long long) + sizeof(int)) + 256;
    const size_t smem = dgemm_smem();
    GPR_CUDA_TRY(cudaFuncSetAttribute(k_oz_dgemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    AdigBuf *buf = nullptr;
    GPR_TRY(adig_acquire(bytes, st, &buf));
    __nv_bfloat16 *dA = (__nv_bfloat16 *)buf->p, *dB = (__nv_bfloat16 *)((char *)buf->p + dig_bytes);
    unsigned long long *cmax = (unsigned long long *)((char *)buf->p + 2 * dig_bytes);
    int *eA = (int *)(cmax + 2 * ncp), *eB = eA + ncp;
    OzG prm;
    prm.M = ncp;
    prm.N = ncp;
    prm.lower_b = 0;
    prm.ea = eA;
    prm.eb = eB;
    prm.C = part;
    prm.ldc = ncp;
    prm.cstride = ncp * ncp;
    prm.status = gpr_status_word();
    gpr_status rs = prm.status ? GPR_OK : GPR_ERR_CUDA;
    for (int64_t c0 = 0; c0 < K && rs == GPR_OK; c0 += kc) {
        const int64_t cnt = K - c0 < kc ? K - c0 : kc, kpad = (cnt + 31) / 32 * 32;
        GPR_CUDA_TRY(cudaMemsetAsync(cmax, 0, sizeof(unsigned long long) * 2 * ncp, st));
        const int64_t rpb = 512;
        const dim3 gmax((unsigned)((nc + 255) / 256), (unsigned)((cnt + rpb - 1) / rpb));
        k_oz_colmax<<<gmax, 256, 0, st>>>(A + c0 * ld, ld, cnt, nc, rpb, cmax);
        k_oz_colmax<<<gmax, 256, 0, st>>>(B + c0 * ld, ld, cnt, nc, rpb, cmax + ncp);
        k_oz_colexp<<<(unsigned)((2 * ncp + 255) / 256), 256, 0, st>>>(cmax, 2 * ncp, eA);
        const dim3 gdig((unsigned)(ncp / 64), (unsigned)(kpad / 32));
        k_oz_coldig<<<gdig, 256, 0, st>>>(A + c0 * ld, ld, cnt, nc, ncp, kpad, 0, eA, dA);
        k_oz_coldig<<<gdig, 256, 0, st>>>(B + c0 * ld, ld, cnt, nc, ncp, kpad, 0, eB, dB);
        for (int q = 0; q < 5; ++q) note_launch();
        CUtensorMap mapA, mapB;
        if (!encode_digits(&mapA, dA, kpad, ncp, TM) || !encode_digits(&mapB, dB, kpad, ncp, TN)) {
            rs = GPR_ERR_UNSUPPORTED;
            break;
        }
        prm.kblocks = kpad / BKE;
        prm.kb_per_split = (prm.kblocks + nsplit - 1) / nsplit;
        prm.accumulate = c0 > 0;
        k_oz_dgemm<S><<<dim3((unsigned)(ncp / TN), (unsigned)((ncp + TM - 1) / TM), (unsigned)nsplit), G_NTHR, smem,
                        st>>>(mapA, mapB, prm);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) rs = GPR_ERR_CUDA;
    }
    adig_release(buf, st);
    return rs;
}

__global__ void k_fill_slot_oz(const int64_t *idx, int64_t count, int64_t npts, int32_t *slot)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count && idx[i] >= 0 && idx[i] < npts) slot[idx[i]] = (int32_t)i;
}

// Test hook (not in the public header): stats15 of listed points through the tensor-core
// digit-split path, for parity tests against the FP64 path and the oracle.
extern "C" gpr_status gpr_stats_points_split(gpr_model *M, const gpr_grid *grid, const int64_t *point_idx,
                                             int64_t count, double *stats, void *stream)
{
    if (!M || !grid_valid(grid) || count <= 0 || !point_idx || !stats) return GPR_ERR_ARG;
    if (!oz_supported(M)) return GPR_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    GridDev g = make_grid(grid);
    size_t te = table_elems(M, g);
    size_t bytes = Carver::round(te * sizeof(float2)) + Carver::round((size_t)g.npts() * 4) +
                   Carver::round((size_t)count * M->mp * 8) + 1024;
    GPR_TRY(ws_reserve(M, 0, bytes, st));
    Carver cv{(char *)ws_ptr(M, 0)};
    float2 *Tu = cv.take<float2>(te);
    int32_t *slot = cv.take<int32_t>((size_t)g.npts());
    float2 *W = cv.take<float2>((size_t)count * M->mp);
    GPR_TRY(oz_prepare(M, st));
    GPR_TRY(oz_unit_tables(M, g, Tu, st));
    GPR_CUDA_TRY(cudaMemsetAsync(slot, 0xff, sizeof(int32_t) * (size_t)g.npts(), st));
    k_fill_slot_oz<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(point_idx, count, g.npts(), slot);
    note_launch();
    GPR_TRY(launch_oz_w(M, g, Tu, point_idx, 0, count, W, st));
    GPR_TRY(launch_stats_ff(M, g, point_idx, count, slot, W, stats, st));
    return GPR_OK;
}

__global__ void k_sum_parts(const double *part, int n, int64_t len, double *out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= len) return;
    double s = 0.0;
    for (int z = 0; z < n; ++z) s += part[z * len + i];
    out[i] = s;
}

// Test hooks (not in the public header) for the FP64-class products: C (nc x nc, device) =
// A^T B with A, B device K x nc (ld nc) in K chunks of kchunk rows (0: default), and
// C (rows x m, ld m) = X L^-1 for device X (rows x m, ld m).
extern "C" gpr_status gpr_oz_mul_tn_test(const double *A, const double *B, int64_t K, int64_t nc, int64_t kchunk,
                                         int32_t nsplit, double *C, void *stream)
{
    if (!A || !B || !C || K < 0 || nc <= 0 || nsplit <= 0 || nsplit > 64) return GPR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t ncp = (nc + 63) / 64 * 64;
    double *part = nullptr, *full = nullptr;
    GPR_CUDA_TRY(cudaMalloc(&part, sizeof(double) * (size_t)nsplit * ncp * ncp));
    GPR_CUDA_TRY(cudaMalloc(&full, sizeof(double) * (size_t)ncp * ncp));
    gpr_status rs = oz_mul_tn(A, B, K, nc, nc, part, nsplit, st, kchunk);
    if (rs == GPR_OK) {
        k_sum_parts<<<(unsigned)((ncp * ncp + 255) / 256), 256, 0, st>>>(part, nsplit, ncp * ncp, full);
        cudaMemcpy2DAsync(C, nc * sizeof(double), full, ncp * sizeof(double), nc * sizeof(double), nc,
                          cudaMemcpyDeviceToDevice, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) rs = GPR_ERR_CUDA;
    }
    cudaFree(part);
    cudaFree(full);
    return rs;
}

extern "C" gpr_status gpr_oz_mul_linv_test(gpr_model *M, const double *X, int64_t rows, double *C, void *stream)
{
    if (!M || !X || !C || rows < 0) return GPR_ERR_ARG;
    if (!oz_supported(M)) return GPR_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    GPR_TRY(oz_mul_linv(M, X, rows, M->m, C, M->m, st));
    GPR_CUDA_TRY(cudaStreamSynchronize(st));
    return GPR_OK;
}
