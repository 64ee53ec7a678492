// Whitened contraction W = K_* L^-T on the 5th-generation tensor cores (tcgen05, sm_103a),
// reduced on the fly to var = k(x,x) - |w|^2 (Eq. 1, whitened form).
//
// One CTA per (128-point row tile, N-column tile).  A (the kernel rows, M x K, K-major) is
// generated by all warps from the separable tables directly into shared memory in the
// canonical 128-byte-swizzled K-major layout, split into TF32 hi/lo or three BF16 slices.
// B = rows of L^-1 (N x K, K-major, pre-split on the device at model set-up) arrives by TMA
// (cp.async.bulk.tensor, 128B swizzle).  One thread issues tcgen05.mma into a TMEM
// accumulator (FP32, 128 lanes x N columns); two pipeline stages overlap the generation of
// the next A tile with the MMAs of the current one.  The epilogue reads TMEM with
// tcgen05.ld and sums w^2 per row; a partial per N tile goes to global memory.
// Split products (Ootomo & Yokota 2022): TF32x3 = hi*hi + hi*lo + lo*hi;
// BF16x3 = sum over slice pairs (i, j) with i + j <= 2 (six products).
// Every mbarrier wait is bounded; a wait that runs out records GPR_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>

#include <mutex>

#include "internal.h"

namespace {

constexpr int TM = 128;          // rows (points) per tile = TMEM lanes
constexpr int NTHR = 256;        // 8 warps
constexpr uint32_t kSpinLimit = 1u << 22;

template <int P>
struct Cfg;
// P = precision code (GPR_P_TF32 .. GPR_P_BF16X3)
template <>
struct Cfg<GPR_P_TF32> {
    static constexpr int NA = 1, NB = 1, NPROD = 1, BKE = 32, ESZ = 4;
    static constexpr bool BF = false;
};
template <>
struct Cfg<GPR_P_TF32X3> {
    static constexpr int NA = 2, NB = 2, NPROD = 3, BKE = 32, ESZ = 4;
    static constexpr bool BF = false;
};
template <>
struct Cfg<GPR_P_BF16> {
    static constexpr int NA = 1, NB = 1, NPROD = 1, BKE = 64, ESZ = 2;
    static constexpr bool BF = true;
};
template <>
struct Cfg<GPR_P_BF16X3> {
    static constexpr int NA = 3, NB = 3, NPROD = 6, BKE = 64, ESZ = 2;
    static constexpr bool BF = true;
};

// slice pairs (a, b) of the split products
__device__ __forceinline__ void prod_pair(int P, int t, int &a, int &b)
{
    if (P == GPR_P_TF32X3) {
        const int pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0};
        a = pa[t]; b = pb[t];
    } else if (P == GPR_P_BF16X3) {
        const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
        a = pa[t]; b = pb[t];
    } else {
        a = 0; b = 0;
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // leading-dimension offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride-dimension offset: 1024 B
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}

// Instruction descriptor: D = F32, A/B = TF32 (kind::tf32) or BF16 (kind::f16), K-major, M x N.
template <bool BF>
__host__ __device__ constexpr uint32_t idesc(int M, int N)
{
    return (1u << 4) | ((BF ? 1u : 2u) << 7) | ((BF ? 1u : 2u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
// Bounded wait on phase `parity`; returns false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity)
{
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(mbar)
        : "memory");
}

template <bool BF>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    if (BF)
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                         tmem_d),
                     "l"(a), "l"(b), "r"(id), "r"(acc));
    else
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                         tmem_d),
                     "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ float tf32_round(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

struct TcParams {
    const float *T32;
    int64_t off1, off2, mp, m;
    int kind;
    float sf2;
    GridDev g;
    const int64_t *pts;
    int64_t pt_base, count;
    float *partial;  // count x nN partial sums of w^2, one per 64 columns
    float *W;        // nullable: the whitened rows themselves (count x mp), plain kernel only
    int64_t plen;    // floats in `partial` (bounds self-check)
    int64_t tlen;    // floats in T32 (bounds self-check)
    int nN;
    int *status;
};

// One 16-byte chunk c (of 8) of row r of the A tile for K block kb, in every A slice of the
// stage: kernel values from the separable FP32 tables, split as the precision wants (TF32 hi/lo
// or three BF16 slices), stored in the 128-byte-swizzled K-major layout.
template <int P>
__device__ __forceinline__ void gen_a_chunk(const TcParams &prm, unsigned char *st, int r, int c, int kb,
                                            const int *gx, const int *gy, const int *gz, const bool *rvalid)
{
    using C = Cfg<P>;
    constexpr int BKE = C::BKE;
    constexpr int A_TILE = TM * 128;
    const int64_t m = prm.m;
    const int64_t k0 = (int64_t)kb * BKE + c * (16 / C::ESZ);
    float v[8];
    constexpr int EPC = 16 / C::ESZ;  // elements per chunk
#pragma unroll
    for (int e = 0; e < EPC; ++e) v[e] = 0.f;
    if (rvalid[r]) {
        const float *tx = prm.T32 + (int64_t)gx[r] * prm.mp, *ty = prm.T32 + prm.off1 + (int64_t)gy[r] * prm.mp,
                    *tz = prm.T32 + prm.off2 + (int64_t)gz[r] * prm.mp;
#pragma unroll
        for (int e = 0; e < EPC; ++e) {
            int64_t j = k0 + e;
            if (j < m && prm.off2 + (int64_t)gz[r] * prm.mp + j >= prm.tlen) {
                atomicCAS(prm.status, 0, (int)GPR_ERR_ARG);  // self-check: never expected
            } else if (j < m) {
                float a = tx[j], b = ty[j], cc = tz[j];
                if (prm.kind == GPR_K_SE) {
                    v[e] = a * b * cc;
                } else {
                    float r2 = a + b + cc, rr = sqrtf(r2), s5r = 2.23606797749979f * rr;
                    v[e] = prm.sf2 * (1.0f + s5r + (5.0f / 3.0f) * r2) * __expf(-s5r);
                }
            }
        }
    }
    const int off = r * 128 + ((c ^ (r & 7)) << 4);
    if (!C::BF) {
        float4 hi, lo;
        float *h = &hi.x, *l = &lo.x;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            h[e] = tf32_round(v[e]);
            l[e] = tf32_round(v[e] - h[e]);
        }
        *(float4 *)(st + off) = hi;
        if (C::NA > 1) *(float4 *)(st + A_TILE + off) = lo;
    } else {
        uint32_t wd[3][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            uint32_t bits[3][2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float x = v[e + h];
                __nv_bfloat16 b0 = __float2bfloat16_rn(x);
                float r1 = x - __bfloat162float(b0);
                __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
                float r2 = r1 - __bfloat162float(b1);
                __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
                bits[0][h] = __bfloat16_as_ushort(b0);
                bits[1][h] = __bfloat16_as_ushort(b1);
                bits[2][h] = __bfloat16_as_ushort(b2);
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) wd[a][e / 2] = bits[a][0] | (bits[a][1] << 16);
        }
#pragma unroll
        for (int a = 0; a < C::NA; ++a)
            *(uint4 *)(st + a * A_TILE + off) = make_uint4(wd[a][0], wd[a][1], wd[a][2], wd[a][3]);
    }
}

// The MMAs of one 128-byte K block, in the order every variant uses (so all give the same bits):
// TF32 K blocks are issued as two 16-element halves, each product over its two K steps in turn
// (the order of the 64-byte-row variant below); BF16 blocks product by product over four K steps.
template <int P, int N>
__device__ __forceinline__ void issue_block128(uint32_t tmem, uint32_t abase0, uint32_t bbase0, bool first)
{
    using C = Cfg<P>;
    constexpr int A_TILE = TM * 128, B_TILE = N * 128;
    constexpr uint32_t ID = idesc<C::BF>(TM, N);
    constexpr int H = C::BF ? 1 : 2;  // halves of the block
#pragma unroll
    for (int h = 0; h < H; ++h)
        for (int t = 0; t < C::NPROD; ++t) {
            int ia, ib;
            prod_pair(P, t, ia, ib);
            const uint32_t abase = abase0 + ia * A_TILE, bbase = bbase0 + ib * B_TILE;
#pragma unroll
            for (int k2 = 0; k2 < 4 / H; ++k2) {
                const int kk = h * (4 / H) + k2;
                const uint32_t acc = (!first || h > 0 || t > 0 || k2 > 0) ? 1u : 0u;
                mma<C::BF>(tmem, desc_sw128(abase + kk * 32), desc_sw128(bbase + kk * 32), ID, acc);
            }
        }
}

// N: output columns per tile (64, 128 or 256; chosen per model size by the autotuner).  The
// squares are summed per 32-column chunk and paired into 64-column partials, the same grouping
// for every N, so all tile widths give the same bits.
template <int P, int N>
__global__ void __launch_bounds__(NTHR, 1) k_tc_sumsq(const __grid_constant__ CUtensorMap mapB0,
                                                     const __grid_constant__ CUtensorMap mapB1,
                                                     const __grid_constant__ CUtensorMap mapB2, TcParams prm)
{
    using C = Cfg<P>;
    constexpr int BKE = C::BKE;
    constexpr int A_TILE = TM * 128;   // bytes per A slice per stage
    constexpr int B_TILE = N * 128;    // bytes per B slice per stage
    constexpr int STAGE = C::NA * A_TILE + C::NB * B_TILE;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(smem + 2 * STAGE);  // full[2], free[2], done
    __shared__ uint32_t tmem_slot;
    __shared__ int gx[TM], gy[TM], gz[TM];
    __shared__ bool rvalid[TM];
    __shared__ float red[N / 32][TM];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row0 = (int64_t)blockIdx.x * TM;
    const int n0 = blockIdx.y * N;
    const int64_t m = prm.m;
    const int64_t kend = (int64_t)n0 + N < m ? (int64_t)n0 + N : m;
    const int nkb = (int)((kend + BKE - 1) / BKE);
    const uint32_t bar_full0 = smem_u32(&bars[0]), bar_free0 = smem_u32(&bars[2]), bar_done = smem_u32(&bars[4]);

    if (tid == 0) {
        mbar_init(bar_full0, 1);
        mbar_init(bar_full0 + 8, 1);
        mbar_init(bar_free0, 1);
        mbar_init(bar_free0 + 8, 1);
        mbar_init(bar_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"((uint32_t)N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int r = tid; r < TM; r += NTHR) {
        int64_t row = row0 + r;
        bool ok = row < prm.count;
        int64_t p = ok ? (prm.pts ? prm.pts[row] : prm.pt_base + row) : 0;
        int64_t nx = prm.g.n[0], ny = prm.g.n[1];
        if (p < 0 || p >= nx * ny * (int64_t)prm.g.n[2]) { ok = false; p = 0; }
        gx[r] = (int)(p % nx);
        gy[r] = (int)((p / nx) % ny);
        gz[r] = (int)(p / (nx * ny));
        rvalid[r] = ok;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    bool ok_all = true;
    const CUtensorMap *maps[3] = {&mapB0, &mapB1, &mapB2};

    for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb & 1, use = kb >> 1;
        unsigned char *st = smem + s * STAGE;
        if (kb >= 2) {
            if (!mbar_wait(bar_free0 + 8 * s, (use - 1) & 1)) ok_all = false;
        }
        if (tid == 0) {
            mbar_expect_tx(bar_full0 + 8 * s, (uint32_t)(C::NB * B_TILE));
            for (int b = 0; b < C::NB; ++b)
                tma_load_2d(smem_u32(st + C::NA * A_TILE + b * B_TILE), maps[b], kb * BKE, n0, bar_full0 + 8 * s);
        }
        // A tile: 128 rows x 128 bytes per slice; one 16-byte chunk per (row, c)
        for (int q = tid; q < TM * 8; q += NTHR) gen_a_chunk<P>(prm, st, q >> 3, q & 7, kb, gx, gy, gz, rvalid);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            if (!mbar_wait(bar_full0 + 8 * s, use & 1)) ok_all = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            issue_block128<P, N>(tmem, smem_u32(st), smem_u32(st + C::NA * A_TILE), kb == 0);
            mma_commit(bar_free0 + 8 * s);
            if (kb == nkb - 1) mma_commit(bar_done);
        }
    }
    // epilogue: warp w reads TMEM lanes 32*(w%4).., column half w/4
    if (!mbar_wait(bar_done, 0)) ok_all = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int lq = warp & 3, half = warp >> 2;
#pragma unroll
    for (int c0 = 0; c0 < N / 2; c0 += 32) {
        uint32_t rr[32];
        const uint32_t taddr = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(half * (N / 2) + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
            "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]), "=r"(rr[7]),
              "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]),
              "=r"(rr[15]), "=r"(rr[16]), "=r"(rr[17]), "=r"(rr[18]), "=r"(rr[19]), "=r"(rr[20]), "=r"(rr[21]),
              "=r"(rr[22]), "=r"(rr[23]), "=r"(rr[24]), "=r"(rr[25]), "=r"(rr[26]), "=r"(rr[27]), "=r"(rr[28]),
              "=r"(rr[29]), "=r"(rr[30]), "=r"(rr[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float sum = 0.f;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            float w = __uint_as_float(rr[i]);
            sum = fmaf(w, w, sum);
        }
        red[(half * (N / 2) + c0) / 32][lq * 32 + lane] = sum;
        if (prm.W) {  // the rows themselves, for the covariances of this precision
            const int64_t row = row0 + lq * 32 + lane;
            const int64_t col0 = n0 + half * (N / 2) + c0;
            if (row < prm.count)
                for (int i = 0; i < 32; ++i)
                    if (col0 + i < prm.mp) prm.W[row * prm.mp + col0 + i] = __uint_as_float(rr[i]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid < TM && row0 + tid < prm.count) {
        const int64_t row = row0 + tid;
#pragma unroll
        for (int q = 0; q < N / 64; ++q) {
            const int64_t idx = row * prm.nN + n0 / 64 + q;
            if (idx < prm.plen) prm.partial[idx] = red[2 * q][tid] + red[2 * q + 1][tid];
            else atomicCAS(prm.status, 0, (int)GPR_ERR_ARG);  // self-check: never expected
        }
    }
    if (!ok_all) atomicCAS(prm.status, 0, (int)GPR_ERR_TIMEOUT);
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)N));
    }
}

// Warp-specialised variant with the same products, order and epilogue grouping (the same bits):
// warp 0 loads the B slices by TMA, warp 1 issues the MMAs, warps 2-9 generate the A tile of each
// stage (waiting only for that stage to be free) and finally drain the accumulator.
constexpr int WS_NTHR = 320;

template <int P, int N>
__global__ void __launch_bounds__(WS_NTHR, 1) k_tc_sumsq_ws(const __grid_constant__ CUtensorMap mapB0,
                                                           const __grid_constant__ CUtensorMap mapB1,
                                                           const __grid_constant__ CUtensorMap mapB2, TcParams prm)
{
    using C = Cfg<P>;
    constexpr int BKE = C::BKE;
    constexpr int A_TILE = TM * 128;
    constexpr int B_TILE = N * 128;
    constexpr int STAGE = C::NA * A_TILE + C::NB * B_TILE;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(smem + 2 * STAGE);  // fullB[2], fullA[2], empty[2], done
    __shared__ uint32_t tmem_slot;
    __shared__ int gx[TM], gy[TM], gz[TM];
    __shared__ bool rvalid[TM];
    __shared__ float red[N / 32][TM];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row0 = (int64_t)blockIdx.x * TM;
    const int n0 = blockIdx.y * N;
    const int64_t m = prm.m;
    const int64_t kend = (int64_t)n0 + N < m ? (int64_t)n0 + N : m;
    const int nkb = (int)((kend + BKE - 1) / BKE);
    const uint32_t fullB0 = smem_u32(&bars[0]), fullA0 = smem_u32(&bars[2]), empty0 = smem_u32(&bars[4]),
                   bar_done = smem_u32(&bars[6]);
    if (tid == 0) {
        mbar_init(fullB0, 1);
        mbar_init(fullB0 + 8, 1);
        mbar_init(fullA0, 256);
        mbar_init(fullA0 + 8, 256);
        mbar_init(empty0, 1);
        mbar_init(empty0 + 8, 1);
        mbar_init(bar_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"((uint32_t)N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int r = tid; r < TM; r += WS_NTHR) {
        int64_t row = row0 + r;
        bool ok = row < prm.count;
        int64_t p = ok ? (prm.pts ? prm.pts[row] : prm.pt_base + row) : 0;
        int64_t nx = prm.g.n[0], ny = prm.g.n[1];
        if (p < 0 || p >= nx * ny * (int64_t)prm.g.n[2]) { ok = false; p = 0; }
        gx[r] = (int)(p % nx);
        gy[r] = (int)((p / nx) % ny);
        gz[r] = (int)(p / (nx * ny));
        rvalid[r] = ok;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    bool ok_all = true;

    if (warp == 0 && lane == 0) {
        const CUtensorMap *maps[3] = {&mapB0, &mapB1, &mapB2};
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb & 1, use = kb >> 1;
            unsigned char *st = smem + s * STAGE;
            if (kb >= 2 && !mbar_wait(empty0 + 8 * s, (use - 1) & 1)) ok_all = false;
            mbar_expect_tx(fullB0 + 8 * s, (uint32_t)(C::NB * B_TILE));
            for (int b = 0; b < C::NB; ++b)
                tma_load_2d(smem_u32(st + C::NA * A_TILE + b * B_TILE), maps[b], kb * BKE, n0, fullB0 + 8 * s);
        }
    } else if (warp == 1 && lane == 0) {
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb & 1, use = kb >> 1;
            unsigned char *st = smem + s * STAGE;
            if (!mbar_wait(fullB0 + 8 * s, use & 1)) ok_all = false;
            if (!mbar_wait(fullA0 + 8 * s, use & 1)) ok_all = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            issue_block128<P, N>(tmem, smem_u32(st), smem_u32(st + C::NA * A_TILE), kb == 0);
            mma_commit(empty0 + 8 * s);
            if (kb == nkb - 1) mma_commit(bar_done);
        }
    } else if (warp >= 2) {
        const int at = tid - 64;  // 0 .. 255
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb & 1, use = kb >> 1;
            unsigned char *st = smem + s * STAGE;
            if (kb >= 2 && !mbar_wait(empty0 + 8 * s, (use - 1) & 1)) ok_all = false;
            for (int q = at; q < TM * 8; q += 256) gen_a_chunk<P>(prm, st, q >> 3, q & 7, kb, gx, gy, gz, rvalid);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(fullA0 + 8 * s) : "memory");
        }
        // epilogue: warp w reads TMEM lanes 32 (w % 4), column half (w - 2) / 4
        if (!mbar_wait(bar_done, 0)) ok_all = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int lq = warp & 3, half = (warp - 2) >> 2;
#pragma unroll
        for (int c0 = 0; c0 < N / 2; c0 += 32) {
            uint32_t rr[32];
            const uint32_t taddr = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(half * (N / 2) + c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
                "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]), "=r"(rr[7]),
                  "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]),
                  "=r"(rr[15]), "=r"(rr[16]), "=r"(rr[17]), "=r"(rr[18]), "=r"(rr[19]), "=r"(rr[20]), "=r"(rr[21]),
                  "=r"(rr[22]), "=r"(rr[23]), "=r"(rr[24]), "=r"(rr[25]), "=r"(rr[26]), "=r"(rr[27]), "=r"(rr[28]),
                  "=r"(rr[29]), "=r"(rr[30]), "=r"(rr[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float sum = 0.f;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                float w = __uint_as_float(rr[i]);
                sum = fmaf(w, w, sum);
            }
            red[(half * (N / 2) + c0) / 32][lq * 32 + lane] = sum;
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");  // the epilogue warps only
        if (at < TM && row0 + at < prm.count) {
            const int64_t row = row0 + at;
#pragma unroll
            for (int q = 0; q < N / 64; ++q) {
                const int64_t idx = row * prm.nN + n0 / 64 + q;
                if (idx < prm.plen) prm.partial[idx] = red[2 * q][at] + red[2 * q + 1][at];
                else atomicCAS(prm.status, 0, (int)GPR_ERR_ARG);  // self-check: never expected
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (!ok_all) atomicCAS(prm.status, 0, (int)GPR_ERR_TIMEOUT);
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)N));
    }
}

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

// One 16-byte chunk c (of 4) of row r of a 64-byte-row A tile (16 TF32 elements per K block),
// hi and lo slices, in the 64-byte-swizzled K-major layout (chunk c of row r at c ^ ((r >> 1) & 3)).
template <int P>
__device__ __forceinline__ void gen_a_chunk64(const TcParams &prm, unsigned char *st, int r, int c, int kb,
                                              const int *gx, const int *gy, const int *gz, const bool *rvalid)
{
    using C = Cfg<P>;
    constexpr int A_TILE = TM * 64;
    const int64_t m = prm.m;
    const int64_t k0 = (int64_t)kb * 16 + c * 4;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (rvalid[r] && k0 < m) {
        const float *tx = prm.T32 + (int64_t)gx[r] * prm.mp, *ty = prm.T32 + prm.off1 + (int64_t)gy[r] * prm.mp,
                    *tz = prm.T32 + prm.off2 + (int64_t)gz[r] * prm.mp;
        if (prm.off2 + (int64_t)gz[r] * prm.mp + k0 + 3 >= prm.tlen) {
            atomicCAS(prm.status, 0, (int)GPR_ERR_ARG);  // self-check: never expected
        } else {
            // table rows are mp (a multiple of 64) floats long and k0 a multiple of 4: 16-byte loads;
            // entries j >= m of a table row are masked below
            const float4 a = *(const float4 *)(tx + k0), b = *(const float4 *)(ty + k0), cc = *(const float4 *)(tz + k0);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w}, cv[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (k0 + e >= m) continue;
                if (prm.kind == GPR_K_SE) {
                    v[e] = av[e] * bv[e] * cv[e];
                } else {
                    const float r2 = av[e] + bv[e] + cv[e], rr = sqrtf(r2), s5r = 2.23606797749979f * rr;
                    v[e] = prm.sf2 * (1.0f + s5r + (5.0f / 3.0f) * r2) * __expf(-s5r);
                }
            }
        }
    }
    const int off = r * 64 + ((c ^ ((r >> 1) & 3)) << 4);
    float4 hi, lo;
    float *h = &hi.x, *l = &lo.x;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        h[e] = tf32_round(v[e]);
        l[e] = tf32_round(v[e] - h[e]);
    }
    *(float4 *)(st + off) = hi;
    if (C::NA > 1) *(float4 *)(st + A_TILE + off) = lo;
}

// TF32 / TF32x3 variant with 64-byte rows (16-element K blocks): two 48 KB stages, so two CTAs
// share an SM (2 x 256 TMEM columns) and one CTA's prologue, generation and drain overlap the
// other's MMAs.  Warp roles as in k_tc_sumsq_ws; the MMA order (per 16-element block: product by
// product over two K steps) and the epilogue grouping equal the other variants', so the bits do.
template <int P>
__global__ void __launch_bounds__(WS_NTHR, 2) k_tc_sumsq_2c(const __grid_constant__ CUtensorMap mapB0,
                                                           const __grid_constant__ CUtensorMap mapB1, TcParams prm)
{
    using C = Cfg<P>;
    static_assert(!C::BF, "64-byte rows: TF32 operands only");
    constexpr int N = 256;
    constexpr int A_TILE = TM * 64;
    constexpr int B_TILE = N * 64;
    constexpr int STAGE = C::NA * A_TILE + C::NB * B_TILE;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(smem + 2 * STAGE);  // fullB[2], fullA[2], empty[2], done
    __shared__ uint32_t tmem_slot;
    __shared__ int gx[TM], gy[TM], gz[TM];
    __shared__ bool rvalid[TM];
    __shared__ float red[N / 32][TM];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row0 = (int64_t)blockIdx.x * TM;
    const int n0 = blockIdx.y * N;
    const int64_t m = prm.m;
    const int64_t kend = (int64_t)n0 + N < m ? (int64_t)n0 + N : m;
    const int nkb = (int)((kend + 15) / 16);
    const uint32_t fullB0 = smem_u32(&bars[0]), fullA0 = smem_u32(&bars[2]), empty0 = smem_u32(&bars[4]),
                   bar_done = smem_u32(&bars[6]);
    if (tid == 0) {
        mbar_init(fullB0, 1);
        mbar_init(fullB0 + 8, 1);
        mbar_init(fullA0, 256);
        mbar_init(fullA0 + 8, 256);
        mbar_init(empty0, 1);
        mbar_init(empty0 + 8, 1);
        mbar_init(bar_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"((uint32_t)N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int r = tid; r < TM; r += WS_NTHR) {
        int64_t row = row0 + r;
        bool ok = row < prm.count;
        int64_t p = ok ? (prm.pts ? prm.pts[row] : prm.pt_base + row) : 0;
        int64_t nx = prm.g.n[0], ny = prm.g.n[1];
        if (p < 0 || p >= nx * ny * (int64_t)prm.g.n[2]) { ok = false; p = 0; }
        gx[r] = (int)(p % nx);
        gy[r] = (int)((p / nx) % ny);
        gz[r] = (int)(p / (nx * ny));
        rvalid[r] = ok;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    bool ok_all = true;
    constexpr uint32_t ID = idesc<false>(TM, N);

    if (warp == 0 && lane == 0) {
        const CUtensorMap *maps[2] = {&mapB0, &mapB1};
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb & 1, use = kb >> 1;
            unsigned char *st = smem + s * STAGE;
            if (kb >= 2 && !mbar_wait(empty0 + 8 * s, (use - 1) & 1)) ok_all = false;
            mbar_expect_tx(fullB0 + 8 * s, (uint32_t)(C::NB * B_TILE));
            for (int b = 0; b < C::NB; ++b)
                tma_load_2d(smem_u32(st + C::NA * A_TILE + b * B_TILE), maps[b], kb * 16, n0, fullB0 + 8 * s);
        }
    } else if (warp == 1 && lane == 0) {
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb & 1, use = kb >> 1;
            unsigned char *st = smem + s * STAGE;
            if (!mbar_wait(fullB0 + 8 * s, use & 1)) ok_all = false;
            if (!mbar_wait(fullA0 + 8 * s, use & 1)) ok_all = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int t = 0; t < C::NPROD; ++t) {
                int ia, ib;
                prod_pair(P, t, ia, ib);
                const uint32_t abase = smem_u32(st + ia * A_TILE), bbase = smem_u32(st + C::NA * A_TILE + ib * B_TILE);
#pragma unroll
                for (int k2 = 0; k2 < 2; ++k2) {
                    uint32_t acc = (kb > 0 || t > 0 || k2 > 0) ? 1u : 0u;
                    mma<false>(tmem, desc_sw64(abase + k2 * 32), desc_sw64(bbase + k2 * 32), ID, acc);
                }
            }
            mma_commit(empty0 + 8 * s);
            if (kb == nkb - 1) mma_commit(bar_done);
        }
    } else if (warp >= 2) {
        const int at = tid - 64;  // 0 .. 255
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb & 1, use = kb >> 1;
            unsigned char *st = smem + s * STAGE;
            if (kb >= 2 && !mbar_wait(empty0 + 8 * s, (use - 1) & 1)) ok_all = false;
            for (int q = at; q < TM * 4; q += 256) gen_a_chunk64<P>(prm, st, q >> 2, q & 3, kb, gx, gy, gz, rvalid);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(fullA0 + 8 * s) : "memory");
        }
        // epilogue: warp w reads TMEM lanes 32 (w % 4), column half (w - 2) / 4
        if (!mbar_wait(bar_done, 0)) ok_all = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int lq = warp & 3, half = (warp - 2) >> 2;
#pragma unroll
        for (int c0 = 0; c0 < N / 2; c0 += 32) {
            uint32_t rr[32];
            const uint32_t taddr = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(half * (N / 2) + c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
                "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]), "=r"(rr[7]),
                  "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]),
                  "=r"(rr[15]), "=r"(rr[16]), "=r"(rr[17]), "=r"(rr[18]), "=r"(rr[19]), "=r"(rr[20]), "=r"(rr[21]),
                  "=r"(rr[22]), "=r"(rr[23]), "=r"(rr[24]), "=r"(rr[25]), "=r"(rr[26]), "=r"(rr[27]), "=r"(rr[28]),
                  "=r"(rr[29]), "=r"(rr[30]), "=r"(rr[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float sum = 0.f;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                float w = __uint_as_float(rr[i]);
                sum = fmaf(w, w, sum);
            }
            red[(half * (N / 2) + c0) / 32][lq * 32 + lane] = sum;
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");  // the epilogue warps only
        if (at < TM && row0 + at < prm.count) {
            const int64_t row = row0 + at;
#pragma unroll
            for (int q = 0; q < N / 64; ++q) {
                const int64_t idx = row * prm.nN + n0 / 64 + q;
                if (idx < prm.plen) prm.partial[idx] = red[2 * q][at] + red[2 * q + 1][at];
                else atomicCAS(prm.status, 0, (int)GPR_ERR_ARG);  // self-check: never expected
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (!ok_all) atomicCAS(prm.status, 0, (int)GPR_ERR_TIMEOUT);
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)N));
    }
}

// ---- Evaluations at arbitrary points (the octree bound's minimiser): TF32x3 whitened rows of
// the kernel vector and, with GRAD, of its three coordinate derivatives, reduced on the fly to
// |w|^2 and w . (L^-1 d_k k): var = sf2 - |w|^2, grad var_d = -2 w . (L^-1 d_k k).

struct TcEvalParams {
    const double *xyz;  // count x 3 evaluation points
    int64_t count;
    const float *X32;   // m x 3 observation sites, float-float: hi, then lo at + 3 mp
    int64_t m, mp;
    int kind;
    float sf2;
    float iell[3], il2[3];
    float *partial;     // (count x T) x nN partial sums, T = 4 with GRAD (|w|^2, w . dw_x, dw_y, dw_z), else 1
    float *mom;         // count x 8: mu and (GRAD) grad mu as float-float pairs (hi, lo), by the last column tile
    const float *alpha32;  // mp FP32 alpha (zero beyond m)
    int nN;
    int64_t plen;
    int *status;
};

// Chunk c (4 elements) of rows r0 and r0 + 64 (r0 < 64): with GRAD, rows 32t .. 32t + 31 hold row
// type t (0: k(x, X_j), 1..3: d k / d x_{t-1}) of the CTA's 32 points, so both rows belong to point
// r0 mod 32 (types t0 and t0 + 2) and share one kernel evaluation; without, they are points r0 and
// r0 + 64.  The sites X_j of the chunk come in three 16-byte loads.
// (h, l) += t with Knuth's error-free two-sum (the rounding error goes to l).
__device__ __forceinline__ void acc2(float &h, float &l, float t)
{
    const float s = h + t, bv = s - h;
    l += (h - (s - bv)) + (t - bv);
    h = s;
}

// The generating thread also sums, for the last column tile (whose K range is every site), the
// mean k . alpha and with GRAD its gradient sum_j dk_j alpha_j of its point(s) over its chunks,
// error-free (alpha reaches ~1e3 for plain and ~1e5 for sparse models): acc[h] = (mu hi, lo, then
// grad hi, lo per axis) of point r0 + 64 h (GRAD: of point r0 mod 32, rows r0 < 32 only).
template <bool GRAD>
__device__ __forceinline__ void gen_eval_chunk64(const TcEvalParams &prm, unsigned char *st, int r0, int c, int kb,
                                                 const float (*pc)[GRAD ? 32 : TM], const bool *rvalid, bool accum,
                                                 float (&acc)[2][8])
{
    constexpr int A_TILE = TM * 64;
    const int64_t k0 = (int64_t)kb * 16 + c * 4;
    float xs[12], xsl[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) xs[i] = xsl[i] = 0.f;
    if (k0 < prm.m) {  // X32 holds 2 x 3 mp floats (zero beyond m) and k0 + 3 < mp
        const float4 *xp = (const float4 *)(prm.X32 + 3 * k0), *xq = (const float4 *)(prm.X32 + 3 * prm.mp + 3 * k0);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float4 a = xp[i], b = xq[i];
            xs[4 * i] = a.x; xs[4 * i + 1] = a.y; xs[4 * i + 2] = a.z; xs[4 * i + 3] = a.w;
            xsl[4 * i] = b.x; xsl[4 * i + 1] = b.y; xsl[4 * i + 2] = b.z; xsl[4 * i + 3] = b.w;
        }
    }
    float al[4] = {0.f, 0.f, 0.f, 0.f};
    if (accum && k0 < prm.m) {
        const float4 a4 = *(const float4 *)(prm.alpha32 + k0);
        al[0] = a4.x; al[1] = a4.y; al[2] = a4.z; al[3] = a4.w;
    }
    const bool acc_here = accum && (!GRAD || r0 < 32);
    float v[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int h = 0; h < (GRAD ? 1 : 2); ++h) {
        const int pr = GRAD ? (r0 & 31) : r0 + 64 * h;
        if (!rvalid[pr] || k0 >= prm.m) continue;
        const float x = pc[0][pr], y = pc[1][pr], z = pc[2][pr], xl = pc[3][pr], yl = pc[4][pr], zl = pc[5][pr];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (k0 + e >= prm.m) continue;
            // float-float differences: near points keep their digits
            const float d0 = (x - xs[3 * e]) + (xl - xsl[3 * e]), d1 = (y - xs[3 * e + 1]) + (yl - xsl[3 * e + 1]),
                        d2 = (z - xs[3 * e + 2]) + (zl - xsl[3 * e + 2]);
            const float a = d0 * prm.iell[0], b = d1 * prm.iell[1], cc = d2 * prm.iell[2];
            const float r2 = a * a + b * b + cc * cc;
            float k, cf;
            if (prm.kind == GPR_K_SE) {
                k = prm.sf2 * __expf(-0.5f * r2);
                cf = -k;
            } else {
                const float rr = sqrtf(r2), s5r = 2.23606797749979f * rr, ex = __expf(-s5r);
                k = prm.sf2 * (1.0f + s5r + (5.0f / 3.0f) * r2) * ex;
                cf = -(5.0f / 3.0f) * prm.sf2 * (1.0f + s5r) * ex;
            }
            const float g0 = cf * d0 * prm.il2[0], g1 = cf * d1 * prm.il2[1], g2 = cf * d2 * prm.il2[2];
            if (GRAD) {
                // row r0: type r0 / 32 (0: k, 1: d/dx); row r0 + 64: type 2 or 3 (d/dy, d/dz)
                v[0][e] = (r0 >> 5) == 0 ? k : g0;
                v[1][e] = (r0 >> 5) == 0 ? g1 : g2;
            } else {
                v[h][e] = k;
            }
            if (acc_here) {
                acc2(acc[h][0], acc[h][1], k * al[e]);
                if (GRAD) {
                    acc2(acc[h][2], acc[h][3], g0 * al[e]);
                    acc2(acc[h][4], acc[h][5], g1 * al[e]);
                    acc2(acc[h][6], acc[h][7], g2 * al[e]);
                }
            }
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int r = r0 + 64 * h;
        const int off = r * 64 + ((c ^ ((r >> 1) & 3)) << 4);
        float4 hi, lo;
        float *hh = &hi.x, *l = &lo.x;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            hh[e] = tf32_round(v[h][e]);
            l[e] = tf32_round(v[h][e] - hh[e]);
        }
        *(float4 *)(st + off) = hi;
        *(float4 *)(st + A_TILE + off) = lo;
    }
}

// The pipeline of k_tc_sumsq_2c (TMA warp, MMA warp, 8 generating and draining warps; two CTAs
// per SM) on the evaluation rows.  GRAD: the drain pairs each derivative row with its point's
// kernel row through shared memory, chunk by chunk.
template <bool GRAD>
__global__ void __launch_bounds__(WS_NTHR, 2) k_tc_eval(const __grid_constant__ CUtensorMap mapB0,
                                                       const __grid_constant__ CUtensorMap mapB1, TcEvalParams prm)
{
    constexpr int P = GPR_P_TF32X3;
    using C = Cfg<P>;
    constexpr int N = 256;
    constexpr int A_TILE = TM * 64;
    constexpr int B_TILE = N * 64;
    constexpr int STAGE = C::NA * A_TILE + C::NB * B_TILE;
    constexpr int PTS = GRAD ? 32 : TM;  // points per CTA
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(smem + 2 * STAGE);  // fullB[2], fullA[2], empty[2], done
    __shared__ uint32_t tmem_slot;
    __shared__ float pc[6][PTS];  // point coordinates x, y, z (hi), then their lo parts
    __shared__ bool rvalid[PTS];
    __shared__ float red[N / 32][TM];
    __shared__ float wbuf[GRAD ? 2 : 1][32][32];  // [column half][column][point]: kernel-row chunk

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t pt0 = (int64_t)blockIdx.x * PTS;
    const int n0 = blockIdx.y * N;
    const int64_t m = prm.m;
    const int64_t kend = (int64_t)n0 + N < m ? (int64_t)n0 + N : m;
    const int nkb = (int)((kend + 15) / 16);
    const uint32_t fullB0 = smem_u32(&bars[0]), fullA0 = smem_u32(&bars[2]), empty0 = smem_u32(&bars[4]),
                   bar_done = smem_u32(&bars[6]);
    if (tid == 0) {
        mbar_init(fullB0, 1);
        mbar_init(fullB0 + 8, 1);
        mbar_init(fullA0, 256);
        mbar_init(fullA0 + 8, 256);
        mbar_init(empty0, 1);
        mbar_init(empty0 + 8, 1);
        mbar_init(bar_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"((uint32_t)N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int r = tid; r < PTS; r += WS_NTHR) {
        const int64_t q = pt0 + r;
        const bool ok = q < prm.count;
        rvalid[r] = ok;
        for (int d = 0; d < 3; ++d) {
            const double v = ok ? prm.xyz[3 * q + d] : 0.0;
            const float h = (float)v;
            pc[d][r] = h;
            pc[3 + d][r] = (float)(v - (double)h);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    bool ok_all = true;
    constexpr uint32_t ID = idesc<false>(TM, N);

    if (warp == 0 && lane == 0) {
        const CUtensorMap *maps[2] = {&mapB0, &mapB1};
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb & 1, use = kb >> 1;
            unsigned char *st = smem + s * STAGE;
            if (kb >= 2 && !mbar_wait(empty0 + 8 * s, (use - 1) & 1)) ok_all = false;
            mbar_expect_tx(fullB0 + 8 * s, (uint32_t)(C::NB * B_TILE));
            for (int b = 0; b < C::NB; ++b)
                tma_load_2d(smem_u32(st + C::NA * A_TILE + b * B_TILE), maps[b], kb * 16, n0, fullB0 + 8 * s);
        }
    } else if (warp == 1 && lane == 0) {
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb & 1, use = kb >> 1;
            unsigned char *st = smem + s * STAGE;
            if (!mbar_wait(fullB0 + 8 * s, use & 1)) ok_all = false;
            if (!mbar_wait(fullA0 + 8 * s, use & 1)) ok_all = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int t = 0; t < C::NPROD; ++t) {
                int ia, ib;
                prod_pair(P, t, ia, ib);
                const uint32_t abase = smem_u32(st + ia * A_TILE), bbase = smem_u32(st + C::NA * A_TILE + ib * B_TILE);
#pragma unroll
                for (int k2 = 0; k2 < 2; ++k2) {
                    uint32_t acc = (kb > 0 || t > 0 || k2 > 0) ? 1u : 0u;
                    mma<false>(tmem, desc_sw64(abase + k2 * 32), desc_sw64(bbase + k2 * 32), ID, acc);
                }
            }
            mma_commit(empty0 + 8 * s);
            if (kb == nkb - 1) mma_commit(bar_done);
        }
    } else if (warp >= 2) {
        const int at = tid - 64;  // 0 .. 255
        const bool accum = blockIdx.y == gridDim.y - 1;  // the last column tile sees every site
        float acc[2][8];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[h][i] = 0.f;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb & 1, use = kb >> 1;
            unsigned char *st = smem + s * STAGE;
            if (kb >= 2 && !mbar_wait(empty0 + 8 * s, (use - 1) & 1)) ok_all = false;
            gen_eval_chunk64<GRAD>(prm, st, at >> 2, at & 3, kb, pc, rvalid, accum, acc);  // rows at/4 and at/4 + 64
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(fullA0 + 8 * s) : "memory");
        }
        if (accum) {
            // the four chunk threads of a point are lanes 4q .. 4q + 3: combine them error-free
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int i = 0; i < 8; i += 2)
#pragma unroll
                    for (int o = 1; o <= 2; o <<= 1) {
                        const float h2 = __shfl_xor_sync(0xffffffffu, acc[h][i], o);
                        const float l2 = __shfl_xor_sync(0xffffffffu, acc[h][i + 1], o);
                        acc2(acc[h][i], acc[h][i + 1], h2);
                        acc[h][i + 1] += l2;
                    }
            const int r0 = at >> 2;
            if ((at & 3) == 0 && (!GRAD || r0 < 32)) {
#pragma unroll
                for (int h = 0; h < (GRAD ? 1 : 2); ++h) {
                    const int pr = GRAD ? r0 : r0 + 64 * h;
                    const int64_t q = pt0 + pr;
                    if (q < prm.count) {
                        float *mo = prm.mom + 8 * q;
#pragma unroll
                        for (int i = 0; i < 8; ++i) mo[i] = acc[h][i];
                    }
                }
            }
        }
        if (!mbar_wait(bar_done, 0)) ok_all = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int lq = warp & 3, half = (warp - 2) >> 2;
#pragma unroll
        for (int c0 = 0; c0 < N / 2; c0 += 32) {
            uint32_t rr[32];
            const uint32_t taddr = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(half * (N / 2) + c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
                "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]), "=r"(rr[7]),
                  "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]),
                  "=r"(rr[15]), "=r"(rr[16]), "=r"(rr[17]), "=r"(rr[18]), "=r"(rr[19]), "=r"(rr[20]), "=r"(rr[21]),
                  "=r"(rr[22]), "=r"(rr[23]), "=r"(rr[24]), "=r"(rr[25]), "=r"(rr[26]), "=r"(rr[27]), "=r"(rr[28]),
                  "=r"(rr[29]), "=r"(rr[30]), "=r"(rr[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float sum = 0.f;
            if (!GRAD || lq == 0) {
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float w = __uint_as_float(rr[i]);
                    sum = fmaf(w, w, sum);
                }
            }
            if (GRAD) {
                if (lq == 0)
#pragma unroll
                    for (int i = 0; i < 32; ++i) wbuf[GRAD ? half : 0][i][lane] = __uint_as_float(rr[i]);
                asm volatile("bar.sync 1, 256;" ::: "memory");
                if (lq != 0)
#pragma unroll
                    for (int i = 0; i < 32; ++i) sum = fmaf(__uint_as_float(rr[i]), wbuf[GRAD ? half : 0][i][lane], sum);
                asm volatile("bar.sync 1, 256;" ::: "memory");
            }
            red[(half * (N / 2) + c0) / 32][lq * 32 + lane] = sum;
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");  // the epilogue warps only
        if (at < TM) {
            const int type = GRAD ? at >> 5 : 0, pr = GRAD ? (at & 31) : at;
            const int64_t q = pt0 + pr;
            if (q < prm.count) {
#pragma unroll
                for (int g2 = 0; g2 < N / 64; ++g2) {
                    const int64_t idx = (q * (GRAD ? 4 : 1) + type) * prm.nN + n0 / 64 + g2;
                    if (idx < prm.plen) prm.partial[idx] = red[2 * g2][at] + red[2 * g2 + 1][at];
                    else atomicCAS(prm.status, 0, (int)GPR_ERR_ARG);  // self-check: never expected
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (!ok_all) atomicCAS(prm.status, 0, (int)GPR_ERR_TIMEOUT);
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)N));
    }
}

__global__ void k_tc_finalize(const float *partial, int nN, int64_t count, double sf2, float *var)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count || nN > 64) return;
    float s = 0.f;
    for (int t = 0; t < nN; ++t) s += partial[i * nN + t];
    var[i] = (float)(sf2 - (double)s);
}

// B slices of L^-1 (rows j, columns i <= j), K-major: TF32 hi/lo (FP32 storage) or BF16 x3.
__global__ void k_split_b(const double *Linv, int64_t mb, int64_t m, int64_t mpt, float *thi, float *tlo,
                          __nv_bfloat16 *b0, __nv_bfloat16 *b1, __nv_bfloat16 *b2)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= mpt * mpt) return;
    int64_t j = idx / mpt, i = idx % mpt;
    double v = (j < m && i <= j) ? Linv[j * mb + i] : 0.0;
    float f = (float)v;
    float h = tf32_round(f);
    thi[idx] = h;
    tlo[idx] = tf32_round((float)(v - (double)h));
    __nv_bfloat16 x0 = __double2bfloat16(v);
    double r1 = v - (double)__bfloat162float(x0);
    __nv_bfloat16 x1 = __double2bfloat16(r1);
    double r2 = r1 - (double)__bfloat162float(x1);
    b0[idx] = x0;
    b1[idx] = x1;
    b2[idx] = __double2bfloat16(r2);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode()
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

bool make_map(CUtensorMap *map, void *base, int64_t mpt, bool bf, int N)
{
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)mpt, (cuuint64_t)mpt};
    cuuint64_t gstride[1] = {(cuuint64_t)mpt * (bf ? 2 : 4)};
    cuuint32_t box[2] = {(cuuint32_t)(bf ? 64 : 32), (cuuint32_t)N};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, gdim, gstride,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool make_map64(CUtensorMap *map, void *base, int64_t mpt)
{
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)mpt, (cuuint64_t)mpt};
    cuuint64_t gstride[1] = {(cuuint64_t)mpt * 4};
    cuuint32_t box[2] = {16, 256};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int P>
gpr_status launch_tc2c(const gpr_model *M, const TcParams &prm, cudaStream_t st)
{
    using C = Cfg<P>;
    CUtensorMap maps[2];
    const TcOperands &B = *M->tc;
    if (!make_map64(&maps[0], B.thi, B.mpt) || !make_map64(&maps[1], B.tlo, B.mpt)) return GPR_ERR_UNSUPPORTED;
    const size_t smem = 2 * ((size_t)C::NA * TM * 64 + (size_t)C::NB * 256 * 64) + 64 + 1024;
    dim3 grid((unsigned)((prm.count + TM - 1) / TM), (unsigned)(B.mpt / 256));
    GPR_CUDA_TRY(cudaFuncSetAttribute(k_tc_sumsq_2c<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps("tc_sumsq", st, (double)prm.count);
    k_tc_sumsq_2c<P><<<grid, WS_NTHR, smem, st>>>(maps[0], maps[1], prm);
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

template <int P, int N>
size_t smem_bytes()
{
    using C = Cfg<P>;
    size_t stage = (size_t)C::NA * TM * 128 + (size_t)C::NB * N * 128;
    return 2 * stage + 64 + 1024;
}

template <int P, int N, bool WS>
gpr_status launch_tc(const gpr_model *M, const TcParams &prm, cudaStream_t st)
{
    using C = Cfg<P>;
    CUtensorMap maps[3];
    const TcOperands &B = *M->tc;
    if (C::BF) {
        void *bases[3] = {B.b0, B.b1, B.b2};
        for (int i = 0; i < 3; ++i)
            if (!make_map(&maps[i], bases[i], B.mpt, true, N)) return GPR_ERR_UNSUPPORTED;
    } else {
        void *bases[3] = {B.thi, B.tlo, B.thi};
        for (int i = 0; i < 3; ++i)
            if (!make_map(&maps[i], bases[i], B.mpt, false, N)) return GPR_ERR_UNSUPPORTED;
    }
    size_t smem = smem_bytes<P, N>();
    dim3 grid((unsigned)((prm.count + TM - 1) / TM), (unsigned)(B.mpt / N));
    if (WS) {
        GPR_CUDA_TRY(cudaFuncSetAttribute(k_tc_sumsq_ws<P, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ProfScope ps("tc_sumsq", st, (double)prm.count);
        k_tc_sumsq_ws<P, N><<<grid, WS_NTHR, smem, st>>>(maps[0], maps[1], maps[2], prm);
    } else {
        GPR_CUDA_TRY(cudaFuncSetAttribute(k_tc_sumsq<P, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ProfScope ps("tc_sumsq", st, (double)prm.count);
        k_tc_sumsq<P, N><<<grid, NTHR, smem, st>>>(maps[0], maps[1], maps[2], prm);
    }
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

}  // namespace

bool tc_precision(gpr_precision p)
{
    return p == GPR_P_TF32 || p == GPR_P_TF32X3 || p == GPR_P_BF16 || p == GPR_P_BF16X3;
}

gpr_status fast_meanvar(gpr_model *M, const GridDev &g, gpr_precision prec, const float *T32, const float2 *Tff,
                        const double *T64, const int64_t *pts, int64_t pt_base, int64_t count, float *mean, float *var,
                        float *partial, cudaStream_t st)
{
    if (count <= 0) return GPR_OK;
    if (tc_precision(prec)) {
        GPR_TRY(tc_prepare(M, st));
        GPR_TRY(launch_tc_var(M, g, prec, T32, pts, pt_base, count, partial, var, st));
    } else {
        launch_meanvar32(M, g, T32, pts, pt_base, count, mean, var, st);
    }
    launch_mean_compensated(M, g, Tff, T64, pts, pt_base, count, mean, st);
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

static gpr_status tc_prepare_locked(gpr_model *M, cudaStream_t st);

// Lazily built per model; under the model's lock, and finished on the stream before another
// thread may use it (fields of one model can run concurrently in the batched path).
gpr_status tc_prepare(gpr_model *M, cudaStream_t st)
{
    std::lock_guard<std::mutex> lock(M->init_mu);
    if (M->tc) return GPR_OK;
    GPR_TRY(tc_prepare_locked(M, st));
    GPR_CUDA_TRY(cudaStreamSynchronize(st));
    return GPR_OK;
}

static gpr_status tc_prepare_locked(gpr_model *M, cudaStream_t st)
{
    if (M->tc) return GPR_OK;
    int64_t mb = (M->m + 31) / 32 * 32;
    TcOperands *B = new TcOperands();
    B->mpt = (M->mp + 255) / 256 * 256;
    int64_t mpt = B->mpt;
    size_t n = (size_t)mpt * mpt;
    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&B->thi, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&B->tlo, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&B->b0, n * 2);
    if (e == cudaSuccess) e = cudaMalloc(&B->b1, n * 2);
    if (e == cudaSuccess) e = cudaMalloc(&B->b2, n * 2);
    if (e != cudaSuccess) {
        cudaFree(B->thi); cudaFree(B->tlo); cudaFree(B->b0); cudaFree(B->b1); cudaFree(B->b2);
        delete B;
        return e == cudaErrorMemoryAllocation ? GPR_ERR_OOM : GPR_ERR_CUDA;
    }
    k_split_b<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M->Linv, mb, M->m, mpt, B->thi, B->tlo,
                                                          (__nv_bfloat16 *)B->b0, (__nv_bfloat16 *)B->b1,
                                                          (__nv_bfloat16 *)B->b2);
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    M->tc = B;
    return GPR_OK;
}

void tc_release(gpr_model *M)
{
    if (!M->tc) return;
    cudaFree(M->tc->thi); cudaFree(M->tc->tlo); cudaFree(M->tc->b0); cudaFree(M->tc->b1); cudaFree(M->tc->b2);
    delete M->tc;
    M->tc = nullptr;
}

size_t tc_partial_elems(gpr_precision p, const gpr_model *M, int64_t count)
{
    (void)p;
    int64_t mpt = (M->mp + 255) / 256 * 256;
    return (size_t)count * (size_t)(mpt / 64);
}

// var of the listed points by the tensor-core contraction; `partial` holds tc_partial_elems floats.
size_t tc_eval_partial_elems(const gpr_model *M, int64_t count)
{
    const int64_t mpt = (M->mp + 255) / 256 * 256;
    return (size_t)count * (4 * (size_t)(mpt / 64) + 8);
}

gpr_status launch_tc_eval(gpr_model *M, const double *xyz, int64_t count, bool grad, float *partial,
                          size_t partial_elems, cudaStream_t st)
{
    if (count <= 0) return GPR_OK;
    GPR_TRY(tc_prepare(M, st));
    const TcOperands &B = *M->tc;
    CUtensorMap maps[2];
    if (!make_map64(&maps[0], B.thi, B.mpt) || !make_map64(&maps[1], B.tlo, B.mpt)) return GPR_ERR_UNSUPPORTED;
    TcEvalParams prm;
    prm.xyz = xyz;
    prm.count = count;
    prm.X32 = M->X32;
    prm.m = M->m;
    prm.mp = M->mp;
    prm.kind = M->kp.kind;
    prm.sf2 = (float)M->kp.sf2;
    for (int d = 0; d < 3; ++d) {
        prm.iell[d] = (float)(1.0 / M->kp.ell[d]);
        prm.il2[d] = (float)(1.0 / (M->kp.ell[d] * M->kp.ell[d]));
    }
    prm.partial = partial;
    prm.nN = (int)(B.mpt / 64);
    prm.plen = (int64_t)count * 4 * prm.nN;  // the moments follow the partial sums
    prm.mom = partial + prm.plen;
    prm.alpha32 = M->alpha32;
    if ((size_t)count * (4 * (size_t)prm.nN + 8) > partial_elems) return GPR_ERR_ARG;
    prm.status = gpr_status_word();
    if (!prm.status) return GPR_ERR_CUDA;
    using C = Cfg<GPR_P_TF32X3>;
    const size_t smem = 2 * ((size_t)C::NA * TM * 64 + (size_t)C::NB * 256 * 64) + 64 + 1024;
    const int pts = grad ? 32 : TM;
    dim3 grid((unsigned)((count + pts - 1) / pts), (unsigned)(B.mpt / 256));
    if (grad) {
        GPR_CUDA_TRY(cudaFuncSetAttribute(k_tc_eval<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_tc_eval<true><<<grid, WS_NTHR, smem, st>>>(maps[0], maps[1], prm);
    } else {
        GPR_CUDA_TRY(cudaFuncSetAttribute(k_tc_eval<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_tc_eval<false><<<grid, WS_NTHR, smem, st>>>(maps[0], maps[1], prm);
    }
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

gpr_status launch_tc_var(const gpr_model *M, const GridDev &g, gpr_precision prec, const float *T32,
                         const int64_t *pts, int64_t pt_base, int64_t count, float *partial, float *var, cudaStream_t st,
                         float *W)
{
    if (count <= 0) return GPR_OK;
    if (!M->tc) return GPR_ERR_ARG;
    TcParams prm;
    prm.T32 = T32;
    prm.off1 = (int64_t)g.n[0] * M->mp;
    prm.off2 = prm.off1 + (int64_t)g.n[1] * M->mp;
    prm.mp = M->mp;
    prm.m = M->m;
    prm.kind = M->kp.kind;
    prm.sf2 = (float)M->kp.sf2;
    prm.g = g;
    prm.pts = pts;
    prm.pt_base = pt_base;
    prm.count = count;
    prm.partial = partial;
    prm.W = W;
    prm.nN = (int)(M->tc->mpt / 64);
    prm.plen = count * prm.nN;
    prm.tlen = prm.off2 + (int64_t)g.n[2] * M->mp;
    prm.status = gpr_status_word();
    if (!prm.status) return GPR_ERR_CUDA;
    // tile width: the autotuner's choice for this precision and model size (results are the same)
    // alternatives (same bits): tile width N and the plain or warp-specialised kernel
    auto run = [&](int c) -> gpr_status {
        const bool wide = c & 1, ws = c >> 1;
        if (c == 4) return prec == GPR_P_TF32 ? launch_tc2c<GPR_P_TF32>(M, prm, st) : launch_tc2c<GPR_P_TF32X3>(M, prm, st);
        switch (prec) {
        case GPR_P_TF32:
            return ws ? (wide ? launch_tc<GPR_P_TF32, 256, true>(M, prm, st) : launch_tc<GPR_P_TF32, 128, true>(M, prm, st))
                      : (wide ? launch_tc<GPR_P_TF32, 256, false>(M, prm, st)
                              : launch_tc<GPR_P_TF32, 128, false>(M, prm, st));
        case GPR_P_TF32X3:
            return ws ? (wide ? launch_tc<GPR_P_TF32X3, 256, true>(M, prm, st)
                              : launch_tc<GPR_P_TF32X3, 128, true>(M, prm, st))
                      : (wide ? launch_tc<GPR_P_TF32X3, 256, false>(M, prm, st)
                              : launch_tc<GPR_P_TF32X3, 128, false>(M, prm, st));
        case GPR_P_BF16:
            return ws ? (wide ? launch_tc<GPR_P_BF16, 256, true>(M, prm, st) : launch_tc<GPR_P_BF16, 128, true>(M, prm, st))
                      : (wide ? launch_tc<GPR_P_BF16, 256, false>(M, prm, st)
                              : launch_tc<GPR_P_BF16, 128, false>(M, prm, st));
        case GPR_P_BF16X3:
            return ws ? (wide ? launch_tc<GPR_P_BF16X3, 128, true>(M, prm, st)
                              : launch_tc<GPR_P_BF16X3, 64, true>(M, prm, st))
                      : (wide ? launch_tc<GPR_P_BF16X3, 128, false>(M, prm, st)
                              : launch_tc<GPR_P_BF16X3, 64, false>(M, prm, st));
        default: return GPR_ERR_ARG;
        }
    };
    static const char *names[] = {"tc_sumsq_fp64", "tc_sumsq_fp32", "tc_sumsq_tf32", "tc_sumsq_tf32x3",
                                  "tc_sumsq_bf16", "tc_sumsq_bf16x3"};
    // key: model size and the order of magnitude of the point count
    int lg = 0;
    while (((int64_t)1 << lg) < count && lg < 62) ++lg;
    if (W) GPR_TRY(run(1));  // rows out: the plain kernel (only it writes them), wide tiles
    else  // TF32 operands also have the two-CTAs-per-SM variant
        GPR_TRY(tune_run(names[(int)prec], (tune_bucket(M->mp) << 6) | lg,
                         prec == GPR_P_TF32 || prec == GPR_P_TF32X3 ? 5 : 4, run, st));
    k_tc_finalize<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(partial, prm.nN, count, M->kp.sf2, var);
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}
