// Posterior statistics at grid points in the whitened form (Eq. 1 for plain GPR):
// w_p = L^-1 k_p (row p of W = K_* L^-T, kernel rows generated on the fly from
// separable per-axis tables, never stored), mu_p = w_p . L^-1 y,
// var_p = k(p,p) - |w_p|^2, cov(p,q) = k(p,q) - w_p . w_q.
#include <math.h>

#include "internal.h"

GridDev make_grid(const gpr_grid *g)
{
    GridDev d;
    for (int k = 0; k < 3; ++k) {
        d.lo[k] = g->lo[k];
        d.h[k] = (g->hi[k] - g->lo[k]) / (double)(g->n[k] - 1);
        d.n[k] = g->n[k];
    }
    return d;
}

bool grid_valid(const gpr_grid *g)
{
    if (!g) return false;
    for (int k = 0; k < 3; ++k) {
        if (g->n[k] < 2 || g->n[k] > (1 << 20)) return false;
        if (!(g->hi[k] > g->lo[k]) || !isfinite(g->lo[k]) || !isfinite(g->hi[k])) return false;
    }
    return (int64_t)g->n[0] * g->n[1] * g->n[2] <= (int64_t)1 << 31;
}

size_t table_elems(const gpr_model *M, const GridDev &g) { return (size_t)(g.n[0] + g.n[1] + g.n[2]) * M->mp; }

// SE: T_d[g][j] = exp(-(x_g - X_jd)^2 / (2 l_d^2)), sf2 folded into axis 0.
// Matern-5/2: T_d[g][j] = ((x_g - X_jd)/l_d)^2.  Columns j >= m are 0.
// Optional float-float copy (hi, lo) of the FP64 table for the compensated mean.
__global__ void k_tables(const double *X, int64_t m, int64_t mp, KernParams kp, GridDev g, double *T64, float *T32,
                         float2 *Tff)
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
        if (kp.kind == GPR_K_SE) {
            v = exp(-0.5 * t * t);
            if (d == 0) v *= kp.sf2;
        } else {
            v = t * t;
        }
    }
    if (T64) T64[idx] = v;
    if (T32) T32[idx] = (float)v;
    if (Tff) {
        float hi = (float)v;
        Tff[idx] = make_float2(hi, (float)(v - (double)hi));
    }
}

gpr_status build_tables(const gpr_model *M, const GridDev &g, double *T64, float *T32, cudaStream_t st,
                        float2 *Tff)
{
    int64_t total = (int64_t)table_elems(M, g);
    k_tables<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(M->X, M->m, M->mp, M->kp, g, T64, T32, Tff);
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

template <typename T>
struct KFun;

template <>
struct KFun<double> {
    static __device__ __forceinline__ double se(double a, double b, double c) { return a * b * c; }
    static __device__ __forceinline__ double matern(double r2, double sf2)
    {
        double r = sqrt(r2), s5r = 2.2360679774997896964 * r;
        return sf2 * (1.0 + s5r + (5.0 / 3.0) * r2) * exp(-s5r);
    }
};
template <>
struct KFun<float> {
    static __device__ __forceinline__ float se(float a, float b, float c) { return a * b * c; }
    static __device__ __forceinline__ float matern(float r2, double sf2)
    {
        float r = sqrtf(r2), s5r = 2.23606797749979f * r;
        return (float)sf2 * (1.0f + s5r + (5.0f / 3.0f) * r2) * __expf(-s5r);
    }
};

// Kernel value k(x_p, X_j) from the tables for grid coordinates (gx, gy, gz).
template <typename T>
__device__ __forceinline__ T kval(const T *Tab, int64_t off1, int64_t off2, int64_t mp, int kind, double sf2,
                                  int gx, int gy, int gz, int64_t j)
{
    T a = Tab[(int64_t)gx * mp + j], b = Tab[off1 + (int64_t)gy * mp + j], c = Tab[off2 + (int64_t)gz * mp + j];
    if (kind == GPR_K_SE) return KFun<T>::se(a, b, c);
    return KFun<T>::matern(a + b + c, sf2);
}

static constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// One 64x64 tile of W = K_* BT for rows [row0, row0+64) and columns [j0, j0+64);
// the K range stops at min(j0 + 64, m) because BT is upper triangular.
template <typename T>
__device__ __forceinline__ void w_tile(const T *Tab, int64_t off1, int64_t off2, int64_t mp, int64_t m, int kind,
                                       double sf2, const T *BT, const int *cx, const int *cy, const int *cz,
                                       const bool *valid, int64_t j0, T (*As)[BM + 4], T (*Bs)[BN + 4],
                                       T acc[4][4])
{
    int t = threadIdx.x, tx = t % 16, ty = t / 16;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = T(0);
    int64_t kend = j0 + BN < m ? j0 + BN : m;
    for (int64_t k0 = 0; k0 < kend; k0 += BK) {
#pragma unroll
        for (int e = 0; e < (BM * BK) / NT; ++e) {
            int idx = t + NT * e, r = idx % BM, kk = idx / BM;
            int64_t j = k0 + kk;
            T v = T(0);
            if (j < m && valid[r]) v = kval<T>(Tab, off1, off2, mp, kind, sf2, cx[r], cy[r], cz[r], j);
            As[kk][r] = v;
        }
#pragma unroll
        for (int e = 0; e < (BK * BN) / NT; ++e) {
            int idx = t + NT * e, kk = idx / BN, c = idx % BN;
            Bs[kk][c] = BT[(k0 + kk) * mp + j0 + c];
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx * 4 + c];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[i][c] = fma(a[i], b[c], acc[i][c]);
        }
        __syncthreads();
    }
}

template <typename T>
__device__ __forceinline__ void load_rows(const GridDev &g, const int64_t *pts, int64_t pt_base, int64_t count, int64_t row0, int *cx,
                                          int *cy, int *cz, bool *valid)
{
    for (int r = threadIdx.x; r < BM; r += blockDim.x) {
        int64_t row = row0 + r;
        bool ok = row < count;
        int64_t p = ok ? (pts ? pts[row] : pt_base + row) : 0;
        int64_t nx = g.n[0], ny = g.n[1];
        if (p < 0 || p >= nx * ny * (int64_t)g.n[2]) { ok = false; p = 0; }  // listed index off the grid
        cx[r] = (int)(p % nx);
        cy[r] = (int)((p / nx) % ny);
        cz[r] = (int)(p / (nx * ny));
        valid[r] = ok;
    }
}

// Stored W rows: grid (mp/64, ceil(count/64)).
template <typename T>
__global__ void __launch_bounds__(NT) k_w_store(const T *Tab, int64_t off1, int64_t off2, int64_t mp, int64_t m,
                                                 int kind, double sf2, const T *BT, GridDev g, const int64_t *pts,
                                                 int64_t pt_base, int64_t count, T *W)
{
    __shared__ T As[BK][BM + 4];
    __shared__ T Bs[BK][BN + 4];
    __shared__ int cx[BM], cy[BM], cz[BM];
    __shared__ bool valid[BM];
    int64_t row0 = (int64_t)blockIdx.y * BM, j0 = (int64_t)blockIdx.x * BN;
    load_rows<T>(g, pts, pt_base, count, row0, cx, cy, cz, valid);
    __syncthreads();
    T acc[4][4];
    w_tile<T>(Tab, off1, off2, mp, m, kind, sf2, BT, cx, cy, cz, valid, j0, As, Bs, acc);
    int t = threadIdx.x, tx = t % 16, ty = t / 16;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t row = row0 + ty * 4 + i;
        if (row >= count) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) W[row * mp + j0 + tx * 4 + c] = acc[i][c];
    }
}

// Fused mean/variance: each CTA owns 64 rows and sweeps every column tile.
template <typename T>
__global__ void __launch_bounds__(NT) k_w_meanvar(const T *Tab, int64_t off1, int64_t off2, int64_t mp, int64_t m,
                                                   int kind, double sf2, const T *BT, const T *vy, GridDev g,
                                                   const int64_t *pts, int64_t pt_base, int64_t count, float *mean,
                                                   float *var)
{
    __shared__ T As[BK][BM + 4];
    __shared__ T Bs[BK][BN + 4];
    __shared__ int cx[BM], cy[BM], cz[BM];
    __shared__ bool valid[BM];
    int64_t row0 = (int64_t)blockIdx.x * BM;
    load_rows<T>(g, pts, pt_base, count, row0, cx, cy, cz, valid);
    __syncthreads();
    int t = threadIdx.x, tx = t % 16, ty = t / 16;
    T sq[4] = {0, 0, 0, 0}, mv[4] = {0, 0, 0, 0};
    for (int64_t j0 = 0; j0 < m; j0 += BN) {
        T acc[4][4];
        w_tile<T>(Tab, off1, off2, mp, m, kind, sf2, BT, cx, cy, cz, valid, j0, As, Bs, acc);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                T w = acc[i][c];
                sq[i] = fma(w, w, sq[i]);
                mv[i] = fma(w, vy[j0 + tx * 4 + c], mv[i]);
            }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            sq[i] += __shfl_xor_sync(0xffffffffu, sq[i], o);
            mv[i] += __shfl_xor_sync(0xffffffffu, mv[i], o);
        }
    if (tx == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int64_t row = row0 + ty * 4 + i;
            if (row < count) {
                mean[row] = (float)mv[i];
                var[row] = (float)(sf2 - (double)sq[i]);
            }
        }
    }
}

static void table_offsets(const gpr_model *M, const GridDev &g, int64_t &o1, int64_t &o2)
{
    o1 = (int64_t)g.n[0] * M->mp;
    o2 = o1 + (int64_t)g.n[1] * M->mp;
}

void launch_w64(const gpr_model *M, const GridDev &g, const double *T64, const int64_t *pts, int64_t pt_base,
                int64_t count, double *W, cudaStream_t st)
{
    if (count <= 0) return;
    int64_t o1, o2;
    table_offsets(M, g, o1, o2);
    dim3 grid((unsigned)(M->mp / BN), (unsigned)((count + BM - 1) / BM));
    {
        ProfScope _ps("w64", st);
        k_w_store<double><<<grid, NT, 0, st>>>(T64, o1, o2, M->mp, M->m, M->kp.kind, M->kp.sf2, M->BT64, g, pts, pt_base, count, W);
    }
    note_launch();
}

void launch_w32(const gpr_model *M, const GridDev &g, const float *T32, const int64_t *pts, int64_t pt_base,
                int64_t count, float *W, cudaStream_t st)
{
    if (count <= 0) return;
    int64_t o1, o2;
    table_offsets(M, g, o1, o2);
    dim3 grid((unsigned)(M->mp / BN), (unsigned)((count + BM - 1) / BM));
    {
        ProfScope _ps("w32", st);
        k_w_store<float><<<grid, NT, 0, st>>>(T32, o1, o2, M->mp, M->m, M->kp.kind, M->kp.sf2, M->BT32, g, pts, pt_base, count, W);
    }
    note_launch();
}

void launch_meanvar32(const gpr_model *M, const GridDev &g, const float *T32, const int64_t *pts, int64_t pt_base,
                      int64_t count, float *mean, float *var, cudaStream_t st)
{
    if (count <= 0) return;
    int64_t o1, o2;
    table_offsets(M, g, o1, o2);
    {
        ProfScope _ps("meanvar32", st);
        k_w_meanvar<float><<<(unsigned)((count + BM - 1) / BM), NT, 0, st>>>(T32, o1, o2, M->mp, M->m, M->kp.kind,
                                                                         M->kp.sf2, M->BT32, M->vy32, g, pts, pt_base, count,
                                                                         mean, var);
    }
    note_launch();
}

// Prior covariance between a grid point and its neighbour at offset e.
static void prior_offsets(const gpr_model *M, const GridDev &g, double kprior[13])
{
    for (int e = 0; e < 13; ++e) {
        double r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            double t = kOff13[e][d] * g.h[d] / M->kp.ell[d];
            r2 += t * t;
        }
        if (M->kp.kind == GPR_K_SE) kprior[e] = M->kp.sf2 * exp(-0.5 * r2);
        else {
            double r = sqrt(r2), s5r = sqrt(5.0) * r;
            kprior[e] = M->kp.sf2 * (1.0 + s5r + 5.0 * r2 / 3.0) * exp(-s5r);
        }
    }
}

struct Prior13 {
    double k[13];
};

__constant__ int c_off13[13][3] = {{1, -1, -1}, {1, -1, 0}, {1, -1, 1}, {1, 0, -1}, {1, 0, 0}, {1, 0, 1}, {1, 1, -1},
                                   {1, 1, 0},   {1, 1, 1},  {0, 1, -1}, {0, 1, 0},  {0, 1, 1}, {0, 0, 1}};

// Warp per listed point: 15 dot products over the W rows of the point and its neighbours.
template <typename T, typename OutT>
__global__ void k_stats_from_w(GridDev g, const int64_t *pts, int64_t pt_base, int64_t count, const int32_t *slot,
                               int64_t slot_base, const T *W,
                               int64_t mp, const T *vy, double sf2, Prior13 pr, OutT *out15, OutT *mean, OutT *var,
                               OutT *cov13)
{
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    int64_t pos = blockIdx.x * (int64_t)(blockDim.x / 32) + warp;
    if (pos >= count) return;
    int64_t p = pts ? pts[pos] : pt_base + pos;
    int64_t nx = g.n[0], ny = g.n[1], nz = g.n[2];
    if (p < 0 || p >= nx * ny * nz) {  // listed index off the grid: the caller gets NaN stats
        if (lane == 0 && out15)
            for (int s = 0; s < 15; ++s) out15[pos * 15 + s] = (OutT)NAN;
        return;
    }
    int ix = (int)(p % nx), iy = (int)((p / nx) % ny), iz = (int)(p / (nx * ny));
    int64_t self = slot ? (int64_t)slot[p] : p - slot_base;
    int64_t nb[13];
#pragma unroll
    for (int e = 0; e < 13; ++e) {
        int a = ix + c_off13[e][0], b = iy + c_off13[e][1], c = iz + c_off13[e][2];
        int64_t r = -1;
        if (a >= 0 && b >= 0 && c >= 0 && a < nx && b < ny && c < nz) {
            int64_t q = a + nx * (b + ny * (int64_t)c);
            r = slot ? (int64_t)slot[q] : q - slot_base;
        }
        nb[e] = r;
    }
    T acc[15];
#pragma unroll
    for (int s = 0; s < 15; ++s) acc[s] = T(0);
    const T *wp = W + self * mp;
    for (int64_t j = lane; j < mp; j += 32) {
        T w = wp[j];
        acc[0] = fma(w, vy[j], acc[0]);
        acc[1] = fma(w, w, acc[1]);
#pragma unroll
        for (int e = 0; e < 13; ++e)
            if (nb[e] >= 0) acc[2 + e] = fma(w, W[nb[e] * mp + j], acc[2 + e]);
    }
#pragma unroll
    for (int s = 0; s < 15; ++s)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[s] += __shfl_xor_sync(0xffffffffu, acc[s], o);
    if (lane == 0) {
        double mu = (double)acc[0], v = sf2 - (double)acc[1];
        if (out15) {
            OutT *o = out15 + pos * 15;
            o[0] = (OutT)mu;
            o[1] = (OutT)v;
#pragma unroll
            for (int e = 0; e < 13; ++e) o[2 + e] = nb[e] >= 0 ? (OutT)(pr.k[e] - (double)acc[2 + e]) : (OutT)NAN;
        } else {
            mean[pos] = (OutT)mu;
            var[pos] = (OutT)v;
            if (cov13)
#pragma unroll
                for (int e = 0; e < 13; ++e)
                    cov13[pos * 13 + e] = nb[e] >= 0 ? (OutT)(pr.k[e] - (double)acc[2 + e]) : (OutT)NAN;
        }
    }
}

void launch_stats_from_w64(const gpr_model *M, const GridDev &g, const int64_t *pts, int64_t pt_base, int64_t count,
                           const int32_t *slot, int64_t slot_base, const double *W, double *out15, double *mean,
                           double *var, double *cov13, cudaStream_t st)
{
    if (count <= 0) return;
    Prior13 pr;
    prior_offsets(M, g, pr.k);
    {
        ProfScope _ps("stats_from_w64", st);
        k_stats_from_w<double, double><<<(unsigned)((count + 7) / 8), 256, 0, st>>>(
        g, pts, pt_base, count, slot, slot_base, W, M->mp, M->vy, M->kp.sf2, pr, out15, mean, var, cov13);
    }
    note_launch();
}

void launch_stats_from_w32(const gpr_model *M, const GridDev &g, const int64_t *pts, int64_t pt_base, int64_t count,
                           const int32_t *slot, int64_t slot_base, const float *W, float *mean, float *var,
                           float *cov13, cudaStream_t st)
{
    if (count <= 0) return;
    Prior13 pr;
    prior_offsets(M, g, pr.k);
    {
        ProfScope _ps("stats_from_w32", st);
        k_stats_from_w<float, float><<<(unsigned)((count + 7) / 8), 256, 0, st>>>(
        g, pts, pt_base, count, slot, slot_base, W, M->mp, M->vy32, M->kp.sf2, pr, nullptr, mean, var, cov13);
    }
    note_launch();
}

// ---------------------------------------------------------------- compensated mean
// mu_p = sum_j k(x_p, X_j) alpha_j evaluated in float-float arithmetic (pairs of FP32
// carrying ~48 bits): the terms k_j alpha_j reach ~1e3 while mu is O(1), so a plain
// FP32 sum loses ~1e-4 of the field scale.  SE kernels: k = E_x E_y E_z from the
// float-float tables; Matern: FP64 arithmetic.
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

__global__ void k_mean_ff(const float2 *Tff, int64_t off1, int64_t off2, int64_t mp, int64_t m, const float2 *aff,
                          GridDev g, const int64_t *pts, int64_t pt_base, int64_t count, float *mean)
{
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    int64_t pos = blockIdx.x * (int64_t)(blockDim.x / 32) + warp;
    if (pos >= count) return;
    int64_t p = pts ? pts[pos] : pt_base + pos;
    int64_t nx = g.n[0], ny = g.n[1];
    if (p < 0 || p >= nx * ny * (int64_t)g.n[2]) return;
    int64_t gx = p % nx, gy = (p / nx) % ny, gz = p / (nx * ny);
    const float2 *tx = Tff + gx * mp, *ty = Tff + off1 + gy * mp, *tz = Tff + off2 + gz * mp;
    // two independent accumulation chains (more loads and float-float products in flight)
    FF acc = {0.f, 0.f}, acc2 = {0.f, 0.f};
    int64_t j = lane;
    for (; j + 32 < m; j += 64) {
        const float2 a = tx[j], b = ty[j], c = tz[j], al = aff[j];
        const float2 a2 = tx[j + 32], b2 = ty[j + 32], c2 = tz[j + 32], al2 = aff[j + 32];
        const FF k = ff_mul(ff_mul(FF{a.x, a.y}, FF{b.x, b.y}), FF{c.x, c.y});
        const FF k2 = ff_mul(ff_mul(FF{a2.x, a2.y}, FF{b2.x, b2.y}), FF{c2.x, c2.y});
        acc = ff_add(acc, ff_mul(k, FF{al.x, al.y}));
        acc2 = ff_add(acc2, ff_mul(k2, FF{al2.x, al2.y}));
    }
    if (j < m) {
        const float2 a = tx[j], b = ty[j], c = tz[j], al = aff[j];
        const FF k = ff_mul(ff_mul(FF{a.x, a.y}, FF{b.x, b.y}), FF{c.x, c.y});
        acc = ff_add(acc, ff_mul(k, FF{al.x, al.y}));
    }
    acc = ff_add(acc, acc2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        FF t = {__shfl_xor_sync(0xffffffffu, acc.h, o), __shfl_xor_sync(0xffffffffu, acc.l, o)};
        acc = ff_add(acc, t);
    }
    if (lane == 0) mean[pos] = acc.h + acc.l;
}

__global__ void k_mean_f64(const double *T64, int64_t off1, int64_t off2, int64_t mp, int64_t m, double sf2,
                           const double *alpha, GridDev g, const int64_t *pts, int64_t pt_base, int64_t count,
                           float *mean)
{
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    int64_t pos = blockIdx.x * (int64_t)(blockDim.x / 32) + warp;
    if (pos >= count) return;
    int64_t p = pts ? pts[pos] : pt_base + pos;
    int64_t nx = g.n[0], ny = g.n[1];
    if (p < 0 || p >= nx * ny * (int64_t)g.n[2]) return;
    int64_t gx = p % nx, gy = (p / nx) % ny, gz = p / (nx * ny);
    double acc = 0.0;
    for (int64_t j = lane; j < m; j += 32) {
        double r2 = T64[gx * mp + j] + T64[off1 + gy * mp + j] + T64[off2 + gz * mp + j];
        acc += KFun<double>::matern(r2, sf2) * alpha[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) mean[pos] = (float)acc;
}

void launch_mean_compensated(const gpr_model *M, const GridDev &g, const float2 *Tff, const double *T64,
                             const int64_t *pts, int64_t pt_base, int64_t count, float *mean, cudaStream_t st)
{
    if (count <= 0) return;
    int64_t o1, o2;
    table_offsets(M, g, o1, o2);
    ProfScope _ps("mean_ff", st);
    if (M->kp.kind == GPR_K_SE)
        k_mean_ff<<<(unsigned)((count + 7) / 8), 256, 0, st>>>(Tff, o1, o2, M->mp, M->m, M->alpha_ff, g, pts, pt_base,
                                                             count, mean);
    else
        k_mean_f64<<<(unsigned)((count + 7) / 8), 256, 0, st>>>(T64, o1, o2, M->mp, M->m, M->kp.sf2, M->alpha, g,
                                                              pts, pt_base, count, mean);
    note_launch();
}
