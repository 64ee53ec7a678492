// Hand-written adjoint of the LCP field (no counterpart in the paper):
//   loss = sum_c dL_dlcp[c] * LCP_c   ->   dloss/dy, dloss/dlog l_d.
//
// Per cell (K9): reverse sweep of the sequential-conditioning estimator (FP32, lanes over
// samples) and the 8x8 Cholesky / jitter adjoint (FP64) give dloss/dmu_8 and dloss/dSigma_8,
// scattered onto the per-point statistics: g_mu[p], G_var[p], G_cov[p][e].
// Through Eq. (1) in the whitened form (K10/K11), with W rows w_p = L^-1 k_p,
// G_pq the symmetric pair weights, Zh_p = sum_q G_pq w_q, Z_p = L^-T Zh_p, t = W^T g_mu:
//   dloss/dy        = L^-T t
//   dloss/dlog l_d  = sum_p g_p kd_p.alpha + sum_(p,e) G_cov[p][e] kd_e - 2 sum_p kd_p.Z_p
//                     + tr(Kd_d L^-T (Zh^T W - v t^T) L^-1)
// with kd = dk/dlog l_d, Kd_d = dK(X,X)/dlog l_d and v = L^-1 y.  The kernel rows K_* are
// regenerated from the tables, never stored; the m x m parts are FP64.
#include <math.h>
#include <string.h>

#include "internal.h"
#include "normal_fast.cuh"

namespace {

__constant__ int c_off[13][3] = {{1, -1, -1}, {1, -1, 0}, {1, -1, 1}, {1, 0, -1}, {1, 0, 0}, {1, 0, 1}, {1, 1, -1},
                                 {1, 1, 0},   {1, 1, 1},  {0, 1, -1}, {0, 1, 0},  {0, 1, 1}, {0, 0, 1}};

struct Pairs {
    int owner[8][8];
    int slot[8][8];
};

Pairs make_pairs()
{
    Pairs t;
    for (int c1 = 0; c1 < 8; ++c1)
        for (int c2 = 0; c2 < 8; ++c2) {
            t.owner[c1][c2] = -1;
            t.slot[c1][c2] = -1;
            if (c1 == c2) continue;
            int d[3] = {(c2 & 1) - (c1 & 1), ((c2 >> 1) & 1) - ((c1 >> 1) & 1), ((c2 >> 2) & 1) - ((c1 >> 2) & 1)};
            for (int e = 0; e < 13; ++e) {
                if (kOff13[e][0] == d[0] && kOff13[e][1] == d[1] && kOff13[e][2] == d[2]) { t.owner[c1][c2] = 0; t.slot[c1][c2] = e; }
                if (kOff13[e][0] == -d[0] && kOff13[e][1] == -d[1] && kOff13[e][2] == -d[2]) { t.owner[c1][c2] = 1; t.slot[c1][c2] = e; }
            }
        }
    return t;
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__device__ __forceinline__ float u01f(uint32_t x) { return (float)(((x >> 9) << 1) | 1u) * (1.0f / 16777216.0f); }
__device__ __forceinline__ float npdf(float x) { return 0.3989422804014327f * __expf(-0.5f * x * x); }

struct Lat {
    uint32_t G[7];
};

// FP32 view of one kept cell's factor for the sampling sweep, rows pre-scaled by 1/L_ii:
// u_i = sg bs_i - sum_{j<i} Ls_ij z_j with Ls_ij = L_ij / L_ii, bs_i = (theta - mu_i) / L_ii.
struct AdjRec {
    float Ls[28];  // strictly lower part, entry (i, j) at trs(i, j)
    float bs[8];
    int active;
    int pad[3];
};
__device__ __forceinline__ int trs(int i, int j) { return i * (i - 1) / 2 + j; }
constexpr int kRed = 1 + 8 + 28;  // P_lo + P_hi, bs adjoint (8), Ls adjoint (28): FP32 sums per cell

// The cell's 8 corner statistics, jitter and FP64 Cholesky factor, exactly as the forward
// estimator forms them; false when the cell is skipped (zero weight, no variance, Boole test).
__device__ bool adj_factor(const GridDev &g, const double *stats, const int32_t *slot, int64_t cidx, float wbar,
                           double theta, double tau, double skip_eps, const Pairs &pt, double Lm[8][8], double mu[8],
                           int slots[8], int &am)
{
    const int64_t cx = g.n[0] - 1, cy = g.n[1] - 1;
    const int64_t i = cidx % cx, j = (cidx / cx) % cy, k = cidx / (cx * cy);
    const double *row[8];
    double S[8][8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int64_t p = (i + (c & 1)) + (int64_t)g.n[0] * ((j + ((c >> 1) & 1)) + (int64_t)g.n[1] * (k + (c >> 2)));
        slots[c] = slot[p];
        row[c] = stats + (int64_t)slots[c] * 15;
        mu[c] = row[c][0];
        S[c][c] = row[c][1];
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = a + 1; b < 8; ++b) {
            const double v = pt.owner[a][b] == 0 ? row[a][2 + pt.slot[a][b]] : row[b][2 + pt.slot[a][b]];
            S[a][b] = v;
            S[b][a] = v;
        }
    double maxd = 0.0;
    am = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (S[c][c] > maxd) { maxd = S[c][c]; am = c; }
    if (wbar == 0.0f || !(maxd > 1e-30)) return false;
    const double jit = tau * maxd;
#pragma unroll
    for (int c = 0; c < 8; ++c) S[c][c] += jit;
    double sa = 0.0, sb = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const double sd = sqrt(S[c][c]);
        sa += normcdf((mu[c] - theta) / sd);
        sb += normcdf((theta - mu[c]) / sd);
    }
    if (sa < skip_eps || sb < skip_eps) return false;
    const double fl = 1e-3 * jit;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            double v = S[a][b];
#pragma unroll
            for (int r = 0; r < b; ++r) v -= Lm[a][r] * Lm[b][r];
            if (a == b) {
                if (!(v > fl)) v = fl;
                Lm[a][a] = sqrt(v);
            } else {
                Lm[a][b] = v / Lm[b][b];
            }
        }
    return true;
}

// K9a: thread per kept cell: the FP64 factor and its FP32 record for the sweep.
__global__ void k_adj_prep(GridDev g, const double *stats, const int32_t *slot, const int64_t *cells, int64_t count,
                           const float *dldlcp, double theta, double tau, double skip_eps, Pairs pt, AdjRec *rec)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= count) return;
    const int64_t cidx = cells[q];
    double Lm[8][8], mu[8];
    int slots[8], am;
    AdjRec &R = rec[q];
    if (!adj_factor(g, stats, slot, cidx, dldlcp[cidx], theta, tau, skip_eps, pt, Lm, mu, slots, am)) {
        R.active = 0;
        return;
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const double inv = 1.0 / Lm[a][a];
        R.bs[a] = (float)((theta - mu[a]) * inv);
#pragma unroll
        for (int b = 0; b < a; ++b) R.Ls[trs(a, b)] = (float)(Lm[a][b] * inv);
    }
    R.active = 1;
}

// K9b: warp per kept cell: the estimator's samples forward and their reverse sweep (FP32,
// lanes over lattice points), reduced over the warp to the kRed sums of the cell.
__global__ void __launch_bounds__(256, 2) k_adj_sample(const AdjRec *rec, const int64_t *cells, int64_t count, const float *dldlcp, int N,
                             uint64_t seed, Lat lat, float *red)
{
    __shared__ AdjRec wc[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = blockIdx.x * (int64_t)(blockDim.x >> 5) + warp;
    if (q >= count) return;
    if (!rec[q].active) return;
    AdjRec &W = wc[warp];
    for (int t = lane; t < (int)(sizeof(AdjRec) / 4); t += 32) ((float *)&W)[t] = ((const float *)&rec[q])[t];
    __syncwarp();
    const int64_t cidx = cells[q];
    const float wbar = dldlcp[cidx];
    uint32_t D = 0;
    if (lane < 7) D = (uint32_t)(splitmix64(seed, (uint64_t)cidx * 8 + lane + 1) >> 32);
    uint32_t Ds[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) Ds[i] = __shfl_sync(0xffffffffu, D, i);
    // bbar: adjoint of bs (orthant sign folded in), Lbar: of Ls, P: both orthant sums
    float bbar[8], Lbar[28];
    float P = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) bbar[i] = 0.f;
#pragma unroll
    for (int t = 0; t < 28; ++t) Lbar[t] = 0.f;
    const float fbar = -wbar / (float)N;
    // the first coordinate does not depend on the sample: its factor and density, per orthant
    const float e0lo = nrm_cdf(W.bs[0]), e0hi = nrm_cdf(-W.bs[0]), pdf0 = npdf(W.bs[0]);
    for (int k = lane; k < N; k += 32) {
        float w[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            uint32_t U = (uint32_t)k * lat.G[i] + Ds[i];
            w[i] = fabsf(2.0f * u01f(U) - 1.0f);
        }
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            float sg = side == 0 ? 1.f : -1.f;
            float pd[8], e[8], z[7];  // pd: the density at u_i, from the exponential of Phi(u_i)
            float f = 1.f;
            // no early exit: once f underflows to 0 the rest stays finite and the sample adds 0
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float s = sg * W.bs[i];
#pragma unroll
                for (int j = 0; j < i; ++j) s = fmaf(-W.Ls[trs(i, j)], z[j], s);
                if (i == 0) {
                    e[0] = side ? e0hi : e0lo;
                    pd[0] = pdf0;
                } else {
                    e[i] = nrm_cdf_pdf(s, pd[i]);
                }
                f *= e[i];
                if (i < 7) z[i] = nrm_ppf(fmaxf(w[i] * e[i], 1e-37f));
            }
            P += f;
            if (!(f > 1e-30f)) continue;  // negligible share of value and gradient (both scale with f)
            float zbar[7];
#pragma unroll
            for (int i = 0; i < 7; ++i) zbar[i] = 0.f;
#pragma unroll
            for (int i = 7; i >= 0; --i) {
                float ebar = fbar * __fdividef(f, e[i]);  // e[i] >= f > 1e-30
                if (i < 7) {
                    const float iph = 2.50662827f * __expf(0.5f * z[i] * z[i]);  // 1 / phi(z)
                    if (iph < INFINITY) ebar = fmaf(zbar[i] * w[i], iph, ebar);
                }
                const float ubar = ebar * pd[i];
                bbar[i] = fmaf(sg, ubar, bbar[i]);
#pragma unroll
                for (int j = 0; j < i; ++j) {
                    Lbar[trs(i, j)] = fmaf(-ubar, z[j], Lbar[trs(i, j)]);
                    zbar[j] = fmaf(-ubar, W.Ls[trs(i, j)], zbar[j]);
                }
            }
        }
    }
    // warp reductions; lane t stores sums t and t + 32
    float out0 = 0.f, out1 = 0.f;
#pragma unroll
    for (int t = 0; t < kRed; ++t) {
        float v = t == 0 ? P : (t < 9 ? bbar[t - 1] : Lbar[t - 9]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (t == lane) out0 = v;
        if (t == lane + 32) out1 = v;
    }
    red[q * kRed + lane] = out0;
    if (lane + 32 < kRed) red[q * kRed + lane + 32] = out1;
}

// K9c: thread per kept cell: the FP64 factor again (same bits as in K9a), the Cholesky /
// jitter adjoint Sbar = L^-T sym(Phi(L^T Lbar)) L^-1, scattered onto the per-point weights.
__global__ void k_adj_chol(GridDev g, const double *stats, const int32_t *slot, const int64_t *cells, int64_t count,
                           const float *dldlcp, double theta, double tau, double skip_eps, int N, Pairs pt,
                           const AdjRec *rec, const float *red, double *G16)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= count || !rec[q].active) return;
    const int64_t cidx = cells[q];
    double L[8][8], mu[8];
    int slots[8], am;
    if (!adj_factor(g, stats, slot, cidx, dldlcp[cidx], theta, tau, skip_eps, pt, L, mu, slots, am)) return;
    const float *rd = red + q * kRed;
    const double lcp = 1.0 - (double)rd[0] / N;
    if (lcp < 0.0 || lcp > 1.0) return;  // clamped: constant in a neighbourhood
    // adjoints of the pre-scaled rows back to L: Ls_ij = L_ij / L_ii, bs_i = (theta - mu_i) / L_ii
    double Lb[8][8], Pm[8][8], T[8][8], Li[8][8], mubar[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const double inv = 1.0 / L[i][i], bsb = (double)rd[1 + i];
        double dg = bsb * (theta - mu[i]) * inv;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j > i) L[i][j] = 0.0;
            Lb[i][j] = 0.0;
        }
#pragma unroll
        for (int j = 0; j < i; ++j) {
            const double lsb = (double)rd[9 + trs(i, j)];
            Lb[i][j] = lsb * inv;
            dg += lsb * L[i][j] * inv;
        }
        Lb[i][i] = -dg * inv;
        mubar[i] = -bsb * inv;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < 8; ++k) s += L[k][i] * Lb[k][j];
            Pm[i][j] = s;
        }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) T[i][j] = j < i ? Pm[i][j] : (j == i ? 0.5 * Pm[i][i] : 0.0);
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) Pm[i][j] = 0.5 * (T[i][j] + T[j][i]);
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
#pragma unroll
            for (int k = 0; k < i; ++k) s -= L[i][k] * Li[k][c];
            Li[i][c] = i < c ? 0.0 : s / L[i][i];
        }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < 8; ++k) s += Pm[i][k] * Li[k][j];
            T[i][j] = s;
        }
    double tr = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < 8; ++k) s += Li[k][i] * T[k][j];
            Pm[i][j] = s;  // Sbar
            if (i == j) tr += s;
        }
    // mu adjoint: b_lo = theta - mu, b_hi = mu - theta; jitter tau * max diag on the argmax
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        double *gp = G16 + (int64_t)slots[i] * 16;
        atomicAdd(gp + 0, mubar[i]);
        atomicAdd(gp + 1, Pm[i][i] + (i == am ? tau * tr : 0.0));
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = a + 1; b < 8; ++b) {
            const int own = pt.owner[a][b] == 0 ? a : b;
            atomicAdd(G16 + (int64_t)slots[own] * 16 + 2 + pt.slot[a][b], 2.0 * Pm[a][b]);
        }
}

// t partial sums: tp[chunk][j] = sum_{p in chunk} g_mu[p] W[p][j].
__global__ void k_wt_vec(const double *W, const double *G16, int64_t np, int64_t mp, int64_t chunk, double *tp)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t c = blockIdx.y;
    if (j >= mp) return;
    int64_t p0 = c * chunk, p1 = p0 + chunk < np ? p0 + chunk : np;
    double s = 0.0;
    for (int64_t p = p0; p < p1; ++p) s += G16[p * 16] * W[p * mp + j];
    tp[c * mp + j] = s;
}

__global__ void k_sum_rows(const double *part, int64_t nrow, int64_t len, double *out)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= len) return;
    double s = 0.0;
    for (int64_t r = 0; r < nrow; ++r) s += part[r * len + j];
    out[j] = s;
}

// Zh_p = G_pp w_p + sum_e (G_cov[p][e]/2) w_{p+e} + sum_e (G_cov[p-e][e]/2) w_{p-e}  (warp per point).
__global__ void k_zhat(GridDev g, const int64_t *pts, int64_t np, const int32_t *slot, const double *W,
                       const double *G16, int64_t mp, double *Zh)
{
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    int64_t pos = blockIdx.x * (int64_t)(blockDim.x / 32) + warp;
    if (pos >= np) return;
    int64_t p = pts[pos];
    int64_t nx = g.n[0], ny = g.n[1], nz = g.n[2];
    int ix = (int)(p % nx), iy = (int)((p / nx) % ny), iz = (int)(p / (nx * ny));
    int64_t rows[27];
    double wts[27];
    int cnt = 0;
    rows[cnt] = pos;
    wts[cnt++] = G16[pos * 16 + 1];
    for (int e = 0; e < 13; ++e) {
        int a = ix + c_off[e][0], b = iy + c_off[e][1], c = iz + c_off[e][2];
        if (a >= 0 && b >= 0 && c >= 0 && a < nx && b < ny && c < nz) {
            int s = slot[a + nx * (b + ny * (int64_t)c)];
            double gv = G16[pos * 16 + 2 + e];
            if (s >= 0 && gv != 0.0) { rows[cnt] = s; wts[cnt++] = 0.5 * gv; }
        }
        a = ix - c_off[e][0]; b = iy - c_off[e][1]; c = iz - c_off[e][2];
        if (a >= 0 && b >= 0 && c >= 0 && a < nx && b < ny && c < nz) {
            int s = slot[a + nx * (b + ny * (int64_t)c)];
            if (s >= 0) {
                double gv = G16[(int64_t)s * 16 + 2 + e];
                if (gv != 0.0) { rows[cnt] = s; wts[cnt++] = 0.5 * gv; }
            }
        }
    }
    for (int64_t j = lane; j < mp; j += 32) {
        double acc = 0.0;
        for (int t = 0; t < cnt; ++t) acc += wts[t] * W[rows[t] * mp + j];
        Zh[pos * mp + j] = acc;
    }
}

// (sh, sl) += (gh + gl)(wh + wl) in float-float (compensated dot product: the product's high
// part joins the running sum by an error-free TwoSum, every rounding error goes to sl).
__device__ __forceinline__ void ff_dot_step(float &sh, float &sl, float gh, float gl, float wh, float wl)
{
    const float p = gh * wh;
    float e = fmaf(gh, wh, -p);
    e = fmaf(gh, wl, fmaf(gl, wh, e));
    const float t = sh + p;
    const float bv = t - sh;
    sl += ((sh - (t - bv)) + (p - bv)) + e;
    sh = t;
}

// Exact FP64 value of a normal FP32 number (or 0) from its bit pattern, without FP64 instructions.
__device__ __forceinline__ double f2d_bits(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t ef = (b >> 23) & 0xFF;
    if (ef == 0) return 0.0;
    const unsigned long long db = ((unsigned long long)(b >> 31) << 63) | ((unsigned long long)(ef + 896) << 52) |
                                  ((unsigned long long)(b & 0x7FFFFF) << 29);
    return __longlong_as_double((long long)db);
}

// k_zhat from the float-float rows (hi, lo pairs, 512-byte aligned rows of even length mp):
// the same sums as float-float compensated dot products, two columns per lane, FP64 out.
__global__ void k_zhat_ff(GridDev g, const int64_t *pts, int64_t np, const int32_t *slot, const float2 *Wff,
                          const double *G16, int64_t mp, double *Zh)
{
    __shared__ int4 lst[8][27];  // per warp: (row, weight hi bits, weight lo bits)
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t pos = blockIdx.x * (int64_t)(blockDim.x / 32) + warp;
    if (pos >= np) return;
    const int64_t p = pts[pos];
    const int64_t nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int ix = (int)(p % nx), iy = (int)((p / nx) % ny), iz = (int)(p / (nx * ny));
    int4 *L = lst[warp];
    int cnt = 0;
    auto add = [&](int64_t r, double w) {
        if (lane == 0) {
            const float h = (float)w;
            L[cnt] = make_int4((int)r, __float_as_int(h), __float_as_int((float)(w - (double)h)), 0);
        }
        ++cnt;
    };
    add(pos, G16[pos * 16 + 1]);
    for (int e = 0; e < 13; ++e) {
        int a = ix + c_off[e][0], b = iy + c_off[e][1], c = iz + c_off[e][2];
        if (a >= 0 && b >= 0 && c >= 0 && a < nx && b < ny && c < nz) {
            const int s = slot[a + nx * (b + ny * (int64_t)c)];
            const double gv = G16[pos * 16 + 2 + e];
            if (s >= 0 && gv != 0.0) add(s, 0.5 * gv);
        }
        a = ix - c_off[e][0]; b = iy - c_off[e][1]; c = iz - c_off[e][2];
        if (a >= 0 && b >= 0 && c >= 0 && a < nx && b < ny && c < nz) {
            const int s = slot[a + nx * (b + ny * (int64_t)c)];
            if (s >= 0) {
                const double gv = G16[(int64_t)s * 16 + 2 + e];
                if (gv != 0.0) add(s, 0.5 * gv);
            }
        }
    }
    __syncwarp();
    for (int64_t j2 = lane; j2 < mp / 2; j2 += 32) {
        float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
        for (int t = 0; t < cnt; ++t) {
            const int4 e = L[t];
            const float gh = __int_as_float(e.y), gl = __int_as_float(e.z);
            const float4 v = *(const float4 *)(Wff + (int64_t)e.x * mp + 2 * j2);
            ff_dot_step(h0, l0, gh, gl, v.x, v.y);
            ff_dot_step(h1, l1, gh, gl, v.z, v.w);
        }
        *(double2 *)(Zh + pos * mp + 2 * j2) = make_double2(f2d_bits(h0) + f2d_bits(l0), f2d_bits(h1) + f2d_bits(l1));
    }
}

// Rows and statistics of the listed points from the model's grid cache (rows and stats15 by
// grid point): float-float rows, their FP64 values and stats15 in list order.  Thread per pair of
// row elements (rows 512-byte aligned, mp even).
__global__ void k_gather_rows(const float2 *Wc, const double *Sc, const int64_t *pts, int64_t np, int64_t mp,
                              float2 *Wff, double *W, double *S15)
{
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t half = mp / 2;
    if (idx >= np * half) return;
    const int64_t r = idx / half, j2 = idx % half, p = pts[r];
    const float4 v = ((const float4 *)(Wc + p * mp))[j2];
    ((float4 *)(Wff + r * mp))[j2] = v;
    ((double2 *)(W + r * mp))[j2] = make_double2(f2d_bits(v.x) + f2d_bits(v.y), f2d_bits(v.z) + f2d_bits(v.w));
    if (j2 < 15) S15[r * 15 + j2] = Sc[p * 15 + j2];
}

// Generic FP64 tiled GEMM: C_z = opA(A) B over the K range of split z (partials stacked by z).
// opA(i,k) = TA ? A[k*lda + i] : A[i*lda + k];  LOWERB: B[k][j] = 0 for k < j (skip those k).
constexpr int GB = 64, GK = 16;
template <bool TA, bool LOWERB>
__global__ void __launch_bounds__(256) k_gemm64(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                                                const double *B, int64_t ldb, double *C, int64_t ldc, int64_t kchunk)
{
    __shared__ double As[GK][GB + 2], Bs[GK][GB + 2];
    int t = threadIdx.x, tx = t % 16, ty = t / 16;
    int64_t i0 = (int64_t)blockIdx.x * GB, j0 = (int64_t)blockIdx.y * GB;
    int64_t kb = (int64_t)blockIdx.z * kchunk, ke = kb + kchunk < K ? kb + kchunk : K;
    if (LOWERB && kb < j0) kb = j0 / GK * GK;
    double acc[4][4] = {};
    for (int64_t k0 = kb; k0 < ke; k0 += GK) {
        for (int e = t; e < GK * GB; e += 256) {
            int kk = e / GB, ii = e % GB;
            int64_t k = k0 + kk, i = i0 + ii;
            double v = 0.0;
            if (k < ke && i < M) v = TA ? A[k * lda + i] : A[i * lda + k];
            As[kk][ii] = v;
            int64_t j = j0 + ii;
            Bs[kk][ii] = (k < ke && j < N) ? B[k * ldb + j] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx * 4 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
    double *Cz = C + (int64_t)blockIdx.z * M * ldc;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int64_t i = i0 + ty * 4 + r;
        if (i >= M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int64_t j = j0 + tx * 4 + c;
            if (j < N) Cz[i * ldc + j] = acc[r][c];
        }
    }
}

template <bool TA, bool LOWERB>
void gemm64(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
            int64_t ldc, int splits, cudaStream_t st)
{
    int64_t kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + GK - 1) / GK * GK;
    dim3 grid((unsigned)((M + GB - 1) / GB), (unsigned)((N + GB - 1) / GB), (unsigned)splits);
    k_gemm64<TA, LOWERB><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, kchunk);
    note_launch();
}

// M = R - v t^T over the m x m block (zero padding elsewhere kept).
__global__ void k_form_m(double *R, const double *vy, const double *t, int64_t m, int64_t mp)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= mp * mp) return;
    int64_t i = idx / mp, j = idx % mp;
    if (i < m && j < m) R[idx] -= vy[i] * t[j];
    else R[idx] = 0.0;
}

__device__ __forceinline__ double kdot(int kind, const double *ell, double sf2, const double *a, const double *b, int d)
{
    double r2 = 0.0;
    for (int q = 0; q < 3; ++q) {
        double t = (a[q] - b[q]) / ell[q];
        r2 += t * t;
    }
    double t = (a[d] - b[d]) / ell[d], t2 = t * t;
    if (kind == GPR_K_SE) return sf2 * exp(-0.5 * r2) * t2;
    double r = sqrt(r2), s5r = 2.2360679774997896964 * r;
    return (5.0 / 3.0) * sf2 * (1.0 + s5r) * exp(-s5r) * t2;
}

// out[d] += sum_ij Kd_d[i][j] N[j][i]  (block reduction, FP64 atomics).
__global__ void k_trace(const double *X, int64_t m, KernParams kp, const double *Nm, int64_t mp, double *out)
{
    __shared__ double red[3][256];
    double acc[3] = {0, 0, 0};
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < m * m;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx / m, j = idx % m;
        double nji = Nm[j * mp + i];
        for (int d = 0; d < 3; ++d) acc[d] += kdot(kp.kind, kp.ell, kp.sf2, X + 3 * i, X + 3 * j, d) * nji;
    }
    for (int d = 0; d < 3; ++d) red[d][threadIdx.x] = acc[d];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int d = 0; d < 3; ++d) red[d][threadIdx.x] += red[d][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 3; ++d) atomicAdd(out + d, red[d][0]);
}

struct KdPrior {
    double k[13][3];
};

// Per-point terms: g_p kd_p.alpha - 2 kd_p.Z_p + sum_e G_cov[p][e] kd_e  (warp per point).
__global__ void k_point_terms(GridDev g, const int64_t *pts, int64_t np, const double *X, int64_t m, KernParams kp,
                              const double *alpha, const double *Z, int64_t mp, const double *G16, KdPrior kdp,
                              double *out)
{
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    int64_t pos = blockIdx.x * (int64_t)(blockDim.x / 32) + warp;
    double acc[3] = {0, 0, 0};
    if (pos < np) {
        int64_t p = pts[pos];
        int64_t nx = g.n[0], ny = g.n[1];
        double x[3] = {g.lo[0] + (double)(p % nx) * g.h[0], g.lo[1] + (double)((p / nx) % ny) * g.h[1],
                       g.lo[2] + (double)(p / (nx * ny)) * g.h[2]};
        double gm = G16[pos * 16];
        const double *zr = Z + pos * mp;
        for (int64_t j = lane; j < m; j += 32) {
            double coef = gm * alpha[j] - 2.0 * zr[j];
            for (int d = 0; d < 3; ++d) acc[d] += kdot(kp.kind, kp.ell, kp.sf2, x, X + 3 * j, d) * coef;
        }
        if (lane == 0)
            for (int e = 0; e < 13; ++e) {
                double gc = G16[pos * 16 + 2 + e];
                if (gc != 0.0)
                    for (int d = 0; d < 3; ++d) acc[d] += gc * kdp.k[e][d];
            }
    }
    for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) acc[d] += __shfl_xor_sync(0xffffffffu, acc[d], o);
    if (lane == 0 && pos < np)
        for (int d = 0; d < 3; ++d) atomicAdd(out + d, acc[d]);
}

// Squared scaled distances per axis, Q_d[g][j] = ((x_g - X_jd) / l_d)^2 (zero for j >= m), laid out
// like the kernel tables.
__global__ void k_sqdist_tables(const double *X, int64_t m, int64_t mp, KernParams kp, GridDev g, double *Q,
                                float2 *Qff)
{
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)(g.n[0] + g.n[1] + g.n[2]) * mp;
    if (idx >= total) return;
    const int64_t row = idx / mp, j = idx % mp;
    int d = 0;
    int64_t gi = row;
    if (gi >= g.n[0]) { gi -= g.n[0]; d = 1; if (gi >= g.n[1]) { gi -= g.n[1]; d = 2; } }
    double v = 0.0;
    if (j < m) {
        const double t = (g.lo[d] + (double)gi * g.h[d] - X[3 * j + d]) / kp.ell[d];
        v = t * t;
    }
    Q[idx] = v;
    const float h = (float)v;
    Qff[idx] = make_float2(h, (float)(v - (double)h));
}

// Float-float value of an FP64 number from its bit pattern (integer steps): hi = x rounded to 24
// bits, lo = the remainder (rounded to 24 bits), |x - hi - lo| <= 2^-48 |x|.  Magnitudes outside
// [2^-60, 2^61) take FP64 conversions instead.
__device__ __forceinline__ float2 d2ff(double x)
{
    const long long b = __double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E < 1023 - 60 || E > 1023 + 60) {
        const float h = (float)x;
        return make_float2(h, (float)(x - (double)h));
    }
    const long long m53 = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);  // x = m53 2^(E-1075)
    const long long r = (m53 + (1LL << 28)) >> 29;                 // 24-bit rounding (2^24 carries)
    const int rem = (int)(m53 - (r << 29));                          // |rem| <= 2^28
    const float h = __int_as_float(((E - 896) << 23) + (int)(r - (1LL << 23)));
    const float l = (float)rem * __int_as_float((E - 948) << 23);   // times 2^(E-1075)
    return b < 0 ? make_float2(-h, -l) : make_float2(h, l);
}

__device__ __forceinline__ float2 ffmul(float2 a, float2 b)
{
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    const float s = p + e;
    return make_float2(s, e - (s - p));
}

__device__ __forceinline__ float2 ffadd(float2 a, float2 b)
{
    const float s = a.x + b.x;
    const float bv = s - a.x;
    const float err = ((a.x - (s - bv)) + (b.x - bv)) + (a.y + b.y);
    const float r = s + err;
    return make_float2(r, err - (r - s));
}

// k_point_terms for the SE kernel from its separable tables, k_pj = Tx Ty Tz (signal variance in
// Tx) and dk_pj/dlog l_d = k_pj Q_d, in float-float arithmetic on the FP32 pipe (the FP64 pipe
// runs at 1/64 of its rate): tables, alpha and g_mu as float-float, Z converted from FP64 by d2ff,
// the three sums as compensated dot products; FP64 from the warp reduction on.
__global__ void k_point_terms_se_ff(GridDev g, const int64_t *pts, int64_t np, const float2 *Tff, const float2 *Qff,
                                    int64_t m, const float2 *alpha_ff, const double *Z, int64_t mp,
                                    const double *G16, KdPrior kdp, double *out)
{
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t pos = blockIdx.x * (int64_t)(blockDim.x / 32) + warp;
    double acc[3] = {0, 0, 0};
    if (pos < np) {
        const int64_t p = pts[pos], nx = g.n[0], ny = g.n[1];
        const int64_t o0 = (p % nx) * mp, o1 = ((int64_t)g.n[0] + (p / nx) % ny) * mp,
                      o2 = ((int64_t)g.n[0] + g.n[1] + p / (nx * ny)) * mp;
        const float2 gm = d2ff(G16[pos * 16]);
        const double *zr = Z + pos * mp;
        float sh[3] = {0.f, 0.f, 0.f}, sl[3] = {0.f, 0.f, 0.f};
#pragma unroll 4
        for (int64_t j = lane; j < m; j += 32) {
            const float2 k = ffmul(ffmul(Tff[o0 + j], Tff[o1 + j]), Tff[o2 + j]);
            const float2 z = d2ff(zr[j]);
            const float2 kc = ffmul(k, ffadd(ffmul(gm, alpha_ff[j]), make_float2(-2.f * z.x, -2.f * z.y)));
            const float2 q[3] = {Qff[o0 + j], Qff[o1 + j], Qff[o2 + j]};
#pragma unroll
            for (int d = 0; d < 3; ++d) ff_dot_step(sh[d], sl[d], kc.x, kc.y, q[d].x, q[d].y);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) acc[d] = f2d_bits(sh[d]) + f2d_bits(sl[d]);
        if (lane == 0)
            for (int e = 0; e < 13; ++e) {
                const double gc = G16[pos * 16 + 2 + e];
                if (gc != 0.0)
                    for (int d = 0; d < 3; ++d) acc[d] += gc * kdp.k[e][d];
            }
    }
    for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) acc[d] += __shfl_xor_sync(0xffffffffu, acc[d], o);
    if (lane == 0 && pos < np)
        for (int d = 0; d < 3; ++d) atomicAdd(out + d, acc[d]);
}

// dy_i = sum_{j >= i} Linv[j][i] t_j.
__global__ void k_dy(const double *Linv, int64_t mb, const double *t, int64_t m, double *dy)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    double s = 0.0;
    for (int64_t j = i; j < m; ++j) s += Linv[j * mb + i] * t[j];
    dy[i] = s;
}

// Cells without weight, or (adaptive field) outside the leaf set S, have a constant LCP.
__global__ void k_mask_keep(uint8_t *keep, const float *dl, const uint8_t *leaf, int64_t nc)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c < nc && (dl[c] == 0.0f || (leaf && !leaf[c]))) keep[c] = 0;
}

__global__ void k_ff_to_double(const float2 *ff, int64_t n, double *out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)ff[i].x + (double)ff[i].y;
}

}  // namespace

// Plain FP64 products for the model set-up of other translation units: C = A B or A^T B
// (row-major, leading dimensions lda/ldb/ldc), no split.
void gemm64_nn(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
               int64_t ldc, cudaStream_t st)
{
    gemm64<false, false>(M, N, K, A, lda, B, ldb, C, ldc, 1, st);
}
void gemm64_tn(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
               int64_t ldc, cudaStream_t st)
{
    gemm64<true, false>(M, N, K, A, lda, B, ldb, C, ldc, 1, st);
}

static gpr_status lcp_backward(gpr_model *M, const gpr_grid *grid, double isovalue, const gpr_lcp_options *opts,
                               const float *dL_dlcp, const uint8_t *leaf, double *dL_dy, double *dL_dloglen,
                               cudaStream_t st)
{
    GridDev g = make_grid(grid);
    int64_t n = g.npts(), nc = g.ncells(), m = M->m, mp = M->mp, mb = (m + 31) / 32 * 32;
    size_t te = table_elems(M, g);
    size_t csb = compact_scratch_bytes(nc > n ? nc : n);
    size_t b1 = Carver::round(te * 4) + Carver::round(te * 8) + Carver::round(te * 8) + 2 * Carver::round((size_t)n * 4) +
                Carver::round((size_t)nc) + Carver::round((size_t)n) + Carver::round((size_t)n * 8) +
                Carver::round((size_t)n * 4) + Carver::round((size_t)nc * 8) + csb +
                Carver::round(tc_partial_elems(GPR_P_BF16X3, M, n) * 4) + 3 * Carver::round(te * 8) + 8192;
    GPR_TRY(ws_reserve(M, 0, b1, st));
    Carver cv{(char *)ws_ptr(M, 0)};
    float *T32 = cv.take<float>(te);
    double *T64 = cv.take<double>(te);
    float2 *Tff = cv.take<float2>(te);
    float *mean = cv.take<float>((size_t)n);
    float *var = cv.take<float>((size_t)n);
    uint8_t *keep = cv.take<uint8_t>((size_t)nc);
    uint8_t *pflag = cv.take<uint8_t>((size_t)n);
    int64_t *plist = cv.take<int64_t>((size_t)n);
    int32_t *slot = cv.take<int32_t>((size_t)n);
    int64_t *clist = cv.take<int64_t>((size_t)nc);
    void *cscr = cv.take<char>(csb);
    float *part = cv.take<float>(tc_partial_elems(GPR_P_BF16X3, M, n));
    float2 *Tu = cv.take<float2>(te);
    double *Q64 = cv.take<double>(te);
    float2 *Qff = cv.take<float2>(te);
    GPR_TRY(build_tables(M, g, T64, T32, st, Tff));
    // The model's grid cache: the per-point FP32-class mean/variance, float-float rows and complete
    // statistics that forward calls on this grid left are reused (what is missing is added).
    GridCache *C = nullptr;
    if (opts->exact == GPR_EXACT_AUTO && oz_supported(M) && opts->prec != GPR_P_FP64)
        GPR_TRY(grid_cache(M, grid, g, opts->prec, &C, st));
    // cells whose LCP is not identically 0 near the current parameters (same cascade as the forward)
    if (opts->prec == GPR_P_FP64) {
        GPR_CUDA_TRY(cudaMemsetAsync(keep, 1, (size_t)nc, st));
    } else if (C) {
        GPR_CUDA_TRY(cudaMemsetAsync(pflag, 1, (size_t)n, st));
        GPR_TRY(cache_fill_mv(M, C, g, pflag, plist, mean, var, part, cscr, csb, st));
        double mv, mm;
        prepass_margins(M, mv, mm);
        if (opts->prec == GPR_P_TF32 || opts->prec == GPR_P_BF16) mv = M->kp.sf2;
        launch_classify_cells_mv(g, C->mv, isovalue, opts->skip_eps, opts->jitter, mv, mm, keep, st);
    } else {
        GPR_TRY(fast_meanvar(M, g, opts->prec, T32, Tff, T64, nullptr, 0, n, mean, var, part, st));
        double mv, mm;
        prepass_margins(M, mv, mm);
        if (opts->prec == GPR_P_TF32 || opts->prec == GPR_P_BF16) mv = M->kp.sf2;
        launch_classify_cells(g, mean, var, isovalue, opts->skip_eps, opts->jitter, mv, mm, keep, st);
    }
    k_mask_keep<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(keep, dL_dlcp, leaf, nc);
    note_launch();
    GPR_CUDA_TRY(cudaMemsetAsync(pflag, 0, (size_t)n, st));
    launch_mark_corners(g, keep, pflag, st);
    int64_t npts = 0, ncell = 0;
    GPR_TRY(compact_flags(pflag, n, plist, slot, &npts, cscr, csb, st));
    GPR_TRY(compact_flags(keep, nc, clist, nullptr, &ncell, cscr, csb, st));
    double h_out[3] = {0, 0, 0};
    if (ncell == 0) {
        memset(dL_dy, 0, sizeof(double) * m);
        memcpy(dL_dloglen, h_out, sizeof h_out);
        return GPR_OK;
    }
    const bool use_oz = opts->exact == GPR_EXACT_AUTO && oz_supported(M);
    const int splits = 32;
    const int64_t chunk = 4096;
    int64_t nchunks = (npts + chunk - 1) / chunk;
    size_t b2 = 2 * Carver::round((size_t)npts * mp * 8) + Carver::round((size_t)npts * 15 * 8) +
                Carver::round((size_t)npts * 16 * 8) + Carver::round((size_t)nchunks * mp * 8) +
                Carver::round((size_t)splits * mp * mp * 8) + 3 * Carver::round((size_t)mp * mp * 8) +
                4 * Carver::round((size_t)mp * 8) + Carver::round((size_t)ncell * sizeof(AdjRec)) +
                Carver::round((size_t)ncell * kRed * 4) + (use_oz ? Carver::round((size_t)npts * mp * 8) : 0) +
                (C && C->W ? Carver::round((size_t)n * 2) + Carver::round((size_t)n * 16) : 0) + 4096;
    GPR_TRY(ws_reserve(M, 1, b2, st));
    Carver cv2{(char *)ws_ptr(M, 1)};
    double *W = cv2.take<double>((size_t)npts * mp);
    double *Zh = cv2.take<double>((size_t)npts * mp);
    double *S15 = cv2.take<double>((size_t)npts * 15);
    double *G16 = cv2.take<double>((size_t)npts * 16);
    double *tp = cv2.take<double>((size_t)nchunks * mp);
    double *Rp = cv2.take<double>((size_t)splits * mp * mp);
    double *R = cv2.take<double>((size_t)mp * mp);
    double *T1 = cv2.take<double>((size_t)mp * mp);
    double *Nm = cv2.take<double>((size_t)mp * mp);
    double *t = cv2.take<double>((size_t)mp);
    double *dy = cv2.take<double>((size_t)mp);
    double *acc = cv2.take<double>(4);
    AdjRec *arec = cv2.take<AdjRec>((size_t)ncell);
    float *ared = cv2.take<float>((size_t)ncell * kRed);
    float2 *Wff = use_oz ? cv2.take<float2>((size_t)npts * mp) : nullptr;
    if (C && C->W) {
        uint8_t *tmpflag = cv2.take<uint8_t>((size_t)n * 2);
        int64_t *list2 = cv2.take<int64_t>((size_t)n * 2);
        std::lock_guard<std::mutex> leaf_lock(M->leaf_mu);
        int64_t nrows = 0;
        GPR_TRY(cache_fill_stats(M, C, g, pflag, tmpflag, list2, cscr, csb, &nrows, st));
        k_gather_rows<<<(unsigned)((npts * (mp / 2) + 255) / 256), 256, 0, st>>>(C->W, C->S15, plist, npts, mp, Wff,
                                                                                 W, S15);
        note_launch();
    } else if (use_oz) {
        // FP64-class rows on the tensor cores (digit split), their float-float statistics, and the
        // rows widened to FP64 for the FP64 chain rule below
        GPR_TRY(oz_prepare(M, st));
        GPR_TRY(oz_unit_tables(M, g, Tu, st));
        GPR_TRY(launch_oz_w(M, g, Tu, plist, 0, npts, Wff, st));
        GPR_TRY(launch_stats_ff(M, g, plist, npts, slot, Wff, S15, st));
        k_ff_to_double<<<(unsigned)((npts * mp + 255) / 256), 256, 0, st>>>(Wff, npts * mp, W);
        note_launch();
    } else {
        launch_w64(M, g, T64, plist, 0, npts, W, st);
        launch_stats_from_w64(M, g, plist, 0, npts, slot, 0, W, S15, nullptr, nullptr, nullptr, st);
    }
    GPR_CUDA_TRY(cudaMemsetAsync(G16, 0, sizeof(double) * (size_t)npts * 16, st));
    GPR_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double) * 4, st));
    static Pairs pt = make_pairs();
    Lat lat;
    {
        static const int primes[7] = {2, 3, 5, 7, 11, 13, 17};
        for (int i = 0; i < 7; ++i) {
            double s = sqrt((double)primes[i]);
            lat.G[i] = (uint32_t)floor((s - floor(s)) * 4294967296.0);
        }
    }
    {
        ProfScope ps("adj_cell", st);
        {
            ProfScope p1("adj_prep", st);
            k_adj_prep<<<(unsigned)((ncell + 127) / 128), 128, 0, st>>>(g, S15, slot, clist, ncell, dL_dlcp, isovalue,
                                                                        opts->jitter, opts->skip_eps, pt, arec);
        }
        {
            ProfScope p2("adj_sample", st);
            k_adj_sample<<<(unsigned)((ncell + 7) / 8), 256, 0, st>>>(arec, clist, ncell, dL_dlcp, opts->n_samples,
                                                                      opts->seed, lat, ared);
        }
        ProfScope p3("adj_chol", st);
        k_adj_chol<<<(unsigned)((ncell + 127) / 128), 128, 0, st>>>(g, S15, slot, clist, ncell, dL_dlcp, isovalue,
                                                                    opts->jitter, opts->skip_eps, opts->n_samples, pt,
                                                                    arec, ared, G16);
    }
    note_launch();
    note_launch();
    note_launch();
    // t = W^T g_mu
    k_wt_vec<<<dim3((unsigned)((mp + 255) / 256), (unsigned)nchunks), 256, 0, st>>>(W, G16, npts, mp, chunk, tp);
    note_launch();
    k_sum_rows<<<(unsigned)((mp + 255) / 256), 256, 0, st>>>(tp, nchunks, mp, t);
    note_launch();
    // Zh rows, R = Zh^T W (split over points), M = R - v t^T, N = L^-T M L^-1
    {
        ProfScope ps("adj_zhat", st);
        if (use_oz) k_zhat_ff<<<(unsigned)((npts + 7) / 8), 256, 0, st>>>(g, plist, npts, slot, Wff, G16, mp, Zh);
        else k_zhat<<<(unsigned)((npts + 7) / 8), 256, 0, st>>>(g, plist, npts, slot, W, G16, mp, Zh);
    }
    note_launch();
    // R splits: 19 x (mp/64) x (mp/128) tiles = 608 CTAs = 4 waves of 152 for mp = 512
    const int rsplits = use_oz ? 19 : splits;
    {
        ProfScope ps("adj_R", st);
        if (use_oz) GPR_TRY(oz_mul_tn(Zh, W, npts, m, mp, Rp, rsplits, st));
        else gemm64<true, false>(mp, mp, npts, Zh, mp, W, mp, Rp, mp, splits, st);
    }
    k_sum_rows<<<(unsigned)((mp * mp + 255) / 256), 256, 0, st>>>(Rp, rsplits, mp * mp, R);
    note_launch();
    k_form_m<<<(unsigned)((mp * mp + 255) / 256), 256, 0, st>>>(R, M->vy, t, m, mp);
    note_launch();
    // Linv (mb x mb) viewed with leading dimension mb; products restricted to the m x m block
    gemm64<false, true>(m, m, m, R, mp, M->Linv, mb, T1, mp, 1, st);     // T1 = M L^-1
    gemm64<true, false>(m, m, m, M->Linv, mb, T1, mp, Nm, mp, 1, st);    // N = L^-T T1
    k_trace<<<(unsigned)num_sms() * 2, 256, 0, st>>>(M->X, m, M->kp, Nm, mp, acc);
    note_launch();
    // Z = Zh L^-1 into the W buffer (W no longer needed), then the per-point terms
    {
        ProfScope ps("adj_Z", st);
        if (use_oz) GPR_TRY(oz_mul_linv(M, Zh, npts, mp, W, mp, st));
        else gemm64<false, true>(npts, m, m, Zh, mp, M->Linv, mb, W, mp, 1, st);
    }
    KdPrior kdp;
    for (int e = 0; e < 13; ++e) {
        double b[3];
        for (int d = 0; d < 3; ++d) b[d] = kOff13[e][d] * g.h[d];
        double r2 = 0.0;
        for (int d = 0; d < 3; ++d) r2 += (b[d] / M->kp.ell[d]) * (b[d] / M->kp.ell[d]);
        for (int d = 0; d < 3; ++d) {
            double t2 = (b[d] / M->kp.ell[d]) * (b[d] / M->kp.ell[d]);
            if (M->kp.kind == GPR_K_SE) kdp.k[e][d] = M->kp.sf2 * exp(-0.5 * r2) * t2;
            else {
                double r = sqrt(r2), s5r = sqrt(5.0) * r;
                kdp.k[e][d] = (5.0 / 3.0) * M->kp.sf2 * (1.0 + s5r) * exp(-s5r) * t2;
            }
        }
    }
    {
        ProfScope ps("adj_points", st);
        if (M->kp.kind == GPR_K_SE) {
            k_sqdist_tables<<<(unsigned)((te + 255) / 256), 256, 0, st>>>(M->X, m, mp, M->kp, g, Q64, Qff);
            k_point_terms_se_ff<<<(unsigned)((npts + 7) / 8), 256, 0, st>>>(g, plist, npts, Tff, Qff, m, M->alpha_ff,
                                                                            W, mp, G16, kdp, acc);
            note_launch();
        } else {
            k_point_terms<<<(unsigned)((npts + 7) / 8), 256, 0, st>>>(g, plist, npts, M->X, m, M->kp, M->alpha, W, mp,
                                                                      G16, kdp, acc);
        }
    }
    note_launch();
    k_dy<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(M->Linv, mb, t, m, dy);
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    GPR_CUDA_TRY(cudaMemcpyAsync(dL_dy, dy, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    GPR_CUDA_TRY(cudaMemcpyAsync(h_out, acc, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
    GPR_CUDA_TRY(cudaStreamSynchronize(st));
    memcpy(dL_dloglen, h_out, sizeof h_out);
    return GPR_OK;
}

extern "C" gpr_status gpr_lcp_backward(gpr_model *M, const gpr_grid *grid, double isovalue,
                                       const gpr_lcp_options *opts, const float *dL_dlcp, double *dL_dy,
                                       double *dL_dloglen, void *stream)
{
    TraceRange trace_("gpr_lcp_backward");
    if (!M || !grid_valid(grid) || !opts_valid(opts) || !dL_dlcp || !dL_dy || !dL_dloglen || !isfinite(isovalue))
        return GPR_ERR_ARG;
    if (opts->est != GPR_EST_SOV_QMC) return GPR_ERR_UNSUPPORTED;  // the indicator MC has no useful gradient
    if (M->sgpr) return GPR_ERR_UNSUPPORTED;                        // written for plain GPR models
    return lcp_backward(M, grid, isovalue, opts, dL_dlcp, nullptr, dL_dy, dL_dloglen, (cudaStream_t)stream);
}

extern "C" gpr_status gpr_lcp_backward_adaptive(gpr_model *M, const gpr_grid *grid, double isovalue,
                                                int32_t max_depth, const gpr_lcp_options *opts, const float *dL_dlcp,
                                                double *dL_dy, double *dL_dloglen, void *stream)
{
    TraceRange trace_("gpr_lcp_backward_adaptive");
    if (!M || !grid_valid(grid) || !opts_valid(opts) || !dL_dlcp || !dL_dy || !dL_dloglen || !isfinite(isovalue))
        return GPR_ERR_ARG;
    if (max_depth < 0 || max_depth > 20) return GPR_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (((int64_t)1 << max_depth) < (int64_t)grid->n[d] - 1) return GPR_ERR_ARG;
    if (opts->est != GPR_EST_SOV_QMC || M->sgpr) return GPR_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    GridDev g = make_grid(grid);
    uint8_t *leaf = nullptr;
    GPR_CUDA_TRY(cudaMallocAsync((void **)&leaf, (size_t)g.ncells(), st));
    gpr_status s = octree_leaf_mask(M, grid, isovalue, max_depth, opts, leaf, st);
    if (s == GPR_OK) s = lcp_backward(M, grid, isovalue, opts, dL_dlcp, leaf, dL_dy, dL_dloglen, st);
    cudaError_t e = cudaFreeAsync(leaf, st);
    if (s == GPR_OK && e != cudaSuccess) {
        gpr_internal_note_cuda_error(e, "cudaFreeAsync(leaf)", __LINE__);
        s = GPR_ERR_CUDA;
    }
    return s;
}
