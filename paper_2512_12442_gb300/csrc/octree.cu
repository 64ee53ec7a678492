// Algorithm 1 (octree adaptive query, Sec. 5.3) on the device, level by level, followed by
// the leaf reconstruction of Sec. 5.3's last paragraph: the cells of S get the dense
// method's LCP, every other cell 0.
//
// Per level: (1) p-test on the observations inside each node (Sec. 5.3: p1 = max P(Y_i<t),
// p2 = max P(Y_i>t) over the node's observations, with the latent posterior at the
// observations); (2) the regional upper bound 1 - B_l^d - B_u^d (Eq. upper_bound, Sec. 5.1)
// for the remaining nodes, B = min over the node of Phi(+-(t - mu)/sigma): exact over the
// grid points when a node has <= 3 points per axis, otherwise a 3x3x3 lattice start plus T
// projected gradient steps (our reading of the paper's L-BFGS-B minimiser); (3) compaction
// of the subdivided nodes into the next frontier (or into S at the last level).
// Evaluations of mu, sigma and their gradients run in FP32 on the whitened form.
#include <math.h>
#include <string.h>

#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

constexpr int64_t kEvalChunk = 131072;  // evaluation points per pipeline pass

// g = (theta - mu)/sigma and grad g at each evaluation point (thread per point) from the tensor-core
// evaluation's sums: |w|^2 and (grad) w . L^-1 d_k k per 64-column group, var = sf2 - |w|^2,
// grad var = -2 w . L^-1 d_k k; mu and grad mu = sum_j dk_j alpha_j as float-float pairs (summed
// error-free in the generating warps).  Without grad the gradient is 0.
__global__ void k_eval_reduce(float sf2, const float *partial, int nN, bool grad, int64_t count, double theta,
                              float4 *out, float *moments)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= count) return;
    const float *mo = partial + count * 4 * nN + 8 * q;
    const int T = grad ? 4 : 1;
    float wsq = 0.f, gv[3] = {0.f, 0.f, 0.f}, gm[3] = {0.f, 0.f, 0.f};
    for (int g2 = 0; g2 < nN; ++g2) {
        wsq += partial[(q * T) * nN + g2];
        if (grad)
            for (int dI = 0; dI < 3; ++dI) gv[dI] += partial[(q * T + 1 + dI) * nN + g2];
    }
    for (int dI = 0; dI < 3; ++dI) {
        gv[dI] *= -2.f;
        if (grad) gm[dI] = mo[2 + 2 * dI] + mo[3 + 2 * dI];
    }
    const float mu = mo[0] + mo[1];
    float var = sf2 - wsq;
    const float fl = 1e-12f * sf2;
    if (!(var > fl)) var = fl;
    const float sd = sqrtf(var);
    const float gg = (float)(theta - (double)mu) / sd;
    float4 o;
    o.x = gg;
    o.y = -gm[0] / sd - gg * gv[0] / (2.f * var);
    o.z = -gm[1] / sd - gg * gv[1] / (2.f * var);
    o.w = -gm[2] / sd - gg * gv[2] / (2.f * var);
    out[q] = o;
    if (moments) {  // test hook: mu, var (unfloored), grad mu, grad var
        float *m8 = moments + 8 * q;
        m8[0] = mu;
        m8[1] = sf2 - wsq;
        for (int dI = 0; dI < 3; ++dI) {
            m8[2 + dI] = gm[dI];
            m8[5 + dI] = gv[dI];
        }
    }
}

struct Geom {
    int64_t p0[3], p1[3];
    double blo[3], bhi[3];
};

// Cells per axis of a node at level l: 2^(D - l) in the octree; in the K-D tree (Sec. 9), which
// halves x, y, z in turn, axis d has been halved floor((l + 2 - d) / 3) times by level l (0 .. 3D).
__host__ __device__ __forceinline__ int64_t axis_extent(int D, int l, int kd, int d)
{
    return (int64_t)1 << (D - (kd ? (l + 2 - d) / 3 : l));
}

__device__ __forceinline__ Geom node_geom(const GridDev &g, int D, int l, int kd, int64_t code)
{
    Geom G;
    int64_t ijk[3] = {code & 0x1FFFFF, (code >> 21) & 0x1FFFFF, (code >> 42) & 0x1FFFFF};
    for (int d = 0; d < 3; ++d) {
        const int64_t s = axis_extent(D, l, kd, d);
        G.p0[d] = ijk[d] * s;
        G.p1[d] = (ijk[d] + 1) * s;
        if (G.p1[d] > g.n[d] - 1) G.p1[d] = g.n[d] - 1;
        G.blo[d] = g.lo[d] + (double)G.p0[d] * g.h[d];
        G.bhi[d] = g.lo[d] + (double)G.p1[d] * g.h[d];
    }
    return G;
}

__device__ __forceinline__ bool is_small(const Geom &G)
{
    return G.p1[0] - G.p0[0] <= 2 && G.p1[1] - G.p0[1] <= 2 && G.p1[2] - G.p0[2] <= 2;
}

__device__ __forceinline__ double log_norm_cdf(double gg)
{
    if (gg >= 0.0) return log1p(-0.5 * erfc(gg * 0.70710678118654752440));
    double c = 0.5 * erfc(-gg * 0.70710678118654752440);
    if (c > 0.0) return log(c);
    return -0.5 * gg * gg - log(-gg * 2.5066282746310005024);
}

__device__ __forceinline__ double bound_of(int sides, double dcount, double glo, double ghi)
{
    double lBlo = (sides & 1) ? log_norm_cdf(glo) : -INFINITY;
    double lBhi = (sides & 2) ? log_norm_cdf(ghi) : -INFINITY;
    if (sides == 3) return -expm1(dcount * lBlo) - exp(dcount * lBhi);
    if (sides == 1) return -expm1(dcount * lBlo);
    return -expm1(dcount * lBhi);
}

// The same in FP32, for bounds from FP32-class values of g (the per-point table and the tensor-core
// evaluations): FP64 erfc, log and expm1 per node cost the FP64 pipe more than the rest of those
// kernels, and add no accuracy to FP32 inputs.  Below Phi = 1e-37 the leading asymptotic term.
__device__ __forceinline__ float log_norm_cdf32(float gg)
{
    if (gg >= 0.0f) return log1pf(-0.5f * erfcf(gg * 0.70710678f));
    const float c = 0.5f * erfcf(-gg * 0.70710678f);
    if (c > 1e-37f) return logf(c);
    return -0.5f * gg * gg - logf(-gg * 2.5066283f);
}

__device__ __forceinline__ float bound_of32(int sides, float dcount, float glo, float ghi)
{
    const float lBlo = (sides & 1) ? log_norm_cdf32(glo) : -INFINITY;
    const float lBhi = (sides & 2) ? log_norm_cdf32(ghi) : -INFINITY;
    if (sides == 3) return -expm1f(dcount * lBlo) - expf(dcount * lBhi);
    if (sides == 1) return -expm1f(dcount * lBlo);
    return -expm1f(dcount * lBhi);
}

// Observation flags for the p-test: bit0 = P(Y_i < theta) > alpha, bit1 = P(Y_i > theta) > alpha.
__global__ void k_obs_flags(const double *mu_obs, const double *var_obs, int64_t m, double theta, double alpha,
                            uint8_t *flags)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    double sd = sqrt(var_obs[i]);
    bool lo = normcdf((theta - mu_obs[i]) / sd) > alpha;
    bool hi = normcdf((mu_obs[i] - theta) / sd) > alpha;
    flags[i] = (uint8_t)((lo ? 1 : 0) | (hi ? 2 : 0));
}

// p-test (warp per node).  decision: 1 = subdivide (p1 > alpha and p2 > alpha), 0 = bound needed;
// sides: bit0 lower bound B_l, bit1 upper bound B_u.
// p-test flags of the octree's nodes at every level, as a pyramid of bytes (bit 2: the node
// holds an observation, bit 0 / bit 1: one with P(Y_i < t) > alpha / P(Y_i > t) > alpha).  The
// finest level has one word per cell; an observation marks every cell whose closed box holds
// it (two per axis on a shared face), with the box edges lo + c h of the node geometry, so the
// OR over a node's cells is exactly "some observation lies in the node's closed box".
struct Pyramid {
    int64_t off[21];     // byte offset of level l in the level buffer
    int32_t dim[21][3];  // nodes per axis at level l: ceil((n_d - 1) / 2^(D - l))
};

__global__ void k_obs_cells(GridDev g, const double *X, int64_t m, const uint8_t *flags, uint32_t *fine)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    int64_t cand[3][2];
    int cnt[3];
    for (int d = 0; d < 3; ++d) {
        const double x = X[3 * i + d];
        const int64_t ncd = g.n[d] - 1;
        const double t = (x - g.lo[d]) / g.h[d];
        cnt[d] = 0;
        if (!(t >= -2.0 && t <= (double)ncd + 2.0)) return;  // outside the grid (or NaN)
        const int64_t c = (int64_t)floor(t);
        for (int64_t cc = c - 1; cc <= c + 1; ++cc) {
            if (cc < 0 || cc >= ncd || cnt[d] == 2) continue;
            if (x >= g.lo[d] + (double)cc * g.h[d] && x <= g.lo[d] + (double)(cc + 1) * g.h[d]) cand[d][cnt[d]++] = cc;
        }
        if (cnt[d] == 0) return;
    }
    const uint32_t v = 4u | (flags[i] & 3u);
    const int64_t cx = g.n[0] - 1, cy = g.n[1] - 1;
    for (int a = 0; a < cnt[0]; ++a)
        for (int b = 0; b < cnt[1]; ++b)
            for (int c = 0; c < cnt[2]; ++c) atomicOr(&fine[cand[0][a] + cx * (cand[1][b] + cy * cand[2][c])], v);
}

__global__ void k_cells_to_bytes(const uint32_t *fine, int64_t n, uint8_t *out)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < n) out[q] = (uint8_t)fine[q];
}

template <typename TC>
__global__ void k_pyr_level(const TC *child, int32_t c0, int32_t c1, int32_t c2, uint8_t *parent, int32_t p0,
                            int32_t p1, int32_t p2)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)p0 * p1 * p2) return;
    const int64_t i = q % p0, j = (q / p0) % p1, k = q / ((int64_t)p0 * p1);
    uint32_t v = 0;
    for (int b = 0; b < 8; ++b) {
        const int64_t a0 = 2 * i + (b & 1), a1 = 2 * j + ((b >> 1) & 1), a2 = 2 * k + (b >> 2);
        if (a0 < c0 && a1 < c1 && a2 < c2) v |= (uint32_t)child[a0 + (int64_t)c0 * (a1 + (int64_t)c1 * a2)];
    }
    parent[q] = (uint8_t)v;
}

__global__ void k_ptest(GridDev g, int D, int l, int kd, const int64_t *nodes, int64_t count, const uint8_t *lvl,
                        int32_t d0, int32_t d1, int32_t d2, int8_t *decision, int8_t *sides)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= count) return;
    const int64_t code = nodes[q];
    const int64_t ijk[3] = {code & 0x1FFFFF, (code >> 21) & 0x1FFFFF, (code >> 42) & 0x1FFFFF};
    // `lvl` is the pyramid level of the node's smallest extent; a K-D node spans 1, 2 or 4 of its
    // entries (2^(q_0 - q_d) along axis d, q_d the halvings of axis d)
    int64_t span[3] = {1, 1, 1}, base[3];
    for (int d = 0; d < 3; ++d) {
        if (kd) span[d] = axis_extent(D, l, kd, d) / axis_extent(D, l, kd, 0);
        base[d] = ijk[d] * span[d];
    }
    uint32_t v = 0;
    for (int64_t c = 0; c < span[2]; ++c)
        for (int64_t b = 0; b < span[1]; ++b)
            for (int64_t a = 0; a < span[0]; ++a) {
                const int64_t ii = base[0] + a, jj = base[1] + b, kk = base[2] + c;
                if (ii < d0 && jj < d1 && kk < d2) v |= lvl[ii + (int64_t)d0 * (jj + (int64_t)d1 * kk)];
            }
    const bool any = v & 4, lo = v & 1, hi = v & 2;
    if (any && lo && hi) {
        decision[q] = 1;
        sides[q] = 0;
    } else {
        decision[q] = 0;
        sides[q] = (!any || (!lo && !hi)) ? 3 : (!hi ? 1 : 2);
    }
}

// Flags the grid points of pending small nodes whose mean/variance is not yet in the table.
__global__ void k_mark_small_points(GridDev g, int D, int l, int kd, const int64_t *nodes, int64_t count,
                                    const int8_t *decision, const uint8_t *have, uint8_t *need)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= count || decision[q] != 0) return;
    Geom G = node_geom(g, D, l, kd, nodes[q]);
    if (!is_small(G)) return;
    for (int64_t c = G.p0[2]; c <= G.p1[2]; ++c)
        for (int64_t b = G.p0[1]; b <= G.p1[1]; ++b)
            for (int64_t a = G.p0[0]; a <= G.p1[0]; ++a) {
                int64_t p = a + (int64_t)g.n[0] * (b + (int64_t)g.n[1] * c);
                if (!have[p]) need[p] = 1;
            }
}

__global__ void k_scatter_mv(const int64_t *pts, int64_t count, const float *mean, const float *var, float2 *mv,
                             uint8_t *have)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    int64_t p = pts[i];
    mv[p] = make_float2(mean[i], var[i]);
    __threadfence();  // the value before its flag, for readers on other streams
    have[p] = 1;
}

// Exact minimum over the grid points of small pending nodes -> bound -> decision.
__global__ void k_small_bound(GridDev g, int D, int l, int kd, const int64_t *nodes, int64_t count, const float2 *mv,
                              double theta, double alpha, double sf2, int8_t *decision, const int8_t *sides,
                              double *bound)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= count || decision[q] != 0) return;
    Geom G = node_geom(g, D, l, kd, nodes[q]);
    if (!is_small(G)) return;
    // g per point in FP32 (the table holds FP32-class values; FP64 division and square roots per
    // point cost the FP64 pipe more than the rest of the kernel); the bound itself in FP64
    const float thf = (float)theta, fl = (float)(1e-12 * sf2);
    float gmin = INFINITY, gmax = -INFINITY;
    for (int64_t c = G.p0[2]; c <= G.p1[2]; ++c)
        for (int64_t b = G.p0[1]; b <= G.p1[1]; ++b)
            for (int64_t a = G.p0[0]; a <= G.p1[0]; ++a) {
                const float2 v = mv[a + (int64_t)g.n[0] * (b + (int64_t)g.n[1] * c)];
                const float gg = (thf - v.x) * rsqrtf(fmaxf(v.y, fl));
                gmin = fminf(gmin, gg);
                gmax = fmaxf(gmax, gg);
            }
    const float dcount = (float)((G.p1[0] - G.p0[0] + 1) * (G.p1[1] - G.p0[1] + 1) * (G.p1[2] - G.p0[2] + 1));
    const double bnd = (double)bound_of32(sides[q], dcount, gmin, -gmax);
    bound[q] = bnd;
    decision[q] = bnd > alpha ? 2 : 0;
}

// Pending large nodes -> compact list (positions in the frontier).
__global__ void k_flag_large(GridDev g, int D, int l, int kd, const int64_t *nodes, int64_t count, const int8_t *decision,
                             uint8_t *flag)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= count) return;
    bool f = false;
    if (decision[q] == 0) f = !is_small(node_geom(g, D, l, kd, nodes[q]));
    flag[q] = f ? 1 : 0;
}

// Lattice points (3x3x3 per node; corners, edge/face midpoints, centre, x fastest).
__global__ void k_lattice_points(GridDev g, int D, int l, int kd, const int64_t *nodes, const int64_t *pend,
                                 const int64_t *ulist, int64_t first, int64_t cnt, double *xyz)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= cnt) return;
    int64_t gi = first + e, q = ulist[gi / 27];
    int t = (int)(gi % 27);
    Geom G = node_geom(g, D, l, kd, nodes[pend[q]]);
    int id[3] = {t % 3, (t / 3) % 3, t / 9};
    for (int d = 0; d < 3; ++d) xyz[3 * e + d] = G.blo[d] + 0.5 * (double)id[d] * (G.bhi[d] - G.blo[d]);
}

// A node is grid-aligned when its 3x3x3 lattice lies on grid points (even extent per axis).
__device__ __forceinline__ bool lattice_aligned(const Geom &G)
{
    return ((G.p1[0] - G.p0[0]) % 2 == 0) && ((G.p1[1] - G.p0[1]) % 2 == 0) && ((G.p1[2] - G.p0[2]) % 2 == 0);
}

__device__ __forceinline__ int64_t lattice_point(const GridDev &g, const Geom &G, int t)
{
    int id[3] = {t % 3, (t / 3) % 3, t / 9};
    int64_t q[3];
    for (int d = 0; d < 3; ++d) q[d] = G.p0[d] + id[d] * ((G.p1[d] - G.p0[d]) / 2);
    return q[0] + (int64_t)g.n[0] * (q[1] + (int64_t)g.n[1] * q[2]);
}

// Marks the lattice grid points of aligned pending large nodes that the table lacks; flags the
// unaligned nodes (their lattice is evaluated point by point).
__global__ void k_mark_lattice(GridDev g, int D, int l, int kd, const int64_t *nodes, const int64_t *pend, int64_t npend,
                               const uint8_t *have, uint8_t *need, uint8_t *unaligned)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= npend) return;
    Geom G = node_geom(g, D, l, kd, nodes[pend[q]]);
    bool al = lattice_aligned(G);
    unaligned[q] = al ? 0 : 1;
    if (!al) return;
    for (int t = 0; t < 27; ++t) {
        int64_t p = lattice_point(g, G, t);
        if (!have[p]) need[p] = 1;
    }
}

// g = (theta - mu)/sigma at the 27 lattice points of aligned nodes, from the table.
__global__ void k_lattice_from_table(GridDev g, int D, int l, int kd, const int64_t *nodes, const int64_t *pend,
                                     int64_t npend, const uint8_t *unaligned, const float2 *mv, double theta,
                                     double sf2, float4 *lat)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= npend * 27) return;
    int64_t q = e / 27;
    if (unaligned[q]) return;
    Geom G = node_geom(g, D, l, kd, nodes[pend[q]]);
    float2 v = mv[lattice_point(g, G, (int)(e % 27))];
    double var = fmax((double)v.y, 1e-12 * sf2);
    lat[e] = make_float4((float)((theta - (double)v.x) / sqrt(var)), 0.f, 0.f, 0.f);
}

// Best lattice point per node and side (lowest g; first in x-fastest order on ties).
struct MinState {
    double x[2][3];
    float g[2];
    float grad[2][3];
};

__global__ void k_scatter_lattice(const float4 *ev, const int64_t *ulist, int64_t first, int64_t cnt, float4 *lat)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= cnt) return;
    int64_t gi = first + e;
    lat[ulist[gi / 27] * 27 + gi % 27] = ev[e];
}

// Start points (best lattice point per side) as evaluation points, for their gradients.
__global__ void k_start_points(const MinState *ms, const int64_t *act, int64_t first, int64_t cnt, double *xyz)
{
    int64_t le = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (le >= cnt) return;
    const int64_t e = act[first + le], q = e / 2;
    const int side = (int)(e % 2);
    for (int d = 0; d < 3; ++d) xyz[3 * le + d] = ms[q].x[side][d];
}

__global__ void k_start_grad(const float4 *ev, const int64_t *act, int64_t first, int64_t cnt, MinState *ms)
{
    int64_t le = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (le >= cnt) return;
    const int64_t e = act[first + le], q = e / 2;
    const int side = (int)(e % 2);
    float sg = side == 0 ? 1.f : -1.f;
    ms[q].g[side] = sg * ev[le].x;
    ms[q].grad[side][0] = sg * ev[le].y;
    ms[q].grad[side][1] = sg * ev[le].z;
    ms[q].grad[side][2] = sg * ev[le].w;
}

__global__ void k_lattice_best(const float4 *ev, int64_t npend, MinState *ms)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= npend) return;
    MinState s;
    for (int side = 0; side < 2; ++side) {
        float sg = side == 0 ? 1.f : -1.f;
        int best = 0;
        float bg = sg * ev[q * 27].x;
        for (int t = 1; t < 27; ++t) {
            float v = sg * ev[q * 27 + t].x;
            if (v < bg) { bg = v; best = t; }
        }
        float4 e = ev[q * 27 + best];
        s.g[side] = bg;
        s.grad[side][0] = sg * e.y;
        s.grad[side][1] = sg * e.z;
        s.grad[side][2] = sg * e.w;
        s.x[side][0] = best % 3;  // lattice indices; converted to coordinates by the caller kernel
        s.x[side][1] = (best / 3) % 3;
        s.x[side][2] = best / 9;
    }
    ms[q] = s;
}

__global__ void k_lattice_coords(GridDev g, int D, int l, int kd, const int64_t *nodes, const int64_t *pend, int64_t npend,
                                 MinState *ms)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= npend) return;
    Geom G = node_geom(g, D, l, kd, nodes[pend[q]]);
    for (int side = 0; side < 2; ++side)
        for (int d = 0; d < 3; ++d) ms[q].x[side][d] = G.blo[d] + 0.5 * ms[q].x[side][d] * (G.bhi[d] - G.blo[d]);
}

// Candidate of projected step t for every (node, side): x' = clamp(x + eta_t w u/|u|_inf), u = -grad g * w.
__global__ void k_candidates(GridDev g, int D, int l, int kd, const int64_t *nodes, const int64_t *pend, const int64_t *act,
                             const MinState *ms, int step, int64_t first, int64_t cnt, double *xyz, uint8_t *valid)
{
    int64_t le = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (le >= cnt) return;
    const int64_t e = act[first + le], q = e / 2;
    const int side = (int)(e % 2);
    Geom G = node_geom(g, D, l, kd, nodes[pend[q]]);
    double w[3], u[3], un = 0.0;
    for (int d = 0; d < 3; ++d) {
        w[d] = G.bhi[d] - G.blo[d];
        u[d] = -(double)ms[q].grad[side][d] * w[d];
        un = fmax(un, fabs(u[d]));
    }
    double eta = 0.25 * ldexp(1.0, -step);
    for (int d = 0; d < 3; ++d) {
        double xn = un > 0.0 ? ms[q].x[side][d] + eta * w[d] * u[d] / un : ms[q].x[side][d];
        xyz[3 * le + d] = xn < G.blo[d] ? G.blo[d] : (xn > G.bhi[d] ? G.bhi[d] : xn);
    }
    valid[le] = un > 0.0 ? 1 : 0;
}

__global__ void k_accept(const double *xyz, const uint8_t *valid, const float4 *ev, const int64_t *act, int64_t first,
                         int64_t cnt, MinState *ms)
{
    int64_t le = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (le >= cnt) return;
    const int64_t e = act[first + le], q = e / 2;
    const int side = (int)(e % 2);
    if (!valid[le]) return;
    float sg = side == 0 ? 1.f : -1.f;
    float v = sg * ev[le].x;
    if (v < ms[q].g[side]) {
        ms[q].g[side] = v;
        ms[q].grad[side][0] = sg * ev[le].y;
        ms[q].grad[side][1] = sg * ev[le].z;
        ms[q].grad[side][2] = sg * ev[le].w;
        for (int d = 0; d < 3; ++d) ms[q].x[side][d] = xyz[3 * le + d];
    }
}

// Bound of each listed pending node from its current minima (act: codes 2q + side of pending
// nodes q; nullptr = every pending node).  With `active` (two flags per pending node), nodes whose
// bound already exceeds alpha are decided (subdivide: the minimiser only lowers g, which only
// raises the bound) and, for the others, each side the bound depends on is flagged for the
// minimiser: a side outside the p-test's sides, or whose B^d is already below 1e-30 (further
// descent moves the bound by less than that), is not minimised.
__global__ void k_large_bound(GridDev g, int D, int l, int kd, const int64_t *nodes, const int64_t *pend, const int64_t *act,
                              int64_t cnt, const MinState *ms, double alpha, int8_t *decision, const int8_t *sides,
                              double *bound, uint8_t *active)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int64_t q = act ? act[t] / 2 : t;
    int64_t node = pend[q];
    Geom G = node_geom(g, D, l, kd, nodes[node]);
    const float dcount = (float)((G.p1[0] - G.p0[0] + 1) * (G.p1[1] - G.p0[1] + 1) * (G.p1[2] - G.p0[2] + 1));
    const double bnd = (double)bound_of32(sides[node], dcount, ms[q].g[0], ms[q].g[1]);
    bound[node] = bnd;
    decision[node] = bnd > alpha ? 2 : 0;
    if (active) {
        for (int sd = 0; sd < 2; ++sd) {
            const bool need = bnd <= alpha && (sides[node] & (1 << sd)) &&
                              dcount * log_norm_cdf32(ms[q].g[sd]) > -69.0f;  // B^d > 1e-30
            active[2 * q + sd] = need ? 1 : 0;
        }
    }
}

// Subdivided nodes -> children (next frontier) or, at the last level, cells of S.
__global__ void k_children(GridDev g, int D, int l, int kd, const int64_t *nodes, int64_t count, const int8_t *decision,
                           int64_t *next, unsigned long long *nnext, uint8_t *leaf, unsigned long long *nsub)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool sub = q < count && decision[q] > 0;
    unsigned mask = __ballot_sync(0xffffffffu, sub);
    if ((threadIdx.x & 31) == 0 && mask) atomicAdd(nsub, (unsigned long long)__popc(mask));
    if (!sub) return;
    int64_t code = nodes[q];
    int64_t i = code & 0x1FFFFF, j = (code >> 21) & 0x1FFFFF, k = (code >> 42) & 0x1FFFFF;
    if (l == (kd ? 3 * D : D)) {
        leaf[i + (int64_t)(g.n[0] - 1) * (j + (int64_t)(g.n[1] - 1) * k)] = 1;
        return;
    }
    int64_t sc[3];
    for (int d = 0; d < 3; ++d) sc[d] = axis_extent(D, l + 1, kd, d);
    int64_t out[8];
    int c = 0;
    // octree: 8 children; K-D tree: 2 children along the axis this level halves (l mod 3)
    const int nch = kd ? 2 : 8, ax = l % 3;
    for (int b = 0; b < nch; ++b) {
        int64_t ci, cj, ck;
        if (kd) {
            ci = ax == 0 ? 2 * i + b : i;
            cj = ax == 1 ? 2 * j + b : j;
            ck = ax == 2 ? 2 * k + b : k;
        } else {
            ci = 2 * i + (b & 1); cj = 2 * j + ((b >> 1) & 1); ck = 2 * k + ((b >> 2) & 1);
        }
        if (ci * sc[0] < g.n[0] - 1 && cj * sc[1] < g.n[1] - 1 && ck * sc[2] < g.n[2] - 1)
            out[c++] = ci | (cj << 21) | (ck << 42);
    }
    unsigned long long base = atomicAdd(nnext, (unsigned long long)c);
    for (int t = 0; t < c; ++t) next[base + t] = out[t];
}

unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---- Local model of Sec. 5.2 (beta >= 0): the bound of a node is minimised on the model
// restricted to the observations M' inside the node box enlarged by beta * l_d per axis.

__device__ __forceinline__ bool in_local_box(const Geom &G, const double *x, double beta, const KernParams &kp)
{
    for (int d = 0; d < 3; ++d)
        if (x[d] < G.blo[d] - beta * kp.ell[d] || x[d] > G.bhi[d] + beta * kp.ell[d]) return false;
    return true;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Pending nodes whose local set is a strict subset of M: flag them (decision 5 keeps the full-model
// kernels off them), track the largest local set, and record each set's size and an
// order-independent hash of its members (nodes with equal sets share one factorisation).
__global__ void k_local_flag(GridDev g, int D, int l, int kd, const int64_t *nodes, int64_t count, int8_t *decision,
                             const double *X, int64_t m, double beta, KernParams kp, uint8_t *flag,
                             unsigned long long *cmax, uint64_t *sig, int32_t *cnt)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= count) return;
    flag[q] = 0;
    if (decision[q] != 0) return;
    Geom G = node_geom(g, D, l, kd, nodes[q]);
    int64_t c = 0;
    uint64_t h = 0;
    for (int64_t i = 0; i < m; ++i)
        if (in_local_box(G, X + 3 * i, beta, kp)) {
            ++c;
            h += mix64((uint64_t)i * 0x9E3779B97F4A7C15ULL + 1);
        }
    if (c == m) return;
    flag[q] = 1;
    decision[q] = 5;
    sig[q] = h;
    cnt[q] = (int32_t)c;
    atomicMax(cmax, (unsigned long long)c);
}

__global__ void k_gather_local(const int64_t *list, int64_t nl, const uint64_t *sig, const int32_t *cnt,
                               uint64_t *osig, int32_t *ocnt)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nl) return;
    osig[t] = sig[list[t]];
    ocnt[t] = cnt[list[t]];
}

__device__ __forceinline__ double kval64(const KernParams &kp, const double *a, const double *b)
{
    double r2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        double t = (a[d] - b[d]) / kp.ell[d];
        r2 += t * t;
    }
    if (kp.kind == GPR_K_SE) return kp.sf2 * exp(-0.5 * r2);
    double r = sqrt(r2), s5r = 2.2360679774997896964 * r;
    return kp.sf2 * (1.0 + s5r + (5.0 / 3.0) * r2) * exp(-s5r);
}

// k(x, b) and d k(x, b) / d x.
__device__ __forceinline__ double kgrad64(const KernParams &kp, const double *x, const double *b, double gr[3])
{
    double r2 = 0.0, dd[3];
    for (int d = 0; d < 3; ++d) {
        dd[d] = x[d] - b[d];
        double t = dd[d] / kp.ell[d];
        r2 += t * t;
    }
    if (kp.kind == GPR_K_SE) {
        double k = kp.sf2 * exp(-0.5 * r2);
        for (int d = 0; d < 3; ++d) gr[d] = -k * dd[d] / (kp.ell[d] * kp.ell[d]);
        return k;
    }
    double r = sqrt(r2), s5r = 2.2360679774997896964 * r, e = exp(-s5r);
    double c = -(5.0 / 3.0) * kp.sf2 * (1.0 + s5r) * e;
    for (int d = 0; d < 3; ++d) gr[d] = c * dd[d] / (kp.ell[d] * kp.ell[d]);
    return kp.sf2 * (1.0 + s5r + (5.0 / 3.0) * r2) * e;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct LocalModel {
    const double *X, *y, *A;  // A: SGPR A_M (m x m), nullptr for plain GPR
    int64_t m;
    KernParams kp;
    double diag;  // noise variance (plain GPR) or K_MM jitter (SGPR)
};

// Per-warp FP64 work space of the local kernel.
struct LocalWs {
    double *L, *A, *v, *al, *k, *dk, *w, *a, *t, *ca;
    int32_t *idx;
};

__device__ LocalWs local_ws(double *base, int32_t *ibase, int64_t warp, int64_t cmax, bool sgpr)
{
    const int64_t per = cmax * cmax * (sgpr ? 2 : 1) + 12 * cmax;
    double *p = base + warp * per;
    LocalWs W;
    W.L = p; p += cmax * cmax;
    W.A = sgpr ? p : nullptr; p += sgpr ? cmax * cmax : 0;
    W.v = p; p += cmax;
    W.al = p; p += cmax;
    W.k = p; p += cmax;
    W.dk = p; p += 3 * cmax;
    W.w = p; p += cmax;
    W.a = p; p += cmax;
    W.t = p; p += cmax;
    W.ca = p; p += cmax;
    W.idx = ibase + warp * cmax;
    return W;
}

// Forward solve x = L^-1 x in place (L column-major c x c, lower), warp-cooperative.
__device__ void fwd_solve(const double *L, int64_t c, double *x, int lane)
{
    for (int64_t j = 0; j < c; ++j) {
        __syncwarp();
        const double xj = x[j] / L[j + j * c];
        __syncwarp();
        if (lane == 0) x[j] = xj;
        for (int64_t r = j + 1 + lane; r < c; r += 32) x[r] -= L[r + j * c] * xj;
    }
    __syncwarp();
}

// Backward solve y = L^-T x (into y; x unchanged).
__device__ void bwd_solve(const double *L, int64_t c, const double *x, double *y, int lane)
{
    for (int64_t j = c - 1; j >= 0; --j) {
        double s = 0.0;
        for (int64_t r = j + 1 + lane; r < c; r += 32) s += L[r + j * c] * y[r];
        s = warp_sum(s);
        if (lane == 0) y[j] = (x[j] - s) / L[j + j * c];
        __syncwarp();
    }
}

// g = (theta - mu(x)) / sigma(x) on the local model, and (want_grad) its gradient.
__device__ double local_eval(const LocalModel &Mo, const LocalWs &W, int64_t c, const double *x, double theta,
                             bool want_grad, double grad[3], int lane)
{
    for (int64_t r = lane; r < c; r += 32) {
        double gr[3];
        const double kv = kgrad64(Mo.kp, x, Mo.X + 3 * W.idx[r], gr);
        W.k[r] = kv;
        W.w[r] = kv;
        for (int d = 0; d < 3; ++d) W.dk[3 * r + d] = gr[d];
    }
    __syncwarp();
    fwd_solve(W.L, c, W.w, lane);  // w = L'^-1 k
    double mu = 0.0, ww = 0.0;
    for (int64_t r = lane; r < c; r += 32) {
        mu += W.w[r] * W.v[r];
        ww += W.w[r] * W.w[r];
    }
    mu = warp_sum(mu);
    const double kxx = kval64(Mo.kp, x, x);
    double var;
    if (Mo.A) {
        // Eq. 1: var = k(x,x) - k^T a + a^T A' a, a = K'^-1 k
        bwd_solve(W.L, c, W.w, W.a, lane);
        for (int64_t r = lane; r < c; r += 32) {
            double s = 0.0;
            for (int64_t q = 0; q < c; ++q) s += W.A[r + q * c] * W.a[q];
            W.ca[r] = s;
        }
        __syncwarp();
        double ka = 0.0, aca = 0.0;
        for (int64_t r = lane; r < c; r += 32) {
            ka += W.k[r] * W.a[r];
            aca += W.a[r] * W.ca[r];
        }
        var = kxx - warp_sum(ka) + warp_sum(aca);
    } else {
        var = kxx - warp_sum(ww);
    }
    const double fl = 1e-12 * Mo.kp.sf2;
    if (!(var > fl)) var = fl;
    const double sd = sqrt(var), gl = (theta - mu) / sd;
    if (!want_grad) return gl;
    // P = Kt'^-1 k (plain) or a - K'^-1 A' a (SGPR); d var = -2 dk^T P, d mu = dk^T alpha'
    if (Mo.A) {
        for (int64_t r = lane; r < c; r += 32) W.t[r] = W.ca[r];
        __syncwarp();
        fwd_solve(W.L, c, W.t, lane);
        bwd_solve(W.L, c, W.t, W.w, lane);  // w = K'^-1 A' a
        for (int64_t r = lane; r < c; r += 32) W.t[r] = W.a[r] - W.w[r];
    } else {
        bwd_solve(W.L, c, W.w, W.t, lane);
    }
    __syncwarp();
    double gm[3] = {0, 0, 0}, gv[3] = {0, 0, 0};
    for (int64_t r = lane; r < c; r += 32)
        for (int d = 0; d < 3; ++d) {
            gm[d] += W.dk[3 * r + d] * W.al[r];
            gv[d] += -2.0 * W.dk[3 * r + d] * W.t[r];
        }
    for (int d = 0; d < 3; ++d) {
        gm[d] = warp_sum(gm[d]);
        gv[d] = warp_sum(gv[d]);
        grad[d] = -gm[d] / sd - gl * gv[d] / (2.0 * var);
    }
    __syncwarp();
    return gl;
}

// One warp per listed node: gather M', factor K' (FP64, left-looking by columns), then the same
// minimiser as the full-model path (exact over grid points for nodes of <= 3 points per axis; else
// the best of the 3x3x3 lattice and T projected steps per side), bound and decision.
__global__ void k_local_nodes(GridDev g, int D, int l, int kd, const int64_t *nodes, const int64_t *list, int64_t nl,
                              LocalModel Mo, double beta, double theta, double alpha, int T, const int8_t *sides,
                              int8_t *decision, double *bound, double *ws, int32_t *iws, int64_t cmax, int *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const LocalWs W = local_ws(ws, iws, warp, cmax, Mo.A != nullptr);
    for (int64_t t = warp; t < nl; t += nwarps) {
        const int64_t q = list[t];
        const Geom G = node_geom(g, D, l, kd, nodes[q]);
        // gather the local set (ascending observation index)
        int64_t c = 0;
        for (int64_t base = 0; base < Mo.m; base += 32) {
            const int64_t i = base + lane;
            const bool in = i < Mo.m && in_local_box(G, Mo.X + 3 * i, beta, Mo.kp);
            const unsigned msk = __ballot_sync(0xffffffffu, in);
            if (in) W.idx[c + __popc(msk & ((1u << lane) - 1))] = (int32_t)i;
            c += __popc(msk);
        }
        __syncwarp();
        // K' (column-major, lower) and, for SGPR, A'
        for (int64_t s2 = 0; s2 < c; ++s2)
            for (int64_t r = s2 + lane; r < c; r += 32)
                W.L[r + s2 * c] = kval64(Mo.kp, Mo.X + 3 * W.idx[r], Mo.X + 3 * W.idx[s2]) + (r == s2 ? Mo.diag : 0.0);
        if (Mo.A)
            for (int64_t s2 = 0; s2 < c; ++s2)
                for (int64_t r = lane; r < c; r += 32) W.A[r + s2 * c] = Mo.A[W.idx[r] * Mo.m + W.idx[s2]];
        __syncwarp();
        for (int64_t j = 0; j < c; ++j) {
            for (int64_t r = j + lane; r < c; r += 32) {
                double a = W.L[r + j * c];
                for (int64_t k = 0; k < j; ++k) a -= W.L[r + k * c] * W.L[j + k * c];
                W.t[r] = a;
            }
            __syncwarp();
            double piv = W.t[j];
            if (!(piv > 0.0)) {
                if (lane == 0) atomicCAS(status, 0, (int)GPR_ERR_NOT_PD);
                piv = 1e-300;
            }
            const double d = sqrt(piv);
            for (int64_t r = j + lane; r < c; r += 32) W.L[r + j * c] = r == j ? d : W.t[r] / d;
            __syncwarp();
        }
        // v' = L'^-1 y', alpha' = L'^-T v'  (y' = y or mu_M restricted to M')
        for (int64_t r = lane; r < c; r += 32) W.v[r] = Mo.y[W.idx[r]];
        __syncwarp();
        fwd_solve(W.L, c, W.v, lane);
        bwd_solve(W.L, c, W.v, W.al, lane);
        const int sd = sides[q];
        double gmin[2] = {INFINITY, INFINITY};
        double gr[3];
        const bool small = G.p1[0] - G.p0[0] <= 2 && G.p1[1] - G.p0[1] <= 2 && G.p1[2] - G.p0[2] <= 2;
        const double dcount =
            (double)((G.p1[0] - G.p0[0] + 1) * (G.p1[1] - G.p0[1] + 1) * (G.p1[2] - G.p0[2] + 1));
        if (small) {
            for (int64_t cz = G.p0[2]; cz <= G.p1[2]; ++cz)
                for (int64_t cy = G.p0[1]; cy <= G.p1[1]; ++cy)
                    for (int64_t cx = G.p0[0]; cx <= G.p1[0]; ++cx) {
                        const double x[3] = {g.lo[0] + (double)cx * g.h[0], g.lo[1] + (double)cy * g.h[1],
                                             g.lo[2] + (double)cz * g.h[2]};
                        const double v = local_eval(Mo, W, c, x, theta, false, gr, lane);
                        gmin[0] = fmin(gmin[0], v);
                        gmin[1] = fmin(gmin[1], -v);
                    }
        } else {
            double bx[2][3], bg[2][3];
            for (int t27 = 0; t27 < 27; ++t27) {
                const int id[3] = {t27 % 3, (t27 / 3) % 3, t27 / 9};
                double x[3];
                for (int d = 0; d < 3; ++d) x[d] = G.blo[d] + 0.5 * (double)id[d] * (G.bhi[d] - G.blo[d]);
                const double v = local_eval(Mo, W, c, x, theta, true, gr, lane);
                for (int s2 = 0; s2 < 2; ++s2) {
                    const double sg = s2 == 0 ? 1.0 : -1.0;
                    if (sg * v < gmin[s2]) {
                        gmin[s2] = sg * v;
                        for (int d = 0; d < 3; ++d) { bx[s2][d] = x[d]; bg[s2][d] = sg * gr[d]; }
                    }
                }
            }
            // the lattice bound already above alpha decides (the steps only lower g)
            if (!(bound_of(sd, dcount, gmin[0], gmin[1]) > alpha)) {
                for (int s2 = 0; s2 < 2; ++s2) {
                    if (!(sd & (1 << s2))) continue;
                    const double sg = s2 == 0 ? 1.0 : -1.0;
                    for (int st = 0; st < T; ++st) {
                        double wv[3], u[3], un = 0.0;
                        for (int d = 0; d < 3; ++d) {
                            wv[d] = G.bhi[d] - G.blo[d];
                            u[d] = -bg[s2][d] * wv[d];
                            un = fmax(un, fabs(u[d]));
                        }
                        if (!(un > 0.0)) break;
                        const double eta = 0.25 * ldexp(1.0, -st);
                        double xc[3];
                        for (int d = 0; d < 3; ++d) {
                            const double xn = bx[s2][d] + eta * wv[d] * u[d] / un;
                            xc[d] = xn < G.blo[d] ? G.blo[d] : (xn > G.bhi[d] ? G.bhi[d] : xn);
                        }
                        const double v = sg * local_eval(Mo, W, c, xc, theta, true, gr, lane);
                        if (v < gmin[s2]) {
                            gmin[s2] = v;
                            for (int d = 0; d < 3; ++d) { bx[s2][d] = xc[d]; bg[s2][d] = sg * gr[d]; }
                        }
                    }
                }
            }
        }
        if (lane == 0) {
            const double bnd = bound_of(sd, dcount, gmin[0], gmin[1]);
            bound[q] = bnd;
            decision[q] = bnd > alpha ? 2 : 0;
        }
        __syncwarp();
    }
}

// ---- Grouped local models (plain GPR): nodes with equal local sets share one factorisation.
// Group record g: grp[4g] = frontier position of a representative node, [4g+1] = |M'| = c,
// [4g+2] = offset of its FP32 data (L'^-1 column-major c x c, then v' = L'^-1 y', alpha'), [4g+3] =
// offset of its c member indices.

// Left-looking Cholesky of the column-major c x c matrix L in place (warp-cooperative, FP64).
__device__ void chol_warp(double *L, double *t, int64_t c, int lane, int *status)
{
    for (int64_t j = 0; j < c; ++j) {
        for (int64_t r = j + lane; r < c; r += 32) {
            double a = L[r + j * c];
            for (int64_t k = 0; k < j; ++k) a -= L[r + k * c] * L[j + k * c];
            t[r] = a;
        }
        __syncwarp();
        double piv = t[j];
        if (!(piv > 0.0)) {
            if (lane == 0) atomicCAS(status, 0, (int)GPR_ERR_NOT_PD);
            piv = 1e-300;
        }
        const double d = sqrt(piv);
        for (int64_t r = j + lane; r < c; r += 32) L[r + j * c] = r == j ? d : t[r] / d;
        __syncwarp();
    }
}

// One warp per group: gather M' of the representative node, factor K' in FP64, and store L'^-1,
// v' and alpha' in FP32 for the evaluations.
__global__ void k_local_factor(GridDev g, int D, int l, int kd, const int64_t *nodes, const int64_t *grp, int64_t ng,
                               LocalModel Mo, double beta, float *F, int32_t *I, double *ws, int64_t cmax, int *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double *L = ws + warp * (cmax * cmax + 3 * cmax);
    double *t = L + cmax * cmax, *x = t + cmax, *v = x + cmax;
    for (int64_t gi = warp; gi < ng; gi += nwarps) {
        const int64_t q = grp[4 * gi], c = grp[4 * gi + 1];
        float *Fg = F + grp[4 * gi + 2];
        int32_t *idx = I + grp[4 * gi + 3];
        const Geom G = node_geom(g, D, l, kd, nodes[q]);
        int64_t cc = 0;
        for (int64_t base = 0; base < Mo.m; base += 32) {
            const int64_t i = base + lane;
            const bool in = i < Mo.m && in_local_box(G, Mo.X + 3 * i, beta, Mo.kp);
            const unsigned msk = __ballot_sync(0xffffffffu, in);
            if (in && cc + __popc(msk & ((1u << lane) - 1)) < c) idx[cc + __popc(msk & ((1u << lane) - 1))] = (int32_t)i;
            cc += __popc(msk);
        }
        __syncwarp();
        if (cc != c && lane == 0) atomicCAS(status, 0, (int)GPR_ERR_ARG);  // self-check: equal sets
        for (int64_t s2 = 0; s2 < c; ++s2)
            for (int64_t r = s2 + lane; r < c; r += 32)
                L[r + s2 * c] = kval64(Mo.kp, Mo.X + 3 * idx[r], Mo.X + 3 * idx[s2]) + (r == s2 ? Mo.diag : 0.0);
        __syncwarp();
        chol_warp(L, t, c, lane, status);
        for (int64_t r = lane; r < c; r += 32) v[r] = Mo.y[idx[r]];
        __syncwarp();
        fwd_solve(L, c, v, lane);
        bwd_solve(L, c, v, t, lane);
        for (int64_t r = lane; r < c; r += 32) {
            Fg[c * c + r] = (float)v[r];
            Fg[c * c + c + r] = (float)t[r];
        }
        // L'^-1 column by column: column j solves L' x = e_j (rows >= j)
        for (int64_t j = 0; j < c; ++j) {
            for (int64_t r = lane; r < c; r += 32) x[r] = r == j ? 1.0 : 0.0;
            __syncwarp();
            for (int64_t jj = j; jj < c; ++jj) {
                const double xj = x[jj] / L[jj + jj * c];
                __syncwarp();
                if (lane == 0) x[jj] = xj;
                for (int64_t r = jj + 1 + lane; r < c; r += 32) x[r] -= L[r + jj * c] * xj;
                __syncwarp();
            }
            for (int64_t r = lane; r < c; r += 32) Fg[r + j * c] = r >= j ? (float)x[r] : 0.f;
            __syncwarp();
        }
    }
}

// g = (theta - mu) / sigma on a group's local model in FP32 (w = L'^-1 k as a triangular mat-vec).
__device__ float local_eval32(const KernParams &kp, const double *X, const int32_t *idx, const float *Fg, int64_t c,
                              const double *x, double theta, bool want_grad, float grad[3], float *wk, int lane)
{
    float *kv = wk, *dk = wk + c, *w = wk + 4 * c;
    const float ix = (float)(1.0 / kp.ell[0]), iy = (float)(1.0 / kp.ell[1]), iz = (float)(1.0 / kp.ell[2]);
    for (int64_t r = lane; r < c; r += 32) {
        const double *b = X + 3 * idx[r];
        const float dx = (float)(x[0] - b[0]), dy = (float)(x[1] - b[1]), dz = (float)(x[2] - b[2]);
        const float a = dx * ix, bb = dy * iy, cz = dz * iz, r2 = a * a + bb * bb + cz * cz;
        float kvl, gcoef;
        if (kp.kind == GPR_K_SE) {
            kvl = (float)kp.sf2 * expf(-0.5f * r2);
            gcoef = -kvl;
        } else {
            const float rr = sqrtf(r2), s5r = 2.23606797749979f * rr, e = expf(-s5r);
            kvl = (float)kp.sf2 * (1.0f + s5r + (5.0f / 3.0f) * r2) * e;
            gcoef = -(5.0f / 3.0f) * (float)kp.sf2 * (1.0f + s5r) * e;
        }
        kv[r] = kvl;
        dk[3 * r] = gcoef * dx * ix * ix;
        dk[3 * r + 1] = gcoef * dy * iy * iy;
        dk[3 * r + 2] = gcoef * dz * iz * iz;
    }
    __syncwarp();
    float mu = 0.f, ww = 0.f;
    for (int64_t r = lane; r < c; r += 32) {
        float a = 0.f;
        for (int64_t j = 0; j <= r; ++j) a = fmaf(Fg[r + j * c], kv[j], a);
        w[r] = a;
        mu = fmaf(a, Fg[c * c + r], mu);
        ww = fmaf(a, a, ww);
    }
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mu += __shfl_xor_sync(0xffffffffu, mu, o);
        ww += __shfl_xor_sync(0xffffffffu, ww, o);
    }
    float var = (float)kp.sf2 - ww;
    const float fl = (float)(1e-12 * kp.sf2);
    if (!(var > fl)) var = fl;
    const float sd = sqrtf(var), gl = (float)((theta - (double)mu) / (double)sd);
    if (!want_grad) return gl;
    // P_j = sum_{r >= j} L'^-1_rj w_r; d mu = dk . alpha', d var = -2 dk . P
    float gm[3] = {0.f, 0.f, 0.f}, gv[3] = {0.f, 0.f, 0.f};
    for (int64_t j = 0; j < c; ++j) {
        float p = 0.f;
        for (int64_t r = j + lane; r < c; r += 32) p = fmaf(Fg[r + j * c], w[r], p);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
        if ((j & 31) == lane) {
            const float al = Fg[c * c + c + j];
            for (int d = 0; d < 3; ++d) {
                gm[d] = fmaf(dk[3 * j + d], al, gm[d]);
                gv[d] = fmaf(-2.f * dk[3 * j + d], p, gv[d]);
            }
        }
    }
    for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            gm[d] += __shfl_xor_sync(0xffffffffu, gm[d], o);
            gv[d] += __shfl_xor_sync(0xffffffffu, gv[d], o);
        }
        grad[d] = -gm[d] / sd - gl * gv[d] / (2.f * var);
    }
    __syncwarp();
    return gl;
}

// One warp per local node of a grouped (plain GPR) level: the minimiser of k_local_nodes on its
// group's FP32 factor.
__global__ void k_local_eval(GridDev g, int D, int l, int kd, const int64_t *nodes, const int64_t *list,
                             const int32_t *node_group, int64_t nl, const int64_t *grp, KernParams kp, const double *X,
                             double theta, double alpha, int T, const int8_t *sides, int8_t *decision, double *bound,
                             const float *F, const int32_t *I, float *ws, int64_t cmax)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float *wk = ws + warp * 5 * cmax;
    for (int64_t t = warp; t < nl; t += nwarps) {
        const int64_t q = list[t], gi = node_group[t];
        const int64_t c = grp[4 * gi + 1];
        const float *Fg = F + grp[4 * gi + 2];
        const int32_t *idx = I + grp[4 * gi + 3];
        const Geom G = node_geom(g, D, l, kd, nodes[q]);
        const int sd = sides[q];
        double gmin[2] = {INFINITY, INFINITY};
        float gr[3];
        const bool small = G.p1[0] - G.p0[0] <= 2 && G.p1[1] - G.p0[1] <= 2 && G.p1[2] - G.p0[2] <= 2;
        const double dcount =
            (double)((G.p1[0] - G.p0[0] + 1) * (G.p1[1] - G.p0[1] + 1) * (G.p1[2] - G.p0[2] + 1));
        if (small) {
            for (int64_t cz = G.p0[2]; cz <= G.p1[2]; ++cz)
                for (int64_t cy = G.p0[1]; cy <= G.p1[1]; ++cy)
                    for (int64_t cx = G.p0[0]; cx <= G.p1[0]; ++cx) {
                        const double x[3] = {g.lo[0] + (double)cx * g.h[0], g.lo[1] + (double)cy * g.h[1],
                                             g.lo[2] + (double)cz * g.h[2]};
                        const double v = local_eval32(kp, X, idx, Fg, c, x, theta, false, gr, wk, lane);
                        gmin[0] = fmin(gmin[0], v);
                        gmin[1] = fmin(gmin[1], -v);
                    }
        } else {
            double bx[2][3], bg[2][3];
            for (int t27 = 0; t27 < 27; ++t27) {
                const int id[3] = {t27 % 3, (t27 / 3) % 3, t27 / 9};
                double x[3];
                for (int d = 0; d < 3; ++d) x[d] = G.blo[d] + 0.5 * (double)id[d] * (G.bhi[d] - G.blo[d]);
                const double v = local_eval32(kp, X, idx, Fg, c, x, theta, true, gr, wk, lane);
                for (int s2 = 0; s2 < 2; ++s2) {
                    const double sg = s2 == 0 ? 1.0 : -1.0;
                    if (sg * v < gmin[s2]) {
                        gmin[s2] = sg * v;
                        for (int d = 0; d < 3; ++d) { bx[s2][d] = x[d]; bg[s2][d] = sg * gr[d]; }
                    }
                }
            }
            if (!(bound_of(sd, dcount, gmin[0], gmin[1]) > alpha)) {
                for (int s2 = 0; s2 < 2; ++s2) {
                    if (!(sd & (1 << s2))) continue;
                    const double sg = s2 == 0 ? 1.0 : -1.0;
                    for (int stp = 0; stp < T; ++stp) {
                        double wv[3], u[3], un = 0.0;
                        for (int d = 0; d < 3; ++d) {
                            wv[d] = G.bhi[d] - G.blo[d];
                            u[d] = -bg[s2][d] * wv[d];
                            un = fmax(un, fabs(u[d]));
                        }
                        if (!(un > 0.0)) break;
                        const double eta = 0.25 * ldexp(1.0, -stp);
                        double xc[3];
                        for (int d = 0; d < 3; ++d) {
                            const double xn = bx[s2][d] + eta * wv[d] * u[d] / un;
                            xc[d] = xn < G.blo[d] ? G.blo[d] : (xn > G.bhi[d] ? G.bhi[d] : xn);
                        }
                        const double v = sg * local_eval32(kp, X, idx, Fg, c, xc, theta, true, gr, wk, lane);
                        if (v < gmin[s2]) {
                            gmin[s2] = v;
                            for (int d = 0; d < 3; ++d) { bx[s2][d] = xc[d]; bg[s2][d] = sg * gr[d]; }
                        }
                    }
                }
            }
        }
        if (lane == 0) {
            const double bnd = bound_of(sd, dcount, gmin[0], gmin[1]);
            bound[q] = bnd;
            decision[q] = bnd > alpha ? 2 : 0;
        }
        __syncwarp();
    }
}

struct OctBuffers {
    int64_t *front[2];
    int8_t *decision, *sides;
    double *bound;
    uint8_t *obs_flags, *have, *need, *lflag, *leaf;
    float2 *mv;
    int64_t *plist, *pend;
    float *tmp_mean, *tmp_var;
    double *xyz;
    float *W;     // partial sums of the tensor-core evaluations
    size_t wlen;  // floats in W
    float4 *ev, *lat;
    float *part;
    uint8_t *unal;
    int64_t *ulist;
    uint8_t *lflag2;  // nodes on the local model (beta >= 0)
    int64_t *llist;
    uint64_t *lsig;   // per node: hash and size of its local set
    int32_t *lcnt;
    uint8_t *cvalid;
    MinState *ms;
    unsigned long long *counters;  // [0] nnext, [1] nsub
    void *cscr;
    size_t csb;
};

}  // namespace

// Trace hook for tests: records one level's frontier, decisions and bounds on the host.
// With leaf_out set (and level -1) the call stops after the last level and copies the leaf-cell
// flags S (one byte per cell, device) there instead of reconstructing the leaves.
struct OctTrace {
    int level;
    int64_t *nodes;
    int8_t *decision;
    double *bound;
    int64_t capacity;
    int64_t count;
    uint8_t *leaf_out;
};

static gpr_status run_eval(gpr_model *M, OctBuffers &B, int64_t cnt, double theta,
                           cudaStream_t st, bool grad = true)
{
    {
        ProfScope ps("oct_eval_w", st);
        GPR_TRY(launch_tc_eval(M, B.xyz, cnt, grad, B.W, B.wlen, st));
    }
    const int nN = (int)(((M->mp + 255) / 256 * 256) / 64);
    k_eval_reduce<<<nb(cnt, 256), 256, 0, st>>>((float)M->kp.sf2, B.W, nN, grad, cnt, theta, B.ev, nullptr);
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

// Local models of the listed nodes (device list), one warp per node, FP64 throughout (gather,
// factor, minimise); work space per warp, bounded to ~2 GB.
static gpr_status local_per_node(gpr_model *M, const GridDev &g, int D, int l, int kd, const int64_t *nodes,
                                 const OctBuffers &B, const int64_t *list, int64_t nlist, int64_t cmax, double theta,
                                 const gpr_lcp_options *opts, int T, cudaStream_t st)
{
    const int64_t c = cmax > 0 ? cmax : 1;
    const size_t dper = (size_t)c * c * (M->sgpr ? 2 : 1) + 12 * (size_t)c;
    const size_t per = sizeof(double) * dper + sizeof(int32_t) * (size_t)c;
    int64_t nw = nlist < 4 * (int64_t)num_sms() ? nlist : 4 * (int64_t)num_sms();
    const int64_t cap = (int64_t)(((size_t)2 << 30) / per);
    if (nw > cap) nw = cap > 0 ? cap : 1;
    void *lws = nullptr;
    GPR_CUDA_TRY(cudaMallocAsync(&lws, per * (size_t)nw + 256, st));
    double *dws = (double *)lws;
    int32_t *iws = (int32_t *)((char *)lws + sizeof(double) * dper * nw);
    LocalModel Mo{M->X, M->y, M->sgpr ? M->A_M : nullptr, M->m, M->kp, M->sgpr ? M->kmm_jitter : M->sn2};
    int *status = gpr_status_word();
    if (!status) return GPR_ERR_CUDA;
    {
        ProfScope ps("oct_local", st, (double)nlist);
        k_local_nodes<<<(unsigned)((nw + 3) / 4), 128, 0, st>>>(g, D, l, kd, nodes, list, nlist, Mo, opts->beta, theta,
                                                                opts->alpha, T, B.sides, B.decision, B.bound, dws, iws,
                                                                c, status);
    }
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    GPR_CUDA_TRY(cudaFreeAsync(lws, st));
    return GPR_OK;
}

// Local models of a level's listed nodes for a plain GPR model: nodes are grouped by their local
// set (hash and size, gathered from the device), one factorisation per group (FP64, stored as
// FP32 L'^-1), then every node is bounded on its group's factor in FP32.  Groups are processed in
// batches whose FP32 data stays within ~2 GB.
static gpr_status local_grouped(gpr_model *M, const GridDev &g, int D, int l, int kd, const int64_t *nodes,
                                const OctBuffers &B, int64_t nl, int64_t cmax, double theta,
                                const gpr_lcp_options *opts, int T, cudaStream_t st)
{
    std::vector<uint64_t> hs((size_t)nl);
    std::vector<int32_t> hc((size_t)nl);
    std::vector<int64_t> hl((size_t)nl);
    {
        void *tmp = nullptr;
        GPR_CUDA_TRY(cudaMallocAsync(&tmp, (size_t)nl * 12 + 256, st));
        uint64_t *ds = (uint64_t *)tmp;
        int32_t *dc = (int32_t *)((char *)tmp + (size_t)nl * 8);
        k_gather_local<<<nb(nl, 256), 256, 0, st>>>(B.llist, nl, B.lsig, B.lcnt, ds, dc);
        note_launch();
        GPR_CUDA_TRY(cudaMemcpyAsync(hs.data(), ds, (size_t)nl * 8, cudaMemcpyDeviceToHost, st));
        GPR_CUDA_TRY(cudaMemcpyAsync(hc.data(), dc, (size_t)nl * 4, cudaMemcpyDeviceToHost, st));
        GPR_CUDA_TRY(cudaMemcpyAsync(hl.data(), B.llist, (size_t)nl * 8, cudaMemcpyDeviceToHost, st));
        GPR_CUDA_TRY(cudaFreeAsync(tmp, st));
        GPR_CUDA_TRY(cudaStreamSynchronize(st));
    }
    // groups in order of first appearance
    std::unordered_map<uint64_t, int32_t> key_to_group;
    std::vector<int32_t> node_group((size_t)nl);
    std::vector<int64_t> rep, gc;
    for (int64_t t = 0; t < nl; ++t) {
        const uint64_t key = hs[t] ^ ((uint64_t)hc[t] * 0xD6E8FEB86659FD93ULL);
        auto it = key_to_group.find(key);
        if (it == key_to_group.end()) {
            it = key_to_group.emplace(key, (int32_t)rep.size()).first;
            rep.push_back(hl[t]);
            gc.push_back(hc[t]);
        }
        node_group[t] = it->second;
    }
    // a set that only one node has is cheaper to factor and solve per node in FP64 than to invert
    std::vector<int64_t> members(rep.size(), 0);
    for (int64_t t = 0; t < nl; ++t) ++members[node_group[t]];
    std::vector<int32_t> remap(rep.size(), -1);
    std::vector<int64_t> rep2, gc2, singles;
    for (size_t gi = 0; gi < rep.size(); ++gi)
        if (members[gi] > 1) {
            remap[gi] = (int32_t)rep2.size();
            rep2.push_back(rep[gi]);
            gc2.push_back(gc[gi]);
        }
    for (int64_t t = 0; t < nl; ++t) {
        if (remap[node_group[t]] < 0) singles.push_back(hl[t]);
        node_group[t] = remap[node_group[t]];
    }
    rep.swap(rep2);
    gc.swap(gc2);
    if (!singles.empty()) {
        int64_t *dl = nullptr;
        GPR_CUDA_TRY(cudaMallocAsync((void **)&dl, singles.size() * 8, st));
        GPR_CUDA_TRY(cudaMemcpyAsync(dl, singles.data(), singles.size() * 8, cudaMemcpyHostToDevice, st));
        GPR_TRY(local_per_node(M, g, D, l, kd, nodes, B, dl, (int64_t)singles.size(), cmax, theta, opts, T, st));
        GPR_CUDA_TRY(cudaFreeAsync(dl, st));
        GPR_CUDA_TRY(cudaStreamSynchronize(st));
    }
    const int64_t ng = (int64_t)rep.size();
    const size_t budget = (size_t)2 << 30;
    LocalModel Mo{M->X, M->y, nullptr, M->m, M->kp, M->sn2};
    int *status = gpr_status_word();
    if (!status) return GPR_ERR_CUDA;
    int64_t g0 = 0;
    while (g0 < ng) {
        // a batch of groups [g0, g1) and the nodes that belong to it
        size_t fbytes = 0, ibytes = 0;
        int64_t g1 = g0;
        std::vector<int64_t> tab;
        while (g1 < ng) {
            const size_t c = (size_t)gc[g1];
            const size_t fb = Carver::round((c * c + 2 * c) * sizeof(float)), ib = Carver::round(c * sizeof(int32_t));
            if (g1 > g0 && fbytes + ib + ibytes + fb > budget) break;
            tab.insert(tab.end(), {rep[g1], (int64_t)c, (int64_t)(fbytes / sizeof(float)), (int64_t)(ibytes / sizeof(int32_t))});
            fbytes += fb;
            ibytes += ib;
            ++g1;
        }
        std::vector<int64_t> blist;
        std::vector<int32_t> bgroup;
        for (int64_t t = 0; t < nl; ++t)
            if (node_group[t] >= 0 && node_group[t] >= g0 && node_group[t] < g1) {
                blist.push_back(hl[t]);
                bgroup.push_back(node_group[t] - (int32_t)g0);
            }
        const int64_t bg = g1 - g0, bn = (int64_t)blist.size();
        const int64_t nwf = bg < 4 * (int64_t)num_sms() ? bg : 4 * (int64_t)num_sms();
        const int64_t nwe = bn < 16 * (int64_t)num_sms() ? bn : 16 * (int64_t)num_sms();
        const size_t wsf = Carver::round((size_t)nwf * (cmax * cmax + 3 * cmax) * sizeof(double));
        const size_t wse = Carver::round((size_t)nwe * 5 * cmax * sizeof(float));
        const size_t total = Carver::round(fbytes) + Carver::round(ibytes) + wsf + wse +
                             Carver::round(tab.size() * 8) + Carver::round(blist.size() * 8) +
                             Carver::round(bgroup.size() * 4) + 1024;
        void *buf = nullptr;
        GPR_CUDA_TRY(cudaMallocAsync(&buf, total, st));
        Carver cv{(char *)buf};
        float *F = cv.take<float>(fbytes / sizeof(float));
        int32_t *I = cv.take<int32_t>(ibytes / sizeof(int32_t));
        double *wf = cv.take<double>((size_t)nwf * (cmax * cmax + 3 * cmax));
        float *we = cv.take<float>((size_t)nwe * 5 * cmax);
        int64_t *dtab = cv.take<int64_t>(tab.size());
        int64_t *dlist = cv.take<int64_t>(blist.size());
        int32_t *dgroup = cv.take<int32_t>(bgroup.size());
        GPR_CUDA_TRY(cudaMemcpyAsync(dtab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, st));
        GPR_CUDA_TRY(cudaMemcpyAsync(dlist, blist.data(), blist.size() * 8, cudaMemcpyHostToDevice, st));
        GPR_CUDA_TRY(cudaMemcpyAsync(dgroup, bgroup.data(), bgroup.size() * 4, cudaMemcpyHostToDevice, st));
        {
            ProfScope ps("oct_local_factor", st, (double)bg);
            k_local_factor<<<(unsigned)((nwf + 3) / 4), 128, 0, st>>>(g, D, l, kd, nodes, dtab, bg, Mo, opts->beta, F, I,
                                                                      wf, cmax, status);
        }
        note_launch();
        {
            ProfScope ps("oct_local", st, (double)bn);
            k_local_eval<<<(unsigned)((nwe + 3) / 4), 128, 0, st>>>(g, D, l, kd, nodes, dlist, dgroup, bn, dtab, M->kp,
                                                                    M->X, theta, opts->alpha, T, B.sides, B.decision,
                                                                    B.bound, F, I, we, cmax);
        }
        note_launch();
        GPR_CUDA_TRY(cudaGetLastError());
        GPR_CUDA_TRY(cudaFreeAsync(buf, st));
        // the host vectors are released at return; the copies above were queued before the free
        GPR_CUDA_TRY(cudaStreamSynchronize(st));
        g0 = g1;
    }
    return GPR_OK;
}

gpr_status octree_lcp(gpr_model *M, const gpr_grid *grid, double theta, int D, const gpr_lcp_options *opts,
                      float *lcp, gpr_adaptive_stats *stats, cudaStream_t st, OctTrace *trace)
{
    GridDev g = make_grid(grid);
    int64_t n = g.npts(), nc = g.ncells(), m = M->m;
    size_t te = table_elems(M, g);
    int T = opts->max_iters_min;
    const int kd = opts->tree == GPR_TREE_KD ? 1 : 0;
    const int last = kd ? 3 * D : D;  // the level whose subdivided nodes are cells of S
    // nodes with >= 4 cells along an axis: at most prod ceil((n_d - 1) / 4) of them in any octree
    // level; a K-D node's extents differ by at most a factor 2, so (4, 2, 2) bounds its count
    int64_t max_large = 1;
    for (int d = 0; d < 3; ++d) max_large *= (int64_t)(g.n[d] - 1 + (kd && d < 2 ? 1 : 3)) / (kd && d < 2 ? 2 : 4);
    // workspace (slot 0): tables, frontier, per-point mean/var table, evaluation chunk
    size_t csb = compact_scratch_bytes(nc > n ? nc : n);
    size_t bytes = 2 * Carver::round((size_t)nc * 8) + 2 * Carver::round((size_t)nc) +
                   Carver::round((size_t)nc * 8) + Carver::round((size_t)m) + 3 * Carver::round((size_t)n) +
                   Carver::round((size_t)nc) + Carver::round((size_t)nc) + Carver::round((size_t)n * 16) +
                   Carver::round((size_t)nc * 8) + 2 * Carver::round((size_t)n * 4) +
                   Carver::round((size_t)kEvalChunk * 24) + Carver::round(tc_eval_partial_elems(M, kEvalChunk) * 4) +
                   Carver::round((size_t)kEvalChunk * 16) + Carver::round((size_t)kEvalChunk) +
                   Carver::round((size_t)nc * sizeof(MinState)) + Carver::round((size_t)max_large * 27 * 16) + 512 +
                   csb + Carver::round(tc_partial_elems(GPR_P_BF16X3, M, n) * 4) + Carver::round((size_t)max_large * 2) +
                   Carver::round((size_t)max_large * 16) + 8192 + Carver::round((size_t)nc * 4) + 2 * Carver::round((size_t)nc) +
                   Carver::round((size_t)nc) + Carver::round((size_t)nc * 8) + Carver::round((size_t)nc * 8) +
                   Carver::round((size_t)nc * 4) + 256 * 26;
    gpr_precision pp = opts->prec == GPR_P_FP64 ? GPR_P_FP32 : opts->prec;
    GridCache *C = nullptr;
    GPR_TRY(grid_cache(M, grid, g, pp, &C, st));
    GPR_TRY(ws_reserve(M, 0, bytes, st));
    Carver cv{(char *)ws_ptr(M, 0)};
    const float *T32 = C->T32;
    const double *T64 = C->T64;
    const float2 *Tff = C->Tff;
    OctBuffers B;
    B.front[0] = cv.take<int64_t>((size_t)nc);
    B.front[1] = cv.take<int64_t>((size_t)nc);
    B.decision = cv.take<int8_t>((size_t)nc);
    B.sides = cv.take<int8_t>((size_t)nc);
    B.bound = cv.take<double>((size_t)nc);
    B.obs_flags = cv.take<uint8_t>((size_t)m);
    Pyramid pyr;
    int64_t pyr_bytes = 0;
    for (int l = D; l >= 0; --l) {
        const int64_t s = (int64_t)1 << (D - l);
        for (int d = 0; d < 3; ++d) pyr.dim[l][d] = (int32_t)((g.n[d] - 1 + s - 1) / s);
        pyr.off[l] = pyr_bytes;
        pyr_bytes += Carver::round((size_t)pyr.dim[l][0] * pyr.dim[l][1] * pyr.dim[l][2]);
    }
    uint32_t *pyr_fine = cv.take<uint32_t>((size_t)nc);
    uint8_t *pyr_lv = cv.take<uint8_t>((size_t)pyr_bytes);
    B.need = cv.take<uint8_t>((size_t)n);
    uint8_t *pflag = cv.take<uint8_t>((size_t)n);
    B.lflag = cv.take<uint8_t>((size_t)nc);
    B.leaf = cv.take<uint8_t>((size_t)nc);
    B.mv = C->mv;
    B.have = C->have_mv;
    B.plist = cv.take<int64_t>((size_t)n * 2);
    B.pend = cv.take<int64_t>((size_t)nc);
    B.tmp_mean = cv.take<float>((size_t)n);
    B.tmp_var = cv.take<float>((size_t)n);
    B.xyz = cv.take<double>((size_t)kEvalChunk * 3);
    B.wlen = tc_eval_partial_elems(M, kEvalChunk);
    B.W = cv.take<float>(B.wlen);
    B.ev = cv.take<float4>((size_t)kEvalChunk);
    B.lat = cv.take<float4>((size_t)max_large * 27);
    B.cvalid = cv.take<uint8_t>((size_t)kEvalChunk);
    B.ms = cv.take<MinState>((size_t)nc);
    B.counters = cv.take<unsigned long long>(4);
    B.csb = csb;
    B.cscr = cv.take<char>(csb);
    B.part = cv.take<float>(tc_partial_elems(GPR_P_BF16X3, M, n));
    B.unal = cv.take<uint8_t>((size_t)max_large * 2);
    B.ulist = cv.take<int64_t>((size_t)max_large * 2);
    B.lflag2 = cv.take<uint8_t>((size_t)nc);
    B.llist = cv.take<int64_t>((size_t)nc);
    B.lsig = cv.take<uint64_t>((size_t)nc);
    B.lcnt = cv.take<int32_t>((size_t)nc);
    const bool local = opts->beta >= 0.0 && isfinite(opts->beta);
    int32_t *slot = (int32_t *)B.tmp_mean;  // reused by the leaf phase (n int32 fits in n floats)
    int64_t *clist = B.pend;                 // reused by the leaf phase (nc int64)


    GPR_CUDA_TRY(cudaMemsetAsync(B.leaf, 0, (size_t)nc, st));
    k_obs_flags<<<nb(m, 128), 128, 0, st>>>(M->mu_obs, M->var_obs, m, theta, opts->alpha, B.obs_flags);
    note_launch();
    GPR_CUDA_TRY(cudaMemsetAsync(pyr_fine, 0, sizeof(uint32_t) * (size_t)nc, st));
    k_obs_cells<<<nb(m, 128), 128, 0, st>>>(g, M->X, m, B.obs_flags, pyr_fine);
    note_launch();
    for (int l = D; l >= 0; --l) {  // level D from the words of the cells, then halving
        const int32_t *pd = pyr.dim[l];
        const int64_t np = (int64_t)pd[0] * pd[1] * pd[2];
        if (l == D) {
            k_cells_to_bytes<<<nb(np, 256), 256, 0, st>>>(pyr_fine, np, pyr_lv + pyr.off[l]);
        } else {
            const int32_t *cd = pyr.dim[l + 1];
            k_pyr_level<uint8_t><<<nb(np, 256), 256, 0, st>>>(pyr_lv + pyr.off[l + 1], cd[0], cd[1], cd[2],
                                                              pyr_lv + pyr.off[l], pd[0], pd[1], pd[2]);
        }
        note_launch();
    }
    int64_t root = 0;
    GPR_CUDA_TRY(cudaMemcpyAsync(B.front[0], &root, sizeof root, cudaMemcpyHostToDevice, st));
    int64_t count = 1;
    int cur = 0;
    if (stats) memset(stats, 0, sizeof *stats);
    TraceRange levels("algorithm1_levels");
    for (int l = 0; l <= last && count > 0; ++l) {
        const int64_t *nodes = B.front[cur];
        const int64_t s = axis_extent(D, l, kd, 2);  // the node's largest extent
        const int lp = kd ? (l + 2) / 3 : l;          // pyramid level of its smallest extent
        ProfScope lvl("oct_level", st);
        k_ptest<<<nb(count, 256), 256, 0, st>>>(g, D, l, kd, nodes, count, pyr_lv + pyr.off[lp], pyr.dim[lp][0],
                                                 pyr.dim[lp][1], pyr.dim[lp][2], B.decision, B.sides);
        note_launch();
        // nodes whose local set (Sec. 5.2) is a strict subset of the observations leave the
        // full-model path below and are bounded on their local model
        int64_t nlocal = 0;
        unsigned long long cmax = 0;
        if (local) {
            GPR_CUDA_TRY(cudaMemsetAsync(B.counters + 2, 0, sizeof(unsigned long long), st));
            k_local_flag<<<nb(count, 128), 128, 0, st>>>(g, D, l, kd, nodes, count, B.decision, M->X, m, opts->beta, M->kp,
                                                         B.lflag2, B.counters + 2, B.lsig, B.lcnt);
            note_launch();
            GPR_TRY(compact_flags(B.lflag2, count, B.llist, nullptr, &nlocal, B.cscr, B.csb, st));
            if (nlocal > 0)
                GPR_CUDA_TRY(cudaMemcpyAsync(&cmax, B.counters + 2, sizeof cmax, cudaMemcpyDeviceToHost, st));
            GPR_CUDA_TRY(cudaStreamSynchronize(st));
        }
        // small nodes: exact minimum over grid points from the per-point table
        {
            MvFillScope fill(M, st);
            GPR_CUDA_TRY(cudaMemsetAsync(B.need, 0, (size_t)n, st));
            k_mark_small_points<<<nb(count, 128), 128, 0, st>>>(g, D, l, kd, nodes, count, B.decision, B.have, B.need);
            note_launch();
            int64_t nneed = 0;
            GPR_TRY(compact_flags(B.need, n, B.plist, nullptr, &nneed, B.cscr, B.csb, st));
            if (nneed > 0) {
                GPR_TRY(fast_meanvar(M, g, pp, T32, Tff, T64, B.plist, 0, nneed, B.tmp_mean, B.tmp_var, B.part, st));
                k_scatter_mv<<<nb(nneed, 256), 256, 0, st>>>(B.plist, nneed, B.tmp_mean, B.tmp_var, B.mv, B.have);
                note_launch();
            }
        }
        k_small_bound<<<nb(count, 128), 128, 0, st>>>(g, D, l, kd, nodes, count, B.mv, theta, opts->alpha, M->kp.sf2,
                                                      B.decision, B.sides, B.bound);
        note_launch();
        // large nodes: lattice start + projected gradient steps
        if (s > 2) {
            k_flag_large<<<nb(count, 256), 256, 0, st>>>(g, D, l, kd, nodes, count, B.decision, B.lflag);
            note_launch();
            int64_t npend = 0;
            GPR_TRY(compact_flags(B.lflag, count, B.pend, nullptr, &npend, B.cscr, B.csb, st));
            if (npend > 0) {
                // lattice values: aligned nodes from the per-point table, unaligned ones evaluated
                {
                    MvFillScope fill(M, st);
                    GPR_CUDA_TRY(cudaMemsetAsync(B.need, 0, (size_t)n, st));
                    k_mark_lattice<<<nb(npend, 128), 128, 0, st>>>(g, D, l, kd, nodes, B.pend, npend, B.have, B.need,
                                                                   B.unal);
                    note_launch();
                    int64_t nneed = 0;
                    GPR_TRY(compact_flags(B.need, n, B.plist, nullptr, &nneed, B.cscr, B.csb, st));
                    if (nneed > 0) {
                        GPR_TRY(fast_meanvar(M, g, pp, T32, Tff, T64, B.plist, 0, nneed, B.tmp_mean, B.tmp_var,
                                             B.part, st));
                        k_scatter_mv<<<nb(nneed, 256), 256, 0, st>>>(B.plist, nneed, B.tmp_mean, B.tmp_var, B.mv,
                                                                     B.have);
                        note_launch();
                    }
                }
                k_lattice_from_table<<<nb(npend * 27, 256), 256, 0, st>>>(g, D, l, kd, nodes, B.pend, npend, B.unal, B.mv,
                                                                          theta, M->kp.sf2, B.lat);
                note_launch();
                int64_t nun = 0;
                GPR_TRY(compact_flags(B.unal, npend, B.ulist, nullptr, &nun, B.cscr, B.csb, st));
                for (int64_t first = 0; first < nun * 27; first += kEvalChunk) {
                    int64_t cnt = nun * 27 - first < kEvalChunk ? nun * 27 - first : kEvalChunk;
                    k_lattice_points<<<nb(cnt, 256), 256, 0, st>>>(g, D, l, kd, nodes, B.pend, B.ulist, first, cnt, B.xyz);
                    note_launch();
                    // lattice values only: the start points' gradients are evaluated afresh below
                    GPR_TRY(run_eval(M, B, cnt, theta, st, false));
                    k_scatter_lattice<<<nb(cnt, 256), 256, 0, st>>>(B.ev, B.ulist, first, cnt, B.lat);
                    note_launch();
                }
                k_lattice_best<<<nb(npend, 128), 128, 0, st>>>(B.lat, npend, B.ms);
                note_launch();
                k_lattice_coords<<<nb(npend, 128), 128, 0, st>>>(g, D, l, kd, nodes, B.pend, npend, B.ms);
                note_launch();
                // nodes whose lattice minima already give a bound above alpha are decided; the
                // minimiser runs on the others (the act list)
                k_large_bound<<<nb(npend, 128), 128, 0, st>>>(g, D, l, kd, nodes, B.pend, nullptr, npend, B.ms, opts->alpha,
                                                             B.decision, B.sides, B.bound, B.unal);
                note_launch();
                int64_t nact = 0;  // (node, side) pairs to minimise
                GPR_TRY(compact_flags(B.unal, 2 * npend, B.ulist, nullptr, &nact, B.cscr, B.csb, st));
                const int64_t *act = B.ulist;
                // g and its gradient at the start point of each side
                for (int64_t first = 0; first < nact; first += kEvalChunk) {
                    int64_t cnt = nact - first < kEvalChunk ? nact - first : kEvalChunk;
                    k_start_points<<<nb(cnt, 256), 256, 0, st>>>(B.ms, act, first, cnt, B.xyz);
                    note_launch();
                    GPR_TRY(run_eval(M, B, cnt, theta, st));
                    k_start_grad<<<nb(cnt, 256), 256, 0, st>>>(B.ev, act, first, cnt, B.ms);
                    note_launch();
                }
                for (int t = 0; t < T && nact > 0; ++t) {
                    for (int64_t first = 0; first < nact; first += kEvalChunk) {
                        int64_t cnt = nact - first < kEvalChunk ? nact - first : kEvalChunk;
                        k_candidates<<<nb(cnt, 256), 256, 0, st>>>(g, D, l, kd, nodes, B.pend, act, B.ms, t, first, cnt,
                                                                   B.xyz, B.cvalid);
                        note_launch();
                        // the last step's gradients are never used: value only
                        GPR_TRY(run_eval(M, B, cnt, theta, st, t < T - 1));
                        k_accept<<<nb(cnt, 256), 256, 0, st>>>(B.xyz, B.cvalid, B.ev, act, first, cnt, B.ms);
                        note_launch();
                    }
                }
                if (nact > 0) {
                    k_large_bound<<<nb(nact, 128), 128, 0, st>>>(g, D, l, kd, nodes, B.pend, act, nact, B.ms, opts->alpha,
                                                                 B.decision, B.sides, B.bound, nullptr);
                    note_launch();
                }
            }
        }
        if (nlocal > 0 && !M->sgpr) {
            GPR_TRY(local_grouped(M, g, D, l, kd, nodes, B, nlocal, (int64_t)cmax, theta, opts, T, st));
        } else if (nlocal > 0) {
            GPR_TRY(local_per_node(M, g, D, l, kd, nodes, B, B.llist, nlocal, (int64_t)cmax, theta, opts, T, st));
        }
        GPR_CUDA_TRY(cudaMemsetAsync(B.counters, 0, 2 * sizeof(unsigned long long), st));
        k_children<<<nb(count, 256), 256, 0, st>>>(g, D, l, kd, nodes, count, B.decision, B.front[1 - cur], B.counters,
                                                   B.leaf, B.counters + 1);
        note_launch();
        GPR_CUDA_TRY(cudaGetLastError());
        unsigned long long hc[2] = {0, 0};
        GPR_CUDA_TRY(cudaMemcpyAsync(hc, B.counters, sizeof hc, cudaMemcpyDeviceToHost, st));
        if (trace && trace->level == l) {
            int64_t c = count < trace->capacity ? count : trace->capacity;
            GPR_CUDA_TRY(cudaMemcpyAsync(trace->nodes, nodes, sizeof(int64_t) * c, cudaMemcpyDeviceToHost, st));
            GPR_CUDA_TRY(cudaMemcpyAsync(trace->decision, B.decision, c, cudaMemcpyDeviceToHost, st));
            GPR_CUDA_TRY(cudaMemcpyAsync(trace->bound, B.bound, sizeof(double) * c, cudaMemcpyDeviceToHost, st));
            trace->count = count;
        }
        GPR_CUDA_TRY(cudaStreamSynchronize(st));
        if (stats && l < 24) {
            stats->nodes_per_level[l] = count;
            stats->subdiv_per_level[l] = (int64_t)hc[1];
        }
        count = (int64_t)hc[0];
        cur = 1 - cur;
    }
    levels.end();
    if (trace) {
        if (trace->leaf_out)
            GPR_CUDA_TRY(cudaMemcpyAsync(trace->leaf_out, B.leaf, (size_t)nc, cudaMemcpyDeviceToDevice, st));
        return GPR_OK;
    }
    int64_t leaf_cells = 0, rp = 0, est = 0;
    gpr_adaptive_stats tmp;
    memset(&tmp, 0, sizeof tmp);
    TraceRange leaf("leaf_lcp");
    GPR_TRY(lcp_from_kept_cells(M, g, T64, B.leaf, pflag, B.plist, slot, clist, B.cscr, B.csb, lcp_opts(opts, theta),
                                lcp, &tmp, st));
    leaf_cells = tmp.leaf_cells;
    rp = tmp.recon_points;
    est = tmp.cells_estimated;
    if (stats) {
        stats->leaf_cells = leaf_cells;
        stats->recon_points = rp;
        stats->cells_estimated = est;
    }
    return GPR_OK;
}

extern "C" gpr_status gpr_lcp_adaptive(gpr_model *M, const gpr_grid *grid, double isovalue, int32_t max_depth,
                                       const gpr_lcp_options *opts, float *lcp, gpr_adaptive_stats *stats,
                                       void *stream)
{
    TraceRange trace_("gpr_lcp_adaptive");
    if (!M || !grid_valid(grid) || !lcp || !opts_valid(opts) || !isfinite(isovalue)) return GPR_ERR_ARG;
    if (max_depth < 0 || max_depth > 20) return GPR_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (((int64_t)1 << max_depth) < (int64_t)grid->n[d] - 1) return GPR_ERR_ARG;
    return octree_lcp(M, grid, isovalue, max_depth, opts, lcp, stats, (cudaStream_t)stream, nullptr);
}

// The leaf cells S of Algorithm 1 only (one byte per cell, device), for the adaptive backward.
gpr_status octree_leaf_mask(gpr_model *M, const gpr_grid *grid, double theta, int D, const gpr_lcp_options *opts,
                            uint8_t *leaf, cudaStream_t st)
{
    OctTrace tr{-1, nullptr, nullptr, nullptr, 0, 0, leaf};
    return octree_lcp(M, grid, theta, D, opts, nullptr, nullptr, st, &tr);
}

// Test hook (not in the public header): the evaluation path of the bound's minimiser (tensor-core
// rows and the warp reduction) at count points (device, count x 3 FP64); out: device float, 8 per
// point: mu, var, grad mu (3), grad var (3) (the gradients 0 without grad).
extern "C" gpr_status gpr_eval_points(gpr_model *M, const double *xyz, int64_t count, int32_t grad, float *out,
                                      void *stream)
{
    TraceRange trace_("gpr_eval_points");
    if (!M || !xyz || !out || count < 0 || count > kEvalChunk) return GPR_ERR_ARG;
    if (count == 0) return GPR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t pe = tc_eval_partial_elems(M, count);
    float *part = nullptr;
    float4 *g4 = nullptr;
    const size_t pe4 = (pe + 3) / 4 * 4;  // the g / grad g records after the partials, 16-byte aligned
    GPR_CUDA_TRY(cudaMallocAsync((void **)&part, pe4 * sizeof(float) + (size_t)count * sizeof(float4), st));
    g4 = (float4 *)(part + pe4);
    gpr_status rc = launch_tc_eval(M, xyz, count, grad != 0, part, pe, st);
    if (rc == GPR_OK) {
        const int nN = (int)(((M->mp + 255) / 256 * 256) / 64);
        k_eval_reduce<<<nb(count, 256), 256, 0, st>>>((float)M->kp.sf2, part, nN, grad != 0, count, 0.0, g4, out);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) rc = GPR_ERR_CUDA;
    }
    cudaFreeAsync(part, st);
    return rc;
}

// Test hook (not in the public header): the frontier, decisions and bounds of one level.
extern "C" gpr_status gpr_octree_trace(gpr_model *M, const gpr_grid *grid, double isovalue, int32_t max_depth,
                                       const gpr_lcp_options *opts, int32_t level, int64_t *nodes, int8_t *decision,
                                       double *bound, int64_t capacity, int64_t *count, void *stream)
{
    TraceRange trace_("gpr_octree_trace");
    if (!M || !grid_valid(grid) || !opts_valid(opts) || !nodes || !decision || !bound || !count) return GPR_ERR_ARG;
    if (max_depth < 0 || max_depth > 20 || level < 0 || level > (opts->tree == GPR_TREE_KD ? 3 : 1) * max_depth)
        return GPR_ERR_ARG;
    OctTrace tr{level, nodes, decision, bound, capacity, 0, nullptr};
    gpr_status s = octree_lcp(M, grid, isovalue, max_depth, opts, nullptr, nullptr, (cudaStream_t)stream, &tr);
    *count = tr.count;
    return s;
}
