// Cell level-crossing probability (Sec. 4): LCP = 1 - P(all 8 corners < theta)
// - P(all 8 corners > theta) for the 8-variate Gaussian of a cell's corners.
// Stage 1 (FP64, thread per cell): assemble (mu_8, Sigma_8) from per-point stats15,
// add the jitter, apply Boole's pre-skip and factor Sigma_8 = L L^T.
// Stage 2 (FP32, warp per cell): the estimator -- Genz sequential conditioning over
// a shifted rank-1 lattice (SOV-QMC), or the paper's Monte Carlo with Philox-4x32-10.
#include <math.h>

#include "internal.h"
#include "normal_fast.cuh"

namespace {

// For the 28 corner pairs (c1 < c2): which corner stores the covariance (0: c1, 1: c2) and the
// offset slot e of that corner's stats15 row.  Built on the host from the offset list.
struct PairTable {
    int owner[8][8];
    int slot[8][8];
};

PairTable make_pair_table()
{
    PairTable t;
    for (int c1 = 0; c1 < 8; ++c1)
        for (int c2 = 0; c2 < 8; ++c2) {
            t.owner[c1][c2] = -1;
            t.slot[c1][c2] = -1;
            if (c1 == c2) continue;
            int d[3] = {((c2 >> 0) & 1) - ((c1 >> 0) & 1), ((c2 >> 1) & 1) - ((c1 >> 1) & 1),
                        ((c2 >> 2) & 1) - ((c1 >> 2) & 1)};
            for (int e = 0; e < 13; ++e) {
                if (kOff13[e][0] == d[0] && kOff13[e][1] == d[1] && kOff13[e][2] == d[2]) { t.owner[c1][c2] = 0; t.slot[c1][c2] = e; }
                if (kOff13[e][0] == -d[0] && kOff13[e][1] == -d[1] && kOff13[e][2] == -d[2]) { t.owner[c1][c2] = 1; t.slot[c1][c2] = e; }
            }
        }
    return t;
}

// One estimator record per cell that survives the pre-skip.
struct CellRec {
    float b[8];       // theta - mu_c
    float L[36];      // lower Cholesky factor, row-major packed (row i: entries 0..i)
    int64_t cell;     // linear cell index (keys the lattice shift / Philox stream)
    float *out;       // output address (the records of several fields share one estimator launch)
};

__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// ---- closed-form cell estimators (FP32 with this library's Phi)

// 12-point Gauss-Legendre rule on [-1, 1] (symmetric half: nodes, weights).
__constant__ float kGLx[6] = {0.1252334085114689f, 0.3678314989981802f, 0.5873179542866175f,
                              0.7699026741943047f, 0.9041172563704748f, 0.9815606342467192f};
__constant__ float kGLw[6] = {0.2491470458134027f, 0.2334925365383546f, 0.20316742672306573f,
                              0.16007832854334642f, 0.10693932599531907f, 0.04717533638651141f};

// Owen's T(h, a) = (1/2pi) int_0^a exp(-h^2 (1 + x^2) / 2) / (1 + x^2) dx for 0 <= a <= 1, by the
// Gauss-Legendre rule on [0, a] (a smooth integrand there).
__device__ float owen_t_small(float h, float a)
{
    const float hh = -0.5f * h * h, half = 0.5f * a;
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int sg = -1; sg <= 1; sg += 2) {
            const float x = half * (1.0f + (float)sg * kGLx[i]);
            const float q = 1.0f + x * x;
            s = fmaf(kGLw[i], __expf(hh * q) / q, s);
        }
    }
    return s * half * 0.15915494309189535f;
}

// Owen's T for any a: odd in a, even in h; for a > 1 through Owen's identity
// T(h, a) + T(ah, 1/a) = (Phi(h) + Phi(ah)) / 2 - Phi(h) Phi(ah)   (h >= 0, a > 0).
__device__ float owen_t(float h, float a)
{
    const float sg = a < 0.f ? -1.f : 1.f;
    a = fabsf(a);
    h = fabsf(h);
    if (a <= 1.0f) return sg * owen_t_small(h, a);
    const float ah = a * h, ph = nrm_cdf(h), pah = nrm_cdf(ah);
    return sg * (0.5f * (ph + pah) - ph * pah - owen_t_small(ah, 1.0f / a));
}

// P(X1 < h, X2 < k), standard bivariate normal with correlation r = rr (FP64 in, for the
// arguments of T, which cancel when r is near 1): Owen's (1956) formula
// Phi2 = Phi(h)/2 + Phi(k)/2 - T(h, (k - r h)/(h s)) - T(k, (h - r k)/(k s)) - beta, s = sqrt(1-r^2),
// beta = 1/2 when h k < 0 or (h k = 0 and h + k < 0).
__device__ float bvn_lower(double h, double k, double r)
{
    const double s = sqrt((1.0 - r) * (1.0 + r));
    if (h == 0.0 && k == 0.0) return 0.25f + asinf((float)r) * 0.15915494309189535f;
    float t1, t2;
    if (h == 0.0) t1 = (k > 0.0) ? 0.25f : (k < 0.0 ? -0.25f : 0.f);
    else t1 = owen_t((float)h, (float)((k - r * h) / (h * s)));
    if (k == 0.0) t2 = (h > 0.0) ? 0.25f : (h < 0.0 ? -0.25f : 0.f);
    else t2 = owen_t((float)k, (float)((h - r * k) / (k * s)));
    const float beta = (h * k < 0.0 || (h * k == 0.0 && h + k < 0.0)) ? 0.5f : 0.f;
    return 0.5f * nrm_cdf((float)h) + 0.5f * nrm_cdf((float)k) - t1 - t2 - beta;
}

// Cholesky factor (pivots floored at fl) of the cell's covariance with its corners taken in
// ascending order of the standardised threshold s (theta - mu_c) / sigma_c (ties: lower corner
// first), and the thresholds s (theta - mu) in that order: the all-below (s = +1) or all-above
// (s = -1) orthant of the ordered estimator.  The order is decided in FP64.
__device__ void ordered_factor(const double (&S)[8][8], const double (&mu)[8], double theta, double s, double fl,
                               CellRec &r)
{
    int perm[8];
    double key[8];
    for (int c = 0; c < 8; ++c) {
        key[c] = (s * (theta - mu[c])) / sqrt(S[c][c]);
        perm[c] = c;
    }
    for (int i = 1; i < 8; ++i) {  // insertion sort, stable
        const int v = perm[i];
        int j = i;
        while (j > 0 && key[v] < key[perm[j - 1]]) {
            perm[j] = perm[j - 1];
            --j;
        }
        perm[j] = v;
    }
    double Lm[8][8];
    for (int a = 0; a < 8; ++a) {
        for (int b = 0; b <= a; ++b) {
            double t = S[perm[a]][perm[b]];
            for (int q = 0; q < b; ++q) t -= Lm[a][q] * Lm[b][q];
            if (a == b) {
                if (!(t > fl)) t = fl;
                Lm[a][a] = sqrt(t);
            } else {
                Lm[a][b] = t / Lm[b][b];
            }
        }
    }
    for (int a = 0; a < 8; ++a) {
        r.b[a] = (float)(s * (theta - mu[perm[a]]));
        for (int b = 0; b <= a; ++b) r.L[tri(a, b)] = (float)Lm[a][b];
    }
}

// CF: 0 = queue records for the sampling estimators, 1 = independent-corner closed form,
// 2 = edge-max closed form (results written in place, no records), 3 = queue records of the
// ordered SOV estimator (the all-below factor in recs, the all-above one in recs2, same index).
template <int CF>
__global__ void k_cell_prep(GridDev g, const double *stats, const int32_t *slot, const int64_t *cells,
                            int64_t count, double theta, double tau, double skip_eps, PairTable pt, float *lcp,
                            bool by_pos, CellRec *recs, unsigned long long *nrec, unsigned long long *nown,
                            int *status, unsigned long long *orth_ctr, CellRec *recs2)
{
    bool closed = false;  // a closed-form estimator evaluated this cell (counted as estimated)
    int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool active = pos < count;
    bool need = false;
    CellRec r, r2;
    int64_t outi = 0;
    if (active) {
        int64_t cidx = cells ? cells[pos] : pos;
        int64_t cx = g.n[0] - 1, cy = g.n[1] - 1;
        if (cidx < 0 || cidx >= cx * cy * (int64_t)(g.n[2] - 1)) {  // listed cell off the grid
            atomicCAS(status, 0, (int)GPR_ERR_ARG);
            active = false;
            cidx = 0;
        }
        outi = by_pos ? pos : cidx;
    }
    if (active) {
        int64_t cidx = cells ? cells[pos] : pos;
        int64_t cx = g.n[0] - 1, cy = g.n[1] - 1;
        int64_t i = cidx % cx, j = (cidx / cx) % cy, k = cidx / (cx * cy);
        const double *row[8];
        double mu[8], S[8][8];
        for (int c = 0; c < 8; ++c) {
            int64_t p = (i + (c & 1)) + (int64_t)g.n[0] * ((j + ((c >> 1) & 1)) + (int64_t)g.n[1] * (k + (c >> 2)));
            int64_t s = slot ? (int64_t)slot[p] : p;
            row[c] = stats + s * 15;
            mu[c] = row[c][0];
            S[c][c] = row[c][1];
        }
        for (int c1 = 0; c1 < 8; ++c1)
            for (int c2 = c1 + 1; c2 < 8; ++c2) {
                double v = pt.owner[c1][c2] == 0 ? row[c1][2 + pt.slot[c1][c2]] : row[c2][2 + pt.slot[c1][c2]];
                S[c1][c2] = v;
                S[c2][c1] = v;
            }
        double maxd = 0.0;
        for (int c = 0; c < 8; ++c) maxd = fmax(maxd, S[c][c]);
        float result = 0.0f;
        if (!(maxd > 1e-30)) {
            bool lo = true, hi = true;
            for (int c = 0; c < 8; ++c) { lo = lo && (mu[c] < theta); hi = hi && (mu[c] > theta); }
            result = (lo || hi) ? 0.0f : 1.0f;
        } else {
            double jit = tau * maxd;
            bool indef = false;
            for (int c = 0; c < 8; ++c) {
                S[c][c] += jit;
                indef = indef || !(S[c][c] > 0.0);
            }
            // P(Y_c > theta), P(Y_c < theta) in FP32 (relative error ~1e-5 down to 1e-30): a test
            // passes only with a 1% margin, so no cell or orthant the FP64 values would keep is dropped
            float sa = 0.f, sb = 0.f, pa[8], pb[8];
            for (int c = 0; c < 8; ++c) {
                const float isd = rsqrtf((float)S[c][c]);
                pa[c] = nrm_cdf((float)(mu[c] - theta) * isd);
                pb[c] = nrm_cdf((float)(theta - mu[c]) * isd);
                sa += pa[c];
                sb += pb[c];
            }
            const float lim = (float)(0.99 * skip_eps);
            if (indef) {
                // a corner variance that stays non-positive after the jitter describes no
                // Gaussian: the cell's LCP is undefined and reported as NaN
                result = nanf("");
            } else if (CF == 1 && !(sa < lim || sb < lim)) {
                // corners taken as independent: 1 - prod P(Y_c < theta) - prod P(Y_c > theta)
                float plo = 1.f, phi = 1.f;
                for (int c = 0; c < 8; ++c) {
                    plo *= pb[c];
                    phi *= pa[c];
                }
                result = fminf(fmaxf(1.f - plo - phi, 0.f), 1.f);
                closed = true;
            } else if (CF == 2 && !(sa < lim || sb < lim)) {
                // largest edge-crossing probability over the 12 edges: P(Y_i < t) + P(Y_j < t) - 2 P(both < t)
                double z[8], isd[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    isd[c] = 1.0 / sqrt(S[c][c]);
                    z[c] = (theta - mu[c]) * isd[c];
                }
                float best = 0.f;
#pragma unroll
                for (int c = 0; c < 8; ++c)
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const int d = c ^ (1 << a);
                        if (d < c) continue;
                        const double r = S[c][d] * isd[c] * isd[d];
                        const double rc = r > 0.9999999999 ? 0.9999999999 : (r < -0.9999999999 ? -0.9999999999 : r);
                        const float pe = pb[c] + pb[d] - 2.f * bvn_lower(z[c], z[d], rc);
                        best = fmaxf(best, pe);
                    }
                result = fminf(fmaxf(best, 0.f), 1.f);
                closed = true;
            } else if (CF == 3 && !(sa < lim || sb < lim)) {
                ordered_factor(S, mu, theta, 1.0, 1e-3 * jit, r);
                ordered_factor(S, mu, theta, -1.0, 1e-3 * jit, r2);
            } else if (CF == 0 && !(sa < lim || sb < lim)) {
                double Lm[8][8];
                double fl = 1e-3 * jit;
                for (int a = 0; a < 8; ++a) {
                    for (int b = 0; b <= a; ++b) {
                        double s = S[a][b];
                        for (int q = 0; q < b; ++q) s -= Lm[a][q] * Lm[b][q];
                        if (a == b) {
                            if (!(s > fl)) s = fl;
                            Lm[a][a] = sqrt(s);
                        } else {
                            Lm[a][b] = s / Lm[b][b];
                        }
                    }
                }
                for (int a = 0; a < 8; ++a) {
                    r.b[a] = (float)(theta - mu[a]);
                    for (int b = 0; b <= a; ++b) r.L[tri(a, b)] = (float)Lm[a][b];
                }
            }
            if ((CF == 0 || CF == 3) && !indef && !(sa < lim || sb < lim)) {
                // Frechet bound: P(all < theta) <= min_c P(Y_c < theta) (and likewise above).  An
                // orthant bounded below 1e-7 is taken as 0: the LCP moves by less than 1e-7.
                float mlo = 1.f, mhi = 1.f;
                for (int c = 0; c < 8; ++c) {
                    mlo = fminf(mlo, pb[c]);
                    mhi = fminf(mhi, pa[c]);
                }
                int64_t mask = (mlo < 0.99e-7f ? 1 : 0) | (mhi < 0.99e-7f ? 2 : 0);
                r.cell = cidx | (mask << 56);
                r.out = lcp + outi;
                need = true;
            }
        }
        if (!need) lcp[outi] = result;
    }
    if (CF == 1 || CF == 2) {  // closed-form estimators: count the cells they evaluated (no records)
        const unsigned cmask = __ballot_sync(0xffffffffu, closed);
        if (cmask && (threadIdx.x & 31) == __ffs(cmask) - 1) atomicAdd(nrec, (unsigned long long)__popc(cmask));
        return;
    }
    // warp-aggregated append of the cells that need the estimator
    unsigned mask = __ballot_sync(0xffffffffu, need);
    if (!mask) return;
    if (orth_ctr) {  // tracing: orthants the estimator will integrate (the Frechet test drops some)
        const unsigned no = need ? 2u - (unsigned)__popcll((unsigned long long)(r.cell >> 56) & 3ull) : 0u;
        const unsigned tot = __reduce_add_sync(0xffffffffu, no);
        if ((threadIdx.x & 31) == 0 && tot) atomicAdd(orth_ctr, (unsigned long long)tot);
    }
    int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) {
        base = atomicAdd(nrec, (unsigned long long)__popc(mask));
        if (nown) atomicAdd(nown, (unsigned long long)__popc(mask));
    }
    base = __shfl_sync(0xffffffffu, base, leader);
    if (need) {
        const unsigned long long at = base + __popc(mask & ((1u << lane) - 1));
        recs[at] = r;
        if (CF == 3) {
            r2.cell = r.cell;
            r2.out = r.out;
            recs2[at] = r2;
        }
    }
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// odd multiples of 2^-24 in (0,1): exact in binary32
__device__ __forceinline__ float u01f(uint32_t x) { return (float)(((x >> 9) << 1) | 1u) * (1.0f / 16777216.0f); }

__global__ void k_normal_eval(const float *x, int64_t n, float *cdf, float *ppf)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    cdf[i] = nrm_cdf(x[i]);
    ppf[i] = (x[i] > 0.0f && x[i] < 1.0f) ? nrm_ppf(x[i]) : 0.0f;
}

struct Lattice {
    uint32_t G[7];
};

// Lattice coordinate |2u - 1| of u = (2k + 1) 2^-24, k = U >> 9 (odd multiples of 2^-24): from the
// float 1 + k 2^-23, 2u - 1 = (2 (1 + k 2^-23) - 3) + 2^-23, each step exact in binary32.
__device__ __forceinline__ float lattice_w(uint32_t U)
{
    const float one_k = __uint_as_float(0x3F800000u | (U >> 9));
    return fabsf(fmaf(2.0f, one_k, -3.0f) + 1.1920929e-07f);
}

// One orthant of the SOV recursion for two samples at once (independent chains, interleaved):
// e_i = Phi(c_i - sum_j Ls_ij z_j) with the rows pre-scaled by 1/L_ii, f = prod e_i,
// z_i = Phi^-1(w_i e_i).  An underflowed product stays 0 (z from the clamped argument).
// The first factor e_0 = Phi(c_0) does not depend on the sample: the caller passes it.
__device__ __forceinline__ void sov_pair(const float (&Ls)[28], const float (&cb)[8], float sg, float e_first,
                                         const float (&w0)[7], const float (&w1)[7], float &f0, float &f1)
{
    float z0[7], z1[7];
    f0 = e_first;
    f1 = e_first;
    z0[0] = nrm_ppf(fmaxf(w0[0] * e_first, 1e-37f));
    z1[0] = nrm_ppf(fmaxf(w1[0] * e_first, 1e-37f));
#pragma unroll
    for (int i = 1; i < 8; ++i) {
        float a0 = sg * cb[i], a1 = a0;
#pragma unroll
        for (int j = 0; j < i; ++j) {
            a0 = fmaf(-Ls[i * (i - 1) / 2 + j], z0[j], a0);
            a1 = fmaf(-Ls[i * (i - 1) / 2 + j], z1[j], a1);
        }
        const float e0 = nrm_cdf(a0), e1 = nrm_cdf(a1);
        f0 *= e0;
        f1 *= e1;
        if (i < 7) {
            z0[i] = nrm_ppf(fmaxf(w0[i] * e0, 1e-37f));
            z1[i] = nrm_ppf(fmaxf(w1[i] * e1, 1e-37f));
        }
    }
}

// MINB: CTAs per SM the register allocation targets (2: 111 registers, 3: 80, both without
// spills); the autotuner picks the variant and the grid.
template <int MINB>
__global__ void __launch_bounds__(256, MINB) k_sov(const CellRec *recs, const unsigned long long *nrec,
                                                  unsigned long long *ticket, int N, uint64_t seed, Lattice lat)
{
    int lane = threadIdx.x & 31;
    int64_t n = (int64_t)*nrec;
    // records taken from a ticket counter, one per warp at a time: records whose Frechet test
    // dropped an orthant cost half, so a fixed stride would leave some warps with more work
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(ticket, 1ull);
        const int64_t q = (int64_t)__shfl_sync(0xffffffffu, t, 0);
        if (q >= n) break;
        const CellRec &r = recs[q];
        float Ls[28], cb[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float inv = 1.0f / r.L[tri(i, i)];
            cb[i] = r.b[i] * inv;
#pragma unroll
            for (int j = 0; j < i; ++j) Ls[i * (i - 1) / 2 + j] = r.L[tri(i, j)] * inv;
        }
        const uint64_t cellid = (uint64_t)r.cell & ((1ull << 56) - 1);
        const int skip = (int)((uint64_t)r.cell >> 56);
        uint32_t D = 0;
        if (lane < 7) D = (uint32_t)(splitmix64(seed, cellid * 8 + lane + 1) >> 32);
        uint32_t Ds[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) Ds[i] = __shfl_sync(0xffffffffu, D, i);
        float acc_lo = 0.f, acc_hi = 0.f;  // <= 50 samples per lane: FP32 sums are exact to ~1e-7
        const float e_first_lo = nrm_cdf(cb[0]), e_first_hi = nrm_cdf(-cb[0]);
        for (int k = lane; k < N; k += 64) {
            const bool two = k + 32 < N;
            float w0[7], w1[7];
#pragma unroll
            for (int i = 0; i < 7; ++i) {
                w0[i] = lattice_w((uint32_t)k * lat.G[i] + Ds[i]);
                w1[i] = lattice_w((uint32_t)(k + 32) * lat.G[i] + Ds[i]);
            }
#pragma unroll 1
            for (int side = 0; side < 2; ++side) {  // one copy of the recursion (instruction cache)
                if (skip & (1 << side)) continue;
                float f0, f1;
                sov_pair(Ls, cb, side ? -1.0f : 1.0f, side ? e_first_hi : e_first_lo, w0, w1, f0, f1);
                const float f = two ? f0 + f1 : f0;
                if (side) acc_hi += f; else acc_lo += f;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc_lo += __shfl_xor_sync(0xffffffffu, acc_lo, o);
            acc_hi += __shfl_xor_sync(0xffffffffu, acc_hi, o);
        }
        if (lane == 0) {
            double v = 1.0 - (double)acc_lo / N - (double)acc_hi / N;
            *r.out = (float)(v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v));
        }
    }
}

// The ordered SOV estimator: the same lattice and recursion as k_sov, but each orthant has its own
// factor and signed thresholds (all-below from recs, all-above from recs2, same index), so the
// two orthants run one after the other with the lattice coordinates recomputed for each.
template <int MINB>
__global__ void __launch_bounds__(256, MINB) k_sov_ord(const CellRec *recs, const CellRec *recs2,
                                                      const unsigned long long *nrec, unsigned long long *ticket,
                                                      int N, uint64_t seed, Lattice lat)
{
    int lane = threadIdx.x & 31;
    int64_t n = (int64_t)*nrec;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(ticket, 1ull);
        const int64_t q = (int64_t)__shfl_sync(0xffffffffu, t, 0);
        if (q >= n) break;
        const uint64_t cellid = (uint64_t)recs[q].cell & ((1ull << 56) - 1);
        const int skip = (int)((uint64_t)recs[q].cell >> 56);
        uint32_t D = 0;
        if (lane < 7) D = (uint32_t)(splitmix64(seed, cellid * 8 + lane + 1) >> 32);
        uint32_t Ds[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) Ds[i] = __shfl_sync(0xffffffffu, D, i);
        float acc_lo = 0.f, acc_hi = 0.f;
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
            if (skip & (1 << side)) continue;
            const CellRec &r = side ? recs2[q] : recs[q];
            float Ls[28], cb[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float inv = 1.0f / r.L[tri(i, i)];
                cb[i] = r.b[i] * inv;
#pragma unroll
                for (int j = 0; j < i; ++j) Ls[i * (i - 1) / 2 + j] = r.L[tri(i, j)] * inv;
            }
            const float e_first = nrm_cdf(cb[0]);
            float a = 0.f;
            for (int k = lane; k < N; k += 64) {
                const bool two = k + 32 < N;
                float w0[7], w1[7];
#pragma unroll
                for (int i = 0; i < 7; ++i) {
                    w0[i] = lattice_w((uint32_t)k * lat.G[i] + Ds[i]);
                    w1[i] = lattice_w((uint32_t)(k + 32) * lat.G[i] + Ds[i]);
                }
                float f0, f1;
                sov_pair(Ls, cb, 1.0f, e_first, w0, w1, f0, f1);
                a += two ? f0 + f1 : f0;
            }
            if (side) acc_hi = a; else acc_lo = a;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc_lo += __shfl_xor_sync(0xffffffffu, acc_lo, o);
            acc_hi += __shfl_xor_sync(0xffffffffu, acc_hi, o);
        }
        if (lane == 0) {
            double v = 1.0 - (double)acc_lo / N - (double)acc_hi / N;
            *recs[q].out = (float)(v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v));
        }
    }
}

// Philox-4x32-10 (Salmon et al., SC'11).
__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

__global__ void k_mc(const CellRec *recs, const unsigned long long *nrec, int N, uint64_t seed)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t n = (int64_t)*nrec;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int64_t q = warp; q < n; q += nw) {
        const CellRec &r = recs[q];
        float L[36], b[8];
#pragma unroll
        for (int t = 0; t < 36; ++t) L[t] = r.L[t];
#pragma unroll
        for (int t = 0; t < 8; ++t) b[t] = r.b[t];
        const uint64_t cellid = (uint64_t)r.cell & ((1ull << 56) - 1);
        uint32_t clo = (uint32_t)cellid, chi = (uint32_t)(cellid >> 32);
        int crossed = 0;
        for (int k = lane; k < N; k += 32) {
            float z[8];
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                uint32_t c[4] = {(uint32_t)k, clo, chi, (uint32_t)rr};
                philox(c, k0, k1);
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    float u1 = u01f(c[2 * p]), u2 = u01f(c[2 * p + 1]);
                    float rad = sqrtf(-2.0f * logf(u1));
                    float sn, cs;
                    sincospif(2.0f * u2, &sn, &cs);
                    z[4 * rr + 2 * p] = rad * cs;
                    z[4 * rr + 2 * p + 1] = rad * sn;
                }
            }
            bool all_lo = true, all_hi = true;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float s = 0.0f;
#pragma unroll
                for (int j = 0; j <= i; ++j) s = fmaf(L[tri(i, j)], z[j], s);
                all_lo = all_lo && (s < b[i]);
                all_hi = all_hi && (s > b[i]);
            }
            crossed += (all_lo || all_hi) ? 0 : 1;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) crossed += __shfl_xor_sync(0xffffffffu, crossed, o);
        if (lane == 0) *r.out = (float)((double)crossed / (double)N);
    }
}

Lattice make_lattice()
{
    static const int primes[7] = {2, 3, 5, 7, 11, 13, 17};
    Lattice L;
    for (int i = 0; i < 7; ++i) {
        double s = sqrt((double)primes[i]);
        L.G[i] = (uint32_t)floor((s - floor(s)) * 4294967296.0);
    }
    return L;
}

}  // namespace

// records and, for the ordered estimator, the parallel all-above records
size_t cell_lcp_scratch_bytes(int64_t count, int est)
{
    return (est == GPR_EST_SOV_ORDERED ? 2 : 1) * Carver::round(sizeof(CellRec) * (size_t)count) + 256;
}

namespace {
thread_local RecordSink *tl_sink = nullptr;
}

void set_record_sink(RecordSink *sink) { tl_sink = sink; }
size_t record_bytes() { return sizeof(CellRec); }

void launch_estimator(const void *recs, const void *recs2, unsigned long long *nrec, int64_t max_records,
                      const LcpOpts &o, cudaStream_t st)
{
    // one warp per record, persistent over the device count (nrec[0]; nrec[1] is the work ticket);
    // the register variant and the CTAs per SM are chosen by the autotuner
    static const int per_sm[4] = {2, 8, 3, 12};
    auto run = [&](int c) -> gpr_status {
        int64_t blocks = (max_records + 7) / 8;
        if (blocks > (int64_t)num_sms() * per_sm[c]) blocks = (int64_t)num_sms() * per_sm[c];
        if (blocks < 1) blocks = 1;
        if (o.est == GPR_EST_SOV_ORDERED) {
            static Lattice lat = make_lattice();
            GPR_CUDA_TRY(cudaMemsetAsync(nrec + 1, 0, sizeof(unsigned long long), st));
            ProfScope _ps("sov_ordered", st);
            if (c < 2)
                k_sov_ord<2><<<(unsigned)blocks, 256, 0, st>>>((const CellRec *)recs, (const CellRec *)recs2, nrec,
                                                               nrec + 1, o.n_samples, o.seed, lat);
            else
                k_sov_ord<3><<<(unsigned)blocks, 256, 0, st>>>((const CellRec *)recs, (const CellRec *)recs2, nrec,
                                                               nrec + 1, o.n_samples, o.seed, lat);
        } else if (o.est == GPR_EST_SOV_QMC) {
            static Lattice lat = make_lattice();
            GPR_CUDA_TRY(cudaMemsetAsync(nrec + 1, 0, sizeof(unsigned long long), st));
            ProfScope _ps("sov", st);
            if (c < 2)
                k_sov<2><<<(unsigned)blocks, 256, 0, st>>>((const CellRec *)recs, nrec, nrec + 1, o.n_samples, o.seed,
                                                           lat);
            else
                k_sov<3><<<(unsigned)blocks, 256, 0, st>>>((const CellRec *)recs, nrec, nrec + 1, o.n_samples, o.seed,
                                                           lat);
        } else {
            ProfScope _ps("mc", st);
            k_mc<<<(unsigned)blocks, 256, 0, st>>>((const CellRec *)recs, nrec, o.n_samples, o.seed);
        }
        note_launch();
        GPR_CUDA_TRY(cudaGetLastError());
        return GPR_OK;
    };
    const bool sov = o.est == GPR_EST_SOV_QMC || o.est == GPR_EST_SOV_ORDERED;
    tune_run(o.est == GPR_EST_SOV_QMC ? "sov_shape" : (sov ? "sov_ordered_shape" : "mc_ctas_per_sm"),
             tune_bucket(max_records), sov ? 4 : 3, run, st);
}

gpr_status run_cell_lcp(const GridDev &g, const double *stats, const int32_t *slot, const int64_t *cells,
                        int64_t count, const LcpOpts &o, float *lcp, bool by_pos, void *scratch,
                        size_t scratch_bytes, int64_t *n_estimated, cudaStream_t st)
{
    if (count <= 0) {
        if (n_estimated) *n_estimated = 0;
        return GPR_OK;
    }
    if (scratch_bytes < cell_lcp_scratch_bytes(count, o.est)) return GPR_ERR_ARG;
    Carver cv{(char *)scratch};
    unsigned long long *nrec = cv.take<unsigned long long>(2);  // record count, estimator ticket
    CellRec *recs = cv.take<CellRec>((size_t)count);
    const bool ordered = o.est == GPR_EST_SOV_ORDERED;
    CellRec *recs2 = ordered ? cv.take<CellRec>((size_t)count) : nullptr;  // all-above records
    // a batch sink with room takes the records; its owner runs one estimator launch for all
    RecordSink *sink = tl_sink;
    bool to_sink = false;
    const bool closed = o.est == GPR_EST_INDEP || o.est == GPR_EST_EDGE_MAX;  // no records, no estimator
    if (sink && !closed && (!ordered || sink->recs2)) {
        int64_t cur = sink->reserved->load();
        while (cur + count <= sink->capacity && !sink->reserved->compare_exchange_weak(cur, cur + count)) {
        }
        to_sink = cur + count <= sink->capacity;
    }
    GPR_CUDA_TRY(cudaMemsetAsync(nrec, 0, sizeof(unsigned long long), st));
    static PairTable pt = make_pair_table();
    int *status = gpr_status_word();
    if (!status) return GPR_ERR_CUDA;
    {
        ProfScope _ps("cell_prep", st);
        const unsigned nb = (unsigned)((count + 127) / 128);
        if (o.est == GPR_EST_INDEP)
            k_cell_prep<1><<<nb, 128, 0, st>>>(g, stats, slot, cells, count, o.theta, o.tau, o.skip_eps, pt, lcp,
                                               by_pos, recs, nrec, nullptr, status, nullptr, nullptr);
        else if (o.est == GPR_EST_EDGE_MAX)
            k_cell_prep<2><<<nb, 128, 0, st>>>(g, stats, slot, cells, count, o.theta, o.tau, o.skip_eps, pt, lcp,
                                               by_pos, recs, nrec, nullptr, status, nullptr, nullptr);
        else if (ordered)
            k_cell_prep<3><<<nb, 128, 0, st>>>(
                g, stats, slot, cells, count, o.theta, o.tau, o.skip_eps, pt, lcp, by_pos,
                to_sink ? (CellRec *)sink->recs : recs, to_sink ? sink->nrec : nrec, to_sink ? nrec : nullptr,
                status, prof_counter(PROF_CTR_ORTHANTS), to_sink ? (CellRec *)sink->recs2 : recs2);
        else
            k_cell_prep<0><<<nb, 128, 0, st>>>(
                g, stats, slot, cells, count, o.theta, o.tau, o.skip_eps, pt, lcp, by_pos,
                to_sink ? (CellRec *)sink->recs : recs, to_sink ? sink->nrec : nrec, to_sink ? nrec : nullptr,
                status, prof_counter(PROF_CTR_ORTHANTS), nullptr);
    }
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    if (!to_sink && !closed) launch_estimator(recs, recs2, nrec, count, o, st);
    GPR_CUDA_TRY(cudaGetLastError());
    if (n_estimated) {
        unsigned long long h = 0;
        GPR_CUDA_TRY(cudaMemcpyAsync(&h, nrec, sizeof h, cudaMemcpyDeviceToHost, st));
        GPR_CUDA_TRY(cudaStreamSynchronize(st));
        *n_estimated = (int64_t)h;
    }
    return GPR_OK;
}

// ------------------------------------------------------------ pre-classification

// Widened Boole test of the pre-classification in FP32: the estimator's Phi is accurate to ~1e-5
// relative down to 1e-30, so a cell is dropped only when a sum is below 0.99 skip_eps (never a cell
// the FP64 test with the same margins keeps; the few extra cells are dropped by the exact test).
__device__ __forceinline__ uint8_t classify_keep(const double (&mu)[8], const double (&v)[8], double maxv,
                                                 double theta, double skip_eps, double tau, double mm)
{
    float sa = 0.f, sb = 0.f;
    for (int c = 0; c < 8; ++c) {
        const float isd = rsqrtf((float)(v[c] + tau * maxv));
        sa += nrm_cdf((float)(mu[c] + mm - theta) * isd);
        sb += nrm_cdf((float)(theta - mu[c] + mm) * isd);
    }
    const float lim = (float)(0.99 * skip_eps);
    return (sa < lim || sb < lim) ? 0 : 1;
}

__global__ void k_classify(GridDev g, const float *mean, const float *var, double theta, double skip_eps,
                           double tau, double mv, double mm, uint8_t *keep)
{
    int64_t cidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t cx = g.n[0] - 1, cy = g.n[1] - 1, cz = g.n[2] - 1;
    if (cidx >= cx * cy * cz) return;
    int64_t i = cidx % cx, j = (cidx / cx) % cy, k = cidx / (cx * cy);
    double mu[8], v[8], maxv = 0.0;
    for (int c = 0; c < 8; ++c) {
        int64_t p = (i + (c & 1)) + (int64_t)g.n[0] * ((j + ((c >> 1) & 1)) + (int64_t)g.n[1] * (k + (c >> 2)));
        mu[c] = mean[p];
        v[c] = fmax((double)var[p], 0.0) + mv;
        maxv = fmax(maxv, v[c]);
    }
    keep[cidx] = classify_keep(mu, v, maxv, theta, skip_eps, tau, mm);
}

void launch_classify_cells(const GridDev &g, const float *mean, const float *var, double theta, double skip_eps,
                           double tau, double margin_var, double margin_mu, uint8_t *keep, cudaStream_t st)
{
    {
        ProfScope _ps("classify", st);
        k_classify<<<(unsigned)((g.ncells() + 255) / 256), 256, 0, st>>>(g, mean, var, theta, skip_eps, tau,
                                                                     margin_var, margin_mu, keep);
    }
    note_launch();
}

__global__ void k_mark_corners(GridDev g, const uint8_t *keep, uint8_t *flag)
{
    int64_t cidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t cx = g.n[0] - 1, cy = g.n[1] - 1, cz = g.n[2] - 1;
    if (cidx >= cx * cy * cz || !keep[cidx]) return;
    int64_t i = cidx % cx, j = (cidx / cx) % cy, k = cidx / (cx * cy);
    for (int c = 0; c < 8; ++c) {
        int64_t p = (i + (c & 1)) + (int64_t)g.n[0] * ((j + ((c >> 1) & 1)) + (int64_t)g.n[1] * (k + (c >> 2)));
        flag[p] = 1;
    }
}

__global__ void k_classify_mv(GridDev g, const float2 *mvt, double theta, double skip_eps, double tau, double mv,
                              double mm, uint8_t *keep)
{
    int64_t cidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t cx = g.n[0] - 1, cy = g.n[1] - 1, cz = g.n[2] - 1;
    if (cidx >= cx * cy * cz) return;
    int64_t i = cidx % cx, j = (cidx / cx) % cy, k = cidx / (cx * cy);
    double mu[8], v[8], maxv = 0.0;
    for (int c = 0; c < 8; ++c) {
        int64_t p = (i + (c & 1)) + (int64_t)g.n[0] * ((j + ((c >> 1) & 1)) + (int64_t)g.n[1] * (k + (c >> 2)));
        float2 t = mvt[p];
        mu[c] = t.x;
        v[c] = fmax((double)t.y, 0.0) + mv;
        maxv = fmax(maxv, v[c]);
    }
    keep[cidx] = classify_keep(mu, v, maxv, theta, skip_eps, tau, mm);
}

void launch_classify_cells_mv(const GridDev &g, const float2 *mvt, double theta, double skip_eps, double tau,
                              double margin_var, double margin_mu, uint8_t *keep, cudaStream_t st)
{
    {
        ProfScope _ps("classify", st);
        k_classify_mv<<<(unsigned)((g.ncells() + 255) / 256), 256, 0, st>>>(g, mvt, theta, skip_eps, tau, margin_var,
                                                                           margin_mu, keep);
    }
    note_launch();
}

void launch_mark_corners(const GridDev &g, const uint8_t *keep_cell, uint8_t *point_flag, cudaStream_t st)
{
    k_mark_corners<<<(unsigned)((g.ncells() + 255) / 256), 256, 0, st>>>(g, keep_cell, point_flag);
    note_launch();
}

// ------------------------------------------------------------ stream compaction

static constexpr int CHUNK = 4096;  // flags per block

__global__ void k_count(const uint8_t *flag, int64_t n, unsigned *counts)
{
    __shared__ unsigned wsum[32];
    int64_t base = (int64_t)blockIdx.x * CHUNK;
    unsigned c = 0;
    for (int t = threadIdx.x; t < CHUNK; t += blockDim.x) {
        int64_t i = base + t;
        if (i < n && flag[i]) ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wsum[w];
        counts[blockIdx.x] = s;
    }
}

// Exclusive scan of nb block counts in one block (serial over chunks of 1024).
__global__ void k_scan_counts(const unsigned *counts, int64_t nb, unsigned long long *offs, unsigned long long *total)
{
    __shared__ unsigned long long sh[1024];
    unsigned long long carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
        int64_t i = b0 + threadIdx.x;
        unsigned long long v = i < nb ? counts[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            unsigned long long t = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) offs[i] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        carry += sh[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scatter(const uint8_t *flag, int64_t n, const unsigned long long *offs, int64_t *out_idx,
                          int32_t *slot)
{
    __shared__ unsigned wsum[32];
    int64_t base = (int64_t)blockIdx.x * CHUNK;
    unsigned long long run = offs[blockIdx.x];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t0 = 0; t0 < CHUNK; t0 += blockDim.x) {
        int64_t i = base + t0 + threadIdx.x;
        bool f = i < n && flag[i];
        unsigned m = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wsum[w] = __popc(m);
        __syncthreads();
        unsigned before = 0, tot = 0;
        for (int q = 0; q < nw; ++q) {
            if (q < w) before += wsum[q];
            tot += wsum[q];
        }
        unsigned long long pos = run + before + __popc(m & ((1u << lane) - 1));
        if (i < n) {
            if (f) out_idx[pos] = i;
            if (slot) slot[i] = f ? (int32_t)pos : -1;
        }
        run += tot;
        __syncthreads();
    }
}

size_t compact_scratch_bytes(int64_t n)
{
    int64_t nb = (n + CHUNK - 1) / CHUNK;
    return Carver::round(sizeof(unsigned) * nb) + Carver::round(sizeof(unsigned long long) * nb) + 512;
}

gpr_status compact_flags(const uint8_t *flag, int64_t n, int64_t *out_idx, int32_t *slot, int64_t *count_host,
                         void *scratch, size_t scratch_bytes, cudaStream_t st)
{
    if (scratch_bytes < compact_scratch_bytes(n)) return GPR_ERR_ARG;
    int64_t nb = (n + CHUNK - 1) / CHUNK;
    Carver cv{(char *)scratch};
    unsigned *counts = cv.take<unsigned>(nb);
    unsigned long long *offs = cv.take<unsigned long long>(nb);
    unsigned long long *total = cv.take<unsigned long long>(1);
    k_count<<<(unsigned)nb, 256, 0, st>>>(flag, n, counts);
    note_launch();
    k_scan_counts<<<1, 1024, 0, st>>>(counts, nb, offs, total);
    note_launch();
    k_scatter<<<(unsigned)nb, 256, 0, st>>>(flag, n, offs, out_idx, slot);
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    unsigned long long h = 0;
    GPR_CUDA_TRY(cudaMemcpyAsync(&h, total, sizeof h, cudaMemcpyDeviceToHost, st));
    GPR_CUDA_TRY(cudaStreamSynchronize(st));
    *count_host = (int64_t)h;
    return GPR_OK;
}

// Bricked order of the grid points: 8 x 8 x 8 bricks (clipped at the far faces), bricks x-fastest
// within 8-row bands, bands within 8-plane slabs; x-fastest inside a brick.  t -> point index.
__device__ __forceinline__ int64_t brick_point(const GridDev &g, int64_t t)
{
    const int64_t nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int64_t slab = nx * ny * 8;
    int64_t bz = t / slab;
    const int64_t nbz = (nz + 7) / 8;
    if (bz > nbz - 1) bz = nbz - 1;
    t -= bz * slab;
    const int64_t hz = nz - 8 * bz < 8 ? nz - 8 * bz : 8;
    const int64_t band = nx * 8 * hz;
    int64_t by = t / band;
    const int64_t nby = (ny + 7) / 8;
    if (by > nby - 1) by = nby - 1;
    t -= by * band;
    const int64_t hy = ny - 8 * by < 8 ? ny - 8 * by : 8;
    const int64_t brick = 8 * hy * hz;
    int64_t bx = t / brick;
    const int64_t nbx = (nx + 7) / 8;
    if (bx > nbx - 1) bx = nbx - 1;
    t -= bx * brick;
    const int64_t hx = nx - 8 * bx < 8 ? nx - 8 * bx : 8;
    const int64_t lx = t % hx, ly = (t / hx) % hy, lz = t / (hx * hy);
    return (8 * bx + lx) + nx * ((8 * by + ly) + ny * (8 * bz + lz));
}

__global__ void k_brick_gather(GridDev g, const uint8_t *flag, uint8_t *bflag)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < (int64_t)g.n[0] * g.n[1] * g.n[2]) bflag[t] = flag[brick_point(g, t)];
}

__global__ void k_brick_map(GridDev g, int64_t *list, int64_t count, int32_t *slot)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t p = brick_point(g, list[i]);
    list[i] = p;
    if (slot) slot[p] = (int32_t)i;
}

gpr_status compact_flags_bricked(const GridDev &g, const uint8_t *flag, uint8_t *bflag, int64_t *out_idx,
                                 int32_t *slot, int64_t *count_host, void *scratch, size_t scratch_bytes,
                                 cudaStream_t st)
{
    const int64_t n = g.npts();
    k_brick_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, flag, bflag);
    note_launch();
    if (slot) GPR_CUDA_TRY(cudaMemsetAsync(slot, 0xff, sizeof(int32_t) * (size_t)n, st));
    GPR_TRY(compact_flags(bflag, n, out_idx, nullptr, count_host, scratch, scratch_bytes, st));
    if (*count_host > 0) {
        k_brick_map<<<(unsigned)((*count_host + 255) / 256), 256, 0, st>>>(g, out_idx, *count_host, slot);
        note_launch();
    }
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

// Same two stages as run_cell_lcp, on caller-provided scratch: `scratch` holds the record
// counter (first 256 bytes) and then `max_records` CellRec records; `status` receives
// GPR_ERR_ARG for listed cells off the grid.  Queues work only (no allocation, no sync).
size_t cell_rec_bytes() { return sizeof(CellRec); }

gpr_status run_cell_lcp_on_scratch(const GridDev &g, const double *stats, const int64_t *cells, int64_t count,
                                   const LcpOpts &o, float *lcp, bool by_pos, void *scratch, int64_t max_records,
                                   int *status, cudaStream_t st)
{
    if (o.est == GPR_EST_SOV_ORDERED) return GPR_ERR_UNSUPPORTED;  // one record per cell only
    if (count <= 0) return GPR_OK;
    if (count > max_records) return GPR_ERR_ARG;
    unsigned long long *nrec = (unsigned long long *)scratch;  // record count, estimator ticket
    CellRec *recs = (CellRec *)((char *)scratch + 256);
    GPR_CUDA_TRY(cudaMemsetAsync(nrec, 0, 2 * sizeof(unsigned long long), st));
    static PairTable pt = make_pair_table();
    const unsigned nb = (unsigned)((count + 127) / 128);
    if (o.est == GPR_EST_INDEP)
        k_cell_prep<1><<<nb, 128, 0, st>>>(g, stats, nullptr, cells, count, o.theta, o.tau, o.skip_eps, pt, lcp,
                                           by_pos, recs, nrec, nullptr, status, nullptr, nullptr);
    else if (o.est == GPR_EST_EDGE_MAX)
        k_cell_prep<2><<<nb, 128, 0, st>>>(g, stats, nullptr, cells, count, o.theta, o.tau, o.skip_eps, pt, lcp,
                                           by_pos, recs, nrec, nullptr, status, nullptr, nullptr);
    else
        k_cell_prep<0><<<nb, 128, 0, st>>>(g, stats, nullptr, cells, count, o.theta, o.tau, o.skip_eps, pt, lcp,
                                           by_pos, recs, nrec, nullptr, status, nullptr, nullptr);
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    if (o.est == GPR_EST_INDEP || o.est == GPR_EST_EDGE_MAX) return GPR_OK;  // evaluated in place
    int64_t blocks = (count + 7) / 8;
    if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
    if (o.est == GPR_EST_SOV_QMC) {
        static Lattice lat = make_lattice();
        k_sov<2><<<(unsigned)blocks, 256, 0, st>>>(recs, nrec, nrec + 1, o.n_samples, o.seed, lat);
    } else {
        k_mc<<<(unsigned)blocks, 256, 0, st>>>(recs, nrec, o.n_samples, o.seed);
    }
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

// Test hook (not in the public header): the estimator's FP32 normal CDF of every x and its
// quantile of every x in (0, 1) (0 elsewhere).  x, cdf, ppf: device, n floats.
extern "C" gpr_status gpr_normal_approx_eval(const float *x, int64_t n, float *cdf, float *ppf, void *stream)
{
    if (n < 0 || (n > 0 && (!x || !cdf || !ppf))) return GPR_ERR_ARG;
    if (n == 0) return GPR_OK;
    k_normal_eval<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, n, cdf, ppf);
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}
