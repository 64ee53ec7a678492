// Model set-up on the device (Sec. 3 / Eq. 1 precomputation): Kt = K(X,X) + sn2 I,
// blocked FP64 Cholesky, L^-1, v = L^-1 y, alpha = Kt^-1 y, latent posterior at the
// observations, and the whitening operand BT = L^-T in FP64 and FP32.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include "internal.h"

static constexpr int NB = 32;  // Cholesky block size

// The status word is a module global, so every device that loads the library has its own copy
// (zero at load); its device address is resolved once per device, with that device current.
static __device__ int g_status_word;
static constexpr int kMaxDevices = 128;

int *gpr_status_word()
{
    static std::mutex mu;
    static int *addr[kMaxDevices] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_status_word);
        if (e != cudaSuccess || !p) {
            gpr_internal_note_cuda_error(e, "cudaGetSymbolAddress(g_status_word)", __LINE__);
            return nullptr;
        }
        addr[dev] = (int *)p;
    }
    return addr[dev];
}

static char g_last_err[256];
void gpr_internal_note_cuda_error(cudaError_t e, const char *what, int line)
{
    snprintf(g_last_err, sizeof g_last_err, "%s (%s) at line %d", cudaGetErrorString(e), what, line);
    if (getenv("GPR_VERBOSE")) fprintf(stderr, "gpr_lcp: %s\n", g_last_err);
}

int num_sms()
{
    static std::atomic<int> cached[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
    int n = cached[dev].load();
    if (!n) {
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
        cached[dev] = n;
    }
    return n;
}

__device__ __forceinline__ double kern64(const KernParams &kp, const double *a, const double *b)
{
    double r2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double t = (a[d] - b[d]) / kp.ell[d];
        r2 += t * t;
    }
    if (kp.kind == GPR_K_SE) return kp.sf2 * exp(-0.5 * r2);
    double r = sqrt(r2), s5r = 2.2360679774997896964 * r;
    return kp.sf2 * (1.0 + s5r + (5.0 / 3.0) * r2) * exp(-s5r);
}

// Kt padded to mb x mb with the identity on the padding.
__global__ void k_build_K(const double *X, int64_t m, int64_t mb, KernParams kp, double sn2, double *A)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= mb * mb) return;
    int64_t i = idx / mb, j = idx % mb;
    double v;
    if (i < m && j < m) v = kern64(kp, X + 3 * i, X + 3 * j) + (i == j ? sn2 : 0.0);
    else v = (i == j) ? 1.0 : 0.0;
    A[idx] = v;
}

// Unblocked Cholesky of the diagonal block kb (one warp; lane = row of the block).
__global__ void k_potrf_diag(double *A, int64_t mb, int kb, int *status)
{
    __shared__ double S[NB][NB + 1];
    int lane = threadIdx.x;
    int64_t r0 = (int64_t)kb * NB;
    for (int c = 0; c < NB; ++c) S[lane][c] = A[(r0 + lane) * mb + r0 + c];
    __syncwarp();
    for (int j = 0; j < NB; ++j) {
        double piv = S[j][j];
        bool bad = !(piv > 0.0);
        if (bad) {
            if (lane == 0) atomicCAS(status, 0, (int)GPR_ERR_NOT_PD);
            piv = 1.0;  // keep going with finite numbers; the status word reports the failure
        }
        const double inv = rsqrt(piv);  // one reciprocal square root for the pivot and the column
        const double ljj = piv * inv;
        __syncwarp();
        if (lane == j) S[j][j] = ljj;
        if (lane > j) S[lane][j] *= inv;
        __syncwarp();
        if (lane > j) {
            double lij = S[lane][j];
            for (int k = j + 1; k <= lane; ++k) S[lane][k] -= lij * S[k][j];
        }
        __syncwarp();
    }
    for (int c = 0; c < NB; ++c) A[(r0 + lane) * mb + r0 + c] = (c <= lane) ? S[lane][c] : 0.0;
}

// Panel solve: rows below block kb, A[r][kb-block] <- A[r][kb-block] L_kk^-T (thread per row).
__global__ void k_trsm_panel(double *A, int64_t mb, int kb)
{
    __shared__ double Lk[NB][NB + 1];
    __shared__ double rd[NB];  // 1 / L_cc: one division per column instead of one per row and column
    int64_t r0 = (int64_t)kb * NB;
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) Lk[t / NB][t % NB] = A[(r0 + t / NB) * mb + r0 + t % NB];
    if (threadIdx.x < NB) rd[threadIdx.x] = 1.0 / A[(r0 + threadIdx.x) * mb + r0 + threadIdx.x];
    __syncthreads();
    int64_t row = r0 + NB + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row >= mb) return;
    double x[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) x[c] = A[row * mb + r0 + c];
#pragma unroll
    for (int c = 0; c < NB; ++c) {
        double s = x[c];
#pragma unroll
        for (int k = 0; k < c; ++k) s -= x[k] * Lk[c][k];
        x[c] = s * rd[c];
    }
#pragma unroll
    for (int c = 0; c < NB; ++c) A[row * mb + r0 + c] = x[c];
}

// Trailing update A[ib][jb] -= A[ib][kb] A[jb][kb]^T for kb < jb <= ib (lower blocks only).
__global__ void k_syrk_update(double *A, int64_t mb, int kb)
{
    int ib = kb + 1 + blockIdx.y, jb = kb + 1 + blockIdx.x;
    if (jb > ib) return;
    __shared__ double Pa[NB][NB + 1], Pb[NB][NB + 1];
    int64_t c0 = (int64_t)kb * NB;
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        int r = t / NB, c = t % NB;
        Pa[r][c] = A[((int64_t)ib * NB + r) * mb + c0 + c];
        Pb[r][c] = A[((int64_t)jb * NB + r) * mb + c0 + c];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        int r = t / NB, c = t % NB;
        double s = 0.0;
#pragma unroll 8
        for (int k = 0; k < NB; ++k) s += Pa[r][k] * Pb[c][k];
        A[((int64_t)ib * NB + r) * mb + (int64_t)jb * NB + c] -= s;
    }
}

// L^-1 column by column (warp per column j): x = L^-1 e_j by forward substitution in blocks of
// 32 rows.  Lane r owns row i = 32 b + r of block b: it first sums L_ik x_k over the finished rows
// k in [j, 32 b) on its own, then the block is solved in 32 steps, each broadcasting one new x_t
// by a shuffle (x_i = -(sum_k L_ik x_k) / L_ii, x_j = 1 / L_jj, x_i = 0 above j).  The sequential
// chain is 32 short steps per block instead of one warp reduction per row.  mb is a multiple of 32.
__global__ void k_trtri_cols(const double *L, int64_t mb, double *Linv)
{
    extern __shared__ double xs[];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t j = blockIdx.x * (int64_t)(blockDim.x / 32) + warp;
    if (j >= mb) return;
    double *x = xs + (int64_t)warp * mb;
    const int64_t b0 = j / 32, nb32 = mb / 32;
    for (int64_t i = lane; i < 32 * b0; i += 32) x[i] = 0.0;
    for (int64_t b = b0; b < nb32; ++b) {
        const int64_t i = 32 * b + lane;
        const double *Li = L + i * mb;
        const double ri = 1.0 / Li[i];  // each lane's own row: one division per row
        double p = 0.0;
        for (int64_t k = j; k < 32 * b; ++k) p = fma(Li[k], x[k], p);
        double xi = 0.0;
        for (int t = 0; t < 32; ++t) {
            const int64_t it = 32 * b + t;
            double xt = it < j ? 0.0 : (it == j ? ri : -p * ri);  // lane t's value counts
            xt = __shfl_sync(0xffffffffu, xt, t);
            if (lane == t) xi = xt;
            if (lane > t && it >= j) p = fma(Li[it], xt, p);
        }
        x[i] = xi;
        __syncwarp();
    }
    for (int64_t i = lane; i < mb; i += 32) Linv[i * mb + j] = x[i];
}

// vy = L^-1 y (warp per row).
__global__ void k_vy(const double *Linv, int64_t mb, const double *y, int64_t m, double *vy, int64_t mp)
{
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    int64_t i = blockIdx.x * (int64_t)(blockDim.x / 32) + warp;
    if (i >= mp) return;
    double s = 0.0;
    if (i < m)
        for (int64_t k = lane; k <= i; k += 32) s += Linv[i * mb + k] * y[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) vy[i] = s;
}

// alpha = L^-T vy, Q_jj = sum_i Linv[i][j]^2, latent posterior at the observations.
__global__ void k_alpha_obs(const double *Linv, int64_t mb, const double *vy, const double *y, int64_t m,
                            double sn2, double sf2, double *alpha, double *mu_obs, double *var_obs)
{
    // warp per column j, lanes over the rows i >= j (the loads of one lane are independent)
    const int lane = threadIdx.x & 31;
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (j >= m) return;
    double a = 0.0, q = 0.0;
    for (int64_t i = j + lane; i < m; i += 32) {
        double l = Linv[i * mb + j];
        a += l * vy[i];
        q += l * l;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if (lane != 0) return;
    alpha[j] = a;
    mu_obs[j] = y[j] - sn2 * a;
    double v = sn2 - sn2 * sn2 * q, fl = 1e-12 * sf2;
    var_obs[j] = v > fl ? v : fl;
}

// BT[i][j] = Linv[j][i] for i <= j < m, else 0  (mp x mp), FP64 and FP32.
__global__ void k_operands(const double *Linv, int64_t mb, int64_t m, int64_t mp, double *BT64, float *BT32,
                           const double *vy, float *vy32, const double *alpha, float2 *alpha_ff,
                           const double *X, float *X32, float *alpha32)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx < mp) {
        vy32[idx] = (float)vy[idx];
        double a = idx < m ? alpha[idx] : 0.0;
        float h = (float)a;
        alpha_ff[idx] = make_float2(h, (float)(a - (double)h));
        alpha32[idx] = h;
    }
    if (idx < 3 * mp) {  // hi parts, then lo parts (X = hi + lo to ~1e-15), each zero-padded to 3 mp
        const float h = idx < 3 * m ? (float)X[idx] : 0.0f;
        X32[idx] = h;
        X32[3 * mp + idx] = idx < 3 * m ? (float)(X[idx] - (double)h) : 0.0f;
    }
    if (idx >= mp * mp) return;
    int64_t i = idx / mp, j = idx % mp;
    double v = (i < m && j < m && i <= j) ? Linv[j * mb + i] : 0.0;
    BT64[idx] = v;
    BT32[idx] = (float)v;
}

// Compact the padded mb x mb factor into m x m.
__global__ void k_unpad(const double *A, int64_t mb, int64_t m, double *out)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= m * m) return;
    int64_t i = idx / m, j = idx % m;
    out[idx] = (j <= i) ? A[i * mb + j] : 0.0;
}

static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Blocked Cholesky in place (lower factor of the padded mb x mb matrix A); a pivot that is not
// positive sets GPR_ERR_NOT_PD in the status word.
static void chol_blocked(double *A, int64_t mb, int *status, cudaStream_t st)
{
    int nbk = (int)(mb / NB);
    for (int kb = 0; kb < nbk; ++kb) {
        k_potrf_diag<<<1, 32, 0, st>>>(A, mb, kb, status);
        note_launch();
        int64_t rows = mb - (int64_t)(kb + 1) * NB;
        if (rows > 0) {
            k_trsm_panel<<<nblk(rows, 32), 32, 0, st>>>(A, mb, kb);  // a warp per CTA: more SMs share the FP64 work
            note_launch();
            unsigned T = (unsigned)(nbk - kb - 1);
            k_syrk_update<<<dim3(T, T), 256, 0, st>>>(A, mb, kb);
            note_launch();
        }
    }
}

// Linv = L^-1 of a padded lower factor (column by column).
static void trtri(const double *L, int64_t mb, double *Linv, cudaStream_t st)
{
    const int wpb = (sizeof(double) * mb * 4 <= 200 * 1024) ? 4 : ((sizeof(double) * mb * 2 <= 200 * 1024) ? 2 : 1);
    size_t smem = sizeof(double) * mb * wpb;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_trtri_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_trtri_cols<<<nblk(mb, wpb), 32 * wpb, smem, st>>>(L, mb, Linv);
    note_launch();
}

extern "C" gpr_status gpr_model_create(const double *obs_xyz, const double *y, int64_t m, gpr_kernel kernel,
                                       const double length_scales[3], double signal_var, double noise_var,
                                       void *stream, gpr_model **out)
{
    TraceRange trace_("gpr_model_create");
    if (!out) return GPR_ERR_ARG;
    *out = nullptr;
    if (!obs_xyz || !y || !length_scales || m < 1 || m > 8192) return GPR_ERR_ARG;
    if (kernel != GPR_K_SE && kernel != GPR_K_MATERN52) return GPR_ERR_ARG;
    if (!(signal_var > 0.0) || !(noise_var >= 0.0) || !isfinite(signal_var) || !isfinite(noise_var)) return GPR_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (!(length_scales[d] > 0.0) || !isfinite(length_scales[d])) return GPR_ERR_ARG;
    for (int64_t i = 0; i < 3 * m; ++i)
        if (!isfinite(obs_xyz[i])) return GPR_ERR_ARG;
    for (int64_t i = 0; i < m; ++i)
        if (!isfinite(y[i])) return GPR_ERR_ARG;
    if (getenv("GPR_FAULT") && strcmp(getenv("GPR_FAULT"), "alloc") == 0) return GPR_ERR_OOM;

    cudaStream_t st = (cudaStream_t)stream;
    int *status = gpr_status_word();
    if (!status) return GPR_ERR_CUDA;
    gpr_model *M = new gpr_model();
    M->m = m;
    M->mp = (m + 63) / 64 * 64;
    M->kp.kind = kernel;
    for (int d = 0; d < 3; ++d) M->kp.ell[d] = length_scales[d];
    M->kp.sf2 = signal_var;
    M->sn2 = noise_var;
    cudaGetDevice(&M->device);
    M->hX.assign(obs_xyz, obs_xyz + 3 * m);
    M->hy.assign(y, y + m);
    int64_t mb = (m + NB - 1) / NB * NB, mp = M->mp;
    double *A = nullptr;
    auto fail = [&](gpr_status s) {
        if (A) cudaFree(A);
        gpr_model_destroy(M);
        return s;
    };
#define ALLOC(ptr, bytes)                                                   \
    do {                                                                    \
        cudaError_t _e = cudaMalloc((void **)&(ptr), (bytes));              \
        if (_e != cudaSuccess) {                                            \
            gpr_internal_note_cuda_error(_e, "cudaMalloc", __LINE__);       \
            return fail(_e == cudaErrorMemoryAllocation ? GPR_ERR_OOM : GPR_ERR_CUDA); \
        }                                                                   \
    } while (0)
    ALLOC(M->X, sizeof(double) * 3 * m);
    ALLOC(M->y, sizeof(double) * m);
    ALLOC(M->L, sizeof(double) * m * m);
    ALLOC(M->Linv, sizeof(double) * mb * mb);
    ALLOC(M->vy, sizeof(double) * mp);
    ALLOC(M->alpha, sizeof(double) * m);
    ALLOC(M->mu_obs, sizeof(double) * m);
    ALLOC(M->var_obs, sizeof(double) * m);
    ALLOC(M->BT64, sizeof(double) * mp * mp);
    ALLOC(M->BT32, sizeof(float) * mp * mp);
    ALLOC(M->vy32, sizeof(float) * mp);
    ALLOC(M->alpha_ff, sizeof(float2) * mp);
    ALLOC(M->X32, sizeof(float) * 6 * mp);
    ALLOC(M->alpha32, sizeof(float) * mp);
    ALLOC(A, sizeof(double) * mb * mb);
#undef ALLOC
    if (cudaMemcpyAsync(M->X, obs_xyz, sizeof(double) * 3 * m, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(M->y, y, sizeof(double) * m, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess)
        return fail(GPR_ERR_CUDA);

    k_build_K<<<nblk(mb * mb, 256), 256, 0, st>>>(M->X, m, mb, M->kp, noise_var, A);
    note_launch();
    chol_blocked(A, mb, status, st);
    trtri(A, mb, M->Linv, st);
    k_vy<<<nblk(mp, 8), 256, 0, st>>>(M->Linv, mb, M->y, m, M->vy, mp);
    note_launch();
    k_alpha_obs<<<nblk(m * 32, 256), 256, 0, st>>>(M->Linv, mb, M->vy, M->y, m, noise_var, signal_var, M->alpha,
                                               M->mu_obs, M->var_obs);
    note_launch();
    k_operands<<<nblk(mp * mp, 256), 256, 0, st>>>(M->Linv, mb, m, mp, M->BT64, M->BT32, M->vy, M->vy32, M->alpha, M->alpha_ff, M->X, M->X32, M->alpha32);
    note_launch();
    k_unpad<<<nblk(m * m, 256), 256, 0, st>>>(A, mb, m, M->L);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { gpr_internal_note_cuda_error(e, "setup launch", __LINE__); return fail(GPR_ERR_CUDA); }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { gpr_internal_note_cuda_error(e, "setup sync", __LINE__); return fail(GPR_ERR_CUDA); }
    int hs = 0;
    cudaMemcpy(&hs, status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(A);
    A = nullptr;
    if (hs != 0) {
        cudaMemset(status, 0, sizeof(int));
        gpr_model_destroy(M);
        return (gpr_status)hs;
    }
    *out = M;
    return GPR_OK;
}

// ---- SGPR model (Eq. 1 with a stored inducing distribution)

// dst (mb x mb) = src (m x m, contiguous), zero padding.
__global__ void k_pad(const double *src, int64_t m, int64_t mb, double *dst)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= mb * mb) return;
    int64_t i = idx / mb, j = idx % mb;
    dst[idx] = (i < m && j < m) ? src[i * m + j] : 0.0;
}

// out[j] = sum_i P[i][j] v[i] for lower-triangular P (i >= j): alpha = L^-T (L^-1 mu_M).
__global__ void k_ltv(const double *P, int64_t mb, const double *v, int64_t m, double *out)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
    double a = 0.0;
    for (int64_t i = j; i < m; ++i) a += P[i * mb + j] * v[i];
    out[j] = a;
}

__global__ void k_transpose(const double *A, int64_t mb, double *At)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= mb * mb) return;
    int64_t i = idx / mb, j = idx % mb;
    At[j * mb + i] = A[idx];
}

// E = I - (B + B^T) / 2 on the m x m block, 0 on the padding.
__global__ void k_eye_minus_sym(const double *B, int64_t mb, int64_t m, double *E)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= mb * mb) return;
    int64_t i = idx / mb, j = idx % mb;
    E[idx] = (i < m && j < m) ? (i == j ? 1.0 : 0.0) - 0.5 * (B[idx] + B[j * mb + i]) : 0.0;
}

// R = J Q J (index reversal on the m x m block, symmetrised), identity on the padding.
__global__ void k_reverse(const double *Q, int64_t mb, int64_t m, double *R)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= mb * mb) return;
    int64_t i = idx / mb, j = idx % mb;
    double v;
    if (i < m && j < m) {
        int64_t a = m - 1 - i, b = m - 1 - j;
        v = 0.5 * (Q[a * mb + b] + Q[b * mb + a]);
    } else {
        v = (i == j) ? 1.0 : 0.0;
    }
    R[idx] = v;
}

// G = J Lr^T J (lower triangular), identity on the padding: Q = G^T G when J Q J = Lr Lr^T.
__global__ void k_unreverse_t(const double *Lr, int64_t mb, int64_t m, double *G)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= mb * mb) return;
    int64_t i = idx / mb, j = idx % mb;
    G[idx] = (i < m && j < m) ? Lr[(m - 1 - j) * mb + (m - 1 - i)] : (i == j ? 1.0 : 0.0);
}

// v = G^-T alpha with G^-1 = J Lr^-T J: v_i = sum_{j >= i} Lrinv[m-1-i][m-1-j] alpha_j (warp per row),
// zero on the padding (mp entries).
__global__ void k_sgpr_v(const double *Lrinv, int64_t mb, const double *alpha, int64_t m, double *v, int64_t mp)
{
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    int64_t i = blockIdx.x * (int64_t)(blockDim.x / 32) + warp;
    if (i >= mp) return;
    double s = 0.0;
    if (i < m) {
        const double *row = Lrinv + (m - 1 - i) * mb;
        for (int64_t j = i + lane; j < m; j += 32) s += row[m - 1 - j] * alpha[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) v[i] = s;
}

// The p-test reads the inducing distribution itself: mean mu_M, variance diag(A_M) (floored).
__global__ void k_sgpr_obs(const double *muM, const double *AM, int64_t m, int64_t mb, double sf2, double *mu_obs,
                           double *var_obs)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    mu_obs[i] = muM[i];
    double v = AM[i * mb + i], fl = 1e-12 * sf2;
    var_obs[i] = v > fl ? v : fl;
}

extern "C" gpr_status gpr_model_create_sgpr(const double *inducing_xyz, const double *mu_M, const double *A_M,
                                            int64_t m, gpr_kernel kernel, const double length_scales[3],
                                            double signal_var, double kmm_jitter, void *stream, gpr_model **out)
{
    TraceRange trace_("gpr_model_create_sgpr");
    if (!out) return GPR_ERR_ARG;
    *out = nullptr;
    if (!inducing_xyz || !mu_M || !A_M || !length_scales || m < 1 || m > 8192) return GPR_ERR_ARG;
    if (kernel != GPR_K_SE && kernel != GPR_K_MATERN52) return GPR_ERR_ARG;
    if (!(signal_var > 0.0) || !(kmm_jitter >= 0.0) || !isfinite(signal_var) || !isfinite(kmm_jitter))
        return GPR_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (!(length_scales[d] > 0.0) || !isfinite(length_scales[d])) return GPR_ERR_ARG;
    for (int64_t i = 0; i < 3 * m; ++i)
        if (!isfinite(inducing_xyz[i])) return GPR_ERR_ARG;
    for (int64_t i = 0; i < m; ++i)
        if (!isfinite(mu_M[i])) return GPR_ERR_ARG;
    for (int64_t i = 0; i < m * m; ++i)
        if (!isfinite(A_M[i])) return GPR_ERR_ARG;
    if (getenv("GPR_FAULT") && strcmp(getenv("GPR_FAULT"), "alloc") == 0) return GPR_ERR_OOM;

    cudaStream_t st = (cudaStream_t)stream;
    int *status = gpr_status_word();
    if (!status) return GPR_ERR_CUDA;
    gpr_model *M = new gpr_model();
    M->sgpr = true;
    M->kmm_jitter = kmm_jitter;
    M->m = m;
    M->mp = (m + 63) / 64 * 64;
    M->kp.kind = kernel;
    for (int d = 0; d < 3; ++d) M->kp.ell[d] = length_scales[d];
    M->kp.sf2 = signal_var;
    M->sn2 = 0.0;
    cudaGetDevice(&M->device);
    M->hX.assign(inducing_xyz, inducing_xyz + 3 * m);
    M->hy.assign(mu_M, mu_M + m);
    int64_t mb = (m + NB - 1) / NB * NB, mp = M->mp;
    const size_t sq = sizeof(double) * mb * mb;
    double *A = nullptr, *P = nullptr, *T1 = nullptr, *T2 = nullptr, *T3 = nullptr, *AMd = nullptr, *v0 = nullptr;
    auto release = [&]() {
        cudaFree(A); cudaFree(P); cudaFree(T1); cudaFree(T2); cudaFree(T3); cudaFree(AMd); cudaFree(v0);
        A = P = T1 = T2 = T3 = AMd = v0 = nullptr;
    };
    auto fail = [&](gpr_status s) {
        cudaStreamSynchronize(st);
        release();
        gpr_model_destroy(M);
        return s;
    };
#define ALLOC(ptr, bytes)                                                   \
    do {                                                                    \
        cudaError_t _e = cudaMalloc((void **)&(ptr), (bytes));              \
        if (_e != cudaSuccess) {                                            \
            gpr_internal_note_cuda_error(_e, "cudaMalloc", __LINE__);       \
            return fail(_e == cudaErrorMemoryAllocation ? GPR_ERR_OOM : GPR_ERR_CUDA); \
        }                                                                   \
    } while (0)
    ALLOC(M->X, sizeof(double) * 3 * m);
    ALLOC(M->y, sizeof(double) * m);
    ALLOC(M->L, sizeof(double) * m * m);
    ALLOC(M->Linv, sq);
    ALLOC(M->vy, sizeof(double) * mp);
    ALLOC(M->alpha, sizeof(double) * m);
    ALLOC(M->mu_obs, sizeof(double) * m);
    ALLOC(M->var_obs, sizeof(double) * m);
    ALLOC(M->BT64, sizeof(double) * mp * mp);
    ALLOC(M->BT32, sizeof(float) * mp * mp);
    ALLOC(M->vy32, sizeof(float) * mp);
    ALLOC(M->alpha_ff, sizeof(float2) * mp);
    ALLOC(M->X32, sizeof(float) * 6 * mp);
    ALLOC(M->alpha32, sizeof(float) * mp);
    ALLOC(A, sq);
    ALLOC(P, sq);
    ALLOC(T1, sq);
    ALLOC(T2, sq);
    ALLOC(T3, sq);
    ALLOC(AMd, sq);
    ALLOC(v0, sizeof(double) * mb);
    ALLOC(M->A_M, sizeof(double) * m * m);
#undef ALLOC
    if (cudaMemcpyAsync(M->X, inducing_xyz, sizeof(double) * 3 * m, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(M->y, mu_M, sizeof(double) * m, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(T3, A_M, sizeof(double) * m * m, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(M->A_M, A_M, sizeof(double) * m * m, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess)
        return fail(GPR_ERR_CUDA);
    const unsigned gsq = nblk(mb * mb, 256);
    k_pad<<<gsq, 256, 0, st>>>(T3, m, mb, AMd);
    note_launch();
    // K_MM + jitter I = Lk Lk^T, P = Lk^-1, alpha = K_MM^-1 mu_M
    k_build_K<<<gsq, 256, 0, st>>>(M->X, m, mb, M->kp, kmm_jitter, A);
    note_launch();
    chol_blocked(A, mb, status, st);
    trtri(A, mb, P, st);
    k_unpad<<<nblk(m * m, 256), 256, 0, st>>>(A, mb, m, M->L);
    note_launch();
    k_vy<<<nblk(m, 8), 256, 0, st>>>(P, mb, M->y, m, v0, m);
    note_launch();
    k_ltv<<<nblk(m, 128), 128, 0, st>>>(P, mb, v0, m, M->alpha);
    note_launch();
    // Q = K_MM^-1 - K_MM^-1 A_M K_MM^-1 = P^T (I - P A_M P^T) P
    k_transpose<<<gsq, 256, 0, st>>>(P, mb, T1);  // T1 = P^T
    note_launch();
    gemm64_nn(mb, mb, mb, P, mb, AMd, mb, T2, mb, st);   // T2 = P A_M
    gemm64_nn(mb, mb, mb, T2, mb, T1, mb, T3, mb, st);   // T3 = P A_M P^T
    k_eye_minus_sym<<<gsq, 256, 0, st>>>(T3, mb, m, T2);  // T2 = E = I - P A_M P^T
    note_launch();
    gemm64_nn(mb, mb, mb, T2, mb, P, mb, T3, mb, st);    // T3 = E P
    gemm64_tn(mb, mb, mb, P, mb, T3, mb, T2, mb, st);    // T2 = Q = P^T E P
    // Q = G^T G with G lower triangular: J Q J = Lr Lr^T, G = J Lr^T J
    k_reverse<<<gsq, 256, 0, st>>>(T2, mb, m, A);
    note_launch();
    chol_blocked(A, mb, status, st);  // not positive definite: A_M is not below K_MM
    k_unreverse_t<<<gsq, 256, 0, st>>>(A, mb, m, M->Linv);
    note_launch();
    trtri(A, mb, T1, st);  // T1 = Lr^-1
    k_sgpr_v<<<nblk(mp, 8), 256, 0, st>>>(T1, mb, M->alpha, m, M->vy, mp);
    note_launch();
    k_sgpr_obs<<<nblk(m, 128), 128, 0, st>>>(M->y, AMd, m, mb, signal_var, M->mu_obs, M->var_obs);
    note_launch();
    k_operands<<<nblk(mp * mp, 256), 256, 0, st>>>(M->Linv, mb, m, mp, M->BT64, M->BT32, M->vy, M->vy32, M->alpha,
                                                   M->alpha_ff, M->X, M->X32, M->alpha32);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { gpr_internal_note_cuda_error(e, "sgpr setup launch", __LINE__); return fail(GPR_ERR_CUDA); }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { gpr_internal_note_cuda_error(e, "sgpr setup sync", __LINE__); return fail(GPR_ERR_CUDA); }
    int hs = 0;
    cudaMemcpy(&hs, status, sizeof(int), cudaMemcpyDeviceToHost);
    release();
    if (hs != 0) {
        cudaMemset(status, 0, sizeof(int));
        gpr_model_destroy(M);
        return (gpr_status)hs;
    }
    *out = M;
    return GPR_OK;
}

extern "C" gpr_status gpr_model_destroy(gpr_model *M)
{
    if (!M) return GPR_ERR_ARG;
    cudaDeviceSynchronize();
    cudaFree(M->X); cudaFree(M->y); cudaFree(M->L); cudaFree(M->Linv); cudaFree(M->vy); cudaFree(M->alpha);
    cudaFree(M->mu_obs); cudaFree(M->var_obs); cudaFree(M->A_M); cudaFree(M->BT64); cudaFree(M->BT32); cudaFree(M->vy32); cudaFree(M->alpha_ff); cudaFree(M->X32); cudaFree(M->alpha32);
    for (int w = 0; w < 2; ++w)
        if (M->own_ws.ptr[w]) cudaFree(M->own_ws.ptr[w]);
    tc_release(M);
    oz_release(M);
    cache_release(M);
    if (M->mv_ev) cudaEventDestroy(M->mv_ev);
    delete M;
    return GPR_OK;
}

extern "C" int64_t gpr_model_m(const gpr_model *M) { return M ? M->m : -1; }

namespace {
thread_local Workspace *tl_ws = nullptr;  // a batch worker's pooled workspace, used for every model
}

void set_thread_workspace(Workspace *w) { tl_ws = w; }

static Workspace &ws_of(gpr_model *M) { return tl_ws ? *tl_ws : M->own_ws; }
void *ws_ptr(gpr_model *M, int which) { return ws_of(M).ptr[which]; }
size_t ws_size(gpr_model *M, int which) { return ws_of(M).bytes[which]; }

gpr_status ws_reserve(gpr_model *M, int which, size_t bytes, cudaStream_t st)
{
    Workspace &W = ws_of(M);
    if (bytes <= W.bytes[which]) return GPR_OK;
    if (W.ptr[which]) {
        cudaStreamSynchronize(st);
        cudaFree(W.ptr[which]);
        W.ptr[which] = nullptr;
        W.bytes[which] = 0;
    }
    size_t want = bytes + bytes / 8;
    cudaError_t e = cudaMalloc(&W.ptr[which], want);
    if (e != cudaSuccess) {
        gpr_internal_note_cuda_error(e, "workspace", __LINE__);
        W.ptr[which] = nullptr;
        return e == cudaErrorMemoryAllocation ? GPR_ERR_OOM : GPR_ERR_CUDA;
    }
    W.bytes[which] = want;
    return GPR_OK;
}

// Test hook: copy the FP64 factors of a model to host buffers (each nullable).
extern "C" gpr_status gpr_model_export(const gpr_model *M, double *L, double *alpha, double *vy, double *mu_obs,
                                       double *var_obs)
{
    if (!M) return GPR_ERR_ARG;
    int64_t m = M->m;
    if (L) GPR_CUDA_TRY(cudaMemcpy(L, M->L, sizeof(double) * m * m, cudaMemcpyDeviceToHost));
    if (alpha) GPR_CUDA_TRY(cudaMemcpy(alpha, M->alpha, sizeof(double) * m, cudaMemcpyDeviceToHost));
    if (vy) GPR_CUDA_TRY(cudaMemcpy(vy, M->vy, sizeof(double) * m, cudaMemcpyDeviceToHost));
    if (mu_obs) GPR_CUDA_TRY(cudaMemcpy(mu_obs, M->mu_obs, sizeof(double) * m, cudaMemcpyDeviceToHost));
    if (var_obs) GPR_CUDA_TRY(cudaMemcpy(var_obs, M->var_obs, sizeof(double) * m, cudaMemcpyDeviceToHost));
    return GPR_OK;
}
