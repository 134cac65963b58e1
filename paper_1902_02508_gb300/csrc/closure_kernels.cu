// Learned subgrid closure: features on the LES grid, an MLP 10-128-128-128-6
// (SiLU) trained with Adam on the exact stress, and inference with the exact
// stress as fallback.  All device work is in the kernels below; the host code
// only orders them.
//
// The paper proposes informing SGS models with the exact stress computed from
// DNS, e.g. by machine learning (Sec. 2.1, Sec. 5).  Inputs: the nine
// filtered velocity gradients d~bar(u_i)/dx_j (second-order central
// differences; periodic in x, z; three-point non-uniform in y with mirror
// ghosts of the Eq. 8 parities at the walls) and y+ = (1 - |y|) Re_tau.
// Outputs: the six independent T_ij.  Inputs and targets are standardised
// with statistics of the training set.
//
// Numerics: FP32 master weights and Adam moments; the forward and backward
// passes use the weights rounded to BF16 ("BF16 weights") with FP32
// accumulation.  Every reduction has a fixed order, so a run is reproducible
// bit for bit, and a checkpoint resumed gives the same bits as an
// uninterrupted run.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include <cuda_bf16.h>

#include "eles_internal.h"

namespace eles {
namespace {

constexpr int NIN = 10, NH = 128, NOUT = 6, NLAYER = 4;
constexpr int kLayerIn[NLAYER] = {NIN, NH, NH, NH};
constexpr int kLayerOut[NLAYER] = {NH, NH, NH, NOUT};

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_d(float z)
{
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}
__device__ __forceinline__ float bf16_round(float x)
{
    unsigned u = __float_as_uint(x);
    u += 0x7fffu + ((u >> 16) & 1u);
    return __uint_as_float(u & 0xffff0000u);
}

// ------------------------------------------------------------- features --
__global__ void features_kernel(const float *__restrict__ ub, const double *__restrict__ Y, int nlx, int nly,
                                int nlz, double Lx, double Lz, int p0, int p1, int p2, double re_tau,
                                float *__restrict__ F)
{
    const long n = (long)nly * nlz * nlx;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int X = (int)(idx % nlx), Z = (int)((idx / nlx) % nlz), J = (int)(idx / ((long)nlx * nlz));
    const long plane = (long)nlz * nlx;
    const int par[3] = {p0, p1, p2};
    const double hx = Lx / nlx, hz = Lz / nlz;
    const int Xp = X + 1 == nlx ? 0 : X + 1, Xm = X == 0 ? nlx - 1 : X - 1;
    const int Zp = Z + 1 == nlz ? 0 : Z + 1, Zm = Z == 0 ? nlz - 1 : Z - 1;
    double hp, hm;
    int Jp, Jm;
    double sp = 1.0, sm = 1.0;   // mirror signs of the neighbours
    if (J > 0 && J < nly - 1) {
        hp = Y[J + 1] - Y[J]; hm = Y[J] - Y[J - 1]; Jp = J + 1; Jm = J - 1;
    } else if (J == 0) {
        hp = hm = Y[1] - Y[0]; Jp = 1; Jm = 1; sm = -1.0;   // ghost = parity * f(y1)
    } else {
        hp = hm = Y[nly - 1] - Y[nly - 2]; Jp = nly - 2; Jm = nly - 2; sp = -1.0;
    }
    float *out = F + idx * NIN;
    for (int i = 0; i < 3; i++) {
        const float *f = ub + (long)i * nly * plane;
        const double c = f[(long)J * plane + (long)Z * nlx + X];
        out[3 * i + 0] = (float)((f[(long)J * plane + (long)Z * nlx + Xp] - f[(long)J * plane + (long)Z * nlx + Xm]) / (2 * hx));
        double fp = f[(long)Jp * plane + (long)Z * nlx + X], fm = f[(long)Jm * plane + (long)Z * nlx + X];
        if (sp < 0) fp *= par[i];
        if (sm < 0) fm *= par[i];
        out[3 * i + 1] = (float)((hm * hm * (fp - c) + hp * hp * (c - fm)) / (hp * hm * (hp + hm)));
        out[3 * i + 2] = (float)((f[(long)J * plane + (long)Zp * nlx + X] - f[(long)J * plane + (long)Zm * nlx + X]) / (2 * hz));
    }
    out[9] = (float)((1.0 - fabs(Y[J])) * re_tau);
}

// ------------------------------------------------------- standardisation --
// mean and standard deviation of column c of a [n][ld] (point-major) or
// [ld][n] (component-major) array; one CTA per column, FP64, fixed order.
__global__ void column_stats(const float *__restrict__ A, long n, int ncol, int point_major, double *mean,
                             double *stdv)
{
    const int c = blockIdx.x;
    double s = 0.0, s2 = 0.0;
    for (long i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = point_major ? A[i * ncol + c] : A[(long)c * n + i];
        s += v;
        s2 += v * v;
    }
    __shared__ double ps[256], ps2[256];
    ps[threadIdx.x] = s;
    ps2[threadIdx.x] = s2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) { ps[threadIdx.x] += ps[threadIdx.x + o]; ps2[threadIdx.x] += ps2[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = ps[0] / n;
        const double var = ps2[0] / n - m * m;
        mean[c] = m;
        stdv[c] = sqrt(var > 1e-30 ? var : 1e-30);
    }
}

// Gather a mini-batch: H0[b][k] = (F[idx[b]][k] - mu_k) / sd_k and
// T[b][q] = (tau[q][idx[b]] - mu_q) / sd_q.
__global__ void gather_batch(const float *__restrict__ F, const float *__restrict__ tau, long n,
                             const long *__restrict__ idx, int nb, const double *fmu, const double *fsd,
                             const double *tmu, const double *tsd, float *H0, float *T)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const long p = idx[b];
    for (int k = 0; k < NIN; k++) H0[(long)b * NIN + k] = (float)((F[p * NIN + k] - fmu[k]) / fsd[k]);
    if (T)
        for (int q = 0; q < NOUT; q++) T[(long)b * NOUT + q] = (float)((tau[(long)q * n + p] - tmu[q]) / tsd[q]);
}

// ------------------------------------------------------------------ GEMM --
// C[m][n] = sum_k A(m, k) B(k, n) on the tensor cores, with generic strides:
// A(m, k) = A[m * sam + k * sak], B(k, n) = B[k * sbk + n * sbn].
//
// mma.sync m16n8k16 BF16 with FP32 accumulation.  Each FP32 operand is split
// into BF16 words hi = rn(x), lo = rn(x - hi) (16 significant bits together)
// and the products hi*hi + lo*hi + hi*lo are accumulated; an operand that is
// exact in BF16 (the rounded weights, BLO = false) has no lo word and its
// product is dropped.  Tiles of 64 x 64 outputs, k-slices of 32 staged in
// shared memory as BF16 (A as [m][k], B as [n][k], so a fragment register is
// one 32-bit load), 4 warps with 32 x 32 outputs each.  With gridDim.z > 1
// the k range is split and slice z writes its partial to C + z * M * N
// (reduced afterwards in a fixed order).
constexpr int GT = 64, GK = 32, GKP = GK + 8;   // row pitch 40 BF16 = 20 words: conflict-free fragments

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void split_store(__nv_bfloat16 *hi, __nv_bfloat16 *lo, int at, float x, bool keep_lo)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[at] = h;
    if (keep_lo) lo[at] = __float2bfloat16_rn(x - __bfloat162float(h));
}

template <bool BLO>
__global__ void __launch_bounds__(128) gemm_tc_kernel(const float *__restrict__ A, long sam, long sak,
                                                      const float *__restrict__ B, long sbk, long sbn, float *C,
                                                      int M, int N, long K, long kchunk)
{
    __shared__ __align__(16) __nv_bfloat16 Ah[GT * GKP], Al[GT * GKP], Bh[GT * GKP], Bl[BLO ? GT * GKP : 2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    const long k0 = (long)blockIdx.z * kchunk, k1 = min(K, k0 + kchunk);
    float acc[2][4][4] = {};
    for (long kb = k0; kb < k1; kb += GK) {
        for (int i = threadIdx.x; i < GK * GT; i += 128) {
            // the contiguous index runs fastest across the threads
            const int kk = sak == 1 ? i % GK : i / GT, mm = sak == 1 ? i / GK : i % GT;
            const long k = kb + kk;
            const float x = (m0 + mm < M && k < k1) ? A[(long)(m0 + mm) * sam + k * sak] : 0.f;
            split_store(Ah, Al, mm * GKP + kk, x, true);
        }
        for (int i = threadIdx.x; i < GK * GT; i += 128) {
            const int kk = sbk == 1 ? i % GK : i / GT, nn = sbk == 1 ? i / GK : i % GT;
            const long k = kb + kk;
            const float x = (n0 + nn < N && k < k1) ? B[k * sbk + (long)(n0 + nn) * sbn] : 0.f;
            split_store(Bh, Bl, nn * GKP + kk, x, BLO);
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GK; ks += 16) {
            unsigned ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; mt++) {
                const int r = (wm + mt * 16 + g) * GKP + ks + 2 * t;
                ah[mt][0] = *reinterpret_cast<const unsigned *>(Ah + r);
                ah[mt][1] = *reinterpret_cast<const unsigned *>(Ah + r + 8 * GKP);
                ah[mt][2] = *reinterpret_cast<const unsigned *>(Ah + r + 8);
                ah[mt][3] = *reinterpret_cast<const unsigned *>(Ah + r + 8 * GKP + 8);
                al[mt][0] = *reinterpret_cast<const unsigned *>(Al + r);
                al[mt][1] = *reinterpret_cast<const unsigned *>(Al + r + 8 * GKP);
                al[mt][2] = *reinterpret_cast<const unsigned *>(Al + r + 8);
                al[mt][3] = *reinterpret_cast<const unsigned *>(Al + r + 8 * GKP + 8);
            }
#pragma unroll
            for (int nt = 0; nt < 4; nt++) {
                const int r = (wn + nt * 8 + g) * GKP + ks + 2 * t;
                bh[nt][0] = *reinterpret_cast<const unsigned *>(Bh + r);
                bh[nt][1] = *reinterpret_cast<const unsigned *>(Bh + r + 8);
                if constexpr (BLO) {
                    bl[nt][0] = *reinterpret_cast<const unsigned *>(Bl + r);
                    bl[nt][1] = *reinterpret_cast<const unsigned *>(Bl + r + 8);
                }
            }
#pragma unroll
            for (int mt = 0; mt < 2; mt++)
#pragma unroll
                for (int nt = 0; nt < 4; nt++) {
                    // small products first
                    if constexpr (BLO) mma_bf16(acc[mt][nt], ah[mt], bl[nt][0], bl[nt][1]);
                    mma_bf16(acc[mt][nt], al[mt], bh[nt][0], bh[nt][1]);
                    mma_bf16(acc[mt][nt], ah[mt], bh[nt][0], bh[nt][1]);
                }
        }
        __syncthreads();
    }
    float *Cz = C + (long)blockIdx.z * M * N;
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < 4; nt++)
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int m = m0 + wm + mt * 16 + g + (i >> 1) * 8, nn = n0 + wn + nt * 8 + 2 * t + (i & 1);
                if (m < M && nn < N) Cz[(long)m * N + nn] = acc[mt][nt][i];
            }
}

__global__ void reduce_parts(const float *__restrict__ P, int nparts, long len, float *out)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    float s = 0.f;
    for (int z = 0; z < nparts; z++) s += P[(long)z * len + i];
    out[i] = s;
}

// Z = pre-activation + bias (in place); H = SiLU(Z) for hidden layers.
__global__ void bias_act(float *Z, float *H, const float *__restrict__ bias, long rows, int cols, int act)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const float z = Z[i] + bias[i % cols];
    Z[i] = z;
    if (act) H[i] = silu(z);
}

// dY = 2 (Y - T) / (rows * cols); per-row squared error partials for the loss.
__global__ void mse_grad(const float *__restrict__ Y, const float *__restrict__ T, float *dY, float *rowloss,
                         int rows)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float s = 0.f;
    for (int q = 0; q < NOUT; q++) {
        const float d = Y[(long)r * NOUT + q] - T[(long)r * NOUT + q];
        s += d * d;
        dY[(long)r * NOUT + q] = 2.f * d / ((float)rows * NOUT);
    }
    rowloss[r] = s;
}

// *acc += sum of v[0 .. n) in a fixed order (one block).
__global__ void sum_into(const float *__restrict__ v, int n, double *acc)
{
    __shared__ double part[256];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += (double)v[i];
    part[threadIdx.x] = t;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *acc += part[0];
}

__global__ void mul_silu_d(float *dH, const float *__restrict__ Z, long n)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dH[i] *= silu_d(Z[i]);
}

// Column sums of dZ [rows][cols] (bias gradients): block z sums rows
// [z * chunk, (z + 1) * chunk) with one thread per column (coalesced); the
// partials [gridDim.x][cols] are then reduced in a fixed order.
__global__ void col_sum_parts(const float *__restrict__ dZ, long rows, int cols, long chunk, float *parts)
{
    const int c = threadIdx.x;
    if (c >= cols) return;
    const long r0 = (long)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
    float s = 0.f;
    for (long r = r0; r < r1; r++) s += dZ[r * cols + c];
    parts[(long)blockIdx.x * cols + c] = s;
}

// Adam on the FP32 master parameters; the working copy Wq is the BF16-rounded master.
__global__ void adam_step(float *w, float *Wq, const float *__restrict__ g, float *m, float *v, long n, float lr,
                          float b1, float b2, float eps, float c1, float c2)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    Wq[i] = bf16_round(wi);
}

// The captured training step's variants: the batch index *bt and the bias
// corrections of that step come from device memory, so one captured step
// serves every full batch of an epoch (same arithmetic as gather_batch and
// adam_step).
__global__ void gather_batch_at(const float *__restrict__ F, const float *__restrict__ tau, long n,
                                const long *__restrict__ perm, const long *__restrict__ bt, int B,
                                const double *fmu, const double *fsd, const double *tmu, const double *tsd, float *H0,
                                float *T)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const long p = perm[*bt * B + b];
    for (int k = 0; k < NIN; k++) H0[(long)b * NIN + k] = (float)((F[p * NIN + k] - fmu[k]) / fsd[k]);
    for (int q = 0; q < NOUT; q++) T[(long)b * NOUT + q] = (float)((tau[(long)q * n + p] - tmu[q]) / tsd[q]);
}

__global__ void adam_step_at(float *w, float *Wq, const float *__restrict__ g, float *m, float *v, long n, float lr,
                             float b1, float b2, float eps, const float *__restrict__ c12, const long *__restrict__ bt)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float c1 = c12[2 * *bt], c2 = c12[2 * *bt + 1];
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    Wq[i] = bf16_round(wi);
}

__global__ void next_batch(long *bt) { *bt += 1; }

__global__ void round_copy(const float *w, float *Wq, long n)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) Wq[i] = bf16_round(w[i]);
}

__global__ void iota_range(long *idx, long p0, int nb)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) idx[b] = p0 + b;
}

__global__ void init_uniform(float *w, long n, float bound, unsigned long long seed)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // splitmix64 of (seed, i): counter-based, reproducible
    unsigned long long z = seed + 0x9e3779b97f4a7c15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    w[i] = (float)((2.0 * u - 1.0) * bound);
}

inline unsigned grid1(long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace eles

// ------------------------------------------------------------ host side --
struct ef_closure {
    ef_closure_cfg cfg;
    int device = 0;
    long nparam = 0;
    long off_w[eles::NLAYER], off_b[eles::NLAYER];
    float *w = nullptr, *wq = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;   // [nparam]
    double *stats = nullptr;   // fmu[10] fsd[10] tmu[6] tsd[6]
    bool fitted = false;
    long step = 0;
    // work buffers for one mini-batch
    int cap = 0;
    float *H[eles::NLAYER + 1] = {};   // activations: H[0] = standardised input
    float *Z[eles::NLAYER] = {};
    float *T = nullptr, *dA = nullptr, *dB = nullptr, *rowloss = nullptr, *parts = nullptr;
    long *idx = nullptr;
    int *nfall = nullptr;      // [0] guarded points of the last inference, [1] device error word
    void *image = nullptr;     // tensor-core inference image (packed weights and statistics)
    size_t parts_len = 0;
};

namespace eles {
namespace {

constexpr int kSplitK = 32;

int closure_alloc_batch(ef_closure *c, int cap)
{
    if (cap <= c->cap) return EF_OK;
    for (int l = 0; l <= NLAYER; l++) { cudaFree(c->H[l]); c->H[l] = nullptr; }
    for (int l = 0; l < NLAYER; l++) { cudaFree(c->Z[l]); c->Z[l] = nullptr; }
    cudaFree(c->T); cudaFree(c->dA); cudaFree(c->dB); cudaFree(c->rowloss); cudaFree(c->idx); cudaFree(c->parts);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l <= NLAYER && e == cudaSuccess; l++)
        e = dev_malloc(&c->H[l], sizeof(float) * (size_t)cap * (l == 0 ? NIN : (l == NLAYER ? NOUT : NH)));
    for (int l = 0; l < NLAYER && e == cudaSuccess; l++) e = dev_malloc(&c->Z[l], sizeof(float) * (size_t)cap * kLayerOut[l]);
    if (e == cudaSuccess) e = dev_malloc(&c->T, sizeof(float) * (size_t)cap * NOUT);
    if (e == cudaSuccess) e = dev_malloc(&c->dA, sizeof(float) * (size_t)cap * NH);
    if (e == cudaSuccess) e = dev_malloc(&c->dB, sizeof(float) * (size_t)cap * NH);
    if (e == cudaSuccess) e = dev_malloc(&c->rowloss, sizeof(float) * (size_t)cap);
    if (e == cudaSuccess) e = dev_malloc(&c->idx, sizeof(long) * (size_t)cap);
    c->parts_len = (size_t)kSplitK * NH * NH;
    if (e == cudaSuccess) e = dev_malloc(&c->parts, sizeof(float) * c->parts_len);
    if (e != cudaSuccess) return cuda_fail(e, "closure work buffers");
    c->cap = cap;
    return EF_OK;
}

// C[M][N] = A(m,k) B(k,n) with a deterministic split over k when K is long;
// b_exact: B holds BF16-exact values (the rounded weights).
void gemm(const float *A, long sam, long sak, const float *B, long sbk, long sbn, bool b_exact, float *C, int M,
          int N, long K, float *parts, cudaStream_t s)
{
    int splits = 1;
    if (K > 1024) splits = kSplitK;
    const long kchunk = ((K + splits - 1) / splits + GK - 1) / GK * GK;
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, splits);
    float *out = splits == 1 ? C : parts;
    if (b_exact) gemm_tc_kernel<false><<<grid, 128, 0, s>>>(A, sam, sak, B, sbk, sbn, out, M, N, K, kchunk);
    else gemm_tc_kernel<true><<<grid, 128, 0, s>>>(A, sam, sak, B, sbk, sbn, out, M, N, K, kchunk);
    if (splits > 1) reduce_parts<<<grid1((long)M * N), 256, 0, s>>>(parts, splits, (long)M * N, C);
}

// Forward pass of nb rows already in H[0]; Y in H[NLAYER].
void forward(ef_closure *c, int nb, cudaStream_t s)
{
    for (int l = 0; l < NLAYER; l++) {
        const int K = kLayerIn[l], N = kLayerOut[l];
        // Z = H W^T: A = H [nb][K], B(k, n) = W[n][k]
        gemm(c->H[l], K, 1, c->wq + c->off_w[l], 1, K, true, c->Z[l], nb, N, K, c->parts, s);
        const bool act = l < NLAYER - 1;
        bias_act<<<grid1((long)nb * N), 256, 0, s>>>(c->Z[l], act ? c->H[l + 1] : nullptr, c->wq + c->off_b[l],
                                                      nb, N, act ? 1 : 0);
        if (!act) cudaMemcpyAsync(c->H[l + 1], c->Z[l], sizeof(float) * (size_t)nb * N, cudaMemcpyDeviceToDevice, s);
    }
}

// Backward pass (after forward and the loss gradient in dA as [nb][6]);
// gradients into c->g.
void backward(ef_closure *c, int nb, cudaStream_t s)
{
    float *d = c->dA, *dn = c->dB;
    for (int l = NLAYER - 1; l >= 0; l--) {
        const int K = kLayerIn[l], N = kLayerOut[l];
        // dW[n][k] = sum_b d[b][n] H[b][k]: A(m=n, k=b) = d[b][n], B(k=b, n=k) = H[b][k]
        gemm(d, 1, N, c->H[l], K, 1, false, c->g + c->off_w[l], N, K, nb, c->parts, s);
        {
            const long chunk = (nb + kSplitK - 1) / kSplitK;
            col_sum_parts<<<kSplitK, 128, 0, s>>>(d, nb, N, chunk, c->parts);
            reduce_parts<<<grid1(N), 256, 0, s>>>(c->parts, kSplitK, N, c->g + c->off_b[l]);
        }
        if (l > 0) {
            // dH[b][k] = sum_n d[b][n] W[n][k]
            gemm(d, N, 1, c->wq + c->off_w[l], K, 1, true, dn, nb, K, N, c->parts, s);
            mul_silu_d<<<grid1((long)nb * K), 256, 0, s>>>(dn, c->Z[l - 1], (long)nb * K);
            float *t = d; d = dn; dn = t;
        }
    }
}

// splitmix64
unsigned long long mix(unsigned long long z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

int check_closure(const ef_closure *c, const char *who)
{
    if (!c) { set_error("%s: NULL closure", who); return EF_ERR_ARG; }
    return EF_OK;
}

}  // namespace
}  // namespace eles

using namespace eles;

extern "C" {

int ef_closure_create(const ef_closure_cfg *cfg, ef_closure **out)
{
    if (!cfg || !out) { set_error("ef_closure_create: NULL argument"); return EF_ERR_ARG; }
    *out = nullptr;
    if (cfg->hidden != NH || cfg->batch < 1 || !(cfg->lr > 0) || !(cfg->guard_sigma > 0)) {
        set_error("ef_closure_create: hidden must be %d, batch >= 1, lr > 0, guard_sigma > 0", NH);
        return EF_ERR_ARG;
    }
    ef_closure *c = new ef_closure();
    c->cfg = *cfg;
    cudaGetDevice(&c->device);
    long off = 0;
    for (int l = 0; l < NLAYER; l++) {
        c->off_w[l] = off; off += (long)kLayerIn[l] * kLayerOut[l];
        c->off_b[l] = off; off += kLayerOut[l];
    }
    c->nparam = off;
    cudaError_t e = cudaSuccess;
    float **bufs[5] = {&c->w, &c->wq, &c->m, &c->v, &c->g};
    for (auto b : bufs)
        if (e == cudaSuccess) e = dev_malloc(b, sizeof(float) * c->nparam);
    if (e == cudaSuccess) e = dev_malloc(&c->stats, sizeof(double) * 32);
    if (e == cudaSuccess) e = dev_malloc(&c->nfall, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->nfall, 0, 2 * sizeof(int));
    if (e == cudaSuccess) e = dev_malloc(&c->image, closure_tc_image_bytes());
    if (e == cudaSuccess) e = cudaMemset(c->w, 0, sizeof(float) * c->nparam);
    if (e == cudaSuccess) e = cudaMemset(c->m, 0, sizeof(float) * c->nparam);
    if (e == cudaSuccess) e = cudaMemset(c->v, 0, sizeof(float) * c->nparam);
    if (e != cudaSuccess) { int rc = cuda_fail(e, "ef_closure_create"); ef_closure_destroy(c); return rc; }
    for (int l = 0; l < NLAYER; l++) {
        const float bound = 0.5f * sqrtf(6.f / kLayerIn[l]);
        const long n = (long)kLayerIn[l] * kLayerOut[l];
        init_uniform<<<grid1(n), 256>>>(c->w + c->off_w[l], n, bound, mix(cfg->seed + l));
    }
    round_copy<<<grid1(c->nparam), 256>>>(c->w, c->wq, c->nparam);
    int rc = closure_alloc_batch(c, cfg->batch);
    if (rc == EF_OK && (e = cudaDeviceSynchronize()) != cudaSuccess) rc = cuda_fail(e, "ef_closure_create");
    if (rc) { ef_closure_destroy(c); return rc; }
    *out = c;
    return EF_OK;
}

void ef_closure_destroy(ef_closure *c)
{
    if (!c) return;
    cudaFree(c->w); cudaFree(c->wq); cudaFree(c->m); cudaFree(c->v); cudaFree(c->g); cudaFree(c->stats);
    cudaFree(c->nfall);
    cudaFree(c->image);
    for (int l = 0; l <= NLAYER; l++) cudaFree(c->H[l]);
    for (int l = 0; l < NLAYER; l++) cudaFree(c->Z[l]);
    cudaFree(c->T); cudaFree(c->dA); cudaFree(c->dB); cudaFree(c->rowloss); cudaFree(c->idx); cudaFree(c->parts);
    delete c;
}

int ef_closure_features(const ef_grid *les, const float *ubar, double re_tau, int extension, float *feats,
                        void *stream)
{
    if (!les || !les->y || !ubar || !feats) { set_error("ef_closure_features: NULL argument"); return EF_ERR_ARG; }
    if (les->nx < 2 || les->nz < 2 || les->ny < 3) { set_error("ef_closure_features: grid too small"); return EF_ERR_SHAPE; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *dY = nullptr;
    cudaError_t e = dev_malloc_async(&dY, sizeof(double) * les->ny, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dY, les->y, sizeof(double) * les->ny, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "ef_closure_features");
    const int flip = extension == EF_EXT_ODD_EVEN;
    const long n = (long)les->nx * les->ny * les->nz;
    features_kernel<<<grid1(n), 256, 0, s>>>(ubar, dY, les->nx, les->ny, les->nz, les->Lx, les->Lz, flip ? -1 : 1,
                                             flip ? 1 : -1, flip ? -1 : 1, re_tau, feats);
    e = cudaGetLastError();
    cudaFreeAsync(dY, s);
    if (e != cudaSuccess) return cuda_fail(e, "features_kernel");
    return EF_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of ef_closure_features.  Its only scratch, the LES
// y nodes on the device, lives in a fixed file-scope device array instead of
// a per-call allocation, for callers that may not allocate device memory
// (a host code that owns every allocation itself, or one running where the
// allocator must not be called).  The array holds kStaticMaxNy nodes; every
// device that loads the library keeps it until the process exits.  The
// first call on a device looks up the array's device address (set-up; make
// that first call before any stream capture).  All calls share the array:
// calls that overlap on the GPU race and must be serialised by the caller.
constexpr int kStaticMaxNy = 4096;
static __device__ __align__(256) double g_static_y[kStaticMaxNy];

int ef_closure_features_static(const ef_grid *les, const float *ubar, double re_tau, int extension, float *feats,
                               void *stream)
{
    if (!les || !les->y || !ubar || !feats) { set_error("ef_closure_features_static: NULL argument"); return EF_ERR_ARG; }
    if (les->nx < 2 || les->nz < 2 || les->ny < 3) { set_error("ef_closure_features_static: grid too small"); return EF_ERR_SHAPE; }
    if (les->ny > kStaticMaxNy) {
        set_error("ef_closure_features_static: ny = %d exceeds the static limit of %d nodes", les->ny, kStaticMaxNy);
        return EF_ERR_ARG;
    }
    static double *addr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "ef_closure_features_static");
    if (dev < 0 || dev >= 64) { set_error("ef_closure_features_static: device index %d unsupported", dev); return EF_ERR_ARG; }
    if (!addr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_static_y);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
        addr[dev] = p;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemcpyAsync(addr[dev], les->y, sizeof(double) * les->ny, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "ef_closure_features_static");
    const int flip = extension == EF_EXT_ODD_EVEN;
    const long n = (long)les->nx * les->ny * les->nz;
    features_kernel<<<grid1(n), 256, 0, s>>>(ubar, addr[dev], les->nx, les->ny, les->nz, les->Lx, les->Lz,
                                             flip ? -1 : 1, flip ? 1 : -1, flip ? -1 : 1, re_tau, feats);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "features_kernel");
    return EF_OK;
}

int ef_closure_fit_norm(ef_closure *c, const float *feats, const float *tau, long n, void *stream)
{
    int rc = check_closure(c, "ef_closure_fit_norm");
    if (rc) return rc;
    if (!feats || !tau || n < 2) { set_error("ef_closure_fit_norm: need features, targets and n >= 2"); return EF_ERR_ARG; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    column_stats<<<NIN, 256, 0, s>>>(feats, n, NIN, 1, c->stats, c->stats + 10);
    column_stats<<<NOUT, 256, 0, s>>>(tau, n, NOUT, 0, c->stats + 20, c->stats + 26);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "column_stats");
    c->fitted = true;
    return EF_OK;
}

int ef_closure_train(ef_closure *c, const float *feats, const float *tau, long n, int epochs, void *stream,
                     float *loss_out)
{
    int rc = check_closure(c, "ef_closure_train");
    if (rc) return rc;
    if (!feats || !tau || n < 1 || epochs < 0) { set_error("ef_closure_train: bad arguments"); return EF_ERR_ARG; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!c->fitted && (rc = ef_closure_fit_norm(c, feats, tau, n, stream))) return rc;
    const int B = c->cfg.batch;
    const long nbatch = (n + B - 1) / B;
    const long nfull = n / B;            // full batches: one captured step replayed; a partial last one launched
    const float b1 = 0.9f, b2 = 0.999f;
    std::vector<long> perm(n);
    std::vector<float> c12(2 * (size_t)nbatch);
    long *d_perm = nullptr, *d_bt = nullptr;
    float *d_c12 = nullptr;
    double *d_loss = nullptr;
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = dev_malloc(&d_perm, sizeof(long) * (size_t)n);
    if (e == cudaSuccess) e = dev_malloc(&d_loss, sizeof(double));
    if (e == cudaSuccess) e = dev_malloc(&d_bt, sizeof(long));
    if (e == cudaSuccess) e = dev_malloc(&d_c12, sizeof(float) * c12.size());
    if (e == cudaSuccess) e = cudaMemsetAsync(d_loss, 0, sizeof(double), s);
    // one training step of a full batch, captured on a private stream: the
    // batch index and the step's bias corrections are read on the device
    if (e == cudaSuccess && nfull > 0 && epochs > 0) {
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            gather_batch_at<<<grid1(B), 256, 0, cs>>>(feats, tau, n, d_perm, d_bt, B, c->stats, c->stats + 10,
                                                        c->stats + 20, c->stats + 26, c->H[0], c->T);
            forward(c, B, cs);
            mse_grad<<<grid1(B), 256, 0, cs>>>(c->H[NLAYER], c->T, c->dA, c->rowloss, B);
            backward(c, B, cs);
            adam_step_at<<<grid1(c->nparam), 256, 0, cs>>>(c->w, c->wq, c->g, c->m, c->v, c->nparam, c->cfg.lr, b1,
                                                             b2, 1e-8f, d_c12, d_bt);
            sum_into<<<1, 256, 0, cs>>>(c->rowloss, B, d_loss);
            next_batch<<<1, 1, 0, cs>>>(d_bt);
            const cudaError_t el = cudaGetLastError();
            e = cudaStreamEndCapture(cs, &graph);
            if (e == cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    }
    for (int ep = 0; ep < epochs && e == cudaSuccess; ep++) {
        // deterministic order: sort points by a hash of (seed, epoch index,
        // point).  The shuffle only decides which points share a batch, so a
        // set that fits one batch is taken in its stored order.
        const unsigned long long key = mix(c->cfg.seed ^ mix(0x5eedull + (unsigned long long)(c->step / nbatch)));
        for (long i = 0; i < n; i++) perm[i] = i;
        for (long i = nbatch > 1 ? n - 1 : 0; i > 0; i--) {
            const long j = (long)(mix(key + (unsigned long long)i) % (unsigned long long)(i + 1));
            const long t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
        for (long bt = 0; bt < nbatch; bt++) {   // Adam's bias corrections of the epoch's steps
            const long st = c->step + 1 + bt;
            c12[2 * bt] = 1.f - powf(b1, (float)st);
            c12[2 * bt + 1] = 1.f - powf(b2, (float)st);
        }
        // the host buffers are refilled next epoch: the copies must have landed
        e = cudaMemcpyAsync(d_perm, perm.data(), sizeof(long) * (size_t)n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_c12, c12.data(), sizeof(float) * c12.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_bt, 0, sizeof(long), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_loss, 0, sizeof(double), s);   // the last epoch's loss is kept
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        for (long bt = 0; bt < nfull && e == cudaSuccess; bt++) e = cudaGraphLaunch(exec, s);
        for (long bt = nfull; bt < nbatch && e == cudaSuccess; bt++) {   // the partial last batch
            const int nb = (int)(n - bt * B);
            gather_batch<<<grid1(nb), 256, 0, s>>>(feats, tau, n, d_perm + bt * B, nb, c->stats, c->stats + 10,
                                                   c->stats + 20, c->stats + 26, c->H[0], c->T);
            forward(c, nb, s);
            mse_grad<<<grid1(nb), 256, 0, s>>>(c->H[NLAYER], c->T, c->dA, c->rowloss, nb);
            backward(c, nb, s);
            adam_step<<<grid1(c->nparam), 256, 0, s>>>(c->w, c->wq, c->g, c->m, c->v, c->nparam, c->cfg.lr, b1, b2,
                                                      1e-8f, c12[2 * bt], c12[2 * bt + 1]);
            sum_into<<<1, 256, 0, s>>>(c->rowloss, nb, d_loss);
            e = cudaGetLastError();
        }
        c->step += nbatch;
    }
    double loss_sum = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&loss_sum, d_loss, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    cudaFree(d_perm);
    cudaFree(d_loss);
    cudaFree(d_bt);
    cudaFree(d_c12);
    if (e != cudaSuccess) return cuda_fail(e, "ef_closure_train");
    if (loss_out) *loss_out = epochs > 0 ? (float)(loss_sum / ((double)n * NOUT)) : 0.f;
    return EF_OK;
}

int ef_closure_infer(ef_closure *c, const float *feats, float *tau_out, long n, const float *exact_tau,
                     long *n_fallback, void *stream)
{
    int rc = check_closure(c, "ef_closure_infer");
    if (rc) return rc;
    if (!feats || !tau_out || n < 1) { set_error("ef_closure_infer: bad arguments"); return EF_ERR_ARG; }
    if (!c->fitted) { set_error("ef_closure_infer: the closure has not been fitted or loaded"); return EF_ERR_ARG; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(c->nfall, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "ef_closure_infer");
    rc = closure_infer_tc(c->wq, c->off_w, c->off_b, c->stats, c->image, feats, n, c->cfg.guard_sigma, exact_tau,
                          tau_out, c->nfall, c->nfall + 1, s);
    if (rc) return rc;
    if (n_fallback) {
        int w[2] = {0, 0};
        e = cudaMemcpyAsync(w, c->nfall, sizeof w, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "fallback count");
        if (w[1]) {
            cudaMemsetAsync(c->nfall + 1, 0, sizeof(int), s);
            set_error("ef_closure_infer: device error %d (a wait ran out)", w[1]);
            return w[1];
        }
        *n_fallback = w[0];
    }
    return EF_OK;
}

int ef_closure_infer_exact(ef_closure *c, const float *feats, float *tau_out, long n, ef_plan *plan, const void *u,
                           long *n_fallback, void *stream)
{
    int rc = check_closure(c, "ef_closure_infer_exact");
    if (rc) return rc;
    if (!plan || !u) { set_error("ef_closure_infer_exact: a plan and its DNS snapshot are required"); return EF_ERR_ARG; }
    if (plan->diff) { set_error("ef_closure_infer_exact: the fallback needs a Gaussian-kernel plan"); return EF_ERR_UNSUPPORTED; }
    if (n != (long)plan->nlx * plan->nly * plan->nlz) {
        set_error("ef_closure_infer_exact: n (%ld) must be the plan's LES point count (%ld)", n,
                  (long)plan->nlx * plan->nly * plan->nlz);
        return EF_ERR_SHAPE;
    }
    if ((rc = ef_closure_infer(c, feats, tau_out, n, nullptr, nullptr, stream))) return rc;
    ExactFallbackArgs a;
    memset(&a, 0, sizeof a);
    a.feats = feats; a.n = n; a.guard = c->cfg.guard_sigma;
    a.image = static_cast<const unsigned char *>(c->image);
    if (plan->prec == EF_PREC_FP64) a.u64 = static_cast<const double *>(u);
    else a.u32 = static_cast<const float *>(u);
    a.np = (size_t)plan->nx * plan->ny * plan->nz;
    a.nx = plan->nx; a.ny = plan->ny; a.nz = plan->nz; a.nlx = plan->nlx; a.nly = plan->nly; a.nlz = plan->nlz;
    a.xstart = plan->bx.d_start; a.xw = plan->bx.d_w64; a.Tx = plan->bx.T;
    a.zstart = plan->bz.d_start; a.zw = plan->bz.d_w64; a.Tz = plan->bz.T;
    a.ystart = plan->d_ystart; a.ycount = plan->d_ycount; a.yw[0] = plan->d_yw64[0]; a.yw[1] = plan->d_yw64[1];
    for (int k = 0; k < 3; k++) a.par[k] = plan->par[k];
    a.tau = tau_out;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = closure_exact_fallback(a, s))) return rc;
    if (n_fallback) {
        int w[2] = {0, 0};
        cudaError_t e = cudaMemcpyAsync(w, c->nfall, sizeof w, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "fallback count");
        if (w[1]) {
            cudaMemsetAsync(c->nfall + 1, 0, sizeof(int), s);
            set_error("ef_closure_infer_exact: device error %d (a wait ran out)", w[1]);
            return w[1];
        }
        *n_fallback = w[0];
    }
    return EF_OK;
}

int ef_closure_check_device_error(ef_closure *c, void *stream)
{
    int rc = check_closure(c, "ef_closure_check_device_error");
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int code = 0;
    cudaError_t e = cudaMemcpyAsync(&code, c->nfall + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->nfall + 1, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "ef_closure_check_device_error");
    if (code) set_error("closure device error %d (a wait ran out)", code);
    return code;
}

int ef_closure_gradients(ef_closure *c, const float *feats, const float *tau, long n, float *grad_out,
                         float *loss_out, void *stream)
{
    int rc = check_closure(c, "ef_closure_gradients");
    if (rc) return rc;
    if (!feats || !tau || n < 1 || n > c->cap) { set_error("ef_closure_gradients: 1 <= n <= batch"); return EF_ERR_ARG; }
    if (!c->fitted) { set_error("ef_closure_gradients: not fitted"); return EF_ERR_ARG; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    iota_range<<<grid1(n), 256, 0, s>>>(c->idx, 0, (int)n);
    gather_batch<<<grid1(n), 256, 0, s>>>(feats, tau, n, c->idx, (int)n, c->stats, c->stats + 10, c->stats + 20,
                                          c->stats + 26, c->H[0], c->T);
    forward(c, (int)n, s);
    mse_grad<<<grid1(n), 256, 0, s>>>(c->H[NLAYER], c->T, c->dA, c->rowloss, (int)n);
    backward(c, (int)n, s);
    std::vector<float> rl(n);
    cudaError_t e = cudaMemcpyAsync(grad_out, c->g, sizeof(float) * c->nparam, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rl.data(), c->rowloss, sizeof(float) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "ef_closure_gradients");
    if (loss_out) {
        double t = 0.0;
        for (long i = 0; i < n; i++) t += rl[i];
        *loss_out = (float)(t / ((double)n * NOUT));
    }
    return EF_OK;
}

long ef_closure_param_count(const ef_closure *c) { return c ? c->nparam : 0; }

int ef_closure_get_params(const ef_closure *c, float *host, double *norm_stats)
{
    int rc = check_closure(c, "ef_closure_get_params");
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    if (host) e = cudaMemcpy(host, c->w, sizeof(float) * c->nparam, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && norm_stats) e = cudaMemcpy(norm_stats, c->stats, sizeof(double) * 32, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "ef_closure_get_params");
    return EF_OK;
}

int ef_closure_set_params(ef_closure *c, const float *host, const double *norm_stats)
{
    int rc = check_closure(c, "ef_closure_set_params");
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    if (host) {
        e = cudaMemcpy(c->w, host, sizeof(float) * c->nparam, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            round_copy<<<grid1(c->nparam), 256>>>(c->w, c->wq, c->nparam);
            e = cudaDeviceSynchronize();
        }
    }
    if (e == cudaSuccess && norm_stats) {
        e = cudaMemcpy(c->stats, norm_stats, sizeof(double) * 32, cudaMemcpyHostToDevice);
        c->fitted = true;
    }
    if (e != cudaSuccess) return cuda_fail(e, "ef_closure_set_params");
    return EF_OK;
}

// Checkpoint: magic, version, counts, step, the four parameter arrays (w, m,
// v) and the statistics, then a CRC-32 of everything before it.
static unsigned crc32(const unsigned char *p, size_t n, unsigned crc = 0)
{
    crc = ~crc;
    for (size_t i = 0; i < n; i++) {
        crc ^= p[i];
        for (int k = 0; k < 8; k++) crc = (crc >> 1) ^ (0xedb88320u & (0u - (crc & 1u)));
    }
    return ~crc;
}

int ef_closure_save(const ef_closure *c, const char *path)
{
    int rc = check_closure(c, "ef_closure_save");
    if (rc) return rc;
    if (!path) { set_error("ef_closure_save: NULL path"); return EF_ERR_ARG; }
    std::vector<unsigned char> buf;
    auto put = [&](const void *p, size_t n) { buf.insert(buf.end(), (const unsigned char *)p, (const unsigned char *)p + n); };
    const char magic[8] = {'E', 'L', 'E', 'S', 'M', 'L', 'P', '1'};
    put(magic, 8);
    const long hdr[4] = {c->nparam, c->step, c->fitted ? 1 : 0, (long)c->cfg.seed};
    put(hdr, sizeof hdr);
    std::vector<float> h(c->nparam);
    const float *arrs[3] = {c->w, c->m, c->v};
    for (auto a : arrs) {
        cudaError_t e = cudaMemcpy(h.data(), a, sizeof(float) * c->nparam, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "ef_closure_save");
        put(h.data(), sizeof(float) * c->nparam);
    }
    double st[32];
    cudaError_t e = cudaMemcpy(st, c->stats, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "ef_closure_save");
    put(st, sizeof st);
    const unsigned crc = crc32(buf.data(), buf.size());
    put(&crc, sizeof crc);
    FILE *f = fopen(path, "wb");
    if (!f) { set_error("ef_closure_save: cannot open %s", path); return EF_ERR_ARG; }
    const size_t wr = fwrite(buf.data(), 1, buf.size(), f);
    fclose(f);
    if (wr != buf.size()) { set_error("ef_closure_save: short write"); return EF_ERR_ARG; }
    return EF_OK;
}

int ef_closure_load(ef_closure *c, const char *path)
{
    int rc = check_closure(c, "ef_closure_load");
    if (rc) return rc;
    if (!path) { set_error("ef_closure_load: NULL path"); return EF_ERR_ARG; }
    FILE *f = fopen(path, "rb");
    if (!f) { set_error("ef_closure_load: cannot open %s", path); return EF_ERR_ARG; }
    std::vector<unsigned char> buf;
    unsigned char tmp[65536];
    size_t r;
    while ((r = fread(tmp, 1, sizeof tmp, f)) > 0) buf.insert(buf.end(), tmp, tmp + r);
    fclose(f);
    const size_t need = 8 + 4 * sizeof(long) + 3 * sizeof(float) * (size_t)c->nparam + 32 * sizeof(double) + 4;
    if (buf.size() != need || memcmp(buf.data(), "ELESMLP1", 8) != 0) {
        set_error("ef_closure_load: not a checkpoint of this closure");
        return EF_ERR_ARG;
    }
    unsigned crc;
    memcpy(&crc, buf.data() + need - 4, 4);
    if (crc != crc32(buf.data(), need - 4)) { set_error("ef_closure_load: checksum mismatch"); return EF_ERR_ARG; }
    long hdr[4];
    memcpy(hdr, buf.data() + 8, sizeof hdr);
    if (hdr[0] != c->nparam) { set_error("ef_closure_load: parameter count differs"); return EF_ERR_ARG; }
    c->step = hdr[1];
    c->fitted = hdr[2] != 0;
    size_t off = 8 + sizeof hdr;
    float *arrs[3] = {c->w, c->m, c->v};
    cudaError_t e = cudaSuccess;
    for (auto a : arrs) {
        if (e == cudaSuccess) e = cudaMemcpy(a, buf.data() + off, sizeof(float) * c->nparam, cudaMemcpyHostToDevice);
        off += sizeof(float) * c->nparam;
    }
    if (e == cudaSuccess) e = cudaMemcpy(c->stats, buf.data() + off, 32 * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        round_copy<<<grid1(c->nparam), 256>>>(c->w, c->wq, c->nparam);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) return cuda_fail(e, "ef_closure_load");
    return EF_OK;
}

}  // extern "C"
