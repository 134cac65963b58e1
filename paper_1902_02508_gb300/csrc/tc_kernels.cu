// Fused x-z kernel with the x-contraction on the tensor cores, split-BF16
// operands and FP32 accumulation (EF_PREC_BF16X3).
//
// The staging, the reference profile, the plane means and the z phase are
// those of the CUDA-core kernel (fused_stage.cuh).  What changes is the x
// contraction of one stage = one chunk of 16 inputs (two row blocks of 8):
//
//   D[16 rows x 8 outputs] += A[16 rows x 16 inputs] * B[16 inputs x 8 outputs]
//
// one warp-wide mma.sync.m16n8k16 per (16-row tile, field, split product).
// B is the same for every chunk (the operator is a strided convolution): the
// chunk whose first block is b0 feeds outputs X0 + n, X0 = b0 + dmin, with
// B[k][n] = W[k % 8][n - k / 8] (zero outside the ring).  Consecutive chunks
// shift the output window by two, so after each chunk the accumulator tile
// emits its first two columns (complete) and slides left by two columns with
// one quad shuffle.  Every operand x is split as x = hi + lo with hi = bf16(x),
// lo = bf16(x - hi) (both round-to-nearest), and the product is
//   A B ~= Ahi Bhi + Alo Bhi + Ahi Blo,
// dropping only Alo Blo (~2^-18 relative).  Each warp owns 32 z-rows (two
// 16-row tiles); rows are the M dimension, so no output is shared between
// warps.
#include <math.h>
#include <string.h>

#include <vector>

#include "eles_internal.h"
#include "fused_stage.cuh"

namespace eles {
namespace {

using namespace fz;

__device__ __forceinline__ unsigned pack_bf16(float lo_k, float hi_k)
{
    unsigned d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi_k), "f"(lo_k));
    return d;
}

// x = hi + lo for a pair (k, k+1): returns the packed hi pair and the packed lo pair.
__device__ __forceinline__ void split_pair(float x0, float x1, unsigned &hi, unsigned &lo)
{
    hi = pack_bf16(x0, x1);
    const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xffff0000u);
    lo = pack_bf16(x0 - h0, x1 - h1);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1)
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <int F>
__device__ __forceinline__ float field(float v0, float v1, float v2)
{
    return F == 0 ? v0 : F == 1 ? v1 : F == 2 ? v2 : F == 3 ? v0 * v0 : F == 4 ? v0 * v1
         : F == 5 ? v0 * v2 : F == 6 ? v1 * v1 : F == 7 ? v1 * v2 : v2 * v2;
}

// z phase on the tensor cores: for the parked columns (col = xo * 9 + f,
// z contiguous in colbuf) and every tile of 16 Z outputs,
//   h[Z][col] = sum_z Az[Z][z] g[z][col],  M = Z, N = col, K = z,
// with the band of each Z tile covered by KS k-steps starting at
// z = 16 RZ zt - zoff.  The A fragments of every k-step are the same for all
// Z tiles (strided convolution) and sit in shared memory (hi, lo); the B
// fragments are split from the FP32 parked values on the fly.
template <int RZ>
__device__ __forceinline__ void zphase_tc(const FusedArgs &a, const float *colbuf, int ld, const uint4 *afrag,
                                          int KS, int zoff, int s, int j, int Xs, int cnt, int warp, int nwarps,
                                          int lane)
{
    const int g = lane >> 2, t = lane & 3;
    const int ncol = a.P * NF, ntile = (ncol + 7) / 8;
    const int nitems = (a.nlz / 16) * ntile;
    for (int it = warp; it < nitems; it += nwarps) {
        const int zt = it / ntile, nt = it - zt * ntile;
        const int colb = nt * 8 + g;                     // this lane's B column
        const bool bval = colb < ncol && colb / NF < cnt;
        const float *cb = colbuf + (size_t)(bval ? colb : 0) * ld;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        int z0 = 16 * RZ * zt - zoff;
        for (int kk = 0; kk < KS; kk++, z0 += 16) {
            const uint4 ah = afrag[(kk * 32 + lane) * 2], al = afrag[(kk * 32 + lane) * 2 + 1];
            int za = z0 + 2 * t, zb = za + 8;
            za = za < 0 ? za + a.nz : (za >= a.nz ? za - a.nz : za);
            zb = zb < 0 ? zb + a.nz : (zb >= a.nz ? zb - a.nz : zb);
            float2 va = *reinterpret_cast<const float2 *>(cb + za);
            float2 vb = *reinterpret_cast<const float2 *>(cb + zb);
            if (!bval) { va = make_float2(0.f, 0.f); vb = va; }
            unsigned bh0, bl0, bh1, bl1;
            split_pair(va.x, va.y, bh0, bl0);
            split_pair(vb.x, vb.y, bh1, bl1);
            mma_bf16(acc, ah.x, ah.y, ah.z, ah.w, bh0, bh1);
            mma_bf16(acc, al.x, al.y, al.z, al.w, bh0, bh1);
            mma_bf16(acc, ah.x, ah.y, ah.z, ah.w, bl0, bl1);
        }
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const int c = nt * 8 + 2 * t + e;
            if (c >= ncol) continue;
            const int xo = c / NF, f = c - xo * NF;
            if (xo >= cnt || f >= a.nf) continue;
            float *hout = a.h + ((((size_t)s * NF + f) * a.ny + j) * a.nlz + 16 * zt) * a.nlx + Xs + xo;
            hout[(size_t)g * a.nlx] = acc[e];
            hout[(size_t)(g + 8) * a.nlx] = acc[2 + e];
        }
    }
}

template <int RZ, int DZ, bool ZTC>
__global__ void __launch_bounds__(kFusedMaxRows) xz_fused_tc(const __grid_constant__ FusedTCArgs ta)
{
    const FusedArgs &a = ta.f;
    constexpr int RX = 8;
    using S = Stg<RX>;
    constexpr int SB = S::SB;                  // 2 blocks per stage = one 16-input chunk
    extern __shared__ float4 smem_dyn[];
    const int ld = ZTC ? a.nz + 8 : a.nz + 1;   // +8: conflict-free 8-byte B loads
    uint4 *afrag = reinterpret_cast<uint4 *>(smem_dyn);                           // [KS][32][2]
    float *colbuf = reinterpret_cast<float *>(afrag + (ZTC ? ta.KS * 64 : 0));
    float *stg;                                                                 // [TSTG][3][nz][TW], 1024-B aligned
    {
        char *end = reinterpret_cast<char *>(colbuf + (size_t)a.P * NF * ld);
        const unsigned sa = smem_u32(end);
        stg = reinterpret_cast<float *>(end + (((sa + 1023u) & ~1023u) - sa));
    }
    const size_t stg_floats = (size_t)3 * a.nz * TW;
    __shared__ alignas(8) unsigned long long full[TSTG];
    __shared__ double red[3][kFusedMaxRows / 32];
    __shared__ float Us[3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int nthr = blockDim.x;
    const int j = blockIdx.x, s = blockIdx.y;
    const size_t np = (size_t)a.nx * a.ny * a.nz;
    const float *plane = a.u + (size_t)s * 3 * np + (size_t)j * a.nz * a.nx;
    const int pc0 = s * 3 * a.ny + j;             // TMA plane coordinate of component 0

    // TMA stage k = row block k of the stream (8 inputs per row)
    auto stage_x = [&](int k) {
        int b = (k - a.bshift) % a.nlx;
        if (b < 0) b += a.nlx;
        return b * RX;
    };
    const int nts = a.nblk_x;                     // TMA stages (one row block each)
    if (tid == 0) {
        for (int i = 0; i < TSTG; i++) mbar_init(&full[i], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < TSTG && k < nts; k++)
            tma_stage(stg + k * stg_floats, &full[k], &a.tmap, a.nz, a.box_rows, stage_x(k), pc0, a.ny);
    }
    if constexpr (ZTC) {
        for (int i = tid; i < ta.KS * 64; i += blockDim.x) afrag[i] = ta.afrag[i];
    }
    for (int c = warp; c < 3; c += nthr / 32) {
        const float *r0 = plane + (size_t)c * np;
        double acc = 0.0;
        for (int i = lane; i < a.nx; i += 32) acc += (double)r0[i];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const float Uc = (float)(acc / a.nx);
            Us[c] = Uc;
            a.uref[((size_t)s * 3 + c) * a.ny + j] = (double)Uc;
        }
    }
    __syncthreads();
    const float U[3] = {Us[0], Us[1], Us[2]};
    const unsigned bh0 = ta.Bh[2 * lane], bh1 = ta.Bh[2 * lane + 1];
    const unsigned bl0 = ta.Bl[2 * lane], bl1 = ta.Bl[2 * lane + 1];

    float acc[2][NF][4];
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int f = 0; f < NF; f++)
#pragma unroll
            for (int i = 0; i < 4; i++) acc[m][f][i] = 0.f;
    float psum[3] = {0.f, 0.f, 0.f};

    const int nchunk = nts / 2;
    for (int sidx = 0; sidx < nchunk; sidx++) {
        const int ka = 2 * sidx, kb = 2 * sidx + 1;  // the chunk's two TMA stages
        mbar_wait(&full[ka % TSTG], (ka / TSTG) & 1, a.err);
        mbar_wait(&full[kb % TSTG], (kb / TSTG) & 1, a.err);
        const float *bufa = stg + (ka % TSTG) * stg_floats, *bufb = stg + (kb % TSTG) * stg_floats;
        const int b0 = sidx * SB - a.bshift;        // first row block of the chunk
        const bool own = b0 >= 0 && b0 < a.nlx;     // both blocks are owned or neither
#pragma unroll
        for (int m = 0; m < 2; m++) {
            float v[3][2][4];
            {
                const int r0 = warp * 32 + 16 * m + g;
#pragma unroll
                for (int c = 0; c < 3; c++)
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const size_t o = ((size_t)c * a.nz + r0 + 8 * h) * TW + 2 * t;
                        const float2 xa = *reinterpret_cast<const float2 *>(bufa + o);
                        const float2 xb = *reinterpret_cast<const float2 *>(bufb + o);
                        v[c][h][0] = xa.x; v[c][h][1] = xa.y; v[c][h][2] = xb.x; v[c][h][3] = xb.y;
                    }
            }
#pragma unroll
            for (int c = 0; c < 3; c++)
#pragma unroll
                for (int h = 0; h < 2; h++)
#pragma unroll
                    for (int e = 0; e < 4; e++) v[c][h][e] -= U[c];
            if (own) {
#pragma unroll
                for (int c = 0; c < 3; c++)
#pragma unroll
                    for (int h = 0; h < 2; h++) psum[c] += (v[c][h][0] + v[c][h][1]) + (v[c][h][2] + v[c][h][3]);
            }
#pragma unroll
            for (int f = 0; f < NF; f++) {
                float x[2][4];
#pragma unroll
                for (int h = 0; h < 2; h++)
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const float v0 = v[0][h][e], v1 = v[1][h][e], v2 = v[2][h][e];
                        x[h][e] = f == 0 ? field<0>(v0, v1, v2) : f == 1 ? field<1>(v0, v1, v2)
                                : f == 2 ? field<2>(v0, v1, v2) : f == 3 ? field<3>(v0, v1, v2)
                                : f == 4 ? field<4>(v0, v1, v2) : f == 5 ? field<5>(v0, v1, v2)
                                : f == 6 ? field<6>(v0, v1, v2) : f == 7 ? field<7>(v0, v1, v2)
                                : field<8>(v0, v1, v2);
                    }
                unsigned ah[4], al[4];
                split_pair(x[0][0], x[0][1], ah[0], al[0]);   // row g,   k 2t, 2t+1
                split_pair(x[1][0], x[1][1], ah[1], al[1]);   // row g+8, k 2t, 2t+1
                split_pair(x[0][2], x[0][3], ah[2], al[2]);   // row g,   k 2t+8, 2t+9
                split_pair(x[1][2], x[1][3], ah[3], al[3]);   // row g+8, k 2t+8, 2t+9
                mma_bf16(acc[m][f], ah[0], ah[1], ah[2], ah[3], bh0, bh1);
                mma_bf16(acc[m][f], al[0], al[1], al[2], al[3], bh0, bh1);
                mma_bf16(acc[m][f], ah[0], ah[1], ah[2], ah[3], bl0, bl1);
            }
        }
        // columns 0 and 1 of the tiles are outputs X0 and X0 + 1: complete
        const int X0 = b0 + a.dmin_x;
#pragma unroll
        for (int n = 0; n < 2; n++) {
            const int X = X0 + n;
            if (X >= 0 && X < a.nlx) {
                if (t == 0) {
#pragma unroll
                    for (int m = 0; m < 2; m++)
#pragma unroll
                        for (int f = 0; f < NF; f++) {
                            float *cb = colbuf + ((X & (a.P - 1)) * NF + f) * ld + warp * 32 + 16 * m + g;
                            cb[0] = acc[m][f][n];
                            cb[8] = acc[m][f][2 + n];
                        }
                }
                if ((X & (a.P - 1)) == a.P - 1 || X == a.nlx - 1) {
                    __syncthreads();
                    if constexpr (ZTC)
                        zphase_tc<RZ>(a, colbuf, ld, afrag, ta.KS, ta.zoff, s, j, X & ~(a.P - 1), (X & (a.P - 1)) + 1,
                                      warp, nthr / 32, lane);
                    else
                        zphase<RZ, DZ>(a, colbuf, ld, s, j, X & ~(a.P - 1), (X & (a.P - 1)) + 1, tid, nthr);
                    __syncthreads();
                }
            }
        }
        // slide every tile left by two columns (one lane of the quad)
#pragma unroll
        for (int m = 0; m < 2; m++)
#pragma unroll
            for (int f = 0; f < NF; f++)
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const float nb = __shfl_down_sync(0xffffffffu, acc[m][f][i], 1);
                    acc[m][f][i] = t == 3 ? 0.f : nb;
                }
        // every thread is done with the chunk's buffers: refill them
        __syncthreads();
        if (tid == 0) {
            proxy_fence();
            for (int k = ka + TSTG; k <= kb + TSTG; k++)
                if (k < nts) tma_stage(stg + (k % TSTG) * stg_floats, &full[k % TSTG], &a.tmap, a.nz, a.box_rows,
                                       stage_x(k), pc0, a.ny);
        }
    }
    if (a.plane_mean) {
        double d[3] = {psum[0], psum[1], psum[2]};
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < 3; c++) d[c] += __shfl_xor_sync(0xffffffffu, d[c], o);
        if (lane == 0) { red[0][warp] = d[0]; red[1][warp] = d[1]; red[2][warp] = d[2]; }
        __syncthreads();
        if (tid < 3) {
            double tt = 0.0;
            for (int w = 0; w < nthr / 32; w++) tt += red[tid][w];
            a.plane_mean[((size_t)s * 3 + tid) * a.ny + j] = (double)Us[tid] + tt / ((double)a.nx * a.nz);
        }
    }
}

template <int RZ, int DZ, bool ZTC>
cudaError_t launch(const FusedTCArgs &ta, int nsnap, cudaStream_t st)
{
    const FusedArgs &a = ta.f;
    const size_t smem = tc_smem_bytes(a.P, a.nz, ZTC ? ta.KS : 0);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(xz_fused_tc<RZ, DZ, ZTC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             222 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    xz_fused_tc<RZ, DZ, ZTC><<<dim3(a.ny, nsnap), a.nz, smem, st>>>(ta);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Warp-specialised variant (x_variant 3), for the tensor-core z phase.  One
// CTA per (snapshot, y-plane) with three roles that synchronise only through
// mbarriers, never through a CTA-wide barrier inside the stream:
//   * nz / 32 x warps (32 z-rows each) contract x on the tensor cores;
//   * one producer warp streams the plane through TMA stages (a full and an
//     empty barrier per stage) and refills a stage as soon as every x warp
//     has released it;
//   * kZW z warps contract z on the tensor cores for the two outputs each
//     chunk completes, from a double-buffered column buffer (a full and an
//     empty barrier per buffer).
// The accumulator tiles do not slide.  Output X lives in tile column
// (X - Xbase) mod 8 for the whole stream, where Xbase is the first output of
// chunk 0; the chunk's B operand is rotated accordingly (one pre-split B
// fragment per rotation q = chunk mod 4), so the two outputs a chunk
// completes always sit in tile columns 2q and 2q + 1, held by the lanes with
// t == q, which write them out and clear them.  A chunk touches at most
// D + 1 <= 7 outputs, so the eighth column (X0 + 7, tile column 2q + 7 mod 8)
// is idle for the chunk: its B column is all ones and it collects the row
// sums of the chunk's fluctuation, which make the plane means.
constexpr int kZW = 3;   // z warps
constexpr int CW = kTcwsStageWidth;   // floats per row per TMA stage: one chunk (two row blocks of 8)
static_assert(CW == 16, "a stage is one chunk of two row blocks of 8");
constexpr int CSTG = 2;  // stages in flight

// Issue chunk stage `buf` (one thread): 3 components x (nz / box rows) boxes of
// CW floats starting at column xstart.
__device__ __forceinline__ void tma_chunk(float *buf, unsigned long long *bar, const CUtensorMap *map, int nz,
                                          int box_rows, int xstart, int pc0, int ny)
{
    mbar_expect_tx(bar, 3u * nz * CW * 4u);
    for (int c = 0; c < 3; c++)
        for (int r0 = 0; r0 < nz; r0 += box_rows)
            tma_load3(buf + ((size_t)c * nz + r0) * CW, map, bar, xstart, r0, pc0 + c * ny);
}

// x = hi + lo for a pair (k, k+1), with a packed FP32 subtraction.
__device__ __forceinline__ void split2(float2 x, unsigned &hi, unsigned &lo)
{
    hi = pack_bf16(x.x, x.y);
    const float2 h = make_float2(__uint_as_float(hi << 16), __uint_as_float(hi & 0xffff0000u));
    const float2 l = __ffma2_rn(h, make_float2(-1.f, -1.f), x);
    lo = pack_bf16(l.x, l.y);
}

template <int F>
__device__ __forceinline__ float2 field2(float2 v0, float2 v1, float2 v2)
{
    if constexpr (F == 0) return v0;
    else if constexpr (F == 1) return v1;
    else if constexpr (F == 2) return v2;
    else if constexpr (F == 3) return __fmul2_rn(v0, v0);
    else if constexpr (F == 4) return __fmul2_rn(v0, v1);
    else if constexpr (F == 5) return __fmul2_rn(v0, v2);
    else if constexpr (F == 6) return __fmul2_rn(v1, v1);
    else if constexpr (F == 7) return __fmul2_rn(v1, v2);
    else return __fmul2_rn(v2, v2);
}

// Fields F.. NF-1 of one 16-row tile: v[c][h][blk] holds component c at rows
// g + 8h and chunk inputs k = 8 blk + 2t, 2t + 1.
template <int F>
__device__ __forceinline__ void x_mma(float (&acc)[NF][4], const float2 (&v)[3][2][2], const uint4 &B)
{
    unsigned ah[4], al[4];
    split2(field2<F>(v[0][0][0], v[1][0][0], v[2][0][0]), ah[0], al[0]);   // row g,     k 2t, 2t+1
    split2(field2<F>(v[0][1][0], v[1][1][0], v[2][1][0]), ah[1], al[1]);   // row g + 8, k 2t, 2t+1
    split2(field2<F>(v[0][0][1], v[1][0][1], v[2][0][1]), ah[2], al[2]);   // row g,     k 2t+8, 2t+9
    split2(field2<F>(v[0][1][1], v[1][1][1], v[2][1][1]), ah[3], al[3]);   // row g + 8, k 2t+8, 2t+9
    mma_bf16(acc[F], ah[0], ah[1], ah[2], ah[3], B.x, B.y);
    mma_bf16(acc[F], al[0], al[1], al[2], al[3], B.x, B.y);
    mma_bf16(acc[F], ah[0], ah[1], ah[2], ah[3], B.z, B.w);
    // order 0 3 4 5 | 1 6 7 | 2 8: each component's pairs die as early as possible
    constexpr int next = F == 0 ? 3 : F == 3 ? 4 : F == 4 ? 5 : F == 5 ? 1 : F == 1 ? 6 : F == 6 ? 7
                       : F == 7 ? 2 : F == 2 ? 8 : -1;
    if constexpr (next >= 0) x_mma<next>(acc, v, B);
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait shared by the roles: once any wait of the CTA has run out, the
// others return at once (the error word tells the host; results are garbage).
__device__ __forceinline__ void wait_or_abort(unsigned long long *bar, unsigned parity, volatile int *abort_flag,
                                              int *err)
{
    if (mbar_try_wait(bar, parity)) return;
    const long long t0 = clock64();
    while (clock64() - t0 < kWaitCycles) {
        if (*abort_flag) return;
        if (mbar_try_wait(bar, parity)) return;
    }
    *abort_flag = 1;
    if (err) atomicCAS(err, 0, (int)EF_ERR_TIMEOUT);
}

// z work of the warp-specialised kernel: Z tile zt (16 outputs) x column
// tiles nt0 .. nt0 + NT - 1 (8 of the 2 NF parked columns each, column
// c = n NF + f for output X0 + n), KS k-steps over the tile's z window.
// The parked columns hold, per 16-row block and pair i < 8, the split
// (hi, lo) words of rows (i, i + 8); the k index of a k-step runs over the
// block's rows in the order k = 2i + e -> row i + 8e, which the A fragments
// follow.  So lane (g, t) loads its B fragment words, pairs t and t + 4, as
// two 8-byte words and splits nothing.  One A fragment load per k-step feeds
// all NT column tiles.  The window starts on a 16-row boundary (zoff is a
// multiple of 16), so a k-step wraps periodically as a whole or not at all.
// Lanes whose column is idle read a zero column.
template <int RZ, int NT>
__device__ __forceinline__ void z_tile(const FusedArgs &a, const float *colb, const float *zero_col, int ld,
                                       const uint4 *afrag, int KS, int zoff, int s, int j, int X0, bool val0,
                                       bool val1, int zt, int nt0, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    const uint2 *cp[NT];
#pragma unroll
    for (int i = 0; i < NT; i++) {
        const int c = (nt0 + i) * 8 + g;          // this lane's B column
        const bool bval = c < 2 * NF && (c < NF ? val0 : val1);
        cp[i] = reinterpret_cast<const uint2 *>(bval ? colb + (size_t)c * ld : zero_col) + t;
    }
    float acc[NT][3][4];   // one accumulator per split product: independent chains
#pragma unroll
    for (int i = 0; i < NT; i++)
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int e = 0; e < 4; e++) acc[i][r][e] = 0.f;
    int z0 = 16 * RZ * zt - zoff;
#pragma unroll 2
    for (int kk = 0; kk < KS; kk++, z0 += 16) {
        const int zr = (z0 < 0 ? z0 + a.nz : (z0 >= a.nz ? z0 - a.nz : z0)) >> 1;   // in 8-byte words
        const uint4 ah = afrag[(2 * kk) * 32 + lane], al = afrag[(2 * kk + 1) * 32 + lane];
#pragma unroll
        for (int i = 0; i < NT; i++) {
            const uint2 w0 = cp[i][zr], w1 = cp[i][zr + 4];     // pairs t and t + 4: (hi, lo)
            mma_bf16(acc[i][0], ah.x, ah.y, ah.z, ah.w, w0.x, w1.x);
            mma_bf16(acc[i][1], al.x, al.y, al.z, al.w, w0.x, w1.x);
            mma_bf16(acc[i][2], ah.x, ah.y, ah.z, ah.w, w0.y, w1.y);
        }
    }
#pragma unroll
    for (int i = 0; i < NT; i++)
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const int cc = (nt0 + i) * 8 + 2 * t + e;
            if (cc >= 2 * NF) continue;
            const int n = cc >= NF ? 1 : 0, f = cc - n * NF;
            if (f >= a.nf || !(n ? val1 : val0)) continue;
            float *hout = a.h + ((((size_t)s * NF + f) * a.ny + j) * a.nlz + 16 * zt) * a.nlx + X0 + n;
            hout[(size_t)g * a.nlx] = (acc[i][0][e] + acc[i][1][e]) + acc[i][2][e];
            hout[(size_t)(g + 8) * a.nlx] = (acc[i][0][2 + e] + acc[i][1][2 + e]) + acc[i][2][2 + e];
        }
}

__device__ __forceinline__ void named_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

template <int RZ, bool PM>   // PM: plane means requested
__global__ void __launch_bounds__(kFusedMaxRows + 32 * (1 + kZW), 1) xz_tc_ws(const __grid_constant__ FusedTCArgs ta)
{
    const FusedArgs &a = ta.f;
    constexpr int RX = 8;
    extern __shared__ float4 smem_dyn[];
    const int nxw = a.nz >> 5;                 // x warps; warp nxw is the producer, the rest z warps
    const int ld = a.nz + 8;                   // column stride (floats); +8: conflict-free 8-byte B loads
    const int KS = ta.KS;
    uint4 *afrag = reinterpret_cast<uint4 *>(smem_dyn);        // [KS][hi, lo][32 lanes]
    uint4 *bvar = afrag + KS * 64;                              // [4 rotations][32 lanes]
    constexpr int NCB = 2 * NF + 3;                             // parked columns: 2 outputs x NF fields, 3 row sums
    float *colbuf = reinterpret_cast<float *>(bvar + 128);      // [2 buffers][NCB][ld], then a zero column
    float *zero_col = colbuf + (size_t)2 * NCB * ld;
    float *stg;                                                 // [CSTG][3][nz][CW], 1024-B aligned
    {
        char *end = reinterpret_cast<char *>(zero_col + ld);
        const unsigned sa = smem_u32(end);
        stg = reinterpret_cast<float *>(end + (((sa + 1023u) & ~1023u) - sa));
    }
    const size_t stg_floats = (size_t)3 * a.nz * CW;
    __shared__ alignas(8) unsigned long long full[CSTG], empty[CSTG], cfull[2], cempty[2];
    __shared__ float Us[3];
    __shared__ int abort_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int j = blockIdx.x, s = blockIdx.y;
    const size_t np = (size_t)a.nx * a.ny * a.nz;
    const int nts = a.nblk_x, nchunk = nts >> 1;
    volatile int *abort_v = &abort_flag;

    if (tid == 0) {
        for (int i = 0; i < CSTG; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 32 * nxw);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&cfull[b], 32 * nxw);
            mbar_init(&cempty[b], 32 * kZW);
        }
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == nxw) {   // producer: stage k = chunk k = row blocks 2k, 2k + 1 of the stream
        if (lane == 0) {
            const int pc0 = s * 3 * a.ny + j;  // TMA plane coordinate of component 0
            int issued = 0;
            for (int k = 0; k < nchunk; k++) {
                const int st = k % CSTG;
                if (k >= CSTG) wait_or_abort(&empty[st], ((k / CSTG) - 1) & 1, abort_v, a.err);
                if (*abort_v) break;
                int b = (2 * k - a.bshift) % a.nlx;   // even, so the pair never wraps (nlx is even)
                if (b < 0) b += a.nlx;
                proxy_fence();
                tma_chunk(stg + st * stg_floats, &full[st], &a.tmap, a.nz, a.box_rows, b * RX, pc0, a.ny);
                issued = k + 1;
            }
            // no copy may be in flight when the CTA exits
            for (int k = issued > CSTG ? issued - CSTG : 0; k < issued; k++)
                mbar_wait(&full[k % CSTG], (k / CSTG) & 1, a.err);
        }
        return;
    }

    // x and z warps: z fragments, rotated x fragments, reference profile
    const int nwork = blockDim.x - 32;
    const int wtid = tid < 32 * nxw ? tid : tid - 32;
    for (int i = wtid; i < KS * 64; i += nwork) {
        const int kk = i >> 6, hl = (i >> 5) & 1, ln = i & 31;
        afrag[i] = ta.afrag_ws[(kk * 32 + ln) * 2 + hl];
    }
    for (int i = wtid; i < ld; i += nwork) zero_col[i] = 0.f;
    for (int i = wtid; i < 128; i += nwork) bvar[i] = ta.bvar[i];
    const float *plane = a.u + (size_t)s * 3 * np + (size_t)j * a.nz * a.nx;
    const int wk = warp < nxw ? warp : warp - 1;  // index among the x and z warps
    if (wk < 3) {
        const float *r0 = plane + (size_t)wk * np;
        double acc = 0.0;
        for (int i = lane; i < a.nx; i += 32) acc += (double)r0[i];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const float Uc = (float)(acc / a.nx);
            Us[wk] = Uc;
            a.uref[((size_t)s * 3 + wk) * a.ny + j] = (double)Uc;
        }
    }
    named_sync(1, nwork);

    if (warp < nxw) {   // ---------------- x warps
        volatile float *Uv = Us;    // re-read per tile: keeps three register pairs free
        float acc[2][NF][4];
#pragma unroll
        for (int m = 0; m < 2; m++)
#pragma unroll
            for (int f = 0; f < NF; f++)
#pragma unroll
                for (int i = 0; i < 4; i++) acc[m][f][i] = 0.f;
        for (int sidx = 0; sidx < nchunk; sidx++) {
            const int st = sidx % CSTG;
            wait_or_abort(&full[st], (sidx / CSTG) & 1, abort_v, a.err);
            const int q = sidx & 3;
            const uint4 B = bvar[q * 32 + lane];
            const float *buf = stg + st * stg_floats;
            const int b0 = 2 * sidx - a.bshift;        // first row block of the chunk
#pragma unroll
            for (int m = 0; m < 2; m++) {
                float2 v[3][2][2];
                const int r0 = warp * 32 + 16 * m + g;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const float nu = -Uv[c];
                    const float2 nU = make_float2(nu, nu);
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        // inputs 4t .. 4t + 3 of the chunk: k slots 2t, 2t + 1, 2t + 8, 2t + 9
                        const float4 x = *reinterpret_cast<const float4 *>(buf + ((size_t)c * a.nz + r0 + 8 * h) * CW + 4 * t);
                        v[c][h][0] = __fadd2_rn(make_float2(x.x, x.y), nU);
                        v[c][h][1] = __fadd2_rn(make_float2(x.z, x.w), nU);
                    }
                }
                x_mma<0>(acc[m], v, B);
            }
            mbar_arrive(&empty[st]);
            // the chunk completes outputs X0 and X0 + 1 (tile columns 2q, 2q + 1)
            const int cb = sidx & 1;
            if (sidx >= 2) wait_or_abort(&cempty[cb], ((sidx >> 1) - 1) & 1, abort_v, a.err);
            const int X0 = b0 + a.dmin_x;
            // park rows (g, g + 8) of each 16-row block as one pair (lanes t == q)
            float *colw = colbuf + (size_t)cb * NCB * ld + warp * 32 + 2 * g;
            if (t == q) {
#pragma unroll
                for (int n = 0; n < 2; n++)
                    if (X0 + n >= 0 && X0 + n < a.nlx) {
#pragma unroll
                        for (int m = 0; m < 2; m++)
#pragma unroll
                            for (int f = 0; f < NF; f++)
                                *reinterpret_cast<float2 *>(colw + (n * NF + f) * ld + 16 * m) =
                                    make_float2(acc[m][f][n], acc[m][f][2 + n]);
                    }
            }
            // the sum column 2 q3 + 1 (lanes t == q3) of fields 0-2 goes to parked
            // columns 2 NF + c when the chunk's blocks are owned (each input once)
            const int q3 = (q + 3) & 3;
            if (PM && t == q3 && b0 >= 0 && b0 < a.nlx) {
#pragma unroll
                for (int m = 0; m < 2; m++)
#pragma unroll
                    for (int c = 0; c < 3; c++)
                        *reinterpret_cast<float2 *>(colw + (2 * NF + c) * ld + 16 * m) =
                            make_float2(acc[m][c][1], acc[m][c][3]);
            }
            // clear the written columns (lanes t == q) and the sum column without a
            // branch; a non-finite value stays in its column, and the y pass flags it
            const float2 keep = make_float2(t == q ? 0.f : 1.f, t == q || t == q3 ? 0.f : 1.f);
#pragma unroll
            for (int m = 0; m < 2; m++)
#pragma unroll
                for (int f = 0; f < NF; f++) {
                    float2 lo = __fmul2_rn(make_float2(acc[m][f][0], acc[m][f][1]), keep);
                    float2 hi = __fmul2_rn(make_float2(acc[m][f][2], acc[m][f][3]), keep);
                    acc[m][f][0] = lo.x; acc[m][f][1] = lo.y; acc[m][f][2] = hi.x; acc[m][f][3] = hi.y;
                }
            // split the warp's parked pairs into (hi, lo) bf16 words in place, all
            // lanes sharing the work: 2 NF columns x 2 blocks x 8 pairs
            __syncwarp();
            {
                float *cw = colbuf + (size_t)cb * NCB * ld + warp * 32;
#pragma unroll
                for (int r = 0; r < NF; r++) {
                    const int pidx = lane + 32 * r, col = pidx >> 4, off = pidx & 15;
                    float2 *pp = reinterpret_cast<float2 *>(cw + (size_t)col * ld) + off;
                    unsigned hi, lo;
                    split2(*pp, hi, lo);
                    *reinterpret_cast<uint2 *>(pp) = make_uint2(hi, lo);
                }
            }
            mbar_arrive(&cfull[cb]);
        }
        return;
    }

    // ---------------- z warps: with three Z tiles z warp zw takes tile zw and
    // every column tile; otherwise the (Z tile, column tile) pairs round robin.
    // z warp c < 3 also sums the parked row sums of component c (plane means).
    const int zw = warp - nxw - 1;
    const int nzt = a.nlz / 16;
    double pmean = 0.0;
    for (int sidx = 0; sidx < nchunk; sidx++) {
        const int cb = sidx & 1;
        wait_or_abort(&cfull[cb], (sidx >> 1) & 1, abort_v, a.err);
        const int X0 = 2 * sidx - a.bshift + a.dmin_x;
        const bool val0 = X0 >= 0 && X0 < a.nlx, val1 = X0 + 1 >= 0 && X0 + 1 < a.nlx;
        const float *colb = colbuf + (size_t)cb * NCB * ld;
        if (PM && zw < 3) {
            const int b0 = 2 * sidx - a.bshift;
            if (b0 >= 0 && b0 < a.nlx) {
                float ssum = 0.f;
                for (int z = lane; z < a.nz; z += 32) ssum += colb[(2 * NF + zw) * ld + z];
                pmean += (double)ssum;
            }
        }
        if (val0 || val1) {
            if (nzt == kZW) {
                z_tile<RZ, 3>(a, colb, zero_col, ld, afrag, KS, ta.zoff, s, j, X0, val0, val1, zw, 0, lane);
            } else {
                for (int p = zw; p < 3 * nzt; p += kZW)
                    z_tile<RZ, 1>(a, colb, zero_col, ld, afrag, KS, ta.zoff, s, j, X0, val0, val1, p / 3, p % 3, lane);
            }
        }
        mbar_arrive(&cempty[cb]);
    }
    if (PM && zw < 3) {
        for (int o = 16; o > 0; o >>= 1) pmean += __shfl_xor_sync(0xffffffffu, pmean, o);
        if (lane == 0)
            a.plane_mean[((size_t)s * 3 + zw) * a.ny + j] = (double)Us[zw] + pmean / ((double)a.nx * a.nz);
    }
}

size_t ws_smem(int nz, int KS)
{
    return sizeof(uint4) * (64 * (size_t)KS + 128) + 1024
         + sizeof(float) * ((size_t)(2 * (2 * NF + 3) + 1) * (nz + 8) + (size_t)CSTG * 3 * nz * CW);
}

template <int RZ, bool PM>
cudaError_t launch_ws(const FusedTCArgs &ta, int nsnap, cudaStream_t st)
{
    const FusedArgs &a = ta.f;
    const size_t smem = ws_smem(a.nz, ta.KS);
    static size_t attr = 0;
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(xz_tc_ws<RZ, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    xz_tc_ws<RZ, PM><<<dim3(a.ny, nsnap), a.nz + 32 * (1 + kZW), smem, st>>>(ta);
    return cudaGetLastError();
}

// Round-to-nearest-even float -> bf16 bits (host).
unsigned short bf16_bits(float x)
{
    unsigned u;
    memcpy(&u, &x, 4);
    const unsigned rounding = 0x7fffu + ((u >> 16) & 1u);
    return (unsigned short)((u + rounding) >> 16);
}
float bf16_value(unsigned short b)
{
    const unsigned u = (unsigned)b << 16;
    float x;
    memcpy(&x, &u, 4);
    return x;
}

}  // namespace

#define ELES_TC_LIST(X) X(8, 8) X(8, 7)

bool tc_supported(int rx, int dx, int rz, int dz, int nlz)
{
    if (rx != 8 || dx > 7) return false;   // window of SB + D - 1 outputs fits one 8-column tile
    if (rz == 8 && nlz % 16 == 0) return true;   // z phase on the tensor cores
#define ELES_CASE(A, B) if (rz == A && dz == B) return true;
    ELES_TC_LIST(ELES_CASE)
#undef ELES_CASE
    return false;
}

// B fragments of the strided-convolution tile for every lane (hi and lo):
// lane (g = lane / 4, t = lane % 4) holds B[2t][g], B[2t+1][g] and
// B[2t+8][g], B[2t+9][g], the lower k in the low half.
void tc_weights(const Ring &rx, FusedTCArgs *ta)
{
    auto Bk = [&](int k, int n) -> double {
        const int lb = k / 8, e = k % 8, dd = n - lb;
        return (dd >= 0 && dd < rx.D) ? rx.W64[e * rx.D + dd] : 0.0;
    };
    for (int lane = 0; lane < 32; lane++) {
        const int g = lane / 4, t = lane % 4;
        for (int q = 0; q < 2; q++) {
            unsigned hi = 0, lo = 0;
            for (int e = 0; e < 2; e++) {
                const double w = Bk(2 * t + 8 * q + e, g);
                const unsigned short h = bf16_bits((float)w);
                const unsigned short l = bf16_bits((float)(w - (double)bf16_value(h)));
                hi |= (unsigned)h << (16 * e);
                lo |= (unsigned)l << (16 * e);
            }
            ta->Bh[2 * lane + q] = hi;
            ta->Bl[2 * lane + q] = lo;
        }
    }
}

cudaError_t launch_fused_tc(int rz, int dz, const FusedTCArgs &ta, int nsnap, cudaStream_t st)
{
    if (ta.KS > 0) {
        if (rz == 8) return launch<8, 8, true>(ta, nsnap, st);
        return cudaErrorInvalidValue;
    }
#define ELES_CASE(A, B) if (rz == A && dz == B) return launch<A, B, false>(ta, nsnap, st);
    ELES_TC_LIST(ELES_CASE)
#undef ELES_CASE
    return cudaErrorInvalidValue;
}

size_t tc_smem_bytes(int P, int nz, int KS)
{
    const int ld = KS > 0 ? nz + 8 : nz + 1;
    return sizeof(uint4) * 64 * (size_t)KS + 1024
         + sizeof(float) * ((size_t)P * NF * ld + (size_t)TSTG * 3 * nz * TW);
}

// TMA view of u [S][3][ny][nz][nx] as a 3-D tensor {nx, nz, 3 ny S}, boxes of
// box_w floats x box_rows rows.
int encode_u_map(const float *u, int nx, int ny, int nz, int nsnap, int box_w, int box_rows, CUtensorMap *map)
{
    typedef CUresult (*encode_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static encode_fn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p) {
            set_error("cuTensorMapEncodeTiled unavailable");
            return EF_ERR_CUDA;
        }
        fn = reinterpret_cast<encode_fn>(p);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)nz, (cuuint64_t)3 * ny * nsnap};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * nz * 4};
    const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(u), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return EF_ERR_CUDA;
    }
    return EF_OK;
}

// A fragments of the z operator for the tensor-core z phase: k-step kk,
// lane (g, t) holds A[g][2t..2t+1], A[g+8][2t..2t+1], A[g][2t+8..2t+9],
// A[g+8][2t+8..2t+9] with A[m][k] = w[16 kk + r(k) - RZ m - zoff], split into
// hi and lo bf16 pairs, where r(k) = k (natural order) or, with pairperm, the
// row order of the pre-split parked pairs, r(2i + e) = i + 8e.  Returns KS
// (0 if the z operator does not qualify).
int tc_zfrags(const Ring &rz, int nlz, std::vector<unsigned> &out, int *zoff_out, bool pairperm)
{
    if (rz.r != 8 || nlz % 16 != 0) return 0;
    const int R = rz.R, RZ = rz.r;
    const int zoff = (R + 15) / 16 * 16;   // window starts on 16-row boundaries
    const int KS = (zoff + 15 * RZ + R + 1 + 15) / 16;
    // Toeplitz weight at offset o = z - RZ Z: W[e][dd] with o = e - RZ (dd + dmin)
    auto w = [&](int o) -> double {
        if (o < -R || o > R) return 0.0;
        const int e = ((o % RZ) + RZ) % RZ;
        const int dd = (e - o) / RZ - rz.dmin;
        return (dd >= 0 && dd < rz.D) ? rz.W64[e * rz.D + dd] : 0.0;
    };
    out.assign((size_t)KS * 32 * 8, 0u);
    for (int kk = 0; kk < KS; kk++)
        for (int lane = 0; lane < 32; lane++) {
            const int g = lane / 4, t = lane % 4;
            const int rows[4] = {g, g + 8, g, g + 8}, kofs[4] = {0, 0, 8, 8};
            for (int r = 0; r < 4; r++) {
                unsigned hi = 0, lo = 0;
                for (int e = 0; e < 2; e++) {
                    const int k = 2 * t + kofs[r] + e;
                    const int row = pairperm ? (k >> 1) + 8 * (k & 1) : k;
                    const double v = w(16 * kk + row - RZ * rows[r] - zoff);
                    const unsigned short h = bf16_bits((float)v);
                    const unsigned short l = bf16_bits((float)(v - (double)bf16_value(h)));
                    hi |= (unsigned)h << (16 * e);
                    lo |= (unsigned)l << (16 * e);
                }
                out[((size_t)(kk * 32 + lane) * 2 + 0) * 4 + r] = hi;
                out[((size_t)(kk * 32 + lane) * 2 + 1) * 4 + r] = lo;
            }
        }
    *zoff_out = zoff;
    return KS;
}

// The warp-specialised kernel: stride 8 in x (window of 8 outputs) and the
// tensor-core z phase (stride 8, whole 16-output Z tiles).
bool tcws_supported(int rx, int dx, int rz, int nlz, int nz)
{
    // dx <= 6: a chunk leaves tile column X0 + 7 idle (the sum column)
    return rx == 8 && dx <= 6 && rz == 8 && nlz % 16 == 0 && nz % 32 == 0 && nz <= kFusedMaxRows;
}

size_t tcws_smem_bytes(int nz, int KS) { return ws_smem(nz, KS); }

// B fragments of the four rotations q of the x-operator tile: rotation q
// maps tile column c to output X0 + ((c - 2q) mod 8); the column of X0 + 7
// is all ones (row sums).  The k slots follow the chunk's inputs in the order
// the A fragments load them: k = 8 h8 + 2 t + e holds input 4 t + 2 h8 + e.
// Layout [q][lane][4]: hi (k 2t, 2t+1), hi (k 2t+8, 2t+9), lo (same), lo
// (same), lower k in the low half of each word.
void tc_bvar(const Ring &rx, std::vector<unsigned> &out)
{
    out.assign(4 * 32 * 4, 0u);
    for (int q = 0; q < 4; q++)
        for (int lane = 0; lane < 32; lane++) {
            const int g = lane / 4, t = lane % 4, n = (g - 2 * q) & 7;
            for (int kq = 0; kq < 2; kq++) {
                unsigned hi = 0, lo = 0;
                for (int e = 0; e < 2; e++) {
                    const int xi = 4 * t + 2 * kq + e;            // chunk input of slot k = 2t + 8kq + e
                    const int dd = n - xi / 8;
                    const double w = n == 7 ? 1.0 : (dd >= 0 && dd < rx.D) ? rx.W64[(xi % 8) * rx.D + dd] : 0.0;
                    const unsigned short h = bf16_bits((float)w);
                    const unsigned short l = bf16_bits((float)(w - (double)bf16_value(h)));
                    hi |= (unsigned)h << (16 * e);
                    lo |= (unsigned)l << (16 * e);
                }
                out[(q * 32 + lane) * 4 + kq] = hi;
                out[(q * 32 + lane) * 4 + 2 + kq] = lo;
            }
        }
}

cudaError_t launch_tcws(const FusedTCArgs &ta, int nsnap, cudaStream_t st)
{
    if (ta.KS <= 0 || !ta.bvar || !ta.afrag_ws) return cudaErrorInvalidValue;
    return ta.f.plane_mean ? launch_ws<8, true>(ta, nsnap, st) : launch_ws<8, false>(ta, nsnap, st);
}

}  // namespace eles
