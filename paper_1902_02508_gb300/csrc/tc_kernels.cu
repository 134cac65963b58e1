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
    // no bulk copy may outlive the CTA: the last stages issued (a wait that
    // ran out above may have left one landing)
    if (tid == 0)
        for (int k = nts > TSTG ? nts - TSTG : 0; k < nts; k++) mbar_wait(&full[k % TSTG], (k / TSTG) & 1, a.err);
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
// A[g+8][2t+8..2t+9] with A[m][k] = w[16 kk + k - RZ m - zoff], split into
// hi and lo bf16 pairs.  Returns KS (0 if the z operator does not qualify).
int tc_zfrags(const Ring &rz, int nlz, std::vector<unsigned> &out, int *zoff_out)
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
                    const double v = w(16 * kk + k - RZ * rows[r] - zoff);
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

}  // namespace eles
