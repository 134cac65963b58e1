// Wall-normal contraction and recovery on the tensor cores (EF_PREC_BF16X3).
//
// Same quantities as the y passes of ypass_kernels.cu (the recovery of
// ~bar(u_a) and T_ab of Eq. 6 about the reference profile U(y)); here the
// banded y operators are contractions on the tensor cores:
//   out[J][p] = sum_j A[J][j] h_f[j][p],   M = LES rows J, K = DNS rows j,
//                                          N = (Z, X) points p.
// The cross bracket C_ab - A_y U_a q_b of the recovery cancels two terms of
// size U q, too large for split BF16 (U ~ 20 u_tau).  It is contracted in
// deviation form instead,
//   C'_ab(J) = sum_j A^{p_a p_b}[J][j] (U_a(j) - Ubar_a(J)) h_b(j),
//   C_ab - Ubar_a q_b = C'_ab + [p_a odd] Ubar_a d_b,
//   d_b = (A^{-p_b} - A^{p_b}) h_b   (nonzero only where the filter meets
//                                     the wall), Ubar_a = A^{p_a} U_a,
// an identity of the sums.  Nine operators per snapshot: 0 A_y^+, 1 A_y^-,
// 2 A_y^- - A_y^+, 3 + 2a + p: A_y^p (U_a(j) - Ubar_a(J)).  An LES row
// tile of 16 rows only meets its band [jb, jb + 16 ks) of DNS rows, so a tile
// runs ks k-steps of 16 rows.  Operands are split as in the x-z kernels
// (x = hi + lo, BF16 round to nearest; A B ~ Ahi Bhi + Alo Bhi + Ahi Blo,
// FP32 accumulation); the operator fragments are built once per snapshot
// from the FP64 operators.
//
// One CTA per (32-point tile, snapshot, field) stages the field's h column
// over the band rows with TMA (rows padded to 36 floats, which makes the B
// fragment loads conflict-free).  Launches: fragments; all nine fields in
// one launch (the velocities: q_a, d_a and C'_ab to the scratch, ~bar(u_a)
// out; the products: q_ab to the scratch); the recovery of T_ab
// (elementwise).
#include <cuda_bf16.h>

#include "eles_internal.h"
#include "fused_stage.cuh"

namespace eles {
namespace {

using namespace fz;

constexpr int YTW = 4;      // warps per CTA
constexpr int YTP = 32;     // points per tile
constexpr int YTS = 36;     // shared row stride (floats): 2t * 36 = 8t (mod 32 banks)

__device__ __forceinline__ unsigned pack2(float lo_k, float hi_k)
{
    unsigned d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi_k), "f"(lo_k));
    return d;
}

// x = hi + lo for the pair (x0: lower k, x1: upper k).
__device__ __forceinline__ void split_b(float x0, float x1, unsigned &hi, unsigned &lo)
{
    hi = pack2(x0, x1);
    const float2 h = make_float2(__uint_as_float(hi << 16), __uint_as_float(hi & 0xffff0000u));
    const float2 l = __ffma2_rn(h, make_float2(-1.f, -1.f), make_float2(x0, x1));
    lo = pack2(l.x, l.y);
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint4 &a, unsigned b0, unsigned b1)
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void tma_load2(void *dst, const CUtensorMap *map, unsigned long long *bar, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n"
                 ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
                 : "memory");
}

// Parity index (0 even, 1 odd) of the product of components a and b.
__host__ __device__ constexpr int pprod(int a, int b) { return ((a == 1) != (b == 1)) ? 1 : 0; }

// Operator fragments: block (k-step kg of all tiles, operator op, snapshot s;
// the operators 0-2 for snapshot 0 only),
// lane (g, t) holds A[g][2t..2t+1], A[g+8][2t..2t+1], A[g][2t+8..2t+9],
// A[g+8][2t+8..2t+9] of the tile's k-step, A[m][k] = op(J = 16 mt + m,
// j = jb + 16 kk + k), the operators numbered as above.
__global__ void yfrag_kernel(const YTcGeom g, const double *__restrict__ we, const double *__restrict__ wo,
                             const double *__restrict__ uref, const double *__restrict__ AU, int ny, int nly,
                             uint4 *frag)
{
    const int kg = blockIdx.x, op = blockIdx.y, s = blockIdx.z, lane = threadIdx.x;
    if (op < 3 && s > 0) return;   // A_y^+, A_y^-, A_y^- - A_y^+ do not depend on U: snapshot 0's serve all
    int mt = 0;
    while (mt + 1 < g.nmt && g.koff[mt + 1] <= kg) mt++;
    const int kk = kg - g.koff[mt];
    const int par = op < 2 ? op : (op - 3) & 1, c = op < 3 ? -1 : (op - 3) >> 1;
    const double *W = par ? wo : we;
    const double *U = uref + ((size_t)s * 3 + (c < 0 ? 0 : c)) * ny;
    const double *Ub = AU + ((size_t)s * 3 + (c < 0 ? 0 : c)) * nly;
    const int gg = lane >> 2, t = lane & 3;
    const int rows[4] = {gg, gg + 8, gg, gg + 8}, kofs[4] = {0, 0, 8, 8};
    unsigned hi[4], lo[4];
    for (int r = 0; r < 4; r++) {
        hi[r] = lo[r] = 0;
        for (int e = 0; e < 2; e++) {
            const int J = 16 * mt + rows[r], j = g.jb[mt] + 16 * kk + 2 * t + kofs[r] + e;
            double v = 0.0;
            if (J < nly && j < ny) {
                if (op == 2) v = wo[(size_t)J * ny + j] - we[(size_t)J * ny + j];
                else v = W[(size_t)J * ny + j];
                if (c >= 0) v *= U[j] - Ub[J];
            }
            const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
            const __nv_bfloat16 l = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
            hi[r] |= (unsigned)__bfloat16_as_ushort(h) << (16 * e);
            lo[r] |= (unsigned)__bfloat16_as_ushort(l) << (16 * e);
        }
    }
    uint4 *o = frag + (((size_t)s * kYOps + op) * g.kstot + kg) * 64;
    o[lane] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    o[32 + lane] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}

// Warp units of one field's column (the h words split in place in hw):
// (LES row tile, operator, NG column tiles of 8 points); a unit streams its
// k-steps with the next k-step's operator fragment loaded ahead.  NOPS 5, a
// velocity (q_F with A_y^{p_F}, d_F, and C'_cF for c = 1..3); NOPS 1, a
// product (q only).  Returns whether a non-finite ~bar(u) was written.
template <int NOPS, int NG>
__device__ __forceinline__ bool ytc_units(const YTcArgs &a, const unsigned *hw, int tile, int s, int F, int warp,
                                          int lane)
{
    const YTcGeom &geo = a.geo;
    const int g = lane >> 2, t = lane & 3;
    const int nplane = a.nplane;
    const size_t nl = (size_t)a.nly * nplane;
    constexpr int NGRP = 4 / NG;                   // column groups per 32-point tile
    bool bad = false;
    for (int unit = warp; unit < geo.nmt * NOPS * NGRP; unit += YTW) {
        const int mt = unit / (NOPS * NGRP), rem = unit - mt * NOPS * NGRP;
        const int o = rem / NGRP, n0 = NG * (rem - o * NGRP);
        float acc[NG][4];
#pragma unroll
        for (int n = 0; n < NG; n++)
#pragma unroll
            for (int i = 0; i < 4; i++) acc[n][i] = 0.f;
        const unsigned *bw = hw + g + 8 * n0 + (size_t)(geo.jb[mt] + 2 * t) * YTS;
        // operator: velocities q (A_y^{p_F}, Eq. 7 (+,-,+) or Eq. 9 (-,+,-)), d, C'_cF;
        // products q (12 and 23 odd)
        const int opo = NOPS == 5 ? (o == 0 ? ((F == 1) != (a.flip != 0) ? 1 : 0)
                                   : o == 1 ? 2 : 3 + 2 * (o - 2) + pprod(o - 2, F))
                                  : ((F == 4 || F == 7) ? 1 : 0);
        const size_t sf = opo < 3 ? 0 : s;            // the U-free operators are built for snapshot 0 only
        const uint4 *fo = a.frag + ((sf * kYOps + opo) * geo.kstot + geo.koff[mt]) * 64 + lane;
        uint4 ah = __ldg(fo), al = __ldg(fo + 32);
        // the wall term d of a row tile that never meets a wall is zero: no MMAs
        const int ks = NOPS == 5 && o == 1 && geo.dzero[mt] ? 0 : geo.ks[mt];
        for (int kk = 0; kk < ks; kk++) {
            uint4 nah = ah, nal = al;
            if (kk + 1 < ks) {
                nah = __ldg(fo + 64 * (kk + 1));
                nal = __ldg(fo + 64 * (kk + 1) + 32);
            }
            const unsigned *x = bw + (size_t)16 * kk * YTS;
            unsigned b0h[NG], b0l[NG], b1h[NG], b1l[NG];
#pragma unroll
            for (int n = 0; n < NG; n++) {
                b0h[n] = x[8 * n];                                                 // rows 2t, 2t + 1
                b0l[n] = x[YTS + 8 * n];
                b1h[n] = x[8 * YTS + 8 * n];                                       // rows 2t + 8, 2t + 9
                b1l[n] = x[9 * YTS + 8 * n];
            }
            // the three split products of one accumulator depend on each other:
            // issue them NG apart (the order within an accumulator is unchanged)
#pragma unroll
            for (int n = 0; n < NG; n++) mma16816(acc[n], ah, b0h[n], b1h[n]);
#pragma unroll
            for (int n = 0; n < NG; n++) mma16816(acc[n], al, b0h[n], b1h[n]);
#pragma unroll
            for (int n = 0; n < NG; n++) mma16816(acc[n], ah, b0l[n], b1l[n]);
            ah = nah;
            al = nal;
        }
        // lane (g, t) holds rows 16 mt + g (+8) and points 8n + 2t (+1) of the tile
#pragma unroll
        for (int hr = 0; hr < 2; hr++) {
            const int J = 16 * mt + g + 8 * hr;
            if (J >= a.nly) continue;
            const size_t o0 = (size_t)J * nplane;
#pragma unroll
            for (int n = 0; n < NG; n++)
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    const int p = tile * YTP + 8 * (n0 + n) + 2 * t + e;
                    if (p >= nplane) continue;
                    float *tmp = a.tmp + (size_t)s * kYTmp * nl + o0 + p;
                    const float v = acc[n][2 * hr + e];
                    if (!in_range((size_t)s * kYTmp * nl + o0 + p + (size_t)(kYTmp - 1) * nl, (size_t)a.nsnap * kYTmp * nl,
                                  a.err))
                        continue;
                    if constexpr (NOPS == 5) {
                        if (o == 0) {
                            const float ub = (float)a.AU[((size_t)s * 3 + F) * a.nly + J] + v;
                            bad |= !isfinite(ub);
                            const int po = a.ptrans ? (p % a.nlz) * a.nlx + p / a.nlz : p;
                            if (in_range(((size_t)s * 3 + F) * nl + o0 + po, (size_t)a.nsnap * 3 * nl, a.err))
                                a.ubar[((size_t)s * 3 + F) * nl + o0 + po] = ub;
                        }
                        if (a.stress) {
                            const int slot = o == 0 ? F : o == 1 ? 12 + F : 3 + 3 * (o - 2) + F;
                            tmp[(size_t)slot * nl] = v;
                        }
                    } else {
                        tmp[(size_t)(15 + F - 3) * nl] = v;
                    }
                }
        }
    }
    return bad;
}

// One field per CTA (blockIdx.z = F: the velocities 0-2, the products 3-8
// when the stress is wanted; one launch, the velocity CTAs first so that the
// lighter product CTAs fill the tail).  After the TMA load the CTA splits its
// h column once, in place: the fp32 pair of rows (2r, 2r + 1) at a point
// becomes the two B fragment words (hi in row 2r's slot, lo in row 2r + 1's).
__global__ void __launch_bounds__(YTW * 32, 5) ytc_kernel(const __grid_constant__ YTcArgs a)
{
    extern __shared__ float4 ysm4[];
    float *hs;                                     // [2 box_rows][YTS], 128-B aligned for TMA
    {
        char *b = reinterpret_cast<char *>(ysm4);
        const unsigned sa = smem_u32(b);
        hs = reinterpret_cast<float *>(b + (((sa + 127u) & ~127u) - sa));
    }
    __shared__ alignas(8) unsigned long long bar;
    const YTcGeom &geo = a.geo;
    const int tile = blockIdx.x, s = blockIdx.y, F = blockIdx.z;
    const int rows = 2 * geo.box_rows;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bar, 2u * geo.box_rows * YTS * 4u);
        const int row0 = (s * 9 + F) * a.ny;
        for (int hf = 0; hf < 2; hf++)
            tma_load2(hs + (size_t)hf * geo.box_rows * YTS, &a.hmap, &bar, tile * YTP, row0 + hf * geo.box_rows);
    }
    const bool landed = mbar_wait(&bar, 0, a.err);
    if (__syncthreads_or(!landed)) {
        // the wait ran out (EF_ERR_TIMEOUT is recorded) and the copy may still
        // be landing: skip the column and wait once more, with the same bound,
        // so that no bulk copy outlives the CTA
        mbar_wait(&bar, 0, nullptr);
        return;
    }
    // split the column once: (rows 2r, 2r + 1) -> (hi word, lo word)
    unsigned *hw = reinterpret_cast<unsigned *>(hs);
    for (int i = threadIdx.x; i < (rows / 2) * YTP; i += YTW * 32) {
        const int r2 = i / YTP, pc = i - r2 * YTP;
        unsigned hi, lo;
        split_b(hs[(2 * r2) * YTS + pc], hs[(2 * r2 + 1) * YTS + pc], hi, lo);
        hw[(2 * r2) * YTS + pc] = hi;
        hw[(2 * r2 + 1) * YTS + pc] = lo;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool bad = F < 3 ? ytc_units<5, 4>(a, hw, tile, s, F, warp, lane)
                           : ytc_units<1, 2>(a, hw, tile, s, F, warp, lane);
    if (bad && a.err) atomicCAS(a.err, 0, (int)EF_ERR_NAN);
}

// T_ab = [A_y(U_a U_b) - A_y U_a A_y U_b] + [C_ab - A_y U_a q_b]
//      + [C_ba - A_y U_b q_a] + [q_ab - q_a q_b], with
// C_ab - A_y U_a q_b = C'_ab + [p_a odd] A_y U_a d_b.  The first bracket,
// the only one that cancels large terms, comes formed in FP64 per row (Kab);
// the rest are O(1) and are summed in FP32.
// The six T_ab of snapshot s, LES row J, plane point r (in h's plane order).
__device__ __forceinline__ bool recover_point(const YTcArgs &a, int s, int J, size_t r, float (&out)[6])
{
    const size_t nl = (size_t)a.nly * a.nplane;
    const float *tmp = a.tmp + (size_t)s * kYTmp * nl + (size_t)J * a.nplane + r;
    const double *AU = a.AU + (size_t)s * 3 * a.nly;
    const float *K = a.Kab + (size_t)s * 6 * a.nly;
    const int PI[6] = {0, 0, 0, 1, 1, 2}, PJ[6] = {0, 1, 2, 1, 2, 2};
    float qv[3], dU[3][3];   // dU[a][b] = [p_a odd] A_y U_a d_b
#pragma unroll
    for (int c = 0; c < 3; c++) qv[c] = tmp[(size_t)c * nl];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const bool odd = (c == 1) != (a.flip != 0);
        // the scratch holds (A^- - A^+) h_c; d_c = (A^{-p_c} - A^{p_c}) h_c
        const float dc = (odd ? -1.f : 1.f) * tmp[(size_t)(12 + c) * nl];
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const bool oddb = (b == 1) != (a.flip != 0);
            dU[b][c] = oddb ? (float)AU[b * a.nly + J] * dc : 0.f;
        }
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const int ia = PI[k], m = PJ[k];
        const float Bim = tmp[(size_t)(3 + 3 * ia + m) * nl] + dU[ia][m];
        const float Bmi = tmp[(size_t)(3 + 3 * m + ia) * nl] + dU[m][ia];
        out[k] = K[k * a.nly + J] + (Bim + Bmi) + fmaf(-qv[ia], qv[m], tmp[(size_t)(15 + k) * nl]);
        bad |= !isfinite(out[k]);
    }
    return bad;
}

// T_ab = [A_y(U_a U_b) - A_y U_a A_y U_b] + [C_ab - A_y U_a q_b]
//      + [C_ba - A_y U_b q_a] + [q_ab - q_a q_b], with
// C_ab - A_y U_a q_b = C'_ab + [p_a odd] A_y U_a d_b.  The first bracket,
// the only one that cancels large terms, comes formed in FP64 per row (Kab);
// the rest are O(1) and are summed in FP32.
__global__ void yrecover_kernel(const __grid_constant__ YTcArgs a, int nsnap)
{
    const size_t nl = (size_t)a.nly * a.nplane;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl * nsnap) return;
    const int s = (int)(i / nl);
    const size_t r = i - (size_t)s * nl;
    const int J = (int)(r / a.nplane);
    float out[6];
    const bool bad = recover_point(a, s, J, r - (size_t)J * a.nplane, out);
#pragma unroll
    for (int k = 0; k < 6; k++)
        if (in_range(((size_t)s * 6 + k) * nl + r, (size_t)nsnap * 6 * nl, a.err)) a.tau[((size_t)s * 6 + k) * nl + r] = out[k];
    if (bad && a.err) atomicCAS(a.err, 0, (int)EF_ERR_NAN);
}

// The same for h planes in (X, Z) order: a 16 x 16 tile of (X, Z) points per
// block, read along Z and written along X through shared memory.
__global__ void __launch_bounds__(256) yrecover_t_kernel(const __grid_constant__ YTcArgs a)
{
    __shared__ float tile[6][16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int X0 = 16 * blockIdx.x, Z0 = 16 * blockIdx.y;
    const int J = blockIdx.z % a.nly, s = blockIdx.z / a.nly;
    const size_t nl = (size_t)a.nly * a.nplane;
    bool bad = false;
    {   // read: thread (ty, tx) takes X = X0 + ty, Z = Z0 + tx
        const int X = X0 + ty, Z = Z0 + tx;
        if (X < a.nlx && Z < a.nlz) {
            float out[6];
            bad = recover_point(a, s, J, (size_t)X * a.nlz + Z, out);
#pragma unroll
            for (int k = 0; k < 6; k++) tile[k][tx][ty] = out[k];
        }
    }
    __syncthreads();
    {   // write: thread (ty, tx) takes Z = Z0 + ty, X = X0 + tx
        const int Z = Z0 + ty, X = X0 + tx;
        if (X < a.nlx && Z < a.nlz) {
#pragma unroll
            for (int k = 0; k < 6; k++) {
                const size_t o = ((size_t)s * 6 + k) * nl + (size_t)J * a.nplane + (size_t)Z * a.nlx + X;
                if (in_range(o, (size_t)a.nsnap * 6 * nl, a.err)) a.tau[o] = tile[k][ty][tx];
            }
        }
    }
    if (bad && a.err) atomicCAS(a.err, 0, (int)EF_ERR_NAN);
}

cudaError_t launch_fields(const YTcArgs &a, int nsnap, int nfields, cudaStream_t st)
{
    const size_t smem = sizeof(float) * 2 * (size_t)a.geo.box_rows * YTS + 128;
    static size_t attr = 0;
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(ytc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    ytc_kernel<<<dim3((a.nplane + YTP - 1) / YTP, nsnap, nfields), YTW * 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Banded tiling of the y operators: tile mt of 16 LES rows meets DNS rows
// [jb, jb + 16 ks); two TMA boxes of box_rows rows stage them all.  False if
// the plan does not fit (rows > 512, a row stride of h that TMA cannot take,
// or the staging beyond one CTA's shared memory).
bool ytc_geometry(const std::vector<int> &ystart, const std::vector<int> &ycount, int ny, int nplane, YTcGeom *g)
{
    const int nly = (int)ycount.size();
    const int nmt = (nly + 15) / 16;
    if (nmt > kYMaxTiles || nplane % 4 != 0) return false;
    g->nmt = nmt;
    int kstot = 0, top = 0;
    for (int mt = 0; mt < nmt; mt++) {
        int lo = ny, hi = 0;
        for (int J = 16 * mt; J < 16 * mt + 16 && J < nly; J++) {
            lo = ystart[J] < lo ? ystart[J] : lo;
            hi = ystart[J] + ycount[J] > hi ? ystart[J] + ycount[J] : hi;
        }
        if (hi <= lo) lo = hi = 0;
        lo &= ~1;                 // even: the split words pair rows (2r, 2r + 1)
        g->jb[mt] = lo;
        g->ks[mt] = (hi - lo + 15) / 16;
        g->koff[mt] = kstot;
        kstot += g->ks[mt];
        top = lo + 16 * g->ks[mt] > top ? lo + 16 * g->ks[mt] : top;
    }
    g->kstot = kstot;
    // a TMA box must land on a 128-byte boundary: box_rows x 144 bytes is a
    // multiple of 128 when box_rows is a multiple of 8
    g->box_rows = ((top + 1) / 2 + 7) / 8 * 8;
    (void)ny;
    return g->box_rows <= 256 && sizeof(float) * 2 * (size_t)g->box_rows * YTS + 128 <= 227 * 1024;
}

cudaError_t launch_yfrag(const YTcGeom &g, const double *yw_even, const double *yw_odd, const double *uref,
                         const double *AU, int ny, int nly, int nsnap, uint4 *frag, cudaStream_t st)
{
    yfrag_kernel<<<dim3(g.kstot, kYOps, nsnap), 32, 0, st>>>(g, yw_even, yw_odd, uref, AU, ny, nly, frag);
    return cudaGetLastError();
}

// TMA view of h [S][9][ny][nplane] as a 2-D tensor {nplane, 9 ny S}, boxes of
// 36 points (a 32-point tile and 4 of padding) x box_rows rows.
int encode_h_map(const float *h, int nplane, int ny, int nsnap, int box_rows, CUtensorMap *map)
{
    typedef CUresult (*encode_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static encode_fn fn = nullptr;
    if (!fn) {
        void *q = nullptr;
        cudaDriverEntryPointQueryResult r;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault, &r) != cudaSuccess ||
            r != cudaDriverEntryPointSuccess || !q) {
            set_error("cuTensorMapEncodeTiled unavailable");
            return EF_ERR_CUDA;
        }
        fn = reinterpret_cast<encode_fn>(q);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)nplane, (cuuint64_t)9 * ny * nsnap};
    const cuuint64_t strides[1] = {(cuuint64_t)nplane * 4};
    const cuuint32_t box[2] = {(cuuint32_t)YTS, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(h), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled (h) failed (%d)", (int)r);
        return EF_ERR_CUDA;
    }
    return EF_OK;
}

cudaError_t launch_ytc(const YTcArgs &a, int nsnap, cudaStream_t st)
{
    YTcArgs c = a;
    c.nsnap = nsnap;
    cudaError_t e = launch_fields(c, nsnap, a.stress ? 9 : 3, st);
    if (e != cudaSuccess || !a.stress) return e;
    YTcArgs b = a;
    b.nsnap = nsnap;
    if (a.ptrans) {
        yrecover_t_kernel<<<dim3((a.nlx + 15) / 16, (a.nlz + 15) / 16, a.nly * nsnap), 256, 0, st>>>(b);
    } else {
        const size_t n = (size_t)a.nly * a.nplane * nsnap;
        yrecover_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(b, nsnap);
    }
    return cudaGetLastError();
}

}  // namespace eles
