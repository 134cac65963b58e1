// Warp-specialised x-z kernel on the tensor cores (x_variant 3), for the
// split-precision plans: EF_PREC_BF16X3 and EF_PREC_TF32X2.
//
// A persistent grid (as many CTAs as fit at once) walks the items (snapshot,
// y-plane, output phase); in each CTA three roles meet only at mbarriers
// (every wait bounded), and the producer streams the next item while the
// other roles finish the current one:
//   * NZ / 32 x warps (32 z-rows each) contract x with mma.sync on the tensor
//     cores, FP32 accumulation;
//   * one producer warp streams the plane through TMA stages of one chunk
//     (16 x-inputs of every row, three components) with a full and an empty
//     barrier per stage;
//   * ZW z warps contract z (split BF16, tensor cores) for the outputs each
//     chunk completes, from a double-buffered column buffer.  (An FP32 z
//     phase on the CUDA cores was measured 2.4 times slower: the z warps are
//     few, and a 63-tap FP32 dot product per output outweighs the banded MMAs.)
//
// The x contraction is a strided convolution: output X (at DNS column rx X)
// takes inputs x with |x - rx X| <= R.  A chunk feeds the outputs in flight,
// held as the 8 columns of the MMA accumulator tile (rows = z-rows).  When the
// band is wide (ring depth D above what 7 columns hold), the outputs are split
// into OP phases X = OP m + p, one CTA per phase, each re-reading the plane
// (from L2: the phases of a plane run side by side).  Every chunk completes
// OPC = 16 / (rx OP) outputs of a phase (1 or 2).  Phase output m lives in
// tile column (m - m0) mod 8 for the whole stream, so the chunk's B operand
// rotates (NR = 8 / OPC rotations, built on the host) and the outputs a
// chunk completes always sit in columns OPC q .. OPC q + OPC - 1 (q = chunk
// mod NR).  The column after the window (OPC q + 7) is idle: its B column is
// all ones and collects the chunk's row sums of the fluctuation (plane means).
//
// Fields: u'_c = u_c - U_c(y) (U_c the mean of the plane's z-row 0) and the
// six products u'_a u'_b, formed in registers.
//   Velocities, BF16X3: x = hi + lo (bf16 pair), weights likewise; the
//           products Ahi Bhi + Alo Bhi + Ahi Blo (m16n8k16).
//   Velocities, TF32X2: hi = x with its 13 low bits cleared (TF32), lo = x -
//           hi (exact; no conversion instruction), against TF32 hi + lo
//           weights: Ahi Bhi + Alo Bhi + Ahi Blo (m16n8k8).
//   Products, both forms: rounded once to an 11-bit significand (the FP16
//           format, TF32's precision: one conversion per pair of values)
//           and contracted against FP16 hi + lo weights: A Bhi + A Blo
//           (m16n8k16).  Exact range for |u'_a u'_b| < 65504; values below
//           2^-14 are kept to 2^-25 absolute as subnormals.
// The z contraction takes the parked x results the same way: the velocity
// columns as bf16 (hi, lo) pairs against bf16 hi + lo weights (three
// products), the product columns rounded once to FP16 against FP16 hi + lo
// weights (two products).
#pragma once

#include "eles_internal.h"
#include "fused_stage.cuh"

namespace eles {
namespace ws {

using namespace fz;

constexpr int CW = 16;               // floats per row per TMA stage: one chunk
constexpr int CSTG = 2;              // stages in flight
enum { MODE_BF16X3 = 0, MODE_TF32X2 = 1 };

// B words per lane and rotation: the velocities' set (one uint4 of bf16 hi,
// lo words for BF16X3; two TF32 k-halves for TF32X2), then the products'
// FP16 hi, lo words (the last uint4).
template <int MODE>
struct Bw { static constexpr int n = MODE == MODE_TF32X2 ? 3 : 2; };

// Parked columns of one buffer (floats): the velocity columns (3 per output,
// LD floats), the product columns (6 per output, LDP(LD) words) and the three
// row-sum columns (LD).  Per 16-row block, pair i < 8 stands for rows
// (i, i + 8).  A velocity block is parked as 8 FP32 pairs and then split into
// bf16 words, stored as 8 uint2 slots: slot i' < 4 holds (hi of pair i', hi
// of pair i' + 4) and slot 4 + i' the two lo words, so that one 8-byte load
// is the B operand (k rows 2t, 2t + 1 and 2t + 8, 2t + 9) of one split
// product.  A product block is 8 FP16x2 words in the order pair 0, 4, 1, 5,
// 2, 6, 3, 7 (one 8-byte load per B operand likewise).  Column strides of 8
// (mod 32) words keep the z warps' 8-byte loads conflict-free.
template <int OPC>
struct Park {
    static constexpr int NV = 3 * OPC, NP = 6 * OPC;   // velocity, product columns
    static constexpr int NVT = 1, NPT = (NP + 7) / 8;  // column tiles of each kind
    __host__ __device__ static constexpr int LDP(int LD) { return LD / 2 + 4; }   // product column stride
    __host__ __device__ static constexpr size_t floats(int LD) { return (size_t)(NV + 3) * LD + (size_t)NP * LDP(LD); }
    __host__ __device__ static constexpr size_t prod0(int LD) { return (size_t)NV * LD; }
    __host__ __device__ static constexpr size_t sum0(int LD) { return (size_t)NV * LD + (size_t)NP * LDP(LD); }
};

struct WsArgs {
    CUtensorMap tmap;     // TMA view of u: {nx, nz, 3 ny S} floats, box {16, box_rows, 1}
    const float *u;       // [S][3][ny][nz][nx]
    float *h;             // [S][9][ny][nlx][nlz]: the plane in (X, Z) order, Z fastest
    const double *uref;   // [S][3][ny]: the reference profile (written by ws_uref before the launch)
    double *plane_mean;   // [S][3][ny] or nullptr
    int *err;             // device error word
    int nx, ny, nz, nlx, nlz;
    int box_rows;
    int nchunk;           // chunks per row stream
    int bshift;           // chunk k starts at x block CB k - bshift (mod nlx)
    int rx, CB;           // DNS columns per LES column, x blocks per chunk (16 / rx)
    int OP;               // output phases (CTAs per plane)
    int xc0[4];           // per phase: first output completed by chunk 0 (may be < 0)
    int RZ, KS, zoff;     // z phase: stride, k-steps per Z tile, window offset
    int nf;               // fields contracted in z (9, or 3 for the velocities only)
    int nsnap;            // snapshots (items are (snapshot, y-plane, phase))
    long long wait_limit; // bound of one wait in SM clocks (kWaitCycles unless set for tests)
    const uint4 *afrag;   // z A fragments [KS][bf16 hi, bf16 lo, f16 hi, f16 lo][32 lanes] (pair order)
    const uint4 *bvar;    // x B fragments [OP][NR][32 lanes][Bw]
};

// One launch over the items of up to kWsMaxPlans plans of one kernel class
// (nz, precision, outputs per chunk): CTAs cta0[i] .. cta0[i + 1] - 1 walk
// plan i's items (a multiple of its OP), so each CTA loads its plan's
// tables once.  Plans of different grids and filter widths share the launch.
constexpr int kWsMaxPlans = 16;
struct WsMulti {
    WsArgs plan[kWsMaxPlans];
    int nplan;
    int cta0[kWsMaxPlans + 1];
};

__device__ __forceinline__ unsigned pack_f16(float lo_k, float hi_k)
{
    unsigned d;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi_k), "f"(lo_k));
    return d;
}

__device__ __forceinline__ void mma_f16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                        unsigned b0, unsigned b1)
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_bf16(float lo_k, float hi_k)
{
    unsigned d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi_k), "f"(lo_k));
    return d;
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1)
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1)
{
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// x = hi + lo for a pair (k, k+1), bf16 words, with a packed FP32 subtraction.
__device__ __forceinline__ void split2(float2 x, unsigned &hi, unsigned &lo)
{
    hi = pack_bf16(x.x, x.y);
    const float2 h = make_float2(__uint_as_float(hi << 16), __uint_as_float(hi & 0xffff0000u));
    const float2 l = __ffma2_rn(h, make_float2(-1.f, -1.f), x);
    lo = pack_bf16(l.x, l.y);
}

__device__ __forceinline__ unsigned pack_f16_2(float2 x) { return pack_f16(x.x, x.y); }

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

// order 0 3 4 5 | 1 6 7 | 2 8: each component's registers die as early as possible
template <int F>
__host__ __device__ constexpr int next_field()
{
    return F == 0 ? 3 : F == 3 ? 4 : F == 4 ? 5 : F == 5 ? 1 : F == 1 ? 6 : F == 6 ? 7 : F == 7 ? 2 : F == 2 ? 8 : -1;
}

// One 16-row tile, all fields, one chunk.  v[c][h][k2] holds component c at
// row g + 8h and chunk inputs 4t + 2k2 (.x) and 4t + 2k2 + 1 (.y).
//   BF16X3 k slots: 2t + 8 k2 + e <-> input 4t + 2 k2 + e.
//   TF32X2, MMA k2: slot t <-> input 4t + 2 k2, slot t + 4 <-> 4t + 2 k2 + 1.
template <int MODE, int F>
__device__ __forceinline__ void x_mma(float (&acc)[NF][4], const float2 (&v)[3][2][2], const uint4 (&B)[Bw<MODE>::n])
{
    if constexpr (F >= 3) {
        // products: one rounding to an 11-bit significand (FP16); k slots as the BF16 velocities
        constexpr int FB = Bw<MODE>::n - 1;
        const unsigned a0 = pack_f16_2(field2<F>(v[0][0][0], v[1][0][0], v[2][0][0]));   // row g,     k 2t, 2t+1
        const unsigned a1 = pack_f16_2(field2<F>(v[0][1][0], v[1][1][0], v[2][1][0]));   // row g + 8, k 2t, 2t+1
        const unsigned a2 = pack_f16_2(field2<F>(v[0][0][1], v[1][0][1], v[2][0][1]));   // row g,     k 2t+8, 2t+9
        const unsigned a3 = pack_f16_2(field2<F>(v[0][1][1], v[1][1][1], v[2][1][1]));   // row g + 8, k 2t+8, 2t+9
        mma_f16(acc[F], a0, a1, a2, a3, B[FB].z, B[FB].w);
        mma_f16(acc[F], a0, a1, a2, a3, B[FB].x, B[FB].y);
    } else if constexpr (MODE == MODE_BF16X3) {
        unsigned ah[4], al[4];
        split2(field2<F>(v[0][0][0], v[1][0][0], v[2][0][0]), ah[0], al[0]);   // row g,     k 2t, 2t+1
        split2(field2<F>(v[0][1][0], v[1][1][0], v[2][1][0]), ah[1], al[1]);   // row g + 8, k 2t, 2t+1
        split2(field2<F>(v[0][0][1], v[1][0][1], v[2][0][1]), ah[2], al[2]);   // row g,     k 2t+8, 2t+9
        split2(field2<F>(v[0][1][1], v[1][1][1], v[2][1][1]), ah[3], al[3]);   // row g + 8, k 2t+8, 2t+9
        mma_bf16(acc[F], ah[0], ah[1], ah[2], ah[3], B[0].x, B[0].y);
        mma_bf16(acc[F], al[0], al[1], al[2], al[3], B[0].x, B[0].y);
        mma_bf16(acc[F], ah[0], ah[1], ah[2], ah[3], B[0].z, B[0].w);
    } else {
#pragma unroll
        for (int k2 = 0; k2 < 2; k2++) {
            const float2 x0 = v[F][0][k2], x1 = v[F][1][k2];     // rows g, g + 8
            const uint4 b = B[k2];           // b0 hi, b1 hi, b0 lo, b1 lo
            const unsigned h00 = __float_as_uint(x0.x) & 0xffffe000u, h01 = __float_as_uint(x0.y) & 0xffffe000u;
            const unsigned h10 = __float_as_uint(x1.x) & 0xffffe000u, h11 = __float_as_uint(x1.y) & 0xffffe000u;
            const float2 m1 = make_float2(-1.f, -1.f);
            const float2 l0 = __ffma2_rn(make_float2(__uint_as_float(h00), __uint_as_float(h01)), m1, x0);
            const float2 l1 = __ffma2_rn(make_float2(__uint_as_float(h10), __uint_as_float(h11)), m1, x1);
            mma_tf32(acc[F], h00, h10, h01, h11, b.x, b.y);
            mma_tf32(acc[F], __float_as_uint(l0.x), __float_as_uint(l1.x), __float_as_uint(l0.y),
                     __float_as_uint(l1.y), b.x, b.y);
            mma_tf32(acc[F], h00, h10, h01, h11, b.z, b.w);
        }
    }
    constexpr int nx = next_field<F>();
    if constexpr (nx >= 0) x_mma<MODE, nx>(acc, v, B);
}

// BF16X3 x contraction with the MMAs of two fields interleaved, so that the
// dependent MMAs of one accumulator are issued apart.  The x warps take the
// pairs (u'1, u'1u'1), (u'2, u'1u'2), (u'3, u'2u'2), (u'2u'3, u'3u'3), then
// u'1u'3 with u'1 reloaded, so that at most two velocity components are live
// (the x-warp loop issues them).
template <int F>
__device__ __forceinline__ void vel_split(const float2 (&v)[3][2][2], unsigned (&ah)[4], unsigned (&al)[4])
{
    split2(field2<F>(v[0][0][0], v[1][0][0], v[2][0][0]), ah[0], al[0]);
    split2(field2<F>(v[0][1][0], v[1][1][0], v[2][1][0]), ah[1], al[1]);
    split2(field2<F>(v[0][0][1], v[1][0][1], v[2][0][1]), ah[2], al[2]);
    split2(field2<F>(v[0][1][1], v[1][1][1], v[2][1][1]), ah[3], al[3]);
}
template <int F>
__device__ __forceinline__ void prod_pack(const float2 (&v)[3][2][2], unsigned (&a)[4])
{
    a[0] = pack_f16_2(field2<F>(v[0][0][0], v[1][0][0], v[2][0][0]));
    a[1] = pack_f16_2(field2<F>(v[0][1][0], v[1][1][0], v[2][1][0]));
    a[2] = pack_f16_2(field2<F>(v[0][0][1], v[1][0][1], v[2][0][1]));
    a[3] = pack_f16_2(field2<F>(v[0][1][1], v[1][1][1], v[2][1][1]));
}
template <int FV, int FP>
__device__ __forceinline__ void vp_pair(float (&acc)[NF][4], const float2 (&v)[3][2][2], const uint4 &bv, const uint4 &bp)
{
    unsigned ah[4], al[4], a[4];
    vel_split<FV>(v, ah, al);
    prod_pack<FP>(v, a);
    mma_bf16(acc[FV], ah[0], ah[1], ah[2], ah[3], bv.x, bv.y);
    mma_f16(acc[FP], a[0], a[1], a[2], a[3], bp.z, bp.w);
    mma_bf16(acc[FV], al[0], al[1], al[2], al[3], bv.x, bv.y);
    mma_f16(acc[FP], a[0], a[1], a[2], a[3], bp.x, bp.y);
    mma_bf16(acc[FV], ah[0], ah[1], ah[2], ah[3], bv.z, bv.w);
}
template <int F1, int F2>
__device__ __forceinline__ void pp_pair(float (&acc)[NF][4], const float2 (&v)[3][2][2], const uint4 &bp)
{
    unsigned a[4], b[4];
    prod_pack<F1>(v, a);
    prod_pack<F2>(v, b);
    mma_f16(acc[F1], a[0], a[1], a[2], a[3], bp.z, bp.w);
    mma_f16(acc[F2], b[0], b[1], b[2], b[3], bp.z, bp.w);
    mma_f16(acc[F1], a[0], a[1], a[2], a[3], bp.x, bp.y);
    mma_f16(acc[F2], b[0], b[1], b[2], b[3], bp.x, bp.y);
}

// TF32X2 x contraction with the first k-half of each velocity field
// interleaved with the MMAs of a product field: (u'1, u'1u'1), (u'1u'2, u'1u'3),
// (u'2, u'2u'2), (u'3, u'2u'3), u'3u'3 (all three components loaded).
template <int FV>
__device__ __forceinline__ void tf32_half(const float2 (&v)[3][2][2], int k2, unsigned (&h)[4], unsigned (&l)[4])
{
    const float2 x0 = v[FV][0][k2], x1 = v[FV][1][k2];     // rows g, g + 8
    h[0] = __float_as_uint(x0.x) & 0xffffe000u; h[2] = __float_as_uint(x0.y) & 0xffffe000u;
    h[1] = __float_as_uint(x1.x) & 0xffffe000u; h[3] = __float_as_uint(x1.y) & 0xffffe000u;
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 l0 = __ffma2_rn(make_float2(__uint_as_float(h[0]), __uint_as_float(h[2])), m1, x0);
    const float2 l1 = __ffma2_rn(make_float2(__uint_as_float(h[1]), __uint_as_float(h[3])), m1, x1);
    l[0] = __float_as_uint(l0.x); l[1] = __float_as_uint(l1.x); l[2] = __float_as_uint(l0.y); l[3] = __float_as_uint(l1.y);
}
template <int FV, int FP>
__device__ __forceinline__ void vp_pair_tf32(float (&acc)[NF][4], const float2 (&v)[3][2][2], const uint4 (&B)[3])
{
    unsigned h[4], l[4], a[4];
    tf32_half<FV>(v, 0, h, l);
    prod_pack<FP>(v, a);
    mma_tf32(acc[FV], h[0], h[1], h[2], h[3], B[0].x, B[0].y);
    mma_f16(acc[FP], a[0], a[1], a[2], a[3], B[2].z, B[2].w);
    mma_tf32(acc[FV], l[0], l[1], l[2], l[3], B[0].x, B[0].y);
    mma_f16(acc[FP], a[0], a[1], a[2], a[3], B[2].x, B[2].y);
    mma_tf32(acc[FV], h[0], h[1], h[2], h[3], B[0].z, B[0].w);
    tf32_half<FV>(v, 1, h, l);
    mma_tf32(acc[FV], h[0], h[1], h[2], h[3], B[1].x, B[1].y);
    mma_tf32(acc[FV], l[0], l[1], l[2], l[3], B[1].x, B[1].y);
    mma_tf32(acc[FV], h[0], h[1], h[2], h[3], B[1].z, B[1].w);
}
__device__ __forceinline__ void x_mma_il_tf32(float (&acc)[NF][4], const float2 (&v)[3][2][2], const uint4 (&B)[3])
{
    vp_pair_tf32<0, 3>(acc, v, B);
    pp_pair<4, 5>(acc, v, B[2]);
    vp_pair_tf32<1, 6>(acc, v, B);
    vp_pair_tf32<2, 7>(acc, v, B);
    unsigned a[4];
    prod_pack<8>(v, a);
    mma_f16(acc[8], a[0], a[1], a[2], a[3], B[2].z, B[2].w);
    mma_f16(acc[8], a[0], a[1], a[2], a[3], B[2].x, B[2].y);
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait shared by the roles (at most `limit` SM clocks after a first
// non-blocking test).  Once any wait of the CTA has run out the others return
// at once and the roles stop: the producer issues no new stage and the
// consumers stop touching the stage and column buffers (a bulk copy issued
// before may still be landing; the producer waits for those, with the long
// bound, before the CTA exits).  The error word tells the host.
__device__ __forceinline__ bool wait_or_abort(unsigned long long *bar, unsigned parity, volatile int *abort_flag,
                                              int *err, long long limit)
{
    if (mbar_test_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (clock64() - t0 < limit) {
        if (*abort_flag) return false;
        if (mbar_try_wait(bar, parity)) return true;
    }
    *abort_flag = 1;
    if (err) atomicCAS(err, 0, (int)EF_ERR_TIMEOUT);
    return false;
}

// z work: Z tile zt (16 outputs) of the velocity column tile (DOV) and of
// product column tiles pt0 .. pt0 + NPTW - 1 (8 columns each; velocity
// column c = 3 n + f, product column c = 6 n + f - 3, for output X0 + OP n),
// KS k-steps over the tile's z window, each A fragment loaded once per
// k-step for all the tiles.  The k index of a k-step runs over a 16-row
// block's rows in the order k = 2i + e -> row i + 8e (pair i, element e),
// which the A fragments follow; each B operand is one 8-byte load (the slot
// order of Park).  The window starts on a 16-row boundary (zoff is a multiple
// of 16), so a k-step wraps periodically as a whole or not at all.  Lanes
// whose column is idle read column 0: an MMA's output column depends on its
// own B column only, and idle output columns are never stored.  Outputs go to
// h in (X, Z) plane order (Z fastest), so that each store instruction writes
// 4 runs of 8 consecutive floats instead of 32 scattered ones (a chunk
// completes whole Z columns of one or two X); the y passes transpose back.
template <int OPC, int LD, bool DOV, int NPTW>
__device__ __forceinline__ void z_tile(const WsArgs &a, const float *colb, const uint4 *afrag,
                                       int s, int j, int X0, bool val0, bool val1, int zt, int pt0, int lane)
{
    using PK = Park<OPC>;
    constexpr int NPA = NPTW > 0 ? NPTW : 1;
    constexpr int LDP = PK::LDP(LD);
    const int g = lane >> 2, t = lane & 3;
    const uint2 *vp = nullptr;                    // slot t of each block: +8 per 16 rows
    if constexpr (DOV) vp = reinterpret_cast<const uint2 *>(colb + (size_t)(g < PK::NV ? g : 0) * LD) + t;
    const uint2 *pp[NPA];                         // word pair t of each block: +4 per 16 rows
#pragma unroll
    for (int i = 0; i < NPTW; i++) {
        const int c = (pt0 + i) * 8 + g;
        pp[i] = reinterpret_cast<const uint2 *>(colb + PK::prod0(LD) + (size_t)(c < PK::NP ? c : 0) * LDP) + t;
    }
    float av[3][4], ap[NPA][2][4];   // one accumulator per split product: independent chains
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int e = 0; e < 4; e++) av[r][e] = 0.f;
#pragma unroll
    for (int i = 0; i < NPA; i++)
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
            for (int e = 0; e < 4; e++) ap[i][r][e] = 0.f;
    // 16-row block index of the first k-step, periodic in the nz / 16 blocks
    const int nb = a.nz >> 4;
    int blk = (16 * a.RZ * zt - a.zoff) >> 4;
    if (blk < 0) blk += nb;
    const uint4 *af = afrag + lane;
#pragma unroll 2
    for (int kk = 0; kk < a.KS; kk++, af += 128) {
        if constexpr (DOV) {
            const uint4 ah = af[0], al = af[32];
            const uint2 bh = vp[8 * blk], bl = vp[8 * blk + 4];   // (hi, hi) and (lo, lo) of pairs t, t + 4
            mma_bf16(av[0], ah.x, ah.y, ah.z, ah.w, bh.x, bh.y);
            mma_bf16(av[1], al.x, al.y, al.z, al.w, bh.x, bh.y);
            mma_bf16(av[2], ah.x, ah.y, ah.z, ah.w, bl.x, bl.y);
        }
        if constexpr (NPTW > 0) {
            const uint4 fh = af[64], fl = af[96];
#pragma unroll
            for (int i = 0; i < NPTW; i++) {
                const uint2 b = pp[i][4 * blk];
                mma_f16(ap[i][0], fl.x, fl.y, fl.z, fl.w, b.x, b.y);
                mma_f16(ap[i][1], fh.x, fh.y, fh.z, fh.w, b.x, b.y);
            }
        }
        if (++blk == nb) blk = 0;
    }
    // h plane in (X, Z) order, Z fastest: the 8 rows g of a store are contiguous
    const size_t nh = (size_t)a.nsnap * NF * a.ny * a.nlz * a.nlx;
    const size_t fstride = (size_t)a.ny * a.nlz * a.nlx;
    const size_t base = ((size_t)s * NF * a.ny + j) * ((size_t)a.nlz * a.nlx) + (size_t)X0 * a.nlz + 16 * zt + g;
    auto put = [&](int f, int n, float r0, float r8) {
        const size_t o = base + (size_t)f * fstride + (size_t)(a.OP * n) * a.nlz;
        if (in_range(o + 8, nh, a.err)) {
            a.h[o] = r0;
            a.h[o + 8] = r8;
        }
    };
    if constexpr (DOV) {
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const int cc = 2 * t + e;
            const int n = cc >= 3 ? 1 : 0;
            if (cc < PK::NV && (n ? val1 : val0))
                put(cc - 3 * n, n, (av[0][e] + av[1][e]) + av[2][e], (av[0][2 + e] + av[1][2 + e]) + av[2][2 + e]);
        }
    }
#pragma unroll
    for (int i = 0; i < NPTW; i++)
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const int cc = (pt0 + i) * 8 + 2 * t + e;
            const int n = cc >= 6 ? 1 : 0;
            if (cc < PK::NP && (n ? val1 : val0))
                put(3 + cc - 6 * n, n, ap[i][0][e] + ap[i][1][e], ap[i][0][2 + e] + ap[i][1][2 + e]);
        }
}

__device__ __forceinline__ void named_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

// Column stride of the parked columns (floats): +8 makes the 8-byte B loads
// of the z warps conflict-free.  z warps: the z work of a chunk grows with
// the LES z count, a larger share of the rows on the narrower grids (64 Z
// outputs for 256 rows at stride 4, against 48 for 384 at stride 8), so the
// 192- and 256-row kernels take as many z warps as their (Z tile, column
// tile) units at stride 4 allow within the 512 threads that one CTA per SM
// can hold at 128 registers (9 and 6); the 64- and 128-row kernels keep 3,
// which lets two or three CTAs share an SM.
template <int NZ>
struct Geo {
    static constexpr int LD = NZ + 8;
    static constexpr int NXW = NZ / 32;                    // x warps
    static constexpr int ZW = NZ == 192 ? 9 : NZ == 256 ? 6 : 3;   // z warps
    static constexpr int THREADS = NZ + 32 * (1 + ZW);
    static_assert(THREADS <= 512, "one CTA of at most 512 threads per SM");
    static constexpr int STGF = 3 * NZ * CW;               // floats per stage
};

template <int NZ, int MODE, int OPC>
__global__ void __launch_bounds__(Geo<NZ>::THREADS, 1) xz_ws(const __grid_constant__ WsMulti mp)
{
    int pi = 0;
    while (pi + 1 < mp.nplan && (int)blockIdx.x >= mp.cta0[pi + 1]) pi++;
    const WsArgs &a = mp.plan[pi];
    const int cta = (int)blockIdx.x - mp.cta0[pi], ncta = mp.cta0[pi + 1] - mp.cta0[pi];
    using G = Geo<NZ>;
    constexpr int LD = G::LD, NXW = G::NXW, STGF = G::STGF, kZW = G::ZW;
    constexpr int NR = 8 / OPC;                  // B rotations
    constexpr int BW = Bw<MODE>::n;
    using PK = Park<OPC>;
    constexpr size_t PF = PK::floats(LD);        // floats per parked-column buffer
    extern __shared__ float4 smem_dyn[];
    const int KS = a.KS;
    uint4 *afrag = reinterpret_cast<uint4 *>(smem_dyn);        // [KS][4][32 lanes]
    uint4 *bvar = afrag + KS * 128;                             // [NR][32 lanes][BW]
    float *colbuf = reinterpret_cast<float *>(bvar + NR * 32 * BW);   // [2 buffers][PF]
    float *stg;                                                 // [CSTG][3][NZ][CW], 128-B aligned
    {
        char *end = reinterpret_cast<char *>(colbuf + 2 * PF);
        const unsigned sa = smem_u32(end);
        stg = reinterpret_cast<float *>(end + (((sa + 127u) & ~127u) - sa));
    }
    __shared__ alignas(8) unsigned long long full[CSTG], empty[CSTG], cfull[2], cempty[2];
    __shared__ int abort_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    // persistent: items (snapshot, plane, phase) = it, it + ncta, ... of the
    // CTA's plan; ncta is a multiple of OP, so the phase of a CTA is fixed
    const int p = cta % a.OP;
    const int nitems = a.ny * a.OP * a.nsnap;
    const size_t np = (size_t)a.nx * a.ny * NZ;
    const int nchunk = a.nchunk;
    const bool pm = a.plane_mean != nullptr && p == 0;
    volatile int *abort_v = &abort_flag;

    if (tid == 0) {
        for (int i = 0; i < CSTG; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 32 * NXW);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&cfull[b], 32 * NXW);
            mbar_init(&cempty[b], 32 * kZW);
        }
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();

    // warp 0: producer; warps 1 .. kZW: z warps; the rest: x warps.  The
    // producer and z warps take the lowest warp ids (the schedulers prefer
    // older warps).
    if (warp == 0) {   // producer: stage k = chunk k = x blocks CB k - bshift .. + CB - 1, item by item
        if (lane == 0) {
            int gk = 0;
            for (int it = cta; it < nitems && !*abort_v; it += ncta) {
                const int j = (it / a.OP) % a.ny, s = it / (a.OP * a.ny);
                const int pc0 = s * 3 * a.ny + j;   // TMA plane coordinate of component 0
                for (int k = 0; k < nchunk; k++, gk++) {
                    const int st = gk % CSTG;
                    if (gk >= CSTG && !wait_or_abort(&empty[st], ((gk / CSTG) - 1) & 1, abort_v, a.err, a.wait_limit)) break;
                    if (*abort_v) break;
                    int b = (a.CB * k - a.bshift) % a.nlx;   // a multiple of CB: the chunk never wraps
                    if (b < 0) b += a.nlx;
                    proxy_fence();
                    float *buf = stg + st * STGF;
                    mbar_expect_tx(&full[st], 3u * NZ * CW * 4u);
                    for (int c = 0; c < 3; c++)
                        for (int r0 = 0; r0 < NZ; r0 += a.box_rows)
                            tma_load3(buf + ((size_t)c * NZ + r0) * CW, &a.tmap, &full[st], b * a.rx, r0,
                                      pc0 + c * a.ny);
                }
            }
            // no copy may be in flight when the CTA exits
            for (int k = gk > CSTG ? gk - CSTG : 0; k < gk; k++) mbar_wait(&full[k % CSTG], (k / CSTG) & 1, a.err);
        }
        return;
    }

    // x and z warps: z fragments, this phase's rotated x fragments
    constexpr int nwork = G::THREADS - 32;
    const int wtid = tid - 32;
    for (int i = wtid; i < KS * 128; i += nwork) afrag[i] = a.afrag[i];
    for (int i = wtid; i < NR * 32 * BW; i += nwork) bvar[i] = a.bvar[(size_t)p * NR * 32 * BW + i];
    named_sync(1, nwork);

    const int xc0 = a.xc0[p];
    const int xw = warp - 1 - kZW;                // x warp index (rows 32 xw ..)
    if (xw >= 0) {   // ---------------- x warps
        const float *xrow = stg + (size_t)(xw * 32 + g) * CW + 4 * t;   // this lane's row g, inputs 4t..
        float *colw0 = colbuf + xw * 32 + 2 * g;  // pair g of the warp's first block, velocity column 0
        // the reference profile U_c(y_j) of each item (uref, written by the
        // launch before), the next item's read one item ahead
        auto uref_of = [&](int it, float (&U)[3]) {
            const int j = (it / a.OP) % a.ny, s = it / (a.OP * a.ny);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const size_t k = ((size_t)s * 3 + c) * a.ny + j;
                U[c] = it < nitems && in_range(k, (size_t)a.nsnap * 3 * a.ny, a.err) ? (float)a.uref[k] : 0.f;
            }
        };
        float Un[3];
        uref_of(cta, Un);
        int gc = 0;                               // chunks of this CTA so far
        for (int it = cta; it < nitems; it += ncta) {
            const float U[3] = {Un[0], Un[1], Un[2]};
            uref_of(it + ncta, Un);
            float acc[2][NF][4];
#pragma unroll
            for (int m = 0; m < 2; m++)
#pragma unroll
                for (int f = 0; f < NF; f++)
#pragma unroll
                    for (int i = 0; i < 4; i++) acc[m][f][i] = 0.f;
            bool stop = false;
            for (int sidx = 0; sidx < nchunk; sidx++, gc++) {
                const int st = gc % CSTG;
                if (!wait_or_abort(&full[st], (gc / CSTG) & 1, abort_v, a.err, a.wait_limit)) { stop = true; break; }
                const int q = sidx % NR;
                uint4 B[BW];
#pragma unroll
                for (int w = 0; w < BW; w++) B[w] = bvar[(q * 32 + lane) * BW + w];
                const float *buf = xrow + st * STGF;
#pragma unroll
                for (int m = 0; m < 2; m++) {
                    if constexpr (MODE == MODE_BF16X3) {
                        // two components live at a time: (u1, u2), then (u2, u3), then (u1 reloaded, u3)
                        float2 v[3][2][2];
                        auto ld = [&](int c) {
                            const float2 nU = make_float2(-U[c], -U[c]);
#pragma unroll
                            for (int h = 0; h < 2; h++) {
                                const float4 x = *reinterpret_cast<const float4 *>(buf + (c * NZ + 16 * m + 8 * h) * CW);
                                v[c][h][0] = __fadd2_rn(make_float2(x.x, x.y), nU);
                                v[c][h][1] = __fadd2_rn(make_float2(x.z, x.w), nU);
                            }
                        };
                        ld(0); ld(1);
                        vp_pair<0, 3>(acc[m], v, B[0], B[1]);
                        vp_pair<1, 4>(acc[m], v, B[0], B[1]);
                        ld(2);
                        vp_pair<2, 6>(acc[m], v, B[0], B[1]);
                        pp_pair<7, 8>(acc[m], v, B[1]);
                        ld(0);
                        unsigned a5[4];
                        prod_pack<5>(v, a5);
                        mma_f16(acc[m][5], a5[0], a5[1], a5[2], a5[3], B[1].z, B[1].w);
                        mma_f16(acc[m][5], a5[0], a5[1], a5[2], a5[3], B[1].x, B[1].y);
                    } else {
                        float2 v[3][2][2];
#pragma unroll
                        for (int c = 0; c < 3; c++) {
                            const float2 nU = make_float2(-U[c], -U[c]);
#pragma unroll
                            for (int h = 0; h < 2; h++) {
                                const float4 x = *reinterpret_cast<const float4 *>(buf + (c * NZ + 16 * m + 8 * h) * CW);
                                v[c][h][0] = __fadd2_rn(make_float2(x.x, x.y), nU);
                                v[c][h][1] = __fadd2_rn(make_float2(x.z, x.w), nU);
                            }
                        }
                        x_mma_il_tf32(acc[m], v, B);
                    }
                }
                mbar_arrive(&empty[st]);
                // the chunk completes phase outputs X0 + OP i, i < OPC (tile columns OPC q + i)
                const int cb = gc & 1;
                if (gc >= 2 && !wait_or_abort(&cempty[cb], ((gc >> 1) - 1) & 1, abort_v, a.err, a.wait_limit)) { stop = true; break; }
                const int X0 = xc0 + a.OP * OPC * sidx;
                const int b0 = a.CB * sidx - a.bshift;     // first x block of the chunk
                float *colw = colw0 + (size_t)cb * PF;
                // product pair g of a block goes to word 2 (g mod 4) + g / 4 (Park's order)
                unsigned *prodw = reinterpret_cast<unsigned *>(colbuf + (size_t)cb * PF + PK::prod0(LD)) + xw * 16 +
                                  2 * (g & 3) + (g >> 2);
                const int csum = (OPC * q + 7) & 7;        // the idle column: row sums
                // rows (g, g + 8) of each 16-row block as one pair: velocities as two
                // FP32 values, products as one FP16x2 word
                auto park = [&](int n, int m, int e) {
#pragma unroll
                    for (int f = 0; f < 3; f++)
                        *reinterpret_cast<float2 *>(colw + (3 * n + f) * LD + 16 * m) =
                            make_float2(acc[m][f][e], acc[m][f][2 + e]);
#pragma unroll
                    for (int f = 3; f < NF; f++)
                        prodw[(6 * n + f - 3) * PK::LDP(LD) + 8 * m] = pack_f16(acc[m][f][e], acc[m][f][2 + e]);
                };
                if constexpr (OPC == 2) {
                    // columns 2q, 2q + 1 (lanes t == q, elements 0 and 1)
                    // block m = 0 first: its MMAs were issued before those of m = 1
                    if (t == q) {
                        const bool ok0 = X0 >= 0 && X0 < a.nlx, ok1 = X0 + a.OP >= 0 && X0 + a.OP < a.nlx;
#pragma unroll
                        for (int m = 0; m < 2; m++) {
                            if (ok0) park(0, m, 0);
                            if (ok1) park(1, m, 1);
                        }
                    }
                } else {
                    // column q (lanes t == q / 2, element q % 2)
                    if (t == (q >> 1) && X0 >= 0 && X0 < a.nlx) {
                        if (q & 1) {
#pragma unroll
                            for (int m = 0; m < 2; m++) park(0, m, 1);
                        } else {
#pragma unroll
                            for (int m = 0; m < 2; m++) park(0, m, 0);
                        }
                    }
                }
                // row sums of fields 0-2 (the idle column) go to the row-sum columns
                // when the chunk's blocks are owned (each input counted once)
                if (pm && t == (csum >> 1) && b0 >= 0 && b0 < a.nlx) {
                    const int es = csum & 1;
#pragma unroll
                    for (int m = 0; m < 2; m++)
#pragma unroll
                        for (int c = 0; c < 3; c++)
                            *reinterpret_cast<float2 *>(colw + PK::sum0(LD) + c * LD + 16 * m) =
                                es ? make_float2(acc[m][c][1], acc[m][c][3]) : make_float2(acc[m][c][0], acc[m][c][2]);
                }
                // clear the completed columns and the sum column without a branch; a
                // non-finite value stays in its column, and the y pass flags it
                {
                    const unsigned clr = (((OPC == 2 ? 3u : 1u) << (OPC * q)) | (1u << csum)) >> (2 * t);
                    const float2 keep = make_float2(clr & 1u ? 0.f : 1.f, clr & 2u ? 0.f : 1.f);
#pragma unroll
                    for (int m = 0; m < 2; m++)
#pragma unroll
                        for (int f = 0; f < NF; f++) {
                            const float2 lo = __fmul2_rn(make_float2(acc[m][f][0], acc[m][f][1]), keep);
                            const float2 hi = __fmul2_rn(make_float2(acc[m][f][2], acc[m][f][3]), keep);
                            acc[m][f][0] = lo.x; acc[m][f][1] = lo.y; acc[m][f][2] = hi.x; acc[m][f][3] = hi.y;
                        }
                }
                // split the warp's parked velocity pairs into (hi, lo) bf16 words,
                // all lanes sharing the work (NV columns x 2 blocks x 8 pairs), and
                // store them in Park's slot order within each block (a round reads
                // its blocks whole before any lane writes)
                __syncwarp();
                {
                    float *cw = colbuf + (size_t)cb * PF + xw * 32;
                    constexpr int NPAIR = PK::NV * 16;
#pragma unroll
                    for (int r = 0; r < (NPAIR + 31) / 32; r++) {
                        const int pidx = lane + 32 * r, col = pidx >> 4, off = pidx & 15, i = off & 7;
                        const bool act = NPAIR % 32 == 0 || pidx < NPAIR;
                        unsigned *blk = reinterpret_cast<unsigned *>(cw + (size_t)(act ? col : 0) * LD + 16 * (off >> 3));
                        unsigned hi = 0u, lo = 0u;
                        if (act) split2(*reinterpret_cast<const float2 *>(blk + 2 * i), hi, lo);
                        __syncwarp();
                        if (act) {
                            blk[2 * (i & 3) + (i >> 2)] = hi;
                            blk[8 + 2 * (i & 3) + (i >> 2)] = lo;
                        }
                    }
                }
                mbar_arrive(&cfull[cb]);
            }
            if (stop) break;
        }
        return;
    }

    // ---------------- z warps: with as many Z tiles as z warps, z warp zw takes
    // tile zw and every column tile; otherwise the (Z tile, column tile) units
    // round robin.  z warp c < 3 also sums the parked row sums of component c.
    constexpr int NPT = PK::NPT;
    const int npt = a.nf > 3 ? NPT : 0;          // product tiles only when the products are contracted
    const int zw = warp - 1;
    const int nzt = a.nlz / 16;
    int gc = 0;
    for (int it = cta; it < nitems; it += ncta) {
        const int j = (it / a.OP) % a.ny, s = it / (a.OP * a.ny);
        double pmean = 0.0;
        bool stop = false;
        for (int sidx = 0; sidx < nchunk; sidx++, gc++) {
            const int cb = gc & 1;
            if (!wait_or_abort(&cfull[cb], (gc >> 1) & 1, abort_v, a.err, a.wait_limit)) { stop = true; break; }
            const int X0 = xc0 + a.OP * OPC * sidx;
            const bool val0 = X0 >= 0 && X0 < a.nlx;
            const bool val1 = OPC == 2 && X0 + a.OP >= 0 && X0 + a.OP < a.nlx;
            const float *colb = colbuf + (size_t)cb * PF;
            if (pm && zw < 3) {
                const int b0 = a.CB * sidx - a.bshift;
                if (b0 >= 0 && b0 < a.nlx) {
                    float ssum = 0.f;
                    for (int z = lane; z < NZ; z += 32) ssum += colb[PK::sum0(LD) + zw * LD + z];
                    pmean += (double)ssum;
                }
            }
            if (val0 || val1) {
                if (nzt == kZW) {
                    if (npt) z_tile<OPC, LD, true, NPT>(a, colb, afrag, s, j, X0, val0, val1, zw, 0, lane);
                    else z_tile<OPC, LD, true, 0>(a, colb, afrag, s, j, X0, val0, val1, zw, 0, lane);
                } else {
                    const int nu = 1 + npt;          // per Z tile: the velocity tile, then each product tile
                    for (int w = zw; w < nu * nzt; w += kZW) {
                        const int u = w % nu, zt = w / nu;
                        if (u == 0) z_tile<OPC, LD, true, 0>(a, colb, afrag, s, j, X0, val0, val1, zt, 0, lane);
                        else z_tile<OPC, LD, false, 1>(a, colb, afrag, s, j, X0, val0, val1, zt, u - 1, lane);
                    }
                }
            }
            mbar_arrive(&cempty[cb]);
        }
        if (stop) break;
        if (pm && zw < 3) {
            for (int o = 16; o > 0; o >>= 1) pmean += __shfl_xor_sync(0xffffffffu, pmean, o);
            const size_t k = ((size_t)s * 3 + zw) * a.ny + j;
            if (lane == 0 && in_range(k, (size_t)a.nsnap * 3 * a.ny, a.err))
                a.plane_mean[k] = (double)(float)a.uref[k] + pmean / ((double)a.nx * NZ);
        }
    }
}

// Dynamic shared memory: z fragments, x B fragments, the parked columns,
// 128-byte alignment, the TMA stages.
template <int NZ, int MODE, int OPC>
size_t ws_smem_bytes(int KS)
{
    using G = Geo<NZ>;
    return sizeof(uint4) * (128 * (size_t)KS + (8 / OPC) * 32 * Bw<MODE>::n) + 128 +
           sizeof(float) * (2 * Park<OPC>::floats(G::LD) + (size_t)CSTG * G::STGF);
}

// Launch over the plans of one class; the grid is as many CTAs as fit at
// once, shared among the plans in proportion to their chunks (each share a
// multiple of the plan's OP and at most its item count).  Dynamic shared
// memory for the largest z-fragment table of the class.
template <int NZ, int MODE, int OPC>
cudaError_t ws_launch(WsMulti m, cudaStream_t st)
{
    size_t smem = 0;
    for (int i = 0; i < m.nplan; i++) {
        const size_t b = ws_smem_bytes<NZ, MODE, OPC>(m.plan[i].KS);
        smem = b > smem ? b : smem;
    }
    static size_t attr = 0;
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(xz_ws<NZ, MODE, OPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xz_ws<NZ, MODE, OPC>, Geo<NZ>::THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    double work = 0.0;
    for (int i = 0; i < m.nplan; i++) work += (double)m.plan[i].ny * m.plan[i].OP * m.plan[i].nsnap * m.plan[i].nchunk;
    m.cta0[0] = 0;
    for (int i = 0; i < m.nplan; i++) {
        const WsArgs &a = m.plan[i];
        const int nitems = a.ny * a.OP * a.nsnap;
        const double w = (double)a.ny * a.OP * a.nsnap * a.nchunk;
        int g = (int)((double)nsm * per_sm * w / work) / a.OP * a.OP;
        if (g < a.OP) g = a.OP;
        if (g > nitems) g = nitems;
        m.cta0[i + 1] = m.cta0[i] + g;
    }
    xz_ws<NZ, MODE, OPC><<<m.cta0[m.nplan], Geo<NZ>::THREADS, smem, st>>>(m);
    return cudaGetLastError();
}

}  // namespace ws
}  // namespace eles
