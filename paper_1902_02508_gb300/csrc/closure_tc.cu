// Learned-closure inference on the 5th-generation tensor cores (tcgen05).
//
// One persistent CTA per SM runs the whole MLP 10 -> 128 -> 128 -> 128 -> 6
// (SiLU) over tiles of 128 points: standardisation and the guard, four
// layers, de-standardisation and the exact-stress fallback, with nothing
// but the features read and the stress written in HBM.
//
// Numerics: the working weights are BF16 (the BF16-rounded FP32 masters the
// training kernels use) and enter the MMA exactly.  Every activation a is
// split into a_hi = bf16(a) and a_lo = bf16(a - a_hi), both multiplied by the
// weights with FP32 accumulation in TMEM, so an activation keeps 16
// significant bits (|a - a_hi - a_lo| <= 2^-16 |a|): the served network is
// the FP32-activation network the training passes evaluate, to a few parts
// in 10^6, not a BF16-activation approximation of it.
//
// Layout: shared memory holds the weight image, every matrix in the K-major
// no-swizzle canonical layout of tcgen05 (8 x 8 BF16 core matrices of 128
// contiguous bytes, core (r/8, k/8) at ((r/8)(K/8) + k/8) * 128 bytes, i.e.
// leading (K) byte offset 128 and stride (row-group) byte offset K * 16).
// Three tile slots of eight warps each keep three tiles in flight: each has
// 128 FP32 accumulator columns in TMEM, and the next layer's A operand (a_hi,
// a_lo) lives in shared memory for slots 0 and 1 (same layout, 64 KB each)
// and in the remaining 128 TMEM columns for slot 2 (two BF16 per 32-bit
// column, written with tcgen05.st and read by the MMA from TMEM).  The MMAs
// of one slot's layer run while the other slots' warps do their epilogues.
// Warp w owns TMEM lanes (rows) 32 (w % 4) .. +31, one row per thread, and
// the two warps of a slot on the same lanes take 64 columns each, so every
// thread carries its point from the features to the output.
#include <cuda_bf16.h>
#include <math.h>

#include <type_traits>

#include "eles_internal.h"
#include "fused_stage.cuh"

namespace eles {
namespace {

constexpr int kRows = 128;                  // points per tile (MMA M)
constexpr int kHid = 128;                   // hidden width
constexpr int kIn = 10, kOut = 6;
constexpr int kK0 = 16;                     // first-layer K, padded
constexpr int kW3Row = 8;                   // output-layer weights, FP32 [k][8] (6 used)

// weight image (bytes); the same image is the device buffer and the head of shared memory
constexpr int kImgW0 = 0;                                  // [128][16]
constexpr int kImgW1 = kImgW0 + kHid * kK0 * 2;            // [128][128]
constexpr int kImgW2 = kImgW1 + kHid * kHid * 2;           // [128][128]
constexpr int kImgW3 = kImgW2 + kHid * kHid * 2;           // float [128][8]
constexpr int kImgBias = kImgW3 + kHid * kW3Row * 4;       // float b0[128] b1[128] b2[128] b3[16]
constexpr int kImgStats = kImgBias + 4 * (3 * kHid + 16);  // float mu[16] inv_sd[16] tmu[8] tsd[8]
constexpr int kImgBytes = kImgStats + 4 * 48;
static_assert(kImgBytes % 128 == 0, "image must keep the operand buffers 128-byte aligned");

constexpr int kSlots = 3;
constexpr int kSmemSlots = 2;                              // slots 0, 1: A operand in shared memory
constexpr int kOperandBytes = kRows * kHid * 2;            // one of a_hi, a_lo: 128 x 128 BF16
constexpr int kAOff = kImgBytes;
constexpr int kXOff = kAOff + kSmemSlots * 2 * kOperandBytes;   // output-layer partials exchanged by the halves
constexpr int kXBytes = kSlots * 2 * kRows * 16;           // [slot][half][row][4] floats
constexpr int kBarOff = kXOff + kXBytes;
constexpr int kSmemBytes = kBarOff + 64;                   // 3 mbarriers, TMEM address, 3 abort flags
constexpr int kSlotThreads = 256;                          // 8 warps per slot
constexpr int kThreads = kSlots * kSlotThreads;
constexpr unsigned kTmemCols = 512;                        // D of slot g at [128 g, 128 g + 128); slot 2's
constexpr unsigned kAhiCol = 384, kAloCol = 448;           // a_hi at [384, 448), a_lo at [448, 512)
static_assert(kSmemBytes <= 227 * 1024, "shared memory");

__host__ __device__ constexpr int core_off(int r, int k, int K)
{
    return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// ----------------------------------------------------------- PTX helpers --
// Shared-memory matrix descriptor, K-major, no swizzle: start address,
// leading-dimension byte offset (between core matrices along K), stride
// byte offset (between 8-row groups), descriptor version 1 (bits 46-47).
__device__ __forceinline__ unsigned long long sdesc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    return (unsigned long long)((saddr & 0x3FFFFu) >> 4) | ((unsigned long long)(lbo >> 4) << 16) |
           ((unsigned long long)(sbo >> 4) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major.
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
// D (+)= A B, A and B from shared memory (descriptors).
__device__ __forceinline__ void mma_bf16_ss(unsigned dtmem, unsigned long long a, unsigned long long b, unsigned id,
                                            unsigned acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(dtmem), "l"(a), "l"(b), "r"(id), "r"(acc));
}
// D (+)= A B with A read from tensor memory (a_tmem: lane 0, first column)
// and B from shared memory (descriptor).
__device__ __forceinline__ void mma_bf16_ts(unsigned dtmem, unsigned a_tmem, unsigned long long b, unsigned id,
                                            unsigned acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
                 ::"r"(dtmem), "r"(a_tmem), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                 ::"r"(fz::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane: the load is
// issued here and completes at tmem_ld16_wait, which carries the registers
// so that no use of them is scheduled before it (a wait covers every load
// issued before it).
__device__ __forceinline__ void tmem_ld16_issue(unsigned taddr, unsigned (&v)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16_wait(unsigned (&v)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
                 :: "memory");
}
__device__ __forceinline__ void tmem_st8(unsigned taddr, const unsigned (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n"
                 ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_st4(unsigned taddr, const unsigned (&v)[4])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};\n"
                 ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]) : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// hi = bf16(a), lo = bf16(a - hi) for a pair, packed as bf16x2 words (the
// lower k in the lower half).  a - hi is exact in FP32.
__device__ __forceinline__ void split2(float2 a, unsigned &hi, unsigned &lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a.x, a.y);
    hi = *reinterpret_cast<const unsigned *>(&h);
    const float2 hf = make_float2(__uint_as_float(hi << 16), __uint_as_float(hi & 0xffff0000u));
    const float2 r = __ffma2_rn(hf, make_float2(-1.f, -1.f), a);
    const __nv_bfloat162 l = __floats2bfloat162_rn(r.x, r.y);
    lo = *reinterpret_cast<const unsigned *>(&l);
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// SiLU of a pair: z / (1 + e^-z) with e^-z = 2^(-z log2 e).  For z below
// about -88 the exponential overflows to +inf and the quotient is -0.
__device__ __forceinline__ float2 silu2(float2 z)
{
    constexpr float kNegLog2e = -1.4426950408889634f;
    const float2 x = __fmul2_rn(z, make_float2(kNegLog2e, kNegLog2e));
    const float2 d = __fadd2_rn(make_float2(ex2_approx(x.x), ex2_approx(x.y)), make_float2(1.f, 1.f));
    return __fmul2_rn(z, make_float2(rcp_approx(d.x), rcp_approx(d.y)));
}

// ------------------------------------------------------------ the image --
// One thread per image element: BF16 weight bits (the working weights are
// already BF16 values), zero padding, FP32 biases and statistics.
__global__ void pack_image(const float *__restrict__ wq, long w0, long b0, long w1, long b1, long w2, long b2,
                           long w3, long b3, const double *__restrict__ stats, unsigned char *img)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nw = kHid * kK0 + 2 * kHid * kHid + kHid * kW3Row;
    auto bits = [&](float v) { return (unsigned short)(__float_as_uint(v) >> 16); };
    if (i < kHid * kK0) {                                       // W0 [128][16], k >= 10 zero
        const int r = i / kK0, k = i % kK0;
        const float v = k < kIn ? wq[w0 + (long)r * kIn + k] : 0.f;
        *reinterpret_cast<unsigned short *>(img + kImgW0 + core_off(r, k, kK0)) = bits(v);
    } else if (i < kHid * kK0 + 2 * kHid * kHid) {              // W1, W2 [128][128]
        const int j = i - kHid * kK0, l = j / (kHid * kHid), e = j % (kHid * kHid);
        const int r = e / kHid, k = e % kHid;
        const float v = wq[(l ? w2 : w1) + (long)r * kHid + k];
        *reinterpret_cast<unsigned short *>(img + (l ? kImgW2 : kImgW1) + core_off(r, k, kHid)) = bits(v);
    } else if (i < nw) {                                        // W3 as FP32 [k][8], q >= 6 zero
        const int e = i - kHid * kK0 - 2 * kHid * kHid, k = e / kW3Row, q = e % kW3Row;
        reinterpret_cast<float *>(img + kImgW3)[e] = q < kOut ? wq[w3 + (long)q * kHid + k] : 0.f;
    } else if (i < nw + 3 * kHid + 16) {                        // biases
        const int e = i - nw;
        float v;
        if (e < 3 * kHid) v = wq[(e < kHid ? b0 : e < 2 * kHid ? b1 : b2) + e % kHid];
        else v = e - 3 * kHid < kOut ? wq[b3 + e - 3 * kHid] : 0.f;
        reinterpret_cast<float *>(img + kImgBias)[e] = v;
    } else if (i < nw + 3 * kHid + 16 + 48) {                   // statistics
        const int e = i - nw - 3 * kHid - 16;
        float v = 0.f;
        if (e < kIn) v = (float)stats[e];                                  // feature means
        else if (e >= 16 && e < 16 + kIn) v = (float)(1.0 / stats[10 + e - 16]);   // 1 / feature sd
        else if (e >= 32 && e < 32 + kOut) v = (float)stats[20 + e - 32];  // target means
        else if (e >= 40 && e < 40 + kOut) v = (float)stats[26 + e - 40];  // target sd
        reinterpret_cast<float *>(img + kImgStats)[e] = v;
    }
}
constexpr int kImgElems = kHid * kK0 + 2 * kHid * kHid + kHid * kW3Row + 3 * kHid + 16 + 48;

// ------------------------------------------------------------ the kernel --
// Slot g (warps 8g .. 8g+7) handles tiles g, g + 3 G, ... of CTA b's
// sequence 3 (b + k G) + g (G CTAs).  The two warps of a TMEM lane quadrant
// split the 128 columns of the epilogue.  Slots 0 and 1 keep the A operand
// in shared memory, slot 2 in tensor memory (512 columns hold three
// accumulators and one hi/lo operand).  Per tile: inputs -> MMA layer 0 ->
// (wait, epilogue, MMA) x 3 -> wait -> output; the next tile's features are
// fetched while the four layers run.  Every wait is bounded; on expiry the
// slot records EF_ERR_TIMEOUT and stops, and the CTA frees its TMEM.

__device__ __forceinline__ void load_feats(const float *__restrict__ feats, long p, long n, float (&f)[kIn])
{
#pragma unroll
    for (int k = 0; k < kIn; k++) f[k] = p < n ? __ldg(feats + p * kIn + k) : 0.f;
}

// bias, SiLU and split of 16 accumulator columns (8 pairs)
__device__ __forceinline__ void act16(const unsigned (&v)[16], const float2 *b2, unsigned (&hw)[8], unsigned (&lw)[8])
{
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const float2 z = __fadd2_rn(make_float2(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1])), b2[j]);
        split2(silu2(z), hw[j], lw[j]);
    }
}

// Epilogue of one thread over its 64 accumulator columns [c0, c0 + 64):
// four pieces of 16, the TMEM load of the next piece in flight while one is
// computed.  tl_d: the warp's lanes at the slot's accumulator; tl_a: the
// warp's lanes at column 0 (the TMEM operand columns are absolute).  The
// hi/lo words go to the slot's operand in TMEM (kTmemA) or shared memory.
template <bool kTmemA>
__device__ __forceinline__ void epilogue64(unsigned tl_d, unsigned tl_a, int c0, const float2 *b2,
                                           unsigned char *Ahi, unsigned char *Alo, int r)
{
    unsigned va[16], vb[16], hw[8], lw[8];
    auto put = [&](int piece) {
        const int k = c0 + 16 * piece;                 // next layer's k of these 16 activations
        if (kTmemA) {
            tmem_st8(tl_a + kAhiCol + k / 2, hw);
            tmem_st8(tl_a + kAloCol + k / 2, lw);
        } else {
            *reinterpret_cast<uint4 *>(Ahi + core_off(r, k, kHid)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4 *>(Ahi + core_off(r, k + 8, kHid)) = make_uint4(hw[4], hw[5], hw[6], hw[7]);
            *reinterpret_cast<uint4 *>(Alo + core_off(r, k, kHid)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            *reinterpret_cast<uint4 *>(Alo + core_off(r, k + 8, kHid)) = make_uint4(lw[4], lw[5], lw[6], lw[7]);
        }
    };
    const unsigned src = tl_d + c0;
    tmem_ld16_issue(src, va);
    tmem_ld16_wait(va);
    tmem_ld16_issue(src + 16, vb);
    act16(va, b2, hw, lw);
    put(0);
    tmem_ld16_wait(vb);
    tmem_ld16_issue(src + 32, va);
    act16(vb, b2 + 8, hw, lw);
    put(1);
    tmem_ld16_wait(va);
    tmem_ld16_issue(src + 48, vb);
    act16(va, b2 + 16, hw, lw);
    put(2);
    tmem_ld16_wait(vb);
    act16(vb, b2 + 24, hw, lw);
    put(3);
}

// Epilogue of the last hidden layer fused with the output layer, on the CUDA
// cores in FP32: y_q += sum over the thread's 64 columns k of W3[q][k] a_k
// with the activations unsplit.  y holds (y0, y1), (y2, y3), (y4, y5).
__device__ __forceinline__ void epilogue64_out(unsigned tl_d, int c0, const float2 *b2, const float *w3,
                                               float2 (&y)[3])
{
    unsigned va[16], vb[16];
    auto acc16 = [&](const unsigned (&v)[16], int piece) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const float2 z = __fadd2_rn(make_float2(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1])),
                                        b2[8 * piece + j]);
            const float2 a = silu2(z);
            const float *w = w3 + (c0 + 16 * piece + 2 * j) * kW3Row;
#pragma unroll
            for (int e = 0; e < 2; e++) {
                const float ae = e ? a.y : a.x;
                const float4 w0 = *reinterpret_cast<const float4 *>(w + e * kW3Row);
                const float2 w1 = *reinterpret_cast<const float2 *>(w + e * kW3Row + 4);
                const float2 aa = make_float2(ae, ae);
                y[0] = __ffma2_rn(make_float2(w0.x, w0.y), aa, y[0]);
                y[1] = __ffma2_rn(make_float2(w0.z, w0.w), aa, y[1]);
                y[2] = __ffma2_rn(w1, aa, y[2]);
            }
        }
    };
    const unsigned src = tl_d + c0;
    tmem_ld16_issue(src, va);
    tmem_ld16_wait(va);
    tmem_ld16_issue(src + 16, vb);
    acc16(va, 0);
    tmem_ld16_wait(vb);
    tmem_ld16_issue(src + 32, va);
    acc16(vb, 1);
    tmem_ld16_wait(va);
    tmem_ld16_issue(src + 48, vb);
    acc16(va, 2);
    tmem_ld16_wait(vb);
    acc16(vb, 3);
}

__global__ void __launch_bounds__(kThreads, 1)
closure_mlp_tc_kernel(const uint4 *__restrict__ img, const float *__restrict__ feats, long n, long ntiles,
                      float guard, const float *__restrict__ exact, float *__restrict__ tau, int *nfall, int *err)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = warp >> 3, quad = warp & 3, half = (warp >> 2) & 1, r = 32 * quad + lane;
    for (int i = tid; i < kImgBytes / 16; i += kThreads) reinterpret_cast<uint4 *>(sm)[i] = img[i];
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(sm + kBarOff);
    unsigned *tmem_holder = reinterpret_cast<unsigned *>(sm + kBarOff + 8 * kSlots);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + kBarOff + 8 * kSlots + 4);
    if (tid == 0) {
        for (int k = 0; k < kSlots; k++) {
            fz::mbar_init(&bar[k], 1);
            abort_flag[k] = 0;
        }
        fz::mbar_fence_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(fz::smem_u32(tmem_holder)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    fz::proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_holder;
    const bool tmemA = g == kSmemSlots;                          // this slot's operand lives in TMEM
    const unsigned dslot = tmem + kRows * g;                     // this slot's accumulator (lane 0)
    const unsigned tlane = dslot + ((unsigned)(32 * quad) << 16);  // this warp's lanes
    const unsigned tlane_a = tmem + ((unsigned)(32 * quad) << 16); // the same lanes, column 0 (operand base)
    unsigned char *Ahi = sm + kAOff + (tmemA ? 0 : g) * 2 * kOperandBytes, *Alo = Ahi + kOperandBytes;
    const float *bias = reinterpret_cast<const float *>(sm + kImgBias);
    const float *st = reinterpret_cast<const float *>(sm + kImgStats);
    const bool issuer = (tid & (kSlotThreads - 1)) == 0;
    const int barid = 1 + g;
    const unsigned sA_hi = fz::smem_u32(Ahi), sA_lo = fz::smem_u32(Alo), sImg = fz::smem_u32(sm);
    constexpr unsigned id128 = idesc_bf16(kRows, kHid);
    const float *w3 = reinterpret_cast<const float *>(sm + kImgW3);
    float *xch = reinterpret_cast<float *>(sm + kXOff) + (size_t)g * 2 * kRows * 4;   // [half][row][4]
    unsigned phase = 0;

    auto slot_sync = [&]() { asm volatile("bar.sync %0, %1;\n" ::"r"(barid), "r"(kSlotThreads) : "memory"); };
    // bounded wait of the slot's MMA barrier by one thread, shared with the slot
    auto slot_wait = [&]() -> bool {
        if (issuer && !fz::mbar_wait(&bar[g], phase, err)) abort_flag[g] = 1;
        slot_sync();
        phase ^= 1u;
        tc_fence_after();
        return abort_flag[g] == 0;
    };
    // the A operand written by every thread (TMEM or shared memory) is
    // complete and visible to the tensor core before the MMA is issued
    auto operand_ready = [&]() {
        if (tmemA) tmem_wait_st();
        else fz::proxy_fence();
        tc_fence_before();
        slot_sync();
    };
    // One layer's MMAs over KS k-steps of 16, hi and lo, B from the image.
    // A k-step advances a descriptor's start address by 256 bytes (16 in its
    // encoded low field) and a TMEM operand by 8 columns; the base
    // descriptors are fixed for the kernel.
    const unsigned long long dA0hi = sdesc(sA_hi, 128, kK0 * 16), dA0lo = sdesc(sA_lo, 128, kK0 * 16);
    const unsigned long long dAhi = sdesc(sA_hi, 128, kHid * 16), dAlo = sdesc(sA_lo, 128, kHid * 16);
    const unsigned long long dW0 = sdesc(sImg + kImgW0, 128, kK0 * 16);
    const unsigned long long dW1 = sdesc(sImg + kImgW1, 128, kHid * 16), dW2 = sdesc(sImg + kImgW2, 128, kHid * 16);
    auto issue = [&](auto ksteps, unsigned long long bw, unsigned long long ahi, unsigned long long alo) {
        tc_fence_after();
#pragma unroll
        for (int ks = 0; ks < decltype(ksteps)::value; ks++) {
            if (tmemA) {
                mma_bf16_ts(dslot, tmem + kAhiCol + 8 * ks, bw + 16 * ks, id128, ks > 0 ? 1u : 0u);
                mma_bf16_ts(dslot, tmem + kAloCol + 8 * ks, bw + 16 * ks, id128, 1u);
            } else {
                mma_bf16_ss(dslot, ahi + 16 * ks, bw + 16 * ks, id128, ks > 0 ? 1u : 0u);
                mma_bf16_ss(dslot, alo + 16 * ks, bw + 16 * ks, id128, 1u);
            }
        }
        mma_commit(&bar[g]);
    };

    long t = g + (long)kSlots * blockIdx.x;
    float f[kIn];
    load_feats(feats, t * kRows + r, n, f);
    for (; t < ntiles; t += (long)kSlots * gridDim.x) {
        const long p = t * kRows + r;
        const bool valid = p < n;
        // standardised inputs and the guard; each half writes 8 of the 16 k
        float h[kK0];
        bool out = false;
#pragma unroll
        for (int k = 0; k < kK0; k++) {
            h[k] = 0.f;
            if (k < kIn && valid) {
                h[k] = (f[k] - st[k]) * st[16 + k];
                out |= fabsf(h[k]) > guard;
            }
        }
        {
            unsigned hv[4], lv[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const float2 a = half ? make_float2(h[8 + 2 * i], h[9 + 2 * i]) : make_float2(h[2 * i], h[2 * i + 1]);
                split2(a, hv[i], lv[i]);
            }
            if (tmemA) {
                tmem_st4(tlane_a + kAhiCol + 4 * half, hv);
                tmem_st4(tlane_a + kAloCol + 4 * half, lv);
            } else {
                *reinterpret_cast<uint4 *>(Ahi + core_off(r, 8 * half, kK0)) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                *reinterpret_cast<uint4 *>(Alo + core_off(r, 8 * half, kK0)) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
            }
        }
        if (half == 0) {
            const unsigned ballot = __ballot_sync(0xffffffffu, out);
            if (lane == 0 && ballot) atomicAdd(nfall, __popc(ballot));
        }
        operand_ready();
        if (issuer) issue(std::integral_constant<int, 1>(), dW0, dA0hi, dA0lo);
        load_feats(feats, (t + (long)kSlots * gridDim.x) * kRows + r, n, f);   // the next tile's, in flight meanwhile
        bool ok = true;
        for (int l = 1; l < 3 && ok; l++) {
            ok = slot_wait();
            if (!ok) break;
            // epilogue of hidden layer l - 1: bias, SiLU, split into the next A operand
            const float2 *b2 = reinterpret_cast<const float2 *>(bias + (l - 1) * kHid) + 32 * half;
            if (tmemA) epilogue64<true>(tlane, tlane_a, 64 * half, b2, Ahi, Alo, r);
            else epilogue64<false>(tlane, tlane_a, 64 * half, b2, Ahi, Alo, r);
            operand_ready();
            if (issuer) issue(std::integral_constant<int, kHid / 16>(), l == 1 ? dW1 : dW2, dAhi, dAlo);
        }
        if (!ok || !slot_wait()) break;
        // last hidden layer and the output layer; the halves exchange their
        // partial sums: half h finishes outputs 3h .. 3h + 2
        float2 y[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        epilogue64_out(tlane, 64 * half, reinterpret_cast<const float2 *>(bias + 2 * kHid) + 32 * half, w3, y);
        {
            const float ys[6] = {y[0].x, y[0].y, y[1].x, y[1].y, y[2].x, y[2].y};
            float *mine = xch + ((size_t)half * kRows + r) * 4;          // the other half's outputs
            mine[0] = ys[half ? 0 : 3];
            mine[1] = ys[half ? 1 : 4];
            mine[2] = ys[half ? 2 : 5];
            slot_sync();
            const float *theirs = xch + ((size_t)(1 - half) * kRows + r) * 4;
            if (valid) {
                const bool fall = out && exact != nullptr;
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const int qq = 3 * half + j;
                    const float yq = (half ? ys[3 + j] : ys[j]) + theirs[j] + bias[3 * kHid + qq];
                    tau[qq * n + p] = fall ? __ldg(exact + qq * n + p) : fmaf(st[40 + qq], yq, st[32 + qq]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// Exact stress at the guarded points (the closure's fallback through a filter
// plan).  Blocks stride over groups of 256 points; each thread repeats the
// inference kernel's guard test (the same FP32 statistics of the packed image,
// the same arithmetic), the block lists its group's guarded points and then
// evaluates T at each of them by direct summation of the plan's banded
// operators over the DNS snapshot in FP64 (Eq. 6):
//   ubar_a = sum_{j,z,x} Ay^{p_a}[J][j] Az[Z][z] Ax[X][x] u_a(j, z, x),
//   bar(u_a u_b) likewise with the parity p_a p_b,  T_ab = bar(u_a u_b) - ubar_a ubar_b,
// at the LES node of point p = (J nlz + Z) nlx + X, overwriting tau there.
__global__ void __launch_bounds__(256) exact_fallback_kernel(const __grid_constant__ ExactFallbackArgs a)
{
    __shared__ int list[256];
    __shared__ int nlist;
    __shared__ double red[8][9];
    const float *st = reinterpret_cast<const float *>(a.image + kImgStats);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nrow_z = a.Tz;
    for (long base = (long)blockIdx.x * 256; base < a.n; base += (long)gridDim.x * 256) {
        if (tid == 0) nlist = 0;
        __syncthreads();
        const long p = base + tid;
        if (p < a.n) {
            bool out = false;
#pragma unroll
            for (int k = 0; k < kIn; k++) out |= fabsf((__ldg(a.feats + p * kIn + k) - st[k]) * st[16 + k]) > a.guard;
            if (out) list[atomicAdd(&nlist, 1)] = tid;
        }
        __syncthreads();
        const int nl = nlist;
        for (int i = 0; i < nl; i++) {
            const long q = base + list[i];
            const int X = (int)(q % a.nlx), Z = (int)((q / a.nlx) % a.nlz), J = (int)(q / ((long)a.nlx * a.nlz));
            const int j0 = a.ystart[J], nj = a.ycount[J];
            double acc[9];
#pragma unroll
            for (int f = 0; f < 9; f++) acc[f] = 0.0;
            for (int r = tid; r < nj * nrow_z; r += 256) {
                const int j = j0 + r / nrow_z, kz = r % nrow_z;
                int z = a.zstart[Z] + kz;
                z = ((z % a.nz) + a.nz) % a.nz;
                const double wz = a.zw[(size_t)Z * a.Tz + kz];
                if (wz == 0.0) continue;
                double s[9];
#pragma unroll
                for (int f = 0; f < 9; f++) s[f] = 0.0;
                const size_t row = ((size_t)j * a.nz + z) * a.nx;
                for (int kx = 0; kx < a.Tx; kx++) {
                    int x = a.xstart[X] + kx;
                    x = ((x % a.nx) + a.nx) % a.nx;
                    const double wx = a.xw[(size_t)X * a.Tx + kx];
                    double v[3];
#pragma unroll
                    for (int c = 0; c < 3; c++)
                        v[c] = a.u64 ? a.u64[(size_t)c * a.np + row + x] : (double)a.u32[(size_t)c * a.np + row + x];
                    s[0] += wx * v[0]; s[1] += wx * v[1]; s[2] += wx * v[2];
                    s[3] += wx * v[0] * v[0]; s[4] += wx * v[0] * v[1]; s[5] += wx * v[0] * v[2];
                    s[6] += wx * v[1] * v[1]; s[7] += wx * v[1] * v[2]; s[8] += wx * v[2] * v[2];
                }
                const double we = wz * a.yw[0][(size_t)J * a.ny + j], wo = wz * a.yw[1][(size_t)J * a.ny + j];
                const int pa[9] = {a.par[0], a.par[1], a.par[2], 1, a.par[0] * a.par[1], a.par[0] * a.par[2], 1,
                                   a.par[1] * a.par[2], 1};
#pragma unroll
                for (int f = 0; f < 9; f++) acc[f] += (pa[f] > 0 ? we : wo) * s[f];
            }
#pragma unroll
            for (int f = 0; f < 9; f++) {
                double v = acc[f];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) red[warp][f] = v;
            }
            __syncthreads();
            if (tid < 6) {
                const int PI[6] = {0, 0, 0, 1, 1, 2}, PJ[6] = {0, 1, 2, 1, 2, 2};
                double ub[3] = {0.0, 0.0, 0.0}, uu = 0.0;
                for (int w = 0; w < 8; w++) {
                    for (int c = 0; c < 3; c++) ub[c] += red[w][c];
                    uu += red[w][3 + tid];
                }
                a.tau[(size_t)tid * a.n + q] = (float)(uu - ub[PI[tid]] * ub[PJ[tid]]);
            }
            __syncthreads();
        }
        __syncthreads();   // every thread has read nlist before the next group resets it
    }
}

}  // namespace

size_t closure_tc_image_bytes() { return kImgBytes; }

int closure_exact_fallback(const ExactFallbackArgs &a, cudaStream_t s)
{
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "closure_exact_fallback");
    const long groups = (a.n + 255) / 256;
    const int grid = (int)(groups < 4L * nsm ? groups : 4L * nsm);
    exact_fallback_kernel<<<grid, 256, 0, s>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? EF_OK : cuda_fail(e, "exact_fallback_kernel");
}

int closure_infer_tc(const float *wq, const long *off_w, const long *off_b, const double *stats, void *image,
                     const float *feats, long n, float guard, const float *exact, float *tau, int *nfall, int *err,
                     cudaStream_t s)
{
    static int smem_set_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && smem_set_dev != dev) {
        e = cudaFuncSetAttribute(closure_mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e == cudaSuccess) smem_set_dev = dev;
    }
    int nsm = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "closure_infer_tc setup");
    pack_image<<<(kImgElems + 255) / 256, 256, 0, s>>>(wq, off_w[0], off_b[0], off_w[1], off_b[1], off_w[2], off_b[2],
                                                      off_w[3], off_b[3], stats, static_cast<unsigned char *>(image));
    const long ntiles = (n + kRows - 1) / kRows;
    const long want = (ntiles + kSlots - 1) / kSlots;
    const int grid = (int)(want < nsm ? want : nsm);
    closure_mlp_tc_kernel<<<grid, kThreads, kSmemBytes, s>>>(static_cast<const uint4 *>(image), feats, n, ntiles, guard,
                                                       exact, tau, nfall, err);
    e = cudaGetLastError();
    return e == cudaSuccess ? EF_OK : cuda_fail(e, "closure_infer_tc");
}

}  // namespace eles
