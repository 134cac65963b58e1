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
// significant bits (|a - a_hi - a_lo| <= 2^-17 |a|): the served network is
// the FP32-activation network the training passes evaluate, to a few parts
// in 10^6, not a BF16-activation approximation of it.
//
// Layout: shared memory holds only the weight image, every matrix in the
// K-major no-swizzle canonical layout of tcgen05 (8 x 8 BF16 core matrices of
// 128 contiguous bytes, core (r/8, k/8) at ((r/8)(K/8) + k/8) * 128 bytes,
// i.e. leading (K) byte offset 128 and stride (row-group) byte offset
// K * 16).  The activations stay in tensor memory: per tile slot, 128 FP32
// accumulator columns and the A operand of the next layer (a_hi and a_lo,
// two BF16 per 32-bit column, 64 columns each), written by the epilogue with
// tcgen05.st and read by the MMA from TMEM.  Two slots of eight warps each
// fill the 512 TMEM columns: the MMAs of one slot's layer run while the other
// slot's warps do their epilogue.  Warp w owns TMEM lanes (rows)
// 32 (w % 4) .. +31, one row per thread, and the two warps of a slot on the
// same lanes take 64 columns each, so every thread carries its point from
// the features to the output.
#include <cuda_bf16.h>
#include <math.h>

#include "eles_internal.h"
#include "fused_stage.cuh"

namespace eles {
namespace {

constexpr int kRows = 128;                  // points per tile (MMA M)
constexpr int kHid = 128;                   // hidden width
constexpr int kIn = 10, kOut = 6;
constexpr int kK0 = 16;                     // first-layer K, padded
constexpr int kN3 = 16;                     // last-layer N, padded (MMA N >= 16 for M = 128)

// weight image (bytes); the same image is the device buffer and the head of shared memory
constexpr int kImgW0 = 0;                                  // [128][16]
constexpr int kImgW1 = kImgW0 + kHid * kK0 * 2;            // [128][128]
constexpr int kImgW2 = kImgW1 + kHid * kHid * 2;           // [128][128]
constexpr int kImgW3 = kImgW2 + kHid * kHid * 2;           // [16][128]
constexpr int kImgBias = kImgW3 + kN3 * kHid * 2;          // float b0[128] b1[128] b2[128] b3[16]
constexpr int kImgStats = kImgBias + 4 * (3 * kHid + kN3); // float mu[16] inv_sd[16] tmu[8] tsd[8]
constexpr int kImgBytes = kImgStats + 4 * 48;
static_assert(kImgBytes % 128 == 0, "image must keep the operand buffers 128-byte aligned");

constexpr int kBarOff = kImgBytes;
constexpr int kSmemBytes = kBarOff + 32;                   // 2 mbarriers, TMEM address, 2 abort flags
constexpr int kThreads = 512;                              // 2 slots x 8 warps
constexpr unsigned kTmemCols = 512;                        // per slot: D [0,128), a_hi [128,192), a_lo [192,256)
constexpr unsigned kSlotCols = 256, kAhiCol = 128, kAloCol = 192;

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

// 32 consecutive FP32 columns of this thread's TMEM lane; the wait carries
// the registers so that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_ld32(unsigned taddr, unsigned (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                   "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]),
                   "+r"(v[22]), "+r"(v[23]), "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]),
                   "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
                 :: "memory");
}
__device__ __forceinline__ void tmem_ld8(unsigned taddr, unsigned (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7])
                 :: "memory");
}

__device__ __forceinline__ void tmem_st16(unsigned taddr, const unsigned (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n"
                 ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
                   "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
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
    const int nw = kHid * kK0 + 2 * kHid * kHid + kN3 * kHid;
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
    } else if (i < nw) {                                        // W3 [16][128], rows >= 6 zero
        const int e = i - kHid * kK0 - 2 * kHid * kHid, r = e / kHid, k = e % kHid;
        const float v = r < kOut ? wq[w3 + (long)r * kHid + k] : 0.f;
        *reinterpret_cast<unsigned short *>(img + kImgW3 + core_off(r, k, kHid)) = bits(v);
    } else if (i < nw + 3 * kHid + kN3) {                       // biases
        const int e = i - nw;
        float v;
        if (e < 3 * kHid) v = wq[(e < kHid ? b0 : e < 2 * kHid ? b1 : b2) + e % kHid];
        else v = e - 3 * kHid < kOut ? wq[b3 + e - 3 * kHid] : 0.f;
        reinterpret_cast<float *>(img + kImgBias)[e] = v;
    } else if (i < nw + 3 * kHid + kN3 + 48) {                  // statistics
        const int e = i - nw - 3 * kHid - kN3;
        float v = 0.f;
        if (e < kIn) v = (float)stats[e];                                  // feature means
        else if (e >= 16 && e < 16 + kIn) v = (float)(1.0 / stats[10 + e - 16]);   // 1 / feature sd
        else if (e >= 32 && e < 32 + kOut) v = (float)stats[20 + e - 32];  // target means
        else if (e >= 40 && e < 40 + kOut) v = (float)stats[26 + e - 40];  // target sd
        reinterpret_cast<float *>(img + kImgStats)[e] = v;
    }
}
constexpr int kImgElems = kHid * kK0 + 2 * kHid * kHid + kN3 * kHid + 3 * kHid + kN3 + 48;

// ------------------------------------------------------------ the kernel --
// Slot g (warps 8g .. 8g+7) handles tiles g, g + 2 G, ... of CTA b's
// sequence 2 (b + k G) + g (G CTAs).  The two warps of a TMEM lane quadrant
// split the 128 columns of the epilogue.  Per tile: inputs -> MMA layer 0 ->
// (wait, epilogue, MMA) x 3 -> wait -> output; the next tile's features are
// fetched while the four layers run.  Every wait is bounded; on expiry the
// slot records EF_ERR_TIMEOUT and stops, and the CTA frees its TMEM.
constexpr int kSlotThreads = 256;

__device__ __forceinline__ void load_feats(const float *__restrict__ feats, long p, long n, float (&f)[kIn])
{
#pragma unroll
    for (int k = 0; k < kIn; k++) f[k] = p < n ? __ldg(feats + p * kIn + k) : 0.f;
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
    unsigned *tmem_holder = reinterpret_cast<unsigned *>(sm + kBarOff + 16);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + kBarOff + 24);
    if (tid == 0) {
        fz::mbar_init(&bar[0], 1);
        fz::mbar_init(&bar[1], 1);
        abort_flag[0] = 0;
        abort_flag[1] = 0;
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
    const unsigned dslot = tmem + kSlotCols * g;                  // this slot's accumulator (lane 0)
    const unsigned tlane = dslot + ((unsigned)(32 * quad) << 16);  // this warp's lanes
    const float *bias = reinterpret_cast<const float *>(sm + kImgBias);
    const float *st = reinterpret_cast<const float *>(sm + kImgStats);
    const bool issuer = (tid & (kSlotThreads - 1)) == 0;
    const int barid = 1 + g;
    const unsigned sImg = fz::smem_u32(sm);
    constexpr unsigned id128 = idesc_bf16(kRows, kHid), id16 = idesc_bf16(kRows, kN3);
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
    // the A operand written by every thread is complete before the MMA is issued
    auto operand_ready = [&]() {
        tmem_wait_st();
        tc_fence_before();
        slot_sync();
    };

    long t = g + 2L * blockIdx.x;
    float f[kIn];
    load_feats(feats, t * kRows + r, n, f);
    for (; t < ntiles; t += 2L * gridDim.x) {
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
            tmem_st4(tlane + kAhiCol + 4 * half, hv);
            tmem_st4(tlane + kAloCol + 4 * half, lv);
        }
        if (half == 0) {
            const unsigned ballot = __ballot_sync(0xffffffffu, out);
            if (lane == 0 && ballot) atomicAdd(nfall, __popc(ballot));
        }
        operand_ready();
        if (issuer) {
            tc_fence_after();
            const unsigned long long bw = sdesc(sImg + kImgW0, 128, kK0 * 16);
            mma_bf16_ts(dslot, dslot + kAhiCol, bw, id128, 0);
            mma_bf16_ts(dslot, dslot + kAloCol, bw, id128, 1);
            mma_commit(&bar[g]);
        }
        load_feats(feats, (t + 2L * gridDim.x) * kRows + r, n, f);   // the next tile's, in flight meanwhile
        bool ok = true;
        for (int l = 1; l < 4 && ok; l++) {
            ok = slot_wait();
            if (!ok) break;
            // epilogue of hidden layer l - 1: bias, SiLU, split into the next A operand
            const float2 *b2 = reinterpret_cast<const float2 *>(bias + (l - 1) * kHid);
#pragma unroll 1
            for (int cc = 0; cc < 2; cc++) {
                const int c = 2 * half + cc;
                unsigned v[32];
                tmem_ld32(tlane + 32 * c, v);
                unsigned hw[16], lw[16];
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const float2 z = __fadd2_rn(make_float2(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1])),
                                                b2[16 * c + j]);
                    split2(silu2(z), hw[j], lw[j]);
                }
                tmem_st16(tlane + kAhiCol + 16 * c, hw);
                tmem_st16(tlane + kAloCol + 16 * c, lw);
            }
            operand_ready();
            if (issuer) {
                tc_fence_after();
                const unsigned wbase = sImg + (l == 1 ? kImgW1 : l == 2 ? kImgW2 : kImgW3);
                const unsigned id = l == 3 ? id16 : id128;
#pragma unroll 1
                for (int ks = 0; ks < kHid / 16; ks++) {
                    const unsigned long long bw = sdesc(wbase + 256 * ks, 128, kHid * 16);
                    mma_bf16_ts(dslot, dslot + kAhiCol + 8 * ks, bw, id, ks > 0 ? 1u : 0u);
                    mma_bf16_ts(dslot, dslot + kAloCol + 8 * ks, bw, id, 1u);
                }
                mma_commit(&bar[g]);
            }
        }
        if (!ok || !slot_wait()) break;
        unsigned v[8];
        tmem_ld8(tlane, v);
        if (valid) {
            const bool fall = out && exact != nullptr;
#pragma unroll
            for (int qq = 0; qq < kOut; qq++) {
                if (qq / 3 != half) continue;
                const float y = __uint_as_float(v[qq]) + bias[3 * kHid + qq];
                tau[qq * n + p] = fall ? __ldg(exact + qq * n + p) : fmaf(st[40 + qq], y, st[32 + qq]);
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

}  // namespace

size_t closure_tc_image_bytes() { return kImgBytes; }

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
    const long want = (ntiles + 1) / 2;
    const int grid = (int)(want < nsm ? want : nsm);
    closure_mlp_tc_kernel<<<grid, kThreads, kSmemBytes, s>>>(static_cast<const uint4 *>(image), feats, n, ntiles, guard,
                                                       exact, tau, nfall, err);
    e = cudaGetLastError();
    return e == cudaSuccess ? EF_OK : cuda_fail(e, "closure_infer_tc");
}

}  // namespace eles
