// Shared pieces of the fused x-z kernels (CUDA-core and tensor-core x
// contraction): the coalesced cp.async staging of a y-plane, and the
// z-contraction of parked output columns.
#pragma once

#include <cuda.h>

#include "eles_internal.h"

namespace eles {
namespace fz {

constexpr int NF = 9;     // fields
constexpr int STG = 2;    // stages in flight

template <int F>
__device__ __forceinline__ float field(float v0, float v1, float v2)
{
    return F == 0 ? v0 : F == 1 ? v1 : F == 2 ? v2 : F == 3 ? v0 * v0 : F == 4 ? v0 * v1
         : F == 5 ? v0 * v2 : F == 6 ? v1 * v1 : F == 7 ? v1 * v2 : v2 * v2;
}

// Blocks per stage: 16 floats (64 bytes) of every row per component, or 12
// for a stride of 6.
template <int RX>
struct Stg {
    static constexpr int SB = RX % 4 == 0 ? 16 / RX : 2;
    static constexpr int W = SB * RX;         // floats per row per component
    static constexpr int NP = W / 4;          // 16-byte pieces per row per component
    static_assert(W % 4 == 0, "stage width must be whole 16-byte pieces");
};

__host__ __device__ constexpr int swz(int p) { return (2 * p) & 7; }

__device__ __forceinline__ void cp16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Copy stage `sidx` of the whole plane: 3 components x nz rows x NP pieces,
// piece index fastest.
template <int RX>
__device__ __forceinline__ void issue_stage(float *buf, const float *plane, size_t np, int nz, int nx,
                                            int xstart, int tid, int nthr)
{
    using S = Stg<RX>;
    // nthr == nz: each thread copies NP pieces per component (compile-time
    // divisions only)
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int m = 0; m < S::NP; m++) {
            const int q = tid + m * nthr;
            const int p = q % S::NP, r = q / S::NP;
            cp16(buf + ((size_t)(c * S::NP + p) * nz + (r ^ swz(p))) * 4,
                 plane + c * np + (size_t)r * nx + xstart + 4 * p);
        }
}

// Row t's RX inputs of local block LB (0 <= LB < SB) of a staged buffer.
template <int RX, int LB>
__device__ __forceinline__ void read_block(const float *buf, int nz, int t, float (&x)[3][RX])
{
    using S = Stg<RX>;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if constexpr (RX % 4 == 0) {
#pragma unroll
            for (int q = 0; q < RX / 4; q++) {
                const int p = LB * RX / 4 + q;
                const float4 v = *reinterpret_cast<const float4 *>(buf + ((size_t)(c * S::NP + p) * nz + (t ^ swz(p))) * 4);
                x[c][4 * q] = v.x; x[c][4 * q + 1] = v.y; x[c][4 * q + 2] = v.z; x[c][4 * q + 3] = v.w;
            }
        } else {   // RX == 6, SB == 2: floats 0..5 or 6..11 of the 12
            static_assert(RX == 6, "unsupported stride");
            constexpr int pa = LB == 0 ? 0 : 1, pb = LB == 0 ? 1 : 2;
            const float4 va = *reinterpret_cast<const float4 *>(buf + ((size_t)(c * S::NP + pa) * nz + (t ^ swz(pa))) * 4);
            const float4 vb = *reinterpret_cast<const float4 *>(buf + ((size_t)(c * S::NP + pb) * nz + (t ^ swz(pb))) * 4);
            if constexpr (LB == 0) {
                x[c][0] = va.x; x[c][1] = va.y; x[c][2] = va.z; x[c][3] = va.w; x[c][4] = vb.x; x[c][5] = vb.y;
            } else {
                x[c][0] = va.z; x[c][1] = va.w; x[c][2] = vb.x; x[c][3] = vb.y; x[c][4] = vb.z; x[c][5] = vb.w;
            }
        }
    }
}


// z phase over the parked columns Xs .. Xs + cnt - 1 of plane (s, j): work
// items (field, column, Z-range) stream one parked column along z with a ring
// of DZ accumulators (weights WZ[e][dd] as kernel parameters) and write the Z
// outputs they own, each exactly once (periodic wrap included).
template <int RZ, int DZ>
__device__ __forceinline__ void zphase(const FusedArgs &a, const float *colbuf, int ld, int s, int j, int Xs, int cnt,
                                       int tid, int nthr)
{
    const int nitems = a.nf * a.P * a.NQ;
    for (int it = tid; it < nitems; it += nthr) {
        const int xo = it & (a.P - 1), fq = it >> a.lP;
        const int q = fq / a.nf, f = fq - q * a.nf;
        if (xo >= cnt) continue;
        const float *col = colbuf + (xo * NF + f) * ld;
        const int Zs = q * a.ZQs;
        const int nbz = a.ZQs + DZ - 1;
        float *hout = a.h + ((((size_t)s * NF + f) * a.ny + j) * a.nlz + Zs) * a.nlx + Xs + xo;
        float zacc[DZ];
#pragma unroll
        for (int d = 0; d < DZ; d++) zacc[d] = 0.f;
        for (int c0 = 0; c0 < nbz; c0 += DZ) {
#pragma unroll
            for (int uz = 0; uz < DZ; uz++) {
                const int bz = c0 + uz;
                if (bz < nbz) {
                    int bb = Zs - a.dmax_z + bz;
                    bb = bb < 0 ? bb + a.nlz : (bb >= a.nlz ? bb - a.nlz : bb);
                    float v[RZ];
#pragma unroll
                    for (int e = 0; e < RZ; e++) v[e] = col[bb * RZ + e];
#pragma unroll
                    for (int e = 0; e < RZ; e++)
#pragma unroll
                        for (int dd = 0; dd < DZ; dd++)
                            zacc[(uz + dd) % DZ] = fmaf(a.WZ[e * DZ + dd], v[e], zacc[(uz + dd) % DZ]);
                    const int Zo = bz - (DZ - 1);
                    if (Zo >= 0) hout[(size_t)Zo * a.nlx] = zacc[uz];
                    zacc[uz] = 0.f;
                }
            }
        }
    }
}

}  // namespace fz
}  // namespace eles

// ---------------------------------------------------------------------------
// TMA staging (cp.async.bulk.tensor) of a y-plane: stages of W = 8 floats
// (32 bytes) of every row, one box per component and row half, completion on
// an mbarrier per stage.  Every wait is bounded: on expiry the kernel records
// EF_ERR_TIMEOUT and carries on (the results are then garbage, but nothing
// hangs).  A stage whose wait ran out may still be landing afterwards: the
// kernels that use these stages wait once more, with the same bound, for every
// stage they issued before the CTA exits, so no bulk copy outlives its CTA
// unless it never completes at all.
namespace eles {
namespace fz {

constexpr int TW = 8;            // floats per row per stage
constexpr int TSTG = 4;          // stages in flight
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at the SM clock: the bound of one wait
constexpr unsigned kSuspendNs = 100000;              // suspend-time hint of one try_wait (the thread
                                                     // wakes as soon as the phase completes)

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
                 : "memory");
    return ok != 0;
}
// Non-blocking test of a phase (no suspend).
__device__ __forceinline__ bool mbar_test_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Bounded wait of at most `limit` SM clocks; returns false (and flags the
// plan) if the phase never completed.
__device__ __forceinline__ bool mbar_wait_for(unsigned long long *bar, unsigned parity, int *err, long long limit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (clock64() - t0 < limit)
        if (mbar_try_wait(bar, parity)) return true;
    if (err) atomicCAS(err, 0, (int)EF_ERR_TIMEOUT);
    return false;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int *err)
{
    return mbar_wait_for(bar, parity, err, kWaitCycles);
}
__device__ __forceinline__ void tma_load3(void *dst, const CUtensorMap *map, unsigned long long *bar, int x, int y, int z)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];\n"
                 ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}

// Issue stage `sidx` into buffer `buf` (thread 0 only): 3 components x
// (nz / box rows) boxes of TW floats starting at column xstart.
__device__ __forceinline__ void tma_stage(float *buf, unsigned long long *bar, const CUtensorMap *map, int nz,
                                          int box_rows, int xstart, int pc0, int ny)
{
    mbar_expect_tx(bar, 3u * nz * TW * 4u);
    for (int c = 0; c < 3; c++)
        for (int r0 = 0; r0 < nz; r0 += box_rows)
            tma_load3(buf + ((size_t)c * nz + r0) * TW, map, bar, xstart, r0, pc0 + c * ny);
}

}  // namespace fz
}  // namespace eles
