// Fused x- and z-contraction of one (snapshot, y-plane) per CTA, FP32 on the
// CUDA cores.  One thread per z-row.
//
//  * reference profile: the first warps average row z = 0 of the plane for
//    u1, u2, u3 (FP64 sum); every thread forms u'_c = u_c - U_c in FP32.
//  * staging: the plane is streamed along x in stages of SB row blocks.  All
//    threads copy a stage with 16-byte cp.async pieces laid out along x, so
//    every warp request reads whole row segments (coalesced); in shared memory
//    piece p of row r lands in slot r ^ swz(p) of plane [c][p], so the per-row
//    reads below and the copies are both free of bank conflicts.  STG stages
//    are in flight.
//  * x phase: each thread streams its row in blocks of RX inputs (RX = nx /
//    nlx) with a ring of DX accumulators per field: input block b feeds the
//    outputs X = b + d, d in [dmin, dmax], with weight W[s][d - dmin]; the
//    slot of an output is a compile-time constant because the block loop is
//    unrolled by DX.  After block b the output X = b + dmin is
//    complete.  The nine fields u'_a and u'_a u'_b are formed in registers.
//  * z phase: every P completed columns are parked in shared memory; work
//    items (field, column, Z-range) stream a parked column along z with a ring
//    of DZ accumulators and write h[s][f][j][Z][X] for the Z outputs they own
//    (each Z exactly once, periodic wrap included).  Only h leaves the SM.
//  * the plane means <u_c>(y_j) come out of the same pass (FP64 reduction of
//    the per-thread FP32 row sums).
// Weights of both rings are kernel parameters (constant bank), indexed with
// compile-time offsets.
#include "eles_internal.h"
#include "fused_stage.cuh"

namespace eles {
namespace {

using namespace fz;

template <int RX, int DX, int RZ, int DZ>
__global__ void __launch_bounds__(kFusedMaxRows) xz_fused(const __grid_constant__ FusedArgs a)
{
    using S = Stg<RX>;
    constexpr int SB = S::SB;
    constexpr int U = DX;                     // unroll of the block loop (ring slots are static)
    extern __shared__ float4 smem_dyn[];
    float *colbuf = reinterpret_cast<float *>(smem_dyn);                        // [P][NF][nz + 1]
    float *stg = colbuf + (((size_t)a.P * NF * (a.nz + 1) + 3) & ~(size_t)3);     // [STG][3][NP][nz][4]
    const size_t stg_floats = (size_t)3 * S::NP * a.nz * 4;
    __shared__ double red[3][kFusedMaxRows / 32];
    __shared__ float Us[3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x;
    const int j = blockIdx.x, s = blockIdx.y;
    const int ld = a.nz + 1;
    const size_t np = (size_t)a.nx * a.ny * a.nz;
    const float *plane = a.u + (size_t)s * 3 * np + (size_t)j * a.nz * a.nx;

    auto stage_x = [&](int sidx) {
        int b = (sidx * SB - a.bshift) % a.nlx;
        if (b < 0) b += a.nlx;
        return b * RX;
    };
    const int nstage = a.nblk_x / SB;
    for (int k = 0; k < STG - 1; k++) {
        if (k < nstage) issue_stage<RX>(stg + k * stg_floats, plane, np, a.nz, a.nx, stage_x(k), tid, nthr);
        cp_commit();
    }

    for (int c = warp; c < 3; c += nthr / 32) {
        const float *r0 = plane + (size_t)c * np;
        double acc = 0.0;
        for (int i = lane; i < a.nx; i += 32) acc += (double)r0[i];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const float Uc = (float)(acc / a.nx);
            Us[c] = Uc;
            a.uref[((size_t)s * 3 + c) * a.ny + j] = (double)Uc;   // the exact value subtracted
        }
    }
    __syncthreads();
    const float U0 = Us[0], U1 = Us[1], U2 = Us[2];

    float acc[NF][DX];
#pragma unroll
    for (int k = 0; k < NF; k++)
#pragma unroll
        for (int d = 0; d < DX; d++) acc[k][d] = 0.f;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;

    for (int b0 = 0; b0 < a.nblk_x; b0 += U) {
#pragma unroll
        for (int uu = 0; uu < U; uu++) {
            const int bi = b0 + uu;
            if (bi < a.nblk_x) {
                const int sidx = bi / SB;
                const int lb = bi % SB;
                if (lb == 0) {                       // first block of a stage
                    cp_wait<STG - 2>();
                    __syncthreads();
                    const int sn = sidx + STG - 1;
                    if (sn < nstage)
                        issue_stage<RX>(stg + (sn % STG) * stg_floats, plane, np, a.nz, a.nx, stage_x(sn), tid, nthr);
                    cp_commit();
                }
                float cur[3][RX];
                const float *sbuf = stg + (sidx % STG) * stg_floats;
                if constexpr (SB == 1) read_block<RX, 0>(sbuf, a.nz, tid, cur);
                else if constexpr (SB == 2) {
                    if (lb == 0) read_block<RX, 0>(sbuf, a.nz, tid, cur);
                    else read_block<RX, SB == 2 ? 1 : 0>(sbuf, a.nz, tid, cur);
                } else {
                    static_assert(SB == 4, "stage blocks");
                    if (lb == 0) read_block<RX, 0>(sbuf, a.nz, tid, cur);
                    else if (lb == 1) read_block<RX, SB == 4 ? 1 : 0>(sbuf, a.nz, tid, cur);
                    else if (lb == 2) read_block<RX, SB == 4 ? 2 : 0>(sbuf, a.nz, tid, cur);
                    else read_block<RX, SB == 4 ? 3 : 0>(sbuf, a.nz, tid, cur);
                }
                const int b = bi - a.bshift;
                const bool own = b >= 0 && b < a.nlx;
#pragma unroll
                for (int e = 0; e < RX; e++) {
                    const float v0 = cur[0][e] - U0, v1 = cur[1][e] - U1, v2 = cur[2][e] - U2;
                    if (own) { s0 += v0; s1 += v1; s2 += v2; }
                    const float fv[NF] = {field<0>(v0, v1, v2), field<1>(v0, v1, v2), field<2>(v0, v1, v2),
                                          field<3>(v0, v1, v2), field<4>(v0, v1, v2), field<5>(v0, v1, v2),
                                          field<6>(v0, v1, v2), field<7>(v0, v1, v2), field<8>(v0, v1, v2)};
#pragma unroll
                    for (int dd = 0; dd < DX; dd++) {
                        const float w = a.WX[e * DX + dd];
#pragma unroll
                        for (int k = 0; k < NF; k++)
                            acc[k][(uu + dd) % DX] = fmaf(w, fv[k], acc[k][(uu + dd) % DX]);
                    }
                }
                const int X = b + a.dmin_x;
                if (X >= 0 && X < a.nlx) {
#pragma unroll
                    for (int k = 0; k < NF; k++) colbuf[((X & (a.P - 1)) * NF + k) * ld + tid] = acc[k][uu % DX];
                }
#pragma unroll
                for (int k = 0; k < NF; k++) acc[k][uu % DX] = 0.f;
                if (X >= 0 && X < a.nlx && ((X & (a.P - 1)) == a.P - 1 || X == a.nlx - 1)) {
                    __syncthreads();
                    // ---- z phase over the parked columns
                    zphase<RZ, DZ>(a, colbuf, ld, s, j, X & ~(a.P - 1), (X & (a.P - 1)) + 1, tid, nthr);
                    __syncthreads();
                }
            }
        }
    }
    cp_wait<0>();
    if (a.plane_mean) {
        double d0 = s0, d1 = s1, d2 = s2;
        for (int o = 16; o > 0; o >>= 1) {
            d0 += __shfl_xor_sync(0xffffffffu, d0, o);
            d1 += __shfl_xor_sync(0xffffffffu, d1, o);
            d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        }
        if (lane == 0) { red[0][warp] = d0; red[1][warp] = d1; red[2][warp] = d2; }
        __syncthreads();
        if (tid < 3) {
            double t = 0.0;
            for (int w = 0; w < nthr / 32; w++) t += red[tid][w];
            a.plane_mean[((size_t)s * 3 + tid) * a.ny + j] = (double)Us[tid] + t / ((double)a.nx * a.nz);
        }
    }
}

template <int RX>
size_t smem_bytes(int P, int nz)
{
    return sizeof(float) * ((((size_t)P * NF * (nz + 1) + 3) & ~(size_t)3) + (size_t)STG * 3 * Stg<RX>::NP * nz * 4);
}

template <int RX, int DX, int RZ, int DZ>
cudaError_t launch(const FusedArgs &a, int nsnap, cudaStream_t st)
{
    const size_t smem = smem_bytes<RX>(a.P, a.nz);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(xz_fused<RX, DX, RZ, DZ>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 222 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    xz_fused<RX, DX, RZ, DZ><<<dim3(a.ny, nsnap), a.nz, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Which (RX, DX, RZ, DZ) rings have a fused instantiation.
#define ELES_FUSED_LIST(X) \
    X(4, 4, 4, 6) X(4, 4, 4, 8) X(4, 6, 4, 8) X(4, 6, 4, 11) X(4, 8, 4, 11) X(4, 11, 4, 16) \
    X(6, 6, 6, 11) X(8, 4, 8, 8) X(8, 6, 8, 8) X(8, 11, 8, 16)

bool fused_supported(int rx, int dx, int rz, int dz)
{
#define ELES_CASE(A, B, C, D) if (rx == A && dx == B && rz == C && dz == D) return true;
    ELES_FUSED_LIST(ELES_CASE)
#undef ELES_CASE
    return false;
}

int fused_stage_blocks(int rx)
{
    return rx == 4 ? Stg<4>::SB : rx == 6 ? Stg<6>::SB : rx == 8 ? Stg<8>::SB : 0;
}

size_t fused_smem_bytes(int rx, int P, int nz)
{
    return rx == 4 ? smem_bytes<4>(P, nz) : rx == 6 ? smem_bytes<6>(P, nz) : rx == 8 ? smem_bytes<8>(P, nz) : 0;
}

cudaError_t launch_fused(int rx, int dx, int rz, int dz, const FusedArgs &a, int nsnap, cudaStream_t st)
{
#define ELES_CASE(A, B, C, D) if (rx == A && dx == B && rz == C && dz == D) return launch<A, B, C, D>(a, nsnap, st);
    ELES_FUSED_LIST(ELES_CASE)
#undef ELES_CASE
    return cudaErrorInvalidValue;
}

}  // namespace eles
