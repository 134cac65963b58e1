// Wall-normal contraction and the recovery of ~bar(u_a) and T_ab (Eq. 6).
//
// With h = A_z A_x f for the nine fields f about the reference profile U(y),
//   q_f   = A_y^{p_f} h_f                       (p_f: parity of field f, Eq. 7)
//   C_ab  = A_y^{p_a p_b} (U_a h_b)
//   ~bar(u_a) = A_y^{p_a} U_a + q_a
//   T_ab  = [A_y(U_a U_b) - A_y U_a A_y U_b] + [C_ab - A_y U_a q_b]
//         + [C_ba - A_y U_b q_a] + [q_ab - q_a q_b],
// every bracket a difference of nearly equal numbers, evaluated in FP64.
// The y-operators fold the wall extension: A_y^+ (even) and A_y^- (odd).
#include "eles_internal.h"

namespace eles {
namespace {

constexpr int YT = 128;

// Per (snapshot, LES row J), one CTA: A_y U_a, A_y (U_a U_b) in FP64 (block
// reduction) and the tap table wy[t] = (w+, w-, U1 w+, U1 w-, U2 w+, U2 w-,
// U3 w+, U3 w-) of row J, one thread per tap.
constexpr int YPT = 128;

template <typename T>
__global__ void __launch_bounds__(YPT) yprofile_kernel(const double *__restrict__ uref, const int *__restrict__ ystart,
                                                       const int *__restrict__ ycount, const double *__restrict__ we,
                                                       const double *__restrict__ wo, int ny, int nly, int flip,
                                                       double *AU, double *AUU, T *wy, float *Kab)
{
    const int J = blockIdx.x, s = blockIdx.y;
    const int pv[3] = {flip ? -1 : 1, flip ? 1 : -1, flip ? -1 : 1};
    const int PI[6] = {0, 0, 0, 1, 1, 2}, PJ[6] = {0, 1, 2, 1, 2, 2};
    const double *U = uref + (size_t)s * 3 * ny;
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int st = ystart[J], cnt = ycount[J];
    for (int t = threadIdx.x; t < cnt; t += YPT) {
        const int j = st + t;
        const double wev = we[(size_t)J * ny + j], wod = wo[(size_t)J * ny + j];
        const double u[3] = {U[j], U[ny + j], U[2 * ny + j]};
        for (int c = 0; c < 3; c++) acc[c] += (pv[c] > 0 ? wev : wod) * u[c];
        for (int k = 0; k < 6; k++) acc[3 + k] += (pv[PI[k]] * pv[PJ[k]] > 0 ? wev : wod) * u[PI[k]] * u[PJ[k]];
        if (wy) {   // the tap table of the CUDA-core y pass (not needed by the tensor-core one)
            T *o = wy + (((size_t)s * nly + J) * ny + t) * 8;
            o[0] = (T)wev; o[1] = (T)wod;
            for (int c = 0; c < 3; c++) { o[2 + 2 * c] = (T)(u[c] * wev); o[3 + 2 * c] = (T)(u[c] * wod); }
        }
    }
    __shared__ double part[9][YPT / 32];
    for (int k = 0; k < 9; k++) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) part[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    __shared__ double tot[9];
    if (threadIdx.x < 9) {
        const int k = threadIdx.x;
        double v = 0.0;
        for (int w = 0; w < YPT / 32; w++) v += part[k][w];
        tot[k] = v;
        if (k < 3) AU[((size_t)s * 3 + k) * nly + J] = v;
        else AUU[((size_t)s * 6 + (k - 3)) * nly + J] = v;
    }
    // the profile bracket of T_ab, A_y(U_a U_b) - A_y U_a A_y U_b: cancels
    // ~U^2 to O(1), so it is formed here in FP64 (once per row)
    __syncthreads();
    if (Kab && threadIdx.x >= 3 && threadIdx.x < 9) {
        const int k = threadIdx.x - 3;
        Kab[((size_t)s * 6 + k) * nly + J] = (float)(tot[3 + k] - tot[PI[k]] * tot[PJ[k]]);
    }
}

// Parity index (0 even, 1 odd) of the product of components a and b.
__host__ __device__ constexpr int podd(int a, int b) { return ((a == 1) != (b == 1)) ? 1 : 0; }

// The eight tap weights of one (row, tap) as vector loads (broadcast).
__device__ __forceinline__ void load8(const float *p, float (&w)[8])
{
    const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
}
__device__ __forceinline__ void load8(const double *p, double (&w)[8])
{
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const double2 v = reinterpret_cast<const double2 *>(p)[i];
        w[2 * i] = v.x; w[2 * i + 1] = v.y;
    }
}

// One thread per (snapshot, block of JB LES rows, Z, X).  The rows of a block
// share most of their taps, so each h(j) is loaded once per block and feeds
// the JB rows whose support contains j.  The CTA shares (s, row block): its
// tap tables are staged in shared memory and read as broadcasts.  The work is
// split in two passes to keep the accumulators few:
//   pass 0: velocity fields -> q_a, C_ab; writes ~bar(u_a) and (q_a, C_ab) to
//           a scratch table;
//   pass 1: product fields -> q_ab; reads the table and writes T_ab.
template <typename T, int JB, int PASS>
__global__ void __launch_bounds__(YT) ypass_kernel(const __grid_constant__ YArgs<T> a)
{
    constexpr int NFP = PASS == 0 ? 3 : 6;     // fields of this pass
    constexpr int F0 = PASS == 0 ? 0 : 3;
    constexpr int NC = PASS == 0 ? 9 : 0;      // cross terms of this pass
    extern __shared__ unsigned char ysm[];
    T *tw = reinterpret_cast<T *>(ysm);        // [JB][ny][8]
    const int J0 = blockIdx.y * JB, s = blockIdx.z;
    int st[JB], en[JB];
    int jlo = a.ny, jhi = 0;
#pragma unroll
    for (int b = 0; b < JB; b++) {
        const int J = J0 + b;
        st[b] = J < a.nly ? a.ystart[J] : a.ny;
        en[b] = J < a.nly ? a.ystart[J] + a.ycount[J] : 0;
        if (J < a.nly) { jlo = min(jlo, st[b]); jhi = max(jhi, en[b]); }
    }
#pragma unroll
    for (int b = 0; b < JB; b++) {
        if (J0 + b >= a.nly) break;
        const T *src = a.wy + ((size_t)s * a.nly + J0 + b) * a.ny * 8;
        for (int i = threadIdx.x; i < (en[b] - st[b]) * 8; i += YT) tw[(size_t)b * a.ny * 8 + i] = src[i];
    }
    __syncthreads();
    const int nplane = a.nlz * a.nlx;
    const int p0 = blockIdx.x * YT + threadIdx.x;
    if (p0 >= nplane) return;
    const bool cross = PASS == 0 && a.stress;
    // weight slot of each field: velocities Eq. 7 (+,-,+) or Eq. 9 (-,+,-);
    // products 11, 12, 13, 22, 23, 33: +, -, +, +, -, +
    int wsl[NFP];
#pragma unroll
    for (int f = 0; f < NFP; f++) {
        if constexpr (PASS == 0) wsl[f] = (f == 1) != (a.flip != 0) ? 1 : 0;
        else wsl[f] = (f == 1 || f == 4) ? 1 : 0;
    }
    T q[JB][NFP], C[JB][NC > 0 ? NC : 1];
#pragma unroll
    for (int b = 0; b < JB; b++) {
#pragma unroll
        for (int f = 0; f < NFP; f++) q[b][f] = T(0);
#pragma unroll
        for (int c = 0; c < (NC > 0 ? NC : 1); c++) C[b][c] = T(0);
    }
    const size_t fstride = (size_t)a.ny * nplane;
    const T *hp = a.h + (size_t)s * 9 * fstride + (size_t)F0 * fstride + p0;
    T hn[NFP];
#pragma unroll
    for (int f = 0; f < NFP; f++) hn[f] = jlo < jhi ? __ldg(hp + f * fstride + (size_t)jlo * nplane) : T(0);
    for (int j = jlo; j < jhi; j++) {
        T hv[NFP];
#pragma unroll
        for (int f = 0; f < NFP; f++) hv[f] = hn[f];
        if (j + 1 < jhi) {
#pragma unroll
            for (int f = 0; f < NFP; f++) hn[f] = __ldg(hp + f * fstride + (size_t)(j + 1) * nplane);
        }
#pragma unroll
        for (int b = 0; b < JB; b++) {
            if (j < st[b] || j >= en[b]) continue;
            T w[8];
            load8(tw + ((size_t)b * a.ny + (j - st[b])) * 8, w);
#pragma unroll
            for (int f = 0; f < NFP; f++) q[b][f] = fma(wsl[f] ? w[1] : w[0], hv[f], q[b][f]);
            if constexpr (NC > 0) {
                if (cross) {
#pragma unroll
                    for (int i = 0; i < 3; i++)
#pragma unroll
                        for (int k = 0; k < 3; k++) C[b][3 * i + k] = fma(w[2 + 2 * i + podd(i, k)], hv[k], C[b][3 * i + k]);
                }
            }
        }
    }
    const size_t nl = (size_t)a.nly * nplane;
    const double *AU = a.AU + (size_t)s * 3 * a.nly;
    const double *AUU = a.AUU + (size_t)s * 6 * a.nly;
    bool bad = false;
#pragma unroll
    for (int b = 0; b < JB; b++) {
        const int J = J0 + b;
        if (J >= a.nly) break;
        const size_t o0 = (size_t)J * nplane + p0;
        // outputs in (Z, X) order; h planes, and the scratch, in h's order
        const size_t oo = (size_t)J * nplane + (a.ptrans ? (size_t)(p0 % a.nlz) * a.nlx + p0 / a.nlz : (size_t)p0);
        T *tmp = a.tmp + (size_t)s * 12 * nl + o0;
        if constexpr (PASS == 0) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const double v = AU[c * a.nly + J] + (double)q[b][c];
                bad |= !isfinite(v);
                if (in_range(((size_t)s * 3 + c) * nl + oo, (size_t)gridDim.z * 3 * nl, a.err))
                    a.ubar[((size_t)s * 3 + c) * nl + oo] = (T)v;
            }
            if (cross) {
#pragma unroll
                for (int c = 0; c < 3; c++) tmp[c * nl] = q[b][c];
#pragma unroll
                for (int c = 0; c < 9; c++) tmp[(3 + c) * nl] = C[b][c];
            }
        } else {
            const int PI[6] = {0, 0, 0, 1, 1, 2}, PJ[6] = {0, 1, 2, 1, 2, 2};
            double qv[3];
#pragma unroll
            for (int c = 0; c < 3; c++) qv[c] = (double)tmp[c * nl];
#pragma unroll
            for (int k = 0; k < 6; k++) {
                const int i = PI[k], m = PJ[k];
                const double Ai = AU[i * a.nly + J], Am = AU[m * a.nly + J];
                const double Cim = (double)tmp[(3 + 3 * i + m) * nl], Cmi = (double)tmp[(3 + 3 * m + i) * nl];
                const double v = (AUU[k * a.nly + J] - Ai * Am) + (Cim - Ai * qv[m])
                               + (Cmi - Am * qv[i]) + ((double)q[b][k] - qv[i] * qv[m]);
                bad |= !isfinite(v);
                if (in_range(((size_t)s * 6 + k) * nl + oo, (size_t)gridDim.z * 6 * nl, a.err))
                    a.tau[((size_t)s * 6 + k) * nl + oo] = (T)v;
            }
        }
    }
    if (bad && a.err) atomicCAS(a.err, 0, (int)EF_ERR_NAN);
}

}  // namespace

template <typename T>
cudaError_t launch_yprofile(const double *uref, const int *ystart, const int *ycount, const double *we,
                            const double *wo, int ny, int nly, int flip, int nsnap, double *AU, double *AUU,
                            T *wy, float *Kab, cudaStream_t st)
{
    yprofile_kernel<T><<<dim3(nly, nsnap), YPT, 0, st>>>(uref, ystart, ycount, we, wo, ny, nly, flip, AU, AUU, wy,
                                                         Kab);
    return cudaGetLastError();
}

template <typename T, int JB, int PASS>
cudaError_t launch_pass(const YArgs<T> &a, int nsnap, cudaStream_t st)
{
    const int nplane = a.nlz * a.nlx;
    const size_t smem = sizeof(T) * 8 * (size_t)JB * a.ny;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(ypass_kernel<T, JB, PASS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             96 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 g((nplane + YT - 1) / YT, (a.nly + JB - 1) / JB, nsnap);
    ypass_kernel<T, JB, PASS><<<g, YT, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ypass(const YArgs<T> &a, int nsnap, cudaStream_t st)
{
    constexpr int JB = sizeof(T) == 4 ? 4 : 2;
    cudaError_t e = launch_pass<T, JB, 0>(a, nsnap, st);
    if (e != cudaSuccess || !a.stress) return e;
    return launch_pass<T, JB, 1>(a, nsnap, st);
}

template cudaError_t launch_yprofile<float>(const double *, const int *, const int *, const double *,
                                            const double *, int, int, int, int, double *, double *, float *,
                                            float *, cudaStream_t);
template cudaError_t launch_yprofile<double>(const double *, const int *, const int *, const double *,
                                             const double *, int, int, int, int, double *, double *, double *,
                                             float *, cudaStream_t);
template cudaError_t launch_ypass<float>(const YArgs<float> &, int, cudaStream_t);
template cudaError_t launch_ypass<double>(const YArgs<double> &, int, cudaStream_t);

}  // namespace eles
