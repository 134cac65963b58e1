// Hot path: the four steps of Sec. 2.1 on a channel snapshot, as separable
// contractions on the CUDA cores.
//
//   1. reference profile U_c(y_j): mean of one z-row per plane (FP64);
//   2. x-contraction A_x of the nine fields about that profile,
//        f = {u'_1, u'_2, u'_3, u'_1u'_1, u'_1u'_2, u'_1u'_3, u'_2u'_2, u'_2u'_3, u'_3u'_3},
//      u'_c = u_c - U_c(y); the fields are formed in registers and never stored;
//   3. z-contraction A_z;
//   4. y-contraction with the wall extension of Eq. 7 folded into the even and
//      odd operators A_y^+, A_y^-, plus the cross terms A_y(U_a h_b), and the
//      recovery of ~bar(u_a) and T_ab (Eq. 6) in FP64.
//
// The recovery uses the identity, exact because A_x and A_z reproduce any
// function of y alone (their rows sum to one) and every operator is linear:
//   A(u_a u_b) = A_y(U_a U_b) + A_y(U_a h_b) + A_y(U_b h_a) + A_y(h_ab),
//   A(u_a)     = A_y U_a + A_y h_a,
// with h = A_z A_x f.  Only fluctuation-sized numbers meet the working
// precision; the large mean-flow terms are FP64.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "eles_internal.h"

namespace eles {
namespace {

constexpr int XT = 128;   // threads (z-rows) per CTA of the x-contraction
constexpr int ZT = 128;
constexpr int YT = 128;

__device__ __forceinline__ void flag_error(int *err, int code)
{
    if (err) atomicCAS(err, 0, code);
}

// ----------------------------------------------------------------- step 1 --
// U_c(y_j) = mean over x of u_c at (j, z = 0).  One CTA per (j, c).
template <typename T>
__global__ void uref_kernel(const T *__restrict__ u, int nx, int ny, int nz, double *uref, T *urefT)
{
    int j = blockIdx.x, c = blockIdx.y;
    const T *row = u + (((size_t)c * ny + j) * nz) * nx;
    double s = 0.0;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) s += (double)row[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
        t /= nx;
        const T tt = (T)t;             // the value subtracted is the one the recovery uses
        uref[c * ny + j] = (double)tt;
        urefT[c * ny + j] = tt;
    }
}

// The nine fields of step 1 about the reference profile, F0..F0+NF-1.
template <typename T, int F0, int NF>
__device__ __forceinline__ void make_fields(T v0, T v1, T v2, T (&fv)[NF])
{
#pragma unroll
    for (int k = 0; k < NF; k++) {
        const int f = F0 + k;
        fv[k] = f == 0 ? v0 : f == 1 ? v1 : f == 2 ? v2 : f == 3 ? v0 * v0 : f == 4 ? v0 * v1
              : f == 5 ? v0 * v2 : f == 6 ? v1 * v1 : f == 7 ? v1 * v2 : v2 * v2;
    }
}

template <typename T, int R>
__device__ __forceinline__ void load_run(const T *__restrict__ p, T (&v)[R])
{
    if constexpr ((R * sizeof(T)) % 16 == 0) {
        constexpr int E = 16 / sizeof(T);
#pragma unroll
        for (int q = 0; q < R / E; q++) {
            float4 t = __ldg(reinterpret_cast<const float4 *>(p) + q);
            const T *tt = reinterpret_cast<const T *>(&t);
#pragma unroll
            for (int e = 0; e < E; e++) v[q * E + e] = tt[e];
        }
    } else if constexpr ((R * sizeof(T)) % 8 == 0) {
        constexpr int E = 8 / sizeof(T);
#pragma unroll
        for (int q = 0; q < R / E; q++) {
            float2 t = __ldg(reinterpret_cast<const float2 *>(p) + q);
            const T *tt = reinterpret_cast<const T *>(&t);
#pragma unroll
            for (int e = 0; e < E; e++) v[q * E + e] = tt[e];
        }
    } else {
#pragma unroll
        for (int s = 0; s < R; s++) v[s] = __ldg(p + s);
    }
}

// ----------------------------------------------------------------- step 2 --
template <typename T>
struct XArgs {
    const T *u;
    const T *uref;
    T *g;                 // [9][ny][nz][nlx]
    double *rowsum;       // [3][ny][nzw] or nullptr
    int nx, ny, nz, nlx, nzw;
    int nblk;             // nlx + D - 1 blocks of r inputs per row
    int dmax;
    T W[kMaxStride * kMaxRing];
};

// One thread streams one z-row of plane j along x in blocks of R inputs
// (R = nx / nlx).  Input block b feeds outputs X = b + d, d in [dmin, dmax],
// with weight W[s][d - dmin]; their accumulators live in a ring of D
// registers per field whose slot indices are compile-time constants because
// the block loop is unrolled by D.  After block b the output X = b + dmin is
// complete; completed columns are staged in shared memory and written out
// P at a time as 32-byte runs of g[f][j][z][X].
template <typename T, int R, int D, int F0, int NF>
__global__ void __launch_bounds__(XT) xpass_ring(const __grid_constant__ XArgs<T> a)
{
    constexpr int P = 32 / sizeof(T);
    __shared__ T colbuf[P][NF][XT + 1];
    const int tid = threadIdx.x;
    const int z = blockIdx.x * XT + tid;
    const int j = blockIdx.y;
    const bool act = z < a.nz;
    const size_t np = (size_t)a.nx * a.ny * a.nz;
    const T *row = a.u + ((size_t)j * a.nz + (act ? z : 0)) * a.nx;
    const T U0 = a.uref[j], U1 = a.uref[a.ny + j], U2 = a.uref[2 * a.ny + j];
    T acc[NF][D];
#pragma unroll
    for (int k = 0; k < NF; k++)
#pragma unroll
        for (int d = 0; d < D; d++) acc[k][d] = T(0);
    T s0 = T(0), s1 = T(0), s2 = T(0);
    const bool sums = (a.rowsum != nullptr);

    for (int b0 = 0; b0 < a.nblk; b0 += D) {
#pragma unroll
        for (int uu = 0; uu < D; uu++) {
            const int bi = b0 + uu;
            if (bi < a.nblk) {
                const int b = bi - a.dmax;
                const int bw = b < 0 ? b + a.nlx : (b >= a.nlx ? b - a.nlx : b);
                T x0[R], x1[R], x2[R];
                load_run<T, R>(row + (size_t)bw * R, x0);
                load_run<T, R>(row + np + (size_t)bw * R, x1);
                load_run<T, R>(row + 2 * np + (size_t)bw * R, x2);
                const bool own = sums && b >= 0 && b < a.nlx;
#pragma unroll
                for (int s = 0; s < R; s++) {
                    const T v0 = x0[s] - U0, v1 = x1[s] - U1, v2 = x2[s] - U2;
                    if (own) { s0 += v0; s1 += v1; s2 += v2; }
                    T fv[NF];
                    make_fields<T, F0, NF>(v0, v1, v2, fv);
#pragma unroll
                    for (int dd = 0; dd < D; dd++) {
                        const T w = a.W[s * D + dd];
#pragma unroll
                        for (int k = 0; k < NF; k++)
                            acc[k][(uu + dd) % D] = fma(w, fv[k], acc[k][(uu + dd) % D]);
                    }
                }
                const int X = bi - (D - 1);
                if (X >= 0) {
#pragma unroll
                    for (int k = 0; k < NF; k++) colbuf[X % P][k][tid] = acc[k][uu];
                }
#pragma unroll
                for (int k = 0; k < NF; k++) acc[k][uu] = T(0);
                if (X >= 0 && ((X % P) == P - 1 || X == a.nlx - 1)) {
                    __syncthreads();
                    const int Xs = X - X % P, cnt = X % P + 1;
                    for (int e = tid; e < NF * XT * P; e += XT) {
                        const int xo = e % P, zl = (e / P) % XT, k = e / (P * XT);
                        const int zg = blockIdx.x * XT + zl;
                        if (xo < cnt && zg < a.nz)
                            a.g[(((size_t)(F0 + k) * a.ny + j) * a.nz + zg) * a.nlx + Xs + xo] = colbuf[xo][k][zl];
                    }
                    __syncthreads();
                }
            }
        }
    }
    if (sums) {
        double d0 = act ? (double)s0 : 0.0, d1 = act ? (double)s1 : 0.0, d2 = act ? (double)s2 : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            d0 += __shfl_xor_sync(0xffffffffu, d0, o);
            d1 += __shfl_xor_sync(0xffffffffu, d1, o);
            d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        }
        if ((tid & 31) == 0) {
            const int w = (blockIdx.x * XT + tid) >> 5;
            if (w < a.nzw) {
                a.rowsum[((size_t)0 * a.ny + j) * a.nzw + w] = d0;
                a.rowsum[((size_t)1 * a.ny + j) * a.nzw + w] = d1;
                a.rowsum[((size_t)2 * a.ny + j) * a.nzw + w] = d2;
            }
        }
    }
}

// Generic banded x-contraction (any DNS/LES ratio): one thread per output.
template <typename T, int NF>
__global__ void xpass_gather(const T *__restrict__ u, const T *__restrict__ uref, T *__restrict__ g,
                             const int *__restrict__ start, const T *__restrict__ w, int taps,
                             int nx, int ny, int nz, int nlx)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)ny * nz * nlx;
    if (idx >= total) return;
    const int X = (int)(idx % nlx);
    const int z = (int)((idx / nlx) % nz);
    const int j = (int)(idx / ((size_t)nlx * nz));
    const size_t np = (size_t)nx * ny * nz;
    const T *row = u + ((size_t)j * nz + z) * nx;
    const T U0 = uref[j], U1 = uref[ny + j], U2 = uref[2 * ny + j];
    T acc[NF];
#pragma unroll
    for (int k = 0; k < NF; k++) acc[k] = T(0);
    int c = start[X];
    for (int t = 0; t < taps; t++, c = (c + 1 == nx) ? 0 : c + 1) {
        const T wt = w[(size_t)X * taps + t];
        const T v0 = row[c] - U0, v1 = row[np + c] - U1, v2 = row[2 * np + c] - U2;
        T fv[NF];
        make_fields<T, 0, NF>(v0, v1, v2, fv);
#pragma unroll
        for (int k = 0; k < NF; k++) acc[k] = fma(wt, fv[k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < NF; k++) g[(((size_t)k * ny + j) * nz + z) * nlx + X] = acc[k];
}

// ----------------------------------------------------------------- step 3 --
template <typename T>
struct ZArgs {
    const T *g;
    T *h;                 // [nf][ny][nlz][nlx]
    int nf, ny, nz, nlz, nlx;
    int nblk, dmax;
    T W[kMaxStride * kMaxRing];
};

// One thread per column (f, j, X) streams z with the same ring scheme as the
// x-contraction; lanes run along X, so every load and store is coalesced.
template <typename T, int R, int D>
__global__ void __launch_bounds__(ZT) zpass_ring(const __grid_constant__ ZArgs<T> a)
{
    const size_t idx = (size_t)blockIdx.x * ZT + threadIdx.x;
    const size_t total = (size_t)a.nf * a.ny * a.nlx;
    if (idx >= total) return;
    const int X = (int)(idx % a.nlx);
    const size_t fj = idx / a.nlx;
    const T *col = a.g + fj * a.nz * a.nlx + X;
    T *out = a.h + fj * a.nlz * a.nlx + X;
    T acc[D];
#pragma unroll
    for (int d = 0; d < D; d++) acc[d] = T(0);
    for (int b0 = 0; b0 < a.nblk; b0 += D) {
#pragma unroll
        for (int uu = 0; uu < D; uu++) {
            const int bi = b0 + uu;
            if (bi < a.nblk) {
                const int b = bi - a.dmax;
                const int bw = b < 0 ? b + a.nlz : (b >= a.nlz ? b - a.nlz : b);
                T v[R];
#pragma unroll
                for (int s = 0; s < R; s++) v[s] = __ldg(col + (size_t)(bw * R + s) * a.nlx);
#pragma unroll
                for (int s = 0; s < R; s++)
#pragma unroll
                    for (int dd = 0; dd < D; dd++)
                        acc[(uu + dd) % D] = fma(a.W[s * D + dd], v[s], acc[(uu + dd) % D]);
                const int Z = bi - (D - 1);
                if (Z >= 0) out[(size_t)Z * a.nlx] = acc[uu];
                acc[uu] = T(0);
            }
        }
    }
}

template <typename T>
__global__ void zpass_gather(const T *__restrict__ g, T *__restrict__ h, const int *__restrict__ start,
                             const T *__restrict__ w, int taps, int nf, int ny, int nz, int nlz, int nlx)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)nf * ny * nlz * nlx;
    if (idx >= total) return;
    const int X = (int)(idx % nlx);
    const int Z = (int)((idx / nlx) % nlz);
    const size_t fj = idx / ((size_t)nlx * nlz);
    const T *col = g + fj * nz * nlx + X;
    T acc = T(0);
    int c = start[Z];
    for (int t = 0; t < taps; t++, c = (c + 1 == nz) ? 0 : c + 1)
        acc = fma(w[(size_t)Z * taps + t], col[(size_t)c * nlx], acc);
    h[(fj * nlz + Z) * nlx + X] = acc;
}

// Plane means by a plain reduction (unfused path).
template <typename T>
__global__ void plane_mean_direct(const T *__restrict__ u, const double *uref, int nx, int ny, int nz, double *out)
{
    int j = blockIdx.x, c = blockIdx.y;
    const T *pl = u + (((size_t)c * ny + j) * nz) * nx;
    const double U = uref[c * ny + j];
    double s = 0.0;
    for (size_t i = threadIdx.x; i < (size_t)nx * nz; i += blockDim.x) s += (double)pl[i] - U;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
        out[c * ny + j] = U + t / ((double)nx * nz);
    }
}

// --------------------------------------------------------------- dispatch --
template <typename T>
const T *band_w(const Band &b);
template <>
const float *band_w<float>(const Band &b) { return b.d_w32; }
template <>
const double *band_w<double>(const Band &b) { return b.d_w64; }

template <typename T>
const T *ring_W(const Ring &r);
template <>
const float *ring_W<float>(const Ring &r) { return r.W32; }
template <>
const double *ring_W<double>(const Ring &r) { return r.W64; }

template <typename T, int R, int D, int F0, int NF>
void launch_x(const XArgs<T> &a, int ny, int nz, cudaStream_t s)
{
    dim3 grid((nz + XT - 1) / XT, ny);
    xpass_ring<T, R, D, F0, NF><<<grid, XT, 0, s>>>(a);
}

// Field grouping: all nine fields in one pass while the ring is short, three
// passes of three fields when it is long (register budget).
template <typename T, int R, int D>
void launch_x_all(XArgs<T> a, int nfields, int ny, int nz, cudaStream_t s)
{
    constexpr bool one_pass = (D * 9 * sizeof(T) <= 8 * 9 * 4);
    if (nfields == 3) { launch_x<T, R, D, 0, 3>(a, ny, nz, s); return; }
    if constexpr (one_pass) {
        launch_x<T, R, D, 0, 9>(a, ny, nz, s);
    } else {
        launch_x<T, R, D, 0, 3>(a, ny, nz, s);
        a.rowsum = nullptr;
        launch_x<T, R, D, 3, 3>(a, ny, nz, s);
        launch_x<T, R, D, 6, 3>(a, ny, nz, s);
    }
}

template <typename T>
bool dispatch_x(const Ring &rg, XArgs<T> &a, int nfields, int ny, int nz, cudaStream_t s)
{
#define ELES_X(RR, DD) \
    if (rg.r == RR && rg.D == DD) { launch_x_all<T, RR, DD>(a, nfields, ny, nz, s); return true; }
    ELES_X(4, 4) ELES_X(4, 6) ELES_X(4, 8) ELES_X(4, 10) ELES_X(4, 11)
    ELES_X(6, 6) ELES_X(8, 6) ELES_X(8, 10) ELES_X(8, 11)
#undef ELES_X
    return false;
}

template <typename T>
bool dispatch_z(const Ring &rg, const ZArgs<T> &a, cudaStream_t s)
{
    const size_t total = (size_t)a.nf * a.ny * a.nlx;
    const unsigned grid = (unsigned)((total + ZT - 1) / ZT);
#define ELES_Z(RR, DD) \
    if (rg.r == RR && rg.D == DD) { zpass_ring<T, RR, DD><<<grid, ZT, 0, s>>>(a); return true; }
    ELES_Z(4, 6) ELES_Z(4, 8) ELES_Z(4, 10) ELES_Z(4, 11) ELES_Z(4, 14) ELES_Z(4, 16)
    ELES_Z(6, 11) ELES_Z(8, 7) ELES_Z(8, 8) ELES_Z(8, 15) ELES_Z(8, 16)
#undef ELES_Z
    return false;
}

// Unfused x and z contractions of one snapshot into h (FP64 path, and any
// grid without a fused instantiation).
template <typename T>
void xz_unfused(ef_plan *p, const T *u, T *h, double *uref, double *plane_mean, int nf, cudaStream_t s)
{
    T *g = static_cast<T *>(p->d_g);
    T *urefT = static_cast<T *>(p->d_urefT);
    uref_kernel<T><<<dim3(p->ny, 3), 256, 0, s>>>(u, p->nx, p->ny, p->nz, uref, urefT);
    bool ring_x = false;
    if (p->rx.ok) {
        XArgs<T> a;
        a.u = u; a.uref = urefT; a.g = g;
        a.rowsum = nullptr;
        a.nx = p->nx; a.ny = p->ny; a.nz = p->nz; a.nlx = p->nlx; a.nzw = p->nzw;
        a.nblk = p->nlx + p->rx.D - 1;
        a.dmax = p->rx.dmax;
        const T *W = ring_W<T>(p->rx);
        for (int i = 0; i < p->rx.r * p->rx.D; i++) a.W[i] = W[i];
        ring_x = dispatch_x<T>(p->rx, a, nf, p->ny, p->nz, s);
    }
    if (!ring_x) {
        const size_t total = (size_t)p->ny * p->nz * p->nlx;
        const unsigned grid = (unsigned)((total + 127) / 128);
        if (nf == 9)
            xpass_gather<T, 9><<<grid, 128, 0, s>>>(u, urefT, g, p->bx.d_start, band_w<T>(p->bx),
                                                    p->bx.T, p->nx, p->ny, p->nz, p->nlx);
        else
            xpass_gather<T, 3><<<grid, 128, 0, s>>>(u, urefT, g, p->bx.d_start, band_w<T>(p->bx),
                                                    p->bx.T, p->nx, p->ny, p->nz, p->nlx);
    }
    bool ring_z = false;
    if (p->rz.ok) {
        ZArgs<T> a;
        a.g = g; a.h = h; a.nf = nf; a.ny = p->ny; a.nz = p->nz; a.nlz = p->nlz; a.nlx = p->nlx;
        a.nblk = p->nlz + p->rz.D - 1;
        a.dmax = p->rz.dmax;
        const T *W = ring_W<T>(p->rz);
        for (int i = 0; i < p->rz.r * p->rz.D; i++) a.W[i] = W[i];
        ring_z = dispatch_z<T>(p->rz, a, s);
    }
    if (!ring_z) {
        const size_t total = (size_t)nf * p->ny * p->nlz * p->nlx;
        zpass_gather<T><<<(unsigned)((total + 127) / 128), 128, 0, s>>>(
            g, h, p->bz.d_start, band_w<T>(p->bz), p->bz.T, nf, p->ny, p->nz, p->nlz, p->nlx);
    }
    if (plane_mean)
        plane_mean_direct<T><<<dim3(p->ny, 3), 256, 0, s>>>(u, uref, p->nx, p->ny, p->nz, plane_mean);
}

// The y contraction and the recovery of ~bar(u) and T (and the y-profile
// terms) for ns snapshots whose h and reference profile are in place.
template <typename T>
int y_stage(ef_plan *p, int ns, T *ubar, T *tau, bool stress, cudaStream_t s, const PhaseEvents *pe)
{
    T *h = static_cast<T *>(p->d_h);
    cudaError_t e = cudaSuccess;
    T *wy = static_cast<T *>(p->d_wy);
    e = launch_yprofile<T>(p->d_uref, p->d_ystart, p->d_ycount, p->d_yw64[0], p->d_yw64[1], p->ny, p->nly,
                           p->ext == EF_EXT_ODD_EVEN, ns, p->d_AU, p->d_AUU,
                           sizeof(T) == 4 && p->ytc_ok ? nullptr : wy, p->d_Kab, s);
    if (e != cudaSuccess) return cuda_fail(e, "yprofile launch");
    if constexpr (sizeof(T) == 4) {
        if (p->ytc_ok) {   // tensor-core y passes (split-precision plans)
            YTcArgs yt;
            memset(&yt, 0, sizeof yt);
            yt.geo = p->ytc;
            const int nplane = p->nlz * p->nlx;
            int rc = encode_h_map(h, nplane, p->ny, ns, p->ytc.box_rows, &yt.hmap);
            if (rc) return rc;
            e = launch_yfrag(p->ytc, p->d_yw64[0], p->d_yw64[1], p->d_uref, p->d_AU, p->ny, p->nly, ns, p->d_yfrag, s);
            if (e != cudaSuccess) return cuda_fail(e, "yfrag launch");
            yt.frag = p->d_yfrag; yt.AU = p->d_AU; yt.Kab = p->d_Kab;
            yt.ubar = ubar; yt.tau = tau; yt.tmp = static_cast<float *>(p->d_ytmp);
            yt.ny = p->ny; yt.nly = p->nly; yt.nplane = nplane;
            yt.nlz = p->nlz; yt.nlx = p->nlx; yt.ptrans = p->fused && p->x_variant == 3;
            yt.stress = stress ? 1 : 0; yt.flip = p->ext == EF_EXT_ODD_EVEN; yt.err = p->d_err;
            e = launch_ytc(yt, ns, s);
            if (e != cudaSuccess) return cuda_fail(e, "ytc launch");
            prof_mark(pe, 3, s);
            prof_mark(pe, 4, s);
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "filter launch");
            return EF_OK;
        }
    }
    YArgs<T> y;
    y.h = h; y.wy = wy; y.AU = p->d_AU; y.AUU = p->d_AUU; y.ystart = p->d_ystart; y.ycount = p->d_ycount;
    y.ubar = ubar; y.tau = tau; y.tmp = static_cast<T *>(p->d_ytmp); y.ny = p->ny; y.nly = p->nly; y.nlz = p->nlz; y.nlx = p->nlx;
    y.stress = stress ? 1 : 0; y.flip = p->ext == EF_EXT_ODD_EVEN; y.err = p->d_err;
    y.ptrans = p->fused && p->x_variant == 3;
    e = launch_ypass<T>(y, ns, s);
    if (e != cudaSuccess) return cuda_fail(e, "ypass launch");
    prof_mark(pe, 3, s);
    prof_mark(pe, 4, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "filter launch");
    return EF_OK;
}

template <typename T>
int run_group(ef_plan *p, int ns, const T *u, T *ubar, T *tau, double *plane_mean, bool stress,
              cudaStream_t s, const PhaseEvents *pe)
{
    const int nf = stress ? 9 : 3;
    const size_t np = (size_t)p->nx * p->ny * p->nz;
    const size_t nh = (size_t)9 * p->ny * p->nlz * p->nlx;
    T *h = static_cast<T *>(p->d_h);
    cudaError_t e = cudaSuccess;
    prof_mark(pe, 0, s);
    if constexpr (sizeof(T) == 4) {
        if (p->fused) {
            FusedArgs a;
            memset(&a, 0, sizeof a);
            a.err = p->d_err;
            a.u = u; a.h = h; a.uref = p->d_uref; a.plane_mean = plane_mean;
            a.nx = p->nx; a.ny = p->ny; a.nz = p->nz; a.nlx = p->nlx; a.nlz = p->nlz;
            a.nblk_x = p->nblk_x; a.bshift = p->bshift; a.dmin_x = p->rx.dmin;
            a.dmax_z = p->rz.dmax; a.ZQs = p->ZQs; a.NQ = p->NQ; a.P = p->P; a.nf = nf;
            a.lP = 0;
            while ((1 << a.lP) < a.P) a.lP++;
            for (int i = 0; i < p->rx.r * p->rx.D; i++) a.WX[i] = p->rx.W32[i];
            for (int i = 0; i < p->rz.r * p->rz.D; i++) a.WZ[i] = p->rz.W32[i];
            if (p->x_variant == 3) {
                int rc = ws_run(p, ns, u, h, p->d_uref, plane_mean, nf, s);
                if (rc) return rc;
            } else if (p->x_variant == 2) {
                FusedTCArgs ta = p->tc;
                a.box_rows = p->nz > 256 ? p->nz / 2 : p->nz;
                a.use_tma = 1;
                int rc = encode_u_map(u, p->nx, p->ny, p->nz, ns, 8, a.box_rows, &a.tmap);
                if (rc) return rc;
                ta.f = a;     // KS, zoff, afrag and the B fragments come from the plan
                e = launch_fused_tc(p->rz.r, p->rz.D, ta, ns, s);
            } else {
                e = launch_fused(p->rx.r, p->rx.D, p->rz.r, p->rz.D, a, ns, s);
            }
            if (e != cudaSuccess) return cuda_fail(e, "xz_fused launch");
        }
    }
    if (!p->fused) {
        for (int k = 0; k < ns; k++)
            xz_unfused<T>(p, u + k * 3 * np, h + k * nh, p->d_uref + (size_t)k * 3 * p->ny,
                          plane_mean ? plane_mean + (size_t)k * 3 * p->ny : nullptr, nf, s);
    }
    prof_mark(pe, 1, s);
    prof_mark(pe, 2, s);
    return y_stage<T>(p, ns, ubar, tau, stress, s, pe);
}

template <typename T>
int run_typed(ef_plan *p, int nsnap, const T *u, T *ubar, T *tau, double *plane_mean, bool stress,
              cudaStream_t s, const PhaseEvents *pe)
{
    const size_t np = (size_t)p->nx * p->ny * p->nz;
    const size_t nl = (size_t)p->nlx * p->nly * p->nlz;
    for (int s0 = 0; s0 < nsnap; s0 += p->reserve) {
        const int ns = nsnap - s0 < p->reserve ? nsnap - s0 : p->reserve;
        const bool last = s0 + ns >= nsnap;
        int rc = run_group<T>(p, ns, u + s0 * 3 * np, ubar + s0 * 3 * nl, stress ? tau + s0 * 6 * nl : nullptr,
                              plane_mean ? plane_mean + (size_t)s0 * 3 * p->ny : nullptr, stress, s,
                              last ? pe : nullptr);
        if (rc) return rc;
    }
    return EF_OK;
}

}  // namespace

int run_y_stage(ef_plan *p, int nsnap, void *ubar, void *tau, bool stress, cudaStream_t s)
{
    if (p->prec == EF_PREC_FP64)
        return y_stage<double>(p, nsnap, static_cast<double *>(ubar), static_cast<double *>(tau), stress, s, nullptr);
    return y_stage<float>(p, nsnap, static_cast<float *>(ubar), static_cast<float *>(tau), stress, s, nullptr);
}

int run_filter(ef_plan *p, int nsnap, const void *u, void *ubar, void *tau, double *plane_mean, bool stress,
               cudaStream_t s, const PhaseEvents *pe)
{
    if (p->diff) return diff_run(p, nsnap, u, ubar, tau, plane_mean, stress, s);
    if (p->prec == EF_PREC_FP64)
        return run_typed<double>(p, nsnap, static_cast<const double *>(u), static_cast<double *>(ubar),
                                 static_cast<double *>(tau), plane_mean, stress, s, pe);
    return run_typed<float>(p, nsnap, static_cast<const float *>(u), static_cast<float *>(ubar),
                            static_cast<float *>(tau), plane_mean, stress, s, pe);
}

}  // namespace eles
