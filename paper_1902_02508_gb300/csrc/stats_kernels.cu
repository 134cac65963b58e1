// The paper's error measures (Sec. 4) as device reductions.
//
//   plane statistics: <u_c>(y_j) and u_c,rms(y_j) = sqrt(<(u_c - <u_c>)^2>)
//                     over the homogeneous directions x and z;
//   Eq. 13:           || a/ut_a - b/ut_b ||_V / || b/ut_b ||_V for one
//                     velocity component (the paper uses u_1);
//   Eq. 14 / Eq. 15:  the same norm of profiles (mean or rms) over x_2 from
//                     the wall to the channel centre.
// Quadrature: x and z periodic and uniform (node sums; their cell sizes
// cancel in the ratios), trapezoid in y; the wall-to-centre integral is that
// of the piecewise-linear interpolant over y in [-1, 0].  All sums are FP64
// and deterministic: blocks write partial sums that one block adds in a
// fixed order.
#include <math.h>
#include <string.h>

#include <vector>

#include "eles_internal.h"

namespace {

constexpr int kStatBlocks = 1024;   // partial sums of the field reductions
constexpr int kStatThreads = 256;

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += sh[i];
    return t;   // valid in thread 0
}

// One block per (y row j, component c).
template <typename T>
__global__ void __launch_bounds__(kStatThreads) plane_stats_kernel(const T *__restrict__ u, int ny, int nxz,
                                                                    double *mean, double *rms)
{
    __shared__ double sh[kStatThreads / 32];
    const int j = blockIdx.x, c = blockIdx.y;
    const T *row = u + ((size_t)c * ny + j) * nxz;
    // sums about the row's first value: no cancellation of the mean in the variance
    const double K = (double)row[0];
    double s = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < nxz; i += blockDim.x) {
        const double v = (double)row[i] - K;
        s += v;
        s2 += v * v;
    }
    s = block_sum(s, sh);
    s2 = block_sum(s2, sh);
    if (threadIdx.x == 0) {
        const double m = s / nxz;
        const double var = s2 / nxz - m * m;
        mean[c * ny + j] = K + m;
        rms[c * ny + j] = sqrt(var > 0.0 ? var : 0.0);
    }
}

// Partial sums of sum_j w_j sum_xz (a/ut_a - b/ut_b)^2 and (b/ut_b)^2.
template <typename T>
__global__ void __launch_bounds__(kStatThreads) error_field_kernel(const T *__restrict__ a, const T *__restrict__ b,
                                                                    const double *__restrict__ wy, int ny, int nxz,
                                                                    double ia, double ib, double *part)
{
    __shared__ double sh[kStatThreads / 32];
    const size_t n = (size_t)ny * nxz;
    double num = 0.0, den = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double w = wy[i / nxz];
        const double vb = (double)b[i] * ib, d = (double)a[i] * ia - vb;
        num += w * d * d;
        den += w * vb * vb;
    }
    num = block_sum(num, sh);
    den = block_sum(den, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = num;
        part[2 * blockIdx.x + 1] = den;
    }
}

// err = sqrt(sum of numerators / sum of denominators), partials in order.
__global__ void __launch_bounds__(kStatThreads) error_finish_kernel(const double *__restrict__ part, int nparts,
                                                                     double *err)
{
    __shared__ double sh[kStatThreads / 32];
    // fixed assignment of partials to threads, then a fixed-order tree
    double num = 0.0, den = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        num += part[2 * i];
        den += part[2 * i + 1];
    }
    num = block_sum(num, sh);
    den = block_sum(den, sh);
    if (threadIdx.x == 0) *err = sqrt(num) / sqrt(den);
}

// Eq. 14 / 15 on profiles of ny nodes with the wall-to-centre weights.
__global__ void __launch_bounds__(kStatThreads) error_profile_kernel(const double *__restrict__ pa,
                                                                      const double *__restrict__ pb,
                                                                      const double *__restrict__ wh, int ny,
                                                                      double ia, double ib, double *err)
{
    __shared__ double sh[kStatThreads / 32];
    double num = 0.0, den = 0.0;
    for (int j = threadIdx.x; j < ny; j += blockDim.x) {
        const double vb = pb[j] * ib, d = pa[j] * ia - vb;
        num += wh[j] * d * d;
        den += wh[j] * vb * vb;
    }
    num = block_sum(num, sh);
    den = block_sum(den, sh);
    if (threadIdx.x == 0) *err = sqrt(num) / sqrt(den);
}

}  // namespace

struct ef_stats {
    int nx = 0, ny = 0, nz = 0, prec = 0;
    double *d_wy = nullptr;     // trapezoid weights in y [ny]
    double *d_wh = nullptr;     // wall-to-centre weights [ny]
    double *d_part = nullptr;   // partial sums [kStatBlocks][2]
};

using namespace eles;

extern "C" {

int ef_stats_create(const ef_grid *g, int precision, ef_stats **out)
{
    if (!g || !out || !g->y || g->nx < 1 || g->ny < 2 || g->nz < 1) {
        set_error("ef_stats_create: bad grid");
        return EF_ERR_ARG;
    }
    if (precision != EF_PREC_FP64 && precision != EF_PREC_FP32 && precision != EF_PREC_BF16X3 &&
        precision != EF_PREC_TF32X2) {
        set_error("ef_stats_create: unknown precision %d", precision);
        return EF_ERR_ARG;
    }
    *out = nullptr;
    const int ny = g->ny;
    for (int j = 1; j < ny; j++)
        if (!(g->y[j] > g->y[j - 1])) { set_error("ef_stats_create: y nodes must ascend"); return EF_ERR_ARG; }
    std::vector<double> wy(ny, 0.0), wh(ny, 0.0);
    for (int j = 0; j + 1 < ny; j++) {
        const double lo = g->y[j], hi = g->y[j + 1], h = hi - lo;
        wy[j] += h / 2;
        wy[j + 1] += h / 2;
        if (hi <= 0.0) {                 // interval in the lower half
            wh[j] += h / 2;
            wh[j + 1] += h / 2;
        } else if (lo < 0.0) {           // the interval holding the centre, clipped at y = 0
            const double t = -lo / h;
            wh[j] += h * (t - t * t / 2);
            wh[j + 1] += h * t * t / 2;
        }
    }
    ef_stats *st = new ef_stats();
    st->nx = g->nx; st->ny = ny; st->nz = g->nz; st->prec = precision;
    cudaError_t e = dev_malloc(&st->d_wy, sizeof(double) * ny);
    if (e == cudaSuccess) e = dev_malloc(&st->d_wh, sizeof(double) * ny);
    if (e == cudaSuccess) e = dev_malloc(&st->d_part, sizeof(double) * 2 * kStatBlocks);
    if (e == cudaSuccess) e = cudaMemcpy(st->d_wy, wy.data(), sizeof(double) * ny, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(st->d_wh, wh.data(), sizeof(double) * ny, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        ef_stats_destroy(st);
        return cuda_fail(e, "ef_stats_create");
    }
    *out = st;
    return EF_OK;
}

void ef_stats_destroy(ef_stats *st)
{
    if (!st) return;
    cudaFree(st->d_wy);
    cudaFree(st->d_wh);
    cudaFree(st->d_part);
    delete st;
}

int ef_plane_stats(ef_stats *st, const void *u, double *mean, double *rms, void *stream)
{
    if (!st || !u || !mean || !rms) { set_error("ef_plane_stats: NULL argument"); return EF_ERR_ARG; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nxz = st->nx * st->nz;
    if (st->prec == EF_PREC_FP64)
        plane_stats_kernel<double><<<dim3(st->ny, 3), kStatThreads, 0, s>>>(static_cast<const double *>(u), st->ny,
                                                                            nxz, mean, rms);
    else
        plane_stats_kernel<float><<<dim3(st->ny, 3), kStatThreads, 0, s>>>(static_cast<const float *>(u), st->ny, nxz,
                                                                           mean, rms);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EF_OK : cuda_fail(e, "ef_plane_stats");
}

int ef_error_field(ef_stats *st, const void *a, const void *b, int component, double utau_a, double utau_b,
                   double *err, void *stream)
{
    if (!st || !a || !b || !err) { set_error("ef_error_field: NULL argument"); return EF_ERR_ARG; }
    if (component < 0 || component > 2) { set_error("ef_error_field: component must be 0, 1 or 2"); return EF_ERR_ARG; }
    if (!(utau_a > 0) || !(utau_b > 0)) { set_error("ef_error_field: u_tau must be > 0"); return EF_ERR_ARG; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nxz = st->nx * st->nz;
    const size_t off = (size_t)component * st->ny * nxz;
    if (st->prec == EF_PREC_FP64)
        error_field_kernel<double><<<kStatBlocks, kStatThreads, 0, s>>>(
            static_cast<const double *>(a) + off, static_cast<const double *>(b) + off, st->d_wy, st->ny, nxz,
            1.0 / utau_a, 1.0 / utau_b, st->d_part);
    else
        error_field_kernel<float><<<kStatBlocks, kStatThreads, 0, s>>>(
            static_cast<const float *>(a) + off, static_cast<const float *>(b) + off, st->d_wy, st->ny, nxz,
            1.0 / utau_a, 1.0 / utau_b, st->d_part);
    error_finish_kernel<<<1, kStatThreads, 0, s>>>(st->d_part, kStatBlocks, err);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EF_OK : cuda_fail(e, "ef_error_field");
}

int ef_error_profile(ef_stats *st, const double *pa, const double *pb, double utau_a, double utau_b, double *err,
                     void *stream)
{
    if (!st || !pa || !pb || !err) { set_error("ef_error_profile: NULL argument"); return EF_ERR_ARG; }
    if (!(utau_a > 0) || !(utau_b > 0)) { set_error("ef_error_profile: u_tau must be > 0"); return EF_ERR_ARG; }
    error_profile_kernel<<<1, kStatThreads, 0, static_cast<cudaStream_t>(stream)>>>(pa, pb, st->d_wh, st->ny,
                                                                                   1.0 / utau_a, 1.0 / utau_b, err);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EF_OK : cuda_fail(e, "ef_error_profile");
}

}  // extern "C"
