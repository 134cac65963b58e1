// Filter-operator construction on the device, in FP64 (one thread per
// operator row).  The operators are those of Eq. 2 with a Gaussian kernel of
// constant width Delta, cut at |s| <= 2.5 Delta, trapezoid weights, every row
// normalised; the wall-normal line is extended across both walls by Eq. 7
// (or Eq. 9); the filtered field is sampled on the LES nodes by linear
// interpolation (the discretization operator of Sec. 3).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <vector>

#include "eles_internal.h"

namespace eles {
namespace {

__device__ __forceinline__ double gauss(double s, double delta)
{
    // sqrt(6/(pi delta^2)) exp(-6 s^2/delta^2); second moment delta^2/12.
    return sqrt(6.0 / (3.14159265358979323846 * delta * delta)) * exp(-6.0 * s * s / (delta * delta));
}

// Row X of the periodic operator A = S F on a uniform line of n nodes and
// length L.  The LES node X L / nl lies at DNS position X n / nl, so
// i0 = floor(X n / nl) and theta = (X n mod nl) / nl exactly.  Row i of F is
// the Gaussian at offsets o (columns i + o mod n), |o h| <= 2.5 Delta, divided
// by its sum; the band of row X covers offsets -K .. K+1 around i0.
__global__ void periodic_rows_kernel(int n, double L, int nl, double delta, int K, int T,
                                     int *start, double *w64, float *w32)
{
    int X = blockIdx.x * blockDim.x + threadIdx.x;
    if (X >= nl) return;
    double h = L / n;
    long num = (long)X * n;
    int i0 = (int)(num / nl);
    double theta = (double)(num % nl) / nl;
    double norm = 0.0;
    for (int o = -K; o <= K; o++) {
        double s = (double)o * h;
        if (fabs(s) <= 2.5 * delta) norm += gauss(s, delta) * h;
    }
    int st = i0 - K;
    st = ((st % n) + n) % n;
    start[X] = st;
    for (int t = 0; t < T; t++) {
        int c = i0 - K + t;                 // unwrapped column
        double v = 0.0;
        for (int q = 0; q < 2; q++) {       // DNS rows i0 and i0 + 1
            double wq = q ? theta : 1.0 - theta;
            if (wq == 0.0) continue;
            double s = (double)(c - (i0 + q)) * h;
            if (fabs(s) <= 2.5 * delta) v += wq * gauss(s, delta) * h / norm;
        }
        w64[(size_t)X * T + t] = v;
        w32[(size_t)X * T + t] = (float)v;
    }
}

// Trapezoid weight of DNS node j on the extended wall-normal line.  A mirror
// image of node j has the mirrors of j - 1 and j + 1 as neighbours, so it
// carries the same weight as the node itself; the wall node's neighbours are
// node 1 and the mirror of node 1.  Truncated mode: half cells at the walls.
__device__ __forceinline__ double wall_trap(const double *y, int ny, int j, int truncated)
{
    if (j == 0) return truncated ? 0.5 * (y[1] - y[0]) : (y[1] - y[0]);
    if (j == ny - 1) return truncated ? 0.5 * (y[ny - 1] - y[ny - 2]) : (y[ny - 1] - y[ny - 2]);
    return 0.5 * (y[j + 1] - y[j - 1]);
}

// Kernel moments over s in [a, b] clipped to |s - yi| <= 2.5 delta:
// I0 = int G(yi - s) ds (erf differences), J1 = int G(yi - s)(s - yi) ds
// (t G(t) integrates to -sigma^2 G(t), sigma^2 = delta^2 / 12).
__device__ void kernel_moments(double yi, double a, double b, double delta, double &I0, double &J1)
{
    const double R = 2.5 * delta, sig = delta / sqrt(12.0);
    a = fmax(a, yi - R);
    b = fmin(b, yi + R);
    I0 = 0.0;
    J1 = 0.0;
    if (!(b > a)) return;
    const double ta = a - yi, tb = b - yi, c = 1.0 / (sig * sqrt(2.0));
    I0 = 0.5 * (erf(tb * c) - erf(ta * c));
    J1 = sig * sig * (gauss(ta, delta) - gauss(tb, delta));
}

// Weight of a node at e of the extended line under the hat quadrature: the
// kernel integrated exactly against the node's hat function, whose left and
// right neighbours lie hl and hr away (0: no neighbour on that side).
__device__ double hat_weight(double yi, double e, double hl, double hr, double delta)
{
    double w = 0.0, I0, J1;
    if (hl > 0.0) {
        kernel_moments(yi, e - hl, e, delta, I0, J1);
        w += (J1 + (yi - (e - hl)) * I0) / hl;
    }
    if (hr > 0.0) {
        kernel_moments(yi, e, e + hr, delta, I0, J1);
        w += ((e + hr - yi) * I0 - J1) / hr;
    }
    return w;
}

// Weight of image e of DNS node j (mirror: the image reflected about a wall)
// at the filtered node yi: trapezoid or hat quadrature.
__device__ double image_weight(const double *y, int ny, int j, bool mirror, double e, double yi, double delta,
                               int truncated, int hat)
{
    if (!hat) {
        const double s = yi - e;
        return fabs(s) <= 2.5 * delta ? gauss(s, delta) * wall_trap(y, ny, j, truncated) : 0.0;
    }
    // gaps to the neighbours on the extended line: the mirror image has its
    // source's gaps swapped; a wall node's outer neighbour is the mirror of
    // its inner one (none on the truncated line)
    double hl = j > 0 ? y[j] - y[j - 1] : (truncated ? 0.0 : y[1] - y[0]);
    double hr = j < ny - 1 ? y[j + 1] - y[j] : (truncated ? 0.0 : y[ny - 1] - y[ny - 2]);
    if (mirror) {
        const double t = hl;
        hl = hr;
        hr = t;
    }
    return hat_weight(yi, e, hl, hr, delta);
}

// Adds (scale x) row i of F^even and F^odd to the dense rows re, ro.
__device__ void wall_row_accumulate(const double *y, int ny, int i, double delta, int truncated, int hat,
                                    double scale, double *re, double *ro)
{
    double yi = y[i];
    double norm = 0.0;
    // pass 1: row sum over every node of the (extended) line within reach
    for (int m = -1; m <= 1; m++) {
        if (truncated && m != 0) continue;
        for (int j = 0; j < ny; j++) {
            norm += image_weight(y, ny, j, false, y[j] + 4.0 * m, yi, delta, truncated, hat);
            if (!truncated && j > 0 && j < ny - 1)
                norm += image_weight(y, ny, j, true, -2.0 - y[j] + 4.0 * m, yi, delta, truncated, hat);
        }
    }
    // pass 2: fold every image onto its source node with the parity sign
    for (int m = -1; m <= 1; m++) {
        if (truncated && m != 0) continue;
        for (int j = 0; j < ny; j++) {
            bool wall = (j == 0 || j == ny - 1);
            double w = image_weight(y, ny, j, false, y[j] + 4.0 * m, yi, delta, truncated, hat);
            if (w != 0.0) {
                w *= scale / norm;
                re[j] += w;
                // a wall node is its own mirror: an odd extension vanishes there
                if (truncated || !wall) ro[j] += w;
            }
            if (!truncated && !wall) {
                w = image_weight(y, ny, j, true, -2.0 - y[j] + 4.0 * m, yi, delta, truncated, hat);
                if (w != 0.0) {
                    w *= scale / norm;
                    re[j] += w;
                    ro[j] -= w;
                }
            }
        }
    }
}

// Row J of A_y^even / A_y^odd on the LES node Y[J]: linear interpolation of
// rows i0, i0+1 of F (i0 = last DNS node <= Y, capped at ny - 2).
__global__ void wall_rows_kernel(const double *y, int ny, const double *Y, int nly, double delta,
                                 int truncated, int hat, double *we, double *wo, float *we32, float *wo32,
                                 int *start, int *count)
{
    int J = blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= nly) return;
    double *re = we + (size_t)J * ny, *ro = wo + (size_t)J * ny;
    int i0 = 0;
    while (i0 < ny - 2 && y[i0 + 1] <= Y[J]) i0++;
    double theta = (Y[J] - y[i0]) / (y[i0 + 1] - y[i0]);
    if (1.0 - theta != 0.0) wall_row_accumulate(y, ny, i0, delta, truncated, hat, 1.0 - theta, re, ro);
    if (theta != 0.0) wall_row_accumulate(y, ny, i0 + 1, delta, truncated, hat, theta, re, ro);
    int lo = ny, hi = -1;
    for (int j = 0; j < ny; j++) {
        if (re[j] != 0.0 || ro[j] != 0.0) { if (j < lo) lo = j; hi = j; }
        we32[(size_t)J * ny + j] = (float)re[j];
        wo32[(size_t)J * ny + j] = (float)ro[j];
    }
    start[J] = lo;
    count[J] = hi >= lo ? hi - lo + 1 : 0;
}

}  // namespace

int build_periodic_band(int n, double L, int nl, double delta, Band *b)
{
    double h = L / n;
    int K = (int)floor(2.5 * delta / h) + 1;
    int T = 2 * K + 2;
    b->n = n; b->nl = nl; b->T = T;
    cudaError_t e;
    if ((e = dev_malloc(&b->d_start, sizeof(int) * nl)) != cudaSuccess) return cuda_fail(e, "cudaMalloc band");
    if ((e = dev_malloc(&b->d_w64, sizeof(double) * (size_t)nl * T)) != cudaSuccess) return cuda_fail(e, "cudaMalloc band");
    if ((e = dev_malloc(&b->d_w32, sizeof(float) * (size_t)nl * T)) != cudaSuccess) return cuda_fail(e, "cudaMalloc band");
    periodic_rows_kernel<<<(nl + 127) / 128, 128>>>(n, L, nl, delta, K, T, b->d_start, b->d_w64, b->d_w32);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "periodic_rows_kernel");
    return EF_OK;
}

// When n = r nl every row is the first one shifted by r: read row 0 back and
// lay its taps out as the table W[s][dd] of the strided convolution.
int build_ring(const Band &b, Ring *rg)
{
    rg->ok = false;
    if (b.n % b.nl) return EF_OK;
    int r = b.n / b.nl;
    std::vector<double> row(b.T);
    std::vector<int> st(1);
    cudaError_t e = cudaMemcpy(row.data(), b.d_w64, sizeof(double) * b.T, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(st.data(), b.d_start, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read operator row");
    // column of tap t is st + t (mod n); its offset from node 0 is o
    int K = (b.T - 2) / 2;
    int R = 0;
    for (int t = 0; t < b.T; t++) {
        int o = t - K;
        if (row[t] != 0.0 && abs(o) > R) R = abs(o);
    }
    int dmin = -(R / r), dmax = (r - 1 + R) / r, D = dmax - dmin + 1;
    if (r > kMaxStride || D > kMaxRing) return EF_OK;
    rg->r = r; rg->R = R; rg->dmin = dmin; rg->dmax = dmax; rg->D = D;
    for (int s = 0; s < r; s++)
        for (int dd = 0; dd < D; dd++) {
            int o = s - r * (dd + dmin);
            double v = (o >= -R && o <= R) ? row[o + K] : 0.0;
            rg->W64[s * D + dd] = v;
            rg->W32[s * D + dd] = (float)v;
        }
    rg->ok = true;
    return EF_OK;
}

int build_wall_rows(ef_plan *p, const double *h_les_y)
{
    cudaError_t e;
    double *dY = nullptr;
    size_t dense = (size_t)p->nly * p->ny;
    if ((e = dev_malloc(&dY, sizeof(double) * p->nly)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    e = cudaMemcpy(dY, h_les_y, sizeof(double) * p->nly, cudaMemcpyHostToDevice);
    for (int q = 0; q < 2 && e == cudaSuccess; q++) {
        e = dev_malloc(&p->d_yw64[q], sizeof(double) * dense);
        if (e == cudaSuccess) e = dev_malloc(&p->d_yw32[q], sizeof(float) * dense);
        if (e == cudaSuccess) e = cudaMemset(p->d_yw64[q], 0, sizeof(double) * dense);
    }
    if (e == cudaSuccess) e = dev_malloc(&p->d_ystart, sizeof(int) * p->nly);
    if (e == cudaSuccess) e = dev_malloc(&p->d_ycount, sizeof(int) * p->nly);
    if (e != cudaSuccess) { cudaFree(dY); return cuda_fail(e, "allocate y operator"); }
    int truncated = (p->ext == EF_EXT_NONE) ? 1 : 0;
    wall_rows_kernel<<<(p->nly + 63) / 64, 64>>>(p->d_ygrid, p->ny, dY, p->nly, p->delta, truncated, p->yquad,
                                                 p->d_yw64[0], p->d_yw64[1], p->d_yw32[0],
                                                 p->d_yw32[1], p->d_ystart, p->d_ycount);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(dY);
    if (e != cudaSuccess) return cuda_fail(e, "wall_rows_kernel");
    std::vector<int> cnt(p->nly);
    e = cudaMemcpy(cnt.data(), p->d_ycount, sizeof(int) * p->nly, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read y counts");
    p->ytaps_max = 0;
    for (int c : cnt) p->ytaps_max = c > p->ytaps_max ? c : p->ytaps_max;
    std::vector<int> sta(p->nly);
    e = cudaMemcpy(sta.data(), p->d_ystart, sizeof(int) * p->nly, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read y starts");
    p->ytc_fit = (p->prec == EF_PREC_BF16X3 || p->prec == EF_PREC_TF32X2) && ytc_geometry(sta, cnt, p->ny, p->nlz * p->nlx, &p->ytc);
    if (p->ytc_fit) {
        // row tiles whose filter never meets a wall: A_y^- and A_y^+ agree on every
        // row, so the wall term d = (A^- - A^+) h is zero there
        std::vector<double> we(dense), wo(dense);
        e = cudaMemcpy(we.data(), p->d_yw64[0], sizeof(double) * dense, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(wo.data(), p->d_yw64[1], sizeof(double) * dense, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "read y operators");
        for (int mt = 0; mt < p->ytc.nmt; mt++) {
            bool same = true;
            for (int J = 16 * mt; J < 16 * mt + 16 && J < p->nly && same; J++)
                for (int j = 0; j < p->ny && same; j++) same = we[(size_t)J * p->ny + j] == wo[(size_t)J * p->ny + j];
            p->ytc.dzero[mt] = same ? 1 : 0;
        }
    }
    p->ytc_ok = p->ytc_fit;
    return EF_OK;
}

}  // namespace eles
