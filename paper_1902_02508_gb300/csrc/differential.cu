// The differential filter of Sec. 3 on the GPU, in FP64.
//
// The filter the paper's simulations use is the Green's function of
// (1 - a^2 lap): ubar solves (1 - a^2 lap) ubar = u on the domain extended
// across the walls (Eq. 7, or Eq. 9), periodic in x and z.  The Laplacian is
// the second-order finite-difference one on the DNS nodes (three-point
// periodic in x and z, the three-point non-uniform stencil in y with mirror
// ghosts of the field's parity at both walls), and a^2 = Delta_f^2 / 40.
// The kernel is not a product of one-dimensional kernels, so this path does
// not share the separable contractions of the Gaussian filter:
//   1. form the field (u_a or u_a u_b) and transform each (y, z) row in x;
//   2. transform each (y, kx) column in z (the periodic stencils become
//      diagonal: lap -> -(2 - 2 cos(k h)) / h^2);
//   3. solve the tridiagonal system in y for every (kx, kz) (Thomas);
//   4. transform back in z only on the LES rows, keeping the LES z nodes;
//   5. transform back in x on those, keeping the LES x nodes (the LES nodes
//      are DNS nodes, so the linear interpolation of Sec. 3 is the identity);
//   6. T_ab = bar(u_a u_b) - ubar_a ubar_b (Eq. 6).
// The transforms are mixed-radix (2 and 3) Stockham FFTs in shared memory
// (the decimation-in-time formulation for GPUs of Govindaraju et al.,
// SC 2008), one row or a few columns per CTA; the inverse is the forward
// transform of the conjugate.  The plane means of u_c are the zero modes.
#include <math.h>
#include <string.h>

#include <vector>

#include "eles_internal.h"

namespace eles {

struct DiffPlan {
    double a = 0;
    int nxh = 0;                          // nx / 2 + 1 kept x modes (real input)
    int radx[32] = {}, nradx = 0, radz[32] = {}, nradz = 0;
    double2 *twx = nullptr, *twz = nullptr;   // exp(-2 pi i m / N), m < N
    double *k2x = nullptr, *k2z = nullptr;    // a^2 (2 - 2 cos(2 pi m / N)) / h^2
    double *dyy = nullptr;                // [3][ny]: D_yy lower, centre, upper (interior and even walls)
    int *jy = nullptr;                    // [nly]: DNS row of each LES row
    int rx = 1, rz = 1;                   // DNS nodes per LES node in x and z
    int zcols = 4;                        // columns per CTA in the z transforms
    double2 *spec = nullptr;              // [ny][nz][nxh] spectrum of one field
    double *fcp = nullptr;                // [2][ny][nz][nxh] Thomas factors per parity (even, odd):
    double *finv = nullptr;               //   modified upper diagonal and pivot reciprocal
    double2 *lesz = nullptr;              // [nly][nlz][nxh]
    double *fld = nullptr;                // [9][nly][nlz][nlx] filtered fields of one snapshot
};

namespace {

constexpr int kDiffThreads = 256;
constexpr int kDiffMaxN = 1024;

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Stockham stages over ncol independent transforms of length N held column
// by column (column c at b + c * N).  Returns the buffer holding the result.
__device__ double2 *smem_fft(double2 *b0, double2 *b1, int N, int ncol, const int *rad, int nrad,
                             const double2 *__restrict__ tw)
{
    int Ns = 1;
    for (int s = 0; s < nrad; s++) {
        const int R = rad[s], NR = N / R, tstride = N / (Ns * R);
        for (int t = threadIdx.x; t < NR * ncol; t += blockDim.x) {
            const int c = t / NR, j = t - c * NR, k = j % Ns;
            const double2 *x = b0 + c * N;
            double2 *yv = b1 + c * N;
            const int d = (j / Ns) * Ns * R + k;
            double2 v0 = x[j], v1 = x[j + NR];
            if (Ns > 1) v1 = cmul(v1, tw[tstride * k]);      // the first stage's twiddles are 1
            if (R == 2) {
                yv[d] = make_double2(v0.x + v1.x, v0.y + v1.y);
                yv[d + Ns] = make_double2(v0.x - v1.x, v0.y - v1.y);
            } else {
                // radix 3: w = exp(-2 pi i / 3); y1,2 = v0 - (v1 + v2) / 2 -/+ i (sqrt 3 / 2)(v1 - v2)
                double2 v2 = x[j + 2 * NR];
                if (Ns > 1) v2 = cmul(v2, tw[2 * tstride * k]);
                const double2 t1 = make_double2(v1.x + v2.x, v1.y + v2.y);
                const double2 t2 = make_double2(v1.x - v2.x, v1.y - v2.y);
                const double h = 0.86602540378443864676;     // sqrt(3) / 2
                const double2 m = make_double2(h * t2.y, -h * t2.x); // -i h t2
                const double2 base = make_double2(v0.x - 0.5 * t1.x, v0.y - 0.5 * t1.y);
                yv[d] = make_double2(v0.x + t1.x, v0.y + t1.y);
                yv[d + Ns] = make_double2(base.x + m.x, base.y + m.y);
                yv[d + 2 * Ns] = make_double2(base.x - m.x, base.y - m.y);
            }
        }
        __syncthreads();
        double2 *tmp = b0;
        b0 = b1;
        b1 = tmp;
        Ns *= R;
    }
    return b0;
}

struct DxFwdArgs {
    const double *u;                      // [3][ny][nz][nx]
    int ca, cb;                           // the field is u_ca (cb < 0) or u_ca u_cb
    int odd;                              // its parity is odd: zero on the walls
    int nx, ny, nz, nxh;
    int rad[32], nrad;
    const double2 *tw;
    double2 *spec;                        // [ny][nz][nxh]
};

// One CTA per (pair of z rows k0 = 2 b, k0 + 1; y row j): the two real rows
// are transformed together as z = f_k0 + i f_k1, and separated by the
// symmetry of real transforms: F_k0[m] = (Z[m] + conj Z[N-m]) / 2,
// F_k1[m] = (Z[m] - conj Z[N-m]) / (2i).
__global__ void __launch_bounds__(kDiffThreads) dx_forward(const DxFwdArgs a)
{
    extern __shared__ double2 sbuf[];
    const int k0 = 2 * blockIdx.x, j = blockIdx.y, N = a.nx;
    const bool two = k0 + 1 < a.nz;
    double2 *b0 = sbuf, *b1 = sbuf + N;
    const size_t plane = (size_t)a.ny * a.nz * a.nx;
    const size_t row = ((size_t)j * a.nz + k0) * a.nx;
    const bool zero = a.odd && (j == 0 || j == a.ny - 1);
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double v0 = a.u[a.ca * plane + row + i], v1 = two ? a.u[a.ca * plane + row + N + i] : 0.0;
        if (a.cb >= 0) {
            v0 *= a.u[a.cb * plane + row + i];
            if (two) v1 *= a.u[a.cb * plane + row + N + i];
        }
        b0[i] = zero ? make_double2(0.0, 0.0) : make_double2(v0, v1);
    }
    __syncthreads();
    const double2 *X = smem_fft(b0, b1, N, 1, a.rad, a.nrad, a.tw);
    double2 *out = a.spec + ((size_t)j * a.nz + k0) * a.nxh;
    for (int m = threadIdx.x; m < a.nxh; m += blockDim.x) {
        const double2 zm = X[m], zc = X[m == 0 ? 0 : N - m];       // conj taken below
        out[m] = make_double2(0.5 * (zm.x + zc.x), 0.5 * (zm.y - zc.y));
        if (two) out[a.nxh + m] = make_double2(0.5 * (zm.y + zc.y), -0.5 * (zm.x - zc.x));
    }
}

struct DzArgs {
    double2 *spec;                        // [ny][nz][nxh]
    int nz, nxh, ncol;
    int rad[32], nrad;
    const double2 *tw;
    // inverse only: LES rows and output
    const int *jy;
    int rz, nlz;
    double2 *lesz;                        // [nly][nlz][nxh]
};

// Forward z transform in place: one CTA per (group of ncol x modes, y row).
__global__ void __launch_bounds__(kDiffThreads) dz_forward(const DzArgs a)
{
    extern __shared__ double2 sbuf[];
    const int N = a.nz, c0 = blockIdx.x * a.ncol, j = blockIdx.y;
    const int nc = min(a.ncol, a.nxh - c0);
    double2 *b0 = sbuf, *b1 = sbuf + (size_t)N * a.ncol;
    double2 *base = a.spec + (size_t)j * N * a.nxh + c0;
    for (int t = threadIdx.x; t < N * a.ncol; t += blockDim.x) {
        const int k = t / a.ncol, c = t - k * a.ncol;
        b0[c * N + k] = c < nc ? base[(size_t)k * a.nxh + c] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const double2 *Z = smem_fft(b0, b1, N, a.ncol, a.rad, a.nrad, a.tw);
    for (int t = threadIdx.x; t < N * a.ncol; t += blockDim.x) {
        const int k = t / a.ncol, c = t - k * a.ncol;
        if (c < nc) base[(size_t)k * a.nxh + c] = Z[c * N + k];
    }
}

// Inverse z transform of the LES rows (conjugate, forward transform,
// conjugate; the 1/(nx nz) scaling is applied at the end), keeping the LES
// z nodes.  One CTA per (group of x modes, LES row).
__global__ void __launch_bounds__(kDiffThreads) dz_inverse(const DzArgs a)
{
    extern __shared__ double2 sbuf[];
    const int N = a.nz, c0 = blockIdx.x * a.ncol, J = blockIdx.y, j = a.jy[J];
    const int nc = min(a.ncol, a.nxh - c0);
    double2 *b0 = sbuf, *b1 = sbuf + (size_t)N * a.ncol;
    const double2 *base = a.spec + (size_t)j * N * a.nxh + c0;
    for (int t = threadIdx.x; t < N * a.ncol; t += blockDim.x) {
        const int k = t / a.ncol, c = t - k * a.ncol;
        const double2 v = c < nc ? base[(size_t)k * a.nxh + c] : make_double2(0.0, 0.0);
        b0[c * N + k] = make_double2(v.x, -v.y);
    }
    __syncthreads();
    const double2 *Z = smem_fft(b0, b1, N, a.ncol, a.rad, a.nrad, a.tw);
    double2 *out = a.lesz + (size_t)J * a.nlz * a.nxh + c0;
    for (int t = threadIdx.x; t < a.nlz * a.ncol; t += blockDim.x) {
        const int K = t / a.ncol, c = t - K * a.ncol;
        const double2 v = Z[c * N + K * a.rz];
        if (c < nc) out[(size_t)K * a.nxh + c] = make_double2(v.x, -v.y);
    }
}

struct DyArgs {
    double2 *spec;                        // [ny][nz][nxh], in place
    const double *fcp, *finv;             // this parity's Thomas factors [ny][nz][nxh]
    const double *k2x, *k2z, *dyy;        // a^2 k~^2 tables; D_yy [3][ny]
    double a2;
    int ny, nz, nxh, odd;
};

// The tridiagonal rows for (kz, kx):
//   -a^2 lo_j v_{j-1} + (1 + a^2 (kx~^2 + kz~^2) - a^2 ce_j) v_j - a^2 up_j v_{j+1} = f_j,
// identity rows on the walls for an odd field.
__device__ __forceinline__ void dy_row(const DyArgs &a, double lam, int j, double &sub, double &dia, double &sup)
{
    if (a.odd && (j == 0 || j == a.ny - 1)) { sub = 0.0; dia = 1.0; sup = 0.0; return; }
    sub = -a.a2 * a.dyy[j];
    dia = 1.0 + lam - a.a2 * a.dyy[a.ny + j];
    sup = -a.a2 * a.dyy[2 * a.ny + j];
}

// Set-up: the LU factors of the Thomas algorithm per line (they depend on
// the mode and the parity only, not on the field): c_j = sup_j / den_j and
// 1 / den_j with den_j = dia_j - sub_j c_{j-1}.
__global__ void __launch_bounds__(kDiffThreads) dy_factor(DyArgs a, double *fcp, double *finv)
{
    const long line = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nline = (long)a.nz * a.nxh;
    if (line >= nline) return;
    const int kz = (int)(line / a.nxh), kx = (int)(line - (long)kz * a.nxh);
    const double lam = a.k2x[kx] + a.k2z[kz];
    double c = 0.0;
    for (int j = 0; j < a.ny; j++) {
        double sub, dia, sup;
        dy_row(a, lam, j, sub, dia, sup);
        const double inv = 1.0 / (dia - sub * c);
        c = sup * inv;
        fcp[(size_t)j * nline + line] = c;
        finv[(size_t)j * nline + line] = inv;
    }
}

// Thomas algorithm per (kz, kx) with the precomputed factors: forward
// d_j = (f_j - sub_j d_{j-1}) / den_j, backward v_j = d_j - c_j v_{j+1}.
// Threads run along kx (coalesced).
__global__ void __launch_bounds__(kDiffThreads) dy_solve(const DyArgs a)
{
    const long line = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nline = (long)a.nz * a.nxh;
    if (line >= nline) return;
    double2 d = make_double2(0.0, 0.0);
    for (int j = 0; j < a.ny; j++) {
        const size_t o = (size_t)j * nline + line;
        const double sub = (a.odd && j == a.ny - 1) ? 0.0 : -a.a2 * a.dyy[j];
        const double inv = a.finv[o];
        const double2 f = a.spec[o];
        d = make_double2((f.x - sub * d.x) * inv, (f.y - sub * d.y) * inv);
        a.spec[o] = d;
    }
    double2 v = d;
    for (int j = a.ny - 2; j >= 0; j--) {
        const size_t o = (size_t)j * nline + line;
        const double cj = a.fcp[o];
        const double2 dj = a.spec[o];
        v = make_double2(dj.x - cj * v.x, dj.y - cj * v.y);
        a.spec[o] = v;
    }
}

struct DxInvArgs {
    const double2 *lesz;                  // [nly][nlz][nxh]
    double *out;                          // [nly][nlz][nlx]
    int nx, nxh, rx, nlx;
    double scale;                         // 1 / (nx nz)
    int rad[32], nrad;
    const double2 *tw;
};

// Inverse x transform of one (LES row, LES z node): the Hermitian spectrum
// completed from the kept modes, conjugated, transformed, real part at the
// LES x nodes.
__global__ void __launch_bounds__(kDiffThreads) dx_inverse(const DxInvArgs a)
{
    extern __shared__ double2 sbuf[];
    const int K = blockIdx.x, J = blockIdx.y, N = a.nx, nlz = gridDim.x;
    double2 *b0 = sbuf, *b1 = sbuf + N;
    const double2 *X = a.lesz + ((size_t)J * nlz + K) * a.nxh;
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        double2 v;
        if (m < a.nxh) v = X[m];
        else {
            const double2 w = X[N - m];
            v = make_double2(w.x, -w.y);
        }
        b0[m] = make_double2(v.x, -v.y);
    }
    __syncthreads();
    const double2 *Y = smem_fft(b0, b1, N, 1, a.rad, a.nrad, a.tw);
    double *o = a.out + ((size_t)J * nlz + K) * a.nlx;
    for (int X0 = threadIdx.x; X0 < a.nlx; X0 += blockDim.x) o[X0] = Y[X0 * a.rx].x * a.scale;
}

// Plane means of a velocity component: the zero mode of each y row.
__global__ void plane_mean_from_spec(const double2 *spec, int ny, int nz, int nxh, double scale, double *pm)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < ny) pm[j] = spec[(size_t)j * nz * nxh].x * scale;
}

// ubar_c = F(u_c); T_q = F(u_i u_j) - F(u_i) F(u_j).
__global__ void diff_stress(const double *fld, long n, double *ubar, double *tau)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int pi[6] = {0, 0, 0, 1, 1, 2}, pj[6] = {0, 1, 2, 1, 2, 2};
    double f[3];
    for (int c = 0; c < 3; c++) {
        f[c] = fld[c * n + i];
        ubar[c * n + i] = f[c];
    }
    if (tau)
        for (int q = 0; q < 6; q++) tau[q * n + i] = fld[(3 + q) * n + i] - f[pi[q]] * f[pj[q]];
}

// (1 - a^2 lap) of a velocity field on one grid, the stencils of the filter.
__global__ void unfilter_kernel(const double *__restrict__ in, double *__restrict__ out, const double *__restrict__ y,
                                int nx, int ny, int nz, double ihx2, double ihz2, double a2, int p0, int p1, int p2)
{
    const long n = (long)nx * ny * nz;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 3 * n) return;
    const int c = (int)(idx / n);
    const long r = idx - (long)c * n;
    const int i = (int)(r % nx), k = (int)((r / nx) % nz), j = (int)(r / ((long)nx * nz));
    const int parity = c == 0 ? p0 : c == 1 ? p1 : p2;
    const double *f = in + (long)c * n;
    const long row = ((long)j * nz + k) * nx;
    const double v = f[row + i];
    if (parity < 0 && (j == 0 || j == ny - 1)) { out[idx] = v; return; }
    const double lx = (f[row + (i + 1 == nx ? 0 : i + 1)] - 2.0 * v + f[row + (i == 0 ? nx - 1 : i - 1)]) * ihx2;
    const long plane = (long)nz * nx;
    const long kp = (long)(k + 1 == nz ? 0 : k + 1) * nx, km = (long)(k == 0 ? nz - 1 : k - 1) * nx;
    const double lz = (f[(long)j * plane + kp + i] - 2.0 * v + f[(long)j * plane + km + i]) * ihz2;
    double ly;
    if (j > 0 && j < ny - 1) {
        const double hm = y[j] - y[j - 1], hp = y[j + 1] - y[j];
        ly = 2.0 / (hm + hp) * ((f[row + plane + i] - v) / hp - (v - f[row - plane + i]) / hm);
    } else {
        const double h = j == 0 ? y[1] - y[0] : y[ny - 1] - y[ny - 2];
        const double inner = f[row + (j == 0 ? plane : -plane) + i];
        ly = 2.0 * (inner - v) / (h * h);
    }
    out[idx] = v - a2 * (lx + lz + ly);
}

bool factor23(int n, int *rad, int *nrad)
{
    *nrad = 0;
    while (n % 3 == 0) { rad[(*nrad)++] = 3; n /= 3; }
    while (n % 2 == 0) { rad[(*nrad)++] = 2; n /= 2; }
    return n == 1 && *nrad <= 32;
}

std::vector<double2> twiddles(int n)
{
    std::vector<double2> t(n);
    for (int m = 0; m < n; m++) {
        const long double ang = -2.0L * 3.141592653589793238462643383279503L * m / n;
        t[m] = make_double2((double)cosl(ang), (double)sinl(ang));
    }
    return t;
}

}  // namespace

int diff_setup(ef_plan *p, const double *dns_y, const double *les_y)
{
    if (p->prec != EF_PREC_FP64) {
        set_error("the differential filter is implemented in FP64 (EF_PREC_FP64)");
        return EF_ERR_UNSUPPORTED;
    }
    if (p->ext != EF_EXT_EVEN_ODD && p->ext != EF_EXT_ODD_EVEN) {
        set_error("the differential filter needs a wall extension (Eq. 7 or Eq. 9)");
        return EF_ERR_ARG;
    }
    DiffPlan *d = new DiffPlan();
    p->diff = d;
    if (!factor23(p->nx, d->radx, &d->nradx) || !factor23(p->nz, d->radz, &d->nradz) || p->nx > kDiffMaxN ||
        p->nz > kDiffMaxN) {
        set_error("the differential filter needs nx and nz of the form 2^p 3^q, at most %d", kDiffMaxN);
        return EF_ERR_SHAPE;
    }
    if (p->nx % p->nlx || p->nz % p->nlz) {
        set_error("the differential filter needs LES x and z nodes on DNS nodes (nx %% nlx = nz %% nlz = 0)");
        return EF_ERR_SHAPE;
    }
    std::vector<int> jy(p->nly);
    for (int J = 0, j = 0; J < p->nly; J++) {
        while (j < p->ny && dns_y[j] < les_y[J]) j++;
        if (j >= p->ny || dns_y[j] != les_y[J]) {
            set_error("the differential filter needs LES y nodes on DNS nodes");
            return EF_ERR_SHAPE;
        }
        jy[J] = j;
    }
    d->a = p->delta / sqrt(40.0);
    d->nxh = p->nx / 2 + 1;
    d->rx = p->nx / p->nlx;
    d->rz = p->nz / p->nlz;
    d->zcols = p->nz <= 512 ? 4 : 2;
    const double a2 = d->a * d->a, hx = p->Lx / p->nx, hz = p->Lz / p->nz;
    std::vector<double> k2x(d->nxh), k2z(p->nz), dyy(3 * (size_t)p->ny, 0.0);
    for (int m = 0; m < d->nxh; m++) k2x[m] = a2 * (2.0 - 2.0 * cos(2.0 * M_PI * m / p->nx)) / (hx * hx);
    for (int m = 0; m < p->nz; m++) k2z[m] = a2 * (2.0 - 2.0 * cos(2.0 * M_PI * m / p->nz)) / (hz * hz);
    const int ny = p->ny;
    for (int j = 0; j < ny; j++) {
        double lo = 0, ce = 0, up = 0;
        if (j > 0 && j < ny - 1) {
            const double hm = dns_y[j] - dns_y[j - 1], hp = dns_y[j + 1] - dns_y[j];
            lo = 2.0 / ((hm + hp) * hm);
            up = 2.0 / ((hm + hp) * hp);
            ce = -(lo + up);
        } else {                                  // even wall row: the mirror ghost is the inner neighbour
            const double h = j == 0 ? dns_y[1] - dns_y[0] : dns_y[ny - 1] - dns_y[ny - 2];
            const double c = 2.0 / (h * h);
            ce = -c;
            (j == 0 ? up : lo) = c;
        }
        dyy[j] = lo;
        dyy[ny + j] = ce;
        dyy[2 * ny + j] = up;
    }
    const auto twx = twiddles(p->nx), twz = twiddles(p->nz);
    const size_t nspec = (size_t)ny * p->nz * d->nxh;
    cudaError_t e = cudaSuccess;
#define DK(x) if (e == cudaSuccess) e = (x)
    DK(cudaMalloc(&d->twx, sizeof(double2) * p->nx));
    DK(cudaMalloc(&d->twz, sizeof(double2) * p->nz));
    DK(cudaMalloc(&d->k2x, sizeof(double) * d->nxh));
    DK(cudaMalloc(&d->k2z, sizeof(double) * p->nz));
    DK(cudaMalloc(&d->dyy, sizeof(double) * dyy.size()));
    DK(cudaMalloc(&d->jy, sizeof(int) * p->nly));
    DK(cudaMalloc(&d->spec, sizeof(double2) * nspec));
    DK(cudaMalloc(&d->fcp, sizeof(double) * 2 * nspec));
    DK(cudaMalloc(&d->finv, sizeof(double) * 2 * nspec));
    DK(cudaMalloc(&d->lesz, sizeof(double2) * (size_t)p->nly * p->nlz * d->nxh));
    DK(cudaMalloc(&d->fld, sizeof(double) * 9 * (size_t)p->nly * p->nlz * p->nlx));
    DK(cudaMemcpy(d->twx, twx.data(), sizeof(double2) * p->nx, cudaMemcpyHostToDevice));
    DK(cudaMemcpy(d->twz, twz.data(), sizeof(double2) * p->nz, cudaMemcpyHostToDevice));
    DK(cudaMemcpy(d->k2x, k2x.data(), sizeof(double) * d->nxh, cudaMemcpyHostToDevice));
    DK(cudaMemcpy(d->k2z, k2z.data(), sizeof(double) * p->nz, cudaMemcpyHostToDevice));
    DK(cudaMemcpy(d->dyy, dyy.data(), sizeof(double) * dyy.size(), cudaMemcpyHostToDevice));
    DK(cudaMemcpy(d->jy, jy.data(), sizeof(int) * p->nly, cudaMemcpyHostToDevice));
    const int zsm = (int)(2 * sizeof(double2) * (size_t)p->nz * d->zcols);
    DK(cudaFuncSetAttribute(dz_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, zsm));
    DK(cudaFuncSetAttribute(dz_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, zsm));
    for (int q = 0; q < 2 && e == cudaSuccess; q++) {
        DyArgs ya = {};
        ya.k2x = d->k2x; ya.k2z = d->k2z; ya.dyy = d->dyy; ya.a2 = a2;
        ya.ny = ny; ya.nz = p->nz; ya.nxh = d->nxh; ya.odd = q;
        const long nline = (long)p->nz * d->nxh;
        dy_factor<<<(unsigned)((nline + kDiffThreads - 1) / kDiffThreads), kDiffThreads>>>(ya, d->fcp + q * nspec,
                                                                                          d->finv + q * nspec);
        e = cudaGetLastError();
    }
    DK(cudaDeviceSynchronize());
#undef DK
    if (e != cudaSuccess) return cuda_fail(e, "differential filter setup");
    return EF_OK;
}

void diff_destroy(DiffPlan *d)
{
    if (!d) return;
    cudaFree(d->twx); cudaFree(d->twz); cudaFree(d->k2x); cudaFree(d->k2z); cudaFree(d->dyy); cudaFree(d->jy);
    cudaFree(d->spec); cudaFree(d->fcp); cudaFree(d->finv); cudaFree(d->lesz); cudaFree(d->fld);
    delete d;
}

int diff_run(ef_plan *p, int nsnap, const void *u_, void *ubar_, void *tau_, double *plane_mean, bool stress,
             cudaStream_t s)
{
    DiffPlan *d = p->diff;
    const int nfield = stress ? 9 : 3;
    const size_t npt = (size_t)p->nx * p->ny * p->nz, nles = (size_t)p->nlx * p->nly * p->nlz;
    const int pi[9] = {0, 1, 2, 0, 0, 0, 1, 1, 2}, pj[9] = {-1, -1, -1, 0, 1, 2, 1, 2, 2};
    const int xsm = (int)(2 * sizeof(double2) * p->nx);
    const int zsm = (int)(2 * sizeof(double2) * (size_t)p->nz * d->zcols);
    for (int sn = 0; sn < nsnap; sn++) {
        const double *u = static_cast<const double *>(u_) + sn * 3 * npt;
        for (int f = 0; f < nfield; f++) {
            const int parity = pj[f] < 0 ? p->par[pi[f]] : p->par[pi[f]] * p->par[pj[f]];
            DxFwdArgs xa;
            xa.u = u; xa.ca = pi[f]; xa.cb = pj[f]; xa.odd = parity < 0;
            xa.nx = p->nx; xa.ny = p->ny; xa.nz = p->nz; xa.nxh = d->nxh;
            memcpy(xa.rad, d->radx, sizeof xa.rad); xa.nrad = d->nradx;
            xa.tw = d->twx; xa.spec = d->spec;
            dx_forward<<<dim3((p->nz + 1) / 2, p->ny), kDiffThreads, xsm, s>>>(xa);
            DzArgs za;
            za.spec = d->spec; za.nz = p->nz; za.nxh = d->nxh; za.ncol = d->zcols;
            memcpy(za.rad, d->radz, sizeof za.rad); za.nrad = d->nradz;
            za.tw = d->twz; za.jy = d->jy; za.rz = d->rz; za.nlz = p->nlz; za.lesz = d->lesz;
            const int zgroups = (d->nxh + d->zcols - 1) / d->zcols;
            dz_forward<<<dim3(zgroups, p->ny), kDiffThreads, zsm, s>>>(za);
            if (f < 3 && plane_mean)
                plane_mean_from_spec<<<(p->ny + 127) / 128, 128, 0, s>>>(
                    d->spec, p->ny, p->nz, d->nxh, 1.0 / ((double)p->nx * p->nz), plane_mean + (sn * 3 + f) * p->ny);
            DyArgs ya;
            const size_t nspec = (size_t)p->ny * p->nz * d->nxh;
            ya.spec = d->spec; ya.k2x = d->k2x; ya.k2z = d->k2z; ya.dyy = d->dyy;
            ya.fcp = d->fcp + (parity < 0 ? nspec : 0);
            ya.finv = d->finv + (parity < 0 ? nspec : 0);
            ya.a2 = d->a * d->a; ya.ny = p->ny; ya.nz = p->nz; ya.nxh = d->nxh; ya.odd = parity < 0;
            const long nline = (long)p->nz * d->nxh;
            dy_solve<<<(unsigned)((nline + kDiffThreads - 1) / kDiffThreads), kDiffThreads, 0, s>>>(ya);
            dz_inverse<<<dim3(zgroups, p->nly), kDiffThreads, zsm, s>>>(za);
            DxInvArgs ia;
            ia.lesz = d->lesz; ia.out = d->fld + f * nles; ia.nx = p->nx; ia.nxh = d->nxh; ia.rx = d->rx;
            ia.nlx = p->nlx; ia.scale = 1.0 / ((double)p->nx * p->nz);
            memcpy(ia.rad, d->radx, sizeof ia.rad); ia.nrad = d->nradx; ia.tw = d->twx;
            dx_inverse<<<dim3(p->nlz, p->nly), kDiffThreads, xsm, s>>>(ia);
        }
        double *ubar = static_cast<double *>(ubar_) + sn * 3 * nles;
        double *tau = stress ? static_cast<double *>(tau_) + sn * 6 * nles : nullptr;
        diff_stress<<<(unsigned)((nles + 255) / 256), 256, 0, s>>>(d->fld, (long)nles, ubar, tau);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EF_OK : cuda_fail(e, "differential filter");
}

}  // namespace eles

using namespace eles;

extern "C" int ef_differential_unfilter(const ef_grid *g, double delta, int extension, const double *in, double *out,
                                        void *stream)
{
    if (!g || !g->y || !in || !out || in == out) {
        set_error("ef_differential_unfilter: NULL or aliased argument");
        return EF_ERR_ARG;
    }
    if (!(delta > 0) || (extension != EF_EXT_EVEN_ODD && extension != EF_EXT_ODD_EVEN)) {
        set_error("ef_differential_unfilter: needs delta > 0 and a wall extension (Eq. 7 or Eq. 9)");
        return EF_ERR_ARG;
    }
    if (g->nx < 3 || g->nz < 3 || g->ny < 3) { set_error("ef_differential_unfilter: grid too small"); return EF_ERR_SHAPE; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *dy = nullptr;
    cudaError_t e = cudaMallocAsync(&dy, sizeof(double) * g->ny, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy, g->y, sizeof(double) * g->ny, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "ef_differential_unfilter");
    const double hx = g->Lx / g->nx, hz = g->Lz / g->nz, a2 = delta * delta / 40.0;
    const int flip = extension == EF_EXT_ODD_EVEN;
    const long n3 = 3L * g->nx * g->ny * g->nz;
    unfilter_kernel<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(in, out, dy, g->nx, g->ny, g->nz, 1.0 / (hx * hx),
                                                                1.0 / (hz * hz), a2, flip ? -1 : 1, flip ? 1 : -1,
                                                                flip ? -1 : 1);
    e = cudaGetLastError();
    cudaFreeAsync(dy, s);
    return e == cudaSuccess ? EF_OK : cuda_fail(e, "ef_differential_unfilter");
}
