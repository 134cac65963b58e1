// The differential filter of Sec. 3 on the GPU, in FP64 or FP32.
//
// The filter the paper's simulations use is the Green's function of
// (1 - a^2 lap): ubar solves (1 - a^2 lap) ubar = u on the domain extended
// across the walls (Eq. 7, or Eq. 9), periodic in x and z.  The Laplacian is
// the second-order finite-difference one on the DNS nodes (three-point
// periodic in x and z, the three-point non-uniform stencil in y with mirror
// ghosts of the field's parity at both walls), and a^2 = Delta_f^2 / 40.
// The kernel is not a product of one-dimensional kernels, so this path does
// not share the separable contractions of the Gaussian filter.  Per field:
//   1. form the field and transform each (y, z) row in x (two real rows per
//      complex transform);
//   2. transform each (y, kx) column in z (the periodic stencils become
//      diagonal: lap -> -(2 - 2 cos(k h)) / h^2);
//   3. solve the tridiagonal system in y for every (kx, kz) (Thomas, with the
//      factors precomputed per parity);
//   4. transform back in z only on the LES rows, keeping the LES z nodes;
//   5. transform back in x on those, keeping the LES x nodes (the LES nodes
//      are DNS nodes, so the linear interpolation of Sec. 3 is the identity).
// FP64 plans filter u_a and u_a u_b and form T_ab = bar(u_a u_b) - ubar_a
// ubar_b (Eq. 6) directly.  FP32 plans (the FP64 rate of GB300 is about a
// seventieth of its FP32 rate) filter fluctuations about the plane-mean
// profile U_c(y) so that no FP32 sum carries the mean: with u = U + u',
//   ubar_a = F(U_a) + F(u'_a),
//   T_ab = [F(U_a U_b) - F(U_a) F(U_b)] + [F(U_a u'_b) - F(U_a) F(u'_b)]
//        + [F(U_b u'_a) - F(U_b) F(u'_a)] + [F(u'_a u'_b) - F(u'_a) F(u'_b)],
// an identity of the linear filter.  The profiles' terms are one-dimensional
// (the kx = kz = 0 system) and solved in FP64, the eighteen fluctuation
// fields go through the FP32 transforms, and the brackets are formed in
// FP64.  The transforms are mixed-radix (2 and 3) Stockham FFTs in shared
// memory (the decimation-in-time formulation for GPUs of Govindaraju et al.,
// SC 2008); the inverse is the forward transform of the conjugate.
#include <math.h>
#include <string.h>

#include <vector>

#include "eles_internal.h"

namespace eles {

struct DiffPlan {
    int fp32 = 0;                         // FP32 transforms with the profile decomposition
    double a = 0;
    int nxh = 0;                          // nx / 2 + 1 kept x modes (real input)
    int n4x = 0, n2x = 0, n3x = 0, n4z = 0, n2z = 0, n3z = 0;   // radix-4, -2, -3 stages per axis
    void *twx = nullptr, *twz = nullptr;  // exp(-2 pi i m / N), m < N (plan precision)
    double *k2x = nullptr, *k2z = nullptr;    // a^2 (2 - 2 cos(2 pi m / N)) / h^2
    double *dyy = nullptr;                // [3][ny]: D_yy lower, centre, upper (interior and even walls)
    int *jy = nullptr;                    // [nly]: DNS row of each LES row
    int rx = 1, rz = 1;                   // DNS nodes per LES node in x and z
    int zcols = 4;                        // columns per CTA in the z transforms
    int nfield = 9;                       // filtered fields per snapshot
    int group = 3;                        // fields transformed and solved together (one launch per step)
    void *spec = nullptr;                 // [group][ny][nz][nxh] spectra of a group of fields
    void *fcp = nullptr, *finv = nullptr; // [2][ny][nz][nxh] Thomas factors per parity (even, odd)
    void *lesz = nullptr;                 // [group][nly][nlz][nxh]
    void *fld = nullptr;                  // [nfield][nly][nlz][nlx] filtered fields of one snapshot
    // FP32 plans: profile U_c(y) (FP64), its filtered terms at the LES rows, solver scratch
    double *U = nullptr;                  // [3][ny]
    double *FU = nullptr, *FUU = nullptr; // [3][nly], [6][nly]
    double *pscr = nullptr;               // [9][2][ny]
};

namespace {

constexpr int kDiffThreads = 256;
constexpr int kXThreads = 128;             // x transforms: N/4 butterflies per radix-4 stage
constexpr int kDiffMaxN = 1024;
constexpr int kMaxGroup = 6;

// A group of fields handled by one launch per step (blockIdx.z = member):
// member z is (u_ca - U_ca) [(u_cb - U_cb)] [U_pa] (profile terms on FP32
// plans only), of odd parity or not, filtered into row slot of fld.
struct FieldGroup {
    int n;
    int ca[kMaxGroup], cb[kMaxGroup], pa[kMaxGroup], odd[kMaxGroup], slot[kMaxGroup];
};

template <typename R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };
template <typename R> using cx = typename Cx<R>::T;

template <typename C> __device__ __forceinline__ C mk(double x, double y);
template <> __device__ __forceinline__ double2 mk<double2>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float2 mk<float2>(double x, double y) { return make_float2((float)x, (float)y); }

template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }

// Stockham stages over ncol independent transforms of length N held column
// by column (column c at b + c * N): n4 radix-4 stages, n2 radix-2 stages,
// then n3 radix-3 stages, so that the sub-transform length Ns is a power of
// two while it matters for the index arithmetic (shifts and masks).  Returns
// the buffer holding the result.
template <typename C>
__device__ C *smem_fft(C *b0, C *b1, int N, int ncol, int n4, int n2, int n3, const C *__restrict__ tw)
{
    using Rt = decltype(b0->x);
    int Ns = 1, lg = 0;
    const int nst = n4 + n2 + n3;
    for (int s = 0; s < nst; s++) {
        const int R = s < n4 ? 4 : s < n4 + n2 ? 2 : 3;
        const int NR = N / R, tstride = N / (Ns * R);
        const bool p2 = R != 3 || (Ns & (Ns - 1)) == 0;
        for (int t = threadIdx.x; t < NR * ncol; t += blockDim.x) {
            const int c = ncol == 1 ? 0 : t / NR, j = t - c * NR;
            const int k = p2 ? (j & (Ns - 1)) : j % Ns, jq = p2 ? (j >> lg) : j / Ns;
            const C *x = b0 + c * N;
            C *yv = b1 + c * N;
            const int d = jq * Ns * R + k;
            C v0 = x[j], v1 = x[j + NR];
            if (Ns > 1) v1 = cmul(v1, tw[tstride * k]);      // the first stage's twiddles are 1
            if (R == 4) {
                C v2 = x[j + 2 * NR], v3 = x[j + 3 * NR];
                if (Ns > 1) {
                    v2 = cmul(v2, tw[2 * tstride * k]);
                    v3 = cmul(v3, tw[3 * tstride * k]);
                }
                // radix 4: w = -i
                const C a0 = cadd(v0, v2), a1 = csub(v0, v2), c0 = cadd(v1, v3), c1 = csub(v1, v3);
                C mc1;
                mc1.x = c1.y; mc1.y = -c1.x;                            // -i c1
                yv[d] = cadd(a0, c0);
                yv[d + Ns] = cadd(a1, mc1);
                yv[d + 2 * Ns] = csub(a0, c0);
                yv[d + 3 * Ns] = csub(a1, mc1);
            } else if (R == 2) {
                yv[d] = cadd(v0, v1);
                yv[d + Ns] = csub(v0, v1);
            } else {
                // radix 3: w = exp(-2 pi i / 3); y1,2 = v0 - (v1 + v2) / 2 -/+ i (sqrt 3 / 2)(v1 - v2)
                C v2 = x[j + 2 * NR];
                if (Ns > 1) v2 = cmul(v2, tw[2 * tstride * k]);
                const C t1 = cadd(v1, v2), t2 = csub(v1, v2);
                const Rt h = (Rt)0.86602540378443864676;               // sqrt(3) / 2
                C m, base;
                m.x = h * t2.y; m.y = -h * t2.x;                        // -i h t2
                base.x = v0.x - (Rt)0.5 * t1.x;
                base.y = v0.y - (Rt)0.5 * t1.y;
                yv[d] = cadd(v0, t1);
                yv[d + Ns] = cadd(base, m);
                yv[d + 2 * Ns] = csub(base, m);
            }
        }
        __syncthreads();
        C *tmp = b0;
        b0 = b1;
        b1 = tmp;
        Ns *= R;
        lg += R == 4 ? 2 : R == 2 ? 1 : 0;
    }
    return b0;
}

template <typename R>
struct DxFwdArgs {
    const R *u;                           // [3][ny][nz][nx]
    FieldGroup grp;                       // the fields (member blockIdx.z)
    const double *U;                      // [3][ny] profile subtracted from u (NULL: none)
    int nx, ny, nz, nxh;
    int n4, n2, n3;                       // radix-4, -2, -3 stages
    const cx<R> *tw;
    cx<R> *spec;                          // [ny][nz][nxh]
};

// One CTA per (pair of z rows k0 = 2 b, k0 + 1; y row j): the two real rows
// are transformed together as z = f_k0 + i f_k1, and separated by the
// symmetry of real transforms: F_k0[m] = (Z[m] + conj Z[N-m]) / 2,
// F_k1[m] = (Z[m] - conj Z[N-m]) / (2i).
template <typename R>
__global__ void __launch_bounds__(kXThreads) dx_forward(const DxFwdArgs<R> a)
{
    using C = cx<R>;
    extern __shared__ __align__(16) unsigned char sraw[];
    C *b0 = reinterpret_cast<C *>(sraw), *b1 = b0 + a.nx;
    const int k0 = 2 * blockIdx.x, j = blockIdx.y, N = a.nx, g = blockIdx.z;
    const int ca = a.grp.ca[g], cb = a.grp.cb[g], pa = a.grp.pa[g];
    const bool two = k0 + 1 < a.nz;
    const size_t plane = (size_t)a.ny * a.nz * a.nx;
    const size_t row = ((size_t)j * a.nz + k0) * a.nx;
    const bool zero = a.grp.odd[g] && (j == 0 || j == a.ny - 1);
    const R Ua = a.U ? (R)a.U[ca * a.ny + j] : (R)0;
    const R Ub = (a.U && cb >= 0) ? (R)a.U[cb * a.ny + j] : (R)0;
    const R Pf = pa >= 0 ? (R)a.U[pa * a.ny + j] : (R)1;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        R v0 = a.u[ca * plane + row + i] - Ua, v1 = two ? a.u[ca * plane + row + N + i] - Ua : (R)0;
        if (cb >= 0) {
            v0 *= a.u[cb * plane + row + i] - Ub;
            if (two) v1 *= a.u[cb * plane + row + N + i] - Ub;
        }
        C z;
        z.x = zero ? (R)0 : v0 * Pf;
        z.y = zero ? (R)0 : v1 * Pf;
        b0[i] = z;
    }
    __syncthreads();
    const C *X = smem_fft(b0, b1, N, 1, a.n4, a.n2, a.n3, a.tw);
    C *out = a.spec + (size_t)g * a.ny * a.nz * a.nxh + ((size_t)j * a.nz + k0) * a.nxh;
    for (int m = threadIdx.x; m < a.nxh; m += blockDim.x) {
        const C zm = X[m], zc = X[m == 0 ? 0 : N - m];       // conj taken below
        C p, q;
        p.x = (R)0.5 * (zm.x + zc.x); p.y = (R)0.5 * (zm.y - zc.y);
        q.x = (R)0.5 * (zm.y + zc.y); q.y = (R)-0.5 * (zm.x - zc.x);
        out[m] = p;
        if (two) out[a.nxh + m] = q;
    }
}

template <typename R>
struct DzArgs {
    cx<R> *spec;                          // [group][ny][nz][nxh]
    int ny, nz, nxh, ncol;
    int n4, n2, n3;                       // radix-4, -2, -3 stages
    const cx<R> *tw;
    // inverse only: LES rows and output
    const int *jy;
    int rz, nlz;
    cx<R> *lesz;                          // [group][nly][nlz][nxh]
    int nly;
};

// Forward z transform in place: one CTA per (group of ncol x modes, y row, member).
template <typename R>
__global__ void __launch_bounds__(kDiffThreads) dz_forward(const DzArgs<R> a)
{
    using C = cx<R>;
    extern __shared__ __align__(16) unsigned char sraw[];
    const int N = a.nz, c0 = blockIdx.x * a.ncol, j = blockIdx.y;
    const int nc = min(a.ncol, a.nxh - c0);
    C *b0 = reinterpret_cast<C *>(sraw), *b1 = b0 + (size_t)N * a.ncol;
    C *base = a.spec + (size_t)blockIdx.z * a.ny * N * a.nxh + (size_t)j * N * a.nxh + c0;
    for (int t = threadIdx.x; t < N * a.ncol; t += blockDim.x) {
        const int k = t / a.ncol, c = t - k * a.ncol;
        b0[c * N + k] = c < nc ? base[(size_t)k * a.nxh + c] : mk<C>(0.0, 0.0);
    }
    __syncthreads();
    const C *Z = smem_fft(b0, b1, N, a.ncol, a.n4, a.n2, a.n3, a.tw);
    for (int t = threadIdx.x; t < N * a.ncol; t += blockDim.x) {
        const int k = t / a.ncol, c = t - k * a.ncol;
        if (c < nc) base[(size_t)k * a.nxh + c] = Z[c * N + k];
    }
}

// Inverse z transform of the LES rows (conjugate, forward transform,
// conjugate; the 1/(nx nz) scaling is applied at the end), keeping the LES
// z nodes.  One CTA per (group of x modes, LES row, member).
template <typename R>
__global__ void __launch_bounds__(kDiffThreads) dz_inverse(const DzArgs<R> a)
{
    using C = cx<R>;
    extern __shared__ __align__(16) unsigned char sraw[];
    const int N = a.nz, c0 = blockIdx.x * a.ncol, J = blockIdx.y, j = a.jy[J];
    const int nc = min(a.ncol, a.nxh - c0);
    C *b0 = reinterpret_cast<C *>(sraw), *b1 = b0 + (size_t)N * a.ncol;
    const C *base = a.spec + (size_t)blockIdx.z * a.ny * N * a.nxh + (size_t)j * N * a.nxh + c0;
    for (int t = threadIdx.x; t < N * a.ncol; t += blockDim.x) {
        const int k = t / a.ncol, c = t - k * a.ncol;
        C v = c < nc ? base[(size_t)k * a.nxh + c] : mk<C>(0.0, 0.0);
        v.y = -v.y;
        b0[c * N + k] = v;
    }
    __syncthreads();
    const C *Z = smem_fft(b0, b1, N, a.ncol, a.n4, a.n2, a.n3, a.tw);
    C *out = a.lesz + (size_t)blockIdx.z * a.nly * a.nlz * a.nxh + (size_t)J * a.nlz * a.nxh + c0;
    for (int t = threadIdx.x; t < a.nlz * a.ncol; t += blockDim.x) {
        const int K = t / a.ncol, c = t - K * a.ncol;
        C v = Z[c * N + K * a.rz];
        v.y = -v.y;
        if (c < nc) out[(size_t)K * a.nxh + c] = v;
    }
}

template <typename R>
struct DyArgs {
    cx<R> *spec;                          // [group][ny][nz][nxh], in place
    const R *fcp, *finv;                  // Thomas factors [2 parities][ny][nz][nxh]
    const double *k2x, *k2z, *dyy;        // a^2 k~^2 tables; D_yy [3][ny]
    double a2;
    int ny, nz, nxh, odd;                 // odd: the parity (set-up of the factors)
    FieldGroup grp;                       // the solve: member blockIdx.y and its parity
};

// The tridiagonal rows for (kz, kx), lam = a^2 (kx~^2 + kz~^2):
//   -a^2 lo_j v_{j-1} + (1 + lam - a^2 ce_j) v_j - a^2 up_j v_{j+1} = f_j,
// identity rows on the walls for an odd field.
__device__ __forceinline__ void dy_row(const double *dyy, double a2, int ny, int odd, double lam, int j, double &sub,
                                       double &dia, double &sup)
{
    if (odd && (j == 0 || j == ny - 1)) { sub = 0.0; dia = 1.0; sup = 0.0; return; }
    sub = -a2 * dyy[j];
    dia = 1.0 + lam - a2 * dyy[ny + j];
    sup = -a2 * dyy[2 * ny + j];
}

// Set-up, in FP64: the LU factors of the Thomas algorithm per line (they
// depend on the mode and the parity only, not on the field): c_j = sup_j /
// den_j and 1 / den_j with den_j = dia_j - sub_j c_{j-1}; stored in the
// plan's precision.
template <typename R>
__global__ void __launch_bounds__(kDiffThreads) dy_factor(DyArgs<R> a, R *fcp, R *finv)
{
    const long line = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nline = (long)a.nz * a.nxh;
    if (line >= nline) return;
    const int kz = (int)(line / a.nxh), kx = (int)(line - (long)kz * a.nxh);
    const double lam = a.k2x[kx] + a.k2z[kz];
    double c = 0.0;
    for (int j = 0; j < a.ny; j++) {
        double sub, dia, sup;
        dy_row(a.dyy, a.a2, a.ny, a.odd, lam, j, sub, dia, sup);
        const double inv = 1.0 / (dia - sub * c);
        c = sup * inv;
        fcp[(size_t)j * nline + line] = (R)c;
        finv[(size_t)j * nline + line] = (R)inv;
    }
}

// Thomas algorithm per (kz, kx) with the precomputed factors: forward
// d_j = (f_j - sub_j d_{j-1}) / den_j, backward v_j = d_j - c_j v_{j+1}.
// Threads run along kx (coalesced).  Rows go in blocks of kTb whose loads are
// issued together (the solve is latency-bound: one line per thread).
constexpr int kTb = 8;

template <typename R>
__global__ void __launch_bounds__(kDiffThreads) dy_solve(const DyArgs<R> a0)
{
    using C = cx<R>;
    const long line = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nline = (long)a0.nz * a0.nxh;
    if (line >= nline) return;
    // this member's spectrum and the factors of its parity
    DyArgs<R> a = a0;
    const int z = blockIdx.y;
    const size_t nspec = (size_t)a0.ny * nline;
    a.odd = a0.grp.odd[z];
    a.spec = a0.spec + (size_t)z * nspec;
    a.fcp = a0.fcp + (a.odd ? nspec : 0);
    a.finv = a0.finv + (a.odd ? nspec : 0);
    C d = mk<C>(0.0, 0.0);
    for (int j0 = 0; j0 < a.ny; j0 += kTb) {
        C f[kTb];
        R inv[kTb];
#pragma unroll
        for (int i = 0; i < kTb; i++)
            if (j0 + i < a.ny) {
                const size_t o = (size_t)(j0 + i) * nline + line;
                f[i] = a.spec[o];
                inv[i] = a.finv[o];
            }
#pragma unroll
        for (int i = 0; i < kTb; i++) {
            const int j = j0 + i;
            if (j < a.ny) {
                const R sub = (a.odd && j == a.ny - 1) ? (R)0 : (R)(-a.a2 * a.dyy[j]);
                d.x = (f[i].x - sub * d.x) * inv[i];
                d.y = (f[i].y - sub * d.y) * inv[i];
                a.spec[(size_t)j * nline + line] = d;
            }
        }
    }
    C v = d;
    for (int j0 = a.ny - 2; j0 >= 0; j0 -= kTb) {
        C dj[kTb];
        R cj[kTb];
#pragma unroll
        for (int i = 0; i < kTb; i++)
            if (j0 - i >= 0) {
                const size_t o = (size_t)(j0 - i) * nline + line;
                dj[i] = a.spec[o];
                cj[i] = a.fcp[o];
            }
#pragma unroll
        for (int i = 0; i < kTb; i++) {
            const int j = j0 - i;
            if (j >= 0) {
                v.x = dj[i].x - cj[i] * v.x;
                v.y = dj[i].y - cj[i] * v.y;
                a.spec[(size_t)j * nline + line] = v;
            }
        }
    }
}

template <typename R>
struct DxInvArgs {
    const cx<R> *lesz;                    // [group][nly][nlz][nxh]
    R *out;                               // fld [nfield][nly][nlz][nlx]; member z writes row grp.slot[z]
    FieldGroup grp;
    int nly;
    int nx, nxh, rx, nlx;
    double scale;                         // 1 / (nx nz)
    int n4, n2, n3;                       // radix-4, -2, -3 stages
    const cx<R> *tw;
};

// Inverse x transform of one (LES z node, LES row, member): the Hermitian spectrum
// completed from the kept modes, conjugated, transformed, real part at the
// LES x nodes.
template <typename R>
__global__ void __launch_bounds__(kXThreads) dx_inverse(const DxInvArgs<R> a)
{
    using C = cx<R>;
    extern __shared__ __align__(16) unsigned char sraw[];
    C *b0 = reinterpret_cast<C *>(sraw), *b1 = b0 + a.nx;
    const int K = blockIdx.x, J = blockIdx.y, N = a.nx, nlz = gridDim.x, z = blockIdx.z;
    const C *X = a.lesz + (size_t)z * a.nly * nlz * a.nxh + ((size_t)J * nlz + K) * a.nxh;
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        C v;
        if (m < a.nxh) { v = X[m]; v.y = -v.y; }
        else v = X[N - m];                                    // conj of the conjugate-symmetric mode
        b0[m] = v;
    }
    __syncthreads();
    const C *Y = smem_fft(b0, b1, N, 1, a.n4, a.n2, a.n3, a.tw);
    R *o = a.out + (size_t)a.grp.slot[z] * a.nly * nlz * a.nlx + ((size_t)J * nlz + K) * a.nlx;
    for (int X0 = threadIdx.x; X0 < a.nlx; X0 += blockDim.x) o[X0] = (R)(Y[X0 * a.rx].x * a.scale);
}

// Plane means of a velocity component: the zero mode of each y row (FP64 plans).
__global__ void plane_mean_from_spec(const double2 *spec, int ny, int nz, int nxh, double scale, double *pm)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < ny) pm[j] = spec[(size_t)j * nz * nxh].x * scale;
}

// Plane means U_c(y_j) in FP64 (FP32 plans): one CTA per (j, c), fixed
// order.  A thread loads blocks of m = 8 of its values at once, sums each
// in FP32 with the error-free transformation s + e = a + b (Knuth's
// two-sum), carrying the rounding errors in e, and adds s and e to an FP64
// total, so FP64 adds and conversions run once per 4 values (FP64
// throughput, not bandwidth, bounded a plain FP64 sum).  Only the sum of the
// errors is rounded: at most m^2 u_32^2 (about 2e-13) of the block's largest
// partial sum.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__global__ void __launch_bounds__(256) plane_mean_sum(const float *__restrict__ u, int ny, int nxz, double *U)
{
    constexpr int kBlock = 8;
    __shared__ double sh[256];
    const int j = blockIdx.x, c = blockIdx.y, nt = blockDim.x;
    const float *row = u + ((size_t)c * ny + j) * nxz;
    double acc = 0.0;
    for (int i0 = threadIdx.x; i0 < nxz; i0 += kBlock * nt) {
        float v[kBlock];
#pragma unroll
        for (int k = 0; k < kBlock; k++) {             // the block's loads are issued together
            const int i = i0 + k * nt;
            v[k] = i < nxz ? __ldg(row + i) : 0.f;
        }
        float s = v[0], e = 0.f;
#pragma unroll
        for (int k = 1; k < kBlock; k++) {
            float err;
            two_sum(s, v[k], s, err);
            e = __fadd_rn(e, err);
        }
        acc += (double)s + (double)e;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) U[c * ny + j] = sh[0] / nxz;
}

// The profiles' filtered terms, FP64: F(U_c) (q < 3) and F(U_a U_b) (q >= 3)
// solve the kx = kz = 0 system; sampled at the LES rows.
__global__ void profile_filter(const double *__restrict__ U, const double *__restrict__ dyy, double a2, int ny,
                               const int *__restrict__ jy, int nly, int p0, int p1, int p2, double *scr, double *FU,
                               double *FUU)
{
    const int q = threadIdx.x;
    if (q >= 9) return;
    const int pi[9] = {0, 1, 2, 0, 0, 0, 1, 1, 2}, pj[9] = {-1, -1, -1, 0, 1, 2, 1, 2, 2};
    const int par[3] = {p0, p1, p2};
    const int odd = (pj[q] < 0 ? par[pi[q]] : par[pi[q]] * par[pj[q]]) < 0;
    double *cp = scr + (size_t)q * 2 * ny, *dp = cp + ny;
    double c = 0.0, d = 0.0;
    for (int j = 0; j < ny; j++) {
        double sub, dia, sup;
        dy_row(dyy, a2, ny, odd, 0.0, j, sub, dia, sup);
        double f = U[pi[q] * ny + j] * (pj[q] < 0 ? 1.0 : U[pj[q] * ny + j]);
        if (odd && (j == 0 || j == ny - 1)) f = 0.0;
        const double inv = 1.0 / (dia - sub * c);
        c = sup * inv;
        d = (f - sub * d) * inv;
        cp[j] = c;
        dp[j] = d;
    }
    double v = d;
    for (int j = ny - 2; j >= 0; j--) {
        v = dp[j] - cp[j] * v;
        dp[j] = v;
    }
    for (int J = 0; J < nly; J++) {
        const double val = dp[jy[J]];
        if (q < 3) FU[q * nly + J] = val;
        else FUU[(q - 3) * nly + J] = val;
    }
}

// FP64 plans: ubar_c = F(u_c); T_q = F(u_i u_j) - F(u_i) F(u_j).
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

// FP32 plans: the decomposition's brackets in FP64.  Fields: 0-2 u'_c,
// 3-8 u'_a u'_b (pair order), 9 + 3a + b U_a u'_b.
__global__ void diff_recover32(const float *__restrict__ fld, long n, int nplane, const double *__restrict__ FU,
                               const double *__restrict__ FUU, int nly, float *ubar, float *tau)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int J = (int)(i / nplane);
    const int pi[6] = {0, 0, 0, 1, 1, 2}, pj[6] = {0, 1, 2, 1, 2, 2};
    double fu[3], fp[3];
    for (int c = 0; c < 3; c++) {
        fu[c] = FU[c * nly + J];
        fp[c] = (double)fld[c * n + i];
        ubar[c * n + i] = (float)(fu[c] + fp[c]);
    }
    if (!tau) return;
    for (int q = 0; q < 6; q++) {
        const int a = pi[q], b = pj[q];
        const double t = (FUU[q * nly + J] - fu[a] * fu[b])
                       + ((double)fld[(9 + 3 * a + b) * n + i] - fu[a] * fp[b])
                       + ((double)fld[(9 + 3 * b + a) * n + i] - fu[b] * fp[a])
                       + ((double)fld[(3 + q) * n + i] - fp[a] * fp[b]);
        tau[q * n + i] = (float)t;
    }
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

// n = 4^n4 2^n2 3^n3 with n2 <= 1; false if n has another prime factor.
bool factor423(int n, int *n4, int *n2, int *n3)
{
    *n4 = *n2 = *n3 = 0;
    while (n % 4 == 0) { (*n4)++; n /= 4; }
    while (n % 2 == 0) { (*n2)++; n /= 2; }
    while (n % 3 == 0) { (*n3)++; n /= 3; }
    return n == 1;
}

template <typename C>
std::vector<C> twiddles(int n)
{
    std::vector<C> t(n);
    for (int m = 0; m < n; m++) {
        const long double ang = -2.0L * 3.141592653589793238462643383279503L * m / n;
        t[m].x = (decltype(t[m].x))cosl(ang);
        t[m].y = (decltype(t[m].x))sinl(ang);
    }
    return t;
}

template <typename R>
int diff_setup_typed(ef_plan *p, DiffPlan *d)
{
    using C = cx<R>;
    const int ny = p->ny;
    const size_t nspec = (size_t)ny * p->nz * d->nxh;
    const size_t nles = (size_t)p->nly * p->nlz * p->nlx;
    const auto twx = twiddles<C>(p->nx), twz = twiddles<C>(p->nz);
    cudaError_t e = cudaSuccess;
#define DK(x) if (e == cudaSuccess) e = (x)
    DK(dev_malloc(&d->twx, sizeof(C) * p->nx));
    DK(dev_malloc(&d->twz, sizeof(C) * p->nz));
    DK(dev_malloc(&d->spec, sizeof(C) * nspec * d->group));
    DK(dev_malloc(&d->fcp, sizeof(R) * 2 * nspec));
    DK(dev_malloc(&d->finv, sizeof(R) * 2 * nspec));
    DK(dev_malloc(&d->lesz, sizeof(C) * (size_t)p->nly * p->nlz * d->nxh * d->group));
    DK(dev_malloc(&d->fld, sizeof(R) * d->nfield * nles));
    DK(cudaMemcpy(d->twx, twx.data(), sizeof(C) * p->nx, cudaMemcpyHostToDevice));
    DK(cudaMemcpy(d->twz, twz.data(), sizeof(C) * p->nz, cudaMemcpyHostToDevice));
    const int zsm = (int)(2 * sizeof(C) * (size_t)p->nz * d->zcols);
    DK(cudaFuncSetAttribute(dz_forward<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, zsm));
    DK(cudaFuncSetAttribute(dz_inverse<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, zsm));
    for (int q = 0; q < 2 && e == cudaSuccess; q++) {
        DyArgs<R> ya = {};
        ya.k2x = d->k2x; ya.k2z = d->k2z; ya.dyy = d->dyy; ya.a2 = d->a * d->a;
        ya.ny = ny; ya.nz = p->nz; ya.nxh = d->nxh; ya.odd = q;
        const long nline = (long)p->nz * d->nxh;
        dy_factor<R><<<(unsigned)((nline + kDiffThreads - 1) / kDiffThreads), kDiffThreads>>>(
            ya, static_cast<R *>(d->fcp) + q * nspec, static_cast<R *>(d->finv) + q * nspec);
        e = cudaGetLastError();
    }
    if (d->fp32) {
        DK(dev_malloc(&d->U, sizeof(double) * 3 * ny));
        DK(dev_malloc(&d->FU, sizeof(double) * 3 * p->nly));
        DK(dev_malloc(&d->FUU, sizeof(double) * 6 * p->nly));
        DK(dev_malloc(&d->pscr, sizeof(double) * 18 * ny));
    }
    DK(cudaDeviceSynchronize());
#undef DK
    if (e != cudaSuccess) return cuda_fail(e, "differential filter setup");
    return EF_OK;
}

// A group of fields through the five transform/solve steps, one launch per
// step for the whole group (member = blockIdx.z; blockIdx.y in the solve);
// member m lands in fld row g.slot[m].  With plane_mean set, members 0..2
// are the velocity components and their plane means are read from the zero
// modes (FP64 plans).
template <typename R>
void run_group(ef_plan *p, DiffPlan *d, const R *u, const FieldGroup &g, const double *U, double *plane_mean,
               cudaStream_t s)
{
    using C = cx<R>;
    const size_t nspec = (size_t)p->ny * p->nz * d->nxh;
    const int xsm = (int)(2 * sizeof(C) * p->nx);
    const int zsm = (int)(2 * sizeof(C) * (size_t)p->nz * d->zcols);
    DxFwdArgs<R> xa;
    xa.u = u; xa.grp = g; xa.U = U;
    xa.nx = p->nx; xa.ny = p->ny; xa.nz = p->nz; xa.nxh = d->nxh;
    xa.n4 = d->n4x; xa.n2 = d->n2x; xa.n3 = d->n3x;
    xa.tw = static_cast<const C *>(d->twx); xa.spec = static_cast<C *>(d->spec);
    dx_forward<R><<<dim3((p->nz + 1) / 2, p->ny, g.n), kXThreads, xsm, s>>>(xa);
    DzArgs<R> za;
    za.spec = static_cast<C *>(d->spec); za.ny = p->ny; za.nz = p->nz; za.nxh = d->nxh; za.ncol = d->zcols;
    za.n4 = d->n4z; za.n2 = d->n2z; za.n3 = d->n3z;
    za.tw = static_cast<const C *>(d->twz); za.jy = d->jy; za.rz = d->rz; za.nlz = p->nlz;
    za.lesz = static_cast<C *>(d->lesz); za.nly = p->nly;
    const int zgroups = (d->nxh + d->zcols - 1) / d->zcols;
    dz_forward<R><<<dim3(zgroups, p->ny, g.n), kDiffThreads, zsm, s>>>(za);
    if (plane_mean)
        for (int c = 0; c < 3; c++)
            plane_mean_from_spec<<<(p->ny + 127) / 128, 128, 0, s>>>(
                static_cast<const double2 *>(d->spec) + c * nspec, p->ny, p->nz, d->nxh,
                1.0 / ((double)p->nx * p->nz), plane_mean + c * p->ny);
    DyArgs<R> ya = {};
    ya.spec = static_cast<C *>(d->spec); ya.k2x = d->k2x; ya.k2z = d->k2z; ya.dyy = d->dyy;
    ya.fcp = static_cast<const R *>(d->fcp);
    ya.finv = static_cast<const R *>(d->finv);
    ya.a2 = d->a * d->a; ya.ny = p->ny; ya.nz = p->nz; ya.nxh = d->nxh; ya.grp = g;
    const long nline = (long)p->nz * d->nxh;
    dy_solve<R><<<dim3((unsigned)((nline + kDiffThreads - 1) / kDiffThreads), g.n), kDiffThreads, 0, s>>>(ya);
    dz_inverse<R><<<dim3(zgroups, p->nly, g.n), kDiffThreads, zsm, s>>>(za);
    DxInvArgs<R> ia;
    ia.lesz = static_cast<const C *>(d->lesz); ia.out = static_cast<R *>(d->fld); ia.grp = g; ia.nly = p->nly;
    ia.nx = p->nx; ia.nxh = d->nxh; ia.rx = d->rx; ia.nlx = p->nlx; ia.scale = 1.0 / ((double)p->nx * p->nz);
    ia.n4 = d->n4x; ia.n2 = d->n2x; ia.n3 = d->n3x; ia.tw = static_cast<const C *>(d->twx);
    dx_inverse<R><<<dim3(p->nlz, p->nly, g.n), kXThreads, xsm, s>>>(ia);
}

// The fields of one snapshot, in fld row order: u'_c (rows 0..2), u'_a u'_b
// (3..8, pairs (a, b) of the upper triangle) and, on FP32 plans, U_a u'_b
// (9 + 3 a + b); split into groups of `group` members.  The parity of a
// product is the product of the parities.
int snapshot_groups(const ef_plan *p, bool fp32, bool stress, int group, FieldGroup *grp)
{
    const int pi[6] = {0, 0, 0, 1, 1, 2}, pj[6] = {0, 1, 2, 1, 2, 2};
    int n = 0;
    auto add = [&](int ca, int cb, int pa, int parity) {
        FieldGroup &g = grp[n / group];
        const int m = n % group;
        g.n = m + 1;
        g.ca[m] = ca; g.cb[m] = cb; g.pa[m] = pa; g.odd[m] = parity < 0; g.slot[m] = n;
        n++;
    };
    for (int c = 0; c < 3; c++) add(c, -1, -1, p->par[c]);
    if (stress) {
        for (int q = 0; q < 6; q++) add(pi[q], pj[q], -1, p->par[pi[q]] * p->par[pj[q]]);
        if (fp32)
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) add(b, -1, a, p->par[a] * p->par[b]);
    }
    return (n + group - 1) / group;
}

}  // namespace

int diff_setup(ef_plan *p, const double *dns_y, const double *les_y)
{
    if (p->prec != EF_PREC_FP64 && p->prec != EF_PREC_FP32) {
        set_error("the differential filter is implemented in FP64 and FP32 (EF_PREC_FP64, EF_PREC_FP32)");
        return EF_ERR_UNSUPPORTED;
    }
    if (p->ext != EF_EXT_EVEN_ODD && p->ext != EF_EXT_ODD_EVEN) {
        set_error("the differential filter needs a wall extension (Eq. 7 or Eq. 9)");
        return EF_ERR_ARG;
    }
    DiffPlan *d = new DiffPlan();
    p->diff = d;
    if (!factor423(p->nx, &d->n4x, &d->n2x, &d->n3x) || !factor423(p->nz, &d->n4z, &d->n2z, &d->n3z) ||
        p->nx > kDiffMaxN || p->nz > kDiffMaxN) {
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
    d->fp32 = p->prec == EF_PREC_FP32;
    d->nfield = d->fp32 ? 18 : 9;
    d->group = d->fp32 ? 6 : 3;
    d->a = p->delta / sqrt(40.0);
    d->nxh = p->nx / 2 + 1;
    d->rx = p->nx / p->nlx;
    d->rz = p->nz / p->nlz;
    // z columns per CTA: shared memory 2 N zcols complex values (<= 48 KB FP32, 96 KB FP64)
    d->zcols = p->prec == EF_PREC_FP32 ? (p->nz <= 384 ? 8 : 4) : (p->nz <= 512 ? 4 : 2);
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
    cudaError_t e = dev_malloc(&d->k2x, sizeof(double) * d->nxh);
    if (e == cudaSuccess) e = dev_malloc(&d->k2z, sizeof(double) * p->nz);
    if (e == cudaSuccess) e = dev_malloc(&d->dyy, sizeof(double) * dyy.size());
    if (e == cudaSuccess) e = dev_malloc(&d->jy, sizeof(int) * p->nly);
    if (e == cudaSuccess) e = cudaMemcpy(d->k2x, k2x.data(), sizeof(double) * d->nxh, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d->k2z, k2z.data(), sizeof(double) * p->nz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d->dyy, dyy.data(), sizeof(double) * dyy.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d->jy, jy.data(), sizeof(int) * p->nly, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "differential filter setup");
    return d->fp32 ? diff_setup_typed<float>(p, d) : diff_setup_typed<double>(p, d);
}

void diff_destroy(DiffPlan *d)
{
    if (!d) return;
    cudaFree(d->twx); cudaFree(d->twz); cudaFree(d->k2x); cudaFree(d->k2z); cudaFree(d->dyy); cudaFree(d->jy);
    cudaFree(d->spec); cudaFree(d->fcp); cudaFree(d->finv); cudaFree(d->lesz); cudaFree(d->fld);
    cudaFree(d->U); cudaFree(d->FU); cudaFree(d->FUU); cudaFree(d->pscr);
    delete d;
}

int diff_run(ef_plan *p, int nsnap, const void *u_, void *ubar_, void *tau_, double *plane_mean, bool stress,
             cudaStream_t s)
{
    NvtxRange nv("differential filter");
    DiffPlan *d = p->diff;
    const size_t npt = (size_t)p->nx * p->ny * p->nz, nles = (size_t)p->nlx * p->nly * p->nlz;
    // the first group holds the three velocity components (d->group >= 3)
    FieldGroup grp[18 / 3];
    const int ng = snapshot_groups(p, d->fp32, stress, d->group, grp);
    for (int sn = 0; sn < nsnap; sn++) {
        if (!d->fp32) {
            const double *u = static_cast<const double *>(u_) + sn * 3 * npt;
            for (int k = 0; k < ng; k++)
                run_group<double>(p, d, u, grp[k], nullptr, (k == 0 && plane_mean) ? plane_mean + sn * 3 * p->ny : nullptr,
                                  s);
            double *ubar = static_cast<double *>(ubar_) + sn * 3 * nles;
            double *tau = stress ? static_cast<double *>(tau_) + sn * 6 * nles : nullptr;
            diff_stress<<<(unsigned)((nles + 255) / 256), 256, 0, s>>>(static_cast<const double *>(d->fld), (long)nles,
                                                                      ubar, tau);
        } else {
            const float *u = static_cast<const float *>(u_) + sn * 3 * npt;
            plane_mean_sum<<<dim3(p->ny, 3), 256, 0, s>>>(u, p->ny, p->nx * p->nz, d->U);
            if (plane_mean)
                cudaMemcpyAsync(plane_mean + sn * 3 * p->ny, d->U, sizeof(double) * 3 * p->ny,
                                cudaMemcpyDeviceToDevice, s);
            profile_filter<<<1, 32, 0, s>>>(d->U, d->dyy, d->a * d->a, p->ny, d->jy, p->nly, p->par[0], p->par[1],
                                            p->par[2], d->pscr, d->FU, d->FUU);
            for (int k = 0; k < ng; k++) run_group<float>(p, d, u, grp[k], d->U, nullptr, s);
            float *ubar = static_cast<float *>(ubar_) + sn * 3 * nles;
            float *tau = stress ? static_cast<float *>(tau_) + sn * 6 * nles : nullptr;
            diff_recover32<<<(unsigned)((nles + 255) / 256), 256, 0, s>>>(
                static_cast<const float *>(d->fld), (long)nles, p->nlx * p->nlz, d->FU, d->FUU, p->nly, ubar, tau);
        }
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
    cudaError_t e = dev_malloc_async(&dy, sizeof(double) * g->ny, s);
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
