// A minimal explicitly filtered LES step driven by the exact subfilter stress
// (Sec. 3, Fig. 2): at every step the DNS field is filtered, T_ij of Eq. 6 is
// formed, and the discrete filtered equations (Eq. 6: Eq. 5 with bar(u_i u_j)
// written as ubar_i ubar_j + T_ij) are advanced on the LES nodes with it.
//
// Discretisation (the paper's LES is a staggered second-order code with a
// fractional-step method and a third-order Runge-Kutta scheme; this is its
// collocated counterpart on the nodes where the filter samples ubar and T):
//   * second-order central differences: periodic in x and z,
//     (f[j+1] - f[j-1]) / (y[j+1] - y[j-1]) in y; the three-point Laplacian
//     (non-uniform in y);
//   * R_i = -d_j (ubar_i ubar_j + T_ij) + nu lap ubar_i + Pi [i = 1] at the
//     interior nodes, Pi the imposed mean pressure gradient;
//   * wall rows (Eq. 10 and Eq. 11): ubar_2 = 0, ubar_1 and ubar_3 the
//     filter-consistent value F(u_i), given by the filtered DNS of the step
//     (zero without one);
//   * low-storage RK3 (gamma 8/15 5/12 3/4, zeta 0 -17/60 -5/12) with a
//     projection after every substep: u = u* - G phi with phi = 0 on the
//     walls and D G phi = D u* at the interior nodes.  That is the orthogonal
//     projection, in the inner product weighted by (y[j+1] - y[j-1]) / 2, onto
//     the fields of zero discrete divergence (G is minus the adjoint of D in
//     that inner product), so the divergence after it is zero to rounding.
//
// The projection: a discrete Fourier transform in x (real to half complex)
// and z, per mode (m, q) the system D G phi = b in y, and the inverse
// transforms.  With central differences D G couples node j to j - 2 and
// j + 2 only, so each mode splits into two tridiagonal chains (even and odd
// j), solved by the Thomas algorithm with real coefficients and a complex
// right-hand side:
//     cm_j phi_{j-2} - (cm_j + cp_j + k^2) phi_j + cp_j phi_{j+2} = b_j,
//     cm_j = 1 / (dl_j dl_{j-1}) if j - 1 is interior, cp_j = 1 / (dl_j dl_{j+1})
//     if j + 1 is interior (dl_j = y[j+1] - y[j-1]), a neighbour on a wall
//     being the fixed phi = 0, and k^2 = s_x^2 + s_z^2 with s = sin(k h) / h
//     the symbol of the periodic central difference.
// A chain whose rows all sum to zero (k^2 = 0 and no end next to a wall row)
// is singular, its null vector a constant on the chain that G maps to zero;
// its first unknown is set to zero (the right-hand side is consistent: the
// divergence telescopes to the wall values of u_2, which are zero).
//
// All arithmetic is FP64.  The transforms are Stockham FFTs (radices 4, 2,
// 3, 5, 7; one warp per line in shared memory, twiddles from host-built
// tables) for lines of at most 1024 points with no other prime factor, and
// plain sums over the same tables otherwise.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "eles_internal.h"

namespace {

constexpr int kLesThreads = 256;
constexpr int kLesMaxN = 4096;          // largest nx, ny, nz of an LES grid
constexpr int kLesMaxStages = 16;       // radix stages of one transform
constexpr int kLesFftMaxN = 1024;       // longest line transformed by the FFT kernels (32 KB per warp)
constexpr long kLesMaxPoints = 1L << 28; // largest LES grid (node indices fit 32-bit arithmetic)

// Twiddle and per-row tables (device), and the sizes they are for.
struct LesGeom {
    int nx, ny, nz, nxh;                 // nxh = nx / 2 + 1 x modes kept
    double hx, hz;
    double ix2, iz2, ixx, izz;           // 1 / (2 hx), 1 / (2 hz), 1 / hx^2, 1 / hz^2
    const double *dlinv;                 // [ny] 1 / (y[j+1] - y[j-1]) (interior rows)
    const double *lapm, *lapp;           // [ny] y-Laplacian weights of f[j-1] and f[j+1]
    const double *cm, *cp;               // [ny] chain couplings (above)
    const double *cosx, *sinx;           // [nx] cos, sin of 2 pi r / nx
    const double *cosz, *sinz;           // [nz]
    const double *k2x, *k2z;             // [nxh] s_x^2, [nz] s_z^2 (exact zeros where the symbol is zero)
    int nfx, nfz;                        // Stockham stages of the x and z transforms (0: plain sums)
    int fx[kLesMaxStages], fz[kLesMaxStages];   // their radices, in order (4, 2, 3, 5, 7)
};

__host__ __device__ inline int pair_of(int a, int b)
{
    // order 11, 12, 13, 22, 23, 33
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
}

template <typename TT>
__host__ __device__ inline double tau_at(const TT *tau, long N, int pair, long idx)
{
    return tau ? (double)tau[(long)pair * N + idx] : 0.0;
}

// Wall rows of u (in place): u_2 = 0, u_1 and u_3 from bc (or zero).
// Item w in [0, 2 nz nx): wall row (w / (nz nx)) (0 bottom, 1 top), node w % (nz nx).
template <typename TT>
__host__ __device__ inline void walls_point(const LesGeom &g, double *u, const TT *bc, long w)
{
    const int nxz = g.nz * g.nx;
    const long N = (long)nxz * g.ny;
    const int wi = (int)w;
    const long idx = (long)((wi / nxz) ? g.ny - 1 : 0) * nxz + wi % nxz;
    u[N + idx] = 0.0;
    u[idx] = bc ? (double)bc[idx] : 0.0;
    u[2 * N + idx] = bc ? (double)bc[2 * N + idx] : 0.0;
}

// R at node idx (interior rows); the RK3 update into ustar and R into rout.
// Wall rows: ustar takes u (its wall values), rout zero.
template <typename TT>
__host__ __device__ inline void rhs_point(const LesGeom &g, const double *u, const TT *tau, double nu,
                                          double forcing, double gdt, double zdt, int use_prev, double *ustar,
                                          double *rout, long idx)
{
    const int nx = g.nx, nz = g.nz, ny = g.ny;
    const long nxz = (long)nx * nz, N = nxz * ny;
    const int id = (int)idx, row = id / nx;
    const int i = id - row * nx, j = row / nz, k = row - j * nz;
    if (j == 0 || j == ny - 1) {
        for (int c = 0; c < 3; c++) {
            ustar[c * N + idx] = u[c * N + idx];
            rout[c * N + idx] = 0.0;
        }
        return;
    }
    const long base = (long)j * nxz + (long)k * nx;
    const long xp = base + (i + 1 == nx ? 0 : i + 1), xm = base + (i == 0 ? nx - 1 : i - 1);
    const long zrow = (long)j * nxz + i;
    const long zp = zrow + (long)(k + 1 == nz ? 0 : k + 1) * nx, zm = zrow + (long)(k == 0 ? nz - 1 : k - 1) * nx;
    const long yp = idx + nxz, ym = idx - nxz;
    const double ix2 = g.ix2, iz2 = g.iz2, ixx = g.ixx, izz = g.izz;
    const double dl = g.dlinv[j], wm = g.lapm[j], wp = g.lapp[j];
    for (int c = 0; c < 3; c++) {
        const double *uc = u + c * N;
        // flux F_cd = u_c u_d + T_cd at the neighbours along d
        const double fxp = uc[xp] * u[xp] + tau_at(tau, N, pair_of(c, 0), xp);
        const double fxm = uc[xm] * u[xm] + tau_at(tau, N, pair_of(c, 0), xm);
        const double fyp = uc[yp] * u[N + yp] + tau_at(tau, N, pair_of(c, 1), yp);
        const double fym = uc[ym] * u[N + ym] + tau_at(tau, N, pair_of(c, 1), ym);
        const double fzp = uc[zp] * u[2 * N + zp] + tau_at(tau, N, pair_of(c, 2), zp);
        const double fzm = uc[zm] * u[2 * N + zm] + tau_at(tau, N, pair_of(c, 2), zm);
        const double u0 = uc[idx];
        const double lapx = (uc[xp] - 2.0 * u0 + uc[xm]) * ixx;
        const double lapz = (uc[zp] - 2.0 * u0 + uc[zm]) * izz;
        const double lapy = wp * uc[yp] - (wp + wm) * u0 + wm * uc[ym];
        double R = -((fxp - fxm) * ix2 + (fyp - fym) * dl + (fzp - fzm) * iz2) + nu * (lapx + lapy + lapz);
        if (c == 0) R += forcing;
        double us = u0 + gdt * R;
        if (use_prev) us += zdt * rout[c * N + idx];
        ustar[c * N + idx] = us;
        rout[c * N + idx] = R;
    }
}

// Discrete divergence of ustar at node idx (zero on the wall rows).
__host__ __device__ inline void div_point(const LesGeom &g, const double *us, double *b, long idx)
{
    const int nx = g.nx, nz = g.nz, ny = g.ny;
    const long nxz = (long)nx * nz, N = nxz * ny;
    const int id = (int)idx, row = id / nx;
    const int i = id - row * nx, j = row / nz, k = row - j * nz;
    if (j == 0 || j == ny - 1) {
        b[idx] = 0.0;
        return;
    }
    const long base = (long)j * nxz + (long)k * nx;
    const long xp = base + (i + 1 == nx ? 0 : i + 1), xm = base + (i == 0 ? nx - 1 : i - 1);
    const long zrow = (long)j * nxz + i;
    const long zp = zrow + (long)(k + 1 == nz ? 0 : k + 1) * nx, zm = zrow + (long)(k == 0 ? nz - 1 : k - 1) * nx;
    b[idx] = (us[xp] - us[xm]) * g.ix2 + (us[N + idx + nxz] - us[N + idx - nxz]) * g.dlinv[j] +
             (us[2 * N + zp] - us[2 * N + zm]) * g.iz2;
}

// Forward x transform: B[j][k][m] = sum_i b[j][k][i] exp(-2 pi i m i / nx).
__host__ __device__ inline void dftx_fwd_point(const LesGeom &g, const double *b, double2 *B, long o)
{
    const int m = (int)(o % g.nxh);
    const long line = o / g.nxh;                       // j nz + k
    const double *row = b + line * g.nx;
    double re = 0.0, im = 0.0;
    int r = 0;                                         // m i mod nx
    for (int i = 0; i < g.nx; i++) {
        re += row[i] * g.cosx[r];
        im -= row[i] * g.sinx[r];
        r += m;
        if (r >= g.nx) r -= g.nx;
    }
    B[o] = make_double2(re, im);
}

// Forward z transform: C[j][q][m] = sum_k B[j][k][m] exp(-2 pi i q k / nz).
// Inverse (sgn = +1, scale 1 / nz) alike.
__host__ __device__ inline void dftz_point(const LesGeom &g, const double2 *src, double2 *dst, double sgn,
                                           double scale, long o)
{
    const int nxh = g.nxh, nz = g.nz;
    const int m = (int)(o % nxh), q = (int)((o / nxh) % nz);
    const long j = o / ((long)nxh * nz);
    const double2 *col = src + j * (long)nz * nxh + m;
    double re = 0.0, im = 0.0;
    int r = 0;                                         // q k mod nz
    for (int k = 0; k < nz; k++) {
        const double2 v = col[(long)k * nxh];
        const double c = g.cosz[r], s = sgn * g.sinz[r];
        re += v.x * c - v.y * s;
        im += v.x * s + v.y * c;
        r += q;
        if (r >= nz) r -= nz;
    }
    dst[o] = make_double2(re * scale, im * scale);
}

// The eliminated coefficients of every chain, which depend only on the mode:
// for chain row j, cw = c'_j and cinv = 1 / (b_j - a_j c'_{j-2}) of the Thomas
// forward sweep (host, at set-up).  The singular chain's first row is
// replaced by phi = 0: cinv = 0 there makes its eliminated right-hand side
// zero.  Layout [j][q][m] as C; wall rows unused.
void les_chain_tables(const LesGeom &g, std::vector<double> &cw, std::vector<double> &cinv)
{
    const int ny = g.ny, nz = g.nz, nxh = g.nxh;
    const long stride = (long)nz * nxh;
    cw.assign((size_t)ny * stride, 0.0);
    cinv.assign((size_t)ny * stride, 0.0);
    for (int q = 0; q < nz; q++)
        for (int m = 0; m < nxh; m++)
            for (int p = 0; p < 2; p++) {
                const int j0 = p ? 1 : 2;
                if (j0 > ny - 2) continue;
                int jl = ny - 2;
                if ((jl & 1) != p) jl--;
                const double k2 = g.k2x[m] + g.k2z[q];
                const bool singular = (k2 == 0.0) && (j0 == 1) && (jl == ny - 2);
                double cprev = 0.0;
                for (int j = j0; j <= jl; j += 2) {
                    const long o = (long)j * stride + (long)q * nxh + m;
                    const double a = (j - 2 >= 1) ? g.cm[j] : 0.0;
                    const double c = (j + 2 <= ny - 2) ? g.cp[j] : 0.0;
                    if (singular && j == j0) {
                        cw[o] = 0.0;
                        cinv[o] = 0.0;
                        cprev = 0.0;
                        continue;
                    }
                    const double den = (-g.cm[j] - g.cp[j] - k2) - a * cprev;
                    cw[o] = c / den;
                    cinv[o] = 1.0 / den;
                    cprev = cw[o];
                }
            }
}

// One chain of one mode: item t = (q nxh + m) * 2 + p, p = 0 for the chain
// of even j (starting at j = 2), 1 for odd j (starting at j = 1).  In place
// on C (right-hand side in, phi out) with the eliminated coefficients of
// les_chain_tables.  The chain's wall rows of C are set to zero (phi = 0 on
// the walls).
__host__ __device__ inline void chain_point(const LesGeom &g, double2 *__restrict__ C,
                                            const double *__restrict__ cw, const double *__restrict__ cinv,
                                            long t)
{
    const int p = (int)(t & 1);
    const int mode = (int)(t >> 1);
    const int q = mode / g.nxh, m = mode - q * g.nxh;
    const int ny = g.ny;
    const long stride = (long)g.nz * g.nxh;            // between rows j of one mode
    const long off = (long)q * g.nxh + m;
    double2 *col = C + off;
    if (p == 0) col[0] = make_double2(0.0, 0.0);
    if (((ny - 1) & 1) == p) col[(long)(ny - 1) * stride] = make_double2(0.0, 0.0);
    const int j0 = p ? 1 : 2;
    if (j0 > ny - 2) return;
    int jl = ny - 2;
    if ((jl & 1) != p) jl--;
    // forward elimination
    double2 dprev = make_double2(0.0, 0.0);
    for (int j = j0; j <= jl; j += 2) {
        const long o = (long)j * stride;
        const double a = (j - 2 >= 1) ? g.cm[j] : 0.0;
        const double2 rhs = col[o];
        const double inv = cinv[off + o];
        const double2 dn = make_double2((rhs.x - a * dprev.x) * inv, (rhs.y - a * dprev.y) * inv);
        col[o] = dn;
        dprev = dn;
    }
    // back substitution
    double2 next = col[(long)jl * stride];
    for (int j = jl - 2; j >= j0; j -= 2) {
        const long o = (long)j * stride;
        const double cn = cw[off + o];
        const double2 d = col[o];
        next = make_double2(d.x - cn * next.x, d.y - cn * next.y);
        col[o] = next;
    }
}

// Inverse x transform (half complex to real, scale 1 / nx) into phi.
__host__ __device__ inline void dftx_inv_point(const LesGeom &g, const double2 *B, double *phi, long idx)
{
    const int nx = g.nx, i = (int)(idx % nx);
    const long line = idx / nx;
    const double2 *row = B + line * g.nxh;
    double s = row[0].x;
    const int mtop = (nx - 1) / 2;                     // modes with a conjugate partner
    int r = i;                                         // m i mod nx
    for (int m = 1; m <= mtop; m++) {
        s += 2.0 * (row[m].x * g.cosx[r] - row[m].y * g.sinx[r]);
        r += i;
        if (r >= nx) r -= nx;
    }
    if ((nx & 1) == 0) s += (i & 1) ? -row[nx / 2].x : row[nx / 2].x;
    phi[idx] = s / nx;
}

// u = ustar - G phi at the interior rows; the wall rows keep ustar.
__host__ __device__ inline void correct_point(const LesGeom &g, const double *us, const double *phi, double *u,
                                              long idx)
{
    const int nx = g.nx, nz = g.nz, ny = g.ny;
    const long nxz = (long)nx * nz, N = nxz * ny;
    const int id = (int)idx, row = id / nx;
    const int i = id - row * nx, j = row / nz, k = row - j * nz;
    if (j == 0 || j == ny - 1) {
        for (int c = 0; c < 3; c++) u[c * N + idx] = us[c * N + idx];
        return;
    }
    const long base = (long)j * nxz + (long)k * nx;
    const long xp = base + (i + 1 == nx ? 0 : i + 1), xm = base + (i == 0 ? nx - 1 : i - 1);
    const long zrow = (long)j * nxz + i;
    const long zp = zrow + (long)(k + 1 == nz ? 0 : k + 1) * nx, zm = zrow + (long)(k == 0 ? nz - 1 : k - 1) * nx;
    u[idx] = us[idx] - (phi[xp] - phi[xm]) * g.ix2;
    u[N + idx] = us[N + idx] - (phi[idx + nxz] - phi[idx - nxz]) * g.dlinv[j];
    u[2 * N + idx] = us[2 * N + idx] - (phi[zp] - phi[zm]) * g.iz2;
}

// One radix-R stage (R in 2, 3, 4, 5, 7) of a length-n Stockham transform
// in natural order: butterfly j in [0, n / R), Ns the product of the radices
// of the earlier stages.  Its R inputs in[j + r n / R] are turned by
// exp(sgn 2 pi i r (j mod Ns) / (Ns R)), transformed by an R-point DFT and
// written to out[(j / Ns) Ns R + (j mod Ns) + q Ns].  sgn = -1 forward,
// +1 inverse (no scaling).  Twiddles from the length-n tables.
template <int R>
__host__ __device__ inline void stockham_stage_r(const double2 *in, double2 *out, int n, int Ns, int j, double sgn,
                                                 const double *cs, const double *sn)
{
    double2 v[R];
    const int k = j % Ns, span = n / R, tstep = n / (Ns * R);
#pragma unroll
    for (int r = 0; r < R; r++) {
        const double2 a = in[j + r * span];
        const int t = (r * k * tstep) % n;
        const double c = cs[t], si = sgn * sn[t];
        v[r] = make_double2(a.x * c - a.y * si, a.x * si + a.y * c);
    }
    const int base = (j / Ns) * Ns * R + k;
    if (R == 2) {
        out[base] = make_double2(v[0].x + v[1].x, v[0].y + v[1].y);
        out[base + Ns] = make_double2(v[0].x - v[1].x, v[0].y - v[1].y);
    } else if (R == 4) {
        const double2 t0 = make_double2(v[0].x + v[2 % R].x, v[0].y + v[2 % R].y);
        const double2 t1 = make_double2(v[0].x - v[2 % R].x, v[0].y - v[2 % R].y);
        const double2 t2 = make_double2(v[1].x + v[3 % R].x, v[1].y + v[3 % R].y);
        const double2 t3 = make_double2(v[1].x - v[3 % R].x, v[1].y - v[3 % R].y);
        const double2 wt3 = make_double2(-sgn * t3.y, sgn * t3.x);   // exp(sgn i pi / 2) t3
        out[base] = make_double2(t0.x + t2.x, t0.y + t2.y);
        out[base + Ns] = make_double2(t1.x + wt3.x, t1.y + wt3.y);
        out[base + 2 * Ns] = make_double2(t0.x - t2.x, t0.y - t2.y);
        out[base + 3 * Ns] = make_double2(t1.x - wt3.x, t1.y - wt3.y);
    } else {
        const int rstep = n / R;
#pragma unroll
        for (int q = 0; q < R; q++) {
            double re = v[0].x, im = v[0].y;
#pragma unroll
            for (int r = 1; r < R; r++) {
                const int t = (r * q * rstep) % n;
                const double c = cs[t], si = sgn * sn[t];
                re += v[r].x * c - v[r].y * si;
                im += v[r].x * si + v[r].y * c;
            }
            out[base + q * Ns] = make_double2(re, im);
        }
    }
}

// One radix-R stage (R in 2, 3, 4, 5, 7) of a length-n Stockham transform
// in natural order: butterfly j in [0, n / R), Ns the product of the radices
// of the earlier stages.  Its R inputs in[j + r n / R] are turned by
// exp(sgn 2 pi i r (j mod Ns) / (Ns R)), transformed by an R-point DFT and
// written to out[(j / Ns) Ns R + (j mod Ns) + q Ns].  sgn = -1 forward,
// +1 inverse (no scaling).  Twiddles from the length-n tables.
__host__ __device__ inline void stockham_stage(const double2 *in, double2 *out, int n, int Ns, int R, int j,
                                               double sgn, const double *cs, const double *sn)
{
    switch (R) {
    case 2: stockham_stage_r<2>(in, out, n, Ns, j, sgn, cs, sn); break;
    case 3: stockham_stage_r<3>(in, out, n, Ns, j, sgn, cs, sn); break;
    case 4: stockham_stage_r<4>(in, out, n, Ns, j, sgn, cs, sn); break;
    case 5: stockham_stage_r<5>(in, out, n, Ns, j, sgn, cs, sn); break;
    default: stockham_stage_r<7>(in, out, n, Ns, j, sgn, cs, sn); break;
    }
}

// ---- kernels: grid-stride loops over the items of each point function ----

#define LES_LOOP(n) for (long it = (long)blockIdx.x * blockDim.x + threadIdx.x; it < (n); it += (long)gridDim.x * blockDim.x)

template <typename TT>
__global__ void __launch_bounds__(kLesThreads) les_walls(LesGeom g, double *u, const TT *bc)
{
    LES_LOOP(2L * g.nz * g.nx) walls_point(g, u, bc, it);
}

template <typename TT>
__global__ void __launch_bounds__(kLesThreads) les_rhs(LesGeom g, const double *u, const TT *tau, double nu,
                                                        double forcing, double gdt, double zdt, int use_prev,
                                                        double *ustar, double *rout)
{
    LES_LOOP((long)g.nx * g.ny * g.nz) rhs_point(g, u, tau, nu, forcing, gdt, zdt, use_prev, ustar, rout, it);
}

__global__ void __launch_bounds__(kLesThreads) les_div(LesGeom g, const double *us, double *b)
{
    LES_LOOP((long)g.nx * g.ny * g.nz) div_point(g, us, b, it);
}

__global__ void __launch_bounds__(kLesThreads) les_dftx_fwd(LesGeom g, const double *b, double2 *B)
{
    LES_LOOP((long)g.nxh * g.ny * g.nz) dftx_fwd_point(g, b, B, it);
}

__global__ void __launch_bounds__(kLesThreads) les_dftz(LesGeom g, const double2 *src, double2 *dst, double sgn,
                                                         double scale)
{
    LES_LOOP((long)g.nxh * g.ny * g.nz) dftz_point(g, src, dst, sgn, scale, it);
}

__global__ void __launch_bounds__(kLesThreads) les_chain(LesGeom g, double2 *C, const double *cw, const double *cinv)
{
    LES_LOOP(2L * g.nxh * g.nz) chain_point(g, C, cw, cinv, it);
}

__global__ void __launch_bounds__(kLesThreads) les_dftx_inv(LesGeom g, const double2 *B, double *phi)
{
    LES_LOOP((long)g.nx * g.ny * g.nz) dftx_inv_point(g, B, phi, it);
}

__global__ void __launch_bounds__(kLesThreads) les_correct(LesGeom g, const double *us, const double *phi, double *u)
{
    LES_LOOP((long)g.nx * g.ny * g.nz) correct_point(g, us, phi, u, it);
}

#undef LES_LOOP

// Transforms by Stockham FFTs, one warp per line, the line in two shared
// buffers of n complex values per warp (lanes split each stage's butterflies;
// __syncwarp between stages).  W warps per block, each walking lines
// line0 = blockIdx.x W + warp, line0 + gridDim.x W, ...
__device__ inline double2 *warp_fft(double2 *a, double2 *b, int n, int nf, const int *f, double sgn,
                                    const double *cs, const double *sn, int lane)
{
    int Ns = 1;
    for (int s = 0; s < nf; s++) {
        const int R = f[s];
        for (int j = lane; j < n / R; j += 32) stockham_stage(a, b, n, Ns, R, j, sgn, cs, sn);
        __syncwarp();
        double2 *t = a; a = b; b = t;
        Ns *= R;
    }
    return a;
}

// Forward x: real rows b[line][0..nx) -> B[line][0..nxh).
__global__ void __launch_bounds__(128) les_fftx_fwd(LesGeom g, const double *b, double2 *B)
{
    extern __shared__ double2 fsm[];
    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31, n = g.nx;
    double2 *a0 = fsm + (size_t)warp * 2 * n, *b0 = a0 + n;
    const long lines = (long)g.ny * g.nz;
    for (long line = (long)blockIdx.x * W + warp; line < lines; line += (long)gridDim.x * W) {
        const double *row = b + line * n;
        for (int i = lane; i < n; i += 32) a0[i] = make_double2(row[i], 0.0);
        __syncwarp();
        const double2 *res = warp_fft(a0, b0, n, g.nfx, g.fx, -1.0, g.cosx, g.sinx, lane);
        double2 *dst = B + line * g.nxh;
        for (int m = lane; m < g.nxh; m += 32) dst[m] = res[m];
        __syncwarp();
    }
}

// Inverse x: B[line][0..nxh) (the Hermitian half) -> real rows phi[line][0..nx), scale 1 / nx.
__global__ void __launch_bounds__(128) les_fftx_inv(LesGeom g, const double2 *B, double *phi)
{
    extern __shared__ double2 fsm[];
    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31, n = g.nx;
    double2 *a0 = fsm + (size_t)warp * 2 * n, *b0 = a0 + n;
    const long lines = (long)g.ny * g.nz;
    const double inv = 1.0 / n;
    for (long line = (long)blockIdx.x * W + warp; line < lines; line += (long)gridDim.x * W) {
        const double2 *src = B + line * g.nxh;
        for (int m = lane; m < n; m += 32) {
            if (m < g.nxh) {
                a0[m] = src[m];
            } else {
                const double2 c = src[n - m];
                a0[m] = make_double2(c.x, -c.y);
            }
        }
        __syncwarp();
        const double2 *res = warp_fft(a0, b0, n, g.nfx, g.fx, 1.0, g.cosx, g.sinx, lane);
        double *dst = phi + line * n;
        for (int i = lane; i < n; i += 32) dst[i] = res[i].x * inv;
        __syncwarp();
    }
}

// z transform of the columns (j, m): src[j][k][m] -> dst[j][q][m], sign sgn, scale.
__global__ void __launch_bounds__(128) les_fftz(LesGeom g, const double2 *src, double2 *dst, double sgn,
                                                double scale)
{
    extern __shared__ double2 fsm[];
    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31, n = g.nz;
    double2 *a0 = fsm + (size_t)warp * 2 * n, *b0 = a0 + n;
    const long lines = (long)g.ny * g.nxh;
    for (long line = (long)blockIdx.x * W + warp; line < lines; line += (long)gridDim.x * W) {
        const long j = line / g.nxh, m = line % g.nxh;
        const double2 *col = src + j * (long)n * g.nxh + m;
        for (int k = lane; k < n; k += 32) a0[k] = col[(long)k * g.nxh];
        __syncwarp();
        const double2 *res = warp_fft(a0, b0, n, g.nfz, g.fz, sgn, g.cosz, g.sinz, lane);
        double2 *out = dst + j * (long)n * g.nxh + m;
        for (int q = lane; q < n; q += 32) out[(long)q * g.nxh] = make_double2(res[q].x * scale, res[q].y * scale);
        __syncwarp();
    }
}

inline int fft_warps(int n) { int w = 49152 / (32 * n); return w < 1 ? 1 : (w > 4 ? 4 : w); }

inline int blocks_for(long n)
{
    long b = (n + kLesThreads - 1) / kLesThreads;
    if (b > 152L * 8) b = 152L * 8;
    return (int)(b < 1 ? 1 : b);
}

// Host tables of LesGeom, packed: dlinv lapm lapp cm cp [ny] each, cosx sinx
// [nx], cosz sinz [nz], k2x [nx/2+1], k2z [nz].
void les_tables(int nx, int ny, int nz, double Lx, double Lz, const double *y, std::vector<double> &tab)
{
    const int nxh = nx / 2 + 1;
    const double hx = Lx / nx, hz = Lz / nz;
    tab.assign(5 * (size_t)ny + 2 * (size_t)nx + 3 * (size_t)nz + nxh, 0.0);
    double *dlinv = tab.data(), *lapm = dlinv + ny, *lapp = lapm + ny, *cm = lapp + ny, *cp = cm + ny;
    double *cosx = cp + ny, *sinx = cosx + nx, *cosz = sinx + nx, *sinz = cosz + nz, *k2x = sinz + nz,
           *k2z = k2x + nxh;
    for (int j = 1; j + 1 < ny; j++) {
        const double span = y[j + 1] - y[j - 1], hm = y[j] - y[j - 1], hp = y[j + 1] - y[j];
        dlinv[j] = 1.0 / span;
        lapm[j] = 2.0 / (span * hm);
        lapp[j] = 2.0 / (span * hp);
    }
    for (int j = 1; j + 1 < ny; j++) {
        if (j - 1 >= 1) cm[j] = dlinv[j] * dlinv[j - 1];
        if (j + 1 <= ny - 2) cp[j] = dlinv[j] * dlinv[j + 1];
    }
    const double twopi = 2.0 * M_PI;
    for (int r = 0; r < nx; r++) { cosx[r] = cos(twopi * r / nx); sinx[r] = sin(twopi * r / nx); }
    for (int r = 0; r < nz; r++) { cosz[r] = cos(twopi * r / nz); sinz[r] = sin(twopi * r / nz); }
    for (int m = 0; m < nxh; m++) {
        const bool zero = m == 0 || 2 * m == nx;       // the central difference annihilates these modes
        const double sx = zero ? 0.0 : sinx[m] / hx;
        k2x[m] = sx * sx;
    }
    for (int q = 0; q < nz; q++) {
        const bool zero = q == 0 || 2 * q == nz;
        const double sz = zero ? 0.0 : sinz[q] / hz;
        k2z[q] = sz * sz;
    }
}

// Radices of a Stockham transform of length n (4 first, then 2, 3, 5, 7);
// 0 if n is longer than kLesFftMaxN or has another prime factor.
int les_radices(int n, int *f)
{
    if (n > kLesFftMaxN) return 0;
    int nf = 0, m = n;
    while (m % 4 == 0) { f[nf++] = 4; m /= 4; }
    while (m % 2 == 0) { f[nf++] = 2; m /= 2; }
    for (int p : {3, 5, 7})
        while (m % p == 0) { f[nf++] = p; m /= p; }
    return m == 1 ? nf : 0;
}

// Point g at tables packed as by les_tables at `base`.
void les_bind(int nx, int ny, int nz, double Lx, double Lz, const double *base, LesGeom *g)
{
    const int nxh = nx / 2 + 1;
    g->nx = nx; g->ny = ny; g->nz = nz; g->nxh = nxh; g->hx = Lx / nx; g->hz = Lz / nz;
    g->ix2 = 1.0 / (2.0 * g->hx); g->iz2 = 1.0 / (2.0 * g->hz);
    g->ixx = 1.0 / (g->hx * g->hx); g->izz = 1.0 / (g->hz * g->hz);
    g->dlinv = base; g->lapm = base + ny; g->lapp = base + 2 * ny; g->cm = base + 3 * ny; g->cp = base + 4 * ny;
    g->cosx = base + 5 * ny; g->sinx = g->cosx + nx; g->cosz = g->sinx + nx; g->sinz = g->cosz + nz;
    g->k2x = g->sinz + nz; g->k2z = g->k2x + nxh;
    g->nfx = les_radices(nx, g->fx);
    g->nfz = les_radices(nz, g->fz);
}

}  // namespace

struct ef_les {
    int device = 0;
    int nx = 0, ny = 0, nz = 0, nxh = 0;
    double Lx = 0, Lz = 0;
    ef_les_cfg cfg{};
    std::vector<double> y;          // host copy of the y nodes
    double *d_tab = nullptr;        // the tables of LesGeom, packed
    double *d_ustar = nullptr;      // [3][N]
    double *d_r = nullptr;          // [3][N] R of the previous substep
    double *d_b = nullptr;          // [N] divergence, then phi
    double *d_cw = nullptr;         // [ny][nz][nxh] chain elimination coefficients c'
    double *d_cinv = nullptr;       // [ny][nz][nxh] their reciprocal pivots
    double2 *d_B = nullptr;         // [ny][nz][nxh] x-transformed
    double2 *d_C = nullptr;         // [ny][nz][nxh] x- and z-transformed
    LesGeom g{};
};

using namespace eles;

namespace {

long les_points(const ef_les *s) { return (long)s->nx * s->ny * s->nz; }

// Projection of ustar into u (u may equal ustar); d_b is overwritten.
cudaError_t launch_projection(ef_les *s, const double *ustar, double *u, cudaStream_t st)
{
    const LesGeom &g = s->g;
    const long N = les_points(s), NH = (long)g.nxh * g.ny * g.nz;
    const long xlines = (long)g.ny * g.nz, zlines = (long)g.ny * g.nxh;
    const int wx = fft_warps(g.nx), wz = fft_warps(g.nz);
    const int bx = (int)std::min<long>((xlines + wx - 1) / wx, 152L * 16);
    const int bz = (int)std::min<long>((zlines + wz - 1) / wz, 152L * 16);
    const size_t shx = sizeof(double2) * 2 * g.nx * wx, shz = sizeof(double2) * 2 * g.nz * wz;
    les_div<<<blocks_for(N), kLesThreads, 0, st>>>(g, ustar, s->d_b);
    if (g.nfx) les_fftx_fwd<<<bx, 32 * wx, shx, st>>>(g, s->d_b, s->d_B);
    else les_dftx_fwd<<<blocks_for(NH), kLesThreads, 0, st>>>(g, s->d_b, s->d_B);
    if (g.nfz) les_fftz<<<bz, 32 * wz, shz, st>>>(g, s->d_B, s->d_C, -1.0, 1.0);
    else les_dftz<<<blocks_for(NH), kLesThreads, 0, st>>>(g, s->d_B, s->d_C, -1.0, 1.0);
    les_chain<<<blocks_for(2L * g.nxh * g.nz), kLesThreads, 0, st>>>(g, s->d_C, s->d_cw, s->d_cinv);
    if (g.nfz) les_fftz<<<bz, 32 * wz, shz, st>>>(g, s->d_C, s->d_B, 1.0, 1.0 / g.nz);
    else les_dftz<<<blocks_for(NH), kLesThreads, 0, st>>>(g, s->d_C, s->d_B, 1.0, 1.0 / g.nz);
    if (g.nfx) les_fftx_inv<<<bx, 32 * wx, shx, st>>>(g, s->d_B, s->d_b);
    else les_dftx_inv<<<blocks_for(N), kLesThreads, 0, st>>>(g, s->d_B, s->d_b);
    les_correct<<<blocks_for(N), kLesThreads, 0, st>>>(g, ustar, s->d_b, u);
    return cudaGetLastError();
}

template <typename TT>
cudaError_t launch_step(ef_les *s, double *u, const TT *tau, const TT *bc, double dt, cudaStream_t st)
{
    static const double kGamma[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
    static const double kZeta[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};
    const LesGeom &g = s->g;
    const long N = les_points(s);
    const int nsub = s->cfg.scheme == EF_LES_EULER ? 1 : 3;
    les_walls<TT><<<blocks_for(2L * g.nz * g.nx), kLesThreads, 0, st>>>(g, u, bc);
    for (int k = 0; k < nsub; k++) {
        const double gam = nsub == 1 ? 1.0 : kGamma[k], zet = nsub == 1 ? 0.0 : kZeta[k];
        les_rhs<TT><<<blocks_for(N), kLesThreads, 0, st>>>(g, u, tau, s->cfg.nu, s->cfg.forcing, dt * gam, dt * zet,
                                                           zet != 0.0, s->d_ustar, s->d_r);
        cudaError_t e = launch_projection(s, s->d_ustar, u, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

bool same_device(const ef_les *s)
{
    int dev = -1;
    return cudaGetDevice(&dev) == cudaSuccess && dev == s->device;
}

}  // namespace

extern "C" {

int ef_les_create(const ef_grid *les, const ef_les_cfg *cfg, ef_les **out)
{
    if (!les || !cfg || !out || !les->y) { set_error("ef_les_create: NULL argument"); return EF_ERR_ARG; }
    *out = nullptr;
    const int nx = les->nx, ny = les->ny, nz = les->nz;
    if (nx < 3 || nz < 3 || ny < 3 || nx > kLesMaxN || ny > kLesMaxN || nz > kLesMaxN) {
        set_error("ef_les_create: grid %dx%dx%d outside 3..%d per direction", nx, ny, nz, kLesMaxN);
        return EF_ERR_SHAPE;
    }
    if ((long)nx * ny * nz > kLesMaxPoints) {
        set_error("ef_les_create: more than %ld nodes", kLesMaxPoints);
        return EF_ERR_SHAPE;
    }
    if (!(les->Lx > 0) || !(les->Lz > 0)) { set_error("ef_les_create: Lx and Lz must be > 0"); return EF_ERR_ARG; }
    for (int j = 1; j < ny; j++)
        if (!(les->y[j] > les->y[j - 1])) { set_error("ef_les_create: y nodes must ascend"); return EF_ERR_ARG; }
    if (!(cfg->nu >= 0) || !isfinite(cfg->forcing)) {
        set_error("ef_les_create: nu must be >= 0 and the forcing finite");
        return EF_ERR_ARG;
    }
    if (cfg->scheme != EF_LES_RK3 && cfg->scheme != EF_LES_EULER) {
        set_error("ef_les_create: unknown scheme %d", cfg->scheme);
        return EF_ERR_ARG;
    }
    ef_les *s = new ef_les();
    cudaGetDevice(&s->device);
    s->nx = nx; s->ny = ny; s->nz = nz; s->nxh = nx / 2 + 1;
    s->Lx = les->Lx; s->Lz = les->Lz;
    s->cfg = *cfg;
    s->y.assign(les->y, les->y + ny);
    const int nxh = s->nxh;
    std::vector<double> tab, cwh, cinvh;
    les_tables(nx, ny, nz, les->Lx, les->Lz, les->y, tab);
    {
        LesGeom hg{};
        les_bind(nx, ny, nz, les->Lx, les->Lz, tab.data(), &hg);
        les_chain_tables(hg, cwh, cinvh);
    }
    const long N = (long)nx * ny * nz, NH = (long)nxh * ny * nz;
    cudaError_t e = dev_malloc(&s->d_tab, sizeof(double) * tab.size());
    if (e == cudaSuccess) e = dev_malloc(&s->d_ustar, sizeof(double) * 3 * N);
    if (e == cudaSuccess) e = dev_malloc(&s->d_r, sizeof(double) * 3 * N);
    if (e == cudaSuccess) e = dev_malloc(&s->d_b, sizeof(double) * N);
    if (e == cudaSuccess) e = dev_malloc(&s->d_cw, sizeof(double) * NH);
    if (e == cudaSuccess) e = dev_malloc(&s->d_cinv, sizeof(double) * NH);
    if (e == cudaSuccess) e = dev_malloc(&s->d_B, sizeof(double2) * NH);
    if (e == cudaSuccess) e = dev_malloc(&s->d_C, sizeof(double2) * NH);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_cw, cwh.data(), sizeof(double) * NH, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_cinv, cinvh.data(), sizeof(double) * NH, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        ef_les_destroy(s);
        return cuda_fail(e, "ef_les_create");
    }
    les_bind(nx, ny, nz, les->Lx, les->Lz, s->d_tab, &s->g);
    *out = s;
    return EF_OK;
}

void ef_les_destroy(ef_les *s)
{
    if (!s) return;
    cudaFree(s->d_tab);
    cudaFree(s->d_ustar);
    cudaFree(s->d_r);
    cudaFree(s->d_b);
    cudaFree(s->d_cw);
    cudaFree(s->d_cinv);
    cudaFree(s->d_B);
    cudaFree(s->d_C);
    delete s;
}

int ef_les_step(ef_les *s, double *ubar, const void *tau, const void *ubar_bc, int precision, double dt,
                void *stream)
{
    NvtxRange nv("ef_les_step");
    if (!s || !ubar) { set_error("ef_les_step: NULL argument"); return EF_ERR_ARG; }
    if (!(dt > 0) || !isfinite(dt)) { set_error("ef_les_step: dt must be finite and > 0"); return EF_ERR_ARG; }
    if (precision != EF_PREC_FP64 && precision != EF_PREC_FP32 && precision != EF_PREC_TF32X2 &&
        precision != EF_PREC_BF16X3) {
        set_error("ef_les_step: unknown precision %d", precision);
        return EF_ERR_ARG;
    }
    if (!same_device(s)) { set_error("ef_les_step: the current device is not the solver's"); return EF_ERR_ARG; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (precision == EF_PREC_FP64)
        e = launch_step<double>(s, ubar, static_cast<const double *>(tau), static_cast<const double *>(ubar_bc), dt, st);
    else
        e = launch_step<float>(s, ubar, static_cast<const float *>(tau), static_cast<const float *>(ubar_bc), dt, st);
    return e == cudaSuccess ? EF_OK : cuda_fail(e, "ef_les_step");
}

int ef_les_project(ef_les *s, const double *ustar, double *u, void *stream)
{
    if (!s || !ustar || !u) { set_error("ef_les_project: NULL argument"); return EF_ERR_ARG; }
    if (!same_device(s)) { set_error("ef_les_project: the current device is not the solver's"); return EF_ERR_ARG; }
    cudaError_t e = launch_projection(s, ustar, u, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EF_OK : cuda_fail(e, "ef_les_project");
}

int ef_les_divergence(ef_les *s, const double *u, double *div, void *stream)
{
    if (!s || !u || !div) { set_error("ef_les_divergence: NULL argument"); return EF_ERR_ARG; }
    if (!same_device(s)) { set_error("ef_les_divergence: the current device is not the solver's"); return EF_ERR_ARG; }
    const long N = les_points(s);
    les_div<<<blocks_for(N), kLesThreads, 0, static_cast<cudaStream_t>(stream)>>>(s->g, u, div);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EF_OK : cuda_fail(e, "ef_les_divergence");
}

int ef_les_rhs(ef_les *s, const double *u, const void *tau, int precision, double *rhs, void *stream)
{
    if (!s || !u || !rhs) { set_error("ef_les_rhs: NULL argument"); return EF_ERR_ARG; }
    if (precision != EF_PREC_FP64 && precision != EF_PREC_FP32 && precision != EF_PREC_TF32X2 &&
        precision != EF_PREC_BF16X3) {
        set_error("ef_les_rhs: unknown precision %d", precision);
        return EF_ERR_ARG;
    }
    if (!same_device(s)) { set_error("ef_les_rhs: the current device is not the solver's"); return EF_ERR_ARG; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long N = les_points(s);
    if (precision == EF_PREC_FP64)
        les_rhs<double><<<blocks_for(N), kLesThreads, 0, st>>>(s->g, u, static_cast<const double *>(tau), s->cfg.nu,
                                                               s->cfg.forcing, 0.0, 0.0, 0, s->d_ustar, rhs);
    else
        les_rhs<float><<<blocks_for(N), kLesThreads, 0, st>>>(s->g, u, static_cast<const float *>(tau), s->cfg.nu,
                                                              s->cfg.forcing, 0.0, 0.0, 0, s->d_ustar, rhs);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EF_OK : cuda_fail(e, "ef_les_rhs");
}

int ef_apost_step(ef_plan *plan, ef_les *s, const void *u_dns, void *ubar_dns, void *tau, double *ubar_les,
                  double dt, void *stream)
{
    NvtxRange nv("ef_apost_step");
    if (!plan || !s || !u_dns || !ubar_dns || !tau || !ubar_les) {
        set_error("ef_apost_step: NULL argument");
        return EF_ERR_ARG;
    }
    if (plan->nlx != s->nx || plan->nly != s->ny || plan->nlz != s->nz || plan->Lx != s->Lx || plan->Lz != s->Lz) {
        set_error("ef_apost_step: the plan's LES grid is not the solver's");
        return EF_ERR_SHAPE;
    }
    if (static_cast<const void *>(ubar_les) == ubar_dns || static_cast<const void *>(ubar_les) == tau) {
        set_error("ef_apost_step: ubar_les must not be ubar_dns or tau");
        return EF_ERR_ARG;
    }
    int rc = ef_subfilter_stress(plan, u_dns, ubar_dns, tau, nullptr, stream);
    if (rc) return rc;
    return ef_les_step(s, ubar_les, tau, ubar_dns, plan->prec, dt, stream);
}

}  // extern "C"
