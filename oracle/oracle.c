/*
 * CPU oracle for the explicit wall-extended channel filter and the exact
 * subfilter stress of Bae & Lozano-Duran, "DNS-aided explicitly filtered LES
 * of channel flow" (arXiv 1902.02508).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or constant generator with the CUDA library, and the
 * CUDA library never calls it.
 *
 * Everything is IEEE double precision and written as plainly as the
 * definitions allow.  Readings of points the paper leaves open:
 *   - kernel: Gaussian of width Delta per direction,
 *       G(s) = sqrt(6/(pi Delta^2)) exp(-6 s^2 / Delta^2),
 *     transfer function exp(-k^2 Delta^2 / 24), the same Delta in x, y, z
 *     (constant filter width, Sec. 2.2);
 *   - support cut at |s| <= 2.5 Delta (the excluded mass is ~5e-18);
 *   - quadrature: trapezoid rule on the (extended) node set, then every row
 *     divided by its own weight sum (a constant is preserved exactly), Eq. 2;
 *     optionally in y, the kernel integrated exactly against the
 *     piecewise-linear interpolant of the extended field (a linear function
 *     is then reproduced exactly away from the walls);
 *   - extension across the walls, Eq. 7: u1, u3 even and u2 odd about each
 *     wall, applied at both walls and repeated (a period-4 line in y);
 *     the alternative of Eq. 9 flips every parity; a "truncated" mode filters
 *     over the physical nodes only; a wall node is its own mirror image, so
 *     an odd extension is zero there (u2 = -u2 at the wall);
 *   - discretization operator: the field filtered at the DNS nodes is
 *     linearly interpolated to the LES nodes (Sec. 3, initial condition);
 *   - T_ij = bar(u_i u_j) - bar(u_i) bar(u_j) evaluated as written (Eq. 6 and
 *     the four-step procedure of Sec. 2.1), no decomposition.
 * Parity pins: tests/test_oracle_pins.py (closed forms, invariants, brute
 * force).  Absolute T_ij values on channel data are not printed in the paper.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* Gaussian filter kernel of width delta (second moment delta^2 / 12). */
static double gauss(double s, double delta)
{
    return sqrt(6.0 / (OR_PI * delta * delta)) * exp(-6.0 * s * s / (delta * delta));
}

static int in_support(double s, double delta) { return fabs(s) <= 2.5 * delta; }

/* Moments of the kernel over s in [a, b] clipped to the support
 * |s - yi| <= 2.5 delta: I0 = int G(yi - s) ds, J1 = int G(yi - s)(s - yi) ds.
 * With sigma^2 = delta^2 / 12, int G = erf differences and t G(t) has the
 * antiderivative -sigma^2 G(t). */
static void gauss_moments(double yi, double a, double b, double delta, double *I0, double *J1)
{
    double R = 2.5 * delta, sig = delta / sqrt(12.0);
    if (a < yi - R) a = yi - R;
    if (b > yi + R) b = yi + R;
    *I0 = 0.0;
    *J1 = 0.0;
    if (!(b > a)) return;
    double ta = a - yi, tb = b - yi;
    *I0 = 0.5 * (erf(tb / (sig * sqrt(2.0))) - erf(ta / (sig * sqrt(2.0))));
    *J1 = sig * sig * (gauss(ta, delta) - gauss(tb, delta));
}

/* Exact integral of G(yi - s) times the hat function of a node at e whose
 * neighbours are el < e < er (has_l / has_r: the neighbour exists). */
static double hat_weight(double yi, double e, int has_l, double el, int has_r, double er, double delta)
{
    double w = 0.0, I0, J1;
    if (has_l) {
        gauss_moments(yi, el, e, delta, &I0, &J1);
        w += (J1 + (yi - el) * I0) / (e - el);
    }
    if (has_r) {
        gauss_moments(yi, e, er, delta, &I0, &J1);
        w += ((er - yi) * I0 - J1) / (er - e);
    }
    return w;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------------------
 * One periodic, uniform direction (x or z), Eq. 2 on the periodic line.
 * F[i][i'] = sum over images m of G(x_i - x_i' - m L) h, row-normalised.
 * A = S F with S the linear interpolation to the LES nodes X L / nl.
 * A is returned dense, row-major [nl][n].
 * ------------------------------------------------------------------------- */
int or_op_periodic(int n, double L, int nl, double delta, double *A)
{
    if (n < 2 || nl < 1 || !(L > 0) || !(delta > 0)) return 1;
    double h = L / n;
    double *F = (double *)calloc((size_t)n * n, sizeof(double));
    if (!F) return 2;
    int M = (int)ceil(2.5 * delta / L) + 1;
    for (int i = 0; i < n; i++) {
        double xi = i * h, norm = 0.0;
        for (int ip = 0; ip < n; ip++) {
            double xip = ip * h;
            for (int m = -M; m <= M; m++) {
                double s = xi - xip - m * L;
                if (in_support(s, delta)) {
                    double w = gauss(s, delta) * h;
                    F[(size_t)i * n + ip] += w;
                    norm += w;
                }
            }
        }
        for (int ip = 0; ip < n; ip++) F[(size_t)i * n + ip] /= norm;
    }
    for (int X = 0; X < nl; X++) {
        /* LES node X sits at X L / nl = (X n / nl) h: exact rational position. */
        long num = (long)X * n;
        int i0 = (int)(num / nl);
        double theta = (double)(num % nl) / nl;
        int i1 = (i0 + 1) % n;
        for (int ip = 0; ip < n; ip++)
            A[(size_t)X * n + ip] = (1.0 - theta) * F[(size_t)i0 * n + ip]
                                    + theta * F[(size_t)i1 * n + ip];
    }
    free(F);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Wall-normal direction, Eq. 7 (mode 0) or truncated (mode 1).
 *
 * mode 0: the y-line is extended by mirror images about y = -1 and y = +1,
 * repeated with period 4.  Node j has the direct images y_j + 4m (sign +1) and,
 * for interior j, the mirror images -2 - y_j + 4m (sign = parity).  Mirror
 * images of the two wall nodes coincide with direct images and are not added
 * twice.  The extended lattice is built explicitly, sorted, and given
 * trapezoid weights from its own neighbour spacings.
 * mode 1: the physical nodes only, trapezoid weights with half cells at the
 * walls (the filter support is cut by the wall).
 *
 * F^p[i][j] = sum_{n -> j} sign_p(n) G(y_i - e_n) h_n / sum_n G(y_i - e_n) h_n
 * A^p = S F^p, S linear interpolation to the LES nodes Y (ascending, within
 * [-1, 1]).  Dense, row-major [nly][ny].
 * ------------------------------------------------------------------------- */
typedef struct { double e; int src; int mirror; } ext_node;

static int cmp_ext(const void *a, const void *b)
{
    double d = ((const ext_node *)a)->e - ((const ext_node *)b)->e;
    return (d > 0) - (d < 0);
}

int or_op_wall_q(int ny, const double *y, int nly, const double *Y, double delta,
                 int mode, int parity, int quad, double *A);

int or_op_wall(int ny, const double *y, int nly, const double *Y, double delta,
               int mode, int parity, double *A)
{
    return or_op_wall_q(ny, y, nly, Y, delta, mode, parity, 0, A);
}

/* quad 0: trapezoid weights G(y_i - e_n) h_n on the extended node set;
 * quad 1: the kernel integrated exactly against the piecewise-linear
 * interpolant of the extended field (hat function of each extended node,
 * its neighbours in the sorted extended set), cut at the support. */
int or_op_wall_q(int ny, const double *y, int nly, const double *Y, double delta,
                 int mode, int parity, int quad, double *A)
{
    if (ny < 3 || nly < 2 || !(delta > 0)) return 1;
    for (int j = 1; j < ny; j++) if (!(y[j] > y[j - 1])) return 1;
    int cap = 5 * 2 * ny;
    ext_node *E = (ext_node *)malloc(sizeof(ext_node) * cap);
    double *h = (double *)malloc(sizeof(double) * cap);
    double *F = (double *)calloc((size_t)ny * ny, sizeof(double));
    if (!E || !h || !F) { free(E); free(h); free(F); return 2; }
    int ne = 0;
    if (mode == 0) {
        for (int m = -2; m <= 2; m++)
            for (int j = 0; j < ny; j++) {
                E[ne].e = y[j] + 4.0 * m; E[ne].src = j; E[ne].mirror = 0; ne++;
                if (j > 0 && j < ny - 1) {
                    E[ne].e = -2.0 - y[j] + 4.0 * m; E[ne].src = j; E[ne].mirror = 1; ne++;
                }
            }
        qsort(E, ne, sizeof(ext_node), cmp_ext);
        h[0] = E[1].e - E[0].e;
        h[ne - 1] = E[ne - 1].e - E[ne - 2].e;
        for (int n = 1; n < ne - 1; n++) h[n] = 0.5 * (E[n + 1].e - E[n - 1].e);
    } else {
        for (int j = 0; j < ny; j++) { E[ne].e = y[j]; E[ne].src = j; E[ne].mirror = 0; ne++; }
        h[0] = 0.5 * (y[1] - y[0]);
        h[ny - 1] = 0.5 * (y[ny - 1] - y[ny - 2]);
        for (int j = 1; j < ny - 1; j++) h[j] = 0.5 * (y[j + 1] - y[j - 1]);
    }
    for (int i = 0; i < ny; i++) {
        double norm = 0.0;
        for (int n = 0; n < ne; n++) {
            double s = y[i] - E[n].e, w;
            if (quad == 0) {
                if (!in_support(s, delta)) continue;
                w = gauss(s, delta) * h[n];
            } else {
                w = hat_weight(y[i], E[n].e, n > 0, n > 0 ? E[n - 1].e : 0.0, n < ne - 1,
                               n < ne - 1 ? E[n + 1].e : 0.0, delta);
                if (w == 0.0) continue;
            }
            norm += w;
            /* A wall node is its own mirror image: an odd extension is zero
             * there, an even one takes the node's value. */
            double sgn = 1.0;
            if (mode == 0 && E[n].mirror) sgn = (double)parity;
            if (mode == 0 && (E[n].src == 0 || E[n].src == ny - 1)) sgn = 0.5 * (1.0 + parity);
            F[(size_t)i * ny + E[n].src] += sgn * w;
        }
        for (int j = 0; j < ny; j++) F[(size_t)i * ny + j] /= norm;
    }
    for (int J = 0; J < nly; J++) {
        int i0 = 0;
        while (i0 < ny - 2 && y[i0 + 1] <= Y[J]) i0++;
        double theta = (Y[J] - y[i0]) / (y[i0 + 1] - y[i0]);
        for (int j = 0; j < ny; j++)
            A[(size_t)J * ny + j] = (1.0 - theta) * F[(size_t)i0 * ny + j]
                                    + theta * F[(size_t)(i0 + 1) * ny + j];
    }
    free(E); free(h); free(F);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Tensor-product application out = (Ay (x) Az (x) Ax) f, one direction after
 * the other (x, then z, then y).  f[ny][nz][nx], out[nly][nlz][nlx]; Ay is
 * [nly][ny], Az [nlz][nz], Ax [nlx][nx].  Only LES rows J in [J0, J1) are
 * produced (the rest of out is left untouched); only the DNS planes those rows
 * reach are filtered in x and z.  Zero operator entries are skipped.
 * ------------------------------------------------------------------------- */
static void row_range(const double *A, int rows, int cols, int *lo, int *hi)
{
    for (int r = 0; r < rows; r++) {
        int a = cols, b = -1;
        for (int c = 0; c < cols; c++)
            if (A[(size_t)r * cols + c] != 0.0) { if (c < a) a = c; b = c; }
        lo[r] = a; hi[r] = b;
    }
}

int or_apply_separable(int nx, int ny, int nz, int nlx, int nly, int nlz,
                       const double *Ax, const double *Ay, const double *Az,
                       const double *f, double *out, int J0, int J1)
{
    if (J0 < 0) J0 = 0;
    if (J1 > nly || J1 <= 0) J1 = nly;
    char *need = (char *)calloc(ny, 1);
    double *gx = (double *)malloc(sizeof(double) * (size_t)ny * nz * nlx);
    double *gz = (double *)malloc(sizeof(double) * (size_t)ny * nlz * nlx);
    int *xlo = (int *)malloc(sizeof(int) * nlx), *xhi = (int *)malloc(sizeof(int) * nlx);
    int *zlo = (int *)malloc(sizeof(int) * nlz), *zhi = (int *)malloc(sizeof(int) * nlz);
    int *ylo = (int *)malloc(sizeof(int) * nly), *yhi = (int *)malloc(sizeof(int) * nly);
    if (!need || !gx || !gz || !xlo || !xhi || !zlo || !zhi || !ylo || !yhi) {
        free(need); free(gx); free(gz); free(xlo); free(xhi); free(zlo); free(zhi);
        free(ylo); free(yhi);
        return 2;
    }
    row_range(Ax, nlx, nx, xlo, xhi);
    row_range(Az, nlz, nz, zlo, zhi);
    row_range(Ay, nly, ny, ylo, yhi);
    for (int J = J0; J < J1; J++)
        for (int j = ylo[J]; j <= yhi[J]; j++) need[j] = 1;
    /* x: gx[j][k][I] = sum_i Ax[I][i] f[j][k][i] */
#pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < ny; j++) {
        if (!need[j]) continue;
        for (int k = 0; k < nz; k++) {
            const double *row = f + ((size_t)j * nz + k) * nx;
            for (int I = 0; I < nlx; I++) {
                double s = 0.0;
                for (int i = xlo[I]; i <= xhi[I]; i++) s += Ax[(size_t)I * nx + i] * row[i];
                gx[((size_t)j * nz + k) * nlx + I] = s;
            }
        }
    }
    /* z: gz[j][K][I] = sum_k Az[K][k] gx[j][k][I] */
#pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < ny; j++) {
        if (!need[j]) continue;
        for (int K = 0; K < nlz; K++)
            for (int I = 0; I < nlx; I++) {
                double s = 0.0;
                for (int k = zlo[K]; k <= zhi[K]; k++)
                    s += Az[(size_t)K * nz + k] * gx[((size_t)j * nz + k) * nlx + I];
                gz[((size_t)j * nlz + K) * nlx + I] = s;
            }
    }
    /* y: out[J][K][I] = sum_j Ay[J][j] gz[j][K][I] */
#pragma omp parallel for collapse(2) schedule(static)
    for (int J = J0; J < J1; J++)
        for (int K = 0; K < nlz; K++)
            for (int I = 0; I < nlx; I++) {
                double s = 0.0;
                for (int j = ylo[J]; j <= yhi[J]; j++)
                    s += Ay[(size_t)J * ny + j] * gz[((size_t)j * nlz + K) * nlx + I];
                out[((size_t)J * nlz + K) * nlx + I] = s;
            }
    free(need); free(gx); free(gz); free(xlo); free(xhi); free(zlo); free(zhi);
    free(ylo); free(yhi);
    return 0;
}

/* Component parities about the wall: Eq. 7 (ext 0), Eq. 9 (ext 1). */
static int comp_parity(int ext, int c)
{
    int p = (c == 1) ? -1 : 1;
    return ext == 1 ? -p : p;
}

static const int PAIR_I[6] = {0, 0, 0, 1, 1, 2};
static const int PAIR_J[6] = {0, 1, 2, 1, 2, 2};

/* ---------------------------------------------------------------------------
 * The four steps of Sec. 2.1 on a whole snapshot, separable evaluation.
 * u: [3][ny][nz][nx]; ubar: [3][nly][nlz][nlx]; tau: [6][nly][nlz][nlx] in the
 * order 11, 12, 13, 22, 23, 33.  ext: 0 Eq. 7, 1 Eq. 9, 2 truncated.
 * Rows J outside [J0, J1) are left untouched (J1 <= 0: all rows).
 * ------------------------------------------------------------------------- */
int or_subfilter_stress_q(int nx, int ny, int nz, double Lx, double Lz, const double *y,
                          int nlx, int nly, int nlz, const double *Y, double delta, int ext, int quad,
                          const double *u, double *ubar, double *tau, int J0, int J1);

int or_subfilter_stress(int nx, int ny, int nz, double Lx, double Lz, const double *y,
                        int nlx, int nly, int nlz, const double *Y, double delta, int ext,
                        const double *u, double *ubar, double *tau, int J0, int J1)
{
    return or_subfilter_stress_q(nx, ny, nz, Lx, Lz, y, nlx, nly, nlz, Y, delta, ext, 0, u, ubar, tau, J0, J1);
}

/* The same with the y quadrature chosen as in or_op_wall_q. */
int or_subfilter_stress_q(int nx, int ny, int nz, double Lx, double Lz, const double *y,
                          int nlx, int nly, int nlz, const double *Y, double delta, int ext, int quad,
                          const double *u, double *ubar, double *tau, int J0, int J1)
{
    size_t np = (size_t)nx * ny * nz, nl = (size_t)nlx * nly * nlz;
    double *Ax = (double *)malloc(sizeof(double) * (size_t)nlx * nx);
    double *Az = (double *)malloc(sizeof(double) * (size_t)nlz * nz);
    double *Ayp = (double *)malloc(sizeof(double) * (size_t)nly * ny);
    double *Aym = (double *)malloc(sizeof(double) * (size_t)nly * ny);
    double *prod = (double *)malloc(sizeof(double) * np);
    double *uu = (double *)malloc(sizeof(double) * nl);
    if (!Ax || !Az || !Ayp || !Aym || !prod || !uu) {
        free(Ax); free(Az); free(Ayp); free(Aym); free(prod); free(uu);
        return 2;
    }
    int rc = or_op_periodic(nx, Lx, nlx, delta, Ax);
    rc |= or_op_periodic(nz, Lz, nlz, delta, Az);
    int wmode = (ext == 2) ? 1 : 0;
    rc |= or_op_wall_q(ny, y, nly, Y, delta, wmode, +1, quad, Ayp);
    rc |= or_op_wall_q(ny, y, nly, Y, delta, wmode, -1, quad, Aym);
    if (rc) { free(Ax); free(Az); free(Ayp); free(Aym); free(prod); free(uu); return 1; }
    if (J1 <= 0 || J1 > nly) J1 = nly;
    /* steps 1-2 for the velocities themselves: bar(u_i) */
    for (int c = 0; c < 3; c++) {
        const double *Ay = comp_parity(ext, c) > 0 ? Ayp : Aym;
        or_apply_separable(nx, ny, nz, nlx, nly, nlz, Ax, Ay, Az, u + c * np, ubar + c * nl, J0, J1);
    }
    /* steps 1-4 for each pair: T_ij = bar(u_i u_j) - bar(u_i) bar(u_j) */
    for (int q = 0; q < 6; q++) {
        int a = PAIR_I[q], b = PAIR_J[q];
        const double *ua = u + a * np, *ub = u + b * np;
#pragma omp parallel for schedule(static)
        for (long p = 0; p < (long)np; p++) prod[p] = ua[p] * ub[p];
        const double *Ay = comp_parity(ext, a) * comp_parity(ext, b) > 0 ? Ayp : Aym;
        or_apply_separable(nx, ny, nz, nlx, nly, nlz, Ax, Ay, Az, prod, uu, J0, J1);
        for (int J = J0; J < J1; J++)
            for (size_t r = 0; r < (size_t)nlz * nlx; r++) {
                size_t o = (size_t)J * nlz * nlx + r;
                tau[q * nl + o] = uu[o] - ubar[a * nl + o] * ubar[b * nl + o];
            }
    }
    free(Ax); free(Az); free(Ayp); free(Aym); free(prod); free(uu);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Direct three-dimensional summation at selected LES points: the filter of
 * Eq. 2 with the product kernel G(dx) G(dy) G(dz) over the periodic images in
 * x, z and the extended lattice in y (Eq. 7), evaluated at each DNS node the
 * LES point's trilinear interpolation touches, then interpolated.  All nine
 * filtered quantities are produced: bar(u_i) and bar(u_i u_j), and from them
 * T_ij.  pts: [npts][3] integer LES indices (I, J, K).  ubar_out [npts][3],
 * tau_out [npts][6].
 * ------------------------------------------------------------------------- */
typedef struct { int n; int *idx; double *w; double *sgn; } tap_list;

static void free_taps(tap_list *t) { free(t->idx); free(t->w); free(t->sgn); }

/* Periodic taps of DNS node i: (index, G * h) pairs over all images. */
static int periodic_taps(int n, double L, double delta, int i, tap_list *t)
{
    double h = L / n;
    int M = (int)ceil(2.5 * delta / L) + 1, cap = (2 * M + 1) * n;
    t->idx = (int *)malloc(sizeof(int) * cap);
    t->w = (double *)malloc(sizeof(double) * cap);
    t->sgn = NULL;
    t->n = 0;
    if (!t->idx || !t->w) return 2;
    for (int ip = 0; ip < n; ip++)
        for (int m = -M; m <= M; m++) {
            double s = i * h - ip * h - m * L;
            if (in_support(s, delta)) { t->idx[t->n] = ip; t->w[t->n] = gauss(s, delta) * h; t->n++; }
        }
    return 0;
}

/* Extended-lattice taps of DNS node i in y: (source index, G * h, mirror flag). */
static int wall_taps(int ny, const double *y, double delta, int mode, int i, tap_list *t)
{
    int cap = 10 * ny;
    ext_node *E = (ext_node *)malloc(sizeof(ext_node) * cap);
    double *h = (double *)malloc(sizeof(double) * cap);
    t->idx = (int *)malloc(sizeof(int) * cap);
    t->w = (double *)malloc(sizeof(double) * cap);
    t->sgn = (double *)malloc(sizeof(double) * cap);
    t->n = 0;
    if (!E || !h || !t->idx || !t->w || !t->sgn) { free(E); free(h); return 2; }
    int ne = 0;
    if (mode == 0) {
        for (int m = -2; m <= 2; m++)
            for (int j = 0; j < ny; j++) {
                E[ne].e = y[j] + 4.0 * m; E[ne].src = j; E[ne].mirror = 0; ne++;
                if (j > 0 && j < ny - 1) {
                    E[ne].e = -2.0 - y[j] + 4.0 * m; E[ne].src = j; E[ne].mirror = 1; ne++;
                }
            }
        qsort(E, ne, sizeof(ext_node), cmp_ext);
        h[0] = E[1].e - E[0].e;
        h[ne - 1] = E[ne - 1].e - E[ne - 2].e;
        for (int n = 1; n < ne - 1; n++) h[n] = 0.5 * (E[n + 1].e - E[n - 1].e);
    } else {
        for (int j = 0; j < ny; j++) { E[ne].e = y[j]; E[ne].src = j; E[ne].mirror = 0; ne++; }
        h[0] = 0.5 * (y[1] - y[0]);
        h[ny - 1] = 0.5 * (y[ny - 1] - y[ny - 2]);
        for (int j = 1; j < ny - 1; j++) h[j] = 0.5 * (y[j + 1] - y[j - 1]);
    }
    for (int n = 0; n < ne; n++) {
        double s = y[i] - E[n].e;
        if (!in_support(s, delta)) continue;
        t->idx[t->n] = E[n].src;
        t->w[t->n] = gauss(s, delta) * h[n];
        /* kind: +1 direct image, -1 mirror image, 0 wall node (its own mirror) */
        t->sgn[t->n] = 1.0;
        if (mode == 0 && E[n].mirror) t->sgn[t->n] = -1.0;
        if (mode == 0 && (E[n].src == 0 || E[n].src == ny - 1)) t->sgn[t->n] = 0.0;
        t->n++;
    }
    free(E); free(h);
    return 0;
}

/* bar(f) at one DNS node for the nine fields (3 velocities, 6 products). */
static void direct_node(int nx, int ny, int nz, const tap_list *tx, const tap_list *ty,
                        const tap_list *tz, int ext, const double *u, double out9[9])
{
    size_t np = (size_t)nx * ny * nz;
    double num[9] = {0}, den = 0.0;
    int par[9];
    for (int c = 0; c < 3; c++) par[c] = comp_parity(ext, c);
    for (int q = 0; q < 6; q++) par[3 + q] = comp_parity(ext, PAIR_I[q]) * comp_parity(ext, PAIR_J[q]);
    for (int b = 0; b < ty->n; b++) {
        int j = ty->idx[b];
        for (int c = 0; c < tz->n; c++) {
            int k = tz->idx[c];
            for (int a = 0; a < tx->n; a++) {
                int i = tx->idx[a];
                double w = tx->w[a] * ty->w[b] * tz->w[c];
                size_t o = ((size_t)j * nz + k) * nx + i;
                double v[3] = {u[o], u[np + o], u[2 * np + o]};
                den += w;
                for (int q = 0; q < 9; q++) {
                    double val = q < 3 ? v[q] : v[PAIR_I[q - 3]] * v[PAIR_J[q - 3]];
                    double s = 1.0;
                    if (ty->sgn[b] < 0) s = par[q];
                    if (ty->sgn[b] == 0.0) s = 0.5 * (1.0 + par[q]);
                    num[q] += s * w * val;
                }
            }
        }
    }
    for (int q = 0; q < 9; q++) out9[q] = num[q] / den;
}

int or_direct3d_points(int nx, int ny, int nz, double Lx, double Lz, const double *y,
                       int nlx, int nly, int nlz, const double *Y, double delta, int ext,
                       const double *u, int npts, const int *pts, double *ubar_out,
                       double *tau_out)
{
    (void)nly;
    int wmode = (ext == 2) ? 1 : 0;
    int fail = 0;
#pragma omp parallel for schedule(dynamic)
    for (int p = 0; p < npts; p++) {
        int I = pts[3 * p], J = pts[3 * p + 1], K = pts[3 * p + 2];
        /* interpolation stencils of the discretization operator */
        long nxn = (long)I * nx;
        int ix0 = (int)(nxn / nlx);
        double thx = (double)(nxn % nlx) / nlx;
        long nzn = (long)K * nz;
        int iz0 = (int)(nzn / nlz);
        double thz = (double)(nzn % nlz) / nlz;
        int iy0 = 0;
        while (iy0 < ny - 2 && y[iy0 + 1] <= Y[J]) iy0++;
        double thy = (Y[J] - y[iy0]) / (y[iy0 + 1] - y[iy0]);
        double acc[9] = {0};
        for (int dx = 0; dx < 2; dx++) {
            double wx = dx ? thx : 1.0 - thx;
            if (wx == 0.0) continue;
            tap_list tx;
            if (periodic_taps(nx, Lx, delta, (ix0 + dx) % nx, &tx)) { fail = 1; continue; }
            for (int dz = 0; dz < 2; dz++) {
                double wz = dz ? thz : 1.0 - thz;
                if (wz == 0.0) continue;
                tap_list tz;
                if (periodic_taps(nz, Lz, delta, (iz0 + dz) % nz, &tz)) { fail = 1; continue; }
                for (int dy = 0; dy < 2; dy++) {
                    double wy = dy ? thy : 1.0 - thy;
                    if (wy == 0.0) continue;
                    tap_list ty;
                    if (wall_taps(ny, y, delta, wmode, iy0 + dy, &ty)) { fail = 1; continue; }
                    double v9[9];
                    direct_node(nx, ny, nz, &tx, &ty, &tz, ext, u, v9);
                    for (int q = 0; q < 9; q++) acc[q] += wx * wy * wz * v9[q];
                    free_taps(&ty);
                }
                free_taps(&tz);
            }
            free_taps(&tx);
        }
        for (int c = 0; c < 3; c++) ubar_out[3 * p + c] = acc[c];
        for (int q = 0; q < 6; q++)
            tau_out[6 * p + q] = acc[3 + q] - acc[PAIR_I[q]] * acc[PAIR_J[q]];
    }
    return fail ? 2 : 0;
}
