/*
 * FP64 CPU oracle for periodic tricubic B-spline orbital evaluation.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. It shares no code,
 * header, table or constant with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Source: Mathuriya, Luo, Benali, Shulenburger, Kim, "Optimization and
 * parallelization of B-spline based orbital evaluations in QMC on
 * multi/many-core shared memory processors" (arXiv:1611.02665).
 *   - Sec. "QMC and B-spline-based SPOs", Eq. (SplineFunc): the 1-D cubic
 *     B-spline sums four basis functions on knots i-1..i+2, i = floor(x/Delta).
 *   - Same section, Eq. (TricubicValue): the 3-D orbital is the tensor product
 *     of three such sums over a coefficient table p[i'][j'][k'][n].
 *   - Sec. "Baseline and miniQMC", Fig. (baselineCode): kernels V, VGL, VGH
 *     return values, gradients and Hessians of all N orbitals at one position.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - The basis is the uniform cubic B-spline (four unit boxes convolved). The
 *     paper's figure of the basis is absent from the text.
 *   - Positions are fractional coordinates in the unit cube, n_d intervals per
 *     axis (Delta_d = 1/n_d), periodic; derivatives are taken with respect to
 *     those coordinates.
 *   - Outputs are written, not accumulated.
 *
 * Parity status: every function below is pinned by the CPU tests (partition
 * of unity, knot closed forms, C2 continuity, linear/quadratic reproduction,
 * brute-force sums over all knots, finite differences, periodicity, library
 * float16/bfloat16 rounding). No function is parity-unpinned.
 *
 * Everything is plain C11 in double precision; OpenMP parallelises over
 * positions only (each position is computed by one thread in a fixed order).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_V = 0, ORC_VGL = 1, ORC_VGH = 2 };

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * The four cubic pieces that are nonzero on one interval, as functions of the
 * fractional offset t in [0,1) (Eq. SplineFunc, knots i-1, i, i+1, i+2 in that
 * order), with their first and second derivatives with respect to t.
 * Reading: uniform cubic B-spline. Piece a is B(t + 1 - a), where B is the
 * centred cubic B-spline written out in orc_centred_bspline below.
 */
void orc_basis(double t, double w[4], double dw[4], double d2w[4])
{
    const double s = 1.0 - t;
    w[0] = s * s * s / 6.0;
    w[1] = (3.0 * t * t * t - 6.0 * t * t + 4.0) / 6.0;
    w[2] = (-3.0 * t * t * t + 3.0 * t * t + 3.0 * t + 1.0) / 6.0;
    w[3] = t * t * t / 6.0;

    dw[0] = -0.5 * s * s;
    dw[1] = 1.5 * t * t - 2.0 * t;
    dw[2] = -1.5 * t * t + t + 0.5;
    dw[3] = 0.5 * t * t;

    d2w[0] = s;
    d2w[1] = 3.0 * t - 2.0;
    d2w[2] = -3.0 * t + 1.0;
    d2w[3] = t;
}

/*
 * Centred cubic B-spline B(s) (support [-2,2]) and its derivatives, in closed
 * form. Used only by the brute-force evaluator, which never reduces a
 * position to a cell.
 */
void orc_centred_bspline(double s, double out[3])
{
    const double a = fabs(s);
    const double sg = s < 0.0 ? -1.0 : 1.0;
    if (a < 1.0) {
        out[0] = 2.0 / 3.0 - a * a + 0.5 * a * a * a;
        out[1] = sg * (-2.0 * a + 1.5 * a * a);
        out[2] = -2.0 + 3.0 * a;
    } else if (a < 2.0) {
        const double r = 2.0 - a;
        out[0] = r * r * r / 6.0;
        out[1] = -sg * 0.5 * r * r;
        out[2] = r;
    } else {
        out[0] = out[1] = out[2] = 0.0;
    }
}

/*
 * Lower-bound cell index and fractional offset along one axis
 * (Eq. SplineFunc: i = floor(x / Delta)), after wrapping x into the unit cell.
 * Reading for the periodic cell: x is first reduced by floor-mod to [0,1]; if
 * rounding lands it on 1 (the far face), the index wraps to 0 with t = 0.
 */
void orc_cell(double x, int n, int *i_out, double *t_out)
{
    double xw = x - floor(x);
    double u = xw * (double)n;
    double fi = floor(u);
    double t = u - fi;
    int i = (int)fi;
    if (i >= n) {
        i -= n;
        t = 0.0;
    }
    *i_out = i;
    *t_out = t;
}

/*
 * The ten output components at one position from 4x4x4 stencil weights:
 * value, d/dx, d/dy, d/dz, d2/dxx, d2/dxy, d2/dxz, d2/dyy, d2/dyz, d2/dzz.
 * Derivatives scale by n_d per order (chain rule for u = x * n_d).
 * coef_at(a, b, c, n) returns p for stencil row (a, b, c) and orbital n.
 */
typedef double (*orc_row_fn)(const void *ctx, int a, int b, int c, int n);

static void write_outputs(int kind, int N, int pos, const double acc[10],
                          int n, double *v, double *g, double *h, double *l)
{
    if (v) v[(size_t)pos * N + n] = acc[0];
    if (kind >= ORC_VGL && g) {
        for (int d = 0; d < 3; ++d) g[((size_t)pos * 3 + d) * N + n] = acc[1 + d];
    }
    if (kind == ORC_VGH && h) {
        for (int d = 0; d < 6; ++d) h[((size_t)pos * 6 + d) * N + n] = acc[4 + d];
    }
    if (kind >= ORC_VGL && l) l[(size_t)pos * N + n] = acc[4] + acc[7] + acc[9];
}

/* Derivative orders (along x, y, z) of the ten components. */
static const int ORDERS[10][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
    {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2},
};

static void eval_one_position(int kind, int nx, int ny, int nz, int N, orc_row_fn row,
                              const void *ctx, int pos, double x, double y, double z,
                              double *v, double *g, double *h, double *l)
{
    const int n3[3] = {nx, ny, nz};
    const double r3[3] = {x, y, z};
    int i3[3];
    double wt[3][3][4]; /* [axis][derivative order][stencil row] */
    for (int d = 0; d < 3; ++d) {
        double t;
        orc_cell(r3[d], n3[d], &i3[d], &t);
        orc_basis(t, wt[d][0], wt[d][1], wt[d][2]);
        const double nd = (double)n3[d];
        for (int a = 0; a < 4; ++a) {
            wt[d][1][a] *= nd;
            wt[d][2][a] *= nd * nd;
        }
    }
    struct { int i, j, k; } cell = {i3[0], i3[1], i3[2]};
    for (int n = 0; n < N; ++n) {
        double acc[10] = {0};
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                for (int c = 0; c < 4; ++c) {
                    const double p = row(ctx, cell.i + a, cell.j + b, cell.k + c, n);
                    for (int q = 0; q < 10; ++q)
                        acc[q] += wt[0][ORDERS[q][0]][a] * wt[1][ORDERS[q][1]][b] *
                                  wt[2][ORDERS[q][2]][c] * p;
                }
        write_outputs(kind, N, pos, acc, n, v, g, h, l);
    }
}

/* Periodic table coef[nx][ny][nz][N]; stencil row a of cell i is knot (i-1+a) mod n. */
typedef struct { int nx, ny, nz, N; const double *coef; } periodic_ctx;

static int wrap(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

static double periodic_row(const void *vctx, int a, int b, int c, int n)
{
    const periodic_ctx *p = (const periodic_ctx *)vctx;
    const int i = wrap(a - 1, p->nx), j = wrap(b - 1, p->ny), k = wrap(c - 1, p->nz);
    return p->coef[(((size_t)i * p->ny + j) * p->nz + k) * p->N + n];
}

/* Padded table [nx+3][ny+3][nz+3][N]; stencil rows of cell i are padded rows i..i+3. */
typedef struct { int nx, ny, nz, N; const double *pad; } padded_ctx;

static double padded_row(const void *vctx, int a, int b, int c, int n)
{
    const padded_ctx *p = (const padded_ctx *)vctx;
    return p->pad[(((size_t)a * (p->ny + 3) + b) * (p->nz + 3) + c) * p->N + n];
}

/*
 * Eq. (TricubicValue) over a periodic coefficient table (knot indices taken
 * mod n_d). kind: 0 = V (v), 1 = VGL (v, g, l), 2 = VGH (v, g, h; l if given).
 * Layouts: v[npos][N], g[npos][3][N], h[npos][6][N] (xx,xy,xz,yy,yz,zz), l[npos][N].
 */
void orc_eval_periodic(int kind, int nx, int ny, int nz, int N, const double *coef,
                       int npos, const double *x, const double *y, const double *z,
                       double *v, double *g, double *h, double *l)
{
    periodic_ctx ctx = {nx, ny, nz, N, coef};
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < npos; ++p)
        eval_one_position(kind, nx, ny, nz, N, periodic_row, &ctx, p, x[p], y[p], z[p],
                          v, g, h, l);
}

/* Eq. (TricubicValue) over a padded table [nx+3][ny+3][nz+3][N]; no index wrap. */
void orc_eval_padded(int kind, int nx, int ny, int nz, int N, const double *pad,
                     int npos, const double *x, const double *y, const double *z,
                     double *v, double *g, double *h, double *l)
{
    padded_ctx ctx = {nx, ny, nz, N, pad};
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < npos; ++p)
        eval_one_position(kind, nx, ny, nz, N, padded_row, &ctx, p, x[p], y[p], z[p],
                          v, g, h, l);
}

/*
 * Brute force over every knot of a periodic table and its periodic images:
 * f(r) = sum_{i,j,k} p[i][j][k] B(x n_x - i) B(y n_y - j) B(z n_z - k), the
 * knot sums of Eq. (TricubicValue) before truncation to the four nonzero
 * terms. Images are taken within +-2 cells of the unit cell, which covers the
 * support of B for any x in [0,1). No cell reduction is used. Intended for
 * tiny grids only (cost npos * nx*ny*nz * 125 * N).
 */
void orc_eval_bruteforce(int kind, int nx, int ny, int nz, int N, const double *coef,
                         int npos, const double *x, const double *y, const double *z,
                         double *v, double *g, double *h, double *l)
{
    for (int p = 0; p < npos; ++p) {
        double *acc = (double *)calloc((size_t)N * 10, sizeof(double));
        for (int i = 0; i < nx; ++i)
            for (int j = 0; j < ny; ++j)
                for (int k = 0; k < nz; ++k)
                    for (int ix = -2; ix <= 2; ++ix)
                        for (int iy = -2; iy <= 2; ++iy)
                            for (int iz = -2; iz <= 2; ++iz) {
                                double bx[3], by[3], bz[3];
                                orc_centred_bspline(x[p] * nx - (i + ix * nx), bx);
                                orc_centred_bspline(y[p] * ny - (j + iy * ny), by);
                                orc_centred_bspline(z[p] * nz - (k + iz * nz), bz);
                                if (bx[0] == 0.0 && bx[1] == 0.0 && bx[2] == 0.0) continue;
                                if (by[0] == 0.0 && by[1] == 0.0 && by[2] == 0.0) continue;
                                if (bz[0] == 0.0 && bz[1] == 0.0 && bz[2] == 0.0) continue;
                                const double sx[3] = {bx[0], bx[1] * nx, bx[2] * (double)nx * nx};
                                const double sy[3] = {by[0], by[1] * ny, by[2] * (double)ny * ny};
                                const double sz[3] = {bz[0], bz[1] * nz, bz[2] * (double)nz * nz};
                                const double *row = coef + (((size_t)i * ny + j) * nz + k) * N;
                                for (int q = 0; q < 10; ++q) {
                                    const double wq = sx[ORDERS[q][0]] * sy[ORDERS[q][1]] *
                                                      sz[ORDERS[q][2]];
                                    for (int n = 0; n < N; ++n) acc[(size_t)n * 10 + q] += wq * row[n];
                                }
                            }
        for (int n = 0; n < N; ++n) write_outputs(kind, N, p, acc + (size_t)n * 10, n, v, g, h, l);
        free(acc);
    }
}

/*
 * Padded table from a periodic one: pad[a][b][c] = coef[(a-1) mod nx]
 * [(b-1) mod ny][(c-1) mod nz], so that the stencil of cell i reads padded
 * rows i..i+3 (knots i-1..i+2 of Eq. SplineFunc) without wrapping.
 */
void orc_pad(int nx, int ny, int nz, int N, const double *coef, double *pad)
{
    periodic_ctx ctx = {nx, ny, nz, N, coef};
    for (int a = 0; a < nx + 3; ++a)
        for (int b = 0; b < ny + 3; ++b)
            for (int c = 0; c < nz + 3; ++c)
                for (int n = 0; n < N; ++n)
                    pad[(((size_t)a * (ny + 3) + b) * (nz + 3) + c) * N + n] =
                        periodic_row(&ctx, a, b, c, n);
}

/*
 * Reduced-precision table (not in the paper; the paper computes in single
 * precision throughout). Per orbital n: s_n = max |p[.][.][.][n]| over the
 * single-precision table (1 if the orbital is all zero), q = p / s_n divided
 * in single precision, then rounded to nearest-even in the target format.
 * dtype 1 = IEEE binary16, 2 = bfloat16. codes[cnt][N] holds the raw 16 bits.
 */
static uint16_t f32_to_bf16_rne(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}

static float bf16_to_f32(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

static uint16_t f32_to_f16_rne(float f)
{
    _Float16 hf = (_Float16)f;
    uint16_t b;
    memcpy(&b, &hf, 2);
    return b;
}

static float f16_to_f32(uint16_t b)
{
    _Float16 hf;
    memcpy(&hf, &b, 2);
    return (float)hf;
}

void orc_quantize(size_t cnt, int N, const float *p, int dtype, uint16_t *codes, float *scale)
{
    for (int n = 0; n < N; ++n) {
        float m = 0.0f;
        for (size_t r = 0; r < cnt; ++r) {
            const float a = fabsf(p[r * N + n]);
            if (a > m) m = a;
        }
        scale[n] = m > 0.0f ? m : 1.0f;
    }
    for (size_t r = 0; r < cnt; ++r)
        for (int n = 0; n < N; ++n) {
            volatile float q = p[r * N + n] / scale[n];
            codes[r * N + n] = dtype == 1 ? f32_to_f16_rne(q) : f32_to_bf16_rne(q);
        }
}

/* Value each code stands for: decoded code times s_n, exact in double. */
void orc_dequantize(size_t cnt, int N, const uint16_t *codes, const float *scale, int dtype,
                    double *out)
{
    for (size_t r = 0; r < cnt; ++r)
        for (int n = 0; n < N; ++n) {
            const float q = dtype == 1 ? f16_to_f32(codes[r * N + n]) : bf16_to_f32(codes[r * N + n]);
            out[r * N + n] = (double)q * (double)scale[n];
        }
}
