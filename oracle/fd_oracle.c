/*
 * fd_oracle.c -- the on-grid derivative step (test infrastructure only).
 *
 * From the 16 arrays g[6], K[6], alpha, beta[3] on a periodic nx x ny x nz grid (x fastest), builds the
 * 43-array input table of the metric-evolution chain: g, K, alpha, beta copied, d_k g_ij and d_j beta_i
 * by centred finite differences, literally:
 *   order 2:  (f(x+h) - f(x-h)) / (2h)
 *   order 4:  (8 (f(x+h) - f(x-h)) - (f(x+2h) - f(x-2h))) / (12h)
 * with neighbour indices wrapped periodically.  The chain oracle then evaluates the table.
 */
#include <stdint.h>

static int64_t wrap(int64_t i, int64_t m)
{
    int64_t r = i % m;
    return r < 0 ? r + m : r;
}

static double deriv(const double *f, int64_t ix, int64_t iy, int64_t iz, int axis, int64_t nx, int64_t ny,
                    int64_t nz, double h, int order)
{
    int64_t c[3] = {ix, iy, iz};
    const int64_t m[3] = {nx, ny, nz};
    double v[5];   /* f at offsets -2..2 along the axis */
    for (int o = -2; o <= 2; ++o) {
        int64_t q[3] = {c[0], c[1], c[2]};
        q[axis] = wrap(c[axis] + o, m[axis]);
        v[o + 2] = f[q[0] + nx * (q[1] + ny * q[2])];
    }
    if (order == 2)
        return (v[3] - v[1]) / (2.0 * h);
    return (8.0 * (v[3] - v[1]) - (v[4] - v[0])) / (12.0 * h);
}

int oracle_fd_inputs(const double *const *in16, int64_t nx, int64_t ny, int64_t nz, double hx, double hy,
                     double hz, int order, double *const *out43)
{
    if (!in16 || !out43 || nx < 1 || ny < 1 || nz < 1 || (order != 2 && order != 4))
        return -1;
    const double h[3] = {hx, hy, hz};
    for (int64_t iz = 0; iz < nz; ++iz)
        for (int64_t iy = 0; iy < ny; ++iy)
            for (int64_t ix = 0; ix < nx; ++ix) {
                const int64_t x = ix + nx * (iy + ny * iz);
                for (int p = 0; p < 6; ++p) {
                    out43[p][x] = in16[p][x];
                    out43[24 + p][x] = in16[6 + p][x];
                    for (int k = 0; k < 3; ++k)
                        out43[6 + 3 * p + k][x] = deriv(in16[p], ix, iy, iz, k, nx, ny, nz, h[k], order);
                }
                out43[30][x] = in16[12][x];
                for (int i = 0; i < 3; ++i) {
                    out43[31 + i][x] = in16[13 + i][x];
                    for (int j = 0; j < 3; ++j)
                        out43[34 + 3 * i + j][x] = deriv(in16[13 + i], ix, iy, iz, j, nx, ny, nz, h[j], order);
                }
            }
    return 0;
}
