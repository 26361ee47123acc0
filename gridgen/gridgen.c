/*
 * gridgen.c -- seeded synthetic grid inputs for the metric-evolution chain.
 *
 * This module holds only input generation: no step of the method's arithmetic.  Both the CPU oracle
 * and the CUDA library are fed from it, so both see bit-identical inputs.
 *
 * Counter-based: every value is a pure function of (seed, stream id, point index), so any chunk of any
 * stream can be produced independently, in any order, by any number of threads.
 *   key(seed, stream) = mix(mix(seed + G) + (stream + 1) * G)
 *   bits(k, c)        = mix(k + (c + 1) * G)
 * where mix is the SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014) and G = 0x9E3779B97F4A7C15.
 *   uniform [0,1): (bits >> 11) * 2^-53
 *   normal:        Box-Muller on the counter pair (2c, 2c+1):
 *                  sqrt(-2 ln(1 - u0)) * cos(2 pi u1)
 *
 * Stream ids follow the 43-array input table of the library (g[6], dg[18], K[6], alpha, beta[3],
 * dbeta[9]) plus a caller-supplied base, so that several grids or extra fields (upstream gradients)
 * draw from disjoint streams.
 */
#include <math.h>
#include <stdint.h>

#define GG_GOLDEN 0x9E3779B97F4A7C15ULL

static uint64_t mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t stream_key(uint64_t seed, uint64_t stream)
{
    return mix(mix(seed + GG_GOLDEN) + (stream + 1) * GG_GOLDEN);
}

static double unif(uint64_t key, uint64_t c)
{
    return (double)(mix(key + (c + 1) * GG_GOLDEN) >> 11) * 0x1.0p-53;
}

static double normal(uint64_t key, uint64_t c)
{
    double u0 = unif(key, 2 * c), u1 = unif(key, 2 * c + 1);
    return sqrt(-2.0 * log(1.0 - u0)) * cos(6.283185307179586 * u1);
}

uint64_t gridgen_bits(uint64_t seed, uint64_t stream, uint64_t c)
{
    return mix(stream_key(seed, stream) + (c + 1) * GG_GOLDEN);
}

/* out[x] = lo + (hi - lo) * U[0,1) for x in [0, n), point indices offset .. offset+n-1 */
void gridgen_uniform(uint64_t seed, uint64_t stream, int64_t offset, int64_t n, double lo, double hi,
                     double *out)
{
    uint64_t k = stream_key(seed, stream);
    for (int64_t x = 0; x < n; ++x)
        out[x] = lo + (hi - lo) * unif(k, (uint64_t)(offset + x));
}

/* out[x] = mean + sigma * N(0,1) */
void gridgen_normal(uint64_t seed, uint64_t stream, int64_t offset, int64_t n, double mean, double sigma,
                    double *out)
{
    uint64_t k = stream_key(seed, stream);
    for (int64_t x = 0; x < n; ++x)
        out[x] = mean + sigma * normal(k, (uint64_t)(offset + x));
}

/*
 * The random-grid recipe, for points offset .. offset+n-1, into 43 arrays of n doubles:
 *   g_ij  = delta_ij + 0.1 * S_ij, S_ij uniform [-1,1]   (symmetric: one draw per stored pair; with
 *           |off-diagonal row sum| <= 0.2 and diagonal >= 0.9 the matrix is SPD, eigenvalues in [0.7,1.3])
 *   d_k g_ij uniform [-0.1, 0.1]
 *   K_ij  normal(0, 0.1) (one draw per stored pair)
 *   alpha uniform [0.5, 1.5]
 *   beta_i normal(0, 0.1)
 *   d_j beta_i normal(0, 0.1) (all 9, not symmetric)
 * Stream id of input array s is stream_base + s.
 */
void gridgen_random_grid(uint64_t seed, uint64_t stream_base, int64_t offset, int64_t n, double *const out[43])
{
    static const int diag[6] = {1, 0, 0, 1, 0, 1};
    for (int p = 0; p < 6; ++p)
        gridgen_uniform(seed, stream_base + p, offset, n, diag[p] - 0.1, diag[p] + 0.1, out[p]);
    for (int s = 6; s < 24; ++s)
        gridgen_uniform(seed, stream_base + s, offset, n, -0.1, 0.1, out[s]);
    for (int s = 24; s < 30; ++s)
        gridgen_normal(seed, stream_base + s, offset, n, 0.0, 0.1, out[s]);
    gridgen_uniform(seed, stream_base + 30, offset, n, 0.5, 1.5, out[30]);
    for (int s = 31; s < 43; ++s)
        gridgen_normal(seed, stream_base + s, offset, n, 0.0, 0.1, out[s]);
}

/*
 * Conformally flat grid: side^3 points x_a = lo + (hi - lo) * a / (side - 1) (endpoints included),
 * row-major with the first coordinate fastest.  psi = 1 + 0.5 exp(-r^2), d_k psi = -x_k exp(-r^2),
 * g_ij = psi^4 delta_ij, d_k g_ij = 4 psi^3 d_k psi delta_ij, alpha = 1, and beta, d beta, K zero.
 * Writes points offset .. offset+n-1 of the flattened grid.
 */
void gridgen_conformal_grid(int64_t side, double lo, double hi, int64_t offset, int64_t n, double *const out[43])
{
    static const int diag[6] = {1, 0, 0, 1, 0, 1};
    for (int64_t t = 0; t < n; ++t) {
        int64_t x = offset + t;
        int64_t a0 = x % side, a1 = (x / side) % side, a2 = x / (side * side);
        double c[3];
        c[0] = lo + (hi - lo) * (double)a0 / (double)(side - 1);
        c[1] = lo + (hi - lo) * (double)a1 / (double)(side - 1);
        c[2] = lo + (hi - lo) * (double)a2 / (double)(side - 1);
        double r2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        double e = exp(-r2);
        double psi = 1.0 + 0.5 * e;
        double psi3 = psi * psi * psi, psi4 = psi3 * psi;
        for (int p = 0; p < 6; ++p) {
            out[p][t] = diag[p] ? psi4 : 0.0;
            for (int k = 0; k < 3; ++k)
                out[6 + 3 * p + k][t] = diag[p] ? 4.0 * psi3 * (-c[k] * e) : 0.0;
            out[24 + p][t] = 0.0;
        }
        out[30][t] = 1.0;
        for (int s = 31; s < 43; ++s)
            out[s][t] = 0.0;
    }
}

/*
 * Smooth periodic fields on an nx x ny x nz grid over the unit box (x fastest, coordinate a / n per
 * axis), 16 arrays laid out as g[6], K[6], alpha, beta[3]: each field is base + amp * sum of three
 * Fourier modes a_m sin(2 pi k_m . x + phi_m), with integer wavevectors k_m (components in [-3, 3]),
 * a_m ~ U[-1/3, 1/3] and phi_m ~ U[0, 2 pi) drawn from (seed, field).  g: base delta_ij, amp 0.05
 * (diagonal >= 0.95, off-diagonal <= 0.05: SPD); K, beta: amp 0.1; alpha: base 1, amp 0.2.
 * Writes points offset .. offset+n-1.
 */
void gridgen_periodic_fields(uint64_t seed, int64_t nx, int64_t ny, int64_t nz, int64_t offset, int64_t n,
                             double *const out[16])
{
    static const int diag[6] = {1, 0, 0, 1, 0, 1};
    double k[16][3][3], am[16][3], ph[16][3], base[16], amp[16];
    for (int f = 0; f < 16; ++f) {
        const uint64_t key = stream_key(seed, 8192 + (uint64_t)f);
        for (int m = 0; m < 3; ++m) {
            for (int d = 0; d < 3; ++d)
                k[f][m][d] = (double)((int)(mix(key + (uint64_t)(16 * m + d + 1) * GG_GOLDEN) % 7) - 3);
            am[f][m] = (2.0 * unif(key, 100 + m) - 1.0) / 3.0;
            ph[f][m] = 6.283185307179586 * unif(key, 200 + m);
        }
        base[f] = f < 6 ? (double)diag[f] : (f == 12 ? 1.0 : 0.0);
        amp[f] = f < 6 ? 0.05 : (f == 12 ? 0.2 : 0.1);
    }
    for (int64_t t = 0; t < n; ++t) {
        const int64_t x = offset + t;
        const double c[3] = {(double)(x % nx) / (double)nx, (double)((x / nx) % ny) / (double)ny,
                             (double)(x / (nx * ny)) / (double)nz};
        for (int f = 0; f < 16; ++f) {
            double s = 0.0;
            for (int m = 0; m < 3; ++m)
                s += am[f][m] * sin(6.283185307179586 * (k[f][m][0] * c[0] + k[f][m][1] * c[1] + k[f][m][2] * c[2]) +
                                    ph[f][m]);
            out[f][t] = base[f] + amp[f] * s;
        }
    }
}
