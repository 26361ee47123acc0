/*
 * expr_oracle.c -- CPU oracle for the benchmark expressions of Sec. 5.1 (Eqs. 9-21).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's CPU legs, never by the CUDA library.
 *
 * Every index runs over the three spatial dimensions; every tensor component is an array of n doubles
 * (structure of arrays).  Component order is row-major over the indices as written (B_i^m -> B[3i+m],
 * E_mjkl -> E[27m+9j+3k+l]); the symmetric g_ij and K_ij of Eq. 21 are packed (00,01,02,11,12,22).
 * Each expression is evaluated literally, left to right, with no fused multiply-add:
 *   Eq.  9-11  A = B                       (3, 9, 27 components)
 *   Eq. 12-14  A_i = B_i + C_i (+ D_i (+ E_i))
 *   Eq. 15-17  A_ij = B_i C_j,  A_ijk = B_i C_j D_k,  A_ijkl = B_i C_j D_k E_l
 *   Eq. 18     A_ijkl = sum_m B_im E_mjkl
 *   Eq. 19     A_ijkl = sum_m sum_n C_jn B_im E_mnkl
 *   Eq. 20     A_ijkl = sum_m sum_n sum_o D_ko C_jn B_im E_mnol
 *   Eq. 21     K_ij = 2 alpha g_ij + beta_i beta_j
 * Input table order: the operands in the order they are named above (Eq. 19: B, C, E; Eq. 20: B, C,
 * D, E; Eq. 21: alpha, g, beta); the output table holds A (or K).
 */
#include <stdint.h>

static int expr_sym(int i, int j)
{
    static const int t[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    return t[i][j];
}

int oracle_expr(int eq, const double *const *in, double *const *out, int64_t n)
{
    if (n < 0 || !in || !out)
        return -1;
    for (int64_t x = 0; x < n; ++x) {
        switch (eq) {
        case 9: case 10: case 11: {
            const int c = eq == 9 ? 3 : eq == 10 ? 9 : 27;
            for (int q = 0; q < c; ++q)
                out[q][x] = in[q][x];
            break;
        }
        case 12: case 13: case 14: {
            const int terms = eq - 10;   /* 2, 3, 4 operands */
            for (int i = 0; i < 3; ++i) {
                double s = in[i][x];
                for (int t = 1; t < terms; ++t)
                    s = s + in[3 * t + i][x];
                out[i][x] = s;
            }
            break;
        }
        case 15:
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    out[3 * i + j][x] = in[i][x] * in[3 + j][x];
            break;
        case 16:
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    for (int k = 0; k < 3; ++k)
                        out[9 * i + 3 * j + k][x] = (in[i][x] * in[3 + j][x]) * in[6 + k][x];
            break;
        case 17:
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    for (int k = 0; k < 3; ++k)
                        for (int l = 0; l < 3; ++l)
                            out[27 * i + 9 * j + 3 * k + l][x] =
                                ((in[i][x] * in[3 + j][x]) * in[6 + k][x]) * in[9 + l][x];
            break;
        case 18:   /* B[9], E[81] */
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    for (int k = 0; k < 3; ++k)
                        for (int l = 0; l < 3; ++l) {
                            double s = 0.0;
                            for (int m = 0; m < 3; ++m)
                                s += in[3 * i + m][x] * in[9 + 27 * m + 9 * j + 3 * k + l][x];
                            out[27 * i + 9 * j + 3 * k + l][x] = s;
                        }
            break;
        case 19:   /* B[9], C[9], E[81] */
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    for (int k = 0; k < 3; ++k)
                        for (int l = 0; l < 3; ++l) {
                            double s = 0.0;
                            for (int m = 0; m < 3; ++m)
                                for (int nn = 0; nn < 3; ++nn)
                                    s += (in[9 + 3 * j + nn][x] * in[3 * i + m][x]) *
                                         in[18 + 27 * m + 9 * nn + 3 * k + l][x];
                            out[27 * i + 9 * j + 3 * k + l][x] = s;
                        }
            break;
        case 20:   /* B[9], C[9], D[9], E[81] */
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    for (int k = 0; k < 3; ++k)
                        for (int l = 0; l < 3; ++l) {
                            double s = 0.0;
                            for (int m = 0; m < 3; ++m)
                                for (int nn = 0; nn < 3; ++nn)
                                    for (int o = 0; o < 3; ++o)
                                        s += ((in[18 + 3 * k + o][x] * in[9 + 3 * j + nn][x]) * in[3 * i + m][x]) *
                                             in[27 + 27 * m + 9 * nn + 3 * o + l][x];
                            out[27 * i + 9 * j + 3 * k + l][x] = s;
                        }
            break;
        case 21:   /* alpha, g[6], beta[3] -> K[6] */
            for (int i = 0; i < 3; ++i)
                for (int j = i; j < 3; ++j)
                    out[expr_sym(i, j)][x] = (2.0 * in[0][x]) * in[1 + expr_sym(i, j)][x] + in[7 + i][x] * in[7 + j][x];
            break;
        default:
            return -1;
        }
    }
    return 0;
}
