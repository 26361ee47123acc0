/*
 * dtg_oracle.c -- the CPU oracle for the fused metric-evolution chain.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link or call this file: only the test
 * suite, the smoke check and the timed CPU baseline of the benchmark use it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * What it computes (Lewis & Pfeiffer, arXiv:1804.10120), one grid point at a time, in IEEE binary64,
 * compiled with floating-point contraction disabled:
 *   1. g^ij, the inverse of the symmetric 3x3 spatial metric g_ij (the paper names it and gives no
 *      method, Sec. 1 after Eq. 6).  Written out as adjugate / determinant, the determinant by first-row
 *      expansion.
 *   2. The Christoffel symbols of the second kind, Eq. 6:
 *          Gamma^i_jk = 1/2 sum_l g^il (d_k g_jl + d_j g_lk - d_l g_jk),
 *      evaluated for all 27 (i,j,k) with the terms in the order Eq. 6 prints them.
 *   3. The covariant derivative of the shift, the footnote to Listing 1 (Sec. 1):
 *          nabla_j beta_i = d_j beta_i - sum_k Gamma^k_ij beta_k.
 *   4. The metric evolution equation, Eq. 5:
 *          d_t g_ij = -2 alpha K_ij + nabla_i beta_j + nabla_j beta_i.
 * and the reverse-mode derivative of any linear functional of the 39 outputs (the adjoint; the paper
 * has none), derived by hand from steps 1-4.
 *
 * Storage convention (the paper keeps one element per symmetric pair through a lookup table, Sec. 2.2,
 * and fixes no order; this file fixes one):
 *   packed symmetric index p(i,j) for i<=j: (0,0)->0 (0,1)->1 (0,2)->2 (1,1)->3 (1,2)->4 (2,2)->5.
 *   Input table (43 arrays of n doubles):
 *     [0..5]   g[p]            g_ij
 *     [6..23]  dg[3*p+k]       d_k g_ij  (derivative index innermost, as dg(i,j)(k) in Listing 3)
 *     [24..29] K[p]            K_ij
 *     [30]     alpha
 *     [31..33] beta[i]         beta_i
 *     [34..42] dbeta[3*i+j]    d_j beta_i
 *   Output table (39 arrays of n doubles):
 *     [0..5]   ginv[p]         g^ij
 *     [6..23]  gamma[6*i+p(j,k)]  Gamma^i_jk
 *     [24..32] dbcov[3*i+j]    nabla_j beta_i
 *     [33..38] dtg[p]          d_t g_ij
 */
#include <stddef.h>
#include <stdint.h>

#define ORACLE_N_IN 43
#define ORACLE_N_OUT 39

static int sym_index(int i, int j)
{
    /* packed position of the unordered pair {i,j} */
    static const int table[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    return table[i][j];
}

/* Everything one point needs, unpacked into full index form. */
typedef struct {
    double G[3][3];       /* g_ij                        */
    double D[3][3][3];    /* D[i][j][k] = d_k g_ij       */
    double Kc[3][3];      /* K_ij                        */
    double alpha;
    double b[3];          /* beta_i                      */
    double B[3][3];       /* B[i][j] = d_j beta_i        */
} point_in;

typedef struct {
    double det;
    double H[3][3];       /* g^ij                        */
    double T[3][3][3];    /* T[l][j][k] = d_k g_jl + d_j g_lk - d_l g_jk (the bracket of Eq. 6) */
    double Gam[3][3][3];  /* Gamma^i_jk                  */
    double Nb[3][3];      /* Nb[i][j] = nabla_j beta_i   */
    double dtg[3][3];     /* d_t g_ij (all 9, symmetric up to rounding) */
} point_out;

static void load_point(const double *const in[ORACLE_N_IN], int64_t x, point_in *P)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            int p = sym_index(i, j);
            P->G[i][j] = in[0 + p][x];
            P->Kc[i][j] = in[24 + p][x];
            P->B[i][j] = in[34 + 3 * i + j][x];
            for (int k = 0; k < 3; ++k)
                P->D[i][j][k] = in[6 + 3 * p + k][x];
        }
    P->alpha = in[30][x];
    for (int i = 0; i < 3; ++i)
        P->b[i] = in[31 + i][x];
}

/* Step 1: inverse by the adjugate.  C[i][j] is the (i,j) cofactor; for a 3x3 matrix the cyclic
 * products carry the checkerboard sign.  g^ij = C[j][i] / det. */
static void inverse(const double G[3][3], double *det_out, double H[3][3])
{
    double C[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
            C[i][j] = G[i1][j1] * G[i2][j2] - G[i1][j2] * G[i2][j1];
        }
    double det = G[0][0] * C[0][0] + G[0][1] * C[0][1] + G[0][2] * C[0][2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            H[i][j] = C[j][i] / det;
    *det_out = det;
}

static void forward_point(const point_in *P, point_out *R)
{
    /* 1. inverse metric */
    inverse(P->G, &R->det, R->H);

    /* 2. Christoffel symbols, Eq. 6, terms in printed order */
    for (int l = 0; l < 3; ++l)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                R->T[l][j][k] = (P->D[j][l][k] + P->D[l][k][j]) - P->D[j][k][l];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                double s = 0.0;
                for (int l = 0; l < 3; ++l)
                    s += R->H[i][l] * R->T[l][j][k];
                R->Gam[i][j][k] = 0.5 * s;
            }

    /* 3. covariant derivative of the shift */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k)
                s += R->Gam[k][i][j] * P->b[k];
            R->Nb[i][j] = P->B[i][j] - s;
        }

    /* 4. Eq. 5: nabla_i beta_j = Nb[j][i], nabla_j beta_i = Nb[i][j] */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            R->dtg[i][j] = (-2.0 * P->alpha * P->Kc[i][j] + R->Nb[j][i]) + R->Nb[i][j];
}

/*
 * Forward over n points.  in: 43 arrays, out: 39 arrays, all of n doubles (see the header comment).
 * Returns 0, or -1 for a NULL table entry or n < 0.  A point with det(g) == 0 produces inf/nan, as the
 * definition does.
 */
int oracle_dtg_forward(const double *const in[ORACLE_N_IN], double *const out[ORACLE_N_OUT], int64_t n)
{
    if (n < 0 || !in || !out)
        return -1;
    for (int s = 0; s < ORACLE_N_IN; ++s)
        if (!in[s])
            return -1;
    for (int s = 0; s < ORACLE_N_OUT; ++s)
        if (!out[s])
            return -1;
    for (int64_t x = 0; x < n; ++x) {
        point_in P;
        point_out R;
        load_point(in, x, &P);
        forward_point(&P, &R);
        for (int i = 0; i < 3; ++i)
            for (int j = i; j < 3; ++j) {
                out[0 + sym_index(i, j)][x] = R.H[i][j];
                out[33 + sym_index(i, j)][x] = R.dtg[i][j];
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = j; k < 3; ++k)
                    out[6 + 6 * i + sym_index(j, k)][x] = R.Gam[i][j][k];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                out[24 + 3 * i + j][x] = R.Nb[i][j];
    }
    return 0;
}

/*
 * Adjoint.  Given upstream gradients gout (39 arrays laid out like the forward outputs; a NULL entry
 * means that output does not enter the functional), writes gin (43 arrays laid out like the inputs):
 * the gradient of  L = sum_x sum_c gout[c][x] * out[c][x]  with respect to every stored input value.
 * A symmetric input stored once (g_ij, K_ij, the pair index of d_k g_ij) receives the sum of the
 * derivatives through both of its index orders.
 *
 * Derivation (reverse order of the forward steps, per point):
 *   Eq. 5     dtg_ij = -2 a K_ij + Nb[j][i] + Nb[i][j]   (i<=j stored)
 *               Kbar_ij = -2 a W_ij;  abar = -2 sum_{i<=j} W_ij K_ij;
 *               Nbar[i][j] += W, Nbar[j][i] += W  (once each for i<j; 2W on the diagonal)
 *   footnote  Nb[i][j] = B[i][j] - sum_k Gam[k][i][j] b[k]
 *               Bbar = Nbar;  bbar_k = -sum_ij Nbar[i][j] Gam[k][i][j];
 *               Gambar[k][i][j] += -Nbar[i][j] b[k]   (then folded onto the stored j<=k entries)
 *   Eq. 6     Gam[i][j][k] = 1/2 sum_l H[i][l] T[l][j][k]   (stored j<=k)
 *               Hbar[i][l] += 1/2 sum_{j<=k} Gambar[i][jk] T[l][j][k];
 *               Tbar[l][jk] = 1/2 sum_i H[i][l] Gambar[i][jk]
 *             T[l][j][k] = D[j][l][k] + D[l][k][j] - D[j][k][l]
 *               scatter Tbar with the signs of the three terms onto D, then fold onto stored dg
 *   inverse   H = G^-1:  d H = -H dG H  =>  Gbar = -H Hbar H  (H symmetric), folded onto stored g.
 */
int oracle_dtg_backward(const double *const in[ORACLE_N_IN], const double *const gout[ORACLE_N_OUT],
                        double *const gin[ORACLE_N_IN], int64_t n)
{
    if (n < 0 || !in || !gout || !gin)
        return -1;
    for (int s = 0; s < ORACLE_N_IN; ++s)
        if (!in[s] || !gin[s])
            return -1;
    for (int64_t x = 0; x < n; ++x) {
        point_in P;
        point_out R;
        load_point(in, x, &P);
        forward_point(&P, &R);

        /* upstream gradients, 0 where absent */
        double Wg[6], Wgam[3][6], Wnb[3][3], Wdt[6];
        for (int p = 0; p < 6; ++p) {
            Wg[p] = gout[0 + p] ? gout[0 + p][x] : 0.0;
            Wdt[p] = gout[33 + p] ? gout[33 + p][x] : 0.0;
        }
        for (int i = 0; i < 3; ++i)
            for (int p = 0; p < 6; ++p)
                Wgam[i][p] = gout[6 + 6 * i + p] ? gout[6 + 6 * i + p][x] : 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                Wnb[i][j] = gout[24 + 3 * i + j] ? gout[24 + 3 * i + j][x] : 0.0;

        /* Eq. 5 */
        double Kbar[6], abar = 0.0, Nbar[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                Nbar[i][j] = Wnb[i][j];
        for (int i = 0; i < 3; ++i)
            for (int j = i; j < 3; ++j) {
                int p = sym_index(i, j);
                Kbar[p] = -2.0 * P.alpha * Wdt[p];
                abar += -2.0 * P.Kc[i][j] * Wdt[p];
                Nbar[j][i] += Wdt[p];
                Nbar[i][j] += Wdt[p];
            }

        /* covariant derivative of the shift */
        double Bbar[3][3], bbar[3], Gambar[3][6];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                Bbar[i][j] = Nbar[i][j];
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    s += Nbar[i][j] * R.Gam[k][i][j];
            bbar[k] = -s;
        }
        for (int k = 0; k < 3; ++k)
            for (int p = 0; p < 6; ++p)
                Gambar[k][p] = Wgam[k][p];
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    Gambar[k][sym_index(i, j)] += -Nbar[i][j] * P.b[k];

        /* Eq. 6 */
        double Hbar[3][3], Tbar[3][6];
        for (int i = 0; i < 3; ++i)
            for (int l = 0; l < 3; ++l) {
                double s = 0.0;
                for (int j = 0; j < 3; ++j)
                    for (int k = j; k < 3; ++k)
                        s += Gambar[i][sym_index(j, k)] * R.T[l][j][k];
                Hbar[i][l] = 0.5 * s;
            }
        for (int l = 0; l < 3; ++l)
            for (int j = 0; j < 3; ++j)
                for (int k = j; k < 3; ++k) {
                    double s = 0.0;
                    for (int i = 0; i < 3; ++i)
                        s += R.H[i][l] * Gambar[i][sym_index(j, k)];
                    Tbar[l][sym_index(j, k)] = 0.5 * s;
                }
        double Dbar[3][3][3] = {{{0}}};
        for (int l = 0; l < 3; ++l)
            for (int j = 0; j < 3; ++j)
                for (int k = j; k < 3; ++k) {
                    double t = Tbar[l][sym_index(j, k)];
                    Dbar[j][l][k] += t;
                    Dbar[l][k][j] += t;
                    Dbar[j][k][l] -= t;
                }
        double dgbar[6][3] = {{0}};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 3; ++c)
                    dgbar[sym_index(a, b)][c] += Dbar[a][b][c];

        /* stored g^ij enters the functional through its i<=j entry */
        for (int i = 0; i < 3; ++i)
            for (int j = i; j < 3; ++j)
                Hbar[i][j] += Wg[sym_index(i, j)];

        /* inverse: Gbar = -H Hbar H */
        double M[3][3], Gbar[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int l = 0; l < 3; ++l)
                    s += Hbar[i][l] * R.H[l][j];
                M[i][j] = s;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int l = 0; l < 3; ++l)
                    s += R.H[i][l] * M[l][j];
                Gbar[i][j] = -s;
            }
        double gbar[6] = {0};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                gbar[sym_index(i, j)] += Gbar[i][j];

        for (int p = 0; p < 6; ++p) {
            gin[0 + p][x] = gbar[p];
            gin[24 + p][x] = Kbar[p];
            for (int k = 0; k < 3; ++k)
                gin[6 + 3 * p + k][x] = dgbar[p][k];
        }
        gin[30][x] = abar;
        for (int i = 0; i < 3; ++i) {
            gin[31 + i][x] = bbar[i];
            for (int j = 0; j < 3; ++j)
                gin[34 + 3 * i + j][x] = Bbar[i][j];
        }
    }
    return 0;
}

/* Determinant of g at each point (step 1's intermediate), exposed for the conditioning checks. */
int oracle_metric_det(const double *const g[6], double *det, int64_t n)
{
    if (n < 0 || !g || !det)
        return -1;
    for (int64_t x = 0; x < n; ++x) {
        double G[3][3], H[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                G[i][j] = g[sym_index(i, j)][x];
        inverse(G, &det[x], H);
    }
    return 0;
}
