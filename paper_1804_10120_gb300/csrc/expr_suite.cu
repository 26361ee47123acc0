// expr_suite.cu -- the benchmark expressions of Sec. 5.1 (Eqs. 9-21), in two forms:
//   TL_EXPR_FUSED  ("Tensors" in Sec. 5.5): one kernel per expression, one thread per grid point
//                  computing every component of the left-hand side, the pointer tables as kernel
//                  parameters;
//   TL_EXPR_ARRAYS ("Arrays" in Sec. 5.5): the explicit component loops of Listing 1 around pointwise
//                  kernels -- one launch per left-hand-side component and per value of every
//                  contracted index.
// Indices are spatial (dimension 3); components are row-major over the indices as written; Eq. 21's
// g_ij and K_ij are packed symmetric (00,01,02,11,12,22).  Sums without a contraction and products
// are evaluated left to right without FMA (the same roundings as the literal expression); the fused
// contractions apply one 3x3 factor at a time with FMA.
#include <algorithm>

#include "tl_common.cuh"
#include "tl_host.h"
#include "tl_kernels.h"

namespace tl {

constexpr int kExprMaxIn = 108, kExprMaxOut = 81;
struct ExprArgs {
    const double *in[kExprMaxIn];
    double *out[kExprMaxOut];
};

__host__ __device__ constexpr int expr_n_in(int eq)
{
    return eq <= 11 ? (eq == 9 ? 3 : eq == 10 ? 9 : 27)
         : eq <= 14 ? 3 * (eq - 10)
         : eq <= 17 ? 3 * (eq - 13)
         : eq == 18 ? 90 : eq == 19 ? 99 : eq == 20 ? 108 : 10;
}
__host__ __device__ constexpr int expr_n_out(int eq)
{
    return eq <= 11 ? expr_n_in(eq) : eq <= 14 ? 3 : eq == 15 ? 9 : eq == 16 ? 27 : eq == 21 ? 6 : 81;
}

// ------------------------------------------------------------------------------------- fused kernels
template <int EQ> __device__ __forceinline__ void expr_point(const ExprArgs &a, int64_t x)
{
    auto L = [&](int s) { return ld_stream(a.in[s] + x); };
    auto S = [&](int s, double v) { st_stream(a.out[s] + x, v); };
    if (EQ <= 11) {
#pragma unroll
        for (int q = 0; q < expr_n_in(EQ); ++q)
            S(q, L(q));
    } else if (EQ <= 14) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double s = L(i);
#pragma unroll
            for (int t = 1; t < EQ - 10; ++t)
                s = __dadd_rn(s, L(3 * t + i));
            S(i, s);
        }
    } else if (EQ <= 17) {
        constexpr int R = EQ - 13;   // rank of the outer product
        double v[4][3];
#pragma unroll
        for (int t = 0; t < R; ++t)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                v[t][i] = L(3 * t + i);
        constexpr int C = R == 2 ? 9 : R == 3 ? 27 : 81;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            int rem = c, idx[4];
#pragma unroll
            for (int t = R - 1; t >= 0; --t) {
                idx[t] = rem % 3;
                rem /= 3;
            }
            // rank 3: every other product on the integer pipes (mul_int, the same IEEE product), which
            // balances the FP64 pipe against instruction issue (3999 -> 4546 GB/s at N = 2^22); at
            // rank 4 the same split measured slower (3079 -> 2066 GB/s) and all products stay FP64
            constexpr bool kMix = R == 3;
            double p = (kMix && (c & 1)) ? mul_int(v[0][idx[0]], v[1][idx[1]]) : __dmul_rn(v[0][idx[0]], v[1][idx[1]]);
#pragma unroll
            for (int t = 2; t < R; ++t)
                p = (kMix && ((c + t) & 1)) ? mul_int(p, v[t][idx[t]]) : __dmul_rn(p, v[t][idx[t]]);
            S(c, p);
        }
    } else if (EQ == 18) {           // A_ijkl = sum_m B_im E_mjkl, one (j,k,l) slice at a time
        // (in 18 and 19 the first product of each contraction is mul_int: 3190 -> 4213 and 1726 ->
        // 2198 GB/s at N = 2^22; in 20 the extra registers cost more than the FP64 slots saved)
        double B[9];
#pragma unroll
        for (int q = 0; q < 9; ++q)
            B[q] = L(q);
#pragma unroll
        for (int r = 0; r < 27; ++r) {
            const double e0 = L(9 + r), e1 = L(9 + 27 + r), e2 = L(9 + 54 + r);
#pragma unroll
            for (int i = 0; i < 3; ++i)
                S(27 * i + r, fma(B[3 * i + 2], e2, fma(B[3 * i + 1], e1, mul_int(B[3 * i], e0))));
        }
    } else if (EQ == 19) {           // A_ijkl = sum_mn C_jn B_im E_mnkl = (B E_kl C^T)_ij per (k,l)
        double B[9], C[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            B[q] = L(q);
            C[q] = L(9 + q);
        }
#pragma unroll
        for (int r = 0; r < 9; ++r) {
            double E[3][3], P[3][3];
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int nn = 0; nn < 3; ++nn)
                    E[m][nn] = L(18 + 27 * m + 9 * nn + r);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int nn = 0; nn < 3; ++nn)
                    P[i][nn] = fma(B[3 * i + 2], E[2][nn], fma(B[3 * i + 1], E[1][nn], mul_int(B[3 * i], E[0][nn])));
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    S(27 * i + 9 * j + r, fma(C[3 * j + 2], P[i][2], fma(C[3 * j + 1], P[i][1], mul_int(C[3 * j], P[i][0]))));
        }
    } else if (EQ == 20) {           // A_ijkl = sum_mno D_ko C_jn B_im E_mnol, per l: three 3x3 factors
        double B[9], C[9], D[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            B[q] = L(q);
            C[q] = L(9 + q);
            D[q] = L(18 + q);
        }
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            double T[27];            // T[mno] = E_mnol, then transformed in place index by index
#pragma unroll
            for (int q = 0; q < 27; ++q)
                T[q] = L(27 + 3 * q + l);
            double U[27];
#pragma unroll
            for (int mn = 0; mn < 9; ++mn)          // apply D on o -> k
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    U[3 * mn + k] = fma(D[3 * k + 2], T[3 * mn + 2], fma(D[3 * k + 1], T[3 * mn + 1], D[3 * k] * T[3 * mn]));
#pragma unroll
            for (int m = 0; m < 3; ++m)             // apply C on n -> j
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        T[9 * m + 3 * j + k] = fma(C[3 * j + 2], U[9 * m + 6 + k],
                                                   fma(C[3 * j + 1], U[9 * m + 3 + k], C[3 * j] * U[9 * m + k]));
#pragma unroll
            for (int i = 0; i < 3; ++i)             // apply B on m -> i
#pragma unroll
                for (int jk = 0; jk < 9; ++jk)
                    S(27 * i + 3 * jk + l, fma(B[3 * i + 2], T[18 + jk], fma(B[3 * i + 1], T[9 + jk], B[3 * i] * T[jk])));
        }
    } else {                         // EQ == 21: K_ij = 2 alpha g_ij + beta_i beta_j
        const double a2 = __dmul_rn(2.0, L(0));
        double b[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            b[i] = L(7 + i);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j)
                S(sym(i, j), __dadd_rn(__dmul_rn(a2, L(1 + sym(i, j))), __dmul_rn(b[i], b[j])));
    }
}

template <int EQ> __global__ void __launch_bounds__(256) expr_fused_kernel(const ExprArgs a, int64_t n)
{
    const GridStride gs;
    for (int64_t x = gs.first; x < n; x += gs.step)
        expr_point<EQ>(a, x);
}

// ---------------------------------------------------------------------------------- pointwise kernels
// One component, one term: out = f0 * f1 * ... (left to right), out = a0 + a1 + ..., out += product,
// out = 2 alpha g + b_i b_j.
enum PwOp { PW_COPY = 0, PW_SUM = 1, PW_PROD = 2, PW_ACC_PROD = 3, PW_KIJ = 4 };
struct PwArgs {
    const double *f[4];
    double *out;
    int nf;
};

template <int OP, int NF> __global__ void __launch_bounds__(256) pointwise_kernel(const PwArgs a, int64_t n)
{
    const GridStride gs;
    for (int64_t x = gs.first; x < n; x += gs.step) {
        double v;
        if (OP == PW_COPY) {
            v = a.f[0][x];
        } else if (OP == PW_SUM) {
            v = a.f[0][x];
#pragma unroll
            for (int t = 1; t < NF; ++t)
                v = __dadd_rn(v, a.f[t][x]);
        } else if (OP == PW_KIJ) {
            v = __dadd_rn(__dmul_rn(__dmul_rn(2.0, a.f[0][x]), a.f[1][x]), __dmul_rn(a.f[2][x], a.f[3][x]));
        } else {
            v = a.f[0][x];
#pragma unroll
            for (int t = 1; t < NF; ++t)
                v = __dmul_rn(v, a.f[t][x]);
            if (OP == PW_ACC_PROD)
                v = __dadd_rn(a.out[x], v);
        }
        a.out[x] = v;
    }
}

template <int OP> static void pw_launch(const PwArgs &a, int64_t n, int grid, cudaStream_t s)
{
    switch (a.nf) {
    case 1: pointwise_kernel<OP, 1><<<grid, 256, 0, s>>>(a, n); break;
    case 2: pointwise_kernel<OP, 2><<<grid, 256, 0, s>>>(a, n); break;
    case 3: pointwise_kernel<OP, 3><<<grid, 256, 0, s>>>(a, n); break;
    default: pointwise_kernel<OP, 4><<<grid, 256, 0, s>>>(a, n); break;
    }
}

static cudaError_t pw(int op, const double *f0, const double *f1, const double *f2, const double *f3, int nf,
                      double *out, int64_t n, int grid, cudaStream_t s)
{
    PwArgs a;
    a.f[0] = f0;
    a.f[1] = f1;
    a.f[2] = f2;
    a.f[3] = f3;
    a.out = out;
    a.nf = nf;
    switch (op) {
    case PW_COPY: pointwise_kernel<PW_COPY, 1><<<grid, 256, 0, s>>>(a, n); break;
    case PW_SUM: pw_launch<PW_SUM>(a, n, grid, s); break;
    case PW_PROD: pw_launch<PW_PROD>(a, n, grid, s); break;
    case PW_ACC_PROD: pw_launch<PW_ACC_PROD>(a, n, grid, s); break;
    default: pointwise_kernel<PW_KIJ, 4><<<grid, 256, 0, s>>>(a, n); break;
    }
    return cudaGetLastError();
}

// The "Arrays" evaluation: loops over components and contracted indices on the host, one launch each.
static cudaError_t expr_arrays(int eq, const double *const *in, double *const *out, int64_t n, int grid, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    auto run = [&](int op, const double *f0, const double *f1, const double *f2, const double *f3, int nf, double *o) {
        if (e == cudaSuccess)
            e = pw(op, f0, f1, f2, f3, nf, o, n, grid, s);
    };
    if (eq <= 11) {
        for (int q = 0; q < expr_n_in(eq); ++q)
            run(PW_COPY, in[q], nullptr, nullptr, nullptr, 1, out[q]);
    } else if (eq <= 14) {
        const int terms = eq - 10;
        for (int i = 0; i < 3; ++i)
            run(PW_SUM, in[i], in[3 + i], terms > 2 ? in[6 + i] : nullptr, terms > 3 ? in[9 + i] : nullptr, terms, out[i]);
    } else if (eq <= 17) {
        const int R = eq - 13, C = R == 2 ? 9 : R == 3 ? 27 : 81;
        for (int c = 0; c < C; ++c) {
            int rem = c, idx[4] = {0, 0, 0, 0};
            for (int t = R - 1; t >= 0; --t) {
                idx[t] = rem % 3;
                rem /= 3;
            }
            run(PW_PROD, in[idx[0]], in[3 + idx[1]], R > 2 ? in[6 + idx[2]] : nullptr, R > 3 ? in[9 + idx[3]] : nullptr, R,
                out[c]);
        }
    } else if (eq == 18) {
        for (int i = 0; i < 3; ++i)
            for (int r = 0; r < 27; ++r)
                for (int m = 0; m < 3; ++m)
                    run(m == 0 ? PW_PROD : PW_ACC_PROD, in[3 * i + m], in[9 + 27 * m + r], nullptr, nullptr, 2, out[27 * i + r]);
    } else if (eq == 19) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int r = 0; r < 9; ++r)
                    for (int m = 0; m < 3; ++m)
                        for (int nn = 0; nn < 3; ++nn)
                            run(m == 0 && nn == 0 ? PW_PROD : PW_ACC_PROD, in[9 + 3 * j + nn], in[3 * i + m],
                                in[18 + 27 * m + 9 * nn + r], nullptr, 3, out[27 * i + 9 * j + r]);
    } else if (eq == 20) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l)
                        for (int m = 0; m < 3; ++m)
                            for (int nn = 0; nn < 3; ++nn)
                                for (int o = 0; o < 3; ++o)
                                    run(m == 0 && nn == 0 && o == 0 ? PW_PROD : PW_ACC_PROD, in[18 + 3 * k + o],
                                        in[9 + 3 * j + nn], in[3 * i + m], in[27 + 27 * m + 9 * nn + 3 * o + l], 4,
                                        out[27 * i + 9 * j + 3 * k + l]);
    } else {
        for (int i = 0; i < 3; ++i)
            for (int j = i; j < 3; ++j)
                run(PW_KIJ, in[0], in[1 + sym(i, j)], in[7 + i], in[7 + j], 4, out[sym(i, j)]);
    }
    return e;
}

template <int EQ> static cudaError_t launch_fused_eq(const ExprArgs &a, int64_t n, int grid, cudaStream_t s)
{
    expr_fused_kernel<EQ><<<grid, 256, 0, s>>>(a, n);
    return cudaGetLastError();
}

static cudaError_t expr_fused(int eq, const ExprArgs &a, int64_t n, int grid, cudaStream_t s)
{
    switch (eq) {
    case 9: return launch_fused_eq<9>(a, n, grid, s);
    case 10: return launch_fused_eq<10>(a, n, grid, s);
    case 11: return launch_fused_eq<11>(a, n, grid, s);
    case 12: return launch_fused_eq<12>(a, n, grid, s);
    case 13: return launch_fused_eq<13>(a, n, grid, s);
    case 14: return launch_fused_eq<14>(a, n, grid, s);
    case 15: return launch_fused_eq<15>(a, n, grid, s);
    case 16: return launch_fused_eq<16>(a, n, grid, s);
    case 17: return launch_fused_eq<17>(a, n, grid, s);
    case 18: return launch_fused_eq<18>(a, n, grid, s);
    case 19: return launch_fused_eq<19>(a, n, grid, s);
    case 20: return launch_fused_eq<20>(a, n, grid, s);
    case 21: return launch_fused_eq<21>(a, n, grid, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace tl

using namespace tl;

extern "C" {

tl_status tl_expr_arity(int32_t eq, int32_t *n_in, int32_t *n_out)
{
    if (eq < 9 || eq > 21)
        return fail(TL_ERR_INVALID_ARG, "expression %d: only Eqs. 9-21 are provided", (int)eq);
    if (n_in)
        *n_in = expr_n_in(eq);
    if (n_out)
        *n_out = expr_n_out(eq);
    return TL_OK;
}

tl_status tl_expr_eval(int32_t eq, const double *const *in, double *const *out, int64_t n, tl_expr_mode mode,
                       tl_stream stream)
{
    if (eq < 9 || eq > 21)
        return fail(TL_ERR_INVALID_ARG, "expression %d: only Eqs. 9-21 are provided", (int)eq);
    if (!in || !out)
        return fail(TL_ERR_INVALID_ARG, "NULL table");
    if (n < 0)
        return fail(TL_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
    if (mode != TL_EXPR_FUSED && mode != TL_EXPR_ARRAYS)
        return fail(TL_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
    const void *const *tabs[2] = {(const void *const *)in, (const void *const *)out};
    const int counts[2] = {expr_n_in(eq), expr_n_out(eq)};
    const bool writes[2] = {false, true}, nullable[2] = {false, false};
    const char *const names[2] = {"in", "out"};
    std::vector<Range> rs;
    tl_status s = collect_ranges(rs, tabs, counts, writes, nullable, names, 2, n, sizeof(double), -1);
    if (s == TL_OK)
        s = check_overlaps(rs);
    if (s != TL_OK || n == 0)
        return s;
    const DeviceInfo *d = nullptr;
    if ((s = device_info(&d)) != TL_OK)
        return s;
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (mode == TL_EXPR_FUSED) {
        ExprArgs a;
        for (int q = 0; q < kExprMaxIn; ++q)
            a.in[q] = q < counts[0] ? in[q] : nullptr;
        for (int q = 0; q < kExprMaxOut; ++q)
            a.out[q] = q < counts[1] ? out[q] : nullptr;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)d->sms * 8));
        e = expr_fused(eq, a, n, grid, st);
    } else {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)d->sms * 8));
        e = expr_arrays(eq, in, out, n, grid, st);
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "expression launch");
    return TL_OK;
}

}  // extern "C"
