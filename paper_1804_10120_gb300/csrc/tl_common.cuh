// tl_common.cuh -- layout constants, argument blocks and small exact helpers shared by the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tl {

// Offsets into the 43-entry input table and the 39-entry output table (see include/tl.h).
enum : int { IN_G = 0, IN_DG = 6, IN_K = 24, IN_ALPHA = 30, IN_BETA = 31, IN_DBETA = 34, N_IN = 43 };
enum : int { OUT_GINV = 0, OUT_GAMMA = 6, OUT_DBCOV = 24, OUT_DTG = 33, N_OUT = 39 };

// Packed position of the unordered index pair {i, j}: (00,01,02,11,12,22) -> 0..5.
__host__ __device__ constexpr int sym(int i, int j)
{
    return (i <= j) ? (i * (5 - i)) / 2 + j : (j * (5 - j)) / 2 + i;
}

// Kernel argument blocks: the component pointer tables travel by value in the parameter space
// (82 pointers = 656 bytes), so a launch needs no device-side table.
template <typename T> struct FwdArgs {
    const T *in[N_IN];
    T *out[N_OUT];
};
template <typename T> struct BwdArgs {
    const T *in[N_IN];
    const T *gout[N_OUT];   // nullptr = output absent from the functional
    T *gin[N_IN];
};
// Forward and adjoint in one pass (164 pointers = 1312 bytes of parameters).
template <typename T> struct FwdBwdArgs {
    const T *in[N_IN];
    T *out[N_OUT];
    const T *gout[N_OUT];   // nullptr = output absent from the functional
    T *gin[N_IN];
};

// Streaming loads and stores: each element is touched exactly once, so keep it out of L1 and mark it
// evict-first in L2.
template <typename T> __device__ __forceinline__ T ld_stream(const T *p) { return __ldcs(p); }
template <typename T> __device__ __forceinline__ void st_stream(T *p, T v) { __stcs(p, v); }

// ---- exact power-of-two scaling of binary64 on the integer pipe (the FP64 pipe is the scarce one) ----
// half_exact(x) == x * 0.5 and twice_exact(x) == x * 2.0 in IEEE round-to-nearest-even for every
// binary64 value, including zeros, subnormals, infinities and NaN.
static __device__ __noinline__ double half_slow(double x) { return x * 0.5; }
static __device__ __noinline__ double twice_slow(double x) { return x + x; }

// The exponent field is adjusted with an inline-asm integer add on the high word, so that the compiler
// cannot turn the bit manipulation back into an FP64 instruction; zeros are handled inline, other
// operands without a normal result (subnormals, the smallest / largest normals, inf, nan) out of line.
__device__ __forceinline__ double half_exact(double x)
{
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
    if (e - 2u < 2045u) {
        int r;
        asm("add.s32 %0, %1, -1048576;" : "=r"(r) : "r"(hi));
        return __hiloint2double(r, lo);
    }
    if (((hi & 0x7fffffff) | lo) == 0)
        return x;
    return half_slow(x);
}

__device__ __forceinline__ double twice_exact(double x)
{
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
    if (e - 1u < 2045u) {
        int r;
        asm("add.s32 %0, %1, 1048576;" : "=r"(r) : "r"(hi));
        return __hiloint2double(r, lo);
    }
    if (((hi & 0x7fffffff) | lo) == 0)
        return x;
    return twice_slow(x);
}

// Out-of-line IEEE quotient for the rare operands outside the binary32 exponent range, kept out of the
// hot path so that the compiler cannot predicate the division sequence into every point.
static __device__ __noinline__ double rcp_f64_slow(double d) { return 1.0 / d; }

// ---- exact binary32 <-> binary64 conversions on the integer pipe ------------------------------------
// F2F conversions issue on the FP64 pipe, which runs at 1/64 of the FP32 rate on this part, so the hot
// paths re-pack the bits instead.  Zeros are handled inline; other operands outside the normal range
// (subnormals, inf, nan, binary32 overflow or underflow) set `rare`, and the caller then evaluates the
// whole point through an out-of-line path that uses the compiler's conversions.

// Exact widening.
__device__ __forceinline__ double f32_to_f64(float f, uint32_t &rare)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t mag = b & 0x7fffffffu;
    rare |= (mag != 0u && mag - 0x00800000u >= 0x7f000000u) ? 1u : 0u;
    const uint32_t hw = (mag == 0u) ? (b & 0x80000000u) : ((b & 0x80000000u) | ((mag >> 3) + (896u << 20)));
    return __hiloint2double((int)hw, (int)(b << 29));
}

// Round-to-nearest-even narrowing.
__device__ __forceinline__ float f64_to_f32(double d, uint32_t &rare)
{
    const uint32_t hw = (uint32_t)__double2hiint(d), lw = (uint32_t)__double2loint(d);
    const uint32_t E = (hw >> 20) & 0x7ffu;
    const bool zero = ((hw & 0x7fffffffu) | lw) == 0u;
    rare |= (!zero && E - 897u >= 254u) ? 1u : 0u;
    const uint32_t t = __funnelshift_l(lw, hw, 3);                    // exponent low bits | 23 fraction bits
    const uint32_t rb = (lw >> 28) & 1u, sticky = lw & 0x0fffffffu;   // round bit, bits below it
    const uint32_t inc = rb & ((sticky != 0u) | (t & 1u));
    const uint32_t r = ((t - 0xC0000000u) & 0x7fffffffu) + inc;       // a carry rounds into the exponent
    return __uint_as_float((zero ? 0u : r) | (hw & 0x80000000u));
}

// -x by flipping the sign bit on the integer pipe (for operands that would otherwise cost an FP64
// instruction to negate).
__device__ __forceinline__ double neg_exact(double x)
{
    return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}

// ---- IEEE binary64 multiplication on the integer pipes --------------------------------------------------
// The FP64 pipe is the binding unit of the binary64 kernels while the integer pipes are nearly idle, so
// some products are formed from the operands' bits: the 106-bit product of the two 53-bit significands
// (two 64-bit integer multiplies), normalised by at most one bit and rounded to nearest-even from the
// bits below the 53 kept -- the definition of the IEEE 754 product, so the result equals a * b bit for
// bit.  Normal operands with a normal result take this path; a zero operand times a finite one gives
// the signed zero; every other case (subnormal, inf, nan, a result near overflow or underflow) calls
// a * b out of line, so no predicated FP64 multiply is left in the common path.
static __device__ __noinline__ double mul_slow(double a, double b) { return a * b; }

__device__ __forceinline__ double mul_int(double a, double b)
{
    const uint64_t ua = (uint64_t)__double_as_longlong(a), ub = (uint64_t)__double_as_longlong(b);
    const uint32_t ea = (uint32_t)(ua >> 52) & 0x7ffu, eb = (uint32_t)(ub >> 52) & 0x7ffu;
    const int e = (int)(ea + eb) - 1023;   // biased exponent of the product, before the normalising shift
    const uint64_t sign = (ua ^ ub) & 0x8000000000000000ull;
    if (ea - 1u < 2046u && eb - 1u < 2046u && (uint32_t)(e - 1) < 2044u) {
        const uint64_t ma = (ua & 0x000fffffffffffffull) | 0x0010000000000000ull;
        const uint64_t mb = (ub & 0x000fffffffffffffull) | 0x0010000000000000ull;
        const uint64_t lo = ma * mb, hi = __umul64hi(ma, mb);    // product in [2^104, 2^106)
        const uint32_t t = (uint32_t)(hi >> 41);                  // 1 when the product is >= 2^105
        // normalise to [2^105, 2^106): one bit left unless it is there already
        const uint64_t h = t ? hi : (hi << 1) | (lo >> 63), l = t ? lo : lo << 1;
        uint64_t m = (h << 11) | (l >> 53);                       // the 53 kept bits
        const uint64_t rem = l & 0x001fffffffffffffull;           // the 53 discarded bits
        m += (rem + (m & 1ull) > 0x0010000000000000ull) ? 1ull : 0ull;   // nearest, ties to even
        // m in [2^52, 2^53]: its leading bit adds one to the exponent field, a rounding carry one more
        return __longlong_as_double((long long)(sign | (((uint64_t)(e + (int)t - 1) << 52) + m)));
    }
    if (((ua << 1) == 0ull && eb != 0x7ffu) || ((ub << 1) == 0ull && ea != 0x7ffu))
        return __longlong_as_double((long long)sign);
    return mul_slow(a, b);
}

// ---- binary64 reciprocal ------------------------------------------------------------------------------
// Seed: binary32 reciprocal (MUFU) of the binary32 truncation of d, both conversions done on integer
// bits; relative seed error |e0| < 2^-21.  Then one third-order step in binary64: with e = 1 - d r,
// 1/d = r / (1 - e) = r (1 + e + e^2 + e^3 + ...), and the series truncated after e^2,
//   r' = r + r (e + e^2),
// leaves a relative error of about e0^3 < 2^-63 (the functional-iteration view of division: M. J. Flynn,
// "On division by functional iteration", IEEE Trans. Computers C-19, 1970).  e is exact up to one
// rounding (fused multiply-add), so r' is r (1 + e + e^2) plus the final rounding: within one ulp of 1/d
// (tests/test_gpu_f64_int.py checks it against the host's IEEE quotient).  Three FP64 operations
// instead of the division sequence.  Outside the binary32 exponent window, d in [2^-124, 2^125) in
// magnitude (and for zero, subnormals, inf, nan), the IEEE quotient 1.0 / d is used.
__device__ __forceinline__ double rcp_f64(double d)
{
    const uint64_t b = (uint64_t)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e > 1023 - 125 && e < 1023 + 125) {
        const uint32_t fb = (uint32_t)((b >> 32) & 0x80000000u) | (uint32_t)((e - 1023 + 127) << 23) |
                            (uint32_t)((b >> 29) & 0x7fffffu);
        float rf;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__uint_as_float(fb)));
        const uint32_t rb = __float_as_uint(rf);
        const uint64_t r64 = ((uint64_t)(rb & 0x80000000u) << 32) |
                             ((uint64_t)(((rb >> 23) & 0xff) - 127 + 1023) << 52) |
                             ((uint64_t)(rb & 0x7fffffu) << 29);
        const double r = __longlong_as_double((long long)r64);
        const double err = fma(-d, r, 1.0);
        return fma(r, fma(err, err, err), r);
    }
    return rcp_f64_slow(d);
}

// Grid-stride bounds for a 1-D launch.
struct GridStride {
    int64_t first, step;
    __device__ __forceinline__ GridStride()
        : first((int64_t)blockIdx.x * blockDim.x + threadIdx.x), step((int64_t)gridDim.x * blockDim.x) {}
};

}  // namespace tl
