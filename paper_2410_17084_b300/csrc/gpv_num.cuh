// gpv_num.cuh -- number types of the Voxel-GPR kernels.
//
// The kernels are written once and instantiated for three arithmetic types:
//   float   plain FP32 (the paper's own precision, cuBLAS S-routines in Alg. 3);
//   double  native FP64;
//   ff      "float-float": an unevaluated sum hi + lo of two FP32 numbers carrying
//           about 48 significant bits, built from the error-free transformations
//           TwoSum (Knuth) and FMA-based TwoProduct (Dekker's product with a fused
//           multiply-add), as used by double-float libraries (Dekker 1971; Hida, Li
//           and Bailey 2001).  It runs entirely on the FP32 pipes, which B300 has at
//           many times its FP64 rate.
//
// Why the extra precision is needed: the posterior variance sf2 - k^T (K+s2 I)^-1 k
// sits five orders of magnitude below its two terms when points are dense, and the
// variance moves by about eps * |w|^2 when the kernel entries carry a relative error
// eps (w the kriging weights).  With eps = 2^-24 that alone is 1e-3 relative, so the
// kernel values, the factor and the solves need more than FP32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gpv {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(float h, float l) { ff r; r.hi = h; r.lo = l; return r; }

// s + e == a + b exactly (no magnitude ordering needed)
__device__ __forceinline__ ff two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff_make(s, e);
}
// s + e == a + b exactly when |a| >= |b| or a == 0
__device__ __forceinline__ ff fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return ff_make(s, e);
}
// p + e == a * b exactly (one fused multiply-add recovers the rounding error)
__device__ __forceinline__ ff two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return ff_make(p, e);
}

__device__ __forceinline__ ff operator+(ff a, ff b)
{
    ff s = two_sum(a.hi, b.hi);
    ff t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff operator-(ff a) { return ff_make(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b)
{
    ff p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff operator*(ff a, float b)
{
    ff p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}
// a / b: one Newton correction of the FP32 quotient
__device__ __forceinline__ ff operator/(ff a, ff b)
{
    float q1 = __fdiv_rn(a.hi, b.hi);
    ff r = a - b * q1;
    float q2 = __fdiv_rn(r.hi, b.hi);
    ff q = fast_two_sum(q1, q2);
    r = a - b * q;
    float q3 = __fdiv_rn(r.hi, b.hi);
    return q + ff_make(q3, 0.f);
}
__device__ __forceinline__ bool operator<(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(ff a, ff b) { return b < a; }

// ---- conversions ---------------------------------------------------------
template <class T> __device__ __forceinline__ T from_f(float x);
template <> __device__ __forceinline__ float from_f<float>(float x) { return x; }
template <> __device__ __forceinline__ double from_f<double>(float x) { return (double)x; }
template <> __device__ __forceinline__ ff from_f<ff>(float x) { return ff_make(x, 0.f); }

template <class T> __device__ __forceinline__ T from_d(double x);
template <> __device__ __forceinline__ float from_d<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ double from_d<double>(double x) { return x; }
template <> __device__ __forceinline__ ff from_d<ff>(double x)
{
    float h = __double2float_rn(x);
    return ff_make(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double to_d(float x) { return (double)x; }
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(ff x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(double x) { return __double2float_rn(x); }
__device__ __forceinline__ float to_f(ff x) { return __fadd_rn(x.hi, x.lo); }
__device__ __forceinline__ float hi_of(float x) { return x; }
__device__ __forceinline__ float hi_of(double x) { return (float)x; }
__device__ __forceinline__ float hi_of(ff x) { return x.hi; }

// Exact difference of two FP32 numbers in the working type (the local
// coordinates of a point relative to its voxel centre).
template <class T> __device__ __forceinline__ T diff_f(float a, float b);
template <> __device__ __forceinline__ float diff_f<float>(float a, float b) { return __fsub_rn(a, b); }
template <> __device__ __forceinline__ double diff_f<double>(float a, float b) { return (double)a - (double)b; }
template <> __device__ __forceinline__ ff diff_f<ff>(float a, float b) { return two_sum(a, -b); }

// ---- square root ------------------------------------------------------------
__device__ __forceinline__ float gsqrt(float x) { return __fsqrt_rn(x); }
__device__ __forceinline__ double gsqrt(double x) { return sqrt(x); }
// Newton step on the FP32 root: s + (x - s^2) * (1 / (2 s)), the correction scaled by
// the FP32 reciprocal (its error multiplies a term already 2^-24 small)
__device__ __forceinline__ ff gsqrt(ff x)
{
    if (!(x.hi > 0.f)) return ff_make(x.hi == 0.f ? 0.f : __int_as_float(0x7fc00000), 0.f);
    const float s = __fsqrt_rn(x.hi);
    const ff r = x - two_prod(s, s);
    return fast_two_sum(s, r.hi * (0.5f * __frcp_rn(s)));
}

// 1 / sqrt(x): the FP32 hardware estimate y, one Newton step y + y (1 - x y^2) / 2 with
// x y^2 formed in float-float (the estimate's error, about 2^-22, squares away)
__device__ __forceinline__ float grsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double grsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ ff grsqrt(ff x)
{
    const float y = rsqrtf(x.hi);
    const ff e = ff_make(1.f, 0.f) - (x * y) * y;
    return fast_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), e.hi));
}

// ---- reciprocal ---------------------------------------------------------------------
__device__ __forceinline__ float grcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double grcp(double x) { return 1.0 / x; }
// 1 / x: FP32 reciprocal q of the leading part, one Newton step q (1 + e), e = 1 - x q
// formed exactly in its leading part (1 - p.hi is exact for p.hi near 1)
__device__ __forceinline__ ff grcp(ff x)
{
    const float q = __frcp_rn(x.hi);
    const ff p = two_prod(x.hi, q);
    float e = __fsub_rn(__fsub_rn(1.f, p.hi), p.lo);
    e = __fmaf_rn(-x.lo, q, e);
    return fast_two_sum(q, q * e);
}

// ---- exponential of a non-positive argument -----------------------------------
__device__ __forceinline__ float gexp(float x) { return expf(x); }
__device__ __forceinline__ double gexp(double x) { return exp(x); }

// exp(x) for ff x <= 0: x = k ln2 + r with |r| <= ln2/2, exp(r) by its Taylor
// series in ff arithmetic (13 terms reach 2^-50 for |r| <= 0.35), scaled by 2^k.
// ln 2 is split as LN2_HI (its nearest float) + LN2_LO (the remainder).
__device__ __forceinline__ ff gexp(ff x)
{
    if (x.hi < -87.0f) return ff_make(0.f, 0.f);
    const float LN2_HI = 0.693147182464599609375f;
    const float LN2_LO = -1.9046542121259336e-09f;
    float k = rintf(__fmul_rn(x.hi, 1.4426950216293335f));
    ff kl = two_prod(k, LN2_HI);
    kl.lo = __fmaf_rn(k, LN2_LO, kl.lo);
    ff r = x - fast_two_sum(kl.hi, kl.lo);
    // Horner: sum_{j=0}^{13} r^j / j!, each 1/j! split into nearest float + remainder
    const float inv_fact_hi[14] = {1.f, 1.f, 0.5f, 0.1666666716337204f, 0.0416666679084301f,
                                   0.008333333767950535f, 0.0013888889225199819f,
                                   0.00019841270113829523f, 2.4801587642286904e-05f,
                                   2.7557318844628753e-06f, 2.755731998149713e-07f,
                                   2.5052107943679403e-08f, 2.0876755879584152e-09f,
                                   1.6059044372074283e-10f};
    const float inv_fact_lo[14] = {0.f, 0.f, 0.f, -4.967053879312289e-09f,
                                   -1.2417634698280722e-09f, -4.34617203337595e-10f,
                                   -3.3631094437103215e-11f, -2.725596874933456e-12f,
                                   -3.40699609366682e-13f, 3.793571224297229e-14f,
                                   -7.575112209051195e-15f, 4.4176230446483665e-16f,
                                   1.1082839147459852e-16f, -5.352526511562726e-18f};
    ff p = ff_make(inv_fact_hi[13], inv_fact_lo[13]);
#pragma unroll
    for (int j = 12; j >= 0; --j) p = p * r + ff_make(inv_fact_hi[j], inv_fact_lo[j]);
    int ki = (int)k;
    return ff_make(ldexpf(p.hi, ki), ldexpf(p.lo, ki));
}

// exp(x) for ff x <= 0 with a table tab[m] = 2^(m/256) (float-float, m = 0..255):
// x = (256 k + m) ln2/256 + r with |r| <= ln2/512, so exp(x) = 2^k tab[m] exp(r), and exp(r)
// is its Taylor polynomial of degree 4 (remainder below r^5/120 < 2^-54).  ln2/256 is split
// as L1 + L2 (floats) + 3.4e-19; n L1 and n L2 are formed exactly (TwoProduct), so the
// reduction errs by |n| 3.4e-19, below 5e-17 of the result's scale for every x.
__device__ __forceinline__ ff gexp_tab(ff x, const ff* tab)
{
    if (x.hi < -87.0f) return ff_make(0.f, 0.f);
    const float L1 = 0.0027076061815023422f;
    const float L2 = -7.440055516116928e-12f;
    const float nf = rintf(__fmul_rn(x.hi, 369.3299255371094f));  // 256 / ln 2
    const ff a = two_prod(nf, L1);
    const ff b = two_prod(nf, L2);
    const ff r = (x - a) - b;
    ff p = ff_make(0.0416666679084301f, -1.2417634698280722e-09f);          // 1/24
    p = p * r + ff_make(0.1666666716337204f, -4.967053879312289e-09f);    // 1/6
    p = p * r + ff_make(0.5f, 0.f);
    p = p * r + ff_make(1.f, 0.f);
    p = p * r + ff_make(1.f, 0.f);
    const int n = (int)nf;
    const int k = n >> 8, m = n & 255;  // floor division: n = 256 k + m, 0 <= m < 256
    const ff t = tab[m] * p;
    return ff_make(ldexpf(t.hi, k), ldexpf(t.lo, k));
}

// exp of the working type: float and double by CUDA's own functions, float-float by the
// table form above
__device__ __forceinline__ float gexpw(float x, const ff*) { return expf(x); }
__device__ __forceinline__ double gexpw(double x, const ff*) { return exp(x); }
__device__ __forceinline__ ff gexpw(ff x, const ff* tab) { return gexp_tab(x, tab); }

// ---- fused multiply-add in the working type -----------------------------------
// c + a b for ff: exact leading product (TwoProduct), cross terms in FP32, exact sum of
// the leading parts (TwoSum), one renormalisation.  The error is bounded relative to
// |c| + |a b| (not to the result), the model of an FP64 operation on these operands.
__device__ __forceinline__ float gfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double gfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ ff gfma(ff a, ff b, ff c)
{
    ff p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    ff s = two_sum(c.hi, p.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(c.lo, p.lo));
    return fast_two_sum(s.hi, s.lo);
}
// c - a b
__device__ __forceinline__ float gfnma(float a, float b, float c) { return __fmaf_rn(-a, b, c); }
__device__ __forceinline__ double gfnma(double a, double b, double c) { return __fma_rn(-a, b, c); }
__device__ __forceinline__ ff gfnma(ff a, ff b, ff c) { return gfma(-a, b, c); }

// acc += a b with an unnormalised accumulator: hi carries the running sum of the exact
// leading products, lo collects every rounding error (TwoSum) and cross term.  Twelve
// FP32 operations per step; acc_norm() renormalises once at the end.
__device__ __forceinline__ void acc_fma(float& acc, float a, float b) { acc = __fmaf_rn(a, b, acc); }
__device__ __forceinline__ void acc_fma(double& acc, double a, double b) { acc = __fma_rn(a, b, acc); }
__device__ __forceinline__ void acc_fma(ff& acc, ff a, ff b)
{
    ff p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    ff s = two_sum(acc.hi, p.hi);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, p.lo));
}
__device__ __forceinline__ float acc_norm(float a) { return a; }
__device__ __forceinline__ double acc_norm(double a) { return a; }
__device__ __forceinline__ ff acc_norm(ff a) { return fast_two_sum(a.hi, a.lo); }

template <class T> __device__ __forceinline__ T zero() { return from_f<T>(0.f); }

// Slice exponent of the tensor-core variance: E with m < 2^(E-1) for the largest magnitude
// m of a row (leading parts; the margin covers their rounding), so the first 8-bit slice
// of every entry holds at most 7 bits (|slice| <= 2^7 grid units, like the later ones);
// kept where the slice grids 2^(E-8) .. 2^(E-48) stay normal FP32 numbers.
__device__ __forceinline__ int tc_exp_above(float m)
{
    if (!(m > 0.f)) return -100;
    int e;
    frexpf(m * 1.000001f, &e);
    return max(-100, min(100, e + 1));
}

template <class T> struct is_ff { static constexpr bool value = false; };
template <> struct is_ff<ff> { static constexpr bool value = true; };

}  // namespace gpv
