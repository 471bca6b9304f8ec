// Device interval arithmetic with outward rounding (section 2.1, Eqs. 3-6).
//
// Every lower endpoint is rounded toward -inf and every upper endpoint toward
// +inf with the CUDA directed-rounding intrinsics (__dadd_rd, __dmul_ru,
// __fadd_rd, ...), giving the optimal outward rounding of each elementary
// operation.  Multiplication uses the sign-case table of Eq. 5 (the two
// endpoint products that attain the extremes), which yields the same
// endpoints as the min/max over all four products; the closed-interval
// convention 0 * inf = 0 is honoured on a slow path taken only when an
// operand endpoint is infinite.  Transcendentals are the CUDA library
// functions in round-to-nearest widened by their documented maximum error
// plus one ulp.  No fast-math intrinsic and no flush-to-zero is used.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gb {

struct iv64 { double lo, hi; };
struct iv32 { float lo, hi; };

// CUDA Math API documented maximum ulp errors (non fast-math): exp 1 (FP64),
// sin/cos 2 (FP64); expf 2, sinf/cosf 2 (FP32).  Widening = bound + 1.
constexpr int K_EXP64 = 2, K_TRIG64 = 3, K_EXP32 = 3, K_TRIG32 = 3;

// ---------------------------------------------------------------------------
// ulp stepping on the bit pattern (monotone integer image of the doubles)
__device__ __forceinline__ double step_up(double x, int k) {
    long long b = __double_as_longlong(x);
    if (b == 0x7ff0000000000000LL) return x;                  // +inf
    // signed ordinal of the value: -0 and +0 both map to 0
    long long t = b < 0 ? -(long long)((unsigned long long)b & 0x7fffffffffffffffULL) : b;
    t += k;
    long long r = t < 0 ? (long long)((unsigned long long)(-t) | 0x8000000000000000ULL) : t;
    return __longlong_as_double(r);
}
__device__ __forceinline__ double step_dn(double x, int k) {
    long long b = __double_as_longlong(x);
    if (b == (long long)0xfff0000000000000ULL) return x;      // -inf
    long long t = b < 0 ? -(long long)((unsigned long long)b & 0x7fffffffffffffffULL) : b;
    t -= k;
    long long r = t < 0 ? (long long)((unsigned long long)(-t) | 0x8000000000000000ULL) : t;
    return __longlong_as_double(r);
}
__device__ __forceinline__ float step_up(float x, int k) {
    int b = __float_as_int(x);
    if (b == 0x7f800000) return x;
    int t = b < 0 ? -(b & 0x7fffffff) : b;
    t += k;
    int r = t < 0 ? ((-t) | (int)0x80000000) : t;
    return __int_as_float(r);
}
__device__ __forceinline__ float step_dn(float x, int k) {
    int b = __float_as_int(x);
    if (b == (int)0xff800000) return x;
    int t = b < 0 ? -(b & 0x7fffffff) : b;
    t -= k;
    int r = t < 0 ? ((-t) | (int)0x80000000) : t;
    return __int_as_float(r);
}

// sign bit and "is infinite" tests on the high word (integer pipe)
__device__ __forceinline__ bool sgn(double x) { return __double2hiint(x) < 0; }
__device__ __forceinline__ bool sgn(float x) { return __float_as_int(x) < 0; }
__device__ __forceinline__ unsigned absbits(double x) { return (unsigned)__double2hiint(x) & 0x7fffffffu; }
__device__ __forceinline__ unsigned absbits(float x) { return (unsigned)__float_as_int(x) & 0x7fffffffu; }
// full magnitude ordering key (|x| compares like these integers for non-NaN x)
__device__ __forceinline__ unsigned long long magkey(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ unsigned magkey(float x) { return absbits(x); }
// IEEE comparisons with zero and equality on the integer pipe (the FP64 pipe
// is kept for the directed arithmetic): false for NaN, +0 == -0.
__device__ __forceinline__ bool gt_zero(double x) {
    long long b = __double_as_longlong(x);
    return b > 0 && b <= 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool lt_zero(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return b > 0x8000000000000000ULL && b <= 0xfff0000000000000ULL;
}
__device__ __forceinline__ bool same_value(double x, double y) {
    unsigned long long a = (unsigned long long)__double_as_longlong(x), b = (unsigned long long)__double_as_longlong(y);
    return (a == b && (a & 0x7fffffffffffffffULL) <= 0x7ff0000000000000ULL) || ((a | b) << 1) == 0;
}
__device__ __forceinline__ bool is_one(double x) { return __double_as_longlong(x) == 0x3ff0000000000000LL; }
__device__ __forceinline__ bool gt_zero(float x) {
    int b = __float_as_int(x);
    return b > 0 && b <= 0x7f800000;
}
__device__ __forceinline__ bool lt_zero(float x) {
    unsigned b = (unsigned)__float_as_int(x);
    return b > 0x80000000u && b <= 0xff800000u;
}
__device__ __forceinline__ bool is_one(float x) { return __float_as_int(x) == 0x3f800000; }

__device__ __forceinline__ bool any_inf(double a, double b, double c, double d) {
    unsigned m = max(max(absbits(a), absbits(b)), max(absbits(c), absbits(d)));
    return m >= 0x7ff00000u;
}
__device__ __forceinline__ bool any_inf(float a, float b, float c, float d) {
    unsigned m = max(max(absbits(a), absbits(b)), max(absbits(c), absbits(d)));
    return m >= 0x7f800000u;
}

// ---------------------------------------------------------------------------
// precision-generic directed primitives
__device__ __forceinline__ double add_rd(double a, double b) { return __dadd_rd(a, b); }
__device__ __forceinline__ double add_ru(double a, double b) { return __dadd_ru(a, b); }
__device__ __forceinline__ double sub_rd(double a, double b) { return __dsub_rd(a, b); }
__device__ __forceinline__ double sub_ru(double a, double b) { return __dsub_ru(a, b); }
__device__ __forceinline__ double mul_rd(double a, double b) { return __dmul_rd(a, b); }
__device__ __forceinline__ double mul_ru(double a, double b) { return __dmul_ru(a, b); }
__device__ __forceinline__ double div_rd(double a, double b) { return __ddiv_rd(a, b); }
__device__ __forceinline__ double div_ru(double a, double b) { return __ddiv_ru(a, b); }
__device__ __forceinline__ double rcp_rd(double a) { return __drcp_rd(a); }
__device__ __forceinline__ double rcp_ru(double a) { return __drcp_ru(a); }
__device__ __forceinline__ double sqrt_rd(double a) { return __dsqrt_rd(a); }
__device__ __forceinline__ double sqrt_ru(double a) { return __dsqrt_ru(a); }
__device__ __forceinline__ float add_rd(float a, float b) { return __fadd_rd(a, b); }
__device__ __forceinline__ float add_ru(float a, float b) { return __fadd_ru(a, b); }
__device__ __forceinline__ float sub_rd(float a, float b) { return __fsub_rd(a, b); }
__device__ __forceinline__ float sub_ru(float a, float b) { return __fsub_ru(a, b); }
__device__ __forceinline__ float mul_rd(float a, float b) { return __fmul_rd(a, b); }
__device__ __forceinline__ float mul_ru(float a, float b) { return __fmul_ru(a, b); }
__device__ __forceinline__ float div_rd(float a, float b) { return __fdiv_rd(a, b); }
__device__ __forceinline__ float div_ru(float a, float b) { return __fdiv_ru(a, b); }
__device__ __forceinline__ float rcp_rd(float a) { return __frcp_rd(a); }
__device__ __forceinline__ float rcp_ru(float a) { return __frcp_ru(a); }
__device__ __forceinline__ float sqrt_rd(float a) { return __fsqrt_rd(a); }
__device__ __forceinline__ float sqrt_ru(float a) { return __fsqrt_ru(a); }

template <typename T> struct ivt;
template <> struct ivt<double> { typedef iv64 type; };
template <> struct ivt<float> { typedef iv32 type; };

template <typename T> __device__ __forceinline__ typename ivt<T>::type mk(T lo, T hi) {
    typename ivt<T>::type r;
    r.lo = lo;
    r.hi = hi;
    return r;
}
template <typename T> __device__ __forceinline__ T inf_v() { return (T)__longlong_as_double(0x7ff0000000000000LL); }
template <> __device__ __forceinline__ float inf_v<float>() { return __int_as_float(0x7f800000); }

// Eq. 3
template <typename I> __device__ __forceinline__ I iadd(I x, I y) {
    I r; r.lo = add_rd(x.lo, y.lo); r.hi = add_ru(x.hi, y.hi); return r;
}
// Eq. 4
template <typename I> __device__ __forceinline__ I isub(I x, I y) {
    I r; r.lo = sub_rd(x.lo, y.hi); r.hi = sub_ru(x.hi, y.lo); return r;
}
template <typename I> __device__ __forceinline__ I ineg(I x) {
    I r; r.lo = -x.hi; r.hi = -x.lo; return r;
}

// endpoint product with 0 * inf = 0
template <typename T> __device__ __forceinline__ T pmul_rd(T a, T b) {
    return (a == (T)0 || b == (T)0) ? (T)0 : mul_rd(a, b);
}
template <typename T> __device__ __forceinline__ T pmul_ru(T a, T b) {
    return (a == (T)0 || b == (T)0) ? (T)0 : mul_ru(a, b);
}

// Eq. 5, sign-case form.  P: lo >= +0 (sign bit clear), N: hi has its sign
// bit set, M: otherwise.  -0 endpoints are classified by sign bit; every
// case still selects the products that attain the extremes because a zero
// endpoint contributes a zero product.
template <typename I> __device__ __forceinline__ I imul(I x, I y) {
    typedef decltype(x.lo) T;
    T a = x.lo, b = x.hi, c = y.lo, d = y.hi;
    I r;
    if (__builtin_expect(any_inf(a, b, c, d), 0)) {
        r.lo = fmin(fmin(pmul_rd(a, c), pmul_rd(a, d)), fmin(pmul_rd(b, c), pmul_rd(b, d)));
        r.hi = fmax(fmax(pmul_ru(a, c), pmul_ru(a, d)), fmax(pmul_ru(b, c), pmul_ru(b, d)));
        return r;
    }
    int cx = !sgn(a) ? 0 : (sgn(b) ? 1 : 2);
    int cy = !sgn(c) ? 0 : (sgn(d) ? 1 : 2);
    switch (cx * 3 + cy) {
    case 0: r.lo = mul_rd(a, c); r.hi = mul_ru(b, d); break;  // P P
    case 1: r.lo = mul_rd(b, c); r.hi = mul_ru(a, d); break;  // P N
    case 2: r.lo = mul_rd(b, c); r.hi = mul_ru(b, d); break;  // P M
    case 3: r.lo = mul_rd(a, d); r.hi = mul_ru(b, c); break;  // N P
    case 4: r.lo = mul_rd(b, d); r.hi = mul_ru(a, c); break;  // N N
    case 5: r.lo = mul_rd(a, d); r.hi = mul_ru(a, c); break;  // N M
    case 6: r.lo = mul_rd(a, d); r.hi = mul_ru(b, d); break;  // M P
    case 7: r.lo = mul_rd(b, c); r.hi = mul_ru(a, c); break;  // M N
    default:                                                   // M M
        r.lo = fmin(mul_rd(a, d), mul_rd(b, c));
        r.hi = fmax(mul_ru(a, c), mul_ru(b, d));
        break;
    }
    return r;
}

// Unit step H(y) = 1 for y >= 0, else 0: exact on an interval wholly on one
// side of the jump, [0, 1] on one that holds it.
template <typename I> __device__ __forceinline__ I istep(I x) {
    typedef decltype(x.lo) T;
    I r;
    if (x.lo >= (T)0) r.lo = r.hi = (T)1;
    else if (x.hi < (T)0) r.lo = r.hi = (T)0;
    else r.lo = (T)0, r.hi = (T)1;
    return r;
}

// square without the dependence widening of x*x
template <typename I> __device__ __forceinline__ I isqr(I x) {
    typedef decltype(x.lo) T;
    I r;
    if (!sgn(x.lo)) { r.lo = mul_rd(x.lo, x.lo); r.hi = mul_ru(x.hi, x.hi); return r; }
    if (sgn(x.hi)) { r.lo = mul_rd(x.hi, x.hi); r.hi = mul_ru(x.lo, x.lo); return r; }
    T m = magkey(x.lo) > magkey(x.hi) ? x.lo : x.hi;     // larger magnitude
    r.lo = (T)0;
    r.hi = mul_ru(m, m);
    return r;
}

// multiplication by a point constant c
template <typename I> __device__ __forceinline__ I iscale(I x, decltype(x.lo) c) {
    typedef decltype(x.lo) T;
    I r;
    if (c == (T)0) { r.lo = r.hi = (T)0; return r; }
    if (c > (T)0) { r.lo = mul_rd(x.lo, c); r.hi = mul_ru(x.hi, c); }
    else { r.lo = mul_rd(x.hi, c); r.hi = mul_ru(x.lo, c); }
    return r;
}

// 1/[y] for Eq. 6; the whole line when 0 is in [y]
template <typename I> __device__ __forceinline__ I ircp(I y) {
    typedef decltype(y.lo) T;
    I r;
    if (y.lo > (T)0 || y.hi < (T)0) { r.lo = rcp_rd(y.hi); r.hi = rcp_ru(y.lo); }
    else { r.lo = -inf_v<T>(); r.hi = inf_v<T>(); }
    return r;
}
// Eq. 6
template <typename I> __device__ __forceinline__ I idiv(I x, I y) { return imul(x, ircp(y)); }

template <typename I> __device__ __forceinline__ I isqrt(I x) {
    typedef decltype(x.lo) T;
    I r;
    r.lo = sqrt_rd(fmax(x.lo, (T)0));
    r.hi = sqrt_ru(fmax(x.hi, (T)0));
    return r;
}

__device__ __forceinline__ double lib_exp(double x) { return exp(x); }
__device__ __forceinline__ float lib_exp(float x) { return expf(x); }
__device__ __forceinline__ double lib_cos(double x) { return cos(x); }
__device__ __forceinline__ float lib_cos(float x) { return cosf(x); }
__device__ __forceinline__ double lib_sin(double x) { return sin(x); }
__device__ __forceinline__ float lib_sin(float x) { return sinf(x); }
template <typename T> __device__ __forceinline__ int k_exp() { return sizeof(T) == 8 ? K_EXP64 : K_EXP32; }
template <typename T> __device__ __forceinline__ int k_trig() { return sizeof(T) == 8 ? K_TRIG64 : K_TRIG32; }

// A point interval (lo == hi, the sample points) calls the library once:
// the same value either way, half the dependent FP64 chain.
template <typename I> __device__ __forceinline__ I iexp(I x) {
    typedef decltype(x.lo) T;
    I r;
    const T a = lib_exp(x.lo);
    const T b = x.hi == x.lo ? a : lib_exp(x.hi);
    r.lo = step_dn(a, k_exp<T>());
    r.hi = step_up(b, k_exp<T>());
    if (r.lo < (T)0) r.lo = (T)0;
    return r;
}

// pi enclosed by adjacent doubles: 0x400921FB54442D18 is the double nearest
// to pi and lies below it.  The float bounds are the outward conversions.
__device__ __forceinline__ iv64 pi_iv(double) {
    iv64 r;
    r.lo = __longlong_as_double(0x400921FB54442D18LL);
    r.hi = __longlong_as_double(0x400921FB54442D19LL);
    return r;
}
__device__ __forceinline__ iv32 pi_iv(float) {
    iv32 r;
    r.lo = __int_as_float(0x40490FDA);   // largest float below pi
    r.hi = __int_as_float(0x40490FDB);   // smallest float above pi
    return r;
}
// e: 0x4005BF0A8B145769 is the double nearest to e and lies below it.
__device__ __forceinline__ iv64 e_iv(double) {
    iv64 r;
    r.lo = __longlong_as_double(0x4005BF0A8B145769LL);
    r.hi = __longlong_as_double(0x4005BF0A8B14576ALL);
    return r;
}
__device__ __forceinline__ iv32 e_iv(float) {
    iv32 r;
    r.lo = __int_as_float(0x402DF854);
    r.hi = __int_as_float(0x402DF855);
    return r;
}

// Interval cos (is_cos) or sin: endpoint values widened, extremum +-1 added
// when an outward enclosure of x/pi (minus 1/2 for sin) contains an integer
// of the right parity; widths >= 2*pi_lo or |x| beyond 2^40 (2^20 in FP32)
// give [-1, 1].
template <typename I> __device__ __forceinline__ I itrig(I x, bool is_cos) {
    typedef decltype(x.lo) T;
    I pi = pi_iv(x.lo);
    const T big = sizeof(T) == 8 ? (T)1099511627776.0 : (T)1048576.0;
    T w = sub_ru(x.hi, x.lo);
    I r;
    r.lo = (T)-1;
    r.hi = (T)1;
    if (!(w < pi.lo * (T)2) || !(fabs(x.lo) <= big) || !(fabs(x.hi) <= big)) return r;
    const T va = is_cos ? lib_cos(x.lo) : lib_sin(x.lo);
    const T vb = x.hi == x.lo ? va : (is_cos ? lib_cos(x.hi) : lib_sin(x.hi));
    int k = k_trig<T>();
    T lo = fmin(step_dn(va, k), step_dn(vb, k));
    T hi = fmax(step_up(va, k), step_up(vb, k));
    T qlo = div_rd(x.lo, x.lo >= (T)0 ? pi.hi : pi.lo);
    T qhi = div_ru(x.hi, x.hi >= (T)0 ? pi.lo : pi.hi);
    if (!is_cos) {
        qlo = sub_rd(qlo, (T)0.5);
        qhi = sub_ru(qhi, (T)0.5);
    }
    T k0 = ceil(qlo), k1 = floor(qhi);
    if (k0 <= k1) {
        long long i0 = (long long)k0;
        bool two = k0 + (T)1 <= k1;
        bool even0 = (i0 & 1LL) == 0;
        if (even0 || two) hi = (T)1;
        if (!even0 || two) lo = (T)-1;
    }
    r.lo = fmax(lo, (T)-1);
    r.hi = fmin(hi, (T)1);
    return r;
}

// Two-lane forms of iexp and itrig for lanes 0 and 1 of a warp that hold the
// same argument (both run the same interpreter; the table kernel does): lane
// h evaluates the library function at endpoint h, and for itrig the
// directed division of endpoint h by pi, and the two lanes exchange them --
// the values of iexp / itrig, with the two endpoint evaluations side by side
// instead of one after the other.  RU(a / b) is taken as -RD(-a / b), the
// same number under IEEE directed rounding.
template <typename T> __device__ __forceinline__ T pair_get(T v, int src) { return __shfl_sync(0x3u, v, src); }

template <typename I> __device__ __forceinline__ I iexp_pair(I x) {
    typedef decltype(x.lo) T;
    const int h = threadIdx.x & 1;
    const T v = lib_exp(h ? x.hi : x.lo);
    const T a = pair_get(v, 0), vb = pair_get(v, 1);
    const T b = x.hi == x.lo ? a : vb;
    I r;
    r.lo = step_dn(a, k_exp<T>());
    r.hi = step_up(b, k_exp<T>());
    if (r.lo < (T)0) r.lo = (T)0;
    return r;
}

template <typename I> __device__ __forceinline__ I itrig_pair(I x, bool is_cos) {
    typedef decltype(x.lo) T;
    const int h = threadIdx.x & 1;
    I pi = pi_iv(x.lo);
    const T big = sizeof(T) == 8 ? (T)1099511627776.0 : (T)1048576.0;
    T w = sub_ru(x.hi, x.lo);
    I r;
    r.lo = (T)-1;
    r.hi = (T)1;
    if (!(w < pi.lo * (T)2) || !(fabs(x.lo) <= big) || !(fabs(x.hi) <= big)) return r;
    const T e = h ? x.hi : x.lo;
    const T v = is_cos ? lib_cos(e) : lib_sin(e);
    const T num = h ? -x.hi : x.lo;
    const T den = h ? (x.hi >= (T)0 ? pi.lo : pi.hi) : (x.lo >= (T)0 ? pi.hi : pi.lo);
    const T q = div_rd(num, den);
    const T va = pair_get(v, 0), v1 = pair_get(v, 1);
    const T vb = x.hi == x.lo ? va : v1;
    int k = k_trig<T>();
    T lo = fmin(step_dn(va, k), step_dn(vb, k));
    T hi = fmax(step_up(va, k), step_up(vb, k));
    T qlo = pair_get(q, 0), qhi = -pair_get(q, 1);
    if (!is_cos) {
        qlo = sub_rd(qlo, (T)0.5);
        qhi = sub_ru(qhi, (T)0.5);
    }
    T k0 = ceil(qlo), k1 = floor(qhi);
    if (k0 <= k1) {
        long long i0 = (long long)k0;
        bool two = k0 + (T)1 <= k1;
        bool even0 = (i0 & 1LL) == 0;
        if (even0 || two) hi = (T)1;
        if (!even0 || two) lo = (T)-1;
    }
    r.lo = fmax(lo, (T)-1);
    r.hi = fmin(hi, (T)1);
    return r;
}

}  // namespace gb
