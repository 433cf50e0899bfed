// df64.cuh -- float-float ("double-single") arithmetic for FP64-accurate
// work on the FP32 pipes.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so the
// mixed-precision solver recomputes its reliable-update residual b - A x with
// each real held as an unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2,
// about 48 significant bits).  The operations are the classical error-free
// transformations: Knuth's two-sum, Dekker's fast two-sum and the FMA-based
// exact product (a*b = p + e with p = fl(a*b), e = fma(a, b, -p)).  Sums use
// the cheap variant that adds the low parts in FP32, whose error is a few
// units of 2^-48 of the operands.
#pragma once

#include "lqcd_internal.cuh"

namespace lqcd {

// internal storage precision: float-float pairs (not part of the C ABI)
constexpr lqcd_prec PREC_DF = (lqcd_prec)4;

// Conversions between doubles and float pairs on the integer bits of the
// IEEE-754 formats.  The direct routes -- hi = RN(d), lo = RN(d - hi): two
// conversions, one subtraction and one more conversion on the FP64 pipe;
// (double) hi + (double) lo: two conversions and one addition -- bound every
// kernel that converts whole fields on a part whose FP64 rate is a small
// fraction of its FP32 rate.  These give the same bits with at most the one
// FP64 addition.
//
// Split, for d = (-1)^s 2^E (1 + f / 2^52) with -74 <= E <= 126 (so that hi
// and every nonzero lo are normal floats):
//   hi keeps the leading 23 of the 52 fraction bits, rounded to nearest-even
//   on the 29 dropped bits t: away from zero iff t > 2^28, or t = 2^28 and
//   the last kept bit is 1.  The rounding increment is added to the pattern
//   (E + 127) << 23 | f23, so a carry out of the fraction raises the exponent
//   as RN(d) requires.
//   d - hi is exact: t units of 2^(E-52) with the sign of d, or, when hi went
//   away from zero, 2^29 - t units with the opposite sign.  The integer (< 2^29)
//   is rounded to 24 bits by the unsigned -> float conversion and scaled by
//   the normal float 2^(E-52) exactly; d = hi gives lo = +0 as d - hi does.
// Zero, subnormal, very small or very large d, Inf and NaN take the direct
// route.
__device__ __forceinline__ void df_split_bits(double d, float &hi, float &lo)
{
    const unsigned long long D = (unsigned long long)__double_as_longlong(d);
    const int E = (int)((D >> 52) & 0x7ffu) - 1023;
    if (E < -74 || E > 126) {
        hi = __double2float_rn(d);
        lo = __double2float_rn(d - (double)hi);
        return;
    }
    const unsigned int sign = (unsigned int)(D >> 32) & 0x80000000u;
    const unsigned int t = (unsigned int)D & 0x1fffffffu;
    const unsigned int f23 = (unsigned int)(D >> 29) & 0x7fffffu;
    const unsigned int away = (t > 0x10000000u) | ((t == 0x10000000u) & f23);
    hi = __uint_as_float(sign | ((((unsigned int)(E + 127) << 23) | f23) + (away & 1u)));
    const unsigned int m = (away & 1u) ? 0x20000000u - t : t;
    const float mag = __uint2float_rn(m) * __uint_as_float((unsigned int)(E + 75) << 23);
    const unsigned int lsign = m == 0u ? 0u : (away & 1u) ? sign ^ 0x80000000u : sign;
    lo = __uint_as_float(__float_as_uint(mag) ^ lsign);
}

// a normal float widened to a double on its bits: exponent rebased by
// 1023 - 127 = 896, fraction moved up by 52 - 23 = 29 bits (exact)
__device__ __forceinline__ double df_widen_normal(unsigned int x)
{
    return __longlong_as_double((long long)((((unsigned long long)(x & 0x7fffffffu) << 29) + (896ull << 52)) |
                                            ((unsigned long long)(x & 0x80000000u) << 32)));
}

// (double) hi + (double) lo: both widened exactly, then the one rounding
// FP64 addition (none when lo is zero); zero, subnormal, Inf or NaN parts
// take the direct route
__device__ __forceinline__ double df_sum_bits(float hi, float lo)
{
    const unsigned int H = __float_as_uint(hi), L = __float_as_uint(lo);
    const unsigned int eh = (H >> 23) & 0xffu, el = (L >> 23) & 0xffu;
    const bool lo_zero = (L & 0x7fffffffu) == 0u;
    if (eh == 0u || eh == 0xffu || el == 0xffu || (el == 0u && !lo_zero)) return (double)hi + (double)lo;
    const double dh = df_widen_normal(H);
    return lo_zero ? dh : dh + df_widen_normal(L);
}

struct Df {
    float hi, lo;
    Df() = default;
    __host__ __device__ __forceinline__ constexpr Df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ __forceinline__ Df(int v) : hi((float)v), lo(0.f) {}
    // exact split of a double: hi = RN(d), lo = RN(d - hi)
    __host__ __device__ __forceinline__ explicit Df(double d)
    {
#ifdef __CUDA_ARCH__
        df_split_bits(d, hi, lo);
#else
        hi = (float)d;
        lo = (float)(d - (double)hi);
#endif
    }
    __device__ __forceinline__ explicit operator double() const { return df_sum_bits(hi, lo); }
    __device__ __forceinline__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ Df df_fast_two_sum(float a, float b) // needs |a| >= |b|
{
    float s = a + b;
    float e = b - (s - a);
    return Df(s, e);
}

__device__ __forceinline__ Df operator+(Df a, Df b)
{
    float s = a.hi + b.hi;
    float v = s - a.hi;
    float e = (a.hi - (s - v)) + (b.hi - v); // two-sum error of the high parts
    e += a.lo + b.lo;
    return df_fast_two_sum(s, e);
}

__device__ __forceinline__ Df operator-(Df a) { return Df(-a.hi, -a.lo); }

// a + b with the same error as operator+, left unnormalised (the pair is
// only ever an operand of the exact products below)
__device__ __forceinline__ Df df_add_raw(Df a, Df b)
{
    float s = a.hi + b.hi;
    float v = s - a.hi;
    float e = (a.hi - (s - v)) + (b.hi - v);
    return Df(s, e + (a.lo + b.lo));
}

__device__ __forceinline__ Df operator-(Df a, Df b) { return a + (-b); }

__device__ __forceinline__ Df operator*(Df a, Df b)
{
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p); // exact error of the high product
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ Df &operator+=(Df &a, Df b)
{
    a = a + b;
    return a;
}

// Accumulator of a sum of float-float products: the leading products are
// added exactly (two-sum into s), all error terms and cross products are
// summed in FP32 into c, and the pair is normalised once at the end.
struct DfAcc {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add_prod(Df a, Df b)
    {
        float p = a.hi * b.hi;
        float e = fmaf(a.hi, b.hi, -p);
        e = fmaf(a.hi, b.lo, e);
        e = fmaf(a.lo, b.hi, e);
        float t = s + p;
        float v = t - s;
        c += ((s - (t - v)) + (p - v)) + e;
        s = t;
    }
    __device__ __forceinline__ void sub_prod(Df a, Df b) { add_prod(Df(-a.hi, -a.lo), b); }
    // the first product of a sum: nothing to add it to, so no two-sum
    __device__ __forceinline__ void set_prod(Df a, Df b)
    {
        s = a.hi * b.hi;
        float e = fmaf(a.hi, b.hi, -s);
        e = fmaf(a.hi, b.lo, e);
        c = fmaf(a.lo, b.hi, e);
    }
    __device__ __forceinline__ void set_neg_prod(Df a, Df b) { set_prod(Df(-a.hi, -a.lo), b); }
    __device__ __forceinline__ void set(Df a)
    {
        s = a.hi;
        c = a.lo;
    }
    __device__ __forceinline__ void add(Df a)
    {
        float t = s + a.hi;
        float v = t - s;
        c += ((s - (t - v)) + (a.hi - v)) + a.lo;
        s = t;
    }
    __device__ __forceinline__ Df value() const { return df_fast_two_sum_any(s, c); }
    // the pair as it stands, not normalised: exact to the bits of c, and a
    // valid operand of add, add_prod and set_prod, which never assume |c| <
    // ulp(s)
    __device__ __forceinline__ Df raw() const { return Df(s, c); }
    // |s| >= |c| holds unless the sum cancelled; normalise with a full two-sum
    __device__ __forceinline__ static Df df_fast_two_sum_any(float a, float b)
    {
        float t = a + b;
        float v = t - a;
        float e = (a - (t - v)) + (b - v);
        return Df(t, e);
    }
};

// conversions used by the generic storage accessors
template <typename R>
__device__ __forceinline__ R df_to(float hi, float lo);
template <>
__device__ __forceinline__ float df_to<float>(float hi, float lo)
{
    return hi + lo;
}
template <>
__device__ __forceinline__ double df_to<double>(float hi, float lo)
{
    return df_sum_bits(hi, lo);
}
template <>
__device__ __forceinline__ Df df_to<Df>(float hi, float lo)
{
    return Df(hi, lo);
}

template <typename R>
__device__ __forceinline__ float4 df_from(const Cx<R> &z);
template <>
__device__ __forceinline__ float4 df_from<Df>(const Cx<Df> &z)
{
    return make_float4(z.re.hi, z.re.lo, z.im.hi, z.im.lo);
}
template <>
__device__ __forceinline__ float4 df_from<double>(const Cx<double> &z)
{
    Df a(z.re), b(z.im);
    return make_float4(a.hi, a.lo, b.hi, b.lo);
}
template <>
__device__ __forceinline__ float4 df_from<float>(const Cx<float> &z)
{
    return make_float4(z.re, 0.f, z.im, 0.f);
}

// spinor: float4 (re.hi, re.lo, im.hi, im.lo) [spin*3+colour][Vh]
template <>
struct SpinorRef<PREC_DF> {
    float4 *d;
    int Vh;
    template <typename R>
    __device__ __forceinline__ Sp<R> load(int cb) const
    {
        Sp<R> s;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            float4 v = ldg(d + (size_t)k * Vh + cb);
            s.c[k / 3][k % 3] = Cx<R>{df_to<R>(v.x, v.y), df_to<R>(v.z, v.w)};
        }
        return s;
    }
    template <typename R>
    __device__ __forceinline__ Sp<R> load_rw(int cb) const
    {
        Sp<R> s;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            float4 v = d[(size_t)k * Vh + cb];
            s.c[k / 3][k % 3] = Cx<R>{df_to<R>(v.x, v.y), df_to<R>(v.z, v.w)};
        }
        return s;
    }
    template <typename R>
    __device__ __forceinline__ Sp<R> load_scaled(int cb, R &scale) const
    {
        scale = R(1);
        return load<R>(cb);
    }
    static constexpr bool has_norm = false;
    template <typename R>
    __device__ __forceinline__ void store(int cb, const Sp<R> &s) const
    {
#pragma unroll
        for (int k = 0; k < 12; k++) d[(size_t)k * Vh + cb] = df_from<R>(s.c[k / 3][k % 3]);
    }
};

// gauge: float4 per complex entry [mu][par][row*3+col][Vh]
template <>
struct GaugeRef<PREC_DF> {
    float4 *d;
    int Vh;
    __device__ __forceinline__ size_t idx(int mu, int par, int k, int cb) const
    {
        return ((size_t)((mu * 2 + par) * 9 + k)) * Vh + cb;
    }
    template <typename R>
    __device__ __forceinline__ M3<R> load(int mu, int par, int cb) const
    {
        M3<R> u;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            float4 v = ldg(d + idx(mu, par, k, cb));
            u.e[k / 3][k % 3] = Cx<R>{df_to<R>(v.x, v.y), df_to<R>(v.z, v.w)};
        }
        return u;
    }
    __device__ __forceinline__ void store(int mu, int par, int cb, const M3<double> &u) const
    {
#pragma unroll
        for (int k = 0; k < 9; k++) d[idx(mu, par, k, cb)] = df_from<double>(u.e[k / 3][k % 3]);
    }
};

template <>
__host__ inline SpinorRef<PREC_DF> spinor_ref<PREC_DF>(const lqcd_field *f, int)
{
    return {reinterpret_cast<float4 *>(f->data), f->Vh};
}

} // namespace lqcd
