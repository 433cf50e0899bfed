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

struct Df {
    float hi, lo;
    Df() = default;
    __host__ __device__ __forceinline__ constexpr Df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ __forceinline__ Df(int v) : hi((float)v), lo(0.f) {}
    // exact split of a double (one FP64 subtraction)
    __host__ __device__ __forceinline__ explicit Df(double d)
    {
        hi = (float)d;
        lo = (float)(d - (double)hi);
    }
    __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
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
    return (double)hi + (double)lo;
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
