// lqcd_internal.cuh -- types and device helpers shared by the library's
// translation units: complex / SU(3) / spinor values in registers, the
// site-coalesced structure-of-arrays field accessors for every storage
// precision, lattice geometry, deterministic block reductions, errors and the
// allocator hook.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <type_traits>
#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "lqcd.h"

// ------------------------------------------------------------------ fields

struct lqcd_field {
    lqcd_lattice lat;
    lqcd_kind kind;
    lqcd_prec prec;
    int recon;
    int Vh;            // sites per parity
    void *data;        // main array
    float *norm;       // FP16N spinors: per-site norm
    size_t bytes;      // bytes of data
    size_t norm_bytes; // bytes of norm
    lqcd_alloc_fn alloc;
    lqcd_free_fn free_fn;
    void *alloc_ctx;
};

namespace lqcd {

// ------------------------------------------------------------------ errors

void set_error(const char *fmt, ...);
lqcd_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define LQCD_CUDA(call)                                                                                    \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) return ::lqcd::cuda_fail(e_, #call, __FILE__, __LINE__);                   \
    } while (0)

#define LQCD_TRY(call)                                                                                     \
    do {                                                                                                   \
        lqcd_status s_ = (call);                                                                           \
        if (s_ != LQCD_OK) return s_;                                                                      \
    } while (0)

#define LQCD_REQUIRE(cond, ...)                                                                            \
    do {                                                                                                   \
        if (!(cond)) {                                                                                     \
            ::lqcd::set_error(__VA_ARGS__);                                                                \
            return LQCD_EINVAL;                                                                            \
        }                                                                                                  \
    } while (0)

// every kernel launch goes through this: counts it and checks the launch
extern std::atomic<uint64_t> g_launches;
#define LQCD_LAUNCHED()                                                                                    \
    do {                                                                                                   \
        ::lqcd::g_launches.fetch_add(1, std::memory_order_relaxed);                                        \
        LQCD_CUDA(cudaGetLastError());                                                                     \
    } while (0)

// optional per-class kernel timing with CUDA events on the launching stream
enum KernelClass {
    K_DSLASH_F64 = 0,
    K_DSLASH_F32,
    K_DSLASH_F16N,
    K_DSLASH_BF16,
    K_DSLASH_DF64, // float-float arithmetic (internal storage precision)
    K_GAUGE_FORCE,
    K_FERMION_FORCE,
    K_LINK_UPDATE,
    K_DSLASH_F16N_PLAIN, // the plain FP16+norm hops alone (also counted in K_DSLASH_F16N)
    K_NCLASS
};
struct KernelTimer { // RAII: events around the launches made while it lives
    int cls;
    cudaStream_t s;
    double bytes; // algorithmic bytes the timed launches move (0: not counted)
    cudaEvent_t a = nullptr, b = nullptr;
    KernelTimer(int cls, cudaStream_t s, double bytes = 0.0);
    ~KernelTimer();
};
inline int dslash_class(lqcd_prec p) { return K_DSLASH_F64 + (int)p; }

// algorithmic bytes of one half spinor site / one link in a storage precision
// (each field element counted once; 12-real links for the low precisions)
inline double spinor_site_bytes(lqcd_prec p)
{
    switch ((int)p) {
    case LQCD_F32: return 96;
    case LQCD_F16N: return 52; // 48 + 4-byte norm
    case LQCD_BF16: return 48;
    default: return 192; // F64, float-float
    }
}
inline double link_bytes(lqcd_prec p)
{
    switch ((int)p) {
    case LQCD_F32: return 48;
    case LQCD_F16N:
    case LQCD_BF16: return 24;
    default: return 144;
    }
}

// ------------------------------------------------------------------ memory

// Allocation through the hook set by lqcd_set_allocator (cudaMalloc default).
struct Allocator {
    lqcd_alloc_fn alloc;
    lqcd_free_fn free_fn;
    void *ctx;
};
Allocator current_allocator();
void *dev_alloc(const Allocator &a, size_t bytes, cudaStream_t s);
void dev_free(const Allocator &a, void *p, cudaStream_t s);

// Device buffer owned by the library for the duration of a call or a state.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    Allocator a{};
    cudaStream_t s = nullptr;
    lqcd_status alloc(size_t n, cudaStream_t st);
    void release();
    ~DevBuf() { release(); }
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
};

// Scoped field (freed on scope exit).
struct FieldPtr {
    lqcd_field *f = nullptr;
    ~FieldPtr() {
        if (f) lqcd_field_free(f);
    }
    FieldPtr() = default;
    FieldPtr(const FieldPtr &) = delete;
    FieldPtr &operator=(const FieldPtr &) = delete;
};

// ------------------------------------------------------------------ geometry

// Division by an invariant divisor d (Granlund-Montgomery): with l = ceil(log2 d)
// and m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(m, n) + n) >> l for
// every n < 2^31 (the sum cannot overflow 32 bits there).
struct FastDiv {
    uint32_t d, m, l;
};
inline FastDiv make_fastdiv(uint32_t d)
{
    uint32_t l = 0;
    while ((1ull << l) < d) l++;
    uint64_t m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
    return FastDiv{d, (uint32_t)m, l};
}
__device__ __forceinline__ int fdiv(int n, const FastDiv &f)
{
    return (int)((__umulhi((uint32_t)n, f.m) + (uint32_t)n) >> f.l);
}

struct Geo {
    int L[4];
    int Lxh; // Lx / 2
    int Vh;
    int t_bc; // +1 / -1
    int aniso;  // the actions are anisotropic (xi0 != 1 or cs != 1)
    double xi0; // gauge: planes with t weigh xi0, spatial planes 1 / xi0
    double cs;  // fermion: weight nu / xi0 of the spatial hops
    float csf, cs_lo; // cs rounded to FP32, and cs - csf (its float-float low part)
    int sY, sZ, sT; // checkerboard strides of y, z, t
    FastDiv dLxh, dLy, dLz;
};

lqcd_status check_lattice(const lqcd_lattice *lat);
Geo make_geo(const lqcd_lattice &lat);
bool same_lattice(const lqcd_lattice &a, const lqcd_lattice &b);

// coordinates of checkerboard site cb of parity par
__device__ __forceinline__ void cb_coords(const Geo &g, int cb, int par, int c[4])
{
    int r = fdiv(cb, g.dLxh);
    int xh = cb - r * g.Lxh;
    int r2 = fdiv(r, g.dLy);
    c[1] = r - r2 * g.L[1];
    c[3] = fdiv(r2, g.dLz);
    c[2] = r2 - c[3] * g.L[2];
    c[0] = 2 * xh + ((c[1] + c[2] + c[3] + par) & 1);
}

// checkerboard indices of the 8 neighbours of (cb, coordinates c) and the
// wrap flags of the t hops: nb[2*mu] forward, nb[2*mu+1] backward
__device__ __forceinline__ void cb_neighbours(const Geo &g, int cb, const int c[4], int nb[8], bool &twrap_f,
                                              bool &twrap_b)
{
    int b = c[0] & 1, xh = c[0] >> 1;
    nb[0] = (b && xh == g.Lxh - 1) ? cb - (g.Lxh - 1) : cb + b;
    nb[1] = (!b && xh == 0) ? cb + (g.Lxh - 1) : cb - (1 - b);
    nb[2] = (c[1] == g.L[1] - 1) ? cb - g.sY * (g.L[1] - 1) : cb + g.sY;
    nb[3] = (c[1] == 0) ? cb + g.sY * (g.L[1] - 1) : cb - g.sY;
    nb[4] = (c[2] == g.L[2] - 1) ? cb - g.sZ * (g.L[2] - 1) : cb + g.sZ;
    nb[5] = (c[2] == 0) ? cb + g.sZ * (g.L[2] - 1) : cb - g.sZ;
    twrap_f = (c[3] == g.L[3] - 1);
    twrap_b = (c[3] == 0);
    nb[6] = twrap_f ? cb - g.sT * (g.L[3] - 1) : cb + g.sT;
    nb[7] = twrap_b ? cb + g.sT * (g.L[3] - 1) : cb - g.sT;
}

// checkerboard index of coordinates (its parity is implied by the coordinates)
__device__ __forceinline__ int coords_cb(const Geo &g, const int c[4])
{
    return (c[0] >> 1) + g.Lxh * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}

__device__ __forceinline__ int coords_lex(const Geo &g, const int c[4])
{
    return c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}

// ------------------------------------------------------------------ values

template <typename R>
struct Cx {
    R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ Cx<R> cx(R re, R im)
{
    return Cx<R>{re, im};
}
template <typename R>
__host__ __device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b)
{
    return {a.re + b.re, a.im + b.im};
}
template <typename R>
__host__ __device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b)
{
    return {a.re - b.re, a.im - b.im};
}
template <typename R>
__host__ __device__ __forceinline__ Cx<R> operator-(Cx<R> a)
{
    return {-a.re, -a.im};
}
template <typename R>
__host__ __device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__host__ __device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a)
{
    return {s * a.re, s * a.im};
}
template <typename R>
__host__ __device__ __forceinline__ Cx<R> conj(Cx<R> a)
{
    return {a.re, -a.im};
}
// a^* b
template <typename R>
__host__ __device__ __forceinline__ Cx<R> cmul_conj(Cx<R> a, Cx<R> b)
{
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// i a
template <typename R>
__host__ __device__ __forceinline__ Cx<R> times_i(Cx<R> a)
{
    return {-a.im, a.re};
}
template <typename R>
__host__ __device__ __forceinline__ R norm2(Cx<R> a)
{
    return a.re * a.re + a.im * a.im;
}

template <typename R>
struct M3 {
    Cx<R> e[3][3];
};

template <typename R>
struct Sp { // 4 spin x 3 colour
    Cx<R> c[4][3];
};

template <typename R>
struct Hs { // projected half spinor: 2 spin x 3 colour
    Cx<R> c[2][3];
};

// the spatial hops' weight nu / xi0 of the anisotropic operator in the
// working precision (1 when isotropic)
template <typename R>
__device__ __forceinline__ R spatial_weight(const Geo &g);
template <>
__device__ __forceinline__ float spatial_weight<float>(const Geo &g)
{
    return g.csf;
}
template <>
__device__ __forceinline__ double spatial_weight<double>(const Geo &g)
{
    return g.cs;
}

template <typename R>
__device__ __forceinline__ Sp<R> sp_zero()
{
    Sp<R> s;
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) s.c[a][b] = cx<R>(0, 0);
    return s;
}

// s *= w, every component
template <typename R>
__device__ __forceinline__ void sp_scale(Sp<R> &s, R w)
{
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) s.c[a][b] = cx<R>(w * s.c[a][b].re, w * s.c[a][b].im);
}

template <typename R>
__device__ __forceinline__ M3<R> m3_mul(const M3<R> &a, const M3<R> &b)
{
    M3<R> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            Cx<R> s = a.e[i][0] * b.e[0][j];
            s = s + a.e[i][1] * b.e[1][j];
            s = s + a.e[i][2] * b.e[2][j];
            r.e[i][j] = s;
        }
    return r;
}

// a * b^dag
template <typename R>
__device__ __forceinline__ M3<R> m3_mul_dag(const M3<R> &a, const M3<R> &b)
{
    M3<R> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            Cx<R> s = a.e[i][0] * conj(b.e[j][0]);
            s = s + a.e[i][1] * conj(b.e[j][1]);
            s = s + a.e[i][2] * conj(b.e[j][2]);
            r.e[i][j] = s;
        }
    return r;
}

// a^dag * b
template <typename R>
__device__ __forceinline__ M3<R> m3_dag_mul(const M3<R> &a, const M3<R> &b)
{
    M3<R> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            Cx<R> s = cmul_conj(a.e[0][i], b.e[0][j]);
            s = s + cmul_conj(a.e[1][i], b.e[1][j]);
            s = s + cmul_conj(a.e[2][i], b.e[2][j]);
            r.e[i][j] = s;
        }
    return r;
}

template <typename R>
__device__ __forceinline__ void reconstruct_row2(M3<R> &u)
{
    u.e[2][0] = conj(u.e[0][1] * u.e[1][2] - u.e[0][2] * u.e[1][1]);
    u.e[2][1] = conj(u.e[0][2] * u.e[1][0] - u.e[0][0] * u.e[1][2]);
    u.e[2][2] = conj(u.e[0][0] * u.e[1][1] - u.e[0][1] * u.e[1][0]);
}

// ------------------------------------------------------------------ storage codecs

__device__ __forceinline__ uint32_t pack_h2(float a, float b)
{
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ float2 unpack_h2(uint32_t v)
{
    __half2 h = *reinterpret_cast<__half2 *>(&v);
    return __half22float2(h);
}
__device__ __forceinline__ uint32_t pack_b2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ float2 unpack_b2(uint32_t v)
{
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&v);
    return __bfloat1622float2(h);
}

template <typename T>
__device__ __forceinline__ T ldg(const T *p)
{
    return __ldg(p);
}

// Spinor field accessors: load / store the 24 reals of checkerboard site cb.
template <lqcd_prec P>
struct SpinorRef;

template <>
struct SpinorRef<LQCD_F64> {
    double2 *d;
    int Vh;
    template <typename R>
    __device__ __forceinline__ Sp<R> load(int cb) const
    {
        Sp<R> s;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            double2 v = ldg(d + (size_t)k * Vh + cb);
            s.c[k / 3][k % 3] = cx<R>((R)v.x, (R)v.y);
        }
        return s;
    }
    template <typename R>
    __device__ __forceinline__ Sp<R> load_rw(int cb) const
    {
        Sp<R> s;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            double2 v = d[(size_t)k * Vh + cb];
            s.c[k / 3][k % 3] = cx<R>((R)v.x, (R)v.y);
        }
        return s;
    }
    template <typename R>
    __device__ __forceinline__ Sp<R> load_scaled(int cb, R &scale) const
    {
        scale = (R)1;
        return load<R>(cb);
    }
    static constexpr bool has_norm = false;
    template <typename R>
    __device__ __forceinline__ void store(int cb, const Sp<R> &s) const
    {
#pragma unroll
        for (int k = 0; k < 12; k++)
            d[(size_t)k * Vh + cb] = make_double2((double)s.c[k / 3][k % 3].re, (double)s.c[k / 3][k % 3].im);
    }
};

template <>
struct SpinorRef<LQCD_F32> {
    float4 *d;
    int Vh;
    template <typename R>
    __device__ __forceinline__ Sp<R> unpack(const float4 (&v)[6]) const
    {
        Sp<R> s;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            int c0 = 2 * k, c1 = 2 * k + 1; // complex components 2k, 2k+1
            s.c[c0 / 3][c0 % 3] = cx<R>(v[k].x, v[k].y);
            s.c[c1 / 3][c1 % 3] = cx<R>(v[k].z, v[k].w);
        }
        return s;
    }
    template <typename R>
    __device__ __forceinline__ Sp<R> load(int cb) const
    {
        float4 v[6];
#pragma unroll
        for (int k = 0; k < 6; k++) v[k] = ldg(d + (size_t)k * Vh + cb);
        return unpack<R>(v);
    }
    template <typename R>
    __device__ __forceinline__ Sp<R> load_rw(int cb) const
    {
        float4 v[6];
#pragma unroll
        for (int k = 0; k < 6; k++) v[k] = d[(size_t)k * Vh + cb];
        return unpack<R>(v);
    }
    template <typename R>
    __device__ __forceinline__ Sp<R> load_scaled(int cb, R &scale) const
    {
        scale = (R)1;
        return load<R>(cb);
    }
    static constexpr bool has_norm = false;
    template <typename R>
    __device__ __forceinline__ void store(int cb, const Sp<R> &s) const
    {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            int c0 = 2 * k, c1 = 2 * k + 1;
            d[(size_t)k * Vh + cb] = make_float4((float)s.c[c0 / 3][c0 % 3].re, (float)s.c[c0 / 3][c0 % 3].im,
                                                 (float)s.c[c1 / 3][c1 % 3].re, (float)s.c[c1 / 3][c1 % 3].im);
        }
    }
};

// FP16 of value / norm, norm = max |real| over the site (FP32).
template <>
struct SpinorRef<LQCD_F16N> {
    uint4 *d;
    float *norm;
    int Vh;
    template <typename R>
    __device__ __forceinline__ Sp<R> unpack(const uint4 (&v)[3], float nrm) const
    {
        Sp<R> s;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint32_t w[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
            for (int q = 0; q < 4; q++) {
                int c = 4 * k + q; // complex component
                float2 f = unpack_h2(w[q]);
                s.c[c / 3][c % 3] = cx<R>((R)(f.x * nrm), (R)(f.y * nrm));
            }
        }
        return s;
    }
    template <typename R>
    __device__ __forceinline__ Sp<R> load(int cb) const
    {
        uint4 v[3];
#pragma unroll
        for (int k = 0; k < 3; k++) v[k] = ldg(d + (size_t)k * Vh + cb);
        return unpack<R>(v, ldg(norm + cb));
    }
    // the stored values (value / norm) and the norm, for callers that apply
    // the norm after a linear map
    template <typename R>
    __device__ __forceinline__ Sp<R> load_scaled(int cb, R &scale) const
    {
        uint4 v[3];
#pragma unroll
        for (int k = 0; k < 3; k++) v[k] = ldg(d + (size_t)k * Vh + cb);
        scale = (R)ldg(norm + cb);
        return unpack<R>(v, 1.0f);
    }
    static constexpr bool has_norm = true;
    template <typename R>
    __device__ __forceinline__ Sp<R> load_rw(int cb) const
    {
        uint4 v[3];
#pragma unroll
        for (int k = 0; k < 3; k++) v[k] = d[(size_t)k * Vh + cb];
        return unpack<R>(v, norm[cb]);
    }
    template <typename R>
    __device__ __forceinline__ void store(int cb, const Sp<R> &s) const
    {
        float m = 0.f;
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) m = fmaxf(m, fmaxf(fabsf((float)s.c[a][b].re), fabsf((float)s.c[a][b].im)));
        float inv = m > 0.f ? 1.0f / m : 0.f;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                int c = 4 * k + q;
                w[q] = pack_h2((float)s.c[c / 3][c % 3].re * inv, (float)s.c[c / 3][c % 3].im * inv);
            }
            d[(size_t)k * Vh + cb] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        norm[cb] = m;
    }
};

template <>
struct SpinorRef<LQCD_BF16> {
    uint4 *d;
    int Vh;
    template <typename R>
    __device__ __forceinline__ Sp<R> unpack(const uint4 (&v)[3]) const
    {
        Sp<R> s;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint32_t w[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
            for (int q = 0; q < 4; q++) {
                int c = 4 * k + q;
                float2 f = unpack_b2(w[q]);
                s.c[c / 3][c % 3] = cx<R>((R)f.x, (R)f.y);
            }
        }
        return s;
    }
    template <typename R>
    __device__ __forceinline__ Sp<R> load(int cb) const
    {
        uint4 v[3];
#pragma unroll
        for (int k = 0; k < 3; k++) v[k] = ldg(d + (size_t)k * Vh + cb);
        return unpack<R>(v);
    }
    template <typename R>
    __device__ __forceinline__ Sp<R> load_rw(int cb) const
    {
        uint4 v[3];
#pragma unroll
        for (int k = 0; k < 3; k++) v[k] = d[(size_t)k * Vh + cb];
        return unpack<R>(v);
    }
    template <typename R>
    __device__ __forceinline__ Sp<R> load_scaled(int cb, R &scale) const
    {
        scale = (R)1;
        return load<R>(cb);
    }
    static constexpr bool has_norm = false;
    template <typename R>
    __device__ __forceinline__ void store(int cb, const Sp<R> &s) const
    {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                int c = 4 * k + q;
                w[q] = pack_b2((float)s.c[c / 3][c % 3].re, (float)s.c[c / 3][c % 3].im);
            }
            d[(size_t)k * Vh + cb] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
};

template <lqcd_prec P>
__host__ inline SpinorRef<P> spinor_ref(const lqcd_field *f, int parity_block = 0);

template <>
__host__ inline SpinorRef<LQCD_F64> spinor_ref<LQCD_F64>(const lqcd_field *f, int parity_block)
{
    return {reinterpret_cast<double2 *>(f->data) + (size_t)parity_block * 12 * f->Vh, f->Vh};
}
template <>
__host__ inline SpinorRef<LQCD_F32> spinor_ref<LQCD_F32>(const lqcd_field *f, int)
{
    return {reinterpret_cast<float4 *>(f->data), f->Vh};
}
template <>
__host__ inline SpinorRef<LQCD_F16N> spinor_ref<LQCD_F16N>(const lqcd_field *f, int)
{
    return {reinterpret_cast<uint4 *>(f->data), f->norm, f->Vh};
}
template <>
__host__ inline SpinorRef<LQCD_BF16> spinor_ref<LQCD_BF16>(const lqcd_field *f, int)
{
    return {reinterpret_cast<uint4 *>(f->data), f->Vh};
}

// Gauge field accessors: link (mu, parity, cb) as a full 3x3 matrix.
template <lqcd_prec P>
struct GaugeRef;

template <>
struct GaugeRef<LQCD_F64> { // 18 reals: double2 [mu][par][9][Vh]
    double2 *d;
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
            double2 v = ldg(d + idx(mu, par, k, cb));
            u.e[k / 3][k % 3] = cx<R>((R)v.x, (R)v.y);
        }
        return u;
    }
    __device__ __forceinline__ void store(int mu, int par, int cb, const M3<double> &u) const
    {
#pragma unroll
        for (int k = 0; k < 9; k++) d[idx(mu, par, k, cb)] = make_double2(u.e[k / 3][k % 3].re, u.e[k / 3][k % 3].im);
    }
};

// 12 reals (rows 0 and 1) in 3 chunks of 4 reals:
//   chunk0 = u00 u01, chunk1 = u02 u10, chunk2 = u11 u12 (re, im each)
template <>
struct GaugeRef<LQCD_F32> {
    float4 *d;
    int Vh;
    __device__ __forceinline__ size_t idx(int mu, int par, int k, int cb) const
    {
        return ((size_t)((mu * 2 + par) * 3 + k)) * Vh + cb;
    }
    template <typename R>
    __device__ __forceinline__ M3<R> load(int mu, int par, int cb) const
    {
        float4 a = ldg(d + idx(mu, par, 0, cb)), b = ldg(d + idx(mu, par, 1, cb)), c = ldg(d + idx(mu, par, 2, cb));
        M3<R> u;
        u.e[0][0] = cx<R>(a.x, a.y);
        u.e[0][1] = cx<R>(a.z, a.w);
        u.e[0][2] = cx<R>(b.x, b.y);
        u.e[1][0] = cx<R>(b.z, b.w);
        u.e[1][1] = cx<R>(c.x, c.y);
        u.e[1][2] = cx<R>(c.z, c.w);
        reconstruct_row2(u);
        return u;
    }
    template <typename R>
    __device__ __forceinline__ void store(int mu, int par, int cb, const M3<R> &u) const
    {
        d[idx(mu, par, 0, cb)] = make_float4((float)u.e[0][0].re, (float)u.e[0][0].im, (float)u.e[0][1].re,
                                             (float)u.e[0][1].im);
        d[idx(mu, par, 1, cb)] = make_float4((float)u.e[0][2].re, (float)u.e[0][2].im, (float)u.e[1][0].re,
                                             (float)u.e[1][0].im);
        d[idx(mu, par, 2, cb)] = make_float4((float)u.e[1][1].re, (float)u.e[1][1].im, (float)u.e[1][2].re,
                                             (float)u.e[1][2].im);
    }
};

template <bool BF>
struct GaugeRef16 {
    uint2 *d;
    int Vh;
    __device__ __forceinline__ size_t idx(int mu, int par, int k, int cb) const
    {
        return ((size_t)((mu * 2 + par) * 3 + k)) * Vh + cb;
    }
    __device__ __forceinline__ float2 un(uint32_t w) const { return BF ? unpack_b2(w) : unpack_h2(w); }
    template <typename R>
    __device__ __forceinline__ uint32_t pk(R a, R b) const
    {
        return BF ? pack_b2((float)a, (float)b) : pack_h2((float)a, (float)b);
    }
    template <typename R>
    __device__ __forceinline__ M3<R> load(int mu, int par, int cb) const
    {
        return decode<R>(ldg(d + idx(mu, par, 0, cb)), ldg(d + idx(mu, par, 1, cb)), ldg(d + idx(mu, par, 2, cb)));
    }
    // the link from its three stored chunks
    template <typename R>
    __device__ __forceinline__ M3<R> decode(uint2 a, uint2 b, uint2 c) const
    {
        M3<R> u;
        float2 t;
        t = un(a.x); u.e[0][0] = cx<R>(t.x, t.y);
        t = un(a.y); u.e[0][1] = cx<R>(t.x, t.y);
        t = un(b.x); u.e[0][2] = cx<R>(t.x, t.y);
        t = un(b.y); u.e[1][0] = cx<R>(t.x, t.y);
        t = un(c.x); u.e[1][1] = cx<R>(t.x, t.y);
        t = un(c.y); u.e[1][2] = cx<R>(t.x, t.y);
        reconstruct_row2(u);
        return u;
    }
    template <typename R>
    __device__ __forceinline__ void store(int mu, int par, int cb, const M3<R> &u) const
    {
        d[idx(mu, par, 0, cb)] = make_uint2(pk(u.e[0][0].re, u.e[0][0].im), pk(u.e[0][1].re, u.e[0][1].im));
        d[idx(mu, par, 1, cb)] = make_uint2(pk(u.e[0][2].re, u.e[0][2].im), pk(u.e[1][0].re, u.e[1][0].im));
        d[idx(mu, par, 2, cb)] = make_uint2(pk(u.e[1][1].re, u.e[1][1].im), pk(u.e[1][2].re, u.e[1][2].im));
    }
};
template <>
struct GaugeRef<LQCD_F16N> : GaugeRef16<false> {};
template <>
struct GaugeRef<LQCD_BF16> : GaugeRef16<true> {};

template <lqcd_prec P>
__host__ inline GaugeRef<P> gauge_ref(const lqcd_field *f)
{
    GaugeRef<P> g;
    g.d = reinterpret_cast<decltype(g.d)>(f->data);
    g.Vh = f->Vh;
    return g;
}

// momentum coefficients: double [mu][par][8][Vh]
struct MomRef {
    double *d;
    int Vh;
    __device__ __forceinline__ size_t idx(int mu, int par, int a, int cb) const
    {
        return ((size_t)((mu * 2 + par) * 8 + a)) * Vh + cb;
    }
};
__host__ inline MomRef mom_ref(const lqcd_field *f) { return {reinterpret_cast<double *>(f->data), f->Vh}; }

// ------------------------------------------------------------------ reductions

// Deterministic sum of N doubles over a block of BLOCK threads; thread 0
// writes partials[k * nblocks + blockIdx.x].  Every thread of the block must
// call it (inactive threads pass zeros).
template <int N, int BLOCK>
__device__ __forceinline__ void block_sum_store(double (&v)[N], double *partials, int nblocks, int slot)
{
    static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "block size");
    __shared__ double sh[N][BLOCK / 32];
#pragma unroll
    for (int k = 0; k < N; k++) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < N; k++) sh[k][warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < N; k++) {
            double x = lane < BLOCK / 32 ? sh[k][lane] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
            if (lane == 0) partials[(size_t)k * nblocks + slot] = x;
        }
    }
}

// the block's sums of v into partials[k * nblocks + blockIdx.x]
template <int N, int BLOCK>
__device__ __forceinline__ void block_sum_store(double (&v)[N], double *partials, int nblocks)
{
    block_sum_store<N, BLOCK>(v, partials, nblocks, (int)blockIdx.x);
}

// The same for one value held in the kernel's working precision R: the warp
// sums run in R (an FP32 kernel stays off the FP64 pipe), the warp totals are
// summed in FP64.  Thread 0 writes partials[blockIdx.x].
template <int BLOCK, typename R>
__device__ __forceinline__ void block_sum_store_wp(R v, double *partials)
{
    static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "block size");
    __shared__ double sh[BLOCK / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = (double)v;
    __syncthreads();
    if (warp == 0) {
        double x = lane < BLOCK / 32 ? sh[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) partials[blockIdx.x] = x;
    }
}

// Fixed-order sum of partials[k * nblocks + i] over i, by one block of 1024
// threads; result in sums[k] (shared by the whole block after the call).
template <int N>
__device__ __forceinline__ void final_sum_block(const double *partials, int nblocks, double (&sums)[N])
{
    __shared__ double sh[N][32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < N; k++) {
        double x = 0;
        for (int i = threadIdx.x; i < nblocks; i += blockDim.x) x += partials[(size_t)k * nblocks + i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) sh[k][warp] = x;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; k++) {
        double x = 0;
        if (warp == 0) {
            x = lane < (int)(blockDim.x >> 5) ? sh[k][lane] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        }
        sums[k] = __shfl_sync(0xffffffffu, x, 0); // valid in warp 0
    }
}

// Host: sum N partial arrays into dst_dev[0..N) (device) with one block.
lqcd_status reduce_partials(const double *partials, int nblocks, int n, double *dst_dev, cudaStream_t s);

// Host: blocking read of n doubles from device memory through pinned memory.
lqcd_status read_scalars(const double *src_dev, double *host, int n, cudaStream_t s);

// ------------------------------------------------------------------ launch helpers

inline int nblocks_for(long n, int block) { return (int)((n + block - 1) / block); }

// internal entry points shared between translation units
lqcd_status dslash_dispatch(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger,
                            const lqcd_field *x, double a, double b, double *partials, cudaStream_t s);
lqcd_status field_alloc_like(const lqcd_field *like, lqcd_kind kind, lqcd_prec prec, int recon, lqcd_field **out);
lqcd_status field_alloc_df(const lqcd_lattice *lat, lqcd_kind kind, lqcd_field **out);
lqcd_status mhat_apply(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, double kappa, int dagger,
                       lqcd_field *tmp_odd, double *partials, cudaStream_t s);

} // namespace lqcd
