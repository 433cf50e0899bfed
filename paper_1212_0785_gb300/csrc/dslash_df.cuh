// dslash_df.cuh -- the float-float hopping term's device code (~48
// significant bits on the FP32 pipes), shared by the single-field kernels
// (dslash_df.cu) and the multi-system kernels (batch.cu).
#pragma once

#include "df64.cuh"
#include "dslash.cuh"
#include "spin.cuh"

namespace lqcd {

// ---------------------------------------------------------------- float-float kernel
//
// The float-float products of the mixed solver's accurate residual are long
// chains of dependent FP32 operations, so this kernel spreads each output
// site over three threads, one per colour a.  Each thread first projects
// colour a of the eight neighbour spinors onto half spinors and leaves them in
// shared memory; after one barrier it multiplies all three colours of each
// half spinor by row a of U (column a of U^dag), accumulating exact leading
// products with a single normalisation per dot product.

constexpr int DF_SITES = 64; // sites per block; blockDim = (64, 3)

// ---------------------------------------------------------------- packed pairs
//
// The two rows (h0, h1) of a projected half spinor enter the same products
// with the same link entries, so the kernel carries them as the two lanes of
// Blackwell's packed FP32x2 instructions (fma.rn.f32x2, add.rn.f32x2,
// mul.rn.f32x2: each lane rounded as its scalar counterpart).  Every lane
// runs exactly the scalar sequence of DfAcc and df_add_raw, so the error-free
// transformations stay exact and the results are those of the scalar form.

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 b2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2f(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2f(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

struct Df2 { // two float-float numbers, lane x and lane y
    float2 hi, lo;
};
__device__ __forceinline__ Df2 neg(const Df2 &a) { return Df2{neg2(a.hi), neg2(a.lo)}; }

// DfAcc in both lanes
struct DfAcc2 {
    float2 s, c;
    __device__ __forceinline__ void add_prod(Df a, const Df2 &b)
    {
        const float2 p = mul2f(b2(a.hi), b.hi);
        float2 e = fma2f(b2(a.hi), b.hi, neg2(p));
        e = fma2f(b2(a.hi), b.lo, e);
        e = fma2f(b2(a.lo), b.hi, e);
        const float2 t = add2(s, p);
        const float2 v = sub2(t, s);
        c = add2(c, add2(add2(sub2(s, sub2(t, v)), sub2(p, v)), e));
        s = t;
    }
    __device__ __forceinline__ void sub_prod(Df a, const Df2 &b) { add_prod(Df(-a.hi, -a.lo), b); }
    __device__ __forceinline__ void set_prod(Df a, const Df2 &b)
    {
        s = mul2f(b2(a.hi), b.hi);
        float2 e = fma2f(b2(a.hi), b.hi, neg2(s));
        e = fma2f(b2(a.hi), b.lo, e);
        c = fma2f(b2(a.lo), b.hi, e);
    }
    __device__ __forceinline__ void set(const Df2 &a) { s = a.hi, c = a.lo; }
    __device__ __forceinline__ void add(const Df2 &a)
    {
        const float2 t = add2(s, a.hi);
        const float2 v = sub2(t, s);
        c = add2(c, add2(add2(sub2(s, sub2(t, v)), sub2(a.hi, v)), a.lo));
        s = t;
    }
    __device__ __forceinline__ Df2 raw() const { return Df2{s, c}; }
};

// df_add_raw in both lanes
__device__ __forceinline__ Df2 add_raw2(const Df2 &a, const Df2 &b)
{
    const float2 s = add2(a.hi, b.hi);
    const float2 v = sub2(s, a.hi);
    const float2 e = add2(sub2(a.hi, sub2(s, v)), sub2(b.hi, v));
    return Df2{s, add2(e, add2(a.lo, b.lo))};
}

// lanes of two Df values, and of a complex pair split into re and im
__device__ __forceinline__ Df2 lanes(Df x, Df y) { return Df2{f2(x.hi, y.hi), f2(x.lo, y.lo)}; }

// the projected half spinors of one block: [hop][colour][site] as two float4,
// re = (h0.re.hi, h1.re.hi, h0.re.lo, h1.re.lo) and im likewise (48 KiB), so
// each pair of lanes is read as it is stored
struct DfHalves {
    float4 re[8][3][DF_SITES], im[8][3][DF_SITES];
};

// colour a of (1 + S gamma_mu) psi at site nb, rows (h0, h1) as lanes (the
// table above project()); k v for k in {+1, -1, +i, -i} is exact, so each lane
// is the scalar float-float sum of the re and im parts
template <int MU, int S>
__device__ __forceinline__ void project_colour_df2(const SpinorRef<PREC_DF> &in, int nb, int a, Df2 &hre, Df2 &him)
{
    Cx<Df> p[4];
#pragma unroll
    for (int sp = 0; sp < 4; sp++) {
        float4 v = ldg(in.d + (size_t)(sp * 3 + a) * in.Vh + nb);
        p[sp] = Cx<Df>{Df(v.x, v.y), Df(v.z, v.w)};
    }
    Cx<Df> q0, q1; // the terms added to p0 (row 0) and p1 (row 1)
    if (MU == 0) {
        q0 = s_i<S>(p[3]);
        q1 = s_i<S>(p[2]);
    } else if (MU == 1) {
        q0 = -s_1<S>(p[3]);
        q1 = s_1<S>(p[2]);
    } else if (MU == 2) {
        q0 = s_i<S>(p[2]);
        q1 = -s_i<S>(p[3]);
    } else {
        q0 = s_1<S>(p[2]);
        q1 = s_1<S>(p[3]);
    }
    hre = add_raw2(lanes(p[0].re, p[1].re), lanes(q0.re, q1.re));
    him = add_raw2(lanes(p[0].im, p[1].im), lanes(q0.im, q1.im));
}

template <int MU, int FS, int BS>
__device__ __forceinline__ void project_dir_df(DfHalves &sh, const SpinorRef<PREC_DF> &in, int x, int a, int nf,
                                               int nbk)
{
    Df2 hr, hi;
    project_colour_df2<MU, FS>(in, nf, a, hr, hi);
    sh.re[2 * MU][a][x] = make_float4(hr.hi.x, hr.hi.y, hr.lo.x, hr.lo.y);
    sh.im[2 * MU][a][x] = make_float4(hi.hi.x, hi.hi.y, hi.lo.x, hi.lo.y);
    project_colour_df2<MU, BS>(in, nbk, a, hr, hi);
    sh.re[2 * MU + 1][a][x] = make_float4(hr.hi.x, hr.hi.y, hr.lo.x, hr.lo.y);
    sh.im[2 * MU + 1][a][x] = make_float4(hi.hi.x, hi.hi.y, hi.lo.x, hi.lo.y);
}

__device__ __forceinline__ Df2 df2_of(float4 v) { return Df2{f2(v.x, v.y), f2(v.z, v.w)}; }

// both lanes times c in float-float (the spatial hops' weight of the anisotropic operator)
__device__ __forceinline__ Df2 scale_lanes(const Df2 &v, Df c)
{
    return lanes(Df(v.hi.x, v.lo.x) * c, Df(v.hi.y, v.lo.y) * c);
}

// accumulators of the four output spin rows: rows (0, 1) and (2, 3) as lanes
struct DfOut {
    DfAcc2 r01, i01, r23, i23;
};

// k v for k = +1, -1, +i, -i (kind 0..3) as (re, im) lane by lane: the kind
// and the source lane can differ between the two lanes
template <int KIND>
__device__ __forceinline__ void kind_of(const Df2 &vr, const Df2 &vi, int lane, Df &r, Df &i)
{
    const Df xr = lane ? Df(vr.hi.y, vr.lo.y) : Df(vr.hi.x, vr.lo.x);
    const Df xi = lane ? Df(vi.hi.y, vi.lo.y) : Df(vi.hi.x, vi.lo.x);
    r = KIND == 0 ? xr : KIND == 1 ? -xr : KIND == 2 ? -xi : xi;
    i = KIND == 0 ? xi : KIND == 1 ? -xi : KIND == 2 ? xr : -xr;
}

// the reconstruction of (1 + S gamma_mu) from rows (v0, v1) = lanes of (vr, vi)
// into the four output rows (the table above project()): rows 0, 1 add v0, v1;
// rows 2, 3 add the multiples of the rows listed in acc_hop
template <int MU, int S, bool FIRST>
__device__ __forceinline__ void acc_hop2(DfOut &o, const Df2 &vr, const Df2 &vi)
{
    if (FIRST) {
        o.r01.set(vr);
        o.i01.set(vi);
    } else {
        o.r01.add(vr);
        o.i01.add(vi);
    }
    constexpr int MI = S > 0 ? 3 : 2; // -S i
    constexpr int PI = S > 0 ? 2 : 3; // +S i
    constexpr int P1 = S > 0 ? 0 : 1; // +S
    constexpr int M1 = S > 0 ? 1 : 0; // -S
    constexpr int K2 = MU == 0 ? MI : MU == 1 ? P1 : MU == 2 ? MI : P1; // row 2 ...
    constexpr int L2 = MU <= 1 ? 1 : 0;                                  // ... of row L2 of (v0, v1)
    constexpr int K3 = MU == 0 ? MI : MU == 1 ? M1 : MU == 2 ? PI : P1; // row 3 ...
    constexpr int L3 = MU <= 1 ? 0 : 1;                                  // ... of row L3
    Df r2, i2, r3, i3;
    kind_of<K2>(vr, vi, L2, r2, i2);
    kind_of<K3>(vr, vi, L3, r3, i3);
    const Df2 ar = lanes(r2, r3), ai = lanes(i2, i3);
    if (FIRST) {
        o.r23.set(ar);
        o.i23.set(ai);
    } else {
        o.r23.add(ar);
        o.i23.add(ai);
    }
}

// Each dot product starts from its first exact product and its sums reach the
// output rows unnormalised; only the output is normalised.
template <int MU, int FS, int BS>
__device__ __forceinline__ void hop_dir_df(DfOut &o, const DfHalves &sh, const GaugeRef<PREC_DF> &U, const Geo &g,
                                           int cb, int out_par, int x, int a, int nbk, bool wrap_f, bool wrap_b)
{
    const bool antip = (MU == 3) && g.t_bc < 0;
    { // forward: row a of U_mu(x)
        DfAcc2 r, i;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            float4 w = ldg(U.d + U.idx(MU, out_par, a * 3 + b, cb));
            Df ur(w.x, w.y), ui(w.z, w.w);
            const Df2 hr = df2_of(sh.re[2 * MU][b][x]), hi = df2_of(sh.im[2 * MU][b][x]);
            if (b == 0) {
                r.set_prod(ur, hr);
                i.set_prod(ur, hi);
            } else {
                r.add_prod(ur, hr);
                i.add_prod(ur, hi);
            }
            r.sub_prod(ui, hi);
            i.add_prod(ui, hr);
        }
        Df2 vr = r.raw(), vi = i.raw();
        if (antip && wrap_f) {
            vr = neg(vr);
            vi = neg(vi);
        }
        if (MU < 3 && g.aniso) {
            vr = scale_lanes(vr, Df(g.cs));
            vi = scale_lanes(vi, Df(g.cs));
        }
        acc_hop2<MU, FS, MU == 0>(o, vr, vi);
    }
    { // backward: column a of U_mu(x - mu), conjugated
        DfAcc2 r, i;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            float4 w = ldg(U.d + U.idx(MU, 1 - out_par, b * 3 + a, nbk));
            Df ur(w.x, w.y), ui(w.z, w.w);
            const Df2 hr = df2_of(sh.re[2 * MU + 1][b][x]), hi = df2_of(sh.im[2 * MU + 1][b][x]);
            if (b == 0) {
                r.set_prod(ur, hr);
                i.set_prod(ur, hi);
            } else {
                r.add_prod(ur, hr);
                i.add_prod(ur, hi);
            }
            r.add_prod(ui, hi);
            i.sub_prod(ui, hr);
        }
        Df2 vr = r.raw(), vi = i.raw();
        if (antip && wrap_b) {
            vr = neg(vr);
            vi = neg(vi);
        }
        if (MU < 3 && g.aniso) {
            vr = scale_lanes(vr, Df(g.cs));
            vi = scale_lanes(vi, Df(g.cs));
        }
        acc_hop2<MU, BS, false>(o, vr, vi);
    }
}

// The block body: output sites blk * DF_SITES + threadIdx.x, colour
// threadIdx.y (the kernels of dslash_df.cu and the multi-system kernels of
// batch.cu).
template <bool DAG, bool XPAY>
__device__ __forceinline__ void df_hop_block(DfHalves &sh, SpinorRef<PREC_DF> out, SpinorRef<PREC_DF> in,
                                             GaugeRef<PREC_DF> U, const Geo &g, int out_par, SpinorRef<PREC_DF> x,
                                             Df b, int blk)
{
    const int tx = threadIdx.x, a = threadIdx.y;
    const int cb = blk * DF_SITES + tx;
    const bool live = cb < g.Vh;
    int c[4], nb[8];
    bool tf = false, tb = false;
    constexpr int FS = DAG ? +1 : -1;
    constexpr int BS = -FS;
    if (live) {
        cb_coords(g, cb, out_par, c);
        cb_neighbours(g, cb, c, nb, tf, tb);
        project_dir_df<0, FS, BS>(sh, in, tx, a, nb[0], nb[1]);
        project_dir_df<1, FS, BS>(sh, in, tx, a, nb[2], nb[3]);
        project_dir_df<2, FS, BS>(sh, in, tx, a, nb[4], nb[5]);
        project_dir_df<3, FS, BS>(sh, in, tx, a, nb[6], nb[7]);
    }
    __syncthreads();
    if (!live) return;
    DfOut o;
    hop_dir_df<0, FS, BS>(o, sh, U, g, cb, out_par, tx, a, nb[1], false, false);
    hop_dir_df<1, FS, BS>(o, sh, U, g, cb, out_par, tx, a, nb[3], false, false);
    hop_dir_df<2, FS, BS>(o, sh, U, g, cb, out_par, tx, a, nb[5], false, false);
    hop_dir_df<3, FS, BS>(o, sh, U, g, cb, out_par, tx, a, nb[7], tf, tb);
#pragma unroll
    for (int sp = 0; sp < 4; sp++) {
        const DfAcc2 &R = sp < 2 ? o.r01 : o.r23, &I = sp < 2 ? o.i01 : o.i23;
        const int ln = sp & 1;
        Cx<Df> v{DfAcc::df_fast_two_sum_any(ln ? R.s.y : R.s.x, ln ? R.c.y : R.c.x),
                 DfAcc::df_fast_two_sum_any(ln ? I.s.y : I.s.x, ln ? I.c.y : I.c.x)};
        size_t k = (size_t)(sp * 3 + a) * out.Vh + cb;
        if (XPAY) {
            float4 xv = x.d[k];
            Cx<Df> xc{Df(xv.x, xv.y), Df(xv.z, xv.w)};
            v = xc + b * v;
        }
        out.d[k] = df_from<Df>(v);
    }
}

// the per-site work of the mixed solver's reliable update (cg.cu and the
// multi-system kernels of batch.cu): x += xs, xs = 0
__device__ __forceinline__ void accum_df_site(const SpinorRef<PREC_DF> &x, const SpinorRef<LQCD_F32> &xs, int cb)
{
    Sp<Df> xv = x.load_rw<Df>(cb);
    Sp<float> dv = xs.load_rw<float>(cb);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            xv.c[a][k].re += Df(dv.c[a][k].re, 0.f);
            xv.c[a][k].im += Df(dv.c[a][k].im, 0.f);
        }
    x.store(cb, xv);
    xs.store(cb, sp_zero<float>());
}

// r = b - t in float-float; returns |r|^2 of the leading parts (FP32)
__device__ __forceinline__ float residual_df_site(const SpinorRef<PREC_DF> &r, const SpinorRef<PREC_DF> &b,
                                                  const SpinorRef<PREC_DF> &t, int cb)
{
    Sp<Df> bv = b.load_rw<Df>(cb), tv = t.load_rw<Df>(cb);
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            bv.c[a][k] = bv.c[a][k] - tv.c[a][k];
            acc += bv.c[a][k].re.hi * bv.c[a][k].re.hi + bv.c[a][k].im.hi * bv.c[a][k].im.hi;
        }
    r.store(cb, bv);
    return acc;
}

} // namespace lqcd
