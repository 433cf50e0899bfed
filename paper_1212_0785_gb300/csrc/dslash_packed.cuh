// dslash_packed.cuh -- the FP16+norm hopping term at one output site with
// Blackwell's packed arithmetic: FP16x2 for the spin projection, FP32x2
// (fma.rn.f32x2 / mul.rn.f32x2, one instruction for two FP32 lanes, each
// rounded as fmaf / a * b) for the link product and the reconstruction.
//
// Each stored word of an FP16+norm spinor is one complex component (re, im)
// of value / norm, so a projected component (1 + S gamma_mu) psi is one FP16x2
// add of two stored words (the factor +-i swaps the halves), rounded once to
// FP16 -- relative error 2^-11, the size of the storage rounding itself --
// and only the 12 projected reals, not the 24 stored ones, are widened to
// FP32: the f16 -> f32 conversions were the busiest instructions of the FMA
// pipe.  The two spin rows of a projected half spinor are then carried as
// pairs: for colour j, re[j] = (row0.re, row1.re) and im[j] = (row0.im,
// row1.im), so the SU(3) matrix times half spinor and the reconstruction of
// spin rows 0, 1 and 2, 3 act on both rows with one packed instruction (the
// x and y hops take the pairs swapped), and so does the scaling of the stored
// output by its norm.  Links are prefetched into shared memory
// as in prefetch_site, and the directions, neighbours, boundary signs and
// per-site norms are those of dslash_site.  The bits differ from forms 0 and
// 1 by the FP16 rounding of the projection and the order of the FP32 products.
#pragma once

#include "dslash_site.cuh"

namespace lqcd {

struct HsP { // two spin rows of a half spinor, packed pairwise
    float2 re[3], im[3];
};
struct SpP { // a spinor: [0] spins (0, 1), [1] spins (2, 3), packed pairwise
    float2 re[2][3], im[2][3];
};

__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 swp(float2 a) { return make_float2(a.y, a.x); }

// U h (FWD) or U^dag h, both rows at once
template <bool FWD>
__device__ __forceinline__ HsP mul_link_p(const M3<float> &u, const HsP &h)
{
    HsP o;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float2 re, im;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            // U h: u = u_aj; U^dag h: u = conj(u_ja)
            const float ur = FWD ? u.e[a][j].re : u.e[j][a].re;
            const float ui = FWD ? u.e[a][j].im : -u.e[j][a].im;
            if (j == 0) {
                re = mul2(bc(ur), h.re[0]);
                im = mul2(bc(ur), h.im[0]);
            } else {
                re = fma2(bc(ur), h.re[j], re);
                im = fma2(bc(ur), h.im[j], im);
            }
            re = fma2(bc(-ui), h.im[j], re);
            im = fma2(bc(ui), h.re[j], im);
        }
        o.re[a] = re;
        o.im[a] = im;
    }
    return o;
}

// acc += sc times the reconstruction of (1 + S gamma_mu) from its rows (o0, o1):
//   rows 0, 1 += (o0, o1);   rows 2, 3 +=
//   x: (-S i o1, -S i o0)   y: (S o1, -S o0)   z: (-S i o0, S i o1)   t: (S o0, S o1)
// (the x and y hops take the rows in swapped order: the pairs are swapped
// first, so every lane is the same fmaf as in scalar form)
template <int MU, int S>
__device__ __forceinline__ void accumulate_p(SpP &acc, const HsP &o, float sc)
{
    const float s = (float)S * sc;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        acc.re[0][a] = fma2(bc(sc), o.re[a], acc.re[0][a]);
        acc.im[0][a] = fma2(bc(sc), o.im[a], acc.im[0][a]);
        if (MU == 0) { // -S i (x + i y) = S y - i S x, rows swapped
            acc.re[1][a] = fma2(swp(o.im[a]), bc(s), acc.re[1][a]);
            acc.im[1][a] = fma2(swp(o.re[a]), bc(-s), acc.im[1][a]);
        } else if (MU == 1) {
            acc.re[1][a] = fma2(swp(o.re[a]), pk(s, -s), acc.re[1][a]);
            acc.im[1][a] = fma2(swp(o.im[a]), pk(s, -s), acc.im[1][a]);
        } else if (MU == 2) {
            acc.re[1][a] = fma2(o.im[a], pk(s, -s), acc.re[1][a]);
            acc.im[1][a] = fma2(o.re[a], pk(-s, s), acc.im[1][a]);
        } else {
            acc.re[1][a] = fma2(o.re[a], bc(s), acc.re[1][a]);
            acc.im[1][a] = fma2(o.im[a], bc(s), acc.im[1][a]);
        }
    }
}

__device__ __forceinline__ __half2 as_h2(uint32_t w) { return *reinterpret_cast<const __half2 *>(&w); }

// (1 + S gamma_mu) psi straight from the stored halves: each stored word is
// one complex component (re, im) of value / norm, and each projected
// component is one FP16 add of two of them (i q = (-q.im, q.re): the swapped
// pair times (-1, 1)), correctly rounded to FP16; only the 12 projected reals
// are widened to FP32 for the link product
template <int MU, int S>
__device__ __forceinline__ HsP load_project_h(const SpinorRef<LQCD_F16N> &in, int cb, float &nrm)
{
    uint4 v[3];
#pragma unroll
    for (int k = 0; k < 3; k++) v[k] = ldg(in.d + (size_t)k * in.Vh + cb);
    nrm = ldg(in.norm + cb);
    const uint32_t w[12] = {v[0].x, v[0].y, v[0].z, v[0].w, v[1].x, v[1].y,
                            v[1].z, v[1].w, v[2].x, v[2].y, v[2].z, v[2].w};
    const __half2 pi = __floats2half2_rn((float)-S, (float)S); // S i: (re, im) -> (-S im, S re)
    const __half2 mi = __floats2half2_rn((float)S, (float)-S); // -S i
    HsP h;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const __half2 p0 = as_h2(w[j]), p1 = as_h2(w[3 + j]), p2 = as_h2(w[6 + j]), p3 = as_h2(w[9 + j]);
        __half2 h0, h1;
        if (MU == 0) {
            h0 = __hfma2(__lowhigh2highlow(p3), pi, p0);
            h1 = __hfma2(__lowhigh2highlow(p2), pi, p1);
        } else if (MU == 1) {
            h0 = S > 0 ? __hsub2(p0, p3) : __hadd2(p0, p3);
            h1 = S > 0 ? __hadd2(p1, p2) : __hsub2(p1, p2);
        } else if (MU == 2) {
            h0 = __hfma2(__lowhigh2highlow(p2), pi, p0);
            h1 = __hfma2(__lowhigh2highlow(p3), mi, p1);
        } else {
            h0 = S > 0 ? __hadd2(p0, p2) : __hsub2(p0, p2);
            h1 = S > 0 ? __hadd2(p1, p3) : __hsub2(p1, p3);
        }
        h.re[j] = make_float2(__low2float(h0), __low2float(h1));
        h.im[j] = make_float2(__high2float(h0), __high2float(h1));
    }
    return h;
}

template <bool DAG, int BLOCK = DS_BLOCK>
__device__ __forceinline__ SpP packed_acc(const SpinorRef<LQCD_F16N> &in, const GaugeRef<LQCD_F16N> &U,
                                          const Geo &g, int cb, int out_par)
{
    __shared__ LinkPrefetchT<BLOCK> lp;
    const int i = threadIdx.x;
    int c[4], nb[8];
    bool tf, tb;
    cb_coords(g, cb, out_par, c);
    cb_neighbours(g, cb, c, nb, tf, tb);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            cp_async8(&lp.u[mu][0][k][i], U.d + U.idx(mu, out_par, k, cb));
            cp_async8(&lp.u[mu][1][k][i], U.d + U.idx(mu, 1 - out_par, k, nb[2 * mu + 1]));
        }
        cp_async_commit();
    }
    constexpr int FS = DAG ? +1 : -1;
    constexpr int BS = -FS;
    const bool antip = g.t_bc < 0;
    SpP acc;
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int a = 0; a < 3; a++) acc.re[h][a] = acc.im[h][a] = make_float2(0.f, 0.f);
    float sc;
#define LQCD_PK_LINK(mu, f) U.template decode<float>(lp.u[mu][f][0][i], lp.u[mu][f][1][i], lp.u[mu][f][2][i])
    // the spatial hops carry the anisotropic operator's weight nu / xi0 in
    // their scale (csf = 1 exactly when isotropic, so nothing changes there)
    // each hop: gather and project the neighbour (its loads issued before
    // the direction's links are waited for), multiply by the link, add
    {
        HsP hp;
        hp = load_project_h<0, FS>(in, nb[0], sc);
        cp_async_wait<3>();
        accumulate_p<0, FS>(acc, mul_link_p<true>(LQCD_PK_LINK(0, 0), hp), sc * g.csf);
        hp = load_project_h<0, BS>(in, nb[1], sc);
        accumulate_p<0, BS>(acc, mul_link_p<false>(LQCD_PK_LINK(0, 1), hp), sc * g.csf);
        hp = load_project_h<1, FS>(in, nb[2], sc);
        cp_async_wait<2>();
        accumulate_p<1, FS>(acc, mul_link_p<true>(LQCD_PK_LINK(1, 0), hp), sc * g.csf);
        hp = load_project_h<1, BS>(in, nb[3], sc);
        accumulate_p<1, BS>(acc, mul_link_p<false>(LQCD_PK_LINK(1, 1), hp), sc * g.csf);
        hp = load_project_h<2, FS>(in, nb[4], sc);
        cp_async_wait<1>();
        accumulate_p<2, FS>(acc, mul_link_p<true>(LQCD_PK_LINK(2, 0), hp), sc * g.csf);
        hp = load_project_h<2, BS>(in, nb[5], sc);
        accumulate_p<2, BS>(acc, mul_link_p<false>(LQCD_PK_LINK(2, 1), hp), sc * g.csf);
        hp = load_project_h<3, FS>(in, nb[6], sc);
        cp_async_wait<0>();
        accumulate_p<3, FS>(acc, mul_link_p<true>(LQCD_PK_LINK(3, 0), hp), (antip && tf) ? -sc : sc);
        hp = load_project_h<3, BS>(in, nb[7], sc);
        accumulate_p<3, BS>(acc, mul_link_p<false>(LQCD_PK_LINK(3, 1), hp), (antip && tb) ? -sc : sc);
    }
#undef LQCD_PK_LINK
    return acc;
}

template <bool DAG, int BLOCK = DS_BLOCK>
__device__ __forceinline__ Sp<float> packed_site(const SpinorRef<LQCD_F16N> &in, const GaugeRef<LQCD_F16N> &U,
                                                 const Geo &g, int cb, int out_par)
{
    const SpP acc = packed_acc<DAG, BLOCK>(in, U, g, cb, out_par);
    Sp<float> out;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        out.c[0][a] = cx<float>(acc.re[0][a].x, acc.im[0][a].x);
        out.c[1][a] = cx<float>(acc.re[0][a].y, acc.im[0][a].y);
        out.c[2][a] = cx<float>(acc.re[1][a].x, acc.im[1][a].x);
        out.c[3][a] = cx<float>(acc.re[1][a].y, acc.im[1][a].y);
    }
    return out;
}

// SpinorRef<F16N>::store of the packed accumulator: the same norm (max
// |component|), the same products value * (1 / norm) lane by lane (FP32x2),
// the same FP16 rounding -- bitwise the same stored site
__device__ __forceinline__ void store_packed(const SpinorRef<LQCD_F16N> &out, int cb, const SpP &acc)
{
    float m = 0.f;
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int a = 0; a < 3; a++)
            m = fmaxf(fmaxf(m, fmaxf(fabsf(acc.re[h][a].x), fabsf(acc.im[h][a].x))),
                      fmaxf(fabsf(acc.re[h][a].y), fabsf(acc.im[h][a].y)));
    const float inv = m > 0.f ? 1.0f / m : 0.f;
    SpP v;
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int a = 0; a < 3; a++) v.re[h][a] = mul2(acc.re[h][a], bc(inv)), v.im[h][a] = mul2(acc.im[h][a], bc(inv));
    // component c = spin * 3 + colour: spin 2h + lane, colour a
    uint32_t w[12];
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            w[(2 * h) * 3 + a] = pack_h2(v.re[h][a].x, v.im[h][a].x);
            w[(2 * h + 1) * 3 + a] = pack_h2(v.re[h][a].y, v.im[h][a].y);
        }
#pragma unroll
    for (int k = 0; k < 3; k++) out.d[(size_t)k * out.Vh + cb] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
    out.norm[cb] = m;
}

} // namespace lqcd
