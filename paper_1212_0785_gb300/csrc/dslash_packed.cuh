// dslash_packed.cuh -- the FP16+norm hopping term at one output site with
// Blackwell's packed FP32 arithmetic (fma.rn.f32x2 / mul.rn.f32x2, one
// instruction for two FP32 lanes, each rounded as fmaf / a * b).
//
// The two spin rows of a projected half spinor are carried as pairs: for
// colour j, re[j] = (row0.re, row1.re) and im[j] = (row0.im, row1.im).  The
// spin projection, the SU(3) matrix times half spinor and the reconstruction
// of spin rows 0, 1 (and, for z and t, rows 2, 3) then act on both rows with
// one packed instruction where the scalar form needs two; the x and y hops
// reconstruct rows 2, 3 from the rows in swapped order, which stays scalar.
// Links are prefetched into shared memory as in prefetch_site, and the
// directions, neighbours, boundary signs and per-site norms are those of
// dslash_site.  The products are rounded in a different order than the
// scalar form, so the bits differ from forms 0 and 1 (within FP32 rounding).
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

// the 24 stored reals of an FP16+norm site (value / norm, not rescaled)
struct SpF {
    float re[4][3], im[4][3];
};
__device__ __forceinline__ SpF load_f16_unscaled(const SpinorRef<LQCD_F16N> &in, int cb, float &nrm)
{
    uint4 v[3];
#pragma unroll
    for (int k = 0; k < 3; k++) v[k] = ldg(in.d + (size_t)k * in.Vh + cb);
    nrm = ldg(in.norm + cb);
    SpF p;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const uint32_t w[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int c = 4 * k + q;
            const float2 f = unpack_h2(w[q]);
            p.re[c / 3][c % 3] = f.x;
            p.im[c / 3][c % 3] = f.y;
        }
    }
    return p;
}

// (1 + S gamma_mu) psi: the two rows (h0, h1) of the DeGrand-Rossi projection
//   x: h0 = p0 + S i p3, h1 = p1 + S i p2     y: h0 = p0 - S p3, h1 = p1 + S p2
//   z: h0 = p0 + S i p2, h1 = p1 - S i p3     t: h0 = p0 + S p2, h1 = p1 + S p3
// with i q = (-q.im, q.re); multiplying by +-1 is exact, so each lane is the
// scalar sum
template <int MU, int S>
__device__ __forceinline__ HsP project_p(const SpF &p)
{
    HsP h;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const float2 r01 = pk(p.re[0][j], p.re[1][j]), i01 = pk(p.im[0][j], p.im[1][j]);
        if (MU == 0) {
            h.re[j] = fma2(pk(p.im[3][j], p.im[2][j]), bc((float)-S), r01);
            h.im[j] = fma2(pk(p.re[3][j], p.re[2][j]), bc((float)S), i01);
        } else if (MU == 1) {
            h.re[j] = fma2(pk(p.re[3][j], p.re[2][j]), pk((float)-S, (float)S), r01);
            h.im[j] = fma2(pk(p.im[3][j], p.im[2][j]), pk((float)-S, (float)S), i01);
        } else if (MU == 2) {
            h.re[j] = fma2(pk(p.im[2][j], p.im[3][j]), pk((float)-S, (float)S), r01);
            h.im[j] = fma2(pk(p.re[2][j], p.re[3][j]), pk((float)S, (float)-S), i01);
        } else {
            h.re[j] = fma2(pk(p.re[2][j], p.re[3][j]), bc((float)S), r01);
            h.im[j] = fma2(pk(p.im[2][j], p.im[3][j]), bc((float)S), i01);
        }
    }
    return h;
}

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
template <int MU, int S>
__device__ __forceinline__ void accumulate_p(SpP &acc, const HsP &o, float sc)
{
    const float s = (float)S * sc;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        acc.re[0][a] = fma2(bc(sc), o.re[a], acc.re[0][a]);
        acc.im[0][a] = fma2(bc(sc), o.im[a], acc.im[0][a]);
        if (MU == 0) { // -S i (x + i y) = S y - i S x, rows swapped
            acc.re[1][a].x = fmaf(s, o.im[a].y, acc.re[1][a].x);
            acc.re[1][a].y = fmaf(s, o.im[a].x, acc.re[1][a].y);
            acc.im[1][a].x = fmaf(-s, o.re[a].y, acc.im[1][a].x);
            acc.im[1][a].y = fmaf(-s, o.re[a].x, acc.im[1][a].y);
        } else if (MU == 1) {
            acc.re[1][a].x = fmaf(s, o.re[a].y, acc.re[1][a].x);
            acc.re[1][a].y = fmaf(-s, o.re[a].x, acc.re[1][a].y);
            acc.im[1][a].x = fmaf(s, o.im[a].y, acc.im[1][a].x);
            acc.im[1][a].y = fmaf(-s, o.im[a].x, acc.im[1][a].y);
        } else if (MU == 2) {
            acc.re[1][a] = fma2(o.im[a], pk(s, -s), acc.re[1][a]);
            acc.im[1][a] = fma2(o.re[a], pk(-s, s), acc.im[1][a]);
        } else {
            acc.re[1][a] = fma2(o.re[a], bc(s), acc.re[1][a]);
            acc.im[1][a] = fma2(o.im[a], bc(s), acc.im[1][a]);
        }
    }
}

template <int MU, int S, bool FWD>
__device__ __forceinline__ void hop_packed(SpP &acc, const SpF &psi, float sc, const M3<float> &u, bool flip)
{
    accumulate_p<MU, S>(acc, mul_link_p<FWD>(u, project_p<MU, S>(psi)), flip ? -sc : sc);
}

template <bool DAG, int BLOCK = DS_BLOCK>
__device__ __forceinline__ Sp<float> packed_site(const SpinorRef<LQCD_F16N> &in, const GaugeRef<LQCD_F16N> &U,
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
    SpF psi;
#define LQCD_PK_LINK(mu, f) U.template decode<float>(lp.u[mu][f][0][i], lp.u[mu][f][1][i], lp.u[mu][f][2][i])
    // the spatial hops' weight (anisotropic operator), folded into the norm
#define LQCD_SP(x) (g.aniso ? (x) * (float)g.cs : (x))
    psi = load_f16_unscaled(in, nb[0], sc);
    cp_async_wait<3>();
    hop_packed<0, FS, true>(acc, psi, LQCD_SP(sc), LQCD_PK_LINK(0, 0), false);
    psi = load_f16_unscaled(in, nb[1], sc);
    hop_packed<0, BS, false>(acc, psi, LQCD_SP(sc), LQCD_PK_LINK(0, 1), false);
    psi = load_f16_unscaled(in, nb[2], sc);
    cp_async_wait<2>();
    hop_packed<1, FS, true>(acc, psi, LQCD_SP(sc), LQCD_PK_LINK(1, 0), false);
    psi = load_f16_unscaled(in, nb[3], sc);
    hop_packed<1, BS, false>(acc, psi, LQCD_SP(sc), LQCD_PK_LINK(1, 1), false);
    psi = load_f16_unscaled(in, nb[4], sc);
    cp_async_wait<1>();
    hop_packed<2, FS, true>(acc, psi, LQCD_SP(sc), LQCD_PK_LINK(2, 0), false);
    psi = load_f16_unscaled(in, nb[5], sc);
    hop_packed<2, BS, false>(acc, psi, LQCD_SP(sc), LQCD_PK_LINK(2, 1), false);
    psi = load_f16_unscaled(in, nb[6], sc);
    cp_async_wait<0>();
    hop_packed<3, FS, true>(acc, psi, sc, LQCD_PK_LINK(3, 0), antip && tf);
    psi = load_f16_unscaled(in, nb[7], sc);
    hop_packed<3, BS, false>(acc, psi, sc, LQCD_PK_LINK(3, 1), antip && tb);
#undef LQCD_PK_LINK
#undef LQCD_SP
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

} // namespace lqcd
