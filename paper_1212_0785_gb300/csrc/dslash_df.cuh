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

// acc += k v with k in {+1, -1, +i, -i} (kind 0..3); FIRST: acc = k v
template <int KIND, bool FIRST>
__device__ __forceinline__ void acc_c(DfAcc &ar, DfAcc &ai, const Cx<Df> &v)
{
    const Df r = KIND == 0 ? v.re : KIND == 1 ? -v.re : KIND == 2 ? -v.im : v.im;
    const Df i = KIND == 0 ? v.im : KIND == 1 ? -v.im : KIND == 2 ? v.re : -v.re;
    if (FIRST) {
        ar.set(r);
        ai.set(i);
    } else {
        ar.add(r);
        ai.add(i);
    }
}

// rows 2, 3 of (1 + S gamma_mu) from the projected rows (v0, v1): see the table above project()
template <int MU, int S, bool FIRST>
__device__ __forceinline__ void acc_hop(DfAcc (&ar)[4], DfAcc (&ai)[4], const Cx<Df> &v0, const Cx<Df> &v1)
{
    acc_c<0, FIRST>(ar[0], ai[0], v0);
    acc_c<0, FIRST>(ar[1], ai[1], v1);
    constexpr int MI = S > 0 ? 3 : 2; // -S i
    constexpr int PI = S > 0 ? 2 : 3; // +S i
    constexpr int P1 = S > 0 ? 0 : 1; // +S
    constexpr int M1 = S > 0 ? 1 : 0; // -S
    if (MU == 0) {
        acc_c<MI, FIRST>(ar[2], ai[2], v1);
        acc_c<MI, FIRST>(ar[3], ai[3], v0);
    } else if (MU == 1) {
        acc_c<P1, FIRST>(ar[2], ai[2], v1);
        acc_c<M1, FIRST>(ar[3], ai[3], v0);
    } else if (MU == 2) {
        acc_c<MI, FIRST>(ar[2], ai[2], v0);
        acc_c<PI, FIRST>(ar[3], ai[3], v1);
    } else {
        acc_c<P1, FIRST>(ar[2], ai[2], v0);
        acc_c<P1, FIRST>(ar[3], ai[3], v1);
    }
}

__device__ __forceinline__ Cx<Df> cx_add_raw(const Cx<Df> &a, const Cx<Df> &b)
{
    return Cx<Df>{df_add_raw(a.re, b.re), df_add_raw(a.im, b.im)};
}

// colour a of (1 + S gamma_mu) psi at site nb, rows 0 and 1 (the table above project())
template <int MU, int S>
__device__ __forceinline__ void project_colour_df(const SpinorRef<PREC_DF> &in, int nb, int a, Cx<Df> &h0,
                                                  Cx<Df> &h1)
{
    Cx<Df> p[4];
#pragma unroll
    for (int sp = 0; sp < 4; sp++) {
        float4 v = ldg(in.d + (size_t)(sp * 3 + a) * in.Vh + nb);
        p[sp] = Cx<Df>{Df(v.x, v.y), Df(v.z, v.w)};
    }
    // sums left unnormalised: they only enter the exact link products
    if (MU == 0) {
        h0 = cx_add_raw(p[0], s_i<S>(p[3]));
        h1 = cx_add_raw(p[1], s_i<S>(p[2]));
    } else if (MU == 1) {
        h0 = cx_add_raw(p[0], -s_1<S>(p[3]));
        h1 = cx_add_raw(p[1], s_1<S>(p[2]));
    } else if (MU == 2) {
        h0 = cx_add_raw(p[0], s_i<S>(p[2]));
        h1 = cx_add_raw(p[1], -s_i<S>(p[3]));
    } else {
        h0 = cx_add_raw(p[0], s_1<S>(p[2]));
        h1 = cx_add_raw(p[1], s_1<S>(p[3]));
    }
}

// the projected half spinors of one block: [hop][row][colour][site], hop 2 mu
// forward, 2 mu + 1 backward (48 KiB)
struct DfHalves {
    float4 h[8][2][3][DF_SITES];
};

template <int MU, int FS, int BS>
__device__ __forceinline__ void project_dir_df(DfHalves &sh, const SpinorRef<PREC_DF> &in, int x, int a, int nf,
                                               int nbk)
{
    Cx<Df> h0, h1;
    project_colour_df<MU, FS>(in, nf, a, h0, h1);
    sh.h[2 * MU][0][a][x] = df_from<Df>(h0);
    sh.h[2 * MU][1][a][x] = df_from<Df>(h1);
    project_colour_df<MU, BS>(in, nbk, a, h0, h1);
    sh.h[2 * MU + 1][0][a][x] = df_from<Df>(h0);
    sh.h[2 * MU + 1][1][a][x] = df_from<Df>(h1);
}

__device__ __forceinline__ Cx<Df> df_cx(float4 v) { return Cx<Df>{Df(v.x, v.y), Df(v.z, v.w)}; }

// Each dot product starts from its first exact product and its sums reach the
// output rows unnormalised; only the output is normalised.
template <int MU, int FS, int BS>
__device__ __forceinline__ void hop_dir_df(DfAcc (&ar)[4], DfAcc (&ai)[4], const DfHalves &sh,
                                           const GaugeRef<PREC_DF> &U, const Geo &g, int cb, int out_par, int x,
                                           int a, int nbk, bool wrap_f, bool wrap_b)
{
    const bool antip = (MU == 3) && g.t_bc < 0;
    { // forward: row a of U_mu(x)
        DfAcc r0, i0, r1, i1;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            float4 w = ldg(U.d + U.idx(MU, out_par, a * 3 + b, cb));
            Df ur(w.x, w.y), ui(w.z, w.w);
            const Cx<Df> h0 = df_cx(sh.h[2 * MU][0][b][x]), h1 = df_cx(sh.h[2 * MU][1][b][x]);
            if (b == 0) {
                r0.set_prod(ur, h0.re);
                i0.set_prod(ur, h0.im);
                r1.set_prod(ur, h1.re);
                i1.set_prod(ur, h1.im);
            } else {
                r0.add_prod(ur, h0.re);
                i0.add_prod(ur, h0.im);
                r1.add_prod(ur, h1.re);
                i1.add_prod(ur, h1.im);
            }
            r0.sub_prod(ui, h0.im);
            i0.add_prod(ui, h0.re);
            r1.sub_prod(ui, h1.im);
            i1.add_prod(ui, h1.re);
        }
        Cx<Df> v0{r0.raw(), i0.raw()}, v1{r1.raw(), i1.raw()};
        if (antip && wrap_f) {
            v0 = -v0;
            v1 = -v1;
        }
        acc_hop<MU, FS, MU == 0>(ar, ai, v0, v1);
    }
    { // backward: column a of U_mu(x - mu), conjugated
        DfAcc r0, i0, r1, i1;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            float4 w = ldg(U.d + U.idx(MU, 1 - out_par, b * 3 + a, nbk));
            Df ur(w.x, w.y), ui(w.z, w.w);
            const Cx<Df> h0 = df_cx(sh.h[2 * MU + 1][0][b][x]), h1 = df_cx(sh.h[2 * MU + 1][1][b][x]);
            if (b == 0) {
                r0.set_prod(ur, h0.re);
                i0.set_prod(ur, h0.im);
                r1.set_prod(ur, h1.re);
                i1.set_prod(ur, h1.im);
            } else {
                r0.add_prod(ur, h0.re);
                i0.add_prod(ur, h0.im);
                r1.add_prod(ur, h1.re);
                i1.add_prod(ur, h1.im);
            }
            r0.add_prod(ui, h0.im);
            i0.sub_prod(ui, h0.re);
            r1.add_prod(ui, h1.im);
            i1.sub_prod(ui, h1.re);
        }
        Cx<Df> v0{r0.raw(), i0.raw()}, v1{r1.raw(), i1.raw()};
        if (antip && wrap_b) {
            v0 = -v0;
            v1 = -v1;
        }
        acc_hop<MU, BS, false>(ar, ai, v0, v1);
    }
}

// The block body: output sites blk * DF_SITES + threadIdx.x, colour
// threadIdx.y (the kernels of dslash_df.cu and the multi-system kernels of
// batch.cu).  RESID (with XPAY): the accurate residual r = b - (x + b D in)
// is stored instead of x + b D in, each component r = b - t in float-float, and the block's partial sum of |r|^2 (leading parts) goes to
// partials[blk]: each thread adds its colour over the four spins in FP32,
// the threads' sums are added in FP64 in a fixed order.
template <bool DAG, bool XPAY, bool RESID = false>
__device__ __forceinline__ void df_hop_block(DfHalves &sh, SpinorRef<PREC_DF> out, SpinorRef<PREC_DF> in,
                                             GaugeRef<PREC_DF> U, const Geo &g, int out_par, SpinorRef<PREC_DF> x,
                                             Df b, int blk, SpinorRef<PREC_DF> bsrc = {}, double *partials = nullptr)
{
    static_assert(!RESID || XPAY, "the residual follows the last term x + b D in");
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
    if (!RESID && !live) return;
    float n2 = 0.f;
    if (live) {
        DfAcc ar[4], ai[4];
        hop_dir_df<0, FS, BS>(ar, ai, sh, U, g, cb, out_par, tx, a, nb[1], false, false);
        hop_dir_df<1, FS, BS>(ar, ai, sh, U, g, cb, out_par, tx, a, nb[3], false, false);
        hop_dir_df<2, FS, BS>(ar, ai, sh, U, g, cb, out_par, tx, a, nb[5], false, false);
        if (g.aniso) { // the spatial hops' weight of the anisotropic operator (a uniform branch)
            const Df w(g.csf, g.cs_lo);
#pragma unroll
            for (int sp = 0; sp < 4; sp++) {
                ar[sp].set(w * ar[sp].value());
                ai[sp].set(w * ai[sp].value());
            }
        }
        hop_dir_df<3, FS, BS>(ar, ai, sh, U, g, cb, out_par, tx, a, nb[7], tf, tb);
#pragma unroll
        for (int sp = 0; sp < 4; sp++) {
            Cx<Df> v{ar[sp].value(), ai[sp].value()};
            size_t k = (size_t)(sp * 3 + a) * out.Vh + cb;
            if (XPAY) {
                float4 xv = x.d[k];
                Cx<Df> xc{Df(xv.x, xv.y), Df(xv.z, xv.w)};
                v = xc + b * v;
            }
            if (RESID) {
                const float4 bv = bsrc.d[k];
                v = Cx<Df>{Df(bv.x, bv.y) - v.re, Df(bv.z, bv.w) - v.im};
                n2 += v.re.hi * v.re.hi + v.im.hi * v.im.hi;
            }
            out.d[k] = df_from<Df>(v);
        }
    }
    if (RESID) { // warps of 32 consecutive sites of one colour; warp sums added in warp order
        __shared__ double wsum[DF_SITES * 3 / 32];
        double t = n2;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
        const int lid = a * DF_SITES + tx;
        if ((lid & 31) == 0) wsum[lid >> 5] = t;
        __syncthreads();
        if (lid == 0) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < DF_SITES * 3 / 32; w++) s += wsum[w];
            partials[blk] = s;
        }
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

} // namespace lqcd
