// dslash.cu -- even-odd Wilson hopping term D_eo / D_oe on the device.
//
// One thread per output site (the paper's one-site-per-thread mapping, Sec. 3),
// fields in site-coalesced structure-of-arrays layout so that a warp's loads
// of one component are contiguous.  For each of the 8 hops the neighbour
// spinor is projected to a half spinor with (1 -+ gamma_mu) (DeGrand-Rossi
// basis: two spin components carry all the information), multiplied by the
// link (or its adjoint) and reconstructed into the accumulator.  The fermion
// boundary factor is applied to the half spinor of a hop across the t
// boundary, never to the links, so 12-real compressed links stay in SU(3).
//
// FP64 storage uses FP64 arithmetic; FP32, FP16+norm and BF16 storage use
// FP32 arithmetic with 12-real links (row 2 = conj(row0 x row1)).
#include "df64.cuh"
#include "dslash.cuh"
#include "dslash_site.cuh"

namespace lqcd {

// ---------------------------------------------------------------- kernels

template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG>
__global__ void __launch_bounds__(DS_BLOCK) dslash_plain_kernel(SpinorRef<SP> out, SpinorRef<SP> in, GaugeRef<GP> U,
                                                                 Geo g, int out_par, const int *skip)
{
    if (skip && *skip) return;
    int cb = blockIdx.x * DS_BLOCK + threadIdx.x;
    if (cb >= g.Vh) return;
    out.store(cb, dslash_site<R, SP, GP, DAG>(in, U, g, cb, out_par));
}

template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG>
__global__ void __launch_bounds__(DS_BLOCK) dslash_xpay_kernel(SpinorRef<SP> out, SpinorRef<SP> in, GaugeRef<GP> U,
                                                                Geo g, int out_par, SpinorRef<SP> x, R b,
                                                                double *partials, int nblocks, const int *skip)
{
    if (skip && *skip) return;
    int cb = blockIdx.x * DS_BLOCK + threadIdx.x;
    R n2 = R(0);
    if (cb < g.Vh) {
        Sp<R> d = dslash_site<R, SP, GP, DAG>(in, U, g, cb, out_par);
        Sp<R> xv = x.template load_rw<R>(cb);
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int k = 0; k < 3; k++) d.c[a][k] = xv.c[a][k] + b * d.c[a][k];
        out.store(cb, d);
        n2 = sp_norm2(d);
    }
    if (partials) block_sum_store_wp<DS_BLOCK>(n2, partials);
}

template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG, lqcd_prec XP>
__global__ void __launch_bounds__(DS_BLOCK) dslash_cg_kernel(SpinorRef<SP> in, GaugeRef<GP> U, Geo g, int out_par,
                                                              SpinorRef<SP> t, R b, SpinorRef<XP> xs, SpinorRef<SP> r,
                                                              SpinorRef<SP> p, double *partials, int nblocks,
                                                              const CgScalars *sc)
{
    if (sc->pause) return;
    const R alpha = (R)sc->alpha;
    int cb = blockIdx.x * DS_BLOCK + threadIdx.x;
    R n2 = R(0);
    if (cb < g.Vh) {
        Sp<R> ap = dslash_site<R, SP, GP, DAG>(in, U, g, cb, out_par);
        {
            Sp<R> tv = t.template load_rw<R>(cb);
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int k = 0; k < 3; k++) ap.c[a][k] = tv.c[a][k] + b * ap.c[a][k];
        }
        Sp<R> pv = p.template load_rw<R>(cb);
        {
            using RX = typename std::conditional<XP == LQCD_F64, double, float>::type;
            Sp<RX> xv = xs.template load_rw<RX>(cb);
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    xv.c[a][k].re += (RX)alpha * (RX)pv.c[a][k].re;
                    xv.c[a][k].im += (RX)alpha * (RX)pv.c[a][k].im;
                }
            xs.store(cb, xv);
        }
        Sp<R> rv = r.template load_rw<R>(cb);
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int k = 0; k < 3; k++) rv.c[a][k] = rv.c[a][k] - alpha * ap.c[a][k];
        r.store(cb, rv);
        n2 = sp_norm2(rv);
    }
    block_sum_store_wp<DS_BLOCK>(n2, partials);
}

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

// acc += k v with k in {+1, -1, +i, -i} (kind 0..3)
template <int KIND>
__device__ __forceinline__ void acc_c(DfAcc &ar, DfAcc &ai, const Cx<Df> &v)
{
    if (KIND == 0) {
        ar.add(v.re);
        ai.add(v.im);
    } else if (KIND == 1) {
        ar.add(-v.re);
        ai.add(-v.im);
    } else if (KIND == 2) { // +i v = (-im, re)
        ar.add(-v.im);
        ai.add(v.re);
    } else { // -i v = (im, -re)
        ar.add(v.im);
        ai.add(-v.re);
    }
}

// rows 2, 3 of (1 + S gamma_mu) from the projected rows (v0, v1): see the table above project()
template <int MU, int S>
__device__ __forceinline__ void acc_hop(DfAcc (&ar)[4], DfAcc (&ai)[4], const Cx<Df> &v0, const Cx<Df> &v1)
{
    acc_c<0>(ar[0], ai[0], v0);
    acc_c<0>(ar[1], ai[1], v1);
    constexpr int MI = S > 0 ? 3 : 2; // -S i
    constexpr int PI = S > 0 ? 2 : 3; // +S i
    constexpr int P1 = S > 0 ? 0 : 1; // +S
    constexpr int M1 = S > 0 ? 1 : 0; // -S
    if (MU == 0) {
        acc_c<MI>(ar[2], ai[2], v1);
        acc_c<MI>(ar[3], ai[3], v0);
    } else if (MU == 1) {
        acc_c<P1>(ar[2], ai[2], v1);
        acc_c<M1>(ar[3], ai[3], v0);
    } else if (MU == 2) {
        acc_c<MI>(ar[2], ai[2], v0);
        acc_c<PI>(ar[3], ai[3], v1);
    } else {
        acc_c<P1>(ar[2], ai[2], v0);
        acc_c<P1>(ar[3], ai[3], v1);
    }
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
    if (MU == 0) {
        h0 = p[0] + s_i<S>(p[3]);
        h1 = p[1] + s_i<S>(p[2]);
    } else if (MU == 1) {
        h0 = p[0] - s_1<S>(p[3]);
        h1 = p[1] + s_1<S>(p[2]);
    } else if (MU == 2) {
        h0 = p[0] + s_i<S>(p[2]);
        h1 = p[1] - s_i<S>(p[3]);
    } else {
        h0 = p[0] + s_1<S>(p[2]);
        h1 = p[1] + s_1<S>(p[3]);
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
            r0.add_prod(ur, h0.re);
            r0.sub_prod(ui, h0.im);
            i0.add_prod(ur, h0.im);
            i0.add_prod(ui, h0.re);
            r1.add_prod(ur, h1.re);
            r1.sub_prod(ui, h1.im);
            i1.add_prod(ur, h1.im);
            i1.add_prod(ui, h1.re);
        }
        Cx<Df> v0{r0.value(), i0.value()}, v1{r1.value(), i1.value()};
        if (antip && wrap_f) {
            v0 = -v0;
            v1 = -v1;
        }
        acc_hop<MU, FS>(ar, ai, v0, v1);
    }
    { // backward: column a of U_mu(x - mu), conjugated
        DfAcc r0, i0, r1, i1;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            float4 w = ldg(U.d + U.idx(MU, 1 - out_par, b * 3 + a, nbk));
            Df ur(w.x, w.y), ui(w.z, w.w);
            const Cx<Df> h0 = df_cx(sh.h[2 * MU + 1][0][b][x]), h1 = df_cx(sh.h[2 * MU + 1][1][b][x]);
            r0.add_prod(ur, h0.re);
            r0.add_prod(ui, h0.im);
            i0.add_prod(ur, h0.im);
            i0.sub_prod(ui, h0.re);
            r1.add_prod(ur, h1.re);
            r1.add_prod(ui, h1.im);
            i1.add_prod(ur, h1.im);
            i1.sub_prod(ui, h1.re);
        }
        Cx<Df> v0{r0.value(), i0.value()}, v1{r1.value(), i1.value()};
        if (antip && wrap_b) {
            v0 = -v0;
            v1 = -v1;
        }
        acc_hop<MU, BS>(ar, ai, v0, v1);
    }
}

// 4 blocks of 192 threads per SM (80 registers, 4 x 48 KiB of half spinors)
template <bool DAG, bool XPAY>
__global__ void __launch_bounds__(DF_SITES * 3, 4) dslash_df_kernel(SpinorRef<PREC_DF> out, SpinorRef<PREC_DF> in,
                                                                 GaugeRef<PREC_DF> U, Geo g, int out_par,
                                                                 SpinorRef<PREC_DF> x, Df b, const int *skip)
{
    __shared__ DfHalves sh;
    if (skip && *skip) return; // the same for the whole block
    const int tx = threadIdx.x, a = threadIdx.y;
    const int cb = blockIdx.x * DF_SITES + tx;
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
    DfAcc ar[4], ai[4];
    hop_dir_df<0, FS, BS>(ar, ai, sh, U, g, cb, out_par, tx, a, nb[1], false, false);
    hop_dir_df<1, FS, BS>(ar, ai, sh, U, g, cb, out_par, tx, a, nb[3], false, false);
    hop_dir_df<2, FS, BS>(ar, ai, sh, U, g, cb, out_par, tx, a, nb[5], false, false);
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
        out.d[k] = df_from<Df>(v);
    }
}

static lqcd_status launch_df(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger,
                             const lqcd_field *x, double b, const int *skip, cudaStream_t s)
{
    Geo g = make_geo(in->lat);
    dim3 block(DF_SITES, 3), grid(nblocks_for(g.Vh, DF_SITES));
    SpinorRef<PREC_DF> xr = x ? spinor_ref<PREC_DF>(x) : SpinorRef<PREC_DF>{nullptr, g.Vh};
    int op = out->kind == LQCD_SPINOR_EVEN ? 0 : 1;
    Df bd(b);
    if (x) {
        if (dagger)
            dslash_df_kernel<true, true><<<grid, block, 0, s>>>(spinor_ref<PREC_DF>(out), spinor_ref<PREC_DF>(in),
                                                                 gauge_ref<PREC_DF>(U), g, op, xr, bd, skip);
        else
            dslash_df_kernel<false, true><<<grid, block, 0, s>>>(spinor_ref<PREC_DF>(out), spinor_ref<PREC_DF>(in),
                                                                  gauge_ref<PREC_DF>(U), g, op, xr, bd, skip);
    } else {
        if (dagger)
            dslash_df_kernel<true, false><<<grid, block, 0, s>>>(spinor_ref<PREC_DF>(out), spinor_ref<PREC_DF>(in),
                                                                  gauge_ref<PREC_DF>(U), g, op, xr, bd, skip);
        else
            dslash_df_kernel<false, false><<<grid, block, 0, s>>>(spinor_ref<PREC_DF>(out), spinor_ref<PREC_DF>(in),
                                                                   gauge_ref<PREC_DF>(U), g, op, xr, bd, skip);
    }
    return LQCD_OK;
}

// ---------------------------------------------------------------- dispatch

static int out_parity(const lqcd_field *f) { return f->kind == LQCD_SPINOR_EVEN ? 0 : 1; }

static lqcd_status check_pair(const lqcd_field *out, const lqcd_field *U, const lqcd_field *in)
{
    LQCD_REQUIRE(out && U && in, "dslash: NULL field");
    LQCD_REQUIRE(U->kind == LQCD_GAUGE, "dslash: U is not a gauge field");
    LQCD_REQUIRE((in->kind == LQCD_SPINOR_EVEN && out->kind == LQCD_SPINOR_ODD) ||
                     (in->kind == LQCD_SPINOR_ODD && out->kind == LQCD_SPINOR_EVEN),
                 "dslash: in/out must be half spinors of opposite parity");
    LQCD_REQUIRE(same_lattice(U->lat, in->lat) && same_lattice(U->lat, out->lat), "dslash: lattices differ");
    LQCD_REQUIRE(in->prec == out->prec, "dslash: in/out precisions differ");
    LQCD_REQUIRE(U->prec == in->prec || (U->prec == LQCD_F64 && in->prec == LQCD_F32),
                 "dslash: link precision %d does not match spinor precision %d", (int)U->prec, (int)in->prec);
    return LQCD_OK;
}

template <lqcd_prec P>
struct ArithOf {
    using type = float;
};
template <>
struct ArithOf<LQCD_F64> {
    using type = double;
};
template <>
struct ArithOf<PREC_DF> {
    using type = Df;
};

template <lqcd_prec P, lqcd_prec GP = P>
static void launch_plain(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger, const int *skip,
                         cudaStream_t s)
{
    using R = typename ArithOf<P>::type;
    Geo g = make_geo(in->lat);
    int nb = dslash_blocks(g.Vh);
    if (dagger)
        dslash_plain_kernel<R, P, GP, true><<<nb, DS_BLOCK, 0, s>>>(spinor_ref<P>(out), spinor_ref<P>(in),
                                                                    gauge_ref<GP>(U), g, out_parity(out), skip);
    else
        dslash_plain_kernel<R, P, GP, false><<<nb, DS_BLOCK, 0, s>>>(spinor_ref<P>(out), spinor_ref<P>(in),
                                                                     gauge_ref<GP>(U), g, out_parity(out), skip);
}

template <lqcd_prec P, lqcd_prec GP = P>
static void launch_xpay(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger, const lqcd_field *x,
                        double b, double *partials, const int *skip, cudaStream_t s)
{
    using R = typename ArithOf<P>::type;
    Geo g = make_geo(in->lat);
    int nb = dslash_blocks(g.Vh);
    if (dagger)
        dslash_xpay_kernel<R, P, GP, true><<<nb, DS_BLOCK, 0, s>>>(spinor_ref<P>(out), spinor_ref<P>(in),
                                                                   gauge_ref<GP>(U), g, out_parity(out),
                                                                   spinor_ref<P>(x), (R)b, partials, nb, skip);
    else
        dslash_xpay_kernel<R, P, GP, false><<<nb, DS_BLOCK, 0, s>>>(spinor_ref<P>(out), spinor_ref<P>(in),
                                                                    gauge_ref<GP>(U), g, out_parity(out),
                                                                    spinor_ref<P>(x), (R)b, partials, nb, skip);
}

template <lqcd_prec P, lqcd_prec XP>
static void launch_cg(const lqcd_field *U, const lqcd_field *in, int dagger, const lqcd_field *t, double b,
                      lqcd_field *xs, lqcd_field *r, const lqcd_field *p, double *partials, const CgScalars *sc,
                      cudaStream_t s)
{
    using R = typename ArithOf<P>::type;
    Geo g = make_geo(in->lat);
    int nb = dslash_blocks(g.Vh);
    int op = out_parity(t);
    if (dagger)
        dslash_cg_kernel<R, P, P, true, XP><<<nb, DS_BLOCK, 0, s>>>(spinor_ref<P>(in), gauge_ref<P>(U), g, op,
                                                                    spinor_ref<P>(t), (R)b, spinor_ref<XP>(xs),
                                                                    spinor_ref<P>(r), spinor_ref<P>(p), partials, nb, sc);
    else
        dslash_cg_kernel<R, P, P, false, XP><<<nb, DS_BLOCK, 0, s>>>(spinor_ref<P>(in), gauge_ref<P>(U), g, op,
                                                                     spinor_ref<P>(t), (R)b, spinor_ref<XP>(xs),
                                                                     spinor_ref<P>(r), spinor_ref<P>(p), partials, nb, sc);
}

lqcd_status dslash_plain(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger, const int *skip,
                         cudaStream_t s)
{
    LQCD_TRY(check_pair(out, U, in));
    double site = 8 * link_bytes(U->prec) + 2 * spinor_site_bytes(in->prec);
    KernelTimer kt(dslash_class(in->prec), s, site * in->Vh);
    switch (in->prec) {
    case LQCD_F64: launch_plain<LQCD_F64>(out, U, in, dagger, skip, s); break;
    case LQCD_F32:
        if (U->prec == LQCD_F64)
            launch_plain<LQCD_F32, LQCD_F64>(out, U, in, dagger, skip, s);
        else
            launch_plain<LQCD_F32>(out, U, in, dagger, skip, s);
        break;
    case LQCD_F16N: launch_plain<LQCD_F16N>(out, U, in, dagger, skip, s); break;
    case LQCD_BF16: launch_plain<LQCD_BF16>(out, U, in, dagger, skip, s); break;
    default: launch_df(out, U, in, dagger, nullptr, 0.0, skip, s); break;
    }
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status dslash_xpay(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger, const lqcd_field *x,
                        double b, double *partials, const int *skip, cudaStream_t s)
{
    LQCD_TRY(check_pair(out, U, in));
    LQCD_REQUIRE(x && x->kind == out->kind && x->prec == out->prec, "dslash_xpay: x must match out");
    double site = 8 * link_bytes(U->prec) + 3 * spinor_site_bytes(in->prec); // + read of x
    KernelTimer kt(dslash_class(in->prec), s, site * in->Vh);
    switch (in->prec) {
    case LQCD_F64: launch_xpay<LQCD_F64>(out, U, in, dagger, x, b, partials, skip, s); break;
    case LQCD_F32:
        if (U->prec == LQCD_F64)
            launch_xpay<LQCD_F32, LQCD_F64>(out, U, in, dagger, x, b, partials, skip, s);
        else
            launch_xpay<LQCD_F32>(out, U, in, dagger, x, b, partials, skip, s);
        break;
    case LQCD_F16N: launch_xpay<LQCD_F16N>(out, U, in, dagger, x, b, partials, skip, s); break;
    case LQCD_BF16: launch_xpay<LQCD_BF16>(out, U, in, dagger, x, b, partials, skip, s); break;
    default:
        LQCD_REQUIRE(partials == nullptr, "float-float hopping term has no norm reduction");
        launch_df(out, U, in, dagger, x, b, skip, s);
        break;
    }
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status dslash_cg(const lqcd_field *U, const lqcd_field *in, int dagger, const lqcd_field *t, double b,
                      lqcd_field *xs, lqcd_field *r, const lqcd_field *p, double *partials, const CgScalars *sc,
                      cudaStream_t s)
{
    // links, input; reads of t, p, r and xs; writes of r and xs (no output of the product)
    double site = 8 * link_bytes(U->prec) + 4 * spinor_site_bytes(in->prec) + spinor_site_bytes(r->prec) +
                  2 * spinor_site_bytes(xs->prec);
    KernelTimer kt(dslash_class(in->prec), s, site * in->Vh);
    switch (in->prec) {
    case LQCD_F64: launch_cg<LQCD_F64, LQCD_F64>(U, in, dagger, t, b, xs, r, p, partials, sc, s); break;
    case LQCD_F32: launch_cg<LQCD_F32, LQCD_F32>(U, in, dagger, t, b, xs, r, p, partials, sc, s); break;
    case LQCD_F16N: launch_cg<LQCD_F16N, LQCD_F32>(U, in, dagger, t, b, xs, r, p, partials, sc, s); break;
    case LQCD_BF16: launch_cg<LQCD_BF16, LQCD_F32>(U, in, dagger, t, b, xs, r, p, partials, sc, s); break;
    }
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status mhat_apply(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, double kappa, int dagger,
                       lqcd_field *tmp_odd, double *partials, cudaStream_t s)
{
    LQCD_TRY(dslash_plain(tmp_odd, U, in, dagger, nullptr, s));
    return dslash_xpay(out, U, tmp_odd, dagger, in, -kappa * kappa, partials, nullptr, s);
}

} // namespace lqcd

using namespace lqcd;

extern "C" {

lqcd_status lqcd_dslash(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger, void *stream)
{
    return dslash_plain(out, U, in, dagger, nullptr, (cudaStream_t)stream);
}

lqcd_status lqcd_mhat(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, double kappa, int dagger,
                      void *stream)
{
    LQCD_REQUIRE(out && U && in, "mhat: NULL field");
    LQCD_REQUIRE(out->kind == LQCD_SPINOR_EVEN && in->kind == LQCD_SPINOR_EVEN, "mhat: in/out must be EVEN spinors");
    LQCD_REQUIRE(out != in, "mhat: out must differ from in");
    FieldPtr tmp;
    LQCD_TRY(lqcd_field_alloc(&in->lat, LQCD_SPINOR_ODD, in->prec, 0, &tmp.f));
    LQCD_TRY(mhat_apply(out, U, in, kappa, dagger, tmp.f, nullptr, (cudaStream_t)stream));
    // the temporary is freed on return: finish the work that reads it first
    LQCD_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return LQCD_OK;
}

} // extern "C"
