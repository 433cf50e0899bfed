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
#include "spin.cuh"

namespace lqcd {

// one direction: forward hop with (1 + FS gamma), backward with (1 + BS gamma)
template <int MU, int FS, int BS, typename R, lqcd_prec SP, lqcd_prec GP>
__device__ __forceinline__ void hop_dir(Sp<R> &acc, const SpinorRef<SP> &in, const GaugeRef<GP> &U, const Geo &g,
                                        const int c[4], int cb, int out_par)
{
    const int in_par = 1 - out_par;
    {   // forward: U_mu(x) psi(x + mu)
        int cf[4] = {c[0], c[1], c[2], c[3]};
        bool wrap = (c[MU] + 1 == g.L[MU]);
        cf[MU] = wrap ? 0 : c[MU] + 1;
        Sp<R> psi = in.template load<R>(coords_cb(g, cf));
        Hs<R> h = project<MU, FS>(psi);
        M3<R> u = U.template load<R>(MU, out_par, cb);
        Hs<R> uh = mul_link(u, h);
        if (MU == 3 && wrap && g.t_bc < 0) negate(uh);
        accumulate<MU, FS>(acc, uh);
    }
    {   // backward: U_mu(x - mu)^dag psi(x - mu)
        int cbk[4] = {c[0], c[1], c[2], c[3]};
        bool wrap = (c[MU] == 0);
        cbk[MU] = wrap ? g.L[MU] - 1 : c[MU] - 1;
        int nb = coords_cb(g, cbk);
        Sp<R> psi = in.template load<R>(nb);
        Hs<R> h = project<MU, BS>(psi);
        M3<R> u = U.template load<R>(MU, in_par, nb);
        Hs<R> uh = mul_link_dag(u, h);
        if (MU == 3 && wrap && g.t_bc < 0) negate(uh);
        accumulate<MU, BS>(acc, uh);
    }
}

template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG>
__device__ __forceinline__ Sp<R> dslash_site(const SpinorRef<SP> &in, const GaugeRef<GP> &U, const Geo &g, int cb,
                                             int out_par)
{
    int c[4];
    cb_coords(g, cb, out_par, c);
    Sp<R> acc = sp_zero<R>();
    // D: (1 - gamma) forward, (1 + gamma) backward; D^dag swaps them
    constexpr int FS = DAG ? +1 : -1;
    constexpr int BS = -FS;
    hop_dir<0, FS, BS, R>(acc, in, U, g, c, cb, out_par);
    hop_dir<1, FS, BS, R>(acc, in, U, g, c, cb, out_par);
    hop_dir<2, FS, BS, R>(acc, in, U, g, c, cb, out_par);
    hop_dir<3, FS, BS, R>(acc, in, U, g, c, cb, out_par);
    return acc;
}

template <typename R>
__device__ __forceinline__ double sp_norm2(const Sp<R> &s)
{
    double n = 0;
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) n += (double)norm2(s.c[a][b]);
    return n;
}

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
    double n2[1] = {0.0};
    if (cb < g.Vh) {
        Sp<R> d = dslash_site<R, SP, GP, DAG>(in, U, g, cb, out_par);
        Sp<R> xv = x.template load_rw<R>(cb);
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int k = 0; k < 3; k++) d.c[a][k] = xv.c[a][k] + b * d.c[a][k];
        out.store(cb, d);
        n2[0] = sp_norm2(d);
    }
    if (partials) block_sum_store<1, DS_BLOCK>(n2, partials, nblocks);
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
    double n2[1] = {0.0};
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
        n2[0] = sp_norm2(rv);
    }
    block_sum_store<1, DS_BLOCK>(n2, partials, nblocks);
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
    KernelTimer kt(dslash_class(in->prec), s);
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
    default: launch_plain<PREC_DF>(out, U, in, dagger, skip, s); break;
    }
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status dslash_xpay(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger, const lqcd_field *x,
                        double b, double *partials, const int *skip, cudaStream_t s)
{
    LQCD_TRY(check_pair(out, U, in));
    LQCD_REQUIRE(x && x->kind == out->kind && x->prec == out->prec, "dslash_xpay: x must match out");
    KernelTimer kt(dslash_class(in->prec), s);
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
    default: launch_xpay<PREC_DF>(out, U, in, dagger, x, b, partials, skip, s); break;
    }
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status dslash_cg(const lqcd_field *U, const lqcd_field *in, int dagger, const lqcd_field *t, double b,
                      lqcd_field *xs, lqcd_field *r, const lqcd_field *p, double *partials, const CgScalars *sc,
                      cudaStream_t s)
{
    KernelTimer kt(dslash_class(in->prec), s);
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
