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
#include <atomic>

#include "df64.cuh"
#include "dslash.cuh"
#include "dslash_packed.cuh"
#include "dslash_site.cuh"
#include "tune.cuh"

namespace lqcd {

// ---------------------------------------------------------------- kernels

// Sp of D in at site cb.  FORM 1 (FP16+norm): the thread prefetches its
// links into shared memory first; FORM 2 (FP16+norm): the same with packed
// FP32x2 arithmetic.  FORM 0: every operand gathered by its thread.  (The
// other precisions' FORM 1, 2 instances are never launched.)
template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG, int FORM, int BLOCK = DS_BLOCK>
__device__ __forceinline__ Sp<R> site_value(const SpinorRef<SP> &in, const GaugeRef<GP> &U, const Geo &g, int cb,
                                            int out_par)
{
    if constexpr (FORM == 1 && SP == LQCD_F16N && GP == LQCD_F16N)
        return prefetch_site<R, DAG>(in, U, g, cb, out_par);
    else if constexpr (FORM == 2 && SP == LQCD_F16N && GP == LQCD_F16N && std::is_same<R, float>::value)
        return packed_site<DAG, BLOCK>(in, U, g, cb, out_par);
    else
        return dslash_site<R, SP, GP, DAG>(in, U, g, cb, out_par);
}

// (BLOCK: threads per block of the launch; 128 except for the tuned packed kernels)
template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG, int FORM, int BLOCK = DS_BLOCK>
__device__ __forceinline__ void plain_body(SpinorRef<SP> out, SpinorRef<SP> in, GaugeRef<GP> U,
                                                                 Geo g, int out_par, const int *skip)
{
    if (skip && *skip) return;
    int cb = blockIdx.x * BLOCK + threadIdx.x;
    if (cb >= g.Vh) return;
    if constexpr (FORM == 2 && SP == LQCD_F16N && GP == LQCD_F16N && std::is_same<R, float>::value)
        store_packed(out, cb, packed_acc<DAG, BLOCK>(in, U, g, cb, out_par));
    else
        out.store(cb, site_value<R, SP, GP, DAG, FORM, BLOCK>(in, U, g, cb, out_par));
}

template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG, int FORM, int BLOCK = DS_BLOCK>
__device__ __forceinline__ void xpay_body(SpinorRef<SP> out, SpinorRef<SP> in, GaugeRef<GP> U,
                                                                Geo g, int out_par, SpinorRef<SP> x, R b,
                                                                double *partials, int nblocks, const int *skip,
                                                                CgScalars *fin)
{
    if (skip && *skip) return;
    int cb = blockIdx.x * BLOCK + threadIdx.x;
    R n2 = R(0);
    if (cb < g.Vh) {
        Sp<R> d = site_value<R, SP, GP, DAG, FORM, BLOCK>(in, U, g, cb, out_par);
        Sp<R> xv = x.template load_rw<R>(cb);
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int k = 0; k < 3; k++) d.c[a][k] = xv.c[a][k] + b * d.c[a][k];
        out.store(cb, d);
        n2 = sp_norm2(d);
    }
    if (partials) {
        block_sum_store_wp<BLOCK>(n2, partials);
        if (fin) cg_finish<BLOCK, false>(fin, partials, nblocks);
    }
}

template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG, lqcd_prec XP, int FORM, int BLOCK = DS_BLOCK>
__device__ __forceinline__ void cg_body(SpinorRef<SP> in, GaugeRef<GP> U, Geo g, int out_par,
                                                              SpinorRef<SP> t, R b, SpinorRef<XP> xs, SpinorRef<SP> r,
                                                              SpinorRef<SP> p, double *partials, int nblocks,
                                                              CgScalars *sc)
{
    if (sc->pause) return;
    const R alpha = (R)sc->alpha;
    int cb = blockIdx.x * BLOCK + threadIdx.x;
    R n2 = R(0);
    if (cb < g.Vh) {
        Sp<R> ap = site_value<R, SP, GP, DAG, FORM, BLOCK>(in, U, g, cb, out_par);
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
    block_sum_store_wp<BLOCK>(n2, partials);
    cg_finish<BLOCK, true>(sc, partials, nblocks);
}

// The kernels: gathered operands, and (FP16+norm) prefetched links with the
// same bodies (7 blocks of 128 per SM, 24 KiB of shared memory each).
template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG>
__global__ void __launch_bounds__(DS_BLOCK) dslash_plain_kernel(SpinorRef<SP> out, SpinorRef<SP> in, GaugeRef<GP> U,
                                                                 Geo g, int out_par, const int *skip)
{
    plain_body<R, SP, GP, DAG, 0>(out, in, U, g, out_par, skip);
}
template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG>
__global__ void __launch_bounds__(DS_BLOCK) dslash_xpay_kernel(SpinorRef<SP> out, SpinorRef<SP> in, GaugeRef<GP> U,
                                                                Geo g, int out_par, SpinorRef<SP> x, R b,
                                                                double *partials, int nblocks, const int *skip,
                                                                CgScalars *fin)
{
    xpay_body<R, SP, GP, DAG, 0>(out, in, U, g, out_par, x, b, partials, nblocks, skip, fin);
}
template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG, lqcd_prec XP>
__global__ void __launch_bounds__(DS_BLOCK) dslash_cg_kernel(SpinorRef<SP> in, GaugeRef<GP> U, Geo g, int out_par,
                                                              SpinorRef<SP> t, R b, SpinorRef<XP> xs, SpinorRef<SP> r,
                                                              SpinorRef<SP> p, double *partials, int nblocks,
                                                              CgScalars *sc)
{
    cg_body<R, SP, GP, DAG, XP, 0>(in, U, g, out_par, t, b, xs, r, p, partials, nblocks, sc);
}

template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG>
__global__ void __launch_bounds__(DS_BLOCK, 7) dslash_plain_prefetch_kernel(SpinorRef<SP> out, SpinorRef<SP> in,
                                                                             GaugeRef<GP> U, Geo g, int out_par,
                                                                             const int *skip)
{
    plain_body<R, SP, GP, DAG, 1>(out, in, U, g, out_par, skip);
}
template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG>
__global__ void __launch_bounds__(DS_BLOCK, 7) dslash_xpay_prefetch_kernel(SpinorRef<SP> out, SpinorRef<SP> in,
                                                                            GaugeRef<GP> U, Geo g, int out_par,
                                                                            SpinorRef<SP> x, R b, double *partials,
                                                                            int nblocks, const int *skip,
                                                                            CgScalars *fin)
{
    xpay_body<R, SP, GP, DAG, 1>(out, in, U, g, out_par, x, b, partials, nblocks, skip, fin);
}
template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG, lqcd_prec XP>
__global__ void __launch_bounds__(DS_BLOCK, 7) dslash_cg_prefetch_kernel(SpinorRef<SP> in, GaugeRef<GP> U, Geo g,
                                                                          int out_par, SpinorRef<SP> t, R b,
                                                                          SpinorRef<XP> xs, SpinorRef<SP> r,
                                                                          SpinorRef<SP> p, double *partials,
                                                                          int nblocks, CgScalars *sc)
{
    cg_body<R, SP, GP, DAG, XP, 1>(in, U, g, out_par, t, b, xs, r, p, partials, nblocks, sc);
}

// The packed form with BLOCK threads per block (64, 128 or 256, chosen per
// lattice by the autotuner), register budgets per SM whatever the block size:
// 640 threads for the plain variant (96 registers at 128 per block, where the
// compiler keeps more neighbour loads in flight) and 768 for the reducing
// variants (80 registers; their block sums want the extra warps).  Measured
// on the 32^3x64 trajectory against the earlier 896 for all three: plain
// 185.5 -> 178.8 ms, reducing 282 -> 277 ms per trajectory; 512 for all
// three, or 640 for the reducing ones, was slower.
constexpr int PK_THREADS_PLAIN = 640, PK_THREADS_REDUCING = 768;
template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG, int BLOCK>
__global__ void __launch_bounds__(BLOCK, PK_THREADS_PLAIN / BLOCK) dslash_plain_packed_kernel(SpinorRef<SP> out, SpinorRef<SP> in,
                                                                                  GaugeRef<GP> U, Geo g, int out_par,
                                                                                  const int *skip)
{
    plain_body<R, SP, GP, DAG, 2, BLOCK>(out, in, U, g, out_par, skip);
}
template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG, int BLOCK>
__global__ void __launch_bounds__(BLOCK, PK_THREADS_REDUCING / BLOCK) dslash_xpay_packed_kernel(SpinorRef<SP> out, SpinorRef<SP> in,
                                                                                 GaugeRef<GP> U, Geo g, int out_par,
                                                                                 SpinorRef<SP> x, R b, double *partials,
                                                                                 int nblocks, const int *skip,
                                                                                 CgScalars *fin)
{
    xpay_body<R, SP, GP, DAG, 2, BLOCK>(out, in, U, g, out_par, x, b, partials, nblocks, skip, fin);
}
template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG, lqcd_prec XP, int BLOCK>
__global__ void __launch_bounds__(BLOCK, PK_THREADS_REDUCING / BLOCK) dslash_cg_packed_kernel(SpinorRef<SP> in, GaugeRef<GP> U, Geo g,
                                                                               int out_par, SpinorRef<SP> t, R b,
                                                                               SpinorRef<XP> xs, SpinorRef<SP> r,
                                                                               SpinorRef<SP> p, double *partials,
                                                                               int nblocks, CgScalars *sc)
{
    cg_body<R, SP, GP, DAG, XP, 2, BLOCK>(in, U, g, out_par, t, b, xs, r, p, partials, nblocks, sc);
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

// the FP16+norm form: 2 prefetched links with packed FP32x2 arithmetic
// (default), 1 prefetched links, 0 gathered
static std::atomic<int> g_form{2};

template <lqcd_prec P, lqcd_prec GP>
static int use_form(const Geo &)
{
    if (P != LQCD_F16N || GP != LQCD_F16N) return 0;
    return g_form.load(std::memory_order_relaxed);
}

// launch kernel K in the form chosen by use_form
#define LQCD_LAUNCH_FORM(form, kern, targs, grid, args)                                                              \
    do {                                                                                                             \
        if (form == 1)                                                                                               \
            kern##_prefetch_kernel<LQCD_UNPAREN targs><<<grid, DS_BLOCK, 0, s>>> args;                               \
        else                                                                                                         \
            kern##_kernel<LQCD_UNPAREN targs><<<grid, DS_BLOCK, 0, s>>> args;                                        \
    } while (0)
#define LQCD_UNPAREN(...) __VA_ARGS__

#define LQCD_UNPAREN_PK(...) __VA_ARGS__
// launch the packed-form kernel K with bs threads per block (64, 128, 256)
#define LQCD_LAUNCH_PACKED(bs, kern, targs, args)                                                                    \
    do {                                                                                                             \
        const int nbp_ = nblocks_for(g.Vh, bs);                                                                      \
        if (bs == 64)                                                                                                \
            kern##_packed_kernel<LQCD_UNPAREN_PK targs, 64><<<nbp_, 64, 0, s>>> args;                                \
        else if (bs == 256)                                                                                          \
            kern##_packed_kernel<LQCD_UNPAREN_PK targs, 256><<<nbp_, 256, 0, s>>> args;                              \
        else                                                                                                         \
            kern##_packed_kernel<LQCD_UNPAREN_PK targs, 128><<<nbp_, 128, 0, s>>> args;                              \
    } while (0)

// threads per block of the packed FP16+norm kernels on this lattice: the
// calling thread's override while the autotuner times a candidate, else the
// autotuner's choice, else DS_BLOCK
static thread_local int t_packed_block = 0;

int dslash_packed_block_override(int bs)
{
    const int prev = t_packed_block;
    t_packed_block = bs;
    return prev;
}

static int packed_block(const lqcd_field *in)
{
    const int b = t_packed_block ? t_packed_block : tuned_block(TK_HOP_F16N, in->lat, DS_BLOCK);
    return (b == 64 || b == 128 || b == 256) ? b : DS_BLOCK;
}

template <lqcd_prec P, lqcd_prec GP = P>
static void launch_plain(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger, const int *skip,
                         cudaStream_t s, int bs = 0)
{
    using R = typename ArithOf<P>::type;
    Geo g = make_geo(in->lat);
    const int st = use_form<P, GP>(g);
    if constexpr (P == LQCD_F16N && GP == LQCD_F16N) {
        if (st == 2) {
            if (bs == 0) bs = packed_block(in);
            if (dagger)
                LQCD_LAUNCH_PACKED(bs, dslash_plain, (R, P, GP, true),
                                   (spinor_ref<P>(out), spinor_ref<P>(in), gauge_ref<GP>(U), g, out_parity(out), skip));
            else
                LQCD_LAUNCH_PACKED(bs, dslash_plain, (R, P, GP, false),
                                   (spinor_ref<P>(out), spinor_ref<P>(in), gauge_ref<GP>(U), g, out_parity(out), skip));
            return;
        }
    }
    int nb = dslash_blocks(g.Vh);
    if (dagger)
        LQCD_LAUNCH_FORM(st, dslash_plain, (R, P, GP, true), nb,
                           (spinor_ref<P>(out), spinor_ref<P>(in), gauge_ref<GP>(U), g, out_parity(out), skip));
    else
        LQCD_LAUNCH_FORM(st, dslash_plain, (R, P, GP, false), nb,
                           (spinor_ref<P>(out), spinor_ref<P>(in), gauge_ref<GP>(U), g, out_parity(out), skip));
}

template <lqcd_prec P, lqcd_prec GP = P>
static void launch_xpay(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger, const lqcd_field *x,
                        double b, double *partials, const int *skip, cudaStream_t s, CgScalars *fin)
{
    using R = typename ArithOf<P>::type;
    Geo g = make_geo(in->lat);
    const int st = use_form<P, GP>(g);
    if constexpr (P == LQCD_F16N && GP == LQCD_F16N) {
        if (st == 2) {
            const int bs = packed_block(in), nb = nblocks_for(g.Vh, bs);
            if (dagger)
                LQCD_LAUNCH_PACKED(bs, dslash_xpay, (R, P, GP, true),
                                   (spinor_ref<P>(out), spinor_ref<P>(in), gauge_ref<GP>(U), g, out_parity(out),
                                    spinor_ref<P>(x), (R)b, partials, nb, skip, fin));
            else
                LQCD_LAUNCH_PACKED(bs, dslash_xpay, (R, P, GP, false),
                                   (spinor_ref<P>(out), spinor_ref<P>(in), gauge_ref<GP>(U), g, out_parity(out),
                                    spinor_ref<P>(x), (R)b, partials, nb, skip, fin));
            return;
        }
    }
    int nb = dslash_blocks(g.Vh);
    if (dagger)
        LQCD_LAUNCH_FORM(st, dslash_xpay, (R, P, GP, true), nb,
                           (spinor_ref<P>(out), spinor_ref<P>(in), gauge_ref<GP>(U), g, out_parity(out),
                            spinor_ref<P>(x), (R)b, partials, nb, skip, fin));
    else
        LQCD_LAUNCH_FORM(st, dslash_xpay, (R, P, GP, false), nb,
                           (spinor_ref<P>(out), spinor_ref<P>(in), gauge_ref<GP>(U), g, out_parity(out),
                            spinor_ref<P>(x), (R)b, partials, nb, skip, fin));
}

template <lqcd_prec P, lqcd_prec XP>
static void launch_cg(const lqcd_field *U, const lqcd_field *in, int dagger, const lqcd_field *t, double b,
                      lqcd_field *xs, lqcd_field *r, const lqcd_field *p, double *partials, CgScalars *sc,
                      cudaStream_t s)
{
    using R = typename ArithOf<P>::type;
    Geo g = make_geo(in->lat);
    int op = out_parity(t);
    const int st = use_form<P, P>(g);
    if constexpr (P == LQCD_F16N) {
        if (st == 2) {
            const int bs = packed_block(in), nb = nblocks_for(g.Vh, bs);
            if (dagger)
                LQCD_LAUNCH_PACKED(bs, dslash_cg, (R, P, P, true, XP),
                                   (spinor_ref<P>(in), gauge_ref<P>(U), g, op, spinor_ref<P>(t), (R)b,
                                    spinor_ref<XP>(xs), spinor_ref<P>(r), spinor_ref<P>(p), partials, nb, sc));
            else
                LQCD_LAUNCH_PACKED(bs, dslash_cg, (R, P, P, false, XP),
                                   (spinor_ref<P>(in), gauge_ref<P>(U), g, op, spinor_ref<P>(t), (R)b,
                                    spinor_ref<XP>(xs), spinor_ref<P>(r), spinor_ref<P>(p), partials, nb, sc));
            return;
        }
    }
    int nb = dslash_blocks(g.Vh);
    if (dagger)
        LQCD_LAUNCH_FORM(st, dslash_cg, (R, P, P, true, XP), nb,
                           (spinor_ref<P>(in), gauge_ref<P>(U), g, op, spinor_ref<P>(t), (R)b, spinor_ref<XP>(xs),
                            spinor_ref<P>(r), spinor_ref<P>(p), partials, nb, sc));
    else
        LQCD_LAUNCH_FORM(st, dslash_cg, (R, P, P, false, XP), nb,
                           (spinor_ref<P>(in), gauge_ref<P>(U), g, op, spinor_ref<P>(t), (R)b, spinor_ref<XP>(xs),
                            spinor_ref<P>(r), spinor_ref<P>(p), partials, nb, sc));
}

// the packed plain hop with bs threads per block, for the autotuner
int dslash_form_set(int form)
{
    if (form < 0) return g_form.load();
    if (form > 2) {
        set_error("dslash_form: unknown form %d (0 gathered, 1 prefetched links, 2 packed)", form);
        return -1;
    }
    return g_form.exchange(form);
}

lqcd_status dslash_plain(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger, const int *skip,
                         cudaStream_t s)
{
    LQCD_TRY(check_pair(out, U, in));
    double site = 8 * link_bytes(U->prec) + 2 * spinor_site_bytes(in->prec);
    KernelTimer kt(dslash_class(in->prec), s, site * in->Vh);
    KernelTimer kt_plain(in->prec == LQCD_F16N ? K_DSLASH_F16N_PLAIN : K_NCLASS, s, site * in->Vh);
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
    default: dslash_df_launch(out, U, in, dagger, nullptr, 0.0, skip, s); break;
    }
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status dslash_xpay(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger, const lqcd_field *x,
                        double b, double *partials, const int *skip, cudaStream_t s, CgScalars *fin)
{
    LQCD_TRY(check_pair(out, U, in));
    LQCD_REQUIRE(x && x->kind == out->kind && x->prec == out->prec, "dslash_xpay: x must match out");
    double site = 8 * link_bytes(U->prec) + 3 * spinor_site_bytes(in->prec); // + read of x
    KernelTimer kt(dslash_class(in->prec), s, site * in->Vh);
    switch (in->prec) {
    case LQCD_F64: launch_xpay<LQCD_F64>(out, U, in, dagger, x, b, partials, skip, s, fin); break;
    case LQCD_F32:
        if (U->prec == LQCD_F64)
            launch_xpay<LQCD_F32, LQCD_F64>(out, U, in, dagger, x, b, partials, skip, s, fin);
        else
            launch_xpay<LQCD_F32>(out, U, in, dagger, x, b, partials, skip, s, fin);
        break;
    case LQCD_F16N: launch_xpay<LQCD_F16N>(out, U, in, dagger, x, b, partials, skip, s, fin); break;
    case LQCD_BF16: launch_xpay<LQCD_BF16>(out, U, in, dagger, x, b, partials, skip, s, fin); break;
    default:
        LQCD_REQUIRE(partials == nullptr, "float-float hopping term has no norm reduction");
        dslash_df_launch(out, U, in, dagger, x, b, skip, s);
        break;
    }
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status dslash_cg(const lqcd_field *U, const lqcd_field *in, int dagger, const lqcd_field *t, double b,
                      lqcd_field *xs, lqcd_field *r, const lqcd_field *p, double *partials, CgScalars *sc,
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

int lqcd_dslash_form(int form) { return dslash_form_set(form); }

} // extern "C"
