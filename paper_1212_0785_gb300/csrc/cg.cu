// cg.cu -- conjugate gradient on Mhat^dag Mhat (the matrix inversion the paper
// hands to QUDA, Sec. 6).
//
// Plain FP64 CG, or reliable-update mixed precision (Clark, Babich, Barros,
// Brower, Rebbi 2010): the iteration runs on sloppy fields (FP32, FP16+norm
// or BF16 storage, FP32 arithmetic, FP64 dot products) and whenever the sloppy
// residual has dropped by delta since the last update the solution increment
// is folded into the accurate solution and the residual recomputed
// accurately.  The accurate solution, source, links and residual of the mixed
// solve are held in float-float storage and the residual is computed in
// float-float arithmetic (about 48 significant bits, see df64.cuh): on GB300
// that runs several times faster than FP64 and is far more accurate than the
// 1e-10 tolerance needs.  The plain FP64 solve uses FP64 throughout.
//
// Every scalar (rr, pAp, alpha, beta) lives on the device: the last block of
// each reducing hop kernel sums the block partials in a fixed order, computes
// them and raises a pause flag when the host must act, and every iteration
// kernel is a no-op while the flag is set.  The
// host therefore synchronises only once per chunk of iterations, yet the
// iteration count is exactly that of a per-iteration check.
#include <atomic>
#include <chrono>
#include <cmath>

#include "cg.cuh"
#include "dslash_df.cuh"
#include "df64.cuh"

namespace lqcd {

constexpr int BB = CG_BLOCK;
constexpr int CG_CHUNK = 4;

__global__ void cg_set_kernel(CgScalars *sc, double rr, double beta, double maxrr2)
{
    sc->rr = rr;
    sc->beta = beta;
    sc->maxrr2 = maxrr2;
    sc->pause = 0;
    sc->reason = PAUSE_NONE;
}

template <lqcd_prec P>
__global__ void p_update_kernel(SpinorRef<P> p, SpinorRef<P> r, const CgScalars *sc, int Vh)
{
    if (sc->pause) return;
    int cb = blockIdx.x * BB + threadIdx.x;
    if (cb >= Vh) return;
    using R = typename std::conditional<P == LQCD_F64, double, float>::type;
    R beta = (R)sc->beta;
    Sp<R> pv = p.template load_rw<R>(cb);
    Sp<R> rv = r.template load_rw<R>(cb);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int k = 0; k < 3; k++) pv.c[a][k] = rv.c[a][k] + beta * pv.c[a][k];
    p.store(cb, pv);
}

// r = b - t and block partials of |r|^2
__global__ void __launch_bounds__(BB) residual_kernel(SpinorRef<LQCD_F64> r, SpinorRef<LQCD_F64> b,
                                                      SpinorRef<LQCD_F64> t, double *partials, int nb, int Vh)
{
    int cb = blockIdx.x * BB + threadIdx.x;
    double n2[1] = {0.0};
    if (cb < Vh) {
        Sp<double> bv = b.load_rw<double>(cb), tv = t.load_rw<double>(cb);
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                bv.c[a][k] = bv.c[a][k] - tv.c[a][k];
                n2[0] += norm2(bv.c[a][k]);
            }
        r.store(cb, bv);
    }
    block_sum_store<1, BB>(n2, partials, nb);
}

// x += xs; xs = 0
__global__ void accum_zero_kernel(SpinorRef<LQCD_F64> x, SpinorRef<LQCD_F32> xs, int Vh)
{
    int cb = blockIdx.x * BB + threadIdx.x;
    if (cb >= Vh) return;
    Sp<double> xv = x.load_rw<double>(cb);
    Sp<double> dv = xs.load_rw<double>(cb);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int k = 0; k < 3; k++) xv.c[a][k] = xv.c[a][k] + dv.c[a][k];
    x.store(cb, xv);
    xs.store(cb, sp_zero<double>());
}

// ---------------------------------------------------------------- float-float helpers

// x += xs (exact float-float sum); xs = 0
__global__ void accum_df_kernel(SpinorRef<PREC_DF> x, SpinorRef<LQCD_F32> xs, int Vh)
{
    int cb = blockIdx.x * BB + threadIdx.x;
    if (cb >= Vh) return;
    accum_df_site(x, xs, cb);
}

template <lqcd_prec PS, lqcd_prec PD, typename R>
__global__ void convert_spinor_kernel(SpinorRef<PD> dst, SpinorRef<PS> src, int Vh)
{
    int cb = blockIdx.x * BB + threadIdx.x;
    if (cb >= Vh) return;
    dst.store(cb, src.template load_rw<R>(cb));
}

__global__ void split_gauge_kernel(GaugeRef<PREC_DF> dst, GaugeRef<LQCD_F64> src, int Vh)
{
    long t = blockIdx.x * (long)BB + threadIdx.x;
    if (t >= 8L * Vh) return;
    int cb = (int)(t % Vh), mp = (int)(t / Vh);
    dst.store(mp >> 1, mp & 1, cb, src.load<double>(mp >> 1, mp & 1, cb));
}

// ---------------------------------------------------------------- minimal residual extrapolation

// d = a - b (FP64 solutions) rounded to FP32
__global__ void mre_diff_kernel(SpinorRef<LQCD_F32> d, SpinorRef<LQCD_F64> a, SpinorRef<LQCD_F64> b, int Vh)
{
    int cb = blockIdx.x * BB + threadIdx.x;
    if (cb >= Vh) return;
    Sp<double> av = a.load_rw<double>(cb), bv = b.load_rw<double>(cb);
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int c = 0; c < 3; c++) av.c[k][c] = av.c[k][c] - bv.c[k][c];
    d.store(cb, av);
}

// block partials of G_ij = Re<w_i, w_j> (i <= j, row by row) and g_i = Re<w_i, r>
// for N directions; r in float-float (its leading parts)
template <int N>
__global__ void __launch_bounds__(BB) mre_dots_kernel(const float4 *const *w, SpinorRef<PREC_DF> r, double *partials,
                                                       int nb, int Vh)
{
    constexpr int NG = N * (N + 1) / 2, NT = NG + N;
    int cb = blockIdx.x * BB + threadIdx.x;
    double v[NT];
#pragma unroll
    for (int k = 0; k < NT; k++) v[k] = 0.0;
    if (cb < Vh) {
        float4 wv[N][6];
#pragma unroll
        for (int j = 0; j < N; j++)
#pragma unroll
            for (int k = 0; k < 6; k++) wv[j][k] = w[j][(size_t)k * Vh + cb];
        Sp<float> rv = r.load_rw<float>(cb);
        float rr[24];
#pragma unroll
        for (int k = 0; k < 12; k++) rr[2 * k] = rv.c[k / 3][k % 3].re, rr[2 * k + 1] = rv.c[k / 3][k % 3].im;
        int q = 0;
#pragma unroll
        for (int i = 0; i < N; i++)
#pragma unroll
            for (int j = i; j < N; j++, q++) {
                float a = 0.f;
#pragma unroll
                for (int k = 0; k < 6; k++)
                    a += wv[i][k].x * wv[j][k].x + wv[i][k].y * wv[j][k].y + wv[i][k].z * wv[j][k].z +
                         wv[i][k].w * wv[j][k].w;
                v[q] = a;
            }
#pragma unroll
        for (int i = 0; i < N; i++) {
            float a = 0.f;
#pragma unroll
            for (int k = 0; k < 6; k++)
                a += wv[i][k].x * rr[4 * k] + wv[i][k].y * rr[4 * k + 1] + wv[i][k].z * rr[4 * k + 2] +
                     wv[i][k].w * rr[4 * k + 3];
            v[NG + i] = a;
        }
    }
    block_sum_store<NT, BB>(v, partials, nb);
}

// x += sum_j c_j d_j and r -= sum_j c_j w_j in float-float; block partials of
// |r|^2 from the leading parts
template <int N>
__global__ void __launch_bounds__(BB) mre_update_kernel(SpinorRef<PREC_DF> x, SpinorRef<PREC_DF> r,
                                                         const float4 *const *d, const float4 *const *w, double c0,
                                                         double c1, double c2, double *partials, int nb, int Vh)
{
    int cb = blockIdx.x * BB + threadIdx.x;
    double n2[1] = {0.0};
    if (cb < Vh) {
        const Df c[3] = {Df(c0), Df(c1), Df(c2)};
        Sp<Df> xv = x.load_rw<Df>(cb), rv = r.load_rw<Df>(cb);
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            Df *xe[4] = {&xv.c[(2 * k) / 3][(2 * k) % 3].re, &xv.c[(2 * k) / 3][(2 * k) % 3].im,
                         &xv.c[(2 * k + 1) / 3][(2 * k + 1) % 3].re, &xv.c[(2 * k + 1) / 3][(2 * k + 1) % 3].im};
            Df *re[4] = {&rv.c[(2 * k) / 3][(2 * k) % 3].re, &rv.c[(2 * k) / 3][(2 * k) % 3].im,
                         &rv.c[(2 * k + 1) / 3][(2 * k + 1) % 3].re, &rv.c[(2 * k + 1) / 3][(2 * k + 1) % 3].im};
#pragma unroll
            for (int j = 0; j < N; j++) {
                const float4 dv = d[j][(size_t)k * Vh + cb], wv = w[j][(size_t)k * Vh + cb];
                const float dd[4] = {dv.x, dv.y, dv.z, dv.w}, ww[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    *xe[q] += c[j] * Df(dd[q], 0.f);
                    *re[q] += -(c[j] * Df(ww[q], 0.f));
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) acc += re[q]->hi * re[q]->hi;
        }
        x.store(cb, xv);
        r.store(cb, rv);
        n2[0] = acc;
    }
    block_sum_store<1, BB>(n2, partials, nb);
}

template <lqcd_prec PS, lqcd_prec PD, typename R>
static lqcd_status convert_spinor(lqcd_field *dst, const lqcd_field *src, cudaStream_t s)
{
    convert_spinor_kernel<PS, PD, R><<<nblocks_for(src->Vh, BB), BB, 0, s>>>(spinor_ref<PD>(dst), spinor_ref<PS>(src),
                                                                             src->Vh);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

// float-float residual -> sloppy residual
static lqcd_status df_to_sloppy(lqcd_field *dst, const lqcd_field *src, cudaStream_t s)
{
    switch (dst->prec) {
    case LQCD_F32: return convert_spinor<PREC_DF, LQCD_F32, float>(dst, src, s);
    case LQCD_F16N: return convert_spinor<PREC_DF, LQCD_F16N, float>(dst, src, s);
    case LQCD_BF16: return convert_spinor<PREC_DF, LQCD_BF16, float>(dst, src, s);
    default: set_error("df_to_sloppy: bad precision"); return LQCD_EINVAL;
    }
}

// ---------------------------------------------------------------- pinned scalars

struct Pinned {
    CgScalars *sc = nullptr;
    double *d = nullptr;
    ~Pinned()
    {
        if (sc) cudaFreeHost(sc);
        if (d) cudaFreeHost(d);
    }
};
static thread_local Pinned g_pinned;

static lqcd_status pinned()
{
    if (!g_pinned.sc) {
        LQCD_CUDA(cudaMallocHost((void **)&g_pinned.sc, sizeof(CgScalars)));
        LQCD_CUDA(cudaMallocHost((void **)&g_pinned.d, 8 * sizeof(double)));
    }
    return LQCD_OK;
}

// ---------------------------------------------------------------- work space

lqcd_status CgWorkspace::ensure_mre(int n, cudaStream_t s)
{
    n = std::min(n, MRE_MAX);
    // the normal equations' block partials: up to 9 sums of CG_BLOCK-site blocks
    const size_t need = 9 * (size_t)nblocks_for(make_geo(lat).Vh, BB) * sizeof(double);
    if (partials.bytes < need) {
        lqcd_status rc = partials.alloc(need, s);
        if (rc != LQCD_OK) { // the old buffer is gone: the next solve rebuilds the work space
            ready = false;
            return rc;
        }
    }
    // each field only if missing, so a call that failed half way can be repeated
    if (!mre_te.f) LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F32, 0, &mre_te.f));
    if (!mre_to.f) LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_ODD, LQCD_F32, 0, &mre_to.f));
    for (; mre_n < n; mre_n++) {
        if (!mre_d[mre_n].f) LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F32, 0, &mre_d[mre_n].f));
        if (!mre_w[mre_n].f) LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F32, 0, &mre_w[mre_n].f));
    }
    return LQCD_OK;
}

lqcd_status CgWorkspace::ensure(const lqcd_lattice &l, lqcd_prec sl, cudaStream_t s)
{
    if (ready && same_lattice(lat, l) && sloppy == sl) return LQCD_OK;
    ready = false;
    bdf_of = nullptr;
    for (FieldPtr *f : {&mre_d[0], &mre_d[1], &mre_d[2], &mre_w[0], &mre_w[1], &mre_w[2], &mre_te, &mre_to}) {
        if (f->f) lqcd_field_free(f->f);
        f->f = nullptr;
    }
    mre_n = 0;
    for (FieldPtr *f : {&r64, &t64a, &t64b, &tmpo64, &p64, &xs, &rs, &ps, &ts, &tmpos, &Udf, &xdf, &bdf, &rdf,
                        &t1df, &tmpodf}) {
        if (f->f) lqcd_field_free(f->f);
        f->f = nullptr;
    }
    lat = l;
    sloppy = sl;
    if (sl == LQCD_F64) {
        LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &r64.f));
        LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &t64a.f));
        LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &t64b.f));
        LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_ODD, LQCD_F64, 0, &tmpo64.f));
        LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &p64.f));
    } else {
        if (temps_only) {
            LQCD_TRY(field_alloc_df(&lat, LQCD_SPINOR_EVEN, &rdf.f));
            LQCD_TRY(field_alloc_df(&lat, LQCD_SPINOR_EVEN, &t1df.f));
            LQCD_TRY(field_alloc_df(&lat, LQCD_SPINOR_ODD, &tmpodf.f));
            ready = true;
            return LQCD_OK;
        }
        if (!udf_ext) LQCD_TRY(field_alloc_df(&lat, LQCD_GAUGE, &Udf.f));
        LQCD_TRY(field_alloc_df(&lat, LQCD_SPINOR_EVEN, &xdf.f));
        LQCD_TRY(field_alloc_df(&lat, LQCD_SPINOR_EVEN, &bdf.f));
        if (!tmp_from) {
            LQCD_TRY(field_alloc_df(&lat, LQCD_SPINOR_EVEN, &rdf.f));
            LQCD_TRY(field_alloc_df(&lat, LQCD_SPINOR_EVEN, &t1df.f));
            LQCD_TRY(field_alloc_df(&lat, LQCD_SPINOR_ODD, &tmpodf.f));
        }
        LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F32, 0, &xs.f));
        LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, sl, 0, &rs.f));
        LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, sl, 0, &ps.f));
        LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, sl, 0, &ts.f));
        LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_ODD, sl, 0, &tmpos.f));
    }
    int Vh = make_geo(lat).Vh;
    // one partial per hop block (down to the 64-thread blocks of a tuned hop) or per CG_BLOCK sites
    size_t np = (size_t)std::max(std::max(nblocks_for(Vh, 64), nblocks_for(Vh, BB)), 2048);
    LQCD_TRY(sc.alloc(sizeof(CgScalars), s));
    LQCD_TRY(partials.alloc(np * sizeof(double), s));
    LQCD_TRY(scalars.alloc(16 * sizeof(double), s));
    ready = true;
    return LQCD_OK;
}

size_t CgWorkspace::bytes() const
{
    size_t n = sc.bytes + partials.bytes + scalars.bytes;
    for (const FieldPtr *f : {&r64, &t64a, &t64b, &tmpo64, &p64, &xs, &rs, &ps, &ts, &tmpos, &Udf, &xdf, &bdf, &rdf,
                              &t1df, &tmpodf, &mre_d[0], &mre_d[1], &mre_d[2], &mre_w[0], &mre_w[1],
                              &mre_w[2], &mre_te, &mre_to})
        if (f->f) n += f->f->bytes + f->f->norm_bytes;
    return n;
}

static lqcd_status launch_p_update(lqcd_field *p, lqcd_field *r, const CgScalars *sc, cudaStream_t s)
{
    int nb = nblocks_for(p->Vh, BB);
    switch (p->prec) {
    case LQCD_F64: p_update_kernel<LQCD_F64><<<nb, BB, 0, s>>>(spinor_ref<LQCD_F64>(p), spinor_ref<LQCD_F64>(r), sc, p->Vh); break;
    case LQCD_F32: p_update_kernel<LQCD_F32><<<nb, BB, 0, s>>>(spinor_ref<LQCD_F32>(p), spinor_ref<LQCD_F32>(r), sc, p->Vh); break;
    case LQCD_F16N: p_update_kernel<LQCD_F16N><<<nb, BB, 0, s>>>(spinor_ref<LQCD_F16N>(p), spinor_ref<LQCD_F16N>(r), sc, p->Vh); break;
    case LQCD_BF16: p_update_kernel<LQCD_BF16><<<nb, BB, 0, s>>>(spinor_ref<LQCD_BF16>(p), spinor_ref<LQCD_BF16>(r), sc, p->Vh); break;
    }
    LQCD_LAUNCHED();
    return LQCD_OK;
}

// accurate residual r = b - A x of the mixed solve in float-float arithmetic
// (x, b, links in float-float storage); |r|^2 into ws.scalars[0] (device),
// not read back
static lqcd_status residual_df_enqueue(CgWorkspace &ws, double kappa, cudaStream_t s)
{
    double k2 = kappa * kappa;
    LQCD_TRY(dslash_plain(ws.tmpo(), ws.udf(), ws.xdf.f, 0, nullptr, s));
    LQCD_TRY(dslash_xpay(ws.t1(), ws.udf(), ws.tmpo(), 0, ws.xdf.f, -k2, nullptr, nullptr, s));
    LQCD_TRY(dslash_plain(ws.tmpo(), ws.udf(), ws.t1(), 1, nullptr, s));
    // the last term writes r = b - (t1 - kappa^2 D^dag tmpo) and its block partials of |r|^2
    LQCD_TRY(dslash_df_residual(ws.rdf_(), ws.udf(), ws.tmpo(), ws.t1(), -k2, ws.bdf.f, (double *)ws.partials.p, s));
    const int nb = nblocks_for(ws.xdf.f->Vh, DF_SITES);
    return reduce_partials((double *)ws.partials.p, nb, 1, (double *)ws.scalars.p, s);
}

// the same, read back: |r|^2 in *rr
static lqcd_status true_residual_df(CgWorkspace &ws, double kappa, double *rr, cudaStream_t s)
{
    LQCD_TRY(residual_df_enqueue(ws, kappa, s));
    LQCD_TRY(pinned());
    LQCD_TRY(read_scalars((double *)ws.scalars.p, g_pinned.d, 1, s));
    *rr = g_pinned.d[0];
    return LQCD_OK;
}

// true residual r64 = b - A x in FP64; |r64|^2 returned in *rr
static lqcd_status true_residual(CgWorkspace &ws, const lqcd_field *x, const lqcd_field *U, const lqcd_field *b,
                                 double kappa, double *rr, cudaStream_t s)
{
    LQCD_TRY(mhat_apply(ws.t64a.f, U, x, kappa, 0, ws.tmpo64.f, nullptr, s));
    LQCD_TRY(mhat_apply(ws.t64b.f, U, ws.t64a.f, kappa, 1, ws.tmpo64.f, nullptr, s));
    int Vh = x->Vh, nb = nblocks_for(Vh, BB);
    residual_kernel<<<nb, BB, 0, s>>>(spinor_ref<LQCD_F64>(ws.r64.f), spinor_ref<LQCD_F64>(b),
                                      spinor_ref<LQCD_F64>(ws.t64b.f), (double *)ws.partials.p, nb, Vh);
    LQCD_LAUNCHED();
    LQCD_TRY(reduce_partials((double *)ws.partials.p, nb, 1, (double *)ws.scalars.p, s));
    LQCD_TRY(pinned());
    LQCD_TRY(read_scalars((double *)ws.scalars.p, g_pinned.d, 1, s));
    *rr = g_pinned.d[0];
    return LQCD_OK;
}

// float-float copy of FP64 links (for owners that share one copy among solves)
lqcd_status df_to_f64(lqcd_field *dst, const lqcd_field *src_df, cudaStream_t s)
{
    return convert_spinor<PREC_DF, LQCD_F64, double>(dst, src_df, s);
}

lqcd_status split_links(lqcd_field *Udf, const lqcd_field *U, cudaStream_t s)
{
    split_gauge_kernel<<<nblocks_for(8L * U->Vh, BB), BB, 0, s>>>(gauge_ref<PREC_DF>(Udf), gauge_ref<LQCD_F64>(U),
                                                                    U->Vh);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

// ---------------------------------------------------------------- one solve as a state machine

lqcd_status CgRun::fail(lqcd_status st)
{
    done = true;
    status = st;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

lqcd_status CgRun::succeed()
{
    done = true;
    status = LQCD_OK;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return LQCD_OK;
}

// Minimal residual extrapolation (Brower, Ivanenko, Levkova, Orginos 1997,
// the chronological inverter of the paper's Sec. 6.2): the guess x_L already
// in x / xdf has its accurate residual r_L in rdf.  Over the directions
// d_j = x_j - x_{j+1} of the last n_mre solutions, the real coefficients c
// minimising |r_L - sum_j c_j A d_j| solve the normal equations G c = g,
// G_ij = Re<A d_i, A d_j>, g_i = Re<A d_i, r_L>; the guess becomes
// x_L + sum_j c_j d_j and its residual r_L - sum_j c_j A d_j.  The products
// A d_j are formed in FP32 arithmetic: they multiply differences of nearby
// solutions, so their rounding error is ~1e-7 of |r_L|, far below the solve's
// tolerance, and the updates of x and r are float-float.  A singular or
// ill-conditioned G leaves the guess as it was.
lqcd_status CgRun::mre_refine(cudaStream_t s, double *rr0)
{
    CgWorkspace &w = *ws;
    const int nd = std::min(n_mre - 1, CgWorkspace::MRE_MAX);
    LQCD_TRY(w.ensure_mre(nd, s));
    const lqcd_field *L = mre_links ? mre_links : U;
    const int nb = nblocks_for(Vh, BB);
    for (int j = 0; j < nd; j++) {
        mre_diff_kernel<<<nb, BB, 0, s>>>(spinor_ref<LQCD_F32>(w.mre_d[j].f), spinor_ref<LQCD_F64>(mre_x[j]),
                                          spinor_ref<LQCD_F64>(mre_x[j + 1]), Vh);
        LQCD_LAUNCHED();
        LQCD_TRY(mhat_apply(w.mre_te.f, L, w.mre_d[j].f, kappa, 0, w.mre_to.f, nullptr, s));
        LQCD_TRY(mhat_apply(w.mre_w[j].f, L, w.mre_te.f, kappa, 1, w.mre_to.f, nullptr, s));
    }
    // the direction pointers in device memory (one small table after the partials' scalars)
    const float4 *ptrs[2 * CgWorkspace::MRE_MAX];
    for (int j = 0; j < nd; j++) {
        ptrs[j] = (const float4 *)w.mre_d[j].f->data;
        ptrs[CgWorkspace::MRE_MAX + j] = (const float4 *)w.mre_w[j].f->data;
    }
    if (w.mre_tab.bytes < sizeof(ptrs)) LQCD_TRY(w.mre_tab.alloc(sizeof(ptrs), s));
    LQCD_CUDA(cudaMemcpyAsync(w.mre_tab.p, ptrs, sizeof(ptrs), cudaMemcpyHostToDevice, s));
    const float4 *const *dtab = (const float4 *const *)w.mre_tab.p;
    const float4 *const *wtab = dtab + CgWorkspace::MRE_MAX;
    double *part = (double *)w.partials.p;
    const int ng = nd * (nd + 1) / 2, nt = ng + nd;
    switch (nd) {
    case 1: mre_dots_kernel<1><<<nb, BB, 0, s>>>(wtab, spinor_ref<PREC_DF>(w.rdf_()), part, nb, Vh); break;
    case 2: mre_dots_kernel<2><<<nb, BB, 0, s>>>(wtab, spinor_ref<PREC_DF>(w.rdf_()), part, nb, Vh); break;
    default: mre_dots_kernel<3><<<nb, BB, 0, s>>>(wtab, spinor_ref<PREC_DF>(w.rdf_()), part, nb, Vh); break;
    }
    LQCD_LAUNCHED();
    LQCD_TRY(reduce_partials(part, nb, nt, (double *)w.scalars.p, s));
    double h[9];
    LQCD_TRY(read_scalars((double *)w.scalars.p, h, nt, s)); // synchronises: ptrs may go out of scope
    // G c = g by Cholesky (G symmetric positive semi-definite)
    double G[3][3], g[3], Lc[3][3] = {}, c[3] = {0, 0, 0};
    for (int i = 0, q = 0; i < nd; i++)
        for (int j = i; j < nd; j++, q++) G[i][j] = G[j][i] = h[q];
    for (int i = 0; i < nd; i++) g[i] = h[ng + i];
    bool ok = true;
    for (int i = 0; i < nd && ok; i++) {
        for (int j = 0; j <= i; j++) {
            double v = G[i][j];
            for (int k = 0; k < j; k++) v -= Lc[i][k] * Lc[j][k];
            if (i == j) {
                ok = std::isfinite(v) && v > 1e-24 * G[0][0] && v > 0;
                Lc[i][i] = ok ? std::sqrt(v) : 0.0;
            } else {
                Lc[i][j] = v / Lc[j][j];
            }
        }
    }
    if (!ok) return LQCD_OK; // keep the extrapolated guess
    double y[3];
    for (int i = 0; i < nd; i++) {
        double v = g[i];
        for (int k = 0; k < i; k++) v -= Lc[i][k] * y[k];
        y[i] = v / Lc[i][i];
    }
    for (int i = nd - 1; i >= 0; i--) {
        double v = y[i];
        for (int k = i + 1; k < nd; k++) v -= Lc[k][i] * c[k];
        c[i] = v / Lc[i][i];
    }
    switch (nd) {
    case 1:
        mre_update_kernel<1><<<nb, BB, 0, s>>>(spinor_ref<PREC_DF>(w.xdf.f), spinor_ref<PREC_DF>(w.rdf_()), dtab, wtab,
                                               c[0], c[1], c[2], part, nb, Vh);
        break;
    case 2:
        mre_update_kernel<2><<<nb, BB, 0, s>>>(spinor_ref<PREC_DF>(w.xdf.f), spinor_ref<PREC_DF>(w.rdf_()), dtab, wtab,
                                               c[0], c[1], c[2], part, nb, Vh);
        break;
    default:
        mre_update_kernel<3><<<nb, BB, 0, s>>>(spinor_ref<PREC_DF>(w.xdf.f), spinor_ref<PREC_DF>(w.rdf_()), dtab, wtab,
                                               c[0], c[1], c[2], part, nb, Vh);
        break;
    }
    LQCD_LAUNCHED();
    LQCD_TRY(reduce_partials(part, nb, 1, (double *)w.scalars.p, s));
    LQCD_TRY(read_scalars((double *)w.scalars.p, h, 1, s));
    *rr0 = h[0];
    mre_used = true;
    inf.guess_refined = 1;
    // the FP64 guess follows the float-float one (a solve that stops at once returns it)
    return convert_spinor<PREC_DF, LQCD_F64, double>(x, w.xdf.f, s);
}

lqcd_status CgRun::start(cudaStream_t s, CgScalars *sc_dev)
{
    t0 = std::chrono::steady_clock::now();
    sc = sc_dev;
    done = false;
    status = LQCD_OK;
    inf = lqcd_cg_info{0, 0, 0.0, 0.0, 0, 0, 0};
    mixed = prm.sloppy != LQCD_F64;
    lqcd_status rc = start_impl(s);
    if (rc != LQCD_OK) return fail(rc);
    return LQCD_OK;
}

lqcd_status CgRun::start_impl(cudaStream_t s)
{
    CgWorkspace &w = *ws;
    LQCD_TRY(w.ensure(x->lat, prm.sloppy, s));
    LQCD_TRY(pinned());
    Vh = x->Vh;
    k2 = kappa * kappa;
    LQCD_TRY(spinor_dot_dev(b, b, (double *)w.scalars.p, w.partials, s));
    LQCD_TRY(read_scalars((double *)w.scalars.p, g_pinned.d, 1, s));
    bb = g_pinned.d[0];
    if (!prm.guess) LQCD_CUDA(cudaMemsetAsync(x->data, 0, x->bytes, s));
    if (!std::isfinite(bb)) {
        set_error("cg: |b|^2 is not finite");
        return LQCD_ENUMERIC;
    }
    if (bb == 0.0) {
        LQCD_CUDA(cudaMemsetAsync(x->data, 0, x->bytes, s));
        LQCD_CUDA(cudaStreamSynchronize(s));
        succeed();
        return LQCD_OK;
    }
    double rr0 = bb;
    if (mixed) {
        LQCD_REQUIRE(Us && Us->kind == LQCD_GAUGE && Us->prec == prm.sloppy && Us->recon == 12,
                     "cg: mixed solve needs a 12-real link copy in the sloppy precision");
        if (!w.udf_ext) { // the float-float links of this solve
            split_gauge_kernel<<<nblocks_for(8L * Vh, BB), BB, 0, s>>>(gauge_ref<PREC_DF>(w.Udf.f),
                                                                       gauge_ref<LQCD_F64>(U), Vh);
            LQCD_LAUNCHED();
        }
        if (!(b_stamp && w.bdf_of == b && w.bdf_stamp == b_stamp)) {
            w.bdf_of = nullptr;
            LQCD_TRY((convert_spinor<LQCD_F64, PREC_DF, double>(w.bdf.f, b, s)));
            w.bdf_of = b;
            w.bdf_stamp = b_stamp;
        }
        LQCD_CUDA(cudaMemsetAsync(w.xs.f->data, 0, w.xs.f->bytes, s));
        if (prm.guess) { // r = b - A x0, accurately
            inf.accurate_residuals++;
            LQCD_TRY((convert_spinor<LQCD_F64, PREC_DF, double>(w.xdf.f, x, s)));
            LQCD_TRY(true_residual_df(w, kappa, &rr0, s));
            if (n_mre >= 2 && std::isfinite(rr0)) LQCD_TRY(mre_refine(s, &rr0));
            LQCD_TRY(df_to_sloppy(w.rs.f, w.rdf_(), s));
            LQCD_TRY(lqcd_field_copy(w.ps.f, w.rs.f, s));
        } else {
            LQCD_CUDA(cudaMemsetAsync(w.xdf.f->data, 0, w.xdf.f->bytes, s));
            LQCD_TRY(lqcd_field_copy(w.rs.f, b, s));
            LQCD_TRY(lqcd_field_copy(w.ps.f, b, s));
        }
        P = w.ps.f, R = w.rs.f, T = w.ts.f, TMP = w.tmpos.f, XS = w.xs.f, UU = Us;
    } else {
        if (prm.guess) {
            inf.accurate_residuals++;
            LQCD_TRY(true_residual(w, x, U, b, kappa, &rr0, s));
        } else {
            LQCD_CUDA(cudaMemcpyAsync(w.r64.f->data, b->data, b->bytes, cudaMemcpyDeviceToDevice, s));
        }
        LQCD_CUDA(cudaMemcpyAsync(w.p64.f->data, w.r64.f->data, b->bytes, cudaMemcpyDeviceToDevice, s));
        P = w.p64.f, R = w.r64.f, T = w.t64a.f, TMP = w.tmpo64.f, XS = x, UU = U;
    }
    inf.true_rel_res = std::sqrt(rr0 / bb);
    if (!std::isfinite(rr0)) {
        set_error("cg: the initial residual is not finite");
        return LQCD_ENUMERIC;
    }
    if (rr0 <= prm.tol * prm.tol * bb) { // the guess already solves the system
        LQCD_CUDA(cudaStreamSynchronize(s));
        succeed();
        return LQCD_OK;
    }
    h0 = CgScalars{};
    h0.rr = rr0;
    h0.stop2 = prm.tol * prm.tol * bb;
    h0.delta2 = mixed ? prm.delta * prm.delta : 0.0;
    h0.maxrr2 = rr0;
    h0.maxiter = prm.maxiter;
    LQCD_CUDA(cudaMemcpyAsync(sc, &h0, sizeof(CgScalars), cudaMemcpyHostToDevice, s));
    LQCD_CUDA(cudaStreamSynchronize(s)); // h0 may be rewritten before the copy otherwise
    return LQCD_OK;
}

lqcd_status CgRun::iterate(cudaStream_t s)
{
    double *partials = (double *)ws->partials.p;
    const int *skip = &sc->pause;
    // the last block of the axpy hop computes alpha, that of the CG-update hop
    // the pause decision and beta (cg_finish)
    LQCD_TRY(dslash_plain(TMP, UU, P, 0, skip, s));
    LQCD_TRY(dslash_xpay(T, UU, TMP, 0, P, -k2, partials, skip, s, sc));
    LQCD_TRY(dslash_plain(TMP, UU, T, 1, skip, s));
    LQCD_TRY(dslash_cg(UU, TMP, 1, T, -k2, XS, R, P, partials, sc, s));
    return launch_p_update(P, R, sc, s);
}

lqcd_status CgRun::on_pause(const CgScalars &h, cudaStream_t s)
{
    lqcd_status rc = on_pause_impl(h, s);
    if (rc != LQCD_OK && !done) return fail(rc);
    return rc;
}

lqcd_status CgRun::on_pause_impl(const CgScalars &h, cudaStream_t s)
{
    if (!mixed) {
        inf.iters = h.iter;
        if (h.reason == PAUSE_NONFINITE) {
            set_error("cg: non-finite value after %d iterations", h.iter);
            return fail(LQCD_ENUMERIC);
        }
        LQCD_TRY(true_residual(*ws, x, U, b, kappa, &rr_true, s));
        return pause_decide(h, s);
    }
    LQCD_TRY(pause_begin(h, s));
    if (done) return status;
    LQCD_TRY(pinned());
    LQCD_TRY(read_scalars(pause_result_dev(), g_pinned.d, 1, s));
    return pause_end(g_pinned.d[0], s);
}

// mixed solve, first half of a pause: accumulate the FP32 increment into the
// float-float solution and enqueue its accurate residual (read by the caller)
bool CgRun::pause_record(const CgScalars &h)
{
    inf.iters = h.iter;
    hp = h;
    if (h.reason == PAUSE_NONFINITE) {
        set_error("cg: non-finite value after %d iterations", h.iter);
        fail(LQCD_ENUMERIC);
        return false;
    }
    return true;
}

lqcd_status CgRun::pause_begin(const CgScalars &h, cudaStream_t s)
{
    CgWorkspace &w = *ws;
    if (!pause_record(h)) return status;
    accum_df_kernel<<<nblocks_for(Vh, BB), BB, 0, s>>>(spinor_ref<PREC_DF>(w.xdf.f), spinor_ref<LQCD_F32>(XS), Vh);
    LQCD_LAUNCHED();
    lqcd_status rc = residual_df_enqueue(w, kappa, s);
    if (rc != LQCD_OK) return fail(rc);
    return LQCD_OK;
}

double *CgRun::pause_result_dev() const { return (double *)ws->scalars.p; }

// second half: the decision on the accurate |r|^2
lqcd_status CgRun::pause_end(double rr, cudaStream_t s)
{
    rr_true = rr;
    lqcd_status rc = pause_decide(hp, s);
    if (rc != LQCD_OK && !done) return fail(rc);
    return rc;
}

lqcd_status CgRun::pause_decide(const CgScalars &h, cudaStream_t s)
{
    CgWorkspace &w = *ws;
    inf.true_rel_res = std::sqrt(rr_true / bb);
    inf.accurate_residuals++;
    if (h.reason == PAUSE_CONVERGED && !(rr_true <= h.stop2)) inf.failed_checks++;
    if (!std::isfinite(rr_true)) {
        set_error("cg: non-finite true residual");
        return fail(LQCD_ENUMERIC);
    }
    if (mixed && (rr_true <= h.stop2 || h.reason == PAUSE_MAXITER || h.iter >= prm.maxiter)) {
        // the FP64 solution is the float-float one rounded
        LQCD_TRY((convert_spinor<PREC_DF, LQCD_F64, double>(x, w.xdf.f, s)));
    }
    if (rr_true <= h.stop2) return succeed();
    if (h.reason == PAUSE_MAXITER || h.iter >= prm.maxiter) {
        set_error("cg: no convergence in %d iterations (true |r|/|b| = %.3e)", h.iter, inf.true_rel_res);
        return fail(LQCD_ENOCONV);
    }
    inf.restarts++;
    double beta;
    if (mixed) { // reliable update: continue with the accurate residual
        LQCD_TRY(df_to_sloppy(w.rs.f, w.rdf_(), s));
        beta = rr_true / h.rr;
    } else { // the iterated residual lied: restart from the true one
        if (inf.restarts > prm.max_restarts) {
            set_error("cg: true residual %.3e above tolerance after %d restarts", inf.true_rel_res,
                      prm.max_restarts);
            return fail(LQCD_ENOCONV);
        }
        beta = 0.0;
    }
    cg_set_kernel<<<1, 1, 0, s>>>(sc, rr_true, beta, rr_true);
    LQCD_LAUNCHED();
    return launch_p_update(P, R, sc, s);
}

uint64_t new_content_stamp()
{
    static std::atomic<uint64_t> next{1};
    return next.fetch_add(1, std::memory_order_relaxed);
}

lqcd_status cg_solve_ws(CgWorkspace &ws, lqcd_field *x, const lqcd_field *U, const lqcd_field *Us,
                        const lqcd_field *b, double kappa, const lqcd_cg_params &prm, lqcd_cg_info *info,
                        cudaStream_t s, const MreInput *mre, uint64_t b_stamp)
{
    LQCD_TRY(ws.ensure(x->lat, prm.sloppy, s));
    CgRun run;
    run.ws = &ws, run.x = x, run.U = U, run.Us = Us, run.b = b, run.kappa = kappa, run.prm = prm;
    run.b_stamp = b_stamp;
    if (mre && prm.guess && prm.sloppy != LQCD_F64) {
        run.n_mre = std::min(mre->n, CgWorkspace::MRE_MAX + 1);
        for (int j = 0; j < run.n_mre; j++) run.mre_x[j] = mre->x[j];
        run.mre_links = mre->links;
    }
    run.start(s, (CgScalars *)ws.sc.p);
    CgScalars &h = *g_pinned.sc;
    while (!run.done) {
        for (int k = 0; k < CG_CHUNK; k++) {
            lqcd_status rc = run.iterate(s);
            if (rc != LQCD_OK) {
                run.fail(rc);
                break;
            }
        }
        if (run.done) break;
        lqcd_status rc = [&]() -> lqcd_status {
            LQCD_CUDA(cudaMemcpyAsync(&h, run.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
            LQCD_CUDA(cudaStreamSynchronize(s));
            return LQCD_OK;
        }();
        if (rc != LQCD_OK) {
            run.fail(rc);
            break;
        }
        if (h.pause) run.on_pause(h, s);
    }
    if (info) *info = run.inf;
    return run.status;
}

} // namespace lqcd

using namespace lqcd;

extern "C" lqcd_status lqcd_cg_solve(lqcd_field *x, const lqcd_field *U, const lqcd_field *U_sloppy,
                                     const lqcd_field *b, double kappa, const lqcd_cg_params *params,
                                     lqcd_cg_info *info, void *stream)
{
    LQCD_REQUIRE(x && U && b && params, "cg_solve: NULL argument");
    LQCD_REQUIRE(x->kind == LQCD_SPINOR_EVEN && b->kind == LQCD_SPINOR_EVEN && x->prec == LQCD_F64 &&
                     b->prec == LQCD_F64,
                 "cg_solve: x and b must be EVEN FP64 spinors");
    LQCD_REQUIRE(x != b, "cg_solve: x must differ from b");
    LQCD_REQUIRE(U->kind == LQCD_GAUGE && U->prec == LQCD_F64, "cg_solve: U must be the FP64 gauge field");
    LQCD_REQUIRE(same_lattice(x->lat, U->lat) && same_lattice(b->lat, U->lat), "cg_solve: lattices differ");
    LQCD_REQUIRE(params->tol > 0 && params->maxiter > 0, "cg_solve: tol and maxiter must be positive");
    LQCD_REQUIRE(params->sloppy >= LQCD_F64 && params->sloppy <= LQCD_BF16, "cg_solve: bad sloppy precision");
    LQCD_REQUIRE(params->sloppy == LQCD_F64 || (params->delta > 0 && params->delta < 1),
                 "cg_solve: delta must lie in (0, 1)");
    cudaStream_t s = (cudaStream_t)stream;
    FieldPtr tmpU;
    const lqcd_field *Us = U_sloppy;
    if (params->sloppy != LQCD_F64 && !Us) {
        LQCD_TRY(lqcd_field_alloc(&U->lat, LQCD_GAUGE, params->sloppy, 12, &tmpU.f));
        LQCD_TRY(lqcd_field_copy(tmpU.f, U, s));
        Us = tmpU.f;
    }
    CgWorkspace ws;
    lqcd_status st = cg_solve_ws(ws, x, U, Us, b, kappa, *params, info, s);
    cudaStreamSynchronize(s); // work space is released on return
    return st;
}
