// service.cu -- a continuous-batching service for Wilson-Dirac solves.
//
// Requests arrive at any time (lqcd_solve_submit) for point-source solves of
// the full Wilson operator M x = b on gauge fields kept resident on the device.
// A worker thread admits queued requests in arrival order while the device
// memory their work needs fits a budget (the paper keeps fields resident and
// manages device memory itself, Sec. 5; here admission replaces spilling), sets
// up each right-hand side, and advances every admitted right-hand side
// together, one graph-captured chunk of CG iterations at a time, with the
// multi-system engine of batch.cu: right-hand sides of new requests join
// between chunks as memory frees up, finished ones leave.  Each solve is
// even-odd reduced: b'_e = b_e + kappa D_eo b_o, CG on Mhat^dag Mhat y =
// Mhat^dag b'_e, x_e = y, x_o = b_o + kappa D_oe x_e; the residual reported is
// that of the full M, |b - M x| / |b|, recomputed in FP64, and a solve whose
// full residual misses the tolerance continues from its solution with a
// tighter normal-equation tolerance.  Every right-hand side gives the same
// result alone or in any mix (per-system arithmetic does not depend on the
// batch).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>

#include "batch.cuh"
#include "df64.cuh"
#include "dslash_site.cuh"

namespace lqcd {

using Clock = std::chrono::steady_clock;

// one element of a point source: component comp (spin*3 + colour) at
// checkerboard site cb set to v, in FP64 or float-float storage
__global__ void point_set_kernel(double2 *f, int Vh, int cb, int comp, double v)
{
    f[(size_t)comp * Vh + cb] = make_double2(v, 0.0);
}
__global__ void point_set_df_kernel(float4 *f, int Vh, int cb, int comp, float v)
{
    f[(size_t)comp * Vh + cb] = make_float4(v, 0.f, 0.f, 0.f);
}

// out = x + b D in at the listed output sites only (FP64; x may be absent).
// A point source and the operators applied to it are non-zero on a few dozen
// sites, so the set-up of a right-hand side touches only those.
template <bool DAG>
__global__ void hop_sites_kernel(SpinorRef<LQCD_F64> out, SpinorRef<LQCD_F64> in, GaugeRef<LQCD_F64> U, Geo g,
                                 int out_par, SpinorRef<LQCD_F64> x, double b, const int *sites, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cb = sites[i];
    Sp<double> d = dslash_site<double, LQCD_F64, LQCD_F64, DAG>(in, U, g, cb, out_par);
    if (x.d) {
        Sp<double> xv = x.load_rw<double>(cb);
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) d.c[s][c] = xv.c[s][c] + b * d.c[s][c];
    } else {
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) d.c[s][c] = b * d.c[s][c];
    }
    out.store(cb, d);
}

__global__ void zero_sites_kernel(SpinorRef<LQCD_F64> f, const int *sites, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Sp<double> z;
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < 3; c++) z.c[s][c] = Cx<double>{0.0, 0.0};
    f.store(sites[i], z);
}

// block partials of |y - b_e|^2 for a float-float field y and the even part
// b_e of a unit point source (component comp at site src_cb; src_cb < 0: none)
__global__ void __launch_bounds__(256) point_residual_kernel(SpinorRef<PREC_DF> y, int src_cb, int comp,
                                                             double *partials, int Vh)
{
    int cb = blockIdx.x * 256 + threadIdx.x;
    double n2[1] = {0.0};
    if (cb < Vh) {
#pragma unroll
        for (int k = 0; k < 12; k++) {
            float4 v = y.d[(size_t)k * Vh + cb];
            double re = (double)v.x + (double)v.y, im = (double)v.z + (double)v.w;
            if (cb == src_cb && k == comp) re -= 1.0;
            n2[0] += re * re + im * im;
        }
    }
    block_sum_store<1, 256>(n2, partials, (int)gridDim.x);
}

struct SvcGauge {
    lqcd_field *U = nullptr; // borrowed FP64 links
    FieldPtr Us, Udf;         // sloppy copy and float-float copy shared by every solve on it
    CgWorkspace shared;       // transient float-float fields shared by its solves
    // set-up (FP64, zero outside the few sites a set-up writes, cleared after
    // each use) and check (float-float) temporaries, used one solve at a time
    FieldPtr bo, bp, to, src, bo_df, xo_df, mxe_df;
    DevBuf part, scal;
    bool ready = false;
    // solver work spaces of finished right-hand sides, reused by the next
    // ones (at most one request's worth; their bytes count against the
    // admission budget like those of running right-hand sides)
    std::vector<std::unique_ptr<CgWorkspace>> idle;
    size_t fixed_bytes = 0; // the link copies and shared temporaries above, once set up
};

constexpr size_t IDLE_WS_MAX = 12;

struct SvcRhs {
    int comp = 0;
    std::unique_ptr<CgWorkspace> ws;
    FieldPtr y, xo; // the solution halves
    CgRun run;
    int refinements = 0;
    double tol_n = 0;
    bool finalized = false;
    double rel_res = 0;
    int iters = 0;
    lqcd_status status = LQCD_OK;
};

struct SvcRequest {
    uint64_t ticket = 0;
    lqcd_solve_req req{};
    // the source's parity and checkerboard index, and the checkerboard sites
    // of b'_e (S1), of D_oe^dag b'_e (T, odd) and of Mhat^dag b'_e (S2)
    int par = 0, cb = 0, n1 = 0, nt = 0, n2 = 0;
    DevBuf sites; // S1, T, S2 in a row
    Clock::time_point t_submit, t_admit, t_done;
    std::vector<std::unique_ptr<SvcRhs>> rhs;
    size_t bytes = 0;
    bool admitted = false, done = false;
    lqcd_solve_result result{};
};

} // namespace lqcd

using namespace lqcd;

struct lqcd_service {
    lqcd_service_params prm{};
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<std::unique_ptr<SvcGauge>> gauges;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<SvcRequest *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<SvcRequest>> reqs;
    std::vector<SvcRequest *> running;
    uint64_t next_ticket = 1;
    size_t bytes_in_use = 0; // admitted right-hand sides and unreleased solutions
    size_t idle_bytes = 0;   // the gauge fields' pools of idle solver work spaces
    bool stop = false;
    BatchSolver bs;
    std::thread worker;
    lqcd_status fatal = LQCD_OK;
    std::string fatal_msg;
};

namespace lqcd {

// device bytes of one right-hand side's solver work space as
// CgWorkspace::ensure allocates it when the float-float links and temporaries
// are the gauge field's: float-float solution and source, FP32 solution
// increment, four sloppy vectors, the scalars and the block partials
static size_t ws_bytes(const lqcd_lattice &lat, lqcd_prec sloppy)
{
    const int Vh = make_geo(lat).Vh;
    const size_t s = sloppy == LQCD_F32 ? 96 : (sloppy == LQCD_F16N ? 52 : 48);
    const size_t np = (size_t)std::max(std::max(nblocks_for(Vh, 64), nblocks_for(Vh, CG_BLOCK)), 2048);
    return (size_t)Vh * (2 * 192 + 96 + 4 * s) + sizeof(CgScalars) + np * sizeof(double) + 16 * sizeof(double);
}

// device bytes one right-hand side holds while admitted: its work space and
// the FP64 solution halves
static size_t rhs_bytes(const lqcd_lattice &lat, lqcd_prec sloppy)
{
    return ws_bytes(lat, sloppy) + (size_t)make_geo(lat).Vh * 2 * 192;
}

static lqcd_status gauge_setup(lqcd_service *S, SvcGauge &g)
{
    if (g.ready) return LQCD_OK;
    cudaStream_t s = S->stream;
    const lqcd_lattice &lat = g.U->lat;
    LQCD_TRY(lqcd_field_alloc(&lat, LQCD_GAUGE, S->prm.cg.sloppy, 12, &g.Us.f));
    LQCD_TRY(lqcd_field_copy(g.Us.f, g.U, s));
    LQCD_TRY(field_alloc_df(&lat, LQCD_GAUGE, &g.Udf.f));
    LQCD_TRY(split_links(g.Udf.f, g.U, s));
    g.shared.temps_only = true;
    LQCD_TRY(g.shared.ensure(lat, S->prm.cg.sloppy, s));
    LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_ODD, LQCD_F64, 0, &g.bo.f));
    LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &g.bp.f));
    LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_ODD, LQCD_F64, 0, &g.to.f));
    LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &g.src.f));
    LQCD_TRY(field_alloc_df(&lat, LQCD_SPINOR_ODD, &g.bo_df.f));
    LQCD_TRY(field_alloc_df(&lat, LQCD_SPINOR_ODD, &g.xo_df.f));
    LQCD_TRY(field_alloc_df(&lat, LQCD_SPINOR_EVEN, &g.mxe_df.f));
    for (lqcd_field *f : {g.bo.f, g.bp.f, g.to.f, g.src.f, g.bo_df.f})
        LQCD_CUDA(cudaMemsetAsync(f->data, 0, f->bytes, s));
    LQCD_TRY(g.part.alloc(sizeof(double) * (nblocks_for(make_geo(lat).Vh, 256) + 1), s));
    LQCD_TRY(g.scal.alloc(sizeof(double) * 4, s));
    size_t fixed = g.shared.bytes() + g.part.bytes + g.scal.bytes;
    for (const FieldPtr *f : {&g.Us, &g.Udf, &g.bo, &g.bp, &g.to, &g.src, &g.bo_df, &g.xo_df, &g.mxe_df})
        fixed += f->f->bytes + f->f->norm_bytes;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        g.fixed_bytes = fixed;
    }
    g.ready = true;
    return LQCD_OK;
}

// the site lists of a request's source (host; periodic neighbours)
static lqcd_status source_sites(SvcRequest &r, const lqcd_lattice &lat, cudaStream_t s)
{
    const int *L = lat.dims;
    auto lex = [&](const int *c) { return c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3])); };
    auto neighbours = [&](int i, std::set<int> &out) {
        int c[4] = {i % L[0], (i / L[0]) % L[1], (i / (L[0] * L[1])) % L[2], i / (L[0] * L[1] * L[2])};
        for (int mu = 0; mu < 4; mu++)
            for (int d : {1, L[mu] - 1}) {
                int n[4] = {c[0], c[1], c[2], c[3]};
                n[mu] = (n[mu] + d) % L[mu];
                out.insert(lex(n));
            }
    };
    int src = lex(r.req.site);
    r.par = (r.req.site[0] + r.req.site[1] + r.req.site[2] + r.req.site[3]) & 1;
    r.cb = src >> 1;
    std::set<int> s1, t, s2;
    if (r.par == 0)
        s1.insert(src);
    else
        neighbours(src, s1);
    for (int i : s1) neighbours(i, t);
    s2 = s1;
    for (int i : t) neighbours(i, s2);
    std::vector<int> all;
    for (const std::set<int> *set : {&s1, &t, &s2})
        for (int i : *set) all.push_back(i >> 1);
    r.n1 = (int)s1.size(), r.nt = (int)t.size(), r.n2 = (int)s2.size();
    LQCD_TRY(r.sites.alloc(all.size() * sizeof(int), s));
    // pageable source: the copy has taken the host data when the call returns
    LQCD_CUDA(cudaMemcpyAsync(r.sites.p, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    return LQCD_OK;
}

template <bool DAG>
static lqcd_status hop_sites(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, const lqcd_field *x,
                             double b, const int *sites, int n, cudaStream_t s)
{
    SpinorRef<LQCD_F64> xr = x ? spinor_ref<LQCD_F64>(x) : SpinorRef<LQCD_F64>{nullptr, in->Vh};
    hop_sites_kernel<DAG><<<nblocks_for(n, 64), 64, 0, s>>>(spinor_ref<LQCD_F64>(out), spinor_ref<LQCD_F64>(in),
                                                            gauge_ref<LQCD_F64>(U), make_geo(U->lat),
                                                            out->kind == LQCD_SPINOR_EVEN ? 0 : 1, xr, b, sites, n);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

static lqcd_status zero_sites(lqcd_field *f, const int *sites, int n, cudaStream_t s)
{
    zero_sites_kernel<<<nblocks_for(n, 64), 64, 0, s>>>(spinor_ref<LQCD_F64>(f), sites, n);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

// start (or restart from its solution) one right-hand side's normal-equation
// solve: b'_e = b_e + kappa D_eo b_o and src = Mhat^dag b'_e on their few
// non-zero sites, then the solver's start, then the temporaries cleared
static lqcd_status rhs_start(lqcd_service *S, SvcGauge &g, SvcRequest &r, SvcRhs &h, bool warm)
{
    cudaStream_t s = S->stream;
    const double kappa = r.req.kappa;
    const int *s1 = (const int *)r.sites.p, *t = s1 + r.n1, *s2 = t + r.nt;
    const int Vh = g.bp.f->Vh;
    if (r.par == 0) {
        point_set_kernel<<<1, 1, 0, s>>>((double2 *)g.bp.f->data, Vh, r.cb, h.comp, 1.0);
    } else {
        point_set_kernel<<<1, 1, 0, s>>>((double2 *)g.bo.f->data, Vh, r.cb, h.comp, 1.0);
        LQCD_LAUNCHED();
        LQCD_TRY(hop_sites<false>(g.bp.f, g.U, g.bo.f, nullptr, kappa, s1, r.n1, s));
        point_set_kernel<<<1, 1, 0, s>>>((double2 *)g.bo.f->data, Vh, r.cb, h.comp, 0.0);
    }
    LQCD_LAUNCHED();
    LQCD_TRY(hop_sites<true>(g.to.f, g.U, g.bp.f, nullptr, 1.0, t, r.nt, s));
    LQCD_TRY(hop_sites<true>(g.src.f, g.U, g.to.f, g.bp.f, -kappa * kappa, s2, r.n2, s));
    h.run = CgRun();
    h.run.ws = h.ws.get(), h.run.x = h.y.f, h.run.U = g.U, h.run.Us = g.Us.f, h.run.b = g.src.f;
    h.run.kappa = kappa;
    h.run.prm = S->prm.cg;
    h.run.prm.tol = h.tol_n;
    h.run.prm.guess = warm ? 1 : 0;
    // start() copies src into the solve's own float-float source before any
    // later work on this stream; a failure leaves the run done with its status
    h.run.start(s, (CgScalars *)h.ws->sc.p);
    LQCD_TRY(zero_sites(g.bp.f, s1, r.n1, s));
    LQCD_TRY(zero_sites(g.to.f, t, r.nt, s));
    LQCD_TRY(zero_sites(g.src.f, s2, r.n2, s));
    if (!h.run.done) S->bs.add(&h.run);
    return LQCD_OK;
}

static lqcd_status admit(lqcd_service *S, SvcRequest &r)
{
    SvcGauge &g = *S->gauges[r.req.gauge];
    LQCD_TRY(gauge_setup(S, g));
    const lqcd_lattice &lat = g.U->lat;
    LQCD_TRY(source_sites(r, lat, S->stream));
    for (int k = 0; k < r.req.nrhs; k++) {
        std::unique_ptr<SvcRhs> h(new SvcRhs());
        h->comp = k;
        h->tol_n = S->prm.cg.tol / 10.0;
        if (!g.idle.empty()) {
            h->ws = std::move(g.idle.back());
            g.idle.pop_back();
            std::lock_guard<std::mutex> lk(S->mu);
            S->idle_bytes -= ws_bytes(lat, S->prm.cg.sloppy);
        } else {
            h->ws.reset(new CgWorkspace());
        }
        h->ws->udf_ext = g.Udf.f;
        h->ws->tmp_from = &g.shared;
        LQCD_TRY(h->ws->ensure(lat, S->prm.cg.sloppy, S->stream));
        LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &h->y.f));
        LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_ODD, LQCD_F64, 0, &h->xo.f));
        LQCD_TRY(rhs_start(S, g, r, *h, false));
        r.rhs.push_back(std::move(h));
    }
    return LQCD_OK;
}

// x_o = b_o + kappa D_oe x_e and the full residual |b - M x| / |b| (|b| = 1),
// both from the solver's float-float solution with float-float links and
// arithmetic; a miss continues from x_e with a tighter normal-equation
// tolerance.  The odd rows of b - M x are b_o - x_o + kappa D_oe x_e, zero by
// the definition of x_o up to its rounding, so the even rows are the residual.
static lqcd_status rhs_check(lqcd_service *S, SvcGauge &g, SvcRequest &r, SvcRhs &h, bool *restarted)
{
    cudaStream_t s = S->stream;
    const double kappa = r.req.kappa;
    *restarted = false;
    h.iters += h.run.inf.iters;
    if (h.run.status != LQCD_OK) {
        h.status = h.run.status;
        h.finalized = true;
        return LQCD_OK;
    }
    const lqcd_field *xdf = h.ws->xdf.f;
    const int Vh = xdf->Vh;
    if (r.par == 1) {
        point_set_df_kernel<<<1, 1, 0, s>>>((float4 *)g.bo_df.f->data, Vh, r.cb, h.comp, 1.f);
        LQCD_LAUNCHED();
    }
    LQCD_TRY(dslash_xpay(g.xo_df.f, g.Udf.f, xdf, 0, g.bo_df.f, kappa, nullptr, nullptr, s));
    LQCD_TRY(dslash_xpay(g.mxe_df.f, g.Udf.f, g.xo_df.f, 0, xdf, -kappa, nullptr, nullptr, s));
    if (r.par == 1) {
        point_set_df_kernel<<<1, 1, 0, s>>>((float4 *)g.bo_df.f->data, Vh, r.cb, h.comp, 0.f);
        LQCD_LAUNCHED();
    }
    int nb = nblocks_for(Vh, 256);
    point_residual_kernel<<<nb, 256, 0, s>>>(spinor_ref<PREC_DF>(g.mxe_df.f), r.par == 0 ? r.cb : -1, h.comp,
                                             (double *)g.part.p, Vh);
    LQCD_LAUNCHED();
    LQCD_TRY(reduce_partials((double *)g.part.p, nb, 1, (double *)g.scal.p, s));
    LQCD_TRY(df_to_f64(h.xo.f, g.xo_df.f, s));
    double rr = 0;
    LQCD_TRY(read_scalars((double *)g.scal.p, &rr, 1, s));
    h.rel_res = std::sqrt(rr);
    if (!std::isfinite(h.rel_res)) {
        h.status = LQCD_ENUMERIC;
        h.finalized = true;
        return LQCD_OK;
    }
    if (h.rel_res <= S->prm.cg.tol || h.refinements >= 3) {
        h.status = h.rel_res <= S->prm.cg.tol ? LQCD_OK : LQCD_ENOCONV;
        h.finalized = true;
        return LQCD_OK;
    }
    // the full residual scales roughly like the normal-equation one: aim at half the tolerance
    h.refinements++;
    h.tol_n *= std::min(0.1, std::max(1e-3, 0.5 * S->prm.cg.tol / h.rel_res));
    LQCD_TRY(rhs_start(S, g, r, h, true));
    if (h.run.done) return rhs_check(S, g, r, h, restarted);
    *restarted = true;
    return LQCD_OK;
}

static void finish_request(lqcd_service *S, SvcRequest &r, lqcd_status st)
{
    r.t_done = Clock::now();
    lqcd_solve_result &o = r.result;
    o.status = st;
    o.nrhs = r.req.nrhs;
    o.iters = 0;
    o.refinements = 0;
    o.true_rel_res_max = 0;
    size_t idle_added = 0;
    for (auto &h : r.rhs) {
        o.iters += h->iters;
        o.refinements += h->refinements;
        o.true_rel_res_max = std::max(o.true_rel_res_max, h->rel_res);
        if (o.status == LQCD_OK && h->status != LQCD_OK) o.status = h->status;
        // the solver fields go back to the gauge field's pool (or are freed);
        // the solution halves stay until release
        SvcGauge &g = *S->gauges[r.req.gauge];
        if (h->ws && h->ws->ready && g.idle.size() < IDLE_WS_MAX) {
            g.idle.push_back(std::move(h->ws));
            idle_added += ws_bytes(g.U->lat, S->prm.cg.sloppy);
        }
        h->ws.reset();
    }
    o.queue_s = std::chrono::duration<double>(r.t_admit - r.t_submit).count();
    o.latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
    std::lock_guard<std::mutex> lk(S->mu);
    S->idle_bytes += idle_added;
    S->bytes_in_use -= r.bytes;
    r.bytes = (size_t)r.req.nrhs * 2 * 192 * (size_t)make_geo(S->gauges[r.req.gauge]->U->lat).Vh;
    S->bytes_in_use += r.bytes; // the solutions until lqcd_solve_release
    r.done = true;
    S->cv.notify_all();
}

static lqcd_status worker_step(lqcd_service *S)
{
    // admit in arrival order while the budget allows (a request alone always
    // runs).  The budget covers the admitted right-hand sides, the unreleased
    // solutions and the pooled idle work spaces; a request reuses its own
    // gauge field's idle work spaces, and those of other gauge fields are
    // freed when the request would not fit beside them.
    std::vector<SvcRequest *> admitted;
    std::vector<std::unique_ptr<CgWorkspace>> evicted;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        std::vector<size_t> claimed(S->gauges.size(), 0);
        while (!S->queue.empty()) {
            SvcRequest *r = S->queue.front();
            const size_t need = r->bytes;
            const int gi = r->req.gauge;
            SvcGauge &gr = *S->gauges[gi];
            const size_t wsb = ws_bytes(gr.U->lat, S->prm.cg.sloppy);
            // the idle work spaces this request will take (those not claimed
            // by a request admitted before it in this pass)
            const size_t take = std::min(gr.idle.size() - claimed[gi], (size_t)r->req.nrhs);
            bool alone = S->running.empty() && admitted.empty();
            bool fits = S->bytes_in_use + need <= S->prm.hbm_budget; // once the other idle work spaces are freed
            bool rhs_ok = S->prm.max_active_rhs <= 0 ||
                          (int)S->bs.active.size() + r->req.nrhs <= S->prm.max_active_rhs;
            if (!alone && !(fits && rhs_ok)) break;
            claimed[gi] += take;
            // free idle work spaces, other gauge fields' first, then the
            // unclaimed ones of this gauge field, while the resident total
            // would exceed the budget
            auto over = [&] { return S->bytes_in_use + need + S->idle_bytes - take * wsb > S->prm.hbm_budget; };
            for (int pass = 0; pass < 2; pass++)
                for (size_t k = 0; k < S->gauges.size(); k++) {
                    if ((pass == 0) == ((int)k == gi)) continue;
                    SvcGauge &g = *S->gauges[k];
                    const size_t b = ws_bytes(g.U->lat, S->prm.cg.sloppy);
                    // admissions take work spaces from the back of a pool
                    while (g.idle.size() > claimed[k] && over()) {
                        evicted.push_back(std::move(g.idle.front()));
                        g.idle.erase(g.idle.begin());
                        S->idle_bytes -= b;
                    }
                }
            S->queue.pop_front();
            S->bytes_in_use += need;
            r->admitted = true;
            r->t_admit = Clock::now();
            admitted.push_back(r);
        }
        if (admitted.empty() && S->running.empty()) {
            if (S->stop) return LQCD_OK;
            S->cv.wait_for(lk, std::chrono::milliseconds(50));
            return LQCD_OK;
        }
    }
    evicted.clear(); // freed before the admissions allocate
    for (SvcRequest *r : admitted) {
        lqcd_status rc = admit(S, *r);
        if (rc != LQCD_OK) {
            for (auto &h : r->rhs) {
                h->finalized = true;
                h->status = rc;
            }
            finish_request(S, *r, rc);
            continue;
        }
        S->running.push_back(r);
    }
    LQCD_TRY(S->bs.step(S->prm.cg.sloppy, S->stream));
    std::vector<SvcRequest *> still;
    for (SvcRequest *r : S->running) {
        SvcGauge &g = *S->gauges[r->req.gauge];
        bool all = true;
        for (auto &h : r->rhs) {
            if (h->finalized) continue;
            if (!h->run.done) {
                all = false;
                continue;
            }
            bool restarted = false;
            LQCD_TRY(rhs_check(S, g, *r, *h, &restarted));
            if (!h->finalized) all = false;
        }
        if (all)
            finish_request(S, *r, LQCD_OK);
        else
            still.push_back(r);
    }
    S->running.swap(still);
    return LQCD_OK;
}

static void worker_main(lqcd_service *S)
{
    cudaSetDevice(S->device);
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->stop && S->queue.empty() && S->running.empty()) break;
        }
        lqcd_status rc = worker_step(S);
        if (rc != LQCD_OK) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->fatal = rc;
            S->fatal_msg = lqcd_last_error();
            for (SvcRequest *r : S->running) {
                r->done = true;
                r->result.status = rc;
            }
            for (SvcRequest *r : S->queue) {
                r->done = true;
                r->result.status = rc;
            }
            S->running.clear();
            S->queue.clear();
            S->cv.notify_all();
            break;
        }
    }
    cudaStreamSynchronize(S->stream);
}

} // namespace lqcd

extern "C" {

lqcd_status lqcd_service_create(const lqcd_service_params *params, lqcd_service **out)
{
    LQCD_REQUIRE(params && out, "service_create: NULL argument");
    LQCD_REQUIRE(params->cg.sloppy != LQCD_F64 && params->cg.tol > 0 && params->cg.maxiter > 0 &&
                     params->cg.delta > 0 && params->cg.delta < 1,
                 "service_create: needs a mixed-precision solver (sloppy F32/F16N/BF16, 0 < delta < 1)");
    LQCD_REQUIRE(params->hbm_budget > 0, "service_create: hbm_budget must be positive");
    lqcd_service *S = new lqcd_service();
    S->prm = *params;
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete S;
        return cuda_fail(e, "service stream", __FILE__, __LINE__);
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return LQCD_OK;
}

lqcd_status lqcd_service_add_gauge(lqcd_service *S, lqcd_field *U, int *id)
{
    LQCD_REQUIRE(S && U && id, "service_add_gauge: NULL argument");
    LQCD_REQUIRE(U->kind == LQCD_GAUGE && U->prec == LQCD_F64, "service_add_gauge: U must be an F64 gauge field");
    std::lock_guard<std::mutex> lk(S->mu);
    std::unique_ptr<SvcGauge> g(new SvcGauge());
    g->U = U;
    S->gauges.push_back(std::move(g));
    *id = (int)S->gauges.size() - 1;
    return LQCD_OK;
}

lqcd_status lqcd_solve_submit(lqcd_service *S, const lqcd_solve_req *req, uint64_t *ticket)
{
    LQCD_REQUIRE(S && req && ticket, "solve_submit: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->fatal != LQCD_OK) {
        set_error("solve_submit: the service stopped after an error: %s", S->fatal_msg.c_str());
        return S->fatal;
    }
    LQCD_REQUIRE(req->gauge >= 0 && req->gauge < (int)S->gauges.size(), "solve_submit: unknown gauge %d", req->gauge);
    LQCD_REQUIRE(req->nrhs >= 1 && req->nrhs <= 12, "solve_submit: nrhs must lie in 1..12");
    const lqcd_lattice &lat = S->gauges[req->gauge]->U->lat;
    for (int mu = 0; mu < 4; mu++)
        LQCD_REQUIRE(req->site[mu] >= 0 && req->site[mu] < lat.dims[mu], "solve_submit: source site outside the lattice");
    std::unique_ptr<SvcRequest> r(new SvcRequest());
    r->ticket = S->next_ticket++;
    r->req = *req;
    r->t_submit = Clock::now();
    r->bytes = (size_t)req->nrhs * rhs_bytes(lat, S->prm.cg.sloppy);
    *ticket = r->ticket;
    S->queue.push_back(r.get());
    S->reqs[r->ticket] = std::move(r);
    S->cv.notify_all();
    return LQCD_OK;
}

lqcd_status lqcd_solve_poll(lqcd_service *S, uint64_t ticket, lqcd_solve_result *out)
{
    LQCD_REQUIRE(S && out, "solve_poll: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    LQCD_REQUIRE(it != S->reqs.end(), "solve_poll: unknown ticket %llu", (unsigned long long)ticket);
    if (!it->second->done) return LQCD_EAGAIN;
    *out = it->second->result;
    return LQCD_OK;
}

lqcd_status lqcd_solve_solution(lqcd_service *S, uint64_t ticket, int k, lqcd_field **x_even, lqcd_field **x_odd)
{
    LQCD_REQUIRE(S && x_even && x_odd, "solve_solution: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    LQCD_REQUIRE(it != S->reqs.end(), "solve_solution: unknown ticket");
    SvcRequest &r = *it->second;
    if (!r.done) return LQCD_EAGAIN;
    LQCD_REQUIRE(k >= 0 && k < (int)r.rhs.size(), "solve_solution: right-hand side %d not available", k);
    *x_even = r.rhs[k]->y.f;
    *x_odd = r.rhs[k]->xo.f;
    return LQCD_OK;
}

lqcd_status lqcd_solve_release(lqcd_service *S, uint64_t ticket)
{
    LQCD_REQUIRE(S, "solve_release: NULL service");
    std::unique_ptr<SvcRequest> r;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        LQCD_REQUIRE(it != S->reqs.end(), "solve_release: unknown ticket");
        if (!it->second->done) return LQCD_EAGAIN;
        S->bytes_in_use -= it->second->bytes;
        r = std::move(it->second);
        S->reqs.erase(it);
        S->cv.notify_all();
    }
    return LQCD_OK; // r's fields are freed here
}

lqcd_status lqcd_service_bytes(lqcd_service *S, size_t *counted, size_t *fixed)
{
    LQCD_REQUIRE(S && counted && fixed, "service_bytes: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *counted = S->bytes_in_use + S->idle_bytes;
    *fixed = 0;
    for (auto &g : S->gauges) *fixed += g->fixed_bytes;
    return LQCD_OK;
}

lqcd_status lqcd_service_destroy(lqcd_service *S)
{
    if (!S) return LQCD_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    S->bs.release();
    S->reqs.clear();
    S->gauges.clear();
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
    return LQCD_OK;
}

} // extern "C"
