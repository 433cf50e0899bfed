// batch.cu -- many CG solves at once.
//
// Independent systems Mhat^dag Mhat x_i = b_i (each on its own lattice, gauge
// field and kappa: the solves of a batch of Markov chains, or the right-hand
// sides of queued solve requests) share their launches: each kernel of a CG
// iteration runs over the union of the systems' sites, every block belonging to
// one system (a block -> system map) and reading that system's geometry,
// fields and scalars from a descriptor table.  Small lattices, which alone fill
// a few of the 152 SMs, then fill the GPU together, and the launch count per
// iteration does not grow with the number of systems.  Per-system arithmetic
// is that of the single-system kernels (same block size, same reduction order),
// so every system's iterates are bitwise those of its solve alone.
//
// A chunk of iterations is captured once as a CUDA graph and replayed while the
// set of systems is unchanged; a system whose device pause flag is raised (a
// reliable update, convergence, maxiter) is handled by its own CgRun between
// chunks, and leaves the batch when done.  Systems can be added between chunks.
#include <algorithm>

#include "batch.cuh"
#include "dslash_df.cuh"
#include "dslash_packed.cuh"
#include "dslash_site.cuh"

namespace lqcd {

constexpr int BCHUNK = 4;

// ---------------------------------------------------------------- kernels

// D (DAG: D^dag) at site cb of one system: FP16+norm in the hopping-term
// form of the single-field kernels (FORM 2 packed FP32x2 arithmetic, else
// the links prefetched into shared memory, which gives the bits of the
// gathered form), other precisions gathered
template <lqcd_prec SP, bool DAG, int FORM>
__device__ __forceinline__ Sp<float> sys_site(const SpinorRef<SP> &in, const GaugeRef<SP> &U, const Geo &g, int cb,
                                              int out_par)
{
    if constexpr (SP == LQCD_F16N && FORM == 2)
        return packed_site<DAG>(in, U, g, cb, out_par);
    else if constexpr (SP == LQCD_F16N)
        return prefetch_site<float, DAG>(in, U, g, cb, out_par);
    else
        return dslash_site<float, SP, SP, DAG>(in, U, g, cb, out_par);
}

// blocks of 128 per SM for the FP16+norm kernels, the register budgets of the
// single-system hop (dslash.cu): 5 for the plain steps, 6 for the reducing
// ones (fewer spills than 7 for all; the 64 chains ran at the same rate)
template <lqcd_prec SP, bool REDUCING>
constexpr int min_blocks() { return SP != LQCD_F16N ? 1 : (REDUCING ? 6 : 5); }

// step 0: tmp = D_oe p; step 2: tmp = D_oe^dag-hop t
template <lqcd_prec SP, bool DAG, int FORM>
__global__ void __launch_bounds__(DS_BLOCK, min_blocks<SP, false>()) batch_dslash_plain(const SysDesc<SP> *sys, const int2 *bmap)
{
    const int2 m = bmap[blockIdx.x];
    const SysDesc<SP> &d = sys[m.x];
    if (d.sc->pause) return;
    int cb = m.y * DS_BLOCK + threadIdx.x;
    if (cb >= d.g.Vh) return;
    const SpinorRef<SP> &in = DAG ? d.t : d.p;
    d.tmp.store(cb, sys_site<SP, DAG, FORM>(in, d.U, d.g, cb, 1));
}

// step 1: t = p - kappa^2 D_eo tmp, block sums of |t|^2
template <lqcd_prec SP, int FORM>
__global__ void __launch_bounds__(DS_BLOCK, min_blocks<SP, true>()) batch_dslash_xpay(const SysDesc<SP> *sys, const int2 *bmap)
{
    const int2 m = bmap[blockIdx.x];
    const SysDesc<SP> &d = sys[m.x];
    if (d.sc->pause) return;
    int cb = m.y * DS_BLOCK + threadIdx.x;
    float n2 = 0.f;
    if (cb < d.g.Vh) {
        Sp<float> v = sys_site<SP, false, FORM>(d.tmp, d.U, d.g, cb, 0);
        Sp<float> pv = d.p.template load_rw<float>(cb);
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int k = 0; k < 3; k++) v.c[a][k] = pv.c[a][k] + d.b * v.c[a][k];
        d.t.store(cb, v);
        n2 = sp_norm2(v);
    }
    // the partial of block m.y of this system, as in the single-system kernel
    double *part = d.partials;
    __shared__ double sh[DS_BLOCK / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) n2 += __shfl_down_sync(0xffffffffu, n2, off);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = (double)n2;
    __syncthreads();
    if (warp == 0) {
        double x = lane < DS_BLOCK / 32 ? sh[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) part[m.y] = x;
    }
    cg_finish<DS_BLOCK, false>(d.sc, part, d.nblocks); // pAp and alpha, as the single-system kernel
}

// step 3: Ap = t - kappa^2 D_eo^dag-hop tmp; xs += alpha p; r -= alpha Ap; block sums of |r|^2
template <lqcd_prec SP, int FORM>
__global__ void __launch_bounds__(DS_BLOCK, min_blocks<SP, true>()) batch_dslash_cg(const SysDesc<SP> *sys, const int2 *bmap)
{
    const int2 m = bmap[blockIdx.x];
    const SysDesc<SP> &d = sys[m.x];
    if (d.sc->pause) return;
    const float alpha = (float)d.sc->alpha;
    int cb = m.y * DS_BLOCK + threadIdx.x;
    float n2 = 0.f;
    if (cb < d.g.Vh) {
        Sp<float> ap = sys_site<SP, true, FORM>(d.tmp, d.U, d.g, cb, 0);
        {
            Sp<float> tv = d.t.template load_rw<float>(cb);
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int k = 0; k < 3; k++) ap.c[a][k] = tv.c[a][k] + d.b * ap.c[a][k];
        }
        Sp<float> pv = d.p.template load_rw<float>(cb);
        {
            Sp<float> xv = d.xs.template load_rw<float>(cb);
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    xv.c[a][k].re += alpha * pv.c[a][k].re;
                    xv.c[a][k].im += alpha * pv.c[a][k].im;
                }
            d.xs.store(cb, xv);
        }
        Sp<float> rv = d.r.template load_rw<float>(cb);
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int k = 0; k < 3; k++) rv.c[a][k] = rv.c[a][k] - alpha * ap.c[a][k];
        d.r.store(cb, rv);
        n2 = sp_norm2(rv);
    }
    double *part = d.partials;
    __shared__ double sh[DS_BLOCK / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) n2 += __shfl_down_sync(0xffffffffu, n2, off);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = (double)n2;
    __syncthreads();
    if (warp == 0) {
        double x = lane < DS_BLOCK / 32 ? sh[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) part[m.y] = x;
    }
    cg_finish<DS_BLOCK, true>(d.sc, part, d.nblocks); // rr, beta and the pause decision
}

// step 4: p = r + beta p
template <lqcd_prec SP>
__global__ void __launch_bounds__(DS_BLOCK) batch_p_update(const SysDesc<SP> *sys, const int2 *bmap)
{
    const int2 m = bmap[blockIdx.x];
    const SysDesc<SP> &d = sys[m.x];
    if (d.sc->pause) return;
    int cb = m.y * DS_BLOCK + threadIdx.x;
    if (cb >= d.g.Vh) return;
    float beta = (float)d.sc->beta;
    Sp<float> pv = d.p.template load_rw<float>(cb);
    Sp<float> rv = d.r.template load_rw<float>(cb);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int k = 0; k < 3; k++) pv.c[a][k] = rv.c[a][k] + beta * pv.c[a][k];
    d.p.store(cb, pv);
}

// after a chunk: every system's scalars into one array (one copy to the host)
template <lqcd_prec SP>
__global__ void batch_gather_scalars(const SysDesc<SP> *sys, CgScalars *out, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = *sys[i].sc;
}

// ---------------------------------------------------------------- reliable updates of many systems
//
// The accurate residual r = b - Mhat^dag Mhat x of every paused system in
// float-float, with shared launches: x += x_s, the four float-float hops (the
// last one forming r = b - t and its block partials), and one fixed-order
// final sum per system.
// Each block runs exactly the code and block decomposition of the
// single-system kernels (cg.cu, dslash_df.cu), so the results are bitwise
// theirs.

struct DfSys {
    Geo g;
    SpinorRef<PREC_DF> xdf, bdf, rdf, t1, tmpo;
    GaugeRef<PREC_DF> U;
    SpinorRef<LQCD_F32> xs;
    Df mk2; // -kappa^2
    double *partials, *scalars;
    int nb; // blocks of DF_SITES sites: the partials of |r|^2
};

__global__ void __launch_bounds__(CG_BLOCK) batch_accum_df_kernel(const DfSys *sys, const int2 *bmap)
{
    const int2 m = bmap[blockIdx.x];
    const DfSys &d = sys[m.x];
    const int cb = m.y * CG_BLOCK + threadIdx.x;
    if (cb < d.g.Vh) accum_df_site(d.xdf, d.xs, cb);
}

template <int STEP>
__global__ void __launch_bounds__(DF_SITES * 3, 4) batch_df_hop_kernel(const DfSys *sys, const int2 *bmap)
{
    __shared__ DfHalves sh;
    const int2 m = bmap[blockIdx.x];
    const DfSys &d = sys[m.x];
    if (STEP == 0) df_hop_block<false, false>(sh, d.tmpo, d.xdf, d.U, d.g, 1, d.xdf, Df(0), m.y);
    if (STEP == 1) df_hop_block<false, true>(sh, d.t1, d.tmpo, d.U, d.g, 0, d.xdf, d.mk2, m.y);
    if (STEP == 2) df_hop_block<true, false>(sh, d.tmpo, d.t1, d.U, d.g, 1, d.t1, Df(0), m.y);
    if (STEP == 3) df_hop_block<true, true, true>(sh, d.rdf, d.tmpo, d.U, d.g, 0, d.t1, d.mk2, m.y, d.bdf, d.partials);
}

__global__ void batch_final_sum_kernel(const DfSys *sys)
{
    const DfSys &d = sys[blockIdx.x];
    double sums[1];
    final_sum_block<1>(d.partials, d.nb, sums);
    if (threadIdx.x == 0) d.scalars[0] = sums[0];
}

// ---------------------------------------------------------------- host side

template <lqcd_prec SP>
static SysDesc<SP> make_desc(const CgRun &r)
{
    SysDesc<SP> d;
    d.g = make_geo(r.x->lat);
    d.p = spinor_ref<SP>(r.P);
    d.r = spinor_ref<SP>(r.R);
    d.t = spinor_ref<SP>(r.T);
    d.tmp = spinor_ref<SP>(r.TMP);
    d.xs = spinor_ref<LQCD_F32>(r.XS);
    d.U = gauge_ref<SP>(r.UU);
    d.b = (float)(-r.k2);
    d.sc = r.sc;
    d.partials = (double *)r.ws->partials.p;
    d.nblocks = dslash_blocks(r.Vh);
    return d;
}

BatchSolver::~BatchSolver() { release(); }

void BatchSolver::drop_graph()
{
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
}

template <lqcd_prec SP>
lqcd_status BatchSolver::enqueue_chunk(cudaStream_t s)
{
    const SysDesc<SP> *d = (const SysDesc<SP> *)descs.p;
    const int2 *bm = (const int2 *)bmap.p;
    int n = (int)active.size();
    const int form = SP == LQCD_F16N ? dslash_form_set(-1) : 1;
    for (int k = 0; k < BCHUNK; k++) {
        if (form == 2) {
            batch_dslash_plain<SP, false, 2><<<nblocks_total, DS_BLOCK, 0, s>>>(d, bm);
            batch_dslash_xpay<SP, 2><<<nblocks_total, DS_BLOCK, 0, s>>>(d, bm);
            batch_dslash_plain<SP, true, 2><<<nblocks_total, DS_BLOCK, 0, s>>>(d, bm);
            batch_dslash_cg<SP, 2><<<nblocks_total, DS_BLOCK, 0, s>>>(d, bm);
        } else {
            batch_dslash_plain<SP, false, 1><<<nblocks_total, DS_BLOCK, 0, s>>>(d, bm);
            batch_dslash_xpay<SP, 1><<<nblocks_total, DS_BLOCK, 0, s>>>(d, bm);
            batch_dslash_plain<SP, true, 1><<<nblocks_total, DS_BLOCK, 0, s>>>(d, bm);
            batch_dslash_cg<SP, 1><<<nblocks_total, DS_BLOCK, 0, s>>>(d, bm);
        }
        batch_p_update<SP><<<nblocks_total, DS_BLOCK, 0, s>>>(d, bm);
    }
    batch_gather_scalars<SP><<<nblocks_for(n, 128), 128, 0, s>>>(d, (CgScalars *)gathered.p, n);
    LQCD_CUDA(cudaGetLastError());
    return LQCD_OK;
}

template <lqcd_prec SP>
lqcd_status BatchSolver::build_tables(cudaStream_t s)
{
    std::vector<SysDesc<SP>> hd;
    std::vector<int2> hb;
    for (size_t i = 0; i < active.size(); i++) {
        const CgRun &r = *active[i];
        hd.push_back(make_desc<SP>(r));
        int nb = dslash_blocks(r.Vh);
        for (int k = 0; k < nb; k++) hb.push_back(make_int2((int)i, k));
    }
    nblocks_total = (int)hb.size();
    if (descs.bytes < hd.size() * sizeof(SysDesc<SP>)) LQCD_TRY(descs.alloc(hd.size() * sizeof(SysDesc<SP>), s));
    if (bmap.bytes < hb.size() * sizeof(int2)) LQCD_TRY(bmap.alloc(hb.size() * sizeof(int2), s));
    if (gathered.bytes < hd.size() * sizeof(CgScalars)) LQCD_TRY(gathered.alloc(hd.size() * sizeof(CgScalars), s));
    LQCD_CUDA(cudaMemcpyAsync(descs.p, hd.data(), hd.size() * sizeof(SysDesc<SP>), cudaMemcpyHostToDevice, s));
    LQCD_CUDA(cudaMemcpyAsync(bmap.p, hb.data(), hb.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    LQCD_CUDA(cudaStreamSynchronize(s)); // host vectors go out of scope
    drop_graph();
    if (use_graph) {
        // capture on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); the graph is launched on s
        if (!capture_stream) LQCD_CUDA(cudaStreamCreateWithFlags(&capture_stream, cudaStreamNonBlocking));
        LQCD_CUDA(cudaStreamBeginCapture(capture_stream, cudaStreamCaptureModeThreadLocal));
        lqcd_status rc = enqueue_chunk<SP>(capture_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(capture_stream, &g);
        if (rc != LQCD_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        LQCD_CUDA(e);
        graph = g;
        LQCD_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    }
    return LQCD_OK;
}

template <lqcd_prec SP>
lqcd_status BatchSolver::run_all(std::vector<CgRun *> &runs, cudaStream_t s)
{
    active.clear();
    for (CgRun *r : runs)
        if (!r->done) active.push_back(r);
    changed = true;
    while (!active.empty()) LQCD_TRY(chunk<SP>(s));
    return LQCD_OK;
}

// one chunk of iterations of every active system, then the pauses; done
// systems leave `active`
template <lqcd_prec SP>
lqcd_status BatchSolver::chunk(cudaStream_t s)
{
    if (changed) {
        LQCD_TRY(build_tables<SP>(s));
        changed = false;
    }
    if (use_graph) {
        LQCD_CUDA(cudaGraphLaunch(exec, s));
        g_launches.fetch_add(5 * BCHUNK + 1, std::memory_order_relaxed);
    } else {
        LQCD_TRY(enqueue_chunk<SP>(s));
        g_launches.fetch_add(5 * BCHUNK + 1, std::memory_order_relaxed);
    }
    // read every active system's scalars (gathered by the chunk's last kernel)
    if (pinned_n < active.size()) {
        if (pinned_h) cudaFreeHost(pinned_h);
        pinned_h = nullptr;
        pinned_n = 0;
        LQCD_CUDA(cudaMallocHost((void **)&pinned_h, sizeof(CgScalars) * active.size()));
        pinned_n = active.size();
    }
    LQCD_CUDA(cudaMemcpyAsync(pinned_h, gathered.p, sizeof(CgScalars) * active.size(), cudaMemcpyDeviceToHost, s));
    LQCD_CUDA(cudaStreamSynchronize(s));
    // Pauses: the systems with their own float-float temporaries enqueue
    // their accurate residuals together and share one read-back; a system
    // that borrows another workspace's temporaries (the solve service) is
    // handled alone, since the next system's residual would overwrite them.
    std::vector<CgRun *> paused;
    for (size_t i = 0; i < active.size(); i++) {
        CgRun *r = active[i];
        if (!pinned_h[i].pause) continue;
        if (r->ws->tmp_from)
            r->on_pause(pinned_h[i], s);
        else if (r->pause_record(pinned_h[i]))
            paused.push_back(r);
    }
    if (!paused.empty()) {
        LQCD_TRY(residuals_df(paused, s));
        if (pinned_rr_n < paused.size()) {
            if (pinned_rr) cudaFreeHost(pinned_rr);
            pinned_rr = nullptr;
            pinned_rr_n = 0;
            LQCD_CUDA(cudaMallocHost((void **)&pinned_rr, sizeof(double) * paused.size()));
            pinned_rr_n = paused.size();
        }
        for (size_t j = 0; j < paused.size(); j++)
            LQCD_CUDA(cudaMemcpyAsync(&pinned_rr[j], paused[j]->pause_result_dev(), sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
        LQCD_CUDA(cudaStreamSynchronize(s));
        for (size_t j = 0; j < paused.size(); j++) paused[j]->pause_end(pinned_rr[j], s);
    }
    std::vector<CgRun *> still;
    for (CgRun *r : active) {
        if (r->done)
            changed = true;
        else
            still.push_back(r);
    }
    active.swap(still);
    return LQCD_OK;
}

// the accurate residuals of the paused systems with shared launches (their
// |r|^2 land in each system's pause_result_dev)
lqcd_status BatchSolver::residuals_df(const std::vector<CgRun *> &runs, cudaStream_t s)
{
    std::vector<DfSys> hd;
    std::vector<int2> hdf, hbb;
    for (size_t i = 0; i < runs.size(); i++) {
        const CgRun &r = *runs[i];
        CgWorkspace &w = *r.ws;
        DfSys d;
        d.g = make_geo(r.x->lat);
        d.xdf = spinor_ref<PREC_DF>(w.xdf.f);
        d.bdf = spinor_ref<PREC_DF>(w.bdf.f);
        d.rdf = spinor_ref<PREC_DF>(w.rdf_());
        d.t1 = spinor_ref<PREC_DF>(w.t1());
        d.tmpo = spinor_ref<PREC_DF>(w.tmpo());
        d.U = gauge_ref<PREC_DF>(w.udf());
        d.xs = spinor_ref<LQCD_F32>(r.XS);
        d.mk2 = Df(-(r.kappa * r.kappa));
        d.partials = (double *)w.partials.p;
        d.scalars = r.pause_result_dev();
        d.nb = nblocks_for(d.g.Vh, DF_SITES);
        hd.push_back(d);
        for (int k = 0; k < d.nb; k++) hdf.push_back(make_int2((int)i, k));
        for (int k = 0; k < nblocks_for(d.g.Vh, CG_BLOCK); k++) hbb.push_back(make_int2((int)i, k));
    }
    if (df_descs.bytes < hd.size() * sizeof(DfSys)) LQCD_TRY(df_descs.alloc(hd.size() * sizeof(DfSys), s));
    if (df_map.bytes < hdf.size() * sizeof(int2)) LQCD_TRY(df_map.alloc(hdf.size() * sizeof(int2), s));
    if (bb_map.bytes < hbb.size() * sizeof(int2)) LQCD_TRY(bb_map.alloc(hbb.size() * sizeof(int2), s));
    // pageable sources: the copies have taken the host data when they return
    LQCD_CUDA(cudaMemcpyAsync(df_descs.p, hd.data(), hd.size() * sizeof(DfSys), cudaMemcpyHostToDevice, s));
    LQCD_CUDA(cudaMemcpyAsync(df_map.p, hdf.data(), hdf.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    LQCD_CUDA(cudaMemcpyAsync(bb_map.p, hbb.data(), hbb.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    const DfSys *d = (const DfSys *)df_descs.p;
    const int2 *mdf = (const int2 *)df_map.p, *mbb = (const int2 *)bb_map.p;
    const int ndf = (int)hdf.size(), nbb = (int)hbb.size();
    const dim3 dfb(DF_SITES, 3);
    batch_accum_df_kernel<<<nbb, CG_BLOCK, 0, s>>>(d, mbb);
    {
        KernelTimer kt(K_DSLASH_DF64, s, 4.0 * 1536.0 * (double)ndf * DF_SITES);
        batch_df_hop_kernel<0><<<ndf, dfb, 0, s>>>(d, mdf);
        batch_df_hop_kernel<1><<<ndf, dfb, 0, s>>>(d, mdf);
        batch_df_hop_kernel<2><<<ndf, dfb, 0, s>>>(d, mdf);
        batch_df_hop_kernel<3><<<ndf, dfb, 0, s>>>(d, mdf);
    }
    batch_final_sum_kernel<<<(unsigned)hd.size(), 1024, 0, s>>>(d);
    LQCD_CUDA(cudaGetLastError());
    g_launches.fetch_add(7, std::memory_order_relaxed);
    return LQCD_OK;
}

lqcd_status BatchSolver::add(CgRun *r)
{
    if (!r->done) {
        active.push_back(r);
        changed = true;
    }
    return LQCD_OK;
}

lqcd_status BatchSolver::step(lqcd_prec p, cudaStream_t s)
{
    if (active.empty()) return LQCD_OK;
    switch (p) {
    case LQCD_F16N: return chunk<LQCD_F16N>(s);
    case LQCD_F32: return chunk<LQCD_F32>(s);
    case LQCD_BF16: return chunk<LQCD_BF16>(s);
    default: set_error("batched solve: the sloppy precision must be F32, F16N or BF16"); return LQCD_EINVAL;
    }
}

BatchSolver::BatchSolver() = default;

lqcd_status BatchSolver::solve(std::vector<CgRun *> &runs, cudaStream_t s)
{
    if (runs.empty()) return LQCD_OK;
    lqcd_prec p = runs[0]->prm.sloppy;
    for (CgRun *r : runs)
        LQCD_REQUIRE(r->prm.sloppy == p, "batched solve: every system must use the same sloppy precision");
    switch (p) {
    case LQCD_F16N: return run_all<LQCD_F16N>(runs, s);
    case LQCD_F32: return run_all<LQCD_F32>(runs, s);
    case LQCD_BF16: return run_all<LQCD_BF16>(runs, s);
    default: set_error("batched solve: the sloppy precision must be F32, F16N or BF16"); return LQCD_EINVAL;
    }
}

void BatchSolver::release()
{
    drop_graph();
    if (capture_stream) cudaStreamDestroy(capture_stream);
    capture_stream = nullptr;
    if (pinned_h) cudaFreeHost(pinned_h);
    pinned_h = nullptr;
    pinned_n = 0;
    if (pinned_rr) cudaFreeHost(pinned_rr);
    pinned_rr = nullptr;
    pinned_rr_n = 0;
}

} // namespace lqcd

using namespace lqcd;

// ---------------------------------------------------------------- C ABI: batched solve

extern "C" lqcd_status lqcd_cg_solve_batch(int n, lqcd_field *const *x, const lqcd_field *const *U,
                                           const lqcd_field *const *U_sloppy, const lqcd_field *const *b,
                                           const double *kappa, const lqcd_cg_params *params, lqcd_cg_info *info,
                                           void *stream)
{
    LQCD_REQUIRE(n >= 0 && (n == 0 || (x && U && U_sloppy && b && kappa && params)), "cg_solve_batch: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<std::unique_ptr<CgWorkspace>> wss;
    std::vector<CgRun> runs(n);
    std::vector<CgRun *> ptrs;
    DevBuf scal;
    LQCD_TRY(scal.alloc(sizeof(CgScalars) * std::max(n, 1), s));
    for (int i = 0; i < n; i++) {
        LQCD_REQUIRE(x[i] && U[i] && U_sloppy[i] && b[i], "cg_solve_batch: NULL field in system %d", i);
        LQCD_REQUIRE(x[i]->kind == LQCD_SPINOR_EVEN && b[i]->kind == LQCD_SPINOR_EVEN && x[i]->prec == LQCD_F64 &&
                         b[i]->prec == LQCD_F64 && x[i] != b[i],
                     "cg_solve_batch: system %d needs distinct EVEN FP64 x and b", i);
        LQCD_REQUIRE(U[i]->kind == LQCD_GAUGE && U[i]->prec == LQCD_F64 && same_lattice(U[i]->lat, x[i]->lat) &&
                         same_lattice(U[i]->lat, b[i]->lat) && same_lattice(U[i]->lat, U_sloppy[i]->lat),
                     "cg_solve_batch: system %d has inconsistent fields", i);
        LQCD_REQUIRE(params->sloppy != LQCD_F64 && params->delta > 0 && params->delta < 1 && params->tol > 0 &&
                         params->maxiter > 0,
                     "cg_solve_batch: needs a mixed-precision solver (sloppy F32/F16N/BF16, 0 < delta < 1)");
        wss.emplace_back(new CgWorkspace());
        LQCD_TRY(wss.back()->ensure(x[i]->lat, params->sloppy, s));
        CgRun &r = runs[i];
        r.ws = wss.back().get(), r.x = x[i], r.U = U[i], r.Us = U_sloppy[i], r.b = b[i], r.kappa = kappa[i];
        r.prm = *params;
        r.start(s, (CgScalars *)scal.p + i);
        ptrs.push_back(&r);
    }
    BatchSolver bs;
    lqcd_status rc = bs.solve(ptrs, s);
    cudaStreamSynchronize(s);
    bs.release();
    lqcd_status worst = rc;
    for (int i = 0; i < n; i++) {
        if (info) info[i] = runs[i].inf;
        if (worst == LQCD_OK && runs[i].status != LQCD_OK) worst = runs[i].status;
    }
    return worst;
}
