// batch.cuh -- the multi-system CG engine shared by the batched chains and
// the solve service.
#pragma once

#include <memory>
#include <vector>

#include "cg.cuh"

namespace lqcd {

// Device descriptor of one system of a batch: its geometry, CG fields, links,
// -kappa^2, scalars and block partial sums.
template <lqcd_prec SP>
struct SysDesc {
    Geo g;
    SpinorRef<SP> p, r, t, tmp;
    SpinorRef<LQCD_F32> xs;
    GaugeRef<SP> U;
    float b;
    CgScalars *sc;
    double *partials;
    int nblocks;
};

// Runs a set of CgRuns (each started, each with its own scalars slot) to
// completion with shared launches.
struct BatchSolver {
    bool use_graph = true;
    std::vector<CgRun *> active;
    DevBuf descs, bmap, gathered;
    DevBuf df_descs, df_map, bb_map; // the paused systems' reliable updates
    int nblocks_total = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    CgScalars *pinned_h = nullptr;
    size_t pinned_n = 0;
    double *pinned_rr = nullptr; // accurate |r|^2 of the systems paused in one chunk
    size_t pinned_rr_n = 0;

    BatchSolver();
    ~BatchSolver();
    BatchSolver(const BatchSolver &) = delete;
    BatchSolver &operator=(const BatchSolver &) = delete;

    bool changed = true;

    lqcd_status solve(std::vector<CgRun *> &runs, cudaStream_t s);
    // continuous use: add started runs between steps; step runs one chunk of
    // all active runs (all with sloppy precision p) and drops finished ones
    lqcd_status add(CgRun *r);
    lqcd_status step(lqcd_prec p, cudaStream_t s);
    void release();

  private:
    void drop_graph();
    lqcd_status residuals_df(const std::vector<CgRun *> &runs, cudaStream_t s);
    template <lqcd_prec SP>
    lqcd_status run_all(std::vector<CgRun *> &runs, cudaStream_t s);
    template <lqcd_prec SP>
    lqcd_status chunk(cudaStream_t s);
    template <lqcd_prec SP>
    lqcd_status build_tables(cudaStream_t s);
    template <lqcd_prec SP>
    lqcd_status enqueue_chunk(cudaStream_t s);
};

} // namespace lqcd
