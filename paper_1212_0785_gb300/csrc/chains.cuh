// chains.cuh -- descriptors and launchers of the shared molecular-dynamics
// launches over a batch of chains (chains.cu).
#pragma once

#include <vector>

#include "df64.cuh"
#include "lqcd_internal.cuh"

namespace lqcd {

// One chain's fields for the FP32 molecular dynamics: links (FP64 master, FP32
// and solver-precision 12-real copies, float-float copy), momenta, the solve's
// solution X and the fermion force's FP32 temporaries, and its couplings.
struct ChainMd {
    Geo g;
    MomRef P;
    GaugeRef<LQCD_F64> U;
    GaugeRef<LQCD_F32> Uf;
    void *us; // solver-precision 12-real copy (its GaugeRef chosen by the launch)
    GaugeRef<PREC_DF> Udf;
    SpinorRef<LQCD_F64> X;
    SpinorRef<LQCD_F32> X32, Ao, Ye, Bo;
    double beta, kappa; // the couplings (the force coefficients are formed as the single chain forms them)
    float mk2;          // -kappa^2 in FP32 (the hopping term's axpy)
};

// The descriptors of a batch and its block -> (chain, block) tables: over
// 8 Vh links per chain (gauge force, link update), Vh sites (hopping terms),
// and the fermion force's interleaved link blocks.
struct ChainMdTables {
    int n = 0, link_blocks = 0, site_blocks = 0, force_link_blocks = 0;
    DevBuf dev_desc, dev_map;
    const int2 *link_map = nullptr, *site_map = nullptr, *force_map = nullptr;
    std::vector<ChainMd> host; // what the device tables hold
    lqcd_status build(const std::vector<ChainMd> &descs, cudaStream_t s);
};

// P -= coeff (beta/6) f_gauge for every chain (FP32 links)
lqcd_status chains_gauge_force(const ChainMdTables &t, double coeff, cudaStream_t s);
// P -= coeff kappa^2 f_fermion for every chain, from its solution X
lqcd_status chains_fermion_force(const ChainMdTables &t, double coeff, cudaStream_t s);
// U <- exp(i step P) U for every chain, with the copies of the FP32 molecular dynamics
lqcd_status chains_link_update(const ChainMdTables &t, double step, lqcd_prec sloppy, cudaStream_t s);

} // namespace lqcd
