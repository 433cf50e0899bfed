// tune.cuh -- threads-per-block autotuning of the kernels whose launch shape
// is free (the paper's Sec. 4: every generated kernel is timed over the
// threads-per-block settings on first use and the fastest is kept in a
// database).  Here the tuning is an explicit call for a lattice
// (lqcd_autotune), its timings can be saved to and loaded from a text table,
// and every launch of a tuned kernel reads its block size from the in-memory
// table (the compiled-in default where there is no entry).
#pragma once

#include "lqcd_internal.cuh"

namespace lqcd {

enum TuneKernel {
    TK_HOP_F16N = 0,     // FP16+norm hopping term, packed form (plain, axpy and CG-update variants)
    TK_GAUGE_FORCE_F32,  // gauge force from the FP32 12-real link copy
    TK_GAUGE_FORCE_F64,  // gauge force in FP64
    TK_FERMION_FORCE_F32, // fermion-force link kernel in FP32
    TK_LINK_UPDATE_F32,  // link update of the FP32 molecular dynamics
    TK_NKERNEL
};

// block size for kernel k on lattice lat (dflt if the table has no entry)
int tuned_block(int k, const lqcd_lattice &lat, int dflt);
const char *tune_kernel_name(int k);

} // namespace lqcd
