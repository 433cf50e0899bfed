// cg.cuh -- CG work space shared between the solver and the HMC driver.
#pragma once

#include "dslash.cuh"

namespace lqcd {

// Fields and scalars of one solver, reusable across solves on one lattice.
struct CgWorkspace {
    lqcd_lattice lat{};
    lqcd_prec sloppy = LQCD_F64;
    bool ready = false;
    FieldPtr r64, t64a, t64b, tmpo64;  // FP64 residual and operator temporaries (FP64 CG)
    FieldPtr p64;                      // FP64 search direction (plain FP64 CG)
    FieldPtr xs, rs, ps, ts, tmpos;    // sloppy fields (mixed CG)
    // mixed CG: the accurate solution, source, residual and operator
    // temporaries in float-float storage, and the float-float link copy
    FieldPtr Udf, xdf, bdf, rdf, t1df, t2df, tmpodf;
    DevBuf sc, partials, scalars;
    lqcd_status ensure(const lqcd_lattice &lat, lqcd_prec sloppy, cudaStream_t s);
};

lqcd_status cg_solve_ws(CgWorkspace &ws, lqcd_field *x, const lqcd_field *U, const lqcd_field *Us,
                        const lqcd_field *b, double kappa, const lqcd_cg_params &prm, lqcd_cg_info *info,
                        cudaStream_t s);

// |v|^2 and Re<a,b> of FP64 fields into a device double (deterministic)
lqcd_status spinor_dot_dev(const lqcd_field *a, const lqcd_field *b, double *dst_dev, DevBuf &part, cudaStream_t s);

} // namespace lqcd
