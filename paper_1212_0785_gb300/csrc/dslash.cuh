// dslash.cuh -- internal interface of the Wilson hopping kernels and the CG
// scalar block shared by dslash.cu and cg.cu.
#pragma once

#include "lqcd_internal.cuh"

namespace lqcd {

// Device-resident scalars of one CG solve.  The reduction kernels update them
// and set `pause` when the host must act (convergence of the iterated
// residual, a reliable update, maxiter, a non-finite value); every iteration
// kernel returns immediately while `pause` is set.
struct CgScalars {
    double rr;      // |r|^2 of the current residual
    double pAp;     // <p, A p> = |Mhat p|^2
    double alpha;   // rr / pAp
    double beta;    // rr_new / rr
    double rr_new;  // |r|^2 after the update
    double stop2;   // tol^2 |b|^2
    double delta2;  // reliable-update threshold factor delta^2 (0: none)
    double maxrr2;  // max |r|^2 since the last reliable update
    int pause;
    int reason;     // 1 iterated residual converged, 2 reliable update due, 3 maxiter, 4 non-finite
    int iter;
    int maxiter;
};

enum { PAUSE_NONE = 0, PAUSE_CONVERGED = 1, PAUSE_RELIABLE = 2, PAUSE_MAXITER = 3, PAUSE_NONFINITE = 4 };

#ifndef LQCD_DS_BLOCK
#define LQCD_DS_BLOCK 128
#endif
// threads per block of the hopping-term kernels (one output site each)
constexpr int DS_BLOCK = LQCD_DS_BLOCK;

inline int dslash_blocks(int Vh) { return nblocks_for(Vh, DS_BLOCK); }

// out = D_{out<-in} in (dagger: D^dag).  Parities from the field kinds.
lqcd_status dslash_plain(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger, const int *skip,
                         cudaStream_t s);

// out = x + b D in; if partials != NULL also the per-block partial sums of
// |out|^2 (dslash_blocks(Vh) of them).
lqcd_status dslash_xpay(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger, const lqcd_field *x,
                        double b, double *partials, const int *skip, cudaStream_t s);

// CG update fused into the last half of Mhat^dag Mhat:
//   Ap = t + b D in;  xs += alpha p;  r -= alpha Ap;  partials of |r|^2
// (alpha from sc).  t, r, p in the sloppy precision of in; xs F64 (plain FP64
// solve) or F32 (mixed solve).
lqcd_status dslash_cg(const lqcd_field *U, const lqcd_field *in, int dagger, const lqcd_field *t, double b,
                      lqcd_field *xs, lqcd_field *r, const lqcd_field *p, double *partials, const CgScalars *sc,
                      cudaStream_t s);

// the FP16+norm hopping-term form: 1 prefetched links (default), 0 gathered;
// returns the previous form (form < 0: query; -1 and an error for an unknown form)
int dslash_form_set(int form);

// out = D in, or x + b D in if x is given, with float-float fields and links
// (precision code 4; dslash_df.cu)
lqcd_status dslash_df_launch(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger,
                             const lqcd_field *x, double b, const int *skip, cudaStream_t s);

} // namespace lqcd
