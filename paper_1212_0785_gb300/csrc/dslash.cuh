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
    unsigned int arrive; // blocks of the current reduction that have stored their partial (0 between kernels)
};

enum { PAUSE_NONE = 0, PAUSE_CONVERGED = 1, PAUSE_RELIABLE = 2, PAUSE_MAXITER = 3, PAUSE_NONFINITE = 4 };

// alpha = rr / pAp from the summed pAp (a non-positive or non-finite pAp pauses)
__device__ __forceinline__ void cg_pap_step(CgScalars *sc, double pAp)
{
    sc->pAp = pAp;
    if (!(pAp > 0.0) || !isfinite(pAp)) {
        sc->alpha = 0.0;
        sc->pause = 1;
        sc->reason = PAUSE_NONFINITE;
    } else {
        sc->alpha = sc->rr / pAp;
    }
}

// the new |r|^2: the pause decision (non-finite, converged, reliable update
// due, maxiter -- in that order) or beta = rr_new / rr
__device__ __forceinline__ void cg_rr_step(CgScalars *sc, double rr_new)
{
    sc->rr_new = rr_new;
    sc->iter += 1;
    int reason = PAUSE_NONE;
    if (!isfinite(rr_new))
        reason = PAUSE_NONFINITE;
    else if (rr_new <= sc->stop2)
        reason = PAUSE_CONVERGED;
    else if (sc->delta2 > 0.0 && rr_new < sc->delta2 * sc->maxrr2)
        reason = PAUSE_RELIABLE;
    else if (sc->iter >= sc->maxiter)
        reason = PAUSE_MAXITER;
    if (reason != PAUSE_NONE) {
        sc->pause = 1;
        sc->reason = reason;
    } else {
        sc->beta = rr_new / sc->rr;
        sc->rr = rr_new;
        sc->maxrr2 = fmax(sc->maxrr2, rr_new);
    }
}

// Fixed-order sum of partials[0..n) by one block of BLOCK threads: thread i
// adds partials[i], partials[i + BLOCK], ... in that order (sixteen loads in
// flight, read from L2 since other blocks wrote them), then the warps reduce
// by shuffles and warp 0 adds the warp totals in warp order.  The result,
// valid in thread 0, does not depend on which block computes it.
template <int BLOCK>
__device__ __forceinline__ double block_final_sum(const double *partials, int n)
{
    __shared__ double wsum[BLOCK / 32];
    double s = 0.0;
    int i = threadIdx.x;
    for (; i + 15 * BLOCK < n; i += 16 * BLOCK) {
        double v[16];
#pragma unroll
        for (int k = 0; k < 16; k++) v[k] = __ldcg(partials + i + k * BLOCK);
#pragma unroll
        for (int k = 0; k < 16; k++) s += v[k];
    }
    for (; i < n; i += BLOCK) s += __ldcg(partials + i);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < BLOCK / 32; w++) t += wsum[w];
    return t;
}

// The scalar step of a CG reduction, done by the grid that produced the block
// partial sums: every block calls it after its thread 0 stored the block's
// partial; thread 0 publishes that store and counts the block in sc->arrive;
// the block that arrives last sums all nblocks partials in a fixed order,
// applies the pAp step (RR false) or the rr step (RR true) and resets the
// count.  No block waits for another.
template <int BLOCK, bool RR>
__device__ __forceinline__ void cg_finish(CgScalars *sc, const double *partials, int nblocks)
{
    __shared__ int last;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(&sc->arrive, 1u);
        last = prev == (unsigned int)(nblocks - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double total = block_final_sum<BLOCK>(partials, nblocks);
    if (threadIdx.x == 0) {
        sc->arrive = 0;
        if (RR)
            cg_rr_step(sc, total);
        else
            cg_pap_step(sc, total);
    }
}

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
// |out|^2 (dslash_blocks(Vh) of them), and if fin != NULL the last block then
// sums them and applies the CG pAp step to fin (cg_finish).
lqcd_status dslash_xpay(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger, const lqcd_field *x,
                        double b, double *partials, const int *skip, cudaStream_t s, CgScalars *fin = nullptr);

// CG update fused into the last half of Mhat^dag Mhat:
//   Ap = t + b D in;  xs += alpha p;  r -= alpha Ap;  partials of |r|^2,
// whose last block applies the CG rr step to sc (alpha from sc).  t, r, p in
// the sloppy precision of in; xs F64 (plain FP64 solve) or F32 (mixed solve).
lqcd_status dslash_cg(const lqcd_field *U, const lqcd_field *in, int dagger, const lqcd_field *t, double b,
                      lqcd_field *xs, lqcd_field *r, const lqcd_field *p, double *partials, CgScalars *sc,
                      cudaStream_t s);

// the FP16+norm hopping-term form: 2 prefetched links with packed FP32x2
// arithmetic (default), 1 prefetched links, 0 gathered; returns the previous
// form (form < 0: query; -1 and an error for an unknown form)
int dslash_form_set(int form);

// out = D in, or x + b D in if x is given, with float-float fields and links
// (precision code 4; dslash_df.cu)
lqcd_status dslash_df_launch(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger,
                             const lqcd_field *x, double b, const int *skip, cudaStream_t s);

// the accurate residual's last float-float term: r = bsrc - (x + b D^dag in),
// with one partial of |r|^2 per block of DF_SITES sites in partials[0 ..
// nblocks_for(Vh, DF_SITES)) (dslash_df.cu)
lqcd_status dslash_df_residual(lqcd_field *r, const lqcd_field *U, const lqcd_field *in, const lqcd_field *x,
                               double b, const lqcd_field *bsrc, double *partials, cudaStream_t s);

} // namespace lqcd
