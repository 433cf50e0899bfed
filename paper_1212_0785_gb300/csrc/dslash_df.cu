// dslash_df.cu -- the hopping term in float-float arithmetic for the mixed
// solver's accurate residual b - Mhat^dag Mhat x: GB300 runs FP64 at a small
// fraction of its FP32 rate, so the reliable updates use float-float storage
// and arithmetic (device code in dslash_df.cuh).
#include "dslash_df.cuh"

namespace lqcd {

// 4 blocks of 192 threads per SM (80 registers, 4 x 48 KiB of half spinors)
template <bool DAG, bool XPAY, bool RESID>
__global__ void __launch_bounds__(DF_SITES * 3, 4) dslash_df_kernel(SpinorRef<PREC_DF> out, SpinorRef<PREC_DF> in,
                                                                 GaugeRef<PREC_DF> U, Geo g, int out_par,
                                                                 SpinorRef<PREC_DF> x, Df b, const int *skip,
                                                                 SpinorRef<PREC_DF> bsrc, double *partials)
{
    __shared__ DfHalves sh;
    if (skip && *skip) return; // the same for the whole block
    df_hop_block<DAG, XPAY, RESID>(sh, out, in, U, g, out_par, x, b, blockIdx.x, bsrc, partials);
}

lqcd_status dslash_df_launch(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger,
                             const lqcd_field *x, double b, const int *skip, cudaStream_t s)
{
    Geo g = make_geo(in->lat);
    dim3 block(DF_SITES, 3), grid(nblocks_for(g.Vh, DF_SITES));
    SpinorRef<PREC_DF> xr = x ? spinor_ref<PREC_DF>(x) : SpinorRef<PREC_DF>{nullptr, g.Vh};
    const SpinorRef<PREC_DF> none{nullptr, g.Vh};
    int op = out->kind == LQCD_SPINOR_EVEN ? 0 : 1;
    Df bd(b);
    const auto o = spinor_ref<PREC_DF>(out), i = spinor_ref<PREC_DF>(in);
    const auto u = gauge_ref<PREC_DF>(U);
    if (x) {
        if (dagger)
            dslash_df_kernel<true, true, false><<<grid, block, 0, s>>>(o, i, u, g, op, xr, bd, skip, none, nullptr);
        else
            dslash_df_kernel<false, true, false><<<grid, block, 0, s>>>(o, i, u, g, op, xr, bd, skip, none, nullptr);
    } else {
        if (dagger)
            dslash_df_kernel<true, false, false><<<grid, block, 0, s>>>(o, i, u, g, op, xr, bd, skip, none, nullptr);
        else
            dslash_df_kernel<false, false, false><<<grid, block, 0, s>>>(o, i, u, g, op, xr, bd, skip, none, nullptr);
    }
    return LQCD_OK;
}

lqcd_status dslash_df_residual(lqcd_field *r, const lqcd_field *U, const lqcd_field *in, const lqcd_field *x,
                               double b, const lqcd_field *bsrc, double *partials, cudaStream_t s)
{
    Geo g = make_geo(in->lat);
    dim3 block(DF_SITES, 3), grid(nblocks_for(g.Vh, DF_SITES));
    const int op = r->kind == LQCD_SPINOR_EVEN ? 0 : 1;
    // links, in, x and b read, r written
    KernelTimer kt(K_DSLASH_DF64, s, (8 * link_bytes(U->prec) + 4 * spinor_site_bytes(in->prec)) * g.Vh);
    dslash_df_kernel<true, true, true><<<grid, block, 0, s>>>(spinor_ref<PREC_DF>(r), spinor_ref<PREC_DF>(in),
                                                              gauge_ref<PREC_DF>(U), g, op, spinor_ref<PREC_DF>(x),
                                                              Df(b), nullptr, spinor_ref<PREC_DF>(bsrc), partials);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

} // namespace lqcd
