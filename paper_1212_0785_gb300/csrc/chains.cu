// chains.cu -- the molecular-dynamics kernels of a batch of Markov chains in
// shared launches: every launch covers the links (or sites) of all chains,
// each block finding its chain and its place in it through a block ->
// (chain, block) table and the chain's fields through a descriptor, like the
// multi-system solver (batch.cu).  Per link and per site the arithmetic is
// that of the single-chain kernels (force.cuh, md_device.cuh, dslash_site.cuh,
// blocks of 128 threads), so every chain's momenta and links are bitwise
// those it would get alone.  Used by the batched trajectory with FP32
// molecular dynamics (force_prec F32): the gauge force from the FP32 12-real
// links, the fermion force's three FP32 hopping terms and its link kernel,
// and the link update with its copies.
#include "chains.cuh"
#include "dslash_site.cuh"
#include "force.cuh"
#include "md_device.cuh"

namespace lqcd {

constexpr int CB = 128; // threads per block of every shared launch

__global__ void __launch_bounds__(CB) chains_gauge_force_kernel(const ChainMd *d, const int2 *bmap, double coeff)
{
    const int2 m = bmap[blockIdx.x];
    const ChainMd &c = d[m.x];
    int mu, par, cb;
    if (!link_seq(c.g.Vh, (long)m.y * CB + threadIdx.x, mu, par, cb)) return;
    int x[4];
    cb_coords(c.g, cb, par, x);
    MomRef P = c.P;
    const GaugeRef<LQCD_F32> U = c.Uf;
    const double cf = coeff * c.beta / 6.0;
    gauge_force_link<float, LQCD_F32>(P, U, c.g, mu, par, cb, x, cf);
}

// X32 = X rounded to FP32 (the fermion force's input), per even site
__global__ void __launch_bounds__(CB) chains_round_x_kernel(const ChainMd *d, const int2 *bmap)
{
    const int2 m = bmap[blockIdx.x];
    const ChainMd &c = d[m.x];
    const int cb = m.y * CB + threadIdx.x;
    if (cb >= c.g.Vh) return;
    c.X32.store(cb, c.X.load_rw<float>(cb));
}

// the fermion force's hopping terms, step 0: Ao = D_oe X32; step 1:
// Ye = X32 - kappa^2 D_eo Ao; step 2: Bo = D_oe^dag Ye (FP32 spinors and links)
template <int STEP>
__global__ void __launch_bounds__(CB) chains_force_hop_kernel(const ChainMd *d, const int2 *bmap)
{
    const int2 m = bmap[blockIdx.x];
    const ChainMd &c = d[m.x];
    const int cb = m.y * CB + threadIdx.x;
    if (cb >= c.g.Vh) return;
    if (STEP == 0) {
        c.Ao.store(cb, dslash_site<float, LQCD_F32, LQCD_F32, false>(c.X32, c.Uf, c.g, cb, 1));
    } else if (STEP == 1) {
        Sp<float> v = dslash_site<float, LQCD_F32, LQCD_F32, false>(c.Ao, c.Uf, c.g, cb, 0);
        const Sp<float> xv = c.X32.load_rw<float>(cb);
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int k = 0; k < 3; k++) v.c[a][k] = xv.c[a][k] + c.mk2 * v.c[a][k];
        c.Ye.store(cb, v);
    } else {
        c.Bo.store(cb, dslash_site<float, LQCD_F32, LQCD_F32, true>(c.Ye, c.Uf, c.g, cb, 1));
    }
}

// the fermion-force link kernel, directions interleaved as in the single-chain launch
__global__ void __launch_bounds__(CB) chains_fermion_force_kernel(const ChainMd *d, const int2 *bmap, double coeff)
{
    const int2 m = bmap[blockIdx.x];
    const ChainMd &c = d[m.x];
    int mu, par, cb;
    if (!link_interleaved(c.g.Vh, m.y, CB, threadIdx.x, mu, par, cb)) return;
    int x[4];
    cb_coords(c.g, cb, par, x);
    const SpinorRef<LQCD_F32> A[2] = {c.X32, c.Ao};
    const SpinorRef<LQCD_F32> B[2] = {c.Ye, c.Bo};
    extern __shared__ float4 pf[]; // FF_SLOTS x CB
    MomRef P = c.P;
    const double cf = coeff * c.kappa * c.kappa;
    switch (mu) {
    case 0: fermion_force_link<0, float, LQCD_F32, LQCD_F32>(P, c.Uf, c.g, par, cb, x, A, B, cf, pf); break;
    case 1: fermion_force_link<1, float, LQCD_F32, LQCD_F32>(P, c.Uf, c.g, par, cb, x, A, B, cf, pf); break;
    case 2: fermion_force_link<2, float, LQCD_F32, LQCD_F32>(P, c.Uf, c.g, par, cb, x, A, B, cf, pf); break;
    default: fermion_force_link<3, float, LQCD_F32, LQCD_F32>(P, c.Uf, c.g, par, cb, x, A, B, cf, pf); break;
    }
}

// the FP32 molecular dynamics' link update with its copies, per link
// (registers capped at 128 like the single-chain kernel's)
template <lqcd_prec PS>
__global__ void __launch_bounds__(CB, 4) chains_link_update_kernel(const ChainMd *d, const int2 *bmap, double step)
{
    const int2 m = bmap[blockIdx.x];
    const ChainMd &c = d[m.x];
    int mu, par, cb;
    if (!link_seq(c.g.Vh, (long)m.y * CB + threadIdx.x, mu, par, cb)) return;
    const GaugeRef<PS> Us{reinterpret_cast<decltype(GaugeRef<PS>::d)>(c.us), c.g.Vh};
    // with a float-float copy the FP64 links lag behind it (written after the molecular dynamics)
    link_update_one<PS, true>(c.U, c.P, step, Us, c.Uf, c.Udf, mu, par, cb, 1, 1, c.Udf.d ? 0 : 1);
}

// ---------------------------------------------------------------- host

lqcd_status ChainMdTables::build(const std::vector<ChainMd> &descs, cudaStream_t s)
{
    n = (int)descs.size();
    std::vector<int2> lm, sm, fm;
    for (int i = 0; i < n; i++) {
        const int Vh = descs[i].g.Vh;
        for (int k = 0; k < nblocks_for(8L * Vh, CB); k++) lm.push_back(make_int2(i, k));
        for (int k = 0; k < nblocks_for(Vh, CB); k++) sm.push_back(make_int2(i, k));
        for (int k = 0; k < 8 * force_blocks(Vh, CB); k++) fm.push_back(make_int2(i, k));
    }
    link_blocks = (int)lm.size(), site_blocks = (int)sm.size(), force_link_blocks = (int)fm.size();
    const size_t nd = descs.size() * sizeof(ChainMd);
    const size_t nm = (lm.size() + sm.size() + fm.size()) * sizeof(int2);
    if (dev_desc.bytes < nd) LQCD_TRY(dev_desc.alloc(nd, s));
    if (dev_map.bytes < nm) LQCD_TRY(dev_map.alloc(nm, s));
    // pageable sources: each copy has taken its data when it returns
    LQCD_CUDA(cudaMemcpyAsync(dev_desc.p, descs.data(), nd, cudaMemcpyHostToDevice, s));
    int2 *mp = (int2 *)dev_map.p;
    LQCD_CUDA(cudaMemcpyAsync(mp, lm.data(), lm.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    LQCD_CUDA(cudaMemcpyAsync(mp + lm.size(), sm.data(), sm.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    LQCD_CUDA(cudaMemcpyAsync(mp + lm.size() + sm.size(), fm.data(), fm.size() * sizeof(int2),
                              cudaMemcpyHostToDevice, s));
    link_map = mp;
    site_map = mp + lm.size();
    force_map = mp + lm.size() + sm.size();
    host = descs;
    return LQCD_OK;
}

lqcd_status chains_gauge_force(const ChainMdTables &t, double coeff, cudaStream_t s)
{
    KernelTimer kt(K_GAUGE_FORCE, s);
    chains_gauge_force_kernel<<<t.link_blocks, CB, 0, s>>>((const ChainMd *)t.dev_desc.p, t.link_map, coeff);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status chains_fermion_force(const ChainMdTables &t, double coeff, cudaStream_t s)
{
    const ChainMd *d = (const ChainMd *)t.dev_desc.p;
    chains_round_x_kernel<<<t.site_blocks, CB, 0, s>>>(d, t.site_map);
    LQCD_LAUNCHED();
    {
        KernelTimer kt(K_DSLASH_F32, s);
        chains_force_hop_kernel<0><<<t.site_blocks, CB, 0, s>>>(d, t.site_map);
        LQCD_LAUNCHED();
        chains_force_hop_kernel<1><<<t.site_blocks, CB, 0, s>>>(d, t.site_map);
        LQCD_LAUNCHED();
        chains_force_hop_kernel<2><<<t.site_blocks, CB, 0, s>>>(d, t.site_map);
        LQCD_LAUNCHED();
    }
    KernelTimer kt(K_FERMION_FORCE, s);
    chains_fermion_force_kernel<<<t.force_link_blocks, CB, FF_SLOTS * CB * sizeof(float4), s>>>(d, t.force_map,
                                                                                                  coeff);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status chains_link_update(const ChainMdTables &t, double step, lqcd_prec sloppy, cudaStream_t s)
{
    KernelTimer kt(K_LINK_UPDATE, s);
    const ChainMd *d = (const ChainMd *)t.dev_desc.p;
    switch (sloppy) {
    case LQCD_F32: chains_link_update_kernel<LQCD_F32><<<t.link_blocks, CB, 0, s>>>(d, t.link_map, step); break;
    case LQCD_F16N: chains_link_update_kernel<LQCD_F16N><<<t.link_blocks, CB, 0, s>>>(d, t.link_map, step); break;
    case LQCD_BF16: chains_link_update_kernel<LQCD_BF16><<<t.link_blocks, CB, 0, s>>>(d, t.link_map, step); break;
    default: set_error("chains: the sloppy links must be F32, F16N or BF16"); return LQCD_EINVAL;
    }
    LQCD_LAUNCHED();
    return LQCD_OK;
}

} // namespace lqcd
