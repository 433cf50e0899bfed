// dslash_site.cuh -- the hopping term at one output site, shared by the
// single-field kernels (dslash.cu) and the multi-system kernels (batch.cu).
#pragma once

#include "dslash.cuh"
#include "spin.cuh"

namespace lqcd {

template <typename R>
__device__ __forceinline__ void scale_hs(Hs<R> &h, R s)
{
#pragma unroll
    for (int k = 0; k < 2; k++)
#pragma unroll
        for (int a = 0; a < 3; a++) h.c[k][a] = s * h.c[k][a];
}

// One direction: forward hop U_mu(x) (1 + FS gamma_mu) psi(x + mu), backward
// hop U_mu(x - mu)^dag (1 + BS gamma_mu) psi(x - mu).  A per-site norm of the
// stored spinor and the fermion boundary sign multiply the 6 complex numbers
// of the projected, link-multiplied half spinor rather than the 12 of the
// spinor.
template <int MU, int FS, int BS, typename R, lqcd_prec SP, lqcd_prec GP>
__device__ __forceinline__ void hop_dir(Sp<R> &acc, const SpinorRef<SP> &in, const GaugeRef<GP> &U, const Geo &g,
                                        int cb, int out_par, int nf, int nbk, bool wrap_f, bool wrap_b)
{
    constexpr bool NORM = SpinorRef<SP>::has_norm;
    const bool antip = (MU == 3) && g.t_bc < 0;
    {   // forward
        R sc;
        Sp<R> psi = in.template load_scaled<R>(nf, sc);
        Hs<R> uh = mul_link(U.template load<R>(MU, out_par, cb), project<MU, FS>(psi));
        if (NORM) {
            if (MU < 3) sc = sc * spatial_weight<R>(g); // 1 exactly when isotropic
            scale_hs(uh, (antip && wrap_f) ? -sc : sc);
        } else if (MU == 3) {
            if (antip && wrap_f) negate(uh);
        }
        accumulate<MU, FS>(acc, uh);
    }
    {   // backward
        R sc;
        Sp<R> psi = in.template load_scaled<R>(nbk, sc);
        Hs<R> uh = mul_link_dag(U.template load<R>(MU, 1 - out_par, nbk), project<MU, BS>(psi));
        if (NORM) {
            if (MU < 3) sc = sc * spatial_weight<R>(g);
            scale_hs(uh, (antip && wrap_b) ? -sc : sc);
        } else if (MU == 3) {
            if (antip && wrap_b) negate(uh);
        }
        accumulate<MU, BS>(acc, uh);
    }
}

// One hop from values already loaded: the stored spinor psi with its
// per-site scale sc (norm, or 1), the link u (U_mu(x) forward, U_mu(x - mu)
// backward), the boundary sign flip.  The same arithmetic as hop_dir.
template <int MU, int S, bool FWD, typename R>
__device__ __forceinline__ void hop_values(Sp<R> &acc, const Sp<R> &psi, R sc, const M3<R> &u, bool flip)
{
    Hs<R> uh = FWD ? mul_link(u, project<MU, S>(psi)) : mul_link_dag(u, project<MU, S>(psi));
    scale_hs(uh, flip ? -sc : sc);
    accumulate<MU, S>(acc, uh);
}

template <typename R, lqcd_prec SP, lqcd_prec GP, bool DAG>
__device__ __forceinline__ Sp<R> dslash_site(const SpinorRef<SP> &in, const GaugeRef<GP> &U, const Geo &g, int cb,
                                             int out_par)
{
    int c[4], nb[8];
    bool tf, tb;
    cb_coords(g, cb, out_par, c);
    cb_neighbours(g, cb, c, nb, tf, tb);
    Sp<R> acc = sp_zero<R>();
    // D: (1 - gamma) forward, (1 + gamma) backward; D^dag swaps them
    constexpr int FS = DAG ? +1 : -1;
    constexpr int BS = -FS;
    hop_dir<0, FS, BS, R>(acc, in, U, g, cb, out_par, nb[0], nb[1], false, false);
    hop_dir<1, FS, BS, R>(acc, in, U, g, cb, out_par, nb[2], nb[3], false, false);
    hop_dir<2, FS, BS, R>(acc, in, U, g, cb, out_par, nb[4], nb[5], false, false);
    // the anisotropic operator weighs the spatial hops: stored spinors with a
    // norm carry the weight in it (hop_dir), the others take it here (a
    // uniform branch)
    if (!SpinorRef<SP>::has_norm && g.aniso) sp_scale(acc, spatial_weight<R>(g));
    hop_dir<3, FS, BS, R>(acc, in, U, g, cb, out_par, nb[6], nb[7], tf, tb);
    return acc;
}

// |s|^2 of one site in the working precision (an FP32 kernel stays off the
// FP64 pipe); the sums over sites are FP64
template <typename R>
__device__ __forceinline__ R sp_norm2(const Sp<R> &s)
{
    R n = R(0);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) n = n + norm2(s.c[a][b]);
    return n;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---------------------------------------------------------------- prefetched links
//
// The other form that keeps the link loads off the critical path: each thread
// first starts asynchronous copies (cp.async, 8 bytes each) of its own eight
// links into shared memory, one commit group per direction, then walks the
// directions gathering the neighbour spinors as usual and waits for a
// direction's group only when it needs that direction's links.  Each thread
// reads back only what it copied, so no block barrier is involved; tail
// threads past Vh take no part.  Same arithmetic, same order as dslash_site.
// Blocks of DS_BLOCK threads (the single-field kernels of dslash.cu and the
// multi-system kernels of batch.cu).

__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int BLOCK>
struct LinkPrefetchT {
    uint2 u[4][2][3][BLOCK]; // [mu][forward, backward][chunk][thread]: 192 bytes per thread
};
using LinkPrefetch = LinkPrefetchT<DS_BLOCK>;

template <typename R, bool DAG>
__device__ __forceinline__ Sp<R> prefetch_site(const SpinorRef<LQCD_F16N> &in, const GaugeRef<LQCD_F16N> &U,
                                               const Geo &g, int cb, int out_par)
{
    __shared__ LinkPrefetch lp;
    const int i = threadIdx.x;
    int c[4], nb[8];
    bool tf, tb;
    cb_coords(g, cb, out_par, c);
    cb_neighbours(g, cb, c, nb, tf, tb);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            cp_async8(&lp.u[mu][0][k][i], U.d + U.idx(mu, out_par, k, cb));
            cp_async8(&lp.u[mu][1][k][i], U.d + U.idx(mu, 1 - out_par, k, nb[2 * mu + 1]));
        }
        cp_async_commit();
    }
    constexpr int FS = DAG ? +1 : -1;
    constexpr int BS = -FS;
    const bool antip = g.t_bc < 0;
    Sp<R> acc = sp_zero<R>();
    R sc;
    Sp<R> psi;
#define LQCD_PF_LINK(mu, f) U.template decode<R>(lp.u[mu][f][0][i], lp.u[mu][f][1][i], lp.u[mu][f][2][i])
    psi = in.template load_scaled<R>(nb[0], sc);
    cp_async_wait<3>();
    hop_values<0, FS, true>(acc, psi, sc * spatial_weight<R>(g), LQCD_PF_LINK(0, 0), false);
    psi = in.template load_scaled<R>(nb[1], sc);
    hop_values<0, BS, false>(acc, psi, sc * spatial_weight<R>(g), LQCD_PF_LINK(0, 1), false);
    psi = in.template load_scaled<R>(nb[2], sc);
    cp_async_wait<2>();
    hop_values<1, FS, true>(acc, psi, sc * spatial_weight<R>(g), LQCD_PF_LINK(1, 0), false);
    psi = in.template load_scaled<R>(nb[3], sc);
    hop_values<1, BS, false>(acc, psi, sc * spatial_weight<R>(g), LQCD_PF_LINK(1, 1), false);
    psi = in.template load_scaled<R>(nb[4], sc);
    cp_async_wait<1>();
    hop_values<2, FS, true>(acc, psi, sc * spatial_weight<R>(g), LQCD_PF_LINK(2, 0), false);
    psi = in.template load_scaled<R>(nb[5], sc);
    hop_values<2, BS, false>(acc, psi, sc * spatial_weight<R>(g), LQCD_PF_LINK(2, 1), false);
    psi = in.template load_scaled<R>(nb[6], sc);
    cp_async_wait<0>();
    hop_values<3, FS, true>(acc, psi, sc, LQCD_PF_LINK(3, 0), antip && tf);
    psi = in.template load_scaled<R>(nb[7], sc);
    hop_values<3, BS, false>(acc, psi, sc, LQCD_PF_LINK(3, 1), antip && tb);
#undef LQCD_PF_LINK
    return acc;
}

} // namespace lqcd
