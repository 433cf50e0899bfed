// dslash_site.cuh -- the hopping term at one output site, shared by the
// single-field kernels (dslash.cu) and the multi-system kernels (batch.cu).
#pragma once

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

} // namespace lqcd
