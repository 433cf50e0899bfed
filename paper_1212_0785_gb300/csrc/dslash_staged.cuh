// dslash_staged.cuh -- the FP16+norm hopping term with its far operands
// staged in shared memory by bulk asynchronous copies (TMA engine,
// cp.async.bulk completing on an mbarrier).
//
// When a block's 128 output sites lie in one (z, t) slab (Lx/2 * Ly a multiple
// of 128), the +-t (and +-z) neighbours of those sites are contiguous 128-site
// ranges of the input field (each shifted by one t or z stride, or wrapped
// across the boundary as a whole), the forward links of the block are its own
// 128-site ranges, and the backward links are the ranges of the -t (-z)
// neighbours.  One thread of the block issues the bulk copies of those ranges
// at once (t only: 14 copies, 19.5 KiB; with z: 28 copies, 39 KiB); the other
// operands, which mostly hit L1 or L2, are loaded as before.  The arithmetic
// per site is that of dslash_site, in the same order, so the results are
// bitwise the same.
#pragma once

#include "dslash_site.cuh"

namespace lqcd {

constexpr int ST_SITES = 128;

// STAGE_Z: stage the +-z operands as well as the +-t ones
#ifndef LQCD_STAGE_Z
#define LQCD_STAGE_Z 0
#endif
constexpr int NSR = LQCD_STAGE_Z ? 4 : 2; // staged neighbour ranges: (+z, -z,) +t, -t
constexpr int NUF = LQCD_STAGE_Z ? 2 : 1; // staged forward links: (U_z,) U_t
constexpr int NUB = NUF;                  // staged backward links: (U_z(x - z),) U_t(x - t)

struct __align__(128) StageF16N {
    uint4 sp[NSR][3][ST_SITES]; // neighbour spinors (the three 16-byte chunks)
    float nrm[NSR][ST_SITES];   // their per-site norms
    uint2 uf[NUF][3][ST_SITES]; // forward links
    uint2 ub[NUB][3][ST_SITES]; // backward links
    unsigned long long bar;
};
constexpr uint32_t STAGE_BYTES = NSR * (3 * ST_SITES * 16 + ST_SITES * 4) + (NUF + NUB) * 3 * ST_SITES * 8;

// set when a block's wait for its copies gave up (read and cleared by the
// host; this header belongs to dslash.cu alone)
static __device__ int g_stage_timeout = 0;

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(bar)
                 : "memory");
}

// Stage the block's far operands; every thread of the block calls it.  The
// wait is bounded: after ~2^22 polls the block flags g_stage_timeout and goes
// on (its results are then wrong, and the host reports LQCD_ETIMEOUT).
__device__ __forceinline__ void stage_block(StageF16N &st, const SpinorRef<LQCD_F16N> &in,
                                            const GaugeRef<LQCD_F16N> &U, const Geo &g, int out_par, int cb0,
                                            int z, int t)
{
    const uint32_t bar = smem_addr(&st.bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(STAGE_BYTES)
                     : "memory");
        const int Lz = g.L[2], Lt = g.L[3];
        const int zs[2] = {z == Lz - 1 ? cb0 - (Lz - 1) * g.sZ : cb0 + g.sZ, z == 0 ? cb0 + (Lz - 1) * g.sZ : cb0 - g.sZ};
        const int ts[2] = {t == Lt - 1 ? cb0 - (Lt - 1) * g.sT : cb0 + g.sT, t == 0 ? cb0 + (Lt - 1) * g.sT : cb0 - g.sT};
        const int start[4] = {NSR == 4 ? zs[0] : ts[0], NSR == 4 ? zs[1] : ts[1], ts[0], ts[1]};
        const size_t Vh = (size_t)in.Vh;
        for (int r = 0; r < NSR; r++) {
            for (int k = 0; k < 3; k++) bulk_g2s(st.sp[r][k], in.d + k * Vh + start[r], ST_SITES * 16, bar);
            bulk_g2s(st.nrm[r], in.norm + start[r], ST_SITES * 4, bar);
        }
        for (int j = 0; j < NUF; j++) {
            const int mu = 4 - NUF + j; // z, t or t
            const int back = j == NUF - 1 ? ts[1] : zs[1];
            for (int k = 0; k < 3; k++) {
                bulk_g2s(st.uf[j][k], U.d + U.idx(mu, out_par, k, cb0), ST_SITES * 8, bar);
                bulk_g2s(st.ub[j][k], U.d + U.idx(mu, 1 - out_par, k, back), ST_SITES * 8, bar);
            }
        }
    }
    for (int it = 0; it < (1 << 22); it++) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(0)
                     : "memory");
        if (done) return;
    }
    g_stage_timeout = 1;
}

template <typename R>
__device__ __forceinline__ Sp<R> staged_spinor(const StageF16N &st, int r, int i, R &sc)
{
    const SpinorRef<LQCD_F16N> codec{nullptr, nullptr, 0};
    const uint4 v[3] = {st.sp[r][0][i], st.sp[r][1][i], st.sp[r][2][i]};
    sc = (R)st.nrm[r][i];
    return codec.template unpack<R>(v, 1.0f);
}

// D (DAG: D^dag) at site cb = cb0 + threadIdx.x of a block whose far operands
// are staged; every thread of the block calls it (Vh is a multiple of 128)
template <typename R, bool DAG>
__device__ __forceinline__ Sp<R> staged_site(const SpinorRef<LQCD_F16N> &in, const GaugeRef<LQCD_F16N> &U,
                                             const Geo &g, int cb, int out_par)
{
    __shared__ StageF16N st;
    const int i = threadIdx.x;
    int c[4], nb[8];
    bool tf, tb;
    cb_coords(g, cb, out_par, c);
    cb_neighbours(g, cb, c, nb, tf, tb);
    stage_block(st, in, U, g, out_par, cb - i, c[2], c[3]);
    constexpr int FS = DAG ? +1 : -1;
    constexpr int BS = -FS;
    const bool antip = g.t_bc < 0;
    Sp<R> acc = sp_zero<R>();
    R sc;
    Sp<R> psi;
    // x and y (and z unless staged): operands gathered as in dslash_site
    psi = in.template load_scaled<R>(nb[0], sc);
    hop_values<0, FS, true>(acc, psi, sc, U.template load<R>(0, out_par, cb), false);
    psi = in.template load_scaled<R>(nb[1], sc);
    hop_values<0, BS, false>(acc, psi, sc, U.template load<R>(0, 1 - out_par, nb[1]), false);
    psi = in.template load_scaled<R>(nb[2], sc);
    hop_values<1, FS, true>(acc, psi, sc, U.template load<R>(1, out_par, cb), false);
    psi = in.template load_scaled<R>(nb[3], sc);
    hop_values<1, BS, false>(acc, psi, sc, U.template load<R>(1, 1 - out_par, nb[3]), false);
    if constexpr (NSR == 4) {
        psi = staged_spinor<R>(st, 0, i, sc);
        hop_values<2, FS, true>(acc, psi, sc, U.template decode<R>(st.uf[0][0][i], st.uf[0][1][i], st.uf[0][2][i]),
                                false);
        psi = staged_spinor<R>(st, 1, i, sc);
        hop_values<2, BS, false>(acc, psi, sc,
                                 U.template decode<R>(st.ub[0][0][i], st.ub[0][1][i], st.ub[0][2][i]), false);
    } else {
        psi = in.template load_scaled<R>(nb[4], sc);
        hop_values<2, FS, true>(acc, psi, sc, U.template load<R>(2, out_par, cb), false);
        psi = in.template load_scaled<R>(nb[5], sc);
        hop_values<2, BS, false>(acc, psi, sc, U.template load<R>(2, 1 - out_par, nb[5]), false);
    }
    // t: staged
    constexpr int RT = NSR - 2, JT = NUF - 1;
    psi = staged_spinor<R>(st, RT, i, sc);
    hop_values<3, FS, true>(acc, psi, sc, U.template decode<R>(st.uf[JT][0][i], st.uf[JT][1][i], st.uf[JT][2][i]),
                            antip && tf);
    psi = staged_spinor<R>(st, RT + 1, i, sc);
    hop_values<3, BS, false>(acc, psi, sc, U.template decode<R>(st.ub[JT][0][i], st.ub[JT][1][i], st.ub[JT][2][i]),
                             antip && tb);
    return acc;
}

// the geometry and block size the staged kernels need
inline bool staging_fits(const Geo &g) { return DS_BLOCK == ST_SITES && g.sZ % ST_SITES == 0; }

} // namespace lqcd
