// force.cuh -- per-link device code of the gauge (staple) force and the
// two-flavour Wilson fermion force, shared by the single-field kernels
// (force.cu) and the shared launches over a batch of chains (chains.cu).
#pragma once

#include "dslash.cuh"
#include "spin.cuh"
#include "su3_device.cuh"

namespace lqcd {

// default threads per block of the force kernels (the autotuner's table
// overrides it per lattice); FB_MAX bounds the launches
constexpr int FB = 128;
constexpr int FB_MAX = 256;

// Link of linear thread index t, direction-major (the batched chains' shared
// launches, whose blocks come from a per-chain table).
__device__ __forceinline__ bool link_seq(int Vh, long t, int &mu, int &par, int &cb)
{
    if (t >= 8L * Vh) return false;
    cb = (int)(t % Vh);
    const int mp = (int)(t / Vh);
    mu = mp >> 1;
    par = mp & 1;
    return true;
}

// Link of thread tid of block b (of bs threads), directions interleaved
// (fermion and gauge force).  The four directions of one range of sites go to four
// consecutive blocks, which run together, so the spinors that all four
// directions read are reused from L2 instead of being fetched again by a
// later sweep over the next direction (measured: 37 -> 28 ms per 32^3x64
// trajectory).  Every warp has one direction.  Grid: 8 * force_blocks(Vh, bs)
// blocks of bs threads.
__host__ __device__ __forceinline__ int force_blocks(int Vh, int bs) { return (Vh + bs - 1) / bs; }

__device__ __forceinline__ bool link_interleaved(int Vh, int b, int bs, int tid, int &mu, int &par, int &cb)
{
    mu = b & 3;
    const int q = b >> 2, nbp = force_blocks(Vh, bs);
    par = q / nbp;
    cb = (q - par * nbp) * bs + tid;
    return cb < Vh;
}
__device__ __forceinline__ bool link_of_thread(int Vh, int &mu, int &par, int &cb)
{
    return link_interleaved(Vh, blockIdx.x, blockDim.x, threadIdx.x, mu, par, cb);
}


template <typename R>
__device__ __forceinline__ void m3_scale(M3<R> &a, R w)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) a.e[i][j] = w * a.e[i][j];
}

template <typename R>
__device__ __forceinline__ void m3_acc(M3<R> &a, const M3<R> &b)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) a.e[i][j] = a.e[i][j] + b.e[i][j];
}


// Gauge force of link (x, mu): P_mu(x) -= cf * Im tr lambda_a U_mu(x) A_mu(x),
// A_mu(x) the sum of the six staples (the plaquettes through the link, each
// plane weighted by the anisotropic action's factor).  The direction mu is a
// run-time value, so one code path serves all four directions: the
// neighbours are reached by lexicographic offsets (+1 and -1 in each
// direction, with the periodic wrap), and an even-odd index is the
// lexicographic one halved.  A version specialised per direction at compile
// time ran the four directions as four code paths; with the directions
// interleaved across blocks (link_of_thread) that one path is 22% faster at
// 32^3x64 and gives the same bits.
__device__ __forceinline__ int sel4(const int v[4], int i)
{
    return i == 0 ? v[0] : i == 1 ? v[1] : i == 2 ? v[2] : v[3];
}

template <typename R, lqcd_prec GP>
__device__ __forceinline__ void gauge_force_link(MomRef &P, const GaugeRef<GP> &U, const Geo &g, int mu, int par,
                                                    int cb, const int c[4], double cf)
{
    int op[4], om[4];
    int stride = 1;
#pragma unroll
    for (int d = 0; d < 4; d++) {
        op[d] = c[d] == g.L[d] - 1 ? -(g.L[d] - 1) * stride : stride;
        om[d] = c[d] == 0 ? (g.L[d] - 1) * stride : -stride;
        stride *= g.L[d];
    }
    const int lex = coords_lex(g, c);
    const int pm = lex + sel4(op, mu);
    const int cb_pm = pm >> 1;
    M3<R> A;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) A.e[i][j] = cx<R>(0, 0);
#pragma unroll
    for (int k = 1; k < 4; k++) {
        const int nu = (mu + k) & 3;
        const int pn = sel4(op, nu), mn = sel4(om, nu);
        const int cb_pn = (lex + pn) >> 1, cb_mn = (lex + mn) >> 1, cb_pmmn = (pm + mn) >> 1;
        // upper: U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
        M3<R> up = m3_mul_dag(U.template load<R>(nu, 1 - par, cb_pm), U.template load<R>(mu, 1 - par, cb_pn));
        up = m3_mul_dag(up, U.template load<R>(nu, par, cb));
        // lower: (U_mu(x-nu) U_nu(x+mu-nu))^dag U_nu(x-nu)
        M3<R> lo = m3_mul(U.template load<R>(mu, 1 - par, cb_mn), U.template load<R>(nu, par, cb_pmmn));
        lo = m3_dag_mul(lo, U.template load<R>(nu, 1 - par, cb_mn));
        if (g.aniso) {
            const R w = (R)((mu == 3 || nu == 3) ? g.xi0 : 1.0 / g.xi0);
            m3_scale(up, w);
            m3_scale(lo, w);
        }
        m3_acc(A, up);
        m3_acc(A, lo);
    }
    M3<R> W = m3_mul(U.template load<R>(mu, par, cb), A);
    R gl[8];
    im_tr_lambda(W, gl);
#pragma unroll
    for (int a = 0; a < 8; a++) P.d[P.idx(mu, par, a, cb)] -= cf * (double)gl[a];
}

// FP32 fermion force: each thread first starts asynchronous 16-byte copies
// (cp.async) of B(x), B(x+mu) and U_mu(x) (one group) and of A(x+mu) (a
// second) into shared memory, so their DRAM latencies overlap instead of
// following one another; A(x) is loaded as before.  The arithmetic is
// unchanged.  Slots: [0, 6) B(x), [6, 12) B(x+mu), [12, 15) U_mu(x),
// [15, 21) A(x+mu), each [slot][thread] in dynamic shared memory (336 bytes
// per thread, so at most FF_MAX threads per block).
constexpr int FF_SLOTS = 21;
constexpr int FF_MAX = 128;

__device__ __forceinline__ void ff_cp16(float4 *dst, const float4 *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(__cvta_generic_to_global(src))
                 : "memory");
}

// a 12-real FP32 link from its three stored chunks (as GaugeRef<F32>::load)
template <typename R>
__device__ __forceinline__ M3<R> ff_link(float4 a, float4 b, float4 c)
{
    M3<R> u;
    u.e[0][0] = cx<R>(a.x, a.y);
    u.e[0][1] = cx<R>(a.z, a.w);
    u.e[0][2] = cx<R>(b.x, b.y);
    u.e[1][0] = cx<R>(b.z, b.w);
    u.e[1][1] = cx<R>(c.x, c.y);
    u.e[1][2] = cx<R>(c.z, c.w);
    reconstruct_row2(u);
    return u;
}

// Fermion force on link (x, mu), x of parity par:
//   Q = sum_spin [s U A(x+mu)] [(1 - gamma_mu) B(x)]^dag - A(x) [s U (1 + gamma_mu) B(x+mu)]^dag
// A = (A_e, A_o), B = (B_e, B_o) full-lattice spinors split by parity.
template <int MU, typename R, lqcd_prec SP, lqcd_prec GP>
__device__ __forceinline__ void fermion_force_link(MomRef &P, const GaugeRef<GP> &U, const Geo &g, int par,
                                                   int cb, const int c[4], const SpinorRef<SP> (&A)[2],
                                                   const SpinorRef<SP> (&B)[2], double cf,
                                                   float4 *pf = nullptr)
{
    int cy[4] = {c[0], c[1], c[2], c[3]};
    bool wrap = (c[MU] + 1 == g.L[MU]);
    cy[MU] = wrap ? 0 : c[MU] + 1;
    int cby = coords_cb(g, cy);
    R s = (MU == 3 && wrap && g.t_bc < 0) ? (R)-1 : (R)1;
    M3<R> u;
    Sp<R> Ay, Ax, Bx, By;
    if constexpr (SP == LQCD_F32 && GP == LQCD_F32) {
        const int i = threadIdx.x, nt = blockDim.x;
        const size_t Vh = (size_t)g.Vh;
        auto slot = [&](int k) -> float4 & { return pf[k * nt + i]; };
#pragma unroll
        for (int k = 0; k < 6; k++) {
            ff_cp16(&slot(k), B[par].d + k * Vh + cb);
            ff_cp16(&slot(6 + k), B[1 - par].d + k * Vh + cby);
        }
#pragma unroll
        for (int k = 0; k < 3; k++) ff_cp16(&slot(12 + k), U.d + U.idx(MU, par, k, cb));
        asm volatile("cp.async.commit_group;" ::: "memory");
#pragma unroll
        for (int k = 0; k < 6; k++) ff_cp16(&slot(15 + k), A[1 - par].d + k * Vh + cby);
        asm volatile("cp.async.commit_group;" ::: "memory");
        Ax = A[par].template load_rw<R>(cb);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        {
            float4 v[6], w[6];
#pragma unroll
            for (int k = 0; k < 6; k++) v[k] = slot(k), w[k] = slot(6 + k);
            Bx = B[par].template unpack<R>(v);
            By = B[1 - par].template unpack<R>(w);
        }
        u = ff_link<R>(slot(12), slot(13), slot(14));
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        {
            float4 v[6];
#pragma unroll
            for (int k = 0; k < 6; k++) v[k] = slot(15 + k);
            Ay = A[1 - par].template unpack<R>(v);
        }
    } else {
        u = U.template load<R>(MU, par, cb);
        Ay = A[1 - par].template load_rw<R>(cby);
        Ax = A[par].template load_rw<R>(cb);
        Bx = B[par].template load_rw<R>(cb);
        By = B[1 - par].template load_rw<R>(cby);
    }
    // w1 = (1 - gamma) B(x) as a full spinor
    Sp<R> w1 = sp_zero<R>();
    accumulate<MU, -1>(w1, project<MU, -1>(Bx));
    // w2 = s U (1 + gamma) B(y): project, multiply the two rows, reconstruct
    Sp<R> w2 = sp_zero<R>();
    {
        Hs<R> h = mul_link(u, project<MU, +1>(By));
        accumulate<MU, +1>(w2, h);
    }
    M3<R> Q;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) Q.e[a][b] = cx<R>(0, 0);
#pragma unroll
    for (int sp = 0; sp < 4; sp++) {
        Cx<R> v1[3];
#pragma unroll
        for (int a = 0; a < 3; a++) v1[a] = u.e[a][0] * Ay.c[sp][0] + u.e[a][1] * Ay.c[sp][1] + u.e[a][2] * Ay.c[sp][2];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++)
                Q.e[a][b] = Q.e[a][b] + s * (v1[a] * conj(w1.c[sp][b]) - Ax.c[sp][a] * conj(w2.c[sp][b]));
    }
    R gl[8];
    im_tr_lambda(Q, gl);
    // P -= coeff * f with f_a = -kappa^2 g_a (a spatial link times its hop's weight)
    if (MU < 3 && g.aniso) cf *= g.cs;
#pragma unroll
    for (int a = 0; a < 8; a++) P.d[P.idx(MU, par, a, cb)] += cf * (double)gl[a];
}

} // namespace lqcd
