// spin.cuh -- Wilson spin projection (1 -+ gamma_mu) onto half spinors in the
// DeGrand-Rossi basis, its reconstruction, and link multiplication of half
// spinors.  Used by the hopping term and the fermion force.
#pragma once

#include "lqcd_internal.cuh"

namespace lqcd {

// ---------------------------------------------------------------- spin projection
//
// SIGN = -1 projects with (1 - gamma_mu), SIGN = +1 with (1 + gamma_mu).
// In the DeGrand-Rossi basis (1 + s gamma_mu) psi has rows 0, 1 = (h0, h1)
// and rows 2, 3 fixed multiples of them:
//   mu=x: h0 = p0 + s i p3, h1 = p1 + s i p2, row2 = -s i h1, row3 = -s i h0
//   mu=y: h0 = p0 - s p3,   h1 = p1 + s p2,   row2 =  s h1,   row3 = -s h0
//   mu=z: h0 = p0 + s i p2, h1 = p1 - s i p3, row2 = -s i h0, row3 =  s i h1
//   mu=t: h0 = p0 + s p2,   h1 = p1 + s p3,   row2 =  s h0,   row3 =  s h1

template <int S, typename R>
__device__ __forceinline__ Cx<R> s_i(Cx<R> a) // s * i * a
{
    return S > 0 ? times_i(a) : -times_i(a);
}
template <int S, typename R>
__device__ __forceinline__ Cx<R> s_1(Cx<R> a) // s * a
{
    return S > 0 ? a : -a;
}

template <int MU, int S, typename R>
__device__ __forceinline__ Hs<R> project(const Sp<R> &p)
{
    Hs<R> h;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if (MU == 0) {
            h.c[0][c] = p.c[0][c] + s_i<S>(p.c[3][c]);
            h.c[1][c] = p.c[1][c] + s_i<S>(p.c[2][c]);
        } else if (MU == 1) {
            h.c[0][c] = p.c[0][c] - s_1<S>(p.c[3][c]);
            h.c[1][c] = p.c[1][c] + s_1<S>(p.c[2][c]);
        } else if (MU == 2) {
            h.c[0][c] = p.c[0][c] + s_i<S>(p.c[2][c]);
            h.c[1][c] = p.c[1][c] - s_i<S>(p.c[3][c]);
        } else {
            h.c[0][c] = p.c[0][c] + s_1<S>(p.c[2][c]);
            h.c[1][c] = p.c[1][c] + s_1<S>(p.c[3][c]);
        }
    }
    return h;
}

template <int MU, int S, typename R>
__device__ __forceinline__ void accumulate(Sp<R> &acc, const Hs<R> &h)
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        acc.c[0][c] = acc.c[0][c] + h.c[0][c];
        acc.c[1][c] = acc.c[1][c] + h.c[1][c];
        if (MU == 0) {
            acc.c[2][c] = acc.c[2][c] - s_i<S>(h.c[1][c]);
            acc.c[3][c] = acc.c[3][c] - s_i<S>(h.c[0][c]);
        } else if (MU == 1) {
            acc.c[2][c] = acc.c[2][c] + s_1<S>(h.c[1][c]);
            acc.c[3][c] = acc.c[3][c] - s_1<S>(h.c[0][c]);
        } else if (MU == 2) {
            acc.c[2][c] = acc.c[2][c] - s_i<S>(h.c[0][c]);
            acc.c[3][c] = acc.c[3][c] + s_i<S>(h.c[1][c]);
        } else {
            acc.c[2][c] = acc.c[2][c] + s_1<S>(h.c[0][c]);
            acc.c[3][c] = acc.c[3][c] + s_1<S>(h.c[1][c]);
        }
    }
}

// U h (per spin row)
template <typename R>
__device__ __forceinline__ Hs<R> mul_link(const M3<R> &u, const Hs<R> &h)
{
    Hs<R> o;
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            Cx<R> v = u.e[a][0] * h.c[s][0];
            v = v + u.e[a][1] * h.c[s][1];
            v = v + u.e[a][2] * h.c[s][2];
            o.c[s][a] = v;
        }
    return o;
}

// U^dag h
template <typename R>
__device__ __forceinline__ Hs<R> mul_link_dag(const M3<R> &u, const Hs<R> &h)
{
    Hs<R> o;
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            Cx<R> v = cmul_conj(u.e[0][a], h.c[s][0]);
            v = v + cmul_conj(u.e[1][a], h.c[s][1]);
            v = v + cmul_conj(u.e[2][a], h.c[s][2]);
            o.c[s][a] = v;
        }
    return o;
}

template <typename R>
__device__ __forceinline__ void negate(Hs<R> &h)
{
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) h.c[s][a] = -h.c[s][a];
}

} // namespace lqcd
