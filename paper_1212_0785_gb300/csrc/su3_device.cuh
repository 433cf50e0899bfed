// su3_device.cuh -- SU(3) algebra helpers on the device: Gell-Mann
// coefficients <-> Hermitian matrices, Im Tr(lambda_a W), the exponential
// exp(iQ) by Cayley-Hamilton, and Philox4x32-10.
#pragma once

#include "lqcd_internal.cuh"

namespace lqcd {

// H = sum_a p_a lambda_a / 2 for the 8 coefficients p (Gell-Mann lambda_1..8).
template <typename R>
__device__ __forceinline__ M3<R> herm_from_coeffs(const R p[8], R scale)
{
    const R inv_sqrt3 = (R)0.57735026918962576451;
    const R z = (R)0;
    M3<R> h;
    R s = (R)0.5 * scale;
    h.e[0][0] = cx<R>(s * (p[2] + p[7] * inv_sqrt3), z);
    h.e[1][1] = cx<R>(s * (-p[2] + p[7] * inv_sqrt3), z);
    h.e[2][2] = cx<R>((R)-2 * s * p[7] * inv_sqrt3, z);
    h.e[0][1] = cx<R>(s * p[0], -s * p[1]);
    h.e[1][0] = cx<R>(s * p[0], s * p[1]);
    h.e[0][2] = cx<R>(s * p[3], -s * p[4]);
    h.e[2][0] = cx<R>(s * p[3], s * p[4]);
    h.e[1][2] = cx<R>(s * p[5], -s * p[6]);
    h.e[2][1] = cx<R>(s * p[5], s * p[6]);
    return h;
}

// g_a = Im Tr(lambda_a W) for a = 1..8.
template <typename R>
__device__ __forceinline__ void im_tr_lambda(const M3<R> &W, R g[8])
{
    const R inv_sqrt3 = (R)0.57735026918962576451;
    g[0] = W.e[1][0].im + W.e[0][1].im;
    g[1] = W.e[0][1].re - W.e[1][0].re;
    g[2] = W.e[0][0].im - W.e[1][1].im;
    g[3] = W.e[2][0].im + W.e[0][2].im;
    g[4] = W.e[0][2].re - W.e[2][0].re;
    g[5] = W.e[2][1].im + W.e[1][2].im;
    g[6] = W.e[1][2].re - W.e[2][1].re;
    g[7] = (W.e[0][0].im + W.e[1][1].im - (R)2 * W.e[2][2].im) * inv_sqrt3;
}

// exp(i Q) for Hermitian traceless Q by the Cayley-Hamilton theorem
// (Morningstar & Peardon, Phys. Rev. D 69 (2004) 054501):
//   exp(iQ) = f0 + f1 Q + f2 Q^2 with c0 = det Q, c1 = Tr Q^2 / 2,
//   theta = arccos(|c0| / c0max), c0max = 2 (c1/3)^(3/2),
//   u = sqrt(c1/3) cos(theta/3), w = sqrt(c1) sin(theta/3),
//   f_j = h_j / (9u^2 - w^2) with
//   h0 = (u^2 - w^2) e^{2iu} + e^{-iu} [8u^2 cos w + 2iu (3u^2 + w^2) xi0(w)]
//   h1 = 2u e^{2iu} - e^{-iu} [2u cos w - i (3u^2 - w^2) xi0(w)]
//   h2 = e^{2iu} - e^{-iu} [cos w + 3iu xi0(w)],   xi0(w) = sin(w)/w,
// and f_j(-c0) = (-1)^j conj(f_j(c0)).
template <typename R>
__device__ __forceinline__ M3<R> expi_cayley_hamilton(const M3<R> &Q)
{
    const R one = (R)1, half = (R)0.5, third = (R)1 / (R)3;
    M3<R> Q2 = m3_mul(Q, Q);
    R c1 = half * (Q2.e[0][0].re + Q2.e[1][1].re + Q2.e[2][2].re);
    // det Q = Tr Q^3 / 3 (real for Hermitian Q)
    R c0 = (R)0;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) c0 += (Q.e[i][k] * Q2.e[k][i]).re;
    c0 *= third;
    M3<R> r;
    // Q ~ 0: I + iQ - Q^2/2 is exact to working precision
    if (c1 < (sizeof(R) == 8 ? (R)1e-28 : (R)1e-12)) {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                r.e[i][j] = cx<R>((i == j ? one : (R)0) - half * Q2.e[i][j].re - Q.e[i][j].im,
                                  Q.e[i][j].re - half * Q2.e[i][j].im);
        return r;
    }
    bool neg = c0 < (R)0;
    R ac0 = fabs(c0);
    R c0max = (R)2 * c1 * third * sqrt(c1 * third);
    R ratio = fmin(ac0 / c0max, one);
    R theta = acos(ratio);
    R u = sqrt(c1 * third) * cos(theta * third);
    R w = sqrt(c1) * sin(theta * third);
    R u2 = u * u, w2 = w * w;
    R cw = cos(w);
    R xi0;
    if (fabs(w) < (R)0.05) {
        xi0 = one - w2 / (R)6 * (one - w2 / (R)20 * (one - w2 / (R)42 * (one - w2 / (R)72)));
    } else {
        xi0 = sin(w) / w;
    }
    R s2u, c2u, su, cu;
    sincos((R)2 * u, &s2u, &c2u);
    sincos(u, &su, &cu);
    Cx<R> e2iu = cx<R>(c2u, s2u);
    Cx<R> emiu = cx<R>(cu, -su);
    Cx<R> h0 = (u2 - w2) * e2iu + emiu * cx<R>((R)8 * u2 * cw, (R)2 * u * ((R)3 * u2 + w2) * xi0);
    Cx<R> h1 = ((R)2 * u) * e2iu - emiu * cx<R>((R)2 * u * cw, -((R)3 * u2 - w2) * xi0);
    Cx<R> h2 = e2iu - emiu * cx<R>(cw, (R)3 * u * xi0);
    R inv = one / ((R)9 * u2 - w2);
    Cx<R> f0 = inv * h0, f1 = inv * h1, f2 = inv * h2;
    if (neg) {
        f0 = conj(f0);
        f1 = -conj(f1);
        f2 = conj(f2);
    }
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            Cx<R> v = f1 * Q.e[i][j] + f2 * Q2.e[i][j];
            if (i == j) v = v + f0;
            r.e[i][j] = v;
        }
    return r;
}

// Gram-Schmidt of rows 0 and 1, row 2 = conj(row0 x row1): the nearest
// special-unitary matrix in the sense used by the reunitarization
__device__ __forceinline__ void reunit_rows(M3<double> &u)
{
    double n0 = rsqrt(norm2(u.e[0][0]) + norm2(u.e[0][1]) + norm2(u.e[0][2]));
    for (int b = 0; b < 3; b++) u.e[0][b] = n0 * u.e[0][b];
    Cx<double> ov = cmul_conj(u.e[0][0], u.e[1][0]) + cmul_conj(u.e[0][1], u.e[1][1]) + cmul_conj(u.e[0][2], u.e[1][2]);
    for (int b = 0; b < 3; b++) u.e[1][b] = u.e[1][b] - ov * u.e[0][b];
    double n1 = rsqrt(norm2(u.e[1][0]) + norm2(u.e[1][1]) + norm2(u.e[1][2]));
    for (int b = 0; b < 3; b++) u.e[1][b] = n1 * u.e[1][b];
    reconstruct_row2(u);
}

// ------------------------------------------------------------------ Philox4x32-10

// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): 10 rounds; each round multiplies counter words 0 and 2 by the two
// round multipliers, mixes the high halves with words 1, 3 and the key, and
// the key is bumped by the two Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    const uint32_t MUL_A = 0xD2511F53u, MUL_B = 0xCD9E8D57u;
    const uint32_t WEYL_A = 0x9E3779B9u, WEYL_B = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        uint32_t hiA = __umulhi(MUL_A, c.x), loA = MUL_A * c.x;
        uint32_t hiB = __umulhi(MUL_B, c.z), loB = MUL_B * c.z;
        c = make_uint4(hiB ^ c.y ^ k.x, loB, hiA ^ c.w ^ k.y, loA);
        k.x += WEYL_A;
        k.y += WEYL_B;
    }
    return c;
}

// (0,1) uniform from a 64-bit word: ((w >> 12) + 1/2) * 2^-52, exact in double.
__device__ __forceinline__ double u52(uint32_t hi, uint32_t lo)
{
    unsigned long long w = ((unsigned long long)hi << 32) | lo;
    return ((double)(w >> 12) + 0.5) * 2.220446049250313080847e-16; // 2^-52
}

// Two standard Gaussians (Box-Muller) from one Philox block.
__device__ __forceinline__ void philox_gauss2(uint32_t seed, uint32_t chain, uint32_t site, uint32_t j,
                                              uint32_t purpose, uint32_t traj, double &g0, double &g1)
{
    uint4 x = philox4x32_10(make_uint4(site, j, purpose, traj), make_uint2(seed, chain));
    double u1 = u52(x.x, x.y), u2 = u52(x.z, x.w);
    double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincos((2.0 * 3.14159265358979323846) * u2, &s, &c);
    g0 = r * c;
    g1 = r * s;
}

} // namespace lqcd
