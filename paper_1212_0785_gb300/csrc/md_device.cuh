// md_device.cuh -- per-link device code of the SU(3) exponential link
// update (paper Sec. 1: "exponentiating of SU(3) matrices"), shared by the
// single-field kernel (field.cu) and the shared launches over a batch of
// chains (chains.cu).
#pragma once

#include "df64.cuh"
#include "lqcd_internal.cuh"
#include "su3_device.cuh"

namespace lqcd {

// 1/sqrt(n) in float-float for n > 0: the FP32 estimate y refined by one
// Newton-Raphson step of the reciprocal square root, y + y (1 - n y^2) / 2
// (relative error ~ (3/8) e^2 for an estimate of relative error e)
__device__ __forceinline__ Df df_rsqrt(Df n)
{
    const float y = rsqrtf(n.hi);
    const Df yy = Df(y, 0.f) * Df(y, 0.f);
    const Df r = Df(1) - n * yy;
    return Df(y, 0.f) + Df(y, 0.f) * Df(0.5f * r.hi, 0.5f * r.lo);
}

// Gram-Schmidt of rows 0 and 1 of an FP32 matrix in float-float arithmetic,
// row 2 = conj(row0 x row1): special unitary to ~2^-46
__device__ __forceinline__ M3<Df> reunit_rows_df(const M3<float> &e)
{
    M3<Df> u;
    DfAcc n0;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        n0.add_prod(Df(e.e[0][b].re, 0.f), Df(e.e[0][b].re, 0.f));
        n0.add_prod(Df(e.e[0][b].im, 0.f), Df(e.e[0][b].im, 0.f));
    }
    const Df s0 = df_rsqrt(n0.value());
#pragma unroll
    for (int b = 0; b < 3; b++) u.e[0][b] = Cx<Df>{s0 * Df(e.e[0][b].re, 0.f), s0 * Df(e.e[0][b].im, 0.f)};
    DfAcc ore, oim; // <row0, row1>
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const Df r1(e.e[1][b].re, 0.f), i1(e.e[1][b].im, 0.f);
        ore.add_prod(u.e[0][b].re, r1);
        ore.add_prod(u.e[0][b].im, i1);
        oim.add_prod(u.e[0][b].re, i1);
        oim.sub_prod(u.e[0][b].im, r1);
    }
    const Cx<Df> ov{ore.value(), oim.value()};
    DfAcc n1;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        u.e[1][b] = Cx<Df>{Df(e.e[1][b].re, 0.f), Df(e.e[1][b].im, 0.f)} - ov * u.e[0][b];
        n1.add_prod(u.e[1][b].re, u.e[1][b].re);
        n1.add_prod(u.e[1][b].im, u.e[1][b].im);
    }
    const Df s1 = df_rsqrt(n1.value());
#pragma unroll
    for (int b = 0; b < 3; b++) u.e[1][b] = Cx<Df>{s1 * u.e[1][b].re, s1 * u.e[1][b].im};
    reconstruct_row2(u);
    return u;
}

// U_mu(x) <- exp(i c P_mu(x)) U_mu(x) for the link (mu, par, cb).  FAST (the
// mixed-precision trajectory): the exponential by Cayley-Hamilton in FP32,
// re-unitarized and multiplied onto the links in float-float arithmetic (~48
// bits, on the FP32 pipes), so that the FP64 links stay in SU(3) to ~1e-14 per
// update; otherwise everything in FP64.  The new link is also written to the
// 12-real copies Us (solver precision) and Uf (FP32) and to the float-float
// copy Udf (the solver's accurate residual) when those are given; a given Udf
// is also the FAST product's input (it holds the current links), which spares
// the FP64 split of U.  write_f64 0 (FAST with Udf only): the FP64 links are
// not written; they lag behind the float-float copy until the caller converts
// it (the molecular dynamics reads only the copies).
template <lqcd_prec PS, bool FAST>
__device__ __forceinline__ void link_update_one(const GaugeRef<LQCD_F64> &U, const MomRef &P, double c,
                                                const GaugeRef<PS> &Us, const GaugeRef<LQCD_F32> &Uf,
                                                const GaugeRef<PREC_DF> &Udf, int mu, int par, int cb,
                                                int write_sloppy, int write_f32, int write_f64 = 1)
{
    M3<double> nu;
    M3<float> nf; // rows 0, 1 of the new link rounded once, for the 12-real copies
    if (FAST) {
        float p[8];
        for (int a = 0; a < 8; a++) p[a] = (float)P.d[P.idx(mu, par, a, cb)];
        const M3<Df> E = reunit_rows_df(expi_cayley_hamilton(herm_from_coeffs(p, (float)c)));
        M3<Df> u;
        if (Udf.d) { // the float-float copy is current: no FP64 split
#pragma unroll
            for (int k = 0; k < 9; k++) {
                float4 v = Udf.d[Udf.idx(mu, par, k, cb)];
                u.e[k / 3][k % 3] = Cx<Df>{Df(v.x, v.y), Df(v.z, v.w)};
            }
        } else {
#pragma unroll
            for (int k = 0; k < 9; k++) {
                double2 v = ldg(U.d + U.idx(mu, par, k, cb));
                u.e[k / 3][k % 3] = Cx<Df>{Df(v.x), Df(v.y)};
            }
        }
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                DfAcc re, im;
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    re.add_prod(E.e[i][k].re, u.e[k][j].re);
                    re.sub_prod(E.e[i][k].im, u.e[k][j].im);
                    im.add_prod(E.e[i][k].re, u.e[k][j].im);
                    im.add_prod(E.e[i][k].im, u.e[k][j].re);
                }
                const Df vr = re.value(), vi = im.value();
                if (write_f64) nu.e[i][j] = cx<double>((double)vr, (double)vi);
                if (i < 2) nf.e[i][j] = cx<float>(vr.hi + vr.lo, vi.hi + vi.lo);
                if (Udf.d) Udf.d[Udf.idx(mu, par, i * 3 + j, cb)] = make_float4(vr.hi, vr.lo, vi.hi, vi.lo);
            }
    } else {
        double p[8];
        for (int a = 0; a < 8; a++) p[a] = P.d[P.idx(mu, par, a, cb)];
        M3<double> E = expi_cayley_hamilton(herm_from_coeffs(p, c));
        nu = m3_mul(E, U.load<double>(mu, par, cb));
        if (Udf.d) Udf.store(mu, par, cb, nu);
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 3; j++) nf.e[i][j] = cx<float>((float)nu.e[i][j].re, (float)nu.e[i][j].im);
    }
    if (write_f64) U.store(mu, par, cb, nu);
    if (write_sloppy || write_f32) {
        if (write_sloppy) Us.store(mu, par, cb, nf);
        if (write_f32) Uf.store(mu, par, cb, nf);
    }
}

} // namespace lqcd
