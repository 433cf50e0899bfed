// force.cu -- gauge (staple) force and two-flavour Wilson fermion force, each
// projected onto su(3) and fused with the momentum update P <- P - coeff F
// (paper Sec. 1: "force term calculation", "projection of fields",
// "momentum updates").  One thread per link.  The arithmetic is FP64, or FP32
// (links read from the FP64 master field, spinors in FP32, the increment
// accumulated into the FP64 momenta) for the mixed-precision trajectory.
//
// Both forces are written as f_a = Im Tr(lambda_a W) of one 3x3 matrix W per
// link: for F = c TA(W) = c [(W - W^dag) - Tr(W - W^dag)/3] the Gell-Mann
// coefficients are 2 Re Tr(T_a F) = Re(c Tr(lambda_a (W - W^dag)))
// = Re(2 i c Im Tr(lambda_a W)), so
//   gauge   F = -(i beta/12) TA(U A):  f_a = (beta / 6) Im Tr(lambda_a U A)
//   fermion F = (i kappa^2/2) TA(Q):   f_a = -kappa^2 Im Tr(lambda_a Q).
#include "force.cuh"
#include "tune.cuh"

namespace lqcd {

// one thread per link, the four directions of a range of sites in four
// consecutive blocks (link_of_thread), so the staple links that all four
// directions read are shared through L2
template <typename R, lqcd_prec GP>
__global__ void __launch_bounds__(FB_MAX) gauge_force_kernel(MomRef P, GaugeRef<GP> U, Geo g, double cf)
{
    int mu, par, cb;
    if (!link_of_thread(g.Vh, mu, par, cb)) return;
    int c[4];
    cb_coords(g, cb, par, c);
    gauge_force_link<R, GP>(P, U, g, mu, par, cb, c, cf);
}

template <typename R, lqcd_prec SP, lqcd_prec GP>
__global__ void __launch_bounds__(FF_MAX) fermion_force_kernel(MomRef P, GaugeRef<GP> U, Geo g, SpinorRef<SP> Ae,
                                                           SpinorRef<SP> Ao, SpinorRef<SP> Be, SpinorRef<SP> Bo,
                                                           double cf)
{
    int mu, par, cb;
    if (!link_of_thread(g.Vh, mu, par, cb)) return;
    int c[4];
    cb_coords(g, cb, par, c);
    const SpinorRef<SP> A[2] = {Ae, Ao};
    const SpinorRef<SP> B[2] = {Be, Bo};
    extern __shared__ float4 pf[]; // FF_SLOTS x blockDim.x (FP32), none otherwise
    switch (mu) {
    case 0: fermion_force_link<0, R, SP, GP>(P, U, g, par, cb, c, A, B, cf, pf); break;
    case 1: fermion_force_link<1, R, SP, GP>(P, U, g, par, cb, c, A, B, cf, pf); break;
    case 2: fermion_force_link<2, R, SP, GP>(P, U, g, par, cb, c, A, B, cf, pf); break;
    default: fermion_force_link<3, R, SP, GP>(P, U, g, par, cb, c, A, B, cf, pf); break;
    }
}

// P -= cf f of the gauge force with bs threads per block; Uf: the FP32
// 12-real link copy, used (and required) when arith is F32
lqcd_status gauge_force_block(lqcd_field *P, const lqcd_field *U, const lqcd_field *Uf, double cf, lqcd_prec arith,
                              int bs, cudaStream_t s)
{
    LQCD_REQUIRE(bs >= 32 && bs <= FB_MAX && bs % 32 == 0, "gauge force: bad block size %d", bs);
    Geo g = make_geo(U->lat);
    const int nb = 8 * force_blocks(g.Vh, bs);
    if (arith == LQCD_F32)
        gauge_force_kernel<float, LQCD_F32><<<nb, bs, 0, s>>>(mom_ref(P), gauge_ref<LQCD_F32>(Uf), g, cf);
    else
        gauge_force_kernel<double, LQCD_F64><<<nb, bs, 0, s>>>(mom_ref(P), gauge_ref<LQCD_F64>(U), g, cf);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status gauge_force_dev(lqcd_field *P, const lqcd_field *U, const lqcd_field *Uf, double beta, double coeff,
                            lqcd_prec arith, cudaStream_t s)
{
    KernelTimer kt(K_GAUGE_FORCE, s);
    const int bs = tuned_block(arith == LQCD_F32 ? TK_GAUGE_FORCE_F32 : TK_GAUGE_FORCE_F64, U->lat, FB);
    return gauge_force_block(P, U, Uf, coeff * beta / 6.0, arith, bs, s);
}

// the fermion-force link kernel with bs threads per block (A = (Xe, Ao), B = (Ye, Bo))
template <typename R, lqcd_prec SP>
static lqcd_status fermion_link_launch(lqcd_field *P, const lqcd_field *L, const lqcd_field *Xe, const lqcd_field *Ao,
                                       const lqcd_field *Ye, const lqcd_field *Bo, double cf, int bs, cudaStream_t s)
{
    LQCD_REQUIRE(bs >= 32 && bs <= FF_MAX && bs % 32 == 0, "fermion force: bad block size %d", bs);
    Geo g = make_geo(L->lat);
    const int nb = 8 * force_blocks(g.Vh, bs);
    const size_t smem = SP == LQCD_F32 ? (size_t)FF_SLOTS * bs * sizeof(float4) : 0;
    fermion_force_kernel<R, SP, SP><<<nb, bs, smem, s>>>(mom_ref(P), gauge_ref<SP>(L), g, spinor_ref<SP>(Xe),
                                                          spinor_ref<SP>(Ao), spinor_ref<SP>(Ye), spinor_ref<SP>(Bo),
                                                          cf);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status fermion_force_link_block(lqcd_field *P, const lqcd_field *Uf, const lqcd_field *Xe, const lqcd_field *Ao,
                                     const lqcd_field *Ye, const lqcd_field *Bo, double cf, int bs, cudaStream_t s)
{
    return fermion_link_launch<float, LQCD_F32>(P, Uf, Xe, Ao, Ye, Bo, cf, bs, s);
}

// A_o = Doe X_e, Y_e = Mhat X_e = X_e - kappa^2 Deo A_o, B_o = Doe^dag-hop Y_e, then the link kernel:
// P -= coeff F with F the force of -2 Re[Y^dag dMhat X].  Y (optional) replaces
// Mhat X (the second term of the Hasenbusch ratio action).  The temporaries'
// precision (F64 or F32) sets the arithmetic; for F32 the links come from the
// FP32 12-real copy Uf and X (and Y) are rounded into Xc (Ye) first.
lqcd_status fermion_force_dev(lqcd_field *P, const lqcd_field *U, const lqcd_field *Uf, const lqcd_field *X,
                              double kappa, double coeff, lqcd_field *Ao, lqcd_field *Ye, lqcd_field *Bo, lqcd_field *Xc,
                              cudaStream_t s, const lqcd_field *Y)
{
    const lqcd_field *Xa = X;
    const lqcd_field *L = Ao->prec == LQCD_F32 ? Uf : U;
    if (Ao->prec != X->prec) {
        LQCD_TRY(lqcd_field_copy(Xc, X, s));
        Xa = Xc;
    }
    LQCD_TRY(dslash_plain(Ao, L, Xa, 0, nullptr, s));
    const lqcd_field *Ya = Ye;
    if (Y) {
        if (Y->prec != Ye->prec)
            LQCD_TRY(lqcd_field_copy(Ye, Y, s));
        else
            Ya = Y;
    } else {
        LQCD_TRY(dslash_xpay(Ye, L, Ao, 0, Xa, -kappa * kappa, nullptr, nullptr, s));
    }
    LQCD_TRY(dslash_plain(Bo, L, Ya, 1, nullptr, s));
    KernelTimer kt(K_FERMION_FORCE, s);
    const double cf = coeff * kappa * kappa;
    if (Ao->prec == LQCD_F32)
        return fermion_link_launch<float, LQCD_F32>(P, Uf, Xa, Ao, Ya, Bo, cf,
                                                    tuned_block(TK_FERMION_FORCE_F32, U->lat, FB), s);
    return fermion_link_launch<double, LQCD_F64>(P, U, Xa, Ao, Ya, Bo, cf, FB, s);
}

} // namespace lqcd

using namespace lqcd;

extern "C" {

lqcd_status lqcd_gauge_force_ex(lqcd_field *P, const lqcd_field *U, double beta, double coeff, lqcd_prec arith,
                                void *stream)
{
    LQCD_REQUIRE(P && U && P->kind == LQCD_MOMENTUM && U->kind == LQCD_GAUGE && U->prec == LQCD_F64,
                 "gauge_force needs a momentum field and an F64 gauge field");
    LQCD_REQUIRE(same_lattice(P->lat, U->lat), "gauge_force: lattices differ");
    LQCD_REQUIRE(arith == LQCD_F64 || arith == LQCD_F32, "gauge_force: arithmetic must be F64 or F32");
    cudaStream_t s = (cudaStream_t)stream;
    FieldPtr Uf;
    if (arith == LQCD_F32) {
        LQCD_TRY(lqcd_field_alloc(&U->lat, LQCD_GAUGE, LQCD_F32, 12, &Uf.f));
        LQCD_TRY(lqcd_field_copy(Uf.f, U, s));
    }
    LQCD_TRY(gauge_force_dev(P, U, Uf.f, beta, coeff, arith, s));
    LQCD_CUDA(cudaStreamSynchronize(s)); // the temporary copy is freed on return
    return LQCD_OK;
}

lqcd_status lqcd_gauge_force(lqcd_field *P, const lqcd_field *U, double beta, double coeff, void *stream)
{
    return lqcd_gauge_force_ex(P, U, beta, coeff, LQCD_F64, stream);
}

lqcd_status lqcd_fermion_force_ex(lqcd_field *P, const lqcd_field *U, const lqcd_field *X_e, double kappa,
                                  double coeff, lqcd_prec arith, void *stream)
{
    LQCD_REQUIRE(P && U && X_e && P->kind == LQCD_MOMENTUM && U->kind == LQCD_GAUGE && U->prec == LQCD_F64,
                 "fermion_force needs a momentum field and an F64 gauge field");
    LQCD_REQUIRE(X_e->kind == LQCD_SPINOR_EVEN && X_e->prec == LQCD_F64, "fermion_force: X_e must be EVEN F64");
    LQCD_REQUIRE(same_lattice(P->lat, U->lat) && same_lattice(X_e->lat, U->lat), "fermion_force: lattices differ");
    LQCD_REQUIRE(arith == LQCD_F64 || arith == LQCD_F32, "fermion_force: arithmetic must be F64 or F32");
    FieldPtr Ao, Ye, Bo, Xc, Uf;
    cudaStream_t s = (cudaStream_t)stream;
    LQCD_TRY(lqcd_field_alloc(&U->lat, LQCD_SPINOR_ODD, arith, 0, &Ao.f));
    LQCD_TRY(lqcd_field_alloc(&U->lat, LQCD_SPINOR_EVEN, arith, 0, &Ye.f));
    LQCD_TRY(lqcd_field_alloc(&U->lat, LQCD_SPINOR_ODD, arith, 0, &Bo.f));
    if (arith != LQCD_F64) {
        LQCD_TRY(lqcd_field_alloc(&U->lat, LQCD_SPINOR_EVEN, arith, 0, &Xc.f));
        LQCD_TRY(lqcd_field_alloc(&U->lat, LQCD_GAUGE, LQCD_F32, 12, &Uf.f));
        LQCD_TRY(lqcd_field_copy(Uf.f, U, s));
    }
    LQCD_TRY(fermion_force_dev(P, U, Uf.f, X_e, kappa, coeff, Ao.f, Ye.f, Bo.f, Xc.f, s, nullptr));
    LQCD_CUDA(cudaStreamSynchronize(s)); // temporaries are freed on return
    return LQCD_OK;
}

lqcd_status lqcd_fermion_force(lqcd_field *P, const lqcd_field *U, const lqcd_field *X_e, double kappa, double coeff,
                               void *stream)
{
    return lqcd_fermion_force_ex(P, U, X_e, kappa, coeff, LQCD_F64, stream);
}

} // extern "C"
