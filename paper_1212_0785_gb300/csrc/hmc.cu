// hmc.cu -- Hybrid Monte Carlo driver: refresh, molecular dynamics with merged
// kicks (leapfrog or Omelyan 2MN, optionally nested on two time scales),
// Hamiltonian, Metropolis and reunitarization, every field operation on the
// device (paper Sec. 1: the whole trajectory runs on the accelerator; Sec. 6.2:
// Nf = 2 Wilson HMC, with mass preconditioning and chronological guesses among
// its production features).
//
// The host only sequences kernels and reads back the scalars it must decide
// on (solver convergence, dH and the Metropolis uniform, the plaquette).
#include <chrono>
#include <cmath>
#include <cstring>

#include "batch.cuh"
#include "cg.cuh"
#include "chains.cuh"
#include "su3_device.cuh"

namespace lqcd {

// defined in field.cu / force.cu
// (weighted: the anisotropic gauge action's plane weights; false: the plaquette observable)
lqcd_status plaquette_sum(const lqcd_field *U, double *dst_dev, DevBuf &part, cudaStream_t s, bool weighted);
lqcd_status plaquette_sum_df(const lqcd_field *Udf, double *dst_dev, DevBuf &part, cudaStream_t s, bool weighted);
lqcd_status kinetic_sum(const lqcd_field *P, double *dst_dev, DevBuf &part, cudaStream_t s);
lqcd_status reunitarize_dev(lqcd_field *U, double *dst_dev, DevBuf &part, cudaStream_t s);
lqcd_status link_update_dev(lqcd_field *U, const lqcd_field *P, double c, lqcd_field *Us, lqcd_field *Uf, bool fast,
                            cudaStream_t s, lqcd_field *Udf, bool write_f64);
lqcd_status links_from_df(lqcd_field *U, const lqcd_field *Udf, cudaStream_t s);
lqcd_status momentum_refresh_dev(lqcd_field *P, uint32_t seed, uint32_t chain, uint32_t traj, cudaStream_t s);
lqcd_status eta_refresh_dev(lqcd_field *E, uint32_t seed, uint32_t chain, uint32_t traj, cudaStream_t s,
                            uint32_t purpose);
lqcd_status gauge_force_dev(lqcd_field *P, const lqcd_field *U, const lqcd_field *Uf, double beta, double coeff,
                            lqcd_prec arith, cudaStream_t s);
lqcd_status fermion_force_dev(lqcd_field *P, const lqcd_field *U, const lqcd_field *Uf, const lqcd_field *X,
                              double kappa, double coeff, lqcd_field *Ao, lqcd_field *Ye, lqcd_field *Bo, lqcd_field *Xc,
                              cudaStream_t s, const lqcd_field *Y);

constexpr double OMELYAN_LAMBDA = 0.1931833275037836;

// first uniform of Philox(counter (0, 0, 3, traj), key (seed, chain))
__global__ void metropolis_uniform_kernel(double *out, uint32_t seed, uint32_t chain, uint32_t traj)
{
    uint4 x = philox4x32_10(make_uint4(0u, 0u, 3u, traj), make_uint2(seed, chain));
    out[0] = u52(x.x, x.y);
}

// out = sum_{i<m} w_i x_i over n double2 elements (m <= 4)
__global__ void combine_kernel(double2 *out, const double2 *x0, const double2 *x1, const double2 *x2,
                               const double2 *x3, double w0, double w1, double w2, double w3, int m, size_t n)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 a = x0[i];
    double2 r = make_double2(w0 * a.x, w0 * a.y);
    if (m > 1) {
        a = x1[i];
        r.x += w1 * a.x, r.y += w1 * a.y;
    }
    if (m > 2) {
        a = x2[i];
        r.x += w2 * a.x, r.y += w2 * a.y;
    }
    if (m > 3) {
        a = x3[i];
        r.x += w3 * a.x, r.y += w3 * a.y;
    }
    out[i] = r;
}

} // namespace lqcd

using namespace lqcd;

constexpr int CHRONO_MAX = 4;

// One pseudofermion action of the trajectory: its field, the last solution of
// its solve and what the chronological guess of its next solve needs.
struct PfTerm {
    lqcd::FieldPtr phi, X;
    lqcd::FieldPtr chi; // ratio action: the right-hand side W^dag phi of its solve
    bool have_guess = false; // X holds a solution for the current phi
    uint64_t phi_stamp = 0;  // stamp of phi's contents (new at every refresh and public entry)
    bool last_ok = false;    // the last solve converged, at molecular-dynamics time last_t
    double last_t = -1;
    // solutions of this trajectory's solves and the molecular-dynamics times
    // (sum of the drifts since the refresh) of their links;
    // hist[(head - 1) mod CHRONO_MAX] is the latest
    lqcd::FieldPtr hist[CHRONO_MAX];
    double hist_t[CHRONO_MAX] = {0, 0, 0, 0};
    int n_hist = 0, head = 0;
    void reset()
    {
        have_guess = last_ok = false;
        n_hist = 0;
        phi_stamp = lqcd::new_content_stamp();
    }
};

// pseudofermion terms: the fermion action (the ratio action when mass
// preconditioned) and the heavy Hasenbusch action
enum { PF_MAIN = 0, PF_HEAVY = 1 };
// force terms of a time-scale level
enum { TERM_GAUGE = 1, TERM_FERMION = 2, TERM_HEAVY = 4 };

struct lqcd_hmc_state {
    lqcd_field *U = nullptr; // borrowed
    uint32_t seed = 0, chain = 0, traj = 0;
    lqcd::FieldPtr P, eta, Ao, Ye, Bo, Ubak, Us;
    lqcd::FieldPtr eta_h, z;                // Hasenbusch refresh (allocated on first use)
    lqcd::FieldPtr Ao32, Ye32, Bo32, X32;   // FP32 fermion-force temporaries (allocated on first use)
    lqcd::FieldPtr Uf;                      // FP32 12-real link copy for the FP32 molecular dynamics
    lqcd::FieldPtr Udf; // float-float link copy of the mixed solver, kept current by every link update
    bool u_lags = false; // U (FP64) not yet written since link updates that wrote only the copies
    PfTerm pf[2];
    lqcd::CgWorkspace ws;
    lqcd::DevBuf part, scal;
    double H0 = 0;
    double md_time = 0;
    double pending[2] = {0, 0}; // kick coefficients of each level not yet applied
    // statistics of the current trajectory
    int cg_iters = 0, n_solves = 0, cg_failures = 0, cg_accurate = 0, cg_failed_checks = 0, cg_refined = 0;
    double cg_res_max = 0;
};

namespace lqcd {

static bool hasenbusch(const lqcd_hmc_params *p) { return p->n_flavors == 2 && p->hasenbusch_kappa != 0.0; }
static int n_levels(const lqcd_hmc_params *p) { return p->gauge_substeps >= 2 ? 2 : 1; }

// the force terms integrated on a level
static int level_terms(const lqcd_hmc_params *p, int level)
{
    if (n_levels(p) == 1) return TERM_GAUGE | TERM_FERMION | TERM_HEAVY;
    if (level == 0) return TERM_FERMION | (p->heavy_inner ? 0 : TERM_HEAVY);
    return TERM_GAUGE | (p->heavy_inner ? TERM_HEAVY : 0);
}

static lqcd_status check_params(const lqcd_hmc_params *p)
{
    LQCD_REQUIRE(p != nullptr, "hmc: params is NULL");
    LQCD_REQUIRE(p->nsteps > 0 && p->tau > 0, "hmc: nsteps and tau must be positive");
    LQCD_REQUIRE(p->integrator == LQCD_LEAPFROG || p->integrator == LQCD_OMELYAN, "hmc: unknown integrator");
    LQCD_REQUIRE(p->n_flavors == 0 || p->n_flavors == 2, "hmc: n_flavors must be 0 or 2");
    if (p->n_flavors == 2) {
        LQCD_REQUIRE(p->cg.tol > 0 && p->cg.maxiter > 0, "hmc: cg tol and maxiter must be positive");
        LQCD_REQUIRE(p->cg.sloppy == LQCD_F64 || (p->cg.delta > 0 && p->cg.delta < 1),
                     "hmc: cg delta must lie in (0, 1) for a mixed solve");
        LQCD_REQUIRE(p->hasenbusch_kappa >= 0 && p->hasenbusch_kappa < p->kappa,
                     "hmc: hasenbusch_kappa must be 0 (off) or lie in (0, kappa)");
    }
    LQCD_REQUIRE(p->force_prec == LQCD_F64 || p->force_prec == LQCD_F32, "hmc: force_prec must be F64 or F32");
    LQCD_REQUIRE(p->chrono >= 0 && p->chrono <= CHRONO_MAX, "hmc: chrono must lie in 0..%d", CHRONO_MAX);
    LQCD_REQUIRE(p->chrono_mre == 0 || p->chrono_mre == 1, "hmc: chrono_mre must be 0 or 1");
    LQCD_REQUIRE(p->gauge_substeps >= 0, "hmc: gauge_substeps must be >= 0");
    return LQCD_OK;
}

// sloppy link copy matching the solver precision (NULL for FP64), and the FP32
// link copy of the FP32 molecular dynamics
static lqcd_status ensure_sloppy(lqcd_hmc_state *st, const lqcd_hmc_params *p, cudaStream_t s)
{
    if (p->force_prec == LQCD_F32) {
        if (!st->Uf.f) LQCD_TRY(lqcd_field_alloc(&st->U->lat, LQCD_GAUGE, LQCD_F32, 12, &st->Uf.f));
        LQCD_TRY(lqcd_field_copy(st->Uf.f, st->U, s));
    }
    if (p->n_flavors == 0 || p->cg.sloppy == LQCD_F64) return LQCD_OK;
    if (st->Us.f && st->Us.f->prec != p->cg.sloppy) {
        lqcd_field_free(st->Us.f);
        st->Us.f = nullptr;
    }
    if (!st->Us.f) LQCD_TRY(lqcd_field_alloc(&st->U->lat, LQCD_GAUGE, p->cg.sloppy, 12, &st->Us.f));
    if (!st->Udf.f) LQCD_TRY(field_alloc_df(&st->U->lat, LQCD_GAUGE, &st->Udf.f));
    LQCD_TRY(split_links(st->Udf.f, st->U, s));
    st->ws.udf_ext = st->Udf.f;
    return lqcd_field_copy(st->Us.f, st->U, s);
}

// allocates f unless it is already there: a call that failed half way (the
// allocator returned NULL) leaves the fields it made, and the next call makes
// only the missing ones
static lqcd_status ensure_field(FieldPtr &f, const lqcd_lattice &lat, lqcd_kind kind, lqcd_prec prec)
{
    return f.f ? LQCD_OK : lqcd_field_alloc(&lat, kind, prec, 0, &f.f);
}

static lqcd_status ensure_hasenbusch(lqcd_hmc_state *st)
{
    const lqcd_lattice &lat = st->U->lat;
    LQCD_TRY(ensure_field(st->eta_h, lat, LQCD_SPINOR_EVEN, LQCD_F64));
    LQCD_TRY(ensure_field(st->z, lat, LQCD_SPINOR_EVEN, LQCD_F64));
    LQCD_TRY(ensure_field(st->pf[PF_MAIN].chi, lat, LQCD_SPINOR_EVEN, LQCD_F64));
    LQCD_TRY(ensure_field(st->pf[PF_HEAVY].phi, lat, LQCD_SPINOR_EVEN, LQCD_F64));
    return ensure_field(st->pf[PF_HEAVY].X, lat, LQCD_SPINOR_EVEN, LQCD_F64);
}

static lqcd_field *sloppy_links(lqcd_hmc_state *st, const lqcd_hmc_params *p)
{
    return (p->n_flavors == 2 && p->cg.sloppy != LQCD_F64) ? st->Us.f : nullptr;
}

// The initial guess of term t's next solve, in its X; returns whether there
// is one.  chrono 1: the previous solution (already in X).  chrono k >= 2: the
// polynomial through the last k solutions at their molecular-dynamics times,
// evaluated at the current time (Lagrange form); the trajectory's solves come
// at evenly spaced times, so this is the extrapolation x_n ~ 2 x_{n-1} -
// x_{n-2} (k = 2), 3 x_{n-1} - 3 x_{n-2} + x_{n-3} (k = 3), ...  A solve at the
// time of the previous one (the action at the end of the trajectory) starts
// from the previous solution.
//
// With chrono_mre the solutions used (latest first) also go to *mre, for the
// solver's minimal residual refinement of the extrapolated guess.
static lqcd_status prepare_guess(lqcd_hmc_state *st, PfTerm &t, const lqcd_hmc_params *p, cudaStream_t s,
                                 int *guess, MreInput *mre = nullptr)
{
    if (mre) mre->n = 0;
    *guess = (p->chrono && t.have_guess) ? 1 : 0;
    if (!*guess || p->chrono < 2 || t.n_hist < 2) return LQCD_OK;
    const int latest = (t.head + CHRONO_MAX - 1) % CHRONO_MAX;
    if (t.hist_t[latest] == st->md_time) return LQCD_OK;
    int idx[CHRONO_MAX], m = 0;
    const int kmax = std::min(p->chrono, CHRONO_MAX);
    for (int k = 0; k < t.n_hist && m < kmax; k++) {
        int i = (t.head + CHRONO_MAX - 1 - k) % CHRONO_MAX;
        bool dup = false;
        for (int j = 0; j < m; j++) dup = dup || t.hist_t[idx[j]] == t.hist_t[i];
        if (!dup) idx[m++] = i;
    }
    if (m < 2) return LQCD_OK;
    double w[CHRONO_MAX] = {0, 0, 0, 0};
    const double2 *x[CHRONO_MAX] = {nullptr, nullptr, nullptr, nullptr};
    for (int a = 0; a < m; a++) {
        double l = 1.0;
        for (int b = 0; b < m; b++)
            if (b != a) l *= (st->md_time - t.hist_t[idx[b]]) / (t.hist_t[idx[a]] - t.hist_t[idx[b]]);
        w[a] = l;
        x[a] = (const double2 *)t.hist[idx[a]].f->data;
    }
    size_t n = t.X.f->bytes / sizeof(double2);
    combine_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((double2 *)t.X.f->data, x[0], x[1], x[2], x[3], w[0],
                                                               w[1], w[2], w[3], m, n);
    LQCD_LAUNCHED();
    if (mre && p->chrono_mre && p->cg.sloppy != LQCD_F64) {
        mre->n = m;
        for (int a = 0; a < m; a++) mre->x[a] = t.hist[idx[a]].f;
        mre->links = p->force_prec == LQCD_F32 ? st->Uf.f : nullptr; // the FP32 copy is current then
    }
    return LQCD_OK;
}

// record a solve's outcome and solution for later guesses
static lqcd_status record_solution(lqcd_hmc_state *st, PfTerm &t, const lqcd_hmc_params *p, lqcd_status rc,
                                   cudaStream_t s)
{
    const bool ok = rc == LQCD_OK || rc == LQCD_ENOCONV;
    t.have_guess = ok;
    t.last_ok = rc == LQCD_OK;
    t.last_t = st->md_time;
    if (!ok || p->chrono < 2) return LQCD_OK;
    lqcd_field *&slot = t.hist[t.head].f;
    if (!slot) LQCD_TRY(lqcd_field_alloc(&st->U->lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &slot));
    LQCD_CUDA(cudaMemcpyAsync(slot->data, t.X.f->data, t.X.f->bytes, cudaMemcpyDeviceToDevice, s));
    t.hist_t[t.head] = st->md_time;
    t.head = (t.head + 1) % CHRONO_MAX;
    t.n_hist = std::min(t.n_hist + 1, CHRONO_MAX);
    return LQCD_OK;
}

static lqcd_status count_solve(lqcd_hmc_state *st, lqcd_status rc, const lqcd_cg_info &info)
{
    st->cg_iters += info.iters;
    st->cg_accurate += info.accurate_residuals;
    st->cg_failed_checks += info.failed_checks;
    st->cg_refined += info.guess_refined;
    st->n_solves++;
    st->cg_res_max = std::max(st->cg_res_max, info.true_rel_res);
    if (rc == LQCD_ENOCONV) {
        st->cg_failures++;
        return LQCD_OK; // the trajectory goes on; the failure is reported in its info
    }
    return rc;
}

// X_t = (Mhat(kappa)^dag Mhat(kappa))^-1 b with the term's chronological guess
static lqcd_status solve(lqcd_hmc_state *st, PfTerm &t, const lqcd_hmc_params *p, double kappa,
                         const lqcd_field *b, cudaStream_t s)
{
    lqcd_cg_info info{};
    lqcd_cg_params cg = p->cg;
    MreInput mre;
    LQCD_TRY(prepare_guess(st, t, p, s, &cg.guess, &mre));
    // phi is constant between refreshes: its float-float copy is made once
    lqcd_status rc = cg_solve_ws(st->ws, t.X.f, st->U, sloppy_links(st, p), b, kappa, cg, &info, s,
                                 mre.n >= 2 ? &mre : nullptr, b == t.phi.f ? t.phi_stamp : 0);
    LQCD_TRY(record_solution(st, t, p, rc, s));
    return count_solve(st, rc, info);
}

static lqcd_status ensure_f32_temps(lqcd_hmc_state *st)
{
    const lqcd_lattice &lat = st->U->lat;
    LQCD_TRY(ensure_field(st->Ao32, lat, LQCD_SPINOR_ODD, LQCD_F32));
    LQCD_TRY(ensure_field(st->Ye32, lat, LQCD_SPINOR_EVEN, LQCD_F32));
    LQCD_TRY(ensure_field(st->Bo32, lat, LQCD_SPINOR_ODD, LQCD_F32));
    return ensure_field(st->X32, lat, LQCD_SPINOR_EVEN, LQCD_F32);
}

// P <- P - c F with F the force of -2 Re[Y^dag dMhat(kappa) X] (Y = Mhat X if Y is NULL)
static lqcd_status fermion_force(lqcd_hmc_state *st, const lqcd_hmc_params *p, const lqcd_field *X,
                                 const lqcd_field *Y, double kappa, double c, cudaStream_t s)
{
    if (p->force_prec == LQCD_F32) {
        LQCD_TRY(ensure_f32_temps(st));
        return fermion_force_dev(st->P.f, st->U, st->Uf.f, X, kappa, c, st->Ao32.f, st->Ye32.f, st->Bo32.f,
                                 st->X32.f, s, Y);
    }
    return fermion_force_dev(st->P.f, st->U, nullptr, X, kappa, c, st->Ao.f, st->Ye.f, st->Bo.f, nullptr, s, Y);
}

// the ratio action's right-hand side chi = W^dag phi_r in FP64 (exact: the
// action) or in the precision of the forces (fast: a force evaluation)
static lqcd_status ratio_rhs(lqcd_hmc_state *st, const lqcd_hmc_params *p, bool exact, cudaStream_t s)
{
    PfTerm &t = st->pf[PF_MAIN];
    if (exact || p->force_prec != LQCD_F32)
        return mhat_apply(t.chi.f, st->U, t.phi.f, p->hasenbusch_kappa, 1, st->Ao.f, nullptr, s);
    LQCD_TRY(ensure_f32_temps(st));
    LQCD_TRY(lqcd_field_copy(st->X32.f, t.phi.f, s));
    LQCD_TRY(mhat_apply(st->Ye32.f, st->Uf.f, st->X32.f, p->hasenbusch_kappa, 1, st->Ao32.f, nullptr, s));
    return lqcd_field_copy(t.chi.f, st->Ye32.f, s);
}

// P <- P - c F of the given force terms at the current links
static lqcd_status apply_forces(lqcd_hmc_state *st, const lqcd_hmc_params *p, int terms, double c, cudaStream_t s)
{
    if (terms & TERM_GAUGE) LQCD_TRY(gauge_force_dev(st->P.f, st->U, st->Uf.f, p->beta, c, p->force_prec, s));
    if (p->n_flavors != 2) return LQCD_OK;
    if (terms & TERM_FERMION) {
        PfTerm &t = st->pf[PF_MAIN];
        if (!hasenbusch(p)) {
            LQCD_TRY(solve(st, t, p, p->kappa, t.phi.f, s));
            LQCD_TRY(fermion_force(st, p, t.X.f, nullptr, p->kappa, c, s));
        } else {
            LQCD_TRY(ratio_rhs(st, p, false, s));
            LQCD_TRY(solve(st, t, p, p->kappa, t.chi.f, s));
            LQCD_TRY(fermion_force(st, p, t.X.f, nullptr, p->kappa, c, s));
            LQCD_TRY(fermion_force(st, p, t.X.f, t.phi.f, p->hasenbusch_kappa, -c, s));
        }
    }
    if ((terms & TERM_HEAVY) && hasenbusch(p)) {
        PfTerm &t = st->pf[PF_HEAVY];
        LQCD_TRY(solve(st, t, p, p->hasenbusch_kappa, t.phi.f, s));
        LQCD_TRY(fermion_force(st, p, t.X.f, nullptr, p->hasenbusch_kappa, c, s));
    }
    return LQCD_OK;
}

// Kicks are queued per level and applied when the links are about to change
// (or at the end), so kicks of adjacent steps at the same links merge into
// one force evaluation with the summed coefficient.
static void kick(lqcd_hmc_state *st, int level, double c) { st->pending[level] += c; }

static lqcd_status flush_kicks(lqcd_hmc_state *st, const lqcd_hmc_params *p, cudaStream_t s)
{
    for (int l = 0; l < n_levels(p); l++) {
        if (st->pending[l] == 0.0) continue;
        const double c = st->pending[l];
        st->pending[l] = 0.0;
        LQCD_TRY(apply_forces(st, p, level_terms(p, l), c, s));
    }
    return LQCD_OK;
}

static lqcd_status drift(lqcd_hmc_state *st, const lqcd_hmc_params *p, double c, cudaStream_t s)
{
    LQCD_TRY(flush_kicks(st, p, s));
    bool fast = p->force_prec == LQCD_F32;
    st->md_time += c;
    // with FP32 forces and the mixed solver the molecular dynamics reads only
    // the link copies, so the FP64 links are written once, after it
    // (sync_master_links), instead of at every update
    lqcd_field *Udf = sloppy_links(st, p) ? st->Udf.f : nullptr;
    const bool lag = fast && Udf;
    if (lag) st->u_lags = true;
    return link_update_dev(st->U, st->P.f, c, sloppy_links(st, p), fast ? st->Uf.f : nullptr, fast, s, Udf, !lag);
}

// the FP64 links from the float-float copy after molecular dynamics that
// updated only the copies
static lqcd_status sync_master_links(lqcd_hmc_state *st, cudaStream_t s)
{
    if (!st->u_lags) return LQCD_OK;
    st->u_lags = false;
    return links_from_df(st->U, st->Udf.f, s);
}

// scalars[0] = plaquette sum, [1] = sum p^2, [2] = fermion term.  With the
// mixed solver the float-float link copy is current (split at the refresh,
// written by every link update), and the plaquette comes from it on the FP32
// pipes instead of the FP64 one.
static lqcd_status hamiltonian_parts(lqcd_hmc_state *st, const lqcd_hmc_params *p, cudaStream_t s)
{
    double *d = (double *)st->scal.p;
    if (sloppy_links(st, p) && st->Udf.f)
        LQCD_TRY(plaquette_sum_df(st->Udf.f, d + 0, st->part, s, true));
    else
        LQCD_TRY(plaquette_sum(st->U, d + 0, st->part, s, true));
    LQCD_TRY(kinetic_sum(st->P.f, d + 1, st->part, s));
    return LQCD_OK;
}

// H = T + S_g + S_f from the sums h: h[0] the plaquette sum weighted by the
// gauge action's plane weights, whose total over all plaquettes is
// V (3 / xi0 + 3 xi0) (6 V when isotropic)
static double hamiltonian_from(const lqcd_hmc_state *st, const lqcd_hmc_params *p, const double *h)
{
    double V = 2.0 * st->U->Vh;
    const Geo g = make_geo(st->U->lat);
    const double W = g.aniso ? V * (3.0 / g.xi0 + 3.0 * g.xi0) : 6.0 * V;
    return 0.5 * h[1] + p->beta * (W - h[0]) + (p->n_flavors == 2 ? h[2] : 0.0);
}

static lqcd_status refresh(lqcd_hmc_state *st, const lqcd_hmc_params *p, double *H0, cudaStream_t s)
{
    for (PfTerm &t : st->pf) t.reset(); // new pseudofermions: old solutions are no guesses
    st->md_time = 0;
    st->pending[0] = st->pending[1] = 0;
    LQCD_TRY(ensure_sloppy(st, p, s));
    LQCD_TRY(momentum_refresh_dev(st->P.f, st->seed, st->chain, st->traj, s));
    double *d = (double *)st->scal.p;
    LQCD_TRY(hamiltonian_parts(st, p, s));
    double h[4] = {0, 0, 0, 0};
    if (p->n_flavors == 2) {
        PfTerm &t = st->pf[PF_MAIN];
        LQCD_TRY(eta_refresh_dev(st->eta.f, st->seed, st->chain, st->traj, s, 2u));
        if (!hasenbusch(p)) {
            LQCD_TRY(mhat_apply(t.phi.f, st->U, st->eta.f, p->kappa, 1, st->Ao.f, nullptr, s));
        } else {
            // phi_h = W^dag eta_h;  phi_r = W (W^dag W)^-1 Mhat^dag eta
            LQCD_TRY(ensure_hasenbusch(st));
            const double kh = p->hasenbusch_kappa;
            LQCD_TRY(eta_refresh_dev(st->eta_h.f, st->seed, st->chain, st->traj, s, 4u));
            LQCD_TRY(mhat_apply(st->pf[PF_HEAVY].phi.f, st->U, st->eta_h.f, kh, 1, st->Ao.f, nullptr, s));
            LQCD_TRY(mhat_apply(t.chi.f, st->U, st->eta.f, p->kappa, 1, st->Ao.f, nullptr, s));
            lqcd_cg_info info{};
            lqcd_cg_params cg = p->cg;
            cg.guess = 0;
            lqcd_status rc = cg_solve_ws(st->ws, st->z.f, st->U, sloppy_links(st, p), t.chi.f, kh, cg, &info, s);
            LQCD_TRY(count_solve(st, rc, info));
            LQCD_TRY(mhat_apply(t.phi.f, st->U, st->z.f, kh, 0, st->Ao.f, nullptr, s));
            LQCD_TRY(spinor_dot_dev(st->eta_h.f, st->eta_h.f, d + 3, st->part, s));
        }
        LQCD_TRY(spinor_dot_dev(st->eta.f, st->eta.f, d + 2, st->part, s));
    }
    LQCD_TRY(read_scalars(d, h, hasenbusch(p) ? 4 : 3, s));
    h[2] += h[3];
    st->H0 = hamiltonian_from(st, p, h);
    if (H0) *H0 = st->H0;
    return LQCD_OK;
}

// the term's solution is reusable for the action at the current links: a
// chronological guess would start from it and stop at once
static bool reusable(const lqcd_hmc_state *st, const PfTerm &t, const lqcd_hmc_params *p)
{
    return p->chrono && t.have_guess && t.last_ok && t.last_t == st->md_time;
}

// H of the current fields.  reuse_last (inside a trajectory, right after the
// last kicks): a term whose last solve was of the same system and converged
// uses that solution as it is (counted as a solve of 0 iterations).
static lqcd_status hamiltonian(lqcd_hmc_state *st, const lqcd_hmc_params *p, double *H, cudaStream_t s,
                               bool reuse_last = false)
{
    double *d = (double *)st->scal.p;
    LQCD_TRY(hamiltonian_parts(st, p, s));
    double h[4] = {0, 0, 0, 0};
    if (p->n_flavors == 2) {
        PfTerm &t = st->pf[PF_MAIN];
        if (!hasenbusch(p)) {
            if (reuse_last && reusable(st, t, p))
                st->n_solves++;
            else
                LQCD_TRY(solve(st, t, p, p->kappa, t.phi.f, s));
            LQCD_TRY(spinor_dot_dev(t.phi.f, t.X.f, d + 2, st->part, s));
        } else {
            // the ratio action needs chi in FP64; the forces may have used FP32
            const bool exact_chi = p->force_prec != LQCD_F32;
            if (reuse_last && exact_chi && reusable(st, t, p)) {
                st->n_solves++;
            } else {
                LQCD_TRY(ratio_rhs(st, p, true, s));
                LQCD_TRY(solve(st, t, p, p->kappa, t.chi.f, s));
            }
            LQCD_TRY(spinor_dot_dev(t.chi.f, t.X.f, d + 2, st->part, s));
            PfTerm &th = st->pf[PF_HEAVY];
            if (reuse_last && reusable(st, th, p))
                st->n_solves++;
            else
                LQCD_TRY(solve(st, th, p, p->hasenbusch_kappa, th.phi.f, s));
            LQCD_TRY(spinor_dot_dev(th.phi.f, th.X.f, d + 3, st->part, s));
        }
    }
    LQCD_TRY(read_scalars(d, h, hasenbusch(p) ? 4 : 3, s));
    h[2] += h[3];
    *H = hamiltonian_from(st, p, h);
    return LQCD_OK;
}

static lqcd_status integrate_level(lqcd_hmc_state *st, const lqcd_hmc_params *p, int level, double t, int n,
                                   cudaStream_t s);

// a drift of a level: the next level's integration, or the link update
static lqcd_status inner(lqcd_hmc_state *st, const lqcd_hmc_params *p, int level, double t, cudaStream_t s)
{
    if (level + 1 < n_levels(p)) return integrate_level(st, p, level + 1, t, p->gauge_substeps, s);
    return drift(st, p, t, s);
}

// n steps of the scheme over time t on one level (Sexton-Weingarten nesting:
// the inner level integrates each drift of the outer one)
static lqcd_status integrate_level(lqcd_hmc_state *st, const lqcd_hmc_params *p, int level, double t, int n,
                                   cudaStream_t s)
{
    const double h = t / n;
    for (int k = 0; k < n; k++) {
        if (p->integrator == LQCD_LEAPFROG) {
            kick(st, level, 0.5 * h);
            LQCD_TRY(inner(st, p, level, h, s));
            kick(st, level, 0.5 * h);
        } else {
            const double lam = OMELYAN_LAMBDA;
            kick(st, level, lam * h);
            LQCD_TRY(inner(st, p, level, 0.5 * h, s));
            kick(st, level, (1.0 - 2.0 * lam) * h);
            LQCD_TRY(inner(st, p, level, 0.5 * h, s));
            kick(st, level, lam * h);
        }
    }
    return LQCD_OK;
}

static lqcd_status integrate(lqcd_hmc_state *st, const lqcd_hmc_params *p, double t, int n, cudaStream_t s)
{
    lqcd_status rc = integrate_level(st, p, 0, t, n, s);
    if (rc == LQCD_OK) rc = flush_kicks(st, p, s);
    // the FP64 links hold the latest update even after a failure half way
    const lqcd_status rs = sync_master_links(st, s);
    return rc != LQCD_OK ? rc : rs;
}

static void reset_stats(lqcd_hmc_state *st)
{
    st->cg_iters = st->n_solves = st->cg_failures = st->cg_accurate = st->cg_failed_checks = st->cg_refined = 0;
    st->cg_res_max = 0;
}

} // namespace lqcd

extern "C" {

lqcd_status lqcd_hmc_state_create(lqcd_field *U, uint32_t seed, uint32_t chain, uint32_t traj0, lqcd_hmc_state **out)
{
    LQCD_REQUIRE(U && out, "hmc_state_create: NULL argument");
    LQCD_REQUIRE(U->kind == LQCD_GAUGE && U->prec == LQCD_F64, "hmc_state_create: U must be an F64 gauge field");
    lqcd_hmc_state *st = new lqcd_hmc_state();
    st->U = U;
    st->seed = seed;
    st->chain = chain;
    st->traj = traj0;
    const lqcd_lattice &lat = U->lat;
    lqcd_status rc = LQCD_OK;
    if (rc == LQCD_OK) rc = lqcd_field_alloc(&lat, LQCD_MOMENTUM, LQCD_F64, 0, &st->P.f);
    if (rc == LQCD_OK) rc = lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &st->eta.f);
    if (rc == LQCD_OK) rc = lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &st->pf[PF_MAIN].phi.f);
    if (rc == LQCD_OK) rc = lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &st->pf[PF_MAIN].X.f);
    if (rc == LQCD_OK) rc = lqcd_field_alloc(&lat, LQCD_SPINOR_ODD, LQCD_F64, 0, &st->Ao.f);
    if (rc == LQCD_OK) rc = lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &st->Ye.f);
    if (rc == LQCD_OK) rc = lqcd_field_alloc(&lat, LQCD_SPINOR_ODD, LQCD_F64, 0, &st->Bo.f);
    if (rc == LQCD_OK) rc = lqcd_field_alloc(&lat, LQCD_GAUGE, LQCD_F64, 18, &st->Ubak.f);
    if (rc == LQCD_OK) rc = st->scal.alloc(8 * sizeof(double), nullptr);
    if (rc != LQCD_OK) {
        delete st;
        return rc;
    }
    *out = st;
    return LQCD_OK;
}

lqcd_status lqcd_hmc_state_destroy(lqcd_hmc_state *s)
{
    cudaDeviceSynchronize();
    delete s;
    return LQCD_OK;
}

lqcd_status lqcd_hmc_state_fields(lqcd_hmc_state *s, lqcd_field **U, lqcd_field **P, lqcd_field **phi)
{
    LQCD_REQUIRE(s, "hmc_state_fields: NULL state");
    if (U) *U = s->U;
    if (P) *P = s->P.f;
    if (phi) *phi = s->pf[PF_MAIN].phi.f;
    return LQCD_OK;
}

lqcd_status lqcd_hmc_state_traj(lqcd_hmc_state *s, uint32_t *traj_out, const uint32_t *traj_in)
{
    LQCD_REQUIRE(s, "hmc_state_traj: NULL state");
    if (traj_in) s->traj = *traj_in;
    if (traj_out) *traj_out = s->traj;
    return LQCD_OK;
}

lqcd_status lqcd_hmc_refresh(lqcd_hmc_state *s, const lqcd_hmc_params *p, double *H0, void *stream)
{
    LQCD_REQUIRE(s, "hmc_refresh: NULL state");
    LQCD_TRY(check_params(p));
    return refresh(s, p, H0, (cudaStream_t)stream);
}

lqcd_status lqcd_hmc_hamiltonian(lqcd_hmc_state *s, const lqcd_hmc_params *p, double *H, void *stream)
{
    LQCD_REQUIRE(s && H, "hmc_hamiltonian: NULL argument");
    LQCD_TRY(check_params(p));
    LQCD_REQUIRE(!hasenbusch(p) || s->eta_h.f, "hmc_hamiltonian: no Hasenbusch refresh has been done");
    LQCD_TRY(ensure_sloppy(s, p, (cudaStream_t)stream));
    for (PfTerm &t : s->pf) t.phi_stamp = new_content_stamp(); // the caller may have written phi
    return hamiltonian(s, p, H, (cudaStream_t)stream);
}

lqcd_status lqcd_md_step(lqcd_hmc_state *s, const lqcd_hmc_params *p, void *stream)
{
    LQCD_REQUIRE(s, "md_step: NULL state");
    LQCD_TRY(check_params(p));
    LQCD_REQUIRE(!hasenbusch(p) || s->eta_h.f, "md_step: no Hasenbusch refresh has been done");
    cudaStream_t st = (cudaStream_t)stream;
    LQCD_TRY(ensure_sloppy(s, p, st));
    s->pending[0] = s->pending[1] = 0;
    for (PfTerm &t : s->pf) t.phi_stamp = new_content_stamp(); // the caller may have written phi
    return integrate(s, p, p->tau / p->nsteps, 1, st);
}

lqcd_status lqcd_hmc_trajectory(lqcd_hmc_state *s, const lqcd_hmc_params *p, lqcd_traj_info *info, void *stream)
{
    LQCD_REQUIRE(s, "hmc_trajectory: NULL state");
    LQCD_TRY(check_params(p));
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    reset_stats(s);
    LQCD_CUDA(cudaMemcpyAsync(s->Ubak.f->data, s->U->data, s->U->bytes, cudaMemcpyDeviceToDevice, st));
    double H0 = 0, H1 = 0;
    lqcd_status rc = refresh(s, p, &H0, st);
    if (rc == LQCD_OK) rc = integrate(s, p, p->tau, p->nsteps, st);
    if (rc == LQCD_OK) rc = hamiltonian(s, p, &H1, st, true);
    double dH = H1 - H0;
    double *d = (double *)s->scal.p;
    metropolis_uniform_kernel<<<1, 1, 0, st>>>(d + 4, s->seed, s->chain, s->traj);
    LQCD_LAUNCHED();
    double u = 0;
    LQCD_TRY(read_scalars(d + 4, &u, 1, st));
    bool accept = rc == LQCD_OK && std::isfinite(dH) && (!p->metropolis || u < std::exp(-dH));
    if (!accept) LQCD_CUDA(cudaMemcpyAsync(s->U->data, s->Ubak.f->data, s->U->bytes, cudaMemcpyDeviceToDevice, st));
    double maxdev = 0;
    if (p->reunitarize) {
        LQCD_TRY(reunitarize_dev(s->U, d + 5, s->part, st));
        LQCD_TRY(read_scalars(d + 5, &maxdev, 1, st));
    }
    LQCD_TRY(plaquette_sum(s->U, d + 6, s->part, st, false));
    double plaq_sum = 0;
    LQCD_TRY(read_scalars(d + 6, &plaq_sum, 1, st));
    if (info) {
        info->dH = dH;
        info->H0 = H0;
        info->H1 = H1;
        info->plaq = plaq_sum / (6.0 * 2.0 * s->U->Vh);
        info->u = u;
        info->max_unitarity_dev = maxdev;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->cg_true_rel_res_max = s->cg_res_max;
        info->accepted = accept ? 1 : 0;
        info->cg_iters = s->cg_iters;
        info->n_solves = s->n_solves;
        info->cg_failures = s->cg_failures;
        info->cg_accurate_residuals = s->cg_accurate;
        info->cg_failed_checks = s->cg_failed_checks;
        info->cg_guesses_refined = s->cg_refined;
        info->traj = s->traj;
    }
    s->traj++;
    if (rc != LQCD_OK) return rc;
    if (!std::isfinite(dH)) {
        set_error("hmc: dH is not finite; trajectory rejected");
        return LQCD_ENUMERIC;
    }
    return LQCD_OK;
}

} // extern "C"

// ================================================================== batched chains

// Streams over which the chains' per-chain kernels (forces, link updates) are
// spread: a small lattice's kernel fills a fraction of the GPU, so the chains
// run side by side.  Created on first use; each chain's kernels stay in order
// on one stream, and the caller's stream waits for all of them.
struct ChainStreams {
    static constexpr int N = 8;
    cudaStream_t st[N] = {};
    cudaEvent_t fork = nullptr, join[N] = {};
    lqcd_status ensure()
    {
        if (fork) return LQCD_OK;
        LQCD_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        for (int k = 0; k < N; k++) {
            LQCD_CUDA(cudaStreamCreateWithFlags(&st[k], cudaStreamNonBlocking));
            LQCD_CUDA(cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming));
        }
        return LQCD_OK;
    }
    ~ChainStreams()
    {
        for (int k = 0; k < N; k++) {
            if (st[k]) cudaStreamDestroy(st[k]);
            if (join[k]) cudaEventDestroy(join[k]);
        }
        if (fork) cudaEventDestroy(fork);
    }
};

struct lqcd_batch {
    std::vector<lqcd_hmc_state *> chains;
    lqcd::BatchSolver bs;
    lqcd::DevBuf scal; // one CgScalars slot per chain
    ChainStreams cs;
    lqcd::ChainMdTables md; // shared launches of the FP32 molecular dynamics
    bool md_shared = false;
};

namespace lqcd {

static lqcd_status check_batch_params(const lqcd_batch *B, const lqcd_hmc_params *p)
{
    LQCD_REQUIRE(p != nullptr, "batch: params is NULL");
    for (size_t i = 0; i < B->chains.size(); i++) {
        LQCD_TRY(check_params(&p[i]));
        LQCD_REQUIRE(p[i].n_flavors == 2, "batch: every chain needs two Wilson flavours");
        LQCD_REQUIRE(p[i].cg.sloppy != LQCD_F64, "batch: the batched solver is the mixed-precision one");
        LQCD_REQUIRE(!hasenbusch(&p[i]) && n_levels(&p[i]) == 1,
                     "batch: chains run one pseudofermion on one time scale (no hasenbusch_kappa, gauge_substeps)");
        LQCD_REQUIRE(p[i].integrator == p[0].integrator && p[i].nsteps == p[0].nsteps && p[i].tau == p[0].tau &&
                         p[i].cg.sloppy == p[0].cg.sloppy && p[i].force_prec == p[0].force_prec,
                     "batch: chains must share integrator, nsteps, tau, solver precision and force precision");
    }
    return LQCD_OK;
}

// every chain's solve of phi for its current links, with shared launches
// (reuse_last: as in hamiltonian())
static lqcd_status batch_solve(lqcd_batch *B, const lqcd_hmc_params *p, cudaStream_t s, bool reuse_last = false)
{
    size_t n = B->chains.size();
    std::vector<CgRun> runs(n);
    std::vector<CgRun *> ptrs;
    std::vector<bool> reused(n, false);
    for (size_t i = 0; i < n; i++) {
        lqcd_hmc_state *st = B->chains[i];
        PfTerm &t = st->pf[PF_MAIN];
        if (reuse_last && reusable(st, t, &p[i])) {
            reused[i] = true;
            st->n_solves++;
            continue;
        }
        CgRun &r = runs[i];
        r.ws = &st->ws, r.x = t.X.f, r.U = st->U, r.Us = sloppy_links(st, &p[i]), r.b = t.phi.f;
        r.b_stamp = t.phi_stamp;
        r.kappa = p[i].kappa;
        r.prm = p[i].cg;
        MreInput mre;
        LQCD_TRY(prepare_guess(st, t, &p[i], s, &r.prm.guess, &mre));
        if (mre.n >= 2 && r.prm.guess) {
            r.n_mre = std::min(mre.n, CgWorkspace::MRE_MAX + 1);
            for (int j = 0; j < r.n_mre; j++) r.mre_x[j] = mre.x[j];
            r.mre_links = mre.links;
        }
        LQCD_TRY(st->ws.ensure(st->U->lat, r.prm.sloppy, s));
        r.start(s, (CgScalars *)B->scal.p + i);
        ptrs.push_back(&r);
    }
    LQCD_TRY(B->bs.solve(ptrs, s));
    for (size_t i = 0; i < n; i++) {
        if (reused[i]) continue;
        lqcd_hmc_state *st = B->chains[i];
        const CgRun &r = runs[i];
        LQCD_TRY(record_solution(st, st->pf[PF_MAIN], &p[i], r.status, s));
        LQCD_TRY(count_solve(st, r.status, r.inf));
    }
    return LQCD_OK;
}

// f(i, stream) for every chain i, chain i on chain stream i mod N, all after
// the work already on s and before the work later enqueued on s
template <class F>
static lqcd_status per_chain(lqcd_batch *B, cudaStream_t s, F f)
{
    ChainStreams &cs = B->cs;
    LQCD_TRY(cs.ensure());
    LQCD_CUDA(cudaEventRecord(cs.fork, s));
    const int ns = (int)std::min<size_t>(ChainStreams::N, B->chains.size());
    for (int k = 0; k < ns; k++) LQCD_CUDA(cudaStreamWaitEvent(cs.st[k], cs.fork, 0));
    lqcd_status rc = LQCD_OK;
    for (size_t i = 0; i < B->chains.size() && rc == LQCD_OK; i++) rc = f(i, cs.st[i % ChainStreams::N]);
    for (int k = 0; k < ns; k++) { // joined also after a failure
        LQCD_CUDA(cudaEventRecord(cs.join[k], cs.st[k]));
        LQCD_CUDA(cudaStreamWaitEvent(s, cs.join[k], 0));
    }
    return rc;
}

// the descriptors of the chains' FP32 molecular dynamics (after the refresh,
// which makes every field they name); false if the batch's forces are FP64
static lqcd_status batch_md_tables(lqcd_batch *B, const lqcd_hmc_params *p, cudaStream_t s)
{
    B->md_shared = p[0].force_prec == LQCD_F32;
    if (!B->md_shared) return LQCD_OK;
    std::vector<ChainMd> d;
    for (size_t i = 0; i < B->chains.size(); i++) {
        lqcd_hmc_state *st = B->chains[i];
        LQCD_TRY(ensure_f32_temps(st));
        ChainMd c{};
        c.g = make_geo(st->U->lat);
        c.P = mom_ref(st->P.f);
        c.U = gauge_ref<LQCD_F64>(st->U);
        c.Uf = gauge_ref<LQCD_F32>(st->Uf.f);
        c.us = st->Us.f->data;
        c.Udf = gauge_ref<PREC_DF>(st->Udf.f);
        c.X = spinor_ref<LQCD_F64>(st->pf[PF_MAIN].X.f);
        c.X32 = spinor_ref<LQCD_F32>(st->X32.f);
        c.Ao = spinor_ref<LQCD_F32>(st->Ao32.f);
        c.Ye = spinor_ref<LQCD_F32>(st->Ye32.f);
        c.Bo = spinor_ref<LQCD_F32>(st->Bo32.f);
        c.beta = p[i].beta;
        c.kappa = p[i].kappa;
        c.mk2 = (float)(-p[i].kappa * p[i].kappa);
        d.push_back(c);
    }
    if (B->md.n == (int)d.size() && !std::memcmp(B->md.host.data(), d.data(), d.size() * sizeof(ChainMd)))
        return LQCD_OK; // the same fields and couplings: the tables stand
    return B->md.build(d, s);
}

static lqcd_status batch_kick(lqcd_batch *B, const lqcd_hmc_params *p, double c, cudaStream_t s)
{
    if (B->md_shared) { // one launch per kernel over every chain
        LQCD_TRY(chains_gauge_force(B->md, c, s));
        LQCD_TRY(batch_solve(B, p, s));
        return chains_fermion_force(B->md, c, s);
    }
    LQCD_TRY(per_chain(B, s, [&](size_t i, cudaStream_t cst) {
        lqcd_hmc_state *st = B->chains[i];
        return gauge_force_dev(st->P.f, st->U, st->Uf.f, p[i].beta, c, p[i].force_prec, cst);
    }));
    LQCD_TRY(batch_solve(B, p, s));
    return per_chain(B, s, [&](size_t i, cudaStream_t cst) {
        lqcd_hmc_state *st = B->chains[i];
        return fermion_force(st, &p[i], st->pf[PF_MAIN].X.f, nullptr, p[i].kappa, c, cst);
    });
}

static lqcd_status batch_drift(lqcd_batch *B, const lqcd_hmc_params *p, double c, cudaStream_t s)
{
    if (B->md_shared) {
        for (lqcd_hmc_state *st : B->chains) {
            st->md_time += c; // (no kicks are queued in a batch)
            if (st->Udf.f) st->u_lags = true;
        }
        return chains_link_update(B->md, c, p[0].cg.sloppy, s);
    }
    return per_chain(B, s, [&](size_t i, cudaStream_t cst) { return drift(B->chains[i], &p[i], c, cst); });
}

static lqcd_status batch_integrate(lqcd_batch *B, const lqcd_hmc_params *p, cudaStream_t s)
{
    double dt = p[0].tau / p[0].nsteps;
    int n = p[0].nsteps;
    if (p[0].integrator == LQCD_LEAPFROG) {
        LQCD_TRY(batch_kick(B, p, 0.5 * dt, s));
        for (int k = 0; k < n; k++) {
            LQCD_TRY(batch_drift(B, p, dt, s));
            LQCD_TRY(batch_kick(B, p, k == n - 1 ? 0.5 * dt : dt, s));
        }
    } else {
        const double lam = OMELYAN_LAMBDA;
        LQCD_TRY(batch_kick(B, p, lam * dt, s));
        for (int k = 0; k < n; k++) {
            LQCD_TRY(batch_drift(B, p, 0.5 * dt, s));
            LQCD_TRY(batch_kick(B, p, (1.0 - 2.0 * lam) * dt, s));
            LQCD_TRY(batch_drift(B, p, 0.5 * dt, s));
            LQCD_TRY(batch_kick(B, p, k == n - 1 ? lam * dt : 2.0 * lam * dt, s));
        }
    }
    return LQCD_OK;
}

} // namespace lqcd

extern "C" {

lqcd_status lqcd_batch_create(lqcd_hmc_state *const *chains, int n, lqcd_batch **out)
{
    LQCD_REQUIRE(chains && out && n > 0, "batch_create: needs at least one chain");
    for (int i = 0; i < n; i++) {
        LQCD_REQUIRE(chains[i], "batch_create: chain %d is NULL", i);
        for (int j = 0; j < i; j++) LQCD_REQUIRE(chains[i] != chains[j], "batch_create: chain %d repeated", i);
    }
    lqcd_batch *B = new lqcd_batch();
    B->chains.assign(chains, chains + n);
    lqcd_status rc = B->scal.alloc(sizeof(CgScalars) * n, nullptr);
    if (rc != LQCD_OK) {
        delete B;
        return rc;
    }
    *out = B;
    return LQCD_OK;
}

lqcd_status lqcd_batch_destroy(lqcd_batch *B)
{
    cudaDeviceSynchronize();
    delete B;
    return LQCD_OK;
}

lqcd_status lqcd_batch_trajectory(lqcd_batch *B, const lqcd_hmc_params *params, lqcd_traj_info *info, void *stream)
{
    LQCD_REQUIRE(B, "batch_trajectory: NULL batch");
    LQCD_TRY(check_batch_params(B, params));
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    size_t n = B->chains.size();
    std::vector<double> H0(n, 0.0), H1(n, 0.0);
    for (size_t i = 0; i < n; i++) {
        lqcd_hmc_state *st = B->chains[i];
        reset_stats(st);
        LQCD_CUDA(cudaMemcpyAsync(st->Ubak.f->data, st->U->data, st->U->bytes, cudaMemcpyDeviceToDevice, s));
        LQCD_TRY(refresh(st, &params[i], &H0[i], s));
    }
    LQCD_TRY(batch_md_tables(B, params, s));
    lqcd_status rc = batch_integrate(B, params, s);
    for (lqcd_hmc_state *st : B->chains) { // the FP64 links from the float-float copies
        const lqcd_status rs = sync_master_links(st, s);
        if (rc == LQCD_OK) rc = rs;
    }
    if (rc == LQCD_OK) {
        for (size_t i = 0; i < n; i++) LQCD_TRY(hamiltonian_parts(B->chains[i], &params[i], s));
        rc = batch_solve(B, params, s, true);
    }
    for (size_t i = 0; i < n; i++) {
        lqcd_hmc_state *st = B->chains[i];
        const lqcd_hmc_params *p = &params[i];
        double *d = (double *)st->scal.p;
        double h[3] = {0, 0, 0};
        if (rc == LQCD_OK) {
            // kinetic and plaquette sums were taken before the batched solve; add phi^dag X
            LQCD_TRY(spinor_dot_dev(st->pf[PF_MAIN].phi.f, st->pf[PF_MAIN].X.f, d + 2, st->part, s));
            LQCD_TRY(read_scalars(d, h, 3, s));
            H1[i] = hamiltonian_from(st, p, h);
        }
        double dH = H1[i] - H0[i];
        metropolis_uniform_kernel<<<1, 1, 0, s>>>(d + 4, st->seed, st->chain, st->traj);
        LQCD_LAUNCHED();
        double u = 0;
        LQCD_TRY(read_scalars(d + 4, &u, 1, s));
        bool accept = rc == LQCD_OK && std::isfinite(dH) && (!p->metropolis || u < std::exp(-dH));
        if (!accept)
            LQCD_CUDA(cudaMemcpyAsync(st->U->data, st->Ubak.f->data, st->U->bytes, cudaMemcpyDeviceToDevice, s));
        double maxdev = 0;
        if (p->reunitarize) {
            LQCD_TRY(reunitarize_dev(st->U, d + 5, st->part, s));
            LQCD_TRY(read_scalars(d + 5, &maxdev, 1, s));
        }
        LQCD_TRY(plaquette_sum(st->U, d + 6, st->part, s, false));
        double plaq_sum = 0;
        LQCD_TRY(read_scalars(d + 6, &plaq_sum, 1, s));
        if (info) {
            lqcd_traj_info &f = info[i];
            f.dH = dH;
            f.H0 = H0[i];
            f.H1 = H1[i];
            f.plaq = plaq_sum / (6.0 * 2.0 * st->U->Vh);
            f.u = u;
            f.max_unitarity_dev = maxdev;
            f.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            f.cg_true_rel_res_max = st->cg_res_max;
            f.accepted = accept ? 1 : 0;
            f.cg_iters = st->cg_iters;
            f.n_solves = st->n_solves;
            f.cg_failures = st->cg_failures;
            f.cg_accurate_residuals = st->cg_accurate;
            f.cg_failed_checks = st->cg_failed_checks;
            f.cg_guesses_refined = st->cg_refined;
            f.traj = st->traj;
        }
        st->traj++;
    }
    return rc;
}

} // extern "C"
