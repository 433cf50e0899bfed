// hmc.cu -- Hybrid Monte Carlo driver: refresh, molecular dynamics with merged
// kicks (leapfrog or Omelyan 2MN), Hamiltonian, Metropolis and
// reunitarization, every field operation on the device (paper Sec. 1: the
// whole trajectory runs on the accelerator; Sec. 6.2: Nf = 2 Wilson HMC).
//
// The host only sequences kernels and reads back the scalars it must decide
// on (solver convergence, dH and the Metropolis uniform, the plaquette).
#include <chrono>
#include <cmath>

#include "batch.cuh"
#include "cg.cuh"
#include "su3_device.cuh"

namespace lqcd {

// defined in field.cu / force.cu
lqcd_status plaquette_sum(const lqcd_field *U, double *dst_dev, DevBuf &part, cudaStream_t s);
lqcd_status kinetic_sum(const lqcd_field *P, double *dst_dev, DevBuf &part, cudaStream_t s);
lqcd_status reunitarize_dev(lqcd_field *U, double *dst_dev, DevBuf &part, cudaStream_t s);
lqcd_status link_update_dev(lqcd_field *U, const lqcd_field *P, double c, lqcd_field *Us, lqcd_field *Uf, bool fast,
                            cudaStream_t s, lqcd_field *Udf);
lqcd_status momentum_refresh_dev(lqcd_field *P, uint32_t seed, uint32_t chain, uint32_t traj, cudaStream_t s);
lqcd_status eta_refresh_dev(lqcd_field *E, uint32_t seed, uint32_t chain, uint32_t traj, cudaStream_t s);
lqcd_status gauge_force_dev(lqcd_field *P, const lqcd_field *U, const lqcd_field *Uf, double beta, double coeff,
                            lqcd_prec arith, cudaStream_t s);
lqcd_status fermion_force_dev(lqcd_field *P, const lqcd_field *U, const lqcd_field *Uf, const lqcd_field *X,
                              double kappa, double coeff, lqcd_field *Ao, lqcd_field *Ye, lqcd_field *Bo, lqcd_field *Xc,
                              cudaStream_t s);

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

struct lqcd_hmc_state {
    lqcd_field *U = nullptr; // borrowed
    uint32_t seed = 0, chain = 0, traj = 0;
    FieldPtr P, eta, phi, X, Ao, Ye, Bo, Ubak, Us;
    FieldPtr Ao32, Ye32, Bo32, X32; // FP32 fermion-force temporaries (allocated on first use)
    FieldPtr Uf;                    // FP32 12-real link copy for the FP32 molecular dynamics
    FieldPtr Udf; // float-float link copy of the mixed solver, kept current by every link update
    CgWorkspace ws;
    DevBuf part, scal;
    double H0 = 0;
    bool have_guess = false; // X holds a solution for the current phi
    // solutions of this trajectory's solves and the molecular-dynamics times
    // (sum of the drifts since the refresh) of their links, for the
    // extrapolated initial guess; hist[(head - 1) mod CHRONO_MAX] is the latest
    double md_time = 0;
    bool last_ok = false; // the last solve converged, at molecular-dynamics time last_t
    double last_t = -1;
    FieldPtr hist[CHRONO_MAX];
    double hist_t[CHRONO_MAX] = {0, 0, 0, 0};
    int n_hist = 0, head = 0;
    // statistics of the current trajectory
    int cg_iters = 0, n_solves = 0, cg_failures = 0;
    double cg_res_max = 0;
};

namespace lqcd {

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
    }
    LQCD_REQUIRE(p->force_prec == LQCD_F64 || p->force_prec == LQCD_F32, "hmc: force_prec must be F64 or F32");
    LQCD_REQUIRE(p->chrono >= 0 && p->chrono <= CHRONO_MAX, "hmc: chrono must lie in 0..%d", CHRONO_MAX);
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

static lqcd_field *sloppy_links(lqcd_hmc_state *st, const lqcd_hmc_params *p)
{
    return (p->n_flavors == 2 && p->cg.sloppy != LQCD_F64) ? st->Us.f : nullptr;
}

// The initial guess of the next solve, in X; returns whether there is one.
// chrono 1: the previous solution (already in X).  chrono k >= 2: the
// polynomial through the last k solutions at their molecular-dynamics times,
// evaluated at the current time (Lagrange form); the trajectory's solves come
// at evenly spaced times, so this is the extrapolation x_n ~ 2 x_{n-1} -
// x_{n-2} (k = 2), 3 x_{n-1} - 3 x_{n-2} + x_{n-3} (k = 3), ...  A solve at the
// time of the previous one (the action at the end of the trajectory) starts
// from the previous solution.
static lqcd_status prepare_guess(lqcd_hmc_state *st, const lqcd_hmc_params *p, cudaStream_t s, int *guess)
{
    *guess = (p->chrono && st->have_guess) ? 1 : 0;
    if (!*guess || p->chrono < 2 || st->n_hist < 2) return LQCD_OK;
    const int latest = (st->head + CHRONO_MAX - 1) % CHRONO_MAX;
    if (st->hist_t[latest] == st->md_time) return LQCD_OK;
    int idx[CHRONO_MAX], m = 0;
    const int kmax = std::min(p->chrono, CHRONO_MAX);
    for (int k = 0; k < st->n_hist && m < kmax; k++) {
        int i = (st->head + CHRONO_MAX - 1 - k) % CHRONO_MAX;
        bool dup = false;
        for (int j = 0; j < m; j++) dup = dup || st->hist_t[idx[j]] == st->hist_t[i];
        if (!dup) idx[m++] = i;
    }
    if (m < 2) return LQCD_OK;
    double w[CHRONO_MAX] = {0, 0, 0, 0};
    const double2 *x[CHRONO_MAX] = {nullptr, nullptr, nullptr, nullptr};
    for (int a = 0; a < m; a++) {
        double l = 1.0;
        for (int b = 0; b < m; b++)
            if (b != a)
                l *= (st->md_time - st->hist_t[idx[b]]) / (st->hist_t[idx[a]] - st->hist_t[idx[b]]);
        w[a] = l;
        x[a] = (const double2 *)st->hist[idx[a]].f->data;
    }
    size_t n = st->X.f->bytes / sizeof(double2);
    combine_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((double2 *)st->X.f->data, x[0], x[1], x[2], x[3],
                                                               w[0], w[1], w[2], w[3], m, n);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

// record a solve's solution for later guesses
static lqcd_status record_solution(lqcd_hmc_state *st, const lqcd_hmc_params *p, bool ok, cudaStream_t s)
{
    st->have_guess = ok;
    if (!ok || p->chrono < 2) return LQCD_OK;
    lqcd_field *&slot = st->hist[st->head].f;
    if (!slot) LQCD_TRY(lqcd_field_alloc(&st->U->lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &slot));
    LQCD_CUDA(cudaMemcpyAsync(slot->data, st->X.f->data, st->X.f->bytes, cudaMemcpyDeviceToDevice, s));
    st->hist_t[st->head] = st->md_time;
    st->head = (st->head + 1) % CHRONO_MAX;
    st->n_hist = std::min(st->n_hist + 1, CHRONO_MAX);
    return LQCD_OK;
}

static lqcd_status solve(lqcd_hmc_state *st, const lqcd_hmc_params *p, cudaStream_t s)
{
    lqcd_cg_info info{};
    lqcd_cg_params cg = p->cg;
    LQCD_TRY(prepare_guess(st, p, s, &cg.guess));
    lqcd_status rc = cg_solve_ws(st->ws, st->X.f, st->U, sloppy_links(st, p), st->phi.f, p->kappa, cg, &info, s);
    st->last_ok = rc == LQCD_OK;
    st->last_t = st->md_time;
    LQCD_TRY(record_solution(st, p, rc == LQCD_OK || rc == LQCD_ENOCONV, s));
    st->cg_iters += info.iters;
    st->n_solves++;
    st->cg_res_max = std::max(st->cg_res_max, info.true_rel_res);
    if (rc == LQCD_ENOCONV) {
        st->cg_failures++;
        return LQCD_OK; // the trajectory goes on; the failure is reported in its info
    }
    return rc;
}

static lqcd_status ensure_f32_temps(lqcd_hmc_state *st)
{
    if (st->Ao32.f) return LQCD_OK;
    const lqcd_lattice &lat = st->U->lat;
    LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_ODD, LQCD_F32, 0, &st->Ao32.f));
    LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F32, 0, &st->Ye32.f));
    LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_ODD, LQCD_F32, 0, &st->Bo32.f));
    LQCD_TRY(lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F32, 0, &st->X32.f));
    return LQCD_OK;
}

// P <- P - c F(U)
static lqcd_status kick(lqcd_hmc_state *st, const lqcd_hmc_params *p, double c, cudaStream_t s)
{
    LQCD_TRY(gauge_force_dev(st->P.f, st->U, st->Uf.f, p->beta, c, p->force_prec, s));
    if (p->n_flavors == 2) {
        LQCD_TRY(solve(st, p, s));
        if (p->force_prec == LQCD_F32) {
            LQCD_TRY(ensure_f32_temps(st));
            LQCD_TRY(fermion_force_dev(st->P.f, st->U, st->Uf.f, st->X.f, p->kappa, c, st->Ao32.f, st->Ye32.f,
                                       st->Bo32.f, st->X32.f, s));
        } else {
            LQCD_TRY(fermion_force_dev(st->P.f, st->U, nullptr, st->X.f, p->kappa, c, st->Ao.f, st->Ye.f, st->Bo.f,
                                       nullptr, s));
        }
    }
    return LQCD_OK;
}

static lqcd_status drift(lqcd_hmc_state *st, const lqcd_hmc_params *p, double c, cudaStream_t s)
{
    bool fast = p->force_prec == LQCD_F32;
    st->md_time += c;
    return link_update_dev(st->U, st->P.f, c, sloppy_links(st, p), fast ? st->Uf.f : nullptr, fast, s,
                           sloppy_links(st, p) ? st->Udf.f : nullptr);
}

// scalars[0] = plaquette sum, [1] = sum p^2, [2] = fermion term
static lqcd_status hamiltonian_parts(lqcd_hmc_state *st, cudaStream_t s)
{
    double *d = (double *)st->scal.p;
    LQCD_TRY(plaquette_sum(st->U, d + 0, st->part, s));
    LQCD_TRY(kinetic_sum(st->P.f, d + 1, st->part, s));
    return LQCD_OK;
}

static double hamiltonian_from(const lqcd_hmc_state *st, const lqcd_hmc_params *p, const double *h)
{
    double V = 2.0 * st->U->Vh;
    return 0.5 * h[1] + p->beta * (6.0 * V - h[0]) + (p->n_flavors == 2 ? h[2] : 0.0);
}

static lqcd_status refresh(lqcd_hmc_state *st, const lqcd_hmc_params *p, double *H0, cudaStream_t s)
{
    st->have_guess = false; // a new phi: the last solution is no guess for it
    st->n_hist = 0;
    st->md_time = 0;
    LQCD_TRY(ensure_sloppy(st, p, s));
    LQCD_TRY(momentum_refresh_dev(st->P.f, st->seed, st->chain, st->traj, s));
    double *d = (double *)st->scal.p;
    LQCD_TRY(hamiltonian_parts(st, s));
    if (p->n_flavors == 2) {
        LQCD_TRY(eta_refresh_dev(st->eta.f, st->seed, st->chain, st->traj, s));
        LQCD_TRY(mhat_apply(st->phi.f, st->U, st->eta.f, p->kappa, 1, st->Ao.f, nullptr, s));
        LQCD_TRY(spinor_dot_dev(st->eta.f, st->eta.f, d + 2, st->part, s));
    }
    double h[3] = {0, 0, 0};
    LQCD_TRY(read_scalars(d, h, 3, s));
    st->H0 = hamiltonian_from(st, p, h);
    if (H0) *H0 = st->H0;
    return LQCD_OK;
}

// H of the current fields.  reuse_last (inside a trajectory, right after the
// last kick): the last solve was of the same system and converged, and with a
// chronological guess a new solve would start from its solution and stop at
// once, so its solution is used as it is (counted as a solve of 0 iterations).
static lqcd_status hamiltonian(lqcd_hmc_state *st, const lqcd_hmc_params *p, double *H, cudaStream_t s,
                               bool reuse_last = false)
{
    double *d = (double *)st->scal.p;
    LQCD_TRY(hamiltonian_parts(st, s));
    if (p->n_flavors == 2) {
        if (reuse_last && p->chrono && st->have_guess && st->last_ok && st->last_t == st->md_time)
            st->n_solves++;
        else
            LQCD_TRY(solve(st, p, s));
        LQCD_TRY(spinor_dot_dev(st->phi.f, st->X.f, d + 2, st->part, s));
    }
    double h[3] = {0, 0, 0};
    LQCD_TRY(read_scalars(d, h, 3, s));
    *H = hamiltonian_from(st, p, h);
    return LQCD_OK;
}

static lqcd_status integrate(lqcd_hmc_state *st, const lqcd_hmc_params *p, cudaStream_t s)
{
    double dt = p->tau / p->nsteps;
    int n = p->nsteps;
    if (p->integrator == LQCD_LEAPFROG) {
        LQCD_TRY(kick(st, p, 0.5 * dt, s));
        for (int k = 0; k < n; k++) {
            LQCD_TRY(drift(st, p, dt, s));
            LQCD_TRY(kick(st, p, k == n - 1 ? 0.5 * dt : dt, s));
        }
    } else {
        const double lam = OMELYAN_LAMBDA;
        LQCD_TRY(kick(st, p, lam * dt, s));
        for (int k = 0; k < n; k++) {
            LQCD_TRY(drift(st, p, 0.5 * dt, s));
            LQCD_TRY(kick(st, p, (1.0 - 2.0 * lam) * dt, s));
            LQCD_TRY(drift(st, p, 0.5 * dt, s));
            LQCD_TRY(kick(st, p, k == n - 1 ? lam * dt : 2.0 * lam * dt, s));
        }
    }
    return LQCD_OK;
}

static void reset_stats(lqcd_hmc_state *st)
{
    st->cg_iters = st->n_solves = st->cg_failures = 0;
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
    if (rc == LQCD_OK) rc = lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &st->phi.f);
    if (rc == LQCD_OK) rc = lqcd_field_alloc(&lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &st->X.f);
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
    if (phi) *phi = s->phi.f;
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
    LQCD_TRY(ensure_sloppy(s, p, (cudaStream_t)stream));
    return hamiltonian(s, p, H, (cudaStream_t)stream);
}

lqcd_status lqcd_md_step(lqcd_hmc_state *s, const lqcd_hmc_params *p, void *stream)
{
    LQCD_REQUIRE(s, "md_step: NULL state");
    LQCD_TRY(check_params(p));
    cudaStream_t st = (cudaStream_t)stream;
    LQCD_TRY(ensure_sloppy(s, p, st));
    double dt = p->tau / p->nsteps;
    if (p->integrator == LQCD_LEAPFROG) {
        LQCD_TRY(kick(s, p, 0.5 * dt, st));
        LQCD_TRY(drift(s, p, dt, st));
        LQCD_TRY(kick(s, p, 0.5 * dt, st));
    } else {
        const double lam = OMELYAN_LAMBDA;
        LQCD_TRY(kick(s, p, lam * dt, st));
        LQCD_TRY(drift(s, p, 0.5 * dt, st));
        LQCD_TRY(kick(s, p, (1.0 - 2.0 * lam) * dt, st));
        LQCD_TRY(drift(s, p, 0.5 * dt, st));
        LQCD_TRY(kick(s, p, lam * dt, st));
    }
    return LQCD_OK;
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
    if (rc == LQCD_OK) rc = integrate(s, p, st);
    if (rc == LQCD_OK) rc = hamiltonian(s, p, &H1, st, true);
    double dH = H1 - H0;
    double *d = (double *)s->scal.p;
    metropolis_uniform_kernel<<<1, 1, 0, st>>>(d + 3, s->seed, s->chain, s->traj);
    LQCD_LAUNCHED();
    double u = 0;
    LQCD_TRY(read_scalars(d + 3, &u, 1, st));
    bool accept = rc == LQCD_OK && std::isfinite(dH) && (!p->metropolis || u < std::exp(-dH));
    if (!accept) LQCD_CUDA(cudaMemcpyAsync(s->U->data, s->Ubak.f->data, s->U->bytes, cudaMemcpyDeviceToDevice, st));
    double maxdev = 0;
    if (p->reunitarize) {
        LQCD_TRY(reunitarize_dev(s->U, d + 4, s->part, st));
        LQCD_TRY(read_scalars(d + 4, &maxdev, 1, st));
    }
    LQCD_TRY(plaquette_sum(s->U, d + 5, s->part, st));
    double plaq_sum = 0;
    LQCD_TRY(read_scalars(d + 5, &plaq_sum, 1, st));
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

struct lqcd_batch {
    std::vector<lqcd_hmc_state *> chains;
    lqcd::BatchSolver bs;
    lqcd::DevBuf scal; // one CgScalars slot per chain
};

namespace lqcd {

static lqcd_status check_batch_params(const lqcd_batch *B, const lqcd_hmc_params *p)
{
    LQCD_REQUIRE(p != nullptr, "batch: params is NULL");
    for (size_t i = 0; i < B->chains.size(); i++) {
        LQCD_TRY(check_params(&p[i]));
        LQCD_REQUIRE(p[i].n_flavors == 2, "batch: every chain needs two Wilson flavours");
        LQCD_REQUIRE(p[i].cg.sloppy != LQCD_F64, "batch: the batched solver is the mixed-precision one");
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
        if (reuse_last && p[i].chrono && st->have_guess && st->last_ok && st->last_t == st->md_time) {
            reused[i] = true;
            st->n_solves++;
            continue;
        }
        CgRun &r = runs[i];
        r.ws = &st->ws, r.x = st->X.f, r.U = st->U, r.Us = sloppy_links(st, &p[i]), r.b = st->phi.f;
        r.kappa = p[i].kappa;
        r.prm = p[i].cg;
        LQCD_TRY(prepare_guess(st, &p[i], s, &r.prm.guess));
        LQCD_TRY(st->ws.ensure(st->U->lat, r.prm.sloppy, s));
        r.start(s, (CgScalars *)B->scal.p + i);
        ptrs.push_back(&r);
    }
    LQCD_TRY(B->bs.solve(ptrs, s));
    for (size_t i = 0; i < n; i++) {
        if (reused[i]) continue;
        lqcd_hmc_state *st = B->chains[i];
        const CgRun &r = runs[i];
        st->last_ok = r.status == LQCD_OK;
        st->last_t = st->md_time;
        st->cg_iters += r.inf.iters;
        st->n_solves++;
        st->cg_res_max = std::max(st->cg_res_max, r.inf.true_rel_res);
        LQCD_TRY(record_solution(st, &p[i], r.status == LQCD_OK || r.status == LQCD_ENOCONV, s));
        if (r.status == LQCD_ENOCONV)
            st->cg_failures++;
        else if (r.status != LQCD_OK)
            return r.status;
    }
    return LQCD_OK;
}

static lqcd_status batch_kick(lqcd_batch *B, const lqcd_hmc_params *p, double c, cudaStream_t s)
{
    size_t n = B->chains.size();
    for (size_t i = 0; i < n; i++) {
        lqcd_hmc_state *st = B->chains[i];
        LQCD_TRY(gauge_force_dev(st->P.f, st->U, st->Uf.f, p[i].beta, c, p[i].force_prec, s));
    }
    LQCD_TRY(batch_solve(B, p, s));
    for (size_t i = 0; i < n; i++) {
        lqcd_hmc_state *st = B->chains[i];
        if (p[i].force_prec == LQCD_F32) {
            LQCD_TRY(ensure_f32_temps(st));
            LQCD_TRY(fermion_force_dev(st->P.f, st->U, st->Uf.f, st->X.f, p[i].kappa, c, st->Ao32.f, st->Ye32.f,
                                       st->Bo32.f, st->X32.f, s));
        } else {
            LQCD_TRY(fermion_force_dev(st->P.f, st->U, nullptr, st->X.f, p[i].kappa, c, st->Ao.f, st->Ye.f,
                                       st->Bo.f, nullptr, s));
        }
    }
    return LQCD_OK;
}

static lqcd_status batch_drift(lqcd_batch *B, const lqcd_hmc_params *p, double c, cudaStream_t s)
{
    for (size_t i = 0; i < B->chains.size(); i++) LQCD_TRY(drift(B->chains[i], &p[i], c, s));
    return LQCD_OK;
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
    lqcd_status rc = batch_integrate(B, params, s);
    if (rc == LQCD_OK) {
        for (size_t i = 0; i < n; i++) LQCD_TRY(hamiltonian_parts(B->chains[i], s));
        rc = batch_solve(B, params, s, true);
    }
    for (size_t i = 0; i < n; i++) {
        lqcd_hmc_state *st = B->chains[i];
        const lqcd_hmc_params *p = &params[i];
        double *d = (double *)st->scal.p;
        double h[3] = {0, 0, 0};
        if (rc == LQCD_OK) {
            // kinetic and plaquette sums were taken before the batched solve; add phi^dag X
            LQCD_TRY(spinor_dot_dev(st->phi.f, st->X.f, d + 2, st->part, s));
            LQCD_TRY(read_scalars(d, h, 3, s));
            H1[i] = hamiltonian_from(st, p, h);
        }
        double dH = H1[i] - H0[i];
        metropolis_uniform_kernel<<<1, 1, 0, s>>>(d + 3, st->seed, st->chain, st->traj);
        LQCD_LAUNCHED();
        double u = 0;
        LQCD_TRY(read_scalars(d + 3, &u, 1, s));
        bool accept = rc == LQCD_OK && std::isfinite(dH) && (!p->metropolis || u < std::exp(-dH));
        if (!accept)
            LQCD_CUDA(cudaMemcpyAsync(st->U->data, st->Ubak.f->data, st->U->bytes, cudaMemcpyDeviceToDevice, s));
        double maxdev = 0;
        if (p->reunitarize) {
            LQCD_TRY(reunitarize_dev(st->U, d + 4, st->part, s));
            LQCD_TRY(read_scalars(d + 4, &maxdev, 1, s));
        }
        LQCD_TRY(plaquette_sum(st->U, d + 5, st->part, s));
        double plaq_sum = 0;
        LQCD_TRY(read_scalars(d + 5, &plaq_sum, 1, s));
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
            f.traj = st->traj;
        }
        st->traj++;
    }
    return rc;
}

} // extern "C"
