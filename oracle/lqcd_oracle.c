/*
 * lqcd_oracle.c -- plain, slow, FP64 CPU oracle for one Hybrid Monte Carlo
 * trajectory of SU(3) lattice gauge theory with two flavours of Wilson fermions.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  It shares nothing with the
 * CUDA library: no headers, no helpers, no tables.
 *
 * The paper (Winter, "Gauge Field Generation on Large-Scale GPU-Enabled
 * Systems", Lattice 2012) names the operations of an HMC trajectory that must run
 * on the accelerator (Sec. 1: pseudofermion refresh, momentum updates, force
 * terms, projection of fields, reunitarization, random numbers, SU(3)
 * exponentiation) and the global reductions `sum`/`sumMulti` (Sec. 1), and it
 * ran Nf=2 Wilson fermions (Sec. 6.2).  It prints no formula for any of them, so
 * every formula below is the textbook reading, written out as plainly as
 * possible:
 *   - Wilson operator M = 1 - kappa*D, D the nearest-neighbour hopping term with
 *     (1 - gamma_mu) on forward hops, DeGrand-Rossi gamma basis, fermion fields
 *     antiperiodic in time; even-odd Schur complement Mhat = 1 - kappa^2 Deo Doe.
 *   - Wilson plaquette gauge action S_g = beta sum_P (1 - Re Tr U_P / 3).
 *   - Two-flavour pseudofermion action S_f = phi^dag (Mhat^dag Mhat)^-1 phi.
 *   - Momenta P = sum_a p_a T_a, T_a = lambda_a / 2, kinetic energy 1/2 sum p_a^2.
 *   - Force coefficient f_a = d/de S(exp(i e T_a) U) at e = 0; P <- P - dt f.
 *   - Philox4x32-10 counter-based RNG (Salmon, Moraes, Dror, Shaw, SC'11),
 *     Box-Muller Gaussians.
 *   - Leapfrog and Omelyan 2MN (Omelyan, Mryglod, Folk 2003) integrators.
 *   - exp of a 3x3 matrix by its power series (scaling and squaring).
 *   - Reunitarization by Gram-Schmidt of rows 0, 1 and row2 = conj(row0 x row1).
 *
 * Parity-pinned by the tests under tests/ (free-field spectrum, gamma5
 * hermiticity, gauge covariance, finite-difference forces, cuRAND's host Philox,
 * scipy expm, reversibility, dH ~ dt^2, Creutz equality).
 *
 * Host layouts (canonical AoS, lexicographic site i = x + Lx(y + Ly(z + Lz t))):
 *   gauge    [site][mu][row][col][re,im]    18 doubles per link
 *   spinor   [site][spin][color][re,im]     24 doubles per site (full lattice)
 *   momentum [site][mu][a]                  8 Gell-Mann coefficients per link
 * Even/odd fields are full-lattice arrays whose other-parity sites are ignored
 * on input and written as zero on output.
 *
 * Built twice from this one source: plainly (serial), and with -fopenmp, where
 * the pragmas split the loops over sites whose iterations write disjoint
 * outputs (hopping term, forces, link update, refresh, start configuration,
 * reunitarization with its exact max) across threads.  Every sum (dot
 * products, plaquette, kinetic energy) stays a serial loop in site order, so
 * both builds give bitwise the same results.
 *
 * Build with -ffp-contract=off so the same source rounds identically on every host.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ geometry */

typedef struct {
    int L[4];
    long V;
    double t_bc; /* +1 periodic, -1 antiperiodic fermion boundary in t */
    double xi0;  /* bare gauge anisotropy: plaquettes in a plane with t weigh xi0, spatial ones 1/xi0 */
    double cs;   /* weight of the spatial hops of the Wilson operator, nu / xi0 (t hops weigh 1) */
} geom;

/* Anisotropy of every later call (the paper's runs use the anisotropic
 * Wilson gauge and fermion actions, Fig. 3): 1, 1 is the isotropic action. */
static double g_xi0 = 1.0, g_nu = 1.0;

void or_set_anisotropy(double xi0, double nu)
{
    g_xi0 = xi0;
    g_nu = nu;
}

static int geom_init(geom *g, const int *dims, int t_bc)
{
    g->xi0 = g_xi0;
    g->cs = g_nu / g_xi0;
    g->V = 1;
    for (int mu = 0; mu < 4; mu++) {
        if (dims[mu] <= 0 || dims[mu] % 2 != 0) return -1;
        g->L[mu] = dims[mu];
        g->V *= dims[mu];
    }
    if (t_bc != 1 && t_bc != -1) return -1;
    g->t_bc = (double)t_bc;
    return 0;
}

static void site_coords(const geom *g, long i, int c[4])
{
    for (int mu = 0; mu < 4; mu++) {
        c[mu] = (int)(i % g->L[mu]);
        i /= g->L[mu];
    }
}

static long site_index(const geom *g, const int c[4])
{
    return c[0] + (long)g->L[0] * (c[1] + (long)g->L[1] * (c[2] + (long)g->L[2] * c[3]));
}

static int site_parity(const geom *g, long i)
{
    int c[4];
    site_coords(g, i, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* Neighbour one step along mu (sign +1 forward, -1 backward).  *phase is the
 * fermion boundary factor of that hop: t_bc when the hop wraps in t, else 1. */
static long hop(const geom *g, long i, int mu, int sign, double *phase)
{
    int c[4];
    site_coords(g, i, c);
    c[mu] += sign;
    *phase = 1.0;
    if (c[mu] == g->L[mu]) {
        c[mu] = 0;
        if (mu == 3) *phase = g->t_bc;
    } else if (c[mu] < 0) {
        c[mu] = g->L[mu] - 1;
        if (mu == 3) *phase = g->t_bc;
    }
    return site_index(g, c);
}

/* ------------------------------------------------------- 3x3 complex matrices */

typedef struct { cplx m[3][3]; } mat3;

static mat3 link_get(const double *U, long i, int mu)
{
    mat3 r;
    const double *p = U + (i * 4 + mu) * 18;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            r.m[a][b] = p[(a * 3 + b) * 2] + I * p[(a * 3 + b) * 2 + 1];
    return r;
}

static void link_set(double *U, long i, int mu, const mat3 *x)
{
    double *p = U + (i * 4 + mu) * 18;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            p[(a * 3 + b) * 2] = creal(x->m[a][b]);
            p[(a * 3 + b) * 2 + 1] = cimag(x->m[a][b]);
        }
}

static mat3 mat_zero(void)
{
    mat3 r;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) r.m[a][b] = 0;
    return r;
}

static mat3 mat_id(void)
{
    mat3 r = mat_zero();
    for (int a = 0; a < 3; a++) r.m[a][a] = 1;
    return r;
}

static mat3 mat_mul(const mat3 *x, const mat3 *y)
{
    mat3 r;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            cplx s = 0;
            for (int k = 0; k < 3; k++) s += x->m[a][k] * y->m[k][b];
            r.m[a][b] = s;
        }
    return r;
}

static mat3 mat_dag(const mat3 *x)
{
    mat3 r;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) r.m[a][b] = conj(x->m[b][a]);
    return r;
}

static mat3 mat_add(const mat3 *x, const mat3 *y)
{
    mat3 r;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) r.m[a][b] = x->m[a][b] + y->m[a][b];
    return r;
}

static mat3 mat_sub(const mat3 *x, const mat3 *y)
{
    mat3 r;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) r.m[a][b] = x->m[a][b] - y->m[a][b];
    return r;
}

static mat3 mat_scale(const mat3 *x, cplx s)
{
    mat3 r;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) r.m[a][b] = s * x->m[a][b];
    return r;
}

static cplx mat_trace(const mat3 *x)
{
    return x->m[0][0] + x->m[1][1] + x->m[2][2];
}

/* Gell-Mann generators T_a = lambda_a / 2, a = 0..7 for lambda_1..lambda_8. */
static mat3 gen_T(int a)
{
    mat3 t = mat_zero();
    switch (a) {
    case 0: t.m[0][1] = 1; t.m[1][0] = 1; break;
    case 1: t.m[0][1] = -I; t.m[1][0] = I; break;
    case 2: t.m[0][0] = 1; t.m[1][1] = -1; break;
    case 3: t.m[0][2] = 1; t.m[2][0] = 1; break;
    case 4: t.m[0][2] = -I; t.m[2][0] = I; break;
    case 5: t.m[1][2] = 1; t.m[2][1] = 1; break;
    case 6: t.m[1][2] = -I; t.m[2][1] = I; break;
    case 7:
        t.m[0][0] = 1 / sqrt(3.0);
        t.m[1][1] = 1 / sqrt(3.0);
        t.m[2][2] = -2 / sqrt(3.0);
        break;
    }
    return mat_scale(&t, 0.5);
}

/* Hermitian traceless matrix sum_a c_a T_a from 8 coefficients. */
static mat3 algebra_to_mat(const double *c)
{
    mat3 r = mat_zero();
    for (int a = 0; a < 8; a++) {
        mat3 t = gen_T(a);
        mat3 s = mat_scale(&t, c[a]);
        r = mat_add(&r, &s);
    }
    return r;
}

/* exp(X) of a 3x3 complex matrix: the power series, with scaling and squaring
 * so that the series is summed for |X / 2^k| <= 1/4 (30 terms, far beyond
 * double precision there). */
static mat3 mat_exp(const mat3 *X)
{
    double nrm = 0;
    for (int a = 0; a < 3; a++) {
        double row = 0;
        for (int b = 0; b < 3; b++) row += cabs(X->m[a][b]);
        if (row > nrm) nrm = row;
    }
    int k = 0;
    while (nrm > 0.25) {
        nrm *= 0.5;
        k++;
    }
    mat3 Y = mat_scale(X, ldexp(1.0, -k));
    mat3 E = mat_id(), term = mat_id();
    for (int n = 1; n <= 30; n++) {
        term = mat_mul(&term, &Y);
        term = mat_scale(&term, 1.0 / n);
        E = mat_add(&E, &term);
    }
    for (int s = 0; s < k; s++) E = mat_mul(&E, &E);
    return E;
}

/* exp(i c H) for Hermitian H. */
static mat3 expi_herm(const mat3 *H, double c)
{
    mat3 X = mat_scale(H, I * c);
    return mat_exp(&X);
}

/* Traceless anti-Hermitian part as used by the forces:
 * TA(W) = (W - W^dag) - Tr(W - W^dag)/3 * 1. */
static mat3 proj_ta(const mat3 *W)
{
    mat3 Wd = mat_dag(W);
    mat3 A = mat_sub(W, &Wd);
    cplx tr = mat_trace(&A) / 3.0;
    for (int a = 0; a < 3; a++) A.m[a][a] -= tr;
    return A;
}

/* Coefficients f_a = 2 Re Tr(T_a F) of a Hermitian traceless F = sum_a f_a T_a. */
static void mat_to_algebra(const mat3 *F, double *f)
{
    for (int a = 0; a < 8; a++) {
        mat3 t = gen_T(a);
        mat3 tf = mat_mul(&t, F);
        f[a] = 2.0 * creal(mat_trace(&tf));
    }
}

/* Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1). */
static mat3 reunit(const mat3 *x)
{
    mat3 r = *x;
    double n0 = 0;
    for (int b = 0; b < 3; b++) n0 += creal(r.m[0][b] * conj(r.m[0][b]));
    n0 = sqrt(n0);
    for (int b = 0; b < 3; b++) r.m[0][b] /= n0;
    cplx ov = 0; /* r0^dag r1 */
    for (int b = 0; b < 3; b++) ov += conj(r.m[0][b]) * r.m[1][b];
    for (int b = 0; b < 3; b++) r.m[1][b] -= ov * r.m[0][b];
    double n1 = 0;
    for (int b = 0; b < 3; b++) n1 += creal(r.m[1][b] * conj(r.m[1][b]));
    n1 = sqrt(n1);
    for (int b = 0; b < 3; b++) r.m[1][b] /= n1;
    r.m[2][0] = conj(r.m[0][1] * r.m[1][2] - r.m[0][2] * r.m[1][1]);
    r.m[2][1] = conj(r.m[0][2] * r.m[1][0] - r.m[0][0] * r.m[1][2]);
    r.m[2][2] = conj(r.m[0][0] * r.m[1][1] - r.m[0][1] * r.m[1][0]);
    return r;
}

/* max_ij |(U U^dag - 1)_ij| */
static double unitarity_dev(const mat3 *x)
{
    mat3 xd = mat_dag(x);
    mat3 p = mat_mul(x, &xd);
    double m = 0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double d = cabs(p.m[a][b] - (a == b ? 1.0 : 0.0));
            if (d > m) m = d;
        }
    return m;
}

/* ------------------------------------------------------------ gamma matrices */

/* DeGrand-Rossi basis; index 0..3 is gamma_1..gamma_4 (x, y, z, t). gamma_5 is
 * computed as the product gamma_1 gamma_2 gamma_3 gamma_4. */
static cplx G[5][4][4];
static int G_ready = 0;

static void gamma_init(void)
{
    if (G_ready) return;
    memset(G, 0, sizeof(G));
    /* gamma_1 */
    G[0][0][3] = I; G[0][1][2] = I; G[0][2][1] = -I; G[0][3][0] = -I;
    /* gamma_2 */
    G[1][0][3] = -1; G[1][1][2] = 1; G[1][2][1] = 1; G[1][3][0] = -1;
    /* gamma_3 */
    G[2][0][2] = I; G[2][1][3] = -I; G[2][2][0] = -I; G[2][3][1] = I;
    /* gamma_4 */
    G[3][0][2] = 1; G[3][1][3] = 1; G[3][2][0] = 1; G[3][3][1] = 1;
    /* gamma_5 = g1 g2 g3 g4 */
    cplx t1[4][4], t2[4][4];
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            cplx s = 0;
            for (int k = 0; k < 4; k++) s += G[0][a][k] * G[1][k][b];
            t1[a][b] = s;
        }
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            cplx s = 0;
            for (int k = 0; k < 4; k++) s += t1[a][k] * G[2][k][b];
            t2[a][b] = s;
        }
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            cplx s = 0;
            for (int k = 0; k < 4; k++) s += t2[a][k] * G[3][k][b];
            G[4][a][b] = s;
        }
    G_ready = 1;
}

/* threads the site loops use: omp_get_max_threads() in the OpenMP build, 1 in
 * the serial one */
#ifdef _OPENMP
#include <omp.h>
int or_num_threads(void) { return omp_get_max_threads(); }
#else
int or_num_threads(void) { return 1; }
#endif

/* Copy of one gamma matrix (0..3 = gamma_1..gamma_4, 4 = gamma_5), row-major
 * [4][4][re,im]. */
void or_gamma(int which, double *out32)
{
    gamma_init();
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            out32[(a * 4 + b) * 2] = creal(G[which][a][b]);
            out32[(a * 4 + b) * 2 + 1] = cimag(G[which][a][b]);
        }
}

/* ------------------------------------------------------------------ spinors */

static cplx *spinor_at(double *psi, long i) { return (cplx *)(psi + i * 24); }
static const cplx *spinor_at_c(const double *psi, long i) { return (const cplx *)(psi + i * 24); }

/* out = gamma_5 in on every site (full lattice) */
static void apply_g5(const geom *g, const double *in, double *out)
{
    gamma_init();
    for (long i = 0; i < g->V; i++) {
        const cplx *s = spinor_at_c(in, i);
        cplx r[12];
        for (int a = 0; a < 4; a++)
            for (int c = 0; c < 3; c++) {
                cplx acc = 0;
                for (int b = 0; b < 4; b++) acc += G[4][a][b] * s[b * 3 + c];
                r[a * 3 + c] = acc;
            }
        memcpy(spinor_at(out, i), r, sizeof(r));
    }
}

/* Hopping term D at one site x (nearest-neighbour Wilson hop):
 *   (D psi)(x) = sum_mu [ s (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                         + s (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
 * with s the fermion boundary factor of the hop. */
static void dslash_site(const geom *g, const double *U, const double *psi, long x, cplx out[12])
{
    gamma_init();
    for (int k = 0; k < 12; k++) out[k] = 0;
    for (int mu = 0; mu < 4; mu++) {
        const double w = mu < 3 ? g->cs : 1.0; /* the hop's weight in the anisotropic operator */
        double s;
        /* forward hop */
        long y = hop(g, x, mu, +1, &s);
        mat3 u = link_get(U, x, mu);
        const cplx *p = spinor_at_c(psi, y);
        cplx v[12]; /* U psi(y), per spin */
        for (int b = 0; b < 4; b++)
            for (int a = 0; a < 3; a++) {
                cplx acc = 0;
                for (int c = 0; c < 3; c++) acc += u.m[a][c] * p[b * 3 + c];
                v[b * 3 + a] = acc;
            }
        for (int al = 0; al < 4; al++)
            for (int a = 0; a < 3; a++) {
                cplx acc = 0;
                for (int be = 0; be < 4; be++) {
                    cplx proj = (al == be ? 1.0 : 0.0) - G[mu][al][be];
                    acc += proj * v[be * 3 + a];
                }
                out[al * 3 + a] += (s * w) * acc;
            }
        /* backward hop */
        y = hop(g, x, mu, -1, &s);
        u = link_get(U, y, mu);
        p = spinor_at_c(psi, y);
        for (int b = 0; b < 4; b++)
            for (int a = 0; a < 3; a++) {
                cplx acc = 0;
                for (int c = 0; c < 3; c++) acc += conj(u.m[c][a]) * p[b * 3 + c];
                v[b * 3 + a] = acc;
            }
        for (int al = 0; al < 4; al++)
            for (int a = 0; a < 3; a++) {
                cplx acc = 0;
                for (int be = 0; be < 4; be++) {
                    cplx proj = (al == be ? 1.0 : 0.0) + G[mu][al][be];
                    acc += proj * v[be * 3 + a];
                }
                out[al * 3 + a] += (s * w) * acc;
            }
    }
}

/* D on sites of parity out_parity (0 even, 1 odd, -1 all); other sites of out
 * are zeroed.  dagger != 0 applies D^dag = gamma_5 D gamma_5. */
static void dslash_full(const geom *g, const double *U, const double *in, double *out, int dagger,
                        int out_parity)
{
    const double *src = in;
    double *tmp = NULL;
    if (dagger) {
        tmp = malloc(sizeof(double) * 24 * g->V);
        apply_g5(g, in, tmp);
        src = tmp;
    }
    gamma_init();
    #pragma omp parallel for schedule(static)
    for (long x = 0; x < g->V; x++) {
        cplx r[12];
        if (out_parity >= 0 && site_parity(g, x) != out_parity) {
            for (int k = 0; k < 12; k++) r[k] = 0;
        } else {
            dslash_site(g, U, src, x, r);
        }
        memcpy(spinor_at(out, x), r, sizeof(r));
    }
    if (dagger) {
        apply_g5(g, out, out);
        free(tmp);
    }
}

/* zero the sites of the other parity */
static void mask_parity(const geom *g, double *psi, int parity)
{
    for (long x = 0; x < g->V; x++)
        if (site_parity(g, x) != parity) memset(psi + x * 24, 0, sizeof(double) * 24);
}

static double dot_re(const geom *g, const double *a, const double *b)
{
    /* Re <a, b> = sum over reals a_k b_k */
    double s = 0;
    for (long k = 0; k < g->V * 24; k++) s += a[k] * b[k];
    return s;
}

/* Mhat x_e = x_e - kappa^2 Deo Doe x_e on the even sites (dagger: the adjoint
 * 1 - kappa^2 Doe^dag Deo^dag, via gamma_5 on both D).  in/out full-lattice
 * arrays, odd sites ignored / zeroed. */
static void mhat(const geom *g, const double *U, double kappa, const double *in, double *out, int dagger)
{
    long n = g->V * 24;
    double *a = malloc(sizeof(double) * n);
    double *t = malloc(sizeof(double) * n);
    double *b = malloc(sizeof(double) * n);
    memcpy(a, in, sizeof(double) * n);
    mask_parity(g, a, 0);
    dslash_full(g, U, a, t, dagger, 1);
    dslash_full(g, U, t, b, dagger, 0);
    for (long k = 0; k < n; k++) out[k] = a[k] - kappa * kappa * b[k];
    mask_parity(g, out, 0);
    free(a);
    free(t);
    free(b);
}

static void mdagm(const geom *g, const double *U, double kappa, const double *in, double *out)
{
    double *t = malloc(sizeof(double) * g->V * 24);
    mhat(g, U, kappa, in, t, 0);
    mhat(g, U, kappa, t, out, 1);
    free(t);
}

/* Conjugate gradient on Mhat^dag Mhat x = b (even sites), x0 = 0.  Stops when
 * the iterated |r|^2 <= tol^2 |b|^2, then recomputes the true residual and
 * restarts from the current x when that fails (at most 3 restarts). */
static int cg_solve(const geom *g, const double *U, double kappa, const double *b, double *x, double tol,
                    int maxiter, int *iters_out, double *true_rel_out)
{
    long n = g->V * 24;
    double *r = malloc(sizeof(double) * n);
    double *p = malloc(sizeof(double) * n);
    double *Ap = malloc(sizeof(double) * n);
    double *bb_ = malloc(sizeof(double) * n);
    memcpy(bb_, b, sizeof(double) * n);
    mask_parity(g, bb_, 0);
    memset(x, 0, sizeof(double) * n);
    double bb = dot_re(g, bb_, bb_);
    int iters = 0, status = 0;
    double true_rel = 0;
    if (bb == 0) {
        *iters_out = 0;
        *true_rel_out = 0;
        free(r); free(p); free(Ap); free(bb_);
        return 0;
    }
    memcpy(r, bb_, sizeof(double) * n);
    for (int restart = 0; restart <= 3; restart++) {
        memcpy(p, r, sizeof(double) * n);
        double rr = dot_re(g, r, r);
        while (iters < maxiter && rr > tol * tol * bb) {
            mdagm(g, U, kappa, p, Ap);
            double pAp = dot_re(g, p, Ap);
            double alpha = rr / pAp;
            for (long k = 0; k < n; k++) x[k] += alpha * p[k];
            for (long k = 0; k < n; k++) r[k] -= alpha * Ap[k];
            double rr_new = dot_re(g, r, r);
            iters++;
            double beta = rr_new / rr;
            rr = rr_new;
            if (rr <= tol * tol * bb) break;
            for (long k = 0; k < n; k++) p[k] = r[k] + beta * p[k];
        }
        /* true residual */
        mdagm(g, U, kappa, x, Ap);
        for (long k = 0; k < n; k++) r[k] = bb_[k] - Ap[k];
        double rt = dot_re(g, r, r);
        true_rel = sqrt(rt / bb);
        if (rt <= tol * tol * bb) break;
        if (iters >= maxiter) {
            status = 1;
            break;
        }
    }
    if (true_rel > tol) status = 1;
    *iters_out = iters;
    *true_rel_out = true_rel;
    free(r); free(p); free(Ap); free(bb_);
    return status;
}

/* -------------------------------------------------------------- gauge action */

/* U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag */
static mat3 plaquette_mat(const geom *g, const double *U, long x, int mu, int nu)
{
    double s;
    long xpm = hop(g, x, mu, +1, &s);
    long xpn = hop(g, x, nu, +1, &s);
    mat3 a = link_get(U, x, mu);
    mat3 b = link_get(U, xpm, nu);
    mat3 c = link_get(U, xpn, mu);
    mat3 d = link_get(U, x, nu);
    mat3 cd = mat_dag(&c), dd = mat_dag(&d);
    mat3 t = mat_mul(&a, &b);
    t = mat_mul(&t, &cd);
    return mat_mul(&t, &dd);
}

/* weight of the plaquettes in plane (mu, nu) in the anisotropic gauge action:
 * xi0 for the planes with t, 1/xi0 for the spatial ones */
static double plane_weight(const geom *g, int mu, int nu)
{
    return (mu == 3 || nu == 3) ? g->xi0 : 1.0 / g->xi0;
}

/* sum_x sum_{mu<nu} w_munu Re Tr U_munu(x) / 3, and the sum of the weights */
static double wplaq_sum(const geom *g, const double *U)
{
    double s = 0;
    for (long x = 0; x < g->V; x++)
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) {
                mat3 p = plaquette_mat(g, U, x, mu, nu);
                s += plane_weight(g, mu, nu) * (creal(mat_trace(&p)) / 3.0);
            }
    return s;
}
static double weight_sum(const geom *g) { return g->V * (3.0 / g->xi0 + 3.0 * g->xi0); }

/* S_g = beta sum_x sum_{mu<nu} w_munu (1 - Re Tr U_munu / 3) */
static double gauge_action(const geom *g, const double *U, double beta)
{
    return beta * (weight_sum(g) - wplaq_sum(g, U));
}

/* sum_x sum_{mu<nu} Re Tr U_munu(x) / 3 */
static double plaq_sum(const geom *g, const double *U)
{
    double s = 0;
    for (long x = 0; x < g->V; x++)
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) {
                mat3 p = plaquette_mat(g, U, x, mu, nu);
                s += creal(mat_trace(&p)) / 3.0;
            }
    return s;
}

/* Staple sum A_mu(x) so that U_mu(x) A_mu(x) is the sum of the 6 plaquettes
 * through the link (x, mu) that start with it, each weighted by its plane's
 * weight in the (anisotropic) gauge action. */
static mat3 staple(const geom *g, const double *U, long x, int mu)
{
    mat3 A = mat_zero();
    double s;
    long xpm = hop(g, x, mu, +1, &s);
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        /* upper: U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag */
        long xpn = hop(g, x, nu, +1, &s);
        mat3 a = link_get(U, xpm, nu);
        mat3 b = link_get(U, xpn, mu);
        mat3 c = link_get(U, x, nu);
        mat3 bd = mat_dag(&b), cd = mat_dag(&c);
        const double w = plane_weight(g, mu < nu ? mu : nu, mu < nu ? nu : mu);
        mat3 t = mat_mul(&a, &bd);
        t = mat_mul(&t, &cd);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) t.m[i][j] *= w;
        A = mat_add(&A, &t);
        /* lower: U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) */
        long xmn = hop(g, x, nu, -1, &s);
        long xpmmn = hop(g, xpm, nu, -1, &s);
        mat3 d = link_get(U, xpmmn, nu);
        mat3 e = link_get(U, xmn, mu);
        mat3 f = link_get(U, xmn, nu);
        mat3 dd = mat_dag(&d), ed = mat_dag(&e);
        t = mat_mul(&dd, &ed);
        t = mat_mul(&t, &f);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) t.m[i][j] *= w;
        A = mat_add(&A, &t);
    }
    return A;
}

/* Gauge force coefficients at one link: F = -(i beta / 12) TA(U A). */
static void gauge_force_link(const geom *g, const double *U, double beta, long x, int mu, double *f)
{
    mat3 A = staple(g, U, x, mu);
    mat3 u = link_get(U, x, mu);
    mat3 W = mat_mul(&u, &A);
    mat3 T = proj_ta(&W);
    mat3 F = mat_scale(&T, -I * beta / 12.0);
    mat_to_algebra(&F, f);
}

/* ----------------------------------------------------------- fermion force */

/* The fields the fermion force needs from X_e (even-site solution):
 * Y_e = Mhat X_e, A = (X_e, Doe X_e), B = (Y_e, Deo^dag Y_e), full lattice. */
static void fermion_force_fields(const geom *g, const double *U, double kappa, const double *X, double *A,
                                 double *B)
{
    long n = g->V * 24;
    double *Xe = malloc(sizeof(double) * n);
    double *Y = malloc(sizeof(double) * n);
    double *t = malloc(sizeof(double) * n);
    memcpy(Xe, X, sizeof(double) * n);
    mask_parity(g, Xe, 0);
    mhat(g, U, kappa, Xe, Y, 0);
    dslash_full(g, U, Xe, t, 0, 1); /* Doe X_e on odd sites */
    for (long k = 0; k < n; k++) A[k] = Xe[k] + t[k];
    dslash_full(g, U, Y, t, 1, 1); /* (D^dag Y_e) on odd sites */
    for (long k = 0; k < n; k++) B[k] = Y[k] + t[k];
    free(Xe);
    free(Y);
    free(t);
}

/* The fields of the force term -2 Re[Y^dag (d Mhat) X] for given even-site
 * X and Y (the standard term has Y = Mhat X): A = (X_e, Doe X_e),
 * B = (Y_e, Deo^dag Y_e), full lattice. */
static void fermion_force_fields_xy(const geom *g, const double *U, const double *X, const double *Y, double *A,
                                    double *B)
{
    long n = g->V * 24;
    double *Xe = malloc(sizeof(double) * n);
    double *Ye = malloc(sizeof(double) * n);
    double *t = malloc(sizeof(double) * n);
    memcpy(Xe, X, sizeof(double) * n);
    mask_parity(g, Xe, 0);
    memcpy(Ye, Y, sizeof(double) * n);
    mask_parity(g, Ye, 0);
    dslash_full(g, U, Xe, t, 0, 1);
    for (long k = 0; k < n; k++) A[k] = Xe[k] + t[k];
    dslash_full(g, U, Ye, t, 1, 1);
    for (long k = 0; k < n; k++) B[k] = Ye[k] + t[k];
    free(Xe);
    free(Ye);
    free(t);
}

/* Fermion force coefficients at one link (x, mu):
 *   Q1 = sum_spin [s U_mu(x) A(x+mu)] [(1 - gamma_mu) B(x)]^dag
 *   Q2 = sum_spin A(x) [s U_mu(x) (1 + gamma_mu) B(x+mu)]^dag
 *   F  = (i kappa^2 / 2) TA(Q1 - Q2)
 * which is the reading of dS_f/de_a = 2 kappa^2 Re[B^dag (dD/de_a) A]. */
static void fermion_force_link(const geom *g, const double *U, double kappa, const double *A, const double *B,
                               long x, int mu, double *f)
{
    gamma_init();
    double s;
    long y = hop(g, x, mu, +1, &s);
    mat3 u = link_get(U, x, mu);
    const cplx *Ay = spinor_at_c(A, y), *Ax = spinor_at_c(A, x);
    const cplx *Bx = spinor_at_c(B, x), *By = spinor_at_c(B, y);
    /* v1[spin][color] = s U A(y);  w1 = (1 - gamma_mu) B(x) */
    cplx v1[12], w1[12], v2[12], w2[12], pb[12];
    for (int b = 0; b < 4; b++)
        for (int a = 0; a < 3; a++) {
            cplx acc = 0;
            for (int c = 0; c < 3; c++) acc += u.m[a][c] * Ay[b * 3 + c];
            v1[b * 3 + a] = s * acc;
        }
    for (int al = 0; al < 4; al++)
        for (int a = 0; a < 3; a++) {
            cplx acc = 0, acc2 = 0;
            for (int be = 0; be < 4; be++) {
                acc += ((al == be ? 1.0 : 0.0) - G[mu][al][be]) * Bx[be * 3 + a];
                acc2 += ((al == be ? 1.0 : 0.0) + G[mu][al][be]) * By[be * 3 + a];
            }
            w1[al * 3 + a] = acc;
            pb[al * 3 + a] = acc2;
        }
    /* w2 = s U (1 + gamma_mu) B(y);  v2 = A(x) */
    for (int b = 0; b < 4; b++)
        for (int a = 0; a < 3; a++) {
            cplx acc = 0;
            for (int c = 0; c < 3; c++) acc += u.m[a][c] * pb[b * 3 + c];
            w2[b * 3 + a] = s * acc;
            v2[b * 3 + a] = Ax[b * 3 + a];
        }
    mat3 Q = mat_zero();
    for (int a = 0; a < 3; a++)
        for (int c = 0; c < 3; c++) {
            cplx acc = 0;
            for (int sp = 0; sp < 4; sp++)
                acc += v1[sp * 3 + a] * conj(w1[sp * 3 + c]) - v2[sp * 3 + a] * conj(w2[sp * 3 + c]);
            Q.m[a][c] = acc;
        }
    mat3 T = proj_ta(&Q);
    mat3 F = mat_scale(&T, I * kappa * kappa / 2.0);
    mat_to_algebra(&F, f);
    /* the link enters the operator through its hop, weighted by the hop's weight */
    const double w = mu < 3 ? g->cs : 1.0;
    for (int k = 0; k < 8; k++) f[k] *= w;
}

/* ------------------------------------------------------------------- Philox */

/* Philox4x32-10 block function (Salmon et al., SC'11): 10 rounds of two 32x32
 * -> 64-bit multiplies with the published multipliers and Weyl key increments. */
void or_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Two uniforms in (0,1) from one Philox call: u = ((w >> 12) + 1/2) 2^-52 with
 * w the 64-bit word (x0 << 32 | x1), resp. (x2 << 32 | x3).  Exact in double. */
static void philox_uniform2(uint32_t seed, uint32_t chain, uint32_t site, uint32_t j, uint32_t purpose,
                            uint32_t traj, double u[2])
{
    uint32_t ctr[4] = {site, j, purpose, traj}, key[2] = {seed, chain}, x[4];
    or_philox4x32_10(ctr, key, x);
    uint64_t w0 = ((uint64_t)x[0] << 32) | x[1];
    uint64_t w1 = ((uint64_t)x[2] << 32) | x[3];
    u[0] = ((double)(w0 >> 12) + 0.5) * ldexp(1.0, -52);
    u[1] = ((double)(w1 >> 12) + 0.5) * ldexp(1.0, -52);
}

/* Box-Muller: r = sqrt(-2 ln u1), theta = 2 pi u2 -> (r cos theta, r sin theta). */
static void philox_gauss2(uint32_t seed, uint32_t chain, uint32_t site, uint32_t j, uint32_t purpose,
                          uint32_t traj, double gz[2])
{
    double u[2];
    philox_uniform2(seed, chain, site, j, purpose, traj, u);
    double r = sqrt(-2.0 * log(u[0]));
    double th = (2.0 * M_PI) * u[1];
    gz[0] = r * cos(th);
    gz[1] = r * sin(th);
}

enum { PURPOSE_GAUGE = 0, PURPOSE_MOM = 1, PURPOSE_ETA = 2, PURPOSE_METRO = 3, PURPOSE_ETA_H = 4 };

void or_uniform2(uint32_t seed, uint32_t chain, uint32_t site, uint32_t j, uint32_t purpose, uint32_t traj,
                 double *u)
{
    philox_uniform2(seed, chain, site, j, purpose, traj, u);
}

void or_gauss2(uint32_t seed, uint32_t chain, uint32_t site, uint32_t j, uint32_t purpose, uint32_t traj,
               double *gz)
{
    philox_gauss2(seed, chain, site, j, purpose, traj, gz);
}

/* ================================================================ exports */

/* Plain wrappers with C types for ctypes.  dims = int[4] (Lx, Ly, Lz, Lt).
 * Return 0 on success, -1 on invalid geometry. */

int or_plaquette(const int *dims, const double *U, double *plaq)
{
    geom g;
    if (geom_init(&g, dims, -1)) return -1;
    *plaq = plaq_sum(&g, U) / (6.0 * g.V);
    return 0;
}

int or_gauge_action(const int *dims, const double *U, double beta, double *S)
{
    geom g;
    if (geom_init(&g, dims, -1)) return -1;
    *S = gauge_action(&g, U, beta);
    return 0;
}

int or_dslash(const int *dims, int t_bc, const double *U, const double *in, double *out, int dagger,
              int out_parity)
{
    geom g;
    if (geom_init(&g, dims, t_bc)) return -1;
    dslash_full(&g, U, in, out, dagger, out_parity);
    return 0;
}

/* D (or D^dag) at a list of sites; out is [n][24]. */
int or_dslash_at(const int *dims, int t_bc, const double *U, const double *in, int dagger, long n,
                 const long *sites, double *out)
{
    geom g;
    if (geom_init(&g, dims, t_bc)) return -1;
    double *src = (double *)in;
    double *tmp = NULL;
    if (dagger) {
        tmp = malloc(sizeof(double) * 24 * g.V);
        apply_g5(&g, in, tmp);
        src = tmp;
    }
    for (long k = 0; k < n; k++) {
        cplx r[12];
        dslash_site(&g, U, src, sites[k], r);
        if (dagger) {
            cplx q[12];
            for (int a = 0; a < 4; a++)
                for (int c = 0; c < 3; c++) {
                    cplx acc = 0;
                    for (int b = 0; b < 4; b++) acc += G[4][a][b] * r[b * 3 + c];
                    q[a * 3 + c] = acc;
                }
            memcpy(r, q, sizeof(r));
        }
        memcpy(out + k * 24, r, sizeof(r));
    }
    free(tmp);
    return 0;
}

int or_mhat(const int *dims, int t_bc, const double *U, double kappa, const double *in, double *out,
            int dagger)
{
    geom g;
    if (geom_init(&g, dims, t_bc)) return -1;
    mhat(&g, U, kappa, in, out, dagger);
    return 0;
}

int or_mdagm(const int *dims, int t_bc, const double *U, double kappa, const double *in, double *out)
{
    geom g;
    if (geom_init(&g, dims, t_bc)) return -1;
    mdagm(&g, U, kappa, in, out);
    return 0;
}

/* returns 0 converged, 1 not converged, -1 bad geometry */
int or_cg(const int *dims, int t_bc, const double *U, double kappa, const double *b, double *x, double tol,
          int maxiter, int *iters, double *true_rel)
{
    geom g;
    if (geom_init(&g, dims, t_bc)) return -1;
    return cg_solve(&g, U, kappa, b, x, tol, maxiter, iters, true_rel);
}

/* F = gauge force coefficients [V][4][8] */
int or_gauge_force(const int *dims, const double *U, double beta, double *F)
{
    geom g;
    if (geom_init(&g, dims, -1)) return -1;
    #pragma omp parallel for schedule(static)
    for (long x = 0; x < g.V; x++)
        for (int mu = 0; mu < 4; mu++) gauge_force_link(&g, U, beta, x, mu, F + (x * 4 + mu) * 8);
    return 0;
}

/* gauge force at a list of links (link = site*4 + mu); F is [n][8] */
int or_gauge_force_at(const int *dims, const double *U, double beta, long n, const long *links, double *F)
{
    geom g;
    if (geom_init(&g, dims, -1)) return -1;
    for (long k = 0; k < n; k++) gauge_force_link(&g, U, beta, links[k] / 4, (int)(links[k] % 4), F + k * 8);
    return 0;
}

/* F = fermion force coefficients [V][4][8] given X_e (full-lattice array, odd
 * sites ignored); n < 0 means every link, else only the listed links into
 * F[n][8]. */
int or_fermion_force(const int *dims, int t_bc, const double *U, double kappa, const double *X, long n,
                     const long *links, double *F)
{
    geom g;
    if (geom_init(&g, dims, t_bc)) return -1;
    double *A = malloc(sizeof(double) * 24 * g.V);
    double *B = malloc(sizeof(double) * 24 * g.V);
    fermion_force_fields(&g, U, kappa, X, A, B);
    gamma_init();
    if (n < 0) {
        #pragma omp parallel for schedule(static)
        for (long x = 0; x < g.V; x++)
            for (int mu = 0; mu < 4; mu++) fermion_force_link(&g, U, kappa, A, B, x, mu, F + (x * 4 + mu) * 8);
    } else {
        for (long k = 0; k < n; k++)
            fermion_force_link(&g, U, kappa, A, B, links[k] / 4, (int)(links[k] % 4), F + k * 8);
    }
    free(A);
    free(B);
    return 0;
}

/* pseudofermion action phi^dag (Mhat^dag Mhat)^-1 phi by CG; returns CG status */
int or_fermion_action(const int *dims, int t_bc, const double *U, double kappa, const double *phi, double tol,
                      int maxiter, double *S, int *iters)
{
    geom g;
    if (geom_init(&g, dims, t_bc)) return -1;
    double *X = malloc(sizeof(double) * 24 * g.V);
    double *ph = malloc(sizeof(double) * 24 * g.V);
    memcpy(ph, phi, sizeof(double) * 24 * g.V);
    mask_parity(&g, ph, 0);
    double rel;
    int st = cg_solve(&g, U, kappa, ph, X, tol, maxiter, iters, &rel);
    *S = dot_re(&g, ph, X);
    free(X);
    free(ph);
    return st;
}

/* single-matrix helpers for tests: exp(i c H) with H Hermitian (18 doubles),
 * TA projection, reunitarization, algebra <-> matrix */
void or_su3_expi(const double *H, double c, double *out)
{
    mat3 h;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) h.m[a][b] = H[(a * 3 + b) * 2] + I * H[(a * 3 + b) * 2 + 1];
    mat3 e = expi_herm(&h, c);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            out[(a * 3 + b) * 2] = creal(e.m[a][b]);
            out[(a * 3 + b) * 2 + 1] = cimag(e.m[a][b]);
        }
}

void or_algebra_to_mat(const double *c8, double *out18)
{
    mat3 m = algebra_to_mat(c8);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            out18[(a * 3 + b) * 2] = creal(m.m[a][b]);
            out18[(a * 3 + b) * 2 + 1] = cimag(m.m[a][b]);
        }
}

void or_reunit_mat(const double *in18, double *out18)
{
    mat3 m;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) m.m[a][b] = in18[(a * 3 + b) * 2] + I * in18[(a * 3 + b) * 2 + 1];
    mat3 r = reunit(&m);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            out18[(a * 3 + b) * 2] = creal(r.m[a][b]);
            out18[(a * 3 + b) * 2 + 1] = cimag(r.m[a][b]);
        }
}

/* Start configuration: U_mu(x) = exp(i eps sum_a h_a T_a), h_a ~ N(0,1) from
 * Philox purpose 0, counter (site, j, 0, 0), j = 0..15 giving coefficients
 * k = 2j, 2j+1 with mu = k / 8, a = k % 8. */
int or_gauge_start(const int *dims, uint32_t seed, uint32_t chain, double eps, double *U)
{
    geom g;
    if (geom_init(&g, dims, -1)) return -1;
    for (long x = 0; x < g.V; x++) {
        double h[32];
        for (int j = 0; j < 16; j++) philox_gauss2(seed, chain, (uint32_t)x, j, PURPOSE_GAUGE, 0, h + 2 * j);
        for (int mu = 0; mu < 4; mu++) {
            mat3 H = algebra_to_mat(h + mu * 8);
            mat3 u = expi_herm(&H, eps);
            link_set(U, x, mu, &u);
        }
    }
    return 0;
}

/* Momenta p_a ~ N(0,1): Philox purpose 1, counter (site, j, 1, traj), same
 * coefficient order as the start configuration.  P is [V][4][8]. */
int or_momentum_refresh(const int *dims, uint32_t seed, uint32_t chain, uint32_t traj, double *P)
{
    geom g;
    if (geom_init(&g, dims, -1)) return -1;
    for (long x = 0; x < g.V; x++)
        for (int j = 0; j < 16; j++) philox_gauss2(seed, chain, (uint32_t)x, j, PURPOSE_MOM, traj, P + x * 32 + 2 * j);
    return 0;
}

/* eta on even sites, each real ~ N(0, 1/2): Philox purpose 2, counter
 * (site, j, 2, traj), j = 0..11 giving reals k = 2j, 2j+1 in [spin][color][re,im]
 * order.  Odd sites are zero. */
static void eta_refresh_purpose(const geom *g, uint32_t seed, uint32_t chain, uint32_t purpose, uint32_t traj,
                                double *eta)
{
    memset(eta, 0, sizeof(double) * 24 * g->V);
    for (long x = 0; x < g->V; x++) {
        if (site_parity(g, x) != 0) continue;
        for (int j = 0; j < 12; j++) {
            double z[2];
            philox_gauss2(seed, chain, (uint32_t)x, j, purpose, traj, z);
            eta[x * 24 + 2 * j] = z[0] * sqrt(0.5);
            eta[x * 24 + 2 * j + 1] = z[1] * sqrt(0.5);
        }
    }
}

/* the second pseudofermion's eta of the Hasenbusch action: as or_eta_refresh
 * with Philox purpose 4 */
int or_eta_refresh_h(const int *dims, uint32_t seed, uint32_t chain, uint32_t traj, double *eta)
{
    geom g;
    if (geom_init(&g, dims, -1)) return -1;
    eta_refresh_purpose(&g, seed, chain, PURPOSE_ETA_H, traj, eta);
    return 0;
}

int or_eta_refresh(const int *dims, uint32_t seed, uint32_t chain, uint32_t traj, double *eta)
{
    geom g;
    if (geom_init(&g, dims, -1)) return -1;
    memset(eta, 0, sizeof(double) * 24 * g.V);
    for (long x = 0; x < g.V; x++) {
        if (site_parity(&g, x) != 0) continue;
        for (int j = 0; j < 12; j++) {
            double z[2];
            philox_gauss2(seed, chain, (uint32_t)x, j, PURPOSE_ETA, traj, z);
            eta[x * 24 + 2 * j] = z[0] * sqrt(0.5);
            eta[x * 24 + 2 * j + 1] = z[1] * sqrt(0.5);
        }
    }
    return 0;
}

/* U <- exp(i c P) U on every link */
int or_link_update(const int *dims, double *U, const double *P, double c)
{
    geom g;
    if (geom_init(&g, dims, -1)) return -1;
    #pragma omp parallel for schedule(static)
    for (long x = 0; x < g.V; x++)
        for (int mu = 0; mu < 4; mu++) {
            mat3 H = algebra_to_mat(P + (x * 4 + mu) * 8);
            mat3 e = expi_herm(&H, c);
            mat3 u = link_get(U, x, mu);
            mat3 r = mat_mul(&e, &u);
            link_set(U, x, mu, &r);
        }
    return 0;
}

/* reunitarize every link; *maxdev = max over links of max |(U U^dag - 1)_ij| before */
int or_reunitarize(const int *dims, double *U, double *maxdev)
{
    geom g;
    if (geom_init(&g, dims, -1)) return -1;
    double m = 0;
#pragma omp parallel for schedule(static) reduction(max : m)
    for (long x = 0; x < g.V; x++)
        for (int mu = 0; mu < 4; mu++) {
            mat3 u = link_get(U, x, mu);
            double d = unitarity_dev(&u);
            if (d > m) m = d;
            mat3 r = reunit(&u);
            link_set(U, x, mu, &r);
        }
    *maxdev = m;
    return 0;
}

/* 1/2 sum p_a^2 over all links */
double or_kinetic(const int *dims, const double *P)
{
    geom g;
    if (geom_init(&g, dims, -1)) return -1;
    double s = 0;
    for (long k = 0; k < g.V * 32; k++) s += P[k] * P[k];
    return 0.5 * s;
}

/* -------------------------------------------------------------- integration */

typedef struct {
    double beta, kappa, tau;
    int nsteps;
    int integrator; /* 0 leapfrog, 1 Omelyan 2MN */
    int n_flavors;  /* 0 pure gauge, 2 Wilson fermions */
    double cg_tol;
    int cg_maxiter;
} md_params;

typedef struct {
    long cg_iters;
    int n_solves;
    int cg_fail;
} md_stats;

/* P <- P - c * F(U), F the total force (gauge + fermion) */
static void kick(const geom *g, const double *U, double *P, const double *phi, const md_params *mp, double c,
                 md_stats *st)
{
    #pragma omp parallel for schedule(static)
    for (long x = 0; x < g->V; x++)
        for (int mu = 0; mu < 4; mu++) {
            double f[8];
            gauge_force_link(g, U, mp->beta, x, mu, f);
            for (int a = 0; a < 8; a++) P[(x * 4 + mu) * 8 + a] -= c * f[a];
        }
    if (mp->n_flavors == 2) {
        double *X = malloc(sizeof(double) * 24 * g->V);
        double *A = malloc(sizeof(double) * 24 * g->V);
        double *B = malloc(sizeof(double) * 24 * g->V);
        int it;
        double rel;
        if (cg_solve(g, U, mp->kappa, phi, X, mp->cg_tol, mp->cg_maxiter, &it, &rel)) st->cg_fail++;
        st->cg_iters += it;
        st->n_solves++;
        fermion_force_fields(g, U, mp->kappa, X, A, B);
        gamma_init();
        #pragma omp parallel for schedule(static)
        for (long x = 0; x < g->V; x++)
            for (int mu = 0; mu < 4; mu++) {
                double f[8];
                fermion_force_link(g, U, mp->kappa, A, B, x, mu, f);
                for (int a = 0; a < 8; a++) P[(x * 4 + mu) * 8 + a] -= c * f[a];
            }
        free(X);
        free(A);
        free(B);
    }
}

static void drift(const geom *g, double *U, const double *P, double c)
{
    #pragma omp parallel for schedule(static)
    for (long x = 0; x < g->V; x++)
        for (int mu = 0; mu < 4; mu++) {
            mat3 H = algebra_to_mat(P + (x * 4 + mu) * 8);
            mat3 e = expi_herm(&H, c);
            mat3 u = link_get(U, x, mu);
            mat3 r = mat_mul(&e, &u);
            link_set(U, x, mu, &r);
        }
}

/* Integrate (U, P) for time tau in nsteps steps.  Adjacent momentum kicks of
 * consecutive steps are merged into one kick of the summed coefficient.
 * Leapfrog: P -= dt/2 F; U <- e^{i dt P} U; P -= dt/2 F.
 * Omelyan 2MN: P -= l dt F; U <- e^{i dt/2 P} U; P -= (1-2l) dt F;
 *              U <- e^{i dt/2 P} U; P -= l dt F,  l = 0.1931833275037836. */
static void md_integrate(const geom *g, double *U, double *P, const double *phi, const md_params *mp,
                         md_stats *st)
{
    double dt = mp->tau / mp->nsteps;
    if (mp->integrator == 0) {
        kick(g, U, P, phi, mp, 0.5 * dt, st);
        for (int s = 0; s < mp->nsteps; s++) {
            drift(g, U, P, dt);
            kick(g, U, P, phi, mp, (s == mp->nsteps - 1) ? 0.5 * dt : dt, st);
        }
    } else {
        const double lam = 0.1931833275037836;
        kick(g, U, P, phi, mp, lam * dt, st);
        for (int s = 0; s < mp->nsteps; s++) {
            drift(g, U, P, 0.5 * dt);
            kick(g, U, P, phi, mp, (1.0 - 2.0 * lam) * dt, st);
            drift(g, U, P, 0.5 * dt);
            kick(g, U, P, phi, mp, (s == mp->nsteps - 1) ? lam * dt : 2.0 * lam * dt, st);
        }
    }
}

/* Molecular dynamics only (no refresh, no accept/reject): integrates U, P in
 * place with a given phi (even-site full-lattice array; ignored if n_flavors
 * is 0).  stats_out: [cg_iters, n_solves, cg_failures]. */
int or_md_integrate(const int *dims, int t_bc, double *U, double *P, const double *phi, double beta,
                    double kappa, double tau, int nsteps, int integrator, int n_flavors, double cg_tol,
                    int cg_maxiter, double *stats_out)
{
    geom g;
    if (geom_init(&g, dims, t_bc)) return -1;
    md_params mp = {beta, kappa, tau, nsteps, integrator, n_flavors, cg_tol, cg_maxiter};
    md_stats st = {0, 0, 0};
    md_integrate(&g, U, P, phi, &mp, &st);
    stats_out[0] = (double)st.cg_iters;
    stats_out[1] = st.n_solves;
    stats_out[2] = st.cg_fail;
    return 0;
}

/* H = 1/2 sum p^2 + S_g + S_f (S_f by CG when n_flavors == 2) */
int or_hamiltonian(const int *dims, int t_bc, const double *U, const double *P, const double *phi, double beta,
                   double kappa, int n_flavors, double cg_tol, int cg_maxiter, double *H)
{
    geom g;
    if (geom_init(&g, dims, t_bc)) return -1;
    double h = or_kinetic(dims, P) + gauge_action(&g, U, beta);
    if (n_flavors == 2) {
        double S;
        int it;
        or_fermion_action(dims, t_bc, U, kappa, phi, cg_tol, cg_maxiter, &S, &it);
        h += S;
    }
    *H = h;
    return 0;
}

/* One HMC trajectory (Sec. 1 of the paper lists its parts):
 *   P from Philox purpose 1; eta from purpose 2, phi_e = Mhat^dag eta_e;
 *   H0 = T + S_g + eta^dag eta;  MD for tau;  H1 = T + S_g + phi^dag X;
 *   accept iff u < exp(-dH), u the first uniform of counter (0, 0, 3, traj);
 *   on reject restore U; then reunitarize (if asked) and measure the plaquette.
 * info_out (doubles): [0] dH [1] accepted [2] plaquette [3] cg_iters
 *   [4] H0 [5] H1 [6] u [7] max unitarity deviation before reunitarization
 *   [8] n_solves [9] cg failures */
int or_hmc_trajectory(const int *dims, int t_bc, double *U, double beta, double kappa, double tau, int nsteps,
                      int integrator, int n_flavors, double cg_tol, int cg_maxiter, uint32_t seed, uint32_t chain,
                      uint32_t traj, int do_reunit, int do_metropolis, double *info_out)
{
    geom g;
    if (geom_init(&g, dims, t_bc)) return -1;
    long nl = g.V * 4 * 18, ns = g.V * 24;
    double *P = malloc(sizeof(double) * g.V * 32);
    double *U0 = malloc(sizeof(double) * nl);
    double *eta = malloc(sizeof(double) * ns);
    double *phi = malloc(sizeof(double) * ns);
    memcpy(U0, U, sizeof(double) * nl);
    or_momentum_refresh(dims, seed, chain, traj, P);
    double H0 = or_kinetic(dims, P) + gauge_action(&g, U, beta);
    if (n_flavors == 2) {
        or_eta_refresh(dims, seed, chain, traj, eta);
        mhat(&g, U, kappa, eta, phi, 1);
        H0 += dot_re(&g, eta, eta);
    } else {
        memset(phi, 0, sizeof(double) * ns);
    }
    md_params mp = {beta, kappa, tau, nsteps, integrator, n_flavors, cg_tol, cg_maxiter};
    md_stats st = {0, 0, 0};
    md_integrate(&g, U, P, phi, &mp, &st);
    double H1 = or_kinetic(dims, P) + gauge_action(&g, U, beta);
    if (n_flavors == 2) {
        double *X = malloc(sizeof(double) * ns);
        int it;
        double rel;
        if (cg_solve(&g, U, kappa, phi, X, cg_tol, cg_maxiter, &it, &rel)) st.cg_fail++;
        st.cg_iters += it;
        st.n_solves++;
        H1 += dot_re(&g, phi, X);
        free(X);
    }
    double dH = H1 - H0;
    double u[2];
    philox_uniform2(seed, chain, 0, 0, PURPOSE_METRO, traj, u);
    int accept = 1;
    if (do_metropolis) accept = isfinite(dH) && (u[0] < exp(-dH));
    if (!accept) memcpy(U, U0, sizeof(double) * nl);
    double maxdev = 0;
    if (do_reunit) or_reunitarize(dims, U, &maxdev);
    info_out[0] = dH;
    info_out[1] = accept;
    info_out[2] = plaq_sum(&g, U) / (6.0 * g.V);
    info_out[3] = (double)st.cg_iters;
    info_out[4] = H0;
    info_out[5] = H1;
    info_out[6] = u[0];
    info_out[7] = maxdev;
    info_out[8] = st.n_solves;
    info_out[9] = st.cg_fail;
    free(P);
    free(U0);
    free(eta);
    free(phi);
    return 0;
}

/* --------------------------------------------- Hasenbusch action, nested integration
 *
 * Mass preconditioning (the production feature named with the chronological
 * guess in Sec. 6.2) splits det(Mhat^dag Mhat) with W = Mhat(kappa_h),
 * kappa_h < kappa, into two pseudofermion actions:
 *   heavy  S_h = phi_h^dag (W^dag W)^-1 phi_h,
 *   ratio  S_r = chi^dag (Mhat^dag Mhat)^-1 chi,  chi = W^dag phi_r,
 * whose Gaussian integrals give det(W^dag W) and det(Mhat^dag Mhat)/det(W^dag W).
 * With X_r = (Mhat^dag Mhat)^-1 chi,
 *   dS_r = -2 Re[(Mhat X_r)^dag dMhat X_r] + 2 Re[phi_r^dag dW X_r],
 * i.e. the standard force term of (X_r, Y = Mhat X_r, kappa) minus the term
 * of (X_r, Y = phi_r, kappa_h).  Refresh: phi_h = W^dag eta_h, and
 * phi_r = W^-dag Mhat^dag eta = W (W^dag W)^-1 Mhat^dag eta, so that
 * S_h = |eta_h|^2 and S_r = |eta|^2 at the start.
 *
 * Nested integration (Sexton-Weingarten): with gauge_substeps m >= 2 the
 * gauge action (and the heavy action if heavy_inner) moves on an inner level
 * that integrates each drift of the outer level in m steps of the same scheme
 * (leapfrog or Omelyan 2MN); the fermion actions stay on the outer level of
 * nsteps steps.  Kicks are applied as they come (none merged). */

enum { TERM_GAUGE = 1, TERM_FERMION = 2, TERM_HEAVY = 4 };

typedef struct {
    double beta, kappa, kappa_h, tau;
    int nsteps, integrator, n_flavors, gauge_substeps, heavy_inner;
    double cg_tol;
    int cg_maxiter;
} hb_params;

/* P <- P - c F_xy with F_xy the force of -2 Re[Y^dag dMhat(kappa) X] */
static void add_force_xy(const geom *g, const double *U, double kappa, const double *X, const double *Y, double *P,
                         double c)
{
    double *A = malloc(sizeof(double) * 24 * g->V);
    double *B = malloc(sizeof(double) * 24 * g->V);
    fermion_force_fields_xy(g, U, X, Y, A, B);
    gamma_init();
    #pragma omp parallel for schedule(static)
    for (long x = 0; x < g->V; x++)
        for (int mu = 0; mu < 4; mu++) {
            double f[8];
            fermion_force_link(g, U, kappa, A, B, x, mu, f);
            for (int a = 0; a < 8; a++) P[(x * 4 + mu) * 8 + a] -= c * f[a];
        }
    free(A);
    free(B);
}

/* X = (Mhat(kappa)^dag Mhat(kappa))^-1 b and Y = Mhat(kappa) X */
static void solve_xy(const geom *g, const double *U, double kappa, const double *b, double *X, double *Y,
                     const hb_params *hp, md_stats *st)
{
    int it;
    double rel;
    if (cg_solve(g, U, kappa, b, X, hp->cg_tol, hp->cg_maxiter, &it, &rel)) st->cg_fail++;
    st->cg_iters += it;
    st->n_solves++;
    if (Y) mhat(g, U, kappa, X, Y, 0);
}

/* P <- P - c F of the selected action terms */
static void hb_kick(const geom *g, const double *U, double *P, const hb_params *hp, const double *phi,
                    const double *phi_h, int terms, double c, md_stats *st)
{
    if (terms & TERM_GAUGE) {
        #pragma omp parallel for schedule(static)
        for (long x = 0; x < g->V; x++)
            for (int mu = 0; mu < 4; mu++) {
                double f[8];
                gauge_force_link(g, U, hp->beta, x, mu, f);
                for (int a = 0; a < 8; a++) P[(x * 4 + mu) * 8 + a] -= c * f[a];
            }
    }
    if (hp->n_flavors != 2) return;
    long n = 24 * g->V;
    double *X = malloc(sizeof(double) * n), *Y = malloc(sizeof(double) * n), *chi = malloc(sizeof(double) * n);
    if (terms & TERM_FERMION) {
        if (hp->kappa_h == 0) {
            solve_xy(g, U, hp->kappa, phi, X, Y, hp, st);
            add_force_xy(g, U, hp->kappa, X, Y, P, c);
        } else {
            mhat(g, U, hp->kappa_h, phi, chi, 1);
            solve_xy(g, U, hp->kappa, chi, X, Y, hp, st);
            add_force_xy(g, U, hp->kappa, X, Y, P, c);
            add_force_xy(g, U, hp->kappa_h, X, phi, P, -c);
        }
    }
    if ((terms & TERM_HEAVY) && hp->kappa_h != 0) {
        solve_xy(g, U, hp->kappa_h, phi_h, X, Y, hp, st);
        add_force_xy(g, U, hp->kappa_h, X, Y, P, c);
    }
    free(X);
    free(Y);
    free(chi);
}

static int hb_levels(const hb_params *hp) { return hp->gauge_substeps >= 2 ? 2 : 1; }

static int hb_terms(const hb_params *hp, int level)
{
    if (hb_levels(hp) == 1) return TERM_GAUGE | TERM_FERMION | TERM_HEAVY;
    if (level == 0) return TERM_FERMION | (hp->heavy_inner ? 0 : TERM_HEAVY);
    return TERM_GAUGE | (hp->heavy_inner ? TERM_HEAVY : 0);
}

static void hb_integrate(const geom *g, double *U, double *P, const hb_params *hp, const double *phi,
                         const double *phi_h, int level, double t, md_stats *st);

/* the drift of one level: the next level's integration, or the link update */
static void hb_inner(const geom *g, double *U, double *P, const hb_params *hp, const double *phi,
                     const double *phi_h, int level, double t, md_stats *st)
{
    if (level + 1 < hb_levels(hp))
        hb_integrate(g, U, P, hp, phi, phi_h, level + 1, t, st);
    else
        drift(g, U, P, t);
}

static void hb_integrate(const geom *g, double *U, double *P, const hb_params *hp, const double *phi,
                         const double *phi_h, int level, double t, md_stats *st)
{
    const int n = level == 0 ? hp->nsteps : hp->gauge_substeps;
    const int terms = hb_terms(hp, level);
    const double h = t / n;
    const double lam = 0.1931833275037836;
    for (int s = 0; s < n; s++) {
        if (hp->integrator == 0) {
            hb_kick(g, U, P, hp, phi, phi_h, terms, 0.5 * h, st);
            hb_inner(g, U, P, hp, phi, phi_h, level, h, st);
            hb_kick(g, U, P, hp, phi, phi_h, terms, 0.5 * h, st);
        } else {
            hb_kick(g, U, P, hp, phi, phi_h, terms, lam * h, st);
            hb_inner(g, U, P, hp, phi, phi_h, level, 0.5 * h, st);
            hb_kick(g, U, P, hp, phi, phi_h, terms, (1.0 - 2.0 * lam) * h, st);
            hb_inner(g, U, P, hp, phi, phi_h, level, 0.5 * h, st);
            hb_kick(g, U, P, hp, phi, phi_h, terms, lam * h, st);
        }
    }
}

/* S_f of the current links: phi^dag (Mhat^dag Mhat)^-1 phi, or S_r + S_h */
static double hb_fermion_action(const geom *g, const double *U, const hb_params *hp, const double *phi,
                                const double *phi_h, md_stats *st)
{
    long n = 24 * g->V;
    double *X = malloc(sizeof(double) * n), *chi = malloc(sizeof(double) * n);
    double S;
    if (hp->kappa_h == 0) {
        solve_xy(g, U, hp->kappa, phi, X, NULL, hp, st);
        S = dot_re(g, phi, X);
    } else {
        mhat(g, U, hp->kappa_h, phi, chi, 1);
        solve_xy(g, U, hp->kappa, chi, X, NULL, hp, st);
        S = dot_re(g, chi, X);
        solve_xy(g, U, hp->kappa_h, phi_h, X, NULL, hp, st);
        S += dot_re(g, phi_h, X);
    }
    free(X);
    free(chi);
    return S;
}

/* The ratio action S_r and its force coefficients F[V][4][8] (NULL: none)
 * for a given phi_r: the pieces of the Hasenbusch trajectory, for tests. */
int or_hasenbusch_ratio(const int *dims, int t_bc, const double *U, double kappa, double kappa_h,
                        const double *phi_r, double tol, int maxiter, double *S, double *F)
{
    geom g;
    if (geom_init(&g, dims, t_bc)) return -1;
    hb_params hp = {0, kappa, kappa_h, 0, 0, 0, 2, 0, 0, tol, maxiter};
    md_stats st = {0, 0, 0};
    long n = 24 * g.V;
    double *X = malloc(sizeof(double) * n), *Y = malloc(sizeof(double) * n), *chi = malloc(sizeof(double) * n);
    mhat(&g, U, kappa_h, phi_r, chi, 1);
    solve_xy(&g, U, kappa, chi, X, Y, &hp, &st);
    *S = dot_re(&g, chi, X);
    if (F) {
        double *P = calloc(g.V * 32, sizeof(double));
        add_force_xy(&g, U, kappa, X, Y, P, -1.0);
        add_force_xy(&g, U, kappa_h, X, phi_r, P, 1.0);
        memcpy(F, P, sizeof(double) * g.V * 32);
        free(P);
    }
    free(X);
    free(Y);
    free(chi);
    return st.cg_fail ? 1 : 0;
}

/* The Hasenbusch refresh: phi_h = W^dag eta_h, phi_r = W (W^dag W)^-1 Mhat^dag eta
 * for given eta, eta_h (even sites). */
int or_hasenbusch_refresh(const int *dims, int t_bc, const double *U, double kappa, double kappa_h,
                          const double *eta, const double *eta_h, double tol, int maxiter, double *phi_r,
                          double *phi_h)
{
    geom g;
    if (geom_init(&g, dims, t_bc)) return -1;
    hb_params hp = {0, kappa, kappa_h, 0, 0, 0, 2, 0, 0, tol, maxiter};
    md_stats st = {0, 0, 0};
    long n = 24 * g.V;
    double *t = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
    mhat(&g, U, kappa_h, eta_h, phi_h, 1);
    mhat(&g, U, kappa, eta, t, 1);
    solve_xy(&g, U, kappa_h, t, z, phi_r, &hp, &st);
    free(t);
    free(z);
    return st.cg_fail ? 1 : 0;
}

/* One HMC trajectory with the Hasenbusch action (kappa_h > 0) and/or the nested
 * integrator (gauge_substeps >= 2); kappa_h = 0 and gauge_substeps <= 1 give
 * the trajectory of or_hmc_trajectory with unmerged kicks.  The second eta
 * comes from Philox purpose 4.  info_out as or_hmc_trajectory. */
int or_hmc_trajectory_hb(const int *dims, int t_bc, double *U, double beta, double kappa, double kappa_h,
                         double tau, int nsteps, int integrator, int n_flavors, int gauge_substeps, int heavy_inner,
                         double cg_tol, int cg_maxiter, uint32_t seed, uint32_t chain, uint32_t traj, int do_reunit,
                         int do_metropolis, double *info_out)
{
    geom g;
    if (geom_init(&g, dims, t_bc)) return -1;
    hb_params hp = {beta, kappa, kappa_h, tau, nsteps, integrator, n_flavors, gauge_substeps, heavy_inner,
                    cg_tol, cg_maxiter};
    md_stats st = {0, 0, 0};
    long nl = g.V * 4 * 18, ns = g.V * 24;
    double *P = malloc(sizeof(double) * g.V * 32);
    double *U0 = malloc(sizeof(double) * nl);
    double *eta = malloc(sizeof(double) * ns), *eta_h = malloc(sizeof(double) * ns);
    double *phi = calloc(ns, sizeof(double)), *phi_h = calloc(ns, sizeof(double));
    memcpy(U0, U, sizeof(double) * nl);
    or_momentum_refresh(dims, seed, chain, traj, P);
    double H0 = or_kinetic(dims, P) + gauge_action(&g, U, beta);
    if (n_flavors == 2) {
        eta_refresh_purpose(&g, seed, chain, PURPOSE_ETA, traj, eta);
        H0 += dot_re(&g, eta, eta);
        if (kappa_h == 0) {
            mhat(&g, U, kappa, eta, phi, 1);
        } else {
            eta_refresh_purpose(&g, seed, chain, PURPOSE_ETA_H, traj, eta_h);
            H0 += dot_re(&g, eta_h, eta_h);
            double *t = malloc(sizeof(double) * ns), *z = malloc(sizeof(double) * ns);
            mhat(&g, U, kappa_h, eta_h, phi_h, 1);
            mhat(&g, U, kappa, eta, t, 1);
            solve_xy(&g, U, kappa_h, t, z, phi, &hp, &st);
            free(t);
            free(z);
        }
    }
    hb_integrate(&g, U, P, &hp, phi, phi_h, 0, tau, &st);
    double H1 = or_kinetic(dims, P) + gauge_action(&g, U, beta);
    if (n_flavors == 2) H1 += hb_fermion_action(&g, U, &hp, phi, phi_h, &st);
    double dH = H1 - H0;
    double u[2];
    philox_uniform2(seed, chain, 0, 0, PURPOSE_METRO, traj, u);
    int accept = 1;
    if (do_metropolis) accept = isfinite(dH) && (u[0] < exp(-dH));
    if (!accept) memcpy(U, U0, sizeof(double) * nl);
    double maxdev = 0;
    if (do_reunit) or_reunitarize(dims, U, &maxdev);
    info_out[0] = dH;
    info_out[1] = accept;
    info_out[2] = plaq_sum(&g, U) / (6.0 * g.V);
    info_out[3] = (double)st.cg_iters;
    info_out[4] = H0;
    info_out[5] = H1;
    info_out[6] = u[0];
    info_out[7] = maxdev;
    info_out[8] = st.n_solves;
    info_out[9] = st.cg_fail;
    free(P);
    free(U0);
    free(eta);
    free(eta_h);
    free(phi);
    free(phi_h);
    return 0;
}
