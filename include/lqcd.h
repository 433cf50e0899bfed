/*
 * lqcd.h -- C ABI of a device-resident Hybrid Monte Carlo for SU(3) lattice
 * gauge theory with two flavours of Wilson fermions on one NVIDIA GB300
 * (sm_103a).
 *
 * The paper this follows (F. Winter, "Gauge Field Generation on Large-Scale
 * GPU-Enabled Systems", Lattice 2012) argues that every part of an HMC
 * trajectory must run on the accelerator, not only the solver (Sec. 1), and
 * lists those parts: pseudofermion refresh, momentum updates, force terms,
 * projection of fields, reunitarization of SU(3) matrices, a random number
 * generator and the exponentiation of SU(3) matrices (Sec. 1), plus global
 * reductions `sum`/`sumMulti` (Sec. 1) and the matrix inversions done by a
 * Krylov solver (Sec. 6).  It ran Nf = 2 Wilson fermions (Sec. 6.2).  It gives
 * no formulas; the conventions fixed here are:
 *
 *   Lattice      dims = (Lx, Ly, Lz, Lt), all even, V = LxLyLzLt, Vh = V/2.
 *                Lexicographic site i = x + Lx(y + Ly(z + Lz t)); parity
 *                (x+y+z+t) mod 2; checkerboard index cb = i/2 within a parity.
 *   Gamma basis  DeGrand-Rossi (Hermitian), gamma_5 = diag(1, 1, -1, -1).
 *   Hopping term (D psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                                      + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ],
 *                each hop across the t boundary multiplied by t_bc (fermions
 *                antiperiodic in t by default; links periodic).
 *   Wilson op.   M = 1 - kappa D; even-odd Mhat = 1 - kappa^2 Deo Doe on
 *                even sites (det M = det Mhat).
 *   Actions      S_g = beta sum_x sum_{mu<nu} (1 - Re Tr U_munu(x) / 3);
 *                S_f = phi_e^dag (Mhat^dag Mhat)^-1 phi_e (two flavours);
 *                T   = sum_links 1/2 sum_a p_a^2 with P = sum_a p_a T_a,
 *                T_a = lambda_a / 2 (Gell-Mann).
 *   MD           dU/dt = i P U, dP/dt = -F, F = sum_a T_a dS/de_a with
 *                dS/de_a = d/de S(exp(i e T_a) U_mu(x)) at e = 0.
 *   RNG          Philox4x32-10 (Salmon et al., SC'11), key (seed, chain),
 *                counter (site, j, purpose, trajectory); purposes 0 gauge
 *                start, 1 momenta, 2 pseudofermion eta, 3 Metropolis.
 *
 * Canonical HOST layouts (FP64, used by upload/download):
 *   LQCD_GAUGE        [site][mu][row][col][re,im]   18 doubles / link
 *   LQCD_MOMENTUM     [site][mu][a]                 8 doubles / link
 *   LQCD_SPINOR_EVEN/ODD  [cb][spin][color][re,im]  24 doubles / site of that
 *                     parity, cb ascending (= lexicographic order of the sites
 *                     of that parity)
 *   LQCD_SPINOR_FULL  [site][spin][color][re,im]    24 doubles / site
 *
 * Conventions of every call:
 *   - The return value is an lqcd_status; on failure lqcd_last_error() gives a
 *     message (thread-local, valid until the next failing call on that thread).
 *     No call aborts the process or raises into the caller.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Kernels
 *     are enqueued asynchronously on it; calls that return host scalars
 *     synchronise that stream before returning.
 *   - Device memory of fields and work buffers comes from the allocator set
 *     by lqcd_set_allocator (default: cudaMalloc / cudaFree).
 *   - Pointers named *_dev are device pointers owned by the caller; all other
 *     pointers to numbers are host pointers owned by the caller.
 *   - Fields are not thread-safe: one call at a time per field.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LQCD_OK = 0,
    LQCD_EINVAL = 1,   /* bad argument: null pointer, odd/zero dims, kind or precision mismatch */
    LQCD_ENOMEM = 2,   /* the allocator returned NULL */
    LQCD_ENOCONV = 3,  /* a solver reached maxiter; its info holds the true residual */
    LQCD_ENUMERIC = 4, /* non-finite value in a reduction (dH, residual) */
    LQCD_ECUDA = 5,    /* a CUDA runtime call failed; message from cudaGetErrorString */
    LQCD_EAGAIN = 6,   /* result not ready yet (asynchronous solve) */
    LQCD_ETIMEOUT = 7  /* a bounded wait gave up (reserved: no kernel of this library waits on
                          another kernel, so no call returns it today) */
} lqcd_status;

typedef struct {
    int dims[4]; /* Lx, Ly, Lz, Lt: positive and even, V < 2^31 */
    int t_bc;    /* fermion boundary factor in t: -1 antiperiodic, +1 periodic */
    double xi0;  /* anisotropic Wilson actions (the paper's runs, Fig. 3): the gauge action weighs the
                    plaquettes of the planes with t by beta xi0 and the spatial ones by beta / xi0;
                    0 or 1: isotropic */
    double nu;   /* the Wilson operator weighs its spatial hops by nu / xi0 (its t hops by 1);
                    0 counts as 1 */
} lqcd_lattice;

typedef enum {
    LQCD_GAUGE = 0,       /* 4 links per site */
    LQCD_MOMENTUM = 1,    /* 8 su(3) coefficients per link, FP64 only */
    LQCD_SPINOR_EVEN = 2, /* 4 spin x 3 colour on even sites */
    LQCD_SPINOR_ODD = 3,  /* 4 spin x 3 colour on odd sites */
    LQCD_SPINOR_FULL = 4  /* both parities, FP64 only */
} lqcd_kind;

typedef enum {
    LQCD_F64 = 0,  /* FP64 storage and arithmetic */
    LQCD_F32 = 1,  /* FP32 storage, FP32 arithmetic */
    LQCD_F16N = 2, /* spinors: FP16 of value / site norm, FP32 norm = max |component|;
                      links: FP16 (entries of SU(3) rows lie in [-1, 1]); FP32 arithmetic */
    LQCD_BF16 = 3  /* BF16 storage, FP32 arithmetic */
} lqcd_prec;

typedef enum { LQCD_LEAPFROG = 0, LQCD_OMELYAN = 1 } lqcd_integrator;

typedef struct lqcd_field lqcd_field;
typedef struct lqcd_hmc_state lqcd_hmc_state;

/* ------------------------------------------------------------ library */

/* Message of the last failing call on this thread ("" if none). */
const char *lqcd_last_error(void);

/* Version string of the library. */
const char *lqcd_version(void);

/* Number of kernels this library has launched in this process (all threads). */
uint64_t lqcd_launch_count(void);

/* Kernel timers: while enabled, launches of the instrumented kernel classes
 * are bracketed by CUDA events recorded on the launching stream.  Classes:
 * "dslash_f64", "dslash_f32", "dslash_f16n", "dslash_bf16" (every half
 * hopping-term launch of that storage precision, fused epilogues included),
 * "dslash_df64" (the mixed solver's float-float residual products),
 * "gauge_force", "fermion_force", "link_update", and "dslash_f16n_plain" (the
 * plain FP16+norm hops alone, without fused epilogues; they are also counted
 * in "dslash_f16n").  Enabling clears the totals.
 * lqcd_kernel_timer_read synchronises the device, then returns the summed
 * event time in milliseconds, the number of launches of one class and, for the
 * hopping-term classes, the algorithmic bytes those launches move (every
 * link, input, output and fused-epilogue field element counted once; 0 for
 * the other classes).  Output pointers may be NULL. */
lqcd_status lqcd_kernel_timers(int enable);
/* The same with only the listed classes timed (comma-separated names; the
 * others run without events).  LQCD_EINVAL on an unknown name. */
lqcd_status lqcd_kernel_timers_only(const char *kernel_classes);
lqcd_status lqcd_kernel_timer_read(const char *kernel_class, double *total_ms, uint64_t *launches,
                                   double *algorithmic_bytes);
/* Sampling: while timers are enabled, time only one launch in every `every`
 * of each class (1, the default: all), counted from the last enable, so that
 * the events disturb a timed run less; the totals then cover the sampled
 * launches (launches and bytes count those, the averages stay per launch).
 * Pick `every` coprime to any period of the launch sequence (a CG iteration
 * cycles through four hopping-term variants).  LQCD_EINVAL if every < 1. */
lqcd_status lqcd_kernel_timers_every(int every);

/* Device allocator hook.  alloc(bytes, stream, ctx) returns device memory or
 * NULL; free(ptr, stream, ctx) releases it.  Passing NULL for both restores
 * cudaMalloc / cudaFree.  Fields remember the hook they were allocated with. */
typedef void *(*lqcd_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*lqcd_free_fn)(void *ptr, void *stream, void *ctx);
lqcd_status lqcd_set_allocator(lqcd_alloc_fn alloc, lqcd_free_fn free_fn, void *ctx);

/* ------------------------------------------------------------ fields */

/* Allocate a field on the current device (contents undefined).  The paper's
 * memory manager (Sec. 5) allocates device memory for a field on first use,
 * from a pool, and keeps it resident; here the caller allocates each field
 * once through the allocator hook and it stays resident until
 * lqcd_field_free. 
 *   kind/prec/link_recon combinations:
 *     LQCD_GAUGE:       (F64, 18) master links; (F32|F16N|BF16, 12) compressed
 *                       copies storing rows 0, 1 (row 2 = conj(row0 x row1)).
 *     LQCD_MOMENTUM:    (F64, 0)
 *     LQCD_SPINOR_EVEN/ODD: any precision, link_recon 0
 *     LQCD_SPINOR_FULL: (F64, 0)
 *   Device layout (structure of arrays, site index fastest, per parity):
 *     gauge F64   double2 [mu][parity][row*3+col][Vh]
 *     gauge 12    F32: float4 [mu][parity][3][Vh]; F16N/BF16: 4 halves [mu][parity][3][Vh]
 *     momentum    double  [mu][parity][a][Vh]
 *     spinor      F64: double2 [spin*3+col][Vh]; F32: float4 [6][Vh];
 *                 F16N: 8 halves [3][Vh] + float norm [Vh]; BF16: 8 halves [3][Vh]
 *     full spinor F64 [parity][12][Vh] double2
 * Errors: LQCD_EINVAL (bad lattice / combination), LQCD_ENOMEM. */
lqcd_status lqcd_field_alloc(const lqcd_lattice *lat, lqcd_kind kind, lqcd_prec prec, int link_recon,
                             lqcd_field **out);
/* Releases the field's device memory through the hook it was allocated with
 * (Sec. 5: the memory manager returns a field's memory to its pool). */
lqcd_status lqcd_field_free(lqcd_field *f);

/* Bytes of device memory the field holds. */
lqcd_status lqcd_field_bytes(const lqcd_field *f, size_t *bytes);

/* Device pointer of the field's main array (and of its norm array, NULL if
 * none), for callers that share memory with another library. */
lqcd_status lqcd_field_data(const lqcd_field *f, void **data_dev, void **norm_dev);

/* Host <-> device transfer of a field (Sec. 5: the memory manager moves a
 * field between host and device memory when a kernel needs it on the device
 * or the host reads it).  Copy a host array in the canonical FP64 layout into the field (converting
 * to the field's precision; gauge 12-real copies keep rows 0 and 1), or the
 * field out to such an array (compressed gauge fields are expanded by
 * reconstructing row 2).  Synchronous with respect to the host buffer: the
 * call returns after the copy completed.  Pinned (page-locked) host memory is
 * read or written directly by the converting kernel; pageable memory goes
 * through a temporary device buffer of the host array's size and one copy. */
lqcd_status lqcd_field_upload(lqcd_field *f, const double *host, void *stream);
lqcd_status lqcd_field_download(const lqcd_field *f, double *host, void *stream);

/* dst <- src for fields of the same kind and lattice, converting precision
 * (e.g. FP64 master links -> 12-real FP16 copy, FP64 spinor -> FP16+norm). */
lqcd_status lqcd_field_copy(lqcd_field *dst, const lqcd_field *src, void *stream);

/* ------------------------------------------------------------ RNG and refresh */

/* Raw Philox4x32-10 blocks: out_dev[4*i .. 4*i+3] = Philox(counter (c0 + i, c1,
 * c2, c3), key (key0, key1)) for i < n_blocks.  out_dev: device, 4*n_blocks
 * uint32. */
lqcd_status lqcd_philox_blocks(uint32_t *out_dev, size_t n_blocks, uint32_t c0, uint32_t c1, uint32_t c2,
                               uint32_t c3, uint32_t key0, uint32_t key1, void *stream);

/* The float-float codec of the mixed solver (the Krylov solver of Sec. 6; its
 * accurate residuals and solutions are held as unevaluated sums hi + lo of
 * two floats in place of FP64, see lqcd_cg_params) on n doubles: pairs_dev[2i] = hi =
 * RN_float(in[i]), pairs_dev[2i+1] = lo = RN_float(in[i] - hi), back_dev[i] =
 * RN_double(hi + lo), exactly as the FP64 operations would give them, computed
 * on the IEEE-754 bit patterns as the field conversions do.  All three arrays
 * on the device (n doubles, 2n floats, n doubles), caller-owned; NULL with
 * n > 0 is LQCD_EINVAL. */
lqcd_status lqcd_df_split(const double *in_dev, size_t n, float *pairs_dev, double *back_dev, void *stream);

/* Start configuration U_mu(x) = exp(i eps sum_a h_a T_a), h_a ~ N(0,1) from
 * Philox purpose 0 (counter (site, j, 0, 0), j = 0..15, Gaussians 2j, 2j+1 are
 * coefficient k = mu*8 + a; uniforms from 52-bit words, Box-Muller).
 * U: LQCD_GAUGE F64 18. */
lqcd_status lqcd_gauge_start(lqcd_field *U, uint32_t seed, uint32_t chain, double eps, void *stream);

/* Momentum refresh (paper Sec. 1, "momentum updates"): p_a ~ N(0,1), Philox
 * purpose 1, counter (site, j, 1, traj), same coefficient order as the start.
 * P: LQCD_MOMENTUM. */
lqcd_status lqcd_momentum_refresh(lqcd_field *P, uint32_t seed, uint32_t chain, uint32_t traj, void *stream);

/* Pseudofermion source eta on even sites (paper Sec. 1, "pseudofermion
 * refresh"): each real ~ N(0, 1/2), Philox purpose 2, counter (site, j, 2,
 * traj), j = 0..11, reals 2j, 2j+1 in [spin][colour][re,im] order.
 * eta: LQCD_SPINOR_EVEN F64.  (phi = Mhat^dag eta is lqcd_mhat with dagger.) */
lqcd_status lqcd_eta_refresh(lqcd_field *eta, uint32_t seed, uint32_t chain, uint32_t traj, void *stream);

/* ------------------------------------------------------------ operators */

/* Half hopping term of the Wilson operator (Sec. 6.2: the Nf = 2 Wilson
 * fermions of the paper's runs; Sec. 6: the even-odd preconditioned operator
 * whose inversion the paper hands to QUDA is Mhat = 1 - kappa^2 Deo Doe, built
 * from these two halves).
 * out = D_{p' p} in, p the parity of `in`, p' = 1 - p the
 * parity of `out` (EVEN/ODD kinds).  dagger != 0 applies D^dag = gamma5 D gamma5.
 * Precisions: U F64/18 with F64 spinors, or U 12-real of precision q with
 * spinors of precision q (q in F32, F16N, BF16; FP32 arithmetic). */
lqcd_status lqcd_dslash(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, int dagger, void *stream);

/* The FP16+norm hopping term comes in three forms:
 *   0  every operand gathered by its thread;
 *   1  each thread first starts asynchronous copies (cp.async) of its eight
 *      links into shared memory, then gathers the neighbour spinors and waits
 *      for each direction's links only when it needs them;
 *   2  (the default) form 1 with the two spin rows of every projected half
 *      spinor carried as pairs in Blackwell's packed FP32x2 instructions.
 * Forms 0 and 1 give bitwise the same results; form 2 rounds its products in
 * another order (agreement within FP32 rounding).  The multi-system solver
 * (lqcd_cg_solve_batch, batched chains, solve service) follows the setting.
 * lqcd_dslash_form(form) selects the form (0, 1, 2; a negative value queries)
 * and returns the previous one (process-wide); an unknown form returns -1,
 * leaves the setting unchanged and sets lqcd_last_error. */
int lqcd_dslash_form(int form);

/* out_e = Mhat in_e = in_e - kappa^2 Deo Doe in_e (dagger: Mhat^dag).  EVEN
 * spinors, precision rules as lqcd_dslash.  Uses one temporary odd spinor. */
lqcd_status lqcd_mhat(lqcd_field *out, const lqcd_field *U, const lqcd_field *in, double kappa, int dagger,
                      void *stream);

/* ------------------------------------------------------------ solver */

typedef struct {
    double tol;           /* stop when the true |r| <= tol |b| (r = b - Mhat^dag Mhat x) */
    int maxiter;          /* total iteration cap (LQCD_ENOCONV when reached) */
    lqcd_prec sloppy;     /* LQCD_F64: plain FP64 CG.  F32/F16N/BF16: reliable-update mixed
                             CG with that sloppy storage (FP32 arithmetic, FP64 sums of the dot
                             products).  Its accurate solution, source, links and residual are
                             held in float-float storage (a pair of FP32 numbers, ~48
                             significant bits) and the residual b - A x is recomputed and the
                             solution accumulated in float-float arithmetic, not FP64 */
    double delta;         /* reliable-update threshold: recompute the true residual when the
                             sloppy |r| drops below delta * max |r| since the last update */
    int max_restarts;     /* FP64 CG only: restarts allowed when the true residual fails */
    int guess;            /* 0: start from x0 = 0; 1: x holds the initial guess on entry (its
                             residual is recomputed accurately before the first iteration) */
} lqcd_cg_params;

typedef struct {
    int iters;            /* CG iterations (sloppy iterations for the mixed solver) */
    int restarts;         /* FP64 restarts / mixed reliable updates */
    double true_rel_res;  /* |b - A x| / |b| at exit, recomputed accurately: in FP64 by the FP64
                             solve; in float-float arithmetic (~48 bits) from the float-float
                             solution by the mixed solve (the FP64 x returned is that solution
                             rounded) */
    double seconds;       /* wall time of the call */
    int accurate_residuals; /* accurate (FP64 or float-float) residuals b - A x computed: of the
                               initial guess, at every reliable update or restart, at the end */
    int failed_checks;    /* times the iterated residual met the tolerance and the accurate one
                             did not (the solve then went on) */
    int guess_refined;    /* 1 if the initial guess was refined by minimal residual extrapolation */
} lqcd_cg_info;

/* Solve Mhat^dag Mhat x = b on the even sites (the matrix inversion of the
 * paper's Sec. 6, done there by QUDA), from x0 = 0 or from x (params->guess).  x, b: EVEN F64 spinors.
 * U: F64/18 master links; for a mixed solve also pass the sloppy 12-real
 * copy U_sloppy in the matching precision (NULL for FP64).
 * Returns LQCD_ENOCONV (x holds the last iterate) when maxiter is reached. */
lqcd_status lqcd_cg_solve(lqcd_field *x, const lqcd_field *U, const lqcd_field *U_sloppy, const lqcd_field *b,
                          double kappa, const lqcd_cg_params *params, lqcd_cg_info *info, void *stream);

/* ------------------------------------------------------------ forces and updates */

/* Gauge (staple) force with its traceless anti-Hermitian projection, fused
 * with the momentum update (paper Sec. 1, "force term calculation",
 * "projection of fields", "momentum updates"):
 *   F = -(i beta / 12) TA(U_mu(x) A_mu(x)), A the staple sum,
 *   TA(W) = (W - W^dag) - Tr(W - W^dag)/3,   P <- P - coeff * F (coefficients).
 * P: MOMENTUM, U: GAUGE F64/18. */
lqcd_status lqcd_gauge_force(lqcd_field *P, const lqcd_field *U, double beta, double coeff, void *stream);

/* The same with the arithmetic chosen: LQCD_F64, or LQCD_F32 (the links
 * rounded once to an FP32 12-real copy, FP32 staples, the increment added to
 * the FP64 momenta). */
lqcd_status lqcd_gauge_force_ex(lqcd_field *P, const lqcd_field *U, double beta, double coeff, lqcd_prec arith,
                                void *stream);

/* Two-flavour fermion force fused with the momentum update, given the even
 * solution X_e = (Mhat^dag Mhat)^-1 phi_e:
 *   Y_e = Mhat X_e, A = (X_e, Doe X_e), B = (Y_e, Deo^dag Y_e),
 *   Q1 = sum_spin [s U A(x+mu)] [(1 - gamma_mu) B(x)]^dag,
 *   Q2 = sum_spin A(x) [s U (1 + gamma_mu) B(x+mu)]^dag,
 *   F = (i kappa^2 / 2) TA(Q1 - Q2),  P <- P - coeff * F.
 * P: MOMENTUM, U: GAUGE F64/18, X_e: EVEN F64.  Uses three temporary spinors. */
lqcd_status lqcd_fermion_force(lqcd_field *P, const lqcd_field *U, const lqcd_field *X_e, double kappa,
                               double coeff, void *stream);

/* The same with the arithmetic chosen (LQCD_F64 or LQCD_F32: X_e and the
 * links rounded to FP32 (12-real links), the three hopping terms and the link
 * kernel in FP32, the increment added to the FP64 momenta). */
lqcd_status lqcd_fermion_force_ex(lqcd_field *P, const lqcd_field *U, const lqcd_field *X_e, double kappa,
                                  double coeff, lqcd_prec arith, void *stream);

/* SU(3) exponential link update (paper Sec. 1, "exponentiating of SU(3)
 * matrices"): U_mu(x) <- exp(i c P_mu(x)) U_mu(x), exp by Cayley-Hamilton
 * (Morningstar & Peardon 2004).  If U_sloppy is not NULL it receives the
 * 12-real copy of the new links in its precision. */
lqcd_status lqcd_link_update(lqcd_field *U, const lqcd_field *P, double c, lqcd_field *U_sloppy, void *stream);

/* The same with the arithmetic chosen: LQCD_F64 as lqcd_link_update;
 * LQCD_F32 (the FP32 molecular dynamics of lqcd_hmc_params.force_prec): the
 * exponential by Cayley-Hamilton in FP32, re-unitarized (Gram-Schmidt) and
 * multiplied onto the FP64 links in float-float arithmetic, so the new links
 * differ from exp(i c P) U by the FP32 exponential's error (~1e-7) but stay in
 * SU(3) to ~1e-14. */
lqcd_status lqcd_link_update_ex(lqcd_field *U, const lqcd_field *P, double c, lqcd_field *U_sloppy, lqcd_prec arith,
                                void *stream);

/* Reunitarization (paper Sec. 1): rows 0, 1 by Gram-Schmidt, row 2 =
 * conj(row0 x row1).  max_dev_out (host, may be NULL) receives the maximum
 * over links of max_ij |(U U^dag - 1)_ij| before the projection. */
lqcd_status lqcd_reunitarize(lqcd_field *U, double *max_dev_out, void *stream);

/* ------------------------------------------------------------ reductions (Sec. 1, `sum`) */

/* Mean plaquette (1/6V) sum_x sum_{mu<nu} Re Tr U_munu(x) / 3 (FP64,
 * deterministic fixed-order reduction).  out: host. */
lqcd_status lqcd_plaquette(const lqcd_field *U, double *out, void *stream);

/* Kinetic energy 1/2 sum p_a^2.  out: host. */
lqcd_status lqcd_kinetic_energy(const lqcd_field *P, double *out, void *stream);

/* Re <a, b> = sum of products of the reals of two FP64 spinor fields of the
 * same kind.  out: host. */
lqcd_status lqcd_spinor_dot(const lqcd_field *a, const lqcd_field *b, double *out, void *stream);

/* ------------------------------------------------------------ autotuning (paper Sec. 4) */

/* The paper times each generated kernel over its threads-per-block settings on
 * first use and keeps the fastest (Sec. 4).  Here that is an explicit call:
 * lqcd_autotune times, on scratch fields of the lattice (allocated and freed
 * inside), every candidate block size of the kernel classes whose launch shape
 * is free -- "dslash_f16n" (the packed FP16+norm hopping term: 64, 128, 256,
 * timed as the solver uses it, one application of Mhat^dag Mhat: two plain
 * hops and two with the fused axpy and norm reduction, whose last block sums
 * the block partials),
 * "gauge_force_f32", "gauge_force_f64" and "link_update_f32" (32 to 256),
 * "fermion_force_f32" (32 to 128) -- keeps the fastest of each in a
 * process-wide table keyed by (kernel class, lattice dims) that every later
 * launch on that lattice reads, and writes all timings to the text file path
 * (lines "class Lx Ly Lz Lt block ms_per_launch best"; NULL: no file).
 * Synchronises stream.  Results do not depend on the block size of the force
 * and link-update kernels; the hopping term's block size sets the order of
 * its block sums, so a tuned size other than 128 changes the solver's
 * rounding (the multi-system solver always uses 128).
 * lqcd_autotune_load reads such a file into the table; lqcd_autotune_block
 * returns a class's block size for a lattice (0: not tuned, the default
 * applies); lqcd_autotune_clear empties the table. */
lqcd_status lqcd_autotune(const lqcd_lattice *lat, const char *path, void *stream);
lqcd_status lqcd_autotune_load(const char *path);
lqcd_status lqcd_autotune_block(const char *kernel_class, const lqcd_lattice *lat, int *block);
lqcd_status lqcd_autotune_clear(void);

/* ------------------------------------------------------------ allocation-free plaquette */

/* Largest lattice (sites) lqcd_plaquette_noalloc accepts. */
#define LQCD_NOALLOC_MAX_SITES 16777216

/* Mean plaquette like lqcd_plaquette, for callers that cannot let the library
 * allocate device memory: code on a thread that must not call back into the
 * allocator hook (for instance a hook that enters the Python interpreter), or
 * a program that fixes its device memory up front.  The paper has no
 * counterpart of this call.
 *   U       F64 gauge field of at most LQCD_NOALLOC_MAX_SITES sites; larger
 *           lattices return LQCD_EINVAL (use lqcd_plaquette).
 *   out_dev device pointer to one double, written asynchronously on stream.
 * It allocates nothing: the per-block partial sums live in one fixed array of
 * LQCD_NOALLOC_MAX_SITES/256 doubles (512 KiB) per device, held by every
 * device that loads the library until the process exits.  The first call on a
 * device looks up that array's device address; make that first call before
 * any stream capture.  All calls on a device share the array and each call
 * overwrites the part it reads, so calls whose kernels may overlap on the
 * device (different streams without ordering) race and must be serialised by
 * the caller. */
lqcd_status lqcd_plaquette_noalloc(const lqcd_field *U, double *out_dev, void *stream);

/* ------------------------------------------------------------ HMC driver */

typedef struct {
    double beta, kappa, tau;
    int nsteps;
    lqcd_integrator integrator; /* leapfrog or Omelyan 2MN (lambda = 0.1931833275037836) */
    int n_flavors;              /* 0: pure gauge, 2: two Wilson flavours */
    lqcd_cg_params cg;          /* solver of every force and action evaluation */
    int reunitarize;            /* 1: reunitarize the links after the accept/reject */
    int metropolis;             /* 1: accept iff u < exp(-dH); 0: always accept */
    int chrono;                 /* chronological initial guess (paper Sec. 6.2) for every solve after
                                   the first of a trajectory: 0 none (x0 = 0); 1 the previous
                                   solution; k = 2..4 the polynomial through the last k solutions
                                   at their molecular-dynamics times, extrapolated to the current
                                   time (a solve at the previous solve's time starts from its
                                   solution).  Reversibility then holds to the solver tolerance only */
    lqcd_prec force_prec;       /* arithmetic of the molecular dynamics: LQCD_F64, or LQCD_F32: both
                                   forces in FP32 from an FP32 12-real copy of the links (increments
                                   accumulated into the FP64 momenta) and the link update's
                                   exponential by Cayley-Hamilton in FP32, re-unitarized and
                                   multiplied onto the FP64 links in float-float arithmetic
                                   (~48 bits: the links stay in SU(3) to ~1e-14 per update) */
    double hasenbusch_kappa;    /* 0: one pseudofermion with Mhat(kappa).  In (0, kappa): mass
                                   preconditioning (paper Sec. 6.2) with W = Mhat(hasenbusch_kappa):
                                   a heavy action phi_h^dag (W^dag W)^-1 phi_h and a ratio action
                                   chi^dag (Mhat^dag Mhat)^-1 chi, chi = W^dag phi; refresh
                                   phi_h = W^dag eta_h (eta_h from Philox purpose 4) and
                                   phi = W (W^dag W)^-1 Mhat^dag eta (one solve) */
    int gauge_substeps;         /* <= 1: every force on one time scale.  m >= 2: nested integration
                                   (Sexton-Weingarten): the gauge force (and the heavy action if
                                   heavy_inner) on an inner level integrating each drift of the
                                   outer level in m steps of the same scheme; the fermion actions
                                   on the outer level of nsteps steps */
    int heavy_inner;            /* with gauge_substeps >= 2: the heavy action on the inner level */
    int chrono_mre;             /* with chrono = k >= 2 and a mixed-precision solver: 1 refines the
                                   extrapolated guess by minimal residual extrapolation (paper Sec.
                                   6.2, the chronological inverter of its production runs): the guess
                                   x_L + sum_j c_j (x_j - x_{j+1}) over the last k solutions x_j whose
                                   real coefficients c minimise |b - A x| for the current operator A;
                                   the products A (x_j - x_{j+1}) in FP32 arithmetic, the residual of
                                   x_L and the update in float-float.  0: the extrapolation alone */
} lqcd_hmc_params;

typedef struct {
    double dH, H0, H1;
    double plaq;               /* after the trajectory (and reunitarization) */
    double u;                  /* Metropolis uniform */
    double max_unitarity_dev;  /* before reunitarization */
    double seconds;
    double cg_true_rel_res_max;
    int accepted;
    int cg_iters;              /* summed over all solves of the trajectory */
    int n_solves;
    int cg_failures;
    uint32_t traj;             /* trajectory counter used for the random numbers */
    int cg_accurate_residuals; /* summed lqcd_cg_info.accurate_residuals of the solves */
    int cg_failed_checks;      /* summed lqcd_cg_info.failed_checks of the solves */
    int cg_guesses_refined;    /* solves whose guess minimal residual extrapolation refined */
} lqcd_traj_info;

/* State of one Markov chain on the device: borrows the caller's FP64 gauge
 * field U (updated in place) and owns the momenta, pseudofermion fields, the
 * backup of U, the sloppy link copy and the solver work space.
 * seed/chain form the Philox key; traj0 is the first trajectory counter. */
lqcd_status lqcd_hmc_state_create(lqcd_field *U, uint32_t seed, uint32_t chain, uint32_t traj0,
                                  lqcd_hmc_state **out);
lqcd_status lqcd_hmc_state_destroy(lqcd_hmc_state *s);

/* Accessors for tests and checkpointing: the borrowed links, the momenta and
 * phi_e; the trajectory counter (read, and set for resume). */
lqcd_status lqcd_hmc_state_fields(lqcd_hmc_state *s, lqcd_field **U, lqcd_field **P, lqcd_field **phi);
lqcd_status lqcd_hmc_state_traj(lqcd_hmc_state *s, uint32_t *traj_out, const uint32_t *traj_in);

/* Refresh of the state for its current trajectory counter: momenta, eta and
 * phi_e = Mhat^dag eta_e; H0 (host, may be NULL) = T + S_g + eta^dag eta. */
lqcd_status lqcd_hmc_refresh(lqcd_hmc_state *s, const lqcd_hmc_params *p, double *H0, void *stream);

/* H = T + S_g + S_f for the state's current (U, P, phi) (S_f by a CG solve). */
lqcd_status lqcd_hmc_hamiltonian(lqcd_hmc_state *s, const lqcd_hmc_params *p, double *H, void *stream);

/* One molecular-dynamics step (Sec. 1: the momentum updates with their force
 * terms, and the link update by the exponential of SU(3) matrices, are among
 * the HMC parts the paper moves to the GPU) of length tau/nsteps with the state's phi, as
 * a whole step (leapfrog: kick dt/2, drift dt, kick dt/2; Omelyan:
 * lambda dt, dt/2, (1-2 lambda) dt, dt/2, lambda dt). */
lqcd_status lqcd_md_step(lqcd_hmc_state *s, const lqcd_hmc_params *p, void *stream);

/* One full trajectory (paper Sec. 1 and 6.2): refresh, nsteps MD steps with
 * adjacent kicks merged, H1, Metropolis with u from Philox purpose 3 counter
 * (0, 0, 3, traj), restore U on reject, optional reunitarization, plaquette.
 * Increments the state's trajectory counter.  info: host. */
lqcd_status lqcd_hmc_trajectory(lqcd_hmc_state *s, const lqcd_hmc_params *p, lqcd_traj_info *info,
                                void *stream);

/* ------------------------------------------------------------ batched solves and chains */

/* n independent mixed-precision solves Mhat^dag Mhat x[i] = b[i] (each on its
 * own lattice, links U[i] with sloppy copy U_sloppy[i], kappa[i]) with shared
 * launches: every kernel of a CG iteration covers all systems that have not
 * converged, each system reading its own geometry, fields and scalars.  Each
 * system's iterates equal those of lqcd_cg_solve on it alone.  params (one
 * for all) must be mixed precision (sloppy F32, F16N or BF16); info[i]
 * receives system i's result.  Returns the first non-OK status of a system
 * (LQCD_ENOCONV if one hit maxiter) after all finished.  Small lattices, each
 * filling a few SMs alone, fill the GPU together. */
lqcd_status lqcd_cg_solve_batch(int n, lqcd_field *const *x, const lqcd_field *const *U,
                                const lqcd_field *const *U_sloppy, const lqcd_field *const *b, const double *kappa,
                                const lqcd_cg_params *params, lqcd_cg_info *info, void *stream);

/* A batch of independent Markov chains (each an lqcd_hmc_state, on lattices of
 * any size) advanced together: per molecular-dynamics force evaluation every
 * chain's solve runs in shared launches (lqcd_cg_solve_batch's engine, each
 * chunk of iterations replayed as a CUDA graph).  The batch borrows the states;
 * they must outlive it. */
typedef struct lqcd_batch lqcd_batch;
lqcd_status lqcd_batch_create(lqcd_hmc_state *const *chains, int n, lqcd_batch **out);
lqcd_status lqcd_batch_destroy(lqcd_batch *batch);

/* One trajectory of every chain; params[i] and info[i] belong to chain i.  All
 * chains must share integrator, nsteps, tau, solver and force precision (beta,
 * kappa, seeds differ freely), have two flavours and a mixed-precision solver.
 * Each chain's trajectory equals lqcd_hmc_trajectory on that chain alone. */
lqcd_status lqcd_batch_trajectory(lqcd_batch *batch, const lqcd_hmc_params *params, lqcd_traj_info *info,
                                  void *stream);

/* ------------------------------------------------------------ solve service */

/* A service for solves of the full Wilson-Dirac operator, M x = b with
 * M = 1 - kappa D, on gauge fields kept resident on the device.  Requests are
 * submitted at any time from any host thread and run on a worker thread of the
 * service with its own stream: it admits queued requests in arrival order
 * while the device memory of the admitted work, the unreleased solutions and
 * the pooled idle solver work spaces fits hbm_budget (a request alone is
 * always admitted; idle work spaces are freed to make room), and advances all admitted right-hand sides
 * together, one chunk of CG iterations at a time, in shared launches (the
 * engine of lqcd_cg_solve_batch); right-hand sides join and leave between
 * chunks (continuous batching).  The paper keeps all fields resident and
 * manages device memory itself (Sec. 5); admission by footprint is this
 * library's analogue for many concurrent solves.
 *
 * Each right-hand side is even-odd reduced: b'_e = b_e + kappa D_eo b_o,
 * Mhat^dag Mhat x_e = Mhat^dag b'_e by the mixed-precision CG of
 * lqcd_cg_solve, x_o = b_o + kappa D_oe x_e.  The residual reported is that of
 * the full operator, |b - M x| / |b|, recomputed in FP64 after the
 * reconstruction; if it is above cg.tol the solve continues from x_e with a
 * tighter normal-equation tolerance (at most 3 times, then LQCD_ENOCONV).
 * Each right-hand side's result does not depend on what else runs with it. */
typedef struct lqcd_service lqcd_service;

typedef struct {
    lqcd_cg_params cg;  /* tol = target full |r|/|b|; sloppy F32, F16N or BF16; guess ignored */
    size_t hbm_budget;  /* device bytes for admitted requests, unreleased solutions, idle work spaces */
    int max_active_rhs; /* admit no request that would make more right-hand sides run at once (<= 0: no limit) */
} lqcd_service_params;

/* A point-source request: nrhs unit sources b = delta(x, site) delta(spin*3 +
 * colour, k) for k = 0 .. nrhs-1 (nrhs <= 12, the spin-colour components in
 * order). */
typedef struct {
    int gauge;    /* id from lqcd_service_add_gauge */
    double kappa;
    int site[4];  /* x, y, z, t of the source */
    int nrhs;     /* 1 .. 12 */
} lqcd_solve_req;

typedef struct {
    lqcd_status status;      /* first non-OK status of a right-hand side, else LQCD_OK */
    int nrhs;
    int iters;               /* CG iterations summed over the right-hand sides */
    int refinements;         /* continuations after a full-residual miss, summed */
    double true_rel_res_max; /* max over the right-hand sides of |b - M x| / |b| */
    double queue_s;          /* submit -> admission, seconds (host clock) */
    double latency_s;        /* submit -> result, seconds (host clock) */
} lqcd_solve_result;

/* Creates a service on the current device and starts its worker thread. */
lqcd_status lqcd_service_create(const lqcd_service_params *params, lqcd_service **out);
/* Registers an F64 gauge field (borrowed: it must outlive the service and not
 * change while the service exists); *id receives its id.  Its sloppy and
 * float-float link copies are made on the first request that uses it. */
lqcd_status lqcd_service_add_gauge(lqcd_service *svc, lqcd_field *U, int *id);
/* Queues a request; *ticket identifies it.  Returns at once. */
lqcd_status lqcd_solve_submit(lqcd_service *svc, const lqcd_solve_req *req, uint64_t *ticket);
/* LQCD_EAGAIN while the request runs; LQCD_OK with *result once done (the
 * request's own failure is in result->status). */
lqcd_status lqcd_solve_poll(lqcd_service *svc, uint64_t ticket, lqcd_solve_result *result);
/* The solution halves x_e, x_o (F64 fields owned by the service) of
 * right-hand side k of a finished request, valid until lqcd_solve_release. */
lqcd_status lqcd_solve_solution(lqcd_service *svc, uint64_t ticket, int k, lqcd_field **x_even,
                                lqcd_field **x_odd);
/* Frees a finished request's solutions (LQCD_EAGAIN while it runs). */
lqcd_status lqcd_solve_release(lqcd_service *svc, uint64_t ticket);
/* Device bytes the service holds: *counted = what hbm_budget covers (the
 * admitted right-hand sides, the solutions not yet released and the idle
 * solver work spaces pooled for reuse); *fixed = what each gauge field holds
 * once it has served a request (its sloppy and float-float link copies and
 * the temporaries its solves share), outside the budget. */
lqcd_status lqcd_service_bytes(lqcd_service *svc, size_t *counted, size_t *fixed);
/* Finishes all submitted requests, stops the worker and frees everything. */
lqcd_status lqcd_service_destroy(lqcd_service *svc);

#ifdef __cplusplus
}
#endif

#endif /* LQCD_H */
