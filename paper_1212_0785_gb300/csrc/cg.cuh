// cg.cuh -- CG work space shared between the solver and the HMC driver.
#pragma once

#include <chrono>

#include "dslash.cuh"

namespace lqcd {

// threads per block of the solver's vector kernels (its block partial sums
// are laid out by it)
constexpr int CG_BLOCK = 256;

// Fields and scalars of one solver, reusable across solves on one lattice.
struct CgWorkspace {
    lqcd_lattice lat{};
    lqcd_prec sloppy = LQCD_F64;
    bool ready = false;
    int mre_n = 0; // directions allocated
    FieldPtr r64, t64a, t64b, tmpo64;  // FP64 residual and operator temporaries (FP64 CG)
    FieldPtr p64;                      // FP64 search direction (plain FP64 CG)
    FieldPtr xs, rs, ps, ts, tmpos;    // sloppy fields (mixed CG)
    // mixed CG: the accurate solution, source, residual and operator
    // temporaries in float-float storage, and the float-float link copy
    FieldPtr Udf, xdf, bdf, rdf, t1df, tmpodf;
    // bdf holds the float-float copy of the source b with stamp bdf_stamp
    // (0: none), so repeated solves of an unchanged source skip the split
    const lqcd_field *bdf_of = nullptr;
    uint64_t bdf_stamp = 0;
    DevBuf sc, partials, scalars;
    // minimal residual extrapolation of the guess (mixed solves): FP32
    // directions d_j, their images w_j = A d_j and the operator temporaries
    static constexpr int MRE_MAX = 3;
    FieldPtr mre_d[MRE_MAX], mre_w[MRE_MAX], mre_te, mre_to;
    DevBuf mre_tab; // device table of the d_j and w_j pointers
    lqcd_status ensure_mre(int n, cudaStream_t s);
    // Optional sharing for many right-hand sides on one lattice: the
    // float-float links kept current by the owner (no per-solve split), and
    // the transient float-float fields of another workspace (used only while a
    // pause is handled, which the owner serialises on one stream).
    const lqcd_field *udf_ext = nullptr;
    CgWorkspace *tmp_from = nullptr;
    bool temps_only = false; // allocate only the transient float-float fields (a tmp_from owner)
    const lqcd_field *udf() const { return udf_ext ? udf_ext : Udf.f; }
    lqcd_field *rdf_() const { return tmp_from ? tmp_from->rdf.f : rdf.f; }
    lqcd_field *t1() const { return tmp_from ? tmp_from->t1df.f : t1df.f; }
    lqcd_field *tmpo() const { return tmp_from ? tmp_from->tmpodf.f : tmpodf.f; }
    lqcd_status ensure(const lqcd_lattice &lat, lqcd_prec sloppy, cudaStream_t s);
    size_t bytes() const;
};

// One solve as a resumable state machine: start() does everything before the
// first iteration, iterate() enqueues one iteration (no-op kernels while the
// device pause flag is set), on_pause() handles a pause read back from the
// device (reliable update, true-residual check, convergence, maxiter).  The
// single-system solve loops over it; the multi-system solver (batch.cu) runs
// many of them with shared launches.
struct CgRun {
    // inputs
    CgWorkspace *ws = nullptr;
    lqcd_field *x = nullptr;
    const lqcd_field *U = nullptr, *Us = nullptr, *b = nullptr;
    double kappa = 0;
    lqcd_cg_params prm{};
    // nonzero: a stamp of b's contents, new whenever they change; a solve of
    // the same b and stamp as the workspace's last reuses its float-float copy
    uint64_t b_stamp = 0;
    // optional minimal residual extrapolation of a mixed solve's guess x:
    // the last n_mre solutions (latest first, FP64), on links mre_links
    // (an FP32 12-real copy, or the FP64 links) for the FP32 products
    const lqcd_field *mre_x[CgWorkspace::MRE_MAX + 1] = {};
    int n_mre = 0;
    const lqcd_field *mre_links = nullptr;
    bool mre_used = false; // the guess was refined
    // state
    bool mixed = false, done = false;
    lqcd_status status = LQCD_OK;
    double bb = 0, rr_true = 0, k2 = 0;
    int Vh = 0;
    lqcd_field *P = nullptr, *R = nullptr, *T = nullptr, *TMP = nullptr, *XS = nullptr;
    const lqcd_field *UU = nullptr;
    CgScalars *sc = nullptr; // device scalars of this solve
    CgScalars h0{};
    lqcd_cg_info inf{};
    std::chrono::steady_clock::time_point t0;

    lqcd_status start(cudaStream_t s, CgScalars *sc_dev);
    lqcd_status iterate(cudaStream_t s);
    lqcd_status on_pause(const CgScalars &h, cudaStream_t s);
    // a mixed solve's pause in two halves, so that many solves' accurate
    // residuals can be enqueued before one read-back: pause_begin enqueues
    // (unless it fails: then done), pause_result_dev is where |r|^2 lands,
    // pause_end takes it and finishes the pause
    lqcd_status pause_begin(const CgScalars &h, cudaStream_t s);
    double *pause_result_dev() const;
    lqcd_status pause_end(double rr, cudaStream_t s);
    // pause_begin without its kernels, for a caller that runs them for many
    // solves at once (batch.cu); false if the pause failed the solve
    bool pause_record(const CgScalars &h);
    lqcd_status fail(lqcd_status st);
    lqcd_status succeed();

  private:
    CgScalars hp{}; // the pause being handled
    lqcd_status start_impl(cudaStream_t s);
    lqcd_status mre_refine(cudaStream_t s, double *rr0);
    lqcd_status on_pause_impl(const CgScalars &h, cudaStream_t s);
    lqcd_status pause_decide(const CgScalars &h, cudaStream_t s);
};

lqcd_status split_links(lqcd_field *Udf, const lqcd_field *U, cudaStream_t s);
// FP64 copy of a float-float spinor field (rounded hi + lo)
lqcd_status df_to_f64(lqcd_field *dst, const lqcd_field *src_df, cudaStream_t s);

// mre (optional): the minimal residual extrapolation inputs of CgRun
struct MreInput {
    const lqcd_field *x[CgWorkspace::MRE_MAX + 1] = {};
    int n = 0;
    const lqcd_field *links = nullptr;
};
lqcd_status cg_solve_ws(CgWorkspace &ws, lqcd_field *x, const lqcd_field *U, const lqcd_field *Us,
                        const lqcd_field *b, double kappa, const lqcd_cg_params &prm, lqcd_cg_info *info,
                        cudaStream_t s, const MreInput *mre = nullptr, uint64_t b_stamp = 0);
// a stamp never handed out before (for CgRun::b_stamp)
uint64_t new_content_stamp();

// |v|^2 and Re<a,b> of FP64 fields into a device double (deterministic)
lqcd_status spinor_dot_dev(const lqcd_field *a, const lqcd_field *b, double *dst_dev, DevBuf &part, cudaStream_t s);

} // namespace lqcd
