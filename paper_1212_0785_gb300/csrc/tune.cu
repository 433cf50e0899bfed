// tune.cu -- the threads-per-block table and the tuning runs (tune.cuh).
#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cg.cuh"
#include "tune.cuh"

namespace lqcd {

// launchers with an explicit block size (dslash.cu, force.cu, field.cu)
int dslash_packed_block_override(int block); // 0: the table's choice
lqcd_status gauge_force_block(lqcd_field *P, const lqcd_field *U, const lqcd_field *Uf, double cf, lqcd_prec arith,
                              int block, cudaStream_t s);
lqcd_status fermion_force_link_block(lqcd_field *P, const lqcd_field *Uf, const lqcd_field *Xe, const lqcd_field *Ao,
                                     const lqcd_field *Ye, const lqcd_field *Bo, double cf, int block, cudaStream_t s);
lqcd_status link_update_block(lqcd_field *U, const lqcd_field *P, double c, lqcd_field *Us, lqcd_field *Uf,
                              lqcd_field *Udf, int block, cudaStream_t s);

static const char *const NAMES[TK_NKERNEL] = {"dslash_f16n", "gauge_force_f32", "gauge_force_f64",
                                              "fermion_force_f32", "link_update_f32"};
// candidate threads per block: the hopping term's shared-memory layout is
// compiled for 64, 128 and 256; the others take any multiple of 32 up to
// their launch bound (the fermion force's staged operands take 336 bytes of
// shared memory per thread, so at most 128)
static const std::vector<int> CANDIDATES[TK_NKERNEL] = {
    {64, 128, 256}, {32, 64, 96, 128, 192, 256}, {32, 64, 96, 128, 192, 256}, {32, 64, 96, 128},
    {32, 64, 96, 128, 192, 256}};

struct TuneEntry {
    int block = 0;
    std::vector<std::pair<int, double>> ms; // (block, time per launch)
};
using TuneKey = std::pair<int, std::array<int, 4>>;
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneEntry> g_tune;

const char *tune_kernel_name(int k) { return k >= 0 && k < TK_NKERNEL ? NAMES[k] : "?"; }

int tuned_block(int k, const lqcd_lattice &lat, int dflt)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(TuneKey{k, {lat.dims[0], lat.dims[1], lat.dims[2], lat.dims[3]}});
    return it == g_tune.end() ? dflt : it->second.block;
}

static int kernel_id(const char *name)
{
    for (int k = 0; k < TK_NKERNEL; k++)
        if (name && !std::strcmp(name, NAMES[k])) return k;
    return -1;
}

// time per launch of f(block) in ms: 3 warm-up launches, then the median of
// 3 repetitions of 10 launches bracketed by events on s
template <class F>
static lqcd_status time_launches(F f, int block, cudaStream_t s, double *ms)
{
    cudaEvent_t a, b;
    LQCD_CUDA(cudaEventCreate(&a));
    LQCD_CUDA(cudaEventCreate(&b));
    lqcd_status rc = LQCD_OK;
    double t[3] = {0, 0, 0};
    for (int w = 0; w < 3 && rc == LQCD_OK; w++) rc = f(block);
    for (int r = 0; r < 3 && rc == LQCD_OK; r++) {
        cudaEventRecord(a, s);
        for (int k = 0; k < 10 && rc == LQCD_OK; k++) rc = f(block);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float e = 0.f;
        cudaEventElapsedTime(&e, a, b);
        t[r] = e / 10.0;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::sort(t, t + 3);
    *ms = t[1];
    return rc;
}

// per_call: kernel launches f makes (the table stores time per launch)
template <class F>
static lqcd_status tune_one(int k, const lqcd_lattice &lat, F f, cudaStream_t s, int per_call = 1)
{
    TuneEntry e;
    double best = 0;
    for (int block : CANDIDATES[k]) {
        double ms = 0;
        LQCD_TRY(time_launches(f, block, s, &ms));
        ms /= per_call;
        e.ms.emplace_back(block, ms);
        if (e.block == 0 || ms < best) e.block = block, best = ms;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[TuneKey{k, {lat.dims[0], lat.dims[1], lat.dims[2], lat.dims[3]}}] = e;
    return LQCD_OK;
}

static lqcd_status save_table(const char *path)
{
    FILE *fp = std::fopen(path, "w");
    LQCD_REQUIRE(fp != nullptr, "autotune: cannot write %s", path);
    std::fprintf(fp, "# kernel Lx Ly Lz Lt block ms_per_launch best\n");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto &kv : g_tune)
        for (const auto &bm : kv.second.ms)
            std::fprintf(fp, "%s %d %d %d %d %d %.6f %d\n", NAMES[kv.first.first], kv.first.second[0],
                         kv.first.second[1], kv.first.second[2], kv.first.second[3], bm.first, bm.second,
                         bm.first == kv.second.block ? 1 : 0);
    std::fclose(fp);
    return LQCD_OK;
}

} // namespace lqcd

using namespace lqcd;

extern "C" {

lqcd_status lqcd_autotune(const lqcd_lattice *lat, const char *path, void *stream)
{
    LQCD_TRY(check_lattice(lat));
    cudaStream_t s = (cudaStream_t)stream;
    // scratch fields of the lattice: the start configuration, its FP32, FP16
    // and float-float copies, momenta and spinors
    FieldPtr U, Uf, Us, Udf, P, Xe, Ao, Ye, Bo, he, ho;
    LQCD_TRY(lqcd_field_alloc(lat, LQCD_GAUGE, LQCD_F64, 18, &U.f));
    LQCD_TRY(lqcd_gauge_start(U.f, 1, 0, 0.3, s));
    LQCD_TRY(lqcd_field_alloc(lat, LQCD_GAUGE, LQCD_F32, 12, &Uf.f));
    LQCD_TRY(lqcd_field_copy(Uf.f, U.f, s));
    LQCD_TRY(lqcd_field_alloc(lat, LQCD_GAUGE, LQCD_F16N, 12, &Us.f));
    LQCD_TRY(lqcd_field_copy(Us.f, U.f, s));
    LQCD_TRY(field_alloc_df(lat, LQCD_GAUGE, &Udf.f));
    LQCD_TRY(split_links(Udf.f, U.f, s));
    LQCD_TRY(lqcd_field_alloc(lat, LQCD_MOMENTUM, LQCD_F64, 0, &P.f));
    LQCD_TRY(lqcd_momentum_refresh(P.f, 1, 0, 0, s));
    LQCD_TRY(lqcd_field_alloc(lat, LQCD_SPINOR_EVEN, LQCD_F64, 0, &he.f));
    LQCD_TRY(lqcd_eta_refresh(he.f, 1, 0, 0, s));
    LQCD_TRY(lqcd_field_alloc(lat, LQCD_SPINOR_EVEN, LQCD_F32, 0, &Xe.f));
    LQCD_TRY(lqcd_field_copy(Xe.f, he.f, s));
    LQCD_TRY(lqcd_field_alloc(lat, LQCD_SPINOR_ODD, LQCD_F32, 0, &Ao.f));
    LQCD_TRY(lqcd_field_alloc(lat, LQCD_SPINOR_EVEN, LQCD_F32, 0, &Ye.f));
    LQCD_TRY(lqcd_field_alloc(lat, LQCD_SPINOR_ODD, LQCD_F32, 0, &Bo.f));
    LQCD_TRY(lqcd_dslash(Ao.f, Uf.f, Xe.f, 0, s));
    LQCD_TRY(lqcd_field_copy(Ye.f, Xe.f, s));
    LQCD_TRY(lqcd_dslash(Bo.f, Uf.f, Ye.f, 1, s));
    // the FP16+norm hopping term is timed as the solver uses it: one
    // application of Mhat^dag Mhat, two plain hops and two with the fused
    // axpy and norm reduction whose last block sums the block partials
    // (cg_finish into scratch scalars; time per hop = a quarter of it)
    FieldPtr p16, o16, t16, u16;
    DevBuf part, fin;
    LQCD_TRY(lqcd_field_alloc(lat, LQCD_SPINOR_EVEN, LQCD_F16N, 0, &p16.f));
    LQCD_TRY(lqcd_field_copy(p16.f, he.f, s));
    LQCD_TRY(lqcd_field_alloc(lat, LQCD_SPINOR_ODD, LQCD_F16N, 0, &o16.f));
    LQCD_TRY(lqcd_field_alloc(lat, LQCD_SPINOR_EVEN, LQCD_F16N, 0, &t16.f));
    LQCD_TRY(lqcd_field_alloc(lat, LQCD_SPINOR_EVEN, LQCD_F16N, 0, &u16.f));
    LQCD_TRY(part.alloc(sizeof(double) * (size_t)nblocks_for(make_geo(*lat).Vh, 64), s));
    LQCD_TRY(fin.alloc(sizeof(CgScalars), s));
    LQCD_CUDA(cudaMemsetAsync(fin.p, 0, sizeof(CgScalars), s));
    const int prev_form = dslash_form_set(2);
    const double k2 = 0.15 * 0.15;
    lqcd_status rc = tune_one(TK_HOP_F16N, *lat, [&](int b) {
        dslash_packed_block_override(b);
        double *pp = (double *)part.p;
        CgScalars *fs = (CgScalars *)fin.p;
        lqcd_status r = dslash_plain(o16.f, Us.f, p16.f, 0, nullptr, s);
        if (r == LQCD_OK) r = dslash_xpay(t16.f, Us.f, o16.f, 0, p16.f, -k2, pp, nullptr, s, fs);
        if (r == LQCD_OK) r = dslash_plain(o16.f, Us.f, t16.f, 1, nullptr, s);
        if (r == LQCD_OK) r = dslash_xpay(u16.f, Us.f, o16.f, 1, t16.f, -k2, pp, nullptr, s, fs);
        dslash_packed_block_override(0);
        return r;
    }, s, 4);
    dslash_form_set(prev_form);
    LQCD_TRY(rc);
    LQCD_TRY(tune_one(TK_GAUGE_FORCE_F32, *lat,
                      [&](int b) { return gauge_force_block(P.f, U.f, Uf.f, 1e-3, LQCD_F32, b, s); }, s));
    LQCD_TRY(tune_one(TK_GAUGE_FORCE_F64, *lat,
                      [&](int b) { return gauge_force_block(P.f, U.f, nullptr, 1e-3, LQCD_F64, b, s); }, s));
    LQCD_TRY(tune_one(TK_FERMION_FORCE_F32, *lat, [&](int b) {
        return fermion_force_link_block(P.f, Uf.f, Xe.f, Ao.f, Ye.f, Bo.f, 1e-3, b, s);
    }, s));
    LQCD_TRY(tune_one(TK_LINK_UPDATE_F32, *lat,
                      [&](int b) { return link_update_block(U.f, P.f, 1e-4, Us.f, Uf.f, Udf.f, b, s); }, s));
    LQCD_CUDA(cudaStreamSynchronize(s));
    if (path && *path) LQCD_TRY(save_table(path));
    return LQCD_OK;
}

lqcd_status lqcd_autotune_load(const char *path)
{
    LQCD_REQUIRE(path != nullptr, "autotune_load: NULL path");
    FILE *fp = std::fopen(path, "r");
    LQCD_REQUIRE(fp != nullptr, "autotune_load: cannot read %s", path);
    char line[256], name[64];
    std::map<TuneKey, TuneEntry> loaded;
    while (std::fgets(line, sizeof line, fp)) {
        if (line[0] == '#') continue;
        int L[4], block, best;
        double ms;
        if (std::sscanf(line, "%63s %d %d %d %d %d %lf %d", name, &L[0], &L[1], &L[2], &L[3], &block, &ms, &best) != 8)
            continue;
        const int k = kernel_id(name);
        if (k < 0) continue;
        bool ok = false;
        for (int c : CANDIDATES[k]) ok = ok || c == block;
        if (!ok) continue; // a block size this build cannot launch
        TuneEntry &e = loaded[TuneKey{k, {L[0], L[1], L[2], L[3]}}];
        e.ms.emplace_back(block, ms);
        if (best) e.block = block;
    }
    std::fclose(fp);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &kv : loaded)
        if (kv.second.block) g_tune[kv.first] = kv.second;
    return LQCD_OK;
}

lqcd_status lqcd_autotune_block(const char *kernel, const lqcd_lattice *lat, int *block)
{
    LQCD_REQUIRE(lat && block, "autotune_block: NULL argument");
    const int k = kernel_id(kernel);
    LQCD_REQUIRE(k >= 0, "autotune_block: unknown kernel class %s", kernel ? kernel : "(null)");
    *block = tuned_block(k, *lat, 0);
    return LQCD_OK;
}

lqcd_status lqcd_autotune_clear(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
    return LQCD_OK;
}

} // extern "C"
