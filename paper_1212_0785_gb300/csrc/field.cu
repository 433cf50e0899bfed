// field.cu -- errors, allocator hook, field allocation and host transfer,
// precision conversion, Philox refresh kernels, start configuration, link
// update, reunitarization and the FP64 reductions (plaquette, kinetic energy,
// spinor dot products).
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "df64.cuh"
#include "lqcd_internal.cuh"
#include "md_device.cuh"
#include "tune.cuh"
#include "su3_device.cuh"

namespace lqcd {

// ------------------------------------------------------------------ errors

static thread_local std::string g_err;
std::atomic<uint64_t> g_launches{0};

void set_error(const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

lqcd_status cuda_fail(cudaError_t e, const char *what, const char *file, int line)
{
    set_error("%s failed at %s:%d: %s", what, file, line, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LQCD_ENOMEM : LQCD_ECUDA;
}

// ------------------------------------------------------------------ kernel timers

static const char *k_class_names[K_NCLASS] = {"dslash_f64",    "dslash_f32",  "dslash_f16n",
                                              "dslash_bf16",   "dslash_df64", "gauge_force",
                                              "fermion_force", "link_update", "dslash_f16n_plain"};
static std::mutex g_timer_mu;
static std::atomic<uint32_t> g_timer_mask{0}; // bit k: class k is timed
static std::atomic<int> g_timer_every{1};      // time one launch in every g_timer_every of a class
static std::atomic<uint64_t> g_timer_seen[K_NCLASS];
static std::vector<cudaEvent_t> g_event_pool;
struct PendingTiming {
    int cls;
    double bytes;
    cudaEvent_t a, b;
};
static std::vector<PendingTiming> g_pending;
static double g_timer_ms[K_NCLASS];
static double g_timer_bytes[K_NCLASS];
static uint64_t g_timer_n[K_NCLASS];

static cudaEvent_t pool_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

KernelTimer::KernelTimer(int c, cudaStream_t st, double nbytes) : cls(c), s(st), bytes(nbytes)
{
    if (!((g_timer_mask.load(std::memory_order_relaxed) >> c) & 1u)) return;
    const int every = g_timer_every.load(std::memory_order_relaxed);
    if (every > 1 && g_timer_seen[c].fetch_add(1, std::memory_order_relaxed) % (uint64_t)every != 0) return;
    std::lock_guard<std::mutex> lk(g_timer_mu);
    a = pool_event();
    b = pool_event();
    if (a && b) cudaEventRecord(a, s);
}

KernelTimer::~KernelTimer()
{
    if (!a || !b) return;
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> lk(g_timer_mu);
    g_pending.push_back({cls, bytes, a, b});
}

// resolve pending event pairs (device synchronised by the caller)
static void drain_timers_locked()
{
    for (auto &p : g_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_timer_ms[p.cls] += ms;
            g_timer_bytes[p.cls] += p.bytes;
            g_timer_n[p.cls] += 1;
        } else {
            cudaGetLastError();
        }
        g_event_pool.push_back(p.a);
        g_event_pool.push_back(p.b);
    }
    g_pending.clear();
}

// ------------------------------------------------------------------ allocator

static std::mutex g_alloc_mu;
static Allocator g_alloc{nullptr, nullptr, nullptr};

Allocator current_allocator()
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return g_alloc;
}

void *dev_alloc(const Allocator &a, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) bytes = 256;
    if (a.alloc) return a.alloc(bytes, (void *)s, a.ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(const Allocator &a, void *p, cudaStream_t s)
{
    if (!p) return;
    if (a.free_fn)
        a.free_fn(p, (void *)s, a.ctx);
    else
        cudaFree(p);
}

lqcd_status DevBuf::alloc(size_t n, cudaStream_t st)
{
    release();
    a = current_allocator();
    s = st;
    p = dev_alloc(a, n, st);
    if (!p) {
        set_error("device allocation of %zu bytes failed", n);
        return LQCD_ENOMEM;
    }
    bytes = n;
    return LQCD_OK;
}

void DevBuf::release()
{
    if (p) dev_free(a, p, s);
    p = nullptr;
    bytes = 0;
}

// ------------------------------------------------------------------ geometry

lqcd_status check_lattice(const lqcd_lattice *lat)
{
    LQCD_REQUIRE(lat != nullptr, "lattice is NULL");
    long long V = 1;
    for (int mu = 0; mu < 4; mu++) {
        LQCD_REQUIRE(lat->dims[mu] > 0 && lat->dims[mu] % 2 == 0,
                     "lattice extent %d in direction %d must be positive and even", lat->dims[mu], mu);
        V *= lat->dims[mu];
    }
    LQCD_REQUIRE(V < (1LL << 31), "lattice volume %lld exceeds 2^31 - 1", V);
    LQCD_REQUIRE(lat->t_bc == 1 || lat->t_bc == -1, "t_bc must be +1 or -1 (got %d)", lat->t_bc);
    LQCD_REQUIRE(lat->xi0 >= 0 && lat->xi0 < 1e6 && lat->nu >= 0 && lat->nu < 1e6,
                 "anisotropy xi0 = %g, nu = %g must be finite and non-negative (0: isotropic)", lat->xi0, lat->nu);
    return LQCD_OK;
}

// the anisotropy of a lattice, 0 read as 1
static double eff_xi0(const lqcd_lattice &l) { return l.xi0 > 0 ? l.xi0 : 1.0; }
static double eff_nu(const lqcd_lattice &l) { return l.nu > 0 ? l.nu : 1.0; }

Geo make_geo(const lqcd_lattice &lat)
{
    Geo g;
    for (int mu = 0; mu < 4; mu++) g.L[mu] = lat.dims[mu];
    g.Lxh = lat.dims[0] / 2;
    g.Vh = (int)((long long)lat.dims[0] * lat.dims[1] * lat.dims[2] * lat.dims[3] / 2);
    g.t_bc = lat.t_bc;
    g.sY = g.Lxh;
    g.sZ = g.Lxh * lat.dims[1];
    g.sT = g.sZ * lat.dims[2];
    g.dLxh = make_fastdiv((uint32_t)g.Lxh);
    g.dLy = make_fastdiv((uint32_t)lat.dims[1]);
    g.dLz = make_fastdiv((uint32_t)lat.dims[2]);
    g.xi0 = eff_xi0(lat);
    g.cs = eff_nu(lat) / g.xi0;
    g.aniso = (g.xi0 != 1.0 || g.cs != 1.0) ? 1 : 0;
    g.csf = (float)g.cs;
    g.cs_lo = (float)(g.cs - (double)g.csf);
    return g;
}

bool same_lattice(const lqcd_lattice &a, const lqcd_lattice &b)
{
    for (int mu = 0; mu < 4; mu++)
        if (a.dims[mu] != b.dims[mu]) return false;
    return a.t_bc == b.t_bc && eff_xi0(a) == eff_xi0(b) && eff_nu(a) == eff_nu(b);
}

// ------------------------------------------------------------------ scalar helpers

template <int N>
__global__ void final_sum_kernel(const double *partials, int nblocks, double *dst)
{
    double sums[N];
    final_sum_block<N>(partials, nblocks, sums);
    if (threadIdx.x == 0)
        for (int k = 0; k < N; k++) dst[k] = sums[k];
}

lqcd_status reduce_partials(const double *partials, int nblocks, int n, double *dst_dev, cudaStream_t s)
{
    switch (n) {
    case 1: final_sum_kernel<1><<<1, 1024, 0, s>>>(partials, nblocks, dst_dev); break;
    case 2: final_sum_kernel<2><<<1, 1024, 0, s>>>(partials, nblocks, dst_dev); break;
    case 3: final_sum_kernel<3><<<1, 1024, 0, s>>>(partials, nblocks, dst_dev); break;
    case 4: final_sum_kernel<4><<<1, 1024, 0, s>>>(partials, nblocks, dst_dev); break;
    case 5: final_sum_kernel<5><<<1, 1024, 0, s>>>(partials, nblocks, dst_dev); break;
    case 9: final_sum_kernel<9><<<1, 1024, 0, s>>>(partials, nblocks, dst_dev); break;
    default: set_error("reduce_partials: n=%d unsupported", n); return LQCD_EINVAL;
    }
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status read_scalars(const double *src_dev, double *host, int n, cudaStream_t s)
{
    LQCD_CUDA(cudaMemcpyAsync(host, src_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    LQCD_CUDA(cudaStreamSynchronize(s));
    return LQCD_OK;
}

// ------------------------------------------------------------------ field allocation

static bool valid_combo(lqcd_kind kind, lqcd_prec prec, int recon)
{
    switch (kind) {
    case LQCD_GAUGE: return (prec == LQCD_F64 && recon == 18) || (prec != LQCD_F64 && recon == 12);
    case LQCD_MOMENTUM: return prec == LQCD_F64 && recon == 0;
    case LQCD_SPINOR_EVEN:
    case LQCD_SPINOR_ODD: return recon == 0 && (prec >= LQCD_F64 && prec <= LQCD_BF16);
    case LQCD_SPINOR_FULL: return prec == LQCD_F64 && recon == 0;
    }
    return false;
}

static size_t field_data_bytes(lqcd_kind kind, lqcd_prec prec, int Vh)
{
    size_t n = (size_t)Vh;
    if (prec == (lqcd_prec)4) prec = LQCD_F64; // float-float pairs: as many bytes as FP64
    switch (kind) {
    case LQCD_GAUGE: return prec == LQCD_F64 ? n * 8 * 18 * 8 : (prec == LQCD_F32 ? n * 8 * 12 * 4 : n * 8 * 12 * 2);
    case LQCD_MOMENTUM: return n * 8 * 8 * 8;
    case LQCD_SPINOR_EVEN:
    case LQCD_SPINOR_ODD: return prec == LQCD_F64 ? n * 24 * 8 : (prec == LQCD_F32 ? n * 24 * 4 : n * 24 * 2);
    case LQCD_SPINOR_FULL: return n * 2 * 24 * 8;
    }
    return 0;
}

lqcd_status field_alloc_like(const lqcd_field *like, lqcd_kind kind, lqcd_prec prec, int recon, lqcd_field **out)
{
    return lqcd_field_alloc(&like->lat, kind, prec, recon, out);
}

static lqcd_status field_alloc_impl(const lqcd_lattice *lat, lqcd_kind kind, lqcd_prec prec, int recon,
                                    lqcd_field **out);

// fields in the internal float-float precision (gauge with 18 reals, half spinors)
lqcd_status field_alloc_df(const lqcd_lattice *lat, lqcd_kind kind, lqcd_field **out)
{
    LQCD_REQUIRE(kind == LQCD_GAUGE || kind == LQCD_SPINOR_EVEN || kind == LQCD_SPINOR_ODD,
                 "float-float fields are gauge or half spinors");
    return field_alloc_impl(lat, kind, (lqcd_prec)4, kind == LQCD_GAUGE ? 18 : 0, out);
}

// ------------------------------------------------------------------ host layout permutation kernels

// canonical gauge AoS [site][mu][row][col][re,im] <-> device SoA
// AoS host layout of a gauge field: links in (lexicographic site, mu) order,
// 18 doubles each (row-major complex 3x3).  A block of GA_LINKS threads moves
// GA_LINKS consecutive links through shared memory, so the AoS side is read
// (or written) contiguously by the whole block -- which matters when it is
// pinned host memory accessed directly over the host link -- and each thread
// converts its own link.
constexpr int GA_LINKS = 128;

template <lqcd_prec P>
__global__ void __launch_bounds__(GA_LINKS) gauge_from_aos(GaugeRef<P> U, const double *aos, Geo g, int V)
{
    __shared__ double sh[GA_LINKS * 18];
    const long t0 = (long)blockIdx.x * GA_LINKS;
    const int nl = (int)min((long)GA_LINKS, 4L * V - t0);
    const double *src = aos + t0 * 18;
    for (int i = threadIdx.x; i < nl * 18; i += GA_LINKS) sh[i] = src[i];
    __syncthreads();
    if ((int)threadIdx.x >= nl) return;
    const long t = t0 + threadIdx.x;
    int lex = (int)(t >> 2), mu = (int)(t & 3);
    int c[4], r = lex;
    for (int m = 0; m < 4; m++) {
        c[m] = r % g.L[m];
        r /= g.L[m];
    }
    int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    const double *e = sh + threadIdx.x * 18;
    M3<double> u;
    for (int k = 0; k < 9; k++) u.e[k / 3][k % 3] = cx<double>(e[2 * k], e[2 * k + 1]);
    U.store(mu, par, lex >> 1, u);
}

template <lqcd_prec P>
__global__ void __launch_bounds__(GA_LINKS) gauge_to_aos(GaugeRef<P> U, double *aos, Geo g, int V)
{
    __shared__ double sh[GA_LINKS * 18];
    const long t0 = (long)blockIdx.x * GA_LINKS;
    const int nl = (int)min((long)GA_LINKS, 4L * V - t0);
    if ((int)threadIdx.x < nl) {
        const long t = t0 + threadIdx.x;
        int lex = (int)(t >> 2), mu = (int)(t & 3);
        int c[4], r = lex;
        for (int m = 0; m < 4; m++) {
            c[m] = r % g.L[m];
            r /= g.L[m];
        }
        int par = (c[0] + c[1] + c[2] + c[3]) & 1;
        M3<double> u = U.template load<double>(mu, par, lex >> 1);
        double *e = sh + threadIdx.x * 18;
        for (int k = 0; k < 9; k++) {
            e[2 * k] = u.e[k / 3][k % 3].re;
            e[2 * k + 1] = u.e[k / 3][k % 3].im;
        }
    }
    __syncthreads();
    double *dst = aos + t0 * 18;
    for (int i = threadIdx.x; i < nl * 18; i += GA_LINKS) dst[i] = sh[i];
}

__global__ void mom_from_aos(MomRef P, const double *aos, Geo g, int V, int to_aos)
{
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= 4L * V) return;
    int lex = (int)(t >> 2), mu = (int)(t & 3);
    int c[4], r = lex;
    for (int m = 0; m < 4; m++) {
        c[m] = r % g.L[m];
        r /= g.L[m];
    }
    int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    double *h = const_cast<double *>(aos) + ((size_t)lex * 4 + mu) * 8;
    for (int a = 0; a < 8; a++) {
        if (to_aos)
            h[a] = P.d[P.idx(mu, par, a, lex >> 1)];
        else
            P.d[P.idx(mu, par, a, lex >> 1)] = h[a];
    }
}

// half spinor: host [cb][24]
template <lqcd_prec P>
__global__ void spinor_from_aos(SpinorRef<P> S, const double *aos, int Vh)
{
    int cb = blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= Vh) return;
    Sp<double> s;
    const double *src = aos + (size_t)cb * 24;
    for (int k = 0; k < 12; k++) s.c[k / 3][k % 3] = cx<double>(src[2 * k], src[2 * k + 1]);
    S.store(cb, s);
}

template <lqcd_prec P>
__global__ void spinor_to_aos(SpinorRef<P> S, double *aos, int Vh)
{
    int cb = blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= Vh) return;
    Sp<double> s = S.template load_rw<double>(cb);
    double *dst = aos + (size_t)cb * 24;
    for (int k = 0; k < 12; k++) {
        dst[2 * k] = s.c[k / 3][k % 3].re;
        dst[2 * k + 1] = s.c[k / 3][k % 3].im;
    }
}

// full spinor: host [lex][24], device [parity][12][Vh]
__global__ void full_spinor_perm(double2 *dev, double *aos, Geo g, int V, int to_aos)
{
    int lex = blockIdx.x * blockDim.x + threadIdx.x;
    if (lex >= V) return;
    int c[4], r = lex;
    for (int m = 0; m < 4; m++) {
        c[m] = r % g.L[m];
        r /= g.L[m];
    }
    int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    int cb = lex >> 1;
    double2 *base = dev + (size_t)par * 12 * g.Vh;
    for (int k = 0; k < 12; k++) {
        if (to_aos) {
            double2 v = base[(size_t)k * g.Vh + cb];
            aos[(size_t)lex * 24 + 2 * k] = v.x;
            aos[(size_t)lex * 24 + 2 * k + 1] = v.y;
        } else {
            base[(size_t)k * g.Vh + cb] = make_double2(aos[(size_t)lex * 24 + 2 * k], aos[(size_t)lex * 24 + 2 * k + 1]);
        }
    }
}

static size_t host_doubles(const lqcd_field *f)
{
    size_t V = 2 * (size_t)f->Vh;
    switch (f->kind) {
    case LQCD_GAUGE: return V * 4 * 18;
    case LQCD_MOMENTUM: return V * 4 * 8;
    case LQCD_SPINOR_EVEN:
    case LQCD_SPINOR_ODD: return (size_t)f->Vh * 24;
    case LQCD_SPINOR_FULL: return V * 24;
    }
    return 0;
}

// the device address of pinned (page-locked, mapped) host memory, else NULL
static double *mapped_host(double *host)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer ? (double *)a.devicePointer : nullptr;
}

// Host <-> device with the layout change done by a kernel.  Pinned host
// memory is read or written by that kernel directly (no device staging copy:
// one pass over the host link); pageable memory goes through a device buffer
// and one copy.
static lqcd_status transfer(lqcd_field *f, double *host, bool upload, cudaStream_t s)
{
    size_t n = host_doubles(f);
    DevBuf tmp;
    double *d = mapped_host(host);
    const bool staged = d == nullptr;
    if (staged) {
        LQCD_TRY(tmp.alloc(n * sizeof(double), s));
        d = (double *)tmp.p;
    }
    Geo g = make_geo(f->lat);
    int V = 2 * f->Vh;
    const int B = 256;
    if (upload && staged) LQCD_CUDA(cudaMemcpyAsync(d, host, n * sizeof(double), cudaMemcpyHostToDevice, s));
    switch (f->kind) {
    case LQCD_GAUGE: {
        const int B = GA_LINKS;
        int nb = nblocks_for(4L * V, B);
        switch (f->prec) {
        case LQCD_F64:
            if (upload) gauge_from_aos<LQCD_F64><<<nb, B, 0, s>>>(gauge_ref<LQCD_F64>(f), d, g, V);
            else gauge_to_aos<LQCD_F64><<<nb, B, 0, s>>>(gauge_ref<LQCD_F64>(f), d, g, V);
            break;
        case LQCD_F32:
            if (upload) gauge_from_aos<LQCD_F32><<<nb, B, 0, s>>>(gauge_ref<LQCD_F32>(f), d, g, V);
            else gauge_to_aos<LQCD_F32><<<nb, B, 0, s>>>(gauge_ref<LQCD_F32>(f), d, g, V);
            break;
        case LQCD_F16N:
            if (upload) gauge_from_aos<LQCD_F16N><<<nb, B, 0, s>>>(gauge_ref<LQCD_F16N>(f), d, g, V);
            else gauge_to_aos<LQCD_F16N><<<nb, B, 0, s>>>(gauge_ref<LQCD_F16N>(f), d, g, V);
            break;
        case LQCD_BF16:
            if (upload) gauge_from_aos<LQCD_BF16><<<nb, B, 0, s>>>(gauge_ref<LQCD_BF16>(f), d, g, V);
            else gauge_to_aos<LQCD_BF16><<<nb, B, 0, s>>>(gauge_ref<LQCD_BF16>(f), d, g, V);
            break;
        }
        break;
    }
    case LQCD_MOMENTUM:
        mom_from_aos<<<nblocks_for(4L * V, B), B, 0, s>>>(mom_ref(f), d, g, V, upload ? 0 : 1);
        break;
    case LQCD_SPINOR_EVEN:
    case LQCD_SPINOR_ODD: {
        int nb = nblocks_for(f->Vh, B);
        switch (f->prec) {
        case LQCD_F64:
            if (upload) spinor_from_aos<LQCD_F64><<<nb, B, 0, s>>>(spinor_ref<LQCD_F64>(f), d, f->Vh);
            else spinor_to_aos<LQCD_F64><<<nb, B, 0, s>>>(spinor_ref<LQCD_F64>(f), d, f->Vh);
            break;
        case LQCD_F32:
            if (upload) spinor_from_aos<LQCD_F32><<<nb, B, 0, s>>>(spinor_ref<LQCD_F32>(f), d, f->Vh);
            else spinor_to_aos<LQCD_F32><<<nb, B, 0, s>>>(spinor_ref<LQCD_F32>(f), d, f->Vh);
            break;
        case LQCD_F16N:
            if (upload) spinor_from_aos<LQCD_F16N><<<nb, B, 0, s>>>(spinor_ref<LQCD_F16N>(f), d, f->Vh);
            else spinor_to_aos<LQCD_F16N><<<nb, B, 0, s>>>(spinor_ref<LQCD_F16N>(f), d, f->Vh);
            break;
        case LQCD_BF16:
            if (upload) spinor_from_aos<LQCD_BF16><<<nb, B, 0, s>>>(spinor_ref<LQCD_BF16>(f), d, f->Vh);
            else spinor_to_aos<LQCD_BF16><<<nb, B, 0, s>>>(spinor_ref<LQCD_BF16>(f), d, f->Vh);
            break;
        }
        break;
    }
    case LQCD_SPINOR_FULL:
        full_spinor_perm<<<nblocks_for(V, B), B, 0, s>>>((double2 *)f->data, d, g, V, upload ? 0 : 1);
        break;
    }
    LQCD_LAUNCHED();
    if (!upload && staged) LQCD_CUDA(cudaMemcpyAsync(host, d, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    LQCD_CUDA(cudaStreamSynchronize(s));
    return LQCD_OK;
}

// ------------------------------------------------------------------ conversions

template <lqcd_prec PS, lqcd_prec PD>
__global__ void gauge_convert(GaugeRef<PD> dst, GaugeRef<PS> src, int Vh)
{
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= 8L * Vh) return;
    int cb = (int)(t % Vh);
    int mp = (int)(t / Vh); // mu*2 + par
    M3<double> u = src.template load<double>(mp >> 1, mp & 1, cb);
    dst.store(mp >> 1, mp & 1, cb, u);
}

template <lqcd_prec PS, lqcd_prec PD>
__global__ void spinor_convert(SpinorRef<PD> dst, SpinorRef<PS> src, int Vh)
{
    int cb = blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= Vh) return;
    Sp<double> s = src.template load_rw<double>(cb);
    dst.store(cb, s);
}

template <lqcd_prec PS>
static void launch_gauge_convert(lqcd_field *dst, const lqcd_field *src, cudaStream_t s)
{
    int nb = nblocks_for(8L * src->Vh, 256);
    switch (dst->prec) {
    case LQCD_F64: gauge_convert<PS, LQCD_F64><<<nb, 256, 0, s>>>(gauge_ref<LQCD_F64>(dst), gauge_ref<PS>(src), src->Vh); break;
    case LQCD_F32: gauge_convert<PS, LQCD_F32><<<nb, 256, 0, s>>>(gauge_ref<LQCD_F32>(dst), gauge_ref<PS>(src), src->Vh); break;
    case LQCD_F16N: gauge_convert<PS, LQCD_F16N><<<nb, 256, 0, s>>>(gauge_ref<LQCD_F16N>(dst), gauge_ref<PS>(src), src->Vh); break;
    case LQCD_BF16: gauge_convert<PS, LQCD_BF16><<<nb, 256, 0, s>>>(gauge_ref<LQCD_BF16>(dst), gauge_ref<PS>(src), src->Vh); break;
    }
}

template <lqcd_prec PS>
static void launch_spinor_convert(lqcd_field *dst, const lqcd_field *src, cudaStream_t s)
{
    int nb = nblocks_for(src->Vh, 256);
    switch (dst->prec) {
    case LQCD_F64: spinor_convert<PS, LQCD_F64><<<nb, 256, 0, s>>>(spinor_ref<LQCD_F64>(dst), spinor_ref<PS>(src), src->Vh); break;
    case LQCD_F32: spinor_convert<PS, LQCD_F32><<<nb, 256, 0, s>>>(spinor_ref<LQCD_F32>(dst), spinor_ref<PS>(src), src->Vh); break;
    case LQCD_F16N: spinor_convert<PS, LQCD_F16N><<<nb, 256, 0, s>>>(spinor_ref<LQCD_F16N>(dst), spinor_ref<PS>(src), src->Vh); break;
    case LQCD_BF16: spinor_convert<PS, LQCD_BF16><<<nb, 256, 0, s>>>(spinor_ref<LQCD_BF16>(dst), spinor_ref<PS>(src), src->Vh); break;
    }
}

// ------------------------------------------------------------------ RNG kernels

// the float-float codec on n doubles: pairs[2i], pairs[2i + 1] = hi, lo of
// in[i]; back[i] = hi + lo rounded to a double
__global__ void df_split_kernel(const double *in, float2 *pairs, double *back, size_t n)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Df v(in[i]);
    pairs[i] = make_float2(v.hi, v.lo);
    back[i] = (double)v;
}

__global__ void philox_blocks_kernel(uint4 *out, size_t n, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = philox4x32_10(make_uint4(c0 + (uint32_t)i, c1, c2, c3), make_uint2(k0, k1));
}

// start links: thread per site (lex), 16 Philox blocks -> 32 Gaussians
__global__ void gauge_start_kernel(GaugeRef<LQCD_F64> U, Geo g, int V, uint32_t seed, uint32_t chain, double eps)
{
    int lex = blockIdx.x * blockDim.x + threadIdx.x;
    if (lex >= V) return;
    int c[4], r = lex;
    for (int m = 0; m < 4; m++) {
        c[m] = r % g.L[m];
        r /= g.L[m];
    }
    int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    for (int mu = 0; mu < 4; mu++) {
        double h[8];
        for (int q = 0; q < 4; q++) {
            int j = mu * 4 + q; // Gaussians 2j, 2j+1 -> coefficients 2q, 2q+1 of link mu
            philox_gauss2(seed, chain, (uint32_t)lex, (uint32_t)j, 0u, 0u, h[2 * q], h[2 * q + 1]);
        }
        M3<double> Q = herm_from_coeffs(h, eps);
        U.store(mu, par, lex >> 1, expi_cayley_hamilton(Q));
    }
}

__global__ void momentum_refresh_kernel(MomRef P, Geo g, int V, uint32_t seed, uint32_t chain, uint32_t traj)
{
    int lex = blockIdx.x * blockDim.x + threadIdx.x;
    if (lex >= V) return;
    int c[4], r = lex;
    for (int m = 0; m < 4; m++) {
        c[m] = r % g.L[m];
        r /= g.L[m];
    }
    int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    int cb = lex >> 1;
    for (int j = 0; j < 16; j++) {
        double g0, g1;
        philox_gauss2(seed, chain, (uint32_t)lex, (uint32_t)j, 1u, traj, g0, g1);
        int k = 2 * j; // coefficient index mu*8 + a
        P.d[P.idx(k >> 3, par, k & 7, cb)] = g0;
        P.d[P.idx((k + 1) >> 3, par, (k + 1) & 7, cb)] = g1;
    }
}

__global__ void eta_refresh_kernel(SpinorRef<LQCD_F64> E, Geo g, uint32_t seed, uint32_t chain, uint32_t traj,
                                   uint32_t purpose)
{
    int cb = blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= g.Vh) return;
    int c[4];
    cb_coords(g, cb, 0, c);
    int lex = coords_lex(g, c);
    const double s = 0.70710678118654752440; // sqrt(1/2)
    Sp<double> v;
    for (int j = 0; j < 12; j++) { // complex component j = spin*3 + colour
        double g0, g1;
        philox_gauss2(seed, chain, (uint32_t)lex, (uint32_t)j, purpose, traj, g0, g1);
        v.c[j / 3][j % 3] = cx<double>(g0 * s, g1 * s);
    }
    E.store(cb, v);
}

// ------------------------------------------------------------------ link update / reunitarize

// U <- exp(i c P) U on every link (link_update_one), one thread per link.
// Registers capped at 128 (two blocks of 256, four of 128 per SM): uncapped it
// took 168 (three blocks of 128) and ran 46.4 ms per 32^3x64 trajectory, capped
// 40.9 ms in a same-box A/B (85 registers, with spills: 41.7 ms).
template <lqcd_prec PS, bool FAST>
__global__ void __launch_bounds__(256, 2) link_update_kernel(GaugeRef<LQCD_F64> U, MomRef P, double c, GaugeRef<PS> Us, GaugeRef<LQCD_F32> Uf,
                                   GaugeRef<PREC_DF> Udf, int Vh, int write_sloppy, int write_f32, int write_f64)
{
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= 8L * Vh) return;
    int cb = (int)(t % Vh);
    int mp = (int)(t / Vh);
    link_update_one<PS, FAST>(U, P, c, Us, Uf, Udf, mp >> 1, mp & 1, cb, write_sloppy, write_f32, write_f64);
}

// U = the float-float links, per link entry (double) hi + (double) lo: bitwise
// what the link update writes when it writes the FP64 links itself
__global__ void links_from_df_kernel(GaugeRef<LQCD_F64> U, GaugeRef<PREC_DF> Udf, int Vh)
{
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= 8L * Vh) return;
    const int cb = (int)(t % Vh), mp = (int)(t / Vh);
    U.store(mp >> 1, mp & 1, cb, Udf.load<double>(mp >> 1, mp & 1, cb));
}

lqcd_status links_from_df(lqcd_field *U, const lqcd_field *Udf, cudaStream_t s)
{
    links_from_df_kernel<<<nblocks_for(8L * U->Vh, 128), 128, 0, s>>>(gauge_ref<LQCD_F64>(U),
                                                                        gauge_ref<PREC_DF>(Udf), U->Vh);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

__global__ void reunitarize_kernel(GaugeRef<LQCD_F64> U, int Vh, double *partials)
{
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    double dev = 0.0;
    if (t < 8L * Vh) {
        int cb = (int)(t % Vh);
        int mp = (int)(t / Vh);
        M3<double> u = U.load<double>(mp >> 1, mp & 1, cb);
        M3<double> p = m3_mul_dag(u, u);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                Cx<double> d = p.e[i][j] - cx<double>(i == j ? 1.0 : 0.0, 0.0);
                dev = fmax(dev, sqrt(norm2(d)));
            }
        double n0 = sqrt(norm2(u.e[0][0]) + norm2(u.e[0][1]) + norm2(u.e[0][2]));
        for (int b = 0; b < 3; b++) u.e[0][b] = (1.0 / n0) * u.e[0][b];
        Cx<double> ov = cmul_conj(u.e[0][0], u.e[1][0]) + cmul_conj(u.e[0][1], u.e[1][1]) + cmul_conj(u.e[0][2], u.e[1][2]);
        for (int b = 0; b < 3; b++) u.e[1][b] = u.e[1][b] - ov * u.e[0][b];
        double n1 = sqrt(norm2(u.e[1][0]) + norm2(u.e[1][1]) + norm2(u.e[1][2]));
        for (int b = 0; b < 3; b++) u.e[1][b] = (1.0 / n1) * u.e[1][b];
        reconstruct_row2(u);
        U.store(mp >> 1, mp & 1, cb, u);
    }
    // block max (order-independent, hence deterministic)
    __shared__ double sh[8];
    for (int off = 16; off > 0; off >>= 1) dev = fmax(dev, __shfl_down_sync(0xffffffffu, dev, off));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = dev;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = fmax(m, sh[w]);
        partials[blockIdx.x] = m;
    }
}

__global__ void max_final_kernel(const double *partials, int n, double *out)
{
    __shared__ double sh[32];
    double m = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, partials[i]);
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) r = fmax(r, sh[w]);
        out[0] = r;
    }
}

// ------------------------------------------------------------------ reductions

constexpr int RB = 256;

// sum over sites of sum_{mu<nu} Re Tr U_munu(x) / 3; thread per site (both parities)
// sum over sites and planes mu < nu of Re Tr U_munu / 3; WEIGHTED (the
// anisotropic gauge action): each plane times its weight, xi0 for the planes
// with t and 1 / xi0 for the spatial ones
__global__ void __launch_bounds__(RB) plaquette_kernel(GaugeRef<LQCD_F64> U, Geo g, double *partials, int nblocks,
                                                       int weighted)
{
    int t = blockIdx.x * RB + threadIdx.x;
    double acc[1] = {0.0};
    if (t < 2 * g.Vh) {
        int par = t / g.Vh, cb = t % g.Vh;
        int c[4];
        cb_coords(g, cb, par, c);
        for (int mu = 0; mu < 3; mu++) {
            int cm[4] = {c[0], c[1], c[2], c[3]};
            cm[mu] = (c[mu] + 1 == g.L[mu]) ? 0 : c[mu] + 1;
            int cb_m = coords_cb(g, cm);
            M3<double> umu = U.load<double>(mu, par, cb);
            for (int nu = mu + 1; nu < 4; nu++) {
                int cn[4] = {c[0], c[1], c[2], c[3]};
                cn[nu] = (c[nu] + 1 == g.L[nu]) ? 0 : c[nu] + 1;
                int cb_n = coords_cb(g, cn);
                M3<double> a = m3_mul(umu, U.load<double>(nu, 1 - par, cb_m));
                M3<double> b = m3_mul(U.load<double>(nu, par, cb), U.load<double>(mu, 1 - par, cb_n));
                // Re Tr(a b^dag)
                double tr = 0;
                for (int i = 0; i < 3; i++)
                    for (int k = 0; k < 3; k++) tr += a.e[i][k].re * b.e[i][k].re + a.e[i][k].im * b.e[i][k].im;
                const double p = tr * (1.0 / 3.0);
                acc[0] += (weighted && g.aniso) ? (nu == 3 ? g.xi0 : 1.0 / g.xi0) * p : p;
            }
        }
    }
    block_sum_store<1, RB>(acc, partials, nblocks);
}

__global__ void __launch_bounds__(RB) sumsq_kernel(const double *d, long n, double *partials, int nblocks)
{
    // each block sums a fixed contiguous chunk
    long chunk = (n + nblocks - 1) / nblocks;
    long lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    double acc[1] = {0.0};
    for (long i = lo + threadIdx.x; i < hi; i += RB) acc[0] += d[i] * d[i];
    block_sum_store<1, RB>(acc, partials, nblocks);
}

__global__ void __launch_bounds__(RB) dot_kernel(const double *a, const double *b, long n, double *partials,
                                                 int nblocks)
{
    long chunk = (n + nblocks - 1) / nblocks;
    long lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    double acc[1] = {0.0};
    for (long i = lo + threadIdx.x; i < hi; i += RB) acc[0] += a[i] * b[i];
    block_sum_store<1, RB>(acc, partials, nblocks);
}

// number of blocks for the flat reductions: a fixed function of n only
static int flat_blocks(long n) { return (int)std::min<long>(1184, std::max<long>(1, (n + RB * 8 - 1) / (RB * 8))); }

// The plaquette sum from float-float links (~48 bits per product, FP64
// accumulation): the FP32 pipes instead of the FP64 one.  Re Tr(a b^dag) with
// a = U_mu(x) U_nu(x+mu), b = U_nu(x) U_mu(x+nu), as plaquette_kernel.
__device__ __forceinline__ M3<Df> df_link(const GaugeRef<PREC_DF> &U, int mu, int par, int cb)
{
    M3<Df> u;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        float4 v = ldg(U.d + U.idx(mu, par, k, cb));
        u.e[k / 3][k % 3] = Cx<Df>{Df(v.x, v.y), Df(v.z, v.w)};
    }
    return u;
}

__device__ __forceinline__ M3<Df> df_mul(const M3<Df> &a, const M3<Df> &b)
{
    M3<Df> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            DfAcc re, im;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                re.add_prod(a.e[i][k].re, b.e[k][j].re);
                re.sub_prod(a.e[i][k].im, b.e[k][j].im);
                im.add_prod(a.e[i][k].re, b.e[k][j].im);
                im.add_prod(a.e[i][k].im, b.e[k][j].re);
            }
            r.e[i][j] = Cx<Df>{re.value(), im.value()};
        }
    return r;
}

__global__ void __launch_bounds__(RB) plaquette_df_kernel(GaugeRef<PREC_DF> U, Geo g, double *partials, int nblocks,
                                                          int weighted)
{
    int t = blockIdx.x * RB + threadIdx.x;
    double acc[1] = {0.0};
    if (t < 2 * g.Vh) {
        int par = t / g.Vh, cb = t % g.Vh;
        int c[4];
        cb_coords(g, cb, par, c);
        for (int mu = 0; mu < 3; mu++) {
            int cm[4] = {c[0], c[1], c[2], c[3]};
            cm[mu] = (c[mu] + 1 == g.L[mu]) ? 0 : c[mu] + 1;
            int cb_m = coords_cb(g, cm);
            for (int nu = mu + 1; nu < 4; nu++) {
                int cn[4] = {c[0], c[1], c[2], c[3]};
                cn[nu] = (c[nu] + 1 == g.L[nu]) ? 0 : c[nu] + 1;
                int cb_n = coords_cb(g, cn);
                M3<Df> a = df_mul(df_link(U, mu, par, cb), df_link(U, nu, 1 - par, cb_m));
                M3<Df> b = df_mul(df_link(U, nu, par, cb), df_link(U, mu, 1 - par, cb_n));
                DfAcc tr;
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        tr.add_prod(a.e[i][k].re, b.e[i][k].re);
                        tr.add_prod(a.e[i][k].im, b.e[i][k].im);
                    }
                const double p = (double)tr.value() * (1.0 / 3.0);
                acc[0] += (weighted && g.aniso) ? (nu == 3 ? g.xi0 : 1.0 / g.xi0) * p : p;
            }
        }
    }
    block_sum_store<1, RB>(acc, partials, nblocks);
}

lqcd_status plaquette_sum_df(const lqcd_field *Udf, double *dst_dev, DevBuf &part, cudaStream_t s, bool weighted)
{
    Geo g = make_geo(Udf->lat);
    int nb = nblocks_for(2L * g.Vh, RB);
    if (part.bytes < sizeof(double) * nb) LQCD_TRY(part.alloc(sizeof(double) * nb, s));
    plaquette_df_kernel<<<nb, RB, 0, s>>>(gauge_ref<PREC_DF>(Udf), g, (double *)part.p, nb, weighted ? 1 : 0);
    LQCD_LAUNCHED();
    return reduce_partials((double *)part.p, nb, 1, dst_dev, s);
}

lqcd_status plaquette_sum(const lqcd_field *U, double *dst_dev, DevBuf &part, cudaStream_t s, bool weighted)
{
    Geo g = make_geo(U->lat);
    int nb = nblocks_for(2L * g.Vh, RB);
    if (part.bytes < sizeof(double) * nb) LQCD_TRY(part.alloc(sizeof(double) * nb, s));
    plaquette_kernel<<<nb, RB, 0, s>>>(gauge_ref<LQCD_F64>(U), g, (double *)part.p, nb, weighted ? 1 : 0);
    LQCD_LAUNCHED();
    return reduce_partials((double *)part.p, nb, 1, dst_dev, s);
}

// block partials of the plaquette sum into caller-provided memory (nblocks
// from plaquette_partial_blocks)
int plaquette_partial_blocks(const lqcd_field *U) { return nblocks_for(2L * U->Vh, RB); }

lqcd_status plaquette_partials_launch(const lqcd_field *U, double *partials, int nblocks, cudaStream_t s)
{
    plaquette_kernel<<<nblocks, RB, 0, s>>>(gauge_ref<LQCD_F64>(U), make_geo(U->lat), partials, nblocks, 0);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status kinetic_sum(const lqcd_field *P, double *dst_dev, DevBuf &part, cudaStream_t s)
{
    long n = (long)P->Vh * 64;
    int nb = flat_blocks(n);
    if (part.bytes < sizeof(double) * nb) LQCD_TRY(part.alloc(sizeof(double) * nb, s));
    sumsq_kernel<<<nb, RB, 0, s>>>((const double *)P->data, n, (double *)part.p, nb);
    LQCD_LAUNCHED();
    return reduce_partials((double *)part.p, nb, 1, dst_dev, s);
}

lqcd_status spinor_dot_dev(const lqcd_field *a, const lqcd_field *b, double *dst_dev, DevBuf &part, cudaStream_t s)
{
    long n = (long)a->bytes / sizeof(double);
    int nb = flat_blocks(n);
    if (part.bytes < sizeof(double) * nb) LQCD_TRY(part.alloc(sizeof(double) * nb, s));
    dot_kernel<<<nb, RB, 0, s>>>((const double *)a->data, (const double *)b->data, n, (double *)part.p, nb);
    LQCD_LAUNCHED();
    return reduce_partials((double *)part.p, nb, 1, dst_dev, s);
}

lqcd_status reunitarize_dev(lqcd_field *U, double *dst_dev, DevBuf &part, cudaStream_t s)
{
    long n = 8L * U->Vh;
    int nb = nblocks_for(n, 256);
    if (part.bytes < sizeof(double) * nb) LQCD_TRY(part.alloc(sizeof(double) * nb, s));
    reunitarize_kernel<<<nb, 256, 0, s>>>(gauge_ref<LQCD_F64>(U), U->Vh, (double *)part.p);
    LQCD_LAUNCHED();
    max_final_kernel<<<1, 1024, 0, s>>>((double *)part.p, nb, dst_dev);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

template <bool FAST>
static lqcd_status launch_link_update(lqcd_field *U, const lqcd_field *P, double c, lqcd_field *Us, lqcd_field *Uf,
                                      lqcd_field *Udf, cudaStream_t s, int bs = 128, bool write_f64 = true)
{
    LQCD_REQUIRE(bs >= 32 && bs <= 256 && bs % 32 == 0, "link update: bad block size %d", bs);
    LQCD_REQUIRE(write_f64 || (FAST && Udf), "link update: only the float-float copy can stand in for the FP64 links");
    const int w64 = write_f64 ? 1 : 0;
    GaugeRef<PREC_DF> ud = Udf ? gauge_ref<PREC_DF>(Udf) : GaugeRef<PREC_DF>{nullptr, U->Vh};
    long n = 8L * U->Vh;
    int nb = nblocks_for(n, bs);
    GaugeRef<LQCD_F32> uf = Uf ? gauge_ref<LQCD_F32>(Uf) : GaugeRef<LQCD_F32>{nullptr, U->Vh};
    int wf = Uf ? 1 : 0;
    switch (Us ? Us->prec : LQCD_F32) {
    case LQCD_F32:
        link_update_kernel<LQCD_F32, FAST><<<nb, bs, 0, s>>>(gauge_ref<LQCD_F64>(U), mom_ref(P), c,
                                                              Us ? gauge_ref<LQCD_F32>(Us) : uf, uf, ud, U->Vh, Us ? 1 : 0, wf, w64);
        break;
    case LQCD_F16N:
        link_update_kernel<LQCD_F16N, FAST><<<nb, bs, 0, s>>>(gauge_ref<LQCD_F64>(U), mom_ref(P), c,
                                                               gauge_ref<LQCD_F16N>(Us), uf, ud, U->Vh, 1, wf, w64);
        break;
    case LQCD_BF16:
        link_update_kernel<LQCD_BF16, FAST><<<nb, bs, 0, s>>>(gauge_ref<LQCD_F64>(U), mom_ref(P), c,
                                                               gauge_ref<LQCD_BF16>(Us), uf, ud, U->Vh, 1, wf, w64);
        break;
    default: set_error("sloppy link copy must be 12-real F32/F16N/BF16"); return LQCD_EINVAL;
    }
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status link_update_dev(lqcd_field *U, const lqcd_field *P, double c, lqcd_field *Us, lqcd_field *Uf, bool fast,
                            cudaStream_t s, lqcd_field *Udf, bool write_f64 = true)
{
    KernelTimer kt(K_LINK_UPDATE, s);
    return fast ? launch_link_update<true>(U, P, c, Us, Uf, Udf, s, tuned_block(TK_LINK_UPDATE_F32, U->lat, 128),
                                           write_f64)
                : launch_link_update<false>(U, P, c, Us, Uf, Udf, s);
}

// the FP32 molecular dynamics' link update with bs threads per block, as the
// mixed trajectory runs it (the FP64 links lag behind the float-float copy)
lqcd_status link_update_block(lqcd_field *U, const lqcd_field *P, double c, lqcd_field *Us, lqcd_field *Uf,
                              lqcd_field *Udf, int bs, cudaStream_t s)
{
    return launch_link_update<true>(U, P, c, Us, Uf, Udf, s, bs, Udf == nullptr);
}

lqcd_status momentum_refresh_dev(lqcd_field *P, uint32_t seed, uint32_t chain, uint32_t traj, cudaStream_t s)
{
    Geo g = make_geo(P->lat);
    int V = 2 * g.Vh;
    momentum_refresh_kernel<<<nblocks_for(V, 128), 128, 0, s>>>(mom_ref(P), g, V, seed, chain, traj);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status eta_refresh_dev(lqcd_field *E, uint32_t seed, uint32_t chain, uint32_t traj, cudaStream_t s,
                            uint32_t purpose)
{
    Geo g = make_geo(E->lat);
    eta_refresh_kernel<<<nblocks_for(g.Vh, 128), 128, 0, s>>>(spinor_ref<LQCD_F64>(E), g, seed, chain, traj,
                                                              purpose);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

} // namespace lqcd

using namespace lqcd;

// ================================================================== C ABI

extern "C" {

const char *lqcd_last_error(void) { return g_err.c_str(); }

const char *lqcd_version(void) { return "lqcd-gb300 0.1 (sm_103a)"; }

uint64_t lqcd_launch_count(void) { return g_launches.load(); }

static lqcd_status timers_set(uint32_t mask)
{
    LQCD_CUDA(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lk(g_timer_mu);
    drain_timers_locked();
    for (int k = 0; k < K_NCLASS; k++) {
        g_timer_ms[k] = 0;
        g_timer_bytes[k] = 0;
        g_timer_n[k] = 0;
    }
    for (int k = 0; k < K_NCLASS; k++) g_timer_seen[k].store(0);
    g_timer_mask.store(mask);
    return LQCD_OK;
}

lqcd_status lqcd_kernel_timers(int enable) { return timers_set(enable ? (1u << K_NCLASS) - 1u : 0u); }

lqcd_status lqcd_kernel_timers_only(const char *kernel_classes)
{
    LQCD_REQUIRE(kernel_classes, "kernel_timers_only: NULL class");
    uint32_t mask = 0;
    const std::string list(kernel_classes);
    size_t at = 0;
    while (at <= list.size()) {
        size_t end = list.find(',', at);
        if (end == std::string::npos) end = list.size();
        const std::string name = list.substr(at, end - at);
        int cls = -1;
        for (int k = 0; k < K_NCLASS; k++)
            if (name == k_class_names[k]) cls = k;
        LQCD_REQUIRE(cls >= 0, "kernel_timers_only: unknown class '%s'", name.c_str());
        mask |= 1u << cls;
        at = end + 1;
    }
    return timers_set(mask);
}

lqcd_status lqcd_kernel_timers_every(int every)
{
    LQCD_REQUIRE(every >= 1, "kernel_timers_every: every must be >= 1");
    g_timer_every.store(every);
    return LQCD_OK;
}

lqcd_status lqcd_kernel_timer_read(const char *kernel_class, double *total_ms, uint64_t *launches,
                                   double *algorithmic_bytes)
{
    LQCD_REQUIRE(kernel_class, "kernel_timer_read: NULL class");
    int cls = -1;
    for (int k = 0; k < K_NCLASS; k++)
        if (std::strcmp(kernel_class, k_class_names[k]) == 0) cls = k;
    LQCD_REQUIRE(cls >= 0, "kernel_timer_read: unknown class '%s'", kernel_class);
    LQCD_CUDA(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lk(g_timer_mu);
    drain_timers_locked();
    if (total_ms) *total_ms = g_timer_ms[cls];
    if (launches) *launches = g_timer_n[cls];
    if (algorithmic_bytes) *algorithmic_bytes = g_timer_bytes[cls];
    return LQCD_OK;
}

lqcd_status lqcd_set_allocator(lqcd_alloc_fn alloc, lqcd_free_fn free_fn, void *ctx)
{
    LQCD_REQUIRE((alloc == nullptr) == (free_fn == nullptr), "allocator: alloc and free must both be set or both NULL");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = Allocator{alloc, free_fn, ctx};
    return LQCD_OK;
}

lqcd_status lqcd_field_alloc(const lqcd_lattice *lat, lqcd_kind kind, lqcd_prec prec, int link_recon, lqcd_field **out)
{
    LQCD_TRY(check_lattice(lat));
    LQCD_REQUIRE(out != nullptr, "out is NULL");
    LQCD_REQUIRE(valid_combo(kind, prec, link_recon), "invalid field combination kind=%d prec=%d recon=%d", (int)kind,
                 (int)prec, link_recon);
    return field_alloc_impl(lat, kind, prec, link_recon, out);
}

} // extern "C"

namespace lqcd {

static lqcd_status field_alloc_impl(const lqcd_lattice *lat, lqcd_kind kind, lqcd_prec prec, int link_recon,
                                    lqcd_field **out)
{
    LQCD_TRY(check_lattice(lat));
    LQCD_REQUIRE(out != nullptr, "out is NULL");
    lqcd_field *f = new lqcd_field();
    f->lat = *lat;
    f->kind = kind;
    f->prec = prec;
    f->recon = link_recon;
    f->Vh = make_geo(*lat).Vh;
    f->bytes = field_data_bytes(kind, prec, f->Vh);
    Allocator a = current_allocator();
    f->alloc = a.alloc;
    f->free_fn = a.free_fn;
    f->alloc_ctx = a.ctx;
    f->data = dev_alloc(a, f->bytes, nullptr);
    if (!f->data) {
        delete f;
        set_error("device allocation of %zu bytes failed", field_data_bytes(kind, prec, make_geo(*lat).Vh));
        return LQCD_ENOMEM;
    }
    if ((kind == LQCD_SPINOR_EVEN || kind == LQCD_SPINOR_ODD) && prec == LQCD_F16N) {
        f->norm_bytes = sizeof(float) * (size_t)f->Vh;
        f->norm = (float *)dev_alloc(a, f->norm_bytes, nullptr);
        if (!f->norm) {
            dev_free(a, f->data, nullptr);
            delete f;
            set_error("device allocation of the norm array failed");
            return LQCD_ENOMEM;
        }
    }
    *out = f;
    return LQCD_OK;
}

} // namespace lqcd

extern "C" {

lqcd_status lqcd_field_free(lqcd_field *f)
{
    if (!f) return LQCD_OK;
    Allocator a{f->alloc, f->free_fn, f->alloc_ctx};
    dev_free(a, f->data, nullptr);
    dev_free(a, f->norm, nullptr);
    delete f;
    return LQCD_OK;
}

lqcd_status lqcd_field_bytes(const lqcd_field *f, size_t *bytes)
{
    LQCD_REQUIRE(f && bytes, "NULL argument");
    *bytes = f->bytes + f->norm_bytes;
    return LQCD_OK;
}

lqcd_status lqcd_field_data(const lqcd_field *f, void **data_dev, void **norm_dev)
{
    LQCD_REQUIRE(f && data_dev, "NULL argument");
    *data_dev = f->data;
    if (norm_dev) *norm_dev = f->norm;
    return LQCD_OK;
}

lqcd_status lqcd_field_upload(lqcd_field *f, const double *host, void *stream)
{
    LQCD_REQUIRE(f && host, "NULL argument");
    return transfer(f, const_cast<double *>(host), true, (cudaStream_t)stream);
}

lqcd_status lqcd_field_download(const lqcd_field *f, double *host, void *stream)
{
    LQCD_REQUIRE(f && host, "NULL argument");
    return transfer(const_cast<lqcd_field *>(f), host, false, (cudaStream_t)stream);
}

lqcd_status lqcd_field_copy(lqcd_field *dst, const lqcd_field *src, void *stream)
{
    LQCD_REQUIRE(dst && src, "NULL argument");
    LQCD_REQUIRE(same_lattice(dst->lat, src->lat), "field_copy: lattices differ");
    cudaStream_t s = (cudaStream_t)stream;
    if (dst->kind == src->kind && dst->prec == src->prec) {
        LQCD_CUDA(cudaMemcpyAsync(dst->data, src->data, src->bytes, cudaMemcpyDeviceToDevice, s));
        if (src->norm) LQCD_CUDA(cudaMemcpyAsync(dst->norm, src->norm, src->norm_bytes, cudaMemcpyDeviceToDevice, s));
        return LQCD_OK;
    }
    if (dst->kind == LQCD_GAUGE && src->kind == LQCD_GAUGE) {
        switch (src->prec) {
        case LQCD_F64: launch_gauge_convert<LQCD_F64>(dst, src, s); break;
        case LQCD_F32: launch_gauge_convert<LQCD_F32>(dst, src, s); break;
        case LQCD_F16N: launch_gauge_convert<LQCD_F16N>(dst, src, s); break;
        case LQCD_BF16: launch_gauge_convert<LQCD_BF16>(dst, src, s); break;
        }
        LQCD_LAUNCHED();
        return LQCD_OK;
    }
    bool half_kinds = (dst->kind == LQCD_SPINOR_EVEN || dst->kind == LQCD_SPINOR_ODD) && dst->kind == src->kind;
    LQCD_REQUIRE(half_kinds, "field_copy: kinds %d -> %d not convertible", (int)src->kind, (int)dst->kind);
    switch (src->prec) {
    case LQCD_F64: launch_spinor_convert<LQCD_F64>(dst, src, s); break;
    case LQCD_F32: launch_spinor_convert<LQCD_F32>(dst, src, s); break;
    case LQCD_F16N: launch_spinor_convert<LQCD_F16N>(dst, src, s); break;
    case LQCD_BF16: launch_spinor_convert<LQCD_BF16>(dst, src, s); break;
    }
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status lqcd_philox_blocks(uint32_t *out_dev, size_t n_blocks, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                               uint32_t key0, uint32_t key1, void *stream)
{
    LQCD_REQUIRE(out_dev || n_blocks == 0, "out_dev is NULL");
    if (n_blocks == 0) return LQCD_OK;
    philox_blocks_kernel<<<nblocks_for((long)n_blocks, 256), 256, 0, (cudaStream_t)stream>>>((uint4 *)out_dev, n_blocks,
                                                                                              c0, c1, c2, c3, key0, key1);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status lqcd_df_split(const double *in_dev, size_t n, float *pairs_dev, double *back_dev, void *stream)
{
    LQCD_REQUIRE((in_dev && pairs_dev && back_dev) || n == 0, "df_split: NULL pointer");
    if (n == 0) return LQCD_OK;
    df_split_kernel<<<nblocks_for((long)n, 256), 256, 0, (cudaStream_t)stream>>>(in_dev, (float2 *)pairs_dev,
                                                                                 back_dev, n);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status lqcd_gauge_start(lqcd_field *U, uint32_t seed, uint32_t chain, double eps, void *stream)
{
    LQCD_REQUIRE(U && U->kind == LQCD_GAUGE && U->prec == LQCD_F64, "gauge_start needs an F64 gauge field");
    Geo g = make_geo(U->lat);
    int V = 2 * g.Vh;
    gauge_start_kernel<<<nblocks_for(V, 128), 128, 0, (cudaStream_t)stream>>>(gauge_ref<LQCD_F64>(U), g, V, seed, chain, eps);
    LQCD_LAUNCHED();
    return LQCD_OK;
}

lqcd_status lqcd_momentum_refresh(lqcd_field *P, uint32_t seed, uint32_t chain, uint32_t traj, void *stream)
{
    LQCD_REQUIRE(P && P->kind == LQCD_MOMENTUM, "momentum_refresh needs a momentum field");
    return momentum_refresh_dev(P, seed, chain, traj, (cudaStream_t)stream);
}

lqcd_status lqcd_eta_refresh(lqcd_field *eta, uint32_t seed, uint32_t chain, uint32_t traj, void *stream)
{
    LQCD_REQUIRE(eta && eta->kind == LQCD_SPINOR_EVEN && eta->prec == LQCD_F64, "eta_refresh needs an even F64 spinor");
    return eta_refresh_dev(eta, seed, chain, traj, (cudaStream_t)stream, 2u);
}

lqcd_status lqcd_link_update(lqcd_field *U, const lqcd_field *P, double c, lqcd_field *U_sloppy, void *stream)
{
    LQCD_REQUIRE(U && P && U->kind == LQCD_GAUGE && U->prec == LQCD_F64 && P->kind == LQCD_MOMENTUM,
                 "link_update needs an F64 gauge field and a momentum field");
    LQCD_REQUIRE(same_lattice(U->lat, P->lat), "link_update: lattices differ");
    if (U_sloppy)
        LQCD_REQUIRE(U_sloppy->kind == LQCD_GAUGE && U_sloppy->recon == 12 && same_lattice(U->lat, U_sloppy->lat),
                     "link_update: U_sloppy must be a 12-real gauge field on the same lattice");
    return link_update_dev(U, P, c, U_sloppy, nullptr, false, (cudaStream_t)stream, nullptr);
}

lqcd_status lqcd_link_update_ex(lqcd_field *U, const lqcd_field *P, double c, lqcd_field *U_sloppy, lqcd_prec arith,
                                void *stream)
{
    LQCD_REQUIRE(arith == LQCD_F64 || arith == LQCD_F32, "link_update_ex: arith must be F64 or F32");
    if (arith == LQCD_F64) return lqcd_link_update(U, P, c, U_sloppy, stream);
    LQCD_REQUIRE(U && P && U->kind == LQCD_GAUGE && U->prec == LQCD_F64 && P->kind == LQCD_MOMENTUM,
                 "link_update_ex needs an F64 gauge field and a momentum field");
    LQCD_REQUIRE(same_lattice(U->lat, P->lat), "link_update_ex: lattices differ");
    if (U_sloppy)
        LQCD_REQUIRE(U_sloppy->kind == LQCD_GAUGE && U_sloppy->recon == 12 && same_lattice(U->lat, U_sloppy->lat),
                     "link_update_ex: U_sloppy must be a 12-real gauge field on the same lattice");
    return link_update_dev(U, P, c, U_sloppy, nullptr, true, (cudaStream_t)stream, nullptr);
}

lqcd_status lqcd_reunitarize(lqcd_field *U, double *max_dev_out, void *stream)
{
    LQCD_REQUIRE(U && U->kind == LQCD_GAUGE && U->prec == LQCD_F64, "reunitarize needs an F64 gauge field");
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf part, out;
    LQCD_TRY(out.alloc(sizeof(double), s));
    LQCD_TRY(reunitarize_dev(U, (double *)out.p, part, s));
    double h = 0;
    LQCD_TRY(read_scalars((double *)out.p, &h, 1, s));
    if (max_dev_out) *max_dev_out = h;
    return LQCD_OK;
}

lqcd_status lqcd_plaquette(const lqcd_field *U, double *out, void *stream)
{
    LQCD_REQUIRE(U && out && U->kind == LQCD_GAUGE && U->prec == LQCD_F64, "plaquette needs an F64 gauge field");
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf part, res;
    LQCD_TRY(res.alloc(sizeof(double), s));
    LQCD_TRY(plaquette_sum(U, (double *)res.p, part, s, false));
    double h = 0;
    LQCD_TRY(read_scalars((double *)res.p, &h, 1, s));
    *out = h / (6.0 * 2.0 * U->Vh);
    return LQCD_OK;
}

lqcd_status lqcd_kinetic_energy(const lqcd_field *P, double *out, void *stream)
{
    LQCD_REQUIRE(P && out && P->kind == LQCD_MOMENTUM, "kinetic_energy needs a momentum field");
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf part, res;
    LQCD_TRY(res.alloc(sizeof(double), s));
    LQCD_TRY(kinetic_sum(P, (double *)res.p, part, s));
    double h = 0;
    LQCD_TRY(read_scalars((double *)res.p, &h, 1, s));
    *out = 0.5 * h;
    return LQCD_OK;
}

lqcd_status lqcd_spinor_dot(const lqcd_field *a, const lqcd_field *b, double *out, void *stream)
{
    LQCD_REQUIRE(a && b && out, "NULL argument");
    LQCD_REQUIRE(a->prec == LQCD_F64 && b->prec == LQCD_F64 && a->kind == b->kind &&
                     (a->kind == LQCD_SPINOR_EVEN || a->kind == LQCD_SPINOR_ODD || a->kind == LQCD_SPINOR_FULL) &&
                     same_lattice(a->lat, b->lat),
                 "spinor_dot needs two FP64 spinor fields of the same kind and lattice");
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf part, res;
    LQCD_TRY(res.alloc(sizeof(double), s));
    LQCD_TRY(spinor_dot_dev(a, b, (double *)res.p, part, s));
    return read_scalars((double *)res.p, out, 1, s);
}

} // extern "C"
