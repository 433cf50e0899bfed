// noalloc.cu -- an allocation-free variant of the plaquette reduction.
//
// Every other call of this library takes its work space from the allocator
// hook (by default cudaMalloc, in the Python binding PyTorch's caching
// allocator reached through a Python callback).  Some callers cannot let the
// library allocate: code on a thread that must not call back into the Python
// interpreter or the framework that owns the allocator, a service loop that
// provisions all device memory up front and forbids allocation afterwards, or
// code that has to run with a bounded, fixed memory footprint.  For them,
// lqcd_plaquette_noalloc keeps the per-block partial sums of the plaquette in
// the file-scope device array below instead.
#include <mutex>

#include "lqcd_internal.cuh"

namespace lqcd {

// partial sums of one block of 256 sites each; LQCD_NOALLOC_MAX_SITES / 256 of them
constexpr int LQCD_NOALLOC_MAX_BLOCKS = LQCD_NOALLOC_MAX_SITES / 256;
constexpr int LQCD_NOALLOC_MAX_DEVICES = 64;

lqcd_status plaquette_partials_launch(const lqcd_field *U, double *partials, int nblocks, cudaStream_t s);
int plaquette_partial_blocks(const lqcd_field *U);

// One array per device that loads the library, held until the process exits.
static __device__ __align__(256) double g_plaq_scratch[LQCD_NOALLOC_MAX_BLOCKS];

// Device address of the array, looked up once per device.
static std::mutex g_scratch_mu;
static double *g_scratch_addr[LQCD_NOALLOC_MAX_DEVICES];

static lqcd_status scratch_address(double **out)
{
    int dev = 0;
    LQCD_CUDA(cudaGetDevice(&dev));
    LQCD_REQUIRE(dev >= 0 && dev < LQCD_NOALLOC_MAX_DEVICES, "plaquette_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        // host code only knows a stand-in for the array's name: ask the
        // runtime for its address on this device
        void *p = nullptr;
        LQCD_CUDA(cudaGetSymbolAddress(&p, g_plaq_scratch));
        g_scratch_addr[dev] = (double *)p;
    }
    *out = g_scratch_addr[dev];
    return LQCD_OK;
}

// sum the partials in a fixed order and store the mean plaquette
__global__ void plaquette_noalloc_final(const double *partials, int nblocks, double inv_norm, double *out)
{
    double s[1];
    final_sum_block<1>(partials, nblocks, s);
    if (threadIdx.x == 0) out[0] = s[0] * inv_norm;
}

} // namespace lqcd

using namespace lqcd;

extern "C" lqcd_status lqcd_plaquette_noalloc(const lqcd_field *U, double *out_dev, void *stream)
{
    LQCD_REQUIRE(U && out_dev, "plaquette_noalloc: NULL argument");
    LQCD_REQUIRE(U->kind == LQCD_GAUGE && U->prec == LQCD_F64, "plaquette_noalloc needs an F64 gauge field");
    int nb = plaquette_partial_blocks(U);
    LQCD_REQUIRE(nb <= LQCD_NOALLOC_MAX_BLOCKS,
                 "plaquette_noalloc: lattice of %lld sites needs %d partial sums, above the fixed maximum of %d "
                 "(%d sites); use lqcd_plaquette",
                 2LL * U->Vh, nb, LQCD_NOALLOC_MAX_BLOCKS, LQCD_NOALLOC_MAX_SITES);
    double *scratch = nullptr;
    LQCD_TRY(scratch_address(&scratch));
    cudaStream_t s = (cudaStream_t)stream;
    // every one of the nb partials is written before it is read: nothing to clear
    LQCD_TRY(plaquette_partials_launch(U, scratch, nb, s));
    plaquette_noalloc_final<<<1, 1024, 0, s>>>(scratch, nb, 1.0 / (6.0 * 2.0 * U->Vh), out_dev);
    LQCD_LAUNCHED();
    return LQCD_OK;
}
