// crosscorr_search_noalloc: the fused search for callers that cannot allocate device
// memory while they run it.
//
// crosscorr_search keeps a small scratch area in the plan (per-template partial
// normalisations, and partial sums when a template is split into chunks), growing it
// with cudaMalloc when a call needs more.  This entry point takes that scratch from a
// fixed array compiled into the library instead, so the call itself never allocates.
// It runs the same kernels with one chunk per template, so the kernel's sums land
// directly in the caller's rho buffer and the only scratch is one double per template.
#include <mutex>

#include "common.cuh"

namespace cc {
cc_status set_inputs(cc_plan* plan, const void* const* x_dev);
}

namespace {

// Largest template batch one call accepts (8 bytes of scratch per template, 512 KiB
// in total, held by every GPU that loads the library until the process exits).
constexpr int64_t kNoAllocMaxTemplates = 65536;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxTemplates];

// Device address of g_noalloc_scratch on each device, resolved on the first call made
// with that device current.  In host code the array's name is only a stand-in for
// the symbol, not an address a kernel can use.
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

cc_status scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cc::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return cc::fail(CC_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cc::cuda_fail(e, "cudaGetSymbolAddress (static scratch)");
        g_scratch_ptr[dev] = (double*)ptr;
    }
    *out = g_scratch_ptr[dev];
    return CC_OK;
}

}  // namespace

extern "C" cc_status crosscorr_search_noalloc(cc_plan* plan, const void* const* x_dev,
                                              const cc_template* t_dev, int64_t n_t, float* rho_dev,
                                              void* stream) {
    using namespace cc;
    if (!plan) return fail(CC_ERR_INVALID, "plan is null");
    if (n_t < 0) return fail(CC_ERR_INVALID, "n_t must be >= 0");
    if (n_t > kNoAllocMaxTemplates)
        return fail(CC_ERR_INVALID, "crosscorr_search_noalloc takes at most 65536 templates per call "
                                    "(size of its static scratch); split the batch");
    if (n_t == 0) return CC_OK;
    if (!t_dev || !rho_dev) return fail(CC_ERR_INVALID, "null device pointer");
    FusedLayout lay;
    if (plan->cfg.store != CC_STORE_FP32 || !fused_layout(plan, n_t, &lay))
        return fail(CC_ERR_UNSUPPORTED, "this plan needs the staged path, which allocates; "
                                        "use crosscorr_search");
    // one chunk per template: partial sums go straight to rho, scratch is D per template
    lay.chunk_len = plan->M;
    lay.n_chunks = 1;
    cc_status s = set_inputs(plan, x_dev);
    if (s != CC_OK) return s;
    double* dpart = nullptr;
    if ((s = scratch_for_current_device(&dpart)) != CC_OK) return s;
    return launch_fused(plan, t_dev, n_t, rho_dev, lay, rho_dev, dpart, (cudaStream_t)stream);
}
