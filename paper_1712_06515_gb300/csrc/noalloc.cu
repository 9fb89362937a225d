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

// Device address of g_noalloc_scratch in each device's current context, resolved on
// the first call made with that device current.  In host code the array's name is only
// a stand-in for the symbol, not an address a kernel can use.  The address belongs to
// the context the module was loaded into: after cudaDeviceReset (or any teardown of the
// primary context) the module is loaded again, possibly elsewhere, so the cache is keyed
// by the context's process-unique id and the next call resolves the address anew.
typedef int (*CtxGetCurrentFn)(void**);                        // cuCtxGetCurrent
typedef int (*CtxGetIdFn)(void*, unsigned long long*);         // cuCtxGetId

std::mutex g_mu;
struct ScratchEntry {
    unsigned long long ctx_id;   // 0: not resolved
    double* ptr;
};
ScratchEntry g_scratch[kMaxDevices] = {};
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

// Id of the context current on this thread, 0 when none is current yet.
cc_status current_context_id(unsigned long long* id) {
    *id = 0;
    if (!g_ctx_current || !g_ctx_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return cc::cuda_fail(e, "cudaGetDriverEntryPointByVersion");
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cc::fail(CC_ERR_CUDA, "driver entry points cuCtxGetCurrent/cuCtxGetId not found");
        g_ctx_current = (CtxGetCurrentFn)f1;
        g_ctx_id = (CtxGetIdFn)f2;
    }
    void* ctx = nullptr;
    if (g_ctx_current(&ctx) != 0) return cc::fail(CC_ERR_CUDA, "cuCtxGetCurrent failed");
    if (ctx && g_ctx_id(ctx, id) != 0) return cc::fail(CC_ERR_CUDA, "cuCtxGetId failed");
    return CC_OK;
}

cc_status scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cc::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return cc::fail(CC_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long id = 0;
    cc_status s = current_context_id(&id);
    if (s != CC_OK) return s;
    if (id == 0 || g_scratch[dev].ctx_id != id) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);   // makes the primary context current if needed
        if (e != cudaSuccess) return cc::cuda_fail(e, "cudaGetSymbolAddress (static scratch)");
        if ((s = current_context_id(&id)) != CC_OK) return s;
        g_scratch[dev].ctx_id = id;
        g_scratch[dev].ptr = (double*)ptr;
    }
    *out = g_scratch[dev].ptr;
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
