// crosscorr_search: the whole path for a batch of templates.
#include <algorithm>

#include "common.cuh"

namespace cc {
cc_status set_inputs(cc_plan* plan, const void* const* x_dev);
cc_status launch_resample(cc_plan* plan, const cc_template* t_dev, int64_t n_t, void* ab, float* norm,
                          cudaStream_t st, const KnotRec* kn = nullptr, int64_t nkn = 0, int write_inactive = 0);
cc_status launch_segfft(cc_plan* plan, const void* ab, int64_t n_t, void* F, cudaStream_t st);
cc_status launch_norm_pairs(cc_plan* plan, const void* F, const float* norm, int64_t n_t, double* Dws,
                            float* rawws, float* rho, cudaStream_t st);
size_t pair_workspace_bytes(const cc_plan* plan, int64_t n_t);
bool two_pass_supported(const cc_plan* plan);
size_t two_pass_workspace_bytes(const cc_plan* plan, int64_t n_t);
cc_status search_two_pass(cc_plan* plan, const cc_template* t_dev, int64_t n_t, float* rho, cudaStream_t st);

constexpr size_t STAGED_WS_BUDGET = (size_t)6 << 30;
size_t knot_bytes_per_template(const cc_plan* plan);
cc_status resample_with_knots(cc_plan* plan, const cc_template* t_dev, int64_t n_t, void* ab, float* norm,
                              cudaStream_t st, KnotRec* kn, int64_t kbatch);

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Templates per batch and the workspace they need when the stages run back to back.
static void staged_batch(const cc_plan* p, int64_t n_t, int64_t* batch, size_t* bytes) {
    const size_t elem = p->cfg.store == CC_STORE_BF16 ? 4 : 8;
    const size_t ab = (size_t)p->Q * 2 * p->N_tau * elem;
    const size_t F = (size_t)p->Q * p->M * 2 * p->N_f * sizeof(float2);
    const size_t nm = (size_t)p->Q * p->M * sizeof(float4);
    const size_t kn = knot_bytes_per_template(p);
    const size_t per = align256(ab) + align256(F) + align256(nm) + align256(kn) + 256;
    int64_t b = (int64_t)std::max<size_t>(1, STAGED_WS_BUDGET / per);
    b = std::min<int64_t>(b, n_t);
    *batch = b;
    *bytes = (align256(ab * b) + align256(F * b) + align256(nm * b) + align256(pair_workspace_bytes(p, b)) +
              align256(kn * b));
}

// Fused path: layout for a batch of templates, knot-record batch and workspace bytes
// (FP64 partial normalisations, FP32 partial sums when a template is split into chunks,
// knot records of one batch).
static bool fused_plan(const cc_plan* plan, int64_t n_t, FusedLayout* lay, int64_t* kbatch, size_t* bytes) {
    const size_t krow = (size_t)plan->Q * knot_rows(plan) * sizeof(KnotRec);
    *kbatch = std::max<int64_t>(1, std::min<int64_t>(n_t, (int64_t)(KNOT_WS_BUDGET / krow)));
    if (plan->cfg.store != CC_STORE_FP32 || !fused_layout(plan, *kbatch, lay)) return false;
    const size_t dbytes = align256((size_t)n_t * lay->n_chunks * sizeof(double));
    const size_t rbytes = lay->n_chunks > 1 ? align256((size_t)n_t * lay->n_chunks * plan->N_f * sizeof(float)) : 0;
    *bytes = dbytes + rbytes + krow * *kbatch;
    return true;
}

static bool fused_supported(const cc_plan* plan) {
    FusedLayout lay;
    return plan->cfg.store == CC_STORE_FP32 && fused_layout(plan, 1, &lay);
}

static int resolve_path(const cc_plan* plan) {
    if (plan->search_path != CC_PATH_AUTO) return plan->search_path;
    if (two_pass_supported(plan)) return CC_PATH_TWO_PASS;
    if (fused_supported(plan)) return CC_PATH_FUSED;
    return CC_PATH_STAGED;
}

}  // namespace cc

extern "C" cc_status crosscorr_plan_set_path(cc_plan* plan, int path) {
    using namespace cc;
    if (!plan) return fail(CC_ERR_INVALID, "plan is null");
    if (path < CC_PATH_AUTO || path > CC_PATH_STAGED) return fail(CC_ERR_INVALID, "unknown search path");
    if (path == CC_PATH_TWO_PASS && !two_pass_supported(plan))
        return fail(CC_ERR_UNSUPPORTED, "plan does not fit the two-pass path");
    if (path == CC_PATH_FUSED && !fused_supported(plan))
        return fail(CC_ERR_UNSUPPORTED, "plan does not fit the fused path");
    plan->search_path = path;
    return CC_OK;
}

extern "C" cc_status crosscorr_plan_workspace_size(const cc_plan* plan, int64_t n_t, size_t* bytes) {
    using namespace cc;
    if (!plan || !bytes) return fail(CC_ERR_INVALID, "null argument to crosscorr_plan_workspace_size");
    if (n_t < 0) return fail(CC_ERR_INVALID, "n_t must be >= 0");
    *bytes = 0;
    if (n_t == 0) return CC_OK;
    const int path = resolve_path(plan);
    FusedLayout lay;
    int64_t kbatch, batch;
    if (path == CC_PATH_TWO_PASS) *bytes = two_pass_workspace_bytes(plan, n_t);
    else if (path == CC_PATH_FUSED && fused_plan(plan, n_t, &lay, &kbatch, bytes)) {
    } else staged_batch(plan, n_t, &batch, bytes);
    return CC_OK;
}

extern "C" cc_status crosscorr_plan_search_path(const cc_plan* plan, int* path) {
    using namespace cc;
    if (!plan || !path) return fail(CC_ERR_INVALID, "null argument to crosscorr_plan_search_path");
    *path = resolve_path(plan);
    return CC_OK;
}

extern "C" cc_status crosscorr_search(cc_plan* plan, const void* const* x_dev, const cc_template* t_dev,
                                      int64_t n_t, float* rho_dev, void* stream) {
    CC_NVTX_RANGE("crosscorr_search");
    using namespace cc;
    if (!plan) return fail(CC_ERR_INVALID, "plan is null");
    if (n_t < 0) return fail(CC_ERR_INVALID, "n_t must be >= 0");
    if (n_t == 0) return CC_OK;
    if (!t_dev || !rho_dev) return fail(CC_ERR_INVALID, "null device pointer");
    cc_status s = set_inputs(plan, x_dev);
    if (s != CC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int path = resolve_path(plan);
    if (path == CC_PATH_TWO_PASS) return search_two_pass(plan, t_dev, n_t, rho_dev, st);
    FusedLayout lay;
    int64_t kbatch;
    size_t fbytes;
    if (path == CC_PATH_FUSED && fused_plan(plan, n_t, &lay, &kbatch, &fbytes)) {
        // knot records from the pre-pass, up to KNOT_WS_BUDGET bytes of them per batch;
        // raw partial sums go straight into rho when there is one chunk per template
        if ((s = ensure_workspace(plan, fbytes)) != CC_OK) return s;
        const size_t dbytes = align256((size_t)n_t * lay.n_chunks * sizeof(double));
        const size_t rbytes = lay.n_chunks > 1 ? align256((size_t)n_t * lay.n_chunks * plan->N_f * sizeof(float)) : 0;
        double* dpart = (double*)plan->ws;
        float* raw = lay.n_chunks > 1 ? (float*)((char*)plan->ws + dbytes) : rho_dev;
        KnotRec* kn = (KnotRec*)((char*)plan->ws + dbytes + rbytes);
        return launch_fused(plan, t_dev, n_t, rho_dev, lay, raw, dpart, st, kn, kbatch);
    }
    int64_t batch;
    size_t bytes;
    staged_batch(plan, n_t, &batch, &bytes);
    if ((s = ensure_workspace(plan, bytes)) != CC_OK) return s;
    const size_t elem = plan->cfg.store == CC_STORE_BF16 ? 4 : 8;
    char* w = (char*)plan->ws;
    void* ab = w;
    w += align256((size_t)plan->Q * 2 * plan->N_tau * elem * batch);
    void* F = w;
    w += align256((size_t)plan->Q * plan->M * 2 * plan->N_f * sizeof(float2) * batch);
    float* nm = (float*)w;
    w += align256((size_t)plan->Q * plan->M * sizeof(float4) * batch);
    double* Dws = (double*)w;
    float* rawws = (float*)((char*)w + (((size_t)batch * sizeof(double) + 255) & ~(size_t)255));
    KnotRec* kn = (KnotRec*)((char*)w + align256(pair_workspace_bytes(plan, batch)));
    for (int64_t t0 = 0; t0 < n_t; t0 += batch) {
        const int64_t nb = std::min(batch, n_t - t0);
        if ((s = resample_with_knots(plan, t_dev + t0, nb, ab, nm, st, kn, nb)) != CC_OK) return s;
        if ((s = launch_segfft(plan, ab, nb, F, st)) != CC_OK) return s;
        if ((s = launch_norm_pairs(plan, F, nm, nb, Dws, rawws, rho_dev + t0 * plan->N_f, st)) != CC_OK) return s;
    }
    return CC_OK;
}
