// Fused search: host side (shared-memory layout, knot pre-pass, finalize, launch).
// The kernel itself is in fused_kernel.cuh, compiled per coset length in fused_l*.cu.
#include <algorithm>

#include "fused_kernel.cuh"

namespace cc {

// rho = sqrt(2) sum_chunks raw / sqrt(sum_chunks D).  With one chunk the caller passes
// raw == rho (the kernel scales rho in place: each thread reads its element before it
// writes it), so neither pointer is declared __restrict__.
__global__ void finalize_kernel(const float* raw, const double* __restrict__ dpart,
                                int64_t N_f, int n_chunks, int64_t t_base, float* rho) {
    const int64_t t = t_base + blockIdx.y;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N_f) return;
    double D = 0.0;
    for (int c = 0; c < n_chunks; ++c) D += dpart[(size_t)t * n_chunks + c];
    float s = 0.f, comp = 0.f;
    for (int c = 0; c < n_chunks; ++c) kahan_add(s, comp, raw[((size_t)t * n_chunks + c) * N_f + k]);
    rho[(size_t)t * N_f + k] = D > 0.0 ? (float)(1.4142135623730951 * (double)s / sqrt(D)) : 0.f;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static size_t al16(size_t b) { return (b + 15) & ~(size_t)15; }

bool fused_layout(const cc_plan* plan, int64_t n_t, FusedLayout* lay) {
    const DevParams& p = plan->dp;
    const int C = p.C;
    int CL = 1;
    while (CL * 2 <= std::min(C, MAX_CLUSTER)) CL *= 2;
    if (C % CL) return false;
    lay->CL = CL;
    const int nblk = (int)((p.N_s + KNOT - 1) / KNOT);
    lay->S = ((nblk + CL - 1) / CL) * KNOT;   // local samples: this CTA's KNOT-sample blocks
    lay->log2CL = 0;
    while ((1 << lay->log2CL) < CL) ++lay->log2CL;
    // bins per CTA: max over ranks of the sum of its cosets' list lengths
    int nb = 0;
    const std::vector<int>& off = plan->coset_off;
    for (int r = 0; r < CL; ++r) {
        int s = 0;
        for (int c = r; c < C; c += CL) s += off[c + 1] - off[c];
        nb = std::max(nb, s);
    }
    lay->nb = std::max(nb, 1);
    lay->nkseg = (int)(p.N_s / KNOT + 5);
    lay->nrec = 2 * ((nblk + CL - 1) / CL);
    lay->ring_q = p.pair_mode == CC_PAIRS_CROSS_ONLY ? p.Q : 1;
    const int ncos_max = (C + CL - 1) / CL;
    size_t o = 0;
    lay->off_slice = o;
    lay->slice_bytes = (size_t)2 * p.Q * 2 * lay->S * sizeof(float2);
    o = al16(o + lay->slice_bytes);
    lay->off_fft = o;
    lay->bothw = p.Q <= 2 ? 1 : 0;
    lay->mmax = plan->N_f > 0 ? (int)((plan->kbar.back() - plan->k0) / C) : 0;
    lay->regpair = (C == CL && p.Q <= 2 && p.R <= 1 && p.pair_mode != CC_PAIRS_CROSS_ONLY &&
                    2 * lay->mmax < p.L) ? 1 : 0;
    lay->regacc = (lay->regpair || (C == CL && lay->nb <= ACC_SLOTS * FUSED_THREADS)) ? 1 : 0;
    o = al16(o + (size_t)(lay->bothw ? 4 : 2) * padded_len(p.L) * sizeof(float2));
    lay->off_ring = o;
    const int64_t nslot = lay->regpair ? 0 : (lay->ring_q > 1 ? p.R + 1 : p.R);
    o = al16(o + (size_t)nslot * lay->ring_q * 2 * lay->nb * sizeof(float2));
    lay->off_same = o;
    o = al16(o + (size_t)(p.Q > 2 ? lay->nb : 0) * sizeof(float2));
    lay->off_rho = o;
    o = al16(o + (size_t)(lay->regacc ? 0 : 2 * lay->nb) * sizeof(float));
    lay->off_dk = o;
    o = al16(o + (size_t)2 * p.Q * lay->nkseg * sizeof(double));
    lay->off_rec = o;
    o = al16(o + (size_t)2 * p.Q * lay->nrec * sizeof(KnotRec));
    lay->off_wpart = o;
    o = al16(o + ((size_t)2 * FUSED_WARPS * p.Q * 4 + (size_t)MAX_CLUSTER * p.Q * 3) * sizeof(float));
    lay->off_nring = o;
    o = al16(o + (size_t)(p.R + 1) * p.Q * sizeof(float4));
    lay->off_bins = o;
    o = al16(o + (size_t)lay->nb * sizeof(int2) + (ncos_max + 1) * sizeof(int));
    lay->off_flags = o;
    o = al16(o + (size_t)SEGACT_DEPTH * CC_MAX_DET * sizeof(int));
    lay->bytes = o;
    if (lay->bytes > 227 * 1024) return false;
    if (p.L > 4096 || p.L < 64) return false;   // one radix-16 butterfly per thread per pass
    if ((int64_t)(p.R + 1) * p.Q > FUSED_THREADS) return false;
    // chunks: enough CTAs to fill the GPU, each chunk at least 4R + 1 segments
    int64_t ctas = (int64_t)C / (C / CL) * n_t;   // = CL * n_t clusters' CTAs
    const int64_t waves = plan->tuning.chunk_waves > 0 ? plan->tuning.chunk_waves : 4;
    int64_t want = std::max<int64_t>(1, (waves * 152 + ctas - 1) / std::max<int64_t>(ctas, 1));
    int64_t maxch = std::max<int64_t>(1, p.M / (4 * p.R + 1));
    int64_t nch = std::min(want, maxch);
    lay->chunk_len = (p.M + nch - 1) / nch;
    lay->n_chunks = (int)((p.M + lay->chunk_len - 1) / lay->chunk_len);
    return true;
}

// Knot records (FP64 delays at every KNOT-th source sample, four per record) for a batch
// of templates: one thread per record of every detector, the block's 256 records plus
// three halo knots.  The binary-orbit part of each delay is computed once for all
// detectors (it depends on the source time only); the barycentric part per detector.
__global__ void __launch_bounds__(256)
knots_kernel(DevParams p, const cc_template* __restrict__ tm, int64_t t_base, int64_t nkn,
             KnotRec* __restrict__ out) {
    __shared__ double dk[CC_MAX_DET][256 + 3];
    __shared__ Orbit orb_s;
    const int Q = p.Q;
    const int64_t tl = blockIdx.z, t = t_base + tl;
    const int64_t k0 = (int64_t)blockIdx.x * 256;
    // the orbit's FP64 set-up (a reciprocal, and trigonometry for e != 0) once per block
    if (threadIdx.x == 0) orb_s = make_orbit(p, tm[t]);
    __syncthreads();
    const Orbit orb = orb_s;
    for (int i = threadIdx.x; i < 256 + 3; i += 256) {
        const double tau = (double)((k0 - 1 + i) * KNOT) * p.dt;
        const double b = knot_binary(orb, tau);
        for (int X = 0; X < Q; ++X) dk[X][i] = knot_ssb(p, X, tau, b);
    }
    __syncthreads();
    const int64_t k = k0 + threadIdx.x;
    if (k < nkn)
        for (int X = 0; X < Q; ++X)
            out[((size_t)tl * Q + X) * nkn + k] =
                make_knot(p, dk[X][threadIdx.x], dk[X][threadIdx.x + 1], dk[X][threadIdx.x + 2],
                          dk[X][threadIdx.x + 3], (double)(k * KNOT) * p.dt);
}

int64_t knot_rows(const cc_plan* plan) { return (plan->N_tau + KNOT - 1) / KNOT; }

// Knot records of templates t_dev[0 .. n_t) into kn ([n_t][Q][knot_rows]).
cc_status launch_knots(cc_plan* plan, const cc_template* t_dev, int64_t n_t, KnotRec* kn, cudaStream_t st) {
    const DevParams& p = plan->dp;
    const int64_t nkn = knot_rows(plan);
    for (int64_t t0 = 0; t0 < n_t; t0 += 65535) {
        const int64_t nt = std::min<int64_t>(65535, n_t - t0);
        dim3 gk((unsigned)((nkn + 255) / 256), 1u, (unsigned)nt);
        knots_kernel<<<gk, 256, 0, st>>>(p, t_dev + t0, 0, nkn, kn + (size_t)t0 * p.Q * nkn);
        count_launch();
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CC_OK : cuda_fail(e, "knots launch");
}

#define CC_FOR_EACH_L(X) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

CC_FOR_EACH_L(CC_FUSED_EXTERN)

static const void* kernel_ptr(int L, bool pre, bool regpair) {
    switch (L) {
#define CC_CASE(LV) case LV: return fused_kernel_ptr<LV>(pre, regpair);
        CC_FOR_EACH_L(CC_CASE)
#undef CC_CASE
    }
    return nullptr;
}

static cudaError_t launch_dispatch(int L, const cudaLaunchConfig_t& cfg, bool pre, bool regpair,
                                   const DevParams& p, const FusedLayout& lay, const cc_template* t_dev,
                                   int64_t tb, float* raw, double* dpart, const KnotRec* kn, int64_t nkn) {
    switch (L) {
#define CC_CASE(LV) case LV: return launch_fused_lt<LV>(cfg, pre, regpair, p, lay, t_dev, tb, raw, dpart, kn, nkn);
        CC_FOR_EACH_L(CC_CASE)
#undef CC_CASE
    }
    return cudaErrorInvalidValue;
}

// kn_ws != nullptr: knot records from the pre-pass, kn_batch templates at a time (the
// workspace holds kn_batch * Q * knot_rows records); otherwise knots are computed in
// the fused kernel.
cc_status launch_fused(cc_plan* plan, const cc_template* t_dev, int64_t n_t, float* rho,
                       const FusedLayout& lay, float* raw, double* dpart, cudaStream_t st,
                       KnotRec* kn_ws, int64_t kn_batch) {
    const DevParams& p = plan->dp;
    const bool pre = kn_ws != nullptr;
    const void* fn = kernel_ptr(p.L, pre, lay.regpair != 0);
    if (!fn) return fail(CC_ERR_UNSUPPORTED, "no fused kernel for this coset length");
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.bytes);
    if (e != cudaSuccess) return cuda_fail(e, "fused smem attribute");
    const int64_t nkn = knot_rows(plan);
    const int64_t step = pre ? std::min<int64_t>(kn_batch, 65535) : 65535;
    for (int64_t tb = 0; tb < n_t; tb += step) {
        const int64_t nt = std::min(step, n_t - tb);
        if (pre) {
            dim3 gk((unsigned)((nkn + 255) / 256), 1u, (unsigned)nt);
            knots_kernel<<<gk, 256, 0, st>>>(p, t_dev, tb, nkn, kn_ws);
            count_launch();
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)lay.CL, (unsigned)lay.n_chunks, (unsigned)nt);
        cfg.blockDim = dim3(FUSED_THREADS);
        cfg.dynamicSmemBytes = lay.bytes;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = lay.CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaEvent_t ev0, ev1;
        timing_pair(plan, &ev0, &ev1);
        if (ev0) cudaEventRecord(ev0, st);
        e = launch_dispatch(p.L, cfg, pre, lay.regpair != 0, p, lay, t_dev, tb, raw, dpart, kn_ws, nkn);
        count_launch();
        if (ev1) cudaEventRecord(ev1, st);
        if (e != cudaSuccess) return cuda_fail(e, "fused launch");
        dim3 g2((unsigned)launch_blocks_for(p.N_f, 256), (unsigned)nt);
        finalize_kernel<<<g2, 256, 0, st>>>(raw, dpart, p.N_f, lay.n_chunks, tb, rho);
        count_launch();
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? CC_OK : cuda_fail(e, "fused launch");
}

}  // namespace cc
