// Plan construction and bookkeeping of the crosscorr C ABI (host code).
//
// The plan derives the frequency resolution, FFT size and output-bin selection
// of Sec. III B 3-4 of the paper (delta-lambda_f = sqrt(6 mu_f/pi)/T_coh,
// N_FFT = 2^ceil(log2 N_FFT0), nu_R = delta-lambda_f dt' N_FFT,
// f_r* = remainder(-f_band/2, 1/T_FFT), k-bar = k0 + floor(nu_R k)) in FP64 on
// the host, splits the N_FFT-point transform into C cosets of L points that fit
// on chip, and copies the detector tables to the device.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <vector>

#include "common.cuh"

namespace {
thread_local std::string g_last_error;

bool is_int_multiple(double v, double dt, int64_t* out) {
    double q = v / dt;
    double r = nearbyint(q);
    if (fabs(q - r) > 1e-9 * fmax(1.0, fabs(q))) return false;
    *out = (int64_t)r;
    return true;
}

// remainder(a, b) = a - sgn(a) floor(|a|/|b|) |b| (the printed definition with the
// final |b| that makes it a remainder).
double paper_remainder(double a, double b) {
    if (a == 0.0) return 0.0;
    return a - copysign(1.0, a) * floor(fabs(a) / fabs(b)) * fabs(b);
}

template <typename T>
cc_status upload(cc_plan* p, const T* host, size_t n, const T** out) {
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
    if (e != cudaSuccess) return cc::cuda_fail(e, "cudaMalloc (plan tables)");
    p->dev_allocs.push_back(d);
    if (n) {
        e = cudaMemcpy(d, host, n * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cc::cuda_fail(e, "cudaMemcpy (plan tables)");
    }
    *out = (const T*)d;
    return CC_OK;
}
}  // namespace

namespace cc {

cc_status fail(cc_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

cc_status cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA;
}

cc_status ensure_workspace(cc_plan* p, size_t bytes) {
    if (p->ws_bytes >= bytes) return CC_OK;
    if (p->ws_external)
        return fail(CC_ERR_OOM, "caller workspace of " + std::to_string(p->ws_bytes) + " bytes; this call needs " +
                                    std::to_string(bytes));
    if (p->ws) {
        cudaFree(p->ws);
        p->ws = nullptr;
        p->ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&p->ws, bytes);
    if (e != cudaSuccess) {
        p->ws = nullptr;
        return cuda_fail(e, ("workspace allocation of " + std::to_string(bytes) + " bytes").c_str());
    }
    p->ws_bytes = bytes;
    return CC_OK;
}

int launch_blocks_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

static std::atomic<uint64_t> g_launches{0};
void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void timing_pair(cc_plan* plan, cudaEvent_t* start, cudaEvent_t* stop) {
    *start = *stop = nullptr;
    if (!plan->kernel_timing) return;
    if (2 * plan->timing_used + 2 > plan->timing_events.size()) {
        cudaEvent_t e[2];
        if (cudaEventCreate(&e[0]) != cudaSuccess) return;
        if (cudaEventCreate(&e[1]) != cudaSuccess) {
            cudaEventDestroy(e[0]);
            return;
        }
        plan->timing_events.push_back(e[0]);
        plan->timing_events.push_back(e[1]);
    }
    *start = plan->timing_events[2 * plan->timing_used];
    *stop = plan->timing_events[2 * plan->timing_used + 1];
    ++plan->timing_used;
}

}  // namespace cc

extern "C" {

const char* crosscorr_status_string(cc_status s) {
    switch (s) {
        case CC_OK: return "ok";
        case CC_ERR_INVALID: return "invalid argument";
        case CC_ERR_OOM: return "out of device memory";
        case CC_ERR_CUDA: return "CUDA error";
        case CC_ERR_TIMEOUT: return "device wait timed out";
        case CC_ERR_UNSUPPORTED: return "unsupported option";
    }
    return "unknown status";
}

const char* crosscorr_last_error(void) { return g_last_error.c_str(); }

uint64_t crosscorr_kernel_launches(void) { return cc::g_launches.load(); }

cc_status crosscorr_plan_set_workspace(cc_plan* plan, void* ws_dev, size_t ws_bytes) {
    if (!plan) return cc::fail(CC_ERR_INVALID, "plan is null");
    if (ws_dev && ((uintptr_t)ws_dev & 255)) return cc::fail(CC_ERR_INVALID, "workspace must be 256-byte aligned");
    if (plan->ws && !plan->ws_external) cudaFree(plan->ws);
    plan->ws = ws_dev;
    plan->ws_bytes = ws_dev ? ws_bytes : 0;
    plan->ws_external = ws_dev != nullptr;
    return CC_OK;
}

cc_status crosscorr_plan_set_tuning(cc_plan* plan, const cc_tuning* tuning) {
    if (!plan || !tuning) return cc::fail(CC_ERR_INVALID, "null argument to crosscorr_plan_set_tuning");
    if (tuning->batch_templates < 0 || tuning->chunk_waves < 0 || tuning->chunk_waves > 1000 ||
        (tuning->transform_len != 0 && tuning->transform_len != 4096))
        return cc::fail(CC_ERR_INVALID, "batch_templates >= 0, 0 <= chunk_waves <= 1000, transform_len 0 or 4096");
    if (tuning->transform_len == 4096 && plan->dp.C4 < 1)
        return cc::fail(CC_ERR_UNSUPPORTED, "transform_len 4096 needs N_FFT >= 4096");
    plan->tuning = *tuning;
    return CC_OK;
}

cc_status crosscorr_plan_set_kernel_timing(cc_plan* plan, int on) {
    if (!plan) return cc::fail(CC_ERR_INVALID, "plan is null");
    plan->kernel_timing = on != 0;
    return CC_OK;
}

cc_status crosscorr_plan_kernel_time(cc_plan* plan, double* ms, int64_t* launches) {
    if (!plan || !ms || !launches) return cc::fail(CC_ERR_INVALID, "null argument to crosscorr_plan_kernel_time");
    double tot = 0.0;
    const size_t n = plan->timing_used;
    plan->timing_used = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaError_t e = cudaEventSynchronize(plan->timing_events[2 * i + 1]);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, plan->timing_events[2 * i], plan->timing_events[2 * i + 1]);
        if (e != cudaSuccess) return cc::cuda_fail(e, "kernel timing events");
        tot += t;
    }
    *ms = tot;
    *launches = (int64_t)n;
    return CC_OK;
}

cc_status crosscorr_plan_set_wait_test(cc_plan* plan, int on) {
    if (!plan) return cc::fail(CC_ERR_INVALID, "plan is null");
    plan->dp.wait_test = on != 0;
    return CC_OK;
}

cc_status crosscorr_plan_check(cc_plan* plan, void* stream) {
    CC_NVTX_RANGE("crosscorr_plan_check");
    if (!plan) return cc::fail(CC_ERR_INVALID, "plan is null");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, plan->dp.err, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cc::cuda_fail(e, "reading the device error word");
    if (h == 0) return CC_OK;
    e = cudaMemsetAsync(plan->dp.err, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cc::cuda_fail(e, "clearing the device error word");
    return cc::fail(CC_ERR_TIMEOUT, "a kernel's bounded wait for its staged samples ran out; "
                                    "the results of the searches since the last check are invalid");
}

void crosscorr_plan_destroy(cc_plan* p) {
    if (!p) return;
    for (void* d : p->dev_allocs) cudaFree(d);
    if (p->ws && !p->ws_external) cudaFree(p->ws);
    for (cudaEvent_t e : p->timing_events) cudaEventDestroy(e);
    for (void* d : {p->demod_z, p->demod_w, p->demod_tw, p->demod_df, p->demod_kbar, p->demod_list, p->demod_boff})
        if (d) cudaFree(d);
    if (p->learned_w) cudaFree(p->learned_w);
    if (p->learned_taps) cudaFree(p->learned_taps);
    if (p->topk_ws) cudaFree(p->topk_ws);
    delete p;
}

cc_status crosscorr_plan(const cc_config* cfg, const cc_detector* dets, cc_plan** out) {
    CC_NVTX_RANGE("crosscorr_plan");
    using cc::fail;
    if (!cfg || !dets || !out) return fail(CC_ERR_INVALID, "null argument to crosscorr_plan");
    *out = nullptr;
    const cc_config& c = *cfg;
    if (c.n_det < 1 || c.n_det > CC_MAX_DET) return fail(CC_ERR_INVALID, "n_det must be 1..4");
    if (c.D < 1 || c.D > cc::MAX_D) return fail(CC_ERR_INVALID, "D must be 1..32");
    if (!(c.dt > 0) || !isfinite(c.dt)) return fail(CC_ERR_INVALID, "dt must be positive");
    if (c.n_samples < 1 || c.n_samples > (int64_t(1) << 30))
        return fail(CC_ERR_INVALID, "n_samples must be in [1, 2^30]");
    if (!(c.f_band > 0) || c.f_band > 1.0 / c.dt + 1e-12)
        return fail(CC_ERR_INVALID, "f_band must be in (0, 1/dt]");
    if (!(c.mu_f > 0) || !isfinite(c.mu_f)) return fail(CC_ERR_INVALID, "mu_f must be positive");
    if (!(c.T_max >= 0) || !isfinite(c.T_max)) return fail(CC_ERR_INVALID, "T_max must be >= 0");
    if (!isfinite(c.f_h) || !isfinite(c.t0)) return fail(CC_ERR_INVALID, "f_h and t0 must be finite");
    if (c.pair_mode < 0 || c.pair_mode > 2) return fail(CC_ERR_INVALID, "pair_mode must be 0..2");
    if (c.store != CC_STORE_FP32 && c.store != CC_STORE_BF16)
        return fail(CC_ERR_INVALID, "store must be CC_STORE_FP32 or CC_STORE_BF16");
    if (c.interp != CC_INTERP_EXACT && c.interp != CC_INTERP_LEARNED)
        return fail(CC_ERR_INVALID, "interp must be CC_INTERP_EXACT or CC_INTERP_LEARNED");
    int64_t nsft;
    if (!(c.T_sft > 0) || !is_int_multiple(c.T_sft, c.dt, &nsft) || nsft < 1)
        return fail(CC_ERR_INVALID, "T_sft must be a positive integer multiple of dt");

    cc_plan* p = new cc_plan();
    p->cfg = c;
    p->Q = c.n_det;
    const double dt = c.dt;
    p->T_short = c.T_short > 0 ? c.T_short : fmax(c.T_max, c.T_sft);
    if (!is_int_multiple(p->T_short, dt, &p->N_s) || p->N_s < 1) {
        delete p;
        return fail(CC_ERR_INVALID, "T_short must be a positive integer multiple of dt");
    }
    p->R = (int64_t)floor(c.T_max / p->T_short + 1e-9);
    p->M = c.n_samples / p->N_s;
    if (p->M < 1) {
        delete p;
        return fail(CC_ERR_INVALID, "n_samples shorter than one T_short segment");
    }
    p->N_tau = p->M * p->N_s;
    p->T_coh = 2.0 * c.T_max + p->T_short;
    p->dlf = sqrt(6.0 * c.mu_f / M_PI) / p->T_coh;
    const double df_load = 1.0 / dt;
    p->N_FFT0 = (df_load / p->dlf) * ceil(p->dlf * p->T_coh);
    if (!(p->N_FFT0 < 16777216.0)) {
        delete p;
        return fail(CC_ERR_UNSUPPORTED, "N_FFT above 2^24");
    }
    int64_t N = 1;
    while ((double)N < p->N_FFT0) N *= 2;
    p->N_FFT = N;
    p->T_FFT = (double)N * dt;
    p->nu_R = p->dlf * dt * (double)N;
    p->N_f = (int64_t)floor(c.f_band / p->dlf);
    if (p->N_f < 1) {
        delete p;
        return fail(CC_ERR_INVALID, "f_band narrower than one frequency bin");
    }
    p->f_r = paper_remainder(-c.f_band / 2.0, 1.0 / p->T_FFT);
    p->f_FFT = c.f_h + p->f_r - 0.5 / dt;
    p->k0 = (int64_t)floor((c.f_h - c.f_band / 2.0 - p->f_FFT) * p->T_FFT + 1e-9);
    p->kbar.resize(p->N_f);
    p->freq.resize(p->N_f);
    for (int64_t k = 0; k < p->N_f; ++k) {
        p->kbar[k] = p->k0 + (int64_t)floor(p->nu_R * (double)k);
        p->freq[k] = p->f_FFT + (double)p->kbar[k] / p->T_FFT;
    }
    if (p->kbar.back() - p->k0 >= N) {
        crosscorr_plan_destroy(p);
        return fail(CC_ERR_INVALID, "output band wider than the FFT");
    }

    // Cosets: X[b0 + C m + c] = L-point DFT of sum over r = pos (mod L) of
    // w_r exp(-2 pi i (b0 + c) r / N_FFT); L covers a segment when it fits on chip.
    int64_t L = 1;
    while (L < p->N_s) L *= 2;
    L = std::min<int64_t>(L, cc::MAX_L);
    L = std::min<int64_t>(L, N);
    L = std::max<int64_t>(L, 4);
    if (L > N) {
        crosscorr_plan_destroy(p);
        return fail(CC_ERR_INVALID, "N_FFT below 4");
    }
    p->L = L;
    p->C = N / L;
    int log2L = 0;
    while ((1LL << log2L) < L) ++log2L;

    // per-detector validation (all of it before the first CUDA call)
    cc::DevParams& dp = p->dp;
    memset(&dp, 0, sizeof(dp));
    for (int q = 0; q < p->Q; ++q) {
        const cc_detector& d = dets[q];
        int64_t abstep, abj0;
        if (!d.ssb_delay || d.n_eph < 2 || !(d.eph_dt > 0) || !isfinite(d.eph_t0)) {
            crosscorr_plan_destroy(p);
            return fail(CC_ERR_INVALID, "detector " + std::to_string(q) + ": bad ssb_delay table");
        }
        if (!d.a_tab || !d.b_tab || d.n_ab < 2 || !(d.ab_dt > 0) ||
            !is_int_multiple(d.ab_dt, dt, &abstep) || abstep < 1 || !is_int_multiple(d.ab_t0, dt, &abj0)) {
            crosscorr_plan_destroy(p);
            return fail(CC_ERR_INVALID, "detector " + std::to_string(q) +
                                            ": a/b tables need n_ab >= 2 and ab_dt, ab_t0 integer multiples of dt");
        }
        if (q == 0) {
            dp.n_ab_step = (int)abstep;
            dp.ab_j0 = abj0;
        } else if (abstep != dp.n_ab_step || abj0 != dp.ab_j0) {
            crosscorr_plan_destroy(p);
            return fail(CC_ERR_INVALID, "all detectors must share the a/b table grid");
        }
        if (!d.sigma || d.n_sigma < 1) {
            crosscorr_plan_destroy(p);
            return fail(CC_ERR_INVALID, "detector " + std::to_string(q) + ": empty sigma table");
        }
        for (int64_t i = 0; i < d.n_ab; ++i)
            if (!isfinite(d.a_tab[i]) || !isfinite(d.b_tab[i])) {
                crosscorr_plan_destroy(p);
                return fail(CC_ERR_INVALID, "non-finite antenna table entry");
            }
        for (int64_t i = 0; i < d.n_sigma; ++i)
            if (!(d.sigma[i] >= 0) || !isfinite(d.sigma[i])) {
                crosscorr_plan_destroy(p);
                return fail(CC_ERR_INVALID, "sigma entries must be finite and >= 0");
            }
        for (int64_t i = 0; i < d.n_eph; ++i)
            if (!isfinite(d.ssb_delay[i])) {
                crosscorr_plan_destroy(p);
                return fail(CC_ERR_INVALID, "non-finite ssb_delay entry");
            }
    }
    // upload
    for (int q = 0; q < p->Q; ++q) {
        const cc_detector& d = dets[q];
        std::vector<float> a(d.n_ab), b(d.n_ab), s2(d.n_sigma);
        std::vector<float2> sw(d.n_sigma);
        for (int64_t i = 0; i < d.n_ab; ++i) {
            a[i] = (float)d.a_tab[i];
            b[i] = (float)d.b_tab[i];
        }
        for (int64_t i = 0; i < d.n_sigma; ++i) {
            const double v = d.sigma[i] * d.sigma[i];
            s2[i] = (float)v;
            sw[i] = s2[i] > 0.f ? make_float2((float)v, (float)(1.0 / v)) : make_float2(0.f, 0.f);
        }
        std::vector<int> lc(d.n_sigma + 1, 0);
        for (int64_t i = 0; i < d.n_sigma; ++i) lc[i + 1] = lc[i] + (s2[i] > 0.f ? 1 : 0);
        cc_status st;
        if ((st = upload(p, d.ssb_delay, (size_t)d.n_eph, &dp.ssb[q])) != CC_OK ||
            (st = upload(p, a.data(), a.size(), &dp.atab[q])) != CC_OK ||
            (st = upload(p, b.data(), b.size(), &dp.btab[q])) != CC_OK ||
            (st = upload(p, sw.data(), sw.size(), &dp.sigw[q])) != CC_OK ||
            (st = upload(p, lc.data(), lc.size(), &dp.lockc[q])) != CC_OK) {
            crosscorr_plan_destroy(p);
            return st;
        }
        dp.eph_t0[q] = d.eph_t0;
        dp.eph_dt[q] = d.eph_dt;
        dp.inv_eph_dt[q] = 1.0 / d.eph_dt;
        dp.n_eph[q] = d.n_eph;
        dp.n_ab[q] = d.n_ab;
        dp.n_sig[q] = d.n_sigma;
    }

    // coset maps
    const int64_t C = p->C;
    std::vector<int> off(C + 1, 0), ck(p->N_f), cm(p->N_f);
    for (int64_t k = 0; k < p->N_f; ++k) off[(p->kbar[k] - p->k0) % C + 1]++;
    for (int64_t c2 = 0; c2 < C; ++c2) off[c2 + 1] += off[c2];
    std::vector<int> fillp(off.begin(), off.end() - 1);
    for (int64_t k = 0; k < p->N_f; ++k) {
        int64_t kp = p->kbar[k] - p->k0;
        int64_t cc2 = kp % C;
        ck[fillp[cc2]] = (int)k;
        cm[fillp[cc2]] = (int)(kp / C);
        fillp[cc2]++;
    }
    std::vector<float2> tw(L);
    for (int64_t j = 0; j < L; ++j) {
        double ang = -2.0 * M_PI * (double)j / (double)L;
        tw[j] = make_float2((float)cos(ang), (float)sin(ang));
    }
    const unsigned zero_word = 0;
    p->coset_off = off;
    // per-coset twiddles of the segment-local sample index (FP64 phase, exact integer index)
    const int64_t b0 = ((p->k0 - N / 2) % N + N) % N;
    std::vector<float2> twc((size_t)C * p->N_s);
    for (int64_t c2 = 0; c2 < C; ++c2) {
        const uint64_t bc = (uint64_t)((b0 + c2) % N);
        for (int64_t r = 0; r < p->N_s; ++r) {
            const uint64_t j = (bc * (uint64_t)r) % (uint64_t)N;
            const double ang = -2.0 * M_PI * (double)j / (double)N;
            twc[(size_t)c2 * p->N_s + r] = make_float2((float)cos(ang), (float)sin(ang));
        }
    }
    // Coset twiddles of the radix-16 passes of the persistent 4096-point kernel, per coset
    // c (bc = b0 + c): the coset twiddle W_N^(bc s) of sample s = t + 256 r (thread t of
    // the first pass) splits into W_N^(256 bc r), applied in the first pass, and the
    // thread factor W_N^(bc t), which passes through the first pass's DFT into the second
    // pass (element r' of second-pass thread j came from first-pass thread (j >> 4) + 16 r'):
    // its part W_N^(16 bc r') joins that pass's twiddle W_L^(16 k r') (k = j mod 16), and
    // its part W_N^(bc (j >> 4)) reaches the last pass as W_N^(bc r3) on element r3.
    // twk[c][r], r < 16: W_N^(256 bc r); twk[c][16 + 16 r + k]: W_N^(16 r (C4 k + bc)), for the
    // C4 = N_FFT / 4096 cosets of that kernel (C4 = C when the plan's coset length is 4096;
    // a plan with shorter cosets may still take it, its segments zero-padded to 4096).
    const int64_t C4 = N >= 4096 ? N / 4096 : 0;
    std::vector<float2> twk((size_t)std::max<int64_t>(C4, 1) * 272);
    for (int64_t c2 = 0; c2 < C4; ++c2) {
        const uint64_t bc = (uint64_t)((b0 + c2) % N);
        for (uint64_t r = 0; r < 16; ++r) {
            const uint64_t j = (256 * bc * r) % (uint64_t)N;
            const double ang = -2.0 * M_PI * (double)j / (double)N;
            twk[(size_t)c2 * 272 + r] = make_float2((float)cos(ang), (float)sin(ang));
            for (uint64_t k = 0; k < 16; ++k) {
                const uint64_t j2 = (16 * r * ((uint64_t)C4 * k + bc)) % (uint64_t)N;
                const double a2 = -2.0 * M_PI * (double)j2 / (double)N;
                twk[(size_t)c2 * 272 + 16 + 16 * r + k] = make_float2((float)cos(a2), (float)sin(a2));
            }
        }
    }
    // coset maps of the 4096-point decomposition (the same as the plan's when L = 4096)
    std::vector<int> off4, ck4, cm4;
    if (C4 > 0 && C4 != C) {
        off4.assign(C4 + 1, 0);
        ck4.resize(p->N_f);
        cm4.resize(p->N_f);
        for (int64_t k = 0; k < p->N_f; ++k) off4[(p->kbar[k] - p->k0) % C4 + 1]++;
        for (int64_t c2 = 0; c2 < C4; ++c2) off4[c2 + 1] += off4[c2];
        std::vector<int> fill4(off4.begin(), off4.end() - 1);
        for (int64_t k = 0; k < p->N_f; ++k) {
            const int64_t kp = p->kbar[k] - p->k0;
            ck4[fill4[kp % C4]] = (int)k;
            cm4[fill4[kp % C4]++] = (int)(kp / C4);
        }
    }
    cc_status st;
    if ((st = upload(p, twc.data(), twc.size(), &dp.twc)) != CC_OK ||
        (st = upload(p, off.data(), off.size(), &dp.coset_off)) != CC_OK ||
        (st = upload(p, ck.data(), ck.size(), &dp.coset_k)) != CC_OK ||
        (st = upload(p, cm.data(), cm.size(), &dp.coset_m)) != CC_OK ||
        (st = upload(p, tw.data(), tw.size(), &dp.twL)) != CC_OK ||
        (st = upload(p, twk.data(), twk.size(), &dp.twk)) != CC_OK ||
        (!off4.empty() && ((st = upload(p, off4.data(), off4.size(), &dp.coset4_off)) != CC_OK ||
                           (st = upload(p, ck4.data(), ck4.size(), &dp.coset4_k)) != CC_OK ||
                           (st = upload(p, cm4.data(), cm4.size(), &dp.coset4_m)) != CC_OK)) ||
        (st = upload(p, &zero_word, 1, (const unsigned**)&dp.err)) != CC_OK) {
        crosscorr_plan_destroy(p);
        return st;
    }

    dp.Q = p->Q;
    dp.D = c.D;
    dp.pair_mode = c.pair_mode;
    dp.store = c.store;
    dp.interp = c.interp;
    dp.ltaps = nullptr;   // crosscorr_plan_set_learned_interp fills it
    dp.L = (int)L;
    dp.C = (int)C;
    dp.C4 = (int)C4;
    if (C4 == C) {
        dp.coset4_off = dp.coset_off;
        dp.coset4_k = dp.coset_k;
        dp.coset4_m = dp.coset_m;
    }
    p->kbar_span4 = C4 > 0 ? (int)((p->kbar.back() - p->k0) / C4) : 0;
    if (C4 > 0) {
        void* ctr = nullptr;
        if (cudaMalloc(&ctr, sizeof(int) * C4) != cudaSuccess) {
            crosscorr_plan_destroy(p);
            return fail(CC_ERR_OOM, "unit counters");
        }
        p->dev_allocs.push_back(ctr);
        p->segfft_ctr = (int*)ctr;
    }
    dp.log2L = log2L;
    dp.nsft = (int)nsft;
    cc::magic_for((uint32_t)nsft, &dp.nsft_m, &dp.nsft_s);
    cc::magic_for((uint32_t)std::max(1, dp.n_ab_step), &dp.ab_m, &dp.ab_s);
    dp.N_t = c.n_samples;
    dp.N_s = p->N_s;
    dp.M = p->M;
    dp.R = p->R;
    dp.N_tau = p->N_tau;
    dp.N_FFT = N;
    dp.N_f = p->N_f;
    dp.b0 = ((p->k0 - N / 2) % N + N) % N;
    dp.dt = dt;
    dp.inv_dt = 1.0 / dt;
    dp.t0 = c.t0;
    dp.f_h = c.f_h;
    dp.f_r = p->f_r;
    dp.f_h_dt = (float)(c.f_h * dt);
    dp.f_r_dt = (float)(p->f_r * dt);
    for (int n = 0; n <= 2 * c.D; ++n)
        dp.ham[n] = (float)(0.54 - 0.46 * cos(2.0 * M_PI * (double)n / (double)(2 * c.D)));
    *out = p;
    return CC_OK;
}

cc_status crosscorr_plan_info(const cc_plan* p, cc_plan_info* info, double* freqs_host,
                              int64_t* kbar_host) {
    if (!p || !info) return cc::fail(CC_ERR_INVALID, "null argument to crosscorr_plan_info");
    info->N_s = p->N_s;
    info->M = p->M;
    info->R = p->R;
    info->N_tau = p->N_tau;
    info->N_FFT = p->N_FFT;
    info->N_f = p->N_f;
    info->k0 = p->k0;
    info->L = p->L;
    info->C = p->C;
    info->T_coh = p->T_coh;
    info->dlf = p->dlf;
    info->N_FFT0 = p->N_FFT0;
    info->T_FFT = p->T_FFT;
    info->nu_R = p->nu_R;
    info->f_r = p->f_r;
    info->f_FFT = p->f_FFT;
    info->ws_bytes = p->ws_bytes;
    if (freqs_host) memcpy(freqs_host, p->freq.data(), sizeof(double) * p->N_f);
    if (kbar_host) memcpy(kbar_host, p->kbar.data(), sizeof(int64_t) * p->N_f);
    return CC_OK;
}

}  // extern "C"
