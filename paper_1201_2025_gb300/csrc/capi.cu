// C ABI of libwdad (declared in include/wdad.h): argument checking, the handle's
// workspace and plan caches, and dispatch to the kernels.  No exception leaves
// this file; every entry point returns a wdad_status.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cstdlib>
#include <map>

#include "batch.h"
#include "cnn.h"
#include "internal.h"

struct wdad_ctx {
    int device = 0;
    int num_sms = 1;
    void* ws = nullptr;        // grow-only device workspace
    size_t ws_bytes = 0;
    struct DwtPlan { int L, taps, J, K; float* A; };
    std::vector<DwtPlan> dwt_plans;
    std::map<long long, int> tuned;  // (D, inner, outer) -> autotuned tile height
    // second stream and events of the host entry point's row-band pipeline
    cudaStream_t aux = nullptr, aux2 = nullptr;
    std::vector<cudaEvent_t> evs;
    // the sequence entry point: its DWT stream (highest priority), ordering events and the
    // DWT's grid
    cudaStream_t seq = nullptr;
    cudaEvent_t seq_ev[5] = {};
    int seq_dwt_ctas = 0;
    std::string err;
};

struct wdad_cnn_ctx {
    wdad_ctx* h = nullptr;
    wdad::cnn::Net net;
};

// A job of at least kBatchDirectPixels pixels fills the GPU on its own: the batch runs it as
// its own DWT and detector launches (in the same graph), the smaller jobs in the persistent
// kernel.  Same kernels and plans as the single-cube entry points, so the same scores.
constexpr int64_t kBatchDirectPixels = 512 * 512;

struct BatchDirect {
    const float* cube;
    const float* A;
    int64_t P;
    int L, K, th;
    wdad::DetectArgs args;  // args.x = the job's approximation matrix
};

struct wdad_batch_ctx {
    wdad_ctx* h = nullptr;
    int n = 0;  // jobs in the persistent kernel
    int nitems = 0;
    size_t smem = 0;
    wdad::BatchJob* d_jobs = nullptr;
    wdad::BatchItem* d_items = nullptr;
    int* d_counters = nullptr;
    float* d_approx = nullptr;
    std::vector<int> th;  // every job's plan, in the caller's order
    std::vector<BatchDirect> direct;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t last = nullptr;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

wdad_status fail(wdad_ctx* h, wdad_status st, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
wdad_status fail(wdad_ctx* h, wdad_status st, const char* fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return st;
}

wdad_status cuda_fail(wdad_ctx* h, cudaError_t e, const char* where) {
    return fail(h, e == cudaErrorMemoryAllocation ? WDAD_ERR_NOMEM : WDAD_ERR_CUDA, "%s: %s", where,
                cudaGetErrorString(e));
}

wdad_status check_params(wdad_ctx* h, const wdad_params* p) {
    if (!p) return fail(h, WDAD_ERR_ARG, "params is NULL");
    if (p->wavelet_taps < 2 || p->wavelet_taps > wdad::kMaxTaps || (p->wavelet_taps & 1))
        return fail(h, WDAD_ERR_ARG, "wavelet_taps must be even, 2..%d (8 = db4), got %d", wdad::kMaxTaps,
                    p->wavelet_taps);
    if (p->level < -1 || p->level > 30) return fail(h, WDAD_ERR_ARG, "level must be -1..30, got %d", p->level);
    if (p->inner < 1 || !(p->inner & 1) || p->outer <= p->inner || !(p->outer & 1) || p->outer > 63)
        return fail(h, WDAD_ERR_ARG, "windows must be odd with 1 <= inner < outer <= 63, got %d/%d", p->inner,
                    p->outer);
    if (!(p->loading >= 0.f) || !std::isfinite(p->loading))
        return fail(h, WDAD_ERR_ARG, "loading must be finite and >= 0");
    if (!(p->cond_gate > 0.f)) return fail(h, WDAD_ERR_ARG, "cond_gate must be > 0");
    if (p->border != 0 && p->border != 1) return fail(h, WDAD_ERR_ARG, "border must be 0 or 1");
    if (p->dwest_mode != 0 && p->dwest_mode != 1) return fail(h, WDAD_ERR_ARG, "dwest_mode must be 0 or 1");
    if (p->precision < 0 || p->precision > 2) return fail(h, WDAD_ERR_ARG, "precision must be 0, 1 or 2");
    if (!(p->dwest_tau >= 0.f) || !std::isfinite(p->dwest_tau))
        return fail(h, WDAD_ERR_ARG, "dwest_tau must be finite and >= 0");
    return WDAD_OK;
}

wdad_status check_cube(wdad_ctx* h, const float* cube, int H, int W, int L) {
    if (H < 0 || W < 0) return fail(h, WDAD_ERR_ARG, "H and W must be >= 0, got %d x %d", H, W);
    if (L < 1) return fail(h, WDAD_ERR_ARG, "L must be >= 1, got %d", L);
    if ((int64_t)H * W > (int64_t)1 << 31) return fail(h, WDAD_ERR_ARG, "H*W above 2^31 pixels");
    if ((int64_t)H * W > 0 && !cube) return fail(h, WDAD_ERR_ARG, "cube is NULL");
    if (((uintptr_t)cube & 15) != 0 && (L % 4 == 0))
        return fail(h, WDAD_ERR_ARG, "cube must be 16-byte aligned");
    return WDAD_OK;
}

wdad_status ensure_ws(wdad_ctx* h, size_t bytes) {
    if (bytes <= h->ws_bytes) return WDAD_OK;
    if (h->ws) {
        cudaError_t e = cudaFree(h->ws);  // synchronises with work still using the old buffer
        h->ws = nullptr;
        h->ws_bytes = 0;
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaFree(workspace)");
    }
    size_t want = std::max(bytes, (size_t)1 << 20);
    cudaError_t e = cudaMalloc(&h->ws, want);
    if (e != cudaSuccess) {
        h->ws = nullptr;
        cudaGetLastError();
        return fail(h, WDAD_ERR_NOMEM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
    }
    h->ws_bytes = want;
    return WDAD_OK;
}

wdad_status get_dwt_plan(wdad_ctx* h, int L, int taps, int level, const float** A, int* K, cudaStream_t s) {
    int k = 0;
    const int J = wdad::dwt_levels(L, level, &k);
    for (auto& p : h->dwt_plans)
        if (p.L == L && p.taps == taps && p.J == J) { *A = p.A; *K = p.K; return WDAD_OK; }
    if (!wdad::dwt_shape_supported(L, k))
        return fail(h, WDAD_ERR_UNSUPPORTED, "DWT with L=%d, K=%d: L <= 1024 (L%%4==0) or L <= 256, K <= 8", L, k);
    float* Am = nullptr;
    cudaError_t e = cudaMalloc(&Am, sizeof(float) * (size_t)k * L);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(dwt matrix)");
    e = wdad::build_dwt_matrix(L, taps, J, k, Am, nullptr, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // later calls may use another stream
    if (e != cudaSuccess) { cudaFree(Am); return cuda_fail(h, e, "build_dwt_matrix"); }
    h->dwt_plans.push_back({L, taps, J, k, Am});
    *A = Am;
    *K = k;
    return WDAD_OK;
}

// Detectors on a D-band device cube x (the reduced cube, or the full-band cube).
wdad_status detect_bands(wdad_ctx* h, const float* x, int H, int W, int D, const wdad_params* p, float* out3[3],
                         uint8_t* flags, void* ws, size_t ws_bytes, cudaStream_t s) {
    if (D <= 8) {
        wdad::DetectArgs a{};
        a.x = x; a.H = H; a.W = W; a.D = D;
        a.inner = p->inner; a.outer = p->outer; a.loading = p->loading; a.border = p->border;
        a.dwest_mode = p->dwest_mode; a.dwest_tau = p->dwest_tau;
        for (int t = 0; t < 3; ++t) a.out[t] = out3[t];
        a.flags = flags;
        if (wdad::detect_small_smem(D, p->inner, p->outer, 1) > 227 * 1024)
            return fail(h, WDAD_ERR_UNSUPPORTED, "window %d/%d too large for %d bands", p->inner, p->outer, D);
        cudaError_t e = wdad::launch_detect_small_th(a, wdad::detect_small_default_th(D, p->inner, p->outer), s);
        if (e != cudaSuccess) return cuda_fail(h, e, "detect_small launch");
        return WDAD_OK;
    }
    wdad::FullArgs a{};
    a.x = x; a.H = H; a.W = W; a.D = D;
    a.inner = p->inner; a.outer = p->outer; a.loading = p->loading; a.cond_gate = p->cond_gate;
    a.border = p->border; a.dwest_mode = p->dwest_mode; a.precision = p->precision; a.dwest_tau = p->dwest_tau;
    for (int t = 0; t < 3; ++t) a.out[t] = out3[t];
    a.flags = flags;
    const size_t need = wdad::fullband_workspace_bytes(a, h->num_sms);
    if (need == 0) return fail(h, WDAD_ERR_UNSUPPORTED, "full-band detectors for %d bands are not supported", D);
    if (need > ws_bytes) return fail(h, WDAD_ERR_NOMEM, "full-band workspace of %zu bytes not available", need);
    cudaError_t e = wdad::launch_detect_full(a, ws, need, h->num_sms, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "detect_full launch");
    return WDAD_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// nwin windows of all three detectors on a D-band device cube x: out[w] = [3][H][W] at
// out + w * 3 * H * W, flags (nullable) [nwin][H][W].  D <= 8: the windows go in groups of up
// to four into single launches; larger D: one full-band pass per window (scratch: ws).
wdad_status detect_windows(wdad_ctx* h, const float* x, int H, int W, int D, int nwin, const wdad_params* params,
                           float* out, uint8_t* flags, void* ws, size_t ws_bytes, cudaStream_t s) {
    const size_t P = (size_t)H * W;
    if (D <= 8) {
        for (int w0 = 0; w0 < nwin; w0 += wdad::kMaxWindowsPerLaunch) {
            const int n = std::min(wdad::kMaxWindowsPerLaunch, nwin - w0);
            wdad::DetectArgs a[wdad::kMaxWindowsPerLaunch];
            for (int i = 0; i < n; ++i) {
                const wdad_params* p = &params[w0 + i];
                if (wdad::detect_small_smem(D, p->inner, p->outer, 1) > 227 * 1024)
                    return fail(h, WDAD_ERR_UNSUPPORTED, "window %d/%d too large for %d bands", p->inner, p->outer, D);
                a[i] = wdad::DetectArgs{};
                a[i].x = x; a[i].H = H; a[i].W = W; a[i].D = D;
                a[i].inner = p->inner; a[i].outer = p->outer; a[i].loading = p->loading; a[i].border = p->border;
                a[i].dwest_mode = p->dwest_mode; a[i].dwest_tau = p->dwest_tau;
                float* o = out + (size_t)(w0 + i) * 3 * P;
                a[i].out[0] = o; a[i].out[1] = o + P; a[i].out[2] = o + 2 * P;
                a[i].flags = flags ? flags + (size_t)(w0 + i) * P : nullptr;
            }
            cudaError_t e = wdad::launch_detect_small_multi(a, n, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "detect_small (windows) launch");
        }
        return WDAD_OK;
    }
    for (int w = 0; w < nwin; ++w) {
        float* o = out + (size_t)w * 3 * P;
        float* out3[3] = {o, o + P, o + 2 * P};
        wdad_status st = detect_bands(h, x, H, W, D, &params[w], out3, flags ? flags + (size_t)w * P : nullptr, ws,
                                      ws_bytes, s);
        if (st != WDAD_OK) return st;
    }
    return WDAD_OK;
}

wdad_status full_ws_need(wdad_ctx* h, int H, int W, int D, const wdad_params* p, size_t* need) {
    *need = 0;
    if (D <= 8) return WDAD_OK;
    wdad::FullArgs a{};
    a.H = H; a.W = W; a.D = D; a.inner = p->inner; a.outer = p->outer; a.precision = p->precision;
    *need = wdad::fullband_workspace_bytes(a, h->num_sms);
    if (*need == 0) return fail(h, WDAD_ERR_UNSUPPORTED, "full-band detectors for %d bands are not supported", D);
    return WDAD_OK;
}

wdad_status run_detect(wdad_ctx* h, const float* cube, int H, int W, int L, int reduce, const wdad_params* p,
                       float* out3[3], uint8_t* flags, cudaStream_t s) {
    wdad_status st = check_params(h, p);
    if (st != WDAD_OK) return st;
    st = check_cube(h, cube, H, W, L);
    if (st != WDAD_OK) return st;
    if (reduce != 0 && reduce != 1) return fail(h, WDAD_ERR_ARG, "reduce must be 0 or 1");
    if ((int64_t)H * W == 0) return WDAD_OK;
    const int64_t P = (int64_t)H * W;
    if (!reduce) {
        size_t need = 0;
        st = full_ws_need(h, H, W, L, p, &need);
        if (st != WDAD_OK) return st;
        if (need) {
            st = ensure_ws(h, need);
            if (st != WDAD_OK) return st;
        }
        return detect_bands(h, cube, H, W, L, p, out3, flags, h->ws, h->ws_bytes, s);
    }
    const int K = wdad_query_K(L, p->wavelet_taps, p->level);
    size_t need = 0;
    st = full_ws_need(h, H, W, K, p, &need);
    if (st != WDAD_OK) return st;
    const size_t off = align256(sizeof(float) * (size_t)P * K);
    st = ensure_ws(h, off + need);
    if (st != WDAD_OK) return st;
    const float* A = nullptr;
    int k2 = 0;
    st = get_dwt_plan(h, L, p->wavelet_taps, p->level, &A, &k2, s);
    if (st != WDAD_OK) return st;
    float* xr = (float*)h->ws;
    cudaError_t e = wdad::launch_dwt_approx(cube, P, L, A, K, xr, h->num_sms, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "dwt_approx launch");
    return detect_bands(h, xr, H, W, K, p, out3, flags, (char*)h->ws + off, h->ws_bytes - off, s);
}

long long tune_key(int D, int inner, int outer) { return ((long long)D << 32) | ((long long)inner << 16) | outer; }

__global__ void fill_pattern_kernel(float* x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t v = (uint32_t)(i * 2654435761u) ^ (uint32_t)(i >> 7) * 40503u;
        v ^= v >> 13;
        v *= 0x5bd1e995u;
        v ^= v >> 15;
        x[i] = 1.0f + 0.25f * (float)(v & 0xFFFFFF) / 16777216.0f;
    }
}

// Tile height for D bands, a window and a cube shape, by measurement.  The candidates are every
// height from 16 down to 4 rows that fits shared memory (two_per_sm: only plans that keep two
// CTAs on an SM, since the batch kernel sizes one plan for all of its jobs), timed on a
// synthetic cube of the given shape (at most 1024 x 1024 pixels) with CUDA events,
// median of five launches after two warm-ups.  The default plan (the tallest tile that keeps
// two CTAs per SM) is the incumbent: another height replaces it only when it is at least 3%
// faster, so a tuned plan is never slower than the default by more than the timing noise.
// Heights above 16 are not candidates: the sliding sums restart every th rows, and taller
// tiles accumulate more FP32 rounding than the parity bars allow.  The block size follows the
// height (one thread per output pixel, 512 threads at 16 rows): layouts with two pixels per
// thread (256 or 384 threads per CTA) measured 5-15% slower on the 512 x 512 workload.
wdad_status autotune(wdad_ctx* h, int D, int inner, int outer, int H, int W, int* out, cudaStream_t s,
                     bool two_per_sm = false) {
    H = std::max(32, std::min(H > 0 ? H : 256, 1024));
    W = std::max(32, std::min(W > 0 ? W : 256, 1024));
    // shape class: the next power of two of each side
    int hb = 32, wb = 32;
    while (hb < H) hb <<= 1;
    while (wb < W) wb <<= 1;
    const long long key = ((tune_key(D, inner, outer) * 2 + (two_per_sm ? 1 : 0)) << 8) ^ ((long long)hb << 4) ^ wb;
    auto it = h->tuned.find(key);
    if (it != h->tuned.end()) { *out = it->second; return WDAD_OK; }
    H = hb;
    W = wb;
    const size_t nx = (size_t)H * W * D, ns = (size_t)3 * H * W;
    wdad_status st = ensure_ws(h, sizeof(float) * (nx + ns) + 256);
    if (st != WDAD_OK) return st;
    float* x = (float*)h->ws;
    float* sc = x + nx;
    fill_pattern_kernel<<<256, 256, 0, s>>>(x, (int64_t)nx);
    wdad::DetectArgs a{};
    a.x = x; a.H = H; a.W = W; a.D = D; a.inner = inner; a.outer = outer; a.loading = 1e-3f;
    a.dwest_tau = 1e-6f;
    for (int t = 0; t < 3; ++t) a.out[t] = sc + (size_t)t * H * W;
    cudaEvent_t ev[6];
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(h, WDAD_ERR_CUDA, "autotune events");
    auto feasible = [&](int th) {
        const size_t need = wdad::detect_small_smem(D, inner, outer, th);
        return need <= 227 * 1024 && (!two_per_sm || need <= wdad::detect_small_two_per_sm_bytes());
    };
    auto time_plan = [&](int th) -> float {
        for (int r = 0; r < 2; ++r)
            if (wdad::launch_detect_small_th(a, th, s) != cudaSuccess) { cudaGetLastError(); return -1.f; }
        float t[5];
        for (int r = 0; r < 5; ++r) {
            cudaEventRecord(ev[r], s);
            wdad::launch_detect_small_th(a, th, s);
            cudaEventRecord(ev[r + 1], s);
            if (cudaEventSynchronize(ev[r + 1]) != cudaSuccess) return -1.f;
            cudaEventElapsedTime(&t[r], ev[r], ev[r + 1]);
        }
        std::sort(t, t + 5);
        return t[2];
    };
    const int th_default = wdad::detect_small_default_th(D, inner, outer);
    int best = 0;
    float best_ms = 1e30f;
    if (th_default > 0 && feasible(th_default)) {
        const float ms = time_plan(th_default);
        if (ms > 0.f) { best = th_default; best_ms = ms; }
    }
    const float incumbent = best_ms;
    int challenger = 0;
    float challenger_ms = 1e30f;
    for (int th = 16; th >= 4; --th) {
        if (th == th_default || !feasible(th)) continue;
        const float ms = time_plan(th);
        if (ms > 0.f && ms < challenger_ms) { challenger_ms = ms; challenger = th; }
    }
    if (challenger && (best == 0 || challenger_ms < 0.97f * incumbent)) { best = challenger; best_ms = challenger_ms; }
    for (auto& e : ev) cudaEventDestroy(e);
    if (best == 0 && two_per_sm) return autotune(h, D, inner, outer, H, W, out, s, false);
    if (best == 0) return fail(h, WDAD_ERR_UNSUPPORTED, "no tile height fits window %d/%d for %d bands", inner, outer, D);
    h->tuned[key] = best;
    *out = best;
    return WDAD_OK;
}

void cnn_free(wdad_cnn_ctx* c) {
    if (!c) return;
    auto& n = c->net;
    cudaFree(n.w); cudaFree(n.wf); cudaFree(n.m); cudaFree(n.v); cudaFree(n.grad); cudaFree(n.wt);
    cudaFree(n.norm); cudaFree(n.stat); cudaFree(n.act); cudaFree(n.loss); cudaFree(n.cx); cudaFree(n.ct);
    cudaFree(n.wpk); cudaFree(n.tcerr); cudaFree(n.gpart);
    delete c;
}

// magic, version, K, bf16, step, norm_mode, nparam (u64), then w, m, v (float32), norm (K + K*K float32)
constexpr uint32_t kCnnMagic = 0x4E4E4357u;  // "WCNN"
constexpr uint32_t kCnnVersion = 2;

void batch_free(wdad_batch_ctx* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->last) cudaEventDestroy(b->last);
    cudaFree(b->d_jobs);
    cudaFree(b->d_items);
    cudaFree(b->d_counters);
    cudaFree(b->d_approx);
    delete b;
}

}  // namespace

extern "C" {

void wdad_default_params(wdad_params* p) {
    if (!p) return;
    p->wavelet_taps = 8;
    p->level = -1;
    p->inner = 3;
    p->outer = 11;
    p->loading = 1e-3f;
    p->cond_gate = 1e6f;
    p->border = 0;
    p->dwest_mode = 0;
    p->precision = WDAD_PREC_FP32;
    p->dwest_tau = 1e-6f;
}

wdad_status wdad_create(wdad_handle* out, int device) {
    if (!out) return WDAD_ERR_ARG;
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) { cudaGetLastError(); return WDAD_ERR_CUDA; }
    if (device < 0 || device >= n) return WDAD_ERR_ARG;
    wdad_ctx* h = new (std::nothrow) wdad_ctx();
    if (!h) return WDAD_ERR_NOMEM;
    h->device = device;
    if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        h->num_sms = 1;
    h->seq_dwt_ctas = std::max(1, 3 * h->num_sms / 4);
    *out = h;
    return WDAD_OK;
}

wdad_status wdad_destroy(wdad_handle h) {
    if (!h) return WDAD_ERR_ARG;
    {
        DeviceGuard g(h->device);
        cudaDeviceSynchronize();
        if (h->ws) cudaFree(h->ws);
        for (auto& p : h->dwt_plans) cudaFree(p.A);
        for (auto e : h->evs) cudaEventDestroy(e);
        if (h->aux) cudaStreamDestroy(h->aux);
        if (h->aux2) cudaStreamDestroy(h->aux2);
        for (auto e : h->seq_ev)
            if (e) cudaEventDestroy(e);
        if (h->seq) cudaStreamDestroy(h->seq);
    }
    delete h;
    return WDAD_OK;
}

wdad_status wdad_last_error_detail(wdad_handle h, char* buf, int len) {
    if (!h || !buf || len <= 0) return WDAD_ERR_ARG;
    std::snprintf(buf, (size_t)len, "%s", h->err.c_str());
    return WDAD_OK;
}

int wdad_query_K(int L, int taps, int level) {
    if (L < 1 || taps < 2 || taps > wdad::kMaxTaps || (taps & 1) || level < -1 || level > 30) return -1;
    int K = 0;
    wdad::dwt_levels(L, level, &K);
    return K;
}

wdad_status wdad_global_rx(wdad_handle h, const float* cube, int H, int W, int L, int reduce, const wdad_params* p,
                           float* score, void* stream) {
    if (!h) return WDAD_ERR_ARG;
    try {
        DeviceGuard g(h->device);
        wdad_status st = check_params(h, p);
        if (st != WDAD_OK) return st;
        st = check_cube(h, cube, H, W, L);
        if (st != WDAD_OK) return st;
        if (reduce != 0 && reduce != 1) return fail(h, WDAD_ERR_ARG, "reduce must be 0 or 1");
        const int64_t P = (int64_t)H * W;
        if (P == 0) return WDAD_OK;
        if (!score) return fail(h, WDAD_ERR_ARG, "score is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        const int D = reduce ? wdad_query_K(L, p->wavelet_taps, p->level) : L;
        if (D < 1 || D > wdad::kGlobalRxMaxBands)
            return fail(h, WDAD_ERR_UNSUPPORTED, "global RX supports 1..%d bands, got %d", wdad::kGlobalRxMaxBands, D);
        const size_t need = wdad::global_rx_workspace_bytes(P, D, h->num_sms);
        if (need == 0) return fail(h, WDAD_ERR_UNSUPPORTED, "global RX workspace for %d bands", D);
        const size_t off = reduce ? align256(sizeof(float) * (size_t)P * D) : 0;
        st = ensure_ws(h, off + need);
        if (st != WDAD_OK) return st;
        const float* x = cube;
        if (reduce) {
            const float* A = nullptr;
            int k2 = 0;
            st = get_dwt_plan(h, L, p->wavelet_taps, p->level, &A, &k2, s);
            if (st != WDAD_OK) return st;
            float* xr = (float*)h->ws;
            cudaError_t e = wdad::launch_dwt_approx(cube, P, L, A, D, xr, h->num_sms, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "dwt_approx launch");
            x = xr;
        }
        cudaError_t e = wdad::launch_global_rx(x, P, D, p->loading, score, (char*)h->ws + off, h->ws_bytes - off,
                                               h->num_sms, s);
        return e == cudaSuccess ? WDAD_OK : cuda_fail(h, e, "global RX launch");
    } catch (...) {
        return fail(h, WDAD_ERR_NOMEM, "host exception");
    }
}

wdad_status wdad_wavelet_filter(int taps, double* h) {
    if (!h) return WDAD_ERR_ARG;
    return wdad::filter_coeffs(taps, h) ? WDAD_OK : WDAD_ERR_ARG;
}

wdad_status wdad_dwt_approx(wdad_handle h, const float* cube, int H, int W, int L, const wdad_params* p,
                            float* approx, int* K_out, void* stream) {
    if (!h) return WDAD_ERR_ARG;
    try {
        DeviceGuard g(h->device);
        wdad_status st = check_params(h, p);
        if (st != WDAD_OK) return st;
        st = check_cube(h, cube, H, W, L);
        if (st != WDAD_OK) return st;
        const int K = wdad_query_K(L, p->wavelet_taps, p->level);
        if (K_out) *K_out = K;
        const int64_t P = (int64_t)H * W;
        if (P == 0) return WDAD_OK;
        if (!approx) return fail(h, WDAD_ERR_ARG, "approx is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        const float* A = nullptr;
        int k2 = 0;
        st = get_dwt_plan(h, L, p->wavelet_taps, p->level, &A, &k2, s);
        if (st != WDAD_OK) return st;
        cudaError_t e = wdad::launch_dwt_approx(cube, P, L, A, k2, approx, h->num_sms, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "dwt_approx launch");
        return WDAD_OK;
    } catch (...) {
        return fail(h, WDAD_ERR_NOMEM, "host exception");
    }
}

wdad_status wdad_detect(wdad_handle h, const float* cube, int H, int W, int L, int detector, int reduce,
                        const wdad_params* p, float* score, uint8_t* flags, void* stream) {
    if (!h) return WDAD_ERR_ARG;
    if (detector < 0 || detector > 2) return fail(h, WDAD_ERR_ARG, "detector must be 0 (LRX), 1 (DWRX) or 2 (DWEST)");
    if ((int64_t)H * W > 0 && !score) return fail(h, WDAD_ERR_ARG, "score is NULL");
    try {
        DeviceGuard g(h->device);
        float* out3[3] = {nullptr, nullptr, nullptr};
        out3[detector] = score;
        return run_detect(h, cube, H, W, L, reduce, p, out3, flags, (cudaStream_t)stream);
    } catch (...) {
        return fail(h, WDAD_ERR_NOMEM, "host exception");
    }
}

wdad_status wdad_detect_all(wdad_handle h, const float* cube, int H, int W, int L, int reduce,
                            const wdad_params* p, float* scores, uint8_t* flags, void* stream) {
    if (!h) return WDAD_ERR_ARG;
    if ((int64_t)H * W > 0 && !scores) return fail(h, WDAD_ERR_ARG, "scores is NULL");
    try {
        DeviceGuard g(h->device);
        const size_t P = (size_t)H * W;
        float* out3[3] = {scores, scores + P, scores + 2 * P};
        return run_detect(h, cube, H, W, L, reduce, p, out3, flags, (cudaStream_t)stream);
    } catch (...) {
        return fail(h, WDAD_ERR_NOMEM, "host exception");
    }
}

wdad_status wdad_detect_windows(wdad_handle h, const float* cube, int H, int W, int L, int reduce, int nwin,
                                const wdad_params* params, float* scores, uint8_t* flags, void* stream) {
    if (!h) return WDAD_ERR_ARG;
    if (nwin < 1 || nwin > 64 || !params) return fail(h, WDAD_ERR_ARG, "nwin must be 1..64 with params[nwin]");
    if (reduce != 0 && reduce != 1) return fail(h, WDAD_ERR_ARG, "reduce must be 0 or 1");
    try {
        DeviceGuard g(h->device);
        for (int w = 0; w < nwin; ++w) {
            wdad_status st = check_params(h, &params[w]);
            if (st != WDAD_OK) return st;
            if (reduce && (params[w].wavelet_taps != params[0].wavelet_taps || params[w].level != params[0].level))
                return fail(h, WDAD_ERR_ARG, "all windows of one call share the wavelet and level");
        }
        wdad_status st = check_cube(h, cube, H, W, L);
        if (st != WDAD_OK) return st;
        const int64_t P = (int64_t)H * W;
        if (P == 0) return WDAD_OK;
        if (!scores) return fail(h, WDAD_ERR_ARG, "scores is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        const int D = reduce ? wdad_query_K(L, params[0].wavelet_taps, params[0].level) : L;
        size_t full = 0;
        for (int w = 0; w < nwin; ++w) {
            size_t need = 0;
            st = full_ws_need(h, H, W, D, &params[w], &need);
            if (st != WDAD_OK) return st;
            full = std::max(full, need);
        }
        const size_t b_red = reduce ? align256(sizeof(float) * (size_t)P * D) : 0;
        st = ensure_ws(h, b_red + full);
        if (st != WDAD_OK) return st;
        const float* x = cube;
        if (reduce) {
            const float* A = nullptr;
            int k2 = 0;
            st = get_dwt_plan(h, L, params[0].wavelet_taps, params[0].level, &A, &k2, s);
            if (st != WDAD_OK) return st;
            float* xr = (float*)h->ws;
            cudaError_t e = wdad::launch_dwt_approx(cube, P, L, A, D, xr, h->num_sms, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "dwt_approx launch");
            x = xr;
        }
        return detect_windows(h, x, H, W, D, nwin, params, scores, flags, (char*)h->ws + b_red, full, s);
    } catch (...) {
        return fail(h, WDAD_ERR_NOMEM, "host exception");
    }
}

// A sequence of cubes: cube i's DWT on the handle's high-priority stream beside cube i - 1's
// detector launch on the caller's stream, through two approximation buffers.  Cube i's DWT
// (buffer i % 2) waits for cube i - 2's detectors, which read that buffer; cube i's detectors
// wait for its DWT.  The DWT kernel is launched on three quarters of the SMs with a shared
// memory reservation that leaves room for exactly one detector CTA beside each of its CTAs:
// launched the ordinary way (two register-heavy DWT CTAs per SM) it fills SMs the detector
// launch then cannot use, and the two launches take as long as one after the other.
wdad_status wdad_detect_sequence(wdad_handle h, int n, const float* const* cubes, int H, int W, int L, int nwin,
                                 const wdad_params* params, float* const* outs, void* const* events, void* stream) {
    if (!h) return WDAD_ERR_ARG;
    if (n < 0 || (n > 0 && (!cubes || !outs))) return fail(h, WDAD_ERR_ARG, "n >= 0 with cubes[n] and outs[n]");
    if (nwin < 1 || nwin > 64 || !params) return fail(h, WDAD_ERR_ARG, "nwin must be 1..64 with params[nwin]");
    try {
        DeviceGuard g(h->device);
        for (int w = 0; w < nwin; ++w) {
            wdad_status st = check_params(h, &params[w]);
            if (st != WDAD_OK) return st;
            if (params[w].wavelet_taps != params[0].wavelet_taps || params[w].level != params[0].level)
                return fail(h, WDAD_ERR_ARG, "all windows of one call share the wavelet and level");
        }
        for (int i = 0; i < n; ++i) {
            wdad_status st = check_cube(h, cubes[i], H, W, L);
            if (st != WDAD_OK) return st;
            if (!outs[i]) return fail(h, WDAD_ERR_ARG, "outs[%d] is NULL", i);
        }
        const int64_t P = (int64_t)H * W;
        if (n == 0 || P == 0) return WDAD_OK;
        const int D = wdad_query_K(L, params[0].wavelet_taps, params[0].level);
        if (D < 1 || D > 8) return fail(h, WDAD_ERR_UNSUPPORTED, "the sequence entry point runs the reduced path (K <= 8)");
        size_t det_smem = 0;
        for (int w = 0; w < nwin; ++w) {
            const int th = wdad::detect_small_default_th(D, params[w].inner, params[w].outer);
            if (th == 0)
                return fail(h, WDAD_ERR_UNSUPPORTED, "window %d/%d too large for %d bands", params[w].inner,
                            params[w].outer, D);
            det_smem = std::max(det_smem, wdad::detect_small_smem(D, params[w].inner, params[w].outer, th));
        }
        const size_t b_red = align256(sizeof(float) * (size_t)P * D);
        wdad_status st = ensure_ws(h, 2 * b_red);
        if (st != WDAD_OK) return st;
        cudaStream_t s = (cudaStream_t)stream;
        const float* A = nullptr;
        int k2 = 0;
        st = get_dwt_plan(h, L, params[0].wavelet_taps, params[0].level, &A, &k2, s);
        if (st != WDAD_OK) return st;
        cudaError_t e = cudaSuccess;
        if (!h->seq) {
            int lo = 0, hi = 0;
            e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
            if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->seq, cudaStreamNonBlocking, hi);
            if (e != cudaSuccess) return cuda_fail(h, e, "sequence stream");
        }
        for (auto& ev : h->seq_ev)
            if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(h, e, "sequence events");
        // the DWT's reservation: at most 100 KiB (measured on the 512 x 512 x 224 workload, where
        // 100 KiB and 3/4 of the SMs gave the shortest step), and no more than what an SM keeps
        // beside one detector CTA: 228 KiB less the runtime's 1 KiB per CTA and the detector's
        // dynamic and static shared memory
        const size_t sm_total = 228 * 1024, overhead = 2 * 1024 + 512;
        const size_t room = det_smem + overhead < sm_total ? sm_total - det_smem - overhead : 0;
        const size_t reserve = std::min<size_t>(room, 100 * 1024);
        float* red[2] = {(float*)h->ws, (float*)((char*)h->ws + b_red)};
        cudaEvent_t ev_start = h->seq_ev[0], *dwt_done = h->seq_ev + 1, *det_done = h->seq_ev + 3;
        auto user_ev = [&](int i, int k) { return events ? (cudaEvent_t)events[4 * (size_t)i + k] : nullptr; };
        // the previous call's work on the caller's stream (detectors reading the buffers) first
        e = cudaEventRecord(ev_start, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->seq, ev_start, 0);
        for (int i = 0; i < n && e == cudaSuccess; ++i) {
            const int b = i & 1;
            if (i >= 2) e = cudaStreamWaitEvent(h->seq, det_done[b], 0);
            if (e == cudaSuccess && user_ev(i, 0)) e = cudaEventRecord(user_ev(i, 0), h->seq);
            if (e == cudaSuccess)
                e = wdad::launch_dwt_approx_beside(cubes[i], P, L, A, D, red[b], h->num_sms, h->seq_dwt_ctas, reserve,
                                                   h->seq);
            if (e == cudaSuccess && user_ev(i, 1)) e = cudaEventRecord(user_ev(i, 1), h->seq);
            if (e == cudaSuccess) e = cudaEventRecord(dwt_done[b], h->seq);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, dwt_done[b], 0);
            if (e == cudaSuccess && user_ev(i, 2)) e = cudaEventRecord(user_ev(i, 2), s);
            if (e != cudaSuccess) break;
            st = detect_windows(h, red[b], H, W, D, nwin, params, outs[i], nullptr, nullptr, 0, s);
            if (st != WDAD_OK) return st;
            if (user_ev(i, 3)) e = cudaEventRecord(user_ev(i, 3), s);
            if (e == cudaSuccess) e = cudaEventRecord(det_done[b], s);
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "sequence launches");
        return WDAD_OK;
    } catch (...) {
        return fail(h, WDAD_ERR_NOMEM, "host exception");
    }
}

wdad_status wdad_detect_all_host(wdad_handle h, const float* host_cube, int H, int W, int L, int reduce,
                                 int nwin, const wdad_params* params, float* host_scores, void* stream) {
    if (!h) return WDAD_ERR_ARG;
    if (nwin < 1 || nwin > 64 || !params) return fail(h, WDAD_ERR_ARG, "nwin must be 1..64 with params[nwin]");
    if (reduce != 0 && reduce != 1) return fail(h, WDAD_ERR_ARG, "reduce must be 0 or 1");
    try {
        DeviceGuard g(h->device);
        for (int w = 0; w < nwin; ++w) {
            wdad_status st = check_params(h, &params[w]);
            if (st != WDAD_OK) return st;
            if (reduce && (params[w].wavelet_taps != params[0].wavelet_taps || params[w].level != params[0].level))
                return fail(h, WDAD_ERR_ARG, "all windows of one call share the wavelet and level");
        }
        if (H < 0 || W < 0 || L < 1) return fail(h, WDAD_ERR_ARG, "bad cube shape %d x %d x %d", H, W, L);
        const int64_t P = (int64_t)H * W;
        if (P == 0) return WDAD_OK;
        if (!host_cube || !host_scores) return fail(h, WDAD_ERR_ARG, "host_cube and host_scores must not be NULL");
        cudaStream_t s = (cudaStream_t)stream;
        const int D = reduce ? wdad_query_K(L, params[0].wavelet_taps, params[0].level) : L;
        size_t full = 0;
        for (int w = 0; w < nwin; ++w) {
            size_t need = 0;
            wdad_status st = full_ws_need(h, H, W, D, &params[w], &need);
            if (st != WDAD_OK) return st;
            full = std::max(full, need);
        }
        // A page-locked, device-mapped cube is read by the DWT in place (over the host link):
        // the reduced path reads every spectrum once, so a staging copy would only add a pass.
        const float* mapped = nullptr;
        if (reduce) {
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, host_cube) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                at.devicePointer)
                mapped = static_cast<const float*>(at.devicePointer);
            else
                cudaGetLastError();  // not registered with CUDA: staged below
        }
        const size_t b_cube = mapped ? 0 : align256(sizeof(float) * (size_t)P * L);
        const size_t b_red = reduce ? align256(sizeof(float) * (size_t)P * D) : 0;
        const size_t b_out = align256(sizeof(float) * (size_t)P * 3 * nwin);
        wdad_status st = ensure_ws(h, b_cube + b_red + b_out + full);
        if (st != WDAD_OK) return st;
        char* base = (char*)h->ws;
        float* d_cube = (float*)base;
        float* d_red = (float*)(base + b_cube);
        float* d_out = (float*)(base + b_cube + b_red);
        void* scratch = base + b_cube + b_red + b_out;
        cudaError_t e = cudaSuccess;
        if (!mapped) {
            e = cudaMemcpyAsync(d_cube, host_cube, sizeof(float) * (size_t)P * L, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "copy cube to device");
        }
        const float* x = mapped ? mapped : d_cube;
        if (reduce && D <= 8) {
            // Row-band pipeline over three streams: the copy engine brings band b to the device
            // (h->aux2) while the SMs run the DWT of band b - 1 (the caller's stream) and the
            // detector tiles of band b - 2, which read reduced rows up to band b - 1 (h->aux),
            // whose score rows go back to the host behind them.  A DWT reading the pinned cube
            // in place would hold the SMs for the whole transfer; the copy engine leaves them
            // free.  The same kernels and plans as the one-pass path, so the same scores.
            const float* A = nullptr;
            int k2 = 0;
            st = get_dwt_plan(h, L, params[0].wavelet_taps, params[0].level, &A, &k2, s);
            if (st != WDAD_OK) return st;
            if (mapped) {  // staged through device memory after all
                const size_t need = align256(sizeof(float) * (size_t)P * L) + b_red + b_out + full;
                st = ensure_ws(h, need);
                if (st != WDAD_OK) return st;
                base = (char*)h->ws;
                d_cube = (float*)base;
                d_red = (float*)(base + align256(sizeof(float) * (size_t)P * L));
                d_out = (float*)((char*)d_red + b_red);
            }
            int ro_max = 0;
            for (int w = 0; w < nwin; ++w) ro_max = std::max(ro_max, params[w].outer / 2);
            const int RC = std::max({64, 2 * (16 + ro_max), (H + 7) / 8});
            const int nb = (H + RC - 1) / RC;
            for (cudaStream_t* q : {&h->aux, &h->aux2})
                if (!*q && cudaStreamCreateWithFlags(q, cudaStreamNonBlocking) != cudaSuccess)
                    return fail(h, WDAD_ERR_CUDA, "host pipeline streams");
            while ((int)h->evs.size() < 2 * nb + 2) {
                cudaEvent_t ev;
                if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
                    return fail(h, WDAD_ERR_CUDA, "host pipeline events");
                h->evs.push_back(ev);
            }
            cudaEvent_t* cev = h->evs.data();           // band b on the device
            cudaEvent_t* dev_ = h->evs.data() + nb;     // band b reduced
            cudaEvent_t ev_start = h->evs[2 * nb], ev_done = h->evs[2 * nb + 1];
            // everything this call touches is free once the caller's stream, which the previous
            // call ended on, gets here
            e = cudaEventRecord(ev_start, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->aux2, ev_start, 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->aux, ev_start, 0);
            for (int b = 0; b < nb && e == cudaSuccess; ++b) {
                const size_t off = (size_t)b * RC * W, npx = (size_t)(std::min(H, (b + 1) * RC) - b * RC) * W;
                e = cudaMemcpyAsync(d_cube + off * L, host_cube + off * L, sizeof(float) * npx * L,
                                    cudaMemcpyHostToDevice, h->aux2);
                if (e == cudaSuccess) e = cudaEventRecord(cev[b], h->aux2);
            }
            for (int b = 0; b < nb && e == cudaSuccess; ++b) {
                const size_t off = (size_t)b * RC * W, npx = (size_t)(std::min(H, (b + 1) * RC) - b * RC) * W;
                e = cudaStreamWaitEvent(s, cev[b], 0);
                if (e == cudaSuccess)
                    e = wdad::launch_dwt_approx(d_cube + off * L, (int64_t)npx, L, A, D, d_red + off * D, h->num_sms, s);
                if (e == cudaSuccess) e = cudaEventRecord(dev_[b], s);
            }
            if (e != cudaSuccess) return cuda_fail(h, e, "host pipeline: copies and DWT");
            for (int b = 0; b < nb && e == cudaSuccess; ++b) {
                const int r0 = b * RC, r1 = std::min(H, r0 + RC);
                e = cudaStreamWaitEvent(h->aux, dev_[std::min(b + 1, nb - 1)], 0);
                for (int w0 = 0; w0 < nwin && e == cudaSuccess; w0 += wdad::kMaxWindowsPerLaunch) {
                    const int n = std::min(wdad::kMaxWindowsPerLaunch, nwin - w0);
                    wdad::DetectArgs a[wdad::kMaxWindowsPerLaunch];
                    for (int i = 0; i < n; ++i) {
                        const wdad_params* p = &params[w0 + i];
                        a[i] = wdad::DetectArgs{};
                        a[i].x = d_red; a[i].H = H; a[i].W = W; a[i].D = D;
                        a[i].inner = p->inner; a[i].outer = p->outer; a[i].loading = p->loading;
                        a[i].border = p->border; a[i].dwest_mode = p->dwest_mode; a[i].dwest_tau = p->dwest_tau;
                        float* o = d_out + (size_t)(w0 + i) * 3 * P;
                        a[i].out[0] = o; a[i].out[1] = o + P; a[i].out[2] = o + 2 * P;
                    }
                    e = wdad::launch_detect_small_multi_rows(a, n, r0, r1, h->aux);
                }
                // the band's rows of all 3 nwin maps in one strided copy
                if (e == cudaSuccess)
                    e = cudaMemcpy2DAsync(host_scores + (size_t)r0 * W, sizeof(float) * (size_t)P, d_out + (size_t)r0 * W,
                                          sizeof(float) * (size_t)P, sizeof(float) * (size_t)(r1 - r0) * W,
                                          (size_t)(3 * nwin), cudaMemcpyDeviceToHost, h->aux);
            }
            // the call is complete on the caller's stream once the other two streams' work is
            if (e == cudaSuccess) e = cudaEventRecord(ev_done, h->aux);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_done, 0);
            if (e != cudaSuccess) return cuda_fail(h, e, "host pipeline: detectors and copies");
            return WDAD_OK;
        }
        if (reduce) {
            const float* A = nullptr;
            int k2 = 0;
            st = get_dwt_plan(h, L, params[0].wavelet_taps, params[0].level, &A, &k2, s);
            if (st != WDAD_OK) return st;
            e = wdad::launch_dwt_approx(x, P, L, A, D, d_red, h->num_sms, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "dwt_approx launch");
            x = d_red;
        }
        st = detect_windows(h, x, H, W, D, nwin, params, d_out, nullptr, scratch, full, s);
        if (st != WDAD_OK) return st;
        e = cudaMemcpyAsync(host_scores, d_out, sizeof(float) * (size_t)P * 3 * nwin, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy scores to host");
        return WDAD_OK;
    } catch (...) {
        return fail(h, WDAD_ERR_NOMEM, "host exception");
    }
}

wdad_status wdad_window_moments(wdad_handle h, const float* cube, int H, int W, int L, const int64_t* pixels,
                                int64_t npix, const wdad_params* p, float* mu_o, float* cov_o, void* stream) {
    if (!h) return WDAD_ERR_ARG;
    try {
        DeviceGuard g(h->device);
        wdad_status st = check_params(h, p);
        if (st != WDAD_OK) return st;
        st = check_cube(h, cube, H, W, L);
        if (st != WDAD_OK) return st;
        if (npix < 0) return fail(h, WDAD_ERR_ARG, "npix must be >= 0");
        if (npix == 0) return WDAD_OK;
        if (!pixels || !mu_o || !cov_o) return fail(h, WDAD_ERR_ARG, "pixels, mu_o and cov_o must not be NULL");
        if (L > 1024) return fail(h, WDAD_ERR_UNSUPPORTED, "window moments for more than 1024 bands");
        wdad::FullArgs a{};
        a.x = cube; a.H = H; a.W = W; a.D = L;
        a.inner = p->inner; a.outer = p->outer; a.precision = p->precision;
        const size_t need = wdad::moments_workspace_bytes(a, npix, h->num_sms);
        if (need == 0) return fail(h, WDAD_ERR_UNSUPPORTED, "window moments for %d bands", L);
        st = ensure_ws(h, need);
        if (st != WDAD_OK) return st;
        cudaError_t e = wdad::launch_window_moments(a, pixels, npix, mu_o, cov_o, h->ws, h->ws_bytes, h->num_sms,
                                                    (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "window moments launch");
        return WDAD_OK;
    } catch (...) {
        return fail(h, WDAD_ERR_NOMEM, "host exception");
    }
}

wdad_status wdad_window_census(wdad_handle h, int H, int W, const wdad_params* p, int64_t* out, void* stream) {
    if (!h) return WDAD_ERR_ARG;
    DeviceGuard g(h->device);
    wdad_status st = check_params(h, p);
    if (st != WDAD_OK) return st;
    if (H < 0 || W < 0) return fail(h, WDAD_ERR_ARG, "H and W must be >= 0");
    if ((int64_t)H * W == 0) return WDAD_OK;
    if (!out) return fail(h, WDAD_ERR_ARG, "out is NULL");
    cudaError_t e = wdad::launch_window_census(H, W, p->inner, p->outer, p->border, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "census launch");
    return WDAD_OK;
}

wdad_status wdad_autotune(wdad_handle h, int D, int inner, int outer, int* tile_h, void* stream) {
    if (!h) return WDAD_ERR_ARG;
    if (!tile_h || D < 1 || D > 8 || inner < 1 || !(inner & 1) || outer <= inner || !(outer & 1) || outer > 63)
        return fail(h, WDAD_ERR_ARG, "autotune: D in 1..8, odd windows 1 <= inner < outer <= 63");
    try {
        DeviceGuard g(h->device);
        return autotune(h, D, inner, outer, 0, 0, tile_h, (cudaStream_t)stream);
    } catch (...) {
        return fail(h, WDAD_ERR_NOMEM, "host exception");
    }
}

// The batch's work on one stream: the persistent kernel for the small jobs, then each large
// job's DWT and detector launches.
static cudaError_t batch_issue(wdad_batch_ctx* b, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (b->n > 0)
        e = wdad::batch_launch(b->d_jobs, b->d_items, b->nitems, b->d_counters, b->n, b->smem, b->h->num_sms, s);
    for (const BatchDirect& d : b->direct) {
        if (e != cudaSuccess) break;
        e = wdad::launch_dwt_approx(d.cube, d.P, d.L, d.A, d.K, const_cast<float*>(d.args.x), b->h->num_sms, s);
        if (e == cudaSuccess) e = wdad::launch_detect_small_th(d.args, d.th, s);
    }
    return e;
}

// The batch with every job's plan from the autotuner (tuned) or the default plans.
static wdad_status batch_build(wdad_handle h, int n, const wdad_job* jobs, int autotune_plans, int use_graph,
                               wdad_batch* out, void* stream) {
    if (!h) return WDAD_ERR_ARG;
    if (!out || n < 1 || !jobs) return fail(h, WDAD_ERR_ARG, "batch: n >= 1 jobs and an output handle");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    wdad_batch_ctx* b = nullptr;
    try {
        DeviceGuard g(h->device);
        std::vector<wdad::BatchJob> hj;
        std::vector<BatchDirect> direct;
        std::vector<int> th_all((size_t)n);
        size_t approx_floats = 0;
        std::vector<size_t> aoff, doff;
        size_t smem = 0;
        for (int i = 0; i < n; ++i) {
            const wdad_job& j = jobs[i];
            wdad_status st = check_params(h, &j.params);
            if (st != WDAD_OK) return st;
            st = check_cube(h, j.cube, j.H, j.W, j.L);
            if (st != WDAD_OK) return st;
            if ((int64_t)j.H * j.W == 0) return fail(h, WDAD_ERR_ARG, "batch job %d is empty", i);
            if (j.detector < 0 || j.detector > 3 || !j.scores) return fail(h, WDAD_ERR_ARG, "batch job %d: detector/scores", i);
            const int K = wdad_query_K(j.L, j.params.wavelet_taps, j.params.level);
            if (!wdad::batch_job_supported(j.L, K))
                return fail(h, WDAD_ERR_UNSUPPORTED, "batch job %d: L %% 4 == 0, L <= 256, K <= 4 (L=%d, K=%d)", i, j.L, K);
            const float* A = nullptr;
            int k2 = 0;
            st = get_dwt_plan(h, j.L, j.params.wavelet_taps, j.params.level, &A, &k2, s);
            if (st != WDAD_OK) return st;
            int th = wdad::detect_small_default_th(K, j.params.inner, j.params.outer);
            if (autotune_plans) {
                // a batch fills the GPU with many jobs: the per-pixel cost of a plan is what counts,
                // so plans are timed on a cube large enough to fill the GPU, not at the job's size
                st = autotune(h, K, j.params.inner, j.params.outer, 1024, 1024, &th, s, true);
                if (st != WDAD_OK) return st;
            }
            if (th < 1) return fail(h, WDAD_ERR_UNSUPPORTED, "batch job %d: window too large", i);
            th_all[(size_t)i] = th;
            const size_t P = (size_t)j.H * j.W;
            if ((int64_t)P >= kBatchDirectPixels) {
                BatchDirect d{};
                d.cube = j.cube; d.A = A; d.P = (int64_t)P; d.L = j.L; d.K = K; d.th = th;
                wdad::DetectArgs& a = d.args;
                a.H = j.H; a.W = j.W; a.D = K;
                a.inner = j.params.inner; a.outer = j.params.outer; a.loading = j.params.loading;
                a.border = j.params.border; a.dwest_mode = j.params.dwest_mode; a.dwest_tau = j.params.dwest_tau;
                if (j.detector == 3) { a.out[0] = j.scores; a.out[1] = j.scores + P; a.out[2] = j.scores + 2 * P; }
                else a.out[j.detector] = j.scores;
                a.flags = j.flags;
                direct.push_back(d);
                doff.push_back(approx_floats);
                approx_floats += ((P * K + 63) / 64) * 64;
                continue;
            }
            smem = std::max(smem, wdad::detect_small_smem(K, j.params.inner, j.params.outer, th));
            smem = std::max(smem, wdad::batch_dwt_smem(j.L));
            hj.emplace_back();
            wdad::BatchJob& bj = hj.back();
            bj = wdad::BatchJob{};
            bj.cube = j.cube; bj.A = A; bj.flags = j.flags;
            bj.H = j.H; bj.W = j.W; bj.L = j.L; bj.K = K;
            bj.inner = j.params.inner; bj.outer = j.params.outer; bj.border = j.params.border;
            bj.dwest_mode = j.params.dwest_mode; bj.loading = j.params.loading; bj.tau = j.params.dwest_tau;
            bj.th = th;
            bj.variant = wdad::batch_variant(j.L);
            if (j.detector == 3) { bj.out[0] = j.scores; bj.out[1] = j.scores + P; bj.out[2] = j.scores + 2 * P; }
            else bj.out[j.detector] = j.scores;
            aoff.push_back(approx_floats);
            approx_floats += ((P * K + 63) / 64) * 64;
        }
        const int np = (int)hj.size();
        int drop = -1;
        if (const char* e = std::getenv("WDAD_FAULT_DROP_DWT_ITEM")) drop = std::atoi(e);
        std::vector<wdad::BatchItem> items;
        std::vector<int> dwt_items;
        if (np > 0) wdad::batch_build_items(hj, items, dwt_items, drop, 4 * 2 * h->num_sms);
        b = new wdad_batch_ctx();
        b->h = h;
        b->n = np;
        b->nitems = (int)items.size();
        b->smem = smem;
        b->th = th_all;
        cudaError_t e = cudaMalloc(&b->d_approx, sizeof(float) * std::max<size_t>(approx_floats, 64));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_jobs, sizeof(wdad::BatchJob) * (size_t)std::max(np, 1));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(wdad::BatchItem) * std::max<size_t>(items.size(), 1));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, sizeof(int) * (size_t)(2 + 2 * std::max(np, 1)));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->last, cudaEventDisableTiming);
        if (e != cudaSuccess) { batch_free(b); return cuda_fail(h, e, "batch allocation"); }
        if (np == 0) e = cudaMemsetAsync(b->d_counters, 0, sizeof(int) * 4, s);  // status word stays 0
        for (int i = 0; i < np; ++i) {
            hj[(size_t)i].approx = b->d_approx + aoff[(size_t)i];
            hj[(size_t)i].dwt_items = dwt_items[(size_t)i];
        }
        for (size_t i = 0; i < direct.size(); ++i) direct[i].args.x = b->d_approx + doff[i];
        b->direct = direct;
        if (e == cudaSuccess && np > 0)
            e = cudaMemcpyAsync(b->d_jobs, hj.data(), sizeof(wdad::BatchJob) * (size_t)np, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !items.empty())
            e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(wdad::BatchItem) * items.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { batch_free(b); return cuda_fail(h, e, "batch upload"); }
        if (use_graph) {
            e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t el = batch_issue(b, b->cap_stream);
                e = cudaStreamEndCapture(b->cap_stream, &b->graph);
                if (el != cudaSuccess) e = el;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
            if (e != cudaSuccess) { batch_free(b); return cuda_fail(h, e, "batch graph capture"); }
        }
        *out = b;
        return WDAD_OK;
    } catch (...) {
        batch_free(b);
        return fail(h, WDAD_ERR_NOMEM, "host exception");
    }
}

// Median device time of `reps` launches of a batch after two warm-up launches (CUDA events on
// `stream`); a negative value when a launch or its status fails.
static float batch_time(wdad_batch b, cudaStream_t s, int reps) {
    for (int r = 0; r < 2; ++r)
        if (wdad_batch_launch(b, s) != WDAD_OK) return -1.f;
    if (wdad_batch_status(b, nullptr) != WDAD_OK) return -1.f;
    std::vector<cudaEvent_t> ev((size_t)reps + 1);
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return -1.f;
    std::vector<float> t;
    bool ok = cudaEventRecord(ev[0], s) == cudaSuccess;
    for (int r = 0; r < reps && ok; ++r)
        ok = wdad_batch_launch(b, s) == WDAD_OK && cudaEventRecord(ev[(size_t)r + 1], s) == cudaSuccess;
    ok = ok && cudaEventSynchronize(ev[(size_t)reps]) == cudaSuccess && wdad_batch_status(b, nullptr) == WDAD_OK;
    for (int r = 0; r < reps && ok; ++r) {
        float ms = 0.f;
        ok = cudaEventElapsedTime(&ms, ev[(size_t)r], ev[(size_t)r + 1]) == cudaSuccess;
        t.push_back(ms);
    }
    for (auto e : ev) cudaEventDestroy(e);
    if (!ok) return -1.f;
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

// With autotune, the plans the autotuner measured one (K, window) class at a time are checked
// on the batch itself: the whole batch is timed with the tuned plans and with the default
// plans, and the tuned set is kept only if it is at least 1% faster, so an autotuned batch is
// never slower than the default one by more than the timing noise.
wdad_status wdad_batch_create(wdad_handle h, int n, const wdad_job* jobs, int autotune_plans, int use_graph,
                              wdad_batch* out, void* stream) {
    if (!autotune_plans) return batch_build(h, n, jobs, 0, use_graph, out, stream);
    wdad_batch tuned = nullptr, plain = nullptr;
    wdad_status st = batch_build(h, n, jobs, 1, use_graph, &tuned, stream);
    if (st != WDAD_OK) return st;
    bool all_default = true;
    for (int i = 0; i < n && all_default; ++i) {
        const wdad_job& j = jobs[i];
        const int K = wdad_query_K(j.L, j.params.wavelet_taps, j.params.level);
        all_default = tuned->th[(size_t)i] == wdad::detect_small_default_th(K, j.params.inner, j.params.outer);
    }
    if (all_default) { *out = tuned; return WDAD_OK; }
    st = batch_build(h, n, jobs, 0, use_graph, &plain, stream);
    if (st != WDAD_OK) { wdad_batch_destroy(tuned); return st; }
    cudaStream_t s = (cudaStream_t)stream;
    const float t_tuned = batch_time(tuned, s, 5), t_plain = batch_time(plain, s, 5);
    if (t_tuned < 0.f || t_plain < 0.f) {
        wdad_batch_destroy(tuned);
        wdad_batch_destroy(plain);
        return fail(h, WDAD_ERR_CUDA, "batch autotune: a timing launch failed");
    }
    const bool keep_tuned = t_tuned < 0.99f * t_plain;
    wdad_batch_destroy(keep_tuned ? plain : tuned);
    *out = keep_tuned ? tuned : plain;
    return WDAD_OK;
}

wdad_status wdad_batch_launch(wdad_batch b, void* stream) {
    if (!b) return WDAD_ERR_ARG;
    DeviceGuard g(b->h->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = b->exec ? cudaGraphLaunch(b->exec, s) : batch_issue(b, s);
    if (e == cudaSuccess) e = cudaEventRecord(b->last, s);
    if (e != cudaSuccess) return cuda_fail(b->h, e, "batch launch");
    return WDAD_OK;
}

wdad_status wdad_batch_status(wdad_batch b, int* tile_h_out) {
    if (!b) return WDAD_ERR_ARG;
    DeviceGuard g(b->h->device);
    if (tile_h_out)
        for (size_t i = 0; i < b->th.size(); ++i) tile_h_out[i] = b->th[i];
    cudaError_t e = cudaEventSynchronize(b->last);
    int dev_status = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&dev_status, b->d_counters + 1 + b->n, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(b->h, e, "batch status");
    if (dev_status == (int)WDAD_ERR_CUDA)
        return fail(b->h, WDAD_ERR_CUDA,
                    "a staged DWT chunk and the copies behind it never landed: unrecoverable, destroy the batch "
                    "and reset the device context");
    if (dev_status != 0) return fail(b->h, (wdad_status)dev_status, "a batched item gave up waiting (DWT chunk or tile)");
    return WDAD_OK;
}

wdad_status wdad_batch_destroy(wdad_batch b) {
    if (!b) return WDAD_ERR_ARG;
    DeviceGuard g(b->h->device);
    cudaEventSynchronize(b->last);
    batch_free(b);
    return WDAD_OK;
}

wdad_status wdad_batch_run(wdad_handle h, int n, const wdad_job* jobs, void* stream) {
    wdad_batch b = nullptr;
    wdad_status st = wdad_batch_create(h, n, jobs, 0, 0, &b, stream);
    if (st != WDAD_OK) return st;
    st = wdad_batch_launch(b, stream);
    if (st == WDAD_OK) st = wdad_batch_status(b, nullptr);
    wdad_batch_destroy(b);
    return st;
}


wdad_status wdad_cnn_create(wdad_handle h, int K, int bf16_weights, uint64_t seed, int64_t max_batch_pixels,
                            wdad_cnn* out) {
    if (!h) return WDAD_ERR_ARG;
    if (!out || K < 1 || K > 8 || max_batch_pixels < 1) return fail(h, WDAD_ERR_ARG, "cnn: K in 1..8, max pixels >= 1");
    *out = nullptr;
    wdad_cnn_ctx* c = nullptr;
    try {
        DeviceGuard g(h->device);
        c = new wdad_cnn_ctx();
        c->h = h;
        auto& n = c->net;
        n.K = K;
        n.bf16 = bf16_weights ? 1 : 0;
        n.max_px = max_batch_pixels;
        wdad::cnn::param_layout(K, n.woff, n.boff, &n.nparam);
        cudaError_t e = cudaSuccess;
        for (float** pp : {&n.w, &n.wf, &n.m, &n.v, &n.grad})
            if (e == cudaSuccess) e = cudaMalloc(pp, sizeof(float) * n.nparam);
        if (e == cudaSuccess) e = cudaMalloc(&n.wt, sizeof(float) * 32 * 32 * 25);
        if (e == cudaSuccess) e = cudaMalloc(&n.norm, sizeof(float) * (size_t)(K + K * K));
        if (e == cudaSuccess)
            e = cudaMalloc(&n.stat, sizeof(double) * wdad::cnn::WHITEN_BLOCKS * wdad::cnn::WHITEN_NQ_MAX);
        if (e == cudaSuccess) e = cudaMalloc(&n.act, sizeof(float) * wdad::cnn::act_floats(max_batch_pixels));
        if (e == cudaSuccess) e = cudaMalloc(&n.loss, sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&n.cx, sizeof(float) * (size_t)max_batch_pixels * K);
        if (e == cudaSuccess) e = cudaMalloc(&n.ct, sizeof(float) * (size_t)max_batch_pixels);
        if (e == cudaSuccess) e = cudaMalloc(&n.wpk, sizeof(__nv_bfloat16) * 2 * 25 * 32 * 32);
        if (e == cudaSuccess) e = cudaMalloc(&n.gpart, sizeof(float) * wdad::cnn::gpart_floats());
        if (e == cudaSuccess) e = cudaMalloc(&n.tcerr, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(n.tcerr, 0, sizeof(int));
        if (e != cudaSuccess) { cnn_free(c); return cuda_fail(h, e, "cnn allocation"); }
        std::vector<float> norm((size_t)(K + K * K), 0.f);  // mu = 0, M = I until a scene sets it
        for (int k = 0; k < K; ++k) norm[K + k * K + k] = 1.f;
        n.norm_mode = 0;
        e = cudaMemcpy(n.norm, norm.data(), sizeof(float) * norm.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = wdad::cnn::net_init(n, seed, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) { cnn_free(c); return cuda_fail(h, e, "cnn init"); }
        *out = c;
        return WDAD_OK;
    } catch (...) {
        cnn_free(c);
        return fail(h, WDAD_ERR_NOMEM, "host exception");
    }
}

wdad_status wdad_cnn_destroy(wdad_cnn c) {
    if (!c) return WDAD_ERR_ARG;
    DeviceGuard g(c->h->device);
    cudaDeviceSynchronize();
    cnn_free(c);
    return WDAD_OK;
}

wdad_status wdad_cnn_set_norm(wdad_cnn c, const float* host_mu_M) {
    if (!c) return WDAD_ERR_ARG;
    auto& n = c->net;
    if (!host_mu_M) { n.norm_mode = 0; return WDAD_OK; }
    const int K = n.K;
    for (int i = 0; i < K + K * K; ++i)
        if (!std::isfinite(host_mu_M[i])) return fail(c->h, WDAD_ERR_ARG, "cnn: input map must be finite");
    DeviceGuard g(c->h->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(n.norm, host_mu_M, sizeof(float) * (size_t)(K + K * K), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c->h, e, "cnn norm");
    n.norm_mode = 1;
    return WDAD_OK;
}

wdad_status wdad_scene_whitening(wdad_handle h, const float* x, int64_t P, int K, float* norm_out, void* stream) {
    if (!h) return WDAD_ERR_ARG;
    if (!x || !norm_out || P < 1 || K < 1 || K > 8) return fail(h, WDAD_ERR_ARG, "whitening: P >= 1, K in 1..8");
    try {
        DeviceGuard g(h->device);
        wdad_status st = ensure_ws(h, sizeof(double) * wdad::cnn::WHITEN_BLOCKS * wdad::cnn::WHITEN_NQ_MAX);
        if (st != WDAD_OK) return st;
        cudaError_t e = wdad::cnn::scene_whitening(x, P, K, (double*)h->ws, norm_out, (cudaStream_t)stream);
        return e == cudaSuccess ? WDAD_OK : cuda_fail(h, e, "scene whitening");
    } catch (...) {
        return fail(h, WDAD_ERR_NOMEM, "host exception");
    }
}

wdad_status wdad_cnn_params(wdad_cnn c, float* host, int64_t* count) {
    if (!c || !count) return WDAD_ERR_ARG;
    DeviceGuard g(c->h->device);
    *count = (int64_t)c->net.nparam;
    if (!host) return WDAD_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host, c->net.w, sizeof(float) * c->net.nparam, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? WDAD_OK : cuda_fail(c->h, e, "cnn params");
}

wdad_status wdad_cnn_set_params(wdad_cnn c, const float* host, int64_t count) {
    if (!c || !host || count != (int64_t)c->net.nparam) return WDAD_ERR_ARG;
    DeviceGuard g(c->h->device);
    auto& n = c->net;
    cudaError_t e = cudaMemcpy(n.w, host, sizeof(float) * n.nparam, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n.m, 0, sizeof(float) * n.nparam);
    if (e == cudaSuccess) e = cudaMemset(n.v, 0, sizeof(float) * n.nparam);
    n.step = 0;
    if (e == cudaSuccess) e = wdad::cnn::net_refresh_forward_copy(n, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e == cudaSuccess ? WDAD_OK : cuda_fail(c->h, e, "cnn set params");
}

wdad_status wdad_cnn_forward(wdad_cnn c, const float* x, int B, int H, int W, float* pred, void* stream) {
    if (!c || !x || !pred || B < 1 || H < 1 || W < 1) return WDAD_ERR_ARG;
    DeviceGuard g(c->h->device);
    wdad_ctx* h = c->h;
    const int64_t px = (int64_t)B * H * W;
    wdad_status st = ensure_ws(h, sizeof(float) * (size_t)px * 96 + 256);
    if (st != WDAD_OK) return st;
    float* a0 = (float*)h->ws;
    cudaError_t e = cudaSuccess;
    if (c->net.norm_mode == 0) e = wdad::cnn::scene_whitening(x, px, c->net.K, c->net.stat, c->net.norm, (cudaStream_t)stream);
    if (e == cudaSuccess)
        e = wdad::cnn::net_forward(c->net, x, B, H, W, c->net.norm, a0, a0 + px * 32, a0 + px * 64, pred,
                                   (cudaStream_t)stream, c->net.bf16 != 0, h->num_sms);
    return e == cudaSuccess ? WDAD_OK : cuda_fail(h, e, "cnn forward");
}

wdad_status wdad_cnn_grad(wdad_cnn c, const float* x, const float* target, int B, int H, int W, float* host_grad,
                          float* host_loss, void* stream) {
    if (!c || !x || !target || B < 1 || H < 15 || W < 15) return WDAD_ERR_ARG;
    if ((int64_t)B * H * W > c->net.max_px) return fail(c->h, WDAD_ERR_ARG, "cnn: batch larger than max pixels");
    DeviceGuard g(c->h->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = wdad::cnn::net_grad(c->net, x, target, B, H, W, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && host_grad)
        e = cudaMemcpy(host_grad, c->net.grad, sizeof(float) * c->net.nparam, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && host_loss) e = cudaMemcpy(host_loss, c->net.loss, sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? WDAD_OK : cuda_fail(c->h, e, "cnn grad");
}

wdad_status wdad_cnn_train(wdad_cnn c, const float* approx, const float* score, int H, int W, int steps, int batch,
                           int crop, float lr, uint64_t seed, float* host_loss, void* stream) {
    if (!c || !approx || !score || steps < 0 || batch < 1 || crop < 15 || crop > H || crop > W || !(lr > 0.f))
        return WDAD_ERR_ARG;
    auto& n = c->net;
    if ((int64_t)batch * crop * crop > n.max_px) return fail(c->h, WDAD_ERR_ARG, "cnn: batch larger than max pixels");
    DeviceGuard g(c->h->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (n.norm_mode == 0) e = wdad::cnn::scene_whitening(approx, (int64_t)H * W, n.K, n.stat, n.norm, s);
    for (int it = 0; it < steps && e == cudaSuccess; ++it) {
        e = wdad::cnn::sample_crops(n, approx, score, H, W, batch, crop, crop, seed, (uint64_t)n.step, n.cx, n.ct, s);
        if (e == cudaSuccess) e = wdad::cnn::net_grad(n, n.cx, n.ct, batch, crop, crop, s);
        if (e == cudaSuccess) e = wdad::cnn::net_adam(n, lr, s);
    }
    if (e == cudaSuccess && host_loss) {
        e = cudaMemcpyAsync(host_loss, n.loss, sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    return e == cudaSuccess ? WDAD_OK : cuda_fail(c->h, e, "cnn train");
}

wdad_status wdad_cnn_save(wdad_cnn c, const char* path) {
    if (!c || !path) return WDAD_ERR_ARG;
    DeviceGuard g(c->h->device);
    auto& n = c->net;
    std::vector<float> w(n.nparam), m(n.nparam), v(n.nparam), norm((size_t)(n.K + n.K * n.K));
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(w.data(), n.w, sizeof(float) * n.nparam, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(m.data(), n.m, sizeof(float) * n.nparam, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(v.data(), n.v, sizeof(float) * n.nparam, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(norm.data(), n.norm, sizeof(float) * norm.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c->h, e, "cnn save");
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(c->h, WDAD_ERR_ARG, "cannot open %s", path);
    const uint32_t hdr[6] = {kCnnMagic, kCnnVersion, (uint32_t)n.K, (uint32_t)n.bf16, (uint32_t)n.step,
                             (uint32_t)n.norm_mode};
    const uint64_t np = n.nparam;
    bool ok = std::fwrite(hdr, sizeof hdr, 1, f) == 1 && std::fwrite(&np, sizeof np, 1, f) == 1 &&
              std::fwrite(w.data(), sizeof(float), np, f) == np && std::fwrite(m.data(), sizeof(float), np, f) == np &&
              std::fwrite(v.data(), sizeof(float), np, f) == np &&
              std::fwrite(norm.data(), sizeof(float), norm.size(), f) == norm.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? WDAD_OK : fail(c->h, WDAD_ERR_ARG, "write failed: %s", path);
}

wdad_status wdad_cnn_load(wdad_handle h, const char* path, int64_t max_batch_pixels, wdad_cnn* out) {
    if (!h || !path || !out) return WDAD_ERR_ARG;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(h, WDAD_ERR_ARG, "cannot open %s", path);
    uint32_t hdr[6];
    uint64_t np = 0;
    if (std::fread(hdr, sizeof hdr, 1, f) != 1 || std::fread(&np, sizeof np, 1, f) != 1 || hdr[0] != kCnnMagic ||
        hdr[1] != kCnnVersion || hdr[2] < 1 || hdr[2] > 8 || hdr[5] > 1) {
        std::fclose(f);
        return fail(h, WDAD_ERR_ARG, "%s is not a version-%u CNN checkpoint", path, kCnnVersion);
    }
    wdad_cnn c = nullptr;
    wdad_status st = wdad_cnn_create(h, (int)hdr[2], (int)hdr[3], 0, max_batch_pixels, &c);
    if (st != WDAD_OK) { std::fclose(f); return st; }
    auto& n = c->net;
    if (np != n.nparam) { std::fclose(f); wdad_cnn_destroy(c); return fail(h, WDAD_ERR_ARG, "checkpoint size mismatch"); }
    std::vector<float> w(np), m(np), v(np), norm((size_t)(n.K + n.K * n.K));
    const bool ok = std::fread(w.data(), sizeof(float), np, f) == np && std::fread(m.data(), sizeof(float), np, f) == np &&
                    std::fread(v.data(), sizeof(float), np, f) == np &&
                    std::fread(norm.data(), sizeof(float), norm.size(), f) == norm.size();
    std::fclose(f);
    if (!ok) { wdad_cnn_destroy(c); return fail(h, WDAD_ERR_ARG, "truncated checkpoint %s", path); }
    DeviceGuard g(h->device);
    cudaError_t e = cudaMemcpy(n.w, w.data(), sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(n.m, m.data(), sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(n.v, v.data(), sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(n.norm, norm.data(), sizeof(float) * norm.size(), cudaMemcpyHostToDevice);
    n.step = (int)hdr[4];
    n.norm_mode = (int)hdr[5];
    if (e == cudaSuccess) e = wdad::cnn::net_refresh_forward_copy(n, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { wdad_cnn_destroy(c); return cuda_fail(h, e, "cnn load"); }
    *out = c;
    return WDAD_OK;
}

wdad_status wdad_screen_run(wdad_handle h, wdad_cnn c, const float* cube, int H, int W, int L, const wdad_params* p,
                            float top_frac, float audit_frac, uint64_t seed, int tile_rows, int exact_reduce,
                            float* score, float* pred_out, uint8_t* selected, int64_t* n_selected, void* stream) {
    if (!h) return WDAD_ERR_ARG;
    if (!c || !score || !(top_frac > 0.f && top_frac <= 1.f) || !(audit_frac >= 0.f && audit_frac < 1.f) ||
        tile_rows < 1 || (exact_reduce != 0 && exact_reduce != 1))
        return fail(h, WDAD_ERR_ARG, "screen: fractions in (0,1], tile_rows >= 1, exact_reduce 0/1");
    try {
        DeviceGuard g(h->device);
        wdad_status st = check_params(h, p);
        if (st != WDAD_OK) return st;
        st = check_cube(h, cube, H, W, L);
        if (st != WDAD_OK) return st;
        const int64_t P = (int64_t)H * W;
        if (P == 0) { if (n_selected) *n_selected = 0; return WDAD_OK; }
        cudaStream_t s = (cudaStream_t)stream;
        auto& n = c->net;
        const int K = wdad_query_K(L, p->wavelet_taps, p->level);
        if (K != n.K) return fail(h, WDAD_ERR_ARG, "screen: the network expects K=%d, the cube gives K=%d", n.K, K);
        if (!wdad::dwt_shape_supported(L, K)) return fail(h, WDAD_ERR_UNSUPPORTED, "screen: DWT shape L=%d", L);
        const int halo = 7, rows_max = std::min(H, tile_rows + 2 * halo);
        const int64_t tpx = (int64_t)rows_max * W;
        const size_t b_ap = align256(sizeof(float) * (size_t)P * K);
        const size_t b_pred = align256(sizeof(float) * (size_t)P);
        const size_t b_act = align256(sizeof(float) * (size_t)tpx * (3 * 32 + 1));
        const size_t b_list = align256(sizeof(int64_t) * (size_t)P);
        const size_t b_hist = align256(sizeof(unsigned int) * 65536 + 64);
        const size_t fixed = b_ap + b_pred + b_act + b_list + b_hist;
        // the exact detector's slabs are sized now (at most one per SM) so that the workspace
        // never moves while it holds the selection
        size_t need_full = 0;
        if (!exact_reduce) {
            wdad::FullArgs probe{};
            probe.H = H; probe.W = W; probe.D = L; probe.inner = p->inner; probe.outer = p->outer;
            probe.precision = p->precision;
            need_full = wdad::fullband_workspace_bytes(probe, h->num_sms);
            if (need_full == 0) return fail(h, WDAD_ERR_UNSUPPORTED, "screen: full-band LRX for %d bands", L);
        }
        st = ensure_ws(h, fixed + need_full);
        if (st != WDAD_OK) return st;
        char* base = (char*)h->ws;
        float* approx = (float*)base;
        float* pred = (float*)(base + b_ap);
        float* act = (float*)(base + b_ap + b_pred);
        int64_t* list = (int64_t*)(base + b_ap + b_pred + b_act);
        unsigned int* hist = (unsigned int*)(base + b_ap + b_pred + b_act + b_list);
        unsigned long long* cnt = (unsigned long long*)(hist + 65536);
        // A1 on the whole cube
        const float* A = nullptr;
        int k2 = 0;
        st = get_dwt_plan(h, L, p->wavelet_taps, p->level, &A, &k2, s);
        if (st != WDAD_OK) return st;
        cudaError_t e = wdad::launch_dwt_approx(cube, P, L, A, K, approx, h->num_sms, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "screen dwt");
        if (n.norm_mode == 0) e = wdad::cnn::scene_whitening(approx, P, K, n.stat, n.norm, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "screen whitening");
        // CNN over row tiles with a 7-row halo (receptive field 15)
        for (int r0 = 0; r0 < H && e == cudaSuccess; r0 += tile_rows) {
            const int r1 = std::min(H, r0 + tile_rows);
            const int h0 = std::max(0, r0 - halo), h1 = std::min(H, r1 + halo);
            const int hr = h1 - h0;
            const int64_t npx = (int64_t)hr * W;
            float* a0 = act;
            float* a1 = a0 + npx * 32;
            float* a2 = a1 + npx * 32;
            float* o = a2 + npx * 32;
            e = wdad::cnn::net_forward(n, approx + (size_t)h0 * W * K, 1, hr, W, n.norm, a0, a1, a2, o, s,
                                       n.bf16 != 0, h->num_sms);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(pred + (size_t)r0 * W, o + (size_t)(r0 - h0) * W, sizeof(float) * (size_t)(r1 - r0) * W,
                                    cudaMemcpyDeviceToDevice, s);
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "screen cnn");
        if (pred_out) {
            e = cudaMemcpyAsync(pred_out, pred, sizeof(float) * (size_t)P, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "screen pred copy");
        }
        // top fraction threshold, audit draw, compaction
        // ceil(top_frac * P) with a slack of one float rounding of top_frac, so that e.g. 0.1f of
        // 2080 pixels counts 208 (0.1f is 0.100000001...)
        const int64_t kth =
            std::max<int64_t>(1, (int64_t)std::ceil((double)top_frac * (double)P * (1.0 - 1.2e-7)));
        uint32_t thr = 0;
        e = wdad::cnn::top_threshold(pred, P, kth, hist, &thr, s);
        if (e == cudaSuccess) e = wdad::cnn::select_pixels(pred, P, thr, audit_frac, seed, selected, list, cnt, s);
        unsigned long long nsel = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&nsel, cnt, sizeof nsel, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "screen selection");
        if (n.bf16) {
            int tcerr = 0;
            e = cudaMemcpy(&tcerr, n.tcerr, sizeof tcerr, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(h, e, "screen status");
            if (tcerr) {
                cudaMemset(n.tcerr, 0, sizeof(int));
                return fail(h, WDAD_ERR_TIMEOUT, "screen: a tensor-core convolution gave up waiting");
            }
        }
        if (n_selected) *n_selected = (int64_t)nsel;
        // unevaluated pixels score -inf; the exact detector fills the selected ones
        e = wdad::cnn::fill(score, P, -INFINITY, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "screen fill");
        if (nsel == 0) return WDAD_OK;
        wdad::FullArgs a{};
        a.x = exact_reduce ? approx : cube;
        a.H = H; a.W = W; a.D = exact_reduce ? K : L;
        a.inner = p->inner; a.outer = p->outer; a.loading = p->loading; a.cond_gate = p->cond_gate;
        a.border = p->border; a.dwest_mode = p->dwest_mode; a.precision = p->precision; a.dwest_tau = p->dwest_tau;
        a.out[0] = score;
        a.pix = list;
        a.npix = (int64_t)nsel;
        if (a.D <= 8) {
            // reduced exact LRX: the whole reduced map is cheap; the selection keeps its values
            wdad::DetectArgs d{};
            d.x = approx; d.H = H; d.W = W; d.D = K;
            d.inner = p->inner; d.outer = p->outer; d.loading = p->loading; d.border = p->border;
            d.dwest_mode = p->dwest_mode; d.dwest_tau = p->dwest_tau;
            d.out[0] = pred;  // the predictions are no longer needed
            e = wdad::launch_detect_small_th(d, wdad::detect_small_default_th(K, p->inner, p->outer), s);
            if (e == cudaSuccess) e = wdad::cnn::scatter_list(pred, list, (int64_t)nsel, score, s);
            return e == cudaSuccess ? WDAD_OK : cuda_fail(h, e, "screen exact reduced detector");
        }
        e = wdad::launch_detect_full(a, base + fixed, h->ws_bytes - fixed, h->num_sms, s);
        return e == cudaSuccess ? WDAD_OK : cuda_fail(h, e, "screen exact detector");
    } catch (...) {
        return fail(h, WDAD_ERR_NOMEM, "host exception");
    }
}

wdad_status wdad_adaptive_threshold(wdad_handle h, const float* score, int64_t n, double z_alpha, uint8_t* mask,
                                    double* host_stats, void* stream) {
    if (!h) return WDAD_ERR_ARG;
    if (n < 0 || (n > 0 && !score) || !std::isfinite(z_alpha))
        return fail(h, WDAD_ERR_ARG, "threshold: n >= 0, score for n > 0, finite z");
    try {
        DeviceGuard g(h->device);
        if (n == 0) {
            if (host_stats) { host_stats[0] = host_stats[1] = host_stats[2] = NAN; host_stats[3] = 0.0; }
            return WDAD_OK;
        }
        wdad_status st = ensure_ws(h, wdad::adaptive_threshold_workspace());
        if (st != WDAD_OK) return st;
        cudaStream_t s = (cudaStream_t)stream;
        cudaError_t e = wdad::launch_adaptive_threshold(score, n, z_alpha, h->ws, mask, host_stats, h->num_sms, s);
        if (e == cudaSuccess && host_stats) e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? WDAD_OK : cuda_fail(h, e, "adaptive threshold");
    } catch (...) {
        return fail(h, WDAD_ERR_NOMEM, "host exception");
    }
}

wdad_status wdad_auc(const float* score, const uint8_t* mask, int64_t n, double* auc) {
    if (!auc || n < 0 || (n > 0 && (!score || !mask))) return WDAD_ERR_ARG;
    try {
        std::vector<std::pair<float, uint8_t>> v((size_t)n);
        int64_t npos = 0;
        for (int64_t i = 0; i < n; ++i) {
            const float s = std::isnan(score[i]) ? -INFINITY : score[i];
            v[(size_t)i] = {s, (uint8_t)(mask[i] ? 1 : 0)};
            npos += mask[i] ? 1 : 0;
        }
        const int64_t nneg = n - npos;
        if (npos == 0 || nneg == 0) { *auc = NAN; return WDAD_OK; }
        std::sort(v.begin(), v.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        double rank_pos = 0.0;
        size_t i = 0;
        while (i < v.size()) {  // tied scores share their mean rank
            size_t j = i;
            while (j + 1 < v.size() && v[j + 1].first == v[i].first) ++j;
            const double r = 0.5 * ((double)i + (double)j) + 1.0;
            for (size_t k = i; k <= j; ++k) rank_pos += v[k].second ? r : 0.0;
            i = j + 1;
        }
        *auc = (rank_pos - 0.5 * (double)npos * (double)(npos + 1)) / ((double)npos * (double)nneg);
        return WDAD_OK;
    } catch (...) {
        return WDAD_ERR_NOMEM;
    }
}

}  // extern "C"
