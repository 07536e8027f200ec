// C ABI of libwdad (declared in include/wdad.h): argument checking, the handle's
// workspace and plan caches, and dispatch to the kernels.  No exception leaves
// this file; every entry point returns a wdad_status.
#include <algorithm>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

struct wdad_ctx {
    int device = 0;
    int num_sms = 1;
    void* ws = nullptr;        // grow-only device workspace
    size_t ws_bytes = 0;
    struct DwtPlan { int L, taps, J, K; float* A; };
    std::vector<DwtPlan> dwt_plans;
    std::string err;
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
    if (p->wavelet_taps != 8 && p->wavelet_taps != 4)
        return fail(h, WDAD_ERR_ARG, "wavelet_taps must be 8 (db4) or 4 (D4), got %d", p->wavelet_taps);
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

// Runs A1 into the workspace (offset 0) and returns the reduced cube.
wdad_status reduce_into_ws(wdad_ctx* h, const float* cube, int H, int W, int L, const wdad_params* p,
                           const float** xr, int* K, cudaStream_t s) {
    const float* A = nullptr;
    wdad_status st = get_dwt_plan(h, L, p->wavelet_taps, p->level, &A, K, s);
    if (st != WDAD_OK) return st;
    const int64_t P = (int64_t)H * W;
    st = ensure_ws(h, sizeof(float) * (size_t)P * (*K) + 256);
    if (st != WDAD_OK) return st;
    cudaError_t e = wdad::launch_dwt_approx(cube, P, L, A, *K, (float*)h->ws, h->num_sms, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "dwt_approx launch");
    *xr = (const float*)h->ws;
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
    const float* x = cube;
    int D = L;
    if (reduce) {
        st = reduce_into_ws(h, cube, H, W, L, p, &x, &D, s);
        if (st != WDAD_OK) return st;
    }
    if (D <= 8) {
        wdad::DetectArgs a{};
        a.x = x; a.H = H; a.W = W; a.D = D;
        a.inner = p->inner; a.outer = p->outer; a.loading = p->loading; a.border = p->border;
        a.dwest_mode = p->dwest_mode; a.dwest_tau = p->dwest_tau;
        for (int t = 0; t < 3; ++t) a.out[t] = out3[t];
        a.flags = flags;
        if (wdad::detect_small_smem(D, p->inner, p->outer, 1) > 227 * 1024)
            return fail(h, WDAD_ERR_UNSUPPORTED, "window %d/%d too large for %d bands", p->inner, p->outer, D);
        cudaError_t e = wdad::launch_detect_small(a, 16, s);
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
    st = ensure_ws(h, need);
    if (st != WDAD_OK) return st;
    cudaError_t e = wdad::launch_detect_full(a, h->ws, h->ws_bytes, h->num_sms, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "detect_full launch");
    return WDAD_OK;
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
    if (L < 1 || (taps != 8 && taps != 4) || level < -1 || level > 30) return -1;
    int K = 0;
    wdad::dwt_levels(L, level, &K);
    return K;
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
