// wdad_detect_all_noalloc: the DWT-reduced LRX + DWRX + DWEST pass without any device
// allocation.
//
// Some callers cannot call cudaMalloc.  A few examples:
//   - embedded or flight software that fixes its whole memory budget at start-up;
//   - a host application whose framework owns the device memory through its own pool,
//     where a foreign allocation would break the pool's accounting or its reserve;
//   - code on a latency-critical path, where cudaMalloc and cudaFree may block on,
//     or synchronise with, work already queued on the device.
// For them this entry point keeps its scratch in a file-scope __device__ array of fixed
// size that lives in the module for as long as the library is loaded: the K x L DWT
// matrix and the H x W x K approximation matrix.  The caller passes the cube and the
// score and flag buffers, as for wdad_detect_all.
#include "internal.h"

namespace {

constexpr size_t kMatFloats = 8 * 1024;             // DWT matrix: K <= 8 rows, L <= 1024 columns
constexpr size_t kApproxFloats = (size_t)1 << 22;   // approximation matrix: H * W * K <= 4,194,304

// Scratch shared by every call on a device (16 MiB + 32 KiB); each call overwrites the
// parts it reads, so nothing has to start at zero.
static __device__ __align__(256) float g_noalloc_scratch[kMatFloats + kApproxFloats];

// Device address of the scratch array in the current context (host code may not use the
// symbol itself as a pointer).  Looked up on every call, with the caller's device current:
// the lookup is not a stream operation, and a context that was torn down and made again
// (cudaDeviceReset) reloads the module, which can place the array elsewhere, so an address
// cached from an earlier context could point at memory the array no longer occupies.
cudaError_t scratch_ptr(float** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<float*>(p);
    return cudaSuccess;
}

bool params_ok(const wdad_params* p) {
    if (!p) return false;
    if (p->wavelet_taps < 2 || p->wavelet_taps > wdad::kMaxTaps || (p->wavelet_taps & 1)) return false;
    if (p->level < -1 || p->level > 30) return false;
    if (p->inner < 1 || !(p->inner & 1) || p->outer <= p->inner || !(p->outer & 1) || p->outer > 63) return false;
    if (!(p->loading >= 0.f) || !(p->loading < 3.0e38f)) return false;
    if (p->border != 0 && p->border != 1) return false;
    if (p->dwest_mode != 0 && p->dwest_mode != 1) return false;
    if (!(p->dwest_tau >= 0.f) || !(p->dwest_tau < 3.0e38f)) return false;
    return true;
}

}  // namespace

extern "C" wdad_status wdad_detect_all_noalloc(const float* cube, int H, int W, int L, const wdad_params* p,
                                               float* scores, uint8_t* flags, void* stream) {
    if (!params_ok(p) || H < 0 || W < 0 || L < 1) return WDAD_ERR_ARG;
    const int64_t P = (int64_t)H * W;
    if (P == 0) return WDAD_OK;
    if (!cube || !scores) return WDAD_ERR_ARG;
    if ((L % 4 == 0) && ((uintptr_t)cube & 15) != 0) return WDAD_ERR_ARG;
    int K = 0;
    const int J = wdad::dwt_levels(L, p->level, &K);
    if (L > 1024 || !wdad::dwt_shape_supported(L, K)) return WDAD_ERR_UNSUPPORTED;
    if ((size_t)P * (size_t)K > kApproxFloats) return WDAD_ERR_ARG;  // beyond the fixed scratch
    if (wdad::detect_small_smem(K, p->inner, p->outer, 1) > 227 * 1024) return WDAD_ERR_UNSUPPORTED;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WDAD_ERR_CUDA;
    float* base = nullptr;
    if (scratch_ptr(&base) != cudaSuccess) return WDAD_ERR_CUDA;
    int num_sms = 1;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WDAD_ERR_CUDA;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* A = base;                  // K x L
    float* approx = base + kMatFloats;  // H x W x K
    if (wdad::build_dwt_matrix(L, p->wavelet_taps, J, K, A, nullptr, s) != cudaSuccess) return WDAD_ERR_CUDA;
    if (wdad::launch_dwt_approx(cube, P, L, A, K, approx, num_sms, s) != cudaSuccess) return WDAD_ERR_CUDA;
    wdad::DetectArgs a{};
    a.x = approx; a.H = H; a.W = W; a.D = K;
    a.inner = p->inner; a.outer = p->outer; a.loading = p->loading; a.border = p->border;
    a.dwest_mode = p->dwest_mode; a.dwest_tau = p->dwest_tau;
    a.out[0] = scores; a.out[1] = scores + P; a.out[2] = scores + 2 * P;
    a.flags = flags;
    if (wdad::launch_detect_small(a, 16, s) != cudaSuccess) return WDAD_ERR_CUDA;
    return WDAD_OK;
}
