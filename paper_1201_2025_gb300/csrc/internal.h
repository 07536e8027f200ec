// Internal C++ interfaces between the C-ABI layer (capi.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <set>
#include <utility>

#include "../../include/wdad.h"

namespace wdad {

// The dynamic shared memory limit of a kernel, raised once per kernel and device to the opt-in
// maximum less the kernel's static shared memory, so that launches of different sizes from
// several host threads never lower it between another thread's set and launch.
template <class Kern>
inline cudaError_t raise_smem_limit(Kern* kernel) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;  // (kernel, device) pairs already raised
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(reinterpret_cast<const void*>(kernel), dev);
    if (done.count(key)) return cudaSuccess;
    int optin = 0;
    cudaFuncAttributes fa{};
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done.insert(key);
    return e;
}

// Device-side reflect-101 (-1 -> 1, n -> n-2), valid for any integer i.
__host__ __device__ __forceinline__ int reflect101(int i, int n) {
    if ((unsigned)i < (unsigned)n) return i;  // interior: no arithmetic
    if (n == 1) return 0;
    const int period = 2 * (n - 1);
    int r = i % period;
    if (r < 0) r += period;
    return r < n ? r : period - r;
}

// Number of approximation coefficients after J halvings; level < 0 = auto (K <= 4).
inline int dwt_levels(int L, int level, int* K) {
    int n = L, J = 0;
    if (level < 0) {
        while (n > 4) { n = (n + 1) / 2; ++J; }
    } else {
        for (J = 0; J < level; ++J) n = (n + 1) / 2;
    }
    if (K) *K = n;
    return J;
}

// Daubechies scaling filters (sum = sqrt 2): taps 8 = db4, taps 4 = D4.
constexpr int kMaxTaps = 20;  // Daubechies filters db1 .. db10
bool filter_coeffs(int taps, double* h);

// ---- A1: DWT approximation ---------------------------------------------------
// Builds the K x L approximation matrix (row-major) by running the Eq. 9
// cascade on the L unit spectra on the GPU (FP64, rounded once to float).
cudaError_t build_dwt_matrix(int L, int taps, int J, int K, float* A, double* scratch, cudaStream_t s);
// approx[P][K] = A x for every pixel spectrum of cube[P][L].
cudaError_t launch_dwt_approx(const float* cube, int64_t P, int L, const float* A, int K, float* approx,
                              int num_sms, cudaStream_t s);
bool dwt_shape_supported(int L, int K);
// The same kernel shaped to run beside another launch: at most ctas CTAs, each launched with
// `reserve` bytes of dynamic shared memory that it does not use, which bounds how many of its
// CTAs share an SM (and so leaves room for the other launch's CTAs).  Same coefficients.
cudaError_t launch_dwt_approx_beside(const float* cube, int64_t P, int L, const float* A, int K, float* approx,
                                     int num_sms, int ctas, size_t reserve, cudaStream_t s);

// ---- A2-A5: detectors on few bands (dim <= 8, the DWT-reduced cube) ---------
struct DetectArgs {
    const float* x;   // [H][W][D]
    int H, W, D;
    int inner, outer;
    float loading;
    int border;
    int dwest_mode;
    float dwest_tau;
    float* out[3];    // LRX, DWRX, DWEST maps (nullptr = not wanted)
    uint8_t* flags;   // nullable
};
cudaError_t launch_detect_small(const DetectArgs& a, int tile_h, cudaStream_t s);
// exact tile height (the plan); default plan of a configuration
cudaError_t launch_detect_small_th(const DetectArgs& a, int th, cudaStream_t s);
// up to kMaxWindowsPerLaunch windows of one cube (same x, H, W, D; default plans) in one launch
constexpr int kMaxWindowsPerLaunch = 4;
cudaError_t launch_detect_small_multi(const DetectArgs* a, int n, cudaStream_t s);
// the same for the tiles whose first row lies in [row0, row1) (a band of the image; the
// tiles read reduced rows up to row1 + th + outer / 2 - 2)
cudaError_t launch_detect_small_multi_rows(const DetectArgs* a, int n, int row0, int row1, cudaStream_t s);
int detect_small_default_th(int D, int inner, int outer);
// Global RX of Eq. 1 on a [P][L] cube (L <= kGlobalRxMaxBands), scores [P]; workspace from
// global_rx_workspace_bytes (0 for unsupported sizes).
constexpr int kGlobalRxMaxBands = 1024;
size_t global_rx_workspace_bytes(int64_t P, int L, int num_sms);
cudaError_t launch_global_rx(const float* x, int64_t P, int L, float loading, float* score, void* ws, size_t ws_bytes,
                             int num_sms, cudaStream_t s);

// Eq. 12 cut-off on a score map (ws: adaptive_threshold_workspace() bytes of device memory);
// stats_out (host, nullable): mu, sigma, tau, count, copied asynchronously on st
size_t adaptive_threshold_workspace();
cudaError_t launch_adaptive_threshold(const float* s, int64_t n, double z, void* ws, uint8_t* mask, double* stats_out,
                                      int num_sms, cudaStream_t st);
// largest dynamic shared memory of a detector tile plan that still lets two CTAs share an SM
size_t detect_small_two_per_sm_bytes();
cudaError_t launch_window_census(int H, int W, int inner, int outer, int border, int64_t* out,
                                 cudaStream_t s);
size_t detect_small_smem(int D, int inner, int outer, int tile_h);

// ---- full-band detectors (dim > 8) -------------------------------------------
struct FullArgs {
    const float* x;   // [H][W][D]
    int H, W, D;
    int inner, outer;
    float loading, cond_gate;
    int border, dwest_mode, precision;
    float dwest_tau;
    float* out[3];
    uint8_t* flags;
    int* status;  // nullable device word: set to a wdad_status when a bounded wait gives up
    const int64_t* pix;  // nullable: only these pixels (linear indices), npix of them
    int64_t npix;
};
size_t fullband_workspace_bytes(const FullArgs& a, int num_sms);
cudaError_t launch_detect_full(const FullArgs& a, void* ws, size_t ws_bytes, int num_sms, cudaStream_t s);
size_t moments_workspace_bytes(const FullArgs& a, int64_t npix, int num_sms);
cudaError_t launch_window_moments(const FullArgs& a, const int64_t* pix, int64_t npix, float* mu, float* cov, void* ws,
                                  size_t ws_bytes, int num_sms, cudaStream_t s);

}  // namespace wdad
