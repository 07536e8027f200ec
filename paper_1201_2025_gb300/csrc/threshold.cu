// Adaptive cut-off of Eq. 12 on a score map: tau = mu_d + z sigma_d, with mu_d and sigma_d
// the mean and the population standard deviation of the map's finite entries; a pixel is
// declared anomalous when its score exceeds tau.  Three launches: FP64 partial sums (count,
// sum, sum of squares) over THR_BLOCKS fixed pixel ranges, their combination by a tree of
// fixed shape (so the statistics are the same on any GPU), and the comparison that writes the
// binary map.  The one-pass variance sum/n - mean^2 is taken in FP64; detector scores have
// mean^2 / variance of order 1-10, so the cancellation costs a few units of 1e-16.
#include "internal.h"

namespace wdad {

constexpr int THR_BLOCKS = 512;
constexpr int THR_THREADS = 256;

__global__ void __launch_bounds__(THR_THREADS) thr_partials_kernel(const float* __restrict__ s, int64_t n,
                                                                   double* __restrict__ part) {
    __shared__ double red[3][THR_THREADS / 32];
    const int64_t chunk = (n + THR_BLOCKS - 1) / THR_BLOCKS;
    const int64_t i0 = blockIdx.x * chunk, i1 = i0 + chunk < n ? i0 + chunk : n;
    double c = 0.0, sum = 0.0, sq = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += THR_THREADS) {
        const float v = s[i];
        if (isfinite(v)) {
            const double d = (double)v;
            c += 1.0;
            sum += d;
            sq += d * d;
        }
    }
    for (int o = 16; o >= 1; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][warp] = c; red[1][warp] = sum; red[2][warp] = sq; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < THR_THREADS / 32; ++w) t += red[threadIdx.x][w];
        part[(size_t)blockIdx.x * 3 + threadIdx.x] = t;
    }
}

// stats = [mu, sigma, tau, count]; one block of THR_BLOCKS threads, pairwise halving
__global__ void __launch_bounds__(THR_BLOCKS) thr_finalize_kernel(const double* __restrict__ part, double z,
                                                                  double* __restrict__ stats) {
    __shared__ double r[3][THR_BLOCKS];
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 3; ++k) r[k][t] = part[3 * t + k];
    __syncthreads();
    for (int h = THR_BLOCKS / 2; h >= 1; h >>= 1) {
        if (t < h) {
#pragma unroll
            for (int k = 0; k < 3; ++k) r[k][t] += r[k][t + h];
        }
        __syncthreads();
    }
    if (t != 0) return;
    const double c = r[0][0], sum = r[1][0], sq = r[2][0];
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const double mu = c > 0.0 ? sum / c : nan;
    const double var = c > 0.0 ? fmax(sq / c - mu * mu, 0.0) : nan;
    const double sd = sqrt(var);
    stats[0] = mu;
    stats[1] = sd;
    stats[2] = mu + z * sd;
    stats[3] = c;
}

__global__ void thr_mask_kernel(const float* __restrict__ s, int64_t n, const double* __restrict__ stats,
                                uint8_t* __restrict__ mask) {
    const double tau = stats[2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = s[i];
        mask[i] = (uint8_t)(isfinite(v) && (double)v > tau);
    }
}

size_t adaptive_threshold_workspace() { return sizeof(double) * (3 * (size_t)THR_BLOCKS + 4) + 256; }

cudaError_t launch_adaptive_threshold(const float* s, int64_t n, double z, void* ws, uint8_t* mask, double* stats_out,
                                      int num_sms, cudaStream_t st) {
    double* part = reinterpret_cast<double*>(ws);
    double* stats = part + 3 * (size_t)THR_BLOCKS;
    thr_partials_kernel<<<THR_BLOCKS, THR_THREADS, 0, st>>>(s, n, part);
    thr_finalize_kernel<<<1, THR_BLOCKS, 0, st>>>(part, z, stats);
    if (mask && n > 0) {
        int64_t g = (n + 255) / 256;
        const int64_t cap = (int64_t)num_sms * 8;
        if (g > cap) g = cap;
        thr_mask_kernel<<<(unsigned)g, 256, 0, st>>>(s, n, stats, mask);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && stats_out) e = cudaMemcpyAsync(stats_out, stats, sizeof(double) * 4, cudaMemcpyDeviceToHost, st);
    return e;
}

}  // namespace wdad
