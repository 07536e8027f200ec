// A1 — band-axis Daubechies DWT, approximation coefficients only (Sec. 4; Eq. 7/9; Fig. 1).
//
// The J-level low-pass cascade with periodic extension is a fixed linear map
// a = A x from L bands to K coefficients.  A is built once per (L, taps, J) by
// running the literal Eq. 9 cascade on the L unit spectra (FP64 on the GPU,
// rounded once to float).  The hot kernel then streams the cube: one warp takes
// a group of PX pixels, each lane loads 16-byte chunks of every pixel's spectrum
// (coalesced 512 B per warp instruction), multiplies them with its slice of A held
// in registers (the "filter bank in registers"), and a 5-step reduce-scatter
// butterfly leaves lane l with coefficient (pixel l / KP, k = l % KP), so the
// PX*K results leave as one coalesced store.  The lane partial sums plus the tree
// of shuffles keep the FP32 rounding error near sqrt(L) ulp instead of L ulp.
#include "dwt_dev.cuh"

namespace wdad {

bool filter_coeffs(int taps, double* h) {
    if (taps == 8) {
        // Daubechies' 4-vanishing-moment scaling filter (Ten Lectures on Wavelets, Table 6.1)
        static const double db4[8] = {0.2303778133088964,  0.7148465705529154,  0.6308807679298587,
                                      -0.0279837694168599, -0.1870348117190931, 0.0308413818355607,
                                      0.0328830116668852,  -0.0105974017850690};
        for (int i = 0; i < 8; ++i) h[i] = db4[i];
        return true;
    }
    if (taps == 4) {
        const double s3 = sqrt(3.0), r = 4.0 * sqrt(2.0);
        h[0] = (1.0 + s3) / r; h[1] = (3.0 + s3) / r; h[2] = (3.0 - s3) / r; h[3] = (1.0 - s3) / r;
        return true;
    }
    return false;
}

struct Filter { double h[8]; int taps; };

// One block per band l: cascade of Eq. 9 steps on the unit spectrum e_l.
__global__ void dwt_matrix_kernel(int L, int J, int K, Filter f, float* __restrict__ A) {
    extern __shared__ double buf[];
    double* a = buf;
    double* b = buf + (L + 2);
    const int l = blockIdx.x;
    for (int i = threadIdx.x; i < L; i += blockDim.x) a[i] = (i == l) ? 1.0 : 0.0;
    __syncthreads();
    int n = L;
    for (int j = 0; j < J; ++j) {
        const int M = n + (n & 1), m = M / 2;
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            double s = 0.0;
            for (int t = 0; t < f.taps; ++t) {
                int idx = (2 * k - t) % M;
                if (idx < 0) idx += M;
                s += f.h[t] * (idx < n ? a[idx] : a[n - 1]);  // odd n: pad with the last sample
            }
            b[k] = s;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += blockDim.x) a[k] = b[k];
        __syncthreads();
        n = m;
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) A[(size_t)k * L + l] = (float)a[k];
}

cudaError_t build_dwt_matrix(int L, int taps, int J, int K, float* A, double* /*scratch*/, cudaStream_t s) {
    Filter f{};
    if (!filter_coeffs(taps, f.h)) return cudaErrorInvalidValue;
    f.taps = taps;
    const size_t smem = sizeof(double) * 2 * (L + 2);
    dwt_matrix_kernel<<<L, 128, smem, s>>>(L, J, K, f, A);
    return cudaGetLastError();
}

static int kpad(int K) { return K <= 1 ? 1 : K <= 2 ? 2 : K <= 4 ? 4 : 8; }

bool dwt_shape_supported(int L, int K) {
    if (L < 1 || K < 1 || K > 8) return false;
    if (L % 4 == 0) return (L + 127) / 128 <= (K <= 4 ? 8 : 2);
    return (L + 31) / 32 <= (K <= 4 ? 8 : 4);
}

template <int VEC, int NCH, int KP>
static cudaError_t launch_one(const float* cube, int64_t P, int L, const float* A, int K, float* out, int num_sms,
                              cudaStream_t s) {
    constexpr int PX = px_per_step(NCH, KP);
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, dwt_apply_kernel<VEC, NCH, KP>, 256, 0);
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    const int64_t ngroups = (P + PX - 1) / PX;
    int64_t grid = (ngroups + 7) / 8;
    const int64_t cap = (int64_t)num_sms * blocks_per_sm;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    dwt_apply_kernel<VEC, NCH, KP><<<(unsigned)grid, 256, 0, s>>>(cube, P, L, A, K, out);
    return cudaGetLastError();
}

// Instantiated (VEC, NCH, KP) combinations; dwt_shape_supported() admits exactly these.
template <int VEC, int KP>
static cudaError_t dispatch_nch(int nch, const float* cube, int64_t P, int L, const float* A, int K, float* out,
                                int num_sms, cudaStream_t s) {
    if (nch <= 1) return launch_one<VEC, 1, KP>(cube, P, L, A, K, out, num_sms, s);
    if (nch <= 2) return launch_one<VEC, 2, KP>(cube, P, L, A, K, out, num_sms, s);
    if constexpr (VEC == 4 && KP == 8) return cudaErrorInvalidValue;
    if (nch <= 3) return launch_one<VEC, 3, KP>(cube, P, L, A, K, out, num_sms, s);
    if (nch <= 4) return launch_one<VEC, 4, KP>(cube, P, L, A, K, out, num_sms, s);
    if constexpr (KP <= 4) {
        if (nch <= 6) return launch_one<VEC, 6, KP>(cube, P, L, A, K, out, num_sms, s);
        if (nch <= 8) return launch_one<VEC, 8, KP>(cube, P, L, A, K, out, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_dwt_approx(const float* cube, int64_t P, int L, const float* A, int K, float* approx, int num_sms,
                              cudaStream_t s) {
    if (P == 0) return cudaSuccess;
    if (!dwt_shape_supported(L, K)) return cudaErrorInvalidValue;
    const int kp = kpad(K);
    if (L % 4 == 0) {
        const int nch = (L / 4 + 31) / 32;
        switch (kp) {
            case 1: return dispatch_nch<4, 1>(nch, cube, P, L, A, K, approx, num_sms, s);
            case 2: return dispatch_nch<4, 2>(nch, cube, P, L, A, K, approx, num_sms, s);
            case 4: return dispatch_nch<4, 4>(nch, cube, P, L, A, K, approx, num_sms, s);
            default: return dispatch_nch<4, 8>(nch, cube, P, L, A, K, approx, num_sms, s);
        }
    }
    const int nch = (L + 31) / 32;
    switch (kp) {
        case 1: return dispatch_nch<1, 1>(nch, cube, P, L, A, K, approx, num_sms, s);
        case 2: return dispatch_nch<1, 2>(nch, cube, P, L, A, K, approx, num_sms, s);
        case 4: return dispatch_nch<1, 4>(nch, cube, P, L, A, K, approx, num_sms, s);
        default: return dispatch_nch<1, 8>(nch, cube, P, L, A, K, approx, num_sms, s);
    }
}

}  // namespace wdad
