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
#include <complex>
#include <vector>

#include "dwt_dev.cuh"

namespace wdad {

// ---- Daubechies scaling filters with taps / 2 vanishing moments, taps = 2 .. kMaxTaps.
// Daubechies' construction (Ten Lectures on Wavelets, Sec. 6.1): with p = taps / 2,
// |m0(w)|^2 = cos^2p(w/2) P(sin^2(w/2)), P(y) = sum_{k<p} C(p-1+k, k) y^k.  Each root y_j of
// P gives the pair z, 1/z of z + 1/z = 2 - 4 y_j; keeping the root outside the unit circle
// for every pair gives the extremal-phase filter, h(w) ~ (1 + w)^p prod_j (w - z_j), scaled
// to sum(h) = sqrt(2) (db4 = taps 8, D4 = taps 4).  Roots of P: Laguerre's method with
// deflation, each root then refined on the undeflated polynomial.
using cplx = std::complex<double>;

static cplx laguerre_root(const std::vector<cplx>& a, cplx z) {
    const int n = (int)a.size() - 1;  // degree, a ascending
    for (int it = 0; it < 100; ++it) {
        cplx p = a[n], dp = 0.0, d2p = 0.0;
        for (int k = n - 1; k >= 0; --k) {
            d2p = d2p * z + dp;
            dp = dp * z + p;
            p = p * z + a[k];
        }
        d2p *= 2.0;
        if (std::abs(p) == 0.0) break;
        const cplx G = dp / p, Hs = G * G - d2p / p;
        const cplx sq = std::sqrt((double)(n - 1) * ((double)n * Hs - G * G));
        const cplx den = std::abs(G + sq) >= std::abs(G - sq) ? G + sq : G - sq;
        const cplx step = std::abs(den) > 0.0 ? (double)n / den : cplx(1e-3 * (1.0 + std::abs(z)), 0.0);
        z -= step;
        if (std::abs(step) <= 4e-16 * std::abs(z)) break;
    }
    return z;
}

bool filter_coeffs(int taps, double* h) {
    if (taps < 2 || taps > kMaxTaps || (taps & 1)) return false;
    const int p = taps / 2, n = p - 1;
    std::vector<cplx> P(n + 1), a;
    double c = 1.0;
    for (int k = 0; k <= n; ++k) {  // C(p-1+k, k)
        P[k] = c;
        c = c * (double)(p + k) / (double)(k + 1);
    }
    std::vector<cplx> w(1, cplx(1.0, 0.0));  // ascending coefficients of the filter polynomial
    auto times = [&w](cplx root) {            // w <- w * (x - root)
        w.push_back(0.0);
        for (int i = (int)w.size() - 1; i >= 1; --i) w[i] = w[i - 1] - root * w[i];
        w[0] = -root * w[0];
    };
    for (int k = 0; k < p; ++k) times(cplx(-1.0, 0.0));
    a = P;
    for (int d = n; d >= 1; --d) {
        cplx y = laguerre_root(a, cplx(0.0, 0.0));
        y = laguerre_root(P, y);
        // deflate a by (x - y)
        std::vector<cplx> b(d);
        b[d - 1] = a[d];
        for (int k = d - 1; k >= 1; --k) b[k - 1] = a[k] + y * b[k];
        a.swap(b);
        const cplx q = 2.0 - 4.0 * y, disc = std::sqrt(q * q - 4.0);
        const cplx z1 = 0.5 * (q + disc), z2 = 0.5 * (q - disc);
        times(std::abs(z1) >= std::abs(z2) ? z1 : z2);
    }
    double sum = 0.0;
    for (int i = 0; i < taps; ++i) sum += w[i].real();
    for (int i = 0; i < taps; ++i) h[i] = w[i].real() * std::sqrt(2.0) / sum;
    return true;
}

struct Filter { double h[kMaxTaps]; int taps; };

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

// ctas > 0 caps the grid at that many CTAs; reserve > 0 launches with that much dynamic shared
// memory, which the kernel does not use: it only limits how many CTAs share an SM.
template <int VEC, int NCH, int KP>
static cudaError_t launch_one(const float* cube, int64_t P, int L, const float* A, int K, float* out, int num_sms,
                              cudaStream_t s, int ctas, size_t reserve) {
    constexpr int PX = px_per_step(NCH, KP);
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, dwt_apply_kernel<VEC, NCH, KP>, 256, 0);
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    const int64_t ngroups = (P + PX - 1) / PX;
    int64_t grid = (ngroups + 7) / 8;
    const int64_t cap = ctas > 0 ? (int64_t)ctas : (int64_t)num_sms * blocks_per_sm;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    if (reserve > 0) {
        cudaError_t e = raise_smem_limit(dwt_apply_kernel<VEC, NCH, KP>);
        if (e != cudaSuccess) return e;
    }
    dwt_apply_kernel<VEC, NCH, KP><<<(unsigned)grid, 256, reserve, s>>>(cube, P, L, A, K, out);
    return cudaGetLastError();
}

// Instantiated (VEC, NCH, KP) combinations; dwt_shape_supported() admits exactly these.
template <int VEC, int KP>
static cudaError_t dispatch_nch(int nch, const float* cube, int64_t P, int L, const float* A, int K, float* out,
                                int num_sms, cudaStream_t s, int ctas, size_t reserve) {
    if (nch <= 1) return launch_one<VEC, 1, KP>(cube, P, L, A, K, out, num_sms, s, ctas, reserve);
    if (nch <= 2) return launch_one<VEC, 2, KP>(cube, P, L, A, K, out, num_sms, s, ctas, reserve);
    if constexpr (VEC == 4 && KP == 8) return cudaErrorInvalidValue;
    if (nch <= 3) return launch_one<VEC, 3, KP>(cube, P, L, A, K, out, num_sms, s, ctas, reserve);
    if (nch <= 4) return launch_one<VEC, 4, KP>(cube, P, L, A, K, out, num_sms, s, ctas, reserve);
    if constexpr (KP <= 4) {
        if (nch <= 6) return launch_one<VEC, 6, KP>(cube, P, L, A, K, out, num_sms, s, ctas, reserve);
        if (nch <= 8) return launch_one<VEC, 8, KP>(cube, P, L, A, K, out, num_sms, s, ctas, reserve);
    }
    return cudaErrorInvalidValue;
}

static cudaError_t dwt_dispatch(const float* cube, int64_t P, int L, const float* A, int K, float* approx,
                                int num_sms, cudaStream_t s, int ctas, size_t reserve) {
    if (P == 0) return cudaSuccess;
    if (!dwt_shape_supported(L, K)) return cudaErrorInvalidValue;
    const int kp = kpad(K);
    if (L % 4 == 0) {
        const int nch = (L / 4 + 31) / 32;
        switch (kp) {
            case 1: return dispatch_nch<4, 1>(nch, cube, P, L, A, K, approx, num_sms, s, ctas, reserve);
            case 2: return dispatch_nch<4, 2>(nch, cube, P, L, A, K, approx, num_sms, s, ctas, reserve);
            case 4: return dispatch_nch<4, 4>(nch, cube, P, L, A, K, approx, num_sms, s, ctas, reserve);
            default: return dispatch_nch<4, 8>(nch, cube, P, L, A, K, approx, num_sms, s, ctas, reserve);
        }
    }
    const int nch = (L + 31) / 32;
    switch (kp) {
        case 1: return dispatch_nch<1, 1>(nch, cube, P, L, A, K, approx, num_sms, s, ctas, reserve);
        case 2: return dispatch_nch<1, 2>(nch, cube, P, L, A, K, approx, num_sms, s, ctas, reserve);
        case 4: return dispatch_nch<1, 4>(nch, cube, P, L, A, K, approx, num_sms, s, ctas, reserve);
        default: return dispatch_nch<1, 8>(nch, cube, P, L, A, K, approx, num_sms, s, ctas, reserve);
    }
}

cudaError_t launch_dwt_approx(const float* cube, int64_t P, int L, const float* A, int K, float* approx, int num_sms,
                              cudaStream_t s) {
    return dwt_dispatch(cube, P, L, A, K, approx, num_sms, s, 0, 0);
}

cudaError_t launch_dwt_approx_beside(const float* cube, int64_t P, int L, const float* A, int K, float* approx,
                                     int num_sms, int ctas, size_t reserve, cudaStream_t s) {
    if (ctas < 1) return cudaErrorInvalidValue;
    return dwt_dispatch(cube, P, L, A, K, approx, num_sms, s, ctas, reserve);
}

}  // namespace wdad
