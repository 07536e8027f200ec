// Global RX (Eq. 1, Sec. 2.1): s(r) = (r - mu)^T (C + delta I)^-1 (r - mu), with mu and
// C = (1/P) sum (x - mu)(x - mu)^T over every pixel of the image and delta = loading tr(C) / L
// (the loading rule of the local detectors).  Six launches:
//   (1) grx_colsum: FP32 band sums over fixed ranges of GRX_CHUNK pixels, stored as FP64;
//   (2) grx_mean: the range sums of each band added by a fixed-shape tree in FP64 -> mu;
//   (3) grx_gram: per fixed pixel range, the centred Gram sum in FP32, one 8 x 8 register tile
//       of the lower triangle per thread, the range staged through shared memory;
//   (4) grx_gram_reduce: the range partials of every entry added in range order in FP64, / P;
//   (5) grx_invert: one block turns C + delta I into its inverse with the symmetric sweep
//       operator (Gauss-Jordan elimination that keeps the matrix symmetric, so only the lower
//       triangle is stored and updated), FP32: in registers (8 x 8 tiles, one per thread) up to
//       248 bands, else in shared memory when it fits, else in global memory;
//   (6) grx_score: per pixel s = d^T B d with d = x - mu, from the strict lower triangle and
//       the diagonal of the symmetric B (about half the multiply-adds of y = B d); lane i reads
//       row k of B at column i (coalesced), eight pixels per warp share every load.
// A pivot at or below the floor (the matrix is not numerically positive definite) sets the
// status word and every score becomes NaN.
#include <float.h>

#include "internal.h"

namespace wdad {
namespace {

constexpr int GRX_CHUNK = 512;      // pixels per band-sum range
constexpr int GRX_THREADS = 512;    // Gram and inversion blocks
constexpr int GRX_SCORE_THREADS = 256;
constexpr int GRX_INV_SMEM_FLOATS = 52 * 1024;  // packed lower triangle held in shared memory up to this size

__host__ __device__ inline int ntri(int n) { return n * (n + 1) / 2; }

__device__ __forceinline__ void tri_decode(int u, int& r, int& c) {  // u = r (r + 1) / 2 + c, c <= r
    r = (int)((sqrtf(8.f * (float)u + 1.f) - 1.f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= u) ++r;
    while (r * (r + 1) / 2 > u) --r;
    c = u - r * (r + 1) / 2;
}

// (1) part[blk][b] = sum of band b over pixels [blk * GRX_CHUNK, ...)
__global__ void __launch_bounds__(256) grx_colsum_kernel(const float* __restrict__ x, int64_t P, int L,
                                                         double* __restrict__ part) {
    const int64_t p0 = (int64_t)blockIdx.x * GRX_CHUNK;
    const int64_t p1 = p0 + GRX_CHUNK < P ? p0 + GRX_CHUNK : P;
    for (int b = threadIdx.x; b < L; b += blockDim.x) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        int64_t p = p0;
        for (; p + 3 < p1; p += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += __ldg(x + (p + u) * L + b);
        }
        for (; p < p1; ++p) acc[0] += __ldg(x + p * L + b);
        part[(size_t)blockIdx.x * L + b] = ((double)acc[0] + (double)acc[1]) + ((double)acc[2] + (double)acc[3]);
    }
}

// (2) one block per band: mu[b] = sum over ranges / P (fixed tree of 256 lanes)
__global__ void __launch_bounds__(256) grx_mean_kernel(const double* __restrict__ part, int nblk, int L, int64_t P,
                                                       float* __restrict__ mu) {
    __shared__ double r[256];
    const int b = blockIdx.x;
    double s = 0.0;
    for (int k = threadIdx.x; k < nblk; k += 256) s += part[(size_t)k * L + b];
    r[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h >= 1; h >>= 1) {
        if (threadIdx.x < h) r[threadIdx.x] += r[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) mu[b] = (float)(r[0] / (double)P);
}

// (3) block (range, group): pixel range blockIdx.x; thread = one 8 x 8 tile (I, K), I >= K, of
// the lower triangle, tile index blockIdx.y * GRX_THREADS + threadIdx.x.  Centred values staged
// S pixels at a time as xs[s][Lp8], zero beyond L and beyond the range.
__global__ void __launch_bounds__(GRX_THREADS, 1) grx_gram_kernel(const float* __restrict__ x, int64_t P, int L,
                                                                  int64_t range, const float* __restrict__ mu,
                                                                  int S, float* __restrict__ part) {
    extern __shared__ __align__(16) float xs[];
    const int nst = (L + 7) / 8, Lp8 = nst * 8, nstl = ntri(nst);
    const int u = blockIdx.y * GRX_THREADS + threadIdx.x;
    const bool own = u < nstl;
    int I = 0, K = 0;
    if (own) tri_decode(u, I, K);
    float acc[64];
#pragma unroll
    for (int e = 0; e < 64; ++e) acc[e] = 0.f;
    const int64_t p0 = (int64_t)blockIdx.x * range;
    const int64_t p1 = p0 + range < P ? p0 + range : P;
    for (int64_t c0 = p0; c0 < p1; c0 += S) {
        __syncthreads();
        const int n = S * Lp8;
        for (int e0 = threadIdx.x; e0 < n; e0 += 4 * GRX_THREADS) {
            float v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = e0 + q * GRX_THREADS;
                const int s = e / Lp8, b = e - s * Lp8;
                const int64_t p = c0 + s;
                v[q] = (e < n && p < p1 && b < L) ? __ldg(x + p * L + b) - __ldg(mu + b) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = e0 + q * GRX_THREADS;
                if (e < n) xs[e] = v[q];
            }
        }
        __syncthreads();
        if (own) {
            for (int s = 0; s < S; ++s) {
                const float4* row = reinterpret_cast<const float4*>(xs + (size_t)s * Lp8);
                const float4 a0 = row[2 * I], a1 = row[2 * I + 1], b0 = row[2 * K], b1 = row[2 * K + 1];
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[r * 8 + c] = fmaf(a[r], bb[c], acc[r * 8 + c]);
            }
        }
    }
    if (own) {
        float* o = part + ((size_t)blockIdx.x * nstl + u) * 64;
#pragma unroll
        for (int e = 0; e < 64; e += 4)
            *reinterpret_cast<float4*>(o + e) = make_float4(acc[e], acc[e + 1], acc[e + 2], acc[e + 3]);
    }
}

// (4) entry (tile u, e) of C: sum over the nblk ranges in range order, / P; written into the
// packed lower triangle M[i (i + 1) / 2 + j], j <= i < L, and the FP64 diagonal diag[i].
__global__ void grx_gram_reduce_kernel(const float* __restrict__ part, int nblk, int L, int64_t P,
                                       float* __restrict__ M, double* __restrict__ diag) {
    const int nst = (L + 7) / 8, nstl = ntri(nst);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nstl * 64) return;
    const int u = t >> 6, e = t & 63;
    int I, K;
    tri_decode(u, I, K);
    const int i = 8 * I + (e >> 3), j = 8 * K + (e & 7);
    if (i >= L || j > i) return;  // the diagonal tiles hold both triangles: keep j <= i
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += (double)part[((size_t)k * nstl + u) * 64 + e];
    s /= (double)P;
    M[(size_t)ntri(i) + j] = (float)s;
    if (i == j) diag[i] = s;
}

// (5) one block: M <- -(M + delta I)^-1 by sweeping every pivot (symmetric sweep operator:
// a_ij -= a_ik a_kj / a_kk, a_ik /= a_kk, a_kk = -1 / a_kk), then B = -M written in full.
__global__ void __launch_bounds__(GRX_THREADS) grx_invert_kernel(float* __restrict__ Mg, const double* __restrict__ diag,
                                                                 int L, float loading, float* __restrict__ B,
                                                                 int* __restrict__ status, int in_smem) {
    extern __shared__ __align__(16) float sm[];
    float* col = sm;                                   // [L] column k before the sweep
    float* M = in_smem ? sm + ((L + 3) & ~3) : Mg;     // packed lower triangle
    __shared__ float s_floor, s_delta;
    __shared__ int s_fail;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = GRX_THREADS / 32;
    const int n = ntri(L);
    if (threadIdx.x == 0) {
        double tr = 0.0, dmax = 0.0;
        for (int i = 0; i < L; ++i) { tr += diag[i]; dmax = fmax(dmax, diag[i]); }
        s_delta = (float)((double)loading * tr / (double)L);
        s_floor = 16.f * FLT_EPSILON * (float)(dmax + (double)s_delta);
        s_fail = 0;
    }
    if (in_smem)
        for (int t = threadIdx.x; t < n; t += GRX_THREADS) M[t] = Mg[t];
    __syncthreads();
    for (int i = threadIdx.x; i < L; i += GRX_THREADS) M[ntri(i) + i] += s_delta;
    __syncthreads();
    for (int k = 0; k < L; ++k) {
        for (int i = threadIdx.x; i < L; i += GRX_THREADS) col[i] = i >= k ? M[ntri(i) + k] : M[ntri(k) + i];
        __syncthreads();
        const float piv = col[k];
        if (!(piv > s_floor)) {  // uniform: every thread reads the same pivot
            if (threadIdx.x == 0) s_fail = 1;
            break;
        }
        const float inv = 1.f / piv;
        for (int i = warp; i < L; i += nw) {
            if (i == k) continue;
            const float ci = col[i] * inv;
            float* row = M + ntri(i);
            for (int j = lane; j <= i; j += 32) {
                if (j == k) continue;
                row[j] = fmaf(-ci, col[j], row[j]);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < L; i += GRX_THREADS) {
            if (i == k) M[ntri(k) + k] = -inv;
            else if (i > k) M[ntri(i) + k] = col[i] * inv;
            else M[ntri(k) + i] = col[i] * inv;
        }
        __syncthreads();
    }
    __syncthreads();
    if (s_fail) {
        if (threadIdx.x == 0) *status = 1;
        return;
    }
    if (threadIdx.x == 0) *status = 0;
    for (int t = threadIdx.x; t < L * L; t += GRX_THREADS) {
        const int i = t / L, j = t - i * L;
        B[t] = -(j <= i ? M[ntri(i) + j] : M[ntri(j) + i]);
    }
}

// column KC of a register tile to col[8 I ..], row KC to col[8 K ..]; the sweep's new values
// of that column / row (compile-time register offsets, selected by a switch on k % 8)
template <int KC>
__device__ __forceinline__ void tile_col_out(const float (&a)[64], float* col, int I) {
#pragma unroll
    for (int r = 0; r < 8; ++r) col[8 * I + r] = a[r * 8 + KC];
}
template <int KC>
__device__ __forceinline__ void tile_row_out(const float (&a)[64], float* col, int K) {
#pragma unroll
    for (int c = 0; c < 8; ++c) col[8 * K + c] = a[KC * 8 + c];
}
template <int KC>
__device__ __forceinline__ void tile_col_set(float (&a)[64], const float (&ci)[8], int I, int k, float inv) {
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r * 8 + KC] = 8 * I + r == k ? -inv : ci[r];
}
template <int KC>
__device__ __forceinline__ void tile_row_set(float (&a)[64], const float (&cj)[8], int K, int k, float inv) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[KC * 8 + c] = 8 * K + c == k ? -inv : cj[c] * inv;
}
#define GRX_SWITCH8(kc, CALL) \
    switch (kc) {                \
        case 0: CALL(0); break;  \
        case 1: CALL(1); break;  \
        case 2: CALL(2); break;  \
        case 3: CALL(3); break;  \
        case 4: CALL(4); break;  \
        case 5: CALL(5); break;  \
        case 6: CALL(6); break;  \
        default: CALL(7); break; \
    }

// (5') the same sweep with the matrix in registers, for L <= 8 * 31: thread u holds the 8 x 8
// tile (I, K) of the lower triangle (diagonal tiles hold both triangles, padding is zero).
// Step k: the owners of column k (and of row k left of the diagonal tile) publish it to col[],
// every tile takes a_ij -= (a_ik / a_kk) a_kj, and the owners then set a_ik = a_ik / a_kk
// and a_kk = -1 / a_kk.  Register arrays are indexed by compile-time offsets only.
__global__ void __launch_bounds__(GRX_THREADS, 1) grx_invert_regs_kernel(const float* __restrict__ Mg,
                                                                         const double* __restrict__ diag, int L,
                                                                         float loading, float* __restrict__ B,
                                                                         int* __restrict__ status) {
    __shared__ __align__(16) float col[8 * 32];
    __shared__ float s_floor, s_delta;
    const int nst = (L + 7) / 8, nstl = ntri(nst);
    const int u = threadIdx.x;
    const bool own = u < nstl;
    int I = 0, K = 0;
    if (own) tri_decode(u, I, K);
    if (threadIdx.x == 0) {
        double tr = 0.0, dmax = 0.0;
        for (int i = 0; i < L; ++i) { tr += diag[i]; dmax = fmax(dmax, diag[i]); }
        s_delta = (float)((double)loading * tr / (double)L);
        s_floor = 16.f * FLT_EPSILON * (float)(dmax + (double)s_delta);
    }
    for (int i = threadIdx.x; i < 8 * 32; i += GRX_THREADS) col[i] = 0.f;
    __syncthreads();
    float a[64];
#pragma unroll
    for (int e = 0; e < 64; ++e) {
        const int i = 8 * I + (e >> 3), j = 8 * K + (e & 7);
        float v = 0.f;
        if (own && i < L && j < L) {
            v = j <= i ? Mg[ntri(i) + j] : Mg[ntri(j) + i];
            if (i == j) v += s_delta;
        }
        a[e] = v;
    }
    bool fail = false;
    for (int k = 0; k < L; ++k) {
        const int kt = k >> 3, kc = k & 7;
        if (own && K == kt) {
#define GRX_C(n) tile_col_out<n>(a, col, I)
            GRX_SWITCH8(kc, GRX_C)
#undef GRX_C
        } else if (own && I == kt) {
#define GRX_R(n) tile_row_out<n>(a, col, K)
            GRX_SWITCH8(kc, GRX_R)
#undef GRX_R
        }
        __syncthreads();
        const float piv = col[k];
        if (!(piv > s_floor)) { fail = true; break; }  // uniform
        const float inv = 1.f / piv;
        if (own) {
            float ci[8], cj[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int i = 8 * I + r;
                ci[r] = i == k ? 0.f : col[i] * inv;
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int j = 8 * K + c;
                cj[c] = j == k ? 0.f : col[j];
            }
#pragma unroll
            for (int e = 0; e < 64; ++e) a[e] = fmaf(-ci[e >> 3], cj[e & 7], a[e]);
            if (K == kt) {
#define GRX_C(n) tile_col_set<n>(a, ci, I, k, inv)
                GRX_SWITCH8(kc, GRX_C)
#undef GRX_C
            }
            if (I == kt) {
#define GRX_R(n) tile_row_set<n>(a, cj, K, k, inv)
                GRX_SWITCH8(kc, GRX_R)
#undef GRX_R
            }
        }
        __syncthreads();
    }
    if (fail) {
        if (threadIdx.x == 0) *status = 1;
        return;
    }
    if (threadIdx.x == 0) *status = 0;
    if (own) {
#pragma unroll
        for (int e = 0; e < 64; ++e) {
            const int i = 8 * I + (e >> 3), j = 8 * K + (e & 7);
            if (i < L && j < L) {
                B[(size_t)i * L + j] = -a[e];
                if (I != K) B[(size_t)j * L + i] = -a[e];
            }
        }
    }
}

// (6) warp w: pixels p0 + w PW .. + PW - 1; lane l: rows i = l + 32 m, m < M
template <int M, int PW>
__global__ void __launch_bounds__(GRX_SCORE_THREADS) grx_score_kernel(const float* __restrict__ x, int64_t P, int L,
                                                                      const float* __restrict__ mu,
                                                                      const float* __restrict__ B,
                                                                      const int* __restrict__ status,
                                                                      float* __restrict__ score) {
    extern __shared__ __align__(16) float ds[];  // [PX][L] centred pixels
    constexpr int PX = PW * (GRX_SCORE_THREADS / 32);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p0 = (int64_t)blockIdx.x * PX;
    for (int e = threadIdx.x; e < PX * L; e += GRX_SCORE_THREADS) {
        const int q = e / L, b = e - q * L;
        const int64_t p = p0 + q;
        ds[e] = p < P ? __ldg(x + p * L + b) - __ldg(mu + b) : 0.f;
    }
    __syncthreads();
    const float* dw = ds + (size_t)warp * PW * L;
    float acc[PW][M];
#pragma unroll
    for (int q = 0; q < PW; ++q)
#pragma unroll
        for (int m = 0; m < M; ++m) acc[q][m] = 0.f;
    // acc_i = sum over k < i of B_ik d_k (the strict lower triangle), k in segments of 32: in
    // segment t only row blocks m >= t take part (compile-time bounds after unrolling t)
#pragma unroll
    for (int t = 0; t < M; ++t) {
        const int k1 = L < 32 * t + 32 ? L : 32 * t + 32;
#pragma unroll 2
        for (int k = 32 * t; k < k1; ++k) {
            float dk[PW];
#pragma unroll
            for (int q = 0; q < PW; ++q) dk[q] = dw[q * L + k];
#pragma unroll
            for (int m = t; m < M; ++m) {
                const int i = lane + 32 * m;
                const float bk = (i < L && k < i) ? __ldg(B + (size_t)k * L + i) : 0.f;
#pragma unroll
                for (int q = 0; q < PW; ++q) acc[q][m] = fmaf(bk, dk[q], acc[q][m]);
            }
        }
    }
    const bool failed = *status != 0;
#pragma unroll
    for (int q = 0; q < PW; ++q) {
        float s = 0.f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int i = lane + 32 * m;
            if (i < L) {  // s = sum_i d_i (B_ii d_i + 2 acc_i)
                const float di = dw[q * L + i];
                s = fmaf(di, fmaf(__ldg(B + (size_t)i * L + i), di, 2.f * acc[q][m]), s);
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const int64_t p = p0 + warp * PW + q;
        if (lane == 0 && p < P) score[p] = failed ? __int_as_float(0x7fc00000) : s;
    }
}

// (6') L % 4 == 0: lane l holds rows 128 g + 4 l .. + 3 (g < G), so one 16-byte load brings
// four entries of row k of B, and four k steps of a pixel's d come in one 16-byte shared load.
// Blocks of 128 x 128 below the diagonal count twice and those above it are skipped.
template <int G, int PW>
__global__ void __launch_bounds__(GRX_SCORE_THREADS, 2) grx_score4_kernel(const float* __restrict__ x, int64_t P, int L,
                                                                       const float* __restrict__ mu,
                                                                       const float* __restrict__ B,
                                                                       const int* __restrict__ status,
                                                                       float* __restrict__ score) {
    extern __shared__ __align__(16) float ds[];  // [PX][L] centred pixels
    constexpr int PX = PW * (GRX_SCORE_THREADS / 32);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p0 = (int64_t)blockIdx.x * PX;
    for (int e = threadIdx.x; e < PX * L; e += GRX_SCORE_THREADS) {
        const int q = e / L, b = e - q * L;
        const int64_t p = p0 + q;
        ds[e] = p < P ? __ldg(x + p * L + b) - __ldg(mu + b) : 0.f;
    }
    __syncthreads();
    const float* dw = ds + (size_t)warp * PW * L;
    float acc[PW][G][4];
#pragma unroll
    for (int q = 0; q < PW; ++q)
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[q][g][j] = 0.f;
    // s = sum over row groups g of d_g^T (B_gg d_g + 2 sum_{h<g} B_gh d_h): the columns k of
    // group h feed row groups g >= h only, twice where g > h (compile-time after unrolling h)
#pragma unroll
    for (int h = 0; h < G; ++h) {
        const int k1 = L < 128 * h + 128 ? L : 128 * h + 128;
        for (int k = 128 * h; k < k1; k += 4) {
            float4 d4[PW];
#pragma unroll
            for (int q = 0; q < PW; ++q) d4[q] = *reinterpret_cast<const float4*>(dw + q * L + k);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                float4 b4[G];
#pragma unroll
                for (int g = h; g < G; ++g) {
                    const int i = 128 * g + 4 * lane;
                    b4[g] = i < L ? __ldg(reinterpret_cast<const float4*>(B + (size_t)(k + kk) * L + i))
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int q = 0; q < PW; ++q) {
                    const float dk = kk == 0 ? d4[q].x : kk == 1 ? d4[q].y : kk == 2 ? d4[q].z : d4[q].w;
#pragma unroll
                    for (int g = h; g < G; ++g) {
                        const float w = g == h ? dk : 2.f * dk;
                        acc[q][g][0] = fmaf(b4[g].x, w, acc[q][g][0]);
                        acc[q][g][1] = fmaf(b4[g].y, w, acc[q][g][1]);
                        acc[q][g][2] = fmaf(b4[g].z, w, acc[q][g][2]);
                        acc[q][g][3] = fmaf(b4[g].w, w, acc[q][g][3]);
                    }
                }
            }
        }
    }
    const bool failed = *status != 0;
#pragma unroll
    for (int q = 0; q < PW; ++q) {
        float s = 0.f;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int i = 128 * g + 4 * lane;
            if (i < L) {
                const float4 di = *reinterpret_cast<const float4*>(dw + q * L + i);
                s = fmaf(di.x, acc[q][g][0], s);
                s = fmaf(di.y, acc[q][g][1], s);
                s = fmaf(di.z, acc[q][g][2], s);
                s = fmaf(di.w, acc[q][g][3], s);
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const int64_t p = p0 + warp * PW + q;
        if (lane == 0 && p < P) score[p] = failed ? __int_as_float(0x7fc00000) : s;
    }
}

struct GrxLayout {
    int64_t P;
    int L, nblk1, nblk2, nst, nstl, ngroups, S;
    int64_t range;
    size_t off_part1, off_mu, off_part2, off_M, off_diag, off_B, off_status, total;
};

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

GrxLayout grx_layout(int64_t P, int L, int num_sms) {
    GrxLayout g{};
    g.P = P;
    g.L = L;
    g.nblk1 = (int)((P + GRX_CHUNK - 1) / GRX_CHUNK);
    g.nst = (L + 7) / 8;
    g.nstl = ntri(g.nst);
    g.ngroups = (g.nstl + GRX_THREADS - 1) / GRX_THREADS;
    // about two blocks per SM in all, and the range partials kept below 64 MB
    int64_t want = (2 * (int64_t)num_sms + g.ngroups - 1) / g.ngroups;
    const int64_t cap = (int64_t)(64u << 20) / ((int64_t)g.nstl * 64 * (int64_t)sizeof(float));
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    int64_t range = (P + want - 1) / want;
    if (range < 256) range = 256;
    g.range = range;
    g.nblk2 = (int)((P + range - 1) / range);
    const int Lp8 = g.nst * 8;
    g.S = Lp8 <= 256 ? 64 : Lp8 <= 512 ? 32 : 16;  // pixels staged per chunk (<= 64 KB)
    size_t o = 0;
    g.off_part1 = o; o = a256(o + sizeof(double) * (size_t)g.nblk1 * L);
    g.off_mu = o; o = a256(o + sizeof(float) * (size_t)L);
    g.off_part2 = o; o = a256(o + sizeof(float) * (size_t)g.nblk2 * g.nstl * 64);
    g.off_M = o; o = a256(o + sizeof(float) * (size_t)ntri(L));
    g.off_diag = o; o = a256(o + sizeof(double) * (size_t)L);
    g.off_B = o; o = a256(o + sizeof(float) * (size_t)L * L);
    g.off_status = o; o = a256(o + sizeof(int));
    g.total = o + 256;
    return g;
}

template <int M, int PW>
cudaError_t launch_score(const float* x, int64_t P, int L, const float* mu, const float* B, const int* status,
                         float* score, cudaStream_t s) {
    constexpr int PX = PW * (GRX_SCORE_THREADS / 32);
    const size_t smem = sizeof(float) * (size_t)PX * L;
    cudaError_t e = raise_smem_limit(grx_score_kernel<M, PW>);
    if (e != cudaSuccess) return e;
    const int64_t grid = (P + PX - 1) / PX;
    grx_score_kernel<M, PW><<<(unsigned)grid, GRX_SCORE_THREADS, smem, s>>>(x, P, L, mu, B, status, score);
    return cudaGetLastError();
}

template <int G, int PW>
cudaError_t launch_score4(const float* x, int64_t P, int L, const float* mu, const float* B, const int* status,
                          float* score, cudaStream_t s) {
    constexpr int PX = PW * (GRX_SCORE_THREADS / 32);
    const size_t smem = sizeof(float) * (size_t)PX * L;
    cudaError_t e = raise_smem_limit(grx_score4_kernel<G, PW>);
    if (e != cudaSuccess) return e;
    const int64_t grid = (P + PX - 1) / PX;
    grx_score4_kernel<G, PW><<<(unsigned)grid, GRX_SCORE_THREADS, smem, s>>>(x, P, L, mu, B, status, score);
    return cudaGetLastError();
}

}  // namespace

size_t global_rx_workspace_bytes(int64_t P, int L, int num_sms) {
    if (P < 1 || L < 1 || L > kGlobalRxMaxBands) return 0;
    return grx_layout(P, L, num_sms).total;
}

cudaError_t launch_global_rx(const float* x, int64_t P, int L, float loading, float* score, void* ws, size_t ws_bytes,
                             int num_sms, cudaStream_t s) {
    if (P == 0) return cudaSuccess;
    if (L < 1 || L > kGlobalRxMaxBands) return cudaErrorInvalidValue;
    const GrxLayout g = grx_layout(P, L, num_sms);
    if (ws_bytes < g.total) return cudaErrorInvalidValue;
    char* base = reinterpret_cast<char*>(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    double* part1 = reinterpret_cast<double*>(base + g.off_part1);
    float* mu = reinterpret_cast<float*>(base + g.off_mu);
    float* part2 = reinterpret_cast<float*>(base + g.off_part2);
    float* M = reinterpret_cast<float*>(base + g.off_M);
    double* diag = reinterpret_cast<double*>(base + g.off_diag);
    float* B = reinterpret_cast<float*>(base + g.off_B);
    int* status = reinterpret_cast<int*>(base + g.off_status);

    grx_colsum_kernel<<<g.nblk1, 256, 0, s>>>(x, P, L, part1);
    grx_mean_kernel<<<L, 256, 0, s>>>(part1, g.nblk1, L, P, mu);
    const size_t smem_g = sizeof(float) * (size_t)g.S * g.nst * 8;
    cudaError_t e = raise_smem_limit(grx_gram_kernel);
    if (e != cudaSuccess) return e;
    grx_gram_kernel<<<dim3(g.nblk2, g.ngroups), GRX_THREADS, smem_g, s>>>(x, P, L, g.range, mu, g.S, part2);
    const int nent = g.nstl * 64;
    grx_gram_reduce_kernel<<<(nent + 255) / 256, 256, 0, s>>>(part2, g.nblk2, L, P, M, diag);
    if (g.nstl <= GRX_THREADS) {
        grx_invert_regs_kernel<<<1, GRX_THREADS, 0, s>>>(M, diag, L, loading, B, status);
    } else {
        const int in_smem = ntri(L) + L + 4 <= GRX_INV_SMEM_FLOATS;
        const size_t smem_i =
            sizeof(float) * (in_smem ? (size_t)(((L + 3) & ~3) + ntri(L)) : (size_t)((L + 3) & ~3));
        e = raise_smem_limit(grx_invert_kernel);
        if (e != cudaSuccess) return e;
        grx_invert_kernel<<<1, GRX_THREADS, smem_i, s>>>(M, diag, L, loading, B, status, in_smem);
    }
    const int mrows = (L + 31) / 32;
    if (L % 4 == 0 && L > 32) {
        const int groups = (L + 127) / 128;
        if (groups <= 1) e = launch_score4<1, 8>(x, P, L, mu, B, status, score, s);
        else if (groups <= 2) e = launch_score4<2, 8>(x, P, L, mu, B, status, score, s);
        else if (groups <= 4) e = launch_score4<4, 4>(x, P, L, mu, B, status, score, s);
        else e = launch_score4<8, 2>(x, P, L, mu, B, status, score, s);
    } else if (mrows <= 1) e = launch_score<1, 8>(x, P, L, mu, B, status, score, s);
    else if (mrows <= 2) e = launch_score<2, 8>(x, P, L, mu, B, status, score, s);
    else if (mrows <= 4) e = launch_score<4, 8>(x, P, L, mu, B, status, score, s);
    else if (mrows <= 8) e = launch_score<8, 8>(x, P, L, mu, B, status, score, s);
    else if (mrows <= 16) e = launch_score<16, 4>(x, P, L, mu, B, status, score, s);
    else e = launch_score<32, 2>(x, P, L, mu, B, status, score, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace wdad
