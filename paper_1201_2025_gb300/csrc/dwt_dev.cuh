// Device code of the band-axis DWT (A1): pixel-group loop and warp butterfly.
#pragma once
#include "internal.h"

namespace wdad {

// Pixels per warp step: at most 8, at most 32/KP (one butterfly), and fewer for long
// spectra so that the staged chunks stay in registers.
__host__ __device__ constexpr int px_per_step(int nch, int kp) {
    int px = 32 / kp < 8 ? 32 / kp : 8;
    const int cap = 16 / nch < 1 ? 1 : 16 / nch;
    return px < cap ? px : cap;
}

// Reduce-scatter of 32 per-lane values: afterwards lane l holds sum over lanes of v[l].
__device__ __forceinline__ float butterfly32(float (&v)[32], int lane) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int j = 0; j < off; ++j) {
            const float send = upper ? v[j] : v[j + off];
            const float keep = upper ? v[j + off] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0];
}

// Reduce-scatter of 8 per-lane values over the 32 lanes: afterwards lanes l, l^8, l^16 and
// l^24 hold the sum over all lanes of v[l & 7].  Folds over lane bits 4 and 3, then the
// butterfly over bits 2, 1, 0: the summation tree butterfly32 builds, so the sums are
// bit-identical to it for the same per-lane inputs.
__device__ __forceinline__ float butterfly8x4(float (&v)[8], int lane) {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], 16);
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], 8);
#pragma unroll
    for (int off = 4; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int j = 0; j < off; ++j) {
            const float send = upper ? v[j] : v[j + off];
            const float keep = upper ? v[j + off] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0];
}

// DWT of npx pixel spectra staged in shared memory (xs: pixel p at xs + p L, L % 4 == 0,
// K <= 4): warp w takes pixels 2w, 2w + 1, then every 2 nwarps-th pair; lane slice a of the
// DWT matrix in registers (zero beyond L and K).  Per-lane sums in dwt_groups' (chunk,
// element) order and butterfly8x4's lane tree give coefficients bit-identical to
// dwt_apply_kernel's.
template <int NCH>
__device__ __forceinline__ void dwt_staged_pairs(const float* __restrict__ xs, int npx, int L,
                                                 const float (&a)[NCH][4][4], int K, float* __restrict__ out,
                                                 int warp, int nwarps) {
    const int lane = threadIdx.x & 31;
    const int LV = L / 4;
    for (int p0 = 2 * warp; p0 < npx; p0 += 2 * nwarps) {
        float v[8];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < NCH; ++i) {
                const int c = lane + 32 * i;
                float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
                if (p0 + p < npx && c < LV) t = reinterpret_cast<const float4*>(xs + (size_t)(p0 + p) * L)[c];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    s[k] = fmaf(t.x, a[i][k][0], s[k]);
                    s[k] = fmaf(t.y, a[i][k][1], s[k]);
                    s[k] = fmaf(t.z, a[i][k][2], s[k]);
                    s[k] = fmaf(t.w, a[i][k][3], s[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) v[p * 4 + k] = s[k];
        }
        const float r = butterfly8x4(v, lane);
        const int t = lane & 7, p = t >> 2, k = t & 3;
        if (lane < 8 && k < K && p0 + p < npx) out[(size_t)(p0 + p) * K + k] = r;
    }
}

// VEC = 4: 16-byte chunks (L % 4 == 0); VEC = 1: 4-byte elements.
// NCH = chunks per lane (NCH * 32 * VEC >= L); KP = K padded to a power of two <= 8.
// Pixel groups [g_begin, g_end) of one cube, group g taken by warp (g - g_begin) % nwarps.
template <int VEC, int NCH, int KP>
__device__ __forceinline__ void dwt_groups(const float* __restrict__ cube, int64_t P, int L,
                                           const float* __restrict__ A, int K, float* __restrict__ out,
                                           int64_t g_begin, int64_t g_end, int64_t warp, int64_t nwarps) {
    constexpr int PX = px_per_step(NCH, KP);
    const int lane = threadIdx.x & 31;
    const int LV = L / VEC;

    float a[NCH][KP][VEC];
#pragma unroll
    for (int i = 0; i < NCH; ++i) {
        const int c = lane + 32 * i;
#pragma unroll
        for (int k = 0; k < KP; ++k)
#pragma unroll
            for (int e = 0; e < VEC; ++e)
                a[i][k][e] = (c < LV && k < K) ? __ldg(A + (size_t)k * L + c * VEC + e) : 0.0f;
    }

    for (int64_t g = g_begin + warp; g < g_end; g += nwarps) {
        const int64_t p0 = g * PX;
        float x[PX][NCH][VEC];
#pragma unroll
        for (int p = 0; p < PX; ++p)
#pragma unroll
            for (int i = 0; i < NCH; ++i) {
                const int c = lane + 32 * i;
                const bool ok = (p0 + p < P) && (c < LV);
                if constexpr (VEC == 4) {
                    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (ok) t = __ldcs(reinterpret_cast<const float4*>(cube + (p0 + p) * L) + c);
                    x[p][i][0] = t.x; x[p][i][1] = t.y; x[p][i][2] = t.z; x[p][i][3] = t.w;
                } else {
                    x[p][i][0] = ok ? __ldcs(cube + (p0 + p) * L + c) : 0.0f;
                }
            }
        float v[32];
#pragma unroll
        for (int t = PX * KP; t < 32; ++t) v[t] = 0.0f;
#pragma unroll
        for (int p = 0; p < PX; ++p)
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                float s = 0.0f;
#pragma unroll
                for (int i = 0; i < NCH; ++i)
#pragma unroll
                    for (int e = 0; e < VEC; ++e) s = fmaf(x[p][i][e], a[i][k][e], s);
                v[p * KP + k] = s;
            }
        const float r = butterfly32(v, lane);
        const int p = lane / KP, k = lane % KP;
        if (k < K && p < PX && p0 + p < P) out[(p0 + p) * K + k] = r;
    }
}

// VEC = 4: 16-byte chunks (L % 4 == 0); VEC = 1: 4-byte elements.
// NCH = chunks per lane (NCH * 32 * VEC >= L); KP = K padded to a power of two <= 8.
template <int VEC, int NCH, int KP>
__global__ void __launch_bounds__(256) dwt_apply_kernel(const float* __restrict__ cube, int64_t P, int L,
                                                        const float* __restrict__ A, int K,
                                                        float* __restrict__ out) {
    constexpr int PX = px_per_step(NCH, KP);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    dwt_groups<VEC, NCH, KP>(cube, P, L, A, K, out, 0, (P + PX - 1) / PX, warp, nwarps);
}

}  // namespace wdad
