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

// Reduce-scatter of 16 per-lane values over the 32 lanes: afterwards lanes l and l ^ 16 both
// hold the sum over all lanes of v[l & 15].  The summation tree (lane pairs over bit 4, then
// bits 3, 2, 1, 0, each addition own + partner) is the one butterfly32 builds for its value
// indices, so the two give bit-identical sums for the same per-lane inputs.
__device__ __forceinline__ float butterfly16x2(float (&v)[16], int lane) {
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], 16);
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
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

// Variant of dwt_groups for the persistent batch kernel (16-byte chunks, K <= 4, 4 pixels per
// warp step): the DWT matrix comes from shared memory, A_s[k * NCH*128 + c] (zero for c >= L
// and k >= K), instead of registers, which keeps the kernel within 64 registers a thread.  The
// per-lane sums take the same (chunk, element) order and butterfly16x2 builds the same lane
// tree as dwt_groups' butterfly32, so the coefficients are bit-identical to dwt_apply_kernel's.
// Groups are 4-pixel groups here.
template <int NCH>
__device__ __forceinline__ void dwt_groups_sA(const float* __restrict__ cube, int64_t P, int L,
                                              const float* __restrict__ A_s, int K, float* __restrict__ out,
                                              int64_t g_begin, int64_t g_end, int64_t warp, int64_t nwarps) {
    constexpr int PX = 4, KP = 4, LS = NCH * 128;
    const int lane = threadIdx.x & 31;
    const int LV = L / 4;
    for (int64_t g = g_begin + warp; g < g_end; g += nwarps) {
        const int64_t p0 = g * PX;
        float x[PX][NCH][4];
#pragma unroll
        for (int p = 0; p < PX; ++p)
#pragma unroll
            for (int i = 0; i < NCH; ++i) {
                const int c = lane + 32 * i;
                float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
                if ((p0 + p < P) && (c < LV)) t = __ldcs(reinterpret_cast<const float4*>(cube + (p0 + p) * L) + c);
                x[p][i][0] = t.x; x[p][i][1] = t.y; x[p][i][2] = t.z; x[p][i][3] = t.w;
            }
        float v[16];
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            float s[PX];
#pragma unroll
            for (int p = 0; p < PX; ++p) s[p] = 0.0f;
#pragma unroll
            for (int i = 0; i < NCH; ++i) {
                const float4 a4 = *reinterpret_cast<const float4*>(A_s + k * LS + (lane + 32 * i) * 4);
#pragma unroll
                for (int p = 0; p < PX; ++p) {
                    s[p] = fmaf(x[p][i][0], a4.x, s[p]);
                    s[p] = fmaf(x[p][i][1], a4.y, s[p]);
                    s[p] = fmaf(x[p][i][2], a4.z, s[p]);
                    s[p] = fmaf(x[p][i][3], a4.w, s[p]);
                }
            }
#pragma unroll
            for (int p = 0; p < PX; ++p) v[p * KP + k] = s[p];
        }
        const float r = butterfly16x2(v, lane);
        const int t = lane & 15, p = t / KP, k = t % KP;
        if (lane < 16 && k < K && p0 + p < P) out[(p0 + p) * K + k] = r;
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
