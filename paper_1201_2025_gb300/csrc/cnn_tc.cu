// A9 — the screening network's 32 -> 32 channel 5x5 convolutions on the tensor cores
// (inference with bfloat16 weights): an implicit GEMM per output tile of 16 rows x 8 pixels,
// M = 128 pixels, N = 32 output channels, K = 25 taps x 32 input channels, as 50
// tcgen05.mma (kind::f16, bfloat16 x bfloat16 -> float32) of depth 16 into 32 columns of
// tensor memory.
//
// The input tile (20 x 12 pixels with the 2-pixel halo, zero outside the image) is staged in
// shared memory as bfloat16 in four planes of 8 channels; inside a plane a pixel is one
// 16-byte row, so 8 consecutive pixels of an input row form one 8 x 16-byte core matrix of
// the canonical K-major layout (no swizzle).  The A operand of tap (ky, kx) is then the same
// tile read at an offset: core matrices along M step one input row (SBO = 12 pixels x 16 B),
// along K one plane (LBO = plane size).  The weights of both layers are packed once per call
// into the matching B layout [tap][channel group][output channel][8 input channels].  Four
// warps read the accumulators back (lane = pixel, column = output channel), add the bias,
// apply ReLU and store float32 NHWC.  Activations are rounded to bfloat16 on staging; the
// sums are float32.  Every wait is bounded; a CTA that gives up sets *err, waits (bounded)
// for its own operations in flight, frees its tensor memory and stops.
#include <cuda_bf16.h>

#include "cnn.h"
#include "tc.cuh"

namespace wdad {
namespace cnn {

constexpr int TT_H = 16, TT_W = 8;                 // output tile
constexpr int IN_H = TT_H + 4, IN_W = TT_W + 4;    // input tile with the 5x5 halo
constexpr int PLANE_BYTES = IN_H * IN_W * 16 + 16; // one 8-channel plane (+16 B: planes start 4 banks apart)
constexpr int XS_BYTES = 4 * PLANE_BYTES;          // 32 channels
constexpr int W5_BYTES = 25 * 4 * 32 * 16;         // packed weights of one layer
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_COLS32 = 32;
constexpr uint32_t TC_SPIN = 1u << 26;

// packed[((tap * 4 + g) * 32 + co) * 8 + e] = w[(8 g + e) * 25 + tap][co]  (w: [ci][tap][co])
__global__ void pack_w5_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ packed) {
    const int n = 25 * 32 * 32;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int e = i & 7, co = (i >> 3) & 31, g = (i >> 8) & 3, tap = i >> 10;
        const int ci = 8 * g + e;
        packed[i] = __float2bfloat16_rn(w[((size_t)ci * 25 + tap) * 32 + co]);
    }
}

__global__ void __launch_bounds__(TC_THREADS) conv5_tc_kernel(const float* __restrict__ in, int B, int H, int W,
                                                              const __nv_bfloat16* __restrict__ wpk,
                                                              const float* __restrict__ bias, int relu,
                                                              float* __restrict__ out, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_ok;
    unsigned char* wsm = smem_raw;
    unsigned char* xs = smem_raw + W5_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // weights into shared memory
    for (int i = tid; i < W5_BYTES / 16; i += TC_THREADS)
        reinterpret_cast<uint4*>(wsm)[i] = reinterpret_cast<const uint4*>(wpk)[i];
    if (tid == 0) {
        tc::mbar_init(&s_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, TC_COLS32);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = tc::idesc_bf16_f32(128, 32);
    const int tiles_x = (W + TT_W - 1) / TT_W, tiles_y = (H + TT_H - 1) / TT_H;
    const int64_t ntiles = (int64_t)tiles_x * tiles_y * B;
    uint32_t phase = 0;
    bool alive = true;
    for (int64_t t = blockIdx.x; t < ntiles && alive; t += gridDim.x) {
        const int b = (int)(t / ((int64_t)tiles_x * tiles_y));
        const int r = (int)(t % ((int64_t)tiles_x * tiles_y));
        const int oy0 = (r / tiles_x) * TT_H, ox0 = (r % tiles_x) * TT_W;
        // stage the input tile as bfloat16 planes (thread: one pixel, one 8-channel group)
        for (int e = tid; e < IN_H * IN_W * 4; e += TC_THREADS) {
            const int g = e & 3, p = e >> 2;
            const int iy = p / IN_W, ix = p - iy * IN_W;
            const int y = oy0 - 2 + iy, x = ox0 - 2 + ix;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (y >= 0 && y < H && x >= 0 && x < W) {
                const float4* src = reinterpret_cast<const float4*>(in + (((size_t)b * H + y) * W + x) * 32 + 8 * g);
                const float4 f0 = __ldg(src), f1 = __ldg(src + 1);
                __nv_bfloat162 h0 = __floats2bfloat162_rn(f0.x, f0.y), h1 = __floats2bfloat162_rn(f0.z, f0.w);
                __nv_bfloat162 h2 = __floats2bfloat162_rn(f1.x, f1.y), h3 = __floats2bfloat162_rn(f1.z, f1.w);
                v.x = *reinterpret_cast<uint32_t*>(&h0);
                v.y = *reinterpret_cast<uint32_t*>(&h1);
                v.z = *reinterpret_cast<uint32_t*>(&h2);
                v.w = *reinterpret_cast<uint32_t*>(&h3);
            }
            *reinterpret_cast<uint4*>(xs + g * PLANE_BYTES + p * 16) = v;
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t xa = tc::smem_u32(xs), wa = tc::smem_u32(wsm);
            for (int tap = 0; tap < 25; ++tap) {
                const int ky = tap / 5, kx = tap - 5 * ky;
#pragma unroll
                for (int gp = 0; gp < 2; ++gp) {
                    const uint64_t ad = tc::smem_desc(xa + (uint32_t)(2 * gp * PLANE_BYTES + (ky * IN_W + kx) * 16),
                                                      PLANE_BYTES, IN_W * 16);
                    const uint64_t bd = tc::smem_desc(wa + (uint32_t)((tap * 4 + 2 * gp) * 512), 512, 128);
                    tc::mma_bf16(tmem, ad, bd, idesc, tap > 0 || gp > 0);
                }
            }
            tc::commit(&s_bar);
            s_ok = tc::mbar_wait_bounded(&s_bar, phase & 1u, TC_SPIN) ? 1 : 0;
        }
        __syncthreads();
        ++phase;
        if (!s_ok) {
            if (tid == 0) atomicExch(err, 1);
            alive = false;
            break;
        }
        tc::fence_after_sync();
        // epilogue: warp w reads tensor-memory lanes 32 w .. 32 w + 31 (pixel m = 8 oy + ox)
        {
            const int m = warp * 32 + lane;
            const int y = oy0 + (m >> 3), x = ox0 + (m & 7);
            float v[32];
            float h[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), h);
#pragma unroll
            for (int c = 0; c < 16; ++c) v[c] = h[c];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + 16u, h);
#pragma unroll
            for (int c = 0; c < 16; ++c) v[16 + c] = h[c];
            if (y < H && x < W) {
                float4* dst = reinterpret_cast<float4*>(out + (((size_t)b * H + y) * W + x) * 32);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float4 o;
                    o.x = v[4 * q] + __ldg(bias + 4 * q);
                    o.y = v[4 * q + 1] + __ldg(bias + 4 * q + 1);
                    o.z = v[4 * q + 2] + __ldg(bias + 4 * q + 2);
                    o.w = v[4 * q + 3] + __ldg(bias + 4 * q + 3);
                    if (relu) { o.x = fmaxf(o.x, 0.f); o.y = fmaxf(o.y, 0.f); o.z = fmaxf(o.z, 0.f); o.w = fmaxf(o.w, 0.f); }
                    dst[q] = o;
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();  // the tile buffer and the accumulator are free again
    }
    if (!alive && tid == 0) {
        // the commit that never arrived: give the tensor cores a last bounded chance to finish
        tc::mbar_wait_bounded(&s_bar, (phase - 1u) & 1u, TC_SPIN);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, TC_COLS32);
}

cudaError_t pack_w5(const float* w, __nv_bfloat16* packed, cudaStream_t s) {
    pack_w5_kernel<<<100, 256, 0, s>>>(w, packed);
    return cudaGetLastError();
}

cudaError_t conv5_tc(const float* in, int B, int H, int W, const __nv_bfloat16* wpk, const float* bias, int relu,
                     float* out, int* err, int num_sms, cudaStream_t s) {
    const size_t smem = (size_t)W5_BYTES + XS_BYTES + 1024;
    cudaError_t e = raise_smem_limit(conv5_tc_kernel);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv5_tc_kernel, TC_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t ntiles = (int64_t)((W + TT_W - 1) / TT_W) * ((H + TT_H - 1) / TT_H) * B;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    conv5_tc_kernel<<<(unsigned)grid, TC_THREADS, smem, s>>>(in, B, H, W, wpk, bias, relu, out, err);
    return cudaGetLastError();
}

}  // namespace cnn
}  // namespace wdad
