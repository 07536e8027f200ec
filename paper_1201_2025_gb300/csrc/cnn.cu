// A9 — learned screening: a 4-layer CNN on the DWT approximation matrix.
//
// Network (fixed): K -> 32 (5x5, ReLU) -> 32 (5x5, ReLU) -> 32 (5x5, ReLU) -> 1 (3x3),
// "same" zero padding, receptive field 15 x 15 (the (5,15) window).  Activations are
// NHWC float32.  Weights of a layer are stored [ci][tap][co] (tap = ky * k + kx): the
// forward kernel reads, for one input value, the contiguous row of its Cout weights.
// FP32 master weights are trained with Adam; the forward and the activation gradients
// use the BF16-rounded copy (BF16 weights, FP32 accumulation), the weight gradients
// update the masters (straight-through).
//
// Kernels: conv_fwd (input tile and weights staged in shared memory, one thread per
// output pixel and all output channels), conv_bwd_weight (one block per (ci, tap), fixed-
// order block reduction), bias gradients, transposed/flipped weights (the data gradient is
// a forward convolution of the output gradient), ReLU masks, MSE loss on the interior of
// each crop, Adam, crop sampling, the scene whitening of the input (the network sees
// z = M (x - mu), with mu and M = L^{-1}, C = L L^T, the mean and covariance of the scene's
// approximation matrix), the output layer of inference (conv3_to1), and for screening a
// radix threshold and an audit draw.  At inference, networks with BF16 weights run their
// two 32-channel layers on the tensor cores (cnn_tc.cu).
// Random numbers come from splitmix64 (Steele, Lea, Flood 2014) on (seed, counter).
#include <algorithm>
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "cnn.h"

namespace wdad {
namespace cnn {

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ float u01(uint64_t seed, uint64_t ctr) {
    return (float)(splitmix64(seed * 0x632BE59BD9B4E019ull + ctr) >> 40) * (1.0f / 16777216.0f);
}

constexpr int CT = 16;  // output tile side of conv_fwd

// out[b][y][x][co] = bias[co] + sum_ci sum_tap in[b][y+ky-p][x+kx-p][ci] * w[ci][tap][co]
// (zero padding), optional ReLU, optional input map z = M (x - mu) (norm = [mu (Cin), M (Cin x Cin)]).
template <int COUT>
__global__ void __launch_bounds__(CT * CT) conv_fwd_kernel(const float* __restrict__ in, int B, int H, int W, int Cin,
                                                           const float* __restrict__ w, const float* __restrict__ bias,
                                                           int k, int relu, const float* __restrict__ norm,
                                                           float* __restrict__ out) {
    extern __shared__ __align__(16) float sm[];
    const int p = k / 2, T = CT + k - 1, taps = k * k, XP = Cin + 1;
    float* ws = sm;                              // [Cin][taps][COUT]
    float* xs = sm + (size_t)Cin * taps * COUT;  // [T][T][Cin + 1]: pixel-major, channel pitch padded
    const int tiles_x = (W + CT - 1) / CT, tiles_y = (H + CT - 1) / CT;
    const int b = blockIdx.x / (tiles_x * tiles_y);
    const int t = blockIdx.x % (tiles_x * tiles_y);
    const int y0 = (t / tiles_x) * CT, x0 = (t % tiles_x) * CT;
    for (int i = threadIdx.x; i < Cin * taps * COUT; i += blockDim.x) ws[i] = w[i];
    if (norm) {  // first layer: z = M (x - mu) per pixel, Cin <= 8, zero padding in z
        for (int i = threadIdx.x; i < T * T; i += blockDim.x) {
            const int y = y0 + i / T - p, x = x0 + i % T - p;
            float xv[8];
            const bool inb = y >= 0 && y < H && x >= 0 && x < W;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                xv[j] = (inb && j < Cin) ? in[(((size_t)b * H + y) * W + x) * Cin + j] - norm[j] : 0.f;
            for (int ci = 0; ci < Cin; ++ci) {
                float z = 0.f;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j < Cin) z = fmaf(norm[Cin + ci * Cin + j], xv[j], z);
                xs[(size_t)i * XP + ci] = z;
            }
        }
    } else {
        // channel fastest: a warp reads whole NHWC pixel records (coalesced)
        for (int i = threadIdx.x; i < Cin * T * T; i += blockDim.x) {
            const int pix = i / Cin, ci = i - pix * Cin;
            const int y = y0 + pix / T - p, x = x0 + pix % T - p;
            xs[(size_t)pix * XP + ci] = (y >= 0 && y < H && x >= 0 && x < W) ? in[(((size_t)b * H + y) * W + x) * Cin + ci] : 0.f;
        }
    }
    __syncthreads();
    const int ty = threadIdx.x / CT, tx = threadIdx.x % CT;
    const int y = y0 + ty, x = x0 + tx;
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = bias ? bias[co] : 0.f;
    for (int ci = 0; ci < Cin; ++ci) {
        const float* xr = xs + ci;
        const float* wr = ws + (size_t)ci * taps * COUT;
        for (int ky = 0; ky < k; ++ky)
            for (int kx = 0; kx < k; ++kx) {
                const float a = xr[(size_t)((ty + ky) * T + tx + kx) * XP];
                const float* wt = wr + (ky * k + kx) * COUT;
#pragma unroll
                for (int co = 0; co < COUT; ++co) acc[co] = fmaf(a, wt[co], acc[co]);
            }
    }
    if (y < H && x < W) {
        float* o = out + (((size_t)b * H + y) * W + x) * COUT;
#pragma unroll
        for (int co = 0; co < COUT; ++co) o[co] = relu ? fmaxf(acc[co], 0.f) : acc[co];
    }
}

// dw[ci][tap][co] = sum over pixels of in[pix + tap offset][ci] * dz[pix][co]; one block per (ci, tap)
template <int COUT>
__global__ void __launch_bounds__(256) conv_bwd_weight_kernel(const float* __restrict__ in, const float* __restrict__ dz,
                                                              int B, int H, int W, int Cin, int k,
                                                              float* __restrict__ dw) {
    __shared__ float red[8][COUT];
    const int taps = k * k, p = k / 2;
    const int ci = blockIdx.x / taps, tap = blockIdx.x % taps;
    const int ky = tap / k, kx = tap % k;
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = 0.f;
    const int64_t n = (int64_t)B * H * W;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int x = (int)(i % W), y = (int)((i / W) % H);
        const int64_t b = i / ((int64_t)H * W);
        const int yy = y + ky - p, xx = x + kx - p;
        if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
        const float a = in[((b * H + yy) * W + xx) * Cin + ci];
        const float* d = dz + i * COUT;
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = fmaf(a, d[co], acc[co]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
        float v = acc[co];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][co] = v;
    }
    __syncthreads();
    for (int co = threadIdx.x; co < COUT; co += blockDim.x) {
        float s = 0.f;
        for (int w2 = 0; w2 < 8; ++w2) s += red[w2][co];
        dw[((size_t)ci * taps + tap) * COUT + co] = s;
    }
}

// The 32-output-channel weight gradient as chunked outer products: block (tap, chunk) stages
// 32 pixels at a time (the activations at the tap's offset and the output gradients) in shared
// memory and accumulates the Cin x 32 products of its chunk's pixels, thread (ci, four co);
// part[chunk][ci][tap][co] receives the chunk's sums, which grad_chunks_sum adds in chunk order
// (deterministic: the same sums on every run).
constexpr int WG_TILE = 32;
__global__ void __launch_bounds__(256) conv_bwd_weight32_kernel(const float* __restrict__ in,
                                                                const float* __restrict__ dz, int B, int H, int W,
                                                                int Cin, int k, int chunk_px,
                                                                float* __restrict__ part) {
    __shared__ float as[WG_TILE][33];
    __shared__ __align__(16) float ds[WG_TILE][32];
    const int taps = k * k, pd = k / 2;
    const int tap = blockIdx.x, chunk = blockIdx.y;
    const int ky = tap / k, kx = tap % k;
    const int ci = threadIdx.x >> 3, c4 = (threadIdx.x & 7) * 4;
    const int64_t n = (int64_t)B * H * W;
    const int64_t p0 = (int64_t)chunk * chunk_px, p1 = min(n, p0 + chunk_px);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t q0 = p0; q0 < p1; q0 += WG_TILE) {
        for (int idx = threadIdx.x; idx < WG_TILE * 32; idx += blockDim.x) {
            const int pp = idx >> 5, cc = idx & 31;
            const int64_t pix = q0 + pp;
            float d = 0.f, a = 0.f;
            if (pix < p1) {
                d = dz[pix * 32 + cc];
                if (cc < Cin) {
                    const int x = (int)(pix % W), y = (int)((pix / W) % H);
                    const int64_t b = pix / ((int64_t)H * W);
                    const int yy = y + ky - pd, xx = x + kx - pd;
                    if (yy >= 0 && yy < H && xx >= 0 && xx < W) a = in[((b * H + yy) * W + xx) * Cin + cc];
                }
            }
            ds[pp][cc] = d;
            as[pp][cc] = a;
        }
        __syncthreads();
        if (ci < Cin) {
#pragma unroll 8
            for (int pp = 0; pp < WG_TILE; ++pp) {
                const float a = as[pp][ci];
                const float4 d = *reinterpret_cast<const float4*>(&ds[pp][c4]);
                acc[0] = fmaf(a, d.x, acc[0]);
                acc[1] = fmaf(a, d.y, acc[1]);
                acc[2] = fmaf(a, d.z, acc[2]);
                acc[3] = fmaf(a, d.w, acc[3]);
            }
        }
        __syncthreads();
    }
    if (ci < Cin) {
        float* o = part + (size_t)chunk * Cin * taps * 32 + ((size_t)ci * taps + tap) * 32 + c4;
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = acc[j];
    }
}

// db partial sums: block `chunk` adds its pixels' output gradients, eight pixel groups per
// channel added in group order
__global__ void __launch_bounds__(256) bias_grad_chunk_kernel(const float* __restrict__ dz, int64_t n, int Cout,
                                                              int chunk_px, float* __restrict__ part) {
    __shared__ float red[8][32];
    const int co = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int64_t p0 = (int64_t)blockIdx.x * chunk_px, p1 = min(n, p0 + chunk_px);
    float acc = 0.f;
    if (co < Cout)
        for (int64_t i = p0 + grp; i < p1; i += 8) acc += dz[i * Cout + co];
    red[grp][co] = acc;
    __syncthreads();
    if (threadIdx.x < Cout) {
        float s = 0.f;
        for (int g = 0; g < 8; ++g) s += red[g][threadIdx.x];
        part[(size_t)blockIdx.x * Cout + threadIdx.x] = s;
    }
}

// out[o] = sum over the chunks in order of part[chunk][o]
__global__ void grad_chunks_sum_kernel(const float* __restrict__ part, int nchunk, int64_t per,
                                       float* __restrict__ out) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < per; o += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * per + o];
        out[o] = s;
    }
}

// wt[co][tap][ci] = w[ci][k*k-1-tap][co]  (the data gradient as a forward convolution)
__global__ void flip_transpose_kernel(const float* __restrict__ w, int Cin, int Cout, int k, float* __restrict__ wt) {
    const int taps = k * k;
    const int n = Cin * taps * Cout;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int co = i % Cout, tap = (i / Cout) % taps, ci = i / (Cout * taps);
        wt[((size_t)co * taps + (taps - 1 - tap)) * Cin + ci] = w[i];
    }
}

__global__ void relu_mask_kernel(float* __restrict__ d, const float* __restrict__ a, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!(a[i] > 0.f)) d[i] = 0.f;
}

// MSE over the interior (border `edge` excluded) of each crop; d = 2 (pred - t) / n, loss
__global__ void __launch_bounds__(1024) mse_kernel(const float* __restrict__ pred, const float* __restrict__ t, int B,
                                                   int H, int W, int edge, float* __restrict__ d,
                                                   float* __restrict__ loss) {
    __shared__ float red[32];
    const int ih = H - 2 * edge, iw = W - 2 * edge;
    const float inv = 1.0f / (float)((int64_t)B * ih * iw);
    float acc = 0.f;
    const int64_t n = (int64_t)B * H * W;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int x = (int)(i % W), y = (int)((i / W) % H);
        const bool in = y >= edge && y < H - edge && x >= edge && x < W - edge;
        const float r = pred[i] - t[i];
        d[i] = in ? 2.f * r * inv : 0.f;
        if (in) acc += r * r;
    }
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w2 = 0; w2 < 32; ++w2) s += red[w2];
        *loss = s * inv;
    }
}

// Adam (Kingma & Ba) on the FP32 masters; refresh the BF16-rounded forward copy
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float* __restrict__ wf, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2, int bf16) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        wf[i] = bf16 ? __bfloat162float(__float2bfloat16_rn(wi)) : wi;
    }
}

__global__ void round_copy_kernel(const float* __restrict__ w, float* __restrict__ wf, int n, int bf16) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        wf[i] = bf16 ? __bfloat162float(__float2bfloat16_rn(w[i])) : w[i];
}

// He-uniform initialisation from splitmix64
__global__ void init_kernel(float* __restrict__ w, int n, int fan_in, uint64_t seed, uint64_t ctr0) {
    const float a = sqrtf(6.f / (float)fan_in);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        w[i] = (2.f * u01(seed, ctr0 + (uint64_t)i) - 1.f) * a;
}

// B random crops (Hc x Wc) of the approximation matrix, mapped by z = M (x - mu), and their targets
// log(1 + score); crop positions from splitmix64(seed, step, b)
__global__ void crops_kernel(const float* __restrict__ approx, const float* __restrict__ score, int H, int W, int K,
                             const float* __restrict__ norm, int B, int Hc, int Wc, uint64_t seed, uint64_t step,
                             float* __restrict__ x, float* __restrict__ t) {
    const int64_t n = (int64_t)B * Hc * Wc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % Wc), r = (int)((i / Wc) % Hc);
        const int b = (int)(i / ((int64_t)Hc * Wc));
        const uint64_t base = step * 1024 + (uint64_t)b * 2;
        const int oy = (int)(u01(seed, base) * (float)(H - Hc + 1)) % (H - Hc + 1);
        const int ox = (int)(u01(seed, base + 1) * (float)(W - Wc + 1)) % (W - Wc + 1);
        const size_t q = (size_t)(oy + r) * W + (ox + c);
        for (int k = 0; k < K; ++k) {
            float z = 0.f;
            for (int j = 0; j < K; ++j) z = fmaf(norm[K + k * K + j], approx[q * K + j] - norm[j], z);
            x[i * K + k] = z;
        }
        t[i] = log1pf(fmaxf(score[q], 0.f));
    }
}

// ---------------------------------------------------------------- scene whitening
// Pass 1: per block, FP64 sums of d = x - x_0 and of d d^T (lower triangle) over a fixed
// contiguous pixel range; thread, warp (butterfly) and block sums in a fixed order, so the
// result does not depend on the GPU.  One partial row of NQ doubles per block.
template <int K>
__global__ void __launch_bounds__(256) scene_moments_kernel(const float* __restrict__ x, int64_t P,
                                                            double* __restrict__ part) {
    constexpr int NQ = K + K * (K + 1) / 2;
    __shared__ double red[8][NQ];
    const int64_t chunk = (P + WHITEN_BLOCKS - 1) / WHITEN_BLOCKS;
    const int64_t p0 = blockIdx.x * chunk, p1 = p0 + chunk < P ? p0 + chunk : P;
    float x0[K];
#pragma unroll
    for (int j = 0; j < K; ++j) x0[j] = x[j];
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
        double d[K];
#pragma unroll
        for (int j = 0; j < K; ++j) d[j] = (double)x[i * K + j] - (double)x0[j];
        int q = K;
#pragma unroll
        for (int a = 0; a < K; ++a) {
            acc[a] += d[a];
#pragma unroll
            for (int c = 0; c <= a; ++c) acc[q++] += d[a] * d[c];
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        for (int o = 16; o >= 1; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) red[warp][q] = acc[q];
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
        part[(size_t)blockIdx.x * NQ + threadIdx.x] = s;
    }
}

// Pass 2 (one block): sum the partials in block order, mean and population covariance, the
// Cholesky factor with the pivot floor 1e-12 trace / K (1 when the trace is 0), and
// M = L^{-1}; writes norm = [mu (K), M (K x K, row-major)].
__global__ void scene_whiten_finalize_kernel(const float* __restrict__ x, int64_t P, int K,
                                             const double* __restrict__ part, float* __restrict__ norm) {
    __shared__ double S[8 + 36];
    __shared__ double C[64], Lf[64], M[64];
    const int NQ = K + K * (K + 1) / 2;
    if (threadIdx.x < NQ) {
        double s = 0.0;
        for (int b = 0; b < WHITEN_BLOCKS; ++b) s += part[(size_t)b * NQ + threadIdx.x];
        S[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double invP = 1.0 / (double)P;
    double m1[8];
    for (int a = 0; a < K; ++a) m1[a] = S[a] * invP;
    int q = K;
    double tr = 0.0;
    for (int a = 0; a < K; ++a)
        for (int c = 0; c <= a; ++c) {
            const double v = S[q++] * invP - m1[a] * m1[c];
            C[a * K + c] = C[c * K + a] = v;
            if (a == c) tr += v;
        }
    const double floor = tr > 0.0 ? 1e-12 * tr / (double)K : 1.0;
    for (int i = 0; i < 64; ++i) Lf[i] = 0.0;
    for (int j = 0; j < K; ++j) {
        double d = C[j * K + j];
        for (int k = 0; k < j; ++k) d -= Lf[j * K + k] * Lf[j * K + k];
        if (!(d > floor)) d = floor;
        Lf[j * K + j] = sqrt(d);
        for (int i = j + 1; i < K; ++i) {
            double v = C[i * K + j];
            for (int k = 0; k < j; ++k) v -= Lf[i * K + k] * Lf[j * K + k];
            Lf[i * K + j] = v / Lf[j * K + j];
        }
    }
    for (int c = 0; c < K; ++c)
        for (int i = 0; i < K; ++i) {
            double v = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= Lf[i * K + k] * M[k * K + c];
            M[i * K + c] = v / Lf[i * K + i];
        }
    for (int a = 0; a < K; ++a) norm[a] = (float)((double)x[a] + m1[a]);
    for (int i = 0; i < K * K; ++i) norm[K + i] = (float)M[i];
}

// order-preserving float -> uint32 key
__device__ __forceinline__ uint32_t fkey(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// 256-bin histogram of key byte (key >> shift) & 0xFF among the keys whose higher bytes equal
// prefix: per-block counts in shared memory, then one global add per non-empty bin
__global__ void __launch_bounds__(256) hist_kernel(const float* __restrict__ v, int64_t n, uint32_t prefix, int shift,
                                                   uint32_t mask_hi, unsigned int* __restrict__ hist) {
    __shared__ unsigned int sh[256];
    sh[threadIdx.x] = 0u;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t kk = fkey(v[i]);
        if ((kk & mask_hi) == prefix) atomicAdd(&sh[(kk >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    const unsigned int c = sh[threadIdx.x];
    if (c) atomicAdd(&hist[threadIdx.x], c);
}

// selection: key >= thr (top fraction) or an audit draw below audit_frac; compacted list
__global__ void select_kernel(const float* __restrict__ v, int64_t n, uint32_t thr, float audit_frac, uint64_t seed,
                              uint8_t* __restrict__ sel, int64_t* __restrict__ list, unsigned long long* __restrict__ cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint8_t s = 0;
        if (fkey(v[i]) >= thr) s = 1;
        else if (u01(seed ^ 0xA5A5A5A5ull, (uint64_t)i) < audit_frac) s = 2;
        if (sel) sel[i] = s;
        if (s) list[atomicAdd(cnt, 1ull)] = i;
    }
}

__global__ void fill_kernel(float* __restrict__ v, int64_t n, float val) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = val;
}

// Output layer of inference (32 -> 1, 3x3, no ReLU): one warp per output pixel, lane = input
// channel, so each neighbouring 32-channel record is one coalesced 128-byte load; the lanes'
// products are summed over the taps and then across the warp (butterfly).
__global__ void __launch_bounds__(256) conv3_to1_kernel(const float* __restrict__ in, int B, int H, int W,
                                                        const float* __restrict__ w, const float* __restrict__ bias,
                                                        float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    float wl[9];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) wl[tap] = __ldg(w + lane * 9 + tap);
    const float b0 = __ldg(bias);
    const int64_t n = (int64_t)B * H * W;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t HW = (int64_t)H * W;
    for (int64_t i = warp; i < n; i += nwarps) {
        // one 64-bit division for the image; the rest in 32 bits (H * W < 2^31)
        const int64_t b = B == 1 ? 0 : i / HW;
        const int r = (int)(i - b * HW);
        const int y = r / W, x = r - y * W;
        float acc = 0.f;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                acc = fmaf(__ldg(in + ((b * H + yy) * W + xx) * 32 + lane), wl[tap], acc);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) out[i] = acc + b0;
    }
}

// ---------------------------------------------------------------- host side
static const int kK[4] = {5, 5, 5, 3};

void layer_dims(int K, int l, int* cin, int* cout, int* k) {
    *cin = (l == 0) ? K : 32;
    *cout = (l == 3) ? 1 : 32;
    *k = kK[l];
}

void param_layout(int K, size_t woff[4], size_t boff[4], size_t* total) {
    size_t o = 0;
    for (int l = 0; l < 4; ++l) {
        int ci, co, k;
        layer_dims(K, l, &ci, &co, &k);
        woff[l] = o;
        o += (size_t)ci * k * k * co;
        boff[l] = o;
        o += co;
    }
    *total = o;
}

static inline int grid_for(int64_t n, int threads, int cap = 4096) {
    int64_t g = (n + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

cudaError_t conv_fwd(const float* in, int B, int H, int W, int Cin, const float* w, const float* bias, int Cout, int k,
                     int relu, const float* norm, float* out, cudaStream_t s) {
    const size_t smem = sizeof(float) * ((size_t)Cin * k * k * Cout + (size_t)(Cin + 1) * (CT + k - 1) * (CT + k - 1));
    const int tiles = ((W + CT - 1) / CT) * ((H + CT - 1) / CT) * B;
    cudaError_t e;
    if (Cout == 32) {
        e = raise_smem_limit(conv_fwd_kernel<32>);
        if (e != cudaSuccess) return e;
        conv_fwd_kernel<32><<<tiles, CT * CT, smem, s>>>(in, B, H, W, Cin, w, bias, k, relu, norm, out);
    } else if (Cout == 4) {
        e = raise_smem_limit(conv_fwd_kernel<4>);
        if (e != cudaSuccess) return e;
        conv_fwd_kernel<4><<<tiles, CT * CT, smem, s>>>(in, B, H, W, Cin, w, bias, k, relu, norm, out);
    } else if (Cout == 1) {
        e = raise_smem_limit(conv_fwd_kernel<1>);
        if (e != cudaSuccess) return e;
        conv_fwd_kernel<1><<<tiles, CT * CT, smem, s>>>(in, B, H, W, Cin, w, bias, k, relu, norm, out);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// pixels per gradient chunk: a multiple of 32, at least 256, at most GRAD_MAX_CHUNKS chunks
static int grad_chunk_px(int64_t n) {
    int64_t c = (n + GRAD_MAX_CHUNKS - 1) / GRAD_MAX_CHUNKS;
    c = std::max<int64_t>(256, (c + 31) / 32 * 32);
    return (int)c;
}

static cudaError_t conv_bwd_weight(const Net& net, const float* in, const float* dz, int B, int H, int W, int Cin,
                                   int Cout, int k, float* dw, cudaStream_t s) {
    if (Cout == 32 && Cin <= 32 && k <= 5) {
        const int64_t n = (int64_t)B * H * W;
        const int chunk_px = grad_chunk_px(n);
        const int nchunk = (int)((n + chunk_px - 1) / chunk_px);
        conv_bwd_weight32_kernel<<<dim3(k * k, nchunk), 256, 0, s>>>(in, dz, B, H, W, Cin, k, chunk_px, net.gpart);
        const int64_t per = (int64_t)Cin * k * k * 32;
        grad_chunks_sum_kernel<<<grid_for(per, 256), 256, 0, s>>>(net.gpart, nchunk, per, dw);
        return cudaGetLastError();
    }
    const int blocks = Cin * k * k;
    if (Cout == 32) conv_bwd_weight_kernel<32><<<blocks, 256, 0, s>>>(in, dz, B, H, W, Cin, k, dw);
    else if (Cout == 1) conv_bwd_weight_kernel<1><<<blocks, 256, 0, s>>>(in, dz, B, H, W, Cin, k, dw);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

static cudaError_t bias_grad(const Net& net, const float* dz, int64_t n, int Cout, float* db, cudaStream_t s) {
    const int chunk_px = grad_chunk_px(n);
    const int nchunk = (int)((n + chunk_px - 1) / chunk_px);
    bias_grad_chunk_kernel<<<nchunk, 256, 0, s>>>(dz, n, Cout, chunk_px, net.gpart);
    grad_chunks_sum_kernel<<<1, 32, 0, s>>>(net.gpart, nchunk, Cout, db);
    return cudaGetLastError();
}

// Forward of the whole net on x [B][H][W][K] (already normalised unless norm != null);
// activations a[0..2] (32 ch) and the prediction out [B][H][W].
cudaError_t net_forward(const Net& n, const float* x, int B, int H, int W, const float* norm, float* a0, float* a1,
                        float* a2, float* out, cudaStream_t s, bool tc, int num_sms) {
    const float* wf = n.wf;
    cudaError_t e = conv_fwd(x, B, H, W, n.K, wf + n.woff[0], wf + n.boff[0], 32, 5, 1, norm, a0, s);
    if (tc) {
        __nv_bfloat16* p1 = n.wpk;
        __nv_bfloat16* p2 = n.wpk + 25 * 32 * 32;
        if (e == cudaSuccess) e = pack_w5(wf + n.woff[1], p1, s);
        if (e == cudaSuccess) e = pack_w5(wf + n.woff[2], p2, s);
        if (e == cudaSuccess) e = conv5_tc(a0, B, H, W, p1, wf + n.boff[1], 1, a1, n.tcerr, num_sms, s);
        if (e == cudaSuccess) e = conv5_tc(a1, B, H, W, p2, wf + n.boff[2], 1, a2, n.tcerr, num_sms, s);
        if (e == cudaSuccess) {
            conv3_to1_kernel<<<grid_for((int64_t)B * H * W * 32, 256), 256, 0, s>>>(a2, B, H, W, wf + n.woff[3],
                                                                                   wf + n.boff[3], out);
            e = cudaGetLastError();
        }
        return e;
    } else {
        if (e == cudaSuccess) e = conv_fwd(a0, B, H, W, 32, wf + n.woff[1], wf + n.boff[1], 32, 5, 1, nullptr, a1, s);
        if (e == cudaSuccess) e = conv_fwd(a1, B, H, W, 32, wf + n.woff[2], wf + n.boff[2], 32, 5, 1, nullptr, a2, s);
    }
    if (e == cudaSuccess) e = conv_fwd(a2, B, H, W, 32, wf + n.woff[3], wf + n.boff[3], 1, 3, 0, nullptr, out, s);
    return e;
}

// Gradients of the interior MSE with respect to every parameter (into n.grad); loss -> n.loss
cudaError_t net_grad(Net& n, const float* x, const float* t, int B, int H, int W, cudaStream_t s) {
    const int64_t px = (int64_t)B * H * W;
    float* a0 = n.act;
    float* a1 = a0 + px * 32;
    float* a2 = a1 + px * 32;
    float* out = a2 + px * 32;
    float* d0 = out + px;  // 32-channel gradient buffers
    float* d1 = d0 + px * 32;
    float* dout = d1 + px * 32;
    cudaError_t e = net_forward(n, x, B, H, W, nullptr, a0, a1, a2, out, s);
    if (e != cudaSuccess) return e;
    mse_kernel<<<1, 1024, 0, s>>>(out, t, B, H, W, 7, dout, n.loss);
    // layer 4 (32 -> 1, 3x3)
    e = conv_bwd_weight(n, a2, dout, B, H, W, 32, 1, 3, n.grad + n.woff[3], s);
    if (e != cudaSuccess) return e;
    if (e == cudaSuccess) e = bias_grad(n, dout, px, 1, n.grad + n.boff[3], s);
    if (e != cudaSuccess) return e;
    flip_transpose_kernel<<<64, 256, 0, s>>>(n.wf + n.woff[3], 32, 1, 3, n.wt);
    e = conv_fwd(dout, B, H, W, 1, n.wt, nullptr, 32, 3, 0, nullptr, d0, s);
    if (e != cudaSuccess) return e;
    relu_mask_kernel<<<grid_for(px * 32, 256), 256, 0, s>>>(d0, a2, px * 32);
    // layers 3, 2 (32 -> 32, 5x5)
    const float* ins[3] = {a0, a1, a2};
    float* dcur = d0;
    float* dnext = d1;
    for (int l = 2; l >= 1; --l) {
        e = conv_bwd_weight(n, ins[l - 1], dcur, B, H, W, 32, 32, 5, n.grad + n.woff[l], s);
        if (e != cudaSuccess) return e;
        if (e == cudaSuccess) e = bias_grad(n, dcur, px, 32, n.grad + n.boff[l], s);
        if (e != cudaSuccess) return e;
        flip_transpose_kernel<<<256, 256, 0, s>>>(n.wf + n.woff[l], 32, 32, 5, n.wt);
        e = conv_fwd(dcur, B, H, W, 32, n.wt, nullptr, 32, 5, 0, nullptr, dnext, s);
        if (e != cudaSuccess) return e;
        relu_mask_kernel<<<grid_for(px * 32, 256), 256, 0, s>>>(dnext, ins[l - 1], px * 32);
        float* tmp = dcur;
        dcur = dnext;
        dnext = tmp;
    }
    // layer 1 (K -> 32, 5x5) on the normalised input
    e = conv_bwd_weight(n, x, dcur, B, H, W, n.K, 32, 5, n.grad + n.woff[0], s);
    if (e != cudaSuccess) return e;
    if (e == cudaSuccess) e = bias_grad(n, dcur, px, 32, n.grad + n.boff[0], s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t net_adam(Net& n, float lr, cudaStream_t s) {
    n.step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)n.step), c2 = 1.f - powf(b2, (float)n.step);
    adam_kernel<<<grid_for((int64_t)n.nparam, 256), 256, 0, s>>>(n.w, n.m, n.v, n.grad, n.wf, (int)n.nparam, lr, b1,
                                                                 b2, 1e-8f, c1, c2, n.bf16);
    return cudaGetLastError();
}

cudaError_t net_init(Net& n, uint64_t seed, cudaStream_t s) {
    uint64_t ctr = 0;
    for (int l = 0; l < 4; ++l) {
        int ci, co, k;
        layer_dims(n.K, l, &ci, &co, &k);
        const int nw = ci * k * k * co;
        init_kernel<<<grid_for(nw, 256), 256, 0, s>>>(n.w + n.woff[l], nw, ci * k * k, seed, ctr);
        ctr += (uint64_t)nw;
        cudaMemsetAsync(n.w + n.boff[l], 0, sizeof(float) * co, s);
    }
    cudaMemsetAsync(n.m, 0, sizeof(float) * n.nparam, s);
    cudaMemsetAsync(n.v, 0, sizeof(float) * n.nparam, s);
    round_copy_kernel<<<grid_for((int64_t)n.nparam, 256), 256, 0, s>>>(n.w, n.wf, (int)n.nparam, n.bf16);
    return cudaGetLastError();
}

cudaError_t net_refresh_forward_copy(Net& n, cudaStream_t s) {
    round_copy_kernel<<<grid_for((int64_t)n.nparam, 256), 256, 0, s>>>(n.w, n.wf, (int)n.nparam, n.bf16);
    return cudaGetLastError();
}

cudaError_t scene_whitening(const float* x, int64_t P, int K, double* part, float* norm, cudaStream_t s) {
    if (P < 1 || K < 1 || K > 8) return cudaErrorInvalidValue;
    switch (K) {
        case 1: scene_moments_kernel<1><<<WHITEN_BLOCKS, 256, 0, s>>>(x, P, part); break;
        case 2: scene_moments_kernel<2><<<WHITEN_BLOCKS, 256, 0, s>>>(x, P, part); break;
        case 3: scene_moments_kernel<3><<<WHITEN_BLOCKS, 256, 0, s>>>(x, P, part); break;
        case 4: scene_moments_kernel<4><<<WHITEN_BLOCKS, 256, 0, s>>>(x, P, part); break;
        case 5: scene_moments_kernel<5><<<WHITEN_BLOCKS, 256, 0, s>>>(x, P, part); break;
        case 6: scene_moments_kernel<6><<<WHITEN_BLOCKS, 256, 0, s>>>(x, P, part); break;
        case 7: scene_moments_kernel<7><<<WHITEN_BLOCKS, 256, 0, s>>>(x, P, part); break;
        default: scene_moments_kernel<8><<<WHITEN_BLOCKS, 256, 0, s>>>(x, P, part); break;
    }
    scene_whiten_finalize_kernel<<<1, 64, 0, s>>>(x, P, K, part, norm);
    return cudaGetLastError();
}

cudaError_t sample_crops(const Net& n, const float* approx, const float* score, int H, int W, int B, int Hc, int Wc,
                         uint64_t seed, uint64_t step, float* x, float* t, cudaStream_t s) {
    const int64_t px = (int64_t)B * Hc * Wc;
    crops_kernel<<<grid_for(px, 256), 256, 0, s>>>(approx, score, H, W, n.K, n.norm, B, Hc, Wc, seed, step, x, t);
    return cudaGetLastError();
}

// k-th largest key (four 8-bit radix passes over 256-bin histograms); the key itself, so
// every value at or above the k-th largest is selected
cudaError_t top_threshold(const float* v, int64_t n, int64_t kth, unsigned int* hist, uint32_t* thr, cudaStream_t s) {
    uint32_t prefix = 0, mask = 0;
    int64_t need = kth;  // rank from the top, 1-based
    unsigned int h[256];
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned int) * 256, s);
        if (e != cudaSuccess) return e;
        hist_kernel<<<grid_for(n, 256, 1024), 256, 0, s>>>(v, n, prefix, shift, mask, hist);
        e = cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        int bin = 255;
        for (; bin > 0; --bin) {
            if ((int64_t)h[bin] >= need) break;
            need -= h[bin];
        }
        prefix |= (uint32_t)bin << shift;
        mask |= 0xFFu << shift;
    }
    *thr = prefix;
    return cudaSuccess;
}

cudaError_t select_pixels(const float* v, int64_t n, uint32_t thr, float audit_frac, uint64_t seed, uint8_t* sel,
                          int64_t* list, unsigned long long* cnt, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    select_kernel<<<grid_for(n, 256), 256, 0, s>>>(v, n, thr, audit_frac, seed, sel, list, cnt);
    return cudaGetLastError();
}

__global__ void scatter_kernel(const float* __restrict__ src, const int64_t* __restrict__ list, int64_t n,
                               float* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[list[i]] = src[list[i]];
}

cudaError_t scatter_list(const float* src, const int64_t* list, int64_t n, float* dst, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, list, n, dst);
    return cudaGetLastError();
}

cudaError_t fill(float* v, int64_t n, float val, cudaStream_t s) {
    fill_kernel<<<grid_for(n, 256), 256, 0, s>>>(v, n, val);
    return cudaGetLastError();
}

}  // namespace cnn
}  // namespace wdad
