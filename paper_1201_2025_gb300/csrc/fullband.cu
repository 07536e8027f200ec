// A3-A5 on the full-band cube (dim D > 8, e.g. L = 224): one CTA per pixel,
// persistent over the pixel list.
//
// Statistics (Sec. 2.1 / 2.2): the background annulus and inner square samples are
// gathered from the cube (reflect-101 borders), their means computed, and the
// centred Gram  sum (x - mu)(x - mu)^T  accumulated into a symmetric matrix stored
// as 4x4 tiles of its lower triangle ("tile-packed").
//   LRX / DWRX (Eq. 1, 5): C_o + delta I, delta = loading * trace(C_o) / D, blocked
//     Cholesky on the tiles bordered by the two right-hand sides r - mu_o and
//     mu_i - mu_o (so it also yields L^-1 d), score = ||L^-1 d||^2.  With fewer
//     background samples than bands (N < D) the same scores come from the N x N sample
//     Gram through the Woodbury identity, so the factorisation runs at dimension N.
//   DWEST (Eq. 2-4): C_diff = C_i - C_o; Householder tridiagonalisation; the
//     eigenvalues above tau = dwest_tau * max|lambda| by Sturm-count bisection (a
//     warp evaluates 32 points per step); their eigenvectors by inverse iteration on
//     the tridiagonal matrix (partial pivoting), re-orthogonalised inside clusters;
//     back-transformation through the stored reflectors, one warp per vector; each
//     vector's largest-|.| entry made positive; score |sum_k v_k^T m_diff|
//     (dwest_mode 0) or ||V^T m_diff|| (mode 1).
// T = float (the FP32 path, matrix in shared memory) or double (FP64 path, matrix in
// the per-CTA slab of the workspace).
#include <float.h>

#include "internal.h"
#include "tc.cuh"

namespace wdad {
namespace {

constexpr int FB_THREADS = 512;
constexpr int FB_WARPS = FB_THREADS / 32;

template <typename T> struct Num;
template <> struct Num<float> {
    static constexpr float eps = 1.1920929e-7f;
    static constexpr int bisect_steps = 6;  // 32-point sections: 6 x 5 = 30 bits
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
};
template <> struct Num<double> {
    static constexpr double eps = 2.220446049250313e-16;
    static constexpr int bisect_steps = 12;  // 60 bits
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
};

// ---- tile-packed symmetric storage: tile (I, K), I >= K, holds rows 4I.., cols 4K..;
// entry e = 4 (a % 4) + (b % 4) of tile u = I(I+1)/2 + K sits at A[e * ntl + u] (entries
// of neighbouring tiles are adjacent, so threads walking tiles hit distinct banks).
__host__ __device__ __forceinline__ int ntiles_of(int nt) { return nt * (nt + 1) / 2; }
__device__ __forceinline__ int tile_idx(int I, int K) { return (I * (I + 1)) / 2 + K; }
template <typename T>
__device__ __forceinline__ T& el(T* A, int ntl, int a, int b) {  // requires a >= b
    return A[(((a & 3) << 2) + (b & 3)) * ntl + tile_idx(a >> 2, b >> 2)];
}
template <typename T>
__device__ __forceinline__ void tile_load(const T* A, int ntl, int u, T (&t)[16]) {
#pragma unroll
    for (int e = 0; e < 16; ++e) t[e] = A[e * ntl + u];
}
template <typename T>
__device__ __forceinline__ void tile_store(T* A, int ntl, int u, const T (&t)[16]) {
#pragma unroll
    for (int e = 0; e < 16; ++e) A[e * ntl + u] = t[e];
}
// linear index u of a lower-triangular tile grid -> (row, col), u = row(row+1)/2 + col
__device__ __forceinline__ void tri_rc(int u, int& r, int& c) {
    r = (int)((sqrtf(8.f * (float)u + 1.f) - 1.f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= u) ++r;
    while (r * (r + 1) / 2 > u) --r;
    c = u - r * (r + 1) / 2;
}

// four consecutive values from a 16-byte aligned shared-memory address
__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&o)[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

// ---- window sample offsets in row-major order (background = outer square minus inner)
__device__ __forceinline__ void bg_offset(int s, int ro, int ri, int& dy, int& dx) {
    const int wo = 2 * ro + 1, wi = 2 * ri + 1, side = ro - ri;
    const int top = side * wo;
    if (s < top) { dy = -ro + s / wo; dx = -ro + s % wo; return; }
    s -= top;
    const int band = wi * (wo - wi);
    if (s < band) {
        const int row = s / (wo - wi), c = s % (wo - wi);
        dy = -ri + row;
        dx = (c < side) ? -ro + c : ri + 1 + (c - side);
        return;
    }
    s -= band;
    dy = ri + 1 + s / wo;
    dx = -ro + s % wo;
}
__device__ __forceinline__ void in_offset(int s, int ri, int& dy, int& dx) {
    const int wi = 2 * ri + 1;
    dy = -ri + s / wi;
    dx = -ri + s % wi;
}

template <typename T>
__device__ T block_sum(T v, T* red) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T s = T(0);
#pragma unroll
    for (int w = 0; w < FB_WARPS; ++w) s += red[w];
    __syncthreads();
    return s;
}
template <typename T>
__device__ T block_max(T v, T* red) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T s = red[0];
#pragma unroll
    for (int w = 1; w < FB_WARPS; ++w) s = max(s, red[w]);
    __syncthreads();
    return s;
}

// ---- shared-memory layout
template <typename T>
struct Smem {
    T* A;     // tile-packed matrix (shared or global)
    T* xs;    // sample chunk [S][Dp]
    T* mu_o;  // [Dp]
    T* mu_i;  // [Dp]
    T* r1;    // [Dp] right-hand side 1 (r - mu_o), then its solution
    T* r2;    // [Dp] right-hand side 2 (mu_i - mu_o), then its solution
    T* v;     // [Dp] Householder vector / scratch
    T* p;     // [Dp]
    T* dd;    // [Dp] tridiagonal diagonal
    T* ee;    // [Dp] tridiagonal off-diagonal
    T* lam;   // [mcap] selected eigenvalues
    T* res;   // [mcap * 2] per-vector sign*projection, projection
    T* red;   // [FB_WARPS]
    T* pan;   // Cholesky panel buffer [Dp + NB + 2][PP]
    int* flag;
};

struct Geo {
    int D, Dp, nt, ntl, S, mcap;
    int N, Np;         // background samples (outer^2 - inner^2), padded to 4
    bool wood;         // LRX / DWRX through the N x N sample Gram (Woodbury), N < D
    bool a_in_smem;
    bool tc;           // mixed precision (BF16 window Gram, condition gate, FP64 re-solve)
    bool tcg;          // window Gram on the tensor cores (D <= 256): tensor memory and chunk buffers
    int pieces;        // BF16 pieces per sample value: 1 (mixed precision) or 3 (FP32-accurate split)
    bool pan_in_tc;    // Cholesky panel buffer inside the (then idle) tensor-core chunk buffers
    bool pan_in_smem;  // else in shared memory after the vectors, else in the slab
};

__host__ __device__ inline int fb_chunk(int elem_size) { return elem_size == 4 ? 32 : 8; }

template <typename T>
__host__ __device__ inline size_t fb_smem_vectors_bytes(int Dp, int S, int mcap) {
    return sizeof(T) * ((size_t)S * Dp + 8 * (size_t)Dp + 3 * (size_t)mcap + FB_WARPS) + 16;
}
constexpr size_t kTcBufBytes = 2 * 256 * 64 * 2;  // two BF16 chunk buffers (TC_MB x TC_KC)

// ---- statistics ---------------------------------------------------------------
// pixel index of sample s of a list (kind 0 = background, 1 = inner) around (py, px)
__device__ __forceinline__ int sample_pixel(int s, int kind, int H, int W, int py, int px, int ro, int ri) {
    int dy, dx;
    if (kind == 0) bg_offset(s, ro, ri, dy, dx); else in_offset(s, ri, dy, dx);
    return reflect101(py + dy, H) * W + reflect101(px + dx, W);
}

// mean over a sample list (kind 0 = background, 1 = inner) into out[0..Dp).  Thread t takes
// the band quad t % Q (Q = Dp / 4) of the samples t / Q, t / Q + G, ... (G groups, G <= S so
// that the partial sums fit the sample-chunk buffer `part`), eight 16-byte loads in flight; the
// samples' pixel indices come from a shared-memory list filled 256 at a time, and the G partial
// sums of a band are added in group order.  Ends with a barrier.
constexpr int kMeanChunk = 256;
template <typename T>
__device__ void sample_mean(const float* __restrict__ x, int H, int W, const Geo& g, int py, int px, int kind,
                            int n, int ro, int ri, T* out, T* part) {
    __shared__ int s_q[kMeanChunk];
    const int D = g.D, Dp = g.Dp, Q = Dp / 4;
    const int G = max(1, min(FB_THREADS / Q, g.S));
    const int grp = threadIdx.x / Q, c = threadIdx.x - grp * Q;
    const bool active = grp < G;
    const bool vec = (D & 3) == 0;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    auto load4 = [&](int q, float (&v)[4]) {
        const float* src = x + (size_t)q * D + 4 * c;
        if (vec) {
            const float4 t = __ldg(reinterpret_cast<const float4*>(src));
            v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = 4 * c + e < D ? __ldg(src + e) : 0.f;
        }
    };
    __syncthreads();  // part and s_q may still be read by a previous call
    for (int s0 = 0; s0 < n; s0 += kMeanChunk) {
        const int m = min(kMeanChunk, n - s0);
        for (int i = threadIdx.x; i < m; i += FB_THREADS) s_q[i] = sample_pixel(s0 + i, kind, H, W, py, px, ro, ri);
        __syncthreads();
        if (active && 4 * c < D) {
            int i = grp;
            for (; i + 7 * G < m; i += 8 * G) {
                float v[8][4];
#pragma unroll
                for (int u = 0; u < 8; ++u) load4(s_q[i + u * G], v[u]);
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[e] += (T)v[u][e];
            }
            for (; i < m; i += G) {
                float v[4];
                load4(s_q[i], v);
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[e] += (T)v[e];
            }
        }
        __syncthreads();  // before s_q is refilled
    }
    if (active) {
#pragma unroll
        for (int e = 0; e < 4; ++e) part[grp * Dp + 4 * c + e] = acc[e];
    }
    __syncthreads();
    for (int b = threadIdx.x; b < Dp; b += FB_THREADS) {
        T sum = T(0);
        for (int gi = 0; gi < G; ++gi) sum += part[gi * Dp + b];
        out[b] = b < D ? sum / (T)n : T(0);
    }
    __syncthreads();
}

// A += sum over samples of (sc (x - mu)) (sc (x - mu))^T, tile by tile, S samples per chunk
template <typename T>
__device__ void gram_accumulate(const float* __restrict__ x, int H, int W, const Geo& g, int py, int px, int kind,
                                int n, int ro, int ri, const T* mu, T sc, T* A, T* xs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ntl = g.ntl;
    for (int s0 = 0; s0 < n; s0 += g.S) {
        __syncthreads();
        for (int ss = warp; ss < g.S; ss += FB_WARPS) {
            T* dst = xs + (size_t)ss * g.Dp;
            const int s = s0 + ss;
            if (s < n) {
                int dy, dx;
                if (kind == 0) bg_offset(s, ro, ri, dy, dx); else in_offset(s, ri, dy, dx);
                const float* src = x + ((size_t)reflect101(py + dy, H) * W + reflect101(px + dx, W)) * g.D;
                for (int b = lane; b < g.Dp; b += 32) dst[b] = b < g.D ? ((T)__ldg(src + b) - mu[b]) * sc : T(0);
            } else {
                for (int b = lane; b < g.Dp; b += 32) dst[b] = T(0);
            }
        }
        __syncthreads();
        const int ns = min(g.S, n - s0);
        for (int u = threadIdx.x; u < ntl; u += FB_THREADS) {
            int I, K;
            tri_rc(u, I, K);
            T acc[16];
            tile_load(A, ntl, u, acc);
            for (int s = 0; s < ns; ++s) {
                const T* row = xs + (size_t)s * g.Dp;
                T ai[4], bk[4];
                ld4(row + 4 * I, ai);
                ld4(row + 4 * K, bk);
#pragma unroll
                for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) acc[rr * 4 + cc] += ai[rr] * bk[cc];
            }
            tile_store(A, ntl, u, acc);
        }
    }
    __syncthreads();
}

// ---- Window Gram on the tensor cores.
// The centred, scaled samples of one chunk are stored transposed, [band][sample], as
// BF16 in the canonical K-major layout of 8 x 16-byte core matrices: element (b, s) at
// byte (b/8)*KC*16 + (s/8)*128 + (b%8)*16 + (s%8)*2.  G = X^T X then reads the same
// buffer as A (M = 128 bands per tile) and as B (N = all bands of the lower block
// triangle), K = 16 samples per MMA; FP32 sums accumulate in tensor memory: tile 0
// (bands 0..127 x 0..127) in columns [0, 128), tile 1 (bands 128..255 x 0..255) in
// columns [128, 384).  Two chunk buffers alternate; each is reused only after the
// tensor cores have signalled (commit -> mbarrier) that they finished reading it.
// Mixed precision stores one BF16 value per sample (64 samples per chunk).  The FP32 path
// splits each FP32 value v into three BF16 pieces, v1 = bf16(v), v2 = bf16(v - v1),
// v3 = bf16(v - v1 - v2) (each difference exact in FP32), which carry v's 24 significant
// bits, and accumulates the six products v1v1, v1v2, v2v1, v2v2, v1v3, v3v1 (each exact in
// FP32; the three dropped ones are below 2^-24 of v^2) over chunks of 16 samples, the three
// piece buffers of a chunk side by side.
constexpr int TC_KC = 64;          // chunk buffer capacity in samples (one piece)
constexpr int TC_MB = 256;         // band rows held per chunk buffer (D <= 256)
constexpr uint32_t TC_COLS = 512;  // tensor-memory columns allocated per CTA
constexpr uint32_t TC_WAIT = 1u << 26;

struct TcState {
    __nv_bfloat16* buf[2];  // 2 x TC_MB x TC_KC
    uint64_t* bar;          // [2] mbarriers
    uint32_t tmem;          // tensor-memory base address
    uint32_t uses[2];       // completed-phase counters per buffer
    int* err;               // shared error word
};

// byte offset of (band b, sample s) in one piece of a chunk of kc samples
__device__ __forceinline__ uint32_t tc_off(int b, int s, int kc) {
    return (uint32_t)((b >> 3) * (kc * 16) + (s >> 3) * 128 + (b & 7) * 16 + (s & 7) * 2);
}

// two floats as packed BF16 (lo at the lower address)
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}
__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// A += scale * (X^T X) over the n samples of one list, X = x - mu (FP32 packed SoA A), with
// NP = 1 (BF16 samples) or 3 (three-piece split).  In the split the tensor memory is added
// into A every kSplitFlush chunks (64 samples), so each FP32 accumulation in the tensor cores
// runs over few terms and the long sum over the window is taken by FP32 adds that round to
// nearest.  Measured against the oracle (48 x 48 scenes, L = 224 at 7/21 and L = 128 at
// 5/15): the largest LRX/DWRX error is 0.033-0.038 u kappa flushing every chunk, 0.06-0.08
// every four chunks, 0.14-0.17 with one accumulation over the whole window, against
// 0.06-0.12 for the SIMT FP32 Gram; every four chunks costs 6.0 ms against 7.4 ms for the
// SIMT Gram on 64 x 64 x 224 at 7/21 (every chunk: 8.4 ms).
constexpr int kSplitFlush = 4;
template <int NP>
__device__ void gram_tc(const float* __restrict__ x, int H, int W, const Geo& g, int py, int px, int kind, int n,
                        int ro, int ri, const float* mu, float scale, float* A, TcState& st) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int MT = (g.Dp + 127) / 128;  // 1 or 2 band tiles
    constexpr int kc = NP == 1 ? TC_KC : 16;  // samples per chunk
    constexpr uint32_t piece_bytes = (uint32_t)(TC_MB * kc * 2);
    const int nchunk = (n + kc - 1) / kc;
    const int F = NP == 1 ? nchunk : kSplitFlush;  // chunks per accumulation in tensor memory
    const uint32_t id128 = tc::idesc_bf16_f32(128, 128), id256 = tc::idesc_bf16_f32(128, 256);
    __shared__ int s_q[2][TC_KC];  // pixel index of each sample of a chunk (by chunk parity)
    bool pend[2] = {false, false};  // MMAs committed on the buffer's barrier and not yet waited for
    auto wait_buf = [&](int b) {
        if (!pend[b]) return;
        if (!tc::mbar_wait_bounded(&st.bar[b], st.uses[b] & 1, TC_WAIT)) *st.err = 1;
        ++st.uses[b];
        pend[b] = false;
    };
    for (int c = 0; c < nchunk; ++c) {
        const int b = c & 1;
        wait_buf(b);  // the tensor cores must be done with this buffer (chunk c - 2)
        if ((int)threadIdx.x < kc && c * kc + (int)threadIdx.x < n)
            s_q[b][threadIdx.x] = sample_pixel(c * kc + threadIdx.x, kind, H, W, py, px, ro, ri);
        __syncthreads();
        if (*st.err) return;
        // fill: one task = 8 consecutive samples x 32 consecutive bands (lane = band)
        __nv_bfloat16* buf = st.buf[b];
        constexpr int ntask = (kc / 8) * (TC_MB / 32);
        for (int t = warp; t < ntask; t += FB_WARPS) {
            const int so = (t % (kc / 8)) * 8, bg = (t / (kc / 8)) * 32;
            const int band = bg + lane;
            const float m = band < g.D ? mu[band] : 0.f;
            float v1[8], v2[8], v3[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int s = c * kc + so + e;
                float val = 0.f;
                if (s < n && band < g.D) val = __ldg(x + (size_t)s_q[b][so + e] * g.D + band) - m;
                if constexpr (NP == 3) {
                    v1[e] = bf16_round(val);
                    const float r1 = val - v1[e];  // exact
                    v2[e] = bf16_round(r1);
                    v3[e] = r1 - v2[e];            // exact; rounded by pack_bf16
                } else {
                    v1[e] = val;
                }
            }
            char* dst = reinterpret_cast<char*>(buf) + tc_off(band, so, kc);
            *reinterpret_cast<uint4*>(dst) =
                make_uint4(pack_bf16(v1[0], v1[1]), pack_bf16(v1[2], v1[3]), pack_bf16(v1[4], v1[5]),
                           pack_bf16(v1[6], v1[7]));
            if constexpr (NP == 3) {
                *reinterpret_cast<uint4*>(dst + piece_bytes) =
                    make_uint4(pack_bf16(v2[0], v2[1]), pack_bf16(v2[2], v2[3]), pack_bf16(v2[4], v2[5]),
                               pack_bf16(v2[6], v2[7]));
                *reinterpret_cast<uint4*>(dst + 2 * piece_bytes) =
                    make_uint4(pack_bf16(v3[0], v3[1]), pack_bf16(v3[2], v3[3]), pack_bf16(v3[4], v3[5]),
                               pack_bf16(v3[6], v3[7]));
            }
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
            const uint32_t base = tc::smem_u32(buf);
            // piece pairs (A, B): v1v1 alone, or v1v1, v1v2, v2v1, v2v2, v1v3, v3v1
            constexpr int npairs = NP == 1 ? 1 : 6;
#pragma unroll
            for (int k = 0; k < kc / 16; ++k) {
                const uint32_t koff = (uint32_t)k * 256;  // two core matrices along K
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int q = 0; q < npairs; ++q) {
                        const uint32_t pa = q == 2 || q == 3 ? 1u : q == 5 ? 2u : 0u;
                        const uint32_t pb = q == 1 || q == 3 ? 1u : q == 4 ? 2u : 0u;
                        const uint64_t ad =
                            tc::smem_desc(base + pa * piece_bytes + (uint32_t)mt * 16 * (kc * 16) + koff, 128, kc * 16);
                        const uint64_t bd = tc::smem_desc(base + pb * piece_bytes + koff, 128, kc * 16);
                        tc::mma_bf16(st.tmem + (uint32_t)(mt * 128), ad, bd, mt == 0 ? id128 : id256,
                                     c % F != 0 || k > 0 || q > 0);
                    }
            }
            tc::commit(&st.bar[b]);
        }
        pend[b] = true;
        if ((c + 1) % F != 0 && c != nchunk - 1) continue;
        // add the tensor-memory sums into A: every warp, lanes of its quarter (warp % 4), a
        // quarter of the 16-column blocks (warp / 4); only the lower triangle is kept
        wait_buf(0);
        wait_buf(1);
        __syncthreads();
        if (*st.err) return;
        tc::fence_after_sync();
        const int lq = warp & 3, cq = warp >> 2;
        for (int mt = 0; mt < MT; ++mt) {
            const int r = mt * 128 + lq * 32 + lane;
            const int clast = mt * 128 + lq * 32 + 31;  // last column any row of this warp keeps
            for (int c0 = 16 * cq; c0 <= clast; c0 += 64) {
                float v[16];
                tc::tmem_ld16(st.tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(mt * 128 + c0), v);
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int col = c0 + e;
                    if (r < g.D && col <= r) el(A, g.ntl, r, col) += scale * v[e];
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
}

// Sample Gram of the background window for the Woodbury form of LRX / DWRX (N < D):
// G = Xt^T Xt (N x N, tile-packed with gw's geometry) and b_k = Xt^T d_k, Xt = sc (X - mu)
// with the N background samples as columns, accumulated over chunks of BC bands.  A chunk
// is staged band-major (xs[b * SP + s], SP = Np + 4): the tile products read four samples
// as one float4.  Staging: thread (bb, s0) loads band c0 + bb of samples s0, s0 + SL, ...
// (coalesced along the bands, eight loads in flight); the samples' pixel offsets are
// computed once into qoff.
template <typename T>
__device__ void gram_samples(const float* __restrict__ x, int H, int W, const Geo& g, const Geo& gw, int py, int px,
                             int ro, int ri, const T* mu, T sc, T* A, T* xs, const T* d1, const T* d2, T* b1, T* b2,
                             int* qoff) {
    const int SP = gw.Dp + 4;
    const int BC = max(4, min(64, (g.S * g.Dp / SP) & ~3));
    const int SL = FB_THREADS / BC;
    const int bb = threadIdx.x % BC, s0 = threadIdx.x / BC;
    for (int smp = threadIdx.x; smp < g.N; smp += FB_THREADS) {
        int dy, dx;
        bg_offset(smp, ro, ri, dy, dx);
        qoff[smp] = reflect101(py + dy, H) * W + reflect101(px + dx, W);
    }
    for (int c0 = 0; c0 < g.Dp; c0 += BC) {
        __syncthreads();
        if (s0 < SL) {
            const int band = c0 + bb;
            const bool inb = band < g.D;
            const T mub = inb ? mu[band] : T(0);
            for (int smp = s0; smp < gw.Dp; smp += 8 * SL) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int sm = smp + u * SL;
                    v[u] = (inb && sm < g.N) ? __ldg(x + (size_t)qoff[sm] * g.D + band) : 0.f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int sm = smp + u * SL;
                    if (sm < gw.Dp) xs[(size_t)bb * SP + sm] = (inb && sm < g.N) ? ((T)v[u] - mub) * sc : T(0);
                }
            }
        }
        __syncthreads();
        const int nbb = min(BC, g.Dp - c0);
        for (int u = threadIdx.x; u < gw.ntl; u += FB_THREADS) {
            int I, K;
            tri_rc(u, I, K);
            T acc[16];
            tile_load(A, gw.ntl, u, acc);
            for (int k = 0; k < nbb; ++k) {
                const T* row = xs + (size_t)k * SP;
                T ai[4], bk[4];
                ld4(row + 4 * I, ai);
                ld4(row + 4 * K, bk);
#pragma unroll
                for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) acc[rr * 4 + cc] += ai[rr] * bk[cc];
            }
            tile_store(A, gw.ntl, u, acc);
        }
        for (int t = threadIdx.x; t < 2 * gw.Dp; t += FB_THREADS) {
            const int smp = t % gw.Dp;
            const T* d = t < gw.Dp ? d1 : d2;
            T acc = T(0);
            for (int k = 0; k < nbb; ++k) acc += xs[(size_t)k * SP + smp] * d[c0 + k];
            (t < gw.Dp ? b1 : b2)[smp] += acc;
        }
    }
    __syncthreads();
}

template <typename T>
__device__ void mat_zero(T* A, const Geo& g) {
    const int n = ntiles_of(g.nt) * 16;
    for (int i = threadIdx.x; i < n; i += FB_THREADS) A[i] = T(0);
    __syncthreads();
}

template <typename T>
__device__ void mat_scale(T* A, const Geo& g, T s) {
    const int n = ntiles_of(g.nt) * 16;
    for (int i = threadIdx.x; i < n; i += FB_THREADS) A[i] *= s;
    __syncthreads();
}

// ---- blocked Cholesky of the tile-packed matrix, bordered by the two right-hand sides.
// Right-looking in steps of NB = 16 columns (4 tile columns; the per-panel critical paths
// of (1) and (2) grow with NB, and 16 beat 32 at every size measured):
//   (1) one warp factors the 16 x 16 diagonal block in registers (lane i holds row i; the
//       column of L each step needs comes by shuffles) and writes L_kk densely at the head
//       of the panel buffer, with 1 / L_jj in column NB;
//   (2) one thread per row below the block, and one for each right-hand side, solves
//       x = a L_kk^-T with the row in registers (L_kk read as shared-memory broadcasts) and
//       writes it to the panel buffer, rows ordered (row within tile, tile) so that the
//       float4 reads of neighbouring tiles in (3) fall on distinct banks;
//   (3) the trailing tiles take A_IK -= X_I X_K^T and the right-hand sides y -= x_b X^T,
//       reading X from the panel buffer.
// The right-hand sides behave as two extra rows appended below the matrix, so on return
// y1 = L^-1 r1 and y2 = L^-1 r2 and no separate solve is needed.  Pivots use rsqrt (1/L_jj
// directly).  Padding rows (D <= b < Dp) are identity.  Returns false, leaving *flag = 1, if
// a pivot is not above `floor`; L_jj is left on A's diagonal.
constexpr int NB = 16;
constexpr int PP = 20;  // panel pitch (16-byte aligned rows; 20 words apart, float4 reads of 8 rows hit distinct banks)
constexpr int LP = 17;  // pitch of the dense diagonal block at the head of the panel buffer

template <typename T>
__host__ __device__ inline size_t pan_bytes(int Dp) {
    return ((size_t)(Dp + NB + 2) * PP * sizeof(T) + 255) & ~(size_t)255;
}
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

template <typename T>
__device__ bool cholesky_bordered(T* A, const Geo& g, T floor, int* flag, T* y1, T* y2, T* pan) {
    const int ntl = g.ntl;
    if (threadIdx.x == 0) *flag = 0;
    for (int b = g.D + threadIdx.x; b < g.Dp; b += FB_THREADS) el(A, ntl, b, b) = T(1);
    __syncthreads();
    for (int c0 = 0; c0 < g.Dp; c0 += NB) {
        const int nb = min(NB, g.Dp - c0);  // a multiple of 4
        const int r0 = c0 + nb, nrows = g.Dp - r0, mI = nrows / 4;
        T* X = pan + NB * PP;              // trailing rows: row r0 + 4 i + rr at X[(rr mI + i) PP]
        T* Yr = X + (size_t)nrows * PP;    // the two right-hand sides
        // (1) diagonal block: warp 0, lane i holding row i in registers, the column of L each
        // step needs taken by shuffles
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            T a[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c)
                a[c] = (lane < nb && c <= lane) ? el(A, ntl, c0 + lane, c0 + c) : T(0);
            bool ok = true;
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                const T d = __shfl_sync(0xffffffffu, a[j], j);
                if (j < nb && ok) {  // warp-uniform
                    if (!(d > floor)) ok = false;
                }
                if (j < nb && ok) {
                    const T inv = rsqrt_t(d);
                    if (lane == j) { a[j] = d * inv; pan[j * LP + NB] = inv; }
                    else if (lane > j) a[j] *= inv;
                    const T lij = a[j];
#pragma unroll
                    for (int c = j + 1; c < NB; ++c) {
                        const T lcj = __shfl_sync(0xffffffffu, a[j], c);
                        if (lane >= c) a[c] -= lij * lcj;
                    }
                }
            }
            if (ok) {
#pragma unroll
                for (int c = 0; c < NB; ++c)
                    if (lane < nb && c <= lane) {
                        el(A, ntl, c0 + lane, c0 + c) = a[c];
                        pan[lane * LP + c] = a[c];
                    }
            } else if (lane == 0) {
                *flag = 1;
            }
        }
        __syncthreads();
        if (*flag) return false;
        // (2) panel rows and the two right-hand sides, one thread per row in registers
        for (int t = threadIdx.x; t < nrows + 2; t += FB_THREADS) {
            T x[NB];
            T* yv = t == nrows ? y1 : y2;
#pragma unroll
            for (int c = 0; c < NB; ++c)
                x[c] = c < nb ? (t < nrows ? el(A, ntl, r0 + t, c0 + c) : yv[c0 + c]) : T(0);
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                if (c < nb) {
                    T v = x[c];
#pragma unroll
                    for (int k = 0; k < c; ++k) v -= x[k] * pan[c * LP + k];
                    x[c] = v * pan[c * LP + NB];
                }
            }
            T* dst = t < nrows ? X + (size_t)((t & 3) * mI + (t >> 2)) * PP : Yr + (size_t)(t - nrows) * PP;
#pragma unroll
            for (int c = 0; c < NB; ++c)
                if (c < nb) {
                    dst[c] = x[c];
                    if (t >= nrows) yv[c0 + c] = x[c];
                }
        }
        __syncthreads();
        // (3) trailing tiles and right-hand sides
        const int T0 = r0 / 4;
        const int ntri = ntiles_of(mI);
        for (int u = threadIdx.x; u < ntri + 2 * mI; u += FB_THREADS) {
            if (u < ntri) {
                int i2, k2;
                tri_rc(u, i2, k2);
                const int uc = tile_idx(T0 + i2, T0 + k2);
                T acc[16];
                tile_load(A, ntl, uc, acc);
                for (int s4 = 0; s4 < nb; s4 += 4) {
                    T xi[4][4], xk[4][4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        ld4(X + (size_t)(r * mI + i2) * PP + s4, xi[r]);
                        ld4(X + (size_t)(r * mI + k2) * PP + s4, xk[r]);
                    }
#pragma unroll
                    for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) {
                            T v = acc[rr * 4 + cc];
#pragma unroll
                            for (int k = 0; k < 4; ++k) v -= xi[rr][k] * xk[cc][k];
                            acc[rr * 4 + cc] = v;
                        }
                }
                tile_store(A, ntl, uc, acc);
            } else {
                const int v0 = u - ntri, k2 = v0 % mI;
                T* yv = v0 < mI ? y1 : y2;
                const T* yr = Yr + (size_t)(v0 < mI ? 0 : 1) * PP;
                T acc[4];
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) acc[cc] = yv[4 * (T0 + k2) + cc];
                for (int s4 = 0; s4 < nb; s4 += 4) {
                    T yb[4], xk[4][4];
                    ld4(yr + s4, yb);
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) ld4(X + (size_t)(cc * mI + k2) * PP + s4, xk[cc]);
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc)
#pragma unroll
                        for (int k = 0; k < 4; ++k) acc[cc] -= yb[k] * xk[cc][k];
                }
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) yv[4 * (T0 + k2) + cc] = acc[cc];
            }
        }
        __syncthreads();
    }
    return true;
}

// ---- Householder tridiagonalisation (in place; reflector k stored in column k below
// the sub-diagonal, unit norm, H_k = I - 2 v v^T).  dd / ee receive the tridiagonal.
// v and p are absolute-index vectors of length Dp, zero outside the trailing block, so
// tile-level products need no masks.
template <typename T>
__device__ void tridiagonalise(T* A, const Geo& g, T* v, T* p, T* dd, T* ee, T* red) {
    const int D = g.D, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, ntl = g.ntl;
    for (int k = 0; k < D - 2; ++k) {
        T part = T(0);
        for (int b = threadIdx.x; b < g.Dp; b += FB_THREADS) {
            const T xb = (b > k && b < D) ? el(A, ntl, b, k) : T(0);
            v[b] = xb;
            if (b > k + 1) part += xb * xb;
        }
        const T rest = block_sum(part, red);
        const T x0 = v[k + 1];
        const bool reflect = rest > T(0);
        T alpha = x0;
        if (reflect) {
            const T nrm = Num<T>::sqrt_(x0 * x0 + rest);
            alpha = (x0 >= T(0)) ? -nrm : nrm;
            const T v0 = x0 - alpha;
            const T inv = T(1) / Num<T>::sqrt_(v0 * v0 + rest);
            if (threadIdx.x == 0) v[k + 1] = v0;
            __syncthreads();
            for (int b = k + 1 + threadIdx.x; b < D; b += FB_THREADS) v[b] *= inv;
            __syncthreads();
            // p = A v over the trailing block: one warp per tile row, lanes over tile columns
            const int T0 = (k + 1) >> 2;
            for (int I = T0 + warp; I < g.nt; I += FB_WARPS) {
                T s4[4] = {T(0), T(0), T(0), T(0)};
                for (int K = T0 + lane; K < g.nt; K += 32) {
                    const bool low = K <= I;
                    T t[16];
                    tile_load(A, ntl, low ? tile_idx(I, K) : tile_idx(K, I), t);
                    T vk[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) vk[c] = v[4 * K + c];
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) s4[r] += (low ? t[r * 4 + c] : t[c * 4 + r]) * vk[c];
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int o = 16; o >= 1; o >>= 1) s4[r] += __shfl_xor_sync(0xffffffffu, s4[r], o);
                if (lane < 4) {
                    const int row = 4 * I + lane;
                    p[row] = (row > k && row < D) ? s4[lane] : T(0);
                }
            }
            for (int b = threadIdx.x; b < 4 * T0; b += FB_THREADS) p[b] = T(0);
            __syncthreads();
            T kp = T(0);
            for (int b = k + 1 + threadIdx.x; b < D; b += FB_THREADS) kp += v[b] * p[b];
            const T K = block_sum(kp, red);
            for (int b = k + 1 + threadIdx.x; b < D; b += FB_THREADS) p[b] = T(2) * p[b] - T(2) * K * v[b];  // q
            __syncthreads();
            // rank-2 update of the trailing lower triangle: A -= v q^T + q v^T
            const int m = g.nt - T0;
            for (int u = threadIdx.x; u < ntiles_of(m); u += FB_THREADS) {
                int i2, k2;
                tri_rc(u, i2, k2);
                const int I = T0 + i2, Kt = T0 + k2;
                const int ut = tile_idx(I, Kt);
                T t[16];
                tile_load(A, ntl, ut, t);
                T va[4], qa[4], vb[4], qb[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    va[r] = v[4 * I + r]; qa[r] = p[4 * I + r];
                    vb[r] = v[4 * Kt + r]; qb[r] = p[4 * Kt + r];
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) t[r * 4 + c] -= va[r] * qb[c] + qa[r] * vb[c];
                tile_store(A, ntl, ut, t);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) { dd[k] = el(A, ntl, k, k); ee[k] = alpha; }
        for (int b = k + 1 + threadIdx.x; b < D; b += FB_THREADS) el(A, ntl, b, k) = reflect ? v[b] : T(0);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        dd[D - 2] = el(A, ntl, D - 2, D - 2);
        dd[D - 1] = el(A, ntl, D - 1, D - 1);
        ee[D - 2] = el(A, ntl, D - 1, D - 2);
        el(A, ntl, D - 1, D - 2) = T(0);  // no reflector for the last column
    }
    __syncthreads();
}

// reciprocal used by the Sturm recurrence
__device__ __forceinline__ float sturm_div(float a, float q) { return a * __frcp_rn(q); }
__device__ __forceinline__ double sturm_div(double a, double q) { return a / q; }

// number of eigenvalues of the tridiagonal (dd, ee) below x (Sturm sequence)
template <typename T>
__device__ int sturm_below(const T* dd, const T* ee, int n, T x, T pivmin) {
    int c = 0;
    T q = dd[0] - x;
    if (q < T(0)) ++c;
    for (int i = 1; i < n; ++i) {
        if (fabs(q) < pivmin) q = (q < T(0)) ? -pivmin : pivmin;
        q = (dd[i] - x) - sturm_div(ee[i - 1] * ee[i - 1], q);
        if (q < T(0)) ++c;
    }
    return c;
}

// j-th smallest eigenvalue (0-based) by warp-parallel 32-section of [lo, hi]
template <typename T>
__device__ T warp_bisect(const T* dd, const T* ee, int n, int j, T lo, T hi, T pivmin) {
    const int lane = threadIdx.x & 31;
    for (int it = 0; it < Num<T>::bisect_steps; ++it) {
        const T h = (hi - lo) / T(32);
        const T x = lo + h * T(lane + 1);  // lanes probe lo + h, ..., lo + 32 h = hi
        const int c = sturm_below(dd, ee, n, x, pivmin);
        // first probe with more than j eigenvalues below it bounds lambda_j from above
        const unsigned ballot = __ballot_sync(0xffffffffu, c > j);
        const int f = ballot ? __ffs(ballot) - 1 : 31;
        const T nlo = lo + h * T(f), nhi = lo + h * T(f + 1);
        lo = nlo;
        hi = nhi;
    }
    return T(0.5) * (lo + hi);
}

// Inverse iteration on (T - lambda I), one thread per eigenvalue; scratch arrays in
// [i][slot] layout so the threads of a warp touch adjacent words.  inv_factor builds
// the LU factors with partial pivoting (zero pivots replaced by `pert`), inv_solve
// overwrites y (a column of n) with (T - lambda I)^-1 y, normalised.
#define IX(i) ((size_t)(i) * nslot + slot)
template <typename T>
__device__ void inv_factor(const T* dd, const T* ee, int n, T lam, T pert, int slot, int nslot, T* Ld, T* Lu,
                           T* Lu2, T* Lf, int* piv) {
    T d_cur = dd[0] - lam, u_cur = (n > 1) ? ee[0] : T(0);
    T u2_prev_next = T(0);
    for (int i = 0; i < n - 1; ++i) {
        const T sub = ee[i];
        const T dnext = dd[i + 1] - lam;
        const T unext = (i + 1 < n - 1) ? ee[i + 1] : T(0);
        if (fabs(d_cur) >= fabs(sub)) {
            const T dn = (d_cur == T(0)) ? pert : d_cur;
            const T f = sub / dn;
            Ld[IX(i)] = dn; Lu[IX(i)] = u_cur; Lu2[IX(i)] = T(0); Lf[IX(i)] = f; piv[IX(i)] = 0;
            d_cur = dnext - f * u_cur;
            u_cur = unext;
        } else {
            const T f = d_cur / sub;
            Ld[IX(i)] = sub; Lu[IX(i)] = dnext; Lu2[IX(i)] = unext; Lf[IX(i)] = f; piv[IX(i)] = 1;
            d_cur = u_cur - f * dnext;
            u_cur = -f * unext;
        }
    }
    (void)u2_prev_next;
    Ld[IX(n - 1)] = (d_cur == T(0)) ? pert : d_cur;
    Lu[IX(n - 1)] = T(0);
    Lu2[IX(n - 1)] = T(0);
}

template <typename T>
__device__ void inv_solve(int n, int slot, int nslot, const T* Ld, const T* Lu, const T* Lu2, const T* Lf,
                          const int* piv, T* y) {
    // forward: apply the interchanges and multipliers
    T b_cur = y[0];
    for (int i = 0; i < n - 1; ++i) {
        const T b_next = y[i + 1];
        if (piv[IX(i)]) {
            y[i] = b_next;
            b_cur = b_cur - Lf[IX(i)] * b_next;
        } else {
            y[i] = b_cur;
            b_cur = b_next - Lf[IX(i)] * b_cur;
        }
    }
    y[n - 1] = b_cur;
    // backward
    T x1 = T(0), x2 = T(0), nrm = T(0);
    for (int i = n - 1; i >= 0; --i) {
        const T xi = (y[i] - Lu[IX(i)] * x1 - Lu2[IX(i)] * x2) / Ld[IX(i)];
        y[i] = xi;
        nrm += xi * xi;
        x2 = x1;
        x1 = xi;
    }
    const T inv = T(1) / Num<T>::sqrt_(nrm);
    for (int i = 0; i < n; ++i) y[i] *= inv;
}
#undef IX

// warp-level argmax |v| (lowest index on ties), sum of v * w
template <typename T>
__device__ void warp_sign_proj(const T* v, const T* w, int n, T& sgn, T& proj) {
    const int lane = threadIdx.x & 31;
    T best = T(-1), pr = T(0);
    int bi = 0x7fffffff;
    T bv = T(0);
    for (int i = lane; i < n; i += 32) {
        const T a = fabs(v[i]);
        if (a > best) { best = a; bi = i; bv = v[i]; }
        pr += v[i] * w[i];
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; bv = ov; }
        pr += __shfl_xor_sync(0xffffffffu, pr, o);
    }
    sgn = (bv >= T(0)) ? T(1) : T(-1);
    proj = pr;
}

// Scratch of one pixel's pipeline: shared-memory vectors (or slab vectors for the FP64
// re-solve) and slab arrays for the eigenvectors and the inverse-iteration factors.
template <typename T>
struct Scratch {
    T *Y, *Ld, *Lu, *Lu2, *Lf;
    int* piv;
};

template <typename T>
__device__ void carve(char* base, const Geo& g, Smem<T>& m, Scratch<T>& sc, bool a_here, char** end) {
    size_t off = 0;
    if (a_here) { m.A = reinterpret_cast<T*>(base); off += sizeof(T) * (size_t)g.ntl * 16; }
    T* v = reinterpret_cast<T*>(base + off);
    m.xs = v; v += (size_t)g.S * g.Dp;
    m.mu_o = v; v += g.Dp;
    m.mu_i = v; v += g.Dp;
    m.r1 = v; v += g.Dp;
    m.r2 = v; v += g.Dp;
    m.v = v; v += g.Dp;
    m.p = v; v += g.Dp;
    m.dd = v; v += g.Dp;
    m.ee = v; v += g.Dp;
    m.lam = v; v += g.mcap;
    m.res = v; v += 2 * g.mcap;
    m.red = v; v += FB_WARPS;
    char* e = reinterpret_cast<char*>(((uintptr_t)v + 255) & ~(uintptr_t)255);
    (void)sc;
    *end = e;
}

template <typename T>
__device__ void carve_scratch(char* base, const Geo& g, Scratch<T>& sc, char** end) {
    const size_t n = (size_t)g.mcap * g.Dp;
    T* t = reinterpret_cast<T*>(base);
    sc.Y = t; t += n;
    sc.Ld = t; t += n;
    sc.Lu = t; t += n;
    sc.Lu2 = t; t += n;
    sc.Lf = t; t += n;
    sc.piv = reinterpret_cast<int*>(t);
    *end = reinterpret_cast<char*>(((uintptr_t)(sc.piv + n) + 255) & ~(uintptr_t)255);
}

template <typename T>
__host__ __device__ size_t vec_bytes(const Geo& g) {
    return sizeof(T) * ((size_t)g.S * g.Dp + 8 * (size_t)g.Dp + 3 * (size_t)g.mcap + FB_WARPS) + 256;
}
template <typename T>
__host__ __device__ size_t scratch_bytes(const Geo& g) {
    return (sizeof(T) * 5 + sizeof(int)) * (size_t)g.mcap * g.Dp + 256;
}

// One pixel, the wanted detectors (bit d = detector d).  Returns, in mixed precision, the
// detectors whose estimated condition exceeds cond_gate (to be re-solved in FP64).
template <typename T>
__device__ unsigned process_pixel(const FullArgs& a, const Geo& g, Smem<T>& m, Scratch<T>& sc, TcState* st, int64_t pix,
                                  unsigned want, uint8_t& flag, int* sflag, int* s_m, T* s_bounds) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ro = a.outer / 2, ri = a.inner / 2;
    const int N = a.outer * a.outer - a.inner * a.inner, ni = a.inner * a.inner;
    const int D = g.D;
    const int py = (int)(pix / a.W), px = (int)(pix % a.W);
    const float fnan = __int_as_float(0x7fc00000);
    const bool gate = g.tc;  // mixed precision: estimate the conditioning
    unsigned redo = 0;
    m.flag = sflag;
    __syncthreads();
    sample_mean<T>(a.x, a.H, a.W, g, py, px, 0, N, ro, ri, m.mu_o, m.xs);
    sample_mean<T>(a.x, a.H, a.W, g, py, px, 1, ni, ro, ri, m.mu_i, m.xs);
    __syncthreads();
    if (want & 3u) {
        for (int b = threadIdx.x; b < g.Dp; b += FB_THREADS) {
            const T c = b < D ? (T)__ldg(a.x + pix * D + b) : T(0);
            m.r1[b] = b < D ? c - m.mu_o[b] : T(0);
            m.r2[b] = b < D ? m.mu_i[b] - m.mu_o[b] : T(0);
        }
        if (g.wood) {
            // Fewer samples than bands: C = Xt Xt^T (Xt = (X - mu_o) / sqrt(N), D x N) has rank
            // below D, and by the Woodbury identity
            //   d^T (C + delta I)^-1 d = (d^T d - |L^-1 Xt^T d|^2) / delta,  L L^T = Xt^T Xt + delta I,
            // so the factorisation runs at dimension N instead of D.  In mixed precision this
            // FP32 form replaces the BF16 Gram: it is both cheaper and more accurate here.
            Geo gw = g;
            gw.D = g.N;
            gw.Dp = g.Np;
            gw.nt = g.Np / 4;
            gw.ntl = ntiles_of(gw.nt);
            for (int b = threadIdx.x; b < gw.Dp; b += FB_THREADS) { m.v[b] = T(0); m.p[b] = T(0); }
            mat_zero(m.A, gw);
            gram_samples<T>(a.x, a.H, a.W, g, gw, py, px, ro, ri, m.mu_o, T(1) / Num<T>::sqrt_((T)N), m.A, m.xs,
                            m.r1, m.r2, m.v, m.p, reinterpret_cast<int*>(m.dd));
            T tr = T(0), dmax = T(0), d1 = T(0), d2 = T(0), fro = T(0);
            for (int b = threadIdx.x; b < N; b += FB_THREADS) {
                tr += el(m.A, gw.ntl, b, b);
                dmax = max(dmax, el(m.A, gw.ntl, b, b));
            }
            if (gate) {  // |G|_F^2: off-diagonal tiles stand for both triangles
                for (int u = threadIdx.x; u < gw.ntl; u += FB_THREADS) {
                    int I, K;
                    tri_rc(u, I, K);
                    T q = T(0);
#pragma unroll
                    for (int e = 0; e < 16; ++e) q += m.A[e * gw.ntl + u] * m.A[e * gw.ntl + u];
                    fro += I == K ? q : T(2) * q;
                }
                fro = block_sum(fro, m.red);
            }
            for (int b = threadIdx.x; b < D; b += FB_THREADS) { d1 += m.r1[b] * m.r1[b]; d2 += m.r2[b] * m.r2[b]; }
            tr = block_sum(tr, m.red);
            dmax = block_max(dmax, m.red);
            d1 = block_sum(d1, m.red);
            d2 = block_sum(d2, m.red);
            const T delta = (T)a.loading * tr / (T)D;
            for (int b = threadIdx.x; b < N; b += FB_THREADS) el(m.A, gw.ntl, b, b) += delta;
            __syncthreads();
            const bool ok = cholesky_bordered(m.A, gw, T(16) * Num<T>::eps * (dmax + delta), m.flag, m.v, m.p, m.pan);
            // kappa(C + delta I) bound: its smallest eigenvalue is delta exactly (C has rank below
            // D), its largest (that of G + delta I) at most |G|_F + delta
            if (ok && gate && !((Num<T>::sqrt_(fro) + delta) / delta <= (T)a.cond_gate)) redo |= want & 3u;
            if (!ok && gate) redo |= want & 3u;
            if (ok) {
                T q1 = T(0), q2 = T(0);
                for (int b = threadIdx.x; b < N; b += FB_THREADS) { q1 += m.v[b] * m.v[b]; q2 += m.p[b] * m.p[b]; }
                q1 = block_sum(q1, m.red);
                q2 = block_sum(q2, m.red);
                if (threadIdx.x == 0) {
                    if ((want & 1u) && a.out[0]) a.out[0][pix] = (float)((d1 - q1) / delta);
                    if ((want & 2u) && a.out[1]) a.out[1][pix] = (float)fabs((d2 - q2) / delta);
                }
            } else {
                flag |= 2;
                if (threadIdx.x == 0) {
                    if ((want & 1u) && a.out[0]) a.out[0][pix] = fnan;
                    if ((want & 2u) && a.out[1]) a.out[1][pix] = fnan;
                }
            }
        } else {
            mat_zero(m.A, g);
            if constexpr (sizeof(T) == 4) {
                if (g.tcg && g.pieces == 3) gram_tc<3>(a.x, a.H, a.W, g, py, px, 0, N, ro, ri, m.mu_o, 1.f / (float)N, m.A, *st);
                else if (g.tcg) gram_tc<1>(a.x, a.H, a.W, g, py, px, 0, N, ro, ri, m.mu_o, 1.f / (float)N, m.A, *st);
            }
            if (!g.tcg) {
                gram_accumulate<T>(a.x, a.H, a.W, g, py, px, 0, N, ro, ri, m.mu_o, T(1), m.A, m.xs);
                mat_scale(m.A, g, T(1) / (T)N);
            }
            T tr = T(0), dmax = T(0);
            for (int b = threadIdx.x; b < D; b += FB_THREADS) {
                tr += el(m.A, g.ntl, b, b);
                dmax = max(dmax, el(m.A, g.ntl, b, b));
            }
            tr = block_sum(tr, m.red);
            dmax = block_max(dmax, m.red);
            const T delta = (T)a.loading * tr / (T)D;
            for (int b = threadIdx.x; b < D; b += FB_THREADS) el(m.A, g.ntl, b, b) += delta;
            __syncthreads();
            bool ok = cholesky_bordered(m.A, g, T(16) * Num<T>::eps * (dmax + delta), m.flag, m.r1, m.r2, m.pan);
            if (ok && gate) {
                // kappa estimate from the factor's diagonal: (max L_ii / min L_ii)^2
                T lmax = T(0), lmin = T(3e38);
                for (int b = threadIdx.x; b < D; b += FB_THREADS) {
                    const T l = el(m.A, g.ntl, b, b);
                    lmax = max(lmax, l);
                    lmin = min(lmin, l);
                }
                lmax = block_max(lmax, m.red);
                lmin = -block_max(-lmin, m.red);
                const T kap = (lmax / lmin) * (lmax / lmin);
                if (!(kap <= (T)a.cond_gate)) redo |= want & 3u;
            }
            if (!ok && gate) redo |= want & 3u;
            if (ok) {
                T q1 = T(0), q2 = T(0);
                for (int b = threadIdx.x; b < D; b += FB_THREADS) { q1 += m.r1[b] * m.r1[b]; q2 += m.r2[b] * m.r2[b]; }
                q1 = block_sum(q1, m.red);
                q2 = block_sum(q2, m.red);
                if (threadIdx.x == 0) {
                    if ((want & 1u) && a.out[0]) a.out[0][pix] = (float)q1;
                    if ((want & 2u) && a.out[1]) a.out[1][pix] = (float)fabs(q2);
                }
            } else {
                flag |= 2;
                if (threadIdx.x == 0) {
                    if ((want & 1u) && a.out[0]) a.out[0][pix] = fnan;
                    if ((want & 2u) && a.out[1]) a.out[1][pix] = fnan;
                }
            }
        }
    }
    if (want & 4u) {
        // C_diff = C_i - C_o (Eq. 2)
        for (int b = threadIdx.x; b < g.Dp; b += FB_THREADS) m.r2[b] = b < D ? m.mu_i[b] - m.mu_o[b] : T(0);
        // the eigenproblem's Gram stays in the working precision in every mode: a BF16 Gram
        // perturbs C_diff by about 2^-9 of its norm, more than the distance of most
        // noise-level eigenvalues to the selection threshold, so it could not decide Eq. 4's
        // selection; in mixed precision FP32 decides it and FP64 takes only the pixels whose
        // selection FP32 cannot decide (the band below)
        mat_zero(m.A, g);
        gram_accumulate<T>(a.x, a.H, a.W, g, py, px, 0, N, ro, ri, m.mu_o, T(1), m.A, m.xs);
        mat_scale(m.A, g, T(-1) / (T)N);
        gram_accumulate<T>(a.x, a.H, a.W, g, py, px, 1, ni, ro, ri, m.mu_i, T(1) / Num<T>::sqrt_((T)ni), m.A, m.xs);
        tridiagonalise(m.A, g, m.v, m.p, m.dd, m.ee, m.red);
        // spectrum bounds (Gershgorin), extreme eigenvalues, threshold, count above it
        T glo, ghi;
        {
            T lo = T(3e38), hi = T(-3e38);
            for (int i = threadIdx.x; i < D; i += FB_THREADS) {
                const T r = (i > 0 ? fabs(m.ee[i - 1]) : T(0)) + (i < D - 1 ? fabs(m.ee[i]) : T(0));
                lo = min(lo, m.dd[i] - r);
                hi = max(hi, m.dd[i] + r);
            }
            glo = -block_max(-lo, m.red);
            ghi = block_max(hi, m.red);
        }
        const T tnorm = max(fabs(glo), fabs(ghi));
        const T pivmin = max(tnorm * Num<T>::eps * Num<T>::eps, T(1e-30));
        const T pad = tnorm * T(4) * Num<T>::eps + pivmin;
        if (warp == 0) {
            const T lmax = warp_bisect(m.dd, m.ee, D, D - 1, glo - pad, ghi + pad, pivmin);
            if (lane == 0) s_bounds[0] = lmax;
        } else if (warp == 1) {
            const T lmin = warp_bisect(m.dd, m.ee, D, 0, glo - pad, ghi + pad, pivmin);
            if (lane == 0) s_bounds[1] = lmin;
        }
        __syncthreads();
        const T maxabs = max(fabs(s_bounds[0]), fabs(s_bounds[1]));
        const T tau = (T)a.dwest_tau * maxabs;
        if (threadIdx.x == 0) {
            const int below = (maxabs > T(0)) ? sturm_below(m.dd, m.ee, D, tau, pivmin) : D;
            *s_m = D - below;
            if (gate && maxabs > T(0)) {
                // selection conditioning: an eigenvalue within max|lambda| / cond_gate of tau, the
                // band never narrower than 64 FP32 roundings of the spectrum's scale (2^-17
                // max|lambda|), a generous bound on what the FP32 Gram, the tridiagonalisation
                // and the Sturm counts can move an eigenvalue by
                const T band = max(maxabs / (T)a.cond_gate, maxabs * T(7.62939453125e-6));
                const int nb = sturm_below(m.dd, m.ee, D, tau + band, pivmin) -
                               sturm_below(m.dd, m.ee, D, tau - band, pivmin);
                if (nb > 0) *s_m = -1 - *s_m;  // mark for the FP64 re-solve
            }
        }
        __syncthreads();
        int msel = *s_m;
        if (msel < 0) { redo |= 4u; msel = -1 - msel; }
        if (msel > g.mcap) { msel = g.mcap; flag |= 8; }  // more than the slab holds: top mcap kept
        // selected eigenvalues lambda_{D-msel} .. lambda_{D-1}
        for (int s = warp; s < msel; s += FB_WARPS) {
            const T l = warp_bisect(m.dd, m.ee, D, D - msel + s, glo - pad, ghi + pad, pivmin);
            if (lane == 0) m.lam[s] = l;
        }
        __syncthreads();
        // eigenvectors of the tridiagonal matrix
        const T pert = max(tnorm * Num<T>::eps, pivmin);
        if (threadIdx.x < msel) {
            const int sl = threadIdx.x;
            T* y = sc.Y + (size_t)sl * g.Dp;
            inv_factor(m.dd, m.ee, D, m.lam[sl], pert, sl, g.mcap, sc.Ld, sc.Lu, sc.Lu2, sc.Lf, sc.piv);
            for (int i = 0; i < D; ++i) y[i] = T(1) + T(0.125) * (T)((i * 7919 + sl * 104729) % 17) / T(17);
            inv_solve(D, sl, g.mcap, sc.Ld, sc.Lu, sc.Lu2, sc.Lf, sc.piv, y);
            inv_solve(D, sl, g.mcap, sc.Ld, sc.Lu, sc.Lu2, sc.Lf, sc.piv, y);
        }
        __syncthreads();
        // re-orthogonalise inside clusters (gap below 1e-3 |T|), one more solve, again
        for (int pass = 0; pass < 2; ++pass) {
            for (int s = 1; s < msel; ++s) {
                for (int s2 = s - 1; s2 >= 0 && fabs(m.lam[s] - m.lam[s2]) <= T(1e-3) * tnorm; --s2) {
                    T* ys = sc.Y + (size_t)s * g.Dp;
                    const T* yo = sc.Y + (size_t)s2 * g.Dp;
                    T dp = T(0);
                    for (int i = threadIdx.x; i < D; i += FB_THREADS) dp += ys[i] * yo[i];
                    dp = block_sum(dp, m.red);
                    T nn = T(0);
                    for (int i = threadIdx.x; i < D; i += FB_THREADS) { ys[i] -= dp * yo[i]; nn += ys[i] * ys[i]; }
                    nn = block_sum(nn, m.red);
                    const T inv = T(1) / Num<T>::sqrt_(nn);
                    for (int i = threadIdx.x; i < D; i += FB_THREADS) ys[i] *= inv;
                    __syncthreads();
                }
            }
            if (pass == 0) {
                if (threadIdx.x < msel)
                    inv_solve(D, (int)threadIdx.x, g.mcap, sc.Ld, sc.Lu, sc.Lu2, sc.Lf, sc.piv,
                              sc.Y + (size_t)threadIdx.x * g.Dp);
                __syncthreads();
            }
        }
        // back-transformation v = H_0 ... H_{D-3} y, one warp per vector (no block barriers)
        for (int s = warp; s < msel; s += FB_WARPS) {
            T* y = sc.Y + (size_t)s * g.Dp;
            for (int k = D - 3; k >= 0; --k) {
                T dp = T(0);
                for (int i = k + 1 + lane; i < D; i += 32) dp += el(m.A, g.ntl, i, k) * y[i];
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) dp += __shfl_xor_sync(0xffffffffu, dp, o);
                for (int i = k + 1 + lane; i < D; i += 32) y[i] -= T(2) * dp * el(m.A, g.ntl, i, k);
                __syncwarp();
            }
            T sg, pr;
            warp_sign_proj(y, m.r2, D, sg, pr);
            if (lane == 0) { m.res[2 * s] = sg * pr; m.res[2 * s + 1] = pr * pr; }
        }
        __syncthreads();
        if (threadIdx.x == 0 && a.out[2]) {
            T acc = T(0), acc2 = T(0);
            for (int s = 0; s < msel; ++s) { acc += m.res[2 * s]; acc2 += m.res[2 * s + 1]; }
            a.out[2][pix] = (float)(a.dwest_mode == 0 ? fabs(acc) : Num<T>::sqrt_(acc2));
        }
        __syncthreads();
    }
    return redo;
}

template <typename T>
__global__ void __launch_bounds__(FB_THREADS, 1) fullband_kernel(FullArgs a, Geo g, Geo g64, char* ws, size_t slab_bytes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int sflag;
    __shared__ int s_m;
    __shared__ T s_bounds[4];
    __shared__ double s_bounds64[4];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_err;
    const int warp = threadIdx.x >> 5;
    char* slab = ws + (size_t)blockIdx.x * slab_bytes;
    TcState st{};
    // shared memory: [tensor-core chunk buffers][matrix if it fits][vectors]
    char* sp = reinterpret_cast<char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    if (g.tcg) {
        st.buf[0] = reinterpret_cast<__nv_bfloat16*>(sp);
        st.buf[1] = reinterpret_cast<__nv_bfloat16*>(sp + kTcBufBytes / 2);
        sp += kTcBufBytes;
    }
    Smem<T> m;
    Scratch<T> sc;
    char* sp_end;
    carve<T>(sp, g, m, sc, g.a_in_smem, &sp_end);
    // slab: [matrix unless in shared memory][eigen scratch][FP64 re-solve area (mixed)]
    char* q = slab;
    if (!g.a_in_smem) { m.A = reinterpret_cast<T*>(q); q += ((sizeof(T) * (size_t)g.ntl * 16 + 255) & ~(size_t)255); }
    if (g.pan_in_tc) m.pan = reinterpret_cast<T*>(st.buf[0]);
    else if (g.pan_in_smem) m.pan = reinterpret_cast<T*>(sp_end);
    else { m.pan = reinterpret_cast<T*>(q); q += pan_bytes<T>(g.Dp); }
    carve_scratch<T>(q, g, sc, &q);
    Smem<double> m64;
    Scratch<double> sc64;
    if (g.tc) {
        carve<double>(q, g64, m64, sc64, true, &q);
        m64.pan = reinterpret_cast<double*>(q);
        q += pan_bytes<double>(g64.Dp);
        carve_scratch<double>(q, g64, sc64, &q);
    }
    if (g.tcg) {
        if (threadIdx.x == 0) {
            s_err = 0;
            tc::mbar_init(&s_bar[0], 1);
            tc::mbar_init(&s_bar[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        if (warp == 0) {
            tc::tmem_alloc(&s_tmem, TC_COLS);
            tc::tmem_relinquish();
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        st.bar = s_bar;
        st.tmem = s_tmem;
        st.err = &s_err;
    }
    const int ro = a.outer / 2;
    const int64_t P = (int64_t)a.H * a.W;
    const unsigned want = (a.out[0] ? 1u : 0u) | (a.out[1] ? 2u : 0u) | (a.out[2] ? 4u : 0u);
    const float fnan = __int_as_float(0x7fc00000);
    const int64_t count = a.pix ? a.npix : P;
    for (int64_t it = blockIdx.x; it < count; it += gridDim.x) {
        const int64_t pix = a.pix ? a.pix[it] : it;
        const int py = (int)(pix / a.W), px = (int)(pix % a.W);
        if (a.border == 1 && (py - ro < 0 || py + ro >= a.H || px - ro < 0 || px + ro >= a.W)) {
            if (threadIdx.x < 3 && a.out[threadIdx.x]) a.out[threadIdx.x][pix] = fnan;
            if (threadIdx.x == 0 && a.flags) a.flags[pix] = 4;
            continue;
        }
        uint8_t flag = 0;
        const unsigned redo = process_pixel<T>(a, g, m, sc, &st, pix, want, flag, &sflag, &s_m, s_bounds);
        if constexpr (sizeof(T) == 4) {
            if (g.tc && redo) {  // estimated condition above the gate: FP64 from the data
                uint8_t f64 = 0;
                process_pixel<double>(a, g64, m64, sc64, nullptr, pix, redo, f64, &sflag, &s_m, s_bounds64);
                flag = (uint8_t)((flag & ~2u) | f64 | 1u);
            }
        }
        if (threadIdx.x == 0 && a.flags) a.flags[pix] = flag;
    }
    if (g.tcg) {
        __syncthreads();
        if (s_err) {  // a wait gave up: give the tensor cores a last bounded chance to finish
            tc::mbar_wait_bounded(&s_bar[0], st.uses[0] & 1, TC_WAIT);
            tc::mbar_wait_bounded(&s_bar[1], st.uses[1] & 1, TC_WAIT);
            if (threadIdx.x == 0 && a.status) atomicExch(a.status, (int)WDAD_ERR_TIMEOUT);
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (warp == 0) tc::tmem_dealloc(st.tmem, TC_COLS);
    }
}

// A3 alone: background mean and covariance (1/N) of the listed pixels, written out
// densely (cov [npix][D][D], row-major, both triangles).  Same statistics code as the
// detectors: SIMT Gram (FP32 / FP64) or the BF16 tensor-core Gram (mixed precision).
template <typename T>
__global__ void __launch_bounds__(FB_THREADS, 1) moments_kernel(FullArgs a, Geo g, const int64_t* __restrict__ pix,
                                                                 int64_t npix, float* __restrict__ mu_out,
                                                                 float* __restrict__ cov_out, char* ws,
                                                                 size_t slab_bytes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_err;
    const int warp = threadIdx.x >> 5;
    char* slab = ws + (size_t)blockIdx.x * slab_bytes;
    TcState st{};
    char* sp = reinterpret_cast<char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    size_t off = 0;
    if (g.tcg) {
        st.buf[0] = reinterpret_cast<__nv_bfloat16*>(sp);
        st.buf[1] = reinterpret_cast<__nv_bfloat16*>(sp + kTcBufBytes / 2);
        off += kTcBufBytes;
    }
    T* A;
    if (g.a_in_smem) { A = reinterpret_cast<T*>(sp + off); off += sizeof(T) * ntiles_of(g.nt) * 16; }
    else A = reinterpret_cast<T*>(slab);
    T* xs = reinterpret_cast<T*>(sp + off);
    T* mu = xs + (size_t)g.S * g.Dp;
    if (g.tcg) {
        if (threadIdx.x == 0) {
            s_err = 0;
            tc::mbar_init(&s_bar[0], 1);
            tc::mbar_init(&s_bar[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        if (warp == 0) {
            tc::tmem_alloc(&s_tmem, TC_COLS);
            tc::tmem_relinquish();
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        st.bar = s_bar;
        st.tmem = s_tmem;
        st.err = &s_err;
    }
    const int ro = a.outer / 2, ri = a.inner / 2;
    const int N = a.outer * a.outer - a.inner * a.inner;
    const int D = g.D;
    for (int64_t t = blockIdx.x; t < npix; t += gridDim.x) {
        const int64_t p = pix[t];
        const int py = (int)(p / a.W), px = (int)(p % a.W);
        __syncthreads();
        sample_mean<T>(a.x, a.H, a.W, g, py, px, 0, N, ro, ri, mu, xs);
        __syncthreads();
        mat_zero(A, g);
        if constexpr (sizeof(T) == 4) {
            if (g.tcg) gram_tc<1>(a.x, a.H, a.W, g, py, px, 0, N, ro, ri, mu, 1.f / (float)N, A, st);
        }
        if (!g.tcg) {
            gram_accumulate<T>(a.x, a.H, a.W, g, py, px, 0, N, ro, ri, mu, T(1), A, xs);
            mat_scale(A, g, T(1) / (T)N);
        }
        for (int b = threadIdx.x; b < D; b += FB_THREADS) mu_out[t * D + b] = (float)mu[b];
        for (int e = threadIdx.x; e < D * D; e += FB_THREADS) {
            const int r = e / D, c = e % D;
            cov_out[t * D * D + e] = (float)(r >= c ? el(A, g.ntl, r, c) : el(A, g.ntl, c, r));
        }
    }
    if (g.tcg) {
        __syncthreads();
        if (s_err) {
            tc::mbar_wait_bounded(&s_bar[0], st.uses[0] & 1, TC_WAIT);
            tc::mbar_wait_bounded(&s_bar[1], st.uses[1] & 1, TC_WAIT);
            if (threadIdx.x == 0 && a.status) atomicExch(a.status, (int)WDAD_ERR_TIMEOUT);
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (warp == 0) tc::tmem_dealloc(st.tmem, TC_COLS);
    }
}

template <typename T>
Geo make_geo_only(const FullArgs& a) {
    Geo g{};
    g.D = a.D;
    g.Dp = (a.D + 3) & ~3;
    g.nt = g.Dp / 4;
    g.ntl = ntiles_of(g.nt);
    g.S = fb_chunk(sizeof(T));
    g.mcap = std::min(g.Dp, a.inner * a.inner + 16);
    g.N = a.outer * a.outer - a.inner * a.inner;
    g.Np = (g.N + 3) & ~3;
    g.wood = g.N < g.D && a.loading > 0.0 && (int64_t)a.H * a.W < (int64_t)INT32_MAX;
    g.tc = false;
    g.tcg = false;
    g.pieces = 1;
    g.a_in_smem = false;
    g.pan_in_tc = false;
    g.pan_in_smem = false;
    return g;
}

template <typename T>
Geo make_geo(const FullArgs& a, bool* smem_ok, size_t* smem_bytes, size_t* slab, Geo* g64_out = nullptr,
             bool split_ok = false) {
    Geo g = make_geo_only<T>(a);
    const size_t amat = sizeof(T) * (size_t)g.ntl * 16;
    const size_t vecs = vec_bytes<T>(g);
    g.tc = (sizeof(T) == 4) && a.precision == WDAD_PREC_MIXED && a.D <= 256;
    // the FP32 detectors' L x L window Gram (LRX / DWRX with N >= D) on the tensor cores in the
    // three-piece split, which keeps FP32 accuracy (only while the matrix still fits shared memory
    // beside the chunk buffers)
    const bool split = split_ok && (sizeof(T) == 4) && a.precision == WDAD_PREC_FP32 && a.D <= 256 && !g.wood &&
                       (a.out[0] || a.out[1]) && amat + vecs + kTcBufBytes <= 210 * 1024;
    g.tcg = g.tc || split;
    g.pieces = g.tc ? 1 : 3;
    const size_t tcb = g.tcg ? kTcBufBytes : 0;
    g.a_in_smem = (sizeof(T) == 4) && (amat + vecs + tcb <= 210 * 1024);
    const size_t panb = pan_bytes<T>(g.Dp);
    size_t sm = vecs + tcb + (g.a_in_smem ? amat : 0);
    g.pan_in_tc = g.tcg && panb <= kTcBufBytes;
    g.pan_in_smem = !g.pan_in_tc && sm + panb <= 210 * 1024;
    if (g.pan_in_smem) sm += panb;
    *smem_bytes = sm + 1024;  // + alignment slack
    *smem_ok = *smem_bytes <= 227 * 1024;
    size_t sl = (g.a_in_smem ? 0 : ((amat + 255) & ~(size_t)255)) + (g.pan_in_tc || g.pan_in_smem ? 0 : panb) +
                scratch_bytes<T>(g);
    Geo g64 = make_geo_only<double>(a);
    if (g.tc) sl += ((sizeof(double) * (size_t)g64.ntl * 16 + 255) & ~(size_t)255) + vec_bytes<double>(g64) +
                    pan_bytes<double>(g64.Dp) + scratch_bytes<double>(g64);
    *slab = (sl + 255) & ~(size_t)255;
    if (g64_out) *g64_out = g64;
    return g;
}

}  // namespace

static int fb_grid(int num_sms, int64_t P) {
    int64_t g = num_sms;
    if (g > P) g = P;
    return (int)(g < 1 ? 1 : g);
}

size_t fullband_workspace_bytes(const FullArgs& a, int num_sms) {
    if (a.D < 9 || a.D > 1024) return 0;
    bool ok;
    size_t smem, slab;
    if (a.precision == WDAD_PREC_FP64) make_geo<double>(a, &ok, &smem, &slab);
    else make_geo<float>(a, &ok, &smem, &slab, nullptr, true);
    if (!ok) return 0;
    return slab * (size_t)fb_grid(num_sms, a.pix ? a.npix : (int64_t)a.H * a.W) + 256;
}

template <typename T>
static cudaError_t launch_fb(const FullArgs& a, void* ws, int num_sms, cudaStream_t s) {
    bool ok;
    size_t smem, slab;
    Geo g64{};
    const Geo g = make_geo<T>(a, &ok, &smem, &slab, &g64, true);
    if (!ok) return cudaErrorInvalidValue;
    cudaError_t e = raise_smem_limit(fullband_kernel<T>);
    if (e != cudaSuccess) return e;
    const int grid = fb_grid(num_sms, a.pix ? a.npix : (int64_t)a.H * a.W);
    char* base = reinterpret_cast<char*>(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    fullband_kernel<T><<<grid, FB_THREADS, smem, s>>>(a, g, g64, base, slab);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_mom(const FullArgs& a, const int64_t* pix, int64_t npix, float* mu, float* cov, void* ws,
                              int num_sms, cudaStream_t s) {
    bool ok;
    size_t smem, slab;
    const Geo g = make_geo<T>(a, &ok, &smem, &slab);
    if (!ok) return cudaErrorInvalidValue;
    cudaError_t e = raise_smem_limit(moments_kernel<T>);
    if (e != cudaSuccess) return e;
    const int grid = fb_grid(num_sms, npix);
    char* base = reinterpret_cast<char*>(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    moments_kernel<T><<<grid, FB_THREADS, smem, s>>>(a, g, pix, npix, mu, cov, base, slab);
    return cudaGetLastError();
}

size_t moments_workspace_bytes(const FullArgs& a, int64_t npix, int num_sms) {
    if (a.D < 1 || a.D > 1024) return 0;
    bool ok;
    size_t smem, slab;
    if (a.precision == WDAD_PREC_FP64) make_geo<double>(a, &ok, &smem, &slab);
    else make_geo<float>(a, &ok, &smem, &slab);
    if (!ok) return 0;
    return slab * (size_t)fb_grid(num_sms, npix) + 256;
}

cudaError_t launch_window_moments(const FullArgs& a, const int64_t* pix, int64_t npix, float* mu, float* cov, void* ws,
                                  size_t ws_bytes, int num_sms, cudaStream_t s) {
    if (npix == 0) return cudaSuccess;
    if (ws_bytes < moments_workspace_bytes(a, npix, num_sms)) return cudaErrorInvalidValue;
    if (a.precision == WDAD_PREC_FP64) return launch_mom<double>(a, pix, npix, mu, cov, ws, num_sms, s);
    return launch_mom<float>(a, pix, npix, mu, cov, ws, num_sms, s);
}

cudaError_t launch_detect_full(const FullArgs& a, void* ws, size_t ws_bytes, int num_sms, cudaStream_t s) {
    if ((int64_t)a.H * a.W == 0 || (a.pix && a.npix == 0)) return cudaSuccess;
    if (ws_bytes < fullband_workspace_bytes(a, num_sms)) return cudaErrorInvalidValue;
    if (a.precision == WDAD_PREC_FP64) return launch_fb<double>(a, ws, num_sms, s);
    return launch_fb<float>(a, ws, num_sms, s);
}

}  // namespace wdad
