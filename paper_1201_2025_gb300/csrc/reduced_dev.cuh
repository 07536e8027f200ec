// A2-A5 on few bands (dim D <= 8, the DWT approximation matrix of Sec. 4):
// dual-window statistics, regularised solve and eigen-decomposition, fused in
// one kernel per output tile of 32 columns x th rows.
//
//  stage 0  warp 0 forms a tile reference spectrum c (the mean of the middle halo
//           row, read from global memory in a fixed order) while every warp
//           fetches its share of the tile plus a halo of outer/2 pixels; after one
//           barrier the pixels are stored shifted, x - c, so that the second
//           moments below are sums of (x - c)(x - c)^T with little cancellation.
//           Every index is reflected at the image border (reflect-101).
//  stage 1  vertical box sums, one work item per (channel group, halo column,
//           outer or inner height): the D first-order and D(D+1)/2 second-order
//           channels of each pixel are formed where they are needed (two groups of
//           channels, so that each pixel is read from shared memory twice), and the
//           sums over the outer and the inner window height slide down the th
//           output rows (a direct sum for the first row, then add the entering
//           and subtract the leaving row).
//  stage 2  horizontal box sums of those, in place, one work item per (channel,
//           output row, outer or inner): segments of 8 output columns, each a
//           direct sum and 7 sliding updates; for radii up to 10 a segment's
//           inputs are held in registers.  Afterwards the planes hold, per
//           output pixel, the sums over the outer square and over the inner
//           square; the background annulus is outer minus inner (Sec. 2.2).
//  stage 3  per pixel: mu_o, C_o (1/N), mu_i, C_i (1/n_i); LRX (Eq. 1) and DWRX
//           (Eq. 5) through a Cholesky factor of C_o + delta I, delta =
//           loading * trace(C_o) / D; DWEST (Eq. 2-4) through a cyclic Jacobi
//           eigen-decomposition of C_i - C_o.
//
// Every sliding sum restarts at least every 16 rows and every 8 columns, which bounds
// the FP32 rounding it accumulates.  Stages 0-2 are templated on the payload, so the
// window census (integer pixel indices instead of spectra) runs exactly the indexing
// and summation code of the detectors and can be checked bit for bit.  Results do not
// depend on the block size (a multiple of 32, at most 512): every sum has a fixed order.
#pragma once
#include <float.h>

#include <cuda.h>

#include "internal.h"
#include "tc.cuh"

namespace wdad {

constexpr int TW = 32;          // tile width in output columns
constexpr int kMaxSmem = 227 * 1024;
constexpr int kSeg = 8;         // horizontal outputs per sliding segment
constexpr int kRegRadius = 10;  // horizontal radii whose segments are held in registers

__host__ __device__ __forceinline__ int halo_pitch(int WR) { return WR | 1; }  // odd pixel pitch
// Row pitch (elements) of a sum plane: at least n and 4 mod 8, so that 16-byte loads of
// eight consecutive rows fall on eight different bank groups.
__host__ __device__ __forceinline__ int plane_pitch(int n) {
    const int p = (n + 3) & ~3;
    return (p & 7) ? p : p + 4;
}

struct TileGeom {
    int H, W, ro, ri, th;        // image, radii, tile height
    int ty0, tx0;                // tile origin
    int HR, WR, XP;              // halo rows / cols, halo row pitch in pixels
    int WI;                      // columns that carry inner sums (TW + 2 ri)
    int VP, VPI;                 // row pitch of the outer / inner sum planes
    __device__ TileGeom(int H_, int W_, int inner, int outer, int th_, int tile_x, int tile_y)
        : H(H_), W(W_), ro(outer / 2), ri(inner / 2), th(th_) {
        ty0 = tile_y * th;
        tx0 = tile_x * TW;
        HR = th + 2 * ro;
        WR = TW + 2 * ro;
        XP = halo_pitch(WR);
        WI = TW + 2 * ri;
        VP = plane_pitch(WR);
        VPI = plane_pitch(WI);
    }
};

// Shared memory of one tile: the halo (words_per_px 4-byte words per pixel, rounded up
// to 16 bytes), the outer and inner sum planes (nc channels of tsize bytes), the tile
// reference (32 bytes).
__host__ __device__ __forceinline__ size_t tile_smem_bytes(int words_per_px, int nc, int tsize, int inner, int outer,
                                                           int th) {
    const int ro = outer / 2, ri = inner / 2;
    const size_t HR = th + 2 * ro, XP = halo_pitch(TW + 2 * ro);
    const size_t xs = (HR * XP * words_per_px * 4 + 15) & ~(size_t)15;
    return xs + (size_t)nc * th * (plane_pitch(TW + 2 * ro) + plane_pitch(TW + 2 * ri)) * tsize + 32;
}

// ---------------------------------------------------------------- payloads
template <int D>
struct SpecPayload {                          // D-band spectra, float
    using T = float;
    static constexpr int DP = (D <= 4) ? 4 : 8;  // padded pixel stride in floats
    static constexpr int NC = D + D * (D + 1) / 2;
    static constexpr int WORDS = DP;             // 4-byte words per halo pixel
    // first- then second-order channels of one shifted spectrum
    static __device__ __forceinline__ void channels(const float* v, float (&ch)[NC]) {
#pragma unroll
        for (int k = 0; k < D; ++k) ch[k] = v[k];
        int q = D;
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b) ch[q++] = v[a] * v[b];
    }
    static constexpr int PX = DP;                // elements of T per halo pixel
    // vertical-pass channel groups [0, QSPLIT) and [QSPLIT, NC): the first-order channels
    // with the products x_0 x_b, then the other products (4 + 4 and 6 channels at D = 4)
    static constexpr int QSPLIT = 2 * D < NC ? 2 * D : NC;
    // the channels of the halo pixel at p
    static __device__ __forceinline__ void pixel_channels(const float* p, float (&ch)[NC]) {
        float v[D];
        if constexpr (D == 4) {
            const float4 q = *reinterpret_cast<const float4*>(p);
            v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else {
#pragma unroll
            for (int k = 0; k < D; ++k) v[k] = p[k];
        }
        channels(v, ch);
    }
};

struct CensusPayload {                        // linear pixel index, int64
    using T = long long;
    static constexpr int NC = 3;                 // 1, q, q^2
    static constexpr int WORDS = 2;
    static constexpr int PX = 1;
    static constexpr int QSPLIT = 2;             // groups (1, q) and (q^2)
    static __device__ __forceinline__ void pixel_channels(const long long* p, long long (&ch)[NC]) {
        const long long q = *p;
        ch[0] = 1; ch[1] = q; ch[2] = q * q;
    }
};

// ---------------------------------------------------------------- stage 0: reflected, shifted halo
// Tile reference: the mean of halo row HR / 2, summed lane-strided then by a fixed
// shuffle tree (one warp; the same value whatever the block size).
template <int D>
__device__ __forceinline__ void tile_reference(const TileGeom& g, const float* __restrict__ x, float* cref, int lane) {
    float acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = 0.f;
    const int gy = reflect101(g.ty0 - g.ro + g.HR / 2, g.H);
    for (int c = lane; c < g.WR; c += 32) {
        const int gx = reflect101(g.tx0 - g.ro + c, g.W);
        const float* px = x + ((size_t)gy * g.W + gx) * D;
        if constexpr (D == 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(px));
            acc[0] += v.x; acc[1] += v.y; acc[2] += v.z; acc[3] += v.w;
        } else {
#pragma unroll
            for (int k = 0; k < D; ++k) acc[k] += __ldg(px + k);
        }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
        float t = acc[k];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) cref[k] = t / (float)g.WR;
    }
}

template <int D>
__device__ __forceinline__ void fetch_pixel(const float* __restrict__ x, int W, int gy, int gx, float (&v)[D]) {
    const float* px = x + ((size_t)gy * W + gx) * D;
    if constexpr (D == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(px));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
#pragma unroll
        for (int k = 0; k < D; ++k) v[k] = __ldg(px + k);
    }
}

template <int D>
__device__ __forceinline__ void store_shifted(float* dst, const float (&v)[D], const float (&c)[D]) {
    if constexpr (D == 4) {
        *reinterpret_cast<float4*>(dst) = make_float4(v[0] - c[0], v[1] - c[1], v[2] - c[2], v[3] - c[3]);
    } else {
#pragma unroll
        for (int k = 0; k < D; ++k) dst[k] = v[k] - c[k];
    }
}

// Warp w takes halo rows w, w + nw, ...; lanes take columns.  The first 64 columns of
// every warp's first kHeld rows are fetched before the barrier that publishes the tile
// reference, so their latency overlaps warp 0's reference sum; the rest after it.
constexpr int kHeld = 2;
// Halo of an interior tile (no reflected row or column) of the 4-band cube by one 2-D tensor
// copy: thread 0 issues the box (HR rows of XP pixels, XP * 16 bytes each, the extra column past
// WR unused) into xs through the tile's mbarrier; the tile reference (the middle row's mean,
// summed in tile_reference's order, so the same value) and the shift (x - reference) then run
// in shared memory.  Returns false if the copy did not land within the bounded wait (then xs
// must not be used).
constexpr uint32_t kHaloWait = 1u << 24;
__device__ __forceinline__ bool load_halo_tma(const TileGeom& g, const CUtensorMap* tm, float* xs, float* cref,
                                              uint64_t* bar) {
    const uint32_t bytes = (uint32_t)(g.HR * g.XP * 16);
    if (threadIdx.x == 0) {
        tc::mbar_arrive_expect_tx(bar, bytes);
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
            ::"r"(tc::smem_u32(xs)), "l"(reinterpret_cast<uint64_t>(tm)), "r"((g.tx0 - g.ro) * 4), "r"(g.ty0 - g.ro),
              "r"(tc::smem_u32(bar))
            : "memory");
    }
    bool ok = tc::mbar_wait_bounded(bar, 0u, kHaloWait);
    if (!ok) ok = tc::mbar_wait_bounded(bar, 0u, 16u * kHaloWait);  // a late copy must land before exit
    if (__syncthreads_and(ok) == 0) return false;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const float* row = xs + (size_t)(g.HR / 2) * g.XP * 4;
        for (int c = lane; c < g.WR; c += 32) {
            const float4 v = *reinterpret_cast<const float4*>(row + c * 4);
            acc[0] += v.x; acc[1] += v.y; acc[2] += v.z; acc[3] += v.w;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float t = acc[k];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) cref[k] = t / (float)g.WR;
        }
    }
    __syncthreads();
    const float4 c = make_float4(cref[0], cref[1], cref[2], cref[3]);
    for (int q = threadIdx.x; q < g.HR * g.XP; q += blockDim.x) {
        float4* p = reinterpret_cast<float4*>(xs) + q;
        const float4 v = *p;
        *p = make_float4(v.x - c.x, v.y - c.y, v.z - c.z, v.w - c.w);
    }
    return true;
}

template <int D>
__device__ __forceinline__ void load_halo_spec(const TileGeom& g, const float* __restrict__ x, float* xs, float* cref) {
    using P = SpecPayload<D>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float v[kHeld][2][D];
    int dst[kHeld][2];
#pragma unroll
    for (int k = 0; k < kHeld; ++k) {
        const int r = warp + k * nw;
        const int gy = reflect101(g.ty0 - g.ro + (r < g.HR ? r : 0), g.H);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            dst[k][h] = -1;
            if (r < g.HR && c < g.WR) {
                fetch_pixel<D>(x, g.W, gy, reflect101(g.tx0 - g.ro + c, g.W), v[k][h]);
                dst[k][h] = r * g.XP + c;
            }
        }
    }
    if (warp == 0) tile_reference<D>(g, x, cref, lane);
    __syncthreads();
    float c[D];
#pragma unroll
    for (int k = 0; k < D; ++k) c[k] = cref[k];
#pragma unroll
    for (int k = 0; k < kHeld; ++k)
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (dst[k][h] >= 0) store_shifted<D>(xs + dst[k][h] * P::DP, v[k][h], c);
    for (int r = warp; r < g.HR; r += nw) {
        // columns the held rows did not cover (halos wider than 64 pixels), then the rest
        const int c0 = (r < warp + kHeld * nw) ? 64 : 0;
        if (c0 >= g.WR) continue;
        const int gy = reflect101(g.ty0 - g.ro + r, g.H);
        for (int cc = lane + c0; cc < g.WR; cc += 32) {
            float t[D];
            fetch_pixel<D>(x, g.W, gy, reflect101(g.tx0 - g.ro + cc, g.W), t);
            store_shifted<D>(xs + (r * g.XP + cc) * P::DP, t, c);
        }
    }
}

__device__ __forceinline__ void load_halo_census(const TileGeom& g, long long* xs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = warp; r < g.HR; r += nw) {
        const int gy = reflect101(g.ty0 - g.ro + r, g.H);
        for (int c = lane; c < g.WR; c += 32)
            xs[(size_t)r * g.XP + c] = (long long)gy * g.W + reflect101(g.tx0 - g.ro + c, g.W);
    }
}

// ---------------------------------------------------------------- stage 1: vertical sums
// Item (channel group, halo column, outer or inner): channels [Q0, Q0 + NQ) of the halo
// column at `in` (its row r0) summed over w rows starting at row r0 + i, for output rows
// i = 0 .. th-1, into out + q * plane + i * pitch.  rs: elements of T per halo row.
template <class P, int Q0, int NQ>
__device__ __forceinline__ void vertical_item(const typename P::T* __restrict__ in, int rs,
                                              typename P::T* __restrict__ out, int plane, int pitch, int th, int w) {
    using T = typename P::T;
    constexpr int NC = P::NC;
    if (w == 1) {  // a window one row high: the channels themselves
        for (int i = 0; i < th; ++i, in += rs, out += pitch) {
            T ch[NC];
            P::pixel_channels(in, ch);
#pragma unroll
            for (int j = 0; j < NQ; ++j) out[(Q0 + j) * plane] = ch[Q0 + j];
        }
        return;
    }
    T acc[NQ];
#pragma unroll
    for (int j = 0; j < NQ; ++j) acc[j] = T(0);
    const T* pe = in;
    for (int k = 0; k < w; ++k, pe += rs) {
        T ch[NC];
        P::pixel_channels(pe, ch);
#pragma unroll
        for (int j = 0; j < NQ; ++j) acc[j] += ch[Q0 + j];
    }
#pragma unroll
    for (int j = 0; j < NQ; ++j) out[(Q0 + j) * plane] = acc[j];
    // pe: the row entering the window of output row i, in: the row leaving it
#pragma unroll 2
    for (int i = 1; i < th; ++i) {
        out += pitch;
        T e[NC], l[NC];
        P::pixel_channels(pe, e);
        P::pixel_channels(in, l);
        pe += rs;
        in += rs;
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
            acc[j] += e[Q0 + j] - l[Q0 + j];  // one rounding at the running-sum magnitude
            out[(Q0 + j) * plane] = acc[j];
        }
    }
}

template <class P, int G>
__device__ __forceinline__ void vertical_group(const typename P::T* in, int rs, typename P::T* out, int plane,
                                               int pitch, int th, int w) {
    constexpr int Q0 = G == 0 ? 0 : P::QSPLIT;
    constexpr int NQ = G == 0 ? P::QSPLIT : P::NC - P::QSPLIT;
    if constexpr (NQ > 0) vertical_item<P, Q0, NQ>(in, rs, out, plane, pitch, th, w);
}

// Items are laid out so that every warp holds one (group, outer or inner) pair: the outer
// columns and the inner columns of a group each start on a warp boundary.  Two channel
// groups: every item reloads its pixels from shared memory, so fewer groups move fewer
// bytes, and two keep enough items in flight.
template <class P>
__device__ __forceinline__ void vertical_sums(const TileGeom& g, const typename P::T* xs, typename P::T* Vo,
                                              typename P::T* Vi) {
    constexpr int NG = P::QSPLIT < P::NC ? 2 : 1;
    const int no = (g.WR + 31) & ~31, ni = (g.WI + 31) & ~31;
    const int per = no + ni;
    const int rs = g.XP * P::PX;
    for (int t = threadIdx.x; t < NG * per; t += blockDim.x) {
        const int grp = t / per, rem = t - grp * per;
        const bool outer = rem < no;
        const int c = outer ? rem : rem - no;
        if (c >= (outer ? g.WR : g.WI)) continue;
        const typename P::T* in = outer ? xs + c * P::PX : xs + ((g.ro - g.ri) * g.XP + c + g.ro - g.ri) * P::PX;
        typename P::T* out = outer ? Vo + c : Vi + c;
        const int pitch = outer ? g.VP : g.VPI;
        const int w = outer ? 2 * g.ro + 1 : 2 * g.ri + 1;
        const int plane = g.th * pitch;
        if (grp == 0) vertical_group<P, 0>(in, rs, out, plane, pitch, g.th, w);
        else vertical_group<P, 1>(in, rs, out, plane, pitch, g.th, w);
    }
}

// ---------------------------------------------------------------- stage 2: horizontal sums, in place
template <class T, int N>
__device__ __forceinline__ void load_row(const T* p, T (&v)[N]) {
    constexpr int V = 16 / sizeof(T);  // elements per 16-byte load (p is 16-byte aligned)
#pragma unroll
    for (int k = 0; k < N; k += V) {
        if constexpr (sizeof(T) == 4) {
            const float4 q = *reinterpret_cast<const float4*>(p + k);
            const float e[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (k + u < N) v[k + u] = e[u];
        } else {
            const longlong2 q = *reinterpret_cast<const longlong2*>(p + k);
            v[k] = q.x;
            if (k + 1 < N) v[k + 1] = q.y;
        }
    }
}

template <class T>
__device__ __forceinline__ void store_seg(T* p, const T (&o)[kSeg]) {
#pragma unroll
    for (int k = 0; k < kSeg; k += 16 / (int)sizeof(T)) {
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4*>(p + k) = make_float4(o[k], o[k + 1], o[k + 2], o[k + 3]);
        } else {
            *reinterpret_cast<longlong2*>(p + k) = make_longlong2(o[k], o[k + 1]);
        }
    }
}

// Row of TW + 2R column sums -> TW window sums of width 2R + 1, in place; segment s reads
// columns [8s, 8s + 8 + 2R) into registers and writes [8s, 8s + 8).
template <class T, int R>
__device__ __forceinline__ void hrow_reg(T* row) {
    constexpr int NV = kSeg + 2 * R;
    if constexpr (R > 0) {  // (a window one column wide: the column sums already are the window sums)
#pragma unroll
        for (int s = 0; s < TW / kSeg; ++s) {
            T v[NV];
            load_row<T, NV>(row + s * kSeg, v);
            T o[kSeg];
            T acc = v[0];
#pragma unroll
            for (int k = 1; k < 2 * R + 1; ++k) acc += v[k];
            o[0] = acc;
#pragma unroll
            for (int j = 1; j < kSeg; ++j) {
                acc += v[j + 2 * R] - v[j - 1];
                o[j] = acc;
            }
            store_seg<T>(row + s * kSeg, o);
        }
    }
}

// The same for any radius, reading shared memory as it goes: the value leaving the window
// at column j - 1 is kept from before that column was overwritten.
template <class T>
__device__ __forceinline__ void hrow_smem(T* row, int R) {
    if (R == 0) return;
    for (int s = 0; s < TW / kSeg; ++s) {
        T* p = row + s * kSeg;
        T acc = p[0];
        for (int k = 1; k < 2 * R + 1; ++k) acc += p[k];
        T carry = p[0];
        p[0] = acc;
        for (int j = 1; j < kSeg; ++j) {
            acc += p[j + 2 * R] - carry;
            carry = p[j];
            p[j] = acc;
        }
    }
}

template <class T>
__device__ __forceinline__ void hrow(T* row, int R) {
    switch (R) {
        case 0: hrow_reg<T, 0>(row); break;
        case 1: hrow_reg<T, 1>(row); break;
        case 2: hrow_reg<T, 2>(row); break;
        case 3: hrow_reg<T, 3>(row); break;
        case 4: hrow_reg<T, 4>(row); break;
        case 5: hrow_reg<T, 5>(row); break;
        case 6: hrow_reg<T, 6>(row); break;
        case 7: hrow_reg<T, 7>(row); break;
        case 8: hrow_reg<T, 8>(row); break;
        case 9: hrow_reg<T, 9>(row); break;
        case 10: hrow_reg<T, 10>(row); break;
        default: hrow_smem<T>(row, R); break;
    }
}

template <class P>
__device__ __forceinline__ void horizontal_sums(const TileGeom& g, typename P::T* Vo, typename P::T* Vi) {
    constexpr int NC = P::NC;
    const int rows = NC * g.th;
    for (int t = threadIdx.x; t < 2 * rows; t += blockDim.x) {
        if (t < rows) hrow(Vo + t * g.VP, g.ro);
        else hrow(Vi + (t - rows) * g.VPI, g.ri);
    }
}

// Stages 0-2 of one tile for a payload: afterwards Vo[(q th + i) VP + j] holds the outer-square
// sum and Vi[(q th + i) VPI + j] the inner-square sum of channel q at output pixel (i, j).
template <class P>
__device__ __forceinline__ void tile_sums(const TileGeom& g, typename P::T* xs, typename P::T* Vo,
                                          typename P::T* Vi) {
    vertical_sums<P>(g, xs, Vo, Vi);
    __syncthreads();
    horizontal_sums<P>(g, Vo, Vi);
    __syncthreads();
}

// ---------------------------------------------------------------- small dense algebra in registers
// Cholesky G = L L^T in place: the strict lower triangle receives L and the diagonal the
// reciprocal pivots 1 / L_jj (one rsqrtf each, so the solves multiply instead of divide).
// Fails when a pivot is not above `floor` (a multiple of the FP32 rounding level of the
// moments the matrix was formed from), so exactly singular covariances are reported instead
// of factorised from rounding noise.
template <int D>
__device__ __forceinline__ bool chol_inplace(float (&G)[D][D], float floor) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
        float s = G[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s = fmaf(-G[j][k], G[j][k], s);
        if (!(s > floor)) return false;
        const float inv = rsqrtf(s);
        G[j][j] = inv;
#pragma unroll
        for (int i = j + 1; i < D; ++i) {
            float t = G[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) t = fmaf(-G[i][k], G[j][k], t);
            G[i][j] = t * inv;
        }
    }
    return true;
}

// ||L^{-1} d||^2 = d^T (L L^T)^{-1} d for the factor chol_inplace leaves in G
template <int D>
__device__ __forceinline__ float chol_quad(const float (&G)[D][D], const float (&d)[D]) {
    float y[D];
    float q = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        float t = d[i];
#pragma unroll
        for (int k = 0; k < i; ++k) t = fmaf(-G[i][k], y[k], t);
        y[i] = t * G[i][i];
        q = fmaf(y[i], y[i], q);
    }
    return q;
}

// Round-robin (circle method) pairing of D indices, D padded to an even count E:
// round r pairs slot 0 with slot 1 + r and slot 1 + (r + k) % (E - 1) with slot
// 1 + (r - k + E - 1) % (E - 1), k = 1 .. E/2 - 1.  Index E - 1 >= D is a bye.
__host__ __device__ constexpr int rr_first(int E, int r, int k) { return k == 0 ? 0 : 1 + (r + k) % (E - 1); }
__host__ __device__ constexpr int rr_second(int E, int r, int k) {
    return k == 0 ? 1 + r : 1 + (r - k + E - 1) % (E - 1);
}

// Parallel-order Jacobi on a symmetric D x D matrix (symmetric Schur rotations,
// Golub & Van Loan Sec. 8.5; the round-robin ordering lets the rotations of one
// round, which act on disjoint index pairs, be computed and applied together).
// Each rotation zeroes a_pq and moves a_pp, a_qq by -/+ t a_pq; the blocks between
// two pairs transform as R_i^T B R_j.  A is first scaled to unit Frobenius norm, so every
// rotation's operands stay normal whatever the data's scale.  Entries at or below the FP32
// rounding level (2^-22 of the norm) are left alone; sweeps end when no off-diagonal entry
// is above that level.  On return A's diagonal holds the eigenvalues divided by ||A||_F (their
// signs and ratios, which is all the DWEST selection uses), V's columns the eigenvectors.
template <int D>
__device__ __forceinline__ void jacobi_inplace(float (&A)[D][D], float (&V)[D][D]) {
    constexpr int E = D + (D & 1);
    constexpr int M = E / 2;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) V[a][b] = (a == b) ? 1.f : 0.f;
    if constexpr (D == 1) return;
    // the eigenvectors are accumulated as row pairs (rows 2h, 2h + 1 of column b in VP[h][b]),
    // so that each rotation of two columns is two packed multiplies and two packed FMAs per
    // row pair; an odd last row stays scalar
    constexpr int HP = D / 2;
    float2 VP[HP > 0 ? HP : 1][D];
    float VL[D];
#pragma unroll
    for (int h = 0; h < HP; ++h)
#pragma unroll
        for (int b = 0; b < D; ++b) VP[h][b] = make_float2(V[2 * h][b], V[2 * h + 1][b]);
#pragma unroll
    for (int b = 0; b < D; ++b) VL[b] = V[D - 1][b];
    float fro = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) fro = fmaf(A[a][b], A[a][b], fro);
    if (!(fro > 0.f)) return;  // zero matrix: already diagonal (NaN input stays NaN); V = I
    const float unit = rsqrtf(fro);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) A[a][b] *= unit;
    const float tol = 2.384185791e-7f;  // 2^-22 of the (unit) norm
    constexpr int kSweeps = (D <= 4) ? 8 : 12;
    for (int sweep = 0; sweep < kSweeps; ++sweep) {
        // a sweep rotates nothing exactly when no off-diagonal entry is above tol at its start
        // (nothing rotated leaves A unchanged), so that sweep is replaced by this check
        bool live = false;
#pragma unroll
        for (int p = 0; p < D; ++p)
#pragma unroll
            for (int q = p + 1; q < D; ++q) live |= fabsf(A[p][q]) > tol;
        if (!live) break;
#pragma unroll
        for (int r = 0; r < E - 1; ++r) {
            float c[M], sn[M];
            // rotation parameters of every pair of the round, from the same A
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int p0 = rr_first(E, r, k), q0 = rr_second(E, r, k);
                const int p = p0 < q0 ? p0 : q0, q = p0 < q0 ? q0 : p0;
                c[k] = 1.f; sn[k] = 0.f;
                if (q >= D) continue;
                const float apq = A[p][q];
                if (!(fabsf(apq) > tol)) continue;
                // t = sgn(theta) / (|theta| + sqrt(theta^2 + 1)) with theta = dq / h, dq = a_qq - a_pp,
                // h = 2 a_pq, written as sgn(dq) h / (|dq| + sqrt(dq^2 + h^2)): one rsqrtf and one
                // approximate division.  c^2 + s^2 = 1 holds to the rsqrtf error, and an inexact
                // angle only changes how much of a_pq the next sweeps still have to remove.
                const float dq = A[q][q] - A[p][p], h = 2.f * apq;
                const float ss = fmaf(dq, dq, h * h);
                const float r = ss * rsqrtf(ss);
                const float tt = __fdividef(h, fabsf(dq) + r);
                const float t = (dq < 0.f) ? -tt : tt;
                c[k] = rsqrtf(fmaf(t, t, 1.f));
                sn[k] = t * c[k];
                A[p][p] = fmaf(-t, apq, A[p][p]);
                A[q][q] = fmaf(t, apq, A[q][q]);
                A[p][q] = 0.f;
                A[q][p] = 0.f;
            }
            // blocks between two pairs: B <- R_i^T B R_j (and the transposed block)
#pragma unroll
            for (int i = 0; i < M; ++i)
#pragma unroll
                for (int j = i + 1; j < M; ++j) {
                    const int pi0 = rr_first(E, r, i), qi0 = rr_second(E, r, i);
                    const int pj0 = rr_first(E, r, j), qj0 = rr_second(E, r, j);
                    const int pi = pi0 < qi0 ? pi0 : qi0, qi = pi0 < qi0 ? qi0 : pi0;
                    const int pj = pj0 < qj0 ? pj0 : qj0, qj = pj0 < qj0 ? qj0 : pj0;
                    if (qi >= D && qj >= D) continue;
                    if (qi >= D) {  // pi is single: row vector A[pi][{pj,qj}] <- . R_j
                        const float x = A[pi][pj], y = A[pi][qj];
                        const float nx = c[j] * x - sn[j] * y, ny = sn[j] * x + c[j] * y;
                        A[pi][pj] = nx; A[pj][pi] = nx; A[pi][qj] = ny; A[qj][pi] = ny;
                        continue;
                    }
                    if (qj >= D) {  // pj is single: column A[{pi,qi}][pj] <- R_i^T .
                        const float x = A[pi][pj], y = A[qi][pj];
                        const float nx = c[i] * x - sn[i] * y, ny = sn[i] * x + c[i] * y;
                        A[pi][pj] = nx; A[pj][pi] = nx; A[qi][pj] = ny; A[pj][qi] = ny;
                        continue;
                    }
                    const float b00 = A[pi][pj], b01 = A[pi][qj], b10 = A[qi][pj], b11 = A[qi][qj];
                    // columns: B R_j
                    const float e00 = c[j] * b00 - sn[j] * b01, e01 = sn[j] * b00 + c[j] * b01;
                    const float e10 = c[j] * b10 - sn[j] * b11, e11 = sn[j] * b10 + c[j] * b11;
                    // rows: R_i^T (B R_j)
                    const float f00 = c[i] * e00 - sn[i] * e10, f10 = sn[i] * e00 + c[i] * e10;
                    const float f01 = c[i] * e01 - sn[i] * e11, f11 = sn[i] * e01 + c[i] * e11;
                    A[pi][pj] = f00; A[pj][pi] = f00; A[pi][qj] = f01; A[qj][pi] = f01;
                    A[qi][pj] = f10; A[pj][qi] = f10; A[qi][qj] = f11; A[qj][qi] = f11;
                }
            // eigenvectors: V <- V J
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int p0 = rr_first(E, r, k), q0 = rr_second(E, r, k);
                const int p = p0 < q0 ? p0 : q0, q = p0 < q0 ? q0 : p0;
                if (q >= D) continue;
                const float2 c2 = make_float2(c[k], c[k]), s2 = make_float2(sn[k], sn[k]);
                const float2 ns2 = make_float2(-sn[k], -sn[k]);
#pragma unroll
                for (int h = 0; h < HP; ++h) {
                    const float2 vp = VP[h][p], vq = VP[h][q];
                    VP[h][p] = __ffma2_rn(vq, ns2, __fmul2_rn(vp, c2));
                    VP[h][q] = __ffma2_rn(vq, c2, __fmul2_rn(vp, s2));
                }
                if constexpr (D & 1) {
                    const float vp = VL[p], vq = VL[q];
                    VL[p] = fmaf(-sn[k], vq, c[k] * vp);
                    VL[q] = fmaf(c[k], vq, sn[k] * vp);
                }
            }
        }
    }
#pragma unroll
    for (int h = 0; h < HP; ++h)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            V[2 * h][b] = VP[h][b].x;
            V[2 * h + 1][b] = VP[h][b].y;
        }
    if constexpr (D & 1) {
#pragma unroll
        for (int b = 0; b < D; ++b) V[D - 1][b] = VL[b];
    }
}

// ---------------------------------------------------------------- detector tile
// One output tile (tile_x, tile_y) of height th; any block size that is a multiple of 32
// and at most 512 gives the same results (every reduction has a fixed order).
// tm (nullable, D = 4): the cube's tensor map for this window's halo box; interior tiles then
// take their halo by one tensor copy (load_halo_tma, mbarrier `bar`), the others as before.
template <int D>
__device__ void detect_tile(const DetectArgs& a, int th, int tile_x, int tile_y, unsigned char* smem_raw,
                            const CUtensorMap* tm = nullptr, uint64_t* bar = nullptr) {
    using P = SpecPayload<D>;
    constexpr int NC = P::NC;
    const TileGeom g(a.H, a.W, a.inner, a.outer, th, tile_x, tile_y);
    float* xs = reinterpret_cast<float*>(smem_raw);
    const int xs_bytes = (g.HR * g.XP * P::DP * 4 + 15) & ~15;
    float* Vo = reinterpret_cast<float*>(smem_raw + xs_bytes);
    float* Vi = Vo + NC * th * g.VP;
    float* cref = Vi + NC * th * g.VPI;  // [8]
    bool interior = false;
    if constexpr (D == 4) {
        const int y0 = g.ty0 - g.ro, x0 = g.tx0 - g.ro;
        interior = tm != nullptr && (tc::smem_u32(xs) & 127u) == 0 && y0 >= 0 && y0 + g.HR <= g.H && x0 >= 0 &&
                   x0 + g.WR <= g.W;
    }
    if (interior) {
        if (!load_halo_tma(g, tm, xs, cref, bar)) {  // the copy never landed: no scores from this tile
            for (int pix = threadIdx.x; pix < th * TW; pix += blockDim.x) {
                const int y = g.ty0 + pix / TW, xq = g.tx0 + pix % TW;
                if (y >= a.H || xq >= a.W) continue;
#pragma unroll
                for (int t = 0; t < 3; ++t)
                    if (a.out[t]) a.out[t][(size_t)y * a.W + xq] = __int_as_float(0x7fc00000);
            }
            return;
        }
    } else {
        load_halo_spec<D>(g, a.x, xs, cref);
    }
    __syncthreads();
    tile_sums<P>(g, xs, Vo, Vi);

    // stage 4, one pixel per thread and step
    const int N = (2 * g.ro + 1) * (2 * g.ro + 1) - (2 * g.ri + 1) * (2 * g.ri + 1);
    const int ni = (2 * g.ri + 1) * (2 * g.ri + 1);
    const float invN = 1.0f / (float)N, invni = 1.0f / (float)ni;
    for (int pix = threadIdx.x; pix < th * TW; pix += blockDim.x) {
        const int i = pix / TW, j = pix - i * TW;
        const int y = g.ty0 + i, xq = g.tx0 + j;
        if (y >= a.H || xq >= a.W) continue;
        const size_t o = (size_t)y * a.W + xq;
        if (a.border == 1 && (y - g.ro < 0 || y + g.ro >= a.H || xq - g.ro < 0 || xq + g.ro >= a.W)) {
#pragma unroll
            for (int t = 0; t < 3; ++t)
                if (a.out[t]) a.out[t][o] = __int_as_float(0x7fc00000);
            if (a.flags) a.flags[o] = 4;
            continue;
        }
        float So[NC], Si[NC];
        {
            const float* po = Vo + i * g.VP + j;
            const float* pi = Vi + i * g.VPI + j;
            const int plo = th * g.VP, pli = th * g.VPI;
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                So[q] = po[q * plo];
                Si[q] = pi[q * pli];
            }
        }
        float mo[D], mi[D], Co[D][D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            mo[k] = (So[k] - Si[k]) * invN;
            mi[k] = Si[k] * invni;
        }
        {
            int q = D;
#pragma unroll
            for (int u = 0; u < D; ++u)
#pragma unroll
                for (int v = u; v < D; ++v) {
                    const float cov = fmaf(-mo[u], mo[v], (So[q] - Si[q]) * invN);
                    Co[u][v] = cov; Co[v][u] = cov;
                    ++q;
                }
        }
        uint8_t flag = 0;
        if (a.out[0] || a.out[1]) {
            float tr = 0.f, smax = 0.f;
            {
                int q = D;
#pragma unroll
                for (int u = 0; u < D; ++u) {
                    tr += Co[u][u];
                    smax = fmaxf(smax, (So[q] - Si[q]) * invN);  // uncentred second moment of the shifted data
                    q += D - u;
                }
            }
            const float delta = a.loading * tr / (float)D;
            float G[D][D];
#pragma unroll
            for (int u = 0; u < D; ++u)
#pragma unroll
                for (int v = 0; v < D; ++v) G[u][v] = Co[u][v] + ((u == v) ? delta : 0.f);
            const bool ok = chol_inplace<D>(G, 16.f * FLT_EPSILON * smax);
            if (!ok) flag |= 2;
            if (a.out[0]) {
                const float* rc = xs + ((size_t)(i + g.ro) * g.XP + (j + g.ro)) * P::DP;  // shifted centre pixel
                float d[D];
#pragma unroll
                for (int k = 0; k < D; ++k) d[k] = rc[k] - mo[k];
                a.out[0][o] = ok ? chol_quad<D>(G, d) : __int_as_float(0x7fc00000);
            }
            if (a.out[1]) {
                float d[D];
#pragma unroll
                for (int k = 0; k < D; ++k) d[k] = mi[k] - mo[k];
                a.out[1][o] = ok ? fabsf(chol_quad<D>(G, d)) : __int_as_float(0x7fc00000);
            }
        }
        if (a.out[2]) {
            float Cd[D][D], V[D][D];
            {
                int q = D;
#pragma unroll
                for (int u = 0; u < D; ++u)
#pragma unroll
                    for (int v = u; v < D; ++v) {
                        const float ci = fmaf(-mi[u], mi[v], Si[q] * invni);
                        Cd[u][v] = ci - Co[u][v];  // Eq. 2
                        Cd[v][u] = Cd[u][v];
                        ++q;
                    }
            }
            jacobi_inplace<D>(Cd, V);
            float lmax = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) lmax = fmaxf(lmax, fabsf(Cd[k][k]));
            const float tau = a.dwest_tau * lmax;
            float acc = 0.f, acc2 = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                if (!(Cd[k][k] > tau)) continue;
                float best = -1.f, sg = 1.f, proj = 0.f;
#pragma unroll
                for (int u = 0; u < D; ++u) {
                    const float v = V[u][k];
                    if (fabsf(v) > best) { best = fabsf(v); sg = (v >= 0.f) ? 1.f : -1.f; }
                    proj = fmaf(v, mi[u] - mo[u], proj);  // v^T m_diff (Eq. 3, 4)
                }
                acc = fmaf(sg, proj, acc);
                acc2 = fmaf(proj, proj, acc2);
            }
            a.out[2][o] = (a.dwest_mode == 0) ? fabsf(acc) : sqrtf(acc2);
        }
        if (a.flags) a.flags[o] = flag;
    }
}

// The census tile: stages 0-2 with linear pixel indices as the payload (channels 1, q, q^2),
// out[p][6] = background count, sum, sum of squares, then the inner ones.
__device__ __forceinline__ void census_tile(int H, int W, int inner, int outer, int border, int th, int tile_x,
                                            int tile_y, long long* __restrict__ out, unsigned char* smem_raw) {
    using P = CensusPayload;
    const TileGeom g(H, W, inner, outer, th, tile_x, tile_y);
    long long* xs = reinterpret_cast<long long*>(smem_raw);
    const size_t xs_bytes = ((size_t)g.HR * g.XP * P::WORDS * 4 + 15) & ~(size_t)15;
    long long* Vo = reinterpret_cast<long long*>(smem_raw + xs_bytes);
    long long* Vi = Vo + (size_t)P::NC * th * g.VP;
    load_halo_census(g, xs);
    __syncthreads();
    tile_sums<P>(g, xs, Vo, Vi);
    for (int pix = threadIdx.x; pix < th * TW; pix += blockDim.x) {
        const int i = pix / TW, j = pix - i * TW;
        const int y = g.ty0 + i, xq = g.tx0 + j;
        if (y >= H || xq >= W) continue;
        long long* o = out + ((size_t)y * W + xq) * 6;
        if (border == 1 && (y - g.ro < 0 || y + g.ro >= H || xq - g.ro < 0 || xq + g.ro >= W)) {
            for (int t = 0; t < 6; ++t) o[t] = -1;
            continue;
        }
        long long So[3], Si[3];
        for (int q = 0; q < 3; ++q) {
            So[q] = Vo[(q * th + i) * g.VP + j];
            Si[q] = Vi[(q * th + i) * g.VPI + j];
        }
        o[0] = So[0] - Si[0]; o[1] = So[1] - Si[1]; o[2] = So[2] - Si[2];
        o[3] = Si[0]; o[4] = Si[1]; o[5] = Si[2];
    }
}

}  // namespace wdad
