// A2-A5 on few bands (dim D <= 8, the DWT approximation matrix of Sec. 4):
// dual-window statistics, regularised solve and eigen-decomposition, fused in
// one kernel per output tile.
//
//  stage 0  the tile plus a halo of outer/2 pixels is loaded into shared memory,
//           every index reflected at the image border (reflect-101);
//  stage 1  (float payload) a tile reference spectrum c = mean of the loaded
//           pixels is subtracted, so the second moments below are sums of
//           (x - c)(x - c)^T with little cancellation;
//  stage 2  horizontal box sums over the outer and the inner window width of the
//           D first-order and D(D+1)/2 second-order channels: one thread per halo
//           row and 8-column segment, a direct sum for the first column and a
//           sliding update (add the entering, subtract the leaving column) after;
//  stage 3  vertical box sums of those, one thread per (channel, column) sliding
//           down the tile rows, written in place over the horizontal sums: sums
//           over the outer square and over the inner square; the background
//           annulus is outer minus inner (Sec. 2.2 dual window);
//  stage 4  per pixel: mu_o, C_o (1/N), mu_i, C_i (1/n_i); LRX (Eq. 1) and DWRX
//           (Eq. 5) through a Cholesky factor of C_o + delta I, delta =
//           loading * trace(C_o) / D; DWEST (Eq. 2-4) through a cyclic Jacobi
//           eigen-decomposition of C_i - C_o.
//
// Stages 0, 2 and 3 are templated on the payload so that the window census
// (integer pixel indices instead of spectra) runs exactly the indexing code of
// the detectors and can be checked bit for bit.
#pragma once
#include <float.h>

#include "internal.h"

namespace wdad {


constexpr int TW = 32;          // tile width = one warp across
constexpr int kMaxSmem = 227 * 1024;

constexpr int SEG = 8;          // output columns per stage-2 thread
constexpr int HP = TW + 1;      // row pitch of the sum planes (words): conflict-free column access

__host__ __device__ __forceinline__ int halo_pitch(int WR) { return WR | 1; }  // odd pixel pitch

struct TileGeom {
    int H, W, ro, ri, th;        // image, radii, tile height
    int ty0, tx0;                // tile origin
    int HR, WR, XP;              // halo region rows / cols, halo row pitch in pixels
    int nin;                     // halo rows that carry inner sums
    __device__ TileGeom(int H_, int W_, int inner, int outer, int th_, int tile_x, int tile_y)
        : H(H_), W(W_), ro(outer / 2), ri(inner / 2), th(th_) {
        ty0 = tile_y * th;
        tx0 = tile_x * TW;
        HR = th + 2 * ro;
        WR = TW + 2 * ro;
        XP = halo_pitch(WR);
        nin = th + 2 * ri;
    }
};

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
};

struct CensusPayload {                        // linear pixel index, int64
    using T = long long;
    static constexpr int NC = 3;                 // 1, q, q^2
    static constexpr int WORDS = 2;
};

// ---------------------------------------------------------------- stage 0: reflected halo load
template <int D>
__device__ __forceinline__ void load_halo_spec(const TileGeom& g, const float* __restrict__ x, float* xs) {
    using P = SpecPayload<D>;
    const int n = g.HR * g.WR;
    if constexpr (D == 4) {
        // eight 16-byte loads in flight per thread before any is stored
        constexpr int B = 8;
        for (int base = threadIdx.x; base < n; base += B * blockDim.x) {
            float4 v[B];
            int dsti[B];
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int idx = base + u * blockDim.x;
                dsti[u] = -1;
                v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (idx < n) {
                    const int r = idx / g.WR, c = idx - r * g.WR;
                    const int gy = reflect101(g.ty0 - g.ro + r, g.H);
                    const int gx = reflect101(g.tx0 - g.ro + c, g.W);
                    v[u] = __ldg(reinterpret_cast<const float4*>(x + ((size_t)gy * g.W + gx) * 4));
                    dsti[u] = r * g.XP + c;
                }
            }
#pragma unroll
            for (int u = 0; u < B; ++u)
                if (dsti[u] >= 0) {
                    *reinterpret_cast<float4*>(xs + (size_t)dsti[u] * P::DP) = v[u];
                }
        }
    } else {
        for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
            const int r = idx / g.WR, c = idx - r * g.WR;
            const int gy = reflect101(g.ty0 - g.ro + r, g.H);
            const int gx = reflect101(g.tx0 - g.ro + c, g.W);
            const float* src = x + ((size_t)gy * g.W + gx) * D;
            float* dst = xs + ((size_t)r * g.XP + c) * P::DP;
#pragma unroll
            for (int k = 0; k < D; ++k) dst[k] = __ldg(src + k);
        }
    }
}

__device__ __forceinline__ void load_halo_census(const TileGeom& g, long long* xs) {
    const int n = g.HR * g.WR;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
        const int r = idx / g.WR, c = idx - r * g.WR;
        const int gy = reflect101(g.ty0 - g.ro + r, g.H);
        const int gx = reflect101(g.tx0 - g.ro + c, g.W);
        xs[(size_t)r * g.XP + c] = (long long)gy * g.W + gx;
    }
}

// ---------------------------------------------------------------- stage 2: horizontal sums
// hso[ch][r][j] = sum over the outer width of channel ch at halo row r, output column j;
// hsi[ch][r'][j] = the same over the inner width for the th + 2 ri halo rows the inner
// squares use (r' = r - (ro - ri)).  Thread (r, seg) owns SEG consecutive output columns
// of one halo row: a direct sum for the first, then sliding updates.
template <class P, int Q0, int Q1, class ChanFn>
__device__ __forceinline__ void horizontal_sums_part(const TileGeom& g, ChanFn chan, typename P::T* hso,
                                                     typename P::T* hsi, int t) {
    using T = typename P::T;
    constexpr int NC = P::NC;
    constexpr int NQ = Q1 - Q0;
    const int wo = 2 * g.ro + 1, i0 = g.ro - g.ri, i1 = g.ro + g.ri;  // inner columns dc in [i0, i1]
    const int rin0 = g.ro - g.ri;
    const int plane_o = g.HR * HP, plane_i = g.nin * HP;
    const int r = t % g.HR, j0 = (t / g.HR) * SEG;
    const bool inner_row = (r >= rin0) && (r < rin0 + g.nin);
    T so[NQ], si[NQ], ch[NC], c2[NC];
#pragma unroll
    for (int q = 0; q < NQ; ++q) { so[q] = T(0); si[q] = T(0); }
    for (int dc = 0; dc < wo; ++dc) {
        chan(r, j0 + dc, ch);
#pragma unroll
        for (int q = 0; q < NQ; ++q) so[q] += ch[Q0 + q];
        if (inner_row && dc >= i0 && dc <= i1) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) si[q] += ch[Q0 + q];
        }
    }
    T* po = hso + Q0 * plane_o + r * HP + j0;
    T* pi = hsi + Q0 * plane_i + (r - rin0) * HP + j0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) po[q * plane_o] = so[q];
    if (inner_row) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) pi[q * plane_i] = si[q];
    }
    for (int jj = 1; jj < SEG; ++jj) {
        const int j = j0 + jj;
        chan(r, j + wo - 1, ch);  // entering column
        chan(r, j - 1, c2);       // leaving column
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            so[q] += ch[Q0 + q] - c2[Q0 + q];  // one rounding at the running-sum magnitude
            po[q * plane_o + jj] = so[q];
        }
        if (inner_row) {
            chan(r, j + i1, ch);
            chan(r, j - 1 + i0, c2);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                si[q] += ch[Q0 + q] - c2[Q0 + q];
                pi[q * plane_i + jj] = si[q];
            }
        }
    }
}

// hso[ch][r][j] = sum over the outer width of channel ch at halo row r, output column j;
// hsi[ch][r'][j] = the same over the inner width for the th + 2 ri halo rows the inner
// squares use (r' = r - (ro - ri)).  Work item (r, seg, half) owns SEG consecutive output
// columns of one halo row and one half of the channels: a direct sum for the first
// column, then sliding updates.  The channel halves run in different warps.
template <class P, class ChanFn>
__device__ __forceinline__ void horizontal_sums(const TileGeom& g, ChanFn chan, typename P::T* hso,
                                                typename P::T* hsi) {
    constexpr int NC = P::NC;
    constexpr int NH = NC / 2;
    const int nwork = g.HR * (TW / SEG);
    const int nwork_pad = (nwork + 31) & ~31;  // each half starts on a warp boundary
    for (int t = threadIdx.x; t < 2 * nwork_pad; t += blockDim.x) {
        const int half = t >= nwork_pad;
        const int u = t - half * nwork_pad;
        if (u >= nwork) continue;
        if (half == 0) horizontal_sums_part<P, 0, NH>(g, chan, hso, hsi, u);
        else horizontal_sums_part<P, NH, NC>(g, chan, hso, hsi, u);
    }
}

// ---------------------------------------------------------------- stage 3: vertical sums, in place
// Thread (ch, j) slides down the tile rows: afterwards hso[ch][i][j] holds the sum over
// the outer square of output pixel (i, j) and hsi[ch][i][j] the sum over its inner square.
template <class P>
__device__ __forceinline__ void vertical_sums_inplace(const TileGeom& g, typename P::T* hso, typename P::T* hsi) {
    using T = typename P::T;
    constexpr int NC = P::NC;
    const int wo = 2 * g.ro + 1, wi = 2 * g.ri + 1;
    const int plane_o = g.HR * HP, plane_i = g.nin * HP;
    for (int t = threadIdx.x; t < NC * TW; t += blockDim.x) {
        const int j = t % TW, q = t / TW;
        T* ho = hso + q * plane_o + j;
        T* hi = hsi + q * plane_i + j;
        T so = T(0), si = T(0);
        for (int dr = 0; dr < wi; ++dr) { so += ho[dr * HP]; si += hi[dr * HP]; }
        for (int dr = wi; dr < wo; ++dr) so += ho[dr * HP];
        for (int i = 1; i < g.th; ++i) {
            const T lo = ho[(i - 1) * HP], eo = ho[(i + wo - 1) * HP];
            const T li = hi[(i - 1) * HP], ei = hi[(i + wi - 1) * HP];
            ho[(i - 1) * HP] = so;
            hi[(i - 1) * HP] = si;
            so += eo - lo;  // one rounding at the running-sum magnitude
            si += ei - li;
        }
        ho[(g.th - 1) * HP] = so;
        hi[(g.th - 1) * HP] = si;
    }
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
    float fro = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) fro = fmaf(A[a][b], A[a][b], fro);
    if (!(fro > 0.f)) return;  // zero matrix: already diagonal (NaN input stays NaN)
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
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    const float vp = V[a][p], vq = V[a][q];
                    V[a][p] = c[k] * vp - sn[k] * vq;
                    V[a][q] = sn[k] * vp + c[k] * vq;
                }
            }
        }
    }
}

// ---------------------------------------------------------------- detector kernel
// One output tile (tile_x, tile_y) of height th; any block size that is a multiple of 32
// and at most 512 gives the same results (every reduction has a fixed order).
template <int D>
__device__ void detect_tile(const DetectArgs& a, int th, int tile_x, int tile_y, unsigned char* smem_raw) {
    using P = SpecPayload<D>;
    constexpr int NC = P::NC;
    const TileGeom g(a.H, a.W, a.inner, a.outer, th, tile_x, tile_y);
    float* xs = reinterpret_cast<float*>(smem_raw);
    float* hso = xs + (size_t)g.HR * g.XP * P::DP;
    float* hsi = hso + (size_t)NC * g.HR * HP;
    // tile reference after the inner sums (in the dynamic buffer, not static shared memory,
    // so that a kernel holding several instantiations keeps its static size small)
    float* cref = hsi + (size_t)NC * g.nin * HP;  // [8]

    // stage 0 + tile reference: the mean of the middle halo row (a tile row), summed by warp 0
    // in a fixed order whatever the block size.  Any value near the tile's data serves: the
    // shift only keeps the second-moment sums from cancelling.
    load_halo_spec<D>(g, a.x, xs);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (warp == 0) {
        float acc[D];
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] = 0.f;
        const int r = g.HR / 2;
        for (int c = lane; c < g.WR; c += 32) {
            const float* px = xs + ((size_t)r * g.XP + c) * P::DP;
#pragma unroll
            for (int k = 0; k < D; ++k) acc[k] += px[k];
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
            float t = acc[k];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) cref[k] = t / (float)g.WR;
        }
    }
    __syncthreads();
    // stage 1: shift in place
    {
        float c[D];
#pragma unroll
        for (int k = 0; k < D; ++k) c[k] = cref[k];
        const int n = g.HR * g.WR;
        for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
            const int r = idx / g.WR, cc = idx - r * g.WR;
            float* v = xs + ((size_t)r * g.XP + cc) * P::DP;
#pragma unroll
            for (int k = 0; k < D; ++k) v[k] -= c[k];
        }
    }
    __syncthreads();
    // stage 2
    auto chan = [&](int r, int col, float (&ch)[NC]) {
        const float* v = xs + ((size_t)r * g.XP + col) * P::DP;
        float t[D];
        if constexpr (D == 4) {
            const float4 q = *reinterpret_cast<const float4*>(v);
            t[0] = q.x; t[1] = q.y; t[2] = q.z; t[3] = q.w;
        } else {
#pragma unroll
            for (int k = 0; k < D; ++k) t[k] = v[k];
        }
        P::channels(t, ch);
    };
    horizontal_sums<P>(g, chan, hso, hsi);
    __syncthreads();
    vertical_sums_inplace<P>(g, hso, hsi);
    __syncthreads();

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
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            So[q] = hso[q * g.HR * HP + i * HP + j];
            Si[q] = hsi[q * g.nin * HP + i * HP + j];
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

}  // namespace wdad
