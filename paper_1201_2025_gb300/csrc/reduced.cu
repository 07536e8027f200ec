// Launchers and kernels of the reduced-band detectors (device code in reduced_dev.cuh).
#include <algorithm>
#include <mutex>

#include "reduced_dev.cuh"

namespace wdad {

template <int D>
__global__ void __launch_bounds__(512) detect_small_kernel(DetectArgs a, int th) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    detect_tile<D>(a, th, blockIdx.x, blockIdx.y, smem_raw);
}

// Several windows of one cube in one launch: the CTAs of window w are blocks
// [first[w], first[w + 1]) of a 1-D grid; each copies its window's arguments to shared
// memory and runs the same tile code (whose results do not depend on the block size), so
// every window's scores equal its own launch's.  One grid leaves no tail between windows.
struct MultiArgs {
    CUtensorMap tmap[kMaxWindowsPerLaunch];  // each window's halo box over the 4-band cube (when use_tma)
    int use_tma;
    DetectArgs a[kMaxWindowsPerLaunch];
    int th[kMaxWindowsPerLaunch];
    int tiles_x[kMaxWindowsPerLaunch];
    int ty0[kMaxWindowsPerLaunch];  // first tile row of each window in this launch
    int first[kMaxWindowsPerLaunch + 1];
    int n;
};

template <int D>
__global__ void __launch_bounds__(512) detect_multi_kernel(const __grid_constant__ MultiArgs m) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ DetectArgs s_args;
    __shared__ int s_w;
    __shared__ __align__(8) uint64_t s_bar;
    if (threadIdx.x == 0) {
        if (m.use_tma) {
            tc::mbar_init(&s_bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        int w = 0;
        while (w + 1 < m.n && (int)blockIdx.x >= m.first[w + 1]) ++w;
        s_w = w;
        // compile-time indices: a runtime index into the parameter array would copy it locally
        if (w == 0) s_args = m.a[0];
        else if (w == 1) s_args = m.a[1];
        else if (w == 2) s_args = m.a[2];
        else s_args = m.a[3];
    }
    __syncthreads();
    const int w = s_w;
    const int t = (int)blockIdx.x - m.first[w];
    const int tx = m.tiles_x[w];
    detect_tile<D>(s_args, m.th[w], t % tx, m.ty0[w] + t / tx, smem_raw, m.use_tma ? &m.tmap[w] : nullptr, &s_bar);
}

// ---------------------------------------------------------------- census kernel
__global__ void __launch_bounds__(512) census_kernel(int H, int W, int inner, int outer, int border, int th,
                                                     long long* __restrict__ out) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    census_tile(H, W, inner, outer, border, th, blockIdx.x, blockIdx.y, out, smem_raw);
}

// ---------------------------------------------------------------- launchers
static int spec_nc(int D) { return D + D * (D + 1) / 2; }
static int spec_dp(int D) { return D <= 4 ? 4 : 8; }

size_t detect_small_smem(int D, int inner, int outer, int tile_h) {
    return tile_smem_bytes(spec_dp(D), spec_nc(D), 4, inner, outer, tile_h);
}

// Tallest tile (<= want, >= 8 rows) that lets two CTAs share an SM; else the tallest that
// fits one.  Two CTAs fit when each takes at most half of the SM's 228 KiB, less the 1 KiB the
// runtime reserves per CTA and 128 B for the kernels' own static shared variables.  Heights
// need not be powers of two: at window (7,21) and D = 4, 11 rows fit two CTAs where 16 do not.
constexpr size_t kTwoPerSm = 228 * 1024 / 2 - 1024 - 128;
size_t detect_small_two_per_sm_bytes() { return kTwoPerSm; }

static int pick_th(int D, int inner, int outer, int want) {
    for (int th = want; th >= 8; --th)
        if (detect_small_smem(D, inner, outer, th) <= kTwoPerSm) return th;
    for (int th = want; th >= 1; th >>= 1)
        if (detect_small_smem(D, inner, outer, th) <= (size_t)kMaxSmem) return th;
    return 0;
}

template <int D>
static cudaError_t launch_d(const DetectArgs& a, int th, cudaStream_t s) {
    const size_t smem = detect_small_smem(D, a.inner, a.outer, th);
    cudaError_t e = raise_smem_limit(detect_small_kernel<D>);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + TW - 1) / TW, (a.H + th - 1) / th);
    const int threads = std::min(512, std::max(256, th * 32));  // one thread per output pixel when th >= 8
    detect_small_kernel<D><<<grid, threads, smem, s>>>(a, th);
    return cudaGetLastError();
}

int detect_small_default_th(int D, int inner, int outer) { return pick_th(D, inner, outer, 16); }

cudaError_t launch_detect_small_th(const DetectArgs& a, int th, cudaStream_t s) {
    if ((int64_t)a.H * a.W == 0) return cudaSuccess;
    if (th < 1 || detect_small_smem(a.D, a.inner, a.outer, th) > (size_t)kMaxSmem) return cudaErrorInvalidValue;
    switch (a.D) {
        case 1: return launch_d<1>(a, th, s);
        case 2: return launch_d<2>(a, th, s);
        case 3: return launch_d<3>(a, th, s);
        case 4: return launch_d<4>(a, th, s);
        case 5: return launch_d<5>(a, th, s);
        case 6: return launch_d<6>(a, th, s);
        case 7: return launch_d<7>(a, th, s);
        case 8: return launch_d<8>(a, th, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_detect_small(const DetectArgs& a, int tile_h, cudaStream_t s) {
    if ((int64_t)a.H * a.W == 0) return cudaSuccess;
    const int th = pick_th(a.D, a.inner, a.outer, tile_h > 0 ? tile_h : 16);
    if (th == 0) return cudaErrorInvalidValue;
    switch (a.D) {
        case 1: return launch_d<1>(a, th, s);
        case 2: return launch_d<2>(a, th, s);
        case 3: return launch_d<3>(a, th, s);
        case 4: return launch_d<4>(a, th, s);
        case 5: return launch_d<5>(a, th, s);
        case 6: return launch_d<6>(a, th, s);
        case 7: return launch_d<7>(a, th, s);
        case 8: return launch_d<8>(a, th, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int D>
static cudaError_t launch_multi_d(const MultiArgs& m, size_t smem, int blocks, cudaStream_t s) {
    cudaError_t e = raise_smem_limit(detect_multi_kernel<D>);
    if (e != cudaSuccess) return e;
    detect_multi_kernel<D><<<blocks, 512, smem, s>>>(m);
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (looked up once)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// The halo box of a window over the 4-band cube x [H][W][4] as a 2-D float32 tensor (W * 4
// elements per row, H rows): HR rows of XP pixels.  False (no tensor copies) when the driver
// entry point or the encoding refuses, or the box does not fit the tensor-copy limits.
static bool encode_halo_map(CUtensorMap* m, const float* x, int H, int W, int HR, int XP) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc || (reinterpret_cast<uintptr_t>(x) & 15) || XP * 4 > 256 || HR > 256 || HR < 1 || XP < 1) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)W * 4, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)W * 4 * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)XP * 4, (cuuint32_t)HR};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(x), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_detect_small_multi(const DetectArgs* a, int n, cudaStream_t s) {
    return launch_detect_small_multi_rows(a, n, 0, a[0].H, s);
}

cudaError_t launch_detect_small_multi_rows(const DetectArgs* a, int n, int row0, int row1, cudaStream_t s) {
    if (n < 1 || n > kMaxWindowsPerLaunch || row0 < 0 || row1 < row0) return cudaErrorInvalidValue;
    MultiArgs m{};
    m.n = n;
    size_t smem = 0;
    int64_t blocks = 0;
    // the widest windows' tiles (the slowest) first, so that the grid ends on short tiles
    int order[kMaxWindowsPerLaunch];
    for (int w = 0; w < n; ++w) order[w] = w;
    std::stable_sort(order, order + n, [&](int p, int q) { return a[p].outer > a[q].outer; });
    for (int j = 0; j < n; ++j) {
        const int w = order[j];
        if (a[w].D != a[0].D || a[w].H != a[0].H || a[w].W != a[0].W || a[w].x != a[0].x)
            return cudaErrorInvalidValue;
        const int th = pick_th(a[w].D, a[w].inner, a[w].outer, 16);
        if (th == 0) return cudaErrorInvalidValue;
        m.a[j] = a[w];
        m.th[j] = th;
        m.tiles_x[j] = (a[w].W + TW - 1) / TW;
        // the tiles whose first row lies in [row0, row1)
        const int y0 = (row0 + th - 1) / th, y1 = std::min((a[w].H + th - 1) / th, (row1 + th - 1) / th);
        m.ty0[j] = y0;
        m.first[j] = (int)blocks;
        blocks += (int64_t)m.tiles_x[j] * std::max(0, y1 - y0);
        smem = std::max(smem, detect_small_smem(a[w].D, a[w].inner, a[w].outer, th));
    }
    m.first[n] = (int)blocks;
    if (blocks == 0) return cudaSuccess;
    // interior tiles take their halo by tensor copies (4-band cubes)
    m.use_tma = 0;
    if (a[0].D == 4) {
        bool ok = true;
        for (int j = 0; j < n && ok; ++j) {
            const int ro = m.a[j].outer / 2;
            ok = encode_halo_map(&m.tmap[j], m.a[j].x, m.a[j].H, m.a[j].W, m.th[j] + 2 * ro, halo_pitch(TW + 2 * ro));
        }
        m.use_tma = ok ? 1 : 0;
    }
    if (blocks > INT32_MAX) return cudaErrorInvalidValue;
    switch (a[0].D) {
        case 1: return launch_multi_d<1>(m, smem, (int)blocks, s);
        case 2: return launch_multi_d<2>(m, smem, (int)blocks, s);
        case 3: return launch_multi_d<3>(m, smem, (int)blocks, s);
        case 4: return launch_multi_d<4>(m, smem, (int)blocks, s);
        case 5: return launch_multi_d<5>(m, smem, (int)blocks, s);
        case 6: return launch_multi_d<6>(m, smem, (int)blocks, s);
        case 7: return launch_multi_d<7>(m, smem, (int)blocks, s);
        case 8: return launch_multi_d<8>(m, smem, (int)blocks, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_window_census(int H, int W, int inner, int outer, int border, int64_t* out, cudaStream_t s) {
    if ((int64_t)H * W == 0) return cudaSuccess;
    int th = 16;
    while (th > 1 && tile_smem_bytes(CensusPayload::WORDS, CensusPayload::NC, 8, inner, outer, th) > (size_t)kMaxSmem)
        th >>= 1;
    const size_t smem = tile_smem_bytes(CensusPayload::WORDS, CensusPayload::NC, 8, inner, outer, th);
    if (smem > (size_t)kMaxSmem) return cudaErrorInvalidValue;
    cudaError_t e = raise_smem_limit(census_kernel);
    if (e != cudaSuccess) return e;
    dim3 grid((W + TW - 1) / TW, (H + th - 1) / th);
    census_kernel<<<grid, th >= 16 ? 512 : 256, smem, s>>>(H, W, inner, outer, border, th,
                                                           reinterpret_cast<long long*>(out));
    return cudaGetLastError();
}

}  // namespace wdad
