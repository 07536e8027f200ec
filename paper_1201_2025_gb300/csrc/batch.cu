// A8 — many cubes of uneven size, band count, window and detector in one persistent
// launch (captured once into a CUDA graph and replayed).
//
// The host builds a work list of DWT items (ranges of 4-pixel groups of one cube) and
// detector tiles: the two streams are merged in proportion to their lengths, so that
// HBM-bound DWT items and ALU-bound tiles run side by side on each SM (two 512-thread CTAs
// per SM when the largest tile plan fits), and every tile of cube j is placed after all DWT
// items of cube j plus a lag of about four times the grid's CTAs.  Persistent CTAs pop items
// with one atomic counter.  A tile of cube j may only start once all DWT items of cube j have
// finished: the DWT items bump done[j] after a fence, and the tile's first thread waits for
// done[j] == dwt_items[j] with a bounded spin.  Items are popped in list order and every DWT
// item of cube j precedes every tile of cube j, so each DWT item a tile waits on is already
// held by a running CTA that will finish it (DWT items never wait); if the spin still runs out
// (about a second), the tile is skipped and the launch status becomes WDAD_ERR_TIMEOUT instead
// of hanging.  The per-item arithmetic gives
// the same bits as the standalone kernels with the same tile plan (the DWT reads its matrix
// from shared memory but sums in the same order), so a batched job's scores are
// bit-identical to the same job run alone.
#include <cstdlib>

#include "batch.h"
#include "dwt_dev.cuh"
#include "tc.cuh"
#include "reduced_dev.cuh"

namespace wdad {

constexpr int BATCH_THREADS = 512;
constexpr int kGroupsPerDwtItem = 512;  // 4-pixel groups: 2048 pixels per DWT item
constexpr int kChunkPx = 32;            // pixels per staged chunk of a DWT item
constexpr int kStages = 3;              // chunks in flight per CTA
constexpr int kStageFloats = kChunkPx * 256;  // stage stride (L <= 256)
constexpr uint32_t kStageWait = 1u << 24;     // polls before a staged chunk counts as lost

// Staged-chunk copy of DWT item chunk q (pixels [p0 + q kChunkPx, ...)) into stage s.
__device__ __forceinline__ void issue_chunk(const BatchJob& j, int64_t p0, int64_t npx_total, int q, int s,
                                            float* stages, uint64_t* full) {
    const int64_t first = p0 + (int64_t)q * kChunkPx;
    const int64_t n = min((int64_t)kChunkPx, npx_total - (int64_t)q * kChunkPx);
    const uint32_t bytes = (uint32_t)(n * j.L * (int64_t)sizeof(float));
    tc::mbar_arrive_expect_tx(&full[s], bytes);
    tc::bulk_g2s(stages + (size_t)s * kStageFloats, j.cube + first * j.L, bytes, &full[s]);
}

__global__ void __launch_bounds__(BATCH_THREADS, 2)
    batch_kernel(const BatchJob* __restrict__ jobs, const BatchItem* __restrict__ items, int nitems, int* counter,
                 int* done, int* status, uint32_t spin_limit) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ int s_ready;
    __shared__ int s_ok;
    __shared__ __align__(8) uint64_t s_full[kStages];
    // the tile's arguments live in shared memory (a kernel parameter in the standalone
    // kernel), which keeps them out of the 64 registers a thread has at two CTAs per SM
    __shared__ DetectArgs s_args;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) tc::mbar_init(&s_full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t gchunk = 0;  // staged chunks this CTA has consumed (stage = g % kStages, parity = g / kStages)
    int ready_job = -1;   // job whose DWT this CTA has seen finished and whose arguments s_args holds
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const BatchItem bi = items[it];
        const BatchJob& j = jobs[bi.job];
        if (bi.kind == 0) {
            // DWT item: its pixels stream through kStages shared-memory stages by bulk copies
            // (one thread issues, mbarriers count the bytes); the lanes keep their slice of the
            // DWT matrix in registers
            const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
            const int64_t P = (int64_t)j.H * j.W;
            const int64_t p0 = 4 * (int64_t)bi.a, p1 = min(P, 4 * (int64_t)bi.b);
            const int64_t npx_total = p1 - p0;
            const int nchunk = (int)((npx_total + kChunkPx - 1) / kChunkPx);
            float* stages = reinterpret_cast<float*>(smem_raw);
            const int LV = j.L / 4;
            float a[2][4][4];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int c = lane + 32 * i;
                        a[i][k][e] = (c < LV && k < j.K) ? __ldg(j.A + (size_t)k * j.L + c * 4 + e) : 0.0f;
                    }
            if (threadIdx.x == 0) {
                tc::fence_proxy_async_smem();  // earlier generic accesses of the stages come first
                for (int q = 0; q < min(kStages, nchunk); ++q)
                    issue_chunk(j, p0, npx_total, q, (int)((gchunk + q) % kStages), stages, s_full);
            }
            int ok = 1;
            int q = 0;
            for (; q < nchunk; ++q) {
                const uint32_t g = gchunk + (uint32_t)q;
                const int s = (int)(g % kStages);
                if (threadIdx.x == 0) s_ok = tc::mbar_wait_bounded(&s_full[s], (g / kStages) & 1u, kStageWait) ? 1 : 0;
                __syncthreads();
                ok = s_ok;
                if (!ok) break;
                const int npx = (int)min((int64_t)kChunkPx, npx_total - (int64_t)q * kChunkPx);
                float* out = j.approx + (size_t)(p0 + (int64_t)q * kChunkPx) * j.K;
                if (j.variant == 0) {
                    const float(&a1)[1][4][4] = *reinterpret_cast<const float(*)[1][4][4]>(&a[0]);
                    dwt_staged_pairs<1>(stages + (size_t)s * kStageFloats, npx, j.L, a1, j.K, out, warp, nw);
                } else {
                    dwt_staged_pairs<2>(stages + (size_t)s * kStageFloats, npx, j.L, a, j.K, out, warp, nw);
                }
                __syncthreads();  // the stage is free again
                if (threadIdx.x == 0 && q + kStages < nchunk) {
                    tc::fence_proxy_async_smem();
                    issue_chunk(j, p0, npx_total, q + kStages, s, stages, s_full);
                }
            }
            if (!ok) {
                // a staged chunk never arrived: report it, let the copies in flight land (with a
                // longer bound), stop.  If one of those copies does not land either, the CTA
                // cannot know when it will write its shared memory: that is reported as
                // WDAD_ERR_CUDA, a state the host must not reuse (destroy the batch, reset the
                // context).
                if (threadIdx.x == 0) {
                    int drained = 1;
                    for (int r = q + 1; r < min(nchunk, q + kStages); ++r) {
                        const uint32_t g = gchunk + (uint32_t)r;
                        drained &= tc::mbar_wait_bounded(&s_full[g % kStages], (g / kStages) & 1u, 16u * kStageWait)
                                       ? 1 : 0;
                    }
                    atomicExch(&status[0], drained ? (int)WDAD_ERR_TIMEOUT : (int)WDAD_ERR_CUDA);
                }
                __syncthreads();
                return;
            }
            gchunk += (uint32_t)nchunk;
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&done[bi.job], 1);
            }
        } else {
            // the first tile of a job this CTA meets waits (bounded) for the job's DWT items and
            // loads the job's arguments; later tiles of the same job reuse both
            if (bi.job != ready_job) {
                if (threadIdx.x == 0) {
                    uint32_t n = 0;
                    int ok = 1;
                    while (atomicAdd(&done[bi.job], 0) < j.dwt_items) {
                        if (atomicAdd(&status[1 + bi.job], 0) != 0 || ++n > spin_limit) {
                            ok = 0;
                            atomicExch(&status[1 + bi.job], 1);
                            atomicExch(&status[0], (int)WDAD_ERR_TIMEOUT);
                            break;
                        }
                        __nanosleep(256);
                    }
                    __threadfence();
                    s_ready = ok;
                    DetectArgs& a = s_args;
                    a.x = j.approx; a.H = j.H; a.W = j.W; a.D = j.K;
                    a.inner = j.inner; a.outer = j.outer; a.loading = j.loading; a.border = j.border;
                    a.dwest_mode = j.dwest_mode; a.dwest_tau = j.tau;
                    for (int t = 0; t < 3; ++t) a.out[t] = j.out[t];
                    a.flags = j.flags;
                }
                __syncthreads();
                ready_job = s_ready ? bi.job : -1;
            }
            if (ready_job == bi.job) {
                const int th = j.th;
                switch (s_args.D) {
                    case 1: detect_tile<1>(s_args, th, bi.a, bi.b, smem_raw); break;
                    case 2: detect_tile<2>(s_args, th, bi.a, bi.b, smem_raw); break;
                    case 3: detect_tile<3>(s_args, th, bi.a, bi.b, smem_raw); break;
                    default: detect_tile<4>(s_args, th, bi.a, bi.b, smem_raw); break;
                }
            }
            __syncthreads();
        }
    }
}

bool batch_job_supported(int L, int K) { return L % 4 == 0 && L <= 256 && K >= 1 && K <= 4; }

int batch_variant(int L) { return L <= 128 ? 0 : 1; }

size_t batch_dwt_smem(int L) {
    (void)L;
    return sizeof(float) * (size_t)kStages * kStageFloats;
}

void batch_build_items(const std::vector<BatchJob>& jobs, std::vector<BatchItem>& items, std::vector<int>& dwt_items,
                       int drop_job, int lag) {
    const size_t n = jobs.size();
    std::vector<BatchItem> dw, tl;
    std::vector<int64_t> left(n, 0);  // DWT items of a job not yet placed
    dwt_items.assign(n, 0);
    for (size_t j = 0; j < n; ++j) {
        const int64_t P = (int64_t)jobs[j].H * jobs[j].W;
        const int64_t ngroups = (P + 3) / 4;
        bool dropped = false;
        for (int64_t g0 = 0; g0 < ngroups; g0 += kGroupsPerDwtItem) {
            dwt_items[j]++;
            if ((int)j == drop_job && !dropped) { dropped = true; continue; }  // fault injection (host only)
            dw.push_back({(int)j, 0, (int)g0, (int)std::min<int64_t>(ngroups, g0 + kGroupsPerDwtItem)});
            left[j]++;
        }
    }
    for (size_t j = 0; j < n; ++j) {
        const int tx = (jobs[j].W + 31) / 32, ty = (jobs[j].H + jobs[j].th - 1) / jobs[j].th;
        for (int y = 0; y < ty; ++y)
            for (int x = 0; x < tx; ++x) tl.push_back({(int)j, 1, x, y});
    }
    // Merge the two streams in proportion to their lengths.  A tile of job j is placed only
    // once every DWT item of job j is in the list and `lag` further items follow the last of
    // them, so that by the time a CTA pops the tile the DWT item has most likely finished.
    std::vector<int64_t> last(n, -(int64_t)1 << 40);
    const size_t nd = dw.size(), nt = tl.size();
    size_t ia = 0, ib = 0;
    items.clear();
    items.reserve(nd + nt);
    auto put_dwt = [&]() {
        const BatchItem it = dw[ia++];
        if (--left[(size_t)it.job] == 0) last[(size_t)it.job] = (int64_t)items.size();
        items.push_back(it);
    };
    while (ia < nd || ib < nt) {
        const bool tile_turn = ib < nt && (ia >= nd || (double)ib * (double)nd <= (double)ia * (double)nt);
        if (!tile_turn) { put_dwt(); continue; }
        const size_t j = (size_t)tl[ib].job;
        const bool ready = left[j] == 0 && (int64_t)items.size() >= last[j] + lag;
        if (!ready && ia < nd) { put_dwt(); continue; }
        items.push_back(tl[ib++]);
    }
}

cudaError_t batch_launch(const BatchJob* d_jobs, const BatchItem* d_items, int nitems, int* d_counters, int njobs,
                         size_t smem, int num_sms, cudaStream_t s) {
    cudaError_t e = raise_smem_limit(batch_kernel);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, BATCH_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // counters: [0] work counter, [1, 1 + njobs) done, then status[0] and one word per job
    e = cudaMemsetAsync(d_counters, 0, sizeof(int) * (size_t)(2 + 2 * njobs), s);
    if (e != cudaSuccess) return e;
    int grid = num_sms * per_sm;
    if (grid > nitems) grid = nitems > 0 ? nitems : 1;
    batch_kernel<<<grid, BATCH_THREADS, smem, s>>>(d_jobs, d_items, nitems, d_counters, d_counters + 1,
                                                   d_counters + 1 + njobs, 4u << 20);
    return cudaGetLastError();
}

}  // namespace wdad
