// Batched launch of many reduced-path jobs (host and device shared declarations).
#pragma once
#include <vector>

#include "internal.h"

namespace wdad {

struct BatchJob {
    const float* cube;   // [H][W][L]
    float* approx;       // [H][W][K] batch-owned
    const float* A;      // K x L DWT matrix (handle plan cache)
    float* out[3];       // score maps (nullptr = not wanted)
    uint8_t* flags;
    int H, W, L, K;
    int inner, outer, border, dwest_mode;
    float loading, tau;
    int th;              // tile height of the detector plan
    int variant;         // DWT register layout: 0 = L <= 128, 1 = L <= 256
    int dwt_items;       // number of DWT items the job's tiles wait for
};

struct BatchItem {
    int job;
    int kind;  // 0 = DWT 4-pixel groups [a, b), 1 = detector tile (a, b) = (tile_x, tile_y)
    int a, b;
};

bool batch_job_supported(int L, int K);
int batch_variant(int L);
// shared memory a DWT item needs (the job's DWT matrix, zero-padded rows)
size_t batch_dwt_smem(int L);
// drop_job >= 0 removes that job's first DWT item from the list (host-side fault injection
// for tests of the bounded wait); -1 in normal use.  lag: items placed between a job's last
// DWT item and its first tile (when DWT items remain to fill the gap).
void batch_build_items(const std::vector<BatchJob>& jobs, std::vector<BatchItem>& items, std::vector<int>& dwt_items,
                       int drop_job, int lag);
cudaError_t batch_launch(const BatchJob* d_jobs, const BatchItem* d_items, int nitems, int* d_counters, int njobs,
                         size_t smem, int num_sms, cudaStream_t s);

}  // namespace wdad
