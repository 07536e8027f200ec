// Host-side declarations of the CNN screener (A9); kernels in cnn.cu.
#pragma once
#include <cuda_bf16.h>

#include "internal.h"

namespace wdad {
namespace cnn {

constexpr int WHITEN_BLOCKS = 256;  // fixed partition of the scene-moment reduction
constexpr int WHITEN_NQ_MAX = 8 + 36;

struct Net {
    int K = 4;             // input channels (DWT approximation coefficients)
    int bf16 = 1;          // forward with BF16-rounded weights
    size_t woff[4], boff[4], nparam = 0;
    int step = 0;          // Adam step counter
    int64_t max_px = 0;    // largest B * H * W of a training call
    float *w = nullptr, *wf = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    float* wt = nullptr;   // flipped/transposed weights of one layer
    int norm_mode = 0;     // 0: whiten each scene with its own statistics; 1: fixed map (set_norm)
    float* norm = nullptr; // [K + K*K] input map z = M (x - mu): mu, then M row-major
    double* stat = nullptr;  // WHITEN_BLOCKS x WHITEN_NQ_MAX partial moments
    float* act = nullptr;  // activations and gradients of one training batch
    float* loss = nullptr; // device scalar
    float *cx = nullptr, *ct = nullptr;  // crop buffers
    __nv_bfloat16* wpk = nullptr;  // the two 32 -> 32 layers' weights packed for the tensor cores
    int* tcerr = nullptr;          // set by a tensor-core convolution that gave up waiting
    float* gpart = nullptr;        // per-chunk partial weight and bias gradients (gpart_floats())
};

// pixel chunks of the gradient reductions: at least 256 pixels each, at most 64 chunks
constexpr int GRAD_MAX_CHUNKS = 64;
inline size_t gpart_floats() { return (size_t)GRAD_MAX_CHUNKS * 32 * 25 * 32; }

void layer_dims(int K, int l, int* cin, int* cout, int* k);
void param_layout(int K, size_t woff[4], size_t boff[4], size_t* total);
inline size_t act_floats(int64_t px) { return (size_t)px * (32 * 5 + 2); }

cudaError_t conv_fwd(const float* in, int B, int H, int W, int Cin, const float* w, const float* bias, int Cout, int k,
                     int relu, const float* norm, float* out, cudaStream_t s);
// tc: the 32 -> 32 layers on the tensor cores (bfloat16 activations; inference of networks
// with bfloat16 weights); otherwise all layers in float32 SIMT
cudaError_t net_forward(const Net& n, const float* x, int B, int H, int W, const float* norm, float* a0, float* a1,
                        float* a2, float* out, cudaStream_t s, bool tc = false, int num_sms = 0);
cudaError_t pack_w5(const float* w, __nv_bfloat16* packed, cudaStream_t s);
cudaError_t conv5_tc(const float* in, int B, int H, int W, const __nv_bfloat16* wpk, const float* bias, int relu,
                     float* out, int* err, int num_sms, cudaStream_t s);
cudaError_t net_grad(Net& n, const float* x, const float* t, int B, int H, int W, cudaStream_t s);
cudaError_t net_adam(Net& n, float lr, cudaStream_t s);
cudaError_t net_init(Net& n, uint64_t seed, cudaStream_t s);
cudaError_t net_refresh_forward_copy(Net& n, cudaStream_t s);
// norm = [mu, M] of the scene whitening of x [P][K] (two launches on s, deterministic)
cudaError_t scene_whitening(const float* x, int64_t P, int K, double* part, float* norm, cudaStream_t s);
cudaError_t sample_crops(const Net& n, const float* approx, const float* score, int H, int W, int B, int Hc, int Wc,
                         uint64_t seed, uint64_t step, float* x, float* t, cudaStream_t s);
cudaError_t top_threshold(const float* v, int64_t n, int64_t kth, unsigned int* hist, uint32_t* thr, cudaStream_t s);
cudaError_t select_pixels(const float* v, int64_t n, uint32_t thr, float audit_frac, uint64_t seed, uint8_t* sel,
                          int64_t* list, unsigned long long* cnt, cudaStream_t s);
cudaError_t fill(float* v, int64_t n, float val, cudaStream_t s);
cudaError_t scatter_list(const float* src, const int64_t* list, int64_t n, float* dst, cudaStream_t s);

}  // namespace cnn
}  // namespace wdad
