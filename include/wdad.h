/*
 * wdad.h — C ABI of libwdad: wavelet-reduced local anomaly detection on one GPU.
 *
 * Method: Zare Baghbidi, Jamshidi, Naghsh Nilchi, Homayouni, "Improvement of
 * anomaly detection algorithms in hyperspectral images using discrete wavelet
 * transform", SIPIJ 2(4), 2011.  Every pixel spectrum of an H x W x L cube goes
 * through a Daubechies DWT along the band axis, only the approximation
 * coefficients are kept (Sec. 4, Eq. 7/9, Fig. 1), and the local detectors LRX
 * (Sec. 2.1, Eq. 1), DWRX (Sec. 2.3, Eq. 5) and DWEST (Sec. 2.2, Eq. 2-4) run on
 * that reduced cube or on the full-band cube.  Also: global RX (Eq. 1 with the whole
 * image as background), the adaptive cut-off of Eq. 12, batches of uneven cubes, and a
 * learned screening pass that runs the exact detector on selected pixels only.
 *
 * Conventions shared by every entry point
 *   - Cubes are float32, band-interleaved-by-pixel: element (y, x, l) sits at
 *     ((y * W) + x) * L + l.  Score maps are float32 [H][W] row-major.
 *   - All array pointers are DEVICE pointers owned by the caller unless the
 *     comment says host; the library never frees them.  Inputs are read-only.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Compute calls
 *     are asynchronous on that stream; the caller synchronises before reading
 *     outputs.  Argument errors are detected on the host before anything is
 *     enqueued and return synchronously.
 *   - Every function returns a wdad_status; no C++ exception crosses the ABI.
 *     wdad_last_error_detail() gives a one-line reason for the last failure on
 *     a handle.
 *   - A handle binds one CUDA device and owns a grow-only device workspace and
 *     plan caches.  Calls on one handle must not run concurrently from several
 *     host threads; use one handle per thread.  Each call reuses the workspace from
 *     its start, so calls on one handle that are given different streams must be
 *     ordered by the caller (an event), or use one handle per stream.
 */
#ifndef WDAD_H
#define WDAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WDAD_OK = 0,
    WDAD_ERR_ARG = 1,         /* invalid argument (checked on the host) */
    WDAD_ERR_CUDA = 2,        /* a CUDA runtime call or launch failed */
    WDAD_ERR_NOMEM = 3,       /* device workspace allocation failed */
    WDAD_ERR_NUMERIC = 4,     /* reported by status readers: non-finite result */
    WDAD_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    WDAD_ERR_UNSUPPORTED = 6  /* valid but not implemented shape or mode */
} wdad_status;

typedef enum { WDAD_LRX = 0, WDAD_DWRX = 1, WDAD_DWEST = 2 } wdad_detector;

typedef enum {
    WDAD_PREC_FP32 = 0,   /* FP32 statistics and solves */
    WDAD_PREC_MIXED = 1,  /* full band: BF16 tensor-core Gram (FP32 sample Gram for LRX/DWRX when N < L),
                             FP32 solve, FP64 re-solve above cond_gate */
    WDAD_PREC_FP64 = 2    /* full band: FP64 statistics and solves for every pixel */
} wdad_precision;

/* Detection parameters.  Fill with wdad_default_params() and override. */
typedef struct {
    int wavelet_taps;  /* Daubechies filter length, even 2..20: 8 = db4, "Daubechies4" of Sec. 4
                          (default); 4 = D4; taps/2 vanishing moments (Sec. 6 other filters) */
    int level;         /* -1 = smallest J whose approximation length is <= 4 (Sec. 4) */
    int inner, outer;  /* odd window sides, 1 <= inner < outer <= 63 (Sec. 2.2, Sec. 5.2) */
    float loading;     /* LRX/DWRX diagonal loading delta = loading * trace(C_o) / dim; default 1e-3 */
    float cond_gate;   /* MIXED: re-solve in FP64 where the estimated condition number exceeds this; 1e6 */
    int border;        /* 0 = reflect-101 (default), 1 = NaN where the outer window leaves the image */
    int dwest_mode;    /* 0 = |sum_k v_k^T m_diff| with each v_k's largest-|.| entry positive (Eq. 4);
                          1 = ||V_S^T m_diff|| (sign free) */
    int precision;     /* wdad_precision, used by the full-band path */
    float dwest_tau;   /* DWEST keeps eigenvalues > dwest_tau * max|lambda|; default 1e-6 */
} wdad_params;

typedef struct wdad_ctx* wdad_handle;

/* Defaults: taps 8, level -1, windows 3/11, loading 1e-3, cond_gate 1e6, reflect-101,
 * dwest_mode 0, FP32, dwest_tau 1e-6. */
void wdad_default_params(wdad_params* p);

/* Create a handle on CUDA device `device`.  Allocates nothing on the device yet. */
wdad_status wdad_create(wdad_handle* h, int device);
/* Release the handle and its workspace (synchronises the device first). */
wdad_status wdad_destroy(wdad_handle h);
/* Copy the last error text of `h` (NUL-terminated, truncated to len). */
wdad_status wdad_last_error_detail(wdad_handle h, char* buf, int len);

/* Number of approximation coefficients K for L bands and a level (-1 = auto, Sec. 4):
 * K = L halved (rounding up) J times.  Returns -1 for invalid input. */
int wdad_query_K(int L, int taps, int level);

/* Global RX, Eq. 1 (Sec. 2.1): score[p] = (r_p - mu)^T (C + delta I)^-1 (r_p - mu) with mu and
 * C = (1/P) sum (r - mu)(r - mu)^T over all P = H*W pixels (one background for the whole
 * image) and delta = p->loading * trace(C) / bands, the loading rule of the local detectors.
 * reduce = 0: on the L bands of cube; reduce = 1: on the K DWT approximation coefficients
 * (p->wavelet_taps, p->level), computed into the handle's workspace.  cube: device
 * [H][W][L] float32; score: device [H][W] float32.  Bands (L or K) up to 1024, otherwise
 * WDAD_ERR_UNSUPPORTED.  Mean and covariance: FP32 partial sums over fixed pixel ranges
 * combined in FP64 in a fixed order; inverse: FP32 symmetric sweep in one block.  If the
 * loaded covariance is not numerically positive definite every score is NaN.  Asynchronous
 * on `stream`; uses the handle's workspace. */
wdad_status wdad_global_rx(wdad_handle h, const float* cube, int H, int W, int L, int reduce, const wdad_params* p,
                           float* score, void* stream);

/* Host-only: the scaling filter h[0..taps-1] the DWT uses (Sec. 4; Daubechies' extremal-phase
 * construction, taps/2 vanishing moments, sum h = sqrt(2)).  taps even, 2..20; h (host, taps
 * doubles) is written on success.  WDAD_ERR_ARG for other taps or a NULL h.  No GPU needed. */
wdad_status wdad_wavelet_filter(int taps, double* h);

/* A1 — approximation matrix (Sec. 4; Eq. 9 cascaded J times, Fig. 1, details discarded).
 * cube: [H][W][L] float32; approx: [H][W][K] float32 (caller allocates H*W*K floats);
 * K_out (host, nullable) receives K.  Periodic extension, odd lengths padded by
 * repeating the last sample.  L <= 1024 when L % 4 == 0, else L <= 256. */
wdad_status wdad_dwt_approx(wdad_handle h, const float* cube, int H, int W, int L,
                            const wdad_params* p, float* approx, int* K_out, void* stream);

/* A2-A6 — one detector on every pixel (Sec. 2, Eq. 1-5).
 * reduce = 1: DWT-reduced path (A1 into the handle's workspace, then the detector
 * on K bands — "DWT-LRX/DWRX/DWEST" of Sec. 5.2); reduce = 0: the detector on
 * the L-band cube as given.  score: [H][W] float32.  On the full band, LRX and DWRX
 * with fewer background samples than bands (N = outer^2 - inner^2 < L, loading > 0) are
 * solved at dimension N: with Xt = (X - mu_o) / sqrt(N) (L x N), C_o = Xt Xt^T and
 * d^T (C_o + delta I)^-1 d = (d^T d - |L_M^-1 Xt^T d|^2) / delta, L_M L_M^T = Xt^T Xt + delta I
 * (Woodbury identity); the result is the same quantity as the L x L solve.
 * flags (nullable): [H][W] uint8 per pixel; bit 0 = re-solved in FP64 (MIXED),
 * bit 1 = covariance not positive definite (score NaN), bit 2 = outside the
 * valid region (border = 1). */
wdad_status wdad_detect(wdad_handle h, const float* cube, int H, int W, int L,
                        int detector, int reduce, const wdad_params* p,
                        float* score, uint8_t* flags, void* stream);

/* All three detectors in one pass over the shared window statistics.
 * scores: [3][H][W] float32 in the order LRX, DWRX, DWEST.  flags as above (OR of the three). */
wdad_status wdad_detect_all(wdad_handle h, const float* cube, int H, int W, int L,
                            int reduce, const wdad_params* p,
                            float* scores, uint8_t* flags, void* stream);

/* All three detectors at nwin windows (params[0..nwin-1], same wavelet and level) in one
 * call: scores [nwin][3][H][W] device float32, flags (nullable) [nwin][H][W] uint8.  On the
 * reduced cube (and any cube of at most 8 bands) up to four windows share one launch, one
 * grid whose blocks each take a tile of one window; every window's maps equal those of
 * wdad_detect_all with the same params.  reduce = 1 runs the DWT first (handle workspace);
 * more than 8 bands run one full-band pass per window.  nwin 1..64. */
wdad_status wdad_detect_windows(wdad_handle h, const float* cube, int H, int W, int L, int reduce, int nwin,
                                const wdad_params* params, float* scores, uint8_t* flags, void* stream);

/* The same pass from HOST memory, for callers whose cube lives on the host: the
 * cube is reduced once (reduce = 1), all three detectors run for each of the nwin
 * parameter sets params[0..nwin-1] (same wavelet and level), and the score maps are
 * copied back to host_scores, laid out [nwin][3][H][W] (LRX, DWRX, DWEST).
 * host_cube and host_scores are HOST pointers.  With reduce = 1 and K <= 8 the call runs
 * in row bands (at least 64 rows, twice the widest halo plus a tile, an eighth of the
 * image) over three streams: the handle's copy stream moves band b of the cube to the
 * workspace, the DWT of band b - 1 runs on `stream`, and the handle's second stream runs
 * the detector tiles of band b - 2 and copies that band's score rows back in one strided
 * copy.  Otherwise the cube is copied to the workspace on `stream` and the one-pass path
 * runs.  The maps equal wdad_detect_windows' bit for bit.  Page-locked memory makes the
 * copies asynchronous, pageable memory makes them synchronous.  The caller synchronises
 * `stream` before reading host_scores, and keeps host_cube unchanged until then. */
wdad_status wdad_detect_all_host(wdad_handle h, const float* host_cube, int H, int W, int L, int reduce,
                                 int nwin, const wdad_params* params, float* host_scores, void* stream);

/* A1-A5 over a sequence of n cubes of one shape (a stream of scenes), reduced path only:
 * for each cube the DWT approximation and all three detectors at nwin windows, maps
 * bit-identical to wdad_detect_windows(reduce = 1) of that cube.  The DWT of cube i runs on
 * a stream the handle owns (created at the device's highest priority) beside the detector
 * launch of cube i - 1 on `stream`, through two approximation buffers in the handle's
 * workspace (2 H W K floats).  The DWT kernel is the standalone one, launched on three
 * quarters of the SMs with an unused shared-memory reservation (at most 100 KiB) that leaves
 * room for one detector CTA beside each of its CTAs, so that the two launches share SMs.
 *   - cubes: host array of n device pointers, each [H][W][L] float32, 16-byte aligned.
 *   - outs: host array of n device pointers, each [nwin][3][H][W] float32 (LRX, DWRX, DWEST);
 *     entries may repeat (the detector launches run in order on `stream`).
 *   - events: NULL, or a host array of 4 n entries, each a cudaEvent_t the caller created or
 *     NULL: for cube i, events[4i] and [4i+1] are recorded around its DWT (on the handle's
 *     stream) and [4i+2], [4i+3] around its detector launch (on `stream`).  Each recorded
 *     timing event costs a few microseconds of overlap; record a sample.
 *   - The call enqueues everything and returns; the work is complete when `stream` reaches
 *     the point after the call.  The cubes must stay unchanged until then.  n = 0 does
 *     nothing.  Windows as for wdad_detect_windows (nwin 1..64, one wavelet and level). */
wdad_status wdad_detect_sequence(wdad_handle h, int n, const float* const* cubes, int H, int W, int L, int nwin,
                                 const wdad_params* params, float* const* outs, void* const* events, void* stream);

/* A3 — background statistics of listed pixels (Sec. 2.1, Sec. 2.2): mean mu_o and covariance
 * C_o = (1/N) sum (x - mu_o)(x - mu_o)^T over the annulus between p->inner and p->outer
 * (reflect-101 borders), on the L-band cube as given.  pixels: device int64 [npix] linear
 * indices y*W + x; mu_o: device [npix][L]; cov_o: device [npix][L][L] row-major (both
 * triangles).  p->precision selects the Gram: FP32 SIMT, MIXED = BF16 tensor cores with
 * FP32 accumulation (L <= 256; larger L uses FP32), FP64.  L <= 1024. */
wdad_status wdad_window_moments(wdad_handle h, const float* cube, int H, int W, int L, const int64_t* pixels,
                                int64_t npix, const wdad_params* p, float* mu_o, float* cov_o, void* stream);

/* A2 — window census computed by the same tile loader and box-sum code as the
 * reduced detectors, with an integer payload: for every pixel, over the
 * background annulus and over the inner window (Sec. 2.2 dual window with
 * reflect-101 borders): count, sum of linear pixel indices, sum of their squares.
 * out: [H][W][6] int64 (nb, sum_b, sumsq_b, ni, sum_i, sumsq_i); -1 entries
 * outside the valid region when border = 1.  Exact integer results. */
wdad_status wdad_window_census(wdad_handle h, int H, int W, const wdad_params* p,
                               int64_t* out, void* stream);

/* The reduced pass of wdad_detect_all (reduce = 1) without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc.  Examples are software that fixes its memory budget at start-up, hosts
 * whose framework owns all device memory through its own pool, and latency-critical code
 * where an allocation could block on or synchronise with queued work.
 * There is no handle.  It works on the current CUDA device and on `stream`.  Its
 * scratch (the DWT matrix and the H x W x K approximation matrix) is a fixed 16 MiB +
 * 32 KiB array inside the library, held by every device that loads the library until
 * the process exits.
 *   - Limits: H * W * K <= 4,194,304 (e.g. 1024 x 1024 pixels at K = 4), L <= 1024,
 *     K <= 8.  Larger sizes return WDAD_ERR_ARG; windows whose tile does not fit
 *     shared memory return WDAD_ERR_UNSUPPORTED.  Other argument rules as wdad_detect_all.
 *   - Every call looks up the array's device address in the current context
 *     (cudaGetSymbolAddress; not a stream operation), so a context torn down and made
 *     again is handled.  The first call on a device may also load the library's module
 *     into the context.  Make that first call before any stream capture.
 *   - Every call on a device shares the one array.  Calls that overlap on the GPU (other
 *     streams, other host threads) race on it and must be serialised by the caller.
 *     Nothing in it needs clearing: each call overwrites what it reads.
 *   - cube: [H][W][L] float32 device; scores: [3][H][W] float32 device (LRX, DWRX, DWEST);
 *     flags: [H][W] uint8 device or NULL, as for wdad_detect. */
wdad_status wdad_detect_all_noalloc(const float* cube, int H, int W, int L, const wdad_params* p,
                                    float* scores, uint8_t* flags, void* stream);

/* A8 — batching.  One job = one cube through the DWT-reduced path (A1 + detectors).
 * Limits of the batched path: L % 4 == 0, L <= 256, K <= 4 (e.g. L in {128, 188, 224}). */
typedef struct {
    const float* cube;    /* [H][W][L] device, read-only */
    int H, W, L;
    int detector;         /* 0 LRX, 1 DWRX, 2 DWEST, 3 = all three */
    wdad_params params;   /* windows, loading, border, DWEST mode, wavelet, level */
    float* scores;        /* device: [H][W], or [3][H][W] (LRX, DWRX, DWEST) when detector == 3 */
    uint8_t* flags;       /* device [H][W] or NULL */
} wdad_job;

typedef struct wdad_batch_ctx* wdad_batch;

/* Tile height the library's autotuner picks for D bands and a window: every height from 16
 * down to 4 rows that fits shared memory (sliding sums restart at least every 16 rows) is
 * timed with CUDA events on a synthetic 256 x 256 cube (the batch tunes on a 1024 x 1024
 * cube, where the per-pixel cost that matters in a full GPU shows); the default plan is kept
 * unless another height is at least 3% faster.  The winner is cached in the handle.  Synchronises `stream`; do not call while
 * `stream` is being captured. */
wdad_status wdad_autotune(wdad_handle h, int D, int inner, int outer, int* tile_h, void* stream);

/* Prepare a batch of n jobs: DWT plans, tile plans (autotune != 0: the autotuner's, kept only
 * if the whole batch, timed with them and with the defaults over five launches each, runs at
 * least 1% faster -- those timing launches write the jobs' outputs; else the defaults that
 * wdad_detect uses), a device work list and per-job scratch owned by the
 * batch, and, when use_graph != 0, a CUDA graph of the whole launch captured on a private
 * stream.  Jobs below 512 x 512 pixels share one persistent kernel (counter reset, then the
 * kernel); a job of at least 512 x 512 pixels fills the GPU alone and runs as its own DWT and
 * detector launches after it, in the same graph (running the two side by side on forked
 * streams measured no faster).  The jobs' pointers are baked in: later
 * launches read and write the same buffers.  With default plans every job's scores are
 * bit-identical to wdad_detect / wdad_detect_all on the same job. */
wdad_status wdad_batch_create(wdad_handle h, int n, const wdad_job* jobs, int autotune, int use_graph,
                              wdad_batch* out, void* stream);
/* Enqueue the batch on `stream` (graph replay when captured). */
wdad_status wdad_batch_launch(wdad_batch b, void* stream);
/* Synchronise the batch's last launch and report its device status: WDAD_OK, or
 * WDAD_ERR_TIMEOUT when a tile gave up waiting for its cube's DWT (that job's scores are
 * then not written) or a staged DWT chunk never arrived, or WDAD_ERR_CUDA when, after such a
 * chunk, the copies queued behind it did not land either: a CTA then left while bulk copies
 * may still write its shared memory, so the batch must be destroyed and the device context
 * reset before further use.  *tile_h_out (nullable, n entries) receives each job's tile height.
 * Fault injection for tests: with the environment variable WDAD_FAULT_DROP_DWT_ITEM=j set
 * when the batch is created, the work list of persistent-kernel job j loses one DWT item, so
 * that job's tiles run into their bounded wait (host-side; no device fault is raised). */
wdad_status wdad_batch_status(wdad_batch b, int* tile_h_out);
wdad_status wdad_batch_destroy(wdad_batch b);
/* One-shot: create (default plans, no graph), launch on `stream`, synchronise, destroy. */
wdad_status wdad_batch_run(wdad_handle h, int n, const wdad_job* jobs, void* stream);

/* A9 — learned screening.  A 4-layer CNN on the DWT approximation matrix:
 * K -> 32 (5x5, ReLU) -> 32 (5x5, ReLU) -> 32 (5x5, ReLU) -> 1 (3x3), "same" zero padding,
 * receptive field 15 x 15, predicting log(1 + DWT-LRX score).  Activations NHWC float32;
 * FP32 master weights trained with Adam, forward with BF16-rounded weights (bf16_weights = 1)
 * or the masters (0); the paper has no such network (it is an addition on top of Sec. 4). */
typedef struct wdad_cnn_ctx* wdad_cnn;

/* New network with He-uniform weights drawn from splitmix64(seed); max_batch_pixels bounds
 * B * H * W of training batches (device buffers are sized for it). */
wdad_status wdad_cnn_create(wdad_handle h, int K, int bf16_weights, uint64_t seed, int64_t max_batch_pixels,
                            wdad_cnn* out);
wdad_status wdad_cnn_destroy(wdad_cnn c);
/* The network's input map z = M (x - mu) applied to raw approximation values x (first layer
 * and training crops).  host_mu_M == NULL (the default of a new network) whitens every scene
 * with its own statistics: each wdad_cnn_forward / wdad_cnn_train / wdad_screen_run call first
 * runs wdad_scene_whitening on its input.  Otherwise host_mu_M = [mu (K), M (K x K,
 * row-major)] is a fixed map used for every call (finite values, else WDAD_ERR_ARG).  The map
 * is stored with the network (checkpoints included); a network serves one stream at a time. */
wdad_status wdad_cnn_set_norm(wdad_cnn c, const float* host_mu_M);
/* Scene whitening of the network's input: for x [P][K] (device, K in 1..8, P >= 1) writes
 * norm_out (device, K + K*K floats) = [mu, M] with mu the mean, C = (1/P) sum (x - mu)(x - mu)^T
 * = L L^T (Cholesky; a pivot not above 1e-12 trace(C)/K is replaced by that floor, by 1 when
 * the trace is 0) and M = L^{-1}.  FP64 sums in a fixed order (deterministic on any GPU);
 * uses the handle's workspace; asynchronous on `stream`.  No paper counterpart (input
 * conditioning of the screening network). */
wdad_status wdad_scene_whitening(wdad_handle h, const float* x, int64_t P, int K, float* norm_out, void* stream);
/* Parameter count (and, when host != NULL, a host copy of the FP32 masters, per layer
 * weights [ci][ky*k+kx][co] then biases). */
wdad_status wdad_cnn_params(wdad_cnn c, float* host, int64_t* count);
/* Replace the masters (resets the Adam state). */
wdad_status wdad_cnn_set_params(wdad_cnn c, const float* host, int64_t count);
/* pred [B][H][W] from raw x [B][H][W][K] (device); the input map is applied inside (per-scene
 * mode: whitened with the statistics of all B * H * W input pixels). */
wdad_status wdad_cnn_forward(wdad_cnn c, const float* x, int B, int H, int W, float* pred, void* stream);
/* Gradients of the interior MSE (7-pixel border excluded) for mapped input z [B][H][W][K] and
 * targets [B][H][W] (device); host_grad [count] and host_loss (both nullable); synchronises. */
wdad_status wdad_cnn_grad(wdad_cnn c, const float* x, const float* target, int B, int H, int W, float* host_grad,
                          float* host_loss, void* stream);
/* `steps` Adam steps on random crop x crop patches (batch per step, positions from
 * splitmix64(seed, step)) of one reduced cube approx [H][W][K] with targets
 * log(1 + score[H][W]); host_loss (nullable) receives the last batch loss. */
wdad_status wdad_cnn_train(wdad_cnn c, const float* approx, const float* score, int H, int W, int steps, int batch,
                           int crop, float lr, uint64_t seed, float* host_loss, void* stream);
/* Versioned checkpoint (version 2): masters, Adam moments, step, input-map mode and map.
 * Loading a file of another version fails with WDAD_ERR_ARG. */
wdad_status wdad_cnn_save(wdad_cnn c, const char* path);
wdad_status wdad_cnn_load(wdad_handle h, const char* path, int64_t max_batch_pixels, wdad_cnn* out);
/* Screened LRX: A1 on the cube, the CNN on row tiles (tile_rows + 7-row halo), the top
 * top_frac of its predictions (every pixel whose prediction is at least the k-th largest,
 * k = max(1, ceil(top_frac * H * W)) up to one float rounding of top_frac; ties at the
 * threshold are all taken) plus a random audit of audit_frac (splitmix64(seed, pixel)),
 * then the exact LRX (exact_reduce = 0: full band; 1: on the reduced cube) on the selected
 * pixels only.  score [H][W]: exact LRX where selected, -inf elsewhere.  pred [H][W] and
 * selected [H][W] (1 = top, 2 = audit, 0 = skipped) are nullable; *n_selected (host,
 * nullable) receives the number of exact evaluations.  Synchronises `stream`. */
wdad_status wdad_screen_run(wdad_handle h, wdad_cnn c, const float* cube, int H, int W, int L, const wdad_params* p,
                            float top_frac, float audit_frac, uint64_t seed, int tile_rows, int exact_reduce,
                            float* score, float* pred, uint8_t* selected, int64_t* n_selected, void* stream);

/* Adaptive cut-off of Eq. 12 (Sec. 5.3.2): tau = mu_d + z_alpha * sigma_d, where mu_d and
 * sigma_d are the mean and the population (1/n) standard deviation of the n finite entries of
 * the anomaly matrix `score` (device, float32; NaN entries, e.g. border pixels, are left out);
 * mask (device, n bytes, nullable) receives 1 where score > tau, else 0 (NaN -> 0).
 * host_stats (host, 4 doubles, nullable) receives mu_d, sigma_d, tau, count, after the call
 * synchronises `stream`; without it the call is asynchronous.  FP64 sums in a fixed order
 * (the same on any GPU).  n == 0 gives NaN statistics and count 0.  Uses the handle's
 * workspace; z_alpha must be finite (WDAD_ERR_ARG otherwise). */
wdad_status wdad_adaptive_threshold(wdad_handle h, const float* score, int64_t n, double z_alpha, uint8_t* mask,
                                    double* host_stats, void* stream);

/* A10 — pixel-level ROC AUC of a score map against a truth mask (Sec. 5.3.1):
 * Mann-Whitney U with ties counted one half.  HOST pointers; NaN scores rank lowest.
 * Writes NaN when the mask has no positive or no negative pixel. */
wdad_status wdad_auc(const float* score, const uint8_t* mask, int64_t n, double* auc);

#ifdef __cplusplus
}
#endif
#endif /* WDAD_H */
