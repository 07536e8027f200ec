/*
 * FP64 CPU oracle of the screening CNN: forward and backward of
 *   K -> 32 (5x5, ReLU) -> 32 (5x5, ReLU) -> 32 (5x5, ReLU) -> 1 (3x3), "same" zero padding,
 * with the mean squared error over the interior of each image (a border of `edge` pixels
 * excluded).  Parameters per layer: weights [ci][ky*k+kx][co], then biases [co].
 * Activations [B][H][W][C].  The network's input is the approximation matrix whitened with
 * the scene's own statistics (or_scene_whiten).  TEST INFRASTRUCTURE ONLY; plain loops, no
 * shared code with the CUDA path.  The network is an addition to the paper's method (no
 * counterpart in it).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static const int KS[4] = {5, 5, 5, 3};

static void dims(int K, int l, int* cin, int* cout, int* k) {
    *cin = l == 0 ? K : 32;
    *cout = l == 3 ? 1 : 32;
    *k = KS[l];
}

long or_cnn_nparam(int K) {
    long n = 0;
    for (int l = 0; l < 4; ++l) {
        int ci, co, k;
        dims(K, l, &ci, &co, &k);
        n += (long)ci * k * k * co + co;
    }
    return n;
}

/* out[b,y,x,co] = bias[co] + sum_{ci,ky,kx} in[b, y+ky-p, x+kx-p, ci] w[ci, ky*k+kx, co] */
static void conv(const double* in, int B, int H, int W, int cin, const double* w, const double* bias, int cout, int k,
                 double* out) {
    int p = k / 2;
    for (int b = 0; b < B; ++b)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                double* o = out + (((long)b * H + y) * W + x) * cout;
                for (int co = 0; co < cout; ++co) o[co] = bias[co];
                for (int ky = 0; ky < k; ++ky) {
                    int yy = y + ky - p;
                    if (yy < 0 || yy >= H) continue;
                    for (int kx = 0; kx < k; ++kx) {
                        int xx = x + kx - p;
                        if (xx < 0 || xx >= W) continue;
                        const double* a = in + (((long)b * H + yy) * W + xx) * cin;
                        for (int ci = 0; ci < cin; ++ci) {
                            const double* wr = w + ((long)ci * k * k + ky * k + kx) * cout;
                            for (int co = 0; co < cout; ++co) o[co] += a[ci] * wr[co];
                        }
                    }
                }
            }
}

/* given dz (gradient w.r.t. conv output): accumulate dw, db and (nullable) din */
static void conv_back(const double* in, const double* dz, int B, int H, int W, int cin, const double* w, int cout,
                      int k, double* dw, double* db, double* din) {
    int p = k / 2;
    if (din) memset(din, 0, sizeof(double) * (size_t)B * H * W * cin);
    for (int b = 0; b < B; ++b)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const double* d = dz + (((long)b * H + y) * W + x) * cout;
                for (int co = 0; co < cout; ++co) db[co] += d[co];
                for (int ky = 0; ky < k; ++ky) {
                    int yy = y + ky - p;
                    if (yy < 0 || yy >= H) continue;
                    for (int kx = 0; kx < k; ++kx) {
                        int xx = x + kx - p;
                        if (xx < 0 || xx >= W) continue;
                        const double* a = in + (((long)b * H + yy) * W + xx) * cin;
                        double* da = din ? din + (((long)b * H + yy) * W + xx) * cin : NULL;
                        for (int ci = 0; ci < cin; ++ci) {
                            const long wb = ((long)ci * k * k + ky * k + kx) * cout;
                            double g = 0.0;
                            for (int co = 0; co < cout; ++co) {
                                dw[wb + co] += a[ci] * d[co];
                                g += w[wb + co] * d[co];
                            }
                            if (da) da[ci] += g;
                        }
                    }
                }
            }
}

/* v rounded to float32 (nearest) and then to bfloat16 (nearest, ties to even): the value a
   float32 activation takes when a tensor-core layer reads it as bfloat16 (finite inputs) */
double or_bf16_round(double v) {
    float f = (float)v;
    unsigned int u;
    memcpy(&u, &f, sizeof u);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    memcpy(&f, &u, sizeof f);
    return (double)f;
}

static int forward_impl(int K, const double* params, const double* x, int B, int H, int W, int bf16_act, double* pred);

int or_cnn_forward(int K, const double* params, const double* x, int B, int H, int W, double* pred) {
    return forward_impl(K, params, x, B, H, W, 0, pred);
}

/* The same network with the inputs of the two 32 -> 32 layers (the ReLU outputs of layers 1
   and 2) rounded to bfloat16: the inference form whose 32 -> 32 convolutions run on the
   tensor cores with bfloat16 operands and float accumulation. */
int or_cnn_forward_bf16act(int K, const double* params, const double* x, int B, int H, int W, double* pred) {
    return forward_impl(K, params, x, B, H, W, 1, pred);
}

static int forward_impl(int K, const double* params, const double* x, int B, int H, int W, int bf16_act, double* pred) {
    long px = (long)B * H * W;
    double* a = (double*)malloc(sizeof(double) * px * 32);
    double* c = (double*)malloc(sizeof(double) * px * 32);
    const double* in = x;
    long off = 0;
    for (int l = 0; l < 4; ++l) {
        int ci, co, k;
        dims(K, l, &ci, &co, &k);
        const double* w = params + off;
        const double* bias = w + (long)ci * k * k * co;
        off += (long)ci * k * k * co + co;
        double* out = (l == 3) ? pred : (l % 2 == 0 ? a : c);
        conv(in, B, H, W, ci, w, bias, co, k, out);
        if (l < 3)
            for (long i = 0; i < px * co; ++i) out[i] = out[i] > 0.0 ? out[i] : 0.0;
        if (bf16_act && (l == 0 || l == 1))
            for (long i = 0; i < px * co; ++i) out[i] = or_bf16_round(out[i]);
        in = out;
    }
    free(a); free(c);
    return 0;
}

/* loss = mean over interior pixels of (pred - t)^2; grad (nparam) */
int or_cnn_grad(int K, const double* params, const double* x, const double* t, int B, int H, int W, int edge,
                double* grad, double* loss) {
    long px = (long)B * H * W;
    double* act[4];
    for (int l = 0; l < 4; ++l) act[l] = (double*)malloc(sizeof(double) * px * 32);
    const double* in = x;
    long woff[4];
    long off = 0;
    for (int l = 0; l < 4; ++l) {
        int ci, co, k;
        dims(K, l, &ci, &co, &k);
        woff[l] = off;
        const double* w = params + off;
        conv(in, B, H, W, ci, w, w + (long)ci * k * k * co, co, k, act[l]);
        if (l < 3)
            for (long i = 0; i < px * co; ++i) act[l][i] = act[l][i] > 0.0 ? act[l][i] : 0.0;
        off += (long)ci * k * k * co + co;
        in = act[l];
    }
    long n = (long)B * (H - 2 * edge) * (W - 2 * edge);
    double* dz = (double*)malloc(sizeof(double) * px * 32);
    double* dnext = (double*)malloc(sizeof(double) * px * 32);
    double s = 0.0;
    for (int b = 0; b < B; ++b)
        for (int y = 0; y < H; ++y)
            for (int xx = 0; xx < W; ++xx) {
                long i = ((long)b * H + y) * W + xx;
                int interior = y >= edge && y < H - edge && xx >= edge && xx < W - edge;
                double r = act[3][i] - t[i];
                dz[i] = interior ? 2.0 * r / n : 0.0;
                if (interior) s += r * r;
            }
    *loss = s / n;
    memset(grad, 0, sizeof(double) * or_cnn_nparam(K));
    for (int l = 3; l >= 0; --l) {
        int ci, co, k;
        dims(K, l, &ci, &co, &k);
        const double* lin = l == 0 ? x : act[l - 1];
        double* dw = grad + woff[l];
        double* db = dw + (long)ci * k * k * co;
        conv_back(lin, dz, B, H, W, ci, params + woff[l], co, k, dw, db, l > 0 ? dnext : NULL);
        if (l > 0) {
            for (long i = 0; i < px * ci; ++i) dnext[i] = lin[i] > 0.0 ? dnext[i] : 0.0;  /* ReLU of layer l-1 */
            double* tmp = dz; dz = dnext; dnext = tmp;
        }
    }
    for (int l = 0; l < 4; ++l) free(act[l]);
    free(dz); free(dnext);
    return 0;
}

/*
 * Scene whitening of the network's input: mean mu and population covariance
 * C = (1/P) sum_p (x_p - mu)(x_p - mu)^T of P pixels with K values each, the Cholesky factor
 * C = L L^T, and M = L^{-1} (lower triangular, positive diagonal), so that z = M (x - mu) has
 * zero mean and identity covariance.  A pivot that is not above 1e-12 * trace(C) / K is
 * replaced by that floor (by 1 when trace(C) == 0), so constant bands give a finite M.
 * Two passes (mean, then centred products); M by forward substitution on the unit vectors.
 */
int or_scene_whiten(int K, const double* x, long P, double* mu, double* M) {
    if (K < 1 || K > 8 || P < 1) return -1;
    double C[64], Lf[64];
    for (int i = 0; i < K; ++i) {
        double s = 0.0;
        for (long p = 0; p < P; ++p) s += x[p * K + i];
        mu[i] = s / (double)P;
    }
    double tr = 0.0;
    for (int i = 0; i < K; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = 0.0;
            for (long p = 0; p < P; ++p) s += (x[p * K + i] - mu[i]) * (x[p * K + j] - mu[j]);
            C[i * K + j] = C[j * K + i] = s / (double)P;
            if (i == j) tr += C[i * K + i];
        }
    const double floor = tr > 0.0 ? 1e-12 * tr / (double)K : 1.0;
    memset(Lf, 0, sizeof Lf);
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
    /* column c of M solves L m = e_c */
    for (int c = 0; c < K; ++c)
        for (int i = 0; i < K; ++i) {
            double v = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= Lf[i * K + k] * M[k * K + c];
            M[i * K + c] = v / Lf[i * K + i];
        }
    return 0;
}
