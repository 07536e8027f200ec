/*
 * FP64 CPU oracle for DWT-reduced local anomaly detection (Zare Baghbidi et al.,
 * "Improvement of anomaly detection algorithms in hyperspectral images using
 * discrete wavelet transform", SIPIJ 2(4), 2011).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
 * Python binding) may include, link, load or call this file.  It shares no
 * code, header, table or constant with the CUDA path: the Daubechies filter is
 * derived here by spectral factorisation, the transform is the literal Eq. 9
 * cascade, the statistics are two-pass sums, the solves are textbook Cholesky
 * and cyclic Jacobi.  Everything is plain double precision, pixel by pixel.
 *
 * Readings of the paper (where it is silent or ambiguous) are fixed here:
 *   - "Daubechies4" = 8-tap db4 (4 vanishing moments); taps=4 gives the D4 variant.
 *   - Eq. 9 literally, a[k] = sum_j h[j] x[(2k - j) mod M], with periodic indices;
 *     odd lengths are padded to even M by repeating the last sample.
 *   - levels: smallest J whose approximation length is <= 4 (Sec. 4), unless given.
 *   - windows: inner = w_i x w_i square incl. the centre, background = w_o x w_o
 *     square minus the inner square (an annulus), border rows/columns reflect-101.
 *   - covariances use 1/n (sample = MLE); LRX and DWRX use diagonal loading
 *     delta = loading * trace(C_o)/dim, DWEST none.
 *   - DWEST keeps eigenvectors with lambda > 1e-6 * max|lambda|; mode 0 makes each
 *     selected eigenvector's largest-magnitude component positive (ties: lowest
 *     index) and returns |sum_k v_k^T m_diff| (Eq. 4); mode 1 returns ||V_S^T m_diff||.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Daubechies scaling filter by spectral factorisation (Daubechies, Ten       */
/* Lectures, Ch. 6): |m0(xi)|^2 = cos^{2p}(xi/2) P(sin^2(xi/2)),              */
/* P(y) = sum_{k<p} C(p-1+k, k) y^k.  Each root y_j of P gives the quadratic  */
/* w + 1/w = 2 - 4 y_j in w = e^{-i xi}; one root per pair is kept and         */
/* H(w) = c (1+w)^p prod_j (w - w_j), scaled so that sum h = sqrt(2).          */
/* ------------------------------------------------------------------------ */
static double binom(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

static double complex poly_eval(const double* c, int deg, double complex z) {
    double complex s = c[deg];
    for (int i = deg - 1; i >= 0; --i) s = s * z + c[i];
    return s;
}

/* taps = 2p, p = 1..10.  Returns 0 on success, -1 on bad taps. */
int or_daub_filter(int taps, double* h) {
    if (taps < 2 || taps > 20 || (taps & 1)) return -1;
    int p = taps / 2, deg = p - 1;
    double c[16];
    for (int k = 0; k <= deg; ++k) c[k] = binom(p - 1 + k, k);
    double complex y[16];
    /* Durand-Kerner on the monic polynomial, then Newton polishing */
    if (deg > 0) {
        double complex seed = 0.4 + 0.9 * I;
        double complex zc = 1.0;
        for (int i = 0; i < deg; ++i) { y[i] = zc; zc *= seed; }
        for (int it = 0; it < 2000; ++it) {
            double moved = 0.0;
            for (int i = 0; i < deg; ++i) {
                double complex den = c[deg];
                for (int j = 0; j < deg; ++j)
                    if (j != i) den *= (y[i] - y[j]);
                double complex step = poly_eval(c, deg, y[i]) / den;
                y[i] -= step;
                moved = fmax(moved, cabs(step));
            }
            if (moved < 1e-17) break;
        }
        for (int i = 0; i < deg; ++i) {
            for (int it = 0; it < 20; ++it) {
                double complex f = poly_eval(c, deg, y[i]);
                double complex d = 0.0;
                for (int k = deg; k >= 1; --k) d = d * y[i] + (double)k * c[k];
                if (cabs(d) == 0.0) break;
                y[i] -= f / d;
            }
        }
    }
    /* polynomial in w, ascending powers, complex during the build */
    double complex poly[24];
    for (int i = 0; i < 24; ++i) poly[i] = 0.0;
    poly[0] = 1.0;
    int len = 1;
    for (int k = 0; k < p; ++k) { /* multiply by (1 + w) */
        for (int i = len; i >= 1; --i) poly[i] += poly[i - 1];
        len++;
    }
    for (int j = 0; j < deg; ++j) {
        double complex b = 2.0 - 4.0 * y[j];
        double complex s = csqrt(b * b - 4.0);
        double complex w1 = 0.5 * (b + s), w2 = 0.5 * (b - s);
        double complex w = (cabs(w1) >= cabs(w2)) ? w1 : w2; /* root outside the unit circle */
        /* multiply by (w - root) */
        for (int i = len; i >= 1; --i) poly[i] = poly[i - 1] - w * poly[i];
        poly[0] = -w * poly[0];
        len++;
    }
    double sum = 0.0;
    for (int i = 0; i < taps; ++i) sum += creal(poly[i]);
    for (int i = 0; i < taps; ++i) h[i] = creal(poly[i]) * sqrt(2.0) / sum;
    return 0;
}

/* quadrature mirror high-pass: g[n] = (-1)^n h[taps-1-n] */
void or_highpass(const double* h, int taps, double* g) {
    for (int n = 0; n < taps; ++n) g[n] = ((n & 1) ? -1.0 : 1.0) * h[taps - 1 - n];
}

/* ------------------------------------------------------------------------ */
/* One analysis step (Eq. 9 / Eq. 8 with f = h / g): out[k] = sum_j f[j] *   */
/* xe[(2k - j) mod M], k < M/2, xe = x padded to even M with its last sample. */
/* ------------------------------------------------------------------------ */
static long mod_pos(long a, long m) { long r = a % m; return r < 0 ? r + m : r; }

int or_dwt_step(const double* x, int n, const double* f, int taps, double* out) {
    if (n < 1) return -1;
    int M = n + (n & 1);
    for (int k = 0; k < M / 2; ++k) {
        double s = 0.0;
        for (int j = 0; j < taps; ++j) {
            long idx = mod_pos(2L * k - j, M);
            double v = (idx < n) ? x[idx] : x[n - 1];
            s += f[j] * v;
        }
        out[k] = s;
    }
    return M / 2;
}

/* Transpose of one analysis step on the padded signal: xe (length 2m) from a, d. */
void or_dwt_synth_step(const double* a, const double* d, int m, const double* h,
                       const double* g, int taps, double* xe) {
    int M = 2 * m;
    for (int i = 0; i < M; ++i) xe[i] = 0.0;
    for (int k = 0; k < m; ++k)
        for (int j = 0; j < taps; ++j) {
            long idx = mod_pos(2L * k - j, M);
            xe[idx] += h[j] * a[k] + g[j] * d[k];
        }
}

/* Number of levels and approximation length K.  level < 0: smallest J with K <= 4. */
int or_dwt_levels(int L, int level, int* K) {
    int n = L, J = 0;
    if (level < 0) {
        while (n > 4) { n = (n + 1) / 2; J++; }
    } else {
        for (J = 0; J < level; ++J) n = (n + 1) / 2;
    }
    if (K) *K = n;
    return J;
}

/* Full decomposition [a_J, d_J, d_{J-1}, ..., d_1] (Fig. 1 order); returns its length. */
int or_dwt_full(const double* x, int L, int taps, int level, double* out) {
    double h[20], g[20];
    if (or_daub_filter(taps, h)) return -1;
    or_highpass(h, taps, g);
    int K;
    int J = or_dwt_levels(L, level, &K);
    double* cur = (double*)malloc(sizeof(double) * (L + 2));
    double* det = (double*)malloc(sizeof(double) * (L + 2) * 2);
    int* dlen = (int*)malloc(sizeof(int) * (J + 1));
    int* doff = (int*)malloc(sizeof(int) * (J + 1));
    memcpy(cur, x, sizeof(double) * L);
    int n = L, dtot = 0;
    double* tmp = (double*)malloc(sizeof(double) * (L + 2));
    for (int j = 0; j < J; ++j) {
        int m = or_dwt_step(cur, n, h, taps, tmp);
        or_dwt_step(cur, n, g, taps, det + dtot);
        dlen[j] = m; doff[j] = dtot; dtot += m;
        memcpy(cur, tmp, sizeof(double) * m);
        n = m;
    }
    int pos = 0;
    for (int i = 0; i < n; ++i) out[pos++] = cur[i];
    for (int j = J - 1; j >= 0; --j)
        for (int i = 0; i < dlen[j]; ++i) out[pos++] = det[doff[j] + i];
    free(cur); free(det); free(dlen); free(doff); free(tmp);
    return pos;
}

/* Inverse of or_dwt_full (synthesis = transpose at every level, padding dropped). */
int or_dwt_inverse(const double* coef, int L, int taps, int level, double* x) {
    double h[20], g[20];
    if (or_daub_filter(taps, h)) return -1;
    or_highpass(h, taps, g);
    int K;
    int J = or_dwt_levels(L, level, &K);
    int* len = (int*)malloc(sizeof(int) * (J + 1)); /* signal length entering level j */
    len[0] = L;
    for (int j = 0; j < J; ++j) len[j + 1] = (len[j] + 1) / 2;
    double* cur = (double*)malloc(sizeof(double) * (L + 2));
    double* xe = (double*)malloc(sizeof(double) * (L + 2));
    memcpy(cur, coef, sizeof(double) * K);
    int pos = K;
    for (int j = J - 1; j >= 0; --j) {
        int m = len[j + 1];
        const double* d = coef + pos;
        pos += m;
        or_dwt_synth_step(cur, d, m, h, g, taps, xe);
        memcpy(cur, xe, sizeof(double) * len[j]); /* drop the pad sample if len[j] is odd */
    }
    memcpy(x, cur, sizeof(double) * L);
    free(len); free(cur); free(xe);
    return 0;
}

/* Approximation matrix: cube [P][L] float32 -> out [P][K] double, cascade of low-pass steps. */
int or_dwt_approx(const float* cube, long P, int L, int taps, int level, double* out, int nthreads) {
    double h[20];
    if (or_daub_filter(taps, h)) return -1;
    int K;
    int J = or_dwt_levels(L, level, &K);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        double* a = (double*)malloc(sizeof(double) * (L + 2));
        double* b = (double*)malloc(sizeof(double) * (L + 2));
#pragma omp for schedule(static)
        for (long p = 0; p < P; ++p) {
            for (int l = 0; l < L; ++l) a[l] = (double)cube[p * L + l];
            int n = L;
            for (int j = 0; j < J; ++j) {
                int m = or_dwt_step(a, n, h, taps, b);
                memcpy(a, b, sizeof(double) * m);
                n = m;
            }
            for (int k = 0; k < K; ++k) out[p * K + k] = a[k];
        }
        free(a); free(b);
    }
    return K;
}

/* ------------------------------------------------------------------------ */
/* Windows: reflect-101 border (-1 -> 1, n -> n-2), repeated for big windows. */
/* ------------------------------------------------------------------------ */
int or_reflect(int i, int n) {
    if (n == 1) return 0;
    long period = 2L * (n - 1);
    long r = mod_pos(i, period);
    return (int)(r < n ? r : period - r);
}

/* Row-major offsets of the inner square and of the background annulus. */
static int window_lists(int inner, int outer, int* in_dy, int* in_dx, int* bg_dy, int* bg_dx, int* nbg) {
    int ri = inner / 2, ro = outer / 2, ni = 0, nb = 0;
    for (int dy = -ro; dy <= ro; ++dy)
        for (int dx = -ro; dx <= ro; ++dx) {
            if (abs(dy) <= ri && abs(dx) <= ri) { in_dy[ni] = dy; in_dx[ni] = dx; ni++; }
            else { bg_dy[nb] = dy; bg_dx[nb] = dx; nb++; }
        }
    *nbg = nb;
    return ni;
}

/* ------------------------------------------------------------------------ */
/* Dense linear algebra (textbook, row-major n x n).                         */
/* ------------------------------------------------------------------------ */
/* Cholesky A = G G^T, G lower, in place.  Returns 0, or -1 if a pivot <= 0. */
static int cholesky(double* A, int n) {
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return -1;
        double gjj = sqrt(s);
        A[j * n + j] = gjj;
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / gjj;
        }
    }
    return 0;
}

/* ||G^{-1} d||^2 with G from cholesky() (= d^T A^{-1} d). */
static double chol_quadform(const double* G, int n, const double* d, double* y) {
    double q = 0.0;
    for (int i = 0; i < n; ++i) {
        double t = d[i];
        for (int k = 0; k < i; ++k) t -= G[i * n + k] * y[k];
        y[i] = t / G[i * n + i];
        q += y[i] * y[i];
    }
    return q;
}

/* Cyclic-by-row Jacobi (Golub & Van Loan, symmetric Schur rotations).  A is
 * destroyed; w = eigenvalues, V (nullable) columns = eigenvectors. */
static void jacobi_eig(double* A, int n, double* V, double* w) {
    if (V) {
        for (int i = 0; i < n * n; ++i) V[i] = 0.0;
        for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    }
    double fro = 0.0;
    for (int i = 0; i < n * n; ++i) fro += A[i] * A[i];
    fro = sqrt(fro);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q)
                if (p != q) off += A[p * n + q] * A[p * n + q];
        if (sqrt(off) <= 1e-14 * fro || fro == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) { /* A <- A J */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) { /* A <- J^T A */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                if (V)
                    for (int k = 0; k < n; ++k) {
                        double vkp = V[k * n + p], vkq = V[k * n + q];
                        V[k * n + p] = c * vkp - s * vkq;
                        V[k * n + q] = s * vkp + c * vkq;
                    }
            }
    }
    for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
}

/* ------------------------------------------------------------------------ */
/* Detectors.  det: 0 = LRX (Sec. 2.1, Eq. 1 on a local background),         */
/* 1 = DWRX (Eq. 5), 2 = DWEST (Eq. 2-4).  cube is [H*W][D] double.           */
/* aux (nullable, OR_NAUX doubles per listed pixel):                         */
/*   LRX/DWRX: [0] lambda_min, [1] lambda_max of C_o + delta I (only when     */
/*             want_cond != 0, else NaN), [2] delta, [3] N, [4] ||d||_2 of    */
/*             the tested difference vector, [5] NaN                          */
/*   DWEST:    [0] selection margin min_k |lambda_k - tau| / max|lambda|,     */
/*             [1] sign margin min over selected v of (|v|_(1) - |v|_(2)),    */
/*             [2] eigen-gap min over selected k, j != k of |l_k - l_j| /     */
/*             max|lambda|, [3] number of selected eigenvectors,              */
/*             [4] ||m_diff||_2, [5] sum over selected k of |v_k^T m_diff|    */
/* Pixels whose outer window leaves the image get NaN when border == 1.       */
/* ------------------------------------------------------------------------ */
#define OR_NAUX 6
int or_naux(void) { return OR_NAUX; }

int or_detect(const double* cube, int H, int W, int D, int det, int inner, int outer,
              double loading, int border, int dwest_mode, const int64_t* pix, int64_t npix,
              double* score, double* aux, int want_cond, int nthreads) {
    if (inner < 1 || outer <= inner || !(inner & 1) || !(outer & 1) || D < 1) return -1;
    int nmax = outer * outer;
    int* in_dy = (int*)malloc(sizeof(int) * nmax);
    int* in_dx = (int*)malloc(sizeof(int) * nmax);
    int* bg_dy = (int*)malloc(sizeof(int) * nmax);
    int* bg_dx = (int*)malloc(sizeof(int) * nmax);
    int N;
    int ni = window_lists(inner, outer, in_dy, in_dx, bg_dy, bg_dx, &N);
    int ro = outer / 2;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        double* mo = (double*)malloc(sizeof(double) * D);
        double* mi = (double*)malloc(sizeof(double) * D);
        double* d = (double*)malloc(sizeof(double) * D);
        double* y = (double*)malloc(sizeof(double) * D);
        double* Co = (double*)malloc(sizeof(double) * D * D);
        double* Ci = (double*)malloc(sizeof(double) * D * D);
        double* V = (double*)malloc(sizeof(double) * D * D);
        double* w = (double*)malloc(sizeof(double) * D);
        double* xc = (double*)malloc(sizeof(double) * D);
#pragma omp for schedule(dynamic, 4)
        for (int64_t t = 0; t < npix; ++t) {
            int64_t p = pix[t];
            int py = (int)(p / W), px = (int)(p % W);
            double* ax = aux ? aux + OR_NAUX * t : NULL;
            if (ax) for (int k = 0; k < OR_NAUX; ++k) ax[k] = NAN;
            if (border == 1 && (py - ro < 0 || py + ro >= H || px - ro < 0 || px + ro >= W)) {
                score[t] = NAN;
                continue;
            }
            /* background mean and covariance (two passes, 1/N) */
            for (int k = 0; k < D; ++k) mo[k] = 0.0;
            for (int s = 0; s < N; ++s) {
                const double* x = cube + ((int64_t)or_reflect(py + bg_dy[s], H) * W + or_reflect(px + bg_dx[s], W)) * D;
                for (int k = 0; k < D; ++k) mo[k] += x[k];
            }
            for (int k = 0; k < D; ++k) mo[k] /= N;
            for (int i = 0; i < D * D; ++i) Co[i] = 0.0;
            for (int s = 0; s < N; ++s) {
                const double* x = cube + ((int64_t)or_reflect(py + bg_dy[s], H) * W + or_reflect(px + bg_dx[s], W)) * D;
                for (int k = 0; k < D; ++k) xc[k] = x[k] - mo[k];
                for (int a = 0; a < D; ++a)
                    for (int b = 0; b < D; ++b) Co[a * D + b] += xc[a] * xc[b];
            }
            for (int i = 0; i < D * D; ++i) Co[i] /= N;
            /* inner mean (and covariance for DWEST) */
            for (int k = 0; k < D; ++k) mi[k] = 0.0;
            for (int s = 0; s < ni; ++s) {
                const double* x = cube + ((int64_t)or_reflect(py + in_dy[s], H) * W + or_reflect(px + in_dx[s], W)) * D;
                for (int k = 0; k < D; ++k) mi[k] += x[k];
            }
            for (int k = 0; k < D; ++k) mi[k] /= ni;

            if (det == 0 || det == 1) {
                const double* r = cube + p * D;
                for (int k = 0; k < D; ++k) d[k] = (det == 0) ? r[k] - mo[k] : mi[k] - mo[k];
                double tr = 0.0;
                for (int k = 0; k < D; ++k) tr += Co[k * D + k];
                double delta = loading * tr / D;
                for (int k = 0; k < D; ++k) Co[k * D + k] += delta;
                if (ax && want_cond) {
                    memcpy(Ci, Co, sizeof(double) * D * D);
                    jacobi_eig(Ci, D, NULL, w);
                    double lmin = w[0], lmax = w[0];
                    for (int k = 1; k < D; ++k) { lmin = fmin(lmin, w[k]); lmax = fmax(lmax, w[k]); }
                    ax[0] = lmin; ax[1] = lmax;
                }
                if (ax) {
                    double nd = 0.0;
                    for (int k = 0; k < D; ++k) nd += d[k] * d[k];
                    ax[2] = delta; ax[3] = N; ax[4] = sqrt(nd);
                }
                if (cholesky(Co, D)) { score[t] = NAN; continue; }
                double q = chol_quadform(Co, D, d, y);
                score[t] = (det == 0) ? q : fabs(q);
            } else {
                for (int i = 0; i < D * D; ++i) Ci[i] = 0.0;
                for (int s = 0; s < ni; ++s) {
                    const double* x = cube + ((int64_t)or_reflect(py + in_dy[s], H) * W + or_reflect(px + in_dx[s], W)) * D;
                    for (int k = 0; k < D; ++k) xc[k] = x[k] - mi[k];
                    for (int a = 0; a < D; ++a)
                        for (int b = 0; b < D; ++b) Ci[a * D + b] += xc[a] * xc[b];
                }
                for (int i = 0; i < D * D; ++i) Ci[i] = Ci[i] / ni - Co[i]; /* Eq. 2 */
                for (int k = 0; k < D; ++k) d[k] = mi[k] - mo[k];           /* Eq. 3 */
                jacobi_eig(Ci, D, V, w);
                double lmax = 0.0;
                for (int k = 0; k < D; ++k) lmax = fmax(lmax, fabs(w[k]));
                double tau = 1e-6 * lmax;
                double acc = 0.0, acc2 = 0.0, accabs = 0.0, selm = INFINITY, sgnm = INFINITY, gap = INFINITY;
                int nsel = 0;
                for (int k = 0; k < D; ++k) {
                    if (lmax > 0.0) selm = fmin(selm, fabs(w[k] - tau) / lmax);
                    if (!(w[k] > tau)) continue;
                    nsel++;
                    /* sign convention: largest-|.| component positive, ties -> lowest index */
                    int im = 0;
                    double b1 = -1.0, b2 = -1.0;
                    for (int a = 0; a < D; ++a) {
                        double v = fabs(V[a * D + k]);
                        if (v > b1) { b2 = b1; b1 = v; im = a; }
                        else if (v > b2) b2 = v;
                    }
                    if (D > 1) sgnm = fmin(sgnm, b1 - b2);
                    double sg = V[im * D + k] >= 0.0 ? 1.0 : -1.0;
                    double proj = 0.0;
                    for (int a = 0; a < D; ++a) proj += V[a * D + k] * d[a];
                    acc += sg * proj;
                    acc2 += proj * proj;
                    accabs += fabs(proj);
                    for (int j = 0; j < D; ++j)
                        if (j != k && lmax > 0.0) gap = fmin(gap, fabs(w[k] - w[j]) / lmax);
                }
                score[t] = (dwest_mode == 0) ? fabs(acc) : sqrt(acc2);
                if (ax) {
                    double nm = 0.0;
                    for (int k = 0; k < D; ++k) nm += d[k] * d[k];
                    ax[0] = selm; ax[1] = sgnm; ax[2] = gap; ax[3] = nsel; ax[4] = sqrt(nm); ax[5] = accabs;
                }
            }
        }
        free(mo); free(mi); free(d); free(y); free(Co); free(Ci); free(V); free(w); free(xc);
    }
    free(in_dy); free(in_dx); free(bg_dy); free(bg_dx);
    return 0;
}

/* Background statistics of listed pixels (Sec. 2.1): mean and covariance (1/N, two
 * passes) over the annulus; mu [npix][D], cov [npix][D][D]. */
int or_window_moments(const double* cube, int H, int W, int D, int inner, int outer, const int64_t* pix,
                      int64_t npix, double* mu, double* cov, int nthreads) {
    if (inner < 1 || outer <= inner || !(inner & 1) || !(outer & 1) || D < 1) return -1;
    int nmax = outer * outer;
    int* in_dy = (int*)malloc(sizeof(int) * nmax);
    int* in_dx = (int*)malloc(sizeof(int) * nmax);
    int* bg_dy = (int*)malloc(sizeof(int) * nmax);
    int* bg_dx = (int*)malloc(sizeof(int) * nmax);
    int N;
    window_lists(inner, outer, in_dy, in_dx, bg_dy, bg_dx, &N);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 2)
    for (int64_t t = 0; t < npix; ++t) {
        int py = (int)(pix[t] / W), px = (int)(pix[t] % W);
        double* m = mu + t * D;
        double* c = cov + t * (int64_t)D * D;
        for (int k = 0; k < D; ++k) m[k] = 0.0;
        for (int s = 0; s < N; ++s) {
            const double* x = cube + ((int64_t)or_reflect(py + bg_dy[s], H) * W + or_reflect(px + bg_dx[s], W)) * D;
            for (int k = 0; k < D; ++k) m[k] += x[k];
        }
        for (int k = 0; k < D; ++k) m[k] /= N;
        for (int64_t i = 0; i < (int64_t)D * D; ++i) c[i] = 0.0;
        for (int s = 0; s < N; ++s) {
            const double* x = cube + ((int64_t)or_reflect(py + bg_dy[s], H) * W + or_reflect(px + bg_dx[s], W)) * D;
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) c[(int64_t)a * D + b] += (x[a] - m[a]) * (x[b] - m[b]);
        }
        for (int64_t i = 0; i < (int64_t)D * D; ++i) c[i] /= N;
    }
    free(in_dy); free(in_dx); free(bg_dy); free(bg_dx);
    return 0;
}

/* Window census: for every listed pixel, the background and inner multisets as
 * (count, sum of linear indices, sum of squared linear indices).  Integer and
 * exact; used to pin the reflect-101 window indexing. */
int or_window_census(int H, int W, int inner, int outer, int border, const int64_t* pix, int64_t npix,
                     int64_t* out /* npix x 6: nb, sum_b, sumsq_b, ni, sum_i, sumsq_i */) {
    if (inner < 1 || outer <= inner || !(inner & 1) || !(outer & 1)) return -1;
    int ri = inner / 2, ro = outer / 2;
    for (int64_t t = 0; t < npix; ++t) {
        int py = (int)(pix[t] / W), px = (int)(pix[t] % W);
        int64_t* o = out + 6 * t;
        for (int k = 0; k < 6; ++k) o[k] = 0;
        if (border == 1 && (py - ro < 0 || py + ro >= H || px - ro < 0 || px + ro >= W)) {
            for (int k = 0; k < 6; ++k) o[k] = -1;
            continue;
        }
        for (int dy = -ro; dy <= ro; ++dy)
            for (int dx = -ro; dx <= ro; ++dx) {
                int64_t q = (int64_t)or_reflect(py + dy, H) * W + or_reflect(px + dx, W);
                int in = abs(dy) <= ri && abs(dx) <= ri;
                int64_t* s = o + (in ? 3 : 0);
                s[0] += 1; s[1] += q; s[2] += q * q;
            }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Pixel-level ROC AUC (Sec. 5.3.1): Mann-Whitney U with tied scores counted  */
/* one half, AUC = U / (n_pos n_neg).  NaN scores rank lowest.                */
/* ------------------------------------------------------------------------ */
typedef struct { double s; int pos; } or_sp;
static int cmp_sp(const void* a, const void* b) {
    double x = ((const or_sp*)a)->s, y = ((const or_sp*)b)->s;
    return (x < y) ? -1 : (x > y) ? 1 : 0;
}
double or_auc(const double* score, const uint8_t* mask, int64_t n) {
    or_sp* v = (or_sp*)malloc(sizeof(or_sp) * n);
    int64_t npos = 0;
    for (int64_t i = 0; i < n; ++i) {
        v[i].s = isnan(score[i]) ? -INFINITY : score[i];
        v[i].pos = mask[i] ? 1 : 0;
        npos += v[i].pos;
    }
    int64_t nneg = n - npos;
    if (npos == 0 || nneg == 0) { free(v); return NAN; }
    qsort(v, n, sizeof(or_sp), cmp_sp);
    double rank_sum = 0.0;
    int64_t i = 0;
    while (i < n) {
        int64_t j = i;
        while (j + 1 < n && v[j + 1].s == v[i].s) j++;
        double mid = 0.5 * ((double)(i + 1) + (double)(j + 1)); /* average 1-based rank */
        for (int64_t k = i; k <= j; ++k) if (v[k].pos) rank_sum += mid;
        i = j + 1;
    }
    free(v);
    double U = rank_sum - 0.5 * (double)npos * (double)(npos + 1);
    return U / ((double)npos * (double)nneg);
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Adaptive cut-off of Eq. 12: tau = mu_d + z * sigma_d, with mu_d and sigma_d the mean and the
 * (population, 1/n) standard deviation of the anomaly matrix over its finite entries; a
 * pixel is declared anomalous when its score exceeds tau (NaN scores never are).  Two
 * passes.  Returns the number of finite scores; mask may be NULL.
 */
int64_t or_adaptive_threshold(const double* score, int64_t n, double z, double* mu, double* sigma, double* tau,
                              uint8_t* mask) {
    int64_t m = 0;
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (isfinite(score[i])) { s += score[i]; ++m; }
    const double mean = m > 0 ? s / (double)m : NAN;
    double ss = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (isfinite(score[i])) ss += (score[i] - mean) * (score[i] - mean);
    const double sd = m > 0 ? sqrt(ss / (double)m) : NAN;
    const double t = mean + z * sd;
    if (mu) *mu = mean;
    if (sigma) *sigma = sd;
    if (tau) *tau = t;
    if (mask)
        for (int64_t i = 0; i < n; ++i) mask[i] = (uint8_t)(isfinite(score[i]) && score[i] > t);
    return m;
}
