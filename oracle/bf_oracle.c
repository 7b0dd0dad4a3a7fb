/*
 * Plain FP64 CPU oracle for the shiftable-kernel bilateral filter.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file; only the tests, the package's smoke check and the bench's
 * CPU-baseline leg use it. It shares no code, header, table or constant with
 * the CUDA path.
 *
 * What it computes is the plain definition of the bilateral filter
 * (Eq. "filter2", Sec. 2):
 *
 *     out(x) = sum_{y in W(x)} w(x,y) f(y) / sum_{y in W(x)} w(x,y)
 *
 * with a box spatial kernel over the square neighbourhood (Sec. 2, the
 * moving-sum window) and the raised-cosine range kernel
 * q_N(t) = cos^N(gamma t), gamma = pi/(2T) (Sec. 3, kernel q_N).
 * The window is truncated at the image border: only pixels inside the image
 * are summed. cos^N is evaluated directly (one cos, then exponentiation by
 * squaring), never through the trigonometric expansion the fast method uses,
 * so the fast path's O(1) result can be compared against the O(r^2) sum.
 *
 * Also here: the exact-Gaussian bilateral filter (the kernel q_N approximates,
 * Theorem "Gaussian approximation", Eq. approx2) and the analytic gradient of
 * L = sum_x g(x) out(x) with respect to the image and to gamma, derived from
 * the direct form of Eq. filter2.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* cos(a)^N by repeated squaring; N >= 0. N = 0 gives 1 (also for cos = 0). */
static double pow_int(double c, int N) {
    double acc = 1.0, base = c;
    int e = N;
    while (e > 0) {
        if (e & 1) acc *= base;
        base *= base;
        e >>= 1;
    }
    return acc;
}

/* Range kernel q_N evaluated at a difference t (Sec. 3): cos^N(gamma t). */
double oracle_weight(double t, double gamma, int N) {
    return pow_int(cos(gamma * t), N);
}

/* d/dt of cos^N(gamma t) = -N gamma cos^{N-1}(gamma t) sin(gamma t). */
static double weight_dt(double t, double gamma, int N) {
    if (N == 0) return 0.0;
    return -(double)N * gamma * pow_int(cos(gamma * t), N - 1) * sin(gamma * t);
}

/* d/dgamma of cos^N(gamma t) = -N t cos^{N-1}(gamma t) sin(gamma t). */
static double weight_dgamma(double t, double gamma, int N) {
    if (N == 0) return 0.0;
    return -(double)N * t * pow_int(cos(gamma * t), N - 1) * sin(gamma * t);
}

static int imin(int a, int b) { return a < b ? a : b; }
static int imax(int a, int b) { return a > b ? a : b; }

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Raised-cosine bilateral filter by its definition (Eq. filter2 with the box
 * spatial kernel of the moving sum, Sec. 2, and range kernel q_N, Sec. 3).
 * f: H x W row-major. Rows [row0, row1) of out/den are written (den may be
 * NULL); the full image is always read. Returns 0, or -1 on bad arguments.
 */
int oracle_bf_cosn_rows(const double* f, int H, int W, int r, double gamma, int N,
                        int row0, int row1, double* out, double* den) {
    if (!f || !out || H <= 0 || W <= 0 || r < 0 || N < 0) return -1;
    if (row0 < 0) row0 = 0;
    if (row1 > H) row1 = H;
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = row0; y < row1; ++y) {
        for (int x = 0; x < W; ++x) {
            const double fx = f[(size_t)y * W + x];
            double num = 0.0, eta = 0.0;
            for (int yy = imax(0, y - r); yy <= imin(H - 1, y + r); ++yy) {
                for (int xx = imax(0, x - r); xx <= imin(W - 1, x + r); ++xx) {
                    const double fy = f[(size_t)yy * W + xx];
                    const double w = oracle_weight(fy - fx, gamma, N);
                    num += w * fy;
                    eta += w;
                }
            }
            out[(size_t)(y - row0) * W + x] = num / eta;
            if (den) den[(size_t)(y - row0) * W + x] = eta;
        }
    }
    return 0;
}

int oracle_bf_cosn(const double* f, int H, int W, int r, double gamma, int N,
                   double* out, double* den) {
    return oracle_bf_cosn_rows(f, H, W, r, gamma, N, 0, H, out, den);
}

/* Values at a list of pixels only (for sampled checks of large images). */
int oracle_bf_cosn_points(const double* f, int H, int W, int r, double gamma, int N,
                          const long long* idx, long long n, double* out, double* den) {
    if (!f || !idx || !out || H <= 0 || W <= 0 || r < 0 || N < 0 || n < 0) return -1;
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) {
        const long long p = idx[i];
        const int y = (int)(p / W), x = (int)(p % W);
        const double fx = f[p];
        double num = 0.0, eta = 0.0;
        for (int yy = imax(0, y - r); yy <= imin(H - 1, y + r); ++yy)
            for (int xx = imax(0, x - r); xx <= imin(W - 1, x + r); ++xx) {
                const double fy = f[(size_t)yy * W + xx];
                const double w = oracle_weight(fy - fx, gamma, N);
                num += w * fy;
                eta += w;
            }
        out[i] = num / eta;
        if (den) den[i] = eta;
    }
    return 0;
}

/*
 * Exact-Gaussian bilateral filter over the same truncated box window, with
 * range kernel exp(-t^2 / (2 sigma^2)): the kernel that q_N approximates
 * (Theorem "Gaussian approximation", Eq. approx2). Used for the approximation
 * error, which is reported, not asserted.
 */
int oracle_bf_gauss(const double* f, int H, int W, int r, double sigma, double* out) {
    if (!f || !out || H <= 0 || W <= 0 || r < 0 || !(sigma > 0)) return -1;
    const double inv = 1.0 / (2.0 * sigma * sigma);
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const double fx = f[(size_t)y * W + x];
            double num = 0.0, eta = 0.0;
            for (int yy = imax(0, y - r); yy <= imin(H - 1, y + r); ++yy)
                for (int xx = imax(0, x - r); xx <= imin(W - 1, x + r); ++xx) {
                    const double fy = f[(size_t)yy * W + xx];
                    const double t = fy - fx;
                    const double w = exp(-t * t * inv);
                    num += w * fy;
                    eta += w;
                }
            out[(size_t)y * W + x] = num / eta;
        }
    return 0;
}

/*
 * Gradient of L = sum_x g(x) out(x), out from Eq. filter2 with q_N, taken on
 * the direct form. With t = f(y) - f(x), w = cos^N(gamma t), w' = dw/dt:
 *   d out(x)/d f(y) = [w + w' (f(y) - out(x))] / den(x)            (y != x)
 *   d out(x)/d f(x) = [1 - sum_{y != x} w' (f(y) - out(x))] / den(x)
 *   d out(x)/d gamma = sum_y (dw/dgamma) (f(y) - out(x)) / den(x)
 * dL/df(p) gathers over the outputs x whose window holds p; the truncated box
 * window is symmetric, so those x are the window of p. grad_gamma may be NULL.
 */
int oracle_bf_grad(const double* f, const double* g, int H, int W, int r,
                   double gamma, int N, double* grad_f, double* grad_gamma) {
    if (!f || !g || !grad_f || H <= 0 || W <= 0 || r < 0 || N < 0) return -1;
    const size_t n = (size_t)H * W;
    double* out = (double*)malloc(n * sizeof(double));
    double* den = (double*)malloc(n * sizeof(double));
    double* self = (double*)malloc(n * sizeof(double)); /* d out(x)/d f(x) */
    if (!out || !den || !self) { free(out); free(den); free(self); return -2; }
    oracle_bf_cosn(f, H, W, r, gamma, N, out, den);
    double ggam = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : ggam)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const size_t px = (size_t)y * W + x;
            const double fx = f[px], o = out[px], d = den[px];
            double s = 0.0, dg = 0.0;
            for (int yy = imax(0, y - r); yy <= imin(H - 1, y + r); ++yy)
                for (int xx = imax(0, x - r); xx <= imin(W - 1, x + r); ++xx) {
                    const double fy = f[(size_t)yy * W + xx];
                    const double t = fy - fx;
                    if (yy != y || xx != x) s += weight_dt(t, gamma, N) * (fy - o);
                    dg += weight_dgamma(t, gamma, N) * (fy - o);
                }
            self[px] = (1.0 - s) / d;
            ggam += g[px] * dg / d;
        }
#pragma omp parallel for schedule(dynamic, 1)
    for (int py = 0; py < H; ++py)
        for (int pxx = 0; pxx < W; ++pxx) {
            const size_t p = (size_t)py * W + pxx;
            const double fp = f[p];
            double acc = g[p] * self[p];
            for (int y = imax(0, py - r); y <= imin(H - 1, py + r); ++y)
                for (int x = imax(0, pxx - r); x <= imin(W - 1, pxx + r); ++x) {
                    if (y == py && x == pxx) continue;
                    const size_t q = (size_t)y * W + x;
                    const double t = fp - f[q];
                    const double w = oracle_weight(t, gamma, N);
                    const double wd = weight_dt(t, gamma, N);
                    acc += g[q] * (w + wd * (fp - out[q])) / den[q];
                }
            grad_f[p] = acc;
        }
    if (grad_gamma) *grad_gamma = ggam;
    free(out); free(den); free(self);
    return 0;
}

/*
 * Generalised neighbourhood filter by its definition, for the variants of
 * Algorithms 1-2 beyond the box / q_N pair (Sec. 2, Sec. 3):
 *
 *   out(x) = sum_{y in W(x)} phi(y - x) w(f(y) - f(x)) f(y)
 *            / sum_{y in W(x)} phi(y - x) w(f(y) - f(x))
 *
 * over the same truncated (2r+1)^2 window.
 *
 * Spatial kernel phi (spatial = 0: box, phi = 1; spatial = 1: the separable
 * kernel q_M(d1) q_M(d2) of Sec. 3 with q_M(d) = cos^M(pi d / (2 Ts)) on
 * [-Ts, Ts], Ts = r + 1/2, so that the window |d| <= r lies inside the
 * kernel's support).
 *
 * Range kernel w (range = 0: none, w = 1, i.e. Algorithm 1's linear
 * filter; 1: q_N, cos^N(gamma t); 2: q_N with its shift expansion cut to the
 * K_keep lowest harmonics, sum_{i < K_keep} a_i cos(k_i gamma t), k_i =
 * N mod 2 + 2i, a_i = 2^(1-N) C(N, (N-k_i)/2) (halved for k = 0) -- the
 * "discard the less significant basis functions" of the end of Sec. 3;
 * 3: p_N(t) = (1 - t^2/T^2)^N with T = Tr).
 * Rows [row0, row1) are written; den may be NULL.
 */
static double binom(int n, int k) {
    double c = 1.0;
    if (k < 0 || k > n) return 0.0;
    if (k > n - k) k = n - k;
    for (int i = 1; i <= k; ++i) c = c * (double)(n - k + i) / (double)i;
    return c;
}

double oracle_trunc_weight(double t, double gamma, int N, int K_keep) {
    double w = 0.0;
    for (int i = 0; i < K_keep && 2 * i + (N & 1) <= N; ++i) {
        const int k = (N & 1) + 2 * i;
        double a = ldexp(binom(N, (N - k) / 2), 1 - N);
        if (k == 0) a *= 0.5;
        w += a * cos((double)k * gamma * t);
    }
    return w;
}

static double range_weight(int range, double t, double gamma, int N, int K_keep, double Tr) {
    switch (range) {
        case 0: return 1.0;
        case 1: return oracle_weight(t, gamma, N);
        case 2: return oracle_trunc_weight(t, gamma, N, K_keep);
        default: {
            const double u = 1.0 - (t * t) / (Tr * Tr);
            return pow_int(u, N);
        }
    }
}

double oracle_spatial_weight(int d, int r, int M) {
    return pow_int(cos(acos(-1.0) * (double)d / (2.0 * ((double)r + 0.5))), M);
}

int oracle_bf_general_rows(const double* f, int H, int W, int r, int spatial, int M, int range,
                           double gamma, int N, int K_keep, double Tr, int row0, int row1,
                           double* out, double* den) {
    if (!f || !out || H <= 0 || W <= 0 || r < 0 || N < 0 || M < 0) return -1;
    if (range < 0 || range > 3 || spatial < 0 || spatial > 1) return -1;
    if (range == 3 && !(Tr > 0)) return -1;
    if (row0 < 0) row0 = 0;
    if (row1 > H) row1 = H;
    double* sw = (double*)malloc((size_t)(2 * r + 1) * sizeof(double));
    if (!sw) return -2;
    for (int d = -r; d <= r; ++d) sw[d + r] = spatial ? oracle_spatial_weight(d, r, M) : 1.0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = row0; y < row1; ++y) {
        for (int x = 0; x < W; ++x) {
            const double fx = f[(size_t)y * W + x];
            double num = 0.0, eta = 0.0;
            for (int yy = imax(0, y - r); yy <= imin(H - 1, y + r); ++yy) {
                for (int xx = imax(0, x - r); xx <= imin(W - 1, x + r); ++xx) {
                    const double fy = f[(size_t)yy * W + xx];
                    const double w = sw[yy - y + r] * sw[xx - x + r] *
                                     range_weight(range, fy - fx, gamma, N, K_keep, Tr);
                    num += w * fy;
                    eta += w;
                }
            }
            out[(size_t)(y - row0) * W + x] = num / eta;
            if (den) den[(size_t)(y - row0) * W + x] = eta;
        }
    }
    free(sw);
    return 0;
}

/* Exact-Gaussian bilateral filter at a list of flat pixel indices only (for
   the approximation error on large images). */
int oracle_bf_gauss_points(const double* f, int H, int W, int r, double sigma,
                           const long long* idx, long long n, double* out) {
    if (!f || !idx || !out || H <= 0 || W <= 0 || r < 0 || !(sigma > 0) || n < 0) return -1;
    const double inv = 1.0 / (2.0 * sigma * sigma);
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) {
        const long long p = idx[i];
        const int y = (int)(p / W), x = (int)(p % W);
        const double fx = f[p];
        double num = 0.0, eta = 0.0;
        for (int yy = imax(0, y - r); yy <= imin(H - 1, y + r); ++yy)
            for (int xx = imax(0, x - r); xx <= imin(W - 1, x + r); ++xx) {
                const double fy = f[(size_t)yy * W + xx];
                const double t = fy - fx;
                const double w = exp(-t * t * inv);
                num += w * fy;
                eta += w;
            }
        out[i] = num / eta;
    }
    return 0;
}
