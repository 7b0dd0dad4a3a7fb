// Host side of the C ABI (include/bf.h): argument checks, the parameter
// rules of the paper (gamma of q_N, order rule, interpolating coefficients),
// tile choice and kernel launches. No device memory is allocated here.
#include <math.h>
#include <string.h>

#include "bf_internal.cuh"
#include "bf_trace.cuh"

namespace bf {

static thread_local int g_last_cuda = 0;

bf_status set_cuda_error(cudaError_t e) {
    g_last_cuda = (int)e;
    return BF_ERR_CUDA;
}

static double gamma_fixed(double T) { return M_PI / (2.0 * T); }

// a_k = 2^(1-N) C(N, (N-k)/2) for k > 0 and 2^(-N) C(N, N/2) for k = 0:
// the binomial expansion of cos^N written with the shift identity of
// Sec. 1 (pairs n, N-n fold onto one harmonic |N - 2n|). Computed as a
// running product so no intermediate exceeds FP64 range.
static int coeffs(int N, double* a, int cap) {
    if (N < 0 || N > BF_N_MAX) return -1;
    const int K = N / 2 + 1;
    if (cap < K || !a) return -1;
    // b[m] = 2^-N C(N, m) for m = 0..N, by b[m+1] = b[m] (N-m)/(m+1).
    double b[BF_N_MAX + 1];
    b[0] = ldexp(1.0, -N);
    for (int m = 0; m < N; ++m) b[m + 1] = b[m] * (double)(N - m) / (double)(m + 1);
    const int kstart = N & 1;
    for (int i = 0; i < K; ++i) {
        const int k = kstart + 2 * i;
        const int m = (N - k) / 2;
        a[i] = (k == 0) ? b[m] : 2.0 * b[m];
    }
    return K;
}

// Number of harmonics of q_N's expansion kept under a kernel tolerance
// (the end of Sec. 3: discard the less significant basis functions). The
// highest harmonics have the smallest a_k; dropping a set of them changes the
// kernel by at most the sum of their a_k (|cos| <= 1), attained at t = 0. The
// dropped sum is kept <= min(tol, 1 / (2 (2r+1)^2)), so the truncated kernel
// is above -1/(2 (2r+1)^2) everywhere and den >= 1 - 1/2 stays positive.
static int trunc_keep(const double* a, int K, int r, double tol) {
    if (!(tol > 0.0)) return K;
    const double n = (double)(2 * r + 1) * (double)(2 * r + 1);
    const double cap = tol < 0.5 / n ? tol : 0.5 / n;
    double tail = 0.0;
    int keep = K;
    while (keep > 1 && tail + a[keep - 1] <= cap) tail += a[--keep];
    return keep;
}

bf_status resolve(int r, float sigma_r, float T, int N, int gamma_mode, float trunc_tol,
                  Resolved* out) {
    if (!(T > 0.f) || !isfinite(T)) return BF_ERR_INVALID_ARG;
    if (r < 0) return BF_ERR_INVALID_ARG;
    if (r > BF_R_MAX) return BF_ERR_UNSUPPORTED;
    if (gamma_mode != BF_GAMMA_FIXED && gamma_mode != BF_GAMMA_FROM_SIGMA)
        return BF_ERR_INVALID_ARG;
    if (N <= 0) {
        if (N < 0 || !(sigma_r > 0.f)) {
            // N == 0 with a valid sigma_r means "derive"; N < 0 too.
            if (!(sigma_r > 0.f)) return BF_ERR_INVALID_ARG;
        }
        N = bf_resolve_N(sigma_r, T);
        if (N < 0) return BF_ERR_INVALID_ARG;
    }
    if (N > BF_N_MAX) return BF_ERR_UNSUPPORTED;
    out->N = N;
    out->kstart = N & 1;
    out->K = coeffs(N, out->a, KCAP);
    if (out->K < 0) return BF_ERR_INTERNAL;
    out->K = trunc_keep(out->a, out->K, r, (double)trunc_tol);
    const double g = bf_gamma(sigma_r, T, N, gamma_mode);
    if (!(g > 0.0)) return BF_ERR_INVALID_ARG;
    out->gamma = g;
    return BF_OK;
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
    return n > 0 ? n : 148;
}

struct Tiles {
    int nt, Tw, Hb, gx, gy;
};

// Strip width: 256 threads (one per input column), Tw = 256 - 2r outputs.
// Band height: enough bands that the grid covers about two waves of SMs.
static bf_status choose_tiles(int H, int W, int r, const bf_opts* o, Tiles* t) {
    int nt = (o && o->tile_w > 0) ? o->tile_w : 256;
    if (nt % 32 != 0 || nt > 256 || nt - 2 * r < 1) return BF_ERR_INVALID_ARG;
    t->nt = nt;
    t->Tw = nt - 2 * r;
    t->gx = (W + t->Tw - 1) / t->Tw;
    if (o && o->tile_h > 0) {
        t->Hb = o->tile_h;
    } else {
        const int target = 2 * sm_count();
        int nb = (target + t->gx - 1) / t->gx;
        if (nb < 1) nb = 1;
        int hb = (H + nb - 1) / nb;
        if (hb < 16) hb = 16;
        t->Hb = hb;
    }
    t->gy = (H + t->Hb - 1) / t->Hb;
    return BF_OK;
}

// Whether launch_sys runs the first-chunk kernels (bf_sys_first*.cu) of
// 64-thread strips for this request: compact rows, plain sums, one harmonic
// chunk, a seed the first chunk specialises (odd N, or even N with harmonics
// beside the constant one), and FP32 input -- or the adjoint, which reads only
// the saved quads.
static bool first_chunk_path(int K, int kstart, int ld, int W, const bf_opts* o, bool kahan,
                             bool adjoint = false) {
    const int dtype = o ? o->in_dtype : BF_F32;
    return (adjoint || dtype == BF_F32) && ld == W && !kahan &&
           sys_chunks(K, false, o ? o->kp_max : 0) == 1 && (kstart == 1 || K > 1);
}

// Band shape of strips of wi threads: one wave of `slots` resident CTAs over
// the B images' strips (rounding the band count up would start a second,
// nearly empty wave), at least 32 rows. Returns the model cost, waves x steps
// per CTA (a CTA of wi lanes sweeps its band, the 2r warm-up rows and the
// wi - 1 steps of the skew ramp; a full SM runs the same number of lane-steps
// per step at either strip width).
static long long band_shape(int H, int W, int r, int wi, int B, int slots, Tiles* t) {
    t->nt = wi;
    t->Tw = wi - 2 * r;
    t->gx = (W + t->Tw - 1) / t->Tw;
    int nb = slots / (t->gx * (B > 1 ? B : 1));
    if (nb < 1) nb = 1;
    int hb = (H + nb - 1) / nb;
    if (hb < 32) hb = 32;
    t->Hb = hb;
    t->gy = (H + t->Hb - 1) / t->Hb;
    const long long ctas = (long long)t->gx * t->gy * (B > 1 ? B : 1);
    const long long waves = (ctas + slots - 1) / slots;
    return waves * (long long)(t->Hb + 2 * r + wi - 1);
}

// The skewed-strip engine (bf_sys.cu) serves every request whose strip of
// Wi threads keeps at least 16 output columns (Wi - 2r >= 16): 128-thread
// strips up to r = 40 (two CTAs per SM: measured faster than wider strips
// with one CTA per SM even at r = 30, where half the lanes are halo),
// 256-thread strips above. Bands: one wave of resident CTAs; the B images of
// a [B, H, W] launch share the wave. When the launch runs the first-chunk
// kernels (narrow64: FP32, compact, one harmonic chunk), 64-thread strips
// (four CTAs per SM) are taken where the model cost says they finish sooner:
// small images, whose 128-thread bands are short next to the skew ramp.
// Measured on a GB300 (forward / fwd+bwd against 128-thread strips): 1024^2
// r = 3 1.48x / 1.51x, r = 10 1.33x / 1.37x; 16 x 512^2 r = 7 1.22x;
// 4096^2 r = 3 1.09x; 4096^2 r = 10 0.85x, where the model keeps 128.
static bool sys_tiles(int H, int W, int ld, int r, const bf_opts* o, Tiles* t, int B = 1,
                      bool narrow64 = false) {
    int wi = (r <= 40) ? 128 : 256;
    const bool fixed_w = o && o->tile_w > 0;
    if (fixed_w) {
        if (o->tile_w > SYS_MAX_THREADS || o->tile_w % 32 != 0) return false;
        wi = o->tile_w;
    }
    if (wi - 2 * r < 16) return false;
    // the engine addresses one image with 32-bit element offsets (rows of the
    // skew ramp above and below the image included)
    if ((long long)(H + 2 * wi + 4 * r) * (ld > W ? ld : W) >= 0x7fffffffLL) return false;
    const int slots = (wi <= 64 ? 4 : wi <= 128 ? 2 : 1) * sm_count();
    const long long cost = band_shape(H, W, r, wi, B, slots, t);
    const bool fixed_h = o && o->tile_h > 0;
    if (!fixed_w && !fixed_h && narrow64 && wi == 128 && 64 - 2 * r >= 16) {
        Tiles t64;
        const long long c64 = band_shape(H, W, r, 64, B, 4 * sm_count(), &t64);
        if (100 * c64 < 97 * cost) *t = t64;  // 3 % margin over the model's error
    }
    if (fixed_h) {
        t->Hb = o->tile_h;
        t->gy = (H + t->Hb - 1) / t->Hb;
    }
    return true;
}

static void fill_sys(const FwdParams& p, SysParams* q) {
    memset(q, 0, sizeof(*q));
    q->img = p.img;
    q->dout = p.den;
    q->H = p.H; q->W = p.W; q->r = p.r; q->K = p.K; q->kstart = p.kstart;
    q->ld = p.ld;
    q->Hb = 0; q->Tw = 0;
    q->k0 = p.kstart;
    q->gamma = p.gamma;
    q->mid = p.mid;
    q->gpi = (float)((double)p.gamma / M_PI);
    for (int i = 0; i < p.K; ++i) {
        q->a[i] = p.a[i];
        q->ak[i] = p.a[i] * (float)(p.kstart + 2 * i);
    }
}

bf_status check_opts(const bf_opts* o) {
    if (!o) return BF_OK;
    if (o->in_dtype != BF_F32 && o->in_dtype != BF_BF16) return BF_ERR_INVALID_ARG;
    if (o->gamma_mode != BF_GAMMA_FIXED && o->gamma_mode != BF_GAMMA_FROM_SIGMA)
        return BF_ERR_INVALID_ARG;
    if (o->tile_h < 0 || o->tile_w < 0) return BF_ERR_INVALID_ARG;
    if (o->kp_max < 0 || o->kp_max > SYS_KP_MAX) return BF_ERR_INVALID_ARG;
    if (!(o->trunc_tol >= 0.f && o->trunc_tol < 1.f)) return BF_ERR_INVALID_ARG;
    if (o->pitch < 0) return BF_ERR_INVALID_ARG;
    return BF_OK;
}

// Row pitch of the image buffers: pitch (from bf_opts or bf_desc) or W when 0;
// -1 when it is shorter than a row.
int row_pitch(int pitch, int W) {
    const int ld = pitch > 0 ? pitch : W;
    return ld < W ? -1 : ld;
}

bf_status fill_fwd_params(const void* img, float* out, void* saved, int H, int W, int pitch,
                          int r, float sigma_r, float T, int N, const bf_opts* opts,
                          FwdParams* pp, int* nt, int* gx, int* gy) {
    if (!img || !out || H < 1 || W < 1) return BF_ERR_INVALID_ARG;
    if ((const void*)out == img) return BF_ERR_INVALID_ARG;
    bf_status st = check_opts(opts);
    if (st != BF_OK) return st;
    const int ld = row_pitch(pitch, W);
    if (ld < 0) return BF_ERR_INVALID_ARG;
    const int gm = opts ? opts->gamma_mode : BF_GAMMA_FIXED;
    Resolved rs;
    st = resolve(r, sigma_r, T, N, gm, opts ? opts->trunc_tol : 0.f, &rs);
    if (st != BF_OK) return st;
    Tiles t;
    st = choose_tiles(H, W, r, opts, &t);
    if (st != BF_OK) return st;
    if (opts && opts->save_for_backward && !saved) return BF_ERR_INVALID_ARG;
    if (saved && ((uintptr_t)saved & 15)) return BF_ERR_INVALID_ARG;  // quads: 16-byte aligned
    FwdParams& p = *pp;
    memset(&p, 0, sizeof(p));
    p.img = img;
    p.out = out;
    p.sv = static_cast<float4*>(saved);
    p.H = H; p.W = W; p.r = r; p.K = rs.K; p.kstart = rs.kstart;
    p.ld = ld;
    p.Hb = t.Hb; p.Tw = t.Tw;
    p.gamma = (float)rs.gamma;
    p.mid = 0.5f * T;
    for (int i = 0; i < rs.K; ++i) p.a[i] = (float)rs.a[i];
    *nt = t.nt; *gx = t.gx; *gy = t.gy;
    return BF_OK;
}

}  // namespace bf

using namespace bf;

extern "C" {

void bf_default_opts(bf_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->gamma_mode = BF_GAMMA_FIXED;
    o->in_dtype = BF_F32;
}

int bf_resolve_N(float sigma_r, float T) {
    if (!(sigma_r > 0.f) || !(T > 0.f) || !isfinite(sigma_r) || !isfinite(T)) return -1;
    const double g = gamma_fixed((double)T);
    const double v = 1.0 / ((g * (double)sigma_r) * (g * (double)sigma_r));
    if (v > 1e9) return BF_N_MAX + 1;
    int n = (int)ceil(v - 1e-9);
    return n < 1 ? 1 : n;
}

int bf_coeffs(int N, double* a, int cap) { return coeffs(N, a, cap); }

int bf_trunc_harmonics(int N, int r, float trunc_tol) {
    if (N < 0 || N > BF_N_MAX || r < 0 || r > BF_R_MAX) return -1;
    if (!(trunc_tol >= 0.f && trunc_tol < 1.f)) return -1;
    double a[KCAP];
    const int K = coeffs(N, a, KCAP);
    if (K < 0) return -1;
    return trunc_keep(a, K, r, (double)trunc_tol);
}

double bf_gamma(float sigma_r, float T, int N, int gamma_mode) {
    if (!(T > 0.f)) return -1.0;
    if (gamma_mode == BF_GAMMA_FIXED) return gamma_fixed((double)T);
    if (gamma_mode == BF_GAMMA_FROM_SIGMA) {
        if (!(sigma_r > 0.f) || N < 1) return -1.0;
        return 1.0 / ((double)sigma_r * sqrt((double)N));
    }
    return -1.0;
}

size_t bf_saved_bytes(int H, int W) {
    if (H < 1 || W < 1) return 0;
    return (size_t)H * (size_t)W * sizeof(float4);
}

static bf_status forward_impl(const void* img, int B, int H, int W, int r, float sigma_r,
                              float T, int N, float* out, const bf_opts* opts, void* saved,
                              void* stream) {
    if (B < 1) return BF_ERR_INVALID_ARG;
    FwdParams p;
    int nt = 0, gx = 0, gy = 0;
    bf_status st = fill_fwd_params(img, out, saved, H, W, opts ? opts->pitch : 0, r, sigma_r, T,
                                   N, opts, &p, &nt, &gx, &gy);
    if (st != BF_OK) return st;
    const int in_dtype = opts ? opts->in_dtype : BF_F32;
    const size_t esz = in_dtype == BF_BF16 ? 2 : 4;
    const bool kahan = opts && opts->kahan;
    Tiles t;
    cudaError_t e = cudaSuccess;
    // harmonic chunks accumulate in the saved buffers, so chunking needs them
    const int kpm = opts ? opts->kp_max : 0;
    if (sys_tiles(H, W, p.ld, r, opts, &t, B, first_chunk_path(p.K, p.kstart, p.ld, W, opts, kahan)) &&
        (sys_chunks(p.K, kahan, kpm) == 1 || saved)) {
        SysParams q;
        fill_sys(p, &q);
        q.out = out;
        q.sv = p.sv;
        q.Hb = t.Hb; q.Tw = t.Tw;
        q.B = B;
        e = launch_sys(q, saved ? 1 : 0, kahan, in_dtype, t.nt, t.gx, t.gy,
                       (cudaStream_t)stream, kpm);
    } else {
        const size_t hw = (size_t)H * W, hp = (size_t)H * p.ld;
        for (int b = 0; b < B && e == cudaSuccess; ++b) {
            FwdParams pb = p;
            pb.img = static_cast<const char*>(img) + b * hp * esz;
            pb.out = out + b * hp;
            if (saved) pb.sv = p.sv + b * hw;
            e = launch_forward(pb, nt, kahan ? 1 : 0, in_dtype, (cudaStream_t)stream);
        }
    }
    if (e != cudaSuccess) return set_cuda_error(e);
    return BF_OK;
}

// Backward workspace layout: per-CTA partial sums, then (when the harmonics
// run in chunks) two H x W float accumulators.
struct BwdWs {
    size_t partial_bytes, acc_offset, total;
    bool chunked;
};

static bf_status bwd_ws(int B, int H, int W, int r, int K, int kstart, const bf_opts* opts,
                        BwdWs* ws, Tiles* t, bool* use_sys) {
    const int ld = row_pitch(opts ? opts->pitch : 0, W);
    if (ld < 0) return BF_ERR_INVALID_ARG;
    // the adjoint always runs plain sums
    *use_sys = sys_tiles(H, W, ld, r, opts, t, B, first_chunk_path(K, kstart, ld, W, opts, false, true));
    if (!*use_sys) {
        bf_status st = choose_tiles(H, W, r, opts, t);
        if (st != BF_OK) return st;
    }
    ws->partial_bytes = (size_t)t->gx * t->gy * B * sizeof(float);
    ws->chunked = *use_sys && sys_chunks(K, false, opts ? opts->kp_max : 0) > 1;
    ws->acc_offset = (ws->partial_bytes + 255) & ~(size_t)255;
    ws->total = ws->chunked ? ws->acc_offset + 2 * (size_t)B * H * W * sizeof(float)
                            : ws->partial_bytes;
    return BF_OK;
}

static size_t backward_ws_impl(int B, int H, int W, int r, float sigma_r, float T, int N,
                               const bf_opts* opts) {
    if (B < 1 || H < 1 || W < 1 || check_opts(opts) != BF_OK) return 0;
    const int gm = opts ? opts->gamma_mode : BF_GAMMA_FIXED;
    Resolved rs;
    if (resolve(r, sigma_r, T, N, gm, opts ? opts->trunc_tol : 0.f, &rs) != BF_OK) return 0;
    BwdWs ws;
    Tiles t;
    bool use_sys = false;
    if (bwd_ws(B, H, W, r, rs.K, rs.kstart, opts, &ws, &t, &use_sys) != BF_OK) return 0;
    return ws.total;
}

static bf_status backward_impl(const void* img, const float* out, const float* grad_out,
                               const void* saved, int B, int H, int W, int r, float sigma_r,
                               float T, int N, float* grad_img, float* grad_sigma, void* workspace,
                               size_t ws_bytes, const bf_opts* opts, void* stream) {
    if (!img || !out || !grad_out || !saved || B < 1 || H < 1 || W < 1) return BF_ERR_INVALID_ARG;
    if (!grad_img && !grad_sigma) return BF_ERR_INVALID_ARG;
    if ((uintptr_t)saved & 15) return BF_ERR_INVALID_ARG;  // quads: 16-byte aligned
    // neighbours' pixels, dL/dout and quads are read while dL/dimg is written
    if (grad_img && ((const void*)grad_img == img || grad_img == out ||
                     grad_img == grad_out || (const void*)grad_img == saved))
        return BF_ERR_INVALID_ARG;
    bf_status st = check_opts(opts);
    if (st != BF_OK) return st;
    const int gm = opts ? opts->gamma_mode : BF_GAMMA_FIXED;
    Resolved rs;
    st = resolve(r, sigma_r, T, N, gm, opts ? opts->trunc_tol : 0.f, &rs);
    if (st != BF_OK) return st;
    Tiles t;
    BwdWs ws;
    bool use_sys = false;
    st = bwd_ws(B, H, W, r, rs.K, rs.kstart, opts, &ws, &t, &use_sys);
    if (st != BF_OK) return st;
    const bool need_ws = ws.chunked || (grad_sigma && gm == BF_GAMMA_FROM_SIGMA);
    if (need_ws && (!workspace || ws_bytes < ws.total)) return BF_ERR_NOMEM;

    cudaStream_t s = (cudaStream_t)stream;
    if (grad_sigma && gm == BF_GAMMA_FIXED) {
        // gamma does not depend on sigma_r: the derivative is exactly 0.
        cudaError_t e = cudaMemsetAsync(grad_sigma, 0, sizeof(float), s);
        if (e != cudaSuccess) return set_cuda_error(e);
        if (!grad_img) return BF_OK;
    }
    const bool want_sigma = grad_sigma && gm == BF_GAMMA_FROM_SIGMA;

    BwdParams p;
    memset(&p, 0, sizeof(p));
    const size_t n = (size_t)H * W;
    p.ld = row_pitch(opts ? opts->pitch : 0, W);
    const size_t np = (size_t)H * p.ld;
    p.img = img; p.gout = grad_out;
    p.sv = static_cast<const float4*>(saved);
    p.gimg = grad_img;
    p.partial = want_sigma ? static_cast<float*>(workspace) : nullptr;
    p.H = H; p.W = W; p.r = r; p.K = rs.K; p.kstart = rs.kstart; p.Hb = t.Hb; p.Tw = t.Tw;
    p.gamma = (float)rs.gamma;
    for (int i = 0; i < rs.K; ++i) p.a[i] = (float)rs.a[i];
    cudaError_t e;
    if (use_sys) {
        FwdParams fp;
        memset(&fp, 0, sizeof(fp));
        fp.img = img; fp.H = H; fp.W = W; fp.r = r; fp.K = p.K; fp.kstart = p.kstart;
        fp.ld = p.ld;
        fp.gamma = p.gamma;
        for (int i = 0; i < p.K; ++i) fp.a[i] = p.a[i];
        SysParams q;
        fill_sys(fp, &q);
        q.gout = grad_out;
        q.bsv = p.sv;
        q.gimg = grad_img; q.partial = p.partial;
        if (ws.chunked) {
            float* acc = reinterpret_cast<float*>(static_cast<char*>(workspace) + ws.acc_offset);
            q.acc_gv = acc;
            q.acc_gt = acc + (size_t)B * H * W;  // both hold B images
        }
        q.Hb = t.Hb; q.Tw = t.Tw;
        q.B = B;
        e = launch_sys(q, 2, false, opts ? opts->in_dtype : BF_F32, t.nt, t.gx, t.gy, s,
                       opts ? opts->kp_max : 0);
    } else {
        const size_t esz = (opts && opts->in_dtype == BF_BF16) ? 2 : 4;
        e = cudaSuccess;
        for (int b = 0; b < B && e == cudaSuccess; ++b) {
            BwdParams pb = p;
            pb.img = static_cast<const char*>(img) + b * np * esz;
            pb.gout = grad_out + b * np;
            pb.sv = p.sv + b * n;
            pb.gimg = grad_img ? grad_img + b * np : nullptr;
            pb.partial = p.partial ? p.partial + (size_t)b * t.gx * t.gy : nullptr;
            e = launch_backward(pb, t.nt, opts ? opts->in_dtype : BF_F32, s);
        }
    }
    if (e != cudaSuccess) return set_cuda_error(e);
    if (want_sigma) {
        // dL/dsigma_r = dL/dgamma * dgamma/dsigma_r, gamma = 1/(sigma_r sqrt N).
        const float scale = (float)(-rs.gamma / (double)sigma_r);
        e = launch_reduce_sigma(p.partial, t.gx * t.gy * B, scale, grad_sigma, s);
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    return BF_OK;
}

size_t bf_backward_workspace_bytes(int H, int W, int r, float sigma_r, float T, int N,
                                   const bf_opts* opts) {
    return backward_ws_impl(1, H, W, r, sigma_r, T, N, opts);
}

size_t bf_backward3d_workspace_bytes(int B, int H, int W, int r, float sigma_r, float T, int N,
                                     const bf_opts* opts) {
    return backward_ws_impl(B, H, W, r, sigma_r, T, N, opts);
}

bf_status bf_forward(const void* img, int H, int W, int r, float sigma_r, float T, int N,
                     float* out, const bf_opts* opts, void* saved, void* stream) {
    BF_TRACE("bf_forward");
    return forward_impl(img, 1, H, W, r, sigma_r, T, N, out, opts, saved, stream);
}

bf_status bf_forward3d(const void* img, int B, int H, int W, int r, float sigma_r, float T, int N,
                       float* out, const bf_opts* opts, void* saved, void* stream) {
    BF_TRACE("bf_forward3d");
    return forward_impl(img, B, H, W, r, sigma_r, T, N, out, opts, saved, stream);
}

bf_status bf_backward(const void* img, const float* out, const float* grad_out,
                      const void* saved, int H, int W, int r, float sigma_r, float T, int N,
                      float* grad_img, float* grad_sigma, void* workspace, size_t ws_bytes,
                      const bf_opts* opts, void* stream) {
    BF_TRACE("bf_backward");
    return backward_impl(img, out, grad_out, saved, 1, H, W, r, sigma_r, T, N, grad_img,
                         grad_sigma, workspace, ws_bytes, opts, stream);
}

bf_status bf_backward3d(const void* img, const float* out, const float* grad_out,
                        const void* saved, int B, int H, int W, int r, float sigma_r, float T,
                        int N, float* grad_img, float* grad_sigma, void* workspace,
                        size_t ws_bytes, const bf_opts* opts, void* stream) {
    BF_TRACE("bf_backward3d");
    return backward_impl(img, out, grad_out, saved, B, H, W, r, sigma_r, T, N, grad_img,
                         grad_sigma, workspace, ws_bytes, opts, stream);
}

const char* bf_status_string(bf_status s) {
    switch (s) {
        case BF_OK: return "ok";
        case BF_ERR_INVALID_ARG: return "invalid argument";
        case BF_ERR_UNSUPPORTED: return "unsupported parameter (N > BF_N_MAX or r > BF_R_MAX)";
        case BF_ERR_CUDA: return "CUDA error (see bf_last_cuda_error)";
        case BF_ERR_TIMEOUT: return "bounded device wait timed out";
        case BF_ERR_INTERNAL: return "internal error";
        case BF_ERR_NOMEM: return "caller-supplied buffer too small";
    }
    return "unknown status";
}

bf_status bf_last_cuda_error(int* code) {
    if (!code) return BF_ERR_INVALID_ARG;
    *code = g_last_cuda;
    return BF_OK;
}

}  // extern "C"
