// Host side of the C ABI (include/bf.h): argument checks, the parameter
// rules of the paper (gamma of q_N, order rule, interpolating coefficients),
// tile choice and kernel launches. No device memory is allocated here.
#include <math.h>
#include <string.h>

#include "bf_internal.cuh"

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

bf_status resolve(int r, float sigma_r, float T, int N, int gamma_mode, Resolved* out) {
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

// The skewed-strip engine serves r <= 32, K <= SYS_KMAX and plain (not
// Kahan) sums; thread count 64, 96 or 128 (one thread per strip column,
// Tw = Wi - 2r outputs). Bands: about two resident CTAs per SM.
static bool sys_tiles(int H, int W, int r, int K, const bf_opts* o, Tiles* t) {
    if (K > SYS_KMAX || (o && o->kahan)) return false;
    int wi = 128;
    if (o && o->tile_w > 0) {
        if (o->tile_w > SYS_MAX_THREADS || o->tile_w % 32 != 0) return false;
        wi = o->tile_w;
    }
    if (wi - 2 * r < 16) return false;
    t->nt = wi;
    t->Tw = wi - 2 * r;
    t->gx = (W + t->Tw - 1) / t->Tw;
    if (o && o->tile_h > 0) {
        t->Hb = o->tile_h;
    } else {
        const int target = 2 * sm_count();
        int nb = (target + t->gx - 1) / t->gx;
        if (nb < 1) nb = 1;
        int hb = (H + nb - 1) / nb;
        if (hb < 32) hb = 32;
        t->Hb = hb;
    }
    t->gy = (H + t->Hb - 1) / t->Hb;
    return true;
}

bf_status check_opts(const bf_opts* o) {
    if (!o) return BF_OK;
    if (o->in_dtype != BF_F32 && o->in_dtype != BF_BF16) return BF_ERR_INVALID_ARG;
    if (o->gamma_mode != BF_GAMMA_FIXED && o->gamma_mode != BF_GAMMA_FROM_SIGMA)
        return BF_ERR_INVALID_ARG;
    if (o->tile_h < 0 || o->tile_w < 0) return BF_ERR_INVALID_ARG;
    return BF_OK;
}

bf_status fill_fwd_params(const void* img, float* out, void* saved, int H, int W, int r,
                          float sigma_r, float T, int N, const bf_opts* opts, FwdParams* pp,
                          int* nt, int* gx, int* gy) {
    if (!img || !out || H < 1 || W < 1) return BF_ERR_INVALID_ARG;
    if ((const void*)out == img) return BF_ERR_INVALID_ARG;
    bf_status st = check_opts(opts);
    if (st != BF_OK) return st;
    const int gm = opts ? opts->gamma_mode : BF_GAMMA_FIXED;
    Resolved rs;
    st = resolve(r, sigma_r, T, N, gm, &rs);
    if (st != BF_OK) return st;
    Tiles t;
    st = choose_tiles(H, W, r, opts, &t);
    if (st != BF_OK) return st;
    if (opts && opts->save_for_backward && !saved) return BF_ERR_INVALID_ARG;
    FwdParams& p = *pp;
    memset(&p, 0, sizeof(p));
    p.img = img;
    p.out = out;
    if (saved) {
        float* s = static_cast<float*>(saved);
        const size_t n = (size_t)H * W;
        p.sv_den = s;
        p.sv_dnum = s + n;
        p.sv_dden = s + 2 * n;
    }
    p.H = H; p.W = W; p.r = r; p.K = rs.K; p.kstart = rs.kstart;
    p.Hb = t.Hb; p.Tw = t.Tw;
    p.gamma = (float)rs.gamma;
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
    return (size_t)3 * (size_t)H * (size_t)W * sizeof(float);
}

bf_status bf_forward(const void* img, int H, int W, int r, float sigma_r, float T, int N,
                     float* out, const bf_opts* opts, void* saved, void* stream) {
    FwdParams p;
    int nt = 0, gx = 0, gy = 0;
    bf_status st = fill_fwd_params(img, out, saved, H, W, r, sigma_r, T, N, opts, &p, &nt,
                                   &gx, &gy);
    if (st != BF_OK) return st;
    const int in_dtype = opts ? opts->in_dtype : BF_F32;
    Tiles t;
    cudaError_t e;
    if (sys_tiles(H, W, r, p.K, opts, &t)) {
        SysParams q;
        memset(&q, 0, sizeof(q));
        q.img = img; q.out = out;
        q.sv_den = p.sv_den; q.sv_dnum = p.sv_dnum; q.sv_dden = p.sv_dden;
        q.H = H; q.W = W; q.r = r; q.K = p.K; q.kstart = p.kstart; q.Hb = t.Hb; q.Tw = t.Tw;
        q.gamma = p.gamma;
        for (int i = 0; i < p.K; ++i) {
            q.a[i] = p.a[i];
            q.ak[i] = p.a[i] * (float)(p.kstart + 2 * i);
        }
        e = launch_sys(q, false, saved != nullptr, in_dtype, t.nt, t.gx, t.gy,
                       (cudaStream_t)stream);
    } else {
        e = launch_forward(p, nt, opts ? opts->kahan : 0, in_dtype, (cudaStream_t)stream);
    }
    if (e != cudaSuccess) return set_cuda_error(e);
    return BF_OK;
}

size_t bf_backward_workspace_bytes(int H, int W, int r, const bf_opts* opts) {
    if (H < 1 || W < 1 || r < 0 || r > BF_R_MAX) return 0;
    Tiles t, u;
    if (choose_tiles(H, W, r, opts, &t) != BF_OK) return 0;
    size_t n = (size_t)t.gx * t.gy;
    if (sys_tiles(H, W, r, 1, opts, &u) && (size_t)u.gx * u.gy > n) n = (size_t)u.gx * u.gy;
    return n * sizeof(float);
}

bf_status bf_backward(const void* img, const float* out, const float* grad_out,
                      const void* saved, int H, int W, int r, float sigma_r, float T, int N,
                      float* grad_img, float* grad_sigma, void* workspace, size_t ws_bytes,
                      const bf_opts* opts, void* stream) {
    if (!img || !out || !grad_out || !saved || H < 1 || W < 1) return BF_ERR_INVALID_ARG;
    if (!grad_img && !grad_sigma) return BF_ERR_INVALID_ARG;
    bf_status st = check_opts(opts);
    if (st != BF_OK) return st;
    const int gm = opts ? opts->gamma_mode : BF_GAMMA_FIXED;
    Resolved rs;
    st = resolve(r, sigma_r, T, N, gm, &rs);
    if (st != BF_OK) return st;
    Tiles t;
    const bool use_sys = sys_tiles(H, W, r, rs.K, opts, &t);
    if (!use_sys) {
        st = choose_tiles(H, W, r, opts, &t);
        if (st != BF_OK) return st;
    }
    const size_t need = (size_t)t.gx * t.gy * sizeof(float);
    if (grad_sigma && gm == BF_GAMMA_FROM_SIGMA && (!workspace || ws_bytes < need))
        return BF_ERR_NOMEM;

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
    const float* sv = static_cast<const float*>(saved);
    const size_t n = (size_t)H * W;
    p.img = img; p.out = out; p.gout = grad_out;
    p.sv_den = sv; p.sv_dnum = sv + n; p.sv_dden = sv + 2 * n;
    p.gimg = grad_img;
    p.partial = want_sigma ? static_cast<float*>(workspace) : nullptr;
    p.H = H; p.W = W; p.r = r; p.K = rs.K; p.kstart = rs.kstart; p.Hb = t.Hb; p.Tw = t.Tw;
    p.gamma = (float)rs.gamma;
    for (int i = 0; i < rs.K; ++i) p.a[i] = (float)rs.a[i];
    cudaError_t e;
    if (use_sys) {
        SysParams q;
        memset(&q, 0, sizeof(q));
        q.img = img; q.fout = out; q.gout = grad_out;
        q.bden = p.sv_den; q.bdnum = p.sv_dnum; q.bdden = p.sv_dden;
        q.gimg = grad_img; q.partial = p.partial;
        q.H = H; q.W = W; q.r = r; q.K = p.K; q.kstart = p.kstart; q.Hb = t.Hb; q.Tw = t.Tw;
        q.gamma = p.gamma;
        for (int i = 0; i < p.K; ++i) {
            q.a[i] = p.a[i];
            q.ak[i] = p.a[i] * (float)(p.kstart + 2 * i);
        }
        e = launch_sys(q, true, false, opts ? opts->in_dtype : BF_F32, t.nt, t.gx, t.gy, s);
    } else {
        e = launch_backward(p, t.nt, opts ? opts->in_dtype : BF_F32, s);
    }
    if (e != cudaSuccess) return set_cuda_error(e);
    if (want_sigma) {
        // dL/dsigma_r = dL/dgamma * dgamma/dsigma_r, gamma = 1/(sigma_r sqrt N).
        const float scale = (float)(-rs.gamma / (double)sigma_r);
        e = launch_reduce_sigma(p.partial, t.gx * t.gy, scale, grad_sigma, s);
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    return BF_OK;
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
