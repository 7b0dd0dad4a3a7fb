// Algorithm 2 with a shiftable SPATIAL kernel as well (Sec. 2), and
// Algorithm 1 (the linear spatial filter) as its case without a range kernel.
//
// Spatial kernel: the separable q_M(d1) q_M(d2) of Sec. 3, q_M(d) =
// cos^M(gs d) with gs = pi / (2r + 1), i.e. q_M on [-Ts, Ts], Ts = r + 1/2,
// sampled on the (2r+1)^2 window (truncated at the image border). Range kernel:
// q_N(t) = cos^N(gamma t) (N = 0: none). With the folded expansions
// cos^M(gs d) = sum_a beta_a cos(a gs d) and cos^N(gamma t) = sum_k alpha_k
// cos(k gamma t) and cos A cos B cos C = 1/4 sum_{+-,+-} cos(A +- B +- C),
// the weight of pixel y for output x is
//
//   phi(y - x) w(f(y) - f(x)) = sum_c coef_c Re(E_c(y) conj(E_c(x))),
//   E_c(z) = e^{i a gs z1} e^{i b gs z2} e^{i k gamma f(z)},
//
// over combos c = (a >= 0, signed b, signed k) (for a = 0 one of each
// conjugate pair), so num and den are moving sums (Sum(F, x, T) of Sec. 2) of
// the planes E_c f and E_c: Algorithm 2's stack, (M+1)^2 (N+1) real basis
// functions, never materialised.
//
// The skewed strip of the box engine carries over because the window width
// 2r + 1 is half a period of every spatial harmonic of the same parity as M:
// e^{i a gs (2r+1)} = (-1)^a = (-1)^M. Thread j keeps, per (b, k), the
// vertical running sums of e^{i b gs z2} e^{i k gamma f} (times f, and not)
// over its own column minus (-1)^M times those of the column 2r + 1 to the
// left; the horizontal sum of combo (a, b, k) then obeys
//   S(j) = S(j - 1) + e^{i a gs cw(j)} D_{b,k}(j),
// passed one lane per step through a shared row double-buffered by step
// parity, one CTA barrier per step.
#include <math.h>
#include <string.h>

#include "bf_internal.cuh"

namespace bf {
namespace spk {

constexpr int WMAX = 128;

template <int M, int N>
struct Dims {
    static constexpr int NA = M / 2 + 1;       // a in {M mod 2, ..., M}
    static constexpr int NB = M + 1;           // signed b in {-M, ..., M}
    static constexpr int NK = N + 1;           // signed k in {-N, ..., N}
    static constexpr int ND = NB * NK;         // (b, k) planes of the vertical sums
    static constexpr int D0 = ND - (ND + 1) / 2;  // first (b, k) kept for a = 0
    // combos: for a > 0 all (b, k); for a = 0 (M even) the upper half
    static constexpr int NS = (M % 2 == 0) ? (NA - 1) * ND + (ND + 1) / 2 : NA * ND;
};

// Largest combo table any instantiation needs.
constexpr int NS_CAP = 64;

struct Params {
    const float* img;
    float* out;
    int H, W, r, Hb, Tw;
    float gamma;           // range kernel frequency (unused when N = 0)
    float coef[NS_CAP];    // coef_c, in combo order
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }

// e^{i m gs n} for integers m, n: the phase is reduced exactly on integers
// (period 2 (2r + 1) in m n) before the sine and cosine.
__device__ __forceinline__ float2 phase(int m, int n, int r) {
    const int P = 2 * (2 * r + 1);
    int q = (int)(((long long)m * (long long)n) % P);
    if (q < 0) q += P;
    float s, c;
    sincospif((float)q / (float)(2 * r + 1), &s, &c);
    return make_float2(c, s);
}

// Range harmonics z_k = e^{i k theta} for signed k = -N, ..., N (step 2).
template <int N>
__device__ __forceinline__ void range_harmonics(float f, float gamma, float2 (&z)[N + 1]) {
    if constexpr (N == 0) {
        z[0] = make_float2(1.f, 0.f);
    } else {
        float s1, c1;
        sincosf(gamma * f, &s1, &c1);
        const float2 w1 = make_float2(c1, s1);
        const float2 w2 = cmul(w1, w1);
        // non-negative k, ascending: k0 = N mod 2, then +2
        float2 zp[N / 2 + 1];
        zp[0] = (N & 1) ? w1 : make_float2(1.f, 0.f);
#pragma unroll
        for (int i = 1; i <= N / 2; ++i) zp[i] = cmul(zp[i - 1], w2);
        // signed index ik: k = -N + 2 ik
#pragma unroll
        for (int ik = 0; ik <= N; ++ik) {
            const int k = -N + 2 * ik;
            const int i = (k >= 0 ? k : -k) / 2;
            z[ik] = k >= 0 ? zp[i] : conj2(zp[i]);
        }
    }
}

// Longest phase table: 2 (2r + 1) entries for r <= 56.
constexpr int PTAB_CAP = 2 * (2 * 56 + 1);

// Row phases e^{i b gs row} for signed b = -M, ..., M (step 2), from the
// table tab[q] = e^{i pi q / (2r+1)} and the row's indices q[b] = b row mod
// 2 (2r + 1) of the non-negative b (ib >= M / 2).
template <int M>
__device__ __forceinline__ void row_phases(const float2* tab, const int (&q)[M + 1],
                                           float2 (&p)[M + 1]) {
#pragma unroll
    for (int ib = M / 2 + (M & 1 ? 1 : 0); ib <= M; ++ib) p[ib] = tab[q[ib]];
#pragma unroll
    for (int ib = 0; ib <= M; ++ib)
        if (-M + 2 * ib < 0) p[ib] = conj2(p[M - ib]);
}

template <int M, int N>
__global__ void __launch_bounds__(WMAX, 2) spk_kernel(Params p) {
    using D = Dims<M, N>;
    constexpr int LD = WMAX + 1;
    constexpr int BUF = D::NS * LD;
    extern __shared__ float4 smem[];  // [2][NS][LD]: (g.re, g.im, h.re, h.im)
    const int Wi = blockDim.x;
    const int j = threadIdx.x;
    const int w = j >> 5;
    const int r = p.r;
    const int W = p.W;
    const int x0 = blockIdx.x * p.Tw;
    const int cw = x0 - r + j;
    const int c2 = cw - 2 * r - 1;
    const int co = cw - r;
    const bool own_in = cw >= 0 && cw < W;
    const bool sec_in = (j >= 2 * r + 1) && c2 >= 0 && c2 < W;
    const bool out_lane = (j >= 2 * r) && co < W;
    const int y0 = blockIdx.y * p.Hb;
    const int rows = min(p.Hb, p.H - y0);
    const int span = rows + 2 * r;
    const int steps = span + Wi - 1;
    const float sgn2 = (M & 1) ? 1.f : -1.f;  // -(-1)^M: weight of the second column

    for (int i = j; i < 2 * BUF; i += Wi) smem[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int P = 2 * (2 * r + 1);  // period of e^{i gs n} in n
    float2* ptab = reinterpret_cast<float2*>(smem + 2 * BUF);
    for (int q = j; q < P; q += Wi) {
        float s, c;
        sincospif((float)q / (float)(2 * r + 1), &s, &c);
        ptab[q] = make_float2(c, s);
    }
    // phase indices b row mod P of the entering row (advanced by b per step)
    // and their offsets to the centre row rho = e - r
    int qe[M + 1], qoff[M + 1];
#pragma unroll
    for (int ib = 0; ib <= M; ++ib) {
        const int b = -M + 2 * ib;
        const int bb = b < 0 ? 0 : b;
        int q0 = (int)(((long long)bb * (long long)(y0 - r - j)) % P);
        if (q0 < 0) q0 += P;
        qe[ib] = q0;
        qoff[ib] = (bb * r) % P;
    }

    // column phases e^{i a gs c} of the own and of the centre column
    float2 cph[D::NA], cphc[D::NA];
#pragma unroll
    for (int ia = 0; ia < D::NA; ++ia) {
        const int a = (M & 1) + 2 * ia;
        cph[ia] = phase(a, cw, r);
        cphc[ia] = phase(a, co, r);
    }

    float2 Dg[D::ND], Dh[D::ND];
#pragma unroll
    for (int d = 0; d < D::ND; ++d) { Dg[d] = make_float2(0.f, 0.f); Dh[d] = Dg[d]; }
    // the five pixels of step tt (own / second column, entering / leaving row,
    // centre), 0 where masked
    float nv[5];
    auto load_step = [&](int tt) {
        const int tau = tt - j;
        const bool act = tau >= 0 && tau < span;
        const int e = y0 - r + tau, l = e - 2 * r - 1, rho = e - r;
        const bool in_e = act && e >= 0 && e < p.H;
        const bool in_l = act && tau >= 2 * r + 1 && l >= 0 && l < p.H;
        const bool out = act && tau >= 2 * r && out_lane;
        nv[0] = (in_e && own_in) ? __ldg(p.img + (size_t)e * W + cw) : 0.f;
        nv[1] = (in_e && sec_in) ? __ldg(p.img + (size_t)e * W + c2) : 0.f;
        nv[2] = (in_l && own_in) ? __ldg(p.img + (size_t)l * W + cw) : 0.f;
        nv[3] = (in_l && sec_in) ? __ldg(p.img + (size_t)l * W + c2) : 0.f;
        nv[4] = out ? __ldg(p.img + (size_t)rho * W + co) : 0.f;
    };
    load_step(w * 32);  // a warp is first active at step 32 w
    __syncthreads();

    for (int t = 0; t < steps; ++t, [&] {
#pragma unroll
             for (int ib = 0; ib <= M; ++ib) {
                 const int b = -M + 2 * ib;
                 if (b > 0) { qe[ib] += b; if (qe[ib] >= P) qe[ib] -= P; }
             }
         }()) {
        const int warp_first = t - (w * 32 + 31);
        const int warp_last = t - w * 32;
        if (warp_last >= 0 && warp_first < span) {
            const int tau = t - j;
            const bool act = tau >= 0 && tau < span;
            const int e = y0 - r + tau;            // entering row
            const int l = e - 2 * r - 1;           // leaving row
            const int rho = e - r;                 // centre (output) row
            const bool in_e = act && e >= 0 && e < p.H;
            const bool in_l = act && tau >= 2 * r + 1 && l >= 0 && l < p.H;
            const bool out = act && tau >= 2 * r && out_lane;
            const bool m0 = in_e && own_in, m1 = in_e && sec_in;
            const bool m2 = in_l && own_in, m3 = in_l && sec_in;
            // this step's pixels were loaded during the previous step; start
            // the loads of the next one so their latency hides under this step
            const float f0 = nv[0], f1 = nv[1], f2 = nv[2], f3 = nv[3], fc = nv[4];
            load_step(t + 1);

            // vertical: entering row's phases; the leaving row's differ by
            // e^{-i b gs (2r+1)} = (-1)^M for every b of this parity
            float2 rp[M + 1];
            row_phases<M>(ptab, qe, rp);
            const float lsg = (M & 1) ? -1.f : 1.f;
            auto accumulate = [&](float f, float wgt, float rsg) {
                float2 z[N + 1];
                range_harmonics<N>(f, p.gamma, z);
                const float wf = wgt * f;
#pragma unroll
                for (int ib = 0; ib <= M; ++ib) {
                    const float2 rb = make_float2(rsg * rp[ib].x, rsg * rp[ib].y);
#pragma unroll
                    for (int ik = 0; ik <= N; ++ik) {
                        const float2 E = cmul(rb, z[ik]);
                        const int d = ib * (N + 1) + ik;
                        Dg[d].x = fmaf(wf, E.x, Dg[d].x);
                        Dg[d].y = fmaf(wf, E.y, Dg[d].y);
                        Dh[d].x = fmaf(wgt, E.x, Dh[d].x);
                        Dh[d].y = fmaf(wgt, E.y, Dh[d].y);
                    }
                }
            };
            // + own enter, -(-1)^M second enter, - own leave, +(-1)^M second leave
            accumulate(f0, m0 ? 1.f : 0.f, 1.f);
            accumulate(f1, m1 ? sgn2 : 0.f, 1.f);
            accumulate(f2, m2 ? -1.f : 0.f, lsg);
            accumulate(f3, m3 ? -sgn2 : 0.f, lsg);

            // horizontal and recombination with the centre's conj(E_c)
            float2 rpc[M + 1];
            {
                int qc[M + 1];
#pragma unroll
                for (int ib = 0; ib <= M; ++ib) {
                    qc[ib] = qe[ib] - qoff[ib];
                    if (qc[ib] < 0) qc[ib] += P;
                }
                row_phases<M>(ptab, qc, rpc);
            }
            float2 zc[N + 1];
            range_harmonics<N>(fc, p.gamma, zc);
            const float4* rd = smem + ((t + 1) & 1) * BUF + j;
            float4* wr = smem + (t & 1) * BUF + j + 1;
            float num = 0.f, den = 0.f;
            int c = 0;
#pragma unroll
            for (int ia = 0; ia < D::NA; ++ia) {
                const int a = (M & 1) + 2 * ia;
#pragma unroll
                for (int d = 0; d < D::ND; ++d) {
                    if (a == 0 && d < D::D0) continue;
                    const int ib = d / (N + 1), ik = d % (N + 1);
                    const float4 A = rd[c * LD];
                    const float2 sg = cmul(cph[ia], Dg[d]);
                    const float2 sh = cmul(cph[ia], Dh[d]);
                    const float2 hg = make_float2(A.x + sg.x, A.y + sg.y);
                    const float2 hh = make_float2(A.z + sh.x, A.w + sh.y);
                    wr[c * LD] = make_float4(hg.x, hg.y, hh.x, hh.y);
                    const float2 E = cmul(cmul(cphc[ia], rpc[ib]), zc[ik]);
                    // Re(conj(E) h) = E.x h.x + E.y h.y
                    num = fmaf(p.coef[c], fmaf(E.x, hg.x, E.y * hg.y), num);
                    den = fmaf(p.coef[c], fmaf(E.x, hh.x, E.y * hh.y), den);
                    ++c;
                }
            }
            if (out) p.out[(size_t)rho * W + co] = num / den;
        }
        __syncthreads();
    }
}

template <int M, int N>
static cudaError_t launch(const Params& p, int gx, int gy, cudaStream_t s) {
    using D = Dims<M, N>;
    static_assert(D::NS <= NS_CAP, "combo table");
    auto kern = spk_kernel<M, N>;
    const size_t smem = sizeof(float4) * 2 * (size_t)D::NS * (WMAX + 1) +
                        sizeof(float2) * PTAB_CAP;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(gx, gy), WMAX, smem, s>>>(p);
    return cudaGetLastError();
}

// Combo order and coefficients, as the kernel enumerates them:
// coef_c = 1/4 beta_a beta_|b| alpha_|k| m_b m_k (m = 2 for b = 0, k = 0:
// both sign choices give the same term), doubled for a = 0 except the
// self-conjugate (0, 0, 0).
static int combo_coefs(int M, int N, const double* beta, const double* alpha, float* coef) {
    const int NB = M + 1, NK = N + 1, ND = NB * NK, D0 = ND - (ND + 1) / 2;
    int c = 0;
    for (int ia = 0; ia <= M / 2; ++ia) {
        const int a = (M & 1) + 2 * ia;
        for (int d = 0; d < ND; ++d) {
            if (a == 0 && d < D0) continue;
            const int b = -M + 2 * (d / NK), k = -N + 2 * (d % NK);
            const int ab = b < 0 ? -b : b, ak = k < 0 ? -k : k;
            double v = 0.25 * beta[(a - (M & 1)) / 2] * beta[(ab - (M & 1)) / 2] *
                       alpha[(ak - (N & 1)) / 2];
            if (b == 0) v *= 2.0;
            if (k == 0) v *= 2.0;
            if (a == 0 && !(b == 0 && k == 0)) v *= 2.0;
            if (c >= NS_CAP) return -1;
            coef[c++] = (float)v;
        }
    }
    return c;
}

static bool supported(int M, int N) {
    if (N == 0) return M >= 1 && M <= 8 && M != 7 && M != 5;
    return (M == 1 || M == 2) && N >= 1 && N <= 4;
}

template <int M>
static cudaError_t dispatch_n(const Params& p, int N, int gx, int gy, cudaStream_t s) {
    if constexpr (M == 1 || M == 2) {
        switch (N) {
            case 0: return launch<M, 0>(p, gx, gy, s);
            case 1: return launch<M, 1>(p, gx, gy, s);
            case 2: return launch<M, 2>(p, gx, gy, s);
            case 3: return launch<M, 3>(p, gx, gy, s);
            case 4: return launch<M, 4>(p, gx, gy, s);
        }
        return cudaErrorInvalidValue;
    } else {
        return N == 0 ? launch<M, 0>(p, gx, gy, s) : cudaErrorInvalidValue;
    }
}

}  // namespace spk
}  // namespace bf

using namespace bf;

extern "C" bf_status bf_spatial_forward(const void* img, int H, int W, int r, int M,
                                        float sigma_r, float T, int N, float* out,
                                        const bf_opts* opts, void* stream) {
    if (!img || !out || H < 1 || W < 1 || r < 0 || M < 1) return BF_ERR_INVALID_ARG;
    if ((const void*)out == img) return BF_ERR_INVALID_ARG;
    if (!(T > 0.f) || !isfinite(T)) return BF_ERR_INVALID_ARG;
    bf_status st = check_opts(opts);
    if (st != BF_OK) return st;
    if (opts && (opts->in_dtype != BF_F32 || opts->kahan || opts->trunc_tol > 0.f))
        return BF_ERR_UNSUPPORTED;
    if (N < 0) {
        N = bf_resolve_N(sigma_r, T);
        if (N < 0) return BF_ERR_INVALID_ARG;
    }
    if (!spk::supported(M, N)) return BF_ERR_UNSUPPORTED;
    if (2 * r + 16 > spk::WMAX) return BF_ERR_UNSUPPORTED;
    if (r == 0) {
        // a 1 x 1 window: every kernel weighs the centre alone, out = f
        cudaError_t e = cudaMemcpyAsync(out, img, sizeof(float) * (size_t)H * W,
                                        cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
        return e == cudaSuccess ? BF_OK : set_cuda_error(e);
    }
    const int gm = opts ? opts->gamma_mode : BF_GAMMA_FIXED;
    double gamma = 0.0;
    if (N > 0) {
        gamma = bf_gamma(sigma_r, T, N, gm);
        if (!(gamma > 0.0)) return BF_ERR_INVALID_ARG;
    }
    double beta[BF_N_MAX / 2 + 1], alpha[BF_N_MAX / 2 + 1];
    if (bf_coeffs(M, beta, BF_N_MAX / 2 + 1) < 0 || bf_coeffs(N, alpha, BF_N_MAX / 2 + 1) < 0)
        return BF_ERR_INTERNAL;
    spk::Params p;
    memset(&p, 0, sizeof(p));
    if (spk::combo_coefs(M, N, beta, alpha, p.coef) < 0) return BF_ERR_INTERNAL;
    p.img = static_cast<const float*>(img);
    p.out = out;
    p.H = H; p.W = W; p.r = r;
    p.gamma = (float)gamma;
    p.Tw = spk::WMAX - 2 * r;
    const int gx = (W + p.Tw - 1) / p.Tw;
    int hb;
    if (opts && opts->tile_h > 0) {
        hb = opts->tile_h;
    } else {
        // one wave of resident CTAs: at most 2 per SM (rounding the band count
        // up would start a second, nearly empty wave)
        const int target = 2 * sm_count();
        int nb = target / gx;
        if (nb < 1) nb = 1;
        hb = (H + nb - 1) / nb;
        if (hb < 32) hb = 32;
    }
    p.Hb = hb;
    const int gy = (H + hb - 1) / hb;
    cudaError_t e;
    cudaStream_t s = (cudaStream_t)stream;
    switch (M) {
        case 1: e = spk::dispatch_n<1>(p, N, gx, gy, s); break;
        case 2: e = spk::dispatch_n<2>(p, N, gx, gy, s); break;
        case 3: e = spk::dispatch_n<3>(p, N, gx, gy, s); break;
        case 4: e = spk::dispatch_n<4>(p, N, gx, gy, s); break;
        case 6: e = spk::dispatch_n<6>(p, N, gx, gy, s); break;
        case 8: e = spk::dispatch_n<8>(p, N, gx, gy, s); break;
        default: return BF_ERR_UNSUPPORTED;
    }
    if (e != cudaSuccess) return set_cuda_error(e);
    return BF_OK;
}
