// Bilateral filter with the polynomial range kernel p_N(t) = (1 - t^2/T^2)^N
// of Sec. 3 (order of shiftability 2N + 1) and the box spatial kernel:
// Algorithm 2 with M = 1 and a polynomial basis instead of q_N's harmonics.
//
// With centred values u = f / T - 1/2 (so f = T (u + 1/2) and t / T = u_y -
// u_x), p_N(f(y) - f(x)) = (1 - (u_y - u_x)^2)^N = sum_{m=0}^{2N} u_y^m
// psi_m(u_x), a polynomial of degree 2N in each variable. Hence
//   num(x) = T sum_m psi_m(u_x) (Box[u^{m+1}] + Box[u^m] / 2)(x),
//   den(x) =   sum_m psi_m(u_x)  Box[u^m](x),
// moving sums (Sec. 2) of the 2N + 2 power images u^0 .. u^{2N+1}. Centring
// keeps |u| <= 1/2 for f in [0, T], which bounds the cancellation of the
// alternating expansion by 2^N (against 5^N for the raw powers); N <= 8.
//
// Tiling is the skewed strip of the harmonic engine: thread j keeps the
// vertical running sums of its own column minus those of the column 2r + 1 to
// its left, the horizontal sum S(j) = S(j - 1) + D(j) passes one lane per
// step through a shared row double-buffered by step parity.
#include <math.h>
#include <string.h>

#include "bf_internal.cuh"
#include "bf_launch.cuh"
#include "bf_trace.cuh"

namespace bf {
namespace poly {

// L2 prefetch of one line (no registers held, nothing returned)
__device__ __forceinline__ void prefetch_l2(const void* ptr) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}

constexpr int WMAX = 128;
constexpr int NMAX = 8;
constexpr int PCAP = 2 * NMAX + 1;  // psi_m, m = 0..2N

struct Params {
    const float* img;      // forward input
    float* out;            // forward output
    float4* sv;            // forward with saved quads: (f, 1/den, out, dnum_s - out dden_s)
    const float4* bsv;     // adjoint: the forward's saved quads
    const float* gout;     // adjoint: dL/dout
    float* gimg;           // adjoint: dL/dimg
    int H, W, r, Hb, Tw;
    float invT, T;
    // psi_m(v) = sum_n c_m[n] v^n (degree 2N - m: the terms u^m v^n of the
    // expansion have m + n <= 2N), kept in pairs for the paired FP32 units:
    // c2[i][n] = (c_{2i}[n], c_{2i+1}[n]) (psi_{2N+1} = 0), and likewise dc2 for
    // psi_m'(v) = sum_n (n + 1) c_m[n + 1] v^n.
    float2 c2[NMAX + 1][PCAP];
    float2 dc2[NMAX + 1][PCAP];
};

__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }

// sum_n c[n] v^n on both lanes by Horner from degree deg (a constant once the
// caller's loop is unrolled).
__device__ __forceinline__ float2 horner2(const float2* c, int deg, float2 V) {
    float2 s = c[deg];
#pragma unroll
    for (int n = PCAP - 2; n >= 0; --n)
        if (n < deg) s = __ffma2_rn(s, V, c[n]);
    return s;
}

// Launch modes: forward, forward that also saves the adjoint's quads, adjoint.
enum Mode { FWD = 0, FWD_SAVE = 1, ADJ = 2 };

// The adjoint (MODE = ADJ) moving-sums alpha u^m and beta u^m (alpha = g / den,
// beta = -alpha out; the window and p_N are symmetric) and forms
//   dL/df(p) = sum_m psi_m(u_p) A_m + (1/T) sum_m psi_m'(u_p) (f(p) A_m + B_m)
//            + alpha(p) X(p),
// A_m = Sum(alpha u^m), B_m = Sum(beta u^m), X = dnum_s - out dden_s saved by
// the forward (dnum_s = sum_m psi_m'(u_p) (Sum(u^{m+1}) + Sum(u^m) / 2),
// dden_s = (1/T) sum_m psi_m'(u_p) Sum(u^m): num and den differentiated
// through the centre value).
template <int N, int MODE>
__global__ void __launch_bounds__(WMAX, 2) poly_kernel(Params p) {
    // forward: power planes u^0 .. u^{2N+1} as pairs (u^{2i}, u^{2i+1});
    // adjoint: pairs (alpha u^m, beta u^m), m <= 2N
    constexpr int NP2 = MODE == ADJ ? 2 * N + 1 : N + 1;  // plane pairs
    constexpr int NQ = (NP2 + 1) / 2;    // float4 slots per lane
    constexpr int LD = WMAX + 1;
    constexpr int BUF = NQ * LD;
    extern __shared__ float4 smem[];     // [2][NQ][LD]
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

    for (int i = j; i < 2 * BUF; i += Wi) smem[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 D[2 * NQ];
#pragma unroll
    for (int m = 0; m < 2 * NQ; ++m) D[m] = make_float2(0.f, 0.f);
    // the five pixels of step tt (own / second column, entering / leaving row,
    // centre), 0 where masked; the adjoint reads the saved quad (whose .x is f)
    // and dL/dout instead
    float4 nq[5];
    float ng[5];
    // pixel (row, col): the image and dL/dout at row * W + col, its saved quad
    // at quad_index (rows sheared, so the diagonal a warp reads is contiguous)
    auto load_one = [&](int k, bool on, int row, int col) {
        if constexpr (MODE == ADJ) {
            nq[k] = on ? __ldg(p.bsv + quad_index(row, col, p.H, W))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
            ng[k] = on ? __ldg(p.gout + (size_t)row * W + col) : 0.f;
        } else {
            nq[k].x = on ? __ldg(p.img + (size_t)row * W + col) : 0.f;
        }
    };
    auto load_step = [&](int tt) {
        const int tau = tt - j;
        const bool act = tau >= 0 && tau < span;
        const int e = y0 - r + tau, l = e - 2 * r - 1, rho = e - r;
        const bool in_e = act && e >= 0 && e < p.H;
        const bool in_l = act && tau >= 2 * r + 1 && l >= 0 && l < p.H;
        const bool out = act && tau >= 2 * r && out_lane;
        load_one(0, in_e && own_in, e, cw);
        load_one(1, in_e && sec_in, e, c2);
        load_one(2, in_l && own_in, l, cw);
        load_one(3, in_l && sec_in, l, c2);
        load_one(4, out, rho, co);
    };
    load_step(w * 32);  // a warp is first active at step 32 w
    __syncthreads();

    for (int t = 0; t < steps; ++t) {
        const int warp_first = t - (w * 32 + 31);
        const int warp_last = t - w * 32;
        if (warp_last >= 0 && warp_first < span) {
            const int tau = t - j;
            const bool act = tau >= 0 && tau < span;
            const int e = y0 - r + tau;
            const int l = e - 2 * r - 1;
            const int rho = e - r;
            const bool in_e = act && e >= 0 && e < p.H;
            const bool in_l = act && tau >= 2 * r + 1 && l >= 0 && l < p.H;
            const bool out = act && tau >= 2 * r && out_lane;
            const bool m0 = in_e && own_in, m1 = in_e && sec_in;
            const bool m2 = in_l && own_in, m3 = in_l && sec_in;
            // this step's pixels were loaded during the previous step; start
            // the loads of the next one so their latency hides under this step
            float4 q[5];
            float gq[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) { q[k] = nq[k]; gq[k] = MODE == ADJ ? ng[k] : 0.f; }
            const float fc = q[4].x;
            load_step(t + 1);
            // pull the entering row of the step 8 ahead into L2 (inside the
            // band's rows only); the other four streams re-read recent rows
            {
                const int ef = e + 8;
                if (own_in && ef >= 0 && ef < p.H && ef < y0 - r + span) {
                    if constexpr (MODE == ADJ) {
                        prefetch_l2(p.bsv + quad_index(ef, cw, p.H, W));
                        prefetch_l2(p.gout + (size_t)ef * W + cw);
                    } else {
                        prefetch_l2(p.img + (size_t)ef * W + cw);
                    }
                }
            }
            // + own enter, - second enter, - own leave, + second leave
            auto accumulate = [&](int k, float wgt) {
                const float u = fmaf(q[k].x, p.invT, -0.5f);
                if constexpr (MODE == ADJ) {
                    const float al = gq[k] * q[k].y;
                    float2 pab = make_float2(wgt * al, -wgt * al * q[k].z);
                    const float2 U = dup(u);
#pragma unroll
                    for (int m = 0; m < NP2; ++m) {
                        D[m] = __fadd2_rn(D[m], pab);
                        pab = __fmul2_rn(pab, U);
                    }
                } else {
                    float2 pw = make_float2(wgt, wgt * u);
                    const float2 U2 = dup(u * u);
#pragma unroll
                    for (int i = 0; i < NP2; ++i) {
                        D[i] = __fadd2_rn(D[i], pw);
                        pw = __fmul2_rn(pw, U2);
                    }
                }
            };
            accumulate(0, m0 ? 1.f : 0.f);
            accumulate(1, m1 ? -1.f : 0.f);
            accumulate(2, m2 ? -1.f : 0.f);
            accumulate(3, m3 ? 1.f : 0.f);

            const float4* rd = smem + ((t + 1) & 1) * BUF + j;
            float4* wr = smem + (t & 1) * BUF + j + 1;
            float2 B[2 * NQ];
#pragma unroll
            for (int qq = 0; qq < NQ; ++qq) {
                const float4 A = rd[qq * LD];
                B[2 * qq] = __fadd2_rn(make_float2(A.x, A.y), D[2 * qq]);
                B[2 * qq + 1] = __fadd2_rn(make_float2(A.z, A.w), D[2 * qq + 1]);
                wr[qq * LD] = make_float4(B[2 * qq].x, B[2 * qq].y, B[2 * qq + 1].x,
                                          B[2 * qq + 1].y);
            }
            if (out) {
                const float2 V = dup(fmaf(fc, p.invT, -0.5f));
                const size_t o = (size_t)rho * W + co;
                float2 NUM = make_float2(0.f, 0.f), DEN = NUM, DN = NUM, DD = NUM;
#pragma unroll
                for (int i = 0; i <= N; ++i) {
                    // (psi_{2i}, psi_{2i+1}) at v: degree 2N - 2i (psi_{2N+1} = 0)
                    const int deg = 2 * N - 2 * i;
                    const float2 ps = horner2(p.c2[i], deg, V);
                    float2 dps = make_float2(0.f, 0.f);
                    if constexpr (MODE != FWD) {
                        if (deg >= 1) dps = horner2(p.dc2[i], deg - 1, V);
                    }
                    if constexpr (MODE == ADJ) {
                        // B[m] = (A_m, B_m) = (Sum(alpha u^m), Sum(beta u^m))
                        const float2 b0 = B[2 * i];
                        NUM.x = fmaf(ps.x, b0.x, NUM.x);
                        DEN.x = fmaf(dps.x, fmaf(fc, b0.x, b0.y), DEN.x);
                        if (i < N) {
                            const float2 b1 = B[2 * i + 1];
                            NUM.y = fmaf(ps.y, b1.x, NUM.y);
                            DEN.y = fmaf(dps.y, fmaf(fc, b1.x, b1.y), DEN.y);
                        }
                    } else {
                        // B[i] = (Sum u^{2i}, Sum u^{2i+1}); g_m = Sum u^m / 2 + Sum u^{m+1}
                        const float2 bm = B[i];
                        const float2 bm1 = make_float2(bm.y, i < N ? B[i + 1].x : 0.f);
                        const float2 g = __ffma2_rn(dup(0.5f), bm, bm1);
                        NUM = __ffma2_rn(ps, g, NUM);
                        DEN = __ffma2_rn(ps, bm, DEN);
                        if constexpr (MODE == FWD_SAVE) {
                            DN = __ffma2_rn(dps, g, DN);
                            DD = __ffma2_rn(dps, bm, DD);
                        }
                    }
                }
                const float num = NUM.x + NUM.y, den = DEN.x + DEN.y;
                if constexpr (MODE == ADJ) {
                    const float al = gq[4] * q[4].y;  // centre quad: (f, 1/den, out, X)
                    p.gimg[o] = num + fmaf(den, p.invT, al * q[4].w);
                } else {
                    const float ov = p.T * num / den;
                    p.out[o] = ov;
                    if constexpr (MODE == FWD_SAVE) {
                        const float dn = DN.x + DN.y, dd = DD.x + DD.y;
                        // streaming store: the adjoint reads the quads after the whole forward
                        __stcs(p.sv + quad_index(rho, co, p.H, W),
                               make_float4(fc, 1.0f / den, ov, fmaf(-ov * p.invT, dd, dn)));
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <int N>
static cudaError_t launch(const Params& p, int mode, int gx, int gy, cudaStream_t s) {
    const int NP = mode == ADJ ? 2 * (2 * N + 1) : 2 * N + 2;  // planes, as in the kernel
    const int NQ = (NP + 3) / 4;
    auto kern = mode == ADJ ? poly_kernel<N, ADJ>
                            : (mode == FWD_SAVE ? poly_kernel<N, FWD_SAVE> : poly_kernel<N, FWD>);
    const size_t smem = sizeof(float4) * 2 * (size_t)NQ * (WMAX + 1);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    Params q = p;
    // one wave of as many CTAs as fit per SM (the adjoint's sheared quad loads
    // coalesce, so it no longer gains from fewer resident CTAs)
    if (q.Hb <= 0) q.Hb = wave_band_rows((const void*)kern, WMAX, smem, q.H, gx);
    gy = (q.H + q.Hb - 1) / q.Hb;
    kern<<<dim3(gx, gy), WMAX, smem, s>>>(q);
    return cudaGetLastError();
}

// Coefficients of (1 - (u - v)^2)^N = sum_j C(N, j) (-1)^j (u - v)^{2j}
//   = sum_j C(N, j) (-1)^j sum_m C(2j, m) u^m (-v)^{2j - m}:
// c[m][n] is the coefficient of u^m v^n (n = 2j - m).
static void expansion(int N, double c[PCAP][PCAP]) {
    for (int m = 0; m < PCAP; ++m)
        for (int n = 0; n < PCAP; ++n) c[m][n] = 0.0;
    double cnj = 1.0;  // C(N, j)
    for (int j = 0; j <= N; ++j) {
        double c2m = 1.0;  // C(2j, m)
        for (int m = 0; m <= 2 * j; ++m) {
            const int n = 2 * j - m;
            const double sgn = ((j + n) & 1) ? -1.0 : 1.0;  // (-1)^j (-1)^n
            c[m][n] += sgn * cnj * c2m;
            c2m = c2m * (double)(2 * j - m) / (double)(m + 1);
        }
        cnj = cnj * (double)(N - j) / (double)(j + 1);
    }
}

// Checks shared by the forward and the adjoint; fills the launch parameters
// (expansion coefficients and their derivatives, tiles) and resolves N.
static bf_status prepare(int H, int W, int r, float sigma_r, float T, int* N,
                         const bf_opts* opts, Params* p, int* gx, int* gy) {
    if (H < 1 || W < 1 || r < 0) return BF_ERR_INVALID_ARG;
    if (!(T > 0.f) || !isfinite(T)) return BF_ERR_INVALID_ARG;
    bf_status st = check_opts(opts);
    if (st != BF_OK) return st;
    if (opts && (opts->in_dtype != BF_F32 || opts->kahan || opts->trunc_tol > 0.f ||
                 opts->gamma_mode != BF_GAMMA_FIXED || (opts->pitch != 0 && opts->pitch != W)))
        return BF_ERR_UNSUPPORTED;
    if (*N <= 0) {
        *N = bf_poly_resolve_N(sigma_r, T);
        if (*N < 0) return BF_ERR_INVALID_ARG;
    }
    if (*N > NMAX) return BF_ERR_UNSUPPORTED;
    if (2 * r + 16 > WMAX) return BF_ERR_UNSUPPORTED;
    memset(p, 0, sizeof(*p));
    double c[PCAP][PCAP];
    expansion(*N, c);
    // psi_m has degree 2N - m: the kernel's Horner starts there
    for (int m = 0; m < PCAP; ++m)
        for (int n = 0; n < PCAP; ++n)
            if (m + n > 2 * *N && c[m][n] != 0.0) return BF_ERR_INTERNAL;
    auto cf = [&](int m, int n) { return m < PCAP && n < PCAP ? c[m][n] : 0.0; };
    for (int i = 0; i <= NMAX; ++i)
        for (int n = 0; n < PCAP; ++n) {
            p->c2[i][n] = make_float2((float)cf(2 * i, n), (float)cf(2 * i + 1, n));
            p->dc2[i][n] = make_float2((float)((n + 1) * cf(2 * i, n + 1)),
                                       (float)((n + 1) * cf(2 * i + 1, n + 1)));
        }
    p->H = H; p->W = W; p->r = r;
    p->T = T;
    p->invT = 1.0f / T;
    p->Tw = WMAX - 2 * r;
    *gx = (W + p->Tw - 1) / p->Tw;
    // band height: the caller's, else (0) one wave of the launched kernel's
    // resident CTAs, chosen at launch
    p->Hb = (opts && opts->tile_h > 0) ? opts->tile_h : 0;
    *gy = 0;
    return BF_OK;
}

static cudaError_t dispatch(const Params& p, int mode, int N, int gx, int gy, cudaStream_t s) {
    switch (N) {
        case 1: return launch<1>(p, mode, gx, gy, s);
        case 2: return launch<2>(p, mode, gx, gy, s);
        case 3: return launch<3>(p, mode, gx, gy, s);
        case 4: return launch<4>(p, mode, gx, gy, s);
        case 5: return launch<5>(p, mode, gx, gy, s);
        case 6: return launch<6>(p, mode, gx, gy, s);
        case 7: return launch<7>(p, mode, gx, gy, s);
        case 8: return launch<8>(p, mode, gx, gy, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace poly
}  // namespace bf

using namespace bf;

extern "C" int bf_poly_resolve_N(float sigma_r, float T) {
    if (!(sigma_r > 0.f) || !(T > 0.f) || !isfinite(sigma_r) || !isfinite(T)) return -1;
    // Eq. approx1: p_N(t / sqrt(N)) -> exp(-t^2 / T^2), i.e. p_N(t) ~
    // exp(-N t^2 / T^2); matching exp(-t^2 / (2 sigma_r^2)) gives
    // N = T^2 / (2 sigma_r^2), rounded up.
    const double v = ((double)T * (double)T) / (2.0 * (double)sigma_r * (double)sigma_r);
    if (v > 1e9) return poly::NMAX + 1;
    const int n = (int)ceil(v - 1e-9);
    return n < 1 ? 1 : n;
}

extern "C" bf_status bf_poly_forward(const void* img, int H, int W, int r, float sigma_r,
                                     float T, int N, float* out, const bf_opts* opts, void* saved,
                                     void* stream) {
    BF_TRACE("bf_poly_forward");
    // the saved quads are indexed in 32 bits here (quad_index)
    if ((long long)H * W >= 0x7fffffffLL) return BF_ERR_UNSUPPORTED;
    if (!img || !out) return BF_ERR_INVALID_ARG;
    if ((const void*)out == img) return BF_ERR_INVALID_ARG;
    if (saved && ((uintptr_t)saved & 15)) return BF_ERR_INVALID_ARG;
    if (opts && opts->save_for_backward && !saved) return BF_ERR_INVALID_ARG;
    poly::Params p;
    int gx = 0, gy = 0;
    bf_status st = poly::prepare(H, W, r, sigma_r, T, &N, opts, &p, &gx, &gy);
    if (st != BF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (r == 0) {
        // a 1 x 1 window: p_N(0) = 1 with slope 0, so out = f and the quads
        // are (f, 1, f, 0)
        cudaError_t e = unit_window(static_cast<const float*>(img), out,
                                    static_cast<float4*>(saved), H, W, s);
        return e == cudaSuccess ? BF_OK : set_cuda_error(e);
    }
    p.img = static_cast<const float*>(img);
    p.out = out;
    p.sv = static_cast<float4*>(saved);
    cudaError_t e = poly::dispatch(p, saved ? poly::FWD_SAVE : poly::FWD, N, gx, gy, s);
    if (e != cudaSuccess) return set_cuda_error(e);
    return BF_OK;
}

extern "C" bf_status bf_poly_backward(const float* grad_out, const void* saved, int H, int W,
                                      int r, float sigma_r, float T, int N, float* grad_img,
                                      const bf_opts* opts, void* stream) {
    BF_TRACE("bf_poly_backward");
    // the saved quads are indexed in 32 bits here (quad_index)
    if ((long long)H * W >= 0x7fffffffLL) return BF_ERR_UNSUPPORTED;
    if (!grad_out || !saved || !grad_img) return BF_ERR_INVALID_ARG;
    if ((uintptr_t)saved & 15) return BF_ERR_INVALID_ARG;
    // neighbours' dL/dout and quads are read while dL/dimg is written
    if ((const void*)grad_img == (const void*)grad_out || (const void*)grad_img == saved)
        return BF_ERR_INVALID_ARG;
    poly::Params p;
    int gx = 0, gy = 0;
    bf_status st = poly::prepare(H, W, r, sigma_r, T, &N, opts, &p, &gx, &gy);
    if (st != BF_OK) return st;
    if (r == 0) {
        // 1 x 1 window: out = f, so dL/df = dL/dout
        cudaError_t e = cudaMemcpyAsync(grad_img, grad_out, sizeof(float) * (size_t)H * W,
                                        cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
        return e == cudaSuccess ? BF_OK : set_cuda_error(e);
    }
    p.bsv = static_cast<const float4*>(saved);
    p.gout = grad_out;
    p.gimg = grad_img;
    cudaError_t e = poly::dispatch(p, poly::ADJ, N, gx, gy, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_cuda_error(e);
    return BF_OK;
}
