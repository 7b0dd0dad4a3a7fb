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

namespace bf {
namespace poly {

constexpr int WMAX = 128;
constexpr int NMAX = 8;
constexpr int PCAP = 2 * NMAX + 1;  // psi_m, m = 0..2N

struct Params {
    const float* img;
    float* out;
    int H, W, r, Hb, Tw;
    float invT, T;
    // psi_m(v) = sum_n c[m][n] v^n, m, n = 0..2N
    float c[PCAP][PCAP];
};

template <int N>
__global__ void __launch_bounds__(WMAX, 2) poly_kernel(Params p) {
    constexpr int NP = 2 * N + 2;        // power planes u^0 .. u^{2N+1}
    constexpr int NQ = (NP + 3) / 4;     // float4 slots per lane
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
    float D[NQ * 4];
#pragma unroll
    for (int m = 0; m < NQ * 4; ++m) D[m] = 0.f;
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
            const float f0 = nv[0], f1 = nv[1], f2 = nv[2], f3 = nv[3], fc = nv[4];
            load_step(t + 1);
            // + own enter, - second enter, - own leave, + second leave
            auto accumulate = [&](float f, float wgt) {
                const float u = fmaf(f, p.invT, -0.5f);
                float pw = wgt;
#pragma unroll
                for (int m = 0; m < NP; ++m) {
                    D[m] += pw;
                    pw *= u;
                }
            };
            accumulate(f0, m0 ? 1.f : 0.f);
            accumulate(f1, m1 ? -1.f : 0.f);
            accumulate(f2, m2 ? -1.f : 0.f);
            accumulate(f3, m3 ? 1.f : 0.f);

            const float4* rd = smem + ((t + 1) & 1) * BUF + j;
            float4* wr = smem + (t & 1) * BUF + j + 1;
            float B[NQ * 4];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const float4 A = rd[q * LD];
                B[4 * q + 0] = A.x + D[4 * q + 0];
                B[4 * q + 1] = A.y + D[4 * q + 1];
                B[4 * q + 2] = A.z + D[4 * q + 2];
                B[4 * q + 3] = A.w + D[4 * q + 3];
                wr[q * LD] = make_float4(B[4 * q], B[4 * q + 1], B[4 * q + 2], B[4 * q + 3]);
            }
            if (out) {
                const float v = fmaf(fc, p.invT, -0.5f);
                float num = 0.f, den = 0.f;
#pragma unroll
                for (int m = 0; m <= 2 * N; ++m) {
                    // psi_m(v) by Horner
                    float psi = p.c[m][2 * N];
#pragma unroll
                    for (int n = 2 * N - 1; n >= 0; --n) psi = fmaf(psi, v, p.c[m][n]);
                    num = fmaf(psi, fmaf(0.5f, B[m], B[m + 1]), num);
                    den = fmaf(psi, B[m], den);
                }
                p.out[(size_t)rho * W + co] = p.T * num / den;
            }
        }
        __syncthreads();
    }
}

template <int N>
static cudaError_t launch(const Params& p, int gx, int gy, cudaStream_t s) {
    constexpr int NQ = (2 * N + 2 + 3) / 4;
    auto kern = poly_kernel<N>;
    const size_t smem = sizeof(float4) * 2 * (size_t)NQ * (WMAX + 1);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(gx, gy), WMAX, smem, s>>>(p);
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
                                     float T, int N, float* out, const bf_opts* opts,
                                     void* stream) {
    if (!img || !out || H < 1 || W < 1 || r < 0) return BF_ERR_INVALID_ARG;
    if ((const void*)out == img) return BF_ERR_INVALID_ARG;
    if (!(T > 0.f) || !isfinite(T)) return BF_ERR_INVALID_ARG;
    bf_status st = check_opts(opts);
    if (st != BF_OK) return st;
    if (opts && (opts->in_dtype != BF_F32 || opts->kahan || opts->trunc_tol > 0.f ||
                 opts->gamma_mode != BF_GAMMA_FIXED))
        return BF_ERR_UNSUPPORTED;
    if (N <= 0) {
        N = bf_poly_resolve_N(sigma_r, T);
        if (N < 0) return BF_ERR_INVALID_ARG;
    }
    if (N > poly::NMAX) return BF_ERR_UNSUPPORTED;
    if (2 * r + 16 > poly::WMAX) return BF_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    if (r == 0) {  // 1 x 1 window: out = f
        cudaError_t e = cudaMemcpyAsync(out, img, sizeof(float) * (size_t)H * W,
                                        cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? BF_OK : set_cuda_error(e);
    }
    poly::Params p;
    memset(&p, 0, sizeof(p));
    double c[poly::PCAP][poly::PCAP];
    poly::expansion(N, c);
    for (int m = 0; m < poly::PCAP; ++m)
        for (int n = 0; n < poly::PCAP; ++n) p.c[m][n] = (float)c[m][n];
    p.img = static_cast<const float*>(img);
    p.out = out;
    p.H = H; p.W = W; p.r = r;
    p.T = T;
    p.invT = 1.0f / T;
    p.Tw = poly::WMAX - 2 * r;
    const int gx = (W + p.Tw - 1) / p.Tw;
    int hb;
    if (opts && opts->tile_h > 0) {
        hb = opts->tile_h;
    } else {
        // one wave of resident CTAs (two per SM)
        int nb = 2 * sm_count() / gx;
        if (nb < 1) nb = 1;
        hb = (H + nb - 1) / nb;
        if (hb < 32) hb = 32;
    }
    p.Hb = hb;
    const int gy = (H + hb - 1) / hb;
    cudaError_t e;
    switch (N) {
        case 1: e = poly::launch<1>(p, gx, gy, s); break;
        case 2: e = poly::launch<2>(p, gx, gy, s); break;
        case 3: e = poly::launch<3>(p, gx, gy, s); break;
        case 4: e = poly::launch<4>(p, gx, gy, s); break;
        case 5: e = poly::launch<5>(p, gx, gy, s); break;
        case 6: e = poly::launch<6>(p, gx, gy, s); break;
        case 7: e = poly::launch<7>(p, gx, gy, s); break;
        case 8: e = poly::launch<8>(p, gx, gy, s); break;
        default: return BF_ERR_UNSUPPORTED;
    }
    if (e != cudaSuccess) return set_cuda_error(e);
    return BF_OK;
}
