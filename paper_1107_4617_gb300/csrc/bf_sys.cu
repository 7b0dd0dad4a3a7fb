// Register-resident skewed-strip engine for the forward filter and its
// adjoint (Algorithm 2 with M = 1 and range kernel q_N, Sec. 2-3).
//
// A CTA owns a strip of Wi = blockDim.x consecutive input columns and a band
// of output rows; thread j owns column cw(j) = x0 - r + j. Two moving sums
// (Sec. 2, Sum(F, x, T)) make the (2r+1)^2 box:
//
//  * vertical: thread j keeps, for every harmonic of the chunk, a running
//    sum over the 2r+1 rows of the window. It keeps it for the DIFFERENCE
//    D = V(cw(j)) - V(cw(j) - 2r - 1) of two columns: per row it adds the
//    entering pixel's planes of both columns and subtracts the leaving ones.
//    All four pixels' planes are regenerated from f (one MUFU sincos per
//    pixel, harmonics by complex rotation z_{k+2} = z_k z_2), so no plane is
//    ever stored.
//  * horizontal: the window sum S(j) = sum_{i=j-2r..j} V(cw(i)) obeys
//    S(j) = S(j-1) + D(j). It flows one lane per step through warp shuffles
//    (and a small shared-memory hand-off between warps): thread j processes
//    output row rho at step t = rho_index + j, one step after thread j-1
//    computed S(j-1) for the same row. The strip is therefore swept on a
//    skew of one row per column; each warp is idle for the first 32 w steps
//    (another resident CTA fills the SM meanwhile).
//
// S(j) is the full box sum centred on column cw(j) - r; thread j combines it
// with that centre pixel's C_k, S_k and a_k (Algorithm 2 step 3). Everything
// per harmonic lives in registers: 8 floats (D and S) per harmonic.
#include "bf_internal.cuh"

namespace bf {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float ld_img(const float* p, size_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_img(const __nv_bfloat16* p, size_t i) {
    return __bfloat162float(p[i]);
}

// Rotation state of one pixel stream: z = current harmonic (cos, sin),
// w = (cos 2 theta, sin 2 theta); u, v = the weights the planes carry
// (forward: f and 1; adjoint: alpha and beta), with the stream's sign folded
// in. A masked stream has z = 0.
struct Stream {
    float zc, zs, wc, ws, u, v;
};

__device__ __forceinline__ void seed(Stream& s, float f, float gamma, int kstart, bool on) {
    float sn, cs;
    __sincosf(gamma * f, &sn, &cs);
    s.wc = (cs - sn) * (cs + sn);
    s.ws = 2.0f * sn * cs;
    s.zc = kstart ? cs : 1.0f;
    s.zs = kstart ? sn : 0.0f;
    if (!on) { s.zc = 0.0f; s.zs = 0.0f; }
}

__device__ __forceinline__ void rot(Stream& s) {
    const float c = s.zc * s.wc - s.zs * s.ws;
    const float n = s.zs * s.wc + s.zc * s.ws;
    s.zc = c;
    s.zs = n;
}

}  // namespace

template <int KC, bool BWD, bool SAVE, typename Tin>
__global__ void __launch_bounds__(128, 2) bf_sys_kernel(SysParams p) {
    __shared__ float4 xfer[2][8][KC];  // lane 31 of warp w -> lane 0 of warp w+1
    const Tin* img = static_cast<const Tin*>(p.img);
    const int Wi = blockDim.x;
    const int j = threadIdx.x;
    const int lane = j & 31;
    const int w = j >> 5;
    const int r = p.r;
    const int x0 = blockIdx.x * p.Tw;
    const int cw = x0 - r + j;            // own column
    const int c2 = cw - 2 * r - 1;        // column leaving the horizontal window
    const int co = cw - r;                // output (centre) column
    const bool own_in = cw >= 0 && cw < p.W;
    const bool sec_in = (j >= 2 * r + 1) && c2 >= 0 && c2 < p.W;
    const bool out_lane = (j >= 2 * r) && co < p.W;
    const int y0 = blockIdx.y * p.Hb;
    const int rows = min(p.Hb, p.H - y0);
    const int span = rows + 2 * r;        // local steps of one thread
    const int steps = span + Wi - 1;
    const int K = p.K;

    for (int i = threadIdx.x; i < 2 * 8 * KC; i += Wi)
        (&xfer[0][0][0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);

    float4 D[KC], S[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) {
        D[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        S[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float gsum = 0.f;
    __syncthreads();

    for (int t = 0; t < steps; ++t) {
        const int warp_first = t - (w * 32 + 31);
        const int warp_last = t - w * 32;
        if (warp_last >= 0 && warp_first < span) {
            const int tau = t - j;
            const bool act = tau >= 0 && tau < span;
            const int e = y0 - r + tau;          // entering row
            const int l = e - 2 * r - 1;         // leaving row
            const int rho = y0 - 2 * r + tau;    // output row
            const bool in_e = act && e >= 0 && e < p.H;
            const bool in_l = act && tau >= 2 * r + 1 && l >= 0 && l < p.H;
            const bool do_out = act && tau >= 2 * r && out_lane;

            Stream s0, s1, s2, s3, sc;  // own-enter, second-enter, own-leave, second-leave, centre
            {
                const bool m0 = in_e && own_in, m1 = in_e && sec_in;
                const bool m2 = in_l && own_in, m3 = in_l && sec_in;
                const size_t re = (size_t)(in_e ? e : 0) * p.W, rl = (size_t)(in_l ? l : 0) * p.W;
                const float f0 = m0 ? ld_img(img, re + cw) : 0.f;
                const float f1 = m1 ? ld_img(img, re + c2) : 0.f;
                const float f2 = m2 ? ld_img(img, rl + cw) : 0.f;
                const float f3 = m3 ? ld_img(img, rl + c2) : 0.f;
                seed(s0, f0, p.gamma, p.kstart, m0);
                seed(s1, f1, p.gamma, p.kstart, m1);
                seed(s2, f2, p.gamma, p.kstart, m2);
                seed(s3, f3, p.gamma, p.kstart, m3);
                if (!BWD) {
                    s0.u = f0; s1.u = -f1; s2.u = -f2; s3.u = f3;
                } else {
                    // alpha = g / den, beta = -alpha * out, at each stream's pixel
                    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f;
                    if (m0) { const size_t q = re + cw; a0 = __ldg(p.gout + q) / __ldg(p.bden + q); b0 = -a0 * __ldg(p.fout + q); }
                    if (m1) { const size_t q = re + c2; a1 = __ldg(p.gout + q) / __ldg(p.bden + q); b1 = -a1 * __ldg(p.fout + q); }
                    if (m2) { const size_t q = rl + cw; a2 = __ldg(p.gout + q) / __ldg(p.bden + q); b2 = -a2 * __ldg(p.fout + q); }
                    if (m3) { const size_t q = rl + c2; a3 = __ldg(p.gout + q) / __ldg(p.bden + q); b3 = -a3 * __ldg(p.fout + q); }
                    s0.u = a0; s0.v = b0;
                    s1.u = -a1; s1.v = -b1;
                    s2.u = -a2; s2.v = -b2;
                    s3.u = a3; s3.v = b3;
                }
            }
            float fc = 0.f, ac = 0.f, bc = 0.f;
            size_t oidx = 0;
            if (do_out) {
                oidx = (size_t)rho * p.W + co;
                fc = ld_img(img, oidx);
                if (BWD) {
                    ac = __ldg(p.gout + oidx) / __ldg(p.bden + oidx);
                    bc = -ac * __ldg(p.fout + oidx);
                }
            }
            seed(sc, fc, p.gamma, p.kstart, do_out);

            float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
            const int rpar = (t + 1) & 1;  // parity written at step t-1
#pragma unroll
            for (int i = 0; i < KC; ++i) {
                if (i < K) {
                    float4 sin;
                    sin.x = __shfl_up_sync(FULL, S[i].x, 1);
                    sin.y = __shfl_up_sync(FULL, S[i].y, 1);
                    sin.z = __shfl_up_sync(FULL, S[i].z, 1);
                    sin.w = __shfl_up_sync(FULL, S[i].w, 1);
                    if (lane == 0) sin = (w == 0) ? make_float4(0.f, 0.f, 0.f, 0.f) : xfer[rpar][w - 1][i];
                    float4 d = D[i];
                    if (!BWD) {
                        d.x = fmaf(s0.zc, s0.u, d.x); d.x = fmaf(s1.zc, s1.u, d.x);
                        d.x = fmaf(s2.zc, s2.u, d.x); d.x = fmaf(s3.zc, s3.u, d.x);
                        d.y = fmaf(s0.zs, s0.u, d.y); d.y = fmaf(s1.zs, s1.u, d.y);
                        d.y = fmaf(s2.zs, s2.u, d.y); d.y = fmaf(s3.zs, s3.u, d.y);
                        d.z = ((d.z + s0.zc) - s1.zc) - s2.zc + s3.zc;
                        d.w = ((d.w + s0.zs) - s1.zs) - s2.zs + s3.zs;
                    } else {
                        d.x = fmaf(s0.zc, s0.u, d.x); d.x = fmaf(s1.zc, s1.u, d.x);
                        d.x = fmaf(s2.zc, s2.u, d.x); d.x = fmaf(s3.zc, s3.u, d.x);
                        d.y = fmaf(s0.zs, s0.u, d.y); d.y = fmaf(s1.zs, s1.u, d.y);
                        d.y = fmaf(s2.zs, s2.u, d.y); d.y = fmaf(s3.zs, s3.u, d.y);
                        d.z = fmaf(s0.zc, s0.v, d.z); d.z = fmaf(s1.zc, s1.v, d.z);
                        d.z = fmaf(s2.zc, s2.v, d.z); d.z = fmaf(s3.zc, s3.v, d.z);
                        d.w = fmaf(s0.zs, s0.v, d.w); d.w = fmaf(s1.zs, s1.v, d.w);
                        d.w = fmaf(s2.zs, s2.v, d.w); d.w = fmaf(s3.zs, s3.v, d.w);
                    }
                    D[i] = d;
                    float4 h;
                    h.x = sin.x + d.x; h.y = sin.y + d.y; h.z = sin.z + d.z; h.w = sin.w + d.w;
                    S[i] = h;
                    const float a = p.a[i];
                    const float ak = a * (float)(p.kstart + 2 * i);
                    if (!BWD) {
                        acc0 = fmaf(a, fmaf(sc.zc, h.x, sc.zs * h.y), acc0);   // num
                        acc1 = fmaf(a, fmaf(sc.zc, h.z, sc.zs * h.w), acc1);   // den
                        if (SAVE) {
                            acc2 = fmaf(ak, fmaf(sc.zc, h.y, -sc.zs * h.x), acc2);  // d num / d s
                            acc3 = fmaf(ak, fmaf(sc.zc, h.w, -sc.zs * h.z), acc3);  // d den / d s
                        }
                    } else {
                        // h = (Box[alpha C], Box[alpha S], Box[beta C], Box[beta S])
                        acc0 = fmaf(a, fmaf(h.x, sc.zc, h.y * sc.zs), acc0);
                        const float pp = fmaf(h.y, sc.zc, -h.x * sc.zs);
                        const float qq = fmaf(h.w, sc.zc, -h.z * sc.zs);
                        acc1 = fmaf(ak, fmaf(fc, pp, qq), acc1);
                    }
                    rot(s0); rot(s1); rot(s2); rot(s3); rot(sc);
                }
            }
            if (lane == 31 && w + 1 < (Wi >> 5)) {
#pragma unroll
                for (int i = 0; i < KC; ++i)
                    if (i < K) xfer[t & 1][w][i] = S[i];
            }
            if (do_out) {
                if (!BWD) {
                    p.out[oidx] = acc0 / acc1;
                    if (SAVE) {
                        p.sv_den[oidx] = acc1;
                        p.sv_dnum[oidx] = acc2;
                        p.sv_dden[oidx] = acc3;
                    }
                } else {
                    const float gt = acc1 + ac * __ldg(p.bdnum + oidx) + bc * __ldg(p.bdden + oidx);
                    if (p.gimg) p.gimg[oidx] = acc0 + p.gamma * gt;
                    gsum = fmaf(fc, gt, gsum);
                }
            }
        }
        __syncthreads();
    }

    if (BWD && p.partial) {
        __shared__ float red[8];
        for (int o = 16; o > 0; o >>= 1) gsum += __shfl_down_sync(FULL, gsum, o);
        if (lane == 0) red[w] = gsum;
        __syncthreads();
        if (j == 0) {
            float v = 0.f;
            for (int q = 0; q < (Wi >> 5); ++q) v += red[q];
            p.partial[blockIdx.y * gridDim.x + blockIdx.x] = v;
        }
    }
}

template <int KC, bool BWD, bool SAVE, typename Tin>
static cudaError_t sys_launch(const SysParams& p, int wi, int gx, int gy, cudaStream_t s) {
    dim3 grid(gx, gy);
    bf_sys_kernel<KC, BWD, SAVE, Tin><<<grid, wi, 0, s>>>(p);
    return cudaGetLastError();
}

template <bool BWD, bool SAVE, typename Tin>
static cudaError_t sys_launch_k(const SysParams& p, int wi, int gx, int gy, cudaStream_t s) {
    if (p.K <= 8) return sys_launch<8, BWD, SAVE, Tin>(p, wi, gx, gy, s);
    if (p.K <= 16) return sys_launch<16, BWD, SAVE, Tin>(p, wi, gx, gy, s);
    return sys_launch<SYS_KMAX, BWD, SAVE, Tin>(p, wi, gx, gy, s);
}

cudaError_t launch_sys(const SysParams& p, bool bwd, bool save, int in_dtype, int wi, int gx,
                       int gy, cudaStream_t s) {
    if (p.K > SYS_KMAX) return cudaErrorInvalidValue;
    if (in_dtype == BF_BF16) {
        if (bwd) return sys_launch_k<true, false, __nv_bfloat16>(p, wi, gx, gy, s);
        return save ? sys_launch_k<false, true, __nv_bfloat16>(p, wi, gx, gy, s)
                    : sys_launch_k<false, false, __nv_bfloat16>(p, wi, gx, gy, s);
    }
    if (bwd) return sys_launch_k<true, false, float>(p, wi, gx, gy, s);
    return save ? sys_launch_k<false, true, float>(p, wi, gx, gy, s)
                : sys_launch_k<false, false, float>(p, wi, gx, gy, s);
}

}  // namespace bf
