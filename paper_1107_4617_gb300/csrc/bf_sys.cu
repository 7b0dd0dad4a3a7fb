// Register-resident skewed-strip engine for the forward filter and its
// adjoint (Algorithm 2 with M = 1 and range kernel q_N, Sec. 2-3).
//
// A CTA owns a strip of Wi = blockDim.x consecutive input columns and a band
// of output rows; thread j owns column cw(j) = x0 - r + j. Two moving sums
// (Sec. 2, Sum(F, x, T)) make the (2r+1)^2 box:
//
//  * vertical: thread j keeps, for every harmonic, a running sum over the
//    2r+1 rows of the window -- of the DIFFERENCE D = V(cw(j)) -
//    V(cw(j) - 2r - 1) of two columns. Per row it adds the entering pixel's
//    planes of both columns and subtracts the leaving ones. All four pixels'
//    planes are regenerated from f (one MUFU sincos per pixel, harmonics by
//    complex rotation z_{k+2} = z_k z_2), so no plane is ever stored.
//  * horizontal: the window sum S(j) = sum_{i=j-2r..j} V(cw(i)) obeys
//    S(j) = S(j-1) + D(j). Thread j processes output row rho at step
//    t = rho_index + j, one step after thread j-1 produced S(j-1) for the
//    same row, and reads it from a one-row shared buffer (a double-buffered
//    slot per warp carries it across warp boundaries). The strip is swept
//    on a skew of one row per column.
//
// S(j) is the full box sum centred on column cw(j) - r; thread j combines it
// with that centre pixel's C_k, S_k and a_k (Algorithm 2 step 3). Per
// harmonic a thread keeps 4 floats of state (D) in registers; S passes
// through shared memory (16 B written and read per harmonic and step).
#include "bf_internal.cuh"

namespace bf {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float ld_img(const float* p, size_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_img(const __nv_bfloat16* p, size_t i) {
    return __bfloat162float(p[i]);
}

// Rotation state of one pixel stream: z = current harmonic (cos, sin),
// w = (cos 2 theta, sin 2 theta). A masked stream has z = 0.
struct Rot {
    float zc, zs, wc, ws;
};

__device__ __forceinline__ Rot seed(float f, float gamma, int kstart, bool on) {
    float sn, cs;
    __sincosf(gamma * f, &sn, &cs);
    Rot s;
    s.wc = (cs - sn) * (cs + sn);
    s.ws = 2.0f * sn * cs;
    s.zc = on ? (kstart ? cs : 1.0f) : 0.0f;
    s.zs = on ? (kstart ? sn : 0.0f) : 0.0f;
    return s;
}

__device__ __forceinline__ void rot(Rot& s) {
    const float c = fmaf(s.zc, s.wc, -s.zs * s.ws);
    const float n = fmaf(s.zs, s.wc, s.zc * s.ws);
    s.zc = c;
    s.zs = n;
}

// Predicated shared store (lane 31's hand-off to the next warp): one
// instruction, no branch inside the unrolled harmonic loop.
__device__ __forceinline__ void st_shared_if(float4* dst, float4 v, bool pred) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %5, 0;\n\t"
        "@p st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n\t}"
        :: "r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"((int)pred) : "memory");
}

// Per-pixel values a stream needs, loaded one step ahead.
template <bool BWD>
struct Px;
template <>
struct Px<false> {
    float f;
};
template <>
struct Px<true> {
    float f, g, den, out;
};

template <bool BWD, typename Tin>
__device__ __forceinline__ void load_px(Px<BWD>& v, const SysParams& p, const Tin* img, bool on,
                                        size_t q) {
    if (!on) {
        v.f = 0.f;
        if constexpr (BWD) { v.g = 0.f; v.den = 1.f; v.out = 0.f; }
        return;
    }
    v.f = ld_img(img, q);
    if constexpr (BWD) {
        v.g = __ldg(p.gout + q);
        v.den = __ldg(p.bden + q);
        v.out = __ldg(p.fout + q);
    }
}

// Row/column geometry of thread j at local step tau.
struct Geo {
    bool m0, m1, m2, m3, out;
    size_t q0, q1, q2, q3, qo;
};

__device__ __forceinline__ Geo geometry(const SysParams& p, int tau, int span, int y0, int cw,
                                        int c2, int co, bool own_in, bool sec_in, bool out_lane) {
    const int r = p.r;
    const bool act = tau >= 0 && tau < span;
    const int e = y0 - r + tau;
    const int l = e - 2 * r - 1;
    const int rho = y0 - 2 * r + tau;
    const bool in_e = act && e >= 0 && e < p.H;
    const bool in_l = act && tau >= 2 * r + 1 && l >= 0 && l < p.H;
    Geo g;
    g.m0 = in_e && own_in;
    g.m1 = in_e && sec_in;
    g.m2 = in_l && own_in;
    g.m3 = in_l && sec_in;
    g.out = act && tau >= 2 * r && out_lane;
    const size_t re = (size_t)(in_e ? e : 0) * p.W, rl = (size_t)(in_l ? l : 0) * p.W;
    g.q0 = re + (g.m0 ? cw : 0);
    g.q1 = re + (g.m1 ? c2 : 0);
    g.q2 = rl + (g.m2 ? cw : 0);
    g.q3 = rl + (g.m3 ? c2 : 0);
    g.qo = g.out ? (size_t)rho * p.W + co : 0;
    return g;
}

}  // namespace

// 128-thread strips, two resident CTAs per SM.
template <int KC, bool BWD, bool SAVE, typename Tin>
__global__ void __launch_bounds__(SYS_MAX_THREADS, 2) bf_sys_kernel(SysParams p) {
    extern __shared__ float4 smem[];
    const int Wi = blockDim.x;
    const int NW = Wi >> 5;
    float4* sbuf = smem;                    // [KC][Wi]: S of each lane, last step
    float4* xfer = smem + KC * Wi;          // [2][NW][KC]: lane 31 -> next warp's lane 0
    float4* zero = xfer + 2 * NW * KC;      // [KC]: carry-in of the first lane
    const Tin* img = static_cast<const Tin*>(p.img);
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

    for (int i = threadIdx.x; i < KC * Wi + 2 * NW * KC + KC; i += Wi)
        smem[i] = make_float4(0.f, 0.f, 0.f, 0.f);

    float4 D[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) D[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    float gsum = 0.f;

    // pixel values of the current step, loaded during the previous one
    Px<BWD> v0, v1, v2, v3, vc;
    // a warp is first active at step 32 w; start its prefetch chain there
    Geo g = geometry(p, w * 32 - j, span, y0, cw, c2, co, own_in, sec_in, out_lane);
    load_px<BWD, Tin>(v0, p, img, g.m0, g.q0);
    load_px<BWD, Tin>(v1, p, img, g.m1, g.q1);
    load_px<BWD, Tin>(v2, p, img, g.m2, g.q2);
    load_px<BWD, Tin>(v3, p, img, g.m3, g.q3);
    load_px<BWD, Tin>(vc, p, img, g.out, g.qo);
    __syncthreads();

    for (int t = 0; t < steps; ++t) {
        const int warp_first = t - (w * 32 + 31);
        const int warp_last = t - w * 32;
        if (warp_last >= 0 && warp_first < span) {
            const Geo gc = g;  // geometry of this step
            const Px<BWD> c0 = v0, c1 = v1, c2v = v2, c3 = v3, cc = vc;
            // prefetch the next step's pixels; their latency hides under this step
            g = geometry(p, t + 1 - j, span, y0, cw, c2, co, own_in, sec_in, out_lane);
            load_px<BWD, Tin>(v0, p, img, g.m0, g.q0);
            load_px<BWD, Tin>(v1, p, img, g.m1, g.q1);
            load_px<BWD, Tin>(v2, p, img, g.m2, g.q2);
            load_px<BWD, Tin>(v3, p, img, g.m3, g.q3);
            load_px<BWD, Tin>(vc, p, img, g.out, g.qo);

            Rot s0 = seed(c0.f, p.gamma, p.kstart, gc.m0);
            Rot s1 = seed(c1.f, p.gamma, p.kstart, gc.m1);
            Rot s2 = seed(c2v.f, p.gamma, p.kstart, gc.m2);
            Rot s3 = seed(c3.f, p.gamma, p.kstart, gc.m3);
            Rot sc = seed(cc.f, p.gamma, p.kstart, gc.out);
            // plane weights with the stream's sign: + own enter, - second enter,
            // - own leave, + second leave
            float u0, u1, u2, u3, b0 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f, ac = 0.f, bc = 0.f;
            if constexpr (!BWD) {
                u0 = c0.f; u1 = -c1.f; u2 = -c2v.f; u3 = c3.f;
            } else {
                const float a0 = __fdividef(c0.g, c0.den), a1 = __fdividef(c1.g, c1.den);
                const float a2 = __fdividef(c2v.g, c2v.den), a3 = __fdividef(c3.g, c3.den);
                u0 = a0; u1 = -a1; u2 = -a2; u3 = a3;
                b0 = -a0 * c0.out; b1 = a1 * c1.out; b2 = a2 * c2v.out; b3 = -a3 * c3.out;
                ac = __fdividef(cc.g, cc.den);
                bc = -ac * cc.out;
            }

            // where this lane reads its left neighbour's S of the previous step
            const float4* rd;
            int rstride;
            if (lane != 0) { rd = sbuf + (j - 1); rstride = Wi; }
            else if (w != 0) { rd = xfer + (((t + 1) & 1) * NW + (w - 1)) * KC; rstride = 1; }
            else { rd = zero; rstride = 1; }
            float4* wr = sbuf + j;
            float4* wx = xfer + ((t & 1) * NW + w) * KC;
            const bool carry = (lane == 31) && (w + 1 < NW);

            float n0 = 0.f, n1 = 0.f, d0 = 0.f, d1 = 0.f, e0 = 0.f, e1 = 0.f, h0 = 0.f, h1 = 0.f;
            // carry-ins are read two harmonics ahead: a slot of harmonic i is only
            // rewritten after the __syncwarp of iteration i, so earlier reads are safe
            float4 sin_a = rd[0];
            float4 sin_b = (KC > 1) ? rd[rstride] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int i = 0; i < KC; ++i) {
                {
                    const float4 sin = sin_a;
                    sin_a = sin_b;
                    if (i + 2 < KC) sin_b = rd[(i + 2) * rstride];
                    float4 d = D[i];
                    d.x = fmaf(s0.zc, u0, d.x); d.x = fmaf(s1.zc, u1, d.x);
                    d.x = fmaf(s2.zc, u2, d.x); d.x = fmaf(s3.zc, u3, d.x);
                    d.y = fmaf(s0.zs, u0, d.y); d.y = fmaf(s1.zs, u1, d.y);
                    d.y = fmaf(s2.zs, u2, d.y); d.y = fmaf(s3.zs, u3, d.y);
                    if constexpr (!BWD) {
                        d.z = ((d.z + s0.zc) - s1.zc) - s2.zc + s3.zc;
                        d.w = ((d.w + s0.zs) - s1.zs) - s2.zs + s3.zs;
                    } else {
                        d.z = fmaf(s0.zc, b0, d.z); d.z = fmaf(s1.zc, b1, d.z);
                        d.z = fmaf(s2.zc, b2, d.z); d.z = fmaf(s3.zc, b3, d.z);
                        d.w = fmaf(s0.zs, b0, d.w); d.w = fmaf(s1.zs, b1, d.w);
                        d.w = fmaf(s2.zs, b2, d.w); d.w = fmaf(s3.zs, b3, d.w);
                    }
                    D[i] = d;
                    float4 h;
                    h.x = sin.x + d.x; h.y = sin.y + d.y; h.z = sin.z + d.z; h.w = sin.w + d.w;
                    __syncwarp();  // every lane has read its neighbour's slot before it changes
                    wr[i * Wi] = h;
                    st_shared_if(wx + i, h, carry);
                    const float a = p.a[i];
                    const float ak = p.ak[i];
                    float& N_ = (i & 1) ? n1 : n0;
                    float& Dn = (i & 1) ? d1 : d0;
                    if constexpr (!BWD) {
                        N_ = fmaf(a, fmaf(sc.zc, h.x, sc.zs * h.y), N_);   // num
                        Dn = fmaf(a, fmaf(sc.zc, h.z, sc.zs * h.w), Dn);   // den
                        if constexpr (SAVE) {
                            float& E_ = (i & 1) ? e1 : e0;
                            float& F_ = (i & 1) ? h1 : h0;
                            E_ = fmaf(ak, fmaf(sc.zc, h.y, -sc.zs * h.x), E_);  // d num / d s
                            F_ = fmaf(ak, fmaf(sc.zc, h.w, -sc.zs * h.z), F_);  // d den / d s
                        }
                    } else {
                        // h = (Box[alpha C], Box[alpha S], Box[beta C], Box[beta S])
                        N_ = fmaf(a, fmaf(h.x, sc.zc, h.y * sc.zs), N_);
                        const float pp = fmaf(h.y, sc.zc, -h.x * sc.zs);
                        const float qq = fmaf(h.w, sc.zc, -h.z * sc.zs);
                        Dn = fmaf(ak, fmaf(cc.f, pp, qq), Dn);
                    }
                    rot(s0); rot(s1); rot(s2); rot(s3); rot(sc);
                }
            }
            if (gc.out) {
                const size_t o = gc.qo;
                const float num = n0 + n1, den = d0 + d1;
                if constexpr (!BWD) {
                    p.out[o] = num / den;
                    if constexpr (SAVE) {
                        p.sv_den[o] = den;
                        p.sv_dnum[o] = e0 + e1;
                        p.sv_dden[o] = h0 + h1;
                    }
                } else {
                    const float gt = den + ac * __ldg(p.bdnum + o) + bc * __ldg(p.bdden + o);
                    if (p.gimg) p.gimg[o] = num + p.gamma * gt;
                    gsum = fmaf(cc.f, gt, gsum);
                }
            }
        }
        __syncthreads();
    }

    if (BWD && p.partial) {
        __shared__ float red[SYS_MAX_THREADS / 32];
        for (int o = 16; o > 0; o >>= 1) gsum += __shfl_down_sync(FULL, gsum, o);
        if (lane == 0) red[w] = gsum;
        __syncthreads();
        if (j == 0) {
            float v = 0.f;
            for (int q = 0; q < NW; ++q) v += red[q];
            p.partial[blockIdx.y * gridDim.x + blockIdx.x] = v;
        }
    }
}

// Harmonic counts with their own instantiation; other K run on the next
// larger one with zero coefficients for the extra harmonics.
static int sys_kc(int K) {
    static const int kcs[] = {1, 2, 3, 4, 6, 8, 11, 14, 17, 21};
    for (int kc : kcs)
        if (K <= kc) return kc;
    return -1;
}

size_t sys_smem_bytes(int K, int wi) {
    const int kc = sys_kc(K);
    return sizeof(float4) * ((size_t)kc * wi + 2 * (size_t)(wi / 32) * kc + kc);
}

template <int KC, bool BWD, bool SAVE, typename Tin>
static cudaError_t sys_launch(const SysParams& p, int wi, int gx, int gy, cudaStream_t s) {
    auto kern = bf_sys_kernel<KC, BWD, SAVE, Tin>;
    const size_t smem = sizeof(float4) * ((size_t)KC * wi + 2 * (size_t)(wi / 32) * KC + KC);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(gx, gy);
    kern<<<grid, wi, smem, s>>>(p);
    return cudaGetLastError();
}

template <bool BWD, bool SAVE, typename Tin>
static cudaError_t sys_launch_k(const SysParams& p, int wi, int gx, int gy, cudaStream_t s) {
    switch (sys_kc(p.K)) {
        case 1: return sys_launch<1, BWD, SAVE, Tin>(p, wi, gx, gy, s);
        case 2: return sys_launch<2, BWD, SAVE, Tin>(p, wi, gx, gy, s);
        case 3: return sys_launch<3, BWD, SAVE, Tin>(p, wi, gx, gy, s);
        case 4: return sys_launch<4, BWD, SAVE, Tin>(p, wi, gx, gy, s);
        case 6: return sys_launch<6, BWD, SAVE, Tin>(p, wi, gx, gy, s);
        case 8: return sys_launch<8, BWD, SAVE, Tin>(p, wi, gx, gy, s);
        case 11: return sys_launch<11, BWD, SAVE, Tin>(p, wi, gx, gy, s);
        case 14: return sys_launch<14, BWD, SAVE, Tin>(p, wi, gx, gy, s);
        case 17: return sys_launch<17, BWD, SAVE, Tin>(p, wi, gx, gy, s);
        case 21: return sys_launch<21, BWD, SAVE, Tin>(p, wi, gx, gy, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sys(const SysParams& p_in, bool bwd, bool save, int in_dtype, int wi, int gx,
                       int gy, cudaStream_t s) {
    if (p_in.K > SYS_KMAX || wi > SYS_MAX_THREADS || wi % 32 != 0) return cudaErrorInvalidValue;
    SysParams p = p_in;
    for (int i = p.K; i < sys_kc(p.K); ++i) { p.a[i] = 0.f; p.ak[i] = 0.f; }  // padding harmonics
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
