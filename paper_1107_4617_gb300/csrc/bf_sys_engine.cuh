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
#pragma once
#include "bf_internal.cuh"

namespace bf {
namespace sysd {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float ld_img(const float* p, size_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_img(const __nv_bfloat16* p, size_t i) {
    return __bfloat162float(p[i]);
}

// Rotation state of one pixel stream, two harmonics at a time (packed FP32
// pairs): zc/zs hold (cos, sin) of harmonics k and k+2; both advance by
// w^2 = e^{4 i theta} per pair. c2, s2, ns2 = (cos 4theta, sin 4theta,
// -sin 4theta) duplicated in both halves. A masked stream has z = 0.
struct Rot2 {
    float2 zc, zs, c2, s2, ns2;
};

// k0 theta reduced to [-pi, pi] (two-term Cody-Waite reduction by 2 pi;
// 2 pi = TWO_PI_HI + TWO_PI_LO with TWO_PI_HI = 6.28125 exact in 9 bits, so
// n * TWO_PI_HI is exact for the n < 2^15 that occur here), then MUFU sincos.
constexpr float TWO_PI_HI = 6.28125f;
constexpr float TWO_PI_LO = 1.9353071795864769e-3f;  // 2 pi - 6.28125
constexpr float INV_TWO_PI = 0.15915494309189535f;

__device__ __forceinline__ void sincos_reduced(float x, float* s, float* c) {
    const float n = rintf(x * INV_TWO_PI);
    const float y = fmaf(-n, TWO_PI_LO, fmaf(-n, TWO_PI_HI, x));
    __sincosf(y, s, c);
}

// k0 = frequency of the first harmonic (k0 <= 1 for an unchunked filter; a
// later harmonic chunk starts at k0 = kstart + 2 i0 and seeds from k0 theta).
__device__ __forceinline__ Rot2 seed2(float f, float gamma, float gpi, int k0, bool on) {
    float sn, cs;
    __sincosf(gamma * f, &sn, &cs);
    const float wc = (cs - sn) * (cs + sn);   // e^{2 i theta}
    const float ws = 2.0f * sn * cs;
    float z0c, z0s;                           // harmonic k0
    if (k0 == 0) { z0c = 1.0f; z0s = 0.0f; }
    else if (k0 == 1) { z0c = cs; z0s = sn; }
    else sincos_reduced((float)k0 * (gamma * f), &z0s, &z0c);
    const float z1c = fmaf(z0c, wc, -z0s * ws);  // harmonic k0 + 2
    const float z1s = fmaf(z0s, wc, z0c * ws);
    const float w2c = fmaf(wc, wc, -ws * ws);    // e^{4 i theta}
    const float w2s = 2.0f * wc * ws;
    Rot2 r;
    r.zc = on ? make_float2(z0c, z1c) : make_float2(0.f, 0.f);
    r.zs = on ? make_float2(z0s, z1s) : make_float2(0.f, 0.f);
    r.c2 = make_float2(w2c, w2c);
    r.s2 = make_float2(w2s, w2s);
    r.ns2 = make_float2(-w2s, -w2s);
    return r;
}

__device__ __forceinline__ void rot2(Rot2& s) {
    const float2 c = __ffma2_rn(s.zs, s.ns2, __fmul2_rn(s.zc, s.c2));
    const float2 n = __ffma2_rn(s.zc, s.s2, __fmul2_rn(s.zs, s.c2));
    s.zc = c;
    s.zs = n;
}

__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }

// Predicated shared store (lane 31's hand-off to the next warp): one
// instruction, no branch inside the unrolled harmonic loop.
__device__ __forceinline__ void st_shared_if(float4* dst, float4 v, bool pred) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %5, 0;\n\t"
        "@p st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n\t}"
        :: "r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"((int)pred) : "memory");
}

// Rows ahead of the current entering row that are pulled into L2.
constexpr int PREFETCH_ROWS = 8;

template <typename T>
__device__ __forceinline__ void prefetch_l2(const T* ptr) {
    asm volatile("prefetch.global.L2 [%0];" :: "l"(ptr));
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
    float dnum, dden;  // centre stream only: saved d num/ds, d den/ds
};

// zo / zs: element offsets of this image in the image-sized and the saved
// (3 planes per image) buffers of a [B, H, W] launch.
template <bool BWD, typename Tin>
__device__ __forceinline__ void load_px(Px<BWD>& v, const SysParams& p, const Tin* img, bool on,
                                        size_t q, size_t zo, size_t zs) {
    if (!on) {
        v.f = 0.f;
        if constexpr (BWD) { v.g = 0.f; v.den = 1.f; v.out = 0.f; v.dnum = 0.f; v.dden = 0.f; }
        return;
    }
    v.f = ld_img(img, q + zo);
    if constexpr (BWD) {
        v.g = __ldg(p.gout + q + zo);
        v.den = __ldg(p.bden + q + zs);
        v.out = __ldg(p.fout + q + zo);
    }
}

// The centre stream also needs the forward's saved centre derivatives.
template <bool BWD, typename Tin>
__device__ __forceinline__ void load_centre(Px<BWD>& v, const SysParams& p, const Tin* img,
                                            bool on, size_t q, size_t zo, size_t zs) {
    load_px<BWD, Tin>(v, p, img, on, q, zo, zs);
    if constexpr (BWD) {
        if (on) {
            v.dnum = __ldg(p.bdnum + q + zs);
            v.dden = __ldg(p.bdden + q + zs);
        }
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


// Shared-memory float4 slots one tile needs (KP harmonic pairs, Wi threads).
__host__ __device__ constexpr int sys_smem_slots(int KP, int Wi) {
    return 2 * KP * Wi + 2 * (Wi / 32) * 2 * KP + 2 * KP;
}

// One strip x band tile (bx, by) of one image, for one chunk of harmonics.
// Called uniformly by every thread of the CTA. gsum accumulates f * dL/dtheta
// (adjoint, last chunk only). KAHAN compensates the vertical running sums.
template <int KP, bool BWD, bool SAVE, bool KAHAN, typename Tin>
__device__ __forceinline__ void sys_tile(const SysParams& p, int bx, int by, size_t zo, size_t zs,
                                         float4* smem, float& gsum) {
    const int Wi = blockDim.x;
    const int NW = Wi >> 5;
    // S of each lane at the last step: [KP][2][Wi] float4, i.e. per harmonic
    // pair (x_k, x_k+2, y_k, y_k+2) and (z_k, z_k+2, w_k, w_k+2)
    float4* sbuf = smem;
    float4* xfer = smem + 2 * KP * Wi;        // [2][NW][KP][2]: lane 31 -> next warp
    float4* zero = xfer + 2 * NW * 2 * KP;    // [KP][2]: carry-in of the first lane
    const Tin* img = static_cast<const Tin*>(p.img);
    const int j = threadIdx.x;
    const int lane = j & 31;
    const int w = j >> 5;
    const int r = p.r;
    const int x0 = bx * p.Tw;
    const int cw = x0 - r + j;            // own column
    const int c2 = cw - 2 * r - 1;        // column leaving the horizontal window
    const int co = cw - r;                // output (centre) column
    const bool own_in = cw >= 0 && cw < p.W;
    const bool sec_in = (j >= 2 * r + 1) && c2 >= 0 && c2 < p.W;
    const bool out_lane = (j >= 2 * r) && co < p.W;
    const int y0 = by * p.Hb;
    const int rows = min(p.Hb, p.H - y0);
    const int span = rows + 2 * r;        // local steps of one thread
    const int steps = span + Wi - 1;

    for (int i = threadIdx.x; i < sys_smem_slots(KP, Wi); i += Wi)
        smem[i] = make_float4(0.f, 0.f, 0.f, 0.f);

    float2 Dx[KP], Dy[KP], Dz[KP], Dw[KP];
    float2 Ex[KAHAN ? KP : 1], Ey[KAHAN ? KP : 1], Ez[KAHAN ? KP : 1], Ew[KAHAN ? KP : 1];
#pragma unroll
    for (int i = 0; i < KP; ++i) {
        Dx[i] = make_float2(0.f, 0.f); Dy[i] = Dx[i]; Dz[i] = Dx[i]; Dw[i] = Dx[i];
        if constexpr (KAHAN) { Ex[i] = Dx[i]; Ey[i] = Dx[i]; Ez[i] = Dx[i]; Ew[i] = Dx[i]; }
    }

    // pixel values of the current step, loaded during the previous one
    Px<BWD> v0, v1, v2, v3, vc;
    // a warp is first active at step 32 w; start its prefetch chain there
    Geo g = geometry(p, w * 32 - j, span, y0, cw, c2, co, own_in, sec_in, out_lane);
    load_px<BWD, Tin>(v0, p, img, g.m0, g.q0, zo, zs);
    load_px<BWD, Tin>(v1, p, img, g.m1, g.q1, zo, zs);
    load_px<BWD, Tin>(v2, p, img, g.m2, g.q2, zo, zs);
    load_px<BWD, Tin>(v3, p, img, g.m3, g.q3, zo, zs);
    load_centre<BWD, Tin>(vc, p, img, g.out, g.qo, zo, zs);
    __syncthreads();

    for (int t = 0; t < steps; ++t) {
        const int warp_first = t - (w * 32 + 31);
        const int warp_last = t - w * 32;
        if (warp_last >= 0 && warp_first < span) {
            const Geo gc = g;  // geometry of this step
            const Px<BWD> c0 = v0, c1 = v1, c2v = v2, c3 = v3, cc = vc;
            // pull the entering row of a later step into L2 (no registers held):
            // the other four streams re-read pixels the strip touched recently
            {
                const int ef = y0 - r + (t + PREFETCH_ROWS - j);
                // (forward only: the adjoint's four extra streams made it slower)
                if (!BWD && own_in && ef >= 0 && ef < p.H)
                    prefetch_l2(static_cast<const Tin*>(p.img) + zo + (size_t)ef * p.W + cw);
            }
            // prefetch the next step's pixels; their latency hides under this step
            g = geometry(p, t + 1 - j, span, y0, cw, c2, co, own_in, sec_in, out_lane);
            load_px<BWD, Tin>(v0, p, img, g.m0, g.q0, zo, zs);
            load_px<BWD, Tin>(v1, p, img, g.m1, g.q1, zo, zs);
            load_px<BWD, Tin>(v2, p, img, g.m2, g.q2, zo, zs);
            load_px<BWD, Tin>(v3, p, img, g.m3, g.q3, zo, zs);
            load_centre<BWD, Tin>(vc, p, img, g.out, g.qo, zo, zs);

            Rot2 s0 = seed2(c0.f, p.gamma, p.gpi, p.k0, gc.m0);
            Rot2 s1 = seed2(c1.f, p.gamma, p.gpi, p.k0, gc.m1);
            Rot2 s2 = seed2(c2v.f, p.gamma, p.gpi, p.k0, gc.m2);
            Rot2 s3 = seed2(c3.f, p.gamma, p.gpi, p.k0, gc.m3);
            Rot2 sc = seed2(cc.f, p.gamma, p.gpi, p.k0, gc.out);
            // plane weights (u: first two planes, v: last two) with the stream's
            // sign: + own enter, - second enter, - own leave, + second leave
            float2 U0, U1, U2, U3, V0, V1, V2, V3;
            float ac = 0.f, bc = 0.f;
            if constexpr (!BWD) {
                U0 = dup(c0.f); U1 = dup(-c1.f); U2 = dup(-c2v.f); U3 = dup(c3.f);
                V0 = dup(1.f); V1 = dup(-1.f); V2 = dup(-1.f); V3 = dup(1.f);
            } else {
                const float a0 = __fdividef(c0.g, c0.den), a1 = __fdividef(c1.g, c1.den);
                const float a2 = __fdividef(c2v.g, c2v.den), a3 = __fdividef(c3.g, c3.den);
                U0 = dup(a0); U1 = dup(-a1); U2 = dup(-a2); U3 = dup(a3);
                V0 = dup(-a0 * c0.out); V1 = dup(a1 * c1.out);
                V2 = dup(a2 * c2v.out); V3 = dup(-a3 * c3.out);
                ac = __fdividef(cc.g, cc.den);
                bc = -ac * cc.out;
            }
            const float2 FC = dup(cc.f);

            // where this lane reads its left neighbour's S of the previous step
            const float4* rd;
            int rstride;
            if (lane != 0) { rd = sbuf + (j - 1); rstride = Wi; }
            else if (w != 0) { rd = xfer + (((t + 1) & 1) * NW + (w - 1)) * 2 * KP; rstride = 1; }
            else { rd = zero; rstride = 1; }
            float4* wr = sbuf + j;
            float4* wx = xfer + ((t & 1) * NW + w) * 2 * KP;
            const bool carry = (lane == 31) && (w + 1 < NW);

            float2 NUM = make_float2(0.f, 0.f), DEN = NUM, DNUM = NUM, DDEN = NUM;
            // carry-ins read one pair ahead: a slot of pair i is only rewritten
            // after the __syncwarp of iteration i, so earlier reads are safe
            float4 ina = rd[0], inb = rd[rstride];
#pragma unroll
            for (int i = 0; i < KP; ++i) {
                const float4 A = ina, B = inb;
                if (i + 1 < KP) { ina = rd[(2 * i + 2) * rstride]; inb = rd[(2 * i + 3) * rstride]; }
                float2 dx, dy, dz, dw;
                if constexpr (!KAHAN) {
                    dx = Dx[i]; dy = Dy[i]; dz = Dz[i]; dw = Dw[i];
                    dx = __ffma2_rn(s0.zc, U0, dx); dx = __ffma2_rn(s1.zc, U1, dx);
                    dx = __ffma2_rn(s2.zc, U2, dx); dx = __ffma2_rn(s3.zc, U3, dx);
                    dy = __ffma2_rn(s0.zs, U0, dy); dy = __ffma2_rn(s1.zs, U1, dy);
                    dy = __ffma2_rn(s2.zs, U2, dy); dy = __ffma2_rn(s3.zs, U3, dy);
                    dz = __ffma2_rn(s0.zc, V0, dz); dz = __ffma2_rn(s1.zc, V1, dz);
                    dz = __ffma2_rn(s2.zc, V2, dz); dz = __ffma2_rn(s3.zc, V3, dz);
                    dw = __ffma2_rn(s0.zs, V0, dw); dw = __ffma2_rn(s1.zs, V1, dw);
                    dw = __ffma2_rn(s2.zs, V2, dw); dw = __ffma2_rn(s3.zs, V3, dw);
                } else {
                    // this row's increment of each running sum, then a
                    // Kahan-compensated add (Kahan 1965): y = inc - e,
                    // t = D + y, e = (t - D) - y, D = t
                    const float2 m1 = dup(-1.f);
                    float2 ix = __fmul2_rn(s0.zc, U0), iy = __fmul2_rn(s0.zs, U0);
                    float2 iz = __fmul2_rn(s0.zc, V0), iw = __fmul2_rn(s0.zs, V0);
                    ix = __ffma2_rn(s1.zc, U1, ix); ix = __ffma2_rn(s2.zc, U2, ix);
                    ix = __ffma2_rn(s3.zc, U3, ix);
                    iy = __ffma2_rn(s1.zs, U1, iy); iy = __ffma2_rn(s2.zs, U2, iy);
                    iy = __ffma2_rn(s3.zs, U3, iy);
                    iz = __ffma2_rn(s1.zc, V1, iz); iz = __ffma2_rn(s2.zc, V2, iz);
                    iz = __ffma2_rn(s3.zc, V3, iz);
                    iw = __ffma2_rn(s1.zs, V1, iw); iw = __ffma2_rn(s2.zs, V2, iw);
                    iw = __ffma2_rn(s3.zs, V3, iw);
                    auto kadd = [&](float2& D, float2& E, float2 inc) {
                        const float2 y = __ffma2_rn(E, m1, inc);
                        const float2 t2 = __fadd2_rn(D, y);
                        E = __ffma2_rn(y, m1, __ffma2_rn(D, m1, t2));
                        D = t2;
                    };
                    kadd(Dx[i], Ex[i], ix); kadd(Dy[i], Ey[i], iy);
                    kadd(Dz[i], Ez[i], iz); kadd(Dw[i], Ew[i], iw);
                    dx = Dx[i]; dy = Dy[i]; dz = Dz[i]; dw = Dw[i];
                }
                Dx[i] = dx; Dy[i] = dy; Dz[i] = dz; Dw[i] = dw;
                const float2 hx = __fadd2_rn(make_float2(A.x, A.y), dx);
                const float2 hy = __fadd2_rn(make_float2(A.z, A.w), dy);
                const float2 hz = __fadd2_rn(make_float2(B.x, B.y), dz);
                const float2 hw = __fadd2_rn(make_float2(B.z, B.w), dw);
                __syncwarp();  // every lane has read its neighbour's slots before they change
                const float4 oa = make_float4(hx.x, hx.y, hy.x, hy.y);
                const float4 ob = make_float4(hz.x, hz.y, hw.x, hw.y);
                wr[(2 * i) * Wi] = oa;
                wr[(2 * i + 1) * Wi] = ob;
                st_shared_if(wx + 2 * i, oa, carry);
                st_shared_if(wx + 2 * i + 1, ob, carry);
                const float2 A2 = make_float2(p.a[2 * i], p.a[2 * i + 1]);
                const float2 AK2 = make_float2(p.ak[2 * i], p.ak[2 * i + 1]);
                const float2 nzs = __fmul2_rn(sc.zs, dup(-1.f));
                if constexpr (!BWD) {
                    NUM = __ffma2_rn(A2, __ffma2_rn(sc.zc, hx, __fmul2_rn(sc.zs, hy)), NUM);
                    DEN = __ffma2_rn(A2, __ffma2_rn(sc.zc, hz, __fmul2_rn(sc.zs, hw)), DEN);
                    if constexpr (SAVE) {
                        DNUM = __ffma2_rn(AK2, __ffma2_rn(sc.zc, hy, __fmul2_rn(nzs, hx)), DNUM);
                        DDEN = __ffma2_rn(AK2, __ffma2_rn(sc.zc, hw, __fmul2_rn(nzs, hz)), DDEN);
                    }
                } else {
                    // h = (Box[alpha C], Box[alpha S], Box[beta C], Box[beta S])
                    NUM = __ffma2_rn(A2, __ffma2_rn(hx, sc.zc, __fmul2_rn(hy, sc.zs)), NUM);
                    const float2 pp = __ffma2_rn(hy, sc.zc, __fmul2_rn(hx, nzs));
                    const float2 qq = __ffma2_rn(hw, sc.zc, __fmul2_rn(hz, nzs));
                    DEN = __ffma2_rn(AK2, __ffma2_rn(FC, pp, qq), DEN);
                }
                rot2(s0); rot2(s1); rot2(s2); rot2(s3); rot2(sc);
            }
            if (gc.out) {
                const size_t o = gc.qo + zo;   // image-sized buffers
                const size_t os = gc.qo + zs;  // saved buffers
                float num = NUM.x + NUM.y, den = DEN.x + DEN.y;
                // chunked harmonics: partial sums live in the output buffers
                // between chunks (acc: 0 single, 1 first, 2 middle, 3 last)
                const int acc = p.acc;
                if constexpr (!BWD) {
                    float dn = DNUM.x + DNUM.y, dd = DDEN.x + DDEN.y;
                    float* dbuf = SAVE ? p.sv_den + zs : p.acc_den + zo;
                    if (acc >= 2) {
                        num += p.out[o];
                        den += dbuf[gc.qo];
                        if constexpr (SAVE) { dn += p.sv_dnum[os]; dd += p.sv_dden[os]; }
                    }
                    p.out[o] = (acc == 0 || acc == 3) ? num / den : num;
                    if (SAVE || acc != 0) dbuf[gc.qo] = den;
                    if constexpr (SAVE) { p.sv_dnum[os] = dn; p.sv_dden[os] = dd; }
                } else {
                    if (acc >= 2) { num += p.acc_gv[o]; den += p.acc_gt[o]; }
                    if (acc == 0 || acc == 3) {
                        const float gt = den + ac * cc.dnum + bc * cc.dden;
                        if (p.gimg) p.gimg[o] = num + p.gamma * gt;
                        gsum = fmaf(cc.f, gt, gsum);
                    } else {
                        p.acc_gv[o] = num;
                        p.acc_gt[o] = den;
                    }
                }
            }
        }
        __syncthreads();
    }
}

// Per-CTA sum of gsum (adjoint), written to partial[slot].
__device__ __forceinline__ void cta_sum_to(float gsum, float* partial, int slot) {
    __shared__ float red[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) gsum += __shfl_down_sync(FULL, gsum, o);
    if (lane == 0) red[w] = gsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += red[q];
        partial[slot] = v;
    }
    __syncthreads();
}

}  // namespace sysd

// One CTA per tile. WMAX = largest strip width (threads) of the instantiation:
// 128-thread strips run two CTAs per SM, 256-thread strips one.
template <int KP, bool BWD, bool SAVE, bool KAHAN, int WMAX, typename Tin>
__global__ void __launch_bounds__(WMAX, 256 / WMAX) bf_sys_kernel(SysParams p) {
    extern __shared__ float4 smem[];
    float gsum = 0.f;
    const size_t z = blockIdx.z;  // image of a [B, H, W] launch
    const size_t hw = (size_t)p.H * p.W;
    sysd::sys_tile<KP, BWD, SAVE, KAHAN, Tin>(p, blockIdx.x, blockIdx.y, z * hw, z * 3 * hw, smem,
                                              gsum);
    if (BWD && p.partial)
        sysd::cta_sum_to(gsum, p.partial, (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
}

template <int KP, bool BWD, bool SAVE, bool KAHAN, int WMAX, typename Tin>
cudaError_t sys_launch_one(const SysParams& p, int wi, int gx, int gy, cudaStream_t s) {
    const int gz = p.B > 0 ? p.B : 1;
    auto kern = bf_sys_kernel<KP, BWD, SAVE, KAHAN, WMAX, Tin>;
    const size_t smem = sizeof(float4) * (size_t)sysd::sys_smem_slots(KP, wi);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(gx, gy, gz), wi, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace bf

