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
//    planes are regenerated from f (one MUFU sincos per pixel, harmonic
//    pairs by a three-term recurrence), so no plane is ever stored.
//  * horizontal: the window sum S(j) = sum_{i=j-2r..j} V(cw(i)) obeys
//    S(j) = S(j-1) + D(j). Thread j processes output row rho at step
//    t = rho_index + j, one step after thread j-1 produced S(j-1) for the
//    same row, and reads it from a shared row buffer that is double-buffered
//    by step parity (so one CTA barrier per step orders every exchange, across
//    warps too). The strip is swept on a skew of one row per column.
//
// S(j) is the full box sum centred on column cw(j) - r; thread j combines it
// with that centre pixel's C_k, S_k and a_k (Algorithm 2 step 3). Per
// harmonic a thread keeps 4 floats of state (D) in registers; S passes
// through shared memory (16 B written and read per harmonic and step).
//
// The forward's planes carry f - mid in place of f (mid = T / 2, the centre
// of the range [0, T]) and it writes out = num / den + mid: num - mid den =
// sum_y (f(y) - mid) w(x, y), so the result is the same while the sums round
// against values half as large. The saved quads keep f and out shifted by
// mid. The adjoint depends on f only through differences (of theta, and of f
// against out), so it runs on the shifted values as they are; that removes
// most of the cancellation between its f and out terms.
//
// Harmonics come in pairs (k, k+2), packed in FP32x2 registers. Pair i+1
// follows from pairs i and i-1 by cos((n+1)x) = 2 cos(x) cos(nx) -
// cos((n-1)x) with x = 4 theta (the shift identity of Sec. 1 applied twice).
// Every stream stores pair i multiplied by s_i = (-1)^(i/2), which turns the
// recurrence into d_{i+1} = (+-m) d_i + d_{i-1}, m = 2 cos 4 theta, with no
// negation; since all planes of pair i carry the same s_i and the
// recombination multiplies two of them, the sign cancels there. An odd
// number of harmonics ends in a half pair (HALF): its one harmonic runs on
// scalar FP32 and passes one float4 per lane through shared memory.
//
// The first two pairs of every stream (the seed) come from one MUFU sincos
// of theta. For the first harmonic chunk the seed is specialised at compile
// time (SEED 1: odd N, harmonics 1, 3, 5, 7; SEED 2: even N, harmonics 2, 4,
// 6, 8, with the constant harmonic k = 0 kept apart as scalar planes); later
// chunks (SEED 0) start from a reduced sincos of k0 theta.
#pragma once
#include "bf_internal.cuh"

namespace bf {
namespace sysd {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float ld_img(const float* p, int i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_img(const __nv_bfloat16* p, int i) {
    return __bfloat162float(p[i]);
}

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

__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }

// One pixel stream: signed harmonic pairs i (c, s) and i+1 (nc, ns), each
// (harmonic k0 + 4i, harmonic k0 + 4i + 2); m = (2 cos 4 theta) twice, nm = -m.
struct Strm {
    float2 c, s, nc, ns, m, nm;
};

// k0 = frequency of the first harmonic of the launch (a later harmonic chunk
// starts at k0 = kstart + 2 i0 and seeds from a reduced sincos of k0 theta).
__device__ __forceinline__ Strm seed_general(float f, float gamma, int k0) {
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
    const float w4c = fmaf(wc, wc, -ws * ws);    // e^{4 i theta}
    const float w4s = 2.0f * wc * ws;
    Strm q;
    q.c = make_float2(z0c, z1c);
    q.s = make_float2(z0s, z1s);
    // pair 1 = pair 0 * e^{4 i theta} (s_1 = +1)
    q.nc = __ffma2_rn(q.s, dup(-w4s), __fmul2_rn(q.c, dup(w4c)));
    q.ns = __ffma2_rn(q.c, dup(w4s), __fmul2_rn(q.s, dup(w4c)));
    q.m = dup(2.0f * w4c);
    q.nm = dup(-2.0f * w4c);
    return q;
}

// Odd N, first chunk: harmonics 2, 3 theta from theta by the Chebyshev
// three-term recurrence in theta, m = 2 cos 4 theta = 4 cos^2 2theta - 2, and
// pair 1 (5, 7 theta) from pair 0 and its mirror (-3, -1 theta) by the
// recurrence in 4 theta.
__device__ __forceinline__ Strm seed_odd(float f, float gamma) {
    float s1, c1;
    __sincosf(gamma * f, &s1, &c1);
    const float cc = c1 + c1;
    const float c2 = fmaf(cc, c1, -1.0f);
    const float s2 = cc * s1;
    const float c3 = fmaf(cc, c2, -c1);
    const float s3 = fmaf(cc, s2, -s1);
    const float m = fmaf(4.0f * c2, c2, -2.0f);
    Strm q;
    q.c = make_float2(c1, c3);
    q.s = make_float2(s1, s3);
    q.nc = make_float2(fmaf(m, c1, -c3), fmaf(m, c3, -c1));
    q.ns = make_float2(fmaf(m, s1, s3), fmaf(m, s3, s1));
    q.m = dup(m);
    q.nm = dup(-m);
    return q;
}

// Even N, first chunk, the constant harmonic apart: pairs from harmonics
// 2, 4 theta; cos 4 theta = m / 2, and pair 1 (6, 8 theta) by the recurrence in
// 4 theta with the mirrors -2 theta and 0.
__device__ __forceinline__ Strm seed_even(float f, float gamma) {
    float s1, c1;
    __sincosf(gamma * f, &s1, &c1);
    const float cc = c1 + c1;
    const float c2 = fmaf(cc, c1, -1.0f);
    const float s2 = cc * s1;
    const float m = fmaf(4.0f * c2, c2, -2.0f);
    const float c4 = 0.5f * m;
    const float s4 = 2.0f * s2 * c2;
    Strm q;
    q.c = make_float2(c2, c4);
    q.s = make_float2(s2, s4);
    q.nc = make_float2(fmaf(m, c2, -c2), fmaf(m, c4, -1.0f));
    q.ns = make_float2(fmaf(m, s2, s2), m * s4);
    q.m = dup(m);
    q.nm = dup(-m);
    return q;
}

template <int SEED>
__device__ __forceinline__ Strm seed(float f, float gamma, int k0) {
    if constexpr (SEED == 1) return seed_odd(f, gamma);
    else if constexpr (SEED == 2) return seed_even(f, gamma);
    else return seed_general(f, gamma, k0);
}

// Step from pair i to pair i+1 and form pair i+2 when it is needed:
// d_{i+2} = (i+1 even ? m : -m) d_{i+1} + d_i. half: pair i+2 is the half
// pair (only its first component is formed).
__device__ __forceinline__ void advance(Strm& q, int i, bool need, bool half = false) {
    if (need) {
        const float2 mm = ((i + 1) & 1) ? q.nm : q.m;
        float2 c2, s2;
        if (half) {
            c2 = make_float2(fmaf(mm.x, q.nc.x, q.c.x), 0.f);
            s2 = make_float2(fmaf(mm.x, q.ns.x, q.s.x), 0.f);
        } else {
            c2 = __ffma2_rn(mm, q.nc, q.c);
            s2 = __ffma2_rn(mm, q.ns, q.s);
        }
        q.c = q.nc; q.s = q.ns; q.nc = c2; q.ns = s2;
    } else {
        q.c = q.nc; q.s = q.ns;
    }
}

// Rows ahead of the current entering row that are pulled into L2.
constexpr int PREFETCH_ROWS = 4;

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
// Adjoint: the forward's saved quad of the pixel (f - mid, 1/den, out - mid,
// dnum - out * dden) and dL/dout.
template <>
struct Px<true> {
    float4 sv;
    float g;
};

// Base pointers of one image of a [B, H, W] launch.
template <typename Tin>
struct Bases {
    const Tin* img;
    const float* gout;
    const float4* bsv;
};

// Masked loads leave neutral values (f = 0; in the adjoint g = 0, so the
// plane weights alpha, beta are 0); the forward masks its own weights.
// Forward: q = element offset in the row-pitched image. Adjoint: q = index
// in the saved quads (quad_index), qg = offset in the row-pitched dL/dout.
template <bool BWD, typename Tin>
__device__ __forceinline__ void load_px(Px<BWD>& v, const Bases<Tin>& b, bool on, int q, int qg) {
    if constexpr (!BWD) {
        v.f = 0.f;
        if (on) v.f = ld_img(b.img, q);
    } else {
        v.sv = make_float4(0.f, 0.f, 0.f, 0.f);
        v.g = 0.f;
        if (on) {
            v.sv = __ldg(b.bsv + q);
            v.g = __ldg(b.gout + qg);
        }
    }
}

template <bool BWD>
__device__ __forceinline__ float pix_f(const Px<BWD>& v) {
    if constexpr (BWD) return v.sv.x; else return v.f;
}

// Masks and element offsets of one step's five pixels (entering and leaving
// row of the own and the second column, centre) in the row-pitched image
// buffers (the forward's image, the adjoint's dL/dout).
struct Geo {
    bool m0, m1, m2, m3, out;
    int q0, q1, q2, q3, qo;
};

// Float4 slots of shared memory one tile needs: two step-parity buffers of
// 2 KP planes x (WMAX + 1) columns (column 0 stays zero: the first lane's
// carry-in), plus one row for the constant (DC) harmonic of even N when it
// runs apart from the pairs.
__host__ __device__ constexpr int sys_smem_slots(int KP, int WMAX, bool dc = false) {
    return 2 * (2 * KP + (dc ? 1 : 0)) * (WMAX + 1);
}

// One strip x band tile (bx, by) of one image, for one chunk of harmonics.
// Called uniformly by every thread of the CTA. gsum accumulates f * dL/dtheta
// (adjoint, last chunk only; f as the saved quads hold it, shifted by mid: the
// same sum, since the dL/dtheta of all pixels sum to 0). KAHAN compensates
// the vertical running sums.
// zo: element offset of this image in the compact buffers (saved quads, chunk
// accumulators); zp: in the row-pitched image buffers (img, out, dL/dout,
// dL/dimg, den), whose rows are p.ld elements apart. PITCH = false builds the
// compact case (p.ld = W) with the pitch terms compiled out.
template <int KP, bool BWD, bool SAVE, bool KAHAN, int WMAX, typename Tin, bool HALF = false,
          int SEED = 0, int FORM = 0, bool PITCH = true>
__device__ __forceinline__ void sys_tile(const SysParams& p, int bx, int by, size_t zo, size_t zp,
                                         float4* smem, float& gsum) {
    // SEED 2 (even N): the constant harmonic k = 0 runs apart from the pairs
    // (planes f and 1, or alpha in the adjoint: its k = 0 phase terms vanish),
    // and pair i holds harmonics 4i + 2, 4i + 4, i.e. coefficients CO + 2i.
    constexpr bool DC = SEED == 2;
    constexpr int CO = DC ? 1 : 0;
    // FORM: bits 0-1 the step-body form, bit 2 the ping-pong step loop, bit 3
    // the combine's sine terms negated on the box sums instead of on the
    // centre's harmonics
    constexpr int BODY = FORM & 3;
    constexpr bool PINGPONG = (FORM & 4) != 0;
    constexpr bool NEGFOLD = (FORM & 8) != 0;
    constexpr int LD = WMAX + 1;          // row of one plane in shared memory
    constexpr int BUF = (2 * KP + (DC ? 1 : 0)) * LD;  // one step-parity buffer
    const int Wi = blockDim.x;
    const int j = threadIdx.x;
    const int w = j >> 5;
    const int r = p.r;
    const int W = p.W;
    const int ld = PITCH ? p.ld : W;      // row pitch of the image buffers
    // row stride of the offsets Geo carries: the row-pitched image buffers
    // (the forward's image, the adjoint's dL/dout); the saved quads are
    // addressed by quad_index (sheared rows, compact)
    const int st = ld;
    const int x0 = bx * p.Tw;
    const int cw = x0 - r + j;            // own column
    const int c2 = cw - 2 * r - 1;        // column leaving the horizontal window
    const int co = cw - r;                // output (centre) column
    const bool own_in = cw >= 0 && cw < W;
    const bool sec_in = (j >= 2 * r + 1) && c2 >= 0 && c2 < W;
    const bool out_lane = (j >= 2 * r) && co < W;
    const int y0 = by * p.Hb;
    const int rows = min(p.Hb, p.H - y0);
    const int span = rows + 2 * r;        // local steps of one thread
    const int steps = span + Wi - 1;
    // rows that enter or leave the window: [elo, elo + ne)
    const int elo = max(0, y0 - r);
    const int ne = min(p.H, y0 + rows + r) - elo;

    Bases<Tin> b;
    b.img = static_cast<const Tin*>(p.img) + zp;
    if constexpr (BWD) {
        b.gout = p.gout + zp;
        b.bsv = p.bsv + zo;
    }

    for (int i = threadIdx.x; i < sys_smem_slots(KP, WMAX, DC); i += Wi)
        smem[i] = make_float4(0.f, 0.f, 0.f, 0.f);

    float2 Dx[KP], Dy[KP], Dz[KP], Dw[KP];
    float Dfa = 0.f, Dfz = 0.f;  // DC planes (f or alpha, and 1)
    float2 Ex[KAHAN ? KP : 1], Ey[KAHAN ? KP : 1], Ez[KAHAN ? KP : 1], Ew[KAHAN ? KP : 1];
#pragma unroll
    for (int i = 0; i < KP; ++i) {
        Dx[i] = make_float2(0.f, 0.f); Dy[i] = Dx[i]; Dz[i] = Dx[i]; Dw[i] = Dx[i];
        if constexpr (KAHAN) { Ex[i] = Dx[i]; Ey[i] = Dx[i]; Ez[i] = Dx[i]; Ew[i] = Dx[i]; }
    }

    // geometry of step t: entering row e = e0 + t, its element offset oe
    const int e0 = y0 - r - j;
    auto geometry = [&](int t) {
        const int e = e0 + t;
        const int tau = t - j;
        const int oe = e * st;
        const bool act = (unsigned)tau < (unsigned)span;
        const bool in_e = act && (unsigned)(e - elo) < (unsigned)ne;
        const bool in_l = act && (unsigned)(e - 2 * r - 1 - elo) < (unsigned)ne &&
                          tau >= 2 * r + 1;
        Geo g;
        g.m0 = in_e && own_in;
        g.m1 = in_e && sec_in;
        g.m2 = in_l && own_in;
        g.m3 = in_l && sec_in;
        g.out = act && out_lane && (unsigned)(e - r - y0) < (unsigned)rows;
        g.q0 = oe + cw;
        g.q1 = oe + c2;
        g.q2 = oe - (2 * r + 1) * st + cw;
        g.q3 = oe - (2 * r + 1) * st + c2;
        g.qo = oe - r * st + co;
        return g;
    };

    // pixel values of the current step, loaded during the previous one
    Px<BWD> vA[5], vB[5];
    // a warp is first active at step 32 w; start its prefetch chain there
    Geo gA = geometry(w * 32), gB = gA;
    // the adjoint's quad offsets (sheared, compact) of the step's pixels:
    // entering row e, leaving row e - 2r - 1, centre row e - r; its dL/dout
    // offsets are Geo's (row-pitched)
    auto quad_at = [&](int row, int col) { return quad_index(row, col, p.H, W); };
    auto load_step = [&](const Geo& gg, int t, Px<BWD> (&v)[5]) {
        if constexpr (BWD) {
            const int e = e0 + t, el = e - 2 * r - 1;
            load_px<BWD, Tin>(v[0], b, gg.m0, quad_at(e, cw), gg.q0);
            load_px<BWD, Tin>(v[1], b, gg.m1, quad_at(e, c2), gg.q1);
            load_px<BWD, Tin>(v[2], b, gg.m2, quad_at(el, cw), gg.q2);
            load_px<BWD, Tin>(v[3], b, gg.m3, quad_at(el, c2), gg.q3);
            load_px<BWD, Tin>(v[4], b, gg.out, quad_at(e - r, co), gg.qo);
        } else {
            load_px<BWD, Tin>(v[0], b, gg.m0, gg.q0, 0);
            load_px<BWD, Tin>(v[1], b, gg.m1, gg.q1, 0);
            load_px<BWD, Tin>(v[2], b, gg.m2, gg.q2, 0);
            load_px<BWD, Tin>(v[3], b, gg.m3, gg.q3, 0);
            load_px<BWD, Tin>(v[4], b, gg.out, gg.qo, 0);
        }
    };
    load_step(gA, w * 32, vA);
    __syncthreads();

    // One step t: its pixels (cur, loaded during step t - 1) are copied out
    // first, then step t + 1's loads are issued into nxt. The plain loop
    // passes one register set as both; the ping-pong loop alternates two sets
    // over pairs of steps, so no copy is made between steps. The two loops
    // compute the same sums; which schedules better differs between
    // instantiations.
    auto step = [&](int t, const Geo& gcur, const Px<BWD> (&cur)[5], Geo& gnext,
                    Px<BWD> (&nxt)[5]) {
        const int warp_first = t - (w * 32 + 31);
        const int warp_last = t - w * 32;
        if (warp_last >= 0 && warp_first < span) {
            const Geo gc = gcur;  // geometry of this step
            const Px<BWD> c0 = cur[0], c1 = cur[1], c2v = cur[2], c3 = cur[3], cc = cur[4];
            // pull the entering row of a later step into L2 (no registers held;
            // only rows that enter this band's window, so nothing past the
            // band is fetched): the other four streams re-read pixels the
            // strip touched recently
            {
                const int ef = e0 + t + PREFETCH_ROWS;
                if (own_in && (unsigned)(ef - elo) < (unsigned)ne) {
                    if constexpr (!BWD) {
                        prefetch_l2(b.img + ef * ld + cw);
                    } else {
                        prefetch_l2(b.bsv + quad_at(ef, cw));
                        prefetch_l2(b.gout + ef * ld + cw);
                    }
                }
            }
            // prefetch the next step's pixels; their latency hides under this step
            gnext = geometry(t + 1);
            load_step(gnext, t + 1, nxt);

            // plane weights (u: first two planes, v: last two) with the stream's
            // sign: + own enter, - second enter, - own leave, + second leave;
            // 0 for a masked stream
            float2 U0, U1, U2, U3, V0, V1, V2, V3;
            float xc = 0.f;  // adjoint: alpha dnum + beta dden of the centre
            if constexpr (!BWD) {
                // u = f - mid, v = 1 (0 for a masked stream)
                V0 = dup(gc.m0 ? 1.f : 0.f); V1 = dup(gc.m1 ? -1.f : 0.f);
                V2 = dup(gc.m2 ? -1.f : 0.f); V3 = dup(gc.m3 ? 1.f : 0.f);
                const float mc = p.mid;
                U0 = dup(gc.m0 ? c0.f - mc : 0.f); U1 = dup(gc.m1 ? mc - c1.f : 0.f);
                U2 = dup(gc.m2 ? mc - c2v.f : 0.f); U3 = dup(gc.m3 ? c3.f - mc : 0.f);
            } else {
                // alpha = g / den, beta = -alpha out
                const float a0 = c0.g * c0.sv.y, a1 = c1.g * c1.sv.y;
                const float a2 = c2v.g * c2v.sv.y, a3 = c3.g * c3.sv.y;
                U0 = dup(a0); U1 = dup(-a1); U2 = dup(-a2); U3 = dup(a3);
                V0 = dup(-a0 * c0.sv.z); V1 = dup(a1 * c1.sv.z);
                V2 = dup(a2 * c2v.sv.z); V3 = dup(-a3 * c3.sv.z);
                xc = cc.g * cc.sv.y * cc.sv.w;
            }
            const float2 FC = dup(pix_f(cc));

            // left neighbour's S of the previous step (column j of the other
            // buffer; column 0 is the zero carry-in of the first lane), and
            // this lane's slot (column j + 1)
            const float4* rd = smem + ((t + 1) & 1) * BUF + j;
            float4* wr = smem + (t & 1) * BUF + j + 1;
            float2 NUM = make_float2(0.f, 0.f), DEN = NUM, DNUM = NUM, DDEN = NUM;
            // the centre pixel's recombination of pair i with its box sums h
            auto combine = [&](const Strm& sc, int i, float2 hx, float2 hy, float2 hz,
                               float2 hw) {
                const float2 A2 = make_float2(p.a[CO + 2 * i], p.a[CO + 2 * i + 1]);
                const float2 AK2 = make_float2(p.ak[CO + 2 * i], p.ak[CO + 2 * i + 1]);
                // -S_k h: the negation on the centre's sines (one product per
                // pair) or on the box sums (folded into the products)
                const float2 nzs = __fmul2_rn(sc.s, dup(-1.f));
                auto msh = [&](float2 h) {
                    if constexpr (NEGFOLD) return __fmul2_rn(sc.s, make_float2(-h.x, -h.y));
                    else return __fmul2_rn(nzs, h);
                };
                auto hms = [&](float2 h) {  // the same, operands in the adjoint's order
                    if constexpr (NEGFOLD) return __fmul2_rn(make_float2(-h.x, -h.y), sc.s);
                    else return __fmul2_rn(h, nzs);
                };
                if constexpr (!BWD) {
                    NUM = __ffma2_rn(A2, __ffma2_rn(sc.c, hx, __fmul2_rn(sc.s, hy)), NUM);
                    DEN = __ffma2_rn(A2, __ffma2_rn(sc.c, hz, __fmul2_rn(sc.s, hw)), DEN);
                    if constexpr (SAVE) {
                        DNUM = __ffma2_rn(AK2, __ffma2_rn(sc.c, hy, msh(hx)), DNUM);
                        DDEN = __ffma2_rn(AK2, __ffma2_rn(sc.c, hw, msh(hz)), DDEN);
                    }
                } else {
                    // h = (Box[alpha C], Box[alpha S], Box[beta C], Box[beta S])
                    NUM = __ffma2_rn(A2, __ffma2_rn(hx, sc.c, __fmul2_rn(hy, sc.s)), NUM);
                    const float2 pp = __ffma2_rn(hy, sc.c, hms(hx));
                    const float2 qq = __ffma2_rn(hw, sc.c, hms(hz));
                    DEN = __ffma2_rn(AK2, __ffma2_rn(FC, pp, qq), DEN);
                }
            };
            // the same for the one harmonic of the half pair (first components)
            auto combine1 = [&](const Strm& sc, int i, float hx, float hy, float hz, float hw) {
                const float a = p.a[CO + 2 * i], ak = p.ak[CO + 2 * i];
                const float c = sc.c.x, sn = sc.s.x;
                if constexpr (!BWD) {
                    NUM.x = fmaf(a, fmaf(c, hx, sn * hy), NUM.x);
                    DEN.x = fmaf(a, fmaf(c, hz, sn * hw), DEN.x);
                    if constexpr (SAVE) {
                        DNUM.x = fmaf(ak, fmaf(c, hy, -sn * hx), DNUM.x);
                        DDEN.x = fmaf(ak, fmaf(c, hw, -sn * hz), DDEN.x);
                    }
                } else {
                    NUM.x = fmaf(a, fmaf(hx, c, hy * sn), NUM.x);
                    const float pp = fmaf(hy, c, -hx * sn);
                    const float qq = fmaf(hw, c, -hz * sn);
                    DEN.x = fmaf(ak, fmaf(FC.x, pp, qq), DEN.x);
                }
            };
            if constexpr (!KAHAN && BODY != 1) {
                // the vertical running sums one stream at a time (only that
                // stream's recurrence is live, and its harmonic pairs update
                // independent sums), then the horizontal step and the centre
                auto accumulate = [&](float f, float2 U, float2 V) {
                    if constexpr (DC) {
                        Dfa += U.x;
                        if constexpr (!BWD) Dfz += V.x;
                    }
                    Strm q = seed<SEED>(f, p.gamma, p.k0);
#pragma unroll
                    for (int i = 0; i < KP; ++i) {
                        if (HALF && i == KP - 1) {
                            Dx[i].x = fmaf(q.c.x, U.x, Dx[i].x);
                            Dy[i].x = fmaf(q.s.x, U.x, Dy[i].x);
                            Dz[i].x = fmaf(q.c.x, V.x, Dz[i].x);
                            Dw[i].x = fmaf(q.s.x, V.x, Dw[i].x);
                        } else {
                            Dx[i] = __ffma2_rn(q.c, U, Dx[i]);
                            Dy[i] = __ffma2_rn(q.s, U, Dy[i]);
                            Dz[i] = __ffma2_rn(q.c, V, Dz[i]);
                            Dw[i] = __ffma2_rn(q.s, V, Dw[i]);
                        }
                        if (i + 1 < KP) advance(q, i, i + 2 < KP, HALF && i + 2 == KP - 1);
                    }
                };
                accumulate(pix_f(c0), U0, V0);
                accumulate(pix_f(c1), U1, V1);
                accumulate(pix_f(c2v), U2, V2);
                accumulate(pix_f(c3), U3, V3);
                Strm sc = seed<SEED>(pix_f(cc), p.gamma, p.k0);
                if constexpr (DC) {
                    // box sums of the constant harmonic: C_0 = 1, S_0 = 0
                    const float4 A = rd[(2 * KP) * LD];
                    const float hf = A.x + Dfa;
                    const float h1 = BWD ? 0.f : A.z + Dfz;
                    wr[(2 * KP) * LD] = make_float4(hf, 0.f, h1, 0.f);
                    NUM.x = fmaf(p.a[0], hf, NUM.x);
                    if constexpr (!BWD) DEN.x = fmaf(p.a[0], h1, DEN.x);
                }
                // BODY 2 / 3: the left neighbour's sums of pair i + PF are loaded
                // before this lane stores pair i (the two step-parity buffers
                // never overlap), so the loads stay in flight across the stores
                constexpr int PF = BODY == 2 ? 2 : (BODY == 3 ? 1 : 0);
                float4 PA[KP], PB[KP];
#pragma unroll
                for (int i = 0; i < PF && i < KP; ++i) {
                    PA[i] = rd[(2 * i) * LD];
                    if (!(HALF && i == KP - 1)) PB[i] = rd[(2 * i + 1) * LD];
                }
#pragma unroll
                for (int i = 0; i < KP; ++i) {
                    if (PF > 0 && i + PF < KP) {
                        PA[i + PF] = rd[(2 * (i + PF)) * LD];
                        if (!(HALF && i + PF == KP - 1)) PB[i + PF] = rd[(2 * (i + PF) + 1) * LD];
                    }
                    if (HALF && i == KP - 1) {
                        // one float4 per lane: (P, Q, U, V) of the single harmonic
                        const float4 A = PF > 0 ? PA[i] : rd[(2 * i) * LD];
                        const float hx = A.x + Dx[i].x, hy = A.y + Dy[i].x;
                        const float hz = A.z + Dz[i].x, hw = A.w + Dw[i].x;
                        wr[(2 * i) * LD] = make_float4(hx, hy, hz, hw);
                        combine1(sc, i, hx, hy, hz, hw);
                    } else {
                        const float4 A = PF > 0 ? PA[i] : rd[(2 * i) * LD];
                        const float4 B = PF > 0 ? PB[i] : rd[(2 * i + 1) * LD];
                        const float2 hx = __fadd2_rn(make_float2(A.x, A.y), Dx[i]);
                        const float2 hy = __fadd2_rn(make_float2(A.z, A.w), Dy[i]);
                        const float2 hz = __fadd2_rn(make_float2(B.x, B.y), Dz[i]);
                        const float2 hw = __fadd2_rn(make_float2(B.z, B.w), Dw[i]);
                        wr[(2 * i) * LD] = make_float4(hx.x, hx.y, hy.x, hy.y);
                        wr[(2 * i + 1) * LD] = make_float4(hz.x, hz.y, hw.x, hw.y);
                        combine(sc, i, hx, hy, hz, hw);
                    }
                    if (i + 1 < KP) advance(sc, i, i + 2 < KP, HALF && i + 2 == KP - 1);
                }
            } else if constexpr (BODY == 1) {
                // all five streams advance together, pair by pair: the four
                // streams' updates of pair i sit between the load of the left
                // neighbour's sums of pair i and their use
                Strm s0 = seed<SEED>(pix_f(c0), p.gamma, p.k0);
                Strm s1 = seed<SEED>(pix_f(c1), p.gamma, p.k0);
                Strm s2 = seed<SEED>(pix_f(c2v), p.gamma, p.k0);
                Strm s3 = seed<SEED>(pix_f(c3), p.gamma, p.k0);
                Strm sc = seed<SEED>(pix_f(cc), p.gamma, p.k0);
                if constexpr (DC) {
                    const float4 A = rd[(2 * KP) * LD];
                    // the same order of adds as the sequential form
                    Dfa += U0.x; Dfa += U1.x; Dfa += U2.x; Dfa += U3.x;
                    const float hf = A.x + Dfa;
                    float h1 = 0.f;
                    if constexpr (!BWD) {
                        Dfz += V0.x; Dfz += V1.x; Dfz += V2.x; Dfz += V3.x;
                        h1 = A.z + Dfz;
                    }
                    wr[(2 * KP) * LD] = make_float4(hf, 0.f, h1, 0.f);
                    NUM.x = fmaf(p.a[0], hf, NUM.x);
                    if constexpr (!BWD) DEN.x = fmaf(p.a[0], h1, DEN.x);
                }
#pragma unroll
                for (int i = 0; i < KP; ++i) {
                    if (HALF && i == KP - 1) {
                        const float4 A = rd[(2 * i) * LD];
                        float dx = Dx[i].x, dy = Dy[i].x, dz = Dz[i].x, dw = Dw[i].x;
                        dx = fmaf(s0.c.x, U0.x, dx); dx = fmaf(s1.c.x, U1.x, dx);
                        dx = fmaf(s2.c.x, U2.x, dx); dx = fmaf(s3.c.x, U3.x, dx);
                        dy = fmaf(s0.s.x, U0.x, dy); dy = fmaf(s1.s.x, U1.x, dy);
                        dy = fmaf(s2.s.x, U2.x, dy); dy = fmaf(s3.s.x, U3.x, dy);
                        dz = fmaf(s0.c.x, V0.x, dz); dz = fmaf(s1.c.x, V1.x, dz);
                        dz = fmaf(s2.c.x, V2.x, dz); dz = fmaf(s3.c.x, V3.x, dz);
                        dw = fmaf(s0.s.x, V0.x, dw); dw = fmaf(s1.s.x, V1.x, dw);
                        dw = fmaf(s2.s.x, V2.x, dw); dw = fmaf(s3.s.x, V3.x, dw);
                        Dx[i].x = dx; Dy[i].x = dy; Dz[i].x = dz; Dw[i].x = dw;
                        const float hx = A.x + dx, hy = A.y + dy, hz = A.z + dz, hw = A.w + dw;
                        wr[(2 * i) * LD] = make_float4(hx, hy, hz, hw);
                        combine1(sc, i, hx, hy, hz, hw);
                    } else {
                        const float4 A = rd[(2 * i) * LD];
                        const float4 B = rd[(2 * i + 1) * LD];
                        float2 dx = Dx[i], dy = Dy[i], dz = Dz[i], dw = Dw[i];
                        dx = __ffma2_rn(s0.c, U0, dx); dx = __ffma2_rn(s1.c, U1, dx);
                        dx = __ffma2_rn(s2.c, U2, dx); dx = __ffma2_rn(s3.c, U3, dx);
                        dy = __ffma2_rn(s0.s, U0, dy); dy = __ffma2_rn(s1.s, U1, dy);
                        dy = __ffma2_rn(s2.s, U2, dy); dy = __ffma2_rn(s3.s, U3, dy);
                        dz = __ffma2_rn(s0.c, V0, dz); dz = __ffma2_rn(s1.c, V1, dz);
                        dz = __ffma2_rn(s2.c, V2, dz); dz = __ffma2_rn(s3.c, V3, dz);
                        dw = __ffma2_rn(s0.s, V0, dw); dw = __ffma2_rn(s1.s, V1, dw);
                        dw = __ffma2_rn(s2.s, V2, dw); dw = __ffma2_rn(s3.s, V3, dw);
                        Dx[i] = dx; Dy[i] = dy; Dz[i] = dz; Dw[i] = dw;
                        const float2 hx = __fadd2_rn(make_float2(A.x, A.y), dx);
                        const float2 hy = __fadd2_rn(make_float2(A.z, A.w), dy);
                        const float2 hz = __fadd2_rn(make_float2(B.x, B.y), dz);
                        const float2 hw = __fadd2_rn(make_float2(B.z, B.w), dw);
                        wr[(2 * i) * LD] = make_float4(hx.x, hx.y, hy.x, hy.y);
                        wr[(2 * i + 1) * LD] = make_float4(hz.x, hz.y, hw.x, hw.y);
                        combine(sc, i, hx, hy, hz, hw);
                    }
                    if (i + 1 < KP) {
                        const bool need = i + 2 < KP, hn = HALF && i + 2 == KP - 1;
                        advance(s0, i, need, hn); advance(s1, i, need, hn);
                        advance(s2, i, need, hn); advance(s3, i, need, hn);
                        advance(sc, i, need, hn);
                    }
                }
            } else {
                // Kahan (forward): every stream's planes are added to the running
                // sums one by one with compensation (Kahan 1965: y = p - e,
                // t = D + y, e = (t - D) - y, D = t). A pixel enters and, 2r+1
                // rows later, leaves a lane's sums with bit-identical products
                // (same stream code, no fused multiply-add into the sum), so
                // with the adds compensated its two contributions cancel and
                // the sums do not drift down a tall band; summing the four
                // streams first (one rounding per step) would not cancel.
                static_assert(!HALF && !BWD && !DC,
                              "the Kahan form runs whole pairs from k0, forward only");
                Strm s0 = seed<SEED>(pix_f(c0), p.gamma, p.k0);
                Strm s1 = seed<SEED>(pix_f(c1), p.gamma, p.k0);
                Strm s2 = seed<SEED>(pix_f(c2v), p.gamma, p.k0);
                Strm s3 = seed<SEED>(pix_f(c3), p.gamma, p.k0);
                Strm sc = seed<SEED>(pix_f(cc), p.gamma, p.k0);
                const float2 m1 = dup(-1.f);
                auto kadd = [&](float2& D, float2& E, float2 v) {
                    const float2 y = __ffma2_rn(E, m1, v);
                    const float2 t2 = __fadd2_rn(D, y);
                    E = __ffma2_rn(y, m1, __ffma2_rn(D, m1, t2));
                    D = t2;
                };
#pragma unroll
                for (int i = 0; i < KP; ++i) {
                    const float4 A = rd[(2 * i) * LD];
                    const float4 B = rd[(2 * i + 1) * LD];
                    auto add_stream = [&](const Strm& q, float2 U, float2 V) {
                        kadd(Dx[i], Ex[i], __fmul2_rn(q.c, U));
                        kadd(Dy[i], Ey[i], __fmul2_rn(q.s, U));
                        kadd(Dz[i], Ez[i], __fmul2_rn(q.c, V));
                        kadd(Dw[i], Ew[i], __fmul2_rn(q.s, V));
                    };
                    add_stream(s0, U0, V0);
                    add_stream(s1, U1, V1);
                    add_stream(s2, U2, V2);
                    add_stream(s3, U3, V3);
                    const float2 hx = __fadd2_rn(make_float2(A.x, A.y), Dx[i]);
                    const float2 hy = __fadd2_rn(make_float2(A.z, A.w), Dy[i]);
                    const float2 hz = __fadd2_rn(make_float2(B.x, B.y), Dz[i]);
                    const float2 hw = __fadd2_rn(make_float2(B.z, B.w), Dw[i]);
                    wr[(2 * i) * LD] = make_float4(hx.x, hx.y, hy.x, hy.y);
                    wr[(2 * i + 1) * LD] = make_float4(hz.x, hz.y, hw.x, hw.y);
                    combine(sc, i, hx, hy, hz, hw);
                    if (i + 1 < KP) {
                        const bool need = i + 2 < KP;
                        advance(s0, i, need); advance(s1, i, need); advance(s2, i, need);
                        advance(s3, i, need); advance(sc, i, need);
                    }
                }
            }
            if (gc.out) {
                // compact buffers (saved quads, chunk accumulators; sheared
                // rows) and row-pitched ones (out, den, dL/dimg)
                const size_t o = (size_t)quad_at(e0 + t - r, co) + zo;
                const size_t op = (size_t)gc.qo + zp;
                float num = NUM.x + NUM.y, den = DEN.x + DEN.y;
                // chunked harmonics: partial sums live in the output buffers
                // between chunks (acc: 0 single, 1 first, 2 middle, 3 last)
                const int acc = p.acc;
                const bool last = acc == 0 || acc == 3;
                if constexpr (!BWD) {
                    float dn = DNUM.x + DNUM.y, dd = DDEN.x + DDEN.y;
                    if constexpr (SAVE) {
                        // between chunks the quad holds the partial (., den,
                        // dnum, dden); the last chunk leaves (f, 1/den, out,
                        // dnum - out dden) for the adjoint
                        if (acc >= 2) {
                            const float4 q = p.sv[o];
                            num += p.out[op]; den += q.y; dn += q.z; dd += q.w;
                        }
                        if (last) {
                            const float qv = num / den;   // out - mid
                            p.out[op] = qv + p.mid;
                            p.sv[o] = make_float4(cc.f - p.mid, 1.0f / den, qv, fmaf(-qv, dd, dn));
                            if constexpr (PITCH) {
                                if (p.dout) p.dout[op] = den;
                            }
                        } else {
                            p.out[op] = num;
                            p.sv[o] = make_float4(cc.f, den, dn, dd);
                        }
                    } else {
                        if (acc >= 2) { num += p.out[op]; den += p.acc_den[o]; }
                        p.out[op] = last ? num / den + p.mid : num;
                        if (acc != 0) p.acc_den[o] = den;
                        if constexpr (PITCH) {
                            if (last && p.dout) p.dout[op] = den;
                        }
                    }
                } else {
                    if (acc >= 2) { num += p.acc_gv[o]; den += p.acc_gt[o]; }
                    if (last) {
                        const float gt = den + xc;
                        if (p.gimg) p.gimg[op] = num + p.gamma * gt;
                        gsum = fmaf(cc.sv.x, gt, gsum);
                    } else {
                        p.acc_gv[o] = num;
                        p.acc_gt[o] = den;
                    }
                }
            }
        }
        __syncthreads();
    };
    if constexpr (PINGPONG) {
        int t = 0;
        for (; t + 1 < steps; t += 2) {
            step(t, gA, vA, gB, vB);
            step(t + 1, gB, vB, gA, vA);
        }
        if (t < steps) step(t, gA, vA, gB, vB);
    } else {
        for (int t = 0; t < steps; ++t) step(t, gA, vA, gA, vA);
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
template <int KP, bool BWD, bool SAVE, bool KAHAN, int WMAX, typename Tin, bool HALF = false,
          int SEED = 0, int FORM = 0, bool PITCH = true>
__global__ void __launch_bounds__(WMAX, 256 / WMAX) bf_sys_kernel(SysParams p) {
    extern __shared__ float4 smem[];
    float gsum = 0.f;
    const size_t z = blockIdx.z;  // image of a [B, H, W] launch
    const size_t hw = (size_t)p.H * p.W;
    const size_t hp = PITCH ? (size_t)p.H * p.ld : hw;
    sysd::sys_tile<KP, BWD, SAVE, KAHAN, WMAX, Tin, HALF, SEED, FORM, PITCH>(
        p, blockIdx.x, blockIdx.y, z * hw, z * hp, smem, gsum);
    if (BWD && p.partial)
        sysd::cta_sum_to(gsum, p.partial, (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
}

template <int KP, bool BWD, bool SAVE, bool KAHAN, int WMAX, typename Tin, bool HALF = false,
          int SEED = 0, int FORM = 0, bool PITCH = true>
cudaError_t sys_launch_one(const SysParams& p, int wi, int gx, int gy, cudaStream_t s) {
    const int gz = p.B > 0 ? p.B : 1;
    auto kern = bf_sys_kernel<KP, BWD, SAVE, KAHAN, WMAX, Tin, HALF, SEED, FORM, PITCH>;
    const size_t smem = sizeof(float4) * (size_t)sysd::sys_smem_slots(KP, WMAX, SEED == 2);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(gx, gy, gz), wi, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace bf
