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
// e^{i a gs (2r+1)} = (-1)^a = (-1)^M. Thread j keeps vertical running sums
// over its own column minus (-1)^M times those of the column 2r + 1 to the
// left; horizontal sums pass one lane per step through a shared row
// double-buffered by step parity, one CTA barrier per step. Two forms:
//   combo-sum (spk_kernel): per combo c, the column-rotated difference
//     D'_c += e^{i a gs cw} e^{i b gs e} Z_k, Z_k the four streams' weighted
//     range harmonics, and S_c(j) = S_c(j - 1) + D'_c(j);
//   plane-sum (spk_plane_kernel): per (b, k) plane the difference D_{b,k} of
//     e^{i b gs z2} e^{i k gamma f} (times f, and not), rotated in the
//     hand-off, S(j) = S(j - 1) + e^{i a gs cw(j)} D_{b,k}(j);
// the first where the combos are few against the planes (every N > 0), the
// second where many combos share a plane (no range kernel, M >= 2).
#include <math.h>
#include <string.h>

#include "bf_internal.cuh"
#include "bf_launch.cuh"
#include "bf_trace.cuh"

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

// Largest combo count any instantiation has, and caps of the factor tables.
constexpr int NS_CAP = 64;
constexpr int FCAP = 8;

// coef_c factors as fa[a] fb[|b|] fk[|k|] (halved for the one self-conjugate
// combo a = b = k = 0): fa = beta_a (x2 for a = 0: one of each conjugate pair
// is kept), fb = beta_|b| m_b / 4, fk = alpha_|k| m_k, with m = 2 for a zero
// index (both sign choices of cos(A +- B +- C) give the same term). Indices
// are half-indices: a = (M mod 2) + 2 ia, |b| = (M mod 2) + 2 ib, |k| = (N
// mod 2) + 2 kk.
struct Params {
    const float* img;      // forward input (forward modes)
    float* out;            // forward output
    float4* sv;            // forward with saved quads: (f, 1/den, out, dnum_s - out dden_s)
    const float4* bsv;     // adjoint: the forward's saved quads
    const float* gout;     // adjoint: dL/dout
    float* gimg;           // adjoint: dL/dimg
    int H, W, r, Hb, Tw;
    float gamma;           // range kernel frequency (unused when N = 0)
    float fa[FCAP], fb[FCAP], fk[FCAP];
    float coef[NS_CAP];    // plane-sum form: coef_c, in combo order
    float ck[NS_CAP];      // plane-sum form: coef_c k_c (k_c: the combo's signed k)
};

// Launch modes: forward, forward that also saves the adjoint's quads, adjoint.
enum Mode { FWD = 0, FWD_SAVE = 1, ADJ = 2 };

__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// A complex number z as the register pairs used by the paired FP32 units:
// v = (Re z, Im z) and iv = i z = (-Im z, Re z), so that w z = w.x v + w.y iv
// for any complex w.
struct Cx {
    float2 v, iv;
};

// (c z) for a complex constant c given as dup(c.x), dup(c.y), dup(-c.y).
__device__ __forceinline__ Cx crot(float2 cx, float2 cy, float2 cyn, const Cx& z) {
    Cx o;
    o.v = __ffma2_rn(cy, z.iv, __fmul2_rn(cx, z.v));
    o.iv = __ffma2_rn(cyn, z.v, __fmul2_rn(cx, z.iv));
    return o;
}

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

// Non-negative range harmonics z_kk = e^{i k theta}, k = (N mod 2) + 2 kk,
// theta = gamma f, from one sine and cosine of theta and complex products.
template <int N>
__device__ __forceinline__ void range_harmonics(float f, float gamma, float2 (&z)[N / 2 + 1]) {
    if constexpr (N == 0) {
        z[0] = make_float2(1.f, 0.f);
    } else {
        float s1, c1;
        __sincosf(gamma * f, &s1, &c1);
        const float2 w1 = make_float2(c1, s1);
        const float2 w2 = cmul(w1, w1);
        z[0] = (N & 1) ? w1 : make_float2(1.f, 0.f);
#pragma unroll
        for (int i = 1; i <= N / 2; ++i) z[i] = cmul(z[i - 1], w2);
    }
}

// Longest phase table: 2 (2r + 1) entries for r <= 56, two float4 each.
constexpr int PTAB_CAP = 2 * (2 * 56 + 1);

__device__ __forceinline__ void prefetch_l2(const void* ptr) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}

// MODE = ADJ runs the same moving sums on the planes (alpha E_c, beta E_c),
// alpha = g / den, beta = -alpha out (the window and the spatial kernel are
// symmetric, so the adjoint's neighbour sums are again moving sums centred
// on the pixel whose gradient is formed), and combines them into
//   dL/df(p) = sum_c coef_c Re(conj E_c(p) A_c)
//            + gamma [sum_c coef_c k_c Im(conj E_c(p) (f(p) A_c + B_c)) + alpha(p) X(p)],
// A_c = Sum(alpha E_c), B_c = Sum(beta E_c), X = dnum_s - out dden_s saved by the
// forward (dnum_s = sum_c coef_c k_c Im(conj E_c S_c(f E)), the derivative of
// num through the centre value, divided by gamma).
//
// Per step and thread: the four entering / leaving pixels' range harmonics,
// weighted and summed into Z_k (real weights, so Z_{-k} = conj Z_k); then per
// combo the column-rotated vertical difference D'_c += e^{i a gs cw} e^{i b gs
// e} Z_k, the horizontal hand-off S_c = S_c(left) + D'_c, and the centre's
// coef_c conj(E_c) S_c, all on (re, im) register pairs.
//
// The adjoint is linear in the combo sums, so it may run as launches over
// consecutive combo ranges [C0, C1) (fewer live sums per launch); a launch
// with C0 > 0 adds its part to dL/df.
template <int M, int N, int MODE, int C0 = 0, int C1 = Dims<M, N>::NS>
__global__ void __launch_bounds__(WMAX, 2) spk_kernel(Params p) {
    using D = Dims<M, N>;
    static_assert(0 <= C0 && C0 < C1 && C1 <= D::NS, "combo range");
    static_assert(MODE == ADJ || (C0 == 0 && C1 == D::NS), "forward runs all combos");
    constexpr int NA = D::NA, NB = D::NB, NK = D::NK;
    constexpr int KH = N / 2 + 1;        // non-negative range harmonics
    constexpr int BH = M / 2 + 1;        // non-negative spatial harmonics |b|
    constexpr int LD = WMAX + 1;
    constexpr int BUF = (C1 - C0) * LD;
    extern __shared__ float4 smem[];  // [2][NS][LD]: (g.re, g.im, h.re, h.im), then the table
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
    // -(-1)^M: weight of the second column; (-1)^M: the leaving row's phase
    // relative to the entering row's, e^{-i b gs (2r+1)} for every b of M's parity
    const float sgn2 = (M & 1) ? 1.f : -1.f;
    const float lsg = (M & 1) ? -1.f : 1.f;

    for (int i = j; i < 2 * BUF; i += Wi) smem[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int P = 2 * (2 * r + 1);  // period of e^{i gs n} in n
    // tab[2q] = (z, i z), tab[2q + 1] = (conj z, i conj z) for z = e^{i pi q / (2r+1)}
    float4* ptab = smem + 2 * BUF;
    for (int q = j; q < P; q += Wi) {
        float s, c;
        sincospif((float)q / (float)(2 * r + 1), &s, &c);
        ptab[2 * q] = make_float4(c, s, -s, c);
        ptab[2 * q + 1] = make_float4(c, -s, s, c);
    }
    // phase indices b e mod P of the entering row e (b > 0, advanced by b per
    // step) and their offsets b r to the centre row rho = e - r
    int qe[BH], qoff[BH];
#pragma unroll
    for (int hb = 0; hb < BH; ++hb) {
        const int b = (M & 1) + 2 * hb;
        int q0 = (int)(((long long)b * (long long)(y0 - r - j)) % P);
        if (q0 < 0) q0 += P;
        qe[hb] = q0;
        qoff[hb] = (b * r) % P;
    }

    // column phases: e^{i a gs cw} of the own column, and coef's a-factor times
    // e^{i a gs co} of the centre column, as dup pairs (x, y, -y)
    float2 cx[NA], cy[NA], cyn[NA], ox[NA], oy[NA], oyn[NA];
#pragma unroll
    for (int ia = 0; ia < NA; ++ia) {
        const int a = (M & 1) + 2 * ia;
        const float2 c = phase(a, cw, r);
        const float2 o = phase(a, co, r);
        const float fa = p.fa[ia];
        cx[ia] = dup(c.x); cy[ia] = dup(c.y); cyn[ia] = dup(-c.y);
        ox[ia] = dup(fa * o.x); oy[ia] = dup(fa * o.y); oyn[ia] = dup(-fa * o.y);
    }
    float fbv[BH], fkv[KH];
#pragma unroll
    for (int hb = 0; hb < BH; ++hb) fbv[hb] = p.fb[hb];
#pragma unroll
    for (int kk = 0; kk < KH; ++kk) fkv[kk] = p.fk[kk];

    // column-rotated vertical differences of the kept combos: (f-weighted,
    // unweighted) in the forward, (alpha, beta)-weighted in the adjoint
    float2 Dg[D::NS], Dh[D::NS];
#pragma unroll
    for (int c = 0; c < D::NS; ++c) { Dg[c] = make_float2(0.f, 0.f); Dh[c] = Dg[c]; }
    // the five pixels of step tt (own / second column, entering / leaving row,
    // centre), 0 where masked; the adjoint reads the saved quad (whose .x
    // is f) and dL/dout instead
    float4 nq[5];
    float ng[5];
    float npart = 0.f;  // adjoint over a later combo range: the earlier ranges' dL/df
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
        if constexpr (MODE == ADJ && C0 > 0) npart = out ? p.gimg[(size_t)rho * W + co] : 0.f;
    };
    load_step(w * 32);  // a warp is first active at step 32 w
    __syncthreads();

    for (int t = 0; t < steps; ++t, [&] {
#pragma unroll
             for (int hb = 0; hb < BH; ++hb) {
                 // P >= 6 (r >= 1): one wrap, two when b = 8 > P
                 qe[hb] += (M & 1) + 2 * hb;
                 if (qe[hb] >= P) qe[hb] -= P;
                 if constexpr (M > 6) {
                     if (qe[hb] >= P) qe[hb] -= P;
                 }
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
            // the loads of the next one so their latency hides under this step,
            // and pull a later entering row into L2
            float4 q[5];
            float gq[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) { q[k] = nq[k]; gq[k] = MODE == ADJ ? ng[k] : 0.f; }
            const float part = npart;
            const float fc = q[4].x;
            load_step(t + 1);
            {
                const int ef = e + 8;
                if (own_in && ef >= 0 && ef < p.H) {
                    if constexpr (MODE == ADJ) {
                        prefetch_l2(p.bsv + quad_index(ef, cw, p.H, W));
                        prefetch_l2(p.gout + (size_t)ef * W + cw);
                    } else {
                        prefetch_l2(p.img + (size_t)ef * W + cw);
                    }
                }
            }

            // Z_k = sum_s u_s z_s(k) over the four streams with signs + own
            // enter, -(-1)^M second enter, -(-1)^M own leave, + second leave
            // (the leaving row's phase folded in): (u_g, u_h) = (f, 1) in the
            // forward, (alpha, beta) in the adjoint
            float zgx[KH], zgy[KH], zhx[KH], zhy[KH];
#pragma unroll
            for (int kk = 0; kk < KH; ++kk) { zgx[kk] = 0.f; zgy[kk] = 0.f; zhx[kk] = 0.f; zhy[kk] = 0.f; }
            const float wsg[4] = {m0 ? 1.f : 0.f, m1 ? sgn2 : 0.f, m2 ? -lsg : 0.f,
                                  m3 ? -sgn2 * lsg : 0.f};
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                float ug, uh;
                if constexpr (MODE == ADJ) {
                    const float al = gq[s] * q[s].y;
                    ug = wsg[s] * al;
                    uh = -ug * q[s].z;
                } else {
                    ug = wsg[s] * q[s].x;
                    uh = wsg[s];
                }
                float2 z[KH];
                range_harmonics<N>(q[s].x, p.gamma, z);
#pragma unroll
                for (int kk = 0; kk < KH; ++kk) {
                    zgx[kk] = fmaf(ug, z[kk].x, zgx[kk]);
                    zgy[kk] = fmaf(ug, z[kk].y, zgy[kk]);
                    zhx[kk] = fmaf(uh, z[kk].x, zhx[kk]);
                    zhy[kk] = fmaf(uh, z[kk].y, zhy[kk]);
                }
            }
            // centre: f-side factors fk |k| z_c(k)
            float2 zc[KH];
            range_harmonics<N>(fc, p.gamma, zc);
#pragma unroll
            for (int kk = 0; kk < KH; ++kk) zc[kk] = make_float2(fkv[kk] * zc[kk].x, fkv[kk] * zc[kk].y);

            // row phases of the entering row (vertical) and, times coef's
            // b-factor, of the centre row (recombination), for signed b
            Cx rp[NB], rc[NB];
#pragma unroll
            for (int hb = 0; hb < BH; ++hb) {
                const int b = (M & 1) + 2 * hb;
                const int ipos = (b + M) / 2, ineg = (M - b) / 2;
                int qc = qe[hb] - qoff[hb];
                if (qc < 0) qc += P;
                const float2 sb = dup(fbv[hb]);
                if (b == 0) {
                    rp[ipos].v = make_float2(1.f, 0.f);
                    rp[ipos].iv = make_float2(0.f, 1.f);
                    rc[ipos].v = make_float2(fbv[hb], 0.f);
                    rc[ipos].iv = make_float2(0.f, fbv[hb]);
                } else {
                    // (z, i z) = (c, s, -s, c); conj z = (c, -s) and i conj z = (s, c)
                    // are the same four values rearranged, so one load serves both
                    // signs of b. The adjoint's later combo range reads the stored
                    // conjugate entry instead: with the rearranged form its registers
                    // fall to 166 and the compiler then issues the next step's pixel
                    // loads late (1.03 against 0.81 ms at M=2, N=4, 4096^2).
                    const float4 t1 = ptab[2 * qe[hb]];
                    const float4 u1 = ptab[2 * qc];
                    rp[ipos].v = make_float2(t1.x, t1.y); rp[ipos].iv = make_float2(t1.z, t1.w);
                    rc[ipos].v = __fmul2_rn(sb, make_float2(u1.x, u1.y));
                    rc[ipos].iv = __fmul2_rn(sb, make_float2(u1.z, u1.w));
                    if constexpr (MODE == ADJ && C0 > 0) {
                        const float4 t2 = ptab[2 * qe[hb] + 1], u2 = ptab[2 * qc + 1];
                        rp[ineg].v = make_float2(t2.x, t2.y);
                        rp[ineg].iv = make_float2(t2.z, t2.w);
                        rc[ineg].v = __fmul2_rn(sb, make_float2(u2.x, u2.y));
                        rc[ineg].iv = __fmul2_rn(sb, make_float2(u2.z, u2.w));
                    } else {
                        rp[ineg].v = make_float2(t1.x, t1.z);
                        rp[ineg].iv = make_float2(t1.y, t1.x);
                        rc[ineg].v = __fmul2_rn(sb, make_float2(u1.x, u1.z));
                        rc[ineg].iv = __fmul2_rn(sb, make_float2(u1.y, u1.x));
                    }
                }
            }

            const float4* rd = smem + ((t + 1) & 1) * BUF + j;
            float4* wr = smem + (t & 1) * BUF + j + 1;
            float2 NUM = make_float2(0.f, 0.f), DEN = NUM, DN = NUM, DD = NUM;
            const float2 FC = dup(fc);
            int cn = 0;  // combo index
#pragma unroll
            for (int ia = 0; ia < NA; ++ia) {
                const int a = (M & 1) + 2 * ia;
#pragma unroll
                for (int ib = 0; ib < NB; ++ib) {
                    // R = e^{i a gs cw} e^{i b gs e}, Q = coef's (a, b) factors times
                    // e^{i a gs co} e^{i b gs rho}
                    Cx R, Q;
                    if (a == 0) {
                        R = rp[ib];
                        Q.v = __fmul2_rn(ox[ia], rc[ib].v);
                        Q.iv = __fmul2_rn(ox[ia], rc[ib].iv);
                    } else {
                        R = crot(cx[ia], cy[ia], cyn[ia], rp[ib]);
                        Q = crot(ox[ia], oy[ia], oyn[ia], rc[ib]);
                    }
#pragma unroll
                    for (int ik = 0; ik < NK; ++ik) {
                        const int d = ib * NK + ik;
                        if (a == 0 && d < D::D0) continue;
                        const int c = cn++;
                        if (c < C0 || c >= C1) continue;
                        const int b = -M + 2 * ib;
                        const int k = -N + 2 * ik;
                        const int kk = (k < 0 ? -k : k) / 2;
                        const bool neg = k < 0;
                        // vertical: D'_c += R Z_k (Z_{-k} = conj Z_k)
                        if (k == 0) {
                            Dg[c] = __ffma2_rn(dup(zgx[kk]), R.v, Dg[c]);
                            Dh[c] = __ffma2_rn(dup(zhx[kk]), R.v, Dh[c]);
                        } else {
                            Dg[c] = __ffma2_rn(dup(neg ? -zgy[kk] : zgy[kk]), R.iv,
                                               __ffma2_rn(dup(zgx[kk]), R.v, Dg[c]));
                            Dh[c] = __ffma2_rn(dup(neg ? -zhy[kk] : zhy[kk]), R.iv,
                                               __ffma2_rn(dup(zhx[kk]), R.v, Dh[c]));
                        }
                        // horizontal hand-off
                        const float4 A = rd[(c - C0) * LD];
                        const float2 hg = __fadd2_rn(make_float2(A.x, A.y), Dg[c]);
                        const float2 hh = __fadd2_rn(make_float2(A.z, A.w), Dh[c]);
                        wr[(c - C0) * LD] = make_float4(hg.x, hg.y, hh.x, hh.y);
                        // E = coef_c E_c(centre) = Q zc_k (conj for k < 0)
                        float2 E;
                        if (k == 0) {
                            E = __fmul2_rn(dup(zc[kk].x), Q.v);
                            if (a == 0 && b == 0) E = __fmul2_rn(dup(0.5f), E);  // self-conjugate
                        } else {
                            E = __ffma2_rn(dup(neg ? -zc[kk].y : zc[kk].y), Q.iv,
                                           __fmul2_rn(dup(zc[kk].x), Q.v));
                        }
                        // Re(conj E h) = E . h; k Im(conj E h) = (-k E.y, k E.x) . h
                        NUM = __ffma2_rn(E, hg, NUM);
                        if constexpr (MODE != ADJ) {
                            DEN = __ffma2_rn(E, hh, DEN);
                            if constexpr (MODE == FWD_SAVE) {
                                if (k != 0) {
                                    const float2 Ek = make_float2(-(float)k * E.y, (float)k * E.x);
                                    DN = __ffma2_rn(Ek, hg, DN);
                                    DD = __ffma2_rn(Ek, hh, DD);
                                }
                            }
                        } else {
                            // hg = A_c = Sum(alpha E_c), hh = B_c = Sum(beta E_c)
                            if (k != 0) {
                                const float2 Ek = make_float2(-(float)k * E.y, (float)k * E.x);
                                DEN = __ffma2_rn(Ek, __ffma2_rn(FC, hg, hh), DEN);
                            }
                        }
                    }
                }
            }
            if (out) {
                const size_t o = (size_t)rho * W + co;
                const float num = NUM.x + NUM.y, den = DEN.x + DEN.y;
                if constexpr (MODE == ADJ) {
                    // centre quad: (f, 1/den, out, X)
                    if constexpr (C0 == 0) {
                        const float al = gq[4] * q[4].y;
                        p.gimg[o] = fmaf(p.gamma, fmaf(al, q[4].w, den), num);
                    } else {
                        p.gimg[o] = part + fmaf(p.gamma, den, num);
                    }
                } else {
                    const float ov = num / den;
                    p.out[o] = ov;
                    if constexpr (MODE == FWD_SAVE) {
                        const float dn = DN.x + DN.y, dd = DD.x + DD.y;
                        // streaming store: the adjoint reads the quads after the whole forward
                        __stcs(p.sv + quad_index(rho, co, p.H, W),
                               make_float4(fc, 1.0f / den, ov, fmaf(-ov, dd, dn)));
                    }
                }
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }

// Range harmonics z_k = e^{i k theta} for signed k = -N, ..., N (step 2), for
// the plane-sum kernel.
template <int N>
__device__ __forceinline__ void range_harmonics_signed(float f, float gamma, float2 (&z)[N + 1]) {
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

// Plane-sum form: the vertical differences are kept per (b, k) plane
// (e^{i b gs z2} e^{i k gamma f}, f-weighted and not) and rotated by each
// combo's column phase e^{i a gs cw} in the horizontal hand-off. Cheaper than
// the combo-sum form when many combos share a plane (no range kernel, M >= 2).
// MODE = ADJ runs the same moving sums on the planes (alpha E_c, beta E_c),
// alpha = g / den, beta = -alpha out (the window and the spatial kernel are
// symmetric, so the adjoint's neighbour sums are again moving sums centred
// on the pixel whose gradient is formed), and combines them into
//   dL/df(p) = sum_c coef_c Re(conj E_c(p) A_c)
//            + gamma [sum_c coef_c k_c Im(conj E_c(p) (f(p) A_c + B_c)) + alpha(p) X(p)],
// A_c = Sum(alpha E_c), B_c = Sum(beta E_c), X = dnum_s - out dden_s saved by the
// forward (dnum_s = sum_c coef_c k_c Im(conj E_c S_c(f E)), the derivative of
// num through the centre value, divided by gamma).
template <int M, int N, int MODE>
__global__ void __launch_bounds__(WMAX, 2) spk_plane_kernel(Params p) {
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
    // centre), 0 where masked; the adjoint reads the saved quad (whose .x
    // is f) and dL/dout instead
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

    for (int t = 0; t < steps; ++t, [&] {
#pragma unroll
             for (int ib = 0; ib <= M; ++ib) {
                 const int b = -M + 2 * ib;
                 if (b > 0) {
                     // P >= 6 (r >= 1): one wrap, two when b = 8 > P
                     qe[ib] += b;
                     if (qe[ib] >= P) qe[ib] -= P;
                     if constexpr (M > 6) {
                         if (qe[ib] >= P) qe[ib] -= P;
                     }
                 }
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
            float4 q[5];
            float gq[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) { q[k] = nq[k]; gq[k] = MODE == ADJ ? ng[k] : 0.f; }
            const float f0 = q[0].x, f1 = q[1].x, f2 = q[2].x, f3 = q[3].x, fc = q[4].x;
            load_step(t + 1);

            // vertical: entering row's phases; the leaving row's differ by
            // e^{-i b gs (2r+1)} = (-1)^M for every b of this parity
            float2 rp[M + 1];
            row_phases<M>(ptab, qe, rp);
            const float lsg = (M & 1) ? -1.f : 1.f;
            // plane weights: (f, 1) in the forward, (alpha, beta) in the adjoint
            auto accumulate = [&](int k, float wgt, float rsg) {
                float2 z[N + 1];
                range_harmonics_signed<N>(q[k].x, p.gamma, z);
                float ug, uh;
                if constexpr (MODE == ADJ) {
                    const float al = gq[k] * q[k].y;
                    ug = wgt * al;
                    uh = -wgt * al * q[k].z;
                } else {
                    ug = wgt * q[k].x;
                    uh = wgt;
                }
#pragma unroll
                for (int ib = 0; ib <= M; ++ib) {
                    const float2 rb = make_float2(rsg * rp[ib].x, rsg * rp[ib].y);
#pragma unroll
                    for (int ik = 0; ik <= N; ++ik) {
                        const float2 E = cmul(rb, z[ik]);
                        const int d = ib * (N + 1) + ik;
                        Dg[d].x = fmaf(ug, E.x, Dg[d].x);
                        Dg[d].y = fmaf(ug, E.y, Dg[d].y);
                        Dh[d].x = fmaf(uh, E.x, Dh[d].x);
                        Dh[d].y = fmaf(uh, E.y, Dh[d].y);
                    }
                }
            };
            // + own enter, -(-1)^M second enter, - own leave, +(-1)^M second leave
            if constexpr (N == 0) {
                // no range kernel: each stream's E is its row phase, so the four
                // streams reduce to one real weight per sum before the phases
                const float wsg[4] = {m0 ? 1.f : 0.f, m1 ? sgn2 : 0.f, m2 ? -lsg : 0.f,
                                      m3 ? -sgn2 * lsg : 0.f};
                float zg = 0.f, zh = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if constexpr (MODE == ADJ) {
                        const float al = wsg[k] * (gq[k] * q[k].y);
                        zg += al;
                        zh = fmaf(-al, q[k].z, zh);
                    } else {
                        zg = fmaf(wsg[k], q[k].x, zg);
                        zh += wsg[k];
                    }
                }
#pragma unroll
                for (int ib = 0; ib <= M; ++ib) {
                    Dg[ib].x = fmaf(zg, rp[ib].x, Dg[ib].x);
                    Dg[ib].y = fmaf(zg, rp[ib].y, Dg[ib].y);
                    Dh[ib].x = fmaf(zh, rp[ib].x, Dh[ib].x);
                    Dh[ib].y = fmaf(zh, rp[ib].y, Dh[ib].y);
                }
            } else {
                accumulate(0, m0 ? 1.f : 0.f, 1.f);
                accumulate(1, m1 ? sgn2 : 0.f, 1.f);
                accumulate(2, m2 ? -1.f : 0.f, lsg);
                accumulate(3, m3 ? -sgn2 : 0.f, lsg);
            }
            (void)f0; (void)f1; (void)f2; (void)f3;

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
            range_harmonics_signed<N>(fc, p.gamma, zc);
            const float4* rd = smem + ((t + 1) & 1) * BUF + j;
            float4* wr = smem + (t & 1) * BUF + j + 1;
            float num = 0.f, den = 0.f, dn = 0.f, dd = 0.f;
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
                    // Re(conj(E) h) = E.x h.x + E.y h.y, Im(conj(E) h) = E.x h.y - E.y h.x
                    if constexpr (MODE != ADJ) {
                        num = fmaf(p.coef[c], fmaf(E.x, hg.x, E.y * hg.y), num);
                        den = fmaf(p.coef[c], fmaf(E.x, hh.x, E.y * hh.y), den);
                        if constexpr (MODE == FWD_SAVE) {
                            dn = fmaf(p.ck[c], fmaf(E.x, hg.y, -E.y * hg.x), dn);
                            dd = fmaf(p.ck[c], fmaf(E.x, hh.y, -E.y * hh.x), dd);
                        }
                    } else {
                        // hg = A_c = Sum(alpha E_c), hh = B_c = Sum(beta E_c)
                        num = fmaf(p.coef[c], fmaf(E.x, hg.x, E.y * hg.y), num);
                        const float vx = fmaf(fc, hg.x, hh.x), vy = fmaf(fc, hg.y, hh.y);
                        den = fmaf(p.ck[c], fmaf(E.x, vy, -E.y * vx), den);
                    }
                    ++c;
                }
            }
            if (out) {
                const size_t o = (size_t)rho * W + co;
                if constexpr (MODE == ADJ) {
                    // centre quad: (f, 1/den, out, X)
                    const float al = gq[4] * q[4].y;
                    p.gimg[o] = fmaf(p.gamma, fmaf(al, q[4].w, den), num);
                } else {
                    const float ov = num / den;
                    p.out[o] = ov;
                    if constexpr (MODE == FWD_SAVE) {
                        // streaming store: the adjoint reads the quads after the whole forward
                        __stcs(p.sv + quad_index(rho, co, p.H, W),
                               make_float4(fc, 1.0f / den, ov, fmaf(-ov, dd, dn)));
                    }
                }
            }
        }
        __syncthreads();
    }
}


// Combo-sum form (one complex FMA per combo and step) while the combos are
// at most 1.6 times the (b, k) planes; the plane-sum form above otherwise,
// whose per-step cost grows with the planes and whose hand-off rotations
// replace the per-(a, b) phase products.
template <int M, int N>
constexpr bool use_combo_sum() {
    return 5 * Dims<M, N>::NS <= 8 * Dims<M, N>::ND;
}

template <typename K>
static cudaError_t launch_one(K kern, size_t smem, const Params& p, int gx, cudaStream_t s) {
    if (p.r < 1) return cudaErrorInvalidValue;  // r = 0 has its closed form
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    Params q = p;
    // one wave of as many CTAs as fit per SM (the adjoint's sheared quad loads
    // coalesce, so it no longer gains from fewer resident CTAs)
    if (q.Hb <= 0) q.Hb = wave_band_rows((const void*)kern, WMAX, smem, q.H, gx);
    const int gy = (q.H + q.Hb - 1) / q.Hb;
    kern<<<dim3(gx, gy), WMAX, smem, s>>>(q);
    return cudaGetLastError();
}

// Combo-sum adjoints with 18 or more combos run as two launches over halves of
// the combos: half the live sums and hand-off rows per launch leave the
// registers to keep the next step's pixel loads in flight.
template <int M, int N>
constexpr int adjoint_split() {
    return Dims<M, N>::NS >= 18 ? (Dims<M, N>::NS + 1) / 2 : Dims<M, N>::NS;
}

template <int M, int N>
static cudaError_t launch(const Params& p, int mode, int gx, int gy, cudaStream_t s) {
    using D = Dims<M, N>;
    static_assert(D::NS <= NS_CAP, "combo table");
    static_assert(D::NA <= FCAP && M / 2 + 1 <= FCAP && N / 2 + 1 <= FCAP, "factor tables");
    const size_t tab = sizeof(float4) * 2 * (size_t)PTAB_CAP;
    if constexpr (use_combo_sum<M, N>()) {
        if (mode == FWD || mode == FWD_SAVE) {
            const size_t smem = sizeof(float4) * 2 * (size_t)D::NS * (WMAX + 1) + tab;
            return mode == FWD_SAVE
                       ? launch_one(spk_kernel<M, N, FWD_SAVE>, smem, p, gx, s)
                       : launch_one(spk_kernel<M, N, FWD>, smem, p, gx, s);
        }
        constexpr int H = adjoint_split<M, N>();
        cudaError_t e = launch_one(spk_kernel<M, N, ADJ, 0, H>,
                                   sizeof(float4) * 2 * (size_t)H * (WMAX + 1) + tab, p, gx, s);
        if constexpr (H < D::NS) {
            if (e == cudaSuccess)
                e = launch_one(spk_kernel<M, N, ADJ, H, D::NS>,
                               sizeof(float4) * 2 * (size_t)(D::NS - H) * (WMAX + 1) + tab, p, gx,
                               s);
        }
        return e;
    } else {
        const size_t smem =
            sizeof(float4) * 2 * (size_t)D::NS * (WMAX + 1) + sizeof(float2) * PTAB_CAP;
        auto kern = mode == ADJ ? spk_plane_kernel<M, N, ADJ>
                                : (mode == FWD_SAVE ? spk_plane_kernel<M, N, FWD_SAVE>
                                                    : spk_plane_kernel<M, N, FWD>);
        return launch_one(kern, smem, p, gx, s);
    }
}

// Combo order and coefficients, as the kernel enumerates them:
// coef_c = 1/4 beta_a beta_|b| alpha_|k| m_b m_k (m = 2 for b = 0, k = 0:
// both sign choices give the same term), doubled for a = 0 except the
// self-conjugate (0, 0, 0). Returns the combo count, or -1.
static int combo_coefs(int M, int N, const double* beta, const double* alpha, double* coef) {
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
            coef[c++] = v;
        }
    }
    return c;
}

// The combo-sum kernel's factors fa, fb, fk of coef_c, checked against every
// combo's coefficient (with the self-conjugate combo halved), and the
// plane-sum kernel's per-combo coef_c and coef_c k_c.
static bool combo_factors(int M, int N, const double* beta, const double* alpha, Params* p) {
    if (M / 2 + 1 > FCAP || N / 2 + 1 > FCAP) return false;
    for (int i = 0; i <= M / 2; ++i) {
        const int a = (M & 1) + 2 * i;
        p->fa[i] = (float)(beta[i] * (a == 0 ? 2.0 : 1.0));
        p->fb[i] = (float)(0.25 * beta[i] * (a == 0 ? 2.0 : 1.0));
    }
    for (int i = 0; i <= N / 2; ++i) {
        const int k = (N & 1) + 2 * i;
        p->fk[i] = (float)(alpha[i] * (k == 0 ? 2.0 : 1.0));
    }
    double coef[NS_CAP];
    if (combo_coefs(M, N, beta, alpha, coef) < 0) return false;
    const int NB = M + 1, NK = N + 1, ND = NB * NK, D0 = ND - (ND + 1) / 2;
    int c = 0;
    for (int ia = 0; ia <= M / 2; ++ia) {
        const int a = (M & 1) + 2 * ia;
        for (int d = 0; d < ND; ++d) {
            if (a == 0 && d < D0) continue;
            const int b = -M + 2 * (d / NK), k = -N + 2 * (d % NK);
            const int ab = b < 0 ? -b : b, ak = k < 0 ? -k : k;
            double v = (double)p->fa[ia] * p->fb[(ab - (M & 1)) / 2] * p->fk[(ak - (N & 1)) / 2];
            if (a == 0 && b == 0 && k == 0) v *= 0.5;
            if (fabs(v - coef[c]) > 1e-6 * fabs(coef[c]) + 1e-30) return false;
            p->coef[c] = (float)coef[c];
            p->ck[c] = (float)(coef[c] * (double)k);
            ++c;
        }
    }
    return true;
}

static bool supported(int M, int N) {
    if (N == 0) return M >= 1 && M <= 8 && M != 7 && M != 5;
    return (M == 1 || M == 2) && N >= 1 && N <= 4;
}

template <int M>
static cudaError_t dispatch_n(const Params& p, int mode, int N, int gx, int gy, cudaStream_t s) {
    if constexpr (M == 1 || M == 2) {
        switch (N) {
            case 0: return launch<M, 0>(p, mode, gx, gy, s);
            case 1: return launch<M, 1>(p, mode, gx, gy, s);
            case 2: return launch<M, 2>(p, mode, gx, gy, s);
            case 3: return launch<M, 3>(p, mode, gx, gy, s);
            case 4: return launch<M, 4>(p, mode, gx, gy, s);
        }
        return cudaErrorInvalidValue;
    } else {
        return N == 0 ? launch<M, 0>(p, mode, gx, gy, s) : cudaErrorInvalidValue;
    }
}

// Checks shared by the forward and the adjoint; fills the launch parameters
// (coefficients, gamma, tiles) and resolves N.
static bf_status prepare(int H, int W, int r, int M, float sigma_r, float T, int* N,
                         const bf_opts* opts, Params* p, int* gx, int* gy) {
    if (H < 1 || W < 1 || r < 0 || M < 1) return BF_ERR_INVALID_ARG;
    if (!(T > 0.f) || !isfinite(T)) return BF_ERR_INVALID_ARG;
    bf_status st = check_opts(opts);
    if (st != BF_OK) return st;
    if (opts && (opts->in_dtype != BF_F32 || opts->kahan || opts->trunc_tol > 0.f ||
                 opts->gamma_mode != BF_GAMMA_FIXED || (opts->pitch != 0 && opts->pitch != W)))
        return BF_ERR_UNSUPPORTED;
    if (*N < 0) {
        *N = bf_resolve_N(sigma_r, T);
        if (*N < 0) return BF_ERR_INVALID_ARG;
    }
    if (!supported(M, *N)) return BF_ERR_UNSUPPORTED;
    if (2 * r + 16 > WMAX) return BF_ERR_UNSUPPORTED;
    double gamma = 0.0;
    if (*N > 0) {
        gamma = bf_gamma(sigma_r, T, *N, BF_GAMMA_FIXED);
        if (!(gamma > 0.0)) return BF_ERR_INVALID_ARG;
    }
    double beta[BF_N_MAX / 2 + 1], alpha[BF_N_MAX / 2 + 1];
    if (bf_coeffs(M, beta, BF_N_MAX / 2 + 1) < 0 || bf_coeffs(*N, alpha, BF_N_MAX / 2 + 1) < 0)
        return BF_ERR_INTERNAL;
    memset(p, 0, sizeof(*p));
    if (!combo_factors(M, *N, beta, alpha, p)) return BF_ERR_INTERNAL;
    p->H = H; p->W = W; p->r = r;
    p->gamma = (float)gamma;
    p->Tw = WMAX - 2 * r;
    *gx = (W + p->Tw - 1) / p->Tw;
    // band height: the caller's, else (0) one wave of the launched kernel's
    // resident CTAs, chosen at launch
    p->Hb = (opts && opts->tile_h > 0) ? opts->tile_h : 0;
    *gy = 0;
    return BF_OK;
}

static cudaError_t dispatch(const Params& p, int mode, int M, int N, int gx, int gy,
                            cudaStream_t s) {
    switch (M) {
        case 1: return dispatch_n<1>(p, mode, N, gx, gy, s);
        case 2: return dispatch_n<2>(p, mode, N, gx, gy, s);
        case 3: return dispatch_n<3>(p, mode, N, gx, gy, s);
        case 4: return dispatch_n<4>(p, mode, N, gx, gy, s);
        case 6: return dispatch_n<6>(p, mode, N, gx, gy, s);
        case 8: return dispatch_n<8>(p, mode, N, gx, gy, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace spk
}  // namespace bf

using namespace bf;

extern "C" bf_status bf_spatial_forward(const void* img, int H, int W, int r, int M,
                                        float sigma_r, float T, int N, float* out,
                                        const bf_opts* opts, void* saved, void* stream) {
    BF_TRACE("bf_spatial_forward");
    // the saved quads are indexed in 32 bits here (quad_index)
    if ((long long)H * W >= 0x7fffffffLL) return BF_ERR_UNSUPPORTED;
    if (!img || !out) return BF_ERR_INVALID_ARG;
    if ((const void*)out == img) return BF_ERR_INVALID_ARG;
    if (saved && ((uintptr_t)saved & 15)) return BF_ERR_INVALID_ARG;
    if (opts && opts->save_for_backward && !saved) return BF_ERR_INVALID_ARG;
    spk::Params p;
    int gx = 0, gy = 0;
    bf_status st = spk::prepare(H, W, r, M, sigma_r, T, &N, opts, &p, &gx, &gy);
    if (st != BF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    p.img = static_cast<const float*>(img);
    p.out = out;
    p.sv = static_cast<float4*>(saved);
    const int mode = saved ? spk::FWD_SAVE : spk::FWD;
    if (r == 0) {
        // a 1 x 1 window weighs the centre alone (q_M(0) = q_N(0) = 1, slope 0):
        // out = f. The strip's hand-off would telescope over all lanes with
        // signed terms here and lose digits to no purpose.
        cudaError_t e = unit_window(static_cast<const float*>(img), out,
                                    static_cast<float4*>(saved), H, W, s);
        return e == cudaSuccess ? BF_OK : set_cuda_error(e);
    }
    cudaError_t e = spk::dispatch(p, mode, M, N, gx, gy, s);
    if (e != cudaSuccess) return set_cuda_error(e);
    return BF_OK;
}

extern "C" bf_status bf_spatial_backward(const float* grad_out, const void* saved, int H, int W,
                                         int r, int M, float sigma_r, float T, int N,
                                         float* grad_img, const bf_opts* opts, void* stream) {
    BF_TRACE("bf_spatial_backward");
    // the saved quads are indexed in 32 bits here (quad_index)
    if ((long long)H * W >= 0x7fffffffLL) return BF_ERR_UNSUPPORTED;
    if (!grad_out || !saved || !grad_img) return BF_ERR_INVALID_ARG;
    if ((uintptr_t)saved & 15) return BF_ERR_INVALID_ARG;
    // neighbours' dL/dout and quads are read while dL/dimg is written
    if ((const void*)grad_img == (const void*)grad_out || (const void*)grad_img == saved)
        return BF_ERR_INVALID_ARG;
    spk::Params p;
    int gx = 0, gy = 0;
    bf_status st = spk::prepare(H, W, r, M, sigma_r, T, &N, opts, &p, &gx, &gy);
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
    cudaError_t e = spk::dispatch(p, spk::ADJ, M, N, gx, gy, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_cuda_error(e);
    return BF_OK;
}
