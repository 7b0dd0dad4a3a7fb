// Forward kernel of the constant-time raised-cosine bilateral filter.
//
// Algorithm 2 (Sec. 2) with M = 1 (box spatial kernel) and range kernel
// q_N(t) = cos^N(gamma t) (Sec. 3). Each harmonic k of q_N's shift expansion
// contributes four pointwise-transformed images (C_k f, S_k f, C_k, S_k),
// C_k = cos(k gamma f), S_k = sin(k gamma f); their box sums over the
// (2r+1)^2 window are recombined with the centre pixel's C_k, S_k and the
// interpolating coefficients a_k into num and den (Algorithm 2, step 3).
//
// Tile organisation (one CTA = a strip of Tw output columns x a band of Hb
// output rows; NT = Tw + 2r threads, one per input column of the strip):
//  * vertical pass: every thread walks its column down the band keeping the
//    vertical running sums V_k of all four planes of every harmonic in
//    registers. Per row it adds the entering pixel's planes and subtracts the
//    leaving pixel's (the moving sum of Sec. 2). The planes are regenerated
//    from f: one sincos per pixel, then the harmonics by complex rotation
//    z_{k+2} = z_k * z_2, so the stack never exists in memory.
//  * horizontal pass: the row of V_k goes to shared memory; each output
//    thread sums its 2r+1 neighbours and combines with its centre pixel.
//  The window is truncated at the image border: pixels outside the image
//  contribute zero planes (their rotation seed is zero).
#include "bf_internal.cuh"
#include "bf_quads.cuh"

namespace bf {

__device__ __forceinline__ float load_px(const float* p, size_t i) { return __ldg(p + i); }
__device__ __forceinline__ float load_px(const __nv_bfloat16* p, size_t i) {
    return __bfloat162float(p[i]);
}

// Seed of the rotation for one pixel value v: z = first harmonic's (cos,
// sin), w = (cos 2 theta, sin 2 theta). A masked pixel gets z = 0, so every
// plane it contributes is zero.
struct Seed {
    float zc, zs, wc, ws;
};

__device__ __forceinline__ Seed make_seed(float v, float gamma, int kstart, bool on) {
    float s, c;
    sincosf(gamma * v, &s, &c);
    Seed q;
    q.wc = (c - s) * (c + s);
    q.ws = 2.0f * s * c;
    if (kstart) { q.zc = c; q.zs = s; } else { q.zc = 1.0f; q.zs = 0.0f; }
    if (!on) { q.zc = 0.0f; q.zs = 0.0f; }
    return q;
}

__device__ __forceinline__ void rotate(float& zc, float& zs, float wc, float ws) {
    const float nc = zc * wc - zs * ws;
    const float ns = zs * wc + zc * ws;
    zc = nc;
    zs = ns;
}

// One strip x band tile (bx, by) of one image. Shared by the single-image
// kernel (grid = tiles) and the persistent batch kernel (tile queue).
template <int KMAX, bool KAHAN, typename Tin>
__device__ __forceinline__ void fwd_tile(const FwdParams& p, int bx, int by, float4* vrow) {
    const Tin* img = static_cast<const Tin*>(p.img);
    const int NT = blockDim.x;
    const int j = threadIdx.x;
    const int x0 = bx * p.Tw;
    const int c = x0 - p.r + j;
    const bool col_in = (c >= 0) && (c < p.W);
    const int y0 = by * p.Hb;
    const int y1 = min(y0 + p.Hb, p.H);
    const int r = p.r;
    const bool is_out = (j >= r) && (j < r + p.Tw) && col_in;

    float4 V[KMAX];
    float4 E[KAHAN ? KMAX : 1];
#pragma unroll
    for (int i = 0; i < KMAX; ++i) {
        V[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (KAHAN) E[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    for (int rho = y0 - 2 * r; rho < y1; ++rho) {
        const int e = rho + r;
        const int l = rho - r - 1;
        const bool me = col_in && e >= 0 && e < p.H;
        const bool ml = col_in && rho > y0 && l >= 0 && l < p.H;
        const float fe = me ? load_px(img, (size_t)e * p.ld + c) : 0.f;
        const float fl = ml ? load_px(img, (size_t)l * p.ld + c) : 0.f;
        Seed se = make_seed(fe, p.gamma, p.kstart, me);
        Seed sl = make_seed(fl, p.gamma, p.kstart, ml);
#pragma unroll
        for (int i = 0; i < KMAX; ++i) {
            if (i < p.K) {
                if (KAHAN) {
                    // each pixel's products added on their own with compensation
                    // (Kahan 1965), so a pixel's entering and leaving
                    // contributions (bit-identical products) cancel
                    auto kadd = [](float& v, float& e, float x) {
                        const float y = x - e;
                        const float t = v + y;
                        e = (t - v) - y;
                        v = t;
                    };
                    kadd(V[i].x, E[i].x, __fmul_rn(se.zc, fe));
                    kadd(V[i].x, E[i].x, -__fmul_rn(sl.zc, fl));
                    kadd(V[i].y, E[i].y, __fmul_rn(se.zs, fe));
                    kadd(V[i].y, E[i].y, -__fmul_rn(sl.zs, fl));
                    kadd(V[i].z, E[i].z, se.zc);
                    kadd(V[i].z, E[i].z, -sl.zc);
                    kadd(V[i].w, E[i].w, se.zs);
                    kadd(V[i].w, E[i].w, -sl.zs);
                } else {
                    float4 d;
                    d.x = se.zc * fe - sl.zc * fl;
                    d.y = se.zs * fe - sl.zs * fl;
                    d.z = se.zc - sl.zc;
                    d.w = se.zs - sl.zs;
                    V[i].x += d.x; V[i].y += d.y; V[i].z += d.z; V[i].w += d.w;
                }
                rotate(se.zc, se.zs, se.wc, se.ws);
                rotate(sl.zc, sl.zs, sl.wc, sl.ws);
            }
        }
        if (rho < y0) continue;  // warm-up rows of the vertical window (uniform)

#pragma unroll
        for (int i = 0; i < KMAX; ++i)
            if (i < p.K) vrow[i * NT + j] = V[i];
        __syncthreads();
        if (is_out) {
            const float fc = load_px(img, (size_t)rho * p.ld + c);
            Seed sc = make_seed(fc, p.gamma, p.kstart, true);
            float num = 0.f, den = 0.f, dnum = 0.f, dden = 0.f;
#pragma unroll 1
            for (int i = 0; i < p.K; ++i) {
                float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4* row = vrow + i * NT + j - r;
                for (int d = 0; d <= 2 * r; ++d) {
                    const float4 v = row[d];
                    h.x += v.x; h.y += v.y; h.z += v.z; h.w += v.w;
                }
                const float a = p.a[i];
                const float ak = a * (float)(p.kstart + 2 * i);
                num += a * (sc.zc * h.x + sc.zs * h.y);
                den += a * (sc.zc * h.z + sc.zs * h.w);
                dnum += ak * (sc.zc * h.y - sc.zs * h.x);
                dden += ak * (sc.zc * h.w - sc.zs * h.z);
                rotate(sc.zc, sc.zs, sc.wc, sc.ws);
            }
            const size_t o = quad_index64(rho, c, p.H, p.W);  // saved quads (sheared)
            const size_t op = (size_t)rho * p.ld + c;  // row-pitched (out, den)
            const float ov = num / den;
            p.out[op] = ov;
            if (p.den) p.den[op] = den;
            // saved for the adjoint: (f - mid, 1/den, out - mid, dnum - out dden)
            if (p.sv) p.sv[o] = make_float4(fc - p.mid, 1.0f / den, ov - p.mid, dnum - ov * dden);
        }
        __syncthreads();
    }
}

template <int KMAX, bool KAHAN, typename Tin>
__global__ void __launch_bounds__(256, 1) bf_fwd_strip_kernel(FwdParams p) {
    extern __shared__ float4 vrow[];  // [K][NT]
    fwd_tile<KMAX, KAHAN, Tin>(p, blockIdx.x, blockIdx.y, vrow);
}

// Persistent batch kernel: each CTA pops tile indices from a device counter
// until the table is exhausted. Images are stored in decreasing order of
// per-tile cost, so the longest tiles start first. No CTA ever waits on
// another, so there is no spin and nothing can hang.
template <bool KAHAN, typename Tin>
__global__ void __launch_bounds__(256, 1) bf_batch_kernel(BatchTable* tab) {
    extern __shared__ float4 vrow[];
    __shared__ int s_tile;
    const int n_img = tab->n_images;
    const int n_tiles = tab->n_tiles;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&tab->counter, 1);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= n_tiles) break;
        // image holding tile t: last image whose first tile is <= t
        int lo = 0, hi = n_img - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tab->img[mid].first_tile <= t) lo = mid; else hi = mid - 1;
        }
        const BatchImage& bi = tab->img[lo];
        const int local = t - bi.first_tile;
        fwd_tile<KCAP, KAHAN, Tin>(bi.p, local % bi.gx, local / bi.gx, vrow);
    }
}

template <bool KAHAN, typename Tin>
static cudaError_t batch_launch_t(BatchTable* tab, int grid, cudaStream_t s) {
    auto kern = bf_batch_kernel<KAHAN, Tin>;
    const size_t smem = (size_t)KCAP * 256 * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 256, smem, s>>>(tab);
    return cudaGetLastError();
}

cudaError_t launch_batch(BatchTable* tab, int grid, int kahan, int in_dtype, cudaStream_t s) {
    if (in_dtype == BF_BF16)
        return kahan ? batch_launch_t<true, __nv_bfloat16>(tab, grid, s)
                     : batch_launch_t<false, __nv_bfloat16>(tab, grid, s);
    return kahan ? batch_launch_t<true, float>(tab, grid, s)
                 : batch_launch_t<false, float>(tab, grid, s);
}

template <int KMAX, bool KAHAN, typename Tin>
static cudaError_t launch_t(const FwdParams& p, int nt, cudaStream_t s) {
    auto kern = bf_fwd_strip_kernel<KMAX, KAHAN, Tin>;
    const size_t smem = (size_t)p.K * nt * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p.W + p.Tw - 1) / p.Tw, (p.H + p.Hb - 1) / p.Hb);
    kern<<<grid, nt, smem, s>>>(p);
    return cudaGetLastError();
}

template <bool KAHAN, typename Tin>
static cudaError_t launch_k(const FwdParams& p, int nt, cudaStream_t s) {
    if (p.K <= 8) return launch_t<8, KAHAN, Tin>(p, nt, s);
    if (p.K <= 16) return launch_t<16, KAHAN, Tin>(p, nt, s);
    if (p.K <= 24) return launch_t<24, KAHAN, Tin>(p, nt, s);
    return launch_t<KCAP, KAHAN, Tin>(p, nt, s);
}

cudaError_t launch_forward(const FwdParams& p, int nt, int kahan, int in_dtype, cudaStream_t s) {
    if (in_dtype == BF_BF16)
        return kahan ? launch_k<true, __nv_bfloat16>(p, nt, s)
                     : launch_k<false, __nv_bfloat16>(p, nt, s);
    return kahan ? launch_k<true, float>(p, nt, s) : launch_k<false, float>(p, nt, s);
}

}  // namespace bf
