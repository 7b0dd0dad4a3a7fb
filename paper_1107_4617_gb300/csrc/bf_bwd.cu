// Adjoint kernel of the constant-time raised-cosine bilateral filter.
//
// For L with dL/dout = g, let alpha = g / den and beta = -alpha * out (per
// pixel). Differentiating num and den of Algorithm 2 (M = 1) with respect to
// f(p), and using that the truncated box window is symmetric (x is in the
// window of p iff p is in the window of x), every neighbour term becomes a box
// sum evaluated at p:
//   A_k = Box[alpha C_k], B_k = Box[alpha S_k], Cb_k = Box[beta C_k],
//   Db_k = Box[beta S_k],
//   dL/df(p) = sum_k a_k (A_k C_k + B_k S_k)                      (value part)
//            + gamma * G_theta(p),
//   G_theta  = sum_k a_k k [f (B_k C_k - A_k S_k) + (Db_k C_k - Cb_k S_k)]
//            + alpha * dnum_s + beta * dden_s                     (phase part)
// with dnum_s = sum_k a_k k (C_k Box[S_k f] - S_k Box[C_k f]) and dden_s the
// same with Box[S_k], Box[C_k] (saved by the forward). Since theta = gamma f,
// dL/dgamma = sum_p f(p) G_theta(p).
//
// Everything here is unchanged when f and out are shifted by one constant c:
// the weights depend on differences of theta only, so sum_p G_theta(p) = 0
// and dL/dgamma = sum_p (f(p) - c) G_theta(p) as well. The saved quads carry
// f and out shifted by the range midpoint (c = T / 2), and this pass uses
// them as they are.
//
// The stack (alpha C_k, alpha S_k, beta C_k, beta S_k) is recomputed from g
// and the forward's saved quads (f - c, 1/den, out - c, dnum - out dden) with the same
// vertical-walker / horizontal-window tile organisation as the forward
// kernel; it is never stored.
#include "bf_internal.cuh"
#include "bf_quads.cuh"

namespace bf {


struct BSeed {
    float zc, zs, wc, ws;
};

__device__ __forceinline__ BSeed bseed(float v, float gamma, int kstart, bool on) {
    float s, c;
    sincosf(gamma * v, &s, &c);
    BSeed q;
    q.wc = (c - s) * (c + s);
    q.ws = 2.0f * s * c;
    if (kstart) { q.zc = c; q.zs = s; } else { q.zc = 1.0f; q.zs = 0.0f; }
    if (!on) { q.zc = 0.0f; q.zs = 0.0f; }
    return q;
}

__device__ __forceinline__ void brot(float& zc, float& zs, float wc, float ws) {
    const float nc = zc * wc - zs * ws;
    const float ns = zs * wc + zc * ws;
    zc = nc;
    zs = ns;
}

template <int KMAX>
__global__ void __launch_bounds__(256, 1) bf_bwd_strip_kernel(BwdParams p) {
    extern __shared__ float4 vrow[];
    __shared__ float red[32];
    const int NT = blockDim.x;
    const int j = threadIdx.x;
    const int x0 = blockIdx.x * p.Tw;
    const int c = x0 - p.r + j;
    const bool col_in = (c >= 0) && (c < p.W);
    const int y0 = blockIdx.y * p.Hb;
    const int y1 = min(y0 + p.Hb, p.H);
    const int r = p.r;
    const bool is_out = (j >= r) && (j < r + p.Tw) && col_in;

    float4 V[KMAX];
#pragma unroll
    for (int i = 0; i < KMAX; ++i) V[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    float gsum = 0.f;

    for (int rho = y0 - 2 * r; rho < y1; ++rho) {
        const int e = rho + r;
        const int l = rho - r - 1;
        const bool me = col_in && e >= 0 && e < p.H;
        const bool ml = col_in && rho > y0 && l >= 0 && l < p.H;
        float fe = 0.f, ae = 0.f, be = 0.f, fl = 0.f, al = 0.f, bl = 0.f;
        if (me) {
            const float4 sv = __ldg(p.sv + quad_index64(e, c, p.H, p.W));
            fe = sv.x;
            ae = __ldg(p.gout + (size_t)e * p.ld + c) * sv.y;
            be = -ae * sv.z;
        }
        if (ml) {
            const float4 sv = __ldg(p.sv + quad_index64(l, c, p.H, p.W));
            fl = sv.x;
            al = __ldg(p.gout + (size_t)l * p.ld + c) * sv.y;
            bl = -al * sv.z;
        }
        BSeed se = bseed(fe, p.gamma, p.kstart, me);
        BSeed sl = bseed(fl, p.gamma, p.kstart, ml);
#pragma unroll
        for (int i = 0; i < KMAX; ++i) {
            if (i < p.K) {
                V[i].x += se.zc * ae - sl.zc * al;
                V[i].y += se.zs * ae - sl.zs * al;
                V[i].z += se.zc * be - sl.zc * bl;
                V[i].w += se.zs * be - sl.zs * bl;
                brot(se.zc, se.zs, se.wc, se.ws);
                brot(sl.zc, sl.zs, sl.wc, sl.ws);
            }
        }
        if (rho < y0) continue;

#pragma unroll
        for (int i = 0; i < KMAX; ++i)
            if (i < p.K) vrow[i * NT + j] = V[i];
        __syncthreads();
        if (is_out) {
            const size_t o = quad_index64(rho, c, p.H, p.W);  // saved quads (sheared)
            const size_t op = (size_t)rho * p.ld + c;  // row-pitched (dL/dout, dL/dimg)
            const float4 svc = __ldg(p.sv + o);
            const float fc = svc.x;
            const float ac = __ldg(p.gout + op) * svc.y;
            BSeed sc = bseed(fc, p.gamma, p.kstart, true);
            float gv = 0.f, gt = 0.f;
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
                gv += a * (h.x * sc.zc + h.y * sc.zs);
                gt += ak * (fc * (h.y * sc.zc - h.x * sc.zs) + (h.w * sc.zc - h.z * sc.zs));
                brot(sc.zc, sc.zs, sc.wc, sc.ws);
            }
            gt += ac * svc.w;
            if (p.gimg) p.gimg[op] = gv + p.gamma * gt;
            gsum += fc * gt;
        }
        __syncthreads();
    }

    if (p.partial) {
        // Deterministic CTA sum of f * G_theta: warp shuffles, then one warp.
        for (int o = 16; o > 0; o >>= 1) gsum += __shfl_down_sync(0xffffffffu, gsum, o);
        if ((j & 31) == 0) red[j >> 5] = gsum;
        __syncthreads();
        if (j < 32) {
            float v = (j < (NT >> 5)) ? red[j] : 0.f;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (j == 0) p.partial[blockIdx.y * gridDim.x + blockIdx.x] = v;
        }
    }
}

// Sums the per-CTA partials in a fixed order (one CTA) and scales.
__global__ void bf_reduce_sigma_kernel(const float* partial, int n, float scale, float* dst) {
    __shared__ double acc[256];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += (double)partial[i];
    acc[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) acc[threadIdx.x] += acc[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *dst = (float)(acc[0] * (double)scale);
}

template <int KMAX>
static cudaError_t blaunch_t(const BwdParams& p, int nt, cudaStream_t s) {
    auto kern = bf_bwd_strip_kernel<KMAX>;
    const size_t smem = (size_t)p.K * nt * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p.W + p.Tw - 1) / p.Tw, (p.H + p.Hb - 1) / p.Hb);
    kern<<<grid, nt, smem, s>>>(p);
    return cudaGetLastError();
}

static cudaError_t blaunch_k(const BwdParams& p, int nt, cudaStream_t s) {
    if (p.K <= 8) return blaunch_t<8>(p, nt, s);
    if (p.K <= 16) return blaunch_t<16>(p, nt, s);
    if (p.K <= 24) return blaunch_t<24>(p, nt, s);
    return blaunch_t<KCAP>(p, nt, s);
}

// The saved quads carry f already decoded to FP32, so the input dtype does
// not matter here.
cudaError_t launch_backward(const BwdParams& p, int nt, int in_dtype, cudaStream_t s) {
    (void)in_dtype;
    return blaunch_k(p, nt, s);
}

cudaError_t launch_reduce_sigma(const float* partial, int n, float scale, float* dst,
                                cudaStream_t s) {
    bf_reduce_sigma_kernel<<<1, 256, 0, s>>>(partial, n, scale, dst);
    return cudaGetLastError();
}

}  // namespace bf
