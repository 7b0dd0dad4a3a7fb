// Internal declarations shared by the CUDA translation units of libbf.
// Nothing here is part of the C ABI (include/bf.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/bf.h"

namespace bf {

// Harmonics of q_N's expansion: k = N mod 2, N mod 2 + 2, ..., N, so
// K = N / 2 + 1 <= 33 for N <= 64.
constexpr int KCAP = BF_N_MAX / 2 + 1;

// Index of pixel (row, col)'s quad in the saved buffer of an H x W image. The
// rows are sheared by (col mod 128) and wrapped at H (for H >= 128; plain
// row-major below): the skewed-strip engine reads and writes one pixel per
// lane on an anti-diagonal (row + col fixed across a warp), and in this
// layout those pixels are consecutive, so a warp's quad loads and stores
// are contiguous instead of one row each.
__host__ __device__ __forceinline__ int quad_index(int row, int col, int H, int W) {
    int rr = row + (col & (H >= 128 ? 127 : 0));
    if (rr >= H) rr -= H;
    return rr * W + col;
}

// Everything one filter launch needs, passed by value as the kernel
// parameter (a_k sits in the constant parameter bank, no __constant__
// symbol, so concurrent launches with different N never race).
struct FwdParams {
    const void* img;      // H x W (row pitch ld), FP32 or BF16
    float* out;           // H x W (row pitch ld)
    float4* sv;           // saved quads (f - mid, 1/den, out - mid, dnum - out dden); nullable, compact
    float* den;           // den of Eq. filter2 (row pitch ld); nullable
    int H, W, r;
    int ld;               // row pitch of img, out and den in elements (>= W)
    int K;                // number of harmonics
    int kstart;           // N mod 2: frequency of harmonic 0
    int Hb;               // output rows per band (grid.y tiles)
    int Tw;               // output columns per strip (grid.x tiles)
    float gamma;
    float mid;            // T / 2, the centre of the range [0, T]
    float a[KCAP];        // a_k for harmonic i (frequency kstart + 2 i)
};

struct BwdParams {
    const void* img;      // forward input
    const float* gout;    // dL/dout (row pitch ld)
    const float4* sv;     // the forward's saved quads (compact)
    float* gimg;          // dL/dimg (nullable, row pitch ld)
    float* partial;       // per-CTA sums of (f - T/2) * dL/dtheta (nullable)
    int H, W, r, K, kstart, Hb, Tw;
    int ld;               // row pitch of gout and gimg in elements (>= W)
    float gamma;
    float a[KCAP];
};

// Skewed-strip engine (bf_sys.cu): forward and adjoint share one kernel
// template. Up to SYS_KMAX harmonics are kept in registers (8 floats each).
constexpr int SYS_MAX_THREADS = 256;

struct SysParams {
    const void* img;
    float* out;                 // forward output
    float4* sv;                 // forward: saved quads (SAVE)
    const float* gout;          // adjoint: dL/dout
    const float4* bsv;          // adjoint: the forward's saved quads
    float* gimg;                // adjoint: dL/dimg (nullable)
    float* partial;             // adjoint: per-CTA sum of (f - T/2) * dL/dtheta (nullable)
    float* acc_den;             // forward chunk accumulator for den when not saving
    float* acc_gv;              // adjoint chunk accumulators (value and phase parts)
    float* acc_gt;
    float* dout;                // forward: den of Eq. filter2 (nullable; row pitch ld)
    int H, W, r, K, kstart, Hb, Tw;
    int ld;          // row pitch (elements) of img, out, gout, gimg, dout; >= W
    int B;           // images of a [B, H, W] launch (grid.z); 0 or 1 = one image
    int k0;          // frequency of this launch's first harmonic
    int acc;         // 0 all harmonics; 1 first, 2 middle, 3 last harmonic chunk
    float gamma;
    float mid;       // forward: T / 2, the value the planes centre f on
    float gpi;       // gamma / pi
    float a[KCAP];   // a_k of harmonic i (of this chunk)
    float ak[KCAP];  // k * a_k (centre-derivative terms)
};

// Largest harmonic pairs per launch (registers); more harmonics run in chunks.
constexpr int SYS_KP_MAX = 11;
constexpr int SYS_KP_KAHAN = 6;

// mode: 0 forward, 1 forward + saved buffers, 2 adjoint.
cudaError_t launch_sys(const SysParams& p, int mode, bool kahan, int in_dtype, int wi, int gx,
                       int gy, cudaStream_t s, int kp_max = 0);
int sys_chunks(int K, bool kahan, int kp_max = 0);
cudaError_t launch_sys_w128(const SysParams& p, int mode, int dtype, int kp, int wi, int gx,
                            int gy, cudaStream_t s);
cudaError_t launch_sys_w256(const SysParams& p, int mode, int dtype, int kp, int wi, int gx,
                            int gy, cudaStream_t s);
cudaError_t launch_sys_kahan(const SysParams& p, int mode, int dtype, int kp, int wi, int gx,
                             int gy, cudaStream_t s);
// First (or only) harmonic chunk of a compact image on strips of up to WMAX =
// 128 or 64 threads: KP pairs (1..11), half = the last pair holds one
// harmonic, seed = 1 (odd N, k0 = 1) or 2 (even N, k0 = 0, the constant
// harmonic kept apart from the pairs). Explicitly instantiated in
// bf_sys_first_*.cu (128, FP32), bf_sys_first64_*.cu (64, FP32) and
// bf_sys_first16_*.cu (128, BF16 input: forward modes only).
template <int KP, int WMAX, typename Tin>
cudaError_t sys_first_kp(const SysParams& p, int mode, bool half, int seed, int wi, int gx,
                         int gy, cudaStream_t s);

// One image of a batch as the persistent kernel sees it: its launch
// parameters, its tile grid width and the index of its first tile.
struct BatchImage {
    FwdParams p;
    int gx;          // strips of this image
    int first_tile;  // prefix sum of tiles over the images before it
    int n_tiles;     // gx * gy
    int pad;
};

// Device tile table in the caller's workspace: header, then images.
struct BatchTable {
    int counter;     // next tile to hand out (reset by each launch)
    int n_tiles;
    int n_images;
    int grid;        // persistent CTAs to launch
    int kahan;
    int in_dtype;
    int pad[2];
    BatchImage img[1];  // n_images entries
};

// Batch on the skewed-strip engine: per image up to two harmonic chunks
// (K <= 33), each with its own launch parameters (coefficients of that chunk,
// first frequency, accumulation mode).
constexpr int SYS_BATCH_MAX_CHUNKS = 2;

struct SysBatchImage {
    SysParams ch[SYS_BATCH_MAX_CHUNKS];
    int kp[SYS_BATCH_MAX_CHUNKS];  // harmonic-pair instantiation of each chunk
    int nch;
    int gx;
    int first_tile;
    int n_tiles;
    int kind;   // index of its specialised kernel (sys_batch_kind), or -1
};

// Work of one persistent launch (one strip width): image range and tiles.
struct SysBatchGroup {
    int n_tiles;
    int img0;       // first image of the group in the image array
    int n_images;
    int wi;         // threads per strip
};

// Groups of one batch, one persistent launch each: on 128-thread strips, 0 =
// harmonics in one chunk of at most SYS_BATCH_SMALL_KP pairs (the first-chunk
// specialisations, compile-time seed and half pair, three CTAs per SM), 1 =
// the rest (general kernel); 2 = 256-thread strips (general kernel).
constexpr int SYS_BATCH_GROUPS = 3;
constexpr int SYS_BATCH_SMALL_KP = 4;

struct SysBatchTable {
    int counters[4];  // next tile of each group (reset by every launch)
    int magic;
    int in_dtype;
    int pad[2];
    SysBatchGroup g[SYS_BATCH_GROUPS];
    SysBatchImage img[1];  // all images, group 0 first
};

// Specialised kernel of a one-chunk image with K harmonics starting at kstart
// (N mod 2): sets *group to 0 and returns the kernel's index within it when
// the harmonics fit SYS_BATCH_SMALL_KP pairs, else -1 (the general kernel).
int sys_batch_kind(int K, int kstart, int* group);
// Resident CTAs of a group's persistent kernel on this device.
int sys_batch_grid(int group, int in_dtype);
cudaError_t launch_sys_batch(SysBatchTable* tab, int group, int grid, int in_dtype,
                             cudaStream_t s);

// Host-side parameter preparation shared by the entry points.
struct Resolved {
    int N, K, kstart;
    double gamma;
    double a[KCAP];
};

bf_status resolve(int r, float sigma_r, float T, int N, int gamma_mode, float trunc_tol,
                  Resolved* out);
bf_status set_cuda_error(cudaError_t e);

// Launchers (defined in the kernel translation units).
cudaError_t launch_forward(const FwdParams& p, int nthreads, int kahan, int in_dtype,
                           cudaStream_t s);
cudaError_t launch_backward(const BwdParams& p, int nthreads, int in_dtype, cudaStream_t s);
cudaError_t launch_batch(BatchTable* tab, int grid, int kahan, int in_dtype, cudaStream_t s);
int sm_count();
bf_status check_opts(const bf_opts* o);
bf_status fill_fwd_params(const void* img, float* out, void* saved, int H, int W, int pitch,
                          int r, float sigma_r, float T, int N, const bf_opts* opts,
                          FwdParams* p, int* nt, int* gx, int* gy);
int row_pitch(int pitch, int W);
cudaError_t launch_reduce_sigma(const float* partial, int n, float scale, float* dst,
                                cudaStream_t s);

}  // namespace bf
