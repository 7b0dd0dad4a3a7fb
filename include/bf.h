/*
 * bf.h -- C ABI of the constant-time raised-cosine bilateral filter on one
 * NVIDIA GB300 (sm_103a).
 *
 * The filter is Eq. "filter2" of Sec. 2 (bilateral filter) with a box spatial
 * kernel over the square window |y - x|_inf <= r and the range kernel
 * q_N(t) = cos^N(gamma t) of Sec. 3, gamma = pi / (2T). Because q_N is
 * shiftable (Eq. "def") with N+1 basis functions, Algorithm 2 with M = 1
 * turns the filter into moving sums (the Sum(F, x, T) of Sec. 2) of a stack of
 * 2(N+1) pointwise transforms of the image:
 *
 *   cos^N(gamma (s - t)) = sum_k a_k [cos(k gamma s) cos(k gamma t)
 *                                     + sin(k gamma s) sin(k gamma t)],
 *   k = N, N-2, ..., N mod 2;  a_k = 2^(1-N) C(N, (N-k)/2) (k > 0),
 *   a_0 = 2^(-N) C(N, N/2),
 *   num(x) = sum_k a_k [C_k(x) Box(C_k f)(x) + S_k(x) Box(S_k f)(x)],
 *   den(x) = sum_k a_k [C_k(x) Box(C_k)(x)   + S_k(x) Box(S_k)(x)],
 *   out(x) = num(x) / den(x),   C_k = cos(k gamma f), S_k = sin(k gamma f).
 *
 * Border: the window is truncated to the image (sums run over in-image
 * pixels only).
 *
 * Conventions shared by every call below:
 *  - Image pointers are DEVICE pointers to row-major H x W arrays, unless the
 *    name says _host. Rows of the image buffers (img, out, grad_out, grad_img,
 *    den) lie `pitch` elements apart: bf_opts.pitch for bf_forward /
 *    bf_backward and their [B, H, W] forms (image b then starts b * H * pitch
 *    elements in), bf_desc.pitch for bf_batch; 0 means W (a compact image),
 *    and a pitch below W is BF_ERR_INVALID_ARG. A pitch lets a caller filter a
 *    region of a larger image, or a strided tensor view, without a copy:
 *    elements between W and pitch in each row are neither read nor written.
 *    The saved quads, workspaces and the variant filters (bf_spatial_*,
 *    bf_poly_*, which reject a pitch other than 0 or W with
 *    BF_ERR_UNSUPPORTED) are always compact. The caller owns every buffer; no
 *    call allocates device memory.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls are
 *    asynchronous on it and never synchronise the host.
 *  - Argument checks run before any launch; on a failed check nothing is
 *    written and the status is returned. A CUDA launch or copy error returns
 *    BF_ERR_CUDA and its cudaError_t code is kept per host thread for
 *    bf_last_cuda_error().
 *  - Precondition (not checked on the hot path): max f - min f <= T. Inside
 *    it every weight is >= 0 and den >= 1. Outside it the result is still the
 *    exact cos^N filter, but den may approach or cross 0.
 *  - Thread safety: all state lives in the arguments; calls from several host
 *    threads on several streams may run concurrently.
 */
#ifndef BF_H_
#define BF_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Largest order N accepted (33 harmonics). */
#define BF_N_MAX 64
/* Largest spatial half-width r accepted (window up to 129 x 129). */
#define BF_R_MAX 64

typedef enum {
    BF_OK = 0,
    BF_ERR_INVALID_ARG = 1,  /* a size, pointer or parameter is out of range */
    BF_ERR_UNSUPPORTED = 2,  /* valid request outside what is built (N > BF_N_MAX, r > BF_R_MAX) */
    BF_ERR_CUDA = 3,         /* a CUDA runtime call failed; see bf_last_cuda_error */
    BF_ERR_TIMEOUT = 4,      /* a bounded device wait ran out */
    BF_ERR_INTERNAL = 5,
    BF_ERR_NOMEM = 6         /* a caller-supplied buffer is too small */
} bf_status;

typedef enum { BF_F32 = 0, BF_BF16 = 1 } bf_dtype;

typedef enum {
    /* gamma = pi / (2T): q_N of Sec. 3 exactly. sigma_r only picks N, so
       dL/dsigma_r is 0. */
    BF_GAMMA_FIXED = 0,
    /* gamma = 1 / (sigma_r sqrt(N)): the Gaussian limit (Eq. approx2) then has
       variance sigma_r^2 exactly (the variance control of Sec. 3); N is
       frozen by the rule, and dL/dsigma_r = -(gamma / sigma_r) dL/dgamma. */
    BF_GAMMA_FROM_SIGMA = 1
} bf_gamma_mode;

typedef struct {
    int kahan;            /* 1: Kahan-compensated vertical running sums */
    int gamma_mode;       /* bf_gamma_mode */
    int in_dtype;         /* bf_dtype of img (output is always FP32) */
    int save_for_backward;/* 1: bf_forward fills `saved` (also implied by saved != NULL) */
    int tile_h;           /* rows per band; 0 = built-in choice */
    int tile_w;           /* threads per strip (multiple of 32, > 2r); 0 = built-in */
    int kp_max;           /* most harmonic pairs per launch, 1..11; 0 = 11. Fewer pairs
                             mean fewer registers per thread; the harmonics then run
                             in chunks, which accumulate in `saved` (forward) or the
                             workspace (adjoint) */
    float trunc_tol;      /* 0: the exact q_N. > 0 (and < 1): keep only the lowest
                             harmonics of q_N's expansion, dropping the highest ones
                             while their a_k sum to at most min(trunc_tol,
                             1/(2 (2r+1)^2)) (end of Sec. 3: discard the less
                             significant basis functions). The range kernel then
                             differs from cos^N(gamma t) by at most that sum
                             anywhere on [-T, T], may dip below 0 by as much, and
                             den >= 1/2 still holds. Forward and backward calls
                             must pass the same value. See bf_trunc_harmonics. */
    int pitch;            /* row pitch of the image buffers in elements; 0 = W */
} bf_opts;

/* One image of a batch (bf_batch). img/out/den are device pointers. */
typedef struct {
    const void* img;      /* H x W, dtype opts->in_dtype */
    float* out;           /* H x W */
    float* den;           /* NULL, or H x W receiving den(x), the normaliser eta(x) of
                             Eq. filter2 (sum of the window's weights; >= 1 inside the
                             precondition); must not alias img or out */
    int H, W;
    int pitch;            /* row pitch of img, out and den in elements; 0 = W */
    int r;                /* spatial half-width, 0..BF_R_MAX */
    int N;                /* order; <= 0 derives it from sigma_r (bf_resolve_N) */
    float sigma_r;
    float T;              /* range bound, > 0 */
} bf_desc;

/* Fills opts with the defaults (no Kahan, fixed gamma, FP32 input). */
void bf_default_opts(bf_opts* opts);

/* Order rule: N = ceil(1 / (gamma sigma_r)^2) with gamma = pi/(2T), from the
   Gaussian-approximation theorem (Eq. approx2: cos^N(gamma t) ~
   exp(-N gamma^2 t^2 / 2)) and the O(T^2/sigma^2) order threshold at the end
   of Sec. 3. Returns -1 if sigma_r <= 0 or T <= 0. Host only. */
int bf_resolve_N(float sigma_r, float T);

/* Interpolating coefficients of q_N's shift expansion (Eq. def applied to
   cos^N): writes a_k for the harmonics k = N mod 2, N mod 2 + 2, ..., N into
   a[0 .. K-1] (K = N/2 + 1, in that order) in FP64 and returns K; returns -1
   if N < 0, N > BF_N_MAX or cap < K. Host only, no GPU needed. */
int bf_coeffs(int N, double* a, int cap);

/* Number of harmonics kept for order N, half-width r and opts->trunc_tol
   (the rule described at bf_opts.trunc_tol; N/2 + 1 when trunc_tol = 0).
   Returns -1 on bad arguments. Host only. */
int bf_trunc_harmonics(int N, int r, float trunc_tol);

/* gamma used for (sigma_r, T, N, gamma_mode); N must already be resolved.
   Returns a negative value on bad arguments. Host only. */
double bf_gamma(float sigma_r, float T, int N, int gamma_mode);

/* Bytes of the `saved` buffer bf_forward fills for bf_backward: H * W
   quads of 4 floats, (f - T/2, 1 / den, out - T/2, dnum_s - out * dden_s),
   where dnum_s, dden_s are num and den of Eq. filter2 differentiated with
   respect to the centre value f(x) (divided by gamma).
   - Layout: pixel (y, x)'s quad sits at index ((y + (x mod 128)) mod H) * W
     + x when H >= 128, and at y * W + x below; [B][...] per image for the
     3-D calls. The rows are sheared so that the anti-diagonals the filter
     sweeps (one pixel per lane, row + column fixed across a warp) are
     contiguous.
   - f and out are stored shifted by the range midpoint T/2: the filter
     commutes with a constant shift of the range, and the adjoint, run on
     the shifted values, rounds against terms half as large (out = quad.z +
     T/2 up to one rounding).
   The adjoint reads one 16-byte quad per pixel instead of several planes.
   The buffer must be 16-byte aligned. */
size_t bf_saved_bytes(int H, int W);

/* Index, in quads, of pixel (y, x)'s quad in the saved buffer of an H x W
   image (the layout above; add b * H * W for image b of a 3-D call). Host
   only; (size_t)-1 when H or W < 1 or (y, x) lies outside the image. */
size_t bf_saved_index(int y, int x, int H, int W);

/*
 * Forward filter (Algorithm 2 with M = 1, box window, range kernel q_N).
 *   img     device, H x W, dtype opts->in_dtype (FP32 or BF16).
 *   r       half-width, 0..BF_R_MAX.   sigma_r > 0 when N <= 0 or in
 *           BF_GAMMA_FROM_SIGMA mode.   T > 0.   N <= 0: derived from sigma_r.
 *   out     device, H x W FP32. Must not alias img.
 *   opts    NULL = defaults.
 *   saved   NULL, or device buffer of bf_saved_bytes(H, W) (16-byte aligned),
 *           written for bf_backward. When N > 43 (or opts->kahan with N > 23) the
 *           harmonics run in chunks that accumulate in this buffer; without
 *           it such calls take a slower single-pass kernel.
 * Errors: BF_ERR_INVALID_ARG (null pointer, H/W < 1, r < 0, T <= 0, bad
 * sigma_r, bad opts), BF_ERR_UNSUPPORTED (N > BF_N_MAX, r > BF_R_MAX),
 * BF_ERR_CUDA.
 */
bf_status bf_forward(const void* img, int H, int W, int r, float sigma_r, float T, int N,
                     float* out, const bf_opts* opts, void* saved, void* stream);

/* Workspace bytes bf_backward needs for the same (H, W, r, sigma_r, T, N,
   opts): the per-CTA dL/dsigma_r partial sums and, when the harmonics of q_N
   run in several chunks (N > 43), two H x W float accumulators. 0 on bad
   arguments. */
size_t bf_backward_workspace_bytes(int H, int W, int r, float sigma_r, float T, int N,
                                   const bf_opts* opts);

/*
 * Adjoint of bf_forward for L with dL/dout = grad_out (derived from Eq.
 * filter2; the box window is symmetric, so the adjoint is again a moving-sum
 * pass over a stack recomputed from img, never stored).
 *   img, out      the forward's input and output (device; the adjoint
 *                 reads both through the saved quads, so they are only
 *                 checked for NULL).
 *   grad_out      device H x W FP32.
 *   saved         the forward's saved buffer (device, bf_saved_bytes).
 *   grad_img      device H x W FP32 output, or NULL.
 *   grad_sigma    device pointer to ONE float receiving dL/dsigma_r, or NULL
 *                 (0 in BF_GAMMA_FIXED mode).
 *   workspace     device, >= bf_backward_workspace_bytes; may be NULL only if
 *                 grad_sigma is NULL (or gamma is fixed) and N <= 43.
 * Same parameters (r, sigma_r, T, N, opts) as the forward call.
 */
bf_status bf_backward(const void* img, const float* out, const float* grad_out,
                      const void* saved, int H, int W, int r, float sigma_r, float T, int N,
                      float* grad_img, float* grad_sigma, void* workspace, size_t ws_bytes,
                      const bf_opts* opts, void* stream);

/*
 * bf_forward over B images of equal size in one launch: img, out are
 * contiguous [B, H, W] arrays (dtype as in bf_forward), saved (NULL or
 * B * bf_saved_bytes(H, W)) is [B][H][W] quads. Same parameters, errors and
 * precondition as bf_forward, for every image.
 */
bf_status bf_forward3d(const void* img, int B, int H, int W, int r, float sigma_r, float T, int N,
                       float* out, const bf_opts* opts, void* saved, void* stream);

/* Workspace bytes of bf_backward3d (B images of H x W). */
size_t bf_backward3d_workspace_bytes(int B, int H, int W, int r, float sigma_r, float T, int N,
                                     const bf_opts* opts);

/*
 * bf_backward over B images in one launch ([B, H, W] arrays, saved as written
 * by bf_forward3d). grad_sigma receives ONE float: dL/dsigma_r summed over
 * the B images. Same errors as bf_backward.
 */
bf_status bf_backward3d(const void* img, const float* out, const float* grad_out,
                        const void* saved, int B, int H, int W, int r, float sigma_r, float T,
                        int N, float* grad_img, float* grad_sigma, void* workspace,
                        size_t ws_bytes, const bf_opts* opts, void* stream);

/* Capacity of the fixed scratch array bf_backward_noalloc uses: this many
   per-CTA partial sums (64 KiB per device). */
#define BF_NOALLOC_MAX_PARTIALS 16384

/*
 * bf_backward for callers that cannot allocate device memory. The paper has
 * no counterpart; this is a deployment variant of the adjoint above.
 *
 * Who needs it: code that may not call cudaMalloc, e.g. a plugin inside a
 * host application that owns all GPU memory through its own pool and forbids
 * libraries from allocating, or a latency-critical loop that cannot afford
 * an allocation's implicit device synchronisation. Such a caller still owns
 * and passes every input and output, but no workspace: the per-CTA
 * dL/dsigma_r partial sums go to a fixed array compiled into the library
 * (BF_NOALLOC_MAX_PARTIALS floats), which every GPU that loads the library
 * holds until the process exits.
 *
 * Arguments and results are those of bf_backward without workspace/ws_bytes.
 * Errors: as bf_backward, plus BF_ERR_UNSUPPORTED, checked before any launch,
 * when the call needs more scratch than the array holds, i.e. when
 * bf_backward_workspace_bytes(H, W, r, sigma_r, T, N, opts) exceeds
 * BF_NOALLOC_MAX_PARTIALS * sizeof(float) (64 KiB): one float per CTA of the
 * launch grid, plus, when the harmonics run in chunks (N > 43), two H x W
 * float accumulators at a 256-byte aligned offset; so chunked calls are
 * accepted only for small images (about 90 x 90 and below).
 *
 * Set-up: every call looks up the array's device address on the current
 * device (cudaGetSymbolAddress, a host-side lookup), so a cudaDeviceReset
 * does not leave it stale. The first call on a device may load the library's
 * device code there; make it before any stream capture. The entry point
 * allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *
 * Sharing: every call on a device uses the same array, which keeps the last
 * call's contents. No slot needs to start at zero (each call writes every
 * slot it reads), but calls whose executions overlap on the GPU (e.g. on two
 * streams at once) race on the array: serialise them.
 */
bf_status bf_backward_noalloc(const void* img, const float* out, const float* grad_out,
                              const void* saved, int H, int W, int r, float sigma_r, float T,
                              int N, float* grad_img, float* grad_sigma, const bf_opts* opts,
                              void* stream);

/*
 * Algorithm 2 with a shiftable spatial kernel as well (Sec. 2), and
 * Algorithm 1 as its case N = 0: the neighbourhood filter
 *   out(x) = sum_y phi(y - x) w(f(y) - f(x)) f(y) / sum_y phi(y - x) w(f(y) - f(x))
 * over the (2r+1)^2 window (truncated at the image border), with the
 * separable spatial kernel phi(d) = q_M(d1) q_M(d2) of Sec. 3, q_M(d) =
 * cos^M(pi d / (2r + 1)) (q_M on [-(r + 1/2), r + 1/2], so the window lies
 * inside its support), and the range kernel w = q_N of bf_forward (N = 0: no
 * range kernel, i.e. the linear spatial filter of Eq. filter1 / Algorithm 1;
 * N < 0: derived from sigma_r like bf_forward's N <= 0). Computed from
 * (M+1)^2 (N+1) shiftable basis functions by moving sums, in one fused pass.
 *   img, out  device H x W FP32 (out must not alias img).
 *   M         1..4, 6 or 8 when N = 0; 1 or 2 when 1 <= N <= 4.
 *   r         0..56.
 *   opts      NULL or defaults; tile_h (rows per band) is honoured, else the
 *             band height fills one wave of the launched kernel's resident
 *             CTAs; BF16 input, Kahan, trunc_tol and BF_GAMMA_FROM_SIGMA give
 *             BF_ERR_UNSUPPORTED.
 *   saved     NULL, or device buffer of bf_saved_bytes(H, W) (16-byte aligned)
 *             receiving the quads (f, 1/den, out, dnum_s - out dden_s),
 *             not shifted by T/2, in the sheared layout of bf_forward's, for
 *             bf_spatial_backward.
 * r = 0 (a 1 x 1 window) is exact: out = img, saved quads (f, 1, f, 0).
 * Errors: BF_ERR_INVALID_ARG, BF_ERR_UNSUPPORTED (other M, N, r; H * W >= 2^31,
 * checked first), BF_ERR_CUDA.
 */
bf_status bf_spatial_forward(const void* img, int H, int W, int r, int M, float sigma_r, float T,
                             int N, float* out, const bf_opts* opts, void* saved, void* stream);

/*
 * Adjoint of bf_spatial_forward for L with dL/dout = grad_out: dL/dimg,
 * derived from Eq. filter2 with the spatial kernel; the window and q_M x q_M
 * are symmetric, so every neighbour term is again a moving sum centred on
 * the pixel whose gradient is formed (the same fused pass on the planes
 * alpha E_c, beta E_c, alpha = g / den, beta = -alpha out).
 *   grad_out  device H x W FP32.
 *   saved     the quads bf_spatial_forward wrote (device, bf_saved_bytes(H, W)).
 *   grad_img  device H x W FP32 output.
 * Same H, W, r, M, sigma_r, T, N, opts as the forward. The range frequency is
 * fixed (gamma = pi / (2T)), so dL/dsigma_r is 0 and not computed. Runs as one
 * or (with 18 or more combos) two launches on `stream`; grad_img must not
 * alias grad_out or saved. r = 0: grad_img = grad_out.
 * Errors: as bf_spatial_forward.
 */
bf_status bf_spatial_backward(const float* grad_out, const void* saved, int H, int W, int r, int M,
                              float sigma_r, float T, int N, float* grad_img, const bf_opts* opts,
                              void* stream);

/* Order of the polynomial range kernel p_N for a target Gaussian width:
   N = ceil(T^2 / (2 sigma_r^2)), from Eq. approx1 (p_N(t / sqrt N) ->
   exp(-t^2 / T^2), so p_N(t) ~ exp(-N t^2 / T^2)). -1 on bad arguments.
   Host only. */
int bf_poly_resolve_N(float sigma_r, float T);

/*
 * Bilateral filter with the box spatial kernel and the polynomial range
 * kernel p_N(t) = (1 - t^2 / T^2)^N of Sec. 3 (order of shiftability 2N+1),
 * by moving sums of the 2N+2 power images of u = f / T - 1/2 (Algorithm 2
 * with a polynomial basis).
 *   img, out  device H x W FP32 (out must not alias img). Precondition as
 *             for bf_forward: values in [0, T].
 *   N         1..8; N <= 0 derives it from sigma_r (bf_poly_resolve_N).
 *   r         0..56.
 *   opts      NULL or defaults (tile_h honoured); BF16 input, Kahan,
 *             trunc_tol or BF_GAMMA_FROM_SIGMA give BF_ERR_UNSUPPORTED.
 *   saved     NULL, or device buffer of bf_saved_bytes(H, W) (16-byte aligned)
 *             receiving the quads (f, 1/den, out, dnum_s - out dden_s),
 *             not shifted by T/2, in the sheared layout of bf_forward's, for
 *             bf_poly_backward.
 * r = 0 (a 1 x 1 window) is exact: out = img, saved quads (f, 1, f, 0), and
 * bf_poly_backward returns grad_out.
 * Errors: BF_ERR_INVALID_ARG, BF_ERR_UNSUPPORTED (N > 8, r > 56; H * W >=
 * 2^31, checked first), BF_ERR_CUDA.
 */
bf_status bf_poly_forward(const void* img, int H, int W, int r, float sigma_r, float T, int N,
                          float* out, const bf_opts* opts, void* saved, void* stream);

/*
 * Adjoint of bf_poly_forward for L with dL/dout = grad_out: dL/dimg (derived
 * from Eq. filter2; the window and p_N are symmetric, so the neighbour terms
 * are moving sums of alpha u^m and beta u^m, alpha = g / den, beta = -alpha out).
 *   grad_out  device H x W FP32.
 *   saved     the quads bf_poly_forward wrote (device, bf_saved_bytes(H, W)).
 *   grad_img  device H x W FP32 output.
 * Same H, W, r, sigma_r, T, N, opts as the forward. Errors: as bf_poly_forward.
 */
bf_status bf_poly_backward(const float* grad_out, const void* saved, int H, int W, int r,
                           float sigma_r, float T, int N, float* grad_img, const bf_opts* opts,
                           void* stream);

/* Workspace bytes bf_batch needs for n descriptors (device tile table). */
size_t bf_batch_workspace_bytes(const bf_desc* descs, int n, const bf_opts* opts);

/*
 * Filters n images of uneven sizes, each with its own r, sigma_r, N, in
 * persistent launches: CTAs pull tiles from device work counters over a tile
 * table held in `workspace`. The images are grouped by kernel (three groups:
 * 128-thread strips whose harmonics fit one chunk of at most 4 pairs, which
 * run the compile-time-specialised kernels at three CTAs per SM; the other
 * 128-thread strips; 256-thread strips for r > 40), one launch per group.
 * descs is a HOST array; each image is validated like bf_forward;
 * opts->tile_w, if set, must be 128 or 256 (else BF_ERR_UNSUPPORTED).
 * Equivalent to bf_batch_prepare followed by bf_batch_launch.
 */
bf_status bf_batch(const bf_desc* descs, int n, const bf_opts* opts, void* workspace,
                   size_t ws_bytes, void* stream);

/* Validates descs and uploads the tile table into workspace (stream-ordered
   copy from host memory). */
bf_status bf_batch_prepare(const bf_desc* descs, int n, const bf_opts* opts, void* workspace,
                           size_t ws_bytes, void* stream);

/* Launches the persistent batch kernels over a table bf_batch_prepare wrote
   into workspace: a memset of the work counters and one kernel per group
   (the Kahan path: one kernel), nothing else, so it can be captured into a
   CUDA graph and replayed. opts must
   carry the same kahan / in_dtype as the prepare call. On the plain (non-
   Kahan) path a table without the tag bf_batch_prepare writes (a workspace
   never prepared, or overwritten) launches no work: outputs stay untouched. */
bf_status bf_batch_launch(void* workspace, size_t ws_bytes, const bf_opts* opts, void* stream);

/* Minimum and maximum of an H x W device image (dtype BF_F32 or BF_BF16), for
   checking the filters' precondition max f - min f <= T (Sec. 3: the range
   kernels are valid kernels on [-T, T] only). Writes the two floats (min,
   max) to the DEVICE pointer minmax (8-byte aligned), asynchronously on
   `stream`. NaN values are not supported. Paper counterpart: the a-priori
   bound on the data that Sec. 3 assumes. Errors: BF_ERR_INVALID_ARG,
   BF_ERR_CUDA. */
bf_status bf_check_range(const void* img, int H, int W, int in_dtype, float* minmax, void* stream);

/* Static message for a status code. */
const char* bf_status_string(bf_status s);

/* cudaError_t code of the last BF_ERR_CUDA on this host thread (0 if none);
   returns BF_OK, or BF_ERR_INVALID_ARG if code is NULL. */
bf_status bf_last_cuda_error(int* code);

#ifdef __cplusplus
}
#endif

#endif /* BF_H_ */
