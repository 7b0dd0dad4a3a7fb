// Launch shape of the strip-engine variants (spatial kernel, polynomial range
// kernel): band height from the launched kernel's occupancy.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace bf {

// Rows per band so that a grid of gx strips is one wave of the CTAs of `kern`
// (threads per CTA, dynamic shared bytes) resident per SM; at least 32 rows.
int wave_band_rows(const void* kern, int threads, size_t smem, int H, int gx);

// r = 0 (a 1 x 1 window) for the variant filters, whose kernels are 1 with
// slope 0 at the origin: out = img (H x W FP32 values) and, if sv is given,
// the saved quads (f, 1/den = 1, out = f, X = 0) at quad_index. Enqueued on s.
cudaError_t unit_window(const float* img, float* out, float4* sv, int H, int W, cudaStream_t s);

// Tag bf_batch_prepare writes into a strip-engine batch table; the persistent
// batch kernels do no work on a table without it (a workspace that was never
// prepared, or was overwritten).
constexpr int SYS_BATCH_MAGIC = 0x42465359;  // "BFSY"

}  // namespace bf
