// 64-bit form of quad_index (bf_internal.cuh): the index of pixel (row, col)'s
// quad in the saved buffer of an H x W image, rows sheared by (col mod 128)
// and wrapped at H for H >= 128, row-major below. The skewed-strip engine's
// launches are limited to 32-bit element offsets and use quad_index; the
// single-pass kernels (which serve larger images), the unit-window quads and
// the host's bf_saved_index use this form, which holds past 2^31 pixels.
#pragma once
#include <cstddef>

namespace bf {

__host__ __device__ __forceinline__ size_t quad_index64(int row, int col, int H, int W) {
    long long rr = (long long)row + (col & (H >= 128 ? 127 : 0));
    if (rr >= H) rr -= H;
    return (size_t)rr * (size_t)W + (size_t)col;
}

}  // namespace bf
