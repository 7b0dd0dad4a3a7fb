// Launch shape of the strip-engine variants (spatial kernel, polynomial range
// kernel): band height from the launched kernel's occupancy.
#pragma once

#include <stddef.h>

namespace bf {

// Rows per band so that a grid of gx strips is one wave of the CTAs of `kern`
// (threads per CTA, dynamic shared bytes) resident per SM, at most max_per_sm
// of them (0: no cap); at least 32 rows.
int wave_band_rows(const void* kern, int threads, size_t smem, int H, int gx, int max_per_sm);

}  // namespace bf
