// Grid-stride walk over the cells of a rows x per_row array that keeps the
// row and column up to date by addition: one integer division per thread at
// the start instead of a 64-bit division per cell.
#pragma once

#include <cstdint>

namespace ts {

struct Walk {
    int64_t i, y, x;
    int64_t stride, dy, dx, per_row;

    __device__ __forceinline__ Walk(int64_t per_row_, int64_t start, int64_t stride_)
        : i(start), stride(stride_), per_row(per_row_)
    {
        y = start / per_row;
        x = start - y * per_row;
        dy = stride / per_row;
        dx = stride - dy * per_row;
    }

    __device__ __forceinline__ void next()
    {
        i += stride;
        x += dx;
        y += dy;
        if (x >= per_row) {
            x -= per_row;
            ++y;
        }
    }
};

}  // namespace ts
