// launch.cuh -- grid sizing of the grid-stride kernels.
#pragma once

#include "common.cuh"

namespace qed {

int sm_count();

// CTAs of `threads` for a grid-stride kernel over `items` work items: at most
// as many as stay resident on the GPU at once (computed once per kernel), since
// a CTA left for a second wave only lengthens the launch
template <auto Kernel>
int resident_grid(int threads, size_t dyn, int64_t items)
{
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, Kernel, threads, dyn);
        if (per_sm <= 0) per_sm = 1;
    }
    const int64_t want = (items + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count() * per_sm;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace qed
