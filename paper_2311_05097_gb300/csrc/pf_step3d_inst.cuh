// Instantiation and dispatch of the 3D step kernel for one precision policy.
#pragma once

#include "pf_internal.h"
#include "pf_kernels3d.cuh"

namespace pf {

template <class P, int TX, int TY, bool MOVING, int MODE>
static bool run3d(int grid, cudaStream_t s, const StepArgs &a, int *occ)
{
    auto kern = k_step3d<P, TX, TY, ZCHUNK3D, MOVING, MODE>;
    if (occ) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, TX * TY, 0) != cudaSuccess) n = 0;
        *occ = n;
        return true;
    }
    kern<<<grid, TX * TY, 0, s>>>(a);
    count_launches(1);
    return true;
}

template <class P, int TX, int TY>
static bool dispatch3d(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s,
                       const StepArgs &a, int *occ)
{
    if (tx != TX || ty != TY) return false;
    if (mode == MODE_MACROS)
        return moving ? run3d<P, TX, TY, true, MODE_MACROS>(grid, s, a, occ)
                      : run3d<P, TX, TY, false, MODE_MACROS>(grid, s, a, occ);
    return moving ? run3d<P, TX, TY, true, MODE_STEP>(grid, s, a, occ)
                  : run3d<P, TX, TY, false, MODE_STEP>(grid, s, a, occ);
}

}  // namespace pf
