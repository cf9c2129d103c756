// Instantiation and dispatch of the 3D step kernel for one precision policy.
#pragma once

#include "pf_internal.h"
#include "pf_kernels3d.cuh"

namespace pf {

template <class P, int TX, int TY, bool MOVING, int MODE, bool EXT, bool UNIT = false>
static bool run3d(int grid, cudaStream_t s, const StepArgs &a, int *occ)
{
    auto kern = k_step3d<P, TX, TY, ZCHUNK3D, MOVING, MODE, EXT, UNIT>;
    // particles with their own contact angle: the W and V plane rings (5
    // planes of the tile + 2 frame each) in dynamic shared memory
    const int dyn = (MOVING && a.wv) ? (int)(2 * 5 * (TX + 4) * (TY + 4) * sizeof(typename P::real)) : 0;
    if (dyn && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess)
        return false;
    if (occ) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, TX * TY, dyn) != cudaSuccess) n = 0;
        *occ = n;
        return true;
    }
    kern<<<grid, TX * TY, dyn, s>>>(a);
    count_launches(1);
    return true;
}

template <class P, int TX, int TY, bool EXT>
static bool dispatch3d_ext(bool moving, bool unit, int mode, int grid, cudaStream_t s, const StepArgs &a, int *occ)
{
    if (mode == MODE_MACROS)
        return moving ? run3d<P, TX, TY, true, MODE_MACROS, EXT>(grid, s, a, occ)
                      : run3d<P, TX, TY, false, MODE_MACROS, EXT>(grid, s, a, occ);
    if constexpr (sizeof(typename P::real) == 4) {
        // unit rates (FP32 arithmetic): the specialised collisions
        if (unit && !moving) return run3d<P, TX, TY, false, MODE_STEP, EXT, true>(grid, s, a, occ);
    }
    return moving ? run3d<P, TX, TY, true, MODE_STEP, EXT>(grid, s, a, occ)
                  : run3d<P, TX, TY, false, MODE_STEP, EXT>(grid, s, a, occ);
}

// mode may carry MODE_EXT: a domain of the launch has walls
template <class P, int TX, int TY>
static bool dispatch3d(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s,
                       const StepArgs &a, int *occ)
{
    if (tx != TX || ty != TY) return false;
    const bool ext = (mode & MODE_EXT) != 0, unit = (mode & MODE_UNIT) != 0;
    mode &= ~(MODE_EXT | MODE_CAC | MODE_UNIT);
    return ext ? dispatch3d_ext<P, TX, TY, true>(moving, unit, mode, grid, s, a, occ)
               : dispatch3d_ext<P, TX, TY, false>(moving, unit, mode, grid, s, a, occ);
}

}  // namespace pf
