// Instantiation and dispatch of the 2D step kernel for one precision policy.
// Included by one translation unit per policy (parallel compilation).
#pragma once

#include "pf_internal.h"
#include "pf_kernels2d.cuh"
#include "pf_kernels2d_pair.cuh"
#include "pf_kernels2d_stage.cuh"
#include "pf_kernels2d_strip.cuh"

namespace pf {

template <class P, int TX, int TY, bool MOVING, int MODE, bool EXT>
static bool run2d(int grid, cudaStream_t s, const StepArgs &a, int *occ)
{
    auto kern = k_step2d<P, TX, TY, MOVING, MODE, EXT>;
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

template <class P, int TX, int TYP, bool CAC, bool MU0 = false>
static bool run2d_pair(int grid, cudaStream_t s, const StepArgs &a, int *occ)
{
    auto kern = k_step2d_pair<P, TX, TYP, CAC, MU0>;
    if (occ) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, TX * TYP, 0) != cudaSuccess) n = 0;
        *occ = n;
        return true;
    }
    kern<<<grid, TX * TYP, 0, s>>>(a);
    count_launches(1);
    return true;
}

// two cells per thread: tiles of tx x ty cells on tx x ty/2 threads
template <class P>
static bool dispatch2d_pair(int tx, int ty, bool moving, bool cac, bool mu0, int grid, cudaStream_t s,
                            const StepArgs &a, int *occ)
{
    if constexpr (P::id == 0) {
        return false;  // FP64 has no packed arithmetic
    } else {
        // far tiles of a particle domain: 32 x 16, Cahn-Hilliard
        if (mu0) return tx == 32 && ty == 16 && !cac && run2d_pair<P, 32, 8, false, true>(grid, s, a, occ);
        if (moving) return false;
        if (tx == 32 && ty == 16)
            return cac ? run2d_pair<P, 32, 8, true>(grid, s, a, occ) : run2d_pair<P, 32, 8, false>(grid, s, a, occ);
        if (tx == 64 && ty == 8)
            return cac ? run2d_pair<P, 64, 4, true>(grid, s, a, occ) : run2d_pair<P, 64, 4, false>(grid, s, a, occ);
        if (tx == 32 && ty == 32)
            return cac ? run2d_pair<P, 32, 16, true>(grid, s, a, occ) : run2d_pair<P, 32, 16, false>(grid, s, a, occ);
        return false;
    }
}

template <class P, int TX, int TYP>
static bool run2d_stage(int grid, cudaStream_t s, const StepArgs &a, int *occ)
{
    auto kern = k_step2d_stage<P, TX, TYP>;
    const int dyn = StageLayout<P, TX, 2 * TYP>::BYTES;
    static bool attr = false;  // set once per instantiation (process-wide, any device)
    if (!attr) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess) return false;
        attr = true;
    }
    if (occ) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, TX * TYP, dyn) != cudaSuccess) n = 0;
        *occ = n;
        return true;
    }
    kern<<<grid, TX * TYP, dyn, s>>>(a);
    count_launches(1);
    return true;
}

// two cells per thread, inputs staged by bulk copies
template <class P>
static bool dispatch2d_stage(int tx, int ty, bool moving, int grid, cudaStream_t s, const StepArgs &a, int *occ)
{
    if constexpr (P::id == 0) {
        return false;
    } else {
        if (moving) return false;
        if (tx == 32 && ty == 16) return run2d_stage<P, 32, 8>(grid, s, a, occ);
        return false;
    }
}

template <class P, int B, bool CAC, bool UNIT, bool WALL>
static bool run2d_strip(int grid, cudaStream_t s, const StepArgs &a, int *occ)
{
    auto kern = k_step2d_strip<P, B, CAC, UNIT, WALL>;
    const int dyn = StripLayout<P, B>::BYTES;
    static bool attr = false;  // set once per instantiation (process-wide, any device)
    if (!attr) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess) return false;
        attr = true;
    }
    if (occ) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 32 * B, dyn) != cudaSuccess) n = 0;
        *occ = n;
        return true;
    }
    kern<<<grid, 32 * B, dyn, s>>>(a);
    count_launches(1);
    return true;
}

template <class P, bool WALL>
static bool dispatch2d_strip_w(bool cac, bool unit, int grid, cudaStream_t s, const StepArgs &a, int *occ)
{
    constexpr int B = strip_band<P>();
    if (cac) return run2d_strip<P, B, true, false, WALL>(grid, s, a, occ);
    return unit ? run2d_strip<P, B, false, true, WALL>(grid, s, a, occ)
                : run2d_strip<P, B, false, false, WALL>(grid, s, a, occ);
}

// strips marched in y (tile_x = strip width, tile_y = segment rows: any), and
// the ghost-column pass it needs (grid = number of domains)
template <class P>
static bool dispatch2d_strip(int tx, bool moving, bool cac, bool unit, bool wall, bool fill, int grid,
                             cudaStream_t s, const StepArgs &a, int *occ)
{
    if constexpr (P::id == 0) {
        return false;
    } else {
        if (fill) {
            if (occ) {
                *occ = 1;
                return true;
            }
            k_fill_ghosts<P><<<dim3(64, grid), 256, 0, s>>>(a.doms, a.par);
            count_launches(1);
            return true;
        }
        if (moving || tx != STRIP_SW) return false;
        return wall ? dispatch2d_strip_w<P, true>(cac, unit, grid, s, a, occ)
                    : dispatch2d_strip_w<P, false>(cac, unit, grid, s, a, occ);
    }
}

template <class P, bool EXT>
static bool dispatch2d_single(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s,
                              const StepArgs &a, int *occ)
{
    if (mode == MODE_MACROS) {
        if (tx == 32 && ty == 8)
            return moving ? run2d<P, 32, 8, true, MODE_MACROS, EXT>(grid, s, a, occ)
                          : run2d<P, 32, 8, false, MODE_MACROS, EXT>(grid, s, a, occ);
        return false;
    }
    if (tx == 32 && ty == 8)
        return moving ? run2d<P, 32, 8, true, MODE_STEP, EXT>(grid, s, a, occ)
                      : run2d<P, 32, 8, false, MODE_STEP, EXT>(grid, s, a, occ);
    if (tx == 64 && ty == 4)
        return moving ? run2d<P, 64, 4, true, MODE_STEP, EXT>(grid, s, a, occ)
                      : run2d<P, 64, 4, false, MODE_STEP, EXT>(grid, s, a, occ);
    if (tx == 32 && ty == 16)
        return moving ? run2d<P, 32, 16, true, MODE_STEP, EXT>(grid, s, a, occ)
                      : run2d<P, 32, 16, false, MODE_STEP, EXT>(grid, s, a, occ);
    return false;
}

template <class P>
static bool dispatch2d(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s,
                       const StepArgs &a, int *occ)
{
    const bool ext = (mode & MODE_EXT) != 0, cac = (mode & MODE_CAC) != 0, mu0 = (mode & MODE_MU0) != 0;
    const bool wall = (mode & MODE_WALL) != 0, unit = (mode & MODE_UNIT) != 0;
    mode &= ~(MODE_EXT | MODE_CAC | MODE_MU0 | MODE_WALL | MODE_UNIT);
    // the tiled two-cells-per-thread kernels have no wall handling: refuse walled launches
    if (mode == MODE_STEP_PAIR) return !wall && dispatch2d_pair<P>(tx, ty, moving, cac, mu0, grid, s, a, occ);
    if (mode == MODE_STEP_STAGE)
        return !wall && !ext && !cac && dispatch2d_stage<P>(tx, ty, moving, grid, s, a, occ);
    if (mode == MODE_STEP_STRIP || mode == MODE_FILL_GHOSTS)
        return dispatch2d_strip<P>(tx, moving, cac, unit, wall, mode == MODE_FILL_GHOSTS, grid, s, a, occ);
    return ext ? dispatch2d_single<P, true>(tx, ty, moving, mode, grid, s, a, occ)
               : dispatch2d_single<P, false>(tx, ty, moving, mode, grid, s, a, occ);
}

}  // namespace pf
