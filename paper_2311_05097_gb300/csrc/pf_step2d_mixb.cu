#include "pf_step2d_inst.cuh"

namespace pf {
bool launch_step2d_mixb(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s,
                      const StepArgs &a, int *occ)
{
    return dispatch2d<PMixB>(tx, ty, moving, mode, grid, s, a, occ);
}
}  // namespace pf
