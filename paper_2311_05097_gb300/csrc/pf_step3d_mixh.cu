#include "pf_step3d_inst.cuh"

namespace pf {
bool launch_step3d_mixh(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s,
                      const StepArgs &a, int *occ)
{
    return dispatch3d<PMixH, 32, 8>(tx, ty, moving, mode, grid, s, a, occ);
}
}  // namespace pf
