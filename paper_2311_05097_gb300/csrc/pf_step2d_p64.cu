#include "pf_step2d_inst.cuh"

namespace pf {
bool launch_step2d_p64(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s,
                      const StepArgs &a, int *occ)
{
    return dispatch2d<P64>(tx, ty, moving, mode, grid, s, a, occ);
}
}  // namespace pf
