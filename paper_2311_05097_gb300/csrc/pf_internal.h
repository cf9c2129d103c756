// Internal declarations shared by the libpf translation units.
#pragma once

#include <cuda_runtime.h>

#include "pf_common.cuh"

namespace pf {

// record the thread-local error message returned by pf_last_error; returns code
int set_error(int code, const char *msg);

// kernel-launch accounting (pf_launch_count)
void count_launches(long long n);

// supported tile shapes of the step kernels
struct TileShape {
    int tx, ty;
};

// 2D fused step (mode 0) or macroscopic-field pass (mode 1).  Returns false
// when the (precision, tile, moving, mode) combination is not compiled.
bool launch_step2d(int prec, int tx, int ty, bool moving, int mode, int grid, cudaStream_t s,
                   const StepArgs &a);
// query of the resident CTAs per SM of one 2D configuration (0 if unsupported)
int occupancy_step2d(int prec, int tx, int ty, bool moving, int mode);
bool launch_step2d_p64(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s, const StepArgs &a, int *occ);
bool launch_step2d_p32(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s, const StepArgs &a, int *occ);
bool launch_step2d_mixh(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s, const StepArgs &a, int *occ);
bool launch_step2d_mixb(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s, const StepArgs &a, int *occ);

// 3D: one CTA marches through ZCHUNK3D planes in z
constexpr int ZCHUNK3D = 32;
bool launch_step3d(int prec, int tx, int ty, bool moving, int mode, int grid, cudaStream_t s,
                   const StepArgs &a);
int occupancy_step3d(int prec, int tx, int ty, bool moving, int mode);
void tile_shape3d(int prec, int *tx, int *ty);
bool launch_step3d_p64(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s, const StepArgs &a, int *occ);
bool launch_step3d_p32(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s, const StepArgs &a, int *occ);
bool launch_step3d_mixh(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s, const StepArgs &a, int *occ);
bool launch_step3d_mixb(int tx, int ty, bool moving, int mode, int grid, cudaStream_t s, const StepArgs &a, int *occ);

void launch_init(int prec, const DomainDev &Dm, int *flags, const double *phi0, const double *phi, const double *u,
                 const double *Pin, double *tmp, const ParticleDev *parts, int np, int wv, cudaStream_t s);
int diag_blocks();
void launch_diag(const DomainDev &Dm, double *partial, double *out, int wv, cudaStream_t s);
// near / far tile lists of a particle domain (single-cell / two-cells step)
void launch_split_tiles(const StepArgs &a, int tx, int ty, unsigned char *sel, cudaStream_t s);
// interface normal (dim planes of N) from Dm.macro's phi plane
void launch_normal(const DomainDev &Dm, double *n, cudaStream_t s);
void launch_particle_update(ParticleDev *parts, int np, const double *partials, int ntiles,
                            const DevParams &p, double *frep, int nx, int ny, int nz, int wall_y,
                            const unsigned char *sel, cudaStream_t s);

}  // namespace pf
