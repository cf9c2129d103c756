// 3D fused time step: D3Q7 order-parameter lattice and D3Q19 flow lattice
// (the 3D extension of Sec. 3; see the readings of the 3D lattices in the
// oracle), pull streaming, Hermite-moment MRT collision.
//
// A CTA owns a TX x TY column of cells and marches through ZC planes in z.
// Shared-memory rings hold the planes the stencils need:
//   phi, phi0       planes z-2 .. z+2 on the tile + 2 frame (ring of 5),
//   mu_phi          planes z-1 .. z+1 on the tile + 1 frame (ring of 4),
//   T = S u - u S   (antisymmetric: xy, xz, yz) of the previous step, planes
//                   z-1 .. z+1 on the tile + 1 frame (ring of 4).
// Each plane costs two barriers.  Halo re-reads hit L2; each cell's own
// populations are read once from DRAM.
#pragma once

#include "pf_common.cuh"

namespace pf {

// D3Q19 velocities: rest, 6 faces, 12 edges; D3Q7 uses the first 7.
__device__ constexpr int C19X[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__device__ constexpr int C19Y[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__device__ constexpr int C19Z[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
// opposite direction (pairs 1-2, 3-4, ..., 17-18)
__device__ __forceinline__ int opp19(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

template <class R>
__device__ __forceinline__ void from_hermite19(const R h[19], R f[19], R cs2);

// Hermite-moment MRT collision of one D3Q19 cell.  Raw moments m = M0 f with
// rows 1, c_a, c_a^2, c_x c_y, c_x c_z, c_y c_z, c_x c_y^2, c_x c_z^2,
// c_y c_x^2, c_y c_z^2, c_z c_x^2, c_z c_y^2, c_x^2 c_y^2, c_x^2 c_z^2,
// c_y^2 c_z^2; Hermite moments h = N_H m; relaxation in h; back by N_H^-1
// and M0^-1.
template <class R>
__device__ __forceinline__ void collide19(R f[19], const R heq[19], const R hF[19], const R S[19],
                                          R cs2)
{
    const R cs4 = cs2 * cs2;
    R m[19];
    m[0] = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8] + f[9] + f[10] + f[11] + f[12] +
           f[13] + f[14] + f[15] + f[16] + f[17] + f[18];
    m[1] = f[1] - f[2] + f[7] - f[8] + f[9] - f[10] + f[11] - f[12] + f[13] - f[14];
    m[2] = f[3] - f[4] + f[7] - f[8] - f[9] + f[10] + f[15] - f[16] + f[17] - f[18];
    m[3] = f[5] - f[6] + f[11] - f[12] - f[13] + f[14] + f[15] - f[16] - f[17] + f[18];
    const R exy = f[7] + f[8] + f[9] + f[10], exz = f[11] + f[12] + f[13] + f[14],
            eyz = f[15] + f[16] + f[17] + f[18];
    m[4] = f[1] + f[2] + exy + exz;
    m[5] = f[3] + f[4] + exy + eyz;
    m[6] = f[5] + f[6] + exz + eyz;
    m[7] = f[7] + f[8] - f[9] - f[10];
    m[8] = f[11] + f[12] - f[13] - f[14];
    m[9] = f[15] + f[16] - f[17] - f[18];
    m[10] = f[7] - f[8] + f[9] - f[10];    // c_x c_y^2
    m[11] = f[11] - f[12] + f[13] - f[14]; // c_x c_z^2
    m[12] = f[7] - f[8] - f[9] + f[10];    // c_y c_x^2
    m[13] = f[15] - f[16] + f[17] - f[18]; // c_y c_z^2
    m[14] = f[11] - f[12] - f[13] + f[14]; // c_z c_x^2
    m[15] = f[15] - f[16] - f[17] + f[18]; // c_z c_y^2
    m[16] = exy;
    m[17] = exz;
    m[18] = eyz;
    R h[19];
    h[0] = m[0];
    h[1] = m[1];
    h[2] = m[2];
    h[3] = m[3];
    h[4] = m[4] - cs2 * m[0];
    h[5] = m[5] - cs2 * m[0];
    h[6] = m[6] - cs2 * m[0];
    h[7] = m[7];
    h[8] = m[8];
    h[9] = m[9];
    h[10] = m[10] - cs2 * m[1];
    h[11] = m[11] - cs2 * m[1];
    h[12] = m[12] - cs2 * m[2];
    h[13] = m[13] - cs2 * m[2];
    h[14] = m[14] - cs2 * m[3];
    h[15] = m[15] - cs2 * m[3];
    h[16] = m[16] - cs2 * (m[4] + m[5]) + cs4 * m[0];
    h[17] = m[17] - cs2 * (m[4] + m[6]) + cs4 * m[0];
    h[18] = m[18] - cs2 * (m[5] + m[6]) + cs4 * m[0];
#pragma unroll
    for (int k = 0; k < 19; ++k)
        h[k] = h[k] - S[k] * (h[k] - heq[k]) + (R(1) - R(0.5) * S[k]) * hF[k];
    from_hermite19<R>(h, f, cs2);
}

// D3Q19 populations from Hermite moments: raw moments m = N_H^-1 h, then
// f = M0^-1 m.
template <class R>
__device__ __forceinline__ void from_hermite19(const R h[19], R f[19], R cs2)
{
    const R cs4 = cs2 * cs2;
    R m[19];
    m[0] = h[0];
    m[1] = h[1];
    m[2] = h[2];
    m[3] = h[3];
    m[4] = h[4] + cs2 * h[0];
    m[5] = h[5] + cs2 * h[0];
    m[6] = h[6] + cs2 * h[0];
    m[7] = h[7];
    m[8] = h[8];
    m[9] = h[9];
    m[10] = h[10] + cs2 * h[1];
    m[11] = h[11] + cs2 * h[1];
    m[12] = h[12] + cs2 * h[2];
    m[13] = h[13] + cs2 * h[2];
    m[14] = h[14] + cs2 * h[3];
    m[15] = h[15] + cs2 * h[3];
    m[16] = h[16] + cs2 * (h[4] + h[5]) + cs4 * h[0];
    m[17] = h[17] + cs2 * (h[4] + h[6]) + cs4 * h[0];
    m[18] = h[18] + cs2 * (h[5] + h[6]) + cs4 * h[0];
    const R hh = R(0.5), q = R(0.25);
    f[0] = m[0] - m[4] - m[5] - m[6] + m[16] + m[17] + m[18];
    f[1] = hh * (m[1] + m[4] - m[10] - m[11] - m[16] - m[17]);
    f[2] = hh * (-m[1] + m[4] + m[10] + m[11] - m[16] - m[17]);
    f[3] = hh * (m[2] + m[5] - m[12] - m[13] - m[16] - m[18]);
    f[4] = hh * (-m[2] + m[5] + m[12] + m[13] - m[16] - m[18]);
    f[5] = hh * (m[3] + m[6] - m[14] - m[15] - m[17] - m[18]);
    f[6] = hh * (-m[3] + m[6] + m[14] + m[15] - m[17] - m[18]);
    f[7] = q * (m[7] + m[10] + m[12] + m[16]);
    f[8] = q * (m[7] - m[10] - m[12] + m[16]);
    f[9] = q * (-m[7] + m[10] - m[12] + m[16]);
    f[10] = q * (-m[7] - m[10] + m[12] + m[16]);
    f[11] = q * (m[8] + m[11] + m[14] + m[17]);
    f[12] = q * (m[8] - m[11] - m[14] + m[17]);
    f[13] = q * (-m[8] + m[11] - m[14] + m[17]);
    f[14] = q * (-m[8] - m[11] + m[14] + m[17]);
    f[15] = q * (m[9] + m[13] + m[15] + m[18]);
    f[16] = q * (m[9] - m[13] - m[15] + m[18]);
    f[17] = q * (-m[9] + m[13] - m[15] + m[18]);
    f[18] = q * (-m[9] - m[13] + m[15] + m[18]);
}

// D3Q7 Hermite collision (rows 1, c_a, c_a^2 - cs^2).
template <class R>
__device__ __forceinline__ void collide7(R f[7], const R heq[7], const R hF[7], const R S[7], R cs2)
{
    R h[7];
    h[0] = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6];
    h[1] = f[1] - f[2];
    h[2] = f[3] - f[4];
    h[3] = f[5] - f[6];
    h[4] = f[1] + f[2] - cs2 * h[0];
    h[5] = f[3] + f[4] - cs2 * h[0];
    h[6] = f[5] + f[6] - cs2 * h[0];
#pragma unroll
    for (int k = 0; k < 7; ++k)
        h[k] = h[k] - S[k] * (h[k] - heq[k]) + (R(1) - R(0.5) * S[k]) * hF[k];
    const R hh = R(0.5), c0 = hh * cs2 * h[0];
    f[0] = (R(1) - R(3) * cs2) * h[0] - h[4] - h[5] - h[6];
    f[1] = c0 + hh * (h[1] + h[4]);
    f[2] = c0 + hh * (-h[1] + h[4]);
    f[3] = c0 + hh * (h[2] + h[5]);
    f[4] = c0 + hh * (-h[2] + h[5]);
    f[5] = c0 + hh * (h[3] + h[6]);
    f[6] = c0 + hh * (-h[3] + h[6]);
}

// The unit-rate collisions (every rate of a non-conserved moment but the
// flow's second-order ones is 1: h* = h - (h - heq) + hF/2 = heq + hF/2,
// Eq. 37).  D3Q7: the result follows from heq and hF alone (moment 0 is phi
// itself); f is only written.
template <class R>
__device__ __forceinline__ void collide7_unit(R f[7], const R heq[7], const R hF[7], R cs2)
{
    R h[7];
    h[0] = heq[0];
#pragma unroll
    for (int k = 1; k < 7; ++k) h[k] = heq[k] + R(0.5) * hF[k];
    const R hh = R(0.5), c0 = hh * cs2 * h[0];
    f[0] = (R(1) - R(3) * cs2) * h[0] - h[4] - h[5] - h[6];
    f[1] = c0 + hh * (h[1] + h[4]);
    f[2] = c0 + hh * (-h[1] + h[4]);
    f[3] = c0 + hh * (h[2] + h[5]);
    f[4] = c0 + hh * (-h[2] + h[5]);
    f[5] = c0 + hh * (h[3] + h[6]);
    f[6] = c0 + hh * (-h[3] + h[6]);
}

// D3Q19 at unit rates s1, s3, s4: moment 0 relaxes at s0 and the second-order
// moments 4-9 at s_2a (diagonal) and s_2b (off-diagonal) of Eq. 35, all from
// f; moments 1-3 and 16-18 at heq + hF/2; 10-15 are zero.
template <class R>
__device__ __forceinline__ void collide19_unit(R f[19], const R heq[19], const R hF[19], R s0, R s2a, R s2b,
                                               R cs2)
{
    R h[19];
    const R m0 = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8] + f[9] + f[10] + f[11] + f[12] +
                 f[13] + f[14] + f[15] + f[16] + f[17] + f[18];
    const R exy = f[7] + f[8] + f[9] + f[10], exz = f[11] + f[12] + f[13] + f[14],
            eyz = f[15] + f[16] + f[17] + f[18];
    h[0] = m0 - s0 * m0 + (R(1) - R(0.5) * s0) * hF[0];  // (heq[0] = 0)
    const R d[3] = {f[1] + f[2] + exy + exz - cs2 * m0, f[3] + f[4] + exy + eyz - cs2 * m0,
                    f[5] + f[6] + exz + eyz - cs2 * m0};
    const R o[3] = {f[7] + f[8] - f[9] - f[10], f[11] + f[12] - f[13] - f[14], f[15] + f[16] - f[17] - f[18]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        h[1 + k] = heq[1 + k] + R(0.5) * hF[1 + k];
        h[4 + k] = d[k] - s2a * (d[k] - heq[4 + k]) + (R(1) - R(0.5) * s2a) * hF[4 + k];
        h[7 + k] = o[k] - s2b * (o[k] - heq[7 + k]) + (R(1) - R(0.5) * s2b) * hF[7 + k];
        h[16 + k] = heq[16 + k] + R(0.5) * hF[16 + k];
    }
#pragma unroll
    for (int k = 10; k < 16; ++k) h[k] = R(0);
    from_hermite19<R>(h, f, cs2);
}

// 1/x: the hardware's approximate reciprocal in FP32 (within 1 ulp; the
// arguments are a density, a bounded 1 - phi0 and rates >= 1/2), the exact
// quotient in FP64 (whose path matches the oracle to 1e-12)
template <class R>
__device__ __forceinline__ R recip(R x)
{
    if constexpr (sizeof(R) == 4) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    } else {
        return R(1) / x;
    }
}

// a store marked streaming (evict first): the new state is read again only in
// the next step, after the rest of the state has passed through the L2
template <class T>
__device__ __forceinline__ void st_stream(T *p, T v)
{
    if constexpr (sizeof(T) == 2)
        __stcs(reinterpret_cast<unsigned short *>(p), *reinterpret_cast<const unsigned short *>(&v));
    else
        __stcs(p, v);
}

// D3Q19 isotropic stencils (weights 1/18 faces, 1/36 edges, cs^2 = 1/3) on
// three shared-memory planes (below, centre, above) of width W.
template <class R, int W>
__device__ __forceinline__ void grad19(const R *lo, const R *mid, const R *hi, int x, int y, R &gx,
                                       R &gy, R &gz)
{
    auto at = [&](const R *pl, int dx, int dy) { return pl[(y + dy) * W + (x + dx)]; };
    const R f6 = R(1) / R(6), f12 = R(1) / R(12);
    gx = f6 * (at(mid, 1, 0) - at(mid, -1, 0)) +
         f12 * (at(mid, 1, 1) + at(mid, 1, -1) - at(mid, -1, 1) - at(mid, -1, -1) + at(hi, 1, 0) +
                at(lo, 1, 0) - at(hi, -1, 0) - at(lo, -1, 0));
    gy = f6 * (at(mid, 0, 1) - at(mid, 0, -1)) +
         f12 * (at(mid, 1, 1) + at(mid, -1, 1) - at(mid, 1, -1) - at(mid, -1, -1) + at(hi, 0, 1) +
                at(lo, 0, 1) - at(hi, 0, -1) - at(lo, 0, -1));
    gz = f6 * (at(hi, 0, 0) - at(lo, 0, 0)) +
         f12 * (at(hi, 1, 0) + at(hi, -1, 0) + at(hi, 0, 1) + at(hi, 0, -1) - at(lo, 1, 0) -
                at(lo, -1, 0) - at(lo, 0, 1) - at(lo, 0, -1));
}

template <class R, int W>
__device__ __forceinline__ R lap19(const R *lo, const R *mid, const R *hi, int x, int y)
{
    auto at = [&](const R *pl, int dx, int dy) { return pl[(y + dy) * W + (x + dx)]; };
    const R c = at(mid, 0, 0);
    const R faces = at(mid, 1, 0) + at(mid, -1, 0) + at(mid, 0, 1) + at(mid, 0, -1) + at(hi, 0, 0) +
                    at(lo, 0, 0);
    const R edges = at(mid, 1, 1) + at(mid, -1, -1) + at(mid, 1, -1) + at(mid, -1, 1) + at(hi, 1, 0) +
                    at(lo, -1, 0) + at(lo, 1, 0) + at(hi, -1, 0) + at(hi, 0, 1) + at(lo, 0, -1) +
                    at(lo, 0, 1) + at(hi, 0, -1);
    // 6 * (1/18 sum_faces (v - c) + 1/36 sum_edges (v - c))
    return R(1) / R(3) * (faces - R(6) * c) + R(1) / R(6) * (edges - R(12) * c);
}

template <class R>
__device__ __forceinline__ R particle_phi0_3d(const ParticleDev &pp, int gx, int gy, int gz, int nx,
                                              int ny, int nz, double D, double cut, R &rx, R &ry,
                                              R &rz)
{
    double dx = (double)gx - pp.x[0], dy = (double)gy - pp.x[1], dz = (double)gz - pp.x[2];
    dx = min_image(dx, nx);
    if (ny > 0) dy = min_image(dy, ny);  // ny <= 0: walls in y, no minimum image
    dz = min_image(dz, nz);
    rx = (R)dx;
    ry = (R)dy;
    rz = (R)dz;
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double lim = pp.R + cut;
    if (r2 >= lim * lim) return R(0);
    const R r = sqrt((R)r2);
    return R(0.5) * (R(1) + tanh(R(2) * ((R)pp.R - r) / (R)D));
}

// EXT: the instantiation also handles domains with walls at the ends of y
// UNIT: every domain of the launch has unit rates for its non-conserved
// moments (FP32 arithmetic only): the collisions above.  FP32 arithmetic
// without particles: three CTAs per SM (80 registers, a few spilled; the step
// waits on global loads, and 24 warps per SM hide more of them than 16 at
// 128 registers: measured 9.8k -> 11.8k MLUPS on the 256^3 drainage, while
// four CTAs at 64 registers spill too much, 10.8k)
template <class P, int TX, int TY, int ZC, bool MOVING, int MODE, bool EXT, bool UNIT = false>
__global__ void __launch_bounds__(TX *TY, (sizeof(typename P::real) == 4 && !MOVING) ? 3 : 1) k_step3d(StepArgs A)
{
    using R = typename P::real;
    using ST = typename P::store;
    using AX = typename P::aux;
    constexpr int NT = TX * TY;
    constexpr int FX = TX + 4, FY = TY + 4, FP = FX * FY;  // tile + 2 frame (one plane)
    constexpr int WX = TX + 2, WY = TY + 2, WP = WX * WY;  // tile + 1 frame
    __shared__ R s_phi[5][FP];
    __shared__ R s_p0[5][FP];
    __shared__ R s_mu[4][WP];
    __shared__ R s_T[4][3][WP];
    __shared__ int s_gx[TX + 6];
    __shared__ int s_gy[TY + 6];   // wrapped row offsets y * pitch
    __shared__ int s_gyi[TY + 6];  // wrapped rows
    __shared__ int s_out[EXT ? TY + 6 : 1];  // walls: the row lies beyond a wall (mirror image)
    __shared__ double s_red[2][NT / 32][6];  // warps' sums, double-buffered over particles
    // particles with their own contact angle (MOVING with A.wv): W and V of
    // every staged phi0 plane (the same ring of 5), in dynamic shared memory
    // (2 * 5 * FP values of R; the launch passes none otherwise)
    extern __shared__ __align__(16) unsigned char s_dyn3d[];
    R *const s_W = reinterpret_cast<R *>(s_dyn3d);
    R *const s_V = s_W + 5 * FP;

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;

    for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
        const DomainDev &Dm = A.doms[A.tile_dom[t]];
        const int2 txy = A.tile_xy[t];
        const int nx = Dm.nx, ny = Dm.ny, nz = Dm.nz;
        const int plane = (int)Dm.plane;  // 26 * plane < 2^31 (checked at create)
        const int zstride = Dm.pitch * ny;
        const int x0 = txy.x * TX;
        const int y0 = (txy.y % Dm.tiles_y) * TY;
        const int zc = Dm.zc;
        const int z0 = (txy.y / Dm.tiles_y) * zc;
        const DevParams &p = Dm.p;
        const KParams<R> &kp = kparams<R>(Dm);

        __syncthreads();
        const int wall = EXT ? Dm.wall_y : 0;
        const int nyw = wall ? 0 : ny;  // minimum image in y only without walls
        for (int k = tid; k < TX + 6; k += NT) s_gx[k] = wrap_idx(x0 - 3 + k, nx);
        for (int k = tid; k < TY + 6; k += NT) {
            if constexpr (EXT) {
                const int y = y0 - 3 + k;
                int yy, out = 0;
                if (wall) {
                    // rows beyond a wall read their mirror image (clamped: the
                    // rows that far out only feed cells beyond the domain)
                    yy = y < 0 ? -1 - y : (y >= ny ? 2 * ny - 1 - y : y);
                    out = y < 0 || y >= ny;
                    yy = min(max(yy, 0), ny - 1);
                } else {
                    yy = wrap_idx(y, ny);
                }
                s_gyi[k] = yy;
                s_gy[k] = yy * Dm.pitch;
                s_out[k] = out;
            } else {
                const int yy = wrap_idx(y0 - 3 + k, ny);
                s_gyi[k] = yy;
                s_gy[k] = yy * Dm.pitch;
            }
        }
        __syncthreads();
        // a tile whose frames reach beyond a wall
        const bool wall_tile = EXT && wall && (y0 - 3 < 0 || y0 + TY + 3 > ny);
        // sign of the y-odd products T_xy, T_yz at table row r under a wall mirror
        auto wsign = [&](int r) -> R {
            if constexpr (EXT) return s_out[r] ? R(-1) : R(1);
            return R(1);
        };

        const ST *fs = reinterpret_cast<const ST *>(Dm.f[A.par]);
        ST *fd = reinterpret_cast<ST *>(Dm.f[A.par ^ 1]);
        const AX *as = reinterpret_cast<const AX *>(Dm.aux[A.par]);
        AX *ad = reinterpret_cast<AX *>(Dm.aux[A.par ^ 1]);
        const AX *ph0 = reinterpret_cast<const AX *>(Dm.phi0);
        const long long *rs = reinterpret_cast<const long long *>(Dm.rest[A.par]);
        long long *rd = reinterpret_cast<long long *>(Dm.rest[A.par ^ 1]);
        const R isc1 = kp.inv_scale[0], isc2 = kp.inv_scale[1];
        const R c_dw = kp.c_dw, c_lap = kp.c_lap, c_pen = kp.c_pen, c_wet = kp.c_wet,
                c_wlap = kp.c_wlap;

        // the planes touched lie in [z0 - 3, min(z0 + zc, nz) + 2], inside
        // [-nz, 2 nz) since nz >= 4
        auto zoff = [&](int z) { return wrap_near(z, nz) * zstride; };
        auto cidx = [&](int tx_, int ty_, int zo) {  // tile+3 table coordinates
            return zo + s_gy[ty_] + s_gx[tx_];
        };
        // offset of the population that table cell (cx, cy) of plane z pulls as
        // direction i of the lattice starting at plane `base`: from cell - c_i,
        // or, where that lies beyond a wall, its own opposite population
        // (halfway bounce-back)
        auto pull = [&](int base, int i, int cx, int cy, int z) -> int {
            if constexpr (EXT) {
                if (wall_tile && s_out[cy - C19Y[i]] && !s_out[cy])
                    return (base + opp19(i)) * plane + cidx(cx, cy, zoff(z));
            }
            return base * plane + i * plane + cidx(cx - C19X[i], cy - C19Y[i], zoff(z - C19Z[i]));
        };
        // phi at (frame x, frame y) of plane z: pull and sum the D3Q7 populations
        auto phi_at = [&](int hx, int hy, int z, R *keep, ST *keepq) -> R {
            const int cx = hx + 1, cy = hy + 1;
            R acc;
            if constexpr (P::MIX) {
                acc = float_of_fixed(rs[cidx(cx, cy, zoff(z))]);
                if (keep) keep[0] = acc;
#pragma unroll
                for (int i = 1; i < 7; ++i) {
                    const ST qv = ldg(fs + pull(0, i, cx, cy, z));
                    const R v = Conv<P>::ld(qv, isc1);
                    if (keep) keep[i] = v;
                    if (keepq) keepq[i] = qv;
                    acc += v;
                }
            } else {
                acc = R(0);
#pragma unroll
                for (int i = 0; i < 7; ++i) {
                    const R v = Conv<P>::ld(ldg(fs + pull(0, i, cx, cy, z)), isc1);
                    if (keep) keep[i] = v;
                    acc += v;
                }
            }
            return acc;
        };
        // total indicator at (frame x, frame y) of plane z; with own particle
        // angles (Wo set) also W = sum_s cos(theta_s) phi0_s and V = sum_s
        // cos(theta_s) phi0_s^3, every solid without an own angle counted as one
        auto phi0_at = [&](int hx, int hy, int z, R *Wo, R *Vo) -> R {
            const int cx = hx + 1, cy = hy + 1;
            R v = (R)ldg(ph0 + cidx(cx, cy, zoff(z)));
            if constexpr (MOVING) {
                const int gx = s_gx[cx], gy = s_gyi[cy], gz = wrap_near(z, nz);
                R dflt = v, w = R(0), vv = R(0);
                for (int k = 0; k < A.np; ++k) {
                    R rx, ry, rz;
                    const R pk = particle_phi0_3d<R>(A.parts[k], gx, gy, gz, nx, nyw, nz, p.D, p.cut, rx, ry, rz);
                    v += pk;
                    if (Wo) {
                        if (A.parts[k].own) {
                            const R ck = (R)A.parts[k].ct;
                            w += ck * pk;
                            vv += ck * pk * pk * pk;
                        } else {
                            dflt += pk;
                        }
                    }
                }
                if (Wo) {
                    const R ct = (R)p.cos_t;
                    *Wo = ct * dflt + w;
                    *Vo = ct * dflt * dflt * dflt + vv;
                }
            }
            return v;
        };
        auto load_phi_plane = [&](int z) {
            const int slot = wrap_idx(z, 5);
            for (int r = tid; r < FP; r += NT) {
                const int hx = r % FX, hy = r / FX;
                s_phi[slot][r] = phi_at(hx, hy, z, nullptr, nullptr);
                if (MOVING && A.wv)
                    s_p0[slot][r] = phi0_at(hx, hy, z, s_W + slot * FP + r, s_V + slot * FP + r);
                else
                    s_p0[slot][r] = phi0_at(hx, hy, z, nullptr, nullptr);
            }
        };
        auto load_T_plane = [&](int z) {
            const int slot = wrap_idx(z, 4);
            const int zo = zoff(z);
            for (int r = tid; r < WP; r += NT) {
                const int wx = r % WX, wy = r / WX;
                const int id = cidx(wx + 2, wy + 2, zo);
                const R ux = (R)ldg(as + 0 * plane + id), uy = (R)ldg(as + 1 * plane + id),
                        uz = (R)ldg(as + 2 * plane + id);
                const R Sx = (R)ldg(as + 3 * plane + id), Sy = (R)ldg(as + 4 * plane + id),
                        Sz = (R)ldg(as + 5 * plane + id);
                const R sg = wsign(wy + 2);  // T_xy and T_yz are odd under the wall mirror
                s_T[slot][0][r] = sg * (Sx * uy - ux * Sy);
                s_T[slot][1][r] = Sx * uz - ux * Sz;
                s_T[slot][2][r] = sg * (Sy * uz - uy * Sz);
            }
        };
        auto mu_plane = [&](int z) {
            const int slot = wrap_idx(z, 4);
            const R *lo = s_phi[wrap_idx(z - 1, 5)], *mid = s_phi[wrap_idx(z, 5)], *hi = s_phi[wrap_idx(z + 1, 5)];
            const R *lo0 = s_p0[wrap_idx(z - 1, 5)], *mid0 = s_p0[wrap_idx(z, 5)], *hi0 = s_p0[wrap_idx(z + 1, 5)];
            for (int r = tid; r < WP; r += NT) {
                const int hx = r % WX + 1, hy = r / WX + 1;
                const R ph = mid[hy * FX + hx], p0 = mid0[hy * FX + hx];
                const R lp = lap19<R, FX>(lo, mid, hi, hx, hy);
                if (MOVING && A.wv) {
                    // wetting summed per solid (own particle angles), through W and V
                    const R *Wl = s_W + wrap_idx(z - 1, 5) * FP, *Wm = s_W + wrap_idx(z, 5) * FP,
                            *Wh = s_W + wrap_idx(z + 1, 5) * FP;
                    const R Wv = Wm[hy * FX + hx], Vv = s_V[wrap_idx(z, 5) * FP + hy * FX + hx];
                    s_mu[slot][r] = c_dw * ph * (ph - R(1)) * (ph + R(1)) - c_lap * lp + c_pen * p0 * p0 * ph +
                                    c_dw * (R(3) * ph * ph * Wv + Vv - Wv) - c_lap * lap19<R, FX>(Wl, Wm, Wh, hx, hy);
                    continue;
                }
                const R lp0 = lap19<R, FX>(lo0, mid0, hi0, hx, hy);
                s_mu[slot][r] = c_dw * ph * (ph - R(1)) * (ph + R(1)) - c_lap * lp + c_pen * p0 * p0 * ph +
                                c_wet * p0 * (R(3) * ph * ph + p0 * p0 - R(1)) - c_wlap * lp0;
            }
        };

        // walls: phi beyond a wall is the mirror image of phi inside (no flux);
        // refills the rows of plane z's slot beyond the wall (after a barrier)
        auto mirror_phi_plane = [&](int z) {
            if constexpr (EXT) {
                const int slot = wrap_idx(z, 5);
                for (int r = tid; r < FP; r += NT) {
                    const int hx = r % FX, hy = r / FX;
                    if (!s_out[hy + 1]) continue;
                    const int y = y0 - 2 + hy;
                    const int hym = (y < 0 ? -1 - y : 2 * ny - 1 - y) - (y0 - 2);
                    if (hym >= 0 && hym < FY && !s_out[hym + 1]) s_phi[slot][r] = s_phi[slot][hym * FX + hx];
                }
            }
        };

        // prologue: phi planes z0-2 .. z0+1, T planes z0-1, z0, mu planes z0-1, z0
        for (int z = z0 - 2; z <= z0 + 1; ++z) load_phi_plane(z);
        if constexpr (MODE == MODE_STEP) {
            load_T_plane(z0 - 1);
            load_T_plane(z0);
        }
        __syncthreads();
        if (wall_tile) {
            for (int z = z0 - 2; z <= z0 + 1; ++z) mirror_phi_plane(z);
            __syncthreads();
        }
        mu_plane(z0 - 1);
        mu_plane(z0);
        __syncthreads();

        // PRE: the own cell's loads of phase 3 (its pulled populations of both
        // lattices, the rest population, the lagged fields) are issued at the
        // top of the plane, so that their round trip overlaps the loads of
        // phase 1 instead of following two barriers
        constexpr bool PRE = MODE == MODE_STEP && !MOVING && sizeof(R) == 4;
        const int zend = min(z0 + zc, nz);
        for (int z = z0; z < zend; ++z) {
            [[maybe_unused]] ST q1p[7], q2p[19];
            [[maybe_unused]] AX lagp[7];
            [[maybe_unused]] long long restp = 0;
            if constexpr (PRE) {
                const int zo0 = zoff(z);
                const int id0 = cidx(lx + 3, ly + 3, zo0);
                if constexpr (P::MIX) restp = rs[id0];
#pragma unroll
                for (int i = P::MIX ? 1 : 0; i < 7; ++i) q1p[i] = ldg(fs + pull(0, i, lx + 3, ly + 3, z));
#pragma unroll
                for (int i = 0; i < 19; ++i) q2p[i] = ldg(fs + pull(7, i, lx + 3, ly + 3, z));
#pragma unroll
                for (int k = 0; k < 7; ++k) lagp[k] = ldg(as + k * plane + id0);
            }
            // phase 1: phi plane z+2 and T plane z+1
            load_phi_plane(z + 2);
            if constexpr (MODE == MODE_STEP) load_T_plane(z + 1);
            __syncthreads();
            if (wall_tile) {
                mirror_phi_plane(z + 2);
                __syncthreads();
            }
            // phase 2: mu plane z+1
            mu_plane(z + 1);
            __syncthreads();

            // phase 3: own cell of plane z
            const int gx = x0 + lx, gy = y0 + ly;
            const bool valid = gx < nx && gy < ny;
            const int zo = zoff(z);
            const int id = cidx(lx + 3, ly + 3, zo);
            const int hx = lx + 2, hy = ly + 2, wxy = (ly + 1) * WX + (lx + 1);
            const R *plo = s_phi[wrap_idx(z - 1, 5)], *pmid = s_phi[wrap_idx(z, 5)], *phi_hi = s_phi[wrap_idx(z + 1, 5)];
            const R *mlo = s_mu[wrap_idx(z - 1, 4)], *mmid = s_mu[wrap_idx(z, 4)], *mhi = s_mu[wrap_idx(z + 1, 4)];

            R f1[7];
            ST q1[7];
            R phi;
            if constexpr (PRE) {
                // phi_at's sum, in its order, from the values loaded at the top
                if constexpr (P::MIX) {
                    R acc = float_of_fixed(restp);
                    f1[0] = acc;
#pragma unroll
                    for (int i = 1; i < 7; ++i) {
                        const R v = Conv<P>::ld(q1p[i], isc1);
                        f1[i] = v;
                        q1[i] = q1p[i];
                        acc += v;
                    }
                    phi = acc;
                } else {
                    R acc = R(0);
#pragma unroll
                    for (int i = 0; i < 7; ++i) {
                        const R v = Conv<P>::ld(q1p[i], isc1);
                        f1[i] = v;
                        acc += v;
                    }
                    phi = acc;
                }
            } else {
                phi = phi_at(hx, hy, z, f1, q1);
            }
            const R phi0 = s_p0[wrap_idx(z, 5)][hy * FX + hx];
            R gpx, gpy, gpz, gmx, gmy, gmz;
            grad19<R, FX>(plo, pmid, phi_hi, hx, hy, gpx, gpy, gpz);
            grad19<R, WX>(mlo, mmid, mhi, lx + 1, ly + 1, gmx, gmy, gmz);
            const R mu = mmid[wxy];
            const R drho = kp.drho;
            const R rho = drho * phi + kp.rhom;
            const R muv = kp.dmu * phi + kp.mum;
            // conservative Allen-Cahn option: theta n = (2/D)(1 - phi^2) grad phi/|grad phi|
            // and the mass flux M (rho1 - rho2)/2 (grad phi - theta n)
            const bool cac = Dm.p.phase_model == 1;
            R tnx = R(0), tny = R(0), tnz = R(0);
            if (cac) {
                const R g2 = gpx * gpx + gpy * gpy + gpz * gpz;
                const R th = kp.two_over_D * (R(1) - phi * phi);
                const R inv = g2 > R(1e-24) ? R(1) / sqrt(g2) : R(0);
                tnx = th * gpx * inv;
                tny = th * gpy * inv;
                tnz = th * gpz * inv;
            }
            const R Sx = cac ? kp.Mdrho * (gpx - tnx) : kp.Mdrho * gmx;
            const R Sy = cac ? kp.Mdrho * (gpy - tny) : kp.Mdrho * gmy;
            const R Sz = cac ? kp.Mdrho * (gpz - tnz) : kp.Mdrho * gmz;
            const R grx = drho * gpx, gry = drho * gpy, grz = drho * gpz;
            R Fx = mu * gpx + kp.Fb[0], Fy = mu * gpy + kp.Fb[1], Fz = mu * gpz + kp.Fb[2];
            if constexpr (MODE == MODE_STEP) {
                // F_c,b = 1/2 sum_a d_a T_ab with T antisymmetric (previous step)
                const int s0_ = wrap_idx(z - 1, 4), s1_ = wrap_idx(z, 4), s2_ = wrap_idx(z + 1, 4);
                R axy, ayx, azx, axz, ayz, azy, dummy;
                // d/dx, d/dy, d/dz of T_xy
                grad19<R, WX>(s_T[s0_][0], s_T[s1_][0], s_T[s2_][0], lx + 1, ly + 1, axy, ayx, azx);
                R bx, by, bz;
                grad19<R, WX>(s_T[s0_][1], s_T[s1_][1], s_T[s2_][1], lx + 1, ly + 1, bx, by, bz);
                R cx_, cy_, cz_;
                grad19<R, WX>(s_T[s0_][2], s_T[s1_][2], s_T[s2_][2], lx + 1, ly + 1, cx_, cy_, cz_);
                (void)azx;
                (void)by;
                (void)cx_;
                (void)dummy;
                (void)axz;
                (void)ayz;
                (void)azy;
                Fx += R(0.5) * (-ayx - bz);   // -d_y T_xy - d_z T_xz
                Fy += R(0.5) * (axy - cz_);   //  d_x T_xy - d_z T_yz
                Fz += R(0.5) * (bx + cy_);    //  d_x T_xz + d_y T_yz
            } else {
                // macroscopic pass: F_c from the lagged fields read directly
                R T[3][3][3][3];
#pragma unroll
                for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
                    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int nid = cidx(lx + 3 + dx, ly + 3 + dy, zoff(z + dz));
                            const R ux = (R)ldg(as + 0 * plane + nid), uy = (R)ldg(as + 1 * plane + nid),
                                    uz = (R)ldg(as + 2 * plane + nid);
                            const R sx = (R)ldg(as + 3 * plane + nid), sy = (R)ldg(as + 4 * plane + nid),
                                    sz = (R)ldg(as + 5 * plane + nid);
                            const R sg = wsign(ly + 3 + dy);
                            T[0][dz + 1][dy + 1][dx + 1] = sg * (sx * uy - ux * sy);
                            T[1][dz + 1][dy + 1][dx + 1] = sx * uz - ux * sz;
                            T[2][dz + 1][dy + 1][dx + 1] = sg * (sy * uz - uy * sz);
                        }
                R g[3][3];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    grad19<R, 3>(&T[c][0][0][0], &T[c][1][0][0], &T[c][2][0][0], 1, 1, g[c][0], g[c][1], g[c][2]);
                Fx += R(0.5) * (-g[0][1] - g[1][2]);
                Fy += R(0.5) * (g[0][0] - g[2][2]);
                Fz += R(0.5) * (g[1][0] + g[2][1]);
            }
            if constexpr (MOVING) {
                const R lphi = lap19<R, FX>(plo, pmid, phi_hi, hx, hy);
                R g0x, g0y, g0z;
                grad19<R, FX>(s_p0[wrap_idx(z - 1, 5)], s_p0[wrap_idx(z, 5)], s_p0[wrap_idx(z + 1, 5)], hx, hy,
                              g0x, g0y, g0z);
                if (A.wv) {
                    // sum over solids of mu_phi0,s grad phi0_s with their own angles
                    const int s0w = wrap_idx(z - 1, 5) * FP, s1w = wrap_idx(z, 5) * FP, s2w = wrap_idx(z + 1, 5) * FP;
                    R gWx, gWy, gWz, gVx, gVy, gVz;
                    grad19<R, FX>(s_W + s0w, s_W + s1w, s_W + s2w, hx, hy, gWx, gWy, gWz);
                    grad19<R, FX>(s_V + s0w, s_V + s1w, s_V + s2w, hx, hy, gVx, gVy, gVz);
                    const R pen = c_pen * phi0 * phi * phi;
                    const R aW = c_dw * phi * (phi * phi - R(1)) - c_lap * lphi, aV = c_dw * phi;
                    Fx += pen * g0x + aW * gWx + aV * gVx;
                    Fy += pen * g0y + aW * gWy + aV * gVy;
                    Fz += pen * g0z + aW * gWz + aV * gVz;
                } else {
                    const R mu0 = c_pen * phi0 * phi * phi +
                                  c_wet * phi * (R(3) * phi0 * phi0 + phi * phi - R(1)) - c_wlap * lphi;
                    Fx += mu0 * g0x;
                    Fy += mu0 * g0y;
                    Fz += mu0 * g0z;
                }
            }

            R f2[19];
#pragma unroll
            for (int i = 0; i < 19; ++i)
                f2[i] = Conv<P>::ld(PRE ? q2p[i] : ldg(fs + pull(7, i, lx + 3, ly + 3, z)), isc2);
            R jx = R(0), jy = R(0), jz = R(0), sum_f = R(0);
#pragma unroll
            for (int i = 1; i < 19; ++i) {
                jx += (R)C19X[i] * f2[i];
                jy += (R)C19Y[i] * f2[i];
                jz += (R)C19Z[i] * f2[i];
                sum_f += f2[i];
            }
            const R irho = recip(rho);
            const R usx = (jx + R(0.5) * Fx) * irho, usy = (jy + R(0.5) * Fy) * irho,
                    usz = (jz + R(0.5) * Fz) * irho;
            R fpx = -phi0 * usx, fpy = -phi0 * usy, fpz = -phi0 * usz;
            if constexpr (MOVING) {
                for (int k = 0; k < A.np; ++k) {
                    const ParticleDev &pp = A.parts[k];
                    R rx, ry, rz;
                    const R pk = particle_phi0_3d<R>(pp, gx, gy, z, nx, nyw, nz, p.D, p.cut, rx, ry, rz);
                    if (pk != R(0)) {
                        fpx += pk * ((R)pp.u[0] + (R)pp.w[1] * rz - (R)pp.w[2] * ry);
                        fpy += pk * ((R)pp.u[1] + (R)pp.w[2] * rx - (R)pp.w[0] * rz);
                        fpz += pk * ((R)pp.u[2] + (R)pp.w[0] * ry - (R)pp.w[1] * rx);
                    }
                }
            }
            const R ux = usx + R(0.5) * fpx, uy = usy + R(0.5) * fpy, uz = usz + R(0.5) * fpz;
            const R Ftx = Fx + rho * fpx, Fty = Fy + rho * fpy, Ftz = Fz + rho * fpz;
            const R upx = (R)(PRE ? lagp[0] : ldg(as + 0 * plane + id)),
                    upy = (R)(PRE ? lagp[1] : ldg(as + 1 * plane + id)),
                    upz = (R)(PRE ? lagp[2] : ldg(as + 2 * plane + id));
            const R Spx = (R)(PRE ? lagp[3] : ldg(as + 3 * plane + id)),
                    Spy = (R)(PRE ? lagp[4] : ldg(as + 4 * plane + id)),
                    Spz = (R)(PRE ? lagp[5] : ldg(as + 5 * plane + id));
            const R php = (R)(PRE ? lagp[6] : ldg(as + 6 * plane + id));

            R solid = R(1) - phi0;
            const R seps = kp.solid_eps;
            solid = solid < seps ? seps : solid;
            R nu;
            if constexpr (sizeof(R) == 4)
                nu = muv * irho * recip(solid);
            else
                nu = muv / (rho * solid);
            const R inv_s2a = R(0.5) + kp.two_over_1md0 * nu;
            const R inv_s2b = R(0.5) + kp.inv_cs2 * nu;
            const R Kf = kp.K;
            const R H = Kf * (kp.Hc0 - kp.Hc1 * inv_s2a);
            const R ugr = ux * grx + uy * gry + uz * grz;
            const R rus_u = (rho * ux - Sx) * ux + (rho * uy - Sy) * uy + (rho * uz - Sz) * uz;
            const R Su = Sx * ux + Sy * uy + Sz * uz, Sup = Spx * upx + Spy * upy + Spz * upz;
            const R dt_term = R(2) * (ux * Ftx + uy * Fty + uz * Ftz) - (Su - Sup);
            const R Pr = kp.Pfac * (sum_f + (R(0.5) + H) * ugr - kp.w0f * rus_u * kp.inv_1mcs2 +
                                      Kf * R(0.5) * dt_term);

            if constexpr (MODE == MODE_MACROS) {
                if (valid) {
                    const long long N = (long long)nx * ny * nz;
                    const long long o = ((long long)z * ny + gy) * nx + gx;
                    double phv = (double)phi;
                    if constexpr (P::MIX) {
                        int sold = 0;
#pragma unroll
                        for (int i = 1; i < 7; ++i) sold += fix24_stored<ST>(q1[i]);
                        const long long acc = rs[id] + fix24_to_rest(sold, p.klog2[0]);
                        phv = double_of_fixed(acc);
                    }
                    Dm.macro[0 * N + o] = phv;
                    Dm.macro[1 * N + o] = (double)rho;
                    Dm.macro[2 * N + o] = (double)ux;
                    Dm.macro[3 * N + o] = (double)uy;
                    Dm.macro[4 * N + o] = (double)uz;
                    Dm.macro[5 * N + o] = (double)Pr;
                    Dm.macro[6 * N + o] = (double)mu;
                    Dm.macro[7 * N + o] = (double)phi0;
                    if (MOVING && A.wv) {
                        Dm.macro[8 * N + o] = (double)s_W[wrap_idx(z, 5) * FP + hy * FX + hx];
                        Dm.macro[9 * N + o] = (double)s_V[wrap_idx(z, 5) * FP + hy * FX + hx];
                    }
                }
                continue;
            } else {
                const R cs2 = kp.cs2, cs4 = kp.cs4;
                // order-parameter lattice (D3Q7)
                const R em = cac ? phi : kp.eta * mu;  // Allen-Cahn: eta mu -> phi
                {
                    R heq[7], hF[7], S[7];
                    heq[0] = phi;
                    heq[1] = phi * ux;
                    heq[2] = phi * uy;
                    heq[3] = phi * uz;
                    heq[4] = heq[5] = heq[6] = cs2 * (em - phi);
                    hF[0] = R(0);
                    hF[1] = phi * ux - php * upx;
                    hF[2] = phi * uy - php * upy;
                    hF[3] = phi * uz - php * upz;
                    if (cac) {
                        hF[1] += cs2 * tnx;
                        hF[2] += cs2 * tny;
                        hF[3] += cs2 * tnz;
                    }
                    hF[4] = hF[5] = hF[6] = R(0);
                    if constexpr (UNIT) {
                        collide7_unit<R>(f1, heq, hF, cs2);
                    } else {
                        S[0] = kp.s0;
                        S[1] = S[2] = S[3] = kp.s1phi;
                        S[4] = S[5] = S[6] = kp.s2;
                        collide7<R>(f1, heq, hF, S, cs2);
                    }
                }
                // flow lattice (D3Q19)
                {
                    R heq[19], hF[19], S[19];
                    const R Xx = rho * ux * ux - Sx * ux, Xy = rho * uy * uy - Sy * uy, Xz = rho * uz * uz - Sz * uz;
                    const R c4r = cs4 * kp.inv_1mcs2;
                    heq[0] = R(0);
                    heq[1] = rho * ux;
                    heq[2] = rho * uy;
                    heq[3] = rho * uz;
                    heq[4] = Pr + Xx;
                    heq[5] = Pr + Xy;
                    heq[6] = Pr + Xz;
                    heq[7] = rho * ux * uy - R(0.5) * (Sx * uy + ux * Sy);
                    heq[8] = rho * ux * uz - R(0.5) * (Sx * uz + ux * Sz);
                    heq[9] = rho * uy * uz - R(0.5) * (Sy * uz + uy * Sz);
#pragma unroll
                    for (int k = 10; k < 16; ++k) heq[k] = R(0);
                    heq[16] = -cs2 * Pr - c4r * Xz;
                    heq[17] = -cs2 * Pr - c4r * Xy;
                    heq[18] = -cs2 * Pr - c4r * Xx;
                    const R c3 = R(1) - R(3) * cs2;
                    const R Mxx = R(2) * ux * Ftx - (Sx * ux - Spx * upx) + R(2) * cs2 * ux * grx + c3 * ugr;
                    const R Myy = R(2) * uy * Fty - (Sy * uy - Spy * upy) + R(2) * cs2 * uy * gry + c3 * ugr;
                    const R Mzz = R(2) * uz * Ftz - (Sz * uz - Spz * upz) + R(2) * cs2 * uz * grz + c3 * ugr;
                    const R Mxy = ux * Fty + Ftx * uy - R(0.5) * ((Sx * uy + ux * Sy) - (Spx * upy + upx * Spy)) +
                                  cs2 * (ux * gry + grx * uy);
                    const R Mxz = ux * Ftz + Ftx * uz - R(0.5) * ((Sx * uz + ux * Sz) - (Spx * upz + upx * Spz)) +
                                  cs2 * (ux * grz + grx * uz);
                    const R Myz = uy * Ftz + Fty * uz - R(0.5) * ((Sy * uz + uy * Sz) - (Spy * upz + upy * Spz)) +
                                  cs2 * (uy * grz + gry * uz);
                    hF[0] = ugr;
                    hF[1] = Ftx;
                    hF[2] = Fty;
                    hF[3] = Ftz;
                    hF[4] = Mxx;
                    hF[5] = Myy;
                    hF[6] = Mzz;
                    hF[7] = Mxy;
                    hF[8] = Mxz;
                    hF[9] = Myz;
#pragma unroll
                    for (int k = 10; k < 16; ++k) hF[k] = R(0);
                    hF[16] = -c4r * Mzz;
                    hF[17] = -c4r * Myy;
                    hF[18] = -c4r * Mxx;
                    const R s2a = recip(inv_s2a), s2b = recip(inv_s2b);
                    if constexpr (UNIT) {
                        collide19_unit<R>(f2, heq, hF, kp.s0, s2a, s2b, cs2);
                    } else {
                        S[0] = kp.s0;
                        S[1] = S[2] = S[3] = kp.s1;
                        S[4] = S[5] = S[6] = s2a;
                        S[7] = S[8] = S[9] = s2b;
#pragma unroll
                        for (int k = 10; k < 16; ++k) S[k] = kp.s3;
                        S[16] = S[17] = S[18] = kp.s4;
                        collide19<R>(f2, heq, hF, S, cs2);
                    }
                }
                if (valid) {
                    if constexpr (P::MIX) {
                        const R sc1 = kp.scale[0];
                        const int k1 = p.klog2[0];
                        int bad = 0, sold = 0, snew = 0;
#pragma unroll
                        for (int i = 1; i < 7; ++i) sold += fix24_stored<ST>(q1[i]);
#pragma unroll
                        for (int i = 1; i < 7; ++i) {
                            ST qv = Conv<P>::st(f1[i], sc1);
                            if constexpr (P::id == 3) qv = bf16_flush(qv);
                            snew += fix24_sat<ST>(qv, &bad);
                            st_stream(fd + i * plane + id, qv);
                        }
                        // exact: sum of the cell's order-parameter populations is unchanged
                        st_stream(rd + id, (PRE ? restp : rs[id]) + fix24_to_rest(sold - snew, k1));
                        if (bad) atomicOr(A.flags, 2);
                    } else {
#pragma unroll
                        for (int i = 0; i < 7; ++i) st_stream(fd + i * plane + id, Conv<P>::st(f1[i], R(1)));
                    }
                    const R sc2 = P::MIX ? kp.scale[1] : R(1);
#pragma unroll
                    for (int i = 0; i < 19; ++i) st_stream(fd + (7 + i) * plane + id, Conv<P>::st(f2[i], sc2));
                    st_stream(ad + 0 * plane + id, (AX)ux);
                    st_stream(ad + 1 * plane + id, (AX)uy);
                    st_stream(ad + 2 * plane + id, (AX)uz);
                    st_stream(ad + 3 * plane + id, (AX)Sx);
                    st_stream(ad + 4 * plane + id, (AX)Sy);
                    st_stream(ad + 5 * plane + id, (AX)Sz);
                    st_stream(ad + 6 * plane + id, (AX)phi);
                    if (!isfinite(phi) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz)) atomicOr(A.flags, 1);
                }
                if constexpr (MOVING) {
                    for (int k = 0; k < A.np; ++k) {
                        const ParticleDev &pp = A.parts[k];
                        double c6[6] = {0, 0, 0, 0, 0, 0};
                        bool hit = false;
                        if (valid) {
                            R rx, ry, rz;
                            const R pk = particle_phi0_3d<R>(pp, gx, gy, z, nx, nyw, nz, p.D, p.cut, rx, ry, rz);
                            if (pk != R(0)) {
                                hit = true;
                                const R vx = (R)pp.u[0] + (R)pp.w[1] * rz - (R)pp.w[2] * ry;
                                const R vy = (R)pp.u[1] + (R)pp.w[2] * rx - (R)pp.w[0] * rz;
                                const R vz = (R)pp.u[2] + (R)pp.w[0] * ry - (R)pp.w[1] * rx;
                                const double fx = (double)(rho * pk * (vx - usx)), fy = (double)(rho * pk * (vy - usy)),
                                             fz = (double)(rho * pk * (vz - usz));
                                c6[0] = -fx;
                                c6[1] = -fy;
                                c6[2] = -fz;
                                c6[3] = -((double)ry * fz - (double)rz * fy);
                                c6[4] = -((double)rz * fx - (double)rx * fz);
                                c6[5] = -((double)rx * fy - (double)ry * fx);
                            }
                        }
                        // warp shuffle tree (skipped by warps whose terms are all 0),
                        // warps in order; one barrier per particle and plane (the
                        // buffer written here is next written after another barrier)
                        const bool wany = __any_sync(0xffffffffu, hit);
                        double(*red)[6] = s_red[k & 1];
#pragma unroll
                        for (int c = 0; c < 6; ++c) {
                            double v = c6[c];
                            if (wany) {
#pragma unroll
                                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                            }
                            if ((tid & 31) == 0) red[tid >> 5][c] = v;
                        }
                        __syncthreads();
                        if (tid < 6) {
                            // per tile and plane: partial sums accumulate over the z loop in order
                            double acc = 0.0;
                            for (int wq = 0; wq < NT / 32; ++wq) acc += red[wq][tid];
                            double *dst = A.partials + ((long long)k * 6 + tid) * A.ntiles + t;
                            *dst = (z == z0 ? 0.0 : *dst) + acc;
                        }
                    }
                }
            }
        }
    }
}

}  // namespace pf
