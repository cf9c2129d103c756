// 2D fused time step of both D2Q9 lattices (Sec. 3.3, steps 2-6 and 7).
//
// One CTA updates a TX x TY tile of one domain per iteration of a persistent
// loop over a tile table (single domain or a batch of uneven domains).  Per
// tile, in shared memory:
//   stage A: phi (pulled and summed, Eq. 31) and phi0 on the tile + 2 halo,
//            w = S_x u_y - u_x S_y of the previous step on the tile + 1 halo;
//   stage B: mu_phi (Eq. 9) on the tile + 1 halo;
//   stage C: per cell gradients, S, F (Eq. 33), u*, f, u, P (Eq. 36),
//            relaxation rates (Eq. 35), Hermite-moment collision of both
//            lattices (Eqs. 29, 37, 38), store (pull streaming: f_i(x) at
//            t+1 is read from x - c_i), lagged fields, particle partial sums.
// Each cell's own populations are read once from DRAM; halo re-reads hit L2.
#pragma once

#include "pf_common.cuh"

namespace pf {

// D2Q9 velocities in the order of the columns of M_0 (Eq. 38), and the
// opposite direction of each.
__device__ constexpr int CX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ constexpr int CY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__device__ constexpr int OPP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};


// Hermite-moment MRT collision of one D2Q9 cell (Eqs. 29, 37, 38 with c = 1):
// h = N_H M_0 f; h* = h - S (h - heq) + (1 - S/2) hF; f* = M_0^-1 N_H^-1 h*.
template <class R>
__device__ __forceinline__ void collide9(R f[9], const R heq[9], const R hF[9], const R S[9],
                                         R cs2)
{
    const R cs4 = cs2 * cs2;
    // raw moments (rows of M_0)
    R a57 = f[5] + f[7], a68 = f[6] + f[8];
    R m0 = f[0] + f[1] + f[2] + f[3] + f[4] + a57 + a68;
    R m1 = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    R m2 = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    R m8 = a57 + a68;
    R m3 = f[1] + f[3] + m8;
    R m4 = f[2] + f[4] + m8;
    R m5 = a57 - a68;
    R m6 = f[5] - f[6] - f[7] + f[8];
    R m7 = f[5] + f[6] - f[7] - f[8];
    // Hermite moments (rows of N_H)
    R h[9];
    h[0] = m0;
    h[1] = m1;
    h[2] = m2;
    h[3] = m3 - cs2 * m0;
    h[4] = m4 - cs2 * m0;
    h[5] = m5;
    h[6] = m6 - cs2 * m1;
    h[7] = m7 - cs2 * m2;
    h[8] = m8 - cs2 * (m3 + m4) + cs4 * m0;
#pragma unroll
    for (int k = 0; k < 9; ++k)
        h[k] = h[k] - S[k] * (h[k] - heq[k]) + (R(1) - R(0.5) * S[k]) * hF[k];
    // back to raw moments (N_H^-1)
    m0 = h[0];
    m1 = h[1];
    m2 = h[2];
    m3 = h[3] + cs2 * h[0];
    m4 = h[4] + cs2 * h[0];
    m5 = h[5];
    m6 = h[6] + cs2 * h[1];
    m7 = h[7] + cs2 * h[2];
    m8 = h[8] + cs2 * (h[3] + h[4]) + cs4 * h[0];
    // populations (M_0^-1)
    const R q = R(0.25), hh = R(0.5);
    f[5] = q * (m8 + m5 + m6 + m7);
    f[6] = q * (m8 - m5 - m6 + m7);
    f[7] = q * (m8 + m5 - m6 - m7);
    f[8] = q * (m8 - m5 + m6 - m7);
    f[1] = hh * (m3 - m8 + m1 - m6);
    f[3] = hh * (m3 - m8 - m1 + m6);
    f[2] = hh * (m4 - m8 + m2 - m7);
    f[4] = hh * (m4 - m8 - m2 + m7);
    f[0] = m0 - m3 - m4 + m8;
}

// Isotropic central stencils on a shared-memory array (Sec. 3.2, last
// paragraph): D2Q9 weights 4/9, 1/9, 1/36 with cs^2 = 1/3.
template <class R, int W>
__device__ __forceinline__ void grad9(const R (*a)[W], int x, int y, R &gx, R &gy)
{
    const R e = a[y][x + 1], w = a[y][x - 1], n = a[y + 1][x], s = a[y - 1][x];
    const R ne = a[y + 1][x + 1], nw = a[y + 1][x - 1], sw = a[y - 1][x - 1],
            se = a[y - 1][x + 1];
    const R third = R(1) / R(3), twelfth = R(1) / R(12);
    gx = third * (e - w) + twelfth * ((ne + se) - (nw + sw));
    gy = third * (n - s) + twelfth * ((ne + nw) - (se + sw));
}

// the same gradient of the cubes a^3
template <class R, int W>
__device__ __forceinline__ void grad9_cubed(const R (*a)[W], int x, int y, R &gx, R &gy)
{
    auto c3 = [](R v) { return v * v * v; };
    const R e = c3(a[y][x + 1]), w = c3(a[y][x - 1]), n = c3(a[y + 1][x]), s = c3(a[y - 1][x]);
    const R ne = c3(a[y + 1][x + 1]), nw = c3(a[y + 1][x - 1]), sw = c3(a[y - 1][x - 1]),
            se = c3(a[y - 1][x + 1]);
    const R third = R(1) / R(3), twelfth = R(1) / R(12);
    gx = third * (e - w) + twelfth * ((ne + se) - (nw + sw));
    gy = third * (n - s) + twelfth * ((ne + nw) - (se + sw));
}

template <class R, int W>
__device__ __forceinline__ R lap9(const R (*a)[W], int x, int y)
{
    const R c = a[y][x];
    const R side = a[y][x + 1] + a[y][x - 1] + a[y + 1][x] + a[y - 1][x];
    const R diag = a[y + 1][x + 1] + a[y + 1][x - 1] + a[y - 1][x - 1] + a[y - 1][x + 1];
    return R(2) / R(3) * (side - R(4) * c) + R(1) / R(6) * (diag - R(4) * c);
}

// Smooth indicator of particle k at cell (gx, gy) (minimum image), 0 beyond
// R + cut where 1/2 (1 + tanh) rounds to 0 in both precisions.
template <class R, bool EXT>
__device__ __forceinline__ R particle_phi0(const ParticleDev &pp, int gx, int gy, int nx, int ny,
                                           double D, double cut, R &rx, R &ry)
{
    double dx = (double)gx - pp.x[0], dy = (double)gy - pp.x[1];
    dx = min_image(dx, nx);
    if (!EXT || ny > 0) dy = min_image(dy, ny);  // ny <= 0: walls in y, no minimum image
    rx = (R)dx;
    ry = (R)dy;
    double r2 = dx * dx + dy * dy;
    double lim = pp.R + cut;
    if (r2 >= lim * lim) return R(0);
    R r = sqrt((R)r2);
    return R(0.5) * (R(1) + tanh(R(2) * ((R)pp.R - r) / (R)D));
}

// The same indicator from the offset (dx, dy) of the cell to the particle's
// centre, given in the arithmetic type (no minimum-image arithmetic).
template <class R>
__device__ __forceinline__ R particle_phi0_rel(R dx, R dy, R Rp, R lim, R D, R &rx, R &ry)
{
    rx = dx;
    ry = dy;
    const R r2 = dx * dx + dy * dy;
    if (r2 >= lim * lim) return R(0);
    const R r = sqrt(r2);
    return R(0.5) * (R(1) + tanh(R(2) * (Rp - r) / D));
}

// Resident CTAs per SM requested from the register allocator: FP64 keeps its
// registers (no cap); the 32 x 8 FP32/16-bit kernels trade a few spills for a
// fourth CTA, 64 x 4 keeps three, 32 x 16 (the near tiles of the split step)
// two; the autotuner picks among the shapes.
template <class P, int TX, int TY>
constexpr int step2d_min_blocks()
{
    return P::id == 0 ? 1 : (TX * TY > 256 ? 2 : ((TX == 32 && TY == 8) ? 4 : 3));
}

// EXT: the instantiation also handles domains with walls at the ends of y;
// without it the wall code is compiled out (it costs registers)
template <class P, int TX, int TY, bool MOVING, int MODE, bool EXT>
__global__ void __launch_bounds__(TX *TY, (step2d_min_blocks<P, TX, TY>())) k_step2d(StepArgs A)
{
    using R = typename P::real;
    using ST = typename P::store;
    using AX = typename P::aux;
    constexpr int NT = TX * TY;
    constexpr int FX = TX + 4, FY = TY + 4;   // tile + 2 frame
    constexpr int WX = TX + 2, WY = TY + 2;   // tile + 1 frame
    __shared__ R s_phi[FY][FX];
    __shared__ R s_p0[FY][FX];
    // free particles with their own contact angle: W = sum_s cos(theta_s) phi0_s,
    // V = sum_s cos(theta_s) phi0_s^3 on the tile + 2 frame
    constexpr int WVY = MOVING ? FY : 1, WVX = MOVING ? FX : 1;
    __shared__ R s_W[WVY][WVX];
    __shared__ R s_V[WVY][WVX];
    __shared__ R s_mu[WY][WX];
    __shared__ R s_w[WY][WX];
    __shared__ int s_gx[TX + 6];
    __shared__ int s_gy[TY + 6];  // row offsets y * pitch (planes hold < 2^31 cells)
    __shared__ int s_gyi[TY + 6];
    __shared__ int s_out[EXT ? TY + 6 : 1];  // walls: the row lies beyond a wall (mirror image)
    // warps' force / torque sums of up to RED_J near particles, reduced behind
    // one barrier (s_redk: their particle indices)
    constexpr int RED_J = 8;
    __shared__ double s_red[MOVING ? RED_J : 1][NT / 32][3];
    __shared__ int s_redk[MOVING ? RED_J : 1];
    __shared__ unsigned long long s_near;  // particles whose indicator reaches this tile
    // particles whose image nearest to the tile is the minimum image of every
    // cell of its frames, and that image's centre in table coordinates (the
    // cells then skip the FP64 minimum-image arithmetic)
    constexpr int PMAX = 64;
    __shared__ unsigned long long s_fast;
    __shared__ R s_pcx[MOVING ? PMAX : 1], s_pcy[MOVING ? PMAX : 1];
    // per near particle, in the arithmetic type: radius, reach R + cut, u_x, u_y,
    // w_z, cos(own angle) (0 without one)
    __shared__ R s_pv[MOVING ? PMAX : 1][6];

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;

    for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
        if (A.tile_sel && A.tile_sel[t] != A.sel) continue;  // (uniform in the block)
        const DomainDev &Dm = A.doms[A.tile_dom[t]];
        const int2 txy = A.tile_xy[t];
        const int nx = Dm.nx, ny = Dm.ny;
        const int plane = (int)Dm.plane;  // (Q1 + Q2) * plane < 2^31 (checked at create)
        const int x0 = txy.x * TX, y0 = txy.y * TY;
        const DevParams &p = Dm.p;
        const KParams<R> &kp = kparams<R>(Dm);

        __syncthreads();  // previous tile's shared-memory readers are done
        if constexpr (MOVING) {
            if (tid == 0) s_near = s_fast = 0ull;
        }
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
        // a tile whose frames reach beyond a wall
        const bool wall_tile = EXT && wall && (y0 - 3 < 0 || y0 + TY + 3 > ny);
        // sign of w = S_x u_y - u_x S_y at table row r: odd under a wall mirror
        auto wsign = [&](int r) -> R {
            if constexpr (EXT) return s_out[r] ? R(-1) : R(1);
            return R(1);
        };
        if constexpr (MOVING) {
            // conservative test of the tile + 2 frame against each particle's
            // reach R + cut (minimum image), one thread per particle
            __syncthreads();
            for (int k = tid; k < A.np; k += NT) {
                const ParticleDev &pp = A.parts[k];
                double dx = (x0 + 0.5 * (TX - 1)) - pp.x[0], dy = (y0 + 0.5 * (TY - 1)) - pp.x[1];
                dx = min_image(dx, nx);
                if (!EXT || !wall) dy = min_image(dy, ny);
                const double ex = fmax(fabs(dx) - (0.5 * TX + 2.0), 0.0);
                const double ey = fmax(fabs(dy) - (0.5 * TY + 2.0), 0.0);
                const double lim = pp.R + p.cut + 1.0;
                if (ex * ex + ey * ey < lim * lim) {
                    atomicOr(&s_near, 1ull << k);
                    s_pv[k][0] = (R)pp.R;
                    s_pv[k][1] = (R)pp.R + (R)p.cut;
                    s_pv[k][2] = (R)pp.u[0];
                    s_pv[k][3] = (R)pp.u[1];
                    s_pv[k][4] = (R)pp.w[2];
                    s_pv[k][5] = pp.own ? (R)pp.ct : R(0);
                    // a cell of the frames farther than nx/2 from this image is at
                    // least R + cut + 1 from every image when the box is this wide
                    const double span = 2.0 * (pp.R + p.cut) + 8.0;
                    const bool fx = nx >= span + TX;
                    const bool fy = (EXT && wall) ? !wall_tile : ny >= span + TY;
                    if (fx && fy) {
                        s_pcx[k] = (R)((x0 + 0.5 * (TX - 1)) - dx - (x0 - 3));
                        s_pcy[k] = (R)((y0 + 0.5 * (TY - 1)) - dy - (y0 - 3));
                        atomicOr(&s_fast, 1ull << k);
                    }
                }
            }
        }
        __syncthreads();
        [[maybe_unused]] const unsigned long long near = MOVING ? s_near : 0ull;
        [[maybe_unused]] const unsigned long long fast = MOVING ? s_fast : 0ull;
        [[maybe_unused]] const R Dr = (R)p.D;
        [[maybe_unused]] const R kp_cos_t = (R)p.cos_t;
        // indicator of particle k at table cell (cx, cy), global cell (gx, gy)
        [[maybe_unused]] auto pphi0 = [&](int k, int cx, int cy, int gx, int gy, R &rx, R &ry) -> R {
            const ParticleDev &pp = A.parts[k];
            if ((fast >> k) & 1ull)
                return particle_phi0_rel<R>(R(cx) - s_pcx[k], R(cy) - s_pcy[k], s_pv[k][0], s_pv[k][1], Dr,
                                            rx, ry);
            return particle_phi0<R, EXT>(pp, gx, gy, nx, nyw, p.D, p.cut, rx, ry);
        };

        const ST *fs = reinterpret_cast<const ST *>(Dm.f[A.par]);
        ST *fd = reinterpret_cast<ST *>(Dm.f[A.par ^ 1]);
        const AX *as = reinterpret_cast<const AX *>(Dm.aux[A.par]);
        AX *ad = reinterpret_cast<AX *>(Dm.aux[A.par ^ 1]);
        const AX *ph0 = reinterpret_cast<const AX *>(Dm.phi0);
        const long long *rs = reinterpret_cast<const long long *>(Dm.rest[A.par]);
        long long *rd = reinterpret_cast<long long *>(Dm.rest[A.par ^ 1]);
        const R isc1 = kp.inv_scale[0], isc2 = kp.inv_scale[1];

        // offset of the population that table cell (cx, cy) pulls as direction
        // i of the lattice starting at plane `base`: from cell - c_i, or, where
        // that lies beyond a wall, its own opposite population (halfway
        // bounce-back)
        auto pull = [&](int base, int i, int cx, int cy) -> int {
            if constexpr (EXT) {
                if (wall_tile && s_out[cy - CY9[i]] && !s_out[cy])
                    return (base + OPP9[i]) * plane + s_gy[cy] + s_gx[cx];
            }
            return base * plane + i * plane + s_gy[cy - CY9[i]] + s_gx[cx - CX9[i]];
        };

        // phi at frame cell (hx, hy) of the tile+2 frame: pull and sum (Eq. 31)
        long long rest_own = 0;
        auto phi_at = [&](int hx, int hy, R *keep, ST *keepq) -> R {
            const int cx = hx + 1, cy = hy + 1;  // tile+3 table coordinates
            R acc;
            if constexpr (P::MIX) {
                const long long rv = rs[s_gy[cy] + s_gx[cx]];
                acc = float_of_fixed(rv);
                if (keep) {
                    keep[0] = acc;
                    rest_own = rv;
                }
                R movers = R(0);  // sum in stored units, scaled once
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    ST q = ldg(fs + pull(0, i, cx, cy));
                    const R v = stored_to_float<ST>(q);
                    if (keep) keep[i] = v * isc1;
                    if (keepq) keepq[i] = q;
                    movers += v;
                }
                acc += movers * isc1;
            } else {
                acc = R(0);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    R v = Conv<P>::ld(ldg(fs + pull(0, i, cx, cy)), isc1);
                    if (keep) keep[i] = v;
                    acc += v;
                }
            }
            return acc;
        };
        auto phi0_at = [&](int hx, int hy) -> R {
            const int cx = hx + 1, cy = hy + 1;
            R v = (R)ldg(ph0 + s_gy[cy] + s_gx[cx]);
            if constexpr (MOVING) {
                const int gx = s_gx[cx], gy = s_gyi[cy];
                R dflt = v, w = R(0), vv = R(0);
                for (int k = 0; k < A.np; ++k) {
                    if (!((near >> k) & 1ull)) continue;
                    R rx, ry;
                    const R pk = pphi0(k, cx, cy, gx, gy, rx, ry);
                    v += pk;
                    if (A.parts[k].own) {
                        const R ck = s_pv[k][5];
                        w += ck * pk;
                        vv += ck * pk * pk * pk;
                    } else {
                        dflt += pk;
                    }
                }
                if (A.wv) {
                    const R ct = kp_cos_t;
                    s_W[hy][hx] = ct * dflt + w;
                    s_V[hy][hx] = ct * dflt * dflt * dflt + vv;
                }
            }
            return v;
        };

        // ---------------- stage A ----------------
        // every load of the own cell is issued here, before the first barrier,
        // so one DRAM round trip per tile covers them all
        const int id = s_gy[ly + 3] + s_gx[lx + 3];
        ST f2raw[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f2raw[i] = ldg(fs + pull(9, i, lx + 3, ly + 3));
        AX lag[5];
        if constexpr (MODE == MODE_STEP) {
#pragma unroll
            for (int k = 0; k < 5; ++k) lag[k] = ldg(as + k * plane + id);
        }
        R f1[9];
        ST q1[9];
        const R phi_own = phi_at(lx + 2, ly + 2, f1, q1);
        // PMIX: the cell's exact fixed-point phi; the pulled movers are dead after this
        [[maybe_unused]] long long racc = 0;
        if constexpr (P::MIX) {
            int sold = 0;
#pragma unroll
            for (int i = 1; i < 9; ++i) sold += fix24_stored<ST>(q1[i]);
            racc = rest_own + fix24_to_rest(sold, p.klog2[0]);
        }
        s_phi[ly + 2][lx + 2] = phi_own;
        s_p0[ly + 2][lx + 2] = phi0_at(lx + 2, ly + 2);
        constexpr int RING = 4 * (TX + 4) + 4 * TY;
        for (int r = tid; r < RING; r += NT) {
            int hx, hy;
            if (r < 2 * FX) {
                hy = r / FX;
                hx = r % FX;
            } else if (r < 4 * FX) {
                int rr = r - 2 * FX;
                hy = TY + 2 + rr / FX;
                hx = rr % FX;
            } else {
                int rr = r - 4 * FX;
                hy = 2 + rr / 4;
                int c = rr % 4;
                hx = c < 2 ? c : TX + c;
            }
            s_phi[hy][hx] = phi_at(hx, hy, nullptr, nullptr);
            s_p0[hy][hx] = phi0_at(hx, hy);
        }
        if constexpr (MODE == MODE_STEP) {
            // w of the own cell from the lagged fields already in registers; the
            // tile+1 ring by the last threads (the first ones did the phi ring)
            // (odd under a wall mirror: rows beyond a wall take the sign change)
            s_w[ly + 1][lx + 1] = wsign(ly + 3) * ((R)lag[2] * (R)lag[1] - (R)lag[0] * (R)lag[3]);
            constexpr int WRING = 2 * WX + 2 * TY;
            static_assert(WRING <= NT, "one tile+1 ring cell per thread at most");
            for (int r = NT - 1 - tid; r >= 0 && r < WRING; r -= NT) {
                int wx, wy;
                if (r < 2 * WX) {
                    wy = r < WX ? 0 : TY + 1;
                    wx = r < WX ? r : r - WX;
                } else {
                    const int rr = r - 2 * WX;
                    wy = 1 + (rr >> 1);
                    wx = (rr & 1) ? TX + 1 : 0;
                }
                const int wid = s_gy[wy + 2] + s_gx[wx + 2];
                const R ux = (R)ldg(as + 0 * plane + wid), uy = (R)ldg(as + 1 * plane + wid);
                const R Sx = (R)ldg(as + 2 * plane + wid), Sy = (R)ldg(as + 3 * plane + wid);
                s_w[wy][wx] = wsign(wy + 2) * (Sx * uy - ux * Sy);
            }
        }
        if constexpr (EXT) {
            if (wall_tile) {
                // phi beyond a wall is the mirror image of phi inside (no flux)
                __syncthreads();
                for (int r = tid; r < FX * FY; r += NT) {
                    const int hx = r % FX, hy = r / FX;
                    if (!s_out[hy + 1]) continue;
                    const int y = y0 - 2 + hy;
                    const int hym = (y < 0 ? -1 - y : 2 * ny - 1 - y) - (y0 - 2);
                    if (hym >= 0 && hym < FY && !s_out[hym + 1]) s_phi[hy][hx] = s_phi[hym][hx];
                }
            }
        }
        __syncthreads();

        // ---------------- stage B: mu_phi on tile+1 (Eq. 9) ----------------
        const R c_dw = kp.c_dw, c_lap = kp.c_lap, c_pen = kp.c_pen, c_wet = kp.c_wet,
                c_wlap = kp.c_wlap;
        for (int r = tid; r < WX * WY; r += NT) {
            const int wx = r % WX, wy = r / WX;
            const int hx = wx + 1, hy = wy + 1;
            const R ph = s_phi[hy][hx], p0 = s_p0[hy][hx];
            const R lp = lap9<R, FX>(s_phi, hx, hy);
            const R base = c_dw * ph * (ph - R(1)) * (ph + R(1)) - c_lap * lp + c_pen * p0 * p0 * ph;
            bool own_wet = false;
            if constexpr (MOVING) {
                if (A.wv) {
                    // wetting summed per solid (own particle angles), through W and V
                    const R Wv = s_W[hy][hx], Vv = s_V[hy][hx];
                    s_mu[wy][wx] =
                        base + c_dw * (R(3) * ph * ph * Wv + Vv - Wv) - c_lap * lap9<R, WVX>(s_W, hx, hy);
                    own_wet = true;
                }
            }
            if (!own_wet) {
                const R lp0 = lap9<R, FX>(s_p0, hx, hy);
                s_mu[wy][wx] = base + c_wet * p0 * (R(3) * ph * ph + p0 * p0 - R(1)) - c_wlap * lp0;
            }
        }
        __syncthreads();

        // ---------------- stage C: own cell ----------------
        const int gx = x0 + lx, gy = y0 + ly;
        const bool valid = gx < nx && gy < ny;
        const int hx = lx + 2, hy = ly + 2, wx = lx + 1, wy = ly + 1;

        const R phi = phi_own, phi0 = s_p0[hy][hx];
        R gpx, gpy, gmx, gmy;
        grad9<R, FX>(s_phi, hx, hy, gpx, gpy);
        grad9<R, WX>(s_mu, wx, wy, gmx, gmy);
        const R mu = s_mu[wy][wx];
        const R drho = kp.drho;
        const R rho = drho * phi + kp.rhom;
        const R muv = kp.dmu * phi + kp.mum;
        // conservative Allen-Cahn option: theta n = (2/D)(1 - phi^2) grad phi/|grad phi|
        const bool cac = EXT && p.phase_model == 1;
        R tnx = R(0), tny = R(0);
        if (cac) {
            const R g2 = gpx * gpx + gpy * gpy;
            const R th = kp.two_over_D * (R(1) - phi * phi);
            const R inv = g2 > R(1e-24) ? R(1) / sqrt(g2) : R(0);
            tnx = th * gpx * inv;
            tny = th * gpy * inv;
        }
        // mass flux: S = M (rho1 - rho2)/2 grad mu, or (grad phi - theta n) for Allen-Cahn
        const R Sx = cac ? kp.Mdrho * (gpx - tnx) : kp.Mdrho * gmx;
        const R Sy = cac ? kp.Mdrho * (gpy - tny) : kp.Mdrho * gmy;
        const R grx = drho * gpx, gry = drho * gpy;
        R Fx = mu * gpx + kp.Fb[0], Fy = mu * gpy + kp.Fb[1];
        if constexpr (MODE == MODE_STEP) {
            // F_c = div(S u - u S)/2 from the previous step: (-d_y w, d_x w)/2
            R wgx, wgy;
            grad9<R, WX>(s_w, wx, wy, wgx, wgy);
            Fx += R(-0.5) * wgy;
            Fy += R(0.5) * wgx;
        } else {
            // macros of the current time use the same lagged F_c
            // (computed below from the aux buffer of the current parity)
        }
        R lphi = R(0);
        if constexpr (MOVING) {
            // mu_phi0 grad phi0 (Eq. 19) for free particles
            lphi = lap9<R, FX>(s_phi, hx, hy);
            R g0x, g0y;
            grad9<R, FX>(s_p0, hx, hy, g0x, g0y);
            if (A.wv) {
                // sum over solids of mu_phi0,s grad phi0_s with their own angles
                R gWx, gWy, gVx, gVy;
                grad9<R, WVX>(s_W, hx, hy, gWx, gWy);
                grad9<R, WVX>(s_V, hx, hy, gVx, gVy);
                const R pen = c_pen * phi0 * phi * phi;
                const R aW = c_dw * phi * (phi * phi - R(1)) - c_lap * lphi, aV = c_dw * phi;
                Fx += pen * g0x + aW * gWx + aV * gVx;
                Fy += pen * g0y + aW * gWy + aV * gVy;
            } else {
                const R mu0 = c_pen * phi0 * phi * phi + c_wet * phi * (R(3) * phi0 * phi0 + phi * phi - R(1)) -
                              c_wlap * lphi;
                Fx += mu0 * g0x;
                Fy += mu0 * g0y;
            }
        } else if constexpr (EXT && MODE == MODE_STEP) {
            if (A.mu0) {
                // far tiles of a particle simulation with walls (split step): the
                // fixed solids' mu_phi0 grad phi0 of Eq. 19; with own particle
                // angles in the simulation, the oracle's W/V form, in which the
                // phi0^2 grad phi0 part is the stencil of phi0^3 over 3
                const R lp = lap9<R, FX>(s_phi, hx, hy);
                R g0x, g0y;
                grad9<R, FX>(s_p0, hx, hy, g0x, g0y);
                if (A.wv) {
                    R g3x, g3y;
                    grad9_cubed<R, FX>(s_p0, hx, hy, g3x, g3y);
                    const R m = c_pen * phi0 * phi * phi + c_wet * phi * (phi * phi - R(1)) - c_wlap * lp;
                    Fx += m * g0x + c_wet * phi * g3x;
                    Fy += m * g0y + c_wet * phi * g3y;
                } else {
                    const R mu0 = c_pen * phi0 * phi * phi +
                                  c_wet * phi * (R(3) * phi0 * phi0 + phi * phi - R(1)) - c_wlap * lp;
                    Fx += mu0 * g0x;
                    Fy += mu0 * g0y;
                }
            }
        }
        if constexpr (MODE == MODE_MACROS) {
            // F_c from the lagged fields of the current parity (no shared tile)
            R wv[3][3];
#pragma unroll
            for (int j = -1; j <= 1; ++j)
#pragma unroll
                for (int i = -1; i <= 1; ++i) {
                    const int nid = s_gy[ly + 3 + j] + s_gx[lx + 3 + i];
                    const R ux = (R)ldg(as + 0 * plane + nid), uy = (R)ldg(as + 1 * plane + nid);
                    const R sx = (R)ldg(as + 2 * plane + nid), sy = (R)ldg(as + 3 * plane + nid);
                    wv[j + 1][i + 1] = wsign(ly + 3 + j) * (sx * uy - ux * sy);
                }
            R wgx, wgy;
            grad9<R, 3>(wv, 1, 1, wgx, wgy);
            Fx += R(-0.5) * wgy;
            Fy += R(0.5) * wgx;
        }

        // the flow populations pulled in stage A
        R f2[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f2[i] = Conv<P>::ld(f2raw[i], isc2);

        // u* (Eq. 36a)
        const R jx = f2[1] - f2[3] + f2[5] - f2[6] - f2[7] + f2[8];
        const R jy = f2[2] - f2[4] + f2[5] + f2[6] - f2[7] - f2[8];
        const R irho = R(1) / rho;
        const R usx = (jx + R(0.5) * Fx) * irho, usy = (jy + R(0.5) * Fy) * irho;
        // penalty force f = phi0 (u_s - u*) (Sec. 3.2, after Eq. 36)
        R fpx = -phi0 * usx, fpy = -phi0 * usy;
        if constexpr (MOVING) {
            for (int k = 0; k < A.np; ++k) {
                if (!((near >> k) & 1ull)) continue;
                R rx, ry;
                const R pk = pphi0(k, lx + 3, ly + 3, gx, gy, rx, ry);
                if (pk != R(0)) {
                    const R usx_k = s_pv[k][2] - s_pv[k][4] * ry;
                    const R usy_k = s_pv[k][3] + s_pv[k][4] * rx;
                    fpx += pk * usx_k;
                    fpy += pk * usy_k;
                }
            }
        }
        const R ux = usx + R(0.5) * fpx, uy = usy + R(0.5) * fpy;
        const R Ftx = Fx + rho * fpx, Fty = Fy + rho * fpy;

        // lagged fields at the own cell (loaded in stage A for a step; the
        // macroscopic pass reads them here)
        if constexpr (MODE == MODE_MACROS) {
#pragma unroll
            for (int k = 0; k < 5; ++k) lag[k] = ldg(as + k * plane + id);
        }
        const R upx = (R)lag[0], upy = (R)lag[1];
        const R Spx = (R)lag[2], Spy = (R)lag[3];
        const R php = (R)lag[4];

        // relaxation rates (Eq. 35, 1 - phi0 bounded below by solid_eps)
        R solid = R(1) - phi0;
        const R seps = kp.solid_eps;
        solid = solid < seps ? seps : solid;
        const R nu = muv / (rho * solid);
        const R inv_s2a = R(0.5) + kp.two_over_1md0 * nu;
        const R inv_s2b = R(0.5) + kp.inv_cs2 * nu;
        const R Kf = kp.K;
        const R H = Kf * (kp.Hc0 - kp.Hc1 * inv_s2a);
        // pressure (Eq. 36b)
        const R sum_f = f2[1] + f2[2] + f2[3] + f2[4] + f2[5] + f2[6] + f2[7] + f2[8];
        const R ugr = ux * grx + uy * gry;
        const R rus_u = (rho * ux - Sx) * ux + (rho * uy - Sy) * uy;
        const R Su = Sx * ux + Sy * uy, Sup = Spx * upx + Spy * upy;
        const R dt_term = R(2) * (ux * Ftx + uy * Fty) - (Su - Sup);
        const R Pr = kp.Pfac * (sum_f + (R(0.5) + H) * ugr - kp.w0f * rus_u * kp.inv_1mcs2 +
                                 Kf * R(0.5) * dt_term);

        if constexpr (MODE == MODE_MACROS) {
            if (valid) {
                const long long N = (long long)nx * ny;
                const long long o = (long long)gy * nx + gx;
                double phv = (double)phi;
                if constexpr (P::MIX) phv = double_of_fixed(racc);
                Dm.macro[0 * N + o] = phv;
                Dm.macro[1 * N + o] = (double)rho;
                Dm.macro[2 * N + o] = (double)ux;
                Dm.macro[3 * N + o] = (double)uy;
                Dm.macro[4 * N + o] = (double)Pr;
                Dm.macro[5 * N + o] = (double)mu;
                Dm.macro[6 * N + o] = (double)phi0;
                if constexpr (MOVING) {
                    if (A.wv) {
                        Dm.macro[7 * N + o] = (double)s_W[hy][hx];
                        Dm.macro[8 * N + o] = (double)s_V[hy][hx];
                    }
                }
            }
            continue;
        } else {
            const R cs2 = kp.cs2, cs4 = kp.cs4;
            // ---- order-parameter lattice (Eq. 30): Hermite equilibria and source
            // (Allen-Cahn: eta mu -> phi, and cs^2 theta n joins the source)
            const R eta_mu = cac ? phi : kp.eta * mu;
            R heq[9], hF[9], S[9];
            heq[0] = phi;
            heq[1] = phi * ux;
            heq[2] = phi * uy;
            heq[3] = cs2 * (eta_mu - phi);
            heq[4] = heq[3];
            heq[5] = R(0);
            heq[6] = R(0);
            heq[7] = R(0);
            heq[8] = cs4 * (phi - eta_mu);
            hF[0] = R(0);
            hF[1] = phi * ux - php * upx;  // d_t(phi u), explicit Euler
            hF[2] = phi * uy - php * upy;
            if (cac) {
                hF[1] += cs2 * tnx;
                hF[2] += cs2 * tny;
            }
#pragma unroll
            for (int k = 3; k < 9; ++k) hF[k] = R(0);
            S[0] = kp.s0;
            S[1] = S[2] = kp.s1phi;
            S[3] = S[4] = S[5] = kp.s2;
            S[6] = S[7] = kp.s3;
            S[8] = kp.s4;
            collide9<R>(f1, heq, hF, S, cs2);

            // ---- flow lattice (Eqs. 32-34)
            heq[0] = R(0);
            heq[1] = rho * ux;
            heq[2] = rho * uy;
            heq[3] = Pr + rho * ux * ux - Sx * ux;
            heq[4] = Pr + rho * uy * uy - Sy * uy;
            heq[5] = rho * ux * uy - R(0.5) * (Sx * uy + ux * Sy);
            heq[6] = R(0);
            heq[7] = R(0);
            heq[8] = -cs2 * Pr;
            const R c3 = R(1) - R(3) * cs2;
            hF[0] = ugr;
            hF[1] = Ftx;
            hF[2] = Fty;
            hF[3] = R(2) * ux * Ftx - (Sx * ux - Spx * upx) + R(2) * cs2 * ux * grx + c3 * ugr;
            hF[4] = R(2) * uy * Fty - (Sy * uy - Spy * upy) + R(2) * cs2 * uy * gry + c3 * ugr;
            hF[5] = ux * Fty + Ftx * uy - R(0.5) * ((Sx * uy + ux * Sy) - (Spx * upy + upx * Spy)) +
                    cs2 * (ux * gry + grx * uy);
            hF[6] = R(0);
            hF[7] = R(0);
            hF[8] = R(0);
            S[0] = kp.s0;
            S[1] = S[2] = kp.s1;
            S[3] = S[4] = R(1) / inv_s2a;
            S[5] = R(1) / inv_s2b;
            S[6] = S[7] = kp.s3;
            S[8] = kp.s4;
            collide9<R>(f2, heq, hF, S, cs2);

            if (valid) {
                // populations (own cell; the next step pulls them)
                if constexpr (P::MIX) {
                    const R sc1 = kp.scale[0];
                    const int k1 = p.klog2[0];
                    int bad = 0, snew = 0;
#pragma unroll
                    for (int i = 1; i < 9; ++i) {
                        ST q = Conv<P>::st(f1[i], sc1);
                        if constexpr (P::id == 3) q = bf16_flush(q);
                        snew += fix24_sat<ST>(q, &bad);
                        fd[i * plane + id] = q;
                    }
                    // exact: sum of the cell's order-parameter populations is unchanged
                    rd[id] = racc - fix24_to_rest(snew, k1);
                    if (bad) atomicOr(A.flags, 2);
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i) fd[i * plane + id] = Conv<P>::st(f1[i], R(1));
                }
                const R sc2 = P::MIX ? kp.scale[1] : R(1);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    ST q = Conv<P>::st(f2[i], sc2);
                    fd[(9 + i) * plane + id] = q;
                }
                // fields of this step, read as the previous step's by the next one
                ad[0 * plane + id] = (AX)ux;
                ad[1 * plane + id] = (AX)uy;
                ad[2 * plane + id] = (AX)Sx;
                ad[3 * plane + id] = (AX)Sy;
                ad[4 * plane + id] = (AX)phi;
                if (!isfinite(phi) || !isfinite(ux) || !isfinite(uy)) atomicOr(A.flags, 1);
            }

            if constexpr (MOVING) {
                // hydrodynamic force and torque on each particle (Eq. 27):
                // F_f = -sum rho phi0_k (u_s,k - u*), T_f = -sum r x (...)
                // 2D: F_x, F_y and T_z (components 0, 1, 5); the others stay 0.
                // The cell terms and the warp's shuffle tree are in the
                // arithmetic type (the terms are computed in it); the warps'
                // sums, the tiles' partials and the update are FP64.  Fixed
                // order: per particle, each warp's shuffle tree (skipped by warps
                // whose terms are all 0: the indicator rounds to 0 well inside
                // the reach used for the tile test), then the warps in order;
                // the warps' sums of up to RED_J near particles wait in s_red for
                // one barrier, after which one thread per particle and component
                // adds them up.
                // particles out of this tile's reach: zero partials
                for (int q = tid; q < 6 * A.np; q += NT)
                    if (!((near >> (q / 6)) & 1ull)) A.partials[(long long)q * A.ntiles + t] = 0.0;
                int nj = 0;
                auto flush = [&]() {
                    __syncthreads();  // the warps' sums of the nj particles are in s_red
                    for (int q = tid; q < 6 * nj; q += NT) {
                        const int j = q / 6, comp = q - 6 * j;
                        double acc = 0.0;
                        if (comp < 2 || comp == 5) {
                            const int c = comp == 5 ? 2 : comp;
                            for (int wq = 0; wq < NT / 32; ++wq) acc += s_red[j][wq][c];
                        }
                        A.partials[((long long)s_redk[j] * 6 + comp) * A.ntiles + t] = acc;
                    }
                    __syncthreads();  // s_red and s_redk are free again
                    nj = 0;
                };
                for (int k = 0; k < A.np; ++k) {
                    if (!((near >> k) & 1ull)) continue;
                    R c6[3] = {R(0), R(0), R(0)};
                    bool hit = false;
                    if (valid) {
                        R rx, ry;
                        const R pk = pphi0(k, lx + 3, ly + 3, gx, gy, rx, ry);
                        if (pk != R(0)) {
                            hit = true;
                            const R usx_k = s_pv[k][2] - s_pv[k][4] * ry;
                            const R usy_k = s_pv[k][3] + s_pv[k][4] * rx;
                            const R fx = rho * pk * (usx_k - usx), fy = rho * pk * (usy_k - usy);
                            c6[0] = -fx;
                            c6[1] = -fy;
                            c6[2] = -(rx * fy - ry * fx);
                        }
                    }
                    const bool wany = __any_sync(0xffffffffu, hit);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        R v = c6[c];
                        if (wany) {
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                        }
                        if ((tid & 31) == 0) s_red[nj][tid >> 5][c] = (double)v;
                    }
                    if (tid == 0) s_redk[nj] = k;
                    if (++nj == RED_J) flush();
                }
                if (nj > 0) flush();
            }
        }
    }
}

}  // namespace pf
