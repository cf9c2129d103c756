// Initialisation (Sec. 3.3 step 1), FP64 diagnostics (Eq. 8, Sec. 2.3) and the
// rigid-particle update (Eqs. 26-28) for 2D and 3D domains.
//
// These kernels run once per call (init, diagnostics) or once per step on a
// handful of particles; they are written for clarity, in double precision.
#include "pf.h"
#include "pf_internal.h"

namespace pf {

// ---- lattice tables (host and device) ------------------------------------------------------
// D2Q9 (order of M_0 in Eq. 38); D3Q19 / D3Q7 share the first 7 velocities.
__device__ const int LX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ const int LY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__device__ const int L19[19][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                   {0, 0, 1},   {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                   {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                   {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

__device__ __forceinline__ long long cell_of(const DomainDev &Dm, int x, int y, int z)
{
    return ((long long)z * Dm.ny + y) * Dm.pitch + x;
}

__device__ __forceinline__ long long lin_of(const DomainDev &Dm, int x, int y, int z)
{
    return ((long long)z * Dm.ny + y) * Dm.nx + x;
}

// row of a neighbour at y: periodic, or, with walls at the ends of y, the
// mirror image of the row inside (zero normal gradient)
__device__ __forceinline__ int row_bc(const DomainDev &Dm, int y)
{
    if (Dm.wall_y) return y < 0 ? -1 - y : (y >= Dm.ny ? 2 * Dm.ny - 1 - y : y);
    return wrap_idx(y, Dm.ny);
}

// FD stencil (D2Q9 or D3Q19 with classical weights, cs^2 = 1/3) on a dense
// x-fastest double array.
__device__ void fd_grad_lap(const DomainDev &Dm, const double *a, int x, int y, int z, double g[3],
                            double *lap)
{
    const int dim = Dm.p.dim;
    const int Q = dim == 2 ? 9 : 19;
    const double c0 = a[lin_of(Dm, x, y, z)];
    double acc = 0.0;
    g[0] = g[1] = g[2] = 0.0;
    for (int i = 1; i < Q; ++i) {
        int cx, cy, cz;
        double w;
        if (dim == 2) {
            cx = LX9[i];
            cy = LY9[i];
            cz = 0;
            w = i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0;
        } else {
            cx = L19[i][0];
            cy = L19[i][1];
            cz = L19[i][2];
            w = i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0;
        }
        const int xx = wrap_idx(x + cx, Dm.nx), yy = row_bc(Dm, y + cy),
                  zz = dim == 2 ? 0 : wrap_idx(z + cz, Dm.nz);
        const double v = a[lin_of(Dm, xx, yy, zz)];
        g[0] += w * cx * v;
        g[1] += w * cy * v;
        g[2] += w * cz * v;
        acc += w * (v - c0);
    }
    g[0] *= 3.0;
    g[1] *= 3.0;
    g[2] *= 3.0;
    if (lap) *lap = 6.0 * acc;
}

__device__ double particle_indicator_d(const ParticleDev &pp, int x, int y, int z, const DomainDev &Dm,
                                       double r[3])
{
    const int dim = Dm.p.dim;
    double d[3] = {(double)x - pp.x[0], (double)y - pp.x[1], dim == 3 ? (double)z - pp.x[2] : 0.0};
    const int n[3] = {Dm.nx, Dm.ny, Dm.nz};
    double r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (a < dim && !(a == 1 && Dm.wall_y)) d[a] = min_image(d[a], n[a]);
        r[a] = d[a];
        r2 += d[a] * d[a];
    }
    const double lim = pp.R + Dm.p.cut;
    if (r2 >= lim * lim) return 0.0;
    return 0.5 * (1.0 + tanh(2.0 * (pp.R - sqrt(r2)) / Dm.p.D));
}

// ---- initialisation: f = f^eq (Sec. 3.3 step 1) ------------------------------------------------
//
// One thread per cell, a grid of (x blocks) x (rows): a row is one (y, z) line
// of the domain, so cell coordinates need no 64-bit division.  Arithmetic is in
// the policy's arithmetic type (double for FP64, float otherwise); the
// fixed-point rest population of the 16-bit policies is formed from the double
// phi, so the bookkeeping is exact whatever the arithmetic type.

// lattice velocities of the order-parameter (Q1) and flow (Q2) lattices
template <int DIM>
struct InitLat;
template <>
struct InitLat<2> {
    static constexpr int Q1 = 9, Q2 = 9;
    static __device__ __forceinline__ int c1(int i, int a) { return a == 0 ? LX9[i] : (a == 1 ? LY9[i] : 0); }
    static __device__ __forceinline__ int c2(int i, int a) { return c1(i, a); }
    template <class R>
    static __device__ __forceinline__ R w1(int i, R d0)
    {
        return i == 0 ? R(1) - R(2) * d0 + d0 * d0 : (i <= 4 ? R(0.5) * (d0 - d0 * d0) : R(0.25) * d0 * d0);
    }
    template <class R>
    static __device__ __forceinline__ R w2(int i, R d0) { return w1<R>(i, d0); }
    static __device__ __forceinline__ int opp(int i) { return i == 0 ? 0 : (i <= 4 ? 1 + (i + 1) % 4 : 5 + (i - 3) % 4); }
    static __device__ __forceinline__ int opp2(int i) { return opp(i); }
};
template <>
struct InitLat<3> {
    static constexpr int Q1 = 7, Q2 = 19;
    static __device__ __forceinline__ int c1(int i, int a) { return L19[i][a]; }
    static __device__ __forceinline__ int c2(int i, int a) { return L19[i][a]; }
    template <class R>
    static __device__ __forceinline__ R w1(int i, R d0)
    {
        return i == 0 ? R(1) - R(3) * d0 : R(0.5) * d0;
    }
    template <class R>
    static __device__ __forceinline__ R w2(int i, R d0)
    {
        return i == 0 ? R(1) - R(3) * d0 + R(3) * d0 * d0
                      : (i <= 6 ? R(0.5) * (d0 - R(2) * d0 * d0) : R(0.25) * d0 * d0);
    }
    // opposite directions: pairs 1-2, 3-4, ..., 17-18 (D3Q7 is the first 7)
    static __device__ __forceinline__ int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
    static __device__ __forceinline__ int opp2(int i) { return opp(i); }
};

__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// FD stencil (D2Q9 or D3Q19 with classical weights, cs^2 = 1/3) on a dense
// x-fastest double array, in arithmetic type R
template <int DIM, class R>
__device__ __forceinline__ void fd_grad_lap_r(const DomainDev &Dm, const double *a, int x, int y, int z,
                                              R g[3], R *lap)
{
    constexpr int Q = DIM == 2 ? 9 : 19;
    const R c0 = (R)a[lin_of(Dm, x, y, z)];
    R acc = R(0);
    g[0] = g[1] = g[2] = R(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int cx = InitLat<DIM>::c2(i, 0), cy = InitLat<DIM>::c2(i, 1), cz = InitLat<DIM>::c2(i, 2);
        const R w = DIM == 2 ? (i <= 4 ? R(1.0 / 9.0) : R(1.0 / 36.0)) : (i <= 6 ? R(1.0 / 18.0) : R(1.0 / 36.0));
        const int xx = wrap1(x + cx, Dm.nx), yy = row_bc(Dm, y + cy), zz = DIM == 2 ? 0 : wrap1(z + cz, Dm.nz);
        const R v = (R)a[lin_of(Dm, xx, yy, zz)];
        g[0] += w * R(cx) * v;
        g[1] += w * R(cy) * v;
        g[2] += w * R(cz) * v;
        acc += w * (v - c0);
    }
    g[0] *= R(3);
    g[1] *= R(3);
    g[2] *= R(3);
    if (lap) *lap = R(6) * acc;
}

#define PF_INIT_ROWS_BEGIN                                                                         \
    const int x = blockIdx.x * blockDim.x + threadIdx.x;                                           \
    const int rows = Dm.ny * Dm.nz;                                                                \
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {                                     \
        const int y = row % Dm.ny, z = row / Dm.ny;                                                \
        if (x >= Dm.nx) continue;                                                                  \
        const long long o = (long long)row * Dm.nx + x;

// total indicator (fixed + particles) and the stored fixed indicator; with
// particles of their own contact angle also W = sum_s cos(theta_s) phi0_s and
// V = sum_s cos(theta_s) phi0_s^3 (all solids without an own angle as one)
template <class P>
__global__ void k_init_phi0(DomainDev Dm, const double *phi0_in, double *phi0tot,
                            const ParticleDev *parts, int np, double *Wf, double *Vf, int wv)
{
    using AX = typename P::aux;
    PF_INIT_ROWS_BEGIN
        double v = phi0_in[o];
        reinterpret_cast<AX *>(Dm.phi0)[cell_of(Dm, x, y, z)] = (AX)v;
        double dflt = v, w = 0.0, vv = 0.0;
        for (int k = 0; k < np; ++k) {
            double r[3];
            const double pk = particle_indicator_d(parts[k], x, y, z, Dm, r);
            v += pk;
            if (parts[k].own) {
                w += parts[k].ct * pk;
                vv += parts[k].ct * pk * pk * pk;
            } else {
                dflt += pk;
            }
        }
        phi0tot[o] = v;
        if (wv) {
            Wf[o] = Dm.p.cos_t * dflt + w;
            Vf[o] = Dm.p.cos_t * dflt * dflt * dflt + vv;
        }
    }
}

// chemical potential of Eq. (9) from the initial phi (with own particle
// angles: the wetting terms summed per solid through W and V)
template <int DIM, class R>
__global__ void k_init_mu(DomainDev Dm, const double *phi, const double *phi0tot, double *mu, const double *Wf,
                          const double *Vf, int wv)
{
    const DevParams &p = Dm.p;
    PF_INIT_ROWS_BEGIN
        R g[3], lp, lp0;
        fd_grad_lap_r<DIM, R>(Dm, phi, x, y, z, g, &lp);
        const R ph = (R)phi[o], p0 = (R)phi0tot[o];
        const R base = (R)p.c_dw * ph * (ph - R(1)) * (ph + R(1)) - (R)p.c_lap * lp + (R)p.c_pen * p0 * p0 * ph;
        if (!wv) {
            fd_grad_lap_r<DIM, R>(Dm, phi0tot, x, y, z, g, &lp0);
            mu[o] = (double)(base + (R)p.c_wet * p0 * (R(3) * ph * ph + p0 * p0 - R(1)) - (R)p.c_wlap * lp0);
        } else {
            R lw;
            fd_grad_lap_r<DIM, R>(Dm, Wf, x, y, z, g, &lw);
            const R W = (R)Wf[o], V = (R)Vf[o];
            mu[o] = (double)(base + (R)p.c_dw * (R(3) * ph * ph * W + V - W) - (R)p.c_lap * lw);
        }
    }
}

// f = f^eq (Eqs. 30, 32) stored for pull streaming: population i of cell x is
// written at x - c_i so that the first step reads f^eq_i(x); where x - c_i
// lies beyond a wall the first step bounces back, reading population opp(i)
// of x itself, so it is written there.  Lagged fields equal the initial ones.
template <class P, int DIM>
__global__ void k_init_f(DomainDev Dm, int *flags, const double *phi, const double *u, const double *Pin,
                         const double *mu)
{
    using ST = typename P::store;
    using AX = typename P::aux;
    using R = typename P::real;
    using LT = InitLat<DIM>;
    const DevParams &p = Dm.p;
    const long long N = (long long)Dm.nx * Dm.ny * Dm.nz;
    ST *f = reinterpret_cast<ST *>(Dm.f[0]);
    AX *aux = reinterpret_cast<AX *>(Dm.aux[0]);
    long long *rest = reinterpret_cast<long long *>(Dm.rest[0]);
    const long long plane = Dm.plane;
    const R cs2 = (R)p.cs2, cs4 = cs2 * cs2, d0 = (R)p.d0;
    PF_INIT_ROWS_BEGIN
        R g[3];
        const bool cac = p.phase_model == 1;  // conservative Allen-Cahn option
        fd_grad_lap_r<DIM, R>(Dm, cac ? phi : mu, x, y, z, g, nullptr);
        if (cac) {
            // S from grad phi - theta n, theta = (2/D)(1 - phi^2), n = grad phi/|grad phi|
            const R pc = (R)phi[o];
            R g2 = R(0);
#pragma unroll
            for (int a = 0; a < DIM; ++a) g2 += g[a] * g[a];
            const R th = R(2.0 / p.D) * (R(1) - pc * pc);
            const R inv = g2 > R(1e-24) ? R(1) / sqrt(g2) : R(0);
#pragma unroll
            for (int a = 0; a < DIM; ++a) g[a] = g[a] - th * g[a] * inv;
        }
        const R Md = (R)p.Mdrho;
        const R S[3] = {Md * g[0], Md * g[1], DIM == 3 ? Md * g[2] : R(0)};
        R uu[3] = {R(0), R(0), R(0)};
        if (u)
#pragma unroll
            for (int a = 0; a < DIM; ++a) uu[a] = (R)u[a * N + o];
        const double phd = phi[o];
        const R ph = (R)phd;
        const R rho = (R)p.drho * ph + (R)p.rhom;
        const R Pv = Pin ? (R)Pin[o] : R(0);
        const R em = cac ? ph : (R)p.eta * (R)mu[o];
        // order-parameter lattice
        int rest_s = 0, bad = 0;
#pragma unroll
        for (int i = 0; i < LT::Q1; ++i) {
            R cu = R(0);
#pragma unroll
            for (int a = 0; a < DIM; ++a) cu += R(LT::c1(i, a)) * uu[a];
            const R wi = LT::template w1<R>(i, d0);
            const R fe = i == 0 ? ph + (wi - R(1)) * em : wi * em + wi * cu * ph / cs2;
            const int ys = y - LT::c1(i, 1);
            const bool bb = Dm.wall_y && (ys < 0 || ys >= Dm.ny);
            const int xx = bb ? x : wrap1(x - LT::c1(i, 0), Dm.nx), yy = bb ? y : wrap1(ys, Dm.ny),
                      zz = DIM == 3 ? (bb ? z : wrap1(z - LT::c1(i, 2), Dm.nz)) : 0;
            const long long id = cell_of(Dm, xx, yy, zz);
            const int slot = bb ? LT::opp(i) : i;
            if constexpr (P::MIX) {
                if (i == 0) continue;
                ST q = Conv<P>::st(fe, (R)p.scale[0]);
                if constexpr (P::id == 3) q = bf16_flush(q);
                rest_s += fix24_sat<ST>(q, &bad);
                f[slot * plane + id] = q;
            } else {
                f[slot * plane + id] = (ST)fe;
            }
        }
        if constexpr (P::MIX) rest[cell_of(Dm, x, y, z)] = fixed_of_double(phd) - fix24_to_rest(rest_s, p.klog2[0]);
        if (bad) atomicOr(flags, 2);
        // flow lattice
#pragma unroll
        for (int i = 0; i < LT::Q2; ++i) {
            R cu = R(0), diag = R(0), off = R(0);
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const R ca = R(LT::c2(i, a));
                cu += ca * uu[a];
                diag += (ca * ca - cs2) * (rho * uu[a] * uu[a] - S[a] * uu[a]);
#pragma unroll
                for (int b = a + 1; b < DIM; ++b)
                    off += ca * R(LT::c2(i, b)) * (rho * uu[a] * uu[b] - R(0.5) * (S[a] * uu[b] + uu[a] * S[b]));
            }
            const R wi = LT::template w2<R>(i, d0);
            const R lam = (i == 0 ? wi - R(1) : wi) * Pv / cs2;
            const R fe = lam + wi * rho * cu / cs2 + wi * (diag / (cs2 - cs4) + off / cs4);
            const int ys = y - LT::c2(i, 1);
            const bool bb = Dm.wall_y && (ys < 0 || ys >= Dm.ny);
            const int xx = bb ? x : wrap1(x - LT::c2(i, 0), Dm.nx), yy = bb ? y : wrap1(ys, Dm.ny),
                      zz = DIM == 3 ? (bb ? z : wrap1(z - LT::c2(i, 2), Dm.nz)) : 0;
            const long long id = cell_of(Dm, xx, yy, zz);
            const int slot = LT::Q1 + (bb ? LT::opp2(i) : i);
            if constexpr (P::MIX) {
                f[slot * plane + id] = Conv<P>::st(fe, (R)p.scale[1]);
            } else {
                f[slot * plane + id] = (ST)fe;
            }
        }
        const long long id = cell_of(Dm, x, y, z);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            aux[a * plane + id] = (AX)uu[a];
            aux[(DIM + a) * plane + id] = (AX)S[a];
        }
        aux[2 * DIM * plane + id] = (AX)ph;
    }
}
#undef PF_INIT_ROWS_BEGIN

// ---- diagnostics --------------------------------------------------------------------------------

// macro = [phi, rho, u (dim), P, mu, phi0] (double, x-fastest)
__global__ void k_diag_partial(DomainDev Dm, double *partial, int wv)
{
    const DevParams &p = Dm.p;
    const int dim = p.dim;
    const long long N = (long long)Dm.nx * Dm.ny * Dm.nz;
    const double *phi = Dm.macro, *rho = Dm.macro + N, *u = Dm.macro + 2 * N;
    const double *phi0 = Dm.macro + (2 + dim + 2) * N;
    const double *Wf = phi0 + N, *Vf = phi0 + 2 * N;  // own particle angles only
    double acc[3] = {0.0, 0.0, 0.0};
    // each thread walks a fixed contiguous range: deterministic order
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long per = (N + nthr - 1) / nthr;
    const long long gtid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long o = gtid * per; o < N && o < (gtid + 1) * per; ++o) {
        const int x = (int)(o % Dm.nx), y = (int)((o / Dm.nx) % Dm.ny), z = (int)(o / ((long long)Dm.nx * Dm.ny));
        double g[3], g0[3];
        fd_grad_lap(Dm, phi, x, y, z, g, nullptr);
        fd_grad_lap(Dm, wv ? Wf : phi0, x, y, z, g0, nullptr);
        const double ph = phi[o], p0 = phi0[o];
        double g2 = 0.0, g0g = 0.0, u2 = 0.0;
        for (int a = 0; a < dim; ++a) {
            g2 += g[a] * g[a];
            g0g += g0[a] * g[a];
            u2 += u[a * N + o] * u[a * N + o];
        }
        const double s = p.sigma, D = p.D, ct = p.cos_t;
        double e = 3.0 * s / (4.0 * D) * (1.0 - ph) * (1.0 - ph) * (1.0 + ph) * (1.0 + ph) +
                   3.0 * D * s / 16.0 * g2 + 9.0 * s / (2.0 * D) * p0 * p0 * ph * ph;
        if (!wv)
            e += 3.0 * s * ct / D * p0 * ph * (ph * ph + p0 * p0 - 1.0) + 3.0 * D * s * ct / 8.0 * g0g;
        else  // wetting energy summed per solid with its own angle (g0 = grad W)
            e += 3.0 * s / D * (ph * (ph * ph - 1.0) * Wf[o] + ph * Vf[o]) + 3.0 * D * s / 8.0 * g0g;
        acc[0] += ph;
        acc[1] += e;
        acc[2] += 0.5 * rho[o] * u2;
    }
    __shared__ double red[256][3];
    for (int c = 0; c < 3; ++c) red[threadIdx.x][c] = acc[c];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int c = 0; c < 3; ++c) red[threadIdx.x][c] += red[threadIdx.x + s][c];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) partial[blockIdx.x * 3 + c] = red[0][c];
}

// interface normal n = grad phi / |grad phi| from the macroscopic phi (central
// isotropic stencil, mirror rows at walls); 0 where |grad phi|^2 <= 1e-24
__global__ void k_normal(DomainDev Dm, double *n)
{
    const int dim = Dm.p.dim;
    const long long N = (long long)Dm.nx * Dm.ny * Dm.nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < N; o += stride) {
        const int x = (int)(o % Dm.nx), y = (int)((o / Dm.nx) % Dm.ny), z = (int)(o / ((long long)Dm.nx * Dm.ny));
        double g[3];
        fd_grad_lap(Dm, Dm.macro, x, y, z, g, nullptr);
        double g2 = 0.0;
        for (int a = 0; a < dim; ++a) g2 += g[a] * g[a];
        const double inv = g2 > 1e-24 ? 1.0 / sqrt(g2) : 0.0;
        for (int a = 0; a < dim; ++a) n[a * N + o] = g[a] * inv;
    }
}

// Split of a particle domain's tiles (tx x ty cells) into those some
// particle's indicator may reach (the same conservative test as the
// single-cell step: its tile + 2 frame against R + cut + 1, minimum image),
// sel[t] = 1, and the rest, sel[t] = 0, whose force partials are zeroed here
// (the step that runs them computes none).  One thread per tile.
__global__ void k_split_tiles(StepArgs A, int tx, int ty, unsigned char *sel)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.ntiles) return;
    const DomainDev &Dm = A.doms[A.tile_dom[t]];
    const int2 txy = A.tile_xy[t];
    const int nx = Dm.nx, ny = Dm.ny;
    const int x0 = txy.x * tx, y0 = txy.y * ty;
    bool near = false;
    for (int k = 0; k < A.np && !near; ++k) {
        const ParticleDev &pp = A.parts[k];
        double dx = (x0 + 0.5 * (tx - 1)) - pp.x[0], dy = (y0 + 0.5 * (ty - 1)) - pp.x[1];
        dx = min_image(dx, nx);
        dy = min_image(dy, ny);
        const double ex = fmax(fabs(dx) - (0.5 * tx + 2.0), 0.0);
        const double ey = fmax(fabs(dy) - (0.5 * ty + 2.0), 0.0);
        const double lim = pp.R + Dm.p.cut + 1.0;
        near = ex * ex + ey * ey < lim * lim;
    }
    sel[t] = near ? 1 : 0;
    if (!near)
        for (int c = 0; c < 6 * A.np; ++c) A.partials[(long long)c * A.ntiles + t] = 0.0;
}

void launch_split_tiles(const StepArgs &a, int tx, int ty, unsigned char *sel, cudaStream_t s)
{
    k_split_tiles<<<(a.ntiles + 255) / 256, 256, 0, s>>>(a, tx, ty, sel);
    count_launches(1);
}

__global__ void k_diag_final(const double *partial, int nblocks, double *out)
{
    __shared__ double red[256][3];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int c = 0; c < 3; ++c) acc[c] += partial[b * 3 + c];
    for (int c = 0; c < 3; ++c) red[threadIdx.x][c] = acc[c];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int c = 0; c < 3; ++c) red[threadIdx.x][c] += red[threadIdx.x + s][c];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) out[c] = red[0][c];
}

// ---- particles: repulsion (Sec. 4.5), per-tile partial sums, Newton-Euler (Eqs. 26, 28) --------
// Force on particle k from the others (as printed: (x_k - x_j)/eps times
// (R_k + R_j + xi - d)^2 within xi of contact, (R_k + R_j - d) overlapping),
// minimum image, and from the nearest wall (the same form with 2 R_k and
// eps/2, x_j the mirror image of particle k across that wall: a box wall at
// y = -1/2 or ny - 1/2, or the circle p.wall_circle along its radius); from
// the positions before this step's update.
// One block per particle k: thread 0 takes the wall term, thread 1 + j the
// pair with particle j, then a fixed-order sum (each warp's shuffle tree, the
// warps in order).  FP64 throughout.
constexpr int REP_THREADS = 96;
static_assert(REP_THREADS >= PF_MAX_PARTICLES + 1, "one thread per partner and one for the wall");
__global__ void __launch_bounds__(REP_THREADS) k_particle_repulsion(const ParticleDev *parts, int np, DevParams p,
                                                                    int nx, int ny, int nz, int wall_y,
                                                                    double *frep)
{
    const int k = blockIdx.x, tid = threadIdx.x;
    if (k >= np) return;
    __shared__ double red[REP_THREADS / 32][3];
    double acc[3] = {0.0, 0.0, 0.0};
    if (p.rep_eps > 0.0) {
        if (tid == 0) {
            double best = INFINITY, dw0 = 0.0, dw1 = 0.0;  // x_k - x'_k
            if (wall_y) {
                const double y = parts[k].x[1];
                const double lo = 2.0 * (y + 0.5), hi = 2.0 * (ny - 0.5 - y);
                if (lo < best) {
                    best = lo;
                    dw0 = 0.0;
                    dw1 = lo;
                }
                if (hi < best) {
                    best = hi;
                    dw0 = 0.0;
                    dw1 = -hi;
                }
            }
            if (p.dim == 2 && p.wall_circle[2] > 0.0) {
                const double ex = parts[k].x[0] - p.wall_circle[0], ey = parts[k].x[1] - p.wall_circle[1];
                const double r = sqrt(ex * ex + ey * ey);
                if (r > 0.0) {
                    const double dd = 2.0 * fabs(p.wall_circle[2] - r);
                    if (dd < best) {
                        const double s = (r - (2.0 * p.wall_circle[2] - r)) / r;
                        best = dd;
                        dw0 = s * ex;
                        dw1 = s * ey;
                    }
                }
            }
            if (best < INFINITY) {
                const double rr = 2.0 * parts[k].R;
                double f = 0.0;
                if (best <= rr + p.rep_xi) {
                    if (best >= rr) f = (rr + p.rep_xi - best) * (rr + p.rep_xi - best) / (0.5 * p.rep_eps);
                    else f = (rr - best) / (0.5 * p.rep_eps);
                }
                acc[0] = f * dw0;
                acc[1] = f * dw1;
            }
        } else if (tid - 1 < np && tid - 1 != k) {
            const int j = tid - 1;
            const int n[3] = {nx, ny, nz};
            double dx[3], d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double v = a < p.dim ? parts[k].x[a] - parts[j].x[a] : 0.0;
                // minimum image (the division only where it can shift: FP64 is slow here)
                if (a < p.dim && !(a == 1 && wall_y) && (v >= 0.5 * n[a] || v <= -0.5 * n[a]))
                    v -= n[a] * floor(v / n[a] + 0.5);
                dx[a] = v;
                d2 += v * v;
            }
            const double rr = parts[k].R + parts[j].R, reach = rr + p.rep_xi;
            if (d2 <= reach * reach) {  // (the pairs farther apart get no force: no square root)
                const double dist = sqrt(d2);
                double f = 0.0;
                if (dist <= reach) {
                    if (dist >= rr) f = (reach - dist) * (reach - dist) / p.rep_eps;
                    else f = (rr - dist) / p.rep_eps;
                }
                for (int a = 0; a < 3; ++a) acc[a] = f * dx[a];
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double v = acc[a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[tid >> 5][a] = v;
    }
    __syncthreads();
    if (tid < 3) {
        double v = 0.0;
        for (int w = 0; w < REP_THREADS / 32; ++w) v += red[w][tid];
        frep[3 * k + tid] = v;
    }
}

// One block per particle; each thread sums a fixed strided set of tiles, then
// each warp's shuffle tree and the warps in order (the order depends only on
// the tile count).
constexpr int UPDATE_THREADS = 256;
// sel: optional per-tile flags; tiles with sel[t] == 0 hold zero partials
// and are skipped (adding them would not change the sums)
__global__ void __launch_bounds__(UPDATE_THREADS) k_particle_update(ParticleDev *parts, int np,
                                                                    const double *partials, int ntiles,
                                  DevParams p, const double *frep, const unsigned char *sel)
{
    const int k = blockIdx.x;
    if (k >= np) return;
    __shared__ double wred[UPDATE_THREADS / 32][6];
    __shared__ double red[1][6];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        if (sel && !sel[t]) continue;
        // component c of tile t: partials[(6 k + c) ntiles + t] (consecutive
        // threads read consecutive tiles); 2D: components 2, 3, 4 stay zero
        const double *q = partials + (long long)k * 6 * ntiles + t;
        acc[0] += q[0];
        acc[1] += q[(long long)ntiles];
        acc[5] += q[5LL * ntiles];
        if (p.dim == 3) {
            acc[2] += q[2LL * ntiles];
            acc[3] += q[3LL * ntiles];
            acc[4] += q[4LL * ntiles];
        }
    }
    // (FP64 adds are slow on this part: 2D sums only F_x, F_y, T_z)
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        if (p.dim == 2 && c >= 2 && c <= 4) {
            if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5][c] = 0.0;
            continue;
        }
        double v = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = 0.0;
        for (int w = 0; w < UPDATE_THREADS / 32; ++w) v += wred[w][threadIdx.x];
        red[0][threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    ParticleDev &pp = parts[k];
    const double R = pp.R;
    double Vp, Mp, Ip;
    if (p.dim == 2) {
        Vp = 3.14159265358979323846 * R * R;
        Mp = pp.rho_p * Vp;
        Ip = 0.5 * Mp * R * R;
    } else {
        Vp = 4.0 / 3.0 * 3.14159265358979323846 * R * R * R;
        Mp = pp.rho_p * Vp;
        Ip = 0.4 * Mp * R * R;
    }
    const double rho_bar = p.rhom;  // fluid density at phi = 0
    const double If = Ip * rho_bar / pp.rho_p;
    double a[3], al[3];
    for (int c = 0; c < 3; ++c) {
        const double Fin = rho_bar * Vp * (pp.u[c] - pp.u_prev[c]);
        const double Tin = If * (pp.w[c] - pp.w_prev[c]);
        a[c] = (red[0][c] + frep[3 * k + c] + Fin + (1.0 - rho_bar / pp.rho_p) * Mp * p.g[c]) / Mp;
        al[c] = (red[0][3 + c] + Tin) / Ip;
    }
    if (p.dim == 2) {
        a[2] = 0.0;
        al[0] = al[1] = 0.0;
    }
    for (int c = 0; c < 3; ++c) {
        pp.F[c] = red[0][c];
        pp.T[c] = red[0][3 + c];
        pp.x[c] += pp.u[c];
        pp.u_prev[c] = pp.u[c];
        pp.w_prev[c] = pp.w[c];
        // held components keep their value (bit 0: all; bits 1-3: translation
        // along x, y, z; bit 4: rotation)
        if (!(pp.prescribed & 1) && !(pp.prescribed & (2 << c))) pp.u[c] += a[c];
        if (!(pp.prescribed & 1) && !(pp.prescribed & 16)) pp.w[c] += al[c];
    }
}

// ---- host launchers ---------------------------------------------------------------------------
static int grid_for(long long N, int bs)
{
    long long g = (N + bs - 1) / bs;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return (int)g;
}

template <class P>
static void init_impl(const DomainDev &Dm, int *flags, const double *phi0, const double *phi, const double *u,
                      const double *Pin, double *tmp, const ParticleDev *parts, int np, int wv,
                      cudaStream_t s)
{
    using R = typename P::real;
    const long long N = (long long)Dm.nx * Dm.ny * Dm.nz;
    double *phi0tot = tmp, *mu = tmp + N, *Wf = tmp + 2 * N, *Vf = tmp + 3 * N;
    // x blocks of 128 cells, one grid row per domain row (at most 65535, the
    // kernels stride over the rest)
    const int bs = 128;
    const int rows = Dm.ny * Dm.nz;
    const dim3 g((Dm.nx + bs - 1) / bs, rows < 65535 ? rows : 65535);
    k_init_phi0<P><<<g, bs, 0, s>>>(Dm, phi0, phi0tot, parts, np, Wf, Vf, wv);
    if (Dm.p.dim == 2) {
        k_init_mu<2, R><<<g, bs, 0, s>>>(Dm, phi, phi0tot, mu, Wf, Vf, wv);
        k_init_f<P, 2><<<g, bs, 0, s>>>(Dm, flags, phi, u, Pin, mu);
    } else {
        k_init_mu<3, R><<<g, bs, 0, s>>>(Dm, phi, phi0tot, mu, Wf, Vf, wv);
        k_init_f<P, 3><<<g, bs, 0, s>>>(Dm, flags, phi, u, Pin, mu);
    }
    count_launches(3);
}

void launch_init(int prec, const DomainDev &Dm, int *flags, const double *phi0, const double *phi, const double *u,
                 const double *Pin, double *tmp, const ParticleDev *parts, int np, int wv, cudaStream_t s)
{
    switch (prec) {
    case 0: init_impl<P64>(Dm, flags, phi0, phi, u, Pin, tmp, parts, np, wv, s); break;
    case 1: init_impl<P32>(Dm, flags, phi0, phi, u, Pin, tmp, parts, np, wv, s); break;
    case 2: init_impl<PMixH>(Dm, flags, phi0, phi, u, Pin, tmp, parts, np, wv, s); break;
    default: init_impl<PMixB>(Dm, flags, phi0, phi, u, Pin, tmp, parts, np, wv, s); break;
    }
}

void launch_normal(const DomainDev &Dm, double *n, cudaStream_t s)
{
    const long long N = (long long)Dm.nx * Dm.ny * Dm.nz;
    k_normal<<<grid_for(N, 256), 256, 0, s>>>(Dm, n);
    count_launches(1);
}

int diag_blocks() { return 120; }

void launch_diag(const DomainDev &Dm, double *partial, double *out, int wv, cudaStream_t s)
{
    k_diag_partial<<<diag_blocks(), 256, 0, s>>>(Dm, partial, wv);
    k_diag_final<<<1, 256, 0, s>>>(partial, diag_blocks(), out);
    count_launches(2);
}

void launch_particle_update(ParticleDev *parts, int np, const double *partials, int ntiles,
                            const DevParams &p, double *frep, int nx, int ny, int nz, int wall_y,
                            const unsigned char *sel, cudaStream_t s)
{
    k_particle_repulsion<<<np, REP_THREADS, 0, s>>>(parts, np, p, nx, ny, nz, wall_y, frep);
    k_particle_update<<<np, UPDATE_THREADS, 0, s>>>(parts, np, partials, ntiles, p, frep, sel);
    count_launches(2);
}

}  // namespace pf
