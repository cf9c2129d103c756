// Initialisation (Sec. 3.3 step 1), FP64 diagnostics (Eq. 8, Sec. 2.3) and the
// rigid-particle update (Eqs. 26-28) for 2D and 3D domains.
//
// These kernels run once per call (init, diagnostics) or once per step on a
// handful of particles; they are written for clarity, in double precision.
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

struct Lat {
    int Q;
    int c[19][3];
    double w[19];
};

__device__ void lattice_of(int dim, int which, double d0, Lat &L)
{
    if (dim == 2) {
        L.Q = 9;
        for (int i = 0; i < 9; ++i) {
            L.c[i][0] = LX9[i];
            L.c[i][1] = LY9[i];
            L.c[i][2] = 0;
        }
        L.w[0] = 1.0 - 2.0 * d0 + d0 * d0;
        for (int i = 1; i <= 4; ++i) L.w[i] = 0.5 * (d0 - d0 * d0);
        for (int i = 5; i <= 8; ++i) L.w[i] = 0.25 * d0 * d0;
    } else if (which == 1) {  // D3Q7, order parameter
        L.Q = 7;
        for (int i = 0; i < 7; ++i)
            for (int a = 0; a < 3; ++a) L.c[i][a] = L19[i][a];
        L.w[0] = 1.0 - 3.0 * d0;
        for (int i = 1; i < 7; ++i) L.w[i] = 0.5 * d0;
    } else {  // D3Q19, flow
        L.Q = 19;
        for (int i = 0; i < 19; ++i)
            for (int a = 0; a < 3; ++a) L.c[i][a] = L19[i][a];
        L.w[0] = 1.0 - 3.0 * d0 + 3.0 * d0 * d0;
        for (int i = 1; i <= 6; ++i) L.w[i] = 0.5 * (d0 - 2.0 * d0 * d0);
        for (int i = 7; i < 19; ++i) L.w[i] = 0.25 * d0 * d0;
    }
}

__device__ __forceinline__ long long cell_of(const DomainDev &Dm, int x, int y, int z)
{
    return ((long long)z * Dm.ny + y) * Dm.pitch + x;
}

__device__ __forceinline__ long long lin_of(const DomainDev &Dm, int x, int y, int z)
{
    return ((long long)z * Dm.ny + y) * Dm.nx + x;
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
        const int xx = wrap_idx(x + cx, Dm.nx), yy = wrap_idx(y + cy, Dm.ny),
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
        if (a < dim) d[a] -= n[a] * rint(d[a] / n[a]);
        r[a] = d[a];
        r2 += d[a] * d[a];
    }
    const double lim = pp.R + Dm.p.cut;
    if (r2 >= lim * lim) return 0.0;
    return 0.5 * (1.0 + tanh(2.0 * (pp.R - sqrt(r2)) / Dm.p.D));
}

// ---- initialisation: f = f^eq (Sec. 3.3 step 1) ------------------------------------------------

// total indicator (fixed + particles) and the stored fixed indicator
template <class P>
__global__ void k_init_phi0(DomainDev Dm, const double *phi0_in, double *phi0tot,
                            const ParticleDev *parts, int np)
{
    using AX = typename P::aux;
    const long long N = (long long)Dm.nx * Dm.ny * Dm.nz;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < N;
         o += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(o % Dm.nx), y = (int)((o / Dm.nx) % Dm.ny), z = (int)(o / ((long long)Dm.nx * Dm.ny));
        double v = phi0_in[o];
        reinterpret_cast<AX *>(Dm.phi0)[cell_of(Dm, x, y, z)] = (AX)v;
        for (int k = 0; k < np; ++k) {
            double r[3];
            v += particle_indicator_d(parts[k], x, y, z, Dm, r);
        }
        phi0tot[o] = v;
    }
}

// chemical potential of Eq. (9) from the initial phi
__global__ void k_init_mu(DomainDev Dm, const double *phi, const double *phi0tot, double *mu)
{
    const DevParams &p = Dm.p;
    const long long N = (long long)Dm.nx * Dm.ny * Dm.nz;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < N;
         o += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(o % Dm.nx), y = (int)((o / Dm.nx) % Dm.ny), z = (int)(o / ((long long)Dm.nx * Dm.ny));
        double g[3], lp, lp0;
        fd_grad_lap(Dm, phi, x, y, z, g, &lp);
        fd_grad_lap(Dm, phi0tot, x, y, z, g, &lp0);
        const double ph = phi[o], p0 = phi0tot[o];
        mu[o] = p.c_dw * ph * (ph - 1.0) * (ph + 1.0) - p.c_lap * lp + p.c_pen * p0 * p0 * ph +
                p.c_wet * p0 * (3.0 * ph * ph + p0 * p0 - 1.0) - p.c_wlap * lp0;
    }
}

// f = f^eq (Eqs. 30, 32) stored for pull streaming: population i of cell x is
// written at x - c_i so that the first step reads f^eq_i(x).  Lagged fields
// equal the initial ones.
template <class P>
__global__ void k_init_f(DomainDev Dm, const double *phi, const double *u, const double *Pin,
                         const double *mu)
{
    using ST = typename P::store;
    using AX = typename P::aux;
    const DevParams &p = Dm.p;
    const int dim = p.dim;
    const long long N = (long long)Dm.nx * Dm.ny * Dm.nz;
    Lat L1, L2;
    lattice_of(dim, 1, p.d0, L1);
    lattice_of(dim, 2, p.d0, L2);
    ST *f = reinterpret_cast<ST *>(Dm.f[0]);
    AX *aux = reinterpret_cast<AX *>(Dm.aux[0]);
    long long *rest = reinterpret_cast<long long *>(Dm.rest[0]);
    const long long plane = Dm.plane;
    const double cs2 = p.cs2, cs4 = cs2 * cs2;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < N;
         o += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(o % Dm.nx), y = (int)((o / Dm.nx) % Dm.ny), z = (int)(o / ((long long)Dm.nx * Dm.ny));
        double g[3];
        fd_grad_lap(Dm, mu, x, y, z, g, nullptr);
        double S[3] = {p.Mdrho * g[0], p.Mdrho * g[1], dim == 3 ? p.Mdrho * g[2] : 0.0};
        double uu[3] = {0.0, 0.0, 0.0};
        if (u)
            for (int a = 0; a < dim; ++a) uu[a] = u[a * N + o];
        const double ph = phi[o];
        const double rho = p.drho * ph + p.rhom;
        const double Pv = Pin ? Pin[o] : 0.0;
        const double em = p.eta * mu[o];
        // order-parameter lattice
        const long long rest_phi = fixed_of_double(ph);
        int rest_s = 0, bad = 0;
        for (int i = 0; i < L1.Q; ++i) {
            double cu = 0.0;
            for (int a = 0; a < dim; ++a) cu += L1.c[i][a] * uu[a];
            const double fe = i == 0 ? ph + (L1.w[0] - 1.0) * em : L1.w[i] * em + L1.w[i] * cu * ph / cs2;
            const int xx = wrap_idx(x - L1.c[i][0], Dm.nx), yy = wrap_idx(y - L1.c[i][1], Dm.ny),
                      zz = dim == 3 ? wrap_idx(z - L1.c[i][2], Dm.nz) : 0;
            const long long id = cell_of(Dm, xx, yy, zz);
            if constexpr (P::MIX) {
                if (i == 0) continue;
                ST q = Conv<P>::st((float)fe, (float)p.scale[0]);
                if constexpr (P::id == 3) q = bf16_flush(q);
                rest_s += fix24<ST>(q, &bad);
                f[i * plane + id] = q;
            } else {
                f[i * plane + id] = (ST)fe;
            }
        }
        if constexpr (P::MIX) rest[cell_of(Dm, x, y, z)] = rest_phi - fix24_to_rest(rest_s, p.klog2[0]);
        (void)bad;
        // flow lattice
        for (int i = 0; i < L2.Q; ++i) {
            double cu = 0.0, diag = 0.0, off = 0.0;
            for (int a = 0; a < dim; ++a) {
                const double ca = L2.c[i][a];
                cu += ca * uu[a];
                diag += (ca * ca - cs2) * (rho * uu[a] * uu[a] - S[a] * uu[a]);
                for (int b = a + 1; b < dim; ++b)
                    off += ca * L2.c[i][b] * (rho * uu[a] * uu[b] - 0.5 * (S[a] * uu[b] + uu[a] * S[b]));
            }
            const double lam = (i == 0 ? L2.w[0] - 1.0 : L2.w[i]) * Pv / cs2;
            const double fe = lam + L2.w[i] * rho * cu / cs2 + L2.w[i] * (diag / (cs2 - cs4) + off / cs4);
            const int xx = wrap_idx(x - L2.c[i][0], Dm.nx), yy = wrap_idx(y - L2.c[i][1], Dm.ny),
                      zz = dim == 3 ? wrap_idx(z - L2.c[i][2], Dm.nz) : 0;
            const long long id = cell_of(Dm, xx, yy, zz);
            if constexpr (P::MIX) {
                ST q = Conv<P>::st((float)fe, (float)p.scale[1]);
                f[(L1.Q + i) * plane + id] = q;
            } else {
                f[(L1.Q + i) * plane + id] = (ST)fe;
            }
        }
        const long long id = cell_of(Dm, x, y, z);
        for (int a = 0; a < dim; ++a) {
            aux[a * plane + id] = (AX)uu[a];
            aux[(dim + a) * plane + id] = (AX)S[a];
        }
        aux[2 * dim * plane + id] = (AX)ph;
    }
}

// ---- diagnostics --------------------------------------------------------------------------------

// macro = [phi, rho, u (dim), P, mu, phi0] (double, x-fastest)
__global__ void k_diag_partial(DomainDev Dm, double *partial)
{
    const DevParams &p = Dm.p;
    const int dim = p.dim;
    const long long N = (long long)Dm.nx * Dm.ny * Dm.nz;
    const double *phi = Dm.macro, *rho = Dm.macro + N, *u = Dm.macro + 2 * N;
    const double *phi0 = Dm.macro + (2 + dim + 2) * N;
    double acc[3] = {0.0, 0.0, 0.0};
    // each thread walks a fixed contiguous range: deterministic order
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long per = (N + nthr - 1) / nthr;
    const long long gtid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long o = gtid * per; o < N && o < (gtid + 1) * per; ++o) {
        const int x = (int)(o % Dm.nx), y = (int)((o / Dm.nx) % Dm.ny), z = (int)(o / ((long long)Dm.nx * Dm.ny));
        double g[3], g0[3];
        fd_grad_lap(Dm, phi, x, y, z, g, nullptr);
        fd_grad_lap(Dm, phi0, x, y, z, g0, nullptr);
        const double ph = phi[o], p0 = phi0[o];
        double g2 = 0.0, g0g = 0.0, u2 = 0.0;
        for (int a = 0; a < dim; ++a) {
            g2 += g[a] * g[a];
            g0g += g0[a] * g[a];
            u2 += u[a * N + o] * u[a * N + o];
        }
        const double s = p.sigma, D = p.D, ct = p.cos_t;
        const double e = 3.0 * s / (4.0 * D) * (1.0 - ph) * (1.0 - ph) * (1.0 + ph) * (1.0 + ph) +
                         3.0 * D * s / 16.0 * g2 + 9.0 * s / (2.0 * D) * p0 * p0 * ph * ph +
                         3.0 * s * ct / D * p0 * ph * (ph * ph + p0 * p0 - 1.0) +
                         3.0 * D * s * ct / 8.0 * g0g;
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

// ---- particles: reduce per-tile partial sums, Newton-Euler (Eqs. 26, 28) ----------------------
__global__ void k_particle_update(ParticleDev *parts, int np, const double *partials, int ntiles,
                                  DevParams p)
{
    const int k = blockIdx.x;
    if (k >= np) return;
    __shared__ double red[256][6];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
        for (int c = 0; c < 6; ++c) acc[c] += partials[((long long)t * np + k) * 6 + c];
    for (int c = 0; c < 6; ++c) red[threadIdx.x][c] = acc[c];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int c = 0; c < 6; ++c) red[threadIdx.x][c] += red[threadIdx.x + s][c];
        __syncthreads();
    }
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
        a[c] = (red[0][c] + Fin + (1.0 - rho_bar / pp.rho_p) * Mp * p.g[c]) / Mp;
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
        pp.u[c] += a[c];
        pp.w_prev[c] = pp.w[c];
        pp.w[c] += al[c];
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
static void init_impl(const DomainDev &Dm, const double *phi0, const double *phi, const double *u,
                      const double *Pin, double *tmp, const ParticleDev *parts, int np,
                      cudaStream_t s)
{
    const long long N = (long long)Dm.nx * Dm.ny * Dm.nz;
    double *phi0tot = tmp, *mu = tmp + N;
    const int g = grid_for(N, 256);
    k_init_phi0<P><<<g, 256, 0, s>>>(Dm, phi0, phi0tot, parts, np);
    k_init_mu<<<g, 256, 0, s>>>(Dm, phi, phi0tot, mu);
    k_init_f<P><<<g, 256, 0, s>>>(Dm, phi, u, Pin, mu);
    count_launches(3);
}

void launch_init(int prec, const DomainDev &Dm, const double *phi0, const double *phi, const double *u,
                 const double *Pin, double *tmp, const ParticleDev *parts, int np, cudaStream_t s)
{
    switch (prec) {
    case 0: init_impl<P64>(Dm, phi0, phi, u, Pin, tmp, parts, np, s); break;
    case 1: init_impl<P32>(Dm, phi0, phi, u, Pin, tmp, parts, np, s); break;
    case 2: init_impl<PMixH>(Dm, phi0, phi, u, Pin, tmp, parts, np, s); break;
    default: init_impl<PMixB>(Dm, phi0, phi, u, Pin, tmp, parts, np, s); break;
    }
}

int diag_blocks() { return 120; }

void launch_diag(const DomainDev &Dm, double *partial, double *out, cudaStream_t s)
{
    k_diag_partial<<<diag_blocks(), 256, 0, s>>>(Dm, partial);
    k_diag_final<<<1, 256, 0, s>>>(partial, diag_blocks(), out);
    count_launches(2);
}

void launch_particle_update(ParticleDev *parts, int np, const double *partials, int ntiles,
                            const DevParams &p, cudaStream_t s)
{
    k_particle_update<<<np, 256, 0, s>>>(parts, np, partials, ntiles, p);
    count_launches(1);
}

}  // namespace pf
