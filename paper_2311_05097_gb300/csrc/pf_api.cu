// C-ABI of libpf (include/pf.h): handles, device memory, CUDA-graph replay of
// the step sequence, batched domains and the launch-configuration autotuner.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <cuda.h>  // CUtensorMap and its encoder's types (the encoder is fetched at run time)
#include <nvtx3/nvToolsExt.h>

#include "../../include/pf.h"
#include "pf_internal.h"

namespace pf {

// NVTX range over a library call (seen by Nsight tools; a no-op otherwise)
struct PfRange {
    explicit PfRange(const char *name) { nvtxRangePushA(name); }
    ~PfRange() { nvtxRangePop(); }
};

static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches += n; }

bool launch_step2d(int prec, int tx, int ty, bool moving, int mode, int grid, cudaStream_t s,
                   const StepArgs &a)
{
    switch (prec) {
    case PF_P64: return launch_step2d_p64(tx, ty, moving, mode, grid, s, a, nullptr);
    case PF_P32: return launch_step2d_p32(tx, ty, moving, mode, grid, s, a, nullptr);
    case PF_PMIX_FP16: return launch_step2d_mixh(tx, ty, moving, mode, grid, s, a, nullptr);
    default: return launch_step2d_mixb(tx, ty, moving, mode, grid, s, a, nullptr);
    }
}

int occupancy_step2d(int prec, int tx, int ty, bool moving, int mode)
{
    StepArgs a{};
    int occ = 0;
    bool ok;
    switch (prec) {
    case PF_P64: ok = launch_step2d_p64(tx, ty, moving, mode, 0, 0, a, &occ); break;
    case PF_P32: ok = launch_step2d_p32(tx, ty, moving, mode, 0, 0, a, &occ); break;
    case PF_PMIX_FP16: ok = launch_step2d_mixh(tx, ty, moving, mode, 0, 0, a, &occ); break;
    default: ok = launch_step2d_mixb(tx, ty, moving, mode, 0, 0, a, &occ); break;
    }
    return ok ? occ : 0;
}

void tile_shape3d(int prec, int *tx, int *ty)
{
    *tx = prec == PF_P64 ? 16 : 32;
    *ty = 8;
}

bool launch_step3d(int prec, int tx, int ty, bool moving, int mode, int grid, cudaStream_t s,
                   const StepArgs &a)
{
    switch (prec) {
    case PF_P64: return launch_step3d_p64(tx, ty, moving, mode, grid, s, a, nullptr);
    case PF_P32: return launch_step3d_p32(tx, ty, moving, mode, grid, s, a, nullptr);
    case PF_PMIX_FP16: return launch_step3d_mixh(tx, ty, moving, mode, grid, s, a, nullptr);
    default: return launch_step3d_mixb(tx, ty, moving, mode, grid, s, a, nullptr);
    }
}

int occupancy_step3d(int prec, int tx, int ty, bool moving, int mode)
{
    StepArgs a{};
    int occ = 0;
    bool ok;
    switch (prec) {
    case PF_P64: ok = launch_step3d_p64(tx, ty, moving, mode, 0, 0, a, &occ); break;
    case PF_P32: ok = launch_step3d_p32(tx, ty, moving, mode, 0, 0, a, &occ); break;
    case PF_PMIX_FP16: ok = launch_step3d_mixh(tx, ty, moving, mode, 0, 0, a, &occ); break;
    default: ok = launch_step3d_mixb(tx, ty, moving, mode, 0, 0, a, &occ); break;
    }
    return ok ? occ : 0;
}

}  // namespace pf

using namespace pf;

// ---------------------------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------------------------
static thread_local std::string t_err = "no error";

static int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                   \
    } while (0)

extern "C" const char *pf_last_error(void) { return t_err.c_str(); }

int pf::set_error(int code, const char *msg)
{
    t_err = msg;
    return code;
}
extern "C" int64_t pf_launch_count(void) { return (int64_t)g_launches.load(); }

// ---------------------------------------------------------------------------------------------
// parameters
// ---------------------------------------------------------------------------------------------
extern "C" int pf_params_default(pf_params *p)
{
    if (!p) return fail(PF_EINVAL, "pf_params_default: NULL");
    memset(p, 0, sizeof(*p));
    p->sigma = 0.01;
    p->D = 4.0;
    p->M = 0.02;
    p->eta = 0.0;
    p->rho1 = p->rho2 = 1.0;
    p->mu1 = p->mu2 = 0.1;
    p->d0 = 0.4;
    p->s0 = p->s1 = p->s2 = p->s3 = p->s4 = 1.0;
    p->theta_deg = 90.0;
    p->solid_eps = 1e-3;
    p->precision = PF_P64;
    return PF_OK;
}

static bool finite_all(const pf_params *p)
{
    const double v[] = {p->sigma, p->D, p->M, p->eta, p->rho1, p->rho2, p->mu1, p->mu2, p->d0,
                        p->s0, p->s1, p->s2, p->s3, p->s4, p->theta_deg, p->Fb[0], p->Fb[1],
                        p->Fb[2], p->g[0], p->g[1], p->g[2], p->solid_eps, p->rep_xi, p->rep_eps,
                        p->wall_circle[0], p->wall_circle[1], p->wall_circle[2]};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

static int validate(const pf_grid *g, const pf_params *p)
{
    if (!g || !p) return fail(PF_EINVAL, "grid or params is NULL");
    if (g->dim != 2 && g->dim != 3) return fail(PF_EINVAL, "dim must be 2 or 3 (got %d)", g->dim);
    const int nz = g->dim == 2 ? 1 : g->nz;
    if (g->nx < 4 || g->ny < 4 || (g->dim == 3 && nz < 4))
        return fail(PF_EINVAL, "grid sizes must be >= 4 (got %d x %d x %d)", g->nx, g->ny, nz);
    const long long pitch = (g->nx + (g->dim == 2 ? 2 * STRIP_GHOST : 0) + 31) / 32 * 32;
    const long long qtot = g->dim == 2 ? 18 : 26;
    if (qtot * (pitch * g->ny * nz + 64) >= (1LL << 31))
        return fail(PF_EINVAL, "grid too large: %lld populations x %lld cells must stay below 2^31 "
                    "(32-bit indexing of the state arrays)", qtot, pitch * g->ny * nz);
    for (int a = 0; a < g->dim; ++a) {
        const bool wall_ok = a == 1 && g->periodic[a] == 0;
        if (g->periodic[a] != 1 && !wall_ok)
            return fail(PF_EINVAL, "boundaries must be periodic, except walls at the ends of y "
                                   "(periodic[1] = 0)");
    }
    if (!finite_all(p)) return fail(PF_EINVAL, "non-finite parameter");
    if (p->sigma < 0) return fail(PF_EINVAL, "sigma must be >= 0");
    if (p->D <= 0) return fail(PF_EINVAL, "D must be > 0");
    if (p->M <= 0) return fail(PF_EINVAL, "M must be > 0");
    if (p->rho1 <= 0 || p->rho2 <= 0) return fail(PF_EINVAL, "densities must be > 0");
    if (p->mu1 <= 0 || p->mu2 <= 0) return fail(PF_EINVAL, "viscosities must be > 0");
    if (!(p->d0 > 0 && p->d0 < 0.5)) return fail(PF_EINVAL, "d0 must lie in (0, 1/2)");
    if (g->dim == 3 && p->d0 > 1.0 / 3.0 + 1e-12)
        return fail(PF_EINVAL, "3D needs d0 <= 1/3 (the D3Q7 rest weight 1 - 3 d0 must be >= 0)");
    const double s[] = {p->s0, p->s1, p->s2, p->s3, p->s4};
    for (double x : s)
        if (!(x > 0 && x < 2)) return fail(PF_EINVAL, "relaxation rates must lie in (0, 2)");
    if (!(p->solid_eps > 0 && p->solid_eps < 1)) return fail(PF_EINVAL, "solid_eps must lie in (0, 1)");
    if (p->rep_xi < 0 || p->rep_eps < 0) return fail(PF_EINVAL, "rep_xi and rep_eps must be >= 0");
    if (p->wall_circle[2] < 0 || (g->dim == 3 && p->wall_circle[2] > 0))
        return fail(PF_EINVAL, "wall_circle: radius >= 0, 2D only");
    if (p->precision < PF_P64 || p->precision > PF_PMIX_BF16)
        return fail(PF_EINVAL, "unknown precision %d", p->precision);
    const double cs2 = p->d0;
    if (p->phase_model != 0 && p->phase_model != 1) return fail(PF_EINVAL, "phase_model must be 0 or 1");
    const double eta = p->phase_model == 1 ? 1.0 : (p->eta > 0 ? p->eta : 2.0 * p->M / cs2);
    const double s1phi = 1.0 / (p->M / (eta * cs2) + 0.5);
    if (!(s1phi > 0 && s1phi < 2)) return fail(PF_EINVAL, "eta gives s_1phi outside (0, 2)");
    for (int k = 0; k < 2; ++k)
        if (p->store_log2_scale[k] < 0 || p->store_log2_scale[k] > 24)
            return fail(PF_EINVAL, "store_log2_scale must lie in [0, 24]");
    return PF_OK;
}

static int default_klog2(double mag)
{
    // map a typical population magnitude to ~2^-2 in the stored format
    int k = (int)std::lround(-std::log2(mag)) - 2;
    if (k < 4) k = 4;
    if (k > 24) k = 24;
    return k;
}

static DevParams derive(int dim, const pf_params *p)
{
    DevParams d{};
    d.sigma = p->sigma;
    d.D = p->D;
    d.M = p->M;
    d.rho1 = p->rho1;
    d.rho2 = p->rho2;
    d.mu1 = p->mu1;
    d.mu2 = p->mu2;
    d.d0 = p->d0;
    d.s0 = p->s0;
    d.s1 = p->s1;
    d.s2 = p->s2;
    d.s3 = p->s3;
    d.s4 = p->s4;
    d.solid_eps = p->solid_eps;
    d.rep_xi = p->rep_xi;
    d.rep_eps = p->rep_eps;
    for (int a = 0; a < 3; ++a) d.wall_circle[a] = p->wall_circle[a];
    d.dim = dim;
    for (int a = 0; a < 3; ++a) {
        d.Fb[a] = a < dim ? p->Fb[a] : 0.0;
        d.g[a] = a < dim ? p->g[a] : 0.0;
    }
    d.cs2 = p->d0;
    d.cs4 = d.cs2 * d.cs2;
    d.inv_cs2 = 1.0 / d.cs2;
    d.phase_model = p->phase_model;
    // Allen-Cahn: eta mu -> phi in the equilibrium, so eta = 1 sets s_1phi
    d.eta = p->phase_model == 1 ? 1.0 : (p->eta > 0 ? p->eta : 2.0 * p->M / d.cs2);
    d.s1phi = 1.0 / (p->M / (d.eta * d.cs2) + 0.5);  // M = (1/s_1phi - 1/2) eta cs^2
    d.unit = (std::fabs(d.s1phi - 1.0) <= 1e-12 && p->s1 == 1.0 && p->s2 == 1.0 && p->s3 == 1.0 && p->s4 == 1.0 &&
              p->phase_model == 0)
                 ? 1
                 : 0;
    d.cos_t = std::cos(p->theta_deg * 3.14159265358979323846 / 180.0);
    const double d0 = p->d0;
    d.w0f = dim == 2 ? 1.0 - 2.0 * d0 + d0 * d0 : 1.0 - 3.0 * d0 + 3.0 * d0 * d0;
    d.drho = 0.5 * (p->rho1 - p->rho2);
    d.rhom = 0.5 * (p->rho1 + p->rho2);
    d.dmu = 0.5 * (p->mu1 - p->mu2);
    d.mum = 0.5 * (p->mu1 + p->mu2);
    d.c_dw = 3.0 * p->sigma / p->D;
    d.c_lap = 3.0 * p->D * p->sigma / 8.0;
    d.c_pen = 9.0 * p->sigma / p->D;
    d.c_wet = 3.0 * p->sigma * d.cos_t / p->D;
    d.c_wlap = 3.0 * p->D * p->sigma * d.cos_t / 8.0;
    d.Mdrho = p->M * d.drho;
    if (dim == 2) {
        d.K = 1.0 - d0;
        d.Hc0 = (1.0 - d0) / p->s0 + 0.5 * (1.0 - 3.0 * d0);
        d.Hc1 = 2.0 - 4.0 * d0;
    } else {
        d.K = 1.0 - 2.0 * d0;
        d.Hc0 = (1.0 - d0) / p->s0 + (1.0 - 3.0 * d0);
        d.Hc1 = 3.0 - 7.0 * d0;
    }
    d.Pfac = d.cs2 / (1.0 - d.w0f);
    d.inv_1mcs2 = 1.0 / (1.0 - d.cs2);
    d.two_over_1md0 = 2.0 / (1.0 - d0);
    d.cut = 10.0 * p->D;
    const bool mix = p->precision >= PF_PMIX_FP16;
    // typical magnitudes: w_1 eta (3 sigma/D) for the order parameter, w_1 (3 sigma/D)/cs2 for flow
    const double w1 = dim == 2 ? 0.5 * (d0 - d0 * d0) : 0.5 * d0;
    const double musc = std::max(3.0 * p->sigma / p->D, 1e-6);
    // order parameter: the exact rest-population bookkeeping needs every stored
    // mover below 8 (stored = value * 2^k1); bound the movers by
    // w_1 (|u|/cs^2 + eta * 2 mu_max) with |u| <= 1 and mu_max = 3 sigma/D
    // (Allen-Cahn: w_1 |phi| (1 + |u|/cs^2) with |phi| <= 3/2)
    const double m1max = p->phase_model == 1 ? 1.5 * w1 * (1.0 + 1.0 / d.cs2)
                                             : w1 * (1.0 / d.cs2 + d.eta * 2.0 * musc);
    int k1 = p->store_log2_scale[0] ? p->store_log2_scale[0]
                                    : (int)std::floor(std::log2(8.0 / m1max));
    k1 = std::max(0, std::min(24, k1));
    // flow: scale typical magnitudes into FP16's normal range, far from overflow
    int k2 = p->store_log2_scale[1] ? p->store_log2_scale[1] : default_klog2(w1 * musc / d.cs2);
    k2 = std::max(0, std::min(12, k2));
    if (!mix) k1 = k2 = 0;
    d.klog2[0] = k1;
    d.klog2[1] = k2;
    d.scale[0] = std::ldexp(1.0, k1);
    d.scale[1] = std::ldexp(1.0, k2);
    d.inv_scale[0] = std::ldexp(1.0, -k1);
    d.inv_scale[1] = std::ldexp(1.0, -k2);
    return d;
}

static size_t store_bytes(int prec)
{
    return prec == PF_P64 ? 8 : (prec == PF_P32 ? 4 : 2);
}
static size_t aux_bytes(int prec) { return prec == PF_P64 ? 8 : 4; }

// ---------------------------------------------------------------------------------------------
// one domain's device memory
// ---------------------------------------------------------------------------------------------
struct DomainMem {
    DomainDev d{};
    void *base = nullptr;  // single allocation for populations, rest, aux, phi0
};

static long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

static int domain_alloc(DomainMem &m, int dim, const pf_grid *g, const DevParams &dp, int prec)
{
    DomainDev &d = m.d;
    d.nx = g->nx;
    d.ny = g->ny;
    d.nz = dim == 2 ? 1 : g->nz;
    d.wall_y = g->periodic[1] == 0 ? 1 : 0;
    // 2D rows carry STRIP_GHOST ghost columns after the row's end and, in the
    // padding of the previous row, before its start (the strip step's periodic
    // images in x)
    d.pitch = (int)round_up(d.nx + (dim == 2 ? 2 * STRIP_GHOST : 0), 32);
    d.plane = round_up((long long)d.pitch * d.ny * d.nz, 64);
    d.p = dp;
    d.kf = make_kparams<float>(dp);
    d.kd = make_kparams<double>(dp);
    const int Q = dim == 2 ? 18 : 26;
    const int naux = 2 * dim + 1;
    const size_t fb = (size_t)Q * d.plane * store_bytes(prec);
    const size_t rb = prec >= PF_PMIX_FP16 ? (size_t)d.plane * 8 : 0;
    const size_t ab = (size_t)naux * d.plane * aux_bytes(prec);
    const size_t pb = (size_t)d.plane * aux_bytes(prec);
    const size_t total = 2 * fb + 2 * rb + 2 * ab + pb + 256 * 8 + 256 * 8;
    CK(cudaMalloc(&m.base, total));
    CK(cudaMemset(m.base, 0, total));
    char *c = (char *)m.base;
    auto take = [&](size_t n) {
        c += 256;  // front pad: the ghost columns left of row 0 of the first plane
        void *r = c;
        c += round_up((long long)n, 256);
        return r;
    };
    d.f[0] = take(fb);
    d.f[1] = take(fb);
    d.rest[0] = rb ? take(rb) : nullptr;
    d.rest[1] = rb ? take(rb) : nullptr;
    d.aux[0] = take(ab);
    d.aux[1] = take(ab);
    d.phi0 = take(pb);
    d.macro = nullptr;
    return PF_OK;
}

// device staging area for init inputs (phi0, phi, u, P) and temporaries of
// one domain; shared by the domains of a batch (their inits are stream-ordered)
struct Staging {
    double *p = nullptr;
    size_t n = 0;
};

static int staging_reserve_n(Staging &st, size_t need)
{
    if (st.n >= need) return PF_OK;
    if (st.p) cudaFree(st.p);
    st.p = nullptr;
    st.n = 0;
    CK(cudaMalloc(&st.p, sizeof(double) * need));
    st.n = need;
    return PF_OK;
}

static int staging_reserve(Staging &st, const DomainMem &m, int dim)
{
    const long long N = (long long)m.d.nx * m.d.ny * m.d.nz;
    return staging_reserve_n(st, (size_t)(2 + dim + 1 + 4) * N);  // phi0, phi, u, P, phi0tot, mu, W, V
}

static void staging_release(Staging &st)
{
    if (st.p) cudaFree(st.p);
    st = Staging{};
}

static void domain_free(DomainMem &m)
{
    if (m.base) cudaFree(m.base);
    m = DomainMem{};
}

// the init kernels of one domain from device arrays (phi0, phi, and u, P or
// NULL, in the caller's layout); tmp: scratch of 4 N doubles (phi0tot, mu, W, V)
static int domain_init_kernels(DomainMem &m, int prec, const double *phi0, const double *phi, const double *u,
                               const double *P, double *tmp, const ParticleDev *d_parts,
                               const ParticleDev *hparts, int np, int *flags, cudaStream_t s)
{
    int wv = 0;
    for (int k = 0; k < np; ++k) wv |= hparts ? hparts[k].own : 0;
    launch_init(prec, m.d, flags, phi0, phi, u, P, tmp, d_parts, np, wv, s);
    CK(cudaGetLastError());
    return PF_OK;
}

// copy caller arrays into the staging area and run the init kernels
static int domain_init(DomainMem &m, Staging &st, int dim, int prec, const double *phi0, const double *phi,
                       const double *u, const double *P, int where, const ParticleDev *d_parts,
                       const ParticleDev *hparts, int np, int *flags, cudaStream_t s)
{
    if (!phi0 || !phi) return fail(PF_EINVAL, "phi0 and phi are required");
    if (where != PF_HOST && where != PF_DEVICE) return fail(PF_EINVAL, "where must be PF_HOST or PF_DEVICE");
    int rc = staging_reserve(st, m, dim);
    if (rc) return rc;
    const long long N = (long long)m.d.nx * m.d.ny * m.d.nz;
    double *sp0 = st.p, *sphi = sp0 + N, *su = sphi + N, *sP = su + dim * N, *tmp = sP + N;
    const cudaMemcpyKind kind = where == PF_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(sp0, phi0, sizeof(double) * N, kind, s));
    CK(cudaMemcpyAsync(sphi, phi, sizeof(double) * N, kind, s));
    if (u) CK(cudaMemcpyAsync(su, u, sizeof(double) * dim * N, kind, s));
    if (P) CK(cudaMemcpyAsync(sP, P, sizeof(double) * N, kind, s));
    return domain_init_kernels(m, prec, sp0, sphi, u ? su : nullptr, P ? sP : nullptr, tmp, d_parts, hparts, np,
                               flags, s);
}

// tile table of a set of domains (2D tiles of tx x ty; 3D column tiles of tx x ty
// cells and zc planes)
static void build_tiles(const std::vector<DomainMem *> &doms, int tx, int ty, std::vector<int> &tdom,
                        std::vector<int2> &txy, int zc = ZCHUNK3D)
{
    tdom.clear();
    txy.clear();
    for (size_t k = 0; k < doms.size(); ++k) {
        DomainDev &d = doms[k]->d;
        d.tiles_x = (d.nx + tx - 1) / tx;
        d.tiles_y = (d.ny + ty - 1) / ty;
        d.zc = zc;
        d.tiles_z = d.p.dim == 3 ? (d.nz + zc - 1) / zc : 1;
        d.tile_base = (int)tdom.size();
        // 3D tiles encode (y tile, z chunk) as y + tiles_y * z
        for (int kz = 0; kz < d.tiles_z; ++kz)
            for (int j = 0; j < d.tiles_y; ++j)
                for (int i = 0; i < d.tiles_x; ++i) {
                    tdom.push_back((int)k);
                    txy.push_back(make_int2(i, j + d.tiles_y * kz));
                }
    }
}

// ---------------------------------------------------------------------------------------------
// shared engine of single and batched handles
// ---------------------------------------------------------------------------------------------
struct Engine {
    int dim = 2, prec = PF_P64;
    std::vector<DomainMem> mem;
    DomainDev *d_doms = nullptr;
    int *d_tdom = nullptr;
    int2 *d_txy = nullptr;
    int ntiles = 0;
    int tx = 32, ty = 8, cps = 0, grid = 0;  // tile shape, CTAs per SM, grid size
    int variant = 0;                         // 2D: 0 one cell per thread, 1 two, 2 two + staging,
                                             // 3 particle domain split: near tiles 0, far tiles 1
    unsigned char *d_sel = nullptr;          // variant 3: per tile 1 near a particle, 0 far
    int sel_cap = 0;
    int grid_far = 0;                        // variant 3: grid of the far-tile launch
    // variant 4 (strips marched in y): work items, tensor maps, ghost columns
    int4 *d_items = nullptr;
    int nitems = 0;
    void *d_maps = nullptr;                  // STRIP_MAPS tensor maps per domain
    bool maps_ok = false;
    bool ghosts_ok = false;                  // the buffer the next step reads has valid ghost columns
    cudaStream_t side = nullptr;             // variant 3: the near tiles run on this stream beside
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;  // the far ones (fork / join)
    bool forced = false;                     // launch configuration set by the caller
    bool tuned = false;
    int nsm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int par = 0;
    int64_t t = 0;
    std::vector<bool> inited;
    Staging staging;
    // macroscopic pass: one output buffer (largest domain) and per-domain tile
    // tables of the macro kernel, built on first use
    double *d_macro = nullptr;
    DomainDev *d_mdoms = nullptr;
    // pf_batch_init_all / pf_batch_get_macros_all: host copies run on a copy
    // stream beside the engine's stream (the input copies of later domains
    // overlap the init kernels of earlier ones; the readback of a domain
    // overlaps the macroscopic passes of the next ones).  The init kernels of
    // consecutive domains go round-robin to the engine's stream and KS - 1
    // more (small domains' kernels are launch-latency bound: they overlap);
    // the macroscopic passes rotate over up to PIPE macro buffers
    static constexpr int PIPE = 4, KS = 8;
    cudaStream_t cstream = nullptr;
    cudaStream_t kstream[KS - 1] = {};
    cudaEvent_t ev_in = nullptr, ev_start = nullptr, ev_k[KS] = {}, ev_c[PIPE] = {};
    int nslots = 0;                          // macro buffers in rotation (d_macro and d_macro_x)
    double *d_macro_x[PIPE - 1] = {};
    DomainDev *d_mdoms_x[PIPE - 1] = {};
    int *d_mtdom = nullptr;
    int2 *d_mtxy = nullptr;
    std::vector<int> mbase, mcount;
    int *d_flags = nullptr;
    int *d_queue = nullptr;  // work-queue counter of the strip step
    double *d_diag = nullptr;  // partials + out
    // particles (single-domain handles)
    ParticleDev hp[PF_MAX_PARTICLES];
    int np = 0;
    int wv = 0;                 // some particle has its own contact angle
    ParticleDev *d_parts = nullptr;
    double *d_frep = nullptr;   // repulsion force per particle (3 doubles each)
    double *d_partials = nullptr;
    size_t partials_cap = 0;
    // graph of CHUNK steps starting at parity 0, and graphs of one step at
    // parity 0 and 1 (the steps of a call that do not fill a chunk: one graph
    // launch per step instead of one launch per kernel), with the kernel
    // launches each replays
    static constexpr int CHUNK = 16;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphExec_t gexec1[2] = {nullptr, nullptr};
    long long glaunch = 0, glaunch1[2] = {0, 0};
    int sticky = PF_OK;
    // polls of one bounded device wait; 0: the kernels' default.  Read from the
    // environment variable PF_WAIT_POLLS at create (fault injection: a tiny
    // value makes the staged kernel's first wait give up -> PF_ETIMEOUT)
    int wait_polls = 0;
    // doubles of the input ring of pf_batch_init_all (at least one domain's
    // inputs); 0: 2^25.  Read from PF_INIT_RING at create (a small value makes
    // the ring wrap after every domain: the ordering test)
    long long init_ring = 0;
};

static int engine_setup(Engine &E, int nd, const pf_grid *g, const pf_params *p)
{
    E.dim = g[0].dim;
    E.prec = p[0].precision;
    if (const char *w = std::getenv("PF_WAIT_POLLS")) E.wait_polls = std::max(0, std::atoi(w));
    if (const char *w = std::getenv("PF_INIT_RING")) E.init_ring = std::max(0LL, std::atoll(w));
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&E.nsm, cudaDevAttrMultiProcessorCount, dev));
    if (p[0].stream) {
        E.stream = (cudaStream_t)p[0].stream;
        E.own_stream = false;
    } else {
        CK(cudaStreamCreateWithFlags(&E.stream, cudaStreamNonBlocking));
        E.own_stream = true;
    }
    E.mem.resize(nd);
    E.inited.assign(nd, false);
    for (int i = 0; i < nd; ++i) {
        const DevParams dp = derive(E.dim, &p[i]);
        int rc = domain_alloc(E.mem[i], E.dim, &g[i], dp, E.prec);
        if (rc) return rc;
    }
    CK(cudaMalloc(&E.d_doms, sizeof(DomainDev) * nd));
    CK(cudaMalloc(&E.d_flags, sizeof(int) * 4));
    CK(cudaMemset(E.d_flags, 0, sizeof(int) * 4));
    CK(cudaMalloc(&E.d_queue, sizeof(int) * 4));
    CK(cudaMalloc(&E.d_diag, sizeof(double) * (3 * diag_blocks() + 8)));
    CK(cudaMalloc(&E.d_parts, sizeof(ParticleDev) * PF_MAX_PARTICLES));
    CK(cudaMalloc(&E.d_frep, sizeof(double) * 3 * PF_MAX_PARTICLES));
    return PF_OK;
}

static void engine_free(Engine &E)
{
    if (E.gexec) cudaGraphExecDestroy(E.gexec);
    for (int p = 0; p < 2; ++p)
        if (E.gexec1[p]) cudaGraphExecDestroy(E.gexec1[p]);
    for (auto &m : E.mem) domain_free(m);
    staging_release(E.staging);
    if (E.d_macro) cudaFree(E.d_macro);
    if (E.d_mdoms) cudaFree(E.d_mdoms);
    for (int k = 0; k < Engine::PIPE - 1; ++k) {
        if (E.d_macro_x[k]) cudaFree(E.d_macro_x[k]);
        if (E.d_mdoms_x[k]) cudaFree(E.d_mdoms_x[k]);
    }
    for (int k = 0; k < Engine::KS - 1; ++k)
        if (E.kstream[k]) cudaStreamDestroy(E.kstream[k]);
    for (int k = 0; k < Engine::KS; ++k)
        if (E.ev_k[k]) cudaEventDestroy(E.ev_k[k]);
    for (int k = 0; k < Engine::PIPE; ++k)
        if (E.ev_c[k]) cudaEventDestroy(E.ev_c[k]);
    if (E.ev_in) cudaEventDestroy(E.ev_in);
    if (E.ev_start) cudaEventDestroy(E.ev_start);
    if (E.cstream) cudaStreamDestroy(E.cstream);
    if (E.d_mtdom) cudaFree(E.d_mtdom);
    if (E.d_mtxy) cudaFree(E.d_mtxy);
    if (E.d_doms) cudaFree(E.d_doms);
    if (E.d_tdom) cudaFree(E.d_tdom);
    if (E.d_txy) cudaFree(E.d_txy);
    if (E.d_flags) cudaFree(E.d_flags);
    if (E.d_queue) cudaFree(E.d_queue);
    if (E.d_diag) cudaFree(E.d_diag);
    if (E.d_parts) cudaFree(E.d_parts);
    if (E.d_frep) cudaFree(E.d_frep);
    if (E.d_partials) cudaFree(E.d_partials);
    if (E.d_sel) cudaFree(E.d_sel);
    if (E.d_items) cudaFree(E.d_items);
    if (E.d_maps) cudaFree(E.d_maps);
    if (E.ev_fork) cudaEventDestroy(E.ev_fork);
    if (E.ev_join) cudaEventDestroy(E.ev_join);
    if (E.side) cudaStreamDestroy(E.side);
    if (E.own_stream && E.stream) cudaStreamDestroy(E.stream);
    E = Engine{};
}

static void drop_graph(Engine &E)
{
    if (E.gexec) cudaGraphExecDestroy(E.gexec);
    E.gexec = nullptr;
    for (int p = 0; p < 2; ++p) {
        if (E.gexec1[p]) cudaGraphExecDestroy(E.gexec1[p]);
        E.gexec1[p] = nullptr;
    }
}

// upload the domain table and the tile table for shape (tx, ty)
static int engine_tiles(Engine &E, int tx, int ty)
{
    std::vector<DomainMem *> ds;
    for (auto &m : E.mem) ds.push_back(&m);
    std::vector<int> tdom;
    std::vector<int2> txy;
    build_tiles(ds, tx, ty, tdom, txy);
    if (E.d_tdom) cudaFree(E.d_tdom);
    if (E.d_txy) cudaFree(E.d_txy);
    E.d_tdom = nullptr;
    E.d_txy = nullptr;
    E.ntiles = (int)tdom.size();
    CK(cudaMalloc(&E.d_tdom, sizeof(int) * E.ntiles));
    CK(cudaMalloc(&E.d_txy, sizeof(int2) * E.ntiles));
    CK(cudaMemcpy(E.d_tdom, tdom.data(), sizeof(int) * E.ntiles, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(E.d_txy, txy.data(), sizeof(int2) * E.ntiles, cudaMemcpyHostToDevice));
    std::vector<DomainDev> hd;
    for (auto &m : E.mem) hd.push_back(m.d);
    CK(cudaMemcpy(E.d_doms, hd.data(), sizeof(DomainDev) * hd.size(), cudaMemcpyHostToDevice));
    E.tx = tx;
    E.ty = ty;
    const size_t need = (size_t)E.ntiles * std::max(E.np, 1) * 6;
    if (need > E.partials_cap) {
        if (E.d_partials) cudaFree(E.d_partials);
        E.d_partials = nullptr;
        CK(cudaMalloc(&E.d_partials, sizeof(double) * need));
        E.partials_cap = need;
    }
    drop_graph(E);
    return PF_OK;
}

// domains only the single-cell kernel handles: walls at the ends of y
static bool any_walls(const Engine &E)
{
    for (auto &m : E.mem)
        if (m.d.wall_y) return true;
    return false;
}

// domains with the Allen-Cahn order parameter
static bool any_cac(const Engine &E)
{
    for (auto &m : E.mem)
        if (m.d.p.phase_model == 1) return true;
    return false;
}

// the instantiation flags of a 2D launch
static bool all_unit(const Engine &E)
{
    for (auto &m : E.mem)
        if (!m.d.p.unit) return false;
    return true;
}

static int mode_flags(const Engine &E)
{
    const bool w = any_walls(E), c = any_cac(E);
    return (w || c ? MODE_EXT : 0) | (c ? MODE_CAC : 0) | (w ? MODE_WALL : 0) | (all_unit(E) ? MODE_UNIT : 0);
}

static bool launch_any(const Engine &E, int tx, int ty, int mode, int grid, const StepArgs &a)
{
    if (E.dim == 3)
        return launch_step3d(E.prec, tx, ty, E.np > 0,
                             mode | (any_walls(E) ? MODE_EXT : 0) | (all_unit(E) ? MODE_UNIT : 0), grid, E.stream, a);
    return launch_step2d(E.prec, tx, ty, E.np > 0, mode | mode_flags(E), grid, E.stream, a);
}

static int step_mode(const Engine &E)
{
    // (variant 3: the single-cell launch of the near tiles; the far tiles are
    // launched beside it in issue_step)
    if (E.variant == 4) return MODE_STEP_STRIP;
    return E.variant == 2 ? MODE_STEP_STAGE : (E.variant == 1 ? MODE_STEP_PAIR : MODE_STEP);
}

// a particle domain whose far tiles the two-cells-per-thread step can run:
// one 2D domain, FP32 or 16-bit storage, no walls, the Cahn-Hilliard lattice,
// no particle with its own contact angle
static bool split_ok(const Engine &E)
{
    // (particles with their own contact angles act only within their reach: on
    // the near tiles, which run the single-cell step)
    // (walls: the far tiles run the single-cell step's wall instantiation)
    return E.dim == 2 && E.np > 0 && E.prec != PF_P64 && E.mem.size() == 1 && !any_cac(E);
}

// the staged 2D step copies 16-byte chunks: every domain's nx must keep its
// rows' chunks and periodic splits aligned
static bool stage_ok(const Engine &E)
{
    if (E.dim != 2 || E.prec == PF_P64 || E.np > 0 || any_walls(E) || any_cac(E)) return false;
    const int q = E.prec == PF_P32 ? 4 : 8;
    for (auto &m : E.mem)
        if (m.d.nx % q) return false;
    return true;
}

// the strip step (variant 4): 2D, FP32 or 16-bit storage, no free particles,
// no walls at the ends of y, every nx even and >= the ghost width
static bool strip_ok(const Engine &E)
{
    if (E.dim != 2 || E.prec == PF_P64 || E.np > 0) return false;
    for (auto &m : E.mem)
        if (m.d.nx % 2 || m.d.nx < STRIP_GHOST || m.d.pitch < m.d.nx + 2 * STRIP_GHOST) return false;
    return true;
}

static int occupancy_any(const Engine &E, int tx, int ty, int mode)
{
    if (E.dim == 3)
        return occupancy_step3d(E.prec, tx, ty, E.np > 0,
                                mode | (any_walls(E) ? MODE_EXT : 0) | (all_unit(E) ? MODE_UNIT : 0));
    return occupancy_step2d(E.prec, tx, ty, E.np > 0, mode | mode_flags(E));
}

static StepArgs step_args(const Engine &E, int par)
{
    StepArgs a{};
    a.doms = E.d_doms;
    a.tile_dom = E.d_tdom;
    a.tile_xy = E.d_txy;
    a.ntiles = E.ntiles;
    a.par = par;
    a.parts = E.d_parts;
    a.np = E.np;
    a.partials = E.d_partials;
    a.flags = E.d_flags;
    a.wv = E.wv;
    a.wait_polls = E.wait_polls;
    a.items = E.d_items;
    a.nitems = E.nitems;
    a.strip_maps = E.d_maps;
    return a;
}

// issue one time step on E.stream (step kernel, then the particle update)
static int issue_step(Engine &E, int par)
{
    const StepArgs a = step_args(E, par);
    if (E.variant == 3) {
        // tiles out of every particle's reach run the two-cells-per-thread
        // step (with the fixed solids' mu_phi0 grad phi0), the others the
        // single-cell step with the particle terms
        launch_split_tiles(a, E.tx, E.ty, E.d_sel, E.stream);
        StepArgs af = a, an = a;
        af.tile_sel = an.tile_sel = E.d_sel;
        af.sel = 0;
        an.sel = 1;
        // the two launches write disjoint tiles and read only the previous
        // parity: the (short, latency-bound) near launch runs on a side
        // stream beside the far one, joined before the particle update
        CK(cudaEventRecord(E.ev_fork, E.stream));
        CK(cudaStreamWaitEvent(E.side, E.ev_fork, 0));
        cudaStream_t main = E.stream;
        E.stream = E.side;
        const bool ok_near = launch_any(E, E.tx, E.ty, MODE_STEP, E.grid, an);
        E.stream = main;
        CK(cudaEventRecord(E.ev_join, E.side));
        bool ok_far;
        if (any_walls(E)) {
            // walls: the single-cell step's wall instantiation without the particle
            // terms, with the fixed solids' mu_phi0 grad phi0
            af.mu0 = 1;
            ok_far = launch_step2d(E.prec, E.tx, E.ty, false, MODE_STEP | mode_flags(E), E.grid_far, E.stream, af);
        } else {
            ok_far = launch_any(E, E.tx, E.ty, MODE_STEP_PAIR | MODE_MU0, E.grid_far, af);
        }
        CK(cudaStreamWaitEvent(E.stream, E.ev_join, 0));
        if (!ok_near || !ok_far) return fail(PF_EINVAL, "split step of tile shape %dx%d not built", E.tx, E.ty);
    } else if (E.variant == 4) {
        if (!E.ghosts_ok && !launch_any(E, STRIP_SW, 0, MODE_FILL_GHOSTS, (int)E.mem.size(), a))
            return fail(PF_EINVAL, "ghost pass not built");
        // the items after each CTA's first come from a work queue
        StepArgs aq = a;
        aq.queue = E.d_queue;
        CK(cudaMemsetAsync(E.d_queue, 0, sizeof(int), E.stream));
        if (!launch_any(E, E.tx, E.ty, MODE_STEP_STRIP, E.grid, aq))
            return fail(PF_EINVAL, "strip step of width %d not built", E.tx);
    } else if (!launch_any(E, E.tx, E.ty, step_mode(E), E.grid, a)) {
        return fail(PF_EINVAL, "tile shape %dx%d (variant %d) not built", E.tx, E.ty, E.variant);
    }
    // the strip step writes the ghost columns of what it stores; the others do not
    E.ghosts_ok = E.variant == 4;
    if (E.np > 0)
        launch_particle_update(E.d_parts, E.np, E.d_partials, E.ntiles, E.mem[0].d.p, E.d_frep, E.mem[0].d.nx,
                               E.mem[0].d.ny, E.mem[0].d.nz, E.mem[0].d.wall_y,
                               E.variant == 3 ? E.d_sel : nullptr, E.stream);
    CK(cudaGetLastError());
    return PF_OK;
}

static int grid_of(Engine &E, int cps)
{
    int occ = occupancy_any(E, E.tx, E.ty, step_mode(E));
    if (occ < 1) occ = 1;
    int c = cps > 0 ? std::min(cps, occ) : occ;
    long long g = (long long)c * E.nsm;
    const long long units = E.variant == 4 ? E.nitems : E.ntiles;
    if (g > units) g = units;
    return (int)std::max(1LL, g);
}

// variant 3: tile lists and the far-tile grid (before any graph capture)
static int split_setup(Engine &E)
{
    if (E.sel_cap < E.ntiles) {
        if (E.d_sel) cudaFree(E.d_sel);
        E.d_sel = nullptr;
        CK(cudaMalloc(&E.d_sel, (size_t)E.ntiles));
        E.sel_cap = E.ntiles;
    }
    if (!E.side) CK(cudaStreamCreateWithFlags(&E.side, cudaStreamNonBlocking));
    if (!E.ev_fork) CK(cudaEventCreateWithFlags(&E.ev_fork, cudaEventDisableTiming));
    if (!E.ev_join) CK(cudaEventCreateWithFlags(&E.ev_join, cudaEventDisableTiming));
    const int occ = std::max(1, any_walls(E) ? occupancy_step2d(E.prec, E.tx, E.ty, false, MODE_STEP | mode_flags(E))
                                             : occupancy_any(E, E.tx, E.ty, MODE_STEP_PAIR | MODE_MU0));
    E.grid_far = (int)std::max(1LL, std::min((long long)occ * E.nsm, (long long)E.ntiles));
    return PF_OK;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, fetched through the runtime (no libcuda link)
static EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    });
    return fn;
}

// One tiled tensor map over a row-major array whose rows carry STRIP_GHOST
// ghost columns on each side: x' = x + STRIP_GHOST in [0, pitch), y in
// [0, ny), then `planes` planes; box = (bx, 1 row, planes).
static int encode_map(CUtensorMap *m, CUtensorMapDataType type, int es, const void *cell0, int pitch, int ny,
                      int planes, long long plane, int bx)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return fail(PF_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const char *base = static_cast<const char *>(cell0) - (size_t)STRIP_GHOST * es;
    const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)ny, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * es, (cuuint64_t)plane * es};
    const cuuint32_t box[3] = {(cuuint32_t)bx, 1u, (cuuint32_t)planes};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const cuuint32_t rank = planes > 1 ? 3u : 2u;
    CUresult r = fn(m, type, rank, const_cast<char *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(PF_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PF_OK;
}

// variant 4: the tensor maps of every domain (both read parities) and the
// work items of segments of `seg` rows (strips of STRIP_SW columns), ordered
// largest first, then by domain, segment and strip (neighbouring strips of a
// segment run side by side and share their halo columns in L2)
static int strip_setup(Engine &E, int seg)
{
    if (!E.maps_ok) {
        const int nd = (int)E.mem.size();
        std::vector<CUtensorMap> maps((size_t)nd * STRIP_MAPS);
        memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
        const bool mix = E.prec >= PF_PMIX_FP16;
        const int es = (int)store_bytes(E.prec);
        const CUtensorMapDataType ft = E.prec == PF_P32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                       : E.prec == PF_PMIX_FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
        const int hs = 16 / es, w1 = STRIP_SW + 2 * hs;
        for (int i = 0; i < nd; ++i) {
            const DomainDev &d = E.mem[i].d;
            CUtensorMap *m = &maps[(size_t)i * STRIP_MAPS];
            int rc = PF_OK;
            for (int par = 0; par < 2 && rc == PF_OK; ++par) {
                CUtensorMap *q = m + par * STRIP_MAPS_PER_PAR;
                const char *f = static_cast<const char *>(d.f[par]);
                const char *aux = static_cast<const char *>(d.aux[par]);
                const int i1 = mix ? 1 : 0;  // (the PMIX rest population is held apart)
                rc = encode_map(q + SM_F, ft, es, f + (size_t)i1 * d.plane * es, d.pitch, d.ny, 18 - i1, d.plane, w1);
                if (!rc && mix)
                    rc = encode_map(q + SM_REST, CU_TENSOR_MAP_DATA_TYPE_INT64, 8, d.rest[par], d.pitch, d.ny, 1,
                                    d.plane, STRIP_SW + 4);
                if (!rc)
                    rc = encode_map(q + SM_US, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, aux, d.pitch, d.ny, 5, d.plane,
                                    STRIP_SW + 8);

            }
            if (!rc)
                rc = encode_map(m + SM_PHI0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d.phi0, d.pitch, d.ny, 1, d.plane,
                                STRIP_SW + 8);
            if (rc) return rc;
        }
        if (E.d_maps) cudaFree(E.d_maps);
        E.d_maps = nullptr;
        CK(cudaMalloc(&E.d_maps, sizeof(CUtensorMap) * maps.size()));
        CK(cudaMemcpy(E.d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice));
        E.maps_ok = true;
    }
    struct It {
        int4 v;
        long long cells;
    };
    std::vector<It> its;
    for (int i = 0; i < (int)E.mem.size(); ++i) {
        const DomainDev &d = E.mem[i].d;
        for (int ya = 0; ya < d.ny; ya += seg)
            for (int x0 = 0; x0 < d.nx; x0 += STRIP_SW) {
                const int yb = std::min(ya + seg, d.ny);
                its.push_back({make_int4(i, x0, ya, yb), (long long)(yb - ya) * std::min(STRIP_SW, d.nx - x0)});
            }
    }
    std::stable_sort(its.begin(), its.end(), [](const It &a, const It &b) { return a.cells > b.cells; });
    std::vector<int4> items;
    for (auto &t : its) items.push_back(t.v);
    if (E.d_items) cudaFree(E.d_items);
    E.d_items = nullptr;
    E.nitems = (int)items.size();
    CK(cudaMalloc(&E.d_items, sizeof(int4) * items.size()));
    CK(cudaMemcpy(E.d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    return PF_OK;
}

// fill the ghost columns of the buffers the next step reads, unless valid
// (before a graph capture or replay: the captured steps then never need it)
static int ensure_ghosts(Engine &E)
{
    if (E.variant != 4 || E.ghosts_ok) return PF_OK;
    const StepArgs a = step_args(E, E.par);
    if (!launch_any(E, STRIP_SW, 0, MODE_FILL_GHOSTS, (int)E.mem.size(), a))
        return fail(PF_EINVAL, "ghost pass not built");
    CK(cudaGetLastError());
    E.ghosts_ok = true;
    return PF_OK;
}

// Autotuner: time a few steps of each compiled tile shape and CTAs-per-SM
// choice on the live state (the state advances; steps are counted), keep the
// fastest; cached per (dim, precision, moving, cell-count bucket, domain count).
static std::mutex g_tune_mu;
// key: (dim, precision, free particles, cell-count bucket, domain count,
// features: bit 0 walls, bit 1 Allen-Cahn, bit 2 own contact angles, bit 3
// the strip step can run it, bit 4 unit relaxation rates)
static std::map<std::tuple<int, int, int, long long, int, int>, std::tuple<int, int, int, int>> g_tune_cache;

// the features of a launch that decide which kernels can run it
static int tune_features(const Engine &E)
{
    return (any_walls(E) ? 1 : 0) | (any_cac(E) ? 2 : 0) | (E.wv ? 4 : 0) | (strip_ok(E) ? 8 : 0) |
           (all_unit(E) ? 16 : 0);
}

// PF_TUNE_LOG set in the environment: the autotuner prints each candidate's
// time per step to stderr
static bool tune_log()
{
    static const bool on = getenv("PF_TUNE_LOG") != nullptr;
    return on;
}

// Returns PF_OK with E.tuned set, or PF_OK with E.tuned unset when nothing is
// cached for this launch and `tune` is false (the caller then takes defaults).
static int engine_configure(Engine &E, bool tune)
{
    long long cells = 0;
    for (auto &m : E.mem) cells += (long long)m.d.nx * m.d.ny * m.d.nz;
    long long bucket = 1;
    while (bucket < cells) bucket <<= 1;
    const auto key = std::make_tuple(E.dim, E.prec, E.np > 0 ? 1 : 0, bucket, (int)E.mem.size(), tune_features(E));
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            int tx, ty, var, cps;
            std::tie(tx, ty, var, cps) = it->second;
            if ((var == 3 && !split_ok(E)) || (var == 4 && !strip_ok(E)) ||
                (var != 0 && (E.dim == 3 || (var != 4 && var != 3 && any_walls(E))))) {  // (the key separates these)
                var = 0;
                tx = 32;
                ty = 8;
            }
            int rc = engine_tiles(E, tx, ty);
            if (rc) return rc;
            E.variant = var;
            E.cps = cps;
            if (var == 3) {
                rc = split_setup(E);
                if (rc) return rc;
            }
            if (var == 4) {
                rc = strip_setup(E, ty);
                if (rc) return rc;
            }
            E.grid = grid_of(E, cps);
            E.tuned = true;
            return PF_OK;
        }
    }
    if (!tune) return PF_OK;
    // (tile x, tile y, variant): one cell per thread, then two (FP32
    // arithmetic policies without free particles)
    // (kernel 2, the bulk-copy staged variant, is selectable with
    // pf_set_config but not a candidate: it measured slower than kernel 1)
    // (kernel 4: tile = strip width x segment rows)
    // (walls: kernels 0 and 4 only)
    int shapes[10][3] = {{32, 8, 0}, {64, 4, 0}, {32, 16, 0}, {32, 16, 1}, {64, 8, 1}, {32, 32, 1}, {64, 96, 4},
                         {64, 128, 4}, {64, 192, 4}, {64, 256, 4}};
    int nshapes = (E.prec != PF_P64 && E.np == 0 && !any_walls(E)) ? 6 : 3;
    if (strip_ok(E)) {
        // on small launches (fewer than 8 work items of 96 rows per SM) also
        // the short segments that give every CTA slot work
        long long items96 = 0;
        for (auto &m : E.mem)
            items96 += (long long)((m.d.nx + STRIP_SW - 1) / STRIP_SW) * ((m.d.ny + 95) / 96);
        if (items96 < 8LL * E.nsm) {
            shapes[6][1] = 8;
            shapes[7][1] = 16;
            shapes[8][1] = 32;
            shapes[9][1] = 64;
        }
        if (nshapes == 3)
            for (int k = 0; k < 4; ++k)
                for (int j = 0; j < 3; ++j) shapes[3 + k][j] = shapes[6 + k][j];
        nshapes += 4;
    }
    if (split_ok(E)) {
        // particle domain: also the split of near (single-cell) and far
        // (two-cells-per-thread) tiles
        shapes[3][0] = 32;
        shapes[3][1] = 16;
        shapes[3][2] = 3;
        nshapes = 4;
    }
    if (E.dim == 3) {
        tile_shape3d(E.prec, &shapes[0][0], &shapes[0][1]);
        shapes[0][2] = 0;
        nshapes = 1;
    }
    float best = 1e30f;
    int bx = 32, by = 8, bv = 0, bc = 0;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int reps = cells > (1 << 22) ? 2 : 4;
    for (int si = 0; si < nshapes; ++si) {
        const int *sh = shapes[si];
        int rc = engine_tiles(E, sh[0], sh[1]);
        if (rc) return rc;
        E.variant = sh[2];
        if (E.variant == 3) {
            rc = split_setup(E);
            if (rc) return rc;
        }
        if (E.variant == 4) {
            rc = strip_setup(E, sh[1]);
            if (rc) return rc;
        }
        const int occ = std::max(1, occupancy_any(E, sh[0], sh[1], step_mode(E)));
        for (int cps = 1; cps <= occ; cps = cps < occ ? std::min(cps * 2, occ) : occ + 1) {
            E.cps = cps;
            E.grid = grid_of(E, cps);
            // warm-up (keeps the parity even so the state stays consistent)
            for (int r = 0; r < 2; ++r) {
                rc = issue_step(E, E.par);
                if (rc) return rc;
                E.par ^= 1;
                E.t++;
            }
            CK(cudaEventRecord(e0, E.stream));
            for (int r = 0; r < 2 * reps; ++r) {
                rc = issue_step(E, E.par);
                if (rc) return rc;
                E.par ^= 1;
                E.t++;
            }
            CK(cudaEventRecord(e1, E.stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (tune_log())
                fprintf(stderr, "pf tune: tile %dx%d kernel %d ctas/SM %d grid %d: %.4f ms per step\n", sh[0], sh[1],
                        sh[2], cps, E.grid, ms / (2 * reps));
            if (ms < best) {
                best = ms;
                bx = sh[0];
                by = sh[1];
                bv = sh[2];
                bc = cps;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int rc = engine_tiles(E, bx, by);
    if (rc) return rc;
    E.variant = bv;
    E.cps = bc;
    if (bv == 3) {
        rc = split_setup(E);
        if (rc) return rc;
    }
    if (bv == 4) {
        rc = strip_setup(E, by);
        if (rc) return rc;
    }
    E.grid = grid_of(E, bc);
    E.tuned = true;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = std::make_tuple(bx, by, bv, bc);
    return PF_OK;
}

static const int64_t TUNE_MIN_STEPS = 256;

static int engine_step(Engine &E, int64_t n, bool autotune)
{
    if (E.sticky) return E.sticky;
    if (n < 0) return fail(PF_EINVAL, "n must be >= 0");
    for (size_t i = 0; i < E.inited.size(); ++i)
        if (!E.inited[i]) return fail(PF_ESTATE, "domain %zu stepped before pf_init_fields", i);
    if (n == 0) return PF_OK;
    int64_t left = n;
    if (!E.tuned) {
        int rc = PF_OK;
        if (autotune) {
            // a configuration cached for this kind of launch is taken at once;
            // otherwise a call of >= TUNE_MIN_STEPS steps runs the tuner: its
            // timed candidate steps are real steps of the simulation and count
            // towards n (every configuration computes the same update)
            const int64_t t0 = E.t;
            rc = engine_configure(E, n >= TUNE_MIN_STEPS);
            left -= E.t - t0;
        }
        if (rc == PF_OK && !E.tuned) {
            int tx = 32, ty = 8;
            if (E.dim == 3) tile_shape3d(E.prec, &tx, &ty);
            E.variant = 0;
            rc = engine_tiles(E, tx, ty);
            E.cps = 0;
            E.grid = autotune ? grid_of(E, 0) : E.ntiles;  // one CTA per tile
            E.tuned = !autotune;
        }
        if (rc) return (E.sticky = rc);
    }
    // one step from the graph of its parity (captured at first use)
    auto one_step = [&]() -> int {
        const int p = E.par;
        int grc = ensure_ghosts(E);
        if (grc) return grc;
        if (!E.gexec1[p]) {
            const long long before = g_launches.load();
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(E.stream, cudaStreamCaptureModeThreadLocal));
            const int rc = issue_step(E, p);
            cudaError_t ce = cudaStreamEndCapture(E.stream, &graph);
            if (rc) return rc;
            CK(ce);
            CK(cudaGraphInstantiate(&E.gexec1[p], graph, 0));
            cudaGraphDestroy(graph);
            E.glaunch1[p] = g_launches.load() - before;
            g_launches = before;  // captured launches run (and are counted) at replay
        }
        CK(cudaGraphLaunch(E.gexec1[p], E.stream));
        count_launches(E.glaunch1[p]);
        E.par ^= 1;
        E.t++;
        return PF_OK;
    };
    while (left > 0 && E.par != 0) {
        int rc = one_step();
        if (rc) return (E.sticky = rc);
        left--;
    }
    if (left >= Engine::CHUNK) {
        int grc = ensure_ghosts(E);
        if (grc) return (E.sticky = grc);
        if (!E.gexec) {
            const long long before = g_launches.load();
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(E.stream, cudaStreamCaptureModeThreadLocal));
            int rc = PF_OK;
            for (int k = 0; k < Engine::CHUNK && rc == PF_OK; ++k) rc = issue_step(E, k & 1);
            cudaError_t ce = cudaStreamEndCapture(E.stream, &graph);
            if (rc) return (E.sticky = rc);
            CK(ce);
            CK(cudaGraphInstantiate(&E.gexec, graph, 0));
            cudaGraphDestroy(graph);
            E.glaunch = g_launches.load() - before;
            g_launches = before;  // captured launches run (and are counted) at replay
        }
        while (left >= Engine::CHUNK) {
            CK(cudaGraphLaunch(E.gexec, E.stream));
            count_launches(E.glaunch);
            left -= Engine::CHUNK;
            E.t += Engine::CHUNK;
        }
    }
    while (left > 0) {
        int rc = one_step();
        if (rc) return (E.sticky = rc);
        left--;
    }
    return PF_OK;
}

static int engine_sync(Engine &E)
{
    if (E.sticky) return E.sticky;
    cudaError_t e = cudaStreamSynchronize(E.stream);
    if (e != cudaSuccess) {
        E.sticky = fail(PF_ECUDA, "asynchronous error: %s", cudaGetErrorString(e));
        return E.sticky;
    }
    int flag = 0;
    CK(cudaMemcpy(&flag, E.d_flags, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag & 4) {
        E.sticky = fail(PF_ETIMEOUT, "a step kernel's bounded wait for its staged inputs ran out");
        return E.sticky;
    }
    if (flag & 1) return fail(PF_ENUMERIC, "a non-finite phi or u appeared");
    if (flag & 2)
        return fail(PF_ENUMERIC, "a 16-bit order-parameter population reached the storage range and was "
                                 "saturated (raise the flow lattice's resolution or lower store_log2_scale[0])");
    return PF_OK;
}

// tile tables and output buffer of the macroscopic pass, built once
static int engine_macro_tables(Engine &E)
{
    if (E.d_mdoms) return PF_OK;
    const int nd = (int)E.mem.size();
    long long nmax = 0;
    for (auto &m : E.mem) nmax = std::max(nmax, (long long)m.d.nx * m.d.ny * m.d.nz);
    // planes: phi, rho, u (dim), P, mu, phi0, W, V, and the interface normal (dim)
    CK(cudaMalloc(&E.d_macro, sizeof(double) * (size_t)(7 + 2 * E.dim) * nmax));
    int mtx = 32, mty = 8;
    if (E.dim == 3) tile_shape3d(E.prec, &mtx, &mty);
    // build_tiles writes the tiling into the DomainDev it is given: tile copies
    std::vector<DomainMem> copies(E.mem.begin(), E.mem.end());
    std::vector<DomainMem *> ds;
    for (auto &c : copies) ds.push_back(&c);
    std::vector<int> tdom;
    std::vector<int2> txy;
    build_tiles(ds, mtx, mty, tdom, txy);
    std::vector<DomainDev> dd(nd);
    E.mbase.assign(nd, 0);
    E.mcount.assign(nd, 0);
    for (int k = 0; k < nd; ++k) {
        dd[k] = copies[k].d;
        dd[k].macro = E.d_macro;
        E.mbase[k] = dd[k].tile_base;
        E.mcount[k] = dd[k].tiles_x * dd[k].tiles_y * dd[k].tiles_z;
    }
    CK(cudaMalloc(&E.d_mdoms, sizeof(DomainDev) * nd));
    CK(cudaMalloc(&E.d_mtdom, sizeof(int) * tdom.size()));
    CK(cudaMalloc(&E.d_mtxy, sizeof(int2) * txy.size()));
    CK(cudaMemcpy(E.d_mdoms, dd.data(), sizeof(DomainDev) * nd, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(E.d_mtdom, tdom.data(), sizeof(int) * tdom.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(E.d_mtxy, txy.data(), sizeof(int2) * txy.size(), cudaMemcpyHostToDevice));
    return PF_OK;
}

// the macro buffers of pf_batch_get_macros_all beyond the first (as many as
// fit in 256 MiB together, 0 .. PIPE - 1) and their domain tables (the first
// table with each domain's macro pointer moved to the buffer)
static int engine_macro_slots(Engine &E)
{
    int rc = engine_macro_tables(E);
    if (rc) return rc;
    if (E.nslots) return PF_OK;
    const int nd = (int)E.mem.size();
    long long nmax = 0;
    for (auto &m : E.mem) nmax = std::max(nmax, (long long)m.d.nx * m.d.ny * m.d.nz);
    const size_t bytes = sizeof(double) * (size_t)(7 + 2 * E.dim) * nmax;
    const int extra = (int)std::min<size_t>(Engine::PIPE - 1, ((size_t)256 << 20) / bytes);
    std::vector<DomainDev> dd(nd);
    CK(cudaMemcpy(dd.data(), E.d_mdoms, sizeof(DomainDev) * nd, cudaMemcpyDeviceToHost));
    for (int k = 0; k < extra; ++k) {
        CK(cudaMalloc(&E.d_macro_x[k], bytes));
        for (auto &d : dd) d.macro = E.d_macro_x[k];
        CK(cudaMalloc(&E.d_mdoms_x[k], sizeof(DomainDev) * nd));
        CK(cudaMemcpy(E.d_mdoms_x[k], dd.data(), sizeof(DomainDev) * nd, cudaMemcpyHostToDevice));
    }
    E.nslots = 1 + extra;
    return PF_OK;
}

// macroscopic pass of domain i into the engine's macro buffer (E.d_macro, or
// E.d_macro_x[slot - 1]; valid until the next macroscopic pass into it)
static int engine_macros(Engine &E, int i, int slot = 0)
{
    int rc = engine_macro_tables(E);
    if (rc) return rc;
    int mtx = 32, mty = 8;
    if (E.dim == 3) tile_shape3d(E.prec, &mtx, &mty);
    StepArgs a{};
    a.doms = slot ? E.d_mdoms_x[slot - 1] : E.d_mdoms;
    a.tile_dom = E.d_mtdom + E.mbase[i];
    a.tile_xy = E.d_mtxy + E.mbase[i];
    a.ntiles = E.mcount[i];
    a.par = E.par;
    a.parts = E.d_parts;
    a.np = E.np;
    a.partials = nullptr;
    a.flags = E.d_flags;
    a.wv = E.wv;
    const int grid = std::min<int>(E.mcount[i], E.nsm * 4);
    if (!launch_any(E, mtx, mty, MODE_MACROS, grid, a))
        return fail(PF_EINVAL, "macro kernel not built");
    CK(cudaGetLastError());
    return PF_OK;
}

// the macroscopic pass of domain i and the copies of the requested fields,
// queued on the engine's stream (the caller waits)
static int engine_queue_macros(Engine &E, int i, double *phi, double *rho, double *u, double *P, double *mu,
                               int where)
{
    int rc = engine_macros(E, i);
    if (rc) return rc;
    const DomainMem &m = E.mem[i];
    const long long N = (long long)m.d.nx * m.d.ny * m.d.nz;
    const cudaMemcpyKind kind = where == PF_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const int d = E.dim;
    const double *mac = E.d_macro;
    // stream-ordered copies after the macroscopic pass, then one wait
    if (phi) CK(cudaMemcpyAsync(phi, mac, sizeof(double) * N, kind, E.stream));
    if (rho) CK(cudaMemcpyAsync(rho, mac + N, sizeof(double) * N, kind, E.stream));
    if (u) CK(cudaMemcpyAsync(u, mac + 2 * N, sizeof(double) * d * N, kind, E.stream));
    if (P) CK(cudaMemcpyAsync(P, mac + (2 + d) * N, sizeof(double) * N, kind, E.stream));
    if (mu) CK(cudaMemcpyAsync(mu, mac + (3 + d) * N, sizeof(double) * N, kind, E.stream));
    return PF_OK;
}

static int engine_get_macros(Engine &E, int i, double *phi, double *rho, double *u, double *P,
                             double *mu, int where)
{
    PfRange range("pf_get_macros");
    if (where != PF_HOST && where != PF_DEVICE) return fail(PF_EINVAL, "where must be PF_HOST or PF_DEVICE");
    if (!E.inited[i]) return fail(PF_ESTATE, "pf_get_macros before pf_init_fields");
    int rc = engine_sync(E);
    if (rc && rc != PF_ENUMERIC) return rc;
    rc = engine_queue_macros(E, i, phi, rho, u, P, mu, where);
    if (rc) return rc;
    CK(cudaStreamSynchronize(E.stream));
    return PF_OK;
}

// interface normal n = grad phi / |grad phi| of domain i (0 where |grad phi|^2 <= 1e-24)
static int engine_get_normal(Engine &E, int i, double *n, int where)
{
    if (!n) return fail(PF_EINVAL, "n is NULL");
    if (where != PF_HOST && where != PF_DEVICE) return fail(PF_EINVAL, "where must be PF_HOST or PF_DEVICE");
    if (!E.inited[i]) return fail(PF_ESTATE, "pf_get_normal before pf_init_fields");
    PfRange range("pf_get_normal");
    int rc = engine_sync(E);
    if (rc && rc != PF_ENUMERIC) return rc;
    rc = engine_macros(E, i);
    if (rc) return rc;
    DomainDev dd = E.mem[i].d;
    dd.macro = E.d_macro;
    const long long N = (long long)dd.nx * dd.ny * dd.nz;
    double *dst = where == PF_DEVICE ? n : E.d_macro + (size_t)(7 + E.dim) * N;
    launch_normal(dd, dst, E.stream);
    CK(cudaGetLastError());
    if (where == PF_HOST)
        CK(cudaMemcpyAsync(n, dst, sizeof(double) * E.dim * N, cudaMemcpyDeviceToHost, E.stream));
    CK(cudaStreamSynchronize(E.stream));
    return PF_OK;
}

static int engine_diag(Engine &E, int i, pf_diag *out)
{
    PfRange range("pf_diagnostics");
    if (!out) return fail(PF_EINVAL, "out is NULL");
    if (!E.inited[i]) return fail(PF_ESTATE, "pf_diagnostics before pf_init_fields");
    int rc = engine_sync(E);
    int nan_flag = 0;
    if (rc == PF_ENUMERIC) CK(cudaMemcpy(&nan_flag, E.d_flags, sizeof(int), cudaMemcpyDeviceToHost));
    if (rc && rc != PF_ENUMERIC) return rc;
    rc = engine_macros(E, i);
    if (rc) return rc;
    DomainDev dd = E.mem[i].d;
    dd.macro = E.d_macro;
    double *partial = E.d_diag, *res = E.d_diag + 3 * diag_blocks();
    launch_diag(dd, partial, res, E.wv, E.stream);
    CK(cudaGetLastError());
    double h[3];
    CK(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, E.stream));
    CK(cudaStreamSynchronize(E.stream));
    out->mass = h[0];
    out->E_F = h[1];
    out->E_K = h[2];
    out->E_total = h[1] + h[2];
    out->nan_flag = nan_flag;
    return PF_OK;
}

static int engine_force(Engine &E, int tile_x, int tile_y, int kernel, int ctas_per_sm);

// ---------------------------------------------------------------------------------------------
// single-domain handle
// ---------------------------------------------------------------------------------------------
struct pf_handle {
    Engine E;
};

extern "C" int pf_create(const pf_grid *g, const pf_params *p, pf_handle **out)
{
    PfRange range("pf_create");
    if (!out) return fail(PF_EINVAL, "out is NULL");
    int rc = validate(g, p);
    if (rc) return rc;
    pf_handle *h = new (std::nothrow) pf_handle();
    if (!h) return fail(PF_ENOMEM, "host allocation failed");
    rc = engine_setup(h->E, 1, g, p);
    if (rc) {
        engine_free(h->E);
        delete h;
        return rc;
    }
    *out = h;
    return PF_OK;
}

extern "C" void pf_destroy(pf_handle *h)
{
    if (!h) return;
    if (h->E.stream) cudaStreamSynchronize(h->E.stream);
    engine_free(h->E);
    delete h;
}

static int upload_particles(Engine &E)
{
    CK(cudaMemcpy(E.d_parts, E.hp, sizeof(ParticleDev) * std::max(E.np, 1), cudaMemcpyHostToDevice));
    return PF_OK;
}

extern "C" int pf_init_fields(pf_handle *h, const double *phi0, const double *phi, const double *u,
                              const double *P, int where)
{
    PfRange range("pf_init_fields");
    if (!h) return fail(PF_EINVAL, "handle is NULL");
    Engine &E = h->E;
    if (E.sticky) return E.sticky;
    CK(cudaStreamSynchronize(E.stream));
    int rc = upload_particles(E);
    if (rc) return rc;
    // the fresh state starts at parity 0; reset previous-velocity memory of particles
    for (int k = 0; k < E.np; ++k)
        for (int a = 0; a < 3; ++a) {
            E.hp[k].u_prev[a] = E.hp[k].u[a];
            E.hp[k].w_prev[a] = E.hp[k].w[a];
        }
    rc = upload_particles(E);
    if (rc) return rc;
    CK(cudaMemsetAsync(E.d_flags, 0, sizeof(int) * 4, E.stream));
    E.ghosts_ok = false;
    rc = domain_init(E.mem[0], E.staging, E.dim, E.prec, phi0, phi, u, P, where, E.d_parts, E.hp, E.np, E.d_flags,
                     E.stream);
    if (rc) return rc;
    CK(cudaStreamSynchronize(E.stream));
    staging_release(E.staging);
    E.par = 0;
    E.t = 0;
    E.inited[0] = true;
    return PF_OK;
}

extern "C" int pf_set_config(pf_handle *h, int tile_x, int tile_y, int kernel, int ctas_per_sm)
{
    if (!h) return fail(PF_EINVAL, "handle is NULL");
    for (size_t i = 0; i < h->E.inited.size(); ++i)
        if (!h->E.inited[i]) return fail(PF_ESTATE, "pf_set_config before pf_init_fields");
    return engine_force(h->E, tile_x, tile_y, kernel, ctas_per_sm);
}

extern "C" int pf_step(pf_handle *h, int64_t n)
{
    PfRange range("pf_step");
    if (!h) return fail(PF_EINVAL, "handle is NULL");
    return engine_step(h->E, n, false);
}

extern "C" int pf_autotune(pf_handle *h, int64_t *steps_taken)
{
    PfRange range("pf_autotune");
    if (!h) return fail(PF_EINVAL, "handle is NULL");
    Engine &E = h->E;
    if (E.sticky) return E.sticky;
    for (size_t i = 0; i < E.mem.size(); ++i)
        if (!E.inited[i]) return fail(PF_ESTATE, "pf_autotune before pf_init_fields");
    const int64_t t0 = E.t;
    while (E.par != 0) {  // the candidates start at parity 0
        int rc = issue_step(E, E.par);
        if (rc) return (E.sticky = rc);
        E.par ^= 1;
        E.t++;
    }
    E.tuned = false;
    E.forced = false;
    int rc = engine_configure(E, true);
    if (rc) return (E.sticky = rc);
    if (steps_taken) *steps_taken = E.t - t0;
    return PF_OK;
}

extern "C" int pf_sync(pf_handle *h)
{
    if (!h) return fail(PF_EINVAL, "handle is NULL");
    return engine_sync(h->E);
}

extern "C" int64_t pf_time(pf_handle *h) { return h ? h->E.t : -1; }

extern "C" int pf_get_macros(pf_handle *h, double *phi, double *rho, double *u, double *P, double *mu,
                             int where)
{
    if (!h) return fail(PF_EINVAL, "handle is NULL");
    return engine_get_macros(h->E, 0, phi, rho, u, P, mu, where);
}

extern "C" int pf_get_normal(pf_handle *h, double *n, int where)
{
    if (!h) return fail(PF_EINVAL, "handle is NULL");
    return engine_get_normal(h->E, 0, n, where);
}

extern "C" int pf_diagnostics(pf_handle *h, pf_diag *out)
{
    if (!h) return fail(PF_EINVAL, "handle is NULL");
    return engine_diag(h->E, 0, out);
}

// ---- checkpoint / resume ----------------------------------------------------------------------
// The state that the next step reads: the current populations, the PMIX rest
// populations, the lagged fields, the fixed indicator, the particles and the
// time.  Loading it into a handle created with the same grid, parameters and
// particle count continues the run bit for bit (the step has no randomness).
struct PfStateHeader {
    char magic[8];
    int version, dim, prec, nx, ny, nz, np, wall_y;
    long long t, fb, rb, ab, pb;
};

static void state_sizes(const Engine &E, size_t &fb, size_t &rb, size_t &ab, size_t &pb)
{
    const DomainDev &d = E.mem[0].d;
    const int Q = E.dim == 2 ? 18 : 26, naux = 2 * E.dim + 1;
    fb = (size_t)Q * d.plane * store_bytes(E.prec);
    rb = E.prec >= PF_PMIX_FP16 ? (size_t)d.plane * 8 : 0;
    ab = (size_t)naux * d.plane * aux_bytes(E.prec);
    pb = (size_t)d.plane * aux_bytes(E.prec);
}

static size_t state_bytes(const Engine &E)
{
    size_t fb, rb, ab, pb;
    state_sizes(E, fb, rb, ab, pb);
    return sizeof(PfStateHeader) + fb + rb + ab + pb + sizeof(ParticleDev) * (size_t)E.np;
}

extern "C" int pf_state_size(pf_handle *h, int64_t *bytes)
{
    if (!h || !bytes) return fail(PF_EINVAL, "NULL argument");
    *bytes = (int64_t)state_bytes(h->E);
    return PF_OK;
}

extern "C" int pf_save_state(pf_handle *h, void *buf, int64_t bytes)
{
    if (!h || !buf) return fail(PF_EINVAL, "NULL argument");
    Engine &E = h->E;
    if (!E.inited[0]) return fail(PF_ESTATE, "pf_save_state before pf_init_fields");
    if (bytes < (int64_t)state_bytes(E)) return fail(PF_EINVAL, "buffer of %lld bytes is smaller than the state (%lld)",
                                                    (long long)bytes, (long long)state_bytes(E));
    PfRange range("pf_save_state");
    int rc = engine_sync(E);
    if (rc) return rc;
    const DomainDev &d = E.mem[0].d;
    PfStateHeader hd{};
    memcpy(hd.magic, "PFSTATE", 8);
    hd.version = 1;
    hd.dim = E.dim;
    hd.prec = E.prec;
    hd.nx = d.nx;
    hd.ny = d.ny;
    hd.nz = d.nz;
    hd.np = E.np;
    hd.wall_y = d.wall_y;
    hd.t = E.t;
    size_t fb, rb, ab, pb;
    state_sizes(E, fb, rb, ab, pb);
    hd.fb = (long long)fb;
    hd.rb = (long long)rb;
    hd.ab = (long long)ab;
    hd.pb = (long long)pb;
    char *o = static_cast<char *>(buf);
    memcpy(o, &hd, sizeof(hd));
    o += sizeof(hd);
    CK(cudaMemcpy(o, d.f[E.par], fb, cudaMemcpyDeviceToHost));
    o += fb;
    if (rb) CK(cudaMemcpy(o, d.rest[E.par], rb, cudaMemcpyDeviceToHost));
    o += rb;
    CK(cudaMemcpy(o, d.aux[E.par], ab, cudaMemcpyDeviceToHost));
    o += ab;
    CK(cudaMemcpy(o, d.phi0, pb, cudaMemcpyDeviceToHost));
    o += pb;
    if (E.np) CK(cudaMemcpy(o, E.d_parts, sizeof(ParticleDev) * E.np, cudaMemcpyDeviceToHost));
    return PF_OK;
}

extern "C" int pf_load_state(pf_handle *h, const void *buf, int64_t bytes)
{
    if (!h || !buf) return fail(PF_EINVAL, "NULL argument");
    Engine &E = h->E;
    if (bytes < (int64_t)sizeof(PfStateHeader)) return fail(PF_EINVAL, "buffer too small for a state header");
    PfStateHeader hd;
    memcpy(&hd, buf, sizeof(hd));
    const DomainDev &d = E.mem[0].d;
    size_t fb, rb, ab, pb;
    state_sizes(E, fb, rb, ab, pb);
    if (memcmp(hd.magic, "PFSTATE", 8) != 0 || hd.version != 1) return fail(PF_EINVAL, "not a libpf state");
    if (hd.dim != E.dim || hd.prec != E.prec || hd.nx != d.nx || hd.ny != d.ny || hd.nz != d.nz ||
        hd.wall_y != d.wall_y || hd.fb != (long long)fb || hd.rb != (long long)rb || hd.ab != (long long)ab ||
        hd.pb != (long long)pb)
        return fail(PF_EINVAL, "the state was saved from another grid or precision");
    if (hd.np != E.np)
        return fail(PF_EINVAL, "the state holds %d particles, the handle %d: set as many before loading", hd.np,
                    E.np);
    if (bytes < (int64_t)state_bytes(E)) return fail(PF_EINVAL, "buffer shorter than the state it announces");
    if (E.sticky) return E.sticky;
    PfRange range("pf_load_state");
    CK(cudaStreamSynchronize(E.stream));
    const char *in = static_cast<const char *>(buf) + sizeof(hd);
    CK(cudaMemcpy(d.f[E.par], in, fb, cudaMemcpyHostToDevice));
    in += fb;
    if (rb) CK(cudaMemcpy(d.rest[E.par], in, rb, cudaMemcpyHostToDevice));
    in += rb;
    CK(cudaMemcpy(d.aux[E.par], in, ab, cudaMemcpyHostToDevice));
    in += ab;
    CK(cudaMemcpy(d.phi0, in, pb, cudaMemcpyHostToDevice));
    in += pb;
    if (E.np) {
        memcpy(E.hp, in, sizeof(ParticleDev) * E.np);
        int wv = 0;
        for (int j = 0; j < E.np; ++j) wv |= E.hp[j].own;
        if (wv != E.wv) drop_graph(E);
        E.wv = wv;
        int rc = upload_particles(E);
        if (rc) return rc;
    }
    E.ghosts_ok = false;
    CK(cudaMemset(E.d_flags, 0, sizeof(int) * 4));
    E.t = hd.t;
    E.inited[0] = true;
    return PF_OK;
}

extern "C" int pf_num_particles(pf_handle *h) { return h ? h->E.np : -1; }

extern "C" int pf_particle_state(pf_handle *h, int k, pf_particle *io, int set)
{
    if (!h || !io) return fail(PF_EINVAL, "NULL argument");
    Engine &E = h->E;
    if (E.sticky) return E.sticky;
    CK(cudaStreamSynchronize(E.stream));
    if (set) {
        if (k < 0 || k > E.np || k >= PF_MAX_PARTICLES)
            return fail(PF_EINVAL, "particle index %d out of range (count %d)", k, E.np);
        if (!(io->R > 0) || !(io->rho_p > 0)) return fail(PF_EINVAL, "particle needs R > 0 and rho_p > 0");
        const bool own = !std::isnan(io->theta_deg);
        if (own && !(io->theta_deg > 0 && io->theta_deg < 180))
            return fail(PF_EINVAL, "particle theta_deg must be NaN or lie in (0, 180)");
        if (io->prescribed < 0 || io->prescribed > 31)
            return fail(PF_EINVAL, "particle prescribed flags must lie in 0..31");
        if (E.np > 0) CK(cudaMemcpy(E.hp, E.d_parts, sizeof(ParticleDev) * E.np, cudaMemcpyDeviceToHost));
        ParticleDev &pp = E.hp[k];
        memset(&pp, 0, sizeof(pp));
        for (int a = 0; a < 3; ++a) {
            pp.x[a] = io->x[a];
            pp.u[a] = io->u[a];
            pp.w[a] = io->w[a];
            pp.u_prev[a] = io->u[a];
            pp.w_prev[a] = io->w[a];
        }
        pp.R = io->R;
        pp.rho_p = io->rho_p;
        pp.theta_deg = own ? io->theta_deg : NAN;
        pp.prescribed = io->prescribed;
        pp.own = own ? 1 : 0;
        pp.ct = own ? std::cos(io->theta_deg * 3.14159265358979323846 / 180.0) : 0.0;
        const bool grew = k == E.np;
        if (grew) E.np++;
        int wv = 0;
        for (int j = 0; j < E.np; ++j) wv |= E.hp[j].own;
        if (wv != E.wv) drop_graph(E);  // the step arguments change
        E.wv = wv;
        if (E.variant == 3 && !split_ok(E)) {  // (not reached: own angles keep the split)
            E.variant = 0;
            int rc0 = engine_tiles(E, E.tx, E.ty);
            if (rc0) return rc0;
            E.grid = grid_of(E, E.cps);
            drop_graph(E);
        }
        int rc = upload_particles(E);
        if (rc) return rc;
        if (grew) {
            // partial-sum table grows with the particle count; graphs bake the count in
            if (E.tuned) {
                if (E.variant) {  // the two-cells-per-thread step has no particle terms
                    E.variant = 0;
                    E.tx = 32;
                    E.ty = 8;
                }
                rc = engine_tiles(E, E.tx, E.ty);
                if (rc) return rc;
                E.grid = E.ntiles;
            }
            drop_graph(E);
        }
        return PF_OK;
    }
    if (k < 0 || k >= E.np) return fail(PF_EINVAL, "particle index %d out of range (count %d)", k, E.np);
    ParticleDev pp;
    CK(cudaMemcpy(&pp, E.d_parts + k, sizeof(pp), cudaMemcpyDeviceToHost));
    for (int a = 0; a < 3; ++a) {
        io->x[a] = pp.x[a];
        io->u[a] = pp.u[a];
        io->w[a] = pp.w[a];
        io->F[a] = pp.F[a];
        io->T[a] = pp.T[a];
    }
    io->R = pp.R;
    io->rho_p = pp.rho_p;
    io->theta_deg = pp.theta_deg;
    io->prescribed = pp.prescribed;
    return PF_OK;
}

// ---------------------------------------------------------------------------------------------
// batched domains
// ---------------------------------------------------------------------------------------------
struct pf_batch {
    Engine E;
};

extern "C" int pf_batch_create(int nd, const pf_grid *g, const pf_params *p, pf_batch **out)
{
    PfRange range("pf_batch_create");
    if (!out || nd < 1 || !g || !p) return fail(PF_EINVAL, "bad arguments");
    for (int i = 0; i < nd; ++i) {
        int rc = validate(&g[i], &p[i]);
        if (rc) return rc;
        if (g[i].dim != g[0].dim || p[i].precision != p[0].precision)
            return fail(PF_EINVAL, "all domains of a batch share dim and precision");
    }
    pf_batch *b = new (std::nothrow) pf_batch();
    if (!b) return fail(PF_ENOMEM, "host allocation failed");
    int rc = engine_setup(b->E, nd, g, p);
    if (rc) {
        engine_free(b->E);
        delete b;
        return rc;
    }
    *out = b;
    return PF_OK;
}

extern "C" int pf_batch_init(pf_batch *b, int i, const double *phi0, const double *phi, const double *u,
                             const double *P, int where)
{
    PfRange range("pf_batch_init");
    if (!b) return fail(PF_EINVAL, "batch is NULL");
    Engine &E = b->E;
    if (i < 0 || i >= (int)E.mem.size()) return fail(PF_EINVAL, "domain index %d out of range", i);
    if (E.sticky) return E.sticky;
    if (E.t != 0) return fail(PF_ESTATE, "all domains are initialised before the first step");
    E.ghosts_ok = false;
    int rc = domain_init(E.mem[i], E.staging, E.dim, E.prec, phi0, phi, u, P, where, E.d_parts, nullptr, 0, E.d_flags,
                         E.stream);
    if (rc) return rc;
    CK(cudaStreamSynchronize(E.stream));
    E.inited[i] = true;
    return PF_OK;
}

extern "C" int pf_batch_init_all(pf_batch *b, const double *const *phi0, const double *const *phi,
                                 const double *const *u, const double *const *P, int where)
{
    PfRange range("pf_batch_init_all");
    if (!b) return fail(PF_EINVAL, "batch is NULL");
    if (!phi0 || !phi) return fail(PF_EINVAL, "phi0 and phi are required");
    if (where != PF_HOST && where != PF_DEVICE) return fail(PF_EINVAL, "where must be PF_HOST or PF_DEVICE");
    Engine &E = b->E;
    if (E.sticky) return E.sticky;
    if (E.t != 0) return fail(PF_ESTATE, "all domains are initialised before the first step");
    const int nd = (int)E.mem.size();
    for (int i = 0; i < nd; ++i)
        if (!phi0[i] || !phi[i]) return fail(PF_EINVAL, "phi0 and phi are required (domain %d)", i);
    E.ghosts_ok = false;
    constexpr int NS = Engine::KS;
    auto cells = [&](int i) { return (size_t)E.mem[i].d.nx * E.mem[i].d.ny * E.mem[i].d.nz; };
    size_t nbig = 0;
    for (int i = 0; i < nd; ++i) nbig = std::max(nbig, cells(i));
    // each kernel stream's scratch for the init kernels (phi0tot, mu, W, V of
    // the largest domain); as many streams as keep the scratch within 512 MiB
    // (the streams help batches of small domains: their kernels are short)
    const size_t per = sizeof(double) * 4 * std::max<size_t>(nbig, 1);
    const int ns = (int)std::min<size_t>(NS, std::max<size_t>(1, ((size_t)512 << 20) / per));
    int rc = staging_reserve_n(E.staging, (size_t)ns * 4 * nbig);
    if (rc) return rc;
    if (!E.cstream) CK(cudaStreamCreateWithFlags(&E.cstream, cudaStreamNonBlocking));
    for (int k = 0; k < ns - 1; ++k)
        if (!E.kstream[k]) CK(cudaStreamCreateWithFlags(&E.kstream[k], cudaStreamNonBlocking));
    for (cudaEvent_t *ev : {&E.ev_in, &E.ev_start})
        if (!*ev) CK(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
    cudaStream_t ks[NS];
    ks[0] = E.stream;
    for (int k = 0; k < ns; ++k) {
        if (!E.ev_k[k]) CK(cudaEventCreateWithFlags(&E.ev_k[k], cudaEventDisableTiming));
        if (k) ks[k] = E.kstream[k - 1];
    }
    const int d = E.dim;
    const bool host = where == PF_HOST;
    // host arrays: copied on the copy stream into a ring of device memory
    // (2^25 doubles, or PF_INIT_RING; at least one domain's inputs), each
    // domain's kernels waiting for its own copies; when the ring wraps, the
    // copy stream first waits for the kernels of every domain queued so far.
    // Device arrays are read in place.
    auto need = [&](int i) { return (size_t)(2 + (u && u[i] ? d : 0) + (P && P[i] ? 1 : 0)) * cells(i); };
    size_t cap = 0;
    double *ring = nullptr;
    if (host) {
        cap = E.init_ring > 0 ? (size_t)E.init_ring : (size_t)1 << 25;
        for (int i = 0; i < nd; ++i) cap = std::max(cap, need(i));
        CK(cudaMalloc(&ring, sizeof(double) * cap));
    }
    bool ok = true;
    auto cuok = [&](cudaError_t e) { ok = ok && e == cudaSuccess; };
    // the other kernel streams start after the work already queued on the batch's stream
    cuok(cudaEventRecord(E.ev_start, E.stream));
    for (int k = 1; k < ns; ++k) cuok(cudaStreamWaitEvent(ks[k], E.ev_start, 0));
    if (host) cuok(cudaStreamWaitEvent(E.cstream, E.ev_start, 0));
    size_t off = 0;
    for (int i = 0; i < nd && ok && rc == PF_OK; ++i) {
        const size_t N = cells(i);
        cudaStream_t s = ks[i % ns];
        const double *a0 = phi0[i], *a1 = phi[i], *au = u ? u[i] : nullptr, *aP = P ? P[i] : nullptr;
        if (host) {
            if (off + need(i) > cap) {
                for (int k = 0; k < ns; ++k) {
                    cuok(cudaEventRecord(E.ev_k[k], ks[k]));
                    cuok(cudaStreamWaitEvent(E.cstream, E.ev_k[k], 0));
                }
                off = 0;
            }
            double *s0 = ring + off, *s1 = s0 + N, *su = s1 + N, *sP = su + (au ? (size_t)d * N : 0);
            cuok(cudaMemcpyAsync(s0, a0, sizeof(double) * N, cudaMemcpyHostToDevice, E.cstream));
            cuok(cudaMemcpyAsync(s1, a1, sizeof(double) * N, cudaMemcpyHostToDevice, E.cstream));
            if (au) cuok(cudaMemcpyAsync(su, au, sizeof(double) * d * N, cudaMemcpyHostToDevice, E.cstream));
            if (aP) cuok(cudaMemcpyAsync(sP, aP, sizeof(double) * N, cudaMemcpyHostToDevice, E.cstream));
            cuok(cudaEventRecord(E.ev_in, E.cstream));
            cuok(cudaStreamWaitEvent(s, E.ev_in, 0));
            off += need(i);
            a0 = s0;
            a1 = s1;
            au = au ? su : nullptr;
            aP = aP ? sP : nullptr;
        }
        if (ok)
            rc = domain_init_kernels(E.mem[i], E.prec, a0, a1, au, aP, E.staging.p + (size_t)(i % ns) * 4 * nbig,
                                     E.d_parts, nullptr, 0, E.d_flags, s);
    }
    const cudaError_t last = cudaGetLastError();
    // the batch's stream continues after every kernel stream
    for (int k = 1; k < ns; ++k) {
        cudaEventRecord(E.ev_k[k], ks[k]);
        cudaStreamWaitEvent(E.stream, E.ev_k[k], 0);
    }
    cudaError_t es = host ? cudaStreamSynchronize(E.cstream) : cudaSuccess;
    for (int k = 0; k < ns; ++k) {
        const cudaError_t e = cudaStreamSynchronize(ks[k]);
        if (es == cudaSuccess) es = e;
    }
    if (ring) cudaFree(ring);
    if (rc) return rc;
    if (!ok) return fail(PF_ECUDA, "init_all: %s", cudaGetErrorString(last));
    if (es != cudaSuccess) return fail(PF_ECUDA, "init_all: %s", cudaGetErrorString(es));
    for (int i = 0; i < nd; ++i) E.inited[i] = true;
    return PF_OK;
}

extern "C" int pf_batch_step(pf_batch *b, int64_t n)
{
    PfRange range("pf_batch_step");
    if (!b) return fail(PF_EINVAL, "batch is NULL");
    return engine_step(b->E, n, true);
}

extern "C" int pf_batch_sync(pf_batch *b)
{
    if (!b) return fail(PF_EINVAL, "batch is NULL");
    return engine_sync(b->E);
}

extern "C" int pf_batch_get_macros(pf_batch *b, int i, double *phi, double *rho, double *u, double *P,
                                   double *mu, int where)
{
    if (!b) return fail(PF_EINVAL, "batch is NULL");
    if (i < 0 || i >= (int)b->E.mem.size()) return fail(PF_EINVAL, "domain index %d out of range", i);
    return engine_get_macros(b->E, i, phi, rho, u, P, mu, where);
}

extern "C" int pf_batch_get_macros_all(pf_batch *b, double *const *phi, double *const *rho, double *const *u,
                                       double *const *P, double *const *mu, int where)
{
    PfRange range("pf_batch_get_macros_all");
    if (!b) return fail(PF_EINVAL, "batch is NULL");
    Engine &E = b->E;
    if (where != PF_HOST && where != PF_DEVICE) return fail(PF_EINVAL, "where must be PF_HOST or PF_DEVICE");
    for (size_t i = 0; i < E.mem.size(); ++i)
        if (!E.inited[i]) return fail(PF_ESTATE, "pf_batch_get_macros_all before every domain is initialised");
    int rc = engine_sync(E);
    if (rc && rc != PF_ENUMERIC) return rc;
    rc = engine_macro_slots(E);
    if (rc) return rc;
    if (!E.cstream) CK(cudaStreamCreateWithFlags(&E.cstream, cudaStreamNonBlocking));
    for (int k = 0; k < E.nslots; ++k) {
        if (!E.ev_k[k]) CK(cudaEventCreateWithFlags(&E.ev_k[k], cudaEventDisableTiming));
        if (!E.ev_c[k]) CK(cudaEventCreateWithFlags(&E.ev_c[k], cudaEventDisableTiming));
    }
    // domain i: its macroscopic pass into buffer i % nslots on the batch's
    // stream (after the copies of domain i - nslots out of that buffer), its
    // copies on the copy stream (after that pass)
    const cudaMemcpyKind kind = where == PF_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const int d = E.dim, ns = E.nslots;
    bool ok = true;
    for (size_t i = 0; i < E.mem.size() && ok && rc == PF_OK; ++i) {
        const int slot = (int)(i % ns);
        if (i >= (size_t)ns) ok = cudaStreamWaitEvent(E.stream, E.ev_c[slot], 0) == cudaSuccess;
        if (ok) rc = engine_macros(E, (int)i, slot);
        if (rc) break;
        const long long N = (long long)E.mem[i].d.nx * E.mem[i].d.ny * E.mem[i].d.nz;
        const double *mac = slot ? E.d_macro_x[slot - 1] : E.d_macro;
        ok = ok && cudaEventRecord(E.ev_k[slot], E.stream) == cudaSuccess &&
             cudaStreamWaitEvent(E.cstream, E.ev_k[slot], 0) == cudaSuccess;
        auto cp = [&](double *const *dst, const double *src, long long n) {
            if (ok && dst && dst[i])
                ok = cudaMemcpyAsync(dst[i], src, sizeof(double) * n, kind, E.cstream) == cudaSuccess;
        };
        cp(phi, mac, N);
        cp(rho, mac + N, N);
        cp(u, mac + 2 * N, (long long)d * N);
        cp(P, mac + (2 + d) * N, N);
        cp(mu, mac + (3 + d) * N, N);
        ok = ok && cudaEventRecord(E.ev_c[slot], E.cstream) == cudaSuccess;
    }
    const cudaError_t last = cudaGetLastError();
    const cudaError_t e1 = cudaStreamSynchronize(E.cstream), e2 = cudaStreamSynchronize(E.stream);
    if (rc) return rc;
    if (!ok) return fail(PF_ECUDA, "get_macros_all: %s", cudaGetErrorString(last));
    if (e1 != cudaSuccess || e2 != cudaSuccess)
        return fail(PF_ECUDA, "get_macros_all: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    return PF_OK;
}

extern "C" int pf_batch_diagnostics(pf_batch *b, int i, pf_diag *out)
{
    if (!b) return fail(PF_EINVAL, "batch is NULL");
    if (i < 0 || i >= (int)b->E.mem.size()) return fail(PF_EINVAL, "domain index %d out of range", i);
    return engine_diag(b->E, i, out);
}

extern "C" int64_t pf_batch_cells(pf_batch *b)
{
    if (!b) return -1;
    long long c = 0;
    for (auto &m : b->E.mem) c += (long long)m.d.nx * m.d.ny * m.d.nz;
    return c;
}

static int engine_config(const Engine &E, int *tile_x, int *tile_y, int *ctas_per_sm, int *kernel)
{
    const bool t = E.tuned;
    if (tile_x) *tile_x = t ? E.tx : -1;
    if (tile_y) *tile_y = t ? E.ty : -1;
    if (ctas_per_sm) *ctas_per_sm = t ? E.cps : -1;
    if (kernel) *kernel = t ? E.variant : -1;
    return PF_OK;
}

extern "C" int pf_batch_config(pf_batch *b, int *tile_x, int *tile_y, int *ctas_per_sm, int *kernel)
{
    if (!b) return fail(PF_EINVAL, "batch is NULL");
    return engine_config(b->E, tile_x, tile_y, ctas_per_sm, kernel);
}

extern "C" int pf_get_config(pf_handle *h, int *tile_x, int *tile_y, int *ctas_per_sm, int *kernel)
{
    if (!h) return fail(PF_EINVAL, "handle is NULL");
    return engine_config(h->E, tile_x, tile_y, ctas_per_sm, kernel);
}

// fixed launch configuration (skips the autotuner)
static int engine_force(Engine &E, int tile_x, int tile_y, int kernel, int ctas_per_sm)
{
    if (E.sticky) return E.sticky;
    const int var = kernel;
    if (var < 0 || var > 4) return fail(PF_EINVAL, "kernel must be 0, 1, 2, 3 or 4");
    if (var == 4 && (!strip_ok(E) || tile_x != STRIP_SW || tile_y < 1))
        return fail(PF_EINVAL, "kernel 4 (strips marched in y) needs 2D domains in FP32 or 16-bit storage without "
                               "particles, every nx even and >= %d, tile_x = %d (the strip width) and tile_y >= 1 "
                               "(the segment rows)", STRIP_GHOST, STRIP_SW);
    if (var == 3 && (!split_ok(E) || tile_x != 32 || tile_y != 16))
        return fail(PF_EINVAL, "kernel 3 (near tiles single-cell with the particle terms, far tiles without) "
                               "needs one 2D particle domain in FP32 or 16-bit storage without the Allen-Cahn "
                               "lattice, and 32x16 tiles");
    if (ctas_per_sm < 0) return fail(PF_EINVAL, "ctas_per_sm must be >= 0");
    if (var != 0 && var != 3 && var != 4 && any_walls(E))
        return fail(PF_EINVAL, "domains with walls run kernels 0, 3 and 4 only");
    if (var == 2 && !stage_ok(E))
        return fail(PF_EINVAL, "kernel 2 needs 2D, FP32 or 16-bit storage, no particles and every nx a "
                               "multiple of %d", E.prec == PF_P32 ? 4 : 8);
    const int mode = var == 4 ? MODE_STEP_STRIP : var == 2 ? MODE_STEP_STAGE : (var == 1 ? MODE_STEP_PAIR : MODE_STEP);
    if (occupancy_any(E, tile_x, tile_y, mode) < 1 ||
        (var == 3 && !any_walls(E) && occupancy_any(E, tile_x, tile_y, MODE_STEP_PAIR | MODE_MU0) < 1)) {
        return fail(PF_EINVAL, "launch configuration %dx%d of kernel %d is not built for this precision / "
                    "particle setting", tile_x, tile_y, var);
    }
    while (E.par != 0) {  // keep graph chunks starting at parity 0
        int rc = issue_step(E, E.par);
        if (rc) return (E.sticky = rc);
        E.par ^= 1;
        E.t++;
    }
    E.variant = var;
    int rc = engine_tiles(E, var == 4 ? 32 : tile_x, var == 4 ? 8 : tile_y);
    if (rc) return (E.sticky = rc);
    E.tx = tile_x;
    E.ty = tile_y;
    E.cps = ctas_per_sm;
    if (var == 3) {
        rc = split_setup(E);
        if (rc) return (E.sticky = rc);
    }
    if (var == 4) {
        rc = strip_setup(E, tile_y);
        if (rc) return (E.sticky = rc);
    }
    E.grid = grid_of(E, ctas_per_sm);
    E.tuned = true;
    E.forced = true;
    return PF_OK;
}

extern "C" int pf_batch_set_config(pf_batch *b, int tile_x, int tile_y, int kernel, int ctas_per_sm)
{
    if (!b) return fail(PF_EINVAL, "batch is NULL");
    return engine_force(b->E, tile_x, tile_y, kernel, ctas_per_sm);
}

extern "C" void pf_batch_destroy(pf_batch *b)
{
    if (!b) return;
    if (b->E.stream) cudaStreamSynchronize(b->E.stream);
    engine_free(b->E);
    delete b;
}
