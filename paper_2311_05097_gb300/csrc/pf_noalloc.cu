// Allocation-free FP64 diagnostics: the same quantities as pf_diagnostics
// (sum phi, the free energy of Eq. (8), the kinetic energy) computed from
// caller-provided device fields, with the reduction's scratch held in a
// fixed-size array in device global memory instead of memory the library
// allocates.
//
// Who needs it: code that must not call cudaMalloc/cudaFree -- work being
// recorded by CUDA stream capture (allocation calls are illegal there),
// real-time or fixed-budget loops, and hosts whose device memory belongs to
// another allocator.  The caller still provides every input and the output.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/pf.h"
#include "pf_internal.h"

namespace pf {

constexpr int NA_THREADS = 256;
constexpr int NA_CELLS_PER_THREAD = 16;
constexpr long long NA_CELLS_PER_BLOCK = (long long)NA_THREADS * NA_CELLS_PER_THREAD;  // 4096

// Scratch: one (mass, E_F, E_K) triple per block plus the final triple.
// Every GPU that loads the library holds this array until the process exits.
__device__ __align__(256) double g_noalloc_scratch[3 * (PF_NOALLOC_MAX_BLOCKS + 1)];

struct NAGeom {
    int dim, nx, ny, nz;
    int wall_y;  // walls at the ends of y (pf_grid.periodic[1] = 0): mirror rows
    double sigma, D, cos_t;
};

// row of a neighbour at y: periodic, or with walls the mirror image of the
// row inside (zero normal gradient, as in pf_diagnostics)
__device__ __forceinline__ int na_row(const NAGeom &g, int y)
{
    if (g.wall_y) return y < 0 ? -1 - y : (y >= g.ny ? 2 * g.ny - 1 - y : y);
    return wrap_idx(y, g.ny);
}

__device__ __forceinline__ long long na_lin(const NAGeom &g, int x, int y, int z)
{
    return ((long long)z * g.ny + y) * g.nx + x;
}

// isotropic gradient (D2Q9 / D3Q19 weights, cs^2 = 1/3): periodic wrap, and
// mirrored rows beyond walls at the ends of y
__device__ void na_grad(const NAGeom &g, const double *a, int x, int y, int z, double out[3])
{
    out[0] = out[1] = out[2] = 0.0;
    auto at = [&](int dx, int dy, int dz) {
        const int xx = wrap_idx(x + dx, g.nx), yy = na_row(g, y + dy),
                  zz = g.dim == 3 ? wrap_idx(z + dz, g.nz) : 0;
        return a[na_lin(g, xx, yy, zz)];
    };
    if (g.dim == 2) {
        out[0] = (at(1, 0, 0) - at(-1, 0, 0)) / 3.0 +
                 (at(1, 1, 0) + at(1, -1, 0) - at(-1, 1, 0) - at(-1, -1, 0)) / 12.0;
        out[1] = (at(0, 1, 0) - at(0, -1, 0)) / 3.0 +
                 (at(1, 1, 0) + at(-1, 1, 0) - at(1, -1, 0) - at(-1, -1, 0)) / 12.0;
        return;
    }
    for (int a = 0; a < 3; ++a) {
        int e[3] = {0, 0, 0};
        e[a] = 1;
        double face = at(e[0], e[1], e[2]) - at(-e[0], -e[1], -e[2]);
        double edge = 0.0;
        for (int b = 0; b < 3; ++b) {
            if (b == a) continue;
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                int pp[3] = {e[0], e[1], e[2]}, mm[3] = {-e[0], -e[1], -e[2]};
                pp[b] = sgn;
                mm[b] = sgn;
                edge += at(pp[0], pp[1], pp[2]) - at(mm[0], mm[1], mm[2]);
            }
        }
        out[a] = face / 6.0 + edge / 12.0;
    }
}

// Each block reduces NA_CELLS_PER_BLOCK consecutive cells; each thread a
// fixed contiguous run of NA_CELLS_PER_THREAD; the block tree is fixed, so
// the result does not depend on scheduling.
__global__ void k_noalloc_partial(NAGeom g, const double *phi, const double *rho, const double *u,
                                  const double *phi0, double *scratch)
{
    const long long N = (long long)g.nx * g.ny * g.nz;
    const long long first = blockIdx.x * NA_CELLS_PER_BLOCK + (long long)threadIdx.x * NA_CELLS_PER_THREAD;
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long o = first; o < first + NA_CELLS_PER_THREAD && o < N; ++o) {
        const int x = (int)(o % g.nx), y = (int)((o / g.nx) % g.ny), z = (int)(o / ((long long)g.nx * g.ny));
        double gp[3], g0[3];
        na_grad(g, phi, x, y, z, gp);
        na_grad(g, phi0, x, y, z, g0);
        const double ph = phi[o], p0 = phi0[o];
        double g2 = 0.0, g0g = 0.0, u2 = 0.0;
        for (int a = 0; a < g.dim; ++a) {
            g2 += gp[a] * gp[a];
            g0g += g0[a] * gp[a];
            u2 += u[a * N + o] * u[a * N + o];
        }
        const double s = g.sigma, D = g.D, ct = g.cos_t;
        acc[0] += ph;
        acc[1] += 3.0 * s / (4.0 * D) * (1.0 - ph) * (1.0 - ph) * (1.0 + ph) * (1.0 + ph) +
                  3.0 * D * s / 16.0 * g2 + 9.0 * s / (2.0 * D) * p0 * p0 * ph * ph +
                  3.0 * s * ct / D * p0 * ph * (ph * ph + p0 * p0 - 1.0) + 3.0 * D * s * ct / 8.0 * g0g;
        acc[2] += 0.5 * rho[o] * u2;
    }
    __shared__ double red[NA_THREADS][3];
    for (int c = 0; c < 3; ++c) red[threadIdx.x][c] = acc[c];
    __syncthreads();
    for (int st = NA_THREADS / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int c = 0; c < 3; ++c) red[threadIdx.x][c] += red[threadIdx.x + st][c];
        __syncthreads();
    }
    // every block overwrites its own triple: nothing carries over between calls
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) scratch[3 * blockIdx.x + c] = red[0][c];
}

__global__ void k_noalloc_final(int nblocks, double *scratch, double *out_dev)
{
    __shared__ double red[NA_THREADS][3];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += NA_THREADS)
        for (int c = 0; c < 3; ++c) acc[c] += scratch[3 * b + c];
    for (int c = 0; c < 3; ++c) red[threadIdx.x][c] = acc[c];
    __syncthreads();
    for (int st = NA_THREADS / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int c = 0; c < 3; ++c) red[threadIdx.x][c] += red[threadIdx.x + st][c];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double *fin = scratch + 3 * PF_NOALLOC_MAX_BLOCKS;
        for (int c = 0; c < 3; ++c) fin[c] = red[0][c];
        if (out_dev) {
            out_dev[0] = red[0][0];
            out_dev[1] = red[0][1];
            out_dev[2] = red[0][2];
            out_dev[3] = red[0][1] + red[0][2];
        }
    }
}

}  // namespace pf

using namespace pf;

// device address of the scratch array, resolved once per device and context:
// the address belongs to the context current at the lookup, so a new context
// on the device (after cudaDeviceReset, say) triggers a new lookup
static std::mutex g_na_mu;
static double *g_na_addr[64] = {};
static void *g_na_ctx[64] = {};

typedef int (*CtxGetCurrentFn)(void **);

// the calling thread's current driver context (nullptr if it cannot be read)
static void *current_context()
{
    static CtxGetCurrentFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrentFn)f;
        tried = true;
    }
    void *ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

static int na_fail(int code, const char *msg) { return set_error(code, msg); }

extern "C" int pf_diagnostics_noalloc(const pf_grid *g, const pf_params *p, const double *phi,
                                      const double *rho, const double *u, const double *phi0,
                                      double *out4, int where, void *stream)
{
    if (!g || !p || !phi || !rho || !u || !phi0 || !out4)
        return na_fail(PF_EINVAL, "pf_diagnostics_noalloc: NULL argument");
    if (g->dim != 2 && g->dim != 3) return na_fail(PF_EINVAL, "pf_diagnostics_noalloc: dim must be 2 or 3");
    if (where != PF_HOST && where != PF_DEVICE)
        return na_fail(PF_EINVAL, "pf_diagnostics_noalloc: where must be PF_HOST or PF_DEVICE");
    const int nz = g->dim == 2 ? 1 : g->nz;
    if (g->nx < 1 || g->ny < 1 || nz < 1) return na_fail(PF_EINVAL, "pf_diagnostics_noalloc: empty grid");
    for (int a = 0; a < g->dim; ++a)
        if (g->periodic[a] != 1 && !(a == 1 && g->periodic[a] == 0))
            return na_fail(PF_EINVAL, "pf_diagnostics_noalloc: boundaries must be periodic, except walls at the "
                                      "ends of y (periodic[1] = 0)");
    const long long N = (long long)g->nx * g->ny * nz;
    if (N > PF_NOALLOC_MAX_CELLS) {
        char buf[200];
        snprintf(buf, sizeof(buf),
                 "pf_diagnostics_noalloc: %lld cells exceed the static scratch maximum of %lld cells",
                 N, (long long)PF_NOALLOC_MAX_CELLS);
        return na_fail(PF_EINVAL, buf);
    }
    if (!(p->D > 0) || !(p->sigma >= 0)) return na_fail(PF_EINVAL, "pf_diagnostics_noalloc: bad sigma or D");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return na_fail(PF_ECUDA, "pf_diagnostics_noalloc: cudaGetDevice failed");
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        void *ctx = current_context();
        if (!g_na_addr[dev] || ctx != g_na_ctx[dev]) {
            // first call on this device (or in a new context): look up the
            // array's device address
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                return na_fail(PF_ECUDA, (std::string("pf_diagnostics_noalloc: cudaGetSymbolAddress failed: ") +
                                          cudaGetErrorString(e)).c_str());
            }
            g_na_addr[dev] = (double *)ptr;
            g_na_ctx[dev] = ctx;
        }
        scratch = g_na_addr[dev];
    }
    NAGeom geo;
    geo.dim = g->dim;
    geo.nx = g->nx;
    geo.ny = g->ny;
    geo.nz = nz;
    geo.wall_y = g->periodic[1] == 0 ? 1 : 0;
    geo.sigma = p->sigma;
    geo.D = p->D;
    geo.cos_t = std::cos(p->theta_deg * 3.14159265358979323846 / 180.0);
    cudaStream_t s = (cudaStream_t)stream;
    const int nblocks = (int)((N + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
    k_noalloc_partial<<<nblocks, NA_THREADS, 0, s>>>(geo, phi, rho, u, phi0, scratch);
    k_noalloc_final<<<1, NA_THREADS, 0, s>>>(nblocks, scratch, where == PF_DEVICE ? out4 : nullptr);
    count_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        return na_fail(PF_ECUDA, (std::string("pf_diagnostics_noalloc: launch failed: ") +
                                  cudaGetErrorString(e)).c_str());
    }
    if (where == PF_HOST) {
        double h[3];
        e = cudaMemcpyAsync(h, scratch + 3 * PF_NOALLOC_MAX_BLOCKS, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            return na_fail(PF_ECUDA, (std::string("pf_diagnostics_noalloc: copy failed: ") +
                                      cudaGetErrorString(e)).c_str());
        }
        out4[0] = h[0];
        out4[1] = h[1];
        out4[2] = h[2];
        out4[3] = h[1] + h[2];
    }
    return PF_OK;
}
