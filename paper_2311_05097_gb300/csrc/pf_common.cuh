// Device-side building blocks shared by the libpf kernels (sm_103a).
//
// Storage layout of one domain (all arrays structure-of-arrays, x fastest):
//   f[q][plane]     populations of both lattices: q in [0, Q1) order parameter,
//                   q in [Q1, Q1+Q2) flow; two buffers (pull streaming A -> B).
//   rest[plane]     PMIX only: rest population of the order-parameter lattice
//                   as a signed 64-bit fixed-point number (REST_FRAC_BITS).
//   aux[k][plane]   lagged fields of the previous step: u (dim), S (dim), phi;
//                   two buffers (neighbours read the old copy).
//   phi0[plane]     indicator of the fixed solids.
// plane = pitch * ny * nz rounded up to 64 elements; cell index
// (z*ny + y)*pitch + x.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace pf {

constexpr int REST_FRAC_BITS = 50;  // rest population = value * 2^-50

// MODE_STEP_PAIR: the 2D step with two cells per thread (FP32 arithmetic
// policies, fixed solids); MODE_STEP_STAGE: the same with the tile's inputs
// staged in shared memory by bulk copies
// MODE_STEP_STRIP: two cells per thread on strips marched in y, inputs staged
// by tensor copies; MODE_FILL_GHOSTS: the pass that refreshes the ghost columns
// the strip step reads
enum Mode {
    MODE_STEP = 0,
    MODE_MACROS = 1,
    MODE_STEP_PAIR = 2,
    MODE_STEP_STAGE = 3,
    MODE_STEP_STRIP = 4,
    MODE_FILL_GHOSTS = 5
};
// or'ed into a 2D mode: the launch holds a domain with walls or the Allen-Cahn
// order parameter (the single-cell kernel's instantiation that handles them)
constexpr int MODE_EXT = 16;
// or'ed into a 2D mode: the launch holds an Allen-Cahn domain (the
// two-cells-per-thread kernels' instantiation that handles it)
constexpr int MODE_CAC = 32;
// or'ed into MODE_STEP_PAIR: the launch runs the far tiles of a particle domain
// (the fixed solids' mu_phi0 grad phi0 term is on)
constexpr int MODE_MU0 = 64;
// or'ed into a 2D mode: the launch holds a domain with walls at the ends of y;
// only the single-cell kernel handles them, so the dispatchers of the other
// 2D kernels refuse a mode carrying this bit
constexpr int MODE_WALL = 128;
// or'ed into a 2D mode: every domain of the launch has unit relaxation rates
// for its non-conserved moments (DevParams::unit); kernels with a
// specialisation for that case take it
constexpr int MODE_UNIT = 256;

// Strip step (MODE_STEP_STRIP): strips of STRIP_SW columns; 2D rows carry
// STRIP_GHOST ghost columns (periodic images) on each side.  Tensor maps of
// one domain: per read parity the populations (the order parameter's staged
// planes, then the flow's), the rest population, the lagged u, S and phi
// (5 planes); then phi0.
constexpr int STRIP_SW = 64;
constexpr int STRIP_GHOST = 8;
constexpr int STRIP_MAPS_PER_PAR = 3;
constexpr int STRIP_MAPS = 2 * STRIP_MAPS_PER_PAR + 1;
enum StripMap { SM_F = 0, SM_REST = 1, SM_US = 2 };
constexpr int SM_PHI0 = 2 * STRIP_MAPS_PER_PAR;

// ---- precision policies ------------------------------------------------------------------
struct P64 {
    using real = double;
    using store = double;
    using aux = double;
    static constexpr bool MIX = false;
    static constexpr int id = 0;
};
struct P32 {
    using real = float;
    using store = float;
    using aux = float;
    static constexpr bool MIX = false;
    static constexpr int id = 1;
};
struct PMixH {
    using real = float;
    using store = __half;
    using aux = float;
    static constexpr bool MIX = true;
    static constexpr int id = 2;
};
struct PMixB {
    using real = float;
    using store = __nv_bfloat16;
    using aux = float;
    static constexpr bool MIX = true;
    static constexpr int id = 3;
};

// ---- per-domain constants (computed on the host in double) ----------------------------------
struct DevParams {
    double sigma, D, M, eta, rho1, rho2, mu1, mu2, d0;
    double s0, s1, s2, s3, s4, s1phi, cos_t, solid_eps;
    double Fb[3], g[3];
    double rep_xi, rep_eps;  // particle-particle repulsion (Sec. 4.5); eps <= 0: off
    double wall_circle[3];   // circular wall of the particle-wall repulsion; radius <= 0: none
    // derived
    double cs2, cs4, inv_cs2;
    double w0f;        // rest weight of the flow lattice
    double drho, rhom; // (rho1 - rho2)/2, (rho1 + rho2)/2
    double dmu, mum;   // (mu1 - mu2)/2, (mu1 + mu2)/2
    double c_dw;       // 3 sigma / D           (double well)
    double c_lap;      // 3 D sigma / 8         (gradient term)
    double c_pen;      // 9 sigma / D           (solid penalty)
    double c_wet;      // 3 sigma cos(theta)/D  (wetting)
    double c_wlap;     // 3 D sigma cos(theta)/8
    double Mdrho;      // M (rho1 - rho2)/2
    double K, Hc0, Hc1;  // H = K [Hc0 - Hc1 / s2a]
    double Pfac;       // cs2 / (1 - w0)
    double inv_1mcs2;  // 1 / (1 - cs2)
    double two_over_1md0;  // 2 / (1 - d0)
    double scale[2], inv_scale[2];  // PMIX population scales 2^k
    double cut;        // particle indicator is exactly 0 beyond R + cut
    int klog2[2];      // PMIX scale exponents k of 2^k
    int dim;
    int phase_model;   // 0: Cahn-Hilliard (Eq. 2); 1: conservative Allen-Cahn
    int unit;          // s_1phi, s1, s2, s3, s4 all 1 (s_1phi to 1e-12), Cahn-Hilliard lattice
};

struct ParticleDev {
    double x[3], u[3], w[3];
    double R, rho_p;
    double u_prev[3], w_prev[3];
    double F[3], T[3];
    double theta_deg;  // own contact angle, NaN for the handle's
    double ct;         // cos(theta_deg) when own
    int own;           // 1 if the particle has its own contact angle
    int prescribed;    // held motion: 1 all of u and w; 2, 4, 8 x, y, z translation; 16 rotation
};

// The constants the step kernels read, in the kernel's arithmetic type (so a
// float kernel never converts from double inside the cell loop).
template <class R>
struct KParams {
    R cs2, cs4, inv_cs2, w0f, drho, rhom, dmu, mum;
    R c_dw, c_lap, c_pen, c_wet, c_wlap, Mdrho;
    R K, Hc0, Hc1, Pfac, inv_1mcs2, two_over_1md0;
    R eta, s0, s1, s2, s3, s4, s1phi, solid_eps;
    R two_over_D;  // conservative Allen-Cahn: theta = (2/D)(1 - phi^2)
    R Fb[3];
    R scale[2], inv_scale[2];
};

template <class R>
inline KParams<R> make_kparams(const DevParams &d)
{
    KParams<R> k;
    k.cs2 = (R)d.cs2;
    k.cs4 = (R)d.cs4;
    k.inv_cs2 = (R)d.inv_cs2;
    k.w0f = (R)d.w0f;
    k.drho = (R)d.drho;
    k.rhom = (R)d.rhom;
    k.dmu = (R)d.dmu;
    k.mum = (R)d.mum;
    k.c_dw = (R)d.c_dw;
    k.c_lap = (R)d.c_lap;
    k.c_pen = (R)d.c_pen;
    k.c_wet = (R)d.c_wet;
    k.c_wlap = (R)d.c_wlap;
    k.Mdrho = (R)d.Mdrho;
    k.K = (R)d.K;
    k.Hc0 = (R)d.Hc0;
    k.Hc1 = (R)d.Hc1;
    k.Pfac = (R)d.Pfac;
    k.inv_1mcs2 = (R)d.inv_1mcs2;
    k.two_over_1md0 = (R)d.two_over_1md0;
    k.eta = (R)d.eta;
    k.s0 = (R)d.s0;
    k.s1 = (R)d.s1;
    k.s2 = (R)d.s2;
    k.s3 = (R)d.s3;
    k.s4 = (R)d.s4;
    k.s1phi = (R)d.s1phi;
    k.solid_eps = (R)d.solid_eps;
    k.two_over_D = (R)(2.0 / d.D);
    for (int a = 0; a < 3; ++a) k.Fb[a] = (R)d.Fb[a];
    for (int a = 0; a < 2; ++a) {
        k.scale[a] = (R)d.scale[a];
        k.inv_scale[a] = (R)d.inv_scale[a];
    }
    return k;
}

// One domain of a (possibly batched) launch.
struct DomainDev {
    int nx, ny, nz, pitch;
    int wall_y;      // 2D: walls at y = -1/2 and ny - 1/2 (halfway bounce-back), else periodic
    long long plane;
    void *f[2];      // population buffers
    void *rest[2];   // PMIX rest populations
    void *aux[2];    // lagged fields
    void *phi0;      // fixed indicator
    double *macro;   // MODE_MACROS output: phi, rho, u(dim), P, mu, phi0 (double)
    int tile_base;   // index of this domain's first tile in the partial-sum table
    int tiles_x, tiles_y, tiles_z;
    int zc;                // 3D: planes per z chunk of a tile (the last chunk may be shorter)
    DevParams p;
    KParams<float> kf;
    KParams<double> kd;
};

template <class R>
__device__ __forceinline__ const KParams<R> &kparams(const DomainDev &d);
template <>
__device__ __forceinline__ const KParams<float> &kparams<float>(const DomainDev &d) { return d.kf; }
template <>
__device__ __forceinline__ const KParams<double> &kparams<double>(const DomainDev &d) { return d.kd; }

// Arguments of the step / macro kernels (2D and 3D).
struct StepArgs {
    const DomainDev *doms;
    const int *tile_dom;   // domain of each tile
    const int2 *tile_xy;   // tile coordinates (x, y) in tiles
    int ntiles;
    int par;               // read buffer parity
    const ParticleDev *parts;
    int np;
    double *partials;      // [particle][6][tile]: F_f and T_f partial sums (Eq. 27)
    int *flags;            // [0]: non-finite value seen
    int wv;                // some particle has its own contact angle (W, V fields)
    int wait_polls;        // polls of one bounded device wait (staged kernel); 0: default
    const unsigned char *tile_sel;  // optional, per tile in device memory: run only the tiles ...
    int sel;                        // ... whose byte equals sel (else every tile)
    int *queue;            // strip step: work-queue counter (zeroed before the launch), or
                           // null: static round-robin over the items
    int mu0;               // single-cell step, wall instantiation, no particle terms: the
                           // tiles out of every particle's reach (split step) carry the
                           // fixed solids' mu_phi0 grad phi0 (Eq. 19)
    const int4 *items;              // strip kernel: work items (domain, x0, first row, end row)
    int nitems;
    const void *strip_maps;         // strip kernel: the tensor maps of every domain (128 bytes each)
};

// ---- helpers -----------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

template <>
__device__ __forceinline__ __half ldg<__half>(const __half *p)
{
    unsigned short v = __ldg(reinterpret_cast<const unsigned short *>(p));
    return __ushort_as_half(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 ldg<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    unsigned short v = __ldg(reinterpret_cast<const unsigned short *>(p));
    return __ushort_as_bfloat16(v);
}

// population store <-> compute conversion
template <class P>
struct Conv;
template <>
struct Conv<P64> {
    static __device__ __forceinline__ double ld(double v, double) { return v; }
    static __device__ __forceinline__ double st(double v, double) { return v; }
};
template <>
struct Conv<P32> {
    static __device__ __forceinline__ float ld(float v, float) { return v; }
    static __device__ __forceinline__ float st(float v, float) { return v; }
};
template <>
struct Conv<PMixH> {
    static __device__ __forceinline__ float ld(__half v, float inv_scale)
    {
        return __half2float(v) * inv_scale;
    }
    static __device__ __forceinline__ __half st(float v, float scale)
    {
        return __float2half_rn(v * scale);
    }
};
template <>
struct Conv<PMixB> {
    // Values whose fixed-point image would carry bits below 2^-REST_FRAC_BITS
    // are flushed to zero so every stored value is exact in fixed point.
    static __device__ __forceinline__ float ld(__nv_bfloat16 v, float inv_scale)
    {
        return __bfloat162float(v) * inv_scale;
    }
    static __device__ __forceinline__ __nv_bfloat16 st(float v, float scale)
    {
        __nv_bfloat16 b = __float2bfloat16_rn(v * scale);
        return b;
    }
};

// Exact integer image of a stored 16-bit order-parameter population, in units
// of 2^-24 of the stored (scaled) value.  Valid for |stored| < 8: then the
// image is below 2^27 and sums of 16 images fit in 32 bits.  FP16 values are
// all multiples of 2^-24; BF16 values are made so by bf16_flush at store time.
// Sets *bad for values outside the range (or inf / nan).
constexpr float FIX24_LIMIT = 8.0f;

__device__ __forceinline__ int fix24_of_float(float v, int *bad)
{
    if (!(fabsf(v) < FIX24_LIMIT)) {
        *bad = 1;
        return 0;
    }
    return __float2int_rn(v * 16777216.0f);
}

template <class S>
__device__ __forceinline__ float stored_to_float(S q);
template <>
__device__ __forceinline__ float stored_to_float<__half>(__half q) { return __half2float(q); }
template <>
__device__ __forceinline__ float stored_to_float<float>(float q) { return q; }
template <>
__device__ __forceinline__ float stored_to_float<__nv_bfloat16>(__nv_bfloat16 q)
{
    return __bfloat162float(q);
}

template <class S>
__device__ __forceinline__ int fix24(S q, int *bad)
{
    return fix24_of_float(stored_to_float<S>(q), bad);
}

// Image of a value that went through fix24_sat when it was stored.
template <class S>
__device__ __forceinline__ int fix24_stored(S q)
{
    return __float2int_rn(stored_to_float<S>(q) * 16777216.0f);
}

// Largest stored magnitude below FIX24_LIMIT.
template <class S>
__device__ __forceinline__ S fix24_max_stored();
template <>
__device__ __forceinline__ __half fix24_max_stored<__half>() { return __float2half_rz(7.99f); }
template <>
__device__ __forceinline__ __nv_bfloat16 fix24_max_stored<__nv_bfloat16>()
{
    return __float2bfloat16_rz(7.99f);
}

// Image of a value about to be stored; a value out of the image's range is
// saturated in place (so the stored value and its image still agree, and the
// cell's bookkeeping stays exact) and *sat is set.
template <class S>
__device__ __forceinline__ int fix24_sat(S &q, int *sat)
{
    float v = stored_to_float<S>(q);
    if (!(fabsf(v) < FIX24_LIMIT)) {
        *sat = 1;
        q = fix24_max_stored<S>();
        if (v < 0.0f) q = -q;
        v = stored_to_float<S>(q);
    }
    return __float2int_rn(v * 16777216.0f);
}

// Zero a BF16 whose value is not a multiple of 2^-24 (|v| < 2^-17; BF16
// carries 8 significant bits).
__device__ __forceinline__ __nv_bfloat16 bf16_flush(__nv_bfloat16 h)
{
    const unsigned int b = __bfloat16_as_ushort(h);
    const int e = (b >> 7) & 0xff;  // biased exponent, value ~ 2^(e - 127)
    if (e < 127 - 17) return __ushort_as_bfloat16(0);
    return h;
}

// Move an integer image in 2^-24 stored units (stored = value * 2^k) to the
// rest population's 2^-50 units: shift by 26 - k.
__device__ __forceinline__ long long fix24_to_rest(int v, int k)
{
    return (long long)v << (26 - k);
}

__device__ __forceinline__ float float_of_fixed(long long v)
{
    // split conversion: hi * 2^32 + lo, both exact in float arithmetic up to rounding of the sum
    int hi = (int)(v >> 32);
    unsigned int lo = (unsigned int)(v & 0xffffffffull);
    return __fmaf_rn((float)hi, 4294967296.0f, (float)lo) * (1.0f / 1125899906842624.0f);
}

__device__ __forceinline__ double double_of_fixed(long long v)
{
    return (double)v * (1.0 / 1125899906842624.0);  // 2^-50, exact for |v| < 2^53
}

__device__ __forceinline__ long long fixed_of_double(double v)
{
    return __double2ll_rn(v * 1125899906842624.0);
}

__device__ __forceinline__ int wrap_idx(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// d - n rint(d / n), the minimum image of a separation: without the FP64
// division (slow on this part) where it cannot shift, |d| <= n/2 (rint of a
// quotient in [-1/2, 1/2] is zero, so the result is the same)
__device__ __forceinline__ double min_image(double d, int n)
{
    return fabs(d) > 0.5 * n ? d - n * rint(d / n) : d;
}

// periodic index for v in [-n, 2n): no division
__device__ __forceinline__ int wrap_near(int v, int n)
{
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

// ---- asynchronous bulk copies into shared memory (mbarrier completion) ------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's earlier shared-memory accesses before later bulk copies
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// global -> shared copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Wait for the phase of parity `parity` to complete, at most max_iter polls
// (with back-off); false if it did not.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, int max_iter)
{
    for (int i = 0; i < max_iter; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (i > 16) __nanosleep(64);
    }
    return false;
}

}  // namespace pf
