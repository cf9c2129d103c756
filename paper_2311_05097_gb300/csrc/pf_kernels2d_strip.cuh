// 2D fused time step on strips marched in y, inputs staged by TMA (FP32
// arithmetic policies, fixed solids).
//
// The update is the one of the two-cells-per-thread step (Sec. 3.3, steps 2-6;
// Eqs. 9, 29-38, the physics shared through pair_physics).  What changes is
// how the inputs reach the cells:
//
//   - A work item is a strip of SW = 64 columns of one domain over a segment of
//     rows [ya, yb).  The CTA marches up the segment in bands of B rows: warp w
//     of the CTA owns row Y + w of the band, lane l the horizontally adjacent
//     cells x0 + 2l, x0 + 2l + 1.
//   - Every staged array row (both lattices' populations, the PMIX rest
//     population, the lagged u, S and phi, phi0) is copied into a ring of
//     R = 2B + 4 shared-memory rows by one 3D / 2D tensor copy per array and row
//     (cp.async.bulk.tensor, completing on an mbarrier).  The copies of band
//     k + 1 are issued early in band k, so DRAM latency hides behind most of a
//     band of work; the update reads nothing from global memory.
//   - phi (Eq. 31), mu_phi (Eq. 9) and w = S_x u_y - u_x S_y are computed once
//     per row and kept in rings of rows: the halo in y costs nothing but the
//     few rows that start a segment; the halo in x is 2 columns on each side.
//   - Periodic wrap in y is the row index taken modulo ny.  Periodic wrap in x
//     comes from ghost columns: every row of every array is followed by 8
//     columns holding copies of its first 8 cells and preceded (in the padding
//     of the previous row) by 8 columns holding copies of its last 8 cells.  The
//     step writes the ghosts of the cells it stores; a separate pass fills them
//     after anything else has written the state.
//
// Walls at the ends of y (the WALL instantiation; the box walls read as
// halfway bounce-back plus mirrored stencil rows): a staged row beyond a wall
// is a copy of its mirror image inside; phi of a row beyond a wall is that of
// its mirror row (w takes the sign change); a pull that would cross a wall
// reads the cell's own opposite population.
//
// Requirements (checked on the host): 2D, no free particles, every nx even
// and >= 8, pitch >= nx + 16.  Every wait on an
// mbarrier is bounded: a wait that runs out sets bit 2 of the flags word
// (PF_ETIMEOUT on the host), waits (bounded) for the copies still in flight
// and ends the CTA.
#pragma once

#include "pf_kernels2d_pair.cuh"
#include "pf_kernels2d_stage.cuh"

namespace pf {

constexpr int up128_c(int v) { return (v + 127) / 128 * 128; }

// Shared-memory layout of one staged row (byte offsets, each 128-aligned: the
// destination of a tensor copy) and of the working rings.
template <class P, int B>
struct StripLayout {
    using ST = typename P::store;
    static constexpr int SW = STRIP_SW;
    static constexpr int ES = (int)sizeof(ST);
    static constexpr int HS = 16 / ES;             // population halo: one 16-byte chunk (>= 3 cells)
    static constexpr int Q1 = P::MIX ? 8 : 9;      // order-parameter planes staged (movers, or all)
    static constexpr int I1 = P::MIX ? 1 : 0;      // first staged order-parameter plane
    static constexpr int W1 = SW + 2 * HS;         // population box: x0 - HS .. x0 + SW + HS
    static constexpr int WR = SW + 4;              // rest: x0 - 2 .. x0 + SW + 2
    static constexpr int WA = SW + 8;              // lagged u, S, phi and phi0: x0 - 4 .. x0 + SW + 4
    static constexpr int B1 = Q1 * W1 * ES, B2 = 9 * W1 * ES, BR = P::MIX ? WR * 8 : 0, BA = 5 * WA * 4,
                         B0 = WA * 4;
    // both lattices' staged planes arrive in one box: order parameter, then flow
    static constexpr int O1 = 0, O2 = O1 + B1, OR = up128_c(O2 + B2), OA = up128_c(OR + BR),
                         O0 = up128_c(OA + BA);
    static constexpr int ROW = up128_c(O0 + B0);   // bytes of one ring row
    static constexpr int ROW_TX = B1 + B2 + BR + BA + B0;  // bytes the copies of one row deliver
    static constexpr int NBOX = P::MIX ? 4 : 3;    // tensor copies per row
    static constexpr int R = 2 * B + 4;            // staged ring rows
    // working rings: phi (x0 - 2 .. x0 + SW + 2) and w (x0 - 1 .. x0 + SW + 1)
    // are written for the next band while the last warps still read them for
    // the current one (2B + 4 and 2B + 2 rows keep the two apart); mu
    // (x0 - 1 .. x0 + SW + 1) is written behind a barrier (B + 4 rows).  When
    // 2B + 4 is a power of two every ring gets that many rows and one slot,
    // row & (R - 1), serves them all (and the copies)
    static constexpr bool POW2 = (R & (R - 1)) == 0;
    static constexpr int RP = R, RWW = POW2 ? R : 2 * B + 2, RM = POW2 ? R : B + 4;
    static constexpr int FP = SW + 4, FM = SW + 2;
    static constexpr int OPHI = R * ROW, OW = OPHI + RP * FP * 4, OMU = OW + RWW * FM * 4;
    // unit rates with 16-bit storage: each cell's exact fixed-point phi
    // (rest + images of its pulled movers, from phase A) on the strip's columns
    static constexpr int ORA = up128_c(OMU + RM * FM * 4);
    static constexpr int BRA = P::MIX ? RP * SW * 8 : 0;
    static constexpr int OKP = up128_c(ORA + BRA);  // the domain's constants
    static constexpr int OIT = up128_c(OKP + (int)sizeof(KParams<float>));  // the item's pointers and scalars
    static constexpr int OBAR = up128_c(OIT + 64);
    static constexpr int BYTES = OBAR + 16;
    static_assert((W1 * ES) % 16 == 0 && (WR * 8) % 16 == 0 && (WA * 4) % 16 == 0,
                  "tensor boxes must be whole 16-byte chunks");
    static_assert(HS >= 3, "the order-parameter pulls of the phi frame reach 3 columns beyond the strip");
};

// rows of the band of the strip kernel (one warp per row): 6 for 16-bit
// storage (two CTAs of 6 warps per SM by shared memory, up to 168 registers
// per thread: measured faster than 8 rows at 128 registers, which spill), 4
// for FP32 storage (its staged rows are larger)
template <class P>
constexpr int strip_band()
{
    return P::MIX ? 6 : 4;
}

// ---- horizontal pairs ---------------------------------------------------------------------------
// Isotropic D2Q9 gradient and Laplacian (weights 4/9, 1/9, 1/36, cs^2 = 1/3) of
// two horizontally adjacent cells, from the 4-wide windows
// w[d] = a[row - 1 + d][left - 1 .. right + 1], d = 0, 1, 2: per row the pairs
// L = (w.x, w.y) of the left neighbours, M = (w.y, w.z) of the cells and
// R = (w.z, w.w) of the right neighbours.
__device__ __forceinline__ void grad9_hpair(const float4 (&w)[3], F2 &gx, F2 &gy)
{
    const F2 Ld = mk2(w[0].x, w[0].y), Md = mk2(w[0].y, w[0].z), Rd = mk2(w[0].z, w[0].w);
    const F2 Lc = mk2(w[1].x, w[1].y), Rc = mk2(w[1].z, w[1].w);
    const F2 Lu = mk2(w[2].x, w[2].y), Mu = mk2(w[2].y, w[2].z), Ru = mk2(w[2].z, w[2].w);
    const F2 third = mk2(1.0f / 3.0f), twelfth = mk2(1.0f / 12.0f);
    gx = fma2(third, Rc - Lc, twelfth * ((Rd - Ld) + (Ru - Lu)));
    gy = fma2(third, Mu - Md, twelfth * ((Ru + Lu) - (Rd + Ld)));
}

__device__ __forceinline__ F2 lap9_hpair(const float4 (&w)[3])
{
    const F2 Ld = mk2(w[0].x, w[0].y), Md = mk2(w[0].y, w[0].z), Rd = mk2(w[0].z, w[0].w);
    const F2 Lc = mk2(w[1].x, w[1].y), Mc = mk2(w[1].y, w[1].z), Rc = mk2(w[1].z, w[1].w);
    const F2 Lu = mk2(w[2].x, w[2].y), Mu = mk2(w[2].y, w[2].z), Ru = mk2(w[2].z, w[2].w);
    // 2/3 (side - 4 c) + 1/6 (diag - 4 c)
    const F2 side = (Rc + Lc) + (Md + Mu);
    const F2 diag = (Rd + Ld) + (Ru + Lu);
    return fma2(mk2(2.0f / 3.0f), side, fma2(mk2(1.0f / 6.0f), diag, mk2(-10.0f / 3.0f) * Mc));
}

// two 16-bit values as one 32-bit word (a in the low half: the lower address)
template <class S>
__device__ __forceinline__ uint32_t pack2(S a, S b);
template <>
__device__ __forceinline__ uint32_t pack2<__half>(__half a, __half b)
{
    return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}
template <>
__device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// two FP32 values rounded to the 16-bit storage type as one 32-bit word (one
// conversion instruction for both), and back
template <class S>
__device__ __forceinline__ uint32_t cvt_pair(F2 v);
template <>
__device__ __forceinline__ uint32_t cvt_pair<__half>(F2 v)
{
    const __half2 h = __float22half2_rn(v.v);
    return *reinterpret_cast<const uint32_t *>(&h);
}
template <>
__device__ __forceinline__ uint32_t cvt_pair<__nv_bfloat16>(F2 v)
{
    const __nv_bfloat162 h = __float22bfloat162_rn(v.v);
    return *reinterpret_cast<const uint32_t *>(&h);
}
template <class S>
__device__ __forceinline__ F2 uncvt_pair(uint32_t w);
template <>
__device__ __forceinline__ F2 uncvt_pair<__half>(uint32_t w)
{
    return {__half22float2(*reinterpret_cast<const __half2 *>(&w))};
}
template <>
__device__ __forceinline__ F2 uncvt_pair<__nv_bfloat16>(uint32_t w)
{
    return {__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w))};
}
// a 16-bit value from its bits
template <class S>
__device__ __forceinline__ S half_of(unsigned short b);
template <>
__device__ __forceinline__ __half half_of<__half>(unsigned short b) { return __ushort_as_half(b); }
template <>
__device__ __forceinline__ __nv_bfloat16 half_of<__nv_bfloat16>(unsigned short b) { return __ushort_as_bfloat16(b); }

// bit pattern of FIX24_LIMIT (8.0) in the 16-bit type: |v| < 8 exactly when
// the magnitude bits of v are below it (NaN and infinity are not)
template <class S>
constexpr uint32_t fix24_limit_bits();
template <>
constexpr uint32_t fix24_limit_bits<__half>() { return 0x4800u; }
template <>
constexpr uint32_t fix24_limit_bits<__nv_bfloat16>() { return 0x4100u; }

// the lane index, read afresh where it is used (volatile: the values derived
// from it are not hoisted out of the band loop, where they would hold
// registers through the update)
__device__ __forceinline__ int lane_now()
{
    int l;
    asm volatile("mov.u32 %0, %%laneid;" : "=r"(l));
    return l;
}

// ---- tensor copies ----------------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(unsigned dst, const void *map, int x, int y, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const void *map, int x, int y, int z, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4}], [%5];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Issue the copies of staged row r (segment coordinates, wrapped to the
// domain, or mirrored at its walls) into its ring row, completing on bar: box `box` of the row (lanes
// 0 .. NBOX - 1 of a warp each issue one).  The expected bytes were
// registered on bar before.  Tensor coordinates: x' = x + STRIP_GHOST (the
// maps start at the left ghost of row 0), y the wrapped row, plane 0 (each
// map starts at its first plane).
template <class P, int B>
__device__ __forceinline__ void strip_copy(const char *maps, int par, int x0, int ya, int ny, int r, int box,
                                           unsigned sbase, unsigned bar, bool wall)
{
    using L = StripLayout<P, B>;
    const char *pm = maps + (size_t)par * STRIP_MAPS_PER_PAR * 128;
    int y;
    if (wall) {  // walls at y = -1/2 and ny - 1/2: the mirror image (period 2 ny)
        const int p2 = 2 * ny;
        y = r % p2;
        if (y < 0) y += p2;
        if (y >= ny) y = p2 - 1 - y;
    } else {
        y = r % ny;
        if (y < 0) y += ny;
    }
    const int slot = L::POW2 ? (r & (L::R - 1)) : (r - ya + 3) % L::R;
    const unsigned row = sbase + (unsigned)(slot * L::ROW);
    const int g = STRIP_GHOST;
    if (box == 0)
        tma_load_3d(row + L::O1, pm + SM_F * 128, x0 - L::HS + g, y, 0, bar);
    else if (box == 1)
        tma_load_3d(row + L::OA, pm + SM_US * 128, x0 - 4 + g, y, 0, bar);
    else if (box == 2)
        tma_load_2d(row + L::O0, maps + SM_PHI0 * 128, x0 - 4 + g, y, bar);
    else
        tma_load_2d(row + L::OR, pm + SM_REST * 128, x0 - 2 + g, y, bar);
}

// what the update of a work item needs besides the constants (kept in shared
// memory: the band loop holds no registers for it)
struct StripItem {
    void *fd;            // populations written this step
    void *ad;            // lagged fields written this step
    void *rd;            // rest populations written this step
    int klog1;           // PMIX scale exponent of the order-parameter lattice
    int phase_model;
    int wall;            // walls at the ends of y
};

// ---- the kernel ---------------------------------------------------------------------------------
// Per band k (rows Y .. Y + B - 1 of the segment) the CTA runs
//   A: phi of rows Y + 2 .. Y + B + 1 and w of rows Y + 1 .. Y + B (every warp)
//   -- barrier 1 (also: every wait on band k's copies succeeded) --
//      every warp issues the copies of one row of band k + 1 (into the ring
//      rows band k - 1 used; all their readers are past barrier 1)
//   B: mu_phi of rows Y + 1 .. Y + B
//   -- barrier 2 --
//   C: the update of row Y + warp
// Phase A of band k + 1 overlaps the last warps' phase C of band k (the phi
// and w rings are long enough to keep the rows apart).
template <class P, int B, bool CAC, bool UNIT, bool WALL>
__global__ void __launch_bounds__(32 * B, 2) k_step2d_strip(StepArgs A)
{
    using ST = typename P::store;
    using AX = typename P::aux;
    using L = StripLayout<P, B>;
    static_assert(sizeof(typename P::real) == 4, "strip kernel: FP32 arithmetic policies only");
    static_assert(sizeof(AX) == 4, "strip kernel: FP32 auxiliary fields");
    static_assert(!(UNIT && CAC), "the Allen-Cahn lattice has s_1phi != 1");
    constexpr int NT = 32 * B, R = L::R, HS = L::HS;
    constexpr int FP = L::FP, FM = L::FM;
    extern __shared__ __align__(128) unsigned char smem[];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned sbase = smem_u32(smem);
    // the two band-group mbarriers (shared addresses), and their phases (bit b:
    // barrier b; kept in one register, not in an indexed array)
    auto bar = [&](int b) -> unsigned { return sbase + L::OBAR + 8u * (unsigned)b; };
    float *s_phi = reinterpret_cast<float *>(smem + L::OPHI);  // [RP][FP]
    float *s_w = reinterpret_cast<float *>(smem + L::OW);      // [RWW][FM]
    float *s_mu = reinterpret_cast<float *>(smem + L::OMU);    // [RM][FM]
    KParams<float> *s_kp = reinterpret_cast<KParams<float> *>(smem + L::OKP);
    StripItem *s_it = reinterpret_cast<StripItem *>(smem + L::OIT);
    if (tid == 0) {
        mbar_init(bar(0), 1);
        mbar_init(bar(1), 1);
    }
    unsigned phases = 0u;
    const int polls = A.wait_polls > 0 ? A.wait_polls : STAGE_WAIT_POLLS;
    const char *maps_all = reinterpret_cast<const char *>(A.strip_maps);

    // items: the first one by block index, the next ones from the work queue
    // (largest first: the short items fill the end of the step), or round-robin
    __shared__ int s_next;
    auto next_item = [&](int it) -> int {
        if (!A.queue) return it + gridDim.x;
        if (tid == 0) s_next = gridDim.x + atomicAdd(A.queue, 1);
        __syncthreads();
        return s_next;
    };
    for (int it = blockIdx.x; it < A.nitems; it = next_item(it)) {
        const int4 item = A.items[it];
        const DomainDev &Dm = A.doms[item.x];
        const int x0 = item.y, ya = item.z, yb = item.w;
        const int nx = Dm.nx, ny = Dm.ny, pitch = Dm.pitch;
        const int plane = (int)Dm.plane;
        const int K = (yb - ya + B - 1) / B;
        auto maps = [&]() { return maps_all + (size_t)item.x * STRIP_MAPS * 128; };

        // the previous item's readers of every ring are done; its copies landed
        fence_proxy_async_smem();
        __syncthreads();
        for (int j = tid; j < (int)(sizeof(KParams<float>) / 4); j += NT)
            reinterpret_cast<float *>(s_kp)[j] = reinterpret_cast<const float *>(&Dm.kf)[j];
        if (tid == NT - 1) {
            s_it->fd = Dm.f[A.par ^ 1];
            s_it->ad = Dm.aux[A.par ^ 1];
            s_it->rd = Dm.rest[A.par ^ 1];
            s_it->klog1 = Dm.p.klog2[0];
            s_it->phase_model = Dm.p.phase_model;
            s_it->wall = WALL ? Dm.wall_y : 0;
        }
        if (tid == 0) mbar_arrive_expect_tx(bar(0), (unsigned)((B + 6) * L::ROW_TX));
        __syncthreads();  // the constants and the item block are visible; the bytes are registered
        // band group 0: rows ya - 3 .. ya + B + 2, one box per lane, rows over the warps
        if (lane < L::NBOX)
            for (int rr = warp; rr < B + 6; rr += B)
                strip_copy<P, B>(maps(), A.par, x0, ya, ny, ya - 3 + rr, lane, sbase, bar(0), WALL && s_it->wall);

        // ring rows of segment row r: the rings hold row Y (the band's first row)
        // in slots bR, bP, bW, bM (advanced per band); r - Y stays within a ring
        int Y = ya, bR = 3, bP = 2, bW = 1, bM = 1;
        auto wrapn = [](int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); };
        constexpr int MSK = L::R - 1;
        auto slotR = [&](int r) { return L::POW2 ? (r & MSK) : wrapn(bR + (r - Y), R); };
        auto slotP = [&](int r) { return L::POW2 ? (r & MSK) : wrapn(bP + (r - Y), L::RP); };
        auto slotW = [&](int r) { return L::POW2 ? (r & MSK) : wrapn(bW + (r - Y), L::RWW); };
        auto slotM = [&](int r) { return L::POW2 ? (r & MSK) : wrapn(bM + (r - Y), L::RM); };
        auto srow_o = [&](int r) -> int { return slotR(r) * L::ROW; };
        auto srow = [&](int r) -> const unsigned char * { return smem + srow_o(r); };
        auto phir = [&](int r) -> float * { return s_phi + slotP(r) * FP; };
        auto wr = [&](int r) -> float * { return s_w + slotW(r) * FM; };
        auto mur = [&](int r) -> float * { return s_mu + slotM(r) * FM; };
        auto rar = [&](int r) -> long long * {  // (same slots as the phi ring)
            return reinterpret_cast<long long *>(smem + L::ORA) + slotP(r) * L::SW;
        };

        // one bounded wait on band group j (its phase advances on success)
        auto wait_group = [&](int j) -> bool {
            const int b = j & 1;
            const bool ok = mbar_wait_bounded(bar(b), (phases >> b) & 1u, polls);
            if (ok) phases ^= 1u << b;
            return ok;
        };
        // a wait ran out (known to every thread at a barrier): report; a thread
        // whose own wait failed gives band group j's copies a second bounded
        // wait to land; end the CTA
        auto give_up = [&](int j, bool my_ok) {
            if (tid == 0) atomicOr(A.flags, 4);
            if (!my_ok) mbar_wait_bounded(bar(j & 1), (phases >> (j & 1)) & 1u, STAGE_WAIT_POLLS);
        };

        // phi of pair m of row r (ring columns 2m, 2m + 1: x0 - 2 + 2m, + 1)
        auto phi_pair = [&](int r, int m) {
            // rs: the row whose phi this is (beyond a wall, the mirror image);
            // blo / bhi: its pulls across the lower / upper wall bounce back
            int rs = r;
            bool blo = false, bhi = false;
            if constexpr (WALL) {
                if (s_it->wall) {
                    if (r < -2 || r > ny + 1) {  // a row no update reads
                        *reinterpret_cast<float2 *>(phir(r) + 2 * m) = make_float2(0.0f, 0.0f);
                        return;
                    }
                    rs = r < 0 ? -1 - r : (r >= ny ? 2 * ny - 1 - r : r);
                    blo = rs == 0;
                    bhi = rs == ny - 1;
                }
            }
            const int c = 2 * m + HS - 2;  // staged column of the left cell
            // rows rs - 1, rs, rs + 1 (byte offsets of the left cell in the order-parameter box)
            const int ro[3] = {srow_o(rs - 1) + L::O1 + c * L::ES, srow_o(rs) + L::O1 + c * L::ES,
                               srow_o(rs + 1) + L::O1 + c * L::ES};
            // the left cell's stored value of population i pulled from plane
            // index k of the box (ko: that of the opposite population)
            auto src = [&](int i, int k, int ko) -> const ST * {
                if constexpr (WALL) {
                    if ((CY9[i] == 1 && blo) || (CY9[i] == -1 && bhi))
                        return reinterpret_cast<const ST *>(smem + ro[1]) + ko * L::W1;
                }
                return reinterpret_cast<const ST *>(smem + ro[1 - CY9[i]]) + k * L::W1 - CX9[i];
            };
            F2 phv;
            if constexpr (P::MIX && UNIT) {
                // the cells' exact fixed-point phi (rest + images of the pulled
                // movers), rounded once to FP32; kept for the update's bookkeeping
                const longlong2 rv = *reinterpret_cast<const longlong2 *>(smem + srow_o(rs) + L::OR + 16 * m);
                int sum[2] = {0, 0};
                const F2 s24 = mk2(16777216.0f);
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    const ST *q = src(i, i - 1, OPP9[i] - 1);
                    const F2 im = mk2(stored_to_float<ST>(q[0]), stored_to_float<ST>(q[1])) * s24;
                    sum[0] += __float2int_rn(im.v.x);
                    sum[1] += __float2int_rn(im.v.y);
                }
                const long long ra = rv.x + fix24_to_rest(sum[0], s_it->klog1);
                const long long rb = rv.y + fix24_to_rest(sum[1], s_it->klog1);
                phv = mk2(float_of_fixed(ra), float_of_fixed(rb));
                if (m >= 1 && m <= L::SW / 2)  // the strip's own columns
                    *reinterpret_cast<longlong2 *>(rar(r) + 2 * (m - 1)) = make_longlong2(ra, rb);
            } else if constexpr (P::MIX) {
                const longlong2 rv = *reinterpret_cast<const longlong2 *>(smem + srow_o(rs) + L::OR + 16 * m);
                F2 movers = mk2(0.0f);
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    const ST *q = src(i, i - 1, OPP9[i] - 1);
                    movers = movers + mk2(stored_to_float<ST>(q[0]), stored_to_float<ST>(q[1]));
                }
                phv = fma2(movers, mk2(s_kp->inv_scale[0]), mk2(float_of_fixed(rv.x), float_of_fixed(rv.y)));
            } else {
                F2 acc = mk2(0.0f);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const ST *q = src(i, i, OPP9[i]);
                    acc = acc + mk2(Conv<P>::ld(q[0], 1.0f), Conv<P>::ld(q[1], 1.0f));
                }
                phv = acc;
            }
            *reinterpret_cast<float2 *>(phir(r) + 2 * m) = phv.v;
        };
        // w of pair m of row r (ring columns 2m, 2m + 1: x0 - 1 + 2m, + 1)
        auto w_pair = [&](int r, int m) {
            const float *us = reinterpret_cast<const float *>(srow(r) + L::OA) + 2 * m + 3;  // left cell
            float wv[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float ux = us[e], uy = us[L::WA + e];
                const float Sx = us[2 * L::WA + e], Sy = us[3 * L::WA + e];
                wv[e] = Sx * uy - ux * Sy;
            }
            if constexpr (WALL) {
                if (s_it->wall && (r < 0 || r >= ny)) {  // odd under the wall mirror
                    wv[0] = -wv[0];
                    wv[1] = -wv[1];
                }
            }
            *reinterpret_cast<float2 *>(wr(r) + 2 * m) = make_float2(wv[0], wv[1]);
        };
        // phi of the four halo cells of row r (ring columns 0, 1, SW + 2, SW + 3:
        // x0 - 2, x0 - 1, x0 + SW, x0 + SW + 1) with unit rates and 16-bit storage,
        // one pulled population per lane: lane 8h + k takes population k + 1 of
        // halo cell h.  The images are integers, so their sum over the 8 lanes
        // of a cell (a shuffle tree) is the one phi_pair forms in sequence.
        // Every lane of the warp takes part (the shuffles).
        auto phi_halo = [&](int r) {
            const int ln = lane_now(), k = ln & 7, h = ln >> 3;
            const int idx = h < 2 ? h : h + L::SW;  // ring column; staged column HS - 2 + idx
            int rs = r;
            bool blo = false, bhi = false;
            if constexpr (WALL) {
                if (s_it->wall) {
                    if (r < -2 || r > ny + 1) {  // a row no update reads
                        if (k == 0) phir(r)[idx] = 0.0f;
                        return;
                    }
                    rs = r < 0 ? -1 - r : (r >= ny ? 2 * ny - 1 - r : r);
                    blo = rs == 0;
                    bhi = rs == ny - 1;
                }
            }
            // c_x + 1, c_y + 1 and the opposite population's plane of population
            // k + 1, four bits each (D2Q9 in the order of CX9 / CY9 / OPP9)
            const int cx = (int)((0x20021012u >> (4 * k)) & 15u) - 1;
            const int cy = (int)((0x00220121u >> (4 * k)) & 15u) - 1;
            const int ko = (int)((0x54761032u >> (4 * k)) & 15u);
            int row = rs - cy, pl = k, col = HS - 2 + idx - cx;
            if constexpr (WALL) {
                if ((cy == 1 && blo) || (cy == -1 && bhi)) {  // bounces back: own opposite population
                    row = rs;
                    pl = ko;
                    col = HS - 2 + idx;
                }
            }
            const ST q = reinterpret_cast<const ST *>(smem + srow_o(row) + L::O1)[pl * L::W1 + col];
            int im = __float2int_rn(__fmul_rn(stored_to_float<ST>(q), 16777216.0f));
            im += __shfl_xor_sync(0xffffffffu, im, 1);
            im += __shfl_xor_sync(0xffffffffu, im, 2);
            im += __shfl_xor_sync(0xffffffffu, im, 4);
            if (k == 0) {
                const long long rv = *reinterpret_cast<const long long *>(smem + srow_o(rs) + L::OR + 8 * idx);
                phir(r)[idx] = float_of_fixed(rv + fix24_to_rest(im, s_it->klog1));
            }
        };
        // phase A: phi (Eq. 31) of rows [rp, rp + np_) on columns x0 - 2 .. x0 + SW + 2
        // and w = S_x u_y - u_x S_y of the previous step on rows [rw, rw + nw),
        // columns x0 - 1 .. x0 + SW + 1; one list of pair items
        auto phase_a = [&](int rp, int np_, int rw, int nw) {
            constexpr int NPP = FP / 2, NPW = FM / 2;
            const int nphi = np_ * NPP, ntot = nphi + nw * NPW;
            for (int j = tid; j < ntot; j += NT) {
                if (j < nphi) {
                    const int rr = j / NPP;
                    phi_pair(rp + rr, j - rr * NPP);
                } else {
                    const int jj = j - nphi, rr = jj / NPW;
                    w_pair(rw + rr, jj - rr * NPW);
                }
            }
        };
        // phase A of a band with unit rates and 16-bit storage, one row per warp:
        // phi of row rp + warp, w of row rw + warp.  Each warp computes its own
        // row's halo (the x halo makes a phi row 34 pairs and a w row 33 pairs
        // wide; handed out as one list over the CTA, the items beyond 32 per row
        // all fell to warp 0, which then reached every barrier last)
        auto phase_a_rows = [&](int rp, int rw) {
            phi_pair(rp + warp, lane + 1);
            phi_halo(rp + warp);
            w_pair(rw + warp, lane);
            if (lane == 0) w_pair(rw + warp, L::SW / 2);
        };
        // mu_phi (Eq. 9) of pair m of row r (ring columns 2m, 2m + 1: x0 - 1 + 2m, + 1)
        auto mu_pair = [&](int r, int m) {
            const KParams<float> &kp = *s_kp;
            const F2 c_dw = mk2(kp.c_dw), c_lap = mk2(-kp.c_lap), c_pen = mk2(kp.c_pen), c_wet = mk2(kp.c_wet),
                     c_wlap = mk2(-kp.c_wlap), one = mk2(1.0f), three = mk2(3.0f);
            // 4-wide windows [left - 1, right + 1] of rows r - 1, r, r + 1
            float4 wp[3], w0[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float *pr = phir(r - 1 + d) + 2 * m;  // phi column of the left cell - 1
                const float2 a = *reinterpret_cast<const float2 *>(pr);
                const float2 b = *reinterpret_cast<const float2 *>(pr + 2);
                wp[d] = make_float4(a.x, a.y, b.x, b.y);
                const float *qr = reinterpret_cast<const float *>(srow(r - 1 + d) + L::O0) + 2 * m + 2;
                const float2 e = *reinterpret_cast<const float2 *>(qr);
                const float2 f = *reinterpret_cast<const float2 *>(qr + 2);
                w0[d] = make_float4(e.x, e.y, f.x, f.y);
            }
            const F2 ph = mk2(wp[1].y, wp[1].z), p0 = mk2(w0[1].y, w0[1].z);
            const F2 lp = lap9_hpair(wp), lp0 = lap9_hpair(w0);
            const F2 p02 = p0 * p0;
            F2 mu = c_dw * ph * ((ph - one) * (ph + one));
            mu = fma2(c_lap, lp, mu);
            mu = fma2(c_pen * p02, ph, mu);
            mu = fma2(c_wet * p0, fma2(three * ph, ph, p02) - one, mu);
            mu = fma2(c_wlap, lp0, mu);
            *reinterpret_cast<float2 *>(mur(r) + 2 * m) = mu.v;
        };
        // mu_phi of the last pair of row r (ring columns SW, SW + 1: x0 + SW - 1,
        // x0 + SW), spread over the warp: lane 16h + p loads stencil point p of
        // cell h (both fields), shuffles form the sums of lap9_hpair in its
        // order and lanes 0 and 16 finish each cell with the operations of
        // mu_pair in its order, one rounding each: the same bits as mu_pair.
        // Every lane of the warp takes part (the shuffles).
        auto mu_halo = [&](int r) {
            const KParams<float> &kp = *s_kp;
            const int ln = lane_now(), h = ln >> 4, p = min(ln & 15, 8), base = ln & 16;
            // stencil point p: Rc, Lc, Md, Mu, Rd, Ld, Ru, Lu, Mc (d: row r - 1, u: row r + 1),
            // dx + 1 and dy + 1 two bits each
            const int dx = (int)((0x12252u >> (2 * p)) & 3u) - 1;
            const int dy = (int)((0x1a085u >> (2 * p)) & 3u) - 1;
            const int j = L::SW + h;  // mu ring column of cell h (x0 - 1 + j)
            const float a = phir(r + dy)[j + 1 + dx];
            const float b = reinterpret_cast<const float *>(srow(r + dy) + L::O0)[j + 3 + dx];
            // (Rc + Lc), (Md + Mu), (Rd + Ld), (Ru + Lu), then side and diag
            const float a1 = __fadd_rn(a, __shfl_xor_sync(0xffffffffu, a, 1));
            const float b1 = __fadd_rn(b, __shfl_xor_sync(0xffffffffu, b, 1));
            const float a2 = __fadd_rn(a1, __shfl_xor_sync(0xffffffffu, a1, 2));
            const float b2 = __fadd_rn(b1, __shfl_xor_sync(0xffffffffu, b1, 2));
            const float adiag = __shfl_sync(0xffffffffu, a2, base + 4), bdiag = __shfl_sync(0xffffffffu, b2, base + 4);
            const float ph = __shfl_sync(0xffffffffu, a, base + 8), p0 = __shfl_sync(0xffffffffu, b, base + 8);
            if ((ln & 15) == 0) {
                const float lp = __fmaf_rn(2.0f / 3.0f, a2, __fmaf_rn(1.0f / 6.0f, adiag, __fmul_rn(-10.0f / 3.0f, ph)));
                const float lp0 = __fmaf_rn(2.0f / 3.0f, b2, __fmaf_rn(1.0f / 6.0f, bdiag, __fmul_rn(-10.0f / 3.0f, p0)));
                const float p02 = __fmul_rn(p0, p0);
                float mu = __fmul_rn(__fmul_rn(kp.c_dw, ph), __fmul_rn(__fsub_rn(ph, 1.0f), __fadd_rn(ph, 1.0f)));
                mu = __fmaf_rn(-kp.c_lap, lp, mu);
                mu = __fmaf_rn(__fmul_rn(kp.c_pen, p02), ph, mu);
                mu = __fmaf_rn(__fmul_rn(kp.c_wet, p0), __fsub_rn(__fmaf_rn(__fmul_rn(3.0f, ph), ph, p02), 1.0f), mu);
                mu = __fmaf_rn(-kp.c_wlap, lp0, mu);
                mur(r)[j] = mu;
            }
        };
        // phase B: mu_phi (Eq. 9), rows [rs, rs + nr), columns x0 - 1 .. x0 + SW + 1
        auto phase_b = [&](int rs, int nr) {
            constexpr int NP = FM / 2;
            for (int j = tid; j < nr * NP; j += NT) {
                const int rr = j / NP;
                mu_pair(rs + rr, j - rr * NP);
            }
        };
        // phase B of a band with unit rates and 16-bit storage, one row per warp
        // (row rs + warp, its halo pair spread over the warp; see phase_a_rows)
        auto phase_b_rows = [&](int rs) {
            mu_pair(rs + warp, lane);
            mu_halo(rs + warp);
        };

        // ---- prologue: rows ya - 3 .. ya + B + 2 staged; phi of ya - 2 .. ya + 1,
        // w and mu of ya - 1 .. ya
        {
            const bool ok = wait_group(0);
            if (ok) phase_a(ya - 2, 4, ya - 1, 2);
            if (__syncthreads_or(!ok)) {
                give_up(0, ok);
                return;
            }
            phase_b(ya - 1, 2);
        }

        for (int k = 0; k < K; ++k) {
            if (k > 0) {
                Y += B;
                if constexpr (!L::POW2) {
                    bR = wrapn(bR + B, R);
                    bP = wrapn(bP + B, L::RP);
                    bW = wrapn(bW + B, L::RWW);
                    bM = wrapn(bM + B, L::RM);
                }
            }
            const bool ok = k == 0 || wait_group(k);
            if constexpr (P::MIX && UNIT) {
                if (__all_sync(0xffffffffu, ok)) phase_a_rows(Y + 2, Y + 1);  // (warp-uniform: shuffles)
            } else {
                if (ok) phase_a(Y + 2, B, Y + 1, B);
            }
            fence_proxy_async_smem();  // this thread's reads of the ring precede the next copies
            if (tid == 0 && k + 1 < K) mbar_arrive_expect_tx(bar((k + 1) & 1), (unsigned)(B * L::ROW_TX));
            if (__syncthreads_or(!ok)) {  // barrier 1
                give_up(k, ok);  // (group k + 1 has its bytes registered but no copy issued)
                return;
            }
            // band group k + 1: rows Y + B + 3 .. Y + 2B + 2, row Y + B + 3 + warp, one box per lane
            if (k + 1 < K && lane < L::NBOX)
                strip_copy<P, B>(maps(), A.par, x0, ya, ny, Y + B + 3 + warp, lane, sbase, bar((k + 1) & 1),
                                 WALL && s_it->wall);
            if constexpr (P::MIX && UNIT)
                phase_b_rows(Y + 1);
            else
                phase_b(Y + 1, B);
            __syncthreads();  // barrier 2

            // ---- phase C: the thread's two cells, row Y + warp, columns x0 + 2 lane, + 1
            const int r = Y + warp, x = x0 + 2 * lane;
            if (r < yb && x < nx) {
                const KParams<float> &kp = *s_kp;
                // phi, mu, w: 4-wide windows of rows r - 1 .. r + 1
                float4 wph[3], wmu[3], ww[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float *pr = phir(r - 1 + d) + 2 * lane;  // columns x - 2 .. x + 3
                    const float2 a = *reinterpret_cast<const float2 *>(pr);
                    const float2 b = *reinterpret_cast<const float2 *>(pr + 2);
                    const float2 e = *reinterpret_cast<const float2 *>(pr + 4);
                    wph[d] = make_float4(a.y, b.x, b.y, e.x);
                    const float *mr = mur(r - 1 + d) + 2 * lane;  // columns x - 1 .. x + 2
                    const float2 ma = *reinterpret_cast<const float2 *>(mr);
                    const float2 mb = *reinterpret_cast<const float2 *>(mr + 2);
                    wmu[d] = make_float4(ma.x, ma.y, mb.x, mb.y);
                    const float *wrr = wr(r - 1 + d) + 2 * lane;
                    const float2 wa = *reinterpret_cast<const float2 *>(wrr);
                    const float2 wb = *reinterpret_cast<const float2 *>(wrr + 2);
                    ww[d] = make_float4(wa.x, wa.y, wb.x, wb.y);
                }
                const int id = r * pitch + x;
                const F2 phi = mk2(wph[1].y, wph[1].z);
                const F2 mu = mk2(wmu[1].y, wmu[1].z);
                F2 gpx, gpy, gmx, gmy, wgx, wgy;
                grad9_hpair(wph, gpx, gpy);
                grad9_hpair(wmu, gmx, gmy);
                grad9_hpair(ww, wgx, wgy);
                const unsigned char *own = srow(r);
                const float2 p0v = *reinterpret_cast<const float2 *>(own + L::O0 + 4 * (2 * lane + 4));
                const F2 phi0 = mk2(p0v.x, p0v.y);
                // previous step's u and S
                const float *us = reinterpret_cast<const float *>(own + L::OA) + 2 * lane + 4;
                const F2 upx = {*reinterpret_cast<const float2 *>(us)};
                const F2 upy = {*reinterpret_cast<const float2 *>(us + L::WA)};
                const F2 Spx = {*reinterpret_cast<const float2 *>(us + 2 * L::WA)};
                const F2 Spy = {*reinterpret_cast<const float2 *>(us + 3 * L::WA)};
                const F2 php = {*reinterpret_cast<const float2 *>(us + 4 * L::WA)};  // previous step's phi
                // pulled populations (Eq. 29): cell (x, r) reads f_i at (x - c_ix, r - c_iy)
                const int c = 2 * lane + HS;  // staged column of the left cell
                const int ro[3] = {srow_o(r - 1) + c * L::ES, srow_o(r) + c * L::ES, srow_o(r + 1) + c * L::ES};
                F2 f1[9], f2[9];
                long long racc[2] = {0, 0};
                // pulls across the lower / upper wall bounce back
                bool blo = false, bhi = false;
                if constexpr (WALL) {
                    if (s_it->wall) {
                        blo = r == 0;
                        bhi = r == ny - 1;
                    }
                }
                // the two cells' stored values of population i (32-bit load where c_x = 0;
                // a pull across a wall: the cells' own opposite population)
                auto pulled = [&](int box, int i, int q) -> F2 {
                    if constexpr (WALL) {
                        if ((CY9[i] == 1 && blo) || (CY9[i] == -1 && bhi)) {
                            const unsigned char *b = smem + ro[1] + box + (q + OPP9[i] - i) * L::W1 * L::ES;
                            if constexpr (P::MIX)
                                return uncvt_pair<ST>(*reinterpret_cast<const uint32_t *>(b));
                            else
                                return {*reinterpret_cast<const float2 *>(b)};
                        }
                    }
                    const unsigned char *b = smem + ro[1 - CY9[i]] + box + q * L::W1 * L::ES;
                    if constexpr (P::MIX) {
                        if (CX9[i] == 0) return uncvt_pair<ST>(*reinterpret_cast<const uint32_t *>(b));
                        const ST *e = reinterpret_cast<const ST *>(b) - CX9[i];
                        return mk2(stored_to_float<ST>(e[0]), stored_to_float<ST>(e[1]));
                    } else {
                        if (CX9[i] == 0) return {*reinterpret_cast<const float2 *>(b)};
                        const float *e = reinterpret_cast<const float *>(b) - CX9[i];
                        return mk2(e[0], e[1]);
                    }
                };
                if constexpr (UNIT) {
                    // the order-parameter collision does not read f1 (unit rates)
                    if constexpr (P::MIX) {
                        const longlong2 rv = *reinterpret_cast<const longlong2 *>(rar(r) + 2 * lane);
                        racc[0] = rv.x;
                        racc[1] = rv.y;
                    }
                } else if constexpr (P::MIX) {
                    const longlong2 rv = *reinterpret_cast<const longlong2 *>(own + L::OR + 8 * (2 * lane + 2));
                    int sold[2] = {0, 0};
                    const F2 s24 = mk2(16777216.0f);
#pragma unroll
                    for (int i = 1; i < 9; ++i) {
                        const F2 v = pulled(L::O1, i, i - 1);
                        const F2 im = v * s24;  // exact: the value in units of 2^-24
                        sold[0] += __float2int_rn(im.v.x);
                        sold[1] += __float2int_rn(im.v.y);
                        f1[i] = v * mk2(kp.inv_scale[0]);
                    }
                    f1[0] = mk2(float_of_fixed(rv.x), float_of_fixed(rv.y));
                    racc[0] = rv.x + fix24_to_rest(sold[0], s_it->klog1);
                    racc[1] = rv.y + fix24_to_rest(sold[1], s_it->klog1);
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i) f1[i] = pulled(L::O1, i, i);
                }
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const F2 v = pulled(L::O2, i, i);
                    f2[i] = P::MIX ? v * mk2(kp.inv_scale[1]) : v;
                }
                // ---- stores: the pair, and its ghost copies near the x ends (each
                // lattice as soon as it has collided), marked as streaming (evict
                // first: they are read again only in the next step, after the rest
                // of the state has passed through the L2, while the halo rows the
                // neighbouring strips and segments read soon should stay)
                ST *fd = reinterpret_cast<ST *>(s_it->fd);
                AX *ad = reinterpret_cast<AX *>(s_it->ad);
                const bool gl = x < STRIP_GHOST;        // copies right of the row's end
                const bool gr = x >= nx - STRIP_GHOST;  // copies left of its start
                int bad = 0;
                auto store1 = [&](const F2 (&g)[9]) {
                    if constexpr (P::MIX) {
                        const F2 sc1 = mk2(kp.scale[0]);
                        uint32_t w[9], amax = 0u;
#pragma unroll
                        for (int i = 1; i < 9; ++i) {
                            w[i] = cvt_pair<ST>(g[i] * sc1);
                            if constexpr (P::id == 3)
                                w[i] = pack2<ST>(bf16_flush(half_of<ST>((unsigned short)(w[i] & 0xffffu))),
                                                 bf16_flush(half_of<ST>((unsigned short)(w[i] >> 16))));
                            amax = __vmaxu2(amax, w[i] & 0x7fff7fffu);
                        }
                        constexpr uint32_t lim = fix24_limit_bits<ST>();
                        if ((amax & 0xffffu) >= lim || (amax >> 16) >= lim) {
                            // a value out of the images' range: saturate it in place (rare)
#pragma unroll
                            for (int i = 1; i < 9; ++i) {
                                ST qa = half_of<ST>((unsigned short)(w[i] & 0xffffu));
                                ST qb = half_of<ST>((unsigned short)(w[i] >> 16));
                                fix24_sat<ST>(qa, &bad);
                                fix24_sat<ST>(qb, &bad);
                                w[i] = pack2<ST>(qa, qb);
                            }
                        }
                        int snew[2] = {0, 0};
                        const F2 s24 = mk2(16777216.0f);
#pragma unroll
                        for (int i = 1; i < 9; ++i) {
                            const F2 im = uncvt_pair<ST>(w[i]) * s24;  // exact: the stored value in 2^-24 units
                            snew[0] += __float2int_rn(im.v.x);
                            snew[1] += __float2int_rn(im.v.y);
                        }
                        // exact: the sum of each cell's order-parameter populations is unchanged
                        const longlong2 rn = make_longlong2(racc[0] - fix24_to_rest(snew[0], s_it->klog1),
                                                           racc[1] - fix24_to_rest(snew[1], s_it->klog1));
                        long long *rd = reinterpret_cast<long long *>(s_it->rd);
                        auto put = [&](int at) {
#pragma unroll
                            for (int i = 1; i < 9; ++i) __stcs(reinterpret_cast<unsigned int *>(fd + i * plane + at), w[i]);
                            __stcs(reinterpret_cast<longlong2 *>(rd + at), rn);
                        };
                        put(id);
                        if (gl) put(id + nx);
                        if (gr) put(id - nx);
                    } else {
                        auto put = [&](int at) {
#pragma unroll
                            for (int i = 0; i < 9; ++i) __stcs(reinterpret_cast<float2 *>(fd + i * plane + at), g[i].v);
                        };
                        put(id);
                        if (gl) put(id + nx);
                        if (gr) put(id - nx);
                    }
                };
                F2 ux, uy, Sx, Sy;
                auto store2 = [&](const F2 (&g)[9], F2 vx, F2 vy, F2 sx, F2 sy) {
                    uint32_t w[9];
                    if constexpr (P::MIX) {
                        const F2 sc2 = mk2(kp.scale[1]);
#pragma unroll
                        for (int i = 0; i < 9; ++i) w[i] = cvt_pair<ST>(g[i] * sc2);
                    }
                    auto put = [&](int at, bool lagged_phi) {
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            if constexpr (P::MIX)
                                __stcs(reinterpret_cast<unsigned int *>(fd + (9 + i) * plane + at), w[i]);
                            else
                                __stcs(reinterpret_cast<float2 *>(fd + (9 + i) * plane + at), g[i].v);
                        }
                        __stcs(reinterpret_cast<float2 *>(ad + 0 * plane + at), vx.v);
                        __stcs(reinterpret_cast<float2 *>(ad + 1 * plane + at), vy.v);
                        __stcs(reinterpret_cast<float2 *>(ad + 2 * plane + at), sx.v);
                        __stcs(reinterpret_cast<float2 *>(ad + 3 * plane + at), sy.v);
                        if (lagged_phi) __stcs(reinterpret_cast<float2 *>(ad + 4 * plane + at), phi.v);
                    };
                    put(id, true);
                    if (gl) put(id + nx, false);
                    if (gr) put(id - nx, false);
                };
                pair_physics<CAC, false, decltype(store1), decltype(store2), UNIT>(
                    s_it->phase_model, kp, phi, phi0, mu, gpx, gpy, gmx, gmy, wgx, wgy, mk2(0.0f), mk2(0.0f),
                    mk2(0.0f), upx, upy, Spx, Spy, php, f1, f2, ux, uy, Sx, Sy, store1, store2);
                if (bad) atomicOr(A.flags, 2);
                // one test for the six values: a non-finite one makes the sum non-finite
                const F2 chk = (phi + ux) + uy;
                if (!isfinite(chk.v.x + chk.v.y)) atomicOr(A.flags, 1);
            }
        }
    }
}

// Refresh the ghost columns of the read buffers (parity par) of every domain:
// the 8 columns after each row's end copy its first 8 cells, the 8 before its
// start (the end of the previous row's padding; before row 0, the front pad of
// the array) copy its last 8 cells.  Populations, the PMIX rest population,
// the lagged u and S and phi0 (the lagged phi is used at the cell only).  Grid
// (any, number of domains); needs nx >= 8.
template <class P>
__global__ void k_fill_ghosts(const DomainDev *doms, int par)
{
    using ST = typename P::store;
    using AX = typename P::aux;
    const DomainDev &Dm = doms[blockIdx.y];
    const int nx = Dm.nx, ny = Dm.ny, pitch = Dm.pitch;
    const long long plane = Dm.plane;
    constexpr int NF = 18, NR = P::MIX ? 1 : 0, NA = 4;
    const long long work = (long long)(NF + NR + NA + 1) * ny * (2 * STRIP_GHOST);
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < work;
         w += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(w % (2 * STRIP_GHOST));
        const long long t = w / (2 * STRIP_GHOST);
        const int y = (int)(t % ny), q = (int)(t / ny);
        const int g = j < STRIP_GHOST ? j - STRIP_GHOST : nx + (j - STRIP_GHOST);  // ghost column
        const int src = g < 0 ? g + nx : g - nx;                                   // the cell it copies
        const long long o = (long long)y * pitch;
        if (q < NF) {
            ST *a = reinterpret_cast<ST *>(Dm.f[par]) + q * plane + o;
            a[g] = a[src];
        } else if (q < NF + NR) {
            long long *a = reinterpret_cast<long long *>(Dm.rest[par]) + o;
            a[g] = a[src];
        } else if (q < NF + NR + NA) {
            AX *a = reinterpret_cast<AX *>(Dm.aux[par]) + (q - NF - NR) * plane + o;
            a[g] = a[src];
        } else {
            AX *a = reinterpret_cast<AX *>(Dm.phi0) + o;
            a[g] = a[src];
        }
    }
}

}  // namespace pf
