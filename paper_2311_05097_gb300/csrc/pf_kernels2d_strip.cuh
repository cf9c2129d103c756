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
//     k + 1 are issued when band k starts, so DRAM latency hides behind a whole
//     band of work; nothing is read from global memory by the threads.
//   - phi (Eq. 31) is computed once per row and kept in a ring of B + 4 rows,
//     mu_phi (Eq. 9) and w = S_x u_y - u_x S_y once per row in rings of B + 4
//     rows: the halo in y costs nothing but the few rows that start a segment;
//     the halo in x is 2 columns on each side of the strip.
//   - Periodic wrap in y is the row index taken modulo ny.  Periodic wrap in x
//     comes from ghost columns: every row of every array is followed by 8
//     columns holding copies of its first 8 cells and preceded (in the padding
//     of the previous row) by 8 columns holding copies of its last 8 cells.  The
//     step writes the ghosts of the cells it stores; a separate pass fills them
//     after anything else has written the state.
//
// Requirements (checked on the host): 2D, no walls at the ends of y, no free
// particles, every nx even and >= 8, pitch >= nx + 16.  Every wait on an
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
    static constexpr int WA = SW + 8;              // u, S and phi0: x0 - 4 .. x0 + SW + 4
    static constexpr int WL = SW;                  // lagged phi: the strip
    static constexpr int B1 = Q1 * W1 * ES, B2 = 9 * W1 * ES, BR = P::MIX ? WR * 8 : 0, BA = 4 * WA * 4,
                         BL = WL * 4, B0 = WA * 4;
    static constexpr int O1 = 0, O2 = up128_c(O1 + B1), OR = up128_c(O2 + B2), OA = up128_c(OR + BR),
                         OL = up128_c(OA + BA), O0 = up128_c(OL + BL);
    static constexpr int ROW = up128_c(O0 + B0);   // bytes of one ring row
    static constexpr int ROW_TX = B1 + B2 + BR + BA + BL + B0;  // bytes the copies of one row deliver
    static constexpr int NBOX = P::MIX ? 6 : 5;    // tensor copies per row
    static constexpr int R = 2 * B + 4;            // staged ring rows
    static constexpr int RW = B + 4;               // working ring rows (phi, mu, w)
    static constexpr int FP = SW + 4;              // phi ring: x0 - 2 .. x0 + SW + 2
    static constexpr int FM = SW + 2;              // mu and w rings: x0 - 1 .. x0 + SW + 1
    static constexpr int OPHI = R * ROW, OMU = OPHI + RW * FP * 4, OW = OMU + RW * FM * 4;
    static constexpr int OBAR = up128_c(OW + RW * FM * 4);
    static constexpr int BYTES = OBAR + 16;
    static_assert((W1 * ES) % 16 == 0 && (WR * 8) % 16 == 0 && (WA * 4) % 16 == 0 && (WL * 4) % 16 == 0,
                  "tensor boxes must be whole 16-byte chunks");
    static_assert(HS >= 3, "the order-parameter pulls of the phi frame reach 3 columns beyond the strip");
};

// rows of the band of the strip kernel (one warp per row)
template <class P>
constexpr int strip_band()
{
    return P::MIX ? 8 : 4;
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

// Issue the copies of the nrows staged rows r0 .. r0 + nrows - 1 (segment rows,
// wrapped to the domain) into their ring rows, completing on bar.  Warp 0 only.
// Tensor coordinates: x' = x + STRIP_GHOST (the maps start at the left ghost
// of row 0), y the wrapped row, plane 0 (each map starts at its first plane).
template <class P, int B>
__device__ __forceinline__ void strip_issue(const char *maps, int par, int x0, int ya, int ny, int r0, int nrows,
                                            unsigned sbase, unsigned bar, int lane)
{
    using L = StripLayout<P, B>;
    if (lane == 0) mbar_arrive_expect_tx(bar, (unsigned)(nrows * L::ROW_TX));
    __syncwarp();
    const char *pm = maps + (size_t)par * STRIP_MAPS_PER_PAR * 128;
    for (int j = lane; j < nrows * L::NBOX; j += 32) {
        const int rr = j / L::NBOX, box = j - rr * L::NBOX;
        const int r = r0 + rr;
        int y = r % ny;
        if (y < 0) y += ny;
        const unsigned row = sbase + (unsigned)(((r - ya + 3) % L::R) * L::ROW);
        const int g = STRIP_GHOST;
        if (box == 0)
            tma_load_3d(row + L::O1, pm + SM_F1 * 128, x0 - L::HS + g, y, 0, bar);
        else if (box == 1)
            tma_load_3d(row + L::O2, pm + SM_F2 * 128, x0 - L::HS + g, y, 0, bar);
        else if (box == 2)
            tma_load_3d(row + L::OA, pm + SM_US * 128, x0 - 4 + g, y, 0, bar);
        else if (box == 3)
            tma_load_2d(row + L::OL, pm + SM_PHIL * 128, x0 + g, y, bar);
        else if (box == 4)
            tma_load_2d(row + L::O0, maps + SM_PHI0 * 128, x0 - 4 + g, y, bar);
        else
            tma_load_2d(row + L::OR, pm + SM_REST * 128, x0 - 2 + g, y, bar);
    }
}

// ---- the kernel ---------------------------------------------------------------------------------
template <class P, int B, bool CAC>
__global__ void __launch_bounds__(32 * B, 2) k_step2d_strip(StepArgs A)
{
    using ST = typename P::store;
    using AX = typename P::aux;
    using L = StripLayout<P, B>;
    static_assert(sizeof(typename P::real) == 4, "strip kernel: FP32 arithmetic policies only");
    static_assert(sizeof(AX) == 4, "strip kernel: FP32 auxiliary fields");
    constexpr int NT = 32 * B, R = L::R, RW = L::RW, HS = L::HS;
    constexpr int FP = L::FP, FM = L::FM;
    extern __shared__ __align__(128) unsigned char smem[];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned sbase = smem_u32(smem);
    const unsigned bar[2] = {sbase + L::OBAR, sbase + L::OBAR + 8};
    float *s_phi = reinterpret_cast<float *>(smem + L::OPHI);  // [RW][FP]
    float *s_mu = reinterpret_cast<float *>(smem + L::OMU);    // [RW][FM]
    float *s_w = reinterpret_cast<float *>(smem + L::OW);      // [RW][FM]
    if (tid == 0) {
        mbar_init(bar[0], 1);
        mbar_init(bar[1], 1);
    }
    __syncthreads();
    unsigned phase[2] = {0u, 0u};
    const int polls = A.wait_polls > 0 ? A.wait_polls : STAGE_WAIT_POLLS;
    const char *maps_all = reinterpret_cast<const char *>(A.strip_maps);

    for (int it = blockIdx.x; it < A.nitems; it += gridDim.x) {
        const int4 item = A.items[it];
        const DomainDev &Dm = A.doms[item.x];
        const int x0 = item.y, ya = item.z, yb = item.w;
        const int nx = Dm.nx, ny = Dm.ny, pitch = Dm.pitch;
        const int plane = (int)Dm.plane;
        const KParams<float> &kp = Dm.kf;
        const DevParams &p = Dm.p;
        const char *maps = maps_all + (size_t)item.x * STRIP_MAPS * 128;
        const int K = (yb - ya + B - 1) / B;
        const float isc1 = kp.inv_scale[0];

        // shared-memory views of staged row r (segment coordinates)
        auto srow = [&](int r) -> const unsigned char * { return smem + ((r - ya + 3) % R) * L::ROW; };
        auto f1s = [&](int r, int q, int c) -> ST {
            return reinterpret_cast<const ST *>(srow(r) + L::O1)[q * L::W1 + c];
        };
        auto f2s = [&](int r, int q, int c) -> ST {
            return reinterpret_cast<const ST *>(srow(r) + L::O2)[q * L::W1 + c];
        };
        auto phir = [&](int r) -> float * { return s_phi + ((r - ya + 2 + RW) % RW) * FP; };
        auto mur = [&](int r) -> float * { return s_mu + ((r - ya + 1 + RW) % RW) * FM; };
        auto wr = [&](int r) -> float * { return s_w + ((r - ya + 1 + RW) % RW) * FM; };

        // one bounded wait on band group j (its phase advances only on success);
        // every thread learns whether any thread's wait ran out
        auto wait_group = [&](int j) -> bool {
            const int b = j & 1;
            const bool ok = mbar_wait_bounded(bar[b], phase[b], polls);
            const bool all = !__syncthreads_or(!ok);
            if (all) phase[b] ^= 1u;
            return all;
        };
        // a wait ran out: report, give the copies still in flight (groups
        // [pending_from, pending_to)) a second bounded wait to land, end the CTA
        auto give_up = [&](int pending_from, int pending_to) {
            if (tid == 0) atomicOr(A.flags, 4);
            for (int j = pending_from; j < pending_to; ++j) {
                const int b = j & 1;
                mbar_wait_bounded(bar[b], phase[b], STAGE_WAIT_POLLS);  // (the default bound, not the injected one)
                phase[b] ^= 1u;
            }
        };

        // phi (Eq. 31) of rows [rs, rs + nr), columns x0 - 2 .. x0 + SW + 2 (pairs)
        auto phase_phi = [&](int rs, int nr) {
            constexpr int NP = FP / 2;
            for (int j = tid; j < nr * NP; j += NT) {
                const int rr = j / NP, m = j - rr * NP;
                const int r = rs + rr;
                const int c = 2 * m + HS - 2;  // staged column of the left cell
                F2 phv;
                if constexpr (P::MIX) {
                    const longlong2 rv = *reinterpret_cast<const longlong2 *>(srow(r) + L::OR + 16 * m);
                    F2 movers = mk2(0.0f);
#pragma unroll
                    for (int i = 1; i < 9; ++i)
                        movers = movers + mk2(stored_to_float<ST>(f1s(r - CY9[i], i - 1, c - CX9[i])),
                                              stored_to_float<ST>(f1s(r - CY9[i], i - 1, c + 1 - CX9[i])));
                    phv = fma2(movers, mk2(isc1), mk2(float_of_fixed(rv.x), float_of_fixed(rv.y)));
                } else {
                    F2 acc = mk2(0.0f);
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        acc = acc + mk2(Conv<P>::ld(f1s(r - CY9[i], i, c - CX9[i]), 1.0f),
                                        Conv<P>::ld(f1s(r - CY9[i], i, c + 1 - CX9[i]), 1.0f));
                    phv = acc;
                }
                *reinterpret_cast<float2 *>(phir(r) + 2 * m) = phv.v;
            }
        };
        // w = S_x u_y - u_x S_y of the previous step, rows [rs, rs + nr),
        // columns x0 - 1 .. x0 + SW + 1
        auto phase_w = [&](int rs, int nr) {
            constexpr int NP = FM / 2;
            for (int j = tid; j < nr * NP; j += NT) {
                const int rr = j / NP, m = j - rr * NP;
                const int r = rs + rr;
                const float *us = reinterpret_cast<const float *>(srow(r) + L::OA);
                const int c = 2 * m + 3;  // u, S column of the left cell (x - x0 + 4)
                float wv[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const float ux = us[0 * L::WA + c + e], uy = us[1 * L::WA + c + e];
                    const float Sx = us[2 * L::WA + c + e], Sy = us[3 * L::WA + c + e];
                    wv[e] = Sx * uy - ux * Sy;
                }
                *reinterpret_cast<float2 *>(wr(r) + 2 * m) = make_float2(wv[0], wv[1]);
            }
        };
        // mu_phi (Eq. 9), rows [rs, rs + nr), columns x0 - 1 .. x0 + SW + 1
        auto phase_mu = [&](int rs, int nr) {
            constexpr int NP = FM / 2;
            const F2 c_dw = mk2(kp.c_dw), c_lap = mk2(-kp.c_lap), c_pen = mk2(kp.c_pen), c_wet = mk2(kp.c_wet),
                     c_wlap = mk2(-kp.c_wlap), one = mk2(1.0f), three = mk2(3.0f);
            for (int j = tid; j < nr * NP; j += NT) {
                const int rr = j / NP, m = j - rr * NP;
                const int r = rs + rr;
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
            }
        };

        // ---- prologue: rows ya - 3 .. ya + B + 2 staged; phi of ya - 2 .. ya + 1,
        // w and mu of ya - 1 .. ya
        if (warp == 0) strip_issue<P, B>(maps, A.par, x0, ya, ny, ya - 3, B + 6, sbase, bar[0], lane);
        if (!wait_group(0)) {
            give_up(0, 1);
            return;
        }
        phase_phi(ya - 2, 4);
        phase_w(ya - 1, 2);
        __syncthreads();
        phase_mu(ya - 1, 2);
        fence_proxy_async_smem();  // this thread's reads of the ring precede the next copies
        __syncthreads();

        for (int k = 0; k < K; ++k) {
            const int Y = ya + k * B;
            if (k + 1 < K && warp == 0)
                strip_issue<P, B>(maps, A.par, x0, ya, ny, Y + B + 3, B, sbase, bar[(k + 1) & 1], lane);
            if (k >= 1 && !wait_group(k)) {
                give_up(k, k + 1 < K ? k + 2 : k + 1);
                return;
            }
            phase_phi(Y + 2, B);
            phase_w(Y + 1, B);
            __syncthreads();
            phase_mu(Y + 1, B);
            __syncthreads();

            // ---- the thread's two cells: row Y + warp, columns x0 + 2 lane, + 1
            const int r = Y + warp, x = x0 + 2 * lane;
            if (r < yb && x < nx) {
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
                const F2 phi = mk2(wph[1].y, wph[1].z);
                const F2 mu = mk2(wmu[1].y, wmu[1].z);
                F2 gpx, gpy, gmx, gmy, wgx, wgy;
                grad9_hpair(wph, gpx, gpy);
                grad9_hpair(wmu, gmx, gmy);
                grad9_hpair(ww, wgx, wgy);
                const unsigned char *own = srow(r);
                const float2 p0v = *reinterpret_cast<const float2 *>(own + L::O0 + 4 * (2 * lane + 4));
                const F2 phi0 = mk2(p0v.x, p0v.y);
                // previous step's u, S (own cells) and phi
                const float *us = reinterpret_cast<const float *>(own + L::OA) + 2 * lane + 4;
                const F2 upx = {*reinterpret_cast<const float2 *>(us)};
                const F2 upy = {*reinterpret_cast<const float2 *>(us + L::WA)};
                const F2 Spx = {*reinterpret_cast<const float2 *>(us + 2 * L::WA)};
                const F2 Spy = {*reinterpret_cast<const float2 *>(us + 3 * L::WA)};
                const F2 php = {*reinterpret_cast<const float2 *>(own + L::OL + 8 * lane)};
                // pulled populations (Eq. 29): cell (x, r) reads f_i at (x - c_ix, r - c_iy)
                const int c = 2 * lane + HS;  // staged column of the left cell
                F2 f1[9], f2[9];
                long long racc[2] = {0, 0};
                long long rest_own[2] = {0, 0};
                if constexpr (P::MIX) {
                    const longlong2 rv = *reinterpret_cast<const longlong2 *>(own + L::OR + 8 * (2 * lane + 2));
                    rest_own[0] = rv.x;
                    rest_own[1] = rv.y;
                    int sold[2] = {0, 0};
#pragma unroll
                    for (int i = 1; i < 9; ++i) {
                        const ST qa = f1s(r - CY9[i], i - 1, c - CX9[i]);
                        const ST qb = f1s(r - CY9[i], i - 1, c + 1 - CX9[i]);
                        sold[0] += fix24_stored<ST>(qa);
                        sold[1] += fix24_stored<ST>(qb);
                        f1[i] = mk2(stored_to_float<ST>(qa), stored_to_float<ST>(qb)) * mk2(isc1);
                    }
                    f1[0] = mk2(float_of_fixed(rest_own[0]), float_of_fixed(rest_own[1]));
                    racc[0] = rest_own[0] + fix24_to_rest(sold[0], p.klog2[0]);
                    racc[1] = rest_own[1] + fix24_to_rest(sold[1], p.klog2[0]);
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        f1[i] = mk2(Conv<P>::ld(f1s(r - CY9[i], i, c - CX9[i]), 1.0f),
                                    Conv<P>::ld(f1s(r - CY9[i], i, c + 1 - CX9[i]), 1.0f));
                }
                const float isc2 = kp.inv_scale[1];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const ST qa = f2s(r - CY9[i], i, c - CX9[i]), qb = f2s(r - CY9[i], i, c + 1 - CX9[i]);
                    if constexpr (P::MIX)
                        f2[i] = mk2(stored_to_float<ST>(qa), stored_to_float<ST>(qb)) * mk2(isc2);
                    else
                        f2[i] = mk2(Conv<P>::ld(qa, 1.0f), Conv<P>::ld(qb, 1.0f));
                }
                F2 ux, uy, Sx, Sy;
                pair_physics<CAC, false>(p, kp, phi, phi0, mu, gpx, gpy, gmx, gmy, wgx, wgy, mk2(0.0f), mk2(0.0f),
                                         mk2(0.0f), upx, upy, Spx, Spy, php, f1, f2, ux, uy, Sx, Sy);

                // ---- stores: the pair, and its ghost copies near the x ends
                ST *fd = reinterpret_cast<ST *>(Dm.f[A.par ^ 1]);
                AX *ad = reinterpret_cast<AX *>(Dm.aux[A.par ^ 1]);
                long long *rd = reinterpret_cast<long long *>(Dm.rest[A.par ^ 1]);
                const int id = r * pitch + x;
                const bool gl = x < STRIP_GHOST;        // copies right of the row's end
                const bool gr = x >= nx - STRIP_GHOST;  // copies left of its start
                int bad = 0;
                uint32_t q1w[9], q2w[9];
                long long rnew[2] = {0, 0};
                if constexpr (P::MIX) {
                    const float sc1 = kp.scale[0], sc2 = kp.scale[1];
                    int snew[2] = {0, 0};
#pragma unroll
                    for (int i = 1; i < 9; ++i) {
                        ST qa = Conv<P>::st(f1[i].v.x, sc1), qb = Conv<P>::st(f1[i].v.y, sc1);
                        if constexpr (P::id == 3) {
                            qa = bf16_flush(qa);
                            qb = bf16_flush(qb);
                        }
                        snew[0] += fix24_sat<ST>(qa, &bad);
                        snew[1] += fix24_sat<ST>(qb, &bad);
                        q1w[i] = pack2<ST>(qa, qb);
                    }
                    // exact: the sum of each cell's order-parameter populations is unchanged
                    rnew[0] = racc[0] - fix24_to_rest(snew[0], p.klog2[0]);
                    rnew[1] = racc[1] - fix24_to_rest(snew[1], p.klog2[0]);
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        q2w[i] = pack2<ST>(Conv<P>::st(f2[i].v.x, sc2), Conv<P>::st(f2[i].v.y, sc2));
                }
                auto store_all = [&](int at, bool lagged_phi) {
                    if constexpr (P::MIX) {
#pragma unroll
                        for (int i = 1; i < 9; ++i) *reinterpret_cast<uint32_t *>(fd + i * plane + at) = q1w[i];
#pragma unroll
                        for (int i = 0; i < 9; ++i)
                            *reinterpret_cast<uint32_t *>(fd + (9 + i) * plane + at) = q2w[i];
                        *reinterpret_cast<longlong2 *>(rd + at) = make_longlong2(rnew[0], rnew[1]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            *reinterpret_cast<float2 *>(fd + i * plane + at) = f1[i].v;
                            *reinterpret_cast<float2 *>(fd + (9 + i) * plane + at) = f2[i].v;
                        }
                    }
                    *reinterpret_cast<float2 *>(ad + 0 * plane + at) = ux.v;
                    *reinterpret_cast<float2 *>(ad + 1 * plane + at) = uy.v;
                    *reinterpret_cast<float2 *>(ad + 2 * plane + at) = Sx.v;
                    *reinterpret_cast<float2 *>(ad + 3 * plane + at) = Sy.v;
                    if (lagged_phi) *reinterpret_cast<float2 *>(ad + 4 * plane + at) = phi.v;
                };
                store_all(id, true);
                if (gl) store_all(id + nx, false);
                if (gr) store_all(id - nx, false);
                if (bad) atomicOr(A.flags, 2);
                if (!isfinite(phi.v.x) || !isfinite(phi.v.y) || !isfinite(ux.v.x) || !isfinite(ux.v.y) ||
                    !isfinite(uy.v.x) || !isfinite(uy.v.y))
                    atomicOr(A.flags, 1);
            }
            fence_proxy_async_smem();  // this thread's reads of the ring precede the next copies
            __syncthreads();
        }
    }
}

// Refresh the ghost columns of the read buffers (parity par) of every domain:
// the 8 columns after each row's end copy its first 8 cells, the 8 before its
// start (the end of the previous row's padding; before row 0, the front pad of
// the array) copy its last 8 cells.  Populations, the PMIX rest population,
// the lagged u and S and phi0; the lagged phi is read at the cell only.  Grid
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
