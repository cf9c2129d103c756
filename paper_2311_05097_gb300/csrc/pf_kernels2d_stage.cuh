// 2D fused time step, two cells per thread, with the tile's inputs staged in
// shared memory by asynchronous bulk copies (FP32 arithmetic policies).
//
// The update is the one of k_step2d_pair (Sec. 3.3, steps 2-6 and 7).  What
// changes is where stage A reads from: before a CTA computes tile t it has
// already copied, for tile t, every row segment the tile needs -- the
// order-parameter movers on the tile + 3 frame, its rest population and phi0
// on the tile + 2 frame, the flow populations and the lagged u, S on the
// tile + 1 frame and the lagged phi on the tile -- into shared memory with
// cp.async.bulk (one copy per row segment, two where the segment crosses the
// periodic edge), completing on an mbarrier.  The copies for the CTA's next
// tile are issued as soon as stage A of the current tile has read the
// buffer, so DRAM latency overlaps stages B and C instead of stalling stage A.
//
// Requirements (checked on the host): nx a multiple of 16 / sizeof(store)
// and of 4 (so every segment and every split starts on a 16-byte boundary),
// fixed solids only.  Every wait on the mbarrier is bounded; a wait that runs
// out sets bit 2 of the flags word (PF_ETIMEOUT on the host), drains with a
// second bounded wait and ends the CTA.
#pragma once

#include "pf_kernels2d_pair.cuh"

namespace pf {

constexpr int round_up_c(int v, int m) { return (v + m - 1) / m * m; }

// Shared-memory staging layout of one tile (byte offsets, each 16-aligned).
template <class P, int TX, int TY>
struct StageLayout {
    using ST = typename P::store;
    using AX = typename P::aux;
    static constexpr int ES = (int)sizeof(ST), EA = (int)sizeof(AX);
    static constexpr int Q1 = P::MIX ? 8 : 9;  // order-parameter planes staged (movers, or all)
    static constexpr int I1 = P::MIX ? 1 : 0;  // first staged plane
    // order-parameter populations: rows y0-3 .. y0+TY+2, halo 3 in x
    static constexpr int M1 = round_up_c(3, 16 / ES), W1 = TX + 2 * M1, R1 = TY + 6;
    // flow populations: rows y0-1 .. y0+TY, halo 1
    static constexpr int M2 = round_up_c(1, 16 / ES), W2 = TX + 2 * M2, R2 = TY + 2;
    // rest population (int64): rows y0-2 .. y0+TY+1, halo 2
    static constexpr int M3 = 2, W3 = TX + 2 * M3, R3 = P::MIX ? TY + 4 : 0;
    // lagged u, S (4 planes): rows y0-1 .. y0+TY, halo 1
    static constexpr int MA = round_up_c(1, 16 / EA), WA = TX + 2 * MA, RA = TY + 2;
    // lagged phi: the tile
    static constexpr int WL = TX, RL = TY;
    // phi0: rows y0-2 .. y0+TY+1, halo 2
    static constexpr int M0 = round_up_c(2, 16 / EA), W0 = TX + 2 * M0, R0 = TY + 4;

    static constexpr int B1 = Q1 * R1 * W1 * ES;
    static constexpr int B2 = 9 * R2 * W2 * ES;
    static constexpr int B3 = R3 * W3 * 8;
    static constexpr int BA = 4 * RA * WA * EA;
    static constexpr int BL = RL * WL * EA;
    static constexpr int B0 = R0 * W0 * EA;
    static constexpr int O1 = 0, O2 = O1 + B1, O3 = O2 + B2, OA = O3 + B3, OL = OA + BA, O0 = OL + BL;
    static constexpr int BYTES = O0 + B0;
    // work units: one row segment of one plane
    static constexpr int U1 = Q1 * R1, U2 = 9 * R2, U3 = R3, UA = 4 * RA, UL = RL, U0 = R0;
    static constexpr int UNITS = U1 + U2 + U3 + UA + UL + U0;
    static_assert((W1 * ES) % 16 == 0 && (W2 * ES) % 16 == 0 && (W3 * 8) % 16 == 0 && (WA * EA) % 16 == 0 &&
                      (WL * EA) % 16 == 0 && (W0 * EA) % 16 == 0,
                  "row segments must be whole 16-byte chunks");
};

// Copy the row segment [xs, xs + w) of one row into shared memory at dst,
// wrapping periodically in x (split where it crosses the edge).
template <class T>
__device__ __forceinline__ void stage_row(unsigned dst, const T *row, int xs, int w, int nx, unsigned bar)
{
    if (xs >= 0 && xs + w <= nx) {  // interior: one copy
        bulk_g2s(dst, row + xs, (unsigned)(w * (int)sizeof(T)), bar);
        return;
    }
    int cur = xs;
    const int end = xs + w;
    while (cur < end) {
        int sx = cur % nx;
        if (sx < 0) sx += nx;
        const int len = min(end - cur, nx - sx);
        bulk_g2s(dst + (unsigned)((cur - xs) * (int)sizeof(T)), row + sx, (unsigned)(len * (int)sizeof(T)), bar);
        cur += len;
    }
}

__device__ __forceinline__ int wrap_row(int y, int ny)
{
    y %= ny;
    return y < 0 ? y + ny : y;
}

// Row offsets (wrapped row * pitch) of tile t's rows y0 - 3 .. y0 + TY + 2,
// written into rows[0 .. TY + 6) by the first threads.
template <int TY, int NT>
__device__ __forceinline__ void stage_rows(const StepArgs &A, int t, int *rows, int tid)
{
    if (tid < TY + 6) {
        const DomainDev &Dm = A.doms[A.tile_dom[t]];
        const int y0 = A.tile_xy[t].y * TY;
        rows[tid] = wrap_row(y0 - 3 + tid, Dm.ny) * Dm.pitch;
    }
}

// Issue every copy of tile t into the staging buffer (all threads; thread 0
// registers the byte count on the mbarrier first).  rows: stage_rows of t.
template <class P, int TX, int TY, int NT>
__device__ __forceinline__ void stage_issue(const StepArgs &A, int t, const int *rows, unsigned sbase, unsigned bar,
                                            int tid)
{
    using L = StageLayout<P, TX, TY>;
    using ST = typename P::store;
    using AX = typename P::aux;
    const DomainDev &Dm = A.doms[A.tile_dom[t]];
    const int x0 = A.tile_xy[t].x * TX;
    const int nx = Dm.nx;
    const long long plane = Dm.plane;
    const ST *fs = reinterpret_cast<const ST *>(Dm.f[A.par]);
    const AX *as = reinterpret_cast<const AX *>(Dm.aux[A.par]);
    const long long *rs = reinterpret_cast<const long long *>(Dm.rest[A.par]);
    const AX *ph0 = reinterpret_cast<const AX *>(Dm.phi0);
    fence_proxy_async_smem();  // this thread's reads of the buffer precede the copies
    if (tid == 0) mbar_arrive_expect_tx(bar, (unsigned)L::BYTES);
#pragma unroll 1
    for (int u = tid; u < L::UNITS; u += NT) {
        // rows[k] holds tile row k - 3
        if (u < L::U1) {
            const int q = u / L::R1, r = u - q * L::R1;
            stage_row<ST>(sbase + L::O1 + (unsigned)(u * L::W1 * L::ES), fs + (q + L::I1) * plane + rows[r],
                          x0 - L::M1, L::W1, nx, bar);
        } else if (u < L::U1 + L::U2) {
            const int v = u - L::U1, q = v / L::R2, r = v - q * L::R2;
            stage_row<ST>(sbase + L::O2 + (unsigned)(v * L::W2 * L::ES), fs + (9 + q) * plane + rows[r + 2],
                          x0 - L::M2, L::W2, nx, bar);
        } else if (u < L::U1 + L::U2 + L::U3) {
            const int r = u - L::U1 - L::U2;
            stage_row<long long>(sbase + L::O3 + (unsigned)(r * L::W3 * 8), rs + rows[r + 1], x0 - L::M3, L::W3, nx,
                                 bar);
        } else if (u < L::U1 + L::U2 + L::U3 + L::UA) {
            const int v = u - L::U1 - L::U2 - L::U3, q = v / L::RA, r = v - q * L::RA;
            stage_row<AX>(sbase + L::OA + (unsigned)(v * L::WA * L::EA), as + q * plane + rows[r + 2], x0 - L::MA,
                          L::WA, nx, bar);
        } else if (u < L::U1 + L::U2 + L::U3 + L::UA + L::UL) {
            const int r = u - L::U1 - L::U2 - L::U3 - L::UA;
            stage_row<AX>(sbase + L::OL + (unsigned)(r * L::WL * L::EA), as + 4 * plane + rows[r + 3], x0, L::WL, nx,
                          bar);
        } else {
            const int r = u - L::U1 - L::U2 - L::U3 - L::UA - L::UL;
            stage_row<AX>(sbase + L::O0 + (unsigned)(r * L::W0 * L::EA), ph0 + rows[r + 1], x0 - L::M0, L::W0, nx,
                          bar);
        }
    }
}

// polls of one bounded mbarrier wait (with 64 ns back-off: well under a second)
constexpr int STAGE_WAIT_POLLS = 1 << 22;

template <class P, int TX, int TYP>
__global__ void __launch_bounds__(TX *TYP, (step2d_pair_min_blocks<TX, TYP>())) k_step2d_stage(StepArgs A)
{
    using ST = typename P::store;
    using AX = typename P::aux;
    static_assert(sizeof(typename P::real) == 4, "staged pair kernel: FP32 arithmetic policies only");
    constexpr int NT = TX * TYP;
    constexpr int TY = 2 * TYP;
    constexpr int FX = TX + 4, FY = TY + 4;
    constexpr int WX = TX + 2, WY = TY + 2;
    using L = StageLayout<P, TX, TY>;
    __shared__ float s_phi[FY][FX];
    __shared__ float s_p0[FY][FX];
    __shared__ float s_mu[WY][WX];
    __shared__ float s_w[WY][WX];
    __shared__ alignas(8) unsigned long long s_bar;
    __shared__ int s_rows[TY + 6];  // row offsets of the tile whose copies are issued next
    extern __shared__ __align__(128) unsigned char s_stage[];

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly0 = 2 * (tid / TX);
    const unsigned bar = smem_u32(&s_bar), sbase = smem_u32(s_stage);
    const ST *S1 = reinterpret_cast<const ST *>(s_stage + L::O1);
    const ST *S2 = reinterpret_cast<const ST *>(s_stage + L::O2);
    const long long *S3 = reinterpret_cast<const long long *>(s_stage + L::O3);
    const AX *SA = reinterpret_cast<const AX *>(s_stage + L::OA);
    const AX *SL = reinterpret_cast<const AX *>(s_stage + L::OL);
    const AX *S0 = reinterpret_cast<const AX *>(s_stage + L::O0);
    auto f1s = [&](int q, int r, int c) -> ST { return S1[(q * L::R1 + r) * L::W1 + c]; };
    auto f2s = [&](int q, int r, int c) -> ST { return S2[(q * L::R2 + r) * L::W2 + c]; };

    if (tid == 0) mbar_init(bar, 1);
    if ((int)blockIdx.x < A.ntiles) stage_rows<TY, NT>(A, blockIdx.x, s_rows, tid);
    __syncthreads();
    if ((int)blockIdx.x < A.ntiles) stage_issue<P, TX, TY, NT>(A, blockIdx.x, s_rows, sbase, bar, tid);
    unsigned phase = 0;
    const int polls = A.wait_polls > 0 ? A.wait_polls : STAGE_WAIT_POLLS;

    for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
        const bool ok = mbar_wait_bounded(bar, phase, polls);
        phase ^= 1u;
        // all threads agree; the barrier also ends the previous tile's
        // shared-memory reads before stage A rewrites the tiles
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(A.flags, 4);
            mbar_wait_bounded(bar, phase ^ 1u, STAGE_WAIT_POLLS);  // let copies in flight land
            return;
        }
        const DomainDev &Dm = A.doms[A.tile_dom[t]];
        const int2 txy = A.tile_xy[t];
        const int nx = Dm.nx, ny = Dm.ny;
        const int plane = (int)Dm.plane;
        const int x0 = txy.x * TX, y0 = txy.y * TY;
        const DevParams &p = Dm.p;
        const KParams<float> &kp = Dm.kf;
        ST *fd = reinterpret_cast<ST *>(Dm.f[A.par ^ 1]);
        AX *ad = reinterpret_cast<AX *>(Dm.aux[A.par ^ 1]);
        long long *rd = reinterpret_cast<long long *>(Dm.rest[A.par ^ 1]);
        const float isc1 = kp.inv_scale[0];

        // phi at frame cell (fx, fy) of the tile + 2 frame (Eq. 31)
        auto phi_frame = [&](int fx, int fy) -> float {
            float acc;
            if constexpr (P::MIX) {
                acc = float_of_fixed(S3[fy * L::W3 + fx]);
                float movers = 0.0f;
#pragma unroll
                for (int i = 1; i < 9; ++i)
                    movers += stored_to_float<ST>(f1s(i - 1, fy + 1 - CY9[i], fx - 2 + L::M1 - CX9[i]));
                acc += movers * isc1;
            } else {
                acc = 0.0f;
#pragma unroll
                for (int i = 0; i < 9; ++i) acc += Conv<P>::ld(f1s(i, fy + 1 - CY9[i], fx - 2 + L::M1 - CX9[i]), 1.0f);
            }
            return acc;
        };

        // ---------------- stage A (from the staging buffer) ----------------
        int id[2];
        ST f2raw[2][9];
        AX lag[2][5];
        ST q1[2][9];
        long long rest_own[2] = {0, 0};
        float rest_f[2] = {0.0f, 0.0f};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int ly = ly0 + c;
            const int gx = x0 + lx, gy = y0 + ly;
            id[c] = (gy < ny ? gy : ny - 1) * Dm.pitch + (gx < nx ? gx : nx - 1);
#pragma unroll
            for (int i = 0; i < 9; ++i) f2raw[c][i] = f2s(i, ly + 1 - CY9[i], lx + L::M2 - CX9[i]);
#pragma unroll
            for (int k = 0; k < 4; ++k) lag[c][k] = SA[(k * L::RA + ly + 1) * L::WA + lx + L::MA];
            lag[c][4] = SL[ly * L::WL + lx];
#pragma unroll
            for (int i = L::I1; i < 9; ++i) q1[c][i] = f1s(i - L::I1, ly + 3 - CY9[i], lx + L::M1 - CX9[i]);
            if constexpr (P::MIX) {
                rest_own[c] = S3[(ly + 2) * L::W3 + lx + 2];
                rest_f[c] = float_of_fixed(rest_own[c]);
            }
        }
        F2 f1[9];
        F2 phi;
        {
            F2 acc = mk2(0.0f);
#pragma unroll
            for (int i = L::I1; i < 9; ++i) {
                const F2 v = P::MIX ? mk2(stored_to_float<ST>(q1[0][i]), stored_to_float<ST>(q1[1][i]))
                                    : mk2(Conv<P>::ld(q1[0][i], 1.0f), Conv<P>::ld(q1[1][i], 1.0f));
                acc = acc + v;
                f1[i] = P::MIX ? v * mk2(isc1) : v;
            }
            if constexpr (P::MIX) {
                f1[0] = mk2(rest_f[0], rest_f[1]);
                phi = fma2(acc, mk2(isc1), f1[0]);
            } else {
                phi = acc;
            }
        }
        // PMIX: the cells' exact fixed-point phi; the pulled movers are dead after this
        long long racc[2] = {0, 0};
        if constexpr (P::MIX) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                int sold = 0;
#pragma unroll
                for (int i = 1; i < 9; ++i) sold += fix24_stored<ST>(q1[c][i]);
                racc[c] = rest_own[c] + fix24_to_rest(sold, p.klog2[0]);
            }
        }
        const int hx = lx + 2, hy = ly0 + 2;
        s_phi[hy][hx] = phi.v.x;
        s_phi[hy + 1][hx] = phi.v.y;
        constexpr int RING = 4 * (TX + 4) + 4 * TY;
        for (int r = tid; r < RING; r += NT) {
            int rx, ry;
            if (r < 2 * FX) {
                ry = r / FX;
                rx = r % FX;
            } else if (r < 4 * FX) {
                const int rr = r - 2 * FX;
                ry = TY + 2 + rr / FX;
                rx = rr % FX;
            } else {
                const int rr = r - 4 * FX;
                ry = 2 + rr / 4;
                const int c = rr % 4;
                rx = c < 2 ? c : TX + c;
            }
            s_phi[ry][rx] = phi_frame(rx, ry);
        }
        // phi0 on the whole tile + 2 frame
        for (int r = tid; r < FX * FY; r += NT) {
            const int fx = r % FX, fy = r / FX;
            (&s_p0[0][0])[r] = (float)S0[fy * L::W0 + fx - 2 + L::M0];
        }
        // row offsets of the CTA's next tile (read after the barrier below)
        if (t + (int)gridDim.x < A.ntiles) stage_rows<TY, NT>(A, t + gridDim.x, s_rows, tid);
        // w = S_x u_y - u_x S_y of the previous step on the tile + 1 frame
        for (int r = tid; r < WX * WY; r += NT) {
            const int wx = r % WX, wy = r / WX;
            const int o = wy * L::WA + wx - 1 + L::MA;
            const float ux = (float)SA[0 * L::RA * L::WA + o], uy = (float)SA[1 * L::RA * L::WA + o];
            const float Sx = (float)SA[2 * L::RA * L::WA + o], Sy = (float)SA[3 * L::RA * L::WA + o];
            (&s_w[0][0])[r] = Sx * uy - ux * Sy;
        }
        __syncthreads();  // the staging buffer is read

        // the CTA's next tile: its copies overlap stages B and C
        if (t + (int)gridDim.x < A.ntiles) stage_issue<P, TX, TY, NT>(A, t + gridDim.x, s_rows, sbase, bar, tid);

        pair_mu<FX, WX, WY, NT>(kp, s_phi, s_p0, s_mu, tid);
        __syncthreads();

        {
            const int gx = x0 + lx, gy0 = y0 + ly0;
            const bool valid0 = gx < nx && gy0 < ny, valid1 = gx < nx && gy0 + 1 < ny;
            pair_cells<P, FX, WX>(A, p, kp, s_phi, s_p0, s_mu, s_w, hx, hy, lx + 1, ly0 + 1, phi, f1, f2raw, lag, racc,
                                  id, valid0, valid1, fd, rd, ad, plane);
        }
    }
}

}  // namespace pf
