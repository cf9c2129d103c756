// 2D fused time step, two cells per thread (FP32 arithmetic policies).
//
// The same update as k_step2d (Sec. 3.3, steps 2-6 and 7; Eqs. 9, 29-38) for
// a tile of TX x 2 TYP cells on TX x TYP threads: thread (lx, j) owns the
// vertically adjacent cells (x0 + lx, y0 + 2j) and (x0 + lx, y0 + 2j + 1).
// Everything a cell computes from its own values and its stencils -- the
// gradients, u*, the penalty force, the pressure, both sets of Hermite
// equilibria and sources and both collisions -- runs on the pair as packed
// FP32 (one f32x2 instruction per operation for both cells), which halves the
// issue slots of the arithmetic that dominates the step.  Loads, stores, the
// conversions of the 16-bit policies and their exact rest bookkeeping stay per
// cell.  Fixed solids only (free particles use k_step2d).
#pragma once

#include "pf_kernels2d.cuh"

namespace pf {

// ---- packed FP32 pairs ------------------------------------------------------------------------
struct F2 {
    float2 v;
};
__device__ __forceinline__ F2 mk2(float a) { return {make_float2(a, a)}; }
__device__ __forceinline__ F2 mk2(float a, float b) { return {make_float2(a, b)}; }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return {__fmul2_rn(a.v, b.v)}; }
// a - b as one fused operation: b * (-1) + a
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    return {__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)};
}
// a * b + c
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }

// 1 / a per lane with the hardware's approximate reciprocal (one instruction,
// within 1 ulp; subnormals flushed): the arguments here are a density, a
// bounded 1 - phi0 and inverse relaxation rates >= 1/2, all normal numbers
__device__ __forceinline__ float rcp_fast(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ F2 rcp2(F2 a) { return mk2(rcp_fast(a.v.x), rcp_fast(a.v.y)); }

// Column values a[y - 1 .. y + 2][x] of a shared array, as the pairs of the
// stencils of rows (y, y + 1).
template <int W>
struct Col4 {
    float r0, r1, r2, r3;
};
template <int W>
__device__ __forceinline__ Col4<W> col4(const float (*a)[W], int x, int y)
{
    return {a[y - 1][x], a[y][x], a[y + 1][x], a[y + 2][x]};
}

// Isotropic D2Q9 gradient and Laplacian (weights 4/9, 1/9, 1/36, cs^2 = 1/3)
// of rows (y, y + 1) at column x, from the columns x - 1, x, x + 1.
template <int W>
__device__ __forceinline__ void grad9_pair(const float (*a)[W], int x, int y, F2 &gx, F2 &gy)
{
    const Col4<W> w = col4<W>(a, x - 1, y), c = col4<W>(a, x, y), e = col4<W>(a, x + 1, y);
    // D_k = e_k - w_k, R_k = e_k + w_k (k = row offset + 1)
    const F2 Dlo = mk2(e.r0, e.r1) - mk2(w.r0, w.r1);
    const F2 Dmid = mk2(e.r1, e.r2) - mk2(w.r1, w.r2);
    const F2 Dhi = mk2(e.r2, e.r3) - mk2(w.r2, w.r3);
    const F2 Rlo = mk2(e.r0, e.r1) + mk2(w.r0, w.r1);
    const F2 Rhi = mk2(e.r2, e.r3) + mk2(w.r2, w.r3);
    const F2 Clo = mk2(c.r0, c.r1), Chi = mk2(c.r2, c.r3);
    const F2 third = mk2(1.0f / 3.0f), twelfth = mk2(1.0f / 12.0f);
    gx = fma2(third, Dmid, twelfth * (Dlo + Dhi));
    gy = fma2(third, Chi - Clo, twelfth * (Rhi - Rlo));
}

// the same gradient of the cubes a^3 (the phi0^3 stencil of the own-angle
// wetting force, reading R18)
template <int W>
__device__ __forceinline__ void grad9_cubed_pair(const float (*a)[W], int x, int y, F2 &gx, F2 &gy)
{
    Col4<W> w = col4<W>(a, x - 1, y), c = col4<W>(a, x, y), e = col4<W>(a, x + 1, y);
    auto cube = [](Col4<W> &q) {
        q.r0 = q.r0 * q.r0 * q.r0;
        q.r1 = q.r1 * q.r1 * q.r1;
        q.r2 = q.r2 * q.r2 * q.r2;
        q.r3 = q.r3 * q.r3 * q.r3;
    };
    cube(w);
    cube(c);
    cube(e);
    const F2 Dlo = mk2(e.r0, e.r1) - mk2(w.r0, w.r1);
    const F2 Dmid = mk2(e.r1, e.r2) - mk2(w.r1, w.r2);
    const F2 Dhi = mk2(e.r2, e.r3) - mk2(w.r2, w.r3);
    const F2 Rlo = mk2(e.r0, e.r1) + mk2(w.r0, w.r1);
    const F2 Rhi = mk2(e.r2, e.r3) + mk2(w.r2, w.r3);
    const F2 Clo = mk2(c.r0, c.r1), Chi = mk2(c.r2, c.r3);
    const F2 third = mk2(1.0f / 3.0f), twelfth = mk2(1.0f / 12.0f);
    gx = fma2(third, Dmid, twelfth * (Dlo + Dhi));
    gy = fma2(third, Chi - Clo, twelfth * (Rhi - Rlo));
}

template <int W>
__device__ __forceinline__ F2 lap9_pair(const float (*a)[W], int x, int y)
{
    const Col4<W> w = col4<W>(a, x - 1, y), c = col4<W>(a, x, y), e = col4<W>(a, x + 1, y);
    const F2 Rlo = mk2(e.r0, e.r1) + mk2(w.r0, w.r1);
    const F2 Rmid = mk2(e.r1, e.r2) + mk2(w.r1, w.r2);
    const F2 Rhi = mk2(e.r2, e.r3) + mk2(w.r2, w.r3);
    const F2 Clo = mk2(c.r0, c.r1), Cmid = mk2(c.r1, c.r2), Chi = mk2(c.r2, c.r3);
    // 2/3 (side - 4 c) + 1/6 (diag - 4 c)
    const F2 side = Rmid + (Clo + Chi);
    const F2 diag = Rlo + Rhi;
    return fma2(mk2(2.0f / 3.0f), side, fma2(mk2(1.0f / 6.0f), diag, mk2(-10.0f / 3.0f) * Cmid));
}

// Populations of two cells from their Hermite moments: raw moments m = N_H^-1 h,
// then f = M_0^-1 m (Eq. 38).
__device__ __forceinline__ void from_hermite9_pair(const F2 h[9], F2 f[9], F2 cs2, F2 cs4)
{
    F2 m[9];
    m[0] = h[0];
    m[1] = h[1];
    m[2] = h[2];
    m[3] = fma2(cs2, h[0], h[3]);
    m[4] = fma2(cs2, h[0], h[4]);
    m[5] = h[5];
    m[6] = fma2(cs2, h[1], h[6]);
    m[7] = fma2(cs2, h[2], h[7]);
    m[8] = fma2(cs4, h[0], fma2(cs2, h[3] + h[4], h[8]));
    const F2 q = mk2(0.25f), hh = mk2(0.5f);
    const F2 p56 = m[8] + m[7], n56 = m[8] - m[7];
    const F2 s56 = m[5] + m[6], d56 = m[5] - m[6];
    f[5] = q * (p56 + s56);
    f[6] = q * (p56 - s56);
    f[7] = q * (n56 + d56);
    f[8] = q * (n56 - d56);
    const F2 a3 = m[3] - m[8], a4 = m[4] - m[8];
    const F2 b1 = m[1] - m[6], b2 = m[2] - m[7];
    f[1] = hh * (a3 + b1);
    f[3] = hh * (a3 - b1);
    f[2] = hh * (a4 + b2);
    f[4] = hh * (a4 - b2);
    f[0] = (m[0] - m[3]) + (m[8] - m[4]);
}

// Hermite-moment MRT collision (Eqs. 29, 37, 38 with c = 1) of two cells:
// h = N_H M_0 f; h* = h - S (h - heq) + (1 - S/2) hF; f* = M_0^-1 N_H^-1 h*.
// nS = -S and cF = 1 - S/2 per moment; ZEQ / ZF flag moments whose
// equilibrium / source is zero (bit k for moment k).
template <unsigned ZEQ, unsigned ZF>
__device__ __forceinline__ void collide9_pair(F2 f[9], const F2 heq[9], const F2 hF[9], const F2 nS[9],
                                              const F2 cF[9], F2 cs2, F2 cs4)
{
    const F2 a57 = f[5] + f[7], a68 = f[6] + f[8];
    const F2 m8r = a57 + a68;
    F2 m[9];
    m[0] = ((f[0] + f[1]) + (f[2] + f[3])) + (f[4] + m8r);
    m[1] = ((f[1] - f[3]) + (f[5] - f[6])) + (f[8] - f[7]);
    m[2] = ((f[2] - f[4]) + (f[5] + f[6])) - (f[7] + f[8]);
    m[3] = (f[1] + f[3]) + m8r;
    m[4] = (f[2] + f[4]) + m8r;
    m[5] = a57 - a68;
    m[6] = (f[5] - f[6]) + (f[8] - f[7]);
    m[7] = (f[5] + f[6]) - (f[7] + f[8]);
    m[8] = m8r;
    // Hermite moments (rows of N_H)
    const F2 ncs2 = mk2(0.0f) - cs2;
    F2 h[9];
    h[0] = m[0];
    h[1] = m[1];
    h[2] = m[2];
    h[3] = fma2(ncs2, m[0], m[3]);
    h[4] = fma2(ncs2, m[0], m[4]);
    h[5] = m[5];
    h[6] = fma2(ncs2, m[1], m[6]);
    h[7] = fma2(ncs2, m[2], m[7]);
    h[8] = fma2(cs4, m[0], fma2(ncs2, m[3] + m[4], m[8]));
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const F2 d = ((ZEQ >> k) & 1u) ? h[k] : h[k] - heq[k];
        F2 r = fma2(nS[k], d, h[k]);
        if (!((ZF >> k) & 1u)) r = fma2(cF[k], hF[k], r);
        h[k] = r;
    }
    from_hermite9_pair(h, f, cs2, cs4);
}

// Stage B: mu_phi (Eq. 9) on the tile + 1 frame, two rows per work item.
template <int FX, int WX, int WY, int NT>
__device__ __forceinline__ void pair_mu(const KParams<float> &kp, const float (*s_phi)[FX],
                                        const float (*s_p0)[FX], float (*s_mu)[WX], int tid)
{
    {
        const F2 c_dw = mk2(kp.c_dw), c_lap = mk2(-kp.c_lap), c_pen = mk2(kp.c_pen),
                 c_wet = mk2(kp.c_wet), c_wlap = mk2(-kp.c_wlap), one = mk2(1.0f), three = mk2(3.0f);
        constexpr int NPAIR = WX * (WY / 2);
        for (int r = tid; r < NPAIR; r += NT) {
            const int wx = r % WX, wy = 2 * (r / WX);
            const int fx = wx + 1, fy = wy + 1;
            const F2 ph = mk2(s_phi[fy][fx], s_phi[fy + 1][fx]);
            const F2 p0 = mk2(s_p0[fy][fx], s_p0[fy + 1][fx]);
            const F2 lp = lap9_pair<FX>(s_phi, fx, fy), lp0 = lap9_pair<FX>(s_p0, fx, fy);
            const F2 p02 = p0 * p0;
            F2 mu = c_dw * ph * ((ph - one) * (ph + one));
            mu = fma2(c_lap, lp, mu);
            mu = fma2(c_pen * p02, ph, mu);
            mu = fma2(c_wet * p0, fma2(three * ph, ph, p02) - one, mu);
            mu = fma2(c_wlap, lp0, mu);
            s_mu[wy][wx] = mu.v.x;
            s_mu[wy + 1][wx] = mu.v.y;
        }
    }
}

// The update of two cells (Eqs. 29-38) from their stencil values, shared by
// every two-cells-per-thread kernel: phi, phi0 and mu_phi of the cells, the
// gradients of phi, mu_phi and w = S_x u_y - u_x S_y (previous step), the
// previous step's u, S, phi (upx .. php), and both lattices' pulled
// populations in the arithmetic scale (f1, f2; replaced by the
// post-collision populations).  Returns u and S of this step.  CAC: the
// instantiation also serves domains with the conservative Allen-Cahn order
// parameter (checked per domain).  MU0: the force carries mu_phi0 grad phi0
// (Eq. 19) of the fixed solids, from lphi (Laplacian of phi) and g0 (grad
// phi0); with wv (some particle of the simulation has its own contact angle,
// reading R18) the phi0^2 grad phi0 part of its wetting term is the stencil
// gradient of phi0^3 over 3, g3 = grad(phi0^3).  done1(f1) runs as soon as the order-parameter lattice has collided
// (a caller can store it and free its registers before the flow lattice
// collides); done2(f2, u_x, u_y, S_x, S_y) at the end.
struct NoEmit {
    template <class... T>
    __device__ __forceinline__ void operator()(T &&...) const {}
};

// UNIT: every relaxation rate that multiplies a non-conserved moment is 1
// (s_1phi, s_1, s_2 = s_3 = s_4 of Eq. 38; the paper's defaults), so for those
// moments h* = h - (h - heq) + hF/2 = heq + hF/2 (Eq. 37): the order-parameter
// populations after collision follow from the macroscopic fields alone (f1 is
// not read), and of the flow moments only 0 (rate s0) and the second-order
// ones (rates s_2a, s_2b of Eq. 35) are taken from f2.
template <bool CAC, bool MU0, class E1 = NoEmit, class E2 = NoEmit, bool UNIT = false>
__device__ __forceinline__ void pair_physics(int phase_model, const KParams<float> &kp, F2 phi, F2 phi0,
                                             F2 mu, F2 gpx, F2 gpy, F2 gmx, F2 gmy, F2 wgx, F2 wgy, F2 lphi,
                                             F2 g0x, F2 g0y, F2 upx, F2 upy, F2 Spx, F2 Spy, F2 php,
                                             F2 (&f1)[9], F2 (&f2)[9], F2 &ux, F2 &uy, F2 &Sx, F2 &Sy,
                                             E1 done1 = E1(), E2 done2 = E2(), bool wv = false,
                                             F2 g3x = mk2(0.0f), F2 g3y = mk2(0.0f))
{
    const F2 drho = mk2(kp.drho), half = mk2(0.5f), one = mk2(1.0f), two = mk2(2.0f);
    const F2 rho = fma2(drho, phi, mk2(kp.rhom));
    const F2 muv = fma2(mk2(kp.dmu), phi, mk2(kp.mum));
    const F2 Mdrho = mk2(kp.Mdrho);
    // conservative Allen-Cahn option: theta n = (2/D)(1 - phi^2) grad phi/|grad phi|
    // and the mass flux M (rho1 - rho2)/2 (grad phi - theta n)
    const bool cac = CAC && phase_model == 1;
    F2 tnx = mk2(0.0f), tny = mk2(0.0f);
    if (cac) {
        const F2 g2 = fma2(gpx, gpx, gpy * gpy);
        const F2 th = mk2(kp.two_over_D) * (one - phi * phi);
        const F2 inv = mk2(g2.v.x > 1e-24f ? 1.0f / sqrtf(g2.v.x) : 0.0f,
                           g2.v.y > 1e-24f ? 1.0f / sqrtf(g2.v.y) : 0.0f);
        tnx = th * gpx * inv;
        tny = th * gpy * inv;
    }
    Sx = cac ? Mdrho * (gpx - tnx) : Mdrho * gmx;
    Sy = cac ? Mdrho * (gpy - tny) : Mdrho * gmy;
    const F2 grx = drho * gpx, gry = drho * gpy;
    // F = mu grad phi + F_b + F_c, F_c = (-d_y w, d_x w)/2 from the previous step
    F2 Fx = fma2(mu, gpx, fma2(mk2(-0.5f), wgy, mk2(kp.Fb[0])));
    F2 Fy = fma2(mu, gpy, fma2(half, wgx, mk2(kp.Fb[1])));
    if constexpr (MU0) {
        if (wv) {
            const F2 m = fma2(mk2(kp.c_pen) * phi0, phi * phi,
                              fma2(mk2(kp.c_wet) * phi, phi * phi - one, mk2(-kp.c_wlap) * lphi));
            const F2 cv = mk2(kp.c_wet) * phi;
            Fx = fma2(m, g0x, fma2(cv, g3x, Fx));
            Fy = fma2(m, g0y, fma2(cv, g3y, Fy));
        } else {
            const F2 mu0 = fma2(mk2(kp.c_pen) * phi0, phi * phi,
                                fma2(mk2(kp.c_wet) * phi, fma2(mk2(3.0f) * phi0, phi0, phi * phi - one),
                                     mk2(-kp.c_wlap) * lphi));
            Fx = fma2(mu0, g0x, Fx);
            Fy = fma2(mu0, g0y, Fy);
        }
    }

    // u* (Eq. 36a)
    const F2 jx = ((f2[1] - f2[3]) + (f2[5] - f2[6])) + (f2[8] - f2[7]);
    const F2 jy = ((f2[2] - f2[4]) + (f2[5] + f2[6])) - (f2[7] + f2[8]);
    const F2 irho = rcp2(rho);
    const F2 usx = fma2(half, Fx, jx) * irho, usy = fma2(half, Fy, jy) * irho;
    // penalty force f = phi0 (u_s - u*) with u_s = 0 (fixed solids)
    const F2 nphi0 = mk2(0.0f) - phi0;
    const F2 fpx = nphi0 * usx, fpy = nphi0 * usy;
    ux = fma2(half, fpx, usx);
    uy = fma2(half, fpy, usy);
    const F2 Ftx = fma2(rho, fpx, Fx), Fty = fma2(rho, fpy, Fy);

    // relaxation rates (Eq. 35, 1 - phi0 bounded below by solid_eps)
    const float seps = kp.solid_eps;
    const F2 solid = one - phi0;
    const F2 solidc = mk2(fmaxf(solid.v.x, seps), fmaxf(solid.v.y, seps));
    const F2 nu = muv * irho * rcp2(solidc);
    const F2 inv_s2a = fma2(mk2(kp.two_over_1md0), nu, half);
    const F2 inv_s2b = fma2(mk2(kp.inv_cs2), nu, half);
    const F2 Kf = mk2(kp.K);
    const F2 H = Kf * (mk2(kp.Hc0) - mk2(kp.Hc1) * inv_s2a);
    // pressure (Eq. 36b)
    const F2 sum_f = ((f2[1] + f2[2]) + (f2[3] + f2[4])) + ((f2[5] + f2[6]) + (f2[7] + f2[8]));
    const F2 ugr = fma2(ux, grx, uy * gry);
    const F2 rus_u = fma2(fma2(rho, ux, mk2(0.0f) - Sx), ux, fma2(rho, uy, mk2(0.0f) - Sy) * uy);
    const F2 Su = fma2(Sx, ux, Sy * uy), Sup = fma2(Spx, upx, Spy * upy);
    const F2 dt_term = fma2(two, fma2(ux, Ftx, uy * Fty), Sup - Su);
    const F2 Pr = mk2(kp.Pfac) *
                  fma2(Kf * half, dt_term,
                       fma2(half + H, ugr, fma2(mk2(-kp.w0f * kp.inv_1mcs2), rus_u, sum_f)));

    const F2 cs2 = mk2(kp.cs2), cs4 = mk2(kp.cs4);
    F2 heq[9], hF[9], nS[9], cF[9];
    // ---- order-parameter lattice (Eq. 30): Hermite equilibria and source
    {
        const F2 eta_mu = cac ? phi : mk2(kp.eta) * mu;  // Allen-Cahn: eta mu -> phi
        heq[0] = phi;
        heq[1] = phi * ux;
        heq[2] = phi * uy;
        heq[3] = cs2 * (eta_mu - phi);
        heq[4] = heq[3];
        heq[8] = cs4 * (phi - eta_mu);
        hF[1] = heq[1] - php * upx;  // d_t(phi u), explicit Euler
        hF[2] = heq[2] - php * upy;
        if (cac) {
            hF[1] = fma2(cs2, tnx, hF[1]);
            hF[2] = fma2(cs2, tny, hF[2]);
        }
        if constexpr (UNIT) {
            // h* = heq + hF/2; moment 0 is phi itself (conserved)
            F2 hs[9];
            hs[0] = phi;
            hs[1] = fma2(half, hF[1], heq[1]);
            hs[2] = fma2(half, hF[2], heq[2]);
            hs[3] = heq[3];
            hs[4] = heq[3];
            hs[5] = hs[6] = hs[7] = mk2(0.0f);
            hs[8] = heq[8];
            from_hermite9_pair(hs, f1, cs2, cs4);
        } else {
            const float s[9] = {kp.s0, kp.s1phi, kp.s1phi, kp.s2, kp.s2, kp.s2, kp.s3, kp.s3, kp.s4};
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                nS[k] = mk2(-s[k]);
                cF[k] = mk2(1.0f - 0.5f * s[k]);
            }
            // zero equilibria: moments 5, 6, 7; zero sources: 0 and 3..8
            collide9_pair<(1u << 5) | (1u << 6) | (1u << 7), 0x1F9u>(f1, heq, hF, nS, cF, cs2, cs4);
        }
        done1(f1);
    }
    // ---- flow lattice (Eqs. 32-34)
    {
        const F2 rux = rho * ux, ruy = rho * uy;
        heq[1] = rux;
        heq[2] = ruy;
        heq[3] = Pr + (rux - Sx) * ux;
        heq[4] = Pr + (ruy - Sy) * uy;
        heq[5] = rux * uy - half * fma2(Sx, uy, ux * Sy);
        heq[8] = (mk2(0.0f) - cs2) * Pr;
        const F2 c3 = one - mk2(3.0f) * cs2;
        const F2 tcs2 = two * cs2;
        hF[0] = ugr;
        hF[1] = Ftx;
        hF[2] = Fty;
        hF[3] = fma2(two * ux, Ftx, fma2(tcs2 * ux, grx, fma2(c3, ugr, Spx * upx - Sx * ux)));
        hF[4] = fma2(two * uy, Fty, fma2(tcs2 * uy, gry, fma2(c3, ugr, Spy * upy - Sy * uy)));
        hF[5] = fma2(ux, Fty, Ftx * uy) -
                half * (fma2(Sx, uy, ux * Sy) - fma2(Spx, upy, upx * Spy)) + cs2 * fma2(ux, gry, grx * uy);
        const F2 s2a = rcp2(inv_s2a);
        const F2 s2b = rcp2(inv_s2b);
        if constexpr (UNIT) {
            // moments 0 (rate s0, zero equilibrium), 3, 4 (s_2a) and 5 (s_2b)
            // from f2; 1, 2 at heq + hF/2; 6, 7 zero; 8 at its equilibrium
            const F2 m8r = (f2[5] + f2[7]) + (f2[6] + f2[8]);
            const F2 m0 = f2[0] + sum_f;
            const F2 ncs2 = mk2(0.0f) - cs2;
            const F2 h0 = m0;
            const F2 h3 = fma2(ncs2, m0, (f2[1] + f2[3]) + m8r);
            const F2 h4 = fma2(ncs2, m0, (f2[2] + f2[4]) + m8r);
            const F2 h5 = (f2[5] + f2[7]) - (f2[6] + f2[8]);
            const F2 ns2a = mk2(0.0f) - s2a, ns2b = mk2(0.0f) - s2b;
            F2 hs[9];
            hs[0] = fma2(mk2(1.0f - 0.5f * kp.s0), hF[0], fma2(mk2(-kp.s0), h0, h0));
            hs[1] = fma2(half, hF[1], heq[1]);
            hs[2] = fma2(half, hF[2], heq[2]);
            hs[3] = fma2(fma2(mk2(-0.5f), s2a, one), hF[3], fma2(ns2a, h3 - heq[3], h3));
            hs[4] = fma2(fma2(mk2(-0.5f), s2a, one), hF[4], fma2(ns2a, h4 - heq[4], h4));
            hs[5] = fma2(fma2(mk2(-0.5f), s2b, one), hF[5], fma2(ns2b, h5 - heq[5], h5));
            hs[6] = hs[7] = mk2(0.0f);
            hs[8] = heq[8];
            from_hermite9_pair(hs, f2, cs2, cs4);
            done2(f2, ux, uy, Sx, Sy);
            return;
        }
        nS[0] = mk2(-kp.s0);
        nS[1] = nS[2] = mk2(-kp.s1);
        nS[3] = nS[4] = mk2(0.0f) - s2a;
        nS[5] = mk2(0.0f) - s2b;
        nS[6] = nS[7] = mk2(-kp.s3);
        nS[8] = mk2(-kp.s4);
        cF[0] = mk2(1.0f - 0.5f * kp.s0);
        cF[1] = cF[2] = mk2(1.0f - 0.5f * kp.s1);
        cF[3] = cF[4] = fma2(mk2(-0.5f), s2a, one);
        cF[5] = fma2(mk2(-0.5f), s2b, one);
        // zero equilibria: moments 0, 6, 7; zero sources: 6, 7, 8
        collide9_pair<(1u << 0) | (1u << 6) | (1u << 7), (1u << 6) | (1u << 7) | (1u << 8)>(f2, heq, hF, nS,
                                                                                           cF, cs2, cs4);
    }
    done2(f2, ux, uy, Sx, Sy);
}

// Stage C of the pair step: the update of the thread's two cells (Eqs. 29-38)
// from the shared tiles (phi, phi0 on tile + 2 at (hx, hy); mu, w on tile + 1
// at (wx, wy)) and the values gathered in stage A, then their stores.  racc:
// PMIX, each cell's exact fixed-point phi (rest + images of the pulled movers).
// CAC: the instantiation also serves domains with the conservative Allen-Cahn
// order parameter (checked per domain).  MU0: the simulation holds free
// particles, so the force carries mu_phi0 grad phi0 (Eq. 19) of the fixed
// solids too (the tiles this kernel gets are out of every particle's reach).
template <class P, int FX, int WX, bool CAC = false, bool MU0 = false>
__device__ __forceinline__ void pair_cells(const StepArgs &A, const DevParams &p, const KParams<float> &kp,
                                           const float (*s_phi)[FX], const float (*s_p0)[FX],
                                           const float (*s_mu)[WX], const float (*s_w)[WX], int hx, int hy,
                                           int wx, int wy, F2 phi, F2 (&f1)[9],
                                           const typename P::store (&f2raw)[2][9],
                                           const typename P::aux (&lag)[2][5],
                                           const long long (&racc)[2], const int (&id)[2], bool valid0, bool valid1, typename P::store *fd,
                                           long long *rd, typename P::aux *ad, int plane)
{
    using ST = typename P::store;
    using AX = typename P::aux;

    const F2 phi0 = mk2(s_p0[hy][hx], s_p0[hy + 1][hx]);
    F2 gpx, gpy, gmx, gmy, wgx, wgy;
    grad9_pair<FX>(s_phi, hx, hy, gpx, gpy);
    grad9_pair<WX>(s_mu, wx, wy, gmx, gmy);
    grad9_pair<WX>(s_w, wx, wy, wgx, wgy);
    const F2 mu = mk2(s_mu[wy][wx], s_mu[wy + 1][wx]);
    F2 lphi = mk2(0.0f), g0x = mk2(0.0f), g0y = mk2(0.0f), g3x = mk2(0.0f), g3y = mk2(0.0f);
    if constexpr (MU0) {
        lphi = lap9_pair<FX>(s_phi, hx, hy);
        grad9_pair<FX>(s_p0, hx, hy, g0x, g0y);
        if (A.wv) grad9_cubed_pair<FX>(s_p0, hx, hy, g3x, g3y);
    }
    F2 f2[9];
    const F2 isc2v = mk2(kp.inv_scale[1]);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const F2 v = P::MIX ? mk2(stored_to_float<ST>(f2raw[0][i]), stored_to_float<ST>(f2raw[1][i]))
                            : mk2(Conv<P>::ld(f2raw[0][i], 1.0f), Conv<P>::ld(f2raw[1][i], 1.0f));
        f2[i] = P::MIX ? v * isc2v : v;
    }
    const F2 upx = mk2((float)lag[0][0], (float)lag[1][0]), upy = mk2((float)lag[0][1], (float)lag[1][1]);
    const F2 Spx = mk2((float)lag[0][2], (float)lag[1][2]), Spy = mk2((float)lag[0][3], (float)lag[1][3]);
    const F2 php = mk2((float)lag[0][4], (float)lag[1][4]);
    F2 ux, uy, Sx, Sy;
    pair_physics<CAC, MU0>(p.phase_model, kp, phi, phi0, mu, gpx, gpy, gmx, gmy, wgx, wgy, lphi, g0x, g0y, upx, upy,
                           Spx, Spy, php, f1, f2, ux, uy, Sx, Sy, NoEmit(), NoEmit(), MU0 && A.wv != 0, g3x, g3y);

    // ---------------- stores (per cell) ----------------
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (!(c == 0 ? valid0 : valid1)) continue;
        const int idc = id[c];
        const float phic = c == 0 ? phi.v.x : phi.v.y;
        const float uxc = c == 0 ? ux.v.x : ux.v.y, uyc = c == 0 ? uy.v.x : uy.v.y;
        if constexpr (P::MIX) {
            const float sc1 = kp.scale[0];
            int bad = 0, snew = 0;
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                ST q = Conv<P>::st(c == 0 ? f1[i].v.x : f1[i].v.y, sc1);
                if constexpr (P::id == 3) q = bf16_flush(q);
                snew += fix24_sat<ST>(q, &bad);
                fd[i * plane + idc] = q;
            }
            // exact: sum of the cell's order-parameter populations is unchanged
            rd[idc] = racc[c] - fix24_to_rest(snew, p.klog2[0]);
            if (bad) atomicOr(A.flags, 2);
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) fd[i * plane + idc] = Conv<P>::st(c == 0 ? f1[i].v.x : f1[i].v.y, 1.0f);
        }
        const float sc2 = P::MIX ? kp.scale[1] : 1.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) fd[(9 + i) * plane + idc] = Conv<P>::st(c == 0 ? f2[i].v.x : f2[i].v.y, sc2);
        // fields of this step, read as the previous step's by the next one
        ad[0 * plane + idc] = (AX)uxc;
        ad[1 * plane + idc] = (AX)uyc;
        ad[2 * plane + idc] = (AX)(c == 0 ? Sx.v.x : Sx.v.y);
        ad[3 * plane + idc] = (AX)(c == 0 ? Sy.v.x : Sy.v.y);
        ad[4 * plane + idc] = (AX)phic;
        if (!isfinite(phic) || !isfinite(uxc) || !isfinite(uyc)) atomicOr(A.flags, 1);
    }
}

// 256-thread pair tiles are register heavy: two resident CTAs per SM.
template <int TX, int TYP>
constexpr int step2d_pair_min_blocks()
{
    return TX * TYP > 256 ? 1 : 2;
}

template <class P, int TX, int TYP, bool CAC, bool MU0 = false>
__global__ void __launch_bounds__(TX *TYP, (step2d_pair_min_blocks<TX, TYP>())) k_step2d_pair(StepArgs A)
{
    using ST = typename P::store;
    using AX = typename P::aux;
    static_assert(sizeof(typename P::real) == 4, "pair kernel: FP32 arithmetic policies only");
    constexpr int NT = TX * TYP;
    constexpr int TY = 2 * TYP;             // tile rows
    constexpr int FX = TX + 4, FY = TY + 4;   // tile + 2 frame
    constexpr int WX = TX + 2, WY = TY + 2;   // tile + 1 frame
    __shared__ float s_phi[FY][FX];
    __shared__ float s_p0[FY][FX];
    __shared__ float s_mu[WY][WX];
    __shared__ float s_w[WY][WX];
    __shared__ int s_gx[TX + 6];
    __shared__ int s_gy[TY + 6];  // row offsets y * pitch (planes hold < 2^31 cells)

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly0 = 2 * (tid / TX);  // first of the thread's two rows

    for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
        if (A.tile_sel && A.tile_sel[t] != A.sel) continue;  // (uniform in the block)
        const DomainDev &Dm = A.doms[A.tile_dom[t]];
        const int2 txy = A.tile_xy[t];
        const int nx = Dm.nx, ny = Dm.ny;
        const int plane = (int)Dm.plane;  // (Q1 + Q2) * plane < 2^31 (checked at create)
        const int x0 = txy.x * TX, y0 = txy.y * TY;
        const DevParams &p = Dm.p;
        const KParams<float> &kp = Dm.kf;

        __syncthreads();  // previous tile's shared-memory readers are done
        for (int k = tid; k < TX + 6; k += NT) s_gx[k] = wrap_idx(x0 - 3 + k, nx);
        for (int k = tid; k < TY + 6; k += NT) s_gy[k] = wrap_idx(y0 - 3 + k, ny) * Dm.pitch;
        __syncthreads();

        const ST *fs = reinterpret_cast<const ST *>(Dm.f[A.par]);
        ST *fd = reinterpret_cast<ST *>(Dm.f[A.par ^ 1]);
        const AX *as = reinterpret_cast<const AX *>(Dm.aux[A.par]);
        AX *ad = reinterpret_cast<AX *>(Dm.aux[A.par ^ 1]);
        const AX *ph0 = reinterpret_cast<const AX *>(Dm.phi0);
        const long long *rs = reinterpret_cast<const long long *>(Dm.rest[A.par]);
        long long *rd = reinterpret_cast<long long *>(Dm.rest[A.par ^ 1]);
        const float isc1 = kp.inv_scale[0];

        // phi at frame cell (hx, hy) of the tile+2 frame: pull and sum (Eq. 31)
        auto phi_ring = [&](int hx, int hy) -> float {
            const int cx = hx + 1, cy = hy + 1;  // tile+3 table coordinates
            float acc;
            if constexpr (P::MIX) {
                acc = float_of_fixed(rs[s_gy[cy] + s_gx[cx]]);
                float movers = 0.0f;
#pragma unroll
                for (int i = 1; i < 9; ++i)
                    movers += stored_to_float<ST>(ldg(fs + i * plane + s_gy[cy - CY9[i]] + s_gx[cx - CX9[i]]));
                acc += movers * isc1;
            } else {
                acc = 0.0f;
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    acc += Conv<P>::ld(ldg(fs + i * plane + s_gy[cy - CY9[i]] + s_gx[cx - CX9[i]]), isc1);
            }
            return acc;
        };

        // ---------------- stage A ----------------
        // own cells: every DRAM load issued before the first barrier
        int id[2];
        ST f2raw[2][9];
        AX lag[2][5];
        ST q1[2][9];
        long long rest_own[2] = {0, 0};
        float rest_f[2] = {0.0f, 0.0f};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int ty = ly0 + c + 3;
            id[c] = s_gy[ty] + s_gx[lx + 3];
#pragma unroll
            for (int i = 0; i < 9; ++i)
                f2raw[c][i] = ldg(fs + (9 + i) * plane + s_gy[ty - CY9[i]] + s_gx[lx + 3 - CX9[i]]);
#pragma unroll
            for (int k = 0; k < 5; ++k) lag[c][k] = ldg(as + k * plane + id[c]);
#pragma unroll
            for (int i = (P::MIX ? 1 : 0); i < 9; ++i)
                q1[c][i] = ldg(fs + i * plane + s_gy[ty - CY9[i]] + s_gx[lx + 3 - CX9[i]]);
            if constexpr (P::MIX) {
                rest_own[c] = rs[id[c]];
                rest_f[c] = float_of_fixed(rest_own[c]);
            }
        }
        // the pair's phi (Eq. 31) and its order-parameter populations
        F2 f1[9];
        F2 phi;
        {
            F2 acc = mk2(0.0f);
#pragma unroll
            for (int i = (P::MIX ? 1 : 0); i < 9; ++i) {
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
        s_p0[hy][hx] = (float)ldg(ph0 + id[0]);
        s_p0[hy + 1][hx] = (float)ldg(ph0 + id[1]);
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
            s_phi[ry][rx] = phi_ring(rx, ry);
            s_p0[ry][rx] = (float)ldg(ph0 + s_gy[ry + 1] + s_gx[rx + 1]);
        }
        // w = S_x u_y - u_x S_y of the previous step: own cells from the lagged
        // fields in registers, the tile+1 ring by the last threads
#pragma unroll
        for (int c = 0; c < 2; ++c)
            s_w[ly0 + c + 1][lx + 1] = (float)lag[c][2] * (float)lag[c][1] - (float)lag[c][0] * (float)lag[c][3];
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
            const float ux = (float)ldg(as + 0 * plane + wid), uy = (float)ldg(as + 1 * plane + wid);
            const float Sx = (float)ldg(as + 2 * plane + wid), Sy = (float)ldg(as + 3 * plane + wid);
            s_w[wy][wx] = Sx * uy - ux * Sy;
        }
        __syncthreads();

        pair_mu<FX, WX, WY, NT>(kp, s_phi, s_p0, s_mu, tid);
        __syncthreads();

        // ---------------- stage C: the thread's two cells ----------------
        {
            const int gx = x0 + lx, gy0 = y0 + ly0;
            const bool valid0 = gx < nx && gy0 < ny, valid1 = gx < nx && gy0 + 1 < ny;
            pair_cells<P, FX, WX, CAC, MU0>(A, p, kp, s_phi, s_p0, s_mu, s_w, hx, hy, lx + 1, ly0 + 1, phi, f1, f2raw, lag, racc,
                                  id, valid0, valid1, fd, rd, ad, plane);
        }
    }
}

}  // namespace pf
