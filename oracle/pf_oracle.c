/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see pf_oracle.h).
 *
 * Plain restatement of the lattice Boltzmann scheme of Sec. 3 of
 * Zhan, Liu, Chai & Shi (arXiv 2311.05097):
 *   - order-parameter lattice, Eqs. (30), (31), with M = (1/s_1phi - 1/2) eta cs^2;
 *   - flow lattice, Eqs. (32)-(36);
 *   - MRT collision, Eq. (29), with Lambda = M_H^-1 S_H M_H, Eqs. (37), (38);
 *   - chemical potentials, Eqs. (9), (19); density and viscosity, Eqs. (17), (18);
 *   - free energy, Eq. (8); kinetic energy, Sec. 2.3;
 *   - rigid particles, Eqs. (26)-(28), explicit Euler (Sec. 3 opening);
 *   - the computational procedure of Sec. 3.3.
 * Every stage is one full-grid pass over plain arrays.  Lattice units:
 * dx = dt = c = 1, cs^2 = d0.
 *
 * Readings of points the paper leaves open (each is a documented choice):
 *   R1  phi0 = (1 + tanh(2 zeta / D)) / 2 with zeta = R - |x - x_p| for a particle
 *       (Eq. 13 and Eq. 39); total phi0 = fixed field + sum of particle indicators.
 *   R2  grad / Laplacian: second-order isotropic central stencils built on the
 *       D2Q9 (2D) or D3Q19 (3D) stencil with the classical weights
 *       (4/9, 1/9, 1/36) or (1/3, 1/18, 1/36) and cs_FD^2 = 1/3.
 *   R3  "c_ia c_ia" in Eqs. (32), (33) is summed over alpha per component.
 *   R4  d_t(rho u u) ~ u F + F u uses F_tot = F + rho f (first moment of Eq. 33).
 *   R5  the other time derivatives are explicit Euler with the previous step's
 *       u, phi, S (stored); at t = 0 the previous values equal the initial ones.
 *   R6  F_c = div(S u - u S)/2 (Eq. 33) is evaluated from the previous step's
 *       S and u; div contracts the first index, as in div[(rho u - S) u] of Eq. (16b).
 *   R7  every step recomputes the macroscopic fields from f, including step 1.
 *   R8  1 - phi0 is bounded below by solid_eps in the viscosity of Eq. (35)
 *       (and hence in s_2a, s_2b and H).
 *   R9  eta <= 0 selects eta = 2M/cs^2 (so s_1phi = 1).
 *   R10 the fluid density in Eqs. (26a), (28) is rho_bar = (rho1 + rho2)/2, the
 *       density at phi = 0 that the penalty term of Eq. (8) drives inside solids;
 *       V_p, M_p, I_p are those of a disc (2D, per unit depth) or a sphere (3D);
 *       F_in^n = rho_bar V_p (u_p^n - u_p^{n-1}), T_in^n = I_f (w^n - w^{n-1}).
 *   R11 mu_phi0 grad phi0 (Eq. 19) is included only when the simulation holds
 *       at least one free particle.
 *   R12 3D: D3Q19 flow lattice and D3Q7 order-parameter lattice with weights
 *       chosen so that sum w c_a c_b = cs^2 delta_ab and sum w c_a^2 c_b^2 = cs^4
 *       (a != b); M_H rows are tensor Hermite polynomials of the velocities; the
 *       viscosity relation of Eq. (35) and the 3D K, H of Sec. 3.2 are used as
 *       printed.
 *   R18 particles with their own contact angle theta_k (Sec. 4.5): the wetting
 *       terms of Eqs. (8), (9), (19) are summed over solids, each with its own
 *       angle; every solid without an own angle (the fixed field and such
 *       particles) forms one solid with the simulation's theta.  The penalty
 *       term keeps the total phi0.  Writing W = sum_s cos(theta_s) phi0_s and
 *       V = sum_s cos(theta_s) phi0_s^3, the wetting part of mu_phi is
 *       3 sigma/D (3 phi^2 W + V - W) - 3 D sigma/8 lap W, and the particle force
 *       sum_s mu_phi0,s grad phi0_s is 9 sigma/D phi0 phi^2 grad phi0 +
 *       3 sigma/D [phi (phi^2 - 1) grad W + phi grad V] - 3 D sigma/8 lap(phi) grad W
 *       (the phi0_s^2 grad phi0_s terms discretised as grad V / 3).
 *   R19 particle-particle repulsion of Sec. 4.5 as printed: (x_k - x_j)/eps times
 *       (R_k + R_j + xi - d)^2 for R_k + R_j <= d <= R_k + R_j + xi, times
 *       (R_k + R_j - d) for d <= R_k + R_j, zero beyond (minimum image), added to
 *       the force of Eq. (26a) from the positions before the update.
 *   R21 box walls (y = -1/2 and y = ny - 1/2, 2D and 3D; the paper's no-flux boxes):
 *       halfway bounce-back of both lattices at resting walls; the stencils read
 *       rows beyond a wall as the mirror image of the rows inside (zero normal
 *       gradient of phi, mu and phi0: no flux), except the products
 *       S_a u_b - u_a S_b of F_c, which change sign under the mirror.
 *   R22 particle-wall repulsion of Sec. 4.5: the imaginary particle is the
 *       mirror image of particle k across the nearest wall (a box wall of R21,
 *       or a circular wall given by centre and radius, mirrored along the
 *       radius), d' its distance; the printed form with 2 R_k for R_k + R_j and
 *       eps/2 for eps; the nearest wall only; added like R19.
 *   R23 conservative Allen-Cahn order parameter (the paper prints none; an
 *       option next to Eq. 2): d_t phi + div(phi u) = div(M (grad phi - theta n))
 *       with theta = (2/D)(1 - phi^2), n = grad phi / |grad phi| (0 where
 *       |grad phi|^2 <= 1e-24), whose flat profile tanh(2 zeta/D) has zero flux.
 *       On the lattice of Eq. (30): eta mu -> phi in the equilibrium (second
 *       Hermite moment zero), s_1phi = 1/(M/cs^2 + 1/2), and cs^2 theta n added
 *       to the source G; the mass flux of the momentum equation becomes
 *       S = M (rho1 - rho2)/2 (grad phi - theta n); mu_phi of Eq. (9) still
 *       gives the surface force, and solids and particles enter it as before.
  *   R25 the two-particle balance of Sec. 4.4 lets the particles move only
 *       vertically: a particle may hold single components of its motion
 *       (translation along an axis, the rotation), which keep their given
 *       value while the hydrodynamic force and torque are still reported.
 */
#include "pf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_QMAX 19
#define ORC_MAXP 64

typedef struct orc_lat {
    int kind, Q;
    int c[ORC_QMAX][3];
    double w[ORC_QMAX];
    double MH[ORC_QMAX * ORC_QMAX];
    double MHinv[ORC_QMAX * ORC_QMAX];
} orc_lat;

struct orc_sim {
    int dim, nx, ny, nz;
    long N;
    orc_params p;
    double cs2, eta, s1phi, cos_t;
    orc_lat L1, L2;
    int np;
    orc_particle parts[ORC_MAXP];
    double *f1, *f2, *g1, *g2;
    double *phi0_fixed, *phi0;
    double *u_prev, *phi_prev, *S_prev;
    /* per-stage work arrays */
    double *phi, *rho, *muv, *lap_phi, *lap_phi0, *mu, *mu0;
    double *gphi, *gphi0, *gmu, *S, *grho, *Fc, *F, *ustar, *fpen, *u, *Ftot;
    double *s2a, *s2b, *P, *tmp, *tmp3;
    /* R18: angle-weighted indicators and their stencils */
    double *wfld, *vfld, *lap_w, *gw, *gv;
    double *tn;  /* R23: theta n of the Allen-Cahn flux */
    int wall_y;  /* R21: walls at the ends of y instead of periodicity */
};

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* small dense linear algebra                                                */
/* ------------------------------------------------------------------------ */

/* Gauss-Jordan inverse with partial pivoting; returns 0 if singular. */
static int mat_inverse(int n, const double *A, double *Ainv)
{
    double a[ORC_QMAX * 2 * ORC_QMAX];
    int m = 2 * n;
    for (int r = 0; r < n; ++r)
        for (int col = 0; col < m; ++col)
            a[r * m + col] = col < n ? A[r * n + col] : (col - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r * m + col]) > fabs(a[piv * m + col])) piv = r;
        if (fabs(a[piv * m + col]) < 1e-300) return 0;
        if (piv != col)
            for (int k = 0; k < m; ++k) {
                double t = a[col * m + k];
                a[col * m + k] = a[piv * m + k];
                a[piv * m + k] = t;
            }
        double d = a[col * m + col];
        for (int k = 0; k < m; ++k) a[col * m + k] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double fct = a[r * m + col];
            if (fct == 0.0) continue;
            for (int k = 0; k < m; ++k) a[r * m + k] -= fct * a[col * m + k];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int col = 0; col < n; ++col) Ainv[r * n + col] = a[r * m + n + col];
    return 1;
}

static void matvec(int n, const double *A, const double *x, double *y)
{
    for (int r = 0; r < n; ++r) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += A[r * n + k] * x[k];
        y[r] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* lattices                                                                  */
/* ------------------------------------------------------------------------ */

/* D2Q9 velocity order fixed by the columns of M_0 in Eq. (38). */
static const int C_D2Q9[9][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
/* M_0 of Eq. (38), as printed. */
static const double M0_D2Q9[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},   {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1}, {0, 1, 0, 1, 0, 1, 1, 1, 1},
    {0, 0, 1, 0, 1, 1, 1, 1, 1},   {0, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, -1, -1, 1}, {0, 0, 0, 0, 0, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, 1, 1, 1, 1}};

static const int C_D3Q19[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static void lattice_setup(orc_lat *L, int kind, double d0)
{
    double cs2 = d0;
    memset(L, 0, sizeof(*L));
    L->kind = kind;
    if (kind == ORC_D2Q9) {
        /* Weights and M_H = N_H C_d M_0 with c = 1 (Sec. 4 opening, Eq. 38). */
        L->Q = 9;
        for (int i = 0; i < 9; ++i)
            for (int a = 0; a < 3; ++a) L->c[i][a] = C_D2Q9[i][a];
        L->w[0] = 1.0 - 2.0 * d0 + d0 * d0;
        for (int i = 1; i <= 4; ++i) L->w[i] = (d0 - d0 * d0) / 2.0;
        for (int i = 5; i <= 8; ++i) L->w[i] = d0 * d0 / 4.0;
        double NH[9][9];
        memset(NH, 0, sizeof(NH));
        for (int i = 0; i < 9; ++i) NH[i][i] = 1.0;
        NH[3][0] = -cs2;
        NH[4][0] = -cs2;
        NH[6][1] = -cs2;
        NH[7][2] = -cs2;
        NH[8][0] = cs2 * cs2;
        NH[8][3] = -cs2;
        NH[8][4] = -cs2;
        for (int r = 0; r < 9; ++r)
            for (int col = 0; col < 9; ++col) {
                double acc = 0.0;
                for (int k = 0; k < 9; ++k) acc += NH[r][k] * M0_D2Q9[k][col];
                L->MH[r * 9 + col] = acc;
            }
    } else if (kind == ORC_D3Q19) {
        L->Q = 19;
        for (int i = 0; i < 19; ++i)
            for (int a = 0; a < 3; ++a) L->c[i][a] = C_D3Q19[i][a];
        L->w[0] = 1.0 - 3.0 * d0 + 3.0 * d0 * d0;
        for (int i = 1; i <= 6; ++i) L->w[i] = (d0 - 2.0 * d0 * d0) / 2.0;
        for (int i = 7; i < 19; ++i) L->w[i] = d0 * d0 / 4.0;
        for (int i = 0; i < 19; ++i) {
            double cx = L->c[i][0], cy = L->c[i][1], cz = L->c[i][2];
            double hx = cx * cx - cs2, hy = cy * cy - cs2, hz = cz * cz - cs2;
            double row[19] = {1.0,     cx,      cy,      cz,      hx,      hy,     hz,
                              cx * cy, cx * cz, cy * cz, cx * hy, cx * hz, cy * hx, cy * hz,
                              cz * hx, cz * hy, hx * hy, hx * hz, hy * hz};
            for (int r = 0; r < 19; ++r) L->MH[r * 19 + i] = row[r];
        }
    } else { /* ORC_D3Q7 */
        L->Q = 7;
        for (int i = 0; i < 7; ++i)
            for (int a = 0; a < 3; ++a) L->c[i][a] = C_D3Q19[i][a];
        L->w[0] = 1.0 - 3.0 * d0;
        for (int i = 1; i <= 6; ++i) L->w[i] = d0 / 2.0;
        for (int i = 0; i < 7; ++i) {
            double cx = L->c[i][0], cy = L->c[i][1], cz = L->c[i][2];
            double row[7] = {1.0, cx, cy, cz, cx * cx - cs2, cy * cy - cs2, cz * cz - cs2};
            for (int r = 0; r < 7; ++r) L->MH[r * 7 + i] = row[r];
        }
    }
    mat_inverse(L->Q, L->MH, L->MHinv);
}

int orc_lattice(int kind, double d0, int *c, double *w, double *MH)
{
    orc_lat L;
    lattice_setup(&L, kind, d0);
    for (int i = 0; i < L.Q; ++i) {
        if (c)
            for (int a = 0; a < 3; ++a) c[i * 3 + a] = L.c[i][a];
        if (w) w[i] = L.w[i];
    }
    if (MH) memcpy(MH, L.MH, sizeof(double) * L.Q * L.Q);
    return L.Q;
}

/* Relaxation vectors: S_H^1 and S_H^2 of Eq. (38) and their 3D analogues. */
void orc_rates(int kind, int k, double s0, double s1, double s2a, double s2b,
               double s3, double s4, double *S)
{
    if (kind == ORC_D2Q9) {
        double v[9] = {s0, s1, s1, s2a, s2a, s2b, s3, s3, s4};
        memcpy(S, v, sizeof(v));
    } else if (kind == ORC_D3Q19) {
        double v[19] = {s0,  s1,  s1,  s1,  s2a, s2a, s2a, s2b, s2b, s2b,
                        s3,  s3,  s3,  s3,  s3,  s3,  s4,  s4,  s4};
        memcpy(S, v, sizeof(v));
    } else {
        double v[7] = {s0, s1, s1, s1, s2a, s2a, s2a};
        memcpy(S, v, sizeof(v));
    }
    (void)k;
}

static void lambda_of(const orc_lat *L, const double *S, double *Lam)
{
    int Q = L->Q;
    double tmp[ORC_QMAX * ORC_QMAX];
    for (int r = 0; r < Q; ++r)
        for (int col = 0; col < Q; ++col) tmp[r * Q + col] = S[r] * L->MH[r * Q + col];
    for (int r = 0; r < Q; ++r)
        for (int col = 0; col < Q; ++col) {
            double acc = 0.0;
            for (int k = 0; k < Q; ++k) acc += L->MHinv[r * Q + k] * tmp[k * Q + col];
            Lam[r * Q + col] = acc;
        }
}

void orc_lambda(int kind, double d0, const double *S, double *Lam)
{
    orc_lat L;
    lattice_setup(&L, kind, d0);
    lambda_of(&L, S, Lam);
}

/* Lambda v computed as M_H^-1 (S (M_H v)), i.e. the product of Eq. (37). */
static void apply_lambda(const orc_lat *L, const double *S, const double *v, double *out)
{
    double m[ORC_QMAX];
    matvec(L->Q, L->MH, v, m);
    for (int r = 0; r < L->Q; ++r) m[r] *= S[r];
    matvec(L->Q, L->MHinv, m, out);
}

/* ------------------------------------------------------------------------ */
/* equilibria and sources                                                    */
/* ------------------------------------------------------------------------ */

static int lat_dim(const orc_lat *L) { return L->kind == ORC_D2Q9 ? 2 : 3; }

/* Eq. (30), equilibrium of the order-parameter lattice. */
static void feq1_lat(const orc_lat *L, double cs2, double phi, const double *u,
                     double mu, double eta, double *feq)
{
    int d = lat_dim(L);
    for (int i = 0; i < L->Q; ++i) {
        double cu = 0.0;
        for (int a = 0; a < d; ++a) cu += L->c[i][a] * u[a];
        if (i == 0)
            feq[i] = phi + (L->w[0] - 1.0) * eta * mu;
        else
            feq[i] = L->w[i] * eta * mu + L->w[i] * cu * phi / cs2;
    }
}

/* Eq. (30), source of the order-parameter lattice, G = d_t(phi u). */
static void src1_lat(const orc_lat *L, double cs2, const double *G, double *F)
{
    int d = lat_dim(L);
    for (int i = 0; i < L->Q; ++i) {
        double cg = 0.0;
        for (int a = 0; a < d; ++a) cg += L->c[i][a] * G[a];
        F[i] = L->w[i] * cg / cs2;
    }
}

/* Eq. (32), equilibrium of the flow lattice (c = 1). */
static void feq2_lat(const orc_lat *L, double cs2, double rho, const double *u,
                     const double *S, double P, double *feq)
{
    int d = lat_dim(L);
    double cs4 = cs2 * cs2;
    for (int i = 0; i < L->Q; ++i) {
        double lam = (i == 0 ? (L->w[0] - 1.0) : L->w[i]) * P / cs2;
        double cu = 0.0;
        for (int a = 0; a < d; ++a) cu += L->c[i][a] * u[a];
        double diag = 0.0, off = 0.0;
        for (int a = 0; a < d; ++a) {
            double ca = L->c[i][a];
            diag += (ca * ca - cs2) * (rho * u[a] * u[a] - S[a] * u[a]);
            for (int b = a + 1; b < d; ++b) {
                double cb = L->c[i][b];
                off += ca * cb * (rho * u[a] * u[b] - 0.5 * (S[a] * u[b] + u[a] * S[b]));
            }
        }
        feq[i] = lam + L->w[i] * rho * cu / cs2 +
                 L->w[i] * (diag / (cs2 - cs4) + off / cs4);
    }
}

/* Eq. (33), forcing distribution of the flow lattice (c = 1). */
static void src2_lat(const orc_lat *L, double cs2, const double *u, const double *gradrho,
                     const double *Ftot, const double *M2F, double *F)
{
    int d = lat_dim(L);
    double cs4 = cs2 * cs2;
    double ugr = 0.0;
    for (int a = 0; a < d; ++a) ugr += u[a] * gradrho[a];
    for (int i = 0; i < L->Q; ++i) {
        double cF = 0.0, diag = 0.0, off = 0.0;
        for (int a = 0; a < d; ++a) {
            double ca = L->c[i][a];
            cF += ca * Ftot[a];
            diag += (ca * ca - cs2) * M2F[a * d + a];
            for (int b = a + 1; b < d; ++b) off += ca * L->c[i][b] * M2F[a * d + b];
        }
        F[i] = L->w[i] * (ugr + cF / cs2 + diag / (cs2 - cs4) + off / cs4);
    }
}

void orc_feq1(int kind, double d0, double phi, const double *u, double mu, double eta,
              double *feq)
{
    orc_lat L;
    lattice_setup(&L, kind, d0);
    feq1_lat(&L, d0, phi, u, mu, eta, feq);
}

void orc_src1(int kind, double d0, const double *dphiu, double *F)
{
    orc_lat L;
    lattice_setup(&L, kind, d0);
    src1_lat(&L, d0, dphiu, F);
}

void orc_feq2(int kind, double d0, double rho, const double *u, const double *S, double P,
              double *feq)
{
    orc_lat L;
    lattice_setup(&L, kind, d0);
    feq2_lat(&L, d0, rho, u, S, P, feq);
}

void orc_src2(int kind, double d0, const double *u, const double *gradrho,
              const double *Ftot, const double *M2F, double *F)
{
    orc_lat L;
    lattice_setup(&L, kind, d0);
    src2_lat(&L, d0, u, gradrho, Ftot, M2F, F);
}

/* ------------------------------------------------------------------------ */
/* finite-difference stencils (Sec. 3.2, last paragraph; reading R2)         */
/* ------------------------------------------------------------------------ */

static long wrap(long i, long n) { return ((i % n) + n) % n; }

static void fd_stencil(int dim, int *Q, int c[][3], double *w)
{
    if (dim == 2) {
        *Q = 9;
        for (int i = 0; i < 9; ++i) {
            for (int a = 0; a < 3; ++a) c[i][a] = C_D2Q9[i][a];
            w[i] = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        }
    } else {
        *Q = 19;
        for (int i = 0; i < 19; ++i) {
            for (int a = 0; a < 3; ++a) c[i][a] = C_D3Q19[i][a];
            w[i] = i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
        }
    }
}

static long nb_index(int nx, int ny, int nz, long x, long y, long z, const int *c)
{
    long xx = wrap(x + c[0], nx), yy = wrap(y + c[1], ny), zz = wrap(z + c[2], nz);
    return (zz * ny + yy) * nx + xx;
}

/* neighbour of (x, y, z) along c with the walls of reading R21: a row beyond a
 * wall is the mirror image of the row inside; *mirrored tells which */
static long nb_index_bc(const orc_sim *s, long x, long y, long z, const int *c, int *mirrored)
{
    long yy = y + c[1];
    *mirrored = 0;
    if (s->wall_y) {
        if (yy < 0) {
            yy = -1 - yy;
            *mirrored = 1;
        } else if (yy >= s->ny) {
            yy = 2L * s->ny - 1 - yy;
            *mirrored = 1;
        }
    } else {
        yy = wrap(yy, s->ny);
    }
    long xx = wrap(x + c[0], s->nx), zz = wrap(z + c[2], s->nz);
    return (zz * s->ny + yy) * s->nx + xx;
}

/* stencils of the simulation's box; parity -1: the field changes sign under
 * the wall mirror */
static void sim_grad(const orc_sim *s, const double *psi, int parity, double *grad)
{
    int Q, c[19][3];
    double w[19];
    fd_stencil(s->dim, &Q, c, w);
    const long N = s->N;
#pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < s->nz; ++z)
        for (long y = 0; y < s->ny; ++y)
            for (long x = 0; x < s->nx; ++x) {
                long id = (z * s->ny + y) * s->nx + x;
                double g[3] = {0.0, 0.0, 0.0};
                for (int i = 1; i < Q; ++i) {
                    int m;
                    double v = psi[nb_index_bc(s, x, y, z, c[i], &m)];
                    if (m && parity < 0) v = -v;
                    for (int a = 0; a < s->dim; ++a) g[a] += w[i] * c[i][a] * v;
                }
                for (int a = 0; a < s->dim; ++a) grad[a * N + id] = 3.0 * g[a];
            }
}

static void sim_lap(const orc_sim *s, const double *psi, int parity, double *lap)
{
    int Q, c[19][3];
    double w[19];
    fd_stencil(s->dim, &Q, c, w);
#pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < s->nz; ++z)
        for (long y = 0; y < s->ny; ++y)
            for (long x = 0; x < s->nx; ++x) {
                long id = (z * s->ny + y) * s->nx + x;
                double acc = 0.0;
                for (int i = 1; i < Q; ++i) {
                    int m;
                    double v = psi[nb_index_bc(s, x, y, z, c[i], &m)];
                    if (m && parity < 0) v = -v;
                    acc += w[i] * (v - psi[id]);
                }
                lap[id] = 6.0 * acc;
            }
}

void orc_grad(int dim, int nx, int ny, int nz, const double *psi, double *grad)
{
    int Q, c[19][3];
    double w[19];
    fd_stencil(dim, &Q, c, w);
    long N = (long)nx * ny * nz;
    const double inv_cs2 = 3.0;
#pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                long id = (z * ny + y) * nx + x;
                double g[3] = {0.0, 0.0, 0.0};
                for (int i = 1; i < Q; ++i) {
                    double v = psi[nb_index(nx, ny, nz, x, y, z, c[i])];
                    for (int a = 0; a < dim; ++a) g[a] += w[i] * c[i][a] * v;
                }
                for (int a = 0; a < dim; ++a) grad[a * N + id] = inv_cs2 * g[a];
            }
}

void orc_lap(int dim, int nx, int ny, int nz, const double *psi, double *lap)
{
    int Q, c[19][3];
    double w[19];
    fd_stencil(dim, &Q, c, w);
    const double two_inv_cs2 = 6.0;
#pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                long id = (z * ny + y) * nx + x;
                double acc = 0.0;
                for (int i = 1; i < Q; ++i)
                    acc += w[i] * (psi[nb_index(nx, ny, nz, x, y, z, c[i])] - psi[id]);
                lap[id] = two_inv_cs2 * acc;
            }
}

/* ------------------------------------------------------------------------ */
/* chemical potentials                                                       */
/* ------------------------------------------------------------------------ */

/* Eq. (9). */
double orc_mu_phi(const orc_params *p, double phi, double phi0, double lap_phi,
                  double lap_phi0)
{
    double s = p->sigma, D = p->D, ct = cos(p->theta_deg * M_PI / 180.0);
    return 3.0 * s / D * phi * (phi - 1.0) * (phi + 1.0) - 3.0 * D * s / 8.0 * lap_phi +
           9.0 * s / D * phi0 * phi0 * phi +
           3.0 * s * ct / D * phi0 * (3.0 * phi * phi + phi0 * phi0 - 1.0) -
           3.0 * D * s * ct / 8.0 * lap_phi0;
}

/* Eq. (19). */
double orc_mu_phi0(const orc_params *p, double phi, double phi0, double lap_phi)
{
    double s = p->sigma, D = p->D, ct = cos(p->theta_deg * M_PI / 180.0);
    return 9.0 * s / D * phi0 * phi * phi +
           3.0 * s * ct / D * phi * (3.0 * phi0 * phi0 + phi * phi - 1.0) -
           3.0 * D * s * ct / 8.0 * lap_phi;
}

/* ------------------------------------------------------------------------ */
/* particles                                                                 */
/* ------------------------------------------------------------------------ */

static void particle_geom(int dim, const orc_particle *pp, double *Vp, double *Mp, double *Ip)
{
    double R = pp->R;
    if (dim == 2) {
        *Vp = M_PI * R * R;
        *Mp = pp->rho_p * *Vp;
        *Ip = 0.5 * *Mp * R * R;
    } else {
        *Vp = 4.0 / 3.0 * M_PI * R * R * R;
        *Mp = pp->rho_p * *Vp;
        *Ip = 0.4 * *Mp * R * R;
    }
}

/* Eqs. (26a-c) with Eq. (28), first-order explicit Euler (reading R10). */
void orc_particle_update(int dim, const orc_params *p, orc_particle *pp, const double *Ff,
                         const double *Tf)
{
    double Vp, Mp, Ip;
    particle_geom(dim, pp, &Vp, &Mp, &Ip);
    double rho_bar = 0.5 * (p->rho1 + p->rho2);
    double If = Ip * rho_bar / pp->rho_p;
    double a[3], al[3];
    for (int k = 0; k < 3; ++k) {
        double Fin = rho_bar * Vp * (pp->u[k] - pp->u_prev[k]);
        double Tin = If * (pp->w[k] - pp->w_prev[k]);
        a[k] = (Ff[k] + Fin + (1.0 - rho_bar / pp->rho_p) * Mp * p->g[k]) / Mp;
        al[k] = (Tf[k] + Tin) / Ip;
    }
    if (dim == 2) {
        a[2] = 0.0;
        al[0] = al[1] = 0.0;
    }
    for (int k = 0; k < 3; ++k) {
        pp->F[k] = Ff[k];
        pp->T[k] = Tf[k];
        pp->x[k] += pp->u[k];
        pp->u_prev[k] = pp->u[k];
        pp->w_prev[k] = pp->w[k];
        /* R25: held components keep their value (bit 0: all; bits 1-3:
         * translation along x, y, z; bit 4: rotation) */
        if (!(pp->prescribed & 1) && !(pp->prescribed & (2 << k))) pp->u[k] += a[k];
        if (!(pp->prescribed & 1) && !(pp->prescribed & 16)) pp->w[k] += al[k];
    }
}

/* Readings R19 and R22: particle-particle and particle-wall repulsion of
 * Sec. 4.5 on each particle. */
void orc_repulsion(int dim, const orc_params *p, const int *n, int wall_y, int np,
                   const orc_particle *parts, double *out)
{
    for (int k = 0; k < np; ++k) {
        for (int a = 0; a < 3; ++a) out[3 * k + a] = 0.0;
        if (!(p->rep_eps > 0.0)) continue;
        /* the wall: x_k - x'_k towards the nearest imaginary particle, the
         * mirror image of particle k across the nearest wall */
        double best = INFINITY, dw[3] = {0.0, 0.0, 0.0};
        if (wall_y) {
            const double y = parts[k].x[1];
            const double d_lo = 2.0 * (y + 0.5), d_hi = 2.0 * (n[1] - 0.5 - y);
            if (d_lo < best) {
                best = d_lo;
                dw[0] = 0.0;
                dw[1] = d_lo;
            }
            if (d_hi < best) {
                best = d_hi;
                dw[0] = 0.0;
                dw[1] = -d_hi;
            }
        }
        if (dim == 2 && p->wall_circle[2] > 0.0) {
            const double ex = parts[k].x[0] - p->wall_circle[0], ey = parts[k].x[1] - p->wall_circle[1];
            const double r = sqrt(ex * ex + ey * ey);
            if (r > 0.0) {
                /* image at radius 2 R_w - r on the same ray */
                const double dd = 2.0 * fabs(p->wall_circle[2] - r);
                if (dd < best) {
                    const double s = (r - (2.0 * p->wall_circle[2] - r)) / r;
                    best = dd;
                    dw[0] = s * ex;
                    dw[1] = s * ey;
                }
            }
        }
        if (best < INFINITY) {
            const double rr = 2.0 * parts[k].R;
            double f;
            if (best > rr + p->rep_xi) f = 0.0;
            else if (best >= rr) f = (rr + p->rep_xi - best) * (rr + p->rep_xi - best) / (0.5 * p->rep_eps);
            else f = (rr - best) / (0.5 * p->rep_eps);
            for (int a = 0; a < 3; ++a) out[3 * k + a] += f * dw[a];
        }
        for (int j = 0; j < np; ++j) {
            if (j == k) continue;
            double dx[3], d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                double v = a < dim ? parts[k].x[a] - parts[j].x[a] : 0.0;
                if (a < dim && !(a == 1 && wall_y)) v -= n[a] * floor(v / n[a] + 0.5);
                dx[a] = v;
                d2 += v * v;
            }
            const double dist = sqrt(d2), rr = parts[k].R + parts[j].R;
            double f;
            if (dist > rr + p->rep_xi) f = 0.0;
            else if (dist >= rr) f = (rr + p->rep_xi - dist) * (rr + p->rep_xi - dist) / p->rep_eps;
            else f = (rr - dist) / p->rep_eps;
            for (int a = 0; a < 3; ++a) out[3 * k + a] += f * dx[a];
        }
    }
}

/* minimum-image offset x - x_p on the periodic box */
static void rel_pos(const orc_sim *s, long x, long y, long z, const double *xp, double *r)
{
    double X[3] = {(double)x, (double)y, (double)z};
    int n[3] = {s->nx, s->ny, s->nz};
    for (int a = 0; a < 3; ++a) {
        double d = X[a] - xp[a];
        if (a < s->dim && !(a == 1 && s->wall_y)) d -= n[a] * floor(d / n[a] + 0.5);
        else if (a >= s->dim) d = 0.0;
        r[a] = d;
    }
}

/* Reading R1. */
static double particle_indicator(const orc_sim *s, const orc_particle *pp, const double *r)
{
    double d2 = 0.0;
    for (int a = 0; a < s->dim; ++a) d2 += r[a] * r[a];
    return 0.5 * (1.0 + tanh(2.0 * (pp->R - sqrt(d2)) / s->p.D));
}

static void solid_velocity(const orc_particle *pp, const double *r, double *us)
{
    /* u_s = u_p + w_p x (x - x_p)  (Sec. 3.2, after Eq. 36) */
    us[0] = pp->u[0] + pp->w[1] * r[2] - pp->w[2] * r[1];
    us[1] = pp->u[1] + pp->w[2] * r[0] - pp->w[0] * r[2];
    us[2] = pp->u[2] + pp->w[0] * r[1] - pp->w[1] * r[0];
}

/* ------------------------------------------------------------------------ */
/* simulation                                                                */
/* ------------------------------------------------------------------------ */

static double *zalloc(long n) { return (double *)calloc((size_t)n, sizeof(double)); }

orc_sim *orc_create(int dim, int nx, int ny, int nz, const orc_params *p)
{
    if (dim != 2 && dim != 3) return NULL;
    if (dim == 2) nz = 1;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->dim = dim;
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->N = (long)nx * ny * nz;
    s->p = *p;
    s->cs2 = p->d0;
    s->eta = p->eta > 0.0 ? p->eta : 2.0 * p->M / s->cs2;
    /* M = (1/s_1phi - 1/2) eta cs^2 dt  (Sec. 3.1); R23: eta = 1 */
    s->s1phi = p->phase_model == 1 ? 1.0 / (p->M / s->cs2 + 0.5) : 1.0 / (p->M / (s->eta * s->cs2) + 0.5);
    s->cos_t = cos(p->theta_deg * M_PI / 180.0);
    lattice_setup(&s->L1, dim == 2 ? ORC_D2Q9 : ORC_D3Q7, p->d0);
    lattice_setup(&s->L2, dim == 2 ? ORC_D2Q9 : ORC_D3Q19, p->d0);
    long N = s->N;
    s->f1 = zalloc(s->L1.Q * N);
    s->g1 = zalloc(s->L1.Q * N);
    s->f2 = zalloc(s->L2.Q * N);
    s->g2 = zalloc(s->L2.Q * N);
    s->phi0_fixed = zalloc(N);
    s->phi0 = zalloc(N);
    s->u_prev = zalloc(3 * N);
    s->phi_prev = zalloc(N);
    s->S_prev = zalloc(3 * N);
    s->phi = zalloc(N);
    s->rho = zalloc(N);
    s->muv = zalloc(N);
    s->lap_phi = zalloc(N);
    s->lap_phi0 = zalloc(N);
    s->mu = zalloc(N);
    s->mu0 = zalloc(N);
    s->gphi = zalloc(3 * N);
    s->gphi0 = zalloc(3 * N);
    s->gmu = zalloc(3 * N);
    s->S = zalloc(3 * N);
    s->grho = zalloc(3 * N);
    s->Fc = zalloc(3 * N);
    s->F = zalloc(3 * N);
    s->ustar = zalloc(3 * N);
    s->fpen = zalloc(3 * N);
    s->u = zalloc(3 * N);
    s->Ftot = zalloc(3 * N);
    s->s2a = zalloc(N);
    s->s2b = zalloc(N);
    s->P = zalloc(N);
    s->tmp = zalloc(N);
    s->tmp3 = zalloc(3 * N);
    s->tn = zalloc(3 * N);
    s->wfld = zalloc(N);
    s->vfld = zalloc(N);
    s->lap_w = zalloc(N);
    s->gw = zalloc(3 * N);
    s->gv = zalloc(3 * N);
    return s;
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    double *bufs[] = {s->f1,  s->g1,   s->f2,   s->g2,   s->phi0_fixed, s->phi0, s->u_prev,
                      s->phi_prev, s->S_prev, s->phi, s->rho, s->muv, s->lap_phi, s->lap_phi0,
                      s->mu,  s->mu0,  s->gphi, s->gphi0, s->gmu, s->S, s->grho, s->Fc, s->F,
                      s->ustar, s->fpen, s->u, s->Ftot, s->s2a, s->s2b, s->P, s->tmp, s->tmp3,
                      s->wfld, s->vfld, s->lap_w, s->gw, s->gv, s->tn};
    for (size_t i = 0; i < sizeof(bufs) / sizeof(bufs[0]); ++i) free(bufs[i]);
    free(s);
}

static int own_angle(const orc_particle *pp) { return isfinite(pp->theta_deg) != 0; }

/* R18: does any particle carry its own contact angle */
static int any_own_angle(const orc_sim *s)
{
    for (int k = 0; k < s->np; ++k)
        if (own_angle(&s->parts[k])) return 1;
    return 0;
}

/* Step 9 of Sec. 3.3: total indicator = fixed solids + particles (reading R1);
 * with own particle angles also W and V of reading R18. */
static void update_phi0(orc_sim *s)
{
    const int own = any_own_angle(s);
#pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < s->nz; ++z)
        for (long y = 0; y < s->ny; ++y)
            for (long x = 0; x < s->nx; ++x) {
                long id = (z * s->ny + y) * s->nx + x;
                double v = s->phi0_fixed[id];
                double dflt = s->phi0_fixed[id], w = 0.0, vv = 0.0;
                for (int k = 0; k < s->np; ++k) {
                    double r[3];
                    rel_pos(s, x, y, z, s->parts[k].x, r);
                    double pk = particle_indicator(s, &s->parts[k], r);
                    v += pk;
                    if (own_angle(&s->parts[k])) {
                        double ck = cos(s->parts[k].theta_deg * M_PI / 180.0);
                        w += ck * pk;
                        vv += ck * pk * pk * pk;
                    } else {
                        dflt += pk;
                    }
                }
                s->phi0[id] = v;
                if (own) {
                    s->wfld[id] = s->cos_t * dflt + w;
                    s->vfld[id] = s->cos_t * dflt * dflt * dflt + vv;
                }
            }
}

/* Sec. 3.3 steps 3-6 (and the pieces of Eqs. 33-36 the collision needs). */
/* R23: theta n = (2/D)(1 - phi^2) grad phi / |grad phi| per cell */
static void cac_theta_n(orc_sim *s)
{
    const long N = s->N;
    for (long id = 0; id < N; ++id) {
        double g2 = 0.0;
        for (int a = 0; a < s->dim; ++a) g2 += s->gphi[a * N + id] * s->gphi[a * N + id];
        const double ph = s->phi[id];
        const double th = 2.0 / s->p.D * (1.0 - ph * ph);
        const double inv = g2 > 1e-24 ? 1.0 / sqrt(g2) : 0.0;
        for (int a = 0; a < 3; ++a) s->tn[a * N + id] = a < s->dim ? th * s->gphi[a * N + id] * inv : 0.0;
    }
}

static void compute_macros(orc_sim *s)
{
    const orc_params *p = &s->p;
    const int d = s->dim;
    const long N = s->N;
    const double cs2 = s->cs2, drho = 0.5 * (p->rho1 - p->rho2);

    update_phi0(s);

    /* step 3: phi (Eq. 31), rho (Eq. 17), viscosity (Eq. 18) */
    for (long id = 0; id < N; ++id) {
        double acc = 0.0;
        for (int i = 0; i < s->L1.Q; ++i) acc += s->f1[i * N + id];
        s->phi[id] = acc;
        s->rho[id] = drho * acc + 0.5 * (p->rho1 + p->rho2);
        s->muv[id] = 0.5 * (p->mu1 - p->mu2) * acc + 0.5 * (p->mu1 + p->mu2);
    }

    /* stencils */
    sim_lap(s, s->phi, 1, s->lap_phi);
    sim_lap(s, s->phi0, 1, s->lap_phi0);
    sim_grad(s, s->phi, 1, s->gphi);
    sim_grad(s, s->phi0, 1, s->gphi0);

    /* chemical potentials, Eqs. (9), (19) */
    const int own = any_own_angle(s);
    if (!own) {
        for (long id = 0; id < N; ++id) {
            s->mu[id] = orc_mu_phi(p, s->phi[id], s->phi0[id], s->lap_phi[id], s->lap_phi0[id]);
            s->mu0[id] = s->np > 0 ? orc_mu_phi0(p, s->phi[id], s->phi0[id], s->lap_phi[id]) : 0.0;
        }
    } else {
        /* reading R18: wetting terms per solid through W and V */
        const double sg = p->sigma, D = p->D;
        sim_lap(s, s->wfld, 1, s->lap_w);
        sim_grad(s, s->wfld, 1, s->gw);
        sim_grad(s, s->vfld, 1, s->gv);
        for (long id = 0; id < N; ++id) {
            const double ph = s->phi[id], p0 = s->phi0[id], W = s->wfld[id], V = s->vfld[id];
            s->mu[id] = 3.0 * sg / D * ph * (ph - 1.0) * (ph + 1.0) - 3.0 * D * sg / 8.0 * s->lap_phi[id] +
                        9.0 * sg / D * p0 * p0 * ph + 3.0 * sg / D * (3.0 * ph * ph * W + V - W) -
                        3.0 * D * sg / 8.0 * s->lap_w[id];
            s->mu0[id] = 0.0;
        }
    }

    /* S = M grad(mu) (rho1 - rho2)/2 (Sec. 2.2), or with R23
     * M (grad phi - theta n)(rho1 - rho2)/2; grad rho from Eq. (17) */
    sim_grad(s, s->mu, 1, s->gmu);
    if (p->phase_model == 1) cac_theta_n(s);
    for (long k = 0; k < 3 * N; ++k) {
        s->S[k] = p->phase_model == 1 ? p->M * (s->gphi[k] - s->tn[k]) * drho : p->M * s->gmu[k] * drho;
        s->grho[k] = drho * s->gphi[k];
    }

    /* F_c = div(S u - u S)/2 from the previous step's S, u (readings R5, R6):
     * F_c,b = 1/2 sum_a d_a (S_a u_b - u_a S_b). */
    for (long k = 0; k < 3 * N; ++k) s->Fc[k] = 0.0;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            if (a == b) continue;
            for (long id = 0; id < N; ++id)
                s->tmp[id] = s->S_prev[a * N + id] * s->u_prev[b * N + id] -
                             s->u_prev[a * N + id] * s->S_prev[b * N + id];
            /* S_a u_b - u_a S_b changes sign under the wall mirror when a or b is y */
            sim_grad(s, s->tmp, (a == 1 || b == 1) ? -1 : 1, s->tmp3);
            for (long id = 0; id < N; ++id) s->Fc[b * N + id] += 0.5 * s->tmp3[a * N + id];
        }

    /* F = mu grad phi + mu0 grad phi0 + F_b + F_c (Eq. 33) */
    for (int a = 0; a < 3; ++a)
        for (long id = 0; id < N; ++id) {
            long k = a * N + id;
            s->F[k] = a < d ? s->mu[id] * s->gphi[k] + s->mu0[id] * s->gphi0[k] + p->Fb[a] +
                                  s->Fc[k]
                            : 0.0;
        }
    if (own) {
        /* reading R18: sum over solids of mu_phi0,s grad phi0_s */
        const double sg = p->sigma, D = p->D;
        for (int a = 0; a < d; ++a)
            for (long id = 0; id < N; ++id) {
                long k = a * N + id;
                const double ph = s->phi[id], p0 = s->phi0[id];
                s->F[k] += 9.0 * sg / D * p0 * ph * ph * s->gphi0[k] +
                           3.0 * sg / D * (ph * (ph * ph - 1.0) * s->gw[k] + ph * s->gv[k]) -
                           3.0 * D * sg / 8.0 * s->lap_phi[id] * s->gw[k];
            }
    }

    /* steps 5-6: u* (Eq. 36a), f, u (Eq. 36b) */
#pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < s->nz; ++z)
        for (long y = 0; y < s->ny; ++y)
            for (long x = 0; x < s->nx; ++x) {
                long id = (z * s->ny + y) * s->nx + x;
                double mom[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < s->L2.Q; ++i)
                    for (int a = 0; a < d; ++a) mom[a] += s->L2.c[i][a] * s->f2[i * N + id];
                double rho = s->rho[id];
                double us_sum[3] = {0.0, 0.0, 0.0};
                for (int k = 0; k < s->np; ++k) {
                    double r[3], us[3];
                    rel_pos(s, x, y, z, s->parts[k].x, r);
                    double ph = particle_indicator(s, &s->parts[k], r);
                    solid_velocity(&s->parts[k], r, us);
                    for (int a = 0; a < 3; ++a) us_sum[a] += ph * us[a];
                }
                for (int a = 0; a < 3; ++a) {
                    long k = a * N + id;
                    if (a >= d) {
                        s->ustar[k] = s->fpen[k] = s->u[k] = s->Ftot[k] = 0.0;
                        continue;
                    }
                    s->ustar[k] = mom[a] / rho + 0.5 * s->F[k] / rho;
                    /* f = phi0 (u_s - u*) / dt, with the fixed solids at rest */
                    s->fpen[k] = us_sum[a] - s->phi0[id] * s->ustar[k];
                    s->u[k] = s->ustar[k] + 0.5 * s->fpen[k];
                    s->Ftot[k] = s->F[k] + rho * s->fpen[k];
                }
            }

    /* relaxation rates (Eq. 35, reading R8) and pressure (Eq. 36b) */
    const double w0 = s->L2.w[0];
    for (long id = 0; id < N; ++id) {
        double solid = 1.0 - s->phi0[id];
        if (solid < p->solid_eps) solid = p->solid_eps;
        double nu = s->muv[id] / (s->rho[id] * solid);
        double inv_s2a = 0.5 + nu / ((1.0 - cs2) / 2.0);
        double inv_s2b = 0.5 + nu / cs2;
        s->s2a[id] = 1.0 / inv_s2a;
        s->s2b[id] = 1.0 / inv_s2b;
        double K, H;
        if (d == 2) {
            K = 1.0 - p->d0;
            H = K * ((1.0 - p->d0) / p->s0 - (2.0 - 4.0 * p->d0) * inv_s2a +
                     (1.0 - 3.0 * p->d0) / 2.0);
        } else {
            K = 1.0 - 2.0 * p->d0;
            H = K * ((1.0 - p->d0) / p->s0 - (3.0 - 7.0 * p->d0) * inv_s2a +
                     (1.0 - 3.0 * p->d0));
        }
        double sum_f = 0.0;
        for (int i = 1; i < s->L2.Q; ++i) sum_f += s->f2[i * N + id];
        double ugr = 0.0, rus_u = 0.0, dt_rhouu = 0.0, Su = 0.0, Su_prev = 0.0;
        for (int a = 0; a < d; ++a) {
            long k = a * N + id;
            ugr += s->u[k] * s->grho[k];
            rus_u += (s->rho[id] * s->u[k] - s->S[k]) * s->u[k];
            dt_rhouu += 2.0 * s->u[k] * s->Ftot[k]; /* trace of u F + F u (R4) */
            Su += s->S[k] * s->u[k];
            Su_prev += s->S_prev[k] * s->u_prev[k];
        }
        double dt_term = dt_rhouu - (Su - Su_prev);
        s->P[id] = cs2 / (1.0 - w0) *
                   (sum_f + (0.5 + H) * ugr - w0 * rus_u / (1.0 - cs2) + K * 0.5 * dt_term);
    }
}

/* Eq. (27) for particle k using the fields of the last compute_macros. */
static void particle_force_current(orc_sim *s, int k, double *F3, double *T3)
{
    const long N = s->N;
    double Fs[3] = {0.0, 0.0, 0.0}, Ts[3] = {0.0, 0.0, 0.0};
    const orc_particle *pp = &s->parts[k];
    for (long z = 0; z < s->nz; ++z)
        for (long y = 0; y < s->ny; ++y)
            for (long x = 0; x < s->nx; ++x) {
                long id = (z * s->ny + y) * s->nx + x;
                double r[3], us[3], rf[3];
                rel_pos(s, x, y, z, pp->x, r);
                double ph = particle_indicator(s, pp, r);
                solid_velocity(pp, r, us);
                for (int a = 0; a < 3; ++a)
                    rf[a] = a < s->dim ? s->rho[id] * ph * (us[a] - s->ustar[a * N + id]) : 0.0;
                Fs[0] -= rf[0];
                Fs[1] -= rf[1];
                Fs[2] -= rf[2];
                Ts[0] -= r[1] * rf[2] - r[2] * rf[1];
                Ts[1] -= r[2] * rf[0] - r[0] * rf[2];
                Ts[2] -= r[0] * rf[1] - r[1] * rf[0];
            }
    for (int a = 0; a < 3; ++a) {
        F3[a] = Fs[a];
        T3[a] = Ts[a];
    }
}

void orc_particle_force(orc_sim *s, int k, double *F3, double *T3)
{
    compute_macros(s);
    particle_force_current(s, k, F3, T3);
}

void orc_init(orc_sim *s, const double *phi0, const double *phi, const double *u,
              const double *P)
{
    const long N = s->N;
    const orc_params *p = &s->p;
    const int d = s->dim;
    const double drho = 0.5 * (p->rho1 - p->rho2);
    memcpy(s->phi0_fixed, phi0, sizeof(double) * N);
    update_phi0(s);
    memcpy(s->phi, phi, sizeof(double) * N);
    for (long k = 0; k < 3 * N; ++k) s->u[k] = (u && k < d * N) ? u[k] : 0.0;
    for (long id = 0; id < N; ++id) {
        s->P[id] = P ? P[id] : 0.0;
        s->rho[id] = drho * phi[id] + 0.5 * (p->rho1 + p->rho2);
    }
    sim_lap(s, s->phi, 1, s->lap_phi);
    sim_lap(s, s->phi0, 1, s->lap_phi0);
    if (!any_own_angle(s)) {
        for (long id = 0; id < N; ++id)
            s->mu[id] = orc_mu_phi(p, s->phi[id], s->phi0[id], s->lap_phi[id], s->lap_phi0[id]);
    } else {
        /* reading R18, as in the steps */
        const double sg = p->sigma, D = p->D;
        sim_lap(s, s->wfld, 1, s->lap_w);
        for (long id = 0; id < N; ++id) {
            const double ph = s->phi[id], p0 = s->phi0[id], W = s->wfld[id], V = s->vfld[id];
            s->mu[id] = 3.0 * sg / D * ph * (ph - 1.0) * (ph + 1.0) - 3.0 * D * sg / 8.0 * s->lap_phi[id] +
                        9.0 * sg / D * p0 * p0 * ph + 3.0 * sg / D * (3.0 * ph * ph * W + V - W) -
                        3.0 * D * sg / 8.0 * s->lap_w[id];
        }
    }
    sim_grad(s, s->mu, 1, s->gmu);
    if (p->phase_model == 1) {
        sim_grad(s, s->phi, 1, s->gphi);
        cac_theta_n(s);
    }
    for (long k = 0; k < 3 * N; ++k)
        s->S[k] = p->phase_model == 1 ? p->M * (s->gphi[k] - s->tn[k]) * drho : p->M * s->gmu[k] * drho;
    /* step 1 of Sec. 3.3: f = f^eq */
    for (long id = 0; id < N; ++id) {
        double uu[3], SS[3], fe[ORC_QMAX];
        for (int a = 0; a < 3; ++a) {
            uu[a] = s->u[a * N + id];
            SS[a] = s->S[a * N + id];
        }
        if (p->phase_model == 1)
            feq1_lat(&s->L1, s->cs2, s->phi[id], uu, s->phi[id], 1.0, fe);
        else
            feq1_lat(&s->L1, s->cs2, s->phi[id], uu, s->mu[id], s->eta, fe);
        for (int i = 0; i < s->L1.Q; ++i) s->f1[i * N + id] = fe[i];
        feq2_lat(&s->L2, s->cs2, s->rho[id], uu, SS, s->P[id], fe);
        for (int i = 0; i < s->L2.Q; ++i) s->f2[i * N + id] = fe[i];
    }
    /* previous-step values equal the initial ones (reading R5) */
    memcpy(s->u_prev, s->u, sizeof(double) * 3 * N);
    memcpy(s->S_prev, s->S, sizeof(double) * 3 * N);
    memcpy(s->phi_prev, s->phi, sizeof(double) * N);
}

/* One time step: Sec. 3.3 steps 3-10 followed by step 2 of the next pass,
 * arranged as macros -> collision (Eq. 29) -> streaming -> particle update. */
static void one_step(orc_sim *s)
{
    const long N = s->N;
    const int d = s->dim;
    const orc_params *p = &s->p;
    const double cs2 = s->cs2;

    compute_macros(s);

    /* step 7: hydrodynamic force and torque, Eq. (27) */
    double Ff[ORC_MAXP][3], Tf[ORC_MAXP][3];
    for (int k = 0; k < s->np; ++k) particle_force_current(s, k, Ff[k], Tf[k]);

    /* collision, Eq. (29) with Lambda of Eq. (37) */
#pragma omp parallel for schedule(static)
    for (long id = 0; id < N; ++id) {
        double uu[3], SS[3], Sp[3], up[3], gr[3], Ft[3];
        for (int a = 0; a < 3; ++a) {
            uu[a] = s->u[a * N + id];
            SS[a] = s->S[a * N + id];
            Sp[a] = s->S_prev[a * N + id];
            up[a] = s->u_prev[a * N + id];
            gr[a] = s->grho[a * N + id];
            Ft[a] = s->Ftot[a * N + id];
        }
        double phi = s->phi[id], rho = s->rho[id];

        /* order-parameter lattice */
        double f[ORC_QMAX], fe[ORC_QMAX], Fs[ORC_QMAX], v[ORC_QMAX], Lv[ORC_QMAX],
            LF[ORC_QMAX], S1[ORC_QMAX], G[3];
        int Q1 = s->L1.Q;
        for (int i = 0; i < Q1; ++i) f[i] = s->f1[i * N + id];
        const int cac = p->phase_model == 1;
        /* R23: eta mu -> phi, and the sharpening flux cs^2 theta n in G */
        feq1_lat(&s->L1, cs2, phi, uu, cac ? phi : s->mu[id], cac ? 1.0 : s->eta, fe);
        for (int a = 0; a < 3; ++a)
            G[a] = phi * uu[a] - s->phi_prev[id] * up[a] + (cac ? cs2 * s->tn[a * N + id] : 0.0);
        src1_lat(&s->L1, cs2, G, Fs);
        orc_rates(s->L1.kind, 1, p->s0, s->s1phi, p->s2, p->s2, p->s3, p->s4, S1);
        for (int i = 0; i < Q1; ++i) v[i] = f[i] - fe[i];
        apply_lambda(&s->L1, S1, v, Lv);
        apply_lambda(&s->L1, S1, Fs, LF);
        for (int i = 0; i < Q1; ++i) s->f1[i * N + id] = f[i] - Lv[i] + Fs[i] - 0.5 * LF[i];

        /* flow lattice */
        double M2F[9], S2[ORC_QMAX];
        int Q2 = s->L2.Q;
        double ugr = 0.0;
        for (int a = 0; a < d; ++a) ugr += uu[a] * gr[a];
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                /* Eq. (34) with d_t(rho u u) ~ u F + F u (R4) and explicit Euler (R5) */
                double dt_ruu = uu[a] * Ft[b] + Ft[a] * uu[b];
                double dt_Su = 0.5 * ((SS[a] * uu[b] + uu[a] * SS[b]) -
                                      (Sp[a] * up[b] + up[a] * Sp[b]));
                M2F[a * d + b] = dt_ruu - dt_Su + cs2 * (uu[a] * gr[b] + gr[a] * uu[b]) +
                                 (a == b ? (1.0 - 3.0 * cs2) * ugr : 0.0);
            }
        for (int i = 0; i < Q2; ++i) f[i] = s->f2[i * N + id];
        feq2_lat(&s->L2, cs2, rho, uu, SS, s->P[id], fe);
        src2_lat(&s->L2, cs2, uu, gr, Ft, M2F, Fs);
        orc_rates(s->L2.kind, 2, p->s0, p->s1, s->s2a[id], s->s2b[id], p->s3, p->s4, S2);
        for (int i = 0; i < Q2; ++i) v[i] = f[i] - fe[i];
        apply_lambda(&s->L2, S2, v, Lv);
        apply_lambda(&s->L2, S2, Fs, LF);
        for (int i = 0; i < Q2; ++i) s->f2[i * N + id] = f[i] - Lv[i] + Fs[i] - 0.5 * LF[i];
    }

    /* streaming, left-hand side of Eq. (29): periodic box, or (reading R21)
     * halfway bounce-back where a population would cross a wall */
    for (int lat = 0; lat < 2; ++lat) {
        const orc_lat *L = lat == 0 ? &s->L1 : &s->L2;
        double *src = lat == 0 ? s->f1 : s->f2;
        double *dst = lat == 0 ? s->g1 : s->g2;
        int opp[ORC_QMAX];
        for (int i = 0; i < L->Q; ++i)
            for (int j = 0; j < L->Q; ++j)
                if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2])
                    opp[i] = j;
#pragma omp parallel for collapse(2) schedule(static)
        for (long z = 0; z < s->nz; ++z)
            for (long y = 0; y < s->ny; ++y)
                for (long x = 0; x < s->nx; ++x) {
                    long id = (z * s->ny + y) * s->nx + x;
                    for (int i = 0; i < L->Q; ++i) {
                        const long yd = y + L->c[i][1];
                        if (s->wall_y && (yd < 0 || yd >= s->ny))
                            dst[opp[i] * N + id] = src[i * N + id];
                        else
                            dst[i * N + nb_index(s->nx, s->ny, s->nz, x, y, z, L->c[i])] = src[i * N + id];
                    }
                }
    }
    double *t1 = s->f1, *t2 = s->f2;
    s->f1 = s->g1;
    s->g1 = t1;
    s->f2 = s->g2;
    s->g2 = t2;

    /* previous-step values for the explicit time derivatives (R5) */
    memcpy(s->u_prev, s->u, sizeof(double) * 3 * N);
    memcpy(s->S_prev, s->S, sizeof(double) * 3 * N);
    memcpy(s->phi_prev, s->phi, sizeof(double) * N);

    /* steps 8-10: particle update (hydrodynamic force plus the repulsion of
     * reading R19 from the positions before the update); the indicator follows
     * at the next pass */
    double Frep[ORC_MAXP * 3];
    const int nn[3] = {s->nx, s->ny, s->nz};
    orc_repulsion(d, p, nn, s->wall_y, s->np, s->parts, Frep);
    for (int k = 0; k < s->np; ++k) {
        double Fk[3];
        for (int a = 0; a < 3; ++a) Fk[a] = Ff[k][a] + Frep[3 * k + a];
        orc_particle_update(d, p, &s->parts[k], Fk, Tf[k]);
        for (int a = 0; a < 3; ++a) s->parts[k].F[a] = Ff[k][a];
    }
}

void orc_step(orc_sim *s, long n)
{
    for (long t = 0; t < n; ++t) one_step(s);
}

void orc_macros(orc_sim *s, double *phi, double *rho, double *u, double *P, double *mu)
{
    const long N = s->N;
    compute_macros(s);
    if (phi) memcpy(phi, s->phi, sizeof(double) * N);
    if (rho) memcpy(rho, s->rho, sizeof(double) * N);
    if (u) memcpy(u, s->u, sizeof(double) * s->dim * N);
    if (P) memcpy(P, s->P, sizeof(double) * N);
    if (mu) memcpy(mu, s->mu, sizeof(double) * N);
}

void orc_normal(orc_sim *s, double *n)
{
    const long N = s->N;
    compute_macros(s);
    for (long id = 0; id < N; ++id) {
        double g2 = 0.0;
        for (int a = 0; a < s->dim; ++a) g2 += s->gphi[a * N + id] * s->gphi[a * N + id];
        const double inv = g2 > 1e-24 ? 1.0 / sqrt(g2) : 0.0;
        for (int a = 0; a < s->dim; ++a) n[a * N + id] = s->gphi[a * N + id] * inv;
    }
}

void orc_get_f(orc_sim *s, double *f1, double *f2)
{
    if (f1) memcpy(f1, s->f1, sizeof(double) * s->L1.Q * s->N);
    if (f2) memcpy(f2, s->f2, sizeof(double) * s->L2.Q * s->N);
}

void orc_get_phi0(orc_sim *s, double *phi0)
{
    update_phi0(s);
    memcpy(phi0, s->phi0, sizeof(double) * s->N);
}

/* Free energy of Eq. (8) and kinetic energy rho u^2/2 (Sec. 2.3), summed over
 * cells (dx = 1) in a fixed serial order. */
void orc_diagnostics(orc_sim *s, double *out4)
{
    const long N = s->N;
    const int d = s->dim;
    const orc_params *p = &s->p;
    compute_macros(s);
    double sg = p->sigma, D = p->D, ct = s->cos_t;
    const int own = any_own_angle(s);
    double mass = 0.0, EF = 0.0, EK = 0.0;
    for (long id = 0; id < N; ++id) {
        double ph = s->phi[id], p0 = s->phi0[id];
        double g2 = 0.0, g0g = 0.0, gwg = 0.0, u2 = 0.0;
        for (int a = 0; a < d; ++a) {
            g2 += s->gphi[a * N + id] * s->gphi[a * N + id];
            g0g += s->gphi0[a * N + id] * s->gphi[a * N + id];
            if (own) gwg += s->gw[a * N + id] * s->gphi[a * N + id];
            u2 += s->u[a * N + id] * s->u[a * N + id];
        }
        double e = 3.0 * sg / (4.0 * D) * (1.0 - ph) * (1.0 - ph) * (1.0 + ph) * (1.0 + ph) +
                   3.0 * D * sg / 16.0 * g2 + 9.0 * sg / (2.0 * D) * p0 * p0 * ph * ph;
        if (!own)
            e += 3.0 * sg * ct / D * p0 * ph * (ph * ph + p0 * p0 - 1.0) + 3.0 * D * sg * ct / 8.0 * g0g;
        else  /* reading R18: sum over solids with their own angles */
            e += 3.0 * sg / D * (ph * (ph * ph - 1.0) * s->wfld[id] + ph * s->vfld[id]) +
                 3.0 * D * sg / 8.0 * gwg;
        mass += ph;
        EF += e;
        EK += 0.5 * s->rho[id] * u2;
    }
    out4[0] = mass;
    out4[1] = EF;
    out4[2] = EK;
    out4[3] = EF + EK;
}

int orc_set_particle(orc_sim *s, int k, const orc_particle *pp)
{
    if (k < 0 || k > s->np || k >= ORC_MAXP) return -1;
    s->parts[k] = *pp;
    for (int a = 0; a < 3; ++a) {
        s->parts[k].u_prev[a] = pp->u[a];
        s->parts[k].w_prev[a] = pp->w[a];
    }
    if (k == s->np) s->np++;
    return 0;
}

int orc_get_particle(orc_sim *s, int k, orc_particle *pp)
{
    if (k < 0 || k >= s->np) return -1;
    *pp = s->parts[k];
    return 0;
}

int orc_num_particles(orc_sim *s) { return s->np; }

int orc_set_walls(orc_sim *s, int wall_y)
{
    s->wall_y = wall_y ? 1 : 0;
    return 0;
}
