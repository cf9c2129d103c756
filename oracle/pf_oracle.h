/*
 * FP64 CPU oracle for the conservative phase-field / consistent Navier-Stokes
 * lattice Boltzmann method of Zhan, Liu, Chai & Shi, "A thermodynamically
 * consistent and conservative diffuse-interface model for gas-liquid-solid
 * multiphase flows" (arXiv 2311.05097).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, plain reference that the
 * CUDA library is checked against.  Nothing in the product path may link,
 * load or call it.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Everything is double precision, plain loops, one full-grid pass per stage,
 * and the collision is applied with the dense matrices
 * Lambda = M_H^-1 S_H M_H of Eq. (37) built from the printed M_0 and N_H of
 * Eq. (38) (2D) or from tensor Hermite polynomials (3D, see pf_oracle.c).
 */
#ifndef PF_ORACLE_H
#define PF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_params {
    double sigma;      /* sigma_12, surface tension (Eq. 1) */
    double D;          /* interface width (Eq. 1) */
    double M;          /* mobility (Eq. 2) */
    double eta;        /* eta of Eq. (30); <= 0 selects 2M/cs^2 (s_1phi = 1) */
    double rho1, rho2; /* Eq. (17) */
    double mu1, mu2;   /* Eq. (18) */
    double d0;         /* cs^2/c^2 (Sec. 3.2) */
    double s0, s1, s2, s3, s4; /* relaxation rates of S_H (Eq. 38) */
    double theta_deg;  /* contact angle (Young's law, Eq. 8) */
    double Fb[3];      /* body force on the fluid (Eq. 16b) */
    double g[3];       /* gravity acting on particles (Eq. 26a) */
    double solid_eps;  /* lower bound on 1 - phi0 in the viscosity (reading of Eq. 35) */
    double rep_xi;     /* particle-particle repulsion range xi (Sec. 4.5) */
    double rep_eps;    /* its stiffness epsilon; <= 0 switches the repulsion off */
    double wall_circle[3]; /* circular wall (centre x, y; radius) seen by the
                              particle-wall repulsion (reading R22); radius <= 0:
                              none */
    int phase_model;   /* 0: Cahn-Hilliard order parameter (Eq. 2, Sec. 3.1);
                          1: conservative Allen-Cahn (reading R23) */
} orc_params;

typedef struct orc_particle {
    double x[3], u[3], w[3];      /* centre, velocity, angular velocity */
    double R, rho_p;              /* radius, density */
    double u_prev[3], w_prev[3];  /* previous-step velocities (Eq. 28) */
    double F[3], T[3];            /* last hydrodynamic force / torque (Eq. 27) */
    double theta_deg;             /* own contact angle (Sec. 4.5), NaN = the simulation's */
    int prescribed;               /* bit flags of held motion (reading R25): 1 all of u and
                                     w kept (prescribed motion); 2, 4, 8 the x, y, z
                                     translation; 16 the rotation; x advances by u */
} orc_particle;

typedef struct orc_sim orc_sim;

/* lattice kinds */
enum { ORC_D2Q9 = 0, ORC_D3Q19 = 1, ORC_D3Q7 = 2 };

orc_sim *orc_create(int dim, int nx, int ny, int nz, const orc_params *p);
void orc_destroy(orc_sim *s);
int orc_num_threads(void);

/* Step 1 of Sec. 3.3: f = f^eq from the initial fields. u and P may be NULL
 * (zero).  Arrays are x-fastest, N = nx*ny*nz; u is component-major (u_x[N],
 * u_y[N], u_z[N]). */
void orc_init(orc_sim *s, const double *phi0, const double *phi,
              const double *u, const double *P);
void orc_step(orc_sim *s, long n);
/* Macroscopic fields at the current time, recomputed from f (Sec. 3.3,
 * steps 3-6).  NULL outputs are skipped. */
void orc_macros(orc_sim *s, double *phi, double *rho, double *u, double *P,
                double *mu);
/* out = {mass, E_F, E_K, E_total} (Eq. 8 and Sec. 2.3). */
void orc_diagnostics(orc_sim *s, double *out4);
/* Distribution functions at the current time (pre-collision), Q*N each. */
void orc_get_f(orc_sim *s, double *f1, double *f2);
/* Particles (Sec. 2.4): add or overwrite particle k (k == count appends). */
int orc_set_particle(orc_sim *s, int k, const orc_particle *pp);
int orc_get_particle(orc_sim *s, int k, orc_particle *pp);
int orc_num_particles(orc_sim *s);
/* Reading R21: walls at y = -1/2 and y = ny - 1/2 (2D and 3D; before init). */
int orc_set_walls(orc_sim *s, int wall_y);
/* Interface normal grad phi / |grad phi| at the current time (dim x N; 0 where
 * |grad phi|^2 <= 1e-24), central stencil with the walls of reading R21. */
void orc_normal(orc_sim *s, double *n);
/* The total solid indicator phi0 at the current time. */
void orc_get_phi0(orc_sim *s, double *phi0);

/* ---- per-cell building blocks, exposed for the oracle's own pins ---- */
/* Lattice tables: c (Q x 3 ints), w (Q), MH (Q x Q, row-major). Returns Q. */
int orc_lattice(int kind, double d0, int *c, double *w, double *MH);
/* Eq. (30): equilibrium of the order-parameter lattice and its source. */
void orc_feq1(int kind, double d0, double phi, const double *u, double mu,
              double eta, double *feq);
void orc_src1(int kind, double d0, const double *dphiu, double *F);
/* Eq. (32): equilibrium of the flow lattice. */
void orc_feq2(int kind, double d0, double rho, const double *u,
              const double *S, double P, double *feq);
/* Eq. (33): forcing distribution of the flow lattice; M2F is d x d row-major. */
void orc_src2(int kind, double d0, const double *u, const double *gradrho,
              const double *Ftot, const double *M2F, double *F);
/* Dense Lambda = M_H^-1 diag(S) M_H (Eq. 37), Q x Q row-major. */
void orc_lambda(int kind, double d0, const double *S, double *Lam);
/* Relaxation vectors of Eq. (38) (and the 3D analogue) for lattice k. */
void orc_rates(int kind, int k, double s0, double s1, double s2a, double s2b,
               double s3, double s4, double *S);
/* Isotropic central stencils (Sec. 3.2 last paragraph) applied on a periodic
 * grid: grad is component-major d*N, lap is N. */
void orc_grad(int dim, int nx, int ny, int nz, const double *psi, double *grad);
void orc_lap(int dim, int nx, int ny, int nz, const double *psi, double *lap);
/* Eq. (9) and Eq. (19) pointwise. */
double orc_mu_phi(const orc_params *p, double phi, double phi0, double lap_phi,
                  double lap_phi0);
double orc_mu_phi0(const orc_params *p, double phi, double phi0, double lap_phi);
/* Newton-Euler update of one particle (Eqs. 26, 28) given F_f, T_f (Eq. 27). */
void orc_particle_update(int dim, const orc_params *p, orc_particle *pp,
                         const double *Ff, const double *Tf);
/* Hydrodynamic force and torque on particle k (Eq. 27) at the current time. */
void orc_particle_force(orc_sim *s, int k, double *F3, double *T3);
/* Short-range repulsion of Sec. 4.5 on each of np particles: from the other
 * particles (minimum image along periodic axes; wall_y: y is bounded by walls
 * at -1/2 and n[1] - 1/2) plus, from the nearest wall (the box walls when
 * wall_y, the circle p->wall_circle), the particle-wall term (reading R22);
 * out is np x 3. */
void orc_repulsion(int dim, const orc_params *p, const int *n, int wall_y, int np,
                   const orc_particle *parts, double *out);

#ifdef __cplusplus
}
#endif
#endif
