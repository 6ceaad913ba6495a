/*
 * sph_oracle.h -- plain FP64 CPU oracle of the weakly compressible SPH
 * (WCSPH) per-step hot path of the DualSPHysics paper (arXiv 2104.00537).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The GPU product path
 * never links, loads or calls it, and it shares no code with the GPU path.
 *
 * Every routine works in double precision on absolute positions, in the
 * paper's notation: particle sets P = F (fluid) u B (boundary), Sect. 2.1.
 * All arrays are caller-owned; nothing here allocates memory that outlives
 * a call.  Functions return 0 on success and a negative value on bad input.
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H
#include <stdint.h>

typedef struct {
  double dp;        /* initial inter-particle spacing; m = rho0 * dp^3     */
  double h;         /* smoothing length, Eq 2                               */
  double rho0;      /* reference density, Eq 28                             */
  double cs0;       /* numerical speed of sound, Eq 28                      */
  double gamma;     /* polytropic index, Eq 28                              */
  double alpha;     /* artificial viscosity coefficient, Eq 21              */
  double delta;     /* density diffusion coefficient, Eq 17                 */
  double cfl;       /* Courant number C_CFL, Eq 35                          */
  double eta2;      /* eta^2 regulariser of Eq 21 and Eq 35                 */
  double g[3];      /* body force f (gravity), Eq 13                        */
  double dmin[3];   /* domain box: particles outside leave the simulation   */
  double dmax[3];
  double dt_fixed;  /* > 0: use this time step instead of Eq 35             */
  int32_t cell_mode;          /* 0: cells of 2h (Sect. 5.1); 1: of h; 2: of 2h/3 */
  int32_t ddt_mode;           /* 0: no density diffusion; 1: Eq 17 + Eq 18;
                               * 2: Eq 17 + Eq 19-20 (dynamic density)     */
  int32_t clamp_boundary_rho; /* 1: boundary density kept >= rho0          */
  int32_t visc_mode;          /* 0: artificial viscosity, Eq 21-22;
                               * 1: laminar viscosity + SPS, Eq 23-27      */
  double nu0;                 /* kinematic viscosity of Eq 23 (m^2/s)      */
  int32_t boundary_mode;      /* 0: DBC, Eq 36; 1: mDBC, Eq 38-39          */
  int32_t mdbc_slip;          /* mDBC velocity of B: 0 the imposed one (Eq 37);
                               * 1 no-slip, 2 v_wall - v_G; 2 free-slip:
                               * tangential part of v_G, normal part of
                               * 2 v_wall - v_G (normal = ghost direction)  */
} orc_params;

/* mDBC: |det| of the corrected-SPH moment matrix below which the ghost node
 * falls back to the Shepard value (Eq 39 form) with a zero gradient. */
#define ORC_MDBC_DET_MIN 1e-3

/* SPS constants of Eq 25: Smagorinsky C_S and C_l; Delta = dp. */
#define ORC_SPS_CS 0.12
#define ORC_SPS_CL 0.0066

/* Imposed sinusoidal translation of a group of boundary particles (Eq 37):
 * displacement D(t) = amp * (sin(omega t + phase) - sin(phase)) along axis. */
typedef struct {
  double axis[3];
  double amp, omega, phase;
} orc_motion;

/* Kernel (Eq 11, 3-D) and the factor F with grad_a W_ab = F(r) * r_ab. */
double orc_wendland_w(double r, double h);
double orc_wendland_gradfac(double r, double h);
/* Tait equation of state, Eq 28. */
double orc_tait(const orc_params *p, double rho);
/* SPS stress of Eq 25 divided by rho, for fluid particle a, from the SPH
 * velocity gradient over its neighbours b in P (Eq 24-25):
 * out = {xx, yy, zz, xy, xz, yz}.  Zero for boundary and frozen particles. */
int orc_sps_tau(const orc_params *p, int64_t n, const double *pos, const double *vel,
                const double *rho, const uint8_t *type, const uint8_t *out, double *tau6);

/* mDBC (Sect. 2.6.2, Eq 38-39): for every in-domain boundary particle B,
 * the ghost node r_G = r_B + ghost[B] (mirror image of B across the wall
 * surface), the corrected SPH estimate (first-order consistent moment
 * equations over b in F) of rho_G and grad rho_G, rho_B = rho_G +
 * (r_B - r_G) . grad rho_G (Eq 38), and v_G by the Shepard sum of Eq 39.
 * Writes rho[B] (not clamped: clamp_boundary_rho applies to Eq 36) and, with
 * mdbc_slip 1 or 2, vel[B] from v_G and B's imposed velocity v_wall at time
 * t (Eq 37; zero for fixed walls).  Without fluid in the ghost's support
 * rho_B = rho0 and v_B = v_wall.  dets (optional, [n]) receives the moment
 * matrix determinant of every boundary particle (0 for the others). */
int orc_mdbc(const orc_params *p, const orc_motion *motions, int32_t nmot, int64_t n,
             const double *pos, double *vel, double *rho, const uint8_t *type,
             const int32_t *group, const uint8_t *out, const double *ghost, double t,
             double *dets);

/* Hydrostatic density difference of Eq 19: the density that Eq 28, solved
 * for rho, gives at the pressure P^H_ab = rho0 g z_ab of Eq 20, minus rho0.
 * With a gravity vector g, rho0 g z_ab reads -rho0 (g . r_ab), which is
 * rho0 |g| (z_a - z_b) when g points down z. */
double orc_rho_hydro(const orc_params *p, const double rab[3]);

/* Cell grid: origin, cell size, cell counts and margin (in cells). */
int orc_grid(const orc_params *p, double origin[3], double *cs, int64_t nc[3],
             int32_t *margin);
/* Linear cell id of each particle, -1 if outside the domain. */
int orc_cells(const orc_params *p, int64_t n, const double *pos, int64_t *cell);
/* Neighbour-list order: stable sort of prev_order by (is_boundary, cell):
 * fluid particles by cell, then boundary particles by cell, out-of-domain
 * particles last.  Returns the number of in-domain particles. */
int64_t orc_sort(const orc_params *p, int64_t n, const double *pos,
                 const uint8_t *type, const uint8_t *out,
                 const int64_t *prev_order, int64_t *order);

/* Ordered neighbour pairs (a, b), a != b, 0 < |r_ab|^2 < (2h)^2 among the
 * in-domain particles, found by brute force (use_cells = 0) or by the cell
 * list (use_cells = 1).  Per-particle count and an order-independent hash of
 * the neighbour ids.  If pairs != NULL, up to cap pairs are stored sorted. */
int64_t orc_pairs(const orc_params *p, int64_t n, const double *pos,
                  const uint8_t *out, int use_cells, int64_t *count,
                  uint64_t *hash, int64_t *pairs, int64_t cap);

/* One evaluation of the particle interaction (PI): for a in F, dv/dt of
 * Eq 22 plus f and drho/dt of Eq 15 (with D_a of Eq 17-18); for a in B,
 * drho/dt of Eq 36; mumax_a = max_b |h v_ab.r_ab| / (r^2 + eta^2) (Eq 35).
 * Returns the number of evaluated ordered pairs. */
int64_t orc_interact(const orc_params *p, int64_t n, const double *pos,
                     const double *vel, const double *rho, const uint8_t *type,
                     const uint8_t *out, int use_cells, double *acc,
                     double *drho, double *mumax);

/* The same evaluation restricted to the particles a in [a0, a1) (their
 * neighbours range over all particles); outputs of other particles are not
 * written.  Used to time bounded samples of a large case. */
int64_t orc_interact_range(const orc_params *p, int64_t n, const double *pos,
                           const double *vel, const double *rho,
                           const uint8_t *type, const uint8_t *out,
                           int use_cells, int64_t a0, int64_t a1, double *acc,
                           double *drho, double *mumax);

/* Variable time step, Eq 35. */
double orc_dt(const orc_params *p, int64_t n, const double *acc,
              const double *mumax, const uint8_t *type, const uint8_t *out);

/* nsteps Symplectic steps (Eq 33-34) with the time step of Eq 35 and the
 * boundary conditions of Eq 36-37.  group[a] >= 0 selects a motion for a
 * boundary particle, -1 keeps it fixed.  order carries the neighbour-list
 * order from step to step.  Returns the number of evaluated pairs. */
int64_t orc_step(const orc_params *p, const orc_motion *motions, int32_t nmot,
                 int64_t n, double *pos, double *vel, double *rho,
                 const uint8_t *type, const int32_t *group, uint8_t *out,
                 int64_t *order, double *t, double *last_dt, int64_t nsteps,
                 const double *ghost);

/* nsteps Verlet steps (Eq 30, with the Eq 31 step whenever the count of
 * completed steps *step is a multiple of ns; so the first step, which has
 * no state n-1, is an Eq 31 step).  vel_prev / rho_prev hold v^{n-1} and
 * rho^{n-1} and are updated with the state.  One PI per step, the time step
 * of Eq 35 from it, boundary conditions as in orc_step.  Returns the number
 * of evaluated pairs. */
int64_t orc_step_verlet(const orc_params *p, const orc_motion *motions, int32_t nmot,
                        int64_t n, double *pos, double *vel, double *rho,
                        double *vel_prev, double *rho_prev, const uint8_t *type,
                        const int32_t *group, uint8_t *out, int64_t *order, double *t,
                        double *last_dt, int64_t *step, int32_t ns, int64_t nsteps,
                        const double *ghost);

/* Diagnostics: res = {total mass, fluid kinetic energy, fluid momentum x, y,
 * z, front (max x of in-domain fluid), number out of domain}. */
int orc_diag(const orc_params *p, int64_t n, const double *pos,
             const double *vel, const uint8_t *type, const uint8_t *out,
             double res[7]);

#endif
