/*
 * sph_oracle.c -- plain FP64 CPU oracle of the WCSPH per-step hot path of
 * the DualSPHysics paper (arXiv 2104.00537): neighbour list (Sect. 5.1),
 * particle interaction (Eq 11, 15-18, 21-22, 28, 36), time step (Eq 35)
 * and Symplectic update (Eq 33-34, 37).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no
 * code with the GPU path.  It is written to be checked against the paper by
 * eye: absolute FP64 positions, one loop per particle, no blocking, no
 * fusion beyond what the equations state.
 *
 * Readings of the paper taken here (each also used by the GPU path):
 *  - grad_a W_ab = -(5 a_D / h^2) (1 - q/2)^3 r_ab, the derivative of Eq 11
 *    with a_D = 21 / (16 pi h^3) (3-D).
 *  - a pair interacts iff 0 < |r_ab|^2 < (2h)^2 (Eq 4 with k = 2).
 *  - the bar of Eq 21 is the mean; c-bar = cs0; rho-bar = (rho_a+rho_b)/2.
 *  - Eq 18 is applied in its diffusive orientation: psi_ab . grad_a W_ab =
 *    -2 (rho_b - rho_a) F, so D_a > 0 when the neighbours are denser.
 *  - V_b = m_b / rho_b; all particles have m = rho0 dp^3.
 *  - the neighbour list is rebuilt before both interaction evaluations of a
 *    Symplectic step; the step size comes from the first evaluation.
 *  - neighbour-list order: fluid particles sorted by cell, then boundary
 *    particles sorted by cell, ties in the previous order (Sect. 5.1 only
 *    says particles are sorted by the cell they belong to).
 *  - |f_a| in Eq 35 is the full fluid acceleration (gravity included) and
 *    Eq 35's v.r is v_ab.r_ab over the same neighbours as the interaction.
 *  - boundary density is clamped to >= rho0 after each update (optional).
 *  - a particle whose position leaves the domain is frozen and excluded.
 */
#include "sph_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---- kernel and equation of state ------------------------------------ */

/* Eq 11, 3-D: W = a_D (1 - q/2)^4 (2q + 1) for 0 <= q <= 2. */
double orc_wendland_w(double r, double h) {
  double q = r / h;
  if (q >= 2.0) return 0.0;
  double aD = 21.0 / (16.0 * M_PI * h * h * h);
  double t = 1.0 - 0.5 * q;
  return aD * t * t * t * t * (2.0 * q + 1.0);
}

/* dW/dr / r, so that grad_a W_ab = F * r_ab (r_ab = r_a - r_b). */
double orc_wendland_gradfac(double r, double h) {
  double q = r / h;
  if (q >= 2.0) return 0.0;
  double aD = 21.0 / (16.0 * M_PI * h * h * h);
  double t = 1.0 - 0.5 * q;
  return -5.0 * aD / (h * h) * t * t * t;
}

/* Eq 28: P = (cs0^2 rho0 / gamma) ((rho/rho0)^gamma - 1). */
double orc_tait(const orc_params *p, double rho) {
  double B = p->cs0 * p->cs0 * p->rho0 / p->gamma;
  return B * (pow(rho / p->rho0, p->gamma) - 1.0);
}

double orc_rho_hydro(const orc_params *p, const double rab[3]) {
  double B = p->cs0 * p->cs0 * p->rho0 / p->gamma;
  double PH = -p->rho0 * (p->g[0] * rab[0] + p->g[1] * rab[1] + p->g[2] * rab[2]);
  return p->rho0 * pow(1.0 + PH / B, 1.0 / p->gamma) - p->rho0;
}

/* ---- grid and neighbour list (Sect. 5.1) ------------------------------ */

int orc_grid(const orc_params *p, double origin[3], double *cs, int64_t nc[3],
             int32_t *margin) {
  if (!(p->h > 0.0)) return -1;
  if (p->cell_mode < 0 || p->cell_mode > 2) return -1;
  int32_t m = p->cell_mode + 1; /* cells needed to cover 2h */
  double c = 2.0 * p->h / m;    /* cells of 2h, h or 2h/3 */
  for (int k = 0; k < 3; k++) {
    if (!(p->dmax[k] > p->dmin[k])) return -1;
    origin[k] = p->dmin[k] - m * c;
    nc[k] = 2 * m + (int64_t)ceil((p->dmax[k] - p->dmin[k]) / c);
  }
  *cs = c;
  *margin = m;
  return 0;
}

/* Integer cell coordinates of a position; returns 1 if inside the domain,
 * i.e. every coordinate in [margin, nc - margin). */
static int cell_coords(const double *origin, double cs, const int64_t *nc,
                       int32_t margin, const double *r, int64_t c[3]) {
  int inside = 1;
  for (int k = 0; k < 3; k++) {
    double f = floor((r[k] - origin[k]) / cs);
    if (!(f >= margin && f < nc[k] - margin)) {
      inside = 0;
      c[k] = 0;
    } else {
      c[k] = (int64_t)f;
    }
  }
  return inside;
}

int orc_cells(const orc_params *p, int64_t n, const double *pos, int64_t *cell) {
  double origin[3], cs;
  int64_t nc[3];
  int32_t margin;
  if (orc_grid(p, origin, &cs, nc, &margin)) return -1;
  for (int64_t a = 0; a < n; a++) {
    int64_t c[3];
    if (cell_coords(origin, cs, nc, margin, pos + 3 * a, c))
      cell[a] = (c[2] * nc[1] + c[1]) * nc[0] + c[0];
    else
      cell[a] = -1;
  }
  return 0;
}

typedef struct {
  int64_t key;  /* is_boundary * 2^40 + cell, out-of-domain: INT64_MAX */
  int64_t rank; /* position in the previous order (makes the sort stable) */
  int64_t id;
} sort_item;

static int cmp_item(const void *x, const void *y) {
  const sort_item *a = (const sort_item *)x, *b = (const sort_item *)y;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  if (a->rank != b->rank) return a->rank < b->rank ? -1 : 1;
  return 0;
}

int64_t orc_sort(const orc_params *p, int64_t n, const double *pos,
                 const uint8_t *type, const uint8_t *out,
                 const int64_t *prev_order, int64_t *order) {
  int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
  sort_item *it = (sort_item *)malloc(sizeof(sort_item) * (n ? n : 1));
  if (!cell || !it || orc_cells(p, n, pos, cell)) {
    free(cell);
    free(it);
    return -1;
  }
  int64_t inside = 0;
  for (int64_t r = 0; r < n; r++) {
    int64_t a = prev_order ? prev_order[r] : r;
    it[r].id = a;
    it[r].rank = r;
    if (cell[a] < 0 || (out && out[a])) {
      it[r].key = INT64_MAX;
    } else {
      it[r].key = (type[a] ? ((int64_t)1 << 40) : 0) + cell[a];
      inside++;
    }
  }
  qsort(it, (size_t)n, sizeof(sort_item), cmp_item);
  for (int64_t r = 0; r < n; r++) order[r] = it[r].id;
  free(cell);
  free(it);
  return inside;
}

/* Cell list: particles of each cell (in neighbour-list order). */
typedef struct {
  double origin[3], cs;
  int64_t nc[3], ncells;
  int32_t margin;
  int64_t *order;  /* in-domain particles sorted by (cell, type) */
  int64_t *start;  /* start[c] .. start[c+1]: particles of cell c in order */
  int64_t *cellof; /* cell of each particle, -1 if out */
} cell_list;

static void cl_free(cell_list *cl) {
  free(cl->order);
  free(cl->start);
  free(cl->cellof);
}

static int cl_build(const orc_params *p, int64_t n, const double *pos,
                    const uint8_t *type, const uint8_t *out, cell_list *cl) {
  memset(cl, 0, sizeof(*cl));
  if (orc_grid(p, cl->origin, &cl->cs, cl->nc, &cl->margin)) return -1;
  cl->ncells = cl->nc[0] * cl->nc[1] * cl->nc[2];
  cl->order = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
  cl->start = (int64_t *)calloc((size_t)cl->ncells + 1, sizeof(int64_t));
  cl->cellof = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
  if (!cl->order || !cl->start || !cl->cellof) return -1;
  orc_cells(p, n, pos, cl->cellof);
  for (int64_t a = 0; a < n; a++)
    if (out && out[a]) cl->cellof[a] = -1;
  /* the lookup structure groups particles by cell only (type ignored) */
  (void)type;
  uint8_t *notype = (uint8_t *)calloc((size_t)(n ? n : 1), 1);
  int64_t inside = notype ? orc_sort(p, n, pos, notype, out, NULL, cl->order) : -1;
  free(notype);
  if (inside < 0) return -1;
  /* counting pass, then prefix sum gives the first index of every cell */
  for (int64_t r = 0; r < inside; r++) cl->start[cl->cellof[cl->order[r]] + 1]++;
  for (int64_t c = 0; c < cl->ncells; c++) cl->start[c + 1] += cl->start[c];
  return 0;
}

/* ---- neighbour pairs -------------------------------------------------- */

static uint64_t splitmix64_mix(uint64_t z) {
  /* finaliser of SplitMix64 (Steele, Lea, Flood 2014) */
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static int cmp_pair(const void *x, const void *y) {
  const int64_t *a = (const int64_t *)x, *b = (const int64_t *)y;
  if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
  if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
  return 0;
}

int64_t orc_pairs(const orc_params *p, int64_t n, const double *pos,
                  const uint8_t *out, int use_cells, int64_t *count,
                  uint64_t *hash, int64_t *pairs, int64_t cap) {
  double R2 = 4.0 * p->h * p->h;
  int64_t total = 0;
  cell_list cl;
  uint8_t *type0 = (uint8_t *)calloc((size_t)(n ? n : 1), 1);
  if (use_cells && cl_build(p, n, pos, type0, out, &cl)) {
    cl_free(&cl);
    free(type0);
    return -1;
  }
  for (int64_t a = 0; a < n; a++) {
    count[a] = 0;
    hash[a] = 0;
  }
  for (int64_t a = 0; a < n; a++) {
    if (out && out[a]) continue;
    if (use_cells && cl.cellof[a] < 0) continue;
    const double *ra = pos + 3 * a;
    if (!use_cells) {
      for (int64_t b = 0; b < n; b++) {
        if (b == a || (out && out[b])) continue;
        double dx = ra[0] - pos[3 * b], dy = ra[1] - pos[3 * b + 1],
               dz = ra[2] - pos[3 * b + 2];
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 > 0.0 && r2 < R2) {
          if (pairs && total < cap) {
            pairs[2 * total] = a;
            pairs[2 * total + 1] = b;
          }
          total++;
          count[a]++;
          hash[a] += splitmix64_mix((uint64_t)b);
        }
      }
    } else {
      int64_t c = cl.cellof[a];
      int64_t cx = c % cl.nc[0], cy = (c / cl.nc[0]) % cl.nc[1],
              cz = c / (cl.nc[0] * cl.nc[1]);
      int32_t M = cl.margin;
      for (int64_t z = cz - M; z <= cz + M; z++)
        for (int64_t y = cy - M; y <= cy + M; y++)
          for (int64_t x = cx - M; x <= cx + M; x++) {
            int64_t cc = (z * cl.nc[1] + y) * cl.nc[0] + x;
            for (int64_t k = cl.start[cc]; k < cl.start[cc + 1]; k++) {
              int64_t b = cl.order[k];
              if (b == a) continue;
              double dx = ra[0] - pos[3 * b], dy = ra[1] - pos[3 * b + 1],
                     dz = ra[2] - pos[3 * b + 2];
              double r2 = dx * dx + dy * dy + dz * dz;
              if (r2 > 0.0 && r2 < R2) {
                if (pairs && total < cap) {
                  pairs[2 * total] = a;
                  pairs[2 * total + 1] = b;
                }
                total++;
                count[a]++;
                hash[a] += splitmix64_mix((uint64_t)b);
              }
            }
          }
    }
  }
  if (pairs) qsort(pairs, (size_t)(total < cap ? total : cap), 2 * sizeof(int64_t), cmp_pair);
  if (use_cells) cl_free(&cl);
  free(type0);
  return total;
}

/* ---- particle interaction (PI) ---------------------------------------- */

/* Contribution of neighbour b to particle a.  Accumulates into acc[3],
 * drho, mu.  Returns 1 if the pair is inside the kernel support. */
static int pair_interaction(const orc_params *p, int a, int b_fluid,
                            const double *ra, const double *rb,
                            const double *va, const double *vb, double rhoa,
                            double rhob, double Pa, double Pb, int a_fluid,
                            const double *tau_a, const double *tau_b,
                            double *acc, double *drho, double *mu) {
  (void)a;
  double rab[3] = {ra[0] - rb[0], ra[1] - rb[1], ra[2] - rb[2]};
  double r2 = rab[0] * rab[0] + rab[1] * rab[1] + rab[2] * rab[2];
  if (!(r2 > 0.0 && r2 < 4.0 * p->h * p->h)) return 0;
  double r = sqrt(r2);
  double F = orc_wendland_gradfac(r, p->h); /* grad_a W_ab = F r_ab */
  double gradW[3] = {F * rab[0], F * rab[1], F * rab[2]};
  double vab[3] = {va[0] - vb[0], va[1] - vb[1], va[2] - vb[2]};
  double vdotgw = vab[0] * gradW[0] + vab[1] * gradW[1] + vab[2] * gradW[2];
  double m = p->rho0 * p->dp * p->dp * p->dp;
  double Vb = m / rhob;
  /* continuity, Eq 15 (fluid a) and Eq 36 (boundary a) */
  *drho += rhoa * Vb * vdotgw;
  if (!a_fluid) return 1;
  /* density diffusion D_a, Eq 17, over fluid neighbours only; psi_ab from
   * Eq 18 (mode 1) or Eq 19-20 (mode 2), in the diffusive sign (drho > 0
   * where the neighbours are denser than the hydrostatic difference) */
  if ((p->ddt_mode == 1 || p->ddt_mode == 2) && b_fluid) {
    double drho_ba = rhob - rhoa;
    if (p->ddt_mode == 2) drho_ba -= orc_rho_hydro(p, rab);
    double psi_dot_gradW = -2.0 * drho_ba * F;
    *drho += p->delta * p->h * p->cs0 * psi_dot_gradW * Vb;
  }
  double vr = vab[0] * rab[0] + vab[1] * rab[1] + vab[2] * rab[2];
  double muab = p->h * vr / (r2 + p->eta2);
  double Pi = 0.0;
  if (p->visc_mode == 0 && vr < 0.0) {
    /* artificial viscosity, Eq 21 */
    double cbar = p->cs0;
    double rhobar = 0.5 * (rhoa + rhob);
    Pi = -p->alpha * cbar * muab / rhobar;
  }
  /* momentum, Eq 22 (Eq 16 with Pi) */
  double s = m * ((Pa + Pb) / (rhoa * rhob) + Pi);
  acc[0] -= s * gradW[0];
  acc[1] -= s * gradW[1];
  acc[2] -= s * gradW[2];
  if (p->visc_mode == 1) {
    /* laminar viscosity, Eq 23: m_b 4 nu0 (r_ab . grad W) v_ab / ((rho_a + rho_b)(r^2 + eta^2)) */
    double rgw = rab[0] * gradW[0] + rab[1] * gradW[1] + rab[2] * gradW[2];
    double cl = m * 4.0 * p->nu0 * rgw / ((rhoa + rhob) * (r2 + p->eta2));
    for (int i = 0; i < 3; i++) acc[i] += cl * vab[i];
    /* SPS stress, Eq 26: m_b (tau_a + tau_b)^{ij} / (rho_a rho_b) grad^j W, with
     * tau = rho (tau / rho) from Eq 25 */
    double T[3][3];
    const int ix[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++)
        T[i][j] = (rhoa * tau_a[ix[i][j]] + rhob * tau_b[ix[i][j]]) / (rhoa * rhob);
    for (int i = 0; i < 3; i++)
      acc[i] += m * (T[i][0] * gradW[0] + T[i][1] * gradW[1] + T[i][2] * gradW[2]);
  }
  /* Eq 35 inner maximum */
  double mu_abs = fabs(muab);
  if (mu_abs > *mu) *mu = mu_abs;
  return 1;
}

/* Candidate neighbours of particle a: every other in-domain particle (brute
 * force, index order) or every particle of the (2M+1)^3 cells around a's
 * cell (cell-list order).  The caller tests the support and the types. */
static int64_t candidates(int use_cells, const cell_list *cl, int64_t n, const uint8_t *out,
                          int64_t a, int64_t **buf, int64_t *cap) {
  int64_t k = 0;
#define ORC_PUSH(b)                                                   \
  do {                                                                \
    if (k == *cap) {                                                  \
      *cap = *cap ? 2 * *cap : 1024;                                  \
      *buf = (int64_t *)realloc(*buf, sizeof(int64_t) * (size_t)*cap); \
    }                                                                 \
    (*buf)[k++] = (b);                                                \
  } while (0)
  if (!use_cells) {
    for (int64_t b = 0; b < n; b++)
      if (b != a && !(out && out[b])) ORC_PUSH(b);
  } else {
    int64_t c = cl->cellof[a];
    int64_t cx = c % cl->nc[0], cy = (c / cl->nc[0]) % cl->nc[1], cz = c / (cl->nc[0] * cl->nc[1]);
    int32_t M = cl->margin;
    for (int64_t z = cz - M; z <= cz + M; z++)
      for (int64_t y = cy - M; y <= cy + M; y++)
        for (int64_t x = cx - M; x <= cx + M; x++) {
          int64_t cc = (z * cl->nc[1] + y) * cl->nc[0] + x;
          for (int64_t q = cl->start[cc]; q < cl->start[cc + 1]; q++)
            if (cl->order[q] != a) ORC_PUSH(cl->order[q]);
        }
  }
#undef ORC_PUSH
  return k;
}

/* Eq 24-25 for every active fluid particle (tau6 = tau / rho, 6 per particle). */
static void sps_tau_all(const orc_params *p, int64_t n, const double *pos, const double *vel,
                        const double *rho, const uint8_t *type, const uint8_t *out,
                        int use_cells, const cell_list *cl, double *tau6) {
  const double m = p->rho0 * p->dp * p->dp * p->dp;
  const double R2 = 4.0 * p->h * p->h;
#pragma omp parallel
  {
    int64_t *buf = NULL, cap = 0;
#pragma omp for schedule(dynamic, 256)
    for (int64_t a = 0; a < n; a++) {
      double *T = tau6 + 6 * a;
      for (int i = 0; i < 6; i++) T[i] = 0.0;
      int active = !(out && out[a]) && (!use_cells || cl->cellof[a] >= 0);
      if (!active || type[a] != 0) continue;
      /* SPH velocity gradient G^{ij} = sum_b V_b (v_b - v_a)^i grad^j_a W_ab */
      double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      const double *ra = pos + 3 * a, *va = vel + 3 * a;
      int64_t nc = candidates(use_cells, cl, n, out, a, &buf, &cap);
      for (int64_t k = 0; k < nc; k++) {
        int64_t b = buf[k];
        double rab[3] = {ra[0] - pos[3 * b], ra[1] - pos[3 * b + 1], ra[2] - pos[3 * b + 2]};
        double r2 = rab[0] * rab[0] + rab[1] * rab[1] + rab[2] * rab[2];
        if (!(r2 > 0.0 && r2 < R2)) continue;
        double F = orc_wendland_gradfac(sqrt(r2), p->h);
        double Vb = m / rho[b];
        for (int i = 0; i < 3; i++)
          for (int j = 0; j < 3; j++) G[i][j] += Vb * (vel[3 * b + i] - va[i]) * F * rab[j];
      }
      /* strain rate S = (G + G^T) / 2 and |S| = (2 S:S)^(1/2) / 2 as printed
       * with Eq 25; nu_SPS = (C_S Delta)^2 |S| (dimensionally consistent
       * reading of the printed square); Delta = dp */
      double S[3][3], SS = 0.0;
      for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
          S[i][j] = 0.5 * (G[i][j] + G[j][i]);
          SS += S[i][j] * S[i][j];
        }
      double Smag = 0.5 * sqrt(2.0 * SS);
      double tr = S[0][0] + S[1][1] + S[2][2];
      double nu = ORC_SPS_CS * p->dp * ORC_SPS_CS * p->dp * Smag;
      double iso = -(2.0 / 3.0) * ORC_SPS_CL * p->dp * p->dp * Smag * Smag;
      T[0] = 2.0 * nu * (S[0][0] - tr / 3.0) + iso;
      T[1] = 2.0 * nu * (S[1][1] - tr / 3.0) + iso;
      T[2] = 2.0 * nu * (S[2][2] - tr / 3.0) + iso;
      T[3] = 2.0 * nu * S[0][1];
      T[4] = 2.0 * nu * S[0][2];
      T[5] = 2.0 * nu * S[1][2];
    }
    free(buf);
  }
}

int orc_sps_tau(const orc_params *p, int64_t n, const double *pos, const double *vel,
                const double *rho, const uint8_t *type, const uint8_t *out, double *tau6) {
  cell_list cl;
  if (cl_build(p, n, pos, type, out, &cl)) {
    cl_free(&cl);
    return -1;
  }
  sps_tau_all(p, n, pos, vel, rho, type, out, 1, &cl, tau6);
  cl_free(&cl);
  return 0;
}

int64_t orc_interact(const orc_params *p, int64_t n, const double *pos,
                     const double *vel, const double *rho, const uint8_t *type,
                     const uint8_t *out, int use_cells, double *acc,
                     double *drho, double *mumax) {
  return orc_interact_range(p, n, pos, vel, rho, type, out, use_cells, 0, n,
                            acc, drho, mumax);
}

int64_t orc_interact_range(const orc_params *p, int64_t n, const double *pos,
                           const double *vel, const double *rho,
                           const uint8_t *type, const uint8_t *out,
                           int use_cells, int64_t a0, int64_t a1, double *acc,
                           double *drho, double *mumax) {
  if (a0 < 0) a0 = 0;
  if (a1 > n) a1 = n;
  cell_list cl;
  if (use_cells && cl_build(p, n, pos, type, out, &cl)) {
    cl_free(&cl);
    return -1;
  }
  double *press = (double *)malloc(sizeof(double) * (n ? n : 1));
  for (int64_t a = 0; a < n; a++) press[a] = orc_tait(p, rho[a]);
  double *tau6 = NULL;
  if (p->visc_mode == 1) {
    tau6 = (double *)malloc(sizeof(double) * 6 * (size_t)(n ? n : 1));
    sps_tau_all(p, n, pos, vel, rho, type, out, use_cells, &cl, tau6);
  }
  static const double zero6[6] = {0, 0, 0, 0, 0, 0};
  int64_t total = 0;

#pragma omp parallel reduction(+ : total)
  {
    int64_t *buf = NULL, cap = 0;
#pragma omp for schedule(dynamic, 256)
    for (int64_t a = a0; a < a1; a++) {
      double ac[3] = {0.0, 0.0, 0.0}, dr = 0.0, mu = 0.0;
      int a_fluid = type[a] == 0;
      int active = !(out && out[a]) && (!use_cells || cl.cellof[a] >= 0);
      /* mDBC: the density of B comes from Eq 38, not from Eq 36 */
      if (p->boundary_mode == 1 && !a_fluid) active = 0;
      if (active) {
        const double *ra = pos + 3 * a;
        int64_t nc = candidates(use_cells, &cl, n, out, a, &buf, &cap);
        for (int64_t k = 0; k < nc; k++) {
          int64_t b = buf[k];
          int b_fluid = type[b] == 0;
          if (!a_fluid && !b_fluid) continue; /* Eq 36: b in F only */
          total += pair_interaction(p, (int)a, b_fluid, ra, pos + 3 * b, vel + 3 * a,
                                    vel + 3 * b, rho[a], rho[b], press[a], press[b], a_fluid,
                                    tau6 ? tau6 + 6 * a : zero6, tau6 ? tau6 + 6 * b : zero6,
                                    ac, &dr, &mu);
        }
        if (a_fluid) {
          ac[0] += p->g[0];
          ac[1] += p->g[1];
          ac[2] += p->g[2];
        }
      }
      acc[3 * a] = ac[0];
      acc[3 * a + 1] = ac[1];
      acc[3 * a + 2] = ac[2];
      drho[a] = dr;
      mumax[a] = mu;
    }
    free(buf);
  }
  free(tau6);
  free(press);
  if (use_cells) cl_free(&cl);
  return total;
}

/* ---- time step, Eq 35 ------------------------------------------------- */

double orc_dt(const orc_params *p, int64_t n, const double *acc,
              const double *mumax, const uint8_t *type, const uint8_t *out) {
  if (p->dt_fixed > 0.0) return p->dt_fixed;
  double dtf = INFINITY, mumx = 0.0;
  for (int64_t a = 0; a < n; a++) {
    if (type[a] != 0 || (out && out[a])) continue;
    double f = sqrt(acc[3 * a] * acc[3 * a] + acc[3 * a + 1] * acc[3 * a + 1] +
                    acc[3 * a + 2] * acc[3 * a + 2]);
    if (f > 0.0) {
      double d = sqrt(p->h / f);
      if (d < dtf) dtf = d;
    }
    if (mumax[a] > mumx) mumx = mumax[a];
  }
  /* min_a h / (cs + mu_a) is reached at the largest mu_a */
  double dtcv = p->h / (p->cs0 + mumx);
  return p->cfl * (dtf < dtcv ? dtf : dtcv);
}

/* ---- Symplectic step, Eq 33-34 with imposed motion Eq 37 ---------------- */

static double motion_disp(const orc_motion *m, double t) {
  return m->amp * (sin(m->omega * t + m->phase) - sin(m->phase));
}
static double motion_vel(const orc_motion *m, double t) {
  return m->amp * m->omega * cos(m->omega * t + m->phase);
}

static int inside_domain(const orc_params *p, const double *r) {
  double origin[3], cs;
  int64_t nc[3], c[3];
  int32_t margin;
  orc_grid(p, origin, &cs, nc, &margin);
  return cell_coords(origin, cs, nc, margin, r, c);
}

int64_t orc_step(const orc_params *p, const orc_motion *motions, int32_t nmot,
                 int64_t n, double *pos, double *vel, double *rho,
                 const uint8_t *type, const int32_t *group, uint8_t *out,
                 int64_t *order, double *t, double *last_dt, int64_t nsteps,
                 const double *ghost) {
  if (p->boundary_mode == 1 && !ghost) return -1;
  size_t N = (size_t)(n ? n : 1);
  double *acc = (double *)malloc(sizeof(double) * 3 * N);
  double *drho = (double *)malloc(sizeof(double) * N);
  double *mu = (double *)malloc(sizeof(double) * N);
  double *pos0 = (double *)malloc(sizeof(double) * 3 * N);
  double *vel0 = (double *)malloc(sizeof(double) * 3 * N);
  double *rho0 = (double *)malloc(sizeof(double) * N);
  int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * N);
  int64_t pairs = 0;
  for (int64_t s = 0; s < nsteps; s++) {
    /* NL + PI on state n */
    if (order) {
      orc_sort(p, n, pos, type, out, order, tmp);
      memcpy(order, tmp, sizeof(int64_t) * (size_t)n);
    }
    if (p->boundary_mode == 1)
      orc_mdbc(p, motions, nmot, n, pos, vel, rho, type, group, out, ghost, *t, NULL);
    int64_t np = orc_interact(p, n, pos, vel, rho, type, out, 1, acc, drho, mu);
    if (np < 0) { pairs = -1; break; }
    pairs += np;
    double dt = orc_dt(p, n, acc, mu, type, out);
    double t0 = *t;
    memcpy(pos0, pos, sizeof(double) * 3 * (size_t)n);
    memcpy(vel0, vel, sizeof(double) * 3 * (size_t)n);
    memcpy(rho0, rho, sizeof(double) * (size_t)n);
    /* predictor: state n+1/2 */
    for (int64_t a = 0; a < n; a++) {
      if (out[a]) continue;
      if (type[a] == 0) {
        for (int k = 0; k < 3; k++) {
          pos[3 * a + k] = pos0[3 * a + k] + 0.5 * dt * vel0[3 * a + k];
          vel[3 * a + k] = vel0[3 * a + k] + 0.5 * dt * acc[3 * a + k];
        }
        rho[a] = rho0[a] + 0.5 * dt * drho[a];
      } else {
        rho[a] = rho0[a] + 0.5 * dt * drho[a];
        if (p->clamp_boundary_rho && rho[a] < p->rho0) rho[a] = p->rho0;
        int g = group ? group[a] : -1;
        if (g >= 0 && g < nmot) {
          const orc_motion *m = motions + g;
          double d = motion_disp(m, t0 + 0.5 * dt) - motion_disp(m, t0);
          double v = motion_vel(m, t0 + 0.5 * dt);
          for (int k = 0; k < 3; k++) {
            pos[3 * a + k] = pos0[3 * a + k] + d * m->axis[k];
            vel[3 * a + k] = v * m->axis[k];
          }
        }
      }
      if (!inside_domain(p, pos + 3 * a)) {
        /* left the domain at the half step: frozen at state n */
        memcpy(pos + 3 * a, pos0 + 3 * a, 3 * sizeof(double));
        memcpy(vel + 3 * a, vel0 + 3 * a, 3 * sizeof(double));
        rho[a] = rho0[a];
        out[a] = 1;
      }
    }
    /* NL + PI on state n+1/2 */
    if (order) {
      orc_sort(p, n, pos, type, out, order, tmp);
      memcpy(order, tmp, sizeof(int64_t) * (size_t)n);
    }
    if (p->boundary_mode == 1)
      orc_mdbc(p, motions, nmot, n, pos, vel, rho, type, group, out, ghost, t0 + 0.5 * dt,
               NULL);
    np = orc_interact(p, n, pos, vel, rho, type, out, 1, acc, drho, mu);
    if (np < 0) { pairs = -1; break; }
    pairs += np;
    /* corrector: state n+1 */
    for (int64_t a = 0; a < n; a++) {
      if (out[a]) continue;
      double eps = -(drho[a] / rho[a]) * dt; /* Eq 34 */
      double rhonew = rho0[a] * (2.0 - eps) / (2.0 + eps);
      if (type[a] == 0) {
        for (int k = 0; k < 3; k++) {
          double vn = vel0[3 * a + k] + dt * acc[3 * a + k];
          pos[3 * a + k] = pos0[3 * a + k] + dt * 0.5 * (vn + vel0[3 * a + k]);
          vel[3 * a + k] = vn;
        }
        rho[a] = rhonew;
      } else {
        if (p->clamp_boundary_rho && rhonew < p->rho0) rhonew = p->rho0;
        rho[a] = rhonew;
        int g = group ? group[a] : -1;
        if (g >= 0 && g < nmot) {
          const orc_motion *m = motions + g;
          double d = motion_disp(m, t0 + dt) - motion_disp(m, t0);
          double v = motion_vel(m, t0 + dt);
          for (int k = 0; k < 3; k++) {
            pos[3 * a + k] = pos0[3 * a + k] + d * m->axis[k];
            vel[3 * a + k] = v * m->axis[k];
          }
        }
      }
      if (!inside_domain(p, pos + 3 * a)) out[a] = 1; /* frozen at n+1 */
    }
    *t = t0 + dt;
    *last_dt = dt;
  }
  free(acc);
  free(drho);
  free(mu);
  free(pos0);
  free(vel0);
  free(rho0);
  free(tmp);
  return pairs;
}


/* ---- modified dynamic boundary condition (Sect. 2.6.2) ------------------- */

/* Solves the 4x4 system A x = b by Gaussian elimination with partial
 * pivoting; returns det(A) (x untouched when det == 0). */
static double solve4(double A[4][4], double b[4], double x[4]) {
  double det = 1.0;
  for (int c = 0; c < 4; c++) {
    int piv = c;
    for (int r = c + 1; r < 4; r++)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (A[piv][c] == 0.0) return 0.0;
    if (piv != c) {
      for (int k = 0; k < 4; k++) {
        double tmp = A[c][k];
        A[c][k] = A[piv][k];
        A[piv][k] = tmp;
      }
      double tb = b[c];
      b[c] = b[piv];
      b[piv] = tb;
      det = -det;
    }
    det *= A[c][c];
    for (int r = c + 1; r < 4; r++) {
      double f = A[r][c] / A[c][c];
      for (int k = c; k < 4; k++) A[r][k] -= f * A[c][k];
      b[r] -= f * b[c];
    }
  }
  for (int r = 3; r >= 0; r--) {
    double v = b[r];
    for (int k = r + 1; k < 4; k++) v -= A[r][k] * x[k];
    x[r] = v / A[r][r];
  }
  return det;
}

int orc_mdbc(const orc_params *p, const orc_motion *motions, int32_t nmot, int64_t n,
             const double *pos, double *vel, double *rho, const uint8_t *type,
             const int32_t *group, const uint8_t *out, const double *ghost, double t,
             double *dets) {
  if (!ghost) return -1;
  double origin[3], cs;
  int64_t nc[3];
  int32_t margin;
  if (orc_grid(p, origin, &cs, nc, &margin)) return -1;
  cell_list cl;
  if (cl_build(p, n, pos, type, out, &cl)) {
    cl_free(&cl);
    return -1;
  }
  const double m = p->rho0 * p->dp * p->dp * p->dp;
  const double R2 = 4.0 * p->h * p->h;
  /* new values go to scratch first: every ghost sees the fluid state only,
   * and boundary values do not feed each other */
  double *nrho = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
  double *nvel = (double *)malloc(sizeof(double) * 3 * (size_t)(n ? n : 1));
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t B = 0; B < n; B++) {
    nrho[B] = rho[B];
    for (int k = 0; k < 3; k++) nvel[3 * B + k] = vel[3 * B + k];
    if (dets) dets[B] = 0.0;
    if (type[B] == 0 || (out && out[B]) || cl.cellof[B] < 0) continue;
    const double *g = ghost + 3 * B;
    double rG[3] = {pos[3 * B] + g[0], pos[3 * B + 1] + g[1], pos[3 * B + 2] + g[2]};
    /* imposed velocity of B at time t (Eq 37) */
    double vw[3] = {0.0, 0.0, 0.0};
    int gi = group ? group[B] : -1;
    if (gi >= 0 && gi < nmot) {
      const orc_motion *mo = motions + gi;
      double v = motion_vel(mo, t);
      for (int k = 0; k < 3; k++) vw[k] = v * mo->axis[k];
    }
    /* moment sums over fluid b in the ghost's support */
    double A[4][4] = {{0}}, rhs[4] = {0}, sv[3] = {0, 0, 0}, sw = 0.0;
    int64_t c[3];
    for (int k = 0; k < 3; k++) c[k] = (int64_t)floor((rG[k] - origin[k]) / cs);
    for (int64_t z = c[2] - margin; z <= c[2] + margin; z++)
      for (int64_t y = c[1] - margin; y <= c[1] + margin; y++)
        for (int64_t x = c[0] - margin; x <= c[0] + margin; x++) {
          if (x < 0 || y < 0 || z < 0 || x >= nc[0] || y >= nc[1] || z >= nc[2]) continue;
          int64_t cc = (z * cl.nc[1] + y) * cl.nc[0] + x;
          for (int64_t q = cl.start[cc]; q < cl.start[cc + 1]; q++) {
            int64_t b = cl.order[q];
            if (type[b] != 0) continue;
            double d[3] = {rG[0] - pos[3 * b], rG[1] - pos[3 * b + 1], rG[2] - pos[3 * b + 2]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < R2)) continue;
            double r = sqrt(r2);
            double W = orc_wendland_w(r, p->h);
            double F = orc_wendland_gradfac(r, p->h); /* grad_G W = F (r_G - r_b) */
            double Vb = m / rho[b];
            double e[3] = {-d[0], -d[1], -d[2]}; /* r_b - r_G */
            A[0][0] += Vb * W;
            for (int k = 0; k < 3; k++) {
              A[0][k + 1] += Vb * e[k] * W;
              A[k + 1][0] += Vb * F * d[k];
              for (int l = 0; l < 3; l++) A[k + 1][l + 1] += Vb * F * d[k] * e[l];
              sv[k] += Vb * vel[3 * b + k] * W;
            }
            rhs[0] += m * W;
            for (int k = 0; k < 3; k++) rhs[k + 1] += m * F * d[k];
            sw += Vb * W;
          }
        }
    if (sw <= 0.0) { /* no fluid near the ghost */
      nrho[B] = p->rho0;
      if (p->mdbc_slip) for (int k = 0; k < 3; k++) nvel[3 * B + k] = vw[k];
      continue;
    }
    double Ac[4][4], bc[4], x[4] = {0, 0, 0, 0};
    for (int r = 0; r < 4; r++) {
      bc[r] = rhs[r];
      for (int k = 0; k < 4; k++) Ac[r][k] = A[r][k];
    }
    double det = solve4(Ac, bc, x);
    if (dets) dets[B] = det;
    double rhoG, grad[3] = {0.0, 0.0, 0.0};
    if (fabs(det) >= ORC_MDBC_DET_MIN) {
      rhoG = x[0];
      for (int k = 0; k < 3; k++) grad[k] = x[k + 1];
    } else {
      rhoG = rhs[0] / sw; /* Shepard */
    }
    /* Eq 38: rho_B = rho_G + (r_B - r_G) . grad rho_G, r_B - r_G = -ghost */
    double rB = rhoG - (g[0] * grad[0] + g[1] * grad[1] + g[2] * grad[2]);
    if (!(rB > 0.0 && rB < 1e30)) rB = rhs[0] / sw; /* not a usable density: Shepard */
    nrho[B] = rB; /* used as is: the rho >= rho0 clamp is a device of Eq 36 */
    /* Eq 39: v_G by the Shepard sum */
    double vG[3] = {sv[0] / sw, sv[1] / sw, sv[2] / sw};
    if (p->mdbc_slip == 1) {
      for (int k = 0; k < 3; k++) nvel[3 * B + k] = 2.0 * vw[k] - vG[k];
    } else if (p->mdbc_slip == 2) {
      double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
      double nn[3] = {0.0, 0.0, 0.0};
      if (gn > 0.0) for (int k = 0; k < 3; k++) nn[k] = g[k] / gn;
      double vn = 0.0, wn = 0.0;
      for (int k = 0; k < 3; k++) {
        vn += vG[k] * nn[k];
        wn += vw[k] * nn[k];
      }
      /* tangential part of v_G kept, normal part reversed about the wall's */
      for (int k = 0; k < 3; k++) nvel[3 * B + k] = vG[k] + (2.0 * wn - 2.0 * vn) * nn[k];
    }
  }
  for (int64_t B = 0; B < n; B++) {
    rho[B] = nrho[B];
    for (int k = 0; k < 3; k++) vel[3 * B + k] = nvel[3 * B + k];
  }
  free(nrho);
  free(nvel);
  cl_free(&cl);
  return 0;
}

/* ---- Verlet scheme (Sect. 2.5.1) ---------------------------------------- */

int64_t orc_step_verlet(const orc_params *p, const orc_motion *motions, int32_t nmot,
                        int64_t n, double *pos, double *vel, double *rho,
                        double *vel_prev, double *rho_prev, const uint8_t *type,
                        const int32_t *group, uint8_t *out, int64_t *order, double *t,
                        double *last_dt, int64_t *step, int32_t ns, int64_t nsteps,
                        const double *ghost) {
  if (ns < 1) return -1;
  if (p->boundary_mode == 1 && !ghost) return -1;
  size_t N = (size_t)(n ? n : 1);
  double *acc = (double *)malloc(sizeof(double) * 3 * N);
  double *drho = (double *)malloc(sizeof(double) * N);
  double *mu = (double *)malloc(sizeof(double) * N);
  int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * N);
  int64_t pairs = 0;
  for (int64_t s = 0; s < nsteps; s++) {
    /* NL + PI on state n: F^n, R^n */
    if (order) {
      orc_sort(p, n, pos, type, out, order, tmp);
      memcpy(order, tmp, sizeof(int64_t) * (size_t)n);
    }
    if (p->boundary_mode == 1)
      orc_mdbc(p, motions, nmot, n, pos, vel, rho, type, group, out, ghost, *t, NULL);
    int64_t np = orc_interact(p, n, pos, vel, rho, type, out, 1, acc, drho, mu);
    if (np < 0) { pairs = -1; break; }
    pairs += np;
    double dt = orc_dt(p, n, acc, mu, type, out);
    double t0 = *t;
    int eq31 = (*step % ns) == 0;
    for (int64_t a = 0; a < n; a++) {
      if (out[a]) continue;
      /* density: Eq 30 (from rho^{n-1}, twice the step) or Eq 31 */
      double rnew = eq31 ? rho[a] + dt * drho[a] : rho_prev[a] + 2.0 * dt * drho[a];
      if (type[a] == 0) {
        for (int k = 0; k < 3; k++) {
          double vn = vel[3 * a + k], F = acc[3 * a + k];
          pos[3 * a + k] += dt * vn + 0.5 * dt * dt * F;
          double vnew = eq31 ? vn + dt * F : vel_prev[3 * a + k] + 2.0 * dt * F;
          vel_prev[3 * a + k] = vn;
          vel[3 * a + k] = vnew;
        }
      } else {
        if (p->clamp_boundary_rho && rnew < p->rho0) rnew = p->rho0;
        for (int k = 0; k < 3; k++) vel_prev[3 * a + k] = vel[3 * a + k];
        int g = group ? group[a] : -1;
        if (g >= 0 && g < nmot) {
          const orc_motion *m = motions + g;
          double d = motion_disp(m, t0 + dt) - motion_disp(m, t0);
          double v = motion_vel(m, t0 + dt);
          for (int k = 0; k < 3; k++) {
            pos[3 * a + k] += d * m->axis[k];
            vel[3 * a + k] = v * m->axis[k];
          }
        }
      }
      rho_prev[a] = rho[a];
      rho[a] = rnew;
      if (!inside_domain(p, pos + 3 * a)) out[a] = 1; /* frozen at n+1 */
    }
    *t = t0 + dt;
    *last_dt = dt;
    *step += 1;
  }
  free(acc);
  free(drho);
  free(mu);
  free(tmp);
  return pairs;
}

/* ---- diagnostics ------------------------------------------------------ */

int orc_diag(const orc_params *p, int64_t n, const double *pos,
             const double *vel, const uint8_t *type, const uint8_t *out,
             double res[7]) {
  double m = p->rho0 * p->dp * p->dp * p->dp;
  double ke = 0.0, px = 0.0, py = 0.0, pz = 0.0, front = -INFINITY;
  double nout = 0.0;
  /* Eq 14: every particle keeps its mass m, so the total is exactly n m */
  double mass = (double)n * m;
  for (int64_t a = 0; a < n; a++) {
    if (out && out[a]) {
      nout += 1.0;
      continue;
    }
    if (type[a] != 0) continue;
    const double *v = vel + 3 * a;
    ke += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    px += m * v[0];
    py += m * v[1];
    pz += m * v[2];
    if (pos[3 * a] > front) front = pos[3 * a];
  }
  res[0] = mass;
  res[1] = ke;
  res[2] = px;
  res[3] = py;
  res[4] = pz;
  res[5] = front;
  res[6] = nout;
  return 0;
}
