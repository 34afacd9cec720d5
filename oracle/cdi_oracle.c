/*
 * FP64 CPU oracle for the pore-scale CDI model (arXiv 2110.13055).
 *
 * TEST INFRASTRUCTURE ONLY: see cdi_oracle.h.  Plain loops in the paper's
 * order; no blocking, fusion or reordering.  Where the paper is silent the
 * following readings are taken (each one named where it is used):
 *
 *   LBM (Sec. 2, Eq. 7-8).  Populations are stored shifted, g_i = f_i - w_i
 *   (rest density 1).  Equilibrium: the Stokes-linear form
 *   g_i^eq = w_i (drho + 3 e_i . j), because Eq. 2 is the Stokes equation and
 *   the sentence that should give f^eq is cut off.  The body force F (the
 *   pressure gradient of Sec. 2) enters as j = sum_i e_i g_i + F/2 and a
 *   source (1 - 1/(2 tau)) 3 w_i e_i . F (Guo's forcing linearised like the
 *   equilibrium).  The velocity is u = j.  Bounce-back is the halfway,
 *   link-wise rule.  "Mirror image" boundaries: the mask is reflected about
 *   its outlet plane, doubling it along x, and the doubled grid is periodic
 *   in x.  Steady state: every K steps the relative change of u over the last
 *   K steps, ||u(t) - u(t-K)|| / ||u(t)|| over pore cells, is compared with a
 *   tolerance.
 *
 *   Potential (Eq. 4-5).  A frozen cell-centred field: the Debye-Hueckel
 *   linearisation of Eq. 4 about the electroneutral initial state, with the
 *   screening length of Eq. 10's denominator; the surface value psi_s is
 *   imposed at the solid faces (half a cell from the pore-cell centre), the
 *   inlet feed is at psi = 0, the outlet and lateral walls carry no flux.
 *
 *   Transport (Eq. 3, Eq. 6).  Explicit finite volumes in conservative form;
 *   face fluxes by Scharfetter-Gummel exponential fitting of advection plus
 *   migration against diffusion; Eq. 6 closed over the half-cell distance,
 *   K_eff = Ka / (1 + Ka dx / (2 D)); inlet ghost at the feed concentration
 *   and zero potential; outlet ghost copies its neighbour (fully developed
 *   outflow); forward Euler.
 */
#include "cdi_oracle.h"

#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Lattices: D2Q9 and D3Q19 (Sec. 2).  Weights follow from |e|^2.            */
/* ------------------------------------------------------------------------ */
static const int E2[9][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0},
                             {0, 1, 0},  {0, -1, 0}, {1, 1, 0},
                             {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
static const int E3[19][3] = {
    {0, 0, 0},   {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
    {0, 0, 1},   {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0},  {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

typedef struct {
  int Q;
  int e[19][3];
  double w[19];
  int opp[19];
} lattice;

static void make_lattice(int dim, lattice *L) {
  L->Q = (dim == 2) ? 9 : 19;
  for (int i = 0; i < L->Q; i++) {
    const int *src = (dim == 2) ? E2[i] : E3[i];
    int n2 = 0;
    for (int a = 0; a < 3; a++) {
      L->e[i][a] = src[a];
      n2 += src[a] * src[a];
    }
    if (dim == 2)
      L->w[i] = (n2 == 0) ? 4.0 / 9.0 : (n2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
    else
      L->w[i] = (n2 == 0) ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  for (int i = 0; i < L->Q; i++)
    for (int k = 0; k < L->Q; k++)
      if (L->e[k][0] == -L->e[i][0] && L->e[k][1] == -L->e[i][1] &&
          L->e[k][2] == -L->e[i][2])
        L->opp[i] = k;
}

/* ------------------------------------------------------------------------ */
/* LBM Stokes solve                                                         */
/* ------------------------------------------------------------------------ */

/* Neighbour of flow-grid site (x,y,z) along (dx,dy,dz): returns the site
 * index, or -1 when the step leaves through a lateral wall. */
static long flow_neighbour(int x, int y, int z, int dx, int dy, int dz,
                           int NX, int ny, int nz, int walls) {
  int X = x + dx, Y = y + dy, Z = z + dz;
  X = ((X % NX) + NX) % NX; /* periodic along the (mirrored) flow axis */
  if (Y < 0 || Y >= ny) {
    if (walls) return -1;
    Y = ((Y % ny) + ny) % ny;
  }
  if (Z < 0 || Z >= nz) {
    if (walls) return -1;
    Z = ((Z % nz) + nz) % nz;
  }
  return ((long)Z * ny + Y) * NX + X;
}

/* u = sum_i e_i g_i + F/2 at every pore site; 0 in solid. */
static void lbm_velocity(const lattice *L, int dim, long N, const uint8_t *solid,
                         const double *g, double fx, double *u) {
#pragma omp parallel for schedule(static)
  for (long s = 0; s < N; s++) {
    for (int a = 0; a < dim; a++) u[a * N + s] = 0.0;
    if (solid[s]) continue;
    double j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L->Q; i++)
      for (int a = 0; a < 3; a++) j[a] += L->e[i][a] * g[(long)i * N + s];
    j[0] += 0.5 * fx;
    for (int a = 0; a < dim; a++) u[a * N + s] = j[a];
  }
}

int orc_lbm(int dim, int nx, int ny, int nz, const uint8_t *mask, int mirror,
            int lateral_walls, double tau, double force_x, double tol,
            int check_every, long max_steps, double *u_flow, long *steps_done,
            double *residual) {
  if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || nz < 1) return -1;
  if (dim == 2 && nz != 1) return -1;
  if (tau <= 0.5 || check_every < 2 || (check_every % 2) != 0) return -1;
  if (max_steps < 0 || (max_steps % check_every) != 0) return -1;
  lattice L;
  make_lattice(dim, &L);
  const int NX = mirror ? 2 * nx : nx;
  const long N = (long)NX * ny * nz;

  /* flow mask: the pore image followed by its mirror image along x */
  uint8_t *solid = (uint8_t *)malloc((size_t)N);
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < NX; x++) {
        int xs = (x < nx) ? x : 2 * nx - 1 - x;
        solid[((long)z * ny + y) * NX + x] = mask[((long)z * ny + y) * nx + xs];
      }

  double *g = (double *)calloc((size_t)L.Q * N, sizeof(double));
  double *gn = (double *)calloc((size_t)L.Q * N, sizeof(double));
  double *u = (double *)malloc(sizeof(double) * dim * N);
  double *uprev = (double *)malloc(sizeof(double) * dim * N);
  lbm_velocity(&L, dim, N, solid, g, force_x, uprev);

  const double F[3] = {force_x, 0.0, 0.0};
  long step = 0;
  double r = NAN;
  int converged = 0;
  while (step < max_steps) {
    /* one step of Eq. 7: collide (Eq. 8) and push to the neighbours (every
     * target slot has exactly one source, so rows may run in any order) */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; z++)
      for (int y = 0; y < ny; y++)
        for (int x = 0; x < NX; x++) {
          long s = ((long)z * ny + y) * NX + x;
          if (solid[s]) continue;
          double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
          for (int i = 0; i < L.Q; i++) {
            double gi = g[(long)i * N + s];
            drho += gi;
            for (int a = 0; a < 3; a++) j[a] += L.e[i][a] * gi;
          }
          for (int a = 0; a < 3; a++) j[a] += 0.5 * F[a];
          for (int i = 0; i < L.Q; i++) {
            double ej = 0.0, eF = 0.0;
            for (int a = 0; a < 3; a++) {
              ej += L.e[i][a] * j[a];
              eF += L.e[i][a] * F[a];
            }
            double geq = L.w[i] * (drho + 3.0 * ej);
            double gi = g[(long)i * N + s];
            double gpost = gi - (gi - geq) / tau +
                           (1.0 - 1.0 / (2.0 * tau)) * 3.0 * L.w[i] * eF;
            long nb = flow_neighbour(x, y, z, L.e[i][0], L.e[i][1], L.e[i][2],
                                     NX, ny, nz, lateral_walls);
            if (nb < 0 || solid[nb])
              gn[(long)L.opp[i] * N + s] = gpost; /* bounce back */
            else
              gn[(long)i * N + nb] = gpost;
          }
        }
    double *t = g;
    g = gn;
    gn = t;
    step++;
    if (step % check_every == 0) {
      lbm_velocity(&L, dim, N, solid, g, force_x, u);
      double num = 0.0, den = 0.0;
      for (long s = 0; s < N; s++) {
        if (solid[s]) continue;
        for (int a = 0; a < dim; a++) {
          double d = u[a * N + s] - uprev[a * N + s];
          num += d * d;
          den += u[a * N + s] * u[a * N + s];
        }
      }
      r = (den > 0.0) ? sqrt(num / den) : 0.0;
      memcpy(uprev, u, sizeof(double) * dim * N);
      if (tol > 0.0 && r < tol) {
        converged = 1;
        break;
      }
    }
  }
  lbm_velocity(&L, dim, N, solid, g, force_x, u_flow);
  if (steps_done) *steps_done = step;
  if (residual) *residual = r;
  free(solid);
  free(g);
  free(gn);
  free(u);
  free(uprev);
  return (tol > 0.0 && !converged) ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Transport-grid face classification (shared by the potential and the      */
/* Nernst-Planck routines of this file).                                     */
/* ------------------------------------------------------------------------ */
enum { FACE_FLUID = 0, FACE_SOLID, FACE_INLET, FACE_OUTLET, FACE_WALL };

/* Face directions: +x, -x, +y, -y, +z, -z. */
static const int FDIR[6][3] = {{1, 0, 0},  {-1, 0, 0}, {0, 1, 0},
                               {0, -1, 0}, {0, 0, 1},  {0, 0, -1}};

static int classify_face(const uint8_t *mask, int nx, int ny, int nz,
                         int walls, int x, int y, int z, int f, long *nb) {
  int X = x + FDIR[f][0], Y = y + FDIR[f][1], Z = z + FDIR[f][2];
  *nb = -1;
  if (X < 0) return FACE_INLET;
  if (X >= nx) return FACE_OUTLET;
  if (Y < 0 || Y >= ny) {
    if (walls) return FACE_WALL;
    Y = (Y + ny) % ny;
  }
  if (Z < 0 || Z >= nz) {
    if (walls) return FACE_WALL;
    Z = (Z + nz) % nz;
  }
  *nb = ((long)Z * ny + Y) * nx + X;
  return mask[*nb] ? FACE_SOLID : FACE_FLUID;
}

/* ------------------------------------------------------------------------ */
/* Potential                                                                */
/* ------------------------------------------------------------------------ */

/* (A v)_P = (sum_f T_f + kdx2) v_P - sum_{pore neighbours} v_nb, with T = 1
 * towards a pore neighbour or the inlet feed, 2 towards a solid face, 0 at
 * the outlet and at lateral walls. */
static void psi_apply(int dim, int nx, int ny, int nz, const uint8_t *mask,
                      int walls, double kdx2, const double *v, double *Av) {
  long N = (long)nx * ny * nz;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        long P = ((long)z * ny + y) * nx + x;
        Av[P] = 0.0;
        if (mask[P]) continue;
        double diag = kdx2, off = 0.0;
        for (int f = 0; f < 2 * dim; f++) {
          long nb;
          int k = classify_face(mask, nx, ny, nz, walls, x, y, z, f, &nb);
          if (k == FACE_FLUID) {
            diag += 1.0;
            off += v[nb];
          } else if (k == FACE_SOLID) {
            diag += 2.0;
          } else if (k == FACE_INLET) {
            diag += 1.0;
          }
        }
        Av[P] = diag * v[P] - off;
      }
  (void)N;
}

int orc_psi(int dim, int nx, int ny, int nz, const uint8_t *mask,
            int lateral_walls, double psi_s, double kdx2, double tol,
            int max_iter, double *psi, int *iters, double *relres) {
  return orc_psi_src(dim, nx, ny, nz, mask, lateral_walls, psi_s, kdx2, NULL, tol,
                     max_iter, psi, iters, relres);
}

int orc_psi_src(int dim, int nx, int ny, int nz, const uint8_t *mask,
                int lateral_walls, double psi_s, double kdx2, const double *src,
                double tol, int max_iter, double *psi, int *iters, double *relres) {
  if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || nz < 1 || kdx2 < 0.0)
    return -1;
  long N = (long)nx * ny * nz;
  double *b = (double *)calloc((size_t)N, sizeof(double));
  /* the charge term of Eq. 4, dx^2 rho_e / (eps_r eps_0), when given */
  if (src)
    for (long P = 0; P < N; P++)
      if (!mask[P]) b[P] = src[P];
  double *r = (double *)malloc(sizeof(double) * N);
  double *p = (double *)malloc(sizeof(double) * N);
  double *Ap = (double *)malloc(sizeof(double) * N);
  /* right-hand side: the Dirichlet surface potential at solid faces */
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        long P = ((long)z * ny + y) * nx + x;
        if (mask[P]) continue;
        for (int f = 0; f < 2 * dim; f++) {
          long nb;
          if (classify_face(mask, nx, ny, nz, lateral_walls, x, y, z, f, &nb) ==
              FACE_SOLID)
            b[P] += 2.0 * psi_s;
        }
      }
  double bb = 0.0;
  for (long P = 0; P < N; P++) bb += b[P] * b[P];
  for (long P = 0; P < N; P++) psi[P] = 0.0;
  int it = 0;
  double rel = 0.0;
  if (bb > 0.0) {
    memcpy(r, b, sizeof(double) * N);
    memcpy(p, b, sizeof(double) * N);
    double rr = bb;
    rel = 1.0;
    while (it < max_iter) {
      psi_apply(dim, nx, ny, nz, mask, lateral_walls, kdx2, p, Ap);
      double pAp = 0.0;
      for (long P = 0; P < N; P++) pAp += p[P] * Ap[P];
      double alpha = rr / pAp;
#pragma omp parallel for schedule(static)
      for (long P = 0; P < N; P++) {
        psi[P] += alpha * p[P];
        r[P] -= alpha * Ap[P];
      }
      double rr_new = 0.0;
      for (long P = 0; P < N; P++) rr_new += r[P] * r[P];
      it++;
      rel = sqrt(rr_new / bb);
      if (rel < tol) break;
      double beta = rr_new / rr;
#pragma omp parallel for schedule(static)
      for (long P = 0; P < N; P++) p[P] = r[P] + beta * p[P];
      rr = rr_new;
    }
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;
  free(b);
  free(r);
  free(p);
  free(Ap);
  return (bb > 0.0 && rel >= tol) ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Nernst-Planck                                                            */
/* ------------------------------------------------------------------------ */

/* Bernoulli function B(x) = x / (exp(x) - 1), with its Taylor series near 0. */
static double bernoulli(double x) {
  if (fabs(x) < 1e-3) return 1.0 - x / 2.0 + x * x / 12.0 - x * x * x * x / 720.0;
  return x / expm1(x);
}

/* Inputs of the flux through face f of pore cell P for species (zi, Di):
 * the face Peclet number (advection plus migration against diffusion).
 * Returns the face kind; *Pf and *Cnb are set for the kinds that have them. */
static int np_face(int dim, int nx, int ny, int nz, const uint8_t *mask,
                   int walls, const double *u, const double *psi, const double *C,
                   double c0, int zi, double Di, double dx, double VT, int x,
                   int y, int z, int f, double *Pf, double *Cnb) {
  long N = (long)nx * ny * nz;
  long P = ((long)z * ny + y) * nx + x;
  long nb;
  int k = classify_face(mask, nx, ny, nz, walls, x, y, z, f, &nb);
  int a = f / 2;                      /* axis of the face normal */
  double sgn = (f % 2 == 0) ? 1.0 : -1.0;
  double uP = u[a * N + P];
  double unb, psinb;
  if (k == FACE_FLUID) {
    unb = u[a * N + nb];
    psinb = psi[nb];
    *Cnb = C[nb];
  } else if (k == FACE_INLET) {
    unb = uP;       /* ghost velocity copies the pore cell */
    psinb = 0.0;    /* bulk feed potential */
    *Cnb = c0;      /* feed concentration */
  } else if (k == FACE_OUTLET) {
    unb = uP;
    psinb = psi[P];
    *Cnb = C[P];    /* zero gradient */
  } else {
    return k;
  }
  double uf = 0.5 * (uP + unb) * sgn;
  *Pf = uf * dx / Di - zi * (psinb - psi[P]) / VT;
  (void)dim;
  return k;
}

double orc_np_dt(int dim, int nx, int ny, int nz, const uint8_t *mask,
                 int lateral_walls, const double *u, const double *psi, int ns,
                 const int *z, const double *D, double dx, double Ka,
                 double VT, double safety) {
  double maxrate = 0.0;
  long N = (long)nx * ny * nz;
  double *dummyC = (double *)calloc((size_t)N, sizeof(double));
  for (int i = 0; i < ns; i++) {
    double Keff = Ka / (1.0 + Ka * dx / (2.0 * D[i]));
#pragma omp parallel for collapse(2) schedule(static) reduction(max : maxrate)
    for (int zz = 0; zz < nz; zz++)
      for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
          long P = ((long)zz * ny + y) * nx + x;
          if (mask[P]) continue;
          double rate = 0.0;
          for (int f = 0; f < 2 * dim; f++) {
            double Pf = 0.0, Cnb = 0.0;
            int k = np_face(dim, nx, ny, nz, mask, lateral_walls, u, psi, dummyC,
                            0.0, z[i], D[i], dx, VT, x, y, zz, f, &Pf, &Cnb);
            if (k == FACE_SOLID)
              rate += Keff / dx;
            else if (k != FACE_WALL)
              rate += D[i] / (dx * dx) * bernoulli(-Pf);
          }
          if (rate > maxrate) maxrate = rate;
        }
  }
  free(dummyC);
  return (maxrate > 0.0) ? safety / maxrate : INFINITY;
}

int orc_np_run(int dim, int nx, int ny, int nz, const uint8_t *mask,
               int lateral_walls, const double *u, const double *psi, int ns,
               const int *z, const double *D, double dx, double Ka, double c0,
               double VT, double dt, long n_steps, double *C, double *Gamma,
               double *In, double *Out) {
  if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || nz < 1 || ns < 1) return -1;
  if (dim == 2 && nz != 1) return -1;
  long N = (long)nx * ny * nz;
  long rows = (long)ny * nz;
  double area = (dim == 2) ? dx : dx * dx; /* face area (per metre in 2D) */
  double *Cn = (double *)malloc(sizeof(double) * N);
  /* per-row sums of the adsorbed, inflow and outflow fluxes (each row summed
   * along x, the rows then summed in row order: the same totals whatever
   * the number of threads) */
  double *racc = (double *)malloc(sizeof(double) * 3 * rows);
  for (long n = 0; n < n_steps; n++) {
    for (int i = 0; i < ns; i++) {
      double *Ci = C + (long)i * N;
      double Keff = Ka / (1.0 + Ka * dx / (2.0 * D[i]));
#pragma omp parallel for collapse(2) schedule(static)
      for (int zz = 0; zz < nz; zz++)
        for (int y = 0; y < ny; y++) {
          double gam = 0.0, in = 0.0, out = 0.0;
          for (int x = 0; x < nx; x++) {
            long P = ((long)zz * ny + y) * nx + x;
            if (mask[P]) {
              Cn[P] = Ci[P];
              continue;
            }
            double sumJ = 0.0;
            for (int f = 0; f < 2 * dim; f++) {
              double Pf = 0.0, Cnb = 0.0, J;
              int k = np_face(dim, nx, ny, nz, mask, lateral_walls, u, psi, Ci,
                              c0, z[i], D[i], dx, VT, x, y, zz, f, &Pf, &Cnb);
              if (k == FACE_WALL) continue;
              if (k == FACE_SOLID) {
                J = Keff * Ci[P]; /* Eq. 6: adsorption into the carbon surface */
                gam += J;
              } else {
                J = D[i] / dx * (bernoulli(-Pf) * Ci[P] - bernoulli(Pf) * Cnb);
                if (k == FACE_INLET) in -= J;
                if (k == FACE_OUTLET) out += J;
              }
              sumJ += J;
            }
            Cn[P] = Ci[P] - dt / dx * sumJ;
          }
          long row = (long)zz * ny + y;
          racc[3 * row] = gam;
          racc[3 * row + 1] = in;
          racc[3 * row + 2] = out;
        }
      memcpy(Ci, Cn, sizeof(double) * N);
      double gam = 0.0, in = 0.0, out = 0.0;
      for (long row = 0; row < rows; row++) {
        gam += racc[3 * row];
        in += racc[3 * row + 1];
        out += racc[3 * row + 2];
      }
      Gamma[i] += dt * area * gam;
      In[i] += dt * area * in;
      Out[i] += dt * area * out;
    }
  }
  free(Cn);
  free(racc);
  return 0;
}

/* The transport operator of one species as a sparse matrix: the face fluxes
 * of orc_np_run are affine in C, (1/dx) sum_f J_f(C)_P = (A C)_P - b_P, with
 *   pore neighbour: A_PP += (D/dx^2) B(-P_f),  A_P,nb += -(D/dx^2) B(P_f)
 *   inlet ghost:    A_PP += (D/dx^2) B(-P_f),  b_P += (D/dx^2) B(P_f) c0
 *   outlet ghost:   A_PP += (D/dx^2) (B(-P_f) - B(P_f))
 *   solid face:     A_PP += K_eff / dx                          (Eq. 6)
 * (rows of solid cells are empty).  The triplets (row, col, val) go to
 * rows/cols/vals (room for 7 per cell; duplicates are to be summed), their
 * count to *nnz; b (N) is overwritten. */
int orc_np_operator(int dim, int nx, int ny, int nz, const uint8_t *mask,
                    int lateral_walls, const double *u, const double *psi, int zi,
                    double Di, double dx, double Ka, double c0, double VT, long *rows,
                    long *cols, double *vals, long *nnz, double *b) {
  if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || nz < 1) return -1;
  long N = (long)nx * ny * nz;
  double Keff = Ka / (1.0 + Ka * dx / (2.0 * Di));
  double *dummyC = (double *)calloc((size_t)N, sizeof(double));
  long k = 0;
  for (int zz = 0; zz < nz; zz++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        long P = ((long)zz * ny + y) * nx + x;
        b[P] = 0.0;
        if (mask[P]) continue;
        double diag = 0.0;
        for (int f = 0; f < 2 * dim; f++) {
          double Pf = 0.0, Cnb = 0.0;
          long nb;
          int kind = np_face(dim, nx, ny, nz, mask, lateral_walls, u, psi, dummyC, c0, zi, Di,
                             dx, VT, x, y, zz, f, &Pf, &Cnb);
          if (kind == FACE_WALL) continue;
          if (kind == FACE_SOLID) {
            diag += Keff / dx;
          } else if (kind == FACE_FLUID) {
            diag += Di / (dx * dx) * bernoulli(-Pf);
            classify_face(mask, nx, ny, nz, lateral_walls, x, y, zz, f, &nb);
            rows[k] = P;
            cols[k] = nb;
            vals[k] = -Di / (dx * dx) * bernoulli(Pf);
            k++;
          } else if (kind == FACE_INLET) {
            diag += Di / (dx * dx) * bernoulli(-Pf);
            b[P] += Di / (dx * dx) * bernoulli(Pf) * c0;
          } else { /* outlet: the ghost copies the cell */
            diag += Di / (dx * dx) * (bernoulli(-Pf) - bernoulli(Pf));
          }
        }
        rows[k] = P;
        cols[k] = P;
        vals[k] = diag;
        k++;
      }
  *nnz = k;
  free(dummyC);
  return 0;
}

/* Coupled Poisson-Nernst-Planck (Eq. 3-5): before every block of K explicit
 * steps, the potential is solved from Eq. 4 with the net charge density of
 * Eq. 5 of the current concentrations (Laplace operator, Dirichlet psi_s at
 * solid faces, psi = 0 in the inlet feed, no flux at the outlet), then the
 * K steps run in that potential.  eps_coef = F dx^2 / (eps_r eps_0), so the
 * source of cell P is eps_coef * sum_i z_i C_i(P).  psi (N) receives the last
 * potential solved. */
int orc_pnp_run(int dim, int nx, int ny, int nz, const uint8_t *mask,
                int lateral_walls, const double *u, int ns, const int *z,
                const double *D, double dx, double Ka, double c0, double VT,
                double dt, long n_steps, long K, double psi_s, double eps_coef,
                double psi_tol, double *C, double *Gamma, double *In, double *Out,
                double *psi) {
  if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || nz < 1 || ns < 1 || K < 1) return -1;
  long N = (long)nx * ny * nz;
  double *src = (double *)malloc(sizeof(double) * N);
  int st = 0;
  for (long s = 0; s < n_steps && st >= 0; s += K) {
    for (long P = 0; P < N; P++) {
      double q = 0.0;
      if (!mask[P])
        for (int i = 0; i < ns; i++) q += z[i] * C[(long)i * N + P];
      src[P] = eps_coef * q;
    }
    int it;
    double rel;
    st = orc_psi_src(dim, nx, ny, nz, mask, lateral_walls, psi_s, 0.0, src, psi_tol,
                     1000000, psi, &it, &rel);
    if (st < 0) break;
    long steps = n_steps - s < K ? n_steps - s : K;
    st = orc_np_run(dim, nx, ny, nz, mask, lateral_walls, u, psi, ns, z, D, dx, Ka, c0, VT,
                    dt, steps, C, Gamma, In, Out);
  }
  free(src);
  return st < 0 ? st : 0;
}

/* Number of host threads of the parallel loops (OpenMP; 1 without it). */
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
