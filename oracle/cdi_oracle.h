/*
 * FP64 CPU oracle for the pore-scale capacitive-deionization model of
 * Liu, Waugh, Komini Babu, Spendelow and Kang (arXiv 2110.13055).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
 * Python binding) may include, link, load or call this code; only the tests,
 * the smoke check and the benchmark's CPU-baseline leg do.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * Conventions shared with the callers (not with the CUDA path):
 *   - grids are x-fastest: cell (x, y, z) is at ((z*ny)+y)*nx + x; 2D has nz=1;
 *   - mask: uint8, 1 = solid, 0 = pore;
 *   - vector fields are component-major: all u_x, then all u_y (then u_z);
 *   - every routine returns 0 on success, a negative value on bad arguments.
 */
#ifndef CDI_ORACLE_H
#define CDI_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Lattice Boltzmann Stokes solve (Sec. 2, Eq. 7-8, bounce-back and body
 * force).  The flow grid is the mask mirrored along x when `mirror` is set
 * (2*nx cells in x), periodic in x; lateral directions periodic, or bounded
 * by bounce-back walls when `lateral_walls` is set.  Steps until the K-lag
 * velocity residual drops below `tol` at a check (every `check_every` steps),
 * or `max_steps` (a multiple of check_every) are done; tol <= 0 runs exactly
 * max_steps.  u_flow receives the lattice-unit velocity on the whole flow grid
 * (dim blocks of NX*ny*nz).  Returns 1 if tol > 0 and it was not reached. */
int orc_lbm(int dim, int nx, int ny, int nz, const uint8_t *mask, int mirror,
            int lateral_walls, double tau, double force_x, double tol,
            int check_every, long max_steps, double *u_flow, long *steps_done,
            double *residual);

/* Frozen potential (Eq. 4 with Dirichlet psi_s at solid faces; screened by
 * kdx2 = (dx/lambda_D)^2, Laplace when kdx2 = 0).  Conjugate gradients to a
 * relative residual of `tol`.  psi (nx*ny*nz, volts) is 0 in solid cells. */
int orc_psi(int dim, int nx, int ny, int nz, const uint8_t *mask,
            int lateral_walls, double psi_s, double kdx2, double tol,
            int max_iter, double *psi, int *iters, double *relres);

/* The same solve with an additional right-hand side: src (N values, ignored
 * in solid cells) is the charge term dx^2 rho_e / (eps_r eps_0) of Eq. 4
 * (NULL: none). */
int orc_psi_src(int dim, int nx, int ny, int nz, const uint8_t *mask,
                int lateral_walls, double psi_s, double kdx2, const double *src,
                double tol, int max_iter, double *psi, int *iters, double *relres);

/* Explicit time step bound: safety / max over cells and species of the
 * outflow rate (the sum of the exponentially fitted outflow coefficients). */
double orc_np_dt(int dim, int nx, int ny, int nz, const uint8_t *mask,
                 int lateral_walls, const double *u, const double *psi, int ns,
                 const int *z, const double *D, double dx, double Ka,
                 double VT, double safety);

/* n_steps explicit finite-volume Nernst-Planck steps (Eq. 3) with the
 * adsorption flux of Eq. 6 at solid faces, a constant-concentration inlet at
 * x = -1/2 and a zero-gradient outlet at x = nx - 1/2.  C (ns*N) is updated in
 * place; Gamma, In and Out (ns each) are accumulated (mol, or mol per metre of
 * depth in 2D). */
int orc_np_run(int dim, int nx, int ny, int nz, const uint8_t *mask,
               int lateral_walls, const double *u, const double *psi, int ns,
               const int *z, const double *D, double dx, double Ka, double c0,
               double VT, double dt, long n_steps, double *C, double *Gamma,
               double *In, double *Out);

/* Coupled Poisson-Nernst-Planck (Eq. 3-5): the potential is re-solved from
 * the charge density of the current concentrations (eps_coef = F dx^2 /
 * (eps_r eps_0)) before every block of K steps; otherwise as orc_np_run.
 * psi receives the last potential solved. */
int orc_pnp_run(int dim, int nx, int ny, int nz, const uint8_t *mask,
                int lateral_walls, const double *u, int ns, const int *z,
                const double *D, double dx, double Ka, double c0, double VT,
                double dt, long n_steps, long K, double psi_s, double eps_coef,
                double psi_tol, double *C, double *Gamma, double *In, double *Out,
                double *psi);

/* The transport operator of species (zi, Di): (1/dx) sum_f J_f(C) = A C - b
 * with the face rules of orc_np_run, as (row, col, val) triplets (room for
 * 7 per cell; duplicates to be summed) and b (N).  The implicit (backward
 * Euler) finite-volume step of Sec. 2 solves (I + dt A) C' = C + dt b. */
int orc_np_operator(int dim, int nx, int ny, int nz, const uint8_t *mask,
                    int lateral_walls, const double *u, const double *psi, int zi,
                    double Di, double dx, double Ka, double c0, double VT, long *rows,
                    long *cols, double *vals, long *nnz, double *b);

/* Host threads used by the loops above (OpenMP).  The loops that run in
 * parallel write disjoint outputs; sums are formed in a fixed order (per
 * grid row, then over rows), so results do not depend on the thread count. */
void orc_set_threads(int n);
int orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
