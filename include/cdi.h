/*
 * cdi.h - C ABI of the GB300 pore-scale capacitive-deionization solver.
 *
 * Method: Liu, Waugh, Komini Babu, Spendelow, Kang, "Numerical Modeling of Ion
 * Transport and Adsorption in Porous Media: A Pore-scale Study for Capacitive
 * Deionization Desalination" (arXiv 2110.13055).
 *
 * One domain = one voxel image of a porous electrode.  The calls follow the
 * paper's pipeline:
 *   cdi_create_domain   voxel mask in (Sec. 2: one grid block per voxel)
 *   cdi_solve_flow      Stokes flow by lattice Boltzmann to steady state
 *                       (Sec. 2, Eq. 1-2 solved with Eq. 7-8, bounce-back,
 *                       body force, mirror image along the flow axis)
 *   cdi_set_potential   electric potential (Eq. 4-5, Dirichlet at the solid)
 *   cdi_init_transport  species, feed concentration, adsorption constant,
 *                       explicit time step (Sec. 4: saturated initial state)
 *   cdi_step_transport  explicit finite-volume Nernst-Planck steps (Eq. 3)
 *                       with the adsorption flux of Eq. 6 at solid faces
 *   cdi_query_*         adsorbed amount, outlet concentration (Sec. 4.1),
 *                       mass balance, vertically averaged profiles
 *
 * Conventions
 *   - Grids are x-fastest: cell (x,y,z) is element ((z*ny)+y)*nx + x; x is the
 *     flow direction (inlet at x = -1/2, outlet at x = nx - 1/2).
 *   - The mask is uint8, 1 = solid (carbon), 0 = pore; host memory owned by
 *     the caller and copied by cdi_create_domain.
 *   - All device memory belongs to the domain.  It is obtained from the
 *     caller's allocator when one is given, else by stream-ordered allocation
 *     on the domain's stream (cudaMallocAsync/cudaFreeAsync, which do not
 *     synchronise the device); everything is released by
 *     cdi_destroy_domain.
 *   - Work runs on the domain's stream: the caller's stream if given, else a
 *     stream the domain creates.  cdi_step_transport returns without waiting;
 *     the queries and cdi_copy_field wait for the stream.
 *   - Calls on one domain must not overlap (not thread-safe per domain);
 *     different domains are independent.
 *   - Every call returns a cdi_status; on failure cdi_last_error(dom) gives a
 *     message (cdi_last_error(NULL) for failures of cdi_create_domain).
 *     A call made out of order (e.g. stepping before cdi_init_transport)
 *     returns CDI_ERR_STATE and changes nothing.
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     computes returns CDI_ERR_CUDA.
 */
#ifndef CDI_H
#define CDI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cdi_domain cdi_domain; /* opaque; owned by the library */

typedef enum {
  CDI_OK = 0,
  CDI_ERR_INVALID_ARG = 1,   /* bad sizes, values or null pointers */
  CDI_ERR_OOM = 2,           /* an allocation failed; nothing leaked */
  CDI_ERR_CUDA = 3,          /* a CUDA call failed (message has the detail) */
  CDI_ERR_NOT_CONVERGED = 4, /* max_steps / max_iter reached; state is valid */
  CDI_ERR_TIMEOUT = 5,       /* reserved for bounded device-side waits */
  CDI_ERR_STATE = 6          /* call out of order */
} cdi_status;

typedef enum {
  CDI_FP64 = 0,      /* populations, velocity, potential, concentrations in FP64 */
  CDI_FP32 = 1,      /* the same fields stored and updated in FP32; reductions,
                        the potential solve and all accumulators stay FP64 */
  CDI_FP32_SPLIT = 2, /* as CDI_FP32, but every population and every
                         concentration is an unevaluated pair of FP32 words
                         (hi + lo) updated with error-free FP32
                         transformations: FP64-class accuracy at FP32
                         arithmetic rates, twice the memory of those fields */
  CDI_BF16_POP = 3,   /* as CDI_FP32, but the populations are stored in BF16
                         (shifted, f - w; collision in FP32): half the
                         population bytes of FP32, about 3 significant digits;
                         an option whose flow error is measured and reported,
                         not held to the FP32 bounds */
  CDI_FP32_CPAIR = 4  /* FP32 populations (as CDI_FP32) and FP32-pair
                         concentrations (as CDI_FP32_SPLIT): for flows that
                         converge in plain FP32 while the transport runs many
                         thousands of steps, over which FP32 rounding of the
                         concentrations would build up */
} cdi_precision;

/* Optional device allocator (e.g. a framework's caching allocator).
 * alloc returns NULL on failure; free receives the pointer and its size. */
typedef struct {
  void *(*alloc)(size_t bytes, void *ctx);
  void (*free)(void *ptr, size_t bytes, void *ctx);
  void *ctx;
} cdi_allocator;

typedef struct {
  int dim;           /* 2 (D2Q9, 5-point faces) or 3 (D3Q19, 7-point) */
  int nx, ny, nz;    /* voxels; nz must be 1 when dim == 2 */
  double dx_m;       /* voxel edge in metres (> 0) */
  int lateral_walls; /* 0: y (and z) periodic; 1: inert walls there */
  int mirror_x;      /* 1: flow grid = image + its mirror image along x,
                        periodic in x (Sec. 2's mirror boundary); 0: the image
                        alone, periodic in x */
  int precision;     /* cdi_precision */
} cdi_domain_desc;

/* Lattice Boltzmann flow parameters (Sec. 2, Eq. 7-8). */
typedef struct {
  double tau;          /* BGK relaxation time (> 1/2); nu = (tau - 1/2) / 3 */
  double force_lu;     /* body force along x in lattice units (the pressure
                          gradient of Sec. 2); the flow is linear in it */
  double tol;          /* steady state when ||u(t)-u(t-K)|| / ||u(t)|| < tol
                          over pore sites; tol <= 0 runs exactly max_steps */
  int check_every;     /* K: even, >= 2 */
  int64_t max_steps;   /* multiple of check_every, >= 0 */
  double U_target_mps; /* pore-mean x velocity U = sum(u) / (N phi) of Sec. 4
                          that the lattice velocity is scaled to (m/s) */
} cdi_flow_params;

/* Potential parameters (Eq. 4-5, Eq. 10). */
typedef struct {
  double T_K;          /* temperature (K) */
  double eps_r;        /* relative permittivity of the solution */
  double c_bulk_molm3; /* bulk salt concentration setting the Debye length of
                          Eq. 10's exponent */
  double lambda_D_m;   /* > 0 overrides that Debye length */
  int mode;            /* 0: screened (Debye-Hueckel) field; 1: Laplace;
                          2: nonlinear Poisson-Boltzmann (Eq. 4 with the
                          Boltzmann charge of Eq. 9 for a 1:1 salt, whose 1D
                          solution is Eq. 10), by Newton's method around the
                          conjugate-gradient solve */
  double tol;          /* relative residual of the conjugate-gradient solve
                          (mode 2: of the nonlinear equation against the
                          surface terms; each linear solve runs to tol / 10) */
  int max_iter;        /* conjugate-gradient iterations (mode 2: per Newton
                          step, at most 200 steps) */
} cdi_elec_params;

typedef struct {
  int z;        /* valence (Eq. 3) */
  double D_m2s; /* diffusion coefficient (Eq. 3) */
} cdi_species;

/* Field ids for cdi_copy_field (all copied out as double). */
enum {
  CDI_FIELD_U_LATTICE = 0, /* dim*NX*ny*nz: flow-grid velocity, lattice units,
                              component-major; NX = 2 nx with mirror_x */
  CDI_FIELD_U = 1,         /* dim*nx*ny*nz: scaled velocity (m/s) */
  CDI_FIELD_PSI = 2,       /* nx*ny*nz: potential (V), 0 in solid */
  CDI_FIELD_C = 3          /* CDI_FIELD_C + k: species k concentration
                              (mol/m^3), nx*ny*nz, 0 in solid */
};

typedef struct {
  double flow_ms;      /* device time of the LBM step kernels */
  int64_t flow_launches;
  double flow_check_ms;/* device time of the residual checks */
  double psi_ms;       /* device time of the potential solve */
  int64_t psi_iters;
  double np_ms;        /* device time of the Nernst-Planck step kernels */
  int64_t np_launches;
  int64_t kernel_launches; /* all kernels this domain launched */
  int32_t lbm_block;   /* threads per block of the LBM step and of the */
  int32_t np_block;    /* transport step, picked by the library's autotuner
                          on the first solve (timing only: every block size
                          computes the same bits); 0 before it ran */
  int32_t lbm_shape;   /* the launch shapes themselves (see */
  int32_t np_shape;    /* cdi_set_launch_shapes); -1 before they are chosen */
} cdi_timing;

/* Create a domain from a voxel mask (Sec. 2: marker-and-cell grid, one grid
 * block per image voxel).  Copies the mask to the device, builds the flow
 * and face neighbour tables there and allocates every field.  The mask needs
 * at least one pore cell in the inlet column x = 0.  stream: a cudaStream_t
 * or NULL.  On success *out owns the domain. */
cdi_status cdi_create_domain(const cdi_domain_desc *desc, const uint8_t *mask,
                             const cdi_allocator *alloc, void *stream,
                             cdi_domain **out);

/* Run the lattice Boltzmann Stokes solve from rest (Sec. 2, Eq. 7-8): BGK
 * collision with the Stokes-linear equilibrium, halfway bounce-back at solid
 * links, body force along x, mirror domain.  Stops at the first residual
 * check below tol, else after max_steps (CDI_ERR_NOT_CONVERGED, state kept).
 * Then scales the velocity to U_target_mps.  Blocks until done.
 * steps_out / residual_out may be NULL. */
cdi_status cdi_solve_flow(cdi_domain *dom, const cdi_flow_params *p,
                          int64_t *steps_out, double *residual_out);

/* Stokes flow of several electrode images at once (the geometry studies of
 * Sec. 4-5 solve Eq. 7-8 on many images): every domain runs the lattice
 * Boltzmann solve of cdi_solve_flow, but all of them advance together, one
 * kernel launch per step over the pore sites of every domain still running;
 * each domain takes its own residual every check_every steps and leaves the
 * batch at its first check below tol (or at max_steps), so its steps,
 * residual and field equal, bit for bit, those of cdi_solve_flow with the
 * same parameters.  Then each velocity is scaled to U_target_mps.
 *   doms: n_doms >= 1 distinct domains on the current device, all of the
 *     same dimension and precision; doms[0]'s stream runs the batch and
 *     doms[0]'s allocator provides a small member table for the call.
 *   steps_out, residual_out, status_out: host arrays of n_doms (any may be
 *     NULL); status_out[i] is CDI_OK, CDI_ERR_NOT_CONVERGED (state kept, as
 *     cdi_solve_flow) or CDI_ERR_CUDA (diverged).
 * Returns CDI_OK when every domain converged, CDI_ERR_NOT_CONVERGED when
 * some did not, another error when the batch itself failed (reported on
 * doms[0]).  Blocks until done. */
cdi_status cdi_solve_flow_batch(cdi_domain *const *doms, int n_doms,
                                const cdi_flow_params *p, int64_t *steps_out,
                                double *residual_out, int *status_out);

/* Rescale the solved Stokes field to another pore-mean velocity U = sum(u) /
 * (N phi) of Sec. 4 (Eq. 2 is linear in the force, so one solve serves every
 * velocity of the Pe sweeps of Sec. 4.1).  Requires a
 * solved flow; invalidates an initialised transport state. */
cdi_status cdi_set_velocity(cdi_domain *dom, double U_target_mps);

/* Solve the potential with surface value psi_s = -applied_V on every solid
 * face (Eq. 4 with the Dirichlet condition of Sec. 2), psi = 0 in the inlet
 * feed, no flux through the outlet and lateral walls.  Invalidates an
 * initialised transport state.  iters_out / relres_out may be NULL. */
cdi_status cdi_set_potential(cdi_domain *dom, double applied_V,
                             const cdi_elec_params *p, int *iters_out,
                             double *relres_out);

/* Set up transport (Sec. 4): n_species (1..4) ions, every pore cell at c0
 * (the saturated start), feed at c0, adsorption constant Ka (Eq. 6) on every
 * solid face.  dt_s > 0 fixes the time step; dt_s == 0 takes
 * 0.9 / (largest outflow rate of any cell and species), which keeps the
 * explicit update positive.  Needs a solved flow (or U_target 0 and no flow
 * solve: then u = 0) and a potential.  Resets Gamma/In/Out to zero. */
cdi_status cdi_init_transport(cdi_domain *dom, const cdi_species *sp,
                              int n_species, double c0_molm3, double Ka_mps,
                              double dt_s, double *dt_used);

/* Coupled Poisson-Nernst-Planck (Eq. 3-5).  every_steps = K > 0: before
 * every block of K transport steps (counted from cdi_init_transport),
 * cdi_step_transport re-solves Eq. 4 with the net charge density of Eq. 5 of
 * the current concentrations, rho_e = F sum_i z_i C_i, as its source
 * (Laplace operator, Dirichlet -applied_V at solid faces, 0 in the inlet
 * feed, no flux at the outlet; eps_r, tolerance and iteration limit of the
 * last cdi_set_potential), and steps in that potential.  0 (the default):
 * the potential stays frozen.  Needs cdi_set_potential first (CDI_ERR_STATE).
 * The explicit scheme resolves the coupling only where the time step is
 * well below the charge relaxation time eps_r eps_0 / conductivity (an
 * electric double layer resolved by the grid, as in Sec. 3's validation);
 * the caller chooses dt accordingly.  With coupling on, cdi_step_transport
 * waits for the stream at every re-solve.  Sweeps and batches always use
 * frozen potentials. */
cdi_status cdi_set_coupling(cdi_domain *dom, int64_t every_steps);

/* Implicit finite-volume transport (Sec. 2: the paper integrates Eq. 3 with
 * an implicit finite-volume scheme).  tol > 0: every later
 * cdi_step_transport step is a backward Euler step, (I + dt A) C' = C +
 * dt b per species with the face fluxes of the explicit step (Eq. 3, Eq. 6),
 * solved by Jacobi-preconditioned BiCGStab in FP64 to a relative residual
 * below tol within max_iter iterations (else CDI_ERR_NOT_CONVERGED with the
 * step not taken).  The step is unconditionally stable and keeps C >= 0, so
 * cdi_init_transport's dt_s may exceed the explicit bound by orders of
 * magnitude; the adsorbed/inflow/outflow accounts take the fluxes at the new
 * concentrations (the mass balance closes as in the explicit scheme).
 * tol <= 0 returns to the explicit scheme.  With cdi_set_coupling the
 * potential is still re-solved before every block of K steps.  Sweeps and
 * batches always step explicitly.  cdi_step_transport waits for the stream
 * at every linear iteration check.  Device memory: (9 or 11 + 7 / species)
 * FP64 values per pore cell, taken on the first call. */
cdi_status cdi_set_implicit(cdi_domain *dom, double tol, int max_iter);

/* Launch shapes of the two step kernels (the paper has no counterpart: it
 * states the method, not its launch configuration).  By default (-1) an autotuner
 * times every candidate shape of the LBM step (0-5) and of the transport
 * step (0-9) on the domain's first flow solve and first transport
 * initialisation and keeps the fastest; every shape computes the same bits
 * (the arithmetic of a lattice site or pore cell, and the per-warp account
 * slots, do not depend on the shape), so the choice changes speed only.
 * lbm_shape / np_shape in range fix the shape from the next step on; -1
 * returns the kernel to the autotuner (its cached choice, if any).  Shapes
 * are those of the FP32 kernels; FP64 maps the resident-grid shapes to plain
 * launches.  Out-of-range values fail with CDI_ERR_INVALID_ARG and change
 * nothing. */
cdi_status cdi_set_launch_shapes(cdi_domain *dom, int32_t lbm_shape, int32_t np_shape);

/* Advance n_steps >= 0 transport steps (Eq. 3 with Eq. 6): explicit unless
 * cdi_set_implicit chose the implicit scheme; explicit steps are
 * asynchronous. */
cdi_status cdi_step_transport(cdi_domain *dom, int64_t n_steps);

/* One member of a transport sweep. */
typedef struct {
  double U_mps;     /* pore-mean velocity (the solved flow rescaled, Sec. 4) */
  double applied_V; /* surface potential -applied_V (Eq. 4, Sec. 2) */
} cdi_combo;

/* Batched transport sweep on one geometry: the parameter studies of Sec. 4.1
 * (velocity), Sec. 4.2 (potential) and Sec. 5 run many transport problems on
 * one electrode image.  Every member reuses the domain's solved Stokes flow
 * rescaled to its velocity (the flow is linear in the driving force, Eq. 2),
 * members with equal applied_V share one potential solve, and all members
 * advance together: one fused kernel launch per step reads the geometry once
 * for all of them.  Each member takes its own explicit time step (the bound
 * of cdi_init_transport) and its result equals, bit for bit, that of a single
 * run (cdi_set_velocity, cdi_set_potential, cdi_init_transport,
 * cdi_step_transport, queries) with the same arguments.  Every member starts
 * from the saturated state (c0) and runs n_steps steps.
 *   gamma_out, cout_out: host, n_combos * n_species doubles (member-major):
 *     adsorbed amount and outlet concentration as cdi_query_adsorbed and
 *     cdi_query_outlet report them;  dt_out: n_combos doubles or NULL.
 * Needs a solved flow; blocks until done.  Replaces the domain's potential
 * and transport state (set them again before cdi_step_transport).  Device
 * memory for the members is taken from the domain's allocator for the call
 * only: about n_combos * (dim + 8) * 4 bytes per cell in FP32. */
cdi_status cdi_sweep_transport(cdi_domain *dom, const cdi_combo *combos, int n_combos,
                               const cdi_elec_params *p, const cdi_species *sp,
                               int n_species, double c0_molm3, double Ka_mps,
                               int64_t n_steps, double *gamma_out, double *cout_out,
                               double *dt_out);

/* Batched transport over several geometries: the parameter studies of
 * Sec. 4.1, 4.2 and Sec. 5 repeated over many electrode images.  Every
 * (domain, combination) pair is a member (member index i * n_combos + c for
 * domain i, combination c); each domain prepares its members exactly as
 * cdi_sweep_transport does (rescaled flow, one potential per distinct
 * applied_V, its own time step), and then all members of all domains advance
 * together: one fused kernel launch per step walks the members' cell blocks,
 * whatever their sizes.  Each member's result equals, bit for bit, that of a
 * single run of its domain with the same arguments.
 *   doms: n_doms >= 1 distinct domains on the current device, all of the same
 *     dimension and precision, each with a solved flow.  doms[0] leads: its
 *     stream runs the batch and its allocator provides the members' device
 *     memory for the call only (about (dim + 8) * 4 bytes per pore cell per
 *     member in FP32, plus one potential per domain and applied_V).
 *   gamma_out, cout_out: host, n_doms * n_combos * n_species doubles;
 *   dt_out: n_doms * n_combos doubles or NULL.
 * Blocks until done; replaces every domain's potential and transport state.
 * An error in a domain's preparation is reported on doms[0]. */
cdi_status cdi_sweep_batch(cdi_domain *const *doms, int n_doms, const cdi_combo *combos,
                           int n_combos, const cdi_elec_params *p, const cdi_species *sp,
                           int n_species, double c0_molm3, double Ka_mps, int64_t n_steps,
                           double *gamma_out, double *cout_out, double *dt_out);

/* Adsorbed amount per species since cdi_init_transport (the time integral of
 * the Eq. 6 flux over the solid faces; the adsorbed amount of Sec. 4.1): mol
 * (3D) or mol per metre of depth (2D).  Waits for the stream. */
cdi_status cdi_query_adsorbed(cdi_domain *dom, double *per_species);

/* Outlet concentration per species (Sec. 4.1), flux weighted over the pore
 * cells of the last column: sum(u_x C) / sum(u_x) (plain mean if the sum of
 * u_x is 0).  Waits for the stream. */
cdi_status cdi_query_outlet(cdi_domain *dom, double *per_species);

/* Per species: dissolved amount M = sum C dx^d, adsorbed Gamma, inflow In
 * and outflow Out (all FP64; M + Gamma + Out - In is conserved, since Eq. 3
 * is solved in conservative form with the Eq. 6 flux at solid faces).  Any
 * pointer may be NULL.  Waits for the stream. */
cdi_status cdi_query_mass_balance(cdi_domain *dom, double *M, double *Gamma,
                                  double *In, double *Out);

/* Geometry of the image (Sec. 4): porosity phi = pore cells / cells, and the
 * specific surface s = pore-solid interface area / image volume (1/m; per
 * metre of depth folded in for 2D, i.e. interface length / image area).
 * Faces across the inlet and outlet planes do not count, nor, with lateral
 * walls, faces across the lateral image boundary; with periodic lateral
 * boundaries the wrapped neighbour decides.  With them Sec. 4 defines
 * l_c = pi / s, Pe = U l_c / D and Da = Ka l_c / D.  Waits for the stream. */
cdi_status cdi_query_geometry(cdi_domain *dom, double *porosity,
                              double *specific_surface_per_m);

/* Dimensionless groups and removal figures of Sec. 4 and Sec. 4.1 for the
 * current transport state (all per species k < n_species, FP64). */
typedef struct {
  double porosity;           /* phi = pore cells / cells */
  double specific_surface;   /* s (1/m), as cdi_query_geometry */
  double l_c_m;              /* characteristic length l_c = pi / s (Sec. 4) */
  double U_mps;              /* pore-mean x velocity U = sum(u_x) / (N phi) */
  double elapsed_s;          /* Delta t: transport steps since cdi_init_transport
                                times the time step */
  double Pe[4];              /* Peclet number U l_c / D_k (Sec. 4) */
  double Da[4];              /* Damkohler number Ka l_c / D_k (Sec. 4) */
  double removal[4];         /* salt removal P_rm = (C_in - C_out) / C_in with
                                C_in the feed and C_out the outlet
                                concentration of cdi_query_outlet (Sec. 4.1) */
  double amount[4];          /* U A P_rm Delta t / (V_t phi) of Sec. 4.1: A the
                                inlet cross-section (ny dx per metre of depth
                                in 2D, ny nz dx^2 in 3D), V_t = nx ny nz dx^d
                                the electrode volume; dimensionless (times
                                C_in: mol removed per m^3 of pore space) */
} cdi_derived;

/* The Pe, Da, l_c, U, P_rm and adsorbed-amount figures the paper reports
 * (Sec. 4: Pe = U l_c / D, Da = Ka l_c / D, U = sum u / (N phi), l_c =
 * pi / s; Sec. 4.1: P_rm and U A P_rm Delta t / (V_t phi)), evaluated for the
 * domain's geometry, velocity field and transport state.  Needs an
 * initialised transport (CDI_ERR_STATE).  Waits for the stream. */
cdi_status cdi_query_derived(cdi_domain *dom, cdi_derived *out);

/* Vertically averaged profile (Fig. 6, Fig. 9): the mean of species k over
 * the pore cells of each x column into out[nx] (0 for all-solid columns). */
cdi_status cdi_query_column_means(cdi_domain *dom, int species, double *out);

/* Copy a field to host memory as doubles (layouts in the CDI_FIELD_* list):
 * the fields the paper maps, e.g. the Na+ concentrations of Fig. 13-15.
 * count is the number of doubles host_dst holds; it must match exactly. */
cdi_status cdi_copy_field(cdi_domain *dom, int field, double *host_dst,
                          size_t count);

/* Device-time counters (CUDA events on the domain stream) since the last
 * reset; no counterpart in the paper.  Waits for the stream.  reset != 0
 * zeroes them afterwards. */
cdi_status cdi_query_timing(cdi_domain *dom, cdi_timing *out, int reset);

/* Dissolved amount and outlet concentration of caller-owned FP64 device
 * fields, with no device allocation by the library.  The paper has no
 * counterpart: this exists for callers that cannot let a library allocate
 * device memory (programs that manage all device memory in their own pool or
 * under a fixed budget, and loops where a cudaMalloc/cudaFree would
 * synchronise the device).
 *   C     device, n_species*nx*ny*nz doubles (species-major, x fastest)
 *   ux    device, nx*ny*nz doubles: x velocity (weights the outlet mean)
 *   mask  device, nx*ny*nz bytes, 1 = solid (excluded)
 *   out   device, 2*n_species doubles: out[k] = sum over pore cells of
 *         C_k dx^dim (mol, or mol per metre in 2D); out[n_species + k] =
 *         sum(u_x C_k)/sum(u_x) over the pore cells of the last column (plain
 *         mean if sum(u_x) = 0)
 *   stream  cudaStream_t or NULL; the call is asynchronous on it.
 * Scratch is a fixed static device array (34,304 bytes per device, held
 * until the process exits); n_species above 4 is rejected with
 * CDI_ERR_INVALID_ARG.  The first call on each device looks up the array's
 * device address, so make that first call before any stream capture; the
 * address is kept for the process, so calls after a cudaDeviceReset of that
 * device are not supported.  All calls share the array: calls that overlap
 * on the GPU race and must be serialised.  Errors: cdi_last_error(NULL). */
cdi_status cdi_transport_sums_noalloc(const double *C, const double *ux,
                                      const uint8_t *mask, int dim, int nx, int ny,
                                      int nz, int n_species, double dx_m,
                                      double *out, void *stream);

/* Checkpoint of the solver state (no counterpart in the paper; its
 * transient runs of Sec. 4-5 are long, and a run stopped and resumed gives
 * the same result bit for bit): the solved flow (populations and lattice
 * velocity), the potential, the scaled velocity, the transport state with
 * its adsorbed/inflow/outflow accounts, and the solver scalars (species, c0,
 * Ka, dt, step counts, coupling).  host_buf NULL: *bytes receives the size
 * needed.  Otherwise *bytes is the buffer's size on entry (too small:
 * CDI_ERR_INVALID_ARG with the size needed in *bytes) and the size written on
 * return.  Host memory of any kind; waits for the stream. */
cdi_status cdi_save_state(cdi_domain *dom, void *host_buf, size_t *bytes);

/* Restore a state saved by cdi_save_state (no counterpart in the paper)
 * into a domain created from the
 * same mask with the same grid options and precision (checked against the
 * state's header, including a hash of the mask: CDI_ERR_INVALID_ARG if they
 * differ).  Replaces the flow, potential and transport state; the next
 * cdi_step_transport continues the saved run.  Waits for the stream. */
cdi_status cdi_load_state(cdi_domain *dom, const void *host_buf, size_t bytes);

/* Message for the last failed call on dom (NULL: the last failed create on
 * this thread).  Valid until the next call on the same domain.  No
 * counterpart in the paper. */
const char *cdi_last_error(const cdi_domain *dom);

/* Release the domain and all its device memory.  NULL is ignored.  No
 * counterpart in the paper. */
void cdi_destroy_domain(cdi_domain *dom);

/* ABI version (major * 100 + minor); no counterpart in the paper. */
int cdi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CDI_H */
