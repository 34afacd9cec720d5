// Frozen electric potential (Eq. 4-5 with the Dirichlet surface value of
// Sec. 2) by Jacobi-preconditioned conjugate gradients in FP64.
//
// For a pore cell P the discrete equation is
//   sum_f T_f (psi_nb - psi_P) - kdx2 psi_P = 0,
// T_f = 1 towards a pore neighbour or the inlet feed (psi = 0), 2 towards a
// solid face (psi = psi_s at half a cell), 0 at the outlet and lateral walls;
// kdx2 = (dx / lambda_D)^2 screens the field (Debye-Hueckel linearisation of
// Eq. 4-5; 0 gives Laplace).  With the coupling of Eq. 3-5 on, the right-hand
// side also carries the charge term dx^2 rho_e / (eps_r eps_0) of every pore
// cell (Eq. 5 from the current concentrations).  All CG scalars stay on the
// device; the host only polls the convergence flag every few iterations.
#include <cmath>

#include "cdi_internal.cuh"

using namespace cdi;

namespace {

struct Geo {
  int nx, ny, nz, dim, walls;
  long long N;
};

// Face f of pore cell (x,y,z): 0 pore neighbour (index in *nb), 1 solid,
// 2 inlet feed, 3 no flux (outlet or lateral wall).
__device__ __forceinline__ int face_kind(const Geo &g, const NFlag *fl, long long P, int x,
                                         int y, int z, int f, long long *nb) {
  const int a = f >> 1;
  const int s = (f & 1) ? -1 : 1;
  if (a == 0) {
    if (x + s < 0) return 2;
    if (x + s >= g.nx) return 3;
    if ((fl[P] >> (kFaceBit + f)) & 1) return 1;
    *nb = P + s;
    return 0;
  }
  int Y = y, Z = z;
  if (a == 1) {
    Y = y + s;
    if (Y < 0 || Y >= g.ny) {
      if (g.walls) return 3;
      Y = (Y + g.ny) % g.ny;
    }
  } else {
    Z = z + s;
    if (Z < 0 || Z >= g.nz) {
      if (g.walls) return 3;
      Z = (Z + g.nz) % g.nz;
    }
  }
  if ((fl[P] >> (kFaceBit + f)) & 1) return 1;
  *nb = ((long long)Z * g.ny + Y) * g.nx + x;
  return 0;
}

__device__ __forceinline__ void coords(const Geo &g, long long P, int &x, int &y, int &z) {
  const long long row = P / g.nx;
  x = (int)(P - row * g.nx);
  z = (int)(row / g.ny);
  y = (int)(row - (long long)z * g.ny);
}

// diag, right-hand side, x = 0, r = b, z = r / diag, p = z; rz and b.b.
__global__ void __launch_bounds__(kRedThreads)
    k_cg_setup(Geo g, const NFlag *__restrict__ fl, double kdx2, double psi_s,
               const double *__restrict__ src, double tol,
               double *__restrict__ x, double *__restrict__ r, double *__restrict__ p,
               double *__restrict__ diag, double *__restrict__ part, unsigned int *counter,
               double *scal) {
  __shared__ double sm[2 * 32];
  double v[2] = {0.0, 0.0};
  for (long long P = blockIdx.x * (long long)blockDim.x + threadIdx.x; P < g.N;
       P += (long long)gridDim.x * blockDim.x) {
    x[P] = 0.0;
    if (fl[P] & 1) {
      r[P] = 0.0;
      p[P] = 0.0;
      diag[P] = 1.0;
      continue;
    }
    int cx, cy, cz;
    coords(g, P, cx, cy, cz);
    double dg = kdx2, b = src ? src[P] : 0.0;
    for (int f = 0; f < 2 * g.dim; f++) {
      long long nb;
      const int k = face_kind(g, fl, P, cx, cy, cz, f, &nb);
      if (k == 0 || k == 2) dg += 1.0;
      if (k == 1) {
        dg += 2.0;
        b += 2.0 * psi_s;
      }
    }
    diag[P] = dg;
    r[P] = b;
    p[P] = b / dg;
    v[0] += b * (b / dg);
    v[1] += b * b;
  }
  block_reduce<2>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = v[0];
    part[gridDim.x + blockIdx.x] = v[1];
  }
  if (last_block(counter, gridDim.x)) {
    combine_partials<2>(part, gridDim.x, v, sm, OpSum(), 0.0);
    if (threadIdx.x == 0) {
      scal[S_CG_RZ] = v[0];
      scal[S_CG_BB] = v[1];
      scal[S_CG_RR] = v[1];
      scal[S_CG_REL] = v[1] > 0.0 ? 1.0 : 0.0;
      scal[S_CG_DONE] = v[1] > 0.0 ? 0.0 : 1.0;
      scal[S_CG_TOL] = tol;
      scal[S_CG_IT] = 0.0;
      *counter = 0;
    }
  }
}

// One Newton step of the nonlinear Poisson-Boltzmann equation (Eq. 4 with
// the Boltzmann charge of Eq. 9 for a 1:1 salt; Eq. 10 in 1D), per pore cell
//   F_P(psi) = (A0 psi)_P - b_P + kdx2 V_T sinh(psi_P / V_T) = 0,
// A0 and b the face rules above.  Newton solves
//   (A0 + kdx2 cosh(psi / V_T)) psi' = b + kdx2 (psi cosh(psi / V_T) - V_T sinh(psi / V_T))
// by the CG below, warm-started at psi' = psi, so its first residual is -F.
// This kernel forms F (F.F and b.b into S_PB_FF / S_PB_BB: the Newton test),
// the CG's diagonal and its start (r = -F, p = r / diag, rz, and the
// right-hand side's b.b for the CG's relative residual).  psi is only read.
__global__ void __launch_bounds__(kRedThreads)
    k_pb_setup(Geo g, const NFlag *__restrict__ fl, double kdx2, double psi_s, double vt,
               double tol, const double *__restrict__ psi, double *__restrict__ r,
               double *__restrict__ p, double *__restrict__ diag, double *__restrict__ part,
               unsigned int *counter, double *scal) {
  __shared__ double sm[4 * 32];
  double v[4] = {0.0, 0.0, 0.0, 0.0};  // rz, rhs.rhs, F.F, b.b
  for (long long P = blockIdx.x * (long long)blockDim.x + threadIdx.x; P < g.N;
       P += (long long)gridDim.x * blockDim.x) {
    if (fl[P] & 1) {
      r[P] = 0.0;
      p[P] = 0.0;
      diag[P] = 1.0;
      continue;
    }
    int cx, cy, cz;
    coords(g, P, cx, cy, cz);
    double t = 0.0, b = 0.0, off = 0.0;
    for (int f = 0; f < 2 * g.dim; f++) {
      long long nb;
      const int k = face_kind(g, fl, P, cx, cy, cz, f, &nb);
      if (k == 0) {
        t += 1.0;
        off += psi[nb];
      } else if (k == 2) {
        t += 1.0;
      } else if (k == 1) {
        t += 2.0;
        b += 2.0 * psi_s;
      }
    }
    const double x = psi[P], ph = x / vt;
    const double sh = sinh(ph), ch = cosh(ph);
    const double F = t * x - off - b + kdx2 * vt * sh;
    const double dg = t + kdx2 * ch;
    const double rhs = b + kdx2 * (x * ch - vt * sh);
    diag[P] = dg;
    r[P] = -F;
    p[P] = -F / dg;
    v[0] += F * (F / dg);
    v[1] += rhs * rhs;
    v[2] += F * F;
    v[3] += b * b;
  }
  block_reduce<4>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; k++) part[k * gridDim.x + blockIdx.x] = v[k];
  if (last_block(counter, gridDim.x)) {
    combine_partials<4>(part, gridDim.x, v, sm, OpSum(), 0.0);
    if (threadIdx.x == 0) {
      scal[S_CG_RZ] = v[0];
      scal[S_CG_BB] = v[1];
      scal[S_CG_RR] = v[2];
      scal[S_CG_REL] = v[1] > 0.0 ? sqrt(v[2] / v[1]) : 0.0;
      scal[S_CG_DONE] = (v[1] > 0.0 && v[2] > 0.0) ? 0.0 : 1.0;
      scal[S_CG_TOL] = tol;
      scal[S_CG_IT] = 0.0;
      scal[S_PB_FF] = v[2];
      scal[S_PB_BB] = v[3];
      *counter = 0;
    }
  }
}

// q = A p and p.q; alpha = rz / p.q.
__global__ void __launch_bounds__(kRedThreads)
    k_cg_spmv(Geo g, const NFlag *__restrict__ fl, const double *__restrict__ p,
              const double *__restrict__ diag, double *__restrict__ q,
              double *__restrict__ part, unsigned int *counter, double *scal) {
  if (scal[S_CG_DONE] != 0.0) return;
  __shared__ double sm[32];
  double v[1] = {0.0};
  for (long long P = blockIdx.x * (long long)blockDim.x + threadIdx.x; P < g.N;
       P += (long long)gridDim.x * blockDim.x) {
    if (fl[P] & 1) {
      q[P] = 0.0;
      continue;
    }
    int cx, cy, cz;
    coords(g, P, cx, cy, cz);
    double off = 0.0;
    for (int f = 0; f < 2 * g.dim; f++) {
      long long nb;
      if (face_kind(g, fl, P, cx, cy, cz, f, &nb) == 0) off += p[nb];
    }
    const double qv = diag[P] * p[P] - off;
    q[P] = qv;
    v[0] += p[P] * qv;
  }
  block_reduce<1>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  if (last_block(counter, gridDim.x)) {
    combine_partials<1>(part, gridDim.x, v, sm, OpSum(), 0.0);
    if (threadIdx.x == 0) {
      scal[S_CG_PQ] = v[0];
      scal[S_CG_ALPHA] = v[0] != 0.0 ? scal[S_CG_RZ] / v[0] : 0.0;
      *counter = 0;
    }
  }
}

// x += alpha p, r -= alpha q, z = r / diag (into q); beta = rz' / rz.
__global__ void __launch_bounds__(kRedThreads)
    k_cg_update(long long N, const NFlag *__restrict__ fl, double *__restrict__ x,
                double *__restrict__ r, const double *__restrict__ p, double *__restrict__ q,
                const double *__restrict__ diag, double *__restrict__ part,
                unsigned int *counter, double *scal) {
  if (scal[S_CG_DONE] != 0.0) return;
  __shared__ double sm[2 * 32];
  const double alpha = scal[S_CG_ALPHA];
  double v[2] = {0.0, 0.0};
  for (long long P = blockIdx.x * (long long)blockDim.x + threadIdx.x; P < N;
       P += (long long)gridDim.x * blockDim.x) {
    if (fl[P] & 1) continue;
    x[P] += alpha * p[P];
    const double rv = r[P] - alpha * q[P];
    r[P] = rv;
    const double zv = rv / diag[P];
    q[P] = zv;
    v[0] += rv * zv;
    v[1] += rv * rv;
  }
  block_reduce<2>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = v[0];
    part[gridDim.x + blockIdx.x] = v[1];
  }
  if (last_block(counter, gridDim.x)) {
    combine_partials<2>(part, gridDim.x, v, sm, OpSum(), 0.0);
    if (threadIdx.x == 0) {
      const double rz_old = scal[S_CG_RZ];
      scal[S_CG_BETA] = rz_old != 0.0 ? v[0] / rz_old : 0.0;
      scal[S_CG_RZ] = v[0];
      scal[S_CG_RR] = v[1];
      const double rel = sqrt(v[1] / scal[S_CG_BB]);
      scal[S_CG_REL] = rel;
      scal[S_CG_IT] += 1.0;
      if (rel < scal[S_CG_TOL] || v[0] == 0.0) scal[S_CG_DONE] = 1.0;
      *counter = 0;
    }
  }
}

// p = z + beta p.
__global__ void k_cg_dir(long long N, double *__restrict__ p, const double *__restrict__ zq,
                         const double *__restrict__ scal) {
  if (scal[S_CG_DONE] != 0.0) return;
  const double beta = scal[S_CG_BETA];
  for (long long P = blockIdx.x * (long long)blockDim.x + threadIdx.x; P < N;
       P += (long long)gridDim.x * blockDim.x)
    p[P] = zq[P] + beta * p[P];
}

// The charge term of Eq. 4 at every pore cell from Eq. 5:
// src = coef * sum_k z_k C_k, coef = F dx^2 / (eps_r eps_0) (lattice order;
// solid cells keep the 0 the caller cleared).
template <typename T>
__global__ void k_charge(int n, int ns, const int *__restrict__ cells, const T *__restrict__ C,
                         const float *__restrict__ Cl, int4 z, double coef,
                         double *__restrict__ src) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int zz[4] = {z.x, z.y, z.z, z.w};
    double q = 0.0;
    for (int k = 0; k < ns; k++)
      q += zz[k] * ((double)C[(size_t)k * n + r] + (Cl ? (double)Cl[(size_t)k * n + r] : 0.0));
    src[cells[r]] = coef * q;
  }
}

// phi = psi / V_T of every pore rank, in the transport kernel's format.
template <typename T>
__global__ void k_phi(int n, const int *__restrict__ cells, const double *__restrict__ psi,
                      typename PhiStore<T>::type *__restrict__ phi, double inv_vt) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    phi[r] = PhiStore<T>::make(psi[cells[r]] * inv_vt);
}

}  // namespace

// CG iterations (the scalars set up by k_cg_setup or k_pb_setup) until the
// device flags convergence or max_iter iterations ran; the host polls the
// flag after 8, 16, 32, ... iterations (at most 256 between polls).
static cdi_status cg_iterate(cdi_domain *d, const Geo &g, double *r, double *p, double *q,
                             const double *dg, int max_iter, bool *done) {
  int launched = 0;
  int chunk = 8;
  *done = false;
  while (launched < max_iter) {
    const int n = std::min(chunk, max_iter - launched);
    for (int k = 0; k < n; k++) {
      k_cg_spmv<<<kRedBlocks, kRedThreads, 0, d->stream>>>(g, d->d_nflags, p, dg, q, d->d_part,
                                                            d->d_counter + C_CG1, d->d_scal);
      k_cg_update<<<kRedBlocks, kRedThreads, 0, d->stream>>>(
          d->N, d->d_nflags, d->d_psi, r, p, q, dg, d->d_part, d->d_counter + C_CG2, d->d_scal);
      k_cg_dir<<<kRedBlocks, kRedThreads, 0, d->stream>>>(d->N, p, q, d->d_scal);
    }
    d->timing.kernel_launches += 3 * n;
    launched += n;
    CDI_TRY(d, cudaGetLastError(), "cg iteration");
    CDI_TRY(d, cudaMemcpyAsync(d->h_scal + S_CG_REL, d->d_scal + S_CG_REL, 4 * sizeof(double),
                               cudaMemcpyDeviceToHost, d->stream),
            "cg poll");
    CDI_TRY(d, cudaStreamSynchronize(d->stream), "cg poll");
    if (d->h_scal[S_CG_DONE] != 0.0) {
      *done = true;
      break;
    }
    chunk = std::min(chunk * 2, 256);
  }
  return CDI_OK;
}

static cdi_status finish_potential(cdi_domain *d, cudaEvent_t ev, bool done, int *iters,
                                   double *relres);

cdi_status cdi_psi_solve(cdi_domain *d, double psi_s, double kdx2, const double *src,
                         double tol, int max_iter, int *iters, double *relres) {
  Geo g{d->nx, d->ny, d->nz, d->dim, d->walls, d->N};
  double *r = d->d_cg, *p = d->d_cg + d->N, *q = d->d_cg + 2 * d->N, *dg = d->d_cg + 3 * d->N;
  cudaEvent_t ev;
  cdi_timing_begin(d, &ev);
  k_cg_setup<<<kRedBlocks, kRedThreads, 0, d->stream>>>(g, d->d_nflags, kdx2, psi_s, src, tol,
                                                         d->d_psi, r, p, dg, d->d_part,
                                                         d->d_counter + C_CG1, d->d_scal);
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "cg setup");
  bool done = false;
  cdi_status cs = cg_iterate(d, g, r, p, q, dg, max_iter, &done);
  if (cs != CDI_OK) return cs;
  return finish_potential(d, ev, done, iters, relres);
}

// phi = psi / V_T for the transport step, the solve's figures to the host.
static cdi_status finish_potential(cdi_domain *d, cudaEvent_t ev, bool done, int *iters,
                                   double *relres) {
  // phi keeps FP64 accuracy in both precisions (a double, or an FP32 hi/lo
  // pair): the Boltzmann factor exp(z phi) of a face turns an absolute error
  // of phi into a relative error of C.
  const double inv_vt = 1.0 / d->VT;
  if (d->prec == CDI_FP64)
    k_phi<double><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        (int)d->n_pore, d->d_cell_list, d->d_psi, (double *)d->d_phi, inv_vt);
  else
    k_phi<float><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        (int)d->n_pore, d->d_cell_list, d->d_psi, (float2 *)d->d_phi, inv_vt);
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "phi");
  CDI_TRY(d, cudaMemcpyAsync(d->h_scal + S_CG_REL, d->d_scal + S_CG_REL, 4 * sizeof(double),
                             cudaMemcpyDeviceToHost, d->stream),
          "cg result");
  cdi_timing_end(d, ev, PH_PSI, 0);
  CDI_TRY(d, cudaStreamSynchronize(d->stream), "potential");
  const int it = (int)d->h_scal[S_CG_IT];
  d->timing.psi_iters += it;
  if (iters) *iters = it;
  if (relres) *relres = d->h_scal[S_CG_REL];
  return (done || d->h_scal[S_CG_DONE] != 0.0) ? CDI_OK : CDI_ERR_NOT_CONVERGED;
}

// Nonlinear Poisson-Boltzmann potential: Newton from psi = 0 (its first step
// is the screened Debye-Hueckel field), each step a CG solve warm-started at
// the current psi (k_pb_setup), until |F| <= tol |b| (b the surface terms).
// The problem is the minimum of a strictly convex energy and, psi keeping the
// sign of psi_s, Newton's iterates approach it monotonically after the first
// step.  Each CG runs to 0.1 tol of its right-hand side, at most max_iter
// iterations.  iters: the CG iterations of all steps; relres: |F| / |b|.
cdi_status cdi_psi_pb(cdi_domain *d, double psi_s, double kdx2, double tol, int max_iter,
                      int *iters, double *relres) {
  constexpr int kMaxNewton = 200;
  Geo g{d->nx, d->ny, d->nz, d->dim, d->walls, d->N};
  double *r = d->d_cg, *p = d->d_cg + d->N, *q = d->d_cg + 2 * d->N, *dg = d->d_cg + 3 * d->N;
  cudaEvent_t ev;
  cdi_timing_begin(d, &ev);
  CDI_TRY(d, cudaMemsetAsync(d->d_psi, 0, (size_t)d->N * 8, d->stream), "pb start");
  bool converged = false;
  double rel = 0.0;
  int cg_total = 0;
  for (int step = 0;; step++) {
    k_pb_setup<<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        g, d->d_nflags, kdx2, psi_s, d->VT, 0.1 * tol, d->d_psi, r, p, dg, d->d_part,
        d->d_counter + C_CG1, d->d_scal);
    d->timing.kernel_launches++;
    CDI_TRY(d, cudaGetLastError(), "pb setup");
    CDI_TRY(d, cudaMemcpyAsync(d->h_scal + S_PB_FF, d->d_scal + S_PB_FF, 2 * sizeof(double),
                               cudaMemcpyDeviceToHost, d->stream),
            "pb residual");
    CDI_TRY(d, cudaStreamSynchronize(d->stream), "pb residual");
    const double ff = d->h_scal[S_PB_FF], bb = d->h_scal[S_PB_BB];
    rel = bb > 0.0 ? std::sqrt(ff / bb) : 0.0;
    if (rel < tol) {
      converged = true;
      break;
    }
    if (step == kMaxNewton) break;
    bool done = false;
    cdi_status cs = cg_iterate(d, g, r, p, q, dg, max_iter, &done);
    if (cs != CDI_OK) return cs;
    cg_total += (int)d->h_scal[S_CG_IT];
  }
  cdi_status s = finish_potential(d, ev, true, nullptr, nullptr);
  if (s != CDI_OK) return s;
  d->timing.psi_iters += cg_total;
  if (iters) *iters = cg_total;
  if (relres) *relres = rel;
  return converged ? CDI_OK : CDI_ERR_NOT_CONVERGED;
}

// Coupled re-solve (Eq. 3-5): the charge term of the current concentrations,
// then Eq. 4 with the Laplace operator and the domain's surface potential.
cdi_status cdi_psi_coupled(cdi_domain *d) {
  CDI_TRY(d, cudaMemsetAsync(d->d_src, 0, (size_t)d->N * 8, d->stream), "charge reset");
  const double F = 96485.0, eps0 = 8.854e-12;
  const double coef = F * d->dx * d->dx / (d->eps_r * eps0);
  const int4 z = make_int4(d->z[0], d->z[1], d->z[2], d->z[3]);
  if (d->prec == CDI_FP64)
    k_charge<double><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        (int)d->n_pore, d->ns, d->d_cell_list, (const double *)d->d_C[d->cur], nullptr, z, coef,
        d->d_src);
  else
    k_charge<float><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        (int)d->n_pore, d->ns, d->d_cell_list, (const float *)d->d_C[d->cur], d->d_Clo[d->cur], z,
        coef, d->d_src);
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "charge");
  int it = 0;
  double rel = 0.0;
  cdi_status s = cdi_psi_solve(d, d->psi_s, 0.0, d->d_src, d->psi_tol, d->psi_max_iter, &it, &rel);
  if (s == CDI_ERR_NOT_CONVERGED)
    return cdi_fail(d, s, "coupled potential did not reach tol within max_iter");
  return s;
}
