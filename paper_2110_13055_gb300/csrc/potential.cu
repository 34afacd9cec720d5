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
  int launched = 0;
  int chunk = 8;
  bool done = false;
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
      done = true;
      break;
    }
    chunk = std::min(chunk * 2, 256);
  }
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
