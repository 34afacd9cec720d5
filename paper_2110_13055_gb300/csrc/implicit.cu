// Implicit (backward Euler) finite-volume transport: the time integration
// Sec. 2 uses for Eq. 3 with the adsorption flux of Eq. 6.  Each step solves,
// per species,
//   (I + dt A) C^{n+1} = C^n + dt b,
// where (1/dx) sum_f J_f(C) = A C - b are the face fluxes of the explicit
// step (Scharfetter-Gummel fluxes with frozen velocity and potential, the
// half-cell Robin closure at solid faces, the feed ghost at the inlet, the
// copying ghost at the outlet).  The operator is assembled once per
// transport state in FP64 (a diagonal, one coefficient per face and the
// inlet source, by pore rank); the solve is matrix-free, Jacobi-
// preconditioned BiCGStab in FP64 with every scalar on the device and
// fixed-order block reductions, so a run is deterministic.  The adsorbed,
// inflow and outflow accounts take the fluxes at C^{n+1}, so the mass balance
// closes as in the explicit scheme.  The step is unconditionally stable and
// positivity-preserving (I + dt A is an M-matrix), so dt may exceed the
// explicit bound by orders of magnitude.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "cdi_internal.cuh"

using namespace cdi;

namespace {

// Scalar slots of the solver (d_iscal).
enum { B_RHO = 0, B_ALPHA, B_OMEGA, B_BETA, B_BB, B_REL, B_DONE, B_TOL, B_IT, B_R0V, B_N };

// Coefficients of species k, component j at ((k * NC) + j) * n + r:
// j = 0 diagonal of A, 1..2 dim its face coefficients (face j - 1: +x, -x,
// +y, -y, +z, -z; 0 across a closed face), then the inlet source b, and the
// account coefficients: ain = (D/dx) B(-P_in), bin = (D/dx) B(P_in) c0 (the
// inflow is bin - ain C_P), aout = (D/dx) (B(-P_out) - B(P_out)) (outflow
// aout C_P), gam = n_solid K_eff (adsorption gam C_P).
template <int DIM> struct ICoef {
  static constexpr int NF = 2 * DIM;
  static constexpr int DIAG = 0, FACE = 1, B = 1 + NF, AIN = 2 + NF, BIN = 3 + NF,
                       AOUT = 4 + NF, GAM = 5 + NF, NC = 6 + NF;
};

struct IGeo {
  const NFlag *fl;   // per rank face flags
  const int *lat;    // lateral neighbour ranks (-1: none)
  int n, walls;
};

// Neighbour rank across face fc of rank r (-1: none) and the face kind.
enum { K_PORE = 0, K_SOLID = 1, K_INLET = 2, K_OUTLET = 3, K_WALL = 4 };
__device__ __forceinline__ int ikind(const IGeo &g, unsigned f, int fc, int r, int &q) {
  const bool solid = (f >> (kFaceBit + fc)) & 1u;
  const bool edge = (f >> (kEdgeBit + fc)) & 1u;
  q = -1;
  if (fc < 2) {
    if (edge) return fc == 0 ? K_OUTLET : K_INLET;
    if (solid) return K_SOLID;
    q = r + (fc == 0 ? 1 : -1);
    return K_PORE;
  }
  if (edge && g.walls) return K_WALL;
  if (solid) return K_SOLID;
  q = g.lat[(size_t)(fc - 2) * g.n + r];
  return q >= 0 ? K_PORE : K_SOLID;
}

__device__ __forceinline__ double phi_of(double v) { return v; }
__device__ __forceinline__ double phi_of(float2 v) { return (double)v.x + (double)v.y; }

// Per-species constants passed by value.
struct PerSpecies {
  double v[kMaxSpecies];
};

template <typename T, int DIM>
__global__ void k_imp_coef(IGeo g, const T *__restrict__ u,
                           const typename PhiStore<T>::type *__restrict__ phi, int ns,
                           PerSpecies dxD, PerSpecies Ddx, PerSpecies Keff, PerSpecies zf,
                           double inv_dx, double c0, double *__restrict__ co) {
  using C = ICoef<DIM>;
  const double *dxDk = dxD.v, *Ddxk = Ddx.v, *Kk = Keff.v, *zk = zf.v;
  const size_t n = (size_t)g.n;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < g.n; r += gridDim.x * blockDim.x) {
    const unsigned f = g.fl[r];
    const double phP = phi_of(phi[r]);
    for (int k = 0; k < ns; k++) {
      double *c = co + (size_t)k * C::NC * n;
      double diag = 0.0, b = 0.0, ain = 0.0, bin = 0.0, aout = 0.0, gam = 0.0;
      for (int fc = 0; fc < C::NF; fc++) {
        int q;
        const int kind = ikind(g, f, fc, r, q);
        double off = 0.0;
        if (kind == K_SOLID) {
          diag += Kk[k] * inv_dx;
          gam += Kk[k];
        } else if (kind != K_WALL) {
          const int a = fc >> 1;
          const double uP = (double)u[(size_t)a * n + r];
          const double un = kind == K_PORE ? (double)u[(size_t)a * n + q] : uP;
          const double phn = kind == K_PORE ? phi_of(phi[q]) : (kind == K_INLET ? 0.0 : phP);
          const double half = (fc & 1) ? -0.5 : 0.5;
          const double P = half * (uP + un) * dxDk[k] - zk[k] * (phn - phP);
          double Bp, Bm;
          bernoulli_pair(P, Bp, Bm);
          if (kind == K_PORE) {
            diag += Ddxk[k] * inv_dx * Bm;
            off = -Ddxk[k] * inv_dx * Bp;
          } else if (kind == K_INLET) {
            diag += Ddxk[k] * inv_dx * Bm;
            b += Ddxk[k] * inv_dx * Bp * c0;
            ain = Ddxk[k] * Bm;
            bin = Ddxk[k] * Bp * c0;
          } else {
            diag += Ddxk[k] * inv_dx * (Bm - Bp);
            aout = Ddxk[k] * (Bm - Bp);
          }
        }
        c[(size_t)(C::FACE + fc) * n + r] = off;
      }
      c[(size_t)C::DIAG * n + r] = diag;
      c[(size_t)C::B * n + r] = b;
      c[(size_t)C::AIN * n + r] = ain;
      c[(size_t)C::BIN * n + r] = bin;
      c[(size_t)C::AOUT * n + r] = aout;
      c[(size_t)C::GAM * n + r] = gam;
    }
  }
}

// (I + dt A) (x / K) at rank r, K = 1 + dt A_PP the Jacobi preconditioner;
// xv(q) supplies x at rank q.
template <int DIM, typename X>
__device__ __forceinline__ double apply_scaled(const IGeo &g, const double *__restrict__ c,
                                               double dt, int r, X xv) {
  using C = ICoef<DIM>;
  const size_t n = (size_t)g.n;
  const unsigned f = g.fl[r];
  double acc = xv(r);  // K x / K
  for (int fc = 0; fc < C::NF; fc++) {
    const double off = c[(size_t)(C::FACE + fc) * n + r];
    if (off == 0.0) continue;
    int q;
    ikind(g, f, fc, r, q);
    acc += dt * off * (xv(q) / (1.0 + dt * c[(size_t)C::DIAG * n + q]));
  }
  return acc;
}

// Start of a step for one species: x = C^n (the first guess), rhs = C^n +
// dt b, r = rhs - M x, r0 = r, p = r; rho = r0.r, bb = rhs.rhs.
template <typename T, int DIM>
__global__ void __launch_bounds__(kRedThreads)
    k_bi_start(IGeo g, const double *__restrict__ c, double dt, const T *__restrict__ Ck,
               const float *__restrict__ Clk, double tol, double *__restrict__ x,
               double *__restrict__ rr, double *__restrict__ r0, double *__restrict__ p,
               double *__restrict__ part, unsigned int *counter, double *scal) {
  using C = ICoef<DIM>;
  __shared__ double sm[2 * 32];
  double v[2] = {0.0, 0.0};
  const size_t n = (size_t)g.n;
  auto cval = [&](int q) {
    return (double)Ck[q] + (Clk ? (double)Clk[q] : 0.0);
  };
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < g.n; r += gridDim.x * blockDim.x) {
    const double cP = cval(r);
    const double rhs = cP + dt * c[(size_t)C::B * n + r];
    // M x with x = C: (1 + dt A_PP) C_P + dt sum off C_nb
    const unsigned f = g.fl[r];
    double Mx = (1.0 + dt * c[(size_t)C::DIAG * n + r]) * cP;
    for (int fc = 0; fc < C::NF; fc++) {
      const double off = c[(size_t)(C::FACE + fc) * n + r];
      if (off == 0.0) continue;
      int q;
      ikind(g, f, fc, r, q);
      Mx += dt * off * cval(q);
    }
    const double res = rhs - Mx;
    x[r] = cP;
    rr[r] = res;
    r0[r] = res;
    p[r] = res;
    v[0] += res * res;
    v[1] += rhs * rhs;
  }
  block_reduce<2>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = v[0];
    part[gridDim.x + blockIdx.x] = v[1];
  }
  if (last_block(counter, gridDim.x)) {
    combine_partials<2>(part, gridDim.x, v, sm, OpSum(), 0.0);
    if (threadIdx.x == 0) {
      scal[B_RHO] = v[0];
      scal[B_BB] = v[1];
      scal[B_TOL] = tol;
      scal[B_IT] = 0.0;
      const double rel = v[1] > 0.0 ? sqrt(v[0] / v[1]) : 0.0;
      scal[B_REL] = rel;
      scal[B_DONE] = (rel < tol || v[0] == 0.0) ? 1.0 : 0.0;
      *counter = 0;
    }
  }
}

// v = M (p / K); alpha = rho / (r0 . v).
template <int DIM>
__global__ void __launch_bounds__(kRedThreads)
    k_bi_v(IGeo g, const double *__restrict__ c, double dt, const double *__restrict__ p,
           const double *__restrict__ r0, double *__restrict__ vv, double *__restrict__ part,
           unsigned int *counter, double *scal) {
  if (scal[B_DONE] != 0.0) return;
  __shared__ double sm[32];
  double v[1] = {0.0};
  auto pv = [&](int q) { return p[q]; };
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < g.n; r += gridDim.x * blockDim.x) {
    const double y = apply_scaled<DIM>(g, c, dt, r, pv);
    vv[r] = y;
    v[0] += r0[r] * y;
  }
  block_reduce<1>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  if (last_block(counter, gridDim.x)) {
    combine_partials<1>(part, gridDim.x, v, sm, OpSum(), 0.0);
    if (threadIdx.x == 0) {
      scal[B_R0V] = v[0];
      scal[B_ALPHA] = v[0] != 0.0 ? scal[B_RHO] / v[0] : 0.0;
      *counter = 0;
    }
  }
}

// s = r - alpha v (stored over r), t = M (s / K); omega = (t . s) / (t . t).
// The neighbours' s are formed on the fly from their r and v.
template <int DIM>
__global__ void __launch_bounds__(kRedThreads)
    k_bi_t(IGeo g, const double *__restrict__ c, double dt, const double *__restrict__ rr,
           const double *__restrict__ vv, double *__restrict__ s, double *__restrict__ t,
           double *__restrict__ part, unsigned int *counter, double *scal) {
  if (scal[B_DONE] != 0.0) return;
  __shared__ double sm[2 * 32];
  const double alpha = scal[B_ALPHA];
  double v[2] = {0.0, 0.0};
  auto sv = [&](int q) { return rr[q] - alpha * vv[q]; };
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < g.n; r += gridDim.x * blockDim.x) {
    const double sP = sv(r);
    const double y = apply_scaled<DIM>(g, c, dt, r, sv);
    s[r] = sP;
    t[r] = y;
    v[0] += y * sP;
    v[1] += y * y;
  }
  block_reduce<2>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = v[0];
    part[gridDim.x + blockIdx.x] = v[1];
  }
  if (last_block(counter, gridDim.x)) {
    combine_partials<2>(part, gridDim.x, v, sm, OpSum(), 0.0);
    if (threadIdx.x == 0) {
      scal[B_OMEGA] = v[1] != 0.0 ? v[0] / v[1] : 0.0;
      *counter = 0;
    }
  }
}

// x += (alpha p + omega s) / K, r = s - omega t; rho' = r0 . r, beta =
// (rho' / rho)(alpha / omega); convergence on ||r|| / ||rhs||.
template <int DIM>
__global__ void __launch_bounds__(kRedThreads)
    k_bi_x(IGeo g, const double *__restrict__ c, double dt, double *__restrict__ x,
           double *__restrict__ rr, const double *__restrict__ r0, const double *__restrict__ p,
           const double *__restrict__ s, const double *__restrict__ t,
           double *__restrict__ part, unsigned int *counter, double *scal) {
  using C = ICoef<DIM>;
  if (scal[B_DONE] != 0.0) return;
  __shared__ double sm[2 * 32];
  const double alpha = scal[B_ALPHA], omega = scal[B_OMEGA];
  double v[2] = {0.0, 0.0};
  const size_t n = (size_t)g.n;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < g.n; r += gridDim.x * blockDim.x) {
    const double K = 1.0 + dt * c[(size_t)C::DIAG * n + r];
    x[r] += (alpha * p[r] + omega * s[r]) / K;
    const double rv = s[r] - omega * t[r];
    rr[r] = rv;
    v[0] += r0[r] * rv;
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
      const double rho = scal[B_RHO];
      scal[B_BETA] = (rho != 0.0 && omega != 0.0) ? (v[0] / rho) * (alpha / omega) : 0.0;
      scal[B_RHO] = v[0];
      const double rel = scal[B_BB] > 0.0 ? sqrt(v[1] / scal[B_BB]) : 0.0;
      scal[B_REL] = rel;
      scal[B_IT] += 1.0;
      // converged, or broken down (no new direction): the host restarts or stops
      if (rel < scal[B_TOL] || v[0] == 0.0 || omega == 0.0) scal[B_DONE] = 1.0;
      *counter = 0;
    }
  }
}

// p = r + beta (p - omega v).
__global__ void k_bi_p(int n, double *__restrict__ p, const double *__restrict__ rr,
                       const double *__restrict__ vv, const double *__restrict__ scal) {
  if (scal[B_DONE] != 0.0) return;
  const double beta = scal[B_BETA], omega = scal[B_OMEGA];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    p[r] = rr[r] + beta * (p[r] - omega * vv[r]);
}

// C^{n+1} = x into the storage type (an FP32 pair splits into hi + lo), and
// the accounts of the step: the adsorbed, inflow and outflow fluxes at
// C^{n+1}, summed per warp of 32 ranks into the domain's per-warp accounts.
template <typename T, int DIM>
__global__ void k_bi_finish(IGeo g, const double *__restrict__ c, const double *__restrict__ x,
                            T *__restrict__ Cout, float *__restrict__ Cout_l, int k,
                            typename std::conditional<std::is_same<T, float>::value, float2,
                                                      double>::type *__restrict__ acc,
                            int naccs) {
  using C = ICoef<DIM>;
  const size_t n = (size_t)g.n;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  double v[3] = {0.0, 0.0, 0.0};
  if (r < g.n) {
    const double xv = x[r];
    if (std::is_same<T, float>::value) {
      const float hi = (float)xv;
      Cout[r] = (T)hi;
      if (Cout_l) Cout_l[r] = (float)(xv - (double)hi);
    } else {
      Cout[r] = (T)xv;
    }
    v[0] = c[(size_t)C::GAM * n + r] * xv;
    v[1] = c[(size_t)C::BIN * n + r] - c[(size_t)C::AIN * n + r] * xv;
    v[2] = c[(size_t)C::AOUT * n + r] * xv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int j = 0; j < 3; j++) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
  const int w = r >> 5;
  if ((threadIdx.x & 31) == 0 && w < naccs) {
    for (int j = 0; j < 3; j++) {
      auto *a = acc + (size_t)(3 * k + j) * naccs + w;
      if constexpr (std::is_same<T, float>::value) {
        // an FP32 pair account: add the FP64 value as hi + lo, each by two-sum
        const float parts[2] = {(float)v[j], (float)(v[j] - (double)(float)v[j])};
        for (float pv : parts) {
          float2 tt = *a;
          const float sum = __fadd_rn(tt.x, pv);
          const float bp = __fsub_rn(sum, tt.x);
          const float e = __fadd_rn(__fsub_rn(tt.x, __fsub_rn(sum, bp)), __fsub_rn(pv, bp));
          tt.x = sum;
          tt.y = __fadd_rn(tt.y, e);
          *a = tt;
        }
      } else {
        *a = __dadd_rn(*a, v[j]);
      }
    }
  }
}

IGeo make_igeo(const cdi_domain *d) {
  return IGeo{d->d_cfl, d->d_latnb, (int)d->n_pore, d->walls};
}

template <typename T, int DIM>
cdi_status imp_coefs(cdi_domain *d) {
  PerSpecies dxD, Ddx, Keff, zf;
  for (int k = 0; k < kMaxSpecies; k++) {
    const double Dk = k < d->ns ? d->D[k] : 1.0;
    dxD.v[k] = d->dx / Dk;
    Ddx.v[k] = Dk / d->dx;
    Keff.v[k] = d->Ka / (1.0 + d->Ka * d->dx / (2.0 * Dk));
    zf.v[k] = k < d->ns ? d->z[k] : 0.0;
  }
  k_imp_coef<T, DIM><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
      make_igeo(d), (const T *)d->d_u, (const typename PhiStore<T>::type *)d->d_phi, d->ns,
      dxD, Ddx, Keff, zf, 1.0 / d->dx, d->c0, d->d_icoef);
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "implicit operator");
  d->imp_stale = false;
  return CDI_OK;
}

template <typename T, int DIM>
cdi_status imp_step(cdi_domain *d) {
  using C = ICoef<DIM>;
  const int n = (int)d->n_pore;
  const size_t nn = (size_t)n;
  double *x = d->d_iwork, *rr = x + nn, *r0 = x + 2 * nn, *p = x + 3 * nn, *vv = x + 4 * nn,
         *s = x + 5 * nn, *t = x + 6 * nn;
  const IGeo g = make_igeo(d);
  const double dt = d->dt;
  const int in = d->cur;
  using A = typename std::conditional<std::is_same<T, float>::value, float2, double>::type;
  for (int k = 0; k < d->ns; k++) {
    const double *c = d->d_icoef + (size_t)k * C::NC * nn;
    const T *Ck = (const T *)d->d_C[in] + (size_t)k * nn;
    const float *Clk = d->d_Clo[in] ? d->d_Clo[in] + (size_t)k * nn : nullptr;
    int iters = 0;
    k_bi_start<T, DIM><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        g, c, dt, Ck, Clk, d->imp_tol, x, rr, r0, p, d->d_part, d->d_counter + C_IMP,
        d->d_iscal);
    d->timing.kernel_launches++;
    CDI_TRY(d, cudaMemcpyAsync(d->h_scal + S_IMP, d->d_iscal, B_N * sizeof(double),
                               cudaMemcpyDeviceToHost, d->stream),
            "implicit start");
    CDI_TRY(d, cudaStreamSynchronize(d->stream), "implicit start");
    int chunk = 4;
    while (d->h_scal[S_IMP + B_DONE] == 0.0 && iters < d->imp_max_iter) {
      const int m = std::min(chunk, d->imp_max_iter - iters);
      for (int j = 0; j < m; j++) {
        k_bi_v<DIM><<<kRedBlocks, kRedThreads, 0, d->stream>>>(g, c, dt, p, r0, vv, d->d_part,
                                                                 d->d_counter + C_IMP,
                                                                 d->d_iscal);
        k_bi_t<DIM><<<kRedBlocks, kRedThreads, 0, d->stream>>>(g, c, dt, rr, vv, s, t,
                                                                 d->d_part,
                                                                 d->d_counter + C_IMP,
                                                                 d->d_iscal);
        k_bi_x<DIM><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
            g, c, dt, x, rr, r0, p, s, t, d->d_part, d->d_counter + C_IMP, d->d_iscal);
        k_bi_p<<<kRedBlocks, kRedThreads, 0, d->stream>>>(n, p, rr, vv, d->d_iscal);
      }
      d->timing.kernel_launches += 4 * m;
      iters += m;
      CDI_TRY(d, cudaGetLastError(), "implicit iteration");
      CDI_TRY(d, cudaMemcpyAsync(d->h_scal + S_IMP, d->d_iscal, B_N * sizeof(double),
                                 cudaMemcpyDeviceToHost, d->stream),
              "implicit poll");
      CDI_TRY(d, cudaStreamSynchronize(d->stream), "implicit poll");
      chunk = std::min(chunk * 2, 64);
    }
    const bool done = d->h_scal[S_IMP + B_REL] < d->imp_tol;
    d->imp_iters += iters;
    d->imp_last_rel = d->h_scal[S_IMP + B_REL];
    if (!done)
      return cdi_fail(d, CDI_ERR_NOT_CONVERGED,
                      "implicit step: the linear solve did not reach tol within max_iter");
    T *Co = (T *)d->d_C[1 - in] + (size_t)k * nn;
    float *Col = d->d_Clo[1 - in] ? d->d_Clo[1 - in] + (size_t)k * nn : nullptr;
    k_bi_finish<T, DIM><<<(n + 127) / 128, 128, 0, d->stream>>>(g, c, x, Co, Col, k, (A *)d->d_acc,
                                                               d->np_accs);
    d->timing.kernel_launches++;
    CDI_TRY(d, cudaGetLastError(), "implicit finish");
  }
  d->cur = 1 - in;
  return CDI_OK;
}

template <typename T, int DIM>
cdi_status imp_steps(cdi_domain *d, int64_t n) {
  if (d->imp_stale) {
    cdi_status s = imp_coefs<T, DIM>(d);
    if (s != CDI_OK) return s;
  }
  cudaEvent_t ev;
  cdi_timing_begin(d, &ev);
  for (int64_t i = 0; i < n; i++) {
    cdi_status s = imp_step<T, DIM>(d);
    if (s != CDI_OK) {
      cdi_timing_end(d, ev, PH_NP, i);
      return s;
    }
    d->np_steps++;
  }
  cdi_timing_end(d, ev, PH_NP, n);
  return CDI_OK;
}

}  // namespace

// Work memory of the implicit scheme (allocated on first use, kept for the
// domain's life): the operator of every species and seven FP64 vectors.
cdi_status cdi_imp_prepare(cdi_domain *d) {
  const int NC = d->dim == 2 ? ICoef<2>::NC : ICoef<3>::NC;
  if (!d->d_icoef) {
    d->d_icoef = (double *)cdi_dev_alloc(d, (size_t)kMaxSpecies * NC * d->n_pore * 8);
    d->d_iwork = (double *)cdi_dev_alloc(d, (size_t)7 * d->n_pore * 8);
    d->d_iscal = (double *)cdi_dev_alloc(d, 16 * 8);
    if (!d->d_icoef || !d->d_iwork || !d->d_iscal)
      return cdi_fail(d, CDI_ERR_OOM, "implicit scheme: device memory");
    CDI_TRY(d, cudaMemsetAsync(d->d_iscal, 0, 16 * 8, d->stream), "implicit scalars");
  }
  d->imp_stale = true;
  return CDI_OK;
}

cdi_status cdi_imp_steps(cdi_domain *d, int64_t n) {
  if (d->prec == CDI_FP64)
    return d->dim == 2 ? imp_steps<double, 2>(d, n) : imp_steps<double, 3>(d, n);
  return d->dim == 2 ? imp_steps<float, 2>(d, n) : imp_steps<float, 3>(d, n);
}
