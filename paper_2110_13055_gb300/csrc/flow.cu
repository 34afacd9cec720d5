// Lattice Boltzmann Stokes solve (Sec. 2, Eq. 7-8) on the GPU.
//
// Layout: populations are stored shifted (g_i = f_i - w_i), structure of
// arrays g[i * Nf + site], sites x-fastest over the flow grid (the image and
// its mirror image along x, periodic in x).  One array only: the AA access
// pattern streams in place.  An "even" step reads and writes the site's own
// slots (writing the post-collision value of direction i into slot opp(i));
// an "odd" step gathers from the neighbours' opposite slots and scatters to
// the neighbours' own slots.  After every even number of steps the array
// holds f_i(x) in slot i ("natural" layout), which is when the residual is
// taken and when a solve may stop.  Halfway bounce-back: a population that
// would enter a solid site (or cross a lateral wall) returns to its source
// in the opposite direction within the same step.
#include <cmath>

#include "cdi_internal.cuh"

using namespace cdi;

namespace {

// s + c += v with s carrying the rounded sum and c the accumulated rounding
// errors (Knuth's two-sum: the error of each addition is exact in FP32).
__device__ __forceinline__ void two_sum_acc(float v, float &s, float &c) {
  const float t = __fadd_rn(s, v);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
  s = t;
  c = __fadd_rn(c, err);
}

template <int DIM>
__global__ void k_flow_flags(const uint8_t *__restrict__ mask,
                             typename FlowFlag<DIM>::type *__restrict__ fl, int nx, int NX,
                             int ny, int nz, int walls) {
  using L = Lat<DIM>;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= NX) return;
  const int y = blockIdx.y, z = blockIdx.z;
  auto solid_at = [&](int X, int Y, int Z) -> bool {
    X = (X + NX) % NX;
    if (Y < 0 || Y >= ny) {
      if (walls) return true;
      Y = (Y + ny) % ny;
    }
    if (Z < 0 || Z >= nz) {
      if (walls) return true;
      Z = (Z + nz) % nz;
    }
    const int xs = X < nx ? X : 2 * nx - 1 - X;  // mirror image along x
    return mask[((size_t)Z * ny + Y) * nx + xs] != 0;
  };
  typename FlowFlag<DIM>::type f = solid_at(x, y, z) ? 1 : 0;
#pragma unroll
  for (int i = 1; i < L::Q; i++)
    if (solid_at(x + L::ex(i), y + L::ey(i), z + L::ez(i))) f |= (1u << i);
  fl[((size_t)z * ny + y) * NX + x] = f;
}

// One full lattice Boltzmann step (stream + collide) at every pore site.
// Collision (Eq. 8) with the Stokes-linear equilibrium
// g_eq_i = w_i (drho + 3 e_i.j), j = sum e_i g_i + F/2, and the force source
// (1 - 1/(2 tau)) 3 w_i e_i.F; omega = 1/tau.
template <typename T, int DIM, bool ODD>
__global__ void __launch_bounds__(kRowBlock)
    k_lbm_step(T *__restrict__ g, const typename FlowFlag<DIM>::type *__restrict__ fl, int NX,
               int ny, int nz, long long Nf, T omega, T fx_half, T fsrc) {
  using L = Lat<DIM>;
  constexpr int Q = L::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= NX) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long s = ((long long)z * ny + y) * NX + x;
  const unsigned f = fl[s];
  if (f & 1u) return;
  const int xp = x + 1 == NX ? 0 : x + 1, xm = x == 0 ? NX - 1 : x - 1;
  const int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
  const int zp = z + 1 == nz ? 0 : z + 1, zm = z == 0 ? nz - 1 : z - 1;
  auto nb = [&](int ex, int ey, int ez) -> long long {
    const int X = ex > 0 ? xp : (ex < 0 ? xm : x);
    const int Y = ey > 0 ? yp : (ey < 0 ? ym : y);
    const int Z = ez > 0 ? zp : (ez < 0 ? zm : z);
    return ((long long)Z * ny + Y) * NX + X;
  };
  T gi[Q];
#pragma unroll
  for (int i = 0; i < Q; i++) {
    if (!ODD) {
      gi[i] = g[(size_t)i * Nf + s];
    } else {
      const int o = L::opp(i);
      if ((f >> o) & 1u)  // the upstream site is solid: take the bounced value
        gi[i] = g[(size_t)i * Nf + s];
      else
        gi[i] = g[(size_t)o * Nf + nb(-L::ex(i), -L::ey(i), -L::ez(i))];
    }
  }
  T drho = T(0), jx = fx_half, jy = T(0), jz = T(0);
#pragma unroll
  for (int i = 0; i < Q; i++) {
    drho += gi[i];
    if (L::ex(i)) jx += T(L::ex(i)) * gi[i];
    if (L::ey(i)) jy += T(L::ey(i)) * gi[i];
    if (DIM == 3 && L::ez(i)) jz += T(L::ez(i)) * gi[i];
  }
  T go_all[Q];
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const T eu = T(L::ex(i)) * jx + T(L::ey(i)) * jy + T(L::ez(i)) * jz;
    const T geq = T(L::w(i)) * (drho + T(3) * eu);
    go_all[i] = gi[i] - omega * (gi[i] - geq) + T(L::w(i) * L::ex(i)) * fsrc;
  }
  if (sizeof(T) == 4) {
    // FP32 storage: the collision conserves mass exactly, but rounding the
    // stored values does not, and the leak is biased; it feeds the slowest
    // (pressure-diffusion) modes of the porous flow.  The rest population
    // closes the balance: g*_0 = sum_i g_i - sum_{i>0} g*_i, both sums carried
    // exactly as (sum, error) pairs by the two-sum transformation.
    float ms = 0.f, mc = 0.f, ss = 0.f, sc = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) two_sum_acc((float)gi[i], ms, mc);
#pragma unroll
    for (int i = 1; i < Q; i++) two_sum_acc((float)go_all[i], ss, sc);
    go_all[0] = (T)__fadd_rn(__fsub_rn(ms, ss), __fsub_rn(mc, sc));
  }
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const T go = go_all[i];
    if (!ODD) {
      g[(size_t)L::opp(i) * Nf + s] = go;
    } else {
      if ((f >> i) & 1u)  // the downstream site is solid: bounce back
        g[(size_t)L::opp(i) * Nf + s] = go;
      else
        g[(size_t)i * Nf + nb(L::ex(i), L::ey(i), L::ez(i))] = go;
    }
  }
}

// Velocity u = j = sum e_i g_i + F/2 from the natural layout, written to
// uflow (FP64); accumulates ||u - u_prev||^2 and ||u||^2 over pore sites and
// leaves the relative K-lag residual in scal[S_RES].
template <typename T, int DIM>
__global__ void __launch_bounds__(kRedThreads)
    k_flow_velocity(const T *__restrict__ g, const typename FlowFlag<DIM>::type *__restrict__ fl,
                    double *__restrict__ uflow, long long Nf, double fx_half,
                    double *__restrict__ part, unsigned int *counter, double *scal) {
  using L = Lat<DIM>;
  __shared__ double sm[2 * 32];
  double v[2] = {0.0, 0.0};
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < Nf;
       s += (long long)gridDim.x * blockDim.x) {
    if (fl[s] & 1u) continue;
    double j[3] = {fx_half, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
      const double gv = (double)g[(size_t)i * Nf + s];
      j[0] += L::ex(i) * gv;
      j[1] += L::ey(i) * gv;
      if (DIM == 3) j[2] += L::ez(i) * gv;
    }
#pragma unroll
    for (int a = 0; a < DIM; a++) {
      const double d = j[a] - uflow[(size_t)a * Nf + s];
      v[0] += d * d;
      v[1] += j[a] * j[a];
      uflow[(size_t)a * Nf + s] = j[a];
    }
  }
  block_reduce<2>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = v[0];
    part[gridDim.x + blockIdx.x] = v[1];
  }
  if (last_block(counter, gridDim.x)) {
    combine_partials<2>(part, gridDim.x, v, sm, OpSum(), 0.0);
    if (threadIdx.x == 0) {
      scal[S_RES_NUM] = v[0];
      scal[S_RES_DEN] = v[1];
      scal[S_RES] = v[1] > 0.0 ? sqrt(v[0] / v[1]) : 0.0;
      *counter = 0;
    }
  }
}

// Pore-mean x velocity over the original (unmirrored) image, U = sum u / (N
// phi) of Sec. 4, and the scale factor U_target / U.
__global__ void __launch_bounds__(kRedThreads)
    k_flow_mean(const double *__restrict__ uflow, const uint8_t *__restrict__ mask, int nx,
                int NX, long long N, double n_pore, double U_target, double *__restrict__ part,
                unsigned int *counter, double *scal) {
  __shared__ double sm[32];
  double v[1] = {0.0};
  for (long long P = blockIdx.x * (long long)blockDim.x + threadIdx.x; P < N;
       P += (long long)gridDim.x * blockDim.x) {
    if (mask[P]) continue;
    const long long row = P / nx;
    const int x = (int)(P - row * nx);
    v[0] += uflow[row * NX + x];
  }
  block_reduce<1>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  if (last_block(counter, gridDim.x)) {
    combine_partials<1>(part, gridDim.x, v, sm, OpSum(), 0.0);
    if (threadIdx.x == 0) {
      const double U = v[0] / n_pore;
      scal[S_ULAT] = U;
      scal[S_SCALE] = (U_target == 0.0 || U == 0.0) ? 0.0 : U_target / U;
      *counter = 0;
    }
  }
}

// u_phys = scale * u_lattice on the transport grid (0 in solid cells).
template <typename T, int DIM>
__global__ void k_flow_scale(const double *__restrict__ uflow, const uint8_t *__restrict__ mask,
                             T *__restrict__ u, int nx, int NX, long long N, long long Nf,
                             const double *__restrict__ scal) {
  const double sc = scal[S_SCALE];
  for (long long P = blockIdx.x * (long long)blockDim.x + threadIdx.x; P < N;
       P += (long long)gridDim.x * blockDim.x) {
    const long long row = P / nx;
    const int x = (int)(P - row * nx);
    const long long s = row * NX + x;
#pragma unroll
    for (int a = 0; a < DIM; a++)
      u[(size_t)a * N + P] = mask[P] ? T(0) : (T)(sc * uflow[(size_t)a * Nf + s]);
  }
}

template <typename T, int DIM>
void launch_step_pair(cdi_domain *d, cudaStream_t st, T omega, T fxh, T fsrc) {
  using FT = typename FlowFlag<DIM>::type;
  dim3 grid((d->NX + kRowBlock - 1) / kRowBlock, d->ny, d->nz);
  k_lbm_step<T, DIM, false><<<grid, kRowBlock, 0, st>>>(
      (T *)d->d_g, (const FT *)d->d_fflags, d->NX, d->ny, d->nz, d->Nf, omega, fxh, fsrc);
  k_lbm_step<T, DIM, true><<<grid, kRowBlock, 0, st>>>(
      (T *)d->d_g, (const FT *)d->d_fflags, d->NX, d->ny, d->nz, d->Nf, omega, fxh, fsrc);
}

template <typename T, int DIM>
cdi_status launch_velocity(cdi_domain *d) {
  using FT = typename FlowFlag<DIM>::type;
  k_flow_velocity<T, DIM><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
      (const T *)d->d_g, (const FT *)d->d_fflags, d->d_uflow, d->Nf, 0.5 * d->force, d->d_part,
      d->d_counter + C_RES, d->d_scal);
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "velocity kernel");
  return CDI_OK;
}

template <typename T, int DIM>
cdi_status flow_run(cdi_domain *d, const cdi_flow_params *p, int64_t *steps_out,
                    double *res_out) {
  const int K = p->check_every;
  d->tau = p->tau;
  d->force = p->force_lu;
  const T omega = T(1.0 / p->tau);
  const T fxh = T(0.5 * p->force_lu);
  const T fsrc = T((1.0 - 0.5 / p->tau) * 3.0 * p->force_lu);
  const int Q = Lat<DIM>::Q;
  // start from rest: g = 0 (f = w), u_prev = u(0)
  CDI_TRY(d, cudaMemsetAsync(d->d_g, 0, (size_t)Q * d->Nf * sizeof(T), d->stream), "reset g");
  cdi_status s = launch_velocity<T, DIM>(d);
  if (s != CDI_OK) return s;
  // K steps captured once as a graph (parameters are baked in)
  if (!d->flow_graph || d->flow_graph_K != K || d->flow_graph_tau != p->tau ||
      d->flow_graph_force != p->force_lu) {
    if (d->flow_graph) cudaGraphExecDestroy(d->flow_graph);
    d->flow_graph = nullptr;
    cudaGraph_t graph;
    CDI_TRY(d, cudaStreamBeginCapture(d->cap_stream, cudaStreamCaptureModeThreadLocal),
            "begin capture");
    for (int k = 0; k < K / 2; k++) launch_step_pair<T, DIM>(d, d->cap_stream, omega, fxh, fsrc);
    cudaError_t e = cudaStreamEndCapture(d->cap_stream, &graph);
    CDI_TRY(d, e, "end capture");
    e = cudaGraphInstantiate(&d->flow_graph, graph, 0);
    cudaGraphDestroy(graph);
    CDI_TRY(d, e, "instantiate flow graph");
    d->flow_graph_K = K;
    d->flow_graph_tau = p->tau;
    d->flow_graph_force = p->force_lu;
  }
  int64_t steps = 0;
  double r = NAN;
  bool converged = false;
  while (steps < p->max_steps) {
    cudaEvent_t a;
    cdi_timing_begin(d, &a);
    CDI_TRY(d, cudaGraphLaunch(d->flow_graph, d->stream), "flow graph");
    cdi_timing_end(d, a, PH_FLOW, K);
    d->timing.kernel_launches += K;
    steps += K;
    cdi_timing_begin(d, &a);
    s = launch_velocity<T, DIM>(d);
    if (s != CDI_OK) return s;
    CDI_TRY(d, cudaMemcpyAsync(d->h_scal + S_RES_NUM, d->d_scal + S_RES_NUM, 3 * sizeof(double),
                               cudaMemcpyDeviceToHost, d->stream),
            "residual copy");
    cdi_timing_end(d, a, PH_CHECK, 1);
    CDI_TRY(d, cudaStreamSynchronize(d->stream), "flow chunk");
    r = d->h_scal[S_RES];
    if (!std::isfinite(r)) return cdi_fail(d, CDI_ERR_CUDA, "flow diverged (non-finite residual)");
    if (p->tol > 0.0 && r < p->tol) {
      converged = true;
      break;
    }
  }
  CDI_TRY(d, cdi_timing_resolve(d), "timing");
  d->flow_steps = steps;
  d->flow_residual = r;
  *steps_out = steps;
  *res_out = r;
  if (p->tol > 0.0 && !converged) return CDI_ERR_NOT_CONVERGED;
  return CDI_OK;
}

template <typename T, int DIM>
cdi_status flow_export(cdi_domain *d, double U_target) {
  k_flow_mean<<<kRedBlocks, kRedThreads, 0, d->stream>>>(
      d->d_uflow, d->d_mask, d->nx, d->NX, d->N, (double)d->n_pore, U_target, d->d_part,
      d->d_counter + C_ULAT, d->d_scal);
  k_flow_scale<T, DIM><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
      d->d_uflow, d->d_mask, (T *)d->d_u, d->nx, d->NX, d->N, d->Nf, d->d_scal);
  d->timing.kernel_launches += 2;
  CDI_TRY(d, cudaGetLastError(), "velocity export");
  CDI_TRY(d, cudaMemcpyAsync(d->h_scal + S_ULAT, d->d_scal + S_ULAT, 2 * sizeof(double),
                             cudaMemcpyDeviceToHost, d->stream),
          "export copy");
  CDI_TRY(d, cudaStreamSynchronize(d->stream), "velocity export");
  d->U_lat = d->h_scal[S_ULAT];
  d->U_target = U_target;
  if (U_target != 0.0 && d->U_lat == 0.0)
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "no net flow through the pore space to scale");
  return CDI_OK;
}

template <int DIM>
cdi_status build_flags(cdi_domain *d) {
  using FT = typename FlowFlag<DIM>::type;
  dim3 grid((d->NX + kRowBlock - 1) / kRowBlock, d->ny, d->nz);
  k_flow_flags<DIM><<<grid, kRowBlock, 0, d->stream>>>(d->d_mask, (FT *)d->d_fflags, d->nx,
                                                       d->NX, d->ny, d->nz, d->walls);
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "flow flags");
  return CDI_OK;
}

}  // namespace

cdi_status cdi_flow_build_flags(cdi_domain *d) {
  return d->dim == 2 ? build_flags<2>(d) : build_flags<3>(d);
}

cdi_status cdi_flow_run(cdi_domain *d, const cdi_flow_params *p, int64_t *steps, double *res) {
  if (d->prec == CDI_FP64)
    return d->dim == 2 ? flow_run<double, 2>(d, p, steps, res) : flow_run<double, 3>(d, p, steps, res);
  return d->dim == 2 ? flow_run<float, 2>(d, p, steps, res) : flow_run<float, 3>(d, p, steps, res);
}

cdi_status cdi_flow_export(cdi_domain *d, double U_target) {
  if (d->prec == CDI_FP64)
    return d->dim == 2 ? flow_export<double, 2>(d, U_target) : flow_export<double, 3>(d, U_target);
  return d->dim == 2 ? flow_export<float, 2>(d, U_target) : flow_export<float, 3>(d, U_target);
}
