// Explicit finite-volume Nernst-Planck transport (Eq. 3) with the adsorption
// flux of Eq. 6, and the transport queries.
//
// Per pore cell P, species k, face f with outward normal n:
//   pore or ghost neighbour:  P_f = (u_f . n) dx / D_k - z_k (phi_nb - phi_P)
//                             J   = (D_k/dx) [B(-P_f) C_P - B(P_f) C_nb]
// (each product is accurate on its own; the equivalent form
// B(-P)(C_P - C_nb) + P C_nb cancels catastrophically for large |P|)
//   solid face (Eq. 6):       J   = K_eff C_P,  K_eff = Ka / (1 + Ka dx/(2 D_k))
//   lateral wall:             J   = 0
// with B(x) = x / (exp(x) - 1) (exponential fitting of advection and
// migration against diffusion), u_f the mean of the two cell velocities,
// phi = psi / V_T (kept to FP64 accuracy; the face difference is rounded to
// the storage precision only after subtraction).  The inlet ghost holds C = c0,
// phi = 0, u = u_P; the outlet ghost copies the cell (zero gradient).  Update: C_P -= (dt/dx) sum_f J.
// Adsorbed / inflow / outflow fluxes are summed per block in FP64 into
// per-block accumulators (fixed block -> cells map, so the totals are
// deterministic).
#include <cmath>

#include "cdi_internal.cuh"

using namespace cdi;

namespace {

enum { F_PORE = 0, F_SOLID = 1, F_INLET = 2, F_OUTLET = 3, F_WALL = 4 };

template <typename T> struct NPConst {
  T dxD[kMaxSpecies];   // dx / D_k
  T Ddx[kMaxSpecies];   // D_k / dx
  T Keff[kMaxSpecies];  // half-cell closure of Eq. 6
  T zf[kMaxSpecies];    // valence
  T dtdx;               // dt / dx
  T c0;                 // feed concentration
};

template <int DIM>
__global__ void k_np_flags(const uint8_t *__restrict__ mask, NFlag *__restrict__ fl, int nx,
                           int ny, int nz, int walls) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long P = ((long long)z * ny + y) * nx + x;
  unsigned f = mask[P] ? 1u : 0u;
  for (int fc = 0; fc < 2 * DIM; fc++) {
    const int a = fc >> 1, s = (fc & 1) ? -1 : 1;
    int X = x, Y = y, Z = z;
    bool edge = false;
    if (a == 0) {
      X += s;
      edge = X < 0 || X >= nx;
    } else if (a == 1) {
      Y += s;
      edge = Y < 0 || Y >= ny;
      Y = (Y + ny) % ny;
    } else {
      Z += s;
      edge = Z < 0 || Z >= nz;
      Z = (Z + nz) % nz;
    }
    if (edge) f |= 1u << (kEdgeBit + fc);
    if ((a == 0 && edge) || (edge && walls)) continue;
    if (mask[((long long)Z * ny + Y) * nx + X]) f |= 1u << (kFaceBit + fc);
  }
  fl[P] = (NFlag)f;
}

// Face kind of face fc of pore cell P and, for a pore neighbour, its index Q,
// from the flag word alone (the edge bits carry the boundary position).
template <int DIM>
__device__ __forceinline__ int np_face(unsigned f, int fc, int nx, int ny, int nz, int walls,
                                       long long P, long long &Q) {
  const int a = fc >> 1, s = (fc & 1) ? -1 : 1;
  const bool edge = (f >> (kEdgeBit + fc)) & 1u;
  if (a == 0) {
    if (edge) return s > 0 ? F_OUTLET : F_INLET;
    if ((f >> (kFaceBit + fc)) & 1u) return F_SOLID;
    Q = P + s;
    return F_PORE;
  }
  if (edge && walls) return F_WALL;
  if ((f >> (kFaceBit + fc)) & 1u) return F_SOLID;
  const long long stride = a == 1 ? (long long)nx : (long long)nx * ny;
  const long long extent = a == 1 ? ny : nz;
  Q = P + (edge ? -s * (extent - 1) * stride : s * stride);
  return F_PORE;
}

// B(P_f) and B(-P_f) for the face Peclet number P_f = adv - z (phi_nb - phi_P).
template <typename T> struct FaceB;

template <> struct FaceB<double> {
  __device__ static void dphi(double nb, double p, double &hi, double &lo) {
    hi = nb - p;
    lo = 0.0;
  }
  __device__ static void eval(double adv, double z, double dhi, double, double &Bp,
                              double &Bm) {
    bernoulli_pair(adv - z * dhi, Bp, Bm);
  }
};

// FP32 carries the potential difference and P_f as unevaluated pairs
// (hi + lo): an exponent |P| rounded to FP32 costs a relative error of about
// |P| * 6e-8 in each Boltzmann factor exp(P), which accumulates across an
// electric double layer.  B is evaluated at hi and corrected to first order
// in lo with B'(x) = B(x) ((1 - B(x)) / x - 1).
template <> struct FaceB<float> {
  __device__ static void dphi(float2 nb, float2 p, float &hi, float &lo) {
    const float d = __fsub_rn(nb.x, p.x);
    const float bv = __fsub_rn(d, nb.x);
    const float e = __fadd_rn(__fsub_rn(nb.x, __fsub_rn(d, bv)), __fsub_rn(-p.x, bv));
    hi = d;
    lo = __fadd_rn(e, __fsub_rn(nb.y, p.y));
  }
  __device__ static void eval(float adv, float z, float dhi, float dlo, float &Bp, float &Bm) {
    const float p = __fmaf_rn(-z, dhi, adv);
    const bool neg = p < 0.f;
    float Ba, Bma;
    if (fabsf(p) < 0.5f) {
      // Almost every face: B(a) from its Taylor series (Bernoulli numbers)
      // through a^8, truncation below 3e-11 for a < 1/2.  Dropping the low
      // part of P shifts B by less than 4e-8 relative here.
      const float a = fabsf(p), a2 = a * a;
      float t = __fmaf_rn(-1.f / 1209600.f, a2, 1.f / 30240.f);
      t = __fmaf_rn(t, a2, -1.f / 720.f);
      t = __fmaf_rn(t, a2, 1.f / 12.f);
      Ba = __fmaf_rn(t, a2, __fmaf_rn(-0.5f, a, 1.f));
      Bma = Ba + a;
    } else {
      // P = adv - z (dhi + dlo) as ph + pl, B at |ph| corrected for pl
      const float zd = __fmul_rn(z, dhi);
      const float zde = __fmaf_rn(z, dhi, -zd);
      const float ph = __fsub_rn(adv, zd);
      const float bb = __fsub_rn(ph, adv);
      const float phe = __fadd_rn(__fsub_rn(adv, __fsub_rn(ph, bb)), __fsub_rn(-zd, bb));
      const float pl = __fsub_rn(__fsub_rn(phe, zde), __fmul_rn(z, dlo));
      const float ah = neg ? -ph : ph, al = neg ? -pl : pl;
      // B(a) = a e^-a / (1 - e^-a) is below 1e-33 beyond a = 80
      Ba = ah > 80.f ? 0.f : __fdividef(ah, expm1f(ah));
      Ba = __fmaf_rn(Ba * al, __fdividef(1.f - Ba, ah) - 1.f, Ba);
      Bma = (Ba + ah) + al;  // B(-a) = B(a) + a, no cancellation
    }
    Bp = neg ? Bma : Ba;
    Bm = neg ? Ba : Bma;
  }
};

// One explicit step of one pore cell P for NS species: writes the new
// concentrations and adds the cell's adsorbed (v[k]), inflow (v[NS+k]) and
// outflow (v[2NS+k]) fluxes.
template <typename T, int DIM, int NS>
__device__ __forceinline__ void np_cell(const T *__restrict__ Cin, T *__restrict__ Cout,
                                        const T *__restrict__ u,
                                        const typename PhiStore<T>::type *__restrict__ phi,
                                        unsigned f, const NPConst<T> &c, int nx, int ny, int nz,
                                        long long N, int walls, long long P, T (&v)[3 * NS]) {
  using PS = PhiStore<T>;
  using PT = typename PS::type;
  constexpr int NF = 2 * DIM;
  // face kinds and neighbour cells first (32-bit indices: N < 2^31); a
  // non-pore face stands in the own cell, whose values an outlet ghost copies
  const int Pi = (int)P;
  int kind[NF], Qi[NF];
#pragma unroll
  for (int fc = 0; fc < NF; fc++) {
    long long Q = P;
    kind[fc] = np_face<DIM>(f, fc, nx, ny, nz, walls, P, Q);
    Qi[fc] = kind[fc] == F_PORE ? (int)Q : Pi;
  }
  // every load issued before any arithmetic (memory-level parallelism)
  T CP[NS], sumJ[NS], un[NF], Cn[NF][NS];
  PT phn[NF];
#pragma unroll
  for (int k = 0; k < NS; k++) {
    CP[k] = Cin[(size_t)k * N + Pi];
    sumJ[k] = T(0);
  }
  const PT phiP = phi[Pi];
  T uP[DIM];
#pragma unroll
  for (int a = 0; a < DIM; a++) uP[a] = u[(size_t)a * N + Pi];
#pragma unroll
  for (int fc = 0; fc < NF; fc++) {
    un[fc] = u[(size_t)(fc >> 1) * N + Qi[fc]];
    phn[fc] = phi[Qi[fc]];
#pragma unroll
    for (int k = 0; k < NS; k++) Cn[fc][k] = Cin[(size_t)k * N + Qi[fc]];
  }
#pragma unroll
  for (int fc = 0; fc < NF; fc++) {
    const int a = fc >> 1;
    const T sg = (fc & 1) ? T(-1) : T(1);
    if (kind[fc] == F_WALL) continue;
    if (kind[fc] == F_SOLID) {
#pragma unroll
      for (int k = 0; k < NS; k++) {
        const T J = c.Keff[k] * CP[k];
        sumJ[k] += J;
        v[k] += J;
      }
      continue;
    }
    if (kind[fc] == F_INLET) {  // feed ghost: C = c0, phi = 0, u = u_P
      phn[fc] = PS::zero();
#pragma unroll
      for (int k = 0; k < NS; k++) Cn[fc][k] = c.c0;
    }
    const T uf = T(0.5) * (uP[a] + un[fc]) * sg;
    T dhi, dlo;
    FaceB<T>::dphi(phn[fc], phiP, dhi, dlo);
#pragma unroll
    for (int k = 0; k < NS; k++) {
      T Bp, Bm;
      FaceB<T>::eval(uf * c.dxD[k], c.zf[k], dhi, dlo, Bp, Bm);
      const T J = c.Ddx[k] * (Bm * CP[k] - Bp * Cn[fc][k]);
      sumJ[k] += J;
      if (kind[fc] == F_INLET) v[NS + k] -= J;
      if (kind[fc] == F_OUTLET) v[2 * NS + k] += J;
    }
  }
#pragma unroll
  for (int k = 0; k < NS; k++) Cout[(size_t)k * N + Pi] = CP[k] - c.dtdx * sumJ[k];
}

// Block sums of v in T, added by thread 0 to the block's own FP64 accounts
// acc[(3*k + kind) * gridDim.x + block], kind 0 Gamma, 1 In, 2 Out (one
// thread per pore cell, so the block -> cells map is fixed and the totals are
// deterministic).  Every thread of the block must call it.
template <typename T, int NS>
__device__ __forceinline__ void np_account(T (&v)[3 * NS], T *sm, double *__restrict__ acc) {
  block_reduce<3 * NS>(v, sm, OpSum(), T(0));
  if (threadIdx.x == 0) {
    const int bid = blockIdx.x, nblocks = gridDim.x;
#pragma unroll
    for (int k = 0; k < NS; k++) {
      acc[(size_t)(3 * k + 0) * nblocks + bid] += (double)v[k];
      acc[(size_t)(3 * k + 1) * nblocks + bid] += (double)v[NS + k];
      acc[(size_t)(3 * k + 2) * nblocks + bid] += (double)v[2 * NS + k];
    }
  }
}

template <typename T, int DIM, int NS>
__global__ void __launch_bounds__(kRowBlock)
    k_np_step(const T *__restrict__ Cin, T *__restrict__ Cout, const T *__restrict__ u,
              const typename PhiStore<T>::type *__restrict__ phi,
              const NFlag *__restrict__ fl, const int *__restrict__ cells, int n_cells,
              NPConst<T> c, double *__restrict__ acc, int nx, int ny, int nz, long long N,
              int walls) {
  __shared__ T sm[3 * NS * 32];
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  T v[3 * NS];
#pragma unroll
  for (int j = 0; j < 3 * NS; j++) v[j] = T(0);
  if (k0 < n_cells) {
    const long long P = cells[k0];
    np_cell<T, DIM, NS>(Cin, Cout, u, phi, fl[P], c, nx, ny, nz, N, walls, P, v);
  }
  np_account<T, NS>(v, sm, acc);
}

// One member of a fused sweep: its own concentrations, velocity, potential,
// constants (time step) and accounts.
template <typename T> struct SweepMember {
  T *C[2];          // concentration buffers (ping-pong)
  const T *u;
  const typename PhiStore<T>::type *phi;
  double *acc;
  NPConst<T> c;
};

// All members of a sweep advance one step in one launch: each block runs the
// same cells for every member in turn (the block -> cells map, the arithmetic
// and the accounts of a member are those of k_np_step, so a member's result
// equals a single run's bit for bit).
template <typename T, int DIM, int NS>
__global__ void __launch_bounds__(kRowBlock)
    k_np_sweep(const SweepMember<T> *__restrict__ members, int n_members, int in,
               const NFlag *__restrict__ fl, const int *__restrict__ cells, int n_cells, int nx,
               int ny, int nz, long long N, int walls) {
  __shared__ T sm[3 * NS * 32];
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  const long long P = k0 < n_cells ? cells[k0] : 0;
  const unsigned f = k0 < n_cells ? fl[P] : 1u;
  for (int m = 0; m < n_members; m++) {
    const SweepMember<T> &mb = members[m];
    T v[3 * NS];
#pragma unroll
    for (int j = 0; j < 3 * NS; j++) v[j] = T(0);
    if (k0 < n_cells)
      np_cell<T, DIM, NS>(mb.C[in], mb.C[1 - in], mb.u, mb.phi, f, mb.c, nx, ny, nz, N, walls,
                          P, v);
    np_account<T, NS>(v, sm, mb.acc);
  }
}

// Largest outflow rate over pore cells and species, in FP64 from the FP64
// lattice velocity and potential:  (1/dx) [sum_{open faces} (D/dx) B(-P_f)
// + n_solid K_eff]; dt = safety / max.
template <int DIM>
__global__ void __launch_bounds__(kRedThreads)
    k_np_rate(const NFlag *__restrict__ fl, const double *__restrict__ uflow,
              const double *__restrict__ psi, NPConst<double> c, int ns, double scale,
              double inv_vt, double inv_dx, double safety, int nx, int NX, int ny, int nz,
              long long N, long long Nf, int walls, double *__restrict__ part,
              unsigned int *counter, double *scal) {
  __shared__ double sm[32];
  double v[1] = {0.0};
  for (long long P = blockIdx.x * (long long)blockDim.x + threadIdx.x; P < N;
       P += (long long)gridDim.x * blockDim.x) {
    const unsigned f = fl[P];
    if (f & 1u) continue;
    const long long row = P / nx;
    const int x = (int)(P - row * nx);
    const long long sP = row * NX + x;
    for (int k = 0; k < ns; k++) {
      double rate = 0.0;
      for (int fc = 0; fc < 2 * DIM; fc++) {
        const int a = fc >> 1;
        const double sg = (fc & 1) ? -1.0 : 1.0;
        long long Q = 0;
        const int kind = np_face<DIM>(f, fc, nx, ny, nz, walls, P, Q);
        if (kind == F_WALL) continue;
        if (kind == F_SOLID) {
          rate += c.Keff[k];
          continue;
        }
        const double uP = scale * uflow[(size_t)a * Nf + sP];
        double unb = uP, psinb = 0.0;
        const double psiP = psi[P];
        if (kind == F_PORE) {
          const long long rq = Q / nx;
          unb = scale * uflow[(size_t)a * Nf + rq * NX + (Q - rq * nx)];
          psinb = psi[Q];
        } else if (kind == F_OUTLET) {
          psinb = psiP;
        }
        const double Pf = 0.5 * (uP + unb) * sg * c.dxD[k] - c.zf[k] * (psinb - psiP) * inv_vt;
        double Bp, Bm;
        bernoulli_pair(Pf, Bp, Bm);
        rate += c.Ddx[k] * Bm;
      }
      v[0] = fmax(v[0], rate * inv_dx);
    }
  }
  block_reduce<1>(v, sm, OpMax(), 0.0);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  if (last_block(counter, gridDim.x)) {
    combine_partials<1>(part, gridDim.x, v, sm, OpMax(), 0.0);
    if (threadIdx.x == 0) {
      scal[S_RATE] = v[0];
      scal[S_DT] = v[0] > 0.0 ? safety / v[0] : 0.0;
      *counter = 0;
    }
  }
}

template <typename T>
__global__ void k_np_init(const NFlag *__restrict__ fl, T *__restrict__ C0, T *__restrict__ C1,
                          long long N, int ns, T c0) {
  for (long long P = blockIdx.x * (long long)blockDim.x + threadIdx.x; P < N;
       P += (long long)gridDim.x * blockDim.x) {
    const bool pore = !(fl[P] & 1);
#pragma unroll
    for (int k = 0; k < kMaxSpecies; k++) {
      const T v = (pore && k < ns) ? c0 : T(0);
      C0[(size_t)k * N + P] = v;
      C1[(size_t)k * N + P] = v;
    }
  }
}

// Dissolved amount, outlet sums (flux weighted and plain) per species.
// Values: [0,4) mass, [4,8) sum u_x C at the outlet, 8 sum u_x, [9,13) plain
// sum of C at the outlet, 13 pore cells in the outlet column.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    k_np_sums(const NFlag *__restrict__ fl, const T *__restrict__ C, const T *__restrict__ u,
              long long N, int nx, int ns, double cell_vol, double *__restrict__ part,
              unsigned int *counter, double *scal) {
  constexpr int NV = 14;
  __shared__ double sm[NV * 32];
  double v[NV];
#pragma unroll
  for (int j = 0; j < NV; j++) v[j] = 0.0;
  for (long long P = blockIdx.x * (long long)blockDim.x + threadIdx.x; P < N;
       P += (long long)gridDim.x * blockDim.x) {
    if (fl[P] & 1u) continue;
    const bool outlet = (P % nx) == nx - 1;
    const double ux = (double)u[P];
#pragma unroll
    for (int k = 0; k < kMaxSpecies; k++) {
      if (k >= ns) break;
      const double ck = (double)C[(size_t)k * N + P];
      v[k] += ck;
      if (outlet) {
        v[4 + k] += ux * ck;
        v[9 + k] += ck;
      }
    }
    if (outlet) {
      v[8] += ux;
      v[13] += 1.0;
    }
  }
  block_reduce<NV>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < NV; j++) part[(size_t)j * gridDim.x + blockIdx.x] = v[j];
  if (last_block(counter, gridDim.x)) {
    combine_partials<NV>(part, gridDim.x, v, sm, OpSum(), 0.0);
    if (threadIdx.x == 0) {
      for (int k = 0; k < kMaxSpecies; k++) {
        scal[S_MASS + k] = v[k] * cell_vol;
        scal[S_OUT + 2 * k] = v[4 + k];
        scal[S_OUT + 2 * k + 1] = v[8];
        scal[S_OUTP + k] = v[9 + k];
      }
      scal[S_OUTN] = v[13];
      *counter = 0;
    }
  }
}

// Pore cells and pore-solid faces inside the image (the interface the
// specific surface of Sec. 4 measures), counted over the pore-cell list.
__global__ void __launch_bounds__(kRedThreads)
    k_geometry(const NFlag *__restrict__ fl, const int *__restrict__ cells, int n, int faces,
               double *__restrict__ part, unsigned int *counter, double *scal) {
  __shared__ double sm[2 * 32];
  double v[2] = {0.0, 0.0};
  const unsigned face_bits = ((1u << faces) - 1u) << kFaceBit;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    v[0] += 1.0;
    v[1] += (double)__popc(fl[cells[k]] & face_bits);
  }
  block_reduce<2>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = v[0];
    part[gridDim.x + blockIdx.x] = v[1];
  }
  if (last_block(counter, gridDim.x)) {
    combine_partials<2>(part, gridDim.x, v, sm, OpSum(), 0.0);
    if (threadIdx.x == 0) {
      scal[S_GEOM] = v[0];
      scal[S_GEOM + 1] = v[1];
      *counter = 0;
    }
  }
}

// Totals of the per-block Gamma/In/Out accumulators (one block, fixed order).
__global__ void __launch_bounds__(kRedThreads)
    k_acc_total(const double *__restrict__ acc, int nblocks, double *scal) {
  constexpr int NV = 3 * kMaxSpecies;
  __shared__ double sm[NV * 32];
  double v[NV];
  combine_partials<NV>(acc, nblocks, v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < NV; j++) scal[S_ACC + j] = v[j];
}

// Mean of species k over the pore cells of each x column.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    k_colmeans(const NFlag *__restrict__ fl, const T *__restrict__ C, int nx, long long rows,
               double *__restrict__ out) {
  __shared__ double sm[2 * 32];
  const int x = blockIdx.x;
  double v[2] = {0.0, 0.0};
  for (long long r = threadIdx.x; r < rows; r += blockDim.x) {
    const long long P = r * nx + x;
    if (fl[P] & 1u) continue;
    v[0] += (double)C[P];
    v[1] += 1.0;
  }
  block_reduce<2>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0) out[x] = v[1] > 0.0 ? v[0] / v[1] : 0.0;
}

template <typename T> NPConst<T> make_const(const cdi_domain *d) {
  NPConst<T> c{};
  for (int k = 0; k < kMaxSpecies; k++) {
    c.dxD[k] = (T)(d->dx / d->D[k]);
    c.Ddx[k] = (T)(d->D[k] / d->dx);
    c.Keff[k] = (T)(d->Ka / (1.0 + d->Ka * d->dx / (2.0 * d->D[k])));
    c.zf[k] = (T)d->z[k];
  }
  c.dtdx = (T)(d->dt / d->dx);
  c.c0 = (T)d->c0;
  return c;
}

template <typename T, int DIM, int NS>
void launch_step_t(cdi_domain *d, cudaStream_t st, int in) {
  // one thread per pore cell; np_blocks blocks, one FP64 account set each
  k_np_step<T, DIM, NS><<<d->np_blocks, kRowBlock, 0, st>>>(
      (const T *)d->d_C[in], (T *)d->d_C[1 - in], (const T *)d->d_u,
      (const typename PhiStore<T>::type *)d->d_phi, d->d_nflags, d->d_cell_list,
      (int)d->n_pore, make_const<T>(d), d->d_acc, d->nx, d->ny, d->nz, d->N, d->walls);
}

template <typename T, int DIM>
void launch_step_d(cdi_domain *d, cudaStream_t st, int in) {
  switch (d->ns) {
    case 1: launch_step_t<T, DIM, 1>(d, st, in); break;
    case 2: launch_step_t<T, DIM, 2>(d, st, in); break;
    case 3: launch_step_t<T, DIM, 3>(d, st, in); break;
    default: launch_step_t<T, DIM, 4>(d, st, in); break;
  }
}

void launch_step(cdi_domain *d, cudaStream_t st, int in) {
  if (d->prec == CDI_FP64) {
    if (d->dim == 2) launch_step_d<double, 2>(d, st, in);
    else launch_step_d<double, 3>(d, st, in);
  } else {
    if (d->dim == 2) launch_step_d<float, 2>(d, st, in);
    else launch_step_d<float, 3>(d, st, in);
  }
}

constexpr int kGraphSteps = 64;  // steps per captured transport graph (even)

}  // namespace

cdi_status cdi_np_build_flags(cdi_domain *d) {
  dim3 grid((d->nx + kRowBlock - 1) / kRowBlock, d->ny, d->nz);
  if (d->dim == 2)
    k_np_flags<2><<<grid, kRowBlock, 0, d->stream>>>(d->d_mask, d->d_nflags, d->nx, d->ny, d->nz,
                                                     d->walls);
  else
    k_np_flags<3><<<grid, kRowBlock, 0, d->stream>>>(d->d_mask, d->d_nflags, d->nx, d->ny, d->nz,
                                                     d->walls);
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "face flags");
  return CDI_OK;
}

cdi_status cdi_np_init(cdi_domain *d, double dt_s, double *dt_used) {
  if (d->np_graph) cudaGraphExecDestroy(d->np_graph);
  d->np_graph = nullptr;
  double dt = dt_s;
  if (dt <= 0.0) {
    cdi_status s = cdi_np_dt(d, d->h_scal[S_SCALE], &dt);
    if (s != CDI_OK) return s;
  }
  d->dt = dt;
  if (dt_used) *dt_used = dt;
  if (d->prec == CDI_FP64)
    k_np_init<double><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        d->d_nflags, (double *)d->d_C[0], (double *)d->d_C[1], d->N, d->ns, d->c0);
  else
    k_np_init<float><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        d->d_nflags, (float *)d->d_C[0], (float *)d->d_C[1], d->N, d->ns, (float)d->c0);
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "transport init");
  CDI_TRY(d, cudaMemsetAsync(d->d_acc, 0, (size_t)3 * kMaxSpecies * d->np_blocks * 8, d->stream),
          "reset accumulators");
  d->cur = 0;
  d->np_steps = 0;
  return CDI_OK;
}

// Explicit time step for the current potential (d_psi) and the solved flow
// scaled by `scale` (the species set in the domain).
cdi_status cdi_np_dt(cdi_domain *d, double scale, double *dt_out) {
  double dt = 0.0;
  {
    NPConst<double> c = make_const<double>(d);
    if (d->dim == 2)
      k_np_rate<2><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
          d->d_nflags, d->d_uflow, d->d_psi, c, d->ns, scale, 1.0 / d->VT, 1.0 / d->dx, 0.9,
          d->nx, d->NX, d->ny, d->nz, d->N, d->Nf, d->walls, d->d_part, d->d_counter + C_DT,
          d->d_scal);
    else
      k_np_rate<3><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
          d->d_nflags, d->d_uflow, d->d_psi, c, d->ns, scale, 1.0 / d->VT, 1.0 / d->dx, 0.9,
          d->nx, d->NX, d->ny, d->nz, d->N, d->Nf, d->walls, d->d_part, d->d_counter + C_DT,
          d->d_scal);
    d->timing.kernel_launches++;
    CDI_TRY(d, cudaGetLastError(), "time step kernel");
    CDI_TRY(d, cudaMemcpyAsync(d->h_scal + S_RATE, d->d_scal + S_RATE, 2 * sizeof(double),
                               cudaMemcpyDeviceToHost, d->stream),
            "time step copy");
    CDI_TRY(d, cudaStreamSynchronize(d->stream), "time step");
    dt = d->h_scal[S_DT];
    if (!(dt > 0.0) || !std::isfinite(dt))
      return cdi_fail(d, CDI_ERR_INVALID_ARG, "no finite time step (no flux anywhere?)");
  }
  *dt_out = dt;
  return CDI_OK;
}

// ---------------------------------------------------------------------------
// Fused sweep: n members on one geometry, one launch per step for all.
// ---------------------------------------------------------------------------
namespace {

template <typename T, int DIM>
void launch_sweep_d(cdi_domain *d, cudaStream_t st, const void *members, int n, int in) {
  const SweepMember<T> *m = (const SweepMember<T> *)members;
  switch (d->ns) {
    case 1:
      k_np_sweep<T, DIM, 1><<<d->np_blocks, kRowBlock, 0, st>>>(
          m, n, in, d->d_nflags, d->d_cell_list, (int)d->n_pore, d->nx, d->ny, d->nz, d->N,
          d->walls);
      break;
    case 2:
      k_np_sweep<T, DIM, 2><<<d->np_blocks, kRowBlock, 0, st>>>(
          m, n, in, d->d_nflags, d->d_cell_list, (int)d->n_pore, d->nx, d->ny, d->nz, d->N,
          d->walls);
      break;
    case 3:
      k_np_sweep<T, DIM, 3><<<d->np_blocks, kRowBlock, 0, st>>>(
          m, n, in, d->d_nflags, d->d_cell_list, (int)d->n_pore, d->nx, d->ny, d->nz, d->N,
          d->walls);
      break;
    default:
      k_np_sweep<T, DIM, 4><<<d->np_blocks, kRowBlock, 0, st>>>(
          m, n, in, d->d_nflags, d->d_cell_list, (int)d->n_pore, d->nx, d->ny, d->nz, d->N,
          d->walls);
      break;
  }
}

void launch_sweep(cdi_domain *d, cudaStream_t st, const void *members, int n, int in) {
  if (d->prec == CDI_FP64) {
    if (d->dim == 2) launch_sweep_d<double, 2>(d, st, members, n, in);
    else launch_sweep_d<double, 3>(d, st, members, n, in);
  } else {
    if (d->dim == 2) launch_sweep_d<float, 2>(d, st, members, n, in);
    else launch_sweep_d<float, 3>(d, st, members, n, in);
  }
}

template <typename T>
cdi_status sweep_run(cdi_domain *d, int n, const double *scale, const int *group,
                     void *const *phi_groups, const double *dts, int64_t n_steps,
                     double *gamma, double *cout) {
  const size_t TN = (size_t)d->N * sizeof(T);
  const int ns = d->ns;
  // per-member device memory: velocity, two concentration buffers, accounts
  std::vector<void *> blocks;
  auto take = [&](size_t bytes) {
    void *p = cdi_dev_alloc(d, bytes);
    if (p) blocks.push_back(p);
    return p;
  };
  std::vector<SweepMember<T>> hm(n);
  bool ok = true;
  for (int m = 0; m < n && ok; m++) {
    void *u = take((size_t)d->dim * TN);
    void *c0 = take((size_t)kMaxSpecies * TN), *c1 = take((size_t)kMaxSpecies * TN);
    void *acc = take((size_t)3 * kMaxSpecies * d->np_blocks * 8);
    ok = u && c0 && c1 && acc;
    if (!ok) break;
    d->dt = dts[m];
    hm[m].C[0] = (T *)c0;
    hm[m].C[1] = (T *)c1;
    hm[m].u = (const T *)u;
    hm[m].phi = (const typename PhiStore<T>::type *)phi_groups[group[m]];
    hm[m].acc = (double *)acc;
    hm[m].c = make_const<T>(d);
  }
  void *dmem = ok ? take(sizeof(SweepMember<T>) * n) : nullptr;
  cdi_status s = CDI_OK;
  if (!ok || !dmem) s = cdi_fail(d, CDI_ERR_OOM, "sweep: device allocation failed");
  for (int m = 0; m < n && s == CDI_OK; m++) {
    s = cdi_flow_scale_to(d, scale[m], (void *)hm[m].u);
    if (s != CDI_OK) break;
    k_np_init<T><<<kRedBlocks, kRedThreads, 0, d->stream>>>(d->d_nflags, hm[m].C[0], hm[m].C[1],
                                                            d->N, ns, (T)d->c0);
    d->timing.kernel_launches++;
    if (cudaMemsetAsync(hm[m].acc, 0, (size_t)3 * kMaxSpecies * d->np_blocks * 8, d->stream) !=
        cudaSuccess)
      s = cdi_fail(d, CDI_ERR_CUDA, "sweep: memset");
  }
  if (s == CDI_OK &&
      cudaMemcpyAsync(dmem, hm.data(), sizeof(SweepMember<T>) * n, cudaMemcpyHostToDevice,
                      d->stream) != cudaSuccess)
    s = cdi_fail(d, CDI_ERR_CUDA, "sweep: member table");
  // steps: graphs of kGraphSteps fused launches (even, so the parity returns)
  cudaGraphExec_t exec = nullptr;
  int64_t done = 0;
  if (s == CDI_OK) {
    cudaEvent_t ev;
    cdi_timing_begin(d, &ev);
    if (n_steps >= kGraphSteps) {
      cudaGraph_t graph;
      cudaError_t e = cudaStreamBeginCapture(d->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        for (int k = 0; k < kGraphSteps; k++) launch_sweep(d, d->cap_stream, dmem, n, k & 1);
        e = cudaStreamEndCapture(d->cap_stream, &graph);
      }
      if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
      }
      if (e != cudaSuccess) s = cdi_cuda_fail(d, e, "sweep graph");
      while (s == CDI_OK && n_steps - done >= kGraphSteps) {
        e = cudaGraphLaunch(exec, d->stream);
        if (e != cudaSuccess) s = cdi_cuda_fail(d, e, "sweep graph launch");
        done += kGraphSteps;
      }
    }
    for (; s == CDI_OK && done < n_steps; done++) launch_sweep(d, d->stream, dmem, n, (int)(done & 1));
    cudaError_t e = cudaGetLastError();
    if (s == CDI_OK && e != cudaSuccess) s = cdi_cuda_fail(d, e, "sweep step");
    cdi_timing_end(d, ev, PH_NP, n_steps);
    d->timing.kernel_launches += n_steps;
  }
  // outputs per member, through the same reductions as a single run
  const int cur = (int)(n_steps & 1);
  const double area = d->dim == 2 ? d->dx : d->dx * d->dx;
  const double vol = d->dim == 2 ? d->dx * d->dx : d->dx * d->dx * d->dx;
  for (int m = 0; m < n && s == CDI_OK; m++) {
    k_np_sums<T><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        d->d_nflags, hm[m].C[cur], hm[m].u, d->N, d->nx, ns, vol, d->d_part,
        d->d_counter + C_MASS, d->d_scal);
    k_acc_total<<<1, kRedThreads, 0, d->stream>>>(hm[m].acc, d->np_blocks, d->d_scal);
    d->timing.kernel_launches += 2;
    cudaError_t e = cudaMemcpyAsync(d->h_scal + S_OUT, d->d_scal + S_OUT,
                                    (S_OUTN - S_OUT + 1) * sizeof(double),
                                    cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) {
      s = cdi_cuda_fail(d, e, "sweep outputs");
      break;
    }
    for (int k = 0; k < ns; k++) {
      gamma[m * ns + k] = d->h_scal[S_ACC + 3 * k] * dts[m] * area;
      const double num = d->h_scal[S_OUT + 2 * k], den = d->h_scal[S_OUT + 2 * k + 1];
      const double cnt = d->h_scal[S_OUTN];
      cout[m * ns + k] = den != 0.0 ? num / den : (cnt > 0 ? d->h_scal[S_OUTP + k] / cnt : 0.0);
    }
  }
  if (s == CDI_OK) {
    cudaError_t e = cdi_timing_resolve(d);
    if (e != cudaSuccess) s = cdi_cuda_fail(d, e, "timing");
  }
  cudaStreamSynchronize(d->stream);
  if (exec) cudaGraphExecDestroy(exec);
  for (void *p : blocks) cdi_dev_release(d, p);
  return s;
}

}  // namespace

cdi_status cdi_np_sweep(cdi_domain *d, int n, const double *scale, const int *group,
                        void *const *phi_groups, const double *dts, int64_t n_steps,
                        double *gamma, double *cout) {
  if (d->prec == CDI_FP64)
    return sweep_run<double>(d, n, scale, group, phi_groups, dts, n_steps, gamma, cout);
  return sweep_run<float>(d, n, scale, group, phi_groups, dts, n_steps, gamma, cout);
}

cdi_status cdi_np_steps(cdi_domain *d, int64_t n) {
  if (n == 0) return CDI_OK;
  cudaEvent_t ev;
  cdi_timing_begin(d, &ev);
  int64_t left = n;
  if (d->cur == 1) {
    launch_step(d, d->stream, 1);
    d->cur = 0;
    left--;
  }
  if (left >= kGraphSteps) {
    if (!d->np_graph) {
      cudaGraph_t graph;
      CDI_TRY(d, cudaStreamBeginCapture(d->cap_stream, cudaStreamCaptureModeThreadLocal),
              "begin capture");
      for (int k = 0; k < kGraphSteps; k++) launch_step(d, d->cap_stream, k & 1);
      cudaError_t e = cudaStreamEndCapture(d->cap_stream, &graph);
      CDI_TRY(d, e, "end capture");
      e = cudaGraphInstantiate(&d->np_graph, graph, 0);
      cudaGraphDestroy(graph);
      CDI_TRY(d, e, "instantiate transport graph");
    }
    while (left >= kGraphSteps) {
      CDI_TRY(d, cudaGraphLaunch(d->np_graph, d->stream), "transport graph");
      left -= kGraphSteps;
    }
  }
  while (left > 0) {
    launch_step(d, d->stream, d->cur);
    d->cur = 1 - d->cur;
    left--;
  }
  CDI_TRY(d, cudaGetLastError(), "transport step");
  cdi_timing_end(d, ev, PH_NP, n);
  d->timing.kernel_launches += n;
  d->np_steps += n;
  return CDI_OK;
}

cdi_status cdi_np_reduce(cdi_domain *d) {
  const double vol = d->dim == 2 ? d->dx * d->dx : d->dx * d->dx * d->dx;
  if (d->prec == CDI_FP64)
    k_np_sums<double><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        d->d_nflags, (const double *)d->d_C[d->cur], (const double *)d->d_u, d->N, d->nx, d->ns,
        vol, d->d_part, d->d_counter + C_MASS, d->d_scal);
  else
    k_np_sums<float><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        d->d_nflags, (const float *)d->d_C[d->cur], (const float *)d->d_u, d->N, d->nx, d->ns,
        vol, d->d_part, d->d_counter + C_MASS, d->d_scal);
  k_acc_total<<<1, kRedThreads, 0, d->stream>>>(d->d_acc, d->np_blocks, d->d_scal);
  d->timing.kernel_launches += 2;
  CDI_TRY(d, cudaGetLastError(), "transport sums");
  CDI_TRY(d, cudaMemcpyAsync(d->h_scal + S_OUT, d->d_scal + S_OUT,
                             (S_OUTN - S_OUT + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                             d->stream),
          "sums copy");
  CDI_TRY(d, cudaStreamSynchronize(d->stream), "transport sums");
  CDI_TRY(d, cdi_timing_resolve(d), "timing");
  return CDI_OK;
}

cdi_status cdi_np_geometry(cdi_domain *d, double *pores, double *faces) {
  k_geometry<<<kRedBlocks, kRedThreads, 0, d->stream>>>(d->d_nflags, d->d_cell_list,
                                                         (int)d->n_pore, 2 * d->dim, d->d_part,
                                                         d->d_counter + C_GEOM, d->d_scal);
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "geometry");
  CDI_TRY(d, cudaMemcpyAsync(d->h_scal + S_GEOM, d->d_scal + S_GEOM, 2 * sizeof(double),
                             cudaMemcpyDeviceToHost, d->stream),
          "geometry copy");
  CDI_TRY(d, cudaStreamSynchronize(d->stream), "geometry");
  *pores = d->h_scal[S_GEOM];
  *faces = d->h_scal[S_GEOM + 1];
  return CDI_OK;
}

cdi_status cdi_np_column_means(cdi_domain *d, int k) {
  const size_t T = d->prec == CDI_FP64 ? 8 : 4;
  const void *C = (const char *)d->d_C[d->cur] + (size_t)k * d->N * T;
  const long long rows = (long long)d->ny * d->nz;
  if (d->prec == CDI_FP64)
    k_colmeans<double><<<d->nx, kRedThreads, 0, d->stream>>>(d->d_nflags, (const double *)C,
                                                             d->nx, rows, d->d_colout);
  else
    k_colmeans<float><<<d->nx, kRedThreads, 0, d->stream>>>(d->d_nflags, (const float *)C, d->nx,
                                                            rows, d->d_colout);
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "column means");
  return CDI_OK;
}
