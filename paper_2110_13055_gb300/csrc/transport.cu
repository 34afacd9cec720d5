// Explicit finite-volume Nernst-Planck transport (Eq. 3) with the adsorption
// flux of Eq. 6, and the transport queries.
//
// Per pore cell P, species k, face f with outward normal n:
//   pore or ghost neighbour:  P_f = (u_f . n) dx / D_k - z_k (phi_nb - phi_P)
//                             J   = (D_k/dx) [B(-P_f) C_P - B(P_f) C_nb]
//     evaluated for |P_f| < 1/2 as (D_k/dx) [E (C_P - C_nb) + (P_f/2)(C_P + C_nb)]
//     with the even series E = B(P) + P/2, and otherwise as the two products
//     (each accurate on its own; B(-P)(C_P - C_nb) + P C_nb would cancel
//     catastrophically for large |P|)
//   solid face (Eq. 6):       J   = K_eff C_P,  K_eff = Ka / (1 + Ka dx/(2 D_k))
//   lateral wall:             J   = 0
// with B(x) = x / (exp(x) - 1) (exponential fitting of advection and
// migration against diffusion), u_f the mean of the two cell velocities,
// phi = psi / V_T (kept to FP64 accuracy; the face difference is rounded to
// the storage precision only after subtraction).  The inlet ghost holds
// C = c0, phi = 0, u = u_P; the outlet ghost copies the cell (zero gradient).
// Update: C_P -= (dt/dx) sum_f J.  Fields are stored by pore rank (see
// NPGeo).  Adsorbed / inflow / outflow fluxes are summed per warp into
// per-warp accounts (FP64, or FP32 pairs in FP32 storage; a fixed warp ->
// cells map, so the totals are deterministic).
#include <algorithm>
#include <cmath>
#include <type_traits>

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
  T c0lo;               // its low word (c0 - (T)c0) for pair storage
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

// Pore rank of the pore lattice cell (x, row): the rank of the first pore
// cell of its 32-cell word plus the pore cells before it in that word.
__device__ __forceinline__ int rank_of(const uint2 *__restrict__ words, int W, int row, int x) {
  const uint2 t = __ldg(words + (size_t)row * W + (x >> 5));
  return (int)t.x + __popc(t.y & ((1u << (x & 31)) - 1u));
}

// Row of the lateral (y: a = 1, z: a = 2) neighbour across face fc; rows wrap
// periodically (a wall face is never asked).  row = z * ny + y.
__device__ __forceinline__ int lateral_row(unsigned f, int fc, int row, int ny, int nz) {
  const int s = (fc & 1) ? -1 : 1;
  const bool edge = (f >> (kEdgeBit + fc)) & 1u;
  const int step = (fc >> 1) == 1 ? 1 : ny;
  const int ext = (fc >> 1) == 1 ? ny : nz;
  return row + (edge ? -s * (ext - 1) * step : s * step);
}

// Face flux divided by D/dx, J' = B(-P) C_P - B(P) C_nb, for the face Peclet
// number P = adv - z (phi_nb - phi_P); dd is phi_nb - phi_P.
__device__ __forceinline__ double face_flux(double adv, double z, double dd, double, double,
                                            double CP, double Cn) {
  double Bp, Bm;
  bernoulli_pair(r_fma(-z, dd, adv), Bp, Bm);
  return r_fma(Bm, CP, -r_mul(Bp, Cn));
}

// FP32: phi and P are carried as unevaluated pairs (hi + lo) where it
// matters: an exponent |P| rounded to FP32 costs a relative error of about
// |P| * 6e-8 in each Boltzmann factor exp(P), which accumulates across an
// electric double layer.
//  * |P| < 1/2 (almost every face): with the even function
//      E(P) = B(P) + P/2 = (P/2) coth(P/2) = 1 + P^2/12 - P^4/720 + P^6/30240 - ...
//    (Bernoulli numbers; the next term is below 3.3e-9 here),
//      J' = E (C_P - C_nb) + (P/2) (C_P + C_nb),
//    a sum of two small, accurately rounded terms.
//  * otherwise: B at the high part of |P| from expm1, corrected to first
//    order in the low part with B'(x) = B(x) ((1 - B(x)) / x - 1), and
//    B(-a) = B(a) + a; J' = B(-P) C_P - B(P) C_nb, each product accurate.
__device__ __noinline__ void bernoulli_pair_split(float adv, float z, float2 nb, float2 pp,
                                                  float &Bp, float &Bm) {
  // phi_nb - phi_P as dhi + dlo (two-sum of the high parts plus the lows)
  const float d = __fsub_rn(nb.x, pp.x);
  const float bv = __fsub_rn(d, nb.x);
  const float e = __fadd_rn(__fsub_rn(nb.x, __fsub_rn(d, bv)), __fsub_rn(-pp.x, bv));
  const float dhi = d, dlo = __fadd_rn(e, __fsub_rn(nb.y, pp.y));
  // P = adv - z (dhi + dlo) as ph + pl
  const float zd = __fmul_rn(z, dhi);
  const float zde = __fmaf_rn(z, dhi, -zd);
  const float ph = __fsub_rn(adv, zd);
  const float bb = __fsub_rn(ph, adv);
  const float phe = __fadd_rn(__fsub_rn(adv, __fsub_rn(ph, bb)), __fsub_rn(-zd, bb));
  const float pl = __fsub_rn(__fsub_rn(phe, zde), __fmul_rn(z, dlo));
  const bool neg = ph < 0.f;
  const float ah = neg ? -ph : ph, al = neg ? -pl : pl;
  // B(a) = a e^-a / (1 - e^-a) is below 1e-33 beyond a = 80
  float Ba = ah > 80.f ? 0.f : __fdividef(ah, expm1f(ah));
  Ba = __fmaf_rn(__fmul_rn(Ba, al), __fsub_rn(__fdividef(__fsub_rn(1.f, Ba), ah), 1.f), Ba);
  const float Bma = __fadd_rn(__fadd_rn(Ba, ah), al);
  Bp = neg ? Bma : Ba;
  Bm = neg ? Ba : Bma;
}

__device__ __forceinline__ float face_flux(float adv, float z, float dd, float2 nb, float2 pp,
                                           float CP, float Cn) {
  const float p = __fmaf_rn(-z, dd, adv);
  if (fabsf(p) < 0.5f) {
    const float p2 = __fmul_rn(p, p);
    float E = __fmaf_rn(p2, 1.f / 30240.f, -1.f / 720.f);
    E = __fmaf_rn(E, p2, 1.f / 12.f);
    E = __fmaf_rn(E, p2, 1.f);
    return __fmaf_rn(E, __fsub_rn(CP, Cn), __fmul_rn(__fmul_rn(0.5f, p), __fadd_rn(CP, Cn)));
  }
  float Bp, Bm;
  bernoulli_pair_split(adv, z, nb, pp, Bp, Bm);
  return r_fma(Bm, CP, -r_mul(Bp, Cn));
}

__device__ __forceinline__ double phi_diff(double nb, double pp) { return __dsub_rn(nb, pp); }
__device__ __forceinline__ float phi_diff(float2 nb, float2 pp) {
  return __fadd_rn(__fsub_rn(nb.x, pp.x), __fsub_rn(nb.y, pp.y));
}

// Geometry of the compact transport layout handed to the step kernels.
struct NPGeo {
  const uint2 *meta;   // per rank {flags | x << 16, row}
  const NFlag *fl;     // per rank: its face flags alone (what the step reads)
  const uint2 *words;  // per 32 cells of a row {first rank, pore bits}
  const int *lat;      // per lateral face f (y+, y-, z+, z-) and rank r, at
                       // (f - 2) * n + r: the pore neighbour's rank, or -1
  int n, W, ny, nz, walls;
  int naccs;           // account sets (one per warp), the same for any launch shape
};

// FP32 storage: warps of 31 home cells.  Warp w holds ranks 31 w - 1 ..
// 31 w + 30 in lanes 0..31; lane 0 (the last home cell of warp w - 1) is a
// halo.  Each lane evaluates the flux through the +x face of its cell; when
// the -x neighbour of a cell is a pore cell it is the rank before it, i.e.
// the lane before it, so that face's flux is the previous lane's +x flux
// with its sign flipped (one shuffle).  Every x face is then evaluated once
// instead of twice, and every lane of the warp takes the same path.
constexpr int kHome = 31;

// The fields of one FP32 transport state as per-species / per-component
// plane pointers: by value as kernel parameters (one launch, one state) or
// in a member table (fused sweeps and batches), so that every access is a
// base pointer plus a 32-bit rank.
struct NPFields {
  const float *C[kMaxSpecies];   // concentrations read (hi words)
  const float *Cl[kMaxSpecies];  // their low words (pair storage), else null
  float *Co[kMaxSpecies];        // concentrations written
  float *Col[kMaxSpecies];       // their low words
  const float *u[3];             // velocity components
  const int *lat[4];             // lateral neighbour ranks (y+, y-, z+, z-)
  const float2 *phi;             // psi / V_T as (hi, lo)
  const NFlag *fl;               // face flags
  float2 *acc;                   // per-warp accounts
};
__host__ __device__ constexpr long long np_warps(long long n) { return (n + kHome - 1) / kHome; }

// One explicit step of the pore cell of rank r for NS species: writes the
// new concentrations and adds the cell's adsorbed (v[k]), inflow (v[NS+k])
// and outflow (v[2NS+k]) fluxes.  Returns whether the cell has an inlet or
// outlet face.
//
// A face that does not lead to a pore cell reads the cell's own values: the
// outlet ghost copies the cell (J = u_x C_P), the inlet ghost then takes
// C = c0 and phi = 0, and a solid or wall face gets u_f = 0, for which the
// flux expression is exactly 0 (C_nb = C_P, dphi = 0); the adsorption flux of
// the n_s solid faces, n_s K_eff C_P, is added once per cell.
template <typename T, int DIM, int NS>
__device__ __forceinline__ bool np_cell(const T *__restrict__ Cin, T *__restrict__ Cout,
                                        const T *__restrict__ u,
                                        const typename PhiStore<T>::type *__restrict__ phi,
                                        const NPGeo &g, uint2 meta, int r, const NPConst<T> &c,
                                        T (&v)[3 * NS]) {
  using PT = typename PhiStore<T>::type;
  constexpr int NF = 2 * DIM;
  const unsigned f = meta.x & 0xffffu;
  const size_t n = (size_t)g.n;
  // neighbour ranks first (x neighbours are the adjacent ranks, lateral ones
  // come from the table)
  int Q[NF];
  bool open[NF];
#pragma unroll
  for (int fc = 0; fc < NF; fc++) {
    const bool solid = (f >> (kFaceBit + fc)) & 1u;
    const bool edge = (f >> (kEdgeBit + fc)) & 1u;
    if (fc < 2) {
      open[fc] = !solid;
      Q[fc] = (solid || edge) ? r : r + ((fc & 1) ? -1 : 1);
    } else {
      // the lateral neighbour's rank, found once at set-up from the row words
      const int q = g.lat[(size_t)(fc - 2) * n + r];
      open[fc] = q >= 0;
      Q[fc] = q >= 0 ? q : r;
    }
  }
  // every load before any arithmetic (memory-level parallelism)
  T CP[NS], Cn[NF][NS], uP[DIM], un[NF];
  PT phn[NF];
#pragma unroll
  for (int k = 0; k < NS; k++) CP[k] = Cin[k * n + r];
#pragma unroll
  for (int a = 0; a < DIM; a++) uP[a] = u[a * n + r];
  const PT phP = phi[r];
#pragma unroll
  for (int fc = 0; fc < NF; fc++) {
    un[fc] = u[(fc >> 1) * n + Q[fc]];
    phn[fc] = phi[Q[fc]];
#pragma unroll
    for (int k = 0; k < NS; k++) Cn[fc][k] = Cin[k * n + Q[fc]];
  }
  // the feed ghost across the inlet face (face 1 at x = 0)
  const bool inlet = (f >> (kEdgeBit + 1)) & 1u, outlet = (f >> kEdgeBit) & 1u;
  if (inlet) {
    phn[1] = PhiStore<T>::zero();
#pragma unroll
    for (int k = 0; k < NS; k++) Cn[1][k] = c.c0;
  }
  // adsorption on the solid faces (Eq. 6)
  const T ns_solid = (T)__popc(f & (((1u << NF) - 1u) << kFaceBit));
  T sumJ[NS];
#pragma unroll
  for (int k = 0; k < NS; k++) {
    const T Ja = r_mul(r_mul(ns_solid, c.Keff[k]), CP[k]);
    sumJ[k] = Ja;
    v[k] = r_add(v[k], Ja);
  }
#pragma unroll
  for (int fc = 0; fc < NF; fc++) {
    const T half = (fc & 1) ? T(-0.5) : T(0.5);
    const T uf = open[fc] ? r_mul(half, r_add(uP[fc >> 1], un[fc])) : T(0);
    const T dd = phi_diff(phn[fc], phP);
#pragma unroll
    for (int k = 0; k < NS; k++) {
      const T J = r_mul(c.Ddx[k], face_flux(r_mul(uf, c.dxD[k]), c.zf[k], dd, phn[fc], phP,
                                            CP[k], Cn[fc][k]));
      sumJ[k] = r_add(sumJ[k], J);
      if (fc == 1 && inlet) v[NS + k] = r_sub(v[NS + k], J);
      if (fc == 0 && outlet) v[2 * NS + k] = r_add(v[2 * NS + k], J);
    }
  }
#pragma unroll
  for (int k = 0; k < NS; k++) Cout[k * n + r] = r_fma(-c.dtdx, sumJ[k], CP[k]);
  return inlet || outlet;
}

// Per-warp account slot: FP64 for FP64 storage; for FP32 storage an
// unevaluated pair of FP32 words (hi + lo, about 48 significant bits) kept
// with the two-sum transformation, so the step issues no FP64 instruction
// (this part's FP64 rate is a small fraction of its FP32 rate).  Both are
// 8 bytes.
template <typename T> struct AccSlot { using type = double; };
template <> struct AccSlot<float> { using type = float2; };

__device__ __forceinline__ void acc_add(double *a, double v) { *a = __dadd_rn(*a, v); }
__device__ __forceinline__ void acc_add(float2 *a, float v) {
  float2 t = *a;
  const float s = __fadd_rn(t.x, v);
  const float bp = __fsub_rn(s, t.x);
  const float e = __fadd_rn(__fsub_rn(t.x, __fsub_rn(s, bp)), __fsub_rn(v, bp));
  t.x = s;
  t.y = __fadd_rn(t.y, e);
  *a = t;
}
__device__ __forceinline__ double acc_value(double a) { return a; }
__device__ __forceinline__ double acc_value(float2 a) { return (double)a.x + (double)a.y; }

// Warp sums of v in T, added by lane 0 to the warp's own accounts
// acc[(3*k + kind) * nw + wid], kind 0 Gamma, 1 In, 2 Out (one thread per
// pore cell, so the warp -> cells map is fixed and the totals are
// deterministic).  A warp without inlet or outlet cells skips the In/Out sums
// (its values are 0).  No block barrier: each warp retires on its own.  All
// 32 lanes of the warp must call it.
template <typename T, int NS>
__device__ __forceinline__ void np_account(T (&v)[3 * NS], bool io,
                                           typename AccSlot<T>::type *__restrict__ acc,
                                           int wid, int nw) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < NS; k++) v[k] = r_add(v[k], __shfl_down_sync(0xffffffffu, v[k], o));
  const bool any_io = __any_sync(0xffffffffu, io);
  if (any_io) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = NS; k < 3 * NS; k++)
        v[k] = r_add(v[k], __shfl_down_sync(0xffffffffu, v[k], o));
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < NS; k++) {
      typename AccSlot<T>::type *a = acc + (size_t)(3 * k) * nw + wid;
      acc_add(a, v[k]);
      if (any_io) {
        acc_add(a + nw, v[NS + k]);
        acc_add(a + 2 * (size_t)nw, v[2 * NS + k]);
      }
    }
  }
}

// (t.x + t.y) + v as a renormalised FP32 pair (two-sum): acc_add without the
// memory access.
__device__ __forceinline__ float2 pair_add(float2 t, float v) {
  const float s = __fadd_rn(t.x, v);
  const float bp = __fsub_rn(s, t.x);
  const float e = __fadd_rn(__fsub_rn(t.x, __fsub_rn(s, bp)), __fsub_rn(v, bp));
  return make_float2(s, __fadd_rn(t.y, e));
}

// The FP32 warp accounts of np_account, with the warp's adsorption slots
// read ahead by lane 0 (np_account_read): a slot belongs to one warp tile, so
// reading it before the tile's arithmetic gives the value acc_add would read
// after it, and its latency no longer ends every tile.  (The inflow and
// outflow slots, touched by the few warps at the inlet and outlet, are read
// at the end as before.)  The same sums and the same bits as np_account.
template <int NS>
__device__ __forceinline__ void np_account_read(float2 (&a)[NS], const float2 *acc, int wid,
                                                int nw) {
  if ((threadIdx.x & 31) != 0) return;
#pragma unroll
  for (int k = 0; k < NS; k++) a[k] = acc[(size_t)(3 * k) * nw + wid];
}
template <int NS>
__device__ __forceinline__ void np_account_f32(float (&v)[3 * NS], bool io,
                                               const float2 (&a)[NS], float2 *acc, int wid,
                                               int nw) {
  const bool any_io = __any_sync(0xffffffffu, io);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < NS; k++) v[k] = r_add(v[k], __shfl_down_sync(0xffffffffu, v[k], o));
  if (any_io) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = NS; k < 3 * NS; k++)
        v[k] = r_add(v[k], __shfl_down_sync(0xffffffffu, v[k], o));
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < NS; k++) {
      float2 *p = acc + (size_t)(3 * k) * nw + wid;
      p[0] = pair_add(a[k], v[k]);
      if (any_io) {
        acc_add(p + nw, v[NS + k]);
        acc_add(p + 2 * (size_t)nw, v[2 * NS + k]);
      }
    }
  }
}

// Two species per packed FP32x2 operation (each component rounded exactly as
// the scalar operation would be).
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 pneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __fadd2_rn(a, pneg(b)); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Flux through one face for a pair of species (k0, k1): the same arithmetic,
// species by species, as face_flux followed by the D/dx factor.  An odd
// species count pads its last pair with a copy of the last species (k1 = k0).
// Scalar flux of one species with pair-stored concentrations C + Cl: the
// difference C_P - C_nb and the two Bernoulli products take the low words
// along; everything else is face_flux.
__device__ __forceinline__ float face_flux_lo(float adv, float z, float dd, float2 nb, float2 pp,
                                              float CP, float Cn, float CPl, float Cnl) {
  const float p = __fmaf_rn(-z, dd, adv);
  if (fabsf(p) < 0.5f) {
    const float p2 = __fmul_rn(p, p);
    float E = __fmaf_rn(p2, 1.f / 30240.f, -1.f / 720.f);
    E = __fmaf_rn(E, p2, 1.f / 12.f);
    E = __fmaf_rn(E, p2, 1.f);
    const float dC = __fadd_rn(__fsub_rn(CP, Cn), __fsub_rn(CPl, Cnl));
    return __fmaf_rn(E, dC, __fmul_rn(__fmul_rn(0.5f, p), __fadd_rn(CP, Cn)));
  }
  float Bp, Bm;
  bernoulli_pair_split(adv, z, nb, pp, Bp, Bm);
  return __fadd_rn(r_fma(Bm, CP, -r_mul(Bp, Cn)), r_fma(Bm, CPl, -r_mul(Bp, Cnl)));
}

// Flux through one face for a pair of species (k0, k1): the same arithmetic,
// species by species, as face_flux (face_flux_lo with PAIR) followed by the
// D/dx factor.  An odd species count pads its last pair with a copy of the
// last species (k1 = k0).
template <bool PAIR>
__device__ __forceinline__ float2 face_flux_pair(float uf, float dd, float2 phn, float2 phP,
                                                 float2 CP, float2 Cn, float2 CPl, float2 Cnl,
                                                 const NPConst<float> &c, int k0, int k1) {
  const float2 adv = pmul(bc(uf), make_float2(c.dxD[k0], c.dxD[k1]));
  const float2 p = pfma(make_float2(-c.zf[k0], -c.zf[k1]), bc(dd), adv);
  float2 J;
  if (fabsf(p.x) < 0.5f && fabsf(p.y) < 0.5f) {
    const float2 p2 = pmul(p, p);
    float2 E = pfma(p2, bc(1.f / 30240.f), bc(-1.f / 720.f));
    E = pfma(E, p2, bc(1.f / 12.f));
    E = pfma(E, p2, bc(1.f));
    float2 dC = psub(CP, Cn);
    if (PAIR) dC = padd(dC, psub(CPl, Cnl));
    J = pfma(E, dC, pmul(pmul(bc(0.5f), p), padd(CP, Cn)));
  } else if (PAIR) {
    J.x = face_flux_lo(adv.x, c.zf[k0], dd, phn, phP, CP.x, Cn.x, CPl.x, Cnl.x);
    J.y = face_flux_lo(adv.y, c.zf[k1], dd, phn, phP, CP.y, Cn.y, CPl.y, Cnl.y);
  } else {
    J.x = face_flux(adv.x, c.zf[k0], dd, phn, phP, CP.x, Cn.x);
    J.y = face_flux(adv.y, c.zf[k1], dd, phn, phP, CP.y, Cn.y);
  }
  return pmul(make_float2(c.Ddx[k0], c.Ddx[k1]), J);
}

// (s, e) with s + e = a + b exactly (two-sum, component-wise).
__device__ __forceinline__ void ptwo_sum(float2 a, float2 b, float2 &s, float2 &e) {
  s = padd(a, b);
  const float2 bp = psub(s, a);
  e = padd(psub(a, psub(s, bp)), psub(b, bp));
}

// One explicit step of the home cells of warp w (FP32, NS species in
// (NS + 1) / 2 packed pairs), with the per-warp accounts of Gamma, In and
// Out.  PAIR: every concentration is an unevaluated pair hi + lo (the low
// words in Cinl/Coutl), updated with the two-sum transformation, so rounding
// does not build up over long runs; the fluxes take the low words into the
// concentration differences.  All 32 lanes of the warp must call it.  Per
// home cell the faces are summed in the order of np_cell (adsorption, +x,
// -x, +y, -y, +z, -z), so without PAIR a cell whose faces all take the
// |P| < 1/2 branch gets the bits np_cell gives.
// The per-lane link data of warp w's tile: the lane's face flags and its
// lateral neighbour ranks (-1 across a solid face or wall, or for the halo
// lane).
template <int DIM> struct NPLinks {
  unsigned f;
  int q[2 * DIM - 2];
};
template <int DIM>
__device__ __forceinline__ NPLinks<DIM> np_links(const NPFields &F, int n_cells, int w) {
  const int lane = threadIdx.x & 31;
  const int r = kHome * w + lane - 1;
  const bool valid = r >= 0 && r < n_cells;
  const bool home = valid && lane != 0;
  NPLinks<DIM> L;
  L.f = valid ? (unsigned)F.fl[r] : 0u;
#pragma unroll
  for (int j = 0; j < 2 * DIM - 2; j++) L.q[j] = home ? F.lat[j][r] : -1;
  return L;
}

template <int DIM, int NS, bool PAIR>
__device__ __forceinline__ void np_warp31(const NPFields &F, int n_cells, int naccs,
                                          const NPConst<float> &c, int w) {
  np_warp31<DIM, NS, PAIR>(F, n_cells, naccs, c, w, np_links<DIM>(F, n_cells, w));
}

// The values one lane of a warp tile works from: its cell's own fields, its
// lateral neighbours' (the cell's own values across a closed face) and its +x
// neighbour's (replaced by the cell's own unless that face is open and inside
// the image).
template <int DIM, int NS> struct NPLane {
  static constexpr int NP = (NS + 1) / 2, NL = 2 * DIM - 2;
  float2 CP[NP], CPl[NP], phP;
  float uP[DIM];
  float2 Cl[NL][NP], Cll[NL][NP], phl[NL];
  float ul[NL];
  float2 Cx[NP], Cxl[NP], phx;
  float ux;
};

// Second species of pair p (a copy of the first when NS is odd).
template <int NS> __device__ __forceinline__ constexpr int np_k1(int p) {
  return 2 * p + 1 < NS ? 2 * p + 1 : 2 * p;
}

// Lateral neighbours' values, read from the field arrays (own values are
// already in V).
template <int DIM, int NS, bool PAIR>
__device__ __forceinline__ void np_load_lateral(const NPFields &F, const int *q,
                                                NPLane<DIM, NS> &V) {
  constexpr int NP = (NS + 1) / 2;
#pragma unroll
  for (int j = 0; j < 2 * DIM - 2; j++) {
    const int fc = j + 2;
    if (q[j] >= 0) {
      const int Q = q[j];
      V.ul[j] = F.u[fc >> 1][Q];
      V.phl[j] = F.phi[Q];
#pragma unroll
      for (int p = 0; p < NP; p++) {
        V.Cl[j][p] = make_float2(F.C[2 * p][Q], F.C[np_k1<NS>(p)][Q]);
        V.Cll[j][p] = PAIR ? make_float2(F.Cl[2 * p][Q], F.Cl[np_k1<NS>(p)][Q])
                           : make_float2(0.f, 0.f);
      }
    } else {
      V.ul[j] = V.uP[fc >> 1];
      V.phl[j] = V.phP;
#pragma unroll
      for (int p = 0; p < NP; p++) {
        V.Cl[j][p] = V.CP[p];
        V.Cll[j][p] = V.CPl[p];
      }
    }
  }
}

// Own, lateral and +x values of warp w's tile, read from the field arrays:
// the +x neighbour is the next lane's cell (np_finish_x, a shuffle), or for
// lane 31 the next tile's first home cell (loaded here).
template <int DIM, int NS, bool PAIR>
__device__ __forceinline__ void np_issue_loads(const NPFields &F, int n_cells, int w,
                                               unsigned f, const int *q, NPLane<DIM, NS> &V) {
  constexpr int NP = (NS + 1) / 2;
  const int lane = threadIdx.x & 31;
  const int r = kHome * w + lane - 1;
  const bool valid = r >= 0 && r < n_cells;
  auto ldC = [&](const float *const *A, int Q, int p) {
    return make_float2(A[2 * p][Q], A[np_k1<NS>(p)][Q]);
  };
  const float2 z2 = make_float2(0.f, 0.f);
#pragma unroll
  for (int p = 0; p < NP; p++) V.CP[p] = V.CPl[p] = z2;
#pragma unroll
  for (int a = 0; a < DIM; a++) V.uP[a] = 0.f;
  V.phP = z2;
  if (valid) {
#pragma unroll
    for (int p = 0; p < NP; p++) {
      V.CP[p] = ldC(F.C, r, p);
      if (PAIR) V.CPl[p] = ldC(F.Cl, r, p);
    }
#pragma unroll
    for (int a = 0; a < DIM; a++) V.uP[a] = F.u[a][r];
    V.phP = F.phi[r];
  }
  np_load_lateral<DIM, NS, PAIR>(F, q, V);
  const bool xp = valid && !((f >> kFaceBit) & 1u) && !((f >> kEdgeBit) & 1u);
  V.ux = 0.f;
  V.phx = z2;
#pragma unroll
  for (int p = 0; p < NP; p++) V.Cx[p] = V.Cxl[p] = z2;
  if (lane == 31 && xp) {  // rank r + 1 is the next warp's first home cell
    V.ux = F.u[0][r + 1];
    V.phx = F.phi[r + 1];
#pragma unroll
    for (int p = 0; p < NP; p++) {
      V.Cx[p] = ldC(F.C, r + 1, p);
      if (PAIR) V.Cxl[p] = ldC(F.Cl, r + 1, p);
    }
  }
}

// The +x neighbour's values of lanes 0-30: the next lane's own values.
template <int DIM, int NS, bool PAIR>
__device__ __forceinline__ void np_finish_x(NPLane<DIM, NS> &V) {
  constexpr int NP = (NS + 1) / 2;
  const bool take = (threadIdx.x & 31) != 31;
  auto sh = [&](float v, float &dst) {
    const float t = __shfl_down_sync(0xffffffffu, v, 1);
    if (take) dst = t;
  };
  sh(V.uP[0], V.ux);
  sh(V.phP.x, V.phx.x);
  sh(V.phP.y, V.phx.y);
#pragma unroll
  for (int p = 0; p < NP; p++) {
    sh(V.CP[p].x, V.Cx[p].x);
    sh(V.CP[p].y, V.Cx[p].y);
    if (PAIR) {
      sh(V.CPl[p].x, V.Cxl[p].x);
      sh(V.CPl[p].y, V.Cxl[p].y);
    }
  }
}

template <int DIM, int NS, bool PAIR>
__device__ __forceinline__ void np_load_global(const NPFields &F, int n_cells, int w,
                                               unsigned f, const int *q, NPLane<DIM, NS> &V) {
  np_issue_loads<DIM, NS, PAIR>(F, n_cells, w, f, q, V);
  np_finish_x<DIM, NS, PAIR>(V);
}

// The update of warp w's tile from the values in V: the +x face flux is
// evaluated once per face and handed to the next lane as its -x flux; then
// adsorption, the x faces and the lateral faces are summed in that order and
// the new concentrations and the warp's accounts written.
template <int DIM, int NS, bool PAIR>
__device__ __forceinline__ void np_tile_update(const NPFields &F, int n_cells, int naccs,
                                               const NPConst<float> &c, int w, unsigned f,
                                               const int *q, NPLane<DIM, NS> &V) {
  constexpr int NF = 2 * DIM;
  constexpr int NP = (NS + 1) / 2;
  const int lane = threadIdx.x & 31;
  const int r = kHome * w + lane - 1;
  const bool valid = r >= 0 && r < n_cells;
  const bool home = valid && lane != 0;
  const float2 z2 = make_float2(0.f, 0.f);
  // the warp's adsorption account slots, read before the arithmetic
  float2 acc_pre[NS];
  np_account_read<NS>(acc_pre, F.acc, w, naccs);
  // +x face: open and inside the image, else the outlet ghost copies the cell
  const bool xs = (f >> kFaceBit) & 1u, xe = (f >> kEdgeBit) & 1u;
  const bool xp = valid && !xs && !xe;
  if (!xp) {
    V.ux = V.uP[0];
    V.phx = V.phP;
#pragma unroll
    for (int p = 0; p < NP; p++) {
      V.Cx[p] = V.CP[p];
      V.Cxl[p] = V.CPl[p];
    }
  }
  float2 Jx[NP];
  {
    const float uf = (valid && !xs) ? r_mul(0.5f, r_add(V.uP[0], V.ux)) : 0.f;
    const float dd = phi_diff(V.phx, V.phP);
#pragma unroll
    for (int p = 0; p < NP; p++)
      Jx[p] = face_flux_pair<PAIR>(uf, dd, V.phx, V.phP, V.CP[p], V.Cx[p], V.CPl[p], V.Cxl[p], c,
                                   2 * p, np_k1<NS>(p));
  }
  // -x face: the previous lane's +x face (pore neighbour), the feed ghost
  // (inlet), or closed (solid)
  const bool ms = (f >> (kFaceBit + 1)) & 1u, me = (f >> (kEdgeBit + 1)) & 1u;
  float2 Jm[NP];
#pragma unroll
  for (int p = 0; p < NP; p++) {
    Jm[p].x = -__shfl_up_sync(0xffffffffu, Jx[p].x, 1);
    Jm[p].y = -__shfl_up_sync(0xffffffffu, Jx[p].y, 1);
    if (ms) Jm[p] = z2;
  }
  if (home && me) {
    const float uf = r_mul(-0.5f, r_add(V.uP[0], V.uP[0]));
    const float dd = phi_diff(z2, V.phP);
#pragma unroll
    for (int p = 0; p < NP; p++)
      Jm[p] = face_flux_pair<PAIR>(uf, dd, z2, V.phP, V.CP[p], bc(c.c0), V.CPl[p], bc(c.c0lo), c,
                                   2 * p, np_k1<NS>(p));
  }
  // adsorption on the solid faces (Eq. 6), then the faces in order
  float v[3 * NS];
#pragma unroll
  for (int j = 0; j < 3 * NS; j++) v[j] = 0.f;
  const float ns_solid = (float)__popc(f & (((1u << NF) - 1u) << kFaceBit));
  float2 sumJ[NP];
#pragma unroll
  for (int p = 0; p < NP; p++) {
    const float2 Ja =
        pmul(pmul(bc(ns_solid), make_float2(c.Keff[2 * p], c.Keff[np_k1<NS>(p)])), V.CP[p]);
    sumJ[p] = padd(padd(Ja, Jx[p]), Jm[p]);
    if (home) {
      v[2 * p] = r_add(0.f, Ja.x);
      if (2 * p + 1 < NS) v[2 * p + 1] = r_add(0.f, Ja.y);
      if (me) {
        v[NS + 2 * p] = r_sub(0.f, Jm[p].x);
        if (2 * p + 1 < NS) v[NS + 2 * p + 1] = r_sub(0.f, Jm[p].y);
      }
      if (xe) {
        v[2 * NS + 2 * p] = r_add(0.f, Jx[p].x);
        if (2 * p + 1 < NS) v[2 * NS + 2 * p + 1] = r_add(0.f, Jx[p].y);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NF - 2; j++) {
    const int fc = j + 2;
    const float half = (fc & 1) ? -0.5f : 0.5f;
    const float uf = q[j] >= 0 ? r_mul(half, r_add(V.uP[fc >> 1], V.ul[j])) : 0.f;
    const float dd = phi_diff(V.phl[j], V.phP);
#pragma unroll
    for (int p = 0; p < NP; p++)
      sumJ[p] = padd(sumJ[p], face_flux_pair<PAIR>(uf, dd, V.phl[j], V.phP, V.CP[p], V.Cl[j][p],
                                                   V.CPl[p], V.Cll[j][p], c, 2 * p,
                                                   np_k1<NS>(p)));
  }
  if (home) {
#pragma unroll
    for (int p = 0; p < NP; p++) {
      float2 Cn, Cnl;
      if (PAIR) {
        // (hi + lo) - dt/dx sum J by two-sum, renormalised
        float2 t, e;
        ptwo_sum(V.CP[p], pmul(bc(-c.dtdx), sumJ[p]), t, e);
        const float2 l = padd(V.CPl[p], e);
        Cn = padd(t, l);
        Cnl = psub(l, psub(Cn, t));
        F.Col[2 * p][r] = Cnl.x;
        if (2 * p + 1 < NS) F.Col[2 * p + 1][r] = Cnl.y;
      } else {
        Cn = pfma(bc(-c.dtdx), sumJ[p], V.CP[p]);
      }
      F.Co[2 * p][r] = Cn.x;
      if (2 * p + 1 < NS) F.Co[2 * p + 1][r] = Cn.y;
    }
  }
  np_account_f32<NS>(v, home && (me || xe), acc_pre, F.acc, w, naccs);
}

template <int DIM, int NS, bool PAIR>
__device__ __forceinline__ void np_warp31(const NPFields &F, int n_cells, int naccs,
                                          const NPConst<float> &c, int w,
                                          const NPLinks<DIM> &lk) {
  NPLane<DIM, NS> V;
  np_load_global<DIM, NS, PAIR>(F, n_cells, w, lk.f, lk.q, V);
  np_tile_update<DIM, NS, PAIR>(F, n_cells, naccs, c, w, lk.f, lk.q, V);
}

template <typename T, int DIM, int NS, bool PAIR>
__device__ __forceinline__ void np_step_body(const T *__restrict__ Cin, T *__restrict__ Cout,
                                             const float *__restrict__ Cinl,
                                             float *__restrict__ Coutl, const T *__restrict__ u,
                                             const typename PhiStore<T>::type *__restrict__ phi,
                                             const NPGeo &g, const NPConst<T> &c,
                                             typename AccSlot<T>::type *__restrict__ acc) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  T v[3 * NS];
#pragma unroll
  for (int j = 0; j < 3 * NS; j++) v[j] = T(0);
  bool io = false;
  if (r < g.n) io = np_cell<T, DIM, NS>(Cin, Cout, u, phi, g, g.meta[r], r, c, v);
  np_account<T, NS>(v, io, acc, r >> 5, g.naccs);
}

// FP32 storage: warps of 31 home cells (np_warp31), fields by plane pointer.
template <int DIM, int NS, int BS, bool PAIR>
__global__ void __launch_bounds__(BS)
    k_np_step32(NPFields F, int n, int naccs, NPConst<float> c) {
  np_warp31<DIM, NS, PAIR>(F, n, naccs, c, (blockIdx.x * BS + threadIdx.x) >> 5);
}

template <int DIM, int NS, int BS, int MINT, bool PAIR>
__global__ void __launch_bounds__(BS, MINT / BS)
    k_np_step32_occ(NPFields F, int n, int naccs, NPConst<float> c) {
  np_warp31<DIM, NS, PAIR>(F, n, naccs, c, (blockIdx.x * BS + threadIdx.x) >> 5);
}

// The same step with a resident grid: each warp walks tiles w, w + W, ...
// (W the warps of the launch) and loads the next tile's link data while it
// computes the current tile, so that load no longer adds a memory round trip
// ahead of the neighbour loads.  Tiles and accounts are those of the other
// launch shapes.  MINB > 0 caps the registers for MINB resident blocks per SM.
template <int DIM, int NS, int BS, int MINB, bool PAIR>
__global__ void __launch_bounds__(BS, MINB)
    k_np_step32_pf(NPFields F, int n, int naccs, NPConst<float> c) {
  const int nw = (int)np_warps(n);
  const int W = gridDim.x * (BS / 32);
  int w = (blockIdx.x * BS + threadIdx.x) >> 5;
  if (w >= nw) return;  // whole warps leave together
  NPLinks<DIM> cur = np_links<DIM>(F, n, w);
  while (true) {
    const int wn = w + W;
    NPLinks<DIM> nxt;
    if (wn < nw) nxt = np_links<DIM>(F, n, wn);
    np_warp31<DIM, NS, PAIR>(F, n, naccs, c, w, cur);
    if (wn >= nw) break;
    w = wn;
    cur = nxt;
  }
}

// Blocks that fill every SM with the kernel at block size bs (once per
// kernel; at most the blocks the work needs).
template <typename K> int resident_grid(K kernel, int bs, long long units) {
  static int blocks = 0;
  if (blocks == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, bs, 0);
    (void)cudaGetLastError();
    blocks = (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
  }
  return (int)std::max<long long>(1, std::min<long long>(blocks, (units + bs - 1) / bs));
}

// BS threads per block, registers as the compiler sees fit.
template <typename T, int DIM, int NS, int BS, bool PAIR>
__global__ void __launch_bounds__(BS)
    k_np_step(const T *__restrict__ Cin, T *__restrict__ Cout, const float *__restrict__ Cinl,
              float *__restrict__ Coutl, const T *__restrict__ u,
              const typename PhiStore<T>::type *__restrict__ phi, NPGeo g, NPConst<T> c,
              typename AccSlot<T>::type *__restrict__ acc) {
  np_step_body<T, DIM, NS, PAIR>(Cin, Cout, Cinl, Coutl, u, phi, g, c, acc);
}

// The same step with registers capped so that MINT threads share an SM (more
// resident warps for the gathered loads, at the price of a few spilled
// values).
template <typename T, int DIM, int NS, int BS, int MINT, bool PAIR>
__global__ void __launch_bounds__(BS, MINT / BS)
    k_np_step_occ(const T *__restrict__ Cin, T *__restrict__ Cout, const float *__restrict__ Cinl,
                  float *__restrict__ Coutl, const T *__restrict__ u,
                  const typename PhiStore<T>::type *__restrict__ phi, NPGeo g, NPConst<T> c,
                  typename AccSlot<T>::type *__restrict__ acc) {
  np_step_body<T, DIM, NS, PAIR>(Cin, Cout, Cinl, Coutl, u, phi, g, c, acc);
}

// One member of a fused sweep: its own concentrations, velocity, potential,
// constants (time step) and accounts.
template <typename T> struct SweepMember {
  T *C[2];          // concentration buffers (ping-pong)
  float *Cl[2];     // their low words (FP32 pair storage), else null
  NPFields f[2];    // FP32: the fields as plane pointers, stepping from buffer 0 / 1
  const T *u;
  const typename PhiStore<T>::type *phi;
  typename AccSlot<T>::type *acc;
  NPConst<T> c;
};

// All members of a sweep advance one step in one launch: each block runs the
// same cells for every member in turn (the block -> cells map, the arithmetic
// and the accounts of a member are those of k_np_step, so a member's result
// equals a single run's bit for bit).
template <typename T, int DIM, int NS, bool PAIR>
__global__ void __launch_bounds__(kRowBlock)
    k_np_sweep(const SweepMember<T> *__restrict__ members, int n_members, int in, NPGeo g) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (std::is_same<T, float>::value) {
    for (int m = 0; m < n_members; m++) {
      const SweepMember<T> &mb = members[m];
      np_warp31<DIM, NS, PAIR>(mb.f[in], g.n, g.naccs, mb.c, r >> 5);
    }
  } else {
    const uint2 meta = r < g.n ? g.meta[r] : make_uint2(1u, 0u);
    for (int m = 0; m < n_members; m++) {
      const SweepMember<T> &mb = members[m];
      T v[3 * NS];
#pragma unroll
      for (int j = 0; j < 3 * NS; j++) v[j] = T(0);
      bool io = false;
      if (r < g.n)
        io = np_cell<T, DIM, NS>(mb.C[in], mb.C[1 - in], mb.u, mb.phi, g, meta, r, mb.c, v);
      np_account<T, NS>(v, io, mb.acc, r >> 5, g.naccs);
    }
  }
}

// One member of a batch over several geometries: a sweep member plus its
// geometry; blocks [block0, block0 + nblocks) of the launch are its own.
template <typename T> struct BatchMember {
  SweepMember<T> s;
  NPGeo g;
  int block0, nblocks;
};

// All members of a batch over uneven geometries advance one step in one
// launch.  Block b of the launch belongs to the member whose block range
// holds it (binary search over the ascending block0), and runs that member's
// local block b - block0: the same cells, arithmetic and accounts as block
// b - block0 of the member's single-run launch, so each member equals its
// single run bit for bit.
template <typename T, int DIM, int NS, bool PAIR>
__global__ void __launch_bounds__(kRowBlock)
    k_np_batch(const BatchMember<T> *__restrict__ members, int n_members, int in) {
  int lo = 0, hi = n_members - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (members[mid].block0 <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const BatchMember<T> &mb = members[lo];
  const int b = (int)blockIdx.x - mb.block0;
  const int r = b * blockDim.x + threadIdx.x;
  if constexpr (std::is_same<T, float>::value) {
    np_warp31<DIM, NS, PAIR>(mb.s.f[in], mb.g.n, mb.g.naccs, mb.s.c, r >> 5);
  } else {
    T v[3 * NS];
#pragma unroll
    for (int j = 0; j < 3 * NS; j++) v[j] = T(0);
    bool io = false;
    if (r < mb.g.n)
      io = np_cell<T, DIM, NS>(mb.s.C[in], mb.s.C[1 - in], mb.s.u, mb.s.phi, mb.g, mb.g.meta[r],
                               r, mb.s.c, v);
    np_account<T, NS>(v, io, mb.s.acc, r >> 5, mb.g.naccs);
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
__global__ void k_np_init(T *__restrict__ C0, T *__restrict__ C1, float *__restrict__ L0,
                          float *__restrict__ L1, int n, int ns, T c0, float c0lo) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < kMaxSpecies; k++) {
      const T v = k < ns ? c0 : T(0);
      C0[(size_t)k * n + r] = v;
      C1[(size_t)k * n + r] = v;
      if (L0) {
        const float l = k < ns ? c0lo : 0.f;
        L0[(size_t)k * n + r] = l;
        L1[(size_t)k * n + r] = l;
      }
    }
  }
}

// Dissolved amount, outlet sums (flux weighted and plain) per species.
// Values: [0,4) mass, [4,8) sum u_x C at the outlet, 8 sum u_x, [9,13) plain
// sum of C at the outlet, 13 pore cells in the outlet column.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    k_np_sums(const uint2 *__restrict__ meta, const T *__restrict__ C,
              const float *__restrict__ Cl, const T *__restrict__ u, int n, int ns,
              double cell_vol, double *__restrict__ part, unsigned int *counter, double *scal) {
  constexpr int NV = 14;
  __shared__ double sm[NV * 32];
  double v[NV];
#pragma unroll
  for (int j = 0; j < NV; j++) v[j] = 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const bool outlet = (meta[r].x >> kEdgeBit) & 1u;
    const double ux = (double)u[r];
#pragma unroll
    for (int k = 0; k < kMaxSpecies; k++) {
      if (k >= ns) break;
      const double ck = (double)C[(size_t)k * n + r] + (Cl ? (double)Cl[(size_t)k * n + r] : 0.0);
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
// specific surface of Sec. 4 measures), counted over the pore ranks, and the
// sum of the x velocity over them (the numerator of Sec. 4's pore mean U).
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    k_geometry(const uint2 *__restrict__ meta, const T *__restrict__ ux, int n, int faces,
               double *__restrict__ part, unsigned int *counter, double *scal) {
  __shared__ double sm[3 * 32];
  double v[3] = {0.0, 0.0, 0.0};
  const unsigned face_bits = ((1u << faces) - 1u) << kFaceBit;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    v[0] += 1.0;
    v[1] += (double)__popc(meta[r].x & face_bits);
    v[2] += (double)ux[r];
  }
  block_reduce<3>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = v[0];
    part[gridDim.x + blockIdx.x] = v[1];
    part[2 * gridDim.x + blockIdx.x] = v[2];
  }
  if (last_block(counter, gridDim.x)) {
    combine_partials<3>(part, gridDim.x, v, sm, OpSum(), 0.0);
    if (threadIdx.x == 0) {
      scal[S_GEOM] = v[0];
      scal[S_GEOM + 1] = v[1];
      scal[S_GEOM + 2] = v[2];
      *counter = 0;
    }
  }
}

// Totals of the per-warp Gamma/In/Out accounts (one block, fixed order).
template <typename A>
__global__ void __launch_bounds__(kRedThreads)
    k_acc_total(const A *__restrict__ acc, int nw, double *scal) {
  constexpr int NV = 3 * kMaxSpecies;
  __shared__ double sm[NV * 32];
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) v[k] = 0.0;
  for (int b = threadIdx.x; b < nw; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] += acc_value(acc[(size_t)k * nw + b]);
  block_reduce<NV>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < NV; j++) scal[S_ACC + j] = v[j];
}

// Launches k_acc_total for the domain's precision.
void acc_total(const cdi_domain *d, const void *acc, cudaStream_t st, double *scal) {
  if (d->prec == CDI_FP64)
    k_acc_total<double><<<1, kRedThreads, 0, st>>>((const double *)acc, d->np_accs, scal);
  else
    k_acc_total<float2><<<1, kRedThreads, 0, st>>>((const float2 *)acc, d->np_accs, scal);
}

// Mean of species k over the pore cells of each x column (the column's
// cells found through the row words).
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    k_colmeans(const uint2 *__restrict__ words, int W, const T *__restrict__ C,
               const float *__restrict__ Cl, int rows, double *__restrict__ out) {
  __shared__ double sm[2 * 32];
  const int x = blockIdx.x;
  double v[2] = {0.0, 0.0};
  for (int row = threadIdx.x; row < rows; row += blockDim.x) {
    const uint2 t = words[(size_t)row * W + (x >> 5)];
    if (!((t.y >> (x & 31)) & 1u)) continue;
    const int r = t.x + __popc(t.y & ((1u << (x & 31)) - 1u));
    v[0] += (double)C[r] + (Cl ? (double)Cl[r] : 0.0);
    v[1] += 1.0;
  }
  block_reduce<2>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0) out[x] = v[1] > 0.0 ? v[0] / v[1] : 0.0;
}

// Per pore rank and lateral face (y+, y-, z+, z-): the rank of the pore
// neighbour across it (rows wrap periodically), or -1 across a solid face or
// a lateral wall.  The step kernels read it instead of the row words, which
// saves them a dependent load and the rank arithmetic.
__global__ void k_lat_nbr(const uint2 *__restrict__ meta, const uint2 *__restrict__ words,
                          int n, int W, int ny, int nz, int walls, int faces,
                          int *__restrict__ lat) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const uint2 m = meta[r];
    const unsigned f = m.x & 0xffffu;
    const int x = (int)(m.x >> 16), row = (int)m.y;
    for (int fc = 2; fc < faces; fc++) {
      const bool solid = (f >> (kFaceBit + fc)) & 1u;
      const bool wall = ((f >> (kEdgeBit + fc)) & 1u) && walls;
      lat[(size_t)(fc - 2) * n + r] =
          (solid || wall) ? -1 : rank_of(words, W, lateral_row(f, fc, row, ny, nz), x);
    }
  }
}

// Per pore rank: its face flags, x and row.
__global__ void k_cmeta(const NFlag *__restrict__ fl, const int *__restrict__ cells, int n,
                        int nx, uint2 *__restrict__ meta, NFlag *__restrict__ cfl) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int P = cells[r];
    const int row = P / nx, x = P - row * nx;
    meta[r] = make_uint2((unsigned)fl[P] | ((unsigned)x << 16), (unsigned)row);
    cfl[r] = fl[P];
  }
}

// Per 32 cells of a row: the pore bits and the rank of the first pore cell at
// or after the word's first cell (binary search of the ascending cell list).
__global__ void k_words(const NFlag *__restrict__ fl, const int *__restrict__ cells, int n,
                        int nx, int W, long long n_words, uint2 *__restrict__ words) {
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < n_words;
       w += (long long)gridDim.x * blockDim.x) {
    const long long row = w / W;
    const int x0 = (int)(w - row * W) * 32;
    const long long P0 = row * nx + x0;
    unsigned bits = 0;
    for (int b = 0; b < 32 && x0 + b < nx; b++)
      if (!(fl[P0 + b] & 1u)) bits |= 1u << b;
    int lo = 0, hi = n;  // first rank with cells[rank] >= P0
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((long long)cells[mid] < P0) lo = mid + 1;
      else hi = mid;
    }
    words[w] = make_uint2((unsigned)lo, bits);
  }
}

// Compact (rank-ordered) field -> FP64 lattice field, 0 in solid cells:
// dst[a * N + cells[r]] = src[a * n + r] for comps components.
template <typename T>
__global__ void k_scatter(const T *__restrict__ src, const float *__restrict__ lo, int comps,
                          const int *__restrict__ cells, int n, long long N,
                          double *__restrict__ dst) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const long long P = cells[r];
    for (int a = 0; a < comps; a++)
      dst[a * N + P] = (double)src[(size_t)a * n + r] + (lo ? (double)lo[(size_t)a * n + r] : 0.0);
  }
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
  c.c0lo = (T)(d->c0 - (double)c.c0);
  return c;
}

// The FP32 fields of a transport state as plane pointers (stepping from
// Cin/Cinl into Cout/Coutl).
NPFields fields32(const cdi_domain *d, const void *Cin, const float *Cinl, void *Cout,
                  float *Coutl, const void *u, const void *phi, void *acc) {
  NPFields F{};
  const size_t n = (size_t)d->n_pore;
  for (int k = 0; k < kMaxSpecies; k++) {
    F.C[k] = (const float *)Cin + (size_t)k * n;
    F.Cl[k] = Cinl ? Cinl + (size_t)k * n : nullptr;
    F.Co[k] = (float *)Cout + (size_t)k * n;
    F.Col[k] = Coutl ? Coutl + (size_t)k * n : nullptr;
  }
  for (int a = 0; a < d->dim; a++) F.u[a] = (const float *)u + (size_t)a * n;
  for (int j = 0; j < 2 * (d->dim - 1); j++) F.lat[j] = d->d_latnb + (size_t)j * n;
  F.phi = (const float2 *)phi;
  F.fl = d->d_cfl;
  F.acc = (float2 *)acc;
  return F;
}

NPGeo make_geo(const cdi_domain *d) {
  return NPGeo{d->d_cmeta, d->d_cfl, d->d_words, d->d_latnb, (int)d->n_pore, d->W, d->ny, d->nz,
               d->walls, d->np_accs};
}

template <typename T, int DIM, int NS, int BS, int MINT, bool PAIR>
void launch_step_bs(cdi_domain *d, cudaStream_t st, int in) {
  // FP64: one thread per pore rank; FP32: warps of 31 home cells (one
  // account set per warp either way)
  const long long units = std::is_same<T, float>::value ? np_warps(d->n_pore) * 32 : d->n_pore;
  const int grid = (int)((units + BS - 1) / BS);
  const float *Cinl = PAIR ? d->d_Clo[in] : nullptr;
  float *Coutl = PAIR ? d->d_Clo[1 - in] : nullptr;
  if constexpr (std::is_same<T, float>::value) {
    const NPFields F = fields32(d, d->d_C[in], Cinl, d->d_C[1 - in], Coutl, d->d_u, d->d_phi,
                                d->d_acc);
    if constexpr (MINT < 0) {
      // -1: registers as the compiler sees fit; -2: capped for 1024 threads
      // per SM; -3: for 768
      constexpr int MINB = MINT == -2 ? 1024 / BS : (MINT == -3 ? 768 / BS : 0);
      auto *kern = k_np_step32_pf<DIM, NS, BS, MINB, PAIR>;
      kern<<<resident_grid(kern, BS, units), BS, 0, st>>>(F, (int)d->n_pore, d->np_accs,
                                                          make_const<float>(d));
    } else if constexpr (MINT == 0)
      k_np_step32<DIM, NS, BS, PAIR><<<grid, BS, 0, st>>>(F, (int)d->n_pore, d->np_accs,
                                                          make_const<float>(d));
    else
      k_np_step32_occ<DIM, NS, BS, MINT, PAIR><<<grid, BS, 0, st>>>(F, (int)d->n_pore, d->np_accs,
                                                                    make_const<float>(d));
  } else if constexpr (MINT <= 0) {
    k_np_step<T, DIM, NS, BS, PAIR><<<grid, BS, 0, st>>>(
        (const T *)d->d_C[in], (T *)d->d_C[1 - in], Cinl, Coutl, (const T *)d->d_u,
        (const typename PhiStore<T>::type *)d->d_phi, make_geo(d), make_const<T>(d),
        (typename AccSlot<T>::type *)d->d_acc);
  } else {
    k_np_step_occ<T, DIM, NS, BS, MINT, PAIR><<<grid, BS, 0, st>>>(
        (const T *)d->d_C[in], (T *)d->d_C[1 - in], Cinl, Coutl, (const T *)d->d_u,
        (const typename PhiStore<T>::type *)d->d_phi, make_geo(d), make_const<T>(d),
        (typename AccSlot<T>::type *)d->d_acc);
  }
}

template <typename T, int DIM, int NS, bool PAIR>
void launch_step_t(cdi_domain *d, cudaStream_t st, int in) {
  switch (d->np_variant) {
    case 0: launch_step_bs<T, DIM, NS, 64, 0, PAIR>(d, st, in); break;
    case 2: launch_step_bs<T, DIM, NS, 256, 0, PAIR>(d, st, in); break;
    case 3: launch_step_bs<T, DIM, NS, 64, 1280, PAIR>(d, st, in); break;
    case 4: launch_step_bs<T, DIM, NS, 128, 1280, PAIR>(d, st, in); break;
    case 5: launch_step_bs<T, DIM, NS, 128, 1024, PAIR>(d, st, in); break;
    case 6: launch_step_bs<T, DIM, NS, 256, 1024, PAIR>(d, st, in); break;
    case 7: launch_step_bs<T, DIM, NS, 128, -1, PAIR>(d, st, in); break;
    case 8: launch_step_bs<T, DIM, NS, 128, -2, PAIR>(d, st, in); break;
    case 9: launch_step_bs<T, DIM, NS, 128, -3, PAIR>(d, st, in); break;
    default: launch_step_bs<T, DIM, NS, 128, 0, PAIR>(d, st, in); break;
  }
}

template <typename T, int DIM, bool PAIR>
void launch_step_d(cdi_domain *d, cudaStream_t st, int in) {
  switch (d->ns) {
    case 1: launch_step_t<T, DIM, 1, PAIR>(d, st, in); break;
    case 2: launch_step_t<T, DIM, 2, PAIR>(d, st, in); break;
    case 3: launch_step_t<T, DIM, 3, PAIR>(d, st, in); break;
    default: launch_step_t<T, DIM, 4, PAIR>(d, st, in); break;
  }
}

void launch_step(cdi_domain *d, cudaStream_t st, int in) {
  if (d->prec == CDI_FP64) {
    if (d->dim == 2) launch_step_d<double, 2, false>(d, st, in);
    else launch_step_d<double, 3, false>(d, st, in);
  } else if (d->cpair) {
    if (d->dim == 2) launch_step_d<float, 2, true>(d, st, in);
    else launch_step_d<float, 3, true>(d, st, in);
  } else {
    if (d->dim == 2) launch_step_d<float, 2, false>(d, st, in);
    else launch_step_d<float, 3, false>(d, st, in);
  }
}

constexpr int kGraphSteps = 64;  // steps per captured transport graph (even)

// Autotuner: times a few transport steps with each candidate launch shape
// (64, 128 or 256 threads per block; for 64 and 128 also a variant compiled
// for 1280 resident threads per SM, for 128 and 256 one for 1024, and FP32
// resident grids that prefetch each warp's next link data, with registers as
// the compiler sees fit or capped for 1024 or 768 threads per SM) on the
// domain's stream and keeps the fastest.  Accounts are kept per warp of 32 ranks whatever the shape, and
// the arithmetic of a thread does not depend on its register allocation, so
// every choice computes the same bits.  Runs once per domain, before
// cdi_np_init overwrites the concentrations and clears the accounts.
constexpr int kNpVariantBlock[10] = {64, 128, 256, 64, 128, 128, 256, 128, 128, 128};
cdi_status tune_np(cdi_domain *d) {
  // variants 7-9 (resident grids with prefetch) are FP32 launch shapes; for
  // FP64 they are plain launches of the same block size again
  static const int cand[] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9};
  const uint64_t key = cdi_tune_key(2, d->dim, d->prec, d->ns, d->n_pore, 0);
  int known = 0;
  if (cdi_tune_lookup(key, &known)) {
    d->np_variant = known;
    d->np_block = kNpVariantBlock[known];
    d->np_tuned = true;
    return CDI_OK;
  }
  cudaEvent_t a, b;
  CDI_TRY(d, cudaEventCreate(&a), "tune event");
  cudaError_t e = cudaEventCreate(&b);
  if (e != cudaSuccess) {
    cudaEventDestroy(a);
    return cdi_cuda_fail(d, e, "tune event");
  }
  float best = 0.f;
  int best_bs = 1;
  for (int bs : cand) {
    d->np_variant = bs;
    launch_step(d, d->stream, 0);  // warm-up
    e = cudaEventRecord(a, d->stream);
    for (int k = 0; k < 8 && e == cudaSuccess; k++) launch_step(d, d->stream, k & 1);
    if (e == cudaSuccess) e = cudaEventRecord(b, d->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) break;
    d->timing.kernel_launches += 9;
    if (bs == cand[0] || ms < best) {
      best = ms;
      best_bs = bs;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  d->np_variant = best_bs;
  d->np_block = kNpVariantBlock[best_bs];
  if (e != cudaSuccess) return cdi_cuda_fail(d, e, "tune transport step");
  d->np_tuned = true;
  cdi_tune_store(key, best_bs);
  return CDI_OK;
}

}  // namespace

int cdi_np_shape_block(int v) { return v >= 0 && v < 10 ? kNpVariantBlock[v] : 0; }

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
  d->imp_stale = true;  // the implicit operator follows u, phi and the species
  double dt = dt_s;
  if (dt <= 0.0) {
    cdi_status s = cdi_np_dt(d, d->h_scal[S_SCALE], &dt);
    if (s != CDI_OK) return s;
  }
  d->dt = dt;
  if (dt_used) *dt_used = dt;
  if (!d->np_tuned) {
    cdi_status s = tune_np(d);
    if (s != CDI_OK) return s;
  }
  if (d->prec == CDI_FP64)
    k_np_init<double><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        (double *)d->d_C[0], (double *)d->d_C[1], nullptr, nullptr, (int)d->n_pore, d->ns, d->c0,
        0.f);
  else
    k_np_init<float><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        (float *)d->d_C[0], (float *)d->d_C[1], d->d_Clo[0], d->d_Clo[1], (int)d->n_pore, d->ns,
        (float)d->c0, (float)(d->c0 - (double)(float)d->c0));
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "transport init");
  CDI_TRY(d, cudaMemsetAsync(d->d_acc, 0, (size_t)3 * kMaxSpecies * d->np_accs * 8, d->stream),
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

template <typename T, int DIM, bool PAIR>
void launch_sweep_d(cdi_domain *d, cudaStream_t st, const void *members, int n, int in) {
  const SweepMember<T> *m = (const SweepMember<T> *)members;
  const NPGeo g = make_geo(d);
  switch (d->ns) {
    case 1: k_np_sweep<T, DIM, 1, PAIR><<<d->np_blocks, kRowBlock, 0, st>>>(m, n, in, g); break;
    case 2: k_np_sweep<T, DIM, 2, PAIR><<<d->np_blocks, kRowBlock, 0, st>>>(m, n, in, g); break;
    case 3: k_np_sweep<T, DIM, 3, PAIR><<<d->np_blocks, kRowBlock, 0, st>>>(m, n, in, g); break;
    default: k_np_sweep<T, DIM, 4, PAIR><<<d->np_blocks, kRowBlock, 0, st>>>(m, n, in, g); break;
  }
}

void launch_sweep(cdi_domain *d, cudaStream_t st, const void *members, int n, int in) {
  if (d->prec == CDI_FP64) {
    if (d->dim == 2) launch_sweep_d<double, 2, false>(d, st, members, n, in);
    else launch_sweep_d<double, 3, false>(d, st, members, n, in);
  } else if (d->cpair) {
    if (d->dim == 2) launch_sweep_d<float, 2, true>(d, st, members, n, in);
    else launch_sweep_d<float, 3, true>(d, st, members, n, in);
  } else {
    if (d->dim == 2) launch_sweep_d<float, 2, false>(d, st, members, n, in);
    else launch_sweep_d<float, 3, false>(d, st, members, n, in);
  }
}

template <typename T>
cdi_status sweep_run(cdi_domain *d, int n, const double *scale, const int *group,
                     void *const *phi_groups, const double *dts, int64_t n_steps,
                     double *gamma, double *cout) {
  const size_t TN = (size_t)d->n_pore * sizeof(T);
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
    void *acc = take((size_t)3 * kMaxSpecies * d->np_accs * 8);
    void *l0 = d->cpair ? take((size_t)kMaxSpecies * d->n_pore * 4) : nullptr;
    void *l1 = d->cpair ? take((size_t)kMaxSpecies * d->n_pore * 4) : nullptr;
    ok = u && c0 && c1 && acc && (!d->cpair || (l0 && l1));
    if (!ok) break;
    d->dt = dts[m];
    hm[m].C[0] = (T *)c0;
    hm[m].C[1] = (T *)c1;
    hm[m].Cl[0] = (float *)l0;
    hm[m].Cl[1] = (float *)l1;
    for (int in = 0; in < 2; in++)
      hm[m].f[in] = fields32(d, in ? c1 : c0, in ? (float *)l1 : (float *)l0, in ? c0 : c1,
                             in ? (float *)l0 : (float *)l1, u, phi_groups[group[m]], acc);
    hm[m].u = (const T *)u;
    hm[m].phi = (const typename PhiStore<T>::type *)phi_groups[group[m]];
    hm[m].acc = (typename AccSlot<T>::type *)acc;
    hm[m].c = make_const<T>(d);
  }
  void *dmem = ok ? take(sizeof(SweepMember<T>) * n) : nullptr;
  cdi_status s = CDI_OK;
  if (!ok || !dmem) s = cdi_fail(d, CDI_ERR_OOM, "sweep: device allocation failed");
  for (int m = 0; m < n && s == CDI_OK; m++) {
    s = cdi_flow_scale_to(d, scale[m], (void *)hm[m].u);
    if (s != CDI_OK) break;
    k_np_init<T><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        hm[m].C[0], hm[m].C[1], hm[m].Cl[0], hm[m].Cl[1], (int)d->n_pore, ns, (T)d->c0,
        (float)(d->c0 - (double)(T)d->c0));
    d->timing.kernel_launches++;
    if (cudaMemsetAsync(hm[m].acc, 0, (size_t)3 * kMaxSpecies * d->np_accs * 8, d->stream) !=
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
        d->d_cmeta, hm[m].C[cur], hm[m].Cl[cur], hm[m].u, (int)d->n_pore, ns, vol, d->d_part,
        d->d_counter + C_MASS, d->d_scal);
    acc_total(d, hm[m].acc, d->stream, d->d_scal);
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

// ---------------------------------------------------------------------------
// Batch over several geometries: every (domain, combination) member in one
// launch per step.
// ---------------------------------------------------------------------------
namespace {

template <typename T, int DIM, bool PAIR>
void launch_batch_d(cudaStream_t st, int ns, const void *members, int n, int blocks, int in) {
  const BatchMember<T> *m = (const BatchMember<T> *)members;
  switch (ns) {
    case 1: k_np_batch<T, DIM, 1, PAIR><<<blocks, kRowBlock, 0, st>>>(m, n, in); break;
    case 2: k_np_batch<T, DIM, 2, PAIR><<<blocks, kRowBlock, 0, st>>>(m, n, in); break;
    case 3: k_np_batch<T, DIM, 3, PAIR><<<blocks, kRowBlock, 0, st>>>(m, n, in); break;
    default: k_np_batch<T, DIM, 4, PAIR><<<blocks, kRowBlock, 0, st>>>(m, n, in); break;
  }
}

template <typename T>
void launch_batch(const cdi_domain *lead, cudaStream_t st, const void *members, int n,
                  int blocks, int in) {
  if (std::is_same<T, float>::value && lead->cpair) {
    if (lead->dim == 2) launch_batch_d<T, 2, true>(st, lead->ns, members, n, blocks, in);
    else launch_batch_d<T, 3, true>(st, lead->ns, members, n, blocks, in);
  } else {
    if (lead->dim == 2) launch_batch_d<T, 2, false>(st, lead->ns, members, n, blocks, in);
    else launch_batch_d<T, 3, false>(st, lead->ns, members, n, blocks, in);
  }
}

template <typename T>
cdi_status batch_run(cdi_domain *const *doms, int n_doms, int n_combos, const double *scale,
                     const int *group, void *const *phis, const double *dts, int64_t n_steps,
                     double *gamma, double *cout) {
  cdi_domain *L = doms[0];  // the lead: its stream, allocator and scratch serve the batch
  const int n = n_doms * n_combos, ns = L->ns;
  std::vector<void *> blocks;
  auto take = [&](size_t bytes) {
    void *p = cdi_dev_alloc(L, bytes);
    if (p) blocks.push_back(p);
    return p;
  };
  std::vector<BatchMember<T>> hm(n);
  bool ok = true;
  int total_blocks = 0;
  for (int m = 0; m < n && ok; m++) {
    cdi_domain *d = doms[m / n_combos];
    const size_t TN = (size_t)d->n_pore * sizeof(T);
    void *u = take((size_t)d->dim * TN);
    void *c0 = take((size_t)kMaxSpecies * TN), *c1 = take((size_t)kMaxSpecies * TN);
    void *acc = take((size_t)3 * kMaxSpecies * d->np_accs * 8);
    void *l0 = d->cpair ? take((size_t)kMaxSpecies * d->n_pore * 4) : nullptr;
    void *l1 = d->cpair ? take((size_t)kMaxSpecies * d->n_pore * 4) : nullptr;
    ok = u && c0 && c1 && acc && (!d->cpair || (l0 && l1));
    if (!ok) break;
    d->dt = dts[m];
    hm[m].s.C[0] = (T *)c0;
    hm[m].s.C[1] = (T *)c1;
    hm[m].s.Cl[0] = (float *)l0;
    hm[m].s.Cl[1] = (float *)l1;
    for (int in = 0; in < 2; in++)
      hm[m].s.f[in] = fields32(d, in ? c1 : c0, in ? (float *)l1 : (float *)l0, in ? c0 : c1,
                               in ? (float *)l0 : (float *)l1, u, phis[group[m]], acc);
    hm[m].s.u = (const T *)u;
    hm[m].s.phi = (const typename PhiStore<T>::type *)phis[group[m]];
    hm[m].s.acc = (typename AccSlot<T>::type *)acc;
    hm[m].s.c = make_const<T>(d);
    hm[m].g = make_geo(d);
    hm[m].block0 = total_blocks;
    hm[m].nblocks = d->np_blocks;
    total_blocks += d->np_blocks;
  }
  void *dmem = ok ? take(sizeof(BatchMember<T>) * n) : nullptr;
  cdi_status s = CDI_OK;
  if (!ok || !dmem) s = cdi_fail(L, CDI_ERR_OOM, "batch: device allocation failed");
  // member velocities on their domains' streams (after the lead's stream
  // has made the members' memory available: stream-ordered allocations),
  // then everything on the lead's
  if (s == CDI_OK && cudaStreamSynchronize(L->stream) != cudaSuccess)
    s = cdi_fail(L, CDI_ERR_CUDA, "batch: member memory");
  for (int m = 0; m < n && s == CDI_OK; m++)
    s = cdi_flow_scale_to(doms[m / n_combos], scale[m], (void *)hm[m].s.u);
  for (int i = 0; i < n_doms && s == CDI_OK; i++)
    if (cudaStreamSynchronize(doms[i]->stream) != cudaSuccess)
      s = cdi_fail(L, CDI_ERR_CUDA, "batch: member setup");
  for (int m = 0; m < n && s == CDI_OK; m++) {
    const cdi_domain *d = doms[m / n_combos];
    k_np_init<T><<<kRedBlocks, kRedThreads, 0, L->stream>>>(
        hm[m].s.C[0], hm[m].s.C[1], hm[m].s.Cl[0], hm[m].s.Cl[1], (int)d->n_pore, ns, (T)d->c0,
        (float)(d->c0 - (double)(T)d->c0));
    L->timing.kernel_launches++;
    if (cudaMemsetAsync(hm[m].s.acc, 0, (size_t)3 * kMaxSpecies * d->np_accs * 8,
                        L->stream) != cudaSuccess)
      s = cdi_fail(L, CDI_ERR_CUDA, "batch: memset");
  }
  if (s == CDI_OK &&
      cudaMemcpyAsync(dmem, hm.data(), sizeof(BatchMember<T>) * n, cudaMemcpyHostToDevice,
                      L->stream) != cudaSuccess)
    s = cdi_fail(L, CDI_ERR_CUDA, "batch: member table");
  cudaGraphExec_t exec = nullptr;
  int64_t done = 0;
  if (s == CDI_OK) {
    cudaEvent_t ev;
    cdi_timing_begin(L, &ev);
    if (n_steps >= kGraphSteps) {
      cudaGraph_t graph;
      cudaError_t e = cudaStreamBeginCapture(L->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        for (int k = 0; k < kGraphSteps; k++)
          launch_batch<T>(L, L->cap_stream, dmem, n, total_blocks, k & 1);
        e = cudaStreamEndCapture(L->cap_stream, &graph);
      }
      if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
      }
      if (e != cudaSuccess) s = cdi_cuda_fail(L, e, "batch graph");
      while (s == CDI_OK && n_steps - done >= kGraphSteps) {
        e = cudaGraphLaunch(exec, L->stream);
        if (e != cudaSuccess) s = cdi_cuda_fail(L, e, "batch graph launch");
        done += kGraphSteps;
      }
    }
    for (; s == CDI_OK && done < n_steps; done++)
      launch_batch<T>(L, L->stream, dmem, n, total_blocks, (int)(done & 1));
    cudaError_t e = cudaGetLastError();
    if (s == CDI_OK && e != cudaSuccess) s = cdi_cuda_fail(L, e, "batch step");
    cdi_timing_end(L, ev, PH_NP, n_steps);
    L->timing.kernel_launches += n_steps;
  }
  // outputs per member, through the same reductions as a single run
  const int cur = (int)(n_steps & 1);
  for (int m = 0; m < n && s == CDI_OK; m++) {
    const cdi_domain *d = doms[m / n_combos];
    const double area = d->dim == 2 ? d->dx : d->dx * d->dx;
    const double vol = d->dim == 2 ? d->dx * d->dx : d->dx * d->dx * d->dx;
    k_np_sums<T><<<kRedBlocks, kRedThreads, 0, L->stream>>>(
        d->d_cmeta, hm[m].s.C[cur], hm[m].s.Cl[cur], hm[m].s.u, (int)d->n_pore, ns, vol,
        L->d_part, L->d_counter + C_MASS, L->d_scal);
    acc_total(d, hm[m].s.acc, L->stream, L->d_scal);
    L->timing.kernel_launches += 2;
    cudaError_t e = cudaMemcpyAsync(L->h_scal + S_OUT, L->d_scal + S_OUT,
                                    (S_OUTN - S_OUT + 1) * sizeof(double),
                                    cudaMemcpyDeviceToHost, L->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
    if (e != cudaSuccess) {
      s = cdi_cuda_fail(L, e, "batch outputs");
      break;
    }
    for (int k = 0; k < ns; k++) {
      gamma[m * ns + k] = L->h_scal[S_ACC + 3 * k] * dts[m] * area;
      const double num = L->h_scal[S_OUT + 2 * k], den = L->h_scal[S_OUT + 2 * k + 1];
      const double cnt = L->h_scal[S_OUTN];
      cout[m * ns + k] = den != 0.0 ? num / den : (cnt > 0 ? L->h_scal[S_OUTP + k] / cnt : 0.0);
    }
  }
  if (s == CDI_OK) {
    cudaError_t e = cdi_timing_resolve(L);
    if (e != cudaSuccess) s = cdi_cuda_fail(L, e, "timing");
  }
  cudaStreamSynchronize(L->stream);
  if (exec) cudaGraphExecDestroy(exec);
  for (void *p : blocks) cdi_dev_release(L, p);
  return s;
}

}  // namespace

cdi_status cdi_np_batch(cdi_domain *const *doms, int n_doms, int n_combos, const double *scale,
                        const int *group, void *const *phis, const double *dts, int64_t n_steps,
                        double *gamma, double *cout) {
  if (doms[0]->prec == CDI_FP64)
    return batch_run<double>(doms, n_doms, n_combos, scale, group, phis, dts, n_steps, gamma,
                             cout);
  return batch_run<float>(doms, n_doms, n_combos, scale, group, phis, dts, n_steps, gamma, cout);
}

cdi_status cdi_np_sweep(cdi_domain *d, int n, const double *scale, const int *group,
                        void *const *phi_groups, const double *dts, int64_t n_steps,
                        double *gamma, double *cout) {
  if (d->prec == CDI_FP64)
    return sweep_run<double>(d, n, scale, group, phi_groups, dts, n_steps, gamma, cout);
  return sweep_run<float>(d, n, scale, group, phi_groups, dts, n_steps, gamma, cout);
}

// Coupled stepping (Eq. 3-5): before every block of couple_K steps (counted
// from cdi_init_transport) the potential is re-solved from the current
// concentrations; the steps of a block are plain launches.
static cdi_status np_steps_coupled(cdi_domain *d, int64_t n) {
  const int64_t K = d->couple_K;
  while (n > 0) {
    if (d->np_steps % K == 0) {
      if (d->np_graph) cudaGraphExecDestroy(d->np_graph);
      d->np_graph = nullptr;
      cdi_status s = cdi_psi_coupled(d);
      if (s != CDI_OK) return s;
    }
    const int64_t block = std::min<int64_t>(n, K - d->np_steps % K);
    if (d->imp_tol > 0.0) {  // implicit steps in the re-solved potential
      d->imp_stale = true;
      cdi_status s = cdi_imp_steps(d, block);
      if (s != CDI_OK) return s;
      n -= block;
      continue;
    }
    cudaEvent_t ev;
    cdi_timing_begin(d, &ev);
    for (int64_t k = 0; k < block; k++) {
      launch_step(d, d->stream, d->cur);
      d->cur = 1 - d->cur;
    }
    CDI_TRY(d, cudaGetLastError(), "transport step");
    cdi_timing_end(d, ev, PH_NP, block);
    d->timing.kernel_launches += block;
    d->np_steps += block;
    n -= block;
  }
  return CDI_OK;
}

cdi_status cdi_np_steps(cdi_domain *d, int64_t n) {
  if (n == 0) return CDI_OK;
  if (d->couple_K > 0) return np_steps_coupled(d, n);
  if (d->imp_tol > 0.0) return cdi_imp_steps(d, n);
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
        d->d_cmeta, (const double *)d->d_C[d->cur], nullptr, (const double *)d->d_u,
        (int)d->n_pore, d->ns, vol, d->d_part, d->d_counter + C_MASS, d->d_scal);
  else
    k_np_sums<float><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        d->d_cmeta, (const float *)d->d_C[d->cur], d->d_Clo[d->cur], (const float *)d->d_u,
        (int)d->n_pore, d->ns, vol, d->d_part, d->d_counter + C_MASS, d->d_scal);
  acc_total(d, d->d_acc, d->stream, d->d_scal);
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

cdi_status cdi_np_geometry(cdi_domain *d, double *pores, double *faces, double *sum_ux) {
  if (d->prec == CDI_FP64)
    k_geometry<double><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        d->d_cmeta, (const double *)d->d_u, (int)d->n_pore, 2 * d->dim, d->d_part,
        d->d_counter + C_GEOM, d->d_scal);
  else
    k_geometry<float><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        d->d_cmeta, (const float *)d->d_u, (int)d->n_pore, 2 * d->dim, d->d_part,
        d->d_counter + C_GEOM, d->d_scal);
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "geometry");
  CDI_TRY(d, cudaMemcpyAsync(d->h_scal + S_GEOM, d->d_scal + S_GEOM, 3 * sizeof(double),
                             cudaMemcpyDeviceToHost, d->stream),
          "geometry copy");
  CDI_TRY(d, cudaStreamSynchronize(d->stream), "geometry");
  *pores = d->h_scal[S_GEOM];
  *faces = d->h_scal[S_GEOM + 1];
  if (sum_ux) *sum_ux = d->h_scal[S_GEOM + 2];
  return CDI_OK;
}

cdi_status cdi_np_column_means(cdi_domain *d, int k) {
  const size_t T = d->prec == CDI_FP64 ? 8 : 4;
  const void *C = (const char *)d->d_C[d->cur] + (size_t)k * d->n_pore * T;
  const float *Cl = d->d_Clo[d->cur] ? d->d_Clo[d->cur] + (size_t)k * d->n_pore : nullptr;
  const int rows = d->ny * d->nz;
  if (d->prec == CDI_FP64)
    k_colmeans<double><<<d->nx, kRedThreads, 0, d->stream>>>(d->d_words, d->W, (const double *)C,
                                                             nullptr, rows, d->d_colout);
  else
    k_colmeans<float><<<d->nx, kRedThreads, 0, d->stream>>>(d->d_words, d->W, (const float *)C,
                                                            Cl, rows, d->d_colout);
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "column means");
  return CDI_OK;
}

// Rank metadata and row words of the compact transport layout (after the
// pore lists and the face flags).
cdi_status cdi_np_build_compact(cdi_domain *d) {
  const int n = (int)d->n_pore;
  const long long n_words = (long long)d->ny * d->nz * d->W;
  k_cmeta<<<kRedBlocks, kRedThreads, 0, d->stream>>>(d->d_nflags, d->d_cell_list, n, d->nx,
                                                     d->d_cmeta, d->d_cfl);
  k_words<<<kRedBlocks, kRedThreads, 0, d->stream>>>(d->d_nflags, d->d_cell_list, n, d->nx, d->W,
                                                     n_words, d->d_words);
  k_lat_nbr<<<kRedBlocks, kRedThreads, 0, d->stream>>>(d->d_cmeta, d->d_words, n, d->W, d->ny,
                                                       d->nz, d->walls, 2 * d->dim, d->d_latnb);
  d->timing.kernel_launches += 3;
  CDI_TRY(d, cudaGetLastError(), "compact layout");
  return CDI_OK;
}

// comps rank-ordered components of the domain's precision -> FP64 lattice
// fields (dst: comps * N doubles, 0 in solid cells).
cdi_status cdi_np_scatter(cdi_domain *d, const void *src, const float *lo, int comps,
                          double *dst) {
  CDI_TRY(d, cudaMemsetAsync(dst, 0, (size_t)comps * d->N * 8, d->stream), "scatter reset");
  if (d->prec == CDI_FP64)
    k_scatter<double><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        (const double *)src, nullptr, comps, d->d_cell_list, (int)d->n_pore, d->N, dst);
  else
    k_scatter<float><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        (const float *)src, lo, comps, d->d_cell_list, (int)d->n_pore, d->N, dst);
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "scatter");
  return CDI_OK;
}
