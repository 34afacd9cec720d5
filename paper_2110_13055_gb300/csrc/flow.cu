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
//
// Four storage modes: FP64; FP32; FP32 pairs (hi + lo in two arrays,
// updated with error-free FP32 transformations: FP64-class accuracy at FP32
// arithmetic rates, which matters on a part whose FP64 rate is low); and BF16
// (collision in FP32, half the bytes of FP32, low accuracy).
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>

#include "cdi_internal.cuh"

using namespace cdi;

namespace {

enum Mode { M_F64 = 0, M_F32 = 1, M_SPLIT = 2, M_BF16 = 3 };

// Arithmetic type of a population storage type (BF16 is widened to FP32).
template <typename S> struct Arith { using type = S; };
template <> struct Arith<__nv_bfloat16> { using type = float; };
__device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ double widen(double v) { return v; }
template <typename S> __device__ __forceinline__ S narrow(typename Arith<S>::type v) {
  return (S)v;
}
template <> __device__ __forceinline__ __nv_bfloat16 narrow<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------------------
// Error-free FP32 transformations (Knuth's two-sum, Dekker's fast two-sum,
// the FMA product error) and unevaluated pairs hi + lo built on them.
// ---------------------------------------------------------------------------
struct F2 {
  float h, l;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
  return {s, e};
}
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const F2 s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ F2 f2_neg(F2 a) { return {-a.h, -a.l}; }
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}
// s + c += v with s the rounded running sum and c the accumulated errors.
__device__ __forceinline__ void two_sum_acc(float v, float &s, float &c) {
  const F2 t = two_sum(s, v);
  s = t.h;
  c = __fadd_rn(c, t.l);
}

F2 host_pair(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

// Site index and neighbour offsets in 32 bits (domains are limited to < 2^31
// flow sites); the periodic wrap is folded into the offsets from the edge
// bits of the flag word, so no coordinates are needed.
template <int DIM> struct SiteIdx {
  int s, oxp, oxm, oyp, oym, ozp, ozm;
  __device__ __forceinline__ SiteIdx(int site, unsigned f, int NX, int ny, int nz) {
    using W = WrapBit<DIM>;
    const int plane = NX * ny;
    s = site;
    oxp = (f >> W::XHI) & 1u ? 1 - NX : 1;
    oxm = (f >> W::XLO) & 1u ? NX - 1 : -1;
    oyp = (f >> W::YHI) & 1u ? (1 - ny) * NX : NX;
    oym = (f >> W::YLO) & 1u ? (ny - 1) * NX : -NX;
    ozp = (f >> W::ZHI) & 1u ? (1 - nz) * plane : plane;
    ozm = (f >> W::ZLO) & 1u ? (nz - 1) * plane : -plane;
  }
  __device__ __forceinline__ int nb(int ex, int ey, int ez) const {
    return s + (ex > 0 ? oxp : (ex < 0 ? oxm : 0)) + (ey > 0 ? oyp : (ey < 0 ? oym : 0)) +
           (ez > 0 ? ozp : (ez < 0 ? ozm : 0));
  }
};

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
  using W = WrapBit<DIM>;
  unsigned f = solid_at(x, y, z) ? 1u : 0u;
#pragma unroll
  for (int i = 1; i < L::Q; i++)
    if (solid_at(x + L::ex(i), y + L::ey(i), z + L::ez(i))) f |= (1u << i);
  if (x == NX - 1) f |= 1u << W::XHI;
  if (x == 0) f |= 1u << W::XLO;
  if (y == ny - 1) f |= 1u << W::YHI;
  if (y == 0) f |= 1u << W::YLO;
  if (z == nz - 1) f |= 1u << W::ZHI;
  if (z == 0) f |= 1u << W::ZLO;
  fl[((size_t)z * ny + y) * NX + x] = (typename FlowFlag<DIM>::type)f;
}

// Populations are stored compactly by pore rank k (the position of the site
// in the ascending pore-site list): g[i * n + k].
//
// Neighbour ranks for the odd step, without a per-direction table.  Per pore
// rank k (site x_k = (x, row), row = (y, z)):
//   lf[k]          the site's solid-neighbour bits (bit i: the site x_k + e_i
//                  is solid or beyond a lateral wall, so the link bounces
//                  back) and kLinkEdge when the site's ranks come from the
//                  overflow table (below);
//   R_o(k)         for each lateral row offset o = (ey, ez) of the lattice
//                  (2 for D2Q9, 8 for D3Q19): the rank the site (x, row + o)
//                  has, or would have if it is solid (the number of pore
//                  sites before it in lattice order).
// Pore sites of one row are consecutive ranks, so the neighbour along e_i is
// k + ex when it stays in the row, and otherwise R_o (ex = 0), R_o - 1
// (ex = -1) or R_o + [site (x, row + o) is pore] (ex = +1).  R_o - k changes
// slowly along the rank order, so it is stored as a per-tile base (lb[o *
// n_ltiles + k / 32], 32 consecutive ranks a tile) plus one signed byte per
// offset and site (ld: byte o of the site's 4-byte words).  Sites at the
// first or last column (where the periodic x neighbour wraps around) and
// sites whose byte would overflow take all Q - 1 ranks from an overflow table
// instead (ovf[(i - 1) * n_ovf + e], -1 for a bounce-back link; e in the
// site's first word): slot 2 * row + (x != 0) for an x-edge site, 2 ny nz +
// (a running count) for the others.  The odd step reads 4 + 8 bytes per site
// in 3D (4 + 4 in 2D) this way, plus a tile's bases once per 32 sites,
// instead of 4 * (Q - 1) bytes.
constexpr unsigned kLinkEdge = 1u << 31;

template <int DIM> struct LatOff;
template <> struct LatOff<2> {
  static constexpr int NO = 2;
  __host__ __device__ static constexpr int ey(int o) { return o == 0 ? 1 : -1; }
  __host__ __device__ static constexpr int ez(int) { return 0; }
};
template <> struct LatOff<3> {
  static constexpr int NO = 8;
  // (ey, ez): (1,0) (-1,0) (0,1) (0,-1) (1,1) (1,-1) (-1,1) (-1,-1)
  __host__ __device__ static constexpr int ey(int o) {
    return o == 0 || o == 4 || o == 5 ? 1 : (o == 1 || o == 6 || o == 7 ? -1 : 0);
  }
  __host__ __device__ static constexpr int ez(int o) {
    return o == 2 || o == 4 || o == 6 ? 1 : (o == 3 || o == 5 || o == 7 ? -1 : 0);
  }
};
// Row offset of direction i (-1 when it stays in the row).
template <int DIM> __host__ __device__ constexpr int off_of(int i) {
  using L = Lat<DIM>;
  using O = LatOff<DIM>;
  if (L::ey(i) == 0 && L::ez(i) == 0) return -1;
  for (int o = 0; o < O::NO; o++)
    if (O::ey(o) == L::ey(i) && O::ez(o) == L::ez(i)) return o;
  return -1;
}
// Direction (0, ey, ez) of row offset o.
template <int DIM> __host__ __device__ constexpr int dir_of_off(int o) {
  using L = Lat<DIM>;
  using O = LatOff<DIM>;
  for (int i = 1; i < L::Q; i++)
    if (L::ex(i) == 0 && L::ey(i) == O::ey(o) && L::ez(i) == O::ez(o)) return i;
  return -1;
}

struct LinkGeo {
  const unsigned *lf;  // n: solid-neighbour bits | kLinkEdge
  const unsigned *ld;  // LinkWords * n: the sites' row-base bytes (or slot)
  const int *lb;       // NO * n_tiles: the tiles' row bases
  const int *ovf;      // (Q - 1) * n_ovf: full neighbour ranks
  int n_ovf;
  int n_tiles;
};
// 4-byte words of row-base bytes per site.
template <int DIM> __host__ __device__ constexpr int link_words() { return (LatOff<DIM>::NO + 3) / 4; }

// Where direction i of pore rank k lives: plane i of the population array
// (plane i = direction i of every pore rank).  Planes<S, Q> passes the Q
// plane base pointers by value, so a kernel reads them from its parameter
// space and an address is one 32-bit-index multiply-add; Strided forms them
// from the array base and the plane length (used where one launch serves
// several domains).
template <typename S, int Q> struct Planes {
  S *p[Q];
  __device__ __forceinline__ S *plane(int i) const { return p[i]; }
};
template <typename S> struct Strided {
  S *g;
  long long n;
  __device__ __forceinline__ S *plane(int i) const { return g + (size_t)i * n; }
};
template <typename S, int Q> Planes<S, Q> make_planes(S *g, long long n) {
  Planes<S, Q> pl;
  for (int i = 0; i < Q; i++) pl.p[i] = g + (size_t)i * n;
  return pl;
}

// Slot read by direction i at rank k (ODD: the upstream neighbour's opposite
// slot, or the own slot after a bounce-back), and slot written by the
// post-collision value of direction i.  nb[j] caches the neighbour rank of
// direction j (-1: bounce-back).  Returned as (plane, index in the plane).
template <int DIM, bool ODD>
__device__ __forceinline__ int read_slot(const int *nb, int k, int i, int &idx) {
  using L = Lat<DIM>;
  idx = k;
  if (!ODD || i == 0) return i;
  const int src = nb[L::opp(i)];  // the site x - e_i
  if (src < 0) return i;          // upstream solid: the bounced value
  idx = src;
  return L::opp(i);
}
template <int DIM, bool ODD>
__device__ __forceinline__ int write_slot(const int *nb, int k, int i, int &idx) {
  using L = Lat<DIM>;
  idx = k;
  if (!ODD || i == 0) return L::opp(i);
  const int dst = nb[i];          // the site x + e_i
  if (dst < 0) return L::opp(i);  // bounce back from a solid
  idx = dst;
  return i;
}
// The address of a slot: the two candidate planes are compile-time indices,
// so only the base pointer and the index are selected at run time.
template <int DIM, bool ODD, bool READ, typename PL>
__device__ __forceinline__ auto slot_ptr(const PL &pl, const int *nb, int k, int i) {
  using L = Lat<DIM>;
  if (!ODD || i == 0) return pl.plane(READ ? i : L::opp(i)) + k;
  const int q = READ ? nb[L::opp(i)] : nb[i];
  const bool bounce = q < 0;
  auto *own = pl.plane(READ ? i : L::opp(i));
  auto *other = pl.plane(READ ? L::opp(i) : i);
  return (bounce ? own : other) + (bounce ? k : q);
}

// The link data of pore rank k: its flag word and row bases.
template <int DIM> struct LinkData {
  unsigned f;
  int R[LatOff<DIM>::NO];
};
// (R[0] holds the overflow slot at a kLinkEdge site.)
template <int DIM>
__device__ __forceinline__ LinkData<DIM> load_link_data(const LinkGeo &lg, int k, long long) {
  constexpr int NO = LatOff<DIM>::NO;
  LinkData<DIM> ld;
  ld.f = lg.lf[k];
  unsigned w[link_words<DIM>()];
  if constexpr (link_words<DIM>() == 2) {
    const uint2 v = reinterpret_cast<const uint2 *>(lg.ld)[k];
    w[0] = v.x;
    w[1] = v.y;
  } else {
    w[0] = lg.ld[k];
  }
  const int t = k >> 5;
#pragma unroll
  for (int o = 0; o < NO; o++) {
    const int b = (int)(w[o >> 2] << (24 - 8 * (o & 3))) >> 24;  // signed byte o
    ld.R[o] = k + lg.lb[(size_t)o * lg.n_tiles + t] + b;
  }
  if (ld.f & kLinkEdge) ld.R[0] = (int)w[0];
  return ld;
}

// Neighbour ranks of pore rank k (all Q-1 directions) from its link data.
template <int DIM>
__device__ __forceinline__ void decode_links(const LinkGeo &lg, const LinkData<DIM> &ld, int k,
                                             int (&nb)[Lat<DIM>::Q]) {
  using L = Lat<DIM>;
  const unsigned f = ld.f;
  const int *R = ld.R;
  nb[0] = k;
#pragma unroll
  for (int i = 1; i < L::Q; i++) {
    const int o = off_of<DIM>(i);
    int r;
    if (o < 0) {
      r = k + L::ex(i);
    } else if (L::ex(i) == 0) {
      r = R[o];
    } else if (L::ex(i) < 0) {
      r = R[o] - 1;
    } else {
      r = R[o] + (int)(((f >> dir_of_off<DIM>(o)) & 1u) ^ 1u);
    }
    nb[i] = ((f >> i) & 1u) ? -1 : r;
  }
  if (f & kLinkEdge) {  // the x neighbours wrap: all ranks from the overflow table
    const int e = R[0];
#pragma unroll
    for (int i = 1; i < L::Q; i++) nb[i] = lg.ovf[(size_t)(i - 1) * lg.n_ovf + e];
  }
}

// Neighbour ranks of pore rank k for the odd step (all Q-1 directions).
template <int DIM, bool ODD>
__device__ __forceinline__ void load_links(const LinkGeo &lg, int k, long long n,
                                           int (&nb)[Lat<DIM>::Q]) {
  nb[0] = k;
  if (!ODD) return;
  decode_links<DIM>(lg, load_link_data<DIM>(lg, k, n), k, nb);
}

__global__ void k_rank_scatter(const int *__restrict__ list, int n, int *__restrict__ rank) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    rank[list[k]] = k;
}

// Builds lf, ld and lb (rank[site]: the pore rank, -1 for a solid site), one
// warp per 32-rank tile.  A tile's base of offset o is R_o - k of its first
// site that uses offset o (one of (x - 1, x, x + 1) in row + o is pore and
// the row is not beyond a wall); a site whose R_o - k - base does not fit a
// signed byte, like an x-edge site, is marked kLinkEdge and gets an overflow
// slot (e in its first word), filled by k_links_ovf once the table is sized.
template <int DIM>
__global__ void k_links(const typename FlowFlag<DIM>::type *__restrict__ fl,
                        const int *__restrict__ list, int n, const int *__restrict__ rank,
                        unsigned *__restrict__ lf, unsigned *__restrict__ ld,
                        int *__restrict__ lb, int n_tiles, unsigned *__restrict__ n_extra,
                        int NX, int ny, int nz, int walls) {
  using L = Lat<DIM>;
  using O = LatOff<DIM>;
  using W = WrapBit<DIM>;
  constexpr int NW = link_words<DIM>();
  constexpr unsigned kSolidBits = ((1u << L::Q) - 1u) & ~1u;
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_tiles; t += warps) {
    const int k = 32 * t + lane;
    const bool valid = k < n;
    const int s = valid ? list[k] : 0;
    const unsigned f = valid ? (unsigned)fl[s] : 0u;
    const int x = s % NX, row = s / NX, y = row % ny, z = row / ny;
    const bool xedge = valid && (((f >> W::XHI) & 1u) || ((f >> W::XLO) & 1u));
    unsigned w[NW];
#pragma unroll
    for (int j = 0; j < NW; j++) w[j] = 0u;
    bool wide = false;
#pragma unroll
    for (int o = 0; o < O::NO; o++) {
      int Y = y + O::ey(o), Z = z + O::ez(o);
      int R = 0;
      bool used = false;
      const bool beyond = Y < 0 || Y >= ny || Z < 0 || Z >= nz;
      if (valid && !xedge && !(beyond && walls)) {
        Y = (Y + ny) % ny;
        Z = (Z + nz) % nz;
        const int sp = (Z * ny + Y) * NX + x;  // x - 1 and x + 1 stay in the row
        used = true;
        if (rank[sp] >= 0) R = rank[sp];
        else if (rank[sp + 1] >= 0) R = rank[sp + 1];
        else if (rank[sp - 1] >= 0) R = rank[sp - 1] + 1;
        else used = false;  // all three links bounce back: R_o is never read
      }
      const unsigned users = __ballot_sync(0xffffffffu, used);
      const int D = R - k;
      const int base = users ? __shfl_sync(0xffffffffu, D, __ffs(users) - 1) : 0;
      if (lane == 0) lb[(size_t)o * n_tiles + t] = base;
      const int b = used ? D - base : 0;
      if (b < -128 || b > 127) wide = true;
      w[o >> 2] |= ((unsigned)b & 0xffu) << (8 * (o & 3));
    }
    if (!valid) continue;
    if (xedge) {
      w[0] = (unsigned)(2 * row + (x != 0 ? 1 : 0));
    } else if (wide) {
      w[0] = (unsigned)(2 * ny * nz) + atomicAdd(n_extra, 1u);
    }
    lf[k] = (f & kSolidBits) | ((xedge || wide) ? kLinkEdge : 0u);
#pragma unroll
    for (int j = 0; j < NW; j++) ld[(size_t)k * NW + j] = w[j];
  }
}

// Fills the overflow slots of the kLinkEdge sites: all Q - 1 neighbour ranks
// (-1 for a bounce-back link).
template <int DIM>
__global__ void k_links_ovf(const typename FlowFlag<DIM>::type *__restrict__ fl,
                            const int *__restrict__ list, int n, const int *__restrict__ rank,
                            const unsigned *__restrict__ lf, const unsigned *__restrict__ ld,
                            int *__restrict__ ovf, int n_ovf, int NX, int ny, int nz) {
  using L = Lat<DIM>;
  constexpr int NW = link_words<DIM>();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    if (!(lf[k] & kLinkEdge)) continue;
    const int s = list[k];
    const unsigned f = fl[s];
    const int e = (int)ld[(size_t)k * NW];
    const SiteIdx<DIM> ix(s, f, NX, ny, nz);
#pragma unroll
    for (int i = 1; i < L::Q; i++)
      ovf[(size_t)(i - 1) * n_ovf + e] =
          ((f >> i) & 1u) ? -1 : rank[ix.nb(L::ex(i), L::ey(i), L::ez(i))];
  }
}

// One full lattice Boltzmann step (stream + collide) at every pore site,
// FP64, FP32 or BF16 storage (S), arithmetic in T = Arith<S>.  Collision (Eq. 8) with the Stokes-linear
// equilibrium g_eq_i = w_i (drho + 3 e_i.j), j = sum e_i g_i + F/2, and the
// force source (1 - 1/(2 tau)) 3 w_i e_i.F; omega = 1/tau.
// (more resident blocks per SM: the step is latency-bound on its scattered
// loads, so occupancy matters more than a few spare registers; the bound is
// chosen per variant so that nothing spills)
template <typename S, int DIM, bool ODD, typename PL>
__device__ __forceinline__ void lbm_body_nb(const PL &g, const int (&nb)[Lat<DIM>::Q], int k0,
                                            typename Arith<S>::type omega,
                                            typename Arith<S>::type fx_half,
                                            typename Arith<S>::type fsrc) {
  using T = typename Arith<S>::type;
  using L = Lat<DIM>;
  constexpr int Q = L::Q;
  T gi[Q];
#pragma unroll
  for (int i = 0; i < Q; i++) gi[i] = widen(*slot_ptr<DIM, ODD, true>(g, nb, k0, i));
  T drho = T(0), jx = fx_half, jy = T(0), jz = T(0);
#pragma unroll
  for (int i = 0; i < Q; i++) {
    drho += gi[i];
    if (L::ex(i)) jx += T(L::ex(i)) * gi[i];
    if (L::ey(i)) jy += T(L::ey(i)) * gi[i];
    if (DIM == 3 && L::ez(i)) jz += T(L::ez(i)) * gi[i];
  }
  // Post-collision values, each stored as soon as it is formed (fewer live
  // registers, so more resident warps for the gathered loads); the rest
  // population last.
  //
  // FP32 storage: the collision conserves mass exactly, but rounding the
  // stored values does not, and the leak is biased; it feeds the slowest
  // (pressure-diffusion) modes of the porous flow.  The rest population
  // closes the balance: g*_0 = sum_i g_i - sum_{i>0} g*_i, both sums carried
  // exactly as (sum, error) pairs.
  constexpr bool kClose = std::is_same<S, float>::value;
  float ms = 0.f, mc = 0.f, ss = 0.f, sc = 0.f;
  if (kClose) {
#pragma unroll
    for (int i = 0; i < Q; i++) two_sum_acc((float)gi[i], ms, mc);
  }
  auto post = [&](int i) {
    const T eu = T(L::ex(i)) * jx + T(L::ey(i)) * jy + T(L::ez(i)) * jz;
    const T geq = T(L::w(i)) * (drho + T(3) * eu);
    return gi[i] - omega * (gi[i] - geq) + T(L::w(i) * L::ex(i)) * fsrc;
  };
#pragma unroll
  for (int i = 1; i < Q; i++) {
    const T go = post(i);
    if (kClose) two_sum_acc((float)go, ss, sc);
    *slot_ptr<DIM, ODD, false>(g, nb, k0, i) = narrow<S>(go);
  }
  const T go0 = kClose ? (T)__fadd_rn(__fsub_rn(ms, ss), __fsub_rn(mc, sc)) : post(0);
  *slot_ptr<DIM, ODD, false>(g, nb, k0, 0) = narrow<S>(go0);
}

template <typename S, int DIM, bool ODD, typename PL>
__device__ __forceinline__ void lbm_body(const PL &g, const LinkGeo &lg, int n, int k0,
                                         typename Arith<S>::type omega,
                                         typename Arith<S>::type fx_half,
                                         typename Arith<S>::type fsrc) {
  int nb[Lat<DIM>::Q];
  load_links<DIM, ODD>(lg, k0, n, nb);
  lbm_body_nb<S, DIM, ODD>(g, nb, k0, omega, fx_half, fsrc);
}

// The odd step as a grid-stride loop: while a site gathers, collides and
// scatters, the link data of the thread's next site is already on its way
// (sites may run in any order: in the AA pattern every slot is read and
// written by one site only), so the link load no longer adds a memory round
// trip ahead of the gathers.  Same arithmetic per site as k_lbm_step.
template <typename S, int DIM, int BS>
__global__ void __launch_bounds__(BS, sizeof(S) == 8 ? 1 : (DIM == 2 ? 8 : 6) * 128 / BS)
    k_lbm_odd_pf(Planes<S, Lat<DIM>::Q> g, LinkGeo lg, int n, typename Arith<S>::type omega,
                 typename Arith<S>::type fx_half, typename Arith<S>::type fsrc) {
  const int stride = gridDim.x * BS;
  int k = blockIdx.x * BS + threadIdx.x;
  if (k >= n) return;
  LinkData<DIM> cur = load_link_data<DIM>(lg, k, n);
  while (true) {
    const int kn = k + stride;
    LinkData<DIM> nxt;
    if (kn < n) nxt = load_link_data<DIM>(lg, kn, n);
    int nb[Lat<DIM>::Q];
    decode_links<DIM>(lg, cur, k, nb);
    lbm_body_nb<S, DIM, true>(g, nb, k, omega, fx_half, fsrc);
    if (kn >= n) break;
    k = kn;
    cur = nxt;
  }
}

template <typename S, int DIM, bool ODD, int BS, int MINT>
__global__ void __launch_bounds__(BS, (MINT > 0 ? MINT : (DIM == 2 ? 8 : (sizeof(S) == 8 ? 4 : 7)) * 128) / BS)
    k_lbm_step(Planes<S, Lat<DIM>::Q> g, LinkGeo lg, int n,
               typename Arith<S>::type omega, typename Arith<S>::type fx_half,
               typename Arith<S>::type fsrc) {
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (k0 >= n) return;
  lbm_body<S, DIM, ODD>(g, lg, n, k0, omega, fx_half, fsrc);
}

// Constants of the pair collision, each an unevaluated FP32 pair.
struct SplitConst {
  F2 omega;     // 1 / tau
  F2 one_minus_omega;
  F2 fx_half;   // F / 2
  F2 src_axis;  // (1 - 1/(2 tau)) 3 F w_axis
  F2 src_diag;  // (1 - 1/(2 tau)) 3 F w_diag
};

// The same step with every population stored as an FP32 pair gh + gl and the
// collision carried out in pair arithmetic.
template <int DIM, bool ODD, bool TAU1, typename PL>
__device__ __forceinline__ void lbm_split_body_nb(const PL &gh, const PL &gl,
                                                  const int (&nb)[Lat<DIM>::Q], int k0,
                                                  const SplitConst &c) {
  using L = Lat<DIM>;
  constexpr int Q = L::Q;
  // lattice weights as FP32 pairs: rest, axis, diagonal
  constexpr double w0 = L::w(0), wa = L::w(1), wd = L::w(Q - 1);
  constexpr F2 kW0 = {(float)w0, (float)(w0 - (double)(float)w0)};
  constexpr F2 kWA = {(float)wa, (float)(wa - (double)(float)wa)};
  constexpr F2 kWD = {(float)wd, (float)(wd - (double)(float)wd)};
  F2 gi[Q];
#pragma unroll
  for (int i = 0; i < Q; i++) {
    int idx;
    const int pl = read_slot<DIM, ODD>(nb, k0, i, idx);
    gi[i] = {gh.plane(pl)[idx], gl.plane(pl)[idx]};
  }
  // moments as pairs: exact sums of the high parts plus the low parts
  float rs = 0.f, rc = 0.f, xs = 0.f, xc = 0.f, ys = 0.f, yc = 0.f, zs = 0.f, zc = 0.f;
#pragma unroll
  for (int i = 0; i < Q; i++) {
    two_sum_acc(gi[i].h, rs, rc);
    rc = __fadd_rn(rc, gi[i].l);
    if (L::ex(i)) {
      two_sum_acc(L::ex(i) > 0 ? gi[i].h : -gi[i].h, xs, xc);
      xc = __fadd_rn(xc, L::ex(i) > 0 ? gi[i].l : -gi[i].l);
    }
    if (L::ey(i)) {
      two_sum_acc(L::ey(i) > 0 ? gi[i].h : -gi[i].h, ys, yc);
      yc = __fadd_rn(yc, L::ey(i) > 0 ? gi[i].l : -gi[i].l);
    }
    if (DIM == 3 && L::ez(i)) {
      two_sum_acc(L::ez(i) > 0 ? gi[i].h : -gi[i].h, zs, zc);
      zc = __fadd_rn(zc, L::ez(i) > 0 ? gi[i].l : -gi[i].l);
    }
  }
  const F2 drho = fast_two_sum(rs, rc);
  const F2 jx = f2_add(fast_two_sum(xs, xc), c.fx_half);
  const F2 jy = fast_two_sum(ys, yc);
  const F2 jz = fast_two_sum(zs, zc);
  // Equilibrium by weight class: g_eq_i = w drho + sum_a e_ia (3 w j_a), with
  // w drho and 3 w j_a formed once per class (rest, axis, diagonal), each
  // scaled by omega unless TAU1 (tau = 1: the collision is g* = g_eq + source).
  const F2 om = TAU1 ? F2{1.f, 0.f} : c.omega;
  const F2 wA3 = f2_mul(om, f2_add(kWA, f2_add(kWA, kWA)));
  const F2 wD3 = f2_mul(om, f2_add(kWD, f2_add(kWD, kWD)));
  const F2 r0 = f2_mul(f2_mul(om, kW0), drho);
  const F2 rA = f2_mul(f2_mul(om, kWA), drho);
  const F2 rD = f2_mul(f2_mul(om, kWD), drho);
  const F2 jA[3] = {f2_mul(wA3, jx), f2_mul(wA3, jy), f2_mul(wA3, jz)};
  const F2 jD[3] = {f2_mul(wD3, jx), f2_mul(wD3, jy), f2_mul(wD3, jz)};
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const int n2 = L::ex(i) * L::ex(i) + L::ey(i) * L::ey(i) + L::ez(i) * L::ez(i);
    const F2 *jw = n2 == 1 ? jA : jD;
    F2 geq = i == 0 ? r0 : (n2 == 1 ? rA : rD);
    if (L::ex(i)) geq = f2_add(geq, L::ex(i) > 0 ? jw[0] : f2_neg(jw[0]));
    if (L::ey(i)) geq = f2_add(geq, L::ey(i) > 0 ? jw[1] : f2_neg(jw[1]));
    if (DIM == 3 && L::ez(i)) geq = f2_add(geq, L::ez(i) > 0 ? jw[2] : f2_neg(jw[2]));
    // g* = g + omega (g_eq - g) = (1 - omega) g + [omega g_eq]
    F2 go = TAU1 ? geq : f2_add(f2_mul(c.one_minus_omega, gi[i]), geq);
    if (L::ex(i)) {
      const bool axis = (L::ey(i) == 0 && L::ez(i) == 0);
      const F2 sv = axis ? c.src_axis : c.src_diag;
      go = f2_add(go, L::ex(i) > 0 ? sv : f2_neg(sv));
    }
    int idx;
    const int pl = write_slot<DIM, ODD>(nb, k0, i, idx);
    gh.plane(pl)[idx] = go.h;
    gl.plane(pl)[idx] = go.l;
  }
}

template <int DIM, bool ODD, bool TAU1, typename PL>
__device__ __forceinline__ void lbm_split_body(const PL &gh, const PL &gl, const LinkGeo &lg,
                                               int n, int k0, const SplitConst &c) {
  int nb[Lat<DIM>::Q];
  load_links<DIM, ODD>(lg, k0, n, nb);
  lbm_split_body_nb<DIM, ODD, TAU1>(gh, gl, nb, k0, c);
}

// The pair-storage odd step as a prefetching grid-stride loop (as
// k_lbm_odd_pf).
template <int DIM, bool TAU1, int BS>
__global__ void __launch_bounds__(BS)
    k_lbm_split_odd_pf(Planes<float, Lat<DIM>::Q> gh, Planes<float, Lat<DIM>::Q> gl,
                       LinkGeo lg, int n, SplitConst c) {
  const int stride = gridDim.x * BS;
  int k = blockIdx.x * BS + threadIdx.x;
  if (k >= n) return;
  LinkData<DIM> cur = load_link_data<DIM>(lg, k, n);
  while (true) {
    const int kn = k + stride;
    LinkData<DIM> nxt;
    if (kn < n) nxt = load_link_data<DIM>(lg, kn, n);
    int nb[Lat<DIM>::Q];
    decode_links<DIM>(lg, cur, k, nb);
    lbm_split_body_nb<DIM, true, TAU1>(gh, gl, nb, k, c);
    if (kn >= n) break;
    k = kn;
    cur = nxt;
  }
}

// Blocks that fill every SM with the kernel at block size bs (once per
// kernel; at most one block per bs sites).
template <typename K> int resident_grid(K kernel, int bs, int n) {
  static int blocks = 0;
  if (blocks == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, bs, 0);
    (void)cudaGetLastError();
    blocks = (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
  }
  return std::max(1, std::min(blocks, (n + bs - 1) / bs));
}

// BS threads per block, registers as the compiler sees fit.
template <int DIM, bool ODD, bool TAU1, int BS>
__global__ void __launch_bounds__(BS)
    k_lbm_step_split(Planes<float, Lat<DIM>::Q> gh, Planes<float, Lat<DIM>::Q> gl, LinkGeo lg,
                     int n, SplitConst c) {
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (k0 >= n) return;
  lbm_split_body<DIM, ODD, TAU1>(gh, gl, lg, n, k0, c);
}

// The same step with registers capped so that MINT threads share an SM.
template <int DIM, bool ODD, bool TAU1, int BS, int MINT>
__global__ void __launch_bounds__(BS, MINT / BS)
    k_lbm_step_split_occ(Planes<float, Lat<DIM>::Q> gh, Planes<float, Lat<DIM>::Q> gl,
                         LinkGeo lg, int n, SplitConst c) {
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (k0 >= n) return;
  lbm_split_body<DIM, ODD, TAU1>(gh, gl, lg, n, k0, c);
}

// One member of a batched flow solve: a domain's populations, neighbour data
// and pore-site count; blocks [block0, block0 + ceil(n / kLbmBatchBlock)) of
// the launch are its own.
template <typename S> struct LbmMember {
  S *g;
  float *glo;  // low words (pair storage) or null
  LinkGeo lg;
  int n, block0;
};
constexpr int kLbmBatchBlock = 128;

// One LBM step of every member of a batch in one launch: block b belongs to
// the member whose block range holds it (binary search over the ascending
// block0) and runs that member's sites with the single-run step's body, so
// every member's populations equal those of its own solve bit for bit.
template <typename S, int DIM, bool ODD, int MODE, bool TAU1>
__global__ void __launch_bounds__(kLbmBatchBlock)
    k_lbm_batch(const LbmMember<S> *__restrict__ members, int n_members,
                typename Arith<S>::type omega, typename Arith<S>::type fx_half,
                typename Arith<S>::type fsrc, SplitConst c) {
  int lo = 0, hi = n_members - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (members[mid].block0 <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const LbmMember<S> &m = members[lo];
  const int k0 = ((int)blockIdx.x - m.block0) * kLbmBatchBlock + threadIdx.x;
  if (k0 >= m.n) return;
  if constexpr (MODE == M_SPLIT)
    lbm_split_body<DIM, ODD, TAU1>(Strided<float>{(float *)m.g, m.n},
                                   Strided<float>{m.glo, m.n}, m.lg, m.n, k0, c);
  else
    lbm_body<S, DIM, ODD>(Strided<S>{m.g, m.n}, m.lg, m.n, k0, omega, fx_half, fsrc);
}

// Velocity u = j = sum e_i g_i + F/2 from the natural layout, written to
// uflow (FP64); accumulates ||u - u_prev||^2 and ||u||^2 over pore sites and
// leaves the relative K-lag residual in scal[S_RES].  glo (pair storage only)
// holds the low parts.
template <typename T, int DIM>
__global__ void __launch_bounds__(kRedThreads)
    k_flow_velocity(const T *__restrict__ g, const float *__restrict__ glo,
                    const int *__restrict__ list, int n, double *__restrict__ uflow,
                    long long Nf, double fx_half, double *__restrict__ part,
                    unsigned int *counter, double *scal) {
  using L = Lat<DIM>;
  __shared__ double sm[2 * 32];
  double v[2] = {0.0, 0.0};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const long long s = list[k];  // populations by rank k, velocity by site s
    // every load of the site first (the kernel is latency-bound otherwise:
    // one site per iteration, few resident warps)
    typename Arith<T>::type gv[L::Q];
    float lv[L::Q];
    double uprev[DIM];
#pragma unroll
    for (int i = 0; i < L::Q; i++) gv[i] = widen(g[(size_t)i * n + k]);
#pragma unroll
    for (int i = 0; i < L::Q; i++) lv[i] = 0.f;
    if (glo) {
#pragma unroll
      for (int i = 1; i < L::Q; i++) lv[i] = glo[(size_t)i * n + k];
    }
#pragma unroll
    for (int a = 0; a < DIM; a++) uprev[a] = uflow[(size_t)a * Nf + s];
    double j[3] = {fx_half, 0.0, 0.0};
    if (!std::is_same<T, double>::value) {
      // exact sums of the FP32 values as (sum, error) pairs: the residual
      // resolves changes far below FP32's relative precision, and FP64 adds
      // are slow on this part
      float ms[3] = {0.f, 0.f, 0.f}, mc[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 1; i < L::Q; i++) {
        const float gi = (float)gv[i], li = lv[i];
        if (L::ex(i)) {
          two_sum_acc(L::ex(i) > 0 ? gi : -gi, ms[0], mc[0]);
          mc[0] = __fadd_rn(mc[0], L::ex(i) > 0 ? li : -li);
        }
        if (L::ey(i)) {
          two_sum_acc(L::ey(i) > 0 ? gi : -gi, ms[1], mc[1]);
          mc[1] = __fadd_rn(mc[1], L::ey(i) > 0 ? li : -li);
        }
        if (DIM == 3 && L::ez(i)) {
          two_sum_acc(L::ez(i) > 0 ? gi : -gi, ms[2], mc[2]);
          mc[2] = __fadd_rn(mc[2], L::ez(i) > 0 ? li : -li);
        }
      }
#pragma unroll
      for (int a = 0; a < 3; a++) j[a] += (double)ms[a] + (double)mc[a];
    } else {
#pragma unroll
      for (int i = 0; i < L::Q; i++) {
        const double gi = (double)gv[i];
        j[0] += L::ex(i) * gi;
        j[1] += L::ey(i) * gi;
        if (DIM == 3) j[2] += L::ez(i) * gi;
      }
    }
#pragma unroll
    for (int a = 0; a < DIM; a++) {
      const double d = j[a] - uprev[a];
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

// u_phys = scale * u_lattice at every pore rank of the transport grid
// (component a of rank r at a * n + r); the scale is scal[S_SCALE], or sc_arg
// when scal is null.
template <typename T, int DIM>
__global__ void k_flow_scale(const double *__restrict__ uflow, const int *__restrict__ cells,
                             int n, T *__restrict__ u, int nx, int NX, long long Nf,
                             const double *__restrict__ scal, double sc_arg) {
  const double sc = scal ? scal[S_SCALE] : sc_arg;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const long long P = cells[r];
    const long long row = P / nx;
    const long long s = row * NX + (P - row * nx);
#pragma unroll
    for (int a = 0; a < DIM; a++) u[(size_t)a * n + r] = (T)(sc * uflow[(size_t)a * Nf + s]);
  }
}

// Storage type of the populations per mode.
template <int M> struct ModeT { using T = float; };
template <> struct ModeT<M_F64> { using T = double; };
template <> struct ModeT<M_BF16> { using T = __nv_bfloat16; };

// One even + one odd step.  MINT: 0 registers as the compiler sees fit; > 0
// capped so that MINT threads share an SM; -1 the odd step as the
// prefetching grid-stride kernel.
template <int M, int DIM, int BS, int MINT>
void step_pair_bs(cdi_domain *d, cudaStream_t st, double tau, double force) {
  using T = typename ModeT<M>::T;
  constexpr int Q = Lat<DIM>::Q;
  constexpr int MI = MINT < 0 ? 0 : MINT;
  // one thread per pore site of the flow grid (pore rank)
  const int n = (int)d->n_flow_pore;
  const int grid = (n + BS - 1) / BS;
  const LinkGeo lk{d->d_lf, d->d_ld, d->d_lb, d->d_lovf, d->n_lovf, d->n_ltiles};
  if (M == M_SPLIT) {
    const double fs = (1.0 - 0.5 / tau) * 3.0 * force;
    const SplitConst c{host_pair(1.0 / tau), host_pair(1.0 - 1.0 / tau), host_pair(0.5 * force),
                       host_pair(fs * Lat<DIM>::w(1)),
                       host_pair(fs * (DIM == 2 ? Lat<2>::w(3) : Lat<3>::w(4)))};
    const Planes<float, Q> gh = make_planes<float, Q>((float *)d->d_g, n);
    const Planes<float, Q> gl = make_planes<float, Q>(d->d_glo, n);
    auto pair = [&](auto tau1) {
      constexpr bool T1 = decltype(tau1)::value;
      if constexpr (MI == 0)
        k_lbm_step_split<DIM, false, T1, BS><<<grid, BS, 0, st>>>(gh, gl, lk, n, c);
      else
        k_lbm_step_split_occ<DIM, false, T1, BS, MI><<<grid, BS, 0, st>>>(gh, gl, lk, n, c);
      if constexpr (MINT < 0) {
        auto *kern = k_lbm_split_odd_pf<DIM, T1, BS>;
        kern<<<resident_grid(kern, BS, n), BS, 0, st>>>(gh, gl, lk, n, c);
      } else if constexpr (MI == 0) {
        k_lbm_step_split<DIM, true, T1, BS><<<grid, BS, 0, st>>>(gh, gl, lk, n, c);
      } else {
        k_lbm_step_split_occ<DIM, true, T1, BS, MI><<<grid, BS, 0, st>>>(gh, gl, lk, n, c);
      }
    };
    if (tau == 1.0) pair(std::true_type());
    else pair(std::false_type());
  } else {
    using A = typename Arith<T>::type;
    const A omega = A(1.0 / tau), fxh = A(0.5 * force);
    const A fsrc = A((1.0 - 0.5 / tau) * 3.0 * force);
    const Planes<T, Q> g = make_planes<T, Q>((T *)d->d_g, n);
    k_lbm_step<T, DIM, false, BS, MI><<<grid, BS, 0, st>>>(g, lk, n, omega, fxh, fsrc);
    if constexpr (MINT < 0) {
      auto *kern = k_lbm_odd_pf<T, DIM, BS>;
      kern<<<resident_grid(kern, BS, n), BS, 0, st>>>(g, lk, n, omega, fxh, fsrc);
    } else {
      k_lbm_step<T, DIM, true, BS, MI><<<grid, BS, 0, st>>>(g, lk, n, omega, fxh, fsrc);
    }
  }
}

// One even + one odd step with the domain's block size.
template <int M, int DIM>
void launch_step_pair(cdi_domain *d, cudaStream_t st, double tau, double force) {
  // pair storage: registers capped for 1280 threads per SM; single-word
  // storage: for 1024 (the single-word kernels hold more live values)
  constexpr int OCC = M == M_SPLIT ? 1280 : 1024;
  switch (d->lbm_variant) {
    case 0: step_pair_bs<M, DIM, 64, 0>(d, st, tau, force); break;
    case 2: step_pair_bs<M, DIM, 256, 0>(d, st, tau, force); break;
    case 3: step_pair_bs<M, DIM, 64, OCC>(d, st, tau, force); break;
    case 4: step_pair_bs<M, DIM, 128, OCC>(d, st, tau, force); break;
    case 5: step_pair_bs<M, DIM, 128, -1>(d, st, tau, force); break;
    default: step_pair_bs<M, DIM, 128, 0>(d, st, tau, force); break;
  }
}

// Autotuner: times a few step pairs with each candidate block size on the
// domain's stream and keeps the fastest.  Every block size computes the same
// bits (one thread per site, no cross-thread arithmetic), so the choice only
// changes speed.  Runs once per domain, before its first solve resets the
// populations.
constexpr int kLbmVariantBlock[6] = {64, 128, 256, 64, 128, 128};
template <int M, int DIM>
cdi_status tune_lbm(cdi_domain *d, double tau, double force) {
  // 64, 128 or 256 threads per block, 64 or 128 with registers capped for
  // more resident warps (FP64 storage skips those: too many spills), and 128
  // with the prefetching odd step
  static const int cand_all[] = {0, 1, 2, 5, 3, 4};
  const int n_cand = M == M_F64 ? 4 : 6;
  const uint64_t key = cdi_tune_key(1, DIM, M, 0, d->n_flow_pore, tau == 1.0 ? 1 : 0);
  int known = 0;
  if (cdi_tune_lookup(key, &known)) {
    d->lbm_variant = known;
    d->lbm_block = kLbmVariantBlock[known];
    d->lbm_tuned = true;
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
  for (int ci = 0; ci < n_cand; ci++) {
    const int bs = cand_all[ci];
    d->lbm_variant = bs;
    launch_step_pair<M, DIM>(d, d->stream, tau, force);  // warm-up
    e = cudaEventRecord(a, d->stream);
    for (int k = 0; k < 6 && e == cudaSuccess; k++) launch_step_pair<M, DIM>(d, d->stream, tau, force);
    if (e == cudaSuccess) e = cudaEventRecord(b, d->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) break;
    d->timing.kernel_launches += 14;
    if (ci == 0 || ms < best) {
      best = ms;
      best_bs = bs;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  d->lbm_variant = best_bs;
  d->lbm_block = kLbmVariantBlock[best_bs];
  if (e != cudaSuccess) return cdi_cuda_fail(d, e, "tune flow step");
  d->lbm_tuned = true;
  cdi_tune_store(key, best_bs);
  return CDI_OK;
}

template <int M, int DIM>
cdi_status launch_velocity(cdi_domain *d, cudaStream_t st = nullptr) {
  using T = typename ModeT<M>::T;
  if (!st) st = d->stream;
  k_flow_velocity<T, DIM><<<kRedBlocks, kRedThreads, 0, st>>>(
      (const T *)d->d_g, M == M_SPLIT ? d->d_glo : nullptr, d->d_flow_list,
      (int)d->n_flow_pore, d->d_uflow, d->Nf, 0.5 * d->force, d->d_part, d->d_counter + C_RES,
      d->d_scal);
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "velocity kernel");
  return CDI_OK;
}

template <int M, int DIM>
cdi_status flow_run(cdi_domain *d, const cdi_flow_params *p, int64_t *steps_out,
                    double *res_out) {
  using T = typename ModeT<M>::T;
  const int K = p->check_every;
  d->tau = p->tau;
  d->force = p->force_lu;
  const int Q = Lat<DIM>::Q;
  if (!d->lbm_tuned) {
    cdi_status ts = tune_lbm<M, DIM>(d, p->tau, p->force_lu);
    if (ts != CDI_OK) return ts;
  }
  // start from rest: g = 0 (f = w), u_prev = u(0)
  const size_t nq = (size_t)Q * d->n_flow_pore;
  CDI_TRY(d, cudaMemsetAsync(d->d_g, 0, nq * sizeof(T), d->stream), "reset g");
  if (M == M_SPLIT)
    CDI_TRY(d, cudaMemsetAsync(d->d_glo, 0, nq * sizeof(float), d->stream), "reset g low parts");
  cdi_status s = launch_velocity<M, DIM>(d);
  if (s != CDI_OK) return s;
  // K steps captured once as a graph (parameters are baked in)
  if (!d->flow_graph || d->flow_graph_K != K || d->flow_graph_tau != p->tau ||
      d->flow_graph_force != p->force_lu) {
    if (d->flow_graph) cudaGraphExecDestroy(d->flow_graph);
    d->flow_graph = nullptr;
    cudaGraph_t graph;
    CDI_TRY(d, cudaStreamBeginCapture(d->cap_stream, cudaStreamCaptureModeThreadLocal),
            "begin capture");
    for (int k = 0; k < K / 2; k++) launch_step_pair<M, DIM>(d, d->cap_stream, p->tau, p->force_lu);
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
    s = launch_velocity<M, DIM>(d);
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

// Batched solve: every active member advances in one launch per step (K
// steps per captured graph on the lead's stream); after each block of K
// steps each member's residual is taken exactly as in its own solve, and a
// member that has converged leaves the batch (its populations then stay as
// its own solve would leave them).
template <int M, int DIM>
cdi_status flow_batch(cdi_domain *const *doms, int n_doms, const cdi_flow_params *p,
                      int64_t *steps_out, double *res_out, int *status_out) {
  using S = typename ModeT<M>::T;
  using A = typename Arith<S>::type;
  cdi_domain *L = doms[0];
  const int K = p->check_every;
  const int Q = Lat<DIM>::Q;
  const double tau = p->tau, force = p->force_lu;
  const A omega = A(1.0 / tau), fxh = A(0.5 * force), fsrc = A((1.0 - 0.5 / tau) * 3.0 * force);
  const double fs = (1.0 - 0.5 / tau) * 3.0 * force;
  const SplitConst c{host_pair(1.0 / tau), host_pair(1.0 - 1.0 / tau), host_pair(0.5 * force),
                     host_pair(fs * Lat<DIM>::w(1)),
                     host_pair(fs * (DIM == 2 ? Lat<2>::w(3) : Lat<3>::w(4)))};
  LbmMember<S> *dtab = (LbmMember<S> *)cdi_dev_alloc(L, sizeof(LbmMember<S>) * n_doms);
  if (!dtab) return cdi_fail(L, CDI_ERR_OOM, "flow batch: member table");
  std::vector<LbmMember<S>> tab;
  std::vector<int> active(n_doms);
  cdi_status s = CDI_OK;
  for (int i = 0; i < n_doms; i++) {
    cdi_domain *d = doms[i];
    active[i] = i;
    steps_out[i] = 0;
    res_out[i] = NAN;
    status_out[i] = CDI_ERR_NOT_CONVERGED;
    d->tau = tau;
    d->force = force;
    if (!d->lbm_tuned) {  // the single solve's block size: kept for later solves
      s = tune_lbm<M, DIM>(d, tau, force);
      if (s != CDI_OK) break;
    }
  }
  auto chk = [&](cudaError_t e, const char *what) {
    if (s == CDI_OK && e != cudaSuccess) s = cdi_cuda_fail(L, e, what);
  };
  // start from rest on the lead's stream (each domain's memory is ready:
  // domains synchronise their streams when created)
  for (int i = 0; i < n_doms && s == CDI_OK; i++) {
    cdi_domain *d = doms[i];
    chk(cudaStreamSynchronize(d->stream), "flow batch: member stream");
    const size_t nq = (size_t)Q * d->n_flow_pore;
    chk(cudaMemsetAsync(d->d_g, 0, nq * sizeof(S), L->stream), "flow batch: reset");
    if (M == M_SPLIT) chk(cudaMemsetAsync(d->d_glo, 0, nq * 4, L->stream), "flow batch: reset");
    if (s == CDI_OK) s = launch_velocity<M, DIM>(d, L->stream);
  }
  cudaGraphExec_t exec = nullptr;
  auto rebuild = [&]() {
    tab.clear();
    int blocks = 0;
    for (int i : active) {
      cdi_domain *d = doms[i];
      LbmMember<S> m;
      m.g = (S *)d->d_g;
      m.glo = d->d_glo;
      m.lg = LinkGeo{d->d_lf, d->d_ld, d->d_lb, d->d_lovf, d->n_lovf, d->n_ltiles};
      m.n = (int)d->n_flow_pore;
      m.block0 = blocks;
      blocks += (m.n + kLbmBatchBlock - 1) / kLbmBatchBlock;
      tab.push_back(m);
    }
    chk(cudaMemcpyAsync(dtab, tab.data(), sizeof(LbmMember<S>) * tab.size(),
                        cudaMemcpyHostToDevice, L->stream), "flow batch: member table");
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    if (s != CDI_OK) return;
    cudaGraph_t graph;
    chk(cudaStreamBeginCapture(L->cap_stream, cudaStreamCaptureModeThreadLocal), "capture");
    if (s != CDI_OK) return;
    const int nm = (int)tab.size();
    for (int k = 0; k < K / 2; k++) {
      const bool t1 = M == M_SPLIT && tau == 1.0;
      if (t1) {
        k_lbm_batch<S, DIM, false, M, true><<<blocks, kLbmBatchBlock, 0, L->cap_stream>>>(
            dtab, nm, omega, fxh, fsrc, c);
        k_lbm_batch<S, DIM, true, M, true><<<blocks, kLbmBatchBlock, 0, L->cap_stream>>>(
            dtab, nm, omega, fxh, fsrc, c);
      } else {
        k_lbm_batch<S, DIM, false, M, false><<<blocks, kLbmBatchBlock, 0, L->cap_stream>>>(
            dtab, nm, omega, fxh, fsrc, c);
        k_lbm_batch<S, DIM, true, M, false><<<blocks, kLbmBatchBlock, 0, L->cap_stream>>>(
            dtab, nm, omega, fxh, fsrc, c);
      }
    }
    cudaError_t e = cudaStreamEndCapture(L->cap_stream, &graph);
    chk(e, "end capture");
    if (e == cudaSuccess) {
      chk(cudaGraphInstantiate(&exec, graph, 0), "instantiate flow batch graph");
      cudaGraphDestroy(graph);
    }
  };
  if (s == CDI_OK && p->max_steps > 0) rebuild();
  int64_t steps = 0;
  while (s == CDI_OK && !active.empty() && steps < p->max_steps) {
    cudaEvent_t a;
    cdi_timing_begin(L, &a);
    chk(cudaGraphLaunch(exec, L->stream), "flow batch graph");
    cdi_timing_end(L, a, PH_FLOW, K);
    L->timing.kernel_launches += K;
    steps += K;
    cdi_timing_begin(L, &a);
    for (int i : active) {
      cdi_domain *d = doms[i];
      if (s == CDI_OK) s = launch_velocity<M, DIM>(d, L->stream);
      chk(cudaMemcpyAsync(d->h_scal + S_RES_NUM, d->d_scal + S_RES_NUM, 3 * sizeof(double),
                          cudaMemcpyDeviceToHost, L->stream), "residual copy");
    }
    cdi_timing_end(L, a, PH_CHECK, (int64_t)active.size());
    chk(cudaStreamSynchronize(L->stream), "flow batch chunk");
    if (s != CDI_OK) break;
    std::vector<int> still;
    for (int i : active) {
      const double r = doms[i]->h_scal[S_RES];
      steps_out[i] = steps;
      res_out[i] = r;
      if (!std::isfinite(r)) {
        status_out[i] = CDI_ERR_CUDA;   // diverged: leaves the batch
      } else if (p->tol > 0.0 && r < p->tol) {
        status_out[i] = CDI_OK;
      } else {
        still.push_back(i);
      }
    }
    if (still.size() != active.size()) {
      active = still;
      if (!active.empty()) rebuild();
    }
  }
  if (p->tol <= 0.0)
    for (int i = 0; i < n_doms; i++)
      if (status_out[i] == CDI_ERR_NOT_CONVERGED) status_out[i] = CDI_OK;
  if (p->max_steps == 0)
    for (int i = 0; i < n_doms; i++) res_out[i] = doms[i]->h_scal[S_RES];
  cudaStreamSynchronize(L->stream);
  if (exec) cudaGraphExecDestroy(exec);
  cdi_dev_release(L, dtab);
  if (s == CDI_OK) {
    cudaError_t e = cdi_timing_resolve(L);
    if (e != cudaSuccess) s = cdi_cuda_fail(L, e, "timing");
  }
  for (int i = 0; i < n_doms; i++) {
    doms[i]->flow_steps = steps_out[i];
    doms[i]->flow_residual = res_out[i];
  }
  return s;
}

template <typename T, int DIM>
cdi_status flow_export(cdi_domain *d, double U_target) {
  k_flow_mean<<<kRedBlocks, kRedThreads, 0, d->stream>>>(
      d->d_uflow, d->d_mask, d->nx, d->NX, d->N, (double)d->n_pore, U_target, d->d_part,
      d->d_counter + C_ULAT, d->d_scal);
  k_flow_scale<T, DIM><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
      d->d_uflow, d->d_cell_list, (int)d->n_pore, (T *)d->d_u, d->nx, d->NX, d->Nf, d->d_scal,
      0.0);
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

int cdi_lbm_shape_block(int v) { return v >= 0 && v < 6 ? kLbmVariantBlock[v] : 0; }

cdi_status cdi_flow_build_flags(cdi_domain *d) {
  return d->dim == 2 ? build_flags<2>(d) : build_flags<3>(d);
}

// Neighbour data of the compact population layout (after the pore lists):
// rank[site] scattered from the list (rank_work: Nf ints, -1 for solid), then
// the flag words, row-base bytes and tile bases of every pore rank; then the
// overflow table, sized by the sites that need it, is taken and filled.
cdi_status cdi_flow_build_links(cdi_domain *d, int *rank_work) {
  const int n = (int)d->n_flow_pore;
  const int Q = d->dim == 2 ? 9 : 19;
  unsigned *n_extra = d->d_counter + C_LINK;
  CDI_TRY(d, cudaMemsetAsync(rank_work, 0xff, (size_t)d->Nf * sizeof(int), d->stream),
          "rank reset");
  CDI_TRY(d, cudaMemsetAsync(n_extra, 0, sizeof(unsigned), d->stream), "overflow count reset");
  k_rank_scatter<<<kRedBlocks, kRedThreads, 0, d->stream>>>(d->d_flow_list, n, rank_work);
  if (d->dim == 2)
    k_links<2><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        (const FlowFlag<2>::type *)d->d_fflags, d->d_flow_list, n, rank_work, d->d_lf, d->d_ld,
        d->d_lb, d->n_ltiles, n_extra, d->NX, d->ny, d->nz, d->walls);
  else
    k_links<3><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        (const FlowFlag<3>::type *)d->d_fflags, d->d_flow_list, n, rank_work, d->d_lf, d->d_ld,
        d->d_lb, d->n_ltiles, n_extra, d->NX, d->ny, d->nz, d->walls);
  CDI_TRY(d, cudaGetLastError(), "neighbour data");
  unsigned extra = 0;
  CDI_TRY(d, cudaMemcpyAsync(&extra, n_extra, sizeof(unsigned), cudaMemcpyDeviceToHost,
                             d->stream), "overflow count");
  CDI_TRY(d, cudaStreamSynchronize(d->stream), "overflow count");
  d->n_lovf = 2 * d->ny * d->nz + (int)extra;
  d->d_lovf = (int *)cdi_dev_alloc(d, (size_t)(Q - 1) * d->n_lovf * sizeof(int));
  if (!d->d_lovf) return cdi_fail(d, CDI_ERR_OOM, "neighbour overflow table");
  CDI_TRY(d, cudaMemsetAsync(d->d_lovf, 0xff, (size_t)(Q - 1) * d->n_lovf * sizeof(int),
                             d->stream), "overflow reset");
  if (d->dim == 2)
    k_links_ovf<2><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        (const FlowFlag<2>::type *)d->d_fflags, d->d_flow_list, n, rank_work, d->d_lf, d->d_ld,
        d->d_lovf, d->n_lovf, d->NX, d->ny, d->nz);
  else
    k_links_ovf<3><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
        (const FlowFlag<3>::type *)d->d_fflags, d->d_flow_list, n, rank_work, d->d_lf, d->d_ld,
        d->d_lovf, d->n_lovf, d->NX, d->ny, d->nz);
  d->timing.kernel_launches += 3;
  CDI_TRY(d, cudaGetLastError(), "neighbour overflow table");
  return CDI_OK;
}

cdi_status cdi_flow_run(cdi_domain *d, const cdi_flow_params *p, int64_t *steps, double *res) {
  switch (d->prec) {
    case CDI_FP64:
      return d->dim == 2 ? flow_run<M_F64, 2>(d, p, steps, res) : flow_run<M_F64, 3>(d, p, steps, res);
    case CDI_FP32:
    case CDI_FP32_CPAIR:
      return d->dim == 2 ? flow_run<M_F32, 2>(d, p, steps, res) : flow_run<M_F32, 3>(d, p, steps, res);
    case CDI_BF16_POP:
      return d->dim == 2 ? flow_run<M_BF16, 2>(d, p, steps, res)
                         : flow_run<M_BF16, 3>(d, p, steps, res);
    default:
      return d->dim == 2 ? flow_run<M_SPLIT, 2>(d, p, steps, res)
                         : flow_run<M_SPLIT, 3>(d, p, steps, res);
  }
}

cdi_status cdi_flow_batch(cdi_domain *const *doms, int n_doms, const cdi_flow_params *p,
                          int64_t *steps, double *res, int *status) {
  const cdi_domain *d = doms[0];
  switch (d->prec) {
    case CDI_FP64:
      return d->dim == 2 ? flow_batch<M_F64, 2>(doms, n_doms, p, steps, res, status)
                         : flow_batch<M_F64, 3>(doms, n_doms, p, steps, res, status);
    case CDI_FP32:
    case CDI_FP32_CPAIR:
      return d->dim == 2 ? flow_batch<M_F32, 2>(doms, n_doms, p, steps, res, status)
                         : flow_batch<M_F32, 3>(doms, n_doms, p, steps, res, status);
    case CDI_BF16_POP:
      return d->dim == 2 ? flow_batch<M_BF16, 2>(doms, n_doms, p, steps, res, status)
                         : flow_batch<M_BF16, 3>(doms, n_doms, p, steps, res, status);
    default:
      return d->dim == 2 ? flow_batch<M_SPLIT, 2>(doms, n_doms, p, steps, res, status)
                         : flow_batch<M_SPLIT, 3>(doms, n_doms, p, steps, res, status);
  }
}

cdi_status cdi_flow_scale_to(cdi_domain *d, double scale, void *dst) {
  if (d->prec == CDI_FP64) {
    if (d->dim == 2)
      k_flow_scale<double, 2><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
          d->d_uflow, d->d_cell_list, (int)d->n_pore, (double *)dst, d->nx, d->NX, d->Nf, nullptr,
          scale);
    else
      k_flow_scale<double, 3><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
          d->d_uflow, d->d_cell_list, (int)d->n_pore, (double *)dst, d->nx, d->NX, d->Nf, nullptr,
          scale);
  } else {
    if (d->dim == 2)
      k_flow_scale<float, 2><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
          d->d_uflow, d->d_cell_list, (int)d->n_pore, (float *)dst, d->nx, d->NX, d->Nf, nullptr,
          scale);
    else
      k_flow_scale<float, 3><<<kRedBlocks, kRedThreads, 0, d->stream>>>(
          d->d_uflow, d->d_cell_list, (int)d->n_pore, (float *)dst, d->nx, d->NX, d->Nf, nullptr,
          scale);
  }
  d->timing.kernel_launches++;
  CDI_TRY(d, cudaGetLastError(), "velocity scale");
  return CDI_OK;
}

cdi_status cdi_flow_export(cdi_domain *d, double U_target) {
  if (d->prec == CDI_FP64)
    return d->dim == 2 ? flow_export<double, 2>(d, U_target) : flow_export<double, 3>(d, U_target);
  return d->dim == 2 ? flow_export<float, 2>(d, U_target) : flow_export<float, 3>(d, U_target);
}
