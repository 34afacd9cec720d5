// Internal declarations of the GB300 CDI library: the domain object, device
// helpers shared by the kernels, and the lattice tables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cdi.h"

namespace cdi {

constexpr int kMaxSpecies = 4;
constexpr int kRowBlock = 128;      // threads per block along x for stencils
constexpr int kRedThreads = 256;    // threads per block for reductions
constexpr int kRedBlocks = 4 * 152; // fixed grid of the grid-stride reductions

// ---------------------------------------------------------------------------
// Lattices (D2Q9 and D3Q19 of Sec. 2).  Direction i and its opposite are
// paired as i <-> i + (Q-1)/2 so that opp() is arithmetic.
// ---------------------------------------------------------------------------
template <int DIM> struct Lat;

template <> struct Lat<2> {
  static constexpr int Q = 9;
  static constexpr int H = 4;
  __host__ __device__ static constexpr int ex(int i) {
    return i == 1 || i == 3 || i == 8 ? 1 : (i == 4 || i == 5 || i == 7 ? -1 : 0);
  }
  __host__ __device__ static constexpr int ey(int i) {
    return i == 2 || i == 3 || i == 4 ? 1 : (i == 6 || i == 7 || i == 8 ? -1 : 0);
  }
  __host__ __device__ static constexpr int ez(int) { return 0; }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : ((ex(i) * ex(i) + ey(i) * ey(i)) == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= H ? i + H : i - H);
  }
};

template <> struct Lat<3> {
  static constexpr int Q = 19;
  static constexpr int H = 9;
  // 1:(1,0,0) 2:(0,1,0) 3:(0,0,1) 4:(1,1,0) 5:(1,-1,0) 6:(1,0,1) 7:(1,0,-1)
  // 8:(0,1,1) 9:(0,1,-1); 10..18 are their negatives.
  __host__ __device__ static constexpr int bx(int k) {
    return k == 1 || k == 4 || k == 5 || k == 6 || k == 7 ? 1 : 0;
  }
  __host__ __device__ static constexpr int by(int k) {
    return k == 2 || k == 4 || k == 8 || k == 9 ? 1 : (k == 5 ? -1 : 0);
  }
  __host__ __device__ static constexpr int bz(int k) {
    return k == 3 || k == 6 || k == 8 ? 1 : (k == 7 || k == 9 ? -1 : 0);
  }
  __host__ __device__ static constexpr int ex(int i) {
    return i == 0 ? 0 : (i <= H ? bx(i) : -bx(i - H));
  }
  __host__ __device__ static constexpr int ey(int i) {
    return i == 0 ? 0 : (i <= H ? by(i) : -by(i - H));
  }
  __host__ __device__ static constexpr int ez(int i) {
    return i == 0 ? 0 : (i <= H ? bz(i) : -bz(i - H));
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0
                  : ((ex(i) * ex(i) + ey(i) * ey(i) + ez(i) * ez(i)) == 1 ? 1.0 / 18.0
                                                                         : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= H ? i + H : i - H);
  }
};

// Flow-site flag word: bit 0 = the site is solid; bit i (1..Q-1) = the
// neighbour along e_i is solid or lies beyond a lateral wall; bits Q..Q+5 =
// the site lies on the high/low x, y, z edge of the flow grid, where the
// periodic neighbour offsets wrap around.
template <int DIM> struct FlowFlag;
template <> struct FlowFlag<2> { using type = uint16_t; };
template <> struct FlowFlag<3> { using type = uint32_t; };
template <int DIM> struct WrapBit {
  static constexpr int XHI = Lat<DIM>::Q, XLO = XHI + 1, YHI = XHI + 2, YLO = XHI + 3,
                       ZHI = XHI + 4, ZLO = XHI + 5;
};

// Transport-cell flag word: bit 0 = solid; bit 1 + f = the neighbour across
// face f (f = +x,-x,+y,-y,+z,-z) is a solid voxel inside the image (after the
// periodic wrap); bit 7 + f = face f lies on the image boundary.
using NFlag = uint16_t;
constexpr int kFaceBit = 1;
constexpr int kEdgeBit = 7;

// ---------------------------------------------------------------------------
// Deterministic block reductions (fixed order, no floating-point atomics).
// ---------------------------------------------------------------------------
template <int NV, typename V, typename Op>
__device__ __forceinline__ void warp_reduce(V (&v)[NV], Op op) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = op(v[k], __shfl_down_sync(0xffffffffu, v[k], o));
}

struct OpSum {
  template <typename V> __device__ V operator()(V a, V b) const { return a + b; }
};
struct OpMax {
  template <typename V> __device__ V operator()(V a, V b) const { return a > b ? a : b; }
};

// Reduces v over the block; the result is valid in thread 0.  smem must hold
// NV * 32 values.  All threads of the block must call it.
template <int NV, typename V, typename Op>
__device__ __forceinline__ void block_reduce(V (&v)[NV], V *smem, Op op, V identity) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  warp_reduce<NV>(v, op);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; k++) smem[k * 32 + w] = v[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = lane < nw ? smem[k * 32 + lane] : identity;
    warp_reduce<NV>(v, op);
  }
  __syncthreads();
}

// Called by every thread after the block wrote its partials: returns true in
// the last block to finish (which then combines all partials in a fixed
// order and must reset *counter to 0).
__device__ __forceinline__ bool last_block(unsigned int *counter, int nblocks) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == (unsigned)(nblocks - 1));
  __syncthreads();
  return am_last;
}

// Sums partials[k * nblocks + b] over b for each k (fixed order) in the last
// block; the result lands in thread 0's v.
template <int NV, typename Op>
__device__ __forceinline__ void combine_partials(const double *partials, int nblocks,
                                                 double (&v)[NV], double *smem, Op op,
                                                 double identity) {
#pragma unroll
  for (int k = 0; k < NV; k++) v[k] = identity;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = op(v[k], __ldcg(partials + (size_t)k * nblocks + b));
  block_reduce<NV>(v, smem, op, identity);
}

// psi / V_T as stored for the transport kernel: FP64, or an unevaluated
// FP32 pair hi + lo (so that face differences keep FP64-like accuracy while
// the arithmetic stays on the FP32 units).
template <typename T> struct PhiStore;
template <> struct PhiStore<double> {
  using type = double;
  __device__ static double make(double v) { return v; }
  __device__ static double zero() { return 0.0; }
};
template <> struct PhiStore<float> {
  using type = float2;
  __device__ static float2 make(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
  }
  __device__ static float2 zero() { return make_float2(0.f, 0.f); }
};

// Arithmetic with explicit rounding (never contracted into FMAs by the
// compiler, so two kernels that inline the same function compute the same
// bits).
__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double r_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float r_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Bernoulli function pair B(x), B(-x) with B(x) = x / (exp(x) - 1), from one
// expm1 of |x|: B(|x|) directly (series near 0) and B(-|x|) = B(|x|) + |x|,
// both positive so neither loses precision.
template <typename T>
__device__ __forceinline__ void bernoulli_pair(T x, T &Bx, T &Bmx) {
  const T a = fabs(x);
  T Ba;
  if (a < T(1e-3)) {
    // 1 - a/2 + a^2/12 - a^4/720
    const T a2 = r_mul(a, a);
    Ba = r_fma(a2, r_fma(a2, T(-1) / T(720), T(1) / T(12)), r_fma(a, T(-0.5), T(1)));
  } else {
    Ba = a / expm1(a);
  }
  const T Bma = r_add(Ba, a);
  if (x >= T(0)) {
    Bx = Ba;
    Bmx = Bma;
  } else {
    Bx = Bma;
    Bmx = Ba;
  }
}

}  // namespace cdi

// ---------------------------------------------------------------------------
// The domain object behind the opaque handle.
// ---------------------------------------------------------------------------
struct cdi_domain {
  // geometry
  int dim = 2, nx = 0, ny = 0, nz = 1, walls = 0, mirror = 1, prec = CDI_FP64;
  double dx = 1e-7;
  int NX = 0;         // flow-grid extent along x (2 nx with the mirror)
  long long N = 0;    // transport cells nx*ny*nz
  long long Nf = 0;   // flow sites NX*ny*nz
  long long n_pore = 0, n_pore_inlet = 0;
  uint64_t mask_hash = 0;  // FNV-1a of the mask bytes (identifies a saved state's geometry)

  // execution
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t cap_stream = nullptr;  // private stream used only for capture
  cdi_allocator alloc{};
  bool has_alloc = false;
  std::string err;
  struct Block {
    void *p;
    size_t bytes;
  };
  std::vector<Block> blocks;

  // device buffers
  uint8_t *d_mask = nullptr;    // N
  void *d_fflags = nullptr;     // Nf flow flags
  cdi::NFlag *d_nflags = nullptr;  // N face flags
  int *d_flow_list = nullptr;   // pore sites of the flow grid, ascending
  long long n_flow_pore = 0;
  // neighbour data of the odd LBM step (see flow.cu): per pore rank a flag
  // word and one signed byte per lateral row offset (the offset's rank base
  // less the rank and the base of the rank's 32-rank tile); per tile the
  // bases; full neighbour ranks of the x-edge sites and of the sites whose
  // bytes overflow in a table of n_lovf = 2 ny nz + (those sites) slots
  unsigned *d_lf = nullptr;     // n_flow_pore
  unsigned *d_ld = nullptr;     // (1 in 2D, 2 in 3D) words * n_flow_pore
  int *d_lb = nullptr;          // (2 in 2D, 8 in 3D) * n_ltiles
  int n_ltiles = 0;             // ceil(n_flow_pore / 32)
  int *d_lovf = nullptr;        // (Q-1) * n_lovf
  int n_lovf = 0;
  int *d_cell_list = nullptr;   // pore cells of the transport grid, ascending:
                                // entry r is the lattice cell of pore rank r
  uint2 *d_cmeta = nullptr;     // n_pore: {face flags | x << 16, row = z*ny + y}
  cdi::NFlag *d_cfl = nullptr;  // n_pore: face flags alone (read by the FP32 step)
  uint2 *d_words = nullptr;     // ny*nz*W: per 32 cells of a row {rank of the
                                // first pore cell at or after it, pore bits}
  int W = 0;                    // words per row, ceil(nx / 32)
  int *d_latnb = nullptr;       // 2*(dim-1)*n_pore lateral neighbour ranks (-1: none)
  void *d_g = nullptr;          // Q*n_flow_pore populations (shifted) by pore rank
  float *d_glo = nullptr;       // their low parts (pair storage only)
  double *d_uflow = nullptr;    // dim*Nf lattice velocity (last check), FP64
  // transport fields by pore rank (component a / species k of rank r at
  // a * n_pore + r)
  void *d_u = nullptr;          // dim*n_pore scaled velocity, precision T
  double *d_psi = nullptr;      // N potential (V), FP64, lattice order
  void *d_phi = nullptr;        // n_pore psi / V_T, 8 bytes a cell: double
                                // (FP64) or a float2 (hi, lo) pair (FP32)
  bool cpair = false;           // concentrations stored as FP32 pairs (hi + lo)
  float *d_Clo[2] = {nullptr, nullptr};  // their low words (pair storage only)
  void *d_C[2] = {nullptr, nullptr};  // kMaxSpecies*n_pore concentrations,
                                      // ping-pong, T
  double *d_acc = nullptr;      // 3*kMaxSpecies*np_accs per-warp sums (8 B each:
                                // FP64, or an FP32 pair in FP32 modes)
  double *d_part = nullptr;     // reduction partials (8*kRedBlocks)
  unsigned int *d_counter = nullptr;  // last-block counters (8 slots)
  double *d_scal = nullptr;     // device scalars (S_COUNT)
  double *h_scal = nullptr;     // pinned host copy of the scalars (S_COUNT)
  double *d_cg = nullptr;       // 4*N CG work vectors (r, p, q, diag)
  double *d_colout = nullptr;   // nx column means

  // state
  bool flow_done = false, psi_done = false, np_ready = false;
  int64_t flow_steps = 0;
  double flow_residual = 0.0;
  double U_lat = 0.0;           // pore-mean lattice x velocity
  double U_target = 0.0;
  double tau = 1.0, force = 0.0;
  int ns = 0;
  int z[cdi::kMaxSpecies] = {0, 0, 0, 0};
  double D[cdi::kMaxSpecies] = {0, 0, 0, 0};
  double c0 = 0.0, Ka = 0.0, dt = 0.0, VT = 0.0;
  // potential parameters of the last cdi_set_potential (for the coupled
  // re-solve) and the coupling period (0: frozen potential)
  double psi_s = 0.0, eps_r = 78.5, psi_tol = 1e-12;
  int psi_max_iter = 100000;
  int64_t couple_K = 0;
  // implicit (backward Euler) transport: on when imp_tol > 0
  double imp_tol = 0.0;
  int imp_max_iter = 0;
  bool imp_stale = true;        // the operator must be rebuilt before a step
  int64_t imp_iters = 0;        // linear iterations so far
  double imp_last_rel = 0.0;    // last relative residual
  double *d_icoef = nullptr;    // operator coefficients of every species (FP64)
  double *d_iwork = nullptr;    // 7 * n_pore FP64 work vectors
  double *d_iscal = nullptr;    // the solver's device scalars (16)
  double *d_src = nullptr;      // N charge terms of Eq. 4 (coupled mode only)
  int cur = 0;                  // which of d_C holds the current state
  int64_t np_steps = 0;
  int np_blocks = 0;            // 128-thread blocks of the fused sweep/batch
                                // steps (FP64: one thread per pore cell; FP32:
                                // warps of 31 home cells)
  int np_accs = 0;              // account sets, one per warp (rounded up to a
                                // multiple of 8: enough for any launch shape)
  // block sizes of the step kernels, picked by the autotuners
  int lbm_block = 128, np_block = 128;
  int np_variant = 1;           // transport launch shape (see tune_np)
  int lbm_variant = 1;          // LBM launch shape (see tune_lbm)
  bool lbm_tuned = false, np_tuned = false;

  // graphs
  cudaGraphExec_t flow_graph = nullptr;
  int flow_graph_K = 0;
  double flow_graph_tau = 0.0, flow_graph_force = 0.0;
  cudaGraphExec_t np_graph = nullptr;
  int np_graph_steps = 0;

  // timing
  struct EvPair {
    cudaEvent_t a, b;
    int phase;
    int64_t launches;
  };
  std::vector<EvPair> pending;
  std::vector<cudaEvent_t> ev_pool;
  cdi_timing timing{};
};

// Scalar slots in d_scal / h_scal.
enum {
  S_RES_NUM = 0, S_RES_DEN = 1, S_RES = 2,  // flow residual
  S_ULAT = 3, S_SCALE = 4,                  // velocity export
  S_CG_RZ = 8, S_CG_PQ = 9, S_CG_ALPHA = 10, S_CG_BETA = 11, S_CG_RR = 12,
  S_CG_BB = 13, S_CG_REL = 14, S_CG_DONE = 15, S_CG_TOL = 16, S_CG_IT = 17,
  S_PB_FF = 18, S_PB_BB = 19,               // Poisson-Boltzmann Newton residual
  S_RATE = 20, S_DT = 21,                   // time step
  S_OUT = 24,                               // 2*kMaxSpecies: outlet sums
  S_MASS = 32,                              // kMaxSpecies
  S_OUTP = 36,                              // kMaxSpecies: plain outlet sums
  S_ACC = 40,                               // 3*kMaxSpecies: Gamma/In/Out sums
  S_OUTN = 52,                              // pore cells in the outlet column
  S_GEOM = 56,                              // pore cells, pore-solid faces, sum u_x
  S_IMP = 64,                               // 16: the implicit solver's scalars (host copy)
  S_COUNT = 80                              // slots in d_scal / h_scal
};

// Counter slots in d_counter.
enum { C_RES = 0, C_ULAT = 1, C_CG1 = 2, C_CG2 = 3, C_DT = 4, C_OUT = 5, C_MASS = 6, C_ACC = 7,
       C_GEOM = 8, C_IMP = 9, C_LINK = 10 };

enum { PH_FLOW = 0, PH_CHECK = 1, PH_PSI = 2, PH_NP = 3 };

// Host helpers (api.cu).
cdi_status cdi_fail(cdi_domain *d, cdi_status s, const std::string &msg);
cdi_status cdi_cuda_fail(cdi_domain *d, cudaError_t e, const char *what);
void *cdi_dev_alloc(cdi_domain *d, size_t bytes);
void cdi_timing_begin(cdi_domain *d, cudaEvent_t *a);
void cdi_timing_end(cdi_domain *d, cudaEvent_t a, int phase, int64_t launches);
cudaError_t cdi_timing_resolve(cdi_domain *d);

// Process-wide memory of the autotuners' choices, keyed by the kernel kind,
// lattice, storage precision, species count, problem size and device: a
// second domain of the same size runs the kernels the first one picked (so
// repeated solves time the same code) without re-timing them.
uint64_t cdi_tune_key(int kind, int dim, int prec, int ns, long long n, int extra);
bool cdi_tune_lookup(uint64_t key, int *variant);
void cdi_tune_store(uint64_t key, int variant);

#define CDI_TRY(d, call, what)                           \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cdi_cuda_fail(d, e_, what); \
  } while (0)

// Kernel-side entry points used by the API layer.
cdi_status cdi_flow_build_flags(cdi_domain *d);
size_t cdi_lists_work_ints(long long n);
cdi_status cdi_flow_build_links(cdi_domain *d, int *rank_work);
cdi_status cdi_build_lists(cdi_domain *d, int *work);
cdi_status cdi_flow_run(cdi_domain *d, const cdi_flow_params *p, int64_t *steps,
                        double *res);
cdi_status cdi_flow_export(cdi_domain *d, double U_target);
cdi_status cdi_flow_batch(cdi_domain *const *doms, int n_doms, const cdi_flow_params *p,
                          int64_t *steps, double *res, int *status);
cdi_status cdi_flow_velocity_lattice(cdi_domain *d);
cdi_status cdi_psi_solve(cdi_domain *d, double psi_s, double kdx2, const double *src,
                         double tol, int max_iter, int *iters, double *relres);
cdi_status cdi_psi_coupled(cdi_domain *d);
cdi_status cdi_np_build_flags(cdi_domain *d);
cdi_status cdi_np_build_compact(cdi_domain *d);
cdi_status cdi_np_scatter(cdi_domain *d, const void *src, const float *lo, int comps,
                          double *dst);
cdi_status cdi_np_init(cdi_domain *d, double dt_s, double *dt_used);
cdi_status cdi_np_dt(cdi_domain *d, double scale, double *dt_out);
cdi_status cdi_np_geometry(cdi_domain *d, double *pores, double *faces, double *sum_ux);
cdi_status cdi_np_sweep(cdi_domain *d, int n, const double *scale, const int *group,
                        void *const *phi_groups, const double *dts, int64_t n_steps,
                        double *gamma, double *cout);
cdi_status cdi_np_batch(cdi_domain *const *doms, int n_doms, int n_combos, const double *scale,
                        const int *group, void *const *phis, const double *dts, int64_t n_steps,
                        double *gamma, double *cout);
cdi_status cdi_flow_scale_to(cdi_domain *d, double scale, void *dst);
void cdi_dev_release(cdi_domain *d, void *p);
cdi_status cdi_np_steps(cdi_domain *d, int64_t n);
cdi_status cdi_np_reduce(cdi_domain *d);
cdi_status cdi_np_column_means(cdi_domain *d, int species);
cdi_status cdi_imp_prepare(cdi_domain *d);
// Nonlinear Poisson-Boltzmann potential (Newton around the device CG).
cdi_status cdi_psi_pb(cdi_domain *d, double psi_s, double kdx2, double tol, int max_iter,
                      int *iters, double *relres);
// Threads per block of LBM / transport launch shape v (0 if v is no shape).
int cdi_lbm_shape_block(int v);
int cdi_np_shape_block(int v);
cdi_status cdi_imp_steps(cdi_domain *d, int64_t n);
