// C ABI of the CDI library: domain lifecycle, argument checking, errors,
// device memory, event timing, field copies and queries.  The numerical work
// lives in flow.cu, potential.cu and transport.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "cdi_internal.cuh"

static thread_local std::string g_create_error;

cdi_status cdi_fail(cdi_domain *d, cdi_status s, const std::string &msg) {
  if (d)
    d->err = msg;
  else
    g_create_error = msg;
  return s;
}

cdi_status cdi_cuda_fail(cdi_domain *d, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                  cudaGetErrorString(e) + ")";
  (void)cudaGetLastError();
  return cdi_fail(d, e == cudaErrorMemoryAllocation ? CDI_ERR_OOM : CDI_ERR_CUDA, m);
}

// Device memory: the caller's allocator when one was given, else
// stream-ordered allocation on the domain's stream (cudaMallocAsync /
// cudaFreeAsync from the device's default memory pool), which, unlike
// cudaMalloc/cudaFree, does not synchronise the device, so domains created
// and destroyed while others run do not stall them.
void *cdi_dev_alloc(cdi_domain *d, size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~size_t(255);
  void *p = nullptr;
  if (d->has_alloc) {
    p = d->alloc.alloc(bytes, d->alloc.ctx);
  } else if (cudaMallocAsync(&p, bytes, d->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    p = nullptr;
  }
  if (p) d->blocks.push_back({p, bytes});
  return p;
}

static void dev_free(cdi_domain *d, void *p, size_t bytes) {
  if (d->has_alloc)
    d->alloc.free(p, bytes, d->alloc.ctx);
  else if (cudaFreeAsync(p, d->stream) != cudaSuccess)
    (void)cudaGetLastError();
}

// Release one block from cdi_dev_alloc (after the stream has finished with
// it: stream-ordered frees take effect in stream order).
void cdi_dev_release(cdi_domain *d, void *p) {
  for (size_t i = 0; i < d->blocks.size(); i++) {
    if (d->blocks[i].p != p) continue;
    dev_free(d, p, d->blocks[i].bytes);
    d->blocks.erase(d->blocks.begin() + (long)i);
    return;
  }
}

// Pinned host blocks for the device scalars, recycled across domains
// (freeing pinned memory would synchronise the device).
static std::mutex g_pinned_mutex;
static std::vector<double *> g_pinned_free;

static cudaError_t pinned_take(double **p) {
  {
    std::lock_guard<std::mutex> lock(g_pinned_mutex);
    if (!g_pinned_free.empty()) {
      *p = g_pinned_free.back();
      g_pinned_free.pop_back();
      return cudaSuccess;
    }
  }
  return cudaMallocHost(reinterpret_cast<void **>(p), S_COUNT * 8);
}

static void pinned_give(double *p) {
  std::lock_guard<std::mutex> lock(g_pinned_mutex);
  g_pinned_free.push_back(p);
}

static void free_all(cdi_domain *d) {
  if (d->stream) cudaStreamSynchronize(d->stream);
  for (auto &b : d->blocks) dev_free(d, b.p, b.bytes);
  d->blocks.clear();
  if (d->stream) cudaStreamSynchronize(d->stream);
  if (d->h_scal) pinned_give(d->h_scal);
  d->h_scal = nullptr;
  if (d->flow_graph) cudaGraphExecDestroy(d->flow_graph);
  if (d->np_graph) cudaGraphExecDestroy(d->np_graph);
  d->flow_graph = d->np_graph = nullptr;
  for (auto &p : d->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  d->pending.clear();
  for (auto e : d->ev_pool) cudaEventDestroy(e);
  d->ev_pool.clear();
  if (d->cap_stream) cudaStreamDestroy(d->cap_stream);
  if (d->own_stream && d->stream) cudaStreamDestroy(d->stream);
  d->cap_stream = d->stream = nullptr;
}

// ---------------------------------------------------------------------------
// Autotuner memory (see cdi_internal.cuh).
// ---------------------------------------------------------------------------
static std::mutex g_tune_mutex;
static std::unordered_map<uint64_t, int> g_tune;

uint64_t cdi_tune_key(int kind, int dim, int prec, int ns, long long n, int extra) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    dev = 0;
  }
  uint64_t h = 1469598103934665603ull;  // FNV-1a over the key fields
  const long long f[7] = {kind, dim, prec, ns, n, extra, dev};
  for (long long v : f)
    for (int b = 0; b < 8; b++) h = (h ^ (uint64_t)((v >> (8 * b)) & 0xff)) * 1099511628211ull;
  return h;
}

bool cdi_tune_lookup(uint64_t key, int *variant) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *variant = it->second;
  return true;
}

void cdi_tune_store(uint64_t key, int variant) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune[key] = variant;
}

// ---------------------------------------------------------------------------
// Event timing: pairs of events on the domain stream around groups of
// launches, resolved at the next synchronisation point.
// ---------------------------------------------------------------------------
static cudaEvent_t take_event(cdi_domain *d) {
  if (!d->ev_pool.empty()) {
    cudaEvent_t e = d->ev_pool.back();
    d->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void cdi_timing_begin(cdi_domain *d, cudaEvent_t *a) {
  *a = take_event(d);
  cudaEventRecord(*a, d->stream);
}

void cdi_timing_end(cdi_domain *d, cudaEvent_t a, int phase, int64_t launches) {
  cudaEvent_t b = take_event(d);
  cudaEventRecord(b, d->stream);
  d->pending.push_back({a, b, phase, launches});
}

cudaError_t cdi_timing_resolve(cdi_domain *d) {
  for (auto &p : d->pending) {
    cudaError_t e = cudaEventSynchronize(p.b);
    if (e != cudaSuccess) return e;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    switch (p.phase) {
      case PH_FLOW: d->timing.flow_ms += ms; d->timing.flow_launches += p.launches; break;
      case PH_CHECK: d->timing.flow_check_ms += ms; break;
      case PH_PSI: d->timing.psi_ms += ms; d->timing.psi_iters += p.launches; break;
      case PH_NP: d->timing.np_ms += ms; d->timing.np_launches += p.launches; break;
    }
    d->ev_pool.push_back(p.a);
    d->ev_pool.push_back(p.b);
  }
  d->pending.clear();
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" {

int cdi_version(void) { return 100; }

const char *cdi_last_error(const cdi_domain *d) {
  return d ? d->err.c_str() : g_create_error.c_str();
}

cdi_status cdi_create_domain(const cdi_domain_desc *desc, const uint8_t *mask,
                             const cdi_allocator *alloc, void *stream, cdi_domain **out) {
  if (!out) return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!desc || !mask) return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "desc or mask is NULL");
  const cdi_domain_desc &D = *desc;
  if (D.dim != 2 && D.dim != 3)
    return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (D.nx < 1 || D.ny < 1 || D.nz < 1 || (D.dim == 2 && D.nz != 1))
    return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "bad grid size (nz must be 1 in 2D)");
  if (D.nx > 65535 || D.ny > 65535 || D.nz > 65535)
    return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "nx, ny and nz must be <= 65535");
  if (!(D.dx_m > 0.0) || !std::isfinite(D.dx_m))
    return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "dx_m must be positive");
  if (D.precision != CDI_FP64 && D.precision != CDI_FP32 && D.precision != CDI_FP32_SPLIT &&
      D.precision != CDI_BF16_POP && D.precision != CDI_FP32_CPAIR)
    return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "unknown precision");
  if (alloc && (!alloc->alloc || !alloc->free))
    return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "allocator needs alloc and free");
  const long long N = (long long)D.nx * D.ny * D.nz;
  const int NX = D.mirror_x ? 2 * D.nx : D.nx;
  const long long Nf = (long long)NX * D.ny * D.nz;
  if (Nf > (1LL << 31) - 1)
    return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "grid too large (flow sites >= 2^31)");
  long long n_pore = 0, n_inlet = 0;
  uint64_t hash = 1469598103934665603ull;
  for (long long i = 0; i < N; i++) {
    if (mask[i] > 1) return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "mask values must be 0 or 1");
    hash = (hash ^ mask[i]) * 1099511628211ull;
    if (!mask[i]) {
      n_pore++;
      if (i % D.nx == 0) n_inlet++;
    }
  }
  if (n_inlet == 0)
    return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "no pore cell in the inlet column x = 0");

  cdi_domain *d = new cdi_domain();
  d->dim = D.dim; d->nx = D.nx; d->ny = D.ny; d->nz = D.nz;
  d->walls = D.lateral_walls ? 1 : 0;
  d->mirror = D.mirror_x ? 1 : 0;
  d->prec = D.precision;
  d->cpair = D.precision == CDI_FP32_SPLIT || D.precision == CDI_FP32_CPAIR;
  d->dx = D.dx_m;
  d->NX = NX; d->N = N; d->Nf = Nf;
  d->n_pore = n_pore; d->n_pore_inlet = n_inlet;
  d->mask_hash = hash;
  if (alloc) {
    d->alloc = *alloc;
    d->has_alloc = true;
  }
  cudaError_t e;
  if (stream) {
    d->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&d->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      cdi_cuda_fail(nullptr, e, "create stream");
      delete d;
      return CDI_ERR_CUDA;
    }
    d->own_stream = true;
  }
  e = cudaStreamCreateWithFlags(&d->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cdi_cuda_fail(nullptr, e, "create capture stream");
    free_all(d);
    delete d;
    return CDI_ERR_CUDA;
  }

  const size_t T = d->prec == CDI_FP64 ? 8 : 4;
  const int Q = D.dim == 2 ? 9 : 19;
  const size_t fflag = D.dim == 2 ? 2 : 4;
  d->n_flow_pore = n_pore * (D.mirror_x ? 2 : 1);
  {
    // FP32 steps run warps of 31 home cells, FP64 steps one thread per cell
    const long long warps31 = (n_pore + 30) / 31;
    const long long units = d->prec == CDI_FP64 ? n_pore : warps31 * 32;
    d->np_blocks = (int)((units + cdi::kRowBlock - 1) / cdi::kRowBlock);
    d->np_accs = (int)((warps31 + 7) / 8) * 8;  // >= the warps of any launch shape
  }
  bool ok = true;
  auto A = [&](size_t bytes) {
    void *p = cdi_dev_alloc(d, bytes);
    if (!p) ok = false;
    return p;
  };
  d->d_mask = (uint8_t *)A(N);
  d->d_fflags = A(Nf * fflag);
  d->d_nflags = (cdi::NFlag *)A(N * sizeof(cdi::NFlag));
  d->d_flow_list = (int *)A((size_t)d->n_flow_pore * sizeof(int));
  d->d_cell_list = (int *)A((size_t)n_pore * sizeof(int));
  int *list_work = (int *)A(cdi_lists_work_ints(Nf) * sizeof(int));
  int *rank_work = (int *)A((size_t)Nf * sizeof(int));
  // populations stored by pore rank: Q * n_flow_pore values
  const size_t nq = (size_t)Q * d->n_flow_pore;
  const size_t Tpop = d->prec == CDI_FP64 ? 8 : d->prec == CDI_BF16_POP ? 2 : 4;
  d->d_g = A(nq * Tpop);
  if (d->prec == CDI_FP32_SPLIT) d->d_glo = (float *)A(nq * 4);
  // (the overflow table is sized and taken while the links are built)
  d->n_ltiles = (int)((d->n_flow_pore + 31) / 32);
  d->d_lf = (unsigned *)A((size_t)d->n_flow_pore * sizeof(unsigned));
  d->d_ld = (unsigned *)A((size_t)(D.dim == 2 ? 1 : 2) * d->n_flow_pore * sizeof(unsigned));
  d->d_lb = (int *)A((size_t)(D.dim == 2 ? 2 : 8) * d->n_ltiles * sizeof(int));
  d->d_uflow = (double *)A((size_t)D.dim * Nf * 8);
  // transport fields by pore rank
  d->W = (D.nx + 31) / 32;
  const size_t n_words = (size_t)D.ny * D.nz * d->W;
  d->d_cmeta = (uint2 *)A((size_t)n_pore * sizeof(uint2));
  d->d_cfl = (cdi::NFlag *)A((size_t)n_pore * sizeof(cdi::NFlag));
  d->d_words = (uint2 *)A(n_words * sizeof(uint2));
  d->d_latnb = (int *)A((size_t)2 * (D.dim - 1) * n_pore * sizeof(int));
  d->d_u = A((size_t)D.dim * n_pore * T);
  d->d_psi = (double *)A(N * 8);
  d->d_phi = A((size_t)n_pore * 8);
  d->d_C[0] = A((size_t)cdi::kMaxSpecies * n_pore * T);
  d->d_C[1] = A((size_t)cdi::kMaxSpecies * n_pore * T);
  if (d->cpair) {
    d->d_Clo[0] = (float *)A((size_t)cdi::kMaxSpecies * n_pore * 4);
    d->d_Clo[1] = (float *)A((size_t)cdi::kMaxSpecies * n_pore * 4);
  }
  d->d_acc = (double *)A((size_t)3 * cdi::kMaxSpecies * d->np_accs * 8);
  d->d_part = (double *)A((size_t)16 * cdi::kRedBlocks * 8);
  d->d_counter = (unsigned int *)A(16 * sizeof(unsigned int));
  d->d_scal = (double *)A(S_COUNT * 8);
  d->d_cg = (double *)A((size_t)4 * N * 8);
  d->d_colout = (double *)A((size_t)D.nx * 8);
  if (!ok) {
    free_all(d);
    delete d;
    return cdi_fail(nullptr, CDI_ERR_OOM, "device allocation failed");
  }
  e = pinned_take(&d->h_scal);
  if (e != cudaSuccess) {
    cdi_cuda_fail(nullptr, e, "pinned scalars");
    free_all(d);
    delete d;
    return CDI_ERR_CUDA;
  }
  std::memset(d->h_scal, 0, S_COUNT * 8);
  cdi_status s = CDI_OK;
  auto chk = [&](cudaError_t ee, const char *w) {
    if (s == CDI_OK && ee != cudaSuccess) s = cdi_cuda_fail(d, ee, w);
  };
  chk(cudaMemcpyAsync(d->d_mask, mask, N, cudaMemcpyHostToDevice, d->stream), "upload mask");
  chk(cudaMemsetAsync(d->d_counter, 0, 16 * sizeof(unsigned int), d->stream), "memset");
  chk(cudaMemsetAsync(d->d_scal, 0, S_COUNT * 8, d->stream), "memset");
  chk(cudaMemsetAsync(d->d_g, 0, nq * Tpop, d->stream), "memset");
  chk(cudaMemsetAsync(d->d_uflow, 0, (size_t)D.dim * Nf * 8, d->stream), "memset");
  chk(cudaMemsetAsync(d->d_u, 0, (size_t)D.dim * n_pore * T, d->stream), "memset");
  chk(cudaMemsetAsync(d->d_psi, 0, N * 8, d->stream), "memset");
  chk(cudaMemsetAsync(d->d_phi, 0, (size_t)n_pore * 8, d->stream), "memset");
  chk(cudaMemsetAsync(d->d_C[0], 0, (size_t)cdi::kMaxSpecies * n_pore * T, d->stream), "memset");
  chk(cudaMemsetAsync(d->d_C[1], 0, (size_t)cdi::kMaxSpecies * n_pore * T, d->stream), "memset");
  for (int b = 0; b < 2 && d->cpair; b++)
    chk(cudaMemsetAsync(d->d_Clo[b], 0, (size_t)cdi::kMaxSpecies * n_pore * 4, d->stream),
        "memset");
  chk(cudaMemsetAsync(d->d_acc, 0, (size_t)3 * cdi::kMaxSpecies * d->np_accs * 8, d->stream),
      "memset");
  if (s == CDI_OK) s = cdi_flow_build_flags(d);
  if (s == CDI_OK) s = cdi_np_build_flags(d);
  if (s == CDI_OK) s = cdi_build_lists(d, list_work);
  if (s == CDI_OK) s = cdi_np_build_compact(d);
  if (s == CDI_OK) s = cdi_flow_build_links(d, rank_work);
  if (s == CDI_OK) chk(cudaStreamSynchronize(d->stream), "create domain");
  if (s == CDI_OK) {  // the work arrays are needed at create time only
    cdi_dev_release(d, rank_work);
    cdi_dev_release(d, list_work);
  }
  if (s != CDI_OK) {
    g_create_error = d->err;
    free_all(d);
    delete d;
    return s;
  }
  *out = d;
  return CDI_OK;
}

void cdi_destroy_domain(cdi_domain *d) {
  if (!d) return;
  free_all(d);
  delete d;
}

cdi_status cdi_solve_flow(cdi_domain *d, const cdi_flow_params *p, int64_t *steps_out,
                          double *residual_out) {
  if (!d || !p) return cdi_fail(d, CDI_ERR_INVALID_ARG, "NULL argument");
  if (!(p->tau > 0.5) || !std::isfinite(p->tau))
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "tau must be > 1/2");
  if (p->check_every < 2 || (p->check_every % 2) != 0)
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "check_every must be even and >= 2");
  if (p->max_steps < 0 || (p->max_steps % p->check_every) != 0)
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "max_steps must be a multiple of check_every");
  if (!std::isfinite(p->force_lu) || !std::isfinite(p->U_target_mps))
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "non-finite force or velocity");
  d->flow_done = false;
  d->np_ready = false;
  int64_t steps = 0;
  double res = 0.0;
  cdi_status s = cdi_flow_run(d, p, &steps, &res);
  if (steps_out) *steps_out = steps;
  if (residual_out) *residual_out = res;
  if (s != CDI_OK && s != CDI_ERR_NOT_CONVERGED) return s;
  cdi_status s2 = cdi_flow_export(d, p->U_target_mps);
  if (s2 != CDI_OK) return s2;
  d->flow_done = true;
  if (s == CDI_ERR_NOT_CONVERGED)
    return cdi_fail(d, s, "flow residual did not reach tol within max_steps");
  return CDI_OK;
}

cdi_status cdi_solve_flow_batch(cdi_domain *const *doms, int n_doms, const cdi_flow_params *p,
                                int64_t *steps_out, double *residual_out, int *status_out) {
  if (!doms || n_doms < 1 || !doms[0])
    return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "flow batch: no domains");
  cdi_domain *L = doms[0];
  if (!p) return cdi_fail(L, CDI_ERR_INVALID_ARG, "NULL argument");
  if (!(p->tau > 0.5) || !std::isfinite(p->tau))
    return cdi_fail(L, CDI_ERR_INVALID_ARG, "tau must be > 1/2");
  if (p->check_every < 2 || (p->check_every % 2) != 0)
    return cdi_fail(L, CDI_ERR_INVALID_ARG, "check_every must be even and >= 2");
  if (p->max_steps < 0 || (p->max_steps % p->check_every) != 0)
    return cdi_fail(L, CDI_ERR_INVALID_ARG, "max_steps must be a multiple of check_every");
  if (!std::isfinite(p->force_lu) || !std::isfinite(p->U_target_mps))
    return cdi_fail(L, CDI_ERR_INVALID_ARG, "non-finite force or velocity");
  for (int i = 0; i < n_doms; i++) {
    if (!doms[i]) return cdi_fail(L, CDI_ERR_INVALID_ARG, "flow batch: NULL domain");
    if (doms[i]->dim != L->dim || doms[i]->prec != L->prec)
      return cdi_fail(L, CDI_ERR_INVALID_ARG,
                      "flow batch: domains differ in dimension or precision");
    for (int j = 0; j < i; j++)
      if (doms[j] == doms[i]) return cdi_fail(L, CDI_ERR_INVALID_ARG, "flow batch: repeated domain");
  }
  std::vector<int64_t> steps(n_doms);
  std::vector<double> res(n_doms);
  std::vector<int> st(n_doms);
  for (int i = 0; i < n_doms; i++) {
    doms[i]->flow_done = false;
    doms[i]->np_ready = false;
  }
  cdi_status s = cdi_flow_batch(doms, n_doms, p, steps.data(), res.data(), st.data());
  if (s != CDI_OK) return s;
  bool all = true;
  for (int i = 0; i < n_doms; i++) {
    if (steps_out) steps_out[i] = steps[i];
    if (residual_out) residual_out[i] = res[i];
    if (status_out) status_out[i] = st[i];
    if (st[i] == CDI_ERR_CUDA) {
      all = false;
      continue;
    }
    cdi_status s2 = cdi_flow_export(doms[i], p->U_target_mps);
    if (s2 != CDI_OK) return cdi_fail(L, s2, std::string("flow batch: ") + doms[i]->err);
    doms[i]->flow_done = true;
    if (st[i] != CDI_OK) all = false;
  }
  if (!all) return cdi_fail(L, CDI_ERR_NOT_CONVERGED, "flow batch: some domains did not converge");
  return CDI_OK;
}

cdi_status cdi_set_velocity(cdi_domain *d, double U) {
  if (!d) return CDI_ERR_INVALID_ARG;
  if (!d->flow_done) return cdi_fail(d, CDI_ERR_STATE, "no solved flow");
  if (!std::isfinite(U)) return cdi_fail(d, CDI_ERR_INVALID_ARG, "non-finite velocity");
  d->np_ready = false;
  return cdi_flow_export(d, U);
}

cdi_status cdi_set_potential(cdi_domain *d, double applied_V, const cdi_elec_params *p,
                             int *iters_out, double *relres_out) {
  if (!d || !p) return cdi_fail(d, CDI_ERR_INVALID_ARG, "NULL argument");
  if (!(p->T_K > 0) || !(p->eps_r > 0) || !std::isfinite(applied_V))
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "T_K and eps_r must be positive");
  if (p->mode < 0 || p->mode > 2)
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "mode must be 0, 1 or 2");
  if (p->mode != 1 && !(p->lambda_D_m > 0) && !(p->c_bulk_molm3 > 0))
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "screened modes need c_bulk or lambda_D");
  if (!(p->tol > 0) || p->max_iter < 1)
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "tol must be > 0 and max_iter >= 1");
  // Physical constants (e and k_B as printed with Eq. 9-10).
  const double e = 1.6e-19, kB = 1.38e-23, F = 96485.0, eps0 = 8.854e-12;
  double kdx2 = 0.0;
  if (p->mode != 1) {
    double lam = p->lambda_D_m > 0
                     ? p->lambda_D_m
                     : std::sqrt(p->eps_r * eps0 * kB * p->T_K / (2.0 * p->c_bulk_molm3 * e * F));
    kdx2 = (d->dx / lam) * (d->dx / lam);
  }
  d->VT = kB * p->T_K / e;
  d->np_ready = false;
  d->psi_done = false;
  int it = 0;
  double rel = 0.0;
  d->psi_s = -applied_V;
  d->eps_r = p->eps_r;
  d->psi_tol = p->tol;
  d->psi_max_iter = p->max_iter;
  cdi_status s =
      p->mode == 2 ? cdi_psi_pb(d, -applied_V, kdx2, p->tol, p->max_iter, &it, &rel)
                   : cdi_psi_solve(d, -applied_V, kdx2, nullptr, p->tol, p->max_iter, &it, &rel);
  if (iters_out) *iters_out = it;
  if (relres_out) *relres_out = rel;
  if (s == CDI_OK || s == CDI_ERR_NOT_CONVERGED) d->psi_done = true;
  if (s == CDI_ERR_NOT_CONVERGED)
    return cdi_fail(d, s, "potential solve did not reach tol within max_iter");
  return s;
}

cdi_status cdi_set_implicit(cdi_domain *d, double tol, int max_iter) {
  if (!d) return CDI_ERR_INVALID_ARG;
  if (!std::isfinite(tol)) return cdi_fail(d, CDI_ERR_INVALID_ARG, "non-finite tolerance");
  if (tol <= 0.0) {
    d->imp_tol = 0.0;
    return CDI_OK;
  }
  if (max_iter < 1) return cdi_fail(d, CDI_ERR_INVALID_ARG, "max_iter must be >= 1");
  cdi_status s = cdi_imp_prepare(d);
  if (s != CDI_OK) return s;
  d->imp_tol = tol;
  d->imp_max_iter = max_iter;
  return CDI_OK;
}

cdi_status cdi_set_launch_shapes(cdi_domain *d, int32_t lbm_shape, int32_t np_shape) {
  if (!d) return CDI_ERR_INVALID_ARG;
  if (lbm_shape < -1 || (lbm_shape >= 0 && cdi_lbm_shape_block(lbm_shape) == 0))
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "no such LBM launch shape");
  if (np_shape < -1 || (np_shape >= 0 && cdi_np_shape_block(np_shape) == 0))
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "no such transport launch shape");
  // captured step graphs hold the old launches: drop them (recaptured on use)
  CDI_TRY(d, cudaStreamSynchronize(d->stream), "launch shapes");
  if (d->flow_graph) cudaGraphExecDestroy(d->flow_graph);
  if (d->np_graph) cudaGraphExecDestroy(d->np_graph);
  d->flow_graph = d->np_graph = nullptr;
  if (lbm_shape >= 0) {
    d->lbm_variant = lbm_shape;
    d->lbm_block = cdi_lbm_shape_block(lbm_shape);
  }
  d->lbm_tuned = lbm_shape >= 0;
  if (np_shape >= 0) {
    d->np_variant = np_shape;
    d->np_block = cdi_np_shape_block(np_shape);
  }
  d->np_tuned = np_shape >= 0;
  return CDI_OK;
}

cdi_status cdi_set_coupling(cdi_domain *d, int64_t every_steps) {
  if (!d) return CDI_ERR_INVALID_ARG;
  if (every_steps < 0) return cdi_fail(d, CDI_ERR_INVALID_ARG, "every_steps < 0");
  if (every_steps > 0 && !d->psi_done)
    return cdi_fail(d, CDI_ERR_STATE, "set the potential first (its parameters are reused)");
  if (every_steps > 0 && !d->d_src) {
    d->d_src = (double *)cdi_dev_alloc(d, (size_t)d->N * 8);
    if (!d->d_src) return cdi_fail(d, CDI_ERR_OOM, "coupling: charge buffer");
  }
  d->couple_K = every_steps;
  return CDI_OK;
}

cdi_status cdi_init_transport(cdi_domain *d, const cdi_species *sp, int n, double c0,
                              double Ka, double dt_s, double *dt_used) {
  if (!d || !sp) return cdi_fail(d, CDI_ERR_INVALID_ARG, "NULL argument");
  if (n < 1 || n > cdi::kMaxSpecies) return cdi_fail(d, CDI_ERR_INVALID_ARG, "1..4 species");
  for (int k = 0; k < n; k++)
    if (!(sp[k].D_m2s > 0) || !std::isfinite(sp[k].D_m2s) || sp[k].z < -8 || sp[k].z > 8)
      return cdi_fail(d, CDI_ERR_INVALID_ARG, "species need D > 0 and |z| <= 8");
  if (!(c0 >= 0) || !(Ka >= 0) || !(dt_s >= 0) || !std::isfinite(c0) || !std::isfinite(Ka) ||
      !std::isfinite(dt_s))
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "c0, Ka, dt must be finite and >= 0");
  if (!d->flow_done) return cdi_fail(d, CDI_ERR_STATE, "solve the flow first");
  if (!d->psi_done) return cdi_fail(d, CDI_ERR_STATE, "set the potential first");
  d->ns = n;
  for (int k = 0; k < cdi::kMaxSpecies; k++) {
    d->z[k] = k < n ? sp[k].z : 0;
    d->D[k] = k < n ? sp[k].D_m2s : 1.0;
  }
  d->c0 = c0;
  d->Ka = Ka;
  d->np_ready = false;
  cdi_status s = cdi_np_init(d, dt_s, dt_used);
  if (s == CDI_OK) d->np_ready = true;
  return s;
}

}  // extern "C"

namespace {

// Argument checks shared by the sweep entry points.
cdi_status check_sweep_args(cdi_domain *d, const cdi_combo *combos, int n_combos,
                            const cdi_elec_params *ep, const cdi_species *sp, int n, double c0,
                            double Ka, int64_t n_steps) {
  if (!combos || !ep || !sp) return cdi_fail(d, CDI_ERR_INVALID_ARG, "NULL argument");
  if (n_combos < 1 || n_combos > 4096)
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "1..4096 combinations");
  if (n_steps < 0) return cdi_fail(d, CDI_ERR_INVALID_ARG, "n_steps < 0");
  if (n < 1 || n > cdi::kMaxSpecies) return cdi_fail(d, CDI_ERR_INVALID_ARG, "1..4 species");
  for (int k = 0; k < n; k++)
    if (!(sp[k].D_m2s > 0) || !std::isfinite(sp[k].D_m2s) || sp[k].z < -8 || sp[k].z > 8)
      return cdi_fail(d, CDI_ERR_INVALID_ARG, "species need D > 0 and |z| <= 8");
  if (!(c0 >= 0) || !(Ka >= 0) || !std::isfinite(c0) || !std::isfinite(Ka))
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "c0 and Ka must be finite and >= 0");
  for (int m = 0; m < n_combos; m++)
    if (!std::isfinite(combos[m].U_mps) || !std::isfinite(combos[m].applied_V))
      return cdi_fail(d, CDI_ERR_INVALID_ARG, "non-finite combination");
  if (!d->flow_done) return cdi_fail(d, CDI_ERR_STATE, "solve the flow first");
  if (d->U_lat == 0.0) {
    for (int m = 0; m < n_combos; m++)
      if (combos[m].U_mps != 0.0)
        return cdi_fail(d, CDI_ERR_INVALID_ARG, "no net flow through the pore space to scale");
  }
  return CDI_OK;
}

// One domain's part of a sweep: the species, one potential per distinct
// applied value (each solved as by cdi_set_potential and kept in a buffer of
// `owner`'s, appended to phis), and each member's velocity scale, potential
// index and time step (as cdi_set_velocity and cdi_init_transport set them).
cdi_status prepare_sweep(cdi_domain *d, cdi_domain *owner, const cdi_combo *combos,
                         int n_combos, const cdi_elec_params *ep, const cdi_species *sp, int n,
                         double c0, double Ka, double *scale, int *group, double *dts,
                         std::vector<void *> &phis) {
  // the sweep replaces the domain's potential and transport state
  d->np_ready = false;
  d->ns = n;
  for (int k = 0; k < cdi::kMaxSpecies; k++) {
    d->z[k] = k < n ? sp[k].z : 0;
    d->D[k] = k < n ? sp[k].D_m2s : 1.0;
  }
  d->c0 = c0;
  d->Ka = Ka;
  std::vector<double> gv;
  std::vector<int> local(n_combos);
  for (int m = 0; m < n_combos; m++) {
    int g = -1;
    for (size_t i = 0; i < gv.size(); i++)
      if (gv[i] == combos[m].applied_V) g = (int)i;
    if (g < 0) {
      g = (int)gv.size();
      gv.push_back(combos[m].applied_V);
    }
    local[m] = g;
    scale[m] = combos[m].U_mps == 0.0 ? 0.0 : combos[m].U_mps / d->U_lat;
  }
  const int base = (int)phis.size();
  cdi_status s = CDI_OK;
  for (size_t g = 0; g < gv.size() && s == CDI_OK; g++) {
    s = cdi_set_potential(d, gv[g], ep, nullptr, nullptr);
    if (s != CDI_OK) break;
    void *ph = cdi_dev_alloc(owner, (size_t)d->n_pore * 8);
    if (!ph) {
      s = cdi_fail(d, CDI_ERR_OOM, "sweep: potential buffer");
      break;
    }
    // stream-ordered allocation on the owner's stream, used on d's stream
    if (owner != d && cudaStreamSynchronize(owner->stream) != cudaSuccess) {
      s = cdi_fail(d, CDI_ERR_CUDA, "sweep: potential buffer");
      break;
    }
    phis.push_back(ph);
    cudaError_t e = cudaMemcpyAsync(ph, d->d_phi, (size_t)d->n_pore * 8,
                                    cudaMemcpyDeviceToDevice, d->stream);
    if (e != cudaSuccess) s = cdi_cuda_fail(d, e, "sweep: potential copy");
    for (int m = 0; m < n_combos && s == CDI_OK; m++)
      if (local[m] == (int)g) s = cdi_np_dt(d, scale[m], &dts[m]);
  }
  for (int m = 0; m < n_combos; m++) group[m] = base + local[m];
  d->psi_done = false;  // the domain's potential is the last group's
  return s;
}

}  // namespace

extern "C" {

cdi_status cdi_sweep_transport(cdi_domain *d, const cdi_combo *combos, int n_combos,
                               const cdi_elec_params *ep, const cdi_species *sp, int n,
                               double c0, double Ka, int64_t n_steps, double *gamma_out,
                               double *cout_out, double *dt_out) {
  if (!d || !gamma_out || !cout_out) return cdi_fail(d, CDI_ERR_INVALID_ARG, "NULL argument");
  cdi_status s = check_sweep_args(d, combos, n_combos, ep, sp, n, c0, Ka, n_steps);
  if (s != CDI_OK) return s;
  std::vector<int> group(n_combos);
  std::vector<double> scale(n_combos), dts(n_combos);
  std::vector<void *> phis;
  s = prepare_sweep(d, d, combos, n_combos, ep, sp, n, c0, Ka, scale.data(), group.data(),
                    dts.data(), phis);
  if (s == CDI_OK)
    s = cdi_np_sweep(d, n_combos, scale.data(), group.data(), phis.data(), dts.data(), n_steps,
                     gamma_out, cout_out);
  cudaStreamSynchronize(d->stream);
  for (void *p : phis) cdi_dev_release(d, p);
  if (s == CDI_OK && dt_out)
    for (int m = 0; m < n_combos; m++) dt_out[m] = dts[m];
  return s;
}

cdi_status cdi_sweep_batch(cdi_domain *const *doms, int n_doms, const cdi_combo *combos,
                           int n_combos, const cdi_elec_params *ep, const cdi_species *sp,
                           int n, double c0, double Ka, int64_t n_steps, double *gamma_out,
                           double *cout_out, double *dt_out) {
  if (!doms || n_doms < 1 || !doms[0])
    return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "batch: no domains");
  cdi_domain *L = doms[0];
  if (!gamma_out || !cout_out) return cdi_fail(L, CDI_ERR_INVALID_ARG, "NULL argument");
  if ((int64_t)n_doms * n_combos > (1 << 20))
    return cdi_fail(L, CDI_ERR_INVALID_ARG, "batch: at most 2^20 members");
  int64_t blocks = 0;
  for (int i = 0; i < n_doms; i++) {
    if (!doms[i]) return cdi_fail(L, CDI_ERR_INVALID_ARG, "batch: NULL domain");
    if (doms[i]->dim != L->dim || doms[i]->prec != L->prec)
      return cdi_fail(L, CDI_ERR_INVALID_ARG, "batch: domains differ in dimension or precision");
    for (int j = 0; j < i; j++)
      if (doms[j] == doms[i]) return cdi_fail(L, CDI_ERR_INVALID_ARG, "batch: repeated domain");
    cdi_status s = check_sweep_args(doms[i], combos, n_combos, ep, sp, n, c0, Ka, n_steps);
    if (s != CDI_OK) return cdi_fail(L, s, std::string("batch: ") + doms[i]->err);
    blocks += (int64_t)doms[i]->np_blocks * n_combos;
  }
  if (blocks > 0x7fffffff) return cdi_fail(L, CDI_ERR_INVALID_ARG, "batch: too many blocks");
  const int nm = n_doms * n_combos;
  std::vector<int> group(nm);
  std::vector<double> scale(nm), dts(nm);
  std::vector<void *> phis;
  cdi_status s = CDI_OK;
  for (int i = 0; i < n_doms && s == CDI_OK; i++) {
    s = prepare_sweep(doms[i], L, combos, n_combos, ep, sp, n, c0, Ka, scale.data() + i * n_combos,
                      group.data() + i * n_combos, dts.data() + i * n_combos, phis);
    if (s != CDI_OK && doms[i] != L) cdi_fail(L, s, std::string("batch: ") + doms[i]->err);
    if (s == CDI_OK && cudaStreamSynchronize(doms[i]->stream) != cudaSuccess)
      s = cdi_fail(L, CDI_ERR_CUDA, "batch: potential");
  }
  if (s == CDI_OK)
    s = cdi_np_batch(doms, n_doms, n_combos, scale.data(), group.data(), phis.data(), dts.data(),
                     n_steps, gamma_out, cout_out);
  cudaStreamSynchronize(L->stream);
  for (void *p : phis) cdi_dev_release(L, p);
  if (s == CDI_OK && dt_out)
    for (int m = 0; m < nm; m++) dt_out[m] = dts[m];
  return s;
}

cdi_status cdi_step_transport(cdi_domain *d, int64_t n) {
  if (!d) return CDI_ERR_INVALID_ARG;
  if (n < 0) return cdi_fail(d, CDI_ERR_INVALID_ARG, "n_steps < 0");
  if (!d->np_ready) return cdi_fail(d, CDI_ERR_STATE, "call cdi_init_transport first");
  return cdi_np_steps(d, n);
}

cdi_status cdi_query_mass_balance(cdi_domain *d, double *M, double *G, double *In, double *Out) {
  if (!d) return CDI_ERR_INVALID_ARG;
  if (!d->np_ready) return cdi_fail(d, CDI_ERR_STATE, "no transport state");
  cdi_status s = cdi_np_reduce(d);
  if (s != CDI_OK) return s;
  const double area = d->dim == 2 ? d->dx : d->dx * d->dx;
  for (int k = 0; k < d->ns; k++) {
    if (M) M[k] = d->h_scal[S_MASS + k];
    if (G) G[k] = d->h_scal[S_ACC + 3 * k + 0] * d->dt * area;
    if (In) In[k] = d->h_scal[S_ACC + 3 * k + 1] * d->dt * area;
    if (Out) Out[k] = d->h_scal[S_ACC + 3 * k + 2] * d->dt * area;
  }
  return CDI_OK;
}

cdi_status cdi_query_adsorbed(cdi_domain *d, double *per_species) {
  if (!d || !per_species) return cdi_fail(d, CDI_ERR_INVALID_ARG, "NULL argument");
  return cdi_query_mass_balance(d, nullptr, per_species, nullptr, nullptr);
}

cdi_status cdi_query_outlet(cdi_domain *d, double *per_species) {
  if (!d || !per_species) return cdi_fail(d, CDI_ERR_INVALID_ARG, "NULL argument");
  if (!d->np_ready) return cdi_fail(d, CDI_ERR_STATE, "no transport state");
  cdi_status s = cdi_np_reduce(d);
  if (s != CDI_OK) return s;
  for (int k = 0; k < d->ns; k++) {
    double num = d->h_scal[S_OUT + 2 * k], den = d->h_scal[S_OUT + 2 * k + 1];
    double cnt = d->h_scal[S_OUTN];
    if (den != 0.0)
      per_species[k] = num / den;
    else
      per_species[k] = cnt > 0 ? d->h_scal[S_OUTP + k] / cnt : 0.0;
  }
  return CDI_OK;
}

cdi_status cdi_query_geometry(cdi_domain *d, double *porosity, double *s_per_m) {
  if (!d || !porosity || !s_per_m) return cdi_fail(d, CDI_ERR_INVALID_ARG, "NULL argument");
  double pores = 0.0, faces = 0.0;
  cdi_status s = cdi_np_geometry(d, &pores, &faces, nullptr);
  if (s != CDI_OK) return s;
  *porosity = pores / (double)d->N;
  *s_per_m = faces / ((double)d->N * d->dx);
  return CDI_OK;
}

cdi_status cdi_query_derived(cdi_domain *d, cdi_derived *out) {
  if (!d || !out) return cdi_fail(d, CDI_ERR_INVALID_ARG, "NULL argument");
  if (!d->np_ready) return cdi_fail(d, CDI_ERR_STATE, "no transport state");
  double pores = 0.0, faces = 0.0, sum_ux = 0.0;
  cdi_status s = cdi_np_geometry(d, &pores, &faces, &sum_ux);
  if (s != CDI_OK) return s;
  double cout[cdi::kMaxSpecies] = {0, 0, 0, 0};
  s = cdi_query_outlet(d, cout);
  if (s != CDI_OK) return s;
  std::memset(out, 0, sizeof(*out));
  const double cells = (double)d->N;
  out->porosity = pores / cells;
  out->specific_surface = faces / (cells * d->dx);
  const double pi = 3.14159265358979323846;
  out->l_c_m = faces > 0.0 ? pi / out->specific_surface : INFINITY;
  out->U_mps = pores > 0.0 ? sum_ux / pores : 0.0;  // sum u / (N phi), N phi = pore cells
  out->elapsed_s = (double)d->np_steps * d->dt;
  // inlet cross-section (per metre of depth in 2D) and electrode volume
  const double A = d->dim == 2 ? d->ny * d->dx : (double)d->ny * d->nz * d->dx * d->dx;
  const double Vt = d->dim == 2 ? cells * d->dx * d->dx : cells * d->dx * d->dx * d->dx;
  for (int k = 0; k < d->ns; k++) {
    out->Pe[k] = out->U_mps * out->l_c_m / d->D[k];
    out->Da[k] = d->Ka * out->l_c_m / d->D[k];
    out->removal[k] = d->c0 != 0.0 ? (d->c0 - cout[k]) / d->c0 : 0.0;
    out->amount[k] = out->porosity > 0.0
                         ? out->U_mps * A * out->removal[k] * out->elapsed_s / (Vt * out->porosity)
                         : 0.0;
  }
  return CDI_OK;
}

cdi_status cdi_query_column_means(cdi_domain *d, int species, double *out) {
  if (!d || !out) return cdi_fail(d, CDI_ERR_INVALID_ARG, "NULL argument");
  if (!d->np_ready) return cdi_fail(d, CDI_ERR_STATE, "no transport state");
  if (species < 0 || species >= d->ns) return cdi_fail(d, CDI_ERR_INVALID_ARG, "bad species");
  cdi_status s = cdi_np_column_means(d, species);
  if (s != CDI_OK) return s;
  CDI_TRY(d, cudaMemcpyAsync(out, d->d_colout, (size_t)d->nx * 8, cudaMemcpyDeviceToHost,
                             d->stream), "copy column means");
  CDI_TRY(d, cudaStreamSynchronize(d->stream), "column means");
  return CDI_OK;
}

cdi_status cdi_copy_field(cdi_domain *d, int field, double *host, size_t count) {
  if (!d || !host) return cdi_fail(d, CDI_ERR_INVALID_ARG, "NULL argument");
  const size_t T = d->prec == CDI_FP64 ? 8 : 4;
  const void *src = nullptr;
  const float *lo = nullptr;
  int comps = 0;
  double *tmp = d->d_cg;  // 4*N doubles of scratch outside a potential solve
  if (field == CDI_FIELD_U_LATTICE) {
    const size_t n = (size_t)d->dim * d->Nf;
    if (count != n) return cdi_fail(d, CDI_ERR_INVALID_ARG, "count mismatch");
    CDI_TRY(d, cudaMemcpyAsync(host, d->d_uflow, n * 8, cudaMemcpyDeviceToHost, d->stream),
            "copy u lattice");
    CDI_TRY(d, cudaStreamSynchronize(d->stream), "copy field");
    return CDI_OK;
  } else if (field == CDI_FIELD_PSI) {
    const size_t n = (size_t)d->N;
    if (count != n) return cdi_fail(d, CDI_ERR_INVALID_ARG, "count mismatch");
    CDI_TRY(d, cudaMemcpyAsync(host, d->d_psi, n * 8, cudaMemcpyDeviceToHost, d->stream),
            "copy psi");
    CDI_TRY(d, cudaStreamSynchronize(d->stream), "copy field");
    return CDI_OK;
  } else if (field == CDI_FIELD_U) {
    comps = d->dim;
    src = d->d_u;
  } else if (field >= CDI_FIELD_C && field < CDI_FIELD_C + cdi::kMaxSpecies) {
    int k = field - CDI_FIELD_C;
    if (!d->np_ready || k >= d->ns) return cdi_fail(d, CDI_ERR_STATE, "no such species state");
    comps = 1;
    src = (const char *)d->d_C[d->cur] + (size_t)k * d->n_pore * T;
    if (d->cpair) lo = d->d_Clo[d->cur] + (size_t)k * d->n_pore;
  } else {
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "unknown field");
  }
  // rank-ordered transport field -> lattice order (0 in solid cells)
  const size_t n = (size_t)comps * d->N;
  if (count != n) return cdi_fail(d, CDI_ERR_INVALID_ARG, "count mismatch");
  cdi_status s = cdi_np_scatter(d, src, lo, comps, tmp);
  if (s != CDI_OK) return s;
  CDI_TRY(d, cudaMemcpyAsync(host, tmp, n * 8, cudaMemcpyDeviceToHost, d->stream), "copy field");
  CDI_TRY(d, cudaStreamSynchronize(d->stream), "copy field");
  return CDI_OK;
}

cdi_status cdi_query_timing(cdi_domain *d, cdi_timing *out, int reset) {
  if (!d || !out) return cdi_fail(d, CDI_ERR_INVALID_ARG, "NULL argument");
  CDI_TRY(d, cdi_timing_resolve(d), "timing events");
  *out = d->timing;
  out->lbm_block = d->lbm_tuned ? d->lbm_block : 0;
  out->np_block = d->np_tuned ? d->np_block : 0;
  out->lbm_shape = d->lbm_tuned ? d->lbm_variant : -1;
  out->np_shape = d->np_tuned ? d->np_variant : -1;
  if (reset) d->timing = cdi_timing{};
  return CDI_OK;
}

}  // extern "C"
