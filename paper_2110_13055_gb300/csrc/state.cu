// Checkpoint and restore of a domain's solver state (cdi_save_state,
// cdi_load_state): the solved flow, the potential, the scaled velocity and
// the transport state with its accounts, so that a long transport run can be
// stopped and resumed (in the same process or another one) with results
// identical, bit for bit, to an uninterrupted run.
//
// Format: a fixed header (geometry, precision, a hash of the mask, the
// solver scalars) followed by the device arrays in a fixed order, each as
// raw bytes of the domain's storage precision.  Loading checks that the
// header describes the same geometry and precision as the domain.
#include <cstring>

#include "cdi_internal.cuh"

namespace {

struct StateHeader {
  char magic[8];
  int32_t version;
  int32_t dim, nx, ny, nz, walls, mirror, prec;
  int64_t n_pore, n_flow_pore;
  uint64_t mask_hash;
  int32_t flow_done, psi_done, np_ready, ns, cur, pad;
  int32_t z[cdi::kMaxSpecies];
  double D[cdi::kMaxSpecies];
  double c0, Ka, dt, VT, U_lat, U_target, tau, force, flow_residual;
  int64_t flow_steps, np_steps;
  double psi_s, eps_r, psi_tol;
  int64_t psi_max_iter, couple_K;
};

constexpr char kMagic[8] = {'C', 'D', 'I', 'S', 'T', 'A', 'T', 'E'};
constexpr int32_t kVersion = 1;

struct Section {
  void *dev;
  size_t bytes;
};

// The device arrays of the state, in file order.
std::vector<Section> sections(cdi_domain *d, int c_buf) {
  const size_t T = d->prec == CDI_FP64 ? 8 : 4;
  const size_t Tpop = d->prec == CDI_FP64 ? 8 : d->prec == CDI_BF16_POP ? 2 : 4;
  const int Q = d->dim == 2 ? 9 : 19;
  const size_t nq = (size_t)Q * d->n_flow_pore;
  std::vector<Section> s;
  s.push_back({d->d_g, nq * Tpop});
  if (d->prec == CDI_FP32_SPLIT) s.push_back({d->d_glo, nq * 4});
  s.push_back({d->d_uflow, (size_t)d->dim * d->Nf * 8});
  s.push_back({d->d_u, (size_t)d->dim * d->n_pore * T});
  s.push_back({d->d_psi, (size_t)d->N * 8});
  s.push_back({d->d_phi, (size_t)d->n_pore * 8});
  s.push_back({d->d_C[c_buf], (size_t)cdi::kMaxSpecies * d->n_pore * T});
  if (d->cpair) s.push_back({d->d_Clo[c_buf], (size_t)cdi::kMaxSpecies * d->n_pore * 4});
  s.push_back({d->d_acc, (size_t)3 * cdi::kMaxSpecies * d->np_accs * 8});
  return s;
}

size_t state_bytes(cdi_domain *d) {
  size_t b = sizeof(StateHeader);
  for (const Section &s : sections(d, 0)) b += s.bytes;
  return b;
}

}  // namespace

extern "C" {

cdi_status cdi_save_state(cdi_domain *d, void *host_buf, size_t *bytes) {
  if (!d || !bytes) return cdi_fail(d, CDI_ERR_INVALID_ARG, "NULL argument");
  const size_t need = state_bytes(d);
  if (!host_buf) {
    *bytes = need;
    return CDI_OK;
  }
  if (*bytes < need) {
    *bytes = need;
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "save_state: buffer too small");
  }
  StateHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.dim = d->dim; h.nx = d->nx; h.ny = d->ny; h.nz = d->nz;
  h.walls = d->walls; h.mirror = d->mirror; h.prec = d->prec;
  h.n_pore = d->n_pore; h.n_flow_pore = d->n_flow_pore;
  h.mask_hash = d->mask_hash;
  h.flow_done = d->flow_done; h.psi_done = d->psi_done; h.np_ready = d->np_ready;
  h.ns = d->ns; h.cur = d->cur;
  for (int k = 0; k < cdi::kMaxSpecies; k++) {
    h.z[k] = d->z[k];
    h.D[k] = d->D[k];
  }
  h.c0 = d->c0; h.Ka = d->Ka; h.dt = d->dt; h.VT = d->VT;
  h.U_lat = d->U_lat; h.U_target = d->U_target; h.tau = d->tau; h.force = d->force;
  h.flow_residual = d->flow_residual;
  h.flow_steps = d->flow_steps; h.np_steps = d->np_steps;
  h.psi_s = d->psi_s; h.eps_r = d->eps_r; h.psi_tol = d->psi_tol;
  h.psi_max_iter = d->psi_max_iter; h.couple_K = d->couple_K;
  char *out = static_cast<char *>(host_buf);
  std::memcpy(out, &h, sizeof(h));
  size_t off = sizeof(h);
  for (const Section &s : sections(d, d->cur)) {
    CDI_TRY(d, cudaMemcpyAsync(out + off, s.dev, s.bytes, cudaMemcpyDeviceToHost, d->stream),
            "save_state copy");
    off += s.bytes;
  }
  CDI_TRY(d, cudaStreamSynchronize(d->stream), "save_state");
  *bytes = off;
  return CDI_OK;
}

cdi_status cdi_load_state(cdi_domain *d, const void *host_buf, size_t bytes) {
  if (!d || !host_buf) return cdi_fail(d, CDI_ERR_INVALID_ARG, "NULL argument");
  if (bytes < sizeof(StateHeader))
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "load_state: buffer too small");
  StateHeader h;
  std::memcpy(&h, host_buf, sizeof(h));
  if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion)
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "load_state: not a state of this format");
  if (h.dim != d->dim || h.nx != d->nx || h.ny != d->ny || h.nz != d->nz ||
      h.walls != d->walls || h.mirror != d->mirror || h.prec != d->prec ||
      h.n_pore != d->n_pore || h.n_flow_pore != d->n_flow_pore || h.mask_hash != d->mask_hash)
    return cdi_fail(d, CDI_ERR_INVALID_ARG,
                    "load_state: the state belongs to another geometry or precision");
  if (h.ns < 0 || h.ns > cdi::kMaxSpecies || (h.cur != 0 && h.cur != 1) || h.couple_K < 0)
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "load_state: corrupt header");
  if (bytes != state_bytes(d))
    return cdi_fail(d, CDI_ERR_INVALID_ARG, "load_state: size does not match the domain");
  if (h.couple_K > 0 && !d->d_src) {
    d->d_src = (double *)cdi_dev_alloc(d, (size_t)d->N * 8);
    if (!d->d_src) return cdi_fail(d, CDI_ERR_OOM, "load_state: charge buffer");
  }
  // the loaded concentrations go to buffer 0; any captured graph is stale
  const char *in = static_cast<const char *>(host_buf);
  size_t off = sizeof(h);
  for (const Section &s : sections(d, 0)) {
    CDI_TRY(d, cudaMemcpyAsync(s.dev, in + off, s.bytes, cudaMemcpyHostToDevice, d->stream),
            "load_state copy");
    off += s.bytes;
  }
  CDI_TRY(d, cudaStreamSynchronize(d->stream), "load_state");
  if (d->np_graph) cudaGraphExecDestroy(d->np_graph);
  d->np_graph = nullptr;
  d->imp_stale = true;
  d->flow_done = h.flow_done != 0;
  d->psi_done = h.psi_done != 0;
  d->np_ready = h.np_ready != 0;
  d->ns = h.ns;
  d->cur = 0;
  for (int k = 0; k < cdi::kMaxSpecies; k++) {
    d->z[k] = h.z[k];
    d->D[k] = h.D[k];
  }
  d->c0 = h.c0; d->Ka = h.Ka; d->dt = h.dt; d->VT = h.VT;
  d->U_lat = h.U_lat; d->U_target = h.U_target; d->tau = h.tau; d->force = h.force;
  d->flow_residual = h.flow_residual;
  d->flow_steps = h.flow_steps; d->np_steps = h.np_steps;
  d->psi_s = h.psi_s; d->eps_r = h.eps_r; d->psi_tol = h.psi_tol;
  d->psi_max_iter = (int)h.psi_max_iter; d->couple_K = h.couple_K;
  return CDI_OK;
}

}  // extern "C"
