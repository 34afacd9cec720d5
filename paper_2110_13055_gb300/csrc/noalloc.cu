// Allocation-free transport sums: the dissolved amount and the outlet
// concentration of caller-owned device fields, computed without any device
// allocation by the library.
//
// Who needs this: programs that own every byte of device memory through
// their own pool or arena and do not let a library call cudaMalloc (host
// applications embedding the solver under a fixed memory budget, services
// that forbid allocation once they are serving, plugins running inside
// another program's memory manager), and loops where a cudaMalloc/cudaFree
// pair would synchronise the device in the middle of the work.
//
// How: the reduction's block partials and its completion counter live in one
// file-scope static device array of fixed size.  Every GPU that loads the
// library holds its own copy of that array until the process exits.  All
// calls on a device share it and it keeps the last call's contents, so the
// counter is cleared on the stream at the start of each call, and calls whose
// work overlaps on the GPU (two streams at once, or two host threads) race on
// it: serialise them.
#include <mutex>

#include "cdi_internal.cuh"

using namespace cdi;

namespace {

constexpr int kNaBlocks = 304;                 // reduction grid: 2 blocks per SM
constexpr int kNaValues = 3 * kMaxSpecies + 2; // per block: mass[4], sum u_x C[4],
                                               // sum u_x, plain sum C[4], count
constexpr size_t kNaPartials = (size_t)kNaBlocks * kNaValues;
constexpr size_t kNaDoubles = kNaPartials + 32;  // + the counter, padded
constexpr int kNaMaxDevices = 64;

// The scratch: kNaDoubles * 8 = 34,304 bytes per device.
static __device__ __align__(256) double g_na_scratch[kNaDoubles];

std::mutex g_na_mutex;
double *g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch on the current device.  The name of the
// array is only a host-side handle, so the address is looked up once per
// device (with that device current) and cached.  A cudaDeviceReset destroys
// the context that held the array, and with it the cached address: this
// entry point is not for use after a reset in the same process.
cudaError_t na_scratch(double **p) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void *q = nullptr;
    e = cudaGetSymbolAddress(&q, g_na_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = static_cast<double *>(q);
  }
  *p = g_na_ptr[dev];
  return cudaSuccess;
}

// Same reduction as the transport sums of a domain, on FP64 fields passed by
// the caller; partials and counter in the static scratch.
__global__ void __launch_bounds__(kRedThreads)
    k_sums_noalloc(const double *__restrict__ C, const double *__restrict__ ux,
                   const uint8_t *__restrict__ mask, long long N, int nx, int ns,
                   double cell_vol, double *__restrict__ scratch, double *__restrict__ out) {
  constexpr int NV = kNaValues;
  __shared__ double sm[NV * 32];
  double *part = scratch;
  unsigned int *counter = reinterpret_cast<unsigned int *>(scratch + kNaPartials);
  double v[NV];
#pragma unroll
  for (int j = 0; j < NV; j++) v[j] = 0.0;
  // grid-stride loop; the x coordinate advances by the stride modulo nx, so
  // no division per cell
  const long long P0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int dxs = (int)(stride % nx);
  int x = (int)(P0 % nx);
  for (long long P = P0; P < N; P += stride) {
    if (!mask[P]) {
      const bool outlet = x == nx - 1;
      const double u = outlet ? ux[P] : 0.0;  // the velocity only weights the outlet
      for (int k = 0; k < ns; k++) {
        const double ck = C[(size_t)k * N + P];
        v[k] += ck;
        if (outlet) {
          v[kMaxSpecies + k] += u * ck;
          v[2 * kMaxSpecies + 1 + k] += ck;
        }
      }
      if (outlet) {
        v[2 * kMaxSpecies] += u;
        v[NV - 1] += 1.0;
      }
    }
    x += dxs;
    if (x >= nx) x -= nx;
  }
  block_reduce<NV>(v, sm, OpSum(), 0.0);
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < NV; j++) part[(size_t)j * gridDim.x + blockIdx.x] = v[j];
  if (last_block(counter, gridDim.x)) {
    combine_partials<NV>(part, gridDim.x, v, sm, OpSum(), 0.0);
    if (threadIdx.x == 0) {
      const double sum_u = v[2 * kMaxSpecies], cnt = v[NV - 1];
      for (int k = 0; k < ns; k++) {
        out[k] = v[k] * cell_vol;
        out[ns + k] = sum_u != 0.0 ? v[kMaxSpecies + k] / sum_u
                                   : (cnt > 0.0 ? v[2 * kMaxSpecies + 1 + k] / cnt : 0.0);
      }
      *counter = 0;
    }
  }
}

}  // namespace

extern "C" cdi_status cdi_transport_sums_noalloc(const double *C, const double *ux,
                                                 const uint8_t *mask, int dim, int nx, int ny,
                                                 int nz, int n_species, double dx_m,
                                                 double *out, void *stream) {
  if (!C || !ux || !mask || !out)
    return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "noalloc sums: NULL pointer");
  if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || nz < 1 || (dim == 2 && nz != 1))
    return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "noalloc sums: bad grid size");
  if (n_species < 1 || n_species > kMaxSpecies)
    return cdi_fail(nullptr, CDI_ERR_INVALID_ARG,
                    "noalloc sums: n_species must be 1..4 (the fixed scratch holds the "
                    "partial sums of at most 4 species)");
  if (!(dx_m > 0.0)) return cdi_fail(nullptr, CDI_ERR_INVALID_ARG, "noalloc sums: dx_m <= 0");
  double *scratch = nullptr;
  cudaError_t e = na_scratch(&scratch);
  if (e != cudaSuccess) return cdi_cuda_fail(nullptr, e, "noalloc sums: scratch address");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  e = cudaMemsetAsync(scratch + kNaPartials, 0, sizeof(double), st);  // the counter
  if (e != cudaSuccess) return cdi_cuda_fail(nullptr, e, "noalloc sums: clear counter");
  const long long N = (long long)nx * ny * nz;
  const double vol = dim == 2 ? dx_m * dx_m : dx_m * dx_m * dx_m;
  k_sums_noalloc<<<kNaBlocks, kRedThreads, 0, st>>>(C, ux, mask, N, nx, n_species, vol,
                                                     scratch, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cdi_cuda_fail(nullptr, e, "noalloc sums: launch");
  return CDI_OK;
}
