// Pore-site lists: the ascending indices of the pore sites of the flow grid
// and of the pore cells of the transport grid, built on the device by stream
// compaction of the flag words (solid bit 0).  The step kernels iterate over
// these lists so that every lane of a warp works on a pore site (a dense
// sweep leaves about half the lanes idle at porosity 0.5).
#include "cdi_internal.cuh"

using namespace cdi;

namespace {

constexpr int kCThreads = 256;
constexpr int kCRounds = 8;
constexpr int kChunk = kCThreads * kCRounds;  // elements per block

template <typename F>
__global__ void __launch_bounds__(kCThreads)
    k_count(const F *__restrict__ fl, long long n, int *__restrict__ counts) {
  const long long base = (long long)blockIdx.x * kChunk;
  int c = 0;
  for (int r = 0; r < kCRounds; r++) {
    const long long i = base + r * kCThreads + threadIdx.x;
    if (i < n && !(fl[i] & 1u)) c++;
  }
  __shared__ int sm[kCThreads / 32];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kCThreads / 32; w++) t += sm[w];
    counts[blockIdx.x] = t;
  }
}

// Exclusive scan of the chunk counts by one block (each thread scans a
// contiguous segment; the segment totals are scanned in order).
__global__ void __launch_bounds__(1024) k_scan(const int *__restrict__ counts, int nchunks,
                                               int *__restrict__ offsets) {
  __shared__ int seg[1024];
  const int per = (nchunks + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per, hi = min(lo + per, nchunks);
  int s = 0;
  for (int i = lo; i < hi; i++) s += counts[i];
  seg[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int t = 0; t < (int)blockDim.x; t++) {
      const int v = seg[t];
      seg[t] = run;
      run += v;
    }
  }
  __syncthreads();
  int run = seg[threadIdx.x];
  for (int i = lo; i < hi; i++) {
    offsets[i] = run;
    run += counts[i];
  }
}

template <typename F>
__global__ void __launch_bounds__(kCThreads)
    k_scatter(const F *__restrict__ fl, long long n, const int *__restrict__ offsets,
              int *__restrict__ list) {
  __shared__ int wtot[kCThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long base = (long long)blockIdx.x * kChunk;
  int out = offsets[blockIdx.x];
  for (int r = 0; r < kCRounds; r++) {
    const long long i = base + r * kCThreads + threadIdx.x;
    const bool p = i < n && !(fl[i] & 1u);
    const unsigned ballot = __ballot_sync(0xffffffffu, p);
    if (lane == 0) wtot[warp] = __popc(ballot);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kCThreads / 32; w++) {
      if (w < warp) before += wtot[w];
      total += wtot[w];
    }
    if (p) list[out + before + __popc(ballot & ((1u << lane) - 1u))] = (int)i;
    out += total;
    __syncthreads();
  }
}

template <typename F>
cdi_status compact(cdi_domain *d, const F *fl, long long n, int *list, int *work) {
  const int nchunks = (int)((n + kChunk - 1) / kChunk);
  int *counts = work, *offsets = work + nchunks;
  k_count<F><<<nchunks, kCThreads, 0, d->stream>>>(fl, n, counts);
  k_scan<<<1, 1024, 0, d->stream>>>(counts, nchunks, offsets);
  k_scatter<F><<<nchunks, kCThreads, 0, d->stream>>>(fl, n, offsets, list);
  d->timing.kernel_launches += 3;
  CDI_TRY(d, cudaGetLastError(), "pore lists");
  return CDI_OK;
}

}  // namespace

size_t cdi_lists_work_ints(long long n) { return 2 * (size_t)((n + kChunk - 1) / kChunk); }

cdi_status cdi_build_lists(cdi_domain *d, int *work) {
  cdi_status s;
  if (d->dim == 2)
    s = compact(d, (const FlowFlag<2>::type *)d->d_fflags, d->Nf, d->d_flow_list, work);
  else
    s = compact(d, (const FlowFlag<3>::type *)d->d_fflags, d->Nf, d->d_flow_list, work);
  if (s != CDI_OK) return s;
  return compact(d, d->d_nflags, d->N, d->d_cell_list, work);
}
