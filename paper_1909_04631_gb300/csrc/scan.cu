// Device-wide exclusive prefix sums (reduce, scan of tile totals, downsweep).
// Three launches, no inter-CTA waiting, deterministic.
#include "sbki_internal.cuh"

namespace sbki {
namespace {

constexpr int kThreads = 256;
constexpr int kIpt = 8;
constexpr int kTile = kThreads * kIpt;

template <typename T>
__device__ T block_exclusive_scan(T v, T* warp_tot, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < kThreads / 32 ? warp_tot[lane] : T(0);
    T winc = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T t = __shfl_up_sync(0xffffffffu, winc, o);
      if (lane >= o) winc += t;
    }
    if (lane < kThreads / 32) warp_tot[lane] = winc - w;
    if (lane == kThreads / 32 - 1) *total = winc;
  }
  __syncthreads();
  return warp_tot[warp] + inc - v;
}

// element count: the launch bound n, or the device count *n_dev (<= n) when given
__device__ __forceinline__ int64_t count_of(int64_t n, const uint32_t* n_dev) {
  return n_dev ? min(n, (int64_t)*n_dev) : n;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) scan_reduce(const T* __restrict__ data, int64_t cap, T* partial,
                                                        const uint32_t* n_dev) {
  __shared__ T warp_tot[kThreads / 32];
  __shared__ T total;
  const int64_t n = count_of(cap, n_dev);
  const int64_t base = (int64_t)blockIdx.x * kTile;
  if (base >= n) return;  // uniform over the CTA
  T s = 0;
  for (int i = threadIdx.x; i < kTile; i += kThreads) {
    int64_t idx = base + i;
    if (idx < n) s += data[idx];
  }
  block_exclusive_scan<T>(s, warp_tot, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// single CTA: exclusive scan of the tile totals, grand total to data[n]
template <typename T>
__global__ void __launch_bounds__(kThreads) scan_partials(T* partial, T* data, int64_t cap, const uint32_t* n_dev) {
  __shared__ T warp_tot[kThreads / 32];
  __shared__ T total;
  const int64_t n = count_of(cap, n_dev);
  const int64_t nparts = (n + kTile - 1) / kTile;
  T carry = 0;
  for (int64_t base = 0; base < nparts; base += kThreads) {
    int64_t i = base + threadIdx.x;
    T v = i < nparts ? partial[i] : T(0);
    T ex = block_exclusive_scan<T>(v, warp_tot, &total);
    if (i < nparts) partial[i] = carry + ex;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) data[n] = carry;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) scan_down(T* data, int64_t cap, const T* __restrict__ partial,
                                                      const uint32_t* n_dev) {
  __shared__ T tile[kTile];
  __shared__ T warp_tot[kThreads / 32];
  __shared__ T total;
  const int64_t n = count_of(cap, n_dev);
  const int64_t base = (int64_t)blockIdx.x * kTile;
  if (base >= n) return;  // uniform over the CTA
  for (int i = threadIdx.x; i < kTile; i += kThreads) {
    int64_t idx = base + i;
    tile[i] = idx < n ? data[idx] : T(0);
  }
  __syncthreads();
  T loc[kIpt];
  T s = 0;
#pragma unroll
  for (int k = 0; k < kIpt; ++k) {
    loc[k] = tile[threadIdx.x * kIpt + k];
    s += loc[k];
  }
  T ex = block_exclusive_scan<T>(s, warp_tot, &total) + partial[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kIpt; ++k) {
    tile[threadIdx.x * kIpt + k] = ex;
    ex += loc[k];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kTile; i += kThreads) {
    int64_t idx = base + i;
    if (idx < n) data[idx] = tile[i];
  }
}

template <typename T>
cudaError_t scan_impl(T* data, int64_t n, void* tmp, cudaStream_t st, const uint32_t* n_dev) {
  if (n <= 0) {
    return cudaMemsetAsync(data, 0, sizeof(T), st);
  }
  int64_t tiles = (n + kTile - 1) / kTile;
  T* partial = (T*)tmp;
  scan_reduce<T><<<(unsigned)tiles, kThreads, 0, st>>>(data, n, partial, n_dev);
  scan_partials<T><<<1, kThreads, 0, st>>>(partial, data, n, n_dev);
  scan_down<T><<<(unsigned)tiles, kThreads, 0, st>>>(data, n, partial, n_dev);
  return cudaGetLastError();
}

}  // namespace

int64_t scan_tmp_bytes(int64_t n) { return ((n + kTile - 1) / kTile + 1) * (int64_t)sizeof(unsigned long long); }

cudaError_t exclusive_scan_u32(uint32_t* data, int64_t n, void* tmp, cudaStream_t st, const uint32_t* n_dev) {
  return scan_impl<uint32_t>(data, n, tmp, st, n_dev);
}
cudaError_t exclusive_scan_u64(unsigned long long* data, int64_t n, void* tmp, cudaStream_t st, const uint32_t* n_dev) {
  return scan_impl<unsigned long long>(data, n, tmp, st, n_dev);
}

}  // namespace sbki
