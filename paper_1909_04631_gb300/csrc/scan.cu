// Device-wide exclusive prefix sums: reduce, scan of tile totals, downsweep
// (three launches, no inter-CTA waiting), and a one-pass form (below) for the
// prefix sum of every update.  Both deterministic (integer sums).
#include <algorithm>

#include "sbki_internal.cuh"

namespace sbki {
namespace {

constexpr int kThreads = 256;
constexpr int kIpt = 8;
constexpr int kTile = kThreads * kIpt;
static_assert(scan_tmp_bytes_ce(kTile) == 24 * 3, "scratch sizing assumes tiles of 2048");
static_assert(kScanSelftestItems == 3 * kTile, "self-test: three tiles");

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

// One-pass form: tiles are claimed in order from a counter; each publishes its
// sum ("aggregate", flag 1), then warp 0 looks back over the preceding tiles
// 32 at a time, adding aggregates until it meets an inclusive prefix (flag 2),
// and publishes its own inclusive prefix (a chained scan with decoupled
// look-back: a tile waits only on earlier tiles, all claimed by running CTAs).
// A value is written before its flag with a fence between, and read after it.
// A wait that outlasts kMaxSpin polls sets SBKI_ERR_TIMEOUT and publishes
// anyway, so no later tile waits on it.  tmp: [counter, pad] u32, flags
// u32[ntiles_cap], then aggregates and inclusive prefixes T[ntiles_cap] each
// (flags and counter zero on entry).
constexpr int kMaxSpin = 1 << 20;

template <typename T>
__device__ __forceinline__ T vload(const T* p) { return *reinterpret_cast<const volatile T*>(p); }
template <typename T>
__device__ __forceinline__ void vstore(T* p, T v) { *reinterpret_cast<volatile T*>(p) = v; }

struct OnePass {
  uint32_t* ctr;
  uint32_t* flags;
  void* agg;
  void* incl;
};
__host__ __device__ inline OnePass onepass_of(void* tmp, int64_t ntiles_cap) {
  OnePass o;
  o.ctr = static_cast<uint32_t*>(tmp);
  o.flags = o.ctr + 2;
  unsigned char* v = reinterpret_cast<unsigned char*>(o.flags + ntiles_cap + (ntiles_cap & 1));  // 8-byte aligned
  o.agg = v;
  o.incl = v + 8 * ntiles_cap;
  return o;
}

// the grand total of the per-point sample counts: hits, free samples, items (capacity check)
__device__ __forceinline__ void finish_counts(unsigned long long total, int64_t items_cap, DevCounters* dc) {
  const uint32_t nv = (uint32_t)(total >> 40);
  const unsigned long long nf = total & kFreeMask;
  dc->n_valid = nv;
  dc->n_free = nf;
  const unsigned long long items = (unsigned long long)nv + nf;
  if (items > (unsigned long long)items_cap) {
    set_error(dc, SBKI_ERR_CAPACITY);
    dc->n_items = 0;
  } else {
    dc->n_items = (uint32_t)items;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) scan_onepass(T* data, int64_t cap, const uint32_t* n_dev, OnePass o,
                                                         DevCounters* dc, int64_t items_cap) {
  __shared__ T tile[kTile];
  __shared__ T warp_tot[kThreads / 32];
  __shared__ T total;
  __shared__ T s_excl;
  __shared__ uint32_t s_t;
  T* agg = static_cast<T*>(o.agg);
  T* incl = static_cast<T*>(o.incl);
  const int64_t n = count_of(cap, n_dev);
  const int64_t nt = (n + kTile - 1) / kTile;
  if (nt == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    data[0] = T(0);
    if (items_cap >= 0) finish_counts(0ull, items_cap, dc);
  }
  const int lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) s_t = atomicAdd(o.ctr, 1u);
    __syncthreads();
    const int64_t t = s_t;
    if (t >= nt) break;
    const int64_t base = t * kTile;
    for (int i = threadIdx.x; i < kTile; i += kThreads) tile[i] = base + i < n ? data[base + i] : T(0);
    __syncthreads();
    T loc[kIpt];
    T sum = 0;
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
      loc[k] = tile[threadIdx.x * kIpt + k];
      sum += loc[k];
    }
    T ex = block_exclusive_scan<T>(sum, warp_tot, &total);
    if (threadIdx.x < 32) {  // warp 0: publish, look back, publish the inclusive prefix
      const T tsum = total;
      T prefix = 0;
      if (t == 0) {
        if (lane == 0) {
          vstore(incl, tsum);
          __threadfence();
          vstore(o.flags, 2u);
        }
      } else {
        if (lane == 0) {
          vstore(agg + t, tsum);
          __threadfence();
          vstore(o.flags + t, 1u);
        }
        int64_t j = t - 1;  // nearest predecessor not yet added
        int spins = 0;
        for (;;) {
          const int64_t q = j - lane;
          const uint32_t f = q >= 0 ? vload(o.flags + q) : 2u;
          const unsigned pre = __ballot_sync(0xffffffffu, f == 2u);
          const unsigned none = __ballot_sync(0xffffffffu, f == 0u);
          const int stop = pre ? __ffs((int)pre) - 1 : 31;  // lanes 0..stop are needed
          const unsigned need = stop == 31 ? 0xffffffffu : ((2u << stop) - 1u);
          if (none & need) {  // a needed predecessor has not published yet
            if (++spins > kMaxSpin) {
              if (lane == 0) set_error(dc, SBKI_ERR_TIMEOUT);
              break;
            }
            __nanosleep(20);
            continue;
          }
          __threadfence();
          T v = 0;
          if (lane <= stop && q >= 0) v = f == 2u ? vload(incl + q) : vload(agg + q);
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
          prefix += v;
          if (pre) break;
          j -= 32;
        }
        if (lane == 0) {
          vstore(incl + t, prefix + tsum);
          __threadfence();
          vstore(o.flags + t, 2u);
        }
      }
      if (lane == 0) s_excl = prefix;
    }
    __syncthreads();
    ex += s_excl;
#pragma unroll
    for (int k = 0; k < kIpt; ++k) {
      tile[threadIdx.x * kIpt + k] = ex;
      ex += loc[k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kTile; i += kThreads)
      if (base + i < n) data[base + i] = tile[i];
    if (t == nt - 1 && threadIdx.x == 0) {
      data[n] = s_excl + total;
      if (items_cap >= 0) finish_counts((unsigned long long)(s_excl + total), items_cap, dc);
    }
    __syncthreads();
  }
}

}  // namespace

int64_t scan_tmp_bytes(int64_t n) { return scan_tmp_bytes_ce(n); }

cudaError_t scan_wait_selftest(unsigned long long* data, void* tmp, DevCounters* dc, cudaStream_t st) {
  const int64_t n = kScanSelftestItems, nt = (n + kTile - 1) / kTile;
  const OnePass o = onepass_of(tmp, nt);
  cudaError_t e = cudaMemsetAsync(tmp, 0, sizeof(uint32_t) * (2 + nt), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(data, 0, sizeof(unsigned long long) * (n + 1), st);
  const uint32_t one = 1u;
  if (e == cudaSuccess) e = cudaMemcpyAsync(o.ctr, &one, sizeof(one), cudaMemcpyHostToDevice, st);  // skip tile 0
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // `one` lives on this stack frame
  if (e != cudaSuccess) return e;
  scan_onepass<unsigned long long><<<2, kThreads, 0, st>>>(data, n, nullptr, o, dc, -1);
  return cudaGetLastError();
}

cudaError_t exclusive_scan_u64_onepass(unsigned long long* data, int64_t n, void* tmp, cudaStream_t st,
                                       const uint32_t* n_dev, int sm_count, DevCounters* dc, int64_t items_cap) {
  if (n <= 0) n = 0;  // the kernel writes data[0] = 0 (and the counts) for an empty input
  const int64_t nt = (n + kTile - 1) / kTile;
  const OnePass o = onepass_of(tmp, nt);
  cudaError_t e = cudaMemsetAsync(tmp, 0, sizeof(uint32_t) * (2 + nt), st);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nt, (int64_t)sm_count * 4));
  scan_onepass<unsigned long long><<<grid, kThreads, 0, st>>>(data, n, n_dev, o, dc, items_cap);
  return cudaGetLastError();
}

cudaError_t exclusive_scan_u32(uint32_t* data, int64_t n, void* tmp, cudaStream_t st, const uint32_t* n_dev) {
  return scan_impl<uint32_t>(data, n, tmp, st, n_dev);
}
cudaError_t exclusive_scan_u64(unsigned long long* data, int64_t n, void* tmp, cudaStream_t st, const uint32_t* n_dev) {
  return scan_impl<unsigned long long>(data, n, tmp, st, n_dev);
}

}  // namespace sbki
