// Stable LSD radix sort of (uint64 key, uint32 value) pairs, 8-bit digits,
// over the low `bits` bits of the key.  Per pass: a per-tile digit histogram,
// a device-wide exclusive scan of the digit-major histogram, and a stable
// scatter in which every tile ranks its items in index order (warp
// match + per-warp digit counts), so equal keys keep their input order.
#include "sbki_internal.cuh"

namespace sbki {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRounds = 16;
constexpr int kTile = kThreads * kRounds;  // items per CTA
constexpr int kRadix = 256;

__global__ void __launch_bounds__(kThreads) digit_hist(const unsigned long long* __restrict__ keys,
                                                       const uint32_t* n_dev, int shift, int ntiles,
                                                       uint32_t* __restrict__ hist, const DevCounters* dc) {
  __shared__ uint32_t h[kRadix];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t n = *n_dev;
  const int64_t base = (int64_t)blockIdx.x * kTile;
  if (dc->err == 0) {
    for (int r = 0; r < kRounds; ++r) {
      int64_t i = base + r * kThreads + threadIdx.x;
      if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & (kRadix - 1)], 1u);
    }
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) digit_scatter(const unsigned long long* __restrict__ keys,
                                                          const uint32_t* __restrict__ vals,
                                                          unsigned long long* __restrict__ keys_out,
                                                          uint32_t* __restrict__ vals_out, const uint32_t* n_dev,
                                                          int shift, int ntiles, const uint32_t* __restrict__ hist,
                                                          const DevCounters* dc) {
  __shared__ uint32_t base_s[kRadix];
  __shared__ uint32_t wc[kWarps][kRadix];
  if (dc->err) return;
  const int64_t n = *n_dev;
  const int64_t tbase = (int64_t)blockIdx.x * kTile;
  if (tbase >= n) return;
  base_s[threadIdx.x] = hist[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int r = 0; r < kRounds; ++r) {
    int64_t i = tbase + r * kThreads + threadIdx.x;
    if (tbase + r * kThreads >= n) break;  // uniform over the CTA
#pragma unroll
    for (int k = 0; k < kWarps; ++k) wc[k][threadIdx.x] = 0;
    __syncthreads();
    bool live = i < n;
    unsigned long long key = live ? keys[i] : 0ull;
    uint32_t val = live ? vals[i] : 0u;
    uint32_t d = live ? ((uint32_t)(key >> shift) & (kRadix - 1)) : kRadix;
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = __popc(peers & lt_mask);
    if (live && rank == 0) wc[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t acc = base_s[threadIdx.x];
#pragma unroll
      for (int k = 0; k < kWarps; ++k) {
        uint32_t t = wc[k][threadIdx.x];
        wc[k][threadIdx.x] = acc;
        acc += t;
      }
      base_s[threadIdx.x] = acc;
    }
    __syncthreads();
    if (live) {
      uint32_t pos = wc[warp][d] + rank;
      keys_out[pos] = key;
      vals_out[pos] = val;
    }
    __syncthreads();
  }
}

}  // namespace

int64_t radix_hist_entries(int64_t cap) { return (int64_t)kRadix * ((cap + kTile - 1) / kTile) + 1; }

cudaError_t radix_sort_pairs(unsigned long long* keys, uint32_t* vals, unsigned long long* keys_alt,
                             uint32_t* vals_alt, const uint32_t* n_dev, int64_t cap, int bits, uint32_t* hist,
                             void* scan_tmp, DevCounters* dc, cudaStream_t st) {
  if (cap <= 0 || bits <= 0) return cudaSuccess;
  const int ntiles = (int)((cap + kTile - 1) / kTile);
  const int passes = (bits + 7) / 8;
  unsigned long long *ks = keys, *kd = keys_alt;
  uint32_t *vs = vals, *vd = vals_alt;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    digit_hist<<<ntiles, kThreads, 0, st>>>(ks, n_dev, shift, ntiles, hist, dc);
    cudaError_t e = exclusive_scan_u32(hist, (int64_t)kRadix * ntiles, scan_tmp, st);
    if (e != cudaSuccess) return e;
    digit_scatter<<<ntiles, kThreads, 0, st>>>(ks, vs, kd, vd, n_dev, shift, ntiles, hist, dc);
    unsigned long long* tk = ks;
    ks = kd;
    kd = tk;
    uint32_t* tv = vs;
    vs = vd;
    vd = tv;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ks != keys) {  // odd number of passes: result lives in the alternate buffers
    e = cudaMemcpyAsync(keys, ks, sizeof(unsigned long long) * cap, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(vals, vs, sizeof(uint32_t) * cap, cudaMemcpyDeviceToDevice, st);
  }
  return e;
}

}  // namespace sbki
