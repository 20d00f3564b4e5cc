// Stable LSD radix sort of (uint64 key, uint32 value) pairs, 8-bit digits,
// over the low `bits` bits of the key, one kernel per digit pass.
//
// One kernel first counts the digits of every pass over all items (the
// global histograms do not depend on the order).  Each pass kernel then
// claims tiles of kTile items in order from a counter and, per tile:
//   1. ranks its items per warp (below) and publishes the tile's digit
//      counts as "aggregate" words in the pass's status array;
//   2. looks back over the preceding tiles (a window of kWindow at a time), per digit, adding aggregates
//      until it meets a tile whose "inclusive prefix" word is published, then
//      publishes its own inclusive prefix (a chained scan with decoupled
//      look-back: a tile never waits on a later one, and every earlier tile
//      was claimed by a running CTA, so the waits end; each wait is bounded
//      and gives SBKI_ERR_TIMEOUT instead of spinning on);
//   3. scatters its items stably: each warp ranks its consecutive items
//      (rounds of 32) with warp matches on the digit and its own digit
//      counters, so equal keys keep their input order; the tile is staged in
//      shared memory in sorted order and written out so that consecutive
//      threads write consecutive positions of a digit's run.
// The last pass can also move a float4 payload: payload_out[pos] = payload[value].
// Destination of an item = (items of smaller digits) + (items of its digit in
// earlier tiles) + (its rank among its digit in this tile).
#include <algorithm>

#include "sbki_internal.cuh"

namespace sbki {
namespace {

constexpr int kRadix = 256;
constexpr int kHistThreads = 256;
constexpr int kThreads = 512;                          // one pass: 16 warps per tile
constexpr int kWarps = kThreads / 32;
constexpr int kRounds = kRadixTile / kThreads;         // rounds of 32 items per warp
constexpr uint32_t kAgg = 1u << 30;   // word holds this tile's count of the digit
constexpr uint32_t kPre = 2u << 30;   // word holds the count through this tile
constexpr uint32_t kValue = kAgg - 1u;
constexpr int kMaxSpin = 1 << 20;     // polls of unpublished status words before giving up
constexpr int kWindow = 16;           // predecessors read at once in the look-back

// layout of the work area (uint32): [2][ntiles][256] status (ping-pong by pass),
// [kMaxPasses][256] global digit counts, [kMaxPasses] tile counters
struct Work {
  uint32_t* status[2];
  uint32_t* ghist;
  uint32_t* tiles;
};

__host__ __device__ inline Work work_of(uint32_t* base, int64_t ntiles) {
  Work w;
  w.status[0] = base;
  w.status[1] = base + ntiles * kRadix;
  w.ghist = base + 2 * ntiles * kRadix;
  w.tiles = w.ghist + kMaxPasses * kRadix;
  return w;
}

// Global digit counts of every pass; also clears the status array of pass 0 and the tile counters.
__global__ void __launch_bounds__(kHistThreads) global_hist_kernel(const unsigned long long* __restrict__ keys,
                                                               const uint32_t* n_dev, int passes, Work w,
                                                               int64_t ntiles, const DevCounters* dc) {
  __shared__ uint32_t h[kMaxPasses][kRadix];
  for (int p = 0; p < passes; ++p) h[p][threadIdx.x] = 0;
  const int64_t stride = (int64_t)gridDim.x * kHistThreads;
  for (int64_t e = (int64_t)blockIdx.x * kHistThreads + threadIdx.x; e < ntiles * kRadix; e += stride) w.status[0][e] = 0;
  __syncthreads();
  const int64_t n = dc->err ? 0 : (int64_t)*n_dev;
  for (int64_t i = (int64_t)blockIdx.x * kHistThreads + threadIdx.x; i < n; i += stride) {
    const unsigned long long k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(uint32_t)(k >> (8 * p)) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  for (int p = 0; p < passes; ++p)
    if (h[p][threadIdx.x]) atomicAdd(&w.ghist[p * kRadix + threadIdx.x], h[p][threadIdx.x]);
}

__device__ __forceinline__ uint32_t load_volatile(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}
__device__ __forceinline__ void store_volatile(uint32_t* p, uint32_t v) { *reinterpret_cast<volatile uint32_t*>(p) = v; }

constexpr size_t kStageBytes = (size_t)kRadixTile * (sizeof(unsigned long long) + sizeof(uint32_t));

__global__ void __launch_bounds__(kThreads) onesweep_kernel(const unsigned long long* __restrict__ keys,
                                                            const uint32_t* __restrict__ vals,
                                                            unsigned long long* __restrict__ keys_out,
                                                            uint32_t* __restrict__ vals_out, const uint32_t* n_dev,
                                                            int pass, int64_t ntiles, Work w,
                                                            const float4* __restrict__ payload,
                                                            float4* __restrict__ payload_out, DevCounters* dc) {
  extern __shared__ __align__(16) unsigned char s_stage[];  // the tile in sorted order: keys, then values
  unsigned long long* s_k = reinterpret_cast<unsigned long long*>(s_stage);
  uint32_t* s_v = reinterpret_cast<uint32_t*>(s_k + kRadixTile);
  __shared__ uint32_t s_dbase[kRadix];         // items of smaller digits (this pass)
  __shared__ uint32_t s_base[kRadix];          // first output position of each digit in this tile
  __shared__ uint32_t s_tstart[kRadix];        // first position of each digit within the tile
  __shared__ uint32_t s_wc[kWarps][kRadix];    // per warp: digit counts, then the warp's offset in the digit
  __shared__ uint32_t s_wsum[kRadix / 32];
  __shared__ uint32_t s_tile;
  __shared__ int s_fail;
  const int shift = 8 * pass;
  uint32_t* status = (pass & 1) ? w.status[1] : w.status[0];  // no dynamic index into the parameter
  uint32_t* next = (pass & 1) ? w.status[0] : w.status[1];
  const int64_t n = dc->err ? 0 : (int64_t)*n_dev;
  const int64_t nt = (n + kRadixTile - 1) / kRadixTile;
  // the next pass's status array was last used by the previous pass, which has finished
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < nt * kRadix; e += (int64_t)gridDim.x * kThreads)
    next[e] = 0;
  const bool dthread = threadIdx.x < kRadix;  // threads 0..255 own one digit each
  {  // exclusive scan of the global counts over digits
    const uint32_t c = dthread ? w.ghist[pass * kRadix + threadIdx.x] : 0u;
    if (dthread) s_base[threadIdx.x] = c;
    __syncthreads();
    for (int o = 1; o < kRadix; o <<= 1) {
      const uint32_t t = (dthread && threadIdx.x >= (unsigned)o) ? s_base[threadIdx.x - o] : 0u;
      __syncthreads();
      if (dthread) s_base[threadIdx.x] += t;
      __syncthreads();
    }
    if (dthread) s_dbase[threadIdx.x] = s_base[threadIdx.x] - c;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_tile = atomicAdd(&w.tiles[pass], 1u);
      s_fail = 0;
    }
    for (int e = threadIdx.x; e < kWarps * kRadix; e += kThreads) (&s_wc[0][0])[e] = 0;
    __syncthreads();
    const int64_t t = s_tile;
    if (t >= nt) break;
    // 1. each warp ranks its 512 consecutive items (16 rounds of 32) by digit,
    //    stably, with warp matches and its own digit counters (no CTA barrier)
    const int64_t wbase = t * kRadixTile + (int64_t)warp * (kRounds * 32);
    unsigned long long kreg[kRounds];
    uint32_t vreg[kRounds], rreg[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const int64_t i = wbase + r * 32 + lane;
      const bool live = i < n;
      kreg[r] = live ? keys[i] : 0ull;
      vreg[r] = live ? vals[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const bool live = wbase + r * 32 + lane < n;
      const uint32_t d = live ? ((uint32_t)(kreg[r] >> shift) & (kRadix - 1)) : kRadix;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const int leader = __ffs(peers) - 1;
      uint32_t before = 0;
      if (live && lane == leader) {
        before = s_wc[warp][d];
        s_wc[warp][d] = before + __popc(peers);
      }
      rreg[r] = __shfl_sync(0xffffffffu, before, leader) + __popc(peers & lt_mask);
    }
    __syncthreads();
    // 2. per digit (one thread each): warp offsets, tile count, look-back
    if (dthread) {
      uint32_t cnt = 0;
#pragma unroll
      for (int k = 0; k < kWarps; ++k) {
        const uint32_t c = s_wc[k][threadIdx.x];
        s_wc[k][threadIdx.x] = cnt;
        cnt += c;
      }
      uint32_t* my = status + t * kRadix + threadIdx.x;
      uint32_t excl = 0;
      if (t == 0) {
        store_volatile(my, kPre | cnt);
      } else {
        store_volatile(my, kAgg | cnt);
        int64_t j = t - 1;
        int spins = 0;
        bool done = false;
        while (!done) {
          // a window of predecessors in flight at once, nearest first
          uint32_t win[kWindow];
#pragma unroll
          for (int k = 0; k < kWindow; ++k) win[k] = j - k >= 0 ? load_volatile(status + (j - k) * kRadix + threadIdx.x) : 0u;
          int used = 0;
          bool stop = false;
#pragma unroll
          for (int k = 0; k < kWindow; ++k) {
            if (!stop && !done) {
              const uint32_t v = win[k];
              if (j - k < 0 || (v & (kAgg | kPre)) == 0) {
                stop = true;  // not published yet: poll again from here
              } else {
                excl += v & kValue;
                ++used;
                done = (v & kPre) != 0;
              }
            }
          }
          if (done) break;
          j -= used;
          if (stop) {
            if (++spins > kMaxSpin) {
              s_fail = 1;
              break;
            }
            __nanosleep(20);
          }
        }
        store_volatile(my, kPre | (excl + cnt));
      }
        s_base[threadIdx.x] = s_dbase[threadIdx.x] + excl;
      // exclusive scan of the tile's digit counts (warps 0..7 hold the 256 digits)
      uint32_t inc = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
      }
      if (lane == 31) s_wsum[warp] = inc;
      s_tstart[threadIdx.x] = inc - cnt;  // within the warp; warp offsets added below
    }
    __syncthreads();
    if (s_fail) {
      if (threadIdx.x == 0) set_error(dc, SBKI_ERR_TIMEOUT);
      break;
    }
    if (dthread) {
      uint32_t off = 0;
      for (int k = 0; k < warp; ++k) off += s_wsum[k];
      s_tstart[threadIdx.x] += off;
    }
    __syncthreads();
    // 3. stage the tile in sorted order in shared memory ...
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      if (wbase + r * 32 + lane < n) {
        const uint32_t d = (uint32_t)(kreg[r] >> shift) & (kRadix - 1);
        const uint32_t lp = s_tstart[d] + s_wc[warp][d] + rreg[r];
        s_k[lp] = kreg[r];
        s_v[lp] = vreg[r];
      }
    }
    __syncthreads();
    // ... and write it out: consecutive threads write consecutive positions of a digit's run
    const int tile_n = (int)(n - t * kRadixTile < kRadixTile ? n - t * kRadixTile : kRadixTile);
    for (int j = threadIdx.x; j < tile_n; j += kThreads) {
      const unsigned long long key = s_k[j];
      const uint32_t val = s_v[j];
      const uint32_t d = (uint32_t)(key >> shift) & (kRadix - 1);
      const uint32_t pos = s_base[d] + (uint32_t)j - s_tstart[d];
      keys_out[pos] = key;
      vals_out[pos] = val;
      if (payload_out) payload_out[pos] = payload[val];
    }
  }
}

}  // namespace

int64_t radix_hist_entries(int64_t cap) { return radix_work_entries(cap); }

cudaError_t radix_sort_pairs(unsigned long long*& keys, uint32_t*& vals, unsigned long long*& keys_alt,
                             uint32_t*& vals_alt, const uint32_t* n_dev, int64_t cap, int bits, uint32_t* hist,
                             int sm_count, DevCounters* dc, cudaStream_t st, const float4* payload,
                             float4* payload_out) {
  if (cap <= 0 || bits <= 0) return cudaSuccess;
  const int passes = (bits + 7) / 8;
  if (passes > kMaxPasses) return cudaErrorInvalidValue;
  const int64_t ntiles = (cap + kRadixTile - 1) / kRadixTile;
  const Work w = work_of(hist, ntiles);
  cudaError_t e = cudaMemsetAsync(w.ghist, 0, sizeof(uint32_t) * (kMaxPasses * kRadix + kMaxPasses), st);
  if (e != cudaSuccess) return e;
  const int hgrid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)sm_count * 8));
  global_hist_kernel<<<hgrid, kHistThreads, 0, st>>>(keys, n_dev, passes, w, ntiles, dc);
  // persistent: as many CTAs as fit at once (tiles are claimed in order, so no CTA waits on one not running)
  e = cudaFuncSetAttribute(onesweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageBytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, onesweep_kernel, kThreads, kStageBytes);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)sm_count * std::max(1, per_sm)));
  for (int p = 0; p < passes; ++p) {
    const bool last = p == passes - 1;
    onesweep_kernel<<<grid, kThreads, kStageBytes, st>>>(keys, vals, keys_alt, vals_alt, n_dev, p, ntiles, w,
                                                         last ? payload : nullptr, last ? payload_out : nullptr, dc);
    std::swap(keys, keys_alt);
    std::swap(vals, vals_alt);
  }
  return cudaGetLastError();
}

cudaError_t radix_wait_selftest(unsigned long long* keys, uint32_t* vals, unsigned long long* keys_out,
                                uint32_t* vals_out, uint32_t* n_dev, uint32_t* work, DevCounters* dc, cudaStream_t st) {
  const int64_t ntiles = (kSelftestItems + kRadixTile - 1) / kRadixTile;
  const Work w = work_of(work, ntiles);
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(uint32_t) * radix_work_entries(kSelftestItems), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * kSelftestItems, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(vals, 0, sizeof(uint32_t) * kSelftestItems, st);
  const uint32_t one = 1u, items = (uint32_t)kSelftestItems;
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.tiles, &one, sizeof(one), cudaMemcpyHostToDevice, st);  // skip tile 0
  if (e == cudaSuccess) e = cudaMemcpyAsync(n_dev, &items, sizeof(items), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(onesweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageBytes);
  if (e != cudaSuccess) return e;
  onesweep_kernel<<<2, kThreads, kStageBytes, st>>>(keys, vals, keys_out, vals_out, n_dev, 0, ntiles, w, nullptr,
                                                    nullptr, dc);
  return cudaGetLastError();
}

}  // namespace sbki
