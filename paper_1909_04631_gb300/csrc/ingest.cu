// Steps a1-a3 of the per-scan update (Sec. III): transform and validate the
// hits, generate the free-space samples along every beam, and downsample hits
// and samples to one centroid per (downsampling cell, label).
//
// Every operation that decides an integer (which points survive, how many
// samples a beam gets, which cell a point falls in) uses round-to-nearest
// intrinsics in a fixed order, so the compiler cannot contract or reorder it:
//   world  = fp32( ((r0 px + r1 py) + r2 pz) + t )      (FP64, then one rounding)
//   r      = sqrt( (dx dx + dy dy) + dz dz ),  d = h - o  (FP32)
//   t_j    = r - fp32(j) * s,   sample = o + d * (t_j / r) (FP32), j >= 1 while t_j > 0
//   cell   = floor( x * fp32(1/ds) )                       (FP32)
// The centroid of a cell is, per axis, the exact mean of its members'
// coordinates rounded once to FP32 (see the centroid kernels).
#include <algorithm>
#include <climits>

#include "sbki_internal.cuh"

namespace sbki {
namespace {

constexpr unsigned long long kValidOne = 1ull << 40;
constexpr unsigned long long kFreeMask = kValidOne - 1;


__device__ __forceinline__ int floor_i(float v) { return (int)floorf(v); }

// sort key: [scan | rel tile x | rel tile y | rel tile z | local cell (z,y,x) | label]
__device__ __forceinline__ unsigned long long make_key(float x, float y, float z, int label, const Geom& g,
                                                       const KeyFrame& kf, const int32_t org[3], int scan,
                                                       DevCounters* dc) {
  int gx = floor_i(__fmul_rn(x, g.inv_ds));
  int gy = floor_i(__fmul_rn(y, g.inv_ds));
  int gz = floor_i(__fmul_rn(z, g.inv_ds));
  int tx = (gx >> kTileShift) - org[0];
  int ty = (gy >> kTileShift) - org[1];
  int tz = (gz >> kTileShift) - org[2];
  if (tx < 0 || ty < 0 || tz < 0 || tx >= (1 << kf.bits[0]) || ty >= (1 << kf.bits[1]) || tz >= (1 << kf.bits[2])) {
    set_error(dc, SBKI_ERR_INVALID_ARG);
    tx = ty = tz = 0;
  }
  const unsigned long long tile = ((unsigned long long)tx << (kf.bits[1] + kf.bits[2])) |
                                  ((unsigned long long)ty << kf.bits[2]) | (unsigned long long)tz;
  unsigned long long local = (unsigned long long)(((gz & (kTileEdge - 1)) << (2 * kTileShift)) |
                                                  ((gy & (kTileEdge - 1)) << kTileShift) | (gx & (kTileEdge - 1)));
  const unsigned long long k = (((tile << kLocalBits) | local) << g.label_bits) | (unsigned long long)label;
  return kf.scan_bits ? (k | ((unsigned long long)scan << kf.total_bits)) : k;
}
__device__ __forceinline__ unsigned long long make_key(float x, float y, float z, int label, const Geom& g,
                                                       const KeyFrame& kf, DevCounters* dc) {
  return make_key(x, y, z, label, g, kf, kf.org, 0, dc);
}

// scan of global point gi: the last s with off[s] <= gi (empty scans are skipped)
__device__ __forceinline__ int scan_of(const int64_t* off, int ns, int64_t gi) {
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= gi) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// the map index a training point's segment belongs to
__device__ __forceinline__ int map_of_segment(unsigned long long key, const KeyFrame& kf, const ScanDesc* desc) {
  return desc[kf.scan_bits ? (int)(key >> kf.total_bits) : 0].map_id;
}

// number of j >= 1 with fp32(j) * s < r  (the set is a prefix since fp32(j)*s is monotone in j)
__device__ __forceinline__ uint32_t free_count(float r, float s) {
  if (!(r > 0.0f)) return 0;
  float q = __fdiv_rn(r, s);
  int j = q < 1.6e7f ? (int)q : 16000000;
  for (int it = 0; it < 4 && j > 0 && !(__fmul_rn((float)j, s) < r); ++it) --j;
  for (int it = 0; it < 4 && __fmul_rn((float)(j + 1), s) < r; ++it) ++j;
  return (uint32_t)(j < 0 ? 0 : j);
}

// a1 for global point i of scan d
__device__ __forceinline__ void transform_count_one(const ScanDesc& d, int64_t i, const int64_t* off, const Geom& g,
                                                    float4* __restrict__ world, unsigned long long* __restrict__ cnt,
                                                    DevCounters* dc, int tlo[3], int thi[3]) {
  const int64_t li = i - d.off;
  const float px = d.pts[3 * li], py = d.pts[3 * li + 1], pz = d.pts[3 * li + 2];
  const int lab = d.labels[li];
  if (lab < 1 || lab > g.K1 - 1) set_error(dc, SBKI_ERR_LABEL_RANGE);
  bool ok = isfinite(px) && isfinite(py) && isfinite(pz);
  unsigned long long c = 0;
  float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
  if (ok) {
    const double dx = px, dy = py, dz = pz;
    const double range = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    ok = range >= g.min_range && range <= g.max_range;
    if (ok) {
      float wc[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        double acc = __dmul_rn(d.r[3 * r], dx);
        acc = __dadd_rn(acc, __dmul_rn(d.r[3 * r + 1], dy));
        acc = __dadd_rn(acc, __dmul_rn(d.r[3 * r + 2], dz));
        acc = __dadd_rn(acc, d.t[r]);
        wc[r] = __double2float_rn(acc);
      }
      const float ex = __fsub_rn(wc[0], d.o[0]);
      const float ey = __fsub_rn(wc[1], d.o[1]);
      const float ez = __fsub_rn(wc[2], d.o[2]);
      const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
      const float rr = __fsqrt_rn(r2);
      c = kValidOne | (unsigned long long)free_count(rr, g.step);
      w = make_float4(wc[0], wc[1], wc[2], (float)lab);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int t = floor_i(__fmul_rn(wc[a], g.inv_ds)) >> kTileShift;
        tlo[a] = min(tlo[a], t);
        thi[a] = max(thi[a], t);
      }
    }
  }
  world[i] = w;
  cnt[i] = c;
}

// Steps a1 (and the free-sample counts of a2) for every point of every scan
// of the update; points are numbered globally, scan after scan.
__global__ void __launch_bounds__(256) transform_count_kernel(const ScanDesc* __restrict__ desc, int ns, Geom g,
                                                               float4* __restrict__ world,
                                                               unsigned long long* __restrict__ cnt, DevCounters* dc) {
  __shared__ int64_t s_off[kMaxScans + 1];
  __shared__ int s_box[6];
  for (int t = threadIdx.x; t <= ns; t += blockDim.x) s_off[t] = desc[t].off;
  if (threadIdx.x < 6) s_box[threadIdx.x] = threadIdx.x < 3 ? INT_MAX : INT_MIN;
  __syncthreads();
  const int64_t total = s_off[ns];
  int tlo[3] = {INT_MAX, INT_MAX, INT_MAX}, thi[3] = {INT_MIN, INT_MIN, INT_MIN};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    transform_count_one(desc[scan_of(s_off, ns, i)], i, s_off, g, world, cnt, dc, tlo, thi);
  // tile bounding box of the kept hits: warp, then CTA, then one global atomic per CTA and bound
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int lo = __reduce_min_sync(0xffffffffu, tlo[a]), hi = __reduce_max_sync(0xffffffffu, thi[a]);
    if ((threadIdx.x & 31) == 0 && lo <= hi) {
      atomicMin(&s_box[a], lo);
      atomicMax(&s_box[3 + a], hi);
    }
  }
  __syncthreads();
  if (threadIdx.x < 3 && s_box[threadIdx.x] <= s_box[3 + threadIdx.x]) {
    atomicMin(&dc->tbox[threadIdx.x], s_box[threadIdx.x]);
    atomicMax(&dc->tbox[3 + threadIdx.x], s_box[3 + threadIdx.x]);
  }
}

__global__ void check_counts_kernel(const unsigned long long* cnt, int64_t cap, DevCounters* dc) {
  const unsigned long long tot = cnt[dc->n_points];
  const uint32_t nv = (uint32_t)(tot >> 40);
  const unsigned long long nf = tot & kFreeMask;
  dc->n_valid = nv;
  dc->n_free = nf;
  const unsigned long long items = (unsigned long long)nv + nf;
  if (items > (unsigned long long)cap) {
    set_error(dc, SBKI_ERR_CAPACITY);
    dc->n_items = 0;
  } else {
    dc->n_items = (uint32_t)items;
  }
}

// Step a2 for every scan of the update: one warp per 32 consecutive points
// (which may belong to different scans); the warp writes each beam's samples
// together.  Hits go to items [0, hits), free samples after all hits.
__global__ void __launch_bounds__(256) emit_kernel(const float4* __restrict__ world,
                                                   const unsigned long long* __restrict__ cnt,
                                                   const ScanDesc* __restrict__ desc, int ns, Geom g, KeyFrame kf,
                                                   float4* __restrict__ items, unsigned long long* __restrict__ keys,
                                                   uint32_t* __restrict__ vals, DevCounters* dc) {
  __shared__ int64_t s_off[kMaxScans + 1];
  for (int t = threadIdx.x; t <= ns; t += blockDim.x) s_off[t] = desc[t].off;
  __syncthreads();
  if (dc->err) return;
  const int64_t n = s_off[ns];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned long long nvalid = cnt[n] >> 40;
  for (int64_t base = warp * 32; base < n; base += nwarps * 32) {
    const int64_t i = base + lane;
    uint32_t nfree = 0;
    unsigned long long fpos = 0;
    float ex = 0.f, ey = 0.f, ez = 0.f, rr = 0.f, ox = 0.f, oy = 0.f, oz = 0.f;
    int sc = 0, og[3] = {0, 0, 0};
    if (i < n) {
      sc = scan_of(s_off, ns, i);
      const ScanDesc& d = desc[sc];
      ox = d.o[0];
      oy = d.o[1];
      oz = d.o[2];
      og[0] = d.org[0];
      og[1] = d.org[1];
      og[2] = d.org[2];
      const unsigned long long c0 = cnt[i], c1 = cnt[i + 1];
      if ((c1 >> 40) != (c0 >> 40)) {  // a kept hit
        const float4 w = world[i];
        const unsigned long long hpos = c0 >> 40;
        items[hpos] = w;
        keys[hpos] = make_key(w.x, w.y, w.z, (int)w.w, g, kf, og, sc, dc);
        vals[hpos] = (uint32_t)hpos;
        nfree = (uint32_t)((c1 & kFreeMask) - (c0 & kFreeMask));
        fpos = nvalid + (c0 & kFreeMask);
        ex = __fsub_rn(w.x, ox);
        ey = __fsub_rn(w.y, oy);
        ez = __fsub_rn(w.z, oz);
        rr = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez)));
      }
    }
    for (int src = 0; src < 32; ++src) {
      const uint32_t m = __shfl_sync(0xffffffffu, nfree, src);
      if (m == 0) continue;
      const float sx = __shfl_sync(0xffffffffu, ex, src);
      const float sy = __shfl_sync(0xffffffffu, ey, src);
      const float sz = __shfl_sync(0xffffffffu, ez, src);
      const float sr = __shfl_sync(0xffffffffu, rr, src);
      const float qx = __shfl_sync(0xffffffffu, ox, src);
      const float qy = __shfl_sync(0xffffffffu, oy, src);
      const float qz = __shfl_sync(0xffffffffu, oz, src);
      const int32_t sorg[3] = {__shfl_sync(0xffffffffu, og[0], src), __shfl_sync(0xffffffffu, og[1], src),
                               __shfl_sync(0xffffffffu, og[2], src)};
      const int ssc = __shfl_sync(0xffffffffu, sc, src);
      const unsigned long long sp = __shfl_sync(0xffffffffu, fpos, src);
      for (uint32_t j = lane + 1; j <= m; j += 32) {
        const float t = __fsub_rn(sr, __fmul_rn((float)j, g.step));
        const float q = __fdiv_rn(t, sr);
        const float x = __fadd_rn(qx, __fmul_rn(sx, q));
        const float y = __fadd_rn(qy, __fmul_rn(sy, q));
        const float z = __fadd_rn(qz, __fmul_rn(sz, q));
        const unsigned long long pos = sp + j - 1;
        items[pos] = make_float4(x, y, z, 0.f);
        keys[pos] = make_key(x, y, z, 0, g, kf, sorg, ssc, dc);
        vals[pos] = (uint32_t)pos;
      }
    }
  }
}

// Segments of the sorted items in one pass: tiles of kSegTile items are claimed
// in order; each counts its segment heads (key differs from its predecessor),
// publishes the count, finds the heads before it by a warp-wide look-back over
// up to 32 preceding tiles at once (bounded waits, SBKI_ERR_TIMEOUT), and
// writes seg_start[head index] = item index.  The tile holding the last item
// writes seg_start[P] = n and the segment count P.  work: [ntiles] status words
// then a tile counter, zero on entry.
constexpr int kSegThreads = 512;
constexpr int kSegPer = 8;
constexpr int kSegTile = kSegThreads * kSegPer;
constexpr uint32_t kSegAgg = 1u << 30, kSegPre = 2u << 30, kSegVal = kSegAgg - 1u;

__global__ void __launch_bounds__(kSegThreads) seg_heads_kernel(const unsigned long long* __restrict__ keys,
                                                               int64_t cap, uint32_t* __restrict__ seg_start,
                                                               uint32_t* __restrict__ work, int64_t ntiles_cap,
                                                               DevCounters* dc) {
  __shared__ uint32_t s_wsum[kSegThreads / 32];
  __shared__ uint32_t s_tile, s_excl;
  __shared__ int s_fail;
  if (dc->err) return;
  const int64_t n = min(cap, (int64_t)dc->n_items);
  const int64_t nt = (n + kSegTile - 1) / kSegTile;
  uint32_t* status = work;
  uint32_t* counter = work + ntiles_cap;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_tile = atomicAdd(counter, 1u);
      s_fail = 0;
    }
    __syncthreads();
    const int64_t t = s_tile;
    if (t >= nt) break;
    const int64_t first = t * kSegTile + (int64_t)threadIdx.x * kSegPer;
    uint32_t heads = 0;  // bit k: item first + k starts a segment
    unsigned long long prev = first > 0 && first <= n ? keys[first - 1] : 0ull;
#pragma unroll
    for (int k = 0; k < kSegPer; ++k) {
      const int64_t i = first + k;
      if (i < n) {
        const unsigned long long key = keys[i];
        if (i == 0 || key != prev) heads |= 1u << k;
        prev = key;
      }
    }
    // exclusive prefix of the head counts over the CTA's threads
    const uint32_t c = __popc(heads);
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    uint32_t wpre = 0, total = 0;
#pragma unroll
    for (int k = 0; k < kSegThreads / 32; ++k) {
      const uint32_t v = s_wsum[k];
      wpre += k < warp ? v : 0u;
      total += v;
    }
    // the tile's place among all heads: publish, then one warp looks back 32 tiles at a time
    if (warp == 0) {
      uint32_t excl = 0;
      if (t == 0) {
        if (lane == 0) *reinterpret_cast<volatile uint32_t*>(status) = kSegPre | total;
      } else {
        if (lane == 0) *reinterpret_cast<volatile uint32_t*>(status + t) = kSegAgg | total;
        int64_t j = t - 1;
        int spins = 0;
        for (;;) {
          const int64_t q = j - lane;
          const uint32_t v = q >= 0 ? *reinterpret_cast<const volatile uint32_t*>(status + q) : kSegPre;
          const unsigned pre = __ballot_sync(0xffffffffu, (v & kSegPre) != 0);
          const unsigned ready = __ballot_sync(0xffffffffu, (v & (kSegAgg | kSegPre)) != 0);
          const int stop = pre ? __ffs(pre) - 1 : 31;  // nearest inclusive prefix in the window
          const unsigned need = stop == 31 ? 0xffffffffu : ((2u << stop) - 1u);
          if ((ready & need) == need) {  // every word up to it is published
            uint32_t part = lane <= stop ? (v & kSegVal) : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            excl += part;
            if (pre) break;
            j -= 32;
          } else if (++spins > (1 << 20)) {
            if (lane == 0) s_fail = 1;
            break;
          } else {
            __nanosleep(20);
          }
        }
        if (lane == 0) *reinterpret_cast<volatile uint32_t*>(status + t) = kSegPre | (excl + total);
      }
      if (lane == 0) s_excl = excl;
    }
    __syncthreads();
    if (s_fail) {
      if (threadIdx.x == 0) set_error(dc, SBKI_ERR_TIMEOUT);
      break;
    }
    uint32_t idx = s_excl + wpre + inc - c;
#pragma unroll
    for (int k = 0; k < kSegPer; ++k)
      if (heads & (1u << k)) seg_start[idx++] = (uint32_t)(first + k);
    if (first <= n - 1 && n - 1 < first + kSegPer) {  // this thread holds the last item
      seg_start[s_excl + total] = (uint32_t)n;
      dc->n_train = s_excl + total;
    }
  }
}

// Centroids: per axis the exact mean of the members' FP32 coordinates,
// rounded once to FP32 (nearest, ties to even).  No floating point is used:
// every nonzero |x| is m 2^e with an integer m < 2^24 and e = its exponent of
// the last mantissa bit; with E the smallest such e in the cell,
//     sum |x| = T 2^E,   T = sum m 2^(e - E)
// is an integer held exactly in 128 bits whenever the members' e span fewer
// than 127 - 24 - ceil(log2 n) binades (cells next to a coordinate plane
// included), and the mean is T 2^E / n, rounded with integer division.  The
// members of a cell share a sign per axis (the cell index fixes it).  Cells
// beyond that span, or whose mean is below the FP32 normal range, take a
// one-thread path with 512-bit arithmetic (exact for every FP32 input).
// Short segments (<= kShort members) are summed by one lane
// (centroid_kernel), longer ones by a warp (mid_centroid_kernel), the longest
// (> kHuge) by a whole CTA (huge_centroid_kernel).
constexpr uint32_t kShort = 16;
constexpr uint32_t kHuge = 1024;

struct U128 {
  unsigned long long lo, hi;
};

__device__ __forceinline__ float axis_of(const float4& p, int ax) { return ax == 0 ? p.x : (ax == 1 ? p.y : p.z); }

// member i of the sorted order: items already in sorted order (perm null) or gathered through perm
__device__ __forceinline__ float4 item_at(const float4* __restrict__ items, const uint32_t* __restrict__ perm, uint32_t i) {
  return perm ? items[perm[i]] : items[i];
}

// |v| = m 2^e (m < 2^24 integer); returns false for zero
__device__ __forceinline__ bool decompose(float v, unsigned& m, int& e) {
  const unsigned b = __float_as_uint(v) & 0x7fffffffu;
  if (b == 0u) return false;
  const unsigned E = b >> 23;
  m = (b & 0x7fffffu) | (E ? 0x800000u : 0u);
  e = E ? (int)E - 150 : -149;
  return true;
}

__device__ __forceinline__ void u128_add(U128& t, unsigned long long lo, unsigned long long hi) {
  t.lo += lo;
  t.hi += hi + (t.lo < lo ? 1ull : 0ull);
}

// t += m 2^sh, 0 <= sh <= 103
__device__ __forceinline__ void u128_add_shifted(U128& t, unsigned long long m, int sh) {
  if (sh == 0) u128_add(t, m, 0ull);
  else if (sh < 64) u128_add(t, m << sh, m >> (64 - sh));
  else u128_add(t, 0ull, m << (sh - 64));
}

__device__ __forceinline__ int bitlen64(unsigned long long v) { return v ? 64 - __clzll((long long)v) : 0; }

struct AxisAcc {
  int emin, emax;  // range of the members' last-mantissa-bit exponents
  bool neg;
  __device__ void init() {
    emin = 1 << 20;
    emax = -(1 << 20);
    neg = false;
  }
  __device__ void see(float v) {
    unsigned m;
    int e;
    if (decompose(v, m, e)) {
      emin = min(emin, e);
      emax = max(emax, e);
      neg |= v < 0.0f;
    }
  }
  __device__ bool empty() const { return emax < emin; }
  __device__ bool fits(uint32_t n) const {  // T stays below 2^127
    int lg = 0;
    while ((1u << lg) < n) ++lg;
    return empty() || emax - emin + 24 + lg <= 126;
  }
  __device__ void add(U128& t, float v) const {
    unsigned m;
    int e;
    if (decompose(v, m, e)) u128_add_shifted(t, m, e - emin);
  }
};

// round(T 2^s / n) to FP32; false when the result is below the normal range
__device__ bool round_mean(U128 T, unsigned long long n, int s, float& out) {
  const int bt = T.hi ? 64 + bitlen64(T.hi) : bitlen64(T.lo);
  const int bn = bitlen64(n);
  const int k = 26 + bn - bt;  // q = floor(T 2^k / n) in [2^24, 2^27)
  unsigned long long q;
  bool sticky;
  if (k >= 0) {
    const unsigned long long num = T.lo << k;  // bt + k = 26 + bn <= 58 bits
    q = num / n;
    sticky = num - q * n != 0ull;
  } else {
    const int m = -k;
    unsigned long long ts, lost;
    if (m < 64) {
      ts = (T.lo >> m) | (m ? (T.hi << (64 - m)) : 0ull);
      lost = T.lo & ((1ull << m) - 1ull);
    } else {
      ts = T.hi >> (m - 64);
      lost = T.lo | (T.hi & ((m - 64 == 0) ? 0ull : ((1ull << (m - 64)) - 1ull)));
    }
    q = ts / n;
    sticky = lost != 0ull || ts - q * n != 0ull;
  }
  const int qb = bitlen64(q);
  if (qb - 1 - k + s < -126) return false;
  const int sh = qb - 24;
  unsigned long long mant = q >> sh;
  const unsigned long long rb = q & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  if (rb > half || (rb == half && (sticky || (mant & 1ull)))) mant += 1ull;
  int e = sh - k + s;
  if (mant == (1ull << 24)) {
    mant >>= 1;
    e += 1;
  }
  out = ldexpf((float)mant, e);
  return true;
}

// One thread: exact mean of axis ax of members [a, b) for any FP32 input.
// The sum is held in 16 32-bit limbs in units of 2^-149 (512 bits).
__device__ float wide_mean(const float4* __restrict__ items, const uint32_t* __restrict__ perm, uint32_t a,
                           uint32_t b, int ax) {
  uint32_t w[16];
  for (int i = 0; i < 16; ++i) w[i] = 0u;
  bool neg = false;
  for (uint32_t i = a; i < b; ++i) {
    const float v = axis_of(item_at(items, perm, i), ax);
    unsigned m;
    int e;
    if (!decompose(v, m, e)) continue;
    neg |= v < 0.0f;
    const int sh = e + 149, li = sh >> 5, bi = sh & 31;
    unsigned long long add = (unsigned long long)m << bi;  // < 2^55
    for (int j = li; j < 16 && add; ++j) {
      const unsigned long long t = (unsigned long long)w[j] + (add & 0xffffffffull);
      w[j] = (uint32_t)t;
      add = (add >> 32) + (t >> 32);
    }
  }
  const unsigned long long n = b - a;
  // quotient of (sum 2^96) / n, limb by limb from the top, in 19 limbs
  uint32_t q[19];
  unsigned long long r = 0ull;
  for (int j = 18; j >= 0; --j) {
    const unsigned long long cur = (r << 32) | (j >= 3 ? w[j - 3] : 0u);
    q[j] = (uint32_t)(cur / n);
    r = cur - (unsigned long long)q[j] * n;
  }
  int qb = 0;
  for (int j = 18; j >= 0 && !qb; --j)
    if (q[j]) qb = 32 * j + 32 - __clz((int)q[j]);
  if (qb == 0) return 0.0f;
  // value = q 2^(-149 - 96); keep 24 bits, fewer for a subnormal result
  const int lead = qb - 1 - 245;
  int keep = lead < -126 ? 24 - (-126 - lead) : 24;
  if (keep < 0) keep = 0;
  const int drop = qb - keep;
  auto bit = [&](int i) -> unsigned { return i >= 0 ? (q[i >> 5] >> (i & 31)) & 1u : 0u; };
  unsigned long long mant = 0ull;
  for (int i = qb - 1; i >= drop; --i) mant = (mant << 1) | bit(i);
  bool sticky = r != 0ull;
  for (int i = 0; i < drop - 1 && !sticky; ++i) sticky = bit(i) != 0u;
  if (bit(drop - 1) && (sticky || (mant & 1ull))) mant += 1ull;
  const float f = ldexpf((float)mant, drop - 245);
  return neg ? -f : f;
}

__device__ float finish_axis(const AxisAcc& s, bool fits, U128 T, uint32_t n, const float4* items,
                             const uint32_t* perm, uint32_t a, uint32_t b, int ax) {
  if (s.empty()) return 0.0f;
  float f;
  if (fits && round_mean(T, n, s.emin, f)) return s.neg ? -f : f;
  return wide_mean(items, perm, a, b, ax);
}

// Single-pass form for an axis whose first member x0 has |x0| >= 2.5 ds: every
// member of the cell lies within ds (plus rounding) of x0, so it has x0's sign
// and its last mantissa bit's exponent is within [e0 - 1, e0 + 1] (e0: x0's);
// in units of 2^E, E = e0 - 1, every |x| is an integer below 2^26 and a 64-bit
// sum is exact for fewer than 2^32 members.  Cells near a coordinate plane
// (|x0| < 2.5 ds) take the two-pass AxisAcc path.
struct FastAxis {
  bool on, neg;
  int E;
  unsigned long long T;
  __device__ void init(float x0, float lim) {
    unsigned m;
    int e;
    on = fabsf(x0) >= lim && decompose(x0, m, e);
    neg = x0 < 0.0f;
    E = on ? e - 1 : 0;
    T = 0ull;
  }
  __device__ void add(float v) {
    unsigned m;
    int e;
    decompose(v, m, e);  // v != 0: |v| > ds
    T += (unsigned long long)m << (e - E);
  }
  __device__ float finish(uint32_t n) const {
    U128 t;
    t.lo = T;
    t.hi = 0ull;
    float f = 0.0f;
    round_mean(t, n, E, f);
    return neg ? -f : f;
  }
};

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ U128 warp_sum_u128(U128 t) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long lo = __shfl_xor_sync(0xffffffffu, t.lo, o);
    const unsigned long long hi = __shfl_xor_sync(0xffffffffu, t.hi, o);
    u128_add(t, lo, hi);
  }
  return t;
}

__device__ __forceinline__ void warp_range(AxisAcc& s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s.emin = min(s.emin, __shfl_xor_sync(0xffffffffu, s.emin, o));
    s.emax = max(s.emax, __shfl_xor_sync(0xffffffffu, s.emax, o));
  }
  s.neg = __any_sync(0xffffffffu, s.neg);
}

__global__ void __launch_bounds__(256) centroid_kernel(const unsigned long long* __restrict__ keys,
                                                       const uint32_t* __restrict__ perm,
                                                       const float4* __restrict__ items,
                                                       const uint32_t* __restrict__ seg_start, Geom g,
                                                       float4* __restrict__ train, const ScanDesc* __restrict__ desc,
                                                       KeyFrame kf, uint32_t* __restrict__ huge,
                                                       uint32_t* __restrict__ mid, DevCounters* dc) {
  if (dc->err) return;
  const uint32_t P = dc->n_train;
  const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nthreads = gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const uint32_t warp = gtid >> 5, nwarps = nthreads >> 5;
  for (uint32_t base = warp * 32; base < P; base += nwarps * 32) {
    const uint32_t s = base + lane;
    const bool valid = s < P;
    const uint32_t a = valid ? seg_start[s] : 0, b = valid ? seg_start[s + 1] : 0;
    const uint32_t n = b - a;
    const bool is_huge = valid && n > kHuge;
    if (is_huge) huge[atomicAdd(&dc->n_huge, 1u)] = s;
    AxisAcc ax[3];
    FastAxis fa[3];
    U128 T[3];
    bool fit[3] = {false, false, false};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ax[c].init();
      T[c].lo = T[c].hi = 0ull;
    }
    if (valid && n <= kShort) {
      const float4 p0 = item_at(items, perm, a);
#pragma unroll
      for (int c = 0; c < 3; ++c) fa[c].init(axis_of(p0, c), g.fast_lim);
      for (uint32_t i = a; i < b; ++i) {
        const float4 p = i == a ? p0 : item_at(items, perm, i);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (fa[c].on) fa[c].add(axis_of(p, c));
          else ax[c].see(axis_of(p, c));
        }
      }
      if (!fa[0].on || !fa[1].on || !fa[2].on) {  // a cell next to a coordinate plane
#pragma unroll
        for (int c = 0; c < 3; ++c) fit[c] = !fa[c].on && ax[c].fits(n);
        for (uint32_t i = a; i < b; ++i) {
          const float4 p = item_at(items, perm, i);
#pragma unroll
          for (int c = 0; c < 3; ++c)
            if (fit[c]) ax[c].add(T[c], axis_of(p, c));
        }
      }
    }
    const bool is_mid = valid && n > kShort && !is_huge;
    if (is_mid) mid[atomicAdd(&dc->n_mid, 1u)] = s;
    if (valid && n <= kShort) {
      const unsigned long long k = keys[a];
      const int label = (int)(k & ((1ull << g.label_bits) - 1));
      float out[3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        out[c] = fa[c].on ? fa[c].finish(n) : finish_axis(ax[c], fit[c], T[c], n, items, perm, a, b, c);
      train[s] = make_float4(out[0], out[1], out[2], (float)(label + 32 * map_of_segment(k, kf, desc)));
    }
  }
}

// Segments of kShort+1 .. kHuge members: one warp each, spread over the grid
// (neighbouring cells near the sensor are all long; a warp per group of 32
// consecutive cells would serialise them).
__global__ void __launch_bounds__(256) mid_centroid_kernel(const unsigned long long* __restrict__ keys,
                                                           const uint32_t* __restrict__ perm,
                                                           const float4* __restrict__ items,
                                                           const uint32_t* __restrict__ seg_start, Geom g,
                                                           float4* __restrict__ train,
                                                           const ScanDesc* __restrict__ desc, KeyFrame kf,
                                                           const uint32_t* __restrict__ mid, DevCounters* dc) {
  if (dc->err) return;
  const uint32_t nm = dc->n_mid;
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t j = warp; j < nm; j += nwarps) {
    const uint32_t s = mid[j];
    const uint32_t a = seg_start[s], b = seg_start[s + 1], n = b - a;
    AxisAcc w[3];
    FastAxis fa[3];
    U128 t[3];
    const float4 p0 = item_at(items, perm, a);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      w[c].init();
      t[c].lo = t[c].hi = 0ull;
      fa[c].init(axis_of(p0, c), g.fast_lim);
    }
    const bool slow = !fa[0].on || !fa[1].on || !fa[2].on;  // warp-uniform
    for (uint32_t i = a + lane; i < b; i += 32) {
      const float4 p = item_at(items, perm, i);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (fa[c].on) fa[c].add(axis_of(p, c));
        else w[c].see(axis_of(p, c));
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (fa[c].on) fa[c].T = warp_sum_u64(fa[c].T);
    bool fit[3] = {false, false, false};
    if (slow) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        warp_range(w[c]);
        fit[c] = !fa[c].on && w[c].fits(n);
      }
      for (uint32_t i = a + lane; i < b; i += 32) {
        const float4 p = item_at(items, perm, i);
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (fit[c]) w[c].add(t[c], axis_of(p, c));
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) t[c] = warp_sum_u128(t[c]);
    }
    if (lane == 0) {
      float out[3];
      for (int c = 0; c < 3; ++c)
        out[c] = fa[c].on ? fa[c].finish(n) : finish_axis(w[c], fit[c], t[c], n, items, perm, a, b, c);
      const unsigned long long k = keys[a];
      const int label = (int)(k & ((1ull << g.label_bits) - 1));
      train[s] = make_float4(out[0], out[1], out[2], (float)(label + 32 * map_of_segment(k, kf, desc)));
    }
  }
}

// Segments of more than kHuge members (cells next to the sensor): one CTA
// each, same arithmetic as centroid_kernel.
__global__ void __launch_bounds__(256) huge_centroid_kernel(const unsigned long long* __restrict__ keys,
                                                            const uint32_t* __restrict__ perm,
                                                            const float4* __restrict__ items,
                                                            const uint32_t* __restrict__ seg_start, Geom g,
                                                            float4* __restrict__ train,
                                                            const ScanDesc* __restrict__ desc, KeyFrame kf,
                                                            const uint32_t* __restrict__ huge, DevCounters* dc) {
  __shared__ int s_emin[3][8], s_emax[3][8], s_neg[3][8];
  __shared__ unsigned long long s_lo[3][8], s_hi[3][8];
  if (dc->err) return;
  const uint32_t nh = dc->n_huge;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t h = blockIdx.x; h < nh; h += gridDim.x) {
    const uint32_t s = huge[h];
    const uint32_t a = seg_start[s], b = seg_start[s + 1], n = b - a;
    AxisAcc w[3];
    FastAxis fa[3];
    const float4 p0 = item_at(items, perm, a);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      w[c].init();
      fa[c].init(axis_of(p0, c), g.fast_lim);
    }
    const bool slow = !fa[0].on || !fa[1].on || !fa[2].on;  // CTA-uniform
    {
      uint32_t i = a + threadIdx.x;
      for (; i + 768 < b; i += 1024) {  // four independent gathers in flight
        const float4 ps[4] = {item_at(items, perm, i), item_at(items, perm, i + 256), item_at(items, perm, i + 512), item_at(items, perm, i + 768)};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            if (fa[c].on) fa[c].add(axis_of(ps[u], c));
            else w[c].see(axis_of(ps[u], c));
          }
      }
      for (; i < b; i += 256) {
        const float4 p = item_at(items, perm, i);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (fa[c].on) fa[c].add(axis_of(p, c));
          else w[c].see(axis_of(p, c));
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (fa[c].on) {
        const unsigned long long tsum = warp_sum_u64(fa[c].T);
        if (lane == 0) {
          s_lo[c][warp] = tsum;
          s_hi[c][warp] = 0ull;
        }
      }
    }
    bool fit[3] = {false, false, false};
    if (slow) {  // an axis next to a coordinate plane: range first, then the 128-bit sums
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        warp_range(w[c]);
        if (lane == 0) {
          s_emin[c][warp] = w[c].emin;
          s_emax[c][warp] = w[c].emax;
          s_neg[c][warp] = w[c].neg ? 1 : 0;
        }
      }
      __syncthreads();
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        int mn = 1 << 20, mx = -(1 << 20), ng = 0;
        for (int k = 0; k < 8; ++k) {
          mn = min(mn, s_emin[c][k]);
          mx = max(mx, s_emax[c][k]);
          ng |= s_neg[c][k];
        }
        w[c].emin = mn;
        w[c].emax = mx;
        w[c].neg = ng != 0;
        fit[c] = !fa[c].on && w[c].fits(n);
      }
      U128 t[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) t[c].lo = t[c].hi = 0ull;
      for (uint32_t i = a + threadIdx.x; i < b; i += 256) {
        const float4 p = item_at(items, perm, i);
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (fit[c]) w[c].add(t[c], axis_of(p, c));
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (!fa[c].on) {
          t[c] = warp_sum_u128(t[c]);
          if (lane == 0) {
            s_lo[c][warp] = t[c].lo;
            s_hi[c][warp] = t[c].hi;
          }
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float out[3];
      for (int c = 0; c < 3; ++c) {
        U128 tt;
        tt.lo = tt.hi = 0ull;
        for (int k = 0; k < 8; ++k) u128_add(tt, s_lo[c][k], s_hi[c][k]);
        if (fa[c].on) {
          fa[c].T = tt.lo;
          out[c] = fa[c].finish(n);
        } else {
          out[c] = finish_axis(w[c], fit[c], tt, n, items, perm, a, b, c);
        }
      }
      const unsigned long long k = keys[a];
      const int label = (int)(k & ((1ull << g.label_bits) - 1));
      train[s] = make_float4(out[0], out[1], out[2], (float)(label + 32 * map_of_segment(k, kf, desc)));
    }
    __syncthreads();
  }
}

// --- given training sets (no sampling or downsampling) ---------------------

__global__ void train_bbox_kernel(const float4* __restrict__ in, int64_t p, Geom g, int* bbox, DevCounters* dc) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p) return;
  const float4 v = in[i];
  const int lab = (int)v.w;
  if (!(v.w == (float)lab) || lab < 0 || lab > g.K1 - 1) set_error(dc, SBKI_ERR_LABEL_RANGE);
  if (!isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z)) {
    set_error(dc, SBKI_ERR_INVALID_ARG);
    return;
  }
  const float c[3] = {v.x, v.y, v.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float q = __fmul_rn(c[a], g.inv_ds);
    if (!(fabsf(q) < 1.0e6f)) {
      set_error(dc, SBKI_ERR_INVALID_ARG);
      return;
    }
    int t = floor_i(q) >> kTileShift;
    atomicMin(&bbox[a], t);
    atomicMax(&bbox[3 + a], t);
  }
}

__global__ void train_keys_kernel(const float4* __restrict__ in, int64_t p, Geom g, KeyFrame kf,
                                  unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals,
                                  DevCounters* dc) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p || dc->err) return;
  const float4 v = in[i];
  keys[i] = make_key(v.x, v.y, v.z, (int)v.w, g, kf, dc);
  vals[i] = (uint32_t)i;
}

// every point is its own segment; gather into tile order, tag the map index
__global__ void train_gather_kernel(const float4* __restrict__ in, const uint32_t* __restrict__ perm, int64_t p,
                                    int map_id, float4* __restrict__ train, uint32_t* __restrict__ seg_start,
                                    DevCounters* dc) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p || dc->err) return;
  float4 v = in[perm[s]];
  v.w = __fadd_rn(v.w, (float)(32 * map_id));  // exact: label < 32, map < 64
  train[s] = v;
  seg_start[s] = (uint32_t)s;
  if (s == p - 1) {
    seg_start[p] = (uint32_t)p;
    dc->n_train = (uint32_t)p;
  }
}

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

// Steps a1-a2 count for the ns scans described in m.s.desc; total_n bounds the
// point count, which the kernels read on the device (dc->n_points, desc[ns].off).
cudaError_t launch_transform_count(MapState& m, int ns, int64_t total_n) {
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(grid_for(total_n, 256), (int64_t)m.sm_count * m.tune.ingest_ctas_per_sm));
  transform_count_kernel<<<blocks, 256, 0, m.stream>>>(m.s.desc, ns, m.g, m.s.world, m.s.cnt, m.dc);
  m.launches += 1 + 3 + 1;  // transform, scan, check
  cudaError_t e = exclusive_scan_u64(m.s.cnt, total_n, m.s.scan_tmp, m.stream, &m.dc->n_points);
  if (e != cudaSuccess) return e;
  check_counts_kernel<<<1, 1, 0, m.stream>>>(m.s.cnt, m.s.s_cap, m.dc);
  return cudaGetLastError();
}

cudaError_t launch_emit(MapState& m, int ns, int64_t total_n, const KeyFrame& kf) {
  const int64_t warps = (total_n + 31) / 32;
  unsigned blocks = (unsigned)std::min<int64_t>((warps + 7) / 8, (int64_t)m.sm_count * m.tune.ingest_ctas_per_sm);
  if (blocks == 0) blocks = 1;
  emit_kernel<<<blocks, 256, 0, m.stream>>>(m.s.world, m.s.cnt, m.s.desc, ns, m.g, kf, m.s.items, m.s.keys, m.s.vals,
                                            m.dc);
  m.launches += 1;
  return cudaGetLastError();
}

// Sorts the items and reduces each (scan, cell, label) segment to its centroid.
// nitems: host-known bound on the item count (the count itself is read on the device).
cudaError_t launch_downsample_n(MapState& m, const KeyFrame& kf, int64_t nitems) {
  Scratch& s = m.s;
  const int bits = kf.total_bits + kf.scan_bits;
  m.launches += 1 + (bits + 7) / 8 + 1 + 3;  // sort, segments, centroids
  // the last pass also moves the items into sorted order (s.sitems), so the centroids read them in a stream
  cudaError_t e = radix_sort_pairs(s.keys, s.vals, s.keys2, s.vals2, &m.dc->n_items, nitems, bits, s.hist,
                                   m.sm_count, m.dc, m.stream, s.items, s.sitems);
  if (e != cudaSuccess) return e;
  {  // segments in one pass; s.flags holds its tile status words and counter
    const int64_t stiles = (nitems + kSegTile - 1) / kSegTile;
    e = cudaMemsetAsync(s.flags, 0, sizeof(uint32_t) * (stiles + 1), m.stream);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, seg_heads_kernel, kSegThreads, 0);
    if (e != cudaSuccess) return e;
    const unsigned sblocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(stiles, (int64_t)m.sm_count * std::max(1, per_sm)));
    seg_heads_kernel<<<sblocks, kSegThreads, 0, m.stream>>>(s.keys, nitems, s.seg_start, s.flags, stiles, m.dc);
  }
  {
    const unsigned cblocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nitems + 255) / 256, (int64_t)m.sm_count * m.tune.ingest_ctas_per_sm));
    centroid_kernel<<<cblocks, 256, 0, m.stream>>>(s.keys, nullptr, s.sitems, s.seg_start, m.g, s.train, s.desc, kf,
                                                   s.huge, s.mid, m.dc);
    mid_centroid_kernel<<<(unsigned)(m.sm_count * std::max(1, m.tune.ingest_ctas_per_sm / 2)), 256, 0, m.stream>>>(s.keys, nullptr, s.sitems, s.seg_start, m.g,
                                                                        s.train, s.desc, kf, s.mid, m.dc);
    huge_centroid_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(nitems / kHuge + 1, 1024)), 256, 0,
                           m.stream>>>(s.keys, nullptr, s.sitems, s.seg_start, m.g, s.train, s.desc, kf, s.huge, m.dc);
  }
  return cudaGetLastError();
}

cudaError_t launch_train_bbox(MapState& m, const float4* in, int64_t p, int* bbox_dev) {
  train_bbox_kernel<<<grid_for(p, 256), 256, 0, m.stream>>>(in, p, m.g, bbox_dev, m.dc);
  m.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_train_prepare(MapState& m, const float4* in, int64_t p, const KeyFrame& kf) {
  Scratch& s = m.s;
  m.launches += 1 + 1 + (kf.total_bits + 7) / 8 + 1;
  train_keys_kernel<<<grid_for(p, 256), 256, 0, m.stream>>>(in, p, m.g, kf, s.keys, s.vals, m.dc);
  cudaError_t e = radix_sort_pairs(s.keys, s.vals, s.keys2, s.vals2, &m.dc->n_items, p, kf.total_bits, s.hist,
                                   m.sm_count, m.dc, m.stream);
  if (e != cudaSuccess) return e;
  train_gather_kernel<<<grid_for(p, 256), 256, 0, m.stream>>>(in, s.vals, p, m.active_map, s.train, s.seg_start,
                                                               m.dc);
  return cudaGetLastError();
}

// Failure-detection self-test: the segment pass over three tiles whose tile
// counter starts at 1, so tile 0 is never claimed and the look-back of the
// others runs out; they must end with SBKI_ERR_TIMEOUT instead of spinning on.
// Buffers are the caller's (device): keys [3 kSegTile] (any values),
// seg_start [3 kSegTile + 1], work [4], dc (zeroed DevCounters).
cudaError_t launch_wait_selftest(unsigned long long* keys, uint32_t* seg_start, uint32_t* work, DevCounters* dc,
                                 cudaStream_t st) {
  const int64_t n = 3 * kSegTile;
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(uint32_t) * 4, st);
  if (e != cudaSuccess) return e;
  const uint32_t one = 1u, items = (uint32_t)n;
  e = cudaMemcpyAsync(work + 3, &one, sizeof(one), cudaMemcpyHostToDevice, st);  // tile counter: skip tile 0
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(&dc->n_items, &items, sizeof(items), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  seg_heads_kernel<<<2, kSegThreads, 0, st>>>(keys, n, seg_start, work, 3, dc);
  return cudaGetLastError();
}

}  // namespace sbki
