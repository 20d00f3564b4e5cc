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

#include "exact_round.cuh"
#include "sbki_internal.cuh"

namespace sbki {
namespace {



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
  int lab;
  if (d.probs) {
    // soft labels: the most probable class (ties to the lowest; class 0 has
    // weight 0 for a hit); every entry finite in [0, 1], at least one above 0
    const float* pr = d.probs + li * (g.K1 - 1);
    lab = 0;
    float best = 0.0f;
    bool bad = false;
    for (int k = 1; k < g.K1; ++k) {
      const float v = pr[k - 1];
      bad = bad || !(v >= 0.0f && v <= 1.0f);
      if (v > best) {
        best = v;
        lab = k;
      }
    }
    if (bad || lab == 0) set_error(dc, SBKI_ERR_LABEL_RANGE);
  } else {
    lab = d.labels[li];
    if (lab < 1 || lab > g.K1 - 1) set_error(dc, SBKI_ERR_LABEL_RANGE);
  }
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

// Step a2 for every scan of the update: one warp per 8 consecutive points
// (which may belong to different scans; 8 rather than 32 so that four times
// the warps hide the latency of the per-beam loop); the warp writes each
// beam's samples together.  Hits go to items [0, hits), free samples after
// all hits.
__global__ void __launch_bounds__(256) emit_kernel(const float4* __restrict__ world,
                                                   const unsigned long long* __restrict__ cnt,
                                                   const ScanDesc* __restrict__ desc, int ns, Geom g, KeyFrame kf,
                                                   float4* __restrict__ items, unsigned long long* __restrict__ keys,
                                                   uint32_t* __restrict__ vals, uint32_t* __restrict__ hit_src,
                                                   DevCounters* dc) {
  __shared__ int64_t s_off[kMaxScans + 1];
  for (int t = threadIdx.x; t <= ns; t += blockDim.x) s_off[t] = desc[t].off;
  __syncthreads();
  if (dc->err) return;
  const int64_t n = s_off[ns];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned long long nvalid = cnt[n] >> 40;
  constexpr int kPerWarp = 8;  // points (beams) per warp task
  for (int64_t base = warp * kPerWarp; base < n; base += nwarps * kPerWarp) {
    const int64_t i = lane < kPerWarp ? base + lane : n;
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
        if (hit_src) hit_src[hpos] = (uint32_t)i;  // soft labels: the point whose probabilities the hit carries
        nfree = (uint32_t)((c1 & kFreeMask) - (c0 & kFreeMask));
        fpos = nvalid + (c0 & kFreeMask);
        ex = __fsub_rn(w.x, ox);
        ey = __fsub_rn(w.y, oy);
        ez = __fsub_rn(w.z, oz);
        rr = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez)));
      }
    }
    for (int src = 0; src < kPerWarp; ++src) {
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

// Centroids: per axis the exact mean of the members' FP32 coordinates,
// rounded once to FP32 (nearest, ties to even), with exact steps only:
// every nonzero |x| is m 2^e with an integer m < 2^24 and e = its exponent of
// the last mantissa bit; with E at or below the smallest such e in the cell,
//     sum |x| = T 2^E,   T = sum m 2^(e - E)
// and the mean is T 2^E / n, rounded with integer division.  The segment pass
// (seg_reduce_kernel) sums x 2^-E as signed 64-bit integers with E fixed by the
// sort tile; the cells it cannot decide go to slow_cell, where the members of
// a cell are taken to share a sign per axis (the cell index fixes it, except
// that x fp32(1/ds) of a negative subnormal x can round to -0 when ds > 1):
// T in 128 bits when the members' e span less than 127 - 24 - ceil(log2 n)
// binades, else (and for a mean below the FP32 normal range, or mixed signs) a
// one-thread signed 512-bit sum, exact for every FP32 input.

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
  bool neg, pos;   // a member below / above zero
  __device__ void init() {
    emin = 1 << 20;
    emax = -(1 << 20);
    neg = pos = false;
  }
  __device__ void see(float v) {
    unsigned m;
    int e;
    if (decompose(v, m, e)) {
      emin = min(emin, e);
      emax = max(emax, e);
      neg |= v < 0.0f;
      pos |= v > 0.0f;
    }
  }
  __device__ bool empty() const { return emax < emin; }
  __device__ bool fits(uint32_t n) const {  // one sign, and T stays below 2^127
    int lg = 0;
    while (lg < 32 && (1ull << lg) < n) ++lg;
    return empty() || (!(neg && pos) && emax - emin + 24 + lg <= 126);
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
// Positive and negative members are summed apart, in 16 32-bit limbs in units
// of 2^-149 each (512 bits), and the smaller sum is subtracted from the larger.
__device__ float wide_mean(const float4* __restrict__ items, const uint32_t* __restrict__ perm, uint32_t a,
                           uint32_t b, int ax) {
  uint32_t wp[16], wn[16];
  for (int i = 0; i < 16; ++i) wp[i] = wn[i] = 0u;
  for (uint32_t i = a; i < b; ++i) {
    const float v = axis_of(item_at(items, perm, i), ax);
    unsigned m;
    int e;
    if (!decompose(v, m, e)) continue;
    uint32_t* w = v < 0.0f ? wn : wp;
    const int sh = e + 149, li = sh >> 5, bi = sh & 31;
    unsigned long long add = (unsigned long long)m << bi;  // < 2^55
    for (int j = li; j < 16 && add; ++j) {
      const unsigned long long t = (unsigned long long)w[j] + (add & 0xffffffffull);
      w[j] = (uint32_t)t;
      add = (add >> 32) + (t >> 32);
    }
  }
  bool neg = false;  // the negative members outweigh the positive ones
  for (int j = 15; j >= 0; --j)
    if (wn[j] != wp[j]) {
      neg = wn[j] > wp[j];
      break;
    }
  uint32_t w[16];
  {
    const uint32_t* hi = neg ? wn : wp;
    const uint32_t* lo = neg ? wp : wn;
    unsigned long long borrow = 0ull;
    for (int j = 0; j < 16; ++j) {
      const unsigned long long d = (unsigned long long)hi[j] - lo[j] - borrow;
      w[j] = (uint32_t)d;
      borrow = (d >> 63) & 1ull;
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
  s.pos = __any_sync(0xffffffffu, s.pos);
}

// Exact mean of a cell the segment pass could not decide (cell s, members
// [seg_start[s], seg_start[s + 1]) of the sorted items), by a whole warp.  An
// axis whose first member has |x0| >= 2.5 ds is summed in one pass in 64 bits
// (FastAxis); any other axis takes its exponent range first, then the 128-bit
// sum, else wide_mean.
__device__ void slow_cell(uint32_t s, const unsigned long long* __restrict__ keys, const float4* __restrict__ items,
                          const uint32_t* __restrict__ seg_start, const Geom& g, float4* __restrict__ train,
                          const ScanDesc* __restrict__ desc, const KeyFrame& kf) {
  const int lane = threadIdx.x & 31;
  const uint32_t* perm = nullptr;
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
  const bool two_pass = !fa[0].on || !fa[1].on || !fa[2].on;  // warp-uniform
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
  if (two_pass) {
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

// --- segments and centroids in one pass ---------------------------------------
// The sorted items are cut into tiles of kSegTile.  seg_count_kernel counts
// each tile's segment heads (items whose key differs from the predecessor's).
// seg_reduce_kernel, a persistent grid, then takes the tiles one by one:
// stages the tile's keys and items through shared memory (coalesced reads),
// marks its heads, sums the head counts of the tiles before it (so it waits on
// no other CTA) and writes seg_start.  Each thread then sums its members: per axis a coordinate x adds
// the integer x 2^-E (an exact FP32 product, converted exactly), with E fixed
// by the member's sort tile of 8^3 cells (kSegShift + 23 below the exponent of
// (8 |t| + 10) ds, t the tile index on that axis, an upper bound of the tile's
// |x|), so a cell's sum is a plain signed 64-bit integer in any order.  A
// nonzero member with |x| 2^-E below 2^23 (it would have a fraction: within
// about 2^-21 ds of a coordinate plane) or a mean below the FP32 normal range
// leaves the cell to slow_cell.
// A thread stores the sums of every cell whose head it holds in shared memory;
// the run before its first head (the end of a cell begun in an earlier thread)
// is added there with shared-memory atomics; then the CTA rounds every cell.
// A cell that continues into the next tile leaves partial sums (the cell's
// part in its head's tile, the run that opens each following tile), which
// finish_cells_kernel joins and rounds.
constexpr int kSegThreads = 256;
constexpr int kSegPer = 8;
constexpr int kSegTile = kSegThreads * kSegPer;
constexpr int kSegWarps = kSegThreads / 32;
constexpr int kSegShift = 24;      // binades between a tile's |x| bound and its members' smallest last bit
constexpr uint32_t kSegMaxN = 1u << (63 - 24 - kSegShift);  // |T| < n 2^(24 + kSegShift) < 2^63 below this
static_assert(kSegTile == kSegTileItems, "segment tile size");

struct SegState {           // sums of a run of members of one cell
  unsigned long long T[3];  // per axis: sum of x 2^-E, two's complement
  uint32_t n;               // members
  uint32_t flags;           // bit 1 kSegBad: see above; bits 2 + 9a: E + 256 of axis a (the same for every
                            // member of a cell, so runs join by OR)
};
constexpr uint32_t kSegBad = 2u;

// Dynamic shared memory: the cells' sums and label words; the first part
// doubles as the load stage (items, then keys, one pad entry per kSegPer so
// that each thread's consecutive entries fall in distinct banks).
__host__ __device__ constexpr int seg_pad(int i) { return i + i / kSegPer; }
constexpr size_t kSegCellBytes = (size_t)kSegTile * sizeof(SegState);
constexpr size_t kSegStageItems = 0;
constexpr size_t kSegStageKeys = (size_t)seg_pad(kSegTile) * 16;
constexpr size_t kSegSmemBytes = kSegCellBytes + (size_t)kSegTile * sizeof(uint32_t);
static_assert(kSegStageKeys + (size_t)seg_pad(kSegTile + 2) * 8 <= kSegCellBytes, "load stage fits the cell stage");

// The tile's cells in shared memory, one array per field (consecutive cells in
// consecutive words, so a warp reading the cells q, q + 1, ... meets no bank conflict).
struct SegCells {
  unsigned long long* T[3];
  uint32_t* n;
  uint32_t* flags;
  __device__ __forceinline__ explicit SegCells(unsigned char* base) {
    T[0] = reinterpret_cast<unsigned long long*>(base);
    T[1] = T[0] + kSegTile;
    T[2] = T[1] + kSegTile;
    n = reinterpret_cast<uint32_t*>(T[2] + kSegTile);
    flags = n + kSegTile;
  }
  __device__ __forceinline__ void store(uint32_t j, const SegState& s) const {
    T[0][j] = s.T[0];
    T[1][j] = s.T[1];
    T[2][j] = s.T[2];
    n[j] = s.n;
    flags[j] = s.flags;
  }
  __device__ __forceinline__ SegState load(uint32_t j) const {
    SegState s;
    s.T[0] = T[0][j];
    s.T[1] = T[1][j];
    s.T[2] = T[2][j];
    s.n = n[j];
    s.flags = flags[j];
    return s;
  }
  __device__ __forceinline__ void add(uint32_t j, const SegState& s) const {  // shared-memory atomics
    atomicAdd(&T[0][j], s.T[0]);
    atomicAdd(&T[1][j], s.T[1]);
    atomicAdd(&T[2][j], s.T[2]);
    atomicAdd(&n[j], s.n);
    atomicOr(&flags[j], s.flags);
  }
};

struct SegCarry {   // partial sums of a cell that crosses a tile boundary
  SegState st;
  uint32_t s;       // part in the head's tile: the cell's index
  uint32_t closed;  // run that opens a tile: 1 when the cell ends inside the tile
  uint32_t pad[2];
};
static_assert(sizeof(SegCarry) == kSegCarryBytes, "segment carry layout");

// The sort tile a key names: E per axis packed as in SegState::flags, the
// scales 2^-E, and kSegBad when a scale is outside the FP32 normal range.
struct TileUnit {
  uint32_t meta, bad;
  float scale[3];
};
__device__ __forceinline__ TileUnit tile_unit(unsigned long long key, const Geom& g, const KeyFrame& kf,
                                              const ScanDesc* __restrict__ desc) {
  int o0 = kf.org[0], o1 = kf.org[1], o2 = kf.org[2];
  if (kf.scan_bits) {
    const ScanDesc& d = desc[(int)(key >> kf.total_bits)];
    o0 = d.org[0];
    o1 = d.org[1];
    o2 = d.org[2];
  }
  const unsigned long long tile = key >> (g.label_bits + kLocalBits);
  const int t[3] = {(int)((tile >> (kf.bits[1] + kf.bits[2])) & ((1ull << kf.bits[0]) - 1)) + o0,
                    (int)((tile >> kf.bits[2]) & ((1ull << kf.bits[1]) - 1)) + o1,
                    (int)(tile & ((1ull << kf.bits[2]) - 1)) + o2};
  TileUnit u;
  u.meta = 0u;
  u.bad = 0u;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int mag = t[a] < 0 ? -t[a] : t[a];
    const float U = __fmul_rn((float)(kTileEdge * mag + kTileEdge + 2), g.ds);
    const int E = (int)(__float_as_uint(U) >> 23) - 150 - kSegShift;  // |x| < U < 2^(E + 48)
    u.meta |= (uint32_t)(E + 256) << (2 + 9 * a);
    const bool ok = E >= -126 && E <= 126;
    u.scale[a] = ok ? __uint_as_float((uint32_t)(127 - E) << 23) : 0.f;
    if (!ok) u.bad = kSegBad;
  }
  return u;
}
__device__ __forceinline__ int meta_E(uint32_t flags, int a) { return (int)((flags >> (2 + 9 * a)) & 511u) - 256; }

__device__ __forceinline__ void seg_clear(SegState& s) {
  s.T[0] = s.T[1] = s.T[2] = 0ull;
  s.n = 0u;
  s.flags = 0u;
}

__device__ __forceinline__ void seg_add(SegState& s, const TileUnit& u, float x, float y, float z) {
  s.n += 1u;
  const float v[3] = {x, y, z};
  bool bad = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float q = __fmul_rn(v[a], u.scale[a]);  // x 2^-E, exact when |q| >= 2^23
    const float aq = fabsf(q);
    bad = bad || (aq < 8388608.0f && aq != 0.0f) || aq >= 281474976710656.0f;
    s.T[a] += (unsigned long long)__float2ll_rz(q);
  }
  s.flags |= u.meta | u.bad | (bad ? kSegBad : 0u);
}

// a := a and b joined (two runs of one cell)
__device__ __forceinline__ void seg_merge(SegState& a, const SegState& b) {
  a.T[0] += b.T[0];
  a.T[1] += b.T[1];
  a.T[2] += b.T[2];
  a.n += b.n;
  a.flags |= b.flags;
}

// The label word of a training point (label + 32 map) from its cell's key
__device__ __forceinline__ uint32_t label_word(unsigned long long key, const Geom& g, const KeyFrame& kf,
                                               const ScanDesc* __restrict__ desc) {
  return (uint32_t)(key & ((1ull << g.label_bits) - 1)) + 32u * (uint32_t)map_of_segment(key, kf, desc);
}

// Training point s from the complete sums of its cell (lw: its label word);
// false, with nothing written, when this form cannot give the exact mean.
__device__ __forceinline__ bool try_round_cell(const SegState& st, uint32_t s, uint32_t lw,
                                               float4* __restrict__ train) {
  bool ok = !(st.flags & kSegBad) && st.n < kSegMaxN;
  float out[3] = {0.f, 0.f, 0.f};
  if (ok) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const long long T = (long long)st.T[a];
      if (T) {
        float f = 0.f;
        ok = round_mean64(T < 0 ? (unsigned long long)(-T) : (unsigned long long)T, st.n, meta_E(st.flags, a), f) &&
             ok;
        out[a] = T < 0 ? -f : f;
      }
    }
  }
  if (ok) train[s] = make_float4(out[0], out[1], out[2], (float)lw);
  return ok;
}

__device__ __forceinline__ void st_carry(SegCarry* dst, const SegState& st, uint32_t s, uint32_t closed) {
  SegCarry c;
  c.st = st;
  c.s = s;
  c.closed = closed;
  c.pad[0] = c.pad[1] = 0u;
  *dst = c;
}

// Heads per tile of the sorted items: counts[t] for every tile t below
// ceil(n / kSegTile), n = min(cap, dc->n_items).  Grid-stride over tiles.
__global__ void __launch_bounds__(kSegThreads) seg_count_kernel(const unsigned long long* __restrict__ keys,
                                                              int64_t cap, uint32_t* __restrict__ counts,
                                                              const DevCounters* dc) {
  __shared__ uint32_t s_w[kSegWarps];
  if (dc->err) return;
  const int64_t n = min(cap, (int64_t)dc->n_items);
  const int64_t nt = (n + kSegTile - 1) / kSegTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    uint32_t c = 0u;
#pragma unroll
    for (int r = 0; r < kSegPer; ++r) {
      const int64_t i = t * kSegTile + r * kSegThreads + threadIdx.x;
      if (i < n) c += (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) s_w[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t total = 0u;
#pragma unroll
      for (int w = 0; w < kSegWarps; ++w) total += s_w[w];
      counts[t] = total;
    }
    __syncthreads();
  }
}

// work: [ntiles_cap] head counts (seg_count_kernel), tile counter, an unused
// word, [ntiles_cap] closing flags (these two zero on entry).  carry: [2 ntiles_cap].
// Dynamic shared memory: kSegSmemBytes.
__global__ void __launch_bounds__(kSegThreads, 3) seg_reduce_kernel(
    const unsigned long long* __restrict__ keys, const float4* __restrict__ items, int64_t cap,
    uint32_t* __restrict__ seg_start, uint32_t* __restrict__ work, int64_t ntiles_cap, SegCarry* __restrict__ carry,
    Geom g, float4* __restrict__ train, const ScanDesc* __restrict__ desc, KeyFrame kf, uint32_t* __restrict__ slow,
    DevCounters* dc) {
  extern __shared__ __align__(16) unsigned char seg_smem[];
  const SegCells s_cell(seg_smem);                                             // by tile-local cell index
  uint32_t* s_head = reinterpret_cast<uint32_t*>(seg_smem + kSegCellBytes);  // the cell's label word
  float4* s_items = reinterpret_cast<float4*>(seg_smem + kSegStageItems);     // load stage (aliases s_cell)
  unsigned long long* s_keys = reinterpret_cast<unsigned long long*>(seg_smem + kSegStageKeys);
  __shared__ SegState s_open;  // the run that opens the tile, of a cell whose head lies in an earlier tile
  __shared__ uint32_t s_wsum[kSegWarps], s_wbefore[kSegWarps];
  __shared__ uint32_t s_tile;
  __shared__ int s_cross;      // the tile's last cell goes on in the next tile
  if (dc->err) return;
  const int64_t n = min(cap, (int64_t)dc->n_items);
  const int64_t nt = (n + kSegTile - 1) / kSegTile;
  const uint32_t* counts = work;
  uint32_t* claim = work + ntiles_cap;
  uint32_t* closing = claim + 2;
  SegCarry* opening_run = carry;
  SegCarry* closing_run = carry + ntiles_cap;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_tile = atomicAdd(claim, 1u);
      s_cross = 0;
      seg_clear(s_open);
    }
    __syncthreads();
    const int64_t t = s_tile;
    if (t >= nt) break;
    const int64_t base = t * kSegTile;
    const int64_t first = base + (int64_t)threadIdx.x * kSegPer;
    const int64_t tile_last = min(n, base + kSegTile) - 1;
    // stage the tile (s_keys[seg_pad(1 + r)] = key of item base + r; entries 0 and
    // kSegTile + 1: the items just before and after the tile), then take the thread's members
#pragma unroll
    for (int r = 0; r < kSegPer; ++r) {
      const int li = r * kSegThreads + (int)threadIdx.x;
      if (base + li < n) {
        s_keys[seg_pad(1 + li)] = keys[base + li];
        s_items[seg_pad(li)] = items[base + li];
      }
    }
    if (threadIdx.x == 0 && base > 0) s_keys[seg_pad(0)] = keys[base - 1];
    if (threadIdx.x == 1 && base + kSegTile < n) s_keys[seg_pad(kSegTile + 1)] = keys[base + kSegTile];
    __syncthreads();
    unsigned long long kk[kSegPer];
    float px[kSegPer], py[kSegPer], pz[kSegPer];
    uint32_t heads = 0u;
    const int l0 = (int)threadIdx.x * kSegPer;
    unsigned long long prev = first > 0 && first <= n ? s_keys[seg_pad(l0)] : 0ull;
#pragma unroll
    for (int k = 0; k < kSegPer; ++k) {
      const int64_t i = first + k;
      kk[k] = 0ull;
      px[k] = py[k] = pz[k] = 0.f;
      if (i < n) {
        kk[k] = s_keys[seg_pad(l0 + k + 1)];
        const float4 p = s_items[seg_pad(l0 + k)];
        px[k] = p.x;
        py[k] = p.y;
        pz[k] = p.z;
        if (i == 0 || kk[k] != prev) heads |= 1u << k;
        prev = kk[k];
      }
    }
    uint32_t ends = heads >> 1;
    if (first + kSegPer < n && s_keys[seg_pad(l0 + kSegPer + 1)] != prev) ends |= 1u << (kSegPer - 1);
    if (first <= n - 1 && n - 1 < first + kSegPer) ends |= 1u << (int)(n - 1 - first);
    const bool has_items = first < n;
    const int last_k = has_items ? (int)(min(n - 1, first + kSegPer - 1) - first) : 0;
    if (has_items && first + last_k == tile_last) s_cross = (ends & (1u << last_k)) ? 0 : 1;
    // heads before this thread in the tile, in the tile, and before the tile
    // (the barrier also ends the stage's reads)
    const uint32_t c = __popc(heads);
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    uint32_t before = 0u;
    for (int64_t q = threadIdx.x; q < t; q += kSegThreads) before += counts[q];
    before = __reduce_add_sync(0xffffffffu, before);
    if (lane == 31) s_wsum[warp] = inc;
    if (lane == 0) s_wbefore[warp] = before;
    __syncthreads();
    uint32_t hthread = inc - c, total = 0u, excl = 0u;
#pragma unroll
    for (int w = 0; w < kSegWarps; ++w) {
      const uint32_t v = s_wsum[w];
      hthread += w < warp ? v : 0u;
      total += v;
      excl += s_wbefore[w];
    }
    {
      uint32_t j = hthread;
#pragma unroll
      for (int k = 0; k < kSegPer; ++k)
        if (heads & (1u << k)) {
          seg_start[excl + j] = (uint32_t)(first + k);
          s_head[j++] = label_word(kk[k], g, kf, desc);
        }
      if (first <= n - 1 && n - 1 < first + kSegPer) {  // this thread holds the last item
        seg_start[excl + total] = (uint32_t)n;
        dc->n_train = excl + total;
      }
    }
    // sum the members: the run before the first head (P), then one run per head,
    // each stored at its cell's tile-local index
    SegState R, P;
    seg_clear(R);
    seg_clear(P);
    bool hashead = false;
    uint32_t j = hthread - 1u;  // tile-local index of the running cell once a head is seen
    const int tshift = g.label_bits + kLocalBits;
    unsigned long long tprev = ~0ull;  // sort tile of the previous member, and its unit
    TileUnit unit;
    unit.meta = unit.bad = 0u;
    unit.scale[0] = unit.scale[1] = unit.scale[2] = 0.f;
#pragma unroll
    for (int k = 0; k < kSegPer; ++k) {
      if (first + k < n) {
        if ((kk[k] >> tshift) != tprev) {
          tprev = kk[k] >> tshift;
          unit = tile_unit(kk[k], g, kf, desc);
        }
        if (heads & (1u << k)) {
          if (!hashead) P = R;
          hashead = true;
          seg_clear(R);
          ++j;
        }
        seg_add(R, unit, px[k], py[k], pz[k]);
        if (hashead && ((ends & (1u << k)) || k == last_k)) s_cell.store(j, R);
      }
    }
    if (!hashead) P = R;
    __syncthreads();
    if (has_items && !(heads & 1u)) {  // the end of a cell begun before this thread
      if (hthread > 0u) {
        s_cell.add(hthread - 1u, P);
      } else {
        atomicAdd(&s_open.T[0], P.T[0]);
        atomicAdd(&s_open.T[1], P.T[1]);
        atomicAdd(&s_open.T[2], P.T[2]);
        atomicAdd(&s_open.n, P.n);
        atomicOr(&s_open.flags, P.flags);
      }
    }
    __syncthreads();
    // round every cell whose head lies in the tile, but a last one that goes on
    const bool cross_out = s_cross && total > 0u;
    const uint32_t nround = total - (cross_out ? 1u : 0u);
    for (uint32_t q = threadIdx.x; q < nround; q += kSegThreads)
      if (!try_round_cell(s_cell.load(q), excl + q, s_head[q], train))
        slow[atomicAdd(&dc->n_slow, 1u)] = excl + q;
    if (threadIdx.x == 0) {
      if (cross_out) {
        st_carry(closing_run + t, s_cell.load(total - 1u), excl + total - 1u, 0u);
        closing[t] = 1u;
      }
      if (s_open.n) st_carry(opening_run + t, s_open, 0u, (total > 0u || !s_cross) ? 1u : 0u);
    }
  }
}

// After seg_reduce_kernel: the cells it left to the slow form (`slow`, one warp
// each), and the cells that cross a tile boundary (one warp per tile whose
// closing flag is set: lane 0 joins the partial sums of the following tiles up
// to the one where the cell ends, in 128 bits (each part holds at most one
// tile's members, but a cell may span many tiles), and rounds them, or the warp
// takes the slow form).  work and carry as seg_reduce_kernel left them.
__device__ __forceinline__ void add_i128(U128& t, unsigned long long v) {  // t += v read as signed 64-bit
  u128_add(t, v, (long long)v < 0 ? ~0ull : 0ull);
}
__global__ void __launch_bounds__(256) finish_cells_kernel(const unsigned long long* __restrict__ keys,
                                                           const float4* __restrict__ items, int64_t cap,
                                                           const uint32_t* __restrict__ seg_start,
                                                           const uint32_t* __restrict__ work, int64_t ntiles_cap,
                                                           const SegCarry* __restrict__ carry, Geom g,
                                                           float4* __restrict__ train,
                                                           const ScanDesc* __restrict__ desc, KeyFrame kf,
                                                           const uint32_t* __restrict__ slow, DevCounters* dc) {
  if (dc->err) return;
  const int64_t n = min(cap, (int64_t)dc->n_items);
  const int64_t nt = (n + kSegTile - 1) / kSegTile;
  const uint32_t ns = dc->n_slow;
  const uint32_t* closing = work + ntiles_cap + 2;
  const SegCarry* opening_run = carry;
  const SegCarry* closing_run = carry + ntiles_cap;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = warp; j < (int64_t)ns + nt; j += nwarps) {
    if (j < (int64_t)ns) {
      slow_cell(slow[j], keys, items, seg_start, g, train, desc, kf);
      continue;
    }
    const int64_t u = j - ns;
    if (!closing[u]) continue;  // warp-uniform
    int done = 0;
    uint32_t s = 0u;
    if (lane == 0) {
      const SegCarry h = closing_run[u];
      U128 T[3];
      uint32_t cn = h.st.n, flags = h.st.flags;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T[c].lo = T[c].hi = 0ull;
        add_i128(T[c], h.st.T[c]);
      }
      for (int64_t v = u + 1; v < nt; ++v) {
        const SegCarry o = opening_run[v];
#pragma unroll
        for (int c = 0; c < 3; ++c) add_i128(T[c], o.st.T[c]);
        cn += o.st.n;
        flags |= o.st.flags;
        if (o.closed) break;
      }
      s = h.s;
      bool ok = !(flags & kSegBad);
      float out[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (!ok || (T[c].lo | T[c].hi) == 0ull) continue;
        const bool neg = (long long)T[c].hi < 0;
        U128 mag = T[c];
        if (neg) {  // two's complement negation
          mag.lo = ~T[c].lo + 1ull;
          mag.hi = ~T[c].hi + (mag.lo == 0ull ? 1ull : 0ull);
        }
        float f = 0.f;
        ok = round_mean(mag, cn, meta_E(flags, c), f);
        out[c] = neg ? -f : f;
      }
      if (ok) {
        const unsigned long long key = keys[(u + 1) * kSegTile - 1];
        const int label = (int)(key & ((1ull << g.label_bits) - 1));
        train[s] = make_float4(out[0], out[1], out[2], (float)(label + 32 * map_of_segment(key, kf, desc)));
      }
      done = ok ? 1 : 0;
    }
    done = __shfl_sync(0xffffffffu, done, 0);
    s = __shfl_sync(0xffffffffu, s, 0);
    if (!done) slow_cell(s, keys, items, seg_start, g, train, desc, kf);
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
  m.launches += 1 + 1;  // transform, prefix sum (which also checks the item count against the capacity)
  cudaError_t e = exclusive_scan_u64_onepass(m.s.cnt, total_n, m.s.scan_tmp, m.stream, &m.dc->n_points, m.sm_count,
                                             m.dc, m.s.s_cap);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_emit(MapState& m, int ns, int64_t total_n, const KeyFrame& kf, uint32_t* hit_src) {
  const int64_t warps = (total_n + 7) / 8;
  unsigned blocks = (unsigned)std::min<int64_t>((warps + 7) / 8, (int64_t)m.sm_count * m.tune.ingest_ctas_per_sm);
  if (blocks == 0) blocks = 1;
  emit_kernel<<<blocks, 256, 0, m.stream>>>(m.s.world, m.s.cnt, m.s.desc, ns, m.g, kf, m.s.items, m.s.keys, m.s.vals,
                                            hit_src, m.dc);
  m.launches += 1;
  return cudaGetLastError();
}

// Sorts the items and reduces each (scan, cell, label) segment to its centroid.
// nitems: host-known bound on the item count (the count itself is read on the device).
cudaError_t launch_downsample_n(MapState& m, const KeyFrame& kf, int64_t nitems) {
  Scratch& s = m.s;
  const int bits = kf.total_bits + kf.scan_bits;
  m.launches += 1 + (bits + 7) / 8 + 3;  // sort, head counts, segment pass, crossing and slow cells
  // the last pass also moves the items into sorted order (s.sitems), so the segment pass reads them in a stream
  cudaError_t e = radix_sort_pairs(s.keys, s.vals, s.keys2, s.vals2, &m.dc->n_items, nitems, bits, s.hist,
                                   m.sm_count, m.dc, m.stream, s.items, s.sitems);
  if (e != cudaSuccess) return e;
  const int64_t stiles = (nitems + kSegTile - 1) / kSegTile;
  e = cudaMemsetAsync(s.flags + stiles, 0, sizeof(uint32_t) * (stiles + 2), m.stream);
  if (e != cudaSuccess) return e;
  seg_count_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(stiles, 65535)), kSegThreads, 0, m.stream>>>(
      s.keys, nitems, s.flags, m.dc);
  e = cudaFuncSetAttribute(seg_reduce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSegSmemBytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, seg_reduce_kernel, kSegThreads, kSegSmemBytes);
  if (e != cudaSuccess) return e;
  const unsigned sblocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(stiles, (int64_t)m.sm_count * std::max(1, per_sm)));
  seg_reduce_kernel<<<sblocks, kSegThreads, kSegSmemBytes, m.stream>>>(s.keys, s.sitems, nitems, s.seg_start, s.flags,
                                                                       stiles, static_cast<SegCarry*>(s.carry), m.g,
                                                                       s.train, s.desc, kf, s.slow, m.dc);
  const unsigned fblocks = (unsigned)std::min<int64_t>(4096, std::max<int64_t>(2 * m.sm_count, (stiles + 7) / 8));
  finish_cells_kernel<<<fblocks, 256, 0, m.stream>>>(s.keys, s.sitems, nitems, s.seg_start, s.flags,
                                                                       stiles, static_cast<const SegCarry*>(s.carry),
                                                                       m.g, s.train, s.desc, kf, s.slow, m.dc);
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

}  // namespace sbki
