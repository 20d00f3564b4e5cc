// Soft labels (reading K15) and per-class length scales (reading K16).
//
// Weights: after the downsampling (groups by cell and most probable class),
// every group of hits (class 1..K) gets, per class 0..K, the exact mean of its
// members' weights rounded once to FP32 (a hit's weights are 0 for class 0 and
// its probability vector for classes 1..K).  Groups of free samples (class 0)
// keep the implicit weight vector one-hot(0) and no row.
//
// Weighted accumulation (Eq. (alpha_kernel) with the one-hot y_i replaced by a
// weight vector, and class k's kernel sigma0 s_k f(d/l_k) with support l_k),
// for what the fast point-major form does not take (class supports beyond 7
// offsets per axis or below half the voxel diagonal, soft labels without the
// fast form's tables):
// one warp per training point sweeps the cube of voxel offsets within
// +-R of the point's voxel, R the largest of its weighted classes' R_k
// (offsets j with |j| - 1/2 >= l_k / res hold no voxel centre within l_k of a
// point in the voxel), decides membership per class
// exactly as the map update does (compensated FP32 offsets, FP64 inside the
// relative band around l_k^2) and adds sigma0 s_k f(d/l_k) w^k into every
// class k with w^k != 0 whose support holds the voxel; a (voxel, point) pair
// counts once when any class's support holds it.
#include <algorithm>
#include <climits>

#include "exact_round.cuh"
#include "kernel_value.cuh"
#include "point_common.cuh"

namespace sbki {
namespace {

// |v| = m 2^e with m < 2^24 an integer; false for zero
__device__ __forceinline__ bool split_float(float v, unsigned& m, int& e) {
  const unsigned b = __float_as_uint(v) & 0x7fffffffu;
  if (b == 0u) return false;
  const unsigned E = b >> 23;
  m = (b & 0x7fffffu) | (E ? 0x800000u : 0u);
  e = E ? (int)E - 150 : -149;
  return true;
}

// Exact mean of n values in [0, 1] rounded once to FP32, 64-bit form: with
// every nonzero value m 2^e (m < 2^24) and E the smallest e, the sum is the
// integer T = sum m 2^(e - E) times 2^E, which fits 64 bits when the values
// span few enough binades; round_mean64 rounds T 2^E / n.  False (nothing
// decided) when they span more, for n >= 2^16, or for a mean below the FP32
// normal range.
template <typename Get>
__device__ bool unit_mean_int(Get get, uint32_t n, float& out) {
  if (n >= (1u << 16)) return false;
  int emin = INT_MAX, emax = INT_MIN;
  for (uint32_t i = 0; i < n; ++i) {
    unsigned m;
    int e;
    if (split_float(get(i), m, e)) {
      emin = min(emin, e);
      emax = max(emax, e);
    }
  }
  if (emin == INT_MAX) {  // all zero
    out = 0.0f;
    return true;
  }
  if (emax - emin + 24 + (32 - __clz((int)n)) > 63) return false;
  unsigned long long T = 0ull;
  for (uint32_t i = 0; i < n; ++i) {
    unsigned m;
    int e;
    if (split_float(get(i), m, e)) T += (unsigned long long)m << (e - emin);
  }
  return round_mean64(T, n, emin, out);
}

// Exact mean of n values in [0, 1] rounded once to FP32 (nearest, ties to
// even): the 64-bit form when it can decide, else the sum is held in units of
// 2^-149 in 6 32-bit limbs (a value below 2^1 needs 150 bits, n < 2^32 adds at
// most 32), divided by n limb by limb from the top with 3 fractional limbs,
// and rounded to 24 significant bits (fewer for a result below the FP32
// normal range).
template <typename Get>
__device__ float unit_mean(Get get, uint32_t n) {
  float f;
  if (unit_mean_int(get, n, f)) return f;
  uint32_t w[6] = {0u, 0u, 0u, 0u, 0u, 0u};
  for (uint32_t i = 0; i < n; ++i) {
    unsigned m;
    int e;
    if (!split_float(get(i), m, e)) continue;
    const int sh = e + 149, li = sh >> 5, bi = sh & 31;
    unsigned long long add = (unsigned long long)m << bi;
    for (int j = li; j < 6 && add; ++j) {
      const unsigned long long t = (unsigned long long)w[j] + (add & 0xffffffffull);
      w[j] = (uint32_t)t;
      add = (add >> 32) + (t >> 32);
    }
  }
  uint32_t q[9];  // (sum 2^96) / n
  unsigned long long r = 0ull;
  for (int j = 8; j >= 0; --j) {
    const unsigned long long cur = (r << 32) | (j >= 3 ? w[j - 3] : 0u);
    q[j] = (uint32_t)(cur / n);
    r = cur - (unsigned long long)q[j] * n;
  }
  int qb = 0;
  for (int j = 8; j >= 0 && !qb; --j)
    if (q[j]) qb = 32 * j + 32 - __clz((int)q[j]);
  if (qb == 0) return 0.0f;
  // value = q 2^(-149 - 96)
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
  return ldexpf((float)mant, drop - 245);
}

// Weight rows of the groups that hold hits: a warp takes 32 consecutive
// training points (groups); a group's class is its members' most probable
// class, which is 1..K for a hit and 0 for a free sample, so a group of class
// k >= 1 holds hits only (class-0 weight 0) and a group of class 0 free
// samples only (no row).  Each group with hits is then taken by the whole
// warp, lane k computing the exact mean of class k (one member: its vector).
__global__ void soft_weights_kernel(const uint32_t* __restrict__ seg_start, const uint32_t* __restrict__ svals,
                                    const uint32_t* __restrict__ hit_src, const float4* __restrict__ train,
                                    const ScanDesc* __restrict__ desc, int32_t* __restrict__ softidx,
                                    float* __restrict__ wsoft, int K1, DevCounters* dc) {
  if (dc->err != 0) return;
  const uint32_t P = dc->n_train;
  const float* probs = desc[0].probs;
  const int K = K1 - 1, lane = threadIdx.x & 31;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < P; base += nw * 32) {
    const uint32_t t = base + lane;
    const bool hits = t < P && (label_of(train[t].w) & ((1 << kLabelBits) - 1)) != 0;
    unsigned todo = __ballot_sync(0xffffffffu, hits);
    uint32_t row0 = 0;
    if (lane == 0 && todo) row0 = atomicAdd(&dc->n_soft, (uint32_t)__popc(todo));
    row0 = __shfl_sync(0xffffffffu, row0, 0);
    if (t < P) softidx[t] = hits ? (int32_t)(row0 + __popc(todo & ((1u << lane) - 1u))) : -1;
    for (uint32_t r = row0; todo; todo &= todo - 1u, ++r) {  // warp-uniform
      const uint32_t tg = base + (uint32_t)(__ffs((int)todo) - 1);
      const uint32_t a = seg_start[tg], n = seg_start[tg + 1] - a;
      if (lane < K1) {
        float w = 0.0f;
        if (lane > 0) {
          if (n == 1)
            w = probs[(size_t)hit_src[svals[a]] * K + (lane - 1)];
          else
            w = unit_mean([&](uint32_t i) -> float { return probs[(size_t)hit_src[svals[a + i]] * K + (lane - 1)]; },
                          n);
        }
        wsoft[(size_t)r * K1 + lane] = w;
      }
    }
  }
}

// Writes a soft training set out: xyz [P,3] and weights [P,K+1] (one-hot for groups without a row).
__global__ void soft_export_kernel(const float4* __restrict__ train, const int32_t* __restrict__ softidx,
                                   const float* __restrict__ wsoft, int K1, int64_t cap, float* __restrict__ xyz,
                                   float* __restrict__ w, const DevCounters* dc) {
  const uint32_t P = dc->n_train;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < P && t < cap; t += gridDim.x * blockDim.x) {
    const float4 p = train[t];
    xyz[3 * (size_t)t] = p.x;
    xyz[3 * (size_t)t + 1] = p.y;
    xyz[3 * (size_t)t + 2] = p.z;
    const int r = softidx[t];
    const int label = label_of(p.w) & ((1 << kLabelBits) - 1);
    for (int k = 0; k < K1; ++k) w[(size_t)t * K1 + k] = r >= 0 ? wsoft[(size_t)r * K1 + k] : (k == label ? 1.0f : 0.0f);
  }
}

constexpr int kWThreads = 128;
constexpr int kWWarps = kWThreads / 32;
constexpr int kWAxis = 16;  // offsets per axis: 2R + 1 <= 15 (and a spare)

struct WArgs {
  Geom g;
  const float4* train;
  const int32_t* softidx;  // null: hard labels (weight one for the point's class)
  const float* wsoft;
  const unsigned long long* hkeys;
  const int32_t* hvals;
  int64_t hash_cap;
  float* alpha;
  int32_t* pairs;
  int32_t sink;
  int Rk[kMaxClasses];     // sweep half-width of class k's support, in voxels
  uint32_t skip;           // hard labels of these classes are the fast form's (per-class supports)
  DevCounters* dc;
};

struct WTables {
  float e2[3][kWAxis];   // squared compensated offset of axis offset j - R
  int part[3][kWAxis];   // block digit (base 3 per axis) | in-block index << 8, per axis
  float* blk[27];        // alpha + pool * (K+1) B^3
  int32_t* cnt[27];
  float w[kMaxClasses];  // the point's weights
};

template <bool kTrack>
__global__ void __launch_bounds__(kWThreads) accumulate_weighted_kernel(WArgs a) {
  __shared__ WTables s_t[kWWarps];
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  WTables& t = s_t[wid];
  if (a.dc->err != 0) return;
  const uint32_t P = a.dc->n_train;
  const int m = g.B - 1;
  uint32_t npairs = 0;
  for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < P; i += (gridDim.x * blockDim.x) >> 5) {
    const float4 p = a.train[i];
    const int lw = label_of(p.w);
    const int label = lw & ((1 << kLabelBits) - 1), map = lw >> kLabelBits;
    const int row = a.softidx ? a.softidx[i] : -1;
    if (row < 0 && ((a.skip >> label) & 1u)) continue;  // warp-uniform
    // weights and the classes that carry one
    float wk = 0.0f;
    if (lane < g.K1) wk = row >= 0 ? a.wsoft[(size_t)row * g.K1 + lane] : (lane == label ? 1.0f : 0.0f);
    const unsigned classes = __ballot_sync(0xffffffffu, lane < g.K1 && wk != 0.0f);
    if (lane < g.K1) t.w[lane] = wk;
    const int R = __reduce_max_sync(0xffffffffu, (lane < g.K1 && wk != 0.0f) ? a.Rk[lane] : 0);
    const int na = 2 * R + 1, ncube = na * na * na;
    // per-axis offsets, digits and in-block indices
    int v0[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const float xa = ax == 0 ? p.x : (ax == 1 ? p.y : p.z);
      v0[ax] = floor_small(__fmul_rn(xa, g.inv_res));
      float hi, lo;
      centre_offset0(v0[ax], xa, g, hi, lo);
      if (lane < na) {
        const float e = centre_offset_at(lane - R, hi, lo, g);
        const int v = v0[ax] + lane - R;
        const int shift = ax == 0 ? 0 : (ax == 1 ? g.B_shift : 2 * g.B_shift);
        const int mul = ax == 0 ? 1 : (ax == 1 ? 3 : 9);
        t.e2[ax][lane] = __fmul_rn(e, e);
        t.part[ax][lane] = (mul * ((v >> g.B_shift) - (v0[ax] >> g.B_shift) + 1)) | ((v & m) << (shift + 8));
      }
    }
    if (lane < 27) {
      const int32_t pool = find_pool_slot(a.hkeys, a.hvals, a.hash_cap,
                                          pack_block((v0[0] >> g.B_shift) - 1 + lane % 3,
                                                     (v0[1] >> g.B_shift) - 1 + (lane / 3) % 3,
                                                     (v0[2] >> g.B_shift) - 1 + lane / 9, map));
      const int32_t pb = pool >= 0 ? pool : a.sink;
      t.blk[lane] = a.alpha + (size_t)pb * g.K1 * g.B3;
      if (kTrack) t.cnt[lane] = a.pairs + (size_t)pb * g.B3;
    }
    __syncwarp();
    for (int c = lane; c - lane < ncube; c += 32) {  // warp-uniform trip count
      const bool live = c < ncube;
      const int cc = live ? c : 0;
      const int jx = cc % na, jy = (cc / na) % na, jz = cc / (na * na);
      const float d2 = __fadd_rn(__fadd_rn(t.e2[0][jx], t.e2[1][jy]), t.e2[2][jz]);
      const int pk = t.part[0][jx] + t.part[1][jy] + t.part[2][jz];
      bool any = false;
      for (unsigned cl = classes; cl; cl &= cl - 1) {  // warp-uniform
        const int k = __ffs(cl) - 1;
        bool in = live && d2 < g.l2k_lo[k];
        const bool band = live && !in && d2 < g.l2k_hi[k];
        if (__any_sync(0xffffffffu, band)) {
          if (band)
            in = in_support64_call(v0[0] + jx - R, v0[1] + jy - R, v0[2] + jz - R, p.x, p.y, p.z, g.res64,
                                   g.l2k_64[k]);
        }
        if (in) {
          const float r = __fmul_rn(sqrtf(d2), g.inv_lk[k]);
          atomicAdd(t.blk[pk & 0xff] + (size_t)k * g.B3 + (pk >> 8), g.sigma0_k[k] * kernel_f_poly(r) * t.w[k]);
        }
        any = any || in;
      }
      if (any) {
        ++npairs;
        if (kTrack) atomicAdd(t.cnt[pk & 0xff] + (pk >> 8), 1);
      }
    }
    __syncwarp();  // the tables are rewritten for the next point
  }
  for (int o = 16; o > 0; o >>= 1) npairs += __shfl_down_sync(0xffffffffu, npairs, o);
  if (lane == 0) atomicAdd(&a.dc->pairs, (unsigned long long)npairs);
}

}  // namespace

cudaError_t launch_soft_weights(MapState& m) {
  const unsigned grid = (unsigned)(m.sm_count * 8);  // persistent: warps stride over the training points
  soft_weights_kernel<<<grid, 128, 0, m.stream>>>(m.s.seg_start, m.s.vals, m.s.hit_src, m.s.train, m.s.desc,
                                                  m.s.softidx, m.s.wsoft, m.g.K1, m.dc);
  m.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_soft_export(MapState& m, float* xyz, float* w, int64_t cap) {
  soft_export_kernel<<<(unsigned)(m.sm_count * 8), 256, 0, m.stream>>>(m.s.train, m.s.softidx, m.s.wsoft, m.g.K1,
                                                                      cap, xyz, w, m.dc);
  m.launches += 1;
  return cudaGetLastError();
}

// Zero-fills the blocks created by this update (unless the fast form ran
// first and did), then the weighted accumulation of the points of every class
// outside `skip`.
cudaError_t launch_accumulate_weighted(MapState& m, bool soft, bool fill, uint32_t skip) {
  if (fill) {
    cudaError_t e = launch_fresh_fill(m);
    if (e != cudaSuccess) return e;
  }
  WArgs a;
  a.g = m.g;
  a.train = m.s.train;
  a.softidx = soft ? m.s.softidx : nullptr;
  a.wsoft = soft ? m.s.wsoft : nullptr;
  a.hkeys = m.hkeys;
  a.hvals = m.hvals;
  a.hash_cap = m.hash_cap;
  a.alpha = m.alpha;
  a.pairs = m.pairs;
  a.sink = (int32_t)m.pool_blocks;
  // offsets j with |j| - 1/2 >= l_k / res hold no voxel centre within l_k of a point in the voxel
  for (int k = 0; k < kMaxClasses; ++k) {
    const double lk = k < m.g.K1 ? m.prm.length_scale * m.prm.l_scale[k] : 0.0;
    a.Rk[k] = k < m.g.K1 ? (int)std::ceil(lk / m.prm.res + 0.5 + 1e-6) - 1 : 0;
    if (2 * a.Rk[k] + 1 > kWAxis - 1) return cudaErrorInvalidValue;
  }
  a.skip = soft ? 0u : skip;
  a.dc = m.dc;
  const unsigned grid = (unsigned)(m.sm_count * 16);
  if (m.pairs) accumulate_weighted_kernel<true><<<grid, kWThreads, 0, m.stream>>>(a);
  else accumulate_weighted_kernel<false><<<grid, kWThreads, 0, m.stream>>>(a);
  m.launches += 1;
  return cudaGetLastError();
}

}  // namespace sbki
