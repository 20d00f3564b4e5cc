// Step a5, point-major form: one warp per training point adds
// sigma0 f(|c_v - x_i| / l) (Eq. alpha_kernel, Eq. kernel) into every voxel
// centre within l, with one global floating-point reduction per pair.
//
// Candidate voxels come from a static table.  Split the voxel of a point into
// 3x3x3 parts by the point's sub-voxel position; for each part the table
// lists every offset d (relative to the point's voxel) whose centre can lie
// within l of some position in that part, widened by 0.01 voxel on every side
// (so FP32 rounding of the position cannot pick too small a list).  For
// l = 3 res a list has at most 154 entries, against ~113 in support.
// Per point the warp
//   1. forms the compensated offsets E0 = c(v0) - x of the point's own voxel
//      centre (hi + lo per axis) and, per axis and per offset d, the squared
//      offset (E0 + d res)^2 and the block / in-block index of voxel v0 + d
//      (shared memory, one lane per entry); looks up the pool slots of the
//      blocks the ball can reach (one lane per block);
//   2. sweeps its part's list, 32 candidates at a time: d^2 is the sum of
//      three looked-up squares; the FP32 test (re-decided in FP64 inside the
//      relative band around l^2), the kernel value, and red.global.add.f32
//      into alpha.  Lists are sorted z, y, x so that neighbouring lanes update
//      neighbouring voxels.
// Training points arrive sorted by their downsampling cell, so the warps in
// flight at any moment update a compact region of the map (L2 locality).
// Blocks allocated by this update are zero-filled before (fresh_fill_kernel).
#include <algorithm>
#include <cmath>
#include <vector>

#include "kernel_value.cuh"
#include "sbki_internal.cuh"

namespace sbki {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kAxisMax = 16;  // offsets per axis: 2R + 1 <= 15

struct PtArgs {
  Geom g;
  const float4* train;
  const unsigned long long* hkeys;
  const int32_t* hvals;
  int64_t hash_cap;
  float* alpha;
  int32_t* pairs;
  const int32_t* ctab;  // [27][tpad] packed (ix | iy << 4 | iz << 8), -1 = none
  int tpad;             // entries per list (multiple of 32)
  int R;                // offsets per axis span [-R, R]
  DevCounters* dc;
};

__device__ __forceinline__ int floor_i(float v) { return (int)floorf(v); }

__device__ int32_t find_pool(const PtArgs& a, unsigned long long key) {
  uint32_t slot = hash_slot(key, a.hash_cap);
  for (int probe = 0; probe < kMaxProbes; ++probe) {
    const unsigned long long k = a.hkeys[slot];
    if (k == key) return a.hvals[slot];
    if (k == kEmpty) return -1;
    slot = (uint32_t)((slot + 1) & (uint32_t)(a.hash_cap - 1));
  }
  return -1;
}

template <bool kTrack>
__global__ void __launch_bounds__(kThreads) accumulate_points_kernel(PtArgs a) {
  __shared__ float s_sq[kWarps][3][kAxisMax];
  __shared__ int s_pk[kWarps][3][kAxisMax];  // (block index weight) << 16 | in-block index weight
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const int B = g.B, K1B3 = g.K1 * g.B3, R = a.R, naxis = 2 * R + 1;
  const uint32_t maxis = small_recip(naxis);
  float(*sq)[kAxisMax] = s_sq[wid];
  int(*pk)[kAxisMax] = s_pk[wid];
  uint32_t npairs = 0;
  if (a.dc->err != 0) return;
  const uint32_t P = a.dc->n_train;
  float4 pnext = gw < P ? a.train[gw] : make_float4(0.f, 0.f, 0.f, 0.f);
  for (uint32_t i = gw; i < P; i += nw) {
    const float4 p = pnext;
    if (i + nw < P) pnext = a.train[i + nw];  // in flight while this point is processed
    const int label = (int)p.w;
    const float xs[3] = {p.x, p.y, p.z};
    int v0[3], part[3], blo[3], nb[3];
    float hi[3], lo[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      v0[ax] = floor_i(__fmul_rn(xs[ax], g.inv_res));
      centre_offset0(v0[ax], xs[ax], g, hi[ax], lo[ax]);
      // sub-voxel position 1/2 - E0/res (accurate anywhere in the map), in thirds
      const float phi = 0.5f - __fmul_rn(__fadd_rn(hi[ax], lo[ax]), g.inv_res);
      part[ax] = min(2, max(0, floor_i(phi * 3.0f)));
      blo[ax] = (v0[ax] - R) >> g.B_shift;
      nb[ax] = ((v0[ax] + R) >> g.B_shift) - blo[ax] + 1;
    }
    const int32_t* tab = a.ctab + (part[0] + 3 * part[1] + 9 * part[2]) * a.tpad;
    // per-axis lookups: lane -> (axis, offset)
    for (int q = lane; q < 3 * naxis; q += 32) {
      const int ax = (int)small_div(q, maxis), j = q - ax * naxis, d = j - R;
      const float h = ax == 0 ? hi[0] : (ax == 1 ? hi[1] : hi[2]);
      const float l0 = ax == 0 ? lo[0] : (ax == 1 ? lo[1] : lo[2]);
      const int vv = (ax == 0 ? v0[0] : (ax == 1 ? v0[1] : v0[2])) + d;
      const int bl = ax == 0 ? blo[0] : (ax == 1 ? blo[1] : blo[2]);
      const int w = ax == 0 ? 1 : (ax == 1 ? nb[0] : nb[0] * nb[1]);
      const int stride = ax == 0 ? 1 : (ax == 1 ? B : B * B);
      const float e = centre_offset_at(d, h, l0, g);
      sq[ax][j] = __fmul_rn(e, e);
      pk[ax][j] = (((vv >> g.B_shift) - bl) * w << 16) | ((vv & (B - 1)) * stride);
    }
    int32_t pool = -1;
    const int nblk = nb[0] * nb[1] * nb[2];
    if (lane < nblk) {
      const uint32_t mx = small_recip(nb[0]), mxy = small_recip(nb[0] * nb[1]);
      const int cz = (int)small_div(lane, mxy), cxy = lane - cz * nb[0] * nb[1];
      const int cy = (int)small_div(cxy, mx), cx = cxy - cy * nb[0];
      pool = find_pool(a, pack_block(blo[0] + cx, blo[1] + cy, blo[2] + cz));
    }
    __syncwarp();
    float* base = a.alpha + (size_t)label * g.B3;
    for (int k = lane; k < a.tpad; k += 32) {  // uniform trip count: full-warp shuffle below
      const int ent = __ldg(tab + k);
      const bool live = ent >= 0;
      const int ix = ent & 15, iy = (ent >> 4) & 15, iz = (ent >> 8) & 15;
      const float d2 = live ? __fadd_rn(__fadd_rn(sq[0][ix], sq[1][iy]), sq[2][iz]) : 3.0e38f;
      const int ps = pk[0][ix] + pk[1][iy] + pk[2][iz];
      bool in = d2 < g.l2_lo;
      if (!in && d2 < g.l2_hi)
        in = in_support64(v0[0] + ix - R, v0[1] + iy - R, v0[2] + iz - R, p.x, p.y, p.z, g);
      const int32_t pl = __shfl_sync(0xffffffffu, pool, live ? (ps >> 16) : 0);
      if (in && pl >= 0) {
        const float d = d2 * rsqrtf(fmaxf(d2, 1e-30f));
        const float u = __fmul_rn(__fsub_rn(g.l, d), g.inv_l);
        const int local = ps & 0xffff;
        atomicAdd(base + (size_t)pl * K1B3 + local, g.sigma0 * kernel_f_poly_u(u));
        if (kTrack) atomicAdd(a.pairs + (size_t)pl * g.B3 + local, 1);
      }
      npairs += (in && pl >= 0) ? 1u : 0u;
    }
    __syncwarp();  // the lookups are rewritten for the next point
  }
  for (int o = 16; o > 0; o >>= 1) npairs += __shfl_down_sync(0xffffffffu, npairs, o);
  if (lane == 0) atomicAdd(&a.dc->pairs, (unsigned long long)npairs);
}

// Blocks created by this update start at zero (and so do their pair counts).
__global__ void fresh_fill_kernel(const uint32_t* fresh, const int32_t* hvals, float* alpha, int32_t* pairs, int K1B3,
                                  int B3, DevCounters* dc) {
  if (dc->err != 0) return;
  const uint32_t n_new = dc->n_new;
  for (uint32_t f = blockIdx.x; f < n_new; f += gridDim.x) {
    const int32_t pl = hvals[fresh[f]];
    float4* dst = reinterpret_cast<float4*>(alpha + (size_t)pl * K1B3);
    for (int e = threadIdx.x; e < K1B3 / 4; e += blockDim.x) dst[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pairs)
      for (int e = threadIdx.x; e < B3; e += blockDim.x) pairs[(size_t)pl * B3 + e] = 0;
  }
}

// min over phi in [lo, hi] of |d + 1/2 - phi| (voxel units)
double min_axis_distance(int d, double lo, double hi) {
  const double c = d + 0.5;
  if (c >= lo && c <= hi) return 0.0;
  return std::min(std::fabs(c - lo), std::fabs(c - hi));
}

}  // namespace

// Candidate lists of the 27 sub-voxel parts (host, once per map).
cudaError_t build_candidate_tables(MapState& m) {
  const double lr = m.prm.length_scale / m.prm.res, delta = 0.01;
  const int R = (int)std::ceil(lr + 0.5 + delta);
  std::vector<std::vector<int32_t>> lists(27);
  size_t longest = 0;
  for (int t = 0; t < 27; ++t) {
    const int pt[3] = {t % 3, (t / 3) % 3, t / 9};
    for (int dz = -R; dz <= R; ++dz)
      for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx) {
          const int d[3] = {dx, dy, dz};
          double m2 = 0.0;
          for (int a = 0; a < 3; ++a) {
            const double md = min_axis_distance(d[a], pt[a] / 3.0 - delta, (pt[a] + 1) / 3.0 + delta);
            m2 += md * md;
          }
          if (m2 < lr * lr * (1.0 + 1e-5))
            lists[t].push_back((dx + R) | ((dy + R) << 4) | ((dz + R) << 8));
        }
    longest = std::max(longest, lists[t].size());
  }
  int maxd = 0;  // offsets actually used
  for (auto& L : lists)
    for (int32_t e : L)
      for (int a = 0; a < 3; ++a) maxd = std::max(maxd, std::abs(((e >> (4 * a)) & 15) - R));
  // re-pack with the tight R (the lookups hold 2R + 1 <= 15 entries per axis)
  const int Rt = maxd;
  const int tpad = (int)((longest + 31) / 32 * 32);
  std::vector<int32_t> flat((size_t)27 * tpad, -1);
  for (int t = 0; t < 27; ++t)
    for (size_t k = 0; k < lists[t].size(); ++k) {
      const int32_t e = lists[t][k];
      const int dx = (e & 15) - R, dy = ((e >> 4) & 15) - R, dz = ((e >> 8) & 15) - R;
      flat[(size_t)t * tpad + k] = (dx + Rt) | ((dy + Rt) << 4) | ((dz + Rt) << 8);
    }
  if (2 * Rt + 1 > kAxisMax) return cudaErrorInvalidValue;
  cudaError_t e = cudaMalloc(&m.ctab, sizeof(int32_t) * flat.size());
  if (e != cudaSuccess) return e;
  m.ctab_pad = tpad;
  m.ctab_R = Rt;
  return cudaMemcpy(m.ctab, flat.data(), sizeof(int32_t) * flat.size(), cudaMemcpyHostToDevice);
}

cudaError_t launch_accumulate_points(MapState& m) {
  fresh_fill_kernel<<<m.sm_count * 4, 256, 0, m.stream>>>(m.s.fresh, m.hvals, m.alpha, m.pairs, m.g.K1 * m.g.B3,
                                                          m.g.B3, m.dc);
  PtArgs a;
  a.g = m.g;
  a.train = m.s.train;
  a.hkeys = m.hkeys;
  a.hvals = m.hvals;
  a.hash_cap = m.hash_cap;
  a.alpha = m.alpha;
  a.pairs = m.pairs;
  a.ctab = m.ctab;
  a.tpad = m.ctab_pad;
  a.R = m.ctab_R;
  a.dc = m.dc;
  int per_sm = 0;
  cudaError_t e;
  if (m.pairs) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, accumulate_points_kernel<true>, kThreads, 0);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, accumulate_points_kernel<false>, kThreads, 0);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, per_sm) * m.sm_count;
  if (m.pairs) accumulate_points_kernel<true><<<grid, kThreads, 0, m.stream>>>(a);
  else accumulate_points_kernel<false><<<grid, kThreads, 0, m.stream>>>(a);
  m.launches += 2;
  return cudaGetLastError();
}

}  // namespace sbki
