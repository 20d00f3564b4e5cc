// Step a5, point-major form: one warp per training point adds
// sigma0 f(|c_v - x_i| / l) (Eq. alpha_kernel, Eq. kernel) into every voxel
// centre within l, with one global floating-point reduction per pair.
//
// Candidate voxels come from a static table.  Split the voxel of a point into
// 8x8x8 parts by the point's sub-voxel position; for each part the table
// lists every offset (dx, dy, dz) (relative to the point's voxel) whose centre
// can lie within l of some position in that part, widened by 0.001 voxel on
// every side (so FP32 rounding of the position cannot pick too small a list).
// For l = 3 res a list has at most 136 entries (94 % of them at most 128, four
// sweeps of 32), against ~113 in support.
// Per point the warp
//   1. forms the compensated offsets E0 = c(v0) - x of the point's own voxel
//      centre (hi + lo per axis) and fills two per-warp lookup tables in
//      shared memory: X[dx] = (ex^2, x-part of the voxel address) and
//      YZ[dy, dz] = (ey^2 + ez^2, y/z-part of the voxel address), where an
//      address part holds the block-offset digit (base 3 per axis) in its low
//      byte and the in-block index above it, so the two parts add up to the
//      full address without carries; and the pointers to class y_i of the
//      (at most 27) blocks the ball can reach;
//   2. sweeps its part's list, 32 candidates at a time (fully unrolled for
//      the common list lengths): a list entry holds the byte offsets of its X
//      and YZ rows, so d^2 and the address are two shared-memory loads and two
//      adds; the FP32 test (re-decided in FP64 inside the relative band around
//      l^2), the kernel value and red.global.add.f32 into alpha.  Padding
//      entries point at an X row with d^2 = 1e30.
// Training points arrive sorted by their downsampling cell, so the warps in
// flight at any moment update a compact region of the map (L2 locality).
// Blocks allocated by this update are zero-filled before (fresh_fill_kernel).
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "kernel_value.cuh"
#include "point_common.cuh"

namespace sbki {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kAxisMax = 15;             // offsets per axis: 2R + 1 <= 15
constexpr int kYZMax = kAxisMax * kAxisMax;
constexpr float kFar = 1.0e30f;          // d^2 of the padding row

struct PtArgs {
  Geom g;
  const float4* train;
  const unsigned long long* hkeys;
  const int32_t* hvals;
  int64_t hash_cap;
  float* alpha;
  int32_t* pairs;
  const uint32_t* ctab;  // [kParts^3][tpad] (X byte offset | YZ byte offset << 8 | dy << 19 | dz << 23)
  const int32_t* clen;   // [kParts^3] entries of each list
  int tpad;              // entries per list (multiple of 32)
  int R;                 // offsets per axis span [-R, R]
  uint32_t recip_na;     // small_recip(2R + 1)
  int chunk;             // consecutive training points per warp (fast set-up form)
  int32_t sink;          // spare pool block that absent neighbour blocks point at
  DevCounters* dc;
};

struct WarpTables {
  float2 x[kAxisMax + 1];  // (e_x^2, address part as int bits); entry 2R+1 is the padding row
  float2 yz[kYZMax];
  float* blk[27];          // alpha + (pool * (K+1) + y_i) * B^3 (pool = the spare block when absent)
  int32_t* cnt[27];        // pair counts of the block (tracking only)
};

// One candidate per lane, branch-free except for the (rare, warp-uniform)
// FP64 re-decision: every lane evaluates the kernel and the reduction is
// predicated.  Every list entry (padding included) yields a block digit in
// 0..26, so the block-pointer load is always in range.  A neighbour block
// that is not in the map holds no voxel within l of any training point of
// this update (the touched-block pass applies the same membership test and
// allocated every block that does), so no in-support pair reaches it; its
// pointer names the spare block after the pool, so the reduction needs no
// null test.  s0 is the point's class scale sigma0 * sigma0_scale[y_i].
// Returns 1 for an in-support pair.
template <bool kTrack>
__device__ __forceinline__ uint32_t candidate(const PtArgs& a, const WarpTables& t, uint32_t ent, const int v0[3],
                                              const float4& p, float s0) {
  const Geom& g = a.g;
  const float2 ex = *reinterpret_cast<const float2*>(reinterpret_cast<const char*>(t.x) + (ent & 0xffu));
  const float2 eyz = *reinterpret_cast<const float2*>(reinterpret_cast<const char*>(t.yz) + ((ent >> 8) & 0x7ffu));
  const float d2 = __fadd_rn(ex.x, eyz.x);
  const int pk = __float_as_int(ex.y) + __float_as_int(eyz.y);
  bool in = d2 < g.l2_lo;
  const bool band = !in && d2 < g.l2_hi;
  if (__any_sync(0xffffffffu, band)) {
    if (band)
      in = in_support64_call(v0[0] + (int)((ent & 0xffu) >> 3) - a.R, v0[1] + (int)((ent >> 19) & 15u) - a.R,
                             v0[2] + (int)((ent >> 23) & 15u) - a.R, p.x, p.y, p.z, g.res64, g.l2_64);
  }
  float* base = t.blk[pk & 0xff];
  const float d = d2 * rsqrtf(fmaxf(d2, 1e-30f));
  const float u = fmaxf(__fmaf_rn(-d, g.inv_l, 1.0f), 0.0f);
  const float w = u * u;
  red_add_if(in, base + (pk >> 8), s0 * (w * w * u * kernel_q(w)));
  if (kTrack) red_add_if(in, t.cnt[pk & 0xff] + (pk >> 8), 1);
  return in ? 1u : 0u;
}

// kNit > 0: lists of exactly kNit x 32 entries, unrolled; 0: any length
template <bool kTrack, int kNit>
__global__ void __launch_bounds__(kThreads, 4) accumulate_points_kernel(PtArgs a) {
  __shared__ WarpTables s_tab[kWarps];
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const int R = a.R, na = 2 * R + 1;
  WarpTables& t = s_tab[wid];
  uint32_t npairs = 0;
  if (a.dc->err != 0) return;
  const uint32_t P = a.dc->n_train;
  if (lane == 0) t.x[na] = make_float2(kFar, __int_as_float(0));
  float4 pnext = gw < P ? a.train[gw] : make_float4(0.f, 0.f, 0.f, 0.f);
  for (uint32_t i = gw; i < P; i += nw) {
    const float4 p = pnext;
    if (i + nw < P) pnext = a.train[i + nw];  // in flight while this point is processed
    const int lm = label_of(p.w);  // label + 32 * map
    const int label = lm & ((1 << kLabelBits) - 1), map = lm >> kLabelBits;
    const float s0 = g.sigma0_k[label];  // class label's kernel scale
    const PointFrame f = point_frame(p.x, p.y, p.z, R, g);
    const uint32_t* tab = a.ctab + f.part * a.tpad;
    const int len = __ldg(a.clen + f.part);
    // X rows
    if (lane < na) {
      const float e = centre_offset_at(lane - R, f.hi[0], f.lo[0], g);
      t.x[lane] = make_float2(__fmul_rn(e, e), __int_as_float(xpart(f, lane, R, g)));
    }
    // Y rows in lanes 0..15, Z rows in lanes 16..31, combined into YZ rows by shuffles
    float sq1 = 0.f;
    int pk1 = 0;
    {
      const int ax = 1 + (lane >> 4), j = min(lane & 15, na - 1);
      const float e = centre_offset_at(j - R, f.hi[ax], f.lo[ax], g);
      const int v = f.v0[ax] + j - R, m = g.B - 1;
      sq1 = __fmul_rn(e, e);
      pk1 = ax == 1 ? (3 * ((v >> g.B_shift) - f.blo[1])) | ((v & m) << (g.B_shift + 8))
                    : (9 * ((v >> g.B_shift) - f.blo[2])) | ((v & m) << (2 * g.B_shift + 8));
    }
    for (int q0 = 0; q0 < na * na; q0 += 32) {  // uniform trip count: full-warp shuffles
      const int q = min(q0 + lane, na * na - 1);
      const int jy = (int)small_div((uint32_t)q, a.recip_na), jz = q - jy * na;
      const float sy = __shfl_sync(0xffffffffu, sq1, jy), sz = __shfl_sync(0xffffffffu, sq1, 16 + jz);
      const int py = __shfl_sync(0xffffffffu, pk1, jy), pz = __shfl_sync(0xffffffffu, pk1, 16 + jz);
      if (q0 + lane < na * na) t.yz[q] = make_float2(__fadd_rn(sy, sz), __int_as_float(py + pz));
    }
    // blocks the ball can reach: digit (bx, by, bz) in base 3
    if (lane < 27) {
      const int32_t pool = digit_pool(f, lane, map, a.hkeys, a.hvals, a.hash_cap);
      t.blk[lane] = a.alpha + ((size_t)(pool >= 0 ? pool : a.sink) * g.K1 + label) * g.B3;
      if (kTrack) t.cnt[lane] = a.pairs + (size_t)(pool >= 0 ? pool : a.sink) * g.B3;
    }
    __syncwarp();
    if (kNit > 0) {
      uint32_t ent[kNit > 0 ? kNit : 1];
#pragma unroll
      for (int it = 0; it < kNit; ++it) ent[it] = it * 32 < len ? __ldg(tab + it * 32 + lane) : 0u;
#pragma unroll
      for (int it = 0; it < kNit; ++it)
        if (it * 32 < len) npairs += candidate<kTrack>(a, t, ent[it], f.v0, p, s0);  // warp-uniform
    } else {
      for (int k = lane; k - lane < len; k += 32) npairs += candidate<kTrack>(a, t, __ldg(tab + k), f.v0, p, s0);
    }
    __syncwarp();  // the tables are rewritten for the next point
  }
  for (int o = 16; o > 0; o >>= 1) npairs += __shfl_down_sync(0xffffffffu, npairs, o);
  if (lane == 0) atomicAdd(&a.dc->pairs, (unsigned long long)npairs);
}

// The same update with a cheaper per-point set-up, for 2R + 1 <= 8 (l up to
// about 3 voxels).  A warp takes kChunk consecutive training points (sorted by
// tile, so mostly one block) in groups of up to kGroup.  For a group, three
// lanes per point (one per axis) form that axis's compensated offsets and
// address parts for offsets -R..R at once, into per-point rows in shared
// memory, with the point's sub-voxel part, block and voxel.  Then, point by
// point, the warp combines the Y and Z rows into YZ rows, refreshes the pool
// slots of the 27 blocks around the point's block when the block (or map)
// changed, and sweeps the candidate list with the point's own X rows.
constexpr int kGroup = 10;  // points whose rows one warp forms at once (3 lanes each)
constexpr int kFastAxis = 8;  // rows per axis: 2R + 1 <= 7 offsets and the padding row

struct alignas(16) PointRows {
  float2 r[3][kFastAxis];  // per axis: (e^2, address part) of offset j - R; r[0][2R + 1] is the padding row
  int pt[4];               // sub-voxel part per axis, label word
  int blk[4];              // block per axis
  int v0[4];               // voxel per axis
};

struct FastTables {
  PointRows pts[kGroup];
  float2 yz[kFastAxis * kFastAxis];  // YZ rows of the point being swept
  float* blk[27];
  int32_t* cnt[27];
};

// As candidate(), with the X rows of one point of the group; the point's
// coordinates are loaded again only on the (rare) FP64 re-decision.
template <bool kTrack>
__device__ __forceinline__ uint32_t candidate_rows(const PtArgs& a, const FastTables& t, const PointRows& pr,
                                                   uint32_t ent, uint32_t i, float s0) {
  const Geom& g = a.g;
  const float2 ex = *reinterpret_cast<const float2*>(reinterpret_cast<const char*>(pr.r[0]) + (ent & 0xffu));
  const float2 eyz = *reinterpret_cast<const float2*>(reinterpret_cast<const char*>(t.yz) + ((ent >> 8) & 0x7ffu));
  const float d2 = __fadd_rn(ex.x, eyz.x);
  const int pk = __float_as_int(ex.y) + __float_as_int(eyz.y);
  bool in = d2 < g.l2_lo;
  const bool band = !in && d2 < g.l2_hi;
  if (__any_sync(0xffffffffu, band)) {
    if (band) {
      const float4 p = a.train[i];
      in = in_support64_call(pr.v0[0] + (int)((ent & 0xffu) >> 3) - a.R, pr.v0[1] + (int)((ent >> 19) & 15u) - a.R,
                             pr.v0[2] + (int)((ent >> 23) & 15u) - a.R, p.x, p.y, p.z, g.res64, g.l2_64);
    }
  }
  float* base = t.blk[pk & 0xff];
  const float d = d2 * rsqrtf(fmaxf(d2, 1e-30f));
  const float u = fmaxf(__fmaf_rn(-d, g.inv_l, 1.0f), 0.0f);
  const float w = u * u;
  red_add_if(in, base + (pk >> 8), s0 * (w * w * u * kernel_q(w)));
  if (kTrack) red_add_if(in, t.cnt[pk & 0xff] + (pk >> 8), 1);
  return in ? 1u : 0u;
}

template <bool kTrack, int kNit>
__global__ void __launch_bounds__(kThreads, 4) accumulate_points_fast_kernel(PtArgs a) {
  __shared__ FastTables s_tab[kWarps];
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const int R = a.R, na = 2 * R + 1, m = g.B - 1;
  FastTables& t = s_tab[wid];
  uint32_t npairs = 0;
  if (a.dc->err != 0) return;
  const uint32_t P = a.dc->n_train;
  // this lane's point of a group and axis (lanes 30, 31 form no rows)
  const int gl = lane / 3, ax = lane - 3 * (lane / 3);
  const int axshift = ax == 0 ? 0 : (ax == 1 ? g.B_shift : 2 * g.B_shift);
  const int dmul = ax == 0 ? 1 : (ax == 1 ? 3 : 9);
  int cb[3] = {INT_MIN, INT_MIN, INT_MIN}, cmap = -1;  // block and map the cached slots belong to
  int32_t pool = -1;                                   // lanes 0..26: slot of block digit `lane`
  const uint32_t chunk = (uint32_t)a.chunk;
  for (uint32_t c = gw; c * chunk < P; c += nw) {
    const uint32_t c1 = min(P, c * chunk + chunk);
    for (uint32_t g0 = c * chunk; g0 < c1; g0 += kGroup) {
      const uint32_t gn = min(c1 - g0, (uint32_t)kGroup);  // warp-uniform
      // 1. rows of every point of the group, three lanes per point
      if (gl < (int)gn) {
        const float4 p = a.train[g0 + gl];
        const float xa = ax == 0 ? p.x : (ax == 1 ? p.y : p.z);
        const int v0 = floor_small(__fmul_rn(xa, g.inv_res));
        float hi, lo;
        centre_offset0(v0, xa, g, hi, lo);
        const float phi = 0.5f - __fmul_rn(__fadd_rn(hi, lo), g.inv_res);
        const int b0 = v0 >> g.B_shift;
        PointRows& pr = t.pts[gl];
#pragma unroll
        for (int j = 0; j < kFastAxis; ++j) {
          if (j < na) {
            const float e = centre_offset_at(j - R, hi, lo, g);
            const int v = v0 + j - R;
            pr.r[ax][j] = make_float2(__fmul_rn(e, e),
                                      __int_as_float(dmul * ((v >> g.B_shift) - (b0 - 1)) | ((v & m) << (axshift + 8))));
          }
        }
        if (ax == 0) pr.r[0][na] = make_float2(kFar, __int_as_float(0));
        pr.pt[ax] = min(kParts - 1, max(0, floor_small(phi * (float)kParts)));
        pr.blk[ax] = b0;
        pr.v0[ax] = v0;
        if (ax == 0) pr.pt[3] = label_of(p.w);
      }
      __syncwarp();
      // 2. point by point: YZ rows, block slots, candidate sweeps
      for (uint32_t k = 0; k < gn; ++k) {
        const PointRows& pr = t.pts[k];
        const int4 ip = *reinterpret_cast<const int4*>(pr.pt);
        const int4 ib = *reinterpret_cast<const int4*>(pr.blk);
        const int part = ip.x + kParts * (ip.y + kParts * ip.z);
        const int label = ip.w & ((1 << kLabelBits) - 1), map = ip.w >> kLabelBits;
        const float s0 = g.sigma0_k[label];  // class label's kernel scale
        for (int q0 = 0; q0 < na * na; q0 += 32) {
          const int q = min(q0 + lane, na * na - 1);
          const int jy = (int)small_div((uint32_t)q, a.recip_na), jz = q - jy * na;
          const float2 ry = pr.r[1][jy], rz = pr.r[2][jz];
          if (q0 + lane < na * na)
            t.yz[q] = make_float2(__fadd_rn(ry.x, rz.x), __int_as_float(__float_as_int(ry.y) + __float_as_int(rz.y)));
        }
        if (ib.x != cb[0] || ib.y != cb[1] || ib.z != cb[2] || map != cmap) {  // warp-uniform
          cb[0] = ib.x;
          cb[1] = ib.y;
          cb[2] = ib.z;
          cmap = map;
          pool = -1;
          if (lane < 27)
            pool = find_pool_slot(a.hkeys, a.hvals, a.hash_cap,
                                  pack_block(ib.x - 1 + lane % 3, ib.y - 1 + (lane / 3) % 3, ib.z - 1 + lane / 9, map));
        }
        if (lane < 27) {
          t.blk[lane] = a.alpha + ((size_t)(pool >= 0 ? pool : a.sink) * g.K1 + label) * g.B3;
          if (kTrack) t.cnt[lane] = a.pairs + (size_t)(pool >= 0 ? pool : a.sink) * g.B3;
        }
        __syncwarp();
        const uint32_t* tab = a.ctab + part * a.tpad;
        const int len = __ldg(a.clen + part);
        const uint32_t i = g0 + k;
        if (kNit > 0) {
          uint32_t ent[kNit > 0 ? kNit : 1];
#pragma unroll
          for (int it = 0; it < kNit; ++it) ent[it] = it * 32 < len ? __ldg(tab + it * 32 + lane) : 0u;
#pragma unroll
          for (int it = 0; it < kNit; ++it)
            if (it * 32 < len) npairs += candidate_rows<kTrack>(a, t, pr, ent[it], i, s0);  // warp-uniform
        } else {
          for (int q = lane; q - lane < len; q += 32)
            npairs += candidate_rows<kTrack>(a, t, pr, __ldg(tab + q), i, s0);
        }
        __syncwarp();  // the YZ rows and block pointers are rewritten for the next point
      }
    }
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

// Candidate lists of the kParts^3 sub-voxel parts (host, once per map).  The
// parts are widened by delta = 1e-3 voxel, far above the FP32 error of the
// sub-voxel position (~1e-6 voxel), so a point's list always holds its ball.
cudaError_t build_candidate_tables(MapState& m) {
  const double lr = m.prm.length_scale / m.prm.res, delta = 1e-3;
  const int R = (int)std::ceil(lr + 0.5 + delta);
  constexpr int kLists = kParts * kParts * kParts;
  std::vector<std::vector<int32_t>> lists(kLists);
  size_t longest = 0;
  for (int t = 0; t < kLists; ++t) {
    const int pt[3] = {t % kParts, (t / kParts) % kParts, t / (kParts * kParts)};
    for (int dz = -R; dz <= R; ++dz)
      for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx) {
          const int d[3] = {dx, dy, dz};
          double m2 = 0.0;
          for (int a = 0; a < 3; ++a) {
            const double md =
                min_axis_distance(d[a], (double)pt[a] / kParts - delta, (double)(pt[a] + 1) / kParts + delta);
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
  // re-pack with the tight R (the lookups hold 2R + 1 <= 15 entries per axis):
  // X row jx at byte offset 8 jx, YZ row (jy, jz) at byte offset 8 (jy (2R+1) + jz);
  // padding entries point at X row 2R + 1 (d^2 = 1e30) and YZ row 0
  const int Rt = maxd, na = 2 * Rt + 1;
  if (na > kAxisMax) return cudaErrorInvalidValue;
  const int tpad = (int)((longest + 31) / 32 * 32);
  std::vector<uint32_t> flat((size_t)kLists * tpad, (uint32_t)(8 * na));
  std::vector<int32_t> len(kLists);
  for (int t = 0; t < kLists; ++t) len[t] = (int32_t)lists[t].size();
  for (int t = 0; t < kLists; ++t)
    for (size_t k = 0; k < lists[t].size(); ++k) {
      const int32_t e = lists[t][k];
      const uint32_t jx = (uint32_t)((e & 15) - R + Rt), jy = (uint32_t)(((e >> 4) & 15) - R + Rt),
                     jz = (uint32_t)(((e >> 8) & 15) - R + Rt);
      flat[(size_t)t * tpad + k] = (8u * jx) | ((8u * (jy * na + jz)) << 8) | (jy << 19) | (jz << 23);
    }
  cudaError_t e = cudaMalloc(&m.ctab, sizeof(uint32_t) * flat.size());
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&m.clen, sizeof(int32_t) * len.size());
  if (e != cudaSuccess) return e;
  m.ctab_pad = tpad;
  m.ctab_R = Rt;
  e = cudaMemcpy(m.clen, len.data(), sizeof(int32_t) * len.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(m.ctab, flat.data(), sizeof(uint32_t) * flat.size(), cudaMemcpyHostToDevice);
}

namespace {

// ctas_per_sm: 0 = as many as fit
template <bool kTrack, int kNit>
cudaError_t launch_points(const PtArgs& a, int sm_count, int ctas_per_sm, cudaStream_t st) {
  int per_sm = 0;
  cudaError_t e;
  if (2 * a.R + 1 <= 8) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, accumulate_points_fast_kernel<kTrack, kNit>, kThreads,
                                                      0);
    if (e != cudaSuccess) return e;
    if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
    accumulate_points_fast_kernel<kTrack, kNit><<<std::max(1, per_sm) * sm_count, kThreads, 0, st>>>(a);
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, accumulate_points_kernel<kTrack, kNit>, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
    accumulate_points_kernel<kTrack, kNit><<<std::max(1, per_sm) * sm_count, kThreads, 0, st>>>(a);
  }
  return cudaGetLastError();
}

template <bool kTrack>
cudaError_t launch_points_nit(const PtArgs& a, int sm_count, int ctas_per_sm, cudaStream_t st) {
  switch (a.tpad / 32) {  // unrolled sweeps for the common list lengths
    case 2: return launch_points<kTrack, 2>(a, sm_count, ctas_per_sm, st);
    case 3: return launch_points<kTrack, 3>(a, sm_count, ctas_per_sm, st);
    case 4: return launch_points<kTrack, 4>(a, sm_count, ctas_per_sm, st);
    case 5: return launch_points<kTrack, 5>(a, sm_count, ctas_per_sm, st);
    case 6: return launch_points<kTrack, 6>(a, sm_count, ctas_per_sm, st);
    default: return launch_points<kTrack, 0>(a, sm_count, ctas_per_sm, st);
  }
}

}  // namespace

cudaError_t launch_fresh_fill(MapState& m) {
  fresh_fill_kernel<<<m.sm_count * 4, 256, 0, m.stream>>>(m.s.fresh, m.hvals, m.alpha, m.pairs, m.g.K1 * m.g.B3,
                                                          m.g.B3, m.dc);
  m.launches += 1;
  return cudaGetLastError();
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
  a.clen = m.clen;
  a.tpad = m.ctab_pad;
  a.R = m.ctab_R;
  a.recip_na = ((1u << 20) + (uint32_t)(2 * m.ctab_R + 1) - 1u) / (uint32_t)(2 * m.ctab_R + 1);
  a.chunk = std::max(1, std::min(64, m.tune.accumulate_chunk));
  a.sink = (int32_t)m.pool_blocks;
  a.dc = m.dc;
  m.launches += 2;
  const int cps = m.tune.accumulate_ctas_per_sm;
  return m.pairs ? launch_points_nit<true>(a, m.sm_count, cps, m.stream)
                 : launch_points_nit<false>(a, m.sm_count, cps, m.stream);
}

}  // namespace sbki
