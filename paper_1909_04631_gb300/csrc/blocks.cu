// Step a4: the set of blocks touched by this scan's training points, and
// their allocation in the device block hash (Sec. IV: voxels grouped into
// blocks; every voxel of a block is a query point of Eq. alpha_kernel).
//
// A block is touched iff one of its voxel centres lies strictly within l of a
// training point under the same membership rule as the accumulation (the
// FP32 block-local test, re-decided in FP64 inside the band).  Because d^2 is
// a sum of per-axis terms, the nearest voxel centre of a block is found per
// axis; the FP32 nearest index is checked with its two neighbours.
//
// The hash is open addressing with linear probing on 64-bit block keys;
// insertion is one atomicCAS per probe, bounded by kMaxProbes (then
// SBKI_ERR_CAPACITY).  New slots go to a list; commit assigns pool indices
// in one pass, or - if the pool would overflow or an error is pending -
// clears exactly the slots this scan created, which restores the table
// (slots created by this scan lie on no older key's probe chain).
#include <algorithm>

#include "sbki_internal.cuh"

namespace sbki {
namespace {

struct TouchArgs {
  Geom g;
  const float4* train;
  unsigned long long* hkeys;
  int32_t* hvals;
  uint32_t* hmark;
  uint32_t* hcnt;
  uint32_t* hcur;
  int64_t hash_cap;
  uint32_t* touched;
  uint32_t* fresh;
  uint32_t* blist;
  uint32_t* ownslot;  // fast accumulation form (or null): per training point, the hash slot of its own block
  uint32_t* nbrslot;  // [hash_cap][32]: per own block, the hash slots of the neighbour blocks its points touch
  DevCounters* dc;
};

__device__ __forceinline__ int floor_i(float v) { return (int)floorf(v); }

// Marks the slot touched by this update; 1 for the call that marked it first.
// kList: that call also appends the slot to the touched list (the block-major
// form walks it; the point-major form only counts the touched blocks).  A plain
// read skips the atomic when the mark is already there (a mark, once set in
// this update, never changes back).
template <bool kList>
__device__ __forceinline__ uint32_t mark_touched(const TouchArgs& a, uint32_t slot) {
  const uint32_t epoch = a.dc->epoch;
  if (a.hmark[slot] == epoch) return 0u;
  if (atomicExch(&a.hmark[slot], epoch) == epoch) return 0u;
  if (kList) {
    const uint32_t t = atomicAdd(&a.dc->n_touched, 1u);
    a.touched[t] = slot;
  }
  return 1u;
}

// returns the slot of key (inserted if new), or -1 when the probe bound is hit;
// first += 1 when this call marked the block touched first.  A slot holds the
// empty key or, for good, one block key, so a plain read that finds the key
// needs no atomic.
template <bool kList = true>
__device__ int64_t insert_block(const TouchArgs& a, unsigned long long key, uint32_t* first = nullptr) {
  uint32_t slot = hash_slot(key, a.hash_cap);
  for (int probe = 0; probe < kMaxProbes; ++probe) {
    const unsigned long long cur = a.hkeys[slot];
    if (cur == key) {
      const uint32_t f = mark_touched<kList>(a, slot);
      if (first) *first += f;
      return slot;
    }
    if (cur == kEmpty) {
      const unsigned long long prev = atomicCAS(&a.hkeys[slot], kEmpty, key);
      if (prev == kEmpty) {
        const uint32_t i = atomicAdd(&a.dc->n_new, 1u);
        a.fresh[i] = slot;
        a.hvals[slot] = -1;
        const uint32_t f = mark_touched<kList>(a, slot);
        if (first) *first += f;
        return slot;
      }
      if (prev == key) {
        const uint32_t f = mark_touched<kList>(a, slot);
        if (first) *first += f;
        return slot;
      }
    }
    slot = (uint32_t)((slot + 1) & (uint32_t)(a.hash_cap - 1));
  }
  set_error(a.dc, SBKI_ERR_CAPACITY);
  return -1;
}

// slot of a key already in the table, or -1
__device__ int64_t find_block(const TouchArgs& a, unsigned long long key) {
  uint32_t slot = hash_slot(key, a.hash_cap);
  for (int probe = 0; probe < kMaxProbes; ++probe) {
    const unsigned long long k = a.hkeys[slot];
    if (k == key) return slot;
    if (k == kEmpty) return -1;
    slot = (uint32_t)((slot + 1) & (uint32_t)(a.hash_cap - 1));
  }
  return -1;
}

// The support of a point's kernel: the common l, or its class's l_k when
// classes have their own length scales (reading K16).
struct Support {
  float l2_lo, l2_hi;
  double l2_64;
};
__device__ __forceinline__ Support support_of(const Geom& g, int label) {
  Support s;
  if (g.lscaled) {
    s.l2_lo = g.l2k_lo[label];
    s.l2_hi = g.l2k_hi[label];
    s.l2_64 = g.l2k_64[label];
  } else {
    s.l2_lo = g.l2_lo;
    s.l2_hi = g.l2_hi;
    s.l2_64 = g.l2_64;
  }
  return s;
}

// candidate block range of a point: at most 3 blocks per axis (l <= 0.75 B res)
__device__ void candidate_blocks(const float xs[3], const Geom& g, const Support& sup, int blo[3], int bhi[3]) {
  const float lw = __fmul_rn(sqrtf(sup.l2_hi), 1.001f);
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int vlo = floor_i(__fmul_rn(__fsub_rn(xs[ax], lw), g.inv_res)) - 1;
    const int vhi = floor_i(__fmul_rn(__fadd_rn(xs[ax], lw), g.inv_res)) + 1;
    blo[ax] = vlo >> g.B_shift;
    bhi[ax] = min(vhi >> g.B_shift, blo[ax] + 2);
  }
}

// Per point and axis, for each candidate block k on that axis: the squared
// offset to the block's voxel nearest the point along the axis (the point's
// own voxel index clamped into the block), from compensated offsets.  A block
// holds a voxel centre within l iff the sum over the axes is below l^2: the
// FP32 sum decides outside the relative band around l^2, FP64 (also trying
// the clamped voxel's neighbours) inside it.
struct PointBlocks {
  float xs[3];
  int v0[3], blo[3], nb[3], vn[3][3];
  float m2[3][3];
  Support sup;
};

__device__ __forceinline__ void point_blocks(const float4& p, const Geom& g, PointBlocks& pb) {
  pb.xs[0] = p.x;
  pb.xs[1] = p.y;
  pb.xs[2] = p.z;
  pb.sup = support_of(g, (int)p.w & ((1 << kLabelBits) - 1));
  int bhi[3];
  candidate_blocks(pb.xs, g, pb.sup, pb.blo, bhi);
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    pb.nb[ax] = bhi[ax] - pb.blo[ax] + 1;
    pb.v0[ax] = floor_i(__fmul_rn(pb.xs[ax], g.inv_res));
    float hi, lo;
    centre_offset0(pb.v0[ax], pb.xs[ax], g, hi, lo);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int first = (pb.blo[ax] + k) << g.B_shift;
      const int vn = min(max(pb.v0[ax], first), first + g.B - 1);
      const float e = centre_offset_at(vn - pb.v0[ax], hi, lo, g);
      pb.vn[ax][k] = vn;
      pb.m2[ax][k] = __fmul_rn(e, e);
    }
  }
}

__device__ __forceinline__ double axis_min64_near(int vn, int first, const Geom& g, float x) {
  double best = 1.0e300;
#pragma unroll
  for (int d = -1; d <= 1; ++d) {
    const int v = vn + d;
    if (v < first || v >= first + g.B) continue;
    best = fmin(best, fabs(__dsub_rn(__dmul_rn(__dadd_rn((double)v, 0.5), g.res64), (double)x)));
  }
  return best;
}

// Does candidate block (kx, ky, kz) (indices into the point's ranges) hold a voxel centre within l?
__device__ bool touches(const PointBlocks& pb, int kx, int ky, int kz, const Geom& g) {
  const float d2 = __fadd_rn(__fadd_rn(pb.m2[0][kx], pb.m2[1][ky]), pb.m2[2][kz]);
  if (d2 < pb.sup.l2_lo) return true;
  if (!(d2 < pb.sup.l2_hi)) return false;
  const int k[3] = {kx, ky, kz};
  double s = 0.0;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const double e = axis_min64_near(pb.vn[ax][k[ax]], (pb.blo[ax] + k[ax]) << g.B_shift, g, pb.xs[ax]);
    s = __dadd_rn(s, __dmul_rn(e, e));
  }
  return s < pb.sup.l2_64;
}

// Extended-block association: only the point's own block and its face neighbours.
__device__ __forceinline__ bool allowed(const PointBlocks& pb, int kx, int ky, int kz, const Geom& g) {
  return !g.assoc || face_or_own(pb.blo[0] + kx - (pb.v0[0] >> g.B_shift), pb.blo[1] + ky - (pb.v0[1] >> g.B_shift),
                                 pb.blo[2] + kz - (pb.v0[2] >> g.B_shift));
}

// The number of blocks a CTA's threads marked touched first, added with one
// atomic per CTA (every thread of the CTA calls it, outside divergent code).
__device__ __forceinline__ void add_touched(uint32_t nfirst, DevCounters* dc) {
  __shared__ uint32_t s_first[8];
  const uint32_t w = __reduce_add_sync(0xffffffffu, nfirst);
  if ((threadIdx.x & 31u) == 0) s_first[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_first[k];
    if (t) atomicAdd(&dc->n_touched, t);
  }
}

// Every lane walks the same cube of candidate blocks around the block of its
// point (warp-uniform trip count, at most 3x3x3), so the warp-wide match that
// lets one lane insert a block reached by several lanes always sees all 32
// lanes.  The
// inserting lane also adds the number of lanes that touch the block to its
// point count (used to lay out the per-block point lists).
template <bool kCount>
__global__ void __launch_bounds__(256, 5) touch_kernel(TouchArgs a) {  // 48 registers: five CTAs per SM
  const Geom& g = a.g;
  if (a.dc->err != 0) return;
  const uint32_t P = a.dc->n_train;
  uint32_t nfirst = 0;  // blocks this thread marked touched first
  for (uint32_t base = blockIdx.x * blockDim.x; base < P; base += gridDim.x * blockDim.x) {  // warp-uniform
    const uint32_t i = base + threadIdx.x;
    const bool active = i < P;
    PointBlocks pb;
    int map = 0;
    if (active) {
      const float4 p = a.train[i];
      map = (int)p.w >> kLabelBits;
      point_blocks(p, g, pb);
    } else {
      pb.nb[0] = pb.nb[1] = pb.nb[2] = 0;
      pb.blo[0] = pb.blo[1] = pb.blo[2] = 0;
    }
    // for the fast accumulation form: the point's own block first (it is always
    // touched: the fast form needs l above half the voxel diagonal), then per
    // touched candidate block its hash slot under the own block's digit
    int64_t own = -1;
    if (a.ownslot) {
      const unsigned long long okey =
          active ? pack_block(pb.v0[0] >> g.B_shift, pb.v0[1] >> g.B_shift, pb.v0[2] >> g.B_shift, map) : kEmpty;
      const unsigned opeers = __match_any_sync(0xffffffffu, okey);
      const int oleader = __ffs(opeers) - 1;
      if (active && oleader == (int)(threadIdx.x & 31u)) own = insert_block<kCount>(a, okey, &nfirst);
      own = __shfl_sync(0xffffffffu, own, oleader);
      if (active) a.ownslot[i] = (uint32_t)own;
    }
    // the warp walks the smallest cube of candidate offsets that covers every lane
    const int mx = __reduce_max_sync(0xffffffffu, (unsigned)pb.nb[0]);
    const int my = __reduce_max_sync(0xffffffffu, (unsigned)pb.nb[1]);
    const int mz = __reduce_max_sync(0xffffffffu, (unsigned)pb.nb[2]);
    const int nc = mx * my * mz;
    int kx = 0, ky = 0, kz = 0;  // candidate c = kx + mx (ky + my kz), stepped without divisions
    for (int c = 0; c < nc; ++c, ++kx) {
      if (kx == mx) {
        kx = 0;
        if (++ky == my) {
          ky = 0;
          ++kz;
        }
      }
      const bool hit = kx < pb.nb[0] && ky < pb.nb[1] && kz < pb.nb[2] && allowed(pb, kx, ky, kz, g) &&
                       touches(pb, kx, ky, kz, g);
      const unsigned long long key =
          hit ? pack_block(pb.blo[0] + kx, pb.blo[1] + ky, pb.blo[2] + kz, map) : kEmpty;
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      const int leader = __ffs(peers) - 1;
      int64_t slot = -1;
      if (hit && leader == (int)(threadIdx.x & 31u)) {
        slot = insert_block<kCount>(a, key, &nfirst);
        if (kCount && slot >= 0) atomicAdd(&a.hcnt[slot], (uint32_t)__popc(peers));
      }
      if (a.ownslot) {  // warp-uniform
        slot = __shfl_sync(0xffffffffu, slot, leader);
        // one write per (own block, neighbour): the leader for its own block, other
        // lanes only when their own block differs from the leader's
        const int64_t lown = __shfl_sync(0xffffffffu, own, leader);
        if (hit && own >= 0 && slot >= 0 && (leader == (int)(threadIdx.x & 31u) || own != lown)) {
          const int digit = (pb.blo[0] + kx - (pb.v0[0] >> g.B_shift) + 1) +
                            3 * (pb.blo[1] + ky - (pb.v0[1] >> g.B_shift) + 1) +
                            9 * (pb.blo[2] + kz - (pb.v0[2] >> g.B_shift) + 1);
          a.nbrslot[(size_t)own * 32 + digit] = (uint32_t)slot;
        }
      }
    }
  }
  if (!kCount) add_touched(nfirst, a.dc);
}

// Counting model, Eq. (alpha): the block of the voxel that holds each training
// point (the voxel key floor(x fp32(1/res)) of the read-off).  Consecutive
// training points mostly share a block, so a warp-wide match lets one lane
// per distinct block insert it.
__global__ void __launch_bounds__(256) touch_cells_kernel(TouchArgs a) {
  const Geom& g = a.g;
  if (a.dc->err != 0) return;
  const uint32_t P = a.dc->n_train;
  uint32_t nfirst = 0;
  for (uint32_t base = blockIdx.x * blockDim.x; base < P; base += gridDim.x * blockDim.x) {  // warp-uniform
    const uint32_t i = base + threadIdx.x;
    unsigned long long key = kEmpty;
    if (i < P) {
      const float4 p = a.train[i];
      key = pack_block(floor_i(__fmul_rn(p.x, g.inv_res)) >> g.B_shift, floor_i(__fmul_rn(p.y, g.inv_res)) >> g.B_shift,
                       floor_i(__fmul_rn(p.z, g.inv_res)) >> g.B_shift, (int)p.w >> kLabelBits);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key != kEmpty && (unsigned)(__ffs(peers) - 1) == (threadIdx.x & 31u)) insert_block<false>(a, key, &nfirst);
  }
  add_touched(nfirst, a.dc);
}

// Same walk as touch_kernel: every (point, touched block) pair takes the next
// entry of the block's list.
__global__ void __launch_bounds__(256) bin_fill_kernel(TouchArgs a) {
  const Geom& g = a.g;
  if (a.dc->err != 0) return;
  const uint32_t P = a.dc->n_train;
  for (uint32_t base = blockIdx.x * blockDim.x; base < P; base += gridDim.x * blockDim.x) {  // warp-uniform
    const uint32_t i = base + threadIdx.x;
    const bool active = i < P;
    PointBlocks pb;
    int map = 0;
    if (active) {
      const float4 p = a.train[i];
      map = (int)p.w >> kLabelBits;
      point_blocks(p, g, pb);
    } else {
      pb.nb[0] = pb.nb[1] = pb.nb[2] = 0;
      pb.blo[0] = pb.blo[1] = pb.blo[2] = 0;
    }
    const uint32_t lane_lt = (1u << (threadIdx.x & 31u)) - 1u;
    // the same walk as touch_kernel, so the same blocks
    const int mx = __reduce_max_sync(0xffffffffu, (unsigned)pb.nb[0]);
    const int my = __reduce_max_sync(0xffffffffu, (unsigned)pb.nb[1]);
    const int mz = __reduce_max_sync(0xffffffffu, (unsigned)pb.nb[2]);
    const int nc = mx * my * mz;
    int kx = 0, ky = 0, kz = 0;  // candidate c = kx + mx (ky + my kz), stepped without divisions
    for (int c = 0; c < nc; ++c, ++kx) {
      if (kx == mx) {
        kx = 0;
        if (++ky == my) {
          ky = 0;
          ++kz;
        }
      }
      const bool hit = kx < pb.nb[0] && ky < pb.nb[1] && kz < pb.nb[2] && allowed(pb, kx, ky, kz, g) &&
                       touches(pb, kx, ky, kz, g);
      const unsigned long long key =
          hit ? pack_block(pb.blo[0] + kx, pb.blo[1] + ky, pb.blo[2] + kz, map) : kEmpty;
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      const int leader = __ffs(peers) - 1;
      uint32_t base = 0;
      if (hit && leader == (int)(threadIdx.x & 31u)) {
        const int64_t slot = find_block(a, key);
        base = slot >= 0 ? atomicAdd(&a.hcur[slot], (uint32_t)__popc(peers)) : 0xffffffffu;
      }
      base = __shfl_sync(0xffffffffu, base, leader);
      if (hit && base != 0xffffffffu) a.blist[base + __popc(peers & lane_lt)] = i;
    }
  }
}

// boff[t] = point count of touched block t (beyond n_touched: 0), then scanned
__global__ void bin_counts_kernel(const uint32_t* touched, const uint32_t* hcnt, uint32_t* boff, uint32_t bound,
                                  const DevCounters* dc) {
  const uint32_t nt = dc->n_touched;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < bound; t += gridDim.x * blockDim.x)
    boff[t] = t < nt ? hcnt[touched[t]] : 0u;
}

// cursors from the scanned offsets; counts back to zero for the next update
__global__ void bin_cursor_kernel(const uint32_t* touched, uint32_t* hcnt, uint32_t* hcur, const uint32_t* boff,
                                  int64_t list_cap, DevCounters* dc) {
  const uint32_t nt = dc->n_touched;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    const uint32_t slot = touched[t];
    hcur[slot] = boff[t];
    hcnt[slot] = 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    dc->n_list = boff[nt];
    if ((int64_t)boff[nt] > list_cap) set_error(dc, SBKI_ERR_CAPACITY);
  }
}

// Pool slots for the blocks this update created, or (an error pending, or the
// pool would overflow) their hash slots cleared again.  The last CTA to finish
// (a counter after a fence) then commits the block count.
__global__ void commit_kernel(unsigned long long* hkeys, int32_t* hvals, const uint32_t* fresh,
                              unsigned long long* pool_keys, int64_t pool_blocks, DevCounters* dc) {
  const uint32_t n_new = dc->n_new;
  const uint32_t nb = dc->n_blocks;
  const bool pending = dc->err != 0;
  const bool overflow = (unsigned long long)nb + n_new > (unsigned long long)pool_blocks;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_new; i += gridDim.x * blockDim.x) {
    const uint32_t slot = fresh[i];
    if (pending || overflow) {
      hkeys[slot] = kEmpty;  // roll back: the map keeps its previous block set
    } else {
      const uint32_t pool = nb + i;
      hvals[slot] = (int32_t)pool;
      pool_keys[pool] = hkeys[slot];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&dc->commit_done, 1u) == gridDim.x - 1) {  // every CTA has read n_blocks
      dc->commit_done = 0u;
      dc->n_blocks_before = nb;
      if (pending) return;
      if (overflow) {
        set_error(dc, SBKI_ERR_CAPACITY);
        return;
      }
      dc->n_blocks = nb + n_new;
    }
  }
}

// Restoring exported contents: the blocks of the given voxel keys (warp-deduplicated
// inserts, like touch_kernel), then the voxels' increments alpha - alpha0.
__global__ void __launch_bounds__(256) import_blocks_kernel(TouchArgs a, const int64_t* __restrict__ keys,
                                                            int64_t count, int map) {
  const Geom& g = a.g;
  if (a.dc->err != 0) return;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < count; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = base + threadIdx.x;
    unsigned long long key = kEmpty;
    if (q < count) {
      const int64_t kx = keys[3 * q], ky = keys[3 * q + 1], kz = keys[3 * q + 2];
      if (kx <= -kKeyLimit || kx >= kKeyLimit || ky <= -kKeyLimit || ky >= kKeyLimit || kz <= -kKeyLimit ||
          kz >= kKeyLimit)
        set_error(a.dc, SBKI_ERR_INVALID_ARG);
      else
        key = pack_block((int32_t)(kx >> g.B_shift), (int32_t)(ky >> g.B_shift), (int32_t)(kz >> g.B_shift), map);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key != kEmpty && (unsigned)(__ffs(peers) - 1) == (threadIdx.x & 31u)) insert_block(a, key);
  }
}

__global__ void __launch_bounds__(256) import_alpha_kernel(Geom g, const unsigned long long* __restrict__ hkeys,
                                                           const int32_t* __restrict__ hvals, int64_t hash_cap,
                                                           const int64_t* __restrict__ keys,
                                                           const float* __restrict__ alpha, int64_t count, int map,
                                                           float alpha0, float* __restrict__ pool,
                                                           DevCounters* dc) {
  if (dc->err != 0) return;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t kx = keys[3 * q], ky = keys[3 * q + 1], kz = keys[3 * q + 2];
    const unsigned long long bkey =
        pack_block((int32_t)(kx >> g.B_shift), (int32_t)(ky >> g.B_shift), (int32_t)(kz >> g.B_shift), map);
    uint32_t slot = hash_slot(bkey, hash_cap);
    int32_t pl = -1;
    for (int probe = 0; probe < kMaxProbes; ++probe) {
      const unsigned long long k = hkeys[slot];
      if (k == bkey) {
        pl = hvals[slot];
        break;
      }
      if (k == kEmpty) break;
      slot = (uint32_t)((slot + 1) & (uint32_t)(hash_cap - 1));
    }
    if (pl < 0) continue;
    const int m = g.B - 1;
    const int local = ((((int)kz & m) << g.B_shift) + ((int)ky & m)) * g.B + ((int)kx & m);
    float* dst = pool + (size_t)pl * g.K1 * g.B3 + local;
    for (int k = 0; k < g.K1; ++k) dst[(size_t)k * g.B3] = __fsub_rn(alpha[q * g.K1 + k], alpha0);
  }
}

TouchArgs touch_args(MapState& m) {
  TouchArgs a;
  a.g = m.g;
  a.train = m.s.train;
  a.hkeys = m.hkeys;
  a.hvals = m.hvals;
  a.hmark = m.hmark;
  a.hash_cap = m.hash_cap;
  a.touched = m.s.touched;
  a.fresh = m.s.fresh;
  a.hcnt = m.hcnt;
  a.hcur = m.hcur;
  a.blist = m.blist;
  a.ownslot = nullptr;
  a.nbrslot = nullptr;
  a.dc = m.dc;
  return a;
}

}  // namespace

cudaError_t launch_touch_cells(MapState& m, int64_t bound) {
  const TouchArgs a = touch_args(m);
  const int64_t blocks =
      std::max<int64_t>(1, std::min<int64_t>((bound + 255) / 256, (int64_t)m.sm_count * m.tune.touch_ctas_per_sm));
  touch_cells_kernel<<<(unsigned)blocks, 256, 0, m.stream>>>(a);
  m.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_touch_blocks(MapState& m, const KeyFrame& /*kf*/, int64_t bound) {
  TouchArgs a = touch_args(m);
  if (m.acc_mode == 0 && fast_form_ready(m)) {  // tables of the fast point-major accumulation
    a.ownslot = m.s.ownslot;
    a.nbrslot = m.nbrslot;
  }
  // bound: the training points never exceed the items of the update
  const int64_t blocks =
      std::max<int64_t>(1, std::min<int64_t>((bound + 255) / 256, (int64_t)m.sm_count * m.tune.touch_ctas_per_sm));
  if (m.acc_mode == 1) touch_kernel<true><<<(unsigned)blocks, 256, 0, m.stream>>>(a);  // counts for the block lists
  else touch_kernel<false><<<(unsigned)blocks, 256, 0, m.stream>>>(a);
  m.launches += 1;
  return cudaGetLastError();
}

// After commit: per touched block the list of training points that touch it.
cudaError_t launch_bin_points(MapState& m, int64_t bound) {
  const TouchArgs a = touch_args(m);
  // touched blocks never exceed 27 per training point nor the hash size
  const int64_t tb = std::min<int64_t>(m.hash_cap, 27 * std::max<int64_t>(bound, 1));
  bin_counts_kernel<<<(unsigned)std::min<int64_t>((tb + 255) / 256, 4096), 256, 0, m.stream>>>(
      m.s.touched, m.hcnt, m.boff, (uint32_t)tb, m.dc);
  cudaError_t e = exclusive_scan_u32(m.boff, tb, m.s.scan_tmp, m.stream);
  if (e != cudaSuccess) return e;
  bin_cursor_kernel<<<m.sm_count * 4, 256, 0, m.stream>>>(m.s.touched, m.hcnt, m.hcur, m.boff, m.list_cap, m.dc);
  const int64_t blocks =
      std::max<int64_t>(1, std::min<int64_t>((bound + 255) / 256, (int64_t)m.sm_count * m.tune.touch_ctas_per_sm));
  bin_fill_kernel<<<(unsigned)blocks, 256, 0, m.stream>>>(a);
  m.launches += 1 + 3 + 1 + 1;
  return cudaGetLastError();
}

cudaError_t launch_import(MapState& m, const int64_t* keys, const float* alpha, int64_t count) {
  TouchArgs a = touch_args(m);
  a.train = nullptr;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, (int64_t)m.sm_count * 8));
  import_blocks_kernel<<<blocks, 256, 0, m.stream>>>(a, keys, count, m.active_map);
  cudaError_t e = launch_commit_blocks(m);
  if (e != cudaSuccess) return e;
  e = launch_fresh_fill(m);
  if (e != cudaSuccess) return e;
  import_alpha_kernel<<<blocks, 256, 0, m.stream>>>(m.g, m.hkeys, m.hvals, m.hash_cap, keys, alpha, count,
                                                    m.active_map, (float)m.prm.alpha0, m.alpha, m.dc);
  m.launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_commit_blocks(MapState& m) {
  commit_kernel<<<m.sm_count * 2, 256, 0, m.stream>>>(m.hkeys, m.hvals, m.s.fresh, m.pool_keys, m.pool_blocks, m.dc);
  m.launches += 1;
  return cudaGetLastError();
}

}  // namespace sbki
