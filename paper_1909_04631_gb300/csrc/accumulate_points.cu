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
#include <type_traits>
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
constexpr int kFastParts = 16;           // fast form: sub-voxel parts per axis of its candidate lists

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
  int chunk;             // consecutive training points per warp (fast form)
  int32_t sink;          // spare pool block that absent neighbour blocks point at
  const uint32_t* ftab;  // fast form: [kFastParts^3][ftpad] (X | Y << 8 | Z << 16 row byte offsets in a slot)
  const int32_t* flen;   // [kFastParts^3] entries of each list
  int ftpad;             // entries per fast list (multiple of 32, at most 32 kFastEntries)
  const uint32_t* ownslot;  // fast form: per training point the hash slot of its own block (touched-block pass)
  const uint32_t* nbrslot;  // fast form: [hash_cap][32] per own block the hash slots of its touched neighbours
  const int32_t* softidx;   // soft labels (fast form), or null: per training point its weight row, or -1
  const float* wsoft;       // weight rows [.][K+1]
  int tab_of[kMaxClasses];  // per-class supports (fast form): each class's list table, or -1 (not this form)
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
  if (g.assoc) in = in && ((kFaceDigits >> (pk & 0xff)) & 1u);  // extended block: own block and face neighbours
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

// The same update for 2R + 1 <= 7 (l up to about 3 voxels), shaped for the
// instruction issue rate, which bounds this loop.
//
// A warp takes a chunk of consecutive training points (sorted by tile, so
// mostly one block) from a work queue and forms their rows in groups of up to
// kGroup: three lanes per point (one per axis) write, for offsets j = 0..2R of
// their axis, the row (e_j^2, address part) into the point's 256-byte slot in
// shared memory (X rows at bytes 0..63, Y rows at 64..127, Z rows at 128..191,
// the point's scalars at 192..255).  An address part holds the block digit of
// the offset (base 3 per axis, times 4: a byte offset into the block table) in
// its top byte and the voxel's in-block index below it (the X part also
// carries the point's class row, label * B^3), so the three parts of a
// candidate add up to (4 digit) << 24 | (label B^3 + in-block index).
//
// A candidate list entry holds the byte offsets of the candidate's X, Y and Z
// rows inside a slot (bytes 0, 1, 2), so with the slot at a 256-byte aligned
// shared address each row address is one byte permute.  Each lane takes two
// entries at a time and evaluates their kernels with packed FP32 instructions
// (two values per instruction).  The block table holds, per digit, the first
// alpha element of the block (the pool slot times (K+1) B^3) minus the digit's
// top byte, so table entry + summed address parts is the alpha element: one
// shared load and one add per candidate.  Tables change only when the point's
// block (or map) changes.  Lists come from a table with kFastParts^3 sub-voxel
// parts; the next point's entries are loaded while the current one is swept.
constexpr int kGroup = 10;         // points whose rows one warp forms at once (3 lanes each)
constexpr int kFastAxis = 8;       // rows per axis: 2R + 1 <= 7 offsets and the X padding row
constexpr int kSlotBytes = 256;    // one point's rows and scalars
constexpr int kFastEntries = 5;    // list entries per lane (lists of at most 160)
constexpr uint32_t kPadEntry = 8u * (kFastAxis - 1) | (64u << 8) | (128u << 16);  // X padding row, Y row 0, Z row 0

struct __align__(256) FastWarp {
  float2 rows[kGroup][kSlotBytes / 8];  // per point: X, Y, Z rows (8 each), scalars (int view, below)
  uint32_t btab[64];                    // alpha element base per block digit (27 used)
  uint32_t ptab[64];                    // pair-count element base per block digit (kTrack)
};
struct __align__(256) FastWarpSoft : FastWarp {
  float cw[kGroup][kMaxClasses];        // soft labels: per point sigma0 s_k w^k by class
};
// scalars of a slot (int index into its last 64 bytes)
constexpr int kScPart = 0, kScLabel = 1, kScS0 = 2, kScPool = 3, kScMask = 4, kScSoft = 5, kScV0 = 8;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ float2 lds_f2(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// d^2 and summed address part of a candidate of the point whose slot starts at `slot`
__device__ __forceinline__ void candidate_rows2(uint32_t e, uint32_t slot, float& d2, uint32_t& pk) {
  const float2 rx = lds_f2(__byte_perm(e, slot, 0x7650));
  const float2 ry = lds_f2(__byte_perm(e, slot, 0x7651));
  const float2 rz = lds_f2(__byte_perm(e, slot, 0x7652));
  d2 = __fadd_rn(__fadd_rn(rx.x, ry.x), rz.x);
  pk = __float_as_uint(rx.y) + __float_as_uint(ry.y) + __float_as_uint(rz.y);
}

// FP64 re-decision of a candidate in the band around l^2 (rare; point loaded again)
__device__ __forceinline__ bool band_decide(uint32_t e, const int* sc, const float4* train, uint32_t i, int R,
                                         double res64, double l2_64) {
  const float4 p = train[i];
  const int jx = (int)((e & 0xffu) >> 3), jy = (int)(((e >> 8) & 0xffu) - 64u) >> 3,
            jz = (int)(((e >> 16) & 0xffu) - 128u) >> 3;
  return in_support64_call(sc[kScV0] + jx - R, sc[kScV0 + 1] + jy - R, sc[kScV0 + 2] + jz - R, p.x, p.y, p.z, res64,
                           l2_64);
}

// Soft labels (kSoft, reading K15): a point with a weight row forms its rows
// for class 0 (no class row in the X parts) with s0 = 1, and each of its
// in-support pairs adds f(d/l) sigma0 s_k w^k into every class k with a
// nonzero weight; a point without one (free samples) is a hard class-0 point.
// Per-class supports (kLk, reading K16): a point's list comes from the table
// of its class's support l_k, its membership test and kernel use l_k; points
// of a class without a table are left to the weighted form.
template <bool kTrack, bool kFace, bool kSoft = false, bool kLk = false>
__global__ void __launch_bounds__(kThreads, 4) accumulate_points_fast_kernel(PtArgs a) {
  using Warp = typename std::conditional<kSoft, FastWarpSoft, FastWarp>::type;
  __shared__ Warp s_w[kWarps];
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Warp& W = s_w[wid];
  const int R = a.R, na = 2 * R + 1, m = g.B - 1;
  if (a.dc->err != 0) return;
  if ((smem_addr(&W) & 255u) != 0u) {  // the byte permutes need 256-byte aligned slots
    if (lane == 0) set_error(a.dc, SBKI_ERR_CUDA);
    return;
  }
  const uint32_t P = a.dc->n_train;
  const uint32_t rows0 = smem_addr(&W.rows[0][0]);
  const uint32_t btab = smem_addr(&W.btab[0]), ptab = smem_addr(&W.ptab[0]);
  // this lane's point of a group and axis (lanes 30, 31 form no rows)
  const int gl = lane / 3, ax = lane - 3 * gl;
  const int axshift = ax == 0 ? 0 : (ax == 1 ? g.B_shift : 2 * g.B_shift);
  const uint32_t dmul = ax == 0 ? 4u : (ax == 1 ? 12u : 36u);
  const uint32_t K1B3 = (uint32_t)(g.K1 * g.B3);
  const float2 neg_inv_l = make_float2(-g.inv_l, -g.inv_l), one2 = make_float2(1.0f, 1.0f);
  int cpool = -1;  // own-block pool slot the tables belong to
  uint32_t npairs = 0;
  const uint32_t chunk = (uint32_t)a.chunk;
  uint32_t c = 0;
  if (lane == 0) c = atomicAdd(&a.dc->acc_next, 1u);
  c = __shfl_sync(0xffffffffu, c, 0);
  while (c * chunk < P) {
    uint32_t cn = 0;  // next chunk, fetched while this one is processed
    if (lane == 0) cn = atomicAdd(&a.dc->acc_next, 1u);
    const uint32_t c1 = min(P, c * chunk + chunk);
    for (uint32_t g0 = c * chunk; g0 < c1; g0 += kGroup) {
      const uint32_t gn = min(c1 - g0, (uint32_t)kGroup);  // warp-uniform
      // 1. rows of every point of the group, three lanes per point; the lane
      //    of axis x also reads the hash slot of the point's own block
      int pt = 0, lw = 0, srow = -1;
      if (gl < (int)gn) {
        const float4 p = a.train[g0 + gl];
        if (kSoft) srow = __ldg(a.softidx + g0 + gl);
        const float xa = ax == 0 ? p.x : (ax == 1 ? p.y : p.z);
        const int v0 = floor_small(__fmul_rn(xa, g.inv_res));
        float hi, lo;
        centre_offset0(v0, xa, g, hi, lo);
        const float phi = 0.5f - __fmul_rn(__fadd_rn(hi, lo), g.inv_res);
        pt = min(kFastParts - 1, max(0, floor_small(phi * (float)kFastParts)));
        const int b0 = v0 >> g.B_shift;
        lw = label_of(p.w);
        if (kSoft && srow >= 0) lw &= ~((1 << kLabelBits) - 1);  // class rows come per class in the sweep
        const uint32_t cls = ax == 0 ? (uint32_t)((lw & ((1 << kLabelBits) - 1)) * g.B3) : 0u;
        float2* r = W.rows[gl] + kFastAxis * ax;
        // offsets in a lane-dependent order, so the lanes of one store spread over the banks
        int j = (gl + 2 * ax) % na;
#pragma unroll
        for (int t = 0; t < kFastAxis - 1; ++t) {
          if (t < na) {
            const float e = centre_offset_at(j - R, hi, lo, g);
            const int v = v0 + j - R;
            const uint32_t part = (dmul * (uint32_t)((v >> g.B_shift) - b0 + 1)) << 24 | (((uint32_t)(v & m) << axshift) + cls);
            r[j] = make_float2(__fmul_rn(e, e), __uint_as_float(part));
            j = j + 1 == na ? 0 : j + 1;
          }
        }
        if (ax == 0) r[kFastAxis - 1] = make_float2(kFar, 0.0f);
        reinterpret_cast<int*>(W.rows[gl] + 3 * kFastAxis)[kScV0 + ax] = v0;
      }
      const int pty = __shfl_sync(0xffffffffu, pt, min(lane + 1, 31));
      const int ptz = __shfl_sync(0xffffffffu, pt, min(lane + 2, 31));
      int list = pt + kFastParts * (pty + kFastParts * ptz);
      if constexpr (kLk) {  // the table of the point's class support, or -1
        const int tb = a.tab_of[lw & ((1 << kLabelBits) - 1)];
        list = tb >= 0 ? list + tb * kFastParts * kFastParts * kFastParts : -1;
      }
      if (ax == 0 && gl < (int)gn)
        *reinterpret_cast<int4*>(reinterpret_cast<int*>(W.rows[gl] + 3 * kFastAxis) + kScPart) =
            make_int4(list, lw,
                      __float_as_int((kSoft && srow >= 0) ? 1.0f : g.sigma0_k[lw & ((1 << kLabelBits) - 1)]),
                      (int)__ldg(a.ownslot + g0 + gl));
      if constexpr (kSoft) {  // class factors sigma0 s_k w^k of the group's soft points
        for (uint32_t k = 0; k < gn; ++k) {
          const int row = __shfl_sync(0xffffffffu, srow, 3 * k);
          float ck = 0.0f;
          if (row >= 0 && lane < g.K1) ck = g.sigma0_k[lane] * __ldg(a.wsoft + (size_t)row * g.K1 + lane);
          const unsigned cm = __ballot_sync(0xffffffffu, ck != 0.0f);
          if (lane < g.K1) W.cw[k][lane] = ck;
          if (lane == 0) {
            int* sc = reinterpret_cast<int*>(W.rows[k] + 3 * kFastAxis);
            sc[kScMask] = (int)cm;
            sc[kScSoft] = row >= 0 ? 1 : 0;
          }
        }
      }
      __syncwarp();
      // 2. point by point: block tables (when the own block changes), candidate sweeps
      uint32_t ent[kFastEntries];
      {
        int part = reinterpret_cast<const int*>(W.rows[0] + 3 * kFastAxis)[kScPart];
        if constexpr (kLk) part = max(0, part);  // a skipped point (-1) loads list 0, unused
        const uint32_t* tab = a.ftab + (size_t)part * a.ftpad;
#pragma unroll
        for (int it = 0; it < kFastEntries; ++it) ent[it] = __ldg(tab + it * 32 + lane);
      }
      for (uint32_t k = 0; k < gn; ++k) {
        const int* sc = reinterpret_cast<const int*>(W.rows[k] + 3 * kFastAxis);
        const int4 sv = *reinterpret_cast<const int4*>(sc + kScPart);  // part, label word, s0, own pool slot
        const bool soft_pt = kSoft && sc[kScSoft] != 0;
        const unsigned cmask = kSoft ? (unsigned)sc[kScMask] : 0u;
        // the next point's list, in flight while this one is swept (lists are
        // padded to kFastEntries x 32 entries, so every load is in range)
        uint32_t nent[kFastEntries];
        {
          int part = k + 1 < gn ? sc[kScPart + kSlotBytes / 4] : sv.x;
          if constexpr (kLk) part = max(0, part);
          const uint32_t* tab = a.ftab + (size_t)part * a.ftpad;
#pragma unroll
          for (int it = 0; it < kFastEntries; ++it) nent[it] = __ldg(tab + it * 32 + lane);
        }
        if (!(kLk && sv.x < 0)) {  // warp-uniform: a point of a class without a table is the weighted form's
          if (sv.w != cpool) {  // warp-uniform: the tables belong to another block
            cpool = sv.w;
            __syncwarp();  // every lane is done with the old tables
            if (lane < 27) {
              // a digit no point of this block touched holds a stale slot; no
              // in-support pair uses it (every reduction is predicated on membership)
              const uint32_t hs = a.nbrslot[(size_t)sv.w * 32 + lane] & (uint32_t)(a.hash_cap - 1);
              const int32_t pool = a.hvals[hs];
              const uint32_t pb = (uint32_t)(pool >= 0 ? pool : a.sink);
              W.btab[lane] = pb * K1B3 - ((4u * (uint32_t)lane) << 24);
              if (kTrack) W.ptab[lane] = pb * (uint32_t)g.B3 - ((4u * (uint32_t)lane) << 24);
            }
            __syncwarp();
          }
          const uint32_t slot = rows0 + (uint32_t)k * kSlotBytes;
          const float s0 = __int_as_float(sv.z);
          const float2 s02 = make_float2(s0, s0);
          const uint32_t cls = (uint32_t)((sv.y & ((1 << kLabelBits) - 1)) * g.B3);
          const int len = __ldg(a.flen + sv.x);
          // the support of the point's class (common l: the kernel's constants)
          const int cl = sv.y & ((1 << kLabelBits) - 1);
          const float l2lo = kLk ? g.l2k_lo[cl] : g.l2_lo, l2hi = kLk ? g.l2k_hi[cl] : g.l2_hi;
          const double l264 = kLk ? g.l2k_64[cl] : g.l2_64;
          const float2 ninv = kLk ? make_float2(-g.inv_lk[cl], -g.inv_lk[cl]) : neg_inv_l;
#pragma unroll
          for (int jp = 0; jp < (kFastEntries + 1) / 2; ++jp) {
            if (jp < 2 || jp * 64 < len) {  // warp-uniform; lists hold more than 64 entries
              const uint32_t ea = ent[2 * jp], eb = 2 * jp + 1 < kFastEntries ? ent[2 * jp + 1] : kPadEntry;
              float d2a, d2b;
              uint32_t pka, pkb;
              candidate_rows2(ea, slot, d2a, pka);
              candidate_rows2(eb, slot, d2b, pkb);
              bool ina = d2a < l2lo, inb = d2b < l2lo;
              const bool bnda = !ina && d2a < l2hi, bndb = !inb && d2b < l2hi;
              if (__any_sync(0xffffffffu, bnda || bndb)) {
                if (bnda) ina = band_decide(ea, sc, a.train, g0 + k, R, g.res64, l264);
                if (bndb) inb = band_decide(eb, sc, a.train, g0 + k, R, g.res64, l264);
              }
              if (kFace) {  // extended block: own block and face neighbours (digit in the top byte, times 4)
                ina = ina && ((kFaceDigits >> (pka >> 26)) & 1u);
                inb = inb && ((kFaceDigits >> (pkb >> 26)) & 1u);
              }
              // kernel of both candidates: f = u^5 Q(u^2), u = 1 - d / l, times sigma0 s_k
              const float2 d = make_float2(sqrt_approx(d2a), sqrt_approx(d2b));
              const float2 u = __ffma2_rn(d, ninv, one2);
              const float2 w = __fmul2_rn(u, u);
              const float2 q = kernel_q2(w);
              const float2 v = __fmul2_rn(__fmul2_rn(__fmul2_rn(__fmul2_rn(w, w), u), q), s02);
              const uint32_t elema = lds_u32(__byte_perm(pka, btab, 0x7653)) + pka;
              const uint32_t elemb = lds_u32(__byte_perm(pkb, btab, 0x7653)) + pkb;
              bool spread = false;
              if constexpr (kSoft) {
                if (soft_pt) {  // warp-uniform: every class with a weight
                  for (unsigned cl = cmask; cl; cl &= cl - 1u) {
                    const int kc = __ffs((int)cl) - 1;
                    const float ck = W.cw[k][kc];
                    const uint32_t off = (uint32_t)kc * (uint32_t)g.B3;
                    if (ina) atomicAdd(a.alpha + elema + off, v.x * ck);
                    if (inb) atomicAdd(a.alpha + elemb + off, v.y * ck);
                  }
                  spread = true;
                }
              }
              if (!spread) {
                if (ina) atomicAdd(a.alpha + elema, v.x);  // result unused: a reduction
                if (inb) atomicAdd(a.alpha + elemb, v.y);
              }
              if (kTrack) {
                red_add_if(ina, a.pairs + (lds_u32(__byte_perm(pka, ptab, 0x7653)) + pka - cls), 1);
                red_add_if(inb, a.pairs + (lds_u32(__byte_perm(pkb, ptab, 0x7653)) + pkb - cls), 1);
              }
              npairs += (ina ? 1u : 0u) + (inb ? 1u : 0u);
            }
          }
        }
#pragma unroll
        for (int it = 0; it < kFastEntries; ++it) ent[it] = nent[it];
      }
      __syncwarp();  // the slots are rewritten by the next group
    }
    c = __shfl_sync(0xffffffffu, cn, 0);
  }
  for (int o = 16; o > 0; o >>= 1) npairs += __shfl_down_sync(0xffffffffu, npairs, o);
  if (lane == 0) atomicAdd(&a.dc->pairs, (unsigned long long)npairs);
}

// Blocks created by this update start at zero (and so do their pair counts).
__global__ void fresh_fill_kernel(const uint32_t* fresh, const int32_t* hvals, float* alpha, int32_t* pairs, int K1B3,
                                  int B3, DevCounters* dc) {
  if (dc->err != 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) dc->acc_next = 0;  // work queue of the accumulation launched next
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

// Candidate offsets of each of parts^3 sub-voxel parts: every (dx, dy, dz) whose
// voxel centre can lie within l of some position in the part, the part widened
// by delta = 1e-3 voxel on every side (far above the FP32 error of the sub-voxel
// position, ~1e-6 voxel), so a point's list always holds its ball.  Offsets are
// packed as (dx + R) | (dy + R) << 4 | (dz + R) << 8; returns R.
int candidate_lists(double lr, int parts, std::vector<std::vector<int32_t>>& lists) {
  const double delta = 1e-3;
  const int R = (int)std::ceil(lr + 0.5 + delta);
  const int n = parts * parts * parts;
  lists.assign(n, {});
  for (int t = 0; t < n; ++t) {
    const int pt[3] = {t % parts, (t / parts) % parts, t / (parts * parts)};
    for (int dz = -R; dz <= R; ++dz)
      for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx) {
          const int d[3] = {dx, dy, dz};
          double m2 = 0.0;
          for (int a = 0; a < 3; ++a) {
            const double md =
                min_axis_distance(d[a], (double)pt[a] / parts - delta, (double)(pt[a] + 1) / parts + delta);
            m2 += md * md;
          }
          if (m2 < lr * lr * (1.0 + 1e-5)) lists[t].push_back((dx + R) | ((dy + R) << 4) | ((dz + R) << 8));
        }
  }
  return R;
}

cudaError_t upload_lists(const std::vector<uint32_t>& flat, const std::vector<int32_t>& len, uint32_t** tab,
                         int32_t** lens) {
  cudaError_t e = cudaMalloc(tab, sizeof(uint32_t) * flat.size());
  if (e != cudaSuccess) return e;
  e = cudaMalloc(lens, sizeof(int32_t) * len.size());
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(*lens, len.data(), sizeof(int32_t) * len.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*tab, flat.data(), sizeof(uint32_t) * flat.size(), cudaMemcpyHostToDevice);
}

}  // namespace

// Candidate lists (host, once per map): kParts^3 lists in the general form and,
// when 2R + 1 <= 7, kFastParts^3 lists in the fast form's entry format.
cudaError_t build_candidate_tables(MapState& m) {
  const double lr = m.prm.length_scale / m.prm.res;
  std::vector<std::vector<int32_t>> lists;
  const int R = candidate_lists(lr, kParts, lists);
  const int kLists = (int)lists.size();
  size_t longest = 0;
  int maxd = 0;  // offsets actually used
  for (auto& L : lists) {
    longest = std::max(longest, L.size());
    for (int32_t e : L)
      for (int a = 0; a < 3; ++a) maxd = std::max(maxd, std::abs(((e >> (4 * a)) & 15) - R));
  }
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
  cudaError_t e = upload_lists(flat, len, &m.ctab, &m.clen);
  if (e != cudaSuccess) return e;
  m.ctab_pad = tpad;
  m.ctab_R = Rt;
  // The fast form: one table of kFastParts^3 lists per distinct class support
  // l_k = l l_scale[k] (one table for the common l).  A support qualifies with
  // 2R + 1 <= 7 offsets per axis and l_k above half the voxel diagonal (a
  // point's own voxel, hence its own block, is then always touched); every
  // list is padded to 32 kFastEntries entries (the sweep loads all of them
  // unconditionally).  Entry = X row byte offset 8 jx | (64 + 8 jy) << 8 |
  // (128 + 8 jz) << 16 inside a point's slot; padding entries name the X
  // padding row.
  const int K1 = m.prm.num_classes + 1;
  const int fpad = 32 * kFastEntries;
  std::vector<double> lrs;                              // distinct supports (voxel units)
  std::vector<std::vector<std::vector<int32_t>>> tabs;  // their lists
  std::vector<int> rfs;                                 // candidate_lists' R of each
  int rmax = 0;
  bool own_touched = true;
  m.ftab_classes = 0;
  for (int k = 0; k < 32; ++k) m.ftab_of[k] = -1;
  for (int k = 0; k < K1; ++k) {
    const double lrk = m.prm.length_scale * m.prm.l_scale[k] / m.prm.res;
    own_touched = own_touched && lrk > 0.8661;
    size_t t = 0;
    while (t < lrs.size() && lrs[t] != lrk) ++t;
    if (t == lrs.size()) {  // a new support: its lists, if it qualifies
      std::vector<std::vector<int32_t>> fl;
      const int Rf = candidate_lists(lrk, kFastParts, fl);
      size_t lng = 0;
      int md = 0;
      for (auto& L : fl) {
        lng = std::max(lng, L.size());
        for (int32_t e : L)
          for (int a2 = 0; a2 < 3; ++a2) md = std::max(md, std::abs(((e >> (4 * a2)) & 15) - Rf));
      }
      if (2 * md + 1 > kFastAxis - 1 || lrk <= 0.8661 || (int)lng > fpad) {
        lrs.push_back(lrk);
        tabs.emplace_back();  // does not qualify
        rfs.push_back(-1);
      } else {
        lrs.push_back(lrk);
        tabs.push_back(std::move(fl));
        rfs.push_back(Rf);
        rmax = std::max(rmax, md);
      }
    }
    if (rfs[t] >= 0) m.ftab_classes |= 1u << k;
  }
  if (m.ftab_classes == 0) return cudaSuccess;
  // tables in order of first use; rows -rmax..rmax for all of them
  const int nf = kFastParts * kFastParts * kFastParts, naf = 2 * rmax + 1;
  std::vector<int> index(lrs.size(), -1);
  int ntab = 0;
  for (size_t t = 0; t < lrs.size(); ++t)
    if (rfs[t] >= 0) index[t] = ntab++;
  std::vector<uint32_t> ff((size_t)ntab * nf * fpad, kPadEntry);
  std::vector<int32_t> fl((size_t)ntab * nf);
  for (size_t t = 0; t < lrs.size(); ++t) {
    if (index[t] < 0) continue;
    const size_t b = (size_t)index[t] * nf;
    for (int q = 0; q < nf; ++q) {
      const auto& L = tabs[t][q];
      fl[b + q] = (int32_t)L.size();
      for (size_t k = 0; k < L.size(); ++k) {
        const int32_t e = L[k];
        const uint32_t jx = (uint32_t)((e & 15) - rfs[t] + rmax), jy = (uint32_t)(((e >> 4) & 15) - rfs[t] + rmax),
                       jz = (uint32_t)(((e >> 8) & 15) - rfs[t] + rmax);
        if (jx >= (uint32_t)naf || jy >= (uint32_t)naf || jz >= (uint32_t)naf) return cudaErrorInvalidValue;
        ff[(b + q) * fpad + k] = (8u * jx) | ((64u + 8u * jy) << 8) | ((128u + 8u * jz) << 16);
      }
    }
  }
  for (int k = 0; k < K1; ++k) {
    size_t t = 0;
    const double lrk = m.prm.length_scale * m.prm.l_scale[k] / m.prm.res;
    while (lrs[t] != lrk) ++t;
    m.ftab_of[k] = index[t];
  }
  e = upload_lists(ff, fl, &m.ftab, &m.flen);
  if (e != cudaSuccess) return e;
  m.ftab_pad = fpad;
  m.ftab_R = rmax;
  m.ftab_own_touched = own_touched;
  return cudaSuccess;
}

namespace {

// ctas_per_sm: 0 = as many as fit
template <typename Kernel>
cudaError_t launch_persistent(Kernel kern, const PtArgs& a, int sm_count, int ctas_per_sm, cudaStream_t st) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
  if (e != cudaSuccess) return e;
  if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
  kern<<<std::max(1, per_sm) * sm_count, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <bool kTrack>
cudaError_t launch_fast(const PtArgs& a, int sm_count, int ctas_per_sm, cudaStream_t st) {
  if (a.g.lscaled)  // per-class supports: the exact association and hard labels only
    return launch_persistent(accumulate_points_fast_kernel<kTrack, false, false, true>, a, sm_count, ctas_per_sm,
                             st);
  if (a.softidx)  // soft labels take the exact association only
    return launch_persistent(accumulate_points_fast_kernel<kTrack, false, true>, a, sm_count, ctas_per_sm, st);
  return a.g.assoc ? launch_persistent(accumulate_points_fast_kernel<kTrack, true>, a, sm_count, ctas_per_sm, st)
                   : launch_persistent(accumulate_points_fast_kernel<kTrack, false>, a, sm_count, ctas_per_sm, st);
}

template <bool kTrack>
cudaError_t launch_general(const PtArgs& a, int sm_count, int ctas_per_sm, cudaStream_t st) {
  switch (a.tpad / 32) {  // unrolled sweeps for the common list lengths
    case 2: return launch_persistent(accumulate_points_kernel<kTrack, 2>, a, sm_count, ctas_per_sm, st);
    case 3: return launch_persistent(accumulate_points_kernel<kTrack, 3>, a, sm_count, ctas_per_sm, st);
    case 4: return launch_persistent(accumulate_points_kernel<kTrack, 4>, a, sm_count, ctas_per_sm, st);
    case 5: return launch_persistent(accumulate_points_kernel<kTrack, 5>, a, sm_count, ctas_per_sm, st);
    case 6: return launch_persistent(accumulate_points_kernel<kTrack, 6>, a, sm_count, ctas_per_sm, st);
    default: return launch_persistent(accumulate_points_kernel<kTrack, 0>, a, sm_count, ctas_per_sm, st);
  }
}

}  // namespace

cudaError_t launch_fresh_fill(MapState& m) {
  fresh_fill_kernel<<<m.sm_count * 4, 256, 0, m.stream>>>(m.s.fresh, m.hvals, m.alpha, m.pairs, m.g.K1 * m.g.B3,
                                                          m.g.B3, m.dc);
  m.launches += 1;
  return cudaGetLastError();
}

// the fast form needs its tables (with per-class supports, every class's l_k
// above half the voxel diagonal, so that the touched-block pass may record
// every point's own block) and addresses alpha and the pair counts with
// 32-bit element indices
bool fast_form_ready(const MapState& m) {
  return m.ftab != nullptr && m.nbrslot != nullptr && (!m.g.lscaled || m.ftab_own_touched) &&
         (uint64_t)(m.pool_blocks + 1) * (uint64_t)(m.g.K1 * m.g.B3) <= (1ull << 32);
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
  // soft labels: a point with a weight row costs up to K+1 times the reductions, so smaller
  // chunks balance the work queue better (20 against 30: 0.53 against 0.60 ms per street scan)
  if (m.soft) a.chunk = std::min(a.chunk, 20);
  a.sink = (int32_t)m.pool_blocks;
  a.ftab = m.ftab;
  a.flen = m.flen;
  a.ftpad = m.ftab_pad;
  a.ownslot = m.s.ownslot;
  a.nbrslot = m.nbrslot;
  a.softidx = m.soft ? m.s.softidx : nullptr;
  a.wsoft = m.soft ? m.s.wsoft : nullptr;
  for (int k = 0; k < kMaxClasses; ++k) a.tab_of[k] = m.ftab_of[k];
  a.dc = m.dc;
  m.launches += 2;
  const int cps = m.tune.accumulate_ctas_per_sm;
  const bool fast = fast_form_ready(m);
  // soft labels and per-class supports without the fast form: the caller takes the weighted form instead
  if ((m.soft || m.g.lscaled) && !fast) return cudaErrorInvalidValue;
  if (fast) a.R = m.ftab_R;
  if (fast)
    return m.pairs ? launch_fast<true>(a, m.sm_count, cps, m.stream) : launch_fast<false>(a, m.sm_count, cps, m.stream);
  return m.pairs ? launch_general<true>(a, m.sm_count, cps, m.stream)
                 : launch_general<false>(a, m.sm_count, cps, m.stream);
}

}  // namespace sbki
