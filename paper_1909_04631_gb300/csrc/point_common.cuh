// Shared device pieces of the point-major passes over a training set: the
// per-point frame (voxel, compensated centre offsets, sub-voxel part, reachable
// blocks), conversion-free integer/float helpers, the block lookup and
// predicated global reductions.  Used by the accumulation of Eq. (alpha_kernel)
// and by its backward pass, so both enumerate exactly the same pairs.
#pragma once
#include "sbki_internal.cuh"

namespace sbki {

// floor of v for |v| < 2^22, without a conversion instruction: adding 1.5 2^23
// rounded toward -inf leaves floor(v) in the low mantissa bits
__device__ __forceinline__ int floor_small(float v) { return __float_as_int(__fadd_rd(v, 12582912.0f)) - 0x4B400000; }

// a class label stored as a float (exact: 0 <= label < 2^22)
__device__ __forceinline__ int label_of(float w) { return __float_as_int(__fadd_rn(w, 8388608.0f)) - 0x4B000000; }

// fire-and-forget global reductions, issued only where p holds
__device__ __forceinline__ void red_add_if(bool p, float* addr, float v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q red.global.add.f32 [%1], %2;\n\t}" ::"r"((int)p),
               "l"(addr), "f"(v)
               : "memory");
}
__device__ __forceinline__ void red_add_if(bool p, int32_t* addr, int32_t v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q red.global.add.s32 [%1], %2;\n\t}" ::"r"((int)p),
               "l"(addr), "r"(v)
               : "memory");
}

// pool slot of a block key, or -1 (bounded linear probing)
__device__ __forceinline__ int32_t find_pool_slot(const unsigned long long* hkeys, const int32_t* hvals, int64_t cap,
                                                  unsigned long long key) {
  uint32_t slot = hash_slot(key, cap);
  for (int probe = 0; probe < kMaxProbes; ++probe) {
    const unsigned long long k = hkeys[slot];
    if (k == key) return hvals[slot];
    if (k == kEmpty) return -1;
    slot = (uint32_t)((slot + 1) & (uint32_t)(cap - 1));
  }
  return -1;
}

// Everything about one training point that every lane of its warp shares.
struct PointFrame {
  int v0[3];        // voxel of the point
  float hi[3], lo[3];  // compensated offset c(v0) - x per axis
  int part;         // sub-voxel part 0..kParts^3-1 (kParts per axis)
  int blo[3], nb[3];   // the 3 x 3 x 3 blocks around the point's block: first block, count (3)
};

__device__ __forceinline__ PointFrame point_frame(float x, float y, float z, int R, const Geom& g) {
  PointFrame f;
  int pt[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const float xa = ax == 0 ? x : (ax == 1 ? y : z);
    f.v0[ax] = floor_small(__fmul_rn(xa, g.inv_res));
    centre_offset0(f.v0[ax], xa, g, f.hi[ax], f.lo[ax]);
    // sub-voxel position 1/2 - E0/res (accurate anywhere in the map), in kParts-ths
    const float phi = 0.5f - __fmul_rn(__fadd_rn(f.hi[ax], f.lo[ax]), g.inv_res);
    pt[ax] = min(kParts - 1, max(0, floor_small(phi * (float)kParts)));
    // every voxel within R <= B of v0 lies in the point's block or a neighbour
    f.blo[ax] = (f.v0[ax] >> g.B_shift) - 1;
    f.nb[ax] = 3;
  }
  f.part = pt[0] + kParts * (pt[1] + kParts * pt[2]);
  return f;
}

// Address part of voxel offset j (in -R..R) along x, and along y and z together:
// the block-offset digit (base 3 per axis) in the low byte, the in-block index
// above it, so an x part and a yz part add up to (digit | local << 8).
__device__ __forceinline__ int xpart(const PointFrame& f, int jx, int R, const Geom& g) {
  const int vx = f.v0[0] + jx - R;
  return ((vx >> g.B_shift) - f.blo[0]) | ((vx & (g.B - 1)) << 8);
}
__device__ __forceinline__ int yzpart(const PointFrame& f, int jy, int jz, int R, const Geom& g) {
  const int vy = f.v0[1] + jy - R, vz = f.v0[2] + jz - R, m = g.B - 1;
  return (3 * ((vy >> g.B_shift) - f.blo[1]) + 9 * ((vz >> g.B_shift) - f.blo[2])) |
         ((((vz & m) << g.B_shift) + (vy & m)) << (g.B_shift + 8));
}

// Pool slot of reachable block `digit` (bx + 3 by + 9 bz) of map `map`, or -1.
__device__ __forceinline__ int32_t digit_pool(const PointFrame& f, int digit, int map,
                                              const unsigned long long* hkeys, const int32_t* hvals, int64_t cap) {
  const int bx = digit % 3, by = (digit / 3) % 3, bz = digit / 9;
  if (bx >= f.nb[0] || by >= f.nb[1] || bz >= f.nb[2]) return -1;
  return find_pool_slot(hkeys, hvals, cap, pack_block(f.blo[0] + bx, f.blo[1] + by, f.blo[2] + bz, map));
}

// Candidate list entry: X row byte offset (8 jx) | YZ row byte offset (8 (jy (2R+1) + jz)) << 8
// | jy << 19 | jz << 23; padding entries point at X row 2R + 1.
__device__ __forceinline__ int entry_jx(uint32_t e) { return (int)((e & 0xffu) >> 3); }
__device__ __forceinline__ int entry_jy(uint32_t e) { return (int)((e >> 19) & 15u); }
__device__ __forceinline__ int entry_jz(uint32_t e) { return (int)((e >> 23) & 15u); }

}  // namespace sbki
