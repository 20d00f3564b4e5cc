// Step a5 of the counting sensor model (S-CSM), Eq. (alpha): every training
// point adds 1 to alpha^{y_i} of the voxel that contains it.  The voxel is the
// read-off's key floor(x * fp32(1/res)) per axis, so a count lands where a
// query of the same point reads.  One global reduction per point; FP32 counts
// stay exact below 2^24 per voxel and class.  The blocks were inserted by
// touch_cells_kernel and committed before this launch, and the ones created
// by this update are zero-filled first.
#include <algorithm>

#include "point_common.cuh"

namespace sbki {
namespace {

struct CountArgs {
  Geom g;
  const float4* train;
  const unsigned long long* hkeys;
  const int32_t* hvals;
  int64_t hash_cap;
  float* alpha;
  int32_t* pairs;  // per-voxel counts of counted points (tracking only), or null
  DevCounters* dc;
};

template <bool kTrack>
__global__ void __launch_bounds__(256) accumulate_counts_kernel(CountArgs a) {
  const Geom& g = a.g;
  if (a.dc->err != 0) return;
  const uint32_t P = a.dc->n_train;
  const int m = g.B - 1;
  uint32_t counted = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    const float4 p = a.train[i];
    const int lm = label_of(p.w);
    const int label = lm & ((1 << kLabelBits) - 1), map = lm >> kLabelBits;
    const int vx = floor_small(__fmul_rn(p.x, g.inv_res)), vy = floor_small(__fmul_rn(p.y, g.inv_res)),
              vz = floor_small(__fmul_rn(p.z, g.inv_res));
    const int32_t pool =
        find_pool_slot(a.hkeys, a.hvals, a.hash_cap, pack_block(vx >> g.B_shift, vy >> g.B_shift, vz >> g.B_shift, map));
    if (pool < 0) continue;
    const int local = ((((vz & m) << g.B_shift) + (vy & m)) << g.B_shift) + (vx & m);
    red_add_if(true, a.alpha + ((size_t)pool * g.K1 + label) * g.B3 + local, 1.0f);
    if (kTrack) red_add_if(true, a.pairs + (size_t)pool * g.B3 + local, 1);
    ++counted;
  }
  counted = __reduce_add_sync(0xffffffffu, counted);
  if ((threadIdx.x & 31u) == 0 && counted) atomicAdd(&a.dc->pairs, (unsigned long long)counted);
}

}  // namespace

cudaError_t launch_accumulate_counts(MapState& m, int64_t bound) {
  cudaError_t e = launch_fresh_fill(m);
  if (e != cudaSuccess) return e;
  CountArgs a;
  a.g = m.g;
  a.train = m.s.train;
  a.hkeys = m.hkeys;
  a.hvals = m.hvals;
  a.hash_cap = m.hash_cap;
  a.alpha = m.alpha;
  a.pairs = m.pairs;
  a.dc = m.dc;
  // the training points never exceed the items of the update
  const unsigned blocks =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>((bound + 255) / 256, (int64_t)m.sm_count * 8));
  if (m.pairs) accumulate_counts_kernel<true><<<blocks, 256, 0, m.stream>>>(a);
  else accumulate_counts_kernel<false><<<blocks, 256, 0, m.stream>>>(a);
  m.launches += 1;
  return cudaGetLastError();
}

}  // namespace sbki
