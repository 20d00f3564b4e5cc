// Read-off of the Dirichlet posterior at query points: Eq. (variance) for the
// mean E[theta^k] = alpha^k / sum alpha and V[theta^k] = E (1 - E) / (sum alpha + 1),
// the occupancy probability of Sec. V-C (sum of the occupied-class
// probabilities), the argmax label (ties to the lowest class) and the
// free / unknown / occupied state with the thresholds of Sec. V-A.  A voxel
// with no kernel mass (never reached, or outside every allocated block) reads
// as the prior alpha_0 and is unknown.
#include <algorithm>

#include "sbki_internal.cuh"

namespace sbki {
namespace {

struct QueryArgs {
  Geom g;
  float alpha0;
  double free_thresh, occ_thresh;
  const unsigned long long* hkeys;
  const int32_t* hvals;
  int64_t hash_cap;
  const float* alpha;
  const float* xyz;
  int64_t q;
  float* probs;
  float* var;
  float* mode;
  int32_t* label;
  float* p_occ;
  int32_t* state;
  int map;
};

__device__ int32_t lookup_block(const QueryArgs& a, unsigned long long key) {
  uint32_t slot = hash_slot(key, a.hash_cap);
  for (int probe = 0; probe < kMaxProbes; ++probe) {
    const unsigned long long k = a.hkeys[slot];
    if (k == key) return a.hvals[slot];
    if (k == kEmpty) return -1;
    slot = (uint32_t)((slot + 1) & (uint32_t)(a.hash_cap - 1));
  }
  return -1;
}

__global__ void __launch_bounds__(256) query_kernel(QueryArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.q) return;
  const Geom& g = a.g;
  const int K1 = g.K1;
  int v[3];
  bool inside = true;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const float s = __fmul_rn(a.xyz[3 * i + ax], g.inv_res);
    inside = inside && fabsf(s) < (float)(kKeyLimit - 64);
    v[ax] = inside ? (int)floorf(s) : 0;
  }
  int32_t pool = -1;
  int local = 0;
  if (inside) {
    pool = lookup_block(a, pack_block(v[0] >> g.B_shift, v[1] >> g.B_shift, v[2] >> g.B_shift, a.map));
    const int m = g.B - 1;
    local = (((v[2] & m) << g.B_shift) + (v[1] & m)) * g.B + (v[0] & m);
  }
  const float* inc = pool >= 0 ? a.alpha + (size_t)pool * K1 * g.B3 + local : nullptr;
  // sums in FP64: 1 - E_k = (S - alpha_k)/S must not cancel when one class dominates
  double S = 0.0, mass = 0.0;
  float amax = -1.f, amin = 3.0e38f;
  int best = 0;
  for (int k = 0; k < K1; ++k) {
    const float d = inc ? inc[(size_t)k * g.B3] : 0.f;
    const float al = a.alpha0 + d;
    mass += d;
    S += al;
    amin = fminf(amin, al);
    if (al > amax) {
      amax = al;
      best = k;
    }
  }
  const bool mode_ok = amin > 1.0f;
  double po = 0.0;
  for (int k = 0; k < K1; ++k) {
    const double al = (double)(a.alpha0 + (inc ? inc[(size_t)k * g.B3] : 0.f));
    a.probs[i * K1 + k] = (float)(al / S);
    if (a.var) a.var[i * K1 + k] = (float)(al * (S - al) / (S * S * (S + 1.0)));
    if (a.mode) a.mode[i * K1 + k] = mode_ok ? (float)((al - 1.0) / (S - (double)K1)) : __int_as_float(0x7fc00000);
    if (k > 0) po += al / S;
  }
  if (a.label) a.label[i] = best;
  if (a.p_occ) a.p_occ[i] = (float)po;
  if (a.state) {
    int st = 1;
    if (mass > 0.0) st = po < a.free_thresh ? 0 : (po > a.occ_thresh ? 2 : 1);
    a.state[i] = st;
  }
}

}  // namespace

cudaError_t launch_query(const MapState& m, const float* xyz, int64_t q, float* probs, float* var, float* mode,
                         int32_t* label, float* p_occ, int32_t* state) {
  if (q <= 0) return cudaSuccess;
  QueryArgs a;
  a.g = m.g;
  a.alpha0 = (float)m.prm.alpha0;
  a.free_thresh = m.prm.free_thresh;
  a.occ_thresh = m.prm.occ_thresh;
  a.hkeys = m.hkeys;
  a.hvals = m.hvals;
  a.hash_cap = m.hash_cap;
  a.alpha = m.alpha;
  a.xyz = xyz;
  a.q = q;
  a.probs = probs;
  a.var = var;
  a.mode = mode;
  a.label = label;
  a.p_occ = p_occ;
  a.state = state;
  a.map = m.active_map;
  query_kernel<<<(unsigned)((q + 255) / 256), 256, 0, m.stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gather_alpha(const MapState& m, float* out, int64_t nblocks) {
  return cudaMemcpyAsync(out, m.alpha, sizeof(float) * (size_t)nblocks * m.g.K1 * m.g.B3, cudaMemcpyDeviceToDevice,
                         m.stream);
}

}  // namespace sbki

namespace sbki {
namespace {

// 1 for every pool block of the selected map (scanned into output rows next)
__global__ void export_flags_kernel(const unsigned long long* __restrict__ pool_keys, uint32_t nb, int map,
                                    uint32_t* __restrict__ flags) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
    flags[b] = map_of_block(pool_keys[b]) == map ? 1u : 0u;
}

// One row per voxel of every selected block: key (x, y, z) and alpha with prior.
__global__ void export_rows_kernel(const unsigned long long* __restrict__ pool_keys, const uint32_t* __restrict__ rowb,
                                   uint32_t nb, int map, Geom g, const float* __restrict__ alpha, float alpha0,
                                   int64_t* __restrict__ keys, float* __restrict__ out) {
  const int64_t total = (int64_t)nb * g.B3;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t b = (uint32_t)(e / g.B3);
    const int li = (int)(e - (int64_t)b * g.B3);
    const unsigned long long k = pool_keys[b];
    if (map_of_block(k) != map) continue;
    const int64_t row = (int64_t)rowb[b] * g.B3 + li;
    int32_t bx, by, bz;
    unpack_block(k, bx, by, bz);
    if (keys) {
      keys[3 * row] = (int64_t)bx * g.B + li % g.B;
      keys[3 * row + 1] = (int64_t)by * g.B + (li / g.B) % g.B;
      keys[3 * row + 2] = (int64_t)bz * g.B + li / (g.B * g.B);
    }
    if (out)
      for (int c = 0; c < g.K1; ++c)
        out[row * g.K1 + c] = __fadd_rn(alpha0, alpha[((size_t)b * g.K1 + c) * g.B3 + li]);
  }
}

}  // namespace

cudaError_t launch_export_rows(const MapState& m, uint32_t nb, uint32_t* rowb, void* scan_tmp, int64_t* keys,
                               float* out) {
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)nb + 255) / 256, 4096));
  export_flags_kernel<<<grid, 256, 0, m.stream>>>(m.pool_keys, nb, m.active_map, rowb);
  cudaError_t e = exclusive_scan_u32(rowb, nb, scan_tmp, m.stream);
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)nb * m.g.B3;
  const unsigned g2 = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)m.sm_count * 16));
  export_rows_kernel<<<g2, 256, 0, m.stream>>>(m.pool_keys, rowb, nb, m.active_map, m.g, m.alpha,
                                               (float)m.prm.alpha0, keys, out);
  return cudaGetLastError();
}

}  // namespace sbki
