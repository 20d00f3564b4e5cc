// sbki_query_points: Eq. (alpha_kernel) at arbitrary points of space (Sec. IV:
// the continuous model can be queried at any resolution, not only at voxel
// centres), from a given training set:
//     alpha^k(x*) = alpha_0 + sum over training points i with |x* - x_i| < l
//                   and y_i = k of sigma0 s_k f(|x* - x_i| / l).
// The accumulation turned around: the training points are binned into cells of
// edge just above l (so every point within l of a query lies in the 3 x 3 x 3
// cells around the query's cell), sorted by cell with the library's radix sort,
// the start of each cell's run entered in a hash; then one warp per query
// walks the 27 cells, evaluates the kernel of every point within l and sums
// per class in shared memory.  Membership is decided in FP32 from the exact
// FP32 offsets' squares and re-decided in FP64 inside the relative band around
// l^2, as in the map update, so it is the plain FP64 definition's.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "kernel_value.cuh"
#include "point_common.cuh"

namespace sbki {
namespace {

constexpr int kQThreads = 256;
constexpr int kQWarps = kQThreads / 32;
constexpr int kCellBits = 21;  // per axis in a packed cell key (offset 2^20)

__device__ __forceinline__ unsigned long long cell_key(float x, float y, float z, float inv_c) {
  const unsigned long long off = 1ull << (kCellBits - 1);
  const unsigned long long m = (1ull << kCellBits) - 1;
  const long long cx = (long long)floorf(x * inv_c), cy = (long long)floorf(y * inv_c), cz = (long long)floorf(z * inv_c);
  return ((((unsigned long long)(cx + (long long)off)) & m) << (2 * kCellBits)) |
         ((((unsigned long long)(cy + (long long)off)) & m) << kCellBits) | (((unsigned long long)(cz + (long long)off)) & m);
}

__device__ __forceinline__ uint32_t cell_hash(unsigned long long k, uint32_t cap) {
  k ^= k >> 31;
  k *= 0x9e3779b97f4a7c15ull;
  k ^= k >> 29;
  return (uint32_t)k & (cap - 1u);
}

__global__ void cell_keys_kernel(const float4* __restrict__ train, int64_t p, float inv_c,
                                 unsigned long long* __restrict__ keys, uint32_t* __restrict__ idx) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 t = train[i];
    keys[i] = cell_key(t.x, t.y, t.z, inv_c);
    idx[i] = (uint32_t)i;
  }
}

// the first position of every cell's run in the sorted order, entered in the hash
__global__ void cell_starts_kernel(const unsigned long long* __restrict__ keys, int64_t p,
                                   unsigned long long* __restrict__ hkeys, uint32_t* __restrict__ hstart, uint32_t cap,
                                   DevCounters* dc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = keys[i];
    if (i > 0 && keys[i - 1] == k) continue;
    uint32_t h = cell_hash(k, cap);
    for (uint32_t probe = 0;; ++probe) {
      if (probe >= cap) {
        set_error(dc, SBKI_ERR_CAPACITY);
        break;
      }
      const unsigned long long prev = atomicCAS(&hkeys[h], kEmpty, k);
      if (prev == kEmpty) {
        hstart[h] = (uint32_t)i;
        break;
      }
      h = (h + 1u) & (cap - 1u);
    }
  }
}

struct QueryArgs {
  Geom g;
  float inv_c;
  const float4* train;   // [p] (x, y, z, label as float)
  const unsigned long long* skeys;  // [p] cell keys, sorted
  const uint32_t* sidx;  // [p] training point of each sorted position
  int64_t p;
  const unsigned long long* hkeys;
  const uint32_t* hstart;
  uint32_t cap;
  const float* pts;      // [q,3]
  int64_t q;
  float* alpha;          // [q,K+1]
  float alpha0;
  DevCounters* dc;
};

// One warp per query point: lane c < 27 finds cell c's run, then the warp
// walks the runs, 32 points at a time, and sums the kernel values per class.
__global__ void __launch_bounds__(kQThreads) query_points_kernel(QueryArgs a) {
  __shared__ float s_acc[kQWarps][kMaxClasses];
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (a.dc->err != 0) return;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t qi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; qi < a.q; qi += nw) {
    const float qx = a.pts[3 * qi], qy = a.pts[3 * qi + 1], qz = a.pts[3 * qi + 2];
    if (lane < g.K1) s_acc[wid][lane] = 0.0f;
    uint32_t start = 0, count = 0;
    if (lane < 27) {
      const unsigned long long k0 = cell_key(qx, qy, qz, a.inv_c);
      const unsigned long long m = (1ull << kCellBits) - 1;
      const long long cx = (long long)((k0 >> (2 * kCellBits)) & m) + lane % 3 - 1;
      const long long cy = (long long)((k0 >> kCellBits) & m) + (lane / 3) % 3 - 1;
      const long long cz = (long long)(k0 & m) + lane / 9 - 1;
      if (cx >= 0 && cy >= 0 && cz >= 0 && cx <= (long long)m && cy <= (long long)m && cz <= (long long)m) {
        const unsigned long long k = ((unsigned long long)cx << (2 * kCellBits)) | ((unsigned long long)cy << kCellBits) |
                                     (unsigned long long)cz;
        uint32_t h = cell_hash(k, a.cap);
        for (uint32_t probe = 0; probe < a.cap; ++probe) {
          const unsigned long long hk = a.hkeys[h];
          if (hk == k) {
            start = a.hstart[h];
            uint32_t e = start;
            while ((int64_t)e < a.p && a.skeys[e] == k) ++e;
            count = e - start;
            break;
          }
          if (hk == kEmpty) break;
          h = (h + 1u) & (a.cap - 1u);
        }
      }
    }
    __syncwarp();
    for (int c = 0; c < 27; ++c) {
      const uint32_t s = __shfl_sync(0xffffffffu, start, c), n = __shfl_sync(0xffffffffu, count, c);
      for (uint32_t j = lane; j < n; j += 32) {
        const float4 t = a.train[a.sidx[s + j]];
        const float ex = __fsub_rn(qx, t.x), ey = __fsub_rn(qy, t.y), ez = __fsub_rn(qz, t.z);
        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
        bool in = d2 < g.l2_lo;
        if (!in && d2 < g.l2_hi) {  // the plain FP64 test, as the definition states it
          const double dx = (double)qx - (double)t.x, dy = (double)qy - (double)t.y, dz = (double)qz - (double)t.z;
          in = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)) < g.l2_64;
        }
        if (in) {
          const int label = label_of(t.w) & ((1 << kLabelBits) - 1);
          const float r = sqrtf(d2) * g.inv_l;
          atomicAdd(&s_acc[wid][label], g.sigma0_k[label] * kernel_f_poly(r));
        }
      }
    }
    __syncwarp();
    if (lane < g.K1) a.alpha[qi * g.K1 + lane] = __fadd_rn(a.alpha0, s_acc[wid][lane]);
    __syncwarp();
  }
}

bool device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

sbki_status fail(sbki_status s, const char* msg) {
  set_global_error(msg);
  return s;
}

}  // namespace
}  // namespace sbki

using namespace sbki;

extern "C" sbki_status sbki_query_points(const sbki_params* params, const float* xyzl, int64_t p, const float* pts,
                                         int64_t q, float* alpha_out) {
  if (!params || p < 0 || q < 0 || (p > 0 && !xyzl) || (q > 0 && (!pts || !alpha_out)))
    return fail(SBKI_ERR_INVALID_ARG, "query points: bad arguments");
  sbki_status st = validate_params(params);
  if (st != SBKI_OK) return st;
  if (params->sensor_model != 0) return fail(SBKI_ERR_INVALID_ARG, "query points: the counting model has no kernel");
  if (p > (int64_t)UINT32_MAX - 1) return fail(SBKI_ERR_INVALID_ARG, "query points: too many training points");
  if (q == 0) return SBKI_OK;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (cudaSetDevice(params->device) != cudaSuccess) return fail(SBKI_ERR_CUDA, "query points: cudaSetDevice failed");
  const Geom g = geometry_of(*params);
  cudaStream_t s = (cudaStream_t)params->cuda_stream;
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, params->device);
  const int64_t np = std::max<int64_t>(p, 1);
  uint32_t cap = 1024;
  while ((int64_t)cap < 2 * np) cap <<= 1;
  // device buffers (this entry point allocates; it is a stateless query)
  float4* dtrain = nullptr;
  float* dpts = nullptr;
  float* dalpha = nullptr;
  unsigned long long *k1 = nullptr, *k2 = nullptr, *hkeys = nullptr;
  uint32_t *v1 = nullptr, *v2 = nullptr, *hstart = nullptr, *work = nullptr, *ndev = nullptr;
  DevCounters* dc = nullptr;
  const int64_t wn = radix_work_entries(np);
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
    return e == cudaSuccess;
  };
  const bool dev_train = p > 0 && device_ptr(xyzl), dev_pts = device_ptr(pts), dev_out = device_ptr(alpha_out);
  ok(cudaMalloc(&k1, sizeof(*k1) * np));
  ok(cudaMalloc(&k2, sizeof(*k2) * np));
  ok(cudaMalloc(&v1, sizeof(*v1) * np));
  ok(cudaMalloc(&v2, sizeof(*v2) * np));
  ok(cudaMalloc(&hkeys, sizeof(*hkeys) * cap));
  ok(cudaMalloc(&hstart, sizeof(*hstart) * cap));
  ok(cudaMalloc(&work, sizeof(*work) * wn));
  ok(cudaMalloc(&ndev, sizeof(*ndev)));
  ok(cudaMalloc(&dc, sizeof(*dc)));
  if (!dev_train && p > 0) ok(cudaMalloc(&dtrain, sizeof(float4) * p));
  if (!dev_pts) ok(cudaMalloc(&dpts, sizeof(float) * 3 * q));
  if (!dev_out) ok(cudaMalloc(&dalpha, sizeof(float) * g.K1 * q));
  const float4* train = dev_train ? reinterpret_cast<const float4*>(xyzl) : dtrain;
  const float* qp = dev_pts ? pts : dpts;
  float* out = dev_out ? alpha_out : dalpha;
  if (e == cudaSuccess && !dev_train && p > 0)
    ok(cudaMemcpyAsync(dtrain, xyzl, sizeof(float4) * p, cudaMemcpyHostToDevice, s));
  if (e == cudaSuccess && !dev_pts) ok(cudaMemcpyAsync(dpts, pts, sizeof(float) * 3 * q, cudaMemcpyHostToDevice, s));
  if (e == cudaSuccess) ok(cudaMemsetAsync(dc, 0, sizeof(*dc), s));
  if (e == cudaSuccess) ok(cudaMemsetAsync(hkeys, 0xff, sizeof(*hkeys) * cap, s));
  const uint32_t n32 = (uint32_t)p;
  if (e == cudaSuccess) ok(cudaMemcpyAsync(ndev, &n32, sizeof(n32), cudaMemcpyHostToDevice, s));
  // cells of edge just above l: every point within l of a query lies in the 27 cells around it
  const float inv_c = (float)(1.0 / (params->length_scale * 1.001));
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((np + 255) / 256, (int64_t)sms * 8));
  if (e == cudaSuccess && p > 0) {
    cell_keys_kernel<<<grid, 256, 0, s>>>(train, p, inv_c, k1, v1);
    ok(cudaGetLastError());
    if (e == cudaSuccess) ok(radix_sort_pairs(k1, v1, k2, v2, ndev, np, 3 * kCellBits, work, sms, dc, s));
    if (e == cudaSuccess) {
      cell_starts_kernel<<<grid, 256, 0, s>>>(k1, p, hkeys, hstart, cap, dc);
      ok(cudaGetLastError());
    }
  }
  if (e == cudaSuccess) {
    QueryArgs a;
    a.g = g;
    a.inv_c = inv_c;
    a.train = train;
    a.skeys = k1;
    a.sidx = v1;
    a.p = p;
    a.hkeys = hkeys;
    a.hstart = hstart;
    a.cap = cap;
    a.pts = qp;
    a.q = q;
    a.alpha = out;
    a.alpha0 = (float)params->alpha0;
    a.dc = dc;
    const unsigned qgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((q + kQWarps - 1) / kQWarps, (int64_t)sms * 16));
    query_points_kernel<<<qgrid, kQThreads, 0, s>>>(a);
    ok(cudaGetLastError());
  }
  if (e == cudaSuccess && !dev_out)
    ok(cudaMemcpyAsync(alpha_out, dalpha, sizeof(float) * g.K1 * q, cudaMemcpyDeviceToHost, s));
  int32_t derr = 0;
  if (e == cudaSuccess) ok(cudaMemcpyAsync(&derr, &dc->err, sizeof(derr), cudaMemcpyDeviceToHost, s));
  if (e == cudaSuccess) ok(cudaStreamSynchronize(s));
  void* bufs[] = {k1, k2, v1, v2, hkeys, hstart, work, ndev, dc, dtrain, dpts, dalpha};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof(msg), "query points: %s", cudaGetErrorString(e));
    return fail(SBKI_ERR_CUDA, msg);
  }
  if (derr != 0) return fail((sbki_status)derr, "query points: device error");
  return SBKI_OK;
}
