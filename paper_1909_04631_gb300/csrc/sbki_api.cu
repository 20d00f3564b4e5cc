// The C ABI of include/sbki.h: argument checks, memory ownership, pointer-kind
// handling and the order of launches of one update.  All arithmetic of the
// update runs in the kernels of ingest.cu, blocks.cu and accumulate.cu.
#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sbki_internal.cuh"

using namespace sbki;

struct sbki_map {
  MapState st;
};

namespace {

char g_create_error[512] = {0};

sbki_status fail(MapState* m, sbki_status s, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
sbki_status fail(MapState* m, sbki_status s, const char* fmt, ...) {
  char* buf = m ? m->last_error : g_create_error;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return s;
}

#define CK(m, expr)                                                                              \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      return fail((m), SBKI_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),   \
                  __FILE__, __LINE__);                                                           \
    }                                                                                            \
  } while (0)

// Restores the caller's current device when a call returns.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int ceil_log2(int64_t v) {
  int b = 0;
  while ((1ll << b) < v) ++b;
  return b;
}

int64_t floor_div64(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

// A named range on the profiler's timeline (NVTX; header-only, a no-op unless a
// tool is attached): the stages of an update appear beside the kernels.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// device temporaries of one call, freed (after the stream drains) when it returns
struct TmpFree {
  void* p[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t st = nullptr;
  ~TmpFree() {
    bool any = false;
    for (void* q : p) any = any || q;
    if (!any) return;
    cudaStreamSynchronize(st);
    for (void* q : p)
      if (q) cudaFree(q);
  }
};

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, sizeof(T) * count);
}

__global__ void begin_kernel(DevCounters* dc, uint32_t epoch, uint32_t n_points) {
  dc->n_points = n_points;
  dc->pairs = 0;
  dc->touched_voxels = 0;
  dc->n_free = 0;
  dc->err = 0;
  dc->n_valid = 0;
  dc->n_items = 0;
  dc->n_train = 0;
  dc->n_tiles = 0;
  dc->n_touched = 0;
  dc->n_new = 0;
  dc->n_slow = 0;
  dc->work_next = 0;
  dc->n_soft = 0;
  dc->epoch = epoch;
  dc->n_blocks_before = dc->n_blocks;
  for (int a = 0; a < 3; ++a) {
    dc->tbox[a] = INT_MAX;
    dc->tbox[3 + a] = INT_MIN;
  }
}

// begin_kernel for a batched update recorded in a graph: the epoch advances on
// the device and the point count comes from the scan descriptors
__global__ void batch_begin_kernel(DevCounters* dc, const ScanDesc* desc, int ns) {
  dc->pairs = 0;
  dc->touched_voxels = 0;
  dc->n_free = 0;
  dc->err = 0;
  dc->n_valid = 0;
  dc->n_items = 0;
  dc->n_train = 0;
  dc->n_tiles = 0;
  dc->n_touched = 0;
  dc->n_new = 0;
  dc->n_slow = 0;
  dc->work_next = 0;
  dc->n_soft = 0;
  dc->epoch = dc->epoch + 1;
  dc->n_blocks_before = dc->n_blocks;
  dc->n_points = (uint32_t)desc[ns].off;
  for (int a = 0; a < 3; ++a) {
    dc->tbox[a] = INT_MAX;
    dc->tbox[3 + a] = INT_MIN;
  }
}

__global__ void bbox_init_kernel(int* bbox) {
  if (threadIdx.x < 3) bbox[threadIdx.x] = INT_MAX;
  else if (threadIdx.x < 6) bbox[threadIdx.x] = INT_MIN;
}

__global__ void set_items_kernel(DevCounters* dc, uint32_t n) { dc->n_items = n; }

sbki_status check_params(const sbki_params* p) {
  if (!p) return fail(nullptr, SBKI_ERR_INVALID_ARG, "params is NULL");
  const double ds = p->ds_res > 0 ? p->ds_res : p->res;
  if (!(p->res > 0) || !std::isfinite(p->res)) return fail(nullptr, SBKI_ERR_INVALID_ARG, "res must be > 0");
  if (!(ds > 0) || !std::isfinite(ds)) return fail(nullptr, SBKI_ERR_INVALID_ARG, "ds_res must be > 0");
  if (!(p->length_scale > 0)) return fail(nullptr, SBKI_ERR_INVALID_ARG, "length_scale must be > 0");
  if (!(p->sigma0 >= 0) || !std::isfinite(p->sigma0)) return fail(nullptr, SBKI_ERR_INVALID_ARG, "sigma0 must be >= 0");
  if (!(p->alpha0 > 0) || !std::isfinite(p->alpha0)) return fail(nullptr, SBKI_ERR_INVALID_ARG, "alpha0 must be > 0");
  if (!(p->free_step > 0)) return fail(nullptr, SBKI_ERR_INVALID_ARG, "free_step must be > 0");
  if (!(p->min_range >= 0) || !(p->max_range >= p->min_range) || !std::isfinite(p->max_range))
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "need 0 <= min_range <= max_range < inf");
  if (p->num_classes < 1 || p->num_classes + 1 > kMaxClasses)
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "num_classes must be in 1..%d", kMaxClasses - 1);
  if (p->block_edge != 4 && p->block_edge != 8)
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "block_edge must be 4 or 8");
  if (p->length_scale > 0.75 * p->block_edge * p->res)
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "length_scale must be <= 0.75 * block_edge * res");
  if (p->pool_blocks < 1 || p->pool_blocks > (1ll << 28))
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "pool_blocks must be in 1..2^28");
  if (p->num_maps < 1 || p->num_maps > kMaxMaps)
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "num_maps must be in 1..%d", kMaxMaps);
  if (p->accumulate_mode != 0 && p->accumulate_mode != 1)
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "accumulate_mode must be 0 (point-major) or 1 (block-major)");
  if (p->sensor_model != 0 && p->sensor_model != 1)
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "sensor_model must be 0 (kernel inference) or 1 (counting)");
  if (p->sensor_model == 1 && p->accumulate_mode != 0)
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "the counting sensor model needs accumulate_mode 0");
  if (p->association != 0 && p->association != 1)
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "association must be 0 (every voxel within l) or 1 (extended block)");
  bool lscaled = false;
  for (int k = 0; k <= p->num_classes; ++k) {
    if (!(p->l_scale[k] > 0) || !std::isfinite(p->l_scale[k]))
      return fail(nullptr, SBKI_ERR_INVALID_ARG, "l_scale[%d] must be finite and > 0", k);
    if (p->length_scale * p->l_scale[k] > 0.75 * p->block_edge * p->res)
      return fail(nullptr, SBKI_ERR_INVALID_ARG, "length_scale * l_scale[%d] must be <= 0.75 * block_edge * res", k);
    lscaled = lscaled || p->l_scale[k] != 1.0;
  }
  if (lscaled && p->sensor_model == 0 && (p->accumulate_mode != 0 || p->association != 0))
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "per-class length scales need accumulate_mode 0 and association 0");
  for (int k = 0; k <= p->num_classes; ++k)
    if (!(p->sigma0_scale[k] > 0) || !std::isfinite(p->sigma0_scale[k]))
      return fail(nullptr, SBKI_ERR_INVALID_ARG, "sigma0_scale[%d] must be finite and > 0", k);
  if (p->sample_capacity < 1 || p->sample_capacity > (1ll << 27))
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "sample_capacity must be in 1..2^27");
  // tiles of training points overlapping one dilated block must stay few
  const double span = p->block_edge * p->res + 2.0 * p->length_scale * 1.001 + 2.0 * ds;
  const int per_axis = (int)std::ceil(span / (kTileEdge * ds)) + 1;
  if (per_axis * per_axis * per_axis > 64)
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "ds_res too small relative to the block size and length scale");
  // a scan's keys must fit in 64 bits
  const int64_t half = (int64_t)std::ceil((p->max_range + 2.0 * ds) / (kTileEdge * ds)) + 2;
  const int bits = ceil_log2(2 * half + 1);
  if (3 * bits + kLocalBits + ceil_log2(p->num_classes + 1) > 64 || p->max_range / p->res > kKeyLimit / 4)
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "max_range too large for res/ds_res");
  return SBKI_OK;
}

Geom make_geom(const sbki_params& p) {
  Geom g;
  const double ds = p.ds_res > 0 ? p.ds_res : p.res;
  const double band = 2e-6;  // relative: the FP32 d^2 is within ~5e-7 (compensated offsets)
  g.res = (float)p.res;
  g.inv_res = (float)(1.0 / p.res);
  g.res_lo = (float)(p.res - (double)g.res);
  g.ds = (float)ds;
  g.inv_ds = (float)(1.0 / ds);
  g.l = (float)p.length_scale;
  g.inv_l = (float)(1.0 / p.length_scale);
  g.l2 = (float)(p.length_scale * p.length_scale);
  g.l2_lo = (float)(p.length_scale * p.length_scale * (1.0 - band));
  g.l2_hi = (float)(p.length_scale * p.length_scale * (1.0 + band));
  g.sigma0 = (float)p.sigma0;
  for (int k = 0; k < 32; ++k) {
    const bool used = k <= p.num_classes;
    g.sigma0_k[k] = used ? (float)(p.sigma0 * p.sigma0_scale[k]) : 0.f;
    g.scale_k[k] = used ? (float)p.sigma0_scale[k] : 0.f;
  }
  g.step = (float)p.free_step;
  g.fast_lim = (float)(2.5 * ds);
  g.res64 = p.res;
  g.l64 = p.length_scale;
  g.l2_64 = p.length_scale * p.length_scale;
  g.min_range = p.min_range;
  g.max_range = p.max_range;
  g.K1 = p.num_classes + 1;
  g.B = p.block_edge;
  g.B_shift = p.block_edge == 8 ? 3 : 2;
  g.B3 = p.block_edge * p.block_edge * p.block_edge;
  g.label_bits = std::max(1, ceil_log2(g.K1));
  g.assoc = p.sensor_model == 0 ? p.association : 0;
  g.lscaled = 0;
  g.lmax64 = p.length_scale;
  for (int k = 0; k < 32; ++k) {
    const bool used = k <= p.num_classes;
    const double lk = p.length_scale * (used ? p.l_scale[k] : 1.0);
    if (used && p.l_scale[k] != 1.0) g.lscaled = 1;
    if (used) g.lmax64 = std::max(g.lmax64, lk);
    g.inv_lk[k] = (float)(1.0 / lk);
    g.l2k_lo[k] = (float)(lk * lk * (1.0 - band));
    g.l2k_hi[k] = (float)(lk * lk * (1.0 + band));
    g.l2k_64[k] = lk * lk;
  }
  return g;
}

// Key frame of a scan: tiles relative to the sensor origin's tile.
KeyFrame scan_frame(const MapState& m, const double T[16]) {
  KeyFrame kf;
  const double ds = m.prm.ds_res > 0 ? m.prm.ds_res : m.prm.res;
  const int64_t half = (int64_t)std::ceil((m.prm.max_range + 2.0 * ds) / (kTileEdge * ds)) + 2;
  kf.bits[0] = kf.bits[1] = kf.bits[2] = ceil_log2(2 * half + 1);
  for (int a = 0; a < 3; ++a) {
    const float o = (float)T[4 * a + 3];
    const float q = o * m.g.inv_ds;
    const int64_t gcell = (int64_t)std::floor(q);
    kf.org[a] = (int32_t)(floor_div64(gcell, kTileEdge) - half);
  }
  kf.total_bits = kf.bits[0] + kf.bits[1] + kf.bits[2] + kLocalBits + m.g.label_bits;
  kf.scan_bits = 0;
  return kf;
}

// Key frame of one scan fitted to its tile bounding box (kept hits and the
// sensor origin, one tile of margin: every free sample lies on a segment
// between the origin and a hit), so the sort covers fewer key bits.
void fit_frame_to_box(const Geom& g, const int32_t tb[6], const double T[16], KeyFrame& kf) {
  for (int a = 0; a < 3; ++a) {
    const int64_t ot = floor_div64((int64_t)std::floor((float)T[4 * a + 3] * g.inv_ds), kTileEdge);
    const int64_t lo = std::min<int64_t>(tb[a], ot) - 1, hi = std::max<int64_t>(tb[3 + a], ot) + 1;
    kf.org[a] = (int32_t)lo;
    kf.bits[a] = std::max(1, ceil_log2(hi - lo + 1));
  }
  kf.total_bits = kf.bits[0] + kf.bits[1] + kf.bits[2] + kLocalBits + g.label_bits;
}

// Descriptor of one scan (device point and label pointers).
void fill_desc(ScanDesc& d, const float* pts, const int32_t* labels, int64_t n, int64_t off, const double T[16],
               const KeyFrame& kf, int map) {
  d.pts = pts;
  d.labels = labels;
  d.n = n;
  d.off = off;
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) d.r[3 * r + c] = T[4 * r + c];
    d.t[r] = T[4 * r + 3];
    d.o[r] = (float)T[4 * r + 3];
    d.org[r] = kf.org[r];
  }
  d.map_id = map;
  d.probs = nullptr;
}

cudaError_t free_scratch_points(Scratch& s) {
  cudaFree(s.pts);
  cudaFree(s.labels);
  cudaFree(s.world);
  cudaFree(s.cnt);
  s.pts = nullptr;
  s.labels = nullptr;
  s.world = nullptr;
  s.cnt = nullptr;
  s.n_cap = 0;
  return cudaSuccess;
}

sbki_status ensure_point_capacity(MapState& m, int64_t n) {
  Scratch& s = m.s;
  if (n <= s.n_cap) return SBKI_OK;
  CK(&m, cudaStreamSynchronize(m.stream));
  free_scratch_points(s);
  int64_t cap = std::max<int64_t>(n, 1 << 16);
  CK(&m, dalloc(&s.pts, 3 * cap));
  CK(&m, dalloc(&s.labels, cap));
  CK(&m, dalloc(&s.world, cap));
  CK(&m, dalloc(&s.cnt, cap + 1));
  s.n_cap = cap;  // scan partials are sized at creation for 2^27 entries
  m.scratch_gen += 1;  // recorded graphs name the old buffers
  return SBKI_OK;
}

// Buffers of the soft-label path, sized for n input points (allocated on first use).
sbki_status ensure_soft_capacity(MapState& m, int64_t n) {
  Scratch& s = m.s;
  if (!s.softidx) CK(&m, dalloc(&s.softidx, s.s_cap));
  if (n <= s.soft_cap) return SBKI_OK;
  CK(&m, cudaStreamSynchronize(m.stream));
  cudaFree(s.probs);
  cudaFree(s.hit_src);
  cudaFree(s.wsoft);
  s.probs = nullptr;
  s.hit_src = nullptr;
  s.wsoft = nullptr;
  s.soft_cap = 0;
  const int64_t cap = std::max<int64_t>(n, 1 << 16);
  CK(&m, dalloc(&s.probs, (size_t)cap * (m.g.K1 - 1)));
  CK(&m, dalloc(&s.hit_src, cap));
  CK(&m, dalloc(&s.wsoft, (size_t)cap * m.g.K1));
  s.soft_cap = cap;
  return SBKI_OK;
}

void profile_collect(MapState& m, const cudaEvent_t* ev);

// Copies the device counters to the host and waits for the stream; the stage
// times of an asynchronous update issued before are complete then, and are added.
sbki_status read_counters(MapState& m) {
  CK(&m, cudaMemcpyAsync(m.hc, m.dc, sizeof(DevCounters), cudaMemcpyDeviceToHost, m.stream));
  CK(&m, cudaStreamSynchronize(m.stream));
  if (m.prof_pending) {
    m.prof_pending = false;
    profile_collect(m, m.ev_alt);
  }
  return SBKI_OK;
}

sbki_status status_from_device(MapState& m) {
  const int e = m.hc->err;
  if (e == 0) return SBKI_OK;
  switch (e) {
    case SBKI_ERR_LABEL_RANGE:
      return fail(&m, SBKI_ERR_LABEL_RANGE, "a label is outside the allowed range; the map is unchanged");
    case SBKI_ERR_CAPACITY:
      return fail(&m, SBKI_ERR_CAPACITY,
                  "capacity exceeded (samples %u of %lld, blocks %u+%u of %lld); the map is unchanged",
                  m.hc->n_items, (long long)m.s.s_cap, m.hc->n_blocks, m.hc->n_new, (long long)m.pool_blocks);
    case SBKI_ERR_TIMEOUT:
      return fail(&m, SBKI_ERR_TIMEOUT, "a bounded device wait ran out");
    default:
      return fail(&m, (sbki_status)e, "device reported error %d", e);
  }
}

void fill_stats(const MapState& m, int64_t n, sbki_stats* st) {
  sbki_stats s{};
  const DevCounters& c = *m.hc;
  s.hits = c.n_valid;
  s.dropped = n - (int64_t)c.n_valid;
  s.free_samples = (int64_t)c.n_free;
  s.train_points = c.n_train;
  s.touched_blocks = c.n_touched;
  s.new_blocks = c.err == 0 ? c.n_new : 0;
  s.pairs = (int64_t)c.pairs;
  s.touched_voxels = (int64_t)c.touched_voxels;
  s.total_blocks = c.n_blocks;
  if (st) *st = s;
}

// Steps a1-a3 on device; leaves the training set in s.train.  On return
// *nitems holds the number of hits + free samples (0 on a pending error).
sbki_status run_ingest(MapState& m, const float* points, const int32_t* labels, int64_t n, const double T[16],
                       KeyFrame& kf, int64_t* nitems, int map, const float* probs = nullptr) {
  NvtxRange range("sbki: ingest (a1-a3)");
  *nitems = 0;
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(T[i])) return fail(&m, SBKI_ERR_INVALID_ARG, "sensor_pose has a non-finite entry");
  for (int a = 0; a < 3; ++a) {
    const double reach = std::fabs(T[4 * a + 3]) + m.prm.max_range;
    if (reach / m.prm.res > (double)(kKeyLimit - 1024))
      return fail(&m, SBKI_ERR_INVALID_ARG, "sensor origin too far from the map origin");
  }
  sbki_status st = ensure_point_capacity(m, n);
  if (st != SBKI_OK) return st;
  const float* dpts = points;
  const int32_t* dlab = labels;
  if (!is_device_ptr(points)) {
    CK(&m, cudaMemcpyAsync(m.s.pts, points, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, m.stream));
    dpts = m.s.pts;
  }
  const float* dprobs = probs;
  if (probs) {  // soft labels: probability vectors instead of labels
    st = ensure_soft_capacity(m, n);
    if (st != SBKI_OK) return st;
    if (!is_device_ptr(probs)) {
      CK(&m, cudaMemcpyAsync(m.s.probs, probs, sizeof(float) * (m.g.K1 - 1) * n, cudaMemcpyHostToDevice, m.stream));
      dprobs = m.s.probs;
    }
    dlab = nullptr;
  } else if (!is_device_ptr(labels)) {
    CK(&m, cudaMemcpyAsync(m.s.labels, labels, sizeof(int32_t) * n, cudaMemcpyHostToDevice, m.stream));
    dlab = m.s.labels;
  }
  m.epoch += 1;
  if (m.profiling) CK(&m, cudaEventRecord(m.ev[0], m.stream));
  begin_kernel<<<1, 1, 0, m.stream>>>(m.dc, m.epoch, (uint32_t)n);
  m.launches += 1;
  kf = scan_frame(m, T);
  fill_desc(m.hdesc[0], dpts, dlab, n, 0, T, kf, map);
  m.hdesc[0].probs = dprobs;
  m.hdesc[1] = ScanDesc{};
  m.hdesc[1].off = n;
  CK(&m, cudaMemcpyAsync(m.s.desc, m.hdesc, 2 * sizeof(ScanDesc), cudaMemcpyHostToDevice, m.stream));
  CK(&m, launch_transform_count(m, 1, n));
  st = read_counters(m);
  if (st != SBKI_OK) return st;
  if (m.hc->err != 0) return status_from_device(m);
  *nitems = m.hc->n_items;
  if (*nitems == 0) return SBKI_OK;
  fit_frame_to_box(m.g, m.hc->tbox, T, kf);
  m.hdesc[0].org[0] = kf.org[0];
  m.hdesc[0].org[1] = kf.org[1];
  m.hdesc[0].org[2] = kf.org[2];
  CK(&m, cudaMemcpyAsync(m.s.desc, m.hdesc, sizeof(ScanDesc), cudaMemcpyHostToDevice, m.stream));
  CK(&m, launch_emit(m, 1, n, kf, probs ? m.s.hit_src : nullptr));
  CK(&m, launch_downsample_n(m, kf, *nitems));
  if (probs) CK(&m, launch_soft_weights(m));
  return SBKI_OK;
}

sbki_status run_update(MapState& m, const KeyFrame& kf, int64_t bound) {
  if (m.profiling) CK(&m, cudaEventRecord(m.ev[1], m.stream));
  if (m.prm.sensor_model == 1) {  // counting model, Eq. (alpha): the block of each point's voxel
    NvtxRange range("sbki: counting model (a4, a5)");
    CK(&m, launch_touch_cells(m, bound));
    CK(&m, launch_commit_blocks(m));
    if (m.profiling) CK(&m, cudaEventRecord(m.ev[2], m.stream));
    CK(&m, launch_accumulate_counts(m, bound));
    if (m.profiling) CK(&m, cudaEventRecord(m.ev[3], m.stream));
    return SBKI_OK;
  }
  {
    NvtxRange range("sbki: touched blocks (a4)");
    CK(&m, launch_touch_blocks(m, kf, bound));
    CK(&m, launch_commit_blocks(m));
    if (m.acc_mode == 1) CK(&m, launch_bin_points(m, bound));
  }
  if (m.profiling) CK(&m, cudaEventRecord(m.ev[2], m.stream));
  {
    NvtxRange range("sbki: accumulation (a5)");
    if (m.g.lscaled && fast_form_ready(m)) {  // per-class l: the fast form for the classes it has tables of
      CK(&m, launch_accumulate_points(m));
      const uint32_t all = m.g.K1 >= 32 ? 0xffffffffu : (1u << m.g.K1) - 1u;
      if ((m.ftab_classes & all) != all) CK(&m, launch_accumulate_weighted(m, false, false, m.ftab_classes));
    } else if (m.g.lscaled || (m.soft && !fast_form_ready(m))) {  // the weighted form alone
      CK(&m, launch_accumulate_weighted(m, m.soft));
    } else if (m.acc_mode == 1) {
      CK(&m, launch_accumulate(m, kf));
    } else {
      CK(&m, launch_accumulate_points(m));
    }
  }
  if (m.profiling) CK(&m, cudaEventRecord(m.ev[3], m.stream));
  return SBKI_OK;
}

// after a synchronising read: add the stage times of a finished update (its events ev[0..3])
void profile_collect(MapState& m, const cudaEvent_t* ev) {
  if (!m.profiling) return;
  float t01 = 0.f, t12 = 0.f, t23 = 0.f;
  if (cudaEventElapsedTime(&t01, ev[0], ev[1]) != cudaSuccess ||
      cudaEventElapsedTime(&t12, ev[1], ev[2]) != cudaSuccess ||
      cudaEventElapsedTime(&t23, ev[2], ev[3]) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  m.prof.inserts += 1;
  m.prof.ingest_ms += t01;
  m.prof.blocks_ms += t12;
  m.prof.accumulate_ms += t23;
}

sbki_status insert_scan_impl(sbki_map* map, const float* points, const int32_t* labels, int64_t n,
                             const double pose[16], bool sync_end, sbki_stats* stats, const float* probs = nullptr) {
  if (!map) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  MapState& m = map->st;
  if (n < 0 || (n > 0 && (!points || (!labels && !probs))) || !pose)
    return fail(&m, SBKI_ERR_INVALID_ARG, "need n >= 0, points/labels non-NULL for n > 0, pose non-NULL");
  if (n > (1ll << 26)) return fail(&m, SBKI_ERR_INVALID_ARG, "n too large");
  DeviceGuard dg(m.device);
  if (n == 0) {
    if (stats) {
      *stats = sbki_stats{};
      stats->total_blocks = m.host_blocks;
    }
    return SBKI_OK;
  }
  KeyFrame kf;
  int64_t nitems = 0;
  sbki_status st = run_ingest(m, points, labels, n, pose, kf, &nitems, m.active_map, probs);
  if (st != SBKI_OK) {
    fill_stats(m, n, &m.last_stats);
    if (stats) *stats = m.last_stats;
    return st;
  }
  if (nitems > 0) {
    m.soft = probs != nullptr;
    st = run_update(m, kf, nitems);
    m.soft = false;
    if (st != SBKI_OK) return st;
  }
  if (!sync_end) {
    // the stage times are read at the next synchronising call, from the other set of events
    if (nitems > 0 && m.profiling) {
      std::swap(m.ev, m.ev_alt);
      m.prof_pending = true;
    }
    return SBKI_OK;
  }
  st = read_counters(m);
  if (st != SBKI_OK) return st;
  if (nitems > 0 && m.hc->err == 0) profile_collect(m, m.ev);
  m.host_blocks = m.hc->n_blocks;
  fill_stats(m, n, &m.last_stats);
  if (stats) *stats = m.last_stats;
  return status_from_device(m);
}

}  // namespace

namespace sbki {
// Shared with entry points defined in other translation units.
sbki_status validate_params(const sbki_params* p) { return check_params(p); }
Geom geometry_of(const sbki_params& p) { return make_geom(p); }
KeyFrame frame_of_scan(const MapState& m, const double T[16]) { return scan_frame(m, T); }
void tighten_frame(const Geom& g, const int32_t tbox[6], const double T[16], KeyFrame& kf) {
  fit_frame_to_box(g, tbox, T, kf);
}
void set_global_error(const char* msg) { snprintf(g_create_error, sizeof(g_create_error), "%s", msg); }
}  // namespace sbki

extern "C" {

sbki_status sbki_default_params(sbki_params* p) {
  if (!p) return SBKI_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->res = 0.1;
  p->length_scale = 0.3;
  p->sigma0 = 0.1;
  p->alpha0 = 0.001;
  p->free_step = 0.3;
  p->ds_res = 0.0;
  p->min_range = 0.0;
  p->max_range = 50.0;
  p->free_thresh = 0.47;
  p->occ_thresh = 0.6;
  p->num_classes = 10;
  p->block_edge = 8;
  p->pool_blocks = 1 << 16;
  p->sample_capacity = 1 << 24;
  p->track_pairs = 0;
  p->device = 0;
  p->accumulate_mode = 0;
  p->num_maps = 1;
  p->cuda_stream = nullptr;
  p->sensor_model = 0;
  for (int k = 0; k < 32; ++k) p->sigma0_scale[k] = 1.0;
  p->association = 0;
  for (int k = 0; k < 32; ++k) p->l_scale[k] = 1.0;
  return SBKI_OK;
}

sbki_status sbki_create_map(const sbki_params* params, sbki_map** out) {
  if (!out) return fail(nullptr, SBKI_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  sbki_status st = check_params(params);
  if (st != SBKI_OK) return st;
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || params->device < 0 || params->device >= ndev)
    return fail(nullptr, SBKI_ERR_CUDA, "no CUDA device %d (%s)", params->device,
                ce != cudaSuccess ? cudaGetErrorString(ce) : "out of range");
  sbki_map* map = new (std::nothrow) sbki_map();
  if (!map) return fail(nullptr, SBKI_ERR_CAPACITY, "host allocation failed");
  MapState& m = map->st;
  m.prm = *params;
  m.device = params->device;
  m.stream = (cudaStream_t)params->cuda_stream;
  m.g = make_geom(m.prm);
  m.acc_mode = params->accumulate_mode;
  DeviceGuard dg(m.device);
  auto bail = [&](const char* what, cudaError_t e) {
    snprintf(g_create_error, sizeof(g_create_error), "%s: %s", what, cudaGetErrorString(e));
    sbki_destroy_map(map);
    return SBKI_ERR_CUDA;
  };
  cudaDeviceProp prop;
  if ((ce = cudaGetDeviceProperties(&prop, m.device)) != cudaSuccess) return bail("cudaGetDeviceProperties", ce);
  m.sm_count = prop.multiProcessorCount;
  m.pool_blocks = params->pool_blocks;
  m.hash_cap = 1024;
  while (m.hash_cap < 2 * m.pool_blocks) m.hash_cap <<= 1;
  const size_t blk = (size_t)m.g.K1 * m.g.B3;
  if ((ce = dalloc(&m.hkeys, m.hash_cap)) != cudaSuccess) return bail("hash keys", ce);
  if ((ce = dalloc(&m.hvals, m.hash_cap)) != cudaSuccess) return bail("hash values", ce);
  if ((ce = dalloc(&m.hmark, m.hash_cap)) != cudaSuccess) return bail("hash marks", ce);
  if ((ce = dalloc(&m.hcnt, m.hash_cap)) != cudaSuccess) return bail("block point counts", ce);
  if ((ce = dalloc(&m.hcur, m.hash_cap)) != cudaSuccess) return bail("block cursors", ce);
  if ((ce = dalloc(&m.boff, m.hash_cap + 1)) != cudaSuccess) return bail("block offsets", ce);
  m.list_cap = std::min<int64_t>(4 * params->sample_capacity, (1ll << 31) - 1);
  if ((ce = dalloc(&m.blist, m.list_cap)) != cudaSuccess) return bail("block point lists", ce);
  // one spare block after the pool: the point-major accumulation points the
  // neighbour blocks a point's ball cannot reach at it (nothing reads it)
  if ((ce = dalloc(&m.alpha, (size_t)(m.pool_blocks + 1) * blk)) != cudaSuccess) return bail("alpha pool", ce);
  if ((ce = dalloc(&m.pool_keys, m.pool_blocks)) != cudaSuccess) return bail("pool keys", ce);
  if (params->track_pairs)
    if ((ce = dalloc(&m.pairs, (size_t)(m.pool_blocks + 1) * m.g.B3)) != cudaSuccess) return bail("pair counts", ce);
  if ((ce = dalloc(&m.dc, 1)) != cudaSuccess) return bail("counters", ce);
  if ((ce = cudaMallocHost((void**)&m.hc, sizeof(DevCounters))) != cudaSuccess) return bail("host counters", ce);
  Scratch& s = m.s;
  const int64_t S = params->sample_capacity;
  s.s_cap = S;
  if ((ce = dalloc(&s.items, S)) != cudaSuccess) return bail("items", ce);
  if ((ce = dalloc(&s.sitems, S)) != cudaSuccess) return bail("sorted items", ce);
  if ((ce = dalloc(&s.keys, S)) != cudaSuccess) return bail("keys", ce);
  if ((ce = dalloc(&s.keys2, S)) != cudaSuccess) return bail("keys2", ce);
  if ((ce = dalloc(&s.vals, S)) != cudaSuccess) return bail("vals", ce);
  if ((ce = dalloc(&s.vals2, S)) != cudaSuccess) return bail("vals2", ce);
  if ((ce = dalloc(&s.flags, std::max<int64_t>(S + 1, 2 * seg_tiles(S) + 2))) != cudaSuccess) return bail("flags", ce);
  if ((ce = dalloc(&s.seg_start, S + 1)) != cudaSuccess) return bail("seg_start", ce);
  if ((ce = dalloc(&s.train, S)) != cudaSuccess) return bail("train", ce);
  s.hist_cap = radix_hist_entries(S);
  if ((ce = dalloc(&s.hist, s.hist_cap)) != cudaSuccess) return bail("histogram", ce);
  const int64_t scan_n = std::max<int64_t>(std::max<int64_t>(s.hist_cap, S + 1), (int64_t)1 << 27);
  if ((ce = cudaMalloc(&s.scan_tmp, scan_tmp_bytes(scan_n))) != cudaSuccess) return bail("scan partials", ce);
  if ((ce = dalloc(&s.touched, m.hash_cap)) != cudaSuccess) return bail("touched list", ce);
  if ((ce = dalloc(&s.bbox, 8)) != cudaSuccess) return bail("bbox", ce);
  if ((ce = dalloc(&s.slow, S + 2)) != cudaSuccess) return bail("slow cells", ce);
  if ((ce = cudaMalloc(&s.carry, (size_t)kSegCarryBytes * 2 * seg_tiles(S))) != cudaSuccess)
    return bail("segment carries", ce);
  if ((ce = dalloc(&s.desc, kMaxScans + 1)) != cudaSuccess) return bail("scan descriptors", ce);
  if ((ce = cudaMallocHost((void**)&m.hdesc, sizeof(ScanDesc) * (kMaxScans + 1))) != cudaSuccess)
    return bail("host scan descriptors", ce);
  if ((ce = dalloc(&s.fresh, m.hash_cap)) != cudaSuccess) return bail("fresh list", ce);
  if ((ce = cudaMemsetAsync(m.hkeys, 0xff, sizeof(unsigned long long) * m.hash_cap, m.stream)) != cudaSuccess)
    return bail("hash init", ce);
  if ((ce = cudaMemsetAsync(m.hmark, 0, sizeof(uint32_t) * m.hash_cap, m.stream)) != cudaSuccess)
    return bail("mark init", ce);
  if ((ce = cudaMemsetAsync(m.hcnt, 0, sizeof(uint32_t) * m.hash_cap, m.stream)) != cudaSuccess)
    return bail("count init", ce);
  if ((ce = cudaMemsetAsync(m.dc, 0, sizeof(DevCounters), m.stream)) != cudaSuccess) return bail("counters init", ce);
  for (int i = 0; i < 4; ++i)
    if ((ce = cudaEventCreate(&m.ev[i])) != cudaSuccess || (ce = cudaEventCreate(&m.ev_alt[i])) != cudaSuccess)
      return bail("events", ce);
  if ((ce = build_candidate_tables(m)) != cudaSuccess) return bail("candidate tables", ce);
  if (m.ftab) {
    if ((ce = dalloc(&m.nbrslot, (size_t)m.hash_cap * 32)) != cudaSuccess) return bail("neighbour slot table", ce);
    if ((ce = dalloc(&m.s.ownslot, S)) != cudaSuccess) return bail("own block slots", ce);
    if ((ce = cudaMemsetAsync(m.nbrslot, 0, sizeof(uint32_t) * (size_t)m.hash_cap * 32, m.stream)) != cudaSuccess)
      return bail("neighbour slot init", ce);
  }
  if ((ce = cudaStreamSynchronize(m.stream)) != cudaSuccess) return bail("create sync", ce);
  std::memset(m.hc, 0, sizeof(DevCounters));
  *out = map;
  return SBKI_OK;
}

void sbki_destroy_map(sbki_map* map) {
  if (!map) return;
  MapState& m = map->st;
  {
    DeviceGuard dg(m.device);
    if (m.stream || m.dc) cudaStreamSynchronize(m.stream);
    void* ptrs[] = {m.clen, m.ftab, m.flen, m.nbrslot, m.s.ownslot, m.s.probs, m.s.hit_src, m.s.softidx, m.s.wsoft, m.gpool, m.dacc, m.ctab, m.hkeys, m.hvals, m.hmark, m.hcnt, m.hcur, m.boff, m.blist, m.alpha, m.pool_keys, m.pairs, m.dc, m.s.items, m.s.sitems, m.s.keys, m.s.keys2,
                    m.s.vals, m.s.vals2, m.s.flags, m.s.seg_start, m.s.train, m.s.hist, m.s.scan_tmp, m.s.touched, m.s.fresh, m.s.bbox, m.s.slow, m.s.carry,
                    m.s.desc};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    free_scratch_points(m.s);
    if (m.hc) cudaFreeHost(m.hc);
    if (m.hdesc) cudaFreeHost(m.hdesc);
    for (int i = 0; i <= kMaxScans; ++i)
      if (m.batch_exec[i]) cudaGraphExecDestroy(m.batch_exec[i]);
    if (m.rec_stream) cudaStreamDestroy(m.rec_stream);
    for (int i = 0; i < 4; ++i) {
      if (m.ev[i]) cudaEventDestroy(m.ev[i]);
      if (m.ev_alt[i]) cudaEventDestroy(m.ev_alt[i]);
    }
  }
  delete map;
}

sbki_status sbki_insert_scan(sbki_map* map, const float* points, const int32_t* labels, int64_t n,
                             const double sensor_pose[16], sbki_stats* stats) {
  return insert_scan_impl(map, points, labels, n, sensor_pose, true, stats);
}

sbki_status sbki_insert_scan_soft(sbki_map* map, const float* points, const float* probs, int64_t n,
                                  const double sensor_pose[16], sbki_stats* stats) {
  if (!map) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  MapState& m = map->st;
  if (m.prm.sensor_model != 0 || m.acc_mode != 0 || m.prm.association != 0 || m.g.lscaled)
    return fail(&m, SBKI_ERR_INVALID_ARG,
                "soft labels need the kernel model, accumulate_mode 0, association 0 and the common l");
  if (n > 0 && !probs) return fail(&m, SBKI_ERR_INVALID_ARG, "probs is NULL");
  return insert_scan_impl(map, points, nullptr, n, sensor_pose, true, stats, probs);
}

sbki_status sbki_training_set_soft(sbki_map* map, const float* points, const float* probs, int64_t n,
                                   const double sensor_pose[16], float* xyz_out, float* w_out, int64_t cap,
                                   int64_t* count) {
  if (!map) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  MapState& m = map->st;
  if (n < 0 || (n > 0 && (!points || !probs)) || !sensor_pose || !count || cap < 0 ||
      (cap > 0 && (!xyz_out || !w_out)))
    return fail(&m, SBKI_ERR_INVALID_ARG, "bad arguments");
  DeviceGuard dg(m.device);
  *count = 0;
  if (n == 0) return SBKI_OK;
  KeyFrame kf;
  int64_t nitems = 0;
  sbki_status st = run_ingest(m, points, nullptr, n, sensor_pose, kf, &nitems, 0, probs);
  if (st != SBKI_OK) return st;
  st = read_counters(m);
  if (st != SBKI_OK) return st;
  if (m.hc->err != 0) return status_from_device(m);
  const int64_t P = nitems > 0 ? m.hc->n_train : 0;
  *count = P;
  const int64_t c = std::min(P, cap);
  if (c > 0) {
    const bool dev = is_device_ptr(xyz_out) && is_device_ptr(w_out);
    float *dx = xyz_out, *dw = w_out;
    TmpFree tf;
    tf.st = m.stream;
    if (!dev) {
      CK(&m, cudaMalloc(&tf.p[0], sizeof(float) * 3 * c));
      CK(&m, cudaMalloc(&tf.p[1], sizeof(float) * m.g.K1 * c));
      dx = static_cast<float*>(tf.p[0]);
      dw = static_cast<float*>(tf.p[1]);
    }
    CK(&m, launch_soft_export(m, dx, dw, c));
    if (!dev) {
      CK(&m, cudaMemcpyAsync(xyz_out, dx, sizeof(float) * 3 * c, cudaMemcpyDeviceToHost, m.stream));
      CK(&m, cudaMemcpyAsync(w_out, dw, sizeof(float) * m.g.K1 * c, cudaMemcpyDeviceToHost, m.stream));
    }
    CK(&m, cudaStreamSynchronize(m.stream));
  }
  if (P > cap) return fail(&m, SBKI_ERR_CAPACITY, "training set has %lld points, cap %lld", (long long)P,
                           (long long)cap);
  return SBKI_OK;
}

sbki_status sbki_get_tuning(const sbki_map* map, sbki_tuning* out) {
  if (!map || !out) return fail(nullptr, SBKI_ERR_INVALID_ARG, "bad arguments");
  *out = map->st.tune;
  return SBKI_OK;
}

sbki_status sbki_set_tuning(sbki_map* map, const sbki_tuning* t) {
  if (!map || !t) return fail(nullptr, SBKI_ERR_INVALID_ARG, "bad arguments");
  MapState& m = map->st;
  if (t->accumulate_ctas_per_sm < 0 || t->accumulate_ctas_per_sm > 32 || t->accumulate_chunk < 1 ||
      t->accumulate_chunk > 64 || t->touch_ctas_per_sm < 1 || t->touch_ctas_per_sm > 64 || t->ingest_ctas_per_sm < 1 ||
      t->ingest_ctas_per_sm > 64)
    return fail(&m, SBKI_ERR_INVALID_ARG, "tuning out of range");
  DeviceGuard dg(m.device);
  CK(&m, cudaStreamSynchronize(m.stream));
  m.tune = *t;
  for (int i = 0; i <= kMaxScans; ++i)
    if (m.batch_exec[i]) {
      cudaGraphExecDestroy(m.batch_exec[i]);
      m.batch_exec[i] = nullptr;
    }
  return SBKI_OK;
}

sbki_status sbki_select_map(sbki_map* map, int32_t map_id) {
  if (!map) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  MapState& m = map->st;
  if (map_id < 0 || map_id >= m.prm.num_maps)
    return fail(&m, SBKI_ERR_INVALID_ARG, "map_id %d outside 0..%d", map_id, m.prm.num_maps - 1);
  m.active_map = map_id;
  return SBKI_OK;
}

sbki_status sbki_insert_batch(sbki_map* map, const sbki_scan* scans, int32_t count, sbki_stats* stats) {
  NvtxRange range("sbki: batched update (a9)");
  if (!map) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  MapState& m = map->st;
  if (!scans || count < 1 || count > kMaxScans)
    return fail(&m, SBKI_ERR_INVALID_ARG, "need 1 <= count <= %d scans", kMaxScans);
  int64_t total = 0;
  for (int i = 0; i < count; ++i) {
    const sbki_scan& sc = scans[i];
    if (sc.n < 0 || (sc.n > 0 && (!sc.points || !sc.labels)))
      return fail(&m, SBKI_ERR_INVALID_ARG, "scan %d: need n >= 0 and points/labels for n > 0", i);
    if (sc.map_id < 0 || sc.map_id >= m.prm.num_maps)
      return fail(&m, SBKI_ERR_INVALID_ARG, "scan %d: map_id %d outside 0..%d", i, sc.map_id, m.prm.num_maps - 1);
    for (int k = 0; k < 16; ++k)
      if (!std::isfinite(sc.pose[k])) return fail(&m, SBKI_ERR_INVALID_ARG, "scan %d: non-finite pose", i);
    for (int a = 0; a < 3; ++a)
      if ((std::fabs(sc.pose[4 * a + 3]) + m.prm.max_range) / m.prm.res > (double)(kKeyLimit - 1024))
        return fail(&m, SBKI_ERR_INVALID_ARG, "scan %d: sensor origin too far from the map origin", i);
    total += sc.n;
  }
  if (total > (1ll << 26)) return fail(&m, SBKI_ERR_INVALID_ARG, "too many points in one batch");
  DeviceGuard dg(m.device);
  if (total == 0) {
    if (stats) {
      *stats = sbki_stats{};
      stats->total_blocks = m.host_blocks;
    }
    return SBKI_OK;
  }
  sbki_status st = ensure_point_capacity(m, total);
  if (st != SBKI_OK) return st;
  // descriptors; host inputs are staged into the map's point buffers (outside the recording)
  KeyFrame kf = scan_frame(m, scans[0].pose);
  kf.scan_bits = count > 1 ? ceil_log2(count) : 0;
  if (kf.total_bits + kf.scan_bits > 64) return fail(&m, SBKI_ERR_INVALID_ARG, "batch keys do not fit 64 bits");
  int64_t off = 0;
  for (int i = 0; i < count; ++i) {
    const sbki_scan& sc = scans[i];
    const float* dp = sc.points;
    const int32_t* dl = sc.labels;
    if (sc.n > 0 && !is_device_ptr(sc.points)) {
      CK(&m, cudaMemcpyAsync(m.s.pts + 3 * off, sc.points, sizeof(float) * 3 * sc.n, cudaMemcpyHostToDevice,
                             m.stream));
      dp = m.s.pts + 3 * off;
    }
    if (sc.n > 0 && !is_device_ptr(sc.labels)) {
      CK(&m, cudaMemcpyAsync(m.s.labels + off, sc.labels, sizeof(int32_t) * sc.n, cudaMemcpyHostToDevice, m.stream));
      dl = m.s.labels + off;
    }
    fill_desc(m.hdesc[i], dp, dl, sc.n, off, sc.pose, scan_frame(m, sc.pose), sc.map_id);
    off += sc.n;
  }
  m.hdesc[count] = ScanDesc{};
  m.hdesc[count].off = total;
  CK(&m, cudaMemcpyAsync(m.s.desc, m.hdesc, sizeof(ScanDesc) * (count + 1), cudaMemcpyHostToDevice, m.stream));
  // the stage sequence, recorded once per scan count (every size it depends on is read on the device)
  if (!m.batch_exec[count] || m.batch_gen[count] != m.scratch_gen) {
    if (m.batch_exec[count]) {
      cudaGraphExecDestroy(m.batch_exec[count]);
      m.batch_exec[count] = nullptr;
    }
    // recorded on a private stream (the legacy default stream cannot be captured),
    // launched on the map's stream
    if (!m.rec_stream) CK(&m, cudaStreamCreateWithFlags(&m.rec_stream, cudaStreamNonBlocking));
    const bool prof = m.profiling;
    const int64_t l0 = m.launches;
    const cudaStream_t user_stream = m.stream;
    m.profiling = false;
    m.stream = m.rec_stream;
    {
      const cudaError_t be = cudaStreamBeginCapture(m.stream, cudaStreamCaptureModeThreadLocal);
      if (be != cudaSuccess) {
        m.stream = user_stream;
        m.profiling = prof;
        return fail(&m, SBKI_ERR_CUDA, "recording the batched update failed: %s", cudaGetErrorString(be));
      }
    }
    batch_begin_kernel<<<1, 1, 0, m.stream>>>(m.dc, m.s.desc, count);
    m.launches += 1;
    cudaError_t ce = launch_transform_count(m, count, m.s.n_cap);
    if (ce == cudaSuccess) ce = launch_emit(m, count, m.s.n_cap, kf);
    if (ce == cudaSuccess) ce = launch_downsample_n(m, kf, m.s.s_cap);
    sbki_status ust = SBKI_OK;
    if (ce == cudaSuccess) ust = run_update(m, kf, m.s.s_cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(m.stream, &graph);
    m.stream = user_stream;
    m.profiling = prof;
    if (ce != cudaSuccess || ee != cudaSuccess || ust != SBKI_OK) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return fail(&m, SBKI_ERR_CUDA, "recording the batched update failed: %s",
                  cudaGetErrorString(ce != cudaSuccess ? ce : ee));
    }
    ce = cudaGraphInstantiate(&m.batch_exec[count], graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      m.batch_exec[count] = nullptr;
      return fail(&m, SBKI_ERR_CUDA, "instantiating the batched update failed: %s", cudaGetErrorString(ce));
    }
    m.batch_kernels[count] = m.launches - l0;
    m.launches = l0;
    m.batch_gen[count] = m.scratch_gen;
  }
  m.epoch += 1;  // the recording advances the device epoch
  if (m.profiling) CK(&m, cudaEventRecord(m.ev[0], m.stream));
  CK(&m, cudaGraphLaunch(m.batch_exec[count], m.stream));
  m.launches += m.batch_kernels[count];
  if (m.profiling) {
    CK(&m, cudaEventRecord(m.ev[1], m.stream));
    CK(&m, cudaEventRecord(m.ev[2], m.stream));
    CK(&m, cudaEventRecord(m.ev[3], m.stream));
  }
  st = read_counters(m);
  if (st != SBKI_OK) return st;
  if (m.hc->err == 0) profile_collect(m, m.ev);
  m.host_blocks = m.hc->n_blocks;
  fill_stats(m, total, &m.last_stats);
  if (stats) *stats = m.last_stats;
  return status_from_device(m);
}

sbki_status sbki_insert_scan_async(sbki_map* map, const float* points, const int32_t* labels, int64_t n,
                                   const double sensor_pose[16]) {
  return insert_scan_impl(map, points, labels, n, sensor_pose, false, nullptr);
}

sbki_status sbki_sync(sbki_map* map, sbki_stats* stats) {
  if (!map) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  MapState& m = map->st;
  DeviceGuard dg(m.device);
  sbki_status st = read_counters(m);
  if (st != SBKI_OK) return st;
  m.host_blocks = m.hc->n_blocks;
  if (stats) {
    sbki_stats s{};
    const DevCounters& c = *m.hc;
    s.hits = c.n_valid;
    s.free_samples = (int64_t)c.n_free;
    s.train_points = c.n_train;
    s.touched_blocks = c.n_touched;
    s.new_blocks = c.err == 0 ? c.n_new : 0;
    s.pairs = (int64_t)c.pairs;
    s.touched_voxels = (int64_t)c.touched_voxels;
    s.total_blocks = c.n_blocks;
    *stats = s;
  }
  return status_from_device(m);
}

sbki_status sbki_training_set(sbki_map* map, const float* points, const int32_t* labels, int64_t n,
                              const double sensor_pose[16], float* xyzl_out, int64_t cap, int64_t* count) {
  if (!map) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  MapState& m = map->st;
  if (n < 0 || (n > 0 && (!points || !labels)) || !sensor_pose || !count || cap < 0 || (cap > 0 && !xyzl_out))
    return fail(&m, SBKI_ERR_INVALID_ARG, "bad arguments");
  DeviceGuard dg(m.device);
  *count = 0;
  if (n == 0) return SBKI_OK;
  KeyFrame kf;
  int64_t nitems = 0;
  sbki_status st = run_ingest(m, points, labels, n, sensor_pose, kf, &nitems, 0);  // labels only in the output
  if (st != SBKI_OK) return st;
  st = read_counters(m);
  if (st != SBKI_OK) return st;
  if (m.hc->err != 0) return status_from_device(m);
  const int64_t P = nitems > 0 ? m.hc->n_train : 0;
  *count = P;
  const int64_t c = std::min(P, cap);
  if (c > 0) {
    CK(&m, cudaMemcpyAsync(xyzl_out, m.s.train, sizeof(float4) * c, cudaMemcpyDefault, m.stream));
    CK(&m, cudaStreamSynchronize(m.stream));
  }
  if (P > cap) return fail(&m, SBKI_ERR_CAPACITY, "training set has %lld points, cap %lld", (long long)P,
                           (long long)cap);
  return SBKI_OK;
}

sbki_status sbki_insert_training(sbki_map* map, const float* xyzl, int64_t p, sbki_stats* stats) {
  if (!map) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  MapState& m = map->st;
  if (p < 0 || (p > 0 && !xyzl)) return fail(&m, SBKI_ERR_INVALID_ARG, "bad arguments");
  if (p > m.s.s_cap) return fail(&m, SBKI_ERR_CAPACITY, "training set larger than sample_capacity");
  DeviceGuard dg(m.device);
  if (p == 0) {
    if (stats) *stats = sbki_stats{};
    return SBKI_OK;
  }
  const float4* din = reinterpret_cast<const float4*>(xyzl);
  if (!is_device_ptr(xyzl)) {
    CK(&m, cudaMemcpyAsync(m.s.items, xyzl, sizeof(float4) * p, cudaMemcpyHostToDevice, m.stream));
    din = m.s.items;
  } else if ((reinterpret_cast<uintptr_t>(xyzl) & 15u) != 0) {
    CK(&m, cudaMemcpyAsync(m.s.items, xyzl, sizeof(float4) * p, cudaMemcpyDeviceToDevice, m.stream));
    din = m.s.items;
  }
  m.epoch += 1;
  if (m.profiling) CK(&m, cudaEventRecord(m.ev[0], m.stream));
  begin_kernel<<<1, 1, 0, m.stream>>>(m.dc, m.epoch, 0u);
  m.launches += 1;
  int* bbox = m.s.bbox;
  sbki_status st = SBKI_OK;
  bbox_init_kernel<<<1, 32, 0, m.stream>>>(bbox);
  m.launches += 1;
  CK(&m, launch_train_bbox(m, din, p, bbox));
  int hb[6];
  CK(&m, cudaMemcpyAsync(hb, bbox, sizeof(hb), cudaMemcpyDeviceToHost, m.stream));
  st = read_counters(m);
  if (st != SBKI_OK) return st;
  if (m.hc->err != 0) return status_from_device(m);
  KeyFrame kf;
  int64_t ext = 1;
  for (int a = 0; a < 3; ++a) {
    kf.org[a] = hb[a];
    ext = std::max<int64_t>(ext, (int64_t)hb[3 + a] - hb[a] + 1);
  }
  kf.bits[0] = kf.bits[1] = kf.bits[2] = std::max(1, ceil_log2(ext));
  kf.total_bits = kf.bits[0] + kf.bits[1] + kf.bits[2] + kLocalBits + m.g.label_bits;
  if (kf.total_bits > 64) return fail(&m, SBKI_ERR_INVALID_ARG, "training set spans too large a region");
  set_items_kernel<<<1, 1, 0, m.stream>>>(m.dc, (uint32_t)p);
  m.launches += 1;
  CK(&m, launch_train_prepare(m, din, p, kf));
  st = run_update(m, kf, p);
  if (st != SBKI_OK) return st;
  st = read_counters(m);
  if (st != SBKI_OK) return st;
  if (m.hc->err == 0) profile_collect(m, m.ev);
  m.host_blocks = m.hc->n_blocks;
  fill_stats(m, 0, &m.last_stats);
  m.last_stats.hits = 0;
  m.last_stats.dropped = 0;
  m.last_stats.free_samples = 0;
  if (stats) *stats = m.last_stats;
  return status_from_device(m);
}

sbki_status sbki_query_probs(const sbki_map* cmap, const float* xyz, int64_t q, float* probs, float* var,
                             float* mode, int32_t* label, float* p_occ, int32_t* state) {
  NvtxRange range("sbki: read-off (a6)");
  if (!cmap) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  sbki_map* map = const_cast<sbki_map*>(cmap);
  MapState& m = map->st;
  if (q < 0 || (q > 0 && (!xyz || !probs))) return fail(&m, SBKI_ERR_INVALID_ARG, "bad arguments");
  if (q == 0) return SBKI_OK;
  DeviceGuard dg(m.device);
  const int K1 = m.g.K1;
  const bool dev_all = is_device_ptr(xyz) && is_device_ptr(probs) && (!var || is_device_ptr(var)) &&
                       (!mode || is_device_ptr(mode)) &&
                       (!label || is_device_ptr(label)) && (!p_occ || is_device_ptr(p_occ)) &&
                       (!state || is_device_ptr(state));
  if (dev_all) {
    CK(&m, launch_query(m, xyz, q, probs, var, mode, label, p_occ, state));
    m.launches += 1;
    CK(&m, cudaStreamSynchronize(m.stream));
    return SBKI_OK;
  }
  // stage through device temporaries
  float *dx = nullptr, *dp = nullptr, *dv = nullptr, *dm = nullptr, *dpo = nullptr;
  int32_t *dl = nullptr, *ds = nullptr;
  sbki_status rs = SBKI_OK;
  cudaError_t e = cudaSuccess;
  do {
    if ((e = dalloc(&dx, 3 * q)) != cudaSuccess) break;
    if ((e = dalloc(&dp, (size_t)K1 * q)) != cudaSuccess) break;
    if (var && (e = dalloc(&dv, (size_t)K1 * q)) != cudaSuccess) break;
    if (mode && (e = dalloc(&dm, (size_t)K1 * q)) != cudaSuccess) break;
    if (label && (e = dalloc(&dl, q)) != cudaSuccess) break;
    if (p_occ && (e = dalloc(&dpo, q)) != cudaSuccess) break;
    if (state && (e = dalloc(&ds, q)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(dx, xyz, sizeof(float) * 3 * q, cudaMemcpyDefault, m.stream)) != cudaSuccess) break;
    if ((e = launch_query(m, dx, q, dp, dv, dm, dl, dpo, ds)) != cudaSuccess) break;
    m.launches += 1;
    if ((e = cudaMemcpyAsync(probs, dp, sizeof(float) * K1 * q, cudaMemcpyDefault, m.stream)) != cudaSuccess) break;
    if (var && (e = cudaMemcpyAsync(var, dv, sizeof(float) * K1 * q, cudaMemcpyDefault, m.stream)) != cudaSuccess)
      break;
    if (mode && (e = cudaMemcpyAsync(mode, dm, sizeof(float) * K1 * q, cudaMemcpyDefault, m.stream)) != cudaSuccess)
      break;
    if (label && (e = cudaMemcpyAsync(label, dl, sizeof(int32_t) * q, cudaMemcpyDefault, m.stream)) != cudaSuccess)
      break;
    if (p_occ && (e = cudaMemcpyAsync(p_occ, dpo, sizeof(float) * q, cudaMemcpyDefault, m.stream)) != cudaSuccess)
      break;
    if (state && (e = cudaMemcpyAsync(state, ds, sizeof(int32_t) * q, cudaMemcpyDefault, m.stream)) != cudaSuccess)
      break;
    e = cudaStreamSynchronize(m.stream);
  } while (0);
  if (e != cudaSuccess) rs = fail(&m, SBKI_ERR_CUDA, "query: %s", cudaGetErrorString(e));
  cudaStreamSynchronize(m.stream);
  void* tmp[] = {dx, dp, dv, dm, dl, dpo, ds};
  for (void* t : tmp)
    if (t) cudaFree(t);
  return rs;
}

sbki_status sbki_voxel_count(const sbki_map* cmap, int64_t* count) {
  if (!cmap || !count) return fail(nullptr, SBKI_ERR_INVALID_ARG, "bad arguments");
  MapState& m = const_cast<sbki_map*>(cmap)->st;
  DeviceGuard dg(m.device);
  sbki_status st = read_counters(m);
  if (st != SBKI_OK) return st;
  const int64_t nb = m.hc->n_blocks;
  if (m.prm.num_maps == 1) {
    *count = nb * m.g.B3;
    return SBKI_OK;
  }
  std::vector<unsigned long long> bkeys((size_t)nb);
  if (nb > 0) {
    CK(&m, cudaMemcpyAsync(bkeys.data(), m.pool_keys, sizeof(unsigned long long) * nb, cudaMemcpyDeviceToHost,
                           m.stream));
    CK(&m, cudaStreamSynchronize(m.stream));
  }
  int64_t mine = 0;
  for (unsigned long long k : bkeys) mine += map_of_block(k) == m.active_map ? 1 : 0;
  *count = mine * m.g.B3;
  return SBKI_OK;
}

sbki_status sbki_export_blocks(const sbki_map* cmap, int64_t* keys, float* alpha, int64_t cap, int64_t* count) {
  if (!cmap || !count || cap < 0) return fail(nullptr, SBKI_ERR_INVALID_ARG, "bad arguments");
  MapState& m = const_cast<sbki_map*>(cmap)->st;
  DeviceGuard dg(m.device);
  sbki_status st = read_counters(m);
  if (st != SBKI_OK) return st;
  const uint32_t nb = m.hc->n_blocks;
  *count = 0;
  if (nb == 0) return SBKI_OK;
  uint32_t* rowb = m.boff;  // [hash_cap + 1] >= nb + 1 (free between updates)
  CK(&m, launch_export_rows(m, nb, rowb, m.s.scan_tmp, nullptr, nullptr));
  uint32_t nsel = 0;
  CK(&m, cudaMemcpyAsync(&nsel, rowb + nb, sizeof(nsel), cudaMemcpyDeviceToHost, m.stream));
  CK(&m, cudaStreamSynchronize(m.stream));
  *count = (int64_t)nsel * m.g.B3;
  if (!keys && !alpha) return SBKI_OK;
  if (cap < *count)
    return fail(&m, SBKI_ERR_CAPACITY, "export needs %lld rows, cap %lld", (long long)*count, (long long)cap);
  const bool dk = !keys || is_device_ptr(keys), da = !alpha || is_device_ptr(alpha);
  TmpFree tf;
  tf.st = m.stream;
  int64_t* ko = keys;
  float* ao = alpha;
  if (!dk) {
    CK(&m, cudaMalloc(&tf.p[0], sizeof(int64_t) * 3 * *count));
    ko = static_cast<int64_t*>(tf.p[0]);
  }
  if (!da) {
    CK(&m, cudaMalloc(&tf.p[1], sizeof(float) * m.g.K1 * *count));
    ao = static_cast<float*>(tf.p[1]);
  }
  CK(&m, launch_export_rows(m, nb, rowb, m.s.scan_tmp, ko, ao));
  if (!dk) CK(&m, cudaMemcpyAsync(keys, ko, sizeof(int64_t) * 3 * *count, cudaMemcpyDeviceToHost, m.stream));
  if (!da) CK(&m, cudaMemcpyAsync(alpha, ao, sizeof(float) * m.g.K1 * *count, cudaMemcpyDeviceToHost, m.stream));
  CK(&m, cudaStreamSynchronize(m.stream));
  return SBKI_OK;
}

sbki_status sbki_export(const sbki_map* cmap, int64_t* keys, float* alpha, int32_t* pairs, int64_t cap,
                        int64_t* count) {
  if (!cmap || !count) return fail(nullptr, SBKI_ERR_INVALID_ARG, "bad arguments");
  MapState& m = const_cast<sbki_map*>(cmap)->st;
  if (pairs && !m.pairs) return fail(&m, SBKI_ERR_INVALID_ARG, "pairs requested but track_pairs is off");
  DeviceGuard dg(m.device);
  sbki_status st = read_counters(m);
  if (st != SBKI_OK) return st;
  const int64_t nb = m.hc->n_blocks;
  const int B = m.g.B, B3 = m.g.B3, K1 = m.g.K1;
  std::vector<unsigned long long> bkeys((size_t)nb);
  if (nb > 0) {
    CK(&m, cudaMemcpyAsync(bkeys.data(), m.pool_keys, sizeof(unsigned long long) * nb, cudaMemcpyDeviceToHost,
                           m.stream));
    CK(&m, cudaStreamSynchronize(m.stream));
  }
  std::vector<int64_t> mine;  // pool blocks of the selected map
  mine.reserve((size_t)nb);
  for (int64_t b = 0; b < nb; ++b)
    if (map_of_block(bkeys[(size_t)b]) == m.active_map) mine.push_back(b);
  *count = (int64_t)mine.size() * B3;
  if (!keys && !alpha && !pairs) return SBKI_OK;
  if (cap < *count) return fail(&m, SBKI_ERR_CAPACITY, "export needs %lld rows, cap %lld", (long long)*count,
                                (long long)cap);
  std::vector<float> a((size_t)nb * K1 * B3);
  std::vector<int32_t> pc(m.pairs ? (size_t)nb * B3 : 0);
  if (nb > 0) {
    CK(&m, cudaMemcpyAsync(a.data(), m.alpha, sizeof(float) * a.size(), cudaMemcpyDeviceToHost, m.stream));
    if (m.pairs)
      CK(&m, cudaMemcpyAsync(pc.data(), m.pairs, sizeof(int32_t) * pc.size(), cudaMemcpyDeviceToHost, m.stream));
    CK(&m, cudaStreamSynchronize(m.stream));
  }
  struct Row {
    int32_t k[3];
    int64_t src;  // pool block * B3 + local
  };
  std::vector<Row> rows(mine.size() * B3);
  for (size_t mb = 0; mb < mine.size(); ++mb) {
    const int64_t b = mine[mb];
    int32_t bx, by, bz;
    unpack_block(bkeys[(size_t)b], bx, by, bz);
    for (int li = 0; li < B3; ++li) {
      Row& r = rows[mb * B3 + li];
      r.k[0] = bx * B + li % B;
      r.k[1] = by * B + (li / B) % B;
      r.k[2] = bz * B + li / (B * B);
      r.src = b * B3 + li;
    }
  }
  std::sort(rows.begin(), rows.end(), [](const Row& x, const Row& y) {
    if (x.k[0] != y.k[0]) return x.k[0] < y.k[0];
    if (x.k[1] != y.k[1]) return x.k[1] < y.k[1];
    return x.k[2] < y.k[2];
  });
  const float a0 = (float)m.prm.alpha0;
  for (size_t i = 0; i < rows.size(); ++i) {
    const Row& r = rows[i];
    if (keys)
      for (int d = 0; d < 3; ++d) keys[3 * i + d] = r.k[d];
    if (alpha) {
      const int64_t b = r.src / B3, li = r.src % B3;
      for (int k = 0; k < K1; ++k) alpha[i * K1 + k] = a0 + a[(size_t)((b * K1 + k) * B3 + li)];
    }
    if (pairs) pairs[i] = pc[(size_t)r.src];
  }
  return SBKI_OK;
}

sbki_status sbki_profile(sbki_map* map, int32_t enable, int32_t reset) {
  if (!map) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  map->st.profiling = enable != 0;
  if (reset) {
    const int64_t l = map->st.prof.launches;
    map->st.prof = sbki_profile_data{};
    map->st.prof.launches = l;
    map->st.prof_pending = false;  // an asynchronous update issued before the reset is not counted
  }
  return SBKI_OK;
}

sbki_status sbki_profile_read(const sbki_map* map, sbki_profile_data* out) {
  if (!map || !out) return fail(nullptr, SBKI_ERR_INVALID_ARG, "bad arguments");
  *out = map->st.prof;
  out->launches = map->st.launches;
  out->readback_bytes = (int64_t)sizeof(DevCounters);
  return SBKI_OK;
}

// ---------------------------------------------------------------- differentiable form

}  // extern "C"

namespace {

// The gradient buffer (pool-shaped, like alpha) and the device accumulators, on first use.
sbki_status ensure_grad(MapState& m) {
  if (m.gpool) return SBKI_OK;
  CK(&m, dalloc(&m.gpool, (size_t)m.pool_blocks * m.g.K1 * m.g.B3));
  CK(&m, dalloc(&m.dacc, 4 + 32));
  CK(&m, cudaMemsetAsync(m.gpool, 0, sizeof(float) * (size_t)m.pool_blocks * m.g.K1 * m.g.B3, m.stream));
  return SBKI_OK;
}

// A device copy of a host or device input; `tmp` receives an allocation to free (or null).
template <typename T>
sbki_status device_input(MapState& m, const T* src, size_t count, const T** dst, void** tmp) {
  *tmp = nullptr;
  if (is_device_ptr(src)) {
    *dst = src;
    return SBKI_OK;
  }
  CK(&m, cudaMalloc(tmp, sizeof(T) * std::max<size_t>(count, 1)));
  CK(&m, cudaMemcpyAsync(*tmp, src, sizeof(T) * count, cudaMemcpyHostToDevice, m.stream));
  *dst = static_cast<const T*>(*tmp);
  return SBKI_OK;
}


}  // namespace

extern "C" {

sbki_status sbki_grad_clear(sbki_map* map) {
  if (!map) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  MapState& m = map->st;
  DeviceGuard dg(m.device);
  sbki_status st = ensure_grad(m);
  if (st != SBKI_OK) return st;
  st = read_counters(m);
  if (st != SBKI_OK) return st;
  CK(&m, cudaMemsetAsync(m.gpool, 0, sizeof(float) * (size_t)m.hc->n_blocks * m.g.K1 * m.g.B3, m.stream));
  return SBKI_OK;
}

sbki_status sbki_heldout_loglik(sbki_map* map, const float* xyz, const int32_t* labels, int64_t h,
                                int32_t accumulate_grad, double* loglik) {
  NvtxRange range("sbki: held-out log-likelihood (a7)");
  if (!map) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  MapState& m = map->st;
  if (h < 0 || (h > 0 && (!xyz || !labels)) || !loglik) return fail(&m, SBKI_ERR_INVALID_ARG, "bad arguments");
  DeviceGuard dg(m.device);
  sbki_status st = ensure_grad(m);
  if (st != SBKI_OK) return st;
  *loglik = 0.0;
  if (h == 0) return SBKI_OK;
  TmpFree tf;
  tf.st = m.stream;
  const float* dx = nullptr;
  const int32_t* dl = nullptr;
  if ((st = device_input(m, xyz, (size_t)h * 3, &dx, &tf.p[0])) != SBKI_OK) return st;
  if ((st = device_input(m, labels, (size_t)h, &dl, &tf.p[1])) != SBKI_OK) return st;
  CK(&m, cudaMemsetAsync(m.dacc, 0, sizeof(double), m.stream));
  CK(&m, cudaMemsetAsync(&m.dc->err, 0, sizeof(int32_t), m.stream));
  CK(&m, launch_heldout(m, dx, dl, h, accumulate_grad ? m.gpool : nullptr, m.dacc));
  m.launches += 1;
  CK(&m, cudaMemcpyAsync(loglik, m.dacc, sizeof(double), cudaMemcpyDeviceToHost, m.stream));
  st = read_counters(m);
  if (st != SBKI_OK) return st;
  if (m.hc->err == SBKI_ERR_LABEL_RANGE) {
    CK(&m, cudaMemsetAsync(&m.dc->err, 0, sizeof(int32_t), m.stream));
    return fail(&m, SBKI_ERR_LABEL_RANGE, "a held-out label is outside 0..K");
  }
  return status_from_device(m);
}

sbki_status sbki_grad_add_alpha(sbki_map* map, const int64_t* keys, const float* grad_alpha, int64_t count,
                                int64_t* missed) {
  if (!map) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  MapState& m = map->st;
  if (count < 0 || (count > 0 && (!keys || !grad_alpha))) return fail(&m, SBKI_ERR_INVALID_ARG, "bad arguments");
  DeviceGuard dg(m.device);
  sbki_status st = ensure_grad(m);
  if (st != SBKI_OK) return st;
  if (missed) *missed = 0;
  if (count == 0) return SBKI_OK;
  TmpFree tf;
  tf.st = m.stream;
  const int64_t* dk = nullptr;
  const float* dg2 = nullptr;
  if ((st = device_input(m, keys, (size_t)count * 3, &dk, &tf.p[0])) != SBKI_OK) return st;
  if ((st = device_input(m, grad_alpha, (size_t)count * m.g.K1, &dg2, &tf.p[1])) != SBKI_OK) return st;
  unsigned long long* dmiss = reinterpret_cast<unsigned long long*>(m.dacc + 3);
  CK(&m, cudaMemsetAsync(dmiss, 0, sizeof(unsigned long long), m.stream));
  CK(&m, launch_grad_scatter(m, dk, dg2, count, m.gpool, dmiss));
  m.launches += 1;
  unsigned long long hm = 0;
  CK(&m, cudaMemcpyAsync(&hm, dmiss, sizeof(hm), cudaMemcpyDeviceToHost, m.stream));
  CK(&m, cudaStreamSynchronize(m.stream));
  if (missed) *missed = (int64_t)hm;
  return SBKI_OK;
}

static sbki_status backward_impl(sbki_map* map, const float* xyzl, int64_t p, double* grad_l, double* grad_sigma0,
                          float* grad_xyz, double* grad_scale) {
  if (!map) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  MapState& m = map->st;
  if (p < 0 || (p > 0 && !xyzl)) return fail(&m, SBKI_ERR_INVALID_ARG, "bad arguments");
  if (m.prm.sensor_model != 0)
    return fail(&m, SBKI_ERR_INVALID_ARG, "the counting sensor model has no kernel to differentiate");
  if (m.prm.association != 0)
    return fail(&m, SBKI_ERR_INVALID_ARG, "the backward pass takes the exact association (association 0)");
  if (m.g.lscaled)
    return fail(&m, SBKI_ERR_INVALID_ARG, "the backward pass takes the common length scale (all l_scale 1)");
  DeviceGuard dg(m.device);
  sbki_status st = ensure_grad(m);
  if (st != SBKI_OK) return st;
  TmpFree tf;
  tf.st = m.stream;
  const float* dxyzl = nullptr;
  if ((st = device_input(m, xyzl, (size_t)p * 4, &dxyzl, &tf.p[0])) != SBKI_OK) return st;
  if (p > 0 && (reinterpret_cast<uintptr_t>(dxyzl) & 15u) != 0) {
    CK(&m, cudaMalloc(&tf.p[1], sizeof(float4) * (size_t)p));
    CK(&m, cudaMemcpyAsync(tf.p[1], dxyzl, sizeof(float4) * (size_t)p, cudaMemcpyDeviceToDevice, m.stream));
    dxyzl = static_cast<const float*>(tf.p[1]);
  }
  float* dgx = grad_xyz;
  if (grad_xyz && !is_device_ptr(grad_xyz)) {
    CK(&m, cudaMalloc(&tf.p[2], sizeof(float) * 3 * std::max<int64_t>(p, 1)));
    dgx = static_cast<float*>(tf.p[2]);
  }
  CK(&m, cudaMemsetAsync(m.dacc + 1, 0, 2 * sizeof(double), m.stream));
  if (grad_scale) CK(&m, cudaMemsetAsync(m.dacc + 4, 0, 32 * sizeof(double), m.stream));
  CK(&m, launch_backward(m, reinterpret_cast<const float4*>(dxyzl), p, m.gpool, m.dacc + 1, dgx,
                         grad_scale ? m.dacc + 4 : nullptr));
  m.launches += 1;
  double acc[2 + 1 + 32] = {};  // sums of G terms, the missed-key word, the per-class sums
  CK(&m, cudaMemcpyAsync(acc, m.dacc + 1, sizeof(acc), cudaMemcpyDeviceToHost, m.stream));
  if (grad_xyz && dgx != grad_xyz && p > 0)
    CK(&m, cudaMemcpyAsync(grad_xyz, dgx, sizeof(float) * 3 * p, cudaMemcpyDeviceToHost, m.stream));
  st = read_counters(m);
  if (st != SBKI_OK) return st;
  if (m.hc->err != 0) return status_from_device(m);
  const double l = m.prm.length_scale;
  if (grad_sigma0) *grad_sigma0 = acc[0];
  if (grad_l) *grad_l = m.prm.sigma0 * acc[1] / (l * l);
  if (grad_scale)
    for (int k = 0; k < m.g.K1; ++k) grad_scale[k] = m.prm.sigma0 * acc[3 + k];
  return SBKI_OK;
}

sbki_status sbki_backward(sbki_map* map, const float* xyzl, int64_t p, double* grad_l, double* grad_sigma0,
                          float* grad_xyz) {
  NvtxRange range("sbki: backward (a8)");
  return backward_impl(map, xyzl, p, grad_l, grad_sigma0, grad_xyz, nullptr);
}

sbki_status sbki_backward_scales(sbki_map* map, const float* xyzl, int64_t p, double* grad_scale) {
  if (!grad_scale) return fail(map ? &map->st : nullptr, SBKI_ERR_INVALID_ARG, "grad_scale is NULL");
  return backward_impl(map, xyzl, p, nullptr, nullptr, nullptr, grad_scale);
}

sbki_status sbki_forward_alpha(const sbki_params* params, const float* xyzl, int64_t p, int64_t* keys_out,
                               float* alpha_out, int64_t cap, int64_t* count) {
  if (!params || !count || p < 0 || (p > 0 && !xyzl)) return fail(nullptr, SBKI_ERR_INVALID_ARG, "bad arguments");
  sbki_map* map = nullptr;
  sbki_status st = sbki_create_map(params, &map);
  if (st != SBKI_OK) return st;
  st = sbki_insert_training(map, xyzl, p, nullptr);
  if (st == SBKI_OK) st = sbki_export(map, keys_out, alpha_out, nullptr, cap, count);
  if (st != SBKI_OK) snprintf(g_create_error, sizeof(g_create_error), "%s", map->st.last_error);
  sbki_destroy_map(map);
  return st;
}

sbki_status sbki_grad(const sbki_params* params, const float* xyzl, int64_t p, const int64_t* keys,
                      const float* grad_alpha, int64_t count, double* grad_l, double* grad_sigma0, float* grad_xyz) {
  if (!params || p < 0 || (p > 0 && !xyzl) || count < 0 || (count > 0 && (!keys || !grad_alpha)))
    return fail(nullptr, SBKI_ERR_INVALID_ARG, "bad arguments");
  sbki_map* map = nullptr;
  sbki_status st = sbki_create_map(params, &map);
  if (st != SBKI_OK) return st;
  st = sbki_insert_training(map, xyzl, p, nullptr);
  if (st == SBKI_OK) st = sbki_grad_clear(map);
  if (st == SBKI_OK) st = sbki_grad_add_alpha(map, keys, grad_alpha, count, nullptr);
  if (st == SBKI_OK) st = sbki_backward(map, xyzl, p, grad_l, grad_sigma0, grad_xyz);
  if (st != SBKI_OK) snprintf(g_create_error, sizeof(g_create_error), "%s", map->st.last_error);
  sbki_destroy_map(map);
  return st;
}

sbki_status sbki_import(sbki_map* map, const int64_t* keys, const float* alpha, int64_t count) {
  if (!map) return fail(nullptr, SBKI_ERR_INVALID_ARG, "map is NULL");
  MapState& m = map->st;
  if (count < 0 || (count > 0 && (!keys || !alpha))) return fail(&m, SBKI_ERR_INVALID_ARG, "bad arguments");
  DeviceGuard dg(m.device);
  if (count == 0) return SBKI_OK;
  TmpFree tf;
  tf.st = m.stream;
  const int64_t* dk = nullptr;
  const float* da = nullptr;
  sbki_status st = device_input(m, keys, (size_t)count * 3, &dk, &tf.p[0]);
  if (st != SBKI_OK) return st;
  if ((st = device_input(m, alpha, (size_t)count * m.g.K1, &da, &tf.p[1])) != SBKI_OK) return st;
  m.epoch += 1;
  begin_kernel<<<1, 1, 0, m.stream>>>(m.dc, m.epoch, 0u);
  m.launches += 1;
  CK(&m, launch_import(m, dk, da, count));
  st = read_counters(m);
  if (st != SBKI_OK) return st;
  m.host_blocks = m.hc->n_blocks;
  return status_from_device(m);
}

sbki_status sbki_selftest_bounded_wait(int32_t device, int32_t* device_status) {
  if (!device_status) return fail(nullptr, SBKI_ERR_INVALID_ARG, "device_status is NULL");
  *device_status = SBKI_OK;
  DeviceGuard dg(device);
  unsigned long long *keys = nullptr, *keys_out = nullptr;
  uint32_t *vals = nullptr, *vals_out = nullptr, *n_dev = nullptr, *work = nullptr;
  DevCounters* dc = nullptr;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = dalloc(&keys, kSelftestItems);
  if (e == cudaSuccess) e = dalloc(&keys_out, kSelftestItems);
  if (e == cudaSuccess) e = dalloc(&vals, kSelftestItems);
  if (e == cudaSuccess) e = dalloc(&vals_out, kSelftestItems);
  if (e == cudaSuccess) e = dalloc(&n_dev, 1);
  if (e == cudaSuccess) e = dalloc(&work, radix_work_entries(kSelftestItems));
  if (e == cudaSuccess) e = dalloc(&dc, 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(dc, 0, sizeof(DevCounters), st);
  if (e == cudaSuccess) e = radix_wait_selftest(keys, vals, keys_out, vals_out, n_dev, work, dc, st);
  int32_t err = 0, err2 = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &dc->err, sizeof(err), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  // the one-pass prefix sum's wait, on the same buffers (keys: the data, work: its scratch)
  static_assert(kScanSelftestItems + 1 <= kSelftestItems, "self-test buffers");
  static_assert(scan_tmp_bytes_ce(kScanSelftestItems) <= 4 * radix_work_entries(kSelftestItems), "self-test scratch");
  if (e == cudaSuccess) e = cudaMemsetAsync(dc, 0, sizeof(DevCounters), st);
  if (e == cudaSuccess) e = scan_wait_selftest(keys, work, dc, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err2, &dc->err, sizeof(err2), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (err == SBKI_ERR_TIMEOUT) err = err2;  // both waits must have run out
  void* ptrs[] = {keys, keys_out, vals, vals_out, n_dev, work, dc};
  for (void* p : ptrs) cudaFree(p);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) return fail(nullptr, SBKI_ERR_CUDA, "bounded-wait self-test: %s", cudaGetErrorString(e));
  *device_status = err;
  return SBKI_OK;
}

const char* sbki_last_error(const sbki_map* map) { return map ? map->st.last_error : g_create_error; }

const char* sbki_status_string(sbki_status s) {
  switch (s) {
    case SBKI_OK: return "ok";
    case SBKI_ERR_INVALID_ARG: return "invalid argument";
    case SBKI_ERR_LABEL_RANGE: return "label out of range";
    case SBKI_ERR_CAPACITY: return "capacity exceeded";
    case SBKI_ERR_CUDA: return "CUDA error";
    case SBKI_ERR_TIMEOUT: return "device wait timed out";
    case SBKI_ERR_NOT_FOUND: return "not found";
  }
  return "unknown status";
}

}  // extern "C"
