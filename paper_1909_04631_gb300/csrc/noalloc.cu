// sbki_training_set_noalloc: the training set of one scan (hits + free-space
// samples, downsampled to one centroid per cell and label) computed without
// any device allocation.
//
// Who needs this: a caller that must not allocate once it is running - a
// robot's real-time mapping loop that pre-reserves all memory at start-up (a
// cudaMalloc can stall or fail mid-run), or a host framework that owns the
// device heap through its own pool and cannot let a library allocate beside
// it.  Such a caller passes device buffers for the inputs and the output;
// every intermediate buffer of the computation
// (transformed points, sample counts, items, radix-sort keys and values,
// segment tables, scan partials, the scan descriptor, device counters) lives in one
// file-scope device array of fixed size, so calling this allocates nothing.
//
// Limits: at most kMaxPoints input points and kMaxItems hits + free samples
// per call; larger inputs are rejected with SBKI_ERR_INVALID_ARG (points) or
// SBKI_ERR_CAPACITY (items, known only after counting on the device).  The
// array (kScratchBytes, about 11 MB) is reserved on every device that loads
// the library, for the life of the process.  All calls share it and it keeps
// the last call's contents; the device counters are cleared at the start of
// each call, every other buffer is written before it is read.  Calls whose
// work overlaps on the GPU (different streams, or different host threads at
// once) race on the array: serialise them.  The first call on a device looks
// up the array's device address (cudaGetSymbolAddress) with that device
// current; make that first call before any stream capture.  The call
// synchronises its stream twice (after counting the items and after the
// downsampling, to read the counts back).
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "sbki_internal.cuh"

namespace {

constexpr int64_t kMaxPoints = 16384;    // input points per call
constexpr int64_t kMaxItems = 1 << 17;   // hits + free samples per call

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffCounters = 0;
constexpr size_t kOffWorld = align256(kOffCounters + sizeof(sbki::DevCounters));
constexpr size_t kOffCnt = align256(kOffWorld + 16 * kMaxPoints);
constexpr size_t kOffItems = align256(kOffCnt + 8 * (kMaxPoints + 1));
constexpr size_t kOffSitems = align256(kOffItems + 16 * kMaxItems);
constexpr size_t kOffKeys = align256(kOffSitems + 16 * kMaxItems);
constexpr size_t kOffKeys2 = align256(kOffKeys + 8 * kMaxItems);
constexpr size_t kOffVals = align256(kOffKeys2 + 8 * kMaxItems);
constexpr size_t kOffVals2 = align256(kOffVals + 4 * kMaxItems);
constexpr size_t kOffFlags = align256(kOffVals2 + 4 * kMaxItems);
constexpr size_t kFlagWords = kMaxItems + 1 > 2 * sbki::seg_tiles(kMaxItems) + 2 ? kMaxItems + 1 : 2 * sbki::seg_tiles(kMaxItems) + 2;
constexpr size_t kOffSeg = align256(kOffFlags + 4 * kFlagWords);
constexpr size_t kOffTrain = align256(kOffSeg + 4 * (kMaxItems + 1));
constexpr size_t kOffSlow = align256(kOffTrain + 16 * kMaxItems);
constexpr size_t kOffCarry = align256(kOffSlow + 4 * (kMaxItems + 2));
constexpr size_t kHistEntries = (size_t)sbki::radix_work_entries(kMaxItems);
constexpr size_t kOffHist = align256(kOffCarry + (size_t)sbki::kSegCarryBytes * 2 * sbki::seg_tiles(kMaxItems));
constexpr size_t kOffScanTmp = align256(kOffHist + 4 * kHistEntries);
constexpr size_t kScanTmpBytes = 8 * ((kMaxItems + 2) / 2048 + 64);  // partial sums of the largest scan
static_assert(kScanTmpBytes >= (size_t)sbki::scan_tmp_bytes_ce(kMaxPoints + 1), "prefix-sum scratch");
constexpr size_t kOffDesc = align256(kOffScanTmp + kScanTmpBytes);
constexpr size_t kScratchBytes = align256(kOffDesc + 2 * sizeof(sbki::ScanDesc));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch[kMaxDevices] = {nullptr};  // device address of the array, per device
int g_sms[kMaxDevices] = {0};

// Once per device, with that device current: the array's device address.
sbki_status setup_device(int dev, unsigned char** ptr, int* sms) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaError_t e = cudaSetDevice(dev);
    void* p = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    int n = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess) {
      char msg[256];
      snprintf(msg, sizeof(msg), "training set without allocation: device %d set-up failed: %s", dev,
               cudaGetErrorString(e));
      sbki::set_global_error(msg);
      return SBKI_ERR_CUDA;
    }
    g_scratch[dev] = static_cast<unsigned char*>(p);
    g_sms[dev] = n;
  }
  *ptr = g_scratch[dev];
  *sms = g_sms[dev];
  return SBKI_OK;
}

bool on_device(const void* p, int dev) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

sbki_status fail(sbki_status s, const char* msg) {
  sbki::set_global_error(msg);
  return s;
}

#define CKN(expr)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (expr);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      char m_[256];                                                                                 \
      snprintf(m_, sizeof(m_), "training set without allocation: %s: %s", #expr, cudaGetErrorString(e_)); \
      return fail(SBKI_ERR_CUDA, m_);                                                               \
    }                                                                                               \
  } while (0)

sbki_status run(const sbki_params* params, const float* points, const int32_t* labels, int64_t n,
                const double pose[16], float* xyzl_out, int64_t cap, int64_t* count) {
  using namespace sbki;
  const int dev = params->device;
  unsigned char* base = nullptr;
  int sms = 0;
  sbki_status st = setup_device(dev, &base, &sms);
  if (st != SBKI_OK) return st;
  if (!on_device(points, dev) || !on_device(labels, dev) || (cap > 0 && !on_device(xyzl_out, dev)))
    return fail(SBKI_ERR_INVALID_ARG, "training set without allocation: points, labels and the output must be device "
                                      "buffers of params->device");
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(pose[i])) return fail(SBKI_ERR_INVALID_ARG, "sensor_pose has a non-finite entry");
  for (int a = 0; a < 3; ++a)
    if ((std::fabs(pose[4 * a + 3]) + params->max_range) / params->res > (double)(kKeyLimit - 1024))
      return fail(SBKI_ERR_INVALID_ARG, "sensor origin too far from the map origin");

  MapState m;  // a view: every pointer below points into the fixed array
  m.prm = *params;
  m.g = geometry_of(*params);
  m.stream = (cudaStream_t)params->cuda_stream;
  m.device = dev;
  m.sm_count = sms;
  m.dc = reinterpret_cast<DevCounters*>(base + kOffCounters);
  Scratch& s = m.s;
  s.world = reinterpret_cast<float4*>(base + kOffWorld);
  s.cnt = reinterpret_cast<unsigned long long*>(base + kOffCnt);
  s.n_cap = kMaxPoints;
  s.items = reinterpret_cast<float4*>(base + kOffItems);
  s.sitems = reinterpret_cast<float4*>(base + kOffSitems);
  s.keys = reinterpret_cast<unsigned long long*>(base + kOffKeys);
  s.keys2 = reinterpret_cast<unsigned long long*>(base + kOffKeys2);
  s.vals = reinterpret_cast<uint32_t*>(base + kOffVals);
  s.vals2 = reinterpret_cast<uint32_t*>(base + kOffVals2);
  s.flags = reinterpret_cast<uint32_t*>(base + kOffFlags);
  s.seg_start = reinterpret_cast<uint32_t*>(base + kOffSeg);
  s.train = reinterpret_cast<float4*>(base + kOffTrain);
  s.slow = reinterpret_cast<uint32_t*>(base + kOffSlow);
  s.carry = base + kOffCarry;
  s.hist = reinterpret_cast<uint32_t*>(base + kOffHist);
  s.hist_cap = (int64_t)kHistEntries;
  s.scan_tmp = base + kOffScanTmp;
  s.desc = reinterpret_cast<ScanDesc*>(base + kOffDesc);
  s.s_cap = kMaxItems;

  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != dev) CKN(cudaSetDevice(dev));
  struct Restore {
    int p, d;
    ~Restore() {
      if (p >= 0 && p != d) cudaSetDevice(p);
    }
  } restore{prev, dev};

  // the counters start cleared (the hits' tile box empty) with this call's point
  // count; every other buffer is written before it is read
  DevCounters init;
  memset(&init, 0, sizeof(init));
  init.n_points = (uint32_t)n;
  for (int a = 0; a < 3; ++a) {
    init.tbox[a] = INT_MAX;
    init.tbox[3 + a] = INT_MIN;
  }
  CKN(cudaMemcpyAsync(m.dc, &init, sizeof(init), cudaMemcpyHostToDevice, m.stream));
  KeyFrame kf = frame_of_scan(m, pose);
  ScanDesc hd[2];  // this scan, then the end marker holding the point count
  memset(hd, 0, sizeof(hd));
  hd[0].pts = points;
  hd[0].labels = labels;
  hd[0].n = n;
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) hd[0].r[3 * r + c] = pose[4 * r + c];
    hd[0].t[r] = pose[4 * r + 3];
    hd[0].o[r] = (float)pose[4 * r + 3];
    hd[0].org[r] = kf.org[r];
  }
  hd[1].off = n;
  CKN(cudaMemcpyAsync(s.desc, hd, sizeof(hd), cudaMemcpyHostToDevice, m.stream));
  CKN(launch_transform_count(m, 1, n));
  DevCounters h;
  CKN(cudaMemcpyAsync(&h, m.dc, sizeof(h), cudaMemcpyDeviceToHost, m.stream));
  CKN(cudaStreamSynchronize(m.stream));
  if (h.err == SBKI_ERR_LABEL_RANGE) return fail(SBKI_ERR_LABEL_RANGE, "a label is outside 1..K");
  if (h.err == SBKI_ERR_CAPACITY)
    return fail(SBKI_ERR_CAPACITY, "training set without allocation: more than 131072 hits + free samples");
  if (h.err != 0) return fail((sbki_status)h.err, "training set without allocation: device error");
  const int64_t nitems = h.n_items;
  if (nitems > 0) {
    // sort keys fitted to the hits' tile box, as in sbki_training_set
    tighten_frame(m.g, h.tbox, pose, kf);
    for (int r = 0; r < 3; ++r) hd[0].org[r] = kf.org[r];
    CKN(cudaMemcpyAsync(s.desc, hd, sizeof(hd), cudaMemcpyHostToDevice, m.stream));
    CKN(launch_emit(m, 1, n, kf));
    CKN(launch_downsample_n(m, kf, nitems));
    CKN(cudaMemcpyAsync(&h, m.dc, sizeof(h), cudaMemcpyDeviceToHost, m.stream));
    CKN(cudaStreamSynchronize(m.stream));
    if (h.err != 0) return fail((sbki_status)h.err, "training set without allocation: device error");
  }
  const int64_t P = nitems > 0 ? (int64_t)h.n_train : 0;
  *count = P;
  const int64_t c = P < cap ? P : cap;
  if (c > 0) {
    CKN(cudaMemcpyAsync(xyzl_out, s.train, sizeof(float4) * c, cudaMemcpyDeviceToDevice, m.stream));
    CKN(cudaStreamSynchronize(m.stream));
  }
  if (P > cap) return fail(SBKI_ERR_CAPACITY, "training set without allocation: output capacity too small");
  return SBKI_OK;
}

}  // namespace

extern "C" sbki_status sbki_training_set_noalloc(const sbki_params* params, const float* points, const int32_t* labels,
                                                 int64_t n, const double sensor_pose[16], float* xyzl_out,
                                                 int64_t cap, int64_t* count) {
  if (!params || !sensor_pose || !count || n < 0 || cap < 0 || (n > 0 && (!points || !labels)) ||
      (cap > 0 && !xyzl_out))
    return fail(SBKI_ERR_INVALID_ARG, "training set without allocation: bad arguments");
  sbki_status st = sbki::validate_params(params);
  if (st != SBKI_OK) return st;
  if (params->device < 0 || params->device >= kMaxDevices)
    return fail(SBKI_ERR_INVALID_ARG, "training set without allocation: device ordinal out of range");
  if (n > kMaxPoints)
    return fail(SBKI_ERR_INVALID_ARG, "training set without allocation: more than 16384 input points");
  *count = 0;
  if (n == 0) return SBKI_OK;
  return run(params, points, labels, n, sensor_pose, xyzl_out, cap, count);
}
