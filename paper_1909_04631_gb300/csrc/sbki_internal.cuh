// Internal declarations shared by the CUDA translation units of libsbki.
// Nothing here is part of the public C ABI (include/sbki.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sbki.h"

namespace sbki {

// ---------------------------------------------------------------- limits
constexpr int kMaxClasses = 32;          // K+1 <= 32 (shared-memory alpha tile)
constexpr int32_t kKeyLimit = 1 << 20;   // |voxel index| < kKeyLimit on every axis
constexpr int kKeyBits = 19;             // bits per axis of a block coordinate in a packed key
constexpr int kMapShift = 3 * kKeyBits;  // map index above the coordinates in a packed key
constexpr int kMaxMaps = 64;             // independent maps in one handle (map index < 2^6)
constexpr int kMaxScans = 64;            // scans of one batched update
constexpr int kLabelBits = 5;            // a training point's float label word = label + 32 * map
constexpr unsigned long long kEmpty = ~0ull;  // never a key: the map field's top bit is always 0
constexpr int kMaxProbes = 4096;         // hash probe bound (then SBKI_ERR_CAPACITY)
constexpr int kTileShift = 3;            // training-point tiles are 8^3 ds cells
constexpr int kTileEdge = 1 << kTileShift;
constexpr int kLocalBits = 3 * kTileShift;
constexpr int kParts = 8;                // candidate lists: sub-voxel parts per axis (kParts^3 lists)
constexpr int kSegTileItems = 2048;      // sorted items per tile of the segment pass
constexpr int kSegCarryBytes = 48;       // one partial cell sum carried across a segment tile
// tiles of the segment pass over n items
constexpr int64_t seg_tiles(int64_t n) { return (n + kSegTileItems - 1) / kSegTileItems; }

// ---------------------------------------------------------------- device counters
// One instance per map, in device memory; every kernel reads its sizes here so
// that the per-scan sequence needs no host round trip.
struct DevCounters {
  unsigned long long pairs;           // in-support (voxel, point) pairs, this scan
  unsigned long long touched_voxels;  // voxels with a nonzero increment, this scan
  unsigned long long n_free;          // free samples, this scan
  int32_t err;                        // first error (sbki_status), 0 = ok
  uint32_t n_valid;                   // kept hits
  uint32_t n_items;                   // hits + free samples
  uint32_t n_train;                   // training points after downsampling
  uint32_t n_tiles;                   // occupied training-point tiles
  uint32_t n_touched;                 // touched blocks, this scan
  uint32_t n_new;                     // blocks allocated by this scan
  uint32_t n_blocks;                  // pool blocks in use (persistent)
  uint32_t work_next;                 // accumulate work queue head
  uint32_t epoch;                     // scan counter (touched marks)
  uint32_t n_blocks_before;           // n_blocks when this scan started
  uint32_t n_list;                    // (training point, touched block) pairs, this scan
  uint32_t n_slow;                    // downsampling cells left to the slow exact mean, this scan
  uint32_t n_points;                  // input points of the update (all scans)
  int32_t tbox[6];                    // ds-tile bounding box of the kept hits (min xyz, max xyz)
  uint32_t acc_next;                  // work queue head of the point-major accumulation (reset before it)
  uint32_t n_soft;                    // soft labels: training points with a weight row, this scan
  uint32_t commit_done;               // CTAs of the commit launch finished (the last one commits the count)
};

// per-point sample counts of a1/a2: kept hits in bits 40.., free samples below
constexpr unsigned long long kValidOne = 1ull << 40;
constexpr unsigned long long kFreeMask = kValidOne - 1;

// ---------------------------------------------------------------- geometry constants
// Every value that decides an integer (key, count, membership) is computed
// with one fixed IEEE operation sequence (see the kernels); these are the
// rounded constants those sequences use.
struct Geom {
  float res, inv_res;      // voxel edge and fp32(1/res)
  float res_lo;            // fp32(res64 - res): res64 = res + res_lo to ~2^-48
  float ds, inv_ds;        // downsampling cell edge and fp32(1/ds)
  float l, inv_l, l2;      // length scale, 1/l, fp32(l*l)
  float l2_lo, l2_hi;      // l2 (1 -/+ band): outside, the fp32 test decides
  float sigma0;
  float sigma0_k[32];      // per class: fp32(sigma0 * sigma0_scale[k]) (0 past K)
  float scale_k[32];       // per class: fp32(sigma0_scale[k]) (0 past K)
  float step;              // fp32(free_step)
  float fast_lim;          // 2.5 ds: cells with |x| above it take the single-pass exact mean
  double res64, l64, l2_64, min_range, max_range;
  int K1;                  // classes incl. free
  int B, B_shift, B3;      // block edge (power of two), log2, B^3
  int label_bits;          // bits for a label in a sort key
  int assoc;               // 1: extended-block association (a voxel takes points of its block and face neighbours)
  int lscaled;             // 1: some class has its own length scale (l_scale[k] != 1)
  float inv_lk[32];        // per class: fp32(1 / l_k), l_k = l * l_scale[k]
  float l2k_lo[32], l2k_hi[32];  // per class: l_k^2 (1 -/+ band)
  double l2k_64[32];       // per class: l_k^2
  double lmax64;           // largest l_k of the classes 0..K
};

// Extended-block association (Sec. IV): a pair counts only when the voxel's
// block is the point's own block or one of its six face neighbours.  Block
// digits d = dx + 3 dy + 9 dz (each of dx, dy, dz in 0..2, 1 = the own block's
// coordinate): the own block is 13, the faces 4, 10, 12, 14, 16, 22.
constexpr uint32_t kFaceDigits = (1u << 13) | (1u << 4) | (1u << 10) | (1u << 12) | (1u << 14) | (1u << 16) | (1u << 22);
__host__ __device__ inline bool face_or_own(int dx, int dy, int dz) {  // block offsets in -1..1
  return (dx < 0 ? -dx : dx) + (dy < 0 ? -dy : dy) + (dz < 0 ? -dz : dz) <= 1;
}

// Per-scan key frame: training-point tiles are packed relative to an origin tile.
struct KeyFrame {
  int32_t org[3];   // lowest tile (ds-tile index) of the region
  int bits[3];      // bits of a relative tile index, per axis
  int total_bits;   // bits of a scan-local sort key (the scan index, if any, sits above)
  int scan_bits;    // bits of the scan index in a batched update (0: one scan)
};

// One scan of an update, in device memory (read by the ingest kernels, so a
// batch of scans needs no per-scan launch arguments).  Entry [count].off holds
// the total point count.
struct ScanDesc {
  const float* pts;       // [n,3] sensor frame (device)
  const int32_t* labels;  // [n] 1..K (device)
  int64_t n;
  int64_t off;            // first global point index of the scan
  double r[9], t[3];      // world_from_sensor
  float o[3];             // fp32 sensor origin
  int32_t org[3];         // key-frame origin tile
  int32_t map_id;         // target map of the handle
  const float* probs;     // soft labels: [n,K] probability vectors over classes 1..K (device), else null
};

// ---------------------------------------------------------------- scratch of one map
struct Scratch {
  // per input point
  float* pts = nullptr;           // staged host points [n_cap,3]
  int32_t* labels = nullptr;      // staged host labels [n_cap]
  float4* world = nullptr;        // [n_cap] world xyz + label bits
  unsigned long long* cnt = nullptr;  // [n_cap+1] packed (valid<<40 | n_free), scanned in place
  int64_t n_cap = 0;
  // per item (hits + free samples)
  float4* items = nullptr;        // [s_cap] xyz + label at source position
  float4* sitems = nullptr;       // [s_cap] the items in sorted (scan, cell, label) order
  unsigned long long* keys = nullptr;   // [s_cap]
  unsigned long long* keys2 = nullptr;  // [s_cap]
  uint32_t* vals = nullptr;       // [s_cap] source positions
  uint32_t* vals2 = nullptr;      // [s_cap]
  uint32_t* flags = nullptr;      // [max(s_cap + 1, 2 seg_tiles(s_cap) + 2)] segment-pass tile words
  uint32_t* seg_start = nullptr;  // [s_cap+1]
  float4* train = nullptr;        // [s_cap] training points (xyz, label bits), tile-sorted
  int64_t s_cap = 0;
  // radix sort / scan temporaries
  uint32_t* hist = nullptr;       // [256 * sort_ctas + 1]
  void* scan_tmp = nullptr;       // partial sums
  int64_t hist_cap = 0;
  // per touched block
  uint32_t* touched = nullptr;    // [hash_cap] hash slots touched this scan
  uint32_t* fresh = nullptr;      // [hash_cap] hash slots created this scan
  int* bbox = nullptr;            // [6] tile bounding box of a given training set
  uint32_t* slow = nullptr;       // [s_cap + 2] downsampling cells left to the slow exact mean
  void* carry = nullptr;          // [2 seg_tiles(s_cap)] partial sums of cells crossing a segment tile
  ScanDesc* desc = nullptr;       // [kMaxScans + 1] scans of the current update
  uint32_t* ownslot = nullptr;    // [s_cap] fast accumulation form: hash slot of each training point's own block
  // soft labels (allocated on first use)
  float* probs = nullptr;         // [n_cap, K] staged host probability vectors
  uint32_t* hit_src = nullptr;    // [n_cap] global point index of each kept hit (by hit rank)
  int32_t* softidx = nullptr;     // [s_cap] weight row of each training point, -1 for none (one-hot label)
  float* wsoft = nullptr;         // [soft_cap, K+1] weight rows
  int64_t soft_cap = 0;           // point capacity the soft buffers were sized for
};

// ---------------------------------------------------------------- the map
struct MapState {
  sbki_params prm;
  Geom g;
  cudaStream_t stream = nullptr;
  int device = 0;
  int sm_count = 0;
  // block hash: key -> pool index
  unsigned long long* hkeys = nullptr;  // [hash_cap]
  int32_t* hvals = nullptr;             // [hash_cap]
  uint32_t* hmark = nullptr;            // [hash_cap] epoch of last touch
  uint32_t* hcnt = nullptr;             // [hash_cap] points touching the block (zero between scans)
  uint32_t* hcur = nullptr;             // [hash_cap] fill cursor of the block's point list
  int64_t hash_cap = 0;                 // power of two
  uint32_t* boff = nullptr;             // [hash_cap + 1] per touched block: first entry in blist
  uint32_t* blist = nullptr;            // [list_cap] training-point indices grouped by touched block
  int64_t list_cap = 0;
  // pool
  float* alpha = nullptr;               // [pool_blocks][K1][B3] increments
  unsigned long long* pool_keys = nullptr;  // [pool_blocks]
  int32_t* pairs = nullptr;             // [pool_blocks][B3] (only if track_pairs)
  int64_t pool_blocks = 0;
  DevCounters* dc = nullptr;            // device counters
  DevCounters* hc = nullptr;            // pinned host mirror
  Scratch s;
  uint32_t epoch = 0;
  uint32_t host_blocks = 0;             // last known n_blocks (host view)
  sbki_status sticky = SBKI_OK;
  int64_t launches = 0;                 // kernels launched on this map
  int acc_mode = 0;                     // 0: point-major (global reductions), 1: block-major (shared tile)
  bool soft = false;                    // the update in progress carries soft labels
  int active_map = 0;                   // map index the single-map calls act on
  sbki_tuning tune{0, 30, 8, 16};       // launch shapes (sbki_set_tuning)
  cudaStream_t rec_stream = nullptr;    // private stream the batched update is recorded on
  cudaGraphExec_t batch_exec[kMaxScans + 1] = {};  // recorded batched updates, by scan count
  int64_t batch_kernels[kMaxScans + 1] = {};       // kernels in each recording
  uint64_t batch_gen[kMaxScans + 1] = {};          // scratch generation each recording used
  uint64_t scratch_gen = 1;             // advances when scratch buffers move
  ScanDesc* hdesc = nullptr;            // pinned host staging of s.desc
  uint32_t* ctab = nullptr;             // point-major candidate lists [kParts^3][ctab_pad]
  int32_t* clen = nullptr;              // [kParts^3] entries of each list
  uint32_t* ftab = nullptr;             // fast accumulation form's candidate lists (2R + 1 <= 7), or null:
                                        // one table of kFastParts^3 lists per distinct class support
  int32_t* flen = nullptr;              // their entry counts
  int ftab_pad = 0;
  int ftab_R = 0;                       // offsets -R..R per axis of the fast form's rows
  int32_t ftab_of[32] = {};             // per class: its table, or -1 (the weighted form takes the class)
  uint32_t ftab_classes = 0;            // classes with a table
  bool ftab_own_touched = false;        // every class's l above half the voxel diagonal (own block always touched)
  uint32_t* nbrslot = nullptr;          // fast form: [hash_cap][32] per own block (hash slot), the hash slots of the
                                        // neighbour blocks its points touched in the last update, by block digit
  float* gpool = nullptr;               // dL/dalpha [pool_blocks][K1][B3] (differentiable form, on first use)
  double* dacc = nullptr;               // [4 + 32]: held-out LL, sum s G f, sum s G u^4 D d, keys missed (as
                                        // u64), then sum G f per class
  int ctab_pad = 0, ctab_R = 0;
  bool profiling = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};      // stage events of the update being issued
  cudaEvent_t ev_alt[4] = {nullptr, nullptr, nullptr, nullptr};  // those of an asynchronous update not yet read
  bool prof_pending = false;                                     // ev_alt holds such an update
  sbki_profile_data prof{};
  char last_error[512] = {0};
  sbki_stats last_stats{};
};

// ---------------------------------------------------------------- device helpers
// Block key: map index (6 bits, top bit of its 7-bit field always 0), then
// x, y, z block coordinates offset by 2^18 (19 bits each; |block| < 2^18).
__host__ __device__ inline unsigned long long pack_block(int32_t bx, int32_t by, int32_t bz, int32_t map) {
  const unsigned long long off = 1ull << (kKeyBits - 1);
  return ((unsigned long long)map << kMapShift) | (((unsigned long long)(bx + (int64_t)off)) << (2 * kKeyBits)) |
         (((unsigned long long)(by + (int64_t)off)) << kKeyBits) | ((unsigned long long)(bz + (int64_t)off));
}
__host__ __device__ inline void unpack_block(unsigned long long k, int32_t& bx, int32_t& by, int32_t& bz) {
  const int64_t off = 1ll << (kKeyBits - 1);
  const unsigned long long m = (1ull << kKeyBits) - 1;
  bx = (int32_t)((int64_t)((k >> (2 * kKeyBits)) & m) - off);
  by = (int32_t)((int64_t)((k >> kKeyBits) & m) - off);
  bz = (int32_t)((int64_t)(k & m) - off);
}
__host__ __device__ inline int32_t map_of_block(unsigned long long k) { return (int32_t)(k >> kMapShift); }
__device__ __forceinline__ uint32_t hash_slot(unsigned long long k, int64_t cap) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return (uint32_t)(k & (unsigned long long)(cap - 1));
}
__device__ __forceinline__ void set_error(DevCounters* dc, int code) { atomicCAS(&dc->err, 0, code); }

// x / n for 0 <= x < 4096 and 1 <= n <= 32, as a multiply and a shift by a
// reciprocal m = ceil(2^20 / n) (exact over that range; checked exhaustively)
__device__ __forceinline__ uint32_t small_recip(uint32_t n) { return ((1u << 20) + n - 1u) / n; }
__device__ __forceinline__ uint32_t small_div(uint32_t x, uint32_t m) { return (x * m) >> 20; }

// ---------------------------------------------------------------- compensated offsets
// Membership d^2 < l^2 is decided in FP32 from offsets e = c_v - x formed to
// about one ulp: for a reference voxel index K the offset of its centre,
// E0 = (K + 1/2) res64 - x, is held as an unevaluated sum hi + lo (the product
// through an exact FMA residual, the difference through an exact two-sum),
// and e(K + d) = E0 + d res64 is rounded once more.  d^2 from such offsets is
// within ~5e-7 relative of the exact value, so a pair whose FP32 d^2 lies in
// the relative band [l2_lo, l2_hi] = l^2 (1 -/+ 2e-6) is re-decided in FP64
// exactly as the plain definition states: c = (v + 0.5)*res64, e = c - x,
// d^2 = (ex^2 + ey^2) + ez^2 < l^2.  Round-to-nearest intrinsics keep the
// compiler from contracting or reordering any of it.
// (float)K for |K| < 2^22, exactly, without a conversion instruction
__device__ __forceinline__ float small_int_to_float(int K) {
  return __fsub_rn(__int_as_float(0x4B400000 + K), 12582912.0f);
}
__device__ __forceinline__ void centre_offset0(int K, float x, const Geom& g, float& hi, float& lo) {
  const float c0 = __fadd_rn(small_int_to_float(K), 0.5f);  // exact: |K| < 2^22
  const float p_hi = __fmul_rn(c0, g.res);
  const float p_lo = __fmaf_rn(c0, g.res_lo, __fmaf_rn(c0, g.res, -p_hi));
  const float s = __fsub_rn(p_hi, x);
  const float bb = __fsub_rn(s, p_hi);
  const float err = __fadd_rn(__fsub_rn(p_hi, __fsub_rn(s, bb)), __fsub_rn(-x, bb));
  hi = s;
  lo = __fadd_rn(err, p_lo);
}
// c_{K+d} - x = E0 + d res, rounded once (d a small integer)
__device__ __forceinline__ float centre_offset_at(int d, float hi, float lo, const Geom& g) {
  const float fd = small_int_to_float(d);
  return __fadd_rn(__fmaf_rn(fd, g.res, hi), __fmaf_rn(fd, g.res_lo, lo));
}
__device__ __forceinline__ bool in_support64(int vx, int vy, int vz, float x, float y, float z, const Geom& g) {
  const double ex = __dsub_rn(__dmul_rn(__dadd_rn((double)vx, 0.5), g.res64), (double)x);
  const double ey = __dsub_rn(__dmul_rn(__dadd_rn((double)vy, 0.5), g.res64), (double)y);
  const double ez = __dsub_rn(__dmul_rn(__dadd_rn((double)vz, 0.5), g.res64), (double)z);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
  return d2 < g.l2_64;
}
// The same test as a call: the FP64 conversions stay inside the (rare) band
// path instead of being hoisted into the caller's loop.
static __device__ __noinline__ bool in_support64_call(int vx, int vy, int vz, float x, float y, float z, double res64,
                                               double l2_64) {
  const double ex = __dsub_rn(__dmul_rn(__dadd_rn((double)vx, 0.5), res64), (double)x);
  const double ey = __dsub_rn(__dmul_rn(__dadd_rn((double)vy, 0.5), res64), (double)y);
  const double ez = __dsub_rn(__dmul_rn(__dadd_rn((double)vz, 0.5), res64), (double)z);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
  return d2 < l2_64;
}

// ---------------------------------------------------------------- shared host helpers (sbki_api.cu)
sbki_status validate_params(const sbki_params* p);
Geom geometry_of(const sbki_params& p);
KeyFrame frame_of_scan(const MapState& m, const double T[16]);
// the key frame of a scan fitted to its hits' tile box (DevCounters::tbox after the transform)
void tighten_frame(const Geom& g, const int32_t tbox[6], const double T[16], KeyFrame& kf);
void set_global_error(const char* msg);

// ---------------------------------------------------------------- launchers (one per .cu)
// scan.cu: exclusive prefix sums in place over n+1 entries (entry n receives the total);
// with n_dev the count is min(n, *n_dev), read on the device (n bounds the launch)
cudaError_t exclusive_scan_u32(uint32_t* data, int64_t n, void* tmp, cudaStream_t st, const uint32_t* n_dev = nullptr);
cudaError_t exclusive_scan_u64(unsigned long long* data, int64_t n, void* tmp, cudaStream_t st,
                               const uint32_t* n_dev = nullptr);
int64_t scan_tmp_bytes(int64_t n);
// scratch of either form for n entries: the partial sums, or a counter, flags and two values per tile of 2048
constexpr int64_t scan_tmp_bytes_ce(int64_t n) { return 24 * ((n + 2047) / 2048 + 2); }
// one launch (chained tiles, bounded look-back: SBKI_ERR_TIMEOUT in dc when a wait runs out); sm_count sizes the grid
// Failure-detection self-test of the one-pass form: a scan of kScanSelftestItems
// zeros (data: that many + 1 entries; tmp: scan_tmp_bytes_ce of them; dc
// zeroed) whose tile counter starts at 1, so tile 0 never publishes and the
// look-back of tile 1 runs out with SBKI_ERR_TIMEOUT.
constexpr int64_t kScanSelftestItems = 3 * 2048;
cudaError_t scan_wait_selftest(unsigned long long* data, void* tmp, DevCounters* dc, cudaStream_t st);
// items_cap >= 0: data are the per-point sample counts of a1/a2 and the grand
// total also sets dc->n_valid, n_free and n_items (SBKI_ERR_CAPACITY and no
// items when they exceed items_cap)
cudaError_t exclusive_scan_u64_onepass(unsigned long long* data, int64_t n, void* tmp, cudaStream_t st,
                                       const uint32_t* n_dev, int sm_count, DevCounters* dc, int64_t items_cap = -1);

// radix_sort.cu: stable LSD sort of (keys, vals) over bits [0, bits) (at most
// 8 passes of 8 bits); count read from *n_dev, cap >= count bounds the work
// area; the pointer pairs are swapped as passes go, so on return (keys, vals)
// name the buffers that hold the result.  hist: radix_work_entries(cap) words.
constexpr int64_t kRadixTile = 4096;  // items per tile of one pass
constexpr int kMaxPasses = 8;
constexpr int64_t radix_work_entries(int64_t cap) {
  return 2 * 256 * ((cap + kRadixTile - 1) / kRadixTile) + kMaxPasses * 256 + kMaxPasses;
}
// The last pass also writes payload_out[pos] = payload[value] when payload_out is given.
cudaError_t radix_sort_pairs(unsigned long long*& keys, uint32_t*& vals, unsigned long long*& keys_alt,
                             uint32_t*& vals_alt, const uint32_t* n_dev, int64_t cap, int bits, uint32_t* hist,
                             int sm_count, DevCounters* dc, cudaStream_t st, const float4* payload = nullptr,
                             float4* payload_out = nullptr);
int64_t radix_hist_entries(int64_t cap);
// Failure-detection self-test of the sort's bounded waits: one digit pass over
// kSelftestItems items (device buffers of that many entries; work:
// radix_work_entries(kSelftestItems) words; n_dev one word; dc zeroed) whose
// tile counter starts at 1, so tile 0 never publishes its counts and the
// look-back of the other tiles runs out with SBKI_ERR_TIMEOUT.
constexpr int64_t kSelftestItems = 3 * kRadixTile;
cudaError_t radix_wait_selftest(unsigned long long* keys, uint32_t* vals, unsigned long long* keys_out,
                                uint32_t* vals_out, uint32_t* n_dev, uint32_t* work, DevCounters* dc, cudaStream_t st);

// ingest.cu
// ingest of the ns scans described in m.s.desc (ns + 1 entries, the last holding the total)
cudaError_t launch_transform_count(MapState& m, int ns, int64_t total_n);
cudaError_t launch_emit(MapState& m, int ns, int64_t total_n, const KeyFrame& kf, uint32_t* hit_src = nullptr);
cudaError_t launch_downsample_n(MapState& m, const KeyFrame& kf, int64_t nitems);
cudaError_t launch_train_bbox(MapState& m, const float4* in, int64_t p, int* bbox_dev);
cudaError_t launch_train_prepare(MapState& m, const float4* in, int64_t p, const KeyFrame& kf);

// blocks.cu
cudaError_t launch_touch_blocks(MapState& m, const KeyFrame& kf, int64_t bound);
cudaError_t launch_touch_cells(MapState& m, int64_t bound);  // counting model: the block of each point's voxel
cudaError_t launch_commit_blocks(MapState& m);
// blocks of the given voxel keys (selected map), commit, zero-fill, then alpha - alpha0 at the keys
cudaError_t launch_import(MapState& m, const int64_t* keys, const float* alpha, int64_t count);
cudaError_t launch_bin_points(MapState& m, int64_t bound);

// accumulate.cu
cudaError_t launch_accumulate(MapState& m, const KeyFrame& kf);
cudaError_t launch_accumulate_points(MapState& m);
bool fast_form_ready(const MapState& m);  // the fast point-major form can run on this map
cudaError_t launch_accumulate_counts(MapState& m, int64_t bound);  // counting model, Eq. (alpha)
cudaError_t launch_fresh_fill(MapState& m);  // zero the blocks created by this update
cudaError_t build_candidate_tables(MapState& m);
// backward.cu: held-out log-likelihood (+ dLL/dalpha into grad), upstream gradient at voxel keys,
// and the backward pass through Eq. (kernel) into acc_dev[0..1] and grad_xyz
cudaError_t launch_heldout(const MapState& m, const float* xyz, const int32_t* labels, int64_t h, float* grad,
                           double* ll_dev);
cudaError_t launch_grad_scatter(const MapState& m, const int64_t* keys, const float* grad, int64_t count, float* gpool,
                                unsigned long long* missed_dev);
cudaError_t launch_backward(const MapState& m, const float4* xyzl, int64_t p, const float* gpool, double* acc_dev,
                            float* grad_xyz, double* acc_class);
size_t accumulate_smem_bytes(const Geom& g);

// soft.cu: weight rows of the groups holding hits (soft labels), their export,
// and the weighted accumulation (soft labels and/or per-class length scales)
cudaError_t launch_soft_weights(MapState& m);
cudaError_t launch_soft_export(MapState& m, float* xyz, float* w, int64_t cap);
cudaError_t launch_accumulate_weighted(MapState& m, bool soft, bool fill = true, uint32_t skip = 0u);

// readoff.cu
cudaError_t launch_query(const MapState& m, const float* xyz, int64_t q, float* probs, float* var, float* mode,
                         int32_t* label, float* p_occ, int32_t* state);
cudaError_t launch_gather_alpha(const MapState& m, float* out, int64_t nblocks);
// rows of the selected map's blocks in pool order: rowb [nb + 1] work (scanned block row offsets)
cudaError_t launch_export_rows(const MapState& m, uint32_t nb, uint32_t* rowb, void* scan_tmp, int64_t* keys,
                               float* out);

}  // namespace sbki
