// S-BKI oracle: a plain, slow, single-threaded FP64 CPU implementation of the
// semantic Bayesian kernel inference map update.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
// this file; only the test suite, the smoke check and the benchmark's CPU
// baseline leg do.  It shares no source, header, table or helper with the CUDA
// library: every step below is written out from the paper's equations.
//
// Method (Gan et al., "Bayesian Spatial Kernel Smoothing for Scalable Dense
// Semantic Mapping"):
//   * Sec. III: labelled points x_i with one-hot y_i form the training data;
//     free-space points interpolated along each beam carry the free class.
//   * Eq. (alpha_kernel), Sec. IV: alpha_*^k = alpha_0^k + sum_i k(x_*, x_i) y_i^k,
//     queried at voxel centroids and applied recursively scan after scan.
//   * Eq. (kernel): sparse kernel of length-scale l and scale sigma0, zero for d >= l.
//   * Eq. (mode), Eq. (variance), Sec. V-C: read-off of mean, variance, mode and
//     occupancy probability from alpha.
//
// Readings where the paper is silent or garbled (each one is listed in the
// design notes of the repository):
//   K1  Eq. (kernel) is typeset with a misplaced bracket; the sparse kernel it
//       cites is f(r) = (2 + cos 2 pi r)(1 - r)/3 + sin(2 pi r)/(2 pi), r = d/l < 1,
//       which is 1 at r = 0, 0 at r = 1, with zero slope at both ends.
//   K2  Class 0 is the free class, classes 1..K are occupied; alpha_0 is the same
//       for all K+1 classes; the map stores increments and adds alpha_0 on read.
//   K3  Free samples: for a hit at range r from the sensor origin o, samples at
//       t_j = r - j*s for j = 1, 2, ... while t_j > 0 (never at the hit itself).
//   K4  Downsampling groups hits and free samples by (ds cell, label); the
//       representative is the centroid: per axis the exact mean of the
//       members' FP32 coordinates, rounded once to FP32 (nearest, ties to
//       even).  Being exact, it does not depend on the order of the members.
//   K5  Every voxel centre with ||c_v - x_i||^2 < l^2 (FP64) receives the pair.
//   K6  Geometry that decides integer keys is a fixed FP32 operation sequence
//       (this file is compiled with -ffp-contract=off): world = fp32(FP64 R p + t)
//       evaluated as ((r0 px + r1 py) + r2 pz) + t; key = floorf(x * fp32(1/res)).
//   K7  A voxel with no kernel mass reads as the prior with state "unknown";
//       otherwise free if p_occ < free_thresh, occupied if p_occ > occ_thresh.
//   K11 Counting model (S-CSM, Eq. (alpha), Sec. IV): the measurements it counts
//       are the training points of steps a1..a3, each of weight 1 (as in K4),
//       and "x_i in cell j" is the voxel key of K6.  Every counted point leaves
//       one (voxel, point) pair, so the pair count of a voxel is its count.
//   K13 Per-class kernel scale (the paper names class-dependent signal
//       variance as the way to let sigma0 matter): class k's kernel is
//       sigma0 * sigma0_scale[k] * f(d/l); all scales 1 is Eq. (kernel) as printed.
//   K14 Extended-block association (Sec. IV, the paper's software): a voxel of
//       block b takes the training points whose own voxel (K6 key) lies in b
//       or in one of b's six face neighbours; pairs from edge or corner
//       neighbours are left out even when d < l.  association = 0 is the
//       exact rule K5, 1 this one.
//   K15 Soft labels (next row f1): a hit carries a probability vector over the
//       occupied classes 1..K instead of one label (free samples stay class 0).
//       Downsampling groups by (cell, most probable class, ties to the lowest),
//       so one-hot vectors give the groups of K4; the representative is the K4
//       centroid with, per class, the exact mean of the members' weights
//       rounded once to FP32.  A training point adds sigma0 s_k f(d/l) w^k into
//       every class k (Eq. alpha_kernel with y_i = w).
//   K16 Per-class support (the rest of next row f1): class k's kernel has the
//       length scale l_k = length_scale * l_scale[k]; a pair counts for class k
//       when d < l_k.  All l_scale 1 is the common l.  The differentiable form
//       takes the common l.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <unordered_map>
#include <vector>

namespace {

struct Params {
  double res, length_scale, sigma0, alpha0, free_step, ds_res, min_range, max_range, free_thresh,
      occ_thresh;
  int32_t num_classes;  // K occupied classes; alpha has K+1 entries
  int32_t block_edge;
  int32_t sensor_model;  // 0: kernel inference, Eq. (alpha_kernel); 1: counting, Eq. (alpha)
  double sigma0_scale[32];  // reading K13: class k's kernel scale is sigma0 * sigma0_scale[k]
  int32_t association;      // reading K14: 0 exact (K5), 1 extended block (face neighbours)
  double l_scale[32];       // reading K16: class k's length scale is length_scale * l_scale[k]
};

const double kPi = 3.14159265358979323846;

// Eq. (kernel), bracket reading K1: f(r) for r = d/l.
double kernel_f(double r) {
  if (r >= 1.0) return 0.0;
  return (2.0 + std::cos(2.0 * kPi * r)) * (1.0 - r) / 3.0 + std::sin(2.0 * kPi * r) / (2.0 * kPi);
}

// d f / d r, differentiated by hand from kernel_f.
double kernel_df(double r) {
  if (r >= 1.0) return 0.0;
  return -2.0 * kPi * std::sin(2.0 * kPi * r) * (1.0 - r) / 3.0 - (2.0 + std::cos(2.0 * kPi * r)) / 3.0 +
         std::cos(2.0 * kPi * r);
}

typedef std::array<int64_t, 3> Key3;

struct Key3Hash {
  size_t operator()(const Key3& k) const {
    uint64_t h = (uint64_t)k[0] * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)k[1] + 0x7F4A7C159E3779B9ull + (h << 6) + (h >> 2);
    h ^= (uint64_t)k[2] + 0x94D049BB133111EBull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
  return q;
}

// Reading K6: the voxel index of an FP32 coordinate.
int64_t voxel_index(float x, float inv_res) {
  float p = x * inv_res;
  return (int64_t)std::floor(p);
}

struct Block {
  std::vector<double> inc;     // [B^3][K+1] kernel-mass increments
  std::vector<int64_t> pairs;  // [B^3] number of in-support training points seen
};

struct Map {
  Params p;
  std::map<Key3, Block> blocks;  // ordered by block key
};

int nclass(const Params& p) { return p.num_classes + 1; }

// Step a1: sensor frame -> world frame, drop non-finite and out-of-range points.
// Returns indices of kept points and their world coordinates.
void transform_validate(const Params& p, const float* pts, int64_t n, const double* T,
                        std::vector<std::array<float, 3>>& world, std::vector<int64_t>& kept) {
  for (int64_t i = 0; i < n; ++i) {
    float px = pts[3 * i], py = pts[3 * i + 1], pz = pts[3 * i + 2];
    if (!std::isfinite(px) || !std::isfinite(py) || !std::isfinite(pz)) continue;
    double dx = px, dy = py, dz = pz;
    double range = std::sqrt((dx * dx + dy * dy) + dz * dz);
    if (!(range >= p.min_range && range <= p.max_range)) continue;
    std::array<float, 3> w;
    for (int r = 0; r < 3; ++r) {
      double acc = T[4 * r + 0] * dx;
      acc = acc + T[4 * r + 1] * dy;
      acc = acc + T[4 * r + 2] * dz;
      acc = acc + T[4 * r + 3];
      w[r] = (float)acc;
    }
    world.push_back(w);
    kept.push_back(i);
  }
}

struct Sample {
  float x, y, z;
  int32_t label;
};

// Step a2 (Sec. III, reading K3): hits then free samples, in source order.
void build_samples(const Params& p, const std::vector<std::array<float, 3>>& world,
                   const std::vector<int32_t>& labels, const double* T, std::vector<Sample>& out,
                   int64_t* n_free) {
  for (size_t i = 0; i < world.size(); ++i) out.push_back({world[i][0], world[i][1], world[i][2], labels[i]});
  float ox = (float)T[3], oy = (float)T[7], oz = (float)T[11];
  float s = (float)p.free_step;
  int64_t nf = 0;
  for (size_t i = 0; i < world.size(); ++i) {
    float dx = world[i][0] - ox;
    float dy = world[i][1] - oy;
    float dz = world[i][2] - oz;
    float r2 = dx * dx;
    r2 = r2 + dy * dy;
    r2 = r2 + dz * dz;
    float r = std::sqrt(r2);
    for (int64_t j = 1;; ++j) {
      float js = (float)j * s;
      float t = r - js;
      if (!(t > 0.0f)) break;
      float q = t / r;
      float x = ox + dx * q;
      float y = oy + dy * q;
      float z = oz + dz * q;
      out.push_back({x, y, z, 0});
      ++nf;
    }
  }
  *n_free = nf;
}

// Exact mean of FP32 values, rounded once to FP32 (nearest, ties to even),
// with plain big-integer fixed point: every FP32 value is an integer multiple
// of 2^-149, so the sum is an integer number of 2^-149 units (below 2^(128+149+32)
// for up to 2^32 values) held in 32-bit limbs.
struct BigFix {
  static const int kLimbs = 14;  // 448 bits
  uint32_t w[kLimbs];
  BigFix() { std::memset(w, 0, sizeof(w)); }
  void add_shifted(uint64_t m, int shift) {  // += m * 2^shift
    int limb = shift / 32, bit = shift % 32;
    unsigned __int128 v = (unsigned __int128)m << bit;
    uint64_t carry = 0;
    for (int i = limb; i < kLimbs; ++i) {
      uint64_t part = (uint64_t)(v & 0xffffffffu);
      v >>= 32;
      uint64_t t = (uint64_t)w[i] + part + carry;
      w[i] = (uint32_t)t;
      carry = t >> 32;
      if (v == 0 && carry == 0) break;
    }
  }
  void sub(const BigFix& o) {  // *this -= o, requires *this >= o
    int64_t borrow = 0;
    for (int i = 0; i < kLimbs; ++i) {
      int64_t t = (int64_t)w[i] - (int64_t)o.w[i] - borrow;
      borrow = t < 0 ? 1 : 0;
      w[i] = (uint32_t)(t + (borrow << 32));
    }
  }
  bool less(const BigFix& o) const {
    for (int i = kLimbs - 1; i >= 0; --i)
      if (w[i] != o.w[i]) return w[i] < o.w[i];
    return false;
  }
  bool zero() const {
    for (int i = 0; i < kLimbs; ++i)
      if (w[i]) return false;
    return true;
  }
  int bitlen() const {
    for (int i = kLimbs - 1; i >= 0; --i)
      if (w[i]) return 32 * i + 32 - __builtin_clz(w[i]);
    return 0;
  }
  bool bit(int i) const { return i >= 0 && ((w[i / 32] >> (i % 32)) & 1u); }
  // divide by n in place, return the remainder
  uint64_t divmod(uint64_t n) {
    unsigned __int128 r = 0;
    for (int i = kLimbs - 1; i >= 0; --i) {
      unsigned __int128 cur = (r << 32) | w[i];
      w[i] = (uint32_t)(cur / n);
      r = cur % n;
    }
    return (uint64_t)r;
  }
};

float exact_mean_f32(const std::vector<float>& v) {
  BigFix pos, neg;
  for (float x : v) {
    if (x == 0.0f) continue;
    int e;
    float m = std::frexp(std::fabs(x), &e);        // |x| = m 2^e, m in [0.5, 1)
    uint64_t mi = (uint64_t)std::ldexp(m, 24);      // exact: 24-bit integer
    int shift = e - 24 + 149;                       // units of 2^-149
    if (shift < 0) {                                // subnormal: mi has trailing zeros
      mi >>= -shift;
      shift = 0;
    }
    (x < 0.0f ? neg : pos).add_shifted(mi, shift);
  }
  bool negative = pos.less(neg);
  BigFix mag = negative ? neg : pos;
  mag.sub(negative ? pos : neg);
  if (mag.zero()) return 0.0f;
  // quotient Q = mag / n in units of 2^-149, scaled up so that it has >= 26 bits
  const uint64_t n = (uint64_t)v.size();
  BigFix q = mag;
  int up = 0;
  while (q.bitlen() < 64 + 27) {  // shift left by limbs until the quotient is long
    for (int i = BigFix::kLimbs - 1; i > 0; --i) q.w[i] = q.w[i - 1];
    q.w[0] = 0;
    up += 32;
  }
  const bool sticky_div = q.divmod(n) != 0;  // q = floor(mag 2^up / n)
  // value = (q + frac) * 2^(-149 - up)
  const int qb = q.bitlen();
  int exp2 = qb - 1 - 149 - up;  // binary exponent of the leading bit
  int keep = 24;                 // significant bits kept (fewer for subnormal results)
  if (exp2 < -126) keep = 24 - (-126 - exp2);
  if (keep <= 0) keep = 0;
  const int drop = qb - keep;    // >= 2 by construction
  uint64_t mant = 0;
  for (int i = qb - 1; i >= drop; --i) mant = (mant << 1) | (q.bit(i) ? 1u : 0u);
  const bool half = q.bit(drop - 1);
  bool sticky = sticky_div;
  for (int i = 0; i < drop - 1 && !sticky; ++i) sticky = q.bit(i);
  if (half && (sticky || (mant & 1u))) mant += 1;  // round to nearest, ties to even
  const float r = std::ldexp((float)mant, drop - 149 - up);
  return negative ? -r : r;
}

// Step a3 (reading K4): centroid per (ds cell, label).
void downsample(const Params& p, const std::vector<Sample>& in, std::vector<Sample>& out) {
  float inv_ds = (float)(1.0 / p.ds_res);
  struct Members {
    std::vector<float> x, y, z;
  };
  std::map<std::array<int64_t, 4>, Members> cells;
  for (const Sample& s : in) {
    std::array<int64_t, 4> k = {voxel_index(s.x, inv_ds), voxel_index(s.y, inv_ds), voxel_index(s.z, inv_ds),
                                (int64_t)s.label};
    Members& m = cells[k];
    m.x.push_back(s.x);
    m.y.push_back(s.y);
    m.z.push_back(s.z);
  }
  for (auto& kv : cells) {
    const Members& m = kv.second;
    out.push_back({exact_mean_f32(m.x), exact_mean_f32(m.y), exact_mean_f32(m.z), (int32_t)kv.first[3]});
  }
}

// Largest per-class length scale (K16): the stencil must reach every class's support.
double max_length_scale(const Params& p) {
  double lm = 0.0;
  for (int c = 0; c < p.num_classes + 1; ++c) lm = std::max(lm, p.length_scale * p.l_scale[c]);
  return lm;
}

// Step a5, Eq. (alpha_kernel) with Eq. (kernel): stencil enumeration per point.
void accumulate(Map& m, const std::vector<Sample>& train) {
  const Params& p = m.p;
  const int K1 = nclass(p);
  const int64_t B = p.block_edge;
  const float inv_res = (float)(1.0 / p.res);
  const int64_t R = (int64_t)std::ceil(max_length_scale(p) / p.res) + 1;
  for (const Sample& s : train) {
    const double l = p.length_scale * p.l_scale[s.label], l2 = l * l;  // K16
    int64_t kx = voxel_index(s.x, inv_res), ky = voxel_index(s.y, inv_res), kz = voxel_index(s.z, inv_res);
    const Key3 pb = {floor_div(kx, B), floor_div(ky, B), floor_div(kz, B)};  // the point's block (K14)
    for (int64_t a = -R; a <= R; ++a)
      for (int64_t b = -R; b <= R; ++b)
        for (int64_t c = -R; c <= R; ++c) {
          int64_t vx = kx + a, vy = ky + b, vz = kz + c;
          double cx = ((double)vx + 0.5) * p.res;
          double cy = ((double)vy + 0.5) * p.res;
          double cz = ((double)vz + 0.5) * p.res;
          double ex = cx - (double)s.x, ey = cy - (double)s.y, ez = cz - (double)s.z;
          double d2 = ex * ex;
          d2 = d2 + ey * ey;
          d2 = d2 + ez * ez;
          if (!(d2 < l2)) continue;
          Key3 bk = {floor_div(vx, B), floor_div(vy, B), floor_div(vz, B)};
          if (p.association == 1 &&
              std::llabs(bk[0] - pb[0]) + std::llabs(bk[1] - pb[1]) + std::llabs(bk[2] - pb[2]) > 1)
            continue;  // K14: only the voxel's own block and its face neighbours
          double kval = p.sigma0 * p.sigma0_scale[s.label] * kernel_f(std::sqrt(d2) / l);
          Block& blk = m.blocks[bk];
          if (blk.inc.empty()) {
            blk.inc.assign((size_t)(B * B * B * K1), 0.0);
            blk.pairs.assign((size_t)(B * B * B), 0);
          }
          int64_t lx = vx - bk[0] * B, ly = vy - bk[1] * B, lz = vz - bk[2] * B;
          int64_t li = (lz * B + ly) * B + lx;
          blk.inc[(size_t)(li * K1 + s.label)] += kval;
          blk.pairs[(size_t)li] += 1;
        }
  }
}

// Step a5 of the counting model, Eq. (alpha) with reading K11: every training
// point adds 1 to alpha^{y_i} of the voxel that contains it.
void accumulate_counts(Map& m, const std::vector<Sample>& train) {
  const Params& p = m.p;
  const int K1 = nclass(p);
  const int64_t B = p.block_edge;
  const float inv_res = (float)(1.0 / p.res);
  for (const Sample& s : train) {
    const int64_t vx = voxel_index(s.x, inv_res), vy = voxel_index(s.y, inv_res), vz = voxel_index(s.z, inv_res);
    Key3 bk = {floor_div(vx, B), floor_div(vy, B), floor_div(vz, B)};
    Block& blk = m.blocks[bk];
    if (blk.inc.empty()) {
      blk.inc.assign((size_t)(B * B * B * K1), 0.0);
      blk.pairs.assign((size_t)(B * B * B), 0);
    }
    const int64_t li = ((vz - bk[2] * B) * B + (vy - bk[1] * B)) * B + (vx - bk[0] * B);
    blk.inc[(size_t)(li * K1 + s.label)] += 1.0;
    blk.pairs[(size_t)li] += 1;
  }
}

// Step a5 of the map's sensor model.
void update(Map& m, const std::vector<Sample>& train) {
  if (m.p.sensor_model == 1)
    accumulate_counts(m, train);
  else
    accumulate(m, train);
}

// ---------------------------------------------------------------- soft labels (reading K15)
struct SoftSample {
  float x, y, z;
  std::vector<float> w;  // K+1 class weights
};

int argmax_lowest(const std::vector<float>& w) {
  int best = 0;
  for (int c = 1; c < (int)w.size(); ++c)
    if (w[c] > w[best]) best = c;
  return best;
}

// Steps a1-a3 with probability vectors probs [n, K] over the occupied classes.
void soft_training_set(const Params& p, const float* pts, const float* probs, int64_t n, const double* T,
                       std::vector<SoftSample>& train, int64_t* stats) {
  const int K1 = nclass(p);
  std::vector<std::array<float, 3>> world;
  std::vector<int64_t> kept;
  transform_validate(p, pts, n, T, world, kept);
  // a2 on one-label samples (the sample positions do not depend on the label),
  // then the weights: the hit's vector for hits, class 0 for free samples
  std::vector<int32_t> idx(kept.size());
  for (size_t i = 0; i < kept.size(); ++i) idx[i] = (int32_t)i + 1;  // a stand-in label > 0 marks hits
  std::vector<Sample> samples;
  int64_t nf = 0;
  build_samples(p, world, idx, T, samples, &nf);
  const float inv_ds = (float)(1.0 / p.ds_res);
  struct Members {
    std::vector<float> x, y, z;
    std::vector<std::vector<float>> w;  // per class
  };
  std::map<std::array<int64_t, 4>, Members> cells;
  for (const Sample& s : samples) {
    std::vector<float> w((size_t)K1, 0.0f);
    if (s.label > 0) {
      const int64_t src = kept[(size_t)(s.label - 1)];
      for (int c = 1; c < K1; ++c) w[c] = probs[src * (K1 - 1) + (c - 1)];
    } else {
      w[0] = 1.0f;
    }
    std::array<int64_t, 4> k = {voxel_index(s.x, inv_ds), voxel_index(s.y, inv_ds), voxel_index(s.z, inv_ds),
                                (int64_t)argmax_lowest(w)};
    Members& m = cells[k];
    m.x.push_back(s.x);
    m.y.push_back(s.y);
    m.z.push_back(s.z);
    if (m.w.empty()) m.w.assign((size_t)K1, {});
    for (int c = 0; c < K1; ++c) m.w[c].push_back(w[c]);
  }
  for (auto& kv : cells) {
    const Members& m = kv.second;
    SoftSample t{exact_mean_f32(m.x), exact_mean_f32(m.y), exact_mean_f32(m.z), std::vector<float>((size_t)K1)};
    for (int c = 0; c < K1; ++c) t.w[c] = exact_mean_f32(m.w[c]);
    train.push_back(t);
  }
  if (stats) {
    stats[0] = (int64_t)kept.size();
    stats[1] = nf;
    stats[2] = (int64_t)train.size();
  }
}

// Step a5 with weight vectors: every class k gets sigma0 s_k f(d/l) w^k.
void accumulate_soft(Map& m, const std::vector<SoftSample>& train) {
  const Params& p = m.p;
  const int K1 = nclass(p);
  const int64_t B = p.block_edge;
  const float inv_res = (float)(1.0 / p.res);
  const int64_t R = (int64_t)std::ceil(max_length_scale(p) / p.res) + 1;
  for (const SoftSample& s : train) {
    int64_t kx = voxel_index(s.x, inv_res), ky = voxel_index(s.y, inv_res), kz = voxel_index(s.z, inv_res);
    for (int64_t a = -R; a <= R; ++a)
      for (int64_t b = -R; b <= R; ++b)
        for (int64_t c = -R; c <= R; ++c) {
          int64_t vx = kx + a, vy = ky + b, vz = kz + c;
          double ex = ((double)vx + 0.5) * p.res - (double)s.x;
          double ey = ((double)vy + 0.5) * p.res - (double)s.y;
          double ez = ((double)vz + 0.5) * p.res - (double)s.z;
          double d2 = ex * ex;
          d2 = d2 + ey * ey;
          d2 = d2 + ez * ez;
          bool any = false;  // a class with weight whose support (K16) holds the voxel
          for (int k = 0; k < K1; ++k) {
            const double lk = p.length_scale * p.l_scale[k];
            any = any || (s.w[k] != 0.0f && d2 < lk * lk);
          }
          if (!any) continue;
          Key3 bk = {floor_div(vx, B), floor_div(vy, B), floor_div(vz, B)};
          Block& blk = m.blocks[bk];
          if (blk.inc.empty()) {
            blk.inc.assign((size_t)(B * B * B * K1), 0.0);
            blk.pairs.assign((size_t)(B * B * B), 0);
          }
          int64_t li = ((vz - bk[2] * B) * B + (vy - bk[1] * B)) * B + (vx - bk[0] * B);
          for (int k = 0; k < K1; ++k) {
            const double lk = p.length_scale * p.l_scale[k];
            if (s.w[k] != 0.0f && d2 < lk * lk)
              blk.inc[(size_t)(li * K1 + k)] += p.sigma0 * p.sigma0_scale[k] * kernel_f(std::sqrt(d2) / lk) *
                                                (double)s.w[k];
          }
          blk.pairs[(size_t)li] += 1;
        }
  }
}

bool labels_ok(const Params& p, const int32_t* labels, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (labels[i] < 1 || labels[i] > p.num_classes) return false;
  return true;
}

void training_set(const Params& p, const float* pts, const int32_t* labels, int64_t n, const double* T,
                  std::vector<Sample>& train, int64_t* stats) {
  std::vector<std::array<float, 3>> world;
  std::vector<int64_t> kept;
  transform_validate(p, pts, n, T, world, kept);
  std::vector<int32_t> lab(kept.size());
  for (size_t i = 0; i < kept.size(); ++i) lab[i] = labels[kept[i]];
  std::vector<Sample> samples;
  int64_t nf = 0;
  build_samples(p, world, lab, T, samples, &nf);
  downsample(p, samples, train);
  if (stats) {
    stats[0] = (int64_t)kept.size();
    stats[1] = nf;
    stats[2] = (int64_t)train.size();
  }
}

// voxel lookup: returns pointer to increments (or null) and pair count
const double* find_voxel(const Map& m, int64_t vx, int64_t vy, int64_t vz, int64_t* pairs) {
  const int64_t B = m.p.block_edge;
  Key3 bk = {floor_div(vx, B), floor_div(vy, B), floor_div(vz, B)};
  auto it = m.blocks.find(bk);
  if (it == m.blocks.end()) return nullptr;
  int64_t li = ((vz - bk[2] * B) * B + (vy - bk[1] * B)) * B + (vx - bk[0] * B);
  if (pairs) *pairs = it->second.pairs[(size_t)li];
  return &it->second.inc[(size_t)(li * nclass(m.p))];
}

}  // namespace

extern "C" {

typedef struct {
  double res, length_scale, sigma0, alpha0, free_step, ds_res, min_range, max_range, free_thresh, occ_thresh;
  int32_t num_classes, block_edge, sensor_model;
  double sigma0_scale[32];
  int32_t association;
  double l_scale[32];
} orc_params;

static Params conv(const orc_params* q) {
  Params p;
  std::memcpy(&p, q, sizeof(Params));
  return p;
}

void* orc_map_create(const orc_params* q) {
  Map* m = new Map();
  m->p = conv(q);
  return m;
}

void orc_map_destroy(void* h) { delete (Map*)h; }

// Kernel value f(r) (Eq. kernel) and its derivative, for tests.
double orc_kernel_f(double r) { return kernel_f(r); }
double orc_kernel_df(double r) { return kernel_df(r); }

// Exact mean of n FP32 values rounded once to FP32 (reading K4), for tests.
float orc_exact_mean_f32(const float* v, int64_t n) { return exact_mean_f32(std::vector<float>(v, v + n)); }

// a1 only: world coordinates of the kept points; returns the kept count.
int64_t orc_transform(const orc_params* q, const float* pts, int64_t n, const double* T, float* world_out,
                      int64_t* kept_idx) {
  Params p = conv(q);
  std::vector<std::array<float, 3>> world;
  std::vector<int64_t> kept;
  transform_validate(p, pts, n, T, world, kept);
  for (size_t i = 0; i < world.size(); ++i) {
    if (world_out) std::memcpy(world_out + 3 * i, world[i].data(), 12);
    if (kept_idx) kept_idx[i] = kept[i];
  }
  return (int64_t)world.size();
}

// a1 + a2: all samples (hits first, then free samples) in source order.
// Call with out = NULL to get the count.  Returns -1 on a label error.
int64_t orc_samples(const orc_params* q, const float* pts, const int32_t* labels, int64_t n, const double* T,
                    float* xyz_out, int32_t* lab_out, int64_t cap) {
  Params p = conv(q);
  if (!labels_ok(p, labels, n)) return -1;
  std::vector<std::array<float, 3>> world;
  std::vector<int64_t> kept;
  transform_validate(p, pts, n, T, world, kept);
  std::vector<int32_t> lab(kept.size());
  for (size_t i = 0; i < kept.size(); ++i) lab[i] = labels[kept[i]];
  std::vector<Sample> samples;
  int64_t nf = 0;
  build_samples(p, world, lab, T, samples, &nf);
  if (xyz_out) {
    int64_t c = std::min<int64_t>(cap, (int64_t)samples.size());
    for (int64_t i = 0; i < c; ++i) {
      xyz_out[3 * i] = samples[i].x;
      xyz_out[3 * i + 1] = samples[i].y;
      xyz_out[3 * i + 2] = samples[i].z;
      lab_out[i] = samples[i].label;
    }
  }
  return (int64_t)samples.size();
}

// a1 + a2 + a3: the training set (centroids + labels), ordered by (ds cell, label).
// stats (nullable) receives {kept hits, free samples, training points}.
// Returns the training-point count, or -1 on a label error.
int64_t orc_training_set(const orc_params* q, const float* pts, const int32_t* labels, int64_t n, const double* T,
                         float* xyz_out, int32_t* lab_out, int64_t cap, int64_t* stats) {
  Params p = conv(q);
  if (!labels_ok(p, labels, n)) return -1;
  std::vector<Sample> train;
  training_set(p, pts, labels, n, T, train, stats);
  if (xyz_out) {
    int64_t c = std::min<int64_t>(cap, (int64_t)train.size());
    for (int64_t i = 0; i < c; ++i) {
      xyz_out[3 * i] = train[i].x;
      xyz_out[3 * i + 1] = train[i].y;
      xyz_out[3 * i + 2] = train[i].z;
      lab_out[i] = train[i].label;
    }
  }
  return (int64_t)train.size();
}

// a5 on a given training set (world FP32 points, labels in 0..K).
int orc_map_insert_training(void* h, const float* xyz, const int32_t* lab, int64_t n) {
  Map* m = (Map*)h;
  std::vector<Sample> train((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    if (lab[i] < 0 || lab[i] > m->p.num_classes) return -1;
    train[i] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lab[i]};
  }
  update(*m, train);
  return 0;
}

// Whole per-scan update a1..a5.  stats: {kept hits, free samples, training points}.
int orc_map_insert_scan(void* h, const float* pts, const int32_t* labels, int64_t n, const double* T,
                        int64_t* stats) {
  Map* m = (Map*)h;
  if (!labels_ok(m->p, labels, n)) return -1;
  std::vector<Sample> train;
  training_set(m->p, pts, labels, n, T, train, stats);
  update(*m, train);
  return 0;
}

// Reading K15: the soft training set of a scan (probs [n,K] over classes 1..K):
// xyz_out [cap,3], w_out [cap,K+1]; returns the count (writes at most cap).
int64_t orc_soft_training_set(const orc_params* q, const float* pts, const float* probs, int64_t n, const double* T,
                              float* xyz_out, float* w_out, int64_t cap, int64_t* stats) {
  Params p = conv(q);
  const int K1 = nclass(p);
  std::vector<SoftSample> train;
  soft_training_set(p, pts, probs, n, T, train, stats);
  const int64_t c = std::min<int64_t>(cap, (int64_t)train.size());
  for (int64_t i = 0; i < c; ++i) {
    xyz_out[3 * i] = train[i].x;
    xyz_out[3 * i + 1] = train[i].y;
    xyz_out[3 * i + 2] = train[i].z;
    for (int k = 0; k < K1; ++k) w_out[i * K1 + k] = train[i].w[k];
  }
  return (int64_t)train.size();
}

// a5 on a soft training set: xyz [n,3], w [n,K+1].
int orc_map_insert_training_soft(void* h, const float* xyz, const float* w, int64_t n) {
  Map* m = (Map*)h;
  const int K1 = nclass(m->p);
  std::vector<SoftSample> train((size_t)n);
  for (int64_t i = 0; i < n; ++i)
    train[i] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], std::vector<float>(w + i * K1, w + (i + 1) * K1)};
  accumulate_soft(*m, train);
  return 0;
}

// Whole per-scan update with soft labels (a1..a5).  stats as orc_map_insert_scan.
int orc_map_insert_scan_soft(void* h, const float* pts, const float* probs, int64_t n, const double* T,
                             int64_t* stats) {
  Map* m = (Map*)h;
  std::vector<SoftSample> train;
  soft_training_set(m->p, pts, probs, n, T, train, stats);
  accumulate_soft(*m, train);
  return 0;
}

int64_t orc_map_num_blocks(void* h) { return (int64_t)((Map*)h)->blocks.size(); }

// Block keys in ascending lexicographic order.
void orc_map_block_keys(void* h, int64_t* keys) {
  Map* m = (Map*)h;
  int64_t i = 0;
  for (auto& kv : m->blocks) {
    keys[3 * i] = kv.first[0];
    keys[3 * i + 1] = kv.first[1];
    keys[3 * i + 2] = kv.first[2];
    ++i;
  }
}

// Every voxel of every allocated block, sorted by voxel key (x, y, z)
// lexicographically: keys [cnt,3], alpha = alpha_0 + increments [cnt,K+1],
// pair counts [cnt].  Returns the voxel count; NULL buffers: count only.
int64_t orc_map_export(void* h, int64_t* keys, double* alpha, int64_t* pairs) {
  Map* m = (Map*)h;
  const int64_t B = m->p.block_edge, B3 = B * B * B;
  const int K1 = nclass(m->p);
  int64_t cnt = (int64_t)m->blocks.size() * B3;
  if (!keys) return cnt;
  struct Row {
    Key3 k;
    const double* inc;
    int64_t pairs;
  };
  std::vector<Row> rows;
  rows.reserve((size_t)cnt);
  for (auto& kv : m->blocks)
    for (int64_t li = 0; li < B3; ++li) {
      int64_t lx = li % B, ly = (li / B) % B, lz = li / (B * B);
      rows.push_back({{kv.first[0] * B + lx, kv.first[1] * B + ly, kv.first[2] * B + lz},
                      &kv.second.inc[(size_t)(li * K1)], kv.second.pairs[(size_t)li]});
    }
  std::sort(rows.begin(), rows.end(), [](const Row& a, const Row& b) { return a.k < b.k; });
  for (size_t i = 0; i < rows.size(); ++i) {
    for (int d = 0; d < 3; ++d) keys[3 * i + d] = rows[i].k[d];
    for (int c = 0; c < K1; ++c) alpha[i * K1 + c] = m->p.alpha0 + rows[i].inc[c];
    if (pairs) pairs[i] = rows[i].pairs;
  }
  return cnt;
}

// alpha (with prior) at given voxel keys; voxels outside allocated blocks read the prior.
void orc_map_alpha_at(void* h, const int64_t* keys, int64_t n, double* alpha, int64_t* pairs) {
  Map* m = (Map*)h;
  const int K1 = nclass(m->p);
  for (int64_t i = 0; i < n; ++i) {
    int64_t pc = 0;
    const double* inc = find_voxel(*m, keys[3 * i], keys[3 * i + 1], keys[3 * i + 2], &pc);
    for (int c = 0; c < K1; ++c) alpha[i * K1 + c] = m->p.alpha0 + (inc ? inc[c] : 0.0);
    if (pairs) pairs[i] = inc ? pc : 0;
  }
}

// Brute force: alpha at given voxel keys from a training set, summing over
// every training point (no neighbour search).  For sampled checks at full size.
void orc_alpha_bruteforce(const orc_params* q, const float* xyz, const int32_t* lab, int64_t n,
                          const int64_t* keys, int64_t nq, double* alpha, int64_t* pairs) {
  Params p = conv(q);
  const int K1 = nclass(p);
  for (int64_t v = 0; v < nq; ++v) {
    double cx = ((double)keys[3 * v] + 0.5) * p.res;
    double cy = ((double)keys[3 * v + 1] + 0.5) * p.res;
    double cz = ((double)keys[3 * v + 2] + 0.5) * p.res;
    for (int c = 0; c < K1; ++c) alpha[v * K1 + c] = p.alpha0;
    int64_t pc = 0;
    for (int64_t i = 0; i < n; ++i) {
      double ex = cx - (double)xyz[3 * i], ey = cy - (double)xyz[3 * i + 1], ez = cz - (double)xyz[3 * i + 2];
      double d2 = ex * ex;
      d2 = d2 + ey * ey;
      d2 = d2 + ez * ez;
      const double l = p.length_scale * p.l_scale[lab[i]], l2 = l * l;  // K16
      if (!(d2 < l2)) continue;
      alpha[v * K1 + lab[i]] += p.sigma0 * p.sigma0_scale[lab[i]] * kernel_f(std::sqrt(d2) / l);
      ++pc;
    }
    if (pairs) pairs[v] = pc;
  }
}

// Eq. (alpha_kernel) at arbitrary query points (Sec. IV: the continuous model
// can be queried at any resolution): alpha [nq,K+1] = alpha_0 + sum over all
// training points within l of sigma0 s_k f(d/l) (exact association).
void orc_alpha_at_points(const orc_params* q, const float* xyz, const int32_t* lab, int64_t n, const double* pts,
                         int64_t nq, double* alpha) {
  Params p = conv(q);
  const int K1 = nclass(p);
  for (int64_t v = 0; v < nq; ++v) {
    for (int c = 0; c < K1; ++c) alpha[v * K1 + c] = p.alpha0;
    for (int64_t i = 0; i < n; ++i) {
      double ex = pts[3 * v] - (double)xyz[3 * i], ey = pts[3 * v + 1] - (double)xyz[3 * i + 1],
             ez = pts[3 * v + 2] - (double)xyz[3 * i + 2];
      double d2 = ex * ex;
      d2 = d2 + ey * ey;
      d2 = d2 + ez * ez;
      const double l = p.length_scale * p.l_scale[lab[i]], l2 = l * l;  // K16
      if (!(d2 < l2)) continue;
      alpha[v * K1 + lab[i]] += p.sigma0 * p.sigma0_scale[lab[i]] * kernel_f(std::sqrt(d2) / l);
    }
  }
}

// Read-off, Eq. (mode), Eq. (variance), Sec. V-C; reading K7 for the state.
// probs = E[theta] [q,K+1]; var, mode nullable [q,K+1]; label, state [q]; p_occ [q].
void orc_map_query(void* h, const float* xyz, int64_t nq, double* probs, double* var, double* mode,
                   int32_t* label, double* p_occ, int32_t* state) {
  Map* m = (Map*)h;
  const Params& p = m->p;
  const int K1 = nclass(p);
  const float inv_res = (float)(1.0 / p.res);
  std::vector<double> a((size_t)K1);
  for (int64_t i = 0; i < nq; ++i) {
    int64_t vx = voxel_index(xyz[3 * i], inv_res), vy = voxel_index(xyz[3 * i + 1], inv_res),
            vz = voxel_index(xyz[3 * i + 2], inv_res);
    const double* inc = find_voxel(*m, vx, vy, vz, nullptr);
    double mass = 0.0;
    for (int c = 0; c < K1; ++c) {
      double d = inc ? inc[c] : 0.0;
      mass += d;
      a[c] = p.alpha0 + d;
    }
    double S = 0.0;
    for (int c = 0; c < K1; ++c) S += a[c];
    bool mode_ok = true;
    for (int c = 0; c < K1; ++c) mode_ok = mode_ok && (a[c] > 1.0);
    int best = 0;
    for (int c = 0; c < K1; ++c) {
      double e = a[c] / S;
      probs[i * K1 + c] = e;
      if (var) var[i * K1 + c] = e * (1.0 - e) / (S + 1.0);
      if (mode) mode[i * K1 + c] = mode_ok ? (a[c] - 1.0) / (S - (double)K1) : NAN;
      if (a[c] > a[best]) best = c;
    }
    double po = 0.0;
    for (int c = 1; c < K1; ++c) po += a[c] / S;
    if (label) label[i] = best;
    if (p_occ) p_occ[i] = po;
    if (state) {
      int st = 1;
      if (mass > 0.0) st = po < p.free_thresh ? 0 : (po > p.occ_thresh ? 2 : 1);
      state[i] = st;
    }
  }
}

// Differentiable form.  Held-out log-likelihood
//   LL = sum_h log( alpha_{v(h)}^{y_h} / sum_k alpha_{v(h)}^k )
// with alpha from the training set (Eq. alpha_kernel), and its exact gradient
// with respect to l, sigma0 and every training point's coordinates.
// Training coordinates are FP64 here so that finite differences can move them
// by less than an FP32 ulp; the stencil centre is the voxel of (float)x.
// held_xyz are world coordinates; v(h) is the voxel containing the point.
// Returns LL; grad_l, grad_sigma0, grad_xyz ([n,3]) and grad_scale (dLL/d
// sigma0_scale[k], [K+1]) are nullable.
static double heldout_grad(const orc_params* q, const double* xyz, const int32_t* lab, int64_t n,
                           const float* held_xyz, const int32_t* held_lab, int64_t nh, double* grad_l,
                           double* grad_sigma0, double* grad_xyz, double* grad_scale) {
  Params p = conv(q);
  const int K1 = nclass(p);
  const float inv_res = (float)(1.0 / p.res);
  const double l = p.length_scale, l2 = l * l;
  const int64_t R = (int64_t)std::ceil(l / p.res) + 1;

  // 1. forward: alpha increments per voxel (Eq. alpha_kernel)
  std::unordered_map<Key3, std::vector<double>, Key3Hash> inc;
  for (int64_t i = 0; i < n; ++i) {
    double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    int64_t kx = voxel_index((float)x, inv_res), ky = voxel_index((float)y, inv_res),
            kz = voxel_index((float)z, inv_res);
    for (int64_t da = -R; da <= R; ++da)
      for (int64_t db = -R; db <= R; ++db)
        for (int64_t dc = -R; dc <= R; ++dc) {
          Key3 v = {kx + da, ky + db, kz + dc};
          double ex = ((double)v[0] + 0.5) * p.res - x;
          double ey = ((double)v[1] + 0.5) * p.res - y;
          double ez = ((double)v[2] + 0.5) * p.res - z;
          double d2 = ex * ex;
          d2 = d2 + ey * ey;
          d2 = d2 + ez * ez;
          if (!(d2 < l2)) continue;
          std::vector<double>& a = inc[v];
          if (a.empty()) a.assign((size_t)K1, 0.0);
          a[(size_t)lab[i]] += p.sigma0 * p.sigma0_scale[lab[i]] * kernel_f(std::sqrt(d2) / l);
        }
  }

  // 2. LL and dLL/dalpha at the voxels holding held-out points
  std::unordered_map<Key3, std::vector<double>, Key3Hash> g;
  double LL = 0.0;
  std::vector<double> a((size_t)K1);
  for (int64_t h = 0; h < nh; ++h) {
    Key3 v = {voxel_index(held_xyz[3 * h], inv_res), voxel_index(held_xyz[3 * h + 1], inv_res),
              voxel_index(held_xyz[3 * h + 2], inv_res)};
    auto it = inc.find(v);
    double S = 0.0;
    for (int c = 0; c < K1; ++c) {
      a[c] = p.alpha0 + (it != inc.end() ? it->second[(size_t)c] : 0.0);
      S += a[c];
    }
    int y = held_lab[h];
    LL += std::log(a[y]) - std::log(S);
    std::vector<double>& gv = g[v];
    if (gv.empty()) gv.assign((size_t)K1, 0.0);
    for (int c = 0; c < K1; ++c) gv[c] -= 1.0 / S;
    gv[y] += 1.0 / a[y];
  }
  if (!grad_l && !grad_sigma0 && !grad_xyz && !grad_scale) return LL;

  // 3. chain rule through every in-support pair (Eq. kernel); class k's kernel
  //    is s sigma0 f with s = sigma0_scale[k]
  double gl = 0.0, gs = 0.0;
  std::vector<double> gsc((size_t)K1, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    int64_t kx = voxel_index((float)x, inv_res), ky = voxel_index((float)y, inv_res),
            kz = voxel_index((float)z, inv_res);
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int64_t da = -R; da <= R; ++da)
      for (int64_t db = -R; db <= R; ++db)
        for (int64_t dc = -R; dc <= R; ++dc) {
          Key3 v = {kx + da, ky + db, kz + dc};
          double ex = ((double)v[0] + 0.5) * p.res - x;
          double ey = ((double)v[1] + 0.5) * p.res - y;
          double ez = ((double)v[2] + 0.5) * p.res - z;
          double d2 = ex * ex;
          d2 = d2 + ey * ey;
          d2 = d2 + ez * ez;
          if (!(d2 < l2)) continue;
          auto it = g.find(v);
          if (it == g.end()) continue;
          double G = it->second[(size_t)lab[i]];
          const double sc = p.sigma0_scale[lab[i]];
          double d = std::sqrt(d2), r = d / l;
          double df = kernel_df(r);
          gs += G * sc * kernel_f(r);
          gsc[(size_t)lab[i]] += G * p.sigma0 * kernel_f(r);
          gl += G * sc * p.sigma0 * df * (-d / l2);
          if (d > 0.0) {
            // d = |c - x|, so dd/dx = (x - c)/d = -e/d
            double coef = G * sc * p.sigma0 * df / (l * d);
            gx -= coef * ex;
            gy -= coef * ey;
            gz -= coef * ez;
          }
        }
    if (grad_xyz) {
      grad_xyz[3 * i] = gx;
      grad_xyz[3 * i + 1] = gy;
      grad_xyz[3 * i + 2] = gz;
    }
  }
  if (grad_l) *grad_l = gl;
  if (grad_sigma0) *grad_sigma0 = gs;
  if (grad_scale)
    for (int c = 0; c < K1; ++c) grad_scale[c] = gsc[(size_t)c];
  return LL;
}

double orc_heldout_grad(const orc_params* q, const double* xyz, const int32_t* lab, int64_t n,
                        const float* held_xyz, const int32_t* held_lab, int64_t nh, double* grad_l,
                        double* grad_sigma0, double* grad_xyz) {
  return heldout_grad(q, xyz, lab, n, held_xyz, held_lab, nh, grad_l, grad_sigma0, grad_xyz, nullptr);
}

// dLL/d sigma0_scale[k] for every class k ([K+1]); returns LL.
double orc_heldout_grad_scale(const orc_params* q, const double* xyz, const int32_t* lab, int64_t n,
                              const float* held_xyz, const int32_t* held_lab, int64_t nh, double* grad_scale) {
  return heldout_grad(q, xyz, lab, n, held_xyz, held_lab, nh, nullptr, nullptr, nullptr, grad_scale);
}

// Held-out log-likelihood alone (same definition as orc_heldout_grad), for
// the finite-difference checks.
double orc_heldout_ll(const orc_params* q, const double* xyz, const int32_t* lab, int64_t n, const float* held_xyz,
                      const int32_t* held_lab, int64_t nh) {
  return heldout_grad(q, xyz, lab, n, held_xyz, held_lab, nh, nullptr, nullptr, nullptr, nullptr);
}

}  // extern "C"
