// Differentiable form of the S-BKI update.
//
// Forward: alpha_v^k = alpha_0 + sum_{i: y_i = k, d_iv < l} sigma0 f(d_iv / l)
// (Eq. alpha_kernel with Eq. kernel, d_iv = |c_v - x_i|).  Given an upstream
// gradient G_v^k = dL/dalpha_v^k, held per voxel in a pool-shaped buffer
// (same block slots and layout as alpha), the backward pass visits every
// in-support pair once more, recomputing the kernel instead of storing pairs:
//   dL/dsigma0 += G f(r)
//   dL/dl      += G sigma0 f'(r) (-d / l^2)
//   dL/dx_i    += G sigma0 f'(r) (x_i - c_v) / (l d)
// with r = d/l, f' = df/dr = -u^4 D(u^2), u = 1 - r (kernel_poly.cuh); the
// x_i term is written with the unit vector (x_i - c_v)/d, which stays bounded
// as d -> 0 (f'(0) = 0).  With per-class kernel scales (class k's kernel is
// sigma0 s_k f) every term of a class-k point carries s_k, applied once per
// point, and dL/ds_k = sigma0 sum_{pairs of class-k points} G f.
//
// The held-out log-likelihood of the differentiable form scores held-out
// labelled points at the voxel containing them:
//   LL = sum_h log(alpha_{v(h)}^{y_h} / sum_k alpha_{v(h)}^k),
//   dLL/dalpha_v^k = sum_{h in v} ([k = y_h] / alpha_v^{y_h} - 1 / sum_j alpha_v^j)
// (the Dirichlet mean of Eq. (variance) as the predictive probability).
//
// Enumeration of pairs is the one of the point-major accumulation (same
// candidate lists, same FP32 test with the FP64 re-decision band), so the
// backward pass sees exactly the pairs the forward pass added.
#include <algorithm>
#include <climits>

#include "kernel_value.cuh"
#include "point_common.cuh"

namespace sbki {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kAxisMax = 15;
constexpr int kYZMax = kAxisMax * kAxisMax;
constexpr float kFar = 1.0e30f;

// ---------------------------------------------------------------- held-out log-likelihood
struct LLArgs {
  Geom g;
  float alpha0;
  const unsigned long long* hkeys;
  const int32_t* hvals;
  int64_t hash_cap;
  const float* alpha;
  float* grad;  // nullable: accumulate dLL/dalpha
  const float* xyz;
  const int32_t* labels;
  int64_t h;
  double* ll;  // device accumulator
  int map;
  DevCounters* dc;
};

__global__ void __launch_bounds__(256) heldout_kernel(LLArgs a) {
  const Geom& g = a.g;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double term = 0.0;
  if (i < a.h) {
    const int y = a.labels[i];
    if (y < 0 || y >= g.K1) {
      set_error(a.dc, SBKI_ERR_LABEL_RANGE);
    } else {
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
        pool = find_pool_slot(a.hkeys, a.hvals, a.hash_cap,
                              pack_block(v[0] >> g.B_shift, v[1] >> g.B_shift, v[2] >> g.B_shift, a.map));
        const int m = g.B - 1;
        local = (((v[2] & m) << g.B_shift) + (v[1] & m)) * g.B + (v[0] & m);
      }
      const float* inc = pool >= 0 ? a.alpha + (size_t)pool * g.K1 * g.B3 + local : nullptr;
      double S = 0.0;
      for (int k = 0; k < g.K1; ++k) S += (double)(a.alpha0 + (inc ? inc[(size_t)k * g.B3] : 0.f));
      const double ay = (double)(a.alpha0 + (inc ? inc[(size_t)y * g.B3] : 0.f));
      term = log(ay) - log(S);
      if (a.grad && pool >= 0) {
        float* gb = a.grad + (size_t)pool * g.K1 * g.B3 + local;
        const float mS = (float)(-1.0 / S);
        for (int k = 0; k < g.K1; ++k) red_add_if(true, gb + (size_t)k * g.B3, mS);
        red_add_if(true, gb + (size_t)y * g.B3, (float)(1.0 / ay));
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) term += __shfl_down_sync(0xffffffffu, term, o);
  if ((threadIdx.x & 31) == 0 && term != 0.0) atomicAdd(a.ll, term);
}

// ---------------------------------------------------------------- upstream gradient at voxel keys
__global__ void __launch_bounds__(256) grad_scatter_kernel(Geom g, const unsigned long long* hkeys,
                                                           const int32_t* hvals, int64_t hash_cap,
                                                           const int64_t* keys, const float* grad, int64_t count,
                                                           int map, float* gpool, unsigned long long* missed) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const int64_t kx = keys[3 * q], ky = keys[3 * q + 1], kz = keys[3 * q + 2];
  const int64_t lim = kKeyLimit;
  int32_t pool = -1;
  if (kx > -lim && kx < lim && ky > -lim && ky < lim && kz > -lim && kz < lim)
    pool = find_pool_slot(hkeys, hvals, hash_cap,
                          pack_block((int32_t)(kx >> g.B_shift), (int32_t)(ky >> g.B_shift), (int32_t)(kz >> g.B_shift),
                                     map));
  if (pool < 0) {
    atomicAdd(missed, 1ull);
    return;
  }
  const int m = g.B - 1;
  const int local = ((((int)kz & m) << g.B_shift) + ((int)ky & m)) * g.B + ((int)kx & m);
  float* gb = gpool + (size_t)pool * g.K1 * g.B3 + local;
  for (int k = 0; k < g.K1; ++k) red_add_if(true, gb + (size_t)k * g.B3, grad[q * g.K1 + k]);
}

// ---------------------------------------------------------------- backward through Eq. (kernel)
struct BwdArgs {
  Geom g;
  const float4* xyzl;  // training set (x, y, z, label)
  int64_t p;
  const unsigned long long* hkeys;
  const int32_t* hvals;
  int64_t hash_cap;
  const float* gpool;  // dL/dalpha, [pool][K1][B3]
  const uint32_t* ctab;
  const int32_t* clen;
  int tpad, R;
  uint32_t recip_na;
  double* acc;         // [2]: sum s G f, sum s G u^4 D d (s: the point's class scale)
  double* acc_class;   // nullable [32]: per class of the point, sum G f
  float* grad_xyz;     // nullable [p][3]: (sigma0 / l) sum G u^4 D (c_v - x)/d
  float xyz_scale;     // sigma0 / l
  DevCounters* dc;
};

struct BwdTables {
  float4 x[kAxisMax + 1];  // (e_x^2, address part, e_x, 0); entry 2R+1 is the padding row
  float4 yz[kYZMax];       // (e_y^2 + e_z^2, address part, e_y, e_z)
  const float* blk[27];    // gpool + (pool (K+1) + y_i) B^3, or null
};

// Adds the warp's sum of one point's lane terms v into the warp's class row
// (lane 0 writes; every lane of the warp calls it).
__device__ __forceinline__ void add_class_sum(double* row, int label, float v, int lane) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0 && label < 32) row[label] += (double)v;
}

__global__ void __launch_bounds__(kThreads, 3) backward_kernel(BwdArgs a) {
  __shared__ BwdTables s_tab[kWarps];
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int R = a.R, na = 2 * R + 1;
  BwdTables& t = s_tab[wid];
  __shared__ double s_cls[kWarps][32];  // per warp: sum G f by class (only with acc_class)
  if (a.dc->err != 0) return;
  if (lane == 0) t.x[na] = make_float4(kFar, __int_as_float(0), 0.f, 0.f);
  s_cls[wid][lane] = 0.0;
  double acc_f = 0.0, acc_l = 0.0;
  for (int64_t i = gw; i < a.p; i += nw) {
    const float4 p = a.xyzl[i];
    const int lm = label_of(p.w);  // label + 32 * map
    const int label = lm & ((1 << kLabelBits) - 1), map = lm >> kLabelBits;
    const PointFrame f = point_frame(p.x, p.y, p.z, R, g);
    const uint32_t* tab = a.ctab + f.part * a.tpad;
    if (lane < na) {
      const float e = centre_offset_at(lane - R, f.hi[0], f.lo[0], g);
      t.x[lane] = make_float4(__fmul_rn(e, e), __int_as_float(xpart(f, lane, R, g)), e, 0.f);
    }
    for (int q = lane; q < na * na; q += 32) {
      const int jy = (int)small_div((uint32_t)q, a.recip_na), jz = q - jy * na;
      const float ey = centre_offset_at(jy - R, f.hi[1], f.lo[1], g);
      const float ez = centre_offset_at(jz - R, f.hi[2], f.lo[2], g);
      t.yz[q] = make_float4(__fadd_rn(__fmul_rn(ey, ey), __fmul_rn(ez, ez)), __int_as_float(yzpart(f, jy, jz, R, g)),
                            ey, ez);
    }
    if (lane < 27) {
      const int32_t pool = (label < g.K1 && map < kMaxMaps) ? digit_pool(f, lane, map, a.hkeys, a.hvals, a.hash_cap)
                                                            : -1;
      t.blk[lane] = pool >= 0 ? a.gpool + ((size_t)pool * g.K1 + label) * g.B3 : nullptr;
    }
    __syncwarp();
    float sf = 0.f, sl = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
    const int len = __ldg(a.clen + f.part);
    for (int k = lane; k - lane < len; k += 32) {  // warp-uniform trip count
      const uint32_t ent = __ldg(tab + k);
      const float4 ex = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(t.x) + 2u * (ent & 0xffu));
      const float4 eyz =
          *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(t.yz) + 2u * ((ent >> 8) & 0x7ffu));
      const float d2 = __fadd_rn(ex.x, eyz.x);
      const int pk = __float_as_int(ex.y) + __float_as_int(eyz.y);
      bool in = d2 < g.l2_lo;
      const bool band = !in && d2 < g.l2_hi;
      if (__any_sync(0xffffffffu, band)) {
        if (band)
          in = in_support64_call(f.v0[0] + entry_jx(ent) - R, f.v0[1] + entry_jy(ent) - R,
                                 f.v0[2] + entry_jz(ent) - R, p.x, p.y, p.z, g.res64, g.l2_64);
      }
      const float* base = t.blk[pk & 0xff];
      if (in && base != nullptr) {
        const float G = __ldg(base + (pk >> 8));
        const float inv_d = rsqrtf(fmaxf(d2, 1e-30f));
        const float d = d2 * inv_d;
        const float u = fmaxf(__fmaf_rn(-d, g.inv_l, 1.0f), 0.0f);
        const float w = u * u;
        const float u4 = w * w;
        const float s = G * u4 * kernel_dq(w);  // -G df/dr
        sf = __fmaf_rn(G * u4 * u, kernel_q(w), sf);
        sl = __fmaf_rn(s, d, sl);
        // e = c_v - x and dr/dx = -e/(l d), so dk/dx = sigma0 u^4 D e / (l d)
        const float c = s * inv_d;
        sx = __fmaf_rn(c, ex.z, sx);
        sy = __fmaf_rn(c, eyz.z, sy);
        sz = __fmaf_rn(c, eyz.w, sz);
      }
    }
    const float s = label < g.K1 ? g.scale_k[label] : 0.f;  // the class's kernel scale
    acc_f += (double)s * (double)sf;
    acc_l += (double)s * (double)sl;
    if (a.acc_class) add_class_sum(s_cls[wid], label, sf, lane);
    if (a.grad_xyz) {
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
        sz += __shfl_down_sync(0xffffffffu, sz, o);
      }
      if (lane == 0) {
        a.grad_xyz[3 * i] = sx * (s * a.xyz_scale);
        a.grad_xyz[3 * i + 1] = sy * (s * a.xyz_scale);
        a.grad_xyz[3 * i + 2] = sz * (s * a.xyz_scale);
      }
    }
    __syncwarp();  // the tables are rewritten for the next point
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc_f += __shfl_down_sync(0xffffffffu, acc_f, o);
    acc_l += __shfl_down_sync(0xffffffffu, acc_l, o);
  }
  if (lane == 0) {
    atomicAdd(&a.acc[0], acc_f);
    atomicAdd(&a.acc[1], acc_l);
  }
  if (a.acc_class) {
    __syncwarp();
    if (s_cls[wid][lane] != 0.0) atomicAdd(&a.acc_class[lane], s_cls[wid][lane]);
  }
}

// The same pass for 2R + 1 <= 8 with the set-up of the fast accumulation: a
// warp takes kBwdChunk consecutive training points in groups of up to
// kBwdGroup; for a group, three lanes per point (one per axis) form the
// axis's offset rows (e^2, address part, e) for offsets -R..R at once, with
// the point's sub-voxel part, block and voxel.  Then, point by point, the
// warp combines the Y and Z rows into YZ rows, refreshes the pool slots of
// the 27 blocks around the point's block when the block (or map) changed,
// and sweeps the candidate list in unrolled rounds of 32.  Rows, tests and
// kernel arithmetic are the ones of backward_kernel, so both give the same
// pairs and the same FP32 terms.
constexpr int kBwdGroup = 10;  // points whose rows one warp forms at once (3 lanes each)
constexpr int kBwdChunk = 20;  // consecutive training points per warp
constexpr int kBwdAxis = 8;    // rows per axis: 2R + 1 <= 7 offsets and the padding row

struct alignas(16) BwdRows {
  float4 r[3][kBwdAxis];  // per axis: (e^2, address part, e, 0) of offset j - R; r[0][2R + 1] is the padding row
  int pt[4];              // sub-voxel part per axis, label word
  int blk[4];             // block per axis
  int v0[4];              // voxel per axis
};

struct BwdFastTables {
  BwdRows pts[kBwdGroup];
  float4 yz[kBwdAxis * kBwdAxis];  // (e_y^2 + e_z^2, address part, e_y, e_z) of the point being swept
  const float* blk[27];            // gpool + (pool (K+1) + y_i) B^3, or null
};

// One candidate of one point: the pair's terms added into sf, sl, sx, sy, sz
// (the point's coordinates are loaded again only on the FP64 re-decision).
__device__ __forceinline__ void bwd_candidate(const BwdArgs& a, const BwdFastTables& t, const BwdRows& pr,
                                              uint32_t ent, int64_t i, float& sf, float& sl, float& sx, float& sy,
                                              float& sz) {
  const Geom& g = a.g;
  const float4 ex = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(pr.r[0]) + 2u * (ent & 0xffu));
  const float4 eyz = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(t.yz) + 2u * ((ent >> 8) & 0x7ffu));
  const float d2 = __fadd_rn(ex.x, eyz.x);
  const int pk = __float_as_int(ex.y) + __float_as_int(eyz.y);
  bool in = d2 < g.l2_lo;
  const bool band = !in && d2 < g.l2_hi;
  if (__any_sync(0xffffffffu, band)) {
    if (band) {
      const float4 p = a.xyzl[i];
      in = in_support64_call(pr.v0[0] + entry_jx(ent) - a.R, pr.v0[1] + entry_jy(ent) - a.R,
                             pr.v0[2] + entry_jz(ent) - a.R, p.x, p.y, p.z, g.res64, g.l2_64);
    }
  }
  const float* base = t.blk[pk & 0xff];
  if (in && base != nullptr) {
    const float G = __ldg(base + (pk >> 8));
    const float inv_d = rsqrtf(fmaxf(d2, 1e-30f));
    const float d = d2 * inv_d;
    const float u = fmaxf(__fmaf_rn(-d, g.inv_l, 1.0f), 0.0f);
    const float w = u * u;
    const float u4 = w * w;
    const float s = G * u4 * kernel_dq(w);  // -G df/dr
    sf = __fmaf_rn(G * u4 * u, kernel_q(w), sf);
    sl = __fmaf_rn(s, d, sl);
    const float c = s * inv_d;
    sx = __fmaf_rn(c, ex.z, sx);
    sy = __fmaf_rn(c, eyz.z, sy);
    sz = __fmaf_rn(c, eyz.w, sz);
  }
}

// kNit > 0: lists of exactly kNit x 32 entries, unrolled; 0: any length
template <int kNit>
__global__ void __launch_bounds__(kThreads, 3) backward_fast_kernel(BwdArgs a) {
  __shared__ BwdFastTables s_tab[kWarps];
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int R = a.R, na = 2 * R + 1, m = g.B - 1;
  BwdFastTables& t = s_tab[wid];
  __shared__ double s_cls[kWarps][32];  // per warp: sum G f by class (only with acc_class)
  if (a.dc->err != 0) return;
  s_cls[wid][lane] = 0.0;
  // this lane's point of a group and axis (lanes 30, 31 form no rows)
  const int gl = lane / 3, ax = lane - 3 * (lane / 3);
  const int axshift = ax == 0 ? 0 : (ax == 1 ? g.B_shift : 2 * g.B_shift);
  const int dmul = ax == 0 ? 1 : (ax == 1 ? 3 : 9);
  int cb[3] = {INT_MIN, INT_MIN, INT_MIN}, cmap = -1;  // block and map the cached slots belong to
  int32_t pool = -1;                                   // lanes 0..26: slot of block digit `lane`
  double acc_f = 0.0, acc_l = 0.0;
  for (int64_t c = gw; c * kBwdChunk < a.p; c += nw) {
    const int64_t c1 = min(a.p, c * kBwdChunk + kBwdChunk);
    for (int64_t g0 = c * kBwdChunk; g0 < c1; g0 += kBwdGroup) {
      const int gn = (int)min(c1 - g0, (int64_t)kBwdGroup);  // warp-uniform
      // 1. rows of every point of the group, three lanes per point
      if (gl < gn) {
        const float4 p = a.xyzl[g0 + gl];
        const float xa = ax == 0 ? p.x : (ax == 1 ? p.y : p.z);
        const int v0 = floor_small(__fmul_rn(xa, g.inv_res));
        float hi, lo;
        centre_offset0(v0, xa, g, hi, lo);
        const float phi = 0.5f - __fmul_rn(__fadd_rn(hi, lo), g.inv_res);
        const int b0 = v0 >> g.B_shift;
        BwdRows& pr = t.pts[gl];
#pragma unroll
        for (int j = 0; j < kBwdAxis; ++j) {
          if (j < na) {
            const float e = centre_offset_at(j - R, hi, lo, g);
            const int v = v0 + j - R;
            pr.r[ax][j] = make_float4(__fmul_rn(e, e),
                                      __int_as_float(dmul * ((v >> g.B_shift) - (b0 - 1)) | ((v & m) << (axshift + 8))),
                                      e, 0.f);
          }
        }
        if (ax == 0) pr.r[0][na] = make_float4(kFar, __int_as_float(0), 0.f, 0.f);
        pr.pt[ax] = min(kParts - 1, max(0, floor_small(phi * (float)kParts)));
        pr.blk[ax] = b0;
        pr.v0[ax] = v0;
        if (ax == 0) pr.pt[3] = label_of(p.w);
      }
      __syncwarp();
      // 2. point by point: YZ rows, block slots, candidate sweeps, the point's terms
      for (int k = 0; k < gn; ++k) {
        const BwdRows& pr = t.pts[k];
        const int4 ip = *reinterpret_cast<const int4*>(pr.pt);
        const int4 ib = *reinterpret_cast<const int4*>(pr.blk);
        const int part = ip.x + kParts * (ip.y + kParts * ip.z);
        const int label = ip.w & ((1 << kLabelBits) - 1), map = ip.w >> kLabelBits;
        for (int q0 = 0; q0 < na * na; q0 += 32) {
          const int q = min(q0 + lane, na * na - 1);
          const int jy = (int)small_div((uint32_t)q, a.recip_na), jz = q - jy * na;
          const float4 ry = pr.r[1][jy], rz = pr.r[2][jz];
          if (q0 + lane < na * na)
            t.yz[q] = make_float4(__fadd_rn(ry.x, rz.x), __int_as_float(__float_as_int(ry.y) + __float_as_int(rz.y)),
                                  ry.z, rz.z);
        }
        if (ib.x != cb[0] || ib.y != cb[1] || ib.z != cb[2] || map != cmap) {  // warp-uniform
          cb[0] = ib.x;
          cb[1] = ib.y;
          cb[2] = ib.z;
          cmap = map;
          pool = -1;
          if (lane < 27 && map < kMaxMaps)
            pool = find_pool_slot(a.hkeys, a.hvals, a.hash_cap,
                                  pack_block(ib.x - 1 + lane % 3, ib.y - 1 + (lane / 3) % 3, ib.z - 1 + lane / 9, map));
        }
        if (lane < 27)
          t.blk[lane] = (pool >= 0 && label < g.K1) ? a.gpool + ((size_t)pool * g.K1 + label) * g.B3 : nullptr;
        __syncwarp();
        const uint32_t* tab = a.ctab + part * a.tpad;
        const int len = __ldg(a.clen + part);
        const int64_t i = g0 + k;
        float sf = 0.f, sl = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
        if (kNit > 0) {
          uint32_t ent[kNit > 0 ? kNit : 1];
#pragma unroll
          for (int it = 0; it < kNit; ++it) ent[it] = it * 32 < len ? __ldg(tab + it * 32 + lane) : 0u;
#pragma unroll
          for (int it = 0; it < kNit; ++it)
            if (it * 32 < len) bwd_candidate(a, t, pr, ent[it], i, sf, sl, sx, sy, sz);  // warp-uniform
        } else {
          for (int q = lane; q - lane < len; q += 32) bwd_candidate(a, t, pr, __ldg(tab + q), i, sf, sl, sx, sy, sz);
        }
        const float s = label < g.K1 ? g.scale_k[label] : 0.f;  // the class's kernel scale
        acc_f += (double)s * (double)sf;
        acc_l += (double)s * (double)sl;
        if (a.acc_class) add_class_sum(s_cls[wid], label, sf, lane);
        if (a.grad_xyz) {
          for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_down_sync(0xffffffffu, sx, o);
            sy += __shfl_down_sync(0xffffffffu, sy, o);
            sz += __shfl_down_sync(0xffffffffu, sz, o);
          }
          if (lane == 0) {
            a.grad_xyz[3 * i] = sx * (s * a.xyz_scale);
            a.grad_xyz[3 * i + 1] = sy * (s * a.xyz_scale);
            a.grad_xyz[3 * i + 2] = sz * (s * a.xyz_scale);
          }
        }
        __syncwarp();  // the YZ rows and block pointers are rewritten for the next point
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc_f += __shfl_down_sync(0xffffffffu, acc_f, o);
    acc_l += __shfl_down_sync(0xffffffffu, acc_l, o);
  }
  if (lane == 0) {
    atomicAdd(&a.acc[0], acc_f);
    atomicAdd(&a.acc[1], acc_l);
  }
  if (a.acc_class) {
    __syncwarp();
    if (s_cls[wid][lane] != 0.0) atomicAdd(&a.acc_class[lane], s_cls[wid][lane]);
  }
}

template <int kNit>
cudaError_t launch_backward_fast(const BwdArgs& a, int sm_count, cudaStream_t st) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, backward_fast_kernel<kNit>, kThreads, 0);
  if (e != cudaSuccess) return e;
  const int64_t want = (a.p + (int64_t)kWarps * kBwdChunk - 1) / ((int64_t)kWarps * kBwdChunk);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)std::max(1, per_sm) * sm_count));
  backward_fast_kernel<kNit><<<grid, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_heldout(const MapState& m, const float* xyz, const int32_t* labels, int64_t h, float* grad,
                           double* ll_dev) {
  if (h <= 0) return cudaSuccess;
  LLArgs a;
  a.g = m.g;
  a.alpha0 = (float)m.prm.alpha0;
  a.hkeys = m.hkeys;
  a.hvals = m.hvals;
  a.hash_cap = m.hash_cap;
  a.alpha = m.alpha;
  a.grad = grad;
  a.xyz = xyz;
  a.labels = labels;
  a.h = h;
  a.ll = ll_dev;
  a.map = m.active_map;
  a.dc = m.dc;
  heldout_kernel<<<(unsigned)((h + 255) / 256), 256, 0, m.stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_grad_scatter(const MapState& m, const int64_t* keys, const float* grad, int64_t count, float* gpool,
                                unsigned long long* missed_dev) {
  if (count <= 0) return cudaSuccess;
  grad_scatter_kernel<<<(unsigned)((count + 255) / 256), 256, 0, m.stream>>>(m.g, m.hkeys, m.hvals, m.hash_cap, keys,
                                                                             grad, count, m.active_map, gpool,
                                                                             missed_dev);
  return cudaGetLastError();
}

cudaError_t launch_backward(const MapState& m, const float4* xyzl, int64_t p, const float* gpool, double* acc_dev,
                            float* grad_xyz, double* acc_class) {
  if (p <= 0) return cudaSuccess;
  BwdArgs a;
  a.g = m.g;
  a.xyzl = xyzl;
  a.p = p;
  a.hkeys = m.hkeys;
  a.hvals = m.hvals;
  a.hash_cap = m.hash_cap;
  a.gpool = gpool;
  a.ctab = m.ctab;
  a.clen = m.clen;
  a.tpad = m.ctab_pad;
  a.R = m.ctab_R;
  a.recip_na = ((1u << 20) + (uint32_t)(2 * m.ctab_R + 1) - 1u) / (uint32_t)(2 * m.ctab_R + 1);
  a.acc = acc_dev;
  a.grad_xyz = grad_xyz;
  a.acc_class = acc_class;
  a.xyz_scale = (float)(m.prm.sigma0 / m.prm.length_scale);
  a.dc = m.dc;
  if (2 * a.R + 1 <= kBwdAxis - 1) {
    switch (a.tpad / 32) {  // unrolled sweeps for the common list lengths
      case 2: return launch_backward_fast<2>(a, m.sm_count, m.stream);
      case 3: return launch_backward_fast<3>(a, m.sm_count, m.stream);
      case 4: return launch_backward_fast<4>(a, m.sm_count, m.stream);
      case 5: return launch_backward_fast<5>(a, m.sm_count, m.stream);
      case 6: return launch_backward_fast<6>(a, m.sm_count, m.stream);
      default: return launch_backward_fast<0>(a, m.sm_count, m.stream);
    }
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, backward_kernel, kThreads, 0);
  if (e != cudaSuccess) return e;
  const int64_t want = (p + kWarps - 1) / kWarps;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)std::max(1, per_sm) * m.sm_count));
  backward_kernel<<<grid, kThreads, 0, m.stream>>>(a);
  return cudaGetLastError();
}

}  // namespace sbki
