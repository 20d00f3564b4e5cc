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
// as d -> 0 (f'(0) = 0).
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
  double* acc;         // [2]: sum G f, sum G u^4 D d
  float* grad_xyz;     // nullable [p][3]: (sigma0 / l) sum G u^4 D (c_v - x)/d
  float xyz_scale;     // sigma0 / l
  DevCounters* dc;
};

struct BwdTables {
  float4 x[kAxisMax + 1];  // (e_x^2, address part, e_x, 0); entry 2R+1 is the padding row
  float4 yz[kYZMax];       // (e_y^2 + e_z^2, address part, e_y, e_z)
  const float* blk[27];    // gpool + (pool (K+1) + y_i) B^3, or null
};

__global__ void __launch_bounds__(kThreads, 3) backward_kernel(BwdArgs a) {
  __shared__ BwdTables s_tab[kWarps];
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int R = a.R, na = 2 * R + 1;
  BwdTables& t = s_tab[wid];
  if (a.dc->err != 0) return;
  if (lane == 0) t.x[na] = make_float4(kFar, __int_as_float(0), 0.f, 0.f);
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
    acc_f += (double)sf;
    acc_l += (double)sl;
    if (a.grad_xyz) {
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
        sz += __shfl_down_sync(0xffffffffu, sz, o);
      }
      if (lane == 0) {
        a.grad_xyz[3 * i] = sx * a.xyz_scale;
        a.grad_xyz[3 * i + 1] = sy * a.xyz_scale;
        a.grad_xyz[3 * i + 2] = sz * a.xyz_scale;
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
                            float* grad_xyz) {
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
  a.xyz_scale = (float)(m.prm.sigma0 / m.prm.length_scale);
  a.dc = m.dc;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, backward_kernel, kThreads, 0);
  if (e != cudaSuccess) return e;
  const int64_t want = (p + kWarps - 1) / kWarps;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)std::max(1, per_sm) * m.sm_count));
  backward_kernel<<<grid, kThreads, 0, m.stream>>>(a);
  return cudaGetLastError();
}

}  // namespace sbki
