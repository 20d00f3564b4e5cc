// Step a5, the S-BKI update of Eq. (alpha_kernel) with the sparse kernel of
// Eq. (kernel):  alpha_v^k += sum_{i: y_i = k, |c_v - x_i| < l} sigma0 f(|c_v - x_i| / l).
// f is evaluated as u^5 Q(u^2), u = 1 - d/l (kernel_value.cuh), and every
// centre-to-point offset is formed in a block-local frame from a compensated
// (hi + lo) offset, so both d and f keep FP32 relative accuracy up to d = l.
//
// One CTA per touched block (a persistent grid pulls blocks from a device
// work counter).  The CTA
//   1. stages the training points that touch the block (the block's list,
//      built by the binning step) into shared memory, as compensated offsets
//      from the block's first voxel centre;
//   2. lists the voxel rows (y, z) of each point's clipped bounding square
//      (a thread per row: the row's x-span from one square root; rows the
//      ball misses get an empty span), then flattens the in-support
//      (voxel, point) pairs of all listed rows and lets every thread walk one
//      contiguous range of them, adding sigma0 f into a shared-memory alpha
//      tile [K+1][B^3];
//   3. adds the tile into the block's alpha in HBM once (write for a block
//      created by this update, read-modify-write of the nonzero entries
//      otherwise) - one pass over each touched block, no global atomics.
#include <algorithm>

#include "kernel_value.cuh"
#include "sbki_internal.cuh"

namespace sbki {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kPts = 512;       // staged points per pass
constexpr int kRows = 3584;     // listed rows per pass (two CTAs per SM fit in shared memory)
constexpr float kMargin = 0.01f;  // voxels: the FP32 span bounds are widened by this; every voxel is re-tested

struct AccArgs {
  Geom g;
  const float4* train;
  const uint32_t* touched;
  const uint32_t* boff;
  const uint32_t* blist;
  const unsigned long long* hkeys;
  const int32_t* hvals;
  float* alpha;
  int32_t* pairs;
  DevCounters* dc;
};

__device__ __forceinline__ int floor_i(float v) { return (int)floorf(v); }
__device__ __forceinline__ int ceil_i(float v) { return (int)ceilf(v); }

// offsets from the block's first voxel centre: e(j) = E0 + j res (compensated)
__device__ __forceinline__ float voxel_offset(int j, float e0_hi, float e0_lo, const Geom& g) {
  return centre_offset_at(j, e0_hi, e0_lo, g);
}
__device__ __forceinline__ void stage_offset(int K0, float x, const Geom& g, float& hi, float& lo) {
  centre_offset0(K0, x, g, hi, lo);
}

// In-place exclusive scan of a[0..n) (n <= 8 kThreads) by the whole CTA;
// a[n] receives the total, which is returned.
__device__ int block_scan(int* a, int n, int* s_wsum) {
  constexpr int kIpt = 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int loc[kIpt];
  int sum = 0;
#pragma unroll
  for (int k = 0; k < kIpt; ++k) {
    const int i = threadIdx.x * kIpt + k;
    loc[k] = i < n ? a[i] : 0;
    sum += loc[k];
  }
  int inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  __syncthreads();  // every thread has read a[] before it is overwritten
  if (lane == 31) s_wsum[warp] = inc;
  __syncthreads();
  int woff = 0, total = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const int v = s_wsum[w];
    woff += (w < warp) ? v : 0;
    total += v;
  }
  int ex = woff + inc - sum;
#pragma unroll
  for (int k = 0; k < kIpt; ++k) {
    const int i = threadIdx.x * kIpt + k;
    if (i < n) a[i] = ex;
    ex += loc[k];
  }
  if (threadIdx.x == 0) a[n] = total;
  __syncthreads();
  return total;
}

template <bool kTrack>
__global__ void __launch_bounds__(kThreads, 2) accumulate_kernel(AccArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Geom& g = a.g;
  const int K1 = g.K1, B3 = g.B3, B = g.B;
  float4* pxy = reinterpret_cast<float4*>(smem_raw);  // [kPts] (x hi, x lo, y hi, y lo)
  float4* pzw = pxy + kPts;                           // [kPts] (z hi, z lo, packed index/label, row rect)
  int2* rows = reinterpret_cast<int2*>(pzw + kPts);   // [kRows] (rd2 bits, packed row)
  int* prs = reinterpret_cast<int*>(rows + kRows);    // [kPts + 4] first row of each point
  int* rps = prs + kPts + 4;                          // [kRows + 4] first pair of each row
  uint16_t* rowpt = reinterpret_cast<uint16_t*>(rps + kRows + 4);  // [kRows] point of each row
  float* asum = reinterpret_cast<float*>(rowpt + kRows);
  int* pcnt = reinterpret_cast<int*>(asum + K1 * B3);
  __shared__ uint32_t s_item;
  __shared__ int s_stop;
  __shared__ int s_wsum[kWarps];
  const int lane = threadIdx.x & 31;
  const float lw = sqrtf(g.l2_hi);
  uint32_t npairs = 0, ntouched = 0;
  // the tile starts at zero; the write-out of every block zeroes it again
  for (int e = threadIdx.x; e < K1 * B3; e += kThreads) asum[e] = 0.0f;
  if (kTrack)
    for (int e = threadIdx.x; e < B3; e += kThreads) pcnt[e] = 0;

  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t it = atomicAdd(&a.dc->work_next, 1u);
      s_item = it;
      s_stop = (a.dc->err != 0 || it >= a.dc->n_touched) ? 1 : 0;
    }
    __syncthreads();
    const uint32_t item = s_item;
    if (s_stop) break;  // uniform over the CTA
    const uint32_t slot = a.touched[item];
    const int32_t pool = a.hvals[slot];
    int bk[3];
    unpack_block(a.hkeys[slot], bk[0], bk[1], bk[2]);
    const bool fresh = pool >= (int32_t)a.dc->n_blocks_before;
    const int K0[3] = {bk[0] << g.B_shift, bk[1] << g.B_shift, bk[2] << g.B_shift};
    const uint32_t beg = a.boff[item], total = a.boff[item + 1] - beg;
    for (uint32_t cb = 0; cb < total; cb += kPts) {
      const int np = (int)min((uint32_t)kPts, total - cb);
      __syncthreads();  // the previous pass is done with the staging arrays
      // 1. stage the points; their (y, z) row square clipped to the block
      for (int k = threadIdx.x; k < np; k += kThreads) {
        const uint32_t idx = a.blist[beg + cb + k];
        const float4 p = a.train[idx];
        float4 xy, zw;
        stage_offset(K0[0], p.x, g, xy.x, xy.y);
        stage_offset(K0[1], p.y, g, xy.z, xy.w);
        stage_offset(K0[2], p.z, g, zw.x, zw.y);
        const int jy0 = max(0, ceil_i(__fmul_rn(-lw - xy.z, g.inv_res) - kMargin));
        const int jy1 = min(B - 1, floor_i(__fmul_rn(lw - xy.z, g.inv_res) + kMargin));
        const int jz0 = max(0, ceil_i(__fmul_rn(-lw - zw.x, g.inv_res) - kMargin));
        const int jz1 = min(B - 1, floor_i(__fmul_rn(lw - zw.x, g.inv_res) + kMargin));
        const int ny = max(0, jy1 - jy0 + 1), nz = max(0, jz1 - jz0 + 1);
        zw.z = __uint_as_float((idx << 5) | ((uint32_t)p.w & 31u));
        zw.w = __int_as_float(jy0 | (ny << 4) | (jz0 << 8));
        pxy[k] = xy;
        pzw[k] = zw;
        prs[k] = ny * nz;
      }
      __syncthreads();
      const int nrow_all = block_scan(prs, np, s_wsum);
      // 2. passes of at most kRows rows
      for (int rb = 0; rb < nrow_all; rb += kRows) {
        const int nrows = min(kRows, nrow_all - rb);
        for (int k = threadIdx.x; k < np; k += kThreads) {  // row -> point map of this pass
          const int r1 = min(prs[k + 1], rb + nrows);
          for (int r = max(prs[k], rb); r < r1; ++r) rowpt[r - rb] = (uint16_t)k;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nrows; t += kThreads) {
          const int r = rb + t;
          const int k = rowpt[t];
          const float4 xy = pxy[k], zw = pzw[k];
          const int inf = __float_as_int(zw.w);
          const int ny = (inf >> 4) & 15, rr = r - prs[k];
          const int qz = (int)small_div(rr, small_recip(ny));
          const int jy = (inf & 15) + (rr - qz * ny), jz = ((inf >> 8) & 15) + qz;
          const float ey = voxel_offset(jy, xy.z, xy.w, g);
          const float ez = voxel_offset(jz, zw.x, zw.y, g);
          const float rd2 = __fmaf_rn(ey, ey, __fmul_rn(ez, ez));
          int i0 = 0, n = 0;
          if (rd2 < g.l2_hi) {
            const float rem = g.l2_hi - rd2;
            const float hx = rem * rsqrtf(rem);
            i0 = max(0, ceil_i(__fmul_rn(-hx - xy.x, g.inv_res) - kMargin));
            const int i1 = min(B - 1, floor_i(__fmul_rn(hx - xy.x, g.inv_res) + kMargin));
            n = max(0, i1 - i0 + 1);
          }
          rows[t] = make_int2(__float_as_int(rd2), k | (jy << 9) | (jz << 12) | (i0 << 15));
          rps[t] = n;
        }
        __syncthreads();
        const int T = block_scan(rps, nrows, s_wsum);
        // 3. every thread walks one contiguous range of the pairs
        const int q0 = (int)(((unsigned)T * threadIdx.x) / kThreads);  // T < 2^22: no overflow
        const int q1 = (int)(((unsigned)T * (threadIdx.x + 1)) / kThreads);
        if (q0 < q1) {
          int lo = 0, hi = nrows - 1;  // last row with rps[r] <= q0 (a row with pairs)
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (rps[mid] <= q0) lo = mid;
            else hi = mid - 1;
          }
          int r = lo;
          int next = rps[r + 1];
          int2 row = rows[r];
          int i = ((row.y >> 15) & 7) + (q0 - rps[r]);
          int kq = row.y & 511;
          float xh = pxy[kq].x, xl = pxy[kq].y;
          uint32_t packed = __float_as_uint(pzw[kq].z);
          int vbase = ((((row.y >> 12) & 7) * B) + ((row.y >> 9) & 7)) * B;
          int abase = (int)(packed & 31u) * B3 + vbase;
          float rd2 = __int_as_float(row.x);
          for (int q = q0; q < q1; ++q, ++i) {
            if (q >= next) {
              do {
                ++r;
                next = rps[r + 1];
              } while (q >= next);
              row = rows[r];
              i = (row.y >> 15) & 7;
              const int k2 = row.y & 511;
              if (k2 != kq) {
                kq = k2;
                xh = pxy[kq].x;
                xl = pxy[kq].y;
                packed = __float_as_uint(pzw[kq].z);
              }
              vbase = ((((row.y >> 12) & 7) * B) + ((row.y >> 9) & 7)) * B;
              abase = (int)(packed & 31u) * B3 + vbase;
              rd2 = __int_as_float(row.x);
            }
            const float ex = voxel_offset(i, xh, xl, g);
            const float d2 = __fmaf_rn(ex, ex, rd2);
            bool in = d2 < g.l2_lo;
            if (!in && d2 < g.l2_hi) {
              const float4 x = a.train[packed >> 5];
              in = in_support64(K0[0] + i, K0[1] + ((row.y >> 9) & 7), K0[2] + ((row.y >> 12) & 7), x.x, x.y,
                                x.z, g);
            }
            if (in) {
              const float d = d2 > 0.0f ? d2 * rsqrtf(d2) : 0.0f;
              const float u = __fmul_rn(__fsub_rn(g.l, d), g.inv_l);
              atomicAdd(&asum[abase + i], g.sigma0_k[packed & 31u] * kernel_f_poly_u(u));
              ++npairs;
              if (kTrack) atomicAdd(&pcnt[vbase + i], 1);
            }
          }
        }
        __syncthreads();  // the row list is reused by the next pass
      }
    }
    __syncthreads();
    // one pass over the block's alpha in HBM (a thread per voxel), zeroing the tile
    float* gblk = a.alpha + (size_t)pool * (size_t)(K1 * B3);
    for (int v = threadIdx.x; v < B3; v += kThreads) {
      bool any = false;
      for (int k = 0; k < K1; ++k) {
        const int e = k * B3 + v;
        const float val = asum[e];
        asum[e] = 0.0f;
        any |= val != 0.0f;
        if (fresh) gblk[e] = val;
        else if (val != 0.0f) gblk[e] += val;
      }
      ntouched += any ? 1u : 0u;
      if (kTrack) {
        int32_t* gp = a.pairs + (size_t)pool * B3 + v;
        *gp = (fresh ? 0 : *gp) + pcnt[v];
        pcnt[v] = 0;
      }
    }
  }
  // CTA totals -> one atomic per warp
  for (int o = 16; o > 0; o >>= 1) {
    npairs += __shfl_down_sync(0xffffffffu, npairs, o);
    ntouched += __shfl_down_sync(0xffffffffu, ntouched, o);
  }
  if (lane == 0) {
    atomicAdd(&a.dc->pairs, (unsigned long long)npairs);
    atomicAdd(&a.dc->touched_voxels, (unsigned long long)ntouched);
  }
}

}  // namespace

size_t accumulate_smem_bytes(const Geom& g) {
  return 2 * sizeof(float4) * kPts + sizeof(int2) * kRows + sizeof(int) * (kPts + 4 + kRows + 4) +
         sizeof(uint16_t) * kRows + sizeof(float) * (size_t)g.K1 * g.B3 + sizeof(int) * (size_t)g.B3;
}

cudaError_t launch_accumulate(MapState& m, const KeyFrame& /*kf*/) {
  AccArgs a;
  a.g = m.g;
  a.train = m.s.train;
  a.touched = m.s.touched;
  a.boff = m.boff;
  a.blist = m.blist;
  a.hkeys = m.hkeys;
  a.hvals = m.hvals;
  a.alpha = m.alpha;
  a.pairs = m.pairs;
  a.dc = m.dc;
  const size_t smem = accumulate_smem_bytes(m.g);
  const bool track = m.pairs != nullptr;
  cudaError_t e;
  int per_sm = 0;
  if (track) {
    e = cudaFuncSetAttribute(accumulate_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, accumulate_kernel<true>, kThreads, smem);
  } else {
    e = cudaFuncSetAttribute(accumulate_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, accumulate_kernel<false>, kThreads, smem);
  }
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, per_sm) * m.sm_count;
  if (track) accumulate_kernel<true><<<grid, kThreads, smem, m.stream>>>(a);
  else accumulate_kernel<false><<<grid, kThreads, smem, m.stream>>>(a);
  m.launches += 1;
  return cudaGetLastError();
}

}  // namespace sbki
