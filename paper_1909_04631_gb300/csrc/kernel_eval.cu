// sbki_kernel_values: the sparse kernel f(r) of Eq. (kernel) at given r, in
// either device form (see kernel_value.cuh).  Diagnostic entry point.
#include "kernel_value.cuh"
#include "sbki_internal.cuh"

namespace {

__global__ void kernel_values_kernel(const float* __restrict__ r, int64_t n, float* __restrict__ f, int method) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x = r[i];
  float v = 0.0f;
  if (x < 1.0f) v = method == 0 ? sbki::kernel_f_poly(x) : sbki::kernel_f_trig(x);
  f[i] = v;
}

}  // namespace

extern "C" sbki_status sbki_kernel_values(const float* r, int64_t n, float* f, int32_t method, void* stream) {
  if (n < 0 || (n > 0 && (!r || !f)) || (method != 0 && method != 1)) return SBKI_ERR_INVALID_ARG;
  if (n == 0) return SBKI_OK;
  cudaPointerAttributes a1, a2;
  if (cudaPointerGetAttributes(&a1, r) != cudaSuccess || cudaPointerGetAttributes(&a2, f) != cudaSuccess ||
      a1.type != cudaMemoryTypeDevice || a2.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return SBKI_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  kernel_values_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(r, n, f, method);
  if (cudaGetLastError() != cudaSuccess) return SBKI_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SBKI_ERR_CUDA;
  return SBKI_OK;
}
