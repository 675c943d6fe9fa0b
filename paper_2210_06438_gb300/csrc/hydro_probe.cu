// hydro_probe.cu -- the binary64 throughput probe: the denominator of the
// binary64 form's roofline, measured on the GPU that runs the form.
//
// The binary64 RHS is bound by the binary64 pipe (about 2 fused multiply-adds
// per SM per clock on this GPU class), not by memory.  Its roofline fraction
// needs the rate that pipe actually reaches, so the library carries a kernel
// that does nothing but independent binary64 fused multiply-adds: every
// thread runs kChains chains of `iters` steps x <- x*a + b.  The caller times
// the launch (CUDA events on `stream`) and divides 2 * flops_per_launch by it.
#include <cuda_runtime.h>

#include "hydro.h"
#include "hydro_internal.h"

namespace hydro_dev {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__device__ double g_probe_sink;

__global__ void __launch_bounds__(kProbeThreads)
fp64_probe_kernel(int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) x[c] = 1e-3 * (threadIdx.x + 1) + c;
#pragma unroll 1
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += x[c];
  // never true for the arguments the host passes (0 < a < 1, b > 0: the
  // chains stay positive and finite); keeps every chain live
  if (s < 0.0) g_probe_sink = s;
}

}  // namespace hydro_dev

extern "C" int hydro_probe_fp64(int32_t blocks_per_sm, int32_t iters, void* stream, double* fma_per_launch) {
  if (blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1 || !fma_per_launch) return HYDRO_EINVAL;
  int dev = 0, n_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return hydro_host::cuda_fail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return hydro_host::cuda_fail(e, "cudaDeviceGetAttribute(SM count)");
  const int grid = n_sm * blocks_per_sm;
  hydro_dev::fp64_probe_kernel<<<grid, hydro_dev::kProbeThreads, 0, (cudaStream_t)stream>>>(
      iters, 0.999999, 1e-7);
  if ((e = cudaGetLastError()) != cudaSuccess) return hydro_host::cuda_fail(e, "fp64 probe launch");
  *fma_per_launch = (double)grid * hydro_dev::kProbeThreads * hydro_dev::kChains * (double)iters;
  return HYDRO_OK;
}
