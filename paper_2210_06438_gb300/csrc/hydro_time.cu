// hydro_time.cu -- the Courant time step on the device, so that explicit
// steps (the three hydro iterations of a time step, Sec. VI-A) can follow one
// another with no host round trip: the step reads the largest signal speeds
// the previous stages wrote (Sec. IV-B: the signal speed sets the Courant
// condition) and leaves dt where the *_stage_dt entry points read it.
#include <cuda_runtime.h>

#include <cmath>

#include "hydro.h"
#include "hydro_internal.h"

namespace hydro_dev {

constexpr int kCourantThreads = 1024;

// One CTA.  a_s = max over the rows r of amax[r * stride + s]; with per-sub-
// grid widths q = cfl * min_s(dx_s / a_s), else q = (cfl * dx) / max_s a_s;
// dt = min(q, t_end - t) (0 once t >= t_end); then clock = {t + dt, dt, k + 1}
// and dt_hist[k] = dt while k < hist_len.
__global__ void __launch_bounds__(kCourantThreads)
courant_kernel(const double* __restrict__ amax, int n_rows, long long stride, long long n,
               const double* __restrict__ dx, double dx_uniform, double cfl, double t_end,
               double* __restrict__ clock, double* __restrict__ dt_hist, long long hist_len) {
  __shared__ double red[kCourantThreads / 32];
  double m = dx ? INFINITY : 0.0;
  for (long long s = threadIdx.x; s < n; s += blockDim.x) {
    double a = amax[s];
    for (int r = 1; r < n_rows; r++) a = fmax(a, amax[r * stride + s]);
    if (dx) m = fmin(m, dx[s] / a);
    else m = fmax(m, a);
  }
  for (int o = 16; o > 0; o >>= 1) {
    double v = __shfl_xor_sync(0xffffffffu, m, o);
    m = dx ? fmin(m, v) : fmax(m, v);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = dx ? fmin(m, red[w]) : fmax(m, red[w]);
    const double q = dx ? cfl * m : (cfl * dx_uniform) / m;
    const double t = clock[0], left = t_end - t;
    const double dt = left > 0.0 ? fmin(q, left) : 0.0;
    const long long k = (long long)clock[2];
    clock[0] = t + dt;
    clock[1] = dt;
    clock[2] = (double)(k + 1);
    if (dt_hist && k < hist_len) dt_hist[k] = dt;
  }
}

}  // namespace hydro_dev

extern "C" int hydro_courant(const double* amax, int32_t n_rows, int64_t row_stride, int64_t n,
                             const double* dx, double dx_uniform, double cfl, double t_end, double* clock,
                             double* dt_hist, int64_t hist_len, void* stream) {
  if (!amax || !clock || n_rows < 1 || n < 1 || row_stride < n || (!dx && !(dx_uniform > 0.0)) ||
      !(cfl > 0.0) || !std::isfinite(cfl) || !std::isfinite(t_end) || hist_len < 0 || (hist_len > 0 && !dt_hist))
    return HYDRO_EINVAL;
  if ((reinterpret_cast<uintptr_t>(amax) | reinterpret_cast<uintptr_t>(clock) |
       reinterpret_cast<uintptr_t>(dx) | reinterpret_cast<uintptr_t>(dt_hist)) & 7)
    return HYDRO_EINVAL;
  hydro_dev::courant_kernel<<<1, hydro_dev::kCourantThreads, 0, (cudaStream_t)stream>>>(
      amax, n_rows, row_stride, n, dx, dx_uniform, cfl, t_end, clock, dt_hist, hist_len);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HYDRO_OK : hydro_host::cuda_fail(e, "courant launch");
}
