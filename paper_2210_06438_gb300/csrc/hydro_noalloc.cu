// hydro_noalloc.cu -- an RHS entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc at all: real-time loops where a device
// allocation (which may synchronise the whole device) is not allowed, or
// hosts whose device memory belongs to another allocator (a framework's
// caching allocator) that must not be bypassed.  For them, hydro_rhs_noalloc
// evaluates a uniform batch with a register-load tile kernel of the same
// per-cell arithmetic as hydro_rhs_ex's, but its only scratch memory -- the
// table of sub-grid descriptors the kernel reads -- lives in the file-scope
// device array below, whose storage exists from module load until process
// exit on every GPU that loads the library.  Nothing is allocated on the
// host heap or the device.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "hydro.h"
#include "hydro_internal.h"
#include "hydro_kernels.cuh"
#include "hydro_uniform.cuh"

namespace hydro_dev {

// The scratch: room for HYDRO_NOALLOC_MAX_SUBGRIDS descriptors (24 bytes
// each, 192 KiB in all).  Every call overwrites the first n_subgrids entries;
// nothing in it has to start at zero.
constexpr size_t kNoallocBytes = (size_t)HYDRO_NOALLOC_MAX_SUBGRIDS * sizeof(hydro_subgrid_t);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

template <int MODE, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
rhs_uniform_kernel(const hydro_subgrid_t* __restrict__ desc, int N, int F, int G, int tpe,
                   int n_tiles, int lch, double* __restrict__ out, double* __restrict__ amax_out,
                   double gamma_d, int prefetch, int scheme) {
  // no status word: nonphysical inputs are not recorded by this entry point;
  // the flux scheme is a run-time argument as in rhs_tiles_kernel (always 0,
  // Kurganov-Tadmor, here), so both kernels compile the same arithmetic
  tile_loop<MODE, NT, 4>(UniformDesc{desc, N, F, G, tpe}, n_tiles, lch, out, amax_out, nullptr,
                         gamma_d, 0, prefetch, scheme == 1);
}

}  // namespace hydro_dev

namespace {

struct NoallocDev {
  bool ready = false;
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
  int n_sm = 0;
  int occ[2] = {0, 0};               // resident CTAs per SM, per precision
};
NoallocDev g_nadev[64];
std::mutex g_namu;

constexpr int kThreads = 256;
constexpr int kLch = 32;
// the launch needs this much dynamic shared memory with F = HYDRO_MAX_FIELDS
// (the layout does not grow with F); a kernel change that outgrows the
// opt-in limit of sm_100-class GPUs (227 KiB per CTA, less the kernels'
// static shared memory) fails here, at build time
static_assert(hydro_dev::smem_layout_bytes<0>(kLch) <= 226 * 1024 &&
                  hydro_dev::smem_layout_bytes<1>(kLch) <= 226 * 1024,
              "shared memory of the allocation-free launch");

void* noalloc_func(hydro_precision_t prec) {
  return prec == HYDRO_FP64 ? (void*)&hydro_dev::rhs_uniform_kernel<0, kThreads, 1>
                            : (void*)&hydro_dev::rhs_uniform_kernel<1, kThreads, 1>;
}

// Once per device, with that device current: resolve the scratch array's
// device address and prepare the kernels' launch attributes.
int noalloc_setup(int dev, NoallocDev** out) {
  std::lock_guard<std::mutex> g(g_namu);
  NoallocDev& D = g_nadev[dev];
  if (!D.ready) {
    cudaError_t e = cudaGetSymbolAddress((void**)&D.scratch, hydro_dev::g_noalloc_scratch);
    if (e != cudaSuccess) return hydro_host::cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&D.n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
      return hydro_host::cuda_fail(e, "cudaDeviceGetAttribute");
    // the same limit as the other entry points' kernels (hydro_api.cu:
    // the opt-in maximum less 1 KiB for the kernels' static shared memory)
    const int limit = optin - 1024;
    for (int m = 0; m < 2; m++) {
      hydro_precision_t prec = (hydro_precision_t)m;
      int smem = hydro_host::smem_bytes(prec, HYDRO_MAX_FIELDS, kLch);
      if (smem > limit) return HYDRO_EINVAL;  // a GPU with less shared memory than sm_100
      if ((e = cudaFuncSetAttribute(noalloc_func(prec), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    limit)) != cudaSuccess)
        return hydro_host::cuda_fail(e, "cudaFuncSetAttribute");
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&D.occ[m], noalloc_func(prec), kThreads,
                                                             smem)) != cudaSuccess)
        return hydro_host::cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      if (D.occ[m] < 1) D.occ[m] = 1;
    }
    D.ready = true;
  }
  *out = &D;
  return HYDRO_OK;
}

}  // namespace

extern "C" int hydro_rhs_noalloc(const hydro_subgrid_t* subgrids, int64_t n_subgrids, int32_t N,
                                 int32_t ghost, int32_t n_fields, double gamma, double* out_dUdt,
                                 double* out_amax, hydro_precision_t prec, void* stream) {
  if (N < 2 || N > HYDRO_MAX_N || n_fields < 6 || n_fields > HYDRO_MAX_FIELDS) return HYDRO_EINVAL;
  if (n_subgrids > HYDRO_NOALLOC_MAX_SUBGRIDS) return HYDRO_ETOOBIG;
  if (n_subgrids < 0) return HYDRO_EINVAL;
  if (prec != HYDRO_FP64 && prec != HYDRO_FP32_FLUX_FP64_ACC) return HYDRO_EINVAL;
  if (ghost < 3 || ghost > 64 || !(gamma > 1.0) || !std::isfinite(gamma)) return HYDRO_EINVAL;
  if (n_subgrids == 0) return HYDRO_OK;
  if (!subgrids || !out_dUdt || !out_amax) return HYDRO_EINVAL;
  for (int64_t s = 0; s < n_subgrids; s++) {
    const hydro_subgrid_t& d = subgrids[s];
    if (!d.U || d.N != N || d.n_fields != n_fields || !(d.dx > 0.0) || !std::isfinite(d.dx) ||
        (reinterpret_cast<uintptr_t>(d.U) & 7))
      return HYDRO_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hydro_host::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return HYDRO_EINVAL;
  NoallocDev* D;
  int rc = noalloc_setup(dev, &D);
  if (rc) return rc;

  cudaStream_t st = (cudaStream_t)stream;
  const hydro_subgrid_t* ddesc = reinterpret_cast<const hydro_subgrid_t*>(D->scratch);
  // the descriptor table: the one piece of scratch every call rewrites
  if ((e = cudaMemcpyAsync((void*)ddesc, subgrids, (size_t)n_subgrids * sizeof(hydro_subgrid_t),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return hydro_host::cuda_fail(e, "cudaMemcpyAsync(descriptors)");
  const int tpe = (N + hydro_dev::TE - 1) / hydro_dev::TE;
  const int64_t n_tiles = n_subgrids * tpe * tpe * tpe;
  if (n_tiles > 0x7fffffff) return HYDRO_EINVAL;
  if (tpe > 1 && (e = cudaMemsetAsync(out_amax, 0, (size_t)n_subgrids * sizeof(double), st)) != cudaSuccess)
    return hydro_host::cuda_fail(e, "cudaMemsetAsync(amax)");
  int G = N + 2 * ghost, F = n_fields, nt = (int)n_tiles, lch = kLch, pf = 0, ntpe = tpe, scheme = 0;
  int64_t grid64 = (int64_t)D->occ[prec == HYDRO_FP64 ? 0 : 1] * D->n_sm;
  int grid = (int)(n_tiles < grid64 ? n_tiles : grid64);
  size_t smem = (size_t)hydro_host::smem_bytes(prec, F, lch);
  void* args[] = {(void*)&ddesc, (void*)&N, (void*)&F, (void*)&G, (void*)&ntpe, (void*)&nt,
                  (void*)&lch, (void*)&out_dUdt, (void*)&out_amax, (void*)&gamma, (void*)&pf,
                  (void*)&scheme};
  if ((e = cudaLaunchKernel(noalloc_func(prec), dim3(grid), dim3(kThreads), args, smem, st)) != cudaSuccess)
    return hydro_host::cuda_fail(e, "launch");
  return HYDRO_OK;
}
