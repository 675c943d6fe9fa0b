// hydro_domain.cu -- the RHS of a periodic domain of same-level sub-grids with
// the ghost shells gathered inside the kernel, and the fused explicit stage.
//
// The sub-grids of the paper's benchmark exchange ghost layers before every
// hydro iteration (the ghost handling that Sec. V-A and VI-B count among the
// per-step work) and an explicit stage update follows each RHS (three hydro
// iterations per step, Sec. VI-A).  Here a domain of nb^3 sub-grids of N^3
// cells is stored without ghosts; each tile reads its 3-deep ghost slabs
// directly from the neighbouring sub-grids' interiors (periodic wrap), so no
// ghost copy and no ghosted storage exist, and the stage
//   U_out = alpha U0 + beta (U + dt dU/dt)
// is applied in the same launch (SSP-RK3: (0,1), (3/4,1/4), (1/3,2/3)).
// The work list is computed on the fly: nothing is allocated per call.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "hydro.h"
#include "hydro_internal.h"
#include "hydro_kernels.cuh"
#include "hydro_quad.cuh"

namespace hydro_host {
int ctx_status_ptr(hydro_dev::Status** st, int* n_sm, int* smem_optin);
}

namespace {

struct Shape {
  int threads, minb, lch;
};
// the launch shapes the autotuner picks for the sub-grid batches (binary64
// 576 threads, mixed the pipelined kernel), then the 26-point kernels
const Shape kShape[4] = {{576, 1, 64},
                         {hydro_host::kPipeThreads, 1, 64},
                         {hydro_dev::QuadShape<0>::NT, 1, 64},
                         {hydro_dev::QuadShape<1>::NT, 1, 64}};
const int kKind[4] = {hydro_host::kKindTiles, hydro_host::kKindPipe, hydro_host::kKindQuad,
                      hydro_host::kKindQuad};

// shape index: precision, plus 2 for the 26-point variant
int shape_of(hydro_precision_t prec, bool quad26) { return (prec == HYDRO_FP64 ? 0 : 1) + (quad26 ? 2 : 0); }

void* domain_func(int k) {
  switch (k) {
    case 0: return (void*)&hydro_dev::rhs_domain_kernel<0, 576, 1, 1>;
    case 1: return (void*)&hydro_dev::rhs_domain_pipe_kernel<hydro_host::kPipeThreads>;
    case 2: return (void*)&hydro_dev::rhs_domain_quad_kernel<0>;
    default: return (void*)&hydro_dev::rhs_domain_quad_kernel<1>;
  }
}

struct DomDev {
  bool ready = false;
  int n_sm = 0, occ[4] = {0, 0, 0, 0};
};
DomDev g_dom[64];
std::mutex g_dmu;

int domain_setup(DomDev** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hydro_host::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return HYDRO_EINVAL;
  std::lock_guard<std::mutex> g(g_dmu);
  DomDev& D = g_dom[dev];
  if (!D.ready) {
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&D.n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
      return hydro_host::cuda_fail(e, "cudaDeviceGetAttribute");
    for (int k = 0; k < 4; k++) {
      hydro_precision_t prec = (k % 2 == 0) ? HYDRO_FP64 : HYDRO_FP32_FLUX_FP64_ACC;
      int smem = hydro_host::smem_bytes(prec, HYDRO_MAX_FIELDS, kShape[k].lch, kKind[k]);
      if ((e = cudaFuncSetAttribute(domain_func(k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    optin - 1024)) != cudaSuccess)
        return hydro_host::cuda_fail(e, "cudaFuncSetAttribute");
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&D.occ[k], domain_func(k), kShape[k].threads,
                                                             smem)) != cudaSuccess)
        return hydro_host::cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      if (D.occ[k] < 1) D.occ[k] = 1;
    }
    D.ready = true;
  }
  *out = &D;
  return HYDRO_OK;
}

int domain_launch(const double* U, const double* U0, double alpha, double beta, double dt, int stage,
                  int32_t nb, int32_t N, int32_t F, double dx, double gamma, double* out,
                  double* amax, hydro_precision_t prec, void* stream, uint32_t flags,
                  const double* dtp = nullptr) {
  if (!U || !out || !amax || (stage && !U0)) return HYDRO_EINVAL;
  if (nb < 1 || N < 2 || N > HYDRO_MAX_N || F < 6 || F > HYDRO_MAX_FIELDS) return HYDRO_EINVAL;
  if (nb * N < 6) return HYDRO_EINVAL;  // the ghost shell must not wrap onto the tile itself
  if (!(dx > 0.0) || !std::isfinite(dx) || !(gamma > 1.0) || !std::isfinite(gamma)) return HYDRO_EINVAL;
  if (prec != HYDRO_FP64 && prec != HYDRO_FP32_FLUX_FP64_ACC) return HYDRO_EINVAL;
  if (stage && (!std::isfinite(alpha) || !std::isfinite(beta) || !std::isfinite(dt))) return HYDRO_EINVAL;
  const long long cells = (long long)nb * nb * nb * N * N * N;
  if (cells * F >= 0x7fffffffLL) return HYDRO_EINVAL;  // 32-bit cell offsets in the kernel
  if ((reinterpret_cast<uintptr_t>(U) | reinterpret_cast<uintptr_t>(out) |
       reinterpret_cast<uintptr_t>(U0)) & 7)
    return HYDRO_EINVAL;
  if (out == U) return HYDRO_EINVAL;  // neighbours' ghosts are read while outputs are written
  DomDev* D;
  int rc = domain_setup(&D);
  if (rc) return rc;
  hydro_dev::Status* status;
  int n_sm, optin;
  if ((rc = hydro_host::ctx_status_ptr(&status, &n_sm, &optin))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int tpe = (N + hydro_dev::TE - 1) / hydro_dev::TE;
  const long long n_tiles = (long long)nb * nb * nb * tpe * tpe * tpe;
  if (n_tiles > 0x7fffffffLL) return HYDRO_EINVAL;
  cudaError_t e;
  if (tpe > 1 && (e = cudaMemsetAsync(amax, 0, (size_t)nb * nb * nb * sizeof(double), st)) != cudaSuccess)
    return hydro_host::cuda_fail(e, "cudaMemsetAsync(amax)");
  int ex2;
  bool pow2 = std::frexp(dx, &ex2) == 0.5 && ex2 > -120 && ex2 < 120;
  hydro_dev::DomainTiles dom{U, nb, N, F, tpe, 1.0 / dx, (short)(pow2 ? 2 : 0)};
  if (dtp && (reinterpret_cast<uintptr_t>(dtp) & 7)) return HYDRO_EINVAL;
  hydro_dev::StageArgs sa{U, stage ? U0 : U, alpha, beta, dt, stage, dtp};
  const int k = shape_of(prec, (flags & HYDRO_F_QUAD26) != 0);
  const Shape& sh = kShape[k];
  int nt = (int)n_tiles, lch = sh.lch, ws = 1, scheme = (flags & HYDRO_F_KNP) ? 1 : 0;
  long long g64 = (long long)D->occ[k] * D->n_sm;
  int grid = (int)(n_tiles < g64 ? n_tiles : g64);
  size_t smem = (size_t)hydro_host::smem_bytes(prec, F, lch, kKind[k]);
  void* args[] = {(void*)&dom, (void*)&nt, (void*)&lch, (void*)&out, (void*)&amax, (void*)&status,
                  (void*)&gamma, (void*)&ws, (void*)&scheme, (void*)&sa};
  if ((e = cudaLaunchKernel(domain_func(k), dim3(grid), dim3(sh.threads), args, smem, st)) != cudaSuccess)
    return hydro_host::cuda_fail(e, "launch");
  return HYDRO_OK;
}

}  // namespace

extern "C" {

int hydro_domain_rhs(const double* U, int32_t nb, int32_t N, int32_t n_fields, double dx,
                     double gamma, double* out_dUdt, double* out_amax, hydro_precision_t prec,
                     void* stream, uint32_t flags) {
  return domain_launch(U, nullptr, 0.0, 0.0, 0.0, 0, nb, N, n_fields, dx, gamma, out_dUdt, out_amax,
                       prec, stream, flags);
}

int hydro_domain_stage(const double* U, const double* U0, double alpha, double beta, double dt,
                       int32_t nb, int32_t N, int32_t n_fields, double dx, double gamma,
                       double* U_out, double* out_amax, hydro_precision_t prec, void* stream,
                       uint32_t flags) {
  return domain_launch(U, U0, alpha, beta, dt, 1, nb, N, n_fields, dx, gamma, U_out, out_amax, prec,
                       stream, flags);
}

int hydro_domain_stage_dt(const double* U, const double* U0, double alpha, double beta, const double* dt,
                          int32_t nb, int32_t N, int32_t n_fields, double dx, double gamma,
                          double* U_out, double* out_amax, hydro_precision_t prec, void* stream,
                          uint32_t flags) {
  if (!dt) return HYDRO_EINVAL;
  return domain_launch(U, U0, alpha, beta, 0.0, 1, nb, N, n_fields, dx, gamma, U_out, out_amax, prec,
                       stream, flags, dt);
}

}  // extern "C"
