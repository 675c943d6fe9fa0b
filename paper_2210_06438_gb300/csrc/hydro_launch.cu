// hydro_launch.cu -- kernel instantiations and launch shapes of libhydro.
#include "hydro_internal.h"
#include "hydro_kernels.cuh"
#include "hydro_quad.cuh"

namespace hydro_host {

using hydro_dev::rhs_tiles_kernel;

// Kernel variants: (threads per CTA, minimum resident CTAs per SM, load
// batch).  The second number caps registers per thread (65536 / (threads *
// minb)), the third sets how many read-region slots a thread loads at once;
// the autotuner picks among them per batch.  {576, 1} is the pipelined mixed
// kernel (no binary64 counterpart), {192, 1} the 26-point kernel.
struct Variant {
  int threads, minb, kc;
};
static const Variant kVariants[] = {{256, 1, 4}, {128, 1, 4}, {512, 1, 4}, {512, 1, 2}, {384, 1, 4},
                                    {384, 1, 2}, {256, 2, 2}, {128, 2, 2}, {kPipeThreads, 1, 0},
                                    {kQuadThreads, 1, 0}};
static constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);
static_assert(kPipeThreads == hydro_dev::PNT, "pipelined kernel block size");
static_assert(kQuadThreads == hydro_dev::QNT, "26-point kernel block size");

template <int MODE>
static void* kfunc(int threads, int minb, int kc) {
  if (threads == kPipeThreads) return MODE == 1 ? (void*)&hydro_dev::rhs_tiles_pipe_kernel<kPipeThreads> : nullptr;
  if (threads == kQuadThreads) return (void*)&hydro_dev::rhs_quad_kernel<MODE>;
  if (threads == 128) return minb == 2 ? (void*)&rhs_tiles_kernel<MODE, 128, 2, 2> : (void*)&rhs_tiles_kernel<MODE, 128, 1, 4>;
  if (threads == 512) return kc == 2 ? (void*)&rhs_tiles_kernel<MODE, 512, 1, 2> : (void*)&rhs_tiles_kernel<MODE, 512, 1, 4>;
  if (threads == 384) return kc == 2 ? (void*)&rhs_tiles_kernel<MODE, 384, 1, 2> : (void*)&rhs_tiles_kernel<MODE, 384, 1, 4>;
  return minb == 2 ? (void*)&rhs_tiles_kernel<MODE, 256, 2, 2> : (void*)&rhs_tiles_kernel<MODE, 256, 1, 4>;
}

static void* pick(hydro_precision_t prec, int threads, int minb, int kc) {
  return prec == HYDRO_FP64 ? kfunc<0>(threads, minb, kc) : kfunc<1>(threads, minb, kc);
}

int num_variants() { return kNumVariants; }
bool variant_exists(hydro_precision_t prec, int threads, int minb, int kc) {
  return pick(prec, threads, minb, kc) != nullptr;
}
void variant(int i, int* threads, int* minb, int* kc) {
  *threads = kVariants[i].threads;
  *minb = kVariants[i].minb;
  *kc = kVariants[i].kc;
}

cudaError_t kernels_init(int smem_optin) {
  for (int m = 0; m < 2; m++)
    for (int i = 0; i < kNumVariants; i++) {
      void* f = pick((hydro_precision_t)m, kVariants[i].threads, kVariants[i].minb, kVariants[i].kc);
      if (!f) continue;
      cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

int smem_bytes(hydro_precision_t prec, int Fmax, int lch, int threads) {
  (void)Fmax;
  if (threads == kPipeThreads && prec != HYDRO_FP64) return (int)hydro_dev::pipe_smem_bytes();
  if (threads == kQuadThreads)
    return (int)(prec == HYDRO_FP64 ? hydro_dev::quad_smem_bytes<0>() : hydro_dev::quad_smem_bytes<1>());
  return (int)(prec == HYDRO_FP64 ? hydro_dev::smem_layout_bytes<0>(lch)
                                  : hydro_dev::smem_layout_bytes<1>(lch));
}

int occupancy(hydro_precision_t prec, int threads, int minb, int smem, int kc) {
  int nb = 0;
  void* f = pick(prec, threads, minb, kc);
  if (!f || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads, smem) != cudaSuccess)
    return 0;
  return nb;
}

LaunchCfg default_cfg(hydro_precision_t prec, int Fmax, int n_sm, int smem_optin,
                      int64_t n_tiles, bool pipelined, bool quad26) {
  LaunchCfg c;
  if (quad26) {
    c.threads = kQuadThreads;
    c.minb = 1;
    c.lch = 64;
    c.smem = smem_bytes(prec, Fmax, c.lch, c.threads);
    c.kc = 0;
    c.ctas_per_sm = occupancy(prec, c.threads, c.minb, c.smem, c.kc);
    if (c.ctas_per_sm < 1) c.ctas_per_sm = 1;
    int64_t g = (int64_t)c.ctas_per_sm * n_sm;
    c.grid = (int)(n_tiles < g ? n_tiles : g);
    if (c.grid < 1) c.grid = 1;
    return c;
  }
  if (prec != HYDRO_FP64 && pipelined && smem_bytes(prec, Fmax, 64, kPipeThreads) <= smem_optin) {
    c.threads = kPipeThreads;
    c.minb = 1;
    c.kc = 0;
    c.lch = 64;
    c.smem = smem_bytes(prec, Fmax, c.lch, c.threads);
    c.ctas_per_sm = 1;
    c.grid = (int)(n_tiles < n_sm ? n_tiles : n_sm);
    if (c.grid < 1) c.grid = 1;
    return c;
  }
  c.threads = 256;
  c.minb = 1;
  c.kc = 4;
  c.lch = prec == HYDRO_FP64 ? 32 : 64;
  c.smem = smem_bytes(prec, Fmax, c.lch);
  while (c.smem > smem_optin && c.lch > 16) {
    c.lch /= 2;
    c.smem = smem_bytes(prec, Fmax, c.lch);
  }
  c.ctas_per_sm = occupancy(prec, c.threads, c.minb, c.smem, c.kc);
  if (c.ctas_per_sm < 1) c.ctas_per_sm = 1;
  int64_t g = (int64_t)c.ctas_per_sm * n_sm;
  c.grid = (int)(n_tiles < g ? n_tiles : g);
  if (c.grid < 1) c.grid = 1;
  return c;
}

cudaError_t launch_tiles(const LaunchCfg& cfg, hydro_precision_t prec, const hydro_dev::Tile* tiles,
                         int n_tiles, int Fmax, double* out, double* amax, hydro_dev::Status* status,
                         double gamma, int write_status, cudaStream_t st, int scheme) {
  int lch = cfg.lch, pf = cfg.prefetch;
  void* args[] = {(void*)&tiles, (void*)&n_tiles, (void*)&Fmax, (void*)&lch, (void*)&out,
                  (void*)&amax, (void*)&status, (void*)&gamma, (void*)&write_status, (void*)&pf,
                  (void*)&scheme};
  return cudaLaunchKernel(pick(prec, cfg.threads, cfg.minb, cfg.kc), dim3(cfg.grid), dim3(cfg.threads), args,
                          (size_t)cfg.smem, st);
}

void kernel_node(const LaunchCfg& cfg, hydro_precision_t prec, void** func) {
  *func = pick(prec, cfg.threads, cfg.minb, cfg.kc);
}

}  // namespace hydro_host
