// hydro_launch.cu -- kernel instantiations and launch shapes of libhydro.
#include "hydro_internal.h"
#include "hydro_kernels.cuh"
#include "hydro_quad.cuh"

namespace hydro_host {

using hydro_dev::rhs_tiles_kernel;

// Kernel variants: (kind, threads per CTA, minimum resident CTAs per SM, load
// batch).  For the register-load kernels the third number caps registers per
// thread (65536 / (threads * minb)) and the fourth sets how many read-region
// slots a thread loads at once; the autotuner picks among the variants per
// batch.  The pipelined kernel exists for the mixed form only.
struct Variant {
  int kind, threads, minb, kc;
};
static const Variant kVariants[] = {
    {kKindTiles, 256, 1, 4}, {kKindTiles, 128, 1, 4}, {kKindTiles, 512, 1, 4}, {kKindTiles, 512, 1, 2},
    {kKindTiles, 384, 1, 4}, {kKindTiles, 384, 1, 2}, {kKindTiles, 192, 1, 4}, {kKindTiles, 256, 2, 2},
    {kKindTiles, 128, 2, 2}, {kKindTiles, 448, 1, 2}, {kKindTiles, 576, 1, 1},
    {kKindPipe, kPipeThreads, 1, 0}, {kKindQuad, 0, 1, 0}};  // 26-point: threads by precision
static constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);
static_assert(kPipeThreads == hydro_dev::PNT, "pipelined kernel block size");

template <int MODE>
static void* kfunc(const LaunchCfg& c) {
  if (c.kind == kKindPipe) return MODE == 1 ? (void*)&hydro_dev::rhs_tiles_pipe_kernel<kPipeThreads> : nullptr;
  if (c.kind == kKindQuad) return (void*)&hydro_dev::rhs_quad_kernel<MODE>;
  switch (c.threads) {
    case 128:
      return c.minb == 2 ? (void*)&rhs_tiles_kernel<MODE, 128, 2, 2> : (void*)&rhs_tiles_kernel<MODE, 128, 1, 4>;
    case 192:
      return (void*)&rhs_tiles_kernel<MODE, 192, 1, 4>;
    case 384:
      return c.kc == 2 ? (void*)&rhs_tiles_kernel<MODE, 384, 1, 2> : (void*)&rhs_tiles_kernel<MODE, 384, 1, 4>;
    case 448:
      return (void*)&rhs_tiles_kernel<MODE, 448, 1, 2>;
    case 512:
      return c.kc == 2 ? (void*)&rhs_tiles_kernel<MODE, 512, 1, 2> : (void*)&rhs_tiles_kernel<MODE, 512, 1, 4>;
    case 576:
      return (void*)&rhs_tiles_kernel<MODE, 576, 1, 1>;
    default:
      return c.minb == 2 ? (void*)&rhs_tiles_kernel<MODE, 256, 2, 2> : (void*)&rhs_tiles_kernel<MODE, 256, 1, 4>;
  }
}

static void* pick(hydro_precision_t prec, const LaunchCfg& c) {
  return prec == HYDRO_FP64 ? kfunc<0>(c) : kfunc<1>(c);
}

int quad_threads(hydro_precision_t prec) {
  return prec == HYDRO_FP64 ? hydro_dev::QuadShape<0>::NT : hydro_dev::QuadShape<1>::NT;
}

int num_variants() { return kNumVariants; }
bool variant_exists(hydro_precision_t prec, const LaunchCfg& c) { return pick(prec, c) != nullptr; }
void variant(int i, LaunchCfg* c) {
  c->kind = kVariants[i].kind;
  c->threads = kVariants[i].threads;
  c->minb = kVariants[i].minb;
  c->kc = kVariants[i].kc;
}

cudaError_t kernels_init(int smem_optin) {
  for (int m = 0; m < 2; m++)
    for (int i = 0; i < kNumVariants; i++) {
      LaunchCfg c;
      variant(i, &c);
      void* f = pick((hydro_precision_t)m, c);
      if (!f) continue;
      cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

int smem_bytes(hydro_precision_t prec, int Fmax, int lch, int kind) {
  (void)Fmax;
  if (kind == kKindPipe) return (int)hydro_dev::pipe_smem_bytes();
  if (kind == kKindQuad)
    return (int)(prec == HYDRO_FP64 ? hydro_dev::quad_smem_bytes<0>() : hydro_dev::quad_smem_bytes<1>());
  return (int)(prec == HYDRO_FP64 ? hydro_dev::smem_layout_bytes<0>(lch)
                                  : hydro_dev::smem_layout_bytes<1>(lch));
}

int occupancy(hydro_precision_t prec, const LaunchCfg& c) {
  int nb = 0;
  void* f = pick(prec, c);
  if (!f || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, c.threads, c.smem) != cudaSuccess)
    return 0;
  return nb;
}

static void finish(LaunchCfg& c, hydro_precision_t prec, int n_sm, int64_t n_tiles) {
  c.ctas_per_sm = occupancy(prec, c);
  if (c.ctas_per_sm < 1) c.ctas_per_sm = 1;
  int64_t g = (int64_t)c.ctas_per_sm * n_sm;
  c.grid = (int)(n_tiles < g ? n_tiles : g);
  if (c.grid < 1) c.grid = 1;
}

LaunchCfg default_cfg(hydro_precision_t prec, int Fmax, int n_sm, int smem_optin,
                      int64_t n_tiles, bool pipelined, bool quad26) {
  LaunchCfg c;
  if (quad26) {
    c.kind = kKindQuad;
    c.threads = quad_threads(prec);
    c.minb = 1;
    c.kc = 0;
    c.lch = 64;
    c.smem = smem_bytes(prec, Fmax, c.lch, c.kind);
    finish(c, prec, n_sm, n_tiles);
    return c;
  }
  if (prec != HYDRO_FP64 && pipelined && smem_bytes(prec, Fmax, 64, kKindPipe) <= smem_optin) {
    c.kind = kKindPipe;
    c.threads = kPipeThreads;
    c.minb = 1;
    c.kc = 0;
    c.lch = 64;
    c.smem = smem_bytes(prec, Fmax, c.lch, c.kind);
    finish(c, prec, n_sm, n_tiles);
    return c;
  }
  c.kind = kKindTiles;
  if (prec == HYDRO_FP64) {
    // the binary64 shape the autotuner settles on for batches of this GPU
    // (18 warps, 96 registers, whole tiles' lines per chunk); no L2 prefetch,
    // which does not pay for buffers in host memory
    c.threads = 576;
    c.minb = 1;
    c.kc = 1;
    c.lch = 64;
  } else {
    c.threads = 256;
    c.minb = 1;
    c.kc = 4;
    c.lch = 64;
  }
  c.smem = smem_bytes(prec, Fmax, c.lch, c.kind);
  while (c.smem > smem_optin && c.lch > 16) {
    c.lch /= 2;
    c.smem = smem_bytes(prec, Fmax, c.lch, c.kind);
  }
  finish(c, prec, n_sm, n_tiles);
  return c;
}

cudaError_t launch_tiles(const LaunchCfg& cfg, hydro_precision_t prec, const hydro_dev::Tile* tiles,
                         int n_tiles, int Fmax, double* out, double* amax, hydro_dev::Status* status,
                         double gamma, int write_status, cudaStream_t st, int scheme) {
  int lch = cfg.lch, pf = cfg.prefetch;
  void* args[] = {(void*)&tiles, (void*)&n_tiles, (void*)&Fmax, (void*)&lch, (void*)&out,
                  (void*)&amax, (void*)&status, (void*)&gamma, (void*)&write_status, (void*)&pf,
                  (void*)&scheme};
  return cudaLaunchKernel(pick(prec, cfg), dim3(cfg.grid), dim3(cfg.threads), args, (size_t)cfg.smem, st);
}

void kernel_node(const LaunchCfg& cfg, hydro_precision_t prec, void** func) { *func = pick(prec, cfg); }

}  // namespace hydro_host
