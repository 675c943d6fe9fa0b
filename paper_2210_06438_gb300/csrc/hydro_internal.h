// hydro_internal.h -- declarations shared by libhydro's host translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "hydro.h"

namespace hydro_dev {
struct Tile;
struct Status;
}  // namespace hydro_dev

namespace hydro_host {

// Kernel families: the register-load tile kernels, the pipelined mixed
// kernel, the 26-point quadrature kernels.
constexpr int kKindTiles = 0, kKindPipe = 1, kKindQuad = 2;
constexpr int kPipeThreads = 576;  // threads of the pipelined mixed kernel

// Launch shape of the tile kernel.
struct LaunchCfg {
  int kind = kKindTiles;
  int threads = 256;   // threads per CTA
  int minb = 1;        // kernel variant: minimum resident CTAs per SM it was compiled for
  int kc = 4;          // kernel variant: read-region slots per load batch (register-load kernels)
  int lch = 32;        // lines per chunk of the reconstruct/flux phases (16, 32 or 64)
  int grid = 0;        // CTAs (persistent: a multiple of the SM count)
  int ctas_per_sm = 1;
  int smem = 0;        // dynamic shared memory bytes
  int prefetch = 0;    // L2 prefetch of the next tile: 0 none, 1 per row, 2 per plane
};

cudaError_t kernels_init(int smem_optin);
int smem_bytes(hydro_precision_t prec, int Fmax, int lch, int kind = kKindTiles);
int occupancy(hydro_precision_t prec, const LaunchCfg& c);  // c.smem must be set
// threads per CTA of the 26-point kernel of a precision
int quad_threads(hydro_precision_t prec);
int num_variants();
void variant(int i, LaunchCfg* c);  // sets kind, threads, minb, kc
bool variant_exists(hydro_precision_t prec, const LaunchCfg& c);
// pipelined: use the pipelined mixed kernel (ignored for binary64);
// quad26: the 26-point quadrature kernel (takes precedence)
LaunchCfg default_cfg(hydro_precision_t prec, int Fmax, int n_sm, int smem_optin, int64_t n_tiles,
                      bool pipelined = true, bool quad26 = false);
// scheme: 0 Kurganov-Tadmor flux, 1 Kurganov-Noelle-Petrova
cudaError_t launch_tiles(const LaunchCfg& cfg, hydro_precision_t prec, const hydro_dev::Tile* tiles,
                         int n_tiles, int Fmax, double* out, double* amax, hydro_dev::Status* status,
                         double gamma, int write_status, cudaStream_t st, int scheme = 0);
// kernel entry and argument block, for graph nodes
void kernel_node(const LaunchCfg& cfg, hydro_precision_t prec, void** func);

extern thread_local std::string g_last_cuda_error;
int cuda_fail(cudaError_t e, const char* what);

}  // namespace hydro_host
