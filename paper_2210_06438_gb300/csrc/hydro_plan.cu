// hydro_plan.cu -- plans: a fixed batch whose work list is built and uploaded
// once, whose launch shape is picked by timing candidates (autotuner), and
// whose launch is recorded once in a CUDA graph and replayed.  This is the
// aggregation region of Sec. V-D made static: the tasks' chunk table is
// fixed, so the "last task launches one large kernel" step becomes a graph
// replay with no host-side packing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "hydro.h"
#include "hydro_internal.h"
#include "hydro_kernels.cuh"

using hydro_dev::Status;
using hydro_dev::Tile;
using namespace hydro_host;

namespace hydro_host {
int ctx_status_ptr(Status** st, int* n_sm, int* smem_optin);
int validate(const hydro_subgrid_t* sg, int64_t n, int32_t N, int32_t ghost, int32_t F, double gamma);
void build_tiles(const hydro_subgrid_t* sg, int64_t n, int32_t ghost, std::vector<Tile>& tiles,
                 std::vector<int64_t>* first_tile, bool sort_by_cost, int* Fmax, bool* any_multi);
int64_t output_doubles(const hydro_subgrid_t* sg, int64_t n);
}  // namespace hydro_host

struct hydro_plan {
  int device = -1;
  hydro_precision_t prec = HYDRO_FP64;
  int64_t n = 0;
  int Fmax = 6;
  bool multi = false;
  Tile* dev_tiles = nullptr;
  LaunchCfg cfg;
  hydro_plan_info_t info;
  // kernel argument block (addresses are taken for the graph node)
  const Tile* a_tiles = nullptr;
  int a_n = 0, a_F = 0, a_lch = 0;
  double* a_out = nullptr;
  double* a_amax = nullptr;
  Status* a_status = nullptr;
  double a_gamma = 0;
  int a_ws = 1;
  int a_pf = 0;
  int a_scheme = 0;
  void* args[11];
  void* func = nullptr;
  bool use_graph = true;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t knode = nullptr, mnode = nullptr;
};

static void plan_free(hydro_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->dev_tiles) cudaFree(p->dev_tiles);
  delete p;
}

static cudaKernelNodeParams kparams(hydro_plan* p) {
  cudaKernelNodeParams kp;
  memset(&kp, 0, sizeof kp);
  kp.func = p->func;
  kp.gridDim = dim3(p->cfg.grid);
  kp.blockDim = dim3(p->cfg.threads);
  kp.sharedMemBytes = (unsigned)p->cfg.smem;
  kp.kernelParams = p->args;
  return kp;
}

static cudaMemsetParams mparams(hydro_plan* p) {
  cudaMemsetParams mp;
  memset(&mp, 0, sizeof mp);
  mp.dst = p->a_amax;
  mp.elementSize = 4;
  mp.width = (size_t)p->n * 2;
  mp.height = 1;
  mp.pitch = 0;
  mp.value = 0;
  return mp;
}

static int build_graph(hydro_plan* p) {
  cudaError_t e;
  if ((e = cudaGraphCreate(&p->graph, 0)) != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
  if (p->multi) {
    cudaMemsetParams mp = mparams(p);
    if ((e = cudaGraphAddMemsetNode(&p->mnode, p->graph, nullptr, 0, &mp)) != cudaSuccess)
      return cuda_fail(e, "cudaGraphAddMemsetNode");
  }
  cudaKernelNodeParams kp = kparams(p);
  if ((e = cudaGraphAddKernelNode(&p->knode, p->graph, p->multi ? &p->mnode : nullptr,
                                  p->multi ? 1 : 0, &kp)) != cudaSuccess)
    return cuda_fail(e, "cudaGraphAddKernelNode");
  if ((e = cudaGraphInstantiate(&p->exec, p->graph, 0)) != cudaSuccess)
    return cuda_fail(e, "cudaGraphInstantiate");
  return HYDRO_OK;
}

static cudaError_t direct_launch(hydro_plan* p, cudaStream_t st) {
  cudaError_t e;
  if (p->multi && (e = cudaMemsetAsync(p->a_amax, 0, p->n * sizeof(double), st)) != cudaSuccess)
    return e;
  return launch_tiles(p->cfg, p->prec, p->a_tiles, p->a_n, p->a_F, p->a_out, p->a_amax,
                      p->a_status, p->a_gamma, p->a_ws, st, p->a_scheme);
}

// Time `reps` launches of configuration c; returns ms per launch or -1.
static float time_cfg(hydro_plan* p, const LaunchCfg& c, cudaStream_t st, int reps) {
  LaunchCfg keep = p->cfg;
  p->cfg = c;
  p->a_lch = c.lch;
  p->a_pf = c.prefetch;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float ms = -1.f;
  if (direct_launch(p, st) == cudaSuccess) {  // warm-up
    cudaEventRecord(a, st);
    bool ok = true;
    for (int r = 0; r < reps && ok; r++) ok = direct_launch(p, st) == cudaSuccess;
    cudaEventRecord(b, st);
    if (ok && cudaEventSynchronize(b) == cudaSuccess) {
      cudaEventElapsedTime(&ms, a, b);
      ms /= reps;
    }
  }
  cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  p->cfg = keep;
  p->a_lch = keep.lch;
  p->a_pf = keep.prefetch;
  return ms;
}

extern "C" {

int hydro_plan_create(const hydro_subgrid_t* sg, int64_t n, int32_t ghost, double gamma,
                      hydro_precision_t prec, uint32_t flags, void* stream,
                      hydro_plan_t** out_plan) {
  if (!out_plan) return HYDRO_EINVAL;
  *out_plan = nullptr;
  int rc = validate(sg, n, 0, ghost, 0, gamma);
  if (rc) return rc;
  if (n < 1) return HYDRO_EINVAL;
  if (prec != HYDRO_FP64 && prec != HYDRO_FP32_FLUX_FP64_ACC) return HYDRO_EINVAL;
  Status* status;
  int n_sm, smem_optin;
  if ((rc = ctx_status_ptr(&status, &n_sm, &smem_optin))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  hydro_plan* p = new hydro_plan();
  cudaGetDevice(&p->device);
  p->prec = prec;
  p->n = n;
  std::vector<Tile> tiles;
  build_tiles(sg, n, ghost, tiles, nullptr, true, &p->Fmax, &p->multi);
  cudaError_t e;
  if ((e = cudaMalloc(&p->dev_tiles, tiles.size() * sizeof(Tile))) != cudaSuccess) {
    plan_free(p);
    return HYDRO_ENOMEM;
  }
  if ((e = cudaMemcpy(p->dev_tiles, tiles.data(), tiles.size() * sizeof(Tile),
                      cudaMemcpyHostToDevice)) != cudaSuccess) {
    plan_free(p);
    return cuda_fail(e, "cudaMemcpy(work list)");
  }
  memset(&p->info, 0, sizeof p->info);
  p->info.n_subgrids = n;
  p->info.n_tiles = (int64_t)tiles.size();
  p->info.out_doubles = output_doubles(sg, n);
  for (int64_t s = 0; s < n; s++) {
    int64_t N = sg[s].N, F = sg[s].n_fields;
    p->info.interior_cells += N * N * N;
    p->info.alg_bytes += ((N * N * N + 6 * 3 * N * N) + N * N * N) * F * 8 + 8;
  }
  const bool quad26 = (flags & HYDRO_PLAN_QUAD26) != 0;
  p->cfg = default_cfg(prec, p->Fmax, n_sm, smem_optin, (int64_t)tiles.size(),
                       !(flags & HYDRO_PLAN_REGISTER_LOADS), quad26);
  p->a_tiles = p->dev_tiles;
  p->a_n = (int)tiles.size();
  p->a_F = p->Fmax;
  p->a_lch = p->cfg.lch;
  p->a_status = status;
  p->a_gamma = gamma;
  p->a_ws = 1;
  p->a_pf = p->cfg.prefetch;
  p->a_scheme = (flags & HYDRO_PLAN_KNP) ? 1 : 0;
  void* a[11] = {&p->a_tiles, &p->a_n, &p->a_F, &p->a_lch, &p->a_out,
                 &p->a_amax, &p->a_status, &p->a_gamma, &p->a_ws, &p->a_pf, &p->a_scheme};
  memcpy(p->args, a, sizeof a);

  if (flags & HYDRO_PLAN_AUTOTUNE) {
    // scratch outputs for timing (allocated here, freed before returning)
    double *o = nullptr, *am = nullptr;
    if (cudaMalloc(&o, (size_t)p->info.out_doubles * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&am, (size_t)n * sizeof(double)) != cudaSuccess) {
      if (o) cudaFree(o);
      plan_free(p);
      return HYDRO_ENOMEM;
    }
    p->a_out = o;
    p->a_amax = am;
    float best = 1e30f;
    LaunchCfg bestc = p->cfg;
    const int lc[3] = {16, 32, 64};
    int cands = 0;
    for (int vi = 0; vi < num_variants(); vi++)
      for (int li = 0; li < 3; li++)
      for (int pf = 0; pf < 3; pf++) {  // L2 prefetch: off, row segments, planes
        LaunchCfg c;
        variant(vi, &c);
        if (c.kind == kKindQuad) c.threads = quad_threads(prec);
        if (!variant_exists(prec, c)) continue;
        if ((c.kind == kKindQuad) != quad26) continue;  // one scheme per plan
        if (quad26 && (li != 2 || pf != 0)) continue;
        const bool pipe = c.kind == kKindPipe;
        if (pipe && (li != 2 || pf != 0)) continue;  // chunking and prefetch do not apply
        if (pipe && (flags & HYDRO_PLAN_REGISTER_LOADS)) continue;
        if (!pipe && prec != HYDRO_FP64 && (flags & HYDRO_PLAN_PIPELINED)) continue;
        c.lch = lc[li];
        c.prefetch = pf;
        c.smem = smem_bytes(prec, p->Fmax, c.lch, c.kind);
        if (c.smem > smem_optin) continue;
        int occ = occupancy(prec, c);
        if (occ < 1) continue;
        for (int k = 1; k <= occ; k++) {
          c.ctas_per_sm = k;
          int64_t gsz = (int64_t)k * n_sm;
          c.grid = (int)std::min<int64_t>(gsz, (int64_t)tiles.size());
          float ms = time_cfg(p, c, st, 3);
          cands++;
          if (ms > 0 && ms < best) {
            best = ms;
            bestc = c;
          }
          if (c.grid == (int)tiles.size()) break;
        }
      }
    cudaStreamSynchronize(st);
    p->cfg = bestc;
    p->a_lch = bestc.lch;
    p->a_pf = bestc.prefetch;
    p->info.tuned_ms = best < 1e29f ? best : 0.f;
    p->info.n_candidates = cands;
    cudaFree(o);
    cudaFree(am);
    p->a_out = nullptr;
    p->a_amax = nullptr;
  }
  p->info.threads_per_cta = p->cfg.threads;
  p->info.ctas_per_sm = p->cfg.ctas_per_sm;
  p->info.grid = p->cfg.grid;
  p->info.smem_bytes = p->cfg.smem;
  p->info.lines_per_chunk = p->cfg.lch;
  p->info.prefetch = p->cfg.prefetch;
  p->info.regs_cap = 65536 / (p->cfg.threads * p->cfg.minb);
  p->info.load_batch = p->cfg.kc;
  kernel_node(p->cfg, prec, &p->func);
  p->use_graph = !(flags & HYDRO_PLAN_NO_GRAPH);
  *out_plan = p;
  return HYDRO_OK;
}

int hydro_plan_execute(hydro_plan_t* p, double* out, double* amax, void* stream) {
  if (!p || !out || !amax) return HYDRO_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  bool changed = out != p->a_out || amax != p->a_amax;
  p->a_out = out;
  p->a_amax = amax;
  if (!p->use_graph) {
    if ((e = direct_launch(p, st)) != cudaSuccess) return cuda_fail(e, "launch");
    return HYDRO_OK;
  }
  if (!p->exec) {
    int rc = build_graph(p);
    if (rc) return rc;
  } else if (changed) {
    cudaKernelNodeParams kp = kparams(p);
    if ((e = cudaGraphExecKernelNodeSetParams(p->exec, p->knode, &kp)) != cudaSuccess)
      return cuda_fail(e, "cudaGraphExecKernelNodeSetParams");
    if (p->multi) {
      cudaMemsetParams mp = mparams(p);
      if ((e = cudaGraphExecMemsetNodeSetParams(p->exec, p->mnode, &mp)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphExecMemsetNodeSetParams");
    }
  }
  if ((e = cudaGraphLaunch(p->exec, st)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return HYDRO_OK;
}

int hydro_plan_info(const hydro_plan_t* p, hydro_plan_info_t* info) {
  if (!p || !info) return HYDRO_EINVAL;
  *info = p->info;
  return HYDRO_OK;
}

int hydro_plan_destroy(hydro_plan_t* p) {
  if (!p) return HYDRO_EINVAL;
  plan_free(p);
  return HYDRO_OK;
}

}  // extern "C"
