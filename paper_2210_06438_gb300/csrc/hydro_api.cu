// hydro_api.cu -- host side of libhydro: argument validation, the tile work
// list (the aggregation allocator's chunk table of Sec. V-D), launches, plans
// with CUDA-graph replay and autotuning, and the sticky device status word.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hydro.h"
#include "hydro_internal.h"
#include "hydro_kernels.cuh"
#include "hydro_uniform.cuh"

using hydro_dev::Tile;
using hydro_dev::Status;

namespace hydro_dev {

// The work list of a uniform batch, built on the device from its sub-grid
// descriptors (24 bytes each instead of 64 per tile from the host).
__global__ void __launch_bounds__(256) expand_uniform_kernel(UniformDesc u, int n_tiles, Tile* __restrict__ tiles) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_tiles) tiles[t] = u(t);
}

}  // namespace hydro_dev

namespace hydro_host {

thread_local std::string g_last_cuda_error = "no CUDA error";

int cuda_fail(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  g_last_cuda_error = buf;
  return HYDRO_ECUDA;
}

// ------------------------------------------------------------ device ctx --
// One per device.  `mu` guards the one-time set-up, the ring cursor and the
// status word; each ring slot has its own lock, held by the call that fills
// the slot's work list until its launch is recorded, so that calls from
// several host threads (or on several devices) build their work lists and
// wait for their slots concurrently.
struct DeviceCtx {
  std::mutex mu;
  bool ready = false;
  int device = -1;
  int n_sm = 0;
  int smem_optin = 0;
  Status* status = nullptr;  // sticky status word (device)
  // ring of work-list slots for the non-plan entry points
  static constexpr int RING = 4;
  std::mutex slot_mu[RING];
  Tile* dev_tiles[RING] = {};
  Tile* host_tiles[RING] = {};  // pinned staging
  size_t cap[RING] = {};
  std::vector<int64_t> first[RING];  // per-sub-grid first tile (hydro_rhs_per_subgrid)
  cudaEvent_t done[RING] = {};
  int next = 0;
};

static DeviceCtx g_ctx[64];

static const Status kStatusClear = {0u, 0u, ~0ull};

int ctx_get(DeviceCtx** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return HYDRO_EINVAL;
  DeviceCtx& c = g_ctx[dev];
  std::lock_guard<std::mutex> g(c.mu);
  if (!c.ready) {
    c.device = dev;
    if ((e = cudaDeviceGetAttribute(&c.n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return cuda_fail(e, "cudaDeviceGetAttribute(SM count)");
    if ((e = cudaDeviceGetAttribute(&c.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
        cudaSuccess)
      return cuda_fail(e, "cudaDeviceGetAttribute(smem)");
    c.smem_optin -= 1024;  // room for the kernels' static shared memory
    if (!c.status && (e = cudaMalloc(&c.status, sizeof(Status))) != cudaSuccess) return HYDRO_ENOMEM;
    if ((e = cudaMemcpy(c.status, &kStatusClear, sizeof(Status), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return cuda_fail(e, "cudaMemcpy(status)");
    for (int i = 0; i < DeviceCtx::RING; i++)
      if (!c.done[i] && (e = cudaEventCreateWithFlags(&c.done[i], cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "cudaEventCreate");
    if ((e = kernels_init(c.smem_optin)) != cudaSuccess) return cuda_fail(e, "kernel attributes");
    c.ready = true;
  }
  *out = &c;
  return HYDRO_OK;
}

int ctx_status_ptr(Status** st, int* n_sm, int* smem_optin) {
  DeviceCtx* c;
  int rc = ctx_get(&c);
  if (rc) return rc;
  *st = c->status;
  *n_sm = c->n_sm;
  *smem_optin = c->smem_optin;
  return HYDRO_OK;
}

// --------------------------------------------------------- validation --
int validate(const hydro_subgrid_t* sg, int64_t n, int32_t N, int32_t ghost, int32_t F,
             double gamma) {
  if (n < 0) return HYDRO_EINVAL;
  if (n > 0 && !sg) return HYDRO_EINVAL;
  if (ghost < 3 || ghost > 64) return HYDRO_EINVAL;
  if (!(gamma > 1.0) || !std::isfinite(gamma)) return HYDRO_EINVAL;
  if (n > (int64_t)1 << 31) return HYDRO_EINVAL;
  for (int64_t s = 0; s < n; s++) {
    const hydro_subgrid_t& d = sg[s];
    if (!d.U) return HYDRO_EINVAL;
    if (d.N < 2 || d.N > HYDRO_MAX_N) return HYDRO_EINVAL;
    if (d.n_fields < 6 || d.n_fields > HYDRO_MAX_FIELDS) return HYDRO_EINVAL;
    if (!(d.dx > 0.0) || !std::isfinite(d.dx)) return HYDRO_EINVAL;
    if (N > 0 && d.N != N) return HYDRO_EINVAL;
    if (F > 0 && d.n_fields != F) return HYDRO_EINVAL;
    if (reinterpret_cast<uintptr_t>(d.U) % 8 != 0) return HYDRO_EINVAL;
  }
  return HYDRO_OK;
}

int64_t output_doubles(const hydro_subgrid_t* sg, int64_t n) {
  int64_t tot = 0;
  for (int64_t s = 0; s < n; s++) tot += (int64_t)sg[s].n_fields * sg[s].N * sg[s].N * sg[s].N;
  return tot;
}

void fill_tile(Tile& t, const hydro_subgrid_t& d, int ghost, int64_t out_off, int64_t amax_off,
               int sub, int tx, int ty, int tz, bool multi) {
  memset(&t, 0, sizeof t);
  t.U = d.U;
  t.out_off = out_off;
  t.amax_off = amax_off;
  t.inv_dx = 1.0 / d.dx;
  t.sub = sub;
  t.N = d.N;
  t.F = d.n_fields;
  t.G = d.N + 2 * ghost;
  t.ox = (short)(tx * hydro_dev::TE);
  t.oy = (short)(ty * hydro_dev::TE);
  t.oz = (short)(tz * hydro_dev::TE);
  int ex2;
  bool pow2 = std::frexp(d.dx, &ex2) == 0.5 && ex2 > -120 && ex2 < 120;
  t.flags = (short)((multi ? 1 : 0) | (pow2 ? 2 : 0));
}

// Size of a batch's work list: tiles, whether any sub-grid spans several
// tiles, the largest field count, whether all sub-grids have one, and
// (uniform_N, if given) whether they all have one edge N.
void count_tiles(const hydro_subgrid_t* sg, int64_t n, int64_t* n_tiles, bool* any_multi, int* Fmax,
                 bool* uniform_F, bool* uniform_N = nullptr) {
  int64_t nt = 0;
  bool multi = false, uni = true, uniN = true;
  int fm = 6;
  for (int64_t s = 0; s < n; s++) {
    const int64_t e = (sg[s].N + hydro_dev::TE - 1) / hydro_dev::TE;
    nt += e * e * e;
    multi |= e > 1;
    fm = std::max(fm, (int)sg[s].n_fields);
    uni &= sg[s].n_fields == sg[0].n_fields;
    uniN &= sg[s].N == sg[0].N;
  }
  *n_tiles = nt;
  *any_multi = multi;
  *Fmax = fm;
  *uniform_F = uni;
  if (uniform_N) *uniform_N = uniN;
}

// Work list: one Tile per 8^3 tile written to `tiles` (room for the count of
// count_tiles), in descriptor order or (sort_by_cost) the largest field
// counts first, so that the longest tiles start first.  The fields of a
// sub-grid's tiles are filled once and copied per tile.  first_tile, if
// given (n + 1 entries), receives each sub-grid's first tile.
void fill_tiles(const hydro_subgrid_t* sg, int64_t n, int32_t ghost, Tile* tiles, int64_t* first_tile,
                bool sort_by_cost) {
  std::vector<int64_t> off, order;
  if (sort_by_cost) {
    off.assign(n + 1, 0);
    for (int64_t s = 0; s < n; s++) off[s + 1] = off[s] + (int64_t)sg[s].n_fields * sg[s].N * sg[s].N * sg[s].N;
    order.resize(n);
    for (int64_t s = 0; s < n; s++) order[s] = s;
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t a, int64_t b) { return sg[a].n_fields > sg[b].n_fields; });
  }
  int64_t k_out = 0, run = 0;  // run: output offset in descriptor order
  double last_dx = -1.0, inv_dx = 0.0;
  short pow2 = 0;
  for (int64_t k = 0; k < n; k++) {
    const int64_t s = sort_by_cost ? order[k] : k;
    const hydro_subgrid_t& d = sg[s];
    const int nt = (d.N + hydro_dev::TE - 1) / hydro_dev::TE;
    if (first_tile) first_tile[s] = k_out;
    if (d.dx != last_dx) {  // 1/dx and the power-of-two test once per run of equal widths
      last_dx = d.dx;
      inv_dx = 1.0 / d.dx;
      int ex2;
      pow2 = (std::frexp(d.dx, &ex2) == 0.5 && ex2 > -120 && ex2 < 120) ? 2 : 0;
    }
    Tile t{d.U, sort_by_cost ? off[s] : run, s, inv_dx, (int)s, d.N, d.n_fields, d.N + 2 * ghost,
           0, 0, 0, (short)((nt > 1 ? 1 : 0) | pow2), {0, 0}};
    run += (int64_t)d.n_fields * d.N * d.N * d.N;
    for (int tz = 0; tz < nt; tz++)
      for (int ty = 0; ty < nt; ty++)
        for (int tx = 0; tx < nt; tx++) {
          t.ox = (short)(tx * hydro_dev::TE);
          t.oy = (short)(ty * hydro_dev::TE);
          t.oz = (short)(tz * hydro_dev::TE);
          tiles[k_out++] = t;
        }
  }
  if (first_tile) first_tile[n] = k_out;
}

// The same into a vector (plans build their work list once).
void build_tiles(const hydro_subgrid_t* sg, int64_t n, int32_t ghost, std::vector<Tile>& tiles,
                 std::vector<int64_t>* first_tile, bool sort_by_cost, int* Fmax, bool* any_multi) {
  int64_t nt;
  bool uni;
  count_tiles(sg, n, &nt, any_multi, Fmax, &uni);
  tiles.resize((size_t)nt);
  if (first_tile) first_tile->assign(n + 1, 0);
  fill_tiles(sg, n, ghost, tiles.data(), first_tile ? first_tile->data() : nullptr, sort_by_cost && !uni);
}

// Take the next ring slot for a work list of `need` tiles: its lock is held
// in *lk until the caller has recorded the slot's event after its launch;
// the slot's previous launch has finished (its host and device buffers are
// free) and they have room for `need` tiles.
int acquire_slot(DeviceCtx* c, int64_t need, int* slot_out, std::unique_lock<std::mutex>* lk) {
  int slot;
  {
    std::lock_guard<std::mutex> g(c->mu);
    slot = c->next;
    c->next = (c->next + 1) % DeviceCtx::RING;
  }
  *lk = std::unique_lock<std::mutex>(c->slot_mu[slot]);
  cudaError_t e;
  if ((e = cudaEventSynchronize(c->done[slot])) != cudaSuccess)
    return cuda_fail(e, "cudaEventSynchronize(ring)");
  if ((size_t)std::max<int64_t>(need, 1) > c->cap[slot]) {
    size_t cap = std::max<size_t>((size_t)need, 1024);
    if (c->dev_tiles[slot]) cudaFree(c->dev_tiles[slot]);
    if (c->host_tiles[slot]) cudaFreeHost(c->host_tiles[slot]);
    c->dev_tiles[slot] = nullptr;
    c->host_tiles[slot] = nullptr;
    c->cap[slot] = 0;
    if (cudaMalloc(&c->dev_tiles[slot], cap * sizeof(Tile)) != cudaSuccess) return HYDRO_ENOMEM;
    if (cudaMallocHost(&c->host_tiles[slot], cap * sizeof(Tile)) != cudaSuccess) return HYDRO_ENOMEM;
    c->cap[slot] = cap;
  }
  *slot_out = slot;
  return HYDRO_OK;
}

}  // namespace hydro_host

using namespace hydro_host;

// ================================================================ C ABI ==
extern "C" {

int hydro_version(void) { return 100; }

const char* hydro_strerror(int s) {
  switch (s) {
    case HYDRO_OK: return "ok";
    case HYDRO_EINVAL: return "invalid argument";
    case HYDRO_ENOMEM: return "out of device or pinned memory";
    case HYDRO_ECUDA: return "CUDA runtime error";
    case HYDRO_ENONPHYS: return "nonphysical input (rho <= 0, p <= 0 or non-finite)";
    case HYDRO_EBUDGET: return "task exceeds the serving memory budget";
    case HYDRO_ETIMEDOUT: return "timed out";
    case HYDRO_EBUSY: return "busy";
    case HYDRO_ETOOBIG: return "batch exceeds the fixed scratch of the no-allocation entry point";
    default: return "unknown status";
  }
}

const char* hydro_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

int64_t hydro_output_doubles(const hydro_subgrid_t* sg, int64_t n) {
  if (n < 0 || (n > 0 && !sg)) return -1;
  for (int64_t s = 0; s < n; s++)
    if (sg[s].N < 2 || sg[s].N > HYDRO_MAX_N || sg[s].n_fields < 6 ||
        sg[s].n_fields > HYDRO_MAX_FIELDS)
      return -1;
  return output_doubles(sg, n);
}

int hydro_rhs_ex(const hydro_subgrid_t* sg, int64_t n, int32_t N, int32_t ghost, int32_t F,
                 double gamma, double* out, double* amax, hydro_precision_t prec, void* stream,
                 uint32_t flags) {
  int rc = validate(sg, n, N, ghost, F, gamma);
  if (rc) return rc;
  if (prec != HYDRO_FP64 && prec != HYDRO_FP32_FLUX_FP64_ACC) return HYDRO_EINVAL;
  if (n == 0) return HYDRO_OK;
  if (!out || !amax) return HYDRO_EINVAL;
  DeviceCtx* c;
  if ((rc = ctx_get(&c))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t nt;
  int Fmax;
  bool multi, uniF, uniN;
  count_tiles(sg, n, &nt, &multi, &Fmax, &uniF, &uniN);
  if (nt > 0x7fffffffLL) return HYDRO_EINVAL;
  // A batch of one N and one field count sends its descriptors and builds
  // the work list on the device (descriptor order, as the host would);
  // others send the work list, sorted by cost when the field counts differ.
  const bool uniform = uniN && uniF;
  const int64_t desc_slots = uniform ? (n * (int64_t)sizeof(hydro_subgrid_t) + sizeof(Tile) - 1) / sizeof(Tile) : 0;
  int slot;
  std::unique_lock<std::mutex> lk;
  if ((rc = acquire_slot(c, nt + desc_slots, &slot, &lk))) return rc;
  cudaError_t e;
  Tile* dt = c->dev_tiles[slot];
  if (uniform) {
    // descriptors behind the work list in the slot's device buffer
    hydro_subgrid_t* dd = reinterpret_cast<hydro_subgrid_t*>(dt + nt);
    memcpy(c->host_tiles[slot], sg, (size_t)n * sizeof(hydro_subgrid_t));
    if ((e = cudaMemcpyAsync(dd, c->host_tiles[slot], (size_t)n * sizeof(hydro_subgrid_t), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpyAsync(descriptors)");
    const int N0 = sg[0].N, tpe = (N0 + hydro_dev::TE - 1) / hydro_dev::TE;
    hydro_dev::UniformDesc u{dd, N0, sg[0].n_fields, N0 + 2 * ghost, tpe};
    hydro_dev::expand_uniform_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(u, (int)nt, dt);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "work-list launch");
  } else {
    fill_tiles(sg, n, ghost, c->host_tiles[slot], nullptr, !uniF);  // a batch of one field count needs no sort
    if ((e = cudaMemcpyAsync(dt, c->host_tiles[slot], (size_t)nt * sizeof(Tile), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return cuda_fail(e, "cudaMemcpyAsync(work list)");
  }
  if (multi && (e = cudaMemsetAsync(amax, 0, n * sizeof(double), st)) != cudaSuccess)
    return cuda_fail(e, "cudaMemsetAsync(amax)");
  LaunchCfg cfg = default_cfg(prec, Fmax, c->n_sm, c->smem_optin, nt, !(flags & HYDRO_F_REGISTER_LOADS),
                              (flags & HYDRO_F_QUAD26) != 0);
  if ((e = launch_tiles(cfg, prec, dt, (int)nt, Fmax, out, amax, c->status, gamma, !(flags & HYDRO_F_NO_STATUS),
                        st, (flags & HYDRO_F_KNP) ? 1 : 0)) != cudaSuccess)
    return cuda_fail(e, "launch");
  if ((e = cudaEventRecord(c->done[slot], st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  return HYDRO_OK;
}

int hydro_rhs(const hydro_subgrid_t* sg, int64_t n, int32_t N, int32_t ghost, int32_t F,
              double gamma, double* out, double* amax) {
  return hydro_rhs_ex(sg, n, N, ghost, F, gamma, out, amax, HYDRO_FP64, nullptr, 0u);
}

int hydro_rhs_per_subgrid(const hydro_subgrid_t* sg, int64_t n, int32_t ghost, double gamma,
                          double* out, double* amax, hydro_precision_t prec, void* const* streams,
                          int32_t n_streams) {
  return hydro_rhs_per_subgrid_ex(sg, n, ghost, gamma, out, amax, prec, streams, n_streams, 0u);
}

int hydro_rhs_per_subgrid_ex(const hydro_subgrid_t* sg, int64_t n, int32_t ghost, double gamma,
                             double* out, double* amax, hydro_precision_t prec, void* const* streams,
                             int32_t n_streams, uint32_t flags) {
  if (flags & ~(uint32_t)(HYDRO_F_NO_STATUS | HYDRO_F_KNP | HYDRO_F_QUAD26 | HYDRO_F_REGISTER_LOADS))
    return HYDRO_EINVAL;
  int rc = validate(sg, n, 0, ghost, 0, gamma);
  if (rc) return rc;
  if (prec != HYDRO_FP64 && prec != HYDRO_FP32_FLUX_FP64_ACC) return HYDRO_EINVAL;
  if (n_streams < 1 || !streams) return HYDRO_EINVAL;
  if (n == 0) return HYDRO_OK;
  if (!out || !amax) return HYDRO_EINVAL;
  DeviceCtx* c;
  if ((rc = ctx_get(&c))) return rc;
  int64_t nt;
  int Fmax;
  bool multi, uniF;
  count_tiles(sg, n, &nt, &multi, &Fmax, &uniF);
  if (nt > 0x7fffffffLL) return HYDRO_EINVAL;
  cudaStream_t s0 = (cudaStream_t)streams[0];
  int slot;
  std::unique_lock<std::mutex> lk;
  if ((rc = acquire_slot(c, nt, &slot, &lk))) return rc;
  std::vector<int64_t>& first = c->first[slot];
  first.assign(n + 1, 0);
  fill_tiles(sg, n, ghost, c->host_tiles[slot], first.data(), false);
  Tile* dt = c->dev_tiles[slot];
  cudaError_t e;
  if ((e = cudaMemcpyAsync(dt, c->host_tiles[slot], (size_t)nt * sizeof(Tile), cudaMemcpyHostToDevice, s0)) !=
      cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync(work list)");
  // every stream starts after the work list is on the device
  cudaEvent_t ready = c->done[slot];
  if ((e = cudaEventRecord(ready, s0)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  for (int i = 1; i < n_streams; i++)
    if ((e = cudaStreamWaitEvent((cudaStream_t)streams[i], ready, 0)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamWaitEvent");
  for (int64_t s = 0; s < n; s++) {
    cudaStream_t st = (cudaStream_t)streams[s % n_streams];
    const int nts = (int)(first[s + 1] - first[s]);
    int F = sg[s].n_fields;
    if (nts > 1 && (e = cudaMemsetAsync(amax + s, 0, sizeof(double), st)) != cudaSuccess)
      return cuda_fail(e, "cudaMemsetAsync(amax)");
    LaunchCfg cfg = default_cfg(prec, F, c->n_sm, c->smem_optin, nts, !(flags & HYDRO_F_REGISTER_LOADS),
                                (flags & HYDRO_F_QUAD26) != 0);
    cfg.grid = nts;
    if ((e = launch_tiles(cfg, prec, dt + first[s], nts, F, out, amax, c->status, gamma,
                          !(flags & HYDRO_F_NO_STATUS), st, (flags & HYDRO_F_KNP) ? 1 : 0)) !=
        cudaSuccess)
      return cuda_fail(e, "launch");
  }
  // the ring slot is free once every stream has finished
  for (int i = 1; i < n_streams; i++) {
    if ((e = cudaEventRecord(ready, (cudaStream_t)streams[i])) != cudaSuccess)
      return cuda_fail(e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(s0, ready, 0)) != cudaSuccess) return cuda_fail(e, "wait");
  }
  if ((e = cudaEventRecord(ready, s0)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  return HYDRO_OK;
}

int hydro_status(void* stream, int64_t* first_bad) {
  DeviceCtx* c;
  int rc;
  if ((rc = ctx_get(&c))) return rc;
  std::lock_guard<std::mutex> g(c->mu);
  cudaError_t e;
  if ((e = cudaStreamSynchronize((cudaStream_t)stream)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamSynchronize");
  Status h;
  if ((e = cudaMemcpy(&h, c->status, sizeof h, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpy(status)");
  if ((e = cudaMemcpy(c->status, &kStatusClear, sizeof h, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpy(status clear)");
  if (h.flags & 1u) {
    if (first_bad) *first_bad = (int64_t)h.first_bad;
    return HYDRO_ENONPHYS;
  }
  if (first_bad) *first_bad = -1;
  return HYDRO_OK;
}

}  // extern "C"
