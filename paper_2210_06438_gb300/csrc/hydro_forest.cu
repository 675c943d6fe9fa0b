// hydro_forest.cu -- the RHS of a multi-level forest of sub-grids (the
// adaptive octree mesh of the paper's application, Sec. III): neighbour links
// built on the host, the ghost slabs between levels transferred on the
// device, the fused tile kernel on every leaf, and the flux correction that
// keeps the RHS conservative across levels.
//
// Per call, three launches on the caller's stream:
//   1. forest_ghost_kernel: for every leaf face towards another level, the
//      three-cell ghost slab is built from the coarser leaf (the containing
//      cell) or the four finer leaves (mean of the eight covered cells) into
//      an auxiliary block laid out like a same-level neighbour;
//   2. rhs_forest_kernel: the persistent tile kernel; a read-region cell
//      outside the leaf is read from the same-level neighbour or the
//      auxiliary block; the fluxes through faces towards other levels are
//      stored in per-face registers;
//   3. forest_reflux_kernel: every coarse cell next to finer leaves gets
//      s (mean of the four fine fluxes - its own flux) / dx added, the flux
//      through that face thereby replaced by the fine one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "hydro.h"
#include "hydro_internal.h"
#include "hydro_kernels.cuh"
#include "hydro_quad.cuh"

namespace hydro_host {
int ctx_status_ptr(hydro_dev::Status** st, int* n_sm, int* smem_optin);
}

namespace hydro_dev {

// One auxiliary block: the ghost slab of face `face` (2 d + side) of leaf
// `owner`, from one coarser leaf (kind 0, src[0]) or four finer leaves
// (kind 1, src[ta + 2 tb] by the tangential child offsets ta, tb).
struct AuxDesc {
  int owner, face, kind, pad;
  int src[4];
};

// Leaf geometry: level and block coordinates.
struct LeafGeo {
  int level, bx, by, bz;
};

__device__ __forceinline__ void tangential(int d, int& ta, int& tb) {
  ta = d == 0 ? 1 : 0;
  tb = d == 2 ? 1 : 2;
}

// One thread per (auxiliary block, ghost cell of its 3 x N x N slab), all
// fields.  The slab sits where a same-level neighbour's cells would: depth k
// is cell N-3+k (neighbour below) or k (neighbour above) along d.
__global__ void __launch_bounds__(256)
forest_ghost_kernel(const double* __restrict__ U, double* __restrict__ aux, const AuxDesc* __restrict__ desc,
                    const LeafGeo* __restrict__ geo, int n_aux, int N, int F, int nb0) {
  const long long nn = (long long)N * N, n3 = nn * N, bsz = (long long)F * n3;
  const long long total = (long long)n_aux * 3 * nn;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / (3 * nn));
    const int r = (int)(i - j * 3 * nn);
    const int k = r / (int)nn, rr = r - k * (int)nn, a = rr % N, b = rr / N;
    const AuxDesc dsc = desc[j];
    const int d = dsc.face >> 1, side = dsc.face & 1;
    const LeafGeo og = geo[dsc.owner];
    const int M = nb0 << og.level;  // blocks per edge at the owner's level
    // the same-level block beyond the face (periodic) and the slab cell in it
    const int st = side ? 1 : -1;
    auto wrap = [M](int q) { return q < 0 ? q + M : (q >= M ? q - M : q); };
    const int px = d == 0 ? wrap(og.bx + st) : og.bx;
    const int py = d == 1 ? wrap(og.by + st) : og.by;
    const int pz = d == 2 ? wrap(og.bz + st) : og.bz;
    const int vd = side ? k : N - 3 + k;
    const int vx = d == 0 ? vd : a;
    const int vy = d == 1 ? vd : (d == 0 ? a : b);
    const int vz = d == 2 ? vd : b;
    double* dst = aux + j * bsz + ((long long)vz * N + vy) * N + vx;
    const int gx = px * N + vx, gy = py * N + vy, gz = pz * N + vz;  // level cell index
    if (dsc.kind == 0) {
      const LeafGeo cg = geo[dsc.src[0]];
      const int lx = (gx >> 1) - cg.bx * N, ly = (gy >> 1) - cg.by * N, lz = (gz >> 1) - cg.bz * N;
      const double* src = U + dsc.src[0] * bsz + ((long long)lz * N + ly) * N + lx;
      for (int f = 0; f < F; f++) dst[f * n3] = __ldg(src + f * n3);
    } else {
      const int fx = 2 * gx, fy = 2 * gy, fz = 2 * gz;  // first covered cell of the finer level
      const int cx = fx / N - 2 * px, cy = fy / N - 2 * py, cz = fz / N - 2 * pz;
      const int ca = d == 0 ? cy : cx, cb = d == 2 ? cy : cz;
      const int leaf = __ldg(&desc[j].src[ca + 2 * cb]);
      const LeafGeo fg = geo[leaf];
      const int lx = fx - fg.bx * N, ly = fy - fg.by * N, lz = fz - fg.bz * N;
      const double* src = U + leaf * bsz + ((long long)lz * N + ly) * N + lx;
      for (int f = 0; f < F; f++) {
        const double* q = src + f * n3;
        double s = __ldg(q);
        s = s + __ldg(q + 1);
        s = s + __ldg(q + N);
        s = s + __ldg(q + N + 1);
        s = s + __ldg(q + nn);
        s = s + __ldg(q + nn + 1);
        s = s + __ldg(q + nn + N);
        s = s + __ldg(q + nn + N + 1);
        dst[f * n3] = s * 0.125;
      }
    }
  }
}

// One thread per cell of the leaves that have finer face neighbours (rf),
// all fields; cells not on such a face return at once.  The corrections of
// the x, y and z faces are added in that order; `scale` is 1 for dU/dt and
// beta dt for a stage (beta *dtp when dtp is set).
__global__ void __launch_bounds__(256)
forest_reflux_kernel(const int* __restrict__ links, const AuxDesc* __restrict__ desc,
                     const int* __restrict__ rf, int n_rf, int nl, int N, int F,
                     const double* __restrict__ reg, double* __restrict__ out, double inv_dx0, double scale,
                     double beta, const double* __restrict__ dtp) {
  if (dtp) scale = beta * __ldg(dtp);  // a stage whose dt is in device memory
  const long long nn = (long long)N * N, n3 = nn * N;
  const long long total = (long long)n_rf * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(i / n3);
    const int m = (int)(i - q * n3);
    const int c[3] = {m % N, (m / N) % N, m / (N * N)};
    const int s = rf[q];
    const int* row = links + 8 * s;
    int jf[3], sd[3];
    bool any = false;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      jf[d] = -1;
      sd[d] = c[d] == 0 ? 0 : (c[d] == N - 1 ? 1 : -1);
      if (sd[d] < 0) continue;
      const int blk = row[2 * d + sd[d]];
      if (blk >= nl && desc[blk - nl].kind == 1) {
        jf[d] = blk - nl;
        any = true;
      }
    }
    if (!any) continue;
    const double inv_dx = inv_dx0 * (double)(1u << row[6]);
    double* o = out + (long long)s * F * n3 + m;
    for (int f = 0; f < F; f++) {
      double v = o[f * n3];
#pragma unroll
      for (int d = 0; d < 3; d++) {
        if (jf[d] < 0) continue;
        int ta, tb;
        tangential(d, ta, tb);
        const int a = c[ta], b = c[tb];
        const double Fc = reg[((long long)jf[d] * F + f) * nn + (long long)b * N + a];
        const int ca = (2 * a) / N, cb = (2 * b) / N;
        const int fine = desc[jf[d]].src[ca + 2 * cb];
        const int jr = links[8 * fine + 2 * d + (1 - sd[d])] - nl;  // the fine leaf's face register
        const int fa = 2 * a - ca * N, fb = 2 * b - cb * N;
        const double* r = reg + ((long long)jr * F + f) * nn + (long long)fb * N + fa;
        double sum = r[0];
        sum = sum + r[1];
        sum = sum + r[N];
        sum = sum + r[N + 1];
        const double corr = (sum * 0.25 - Fc) * inv_dx;
        v = v + scale * (sd[d] == 0 ? corr : -corr);
      }
      o[f * n3] = v;
    }
  }
}

// The 26-point variant reads edge and corner ghosts too: each leaf's ghosted
// block (G = N + 6) is gathered whole.  One CTA per leaf (grid-stride over
// the leaves); its threads take the cells of the block with each coordinate
// in [-3, N+2] and at most one at -3 or N+2, all fields, so that the block is
// written contiguously.  nb26[27 s + (dx+1) + 3 (dy+1) + 9 (dz+1)] describes
// the block of the leaf's level at offset (dx, dy, dz): x = 0 a leaf of that
// level (y), -1 inside the coarser leaf y, +1 refined: kids[8 y + i + 2j + 4k]
// are its children (those next to the leaf are leaves).  The leaf's 27
// entries, its geometry and those of the leaves its ghosts come from are read
// once into shared memory; each cell then loads all its fields before it
// stores them.
__global__ void __launch_bounds__(256, 4)
forest_gather26_kernel(const double* __restrict__ U, double* __restrict__ ghost, const int2* __restrict__ nb26,
                       const int* __restrict__ kids, const LeafGeo* __restrict__ geo, int nl, int N, int F,
                       int nb0) {
  constexpr int MAXF = HYDRO_MAX_FIELDS;
  __shared__ int2 nbs[27];
  __shared__ LeafGeo gs;
  // per offset j and child c (8 j + c): the leaf a ghost cell is read from and
  // its geometry; a coarser source in c = 0
  __shared__ int src_leaf[27 * 8];
  __shared__ LeafGeo src_geo[27 * 8];
  const int G = N + 6, g3 = G * G * G, n3 = N * N * N, nn = N * N;
  for (int s = blockIdx.x; s < nl; s += gridDim.x) {
    __syncthreads();  // the previous leaf's readers are done with the tables
    if (threadIdx.x < 27) nbs[threadIdx.x] = nb26[27 * s + threadIdx.x];
    if (threadIdx.x == 0) gs = geo[s];
    __syncthreads();
    if (threadIdx.x < 27 * 8) {
      const int j = threadIdx.x >> 3, c = threadIdx.x & 7;
      const int jx = j % 3 - 1, jy = (j / 3) % 3 - 1, jz = j / 9 - 1;
      const int2 e = nbs[j];
      // the children that ghost cells at this offset fall in: along an axis
      // with offset +1 the low one, with -1 the high one, with 0 both
      const bool next = (jx == 0 || (c & 1) == (jx < 0)) && (jy == 0 || ((c >> 1) & 1) == (jy < 0)) &&
                        (jz == 0 || (c >> 2) == (jz < 0));
      if (j != 13 && e.x > 0 && next) {
        const int leaf = __ldg(kids + 8 * e.y + c);
        src_leaf[threadIdx.x] = leaf;
        src_geo[threadIdx.x] = geo[leaf];
      } else if (j != 13 && e.x < 0 && c == 0) {
        src_geo[threadIdx.x] = geo[e.y];
      }
    }
    __syncthreads();
    const LeafGeo og = gs;
    const int M = nb0 << og.level;
    const double* own = U + (long long)s * F * n3;
    double* blk = ghost + (long long)s * F * g3;
    for (int r = threadIdx.x; r < g3; r += blockDim.x) {
      const int cx = r % G - 3, cy = (r / G) % G - 3, cz = r / (G * G) - 3;
      const int far = (cx == -3 || cx == N + 2) + (cy == -3 || cy == N + 2) + (cz == -3 || cz == N + 2);
      if (far > 1) continue;
      double* dst = blk + r;
      const int sx = cx < 0 ? -1 : (cx >= N ? 1 : 0), sy = cy < 0 ? -1 : (cy >= N ? 1 : 0),
                sz = cz < 0 ? -1 : (cz >= N ? 1 : 0);
      const double* src;
      bool restrict8 = false;
      if (sx == 0 && sy == 0 && sz == 0) {
        src = own + (cz * N + cy) * N + cx;
      } else {
        const int j = (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1);
        const int2 e = nbs[j];
        auto wrap = [M](int q) { return q < 0 ? q + M : (q >= M ? q - M : q); };
        const int px = wrap(og.bx + sx), py = wrap(og.by + sy), pz = wrap(og.bz + sz);
        const int vx = cx - sx * N, vy = cy - sy * N, vz = cz - sz * N;  // cell in block p
        const int gx = px * N + vx, gy = py * N + vy, gz = pz * N + vz;  // level cell index
        if (e.x == 0) {
          src = U + (long long)e.y * F * n3 + (vz * N + vy) * N + vx;
        } else if (e.x < 0) {
          const LeafGeo cg = src_geo[8 * j];
          const int lx = (gx >> 1) - cg.bx * N, ly = (gy >> 1) - cg.by * N, lz = (gz >> 1) - cg.bz * N;
          src = U + (long long)e.y * F * n3 + (lz * N + ly) * N + lx;
        } else {
          const int fx = 2 * gx, fy = 2 * gy, fz = 2 * gz;
          const int ch = (fx / N - 2 * px) + 2 * (fy / N - 2 * py) + 4 * (fz / N - 2 * pz);
          const int leaf = src_leaf[8 * j + ch];
          const LeafGeo fg = src_geo[8 * j + ch];
          const int lx = fx - fg.bx * N, ly = fy - fg.by * N, lz = fz - fg.bz * N;
          src = U + (long long)leaf * F * n3 + (lz * N + ly) * N + lx;
          restrict8 = true;
        }
      }
      if (!restrict8) {
        double v[MAXF];
#pragma unroll
        for (int f = 0; f < MAXF; f++)
          if (f < F) v[f] = __ldg(src + (long long)f * n3);
#pragma unroll
        for (int f = 0; f < MAXF; f++)
          if (f < F) dst[(long long)f * g3] = v[f];
      } else {
#pragma unroll
        for (int f = 0; f < MAXF; f++) {
          if (f < F) {
            const double* q = src + (long long)f * n3;
            double t = __ldg(q);
            t = t + __ldg(q + 1);
            t = t + __ldg(q + N);
            t = t + __ldg(q + N + 1);
            t = t + __ldg(q + nn);
            t = t + __ldg(q + nn + 1);
            t = t + __ldg(q + nn + N);
            t = t + __ldg(q + nn + N + 1);
            dst[(long long)f * g3] = t * 0.125;
          }
        }
      }
    }
  }
}

}  // namespace hydro_dev

using hydro_dev::AuxDesc;
using hydro_dev::LeafGeo;

struct hydro_forest {
  int device = -1;
  int nl = 0, N = 0, F = 0, nb0 = 0, max_level = 0, n_aux = 0, n_rf = 0;
  int* links = nullptr;       // [nl][8]
  LeafGeo* geo = nullptr;     // [nl]
  AuxDesc* desc = nullptr;    // [n_aux]
  int* rf = nullptr;          // [n_rf]
  double* aux = nullptr;      // [n_aux][F][N^3]
  double* reg = nullptr;      // [n_aux][F][N^2]
  bool full = false;          // 26-neighbour 2:1 balance: the 26-point variant is available
  int2* nb26 = nullptr;       // [nl][27]
  int* kids = nullptr;
  double* ghost = nullptr;    // [nl][F][(N+6)^3], allocated by the first 26-point call
  long long bytes = 0;
};

namespace {

// Forest tile kernels (the shapes the autotuner picks for sub-grid batches):
// 0 binary64, register loads, 576 threads; 1 mixed, pipelined (576 threads);
// 2 mixed, register loads, 256 threads (HYDRO_F_REGISTER_LOADS); 3 and 4
// the 26-point variant, binary64 and mixed.
constexpr int kLch = 64, kNumKernels = 5;
constexpr int kThreads[kNumKernels] = {576, hydro_host::kPipeThreads, 256, hydro_dev::QuadShape<0>::NT,
                                       hydro_dev::QuadShape<1>::NT};
constexpr int kKinds[kNumKernels] = {hydro_host::kKindTiles, hydro_host::kKindPipe, hydro_host::kKindTiles,
                                     hydro_host::kKindQuad, hydro_host::kKindQuad};

void* forest_func(int k) {
  switch (k) {
    case 0: return (void*)&hydro_dev::rhs_forest_kernel<0, 576, 1, 1>;
    case 1: return (void*)&hydro_dev::rhs_forest_pipe_kernel<hydro_host::kPipeThreads>;
    case 2: return (void*)&hydro_dev::rhs_forest_kernel<1, 256, 1, 4>;
    case 3: return (void*)&hydro_dev::rhs_forest_quad_kernel<0>;
    default: return (void*)&hydro_dev::rhs_forest_quad_kernel<1>;
  }
}

struct ForestDev {
  bool ready = false;
  int n_sm = 0, occ[kNumKernels] = {0, 0, 0, 0, 0};
  int occ_gather = 1;  // resident CTAs of the 26-point gather per SM
};
ForestDev g_fdev[64];
std::mutex g_fmu;

int forest_setup(int dev, ForestDev** out) {
  if (dev < 0 || dev >= 64) return HYDRO_EINVAL;
  std::lock_guard<std::mutex> g(g_fmu);
  ForestDev& D = g_fdev[dev];
  if (!D.ready) {
    cudaError_t e;
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&D.n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
      return hydro_host::cuda_fail(e, "cudaDeviceGetAttribute");
    for (int m = 0; m < kNumKernels; m++) {
      hydro_precision_t prec = (m == 0 || m == 3) ? HYDRO_FP64 : HYDRO_FP32_FLUX_FP64_ACC;
      int smem = hydro_host::smem_bytes(prec, HYDRO_MAX_FIELDS, kLch, kKinds[m]);
      if ((e = cudaFuncSetAttribute(forest_func(m), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    optin - 1024)) != cudaSuccess)
        return hydro_host::cuda_fail(e, "cudaFuncSetAttribute");
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&D.occ[m], forest_func(m), kThreads[m], smem)) !=
          cudaSuccess)
        return hydro_host::cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      if (D.occ[m] < 1) D.occ[m] = 1;
    }
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&D.occ_gather, hydro_dev::forest_gather26_kernel, 256,
                                                           0)) != cudaSuccess)
      return hydro_host::cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (D.occ_gather < 1) D.occ_gather = 1;
    D.ready = true;
  }
  *out = &D;
  return HYDRO_OK;
}

// ---------------------------------------------------------- host tables --
// Leaf key: level in bits 60-63, block coordinates in 20 bits each.
constexpr int kCoordBits = 20;
static_assert(HYDRO_FOREST_MAX_LEVEL < 16, "the level must fit the key's 4 bits");
inline uint64_t key_of(int L, int x, int y, int z) {
  return ((uint64_t)L << 60) | ((uint64_t)(uint32_t)x << 40) | ((uint64_t)(uint32_t)y << 20) |
         (uint64_t)(uint32_t)z;
}

struct Tables {
  std::vector<int> links;  // [nl][8]
  std::vector<int> kind;   // [nl][6]: -1 coarser, 0 same, +1 finer
  std::vector<int> nbr;    // [nl][6]
  std::vector<AuxDesc> desc;
  std::vector<int> rf;
  int max_level = 0;
  // the 26-neighbour tables of the 26-point variant (built when every leaf's
  // edge and corner neighbours also differ from it by at most one level)
  bool full = false;
  std::vector<int2> nb26;  // [nl][27]
  std::vector<int> kids;   // [8 per refined neighbour block]
};

// Validate the forest and build its neighbour tables.
int build_tables(const hydro_leaf_t* lv, int32_t n, int32_t nb0, int32_t N, Tables& T) {
  if (!lv || n < 1 || nb0 < 1 || N < 6 || N > HYDRO_MAX_N || (N & 1)) return HYDRO_EINVAL;
  std::unordered_map<uint64_t, int> idx;
  idx.reserve((size_t)n * 2);
  int lmax = 0;
  for (int s = 0; s < n; s++) {
    const hydro_leaf_t& l = lv[s];
    if (l.level < 0 || l.level > HYDRO_FOREST_MAX_LEVEL) return HYDRO_EINVAL;
    const int64_t M = (int64_t)nb0 << l.level;
    if (M >= (1 << kCoordBits)) return HYDRO_EINVAL;
    if (l.bx < 0 || l.by < 0 || l.bz < 0 || l.bx >= M || l.by >= M || l.bz >= M) return HYDRO_EINVAL;
    if (!idx.emplace(key_of(l.level, l.bx, l.by, l.bz), s).second) return HYDRO_EINVAL;  // duplicate
    lmax = std::max(lmax, l.level);
  }
  // disjoint: no leaf has an ancestor that is a leaf; cover: the volumes,
  // counted in blocks of the finest level, add up to the cube
  unsigned __int128 vol = 0;
  for (int s = 0; s < n; s++) {
    const hydro_leaf_t& l = lv[s];
    for (int a = 1; a <= l.level; a++)
      if (idx.count(key_of(l.level - a, l.bx >> a, l.by >> a, l.bz >> a))) return HYDRO_EINVAL;
    vol += (unsigned __int128)1 << (3 * (lmax - l.level));
  }
  const unsigned __int128 M = (unsigned __int128)nb0 << lmax;
  if (vol != M * M * M) return HYDRO_EINVAL;

  T.max_level = lmax;
  T.links.assign((size_t)n * 8, 0);
  T.kind.assign((size_t)n * 6, 0);
  T.nbr.assign((size_t)n * 6, 0);
  T.desc.clear();
  T.rf.clear();
  auto find = [&](int L, int x, int y, int z) -> int {
    const int lim = 1 << kCoordBits;
    if (L < 0 || L > HYDRO_FOREST_MAX_LEVEL || x < 0 || y < 0 || z < 0 || x >= lim || y >= lim || z >= lim)
      return -1;
    auto it = idx.find(key_of(L, x, y, z));
    return it == idx.end() ? -1 : it->second;
  };
  for (int s = 0; s < n; s++) {
    const hydro_leaf_t& l = lv[s];
    const int L = l.level, M_L = nb0 << L;
    bool finer = false;
    for (int face = 0; face < 6; face++) {
      const int d = face >> 1, side = face & 1;
      int p[3] = {l.bx, l.by, l.bz};
      p[d] = side ? (p[d] + 1) % M_L : (p[d] + M_L - 1) % M_L;
      int t = find(L, p[0], p[1], p[2]);
      if (t >= 0) {
        T.links[8 * s + face] = t;
        T.kind[6 * s + face] = 0;
        T.nbr[6 * s + face] = t;
        continue;
      }
      AuxDesc a{};
      a.owner = s;
      a.face = face;
      if (L > 0 && (t = find(L - 1, p[0] >> 1, p[1] >> 1, p[2] >> 1)) >= 0) {
        a.kind = 0;
        a.src[0] = a.src[1] = a.src[2] = a.src[3] = t;
        T.kind[6 * s + face] = -1;
        T.nbr[6 * s + face] = t;
      } else {
        const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
        a.kind = 1;
        for (int cb = 0; cb < 2; cb++)
          for (int ca = 0; ca < 2; ca++) {
            int c[3];
            c[d] = 2 * p[d] + (side ? 0 : 1);  // the children touching the face
            c[ta] = 2 * p[ta] + ca;
            c[tb] = 2 * p[tb] + cb;
            if ((t = find(L + 1, c[0], c[1], c[2])) < 0)
              return HYDRO_EINVAL;  // neither same, coarser by one nor finer by one: not 2:1
            a.src[ca + 2 * cb] = t;
          }
        T.kind[6 * s + face] = 1;
        T.nbr[6 * s + face] = a.src[0];
        finer = true;
      }
      T.links[8 * s + face] = n + (int)T.desc.size();
      T.desc.push_back(a);
    }
    T.links[8 * s + 6] = L;
    if (finer) T.rf.push_back(s);
  }
  // 26 neighbours (the face ones included): same level, coarser by one, or
  // refined with every child next to the leaf a leaf of the next level
  T.full = true;
  T.nb26.assign((size_t)n * 27, make_int2(2, -1));
  T.kids.clear();
  for (int s = 0; s < n && T.full; s++) {
    const hydro_leaf_t& l = lv[s];
    const int L = l.level, M_L = nb0 << L;
    for (int k = 0; k < 27 && T.full; k++) {
      const int o[3] = {k % 3 - 1, (k / 3) % 3 - 1, k / 9 - 1};
      if (!o[0] && !o[1] && !o[2]) continue;
      const int p[3] = {(l.bx + o[0] + M_L) % M_L, (l.by + o[1] + M_L) % M_L, (l.bz + o[2] + M_L) % M_L};
      int t = find(L, p[0], p[1], p[2]);
      if (t >= 0) {
        T.nb26[27 * s + k] = make_int2(0, t);
      } else if (L > 0 && (t = find(L - 1, p[0] >> 1, p[1] >> 1, p[2] >> 1)) >= 0) {
        T.nb26[27 * s + k] = make_int2(-1, t);
      } else {
        const int base = (int)(T.kids.size() / 8);
        for (int c = 0; c < 8; c++) {
          const int b[3] = {c & 1, (c >> 1) & 1, c >> 2};
          bool next = true;  // the child touches the leaf
          for (int e = 0; e < 3; e++)
            if ((o[e] == 1 && b[e] == 1) || (o[e] == -1 && b[e] == 0)) next = false;
          t = find(L + 1, 2 * p[0] + b[0], 2 * p[1] + b[1], 2 * p[2] + b[2]);
          if (next && t < 0) T.full = false;
          T.kids.push_back(next ? t : -1);
        }
        T.nb26[27 * s + k] = make_int2(1, base);
      }
    }
  }
  if (!T.full) {
    T.nb26.clear();
    T.kids.clear();
  }
  return HYDRO_OK;
}

template <class T>
int upload(T** dst, const std::vector<T>& v, long long& bytes) {
  *dst = nullptr;
  if (v.empty()) return HYDRO_OK;
  size_t sz = v.size() * sizeof(T);
  if (cudaMalloc((void**)dst, sz) != cudaSuccess) return HYDRO_ENOMEM;
  bytes += (long long)sz;
  cudaError_t e = cudaMemcpy(*dst, v.data(), sz, cudaMemcpyHostToDevice);
  return e == cudaSuccess ? HYDRO_OK : hydro_host::cuda_fail(e, "cudaMemcpy(forest tables)");
}

void release(hydro_forest* f) {
  cudaFree(f->nb26);
  cudaFree(f->kids);
  cudaFree(f->ghost);
  cudaFree(f->links);
  cudaFree(f->geo);
  cudaFree(f->desc);
  cudaFree(f->rf);
  cudaFree(f->aux);
  cudaFree(f->reg);
}

int forest_launch(hydro_forest* fo, const double* U, const double* U0, double alpha, double beta, double dt,
                  int stage, double dx0, double gamma, double* out, double* amax, hydro_precision_t prec,
                  void* stream, uint32_t flags, const double* dtp = nullptr) {
  if (!fo || !U || !out || !amax || (stage && !U0)) return HYDRO_EINVAL;
  if (flags & ~(uint32_t)(HYDRO_F_KNP | HYDRO_F_REGISTER_LOADS | HYDRO_F_QUAD26)) return HYDRO_EINVAL;
  const bool quad26 = (flags & HYDRO_F_QUAD26) != 0;
  if (quad26 && !fo->full) return HYDRO_EINVAL;  // edge/corner neighbours more than one level apart
  if (!(dx0 > 0.0) || !std::isfinite(dx0) || !(gamma > 1.0) || !std::isfinite(gamma)) return HYDRO_EINVAL;
  if (prec != HYDRO_FP64 && prec != HYDRO_FP32_FLUX_FP64_ACC) return HYDRO_EINVAL;
  if (stage && (!std::isfinite(alpha) || !std::isfinite(beta) || !std::isfinite(dt))) return HYDRO_EINVAL;
  if ((reinterpret_cast<uintptr_t>(U) | reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(U0)) &
      7)
    return HYDRO_EINVAL;
  if (out == U) return HYDRO_EINVAL;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hydro_host::cuda_fail(e, "cudaGetDevice");
  if (dev != fo->device) return HYDRO_EINVAL;
  ForestDev* D;
  int rc = forest_setup(dev, &D);
  if (rc) return rc;
  hydro_dev::Status* status;
  int n_sm, optin;
  if ((rc = hydro_host::ctx_status_ptr(&status, &n_sm, &optin))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int N = fo->N, F = fo->F;
  const int tpe = (N + hydro_dev::TE - 1) / hydro_dev::TE;
  const long long n_tiles = (long long)fo->nl * tpe * tpe * tpe;
  if (tpe > 1 && (e = cudaMemsetAsync(amax, 0, (size_t)fo->nl * sizeof(double), st)) != cudaSuccess)
    return hydro_host::cuda_fail(e, "cudaMemsetAsync(amax)");
  int ex2;
  const bool pow2 = std::frexp(dx0, &ex2) == 0.5 && ex2 > -120 && ex2 < 120;
  if (dtp && (reinterpret_cast<uintptr_t>(dtp) & 7)) return HYDRO_EINVAL;
  hydro_dev::StageArgs sa{U, stage ? U0 : U, alpha, beta, dt, stage, dtp};
  int nt = (int)n_tiles, lch = kLch, ws = 1, scheme = (flags & HYDRO_F_KNP) ? 1 : 0;
  if (quad26) {
    // 1. the ghosted blocks, edges and corners included
    const int G = N + 6;
    if (!fo->ghost) {
      const size_t gb = (size_t)fo->nl * F * G * G * G * sizeof(double);
      if (cudaMalloc(&fo->ghost, gb) != cudaSuccess) {
        fo->ghost = nullptr;
        return HYDRO_ENOMEM;
      }
      fo->bytes += (long long)gb;
    }
    // one wave of resident CTAs over the leaves
    const int gg = (int)std::min<long long>((long long)fo->nl, (long long)D->n_sm * D->occ_gather);
    hydro_dev::forest_gather26_kernel<<<gg, 256, 0, st>>>(U, fo->ghost, fo->nb26, fo->kids, fo->geo, fo->nl, N,
                                                          F, fo->nb0);
    if ((e = cudaGetLastError()) != cudaSuccess) return hydro_host::cuda_fail(e, "forest gather launch");
    // 2. the 26-point tiles
    const int m = prec == HYDRO_FP64 ? 3 : 4;
    hydro_dev::ForestQuadTiles fq{fo->ghost, fo->links, fo->reg, fo->nl, N, F, tpe, 1.0 / dx0,
                                  (short)(pow2 ? 2 : 0)};
    const long long g64 = (long long)D->occ[m] * D->n_sm;
    const int grid = (int)(n_tiles < g64 ? n_tiles : g64);
    size_t smem = (size_t)hydro_host::smem_bytes(prec, F, lch, kKinds[m]);
    void* args[] = {(void*)&fq, (void*)&nt, (void*)&lch, (void*)&out, (void*)&amax, (void*)&status,
                    (void*)&gamma, (void*)&ws, (void*)&scheme, (void*)&sa};
    if ((e = cudaLaunchKernel(forest_func(m), dim3(grid), dim3(kThreads[m]), args, smem, st)) != cudaSuccess)
      return hydro_host::cuda_fail(e, "forest 26-point launch");
  } else {
    // 1. level transfer
    if (fo->n_aux > 0) {
      const long long cells = (long long)fo->n_aux * 3 * N * N;
      const int grid = (int)std::min<long long>((cells + 255) / 256, (long long)D->n_sm * 8);
      hydro_dev::forest_ghost_kernel<<<grid, 256, 0, st>>>(U, fo->aux, fo->desc, fo->geo, fo->n_aux, N, F,
                                                           fo->nb0);
      if ((e = cudaGetLastError()) != cudaSuccess) return hydro_host::cuda_fail(e, "forest ghost launch");
    }
    // 2. tiles
    hydro_dev::ForestTiles ft{U, fo->aux, fo->links, fo->reg, fo->nl, N, F, tpe, 1.0 / dx0, (short)(pow2 ? 2 : 0)};
    const int m = prec == HYDRO_FP64 ? 0 : ((flags & HYDRO_F_REGISTER_LOADS) ? 2 : 1);
    const long long g64 = (long long)D->occ[m] * D->n_sm;
    const int grid = (int)(n_tiles < g64 ? n_tiles : g64);
    size_t smem = (size_t)hydro_host::smem_bytes(prec, F, lch, kKinds[m]);
    void* args[] = {(void*)&ft, (void*)&nt, (void*)&lch, (void*)&out, (void*)&amax, (void*)&status,
                    (void*)&gamma, (void*)&ws, (void*)&scheme, (void*)&sa};
    if ((e = cudaLaunchKernel(forest_func(m), dim3(grid), dim3(kThreads[m]), args, smem, st)) != cudaSuccess)
      return hydro_host::cuda_fail(e, "forest tile launch");
  }
  // 3. flux correction
  if (fo->n_rf > 0) {
    const long long cells = (long long)fo->n_rf * N * N * N;
    const int g = (int)std::min<long long>((cells + 255) / 256, (long long)D->n_sm * 8);
    const double scale = stage ? beta * dt : 1.0;
    hydro_dev::forest_reflux_kernel<<<g, 256, 0, st>>>(fo->links, fo->desc, fo->rf, fo->n_rf, fo->nl, N, F,
                                                       fo->reg, out, 1.0 / dx0, scale, beta, stage ? dtp : nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return hydro_host::cuda_fail(e, "forest reflux launch");
  }
  return HYDRO_OK;
}

}  // namespace

extern "C" {

int hydro_forest_links(const hydro_leaf_t* leaves, int32_t n_leaves, int32_t nb0, int32_t N, int32_t* kind,
                       int32_t* nbr) {
  Tables T;
  int rc = build_tables(leaves, n_leaves, nb0, N, T);
  if (rc) return rc;
  if (kind) std::copy(T.kind.begin(), T.kind.end(), kind);
  if (nbr) std::copy(T.nbr.begin(), T.nbr.end(), nbr);
  return HYDRO_OK;
}

int hydro_forest_create(const hydro_leaf_t* leaves, int32_t n_leaves, int32_t nb0, int32_t N, int32_t n_fields,
                        hydro_forest_t** out) {
  if (!out) return HYDRO_EINVAL;
  *out = nullptr;
  if (n_fields < 6 || n_fields > HYDRO_MAX_FIELDS) return HYDRO_EINVAL;
  Tables T;
  int rc = build_tables(leaves, n_leaves, nb0, N, T);
  if (rc) return rc;
  const int tpe = (N + hydro_dev::TE - 1) / hydro_dev::TE;
  if ((long long)n_leaves * tpe * tpe * tpe > 0x7fffffffLL) return HYDRO_EINVAL;
  hydro_forest* f = new hydro_forest();
  cudaError_t e = cudaGetDevice(&f->device);
  if (e != cudaSuccess) {
    delete f;
    return hydro_host::cuda_fail(e, "cudaGetDevice");
  }
  f->nl = n_leaves;
  f->N = N;
  f->F = n_fields;
  f->nb0 = nb0;
  f->max_level = T.max_level;
  f->n_aux = (int)T.desc.size();
  f->n_rf = (int)T.rf.size();
  f->full = T.full;
  std::vector<LeafGeo> geo((size_t)n_leaves);
  for (int s = 0; s < n_leaves; s++) geo[s] = {leaves[s].level, leaves[s].bx, leaves[s].by, leaves[s].bz};
  if ((rc = upload(&f->links, T.links, f->bytes)) || (rc = upload(&f->geo, geo, f->bytes)) ||
      (rc = upload(&f->desc, T.desc, f->bytes)) || (rc = upload(&f->rf, T.rf, f->bytes)) ||
      (rc = upload(&f->nb26, T.nb26, f->bytes)) || (rc = upload(&f->kids, T.kids, f->bytes))) {
    release(f);
    delete f;
    return rc;
  }
  if (f->n_aux > 0) {
    const size_t aux = (size_t)f->n_aux * n_fields * N * N * N * sizeof(double);
    const size_t reg = (size_t)f->n_aux * n_fields * N * N * sizeof(double);
    if (cudaMalloc(&f->aux, aux) != cudaSuccess || cudaMalloc(&f->reg, reg) != cudaSuccess) {
      release(f);
      delete f;
      return HYDRO_ENOMEM;
    }
    f->bytes += (long long)(aux + reg);
  }
  *out = f;
  return HYDRO_OK;
}

int hydro_forest_info(const hydro_forest_t* f, hydro_forest_info_t* info) {
  if (!f || !info) return HYDRO_EINVAL;
  std::memset(info, 0, sizeof(*info));
  info->n_leaves = f->nl;
  info->N = f->N;
  info->n_fields = f->F;
  info->nb0 = f->nb0;
  info->max_level = f->max_level;
  info->n_level_faces = f->n_aux;
  info->n_reflux_leaves = f->n_rf;
  info->quad26 = f->full ? 1 : 0;
  info->device_bytes = f->bytes;
  return HYDRO_OK;
}

int hydro_forest_rhs(hydro_forest_t* forest, const double* U, double dx0, double gamma, double* out_dUdt,
                     double* out_amax, hydro_precision_t prec, void* stream, uint32_t flags) {
  return forest_launch(forest, U, nullptr, 0.0, 0.0, 0.0, 0, dx0, gamma, out_dUdt, out_amax, prec, stream, flags);
}

int hydro_forest_stage(hydro_forest_t* forest, const double* U, const double* U0, double alpha, double beta,
                       double dt, double dx0, double gamma, double* U_out, double* out_amax,
                       hydro_precision_t prec, void* stream, uint32_t flags) {
  return forest_launch(forest, U, U0, alpha, beta, dt, 1, dx0, gamma, U_out, out_amax, prec, stream, flags);
}

int hydro_forest_stage_dt(hydro_forest_t* forest, const double* U, const double* U0, double alpha, double beta,
                          const double* dt, double dx0, double gamma, double* U_out, double* out_amax,
                          hydro_precision_t prec, void* stream, uint32_t flags) {
  if (!dt) return HYDRO_EINVAL;
  return forest_launch(forest, U, U0, alpha, beta, 0.0, 1, dx0, gamma, U_out, out_amax, prec, stream, flags, dt);
}

int hydro_forest_destroy(hydro_forest_t* f) {
  if (!f) return HYDRO_EINVAL;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != f->device) cudaSetDevice(f->device);
  cudaDeviceSynchronize();
  release(f);
  if (prev >= 0 && prev != f->device) cudaSetDevice(prev);
  delete f;
  return HYDRO_OK;
}

}  // extern "C"
