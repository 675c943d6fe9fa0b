// hydro_kernels.cuh -- device code of the aggregated hydro RHS (sm_103a).
//
// One work item is an 8x8x8 tile of a sub-grid (an 8^3 sub-grid is one tile,
// a 16^3 sub-grid eight; other N give partial edge tiles).  The RHS of a
// sub-grid is the union of its tiles' RHS: every face flux depends only on
// the cells within 3 of the face along its normal, so a flux on a face shared
// by two tiles is computed twice from the same inputs by the same code and is
// bitwise identical both times.  This is the "larger sub-problem" of Sec. V-B
// turned around: the GPU always sees 8^3 work items, whatever the sub-grid
// size, and many of them per launch (the aggregated kernel of Sec. V-D).
//
// Per tile, one CTA:
//   1. stage the tile's read region (interior rows with their x ghosts, plus
//      the y and z ghost slabs: 1664 cells) from HBM, converting to primitive
//      variables on the way into shared memory                    (step A0-A1)
//   2. for each direction, in chunks of lines: PPM face states of every
//      (line, field) (step A2), then the central flux of every face with its
//      signal speed (step A3), written back in place
//   3. every thread owns fixed cells and accumulates the flux differences of
//      x, then y, then z in registers (step A4); the result is scaled by
//      -1/dx and stored.  The largest signal speed is reduced with warp
//      shuffles and one atomic per tile (step A5).
//
// MODE 0 runs every step in binary64.  MODE 1 (mixed) keeps the primitive
// recovery and the dual-energy decision in binary64, rounds primitives to
// binary32, reconstructs and fluxes in binary32, and carries the flux
// differences and their sum as exact binary32 pairs (error-free two-sums) so
// that the binary64 result telescopes like the binary64 form.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hydro_dev {

constexpr int TE = 8;             // tile edge
constexpr int LL = TE + 6;        // line length with 3 ghosts on each side
constexpr int NFC = TE + 1;       // faces per line
constexpr int NLN = TE * TE;      // lines per direction
constexpr int XROWS = TE * TE * LL;         // interior rows with x ghosts: 896
constexpr int YSLAB = TE * 6 * TE;          // y ghost slabs: 384
constexpr int STAR = XROWS + 2 * YSLAB;     // 1664 cells read per tile
constexpr int MAXF = 11;
constexpr double ETA = 1e-3;      // dual-energy switch threshold

struct __align__(16) Tile {
  const double* U;     // sub-grid input base
  long long out_off;   // first output double of the sub-grid
  double inv_dx;       // 1/dx
  int sub;             // sub-grid index within the batch
  int N;               // sub-grid interior edge
  int F;               // fields
  int G;               // stored edge N + 2*ghost
  int ghost;
  short ox, oy, oz;    // tile origin (cells)
  short multi;         // 1 if the sub-grid has more than one tile
};
static_assert(sizeof(Tile) == 64, "tile descriptor is 64 bytes");

struct Status {
  unsigned int flags;          // bit 0: nonphysical input
  unsigned int pad;
  unsigned long long first_bad;  // smallest flagged sub-grid index
};

// ----------------------------------------------------------- star slots --
// Shared-memory slot of tile-local cell (x, y, z) of the read region.
__device__ __forceinline__ int slot_of(int x, int y, int z) {
  if ((unsigned)y < (unsigned)TE && (unsigned)z < (unsigned)TE) return (z * TE + y) * LL + (x + 3);
  if ((unsigned)z < (unsigned)TE) {
    int yg = y < 0 ? y + 3 : y - TE + 3;
    return XROWS + (z * 6 + yg) * TE + x;
  }
  int zg = z < 0 ? z + 3 : z - TE + 3;
  return XROWS + YSLAB + (zg * TE + y) * TE + x;
}

__device__ __forceinline__ void cell_of(int s, int& x, int& y, int& z) {
  if (s < XROWS) {
    z = s / (TE * LL);
    int r = s - z * (TE * LL);
    y = r / LL;
    x = r - y * LL - 3;
  } else if (s < XROWS + YSLAB) {
    int t = s - XROWS;
    z = t / (6 * TE);
    int r = t - z * (6 * TE);
    int yg = r / TE;
    x = r - yg * TE;
    y = yg < 3 ? yg - 3 : yg + TE - 3;
  } else {
    int t = s - XROWS - YSLAB;
    int zg = t / (TE * TE);
    int r = t - zg * (TE * TE);
    y = r / TE;
    x = r - y * TE;
    z = zg < 3 ? zg - 3 : zg + TE - 3;
  }
}

// tile-local coordinates of position c (0..LL-1, cell c-3) of line l along d
__device__ __forceinline__ int line_slot(int d, int l, int c) {
  int a = l % TE, b = l / TE;
  if (d == 0) return slot_of(c - 3, a, b);
  if (d == 1) return slot_of(a, c - 3, b);
  return slot_of(a, b, c - 3);
}

// ------------------------------------------------------------ step A1 --
// Conserved -> primitive (rho, v, p, phi = tau/rho, X_k = rho_k/rho).  The
// quantities that decide the dual-energy branch (|s|^2, e_kin, e_int and the
// threshold) are formed with explicitly rounded operations in the same order
// as the reference definition, so that the branch is taken identically.
__device__ __forceinline__ bool primitives64(const double* u, int F, double gamma, double* w) {
  double rho = u[0];
  double ssq = __dadd_rn(__dadd_rn(__dmul_rn(u[1], u[1]), __dmul_rn(u[2], u[2])),
                         __dmul_rn(u[3], u[3]));
  double ekin = __ddiv_rn(__dmul_rn(0.5, ssq), rho);
  double E = u[4];
  double eint = __dsub_rn(E, ekin);
  if (eint < __dmul_rn(ETA, E)) eint = pow(u[5], gamma);
  double p = __dmul_rn(gamma - 1.0, eint);
  w[0] = rho;
  w[1] = u[1] / rho;
  w[2] = u[2] / rho;
  w[3] = u[3] / rho;
  w[4] = p;
  w[5] = u[5] / rho;
#pragma unroll
  for (int f = 6; f < MAXF; f++)
    if (f < F) w[f] = u[f] / rho;
  bool bad = !(rho > 0.0) || !(p > 0.0);
#pragma unroll
  for (int f = 0; f < MAXF; f++)
    if (f < F) bad |= !isfinite(u[f]) || !isfinite(w[f]);
  return bad;
}

// ------------------------------------------------------------ step A2 --
// PPM along one line of LL cells (Colella & Woodward 1984): monotonised
// central slopes, 4th-order face values, parabola limiter.  Produces the
// states left and right of the NFC faces i-1/2, i = 0..TE:
//   left[i]  = q+ of cell i-1,  right[i] = q- of cell i.
template <typename R>
__device__ __forceinline__ void ppm_line(const R* q, R* left, R* right) {
  const R half = R(0.5), sixth = R(1.0 / 6.0);
  R delta[LL];
#pragma unroll
  for (int c = 1; c <= LL - 2; c++) {
    R dp = q[c + 1] - q[c];
    R dm = q[c] - q[c - 1];
    R dbar = half * (q[c + 1] - q[c - 1]);
    bool mono = (dp > R(0) && dm > R(0)) || (dp < R(0) && dm < R(0));
    R m = fmin(fabs(dbar), fmin(R(2) * fabs(dm), R(2) * fabs(dp)));
    delta[c] = mono ? copysign(m, dbar) : R(0);
  }
  R face[LL];
#pragma unroll
  for (int c = 1; c <= LL - 3; c++) face[c] = half * (q[c] + q[c + 1]) - (delta[c + 1] - delta[c]) * sixth;
#pragma unroll
  for (int c = 2; c <= LL - 3; c++) {  // cells -1 .. TE
    R qc = q[c], lo = face[c - 1], hi = face[c];
    R up = hi - qc, dn = qc - lo;
    bool ext = !((up > R(0) && dn > R(0)) || (up < R(0) && dn < R(0)));
    R D = hi - lo;
    R mid = qc - half * (lo + hi);
    R Dm = D * mid, D2 = D * D * sixth;
    R lo2 = (Dm > D2) ? R(3) * qc - R(2) * hi : lo;
    R hi2 = (!(Dm > D2) && Dm < -D2) ? R(3) * qc - R(2) * lo : hi;
    lo = ext ? qc : lo2;
    hi = ext ? qc : hi2;
    int j = c - 3;               // cell index -1 .. TE
    if (j >= 0) right[j] = lo;   // face j-1/2 sees q- of cell j
    if (j + 1 <= TE) left[j + 1] = hi;  // face j+1/2 sees q+ of cell j
  }
}

// ------------------------------------------------------------ step A3 --
// Central flux (Kurganov & Tadmor 2000) through a face normal to axis d:
//   Fhat = (F(wl) + F(wr))/2 - a (U(wr) - U(wl))/2,
//   a = max(|u_l| + c_l, |u_r| + c_r), c = sqrt(gamma p / rho).
template <typename R>
__device__ __forceinline__ R kt_flux(const R* wl, const R* wr, int F, int d, R gamma, R* fhat) {
  const R half = R(0.5);
  R Ul[MAXF], Fl[MAXF], Ur[MAXF], Fr[MAXF];
  R al, ar;
#pragma unroll
  for (int side = 0; side < 2; side++) {
    const R* w = side ? wr : wl;
    R* U = side ? Ur : Ul;
    R* Fx = side ? Fr : Fl;
    R rho = w[0], vx = w[1], vy = w[2], vz = w[3], p = w[4];
    R u = d == 0 ? vx : (d == 1 ? vy : vz);
    R vsq = (vx * vx + vy * vy) + vz * vz;
    R E = p / (gamma - R(1)) + half * rho * vsq;
    U[0] = rho;
    U[1] = rho * vx;
    U[2] = rho * vy;
    U[3] = rho * vz;
    U[4] = E;
#pragma unroll
    for (int f = 5; f < MAXF; f++)
      if (f < F) U[f] = rho * w[f];
    Fx[0] = rho * u;
    Fx[1] = U[1] * u + (d == 0 ? p : R(0));
    Fx[2] = U[2] * u + (d == 1 ? p : R(0));
    Fx[3] = U[3] * u + (d == 2 ? p : R(0));
    Fx[4] = (E + p) * u;
#pragma unroll
    for (int f = 5; f < MAXF; f++)
      if (f < F) Fx[f] = U[f] * u;
    R c = sqrt(gamma * p / rho);
    if (side) ar = fabs(u) + c; else al = fabs(u) + c;
  }
  R a = fmax(al, ar);
  R ha = half * a;
#pragma unroll
  for (int f = 0; f < MAXF; f++)
    if (f < F) fhat[f] = half * (Fl[f] + Fr[f]) - ha * (Ur[f] - Ul[f]);
  return a;
}

// ------------------------------------------------- exact binary32 pairs --
struct F2 { float h, l; };
__device__ __forceinline__ F2 two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 pair_add(F2 a, F2 b) {
  F2 s = two_sum(a.h, b.h);
  F2 t = two_sum(a.l, b.l);
  s.l = __fadd_rn(s.l, t.h);
  s = fast_two_sum(s.h, s.l);
  s.l = __fadd_rn(s.l, t.l);
  return fast_two_sum(s.h, s.l);
}

// ------------------------------------------------------------- kernel --
template <int MODE> struct Prec;
template <> struct Prec<0> { typedef double R; typedef double Acc; };
template <> struct Prec<1> { typedef float R; typedef F2 Acc; };

__device__ __forceinline__ double acc_to_double(double a) { return a; }
__device__ __forceinline__ double acc_to_double(F2 a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ void acc_diff(double& acc, double hi, double lo, bool first) {
  double d = hi - lo;
  acc = first ? d : acc + d;
}
__device__ __forceinline__ void acc_diff(F2& acc, float hi, float lo, bool first) {
  F2 d = two_sum(hi, -lo);
  acc = first ? d : pair_add(acc, d);
}

// Shared memory (R = element type of the mode):
//   W  [Fmax][STAR]          primitives of the read region
//   QS [2][Fmax][lch][NFC]   left/right face states, then fluxes in place
template <int MODE, int NT>
__global__ void __launch_bounds__(NT, 1)
rhs_tiles_kernel(const Tile* __restrict__ tiles, int n_tiles, int Fmax, int lch, double* __restrict__ out,
                 double* __restrict__ amax_out, Status* __restrict__ status, double gamma_d,
                 int write_status) {
  typedef typename Prec<MODE>::R R;
  typedef typename Prec<MODE>::Acc Acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* W = reinterpret_cast<R*>(smem_raw);
  R* QS = W + (size_t)Fmax * STAR;
  __shared__ double red[NT / 32];
  const int tid = threadIdx.x;
  const R gamma = R(gamma_d);
  constexpr int CPT = (TE * TE * TE + NT - 1) / NT;  // owned cells per thread

  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const Tile tile = tiles[t];
    const int F = tile.F, G = tile.G, N = tile.N, gh = tile.ghost;
    const int ex = min(TE, N - tile.ox), ey = min(TE, N - tile.oy), ez = min(TE, N - tile.oz);
    const long long plane = (long long)G * G * G;

    // ---- A0/A1: stage the read region as primitives
    bool bad = false;
    for (int s = tid; s < STAR; s += NT) {
      int x, y, z;
      cell_of(s, x, y, z);
      // read region of a (possibly partial) tile: at most one coordinate
      // outside the tile, and that one at most 3 cells out
      int outside = (x < 0 || x >= ex) + (y < 0 || y >= ey) + (z < 0 || z >= ez);
      bool valid = outside <= 1 && x < ex + 3 && y < ey + 3 && z < ez + 3;
      double u[MAXF], w[MAXF];
      if (valid) {
        const double* p = tile.U + ((long long)(tile.oz + z + gh) * G + (tile.oy + y + gh)) * G +
                          (tile.ox + x + gh);
#pragma unroll
        for (int f = 0; f < MAXF; f++)
          if (f < F) u[f] = __ldg(p + f * plane);
        bad |= primitives64(u, F, gamma_d, w);
      } else {
#pragma unroll
        for (int f = 0; f < MAXF; f++) w[f] = (f == 0 || f == 4) ? 1.0 : 0.0;
      }
#pragma unroll
      for (int f = 0; f < MAXF; f++)
        if (f < F) W[f * STAR + s] = R(w[f]);
    }
    bad = __syncthreads_or(bad);
    if (bad && tid == 0 && write_status) {
      atomicOr(&status->flags, 1u);
      atomicMin(&status->first_bad, (unsigned long long)tile.sub);
    }

    Acc acc[CPT][MAXF];
    R amax = R(0);
    for (int d = 0; d < 3; d++) {
      const int e_d = d == 0 ? ex : (d == 1 ? ey : ez);
      const int e_a = d == 0 ? ey : ex;  // first tangential axis extent
      const int e_b = d == 2 ? ey : ez;  // second tangential axis extent
      for (int l0 = 0; l0 < NLN; l0 += lch) {
        // ---- A2: PPM per (line, field)
        for (int task = tid; task < lch * F; task += NT) {
          int ll = task % lch, f = task / lch;
          int l = l0 + ll;
          R q[LL], lf[NFC], rt[NFC];
#pragma unroll
          for (int c = 0; c < LL; c++) q[c] = W[f * STAR + line_slot(d, l, c)];
          ppm_line<R>(q, lf, rt);
          R* qs = QS + ((size_t)f * lch + ll) * NFC;
          R* qr = QS + ((size_t)(Fmax + f) * lch + ll) * NFC;
#pragma unroll
          for (int i = 0; i < NFC; i++) { qs[i] = lf[i]; qr[i] = rt[i]; }
        }
        __syncthreads();
        // ---- A3: central flux per face, written over the left states
        for (int task = tid; task < lch * NFC; task += NT) {
          int ll = task / NFC, i = task - ll * NFC;
          int l = l0 + ll;
          R wl[MAXF], wr[MAXF], fh[MAXF];
#pragma unroll
          for (int f = 0; f < MAXF; f++)
            if (f < F) {
              wl[f] = QS[((size_t)f * lch + ll) * NFC + i];
              wr[f] = QS[((size_t)(Fmax + f) * lch + ll) * NFC + i];
            }
          R a = kt_flux<R>(wl, wr, F, d, gamma, fh);
          bool fvalid = (l % TE) < e_a && (l / TE) < e_b && i <= e_d;
          if (fvalid) amax = fmax(amax, a);
#pragma unroll
          for (int f = 0; f < MAXF; f++)
            if (f < F) QS[((size_t)f * lch + ll) * NFC + i] = fh[f];
        }
        __syncthreads();
        // ---- A4: flux differences into the owned cells, x then y then z
#pragma unroll
        for (int k = 0; k < CPT; k++) {
          int m = tid + k * NT;
          if (m < TE * TE * TE) {
            int x = m % TE, y = (m / TE) % TE, z = m / (TE * TE);
            int l = d == 0 ? z * TE + y : (d == 1 ? z * TE + x : y * TE + x);
            int pos = d == 0 ? x : (d == 1 ? y : z);
            if (l >= l0 && l < l0 + lch) {
              const R* fl = QS + (size_t)(l - l0) * NFC + pos;
#pragma unroll
              for (int f = 0; f < MAXF; f++)
                if (f < F) acc_diff(acc[k][f], fl[(size_t)f * lch * NFC + 1], fl[(size_t)f * lch * NFC], d == 0);
            }
          }
        }
        __syncthreads();
      }
    }
    // ---- store dU/dt = -(sum of differences)/dx
    const long long n3 = (long long)N * N * N;
    const double scale = -tile.inv_dx;
#pragma unroll
    for (int k = 0; k < CPT; k++) {
      int m = tid + k * NT;
      if (m < TE * TE * TE) {
        int x = m % TE, y = (m / TE) % TE, z = m / (TE * TE);
        if (x < ex && y < ey && z < ez) {
          double* o = out + tile.out_off + ((long long)(tile.oz + z) * N + (tile.oy + y)) * N + (tile.ox + x);
#pragma unroll
          for (int f = 0; f < MAXF; f++)
            if (f < F) o[f * n3] = acc_to_double(acc[k][f]) * scale;
        }
      }
    }
    // ---- A5: largest signal speed of the tile
    double am = (double)amax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) am = fmax(am, __shfl_xor_sync(0xffffffffu, am, o));
    if ((tid & 31) == 0) red[tid >> 5] = am;
    __syncthreads();
    if (tid == 0) {
      double m = red[0];
      for (int w = 1; w < NT / 32; w++) m = fmax(m, red[w]);
      if (tile.multi)
        atomicMax(reinterpret_cast<unsigned long long*>(amax_out + tile.sub),
                  (unsigned long long)__double_as_longlong(m));
      else
        amax_out[tile.sub] = m;
    }
    __syncthreads();
  }
}

}  // namespace hydro_dev
