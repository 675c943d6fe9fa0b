// hydro_quad.cuh -- the 26-point quadrature variant of the hydro RHS.
//
// Sec. IV-B: PPM values at 26 points on the surface of every cell (6 face
// centres, 12 edge midpoints, 8 vertices), central-upwind fluxes at those
// points and Newton-Cotes quadrature of the fluxes over each face.  The value
// of a cell at its surface point c + v/2 (v in {-1,0,1}^3) is the PPM face
// value of the one-dimensional reconstruction along the line of cells
// c + m v (cells m = -2..2 enter); a face normal to axis d carries the 9
// points e_d + o1 e_a + o2 e_b, the left state from the low cell's line along
// that vector (upper end), the right state from the high cell's line along
// e_d - o1 e_a - o2 e_b (lower end), and the face flux is Simpson's rule in
// both tangential directions, sum_p c_p Fhat_p / 36, c_p = (1,4,1)x(1,4,1).
//
// One CTA per 8^3 tile (persistent over the tile list, one CTA per SM):
//   load   hydro primitives and 1/rho of the tile's read region (every cell
//          with each coordinate in [-3, e+2] and at most one of them at -3 or
//          e+2) into shared memory.  Species: binary64 reads them through the
//          read-only cache and divides by rho on use; the mixed form stores
//          X_k = rho_k/rho of the region in binary32 once per tile;
//   faces  per direction.  Binary64 (192 threads): each thread owns three
//          consecutive faces of one line, walked with the points in pairs
//          (o, -o) so that each single-cell reconstruction gives a state at
//          two points; the weighted point fluxes are summed in shared memory.
//          Mixed: each thread owns 576 / HYDRO_QUAD_MIXED_THREADS faces,
//          reconstructs both states of every point and sums the weighted
//          fluxes in registers;
//   A4     each thread owns up to three cells and accumulates x, y, z flux
//          differences (binary64, or exact binary32 pairs in the mixed form).
#pragma once

#include "hydro_kernels.cuh"

namespace hydro_dev {

constexpr int QBLK = LL * LL * LL;        // 2744 cells of the ghosted 14^3 neighbourhood
constexpr int QFACES = NLN * NFC;         // 576 faces per direction
#ifndef HYDRO_QUAD_MIXED_THREADS
#define HYDRO_QUAD_MIXED_THREADS 576
#endif
// Threads per CTA: binary64 192 (3 faces per thread and direction, one CTA
// per SM); mixed HYDRO_QUAD_MIXED_THREADS (faces per thread 576 / that).
template <int MODE>
struct QuadShape {
  static constexpr int NT = MODE == 0 ? 192 : HYDRO_QUAD_MIXED_THREADS;
  static constexpr int FPT = QFACES / NT;                    // faces per thread and direction
  static constexpr int CPT = (TE * TE * TE + NT - 1) / NT;   // accumulated cells per thread
  static_assert(QFACES % NT == 0 && NT % 32 == 0, "faces divide evenly over whole warps");
};

// Shared memory: hydro primitives and 1/rho of the neighbourhood, the face
// fluxes of one direction, and (mixed form) the species X_k = rho_k/rho of
// the neighbourhood, formed once per tile.
template <int MODE>
__host__ __device__ constexpr size_t quad_smem_bytes() {
  return (MODE == 0 ? 8 : 4) *
         ((size_t)6 * QBLK + QBLK + (size_t)QFACES * MAXF + (MODE == 0 ? 0 : (size_t)(MAXF - 6) * QBLK));
}

__device__ __forceinline__ int qidx(int x, int y, int z) { return ((z + 3) * LL + (y + 3)) * LL + (x + 3); }

// PPM face values of the middle cell of five line values q[0..4] (cells
// -2..2), in the offset form of ppm_line64: up = dq_0/2 - (delta_1 -
// delta_0)/6 and dn = dq_-1 - up_-1 (subscripts relative to the middle cell).
__device__ __forceinline__ void ppm5_64(const double* q, double& lo, double& hi) {
  const double sixth = 1.0 / 6.0;
  double dq[4];
#pragma unroll
  for (int c = 0; c < 4; c++) dq[c] = q[c + 1] - q[c];
  double del[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {  // cells -1, 0, 1
    const double dm = dq[c], dp = dq[c + 1];
    double dbar = dhalf(dp + dm);
    double m = dminp(dabs(dbar), dtwice(dminp(dabs(dm), dabs(dp))));
    del[c] = dsame(dp, dm) ? dcopysign(m, dbar) : 0.0;
  }
  const double qc = q[2];
  const double upm = fma(del[0] - del[1], sixth, dhalf(dq[1]));  // up of cell -1
  const double up = fma(del[1] - del[2], sixth, dhalf(dq[2]));   // up of the middle cell
  const double dn = dq[1] - upm;
  bool ext = !dsame(up, dn);
  bool A = dabs_gt(dn, dtwice(up)), B = dabs_gt(up, dtwice(dn));
  lo = ext ? qc : qc - (A ? dtwice(up) : dn);
  hi = ext ? qc : qc + (B ? dtwice(dn) : up);
}

// The same for binary32, in ppm_line32x2's half-slope and clamp form.
__device__ __forceinline__ void ppm5_32(const float* q, float& lo, float& hi) {
  float d0 = q[1] - q[0], d1 = q[2] - q[1], d2 = q[3] - q[2], d3 = q[4] - q[3];
  float h1 = hslope1(d0, d1, (d0 + d1) * 0.25f, d0 * d1);
  float h2 = hslope1(d1, d2, (d1 + d2) * 0.25f, d1 * d2);
  float h3 = hslope1(d2, d3, (d2 + d3) * 0.25f, d2 * d3);
  const float qc = q[2];
  float l = fmaf(h1 - h2, 1.0f / 3.0f, (q[1] + q[2]) * 0.5f);
  float h = fmaf(h2 - h3, 1.0f / 3.0f, (q[2] + q[3]) * 0.5f);
  float up = h - qc, dn = qc - l;
  float uu = up + up, du = dn + dn;
  limit1(qc, l, h, up, dn, up * dn, uu, du, qc - uu, qc + du, lo, hi);
}
// ppm5_32 on two fields at once: the additions and products as packed
// binary32 pairs (each lane rounded as the scalar instruction rounds it),
// the slope and limiter selections per lane -- the same bits as two calls.
__device__ __forceinline__ void ppm5_32x2(const float2* q, float2& lo, float2& hi) {
  const float2 d0 = sub2(q[1], q[0]), d1 = sub2(q[2], q[1]), d2 = sub2(q[3], q[2]), d3 = sub2(q[4], q[3]);
  const float2 h1 = hslope32x2(d0, d1), h2 = hslope32x2(d1, d2), h3 = hslope32x2(d2, d3);
  const float2 qc = q[2];
  const float2 l = fma2(sub2(h1, h2), f2(1.0f / 3.0f), mul2(add2(q[1], q[2]), f2(0.5f)));
  const float2 h = fma2(sub2(h2, h3), f2(1.0f / 3.0f), mul2(add2(q[2], q[3]), f2(0.5f)));
  const float2 up = sub2(h, qc), dn = sub2(qc, l);
  const float2 uu = add2(up, up), du = add2(dn, dn);
  const float2 e = mul2(up, dn), lc = sub2(qc, uu), hc = add2(qc, du);
  limit1(qc.x, l.x, h.x, up.x, dn.x, e.x, uu.x, du.x, lc.x, hc.x, lo.x, hi.x);
  limit1(qc.y, l.y, h.y, up.y, dn.y, e.y, uu.y, du.y, lc.y, hc.y, lo.y, hi.y);
}

template <int MODE>
struct QuadPrec;
template <>
struct QuadPrec<0> {
  typedef double R;
  typedef double Acc;
};
template <>
struct QuadPrec<1> {
  typedef float R;
  typedef F2 Acc;  // exact binary32 pair (h + l)
};

__device__ __forceinline__ void two_diff1(float a, float b, float& s, float& e) {
  s = a - b;
  float bb = s - a;
  e = (a - (s - bb)) - (b + bb);
}

// DOMAIN: the tiles belong to a periodic cube of pad[0]^3 sub-grids stored
// without ghosts (as in tile_loop); `stage` may turn the output into an
// explicit stage update.  CAP: forest leaves read from their gathered
// ghosted blocks; the fluxes through faces towards other levels are recorded
// (`fetch.capture`), and `stage` applies (outputs in the forest layout).
template <int MODE, class Fetch, bool DOMAIN = false, bool CAP = false>
__device__ __forceinline__ void tile_loop_quad(const Fetch& fetch, int n_tiles, double* __restrict__ out,
                                               double* __restrict__ amax_out, Status* __restrict__ status,
                                               double gamma_d, int write_status, bool knp,
                                               const StageArgs& stage = StageArgs{nullptr, nullptr, 0.0, 0.0,
                                                                                  0.0, 0}) {
  typedef typename QuadPrec<MODE>::R R;
  typedef typename QuadPrec<MODE>::Acc Acc;
  constexpr int QNT = QuadShape<MODE>::NT, QFPT = QuadShape<MODE>::FPT, QCPT = QuadShape<MODE>::CPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* P = reinterpret_cast<R*>(smem_raw);  // [6][QBLK] hydro primitives
  R* RR = P + 6 * QBLK;                    // [QBLK] 1/rho
  R* FF = RR + QBLK;                       // [MAXF][QFACES] face fluxes of one direction
  R* XS = FF + MAXF * QFACES;              // mixed: [MAXF - 6][QBLK] species X_k
  __shared__ double red[QNT / 32];
  const int tid = threadIdx.x;
  const float gamf = (float)gamma_d, gm1f = (float)(gamma_d - 1.0);
  const R gamma = R(gamma_d), inv_gm1 = R(1.0 / (gamma_d - 1.0));
  const bool g53 = gamma_d == 5.0 / 3.0;

  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const Tile tile = fetch(t);
    const int F = tile.F, N = tile.N, G = tile.G, gh = (G - N) >> 1, nsp = F - 6;
    const int ex = min(TE, N - tile.ox), ey = min(TE, N - tile.oy), ez = min(TE, N - tile.oz);
    const long long plane = DOMAIN ? (long long)N * N * N : (long long)G * G * G;  // field stride
    // offset (within one field) of tile cell (x, y, z); in a domain the cell is
    // located by its periodic global coordinates
    DomainPos dp;
    if constexpr (DOMAIN) dp.init(tile.sub, tile.pad[0], N, F);
    auto off_of = [&](int x, int y, int z) {
      if constexpr (DOMAIN) {
        return dp.off(tile.ox + x, tile.oy + y, tile.oz + z);
      } else {
        return ((tile.oz + z + gh) * G + (tile.oy + y + gh)) * G + (tile.ox + x + gh);
      }
    };

    // ---- A0/A1: hydro primitives of the read region
    bool bad = false;
    for (int s = tid; s < QBLK; s += QNT) {
      const int x = s % LL - 3, y = (s / LL) % LL - 3, z = s / (LL * LL) - 3;
      const int far = (x == -3 || x == ex + 2) + (y == -3 || y == ey + 2) + (z == -3 || z == ez + 2);
      if (x > ex + 2 || y > ey + 2 || z > ez + 2 || far > 1) continue;
      const double* src = tile.U + off_of(x, y, z);
      double u[6];
#pragma unroll
      for (int f = 0; f < 6; f++) u[f] = __ldg(src + f * plane);
      if constexpr (MODE == 0) {
        double w[6], r;
        bad |= prim64(u, gamma_d, g53, w, r);
#pragma unroll
        for (int f = 0; f < 6; f++) P[f * QBLK + s] = w[f];
        RR[s] = r;
        for (int k = 0; k < nsp; k++) bad |= !dfinite(__ldg(src + (6 + k) * plane));
      } else {
        float w[6], r;
        bad |= prim_mixed(u, gamma_d, gamf, gm1f, g53, w, r);
#pragma unroll
        for (int f = 0; f < 6; f++) P[f * QBLK + s] = w[f];
        RR[s] = r;
        // species X_k = rho_k / rho in binary32 (rho_k converted, times the
        // binary32 1/rho), once per cell and tile: positive densities on the
        // integer pipe, the cell again with the conversion instruction if any
        // value is outside that path's range
        double us[MAXF - 6];
        float xs[MAXF - 6];
        unsigned oor = 0;
#pragma unroll
        for (int k = 0; k < MAXF - 6; k++)
          if (k < nsp) {
            us[k] = __ldg(src + (6 + k) * plane);
            xs[k] = d2f_fast_pos(us[k], oor);
          }
        if (oor >= D2F_OOR) {
#pragma unroll
          for (int k = 0; k < MAXF - 6; k++)
            if (k < nsp) xs[k] = d2f_slow(us[k]);
        }
#pragma unroll
        for (int k = 0; k < MAXF - 6; k++)
          if (k < nsp) {
            bad |= !dfinite(us[k]);
            XS[k * QBLK + s] = xs[k] * r;
          }
      }
    }
    bad = __syncthreads_or(bad);
    if (bad && tid == 0 && write_status) {
      atomicOr(&status->flags, 1u);
      atomicMin(&status->first_bad, (unsigned long long)tile.sub);
    }

    R amax = R(0);
    Acc acc[QCPT][MAXF];
    const int ogl = off_of(0, 0, 0);  // stored-block offset of tile cell (0, 0, 0)
    for (int d = 0; d < 3; d++) {
      const int e_d = d == 0 ? ex : (d == 1 ? ey : ez);
      const int e_a = d == 0 ? ey : ex, e_b = d == 2 ? ey : ez;
      // index strides along d and the two tangential axes (a: x or y, b: y or z),
      // in the shared-memory block (LL^axis) and in the stored block (G^axis)
      const int Sd = d == 0 ? 1 : (d == 1 ? LL : LL * LL);
      const int Sa = d == 0 ? LL : 1, Sb = d == 2 ? LL : LL * LL;
      const int Gd = d == 0 ? 1 : (d == 1 ? G : G * G);
      const int Ga = d == 0 ? G : 1, Gb = d == 2 ? G : G * G;
      if constexpr (MODE == 0) {
        // ---- A2/A3: the faces of this direction, 9 points each.  Thread t
        // walks three consecutive faces i0..i0+2 of line l = t/3.  The points
        // are taken in pairs (o, -o): one reconstruction of cell c along
        // e_d + o gives the left state at +o of face (c, c+1) (upper end) and
        // the right state at -o of face (c-1, c) (lower end), one along e_d - o
        // the other two, so every reconstruction serves two points; the centre
        // point (o = 0) is one line along e_d.  The weighted point fluxes are
        // summed in FF (the thread owns its faces' entries).
        const int l = tid / 3, i0 = 3 * (tid - 3 * l);
        const int ca = l % TE, cb = l / TE;
        const bool lvalid = ca < e_a && cb < e_b;
        const int c_last = min(i0 + 2, e_d);  // the high cell of the last valid face
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
          for (int f = 0; f < MAXF; f++)
            if (f < F) FF[f * QFACES + l * NFC + i0 + k] = R(0);
        // shared-memory index and stored-block offset of the line's cell 0
        const int is0 = qidx(0, 0, 0) + ca * Sa + cb * Sb;
        const int gs0 = ogl + ca * Ga + cb * Gb;
        // the 5 values of field f along e_d + s (o1 e_a + o2 e_b) through cell c
        auto stencil = [&](int f, int c, int o1, int o2, int s, R* q) {
          const int sm = Sd + s * (o1 * Sa + o2 * Sb), ic = is0 + c * Sd;
          if (f < 6) {
#pragma unroll
            for (int m = 0; m < 5; m++) q[m] = P[f * QBLK + ic + (m - 2) * sm];
            return;
          }
          const double* base = tile.U + f * plane;
#pragma unroll
          for (int m = 0; m < 5; m++) {
            int og;
            if constexpr (DOMAIN) {
              const int t = c + (m - 2), u = ca + (m - 2) * s * o1, v = cb + (m - 2) * s * o2;
              const int x = d == 0 ? t : u, y = d == 1 ? t : (d == 0 ? u : v), z = d == 2 ? t : v;
              og = off_of(x, y, z);
            } else {
              og = gs0 + c * Gd + (m - 2) * (Gd + s * (o1 * Ga + o2 * Gb));
            }
            q[m] = __ldg(base + og) * RR[ic + (m - 2) * sm];
          }
        };
        // lower and upper PPM values of every field of cell c along e_d + s o
        auto ends = [&](int c, int o1, int o2, int s, R* lo, R* hi) {
#pragma unroll
          for (int f = 0; f < MAXF; f++) {
            if (f >= F) break;
            R q[5];
            stencil(f, c, o1, o2, s, q);
            ppm5_64(q, lo[f], hi[f]);
          }
        };
        // central-upwind flux at one point of face i, weighted into FF
        auto point = [&](int i, const R* wl, const R* wr, R cw) {
          R fh[6], g_l, g_r;
          const R a = kt_hydro64(wl, wr, d, gamma, inv_gm1, knp, fh, 1, g_l, g_r);
          R* ff = FF + l * NFC + i;
#pragma unroll
          for (int f = 0; f < 6; f++) ff[f * QFACES] = fma(cw, fh[f], ff[f * QFACES]);
#pragma unroll
          for (int f = 6; f < MAXF; f++)
            if (f - 6 < nsp) ff[f * QFACES] = fma(cw, fma(wl[f], g_l, wr[f] * g_r), ff[f * QFACES]);
          amax = dmaxp(amax, a);
        };
        // pairs (o, -o) with o = (-1,-1), (0,-1), (1,-1), (-1,0), then the centre
#pragma unroll 1
        for (int pp = 0; pp < (lvalid && i0 <= e_d ? 5 : 0); pp++) {
          const int o1 = pp < 4 ? pp % 3 - 1 : 0, o2 = pp < 4 ? pp / 3 - 1 : 0;
          const R cw = R((o1 == 0 ? 4 : 1) * (o2 == 0 ? 4 : 1));  // Simpson weight, same for -o
          R Lp[MAXF], Lm[MAXF];  // left states at +o and -o of face (c, c+1), from cell c
#pragma unroll 1
          for (int c = i0 - 1; c <= c_last; c++) {
            if (pp < 4) {
              // face (c-1, c): the right state at +o is the lower end along
              // e_d - o, at -o the lower end along e_d + o
              R lo_m[MAXF], hi_m[MAXF];
              ends(c, o1, o2, -1, lo_m, hi_m);
              if (c >= i0) point(c, Lp, lo_m, cw);
              R lo_p[MAXF], hi_p[MAXF];
              ends(c, o1, o2, 1, lo_p, hi_p);
              if (c >= i0) point(c, Lm, lo_p, cw);
#pragma unroll
              for (int f = 0; f < MAXF; f++) {
                Lp[f] = hi_p[f];
                Lm[f] = hi_m[f];
              }
            } else {
              R lo_p[MAXF], hi_p[MAXF];
              ends(c, 0, 0, 1, lo_p, hi_p);
              if (c >= i0) point(c, Lp, lo_p, cw);
#pragma unroll
              for (int f = 0; f < MAXF; f++) Lp[f] = hi_p[f];
            }
          }
        }
        // Simpson's 1/36 as a product with its rounded reciprocal (within an
        // ulp of the quotient; a binary64 division costs ~9 operations of
        // the pipe this kernel is bound by)
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
          for (int f = 0; f < MAXF; f++)
            if (f < F) FF[f * QFACES + l * NFC + i0 + k] *= 1.0 / 36.0;
      } else {
        // ---- A2/A3 (mixed form): the faces of this direction, 9 points each
#pragma unroll 1
        for (int k = 0; k < QFPT; k++) {
          const int face = tid + k * QNT, l = face / NFC, i = face - l * NFC;
          const int ca = l % TE, cb = l / TE;
          const bool fvalid = ca < e_a && cb < e_b && i <= e_d;
          // the low cell (i-1 along d) and the high cell (i)
          const int il = qidx(0, 0, 0) + (i - 1) * Sd + ca * Sa + cb * Sb, ir = il + Sd;
          R fsum[MAXF];
#pragma unroll
          for (int f = 0; f < MAXF; f++) fsum[f] = R(0);
          // faces outside a partial tile are skipped: their stencils may leave
          // the stored block
#pragma unroll 1
          for (int p = 0; p < (fvalid ? 9 : 0); p++) {
            const int o1 = p % 3 - 1, o2 = p / 3 - 1;
            // lines e_d + o1 e_a + o2 e_b through the low cell, e_d - o1 e_a - o2 e_b
            // through the high cell
            const int sl = Sd + o1 * Sa + o2 * Sb, sr = Sd - o1 * Sa - o2 * Sb;
            R wl[MAXF], wr[MAXF];
            // fields f, f + 1 of the 5-cell stencils of both sides, one
            // packed reconstruction per side; a: the field's array
            auto pair = [&](const R* a0, const R* a1, int f) {
              float2 ql[5], qr[5], lo, hi;
#pragma unroll
              for (int m = 0; m < 5; m++) {
                ql[m] = make_float2(a0[il + (m - 2) * sl], a1[il + (m - 2) * sl]);
                qr[m] = make_float2(a0[ir + (m - 2) * sr], a1[ir + (m - 2) * sr]);
              }
              ppm5_32x2(ql, lo, hi);
              wl[f] = hi.x;
              wl[f + 1] = hi.y;
              ppm5_32x2(qr, lo, hi);
              wr[f] = lo.x;
              wr[f + 1] = lo.y;
            };
#pragma unroll
            for (int f = 0; f < 6; f += 2) pair(P + f * QBLK, P + (f + 1) * QBLK, f);
            // species X_k on the stencil cells, formed once per tile; an odd
            // last species alone
#pragma unroll
            for (int f = 6; f < MAXF; f += 2) {
              if (f - 6 >= nsp) break;
              const R* xk = XS + (f - 6) * QBLK;
              if (f + 1 < MAXF && f - 6 + 1 < nsp) {  // (f + 1 < MAXF: known when unrolled)
                pair(xk, xk + QBLK, f);
              } else {
                R ql[5], qr[5], lo, hi;
#pragma unroll
                for (int m = 0; m < 5; m++) {
                  ql[m] = xk[il + (m - 2) * sl];
                  qr[m] = xk[ir + (m - 2) * sr];
                }
                ppm5_32(ql, lo, hi);
                wl[f] = hi;
                ppm5_32(qr, lo, hi);
                wr[f] = lo;
              }
            }
            // central-upwind flux at the point
            float fh[MAXF], g_l, g_r;
            float2 pl[3] = {make_float2(wl[0], wl[1]), make_float2(wl[2], wl[3]), make_float2(wl[4], wl[5])};
            float2 pr[3] = {make_float2(wr[0], wr[1]), make_float2(wr[2], wr[3]), make_float2(wr[4], wr[5])};
            float2 fo[3];
            const float a = kt_hydro32(pl, pr, d, gamma, inv_gm1, knp, fo, 1, g_l, g_r);
            fh[0] = fo[0].x, fh[1] = fo[0].y, fh[2] = fo[1].x, fh[3] = fo[1].y, fh[4] = fo[2].x, fh[5] = fo[2].y;
#pragma unroll
            for (int f = 6; f < MAXF; f++)
              if (f - 6 < nsp) fh[f] = fmaf(wl[f], g_l, wr[f] * g_r);
            const float cw = (float)((o1 == 0 ? 4 : 1) * (o2 == 0 ? 4 : 1));
#pragma unroll
            for (int f = 0; f < MAXF; f++)
              if (f < F) fsum[f] = fmaf(cw, fh[f], fsum[f]);
            amax = fmaxf(amax, a);
          }
#pragma unroll
          for (int f = 0; f < MAXF; f++)
            if (f < F) FF[f * QFACES + face] = fsum[f] / R(36);
        }
      }
      __syncthreads();
      if constexpr (CAP) fetch.capture(tile, 0).template faces<QNT>(FF, QFACES, NLN, 0, F, d, ex, ey, ez);
      // ---- A4: flux differences of the owned cells
#pragma unroll
      for (int k = 0; k < QCPT; k++) {
        const int m = tid + k * QNT;
        if (m < TE * TE * TE) {
          const int x = m % TE, y = (m / TE) % TE, z = m / (TE * TE);
          const int l = d == 0 ? z * TE + y : (d == 1 ? z * TE + x : y * TE + x);
          const int pos = d == 0 ? x : (d == 1 ? y : z);
          const R* fl = FF + l * NFC + pos;
#pragma unroll
          for (int f = 0; f < MAXF; f++)
            if (f < F) {
              const R hi = fl[f * QFACES + 1], lo = fl[f * QFACES];
              if constexpr (MODE == 0) {
                acc[k][f] = d == 0 ? hi - lo : acc[k][f] + (hi - lo);
              } else {
                float dh, dl;
                two_diff1(hi, lo, dh, dl);
                if (d == 0) {
                  acc[k][f].h = dh;
                  acc[k][f].l = dl;
                } else {
                  F2 s = two_sum(acc[k][f].h, dh);
                  acc[k][f].h = s.h;
                  acc[k][f].l = (acc[k][f].l + dl) + s.l;
                }
              }
            }
        }
      }
      __syncthreads();
    }

    // ---- store dU/dt = -(sum of differences)/dx
    const long long n3 = (long long)N * N * N;
    const double scale = -tile.inv_dx;
    const bool pow2 = (tile.flags & 2) != 0;
    const float sf = pow2 ? d2f_int(scale) : 0.0f;
#pragma unroll
    for (int k = 0; k < QCPT; k++) {
      const int m = tid + k * QNT;
      if (m < TE * TE * TE) {
        const int x = m % TE, y = (m / TE) % TE, z = m / (TE * TE);
        if (x < ex && y < ey && z < ez) {
          double* o = out + tile.out_off + ((long long)(tile.oz + z) * N + (tile.oy + y)) * N + (tile.ox + x);
#pragma unroll
          for (int f = 0; f < MAXF; f++)
            if (f < F) {
              double v;
              if constexpr (MODE == 0) v = acc[k][f] * scale;
              else v = pair_value(acc[k][f].h, acc[k][f].l, scale, sf, pow2);
              if constexpr (DOMAIN || CAP) {
                if (stage.on) {
                  long long e = (o - out) + f * n3;  // same index in U, U0 and out
                  v = fma(stage.alpha, __ldg(stage.U0 + e), stage.beta * fma(stage.step(), v, __ldg(stage.U + e)));
                }
              }
              o[f * n3] = v;
            }
        }
      }
    }

    // ---- A5: largest signal speed of the tile
    double am = (double)amax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) am = dmaxp(am, __shfl_xor_sync(0xffffffffu, am, o));
    if ((tid & 31) == 0) red[tid >> 5] = am;
    __syncthreads();
    if (tid == 0) {
      double mx = red[0];
      for (int w = 1; w < QNT / 32; w++) mx = dmaxp(mx, red[w]);
      if (tile.flags & 1)
        atomicMax(reinterpret_cast<unsigned long long*>(amax_out + tile.amax_off),
                  (unsigned long long)__double_as_longlong(mx));
      else
        amax_out[tile.amax_off] = mx;
    }
    __syncthreads();
  }
}

// Same arguments as rhs_tiles_kernel; lch and prefetch do not apply.  One
// CTA per SM (shared memory: binary64 204 KB, mixed 157 KB).
template <int MODE>
__global__ void __launch_bounds__(QuadShape<MODE>::NT, 1)
rhs_quad_kernel(const Tile* __restrict__ tiles, int n_tiles, int Fmax, int lch, double* __restrict__ out,
                double* __restrict__ amax_out, Status* __restrict__ status, double gamma_d,
                int write_status, int prefetch, int scheme) {
  (void)Fmax;
  (void)lch;
  (void)prefetch;
  tile_loop_quad<MODE>(TileList{tiles}, n_tiles, out, amax_out, status, gamma_d, write_status, scheme == 1);
}

// The 26-point variant of the domain form (rhs_domain_kernel's arguments).
template <int MODE>
__global__ void __launch_bounds__(QuadShape<MODE>::NT, 1)
rhs_domain_quad_kernel(DomainTiles dom, int n_tiles, int lch, double* __restrict__ out,
                       double* __restrict__ amax_out, Status* __restrict__ status, double gamma_d,
                       int write_status, int scheme, StageArgs stage) {
  (void)lch;
  tile_loop_quad<MODE, DomainTiles, true>(dom, n_tiles, out, amax_out, status, gamma_d, write_status,
                                          scheme == 1, stage);
}

// Forest leaves for the 26-point variant: leaf s = t / tpe^3 read from its
// ghosted block ghost + s F G^3 (G = N + 6, gathered across levels before
// the launch); outputs, amax and the flux registers as for ForestTiles.
struct ForestQuadTiles {
  const double* __restrict__ ghost;
  const int* __restrict__ links;
  double* __restrict__ reg;
  int nl, N, F, tpe;
  double inv_dx0;
  short flags;  // bit 1: dx0 a power of two
  __device__ __forceinline__ Tile operator()(int t) const {
    const int tps = tpe * tpe * tpe;
    const int s = t / tps, k = t - s * tps;
    const int G = N + 6;
    Tile tile;
    tile.U = ghost + (long long)s * F * G * G * G;
    tile.out_off = (long long)s * F * N * N * N;
    tile.amax_off = s;
    tile.inv_dx = inv_dx0 * (double)(1u << __ldg(links + 8 * s + 6));
    tile.sub = s;
    tile.N = N;
    tile.F = F;
    tile.G = G;
    tile.ox = (short)((k % tpe) * TE);
    tile.oy = (short)(((k / tpe) % tpe) * TE);
    tile.oz = (short)((k / (tpe * tpe)) * TE);
    tile.flags = (short)((tps > 1 ? 1 : 0) | (flags & 2));
    tile.pad[0] = 0;
    tile.pad[1] = 0;
    return tile;
  }
  __device__ __forceinline__ ForestCapture capture(const Tile& tile, int f0) const {
    return ForestCapture{reg, links + 8 * tile.sub, nl, N, F, tile.ox, tile.oy, tile.oz, f0};
  }
};

template <int MODE>
__global__ void __launch_bounds__(QuadShape<MODE>::NT, 1)
rhs_forest_quad_kernel(ForestQuadTiles ft, int n_tiles, int lch, double* __restrict__ out,
                       double* __restrict__ amax_out, Status* __restrict__ status, double gamma_d,
                       int write_status, int scheme, StageArgs stage) {
  (void)lch;
  tile_loop_quad<MODE, ForestQuadTiles, false, true>(ft, n_tiles, out, amax_out, status, gamma_d, write_status,
                                                     scheme == 1, stage);
}

}  // namespace hydro_dev
