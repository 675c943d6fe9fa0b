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
// Per tile, one CTA (the register-load kernels, tile_loop):
//   1. stage the tile's read region (interior rows with their x ghosts, plus
//      the y and z ghost slabs: 1664 cells) from HBM, converting to primitive
//      variables on the way into shared memory                    (steps A0-A1)
//   2. for each direction, in chunks of lines: PPM face states of every
//      (line, field) (step A2), then the central flux of every face with its
//      signal speed (step A3), written back in place
//   3. every thread owns fixed cells and accumulates the flux differences of
//      x, then y, then z in registers (step A4); the result is scaled by
//      -1/dx and stored.  The largest signal speed is reduced with warp
//      shuffles and one atomic per tile (step A5).
// The pipelined mixed kernel (tile_loop_pipe, further down) moves the read
// region by asynchronous copies one field group ahead and reconstructs the
// three directions together; the 26-point variant lives in hydro_quad.cuh.
//
// MODE 0 runs every step in binary64.  On this GPU the binary64 pipe issues
// about 2 operations per SM per clock (1/64 of binary32), so the binary64 form
// is bound by that pipe: comparisons, absolute values, minima, sign tests and
// scalings by powers of two run on the integer pipe on the bit patterns, and
// the flux is written in an algebraically reduced form (see kt_hydro64).
//
// MODE 1 (mixed) rounds the binary64 inputs to binary32 (to nearest even,
// mostly with integer operations), forms primitives in binary32 (the
// dual-energy decision and the internal energy near it are evaluated in
// binary64, as the binary64 form does), reconstructs and
// fluxes in binary32, and carries the flux differences and their sum as exact
// binary32 pairs (error-free transformations, Knuth's TwoSum), so that the
// binary64 result telescopes across faces like the binary64 form.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <type_traits>

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
  long long out_off;   // first output double of the sub-grid, relative to the launch's out pointer
  long long amax_off;  // signal-speed slot of the sub-grid, relative to the launch's amax pointer
  double inv_dx;       // 1/dx
  int sub;             // sub-grid index reported in the status word
  int N;               // sub-grid interior edge
  int F;               // fields
  int G;               // stored edge N + 2*ghost
  short ox, oy, oz;    // tile origin (cells)
  short flags;         // bit 0: the sub-grid has more than one tile; bit 1: dx is a power of 2
  int pad[2];          // domain tiles: pad[0] = sub-grids per domain edge
};
static_assert(sizeof(Tile) == 64, "tile descriptor is 64 bytes");

struct Status {
  unsigned int flags;            // bit 0: nonphysical input
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

// Addressing of line l along direction d in the read-region layout: three
// segments (3 low ghosts, TE interior cells, 3 high ghosts), each with a
// base slot and a constant stride.
struct LineAddr {
  int lo, in, hi, sg, si;
  __device__ __forceinline__ int at(int c) const {
    return c < 3 ? lo + c * sg : (c < 3 + TE ? in + (c - 3) * si : hi + (c - 3 - TE) * sg);
  }
};
__device__ __forceinline__ LineAddr line_addr(int d, int l) {
  int a = l % TE, b = l / TE;
  if (d == 0) {
    int base = (b * TE + a) * LL;
    return {base, base + 3, base + 3 + TE, 1, 1};
  }
  if (d == 1)
    return {XROWS + b * 6 * TE + a, b * TE * LL + a + 3, XROWS + b * 6 * TE + 3 * TE + a, TE, LL};
  return {XROWS + YSLAB + b * TE + a, b * LL + a + 3, XROWS + YSLAB + 3 * TE * TE + b * TE + a,
          TE * TE, TE * LL};
}

// --------------------------------------------------- periodic domains --
// Position of a domain tile's sub-grid in a periodic cube of nb^3 sub-grids
// of N^3 cells stored without ghosts ([s][f][N^3], s = bx + nb (by + nb bz)),
// computed once per tile.  off() locates a cell given by coordinates within
// the sub-grid that may lie outside [0, N): a read-region cell is at most 3
// cells outside its tile, so for N >= 3 it lies in the sub-grid or in a direct
// neighbour (one compare and step per axis, wrapping around the cube); for
// N < 3 the periodic global coordinates are reduced with divisions.
struct DomainPos {
  int bx, by, bz, nb, N, bsz;  // bsz: doubles per stored sub-grid (F N^3)
  __device__ __forceinline__ void init(int sub, int nb_, int N_, int F) {
    nb = nb_;
    N = N_;
    bsz = F * N * N * N;
    bx = sub % nb;
    by = (sub / nb) % nb;
    bz = sub / (nb * nb);
  }
  __device__ __forceinline__ void step(int& c, int& b) const {
    if (c < 0) {
      c += N;
      b = b == 0 ? nb - 1 : b - 1;
    } else if (c >= N) {
      c -= N;
      b = b == nb - 1 ? 0 : b + 1;
    }
  }
  __device__ __forceinline__ int off(int cx, int cy, int cz) const {
    int ax = bx, ay = by, az = bz;
    if (N >= 3) {
      step(cx, ax);
      step(cy, ay);
      step(cz, az);
    } else {
      const int L = nb * N;
      const int gx = (bx * N + cx + L) % L, gy = (by * N + cy + L) % L, gz = (bz * N + cz + L) % L;
      ax = gx / N, ay = gy / N, az = gz / N;
      cx = gx % N, cy = gy % N, cz = gz % N;
    }
    return ((az * nb + ay) * nb + ax) * bsz + (cz * N + cy) * N + cx;
  }
};

// ============================================= binary64 on the integer pipe ==
// Bit-pattern helpers.  They are exact for zero and for normal numbers of
// magnitude >= 2^-1021 (far below any value a hydro state produces); the
// tests feed values within that range.
__device__ __forceinline__ int hiw(double x) { return __double2hiint(x); }
__device__ __forceinline__ double dabs(double x) {
  return __hiloint2double(hiw(x) & 0x7fffffff, __double2loint(x));
}
__device__ __forceinline__ double dcopysign(double m, double s) {  // |m| with the sign of s
  return __hiloint2double((hiw(m) & 0x7fffffff) | (hiw(s) & 0x80000000), __double2loint(m));
}
// 2x, x non-zero: one integer add to the exponent field.  Written in PTX so
// that the compiler keeps it on the integer pipe (in plain C it may be
// recognised as x + x and issued to the binary64 pipe, the scarce one here).
__device__ __forceinline__ double dtwice(double x) {
  long long b = __double_as_longlong(x);
  asm("add.s64 %0, %0, 0x0010000000000000;" : "+l"(b));
  return __longlong_as_double(b);
}
__device__ __forceinline__ double dhalf(double x) {  // x/2 (zero stays zero)
  int h = hiw(x);
  return __hiloint2double((h & 0x7ff00000) ? h - 0x00100000 : h, __double2loint(x));
}
// a*b > 0, i.e. both non-zero with the same sign (tested on the signs)
__device__ __forceinline__ bool dsame(double a, double b) {
  int x = hiw(a), y = hiw(b);
  return ((x ^ y) >= 0) && (x & 0x7fffffff) && (y & 0x7fffffff);
}
// |a| > |b|, compared exactly on the bit patterns
__device__ __forceinline__ bool dabs_gt(double a, double b) {
  return (__double_as_longlong(a) & 0x7fffffffffffffffLL) > (__double_as_longlong(b) & 0x7fffffffffffffffLL);
}
// order-preserving integer key of a double (NaN excluded)
__device__ __forceinline__ long long dkey(double x) {
  long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool dgt(double a, double b) { return dkey(a) > dkey(b); }
__device__ __forceinline__ double dminp(double a, double b) {  // a, b >= 0
  return __double_as_longlong(a) < __double_as_longlong(b) ? a : b;
}
__device__ __forceinline__ double dmaxp(double a, double b) {  // a, b >= 0
  return __double_as_longlong(a) > __double_as_longlong(b) ? a : b;
}
__device__ __forceinline__ bool dfinite(double x) { return (hiw(x) & 0x7ff00000) != 0x7ff00000; }
__device__ __forceinline__ double dmax_s(double a, double b) { return dgt(a, b) ? a : b; }  // any signs

// Reciprocal and reciprocal square root: the hardware seed y refined by one
// third-order step, each from the series of its function in the seed's
// relative defect e (a seed accurate to ~2^-23 leaves a term below 2^-66, so
// the result is within about an ulp, as two Newton-Raphson steps would give,
// for one binary64 operation fewer):
//   1/x       = y / (1 - e)       with e = 1 - x y:    y (1 + e + e^2)
//   1/sqrt(z) = y (1 - e)^(-1/2)  with e = 1 - z y^2:  y (1 + e/2 + 3e^2/8)
__device__ __forceinline__ double rcp64(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}
__device__ __forceinline__ double rsqrt64(double z) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(z));
  const double e = fma(-(z * y), y, 1.0);
  return fma(y * e, fma(e, 0.375, 0.5), y);
}

// binary64 <-> binary32 on the integer pipe for positive normal values well
// inside the binary32 range: truncation to binary32 (a seed), and the exact
// widening.
__device__ __forceinline__ float d2f_trunc_pos(double d) {
  return __uint_as_float(__funnelshift_l((unsigned)__double2loint(d), (unsigned)__double2hiint(d), 3) +
                         (128u << 23));
}
__device__ __forceinline__ double f2d_pos(float f) {
  const unsigned a = __float_as_uint(f);
  return __hiloint2double((int)((a >> 3) + (896u << 20)), (int)(a << 29));
}

// tau^gamma.  For gamma = 5/3: tau^(5/3) = tau^2 z with z = tau^(-1/3), seeded
// in binary32 (log2/exp2, relative error ~2^-22) and refined by one
// third-order step without division: with e = 1 - tau z^3,
// z' = z (1 - e)^(-1/3) ~ z (1 + e/3 + 2 e^2/9) (the series' next term,
// 14 e^3/81, is below 2^-60); ~2 ulp in all.  Other gamma, or tau outside
// [1e-30, 1e30]: pow().
__device__ __forceinline__ double tau_pow64(double tau, double gamma, bool g53) {
  if (!g53 || !(tau > 1e-30 && tau < 1e30)) return pow(tau, gamma);
  double z = f2d_pos(exp2f((-1.0f / 3.0f) * __log2f(d2f_trunc_pos(tau))));
  const double z3 = z * z * z;
  const double e = fma(-tau, z3, 1.0);
  z = fma(z, e * fma(e, 2.0 / 9.0, 1.0 / 3.0), z);
  return tau * (tau * z);
}

// ---------------------------------------------------- step A1, binary64 --
// Conserved -> primitive (rho, v, p, phi = tau/rho; the species X_k =
// rho_k/rho are formed by the caller with the returned r = 1/rho).
// The dual-energy branch is decided on e_int = E - |s|^2/(2 rho) against
// eta*E.  Far from the threshold a fast estimate (reciprocal, fused
// operations) decides it from the binary exponents alone (integer pipe):
// with k = expo(e_int) - expo(E), both positive and normal,
// 2^(k-1) < e_int/E < 2^(k+1), so k <= -12 means e_int < 2^-11 E < eta E
// (switched) and k >= -4 means e_int > 2^-5 E > eta E (not switched).  In
// between, and for values that are not positive and normal, e_int and the
// branch are recomputed with correctly rounded operations in the reference
// order, so the branch is taken exactly as the reference definition takes it.
__device__ __forceinline__ bool prim64(const double* u, double gamma, bool g53, double* w,
                                       double& r) {
  double rho = u[0], E = u[4], tau = u[5];
  r = rcp64(rho);
  double ssq = fma(u[3], u[3], fma(u[2], u[2], u[1] * u[1]));
  double eint = fma(-dhalf(ssq), r, E);
  const int xe = hiw(eint) >> 20, xE = hiw(E) >> 20;  // biased exponents; negative values give < 0
  const bool normal = xe > 0 && xe < 0x7ff && xE > 0 && xE < 0x7ff;
  const int k = xe - xE;
  double e;
  if (normal && k <= -12) {
    e = tau_pow64(tau, gamma, g53);
  } else if (normal && k >= -4) {
    e = eint;
  } else {  // near the switch: the reference order
    double ss = __dadd_rn(__dadd_rn(__dmul_rn(u[1], u[1]), __dmul_rn(u[2], u[2])), __dmul_rn(u[3], u[3]));
    double ex = __dsub_rn(E, __ddiv_rn(__dmul_rn(0.5, ss), rho));
    e = ex < __dmul_rn(ETA, E) ? tau_pow64(tau, gamma, g53) : ex;
  }
  double p = (gamma - 1.0) * e;
  w[0] = rho;
  w[1] = u[1] * r;
  w[2] = u[2] * r;
  w[3] = u[3] * r;
  w[4] = p;
  w[5] = tau * r;
  bool bad = !dgt(rho, 0.0) || !dgt(p, 0.0) || !dfinite(p);
#pragma unroll
  for (int f = 0; f < 6; f++) bad |= !dfinite(u[f]);
  return bad;
}

// ---------------------------------------------------- step A2, binary64 --
// PPM along one line of LL cells (Colella & Woodward 1984): monotonised
// central slopes, 4th-order face values, parabola limiter.  Produces the
// states on both sides of the NFC faces i-1/2, i = 0..TE:
//   left[i] = q+ of cell i-1,  right[i] = q- of cell i   (shared memory).
// With up = q+ - q and dn = q - q- (same sign s, else the cell is an
// extremum and flattened), m = q - (q- + q+)/2 = (dn - up)/2 and D = up + dn,
// the parabola tests become comparisons of magnitudes:
//   D m >  D^2/6  <=>  s (dn - 2 up) > 0  <=>  |dn| > 2|up|  ->  q- = q - 2 up  (= 3q - 2q+)
//   D m < -D^2/6  <=>  s (2 dn - up) < 0  <=>  |up| > 2|dn|  ->  q+ = q + 2 dn  (= 3q - 2q-)
// evaluated exactly on the integer pipe; the two cases exclude each other,
// so one fused multiply-add gives whichever new face value is needed.  The
// limiter is continuous at both switching surfaces, so evaluating the tests
// with different rounding than the reference moves results by rounding
// errors only.
// One pass along the line keeping a short window of values live (as
// ppm_line32x2).  The faces enter only through their offsets from the cell
// values: with dq_c = q_c+1 - q_c,
//   up_c = q_c+1/2 - q_c = dq_c/2 - (delta_c+1 - delta_c)/6,
//   dn_c+1 = q_c+1 - q_c+1/2 = dq_c - up_c,
// and the limited states are q - dn' and q + up' (dn' = 2 up where |dn| > 2|up|,
// up' = 2 dn where |up| > 2|dn|, both 0 at an extremum).  At step c: the
// slope of cell c, up of cell c-1, the states of cell c-1, dn of cell c.
// w: the line in shared memory (la addresses it).
__device__ __forceinline__ void ppm_line64(const double* w, const LineAddr& la, double* left,
                                           double* right) {
  const double sixth = 1.0 / 6.0;
  auto slope = [](double dm, double dp) {
    double dbar = dhalf(dp + dm);
    double m = dminp(dabs(dbar), dtwice(dminp(dabs(dm), dabs(dp))));
    return dsame(dp, dm) ? dcopysign(m, dbar) : 0.0;
  };
  double q0 = w[la.at(0)], q1 = w[la.at(1)], q2 = w[la.at(2)];
  double dm = q2 - q1;                   // dq of cell 1
  double del_prev = slope(q1 - q0, dm);  // cell c = 1
  double dn = 0.0;                       // dn of cell c-1
  double qm = q1, qc = q2;               // q[c-1], q[c] for c = 2
#pragma unroll
  for (int c = 2; c <= LL - 2; c++) {
    double qp = w[la.at(c + 1)];
    double dp = qp - qc;
    double del = slope(dm, dp);                           // slope of cell c
    double up = fma(del_prev - del, sixth, dhalf(dm));    // up of cell c-1
    if (c >= 3) {  // states of cell c-1
      bool ext = !dsame(up, dn);
      bool A = dabs_gt(dn, dtwice(up));  // |dn| > 2|up|
      bool B = dabs_gt(up, dtwice(dn));  // |up| > 2|dn| (excludes A)
      double lo = qm - (A ? dtwice(up) : dn);
      double hi = qm + (B ? dtwice(dn) : up);
      lo = ext ? qm : lo;
      hi = ext ? qm : hi;
      int j = c - 4;  // cell index of c-1
      if (j >= 0) right[j] = lo;
      if (j + 1 <= TE) left[j + 1] = hi;
    }
    dn = dm - up;  // dn of cell c
    del_prev = del;
    dm = dp;
    qm = qc;
    qc = qp;
  }
}

// ---------------------------------------------------- step A3, binary64 --
// Central flux (Kurganov & Tadmor 2000) through a face normal to axis d,
//   Fhat = (F_l + F_r)/2 - a (U_r - U_l)/2,  a = max(|u_l| + c_l, |u_r| + c_r),
// evaluated as Fhat = [(F_l + a U_l) + (F_r - a U_r)]/2, which for every
// advected quantity q (U = rho q, F = rho q u) is
//   Fhat_q = (q_l g_l + q_r g_r)/2,  g_l = rho_l (u_l + a),  g_r = rho_r (u_r - a),
// plus the pressure terms for momentum and energy.  Mathematically identical
// to the definition; rounding differs by a few ulps of the flux magnitude.
// w: (rho, vx, vy, vz, p, phi) on each side.  Writes the six fluxes of the
// hydro group (rho, s, E, tau) to fout[f*fstride]; returns a and the two g
// factors the species use.
__device__ __forceinline__ double kt_hydro64(const double* wl, const double* wr, int d,
                                             double gamma, double inv_gm1, bool knp, double* fout,
                                             int fstride, double& gl, double& gr) {
  double rl = wl[0], rr = wr[0], pl = wl[4], pr = wr[4];
  double ul = d == 0 ? wl[1] : (d == 1 ? wl[2] : wl[3]);
  double ur = d == 0 ? wr[1] : (d == 1 ? wr[2] : wr[3]);
  double vl2 = fma(wl[3], wl[3], fma(wl[2], wl[2], wl[1] * wl[1]));
  double vr2 = fma(wr[3], wr[3], fma(wr[2], wr[2], wr[1] * wr[1]));
  double El = fma(dhalf(rl), vl2, pl * inv_gm1);
  double Er = fma(dhalf(rr), vr2, pr * inv_gm1);
  double gpl = gamma * pl, gpr = gamma * pr;
  double cl = gpl * rsqrt64(gpl * rl);
  double cr = gpr * rsqrt64(gpr * rr);
  double a = dmaxp(dabs(ul) + cl, dabs(ur) + cr);
  if (!knp) {
    double hl = ul + a, hr = ur - a;
    gl = rl * hl;
    gr = rr * hr;
    fout[0] = dhalf(gl + gr);
    double pp = pl + pr;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      double t = fma(wl[1 + c], gl, wr[1 + c] * gr);
      fout[(1 + c) * fstride] = dhalf(c == d ? t + pp : t);
    }
    fout[4 * fstride] = dhalf(fma(El, hl, fma(pl, ul, fma(Er, hr, pr * ur))));
    fout[5 * fstride] = dhalf(fma(wl[5], gl, wr[5] * gr));
    gl = dhalf(gl);  // the species use Fhat_q = q_l gl + q_r gr
    gr = dhalf(gr);
    return a;
  }
  // Kurganov-Noelle-Petrova: one-sided speeds ap >= 0 >= am,
  //   Fhat = (ap F_l - am F_r + ap am (U_r - U_l)) / (ap - am)
  // which for advected quantities is q_l g_l + q_r g_r with
  //   wl = ap/(ap - am), wr = -am/(ap - am), k_l = wl (u_l - am),
  //   k_r = wr (u_r - ap), g = rho k; pressure enters with weights wl, wr.
  double ap = dmaxp(dmax_s(ul + cl, ur + cr), 0.0);
  double am = -dmaxp(dmax_s(cl - ul, cr - ur), 0.0);
  double den = ap - am;
  double rd = rcp64(den);
  bool ok = dgt(den, 0.0);
  double wL = ok ? ap * rd : 0.5, wR = ok ? -am * rd : 0.5;
  double kl = wL * (ul - am), kr = wR * (ur - ap);
  gl = rl * kl;
  gr = rr * kr;
  fout[0] = gl + gr;
  double pw = fma(pl, wL, pr * wR);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    double t = fma(wl[1 + c], gl, wr[1 + c] * gr);
    fout[(1 + c) * fstride] = c == d ? t + pw : t;
  }
  fout[4 * fstride] = fma(El, kl, fma(Er, kr, fma(wL, pl * ul, wR * (pr * ur))));
  fout[5 * fstride] = fma(wl[5], gl, wr[5] * gr);
  return a;
}

// ====================================================== binary32 (mixed) ==
// binary64 -> binary32, rounded to nearest with ties to even: the IEEE
// conversion, bit for bit.  d2f_fast converts magnitudes in the binary32
// normal range below the top binade, [2^-126, 2^127), on the integer pipe
// (the conversion instruction runs on the slow binary64 pipe of this GPU):
// the funnel shift takes the low 9 bits of the binary64 exponent and the top
// 23 fraction bits; adding 128 to that 9-bit exponent field (mod 512)
// rebiases it to binary32 for every exponent of the range; the 29 dropped
// bits round the result (up when above one half, or exactly one half with an
// odd result; a carry out of the fraction steps the exponent), and zero.  For
// values outside that range its result is meaningless and `oor` (an unsigned
// maximum over the values of a cell) becomes >= D2F_OOR, so that the caller
// converts that cell again with the instruction (d2f_slow): results below
// the normal range, the top binade (which may round to infinity) and
// non-finite values.  d2f_fast_pos takes the same path for positive values
// only (zero and negative ones count as out of range).
constexpr unsigned D2F_OOR = 253u << 20;
__device__ __forceinline__ float d2f_fast(double d, unsigned& oor) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned ahi = hi & 0x7fffffffu;
  // zero (or a magnitude below 2^-1042): signed zero, exactly as the
  // conversion rounds it -- momenta of gas at rest are zero
  const bool z = ahi == 0u;
  oor = max(oor, z ? 0u : ahi - (897u << 20));
  unsigned t = __funnelshift_l(lo, ahi, 3);
  const bool up = ((lo & 0x1fffffffu) | (t & 1u)) > 0x10000000u;
  t += (128u << 23) + (up ? 1u : 0u);
  return __uint_as_float((z ? 0u : t) | (hi & 0x80000000u));
}
__device__ __forceinline__ float d2f_fast_pos(double d, unsigned& oor) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  oor = max(oor, hi - (897u << 20));
  unsigned t = __funnelshift_l(lo, hi, 3);
  const bool up = ((lo & 0x1fffffffu) | (t & 1u)) > 0x10000000u;
  return __uint_as_float(t + (128u << 23) + (up ? 1u : 0u));
}
// Not inlined, so that the compiler cannot evaluate it speculatively (it has
// no side effects) in the common case that does not need it.
static __device__ __noinline__ float d2f_slow(double d) { return __double2float_rn(d); }
// one value, any magnitude
__device__ __forceinline__ float d2f_int(double d) {
  unsigned oor = 0;
  const float f = d2f_fast(d, oor);
  return oor >= D2F_OOR ? d2f_slow(d) : f;
}
// binary32 -> binary64 (exact), on the integer pipe; zero and subnormal
// binary32 values give signed zero.
__device__ __forceinline__ double f2d_int(float f) {
  unsigned b = __float_as_uint(f);
  unsigned sg = b & 0x80000000u, a = b & 0x7fffffffu;
  bool small = a < 0x00800000u;
  unsigned hi = small ? sg : (sg | ((a >> 3) + (896u << 20)));
  unsigned lo = small ? 0u : (a << 29);
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float rcp32(float x) {  // seed + one Newton step
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return fmaf(fmaf(-x, y, 1.0f), y, y);
}

// tau^(5/3) in binary32 for tau in (1e-18, 1e18): tau * w with w^3 = tau^2
// (seed exp2(2/3 log2 tau), one Halley step).
__device__ __forceinline__ float tau53_32(float tau) {
  float w = exp2f((2.0f / 3.0f) * __log2f(tau));
  const float A = tau * tau;
  const float w3 = w * w * w;
  w = w * fmaf(2.0f, A, w3) * rcp32(fmaf(2.0f, w3, A));
  return tau * w;
}
__device__ __forceinline__ bool tau53_ok(float tau) { return tau > 1e-18f && tau < 1e18f; }
// tau^gamma in binary32: tau53_32 where it applies, else exp2(gamma log2 tau)
__device__ __forceinline__ float tau_pow32(float tau, float gamma, bool g53) {
  return (g53 && tau53_ok(tau)) ? tau53_32(tau) : exp2f(gamma * __log2f(tau));
}

// ------------------------------------------------------ step A1, mixed --
// The mixed form's primitives (declared reading): the conserved values are
// rounded to binary32 (d2f_int, the IEEE conversion); rho, v = s/rho and
// phi = tau/rho are formed in binary32 from them (reciprocal with one Newton
// step, then products: within ~1.5 ulp of the quotients); the internal
// energy and the dual-energy switch are those of the binary64 form, on the
// binary64 inputs, and p = (gamma - 1) e rounded to binary32.  Where the
// binary32 estimate e32 = E - |s|^2/(2 rho) settles the branch with room to
// spare -- e32 >= E/2 (not switched; e32 within ~4 ulp of e) or
// e32 <= eta E/2 (switched; tau^gamma in binary32, within ~3 ulp) -- the
// binary32 values are used; in between, e and the branch are evaluated in
// binary64 in the reference order of operations.
// u: the binary64 hydro inputs of one cell (fields 0-5); writes binary32
// primitives (rho, vx, vy, vz, p, phi) and r = 1/rho.
// The common path, without branches: every value in the fast conversion's
// range and the binary32 estimate of e settling the branch.  Returns true
// where that does not hold, and the cell takes prim_mixed_slow.
__device__ __forceinline__ bool prim_mixed_fast(const double* u, float gamf, float gm1f, bool g53, float* w,
                                                float& r) {
  unsigned oor = 0;
  const float rho = d2f_fast_pos(u[0], oor);
  const float s1 = d2f_fast(u[1], oor), s2 = d2f_fast(u[2], oor), s3 = d2f_fast(u[3], oor);
  const float E = d2f_fast_pos(u[4], oor), tau = d2f_fast_pos(u[5], oor);
  r = rcp32(rho);
  const float ssq = fmaf(s3, s3, fmaf(s2, s2, s1 * s1));
  const float eint = fmaf(-0.5f * ssq, r, E);
  const bool kin = eint >= 0.5f * E;                          // not switched
  // switched, with tau^(5/3) in its range (other gamma, or tau out of range,
  // take the careful path)
  const bool sw = eint <= (float)(0.5 * ETA) * E && g53 && tau53_ok(tau);
  const float ptau = gm1f * tau53_32(tau);
  w[0] = rho;
  w[1] = s1 * r;
  w[2] = s2 * r;
  w[3] = s3 * r;
  w[4] = kin ? gm1f * eint : ptau;
  w[5] = tau * r;
  return oor >= D2F_OOR || !(kin || sw);
}
// The careful path: values outside the fast conversion's range converted
// with the instruction, and e and the branch in binary64 inside the window.
__device__ __forceinline__ void prim_mixed_slow(const double* u, double gamma, float gamf, float gm1f, bool g53,
                                                float* w, float& r) {
  unsigned oor = 0;
  float rho = d2f_fast_pos(u[0], oor);
  float s1 = d2f_fast(u[1], oor), s2 = d2f_fast(u[2], oor), s3 = d2f_fast(u[3], oor);
  float E = d2f_fast_pos(u[4], oor), tau = d2f_fast_pos(u[5], oor);
  if (oor >= D2F_OOR) {
    rho = d2f_slow(u[0]);
    s1 = d2f_slow(u[1]);
    s2 = d2f_slow(u[2]);
    s3 = d2f_slow(u[3]);
    E = d2f_slow(u[4]);
    tau = d2f_slow(u[5]);
  }
  r = rcp32(rho);
  float ssq = fmaf(s3, s3, fmaf(s2, s2, s1 * s1));
  float eint = fmaf(-0.5f * ssq, r, E);
  float p;
  if (eint >= 0.5f * E) {
    p = gm1f * eint;
  } else if (eint <= (float)(0.5 * ETA) * E) {
    p = gm1f * tau_pow32(tau, gamf, g53);
  } else {
    double ss = __dadd_rn(__dadd_rn(__dmul_rn(u[1], u[1]), __dmul_rn(u[2], u[2])), __dmul_rn(u[3], u[3]));
    double ex = __dsub_rn(u[4], __ddiv_rn(__dmul_rn(0.5, ss), u[0]));
    double e = ex < __dmul_rn(ETA, u[4]) ? tau_pow64(u[5], gamma, g53) : ex;
    p = d2f_int(__dmul_rn(gamma - 1.0, e));
  }
  w[0] = rho;
  w[1] = s1 * r;
  w[2] = s2 * r;
  w[3] = s3 * r;
  w[4] = p;
  w[5] = tau * r;
}
// nonphysical: rho <= 0, p <= 0 or a non-finite value.  A non-finite input
// (or one beyond the binary32 range) leaves a non-finite primitive, so the
// binary32 primitives alone decide it, as the binary32 quotients do in the
// reference definition of the mixed form.
__device__ __forceinline__ bool prim_mixed_bad(const float* w) {
  bool bad = !(w[0] > 0.0f) || !(w[4] > 0.0f);
#pragma unroll
  for (int f = 0; f < 6; f++) bad |= !isfinite(w[f]);
  return bad;
}
__device__ __forceinline__ bool prim_mixed(const double* u, double gamma, float gamf, float gm1f,
                                           bool g53, float* w, float& r) {
  if (prim_mixed_fast(u, gamf, gm1f, g53, w, r)) prim_mixed_slow(u, gamma, gamf, gm1f, g53, w, r);
  return prim_mixed_bad(w);
}

// -------------------------------------------- packed binary32 arithmetic --
// Two independent fields are processed per thread with the paired binary32
// instructions of sm_100+ (one instruction, two lanes of arithmetic).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// ------------------------------------------------------ step A2, mixed --
// ppm_line64's steps in binary32 on a pair of fields, in half-slope form:
// with dm = q - q_-1 and dp = q_+1 - q, half the monotonised central slope is
//   h = sign(dm + dp) min(|dm + dp|/4, |dm|, |dp|)  if dm, dp have one sign,
//   h = 0 otherwise,
// and the face between cells c-1 and c is (q_c-1 + q_c)/2 - (h_c - h_c-1)/3.
// The same-sign tests run on products (a product of two differences that
// underflows reads as "not the same sign", which changes results by less
// than those differences).  The parabola limiter in clamp form: with
// up = q+ - q and dn = q - q- of one sign, q+ = q + 2dn where |up| > 2|dn|
// and q- = q - 2up where |dn| > 2|up| (CW84 eq. 1.10); a cell with
// up dn <= 0 is flattened.
// min(|a|, |b|) with the sign of a (min.xorsign.abs with |b|)
__device__ __forceinline__ float min_signed(float a, float b) {
  float r;
  asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(fabsf(b)));
  return r;
}
__device__ __forceinline__ float hslope1(float dm, float dp, float s4, float pr) {
  float m = fminf(fminf(fabsf(s4), fabsf(dm)), fabsf(dp));
  return pr > 0.0f ? copysignf(m, s4) : 0.0f;
}
__device__ __forceinline__ float2 hslope32x2(float2 dm, float2 dp) {
  float2 s4 = mul2(add2(dm, dp), f2(0.25f));
  float2 pr = mul2(dm, dp);
  return make_float2(hslope1(dm.x, dp.x, s4.x, pr.x), hslope1(dm.y, dp.y, s4.y, pr.y));
}
__device__ __forceinline__ void limit1(float q, float lo, float hi, float up, float dn, float e, float uu,
                                       float du, float lc, float hc, float& L, float& H) {
  const bool ext = !(e > 0.0f);
  L = ext ? q : (fabsf(dn) > fabsf(uu) ? lc : lo);
  H = ext ? q : (fabsf(up) > fabsf(du) ? hc : hi);
}
// One pass along the line keeping a short window of values live, in the
// offset form of ppm_line64 (up = face - q from the half slopes, dn of the next
// cell = dq - up): at step c the half slope of cell c, up of cell c-1, the
// states of cell c-1 and dn of cell c.  w: the line in shared memory.
__device__ __forceinline__ void ppm_line32x2(const float2* w, const LineAddr& la, float2* left,
                                             float2* right) {
  float2 q0 = w[la.at(0)], q1 = w[la.at(1)], q2 = w[la.at(2)];
  float2 dm = sub2(q2, q1);                      // dq of cell 1
  float2 h_prev = hslope32x2(sub2(q1, q0), dm);  // cell c = 1
  float2 dn = f2(0.0f);                          // dn of cell c-1
  float2 qm = q1, qc = q2;                       // q[c-1], q[c] for c = 2
#pragma unroll
  for (int c = 2; c <= LL - 2; c++) {
    float2 qp = w[la.at(c + 1)];
    float2 dp = sub2(qp, qc);
    float2 h = hslope32x2(dm, dp);  // half slope of cell c
    // up of cell c-1: dq/2 - (h_c - h_c-1)/3
    float2 up = fma2(sub2(h_prev, h), f2(1.0f / 3.0f), mul2(dm, f2(0.5f)));
    if (c >= 3) {  // states of cell c-1
      float2 e = mul2(up, dn);
      float2 uu = add2(up, up), du = add2(dn, dn);
      // the offsets after clamping: with up, dn of one sign, the smaller of
      // |dn| and 2|up| with the sign of dn, the smaller of |up| and 2|dn| with
      // the sign of up (one instruction each)
      float2 a, b;
      a.x = min_signed(dn.x, uu.x);
      a.y = min_signed(dn.y, uu.y);
      b.x = min_signed(up.x, du.x);
      b.y = min_signed(up.y, du.y);
      float2 L = sub2(qm, a), H = add2(qm, b);
      L.x = e.x > 0.0f ? L.x : qm.x;
      L.y = e.y > 0.0f ? L.y : qm.y;
      H.x = e.x > 0.0f ? H.x : qm.x;
      H.y = e.y > 0.0f ? H.y : qm.y;
      int j = c - 4;  // cell index of c-1
      if (j >= 0) right[j] = L;
      if (j + 1 <= TE) left[j + 1] = H;
    }
    dn = sub2(dm, up);  // dn of cell c
    h_prev = h;
    dm = dp;
    qm = qc;
    qc = qp;
  }
}

// ------------------------------------------------------ step A3, mixed --
// kt_hydro64's flux in binary32.  w: three pairs (rho, vx), (vy, vz), (p, phi).
__device__ __forceinline__ float kt_hydro32(const float2* wl, const float2* wr, int d, float gamma,
                                            float inv_gm1, bool knp, float2* fout, int fstride,
                                            float& gl, float& gr) {
  float rl = wl[0].x, rr = wr[0].x, pl = wl[2].x, pr = wr[2].x;
  float vl[3] = {wl[0].y, wl[1].x, wl[1].y}, vr[3] = {wr[0].y, wr[1].x, wr[1].y};
  float ul = d == 0 ? vl[0] : (d == 1 ? vl[1] : vl[2]);
  float ur = d == 0 ? vr[0] : (d == 1 ? vr[1] : vr[2]);
  float vl2 = fmaf(vl[2], vl[2], fmaf(vl[1], vl[1], vl[0] * vl[0]));
  float vr2 = fmaf(vr[2], vr[2], fmaf(vr[1], vr[1], vr[0] * vr[0]));
  float El = fmaf(0.5f * rl, vl2, pl * inv_gm1);
  float Er = fmaf(0.5f * rr, vr2, pr * inv_gm1);
  float gpl = gamma * pl, gpr = gamma * pr;
  float cl = gpl * rsqrtf(gpl * rl);
  float cr = gpr * rsqrtf(gpr * rr);
  float a = fmaxf(fabsf(ul) + cl, fabsf(ur) + cr);
  // weights of the left and right states (kt_hydro64): KT wl = wr = 1/2
  float wL = 0.5f, wR = 0.5f, kl = 0.5f * (ul + a), kr = 0.5f * (ur - a);
  if (knp) {
    float ap = fmaxf(fmaxf(ul + cl, ur + cr), 0.0f);
    float am = fminf(fminf(ul - cl, ur - cr), 0.0f);
    float den = ap - am;
    if (den > 0.0f) {
      float rd = rcp32(den);
      wL = ap * rd;
      wR = -am * rd;
    }
    kl = wL * (ul - am);
    kr = wR * (ur - ap);
  }
  gl = rl * kl;
  gr = rr * kr;
  float pw = fmaf(pl, wL, pr * wR);
  float m[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    float t = fmaf(vl[c], gl, vr[c] * gr);
    m[c] = c == d ? t + pw : t;
  }
  fout[0] = make_float2(gl + gr, m[0]);
  fout[fstride] = make_float2(m[1], m[2]);
  fout[2 * fstride] = make_float2(fmaf(El, kl, fmaf(Er, kr, fmaf(wL, pl * ul, wR * (pr * ur)))),
                                  fmaf(wl[2].y, gl, wr[2].y * gr));
  return a;
}

// --------------------------------------------- exact binary32 pair sums --
struct F2 {
  float h, l;
};
__device__ __forceinline__ F2 two_sum(float a, float b) {  // a + b = s + e exactly (Knuth)
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// Packed: two independent running sums (H, L) += (hi - lo), one per lane.
// The difference is split exactly with a two-sum, its high part is added to
// H with an exact two-sum, the low parts are summed in binary32 (their
// rounding is ~2^-24 of a quantity already ~2^-24 smaller than H).
struct P2 {
  float2 h, l;
};
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  float2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// a - b = s + e exactly (Knuth's two-sum with the subtraction folded in)
__device__ __forceinline__ void two_diff2(float2 a, float2 b, float2& s, float2& e) {
  s = sub2(a, b);
  float2 bb = sub2(s, a);  // ~ -b
  e = sub2(sub2(a, sub2(s, bb)), add2(b, bb));
}
__device__ __forceinline__ void acc_pair2(P2& acc, float2 hi, float2 lo, bool first) {
  float2 dh, dl;
  two_diff2(hi, lo, dh, dl);
  if (first) {
    acc.h = dh;
    acc.l = dl;
  } else {
    float2 sh, sl;
    two_sum2(acc.h, dh, sh, sl);
    acc.h = sh;
    acc.l = add2(add2(acc.l, dl), sl);
  }
}

// ------------------------------------------------ L2 prefetch (TMA) --
// Issue bulk L2 prefetches (cp.async.bulk.prefetch, executed by the TMA unit)
// for the read region of a tile: every row segment of the region, widened to
// 16-byte boundaries.  Used for the CTA's next tile while it computes the
// current one, so that its loads hit L2.  Requires a 16-byte aligned block
// and an even edge G (row pitch a multiple of 16 bytes); otherwise nothing is
// issued.  Every address lies inside the sub-grid's stored block.
__device__ __forceinline__ void prefetch_tile_l2(const Tile& tile, int tid, int nt, int mode) {
  const int G = tile.G, N = tile.N, F = tile.F;
  const int gh = (G - N) >> 1;
  if ((G & 1) || (reinterpret_cast<uintptr_t>(tile.U) & 15)) return;
  const int ex = min(TE, N - tile.ox), ey = min(TE, N - tile.oy), ez = min(TE, N - tile.oz);
  const long long plane = (long long)G * G * G;
  if (mode == 1) {  // one prefetch per row segment
    const int ny = ey + 6, nz = ez + 6;
    const int rows = ny * nz;  // candidate rows (y, z) of the tile's bounding box
    for (int r = tid; r < rows * F; r += nt) {
      int f = r / rows, rr = r - f * rows;
      int y = rr % ny - 3, z = rr / ny - 3;
      bool yin = y >= 0 && y < ey, zin = z >= 0 && z < ez;
      if (!yin && !zin) continue;  // edge/corner rows hold no read cell
      int x0 = (yin && zin) ? -3 : 0, x1 = (yin && zin) ? ex + 3 : ex;
      int c0 = (tile.ox + x0 + gh) & ~1, c1 = (tile.ox + x1 + gh + 1) & ~1;  // 16-byte bounds
      const double* row = tile.U + f * plane + ((long long)(tile.oz + z + gh) * G + (tile.oy + y + gh)) * G;
      unsigned bytes = (unsigned)(c1 - c0) * 8u;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(row + c0), "r"(bytes) : "memory");
    }
  } else {  // one prefetch per z plane: the byte range from its first to its last read cell
    const int nz = ez + 6;
    for (int r = tid; r < nz * F; r += nt) {
      int f = r / nz, z = r - f * nz - 3;
      bool zin = z >= 0 && z < ez;
      int y0 = zin ? -3 : 0, y1 = zin ? ey + 2 : ey - 1;  // first and last row
      const int xa = 0, xb = ex;  // first cell of the first row, end of the last row
      const double* pl = tile.U + f * plane + (long long)(tile.oz + z + gh) * G * G;
      long long a = (long long)(tile.oy + y0 + gh) * G + (tile.ox + xa + gh);
      long long b = (long long)(tile.oy + y1 + gh) * G + (tile.ox + xb + gh);  // one past the last
      a &= ~1LL;
      b = (b + 1) & ~1LL;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(pl + a), "r"((unsigned)(b - a) * 8u)
                   : "memory");
    }
  }
}

// ------------------------------------------------------------- layout --
template <int MODE> struct Prec;
template <> struct Prec<0> { typedef double R; typedef double V; typedef double Acc; static constexpr int PACK = 1; };
template <> struct Prec<1> { typedef float R; typedef float2 V; typedef P2 Acc; static constexpr int PACK = 2; };

// The per-face factors (g_l, g_r) of the species fluxes as one vector access
// (conflict-free in shared memory, unlike two strided scalar ones).
__device__ __forceinline__ void store_pair(float* g, float a, float b) {
  *reinterpret_cast<float2*>(g) = make_float2(a, b);
}
__device__ __forceinline__ void store_pair(double* g, double a, double b) {
  *reinterpret_cast<double2*>(g) = make_double2(a, b);
}
__device__ __forceinline__ void load_pair(const float* g, float& a, float& b) {
  const float2 v = *reinterpret_cast<const float2*>(g);
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void load_pair(const double* g, double& a, double& b) {
  const double2 v = *reinterpret_cast<const double2*>(g);
  a = v.x;
  b = v.y;
}

// Source of the tile descriptors: a prepared work list in global memory.
struct TileList {
  const Tile* __restrict__ tiles;
  __device__ __forceinline__ Tile operator()(int t) const { return tiles[t]; }
};

constexpr int NGRP = 6;  // fields per group: hydro (rho, vx, vy, vz, p, phi) or species (<= 5)

// Shared memory of one CTA.  V = R (binary64) or a pair of binary32 values
// (mixed form: fields 2k and 2k+1 of a group share one 8-byte element):
//   W  [NGRP/PACK][STAR] V   primitives of the read region: the hydro group,
//                            then (after the hydro pass) the species
//   RR [STAR] R              1/rho of every read cell
//   GG [3][NLN][NFC][2] R    per face the factors g_l, g_r of the species fluxes
//   QS [2][NGRP/PACK][lch][NFC] V   face states of a chunk of lines, then fluxes
template <int MODE>
__host__ __device__ constexpr size_t smem_layout_bytes(int lch) {
  return (MODE == 0 ? 8 : 4) *
         ((size_t)NGRP * STAR + STAR + 3 * NLN * NFC * 2 + 2 * (size_t)NGRP * lch * NFC);
}

// ------------------------------------------------------------ forests --
// Leaves of an octree forest of several refinement levels, N^3 cells each,
// stored without ghosts ([s][f][N^3]).  links[8 s + k], k < 6 (face k = 2 d +
// side, side 1 the high face): the face neighbour, a leaf of the same level
// (< nl) or nl + j for auxiliary block j, which holds that face's ghost slab
// transferred from a coarser or finer level (in the layout of a same-level
// neighbour, [j][f][N^3]); links[8 s + 6]: the leaf's level.
//
// ForestLoc locates a read-region cell given by leaf-local coordinates, at
// most one of which lies outside [0, N).
struct ForestLoc {
  const double* U;
  const double* aux;
  const int* row;  // links of the leaf
  int s, nl, N;
  long long bsz;   // doubles per stored block (F N^3)
  __device__ __forceinline__ const double* ptr(int cx, int cy, int cz) const {
    int face = -1;
    if (cx < 0) {
      face = 0;
      cx += N;
    } else if (cx >= N) {
      face = 1;
      cx -= N;
    } else if (cy < 0) {
      face = 2;
      cy += N;
    } else if (cy >= N) {
      face = 3;
      cy -= N;
    } else if (cz < 0) {
      face = 4;
      cz += N;
    } else if (cz >= N) {
      face = 5;
      cz -= N;
    }
    const int blk = face < 0 ? s : __ldg(row + face);
    const double* base = blk < nl ? U + blk * bsz : aux + (blk - nl) * bsz;
    return base + (cz * N + cy) * N + cx;
  }
};

// Flux registers: for auxiliary block j (a leaf face towards another level),
// reg[(j F + f) N^2 + b N + a] receives the flux of field f through the
// face's cell column (a, b); the tangential axes of a face normal to d are
// (y, z), (x, z), (x, y) for d = x, y, z.
struct ForestCapture {
  double* reg;
  const int* row;
  int nl, N, F, ox, oy, oz, f0;
  // Record the fluxes of the lines [l0, l0 + lch) of direction d, just
  // computed in QS (slot j = field f0 + j, or for binary32 pairs the fields
  // f0 + 2j, f0 + 2j + 1), through the faces that lie on the leaf's boundary
  // towards another level.
  template <int NT, class V>
  __device__ __forceinline__ void faces(const V* QS, int fs, int lch, int l0, int ng, int d, int ex, int ey,
                                        int ez) const {
    const int e_d = d == 0 ? ex : (d == 1 ? ey : ez);
    const int e_a = d == 0 ? ey : ex, e_b = d == 2 ? ey : ez;
    const int o_d = d == 0 ? ox : (d == 1 ? oy : oz);
    const int o_a = d == 0 ? oy : ox, o_b = d == 2 ? oy : oz;
    const int lo = o_d == 0 ? __ldg(row + 2 * d) : -1;
    const int hi = o_d + e_d == N ? __ldg(row + 2 * d + 1) : -1;
    if (lo < nl && hi < nl) return;
    const long long nn = (long long)N * N;
    for (int task = threadIdx.x; task < 2 * lch * ng; task += NT) {
      const int ll = task % lch, r = task / lch, side = r & 1, j = r >> 1;
      const int blk = side ? hi : lo;
      const int l = l0 + ll, a = l % TE, b = l / TE;
      if (blk < nl || a >= e_a || b >= e_b) continue;
      const V v = QS[j * fs + ll * NFC + (side ? e_d : 0)];
      double* dst = reg + (long long)(blk - nl) * F * nn + (long long)(o_b + b) * N + (o_a + a);
      if constexpr (std::is_same<V, float2>::value) {
        const int f = f0 + 2 * j;
        dst[f * nn] = (double)v.x;
        if (f + 1 < F) dst[(f + 1) * nn] = (double)v.y;
      } else {
        dst[(f0 + j) * nn] = (double)v;
      }
    }
  }
};

// Source of forest tiles: leaf s = t / tpe^3, cell width dx0 / 2^level.
struct ForestTiles {
  const double* __restrict__ U;
  const double* __restrict__ aux;
  const int* __restrict__ links;
  double* __restrict__ reg;
  int nl, N, F, tpe;
  double inv_dx0;
  short flags;  // bit 1: dx0 a power of two
  __device__ __forceinline__ Tile operator()(int t) const {
    const int tps = tpe * tpe * tpe;
    const int s = t / tps, k = t - s * tps;
    Tile tile;
    tile.U = U;
    tile.out_off = (long long)s * F * N * N * N;
    tile.amax_off = s;
    tile.inv_dx = inv_dx0 * (double)(1u << __ldg(links + 8 * s + 6));
    tile.sub = s;
    tile.N = N;
    tile.F = F;
    tile.G = N;
    tile.ox = (short)((k % tpe) * TE);
    tile.oy = (short)(((k / tpe) % tpe) * TE);
    tile.oz = (short)((k / (tpe * tpe)) * TE);
    tile.flags = (short)((tps > 1 ? 1 : 0) | (flags & 2));
    tile.pad[0] = 0;
    tile.pad[1] = 0;
    return tile;
  }
  __device__ __forceinline__ ForestLoc loc(const Tile& tile) const {
    return ForestLoc{U, aux, links + 8 * tile.sub, tile.sub, nl, N, (long long)F * N * N * N};
  }
  __device__ __forceinline__ ForestCapture capture(const Tile& tile, int f0) const {
    return ForestCapture{reg, links + 8 * tile.sub, nl, N, F, tile.ox, tile.oy, tile.oz, f0};
  }
};

struct NoCapture {
  template <int NT, class V>
  __device__ __forceinline__ void faces(const V*, int, int, int, int, int, int, int, int) const {}
};

// One pass of steps A2-A4 over a group of `ng` field slots (V elements) for
// all three directions.  HYD: the hydro group (Kurganov-Tadmor flux, records
// g_l, g_r and the signal speed); else the species (flux from g_l, g_r).
// acc[k][j] receives, for the thread's owned cells k, the sum of the flux
// differences x, then y, then z of slot j.  `cap` may record face fluxes.
template <int MODE, int NT, bool HYD, class Cap = NoCapture>
__device__ __forceinline__ void group_pass(
    const typename Prec<MODE>::V* W, typename Prec<MODE>::R* GG, typename Prec<MODE>::V* QS,
    int lch, int ng, int ex, int ey, int ez, typename Prec<MODE>::R gamma,
    typename Prec<MODE>::R inv_gm1, bool knp,
    typename Prec<MODE>::Acc (&acc)[(TE * TE * TE + NT - 1) / NT][NGRP / Prec<MODE>::PACK],
    typename Prec<MODE>::R& amax, const Cap& cap = Cap{}) {
  typedef typename Prec<MODE>::R R;
  typedef typename Prec<MODE>::V V;
  constexpr int CPT = (TE * TE * TE + NT - 1) / NT;
  constexpr int NS = NGRP / Prec<MODE>::PACK;  // V slots of a full group
  const int tid = threadIdx.x;
  const int fs = lch * NFC;  // slot stride of QS
  V* QR = QS + NS * fs;      // right states
  for (int d = 0; d < 3; d++) {
    const int e_d = d == 0 ? ex : (d == 1 ? ey : ez);
    const int e_a = d == 0 ? ey : ex;  // first tangential axis extent
    const int e_b = d == 2 ? ey : ez;  // second tangential axis extent
    R* gg = GG + d * NLN * NFC * 2;
    for (int l0 = 0; l0 < NLN; l0 += lch) {
      // ---- A2: PPM per (line, slot)
      for (int task = tid; task < lch * ng; task += NT) {
        int ll = task % lch, j = task / lch;
        LineAddr la = line_addr(d, l0 + ll);
        const V* w = W + j * STAR;
        if constexpr (MODE == 0) {
          ppm_line64(w, la, QS + j * fs + ll * NFC, QR + j * fs + ll * NFC);
        } else {
          ppm_line32x2(w, la, QS + j * fs + ll * NFC, QR + j * fs + ll * NFC);
        }
      }
      __syncthreads();
      // ---- A3: flux per face, written over the left states
      for (int task = tid; task < lch * NFC; task += NT) {
        int ll = task / NFC, i = task - ll * NFC;
        int l = l0 + ll;
        V* fo = QS + ll * NFC + i;
        const V* fr = QR + ll * NFC + i;
        R* g = gg + (l * NFC + i) * 2;
        if constexpr (HYD) {
          V wl[NS], wr[NS];
#pragma unroll
          for (int j = 0; j < NS; j++) {
            wl[j] = fo[j * fs];
            wr[j] = fr[j * fs];
          }
          R a, gl, gr;
          if constexpr (MODE == 0) a = kt_hydro64(wl, wr, d, gamma, inv_gm1, knp, fo, fs, gl, gr);
          else a = kt_hydro32(wl, wr, d, gamma, inv_gm1, knp, fo, fs, gl, gr);
          store_pair(g, gl, gr);  // one 8- or 16-byte store
          bool fvalid = (l % TE) < e_a && (l / TE) < e_b && i <= e_d;
          if constexpr (MODE == 0) {
            if (fvalid) amax = dmaxp(amax, a);
          } else {
            if (fvalid) amax = fmaxf(amax, a);
          }
        } else {
          R gl, gr;
          load_pair(g, gl, gr);
#pragma unroll
          for (int j = 0; j < NS; j++)
            if (j < ng) {
              if constexpr (MODE == 0) fo[j * fs] = fma(fo[j * fs], gl, fr[j * fs] * gr);
              else fo[j * fs] = fma2(fo[j * fs], f2(gl), mul2(fr[j * fs], f2(gr)));
            }
        }
      }
      __syncthreads();
      cap.template faces<NT>(QS, fs, lch, l0, ng, d, ex, ey, ez);
      // ---- A4: flux differences into the owned cells, x then y then z
#pragma unroll
      for (int k = 0; k < CPT; k++) {
        int m = tid + k * NT;
        if (m < TE * TE * TE) {
          int x = m % TE, y = (m / TE) % TE, z = m / (TE * TE);
          int l = d == 0 ? z * TE + y : (d == 1 ? z * TE + x : y * TE + x);
          int pos = d == 0 ? x : (d == 1 ? y : z);
          if (l >= l0 && l < l0 + lch) {
            const V* fl = QS + (l - l0) * NFC + pos;
#pragma unroll
            for (int j = 0; j < NS; j++)
              if (j < ng) {
                V hi = fl[j * fs + 1], lo = fl[j * fs];
                if constexpr (MODE == 0) {
                  acc[k][j] = d == 0 ? hi - lo : acc[k][j] + (hi - lo);
                } else {
                  acc_pair2(acc[k][j], hi, lo, d == 0);
                }
              }
          }
        }
      }
      __syncthreads();
    }
  }
}

// binary64 value of a mixed-form running sum (one lane), scaled by -1/dx
// (sf: the same scale in binary32, exact when dx is a power of two)
__device__ __forceinline__ double pair_value(float h, float l, double scale, float sf, bool pow2) {
  if (pow2) return f2d_int(h * sf) + f2d_int(l * sf);  // exact scaling in binary32
  return (f2d_int(h) + f2d_int(l)) * scale;
}

// A fused explicit stage: out = alpha U0 + beta (U + dt dU/dt), with U, U0
// and out in the domain layout (the packed output layout of the sub-grids).
struct StageArgs {
  const double* __restrict__ U;
  const double* __restrict__ U0;
  double alpha, beta, dt;
  int on;
  const double* __restrict__ dtp;  // if set, dt is read here (device memory)
  __device__ __forceinline__ double step() const { return dtp ? __ldg(dtp) : dt; }
};

// Store dU/dt = -(sum of differences)/dx of the fields f0 .. f0+nf-1 (or,
// with a stage, the updated state).
template <int MODE, int NT, bool STAGE = false>
__device__ __forceinline__ void store_group(
    double* __restrict__ out, const Tile& tile, int ex, int ey, int ez, int f0, int nf,
    const typename Prec<MODE>::Acc (&acc)[(TE * TE * TE + NT - 1) / NT][NGRP / Prec<MODE>::PACK],
    const StageArgs& stage = StageArgs{nullptr, nullptr, 0.0, 0.0, 0.0, 0}) {
  constexpr int CPT = (TE * TE * TE + NT - 1) / NT;
  const int tid = threadIdx.x, N = tile.N;
  const long long n3 = (long long)N * N * N;
  const double scale = -tile.inv_dx;
  const bool pow2 = (tile.flags & 2) != 0;
  const float sf = pow2 ? d2f_int(scale) : 0.0f;
#pragma unroll
  for (int k = 0; k < CPT; k++) {
    int m = tid + k * NT;
    if (m < TE * TE * TE) {
      int x = m % TE, y = (m / TE) % TE, z = m / (TE * TE);
      if (x < ex && y < ey && z < ez) {
        double* o = out + tile.out_off + f0 * n3 +
                    ((long long)(tile.oz + z) * N + (tile.oy + y)) * N + (tile.ox + x);
#pragma unroll
        for (int j = 0; j < NGRP; j++)
          if (j < nf) {
            double v;
            if constexpr (MODE == 0) {
              v = acc[k][j] * scale;
            } else {
              const P2& a = acc[k][j / 2];
              v = (j & 1) ? pair_value(a.h.y, a.l.y, scale, sf, pow2)
                          : pair_value(a.h.x, a.l.x, scale, sf, pow2);
            }
            if constexpr (STAGE) {
              if (stage.on) {
                long long e = (o - out) + j * n3;  // same index in U, U0 and out
                v = fma(stage.alpha, __ldg(stage.U0 + e), stage.beta * fma(stage.step(), v, __ldg(stage.U + e)));
              }
            }
            o[j * n3] = v;
          }
      }
    }
  }
}

// The persistent tile loop; `fetch(t)` returns tile t's descriptor; KC read-
// region slots of a thread are loaded per batch.  DOM says where a tile's
// read region lives:
//   0  its sub-grid's ghosted block;
//   1  a periodic cube of pad[0]^3 sub-grids stored without ghosts ([s][f][N^3],
//      s = bx + nb (by + nb bz)): the ghost slabs are read from the
//      neighbouring sub-grids' interiors;
//   2  a forest of leaves of several refinement levels stored without ghosts:
//      a ghost slab is read from the face neighbour of the same level or from
//      an auxiliary block holding the slab transferred from another level
//      (`fetch.loc`), and the fluxes through faces towards other levels are
//      recorded for the flux correction (`fetch.capture`).
// With DOM != 0, `stage` may turn the output into an explicit stage update.
template <int MODE, int NT, int KC, class Fetch, int DOM = 0>
__device__ __forceinline__ void tile_loop(const Fetch& fetch, int n_tiles, int lch,
                                          double* __restrict__ out, double* __restrict__ amax_out,
                                          Status* __restrict__ status, double gamma_d,
                                          int write_status, int prefetch, bool knp,
                                          const StageArgs& stage = StageArgs{nullptr, nullptr, 0.0, 0.0, 0.0, 0}) {
  typedef typename Prec<MODE>::R R;
  typedef typename Prec<MODE>::V V;
  typedef typename Prec<MODE>::Acc Acc;
  constexpr int PK = Prec<MODE>::PACK;
  constexpr int NS = NGRP / PK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* W = reinterpret_cast<V*>(smem_raw);
  R* RR = reinterpret_cast<R*>(W + NS * STAR);
  R* GG = RR + STAR;
  V* QS = reinterpret_cast<V*>(GG + 3 * NLN * NFC * 2);
  __shared__ double red[NT / 32];
  const int tid = threadIdx.x;
  const R gamma = R(gamma_d);
  const R inv_gm1 = R(1.0 / (gamma_d - 1.0));
  const float gm1f = (float)(gamma_d - 1.0), gamf = (float)gamma_d;
  const bool g53 = gamma_d == 5.0 / 3.0;
  constexpr int CPT = (TE * TE * TE + NT - 1) / NT;  // owned cells per thread
  constexpr int SPT = (STAR + NT - 1) / NT;          // read-region slots per thread

  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const Tile tile = fetch(t);
    const int F = tile.F, G = tile.G, N = tile.N, gh = (tile.G - tile.N) >> 1;
    const int ex = min(TE, N - tile.ox), ey = min(TE, N - tile.oy), ez = min(TE, N - tile.oz);
    const long long plane = DOM ? (long long)N * N * N : (long long)G * G * G;  // field stride
    DomainPos dp;
    if constexpr (DOM == 1) dp.init(tile.sub, tile.pad[0], N, F);
    ForestLoc fl;
    if constexpr (DOM == 2) fl = fetch.loc(tile);

    // offset of read-region slot s within a field of the stored block; -1 if
    // the slot is outside the (possibly partial) tile's read region: at most
    // one coordinate outside the tile, and that one at most 3 cells out.  In
    // a domain the cell is located by its periodic global coordinates.
    auto slot_offset = [&](int s) -> int {
      int x, y, z;
      cell_of(s < STAR ? s : 0, x, y, z);
      int outside = (x < 0 || x >= ex) + (y < 0 || y >= ey) + (z < 0 || z >= ez);
      bool valid = s < STAR && outside <= 1 && x < ex + 3 && y < ey + 3 && z < ez + 3;
      if (!valid) return -1;
      if constexpr (DOM == 1) {
        return dp.off(tile.ox + x, tile.oy + y, tile.oz + z);
      } else {
        return ((tile.oz + z + gh) * G + (tile.oy + y + gh)) * G + (tile.ox + x + gh);
      }
    };
    // forests: the address of slot s's cell in field 0, or null if not read
    auto slot_src = [&](int s) -> const double* {
      int x, y, z;
      cell_of(s < STAR ? s : 0, x, y, z);
      int outside = (x < 0 || x >= ex) + (y < 0 || y >= ey) + (z < 0 || z >= ez);
      bool valid = s < STAR && outside <= 1 && x < ex + 3 && y < ey + 3 && z < ez + 3;
      return valid ? fl.ptr(tile.ox + x, tile.oy + y, tile.oz + z) : nullptr;
    };

    // ---- A0/A1 (hydro group): rho, s, E, tau -> rho, v, p, phi.  In each
    // batch every load is issued before any result is used.
    bool bad = false;
#pragma unroll 1
    for (int k0 = 0; k0 < SPT; k0 += KC) {
      double u[KC][6];
      int off[KC];
      const double* src[KC];
#pragma unroll
      for (int kk = 0; kk < KC; kk++) {
        if constexpr (DOM == 2) {
          src[kk] = slot_src(tid + (k0 + kk) * NT);
          off[kk] = src[kk] ? 0 : -1;
        } else {
          off[kk] = slot_offset(tid + (k0 + kk) * NT);
        }
#pragma unroll
        for (int f = 0; f < 6; f++)
          if (k0 + kk < SPT && off[kk] >= 0) {
            if constexpr (DOM == 2) u[kk][f] = __ldg(src[kk] + f * plane);
            else u[kk][f] = __ldg(tile.U + f * plane + off[kk]);
          }
      }
#pragma unroll
      for (int kk = 0; kk < KC; kk++) {
        int k = k0 + kk;
        int s = tid + k * NT;
        if (k >= SPT || s >= STAR) continue;
        R w[6], r;
        if (off[kk] >= 0) {
          if constexpr (MODE == 0) bad |= prim64(u[kk], gamma_d, g53, w, r);
          else bad |= prim_mixed(u[kk], gamma_d, gamf, gm1f, g53, w, r);
        } else {
#pragma unroll
          for (int f = 0; f < 6; f++) w[f] = (f == 0 || f == 4) ? R(1) : R(0);
          r = R(1);
        }
        if constexpr (MODE == 0) {
#pragma unroll
          for (int f = 0; f < 6; f++) W[f * STAR + s] = w[f];
        } else {
#pragma unroll
          for (int j = 0; j < 3; j++) W[j * STAR + s] = make_float2(w[2 * j], w[2 * j + 1]);
        }
        RR[s] = r;
      }
    }
    bad = __syncthreads_or(bad);
    if (!DOM && prefetch && t + (int)gridDim.x < n_tiles)
      prefetch_tile_l2(fetch(t + gridDim.x), tid, NT, prefetch);

    // ---- hydro group: rho, momentum, E, tau
    R amax = R(0);
    {
      Acc acc[CPT][NS];
      if constexpr (DOM == 2)
        group_pass<MODE, NT, true>(W, GG, QS, lch, NS, ex, ey, ez, gamma, inv_gm1, knp, acc, amax,
                                   fetch.capture(tile, 0));
      else
        group_pass<MODE, NT, true>(W, GG, QS, lch, NS, ex, ey, ez, gamma, inv_gm1, knp, acc, amax);
      store_group<MODE, NT, (DOM != 0)>(out, tile, ex, ey, ez, 0, 6, acc, stage);
    }

    // ---- A0/A1 (species): X_k = rho_k / rho into the group slots
    const int nsp = F - 6;
    if (nsp > 0) {
#pragma unroll 1
      for (int k0 = 0; k0 < SPT; k0 += KC) {
        double v[KC][MAXF - 6];
        int off[KC];
        const double* src[KC];
#pragma unroll
        for (int kk = 0; kk < KC; kk++) {
          if constexpr (DOM == 2) {
            src[kk] = slot_src(tid + (k0 + kk) * NT);
            off[kk] = src[kk] ? 0 : -1;
          } else {
            off[kk] = slot_offset(tid + (k0 + kk) * NT);
          }
#pragma unroll
          for (int f = 0; f < MAXF - 6; f++)
            if (k0 + kk < SPT && off[kk] >= 0 && f < nsp) {
              if constexpr (DOM == 2) v[kk][f] = __ldg(src[kk] + (6 + f) * plane);
              else v[kk][f] = __ldg(tile.U + (6 + f) * plane + off[kk]);
            }
        }
#pragma unroll
        for (int kk = 0; kk < KC; kk++) {
          int k = k0 + kk;
          int s = tid + k * NT;
          if (k >= SPT || s >= STAR) continue;
          R r = RR[s];
          R x[MAXF - 6];
          unsigned oor = 0;
#pragma unroll
          for (int f = 0; f < MAXF - 6; f++) {
            x[f] = R(0);
            if (f < nsp && off[kk] >= 0) {
              if constexpr (MODE == 0) {
                bad |= !dfinite(v[kk][f]);
                x[f] = v[kk][f] * r;
              } else {
                x[f] = d2f_fast_pos(v[kk][f], oor) * r;
              }
            }
          }
          if constexpr (MODE == 1) {
            if (oor >= D2F_OOR) {  // rare: convert the cell's species again
#pragma unroll
              for (int f = 0; f < MAXF - 6; f++)
                if (f < nsp && off[kk] >= 0) x[f] = d2f_slow(v[kk][f]) * r;
            }
#pragma unroll
            for (int f = 0; f < MAXF - 6; f++)  // a non-finite input leaves a non-finite quotient
              if (f < nsp) bad |= !isfinite(x[f]);
          }
          if constexpr (MODE == 0) {
#pragma unroll
            for (int f = 0; f < MAXF - 6; f++)
              if (f < nsp) W[f * STAR + s] = x[f];
          } else {
#pragma unroll
            for (int j = 0; j < 3; j++)
              if (2 * j < nsp) W[j * STAR + s] = make_float2(x[2 * j], 2 * j + 1 < MAXF - 6 ? x[2 * j + 1] : 0.0f);
          }
        }
      }
    }
    bad = __syncthreads_or(bad);
    if (bad && tid == 0 && write_status) {
      atomicOr(&status->flags, 1u);
      atomicMin(&status->first_bad, (unsigned long long)tile.sub);
    }

    // ---- species group
    if (nsp > 0) {
      Acc acc[CPT][NS];
      if constexpr (DOM == 2)
        group_pass<MODE, NT, false>(W, GG, QS, lch, (nsp + PK - 1) / PK, ex, ey, ez, gamma, inv_gm1,
                                    knp, acc, amax, fetch.capture(tile, 6));
      else
        group_pass<MODE, NT, false>(W, GG, QS, lch, (nsp + PK - 1) / PK, ex, ey, ez, gamma, inv_gm1,
                                    knp, acc, amax);
      store_group<MODE, NT, (DOM != 0)>(out, tile, ex, ey, ez, 6, nsp, acc, stage);
    }

    // ---- A5: largest signal speed of the tile
    double am = (double)amax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) am = dmaxp(am, __shfl_xor_sync(0xffffffffu, am, o));
    if ((tid & 31) == 0) red[tid >> 5] = am;
    __syncthreads();
    if (tid == 0) {
      double m = red[0];
      for (int w = 1; w < NT / 32; w++) m = dmaxp(m, red[w]);
      if (tile.flags & 1)
        atomicMax(reinterpret_cast<unsigned long long*>(amax_out + tile.amax_off),
                  (unsigned long long)__double_as_longlong(m));
      else
        amax_out[tile.amax_off] = m;
    }
    __syncthreads();
  }
}

// KC: read-region slots per load batch (more loads in flight with more
// registers per thread; the autotuner picks among compiled variants).
template <int MODE, int NT, int MINB, int KC = (MINB == 1 ? 4 : 2)>
__global__ void __launch_bounds__(NT, MINB)
rhs_tiles_kernel(const Tile* __restrict__ tiles, int n_tiles, int Fmax, int lch,
                 double* __restrict__ out, double* __restrict__ amax_out,
                 Status* __restrict__ status, double gamma_d, int write_status, int prefetch,
                 int scheme) {
  (void)Fmax;  // the shared-memory layout does not depend on the field count
  // scheme: 0 Kurganov-Tadmor, 1 Kurganov-Noelle-Petrova.
  tile_loop<MODE, NT, KC>(TileList{tiles}, n_tiles, lch, out, amax_out, status, gamma_d, write_status,
                          prefetch, scheme == 1);
}

// ================================================ pipelined mixed kernel ==
// The mixed form with the read region moved by asynchronous copies
// (cp.async, global -> shared, no registers held) into a staging buffer, one
// field group ahead: the species of tile t arrive while its hydro group is
// reconstructed and fluxed, and the hydro group of the CTA's next tile while
// its species are.  Full tiles of ghosted blocks whose rows start 16-byte
// aligned move in 16-byte copies: the interior rows with their x ghosts
// (7 per row) and every ghost-slab row as the aligned span x = -1 .. TE
// (5 per row; the 32-byte sectors the cells x = 0 .. TE-1 occupy in any
// case).  Full tiles of a ghost-free domain with even N move in 16-byte
// copies too, each located in its periodic sub-grid (8 per interior row
// x = -4 .. 11, 4 per ghost-slab row x = 0 .. TE-1; staged in the domain
// layout below).  Other tiles (partial, forests, misaligned blocks) use one
// 8-byte copy per cell.  One CTA of PNT threads per SM; the
// three directions are reconstructed together, so every phase divides
// evenly over the threads:
//   PPM   3 directions x 64 lines x 3 field pairs = 576 tasks
//   flux  3 rounds (one per direction) of 64 lines x 9 faces = 576 faces
//   A4    one interior cell per thread (threads 0..511)
// Shared memory (bytes): S  [6][SSTAR] binary64 staging     89088
//                        W  [3][STAR] float2 primitives     39936
//                        GG [3][NLN][NFC][2] float          13824
//                        QS [3][2][3][NLN][NFC] float2      82944
// Staging layout of one field: the interior rows [z][y][LL] as in the read
// region (XROWS), then the y-ghost rows [z][yg][SROW] and the z-ghost rows
// [zg][y][SROW], each holding x = -1 .. TE.  (Domain tiles: sslot_dom.)
constexpr int PNT = 3 * NLN * 3;  // 576
constexpr int PSPT = (STAR + PNT - 1) / PNT;  // read-region slots per thread: 3
constexpr int SROW = TE + 2;                  // a staged ghost-slab row
constexpr int SSTAR = XROWS + 2 * 6 * TE * SROW;  // 1856 staged values per field
__host__ __device__ constexpr size_t pipe_smem_bytes() {
  return (size_t)6 * SSTAR * 8 + 3 * STAR * 8 + 3 * NLN * NFC * 2 * 4 + 3 * 2 * 3 * NLN * NFC * 8;
}
// staging slot of read-region slot s
__host__ __device__ __forceinline__ int sslot(int s) {
  if (s < XROWS) return s;
  const int t = s - XROWS;  // ghost-slab cell: row t / TE, x = t % TE
  return XROWS + (t / TE) * SROW + (t % TE) + 1;
}
// The domain form's staging layout (ghost-free storage, where a tile's row
// x = 0..7 starts 16-byte aligned in its sub-grid when N is even): interior
// rows of DROW values x = -4..11, then the ghost-slab rows of the 8 values
// x = 0..7, so that every 2-cell chunk of an even x is 16-byte aligned in the
// stored rows and in shared memory.  It fits in one field's SSTAR.
constexpr int DROW = TE + 8;                           // 16
constexpr int DSTAR = TE * TE * DROW + 2 * 6 * TE * TE;  // 1792
static_assert(DSTAR <= SSTAR, "the domain staging layout fits a field's staging");
__host__ __device__ __forceinline__ int sslot_dom(int s) {
  if (s < XROWS) return (s / LL) * DROW + s % LL + 1;
  return TE * TE * DROW + (s - XROWS);
}
template <int DOM>
__host__ __device__ __forceinline__ int stage_slot(int s) {
  return DOM != 0 ? sslot_dom(s) : sslot(s);  // forests are ghost-free too
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Fetch tile t's descriptor into shared memory (one thread): a work list's
// entry by asynchronous copies (complete at the thread's next wait), other
// tile sources by computing it.
template <class Fetch>
__device__ __forceinline__ void prefetch_desc(const Fetch& fetch, int t, Tile* dst) {
  *dst = fetch(t);
}
__device__ __forceinline__ void prefetch_desc(const TileList& fetch, int t, Tile* dst) {
  const char* src = reinterpret_cast<const char*>(fetch.tiles + t);
#pragma unroll
  for (int i = 0; i < 4; i++) cp_async16(reinterpret_cast<char*>(dst) + 16 * i, src + 16 * i);
  cp_async_commit();
}

__device__ __forceinline__ void cp_async16cg(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// 16-byte copies: a full tile of a ghosted block whose rows start 16-byte
// aligned (G even, odd ghost width, block 16-byte aligned), so that the
// interior rows (from x = -3) and the ghost-slab rows (from x = -1) do.
template <int DOM>
__device__ __forceinline__ bool chunk_ok(const Tile& tile) {
  if constexpr (DOM == 2) {
    return false;
  } else if constexpr (DOM == 1) {
    // full tile of a domain with even N: every even-x chunk of 2 cells lies
    // in one sub-grid row, 16-byte aligned
    return tile.N - tile.ox >= TE && tile.N - tile.oy >= TE && tile.N - tile.oz >= TE && (tile.N & 1) == 0 &&
           (reinterpret_cast<uintptr_t>(tile.U) & 15) == 0;
  } else {
    const int gh = (tile.G - tile.N) >> 1;
    return tile.N - tile.ox >= TE && tile.N - tile.oy >= TE && tile.N - tile.oz >= TE && (tile.G & 1) == 0 &&
           (gh & 1) == 1 && (reinterpret_cast<uintptr_t>(tile.U) & 15) == 0;
  }
}
// The 16-byte chunks of one field's staging; every thread takes chunks tid
// and tid + PNT.  A chunk is (z, y, x0) of its first cell and its staging
// slot.  Ghosted blocks: 7 per interior row (64 rows, x0 in -3 + 2k), 5 per
// ghost-slab row (96 rows, x0 in -1 + 2k).  Domain form: 8 per interior row
// (x0 in -4 + 2k), 4 per ghost-slab row (x0 in 2k); forests the same.
constexpr int NCHUNK = TE * TE * (LL / 2) + 2 * 6 * TE * (SROW / 2);  // 928
constexpr int NCHUNK_D = TE * TE * (DROW / 2) + 2 * 6 * TE * (TE / 2);  // 896
constexpr int PCPT = (NCHUNK + PNT - 1) / PNT;                          // chunks per thread: 2
static_assert(NCHUNK_D <= PCPT * PNT, "the domain chunks fit the same count per thread");
struct ChunkGeom {
  int zyx[PCPT];  // z, y, x0 as signed bytes; 0x7f7f7f7f: none
  int st[PCPT];   // staging slot of the first double
  template <int DOM>
  __device__ __forceinline__ void init(int tid) {
    // chunks per interior row and per slab row, their first x, the slab rows' slot base and width
    constexpr bool GF = DOM != 0;  // ghost-free storage: domains and forests
    constexpr int CR = GF ? DROW / 2 : LL / 2, CS = GF ? TE / 2 : SROW / 2;
    constexpr int X0R = GF ? -4 : -3, X0S = GF ? 0 : -1;
    constexpr int RW = GF ? DROW : LL, SBASE = GF ? TE * TE * DROW : XROWS, SW = GF ? TE : SROW;
    constexpr int NC = TE * TE * CR + 2 * 6 * TE * CS;
#pragma unroll
    for (int k = 0; k < PCPT; k++) {
      const int c = tid + k * PNT;
      int z = 0, y = 0, x0 = 0, slot = 0;
      if (c < TE * TE * CR) {
        const int row = c / CR, q = c % CR;
        z = row / TE;
        y = row % TE;
        x0 = X0R + 2 * q;
        slot = row * RW + 2 * q;
      } else if (c < NC) {
        const int c2 = c - TE * TE * CR, r = c2 / CS, q = c2 % CS;
        if (r < 6 * TE) {
          z = r / 6;
          const int yg = r % 6;
          y = yg < 3 ? yg - 3 : yg + TE - 3;
        } else {
          const int r2 = r - 6 * TE, zg = r2 / TE;
          y = r2 % TE;
          z = zg < 3 ? zg - 3 : zg + TE - 3;
        }
        x0 = X0S + 2 * q;
        slot = SBASE + r * SW + 2 * q;
      }
      zyx[k] = c < NC ? ((z & 0xff) | ((y & 0xff) << 8) | ((x0 & 0xff) << 16)) : 0x7f7f7f7f;
      st[k] = slot;
    }
  }
};
// Issue the 16-byte copies of fields f0 .. f0+nf-1 of a domain tile
// (chunk_ok<1>): each chunk located in its (periodic) sub-grid.
__device__ __forceinline__ void chunk_issue_dom(const Tile& tile, const ChunkGeom& cg, double* S, int f0, int nf) {
  const int N = tile.N;
  const long long plane = (long long)N * N * N;
  DomainPos dp;
  dp.init(tile.sub, tile.pad[0], N, tile.F);
  const double* base = tile.U + (long long)f0 * plane;
#pragma unroll
  for (int k = 0; k < PCPT; k++) {
    if (cg.zyx[k] == 0x7f7f7f7f) continue;
    const int z = (int)(signed char)(cg.zyx[k] & 0xff), y = (int)(signed char)((cg.zyx[k] >> 8) & 0xff),
              x0 = (int)(signed char)((cg.zyx[k] >> 16) & 0xff);
    const double* src = base + dp.off(tile.ox + x0, tile.oy + y, tile.oz + z);
#pragma unroll
    for (int f = 0; f < 6; f++)
      if (f < nf) cp_async16cg(S + f * SSTAR + cg.st[k], src + f * plane);
  }
}
// The same for a forest leaf (a full tile of even N whose leaf and
// auxiliary blocks start 16-byte aligned): each chunk in the block that
// ForestLoc locates -- the leaf, a same-level neighbour or the auxiliary
// block of a face towards another level, all stored [F][N^3].  A chunk
// never straddles two blocks (N even, x0 even); the cells x = -4 and 11 it
// also copies go to staging slots that nothing reads.
__device__ __forceinline__ void chunk_issue_forest(const ForestLoc& fl, const Tile& tile, const ChunkGeom& cg,
                                                   double* S, int f0, int nf) {
  const long long plane = (long long)tile.N * tile.N * tile.N;
#pragma unroll
  for (int k = 0; k < PCPT; k++) {
    if (cg.zyx[k] == 0x7f7f7f7f) continue;
    const int z = (int)(signed char)(cg.zyx[k] & 0xff), y = (int)(signed char)((cg.zyx[k] >> 8) & 0xff),
              x0 = (int)(signed char)((cg.zyx[k] >> 16) & 0xff);
    const double* src = fl.ptr(tile.ox + x0, tile.oy + y, tile.oz + z) + (long long)f0 * plane;
#pragma unroll
    for (int f = 0; f < 6; f++)
      if (f < nf) cp_async16cg(S + f * SSTAR + cg.st[k], src + f * plane);
  }
}
// Issue the 16-byte copies of fields f0 .. f0+nf-1 (chunk_ok tiles).
__device__ __forceinline__ void chunk_issue(const Tile& tile, const ChunkGeom& cg, double* S, int f0, int nf) {
  const int G = tile.G, gh = (G - tile.N) >> 1;
  const long long plane = (long long)G * G * G;
  const double* base = tile.U + (long long)f0 * plane +
                       ((long long)(tile.oz + gh) * G + (tile.oy + gh)) * G + (tile.ox + gh);
#pragma unroll
  for (int k = 0; k < PCPT; k++) {
    if (cg.zyx[k] == 0x7f7f7f7f) continue;
    const int z = (int)(signed char)(cg.zyx[k] & 0xff), y = (int)(signed char)((cg.zyx[k] >> 8) & 0xff),
              x0 = (int)(signed char)((cg.zyx[k] >> 16) & 0xff);
    const double* src = base + ((long long)z * G + y) * G + x0;
#pragma unroll
    for (int f = 0; f < 6; f++)
      if (f < nf) cp_async16cg(S + f * SSTAR + cg.st[k], src + f * plane);
  }
}

// Read-region geometry of one thread's slots, computed once per kernel:
// tile-local (x, y, z) packed as three signed bytes, and the staging slot.
struct SlotXYZ {
  int p[PSPT];
  int ss[PSPT];
  template <int DOM>
  __device__ __forceinline__ void init(int tid) {
#pragma unroll
    for (int k = 0; k < PSPT; k++) {
      int s = tid + k * PNT, x = 0, y = 0, z = 0;
      if (s < STAR) cell_of(s, x, y, z);
      p[k] = (x & 0xff) | ((y & 0xff) << 8) | ((z & 0xff) << 16);
      ss[k] = stage_slot<DOM>(s < STAR ? s : 0);
    }
  }
  __device__ __forceinline__ void get(int k, int& x, int& y, int& z) const {
    x = (int)(signed char)(p[k] & 0xff);
    y = (int)(signed char)((p[k] >> 8) & 0xff);
    z = (int)(signed char)((p[k] >> 16) & 0xff);
  }
};

// Offset (doubles, within one field) of read-region cell (x, y, z) of the
// tile, or -1 if the (possibly partial) tile does not read it.
__device__ __forceinline__ bool pipe_valid(int x, int y, int z, int ex, int ey, int ez) {
  int outside = (x < 0 || x >= ex) + (y < 0 || y >= ey) + (z < 0 || z >= ez);
  return outside <= 1 && x < ex + 3 && y < ey + 3 && z < ez + 3;
}
template <bool DOMAIN>
__device__ __forceinline__ int pipe_offset(const Tile& tile, const DomainPos& dp, int x, int y, int z, int ex,
                                           int ey, int ez) {
  if (!pipe_valid(x, y, z, ex, ey, ez)) return -1;
  const int N = tile.N;
  if constexpr (DOMAIN) {
    return dp.off(tile.ox + x, tile.oy + y, tile.oz + z);
  } else {
    const int G = tile.G, gh = (G - N) >> 1;
    return ((tile.oz + z + gh) * G + (tile.oy + y + gh)) * G + (tile.ox + x + gh);
  }
}

// Issue the copies of fields f0 .. f0+nf-1 of the tile's read region into S:
// 16-byte copies where chunk_ok, else one 8-byte copy per cell (DOM as in
// tile_loop; a forest locates cells through fetch.loc).
template <int DOM, class Fetch>
__device__ __forceinline__ void pipe_issue(const Fetch& fetch, const Tile& tile, const SlotXYZ& sx,
                                           const ChunkGeom& cg, double* S, int f0, int nf) {
  bool chunks;
  if constexpr (DOM == 2) {
    chunks = tile.N - tile.ox >= TE && tile.N - tile.oy >= TE && tile.N - tile.oz >= TE && (tile.N & 1) == 0 &&
             ((reinterpret_cast<uintptr_t>(fetch.U) | reinterpret_cast<uintptr_t>(fetch.aux)) & 15) == 0;
  } else {
    chunks = chunk_ok<DOM>(tile);
  }
  if (chunks) {
    if constexpr (DOM == 1) chunk_issue_dom(tile, cg, S, f0, nf);
    else if constexpr (DOM == 2) chunk_issue_forest(fetch.loc(tile), tile, cg, S, f0, nf);
    else chunk_issue(tile, cg, S, f0, nf);
    cp_async_commit();
    return;
  }
  const int N = tile.N;
  const int ex = min(TE, N - tile.ox), ey = min(TE, N - tile.oy), ez = min(TE, N - tile.oz);
  const long long plane = DOM ? (long long)N * N * N : (long long)tile.G * tile.G * tile.G;
  DomainPos dp;
  if constexpr (DOM == 1) dp.init(tile.sub, tile.pad[0], N, tile.F);
  ForestLoc fl;
  if constexpr (DOM == 2) fl = fetch.loc(tile);
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < PSPT; k++) {
    int s = tid + k * PNT;
    if (s >= STAR) continue;
    int x, y, z;
    sx.get(k, x, y, z);
    const double* src;
    if constexpr (DOM == 2) {
      if (!pipe_valid(x, y, z, ex, ey, ez)) continue;
      src = fl.ptr(tile.ox + x, tile.oy + y, tile.oz + z) + (long long)f0 * plane;
    } else {
      int off = pipe_offset<DOM == 1>(tile, dp, x, y, z, ex, ey, ez);
      if (off < 0) continue;
      src = tile.U + (long long)f0 * plane + off;
    }
#pragma unroll
    for (int f = 0; f < 6; f++)
      if (f < nf) cp_async8(S + f * SSTAR + sx.ss[k], src + f * plane);
  }
  cp_async_commit();
}
template <class Fetch, int DOM>
__device__ __forceinline__ void tile_loop_pipe(const Fetch& fetch, int n_tiles, double* __restrict__ out,
                                               double* __restrict__ amax_out, Status* __restrict__ status,
                                               double gamma_d, int write_status, bool knp,
                                               const StageArgs& stage) {
  typedef P2 Acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* S = reinterpret_cast<double*>(smem_raw);
  float2* W = reinterpret_cast<float2*>(S + 6 * SSTAR);
  float* GG = reinterpret_cast<float*>(W + 3 * STAR);
  float2* QS = reinterpret_cast<float2*>(GG + 3 * NLN * NFC * 2);
  __shared__ double red[PNT / 32];
  const int tid = threadIdx.x;
  const float gamma = (float)gamma_d;
  const float inv_gm1 = (float)(1.0 / (gamma_d - 1.0));
  const float gm1f = (float)(gamma_d - 1.0);
  const bool g53 = gamma_d == 5.0 / 3.0;
  constexpr int FS = NLN * NFC;  // stride between pair slots of QS (576)
  // QS block of (direction d, side 0 left / 1 right, pair j)
  auto qs = [&](int d, int side, int j) { return QS + ((d * 2 + side) * 3 + j) * FS; };
  SlotXYZ sx;
  sx.template init<DOM>(tid);
  ChunkGeom cg;
  cg.template init<DOM>(tid);
  // Tile descriptors, double-buffered in shared memory: thread 0 fetches the
  // next tile's while the current one is converted, so that its latency is
  // hidden before the next tile's copies are issued.
  __shared__ Tile tsm[2];

  int t = blockIdx.x;
  if (tid == 0 && t < n_tiles) tsm[0] = fetch(t);
  __syncthreads();
  if (t < n_tiles) pipe_issue<DOM>(fetch, tsm[0], sx, cg, S, 0, 6);
  for (int it = 0; t < n_tiles; t += gridDim.x, it ^= 1) {
    const Tile tile = tsm[it];
    const int F = tile.F, N = tile.N, nsp = F - 6;
    const int ex = min(TE, N - tile.ox), ey = min(TE, N - tile.oy), ez = min(TE, N - tile.oz);
    const bool full = ex == TE && ey == TE && ez == TE;
    const int tn = t + (int)gridDim.x;

    // ---- A0/A1 hydro: staged binary64 (rho, s, E, tau) -> binary32 primitives.
    // The common path of every slot first (straight-line code, so that the
    // slots' long latency chains interleave), then the careful path for the
    // few cells that need it.
    cp_async_wait_all();
    __syncthreads();
    if (tid == 0 && tn < n_tiles) prefetch_desc(fetch, tn, &tsm[it ^ 1]);
    bool bad = false;
    {
      float w[PSPT][6], r[PSPT];
      bool need[PSPT], valid[PSPT];
#pragma unroll
      for (int k = 0; k < PSPT; k++) {
        const int s = tid + k * PNT;
        int x, y, z;
        sx.get(k, x, y, z);
        valid[k] = s < STAR && (full || pipe_valid(x, y, z, ex, ey, ez));
        need[k] = false;
        if (valid[k]) {
          double u[6];
#pragma unroll
          for (int f = 0; f < 6; f++) u[f] = S[f * SSTAR + sx.ss[k]];
          need[k] = prim_mixed_fast(u, gamma, gm1f, g53, w[k], r[k]);
        } else {
#pragma unroll
          for (int f = 0; f < 6; f++) w[k][f] = (f == 0 || f == 4) ? 1.0f : 0.0f;
          r[k] = 1.0f;
        }
      }
#pragma unroll
      for (int k = 0; k < PSPT; k++) {
        if (need[k]) {
          double u[6];
#pragma unroll
          for (int f = 0; f < 6; f++) u[f] = S[f * SSTAR + sx.ss[k]];
          prim_mixed_slow(u, gamma_d, gamma, gm1f, g53, w[k], r[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < PSPT; k++) {
        const int s = tid + k * PNT;
        if (s >= STAR) continue;
        if (valid[k]) bad |= prim_mixed_bad(w[k]);
#pragma unroll
        for (int j = 0; j < 3; j++) W[j * STAR + s] = make_float2(w[k][2 * j], w[k][2 * j + 1]);
      }
    }
    if (tid == 0) cp_async_wait_all();  // the next tile's descriptor
    bad = __syncthreads_or(bad);
    // the staging buffer is free: species of this tile, or the next tile
    if (nsp > 0) pipe_issue<DOM>(fetch, tile, sx, cg, S, 6, nsp);
    else if (tn < n_tiles) pipe_issue<DOM>(fetch, tsm[it ^ 1], sx, cg, S, 0, 6);

    float amax = 0.0f;
    Acc acc[1][3];
    // ---- A2 hydro, three directions at once
    {
      const int d = tid / (3 * NLN), rem = tid - d * 3 * NLN, j = rem / NLN, l = rem - j * NLN;
      LineAddr la = line_addr(d, l);
      ppm_line32x2(W + j * STAR, la, qs(d, 0, j) + l * NFC, qs(d, 1, j) + l * NFC);
    }
    __syncthreads();
    // ---- A3 hydro: one direction per round, 576 faces each
    {
      const int l = tid / NFC, i = tid - l * NFC;
#pragma unroll 1
      for (int d = 0; d < 3; d++) {
        float2* fo = qs(d, 0, 0) + l * NFC + i;
        const float2* fr = qs(d, 1, 0) + l * NFC + i;
        float2 wl[3], wr[3];
#pragma unroll
        for (int j = 0; j < 3; j++) {
          wl[j] = fo[j * FS];
          wr[j] = fr[j * FS];
        }
        float gl, gr;
        float a = kt_hydro32(wl, wr, d, gamma, inv_gm1, knp, fo, FS, gl, gr);
        float* g = GG + ((d * NLN + l) * NFC + i) * 2;
        store_pair(g, gl, gr);
        const int e_d = d == 0 ? ex : (d == 1 ? ey : ez);
        const int e_a = d == 0 ? ey : ex;
        const int e_b = d == 2 ? ey : ez;
        if ((l % TE) < e_a && (l / TE) < e_b && i <= e_d) amax = fmaxf(amax, a);
      }
    }
    __syncthreads();
    // ---- A4 hydro: the flux differences of the thread's cell, x, y, z
    auto diff_pass = [&](int npair) {
      if (tid < TE * TE * TE) {
        const int x = tid % TE, y = (tid / TE) % TE, z = tid / (TE * TE);
#pragma unroll
        for (int d = 0; d < 3; d++) {
          const int l = d == 0 ? z * TE + y : (d == 1 ? z * TE + x : y * TE + x);
          const int pos = d == 0 ? x : (d == 1 ? y : z);
          const float2* fl = qs(d, 0, 0) + l * NFC + pos;
#pragma unroll
          for (int j = 0; j < 3; j++)
            if (j < npair) acc_pair2(acc[0][j], fl[j * FS + 1], fl[j * FS], d == 0);
        }
      }
    };
    if constexpr (DOM == 2) {
      const ForestCapture cap = fetch.capture(tile, 0);
#pragma unroll 1
      for (int d = 0; d < 3; d++) cap.template faces<PNT>(qs(d, 0, 0), FS, NLN, 0, 3, d, ex, ey, ez);
    }
    diff_pass(3);
    store_group<1, PNT, (DOM != 0)>(out, tile, ex, ey, ez, 0, 6, acc, stage);

    if (nsp > 0) {
      const int npair = (nsp + 1) / 2;
      // ---- A0/A1 species: X_k = rho_k / rho (every slot first, then the
      // rare cells with a value outside the fast conversion's range); 1/rho
      // is formed again from the staged rho, bit for bit the hydro pass's
      cp_async_wait_all();
      __syncthreads();
      {
        float xs[PSPT][6], rs[PSPT];
        unsigned oor[PSPT];
        bool valid[PSPT];
#pragma unroll
        for (int k = 0; k < PSPT; k++) {
          const int s = tid + k * PNT;
          int x, y, z;
          sx.get(k, x, y, z);
          valid[k] = s < STAR && (full || pipe_valid(x, y, z, ex, ey, ez));
          rs[k] = s < STAR ? rcp32(W[s].x) : 0.0f;
          oor[k] = 0;
#pragma unroll
          for (int f = 0; f < 6; f++) {
            xs[k][f] = 0.0f;
            if (f < nsp && valid[k]) xs[k][f] = d2f_fast_pos(S[f * SSTAR + sx.ss[k]], oor[k]) * rs[k];
          }
        }
#pragma unroll
        for (int k = 0; k < PSPT; k++) {
          if (oor[k] >= D2F_OOR) {
#pragma unroll
            for (int f = 0; f < 6; f++)
              if (f < nsp) xs[k][f] = d2f_slow(S[f * SSTAR + sx.ss[k]]) * rs[k];
          }
        }
#pragma unroll
        for (int k = 0; k < PSPT; k++) {
          const int s = tid + k * PNT;
          if (s >= STAR) continue;
#pragma unroll
          for (int f = 0; f < 6; f++)  // a non-finite input leaves a non-finite quotient
            if (f < nsp) bad |= !isfinite(xs[k][f]);
#pragma unroll
          for (int j = 0; j < 3; j++)
            if (j < npair) W[j * STAR + s] = make_float2(xs[k][2 * j], xs[k][2 * j + 1]);
        }
      }
      bad = __syncthreads_or(bad);
      if (tn < n_tiles) pipe_issue<DOM>(fetch, tsm[it ^ 1], sx, cg, S, 0, 6);
      // ---- A2 species
      {
        const int d = tid / (3 * NLN), rem = tid - d * 3 * NLN, j = rem / NLN, l = rem - j * NLN;
        if (j < npair) {
          LineAddr la = line_addr(d, l);
          ppm_line32x2(W + j * STAR, la, qs(d, 0, j) + l * NFC, qs(d, 1, j) + l * NFC);
        }
      }
      __syncthreads();
      // ---- A3 species: q_l g_l + q_r g_r
      {
        const int l = tid / NFC, i = tid - l * NFC;
#pragma unroll 1
        for (int d = 0; d < 3; d++) {
          float2* fo = qs(d, 0, 0) + l * NFC + i;
          const float2* fr = qs(d, 1, 0) + l * NFC + i;
          const float* g = GG + ((d * NLN + l) * NFC + i) * 2;
          float gl, gr;
          load_pair(g, gl, gr);
#pragma unroll
          for (int j = 0; j < 3; j++)
            if (j < npair) fo[j * FS] = fma2(fo[j * FS], f2(gl), mul2(fr[j * FS], f2(gr)));
        }
      }
      __syncthreads();
      if constexpr (DOM == 2) {
        const ForestCapture cap = fetch.capture(tile, 6);
#pragma unroll 1
        for (int d = 0; d < 3; d++) cap.template faces<PNT>(qs(d, 0, 0), FS, NLN, 0, npair, d, ex, ey, ez);
      }
      diff_pass(npair);
      store_group<1, PNT, (DOM != 0)>(out, tile, ex, ey, ez, 6, nsp, acc, stage);
    }
    if (bad && tid == 0 && write_status) {
      atomicOr(&status->flags, 1u);
      atomicMin(&status->first_bad, (unsigned long long)tile.sub);
    }

    // ---- A5: largest signal speed of the tile
    double am = (double)amax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) am = dmaxp(am, __shfl_xor_sync(0xffffffffu, am, o));
    if ((tid & 31) == 0) red[tid >> 5] = am;
    __syncthreads();
    if (tid == 0) {
      double m = red[0];
      for (int w = 1; w < PNT / 32; w++) m = dmaxp(m, red[w]);
      if (tile.flags & 1)
        atomicMax(reinterpret_cast<unsigned long long*>(amax_out + tile.amax_off),
                  (unsigned long long)__double_as_longlong(m));
      else
        amax_out[tile.amax_off] = m;
    }
  }
  cp_async_wait_all();
}

// Same arguments as rhs_tiles_kernel; lch and prefetch do not apply.
// (A template so that every translation unit may instantiate it.)
template <int NT>
__global__ void __launch_bounds__(NT, 1)
rhs_tiles_pipe_kernel(const Tile* __restrict__ tiles, int n_tiles, int Fmax, int lch,
                      double* __restrict__ out, double* __restrict__ amax_out,
                      Status* __restrict__ status, double gamma_d, int write_status, int prefetch,
                      int scheme) {
  static_assert(NT == PNT, "the pipelined kernel runs PNT threads");
  (void)Fmax;
  (void)lch;
  (void)prefetch;
  tile_loop_pipe<TileList, 0>(TileList{tiles}, n_tiles, out, amax_out, status, gamma_d, write_status,
                                  scheme == 1, StageArgs{nullptr, nullptr, 0.0, 0.0, 0.0, 0});
}

// Tiles of a periodic domain of nb^3 sub-grids of N^3 (F fields each),
// stored without ghosts; computed on the fly, no work list.
struct DomainTiles {
  const double* __restrict__ U;
  int nb, N, F, tpe;  // tpe: tiles per sub-grid edge
  double inv_dx;
  short flags;        // bit 1: dx a power of two
  __device__ __forceinline__ Tile operator()(int t) const {
    const int tps = tpe * tpe * tpe;
    const int s = t / tps, k = t - s * tps;
    Tile tile;
    tile.U = U;
    tile.out_off = (long long)s * F * N * N * N;
    tile.amax_off = s;
    tile.inv_dx = inv_dx;
    tile.sub = s;
    tile.N = N;
    tile.F = F;
    tile.G = N;
    tile.ox = (short)((k % tpe) * TE);
    tile.oy = (short)(((k / tpe) % tpe) * TE);
    tile.oz = (short)((k / (tpe * tpe)) * TE);
    tile.flags = (short)((tps > 1 ? 1 : 0) | (flags & 2));
    tile.pad[0] = nb;
    tile.pad[1] = 0;
    return tile;
  }
};

template <int MODE, int NT, int MINB, int KC = (MINB == 1 ? 4 : 2)>
__global__ void __launch_bounds__(NT, MINB)
rhs_domain_kernel(DomainTiles dom, int n_tiles, int lch, double* __restrict__ out,
                  double* __restrict__ amax_out, Status* __restrict__ status, double gamma_d,
                  int write_status, int scheme, StageArgs stage) {
  tile_loop<MODE, NT, KC, DomainTiles, 1>(dom, n_tiles, lch, out, amax_out, status, gamma_d, write_status,
                                             0, scheme == 1, stage);
}

// Forest tiles (register-load kernel; see ForestTiles).
template <int MODE, int NT, int MINB, int KC = (MINB == 1 ? 4 : 2)>
__global__ void __launch_bounds__(NT, MINB)
rhs_forest_kernel(ForestTiles ft, int n_tiles, int lch, double* __restrict__ out,
                  double* __restrict__ amax_out, Status* __restrict__ status, double gamma_d,
                  int write_status, int scheme, StageArgs stage) {
  tile_loop<MODE, NT, KC, ForestTiles, 2>(ft, n_tiles, lch, out, amax_out, status, gamma_d, write_status, 0,
                                          scheme == 1, stage);
}

template <int NT>
__global__ void __launch_bounds__(NT, 1)
rhs_domain_pipe_kernel(DomainTiles dom, int n_tiles, int lch, double* __restrict__ out,
                       double* __restrict__ amax_out, Status* __restrict__ status, double gamma_d,
                       int write_status, int scheme, StageArgs stage) {
  static_assert(NT == PNT, "the pipelined kernel runs PNT threads");
  (void)lch;
  tile_loop_pipe<DomainTiles, 1>(dom, n_tiles, out, amax_out, status, gamma_d, write_status, scheme == 1,
                                    stage);
}

// Forest tiles, pipelined mixed kernel.
template <int NT>
__global__ void __launch_bounds__(NT, 1)
rhs_forest_pipe_kernel(ForestTiles ft, int n_tiles, int lch, double* __restrict__ out,
                       double* __restrict__ amax_out, Status* __restrict__ status, double gamma_d,
                       int write_status, int scheme, StageArgs stage) {
  static_assert(NT == PNT, "the pipelined kernel runs PNT threads");
  (void)lch;
  tile_loop_pipe<ForestTiles, 2>(ft, n_tiles, out, amax_out, status, gamma_d, write_status, scheme == 1, stage);
}

}  // namespace hydro_dev
