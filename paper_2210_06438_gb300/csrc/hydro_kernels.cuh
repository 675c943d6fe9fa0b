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
//      variables on the way into shared memory                    (steps A0-A1)
//   2. for each direction, in chunks of lines: PPM face states of every
//      (line, field) (step A2), then the central flux of every face with its
//      signal speed (step A3), written back in place
//   3. every thread owns fixed cells and accumulates the flux differences of
//      x, then y, then z in registers (step A4); the result is scaled by
//      -1/dx and stored.  The largest signal speed is reduced with warp
//      shuffles and one atomic per tile (step A5).
//
// MODE 0 runs every step in binary64.  On this GPU the binary64 pipe issues
// about 2 operations per SM per clock (1/64 of binary32), so the binary64 form
// is bound by that pipe: comparisons, absolute values, minima, sign tests and
// scalings by powers of two run on the integer pipe on the bit patterns, and
// the flux is written in an algebraically reduced form (see kt_face64).
//
// MODE 1 (mixed) converts the binary64 inputs to binary32 with integer
// operations, forms primitives in binary32 (the dual-energy decision and the
// internal energy near it are recomputed in binary64), reconstructs and
// fluxes in binary32, and carries the flux differences and their sum as exact
// binary32 pairs (error-free transformations, Knuth's TwoSum), so that the
// binary64 result telescopes across faces like the binary64 form.
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
  long long out_off;   // first output double of the sub-grid, relative to the launch's out pointer
  long long amax_off;  // signal-speed slot of the sub-grid, relative to the launch's amax pointer
  double inv_dx;       // 1/dx
  int sub;             // sub-grid index reported in the status word
  int N;               // sub-grid interior edge
  int F;               // fields
  int G;               // stored edge N + 2*ghost
  short ox, oy, oz;    // tile origin (cells)
  short flags;         // bit 0: the sub-grid has more than one tile; bit 1: dx is a power of 2
  int pad[2];
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

// slot of position c (0..LL-1, cell c-3) of line l along direction d
__device__ __forceinline__ int line_slot(int d, int l, int c) {
  int a = l % TE, b = l / TE;
  if (d == 0) return slot_of(c - 3, a, b);
  if (d == 1) return slot_of(a, c - 3, b);
  return slot_of(a, b, c - 3);
}

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
__device__ __forceinline__ double dtwice(double x) {  // 2x, x non-zero
  return __hiloint2double(hiw(x) + 0x00100000, __double2loint(x));
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

// Reciprocal and reciprocal square root: the hardware seed refined by two
// Newton-Raphson steps (quadratic convergence; Markstein 1990), ~1 ulp.
__device__ __forceinline__ double rcp64(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ double rsqrt64(double z) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(z));
  double hz = dhalf(z);
  double t = fma(-(hz * y), y, 1.5);
  y = y * t;
  t = fma(-(hz * y), y, 1.5);
  return y * t;
}

// tau^gamma.  For gamma = 5/3: tau^(5/3) = tau * w with w^3 = tau^2, w seeded
// in binary32 (log2/exp2) and refined by one Halley step (cubic convergence),
// then ~1 ulp.  Other gamma, or tau outside [1e-30, 1e30]: pow().
__device__ __forceinline__ double tau_pow64(double tau, double gamma, bool g53) {
  if (!g53 || !(tau > 1e-30 && tau < 1e30)) return pow(tau, gamma);
  float tf = __double2float_rn(tau);
  double w = (double)exp2f((2.0f / 3.0f) * __log2f(tf));
  double A = tau * tau;
  double w3 = w * w * w;
  w = w * fma(2.0, A, w3) * rcp64(fma(2.0, w3, A));
  return tau * w;
}

// ---------------------------------------------------- step A1, binary64 --
// Conserved -> primitive (rho, v, p, phi = tau/rho; the species X_k =
// rho_k/rho are formed by the caller with the returned r = 1/rho).
// The dual-energy branch is decided on e_int = E - |s|^2/(2 rho) against
// eta*E.  A fast estimate (reciprocal, fused operations) decides it when it
// is far from the threshold; inside [eta/2, 20 eta]*E the quantities are
// recomputed with correctly rounded operations in the reference order, so the
// branch is taken exactly as the reference definition takes it.
__device__ __forceinline__ bool prim64(const double* u, double gamma, bool g53, double* w,
                                       double& r) {
  double rho = u[0], E = u[4], tau = u[5];
  r = rcp64(rho);
  double ssq = fma(u[3], u[3], fma(u[2], u[2], u[1] * u[1]));
  double eint = fma(-dhalf(ssq), r, E);
  double thr = ETA * E;
  double e;
  if (dgt(eint, dhalf(thr)) && dgt(20.0 * thr, eint)) {  // near the switch: exact path
    double ss = __dadd_rn(__dadd_rn(__dmul_rn(u[1], u[1]), __dmul_rn(u[2], u[2])), __dmul_rn(u[3], u[3]));
    double ex = __dsub_rn(E, __ddiv_rn(__dmul_rn(0.5, ss), rho));
    e = ex < __dmul_rn(ETA, E) ? tau_pow64(tau, gamma, g53) : ex;
  } else {
    e = dgt(thr, eint) ? tau_pow64(tau, gamma, g53) : eint;
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
//   left[i] = q+ of cell i-1,  right[i] = q- of cell i.
// The parabola tests D*m > D^2/6 and D*m < -D^2/6 (m = q - (q- + q+)/2,
// D = q+ - q-) are evaluated as (D X) vs +-(D D/3) with X = 2m; the limiter is
// continuous at both switching surfaces, so the different rounding of the
// tests moves results by rounding errors only.
__device__ __forceinline__ void ppm_line64(const double* q, double* left, double* right) {  // left/right: shared memory
  double dq[LL - 1];
#pragma unroll
  for (int c = 0; c < LL - 1; c++) dq[c] = q[c + 1] - q[c];
  double del[LL];
#pragma unroll
  for (int c = 1; c <= LL - 2; c++) {
    double dp = dq[c], dm = dq[c - 1];
    double dbar = dhalf(q[c + 1] - q[c - 1]);
    double m = dminp(dabs(dbar), dtwice(dminp(dabs(dm), dabs(dp))));
    del[c] = dsame(dp, dm) ? dcopysign(m, dbar) : 0.0;
  }
  const double sixth = 1.0 / 6.0, third = 1.0 / 3.0;
  double fc[LL];
#pragma unroll
  for (int c = 1; c <= LL - 3; c++) fc[c] = fma(del[c] - del[c + 1], sixth, dhalf(q[c] + q[c + 1]));
#pragma unroll
  for (int c = 2; c <= LL - 3; c++) {  // cells -1 .. TE
    double qc = q[c], lo = fc[c - 1], hi = fc[c];
    double up = hi - qc, dn = qc - lo;
    bool ext = !dsame(up, dn);
    double D = up + dn;
    double X = dn - up;
    double Y = D * X;
    double Z = D * (D * third);
    bool A = dgt(Y, Z);
    bool B = !A && dgt(-Z, Y);
    double lo2 = fma(-2.0, up, qc);
    double hi2 = fma(2.0, dn, qc);
    lo = ext ? qc : (A ? lo2 : lo);
    hi = ext ? qc : (B ? hi2 : hi);
    int j = c - 3;
    if (j >= 0) right[j] = lo;
    if (j + 1 <= TE) left[j + 1] = hi;
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
// Writes Fhat_f to fout[f*fstride]; returns a.
__device__ __forceinline__ double kt_face64(const double* wl, const double* wr, int F, int d,
                                            double gamma, double inv_gm1, double* fout,
                                            int fstride) {
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
  double hl = ul + a, hr = ur - a;
  double gl = rl * hl, gr = rr * hr;
  fout[0] = dhalf(gl + gr);
  double pp = pl + pr;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    double t = fma(wl[1 + c], gl, wr[1 + c] * gr);
    fout[(1 + c) * fstride] = dhalf(c == d ? t + pp : t);
  }
  fout[4 * fstride] = dhalf(fma(El, hl, fma(pl, ul, fma(Er, hr, pr * ur))));
#pragma unroll
  for (int f = 5; f < MAXF; f++)
    if (f < F) fout[f * fstride] = dhalf(fma(wl[f], gl, wr[f] * gr));
  return a;
}

// ====================================================== binary32 (mixed) ==
// binary64 -> binary32, round to nearest even, on the integer pipe.
// Magnitudes below the smallest normal binary32 become signed zero; above
// the largest, infinity (such inputs are flagged as nonphysical anyway).
__device__ __forceinline__ float d2f_int(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  unsigned hi = (unsigned)(b >> 32);
  unsigned sg = hi & 0x80000000u, ahi = hi & 0x7fffffffu;
  unsigned long long m = (b & 0x7fffffffffffffffull) - (896ull << 52) + 0x0fffffffull + ((b >> 29) & 1ull);
  unsigned bits = (unsigned)(m >> 29) | sg;
  bits = ahi < (897u << 20) ? sg : bits;
  bits = ahi >= (1151u << 20) ? (sg | 0x7f800000u) : bits;
  return __uint_as_float(bits);
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

// tau^gamma in binary32 (gamma = 5/3: seed + one Halley step on w^3 = tau^2)
__device__ __forceinline__ float tau_pow32(float tau, float gamma, bool g53) {
  if (!g53 || !(tau > 1e-18f && tau < 1e18f)) return exp2f(gamma * __log2f(tau));
  float w = exp2f((2.0f / 3.0f) * __log2f(tau));
  float A = tau * tau;
  float w3 = w * w * w;
  w = w * fmaf(2.0f, A, w3) * rcp32(fmaf(2.0f, w3, A));
  return tau * w;
}

// ------------------------------------------------------ step A1, mixed --
// u: the binary64 hydro inputs of one cell (fields 0-5); writes binary32
// primitives and r = 1/rho.  Where e_int is within a factor 4 of E (where
// binary32 cancellation would cost more than ~20 ulp) or near the switch, it
// is recomputed in binary64 in the reference order.
__device__ __forceinline__ bool prim_mixed(const double* u, double gamma, float gm1f, bool g53,
                                           float* w, float& r) {
  float rho = d2f_int(u[0]);
  float s1 = d2f_int(u[1]), s2 = d2f_int(u[2]), s3 = d2f_int(u[3]);
  float E = d2f_int(u[4]), tau = d2f_int(u[5]);
  r = rcp32(rho);
  float ssq = fmaf(s3, s3, fmaf(s2, s2, s1 * s1));
  float eint = fmaf(-0.5f * ssq, r, E);
  float thr = (float)ETA * E;
  float p;
  if (eint > 0.5f * thr && eint < 0.25f * E) {  // near the switch, or too inexact in binary32
    double ss = __dadd_rn(__dadd_rn(__dmul_rn(u[1], u[1]), __dmul_rn(u[2], u[2])), __dmul_rn(u[3], u[3]));
    double ex = __dsub_rn(u[4], __ddiv_rn(__dmul_rn(0.5, ss), u[0]));
    double e = ex < __dmul_rn(ETA, u[4]) ? tau_pow64(u[5], gamma, g53) : ex;
    p = __double2float_rn((gamma - 1.0) * e);
  } else {
    float e = eint <= 0.5f * thr ? tau_pow32(tau, (float)gamma, g53) : eint;
    p = gm1f * e;
  }
  w[0] = rho;
  w[1] = s1 * r;
  w[2] = s2 * r;
  w[3] = s3 * r;
  w[4] = p;
  w[5] = tau * r;
  bool bad = !(rho > 0.0f) || !(p > 0.0f) || !isfinite(p);
#pragma unroll
  for (int f = 0; f < 6; f++) bad |= !dfinite(u[f]);
  return bad;
}

// ------------------------------------------------------ step A2, mixed --
__device__ __forceinline__ void ppm_line32(const float* q, float* left, float* right) {  // left/right: shared memory
  float dq[LL - 1];
#pragma unroll
  for (int c = 0; c < LL - 1; c++) dq[c] = q[c + 1] - q[c];
  float del[LL];
#pragma unroll
  for (int c = 1; c <= LL - 2; c++) {
    float dp = dq[c], dm = dq[c - 1];
    float dbar = 0.5f * (q[c + 1] - q[c - 1]);
    float m = fminf(fabsf(dbar), 2.0f * fminf(fabsf(dm), fabsf(dp)));
    bool mono = ((__float_as_int(dp) ^ __float_as_int(dm)) >= 0) && dp != 0.0f && dm != 0.0f;
    del[c] = mono ? copysignf(m, dbar) : 0.0f;
  }
  float fc[LL];
#pragma unroll
  for (int c = 1; c <= LL - 3; c++) fc[c] = fmaf(del[c] - del[c + 1], 1.0f / 6.0f, 0.5f * (q[c] + q[c + 1]));
#pragma unroll
  for (int c = 2; c <= LL - 3; c++) {
    float qc = q[c], lo = fc[c - 1], hi = fc[c];
    float up = hi - qc, dn = qc - lo;
    bool ext = !(((__float_as_int(up) ^ __float_as_int(dn)) >= 0) && up != 0.0f && dn != 0.0f);
    float D = up + dn, X = dn - up;
    float Y = D * X, Z = D * (D * (1.0f / 3.0f));
    bool A = Y > Z;
    bool B = !A && Y < -Z;
    float lo2 = fmaf(-2.0f, up, qc), hi2 = fmaf(2.0f, dn, qc);
    lo = ext ? qc : (A ? lo2 : lo);
    hi = ext ? qc : (B ? hi2 : hi);
    int j = c - 3;
    if (j >= 0) right[j] = lo;
    if (j + 1 <= TE) left[j + 1] = hi;
  }
}

// ------------------------------------------------------ step A3, mixed --
__device__ __forceinline__ float kt_face32(const float* wl, const float* wr, int F, int d,
                                           float gamma, float inv_gm1, float* fout, int fstride) {
  float rl = wl[0], rr = wr[0], pl = wl[4], pr = wr[4];
  float ul = d == 0 ? wl[1] : (d == 1 ? wl[2] : wl[3]);
  float ur = d == 0 ? wr[1] : (d == 1 ? wr[2] : wr[3]);
  float vl2 = fmaf(wl[3], wl[3], fmaf(wl[2], wl[2], wl[1] * wl[1]));
  float vr2 = fmaf(wr[3], wr[3], fmaf(wr[2], wr[2], wr[1] * wr[1]));
  float El = fmaf(0.5f * rl, vl2, pl * inv_gm1);
  float Er = fmaf(0.5f * rr, vr2, pr * inv_gm1);
  float gpl = gamma * pl, gpr = gamma * pr;
  float cl = gpl * rsqrtf(gpl * rl);
  float cr = gpr * rsqrtf(gpr * rr);
  float a = fmaxf(fabsf(ul) + cl, fabsf(ur) + cr);
  float hl = ul + a, hr = ur - a;
  float gl = rl * hl, gr = rr * hr;
  fout[0] = 0.5f * (gl + gr);
  float pp = pl + pr;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    float t = fmaf(wl[1 + c], gl, wr[1 + c] * gr);
    fout[(1 + c) * fstride] = 0.5f * (c == d ? t + pp : t);
  }
  fout[4 * fstride] = 0.5f * fmaf(El, hl, fmaf(pl, ul, fmaf(Er, hr, pr * ur)));
#pragma unroll
  for (int f = 5; f < MAXF; f++)
    if (f < F) fout[f * fstride] = 0.5f * fmaf(wl[f], gl, wr[f] * gr);
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
// running pair (H, L) += (hi - lo): the difference is split exactly, its high
// part is added with an exact two-sum, the low parts are summed in binary32
// (their rounding is ~2^-24 of a quantity already ~2^-24 smaller than H).
__device__ __forceinline__ void acc_pair(F2& acc, float hi, float lo, bool first) {
  F2 d = two_sum(hi, -lo);
  if (first) {
    acc = d;
  } else {
    F2 s = two_sum(acc.h, d.h);
    acc.h = s.h;
    acc.l = __fadd_rn(__fadd_rn(acc.l, d.l), s.l);
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

// ------------------------------------------------------------- kernel --
template <int MODE> struct Prec;
template <> struct Prec<0> { typedef double R; typedef double Acc; };
template <> struct Prec<1> { typedef float R; typedef F2 Acc; };

// Source of the tile descriptors: a prepared work list in global memory.
struct TileList {
  const Tile* __restrict__ tiles;
  __device__ __forceinline__ Tile operator()(int t) const { return tiles[t]; }
};

// Shared memory (R = element type of the mode):
//   W  [Fmax][STAR]          primitives of the read region
//   QS [2][Fmax][lch][NFC]   left/right face states, then fluxes in place
// The persistent tile loop; `fetch(t)` returns tile t's descriptor.
template <int MODE, int NT, class Fetch>
__device__ __forceinline__ void tile_loop(const Fetch& fetch, int n_tiles, int Fmax, int lch,
                                          double* __restrict__ out, double* __restrict__ amax_out,
                                          Status* __restrict__ status, double gamma_d,
                                          int write_status, int prefetch) {
  typedef typename Prec<MODE>::R R;
  typedef typename Prec<MODE>::Acc Acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* W = reinterpret_cast<R*>(smem_raw);
  R* QS = W + (size_t)Fmax * STAR;
  __shared__ double red[NT / 32];
  const int tid = threadIdx.x;
  const R gamma = R(gamma_d);
  const R inv_gm1 = R(1.0 / (gamma_d - 1.0));
  const float gm1f = (float)(gamma_d - 1.0);
  const bool g53 = gamma_d == 5.0 / 3.0;
  constexpr int CPT = (TE * TE * TE + NT - 1) / NT;  // owned cells per thread
  constexpr int SPT = (STAR + NT - 1) / NT;          // read-region slots per thread

  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const Tile tile = fetch(t);
    const int F = tile.F, G = tile.G, N = tile.N, gh = (tile.G - tile.N) >> 1;
    const int ex = min(TE, N - tile.ox), ey = min(TE, N - tile.oy), ez = min(TE, N - tile.oz);
    const long long plane = (long long)G * G * G;

    // ---- A0/A1: stage the read region as primitives.  Two passes over the
    // thread's slots (hydro fields, then species); in each pass every load is
    // issued before any result is used.
    bool bad = false;
    {
      int off[SPT];
      bool valid[SPT];
#pragma unroll
      for (int k = 0; k < SPT; k++) {
        int s = tid + k * NT;
        int x, y, z;
        cell_of(s < STAR ? s : 0, x, y, z);
        // read region of a (possibly partial) tile: at most one coordinate
        // outside the tile, and that one at most 3 cells out
        int outside = (x < 0 || x >= ex) + (y < 0 || y >= ey) + (z < 0 || z >= ez);
        valid[k] = s < STAR && outside <= 1 && x < ex + 3 && y < ey + 3 && z < ez + 3;
        off[k] = ((tile.oz + z + gh) * G + (tile.oy + y + gh)) * G + (tile.ox + x + gh);
      }
      R rr[SPT];
      constexpr int KC = 4;  // slots per load batch
#pragma unroll
      for (int k0 = 0; k0 < SPT; k0 += KC) {
        double u[KC][6];
#pragma unroll
        for (int kk = 0; kk < KC; kk++)
#pragma unroll
          for (int f = 0; f < 6; f++)
            if (k0 + kk < SPT && valid[k0 + kk]) u[kk][f] = __ldg(tile.U + f * plane + off[k0 + kk]);
#pragma unroll
        for (int kk = 0; kk < KC; kk++) {
          int k = k0 + kk;
          int s = tid + k * NT;
          if (k >= SPT || s >= STAR) continue;
          R w[6];
          if (valid[k]) {
            if constexpr (MODE == 0) {
              bad |= prim64(u[kk], gamma_d, g53, w, rr[k]);
            } else {
              bad |= prim_mixed(u[kk], gamma_d, gm1f, g53, w, rr[k]);
            }
          } else {
#pragma unroll
            for (int f = 0; f < 6; f++) w[f] = (f == 0 || f == 4) ? R(1) : R(0);
            rr[k] = R(1);
          }
#pragma unroll
          for (int f = 0; f < 6; f++) W[f * STAR + s] = w[f];
        }
      }
      if (F > 6) {
#pragma unroll
        for (int k0 = 0; k0 < SPT; k0 += KC) {
          double v[KC][MAXF - 6];
#pragma unroll
          for (int kk = 0; kk < KC; kk++)
#pragma unroll
            for (int f = 6; f < MAXF; f++)
              if (k0 + kk < SPT && valid[k0 + kk] && f < F)
                v[kk][f - 6] = __ldg(tile.U + f * plane + off[k0 + kk]);
#pragma unroll
          for (int kk = 0; kk < KC; kk++) {
            int k = k0 + kk;
            int s = tid + k * NT;
            if (k >= SPT || s >= STAR) continue;
#pragma unroll
            for (int f = 6; f < MAXF; f++)
              if (f < F) {
                R x = R(0);
                if (valid[k]) {
                  bad |= !dfinite(v[kk][f - 6]);
                  if constexpr (MODE == 0) x = v[kk][f - 6] * rr[k]; else x = d2f_int(v[kk][f - 6]) * rr[k];
                }
                W[f * STAR + s] = x;
              }
          }
        }
      }
    }
    bad = __syncthreads_or(bad);
    if (prefetch && t + (int)gridDim.x < n_tiles) prefetch_tile_l2(fetch(t + gridDim.x), tid, NT, prefetch);
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
      const int fs = lch * NFC;          // field stride of QS
      for (int l0 = 0; l0 < NLN; l0 += lch) {
        // ---- A2: PPM per (line, field)
        for (int task = tid; task < lch * F; task += NT) {
          int ll = task % lch, f = task / lch;
          int l = l0 + ll;
          R q[LL];
#pragma unroll
          for (int c = 0; c < LL; c++) q[c] = W[f * STAR + line_slot(d, l, c)];
          R* qs = QS + f * fs + ll * NFC;
          R* qr = QS + (Fmax + f) * fs + ll * NFC;
          if constexpr (MODE == 0) ppm_line64(q, qs, qr); else ppm_line32(q, qs, qr);
        }
        __syncthreads();
        // ---- A3: central flux per face, written over the left states
        for (int task = tid; task < lch * NFC; task += NT) {
          int ll = task / NFC, i = task - ll * NFC;
          int l = l0 + ll;
          R wl[MAXF], wr[MAXF];
          R* fo = QS + ll * NFC + i;
          const R* fr = fo + Fmax * fs;
#pragma unroll
          for (int f = 0; f < MAXF; f++)
            if (f < F) {
              wl[f] = fo[f * fs];
              wr[f] = fr[f * fs];
            }
          R a;
          if constexpr (MODE == 0) {
            a = kt_face64(wl, wr, F, d, gamma, inv_gm1, fo, fs);
          } else {
            a = kt_face32(wl, wr, F, d, gamma, inv_gm1, fo, fs);
          }
          bool fvalid = (l % TE) < e_a && (l / TE) < e_b && i <= e_d;
          if constexpr (MODE == 0) {
            if (fvalid) amax = dmaxp(amax, a);
          } else {
            if (fvalid) amax = fmaxf(amax, a);
          }
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
              const R* fl = QS + (l - l0) * NFC + pos;
#pragma unroll
              for (int f = 0; f < MAXF; f++)
                if (f < F) {
                  R hi = fl[f * fs + 1], lo = fl[f * fs];
                  if constexpr (MODE == 0) {
                    acc[k][f] = d == 0 ? hi - lo : acc[k][f] + (hi - lo);
                  } else {
                    acc_pair(acc[k][f], hi, lo, d == 0);
                  }
                }
            }
          }
        }
        __syncthreads();
      }
    }
    // ---- store dU/dt = -(sum of differences)/dx
    const long long n3 = (long long)N * N * N;
    const double scale = -tile.inv_dx;
    const bool pow2 = (tile.flags & 2) != 0;
#pragma unroll
    for (int k = 0; k < CPT; k++) {
      int m = tid + k * NT;
      if (m < TE * TE * TE) {
        int x = m % TE, y = (m / TE) % TE, z = m / (TE * TE);
        if (x < ex && y < ey && z < ez) {
          double* o = out + tile.out_off + ((long long)(tile.oz + z) * N + (tile.oy + y)) * N + (tile.ox + x);
#pragma unroll
          for (int f = 0; f < MAXF; f++)
            if (f < F) {
              double v;
              if constexpr (MODE == 0) {
                v = acc[k][f] * scale;
              } else {
                if (pow2) {  // scaling by a power of two is exact in binary32
                  float sf = (float)scale;
                  v = f2d_int(acc[k][f].h * sf) + f2d_int(acc[k][f].l * sf);
                } else {
                  v = (f2d_int(acc[k][f].h) + f2d_int(acc[k][f].l)) * scale;
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

template <int MODE, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
rhs_tiles_kernel(const Tile* __restrict__ tiles, int n_tiles, int Fmax, int lch,
                 double* __restrict__ out, double* __restrict__ amax_out,
                 Status* __restrict__ status, double gamma_d, int write_status, int prefetch) {
  tile_loop<MODE, NT>(TileList{tiles}, n_tiles, Fmax, lch, out, amax_out, status, gamma_d,
                      write_status, prefetch);
}

}  // namespace hydro_dev
