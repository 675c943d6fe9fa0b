/*
 * hydro_oracle.c -- plain, slow, obviously correct CPU reference of the
 * per-sub-grid hydro right-hand side (RHS).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * What it computes (Sec. IV-B of "From Task-Based GPU Work Aggregation to
 * Stellar Mergers"): the inviscid Euler equations (mass, momentum, energy)
 * discretised by finite volumes; cell values are reconstructed with the
 * piecewise-parabolic method (Colella & Woodward 1984, eqs. 1.6-1.10) and
 * face fluxes are evaluated with the central(-upwind) scheme of Kurganov &
 * Tadmor (2000); the largest signal speed feeds the Courant condition
 * (Sec. IV-B).  Each sub-grid carries a ghost layer of thickness 3 and
 * reconstruction/flux also cover the innermost ghost layer (Sec. V-A).
 *
 * The paper prints no formulas for the scheme, so the steps below are the
 * declared reading (face-centre, dimension-by-dimension; reconstruction of
 * primitives; CW84 slope and parabola limiters without steepening or
 * flattening; single-speed KT flux; dual-energy switch on the entropy tracer
 * tau with eta = 1e-3).  Each function names the step it follows.
 *
 * Evaluation order is fixed and written out; compile with
 *   -O2 -ffp-contract=off
 * so that no multiply-add is fused.  The mixed mode (mode 1) forms the
 * primitives in binary32 from the binary32-rounded conserved values (the
 * internal energy and the dual-energy switch stay binary64; see
 * primitives_mixed), runs steps 2-3 in IEEE binary32 and step 4 in binary64.
 *
 * Layout: U[f][k][j][i] with i (x) fastest; a block has interior nx*ny*nz
 * cells and `ghost` >= 3 ghost layers on every side (only the innermost 3 are
 * read).  Output dUdt[f][k][j][i] over the interior only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_ETA 1e-3 /* dual-energy switch threshold (declared reading) */
#define ORA_MAXF 16
#define ORA_MAXN 4096

/* status bits returned by ora_rhs_block */
#define ORA_NONPHYS 1 /* rho <= 0, p <= 0 or a non-finite value in the read region */
#define ORA_EINVAL 2

typedef struct {
  int nx, ny, nz;   /* interior cells per axis */
  int gh;           /* ghost layers stored */
  int gx, gy, gz;   /* stored extents nx+2gh ... */
  int nf;           /* fields */
} ora_geom;

static size_t at(const ora_geom* g, int f, int i, int j, int k) {
  /* i, j, k are interior coordinates; -gh <= i < nx+gh */
  return (((size_t)f * g->gz + (size_t)(k + g->gh)) * g->gy + (size_t)(j + g->gh)) * g->gx +
         (size_t)(i + g->gh);
}

/* A cell is read by the scheme iff at most one of its coordinates lies outside
 * the interior and that one is within 3 cells of it (the "star" region:
 * lines of 3 ghost cells on each side of every interior line). */
static int in_star(const ora_geom* g, int i, int j, int k) {
  int n[3] = {g->nx, g->ny, g->nz}, c[3] = {i, j, k}, out = 0;
  for (int d = 0; d < 3; d++) {
    if (c[d] < -3 || c[d] >= n[d] + 3) return 0;
    if (c[d] < 0 || c[d] >= n[d]) out++;
  }
  return out <= 1;
}

/* The 26-point variant reads every cell within 3 of the interior along its
 * face-normal axis and within 2 along the other two: each coordinate in
 * [-3, n+2] with at most one of them at -3 or n+2 (the stencils of the
 * lines through the cells next to interior faces, see quad26_face). */
static int in_read26(const ora_geom* g, int i, int j, int k) {
  int n[3] = {g->nx, g->ny, g->nz}, c[3] = {i, j, k}, far = 0;
  for (int d = 0; d < 3; d++) {
    if (c[d] < -3 || c[d] > n[d] + 2) return 0;
    if (c[d] == -3 || c[d] == n[d] + 2) far++;
  }
  return far <= 1;
}

/* ---------------------------------------------------------------- step 1 --
 * Conserved -> primitive variables (declared reading; the paper names the
 * conserved quantities only).  Fields: 0 rho, 1..3 momentum s, 4 total energy
 * E, 5 entropy tracer tau = (rho*eps)^(1/gamma), 6.. species densities.
 * Primitives: rho, v = s/rho, p, phi = tau/rho, X_k = rho_k/rho.
 * Internal energy e = E - |s|^2/(2 rho); if e < eta*E the tracer is used
 * instead: e = tau^gamma.  p = (gamma-1) e.  Returns 1 if nonphysical. */
static int primitives(const double* u, int nf, double gamma, double* w) {
  double rho = u[0];
  double s1 = u[1], s2 = u[2], s3 = u[3], E = u[4], tau = u[5];
  double ssq = (s1 * s1 + s2 * s2) + s3 * s3;
  double ekin = (0.5 * ssq) / rho;
  double eint = E - ekin;
  if (eint < ORA_ETA * E) eint = pow(tau, gamma);
  double p = (gamma - 1.0) * eint;
  w[0] = rho;
  w[1] = s1 / rho;
  w[2] = s2 / rho;
  w[3] = s3 / rho;
  w[4] = p;
  w[5] = tau / rho;
  for (int f = 6; f < nf; f++) w[f] = u[f] / rho;
  int bad = !(rho > 0.0) || !(p > 0.0);
  for (int f = 0; f < nf; f++)
    if (!isfinite(u[f]) || !isfinite(w[f])) bad = 1;
  return bad;
}

/* Step 1 of the mixed mode (declared reading): the conserved values are
 * rounded to binary32 (C's conversion: to nearest, ties to even); rho,
 * v = s/rho, phi = tau/rho and X_k = rho_k/rho are formed from them in
 * binary32 (one binary32 division each); the internal energy and the
 * dual-energy switch are those of `primitives` on the binary64 inputs, and
 * p = (gamma-1) e is rounded to binary32.  w receives the binary32 values
 * (exactly, as doubles).  Returns 1 if nonphysical. */
static int primitives_mixed(const double* u, int nf, double gamma, double* w) {
  double w64[ORA_MAXF];
  int bad = primitives(u, nf, gamma, w64); /* e, the switch and p in binary64 */
  float q[ORA_MAXF];
  for (int f = 0; f < nf; f++) q[f] = (float)u[f];
  float rho = q[0];
  w[0] = rho;
  w[1] = q[1] / rho;
  w[2] = q[2] / rho;
  w[3] = q[3] / rho;
  w[4] = (float)w64[4];
  w[5] = q[5] / rho;
  for (int f = 6; f < nf; f++) w[f] = q[f] / rho;
  for (int f = 0; f < nf; f++)
    if (!isfinite(w[f])) bad = 1;
  return bad;
}

/* ---------------------------------------------------------------- step 2 --
 * PPM along one line (Colella & Woodward 1984).  q[c] holds cell c-3 of the
 * line, c = 0 .. n+5.  Outputs for cells j = -1 .. n (stored at j+1); delta and
 * face are work arrays of n+6 entries:
 *   qm[j+1] = value at the left face of cell j, qp[j+1] = at its right face.
 *
 *  slope (CW84 eq. 1.7-1.8): dbar_j = (q_{j+1} - q_{j-1})/2 ;
 *    if (q_{j+1}-q_j)(q_j-q_{j-1}) > 0, i.e. both non-zero with the same sign
 *      delta_j = sgn(dbar_j) min(|dbar_j|, 2|q_j-q_{j-1}|, 2|q_{j+1}-q_j|)
 *    else delta_j = 0
 *  face (CW84 eq. 1.6, uniform grid):
 *    q_{j+1/2} = (q_j + q_{j+1})/2 - (delta_{j+1} - delta_j)/6
 *  parabola limiter (CW84 eq. 1.10):
 *    if (q+ - q)(q - q-) <= 0 : q- = q+ = q   (tested on the signs of the two
 *      factors, so that an underflowing product cannot change the branch)
 *    else with D = q+ - q-, m = q - (q- + q+)/2 :
 *      D*m >  D*D/6 : q- = 3q - 2q+
 *      D*m < -D*D/6 : q+ = 3q - 2q-
 */
static void ppm_line_d(const double* q, int n, double* qm, double* qp, double* delta,
                       double* face) {
  /* delta for cells j = -2 .. n+1 -> index c = j+3 in 1 .. n+4 */
  for (int c = 1; c <= n + 4; c++) {
    double dp = q[c + 1] - q[c];
    double dm = q[c] - q[c - 1];
    double dbar = 0.5 * (q[c + 1] - q[c - 1]);
    if ((dp > 0.0 && dm > 0.0) || (dp < 0.0 && dm < 0.0)) {
      double m = fmin(fabs(dbar), fmin(2.0 * fabs(dm), 2.0 * fabs(dp)));
      delta[c] = copysign(m, dbar);
    } else {
      delta[c] = 0.0;
    }
  }
  /* face j+1/2 for j = -2 .. n  (c = j+3 in 1 .. n+3): face[c] between c, c+1 */
  for (int c = 1; c <= n + 3; c++)
    face[c] = 0.5 * (q[c] + q[c + 1]) - (delta[c + 1] - delta[c]) / 6.0;
  /* cells j = -1 .. n (c = 2 .. n+3) */
  for (int c = 2; c <= n + 3; c++) {
    double qc = q[c], lo = face[c - 1], hi = face[c];
    double up = hi - qc, dn = qc - lo;
    if (!((up > 0.0 && dn > 0.0) || (up < 0.0 && dn < 0.0))) { /* local extremum */
      lo = qc;
      hi = qc;
    } else {
      double D = hi - lo;
      double m = qc - 0.5 * (lo + hi);
      double D2 = D * D / 6.0;
      if (D * m > D2)
        lo = 3.0 * qc - 2.0 * hi;
      else if (D * m < -D2)
        hi = 3.0 * qc - 2.0 * lo;
    }
    qm[c - 2] = lo;
    qp[c - 2] = hi;
  }
}

/* the same steps in binary32 (mixed mode) */
static void ppm_line_f(const float* q, int n, float* qm, float* qp, float* delta, float* face) {
  for (int c = 1; c <= n + 4; c++) {
    float dp = q[c + 1] - q[c];
    float dm = q[c] - q[c - 1];
    float dbar = 0.5f * (q[c + 1] - q[c - 1]);
    if ((dp > 0.0f && dm > 0.0f) || (dp < 0.0f && dm < 0.0f)) {
      float m = fminf(fabsf(dbar), fminf(2.0f * fabsf(dm), 2.0f * fabsf(dp)));
      delta[c] = copysignf(m, dbar);
    } else {
      delta[c] = 0.0f;
    }
  }
  for (int c = 1; c <= n + 3; c++)
    face[c] = 0.5f * (q[c] + q[c + 1]) - (delta[c + 1] - delta[c]) / 6.0f;
  for (int c = 2; c <= n + 3; c++) {
    float qc = q[c], lo = face[c - 1], hi = face[c];
    float up = hi - qc, dn = qc - lo;
    if (!((up > 0.0f && dn > 0.0f) || (up < 0.0f && dn < 0.0f))) { /* local extremum */
      lo = qc;
      hi = qc;
    } else {
      float D = hi - lo;
      float m = qc - 0.5f * (lo + hi);
      float D2 = D * D / 6.0f;
      if (D * m > D2)
        lo = 3.0f * qc - 2.0f * hi;
      else if (D * m < -D2)
        hi = 3.0f * qc - 2.0f * lo;
    }
    qm[c - 2] = lo;
    qp[c - 2] = hi;
  }
}

/* ---------------------------------------------------------------- step 3 --
 * Central flux of Kurganov & Tadmor (2000) at one face normal to axis d:
 *   left state wl = q+ of the cell on the low side, right wr = q- of the
 *   cell on the high side (primitives).  For each side:
 *     E = p/(gamma-1) + rho|v|^2/2,  U = (rho, rho v, E, rho phi, rho X_k)
 *     F = (rho u, rho v u + p e_d, (E + p) u, rho phi u, rho X_k u), u = v_d
 *     c = sqrt(gamma p / rho)
 *   a = max(|u_l| + c_l, |u_r| + c_r)
 *   Fhat = (F_l + F_r)/2 - a (U_r - U_l)/2
 * Returns a. */
static void cons_flux_d(const double* w, int nf, int d, double gamma, double* U, double* F,
                        double* speed, double* un, double* cs) {
  double rho = w[0], vx = w[1], vy = w[2], vz = w[3], p = w[4];
  double v[3] = {vx, vy, vz};
  double u = v[d];
  double vsq = (vx * vx + vy * vy) + vz * vz;
  double E = p / (gamma - 1.0) + 0.5 * rho * vsq;
  U[0] = rho;
  U[1] = rho * vx;
  U[2] = rho * vy;
  U[3] = rho * vz;
  U[4] = E;
  U[5] = rho * w[5];
  for (int f = 6; f < nf; f++) U[f] = rho * w[f];
  F[0] = rho * u;
  for (int c = 0; c < 3; c++) F[1 + c] = U[1 + c] * u + (c == d ? p : 0.0);
  F[4] = (E + p) * u;
  for (int f = 5; f < nf; f++) F[f] = U[f] * u;
  *cs = sqrt(gamma * p / rho);
  *un = u;
  *speed = fabs(u) + *cs;
}

static double kt_flux_d(const double* wl, const double* wr, int nf, int d, double gamma,
                        double* fhat) {
  double Ul[ORA_MAXF], Fl[ORA_MAXF], Ur[ORA_MAXF], Fr[ORA_MAXF], al, ar, ul, ur, cl, cr;
  cons_flux_d(wl, nf, d, gamma, Ul, Fl, &al, &ul, &cl);
  cons_flux_d(wr, nf, d, gamma, Ur, Fr, &ar, &ur, &cr);
  double a = fmax(al, ar);
  for (int f = 0; f < nf; f++) fhat[f] = 0.5 * (Fl[f] + Fr[f]) - 0.5 * a * (Ur[f] - Ul[f]);
  return a;
}

/* Central-upwind flux with one-sided local speeds (Kurganov, Noelle &
 * Petrova 2001):
 *   ap = max(u_l + c_l, u_r + c_r, 0),  am = min(u_l - c_l, u_r - c_r, 0)
 *   Fhat = (ap F_l - am F_r)/(ap - am) + ap am (U_r - U_l)/(ap - am)
 * (if ap = am = 0, Fhat = (F_l + F_r)/2).  The signal speed returned for the
 * Courant condition is max(ap, -am) = max(|u_l| + c_l, |u_r| + c_r). */
static double knp_flux_d(const double* wl, const double* wr, int nf, int d, double gamma,
                         double* fhat) {
  double Ul[ORA_MAXF], Fl[ORA_MAXF], Ur[ORA_MAXF], Fr[ORA_MAXF], al, ar, ul, ur, cl, cr;
  cons_flux_d(wl, nf, d, gamma, Ul, Fl, &al, &ul, &cl);
  cons_flux_d(wr, nf, d, gamma, Ur, Fr, &ar, &ur, &cr);
  double ap = fmax(fmax(ul + cl, ur + cr), 0.0);
  double am = fmin(fmin(ul - cl, ur - cr), 0.0);
  double den = ap - am;
  for (int f = 0; f < nf; f++) {
    if (den > 0.0)
      fhat[f] = (ap * Fl[f] - am * Fr[f]) / den + ap * am * (Ur[f] - Ul[f]) / den;
    else
      fhat[f] = 0.5 * (Fl[f] + Fr[f]);
  }
  return fmax(al, ar);
}

static void cons_flux_f(const float* w, int nf, int d, float gamma, float* U, float* F,
                        float* speed, float* un, float* cs) {
  float rho = w[0], vx = w[1], vy = w[2], vz = w[3], p = w[4];
  float v[3] = {vx, vy, vz};
  float u = v[d];
  float vsq = (vx * vx + vy * vy) + vz * vz;
  float E = p / (gamma - 1.0f) + 0.5f * rho * vsq;
  U[0] = rho;
  U[1] = rho * vx;
  U[2] = rho * vy;
  U[3] = rho * vz;
  U[4] = E;
  U[5] = rho * w[5];
  for (int f = 6; f < nf; f++) U[f] = rho * w[f];
  F[0] = rho * u;
  for (int c = 0; c < 3; c++) F[1 + c] = U[1 + c] * u + (c == d ? p : 0.0f);
  F[4] = (E + p) * u;
  for (int f = 5; f < nf; f++) F[f] = U[f] * u;
  *cs = sqrtf(gamma * p / rho);
  *un = u;
  *speed = fabsf(u) + *cs;
}

static float kt_flux_f(const float* wl, const float* wr, int nf, int d, float gamma,
                       float* fhat) {
  float Ul[ORA_MAXF], Fl[ORA_MAXF], Ur[ORA_MAXF], Fr[ORA_MAXF], al, ar, ul, ur, cl, cr;
  cons_flux_f(wl, nf, d, gamma, Ul, Fl, &al, &ul, &cl);
  cons_flux_f(wr, nf, d, gamma, Ur, Fr, &ar, &ur, &cr);
  float a = fmaxf(al, ar);
  for (int f = 0; f < nf; f++) fhat[f] = 0.5f * (Fl[f] + Fr[f]) - 0.5f * a * (Ur[f] - Ul[f]);
  return a;
}

static float knp_flux_f(const float* wl, const float* wr, int nf, int d, float gamma,
                        float* fhat) {
  float Ul[ORA_MAXF], Fl[ORA_MAXF], Ur[ORA_MAXF], Fr[ORA_MAXF], al, ar, ul, ur, cl, cr;
  cons_flux_f(wl, nf, d, gamma, Ul, Fl, &al, &ul, &cl);
  cons_flux_f(wr, nf, d, gamma, Ur, Fr, &ar, &ur, &cr);
  float ap = fmaxf(fmaxf(ul + cl, ur + cr), 0.0f);
  float am = fminf(fminf(ul - cl, ur - cr), 0.0f);
  float den = ap - am;
  for (int f = 0; f < nf; f++) {
    if (den > 0.0f)
      fhat[f] = (ap * Fl[f] - am * Fr[f]) / den + ap * am * (Ur[f] - Ul[f]) / den;
    else
      fhat[f] = 0.5f * (Fl[f] + Fr[f]);
  }
  return fmaxf(al, ar);
}

/* ------------------------------------------------ 26-point variant --
 * Sec. IV-B: PPM values at 26 points on the surface of each cell (the
 * centres of its 6 faces, the midpoints of its 12 edges and its 8
 * vertices), central-upwind fluxes at those points, and Newton-Cotes
 * quadrature of the fluxes over each face.  Declared reading: the value of
 * cell c at its surface point c + v/2 (v in {-1,0,1}^3, v != 0) is the PPM
 * face value of the one-dimensional reconstruction along the line of cells
 * c + m v, i.e. ppm_line on that line (cell c depends on cells m = -2..2
 * only).  A face normal to axis d has the 9 points v = e_d + o1 e_a + o2 e_b
 * (o1, o2 in {-1, 0, 1}); at each one the left state is the low cell's value
 * there (its line along v, upper end) and the right state the high cell's
 * value there (its line along e_d - o1 e_a - o2 e_b, lower end).  The face
 * flux is Simpson's rule in both tangential directions,
 *   Fhat = sum_p c_p Fhat_p / 36,  c_p = (1, 4, 1) x (1, 4, 1),
 * and the signal speed is the largest over all points. */
static void ppm_cell_d(const double* W, const ora_geom* g, int f, const int* c, const int* v,
                       double* qm, double* qp) {
  double q[7], lm[3], lp[3], work[14];
  for (int m = -2; m <= 2; m++)
    q[m + 3] = W[at(g, f, c[0] + m * v[0], c[1] + m * v[1], c[2] + m * v[2])];
  q[0] = q[1]; /* cells -3 and +3 of the line do not enter cell 0 */
  q[6] = q[5];
  ppm_line_d(q, 1, lm, lp, work, work + 7);
  *qm = lm[1];
  *qp = lp[1];
}

static void ppm_cell_f(const double* W, const ora_geom* g, int f, const int* c, const int* v,
                       float* qm, float* qp) {
  float q[7], lm[3], lp[3], work[14];
  for (int m = -2; m <= 2; m++)
    q[m + 3] = (float)W[at(g, f, c[0] + m * v[0], c[1] + m * v[1], c[2] + m * v[2])];
  q[0] = q[1];
  q[6] = q[5];
  ppm_line_f(q, 1, lm, lp, work, work + 7);
  *qm = lm[1];
  *qp = lp[1];
}

/* Flux through the face between cell cl and cl + e_d (mode as in
 * ora_rhs_block); returns the largest signal speed of its 9 points. */
static double quad26_face(const double* W, const ora_geom* g, int nf, int d, const int* cl,
                          double gamma, int mode, int knp, double* fhat) {
  const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
  int cr[3] = {cl[0], cl[1], cl[2]};
  cr[d] += 1;
  double acc_d[ORA_MAXF] = {0};
  float acc_f[ORA_MAXF] = {0};
  double amax = 0.0;
  float amax_f = 0.0f;
  for (int o2 = -1; o2 <= 1; o2++)
    for (int o1 = -1; o1 <= 1; o1++) {
      int vl[3] = {0, 0, 0}, vr[3] = {0, 0, 0};
      vl[d] = 1, vl[t1] = o1, vl[t2] = o2;
      vr[d] = 1, vr[t1] = -o1, vr[t2] = -o2;
      const int cw = (o1 == 0 ? 4 : 1) * (o2 == 0 ? 4 : 1);
      if (mode == 0) {
        double wl[ORA_MAXF], wr[ORA_MAXF], fh[ORA_MAXF], lo, hi;
        for (int f = 0; f < nf; f++) {
          ppm_cell_d(W, g, f, cl, vl, &lo, &hi);
          wl[f] = hi;
          ppm_cell_d(W, g, f, cr, vr, &lo, &hi);
          wr[f] = lo;
        }
        double sp = knp ? knp_flux_d(wl, wr, nf, d, gamma, fh) : kt_flux_d(wl, wr, nf, d, gamma, fh);
        if (!(sp <= amax)) amax = sp;
        for (int f = 0; f < nf; f++) acc_d[f] += cw * fh[f];
      } else {
        float wl[ORA_MAXF], wr[ORA_MAXF], fh[ORA_MAXF], lo, hi;
        for (int f = 0; f < nf; f++) {
          ppm_cell_f(W, g, f, cl, vl, &lo, &hi);
          wl[f] = hi;
          ppm_cell_f(W, g, f, cr, vr, &lo, &hi);
          wr[f] = lo;
        }
        float sp = knp ? knp_flux_f(wl, wr, nf, d, (float)gamma, fh)
                       : kt_flux_f(wl, wr, nf, d, (float)gamma, fh);
        if (!(sp <= amax_f)) amax_f = sp;
        for (int f = 0; f < nf; f++) acc_f[f] += (float)cw * fh[f];
      }
    }
  for (int f = 0; f < nf; f++) fhat[f] = mode == 0 ? acc_d[f] / 36.0 : (double)(acc_f[f] / 36.0f);
  return mode == 0 ? amax : (double)amax_f;
}

/* --------------------------------------------------------- steps 1 - 5 --
 * One block (a sub-grid, or any nx*ny*nz box used by the tests).
 *   mode bit 0: 0 all binary64, 1 steps 2-3 in binary32 and step 4 binary64.
 *   mode bit 1: 0 Kurganov-Tadmor flux, 1 Kurganov-Noelle-Petrova flux.
 *   mode bit 2: 0 face-centre fluxes, 1 the 26-point variant (quad26_face).
 * face_out (optional, may be NULL): receives the face fluxes as doubles,
 *   x faces [nf][nz][ny][nx+1], then y faces [nf][nz][ny+1][nx], then z
 *   faces [nf][nz+1][ny][nx].
 * Returns a bit set of ORA_* flags; outputs are written in every case. */
int ora_rhs_block(const double* U, int nx, int ny, int nz, int ghost, int nf, double gamma,
                  double dx, int mode, double* dUdt, double* amax_out, double* face_out) {
  if (nx < 1 || ny < 1 || nz < 1 || nx > ORA_MAXN || ny > ORA_MAXN || nz > ORA_MAXN || ghost < 3 || nf < 6 ||
      nf > ORA_MAXF || !(gamma > 1.0) || !(dx > 0.0) || mode < 0 || mode > 7)
    return ORA_EINVAL;
  ora_geom g = {nx, ny, nz, ghost, nx + 2 * ghost, ny + 2 * ghost, nz + 2 * ghost, nf};
  const int knp = (mode >> 1) & 1;
  const int q26 = (mode >> 2) & 1;
  mode &= 1;
  int flags = 0;
  size_t ncell = (size_t)g.gx * g.gy * g.gz;

  /* step 1 over the star region; W[f][cell] in the same indexing as U (in
   * mode 1 the binary32 primitives, held exactly as doubles) */
  double* W = (double*)calloc((size_t)nf * ncell, sizeof(double));
  for (int k = -3; k < nz + 3; k++)
    for (int j = -3; j < ny + 3; j++)
      for (int i = -3; i < nx + 3; i++) {
        if (!(q26 ? in_read26(&g, i, j, k) : in_star(&g, i, j, k))) continue;
        double u[ORA_MAXF], w[ORA_MAXF];
        for (int f = 0; f < nf; f++) u[f] = U[at(&g, f, i, j, k)];
        flags |= (mode == 1 ? primitives_mixed(u, nf, gamma, w) : primitives(u, nf, gamma, w)) ? ORA_NONPHYS : 0;
        for (int f = 0; f < nf; f++) W[at(&g, f, i, j, k)] = w[f];
      }

  /* face flux storage per direction (as double; in mode 1 they hold the
   * binary32 values exactly) */
  int n[3] = {nx, ny, nz};
  size_t nface[3];
  double* FH[3];
  for (int d = 0; d < 3; d++) {
    size_t m = 1;
    for (int e = 0; e < 3; e++) m *= (size_t)(n[e] + (e == d ? 1 : 0));
    nface[d] = m;
    FH[d] = (double*)calloc((size_t)nf * m, sizeof(double));
  }
  double amax = 0.0;
  float amax_f = 0.0f;
  int nmax = nx > ny ? nx : ny;
  if (nz > nmax) nmax = nz;
  size_t L = (size_t)nmax + 6; /* line buffers */
  double* lbuf_d = (double*)malloc(3 * (size_t)nf * L * sizeof(double));
  float* lbuf_f = (float*)malloc(3 * (size_t)nf * L * sizeof(float));
  double* work_d = (double*)malloc(2 * L * sizeof(double));
  float* work_f = (float*)malloc(2 * L * sizeof(float));

  /* steps 2-3, 26-point variant: every face of an interior cell */
  for (int d = 0; q26 && d < 3; d++) {
    int ext[3] = {n[0] + (d == 0), n[1] + (d == 1), n[2] + (d == 2)};
    for (int k = 0; k < ext[2]; k++)
      for (int j = 0; j < ext[1]; j++)
        for (int i = 0; i < ext[0]; i++) {
          int cl[3] = {i, j, k};
          cl[d] -= 1; /* face i-1/2 along d: low cell i-1 */
          double fh[ORA_MAXF];
          double sp = quad26_face(W, &g, nf, d, cl, gamma, mode, knp, fh);
          if (mode == 0 ? !(sp <= amax) : !((float)sp <= amax_f)) {
            if (mode == 0) amax = sp; else amax_f = (float)sp;
          }
          if (!isfinite(sp)) flags |= ORA_NONPHYS;
          size_t fidx = ((size_t)k * ext[1] + (size_t)j) * ext[0] + (size_t)i;
          for (int f = 0; f < nf; f++) FH[d][(size_t)f * nface[d] + fidx] = fh[f];
        }
  }

  /* steps 2-3: for each direction and each interior line along it */
  for (int d = 0; !q26 && d < 3; d++) {
    int nd = n[d];
    int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2; /* tangential axes */
    for (int b = 0; b < n[t2]; b++)
      for (int a = 0; a < n[t1]; a++) {
        double *qd[ORA_MAXF], *qmd[ORA_MAXF], *qpd[ORA_MAXF];
        float *qf[ORA_MAXF], *qmf[ORA_MAXF], *qpf[ORA_MAXF];
        for (int f = 0; f < nf; f++) {
          qd[f] = lbuf_d + (size_t)(3 * f + 0) * L;
          qmd[f] = lbuf_d + (size_t)(3 * f + 1) * L;
          qpd[f] = lbuf_d + (size_t)(3 * f + 2) * L;
          qf[f] = lbuf_f + (size_t)(3 * f + 0) * L;
          qmf[f] = lbuf_f + (size_t)(3 * f + 1) * L;
          qpf[f] = lbuf_f + (size_t)(3 * f + 2) * L;
        }
        for (int c = 0; c < nd + 6; c++) {
          int cc[3];
          cc[d] = c - 3;
          cc[t1] = a;
          cc[t2] = b;
          for (int f = 0; f < nf; f++) {
            double v = W[at(&g, f, cc[0], cc[1], cc[2])];
            qd[f][c] = v;
            qf[f][c] = (float)v;
          }
        }
        for (int f = 0; f < nf; f++) {
          if (mode == 0)
            ppm_line_d(qd[f], nd, qmd[f], qpd[f], work_d, work_d + L);
          else
            ppm_line_f(qf[f], nd, qmf[f], qpf[f], work_f, work_f + L);
        }
        /* faces i-1/2, i = 0 .. nd: left cell i-1 (row i), right cell i (row i+1) */
        for (int i = 0; i <= nd; i++) {
          int fc[3];
          fc[d] = i;
          fc[t1] = a;
          fc[t2] = b;
          int ext[3] = {n[0] + (d == 0), n[1] + (d == 1), n[2] + (d == 2)};
          size_t fidx = ((size_t)fc[2] * ext[1] + (size_t)fc[1]) * ext[0] + (size_t)fc[0];
          if (mode == 0) {
            double wl[ORA_MAXF], wr[ORA_MAXF], fh[ORA_MAXF];
            for (int f = 0; f < nf; f++) {
              wl[f] = qpd[f][i];
              wr[f] = qmd[f][i + 1];
            }
            double sp = knp ? knp_flux_d(wl, wr, nf, d, gamma, fh) : kt_flux_d(wl, wr, nf, d, gamma, fh);
            if (sp > amax) amax = sp;
            if (!isfinite(sp)) flags |= ORA_NONPHYS;
            for (int f = 0; f < nf; f++) FH[d][(size_t)f * nface[d] + fidx] = fh[f];
          } else {
            float wl[ORA_MAXF], wr[ORA_MAXF], fh[ORA_MAXF];
            for (int f = 0; f < nf; f++) {
              wl[f] = qpf[f][i];
              wr[f] = qmf[f][i + 1];
            }
            float sp = knp ? knp_flux_f(wl, wr, nf, d, (float)gamma, fh)
                           : kt_flux_f(wl, wr, nf, d, (float)gamma, fh);
            if (sp > amax_f) amax_f = sp;
            if (!isfinite(sp)) flags |= ORA_NONPHYS;
            for (int f = 0; f < nf; f++) FH[d][(size_t)f * nface[d] + fidx] = (double)fh[f];
          }
        }
      }
  }
  if (mode == 1) amax = (double)amax_f;

  /* step 4: dU/dt = -((Dx + Dy) + Dz) / dx in binary64 */
  for (int f = 0; f < nf; f++)
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
          const double* fx = FH[0] + (size_t)f * nface[0];
          const double* fy = FH[1] + (size_t)f * nface[1];
          const double* fz = FH[2] + (size_t)f * nface[2];
          double Dx = fx[((size_t)k * ny + j) * (nx + 1) + i + 1] - fx[((size_t)k * ny + j) * (nx + 1) + i];
          double Dy = fy[((size_t)k * (ny + 1) + j + 1) * nx + i] - fy[((size_t)k * (ny + 1) + j) * nx + i];
          double Dz = fz[((size_t)(k + 1) * ny + j) * nx + i] - fz[((size_t)k * ny + j) * nx + i];
          dUdt[(((size_t)f * nz + k) * ny + j) * nx + i] = -((Dx + Dy) + Dz) / dx;
        }
  /* step 5 */
  *amax_out = amax;

  if (face_out) {
    size_t off = 0;
    for (int d = 0; d < 3; d++) {
      memcpy(face_out + off, FH[d], (size_t)nf * nface[d] * sizeof(double));
      off += (size_t)nf * nface[d];
    }
  }
  for (int d = 0; d < 3; d++) free(FH[d]);
  free(W);
  free(lbuf_d);
  free(lbuf_f);
  free(work_d);
  free(work_f);
  return flags;
}

/* A batch of cubic sub-grids, one per task, run by OpenMP threads over the
 * sub-grids (the CPU decomposition of Sec. V-A: one sub-grid per core at a
 * time).  U[s] points at sub-grid s ([nf_s][G][G][G], G = N_s + 2 ghost);
 * out[s] at its [nf_s][N_s]^3 result.  flags[s] receives the block flags. */
int ora_rhs_batch(const double* const* U, const int* N, const int* nf, const double* dx,
                  int64_t n, int ghost, double gamma, int mode, double* const* out, double* amax,
                  int* flags, int nthreads) {
  int any = 0;
#if defined(_OPENMP)
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) reduction(| : any)
#endif
  for (int64_t s = 0; s < n; s++) {
    int fl = ora_rhs_block(U[s], N[s], N[s], N[s], ghost, nf[s], gamma, dx[s], mode, out[s],
                           &amax[s], NULL);
    flags[s] = fl;
    any |= fl;
  }
  (void)nthreads;
  return any;
}

int ora_max_threads(void) {
#if defined(_OPENMP)
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
