/*
 * Oracle for the real spherical harmonics R_l^m and the fused projectors.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this code.  The
 * product path (libshm and its kernels) never links, includes or calls it,
 * and it includes nothing from the product path.
 *
 * Plain, slow, obviously correct FP64 code written from the definitions of
 * "SHarmonic: A fast and accurate implementation of spherical harmonics for
 * electronic-structure calculations" (arXiv 2510.05282):
 *
 *   Sec. II, Eq. 3-4   theta = angle from +z, phi = atan2(y, x).
 *                      theta is taken as atan2(rho, z), rho = sqrt(x^2+y^2),
 *                      which is the same angle as acos(z/r) but keeps full
 *                      precision next to the poles.
 *   Sec. II, Eq. 5     Y_l^m = (-1)^m N_l^m P_l^m(cos theta) e^{i m phi}, m >= 0,
 *                      N_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), where P_l^m
 *                      is the associated Legendre function WITHOUT its own
 *                      Condon-Shortley sign (the (-1)^m is written explicitly).
 *   Sec. III, Eq. 10   Y_l^{-m} = (-1)^m (Y_l^m)^*  (used for negative m).
 *   Sec. II, Eq. 6     R_l^m from Y_l^{+-m}.
 *   Sec. II, Eq. 7     spinor harmonics (spin 1/2) from the complex Y_l^m.
 *   Sec. II            at r = 0 every harmonic is 0 except l = 0, which is the
 *                      constant 1/sqrt(4 pi).
 *
 * P_l^m is computed by the textbook three-term recurrence in l for fixed m:
 *   P_m^m     = (2m-1)!! sin^m(theta)
 *   P_{m+1}^m = (2m+1) cos(theta) P_m^m
 *   (l-m) P_l^m = (2l-1) cos(theta) P_{l-1}^m - (l+m-1) P_{l-2}^m.
 *
 * Output layout: row-major [n, (lmax+1)^2], column k = l*l + l + m with m
 * ascending from -l to l (the appendix lists each l from m = -l upwards).
 *
 * Non-finite inputs are not special-cased: NaN propagates.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_LMAX_CAP 16
#define ORACLE_PI 3.14159265358979323846264338327950288

/* n! (exact in binary64 up to 18!; one rounding beyond, up to 32! for l = 16). */
static double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= (double)i;
  return f;
}

/* N_l^m of Eq. 5 for m >= 0. */
static double norm_lm(int l, int m) {
  return sqrt((2.0 * l + 1.0) / (4.0 * ORACLE_PI) * factorial(l - m) / factorial(l + m));
}

/* P[l][m] = P_l^m(cos theta) without the Condon-Shortley sign, 0 <= m <= l <= lmax. */
static void legendre_table(int lmax, double ct, double st, double P[ORACLE_LMAX_CAP + 1][ORACLE_LMAX_CAP + 1]) {
  P[0][0] = 1.0;
  for (int m = 1; m <= lmax; ++m) P[m][m] = (2.0 * m - 1.0) * st * P[m - 1][m - 1];
  for (int m = 0; m < lmax; ++m) P[m + 1][m] = (2.0 * m + 1.0) * ct * P[m][m];
  for (int m = 0; m <= lmax; ++m)
    for (int l = m + 2; l <= lmax; ++l)
      P[l][m] = ((2.0 * l - 1.0) * ct * P[l - 1][m] - (double)(l + m - 1) * P[l - 2][m]) / (double)(l - m);
}

/* All R_l^m, l <= lmax, at the direction (theta, phi), written to row[k]. */
static void real_sh_from_angles(int lmax, double theta, double phi, double* row) {
  double P[ORACLE_LMAX_CAP + 1][ORACLE_LMAX_CAP + 1];
  legendre_table(lmax, cos(theta), sin(theta), P);
  const double rs2 = 1.0 / sqrt(2.0);
  for (int l = 0; l <= lmax; ++l) {
    /* complex Y_l^m for m = 0..l by Eq. 5 */
    double complex Yp[ORACLE_LMAX_CAP + 1];
    for (int m = 0; m <= l; ++m) {
      const double sgn = (m & 1) ? -1.0 : 1.0;
      Yp[m] = sgn * norm_lm(l, m) * P[l][m] * (cos(m * phi) + I * sin(m * phi));
    }
    for (int m = -l; m <= l; ++m) {
      double v;
      if (m == 0) {
        v = creal(Yp[0]);
      } else {
        const int a = m < 0 ? -m : m;
        const double sa = (a & 1) ? -1.0 : 1.0;          /* (-1)^|m| = (-1)^m */
        const double complex Ypos = Yp[a];               /* Y_l^{|m|}  */
        const double complex Yneg = sa * conj(Yp[a]);    /* Y_l^{-|m|}, Eq. 10 */
        if (m > 0) /* Eq. 6, m > 0: (Y_l^{-m} + (-1)^m Y_l^m) / sqrt 2 */
          v = creal(rs2 * (Yneg + sa * Ypos));
        else       /* Eq. 6, m < 0: i (Y_l^m - (-1)^m Y_l^{-m}) / sqrt 2 */
          v = creal(I * rs2 * (Yneg - sa * Ypos));
      }
      row[l * l + l + m] = v;
    }
  }
}

static int check_lmax(int lmax) { return lmax >= 0 && lmax <= ORACLE_LMAX_CAP; }

/* nthreads > 0: that many OpenMP threads; 0: every processor (also after an
 * earlier call asked for fewer). */
static void set_threads(int nthreads) {
#ifdef _OPENMP
  omp_set_num_threads(nthreads > 0 ? nthreads : omp_get_num_procs());
#else
  (void)nthreads;
#endif
}

/* Number of threads an OpenMP region would use (1 without OpenMP). */
int oracle_max_threads(int nthreads) {
  set_threads(nthreads);
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* All R_l^m, l <= lmax, at one Cartesian point p[3] (any r, r = 0 allowed). */
static void real_sh_point(const double* p, int lmax, double* row) {
  const int L2 = (lmax + 1) * (lmax + 1);
  const double x = p[0], y = p[1], z = p[2];
  if (x == 0.0 && y == 0.0 && z == 0.0) { /* r = 0 convention, Sec. II */
    row[0] = 1.0 / sqrt(4.0 * ORACLE_PI);
    for (int k = 1; k < L2; ++k) row[k] = 0.0;
    return;
  }
  const double rho = sqrt(x * x + y * y);
  real_sh_from_angles(lmax, atan2(rho, z), atan2(y, x), row);
}

/* Real harmonics at Cartesian points xyz[n][3]. */
int oracle_real_sh(const double* xyz, int64_t n, int lmax, double* out, int nthreads) {
  if (!check_lmax(lmax) || n < 0 || (n > 0 && (!xyz || !out))) return 1;
  const int L2 = (lmax + 1) * (lmax + 1);
  set_threads(nthreads);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) real_sh_point(xyz + 3 * i, lmax, out + i * (int64_t)L2);
  return 0;
}

/* Complex harmonics Y_l^m (Eq. 5 for m >= 0, Eq. 10 for m < 0) at Cartesian
 * points: out[i][k][0..1] = (Re, Im) of Y_l^m, k = l*l + l + m; at r = 0 only
 * Y_0^0 = 1/sqrt(4 pi) is nonzero (Sec. II). */
static void complex_sh_point(const double* p, int lmax, double* row) {
  const int L2 = (lmax + 1) * (lmax + 1);
  const double x = p[0], y = p[1], z = p[2];
  if (x == 0.0 && y == 0.0 && z == 0.0) {
    for (int k = 0; k < 2 * L2; ++k) row[k] = 0.0;
    row[0] = 1.0 / sqrt(4.0 * ORACLE_PI);
    return;
  }
  const double theta = atan2(sqrt(x * x + y * y), z), phi = atan2(y, x);
  double P[ORACLE_LMAX_CAP + 1][ORACLE_LMAX_CAP + 1];
  legendre_table(lmax, cos(theta), sin(theta), P);
  for (int l = 0; l <= lmax; ++l) {
    for (int m = 0; m <= l; ++m) {
      const double sgn = (m & 1) ? -1.0 : 1.0;
      const double complex Y = sgn * norm_lm(l, m) * P[l][m] * (cos(m * phi) + I * sin(m * phi));
      row[2 * (l * l + l + m)] = creal(Y);
      row[2 * (l * l + l + m) + 1] = cimag(Y);
      if (m > 0) { /* Eq. 10: Y_l^{-m} = (-1)^m conj(Y_l^m) */
        const double complex Yn = sgn * conj(Y);
        row[2 * (l * l + l - m)] = creal(Yn);
        row[2 * (l * l + l - m) + 1] = cimag(Yn);
      }
    }
  }
}

int oracle_complex_sh(const double* xyz, int64_t n, int lmax, double* out, int nthreads) {
  if (!check_lmax(lmax) || n < 0 || (n > 0 && (!xyz || !out))) return 1;
  const int L2 = (lmax + 1) * (lmax + 1);
  set_threads(nthreads);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) complex_sh_point(xyz + 3 * i, lmax, out + i * (int64_t)L2 * 2);
  return 0;
}

/* Spinor harmonics for spin 1/2 (Sec. II, Eq. 7) at Cartesian points, from
 * the complex harmonics of the same point.  For orbital l and total angular
 * momentum j = l + s/2 (s = +1, or s = -1 when l >= 1), m_j = -j .. j:
 *   upper = s sqrt(l + s m_j + 1/2) / sqrt(2l+1) * Y_l^{m_j - 1/2}
 *   lower =   sqrt(l - s m_j + 1/2) / sqrt(2l+1) * Y_l^{m_j + 1/2}
 * (Eq. 7 with its +- read as s and l = j -+ 1/2), where Y_l^m = 0 for |m| > l.
 * Output out[i][q][c][re/im]: spinor q = 2 l^2 + (s < 0 ? 0 : 2l) + (m_j + j),
 * component c = 0 (upper), 1 (lower); 2 (lmax+1)^2 spinors per point.  */
int oracle_spinor_sh(const double* xyz, int64_t n, int lmax, double* out, int nthreads) {
  if (!check_lmax(lmax) || n < 0 || (n > 0 && (!xyz || !out))) return 1;
  const int L2 = (lmax + 1) * (lmax + 1);
  set_threads(nthreads);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double Y[2 * (ORACLE_LMAX_CAP + 1) * (ORACLE_LMAX_CAP + 1)];
    complex_sh_point(xyz + 3 * i, lmax, Y);
    double* row = out + i * (int64_t)L2 * 8;
    for (int l = 0; l <= lmax; ++l) {
      const double pre = 1.0 / sqrt(2.0 * l + 1.0);
      for (int s = -1; s <= 1; s += 2) {
        if (s < 0 && l == 0) continue;
        const double j = l + 0.5 * s;
        const int q0 = 2 * l * l + (s < 0 ? 0 : 2 * l);
        const int nmj = (int)(2.0 * j + 1.0);
        for (int t = 0; t < nmj; ++t) {
          const double mj = -j + t;
          const int mu = (int)lround(mj - 0.5), md = (int)lround(mj + 0.5); /* m of the two Y */
          const double cu = s * sqrt(l + s * mj + 0.5) * pre, cd = sqrt(l - s * mj + 0.5) * pre;
          double* o = row + 4 * (q0 + t);
          o[0] = o[1] = o[2] = o[3] = 0.0;
          if (mu >= -l && mu <= l) {
            o[0] = cu * Y[2 * (l * l + l + mu)];
            o[1] = cu * Y[2 * (l * l + l + mu) + 1];
          }
          if (md >= -l && md <= l) {
            o[2] = cd * Y[2 * (l * l + l + md)];
            o[3] = cd * Y[2 * (l * l + l + md) + 1];
          }
        }
      }
    }
  }
  return 0;
}

/* Real harmonics at angular inputs (theta[i], phi[i]) (the angular interface). */
int oracle_real_sh_angles(const double* theta, const double* phi, int64_t n, int lmax, double* out) {
  if (!check_lmax(lmax) || n < 0 || (n > 0 && (!theta || !phi || !out))) return 1;
  const int L2 = (lmax + 1) * (lmax + 1);
  for (int64_t i = 0; i < n; ++i) real_sh_from_angles(lmax, theta[i], phi[i], out + i * (int64_t)L2);
  return 0;
}

/*
 * Fused non-local projectors (the paper's motivating use, Sec. I: projectors
 * of pseudopotential / PAW methods on a real-space grid need Y_lm at every
 * grid point of each atom's sphere).  The paper gives no further detail, so
 * the following choices are this project's and are stated once here:
 *
 *   grid point g (linear index, g = (i*ng + j)*ng + k) sits at (i, j, k) * h;
 *   d = minimum image of (grid point - atom position) in a cubic periodic box
 *       of side `box`: each component d_c -= box * rint(d_c / box);
 *   r = |d|, direction d / r (r = 0 uses the r = 0 convention);
 *   the radial function f_{s,l} is tabulated at r_i = r_min exp(i dlog),
 *   i = 0..n_rad-1; it is read at the continuous index t = ln(r / r_min) / dlog
 *   clamped to [0, n_rad-1] (t = 0 for r = 0), by 4-point Lagrange
 *   interpolation through the nodes i0..i0+3, i0 = clamp(floor(t) - 1, 0, n_rad-4);
 *   out[out_offsets[a] + (p - point_offsets[a]) * (lmax_s+1)^2 + l*l + l + m]
 *       = f_{s,l}(r) * R_l^m(d / r)          for every sphere point p of atom a.
 *
 * radial is [n_species][radial_lstride][n_rad] (radial_lstride >= 1 + max lmax).
 */
static double lagrange4(const double* F, int n_rad, double t) {
  int i0 = (int)floor(t) - 1;
  if (i0 < 0) i0 = 0;
  if (i0 > n_rad - 4) i0 = n_rad - 4;
  double f = 0.0;
  for (int j = 0; j < 4; ++j) {
    double w = 1.0;
    for (int q = 0; q < 4; ++q)
      if (q != j) w *= (t - (double)(i0 + q)) / (double)(j - q);
    f += w * F[i0 + j];
  }
  return f;
}

int oracle_projectors(int64_t n_atoms, const double* atom_pos, const int32_t* atom_species,
                      const int32_t* species_lmax, int n_species,
                      const double* radial, int radial_lstride, int n_rad, double r_min, double dlog,
                      double box, int ng, double h,
                      const int64_t* point_offsets, const int32_t* point_index,
                      const int64_t* out_offsets, double* out, int nthreads) {
  if (n_atoms < 0 || n_rad < 4 || ng <= 0 || !(box > 0.0) || !(h > 0.0) || !(dlog > 0.0) || !(r_min > 0.0)) return 1;
  for (int64_t a = 0; a < n_atoms; ++a) {
    const int s = atom_species[a];
    if (s < 0 || s >= n_species) return 1;
    const int lm = species_lmax[s];
    if (!check_lmax(lm) || lm + 1 > radial_lstride) return 1;
  }
  set_threads(nthreads);
  for (int64_t a = 0; a < n_atoms; ++a) {
    const int s = atom_species[a];
    const int lmax = species_lmax[s];
    const int L2 = (lmax + 1) * (lmax + 1);
    const double ax = atom_pos[3 * a], ay = atom_pos[3 * a + 1], az = atom_pos[3 * a + 2];
    const int64_t p0 = point_offsets[a], p1 = point_offsets[a + 1];
#pragma omp parallel for schedule(static)
    for (int64_t p = p0; p < p1; ++p) {
      const int64_t g = point_index[p];
      const int64_t gi = g / ((int64_t)ng * ng), gj = (g / ng) % ng, gk = g % ng;
      double d[3] = {(double)gi * h - ax, (double)gj * h - ay, (double)gk * h - az};
      for (int c = 0; c < 3; ++c) d[c] -= box * rint(d[c] / box);
      const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double t = (r > 0.0) ? log(r / r_min) / dlog : 0.0;
      if (t < 0.0) t = 0.0;
      if (t > (double)(n_rad - 1)) t = (double)(n_rad - 1);
      double Y[(ORACLE_LMAX_CAP + 1) * (ORACLE_LMAX_CAP + 1)];
      real_sh_point(d, lmax, Y);
      double* row = out + out_offsets[a] + (p - p0) * (int64_t)L2;
      for (int l = 0; l <= lmax; ++l) {
        const double f = lagrange4(radial + ((int64_t)s * radial_lstride + l) * n_rad, n_rad, t);
        for (int m = -l; m <= l; ++m) row[l * l + l + m] = f * Y[l * l + l + m];
      }
    }
  }
  return 0;
}
