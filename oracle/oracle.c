/*
 * oracle.c -- plain, slow, FP64 CPU reference for non-linear digital tracking
 * (Golovich et al., arXiv 2503.08854).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or constant with the
 * CUDA library; every constant below is written out here from its published
 * value.
 *
 * What it computes (paper section 3, Algorithm 1, "SearchImages" +
 * "FilterGPUIntersections" + "FindLocalSignal" + "FindSignificantResults"):
 *   for every candidate orbit (heliocentric Cartesian state at epoch t0)
 *   and every exposure of its family:
 *     1. two-body propagation about an inertial Sun (sec. 3, "elliptical
 *        two-body motion around the Sun"), universal-variable Kepler solve;
 *     2. light-time iteration against the observer position of the exposure;
 *     3. ecliptic -> equatorial rotation, gnomonic (TAN) projection about the
 *        exposure's tangent point and inverse CD matrix to pixels (sec. 3,
 *        World Coordinate System projection, Calabretta & Greisen 2002);
 *     4. keep the sample only if the nearest pixel lies inside the image
 *        (sec. 3: intersections outside the image are discarded);
 *     5. matched filter with a Gaussian PSF (sec. 3): psi = sum P*I/V and
 *        phi = sum P^2/V over the truncated PSF window at that pixel;
 *     6. constant-flux combination (sec. 3): Psi = sum psi, Phi = sum phi,
 *        stacked SNR nu = Psi / sqrt(Phi);
 *     7. ranking by nu, ties broken by the lower orbit index.
 * Every step is written as its plain definition, with no blocking or fusion.
 *
 * Units: AU, days, radians inside, degrees in the WCS.  Frame: heliocentric
 * ecliptic, Sun fixed at the origin.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* Gaussian gravitational constant k (AU^1.5 / day); GM_sun = k^2. */
double orc_gm_sun(void) { return 0.01720209895 * 0.01720209895; }
/* Speed of light in AU/day: 299792.458 km/s * 86400 s / 149597870.7 km. */
double orc_c_light(void) { return 299792.458 * 86400.0 / 149597870.7; }
/* IAU 2006 obliquity of the ecliptic at J2000, 84381.406 arcsec, in radians. */
double orc_obliquity(void) { return 84381.406 / 3600.0 * ORC_PI / 180.0; }

static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/*
 * Stumpff functions C(z) = sum_k (-z)^k/(2k+2)!, S(z) = sum_k (-z)^k/(2k+3)!.
 * Closed forms for |z| >= 1, the Maclaurin series otherwise (40 terms, far
 * beyond double precision for |z| < 1).
 */
static void stumpff(double z, double *C, double *S) {
  if (z >= 1.0) {
    double s = sqrt(z);
    *C = (1.0 - cos(s)) / z;
    *S = (s - sin(s)) / (z * s);
  } else if (z <= -1.0) {
    double s = sqrt(-z);
    *C = (cosh(s) - 1.0) / (-z);
    *S = (sinh(s) - s) / ((-z) * s);
  } else {
    double c = 0.0, sv = 0.0, term_c = 0.5, term_s = 1.0 / 6.0;
    for (int k = 0; k < 40; ++k) {
      c += term_c;
      sv += term_s;
      term_c *= -z / ((2.0 * k + 3.0) * (2.0 * k + 4.0));
      term_s *= -z / ((2.0 * k + 4.0) * (2.0 * k + 5.0));
    }
    *C = c;
    *S = sv;
  }
}

/*
 * Two-body propagation by the universal-variable formulation (Bate, Mueller
 * & White 1971, ch. 4; Curtis, Orbital Mechanics, Algorithms 3.3-3.4).
 * Given the state (r0, v0) and a time step dt, solves the universal Kepler
 * equation
 *   F(x) = (r0.v0/sqrt(mu)) x^2 C(a x^2) + (1 - a |r0|) x^3 S(a x^2)
 *          + |r0| x - sqrt(mu) dt = 0,   a = 2/|r0| - |v0|^2/mu,
 * by Newton's method guarded by bisection (F is increasing: F'(x) = |r| > 0),
 * then forms the Lagrange coefficients f, g, fdot, gdot.  Elliptic steps are
 * first reduced modulo the orbital period.  fg (optional) receives
 * {f, g, fdot, gdot}.  Returns the number of iterations, or -1 on failure.
 * A non-positive mu is treated as force-free motion (straight line).
 */
int orc_kepler_uv(const double r0[3], const double v0[3], double dt, double mu,
                  double r[3], double v[3], double fg[4]) {
  if (!(mu > 0.0)) {
    for (int i = 0; i < 3; ++i) {
      r[i] = r0[i] + v0[i] * dt;
      v[i] = v0[i];
    }
    if (fg) { fg[0] = 1.0; fg[1] = dt; fg[2] = 0.0; fg[3] = 1.0; }
    return 0;
  }
  const double sqmu = sqrt(mu);
  const double r0n = sqrt(dot3(r0, r0));
  const double v0sq = dot3(v0, v0);
  const double sig0 = dot3(r0, v0) / sqmu;
  const double alpha = 2.0 / r0n - v0sq / mu;

  if (alpha > 0.0) { /* bound orbit: reduce dt modulo the period */
    double period = 2.0 * ORC_PI / (sqmu * alpha * sqrt(alpha));
    dt = dt - period * nearbyint(dt / period);
  }

  /* residual and derivative of the universal Kepler equation */
#define UV_EVAL(xx, Fo, dFo)                                                  \
  do {                                                                        \
    double z_ = alpha * (xx) * (xx), C_, S_;                                  \
    stumpff(z_, &C_, &S_);                                                    \
    Fo = sig0 * (xx) * (xx) * C_ + (1.0 - alpha * r0n) * (xx) * (xx) * (xx) * S_ + \
         r0n * (xx) - sqmu * dt;                                              \
    dFo = sig0 * (xx) * (1.0 - z_ * S_) + (1.0 - alpha * r0n) * (xx) * (xx) * C_ + r0n; \
  } while (0)

  /* bracket [lo, hi] with F(lo) <= 0 <= F(hi) */
  double lo, hi, Flo, Fhi, dtmp;
  if (dt >= 0.0) {
    lo = 0.0;
    hi = sqmu * dt / r0n + 1e-300;
    UV_EVAL(hi, Fhi, dtmp);
    while (Fhi < 0.0) { lo = hi; hi *= 2.0; UV_EVAL(hi, Fhi, dtmp); }
    UV_EVAL(lo, Flo, dtmp);
  } else {
    hi = 0.0;
    lo = sqmu * dt / r0n - 1e-300;
    UV_EVAL(lo, Flo, dtmp);
    while (Flo > 0.0) { hi = lo; lo *= 2.0; UV_EVAL(lo, Flo, dtmp); }
    UV_EVAL(hi, Fhi, dtmp);
  }
  (void)dtmp;
  if (!(Flo <= 0.0 && Fhi >= 0.0)) return -1;

  /* Newton from the straight-line guess, falling back to bisection */
  double x = sqmu * dt / r0n;
  if (x < lo || x > hi) x = 0.5 * (lo + hi);
  int it, converged = 0;
  for (it = 1; it <= 200; ++it) {
    double F, dF;
    UV_EVAL(x, F, dF);
    if (F == 0.0) { converged = 1; break; }
    if (F < 0.0) lo = x; else hi = x;
    double xn = x - F / dF;
    if (!(xn >= lo && xn <= hi)) xn = 0.5 * (lo + hi);
    double step = fabs(xn - x);
    x = xn;
    if (step <= 1e-15 * fmax(1.0, fabs(x)) || hi - lo <= 1e-15 * fmax(1.0, fabs(x))) {
      converged = 1;
      break;
    }
  }
  if (!converged) {
    /* Newton wandering at rounding level: accept a residual that is small
       against the magnitude of the terms of F */
    double F, dF;
    UV_EVAL(x, F, dF);
    (void)dF;
    if (fabs(F) <= 1e-13 * (r0n * fabs(x) + sqmu * fabs(dt) + 1e-300)) converged = 1;
  }
#undef UV_EVAL
  if (!converged) return -1;

  double z = alpha * x * x, C, S;
  stumpff(z, &C, &S);
  double f = 1.0 - x * x * C / r0n;
  double g = dt - x * x * x * S / sqmu;
  for (int i = 0; i < 3; ++i) r[i] = f * r0[i] + g * v0[i];
  double rn = sqrt(dot3(r, r));
  double fdot = sqmu / (rn * r0n) * x * (z * S - 1.0);
  double gdot = 1.0 - x * x * C / rn;
  for (int i = 0; i < 3; ++i) v[i] = fdot * r0[i] + gdot * v0[i];
  if (fg) { fg[0] = f; fg[1] = g; fg[2] = fdot; fg[3] = gdot; }
  return it;
}

/*
 * Light-time corrected topocentric vector (paper sec. 3: the object's
 * location at the time of every image, seen from the observer).  The object
 * seen at t_obs left its position at t_obs - tau with tau = |rho| / c; tau is
 * found by fixed-point iteration, each iterate a full two-body propagation
 * from the epoch t0.  rho = r(t_obs - tau) - obs.  Returns 0 on success.
 */
int orc_apparent(const double state[6], double t0, double t_obs, const double obs[3],
                 double mu, double c, double rho[3], double *tau_out) {
  double tau = 0.0, r[3], v[3];
  for (int it = 0; it < 50; ++it) {
    if (orc_kepler_uv(state, state + 3, (t_obs - tau) - t0, mu, r, v, NULL) < 0) return -1;
    for (int i = 0; i < 3; ++i) rho[i] = r[i] - obs[i];
    double tau_new = sqrt(dot3(rho, rho)) / c;
    double diff = fabs(tau_new - tau);
    tau = tau_new;
    if (diff <= 1e-16 * tau + 1e-20) {
      /* re-evaluate at the converged tau so that tau * c == |rho| */
      if (orc_kepler_uv(state, state + 3, (t_obs - tau) - t0, mu, r, v, NULL) < 0) return -1;
      for (int i = 0; i < 3; ++i) rho[i] = r[i] - obs[i];
      if (tau_out) *tau_out = tau;
      return 0;
    }
  }
  if (tau_out) *tau_out = tau;
  return 0; /* converged to rounding level without meeting the strict test */
}

/*
 * Sky position and TAN (gnomonic) projection (Calabretta & Greisen 2002,
 * sec. 5.1.3), then pixel coordinates through the inverse CD matrix:
 *   rho_eq = R_x(+eps) rho_ecl;  ra = atan2(y, x), dec = atan2(z, hypot(x, y));
 *   cos c = sin d0 sin d + cos d0 cos d cos(ra - a0);
 *   xi  = cos d sin(ra - a0) / cos c;
 *   eta = (cos d0 sin d - sin d0 cos d cos(ra - a0)) / cos c;   (radians -> deg)
 *   [x, y] = crpix + CD^{-1} [xi, eta].
 * CRPIX is 0-based (FITS CRPIX minus one).  Returns 1 and writes (x, y) when
 * cos c > 0, otherwise returns 0 (the point lies 90 deg or more away).
 */
int orc_project(const double rho[3], double eps, const double crval[2], const double crpix[2],
                const double cd[4], double *x, double *y, double radec_out[2]) {
  double ce = cos(eps), se = sin(eps);
  double qx = rho[0];
  double qy = ce * rho[1] - se * rho[2];
  double qz = se * rho[1] + ce * rho[2];
  double ra = atan2(qy, qx);
  double dec = atan2(qz, sqrt(qx * qx + qy * qy));
  if (radec_out) { radec_out[0] = ra; radec_out[1] = dec; }
  double d2r = ORC_PI / 180.0;
  double a0 = crval[0] * d2r, d0 = crval[1] * d2r;
  double cosc = sin(d0) * sin(dec) + cos(d0) * cos(dec) * cos(ra - a0);
  if (!(cosc > 0.0)) return 0;
  double xi = cos(dec) * sin(ra - a0) / cosc / d2r;
  double eta = (cos(d0) * sin(dec) - sin(d0) * cos(dec) * cos(ra - a0)) / cosc / d2r;
  double det = cd[0] * cd[3] - cd[1] * cd[2];
  *x = crpix[0] + (cd[3] * xi - cd[1] * eta) / det;
  *y = crpix[1] + (-cd[2] * xi + cd[0] * eta) / det;
  return 1;
}

/*
 * Truncated Gaussian PSF of the matched filter (paper sec. 3: Gaussian point
 * spread function whose width is in the image header).  Window radius
 * R = ceil(4 sigma); P(kx, ky) = exp(-(kx^2 + ky^2) / (2 sigma^2)) normalised
 * so that the sum over the (2R+1)^2 window is one.  Writes the window
 * row-major into P (capacity at least (2R+1)^2) and returns R.
 */
int orc_psf_kernel(double sigma, double *P, int cap) {
  int R = (int)ceil(4.0 * sigma);
  int n = 2 * R + 1;
  if (n * n > cap) return -1;
  double sum = 0.0;
  for (int ky = -R; ky <= R; ++ky)
    for (int kx = -R; kx <= R; ++kx) {
      double w = exp(-(double)(kx * kx + ky * ky) / (2.0 * sigma * sigma));
      P[(ky + R) * n + (kx + R)] = w;
      sum += w;
    }
  for (int i = 0; i < n * n; ++i) P[i] /= sum;
  return R;
}

/*
 * Matched-filter planes at one pixel (px, py), by their definition:
 *   psi(p) = sum_k P(k) I(p + k) / V(p + k),  phi(p) = sum_k P(k)^2 / V(p + k),
 * summed over the PSF window, dropping terms outside the W x H image.
 * V is the per-pixel variance plane if var != NULL, else the constant var_c.
 * Images are row-major FP32, index y * W + x.
 */
static void plane_value(const float *img, const float *var, double var_c, int W, int H,
                        const double *P, int R, int px, int py, double *psi, double *phi) {
  int n = 2 * R + 1;
  double s_psi = 0.0, s_phi = 0.0;
  for (int ky = -R; ky <= R; ++ky) {
    int y = py + ky;
    if (y < 0 || y >= H) continue;
    for (int kx = -R; kx <= R; ++kx) {
      int x = px + kx;
      if (x < 0 || x >= W) continue;
      double Pk = P[(ky + R) * n + (kx + R)];
      double V = var ? (double)var[(size_t)y * W + x] : var_c;
      s_psi += Pk * (double)img[(size_t)y * W + x] / V;
      s_phi += Pk * Pk / V;
    }
  }
  *psi = s_psi;
  *phi = s_phi;
}

/* Full psi / phi planes of one image (row-major FP64 outputs). */
int orc_planes(const float *img, const float *var, double var_c, int W, int H, double sigma,
               double *psi, double *phi) {
  int R = (int)ceil(4.0 * sigma);
  int n = 2 * R + 1;
  double *P = (double *)malloc(sizeof(double) * n * n);
  if (!P) return -1;
  orc_psf_kernel(sigma, P, n * n);
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px)
      plane_value(img, var, var_c, W, H, P, R, px, py, &psi[(size_t)py * W + px],
                  &phi[(size_t)py * W + px]);
  free(P);
  return 0;
}

/* Exposure table, one entry per image (structure of arrays). */
typedef struct {
  int n;
  const double *mjd;     /* [n]    epoch, days                              */
  const double *obs;     /* [n*3]  observer heliocentric ecliptic, AU       */
  const double *crval;   /* [n*2]  tangent point RA, Dec, deg               */
  const double *crpix;   /* [n*2]  0-based pixel of the tangent point       */
  const double *cd;      /* [n*4]  CD matrix row-major, deg / px            */
  const double *sigma;   /* [n]    PSF sigma, px                            */
  const double *var;     /* [n]    constant per-pixel variance              */
  const int32_t *width;  /* [n]                                             */
  const int32_t *height; /* [n]                                             */
} orc_exposures;

/*
 * Predicted positions: xy[(o * n_exp + j) * 2 + {0,1}] = pixel coordinates
 * of orbit o in exposure j (light-time corrected), or NaN when cos c <= 0.
 * States are row-major [n_o][6] = x, y, z, vx, vy, vz at epoch t0.
 */
int orc_predict(const double *states, int64_t n_o, double t0, const orc_exposures *ex, double mu,
                double c, double eps, double *xy, int nthreads) {
  int fail = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64) reduction(| : fail)
#endif
  for (int64_t o = 0; o < n_o; ++o) {
    for (int j = 0; j < ex->n; ++j) {
      double rho[3], x, y;
      double *out = xy + ((size_t)o * ex->n + j) * 2;
      if (orc_apparent(states + 6 * o, t0, ex->mjd[j], ex->obs + 3 * j, mu, c, rho, NULL) != 0) {
        fail = 1;
        out[0] = out[1] = NAN;
        continue;
      }
      if (orc_project(rho, eps, ex->crval + 2 * j, ex->crpix + 2 * j, ex->cd + 4 * j, &x, &y, NULL)) {
        out[0] = x;
        out[1] = y;
      } else {
        out[0] = out[1] = NAN;
      }
    }
  }
  return fail ? -1 : 0;
}

/* Nearest pixel: pixel i spans [i - 1/2, i + 1/2). */
static int64_t nearest(double x) { return (int64_t)floor(x + 0.5); }

/*
 * Brute-force stacking over every (orbit, exposure) pair of every family.
 *
 * Families (CSR): family f owns orbits [fam_orb_off[f], fam_orb_off[f+1]) and
 * tests exposures fam_exp_idx[fam_exp_off[f] .. fam_exp_off[f+1]).  With
 * n_fam == 0 every orbit tests every exposure.
 *
 * Plane values come from psi_planes / phi_planes (one FP64 W x H plane per
 * exposure) when given, else they are computed at the gathered pixel from
 * the images by their definition.
 *
 * Outputs per orbit: Psi, Phi (FP64 sums) and n_obs.  Samples whose predicted
 * coordinate lies within amb_px of a pixel edge are "ambiguous": the other
 * side of the edge is an equally valid nearest pixel at FP64 rounding level.
 * For them the outputs psi_lo/psi_hi, phi_lo/phi_hi, n_lo/n_hi bracket every
 * combination of choices (an alternative outside the image contributes
 * nothing); n_amb counts them.  Any of the range outputs may be NULL.
 */
int orc_stack(const double *states, int64_t n_o, double t0, const orc_exposures *ex,
              const float *const *images, const float *const *var_planes,
              const double *const *psi_planes, const double *const *phi_planes,
              int32_t n_fam, const int64_t *fam_orb_off, const int64_t *fam_exp_off,
              const int32_t *fam_exp_idx, double mu, double c, double eps, double amb_px,
              double *Psi, double *Phi, int32_t *nobs, double *psi_lo, double *psi_hi,
              double *phi_lo, double *phi_hi, int32_t *n_lo, int32_t *n_hi, int32_t *n_amb,
              int nthreads) {
  /* PSF windows per exposure, only needed when planes are evaluated on demand */
  double **P = (double **)calloc(ex->n, sizeof(double *));
  int *R = (int *)calloc(ex->n, sizeof(int));
  if (!P || !R) return -1;
  if (!psi_planes) {
    for (int j = 0; j < ex->n; ++j) {
      R[j] = (int)ceil(4.0 * ex->sigma[j]);
      int n = 2 * R[j] + 1;
      P[j] = (double *)malloc(sizeof(double) * n * n);
      orc_psf_kernel(ex->sigma[j], P[j], n * n);
    }
  }
  int fail = 0;
  int32_t nf = n_fam > 0 ? n_fam : 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  for (int32_t f = 0; f < nf; ++f) {
    int64_t o_begin = n_fam > 0 ? fam_orb_off[f] : 0;
    int64_t o_end = n_fam > 0 ? fam_orb_off[f + 1] : n_o;
    int64_t e_begin = n_fam > 0 ? fam_exp_off[f] : 0;
    int64_t e_end = n_fam > 0 ? fam_exp_off[f + 1] : ex->n;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) reduction(| : fail)
#endif
    for (int64_t o = o_begin; o < o_end; ++o) {
      double S_psi = 0, S_phi = 0, lo_psi = 0, hi_psi = 0, lo_phi = 0, hi_phi = 0;
      int32_t cnt = 0, lo_n = 0, hi_n = 0, amb = 0;
      for (int64_t e = e_begin; e < e_end; ++e) {
        int j = n_fam > 0 ? fam_exp_idx[e] : (int)e;
        double rho[3], x, y;
        if (orc_apparent(states + 6 * o, t0, ex->mjd[j], ex->obs + 3 * j, mu, c, rho, NULL) != 0) {
          fail = 1;
          continue;
        }
        if (!orc_project(rho, eps, ex->crval + 2 * j, ex->crpix + 2 * j, ex->cd + 4 * j, &x, &y, NULL))
          continue;
        int W = ex->width[j], H = ex->height[j];
        /* candidate pixels along each axis: the nearest one plus, near an
           edge, its neighbour across that edge */
        int64_t cx[2], cy[2];
        int ncx = 1, ncy = 1;
        cx[0] = nearest(x);
        cy[0] = nearest(y);
        double fx = (x + 0.5) - floor(x + 0.5), fy = (y + 0.5) - floor(y + 0.5);
        if (fx < amb_px) cx[ncx++] = cx[0] - 1;
        else if (fx > 1.0 - amb_px) cx[ncx++] = cx[0] + 1;
        if (fy < amb_px) cy[ncy++] = cy[0] - 1;
        else if (fy > 1.0 - amb_px) cy[ncy++] = cy[0] + 1;
        double vmin_psi = INFINITY, vmax_psi = -INFINITY, vmin_phi = INFINITY, vmax_phi = -INFINITY;
        int nmin = 1, nmax = 0;
        for (int a = 0; a < ncx; ++a)
          for (int b = 0; b < ncy; ++b) {
            double vpsi = 0.0, vphi = 0.0;
            int in = cx[a] >= 0 && cx[a] < W && cy[b] >= 0 && cy[b] < H;
            if (in) {
              if (psi_planes) {
                size_t idx = (size_t)cy[b] * W + (size_t)cx[a];
                vpsi = psi_planes[j][idx];
                vphi = phi_planes[j][idx];
              } else {
                plane_value(images[j], var_planes ? var_planes[j] : NULL, ex->var[j], W, H, P[j],
                            R[j], (int)cx[a], (int)cy[b], &vpsi, &vphi);
              }
            }
            if (a == 0 && b == 0 && in) { /* the nearest pixel itself */
              S_psi += vpsi;
              S_phi += vphi;
              cnt += 1;
            }
            vmin_psi = fmin(vmin_psi, vpsi);
            vmax_psi = fmax(vmax_psi, vpsi);
            vmin_phi = fmin(vmin_phi, vphi);
            vmax_phi = fmax(vmax_phi, vphi);
            nmin = in < nmin ? in : nmin;
            nmax = in > nmax ? in : nmax;
          }
        lo_psi += vmin_psi;
        hi_psi += vmax_psi;
        lo_phi += vmin_phi;
        hi_phi += vmax_phi;
        lo_n += nmin;
        hi_n += nmax;
        if (ncx * ncy > 1) amb += 1;
      }
      Psi[o] = S_psi;
      Phi[o] = S_phi;
      nobs[o] = cnt;
      if (psi_lo) psi_lo[o] = lo_psi;
      if (psi_hi) psi_hi[o] = hi_psi;
      if (phi_lo) phi_lo[o] = lo_phi;
      if (phi_hi) phi_hi[o] = hi_phi;
      if (n_lo) n_lo[o] = lo_n;
      if (n_hi) n_hi[o] = hi_n;
      if (n_amb) n_amb[o] = amb;
    }
  }
  if (!psi_planes)
    for (int j = 0; j < ex->n; ++j) free(P[j]);
  free(P);
  free(R);
  return fail ? -1 : 0;
}

/*
 * Stacked detection statistic (paper sec. 3, constant flux in every image):
 * maximum-likelihood flux Psi/Phi with standard error 1/sqrt(Phi), so
 * nu = Psi / sqrt(Phi).  Orbits with Phi <= 0 or n_obs < min_obs get -inf.
 */
void orc_snr(const double *Psi, const double *Phi, const int32_t *nobs, int64_t n, int32_t min_obs,
             double *nu) {
  for (int64_t o = 0; o < n; ++o)
    nu[o] = (Phi[o] > 0.0 && nobs[o] >= min_obs) ? Psi[o] / sqrt(Phi[o]) : -INFINITY;
}

/* Ranking (paper Algorithm 1, FindSignificantResults): nu descending, then
   orbit index ascending.  Writes the first k indices and values. */
typedef struct {
  double nu;
  int64_t idx;
} orc_rank_item;

static int rank_cmp(const void *pa, const void *pb) {
  const orc_rank_item *a = (const orc_rank_item *)pa, *b = (const orc_rank_item *)pb;
  if (a->nu > b->nu) return -1;
  if (a->nu < b->nu) return 1;
  return (a->idx > b->idx) - (a->idx < b->idx);
}

int orc_topk(const double *nu, int64_t n, int64_t k, int64_t *idx_out, double *nu_out) {
  orc_rank_item *items = (orc_rank_item *)malloc(sizeof(orc_rank_item) * (n > 0 ? n : 1));
  if (!items) return -1;
  for (int64_t o = 0; o < n; ++o) {
    items[o].nu = nu[o];
    items[o].idx = o;
  }
  qsort(items, (size_t)n, sizeof(orc_rank_item), rank_cmp);
  if (k > n) k = n;
  for (int64_t i = 0; i < k; ++i) {
    idx_out[i] = items[i].idx;
    nu_out[i] = items[i].nu;
  }
  free(items);
  return (int)k;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
