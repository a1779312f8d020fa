/*
 * dm_oracle.c -- plain FP64 CPU oracle for the dual messenger Wiener filter of
 * joint T/Q/U CMB maps (Kodi Ramanah, Lavaux & Wandelt, arXiv:1801.05358),
 * carried onto the HEALPix sphere.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  The CUDA
 * product path never calls it, shares no code, header, table or helper with
 * it, and must not fall back to it.
 *
 * Everything here is written for a reader checking it against the paper:
 * no blocking, no fusion, no reordering beyond factoring Y_lm(theta, phi) =
 * lambda_lm(theta) e^{i m phi} per iso-latitude ring.  All arithmetic is FP64.
 * Loops that OpenMP splits are over independent outputs only, so results do
 * not depend on the thread count.
 *
 * Conventions (the paper is flat-sky; these are the sphere readings):
 *  - HEALPix RING pixelisation (Gorski et al. 2005): rings i = 1..4nside-1.
 *  - Spin-weighted harmonics of Goldberg et al. (1967):
 *        sY_lm(theta, phi) = sqrt((2l+1)/4pi) d^l_{m,-s}(theta) e^{i m phi},
 *    which at s = 0 is the usual Y_lm with the Condon-Shortley phase.
 *  - Polarisation: (Q + iU) = sum a_{2,lm} 2Y_lm, (Q - iU) = sum a_{-2,lm} -2Y_lm,
 *    a_{+-2} = -(a_E +- i a_B).  This is the sphere form of the E/B rotation
 *    of Section 2.1 (Eqs. 12-16).
 *  - Synthesis Y: a_lm -> map.  Analysis A = Omega Y^dagger, Omega = 4pi/Npix,
 *    the sphere counterpart of sigma^{-1} F^dagger in Algorithm 1 (no ring
 *    weights, no iteration).
 *  - alm storage: m-major, index(l, m) = m(2 lmax + 1 - m)/2 + l, m = 0..lmax,
 *    complex interleaved (re, im); fields T, E, B.  Maps: [3][Npix] (I, Q, U).
 *
 * Functions whose results are pinned by the -m "not gpu" tests: geometry,
 * harmonics, ring DFTs, synthesis/analysis, per-l filter, the messenger
 * update, the level loop, chi^2, Philox and the constrained-realisation draws,
 * the correlated-noise model (Appendix B) with its update, solve and CR
 * noise draws, and the modified Jacobi refinement (Appendix A).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* HEALPix RING geometry (Gorski et al. 2005; the paper works on a flat grid,  */
/* Section 3.1, and names the sphere as future work in Section 4).            */
/* ------------------------------------------------------------------------ */

long orc_npix(int nside) { return 12L * nside * nside; }
int orc_nrings(int nside) { return 4 * nside - 1; }
long orc_nalm(int lmax) { return (long)(lmax + 1) * (lmax + 2) / 2; }
long orc_almidx(int lmax, int l, int m) { return (long)m * (2 * lmax + 1 - m) / 2 + l; }

/* Ring i (1-based).  Returns the pixel count, first pixel, z = cos(theta),
 * 1 - z and 1 + z (the latter two without cancellation near the poles) and
 * the azimuth phi0 of the ring's first pixel. */
void orc_ring_info(int nside, int i, long *nr, long *start, double *z,
                   double *omz, double *opz, double *phi0) {
  long ns = nside;
  long npix = 12 * ns * ns, ncap = 2 * ns * (ns - 1);
  if (i < nside) { /* north polar cap */
    *nr = 4L * i;
    *start = 2L * i * (i - 1);
    *omz = (double)((long)i * i) / (3.0 * (double)(ns * ns));
    *opz = 2.0 - *omz;
    *z = 1.0 - *omz;
    *phi0 = M_PI / (4.0 * i);
  } else if (i <= 3 * nside) { /* equatorial belt */
    *nr = 4 * ns;
    *start = ncap + (long)(i - nside) * 4 * ns;
    *z = 4.0 / 3.0 - 2.0 * i / (3.0 * ns);
    *omz = 1.0 - *z;
    *opz = 1.0 + *z;
    *phi0 = ((i - nside + 1) % 2 == 1) ? M_PI / (4.0 * ns) : 0.0;
  } else { /* south polar cap, mirror of ring 4nside - i */
    long ip = 4 * ns - i;
    *nr = 4 * ip;
    *start = npix - 2 * ip * (ip + 1);
    *opz = (double)(ip * ip) / (3.0 * (double)(ns * ns));
    *omz = 2.0 - *opz;
    *z = *opz - 1.0;
    *phi0 = M_PI / (4.0 * ip);
  }
}

/* Pixel centre (z, phi) of every pixel, RING order. */
void orc_pix_centers(int nside, double *z, double *phi) {
  for (int i = 1; i <= 4 * nside - 1; ++i) {
    long nr, st;
    double zz, omz, opz, p0;
    orc_ring_info(nside, i, &nr, &st, &zz, &omz, &opz, &p0);
    for (long j = 0; j < nr; ++j) {
      z[st + j] = zz;
      phi[st + j] = p0 + 2.0 * M_PI * (double)j / (double)nr;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Spin-weighted harmonics by the three-term Wigner-d recurrence in l.          */
/*   f_l = sqrt((2l+1)/4pi) d^l_{m,k}(theta),  k in {0, -2, +2}                */
/*   k = 0 -> lambda_lm, k = -2 -> 2lambda_lm, k = +2 -> -2lambda_lm.          */
/* Recurrence (e.g. Varshalovich et al. 1988, Sec. 4.8):                        */
/*   sqrt(((l+1)^2-m^2)((l+1)^2-k^2))/(l+1) d^{l+1}                             */
/*     = (2l+1)(x - mk/(l(l+1))) d^l - sqrt((l^2-m^2)(l^2-k^2))/l d^{l-1}       */
/* Values are carried as v * 2^E so that nothing underflows near the poles.    */
/* ------------------------------------------------------------------------ */

#define ORC_RESCALE_EXP 300

/* Seed f_{l0}, l0 = max(m, |k|), as mantissa * 2^exp.  c = cos(theta/2),
 * s = sin(theta/2). */
static void wigner_seed(int m, int k, double c, double s, double *mant, int *ex) {
  if (m < abs(k)) {
    /* l0 = |k| = 2: explicit small closed forms of d^2_{m,+-2}, m = 0, 1. */
    double n2 = sqrt(5.0 / (4.0 * M_PI));
    double v;
    if (k > 0) { /* d^2_{m,2} = sqrt(C(4, 2+m)) c^{2+m} s^{2-m} */
      double binom = (m == 0) ? 6.0 : 4.0;
      v = sqrt(binom) * pow(c, 2 + m) * pow(s, 2 - m);
    } else { /* d^2_{m,-2} = (-1)^m sqrt(C(4, 2-m)) c^{2-m} s^{2+m} */
      double binom = (m == 0) ? 6.0 : 4.0;
      v = ((m & 1) ? -1.0 : 1.0) * sqrt(binom) * pow(c, 2 - m) * pow(s, 2 + m);
    }
    *mant = frexp(n2 * v, ex);
    return;
  }
  /* lambda_mm = sqrt((2m+1)/4pi) d^m_{m,0}: product over j of
   * -sqrt((2j+1)/(2j)) sin(theta), starting from 1/sqrt(4pi). */
  double sth = 2.0 * s * c;
  int e = 0;
  double v = frexp(1.0 / sqrt(4.0 * M_PI), &e);
  for (int j = 1; j <= m; ++j) {
    int de;
    v *= -sqrt((2.0 * j + 1.0) / (2.0 * j)) * sth;
    v = frexp(v, &de);
    e += de;
  }
  if (k != 0) {
    /* d^m_{m,k} / d^m_{m,0} = (-1)^k sqrt(C(2m,m+k)/C(2m,m)) (c/s)^k, and
     * C(2m, m+-2)/C(2m, m) = m(m-1)/((m+1)(m+2)). */
    double r = sqrt((double)m * (m - 1) / ((double)(m + 1) * (m + 2)));
    double cs = c / s;
    v *= r * ((k > 0) ? cs * cs : 1.0 / (cs * cs));
    int de;
    v = frexp(v, &de);
    e += de;
  }
  *mant = v;
  *ex = e;
}

/* out[l] = f_l for l = 0..lmax (zero below l0). */
static void wigner_column(int lmax, int m, int k, double x, double c, double s, double *out) {
  for (int l = 0; l <= lmax; ++l) out[l] = 0.0;
  int l0 = m > abs(k) ? m : abs(k);
  if (l0 > lmax) return;
  double v0, vm1 = 0.0;
  int E;
  wigner_seed(m, k, c, s, &v0, &E);
  out[l0] = ldexp(v0, E);
  double mm = (double)m * m, kk = (double)k * k;
  for (int l = l0; l < lmax; ++l) {
    double lp = l + 1.0;
    double r1 = sqrt((lp * lp - mm) * (lp * lp - kk));
    double r0 = sqrt(((double)l * l - mm) * ((double)l * l - kk));
    double a = sqrt((2.0 * l + 3.0) / (2.0 * l + 1.0)) * lp * (2.0 * l + 1.0) / r1;
    double xt = (l == 0) ? x : x - (double)m * k / ((double)l * lp);
    double b = (r0 == 0.0) ? 0.0 : sqrt((2.0 * l + 3.0) / (2.0 * l - 1.0)) * lp * r0 / ((double)l * r1);
    double v1 = a * xt * v0 - b * vm1;
    vm1 = v0;
    v0 = v1;
    if (fabs(v0) > ldexp(1.0, ORC_RESCALE_EXP)) {
      v0 = ldexp(v0, -ORC_RESCALE_EXP);
      vm1 = ldexp(vm1, -ORC_RESCALE_EXP);
      E += ORC_RESCALE_EXP;
    }
    out[l + 1] = ldexp(v0, E);
  }
}

/* lambda_lm, 2lambda_lm and -2lambda_lm at the ring with 1 -+ z given. */
void orc_lambda(int lmax, int m, double omz, double opz, double *l0, double *lp2, double *lm2) {
  double x = 0.5 * (opz - omz);
  double c = sqrt(0.5 * opz), s = sqrt(0.5 * omz);
  wigner_column(lmax, m, 0, x, c, s, l0);
  wigner_column(lmax, m, -2, x, c, s, lp2);
  wigner_column(lmax, m, +2, x, c, s, lm2);
}

/* Convenience for tests: harmonics at an arbitrary theta. */
void orc_lambda_theta(int lmax, int m, double theta, double *l0, double *lp2, double *lm2) {
  double c = cos(0.5 * theta), s = sin(0.5 * theta);
  orc_lambda(lmax, m, 2.0 * s * s, 2.0 * c * c, l0, lp2, lm2);
}

/* ------------------------------------------------------------------------ */
/* Naive ring DFTs (the phi part of the transforms; paper: "Fourier transforms" */
/* counted in Section 3.4).  Angles are reduced exactly: m phi_j = m phi0 +     */
/* 2 pi (m j mod n)/n.                                                          */
/* ------------------------------------------------------------------------ */

/* G_m = sum_j f_j e^{-i m (phi0 + 2 pi j / n)}, m = 0..mmax. out: [mmax+1][2]. */
static void ring_dft_fwd(long n, double phi0, const double *f, int mmax, double *out) {
  double *ct = malloc(sizeof(double) * n), *st = malloc(sizeof(double) * n);
  for (long k = 0; k < n; ++k) {
    ct[k] = cos(2.0 * M_PI * (double)k / (double)n);
    st[k] = sin(2.0 * M_PI * (double)k / (double)n);
  }
  for (int m = 0; m <= mmax; ++m) {
    double re = 0.0, im = 0.0;
    for (long j = 0; j < n; ++j) {
      long k = ((long)m * j) % n;
      re += f[j] * ct[k];
      im -= f[j] * st[k];
    }
    double cp = cos(m * phi0), sp = sin(m * phi0);
    out[2 * m] = re * cp + im * sp; /* (re + i im) e^{-i m phi0} */
    out[2 * m + 1] = im * cp - re * sp;
  }
  free(ct);
  free(st);
}

/* f_j = Re F_0 + 2 sum_{m=1}^{mmax} Re(F_m e^{i m (phi0 + 2 pi j/n)}): the
 * real map whose m < 0 coefficients are the conjugates of the m > 0 ones. */
static void ring_dft_inv(long n, double phi0, const double *F, int mmax, double *f) {
  double *ct = malloc(sizeof(double) * n), *st = malloc(sizeof(double) * n);
  double *gr = malloc(sizeof(double) * (mmax + 1)), *gi = malloc(sizeof(double) * (mmax + 1));
  for (long k = 0; k < n; ++k) {
    ct[k] = cos(2.0 * M_PI * (double)k / (double)n);
    st[k] = sin(2.0 * M_PI * (double)k / (double)n);
  }
  for (int m = 0; m <= mmax; ++m) { /* G_m = F_m e^{i m phi0} */
    double cp = cos(m * phi0), sp = sin(m * phi0);
    gr[m] = F[2 * m] * cp - F[2 * m + 1] * sp;
    gi[m] = F[2 * m] * sp + F[2 * m + 1] * cp;
  }
  for (long j = 0; j < n; ++j) {
    double acc = gr[0];
    for (int m = 1; m <= mmax; ++m) {
      long k = ((long)m * j) % n;
      acc += 2.0 * (gr[m] * ct[k] - gi[m] * st[k]);
    }
    f[j] = acc;
  }
  free(ct);
  free(st);
  free(gr);
  free(gi);
}

/* Ring DFTs of a whole map. rc: [nrings][mmax+1][2]. */
void orc_ring_dft_forward(int nside, int mmax, const double *map, double *rc) {
  int nr_ = orc_nrings(nside);
#pragma omp parallel for schedule(dynamic)
  for (int i = 1; i <= nr_; ++i) {
    long nr, st;
    double z, omz, opz, p0;
    orc_ring_info(nside, i, &nr, &st, &z, &omz, &opz, &p0);
    ring_dft_fwd(nr, p0, map + st, mmax, rc + (long)(i - 1) * (mmax + 1) * 2);
  }
}

void orc_ring_dft_inverse(int nside, int mmax, const double *rc, double *map) {
  int nr_ = orc_nrings(nside);
#pragma omp parallel for schedule(dynamic)
  for (int i = 1; i <= nr_; ++i) {
    long nr, st;
    double z, omz, opz, p0;
    orc_ring_info(nside, i, &nr, &st, &z, &omz, &opz, &p0);
    ring_dft_inv(nr, p0, rc + (long)(i - 1) * (mmax + 1) * 2, mmax, map + st);
  }
}

/* ------------------------------------------------------------------------ */
/* Legendre stages: per ring, per m.                                           */
/* Synthesis (F in Algorithm 1):                                               */
/*   F^T_m = sum_l aT lambda                                                   */
/*   F^Q_m = -sum_l [aE lam+ + i aB lam-],  F^U_m = -sum_l [aB lam+ - i aE lam-] */
/*   lam+- = (2lambda +- -2lambda)/2                                           */
/* Analysis (sigma^{-1} F^dagger in Algorithm 1, here Omega Y^dagger):         */
/*   aT = Om sum_r lambda G^T,  aE = -Om sum_r [lam+ G^Q + i lam- G^U],         */
/*   aB = -Om sum_r [lam+ G^U - i lam- G^Q].                                    */
/* rc layout: [3][nrings][lmax+1][2].                                          */
/* ------------------------------------------------------------------------ */

void orc_legendre_synthesis(int nside, int lmax, const double *alm, double *rc) {
  int nrg = orc_nrings(nside);
  long nalm = orc_nalm(lmax);
  long rstride = (long)(lmax + 1) * 2, fstride = (long)nrg * rstride;
#pragma omp parallel
  {
    double *l0 = malloc(sizeof(double) * (lmax + 1));
    double *lp = malloc(sizeof(double) * (lmax + 1));
    double *lm = malloc(sizeof(double) * (lmax + 1));
#pragma omp for schedule(dynamic)
    for (int i = 1; i <= nrg; ++i) {
      long nr, st;
      double z, omz, opz, p0;
      orc_ring_info(nside, i, &nr, &st, &z, &omz, &opz, &p0);
      for (int m = 0; m <= lmax; ++m) {
        orc_lambda(lmax, m, omz, opz, l0, lp, lm);
        double tr = 0, ti = 0, qr = 0, qi = 0, ur = 0, ui = 0;
        for (int l = m; l <= lmax; ++l) {
          long ix = orc_almidx(lmax, l, m);
          const double *aT = alm + 2 * ix, *aE = alm + 2 * (nalm + ix), *aB = alm + 2 * (2 * nalm + ix);
          double lpl = 0.5 * (lp[l] + lm[l]), lmi = 0.5 * (lp[l] - lm[l]);
          tr += aT[0] * l0[l];
          ti += aT[1] * l0[l];
          /* -(aE lam+ + i aB lam-) */
          qr += -(aE[0] * lpl - aB[1] * lmi);
          qi += -(aE[1] * lpl + aB[0] * lmi);
          /* -(aB lam+ - i aE lam-) */
          ur += -(aB[0] * lpl + aE[1] * lmi);
          ui += -(aB[1] * lpl - aE[0] * lmi);
        }
        double *o = rc + (long)(i - 1) * rstride + 2 * m;
        o[0] = tr; o[1] = ti;
        o[fstride] = qr; o[fstride + 1] = qi;
        o[2 * fstride] = ur; o[2 * fstride + 1] = ui;
      }
    }
    free(l0); free(lp); free(lm);
  }
}

void orc_legendre_analysis(int nside, int lmax, const double *rc, double *alm) {
  int nrg = orc_nrings(nside);
  long nalm = orc_nalm(lmax);
  long rstride = (long)(lmax + 1) * 2, fstride = (long)nrg * rstride;
  double omega = 4.0 * M_PI / (double)orc_npix(nside);
  memset(alm, 0, sizeof(double) * 6 * nalm);
#pragma omp parallel
  {
    double *l0 = malloc(sizeof(double) * (lmax + 1));
    double *lp = malloc(sizeof(double) * (lmax + 1));
    double *lm = malloc(sizeof(double) * (lmax + 1));
#pragma omp for schedule(dynamic)
    for (int m = 0; m <= lmax; ++m) {
      for (int i = 1; i <= nrg; ++i) {
        long nr, st;
        double z, omz, opz, p0;
        orc_ring_info(nside, i, &nr, &st, &z, &omz, &opz, &p0);
        orc_lambda(lmax, m, omz, opz, l0, lp, lm);
        const double *g = rc + (long)(i - 1) * rstride + 2 * m;
        double gtr = g[0], gti = g[1];
        double gqr = g[fstride], gqi = g[fstride + 1];
        double gur = g[2 * fstride], gui = g[2 * fstride + 1];
        for (int l = m; l <= lmax; ++l) {
          long ix = orc_almidx(lmax, l, m);
          double *aT = alm + 2 * ix, *aE = alm + 2 * (nalm + ix), *aB = alm + 2 * (2 * nalm + ix);
          double lpl = 0.5 * (lp[l] + lm[l]), lmi = 0.5 * (lp[l] - lm[l]);
          aT[0] += omega * l0[l] * gtr;
          aT[1] += omega * l0[l] * gti;
          /* -(lam+ G^Q + i lam- G^U) */
          aE[0] += -omega * (lpl * gqr - lmi * gui);
          aE[1] += -omega * (lpl * gqi + lmi * gur);
          /* -(lam+ G^U - i lam- G^Q) */
          aB[0] += -omega * (lpl * gur + lmi * gqi);
          aB[1] += -omega * (lpl * gui - lmi * gqr);
        }
      }
    }
    free(l0); free(lp); free(lm);
  }
}

/* Sampled transforms, for parity checks at sizes where the full oracle
 * transforms take too long.  They restrict the sums of orc_legendre_synthesis
 * + orc_ring_dft_inverse to one ring, and those of orc_ring_dft_forward +
 * orc_legendre_analysis to one order m; the arithmetic is the same. */

/* G_m = sum_j f_j e^{-i m (phi0 + 2 pi j / n)} for one m (the m-th output of ring_dft_fwd) */
static void ring_dft_fwd_one(long n, double phi0, const double *f, int m, double *out) {
  double re = 0.0, im = 0.0;
  for (long j = 0; j < n; ++j) {
    long k = ((long)m * j) % n;
    re += f[j] * cos(2.0 * M_PI * (double)k / (double)n);
    im -= f[j] * sin(2.0 * M_PI * (double)k / (double)n);
  }
  double cp = cos(m * phi0), sp = sin(m * phi0);
  out[0] = re * cp + im * sp;
  out[1] = im * cp - re * sp;
}

/* The three maps of Y a on ring i (1-based): out[3][n_r]. */
void orc_ring_alm2map(int nside, int lmax, const double *alm, int i, double *out) {
  long nr, st;
  double z, omz, opz, p0;
  orc_ring_info(nside, i, &nr, &st, &z, &omz, &opz, &p0);
  long nalm = orc_nalm(lmax);
  long fs = (long)(lmax + 1) * 2;
  double *F = malloc(sizeof(double) * 3 * fs);
#pragma omp parallel
  {
    double *l0 = malloc(sizeof(double) * (lmax + 1));
    double *lp = malloc(sizeof(double) * (lmax + 1));
    double *lm = malloc(sizeof(double) * (lmax + 1));
#pragma omp for schedule(dynamic)
    for (int m = 0; m <= lmax; ++m) {
      orc_lambda(lmax, m, omz, opz, l0, lp, lm);
      double tr = 0, ti = 0, qr = 0, qi = 0, ur = 0, ui = 0;
      for (int l = m; l <= lmax; ++l) {
        long ix = orc_almidx(lmax, l, m);
        const double *aT = alm + 2 * ix, *aE = alm + 2 * (nalm + ix), *aB = alm + 2 * (2 * nalm + ix);
        double lpl = 0.5 * (lp[l] + lm[l]), lmi = 0.5 * (lp[l] - lm[l]);
        tr += aT[0] * l0[l];
        ti += aT[1] * l0[l];
        qr += -(aE[0] * lpl - aB[1] * lmi);
        qi += -(aE[1] * lpl + aB[0] * lmi);
        ur += -(aB[0] * lpl + aE[1] * lmi);
        ui += -(aB[1] * lpl - aE[0] * lmi);
      }
      F[2 * m] = tr; F[2 * m + 1] = ti;
      F[fs + 2 * m] = qr; F[fs + 2 * m + 1] = qi;
      F[2 * fs + 2 * m] = ur; F[2 * fs + 2 * m + 1] = ui;
    }
    free(l0); free(lp); free(lm);
  }
  for (int f = 0; f < 3; ++f) ring_dft_inv(nr, p0, F + f * fs, lmax, out + f * nr);
  free(F);
}

/* Column m of A f = Omega Y^dagger f: out[3][lmax+1] complex (entries l < m zero). */
void orc_map2alm_m(int nside, int lmax, const double *map, int m, double *out) {
  int nrg = orc_nrings(nside);
  long npix = orc_npix(nside);
  double omega = 4.0 * M_PI / (double)npix;
  long fs = (long)(lmax + 1) * 2;
  memset(out, 0, sizeof(double) * 3 * fs);
#pragma omp parallel
  {
    double *l0 = malloc(sizeof(double) * (lmax + 1));
    double *lp = malloc(sizeof(double) * (lmax + 1));
    double *lm = malloc(sizeof(double) * (lmax + 1));
    double *acc = calloc(3 * fs, sizeof(double));
#pragma omp for schedule(dynamic)
    for (int i = 1; i <= nrg; ++i) {
      long nr, st;
      double z, omz, opz, p0, g[6];
      orc_ring_info(nside, i, &nr, &st, &z, &omz, &opz, &p0);
      for (int f = 0; f < 3; ++f) ring_dft_fwd_one(nr, p0, map + f * npix + st, m, g + 2 * f);
      orc_lambda(lmax, m, omz, opz, l0, lp, lm);
      for (int l = m; l <= lmax; ++l) {
        double lpl = 0.5 * (lp[l] + lm[l]), lmi = 0.5 * (lp[l] - lm[l]);
        double *aT = acc + 2 * l, *aE = acc + fs + 2 * l, *aB = acc + 2 * fs + 2 * l;
        aT[0] += omega * l0[l] * g[0];
        aT[1] += omega * l0[l] * g[1];
        aE[0] += -omega * (lpl * g[2] - lmi * g[5]);
        aE[1] += -omega * (lpl * g[3] + lmi * g[4]);
        aB[0] += -omega * (lpl * g[4] + lmi * g[3]);
        aB[1] += -omega * (lpl * g[5] - lmi * g[2]);
      }
    }
#pragma omp critical
    for (long k = 0; k < 3 * fs; ++k) out[k] += acc[k];
    free(l0); free(lp); free(lm); free(acc);
  }
}

/* Full transforms: Y (alm -> map) and A = Omega Y^dagger (map -> alm). */
void orc_alm2map(int nside, int lmax, const double *alm, double *map) {
  int nrg = orc_nrings(nside);
  long npix = orc_npix(nside);
  long fstride = (long)nrg * (lmax + 1) * 2;
  double *rc = malloc(sizeof(double) * 3 * fstride);
  orc_legendre_synthesis(nside, lmax, alm, rc);
  for (int f = 0; f < 3; ++f) orc_ring_dft_inverse(nside, lmax, rc + f * fstride, map + f * npix);
  free(rc);
}

void orc_map2alm(int nside, int lmax, const double *map, double *alm) {
  int nrg = orc_nrings(nside);
  long npix = orc_npix(nside);
  long fstride = (long)nrg * (lmax + 1) * 2;
  double *rc = malloc(sizeof(double) * 3 * fstride);
  for (int f = 0; f < 3; ++f) orc_ring_dft_forward(nside, lmax, map + f * npix, rc + f * fstride);
  orc_legendre_analysis(nside, lmax, rc, alm);
  free(rc);
}

/* ------------------------------------------------------------------------ */
/* Per-l TEB filter (Eq. 8 with Sbar = Theta(S - U), Algorithm 1):             */
/*   u = R^T diag(f_e) R t,  f_e = max(S_e, mu) / (max(S_e, mu) + T_h)          */
/* where S_e are the eigenvalues of the 3x3 block of Eq. 10 (2x2 TE block plus */
/* BB), U = mu 1, xi = mu + T_h.  cl: [4][lmax+1] = TT, EE, BB, TE.            */
/* coef: [lmax+1][4] = F_TT, F_TE, F_EE, F_BB.                                 */
/* ------------------------------------------------------------------------ */

/* Eigen-decomposition of [[a, b], [b, c]]: e1 >= e2, (v1, v2) orthonormal. */
static void eig2(double a, double b, double c, double *e1, double *e2, double v1[2], double v2[2]) {
  if (b == 0.0) {
    if (a >= c) { *e1 = a; *e2 = c; v1[0] = 1; v1[1] = 0; v2[0] = 0; v2[1] = 1; }
    else { *e1 = c; *e2 = a; v1[0] = 0; v1[1] = 1; v2[0] = 1; v2[1] = 0; }
    return;
  }
  double h = 0.5 * (a - c);
  double disc = sqrt(h * h + b * b);
  *e1 = 0.5 * (a + c) + disc;
  *e2 = (*e1 != 0.0) ? (a * c - b * b) / *e1 : 0.5 * (a + c) - disc;
  /* eigenvector of e1: (b, e1 - a) or (e1 - c, b), whichever is larger */
  double x1 = b, y1 = *e1 - a, x2 = *e1 - c, y2 = b;
  double n1 = hypot(x1, y1), n2 = hypot(x2, y2);
  if (n1 >= n2) { v1[0] = x1 / n1; v1[1] = y1 / n1; }
  else { v1[0] = x2 / n2; v1[1] = y2 / n2; }
  v2[0] = -v1[1];
  v2[1] = v1[0];
}

void orc_filter_coefs(int lmax, const double *cl, double mu, double th, double *coef) {
  const double *tt = cl, *ee = cl + (lmax + 1), *bb = cl + 2 * (lmax + 1), *te = cl + 3 * (lmax + 1);
  for (int l = 0; l <= lmax; ++l) {
    double e1, e2, v1[2], v2[2];
    eig2(tt[l], te[l], ee[l], &e1, &e2, v1, v2);
    if (e1 < 0) e1 = 0;
    if (e2 < 0) e2 = 0;
    double s1 = fmax(e1, mu), s2 = fmax(e2, mu), s3 = fmax(bb[l] < 0 ? 0 : bb[l], mu);
    double f1 = (s1 + th > 0) ? s1 / (s1 + th) : 0.0;
    double f2 = (s2 + th > 0) ? s2 / (s2 + th) : 0.0;
    double f3 = (s3 + th > 0) ? s3 / (s3 + th) : 0.0;
    coef[4 * l + 0] = f1 * v1[0] * v1[0] + f2 * v2[0] * v2[0];
    coef[4 * l + 1] = f1 * v1[0] * v1[1] + f2 * v2[0] * v2[1];
    coef[4 * l + 2] = f1 * v1[1] * v1[1] + f2 * v2[1] * v2[1];
    coef[4 * l + 3] = f3;
  }
}

void orc_apply_filter(int lmax, const double *coef, double *alm) {
  long nalm = orc_nalm(lmax);
  for (int m = 0; m <= lmax; ++m)
    for (int l = m; l <= lmax; ++l) {
      long ix = orc_almidx(lmax, l, m);
      const double *c = coef + 4 * l;
      for (int p = 0; p < 2; ++p) {
        double t = alm[2 * ix + p], e = alm[2 * (nalm + ix) + p];
        alm[2 * ix + p] = c[0] * t + c[1] * e;
        alm[2 * (nalm + ix) + p] = c[1] * t + c[2] * e;
        alm[2 * (2 * nalm + ix) + p] *= c[3];
      }
    }
}

/* ------------------------------------------------------------------------ */
/* Noise: diagonal N = sigma^2 per pixel and Stokes component, masked pixels   */
/* carry N^{-1} = 0 (Appendix B: Sigma^{-1} = 0 on the mask).  T = alpha 1,     */
/* alpha = min N over observed pixel-components (Section 2).  The messenger    */
/* update of Eq. 9 is then t = (1 - w) s + w d with w = alpha/N (w = 0 masked), */
/* which also covers the N = T corner case (w = 1, t = d) of Section 2.1.      */
/* ------------------------------------------------------------------------ */

double orc_alpha(long npix, const double *sigma, const uint8_t *mask) {
  double a = INFINITY;
  for (int f = 0; f < 3; ++f)
    for (long p = 0; p < npix; ++p)
      if (!mask || mask[p]) {
        double n = sigma[f * npix + p] * sigma[f * npix + p];
        if (n < a) a = n;
      }
  return a;
}

void orc_weights(long npix, const double *sigma, const uint8_t *mask, double alpha, double *w) {
  for (int f = 0; f < 3; ++f)
    for (long p = 0; p < npix; ++p) {
      double n = sigma[f * npix + p] * sigma[f * npix + p];
      w[f * npix + p] = (!mask || mask[p]) ? alpha / n : 0.0;
    }
}

void orc_messenger_update(long n, const double *w, const double *d, const double *s, double *t) {
  for (long i = 0; i < n; ++i) t[i] = (w[i] > 0.0) ? (1.0 - w[i]) * s[i] + w[i] * d[i] : s[i];
}

/* ------------------------------------------------------------------------ */
/* The dual messenger loop (Algorithm 1) on the sphere.                        */
/*                                                                              */
/* Algorithm 1 analyses the messenger with sigma^{-1} F^dagger, the exact       */
/* inverse of the synthesis F because F F^dagger = sigma 1 (Section 2.1).  On   */
/* HEALPix the plain analysis A = Omega Y^dagger is only an approximate inverse */
/* (A Y != 1), so the exact inverse is applied to t as the warm-started one-step */
/* iterative analysis  a + A (t - Y a)  around the current harmonic iterate a.  */
/* Whenever A Y = 1 this is A t, i.e. Algorithm 1 verbatim; on HEALPix it makes */
/* the fixed point the exact Wiener filter (S'^{-1} + Y^T N^{-1} Y) a =          */
/* Y^T N^{-1} d with S' = Sbar + U at each level (Eqs. 2, 8, 9).                */
/*                                                                              */
/*  s_0 = 0, a_0 = 0, t_0 = d (masked pixels of d carry no data: set to 0)     */
/*  level k: lambda_k = xi_k / T_h, mu_k = (lambda_k - 1) T_h                   */
/*  repeat:  a <- F_k [a + A (t - s)]        harmonic step, Eq. 8               */
/*           s <- Y a                        synthesis                          */
/*           t <- (1 - w) s + w d            messenger update, Eq. 9            */
/*  until ||s_i - s_{i-1}|| / ||s_i|| < eps_k  (or a fixed count per level)      */
/* levels: lambda_k given (last = 1, i.e. mu = 0, xi = T_h).                    */
/* forced_iters: if non-NULL, exactly forced_iters[k] iterations at level k.   */
/* Returns the total iteration count; iters_out[k] per level, cauchy_out[i]    */
/* the Cauchy ratio of iteration i (length max_iter), may be NULL.             */
/* ------------------------------------------------------------------------ */

int orc_dm_solve(int nside, int lmax, const double *cl, const double *sigma, const uint8_t *mask,
                 const double *d, int nlev, const double *lambdas, const double *eps,
                 const int *forced_iters, int max_iter, double *s_out, double *alm_out,
                 int *iters_out, double *cauchy_out) {
  long npix = orc_npix(nside), nalm = orc_nalm(lmax);
  long n3 = 3 * npix;
  double alpha = orc_alpha(npix, sigma, mask);
  double omega = 4.0 * M_PI / (double)npix;
  double th = alpha * omega;
  double *w = malloc(sizeof(double) * n3), *t = malloc(sizeof(double) * n3);
  double *s = malloc(sizeof(double) * n3), *sn = malloc(sizeof(double) * n3);
  double *r = malloc(sizeof(double) * n3);
  double *a = malloc(sizeof(double) * 6 * nalm), *ar = malloc(sizeof(double) * 6 * nalm);
  double *coef = malloc(sizeof(double) * 4 * (lmax + 1));
  orc_weights(npix, sigma, mask, alpha, w);
  for (long i = 0; i < n3; ++i) {
    s[i] = 0.0;
    t[i] = (w[i] > 0.0) ? d[i] : 0.0;
  }
  memset(a, 0, sizeof(double) * 6 * nalm);
  int it = 0;
  for (int k = 0; k < nlev; ++k) {
    double mu = (lambdas[k] - 1.0) * th;
    orc_filter_coefs(lmax, cl, mu, th, coef);
    int nk = 0;
    for (;;) {
      if (!forced_iters && it >= max_iter) break;
      if (forced_iters && nk >= forced_iters[k]) break;
      for (long i = 0; i < n3; ++i) r[i] = t[i] - s[i];
      orc_map2alm(nside, lmax, r, ar);
      for (long i = 0; i < 6 * nalm; ++i) a[i] += ar[i];
      orc_apply_filter(lmax, coef, a);
      orc_alm2map(nside, lmax, a, sn);
      double dd = 0.0, ss = 0.0;
      for (long i = 0; i < n3; ++i) {
        dd += (sn[i] - s[i]) * (sn[i] - s[i]);
        ss += sn[i] * sn[i];
      }
      double cauchy = (ss > 0.0) ? sqrt(dd / ss) : 0.0;
      memcpy(s, sn, sizeof(double) * n3);
      orc_messenger_update(n3, w, d, s, t);
      if (cauchy_out && it < max_iter) cauchy_out[it] = cauchy;
      ++it;
      ++nk;
      if (!forced_iters && cauchy < eps[k]) break;
    }
    if (iters_out) iters_out[k] = nk;
  }
  memcpy(s_out, s, sizeof(double) * n3);
  if (alm_out) memcpy(alm_out, a, sizeof(double) * 6 * nalm);
  free(w); free(t); free(s); free(sn); free(r); free(a); free(ar); free(coef);
  return it;
}

/* chi^2 of Eq. 3 for a solution (map s, alm a): (d-s)^T N^{-1} (d-s) over
 * observed pixel-components plus a^dagger S^{-1} a over the harmonic modes of
 * a real field (m = 0 once, m > 0 twice), S^{-1} taken on the non-zero
 * eigenvalues of the per-l block of Eq. 10. */
/* a^dagger S^-1 a over the harmonic modes of a real field (m = 0 once,
 * m > 0 twice), S^-1 on the non-zero eigenvalues of each l's block */
static double chi2_prior(int lmax, const double *cl, const double *alm) {
  long nalm = orc_nalm(lmax);
  double chi = 0.0;
  const double *tt = cl, *ee = cl + (lmax + 1), *bb = cl + 2 * (lmax + 1), *te = cl + 3 * (lmax + 1);
  for (int l = 0; l <= lmax; ++l) {
    double e1, e2, v1[2], v2[2];
    eig2(tt[l], te[l], ee[l], &e1, &e2, v1, v2);
    for (int m = 0; m <= l; ++m) {
      long ix = orc_almidx(lmax, l, m);
      double wm = (m == 0) ? 1.0 : 2.0;
      for (int p = 0; p < 2; ++p) {
        double at = alm[2 * ix + p], ae = alm[2 * (nalm + ix) + p], ab = alm[2 * (2 * nalm + ix) + p];
        double p1 = v1[0] * at + v1[1] * ae, p2 = v2[0] * at + v2[1] * ae;
        if (e1 > 0) chi += wm * p1 * p1 / e1;
        if (e2 > 0) chi += wm * p2 * p2 / e2;
        if (bb[l] > 0) chi += wm * ab * ab / bb[l];
      }
    }
  }
  return chi;
}

double orc_chi2(int nside, int lmax, const double *cl, const double *sigma, const uint8_t *mask,
                const double *d, const double *s, const double *alm) {
  long npix = orc_npix(nside);
  double chi = 0.0;
  for (int f = 0; f < 3; ++f)
    for (long p = 0; p < npix; ++p)
      if (!mask || mask[p]) {
        double r = d[f * npix + p] - s[f * npix + p];
        double n = sigma[f * npix + p] * sigma[f * npix + p];
        chi += r * r / n;
      }
  return chi + chi2_prior(lmax, cl, alm);
}

/* ------------------------------------------------------------------------ */
/* Correlated noise with distinct temperature and polarisation masks           */
/* (the 3x3 per-pixel noise covariance of Section 2.1 and Appendix B).         */
/*                                                                              */
/* Per pixel N = Sigma C Sigma, Sigma = diag(sigma_I, sigma_Q, sigma_U) and C  */
/* the unit-diagonal correlation matrix of (rho_IQ, rho_IU, rho_QU).  Masked    */
/* components carry Sigma^{-1} = 0 (Appendix B): maskT for I, maskP for Q, U,  */
/* so N^{-1} = Sigma^{-1} C^{-1} Sigma^{-1} has zero rows and columns there.    */
/* T = alpha 1, alpha the smallest eigenvalue of N (Algorithm 1), taken over   */
/* the observed components of each pixel: alpha = min_i 1 / lambda_max(N_i^{-1}).*/
/* The messenger equation of Appendix B,                                        */
/*   t = (Nbar^{-1} + T^{-1})^{-1} (T^{-1} s + Nbar^{-1} d),  Nbar = N - T,     */
/* written with Nbar^{-1} = Sigma^{-1} P^T (Delta - alpha P Sigma^{-2} P^T)^{-1} */
/* P Sigma^{-1} (C = P^T Delta P), equals t = s + W (d - s) with               */
/* W = alpha N^{-1}: with G = Sigma^{-1} P^T and M = Delta - alpha G^T G,       */
/* (G M^{-1} G^T + 1/alpha)^{-1} G M^{-1} G^T = alpha G (M + alpha G^T G)^{-1} G^T */
/* = alpha G Delta^{-1} G^T.  The last form needs no M^{-1}, so it also holds  */
/* in the corner case Nbar = 0 of Section 2.1, where W has eigenvalue 1 and    */
/* t = d along that direction.                                                   */
/* ------------------------------------------------------------------------ */

/* Largest eigenvalue of a symmetric 3x3 matrix (cyclic Jacobi rotations). */
static double eigmax3(const double A_in[9]) {
  double A[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[i][j] = A_in[3 * i + j];
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
    double scale = fabs(A[0][0]) + fabs(A[1][1]) + fabs(A[2][2]);
    if (off <= 1e-300 || off <= 1e-17 * scale) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < 3; ++k) {  /* A <- A J */
          double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - sn * akq;
          A[k][q] = sn * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {  /* A <- J^T A */
          double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - sn * aqk;
          A[q][k] = sn * apk + c * aqk;
        }
      }
  }
  double e = A[0][0];
  if (A[1][1] > e) e = A[1][1];
  if (A[2][2] > e) e = A[2][2];
  return e;
}

/* ninv[p][9] = N_p^{-1} (row-major 3x3, components I, Q, U). */
void orc_cov_ninv(long npix, const double *sigma, const double *rho, const uint8_t *maskT, const uint8_t *maskP,
                  double *ninv) {
  for (long p = 0; p < npix; ++p) {
    const double r01 = rho[p], r02 = rho[npix + p], r12 = rho[2 * npix + p];
    /* C^{-1} by cofactors (C symmetric, unit diagonal) */
    const double c00 = 1.0 - r12 * r12, c11 = 1.0 - r02 * r02, c22 = 1.0 - r01 * r01;
    const double c01 = r02 * r12 - r01, c02 = r01 * r12 - r02, c12 = r01 * r02 - r12;
    const double det = 1.0 + 2.0 * r01 * r02 * r12 - r01 * r01 - r02 * r02 - r12 * r12;
    const double ci[9] = {c00 / det, c01 / det, c02 / det, c01 / det, c11 / det, c12 / det,
                          c02 / det, c12 / det, c22 / det};
    double si[3];
    si[0] = (!maskT || maskT[p]) ? 1.0 / sigma[p] : 0.0;
    si[1] = (!maskP || maskP[p]) ? 1.0 / sigma[npix + p] : 0.0;
    si[2] = (!maskP || maskP[p]) ? 1.0 / sigma[2 * npix + p] : 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) ninv[9 * p + 3 * i + j] = si[i] * ci[3 * i + j] * si[j];
  }
}

double orc_cov_alpha(long npix, const double *ninv) {
  double a = INFINITY;
  for (long p = 0; p < npix; ++p) {
    const double e = eigmax3(ninv + 9 * p);
    if (e > 0.0 && 1.0 / e < a) a = 1.0 / e;
  }
  return a;
}

/* t = s + alpha N^{-1} (d - s), per pixel over its three components. */
void orc_messenger_update_cov(long npix, double alpha, const double *ninv, const double *d, const double *s,
                              double *t) {
  for (long p = 0; p < npix; ++p) {
    double r[3];
    for (int i = 0; i < 3; ++i) r[i] = d[i * npix + p] - s[i * npix + p];
    for (int i = 0; i < 3; ++i) {
      double acc = 0.0;
      for (int j = 0; j < 3; ++j) acc += ninv[9 * p + 3 * i + j] * r[j];
      t[i * npix + p] = s[i * npix + p] + alpha * acc;
    }
  }
}

/* The dual messenger loop of orc_dm_solve with the noise model above: the
 * same harmonic step, synthesis, Cauchy test and level control; the
 * messenger update is orc_messenger_update_cov, and t_0 is d on the observed
 * components (0 on masked ones). */
int orc_dm_solve_cov(int nside, int lmax, const double *cl, const double *sigma, const double *rho,
                     const uint8_t *maskT, const uint8_t *maskP, const double *d, int nlev, const double *lambdas,
                     const double *eps, const int *forced_iters, int max_iter, double *s_out, double *alm_out,
                     int *iters_out, double *cauchy_out) {
  long npix = orc_npix(nside), nalm = orc_nalm(lmax);
  long n3 = 3 * npix;
  double *ninv = malloc(sizeof(double) * 9 * npix);
  orc_cov_ninv(npix, sigma, rho, maskT, maskP, ninv);
  double alpha = orc_cov_alpha(npix, ninv);
  double omega = 4.0 * M_PI / (double)npix;
  double th = alpha * omega;
  double *t = malloc(sizeof(double) * n3), *s = malloc(sizeof(double) * n3), *sn = malloc(sizeof(double) * n3);
  double *r = malloc(sizeof(double) * n3);
  double *a = malloc(sizeof(double) * 6 * nalm), *ar = malloc(sizeof(double) * 6 * nalm);
  double *coef = malloc(sizeof(double) * 4 * (lmax + 1));
  for (long p = 0; p < npix; ++p) {
    const int obs[3] = {!maskT || maskT[p], !maskP || maskP[p], !maskP || maskP[p]};
    for (int f = 0; f < 3; ++f) {
      s[f * npix + p] = 0.0;
      t[f * npix + p] = obs[f] ? d[f * npix + p] : 0.0;
    }
  }
  memset(a, 0, sizeof(double) * 6 * nalm);
  int it = 0;
  for (int k = 0; k < nlev; ++k) {
    double mu = (lambdas[k] - 1.0) * th;
    orc_filter_coefs(lmax, cl, mu, th, coef);
    int nk = 0;
    for (;;) {
      if (!forced_iters && it >= max_iter) break;
      if (forced_iters && nk >= forced_iters[k]) break;
      for (long i = 0; i < n3; ++i) r[i] = t[i] - s[i];
      orc_map2alm(nside, lmax, r, ar);
      for (long i = 0; i < 6 * nalm; ++i) a[i] += ar[i];
      orc_apply_filter(lmax, coef, a);
      orc_alm2map(nside, lmax, a, sn);
      double dd = 0.0, ss = 0.0;
      for (long i = 0; i < n3; ++i) {
        dd += (sn[i] - s[i]) * (sn[i] - s[i]);
        ss += sn[i] * sn[i];
      }
      double cauchy = (ss > 0.0) ? sqrt(dd / ss) : 0.0;
      memcpy(s, sn, sizeof(double) * n3);
      orc_messenger_update_cov(npix, alpha, ninv, d, s, t);
      if (cauchy_out && it < max_iter) cauchy_out[it] = cauchy;
      ++it;
      ++nk;
      if (!forced_iters && cauchy < eps[k]) break;
    }
    if (iters_out) iters_out[k] = nk;
  }
  memcpy(s_out, s, sizeof(double) * n3);
  if (alm_out) memcpy(alm_out, a, sizeof(double) * 6 * nalm);
  free(ninv); free(t); free(s); free(sn); free(r); free(a); free(ar); free(coef);
  return it;
}

/* ------------------------------------------------------------------------ */
/* Constrained realisations (Section 2.2, Eq. 19):                             */
/*   s_CR = W(d - dhat) + shat,  shat = Y ahat with ahat ~ S,                  */
/*   dhat = shat + nhat with nhat ~ N on observed pixels.                      */
/* The draws come from Philox4x32-10 (Salmon et al. 2011) keyed by the seed.   */
/* ------------------------------------------------------------------------ */

static uint32_t mulhilo32(uint32_t a, uint32_t b, uint32_t *hi) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  return (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t hi0, hi1;
    uint32_t lo0 = mulhilo32(0xD2511F53u, c[0], &hi0);
    uint32_t lo1 = mulhilo32(0xCD9E8D57u, c[2], &hi1);
    uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/* Two standard normals from one Philox block: two 53-bit uniforms in (0,1)
 * from words (0,1) and (2,3), then Box-Muller. */
void orc_gauss_pair(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, double *z0, double *z1) {
  uint32_t ctr[4] = {c0, c1, c2, 0u}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)}, o[4];
  orc_philox4x32_10(ctr, key, o);
  double u1 = ((double)(((uint64_t)(o[0] >> 5) << 26) | (o[1] >> 6)) + 0.5) * 0x1.0p-53;
  double u2 = ((double)(((uint64_t)(o[2] >> 5) << 26) | (o[3] >> 6)) + 0.5) * 0x1.0p-53;
  double r = sqrt(-2.0 * log(u1));
  *z0 = r * cos(2.0 * M_PI * u2);
  *z1 = r * sin(2.0 * M_PI * u2);
}

/* ahat: per (l, m) (m-major index i) blocks (i, j, 0) for j = 0, 1, 2 give
 * unit normals for T, E, B (re from z0, im from z1).  ahat = L z with L the
 * Cholesky factor of [[TT, TE], [TE, EE]] and sqrt(BB) for B; m = 0 takes the
 * real part at full variance, m > 0 re and im each at half variance. */
void orc_draw_signal_alm(int lmax, const double *cl, uint64_t seed, double *alm) {
  long nalm = orc_nalm(lmax);
  const double *tt = cl, *ee = cl + (lmax + 1), *bb = cl + 2 * (lmax + 1), *te = cl + 3 * (lmax + 1);
  for (int m = 0; m <= lmax; ++m)
    for (int l = m; l <= lmax; ++l) {
      long ix = orc_almidx(lmax, l, m);
      double zt[2], ze[2], zb[2];
      orc_gauss_pair(seed, (uint32_t)ix, 0u, 0u, &zt[0], &zt[1]);
      orc_gauss_pair(seed, (uint32_t)ix, 1u, 0u, &ze[0], &ze[1]);
      orc_gauss_pair(seed, (uint32_t)ix, 2u, 0u, &zb[0], &zb[1]);
      double l11 = sqrt(tt[l] > 0 ? tt[l] : 0.0);
      double l21 = (l11 > 0.0) ? te[l] / l11 : 0.0;
      double r22 = ee[l] - l21 * l21;
      double l22 = sqrt(r22 > 0 ? r22 : 0.0);
      double lbb = sqrt(bb[l] > 0 ? bb[l] : 0.0);
      double sc = (m == 0) ? 1.0 : sqrt(0.5);
      for (int p = 0; p < 2; ++p) {
        double ft = (m == 0 && p == 1) ? 0.0 : sc;
        alm[2 * ix + p] = ft * l11 * zt[p];
        alm[2 * (nalm + ix) + p] = ft * (l21 * zt[p] + l22 * ze[p]);
        alm[2 * (2 * nalm + ix) + p] = ft * lbb * zb[p];
      }
    }
}

/* nhat: per pixel p blocks (p, 0, 1) -> (I, Q) and (p, 1, 1) -> (U, unused);
 * nhat = sigma z on observed pixels, 0 on masked ones. */
void orc_draw_noise(int nside, const double *sigma, const uint8_t *mask, uint64_t seed, double *n) {
  long npix = orc_npix(nside);
  for (long p = 0; p < npix; ++p) {
    double z0, z1, z2, z3;
    orc_gauss_pair(seed, (uint32_t)p, 0u, 1u, &z0, &z1);
    orc_gauss_pair(seed, (uint32_t)p, 1u, 1u, &z2, &z3);
    int obs = (!mask || mask[p]);
    n[p] = obs ? sigma[p] * z0 : 0.0;
    n[npix + p] = obs ? sigma[npix + p] * z1 : 0.0;
    n[2 * npix + p] = obs ? sigma[2 * npix + p] * z2 : 0.0;
  }
}

/* shat = Y ahat and dhat = shat + nhat (masked pixels of dhat set to 0). */
void orc_cr_inputs(int nside, int lmax, const double *cl, const double *sigma, const uint8_t *mask,
                   uint64_t seed, double *ahat, double *shat, double *dhat) {
  long npix = orc_npix(nside);
  orc_draw_signal_alm(lmax, cl, seed, ahat);
  orc_alm2map(nside, lmax, ahat, shat);
  orc_draw_noise(nside, sigma, mask, seed, dhat);
  for (int f = 0; f < 3; ++f)
    for (long p = 0; p < npix; ++p) {
      long i = f * npix + p;
      dhat[i] = (!mask || mask[p]) ? shat[i] + dhat[i] : 0.0;
    }
}


/* ------------------------------------------------------------------------ */
/* Constrained-realisation inputs with the correlated noise model above.       */
/* Eq. 18 needs nhat drawn with the covariance the solve's precision implies.  */
/* On a fully observed pixel that is N = Sigma C Sigma: nhat = Sigma x with    */
/* x = L z, C = L L^T (Cholesky) and z the three normals of orc_draw_noise     */
/* (the same Philox counters). Where Sigma^{-1} = 0 on some components the     */
/* precision of the observed block o is (Sigma^{-1} C^{-1} Sigma^{-1})_oo,     */
/* whose inverse is Sigma_o (C_oo - C_om C_mm^{-1} C_mo) Sigma_o: the          */
/* covariance of x_o given x_m = 0, drawn as x_o - C_om C_mm^{-1} x_m. Masked  */
/* components are 0; dhat = shat + nhat on observed components.               */
/* ------------------------------------------------------------------------ */
void orc_draw_noise_cov(int nside, const double *sigma, const double *rho, const uint8_t *maskT,
                        const uint8_t *maskP, uint64_t seed, double *n) {
  long npix = orc_npix(nside);
  for (long p = 0; p < npix; ++p) {
    double z[4];
    orc_gauss_pair(seed, (uint32_t)p, 0u, 1u, &z[0], &z[1]);
    orc_gauss_pair(seed, (uint32_t)p, 1u, 1u, &z[2], &z[3]);
    const double r01 = rho[p], r02 = rho[npix + p], r12 = rho[2 * npix + p];
    /* Cholesky factor of the correlation matrix, row by row */
    const double l10 = r01, l20 = r02;
    const double l11 = sqrt(1.0 - l10 * l10);
    const double l21 = (r12 - l20 * l10) / l11;
    const double l22 = sqrt(1.0 - l20 * l20 - l21 * l21);
    double x[3] = {z[0], l10 * z[0] + l11 * z[1], l20 * z[0] + l21 * z[1] + l22 * z[2]};
    const int ot = !maskT || maskT[p], op = !maskP || maskP[p];
    if (!ot && op) { /* m = {I}: C_mm = 1, C_om = (r01, r02) */
      x[1] -= r01 * x[0];
      x[2] -= r02 * x[0];
    } else if (ot && !op) { /* m = {Q, U}: C_mm^{-1} = [[1, -r12], [-r12, 1]] / (1 - r12^2) */
      const double y1 = (x[1] - r12 * x[2]) / (1.0 - r12 * r12);
      const double y2 = (x[2] - r12 * x[1]) / (1.0 - r12 * r12);
      x[0] -= r01 * y1 + r02 * y2;
    }
    n[p] = ot ? sigma[p] * x[0] : 0.0;
    n[npix + p] = op ? sigma[npix + p] * x[1] : 0.0;
    n[2 * npix + p] = op ? sigma[2 * npix + p] * x[2] : 0.0;
  }
}

void orc_cr_inputs_cov(int nside, int lmax, const double *cl, const double *sigma, const double *rho,
                       const uint8_t *maskT, const uint8_t *maskP, uint64_t seed, double *ahat, double *shat,
                       double *dhat) {
  long npix = orc_npix(nside);
  orc_draw_signal_alm(lmax, cl, seed, ahat);
  orc_alm2map(nside, lmax, ahat, shat);
  orc_draw_noise_cov(nside, sigma, rho, maskT, maskP, seed, dhat);
  for (int f = 0; f < 3; ++f)
    for (long p = 0; p < npix; ++p) {
      const int obs = f == 0 ? (!maskT || maskT[p]) : (!maskP || maskP[p]);
      long i = f * npix + p;
      dhat[i] = obs ? shat[i] + dhat[i] : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* The modified Jacobi refinement of Appendix A, in the harmonic form the     */
/* sphere allows: a <- a + W~(P g(a)).                                         */
/* - W~ is the dual messenger operator at the per-level iteration counts of   */
/*   the usual solve, driven by a harmonic source g instead of data: from     */
/*   a = 0, counts[k] times a <- F_k [a + g - A(w Y a)].  With g = A(w d) this */
/*   is the iteration of orc_dm_solve after its first step.                    */
/* - g(a) = A(w (d - Y a)) - alpha Omega C^+ a is the harmonic image of the    */
/*   correction's data term w d - T Z, where T Z = alpha (S^+ + N^-1) s is     */
/*   Appendix A's rewriting of the data term of W^+ s = N (S^-1 + N^-1) s; on  */
/*   the sphere A S^+ (Y a) = Omega C^+ a, so no pixel-space inverse is needed. */
/*   At the fixed point of the usual iteration at lambda = 1, g = 0 on the    */
/*   range of C (there F^-1 a = a + A(w(d - Y a)) with F = C (C + T_h)^-1).     */
/* - P projects onto the range of each l's block: along its null directions   */
/*   (C_0^TT = 0, E and B below l = 2) no equation holds, yet W~ at mu > 0     */
/*   would pass them.                                                          */
/* ------------------------------------------------------------------------ */

/* Per-l pseudo-inverse C^+ and range projector of the (TT, TE, EE; BB) block,
 * in the [4(lmax+1)] layout orc_apply_filter takes. */
void orc_cl_pinv(int lmax, const double *cl, double *pinv, double *proj) {
  const double *tt = cl, *ee = cl + (lmax + 1), *bb = cl + 2 * (lmax + 1), *te = cl + 3 * (lmax + 1);
  for (int l = 0; l <= lmax; ++l) {
    double e1, e2, v1[2], v2[2];
    eig2(tt[l], te[l], ee[l], &e1, &e2, v1, v2);
    const double i1 = e1 > 0.0 ? 1.0 / e1 : 0.0, i2 = e2 > 0.0 ? 1.0 / e2 : 0.0;
    const double p1 = e1 > 0.0 ? 1.0 : 0.0, p2 = e2 > 0.0 ? 1.0 : 0.0;
    pinv[4 * l + 0] = i1 * v1[0] * v1[0] + i2 * v2[0] * v2[0];
    pinv[4 * l + 1] = i1 * v1[0] * v1[1] + i2 * v2[0] * v2[1];
    pinv[4 * l + 2] = i1 * v1[1] * v1[1] + i2 * v2[1] * v2[1];
    pinv[4 * l + 3] = bb[l] > 0.0 ? 1.0 / bb[l] : 0.0;
    proj[4 * l + 0] = p1 * v1[0] * v1[0] + p2 * v2[0] * v2[0];
    proj[4 * l + 1] = p1 * v1[0] * v1[1] + p2 * v2[0] * v2[1];
    proj[4 * l + 2] = p1 * v1[1] * v1[1] + p2 * v2[1] * v2[1];
    proj[4 * l + 3] = bb[l] > 0.0 ? 1.0 : 0.0;
  }
}

/* g = P [A(w (d - Y a)) - alpha Omega C^+ a] */
void orc_jacobi_source(int nside, int lmax, const double *cl, const double *sigma, const uint8_t *mask,
                       const double *d, const double *alm, double *g) {
  long npix = orc_npix(nside), nalm = orc_nalm(lmax), n3 = 3 * npix;
  double alpha = orc_alpha(npix, sigma, mask);
  double omega = 4.0 * M_PI / (double)npix;
  double *w = malloc(sizeof(double) * n3), *s = malloc(sizeof(double) * n3);
  double *ca = malloc(sizeof(double) * 6 * nalm);
  double *pinv = malloc(sizeof(double) * 4 * (lmax + 1)), *proj = malloc(sizeof(double) * 4 * (lmax + 1));
  orc_weights(npix, sigma, mask, alpha, w);
  orc_cl_pinv(lmax, cl, pinv, proj);
  orc_alm2map(nside, lmax, alm, s);
  for (long i = 0; i < n3; ++i) s[i] = w[i] * (d[i] - s[i]);
  orc_map2alm(nside, lmax, s, g);
  memcpy(ca, alm, sizeof(double) * 6 * nalm);
  orc_apply_filter(lmax, pinv, ca);
  for (long i = 0; i < 6 * nalm; ++i) g[i] -= alpha * omega * ca[i];
  orc_apply_filter(lmax, proj, g);
  free(w); free(s); free(ca); free(pinv); free(proj);
}

/* a = W~(g): from a = 0, counts[k] times a <- F_k [a + g - A(w Y a)]. */
void orc_dm_frozen(int nside, int lmax, const double *cl, const double *sigma, const uint8_t *mask,
                   const double *g, int nlev, const double *lambdas, const int *counts, double *alm) {
  long npix = orc_npix(nside), nalm = orc_nalm(lmax), n3 = 3 * npix;
  double alpha = orc_alpha(npix, sigma, mask);
  double th = alpha * 4.0 * M_PI / (double)npix;
  double *w = malloc(sizeof(double) * n3), *s = malloc(sizeof(double) * n3);
  double *ar = malloc(sizeof(double) * 6 * nalm), *coef = malloc(sizeof(double) * 4 * (lmax + 1));
  orc_weights(npix, sigma, mask, alpha, w);
  memset(alm, 0, sizeof(double) * 6 * nalm);
  for (int k = 0; k < nlev; ++k) {
    orc_filter_coefs(lmax, cl, (lambdas[k] - 1.0) * th, th, coef);
    for (int it = 0; it < counts[k]; ++it) {
      orc_alm2map(nside, lmax, alm, s);
      for (long i = 0; i < n3; ++i) s[i] *= w[i];
      orc_map2alm(nside, lmax, s, ar);
      for (long i = 0; i < 6 * nalm; ++i) alm[i] += g[i] - ar[i];
      orc_apply_filter(lmax, coef, alm);
    }
  }
  free(w); free(s); free(ar); free(coef);
}

/* ------------------------------------------------------------------------ */
/* True residual of the Wiener-filter equation, the diagnostic the paper      */
/* reports beside its solutions (Section 3.2, Appendix C): ||A x - y|| / ||y|| */
/* with A = 1 + S^1/2 Y^T N^-1 Y S^1/2, x = S^-1/2 a, y = S^1/2 Y^T N^-1 d.    */
/* In the iteration's own terms Y^T N^-1 (d - Y a) - S^-1 a is proportional   */
/* to g(a) = A(w (d - Y a)) - alpha Omega C^+ a and Y^T N^-1 d to A(w d), so   */
/* the ratio is ||C^1/2 g|| / ||C^1/2 A(w d)|| with each (l, m > 0) counted    */
/* twice (its -m partner) and C^1/2 per l from the (TT, TE, EE; BB) block.     */
/* ------------------------------------------------------------------------ */
static double weighted_half_norm2(int lmax, const double *half, const double *alm) {
  long nalm = orc_nalm(lmax);
  double acc = 0.0;
  for (int m = 0; m <= lmax; ++m)
    for (int l = m; l <= lmax; ++l) {
      long ix = orc_almidx(lmax, l, m);
      const double *c = half + 4 * l;
      const double fac = m == 0 ? 1.0 : 2.0;
      for (int p = 0; p < 2; ++p) {
        double t = alm[2 * ix + p], e = alm[2 * (nalm + ix) + p], b = alm[2 * (2 * nalm + ix) + p];
        double ht = c[0] * t + c[1] * e, he = c[1] * t + c[2] * e, hb = c[3] * b;
        acc += fac * (ht * ht + he * he + hb * hb);
      }
    }
  return acc;
}

/* ||C^1/2 (A r - alpha Omega C^+ a)|| / ||C^1/2 A y|| for the weighted pixel
 * maps r = W (d - Y a) and y = W d (each (l, m > 0) counted twice). */
static double residual_ratio(int nside, int lmax, const double *cl, double alpha, const double *r, const double *y,
                             const double *alm) {
  long nalm = orc_nalm(lmax);
  const double *tt = cl, *ee = cl + (lmax + 1), *bb = cl + 2 * (lmax + 1), *te = cl + 3 * (lmax + 1);
  double omega = 4.0 * M_PI / (double)orc_npix(nside);
  double *g = malloc(sizeof(double) * 6 * nalm), *ya = malloc(sizeof(double) * 6 * nalm);
  double *ca = malloc(sizeof(double) * 6 * nalm);
  double *pinv = malloc(sizeof(double) * 4 * (lmax + 1)), *proj = malloc(sizeof(double) * 4 * (lmax + 1));
  double *half = malloc(sizeof(double) * 4 * (lmax + 1));
  orc_cl_pinv(lmax, cl, pinv, proj);
  for (int l = 0; l <= lmax; ++l) {
    double e1, e2, v1[2], v2[2];
    eig2(tt[l], te[l], ee[l], &e1, &e2, v1, v2);
    const double r1 = e1 > 0.0 ? sqrt(e1) : 0.0, r2 = e2 > 0.0 ? sqrt(e2) : 0.0;
    half[4 * l + 0] = r1 * v1[0] * v1[0] + r2 * v2[0] * v2[0];
    half[4 * l + 1] = r1 * v1[0] * v1[1] + r2 * v2[0] * v2[1];
    half[4 * l + 2] = r1 * v1[1] * v1[1] + r2 * v2[1] * v2[1];
    half[4 * l + 3] = bb[l] > 0.0 ? sqrt(bb[l]) : 0.0;
  }
  orc_map2alm(nside, lmax, y, ya);
  orc_map2alm(nside, lmax, r, g);
  memcpy(ca, alm, sizeof(double) * 6 * nalm);
  orc_apply_filter(lmax, pinv, ca);
  for (long i = 0; i < 6 * nalm; ++i) g[i] -= alpha * omega * ca[i];
  const double num = weighted_half_norm2(lmax, half, g), den = weighted_half_norm2(lmax, half, ya);
  free(g); free(ya); free(ca); free(pinv); free(proj); free(half);
  return den > 0.0 ? sqrt(num / den) : 0.0;
}

double orc_wf_residual(int nside, int lmax, const double *cl, const double *sigma, const uint8_t *mask,
                       const double *d, const double *alm) {
  long npix = orc_npix(nside), n3 = 3 * npix;
  double alpha = orc_alpha(npix, sigma, mask);
  double *w = malloc(sizeof(double) * n3), *r = malloc(sizeof(double) * n3), *y = malloc(sizeof(double) * n3);
  orc_weights(npix, sigma, mask, alpha, w);
  orc_alm2map(nside, lmax, alm, r);
  for (long i = 0; i < n3; ++i) {
    y[i] = w[i] * d[i];
    r[i] = w[i] * (d[i] - r[i]);
  }
  const double out = residual_ratio(nside, lmax, cl, alpha, r, y, alm);
  free(w); free(r); free(y);
  return out;
}

/* chi^2 of Eq. 3 with the correlated noise model: (d - s)^T N^-1 (d - s) with
 * the per-pixel block N^-1 (zero rows and columns on masked components), plus
 * the prior term of orc_chi2. */
double orc_chi2_cov(int nside, int lmax, const double *cl, const double *sigma, const double *rho,
                    const uint8_t *maskT, const uint8_t *maskP, const double *d, const double *s,
                    const double *alm) {
  long npix = orc_npix(nside);
  double *ninv = malloc(sizeof(double) * 9 * npix);
  orc_cov_ninv(npix, sigma, rho, maskT, maskP, ninv);
  double chi = 0.0;
  for (long p = 0; p < npix; ++p) {
    double r[3];
    for (int f = 0; f < 3; ++f) r[f] = d[f * npix + p] - s[f * npix + p];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) chi += r[a] * ninv[9 * p + 3 * a + b] * r[b];
  }
  free(ninv);
  return chi + chi2_prior(lmax, cl, alm);
}

/* The same with the correlated noise model: W = alpha N^-1 per pixel (3 x 3). */
double orc_wf_residual_cov(int nside, int lmax, const double *cl, const double *sigma, const double *rho,
                           const uint8_t *maskT, const uint8_t *maskP, const double *d, const double *alm) {
  long npix = orc_npix(nside), n3 = 3 * npix;
  double *ninv = malloc(sizeof(double) * 9 * npix), *s = malloc(sizeof(double) * n3);
  double *r = malloc(sizeof(double) * n3), *y = malloc(sizeof(double) * n3), *z = malloc(sizeof(double) * n3);
  orc_cov_ninv(npix, sigma, rho, maskT, maskP, ninv);
  double alpha = orc_cov_alpha(npix, ninv);
  orc_alm2map(nside, lmax, alm, s);
  memset(z, 0, sizeof(double) * n3);
  orc_messenger_update_cov(npix, alpha, ninv, d, z, y);  /* y = 0 + alpha N^-1 (d - 0) */
  orc_messenger_update_cov(npix, alpha, ninv, d, s, r);  /* r = s + alpha N^-1 (d - s) */
  for (long i = 0; i < n3; ++i) r[i] -= s[i];
  const double out = residual_ratio(nside, lmax, cl, alpha, r, y, alm);
  free(ninv); free(s); free(r); free(y); free(z);
  return out;
}
