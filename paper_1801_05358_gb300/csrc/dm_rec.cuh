// dm_rec.cuh -- the FP64 Legendre / Wigner-d recurrence in l of one ring
// pair, shared by every kernel that runs it on the fly (the FP64 Legendre
// stages, the table generator of the mixed modes and the allocation-free
// analysis), so that a change to the recurrence reaches all of them.
//
// Per (m, l) the coefficients come from RecCoef (dm_internal.h):
//   spin 0:  lambda_{l+1} = al x lambda_l - bl lambda_{l-1}
//   spin 2:  2lambda_{l+1} = (a x + ac) 2lambda_l - b 2lambda_{l-1}
//           -2lambda_{l+1} = (a x - ac) -2lambda_l - b -2lambda_{l-1}
// seeded at l = m (spin 0) and l = max(m, 2) (spin 2) from per-(m, pair)
// seeds; values below 2^-600 are carried as v 2^-S and advanced without
// being used until they become representable (the negligible region).
#pragma once

#include "dm_internal.h"

namespace dmwf {

// Recurrence state of one ring pair: current and previous values.
// The two spin-2 functions run as separate recurrences,
//   2lambda_{l+1} = (a x + ac) 2lambda_l - b 2lambda_{l-1},
//  -2lambda_{l+1} = (a x - ac) -2lambda_l - b -2lambda_{l-1},
// and lam+- = (2lambda +- -2lambda)/2 are formed where they are used: near the
// poles one function is many orders of magnitude below the other, and the
// coupled lam+- form would inject the large one's rounding into the small one,
// whose recurrence then amplifies it by about (l/m)^(m+2).
struct Rec {
  double l0, l1;    // lambda_l, lambda_{l-1}
  double p0, p1;    // 2lambda_l, 2lambda_{l-1}
  double q0, q1;    // -2lambda_l, -2lambda_{l-1}
  int S;            // scale: true = value * 2^-S (0 = plain)
};

// advance from l to l+1 with the coefficients of target l+1
__device__ __forceinline__ void rec_step(Rec &s, const RecCoef &c, double x) {
  double nl = fma(c.al * x, s.l0, -c.bl * s.l1);
  const double cp = fma(c.a, x, c.ac), cm = fma(c.a, x, -c.ac);
  double np = fma(cp, s.p0, -c.b * s.p1);
  double nq = fma(cm, s.q0, -c.b * s.q1);
  s.l1 = s.l0;
  s.l0 = nl;
  s.p1 = s.p0;
  s.p0 = np;
  s.q1 = s.q0;
  s.q0 = nq;
}

// negligible-region bookkeeping (only when S > 0)
__device__ __forceinline__ void rec_rescale(Rec &s) {
  const double big = 0x1p300;
  if (fabs(s.l0) > big || fabs(s.p0) > big || fabs(s.q0) > big) {
    s.l0 *= 0x1p-300; s.l1 *= 0x1p-300;
    s.p0 *= 0x1p-300; s.p1 *= 0x1p-300;
    s.q0 *= 0x1p-300; s.q1 *= 0x1p-300;
    s.S -= 300;
    if (s.S < 600) {
      double f = ldexp(1.0, -s.S);
      s.l0 *= f; s.l1 *= f; s.p0 *= f; s.p1 *= f; s.q0 *= f; s.q1 *= f;
      s.S = 0;
    }
  }
}

// Initial state at l = m.  Spin 2 starts at l0 = max(m, 2); for m < 2 its
// values are zero until the seed is injected when advancing to l = 2.
__device__ __forceinline__ void rec_init(Rec &s, const double *seed, const int *seed_exp, int m, int p,
                                         int npairs) {
  int64_t o = (int64_t)m * npairs + p;
  s.l0 = seed[3 * o];
  s.l1 = 0.0;
  s.S = seed_exp[o];
  if (m >= 2) {
    s.p0 = seed[3 * o + 1];
    s.q0 = seed[3 * o + 2];
  } else {
    s.p0 = 0.0;
    s.q0 = 0.0;
  }
  s.p1 = 0.0;
  s.q1 = 0.0;
}

__device__ __forceinline__ void rec_advance(Rec &s, const RecCoef &c, double x, int m, int l, const double *seed,
                                            int p, int npairs) {
  // l -> l+1
  if (m < 2 && l + 1 == 2) {
    int64_t o = (int64_t)m * npairs + p;
    double nl = fma(c.al * x, s.l0, -c.bl * s.l1);
    s.l1 = s.l0;
    s.l0 = nl;
    s.p1 = 0.0;
    s.q1 = 0.0;
    s.p0 = seed[3 * o + 1];
    s.q0 = seed[3 * o + 2];
  } else {
    rec_step(s, c, x);
  }
  if (s.S) rec_rescale(s);
}

}  // namespace dmwf
