// dm_setup.cu -- plan tables built once on the device: ring-pair latitudes,
// FFT phase/chirp/twiddle tables, Wigner-d recurrence coefficients and seeds,
// the per-level TEB filters (Eq. 8, Algorithm 1) and the noise weights
// w = alpha / N (Section 2, Appendix B).
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "dm_fft.cuh"
#include "dm_internal.h"

namespace dmwf {

cudaError_t dyn_smem_allow_fn(const void *func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, size_t> granted;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t &g = granted[{dev, func}];
  if (bytes <= g) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (!e) g = bytes;
  return e;
}

// ---------------------------------------------------------------- geometry
// Pair p joins northern ring i = p + 1 (1 <= i <= 2 nside) with its mirror.
__global__ void k_pairs(PairDev *pairs, int nside, int npairs) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  int i = p + 1;
  double ns = nside;
  PairDev q;
  if (i < nside) {
    q.omz = ((double)i * (double)i) / (3.0 * ns * ns);
    q.opz = 2.0 - q.omz;
    q.x = 1.0 - q.omz;
  } else {
    q.x = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * ns);
    q.omz = 1.0 - q.x;
    q.opz = 1.0 + q.x;
  }
  pairs[p] = q;
}

// e^{-i pi q / n} for n = 4i, q < 2n; table of ring length n starts at 4 i (i - 1).
__global__ void k_phase(double2 *ph, int nside) {
  int i = blockIdx.y + 1;  // ring "radius" 1..nside
  int n = 4 * i;
  int64_t off = 4LL * i * (i - 1);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 2 * n; q += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-(double)q / (double)n, &s, &c);
    ph[off + q] = make_double2(c, s);
  }
}

// Stage twiddles: tw[len - 1 + j] = e^{-i pi j / len}, len = 1, 2, 4, ..., Mtab / 2.
__global__ void k_twiddle(double2 *tw, int Mtab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Mtab - 1) return;
  const int len = 1 << (31 - __clz(i + 1));
  const int j = i + 1 - len;
  double s, c;
  sincospi(-(double)j / (double)len, &s, &c);
  tw[i] = make_double2(c, s);
}

// Bluestein chirp of one ring radius: c_j = e^{-i pi j^2 / h}, j < h, with the
// exponent reduced exactly: j^2 mod 2h (j < h <= 2^15).
__global__ void k_chirp(const RingDev *rings, const int *ring_ids, double2 *chirp) {
  const RingDev R = rings[ring_ids[blockIdx.x]];
  for (int j = threadIdx.x; j < R.h; j += blockDim.x) {
    const int k = (int)(((int64_t)j * j) % (2 * R.h));
    double s, c;
    sincospi(-(double)k / (double)R.h, &s, &c);
    chirp[R.ch_off + j] = make_double2(c, s);
  }
}

// Pass tables of the fixed-size transforms of M = 2^LOGM and radix R = 2^LR
// (dm_fft.cuh): entry off(P) + (q - 1) L + j = e^{-2 pi i j q / (R L)} for the
// DIF pass P of stride L = M / R^(P + 1) > 1, q = 1..R-1, j < L.
__global__ void k_twr(double2 *tw, int LOGM, int LR) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= fftr_tw_words(LOGM, LR)) return;
  const int R = 1 << LR;
  for (int P = 0; P < LOGM / LR; ++P) {
    const int o = fftr_tw_off(LOGM, LR, P), L = (1 << LOGM) >> (LR * (P + 1));
    if (L > 1 && i < o + (R - 1) * L) {
      const int q = (i - o) / L + 1, j = (i - o) % L;
      const int k = (j * q) % (R * L);
      double s, c;
      sincospi(-2.0 * (double)k / (double)(R * L), &s, &c);
      tw[i] = make_double2(c, s);
      return;
    }
  }
}

// Bluestein kernel spectrum for one ring length: FFT_M of b_j = e^{+i pi j^2/h}
// placed at j and M - j (|j| < h), zero elsewhere, stored in bit-reversed order
// (the order in which the ring kernel's DIF transform leaves its data).
// The Bluestein spectrum of a ring transposed for the fixed-size kernels whose
// threads hold E consecutive entries: entry E t + i moves to i (M / E) + t.
__global__ void k_bhat_t(const RingDev *rings, const int *ring_ids, const double2 *bhat, double2 *out, int E) {
  const RingDev R = rings[ring_ids[blockIdx.x]];
  const int M = R.M;
  if (M % E != 0) return;
  const int nt = M / E;
  for (int k = threadIdx.x; k < M; k += blockDim.x)
    out[R.bh_off + (int64_t)(k % E) * nt + k / E] = bhat[R.bh_off + k];
}

__global__ void k_bhat(const RingDev *rings, const int *ring_ids, const double2 *ph, double2 *bhat,
                       const double2 *twid) {
  extern __shared__ double2 sm_b[];
  RingDev R = rings[ring_ids[blockIdx.x]];
  const double2 *p = ph + R.ph_off;
  int h = R.h, M = R.M;
  int64_t n2 = 4LL * h;
  for (int j = threadIdx.x; j < M; j += blockDim.x) sm_b[spad(j)] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int j = threadIdx.x; j < h; j += blockDim.x) {
    double2 c = p[(2LL * j * j) % n2];
    double2 b = make_double2(c.x, -c.y);
    sm_b[spad(j)] = b;
    if (j > 0) sm_b[spad(M - j)] = b;
  }
  __syncthreads();
  fft_dif(sm_b, M, twid);
  for (int k = threadIdx.x; k < M; k += blockDim.x) bhat[R.bh_off + k] = sm_b[spad(k)];
}

// --------------------------------------------------- recurrence coefficients
// For target l and order m (entry idx(l, m)):
//   spin 0 (l > m): al = sqrt((4l^2-1)/(l^2-m^2)),
//                   bl = sqrt((2l+1)((l-1)^2-m^2) / ((2l-3)(l^2-m^2)))
//   spin 2 (source L = l - 1 >= max(m, 2)), R(l) = sqrt((l^2-m^2)(l^2-4)):
//     a  = sqrt((2L+3)/(2L+1)) (L+1)(2L+1) / R(L+1)
//     ac = a * 2m / (L(L+1))
//     b  = sqrt((2L+3)/(2L-1)) (L+1) R(L) / (L R(L+1))
// (three-term Wigner-d recurrence with k = -+2 written for lam+- =
//  (2lambda +- -2lambda)/2).
__global__ void k_reccoef(RecCoef *rec, int lmax, int mmax) {
  int m = blockIdx.y;
  if (m > mmax) return;
  int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2;
  for (int l = m + blockIdx.x * blockDim.x + threadIdx.x; l <= lmax; l += gridDim.x * blockDim.x) {
    RecCoef c = {0, 0, 0, 0, 0, 0};
    double dl = l, dm = m;
    if (l > m) {
      double l2m2 = dl * dl - dm * dm;
      c.al = sqrt((4.0 * dl * dl - 1.0) / l2m2);
      c.bl = sqrt((2.0 * dl + 1.0) * ((dl - 1.0) * (dl - 1.0) - dm * dm) / ((2.0 * dl - 3.0) * l2m2));
    }
    int L = l - 1;
    int l0 = m > 2 ? m : 2;
    if (L >= l0) {
      double dL = L;
      double R1 = sqrt(((dL + 1) * (dL + 1) - dm * dm) * ((dL + 1) * (dL + 1) - 4.0));
      double R0 = sqrt((dL * dL - dm * dm) * (dL * dL - 4.0));
      c.a = sqrt((2.0 * dL + 3.0) / (2.0 * dL + 1.0)) * (dL + 1.0) * (2.0 * dL + 1.0) / R1;
      c.ac = c.a * 2.0 * dm / (dL * (dL + 1.0));
      c.b = (R0 == 0.0) ? 0.0 : sqrt((2.0 * dL + 3.0) / (2.0 * dL - 1.0)) * (dL + 1.0) * R0 / (dL * R1);
    }
    rec[base + l] = c;
  }
}

// ------------------------------------------------------------------- seeds
// Per pair and m: lambda_mm, 2lambda and -2lambda at l0 = max(m, 2), carried as
// v * 2^-S.  The two spin-2 functions are kept apart (not as their half sum and
// difference lam+-): near the poles they differ by many orders of magnitude and
// the sum would lose the small one.
//   lambda_mm = prod_{j<=m} (-sqrt((2j+1)/(2j)) sin theta) / sqrt(4 pi)
//   m >= 2: 2lambda_mm = lambda_mm r tan^2(theta/2), -2lambda_mm = lambda_mm r cot^2(theta/2),
//           r = sqrt(m(m-1)/((m+1)(m+2)))
//   m < 2 : closed forms of 2lambda_2m and -2lambda_2m.
// S = 0 when the value is representable above 2^-600, else S >= 600.
__global__ void k_seeds(const PairDev *pairs, double *seed, int *seed_exp, int mmax, int npairs) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  PairDev q = pairs[p];
  double sth = sqrt(q.omz * q.opz);
  double c2 = 0.5 * q.opz, s2 = 0.5 * q.omz;  // cos^2(theta/2), sin^2(theta/2)
  double t2 = q.omz / q.opz;                   // tan^2(theta/2)
  int e = 0;
  double v = frexp(0.28209479177387814347403972578039 /* 1/sqrt(4pi) */, &e);
  const double n2 = 0.63078313050504001190 /* sqrt(5/(4pi)) */;
  double c = sqrt(c2), s = sqrt(s2);
  for (int m = 0; m <= mmax; ++m) {
    if (m > 0) {
      int de;
      v *= -sqrt((2.0 * m + 1.0) / (2.0 * m)) * sth;
      v = frexp(v, &de);
      e += de;
    }
    double l0, lp, lm;
    int S;
    if (m < 2) {
      // lambda_mm plain (m = 0, 1 are O(1)); spin-2 seeds at l = 2
      double pv, mv;
      if (m == 0) {
        pv = n2 * sqrt(6.0) * c2 * s2;          // 2lambda_20  (k = -2)
        mv = n2 * sqrt(6.0) * c2 * s2;          // -2lambda_20 (k = +2)
      } else {
        pv = -n2 * 2.0 * c * s2 * s;            // 2lambda_21 = -N2 2 c s^3
        mv = n2 * 2.0 * c2 * c * s;             // -2lambda_21 = N2 2 c^3 s
      }
      l0 = ldexp(v, e);
      lp = pv;
      lm = mv;
      S = 0;
    } else {
      double r = sqrt((double)m * (m - 1) / ((double)(m + 1) * (m + 2)));
      double pv = v * r * t2, mv = v * r / t2;
      if (e >= -600) {
        l0 = ldexp(v, e);
        lp = ldexp(pv, e);
        lm = ldexp(mv, e);
        S = 0;
      } else {
        l0 = v;
        lp = pv;
        lm = mv;
        S = -e;
      }
    }
    int64_t o = (int64_t)m * npairs + p;
    seed[3 * o + 0] = l0;
    seed[3 * o + 1] = lp;
    seed[3 * o + 2] = lm;
    seed_exp[o] = S;
  }
}

// ---------------------------------------------------------------- filters
// Per l: eigen-decomposition of [[TT, TE], [TE, EE]] (closed form), BB apart;
// f_e = max(S_e, mu) / (max(S_e, mu) + T_h); coef = (F_TT, F_TE, F_EE, F_BB).
__device__ void filter_one_l(const double *cl, int lmax, int l, double mu, double th, double *out) {
  double tt = cl[l], ee = cl[(lmax + 1) + l], bb = cl[2 * (lmax + 1) + l], te = cl[3 * (lmax + 1) + l];
  double e1, e2, v1x, v1y;
  if (te == 0.0) {
    if (tt >= ee) { e1 = tt; e2 = ee; v1x = 1.0; v1y = 0.0; }
    else { e1 = ee; e2 = tt; v1x = 0.0; v1y = 1.0; }
  } else {
    // decomposed at unit scale: the spectra fall below 1e-150 at high l, where
    // their squares and products would be subnormal and the eigenvector would
    // lose its unit length
    const double sc = fmax(fmax(fabs(tt), fabs(ee)), fabs(te));
    const double a = tt / sc, c = ee / sc, b = te / sc;
    const double hd = 0.5 * (a - c);
    const double disc = hypot(hd, b);
    const double u1 = 0.5 * (a + c) + disc;
    const double u2 = (a * c - b * b) / u1;
    const double ax = b, ay = u1 - a, bx = u1 - c, by = b;
    const double na = hypot(ax, ay), nb = hypot(bx, by);
    if (na >= nb) { v1x = ax / na; v1y = ay / na; }
    else { v1x = bx / nb; v1y = by / nb; }
    e1 = u1 * sc;
    e2 = u2 * sc;
  }
  double v2x = -v1y, v2y = v1x;
  e1 = fmax(e1, 0.0);
  e2 = fmax(e2, 0.0);
  double s1 = fmax(e1, mu), s2 = fmax(e2, mu), s3 = fmax(fmax(bb, 0.0), mu);
  double f1 = s1 / (s1 + th), f2 = s2 / (s2 + th), f3 = s3 / (s3 + th);
  out[0] = f1 * v1x * v1x + f2 * v2x * v2x;
  out[1] = f1 * v1x * v1y + f2 * v2x * v2y;
  out[2] = f1 * v1y * v1y + f2 * v2y * v2y;
  out[3] = f3;
}

__global__ void k_filter(const double *cl, int lmax, double mu, double th, double *coef, float *coef32) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  filter_one_l(cl, lmax, l, mu, th, coef + 4 * l);
  if (coef32 != nullptr)
    for (int k = 0; k < 4; ++k) coef32[4 * l + k] = (float)coef[4 * l + k];
}

// ------------------------------------------------------------------- noise
__global__ void k_min_n(const double *sigma, const uint8_t *mask, int64_t npix, double *partial) {
  __shared__ double red[256];
  double mn = INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * npix;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = i % npix;
    if (mask == nullptr || mask[p]) mn = fmin(mn, sigma[i] * sigma[i]);
  }
  red[threadIdx.x] = mn;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_min_final(double *partial, int n) {
  __shared__ double red[256];
  double mn = INFINITY;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mn = fmin(mn, partial[i]);
  red[threadIdx.x] = mn;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[0] = red[0];
}

__global__ void k_weights(const double *sigma, const uint8_t *mask, int64_t npix, const double *alpha_dev,
                          double *w) {
  double alpha = alpha_dev[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * npix;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = i % npix;
    bool obs = (mask == nullptr) || mask[p];
    w[i] = obs ? alpha / (sigma[i] * sigma[i]) : 0.0;
  }
}

// ------------------------------------------------------------- launchers
static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
static int next_pow2(int v) {
  int r = 1;
  while (r < v) r <<= 1;
  return r;
}

// e^{-i pi q / n}, q in [0, 2n), for one ring length n (flat-sky rows)
__global__ void k_phase_n(double2 *ph, int n) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 2 * n; q += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-(double)q / (double)n, &s, &c);
    ph[q] = make_double2(c, s);
  }
}

// Flat-sky geometry: the N rows of an N x N grid (row-major maps) are N
// rings of n = N pixels at phi_j = 2 pi j / N (no half-pixel shift), FFT
// size M = N / 2 (a power of two, no Bluestein), paired as (y, N - 1 - y) so
// that the paired ring kernels apply; one size class.
cudaError_t build_tables_flat(dm_plan *p) {
  const int N = p->flatN;
  p->rings_h.resize(N);
  for (int y = 0; y < N; ++y) {
    RingDev R{};
    R.start = (int64_t)y * N;
    R.n = N;
    R.h = N / 2;
    R.M = N / 2;
    R.bluestein = 0;
    R.shift = 0;
    R.pair = y < N / 2 ? y : N - 1 - y;
    R.side = y < N / 2 ? 0 : 1;
    R.ph_off = 0;
    R.bh_off = -1;
    R.ch_off = -1;
    p->rings_h[y] = R;
  }
  p->fft_M_max = N;  // the column transforms are N points (the row transforms N / 2)
  p->bh_total = 0;
  p->ch_total = 0;
  p->ring_classes.clear();
  p->ring_classes.push_back(RingClass{0, N, N / 2, N, 0, N / 2});
  p->ring_order_h.resize(N);
  for (int y = 0; y < N; ++y) p->ring_order_h[y] = y;
  p->pair_order_h.resize(N / 2);
  for (int y = 0; y < N / 2; ++y) p->pair_order_h[y] = y;
  cudaError_t e;
  if ((e = cudaMalloc(&p->rings, sizeof(RingDev) * N))) return e;
  if ((e = cudaMalloc(&p->phase, sizeof(double2) * 2 * N))) return e;
  if ((e = cudaMalloc(&p->twid, sizeof(double2) * (p->fft_M_max - 1)))) return e;
  if ((e = cudaMalloc(&p->bhat, sizeof(double2)))) return e;
  if ((e = cudaMalloc(&p->chirp, sizeof(double2)))) return e;
  if ((e = cudaMalloc(&p->ring_order, sizeof(int) * N))) return e;
  if ((e = cudaMalloc(&p->pair_order, sizeof(int) * (N / 2)))) return e;
  p->ph_total = 2 * N;
  p->bytes += sizeof(RingDev) * N + sizeof(double2) * (2 * N + p->fft_M_max + 1) + sizeof(int) * (N + N / 2);
  cudaMemcpy(p->rings, p->rings_h.data(), sizeof(RingDev) * N, cudaMemcpyHostToDevice);
  cudaMemcpy(p->ring_order, p->ring_order_h.data(), sizeof(int) * N, cudaMemcpyHostToDevice);
  cudaMemcpy(p->pair_order, p->pair_order_h.data(), sizeof(int) * (N / 2), cudaMemcpyHostToDevice);
  k_phase_n<<<(2 * N + 255) / 256, 256>>>(p->phase, N);
  k_twiddle<<<(p->fft_M_max + 255) / 256, 256>>>(p->twid, p->fft_M_max);
  {  // pass tables of the fixed-size transforms when N / 2 is 2^9 .. 2^12
    int total = 0;
    for (int r = 0; r < 2; ++r)
      for (int k = 0; k < 16; ++k) p->twr_off[r][k] = -1;
    const int logm = 31 - __builtin_clz((unsigned)(N / 2));
    if ((N / 2) == (1 << logm) && logm >= 9 && logm <= 12)
      for (int lr = 3; lr <= 4; ++lr) {
        p->twr_off[lr - 3][logm] = total;
        total += fftr_tw_words(logm, lr);
      }
    if ((e = cudaMalloc(&p->twr, sizeof(double2) * (total > 0 ? total : 1)))) return e;
    p->twr_words = total;
    p->bytes += sizeof(double2) * (total > 0 ? total : 1);
    for (int lr = 3; lr <= 4; ++lr)
      if (p->twr_off[lr - 3][logm] >= 0 && logm <= 12 && logm >= 9)
        k_twr<<<(fftr_tw_words(logm, lr) + 255) / 256, 256>>>(p->twr + p->twr_off[lr - 3][logm], logm, lr);
  }
  if ((e = cudaGetLastError())) return e;
  return cudaDeviceSynchronize();
}

// Filters of every index of spectra cl4[4][n] for one level (mu, T_h):
// coef[n][4], the per-l filter math applied to per-mode spectra.
cudaError_t build_filter_table(const double *cl4, int64_t n, double mu, double th, double *coef, cudaStream_t st) {
  k_filter<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(cl4, (int)(n - 1), mu, th, coef, nullptr);
  return cudaGetLastError();
}

cudaError_t build_tables(dm_plan *p) {
  const int ns = p->nside;
  // host-side ring metadata (integer geometry of the RING scheme)
  p->rings_h.resize(p->nrings);
  int Mmax = 1;
  for (int r = 0; r < p->nrings; ++r) {
    int i = r + 1;
    RingDev R{};
    int64_t n64 = ns;
    if (i < ns) {
      R.n = 4 * i;
      R.start = 2LL * i * (i - 1);
      R.shift = 1;
      R.pair = i - 1;
      R.side = 0;
    } else if (i <= 3 * ns) {
      R.n = 4 * ns;
      R.start = 2LL * ns * (ns - 1) + (int64_t)(i - ns) * 4 * n64;
      R.shift = ((i - ns + 1) % 2 == 1) ? 1 : 0;
      if (i <= 2 * ns) {
        R.pair = i - 1;
        R.side = 0;
      } else {
        R.pair = 4 * ns - i - 1;
        R.side = 1;
      }
    } else {
      int ip = 4 * ns - i;
      R.n = 4 * ip;
      R.start = 12LL * n64 * n64 - 2LL * ip * (ip + 1);
      R.shift = 1;
      R.pair = ip - 1;
      R.side = 1;
    }
    R.h = R.n / 2;
    R.bluestein = is_pow2(R.h) ? 0 : 1;
    R.M = R.bluestein ? next_pow2(2 * R.h - 1) : R.h;
    int rad = R.n / 4;
    R.ph_off = 4LL * rad * (rad - 1);
    R.bh_off = -1;
    R.ch_off = -1;
    Mmax = R.M > Mmax ? R.M : Mmax;
    p->rings_h[r] = R;
  }
  p->fft_M_max = Mmax < 2 ? 2 : Mmax;
  // Bluestein spectra: one per distinct ring radius (north and south share)
  std::vector<int> bl_ring;  // representative ring per radius needing bluestein
  std::vector<int64_t> bl_off_by_rad(ns + 1, -1), ch_off_by_rad(ns + 1, -1);
  int64_t bh_total = 0, ch_total = 0;
  for (int r = 0; r < p->nrings; ++r) {
    RingDev &R = p->rings_h[r];
    if (!R.bluestein) continue;
    int rad = R.n / 4;
    if (bl_off_by_rad[rad] < 0) {
      bl_off_by_rad[rad] = bh_total;
      bh_total += R.M;
      ch_off_by_rad[rad] = ch_total;
      ch_total += R.h;
      bl_ring.push_back(r);
    }
    R.bh_off = bl_off_by_rad[rad];
    R.ch_off = ch_off_by_rad[rad];
  }
  // Size classes of the ring kernel: rings sorted by FFT size M (largest first),
  // one class per M, the rings with M <= 256 together.
  {
    std::vector<int> ids(p->nrings);
    for (int r = 0; r < p->nrings; ++r) ids[r] = r;
    std::stable_sort(ids.begin(), ids.end(),
                     [&](int a, int b) { return p->rings_h[a].M > p->rings_h[b].M; });
    p->ring_classes.clear();
    int last_key = -1;
    for (int i = 0; i < p->nrings; ++i) {
      const RingDev &R = p->rings_h[ids[i]];
      const int key = R.M > 256 ? R.M : 256;
      if (key != last_key) {
        p->ring_classes.push_back(RingClass{i, 0, R.M, R.n, 0, 0});  // poff, pcount set below
        last_key = key;
      }
      RingClass &c = p->ring_classes.back();
      ++c.count;
      c.M = std::max(c.M, R.M);
      c.n = std::max(c.n, R.n);
    }
    p->ring_order_h = ids;
    // the northern (or equatorial) member of each pair, class by class: the
    // paired ring kernels take a pair per block (both members have one size)
    p->pair_order_h.clear();
    for (RingClass &c : p->ring_classes) {
      c.poff = (int)p->pair_order_h.size();
      for (int i = c.off; i < c.off + c.count; ++i)
        if (p->rings_h[ids[i]].side == 0) p->pair_order_h.push_back(ids[i]);
      c.pcount = (int)p->pair_order_h.size() - c.poff;
    }
  }
  cudaError_t e;
  size_t ph_n = 4ull * ns * (ns + 1);
  if ((e = cudaMalloc(&p->rings, sizeof(RingDev) * p->nrings))) return e;
  if ((e = cudaMalloc(&p->pairs, sizeof(PairDev) * p->npairs))) return e;
  if ((e = cudaMalloc(&p->phase, sizeof(double2) * ph_n))) return e;
  if ((e = cudaMalloc(&p->twid, sizeof(double2) * (p->fft_M_max - 1)))) return e;
  if ((e = cudaMalloc(&p->bhat, sizeof(double2) * (bh_total > 0 ? bh_total : 1)))) return e;
  p->bh_total = bh_total;
  if ((e = cudaMalloc(&p->chirp, sizeof(double2) * (ch_total > 0 ? ch_total : 1)))) return e;
  p->ch_total = ch_total;
  p->bytes += sizeof(double2) * (ch_total > 0 ? ch_total : 1);
  p->ph_total = (int64_t)ph_n;
  if ((e = cudaMalloc(&p->rec, sizeof(RecCoef) * (p->nalm + 1)))) return e;
  size_t nseed = (size_t)(p->mmax + 1) * p->npairs;
  if ((e = cudaMalloc(&p->seed, sizeof(double) * 3 * nseed))) return e;
  if ((e = cudaMalloc(&p->seed_exp, sizeof(int) * nseed))) return e;
  p->bytes += sizeof(RingDev) * p->nrings + sizeof(PairDev) * p->npairs + sizeof(double2) * ph_n +
              sizeof(double2) * (p->fft_M_max - 1 + bh_total) + sizeof(RecCoef) * (p->nalm + 1) +
              (sizeof(double) * 3 + sizeof(int)) * nseed;
  if ((e = cudaMemcpy(p->rings, p->rings_h.data(), sizeof(RingDev) * p->nrings, cudaMemcpyHostToDevice)))
    return e;
  if ((e = cudaMalloc(&p->ring_order, sizeof(int) * p->nrings))) return e;
  if ((e = cudaMemcpy(p->ring_order, p->ring_order_h.data(), sizeof(int) * p->nrings, cudaMemcpyHostToDevice)))
    return e;
  const size_t npo = p->pair_order_h.size();
  if ((e = cudaMalloc(&p->pair_order, sizeof(int) * (npo > 0 ? npo : 1)))) return e;
  if (npo > 0 &&
      (e = cudaMemcpy(p->pair_order, p->pair_order_h.data(), sizeof(int) * npo, cudaMemcpyHostToDevice)))
    return e;
  cudaMemset(p->rec, 0, sizeof(RecCoef) * (p->nalm + 1));
  k_pairs<<<(p->npairs + 127) / 128, 128>>>(p->pairs, ns, p->npairs);
  k_phase<<<dim3(8, ns), 256>>>(p->phase, ns);
  k_twiddle<<<(p->fft_M_max - 1 + 255) / 256, 256>>>(p->twid, p->fft_M_max);
  {  // pass tables of the fixed-size transforms for the sizes the ring classes use
    int total = 0;
    for (int r = 0; r < 2; ++r)
      for (int k = 0; k < 16; ++k) p->twr_off[r][k] = -1;
    for (const RingClass &c : p->ring_classes)
      for (int k = 9; k <= 12; ++k)
        if (c.M == (1 << k) && p->twr_off[0][k] < 0)
          for (int lr = 3; lr <= 4; ++lr) {
            p->twr_off[lr - 3][k] = total;
            total += fftr_tw_words(k, lr);
          }
    if ((e = cudaMalloc(&p->twr, sizeof(double2) * (total > 0 ? total : 1)))) return e;
    p->twr_words = total;
    p->bytes += sizeof(double2) * (total > 0 ? total : 1);
    for (int lr = 3; lr <= 4; ++lr)
      for (int k = 9; k <= 12; ++k)
        if (p->twr_off[lr - 3][k] >= 0)
          k_twr<<<(fftr_tw_words(k, lr) + 255) / 256, 256>>>(p->twr + p->twr_off[lr - 3][k], k, lr);
  }
  if (!bl_ring.empty()) {
    int *ids;
    if ((e = cudaMalloc(&ids, sizeof(int) * bl_ring.size()))) return e;
    cudaMemcpy(ids, bl_ring.data(), sizeof(int) * bl_ring.size(), cudaMemcpyHostToDevice);
    size_t smem = sizeof(double2) * (p->fft_M_max + p->fft_M_max / 32 + 1);  // slots spad(0..M-1)
    dyn_smem_allow(k_bhat, smem);
    k_bhat<<<(unsigned)bl_ring.size(), 256, smem>>>(p->rings, ids, p->phase, p->bhat, p->twid);
    k_chirp<<<(unsigned)bl_ring.size(), 256>>>(p->rings, ids, p->chirp);
    for (int lr = 3; lr <= 4 && !e; ++lr) {  // transposed copies for the fixed-size kernels of radix 2^lr
      if ((e = cudaMalloc(&p->bhatT[lr - 3], sizeof(double2) * bh_total))) break;
      p->bytes += (int64_t)(sizeof(double2) * bh_total);
      k_bhat_t<<<(unsigned)bl_ring.size(), 256>>>(p->rings, ids, p->bhat, p->bhatT[lr - 3], 1 << lr);
    }
    if (e) {
      cudaFree(ids);
      return e;
    }
    e = cudaDeviceSynchronize();
    cudaFree(ids);
    if (e) return e;
  }
  k_reccoef<<<dim3(4, p->mmax + 1), 256>>>(p->rec, p->lmax, p->mmax);
  k_seeds<<<(p->npairs + 63) / 64, 64>>>(p->pairs, p->seed, p->seed_exp, p->mmax, p->npairs);
  e = cudaGetLastError();
  if (e) return e;
  return cudaDeviceSynchronize();
}

__global__ void k_d2f2(const double2 *in, float2 *out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

cudaError_t gen_tables32(dm_plan *p);  // dm_legendre.cu

// Buffers of DM_MIXED_FP32 and DM_FLOAT_FLOAT: FP32 copies of the FFT tables,
// FP32 ring coefficients and maps.  The FP32 Legendre tables are not made
// here: the kernels that read them build them on first use (ensure_ptab).
cudaError_t setup_fp32(dm_plan *p) {
  if (p->fp32_ready) return cudaSuccess;  // set only after everything below succeeded
  cudaError_t e;
  // all or nothing: on any error every buffer allocated here is freed again,
  // so that a later call starts over instead of finding a half-built state
  void **owned[] = {(void **)&p->phase32, (void **)&p->bhat32, (void **)&p->bhatT32[0], (void **)&p->bhatT32[1],
                    (void **)&p->chirp32, (void **)&p->twid32,
                    (void **)&p->twr32,   (void **)&p->rc32,
                    (void **)&p->apart32, (void **)&p->s32,    (void **)&p->w32,     (void **)&p->wd32,
                    (void **)&p->a_hi,    (void **)&p->g_hi,   (void **)&p->shi32,   (void **)&p->e32,
                    (void **)&p->c32,     (void **)&p->clev,   (void **)&p->tc_err};
  // the workspace figure goes back to what it was on entry, so a failed
  // set-up (and its retries) does not inflate dm_plan_info's byte count
  const int64_t bytes_on_entry = p->bytes;
  auto undo = [&](cudaError_t err) {
    for (void **q : owned) {
      if (*q) cudaFree(*q);
      *q = nullptr;
    }
    p->bytes = bytes_on_entry;
    return err;
  };
  const int64_t B = p->batch, n3 = 3 * p->npix;
  auto al = [&](auto **ptr, size_t cnt) {
    size_t bytes = sizeof(**ptr) * (cnt > 0 ? cnt : 1);
    cudaError_t r = cudaMalloc((void **)ptr, bytes);
    if (!r) p->bytes += (int64_t)bytes;
    return r;
  };
  if ((e = al(&p->phase32, p->ph_total))) return undo(e);
  if ((e = al(&p->bhat32, p->bh_total))) return undo(e);
  if (p->bhatT[0] && (e = al(&p->bhatT32[0], p->bh_total))) return undo(e);
  if (p->bhatT[1] && (e = al(&p->bhatT32[1], p->bh_total))) return undo(e);
  if ((e = al(&p->chirp32, p->ch_total))) return undo(e);
  if ((e = al(&p->twid32, p->fft_M_max - 1))) return undo(e);
  if ((e = al(&p->twr32, p->twr_words))) return undo(e);
  if ((e = al(&p->rc32, (size_t)B * 3 * (p->mmax + 1) * p->npairs * 2))) return undo(e);
  {
    const double full = (double)B * p->nchunk * 3 * p->nalm * sizeof(float2);
    p->nchunk32 = full <= 24.0 * (1u << 30) ? p->nchunk : 1;
  }
  if ((e = al(&p->apart32, (size_t)B * p->nchunk32 * 3 * p->nalm))) return undo(e);
  if ((e = al(&p->s32, (size_t)B * n3))) return undo(e);
  if ((e = al(&p->w32, (size_t)B * n3))) return undo(e);
  if ((e = al(&p->wd32, (size_t)B * n3))) return undo(e);
  if ((e = al(&p->a_hi, (size_t)B * 3 * p->nalm))) return undo(e);
  if ((e = al(&p->g_hi, (size_t)B * 3 * p->nalm))) return undo(e);
  if ((e = al(&p->shi32, (size_t)B * n3))) return undo(e);
  if ((e = al(&p->e32, (size_t)B * 3 * p->nalm))) return undo(e);
  if ((e = al(&p->c32, (size_t)B * 3 * p->nalm))) return undo(e);
  if ((e = al(&p->clev, (size_t)B))) return undo(e);
  if ((e = al(&p->tc_err, 1))) return undo(e);
  cudaMemset(p->tc_err, 0, sizeof(int));
  cudaMemset(p->rc32, 0, sizeof(float2) * (size_t)B * 3 * (p->mmax + 1) * p->npairs * 2);
  k_d2f2<<<512, 256>>>(p->phase, p->phase32, p->ph_total);
  if (p->bh_total > 0) k_d2f2<<<512, 256>>>(p->bhat, p->bhat32, p->bh_total);
  for (int k = 0; k < 2; ++k)
    if (p->bhatT32[k]) k_d2f2<<<512, 256>>>(p->bhatT[k], p->bhatT32[k], p->bh_total);
  if (p->ch_total > 0) k_d2f2<<<512, 256>>>(p->chirp, p->chirp32, p->ch_total);
  k_d2f2<<<64, 256>>>(p->twid, p->twid32, p->fft_M_max - 1);
  if (p->twr_words > 0) k_d2f2<<<64, 256>>>(p->twr, p->twr32, p->twr_words);
  if ((e = cudaDeviceSynchronize())) return undo(e);
  p->fp32_ready = true;
  return cudaSuccess;
}

// The full FP32 Legendre tables (3 x nalm x npairs, hi and lo), made once.
cudaError_t ensure_ptab(dm_plan *p) {
  if (p->ptab) return cudaSuccess;
  const size_t n = (size_t)3 * p->nalm * p->npairs;
  float *hi = nullptr, *lo = nullptr;
  cudaError_t e = cudaMalloc(&hi, sizeof(float) * n);
  if (!e) e = cudaMalloc(&lo, sizeof(float) * n);
  if (!e) e = gen_tables32_slab(p, hi, lo, 0, p->mmax + 1, 0);
  if (!e) e = cudaDeviceSynchronize();
  if (e) {
    cudaFree(hi);
    cudaFree(lo);
    return e;
  }
  p->ptab = hi;
  p->ptab_lo = lo;
  p->bytes += (int64_t)(2 * sizeof(float) * n);
  return cudaSuccess;
}

// When coef lies in p->filt, its FP32 copy goes to the same place of p->filt32.
cudaError_t build_filter_one(dm_plan *p, double lambda, double th, double *coef, cudaStream_t st) {
  double mu = (lambda - 1.0) * th;
  float *coef32 = nullptr;
  if (p->filt32 != nullptr && p->filt != nullptr && coef >= p->filt) {
    const size_t off = (size_t)(coef - p->filt);
    const size_t len = (size_t)4 * (p->lmax + 1) * p->filt_levels * p->batch;
    if (off + (size_t)4 * (p->lmax + 1) <= len) coef32 = p->filt32 + off;
  }
  k_filter<<<(p->lmax + 1 + 127) / 128, 128, 0, st>>>(p->cl, p->lmax, mu, th, coef, coef32);
  return cudaGetLastError();
}

// filters of RHS b for every level: filt[b][k][l][4]; a flat-sky plan keeps
// one table per level for every RHS, filt[k][mode][4] (its noise is shared)
cudaError_t build_filters(dm_plan *p, int b, cudaStream_t st) {
  const int nl = (int)p->lambdas.size();
  if (p->flat) {
    if (b != 0) return cudaSuccess;
    if (p->filt == nullptr || p->filt_levels < nl) {
      if (p->filt) cudaFree(p->filt);
      p->filt = nullptr;
      cudaError_t e = cudaMalloc(&p->filt, sizeof(double) * 4 * (size_t)p->nmodes * nl);
      if (e) return e;
      p->filt_levels = nl;
    }
    for (int k = 0; k < nl; ++k) {
      const double th = p->t_h[0];
      cudaError_t e = build_filter_table(p->cl, p->nmodes, (p->lambdas[k] - 1.0) * th, th,
                                         p->filt + (size_t)k * 4 * p->nmodes, st);
      if (e) return e;
    }
    return cudaGetLastError();
  }
  if (p->filt == nullptr || p->filt_levels < nl) {
    if (p->filt) cudaFree(p->filt);
    if (p->filt32) cudaFree(p->filt32);
    p->filt = nullptr;
    p->filt32 = nullptr;
    cudaError_t e = cudaMalloc(&p->filt, sizeof(double) * 4 * (p->lmax + 1) * (size_t)nl * p->batch);
    if (e) return e;
    e = cudaMalloc(&p->filt32, sizeof(float) * 4 * (p->lmax + 1) * (size_t)nl * p->batch);
    if (e) return e;
    p->filt_levels = nl;
    // every RHS must be (re)built after a reallocation
    for (int bb = 0; bb < p->batch; ++bb)
      for (int k = 0; k < nl; ++k) {
        e = build_filter_one(p, p->lambdas[k], p->t_h[bb], p->filt + ((size_t)bb * nl + k) * 4 * (p->lmax + 1), st);
        if (e) return e;
      }
    return cudaGetLastError();
  }
  for (int k = 0; k < nl; ++k) {
    cudaError_t e = build_filter_one(p, p->lambdas[k], p->t_h[b], p->filt + ((size_t)b * p->filt_levels + k) * 4 * (p->lmax + 1), st);
    if (e) return e;
  }
  return cudaGetLastError();
}

// alpha of RHS b (min over its observed pixel-components) and its weights w
cudaError_t build_noise(dm_plan *p, int b, cudaStream_t st) {
  int nb = 256;
  double *partial;
  cudaError_t e = cudaMalloc(&partial, sizeof(double) * nb);
  if (e) return e;
  const int64_t n3 = 3 * p->npix;
  const double *sg = p->sigma + (size_t)b * n3;
  const uint8_t *mk = p->mask + (size_t)b * p->npix;
  k_min_n<<<nb, 256, 0, st>>>(sg, mk, p->npix, partial);
  k_min_final<<<1, 256, 0, st>>>(partial, nb);
  k_weights<<<1024, 256, 0, st>>>(sg, mk, p->npix, partial, p->w + (size_t)b * n3);
  double alpha = 0.0;
  cudaMemcpyAsync(&alpha, partial, sizeof(double), cudaMemcpyDeviceToHost, st);
  e = cudaStreamSynchronize(st);
  cudaFree(partial);
  if (e) return e;
  p->alpha[b] = alpha;
  p->t_h[b] = alpha * 4.0 * M_PI / (double)p->npix;
  return cudaGetLastError();
}

}  // namespace dmwf
