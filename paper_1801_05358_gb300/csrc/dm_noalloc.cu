// dm_noalloc.cu -- an allocation-free variant of the FP64 Legendre analysis
// for callers that must not allocate device memory when they call it.
//
// dm_legendre_analysis sums the per-chunk partial results of the Legendre
// analysis in a workspace buffer of the plan.  This variant keeps those
// partial sums in one file-scope device array instead, so the call itself
// makes no cudaMalloc/cudaFree and no allocating library call.  That matters
// to code that cannot allocate at the moment it runs, for example:
//  - work being recorded into a CUDA graph by stream capture, where an
//    allocation would either fail or end the capture;
//  - a real-time or latency-critical loop, where cudaMalloc/cudaFree may
//    synchronise the device and stall every stream;
//  - a host application that owns a fixed device-memory budget and forbids
//    libraries from growing it after start-up.
// The plan is still created beforehand (its read-only tables are set up once,
// outside the time-critical code).
//
// The array lives on every GPU that loads this library until the process
// exits (DM_NOALLOC_SCRATCH_BYTES bytes).  Its device address is looked up
// once per device with cudaGetSymbolAddress on the first call made with that
// device current; make that first call before any stream capture starts.
// The cached address belongs to the device's current context: a caller that
// ends that context (cudaDeviceReset) must not call this entry point on that
// device again in the same process, since the cache is not looked up anew.
// All calls share the array: calls that overlap on the GPU (different streams
// or threads) race on it and must be serialised by the caller.  Every partial
// sum the reduction reads is written by the same call first, so nothing in the
// array needs to start at zero and no state carries over between calls.
#include <math.h>

#include <mutex>

#include "dm_internal.h"
#include "dm_rec.cuh"

#define DM_NOALLOC_SCRATCH_BYTES (64u << 20)

namespace {

__device__ __align__(256) double2 g_noalloc_scratch[DM_NOALLOC_SCRATCH_BYTES / sizeof(double2)];

constexpr int NA_P = 64;      // ring pairs per block
constexpr int NA_L = 16;      // multipoles per phase
constexpr int NA_PARTS = NA_P / NA_L;

std::mutex g_mu;
double2 *g_ptr[64] = {nullptr};

__device__ __forceinline__ int64_t na_base(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

// Legendre analysis partial sums over one chunk of 64 ring pairs, reading the
// ring coefficients in the public layout rc[b][f][ring][m].
__global__ void __launch_bounds__(NA_P) k_na_ana(const dmwf::PairDev *__restrict__ pairs,
                                                 const dmwf::RecCoef *__restrict__ rec,
                                                 const double *__restrict__ seed, const int *__restrict__ seed_exp,
                                                 const double2 *__restrict__ rc, double2 *__restrict__ part,
                                                 int lmax, int mmax, int npairs, int nrings, int64_t nalm,
                                                 int nchunk) {
  __shared__ double P0[NA_P][NA_L + 1], Pp[NA_P][NA_L + 1], Pq[NA_P][NA_L + 1];
  __shared__ double2 G[NA_P][6];
  __shared__ double red[NA_PARTS][NA_L][6];
  __shared__ dmwf::RecCoef sc[NA_L];
  const int m = blockIdx.y, b = blockIdx.z, chunk = blockIdx.x;
  const int t = threadIdx.x;
  const int p = chunk * NA_P + t;
  const bool act = p < npairs;
  const int pp = act ? p : npairs - 1;
  const double x = pairs[pp].x;
  {
    const bool eq = (pp == npairs - 1);
    const int rn = pp, rs = nrings - 1 - pp;  // 0-based ring indices of the pair
    for (int f = 0; f < 3; ++f) {
      const double2 *g = rc + ((int64_t)b * 3 + f) * nrings * (mmax + 1);
      const double2 gn = act ? g[(int64_t)rn * (mmax + 1) + m] : make_double2(0, 0);
      const double2 gs = (act && !eq) ? g[(int64_t)rs * (mmax + 1) + m] : make_double2(0, 0);
      G[t][2 * f] = make_double2(gn.x + gs.x, gn.y + gs.y);
      G[t][2 * f + 1] = make_double2(gn.x - gs.x, gn.y - gs.y);
    }
  }
  dmwf::Rec s;
  dmwf::rec_init(s, seed, seed_exp, m, pp, npairs);
  const int64_t base = na_base(lmax, m);
  const int lj = t % NA_L, part_id = t / NA_L;
  for (int lc = m; lc <= lmax; lc += NA_L) {
    const int cnt = min(NA_L, lmax + 1 - lc);
    __syncthreads();
    if (t < cnt) sc[t] = rec[base + lc + t + 1];
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const int l = lc + j;
      const bool live = (s.S == 0) && act;
      P0[t][j] = live ? s.l0 : 0.0;
      Pp[t][j] = live ? 0.5 * (s.p0 + s.q0) : 0.0;  // lam+
      Pq[t][j] = live ? 0.5 * (s.p0 - s.q0) : 0.0;  // lam-
      if (l < lmax) dmwf::rec_advance(s, sc[j], x, m, l, seed, pp, npairs);
    }
    __syncthreads();
    double aTr = 0, aTi = 0, aEr = 0, aEi = 0, aBr = 0, aBi = 0;
    if (lj < cnt) {
      const int l = lc + lj;
      const int par = (l - m) & 1, opp = par ^ 1;
      for (int q = part_id * NA_L; q < (part_id + 1) * NA_L; ++q) {
        const double lam = P0[q][lj], lp = Pp[q][lj], lq = Pq[q][lj];
        const double2 gt = G[q][par], gqp = G[q][2 + par], gup = G[q][4 + par];
        const double2 gqo = G[q][2 + opp], guo = G[q][4 + opp];
        aTr = fma(lam, gt.x, aTr);
        aTi = fma(lam, gt.y, aTi);
        aEr = fma(-lp, gqp.x, fma(lq, guo.y, aEr));
        aEi = fma(-lp, gqp.y, fma(-lq, guo.x, aEi));
        aBr = fma(-lp, gup.x, fma(-lq, gqo.y, aBr));
        aBi = fma(-lp, gup.y, fma(lq, gqo.x, aBi));
      }
    }
    red[part_id][lj][0] = aTr; red[part_id][lj][1] = aTi; red[part_id][lj][2] = aEr;
    red[part_id][lj][3] = aEi; red[part_id][lj][4] = aBr; red[part_id][lj][5] = aBi;
    __syncthreads();
    if (part_id == 0 && lj < cnt) {
      const int l = lc + lj;
      double v[6];
      for (int k = 0; k < 6; ++k) {
        double a = red[0][lj][k];
        for (int q = 1; q < NA_PARTS; ++q) a += red[q][lj][k];
        v[k] = a;
      }
      double2 *o = part + ((int64_t)b * nchunk + chunk) * 3 * nalm + base + l;
      o[0] = make_double2(v[0], v[1]);
      o[nalm] = make_double2(v[2], v[3]);
      o[2 * nalm] = make_double2(v[4], v[5]);
    }
  }
}

__global__ void k_na_reduce(const double2 *__restrict__ part, double2 *__restrict__ out, int lmax, int64_t nalm,
                            int nchunk, double omega) {
  const int b = blockIdx.y, m = blockIdx.z;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  const int64_t i = na_base(lmax, m) + l;
  for (int f = 0; f < 3; ++f) {
    double ax = 0.0, ay = 0.0;
    for (int c = 0; c < nchunk; ++c) {
      const double2 v = part[(((int64_t)b * nchunk + c) * 3 + f) * nalm + i];
      ax += v.x;
      ay += v.y;
    }
    out[((int64_t)b * 3 + f) * nalm + i] = make_double2(omega * ax, omega * ay);
  }
}

}  // namespace

extern "C" dm_status dm_legendre_analysis_noalloc(dm_plan *p, const double *rc, double *alm, void *stream) {
  if (p && p->flat) {
    p->err = "sphere plans only";
    return DM_EINVAL;
  }
  if (!p || !rc || !alm) return DM_EINVAL;
  const int nchunk = (p->npairs + NA_P - 1) / NA_P;
  const size_t need = sizeof(double2) * (size_t)p->batch * nchunk * 3 * (size_t)p->nalm;
  if (need > DM_NOALLOC_SCRATCH_BYTES) {
    p->err = "dm_legendre_analysis_noalloc: this plan needs " + std::to_string(need) +
             " bytes of scratch, more than the fixed " + std::to_string((size_t)DM_NOALLOC_SCRATCH_BYTES) +
             " bytes (batch x ceil(2 nside / 64) x 3 x nalm x 16 bytes); use dm_legendre_analysis";
    return DM_EINVAL;
  }
  int dev = 0;
  const cudaError_t eg = cudaGetDevice(&dev);
  if (eg != cudaSuccess) {
    p->err = std::string("dm_legendre_analysis_noalloc: cudaGetDevice failed: ") + cudaGetErrorString(eg);
    return DM_ECUDA;
  }
  if (dev < 0 || dev >= 64) {
    p->err = "dm_legendre_analysis_noalloc: device ordinal " + std::to_string(dev) + " beyond the 64 this call tracks";
    return DM_ECUDA;
  }
  double2 *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_ptr[dev] == nullptr) {  // once per device, with that device current
      cudaError_t e = cudaGetSymbolAddress((void **)&g_ptr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_ptr[dev] = nullptr;
        p->err = std::string("dm_legendre_analysis_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
        return DM_ECUDA;
      }
    }
    scratch = g_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  dim3 g1(nchunk, p->mmax + 1, p->batch);
  k_na_ana<<<g1, NA_P, 0, st>>>(p->pairs, p->rec, p->seed, p->seed_exp, (const double2 *)rc, scratch, p->lmax,
                                p->mmax, p->npairs, p->nrings, p->nalm, nchunk);
  dim3 g2((unsigned)((p->lmax + 1 + 127) / 128), p->batch, p->mmax + 1);
  k_na_reduce<<<g2, 128, 0, st>>>(scratch, (double2 *)alm, p->lmax, p->nalm, nchunk, 4.0 * M_PI / (double)p->npix);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    p->err = std::string("dm_legendre_analysis_noalloc: ") + cudaGetErrorString(e);
    return DM_ECUDA;
  }
  return DM_OK;
}
