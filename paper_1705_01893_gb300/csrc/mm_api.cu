// C ABI of the messenger mapmaker: plan layout in the caller's workspace, set-up kernels
// (hit counts, weight blocks, pixel cut, noise tables, data spectrum), the messenger and
// PCG drivers, and the per-pixel kernels of the map step.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cstddef>
#include <map>
#include <tuple>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "mm_internal.cuh"

using namespace mm;

// ------------------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

void mm_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" const char* mm_last_error(void) { return g_err; }

#define MM_ARG(cond, ...)          \
  do {                             \
    if (!(cond)) {                 \
      mm_set_error(__VA_ARGS__);   \
      return MM_ERR_ARG;           \
    }                              \
  } while (0)

#define MM_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      mm_set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                   __LINE__);                                                      \
      return MM_ERR_CUDA;                                                          \
    }                                                                              \
  } while (0)

static inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

cudaError_t mm::resident_ctas(const void* kernel, int threads, size_t smem, int* out) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int, size_t>, int> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const auto key = std::make_tuple(kernel, dev, threads, smem);
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) { *out = it->second; return cudaSuccess; }
  }
  // allow the kernel the device's whole opt-in shared memory once, so that launches of the
  // same kernel with different tile sizes never depend on which one came first
  int optin = 0;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess) return e;
  const int dyn_max = optin - (int)fa.sharedSizeBytes;   // opt-in limit minus static shared memory
  if (dyn_max < 0 || smem > (size_t)dyn_max) return cudaErrorInvalidValue;
  if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max)) !=
      cudaSuccess)
    return e;
  int nsm = 0, occ = 0;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem)) != cudaSuccess)
    return e;
  const int r = (occ < 1 ? 1 : occ) * nsm;
  std::lock_guard<std::mutex> g(mu);
  cache[key] = r;
  *out = r;
  return cudaSuccess;
}

// ------------------------------------------------------------------------ FFT shapes
// Slots a chunk of complex length M takes in the spectrum-sized buffers (d~, Nbar, the
// adjoint's kept spectra): M rounded up to a multiple of 4, so that every chunk's block
// starts on 16 bytes of the FP32 table and 32 bytes of the complex ones (bulk prefetches
// of its rows need 16-byte alignment, whatever lengths come before it in the plan).
static inline int64_t spec_slots(int64_t M) { return (M + 3) & ~int64_t(3); }

// M = 2^p complex points per chunk (n = 2M real samples): columns M1, rows M2 = M / M1.
// Columns up to 512 points, then rows stay at 4096 (a row pair in 64 KB of shared memory,
// two CTAs per SM) and the columns grow to 1024 and 2048 points (tiles of 8 and 4 columns,
// also 64 KB).
static bool fft_shape(int64_t n, int* M, int* M1, int* M2) {
  if (n < 512 || (n & 1)) return false;
  const int64_t m = n / 2;
  if (m & (m - 1)) return false;
  int p = 0;
  while ((int64_t(1) << p) < m) ++p;
  if (p < 8 || p > 23) return false;
  constexpr int kRowLog = 12;
  int lo = p / 2;
  if (lo > 9) lo = 9;
  if (p - lo > kRowLog) lo = p - kRowLog;
  *M = (int)m;
  *M1 = 1 << lo;
  *M2 = (int)(m >> lo);
  return true;
}

static bool smooth235(int64_t x) {
  if (x < 1) return false;
  for (int f : {2, 3, 5})
    while (x % f == 0) x /= f;
  return x == 1;
}

// General path: n with prime factors 2, 3, 5 only.  Even n: M = n / 2 (packed real FFT),
// odd n: M = n (complex FFT of the real sequence).  M1 is the divisor of M nearest sqrt(M)
// with M1 <= kGenMaxM1 and M2 = M / M1 <= kGenMaxM2.
static bool gen_shape(int64_t n, int* M, int* M1, int* M2, int* cplx) {
  if (n < 4 || n > (int64_t(1) << 24) || !smooth235(n)) return false;
  const int64_t m = (n & 1) ? n : n / 2;
  int best = 0;
  double bd = 1e300;
  for (int64_t d = 1; d <= kGenMaxM1 && d <= m; ++d) {
    if (m % d || m / d > kGenMaxM2) continue;
    const double dist = fabs(log((double)d) - 0.5 * log((double)m));
    if (dist < bd) { bd = dist; best = (int)d; }
  }
  if (best == 0) return false;
  *M = (int)m;
  *M1 = best;
  *M2 = (int)(m / best);
  *cplx = (int)(n & 1);
  return true;
}

// Radix sequence of a general DFT length (any order is a valid Stockham schedule; larger
// radices mean fewer passes).  order 0: radix 8 while 8 divides, then 4 or 2, then 5s, then
// 3s; order 1: radix 4 in place of 8; order 2: the 3s and 5s first, then 8, 4, 2.
static int radix_plan(int L, int8_t* rad, int order = 0) {
  int n = 0;
  auto twos = [&]() {
    if (order != 1)
      while (L % 8 == 0 && n < kMaxRadices) { rad[n++] = 8; L /= 8; }
    while (L % 4 == 0 && n < kMaxRadices) { rad[n++] = 4; L /= 4; }
    if (L % 2 == 0 && n < kMaxRadices) { rad[n++] = 2; L /= 2; }
  };
  auto odds = [&]() {
    while (L % 5 == 0 && n < kMaxRadices) { rad[n++] = 5; L /= 5; }
    while (L % 3 == 0 && n < kMaxRadices) { rad[n++] = 3; L /= 3; }
  };
  if (order == 2) { odds(); twos(); } else { twos(); odds(); }
  return L == 1 ? n : -1;
}

static int log_lo_of(int M) {
  int p = 0;
  while ((1 << p) < M) ++p;
  return (p + 1) / 2;
}

static const int kGenLogLo = 10;

static size_t tw_count(int M, int M1, int M2, bool general) {
  // general lengths: per-pass tables of the column and row DFTs (fewer than 2 L entries for
  // any radix plan of L), then the four-step and packing tables
  if (general)
    return (size_t)2 * M1 + 2 * M2 + (size_t(1) << kGenLogLo) + (size_t)(M >> kGenLogLo) + 1 + M1 + M2;
  const int lo = log_lo_of(M);
  return (size_t)tw_size(M1) + tw_size(M2) + (size_t(1) << lo) + (size_t)(M >> lo) + M1 + M2;
}

// -------------------------------------------------------------------- workspace layout
struct Layout {
  size_t desc, chunks, params, tw, hits, valid, W, Minv, acc, acc12, map4, bvec, dtab, nbar, nyq, c0,
      ybuf, scal, tpix, tcos, tsin, lam, iter, map64, groups, gen, gen_rec, gen_ctab, gen_rtab,
      adapt, queue, fitems, fctr, fault, total, ybytes;
  int64_t gen_ccap, gen_rcap;
  int lam_cap;
  int n_groups;
  int gM[kMaxGroups], gM1[kMaxGroups], gM2[kMaxGroups], gcount[kMaxGroups], gbatch[kMaxGroups];
  int gn[kMaxGroups], ggen[kMaxGroups], gcplx[kMaxGroups];
  std::vector<int> chunk_group;
  std::vector<int> gen_list;            // general chunks in plan order
  std::vector<Batch> gen_batches;
  int64_t spec_total, n_total;
};

static size_t up(size_t x) { return (x + 255) & ~size_t(255); }

// Bytes of four-step intermediate one batch may use (MM_YBUF_MB overrides; default 2 GB).
// Small budgets (a quarter of L2) keep a batch's intermediate L2-resident between passes,
// but the extra launches cost more than the saved HBM traffic on the 8 x 2^22 workload;
// 2 GB puts the 32 chunks of 2^24 samples of the 2048^2 workload in one batch (one fused
// launch per iteration: 9.15 -> 9.08 ms against two batches of 16).
static size_t ybuf_budget() {
  const char* e = getenv("MM_YBUF_MB");
  const long mb = e ? atol(e) : 2048;
  return (size_t)(mb > 0 ? mb : 2048) << 20;
}

static mm_status make_layout(int n_chunks, const int64_t* off, int64_t n_pix, int ncomp,
                             int wdtype, Layout* L, bool force_general = false) {
  MM_ARG(n_chunks >= 1, "n_chunks must be >= 1 (got %d)", n_chunks);
  MM_ARG(off != nullptr, "offsets is NULL");
  MM_ARG(n_pix >= 1 && n_pix < (int64_t(1) << 31), "n_pix out of range (%lld)", (long long)n_pix);
  MM_ARG(ncomp == 1 || ncomp == 3, "ncomp must be 1 or 3 (got %d)", ncomp);
  MM_ARG(off[0] >= 0, "offsets[0] must be >= 0");
  L->n_groups = 0;
  L->chunk_group.assign(n_chunks, -1);
  L->gen_list.clear();
  L->gen_batches.clear();
  L->spec_total = 0;
  // Power-of-two chunks on 16-byte boundaries take the compile-time kernels (vector loads),
  // one batch per length.  When the plan has a general batch anyway, a length whose chunks
  // hold at most 2^20 samples in all joins it instead: its own batch would add three
  // launches of a few small waves (about 25 us per iteration for one chunk of 2^17 samples
  // beside 24.6 M general samples: 0.851 -> 0.827 ms), more than the general kernels' lower
  // rate costs on that many samples.
  bool any_general = force_general;
  std::vector<std::pair<int64_t, int64_t>> pow2_total;   // (length, samples of that length)
  for (int c = 0; c < n_chunks; ++c) {
    const int64_t n = off[c + 1] - off[c];
    int M_, M1_, M2_;
    if (n < 1) continue;   // reported below
    if (!(fft_shape(n, &M_, &M1_, &M2_) && off[c] % 4 == 0)) { any_general = true; continue; }
    bool found = false;
    for (auto& e : pow2_total)
      if (e.first == n) { e.second += n; found = true; }
    if (!found) pow2_total.push_back({n, n});
  }
  auto joins_general = [&](int64_t n) {
    if (!any_general) return false;
    for (const auto& e : pow2_total)
      if (e.first == n) return e.second <= (int64_t(1) << 20);
    return false;
  };
  for (int c = 0; c < n_chunks; ++c) {
    const int64_t n = off[c + 1] - off[c];
    MM_ARG(n >= 1, "chunk %d is empty or offsets decrease", c);
    int M, M1, M2, cplx = 0;
    bool general = false;
    if (force_general || joins_general(n) || !(fft_shape(n, &M, &M1, &M2) && off[c] % 4 == 0)) {
      if (!gen_shape(n, &M, &M1, &M2, &cplx)) {
        mm_set_error("chunk %d: length %lld unsupported (need prime factors 2, 3, 5 only and "
                     "n <= 2^24; n/2 up to 2^21 for lengths that are not powers of two)",
                     c, (long long)n);
        return MM_ERR_UNSUPPORTED;
      }
      general = true;
    }
    int g = -1;
    for (int i = 0; i < L->n_groups; ++i)
      if (L->gn[i] == n && L->ggen[i] == (int)general) g = i;
    if (g < 0) {
      if (L->n_groups == kMaxGroups) {
        mm_set_error("more than %d distinct chunk lengths", kMaxGroups);
        return MM_ERR_UNSUPPORTED;
      }
      g = L->n_groups++;
      L->gM[g] = M; L->gM1[g] = M1; L->gM2[g] = M2; L->gcount[g] = 0;
      L->gn[g] = (int)n; L->ggen[g] = general; L->gcplx[g] = cplx;
    }
    L->gcount[g]++;
    L->chunk_group[c] = g;
    L->spec_total += spec_slots(M);
    if (general) L->gen_list.push_back(c);
  }
  L->n_total = off[n_chunks];
  MM_ARG(L->n_total < (int64_t(1) << 31) * 2, "too many samples");
  size_t tw = 0, ybytes = 0;
  const size_t budget = ybuf_budget();
  for (int g = 0; g < L->n_groups; ++g) {
    tw += tw_count(L->gM[g], L->gM1[g], L->gM2[g], L->ggen[g]);
    L->gbatch[g] = 0;
    if (L->ggen[g]) continue;
    const size_t per = sizeof(float2) * (size_t)L->gM[g];
    size_t b = budget / per;
    if (b < 1) b = 1;
    if (b > (size_t)L->gcount[g]) b = L->gcount[g];
    L->gbatch[g] = (int)b;
    if (b * per > ybytes) ybytes = b * per;
  }
  // general chunks: consecutive runs of the general list within the same budget
  {
    size_t cur = 0;
    int first = 0;
    const int ng = (int)L->gen_list.size();
    for (int i = 0; i < ng; ++i) {
      const size_t per = sizeof(float2) * (size_t)L->gM[L->chunk_group[L->gen_list[i]]];
      if (i > first && cur + per > budget) {
        L->gen_batches.push_back(Batch{-1, first, i - first});
        first = i;
        cur = 0;
      }
      cur += per;
      if (cur > ybytes) ybytes = cur;
    }
    if (ng > first) L->gen_batches.push_back(Batch{-1, first, ng - first});
  }
  const size_t ngen = L->gen_list.size();
  const size_t np = (size_t)n_pix;
  const size_t blk = ncomp == 3 ? 6 : 1;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o += up(bytes); return r; };
  L->desc = take(sizeof(ChunkDesc) * n_chunks);
  L->chunks = take(sizeof(int) * n_chunks);
  L->params = take(sizeof(double) * 4 * n_chunks);
  L->tw = take(sizeof(float2) * tw);
  L->hits = take(sizeof(int32_t) * np);
  L->valid = take(np);
  L->W = take(sizeof(double) * blk * np);
  L->Minv = take(sizeof(double) * blk * np);
  L->acc = take(sizeof(double) * ncomp * (size_t)acc_stride_of((int64_t)np, ncomp));
  L->acc12 = take(sizeof(double) * 2 * blk * np);
  L->map4 = take((ncomp == 3 ? 16 : 4) * np);
  L->bvec = take(sizeof(double) * ncomp * np);
  L->dtab = take(sizeof(float2) * L->spec_total);
  L->nbar = take(sizeof(float) * L->spec_total);
  L->nyq = take(sizeof(float) * n_chunks);
  L->c0 = take(sizeof(double) * n_chunks);
  L->ybuf = take(ybytes);
  L->ybytes = ybytes;
  L->scal = take(sizeof(double) * kScalCount);
  // pointing copied into column-tile order for the streaming passes
  const size_t wb = ncomp == 3 ? (wdtype == MM_W_F16 ? 2 : 4) : 0;
  L->tpix = take(sizeof(int32_t) * (size_t)L->n_total);
  L->tcos = take(wb * (size_t)L->n_total);
  L->tsin = take(wb * (size_t)L->n_total);
  // graph mode: schedule table, iteration counter + chi^2 pointer slot, FP64 map
  L->lam_cap = 65536;
  L->lam = take(sizeof(double) * L->lam_cap);
  L->iter = take(128);
  L->map64 = take(sizeof(double) * ncomp * np);
  // general path: device groups, chunk list, three prefix arrays, per-chunk records and the
  // work-item tables (column tiles sized for the narrowest tile width)
  int64_t ctiles = 0, rjobs = 0;
  for (int c : L->gen_list) {
    const int g = L->chunk_group[c];
    ctiles += (L->gM2[g] + 7) / 8;
    rjobs += L->gM1[g] / 2 + 1;
  }
  L->gen_ccap = ctiles;
  L->gen_rcap = rjobs;
  L->groups = take(sizeof(Group) * L->n_groups);
  L->gen = take(sizeof(int) * (ngen + 1) + 3 * sizeof(int64_t) * (ngen + 1) + 64);
  L->gen_rec = take(sizeof(GenChunk) * ngen);
  L->gen_ctab = take(sizeof(int2) * ctiles);
  L->gen_rtab = take(sizeof(int4) * rjobs);
  L->adapt = take(sizeof(AdaptState));
  L->queue = take(64);
  // fused iteration kernel: item lists of the batches it covers, counters, fault flag
  size_t fitems = 0;
  for (int g = 0; g < L->n_groups; ++g)
    fitems += (size_t)L->gcount[g] * fused_items_per_chunk(L->gM1[g], L->gM2[g], L->ggen[g]);
  L->fitems = take(sizeof(int2) * (fitems > 0 ? fitems : 1));
  L->fctr = take(sizeof(unsigned) * (2 + 2 * (size_t)n_chunks));
  L->fault = take(16);
  L->total = o;
  return MM_OK;
}

extern "C" mm_status mm_plan_workspace_size(int n_chunks, const int64_t* offsets, int64_t n_pix,
                                            int ncomp, int weight_dtype, size_t* bytes) {
  MM_ARG(bytes != nullptr, "bytes is NULL");
  MM_ARG(weight_dtype == MM_W_F32 || weight_dtype == MM_W_F16, "bad weight_dtype %d",
         weight_dtype);
  Layout L;
  mm_status st = make_layout(n_chunks, offsets, n_pix, ncomp, weight_dtype, &L);
  if (st != MM_OK) return st;
  *bytes = L.total;
  return MM_OK;
}

extern "C" mm_status mm_plan_workspace_size_composite(int n_chunks, const int64_t* offsets,
                                                      int64_t n_pix, int ncomp, int weight_dtype,
                                                      size_t* bytes) {
  MM_ARG(bytes != nullptr, "bytes is NULL");
  MM_ARG(weight_dtype == MM_W_F32 || weight_dtype == MM_W_F16, "bad weight_dtype %d",
         weight_dtype);
  Layout L;
  mm_status st = make_layout(n_chunks, offsets, n_pix, ncomp, weight_dtype, &L, true);
  if (st != MM_OK) return st;
  *bytes = L.total;
  return MM_OK;
}

// ---------------------------------------------------------------------- set-up kernels
// Per-pass Stockham twiddles of a length-L DFT: entry r * Ns + k of pass (Ns, R) holds
// w_{Ns R}^{r k}, computed in FP64 and rounded to FP32.
__global__ void k_pass_twiddles(float2* out, int L) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= tw_size(L)) return;
  int off = 0, ns = 1;
  while (true) {
    const int r = pick_radix(L / ns);
    if (e < off + ns * r) {
      const int loc = e - off, rr = loc / ns, k = loc % ns;
      double sn, cs;
      sincospi(-2.0 * (double)(rr * k) / (double)(ns * r), &sn, &cs);
      out[e] = make_float2((float)cs, (float)sn);
      return;
    }
    off += ns * r;
    ns *= r;
  }
}

// Per-pass twiddles of a mixed-radix Stockham plan of length L: pass p (sub-transforms of
// length Ns, radix R) stores w_{Ns R}^{r k} at [off_p + r Ns + k], r < R, k < Ns, so the
// lanes of a pass (consecutive k) read consecutive words.  FP64, rounded to FP32.
struct PassPlan {
  int nr;
  int8_t rad[kMaxRadices];
};
__global__ void k_plan_twiddles(float2* out, PassPlan pl) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  int off = 0, ns = 1;
  for (int p = 0; p < pl.nr; ++p) {
    const int r = pl.rad[p];
    if (e < off + ns * r) {
      const int loc = e - off, rr = loc / ns, k = loc % ns;
      double sn, cs;
      sincospi(-2.0 * (double)(rr * k) / (double)(ns * r), &sn, &cs);
      out[e] = make_float2((float)cs, (float)sn);
      return;
    }
    off += ns * r;
    ns *= r;
  }
}

static int plan_twiddle_count(const PassPlan& pl) {
  int off = 0, ns = 1;
  for (int p = 0; p < pl.nr; ++p) { off += ns * pl.rad[p]; ns *= pl.rad[p]; }
  return off;
}

__global__ void k_twiddles(float2* out, int count, int denom_mul, int L) {
  // out[m] = exp(-2 pi i m * denom_mul / L) computed in FP64, rounded to FP32
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= count) return;
  double s, c;
  sincospi(-2.0 * (double)m * (double)denom_mul / (double)L, &s, &c);
  out[m] = make_float2((float)c, (float)s);
}

__global__ void k_hits(const int32_t* __restrict__ pix, int64_t n, int64_t n_pix,
                       int32_t* __restrict__ hits, double* __restrict__ flag) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int p = pix[s];
  if (p < -1 || p >= n_pix) {
    flag[0] = 1.0;  // any nonzero marks an out-of-range pixel index
    return;
  }
  if (p >= 0) atomicAdd(hits + p, 1);
}

struct NoiseArgs {
  const ChunkDesc* desc;
  const double* psd;       // table or nullptr
  const double* params;    // device [n_chunks][4] when psd == nullptr
  float* nbar;
  float* nyq;
  double* c0;
  double* scal;            // lambda max bits, min(Nbar) check at kScalTmp
};

__device__ __forceinline__ double psd_value(const NoiseArgs& a, int c, const ChunkDesc& d, int k) {
  if (a.psd) return a.psd[d.nat + k];
  const double* q = a.params + 4 * c;      // sigma, f_knee, alpha, f_sample
  const int kk = k == 0 ? 1 : k;           // DC bin floored to bin 1
  const double f = (double)kk * q[3] / (double)d.n;
  const double x = q[1] / f, alpha = q[2];
  // small integer slopes by multiplication: the FP64 pow runs on the narrow FP64 pipe, once
  // per mode of every chunk (set-up of 32 x 2^24 samples at alpha = 2: 64 -> 22 ms)
  const double xa = alpha == 1.0 ? x : alpha == 2.0 ? x * x : alpha == 3.0 ? x * x * x
                                                                            : pow(x, alpha);
  return q[0] * q[0] * (1.0 + xa);
}

// Nbar = N - tau on every rfft bin of chunk blockIdx.y, stored on the row-layout slots;
// also c0 = (1/n) sum_k w_k / N_k, lambda_max and min(Nbar) (Sec. 2.1 needs Nbar >= 0).
__global__ void k_noise(NoiseArgs a) {
  const int c = blockIdx.y;
  const ChunkDesc d = a.desc[c];
  double sum = 0.0, mx = 0.0, mn = 1e300;
  for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < d.M; slot += gridDim.x * blockDim.x) {
    const int k1 = slot / d.M2, k2 = slot % d.M2;
    const int k = k1 + d.M1 * k2;
    // complex chunks hold every frequency 0..n-1; frequency k is rfft bin min(k, n - k)
    const int kb = d.cplx && 2 * k > d.n ? d.n - k : k;
    const double N = psd_value(a, c, d, kb);
    const double nb = N - d.tau;
    a.nbar[d.spec + slot] = (float)nb;
    double w = k == 0 || d.cplx ? 1.0 : 2.0;
    sum += w / N;
    mx = fmax(mx, nb / d.tau);
    mn = fmin(mn, nb);
    if (k == 0 && d.cplx) a.nyq[c] = 0.f;
    if (k == 0 && !d.cplx) {
      const double NM = psd_value(a, c, d, d.M);
      const double nbM = NM - d.tau;
      a.nyq[c] = (float)nbM;
      sum += 1.0 / NM;
      mx = fmax(mx, nbM / d.tau);
      mn = fmin(mn, nbM);
    }
  }
  __shared__ double rs[32], rx[32], rn[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_down_sync(0xffffffffu, sum, o);
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    rs[threadIdx.x >> 5] = sum; rx[threadIdx.x >> 5] = mx; rn[threadIdx.x >> 5] = mn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      sum += rs[i]; mx = fmax(mx, rx[i]); mn = fmin(mn, rn[i]);
    }
    atomicAdd(a.c0 + c, sum / (double)d.n);
    atomicMax(reinterpret_cast<unsigned long long*>(a.scal + kScalLambdaMax),
              (unsigned long long)__double_as_longlong(fmax(mx, 0.0)));
    if (mn < 0.0) a.scal[kScalTmp] = fmin(a.scal[kScalTmp], mn);
  }
}

__global__ void k_min_psd(const ChunkDesc* desc, const double* psd, double* out) {
  const int c = blockIdx.x;
  const ChunkDesc d = desc[c];
  double mn = 1e300;
  for (int k = threadIdx.x; k <= d.n / 2; k += blockDim.x) mn = fmin(mn, psd[d.nat + k]);
  for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
  __shared__ double r[32];
  if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = mn;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) mn = fmin(mn, r[i]);
    out[c] = mn;
  }
}

// Weight blocks: acc12[p][0..B) += (1/tau_c) w w^T, acc12[p][B..2B) += c0_c w w^T
// (upper triangle 00 01 02 11 12 22 for IQU), w = (1, cos 2psi, sin 2psi).
__global__ void k_weights_accum(const ChunkDesc* __restrict__ desc, int c,
                                const int32_t* __restrict__ pix, const void* cosw,
                                const void* sinw, int half_w, int ncomp,
                                const double* __restrict__ c0, int64_t n0, int64_t n,
                                double* __restrict__ acc12, double scale) {
  const int64_t s = n0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int p = pix[s];
  if (p < 0) return;
  const double s1 = scale / desc[c].tau, s2 = c0[c];
  if (ncomp == 1) {
    atomicAdd(acc12 + 2 * (int64_t)p, s1);
    atomicAdd(acc12 + 2 * (int64_t)p + 1, s2);
    return;
  }
  double cw, sw;
  if (half_w) {
    cw = __half2float(reinterpret_cast<const __half*>(cosw)[s]);
    sw = __half2float(reinterpret_cast<const __half*>(sinw)[s]);
  } else {
    cw = reinterpret_cast<const float*>(cosw)[s];
    sw = reinterpret_cast<const float*>(sinw)[s];
  }
  const double pr[6] = {1.0, cw, sw, cw * cw, cw * sw, sw * sw};
  double* a = acc12 + 12 * (int64_t)p;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    atomicAdd(a + i, s1 * pr[i]);
    atomicAdd(a + 6 + i, s2 * pr[i]);
  }
}

// Eigenvalues of a symmetric 3x3 matrix by the trigonometric closed form (Smith 1961).
__device__ void sym3_eig(const double* m, double* emin, double* emax) {
  const double a00 = m[0], a01 = m[1], a02 = m[2], a11 = m[3], a12 = m[4], a22 = m[5];
  const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
  const double q = (a00 + a11 + a22) / 3.0;
  const double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
  const double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * p1;
  if (p2 <= 0.0) { *emin = *emax = q; return; }
  const double pp = sqrt(p2 / 6.0);
  const double det = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) +
                     a02 * (a01 * a12 - b11 * a02);
  double r = det / (2.0 * pp * pp * pp);
  r = fmin(1.0, fmax(-1.0, r));
  const double phi = acos(r) / 3.0;
  const double e1 = q + 2.0 * pp * cos(phi);
  const double e3 = q + 2.0 * pp * cos(phi + 2.0943951023931954923);
  *emax = e1;
  *emin = e3;
}

__device__ bool sym3_inv(const double* m, double* o) {
  const double a = m[0], b = m[1], c = m[2], d = m[3], e = m[4], f = m[5];
  const double c00 = d * f - e * e, c01 = c * e - b * f, c02 = b * e - c * d;
  const double det = a * c00 + b * c01 + c * c02;
  if (!(det > 0.0) && !(det < 0.0)) return false;
  const double id = 1.0 / det;
  o[0] = c00 * id;
  o[1] = c01 * id;
  o[2] = c02 * id;
  o[3] = (a * f - c * c) * id;
  o[4] = (b * c - a * e) * id;
  o[5] = (a * d - b * b) * id;
  return true;
}

// Per pixel: cut decision, W = (P^T T^-1 P)^-1 and the PCG block preconditioner inverse.
__global__ void k_pixel_solve(int64_t n_pix, int ncomp, double rcond_min,
                              const int32_t* __restrict__ hits, const double* __restrict__ acc12,
                              uint8_t* __restrict__ valid, double* __restrict__ W,
                              double* __restrict__ Minv, unsigned long long* n_valid) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  bool ok = hits[p] >= 1;
  if (ncomp == 1) {
    const double a = acc12[2 * p], b = acc12[2 * p + 1];
    ok = ok && a > 0.0 && b > 0.0;
    W[p] = ok ? 1.0 / a : 0.0;
    Minv[p] = ok ? 1.0 / b : 0.0;
  } else {
    const double* A = acc12 + 12 * p;
    double wi[6] = {0, 0, 0, 0, 0, 0}, mi[6] = {0, 0, 0, 0, 0, 0};
    if (ok) {
      double emin, emax;
      sym3_eig(A, &emin, &emax);
      ok = emax > 0.0 && emin / emax >= rcond_min;
    }
    if (ok) ok = sym3_inv(A, wi) && sym3_inv(A + 6, mi);
    if (!ok)
      for (int i = 0; i < 6; ++i) wi[i] = mi[i] = 0.0;
    for (int i = 0; i < 6; ++i) {
      W[6 * p + i] = wi[i];
      Minv[6 * p + i] = mi[i];
    }
  }
  valid[p] = ok ? 1 : 0;
  if (ok) atomicAdd(n_valid, 1ull);
}

// ------------------------------------------------------------------ map-step kernels
template <int NC>
__device__ __forceinline__ void sym_apply(const double* W, const double* a, double* m) {
  if constexpr (NC == 1) {
    m[0] = W[0] * a[0];
  } else {
    m[0] = W[0] * a[0] + W[1] * a[1] + W[2] * a[2];
    m[1] = W[1] * a[0] + W[3] * a[1] + W[4] * a[2];
    m[2] = W[2] * a[0] + W[4] * a[1] + W[5] * a[2];
  }
}

template <int NC>
__device__ __forceinline__ void store_map4(void* map4, int64_t p, const double* m) {
  if constexpr (NC == 1) reinterpret_cast<float*>(map4)[p] = (float)m[0];
  else reinterpret_cast<float4*>(map4)[p] = make_float4((float)m[0], (float)m[1], (float)m[2], 0.f);
}

// m = (P^T T^-1 P)^-1 acc (the map step of Sec. 2.1); acc is cleared for the next pass.
template <int NC>
__global__ void k_bin_apply(int64_t n_pix, double* __restrict__ acc, const double* __restrict__ W,
                            void* map4, double* __restrict__ map_out, int* iter = nullptr) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (iter && p == 0) *iter += 1;   // graph mode: next iteration of the schedule
  if (p >= n_pix) return;
  constexpr int B = NC == 3 ? 6 : 1;
  double a[NC], w[B], m[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    const int64_t j_ = i * acc_stride_of(n_pix, NC) + p;   // planar accumulators
    a[i] = acc[j_];
    acc[j_] = 0.0;
  }
#pragma unroll
  for (int i = 0; i < B; ++i) w[i] = W[B * p + i];
  sym_apply<NC>(w, a, m);
  store_map4<NC>(map4, p, m);
  if (map_out)
#pragma unroll
    for (int i = 0; i < NC; ++i) map_out[NC * p + i] = m[i];
}

// Composite map step (App. B, compact form): m += D^-1 acc with D^-1 in W; acc cleared; the
// FP32 gather copy holds m on kept pixels and 0 on cut ones (whose entries drop out of P).
template <int NC>
__global__ void k_bin_resid(int64_t n_pix, double* __restrict__ acc, const double* __restrict__ W,
                            const uint8_t* __restrict__ valid, double* __restrict__ m64,
                            void* map4, double* __restrict__ map_out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  constexpr int B = NC == 3 ? 6 : 1;
  double a[NC], w[B], u[NC], m[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    const int64_t j_ = i * acc_stride_of(n_pix, NC) + p;   // planar accumulators
    a[i] = acc[j_];
    acc[j_] = 0.0;
  }
#pragma unroll
  for (int i = 0; i < B; ++i) w[i] = W[B * p + i];
  sym_apply<NC>(w, a, u);
#pragma unroll
  for (int i = 0; i < NC; ++i) { m[i] = m64[NC * p + i] + u[i]; m64[NC * p + i] = m[i]; }
  double g[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) g[i] = valid[p] ? m[i] : 0.0;
  store_map4<NC>(map4, p, g);
  if (map_out)
#pragma unroll
    for (int i = 0; i < NC; ++i) map_out[NC * p + i] = m[i];
}

// map4 = float(map) on valid pixels, 0 on cut ones.
template <int NC>
__global__ void k_map_to4(int64_t n_pix, const double* __restrict__ map,
                          const uint8_t* __restrict__ valid, void* map4) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  double m[NC];
  const bool ok = valid[p] != 0;
#pragma unroll
  for (int i = 0; i < NC; ++i) m[i] = ok ? map[NC * p + i] : 0.0;
  store_map4<NC>(map4, p, m);
}

// ----------------------------------------------------------------- operator kernels
template <int NC>
__global__ void k_gather(int64_t n, const int32_t* __restrict__ pix, const void* cosw,
                         const void* sinw, int half_w, const void* map4, float* __restrict__ out) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int p = pix[s];
  float v = 0.f;
  if (p >= 0) {
    if constexpr (NC == 1) {
      v = reinterpret_cast<const float*>(map4)[p];
    } else {
      float cw, sw;
      if (half_w) {
        cw = __half2float(reinterpret_cast<const __half*>(cosw)[s]);
        sw = __half2float(reinterpret_cast<const __half*>(sinw)[s]);
      } else {
        cw = reinterpret_cast<const float*>(cosw)[s];
        sw = reinterpret_cast<const float*>(sinw)[s];
      }
      const float4 m = reinterpret_cast<const float4*>(map4)[p];
      v = fmaf(sw, m.z, fmaf(cw, m.y, m.x));
    }
  }
  out[s] = v;
}

template <int NC>
__global__ void k_scatter(int64_t n, const int32_t* __restrict__ pix, const void* cosw,
                          const void* sinw, int half_w, const float* __restrict__ tod,
                          double* __restrict__ acc) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int p = pix[s];
  if (p < 0) return;
  const double t = tod[s];
  double* a = acc + (int64_t)p * NC;
  atomicAdd(a, t);
  if constexpr (NC == 3) {
    float cw, sw;
    if (half_w) {
      cw = __half2float(reinterpret_cast<const __half*>(cosw)[s]);
      sw = __half2float(reinterpret_cast<const __half*>(sinw)[s]);
    } else {
      cw = reinterpret_cast<const float*>(cosw)[s];
      sw = reinterpret_cast<const float*>(sinw)[s];
    }
    atomicAdd(a + 1, t * (double)cw);
    atomicAdd(a + 2, t * (double)sw);
  }
}

template <int NC>
__global__ void k_expand_weights(int64_t n_pix, const double* __restrict__ W, double* __restrict__ out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  if constexpr (NC == 1) {
    out[p] = W[p];
  } else {
    const double* w = W + 6 * p;
    double* o = out + 9 * p;
    o[0] = w[0]; o[1] = w[1]; o[2] = w[2];
    o[3] = w[1]; o[4] = w[3]; o[5] = w[4];
    o[6] = w[2]; o[7] = w[4]; o[8] = w[5];
  }
}

// b = P^T N^-1 d on valid pixels; acc cleared.
__global__ void k_finish_b(int64_t len, int ncomp, double* __restrict__ acc,
                           const uint8_t* __restrict__ valid, double* __restrict__ b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= len) return;
  const int64_t a = (i % ncomp) * acc_stride_of(len / ncomp, ncomp) + i / ncomp;   // planar
  b[i] = valid[i / ncomp] ? acc[a] : 0.0;
  acc[a] = 0.0;
}

// ------------------------------------------------------------------------ PCG kernels
// State: r, z, p, q ([len] doubles each) then scalars.
enum { kPcgRz0 = 0, kPcgRz1 = 1, kPcgPq = 2, kPcgXb = 3, kPcgXr = 4, kPcgNs = 8 };

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  __syncthreads();
  return s;
}

template <int NC>
__device__ __forceinline__ void block_apply(const double* Minv, int64_t pixel, const double* r,
                                            double* z) {
  constexpr int B = NC == 3 ? 6 : 1;
  double w[B];
#pragma unroll
  for (int i = 0; i < B; ++i) w[i] = Minv[B * pixel + i];
  sym_apply<NC>(w, r, z);
}

// r = b - A x (A x in acc), z = M^-1 r, p = z, map4 = p; rz, x.b, x.r.
template <int NC>
__global__ void k_pcg_init(int64_t n_pix, double* __restrict__ acc, const double* __restrict__ bvec,
                           const double* __restrict__ x, const uint8_t* __restrict__ valid,
                           const double* __restrict__ Minv, double* __restrict__ r,
                           double* __restrict__ z, double* __restrict__ pv, void* map4,
                           double* sc) {
  __shared__ double red[32];
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double rz = 0, xb = 0, xr = 0;
  if (p < n_pix) {
    const bool ok = valid[p] != 0;
    double rr[NC], zz[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      const int64_t j = NC * p + i;
      const int64_t ja = i * acc_stride_of(n_pix, NC) + p;   // planar accumulators
      rr[i] = ok ? bvec[j] - acc[ja] : 0.0;
      acc[ja] = 0.0;
    }
    block_apply<NC>(Minv, p, rr, zz);
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      const int64_t j = NC * p + i;
      const double xv = ok ? x[j] : 0.0;
      r[j] = rr[i]; z[j] = zz[i]; pv[j] = zz[i];
      rz += rr[i] * zz[i];
      xb += xv * bvec[j];
      xr += xv * rr[i];
    }
    store_map4<NC>(map4, p, zz);
  }
  rz = block_sum(rz, red);
  xb = block_sum(xb, red);
  xr = block_sum(xr, red);
  if (threadIdx.x == 0) {
    atomicAdd(sc + kPcgRz0, rz);
    atomicAdd(sc + kPcgXb, xb);
    atomicAdd(sc + kPcgXr, xr);
  }
}

// q = A p on valid pixels (acc cleared), p.q; block 0 records chi^2 of the current iterate
// and clears the accumulators the update kernel fills.
__global__ void k_pcg_q(int64_t len, int ncomp, double* __restrict__ acc, const uint8_t* __restrict__ valid,
                        const double* __restrict__ pv, double* __restrict__ q, double* sc, int rz_next,
                        const double* cdd, double* chi2_slot) {
  __shared__ double red[32];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < len) {
    const int64_t a = (i % ncomp) * acc_stride_of(len / ncomp, ncomp) + i / ncomp;   // planar
    const double qq = valid[i / ncomp] ? acc[a] : 0.0;
    acc[a] = 0.0;
    q[i] = qq;
    s = pv[i] * qq;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) atomicAdd(sc + kPcgPq, s);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (chi2_slot) *chi2_slot = *cdd - sc[kPcgXb] - sc[kPcgXr];
    sc[kPcgXb] = 0.0;
    sc[kPcgXr] = 0.0;
    sc[rz_next] = 0.0;
  }
}

// alpha = rz / pq; x += alpha p; r -= alpha q; z = M^-1 r; rz_next, x.b, x.r.
template <int NC>
__global__ void k_pcg_update(int64_t n_pix, double* __restrict__ x, double* __restrict__ r,
                             double* __restrict__ z, const double* __restrict__ pv,
                             const double* __restrict__ q, const double* __restrict__ bvec,
                             const double* __restrict__ Minv, double* sc, int rz_cur, int rz_next) {
  __shared__ double red[32];
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double alpha = sc[rz_cur] / sc[kPcgPq];
  double rz = 0, xb = 0, xr = 0;
  if (p < n_pix) {
    double rr[NC], zz[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      const int64_t j = NC * p + i;
      const double xv = x[j] + alpha * pv[j];
      x[j] = xv;
      rr[i] = r[j] - alpha * q[j];
      r[j] = rr[i];
      xb += xv * bvec[j];
      xr += xv * rr[i];
    }
    block_apply<NC>(Minv, p, rr, zz);
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      z[NC * p + i] = zz[i];
      rz += rr[i] * zz[i];
    }
  }
  rz = block_sum(rz, red);
  xb = block_sum(xb, red);
  xr = block_sum(xr, red);
  if (threadIdx.x == 0) {
    atomicAdd(sc + rz_next, rz);
    atomicAdd(sc + kPcgXb, xb);
    atomicAdd(sc + kPcgXr, xr);
  }
}

// beta = rz_next / rz_cur; p = z + beta p; map4 = p; pq cleared by the next k_pcg_q's
// predecessor (this kernel's last block is not known, so pq is reset by the driver).
template <int NC>
__global__ void k_pcg_dir(int64_t n_pix, const double* __restrict__ z, double* __restrict__ pv,
                          void* map4, const double* sc, int rz_cur, int rz_next) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  const double beta = sc[rz_next] / sc[rz_cur];
  double m[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    const int64_t j = NC * p + i;
    m[i] = z[j] + beta * pv[j];
    pv[j] = m[i];
  }
  store_map4<NC>(map4, p, m);
}

// ------------------------------------------------------------------------- plan API
static unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Tables of the general path for the current schedule (p->gen_tune): prefix sums over the
// general chunk list, one record per general chunk (descriptor, twiddle tables, radix
// sequences of the chosen order) and the work-item tables (chunk, tile / row) of the column
// and row kernels; uploaded and synchronised.
static cudaError_t gen_upload(mm_plan_s* p, cudaStream_t s) {
  const int ng = p->n_gen, nb = p->gen_tune.col_nb;
  std::vector<GenChunk> rec(ng);
  std::vector<int2> ct;
  std::vector<int4> rt;
  int64_t ct_n = 0, rj = 0, yo = 0;
  for (int i = 0; i < ng; ++i) {
    const int c = p->h_gen_chunks[i];
    ChunkDesc& d = p->h_desc[c];
    const Group& G = p->groups[d.grp];
    p->h_gen_ctile[i] = ct_n;
    p->h_gen_rjob[i] = rj;
    p->h_gen_yoff[i] = yo;
    const int tiles = (d.M2 + nb - 1) / nb;
    for (int t = 0; t < tiles; ++t) ct.push_back(make_int2(i, t * nb));
    // row jobs: row 0 alone, pairs (k1, M1 - k1) in groups, row M1/2 alone for even M1
    const size_t r0 = rt.size();
    rt.push_back(make_int4(i, 0, 0, 0));
    const int h = (d.M1 - 1) / 2, np = gen_row_pairs(d.M1, d.M2);
    for (int f = 1; f <= h; f += np) rt.push_back(make_int4(i, f, h - f + 1 < np ? h - f + 1 : np, 0));
    if (d.M1 % 2 == 0 && d.M1 >= 2) rt.push_back(make_int4(i, d.M1 / 2, 0, 0));
    const int jobs = (int)(rt.size() - r0);
    GenChunk& R = rec[i];
    memset(&R, 0, sizeof(R));
    R.d = d;
    R.c = c;
    R.log_lo = G.log_lo;
    R.yoff = yo;
    R.tw_col = G.tw_col; R.tw_row = G.tw_row; R.tw_lo = G.tw_lo; R.tw_hi = G.tw_hi;
    R.pack_a = G.tw_pack_a; R.pack_b = G.tw_pack_b;
    R.nr1 = radix_plan(d.M1, R.rad1, p->gen_tune.radix_order);
    R.nr2 = radix_plan(d.M2, R.rad2, p->gen_tune.radix_order);
    ct_n += tiles;
    rj += jobs;
    yo += d.M;
  }
  p->h_gen_ctile[ng] = ct_n;
  p->h_gen_rjob[ng] = rj;
  p->h_gen_yoff[ng] = yo;
  if (ct_n > p->gen_ccap) return cudaErrorInvalidValue;
  // per-pass DFT tables of every general group, for the radix order in use
  for (int g = 0; g < p->n_groups; ++g) {
    const Group& G = p->groups[g];
    if (!G.general) continue;
    for (int dim = 0; dim < 2; ++dim) {
      PassPlan pl;
      memset(&pl, 0, sizeof(pl));
      pl.nr = radix_plan(dim ? G.M2 : G.M1, pl.rad, p->gen_tune.radix_order);
      if (pl.nr < 0) return cudaErrorInvalidValue;
      const int cnt = plan_twiddle_count(pl);
      if (cnt > 2 * (dim ? G.M2 : G.M1)) return cudaErrorInvalidValue;
      if (cnt > 0)   // a length-1 DFT has no pass
        k_plan_twiddles<<<blocks_for(cnt, 256), 256, 0, s>>>(dim ? G.tw_row : G.tw_col, pl);
    }
  }
  cudaError_t ek = cudaGetLastError();
  if (ek != cudaSuccess) return ek;
  cudaError_t e;
  const size_t b = sizeof(int64_t) * (ng + 1);
  if ((e = cudaMemcpyAsync(p->gen_ctile, p->h_gen_ctile, b, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(p->gen_rjob, p->h_gen_rjob, b, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(p->gen_yoff, p->h_gen_yoff, b, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(p->gen_chunks, p->h_gen_chunks, sizeof(int) * ng, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(p->gen_rec, rec.data(), sizeof(GenChunk) * ng, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(p->gen_ctab, ct.data(), sizeof(int2) * ct.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(p->gen_rtab, rt.data(), sizeof(int4) * rt.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  // the column kernels read the pointing in tile order for this schedule's tile width
  if ((e = launch_gen_tile_pointing(p, s)) != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

// Second pointing component of a composite plan (App. B).
struct CompArgs {
  const int32_t* pix_b;
  const void* cos_b;
  const void* sin_b;
  float gain_a, gain_b;
};

static mm_status plan_create(mm_plan* out, int n_chunks, const int64_t* offsets,
                             const int32_t* pix, const void* cos2psi, const void* sin2psi,
                             int weight_dtype, int64_t n_pix, int ncomp, double rcond_min,
                             void* workspace, size_t workspace_bytes, void* stream,
                             const CompArgs* cp);

extern "C" mm_status mm_plan_pointing(mm_plan* out, int n_chunks, const int64_t* offsets,
                                      const int32_t* pix, const void* cos2psi,
                                      const void* sin2psi, int weight_dtype, int64_t n_pix,
                                      int ncomp, double rcond_min, void* workspace,
                                      size_t workspace_bytes, void* stream) {
  MmRange nvtx_range_("mm_plan_pointing");
  return plan_create(out, n_chunks, offsets, pix, cos2psi, sin2psi, weight_dtype, n_pix, ncomp,
                     rcond_min, workspace, workspace_bytes, stream, nullptr);
}

extern "C" mm_status mm_plan_composite(mm_plan* out, int n_chunks, const int64_t* offsets,
                                       const int32_t* pix_a, const void* cos_a, const void* sin_a,
                                       float gain_a, const int32_t* pix_b, const void* cos_b,
                                       const void* sin_b, float gain_b, int weight_dtype,
                                       int64_t n_pix, int ncomp, double rcond_min, void* workspace,
                                       size_t workspace_bytes, void* stream) {
  MmRange nvtx_range_("mm_plan_composite");
  MM_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  MM_ARG(pix_b != nullptr, "pix_b is NULL");
  MM_ARG((ncomp == 3) == (cos_b != nullptr && sin_b != nullptr),
         "cos_b/sin_b must be given iff ncomp == 3");
  MM_ARG(isfinite(gain_a) && isfinite(gain_b) && (gain_a != 0.f || gain_b != 0.f),
         "gains must be finite and not both zero");
  const CompArgs cp{pix_b, cos_b, sin_b, gain_a, gain_b};
  return plan_create(out, n_chunks, offsets, pix_a, cos_a, sin_a, weight_dtype, n_pix, ncomp,
                     rcond_min, workspace, workspace_bytes, stream, &cp);
}

static mm_status plan_create(mm_plan* out, int n_chunks, const int64_t* offsets,
                             const int32_t* pix, const void* cos2psi, const void* sin2psi,
                             int weight_dtype, int64_t n_pix, int ncomp, double rcond_min,
                             void* workspace, size_t workspace_bytes, void* stream,
                             const CompArgs* cp) {
  MM_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  MM_ARG(pix != nullptr, "pix is NULL");
  MM_ARG(weight_dtype == MM_W_F32 || weight_dtype == MM_W_F16, "bad weight_dtype %d",
         weight_dtype);
  Layout L;
  mm_status st = make_layout(n_chunks, offsets, n_pix, ncomp, weight_dtype, &L, cp != nullptr);
  if (st != MM_OK) return st;
  MM_ARG((ncomp == 3) == (cos2psi != nullptr && sin2psi != nullptr),
         "cos2psi/sin2psi must be given iff ncomp == 3");
  MM_ARG(ncomp == 1 || (cos2psi != nullptr && sin2psi != nullptr), "weights missing");
  MM_ARG(workspace != nullptr, "workspace is NULL");
  MM_ARG(((uintptr_t)workspace & 255) == 0, "workspace must be 256-byte aligned");
  if (workspace_bytes < L.total) {
    mm_set_error("workspace too small: %zu < %zu bytes", workspace_bytes, L.total);
    return MM_ERR_NOMEM;
  }
  MM_ARG(rcond_min >= 0.0 && rcond_min <= 1.0, "rcond_min must be in [0, 1]");

  mm_plan_s* p = new (std::nothrow) mm_plan_s();
  if (!p) { mm_set_error("host allocation failed"); return MM_ERR_NOMEM; }
  p->n_chunks = n_chunks; p->ncomp = ncomp; p->wdtype = weight_dtype;
  p->n_pix = n_pix; p->n_total = L.n_total; p->spec_total = L.spec_total;
  p->rcond_min = rcond_min; p->pix = pix; p->cosw = cos2psi; p->sinw = sin2psi;
  p->noise_set = false;
  p->composite = cp != nullptr;
  p->pix_b = cp ? cp->pix_b : nullptr;
  p->cos_b = cp ? cp->cos_b : nullptr;
  p->sin_b = cp ? cp->sin_b : nullptr;
  p->gain_a = cp ? cp->gain_a : 1.f;
  p->gain_b = cp ? cp->gain_b : 0.f;
  char* ws = static_cast<char*>(workspace);
  p->d_desc = reinterpret_cast<ChunkDesc*>(ws + L.desc);
  int* d_chunks = reinterpret_cast<int*>(ws + L.chunks);
  p->tw_pool = reinterpret_cast<float2*>(ws + L.tw);
  p->hits = reinterpret_cast<int32_t*>(ws + L.hits);
  p->valid = reinterpret_cast<uint8_t*>(ws + L.valid);
  p->W = reinterpret_cast<double*>(ws + L.W);
  p->Minv = reinterpret_cast<double*>(ws + L.Minv);
  p->acc = reinterpret_cast<double*>(ws + L.acc);
  p->acc12 = reinterpret_cast<double*>(ws + L.acc12);
  p->map4 = ws + L.map4;
  p->bvec = reinterpret_cast<double*>(ws + L.bvec);
  p->dtab = reinterpret_cast<float2*>(ws + L.dtab);
  p->nbar = reinterpret_cast<float*>(ws + L.nbar);
  p->nyq = reinterpret_cast<float*>(ws + L.nyq);
  p->c0 = reinterpret_cast<double*>(ws + L.c0);
  p->ybuf = reinterpret_cast<float2*>(ws + L.ybuf);
  p->ybuf_bytes = L.ybytes;
  p->theta_ok = false;
  p->graph_exec = nullptr;
  p->graph_stream = nullptr;
  p->lam_cap = L.lam_cap;
  p->lam_table = reinterpret_cast<double*>(ws + L.lam);
  p->iter = reinterpret_cast<int*>(ws + L.iter);
  p->chi2_base = reinterpret_cast<double**>(ws + L.iter + 64);
  p->map64 = reinterpret_cast<double*>(ws + L.map64);
  p->adapt_exec = nullptr;
  p->adapt_st = ws + L.adapt;
  p->row_queue = reinterpret_cast<unsigned*>(ws + L.queue);
  p->fused_items = reinterpret_cast<int2*>(ws + L.fitems);
  p->fused_ctr = reinterpret_cast<unsigned*>(ws + L.fctr);
  p->fault = reinterpret_cast<int*>(ws + L.fault);
  p->wait_polls = 1 << 22;
  p->check_on_return = 0;
  p->h_fused_first = nullptr;
  p->h_fused_n = nullptr;
  p->scal = reinterpret_cast<double*>(ws + L.scal);
  p->params = reinterpret_cast<double*>(ws + L.params);
  p->tpix = reinterpret_cast<int32_t*>(ws + L.tpix);
  p->tcos = ncomp == 3 ? static_cast<void*>(ws + L.tcos) : nullptr;
  p->tsin = ncomp == 3 ? static_cast<void*>(ws + L.tsin) : nullptr;
  p->d_groups = reinterpret_cast<Group*>(ws + L.groups);
  p->n_gen = (int)L.gen_list.size();
  {
    char* gb = ws + L.gen;
    const size_t ng1 = (size_t)p->n_gen + 1;
    p->gen_ctile = reinterpret_cast<int64_t*>(gb);
    p->gen_rjob = p->gen_ctile + ng1;
    p->gen_yoff = p->gen_rjob + ng1;
    p->gen_chunks = reinterpret_cast<int*>(p->gen_yoff + ng1);
  }
  p->gen_rec = reinterpret_cast<GenChunk*>(ws + L.gen_rec);
  p->gen_ctab = reinterpret_cast<int2*>(ws + L.gen_ctab);
  p->gen_rtab = reinterpret_cast<int4*>(ws + L.gen_rtab);
  p->gen_ccap = L.gen_ccap;
  p->h_gen_ctile = p->h_gen_rjob = p->h_gen_yoff = nullptr;
  p->h_gen_chunks = nullptr;
  p->gen_tune = GenTune{8, 256, 256, 0};

  // host descriptors, grouped chunk lists
  p->h_desc = new (std::nothrow) ChunkDesc[n_chunks];
  p->h_chunk_group = new (std::nothrow) int[n_chunks];
  std::vector<int> order;
  if (!p->h_desc || !p->h_chunk_group) { mm_plan_destroy(p); mm_set_error("host allocation failed"); return MM_ERR_NOMEM; }
  int64_t spec = 0, nat = 0;
  for (int c = 0; c < n_chunks; ++c) {
    ChunkDesc& d = p->h_desc[c];
    const int g = L.chunk_group[c];
    d.off = offsets[c];
    d.spec = spec;
    d.nat = nat;
    d.n = (int)(offsets[c + 1] - offsets[c]);
    d.M = L.gM[g]; d.M1 = L.gM1[g]; d.M2 = L.gM2[g];
    d.grp = g;
    d.cplx = L.gcplx[g];
    d.tau = 1.0;
    spec += spec_slots(d.M);
    nat += d.n / 2 + 1;
    p->h_chunk_group[c] = g;
  }
  p->n_groups = L.n_groups;
  p->h_batches = nullptr;
  p->n_batches = 0;
  size_t tw_off = 0;
  for (int g = 0; g < L.n_groups; ++g) {
    Group& G = p->groups[g];
    G.M = L.gM[g]; G.M1 = L.gM1[g]; G.M2 = L.gM2[g];
    G.general = L.ggen[g];
    G.cplx = L.gcplx[g];
    G.log_lo = G.general ? kGenLogLo : log_lo_of(G.M);
    G.nr1 = G.nr2 = 0;
    if (G.general) {
      G.nr1 = radix_plan(G.M1, G.rad1);
      G.nr2 = radix_plan(G.M2, G.rad2);
    }
    G.chunks = d_chunks + order.size();
    G.n_chunks = 0;
    G.batch = L.gbatch[g];
    for (int c = 0; c < n_chunks; ++c)
      if (L.chunk_group[c] == g) { order.push_back(c); G.n_chunks++; }
    float2* t = p->tw_pool + tw_off;
    G.tw_col = t; t += G.general ? 2 * G.M1 : tw_size(G.M1);
    G.tw_row = t; t += G.general ? 2 * G.M2 : tw_size(G.M2);
    G.tw_lo = t; t += (1 << G.log_lo);
    G.tw_hi = t; t += (G.M >> G.log_lo) + (G.general ? 1 : 0);
    G.tw_pack_a = t; t += G.M1;
    G.tw_pack_b = t; t += G.M2;
    tw_off += tw_count(G.M, G.M1, G.M2, G.general);
  }
  {
    int nb = (int)L.gen_batches.size();
    for (int g = 0; g < L.n_groups; ++g)
      if (!L.ggen[g]) nb += (p->groups[g].n_chunks + L.gbatch[g] - 1) / L.gbatch[g];
    p->h_batches = new (std::nothrow) Batch[nb > 0 ? nb : 1];
    if (!p->h_batches) { mm_plan_destroy(p); mm_set_error("host allocation failed"); return MM_ERR_NOMEM; }
    for (int g = 0; g < L.n_groups; ++g) {
      if (L.ggen[g]) continue;
      for (int f = 0; f < p->groups[g].n_chunks; f += L.gbatch[g]) {
        const int cnt = p->groups[g].n_chunks - f < L.gbatch[g] ? p->groups[g].n_chunks - f : L.gbatch[g];
        p->h_batches[p->n_batches++] = Batch{g, f, cnt};
      }
    }
    for (const Batch& b : L.gen_batches) p->h_batches[p->n_batches++] = b;
  }
  // item lists of the batches the fused iteration kernel covers
  std::vector<int2> fitems;
  {
    p->h_fused_first = new (std::nothrow) int[p->n_batches > 0 ? p->n_batches : 1];
    p->h_fused_n = new (std::nothrow) int[p->n_batches > 0 ? p->n_batches : 1];
    if (!p->h_fused_first || !p->h_fused_n) { mm_plan_destroy(p); mm_set_error("host allocation failed"); return MM_ERR_NOMEM; }
    for (int b = 0; b < p->n_batches; ++b) {
      const Batch& B = p->h_batches[b];
      p->h_fused_first[b] = (int)fitems.size();
      p->h_fused_n[b] = 0;
      if (B.group < 0 || p->composite) continue;
      const Group& G = p->groups[B.group];
      const int per = fused_items_per_chunk(G.M1, G.M2, G.general);
      if (per == 0) continue;
      fitems.resize(fitems.size() + (size_t)per * B.count);
      p->h_fused_n[b] = fused_build_items(G.M1, G.M2, B.count, fitems.data() + p->h_fused_first[b]);
    }
  }
  // general list and its prefix sums (column tiles of the tuned width, row jobs, offsets)
  if (p->n_gen > 0) {
    const int ng = p->n_gen;
    p->h_gen_chunks = new (std::nothrow) int[ng];
    p->h_gen_ctile = new (std::nothrow) int64_t[3 * (ng + 1)];
    if (!p->h_gen_chunks || !p->h_gen_ctile) { mm_plan_destroy(p); mm_set_error("host allocation failed"); return MM_ERR_NOMEM; }
    p->h_gen_rjob = p->h_gen_ctile + (ng + 1);
    p->h_gen_yoff = p->h_gen_rjob + (ng + 1);
    for (int i = 0; i < ng; ++i) p->h_gen_chunks[i] = L.gen_list[i];
  }
  cudaStream_t s = S(stream);
  auto fail = [&](const char* what, cudaError_t e) {
    mm_set_error("%s: %s", what, cudaGetErrorString(e));
    mm_plan_destroy(p);
    return MM_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = cudaMemcpyAsync(p->d_desc, p->h_desc, sizeof(ChunkDesc) * n_chunks,
                           cudaMemcpyHostToDevice, s)) != cudaSuccess) return fail("desc upload", e);
  if ((e = cudaMemcpyAsync(d_chunks, order.data(), sizeof(int) * n_chunks,
                           cudaMemcpyHostToDevice, s)) != cudaSuccess) return fail("chunk list upload", e);
  for (int g = 0; g < L.n_groups; ++g) {
    const Group& G = p->groups[g];
    if (G.general) {
      // per-pass DFT tables: built for the tuned radix order by gen_upload
    } else {
      k_pass_twiddles<<<blocks_for(tw_size(G.M1), 256), 256, 0, s>>>(G.tw_col, G.M1);
      k_pass_twiddles<<<blocks_for(tw_size(G.M2), 256), 256, 0, s>>>(G.tw_row, G.M2);
    }
    const int nhi = (G.M >> G.log_lo) + (G.general ? 1 : 0);
    struct { float2* o; int cnt, mul, L; } tabs[4] = {
        {G.tw_lo, 1 << G.log_lo, 1, G.M}, {G.tw_hi, nhi, 1 << G.log_lo, G.M},
        {G.tw_pack_a, G.M1, 1, 2 * G.M}, {G.tw_pack_b, G.M2, G.M1, 2 * G.M}};
    for (auto& tb : tabs) {
      k_twiddles<<<blocks_for(tb.cnt, 256), 256, 0, s>>>(tb.o, tb.cnt, tb.mul, tb.L);
    }
  }
  if ((e = cudaMemcpyAsync(p->d_groups, p->groups, sizeof(Group) * L.n_groups,
                           cudaMemcpyHostToDevice, s)) != cudaSuccess) return fail("group upload", e);
  if (p->n_gen > 0) {
    if ((e = gen_upload(p, s)) != cudaSuccess) return fail("general chunk tables", e);
  }
  if ((e = cudaMemsetAsync(p->hits, 0, sizeof(int32_t) * n_pix, s)) != cudaSuccess) return fail("memset", e);
  if ((e = cudaMemsetAsync(p->scal, 0, sizeof(double) * kScalCount, s)) != cudaSuccess) return fail("memset", e);
  if ((e = cudaMemsetAsync(p->acc, 0, sizeof(double) * ncomp * acc_stride_of(n_pix, ncomp), s)) != cudaSuccess)
    return fail("memset", e);
  if ((e = cudaMemsetAsync(p->row_queue, 0, 64, s)) != cudaSuccess) return fail("memset", e);
  if ((e = cudaMemsetAsync(p->fused_ctr, 0, sizeof(unsigned) * (2 + 2 * (size_t)n_chunks), s)) != cudaSuccess)
    return fail("memset", e);
  if ((e = cudaMemsetAsync(p->fault, 0, 16, s)) != cudaSuccess) return fail("memset", e);
  if (!fitems.empty() &&
      (e = cudaMemcpyAsync(p->fused_items, fitems.data(), sizeof(int2) * fitems.size(),
                           cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return fail("fused item lists", e);
  if (L.n_total > 0)
    k_hits<<<blocks_for(L.n_total, 256), 256, 0, s>>>(pix, L.n_total, n_pix, p->hits, p->scal + kScalTmp);
  if (L.n_total > 0 && p->composite)
    k_hits<<<blocks_for(L.n_total, 256), 256, 0, s>>>(p->pix_b, L.n_total, n_pix, p->hits, p->scal + kScalTmp);
  if ((e = launch_tile_pointing(p, s)) != cudaSuccess) return fail("pointing tile copy", e);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail("set-up kernels", e);
  double flag = 0.0;
  if ((e = cudaMemcpyAsync(&flag, p->scal + kScalTmp, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return fail("flag read", e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail("plan synchronise", e);
  if (flag != 0.0) {
    mm_plan_destroy(p);
    mm_set_error("pix holds a value outside [-1, n_pix)");
    return MM_ERR_ARG;
  }
  *out = p;
  return MM_OK;
}

extern "C" void mm_plan_destroy(mm_plan p) {
  if (!p) return;
  delete[] p->h_gen_chunks;
  delete[] p->h_gen_ctile;
  delete[] p->h_desc;
  delete[] p->h_chunk_group;
  delete[] p->h_batches;
  delete[] p->h_fused_first;
  delete[] p->h_fused_n;
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  if (p->adapt_exec) cudaGraphExecDestroy(p->adapt_exec);
  if (p->graph_stream) cudaStreamDestroy(p->graph_stream);
  delete p;
}

// Run a sequence of launches over every batch (in order, on one stream), failing on the
// first launch error.  `B` names the current batch inside `seq`.
#define FOR_BATCHES(seq)                                                  \
  for (int b_ = 0; b_ < p->n_batches; ++b_) {                             \
    const Batch& B = p->h_batches[b_];                                    \
    (void)B;                                                              \
    cudaError_t e_ = cudaSuccess;                                         \
    seq;                                                                  \
    if (e_ != cudaSuccess) {                                              \
      mm_set_error("%s: %s", #seq, cudaGetErrorString(e_));               \
      return MM_ERR_CUDA;                                                 \
    }                                                                     \
  }
#define L_(call) if (e_ == cudaSuccess) e_ = (call)

static mm_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mm_set_error("%s: %s", what, cudaGetErrorString(e));
    return MM_ERR_CUDA;
  }
  return MM_OK;
}
#define LAUNCHED(what)                                   \
  do {                                                   \
    mm_status st_ = check_launch(what);             \
    if (st_ != MM_OK) return st_;                        \
  } while (0)

extern "C" mm_status mm_set_noise_psd(mm_plan p, const double* psd_dev, const double* params,
                                      const double* tau, const float* tod, void* stream) {
  MmRange nvtx_range_("mm_set_noise_psd");
  MM_ARG(p != nullptr, "plan is NULL");
  MM_ARG((psd_dev != nullptr) != (params != nullptr), "give exactly one of psd / params");
  MM_ARG(tod != nullptr, "tod is NULL");
  MM_ARG(((uintptr_t)tod & 7) == 0, "tod must be 8-byte aligned");
  cudaStream_t s = S(stream);
  const int C = p->n_chunks;
  std::vector<double> taus(C);
  if (params) {
    for (int c = 0; c < C; ++c) {
      const double* q = params + 4 * c;
      MM_ARG(q[0] > 0 && q[1] >= 0 && q[3] > 0 && isfinite(q[2]),
             "chunk %d: params (sigma, f_knee, alpha, f_sample) invalid", c);
      taus[c] = tau ? tau[c] : q[0] * q[0];
    }
  } else if (tau) {
    for (int c = 0; c < C; ++c) taus[c] = tau[c];
  } else {
    // tau_c = min_k N_c(f_k)
    k_min_psd<<<C, 256, 0, s>>>(p->d_desc, psd_dev, p->params);
    LAUNCHED("k_min_psd");
    MM_CUDA(cudaMemcpyAsync(taus.data(), p->params, sizeof(double) * C, cudaMemcpyDeviceToHost, s));
    MM_CUDA(cudaStreamSynchronize(s));
  }
  for (int c = 0; c < C; ++c) {
    MM_ARG(taus[c] > 0 && isfinite(taus[c]), "chunk %d: tau must be positive", c);
    p->h_desc[c].tau = taus[c];
  }
  MM_CUDA(cudaMemcpyAsync(p->d_desc, p->h_desc, sizeof(ChunkDesc) * C, cudaMemcpyHostToDevice, s));
  if (p->n_gen > 0) MM_CUDA(gen_upload(p, s));     // the general records carry tau too
  const double* d_params = nullptr;
  if (params) {
    MM_CUDA(cudaMemcpyAsync(p->params, params, sizeof(double) * 4 * C, cudaMemcpyHostToDevice, s));
    d_params = p->params;
  }
  MM_CUDA(cudaMemsetAsync(p->c0, 0, sizeof(double) * C, s));
  MM_CUDA(cudaMemsetAsync(p->scal, 0, sizeof(double) * kScalCount, s));
  NoiseArgs na{p->d_desc, psd_dev, d_params, p->nbar, p->nyq, p->c0, p->scal};
  {
    int maxM = 0;
    for (int c = 0; c < C; ++c) maxM = p->h_desc[c].M > maxM ? p->h_desc[c].M : maxM;
    const int per = 256 * 16;
    k_noise<<<dim3((maxM + per - 1) / per, C), 256, 0, s>>>(na);
    LAUNCHED("k_noise");
  }
  // scal[kScalTmp] holds min(Nbar) if it went negative
  double mn = 0.0;
  MM_CUDA(cudaMemcpyAsync(&mn, p->scal + kScalTmp, sizeof(double), cudaMemcpyDeviceToHost, s));
  MM_CUDA(cudaStreamSynchronize(s));
  if (mn < 0.0) {
    mm_set_error("Nbar = N - tau is negative (min %.3e): tau exceeds the noise spectrum", mn);
    return MM_ERR_ARG;
  }

  // weight blocks, pixel cut, W and the PCG preconditioner
  const int blk = p->ncomp == 3 ? 6 : 1;
  MM_CUDA(cudaMemsetAsync(p->acc12, 0, sizeof(double) * 2 * blk * p->n_pix, s));
  // one launch per chunk keeps the chunk's scales without a per-sample search
  for (int c = 0; c < C; ++c) {
    const ChunkDesc& d = p->h_desc[c];
    if (!p->composite) {
      k_weights_accum<<<blocks_for(d.n, 256), 256, 0, s>>>(
          p->d_desc, c, p->pix, p->cosw, p->sinw, p->wdtype == MM_W_F16, p->ncomp, p->c0, d.off,
          d.off + d.n, p->acc12, 1.0);
    } else {
      // D = P_A^T T_A^-1 P_A + P_B^T T_B^-1 P_B with T_A = T_B = tau / 2 (App. B); the gains
      // enter squared
      k_weights_accum<<<blocks_for(d.n, 256), 256, 0, s>>>(
          p->d_desc, c, p->pix, p->cosw, p->sinw, p->wdtype == MM_W_F16, p->ncomp, p->c0, d.off,
          d.off + d.n, p->acc12, 2.0 * (double)p->gain_a * p->gain_a);
      k_weights_accum<<<blocks_for(d.n, 256), 256, 0, s>>>(
          p->d_desc, c, p->pix_b, p->cos_b, p->sin_b, p->wdtype == MM_W_F16, p->ncomp, p->c0,
          d.off, d.off + d.n, p->acc12, 2.0 * (double)p->gain_b * p->gain_b);
    }
  }
  LAUNCHED("k_weights_accum");
  unsigned long long* d_nvalid = reinterpret_cast<unsigned long long*>(p->scal + kScalTmp + 1);
  MM_CUDA(cudaMemsetAsync(d_nvalid, 0, 8, s));
  k_pixel_solve<<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, p->ncomp, p->rcond_min, p->hits,
                                                          p->acc12, p->valid, p->W, p->Minv, d_nvalid);
  LAUNCHED("k_pixel_solve");

  // d~ = rfft(d) into the row-layout table
  {
    RowArgs a{kRowSpectrum, 1.0, nullptr, nullptr};
    FOR_BATCHES(L_(launch_col_forward(p, B, kSrcTod, tod, s)); L_(launch_row(p, B, a, s)));
  }
  // b = P^T N^-1 d and d^T N^-1 d
  {
    MM_CUDA(cudaMemsetAsync(p->acc, 0, sizeof(double) * p->ncomp * acc_stride_of(p->n_pix, p->ncomp), s));
    RowArgs a{kRowPcgRhs, 1.0, p->scal + kScalCdd, nullptr};
    FOR_BATCHES(L_(launch_row(p, B, a, s)); L_(launch_col_inverse(p, B, s)));
    const int64_t len = p->ncomp * p->n_pix;
    k_finish_b<<<blocks_for(len, 256), 256, 0, s>>>(len, p->ncomp, p->acc, p->valid, p->bvec);
    LAUNCHED("k_finish_b");
  }
  unsigned long long nvalid = 0;
  MM_CUDA(cudaMemcpyAsync(&nvalid, d_nvalid, 8, cudaMemcpyDeviceToHost, s));
  MM_CUDA(cudaStreamSynchronize(s));
  if (nvalid == 0) {
    mm_set_error("every pixel was cut (no pixel with hits and rcond >= %g)", p->rcond_min);
    return MM_ERR_SINGULAR;
  }
  p->theta_ok = params != nullptr && tau == nullptr;
  p->noise_set = true;
  return MM_OK;
}

extern "C" mm_status mm_lambda_max(mm_plan p, double* out, void* stream) {
  MM_ARG(p != nullptr && out != nullptr, "NULL argument");
  if (!p->noise_set) { mm_set_error("mm_set_noise_psd has not run"); return MM_ERR_STATE; }
  MM_CUDA(cudaMemcpyAsync(out, p->scal + kScalLambdaMax, sizeof(double), cudaMemcpyDeviceToHost, S(stream)));
  MM_CUDA(cudaStreamSynchronize(S(stream)));
  return MM_OK;
}

static mm_status load_map(mm_plan p, const double* map, cudaStream_t s) {
  if (p->ncomp == 3) k_map_to4<3><<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, map, p->valid, p->map4);
  else k_map_to4<1><<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, map, p->valid, p->map4);
  LAUNCHED("k_map_to4");
  return MM_OK;
}

static mm_status check_waits(mm_plan p, cudaStream_t s, const char* who);

extern "C" mm_status mm_messenger_iterate(mm_plan p, const double* lambdas, int n_iter, int precision,
                                          double* map_inout, double* chi2_out, void* stream) {
  MmRange nvtx_range_("mm_messenger_iterate");
  MM_ARG(p != nullptr, "plan is NULL");
  MM_ARG(n_iter >= 0, "n_iter must be >= 0");
  MM_ARG(n_iter == 0 || lambdas != nullptr, "lambdas is NULL");
  MM_ARG(map_inout != nullptr, "map_inout is NULL");
  if (precision != MM_FP32_MIXED) {
    mm_set_error("precision mode %d not supported", precision);
    return MM_ERR_UNSUPPORTED;
  }
  if (!p->noise_set) { mm_set_error("mm_set_noise_psd has not run"); return MM_ERR_STATE; }
  for (int i = 0; i < n_iter; ++i)
    MM_ARG(lambdas[i] >= 1.0 || isinf(lambdas[i]), "lambdas[%d] = %g must be >= 1 or inf", i, lambdas[i]);
  if (n_iter == 0) return MM_OK;
  cudaStream_t s = S(stream);
  mm_status st = load_map(p, map_inout, s);
  if (st != MM_OK) return st;
  if (chi2_out) MM_CUDA(cudaMemsetAsync(chi2_out, 0, sizeof(double) * n_iter, s));
  if (p->composite) {
    // App. B: m' = m + D^-1 P^T (Nbar / lambda + T)^-1 (d - P m), the map kept in FP64
    MM_CUDA(cudaMemcpyAsync(p->map64, map_inout, sizeof(double) * p->ncomp * p->n_pix,
                            cudaMemcpyDeviceToDevice, s));
    for (int it = 0; it < n_iter; ++it) {
      RowArgs a{kRowResidual, lambdas[it], chi2_out ? chi2_out + it : nullptr, nullptr};
      FOR_BATCHES(L_(launch_col_forward(p, B, kSrcGather, nullptr, s)); L_(launch_row(p, B, a, s));
                  L_(launch_col_inverse(p, B, s)));
      double* mo = it == n_iter - 1 ? map_inout : nullptr;
      if (p->ncomp == 3)
        k_bin_resid<3><<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, p->acc, p->W, p->valid, p->map64, p->map4, mo);
      else
        k_bin_resid<1><<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, p->acc, p->W, p->valid, p->map64, p->map4, mo);
      LAUNCHED("k_bin_resid");
    }
    return MM_OK;
  }
  for (int it = 0; it < n_iter; ++it) {
    RowArgs a{kRowMessenger, lambdas[it], chi2_out ? chi2_out + it : nullptr, nullptr};
    FOR_BATCHES(if (fused_eligible(p, B)) { L_(launch_fused(p, B, a, s)); } else {
                  L_(launch_col_forward(p, B, kSrcGather, nullptr, s)); L_(launch_row(p, B, a, s));
                  L_(launch_col_inverse(p, B, s)); });
    double* mo = it == n_iter - 1 ? map_inout : nullptr;
    if (p->ncomp == 3) k_bin_apply<3><<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, p->acc, p->W, p->map4, mo);
    else k_bin_apply<1><<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, p->acc, p->W, p->map4, mo);
    LAUNCHED("k_bin_apply");
  }
  return check_waits(p, s, "mm_messenger_iterate");
}

mm_status mm::messenger_step_keep(mm_plan_s* p, double lambda, double* map_inout, float2* keep,
                                  cudaStream_t s) {
  mm_status st = load_map(p, map_inout, s);
  if (st != MM_OK) return st;
  RowArgs a{kRowMessengerKeep, lambda, nullptr, keep};
  FOR_BATCHES(L_(launch_col_forward(p, B, kSrcGather, nullptr, s)); L_(launch_row(p, B, a, s));
              L_(launch_col_inverse(p, B, s)));
  if (p->ncomp == 3) k_bin_apply<3><<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, p->acc, p->W, p->map4, map_inout);
  else k_bin_apply<1><<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, p->acc, p->W, p->map4, map_inout);
  LAUNCHED("k_bin_apply");
  return MM_OK;
}

// ------------------------------------------------------- map-sized form of the iteration
// Sec. 2.1 writes the step as m' = m_d(lambda) + F(lambda) m with
//   m_d(lambda) = W P^T T^-1 F^-1[ lambda tau d~ / (lambda tau + Nbar) ]   (data only)
//   F(lambda) m = W P^T T^-1 F^-1[ Nbar (P m)~ / (lambda tau + Nbar) ]     (map only).
// m_d is formed once per distinct lambda, after which an iteration no longer reads d~.  Its
// chi^2 (Eq. 3) is assembled without d~ as
//   chi^2(m) = d^T N^-1 d - 2 m . b + sum_k w_k |(P m)~_k|^2 / (n N_k),  b = P^T N^-1 d,
// the first two terms by the map step that produces m, the last by the row pass that reads
// it.

// out = m_d + W acc (m_d may be NULL); acc cleared; map4 (FP32 gather copy) and map_out
// written when given; chi2_next (when given) receives d^T N^-1 d - 2 out . b.
template <int NC>
__global__ void k_bin_md(int64_t n_pix, double* __restrict__ acc, const double* __restrict__ W,
                         const double* __restrict__ md, void* map4, double* __restrict__ map_out,
                         const double* __restrict__ bvec, const double* __restrict__ cdd,
                         double* __restrict__ chi2_next) {
  __shared__ double red[32];
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double dot = 0.0;
  if (p < n_pix) {
    constexpr int B = NC == 3 ? 6 : 1;
    double a[NC], w[B], m[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
    const int64_t j_ = i * acc_stride_of(n_pix, NC) + p;   // planar accumulators
    a[i] = acc[j_];
    acc[j_] = 0.0;
  }
#pragma unroll
    for (int i = 0; i < B; ++i) w[i] = W[B * p + i];
    sym_apply<NC>(w, a, m);
    if (md)
#pragma unroll
      for (int i = 0; i < NC; ++i) m[i] += md[NC * p + i];
    if (map4) store_map4<NC>(map4, p, m);
    if (map_out)
#pragma unroll
      for (int i = 0; i < NC; ++i) map_out[NC * p + i] = m[i];
    if (chi2_next)
#pragma unroll
      for (int i = 0; i < NC; ++i) dot += m[i] * bvec[NC * p + i];
  }
  if (chi2_next == nullptr) return;
  const double sum = block_sum(dot, red);
  if (threadIdx.x == 0) {
    atomicAdd(chi2_next, -2.0 * sum);
    if (blockIdx.x == 0) atomicAdd(chi2_next, *cdd);
  }
}

// chi2 slot of the first iteration: d^T N^-1 d - 2 m . b for the caller's map (b is zero on
// cut pixels).
__global__ void k_chi2_md_start(int64_t len, const double* __restrict__ m,
                                const double* __restrict__ bvec, const double* __restrict__ cdd,
                                double* __restrict__ chi2) {
  __shared__ double red[32];
  double dot = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    dot += m[i] * bvec[i];
  const double sum = block_sum(dot, red);
  if (threadIdx.x == 0) {
    atomicAdd(chi2, -2.0 * sum);
    if (blockIdx.x == 0) atomicAdd(chi2, *cdd);
  }
}

extern "C" mm_status mm_messenger_md_bytes(mm_plan p, int n_levels, size_t* bytes) {
  MM_ARG(p != nullptr && bytes != nullptr, "NULL argument");
  MM_ARG(n_levels >= 1, "n_levels must be >= 1");
  *bytes = sizeof(double) * (size_t)p->ncomp * (size_t)p->n_pix * (size_t)n_levels;
  return MM_OK;
}

extern "C" mm_status mm_messenger_iterate_md(mm_plan p, const double* lambdas, int n_iter,
                                             double* map_inout, double* chi2_out, void* work,
                                             size_t work_bytes, void* stream) {
  MmRange nvtx_range_("mm_messenger_iterate_md");
  if (p && p->composite) {
    mm_set_error("mm_messenger_iterate_md: not available for composite-pointing plans");
    return MM_ERR_UNSUPPORTED;
  }
  MM_ARG(p != nullptr, "plan is NULL");
  MM_ARG(n_iter >= 0, "n_iter must be >= 0");
  MM_ARG(n_iter == 0 || lambdas != nullptr, "lambdas is NULL");
  MM_ARG(map_inout != nullptr, "map_inout is NULL");
  if (!p->noise_set) { mm_set_error("mm_set_noise_psd has not run"); return MM_ERR_STATE; }
  for (int i = 0; i < n_iter; ++i)
    MM_ARG(lambdas[i] >= 1.0 || isinf(lambdas[i]), "lambdas[%d] = %g must be >= 1 or inf", i, lambdas[i]);
  if (n_iter == 0) return MM_OK;
  // distinct lambdas in order of first use: one m_d map each
  std::vector<double> lv;
  std::vector<int> lev(n_iter);
  for (int i = 0; i < n_iter; ++i) {
    int j = 0;
    while (j < (int)lv.size() && !(lv[j] == lambdas[i])) ++j;
    if (j == (int)lv.size()) lv.push_back(lambdas[i]);
    lev[i] = j;
  }
  const size_t per = sizeof(double) * (size_t)p->ncomp * (size_t)p->n_pix;
  MM_ARG(work != nullptr && ((uintptr_t)work & 255) == 0, "work must be 256-byte aligned");
  if (work_bytes < per * lv.size()) {
    mm_set_error("work holds %zu m_d maps, the schedule has %zu distinct lambdas",
                 work_bytes / per, lv.size());
    return MM_ERR_NOMEM;
  }
  double* md = static_cast<double*>(work);
  const int64_t len = p->ncomp * p->n_pix;
  cudaStream_t s = S(stream);
  const unsigned nbp = blocks_for(p->n_pix, 256);
  MM_CUDA(cudaMemsetAsync(p->acc, 0, sizeof(double) * p->ncomp * acc_stride_of(p->n_pix, p->ncomp), s));
  for (size_t j = 0; j < lv.size(); ++j) {
    RowArgs a{kRowMd, lv[j], nullptr, nullptr};
    FOR_BATCHES(L_(launch_row(p, B, a, s)); L_(launch_col_inverse(p, B, s)));
    double* out = md + (size_t)p->ncomp * p->n_pix * j;
    if (p->ncomp == 3)
      k_bin_md<3><<<nbp, 256, 0, s>>>(p->n_pix, p->acc, p->W, nullptr, nullptr, out, nullptr, nullptr, nullptr);
    else
      k_bin_md<1><<<nbp, 256, 0, s>>>(p->n_pix, p->acc, p->W, nullptr, nullptr, out, nullptr, nullptr, nullptr);
    LAUNCHED("k_bin_md (m_d)");
  }
  mm_status st = load_map(p, map_inout, s);
  if (st != MM_OK) return st;
  if (chi2_out) {
    MM_CUDA(cudaMemsetAsync(chi2_out, 0, sizeof(double) * n_iter, s));
    k_chi2_md_start<<<blocks_for(len, 256) < 1024 ? blocks_for(len, 256) : 1024, 256, 0, s>>>(
        len, map_inout, p->bvec, p->scal + kScalCdd, chi2_out);
    LAUNCHED("k_chi2_md_start");
  }
  for (int it = 0; it < n_iter; ++it) {
    RowArgs a{kRowMessengerF, lambdas[it], chi2_out ? chi2_out + it : nullptr, nullptr};
    FOR_BATCHES(if (fused_eligible(p, B)) { L_(launch_fused(p, B, a, s)); } else {
                  L_(launch_col_forward(p, B, kSrcGather, nullptr, s)); L_(launch_row(p, B, a, s));
                  L_(launch_col_inverse(p, B, s)); });
    const double* mdl = md + (size_t)p->ncomp * p->n_pix * lev[it];
    double* mo = it == n_iter - 1 ? map_inout : nullptr;
    double* cn = chi2_out && it + 1 < n_iter ? chi2_out + it + 1 : nullptr;
    if (p->ncomp == 3)
      k_bin_md<3><<<nbp, 256, 0, s>>>(p->n_pix, p->acc, p->W, mdl, p->map4, mo, p->bvec, p->scal + kScalCdd, cn);
    else
      k_bin_md<1><<<nbp, 256, 0, s>>>(p->n_pix, p->acc, p->W, mdl, p->map4, mo, p->bvec, p->scal + kScalCdd, cn);
    LAUNCHED("k_bin_md");
  }
  return check_waits(p, s, "mm_messenger_iterate_md");
}

extern "C" mm_status mm_plan_fault_flags(mm_plan p, int* flags, void* stream) {
  MM_ARG(p != nullptr && flags != nullptr, "NULL argument");
  cudaStream_t s = S(stream);
  int f = 0;
  MM_CUDA(cudaMemcpyAsync(&f, p->fault, sizeof(int), cudaMemcpyDeviceToHost, s));
  MM_CUDA(cudaStreamSynchronize(s));
  MM_CUDA(cudaMemsetAsync(p->fault, 0, sizeof(int), s));
  *flags = f;
  return MM_OK;
}

// With the plan's check-on-return policy: synchronise `s` and report a bounded wait that
// ran out in the launches queued so far (MM_ERR_TIMEOUT; the flag is cleared).
static mm_status check_waits(mm_plan p, cudaStream_t s, const char* who) {
  if (!p->check_on_return) return MM_OK;
  int f = 0;
  MM_CUDA(cudaMemcpyAsync(&f, p->fault, sizeof(int), cudaMemcpyDeviceToHost, s));
  MM_CUDA(cudaStreamSynchronize(s));
  if (f) {
    MM_CUDA(cudaMemsetAsync(p->fault, 0, sizeof(int), s));
    mm_set_error("%s: a bounded wait of the fused launch ran out (its results are wrong)", who);
    return MM_ERR_TIMEOUT;
  }
  return MM_OK;
}

extern "C" mm_status mm_plan_set_wait_policy(mm_plan p, int n_polls, int check_on_return) {
  MM_ARG(p != nullptr, "plan is NULL");
  MM_ARG(n_polls >= 1 && n_polls <= (1 << 22), "n_polls must be in [1, 2^22]");
  MM_ARG(check_on_return == 0 || check_on_return == 1, "check_on_return must be 0 or 1");
  if (n_polls != p->wait_polls) {   // captured graphs hold the old limit: capture again
    if (p->graph_exec) { cudaGraphExecDestroy(p->graph_exec); p->graph_exec = nullptr; }
    if (p->adapt_exec) { cudaGraphExecDestroy(p->adapt_exec); p->adapt_exec = nullptr; }
  }
  p->wait_polls = n_polls;
  p->check_on_return = check_on_return;
  return MM_OK;
}

extern "C" mm_status mm_plan_fused_batches(mm_plan p, int* n_fused) {
  MM_ARG(p != nullptr && n_fused != nullptr, "NULL argument");
  int n = 0;
  for (int b = 0; b < p->n_batches; ++b) n += fused_eligible(p, p->h_batches[b]) ? 1 : 0;
  *n_fused = n;
  return MM_OK;
}

extern "C" mm_status mm_plan_batches(mm_plan p, int* n_batches) {
  MM_ARG(p != nullptr && n_batches != nullptr, "NULL argument");
  *n_batches = p->n_batches;
  return MM_OK;
}

extern "C" mm_status mm_messenger_stage(mm_plan p, int stage, int batch, double lambda,
                                        double* map_inout, double* chi2_slot, void* stream) {
  if (p && p->composite) {
    mm_set_error("mm_messenger_stage: not available for composite-pointing plans");
    return MM_ERR_UNSUPPORTED;
  }
  MM_ARG(p != nullptr, "plan is NULL");
  if (!p->noise_set) { mm_set_error("mm_set_noise_psd has not run"); return MM_ERR_STATE; }
  cudaStream_t s = S(stream);
  const bool per_batch = stage == MM_STAGE_GATHER_FFT || stage == MM_STAGE_FILTER ||
                         stage == MM_STAGE_IFFT_BIN || stage == MM_STAGE_FUSED;
  if (per_batch) MM_ARG(batch >= 0 && batch < p->n_batches, "batch %d out of range", batch);
  cudaError_t e = cudaSuccess;
  switch (stage) {
    case MM_STAGE_LOAD:
      MM_ARG(map_inout != nullptr, "map_inout is NULL");
      return load_map(p, map_inout, s);
    case MM_STAGE_GATHER_FFT:
      e = launch_col_forward(p, p->h_batches[batch], kSrcGather, nullptr, s);
      break;
    case MM_STAGE_FILTER: {
      MM_ARG(lambda >= 1.0 || isinf(lambda), "lambda = %g must be >= 1 or inf", lambda);
      RowArgs a{kRowMessenger, lambda, chi2_slot, nullptr};
      e = launch_row(p, p->h_batches[batch], a, s);
      break;
    }
    case MM_STAGE_IFFT_BIN:
      e = launch_col_inverse(p, p->h_batches[batch], s);
      break;
    case MM_STAGE_FUSED: {
      MM_ARG(lambda >= 1.0 || isinf(lambda), "lambda = %g must be >= 1 or inf", lambda);
      if (!fused_eligible(p, p->h_batches[batch])) {
        mm_set_error("batch %d does not run as one fused launch", batch);
        return MM_ERR_UNSUPPORTED;
      }
      RowArgs a{kRowMessenger, lambda, chi2_slot, nullptr};
      e = launch_fused(p, p->h_batches[batch], a, s);
      break;
    }
    case MM_STAGE_MAP:
      if (p->ncomp == 3) k_bin_apply<3><<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, p->acc, p->W, p->map4, map_inout);
      else k_bin_apply<1><<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, p->acc, p->W, p->map4, map_inout);
      LAUNCHED("k_bin_apply");
      return MM_OK;
    default:
      mm_set_error("unknown stage %d", stage);
      return MM_ERR_ARG;
  }
  if (e != cudaSuccess) {
    mm_set_error("stage %d launch: %s", stage, cudaGetErrorString(e));
    return MM_ERR_CUDA;
  }
  return MM_OK;
}

// Capture one messenger iteration (every batch's three kernels, then the map step) as a CUDA
// graph whose cooling parameter and chi^2 slot come from device memory.
// The kernels of one graph-mode iteration (lambda and the chi^2 slot from device memory,
// the iteration counter advanced by the map step) launched on s.
static cudaError_t launch_iteration(mm_plan p, cudaStream_t s) {
  RowArgs a{kRowMessenger, 1.0, nullptr, nullptr};
  a.lam_table = p->lam_table;
  a.iter = p->iter;
  a.chi2_base = p->chi2_base;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < p->n_batches && e == cudaSuccess; ++b) {
    const Batch& B = p->h_batches[b];
    if (fused_eligible(p, B)) {
      e = launch_fused(p, B, a, s);
      continue;
    }
    if ((e = launch_col_forward(p, B, kSrcGather, nullptr, s)) != cudaSuccess) break;
    if ((e = launch_row(p, B, a, s)) != cudaSuccess) break;
    e = launch_col_inverse(p, B, s);
  }
  if (e != cudaSuccess) return e;
  if (p->ncomp == 3)
    k_bin_apply<3><<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, p->acc, p->W, p->map4, p->map64, p->iter);
  else
    k_bin_apply<1><<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, p->acc, p->W, p->map4, p->map64, p->iter);
  return cudaGetLastError();
}

static mm_status capture_iteration_graph(mm_plan p) {
  if (p->graph_exec) return MM_OK;
  if (!p->graph_stream)
    MM_CUDA(cudaStreamCreateWithFlags(&p->graph_stream, cudaStreamNonBlocking));
  cudaStream_t s = p->graph_stream;
  // relaxed: the launchers may query occupancy / set kernel attributes on first use
  MM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  cudaError_t e = launch_iteration(p, s);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(s, &graph);
  if (e != cudaSuccess || ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    mm_set_error("graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : ec));
    return MM_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&p->graph_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    p->graph_exec = nullptr;
    mm_set_error("graph instantiate failed: %s", cudaGetErrorString(e));
    return MM_ERR_CUDA;
  }
  return MM_OK;
}

// Plateau-driven cooling (Sec. 3.1), one thread after each iteration's map step: decides
// the next iteration's lambda from the chi^2 of the maps entering the last two iterations
// and ends the loop (condition 0) after the last level's plateau or max_iter iterations.
__global__ void k_adapt(AdaptState* __restrict__ st, double* __restrict__ lam_table,
                        const int* __restrict__ iter, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0) return;
  const int it = *iter;                    // iterations done
  bool go = it < st->max_iter;
  if (go) {
    if (st->level < 0) {
      st->level = 0;
      st->start = it;
    } else {
      const int count = it - st->start;
      bool plateau = false;
      if (it - 2 >= st->start) {
        const double rel = (st->chi2[it - 2] - st->chi2[it - 1]) / st->chi2[it - 1];
        plateau = rel < st->rel_tol;
      }
      const bool last = st->level == st->n_levels - 1;
      if ((count >= st->min_per && plateau) || (!last && count >= st->max_per)) {
        if (last) {
          go = false;
        } else {
          st->level += 1;
          st->start = it;
        }
      }
    }
  }
  if (go) {
    const double lam = st->levels[st->level];
    lam_table[it] = lam;
    st->lambda_out[it] = lam;
  } else {
    st->n_done = it;
  }
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// One graph: a WHILE conditional node whose body is one iteration plus the controller.
static mm_status build_adaptive_graph(mm_plan p) {
  if (p->adapt_exec) return MM_OK;
  if (!p->graph_stream)
    MM_CUDA(cudaStreamCreateWithFlags(&p->graph_stream, cudaStreamNonBlocking));
  cudaStream_t s = p->graph_stream;
  cudaGraph_t g = nullptr;
  MM_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  // the parameter union has no default constructor: zero-filled storage stands in for it
  alignas(cudaGraphNodeParams) unsigned char np_buf[sizeof(cudaGraphNodeParams)];
  memset(np_buf, 0, sizeof(np_buf));
  cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_buf);
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  if (e == cudaSuccess) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t el = launch_iteration(p, s);
      if (el == cudaSuccess) {
        k_adapt<<<1, 32, 0, s>>>(static_cast<AdaptState*>(p->adapt_st), p->lam_table, p->iter, h);
        el = cudaGetLastError();
      }
      cudaGraph_t out = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(s, &out);
      e = el != cudaSuccess ? el : ec;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->adapt_exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    p->adapt_exec = nullptr;
    mm_set_error("adaptive graph: %s", cudaGetErrorString(e));
    return MM_ERR_CUDA;
  }
  return MM_OK;
}

extern "C" mm_status mm_messenger_adaptive(mm_plan p, const double* levels, int n_levels,
                                           double rel_tol, int min_per_level, int max_per_level,
                                           int max_iter, double* map_inout, double* chi2_out,
                                           double* lambda_out, int* n_done, void* stream) {
  MmRange nvtx_range_("mm_messenger_adaptive");
  if (p && p->composite) {
    mm_set_error("mm_messenger_adaptive: not available for composite-pointing plans");
    return MM_ERR_UNSUPPORTED;
  }
  MM_ARG(p != nullptr && levels != nullptr && map_inout != nullptr && chi2_out != nullptr &&
         lambda_out != nullptr && n_done != nullptr, "NULL argument");
  MM_ARG(n_levels >= 1 && n_levels <= kMaxLevels, "n_levels must be in [1, %d]", kMaxLevels);
  MM_ARG(max_iter >= 1 && max_iter <= p->lam_cap, "max_iter must be in [1, %d]", p->lam_cap);
  MM_ARG(min_per_level >= 2 && max_per_level >= min_per_level,
         "need 2 <= min_per_level <= max_per_level");
  MM_ARG(!isnan(rel_tol), "rel_tol is NaN");
  for (int j = 0; j < n_levels; ++j) {
    MM_ARG(isfinite(levels[j]) && levels[j] >= 1.0, "levels[%d] must be finite and >= 1", j);
    MM_ARG(j == 0 || levels[j] <= levels[j - 1], "levels must not increase");
  }
  if (!p->noise_set) { mm_set_error("mm_set_noise_psd has not run"); return MM_ERR_STATE; }
  mm_status st = build_adaptive_graph(p);
  if (st != MM_OK) return st;
  cudaStream_t s = S(stream);
  AdaptState h;
  memset(&h, 0, sizeof(h));
  h.level = -1;
  h.n_levels = n_levels;
  h.min_per = min_per_level;
  h.max_per = max_per_level;
  h.max_iter = max_iter;
  h.rel_tol = rel_tol;
  h.chi2 = chi2_out;
  h.lambda_out = lambda_out;
  for (int j = 0; j < n_levels; ++j) h.levels[j] = levels[j];
  const double inf = INFINITY;
  MM_CUDA(cudaMemcpyAsync(p->adapt_st, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  MM_CUDA(cudaMemcpyAsync(p->lam_table, &inf, sizeof(double), cudaMemcpyHostToDevice, s));
  MM_CUDA(cudaMemsetAsync(p->iter, 0, sizeof(int), s));
  MM_CUDA(cudaMemcpyAsync(p->chi2_base, &chi2_out, sizeof(double*), cudaMemcpyHostToDevice, s));
  MM_CUDA(cudaMemsetAsync(chi2_out, 0, sizeof(double) * max_iter, s));
  MM_CUDA(cudaMemsetAsync(lambda_out, 0, sizeof(double) * max_iter, s));
  MM_CUDA(cudaMemcpyAsync(lambda_out, &inf, sizeof(double), cudaMemcpyHostToDevice, s));
  st = load_map(p, map_inout, s);
  if (st != MM_OK) return st;
  MM_CUDA(cudaGraphLaunch(p->adapt_exec, s));
  MM_CUDA(cudaMemcpyAsync(map_inout, p->map64, sizeof(double) * p->ncomp * p->n_pix,
                          cudaMemcpyDeviceToDevice, s));
  MM_CUDA(cudaMemcpyAsync(n_done, reinterpret_cast<char*>(p->adapt_st) + offsetof(AdaptState, n_done),
                          sizeof(int), cudaMemcpyDeviceToDevice, s));
  return check_waits(p, s, "mm_messenger_adaptive");
}

extern "C" mm_status mm_messenger_graph(mm_plan p, const double* lambdas, int n_iter,
                                        double* map_inout, double* chi2_out, void* stream) {
  MmRange nvtx_range_("mm_messenger_graph");
  if (p && p->composite) {
    mm_set_error("mm_messenger_graph: not available for composite-pointing plans");
    return MM_ERR_UNSUPPORTED;
  }
  MM_ARG(p != nullptr && map_inout != nullptr, "NULL argument");
  MM_ARG(n_iter >= 0 && n_iter <= p->lam_cap, "n_iter must be in [0, %d]", p->lam_cap);
  MM_ARG(n_iter == 0 || lambdas != nullptr, "lambdas is NULL");
  if (!p->noise_set) { mm_set_error("mm_set_noise_psd has not run"); return MM_ERR_STATE; }
  for (int i = 0; i < n_iter; ++i)
    MM_ARG(lambdas[i] >= 1.0 || isinf(lambdas[i]), "lambdas[%d] = %g must be >= 1 or inf", i, lambdas[i]);
  if (n_iter == 0) return MM_OK;
  mm_status st = capture_iteration_graph(p);
  if (st != MM_OK) return st;
  cudaStream_t s = S(stream);
  MM_CUDA(cudaMemcpyAsync(p->lam_table, lambdas, sizeof(double) * n_iter, cudaMemcpyHostToDevice, s));
  MM_CUDA(cudaMemsetAsync(p->iter, 0, sizeof(int), s));
  MM_CUDA(cudaMemcpyAsync(p->chi2_base, &chi2_out, sizeof(double*), cudaMemcpyHostToDevice, s));
  if (chi2_out) MM_CUDA(cudaMemsetAsync(chi2_out, 0, sizeof(double) * n_iter, s));
  st = load_map(p, map_inout, s);
  if (st != MM_OK) return st;
  for (int it = 0; it < n_iter; ++it) MM_CUDA(cudaGraphLaunch(p->graph_exec, s));
  MM_CUDA(cudaMemcpyAsync(map_inout, p->map64, sizeof(double) * p->ncomp * p->n_pix,
                          cudaMemcpyDeviceToDevice, s));
  return check_waits(p, s, "mm_messenger_graph");
}

extern "C" mm_status mm_pcg_state_bytes(mm_plan p, size_t* bytes) {
  MM_ARG(p != nullptr && bytes != nullptr, "NULL argument");
  *bytes = up(sizeof(double) * 4 * p->ncomp * p->n_pix) + up(sizeof(double) * kPcgNs);
  return MM_OK;
}

static mm_status apply_A(mm_plan p, cudaStream_t s) {
  RowArgs a{kRowPcgApply, 1.0, nullptr, nullptr};
  FOR_BATCHES(if (fused_eligible(p, B)) { L_(launch_fused(p, B, a, s)); } else {
                L_(launch_col_forward(p, B, kSrcGather, nullptr, s)); L_(launch_row(p, B, a, s));
                L_(launch_col_inverse(p, B, s)); });
  return MM_OK;
}

extern "C" mm_status mm_pcg_iterate(mm_plan p, int n_iter, double* map_inout, void* state, int restart,
                                    double* chi2_out, void* stream) {
  MmRange nvtx_range_("mm_pcg_iterate");
  if (p && p->composite) {
    mm_set_error("mm_pcg_iterate: not available for composite-pointing plans");
    return MM_ERR_UNSUPPORTED;
  }
  MM_ARG(p != nullptr && map_inout != nullptr && state != nullptr, "NULL argument");
  MM_ARG(((uintptr_t)state & 255) == 0, "state must be 256-byte aligned");
  MM_ARG(n_iter >= 0, "n_iter must be >= 0");
  if (!p->noise_set) { mm_set_error("mm_set_noise_psd has not run"); return MM_ERR_STATE; }
  cudaStream_t s = S(stream);
  const int64_t len = p->ncomp * p->n_pix;
  double* r = static_cast<double*>(state);
  double* z = r + len;
  double* pv = z + len;
  double* q = pv + len;
  double* sc = reinterpret_cast<double*>(static_cast<char*>(state) + up(sizeof(double) * 4 * len));
  const unsigned nb = blocks_for(p->n_pix, 256), nbl = blocks_for(len, 256);
  const bool tri = p->ncomp == 3;
  if (restart) {
    MM_CUDA(cudaMemsetAsync(sc, 0, sizeof(double) * kPcgNs, s));
    mm_status st = load_map(p, map_inout, s);
    if (st != MM_OK) return st;
    st = apply_A(p, s);
    if (st != MM_OK) return st;
    if (tri) k_pcg_init<3><<<nb, 256, 0, s>>>(p->n_pix, p->acc, p->bvec, map_inout, p->valid, p->Minv, r, z, pv, p->map4, sc);
    else k_pcg_init<1><<<nb, 256, 0, s>>>(p->n_pix, p->acc, p->bvec, map_inout, p->valid, p->Minv, r, z, pv, p->map4, sc);
    LAUNCHED("k_pcg_init");
  } else {
    // continue: map4 must hold the current direction p
    if (tri) k_map_to4<3><<<nb, 256, 0, s>>>(p->n_pix, pv, p->valid, p->map4);
    else k_map_to4<1><<<nb, 256, 0, s>>>(p->n_pix, pv, p->valid, p->map4);
    LAUNCHED("k_map_to4");
  }
  for (int it = 0; it < n_iter; ++it) {
    // the parity of rz slots is kept in scalar slot 7 across calls
    MM_CUDA(cudaMemsetAsync(sc + kPcgPq, 0, sizeof(double), s));
    mm_status st = apply_A(p, s);
    if (st != MM_OK) return st;
    int cur = kPcgRz0, nxt = kPcgRz1;
    // parity bookkeeping on the host: each call restarts parity at slot 0 after copying
    k_pcg_q<<<nbl, 256, 0, s>>>(len, p->ncomp, p->acc, p->valid, pv, q, sc, nxt,
                                p->scal + kScalCdd, chi2_out ? chi2_out + it : nullptr);
    LAUNCHED("k_pcg_q");
    if (tri) k_pcg_update<3><<<nb, 256, 0, s>>>(p->n_pix, map_inout, r, z, pv, q, p->bvec, p->Minv, sc, cur, nxt);
    else k_pcg_update<1><<<nb, 256, 0, s>>>(p->n_pix, map_inout, r, z, pv, q, p->bvec, p->Minv, sc, cur, nxt);
    LAUNCHED("k_pcg_update");
    if (tri) k_pcg_dir<3><<<nb, 256, 0, s>>>(p->n_pix, z, pv, p->map4, sc, cur, nxt);
    else k_pcg_dir<1><<<nb, 256, 0, s>>>(p->n_pix, z, pv, p->map4, sc, cur, nxt);
    LAUNCHED("k_pcg_dir");
    // rz_cur <- rz_next for the next iteration
    MM_CUDA(cudaMemcpyAsync(sc + kPcgRz0, sc + kPcgRz1, sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  return check_waits(p, s, "mm_pcg_iterate");
}

extern "C" mm_status mm_chi2(mm_plan p, const double* map, double lambda, double* chi2_dev, void* stream) {
  MmRange nvtx_range_("mm_chi2");
  MM_ARG(p != nullptr && map != nullptr && chi2_dev != nullptr, "NULL argument");
  MM_ARG(lambda >= 1.0 && isfinite(lambda), "lambda must be finite and >= 1");
  if (!p->noise_set) { mm_set_error("mm_set_noise_psd has not run"); return MM_ERR_STATE; }
  cudaStream_t s = S(stream);
  MM_CUDA(cudaMemsetAsync(chi2_dev, 0, sizeof(double), s));
  mm_status st = load_map(p, map, s);
  if (st != MM_OK) return st;
  RowArgs a{kRowChi2, lambda, chi2_dev, nullptr};
  FOR_BATCHES(L_(launch_col_forward(p, B, kSrcGather, nullptr, s)); L_(launch_row(p, B, a, s)));
  return MM_OK;
}

// In place over `io`: on entry the natural-order rfft X_k of P m for every chunk (float2,
// chunk c at desc[c].spec + c, M + 1 bins), on exit |d~_k - X_k|^2 / (n N'_k) as float64
// (same 8 bytes per bin).  One thread per bin; the chunk is found by bisection on the
// bin offsets.  The weighted block sums go to *chi2 (when given) by one FP64 atomic each.
__global__ void k_chi2_modes(const ChunkDesc* __restrict__ desc, int n_chunks, int64_t n_bins,
                             const float2* __restrict__ dtab, const float* __restrict__ nbar,
                             const float* __restrict__ nyq, double lambda, void* io,
                             double* chi2) {
  double w = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_bins;
       i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = n_chunks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (desc[mid].nat <= i) lo = mid; else hi = mid - 1;
    }
    const ChunkDesc d = desc[lo];
    const int k = (int)(i - d.nat);
    const float2 X = reinterpret_cast<const float2*>(io)[i];
    double dre, dim = 0.0, nb;
    if (k == 0 && !d.cplx) { dre = dtab[d.spec].x; nb = nbar[d.spec]; }
    else if (k == d.M && !d.cplx) { dre = dtab[d.spec].y; nb = nyq[lo]; }
    else {
      const int64_t slot = d.spec + (int64_t)(k % d.M1) * d.M2 + k / d.M1;
      const float2 D = dtab[slot];
      dre = D.x; dim = D.y; nb = nbar[slot];
    }
    // FP32 per bin (the narrow FP64 pipe made this kernel the cost of the call), FP64 sums
    const float er = (float)dre - X.x, ei = (float)dim - X.y;
    const double v = (double)__fdividef(er * er + ei * ei, (float)(nb + lambda * d.tau)) / d.n;
    reinterpret_cast<double*>(io)[i] = v;
    w += (k == 0 || 2 * k == d.n) ? v : 2.0 * v;
  }
  if (chi2 == nullptr) return;
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x < 32) {
    w = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) atomicAdd(chi2, w);
  }
}

extern "C" mm_status mm_chi2_modes(mm_plan p, const double* map, double lambda, double* chi2_dev,
                                   double* modes, void* stream) {
  MmRange nvtx_range_("mm_chi2_modes");
  MM_ARG(p != nullptr && map != nullptr && modes != nullptr, "NULL argument");
  MM_ARG(((uintptr_t)modes & 7) == 0, "modes must be 8-byte aligned");
  MM_ARG(lambda >= 1.0 && isfinite(lambda), "lambda must be finite and >= 1");
  if (!p->noise_set) { mm_set_error("mm_set_noise_psd has not run"); return MM_ERR_STATE; }
  cudaStream_t s = S(stream);
  if (chi2_dev) MM_CUDA(cudaMemsetAsync(chi2_dev, 0, sizeof(double), s));
  mm_status st = load_map(p, map, s);
  if (st != MM_OK) return st;
  if (p->n_gen == 0) {
    // compile-time lengths: the row jobs write each mode's chi^2 to its natural-order slot
    // and add the total, in one forward pass
    RowArgs a{kRowChi2Modes, lambda, chi2_dev, reinterpret_cast<float2*>(modes)};
    FOR_BATCHES(L_(launch_col_forward(p, B, kSrcGather, nullptr, s)); L_(launch_row(p, B, a, s)));
    return MM_OK;
  }
  // general lengths: the spectrum of P m, natural order, into the caller's buffer (8 bytes
  // per bin either way), then one thread per bin
  RowArgs a{kRowNatural, 1.0, nullptr, reinterpret_cast<float2*>(modes)};
  FOR_BATCHES(L_(launch_col_forward(p, B, kSrcGather, nullptr, s)); L_(launch_row(p, B, a, s)));
  const ChunkDesc& last = p->h_desc[p->n_chunks - 1];
  const int64_t n_bins = last.nat + last.n / 2 + 1;
  int grid = 0;
  MM_CUDA(persistent_grid(k_chi2_modes, 256, 0, (int)std::min<int64_t>(blocks_for(n_bins, 256), 1 << 20), &grid));
  k_chi2_modes<<<grid, 256, 0, s>>>(
      p->d_desc, p->n_chunks, n_bins, p->dtab, p->nbar, p->nyq, lambda, modes, chi2_dev);
  LAUNCHED("k_chi2_modes");
  return MM_OK;
}

// ------------------------------------------------------------------- general-path schedule
static mm_status apply_tune(mm_plan p, const GenTune& t, cudaStream_t s) {
  p->gen_tune = t;
  cudaError_t e = gen_upload(p, s);
  if (e != cudaSuccess) {
    mm_set_error("general schedule upload: %s", cudaGetErrorString(e));
    return MM_ERR_CUDA;
  }
  if (p->graph_exec) {            // the captured iteration holds the old launch shapes
    cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
  }
  if (p->adapt_exec) {
    cudaGraphExecDestroy(p->adapt_exec);
    p->adapt_exec = nullptr;
  }
  return MM_OK;
}

extern "C" mm_status mm_get_tune(mm_plan p, int* col_nb, int* col_threads, int* row_threads,
                                 int* radix_order) {
  MM_ARG(p != nullptr, "plan is NULL");
  if (col_nb) *col_nb = p->gen_tune.col_nb;
  if (col_threads) *col_threads = p->gen_tune.col_threads;
  if (row_threads) *row_threads = p->gen_tune.row_threads;
  if (radix_order) *radix_order = p->gen_tune.radix_order;
  return MM_OK;
}

extern "C" mm_status mm_set_tune(mm_plan p, int col_nb, int col_threads, int row_threads,
                                 int radix_order, void* stream) {
  MM_ARG(p != nullptr, "plan is NULL");
  MM_ARG(col_nb == 8 || col_nb == 16, "col_nb must be 8 or 16");
  MM_ARG(col_threads == 256 || col_threads == 512, "col_threads must be 256 or 512");
  MM_ARG(row_threads == 256 || row_threads == 512 || row_threads == 1024,
         "row_threads must be 256, 512 or 1024");
  MM_ARG(radix_order >= 0 && radix_order <= 2, "radix_order must be 0, 1 or 2");
  if (p->n_gen == 0) return MM_OK;
  return apply_tune(p, GenTune{col_nb, col_threads, row_threads, radix_order}, S(stream));
}

// Time `reps` runs of `fn` on stream s (after one untimed run); fastest run in ms.
template <typename F>
static cudaError_t time_min(cudaStream_t s, int reps, F fn, float* best) {
  cudaEvent_t a, b;
  cudaError_t e;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return e; }
  *best = 1e30f;
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
    if ((e = cudaEventRecord(a, s)) != cudaSuccess) break;
    if ((e = fn()) != cudaSuccess) break;
    if ((e = cudaEventRecord(b, s)) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, a, b)) != cudaSuccess) break;
    if (r > 0 && ms < *best) *best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e;
}

extern "C" mm_status mm_autotune(mm_plan p, void* stream) {
  MmRange nvtx_range_("mm_autotune");
  MM_ARG(p != nullptr, "plan is NULL");
  if (p->n_gen == 0) return MM_OK;
  if (!p->noise_set) { mm_set_error("mm_set_noise_psd has not run"); return MM_ERR_STATE; }
  cudaStream_t s = S(stream);
  const GenTune keep = p->gen_tune;
  // the candidates run the column passes (gather from the current map, bin into acc) and
  // the row pass in PCG-operator mode, which touch only scratch (ybuf, acc), cleared below
  auto cols = [&]() -> cudaError_t {
    for (int b = 0; b < p->n_batches; ++b) {
      const Batch& B = p->h_batches[b];
      if (B.group >= 0) continue;
      cudaError_t e = launch_gen_col_forward(p, B, kSrcGather, nullptr, s);
      if (e == cudaSuccess) e = launch_gen_col_inverse(p, B, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  const RowArgs ra{kRowPcgApply, 1.0, nullptr, nullptr};
  auto rows = [&]() -> cudaError_t {
    for (int b = 0; b < p->n_batches; ++b) {
      const Batch& B = p->h_batches[b];
      if (B.group < 0) {
        cudaError_t e = launch_gen_row(p, B, ra, s);
        if (e != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  };
  const int nbs[2] = {8, 16}, cts[2] = {256, 512}, rts[3] = {256, 512, 1024};
  GenTune best = keep;
  float best_total = 1e30f;
  for (int order = 0; order < 3; ++order) {
    GenTune t = keep;
    t.radix_order = order;
    float bc = 1e30f, br = 1e30f;
    GenTune tc = t;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        t.col_nb = nbs[i];
        t.col_threads = cts[j];
        mm_status st = apply_tune(p, t, s);
        if (st != MM_OK) return st;
        float ms;
        MM_CUDA(time_min(s, 3, cols, &ms));
        if (ms < bc) { bc = ms; tc.col_nb = t.col_nb; tc.col_threads = t.col_threads; }
      }
    t = tc;
    for (int k = 0; k < 3; ++k) {
      t.row_threads = rts[k];
      mm_status st = apply_tune(p, t, s);
      if (st != MM_OK) return st;
      float ms;
      MM_CUDA(time_min(s, 3, rows, &ms));
      if (ms < br) { br = ms; tc.row_threads = t.row_threads; }
    }
    if (bc + br < best_total) { best_total = bc + br; best = tc; }
  }
  mm_status st = apply_tune(p, best, s);
  if (st != MM_OK) return st;
  MM_CUDA(cudaMemsetAsync(p->acc, 0, sizeof(double) * p->ncomp * acc_stride_of(p->n_pix, p->ncomp), s));
  MM_CUDA(cudaStreamSynchronize(s));
  return MM_OK;
}

extern "C" mm_status mm_apply_pointing(mm_plan p, const double* map, float* tod_out, void* stream) {
  if (p && p->composite) {
    mm_set_error("mm_apply_pointing: not available for composite-pointing plans");
    return MM_ERR_UNSUPPORTED;
  }
  MM_ARG(p != nullptr && map != nullptr && tod_out != nullptr, "NULL argument");
  if (!p->noise_set) { mm_set_error("mm_set_noise_psd has not run (pixel cut unknown)"); return MM_ERR_STATE; }
  cudaStream_t s = S(stream);
  mm_status st = load_map(p, map, s);
  if (st != MM_OK) return st;
  const unsigned nb = blocks_for(p->n_total, 256);
  if (p->ncomp == 3) k_gather<3><<<nb, 256, 0, s>>>(p->n_total, p->pix, p->cosw, p->sinw, p->wdtype == MM_W_F16, p->map4, tod_out);
  else k_gather<1><<<nb, 256, 0, s>>>(p->n_total, p->pix, p->cosw, p->sinw, p->wdtype == MM_W_F16, p->map4, tod_out);
  LAUNCHED("k_gather");
  return MM_OK;
}

extern "C" mm_status mm_apply_pointing_T(mm_plan p, const float* tod, double* acc_out, void* stream) {
  if (p && p->composite) {
    mm_set_error("mm_apply_pointing_T: not available for composite-pointing plans");
    return MM_ERR_UNSUPPORTED;
  }
  MM_ARG(p != nullptr && tod != nullptr && acc_out != nullptr, "NULL argument");
  cudaStream_t s = S(stream);
  MM_CUDA(cudaMemsetAsync(acc_out, 0, sizeof(double) * p->ncomp * p->n_pix, s));
  const unsigned nb = blocks_for(p->n_total, 256);
  if (p->ncomp == 3) k_scatter<3><<<nb, 256, 0, s>>>(p->n_total, p->pix, p->cosw, p->sinw, p->wdtype == MM_W_F16, tod, acc_out);
  else k_scatter<1><<<nb, 256, 0, s>>>(p->n_total, p->pix, p->cosw, p->sinw, p->wdtype == MM_W_F16, tod, acc_out);
  LAUNCHED("k_scatter");
  return MM_OK;
}

extern "C" mm_status mm_rfft(mm_plan p, const float* tod, float* spec_out, void* stream) {
  MM_ARG(p != nullptr && tod != nullptr && spec_out != nullptr, "NULL argument");
  MM_ARG(((uintptr_t)tod & 7) == 0 && ((uintptr_t)spec_out & 7) == 0,
         "tod and spec_out must be 8-byte aligned");
  cudaStream_t s = S(stream);
  RowArgs a{kRowNatural, 1.0, nullptr, reinterpret_cast<float2*>(spec_out)};
  FOR_BATCHES(L_(launch_col_forward(p, B, kSrcTod, tod, s)); L_(launch_row(p, B, a, s)));
  return MM_OK;
}

extern "C" mm_status mm_plan_maps(mm_plan p, int32_t* hits, uint8_t* valid, double* weight, void* stream) {
  MM_ARG(p != nullptr, "plan is NULL");
  cudaStream_t s = S(stream);
  if (hits) MM_CUDA(cudaMemcpyAsync(hits, p->hits, sizeof(int32_t) * p->n_pix, cudaMemcpyDeviceToDevice, s));
  if ((valid || weight) && !p->noise_set) {
    mm_set_error("valid / weight need mm_set_noise_psd first");
    return MM_ERR_STATE;
  }
  if (valid) MM_CUDA(cudaMemcpyAsync(valid, p->valid, p->n_pix, cudaMemcpyDeviceToDevice, s));
  if (weight) {
    if (p->ncomp == 3) k_expand_weights<3><<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, p->W, weight);
    else k_expand_weights<1><<<blocks_for(p->n_pix, 256), 256, 0, s>>>(p->n_pix, p->W, weight);
    LAUNCHED("k_expand_weights");
  }
  return MM_OK;
}
