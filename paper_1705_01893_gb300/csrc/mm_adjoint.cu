// Adjoint of K messenger iterations (gradient of a scalar loss of the final map with
// respect to the data d and to each chunk's noise parameters theta = (sigma, f_knee, alpha),
// with tau = sigma^2 and the cooling sequence held constant).
//
// One step m' = W sum_c P_c^T t_c / tau_c, t_c = irfft(a d~ + b (P m)~) (Sec. 2.1; a and b
// = 1 - a the per-mode weights of the messenger update) has, for gbar = dL/dm',
//   u = W gbar,  v_c = P_c u,
//   dL/dd_c += irfft(a v~) / tau = v/tau - irfft(b v~)/tau,
//   dL/dm   = sum_c P_c^T irfft(b v~) / tau_c,
//   dL/dtheta_c += <v/tau, dt/dtheta> + <v, P m' - t> dtau/dtheta / tau^2,
// the last term from W's dependence on tau.  The transposed step reuses the forward
// gather + column-DFT kernel for v, a row kernel that transforms it and forms the filtered
// adjoint spectrum (and the theta sums), and an inverse column kernel that bins P^T t and
// accumulates dL/dd.  Forward iterates are recomputed from checkpoints taken every
// `ckpt_every` iterations; the recomputation keeps each iteration's forward spectrum
// (P m_i)~, which the theta sums read (without a theta gradient nothing is recomputed).
#include <math.h>

#include "mm_colcommon.cuh"

namespace mm {

// Per chunk: A0 = sum w Re(conj V (R - D)) lt Nbar / den^2, Aal = same x ln(f_knee / f),
// Atau = sum w Re(conj V (D - R)) lam Nbar / den^2, AT = sum w Re(conj V T~), DOT = <v, P m'>.
enum { kAdjA0 = 0, kAdjAal = 1, kAdjAtau = 2, kAdjAT = 3, kAdjDot = 4, kAdjN = 5 };

struct AdjRowParams {
  const ChunkDesc* desc;
  const int* chunks;
  int count;
  Group g;
  float2* yV;                 // adjoint intermediate (in: column pass of v; out: of b v~)
  const float2* rspec;        // forward spectrum (P m_i)~ in row layout (theta only)
  const float2* dtab;
  const float* nbar;
  const float* nyq;
  const double* params;       // [n_chunks][4] sigma, f_knee, alpha, f_sample (or nullptr)
  double lambda;
  double* acc;                // [n_chunks][kAdjN]
};

struct Src2Rows {             // rows rA (b = 0) and rB (b = 1) of yV
  const float2* yV;
  int offA, offB;
  __device__ __forceinline__ float2 operator()(int b, int i) const {
    return yV[(b ? offB : offA) + i];
  }
};

struct DstRowsAdj {           // inverse row DFT output with the conjugate four-step twiddle
  float2* y;
  const Group* g;
  int rA, rB;
  bool self;
  __device__ __forceinline__ void operator()(int b, int i, float2 v) const {
    if (b && self) return;
    const int r = b ? rB : rA;
    y[(int64_t)r * g->M2 + i] = cmulc(v, tw_big(*g, r * i));
  }
};

// The filtered adjoint spectrum b v~ of rows rA, rB of yV; THETA: also the theta sums, with
// the forward spectrum read from rspec.
template <int M2, int T, bool THETA>
__global__ void __launch_bounds__(T, 2) k_row_adjoint(AdjRowParams q) {
  extern __shared__ float2 sm[];
  using Lay = RowLayout<M2>;
  __shared__ double red[kAdjN - 1][32];
  float2* tws = sm + 2 * M2;
  for (int i = threadIdx.x; i < tw_size(M2); i += T) tws[i] = q.g.tw_row[i];
  __syncthreads();
  const int jobs_pc = q.g.M1 / 2 + 1;
  const int njobs = q.count * jobs_pc;
  const bool lam_inf = isinf(q.lambda);
  for (int job = blockIdx.x; job < njobs; job += gridDim.x) {
    const int ci = job / jobs_pc;
    const int c = q.chunks[ci];
    const ChunkDesc d = q.desc[c];
    const int M1 = d.M1, M = d.M;
    const int rA = job % jobs_pc;
    const int rB = (M1 - rA) & (M1 - 1);
    const bool self = rA == rB;
    float2* yV = q.yV + (int64_t)ci * M;
    smem_fft<M2, 2, Lay, T, -1>(sm, tws, Src2Rows{yV, rA * M2, rB * M2});

    const float tau = (float)d.tau;
    const float lt = lam_inf ? 0.f : (float)(q.lambda * d.tau);
    const float lam = lam_inf ? 0.f : (float)q.lambda;
    const float sc = 1.0f / ((float)d.n * tau);        // irfft 1/n and T^-1
    float fk = 1.f, fs = 1.f;
    const bool has_par = THETA && q.params != nullptr;
    if (has_par) { fk = (float)q.params[4 * c + 1]; fs = (float)q.params[4 * c + 3]; }
    const float2* dt = q.dtab + d.spec;
    const float2* rs = THETA ? q.rspec + d.spec : nullptr;
    const float* nb = q.nbar + d.spec;
    const float2 wa = q.g.tw_pack_a[rA];
    float s0 = 0.f, sal = 0.f, stau = 0.f, sT = 0.f;

    // terms of one Fourier mode (index kk, multiplicity wt); returns the adjoint output b V sc
    auto mode = [&](float2 V, float2 R, float2 D, float nbv, int kk, float wt) -> float2 {
      if constexpr (!THETA) {
        if (lam_inf) return make_float2(0.f, 0.f);
        const float b = nbv / (lt + nbv);
        return make_float2(b * V.x * sc, b * V.y * sc);
      }
      float2 Tm, Y;
      if (lam_inf) {
        Tm = D;
        Y = make_float2(0.f, 0.f);
      } else {
        const float den = lt + nbv;
        const float a = lt / den, b = nbv / den;
        Tm = make_float2(a * D.x + b * R.x, a * D.y + b * R.y);
        const float c1 = V.x * (R.x - D.x) + V.y * (R.y - D.y);   // Re(conj V (R - D))
        const float g1 = lt * nbv / (den * den);
        s0 += wt * c1 * g1;
        if (has_par) {
          const float f = (kk == 0 ? 1.f : (float)kk) * fs / (float)d.n;
          sal += wt * c1 * g1 * logf(fk / f);
        }
        stau -= wt * c1 * lam * nbv / (den * den);
        Y = make_float2(b * V.x * sc, b * V.y * sc);
      }
      sT += wt * (V.x * Tm.x + V.y * Tm.y);
      return Y;
    };

    for (int p = threadIdx.x; p < M2; p += T) {
      int qs = 1, qi = M2 - 1 - p;
      if (self) {
        qs = 0;
        qi = rA == 0 ? ((M2 - p) & (M2 - 1)) : (M2 - 1 - p);
        if (p > qi) continue;
      }
      const int rowq = qs ? rB : rA;
      const int sk = rA * M2 + p, sp = rowq * M2 + qi;
      const float2 ZVk = sm[Lay::at(0, p)], ZVp = sm[Lay::at(qs, qi)];
      if (rA == 0 && p == 0) {
        // k = 0 and k = M, both real: X_0 = Re Z_0 + Im Z_0, X_M = Re Z_0 - Im Z_0
        const float2 D = THETA ? dt[0] : make_float2(0.f, 0.f);
        const float2 R0 = THETA ? rs[0] : make_float2(0.f, 0.f);   // (X_0, X_M)
        const float n0 = nb[0], nM = q.nyq[c];
        const float2 Y0 = mode(make_float2(ZVk.x + ZVk.y, 0.f), make_float2(R0.x, 0.f),
                               make_float2(D.x, 0.f), n0, 0, 1.f);
        const float2 YM = mode(make_float2(ZVk.x - ZVk.y, 0.f), make_float2(R0.y, 0.f),
                               make_float2(D.y, 0.f), nM, M, 1.f);
        sm[Lay::at(0, 0)] = make_float2(Y0.x + YM.x, Y0.x - YM.x);
        continue;
      }
      const float2 w = cmul(wa, q.g.tw_pack_b[p]);
      auto split = [&](float2 Zk, float2 Zp, float2& Xk, float2& Xp) {
        const float2 E = cscale(cadd(Zk, cconj(Zp)), 0.5f);
        const float2 O = cscale(mul_i<-1>(csub(Zk, cconj(Zp))), 0.5f);
        const float2 wO = cmul(w, O);
        Xk = cadd(E, wO);
        Xp = cconj(csub(E, wO));
      };
      float2 Vk, Vp;
      split(ZVk, ZVp, Vk, Vp);
      const bool same = (qs == 0 && qi == p);
      const float2 Rk = THETA ? rs[sk] : make_float2(0.f, 0.f);
      const float2 Rp = THETA && !same ? rs[sp] : make_float2(0.f, 0.f);
      const int k = rA + M1 * p;
      const float2 Dk = THETA ? dt[sk] : make_float2(0.f, 0.f);
      const float2 Dq = THETA && !same ? dt[sp] : make_float2(0.f, 0.f);
      const float2 Yk = mode(Vk, Rk, Dk, nb[sk], k, 2.f);
      const float2 Yp = same ? Yk : mode(Vp, Rp, Dq, nb[sp], M - k, 2.f);
      sm[Lay::at(0, p)] = cadd(cadd(Yk, cconj(Yp)), mul_i<+1>(cmulc(csub(Yk, cconj(Yp)), w)));
      if (!same)
        sm[Lay::at(qs, qi)] = csub(cadd(Yp, cconj(Yk)), mul_i<+1>(cmul(w, csub(Yp, cconj(Yk)))));
    }
    if constexpr (THETA) {
      // block sums (FP32 within a warp, FP64 across warps), one FP64 add per chunk and term
      float v4[4] = {s0, sal, stau, sT};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v4[j] += __shfl_down_sync(0xffffffffu, v4[j], o);
        if ((threadIdx.x & 31) == 0) red[j][threadIdx.x >> 5] = v4[j];
      }
      __syncthreads();
      if (threadIdx.x < 4) {
        double s = 0.0;
        for (int i = 0; i < T / 32; ++i) s += red[threadIdx.x][i];
        const int slot = threadIdx.x == 0 ? kAdjA0 : threadIdx.x == 1 ? kAdjAal
                         : threadIdx.x == 2 ? kAdjAtau : kAdjAT;
        atomicAdd(q.acc + kAdjN * c + slot, s);
      }
    } else {
      __syncthreads();
    }
    smem_fft<M2, 2, Lay, T, +1>(sm, tws, SmemIO{}, DstRowsAdj{yV, &q.g, rA, rB, self});
    __syncthreads();
  }
}

struct AdjColExtra {
  const void* mapV4;          // u = W gbar (FP32)
  const void* mapRp4;         // m' (FP32)
  float* grad_tod;            // dL/dd, original sample order
  double* acc;                // [n_chunks][kAdjN]
};

template <int NC>
__device__ __forceinline__ float4 gather4_map(const ColParams& q, const void* map4, int64_t s) {
  ColParams qq = q;
  qq.map4 = map4;
  return gather4<NC>(qq, s);
}

// Inverse column DFTs of the adjoint spectrum -> t = irfft(b v~)/tau; bin P^T t (the next
// gbar), accumulate dL/dd += v/tau - t and (THETA) <v, P m'> per chunk.
template <int M1, int CB, int T, int NC, bool THETA>
__global__ void __launch_bounds__(T, (T <= 512 ? 2 : 1)) k_col_inverse_adjoint(ColParams q,
                                                                             AdjColExtra x) {
  extern __shared__ float2 sm[];
  __shared__ double red[32];
  const int M2 = q.g.M2;
  const int tpc = M2 / CB;
  const int ntiles = q.count * tpc;
  constexpr int RUN = 2 * CB;
  constexpr int NS = M1 * RUN;
  static_assert(RUN == 32 && (NS / 4) % T == 0 && T % 32 == 0, "rows of 8 lanes");
  const float* smf = reinterpret_cast<const float*>(sm);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int ci = t / tpc;
    const int c = q.chunks[ci];
    const ChunkDesc d = q.desc[c];
    const int cb = t % tpc;
    smem_fft<M1, CB, ColLayout<CB>, T, +1>(sm, q.g.tw_col,
                                           SrcY<>{q.ybuf + (int64_t)ci * d.M, cb * CB, M2});
    const int64_t tbase = d.off + (int64_t)cb * NS;
    const float itau = (float)(1.0 / d.tau);
    float dot = 0.f;
    for (int e4 = threadIdx.x; e4 < NS / 4; e4 += T) {
      const int e = 4 * e4;
      const float4 t4 = *reinterpret_cast<const float4*>(smf + e);
      scatter4<NC>(q, tbase + e, t4, e4 & 7);
      const float4 v4 = gather4_map<NC>(q, x.mapV4, tbase + e);
      if constexpr (THETA) {
        const float4 r4 = gather4_map<NC>(q, x.mapRp4, tbase + e);
        dot += v4.x * r4.x + v4.y * r4.y + v4.z * r4.z + v4.w * r4.w;
      }
      // tile sample e -> original sample off + 2 (j1 M2 + cb CB) + (e mod 2 CB)
      const int j1 = e / RUN, wpos = e % RUN;
      float4* gt = reinterpret_cast<float4*>(x.grad_tod + d.off + 2ll * j1 * M2 + RUN * cb + wpos);
      float4 g = *gt;
      g.x += v4.x * itau - t4.x;
      g.y += v4.y * itau - t4.y;
      g.z += v4.z * itau - t4.z;
      g.w += v4.w * itau - t4.w;
      *gt = g;
    }
    if constexpr (THETA) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dot;
      __syncthreads();
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < T / 32; ++i) s += red[i];
        atomicAdd(x.acc + kAdjN * c + kAdjDot, s);
      }
    }
    __syncthreads();
  }
}

// u = W gbar (FP32 copy for the gathers), and FP32 copies of m and m'.
template <int NC>
__global__ void k_adj_prep(int64_t n_pix, const double* __restrict__ W, const double* __restrict__ g,
                           const double* __restrict__ m, const double* __restrict__ mp,
                           const uint8_t* __restrict__ valid, void* u4, void* m4, void* mp4) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  constexpr int B = NC == 3 ? 6 : 1;
  const bool ok = valid[p] != 0;
  double a[NC], u[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) a[i] = g[NC * p + i];
  const double* w = W + B * p;
  if constexpr (NC == 1) {
    u[0] = w[0] * a[0];
    reinterpret_cast<float*>(u4)[p] = (float)u[0];
    reinterpret_cast<float*>(m4)[p] = ok ? (float)m[p] : 0.f;
    reinterpret_cast<float*>(mp4)[p] = ok ? (float)mp[p] : 0.f;
  } else {
    u[0] = w[0] * a[0] + w[1] * a[1] + w[2] * a[2];
    u[1] = w[1] * a[0] + w[3] * a[1] + w[4] * a[2];
    u[2] = w[2] * a[0] + w[4] * a[1] + w[5] * a[2];
    reinterpret_cast<float4*>(u4)[p] = make_float4((float)u[0], (float)u[1], (float)u[2], 0.f);
    reinterpret_cast<float4*>(m4)[p] =
        ok ? make_float4((float)m[3 * p], (float)m[3 * p + 1], (float)m[3 * p + 2], 0.f)
           : make_float4(0.f, 0.f, 0.f, 0.f);
    reinterpret_cast<float4*>(mp4)[p] =
        ok ? make_float4((float)mp[3 * p], (float)mp[3 * p + 1], (float)mp[3 * p + 2], 0.f)
           : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// gbar for the previous step: the binned adjoint, on kept pixels; clears the accumulators.
__global__ void k_adj_take_g(int64_t len, int ncomp, double* __restrict__ acc,
                             const uint8_t* __restrict__ valid, double* __restrict__ g) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= len) return;
  const int64_t a = (i % ncomp) * acc_stride_of(len / ncomp, ncomp) + i / ncomp;   // planar
  g[i] = valid[i / ncomp] ? acc[a] : 0.0;
  acc[a] = 0.0;
}

// dL/dtheta from the per-chunk sums (tau = sigma^2, Nbar = sigma^2 (f_knee / f)^alpha).
__global__ void k_adj_theta(int n_chunks, const ChunkDesc* desc, const double* params,
                            const double* acc, double* grad_theta) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  const double sigma = params[4 * c], fk = params[4 * c + 1], alpha = params[4 * c + 2];
  const double tau = desc[c].tau, n = (double)desc[c].n;
  const double* a = acc + kAdjN * c;
  const double w_term = a[kAdjDot] - a[kAdjAT] / n;          // <v, P m' - t>
  grad_theta[3 * c + 0] = a[kAdjA0] * (2.0 / sigma) / (n * tau) +
                          a[kAdjAtau] * 2.0 * sigma / (n * tau) + w_term * 2.0 * sigma / (tau * tau);
  grad_theta[3 * c + 1] = a[kAdjA0] * (alpha / fk) / (n * tau);
  grad_theta[3 * c + 2] = a[kAdjAal] / (n * tau);
}

// ------------------------------------------------------------------------ launchers
template <int M2>
static cudaError_t row_adjoint_m2(const mm_plan_s* p, const Batch& b, float2* yV,
                                  const float2* rspec, double lambda, double* acc,
                                  cudaStream_t st) {   // rspec == NULL: no theta sums
  constexpr int T = M2 / 8 < 32 ? 32 : (M2 / 8 > 1024 ? 1024 : M2 / 8);
  const Group& g = p->groups[b.group];
  AdjRowParams q;
  q.desc = p->d_desc;
  q.chunks = g.chunks + b.first;
  q.count = b.count;
  q.g = g;
  q.yV = yV;
  q.rspec = rspec;
  q.dtab = p->dtab;
  q.nbar = p->nbar;
  q.nyq = p->nyq;
  q.params = p->theta_ok ? p->params : nullptr;
  q.lambda = lambda;
  q.acc = acc;
  const bool theta = rspec != nullptr;
  const size_t smem = sizeof(float2) * (2 * M2 + tw_size(M2));
  auto k = theta ? k_row_adjoint<M2, T, true> : k_row_adjoint<M2, T, false>;
  int grid = 0;
  cudaError_t e = persistent_grid(k, T, smem, (g.M1 / 2 + 1) * b.count, &grid);
  if (e != cudaSuccess) return e;
  k<<<grid, T, smem, st>>>(q);
  return cudaGetLastError();
}

static cudaError_t launch_row_adjoint(const mm_plan_s* p, const Batch& b, float2* yV,
                                      const float2* rspec, double lambda, double* acc,
                                      cudaStream_t st) {
  switch (p->groups[b.group].M2) {
    case 16: return row_adjoint_m2<16>(p, b, yV, rspec, lambda, acc, st);
    case 32: return row_adjoint_m2<32>(p, b, yV, rspec, lambda, acc, st);
    case 64: return row_adjoint_m2<64>(p, b, yV, rspec, lambda, acc, st);
    case 128: return row_adjoint_m2<128>(p, b, yV, rspec, lambda, acc, st);
    case 256: return row_adjoint_m2<256>(p, b, yV, rspec, lambda, acc, st);
    case 512: return row_adjoint_m2<512>(p, b, yV, rspec, lambda, acc, st);
    case 1024: return row_adjoint_m2<1024>(p, b, yV, rspec, lambda, acc, st);
    case 2048: return row_adjoint_m2<2048>(p, b, yV, rspec, lambda, acc, st);
    case 4096: return row_adjoint_m2<4096>(p, b, yV, rspec, lambda, acc, st);
  }
  return cudaErrorInvalidValue;
}

template <int M1, bool THETA>
static cudaError_t col_adjoint_m1(const mm_plan_s* p, const Batch& b, const AdjColExtra& x,
                                  cudaStream_t st) {
  constexpr int T = col_threads(M1);
  const Group& g = p->groups[b.group];
  ColParams q;
  q.desc = p->d_desc;
  q.chunks = g.chunks + b.first;
  q.count = b.count;
  q.g = g;
  q.pix = p->tpix;
  q.cosw = p->tcos;
  q.sinw = p->tsin;
  q.half_w = p->wdtype == MM_W_F16;
  q.map4 = x.mapV4;
  q.tod = nullptr;
  q.ybuf = p->ybuf;
  q.acc = p->acc;
  q.acc_stride = acc_stride_of(p->n_pix, p->ncomp);
  static_assert(col_cb(M1) == kColCB, "the adjoint takes chunks of at most 2^22 samples");
  const int ntiles = (g.M2 / kColCB) * b.count;
  const size_t smem = sizeof(float2) * M1 * kColCB;
  int grid = 0;
  cudaError_t e;
  if (p->ncomp == 3) {
    auto k = k_col_inverse_adjoint<M1, kColCB, T, 3, THETA>;
    if ((e = persistent_grid(k, T, smem, ntiles, &grid)) != cudaSuccess) return e;
    k<<<grid, T, smem, st>>>(q, x);
  } else {
    auto k = k_col_inverse_adjoint<M1, kColCB, T, 1, THETA>;
    if ((e = persistent_grid(k, T, smem, ntiles, &grid)) != cudaSuccess) return e;
    k<<<grid, T, smem, st>>>(q, x);
  }
  return cudaGetLastError();
}

template <bool THETA>
static cudaError_t col_adjoint(const mm_plan_s* p, const Batch& b, const AdjColExtra& x,
                               cudaStream_t st) {
  switch (p->groups[b.group].M1) {
    case 16: return col_adjoint_m1<16, THETA>(p, b, x, st);
    case 32: return col_adjoint_m1<32, THETA>(p, b, x, st);
    case 64: return col_adjoint_m1<64, THETA>(p, b, x, st);
    case 128: return col_adjoint_m1<128, THETA>(p, b, x, st);
    case 256: return col_adjoint_m1<256, THETA>(p, b, x, st);
    case 512: return col_adjoint_m1<512, THETA>(p, b, x, st);
  }
  return cudaErrorInvalidValue;
}

static cudaError_t launch_col_adjoint(const mm_plan_s* p, const Batch& b, const AdjColExtra& x,
                                      bool theta, cudaStream_t st) {
  return theta ? col_adjoint<true>(p, b, x, st) : col_adjoint<false>(p, b, x, st);
}

}  // namespace mm

using namespace mm;

static size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

struct AdjLayout {
  size_t ckpt, seg, g, u4, m4, mp4, keep, acc, total;
  int nseg;
};

static AdjLayout adj_layout(const mm_plan_s* p, int n_iter, int every) {
  AdjLayout L;
  const size_t map = sizeof(double) * p->ncomp * (size_t)p->n_pix;
  const size_t m4 = (p->ncomp == 3 ? 16 : 4) * (size_t)p->n_pix;
  L.nseg = (n_iter + every - 1) / every;
  size_t o = 0;
  auto take = [&](size_t b) { size_t r = o; o += up256(b); return r; };
  L.ckpt = take(map * (size_t)(L.nseg > 0 ? L.nseg : 1));
  L.seg = take(map * (size_t)(every + 1));
  L.g = take(map);
  L.u4 = take(m4);
  L.m4 = take(m4);
  L.mp4 = take(m4);
  // forward spectra (P m_i)~ of one segment's iterations, row layout, for the theta sums
  L.keep = take(sizeof(float2) * (size_t)p->spec_total * (size_t)every);
  L.acc = take(sizeof(double) * kAdjN * (size_t)p->n_chunks);
  L.total = o;
  return L;
}

extern "C" mm_status mm_adjoint_work_bytes(mm_plan p, int n_iter, int ckpt_every, size_t* bytes) {
  if (!p || !bytes || n_iter < 1 || ckpt_every < 1) {
    mm_set_error("mm_adjoint_work_bytes: bad argument");
    return MM_ERR_ARG;
  }
  if (p->n_gen > 0) {
    mm_set_error("mm_adjoint_work_bytes: chunk lengths that are not powers of two are not supported");
    return MM_ERR_UNSUPPORTED;
  }
  *bytes = adj_layout(p, n_iter, ckpt_every).total;
  return MM_OK;
}

#define ADJ_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      mm_set_error("mm_messenger_adjoint: %s: %s", #call, cudaGetErrorString(e_));         \
      return MM_ERR_CUDA;                                                                  \
    }                                                                                      \
  } while (0)

// Checks shared by the adjoint entry points.
static mm_status adjoint_check(mm_plan p, const double* lambdas, int n_iter, int ckpt_every,
                               const char* fn) {
  if (!p || !lambdas || n_iter < 1 || ckpt_every < 1) {
    mm_set_error("%s: NULL pointer or non-positive count", fn);
    return MM_ERR_ARG;
  }
  if (!p->noise_set) {
    mm_set_error("%s: mm_set_noise_psd has not run", fn);
    return MM_ERR_STATE;
  }
  if (p->n_gen > 0) {
    mm_set_error("%s: chunk lengths that are not powers of two are not supported", fn);
    return MM_ERR_UNSUPPORTED;
  }
  for (int g = 0; g < p->n_groups; ++g)
    if (p->groups[g].M2 > 4096) {
      mm_set_error("%s: chunks longer than 2^22 samples are not supported", fn);
      return MM_ERR_UNSUPPORTED;
    }
  for (int i = 0; i < n_iter; ++i)
    if (!(lambdas[i] >= 1.0 || isinf(lambdas[i]))) {
      mm_set_error("%s: lambdas[%d] must be >= 1 or inf", fn, i);
      return MM_ERR_ARG;
    }
  return MM_OK;
}

// n_iter iterations on map_inout in segments of ckpt_every, m_{kE} copied to ckpt[k] first.
static mm_status forward_ckpt(mm_plan p, const double* lambdas, int n_iter, double* map_inout,
                              int every, double* ckpt, cudaStream_t s) {
  const size_t mapb = sizeof(double) * p->ncomp * (size_t)p->n_pix;
  const size_t mstride = (size_t)p->ncomp * (size_t)p->n_pix;
  for (int i0 = 0; i0 < n_iter; i0 += every) {
    ADJ_CUDA(cudaMemcpyAsync(ckpt + (i0 / every) * mstride, map_inout, mapb,
                             cudaMemcpyDeviceToDevice, s));
    const int n = i0 + every < n_iter ? every : n_iter - i0;
    mm_status st = mm_messenger_iterate(p, lambdas + i0, n, MM_FP32_MIXED, map_inout, nullptr, s);
    if (st != MM_OK) return st;
  }
  return MM_OK;
}

// The backward sweep from the checkpoints m_0, m_E, ... (segments recomputed in `work`).
static mm_status adjoint_backward(mm_plan p, const double* lambdas, int n_iter,
                                  const double* ckpt, const double* grad_map_out,
                                  float* grad_tod, double* grad_theta, int ckpt_every,
                                  const AdjLayout& L, char* w, cudaStream_t s) {
  const size_t mapb = sizeof(double) * p->ncomp * (size_t)p->n_pix;
  double* seg = reinterpret_cast<double*>(w + L.seg);
  double* g = reinterpret_cast<double*>(w + L.g);
  void* u4 = w + L.u4;
  void* m4 = w + L.m4;
  void* mp4 = w + L.mp4;
  float2* keep = reinterpret_cast<float2*>(w + L.keep);
  const size_t kstride = (size_t)p->spec_total;
  double* acc = reinterpret_cast<double*>(w + L.acc);
  const int64_t len = p->ncomp * p->n_pix;
  const size_t mstride = (size_t)len;
  const bool theta = grad_theta != nullptr;

  ADJ_CUDA(cudaMemcpyAsync(g, grad_map_out, mapb, cudaMemcpyDeviceToDevice, s));
  ADJ_CUDA(cudaMemsetAsync(grad_tod, 0, sizeof(float) * (size_t)p->n_total, s));
  ADJ_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * kAdjN * p->n_chunks, s));
  const unsigned nbp = (unsigned)((p->n_pix + 255) / 256), nbl = (unsigned)((len + 255) / 256);
  // transposed step i (mi = m_i, mo = m_{i+1}, rs = (P m_i)~: read only for the theta terms)
  auto step = [&](int i, const double* mi, const double* mo, const float2* rs) -> mm_status {
    if (p->ncomp == 3)
      k_adj_prep<3><<<nbp, 256, 0, s>>>(p->n_pix, p->W, g, mi, mo, p->valid, u4, m4, mp4);
    else
      k_adj_prep<1><<<nbp, 256, 0, s>>>(p->n_pix, p->W, g, mi, mo, p->valid, u4, m4, mp4);
    ADJ_CUDA(cudaGetLastError());
    const AdjColExtra x{u4, mp4, grad_tod, acc};
    for (int b = 0; b < p->n_batches; ++b) {
      const Batch& B = p->h_batches[b];
      ADJ_CUDA(launch_col_forward_ex(p, B, kSrcGather, nullptr, u4, p->ybuf, s));
      ADJ_CUDA(launch_row_adjoint(p, B, p->ybuf, theta ? rs : nullptr, lambdas[i], acc, s));
      ADJ_CUDA(launch_col_adjoint(p, B, x, theta, s));
    }
    k_adj_take_g<<<nbl, 256, 0, s>>>(len, p->ncomp, p->acc, p->valid, g);
    ADJ_CUDA(cudaGetLastError());
    return MM_OK;
  };
  if (!theta) {
    // with lambda held constant the step is affine in (m, d): its transpose does not depend
    // on the iterates, so no checkpoint is read and nothing is recomputed
    for (int i = n_iter - 1; i >= 0; --i) {
      mm_status st = step(i, g, g, nullptr);
      if (st != MM_OK) return st;
    }
    return MM_OK;
  }
  for (int sg = L.nseg - 1; sg >= 0; --sg) {
    const int i0 = sg * ckpt_every;
    const int i1 = i0 + ckpt_every < n_iter ? i0 + ckpt_every : n_iter;
    ADJ_CUDA(cudaMemcpyAsync(seg, ckpt + sg * mstride, mapb, cudaMemcpyDeviceToDevice, s));
    for (int i = i0; i < i1; ++i) {
      // recompute m_{i+1} from m_i, keeping the forward spectrum (P m_i)~
      double* nxt = seg + (i - i0 + 1) * mstride;
      ADJ_CUDA(cudaMemcpyAsync(nxt, seg + (i - i0) * mstride, mapb, cudaMemcpyDeviceToDevice, s));
      mm_status st = messenger_step_keep(p, lambdas[i], nxt, keep + (i - i0) * kstride, s);
      if (st != MM_OK) return st;
    }
    for (int i = i1 - 1; i >= i0; --i) {
      mm_status st = step(i, seg + (i - i0) * mstride, seg + (i - i0 + 1) * mstride,
                          keep + (i - i0) * kstride);
      if (st != MM_OK) return st;
    }
  }
  if (theta) {
    k_adj_theta<<<(p->n_chunks + 127) / 128, 128, 0, s>>>(p->n_chunks, p->d_desc, p->params, acc,
                                                        grad_theta);
    ADJ_CUDA(cudaGetLastError());
  }
  return MM_OK;
}

static mm_status adjoint_outputs_check(mm_plan p, const double* grad_map_out,
                                       const float* grad_tod, const double* grad_theta,
                                       void* work, size_t work_bytes, const AdjLayout& L,
                                       const char* fn) {
  if (!grad_map_out || !grad_tod || !work) {
    mm_set_error("%s: NULL pointer", fn);
    return MM_ERR_ARG;
  }
  if (((uintptr_t)grad_tod & 15) != 0) {
    mm_set_error("%s: grad_tod must be 16-byte aligned", fn);
    return MM_ERR_ARG;
  }
  if (grad_theta && !p->theta_ok) {
    mm_set_error("%s: theta gradients need the parametric noise model with tau = sigma^2", fn);
    return MM_ERR_UNSUPPORTED;
  }
  if (((uintptr_t)work & 255) != 0 || work_bytes < L.total) {
    mm_set_error("%s: work must be 256-byte aligned and >= %zu bytes", fn, L.total);
    return MM_ERR_NOMEM;
  }
  return MM_OK;
}

extern "C" mm_status mm_messenger_adjoint(mm_plan p, const double* lambdas, int n_iter,
                                          const double* map_in, const double* grad_map_out,
                                          float* grad_tod, double* grad_theta, int ckpt_every,
                                          void* work, size_t work_bytes, void* stream) {
  MmRange nvtx_range_("mm_messenger_adjoint");
  const char* fn = "mm_messenger_adjoint";
  mm_status st = adjoint_check(p, lambdas, n_iter, ckpt_every, fn);
  if (st != MM_OK) return st;
  if (!map_in) {
    mm_set_error("%s: map_in is NULL", fn);
    return MM_ERR_ARG;
  }
  const AdjLayout L = adj_layout(p, n_iter, ckpt_every);
  st = adjoint_outputs_check(p, grad_map_out, grad_tod, grad_theta, work, work_bytes, L, fn);
  if (st != MM_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(work);
  double* ckpt = reinterpret_cast<double*>(w + L.ckpt);
  double* seg = reinterpret_cast<double*>(w + L.seg);
  const size_t mapb = sizeof(double) * p->ncomp * (size_t)p->n_pix;
  if (grad_theta) {
    // forward sweep (in the segment buffer), checkpoints into the work space; the data
    // gradient alone needs no forward iterate
    ADJ_CUDA(cudaMemcpyAsync(seg, map_in, mapb, cudaMemcpyDeviceToDevice, s));
    st = forward_ckpt(p, lambdas, n_iter, seg, ckpt_every, ckpt, s);
    if (st != MM_OK) return st;
  }
  return adjoint_backward(p, lambdas, n_iter, ckpt, grad_map_out, grad_tod, grad_theta,
                          ckpt_every, L, w, s);
}

extern "C" mm_status mm_messenger_forward_ckpt(mm_plan p, const double* lambdas, int n_iter,
                                               double* map_inout, int ckpt_every, double* ckpt,
                                               void* stream) {
  MmRange nvtx_range_("mm_messenger_forward_ckpt");
  const char* fn = "mm_messenger_forward_ckpt";
  mm_status st = adjoint_check(p, lambdas, n_iter, ckpt_every, fn);
  if (st != MM_OK) return st;
  if (!map_inout || !ckpt) {
    mm_set_error("%s: NULL map or checkpoint buffer", fn);
    return MM_ERR_ARG;
  }
  return forward_ckpt(p, lambdas, n_iter, map_inout, ckpt_every, ckpt,
                      reinterpret_cast<cudaStream_t>(stream));
}

extern "C" mm_status mm_messenger_adjoint_ckpt(mm_plan p, const double* lambdas, int n_iter,
                                               const double* ckpt, const double* grad_map_out,
                                               float* grad_tod, double* grad_theta,
                                               int ckpt_every, void* work, size_t work_bytes,
                                               void* stream) {
  MmRange nvtx_range_("mm_messenger_adjoint_ckpt");
  const char* fn = "mm_messenger_adjoint_ckpt";
  mm_status st = adjoint_check(p, lambdas, n_iter, ckpt_every, fn);
  if (st != MM_OK) return st;
  if (!ckpt) {
    mm_set_error("%s: ckpt is NULL", fn);
    return MM_ERR_ARG;
  }
  const AdjLayout L = adj_layout(p, n_iter, ckpt_every);
  st = adjoint_outputs_check(p, grad_map_out, grad_tod, grad_theta, work, work_bytes, L, fn);
  if (st != MM_OK) return st;
  return adjoint_backward(p, lambdas, n_iter, ckpt, grad_map_out, grad_tod, grad_theta,
                          ckpt_every, L, static_cast<char*>(work),
                          reinterpret_cast<cudaStream_t>(stream));
}
