// Row pass of the four-step FFT with the Fourier-diagonal messenger update in the middle
// (the job body of kernel B, shared by the row kernel and the fused iteration kernel).  A
// job owns rows k1 and M1-k1 of one chunk's intermediate: after the forward row DFTs it
// holds Z_k and Z_{M-k} for all its frequencies, exactly the pairs that the real-to-complex
// split needs:
//   E_k = (Z_k + conj Z_{M-k}) / 2,  O_k = -i (Z_k - conj Z_{M-k}) / 2,
//   X_k = E_k + w_{2M}^k O_k,        X_{M-k} = conj(E_k - w_{2M}^k O_k),
// with X = rfft(x) of the chunk.  It applies the per-mode filter (Sec. 2.1 with T = tau I:
//   t~ = (lambda tau d~ + Nbar (Pm)~) / (lambda tau + Nbar)),
// accumulates chi^2 = (1/n) sum_k w_k |d~ - (Pm)~|^2 / N (Eq. 3 evaluated per Fourier mode,
// Sec. 3.1), merges the filtered Hermitian spectrum back into the packed form
//   Z'_k = (Y_k + conj Y_{M-k}) + i conj(w_{2M}^k) (Y_k - conj Y_{M-k})
// and runs the inverse row DFTs, so the spectrum never leaves the chip between the forward
// and inverse transforms.
#pragma once

#include "mm_internal.cuh"

namespace mm {

struct RowParams {
  const ChunkDesc* desc;
  const int* chunks;
  Group g;
  float2* ybuf;                  // batch slot: chunk ci of the batch at ybuf + ci * M
  int count;                     // chunks in the batch
  float2* dtab;
  const float* __restrict__ nbar;
  const float* __restrict__ nyq;
  unsigned* queue;               // [2] job counter, finished CTAs (zero between launches)
  RowArgs a;
};

// First pass of the forward row DFTs reads rows rA (b = 0) and rB (b = 1) straight from the
// intermediate; the last inverse pass writes them back with the conjugate four-step twiddle.
// kStream (separate row kernel): the rows are read and written back with evict-first
// priority, their next use being a whole batch away; otherwise (fused iteration kernel)
// they are read from L2 only, because other CTAs wrote them in this launch.
template <bool kStream = false>
struct SrcRows {
  const float2* y;
  int offA, offB;
  __device__ __forceinline__ float2 operator()(int b, int i) const {
    if constexpr (kStream) return __ldcs(y + (b ? offB : offA) + i);
    return __ldcg(y + (b ? offB : offA) + i);
  }
};

template <bool kStream = false>
struct DstRows {
  float2* y;
  const Group* g;
  int rA, rB;
  bool self;
  __device__ __forceinline__ void operator()(int b, int i, float2 v) const {
    if (b && self) return;
    const int r = b ? rB : rA;
    const float2 o = cmulc(v, tw_big(*g, r * i));
    if constexpr (kStream) __stcs(y + (int64_t)r * g->M2 + i, o);
    else y[(int64_t)r * g->M2 + i] = o;
  }
};

template <int M2, int T, int MODE, bool kStream = false>
__device__ __forceinline__ void kernel_body_job(const RowParams& q, float2* sm, const float2* tws,
                                                float* red, int ci, int rA_) {
  using Lay = RowLayout<M2>;
  const int c = q.chunks[ci];
  const ChunkDesc d = q.desc[c];
  const int M1 = d.M1, M = d.M;
  const int rA = rA_;
  const int rB = (M1 - rA) & (M1 - 1);
  const bool self = rA == rB;
  const int mode = MODE >= 0 ? MODE : q.a.mode;   // compile-time for the hot mode
  float2* y = q.ybuf + (int64_t)ci * d.M;
  const bool fwd = mode != kRowPcgRhs && mode != kRowMd;
  const bool mess = mode == kRowMessenger || mode == kRowMessengerF || mode == kRowMd ||
                    mode == kRowMessengerKeep;
  const bool inv = mess || mode == kRowPcgApply || mode == kRowPcgRhs;

  if (fwd) {
    const SrcRows<kStream> src{y, rA * M2, rB * M2};
    smem_fft<M2, 2, Lay, T, -1>(sm, tws, src);
  }

  // per-mode constants
  const float tau = (float)d.tau;
  const float inv_n = 1.0f / (float)d.n;
  double lambda = q.a.lambda;
  double* chi2 = q.a.chi2;
  if (q.a.lam_table) {          // graph mode: schedule and chi^2 slot from device memory
    const int it = *q.a.iter;
    lambda = q.a.lam_table[it];
    chi2 = q.a.chi2_base[0] ? q.a.chi2_base[0] + it : nullptr;
  }
  float lt = 0.f;               // lambda * tau
  bool lam_inf = false;
  if (mess) {
    lam_inf = isinf(lambda);
    lt = lam_inf ? 0.f : (float)(lambda * d.tau);
  }
  // N' = Nbar + cn for chi^2: tau (Eq. 3) or lambda tau (chi^2(m, lambda))
  const float cn = (mode == kRowChi2 || mode == kRowChi2Modes) ? (float)(lambda * d.tau) : tau;
  // output scale: irfft normalisation 1/n, and T^-1 = 1/tau for the messenger map step
  const float sc = mess ? inv_n / tau : inv_n;
  const float2* dt = q.dtab + d.spec;
  const float* nb = q.nbar + d.spec;
  const float2 wa = __ldg(&q.g.tw_pack_a[rA]);
  float x2 = 0.f;

  auto filt = [&](float2 X, float2 D, float nbv) -> float2 {
    if (mess) {
      if (lam_inf) return cscale(D, sc);
      const float r = __fdividef(sc, lt + nbv);
      return make_float2((lt * D.x + nbv * X.x) * r, (lt * D.y + nbv * X.y) * r);
    }
    if (mode == kRowPcgApply) return cscale(X, __fdividef(sc, nbv + tau));
    return cscale(D, __fdividef(sc, nbv + tau));  // kRowPcgRhs
  };
  const bool want_x2 = chi2 != nullptr &&
                       (mode == kRowMessenger || mode == kRowMessengerF || mode == kRowChi2 ||
                        mode == kRowChi2Modes ||
                        mode == kRowPcgRhs);
  const bool spec_out = mode == kRowSpectrum || mode == kRowNatural;
  const bool load_d = !spec_out && mode != kRowPcgApply && mode != kRowMessengerF;

  // Pairs (k, M - k): p in row rA with partner qi in row rB (or in row rA itself when the
  // row pairs with itself).  PB pairs per thread have their d~ / Nbar loads in flight at once.
  constexpr int PB = M2 >= 8192 ? 2 : 4;   // fewer in flight where the 1024-thread jobs spill
  for (int p0 = threadIdx.x; p0 < M2; p0 += PB * T) {
    float2 Dk[PB], Dp[PB];
    float nk[PB], np[PB];
    int qsv[PB], qiv[PB];
    bool act[PB];
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      const int p = p0 + u * T;
      int qs = 1, qi = M2 - 1 - p;
      bool a = p < M2;
      if (self) {
        qs = 0;
        qi = rA == 0 ? ((M2 - p) & (M2 - 1)) : (M2 - 1 - p);
        a = a && p <= qi;
      }
      act[u] = a; qsv[u] = qs; qiv[u] = qi;
      Dk[u] = Dp[u] = make_float2(0.f, 0.f);
      nk[u] = np[u] = 0.f;
      if (a && !spec_out) {
        const int sk = rA * M2 + p, sp = (qs ? rB : rA) * M2 + qi;
        if (load_d) { Dk[u] = __ldcs(dt + sk); Dp[u] = __ldcs(dt + sp); }
        nk[u] = __ldcs(nb + sk);
        np[u] = __ldcs(nb + sp);
      }
    }
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      if (!act[u]) continue;
      const int p = p0 + u * T;
      const int qs = qsv[u], qi = qiv[u];
      const int rowq = qs ? rB : rA;
      const int sk = rA * M2 + p, sp = rowq * M2 + qi;   // spectrum slots of k and M-k
      const float2 Zk = fwd ? sm[Lay::at(0, p)] : make_float2(0.f, 0.f);
      const float2 Zp = fwd ? sm[Lay::at(qs, qi)] : make_float2(0.f, 0.f);

      if (rA == 0 && p == 0) {
        // k = 0 and k = M (both real): X_0 = Re Z_0 + Im Z_0, X_M = Re Z_0 - Im Z_0;
        // slot 0 of d~ holds (d~_0, d~_M) and the Nyquist Nbar is kept per chunk
        const float X0 = Zk.x + Zk.y, XM = Zk.x - Zk.y;
        if (mode == kRowSpectrum) { q.dtab[d.spec] = make_float2(X0, XM); continue; }
        if (mode == kRowNatural) {
          float2* o = q.a.natural + d.nat;
          o[0] = make_float2(X0, 0.f);
          o[M] = make_float2(XM, 0.f);
          continue;
        }
        if (mode == kRowMessengerKeep) q.a.natural[d.spec] = make_float2(X0, XM);
        const float2 D = load_d ? dt[0] : make_float2(0.f, 0.f);
        const float n0 = nb[0], nM = __ldg(q.nyq + c);
        if (mode == kRowChi2Modes) {
          const float e0 = D.x - X0, eM = D.y - XM;
          const float v0 = __fdividef(e0 * e0, n0 + cn), vM = __fdividef(eM * eM, nM + cn);
          x2 += v0 + vM;
          double* o = reinterpret_cast<double*>(q.a.natural) + d.nat;
          o[0] = (double)(v0 * inv_n);
          o[M] = (double)(vM * inv_n);
        } else if (want_x2) {
          const float e0 = D.x - X0, eM = D.y - XM;
          x2 += __fdividef(e0 * e0, n0 + cn) + __fdividef(eM * eM, nM + cn);
        }
        if (!inv) continue;
        const float Y0 = filt(make_float2(X0, 0.f), make_float2(D.x, 0.f), n0).x;
        const float YM = filt(make_float2(XM, 0.f), make_float2(D.y, 0.f), nM).x;
        sm[Lay::at(0, 0)] = make_float2(Y0 + YM, Y0 - YM);
        continue;
      }

      const float2 w = cmul(wa, __ldg(&q.g.tw_pack_b[p]));   // w_{2M}^k, k = rA + M1 p
      const float2 E = cscale(cadd(Zk, cconj(Zp)), 0.5f);
      const float2 O = cscale(mul_i<-1>(csub(Zk, cconj(Zp))), 0.5f);
      const float2 wO = cmul(w, O);
      const float2 Xk = cadd(E, wO);
      const float2 Xp = cconj(csub(E, wO));
      const bool same = (qs == 0 && qi == p);   // k == M - k (k = M/2)
      if (mode == kRowSpectrum) {
        q.dtab[d.spec + sk] = Xk;
        if (!same) q.dtab[d.spec + sp] = Xp;
        continue;
      }
      if (mode == kRowNatural) {
        float2* o = q.a.natural + d.nat;
        const int k = rA + M1 * p;
        o[k] = Xk;
        o[M - k] = Xp;
        continue;
      }
      if (mode == kRowMessengerKeep) {
        q.a.natural[d.spec + sk] = Xk;
        if (!same) q.a.natural[d.spec + sp] = Xp;
      }
      if (mode == kRowChi2Modes) {
        // each mode's term at its natural-order slot: k = rA + M1 p, partner M - k
        const float2 ek = csub(Dk[u], Xk), ep = csub(Dp[u], Xp);
        const float tk = __fdividef(ek.x * ek.x + ek.y * ek.y, nk[u] + cn);
        const float tp = same ? 0.f : __fdividef(ep.x * ep.x + ep.y * ep.y, np[u] + cn);
        x2 += 2.f * (tk + tp);
        double* o = reinterpret_cast<double*>(q.a.natural) + d.nat;
        const int k = rA + M1 * p;
        o[k] = (double)(tk * inv_n);
        if (!same) o[M - k] = (double)(tp * inv_n);
      } else if (want_x2) {
        const float2 ek = csub(Dk[u], Xk), ep = csub(Dp[u], Xp);
        float t = __fdividef(ek.x * ek.x + ek.y * ek.y, nk[u] + cn);
        if (!same) t += __fdividef(ep.x * ep.x + ep.y * ep.y, np[u] + cn);
        x2 += 2.f * t;
      }
      if (!inv) continue;
      const float2 Yk = filt(Xk, Dk[u], nk[u]);
      const float2 Yp = filt(Xp, Dp[u], np[u]);
      // Z'_k = (Y_k + conj Y_p) + i conj(w) (Y_k - conj Y_p);
      // Z'_p = (Y_p + conj Y_k) - i w (Y_p - conj Y_k)
      const float2 zk = cadd(cadd(Yk, cconj(Yp)), mul_i<+1>(cmulc(csub(Yk, cconj(Yp)), w)));
      sm[Lay::at(0, p)] = zk;
      if (!same) {
        const float2 zp = csub(cadd(Yp, cconj(Yk)), mul_i<+1>(cmul(w, csub(Yp, cconj(Yk)))));
        sm[Lay::at(qs, qi)] = zp;
      }
    }
  }

  if (want_x2) {
    // block reduction: FP32 within warps, FP64 across warps and CTAs
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x2 += __shfl_down_sync(0xffffffffu, x2, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < T / 32; ++i) s += red[i];
      atomicAdd(chi2, s / (double)d.n);
    }
  }
  if (!inv) return;
  __syncthreads();
  smem_fft<M2, 2, Lay, T, +1>(sm, tws, SmemIO{}, DstRows<kStream>{y, &q.g, rA, rB, self});
}

// The row kernel's parameters for batch b and row mode a.
RowParams make_row_params(const mm_plan_s* p, const Batch& b, const RowArgs& a);

}  // namespace mm
