// General-length chunks: the three FFT stages of the messenger step (kernels A, B and C of
// the power-of-two path) for chunk lengths whose prime factors are 2, 3 and 5, with the
// radix sequence chosen at run time, so that chunks of many different lengths run in ONE
// persistent launch per stage.  Same four-step decomposition (M = M1 * M2, column DFTs of
// length M1, twiddle w_M^{k1 j2}, row DFTs of length M2), same row layout of the
// intermediate (slot k1 M2 + k2 holds frequency k1 + M1 k2) and the same scale
// conventions, so every mode of the row stage (messenger filter of Sec. 2.1, chi^2 of
// Eq. 3 per Fourier mode, PCG operator, spectra) is available for these chunks too.
//
// Even n: complex FFT of M = n/2 points over z_j = x_2j + i x_2j+1 with the real-to-complex
// split in the row stage (rows k1 and M1 - k1 of one chunk in one CTA).  Odd n: complex FFT
// of M = n points over z_j = x_j; every frequency is filtered on its own and the inverse
// keeps the real part.
//
// Each Stockham pass of radix R over a length-L sequence (Ns = product of the radices of
// the earlier passes) maps butterfly i, k = i mod Ns, to
//   v_r = src[i + r L/R] * w_{Ns R}^{r k},  v = DFT_R(v),  dst[(i - k) R + k + r Ns] = v_r,
// which leaves the result in natural order after the last pass.  The passes ping-pong
// between two shared-memory tiles.
#include "mm_colcommon.cuh"

namespace mm {

struct GenParams {
  const GenChunk* __restrict__ rec;     // per general chunk
  const int2* __restrict__ items;       // column tiles: (general index, first column)
  const int4* __restrict__ jobs;        // row jobs: (general index, first row, pairs or 0, -)
  int tile;                             // row tile capacity (elements, padded layout)
  int64_t base, n_items, base_y;        // the batch's items and intermediate offset
  int nb;                               // columns per tile (A, C)
  const int32_t* __restrict__ pix;      // caller's pointing, natural order
  const void* cosw;
  const void* sinw;
  // the same pointing in column-tile order (k_gen_tile_pointing): the samples of the tile
  // at first column j2_0 and width w are contiguous, row j1 after row j1 - 1
  const int32_t* __restrict__ tpix;
  const void* tcos;
  const void* tsin;
  int half_w;
  const void* map4;
  const float* tod;
  float2* ybuf;
  double* acc;
  int64_t acc_stride;   // planar accumulators: component k of pixel p at k * acc_stride + p
  float2* dtab;
  const float* __restrict__ nbar;
  const float* __restrict__ nyq;
  RowArgs a;
  // composite pointing (App. B): P = ga P_1 + gb P_2, the second component below
  int composite;
  float ga, gb;
  const int32_t* __restrict__ pix2;
  const void* cos2;
  const void* sin2;
};

// k mod d for 0 <= k < 2^22 with d uniform: float reciprocal, then one correction step
// each way (the float quotient is within one of the true one).
struct FastDiv {
  int d;
  float inv;
  __device__ __forceinline__ explicit FastDiv(int dd) : d(dd), inv(1.0f / (float)dd) {}
  __device__ __forceinline__ int mod(int k) const {
    const int q = __float2int_rz((float)k * inv);
    int r = k - q * d;
    if (r < 0) r += d;
    if (r >= d) r -= d;
    return r;
  }
  __device__ __forceinline__ int div(int k) const {
    int q = __float2int_rz((float)k * inv);
    const int r = k - q * d;
    if (r < 0) --q;
    if (r >= d) ++q;
    return q;
  }
};

// Row tiles hold nseq sequences of length L (sequence s at s L) in one of two layouts:
// plain, or padded with one spare slot per 16 elements.  Each pass writes the layout that
// suits it (padded after an even radix, whose stride-R stores would otherwise hit the same
// banks), and the next pass reads that layout.
__device__ __forceinline__ int lay(int e, bool pad) { return pad ? e + (e >> 4) : e; }

// ----------------------------------------------------------------- Stockham passes
// Column tiles: element (j, c) of the tile's NB interleaved sequences at j * NB + c.  A
// thread keeps its column c and walks butterflies i = i0, i0 + T/NB, ...; k = i mod Ns is
// advanced by the same step instead of being recomputed.
template <int R, int DIR>
__device__ __forceinline__ void gpass_cols(const float2* src, float2* dst, int L, int Ns, int NB,
                                           int lnb, const float2* __restrict__ tw, int T) {
  const int nb = L / R;
  const int c = threadIdx.x & (NB - 1);
  const int di = T >> lnb;
  int i = threadIdx.x >> lnb;
  if (i >= nb) return;
  const FastDiv fd(Ns);
  int k = fd.mod(i);
  const int dk = fd.mod(di);
  for (; i < nb; i += di) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(i + r * nb) * NB + c];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = __ldg(tw + r * Ns + k);   // this pass's table: w_{Ns R}^{r k}
        v[r] = DIR < 0 ? cmul(v[r], w) : cmulc(v[r], w);
      }
    }
    dftR<R, DIR>(v);
    const int o = (i - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(o + r * Ns) * NB + c] = v[r];
    k += dk;
    if (k >= Ns) k -= Ns;
  }
}

// Row jobs: nseq contiguous sequences of length L; PS / PD: the source / destination tile is
// in the padded layout.  Butterfly b = sq nb + i advances by T per step as (sq, i, k) with
// carries (nb is a multiple of Ns, so wrapping i keeps k = i mod Ns).
template <int R, int DIR, bool PS, bool PD>
__device__ __forceinline__ void gpass_rows(const float2* src, float2* dst, int L, int Ns, int nseq,
                                           const float2* __restrict__ tw, int T) {
  const int nb = L / R;
  const int total = nb * nseq;
  int b = threadIdx.x;
  if (b >= total) return;
  const FastDiv fs(nb), fd(Ns);
  int sq = fs.div(b);
  int i = b - sq * nb;
  int k = fd.mod(i);
  const int dsq = fs.div(T), di = T - dsq * nb, dk = fd.mod(di);
  for (; b < total; b += T) {
    const int base = sq * L;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[lay(base + i + r * nb, PS)];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = __ldg(tw + r * Ns + k);   // this pass's table: w_{Ns R}^{r k}
        v[r] = DIR < 0 ? cmul(v[r], w) : cmulc(v[r], w);
      }
    }
    dftR<R, DIR>(v);
    const int o = base + (i - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[lay(o + r * Ns, PD)] = v[r];
    i += di;
    sq += dsq;
    k += dk;
    if (k >= Ns) k -= Ns;
    if (i >= nb) { i -= nb; ++sq; }
  }
}

// All passes of the row DFTs of a job, starting from layout `pad` in tile a; returns the
// tile holding the result and sets `pad` to its layout (padded after an even radix).
template <int DIR>
__device__ float2* gen_dft_rows(float2* a, float2* b, bool& pad, int L, int nr, const int8_t* rad,
                                const float2* tw, int nseq, int T) {
  int Ns = 1;
  for (int p = 0; p < nr; ++p) {
    const int R = rad[p];
    if (pad) {
      switch (R) {
        case 2: gpass_rows<2, DIR, true, true>(a, b, L, Ns, nseq, tw, T); break;
        case 3: gpass_rows<3, DIR, true, false>(a, b, L, Ns, nseq, tw, T); break;
        case 4: gpass_rows<4, DIR, true, true>(a, b, L, Ns, nseq, tw, T); break;
        case 5: gpass_rows<5, DIR, true, false>(a, b, L, Ns, nseq, tw, T); break;
        default: gpass_rows<8, DIR, true, true>(a, b, L, Ns, nseq, tw, T); break;
      }
    } else {
      switch (R) {
        case 2: gpass_rows<2, DIR, false, true>(a, b, L, Ns, nseq, tw, T); break;
        case 3: gpass_rows<3, DIR, false, false>(a, b, L, Ns, nseq, tw, T); break;
        case 4: gpass_rows<4, DIR, false, true>(a, b, L, Ns, nseq, tw, T); break;
        case 5: gpass_rows<5, DIR, false, false>(a, b, L, Ns, nseq, tw, T); break;
        default: gpass_rows<8, DIR, false, true>(a, b, L, Ns, nseq, tw, T); break;
      }
    }
    __syncthreads();
    float2* t = a; a = b; b = t;
    pad = (R & 1) == 0;
    tw += Ns * R;   // the next pass's table
    Ns *= R;
  }
  return a;
}

// All passes of the column DFTs of a tile; returns the tile holding the result (a or b).
template <int DIR>
__device__ float2* gen_dft_cols(float2* a, float2* b, int L, int nr, const int8_t* rad,
                                const float2* tw, int NB, int lnb, int T) {
  int Ns = 1;
  for (int p = 0; p < nr; ++p) {
    const int R = rad[p];
    switch (R) {
      case 2: gpass_cols<2, DIR>(a, b, L, Ns, NB, lnb, tw, T); break;
      case 3: gpass_cols<3, DIR>(a, b, L, Ns, NB, lnb, tw, T); break;
      case 4: gpass_cols<4, DIR>(a, b, L, Ns, NB, lnb, tw, T); break;
      case 5: gpass_cols<5, DIR>(a, b, L, Ns, NB, lnb, tw, T); break;
      default: gpass_cols<8, DIR>(a, b, L, Ns, NB, lnb, tw, T); break;
    }
    __syncthreads();
    float2* t = a; a = b; b = t;
    tw += Ns * R;   // the next pass's table
    Ns *= R;
  }
  return a;
}

__device__ __forceinline__ float2 gen_tw_big(const GenChunk& g, int e) {
  return cmul(__ldg(&g.tw_hi[e >> g.log_lo]), __ldg(&g.tw_lo[e & ((1 << g.log_lo) - 1)]));
}

// One pointing component's (P m)_s (Eq. 1); weights from the caller's natural-order arrays.
template <int NC>
__device__ __forceinline__ float gen_pm1(const GenParams& q, const int32_t* __restrict__ pix,
                                         const void* cosw, const void* sinw, int64_t s) {
  const int p = __ldg(pix + s);
  if (p < 0) return 0.f;
  if constexpr (NC == 1) {
    return __ldg(reinterpret_cast<const float*>(q.map4) + p);
  } else {
    float cw, sw;
    if (q.half_w) {
      cw = __half2float(static_cast<const __half*>(cosw)[s]);
      sw = __half2float(static_cast<const __half*>(sinw)[s]);
    } else {
      cw = __ldg(static_cast<const float*>(cosw) + s);
      sw = __ldg(static_cast<const float*>(sinw) + s);
    }
    const float4 m = __ldg(reinterpret_cast<const float4*>(q.map4) + p);
    return fmaf(sw, m.z, fmaf(cw, m.y, m.x));
  }
}

// (P m)_s: one component, or g_a P_a m + g_b P_b m for a composite plan (App. B).
template <int NC>
__device__ __forceinline__ float gen_pm(const GenParams& q, int64_t s) {
  const float v = gen_pm1<NC>(q, q.pix, q.cosw, q.sinw, s);
  if (!q.composite) return v;
  return fmaf(q.gb, gen_pm1<NC>(q, q.pix2, q.cos2, q.sin2, s), q.ga * v);
}

// (P m) of a tile of one pointing component into tile a (element e = j1 NB + c holds samples
// 2 (j1 M2 + j2_0 + c) + {0, 1}, or the one sample j1 M2 + j2_0 + c of an odd-length chunk).
// U elements per thread are in flight at once: their pointing loads first, then the map
// loads that depend on them (one element at a time leaves both round trips exposed).
template <int NC>
__device__ __forceinline__ void gen_gather_tile(const GenParams& q, const ChunkDesc& d, int j2_0,
                                                int width, float2* a, int NB, int lnb, int T) {
  constexpr int U = 4;
  const int n = d.M1 * NB;
  const int nh = d.cplx ? 1 : 2;
  const int64_t tb = d.off + (int64_t)d.M1 * j2_0 * nh;   // the tile's first sample
  for (int e0 = threadIdx.x; e0 < n; e0 += U * T) {
    int pi[U][2];
    float cw[U][2], sw[U][2];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * T;
      const int j1 = e >> lnb, c = e & (NB - 1);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        pi[u][h] = -1;
        cw[u][h] = sw[u][h] = 0.f;
        if (e < n && c < width && h < nh) {
          const int64_t s = tb + ((int64_t)j1 * width + c) * nh + h;
          pi[u][h] = __ldg(q.tpix + s);
          if constexpr (NC == 3) {
            if (q.half_w) {
              cw[u][h] = __half2float(static_cast<const __half*>(q.tcos)[s]);
              sw[u][h] = __half2float(static_cast<const __half*>(q.tsin)[s]);
            } else {
              cw[u][h] = __ldg(static_cast<const float*>(q.tcos) + s);
              sw[u][h] = __ldg(static_cast<const float*>(q.tsin) + s);
            }
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * T;
      if (e >= n) continue;
      float z[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int pp = pi[u][h];
        if (pp < 0) {
          z[h] = 0.f;
        } else if constexpr (NC == 1) {
          z[h] = __ldg(reinterpret_cast<const float*>(q.map4) + pp);
        } else {
          const float4 m = __ldg(reinterpret_cast<const float4*>(q.map4) + pp);
          z[h] = fmaf(sw[u][h], m.z, fmaf(cw[u][h], m.y, m.x));
        }
      }
      a[e] = make_float2(z[0], z[1]);   // odd-length chunk: z[1] = 0 (imaginary part)
    }
  }
}

// ------------------------------------------------------------ kernel A: columns forward
template <int NC, int SRC>
__global__ void __launch_bounds__(512) k_gen_col_forward(GenParams q) {
  extern __shared__ float2 gsm[];
  const int T = blockDim.x, NB = q.nb, lnb = NB == 16 ? 4 : 3;
  for (int64_t t = blockIdx.x; t < q.n_items; t += gridDim.x) {
    const int2 it = __ldg(q.items + q.base + t);
    const GenChunk& G = q.rec[it.x];
    const ChunkDesc d = G.d;
    const int M1 = d.M1, M2 = d.M2;
    const int j2_0 = it.y;
    const int width = min(NB, M2 - j2_0);
    float2* a = gsm;
    float2* b = gsm + M1 * NB;
    if (SRC == kSrcGather && !q.composite) {
      gen_gather_tile<NC>(q, d, j2_0, width, a, NB, lnb, T);
    } else for (int e = threadIdx.x; e < M1 * NB; e += T) {
      const int j1 = e >> lnb, c = e & (NB - 1);
      float2 z = make_float2(0.f, 0.f);
      if (c < width) {
        const int64_t j = (int64_t)j1 * M2 + j2_0 + c;
        if (d.cplx) {
          z.x = SRC == kSrcTod ? __ldg(q.tod + d.off + j) : gen_pm<NC>(q, d.off + j);
        } else if constexpr (SRC == kSrcTod) {
          z = make_float2(__ldg(q.tod + d.off + 2 * j), __ldg(q.tod + d.off + 2 * j + 1));
        } else {
          z = make_float2(gen_pm<NC>(q, d.off + 2 * j), gen_pm<NC>(q, d.off + 2 * j + 1));
        }
      }
      a[e] = z;
    }
    __syncthreads();
    const float2* r = gen_dft_cols<-1>(a, b, M1, G.nr1, G.rad1, G.tw_col, NB, lnb, T);
    float2* y = q.ybuf + (G.yoff - q.base_y);
    for (int e = threadIdx.x; e < M1 * NB; e += T) {
      const int k1 = e >> lnb, c = e & (NB - 1);
      if (c < width) {
        const int j2 = j2_0 + c;
        y[(int64_t)k1 * M2 + j2] = cmul(r[e], gen_tw_big(G, k1 * j2));
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------- kernel C: columns inverse + P^T
// Warp-segmented binning: the lanes of a warp hold 32 consecutive samples of the tile (in
// sample order); runs of lanes on the same pixel are summed by a segmented suffix scan and
// the first lane of each run issues one FP64 add per component.
template <int NC>
__device__ __forceinline__ void gen_scatter(const GenParams& q, const ChunkDesc& d, int j2_0,
                                            int width, const float* smf, int NB, int lnb, int T,
                                            const int32_t* __restrict__ pix, const void* cosw,
                                            const void* sinw, float gain, bool tiled) {
  const int rw = d.cplx ? NB : 2 * NB;          // samples per tile row
  const int lrw = d.cplx ? lnb : lnb + 1;
  const int valid_u = d.cplx ? width : 2 * width;
  const int64_t tb = d.off + (int64_t)d.M1 * j2_0 * (d.cplx ? 1 : 2);   // tile order
  const int total = d.M1 * rw;
  const int lane = threadIdx.x & 31;
  // two rounds of 32 samples per warp: both rounds' pointing loads are issued before the
  // first scan
  constexpr int U = 2;
  for (int base0 = threadIdx.x - lane; base0 < total; base0 += U * T) {
    int pv[U];
    float tv[U], cv[U], sv[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int e = base0 + k * T + lane;
      pv[k] = -1;
      tv[k] = cv[k] = sv[k] = 0.f;
      if (e < total) {
        const int j1 = e >> lrw, u = e & (rw - 1);
        if (u < valid_u) {
          const int64_t s = tiled ? tb + (int64_t)j1 * valid_u + u
                                  : d.off + (d.cplx ? (int64_t)j1 * d.M2 + j2_0 + u
                                                    : 2 * ((int64_t)j1 * d.M2 + j2_0) + u);
          pv[k] = __ldg(pix + s);
          tv[k] = gain * (d.cplx ? smf[2 * e] : smf[e]);
          if constexpr (NC == 3) {
            if (q.half_w) {
              cv[k] = __half2float(static_cast<const __half*>(cosw)[s]);
              sv[k] = __half2float(static_cast<const __half*>(sinw)[s]);
            } else {
              cv[k] = __ldg(static_cast<const float*>(cosw) + s);
              sv[k] = __ldg(static_cast<const float*>(sinw) + s);
            }
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (base0 + k * T >= total) break;   // warp-uniform
      const int p = pv[k];
      float v0 = tv[k], v1 = 0.f, v2 = 0.f;
      if constexpr (NC == 3) {
        v1 = tv[k] * cv[k];
        v2 = tv[k] * sv[k];
      }
      const int pp = __shfl_up_sync(0xffffffffu, p, 1);
      const bool head = lane == 0 || p != pp;
      const unsigned hm = __ballot_sync(0xffffffffu, head);
      const int seg = __popc(hm & (0xffffffffu >> (31 - lane)));
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float a0 = __shfl_down_sync(0xffffffffu, v0, o);
        const float a1 = __shfl_down_sync(0xffffffffu, v1, o);
        const float a2 = __shfl_down_sync(0xffffffffu, v2, o);
        const int so = __shfl_down_sync(0xffffffffu, seg, o);
        if (lane + o < 32 && so == seg) { v0 += a0; v1 += a1; v2 += a2; }
      }
      if (head) emit_run<NC>(q.acc, q.acc_stride, p, v0, v1, v2, l2_policy_evict_last());
    }
  }
}

template <int NC>
__global__ void __launch_bounds__(512) k_gen_col_inverse(GenParams q) {
  extern __shared__ float2 gsm[];
  const int T = blockDim.x, NB = q.nb, lnb = NB == 16 ? 4 : 3;
  for (int64_t t = blockIdx.x; t < q.n_items; t += gridDim.x) {
    const int2 it = __ldg(q.items + q.base + t);
    const GenChunk& G = q.rec[it.x];
    const ChunkDesc d = G.d;
    const int M1 = d.M1, M2 = d.M2;
    const int j2_0 = it.y;
    const int width = min(NB, M2 - j2_0);
    float2* a = gsm;
    float2* b = gsm + M1 * NB;
    const float2* y = q.ybuf + (G.yoff - q.base_y);
    for (int e = threadIdx.x; e < M1 * NB; e += T) {
      const int k1 = e >> lnb, c = e & (NB - 1);
      a[e] = c < width ? y[(int64_t)k1 * M2 + j2_0 + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* r = gen_dft_cols<+1>(a, b, M1, G.nr1, G.rad1, G.tw_col, NB, lnb, T);
    const float* rf = reinterpret_cast<const float*>(r);
    if (!q.composite) {
      gen_scatter<NC>(q, d, j2_0, width, rf, NB, lnb, T, q.tpix, q.tcos, q.tsin, 1.f, true);
    } else {   // P^T t = g_a P_a^T t + g_b P_b^T t (App. B), natural-order pointing
      gen_scatter<NC>(q, d, j2_0, width, rf, NB, lnb, T, q.pix, q.cosw, q.sinw, q.ga, false);
      gen_scatter<NC>(q, d, j2_0, width, rf, NB, lnb, T, q.pix2, q.cos2, q.sin2, q.gb, false);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------- kernel B: rows, filter, inverse rows
// A job is either one row that pairs with itself (k1 = 0, or k1 = M1/2 for even M1) or
// `count` consecutive pairs of rows (k1, M1 - k1), k1 = first .. first + count - 1; tile
// sequence 2j holds row first + j and sequence 2j + 1 its partner.
// MODE >= 0: the row mode folded in at compile time (the messenger step and its map-sized
// form); -1: read from q.a.mode (set-up, PCG, chi^2, composite and the other modes).
template <int MODE>
__global__ void __launch_bounds__(1024) k_gen_row(GenParams q) {
  extern __shared__ float2 gsm[];
  __shared__ double red[32];
  const int T = blockDim.x;
  const int mode = MODE >= 0 ? MODE : q.a.mode;
  const bool fwd = mode != kRowPcgRhs && mode != kRowMd;
  const bool mess = mode == kRowMessenger || mode == kRowMessengerF || mode == kRowMd;
  const bool resid = mode == kRowResidual;
  const bool inv = mess || resid || mode == kRowPcgApply || mode == kRowPcgRhs;
  const bool load_d = mode != kRowSpectrum && mode != kRowNatural && mode != kRowPcgApply &&
                      mode != kRowMessengerF;
  double lambda = q.a.lambda;
  double* chi2 = q.a.chi2;
  if (q.a.lam_table) {          // graph mode: schedule and chi^2 slot from device memory
    const int it = *q.a.iter;
    lambda = q.a.lam_table[it];
    chi2 = q.a.chi2_base[0] ? q.a.chi2_base[0] + it : nullptr;
  }
  const bool want_x2 = chi2 != nullptr &&
                       (mode == kRowMessenger || mode == kRowMessengerF || mode == kRowChi2 ||
                        mode == kRowPcgRhs || mode == kRowResidual);
  for (int64_t job = blockIdx.x; job < q.n_items; job += gridDim.x) {
    const int4 it = __ldg(q.jobs + q.base + job);
    const GenChunk& G = q.rec[it.x];
    const ChunkDesc d = G.d;
    const int c = G.c;
    const int M1 = d.M1, M2 = d.M2, M = d.M;
    const bool self = it.z == 0;
    const int first = it.y, count = self ? 1 : it.z;
    const int nseq = self ? 1 : 2 * count;
    const FastDiv fm2(M2);
    auto row_of = [&](int sq) { return self ? first : ((sq & 1) ? M1 - first - (sq >> 1) : first + (sq >> 1)); };
    float2* y = q.ybuf + (G.yoff - q.base_y);
    float2* a = gsm;
    float2* b = gsm + q.tile;
    bool pz = false;
    float2* z = a;
    if (threadIdx.x == 0 && job + gridDim.x < q.n_items) {
      // the next job's rows (and its d~ / Nbar rows) into L2 while this one runs
      const int4 nj = __ldg(q.jobs + q.base + job + gridDim.x);
      const GenChunk& Gn = q.rec[nj.x];
      const int nM1 = Gn.d.M1, nM2 = Gn.d.M2;
      const int ncount = nj.z == 0 ? 1 : nj.z;
      const float2* yn = q.ybuf + (Gn.yoff - q.base_y);
      for (int s = 0; s < (nj.z == 0 ? 1 : 2 * ncount); ++s) {
        const int r = nj.z == 0 ? nj.y : ((s & 1) ? nM1 - nj.y - (s >> 1) : nj.y + (s >> 1));
        // rows of general chunks need not start on 16 bytes: prefetch their aligned interior
        if (fwd) prefetch_l2_inner(yn + (int64_t)r * nM2, 8 * (size_t)nM2);
        if (load_d) prefetch_l2_inner(q.dtab + Gn.d.spec + (int64_t)r * nM2, 8 * (size_t)nM2);
        prefetch_l2_inner(q.nbar + Gn.d.spec + (int64_t)r * nM2, 4 * (size_t)nM2);
      }
    }
    if (fwd) {
      // four elements' loads in flight per thread before their stores
      const int ne = nseq * M2;
      for (int e0 = threadIdx.x; e0 < ne; e0 += 4 * T) {
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = e0 + u * T;
          if (e < ne) {
            const int sq = fm2.div(e), p = e - sq * M2;
            v[u] = y[(int64_t)row_of(sq) * M2 + p];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (e0 + u * T < ne) a[e0 + u * T] = v[u];
      }
      __syncthreads();
      z = gen_dft_rows<-1>(a, b, pz, M2, G.nr2, G.rad2, G.tw_row, nseq, T);
    }
    float2* other = z == a ? b : a;

    const float tau = (float)d.tau;
    const float inv_n = 1.0f / (float)d.n;
    float lt = 0.f;
    bool lam_inf = false;
    if (mess || resid) {
      lam_inf = isinf(lambda);
      lt = lam_inf ? 0.f : (float)(lambda * d.tau);
    }
    const float lamf = lam_inf ? 1.f : (float)lambda;
    const float cn = mode == kRowChi2 ? (float)(lambda * d.tau) : tau;
    const float sc = mess ? inv_n / tau : inv_n;
    const float2* dt = q.dtab + d.spec;
    const float* nb = q.nbar + d.spec;
    auto filt = [&](float2 X, float2 D, float nbv) -> float2 {
      if (mess) {
        if (lam_inf) return cscale(D, sc);
        const float r = __fdividef(sc, lt + nbv);
        return make_float2((lt * D.x + nbv * X.x) * r, (lt * D.y + nbv * X.y) * r);
      }
      if (resid)   // (d~ - X) / (n (Nbar / lambda + tau)); lambda = inf: / (n tau)
        return cscale(csub(D, X), lam_inf ? __fdividef(sc, tau) : __fdividef(sc, __fdividef(nbv, lamf) + tau));
      if (mode == kRowPcgApply) return cscale(X, __fdividef(sc, nbv + tau));
      return cscale(D, __fdividef(sc, nbv + tau));  // kRowPcgRhs
    };
    float x2 = 0.f;

    if (d.cplx) {
      // every frequency on its own: k = r + M1 p for element p of row r
      for (int e = threadIdx.x; e < nseq * M2; e += T) {
        const int sq = fm2.div(e), p = e - sq * M2;
        const int r = row_of(sq);
        const int slot = r * M2 + p;
        const int k = r + M1 * p;
        const int ze = lay(e, pz);
        const float2 X = fwd ? z[ze] : make_float2(0.f, 0.f);
        if (mode == kRowSpectrum) { q.dtab[d.spec + slot] = X; continue; }
        if (mode == kRowNatural) {
          if (2 * k <= d.n) q.a.natural[d.nat + k] = X;
          continue;
        }
        const float2 D = load_d ? __ldcs(dt + slot) : make_float2(0.f, 0.f);
        const float nbv = __ldcs(nb + slot);
        if (want_x2) {
          const float2 er = csub(D, X);
          x2 += __fdividef(er.x * er.x + er.y * er.y, nbv + cn);
        }
        if (inv) z[ze] = filt(X, D, nbv);
      }
    } else {
      // pairs (k, M - k): element p of a row with its partner qi in the partner row (or in
      // the same row for a self-paired row)
      const int npair = self ? M2 : count * M2;
      for (int e = threadIdx.x; e < npair; e += T) {
        int j = 0, p = e, qi, rA, rB, sA, sB;
        if (self) {
          rA = rB = first;
          sA = sB = 0;
          qi = rA == 0 ? (p == 0 ? 0 : M2 - p) : M2 - 1 - p;
          if (p > qi) continue;
        } else {
          j = fm2.div(e);
          p = e - j * M2;
          rA = first + j;
          rB = M1 - rA;
          sA = 2 * j;
          sB = 2 * j + 1;
          qi = M2 - 1 - p;
        }
        const int sk = rA * M2 + p, sp = rB * M2 + qi;                 // spectrum slots
        const int ek = lay(sA * M2 + p, pz), ep = lay(sB * M2 + qi, pz);   // tile positions
        const float2 Zk = fwd ? z[ek] : make_float2(0.f, 0.f);
        const float2 Zp = fwd ? z[ep] : make_float2(0.f, 0.f);
        if (rA == 0 && p == 0) {
          const float X0 = Zk.x + Zk.y, XM = Zk.x - Zk.y;
          if (mode == kRowSpectrum) { q.dtab[d.spec] = make_float2(X0, XM); continue; }
          if (mode == kRowNatural) {
            q.a.natural[d.nat] = make_float2(X0, 0.f);
            q.a.natural[d.nat + M] = make_float2(XM, 0.f);
            continue;
          }
          const float2 D = load_d ? dt[0] : make_float2(0.f, 0.f);
          const float n0 = nb[0], nM = __ldg(q.nyq + c);
          if (want_x2) {
            const float e0 = D.x - X0, eM = D.y - XM;
            x2 += __fdividef(e0 * e0, n0 + cn) + __fdividef(eM * eM, nM + cn);
          }
          if (!inv) continue;
          const float Y0 = filt(make_float2(X0, 0.f), make_float2(D.x, 0.f), n0).x;
          const float YM = filt(make_float2(XM, 0.f), make_float2(D.y, 0.f), nM).x;
          z[ek] = make_float2(Y0 + YM, Y0 - YM);
          continue;
        }
        const float2 w = cmul(__ldg(&G.pack_a[rA]), __ldg(&G.pack_b[p]));   // w_{2M}^k
        const float2 E = cscale(cadd(Zk, cconj(Zp)), 0.5f);
        const float2 O = cscale(mul_i<-1>(csub(Zk, cconj(Zp))), 0.5f);
        const float2 wO = cmul(w, O);
        const float2 Xk = cadd(E, wO);
        const float2 Xp = cconj(csub(E, wO));
        const bool same = self && qi == p;                 // k == M - k
        if (mode == kRowSpectrum) {
          q.dtab[d.spec + sk] = Xk;
          if (!same) q.dtab[d.spec + sp] = Xp;
          continue;
        }
        if (mode == kRowNatural) {
          const int k = rA + M1 * p;
          q.a.natural[d.nat + k] = Xk;
          q.a.natural[d.nat + M - k] = Xp;
          continue;
        }
        const float2 Dk = load_d ? __ldcs(dt + sk) : make_float2(0.f, 0.f);
        const float2 Dp = load_d ? __ldcs(dt + sp) : make_float2(0.f, 0.f);
        const float nk = __ldcs(nb + sk), np = __ldcs(nb + sp);
        if (want_x2) {
          const float2 e1 = csub(Dk, Xk), e2 = csub(Dp, Xp);
          float tt = __fdividef(e1.x * e1.x + e1.y * e1.y, nk + cn);
          if (!same) tt += __fdividef(e2.x * e2.x + e2.y * e2.y, np + cn);
          x2 += 2.f * tt;
        }
        if (!inv) continue;
        const float2 Yk = filt(Xk, Dk, nk);
        const float2 Yp = filt(Xp, Dp, np);
        // Z'_k = (Y_k + conj Y_p) + i conj(w) (Y_k - conj Y_p)
        // Z'_p = (Y_p + conj Y_k) - i w (Y_p - conj Y_k)
        z[ek] = cadd(cadd(Yk, cconj(Yp)), mul_i<+1>(cmulc(csub(Yk, cconj(Yp)), w)));
        if (!same) z[ep] = csub(cadd(Yp, cconj(Yk)), mul_i<+1>(cmul(w, csub(Yp, cconj(Yk)))));
      }
    }
    if (want_x2) {
      // block reduction: FP32 within warps, FP64 across warps and CTAs
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x2 += __shfl_down_sync(0xffffffffu, x2, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x2;
      __syncthreads();
      if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < T / 32; ++w) sum += red[w];
        atomicAdd(chi2, sum / (double)d.n);
      }
    }
    if (inv) {
      __syncthreads();
      const float2* r = gen_dft_rows<+1>(z, other, pz, M2, G.nr2, G.rad2, G.tw_row, nseq, T);
      for (int e = threadIdx.x; e < nseq * M2; e += T) {
        const int sq = fm2.div(e), p = e - sq * M2;
        const int row = row_of(sq);
        y[(int64_t)row * M2 + p] = cmulc(r[lay(e, pz)], gen_tw_big(G, row * p));
      }
    }
    __syncthreads();
  }
}

// Copy one general chunk's pointing into column-tile order for tiles of nb columns: sample
// (j1, j2, h) (even n: s = 2 (j1 M2 + j2) + h; odd n: s = j1 M2 + j2, h = 0) goes to
// tile t = j2 / nb (first column j2_0 = t nb, width w = min(nb, M2 - j2_0)) at
// M1 j2_0 nh + (j1 w + j2 - j2_0) nh + h, nh = 2 (even) or 1 (odd): a bijection of the
// chunk's samples.
__global__ void k_gen_tile_pointing(const int32_t* __restrict__ pix, const void* cosw,
                                    const void* sinw, int wbytes, int64_t off, int n, int M1,
                                    int M2, int cplx, int nb, int32_t* __restrict__ tpix,
                                    void* tcos, void* tsin) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int nh = cplx ? 1 : 2;
  const int64_t j = cplx ? i : i >> 1;
  const int h = cplx ? 0 : (int)(i & 1);
  const int j1 = (int)(j / M2), j2 = (int)(j % M2);
  const int j2_0 = j2 - j2 % nb;
  const int w = min(nb, M2 - j2_0);
  const int64_t o = off + ((int64_t)M1 * j2_0 + (int64_t)j1 * w + (j2 - j2_0)) * nh + h;
  tpix[o] = pix[off + i];
  if (cosw) {
    if (wbytes == 2) {
      static_cast<__half*>(tcos)[o] = static_cast<const __half*>(cosw)[off + i];
      static_cast<__half*>(tsin)[o] = static_cast<const __half*>(sinw)[off + i];
    } else {
      static_cast<float*>(tcos)[o] = static_cast<const float*>(cosw)[off + i];
      static_cast<float*>(tsin)[o] = static_cast<const float*>(sinw)[off + i];
    }
  }
}

cudaError_t launch_gen_tile_pointing(const mm_plan_s* p, cudaStream_t st) {
  if (p->composite) return cudaSuccess;   // composite plans read the natural order
  const int wb = p->wdtype == MM_W_F16 ? 2 : 4;
  for (int i = 0; i < p->n_gen; ++i) {
    const ChunkDesc& d = p->h_desc[p->h_gen_chunks[i]];
    k_gen_tile_pointing<<<(unsigned)((d.n + 255) / 256), 256, 0, st>>>(
        p->pix, p->cosw, p->sinw, wb, d.off, d.n, d.M1, d.M2, d.cplx, p->gen_tune.col_nb,
        p->tpix, p->tcos, p->tsin);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------ launchers
static GenParams gen_params(const mm_plan_s* p, const Batch& b, const int2* items,
                            const int64_t* h_prefix) {
  GenParams q{};
  q.rec = p->gen_rec;
  q.items = items;
  q.base = h_prefix[b.first];
  q.n_items = h_prefix[b.first + b.count] - q.base;
  q.base_y = p->h_gen_yoff[b.first];
  q.pix = p->pix;
  q.cosw = p->cosw;
  q.sinw = p->sinw;
  q.tpix = p->tpix;
  q.tcos = p->tcos;
  q.tsin = p->tsin;
  q.half_w = p->wdtype == MM_W_F16;
  q.map4 = p->map4;
  q.ybuf = p->ybuf;
  q.acc = p->acc;
  q.acc_stride = acc_stride_of(p->n_pix, p->ncomp);
  q.dtab = p->dtab;
  q.nbar = p->nbar;
  q.nyq = p->nyq;
  q.composite = p->composite;
  q.ga = p->gain_a;
  q.gb = p->gain_b;
  q.pix2 = p->pix_b;
  q.cos2 = p->cos_b;
  q.sin2 = p->sin_b;
  return q;
}

// Largest M1 / M2 among the batch's chunks (shared-memory size of the launch).
static void gen_extent(const mm_plan_s* p, const Batch& b, int* m1, int* m2) {
  *m1 = 1; *m2 = 1;
  for (int i = b.first; i < b.first + b.count; ++i) {
    const ChunkDesc& d = p->h_desc[p->h_gen_chunks[i]];
    if (d.M1 > *m1) *m1 = d.M1;
    if (d.M2 > *m2) *m2 = d.M2;
  }
}

template <typename K>
static cudaError_t gen_launch(K kernel, int threads, size_t smem, int64_t items,
                              const GenParams& q, cudaStream_t st) {
  if (items <= 0) return cudaSuccess;
  int grid = 0;
  const int work = items > (1 << 30) ? (1 << 30) : (int)items;
  cudaError_t e = persistent_grid(kernel, threads, smem, work, &grid);
  if (e != cudaSuccess) return e;
  if (grid < 1) return cudaErrorInvalidConfiguration;
  kernel<<<grid, threads, smem, st>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_gen_col_forward(const mm_plan_s* p, const Batch& b, int src, const float* tod,
                                   cudaStream_t st) {
  GenParams q = gen_params(p, b, p->gen_ctab, p->h_gen_ctile);
  q.nb = p->gen_tune.col_nb;
  q.tod = tod;
  int m1, m2;
  gen_extent(p, b, &m1, &m2);
  const size_t smem = 2 * sizeof(float2) * (size_t)m1 * q.nb;
  const int T = p->gen_tune.col_threads;
  if (src == kSrcTod) return gen_launch(k_gen_col_forward<1, kSrcTod>, T, smem, q.n_items, q, st);
  if (p->ncomp == 3) return gen_launch(k_gen_col_forward<3, kSrcGather>, T, smem, q.n_items, q, st);
  return gen_launch(k_gen_col_forward<1, kSrcGather>, T, smem, q.n_items, q, st);
}

cudaError_t launch_gen_col_inverse(const mm_plan_s* p, const Batch& b, cudaStream_t st) {
  GenParams q = gen_params(p, b, p->gen_ctab, p->h_gen_ctile);
  q.nb = p->gen_tune.col_nb;
  int m1, m2;
  gen_extent(p, b, &m1, &m2);
  const size_t smem = 2 * sizeof(float2) * (size_t)m1 * q.nb;
  const int T = p->gen_tune.col_threads;
  if (p->ncomp == 3) return gen_launch(k_gen_col_inverse<3>, T, smem, q.n_items, q, st);
  return gen_launch(k_gen_col_inverse<1>, T, smem, q.n_items, q, st);
}

cudaError_t launch_gen_row(const mm_plan_s* p, const Batch& b, const RowArgs& a, cudaStream_t st) {
  GenParams q = gen_params(p, b, nullptr, p->h_gen_rjob);
  q.jobs = p->gen_rtab;
  q.a = a;
  // the largest job of the batch (sequences x row length), in the padded layout
  int emax = 1;
  for (int i = b.first; i < b.first + b.count; ++i) {
    const ChunkDesc& d = p->h_desc[p->h_gen_chunks[i]];
    const int e = gen_row_pairs(d.M1, d.M2) * 2 * d.M2;
    if (e > emax) emax = e;
    if (d.M2 > emax) emax = d.M2;
  }
  q.tile = emax + (emax >> 4) + 1;
  const size_t smem = 2 * sizeof(float2) * (size_t)q.tile;
  auto k = a.mode == kRowMessenger    ? k_gen_row<kRowMessenger>
           : a.mode == kRowMessengerF ? k_gen_row<kRowMessengerF>
                                      : k_gen_row<-1>;
  return gen_launch(k, p->gen_tune.row_threads, smem, q.n_items, q, st);
}

}  // namespace mm
