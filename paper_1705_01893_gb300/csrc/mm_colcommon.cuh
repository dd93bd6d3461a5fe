// Device code shared by the column passes of the messenger step and of its adjoint:
// kernel parameters, pointing gathers, the reduce-by-pixel binning of four samples per
// lane, and the first-pass sources / last-pass sink of the column DFTs.
#pragma once

#include "mm_internal.cuh"

namespace mm {

struct ColParams {
  const ChunkDesc* desc;
  const int* chunks;
  Group g;
  // pointing in tile order: the samples of tile (chunk, column block cb) are contiguous,
  // row j1 after row j1 - 1, 2*CB samples per row (see k_tile_pointing)
  const int32_t* __restrict__ pix;
  const void* cosw;
  const void* sinw;
  int half_w;          // weights are FP16
  const void* map4;    // float4 [n_pix] (IQU) or float [n_pix] (T)
  const float* tod;
  float2* ybuf;        // batch slot: chunk ci of the batch at ybuf + ci * M
  int count;           // chunks in the batch
  double* acc;         // planar FP64 accumulators: component k of pixel p at k * acc_stride + p
  int64_t acc_stride;  // n_pix
};

// The column kernels' parameters for batch b (plan-owned tile-order pointing, map, buffers).
ColParams make_col_params(const mm_plan_s* p, const Batch& b);

// Four consecutive samples (s a multiple of 4): one 16-byte load per stream.
__device__ __forceinline__ float4 load_w4(const void* w, int half_w, int64_t s) {
  if (half_w) {
    const uint2 b = __ldcs(reinterpret_cast<const uint2*>(static_cast<const __half*>(w) + s));
    const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&b.x));
    const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&b.y));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
  }
  return __ldcs(reinterpret_cast<const float4*>(static_cast<const float*>(w) + s));
}

template <int NC>
__device__ __forceinline__ float gather_one(const ColParams& q, int p, float cw, float sw) {
  if (p < 0) return 0.f;
  if constexpr (NC == 1) {
    return __ldg(reinterpret_cast<const float*>(q.map4) + p);
  } else {
    const float4 m = __ldg(reinterpret_cast<const float4*>(q.map4) + p);
    return fmaf(sw, m.z, fmaf(cw, m.y, m.x));
  }
}

// (P m) for samples s..s+3.
template <int NC>
__device__ __forceinline__ float4 gather4(const ColParams& q, int64_t s) {
  const int4 p = __ldcs(reinterpret_cast<const int4*>(q.pix + s));
  float4 c = make_float4(0.f, 0.f, 0.f, 0.f), w = c;
  if constexpr (NC == 3) {
    c = load_w4(q.cosw, q.half_w, s);
    w = load_w4(q.sinw, q.half_w, s);
  }
  return make_float4(gather_one<NC>(q, p.x, c.x, w.x), gather_one<NC>(q, p.y, c.y, w.y),
                     gather_one<NC>(q, p.z, c.z, w.z), gather_one<NC>(q, p.w, c.w, w.w));
}

// One FP64 add per component into the planar accumulators.  Planar, because the lanes of a
// warp close runs on neighbouring pixels: one reduction instruction then touches a third of
// the L2 sectors it would with [n_pix][3] (measured on 8 x 2^22 samples: 160 -> 141 us per
// binning launch, which is bound by L2 reduction requests).
template <int NC>
__device__ __forceinline__ void emit_run(double* acc, int64_t stride, int p, float a0, float a1,
                                         float a2, uint64_t pol) {
  if (p < 0) return;
  double* a = acc + p;
  red_add_f64(a, f32_to_f64(a0), pol);
  if constexpr (NC == 3) {
    red_add_f64(a + stride, f32_to_f64(a1), pol);
    red_add_f64(a + 2 * stride, f32_to_f64(a2), pol);
  }
}

// P^T t for samples s..s+3 (t4 = t_s..t_s+3), one lane of a row of ROWL lanes (4 ROWL
// consecutive samples; ROWL = 8, 4 or 2, a power of two dividing the warp).
// Reduce by pixel: runs inside the lane are summed in registers; runs that cross lanes are
// closed by a linear-recurrence scan over the lanes of the row (S_u = X_u + G_u S_{u+1},
// X_u = the lane's leading run when it continues the previous lane's trailing run, G_u = the
// lane is one such run and the next lane continues it).  Each run's first sample's lane
// issues one FP64 add per component.
template <int NC, int ROWL = 8>
__device__ __forceinline__ void scatter4(const ColParams& q, int64_t s, float4 t4, int qpos) {
  static_assert(ROWL == 2 || ROWL == 4 || ROWL == 8, "rows of 2, 4 or 8 lanes");
  const uint64_t pol = l2_policy_evict_last();
  const int4 p4 = __ldcs(reinterpret_cast<const int4*>(q.pix + s));
  const int p[4] = {p4.x, p4.y, p4.z, p4.w};
  const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
  float v[3][4];
  float4 c = make_float4(0.f, 0.f, 0.f, 0.f), w = c;
  if constexpr (NC == 3) {
    c = load_w4(q.cosw, q.half_w, s);
    w = load_w4(q.sinw, q.half_w, s);
  }
  const float cw[4] = {c.x, c.y, c.z, c.w}, sw[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[0][i] = tv[i];
    v[1][i] = tv[i] * cw[i];
    v[2][i] = tv[i] * sw[i];
  }
  const bool b1 = p[1] != p[0], b2 = p[2] != p[1], b3 = p[3] != p[2];
  const bool single = !(b1 || b2 || b3);
  const int f = b1 ? 1 : (b2 ? 2 : (b3 ? 3 : 4));   // leading run [0, f)
  const int l = b3 ? 3 : (b2 ? 2 : (b1 ? 1 : 0));   // trailing run [l, 4)
  float lead[3], trail[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lead[k] = 0.f;
    trail[k] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      lead[k] += i < f ? v[k][i] : 0.f;
      trail[k] += i >= l ? v[k][i] : 0.f;
    }
  }
  const int prev3 = __shfl_up_sync(0xffffffffu, p[3], 1);
  const bool cont = qpos != 0 && p[0] == prev3;
  float S[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) S[k] = cont ? lead[k] : 0.f;
  bool Gs = cont && single && qpos != ROWL - 1;
#pragma unroll
  for (int d = 1; d < ROWL; d <<= 1) {
    float Sd[3];
#pragma unroll
    for (int k = 0; k < NC; ++k) Sd[k] = __shfl_down_sync(0xffffffffu, S[k], d);
    const bool Gd = __shfl_down_sync(0xffffffffu, Gs, d);
    if (Gs) {
#pragma unroll
      for (int k = 0; k < NC; ++k) S[k] += Sd[k];
    }
    Gs = Gs && Gd;
  }
  float carry[3];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const float cd = __shfl_down_sync(0xffffffffu, S[k], 1);
    carry[k] = qpos != ROWL - 1 ? cd : 0.f;
  }
  if (!(single && cont))
    emit_run<NC>(q.acc, q.acc_stride, p[3], trail[0] + carry[0], trail[1] + carry[1], trail[2] + carry[2], pol);
  if (!cont && !single) emit_run<NC>(q.acc, q.acc_stride, p[0], lead[0], lead[1], lead[2], pol);
  if (b1 && l > 1) {   // middle run [1, e)
    const bool two = b2;
    emit_run<NC>(q.acc, q.acc_stride, p[1], two ? v[0][1] : v[0][1] + v[0][2], two ? v[1][1] : v[1][1] + v[1][2],
                 two ? v[2][1] : v[2][1] + v[2][2], pol);
  }
  if (b2 && l > 2) emit_run<NC>(q.acc, q.acc_stride, p[2], v[0][2], v[1][2], v[2][2], pol);
}

// First-pass sources and last-pass sink of the column DFTs.  Element (b, i) of a tile is
// column j2 = j2_0 + b, row j1 = i: samples s = base + 2 (i M2 + b) and s + 1.
template <int NC, int CB>
struct SrcGather {   // z = ((P m)_s, (P m)_s+1), Eq. 1; tile-ordered pointing from `tbase`
  const ColParams* q;
  int64_t tbase;
  __device__ __forceinline__ float2 operator()(int b, int i) const {
    const int64_t s = tbase + 2 * (CB * i + b);
    const int2 p = __ldcs(reinterpret_cast<const int2*>(q->pix + s));
    float cw0 = 0.f, cw1 = 0.f, sw0 = 0.f, sw1 = 0.f;
    if constexpr (NC == 3) {
      if (q->half_w) {
        const float2 c = __half22float2(__ldcs(reinterpret_cast<const __half2*>(static_cast<const __half*>(q->cosw) + s)));
        const float2 w = __half22float2(__ldcs(reinterpret_cast<const __half2*>(static_cast<const __half*>(q->sinw) + s)));
        cw0 = c.x; cw1 = c.y; sw0 = w.x; sw1 = w.y;
      } else {
        const float2 c = __ldcs(reinterpret_cast<const float2*>(static_cast<const float*>(q->cosw) + s));
        const float2 w = __ldcs(reinterpret_cast<const float2*>(static_cast<const float*>(q->sinw) + s));
        cw0 = c.x; cw1 = c.y; sw0 = w.x; sw1 = w.y;
      }
    }
    return make_float2(gather_one<NC>(*q, p.x, cw0, sw0), gather_one<NC>(*q, p.y, cw1, sw1));
  }
};

struct SrcTod {      // z = (d_s, d_s+1)
  const float* tod;
  int64_t base;
  int M2;
  __device__ __forceinline__ float2 operator()(int b, int i) const {
    return __ldcs(reinterpret_cast<const float2*>(tod + base + 2ll * ((int64_t)i * M2 + b)));
  }
};

// y[k1][j2] = Z * w_M^(k1 j2): the four-step twiddle on the way out.  kStream: the
// intermediate is written with evict-first priority (separate pass kernels, whose next
// reader comes a whole batch later), leaving L2 to the map and the accumulators.
template <bool kStream = false>
struct DstY {
  float2* y;
  const Group* g;
  int j2_0;
  int M2;
  __device__ __forceinline__ void operator()(int b, int k1, float2 v) const {
    const int j2 = j2_0 + b;
    const float2 o = cmul(v, tw_big(*g, k1 * j2));
    if constexpr (kStream) __stcs(y + (int64_t)k1 * M2 + j2, o);
    else y[(int64_t)k1 * M2 + j2] = o;
  }
};

// Filtered spectrum rows for the inverse column DFTs.  kStream: the last read of the
// intermediate (separate pass kernel), evict-first; otherwise L2 only, because in the fused
// iteration kernel other CTAs wrote these rows in this launch.
template <bool kStream = false>
struct SrcY {
  const float2* y;
  int j2_0;
  int M2;
  __device__ __forceinline__ float2 operator()(int b, int k1) const {
    if constexpr (kStream) return __ldcs(y + (int64_t)k1 * M2 + j2_0 + b);
    return __ldcg(y + (int64_t)k1 * M2 + j2_0 + b);
  }
};

}  // namespace mm
