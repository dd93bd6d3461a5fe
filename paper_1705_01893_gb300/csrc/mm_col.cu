// Column passes of the four-step FFT, fused with the pointing operators:
//   kernel A (k_col_forward): gather (P m)_s (Eq. 1) or read d_s, pack z_j = x_2j + i x_2j+1,
//            length-M1 column DFTs, twiddle w_M^{k1 j2}, write the row-layout intermediate;
//   kernel C (k_col_inverse): length-M1 inverse column DFTs of the filtered spectrum, unpack
//            t_s, and bin P^T t into FP64 per-pixel accumulators (the co-addition of t in
//            the map step of Sec. 2.1).
// Each CTA owns CB consecutive columns j2 of one chunk, i.e. runs of 2*CB consecutive
// samples at M1 places, so every global access is a contiguous run.
#include "mm_internal.cuh"

namespace mm {

struct ColParams {
  const ChunkDesc* desc;
  const int* chunks;
  Group g;
  const int32_t* pix;
  const void* cosw;
  const void* sinw;
  int half_w;          // weights are FP16
  const void* map4;    // float4 [n_pix] (IQU) or float [n_pix] (T)
  const float* tod;
  float2* ybuf;
  double* acc;         // [n_pix][NC]
};

__device__ __forceinline__ float load_w(const void* w, int half_w, int64_t s) {
  if (half_w) return __half2float(__ldg(reinterpret_cast<const __half*>(w) + s));
  return __ldg(reinterpret_cast<const float*>(w) + s);
}

template <int NC>
__device__ __forceinline__ float gather_sample(const ColParams& q, int64_t s) {
  const int p = __ldg(q.pix + s);
  if (p < 0) return 0.f;
  if constexpr (NC == 1) {
    return __ldg(reinterpret_cast<const float*>(q.map4) + p);
  } else {
    const float cw = load_w(q.cosw, q.half_w, s);
    const float sw = load_w(q.sinw, q.half_w, s);
    const float4 m = __ldg(reinterpret_cast<const float4*>(q.map4) + p);
    return fmaf(sw, m.z, fmaf(cw, m.y, m.x));
  }
}

template <int M1, int CB, int T, int NC, int SRC>
__global__ void __launch_bounds__(T) k_col_forward(ColParams q) {
  extern __shared__ float2 sm[];
  const ChunkDesc d = q.desc[q.chunks[blockIdx.y]];
  const int M2 = d.M2;
  const int j2_0 = blockIdx.x * CB;
  const int64_t base = d.off + 2ll * j2_0;
  constexpr int RUN = 2 * CB;
  constexpr int NS = M1 * RUN;
  float* smf = reinterpret_cast<float*>(sm);
#pragma unroll 4
  for (int e = threadIdx.x; e < NS; e += T) {
    const int j1 = e / RUN, h = e % RUN;
    const int64_t s = base + 2ll * j1 * M2 + h;
    float v;
    if constexpr (SRC == kSrcTod) v = __ldg(q.tod + s);
    else v = gather_sample<NC>(q, s);
    smf[e] = v;  // float2 slot j1*CB + h/2 = column layout element (h/2, j1)
  }
  __syncthreads();
  smem_fft<M1, CB, ColLayout<CB>, T, -1>(sm, q.g.tw_col);
  float2* y = q.ybuf + d.spec;
#pragma unroll 4
  for (int e = threadIdx.x; e < M1 * CB; e += T) {
    const int k1 = e / CB, col = e % CB;
    const int j2 = j2_0 + col;
    y[(int64_t)k1 * M2 + j2] = cmul(sm[e], tw_big(q.g, k1 * j2));
  }
}

template <int M1, int CB, int T, int NC>
__global__ void __launch_bounds__(T) k_col_inverse(ColParams q) {
  extern __shared__ float2 sm[];
  const ChunkDesc d = q.desc[q.chunks[blockIdx.y]];
  const int M2 = d.M2;
  const int j2_0 = blockIdx.x * CB;
  const float2* y = q.ybuf + d.spec;
#pragma unroll 4
  for (int e = threadIdx.x; e < M1 * CB; e += T) {
    const int k1 = e / CB, col = e % CB;
    sm[e] = y[(int64_t)k1 * M2 + j2_0 + col];
  }
  __syncthreads();
  smem_fft<M1, CB, ColLayout<CB>, T, +1>(sm, q.g.tw_col);

  constexpr int RUN = 2 * CB;
  constexpr int NS = M1 * RUN;
  static_assert(NS % 32 == 0 && T % 32 == 0, "warp-uniform scatter loop");
  const int64_t base = d.off + 2ll * j2_0;
  const float* smf = reinterpret_cast<const float*>(sm);
  const int lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < NS; e += T) {
    const int j1 = e / RUN, h = e % RUN;
    const int64_t s = base + 2ll * j1 * M2 + h;
    const float t = smf[e];
    const int p = __ldg(q.pix + s);
    float v0 = t, v1 = 0.f, v2 = 0.f;
    if constexpr (NC == 3) {
      v1 = t * load_w(q.cosw, q.half_w, s);
      v2 = t * load_w(q.sinw, q.half_w, s);
    }
    // Segmented suffix sums over runs of equal pixel inside this warp's contiguous samples;
    // the first lane of each run then holds the run total and issues the FP64 adds.
    const int pn = __shfl_down_sync(0xffffffffu, p, 1);
    const int pp = __shfl_up_sync(0xffffffffu, p, 1);
    bool tail = (lane == 31) || (h == RUN - 1) || (pn != p);
    const bool head = (lane == 0) || (h == 0) || (pp != p);
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const float a0 = __shfl_down_sync(0xffffffffu, v0, dd);
      float a1 = 0.f, a2 = 0.f;
      if constexpr (NC == 3) {
        a1 = __shfl_down_sync(0xffffffffu, v1, dd);
        a2 = __shfl_down_sync(0xffffffffu, v2, dd);
      }
      const bool tf = __shfl_down_sync(0xffffffffu, tail, dd);
      if (!tail) {
        v0 += a0;
        if constexpr (NC == 3) { v1 += a1; v2 += a2; }
        tail = tf;
      }
    }
    if (head && p >= 0) {
      double* a = q.acc + (int64_t)p * NC;
      atomicAdd(a, (double)v0);
      if constexpr (NC == 3) {
        atomicAdd(a + 1, (double)v1);
        atomicAdd(a + 2, (double)v2);
      }
    }
  }
}

// ------------------------------------------------------------------------ launchers
constexpr int kColCB = 16;
// 16 complex values per thread per FFT pass keeps registers near 64/thread.
constexpr int col_threads(int M1) {
  return M1 * kColCB / 16 < 64 ? 64 : (M1 * kColCB / 16 > 1024 ? 1024 : M1 * kColCB / 16);
}

template <typename K>
static cudaError_t prep(K kernel, size_t smem) {
  // Opt in to large dynamic shared memory (idempotent).
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

static ColParams make_params(const mm_plan_s* p, const Group& g, const float* tod) {
  ColParams q;
  q.desc = p->d_desc;
  q.chunks = g.chunks;
  q.g = g;
  q.pix = p->pix;
  q.cosw = p->cosw;
  q.sinw = p->sinw;
  q.half_w = p->wdtype == MM_W_F16;
  q.map4 = p->map4;
  q.tod = tod;
  q.ybuf = p->ybuf;
  q.acc = p->acc;
  return q;
}

template <int M1>
static cudaError_t col_forward_m1(const mm_plan_s* p, const Group& g, int src, const float* tod,
                                  cudaStream_t st) {
  constexpr int kColT = col_threads(M1);
  const ColParams q = make_params(p, g, tod);
  const dim3 grid(g.M2 / kColCB, g.n_chunks);
  const size_t smem = sizeof(float2) * M1 * kColCB;
  cudaError_t e;
  if (src == kSrcTod) {
    auto k = k_col_forward<M1, kColCB, kColT, 1, kSrcTod>;
    if ((e = prep(k, smem)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  } else if (p->ncomp == 3) {
    auto k = k_col_forward<M1, kColCB, kColT, 3, kSrcGather>;
    if ((e = prep(k, smem)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  } else {
    auto k = k_col_forward<M1, kColCB, kColT, 1, kSrcGather>;
    if ((e = prep(k, smem)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  }
  return cudaGetLastError();
}

template <int M1>
static cudaError_t col_inverse_m1(const mm_plan_s* p, const Group& g, cudaStream_t st) {
  constexpr int kColT = col_threads(M1);
  const ColParams q = make_params(p, g, nullptr);
  const dim3 grid(g.M2 / kColCB, g.n_chunks);
  const size_t smem = sizeof(float2) * M1 * kColCB;
  cudaError_t e;
  if (p->ncomp == 3) {
    auto k = k_col_inverse<M1, kColCB, kColT, 3>;
    if ((e = prep(k, smem)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  } else {
    auto k = k_col_inverse<M1, kColCB, kColT, 1>;
    if ((e = prep(k, smem)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  }
  return cudaGetLastError();
}

cudaError_t launch_col_forward(const mm_plan_s* p, const Group& g, int src, const float* tod,
                               cudaStream_t st) {
  switch (g.M1) {
    case 16: return col_forward_m1<16>(p, g, src, tod, st);
    case 32: return col_forward_m1<32>(p, g, src, tod, st);
    case 64: return col_forward_m1<64>(p, g, src, tod, st);
    case 128: return col_forward_m1<128>(p, g, src, tod, st);
    case 256: return col_forward_m1<256>(p, g, src, tod, st);
    case 512: return col_forward_m1<512>(p, g, src, tod, st);
    case 1024: return col_forward_m1<1024>(p, g, src, tod, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_col_inverse(const mm_plan_s* p, const Group& g, cudaStream_t st) {
  switch (g.M1) {
    case 16: return col_inverse_m1<16>(p, g, st);
    case 32: return col_inverse_m1<32>(p, g, st);
    case 64: return col_inverse_m1<64>(p, g, st);
    case 128: return col_inverse_m1<128>(p, g, st);
    case 256: return col_inverse_m1<256>(p, g, st);
    case 512: return col_inverse_m1<512>(p, g, st);
    case 1024: return col_inverse_m1<1024>(p, g, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mm
