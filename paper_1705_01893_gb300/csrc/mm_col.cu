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
  const int32_t* __restrict__ pix;
  const void* cosw;
  const void* sinw;
  int half_w;          // weights are FP16
  const void* map4;    // float4 [n_pix] (IQU) or float [n_pix] (T)
  const float* tod;
  float2* ybuf;        // batch slot: chunk ci of the batch at ybuf + ci * M
  int count;           // chunks in the batch
  double* acc;         // [n_pix][NC]
};

// Pointing streams through once per pass: evict-first loads keep the batch's intermediate
// resident in L2.
__device__ __forceinline__ float load_w(const void* w, int half_w, int64_t s) {
  if (half_w) {
    const unsigned short b = __ldcs(reinterpret_cast<const unsigned short*>(w) + s);
    return __half2float(__ushort_as_half(b));
  }
  return __ldcs(reinterpret_cast<const float*>(w) + s);
}

template <int NC>
__device__ __forceinline__ float gather_sample(const ColParams& q, int64_t s) {
  const int p = __ldcs(q.pix + s);
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

// L2 prefetch (TMA bulk prefetch, no registers or shared memory) of one tile's streamed
// input: M1 runs of 2*CB consecutive samples of the pointing (or of the source timestream).
template <int M1, int CB, int T, int NC, bool POINTING>
__device__ __forceinline__ void prefetch_tile(const ColParams& q, int64_t base, int M2) {
  for (int j1 = threadIdx.x; j1 < M1; j1 += T) {
    const int64_t s = base + 2ll * j1 * M2;
    if constexpr (POINTING) {
      prefetch_l2(q.pix + s, 8 * CB);
      if constexpr (NC == 3) {
        const int wb = q.half_w ? 2 : 4;
        prefetch_l2(static_cast<const char*>(q.cosw) + s * wb, 2 * CB * wb);
        prefetch_l2(static_cast<const char*>(q.sinw) + s * wb, 2 * CB * wb);
      }
    } else {
      prefetch_l2(q.tod + s, 8 * CB);
    }
  }
}

// Persistent over the batch's tiles (chunk ci, column block cb); each CTA prefetches its
// next tile into L2 before working on the current one, so the HBM stream of the pointing
// overlaps the FFT arithmetic.
template <int M1, int CB, int T, int NC, int SRC>
__global__ void __launch_bounds__(T) k_col_forward(ColParams q) {
  extern __shared__ float2 sm[];
  const int M2 = q.g.M2;
  const int tpc = M2 / CB;
  const int ntiles = q.count * tpc;
  constexpr int RUN = 2 * CB;
  constexpr int NS = M1 * RUN;
  float* smf = reinterpret_cast<float*>(sm);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int ci = t / tpc;
    const ChunkDesc d = q.desc[q.chunks[ci]];
    const int j2_0 = (t % tpc) * CB;
    const int64_t base = d.off + 2ll * j2_0;
    const int tn = t + gridDim.x;
    if (tn < ntiles) {
      const int64_t nb = q.desc[q.chunks[tn / tpc]].off + 2ll * (tn % tpc) * CB;
      prefetch_tile<M1, CB, T, NC, SRC == kSrcGather>(q, nb, M2);
    }
#pragma unroll 4
    for (int e = threadIdx.x; e < NS; e += T) {
      const int j1 = e / RUN, h = e % RUN;
      const int64_t s = base + 2ll * j1 * M2 + h;
      float v;
      if constexpr (SRC == kSrcTod) v = __ldcs(q.tod + s);
      else v = gather_sample<NC>(q, s);
      smf[e] = v;  // float2 slot j1*CB + h/2 = column layout element (h/2, j1)
    }
    __syncthreads();
    smem_fft<M1, CB, ColLayout<CB>, T, -1>(sm, q.g.tw_col);
    float2* y = q.ybuf + (int64_t)ci * d.M;
#pragma unroll 4
    for (int e = threadIdx.x; e < M1 * CB; e += T) {
      const int k1 = e / CB, col = e % CB;
      const int j2 = j2_0 + col;
      y[(int64_t)k1 * M2 + j2] = cmul(sm[e], tw_big(q.g, k1 * j2));
    }
    __syncthreads();
  }
}

template <int M1, int CB, int T, int NC>
__global__ void __launch_bounds__(T) k_col_inverse(ColParams q) {
  extern __shared__ float2 sm[];
  const int M2 = q.g.M2;
  const int tpc = M2 / CB;
  const int ntiles = q.count * tpc;
  constexpr int RUN = 2 * CB;
  constexpr int NS = M1 * RUN;
  static_assert(NS % 32 == 0 && T % 32 == 0, "warp-uniform scatter loop");
  const float* smf = reinterpret_cast<const float*>(sm);
  const int lane = threadIdx.x & 31;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int ci = t / tpc;
    const ChunkDesc d = q.desc[q.chunks[ci]];
    const int j2_0 = (t % tpc) * CB;
    const int tn = t + gridDim.x;
    if (tn < ntiles) {
      const int64_t nb = q.desc[q.chunks[tn / tpc]].off + 2ll * (tn % tpc) * CB;
      prefetch_tile<M1, CB, T, NC, true>(q, nb, M2);
    }
    const float2* y = q.ybuf + (int64_t)ci * d.M;
#pragma unroll 4
    for (int e = threadIdx.x; e < M1 * CB; e += T) {
      const int k1 = e / CB, col = e % CB;
      sm[e] = y[(int64_t)k1 * M2 + j2_0 + col];
    }
    __syncthreads();
    smem_fft<M1, CB, ColLayout<CB>, T, +1>(sm, q.g.tw_col);

    const int64_t base = d.off + 2ll * j2_0;
    for (int e = threadIdx.x; e < NS; e += T) {
      const int j1 = e / RUN, h = e % RUN;
      const int64_t s = base + 2ll * j1 * M2 + h;
      const float tv = smf[e];
      const int p = __ldcs(q.pix + s);
      float v0 = tv, v1 = 0.f, v2 = 0.f;
      if constexpr (NC == 3) {
        v1 = tv * load_w(q.cosw, q.half_w, s);
        v2 = tv * load_w(q.sinw, q.half_w, s);
      }
      // Runs of equal pixel among this warp's contiguous samples: the head lane of each run
      // gathers the run total by suffix doubling (as many steps as the longest run needs)
      // and issues the FP64 adds.
      const int pp = __shfl_up_sync(0xffffffffu, p, 1);
      const bool head = (lane == 0) || (h == 0) || (pp != p);
      const unsigned H = __ballot_sync(0xffffffffu, head);
      const unsigned after = H & (0xfffffffeu << lane);
      const int end = after ? (__ffs(after) - 2) : 31;
      const int maxlen =
          (int)__reduce_max_sync(0xffffffffu, head ? (unsigned)(end - lane + 1) : 0u);
      for (int dd = 1; dd < maxlen; dd <<= 1) {
        const float a0 = __shfl_down_sync(0xffffffffu, v0, dd);
        float a1 = 0.f, a2 = 0.f;
        if constexpr (NC == 3) {
          a1 = __shfl_down_sync(0xffffffffu, v1, dd);
          a2 = __shfl_down_sync(0xffffffffu, v2, dd);
        }
        if (lane + dd <= end) {
          v0 += a0;
          if constexpr (NC == 3) { v1 += a1; v2 += a2; }
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
    __syncthreads();
  }
}

// ------------------------------------------------------------------------ launchers
constexpr int kColCB = 16;
// 16 complex values per thread per FFT pass keeps registers near 64/thread.
constexpr int col_threads(int M1) {
  return M1 * kColCB / 16 < 64 ? 64 : (M1 * kColCB / 16 > 1024 ? 1024 : M1 * kColCB / 16);
}


static ColParams make_params(const mm_plan_s* p, const Batch& b, const float* tod) {
  ColParams q;
  const Group& g = p->groups[b.group];
  q.desc = p->d_desc;
  q.chunks = g.chunks + b.first;
  q.count = b.count;
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
static cudaError_t col_forward_m1(const mm_plan_s* p, const Batch& b, int src, const float* tod,
                                  cudaStream_t st) {
  constexpr int kColT = col_threads(M1);
  const ColParams q = make_params(p, b, tod);
  const int ntiles = (q.g.M2 / kColCB) * b.count;
  const size_t smem = sizeof(float2) * M1 * kColCB;
  cudaError_t e;
  int grid = 0;
  if (src == kSrcTod) {
    auto k = k_col_forward<M1, kColCB, kColT, 1, kSrcTod>;
    if ((e = persistent_grid(k, kColT, smem, ntiles, &grid)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  } else if (p->ncomp == 3) {
    auto k = k_col_forward<M1, kColCB, kColT, 3, kSrcGather>;
    if ((e = persistent_grid(k, kColT, smem, ntiles, &grid)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  } else {
    auto k = k_col_forward<M1, kColCB, kColT, 1, kSrcGather>;
    if ((e = persistent_grid(k, kColT, smem, ntiles, &grid)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  }
  return cudaGetLastError();
}

template <int M1>
static cudaError_t col_inverse_m1(const mm_plan_s* p, const Batch& b, cudaStream_t st) {
  constexpr int kColT = col_threads(M1);
  const ColParams q = make_params(p, b, nullptr);
  const int ntiles = (q.g.M2 / kColCB) * b.count;
  const size_t smem = sizeof(float2) * M1 * kColCB;
  cudaError_t e;
  int grid = 0;
  if (p->ncomp == 3) {
    auto k = k_col_inverse<M1, kColCB, kColT, 3>;
    if ((e = persistent_grid(k, kColT, smem, ntiles, &grid)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  } else {
    auto k = k_col_inverse<M1, kColCB, kColT, 1>;
    if ((e = persistent_grid(k, kColT, smem, ntiles, &grid)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  }
  return cudaGetLastError();
}

cudaError_t launch_col_forward(const mm_plan_s* p, const Batch& b, int src, const float* tod,
                               cudaStream_t st) {
  const Group& g = p->groups[b.group];
  switch (g.M1) {
    case 16: return col_forward_m1<16>(p, b, src, tod, st);
    case 32: return col_forward_m1<32>(p, b, src, tod, st);
    case 64: return col_forward_m1<64>(p, b, src, tod, st);
    case 128: return col_forward_m1<128>(p, b, src, tod, st);
    case 256: return col_forward_m1<256>(p, b, src, tod, st);
    case 512: return col_forward_m1<512>(p, b, src, tod, st);
    case 1024: return col_forward_m1<1024>(p, b, src, tod, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_col_inverse(const mm_plan_s* p, const Batch& b, cudaStream_t st) {
  const Group& g = p->groups[b.group];
  switch (g.M1) {
    case 16: return col_inverse_m1<16>(p, b, st);
    case 32: return col_inverse_m1<32>(p, b, st);
    case 64: return col_inverse_m1<64>(p, b, st);
    case 128: return col_inverse_m1<128>(p, b, st);
    case 256: return col_inverse_m1<256>(p, b, st);
    case 512: return col_inverse_m1<512>(p, b, st);
    case 1024: return col_inverse_m1<1024>(p, b, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mm
