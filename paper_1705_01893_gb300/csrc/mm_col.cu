// Column passes of the four-step FFT, fused with the pointing operators:
//   kernel A (k_col_forward): gather (P m)_s (Eq. 1) or read d_s, pack z_j = x_2j + i x_2j+1,
//            length-M1 column DFTs, twiddle w_M^{k1 j2}, write the row-layout intermediate;
//   kernel C (k_col_inverse): length-M1 inverse column DFTs of the filtered spectrum, unpack
//            t_s, and bin P^T t into FP64 per-pixel accumulators (the co-addition of t in
//            the map step of Sec. 2.1).
// Each CTA owns CB consecutive columns j2 of one chunk, i.e. runs of 2*CB consecutive
// samples at M1 places, so every global access is a contiguous run.
#include "mm_colcommon.cuh"

namespace mm {

// Persistent over the batch's tiles (chunk ci, column block cb).
template <int M1, int CB, int T, int NC, int SRC>
__global__ void __launch_bounds__(T, (T <= 512 ? 2 : 1)) k_col_forward(ColParams q) {
  extern __shared__ float2 sm[];
  const int M2 = q.g.M2;
  const int tpc = M2 / CB;
  const int ntiles = q.count * tpc;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int ci = t / tpc;
    const ChunkDesc d = q.desc[q.chunks[ci]];
    const int cb = t % tpc;
    const int j2_0 = cb * CB;
    const DstY<true> dst{q.ybuf + (int64_t)ci * d.M, &q.g, j2_0, M2};
    if constexpr (SRC == kSrcTod)
      smem_fft<M1, CB, ColLayout<CB>, T, -1>(sm, q.g.tw_col,
                                             SrcTod{q.tod, d.off + 2ll * j2_0, M2}, dst);
    else
      smem_fft<M1, CB, ColLayout<CB>, T, -1>(
          sm, q.g.tw_col, SrcGather<NC, CB>{&q, d.off + (int64_t)cb * (2 * CB * M1)}, dst);
    __syncthreads();
  }
}

template <int M1, int CB, int T, int NC>
__global__ void __launch_bounds__(T, (T <= 512 ? 2 : 1)) k_col_inverse(ColParams q) {
  extern __shared__ float2 sm[];
  const int M2 = q.g.M2;
  const int tpc = M2 / CB;
  const int ntiles = q.count * tpc;
  constexpr int RUN = 2 * CB;
  constexpr int NS = M1 * RUN;
  constexpr int ROWL = RUN / 4;   // lanes per row of the tile (4 samples per lane)
  static_assert((RUN == 32 || RUN == 16 || RUN == 8) && (NS / 4) % T == 0 && T % 32 == 0,
                "rows of 8, 4 or 2 lanes and a warp-uniform scatter loop");
  using Lay = ColLayout<CB>;
  const float* smf = reinterpret_cast<const float*>(sm);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int ci = t / tpc;
    const ChunkDesc d = q.desc[q.chunks[ci]];
    const int cb = t % tpc;
    smem_fft<M1, CB, ColLayout<CB>, T, +1>(sm, q.g.tw_col,
                                           SrcY<true>{q.ybuf + (int64_t)ci * d.M, cb * CB, M2});
    // tile-ordered pointing: the tile's samples are contiguous, in the same order as t
    const int64_t tbase = d.off + (int64_t)cb * NS;
#pragma unroll 4
    for (int e4 = threadIdx.x; e4 < NS / 4; e4 += T) {
      const int e = 4 * e4;
      // sample e = 2 (i CB + b) + h sits at float 2 Lay::at(b, i) + h; a lane's 4 samples
      // lie in one row i
      const int i = e / RUN;
      const int so = e + (Lay::kPad ? 2 * (i >> 4) * Lay::kPad : 0);
      scatter4<NC, ROWL>(q, tbase + e, *reinterpret_cast<const float4*>(smf + so), e4 & (ROWL - 1));
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------ launchers


// Copy the caller's pointing into tile order: sample 2 (j1 M2 + j2) + h of a chunk goes to
// cb (2 CB M1) + j1 (2 CB) + 2 (j2 - cb CB) + h with cb = j2 / CB (CB = col_cb(M1), the
// column kernels' tile width).  Coalesced writes.
template <int CB>
__global__ void k_tile_pointing(const int32_t* __restrict__ pix, const void* cosw, const void* sinw,
                                int wbytes, int64_t off, int M1, int M2, int32_t* __restrict__ tpix,
                                void* tcos, void* tsin) {
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= 2ll * M1 * M2) return;
  const int64_t tile = 2ll * CB * M1;
  const int cb = (int)(o / tile);
  const int r = (int)(o % tile);
  const int j1 = r / (2 * CB), w = r % (2 * CB);
  const int64_t src = off + 2ll * ((int64_t)j1 * M2 + cb * CB) + w;
  tpix[off + o] = pix[src];
  if (cosw) {
    if (wbytes == 2) {
      static_cast<__half*>(tcos)[off + o] = static_cast<const __half*>(cosw)[src];
      static_cast<__half*>(tsin)[off + o] = static_cast<const __half*>(sinw)[src];
    } else {
      static_cast<float*>(tcos)[off + o] = static_cast<const float*>(cosw)[src];
      static_cast<float*>(tsin)[off + o] = static_cast<const float*>(sinw)[src];
    }
  }
}

cudaError_t launch_tile_pointing(const mm_plan_s* p, cudaStream_t st) {
  const int wb = p->wdtype == MM_W_F16 ? 2 : 4;
  for (int c = 0; c < p->n_chunks; ++c) {
    const ChunkDesc& d = p->h_desc[c];
    if (p->groups[d.grp].general) continue;   // the general path reads the caller's order
    const int64_t n = d.n;
    if (col_cb(d.M1) == 4)
      k_tile_pointing<4><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
          p->pix, p->cosw, p->sinw, wb, d.off, d.M1, d.M2, p->tpix, p->tcos, p->tsin);
    else if (col_cb(d.M1) == 8)
      k_tile_pointing<8><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
          p->pix, p->cosw, p->sinw, wb, d.off, d.M1, d.M2, p->tpix, p->tcos, p->tsin);
    else
      k_tile_pointing<kColCB><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
          p->pix, p->cosw, p->sinw, wb, d.off, d.M1, d.M2, p->tpix, p->tcos, p->tsin);
  }
  return cudaGetLastError();
}

static ColParams make_params(const mm_plan_s* p, const Batch& b, const float* tod,
                             const void* map4 = nullptr, float2* ybuf = nullptr) {
  ColParams q;
  const Group& g = p->groups[b.group];
  q.desc = p->d_desc;
  q.chunks = g.chunks + b.first;
  q.count = b.count;
  q.g = g;
  q.pix = p->tpix;
  q.cosw = p->tcos;
  q.sinw = p->tsin;
  q.half_w = p->wdtype == MM_W_F16;
  q.map4 = map4 ? map4 : p->map4;
  q.tod = tod;
  q.ybuf = ybuf ? ybuf : p->ybuf;
  q.acc = p->acc;
  q.acc_stride = acc_stride_of(p->n_pix, p->ncomp);
  return q;
}

ColParams make_col_params(const mm_plan_s* p, const Batch& b) {
  return make_params(p, b, nullptr);
}

template <int M1>
static cudaError_t col_forward_m1(const mm_plan_s* p, const Batch& b, int src, const float* tod,
                                  const void* map4, float2* ybuf, cudaStream_t st) {
  constexpr int kColT = col_threads(M1);
  constexpr int CB = col_cb(M1);
  const ColParams q = make_params(p, b, tod, map4, ybuf);
  const int ntiles = (q.g.M2 / CB) * b.count;
  const size_t smem = sizeof(float2) * ColLayout<CB>::size(M1);
  cudaError_t e;
  int grid = 0;
  if (src == kSrcTod) {
    auto k = k_col_forward<M1, CB, kColT, 1, kSrcTod>;
    if ((e = persistent_grid(k, kColT, smem, ntiles, &grid)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  } else if (p->ncomp == 3) {
    auto k = k_col_forward<M1, CB, kColT, 3, kSrcGather>;
    if ((e = persistent_grid(k, kColT, smem, ntiles, &grid)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  } else {
    auto k = k_col_forward<M1, CB, kColT, 1, kSrcGather>;
    if ((e = persistent_grid(k, kColT, smem, ntiles, &grid)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  }
  return cudaGetLastError();
}

template <int M1>
static cudaError_t col_inverse_m1(const mm_plan_s* p, const Batch& b, cudaStream_t st) {
  constexpr int kColT = col_threads(M1);
  constexpr int CB = col_cb(M1);
  const ColParams q = make_params(p, b, nullptr);
  const int ntiles = (q.g.M2 / CB) * b.count;
  const size_t smem = sizeof(float2) * ColLayout<CB>::size(M1);
  cudaError_t e;
  int grid = 0;
  if (p->ncomp == 3) {
    auto k = k_col_inverse<M1, CB, kColT, 3>;
    if ((e = persistent_grid(k, kColT, smem, ntiles, &grid)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  } else {
    auto k = k_col_inverse<M1, CB, kColT, 1>;
    if ((e = persistent_grid(k, kColT, smem, ntiles, &grid)) != cudaSuccess) return e;
    k<<<grid, kColT, smem, st>>>(q);
  }
  return cudaGetLastError();
}

cudaError_t launch_col_forward(const mm_plan_s* p, const Batch& b, int src, const float* tod,
                               cudaStream_t st) {
  return launch_col_forward_ex(p, b, src, tod, nullptr, nullptr, st);
}

cudaError_t launch_col_forward_ex(const mm_plan_s* p, const Batch& b, int src, const float* tod,
                                  const void* map4, float2* ybuf, cudaStream_t st) {
  if (b.group < 0) {
    if (map4 || ybuf) return cudaErrorInvalidValue;
    return launch_gen_col_forward(p, b, src, tod, st);
  }
  const Group& g = p->groups[b.group];
  switch (g.M1) {
    case 16: return col_forward_m1<16>(p, b, src, tod, map4, ybuf, st);
    case 32: return col_forward_m1<32>(p, b, src, tod, map4, ybuf, st);
    case 64: return col_forward_m1<64>(p, b, src, tod, map4, ybuf, st);
    case 128: return col_forward_m1<128>(p, b, src, tod, map4, ybuf, st);
    case 256: return col_forward_m1<256>(p, b, src, tod, map4, ybuf, st);
    case 512: return col_forward_m1<512>(p, b, src, tod, map4, ybuf, st);
    case 1024: return col_forward_m1<1024>(p, b, src, tod, map4, ybuf, st);
    case 2048: return col_forward_m1<2048>(p, b, src, tod, map4, ybuf, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_col_inverse(const mm_plan_s* p, const Batch& b, cudaStream_t st) {
  if (b.group < 0) return launch_gen_col_inverse(p, b, st);
  const Group& g = p->groups[b.group];
  switch (g.M1) {
    case 16: return col_inverse_m1<16>(p, b, st);
    case 32: return col_inverse_m1<32>(p, b, st);
    case 64: return col_inverse_m1<64>(p, b, st);
    case 128: return col_inverse_m1<128>(p, b, st);
    case 256: return col_inverse_m1<256>(p, b, st);
    case 512: return col_inverse_m1<512>(p, b, st);
    case 1024: return col_inverse_m1<1024>(p, b, st);
    case 2048: return col_inverse_m1<2048>(p, b, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mm
