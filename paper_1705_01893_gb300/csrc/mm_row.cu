// Row pass of the four-step FFT (kernel B): persistent over the batch's row-pair jobs; the
// job body (split, filter, chi^2, merge between the forward and inverse row DFTs) is in
// mm_rowcommon.cuh.
#include "mm_rowcommon.cuh"

namespace mm {

template <int M2, int T, int MODE>
__global__ void __launch_bounds__(T, (T <= 512 ? 2 : 1)) k_row(RowParams q) {
  extern __shared__ float2 sm[];
  using Lay = RowLayout<M2>;
  __shared__ float red[32];
  const int jobs_pc = q.g.M1 / 2 + 1;
  const int njobs = q.count * jobs_pc;
  const int mode = MODE >= 0 ? MODE : q.a.mode;
  const bool reads_d = mode == kRowMessenger || mode == kRowPcgRhs || mode == kRowChi2 ||
                       mode == kRowPcgApply || mode == kRowMd;
  // per-pass twiddles of the row DFT, staged once per CTA after the 2 rows of data
  float2* tws = sm + 2 * M2;
  for (int i = threadIdx.x; i < tw_size(M2); i += T) tws[i] = q.g.tw_row[i];
  __syncthreads();
  // Jobs are handed out by a counter: a CTA's first job is its index, the next one is taken
  // from the counter as the current one starts (measured: -7 us per launch on 8 x 2^22
  // samples against a fixed stride, whose CTAs stay in lock step through the memory and
  // the arithmetic phases of their jobs).  The last CTA to finish resets the counters.
  __shared__ int s_next;
  for (int job = blockIdx.x; job < njobs;) {
    const int ci = job / jobs_pc;
    int jn = 0;
    if (threadIdx.x == 0) {
      jn = (int)gridDim.x + (int)atomicAdd(q.queue, 1u);
      s_next = jn;
    }
    if (threadIdx.x == 0 && jn < njobs) {
      // the next job's two intermediate rows into L2 while this job runs (measured: -7 us
      // per launch on 8 x 2^22 samples; prefetching its d~ / Nbar rows as well was slower)
      const int cin = jn / jobs_pc;
      const ChunkDesc dn = q.desc[q.chunks[cin]];
      const int ra = jn % jobs_pc, rb = (dn.M1 - ra) & (dn.M1 - 1);
      const float2* yn = q.ybuf + (int64_t)cin * dn.M;
      prefetch_l2(yn + (int64_t)ra * M2, 8 * M2);
      if (rb != ra) prefetch_l2(yn + (int64_t)rb * M2, 8 * M2);
    }
    if (reads_d && threadIdx.x == 0) {
      // this job's d~ and Nbar rows into L2 while the forward row DFTs run
      const ChunkDesc dn = q.desc[q.chunks[ci]];
      const int ra = job % jobs_pc, rb = (dn.M1 - ra) & (dn.M1 - 1);
      prefetch_l2(q.dtab + dn.spec + (int64_t)ra * M2, 8 * M2);
      prefetch_l2(q.nbar + dn.spec + (int64_t)ra * M2, 4 * M2);
      if (rb != ra) {
        prefetch_l2(q.dtab + dn.spec + (int64_t)rb * M2, 8 * M2);
        prefetch_l2(q.nbar + dn.spec + (int64_t)rb * M2, 4 * M2);
      }
    }
    kernel_body_job<M2, T, MODE, true>(q, sm, tws, red, ci, job % jobs_pc);
    __syncthreads();
    job = s_next;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(q.queue + 1, 1u) == gridDim.x - 1) {
      q.queue[0] = 0u;
      q.queue[1] = 0u;
      __threadfence();
    }
  }
}

constexpr int row_threads(int M2) {
  return M2 / 8 < 32 ? 32 : (M2 / 8 > 1024 ? 1024 : M2 / 8);
}

RowParams make_row_params(const mm_plan_s* p, const Batch& b, const RowArgs& a) {
  const Group& g = p->groups[b.group];
  RowParams q;
  q.desc = p->d_desc;
  q.chunks = g.chunks + b.first;
  q.count = b.count;
  q.g = g;
  q.ybuf = p->ybuf;
  q.dtab = p->dtab;
  q.nbar = p->nbar;
  q.nyq = p->nyq;
  q.queue = p->row_queue;
  q.a = a;
  return q;
}

template <int M2>
static cudaError_t row_m2(const mm_plan_s* p, const Batch& b, const RowArgs& a,
                          cudaStream_t st) {
  constexpr int T = row_threads(M2);
  const Group& g = p->groups[b.group];
  const RowParams q = make_row_params(p, b, a);
  const size_t smem = sizeof(float2) * (2 * M2 + tw_size(M2));
  // the per-iteration modes (messenger step, its map-sized form) get their own instances
  // with the mode folded in; the set-up, PCG and chi^2 modes share one
  auto k = a.mode == kRowMessenger    ? k_row<M2, T, kRowMessenger>
           : a.mode == kRowMessengerF ? k_row<M2, T, kRowMessengerF>
                                      : k_row<M2, T, -1>;
  int grid = 0;
  cudaError_t e = persistent_grid(k, T, smem, (g.M1 / 2 + 1) * b.count, &grid);
  if (e != cudaSuccess) return e;
  k<<<grid, T, smem, st>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_row(const mm_plan_s* p, const Batch& b, const RowArgs& a, cudaStream_t st) {
  if (b.group < 0) return launch_gen_row(p, b, a, st);
  switch (p->groups[b.group].M2) {
    case 16: return row_m2<16>(p, b, a, st);
    case 32: return row_m2<32>(p, b, a, st);
    case 64: return row_m2<64>(p, b, a, st);
    case 128: return row_m2<128>(p, b, a, st);
    case 256: return row_m2<256>(p, b, a, st);
    case 512: return row_m2<512>(p, b, a, st);
    case 1024: return row_m2<1024>(p, b, a, st);
    case 2048: return row_m2<2048>(p, b, a, st);
    case 4096: return row_m2<4096>(p, b, a, st);
    case 8192: return row_m2<8192>(p, b, a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mm
