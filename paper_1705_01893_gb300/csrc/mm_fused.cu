// One launch for the three streaming passes of a messenger iteration over a batch of
// equal-length chunks (the column pass A, the row pass B with the Fourier-diagonal update of
// Sec. 2.1, and the inverse column pass C with the binning of P^T T^-1 t).
//
// The batch's work is a list of items -- A tiles, B row-pair jobs, C tiles -- in chunk
// order with a lag: step s holds the A tiles of chunk s, the B jobs of chunk s - 2 and the
// C tiles of chunk s - 5, interleaved.  CTAs take items from a queue counter; a B job of
// chunk c waits until all A tiles of c are done, a C tile until all B jobs of c are done
// (per-chunk counters).  The tails of three separate kernels (each ends on a partly filled
// wave of 20-30 us items) and the gaps between their launches disappear.  Every item, including a CTA's first, comes from the queue, so a CTA
// only ever waits for items that CTAs already running hold: no deadlock whatever number of
// CTAs is resident.  Waits are bounded (about a second): on expiry the kernel sets the plan's
// fault flag and carries on (the result is then wrong, and mm_plan_fault_flags reports it).
#include <vector>

#include "mm_colcommon.cuh"
#include "mm_rowcommon.cuh"

namespace mm {

struct FusedParams {
  ColParams c;            // A and C
  RowParams r;            // B
  const int2* items;      // x = kind << 16 | chunk of the batch, y = tile / job of the chunk
  int n_items;
  unsigned* ctr;          // [0] queue, [1] CTAs done, [2, 2 + count) A tiles done per chunk,
                          // [2 + count, 2 + 2 count) B jobs done per chunk; zero between launches
  int* fault;
  int n_polls;            // poll limit of each wait (the plan's wait policy)
};

enum { kItemA = 0, kItemB = 1, kItemC = 2 };

// Poll *c (acquire, GPU scope) until it reaches target, at most n_polls times (about 256 ns
// apart); on expiry set *fault and return.
__device__ __forceinline__ void wait_count(const unsigned* c, unsigned target, int* fault,
                                           int n_polls = 1 << 22) {   // about a second
  for (int n = 0; n < n_polls; ++n) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
    if (v >= target) return;
    __nanosleep(256);
  }
  atomicExch(fault, 1);
}

// MODE: the row jobs' mode, kRowMessenger (the messenger step), kRowMessengerF (its
// map-sized form, F(lambda) m) or kRowPcgApply (the PCG operator A p of the comparison
// solver).
template <int M1, int M2, int CB, int T, int NC, int MODE>
__global__ void __launch_bounds__(T, 2) k_fused(FusedParams q) {
  extern __shared__ float2 sm[];
  __shared__ float red[32];
  __shared__ int2 s_it;
  // chunks this CTA has already seen complete (A tiles, B jobs): no second acquire poll
  constexpr int kMaskWords = 64;
  __shared__ unsigned s_mask[2][kMaskWords];
  // the launch sizes the dynamic buffer for the larger of a row-pair job (2 M2 words) and a
  // column tile (ColLayout<CB>::size(M1) words)
  // The row twiddles stay in global memory (L1 / L2): staging them in shared memory, as the
  // row kernel does, would take the shared-memory reservation of every item from 64 to
  // 100 KB, and the column items lose the L1 their map gathers hit (measured: a separate
  // column pass slows from 140 to 202 us with the larger reservation).
  const float2* tws = q.r.g.tw_row;
  for (int i = threadIdx.x; i < 2 * kMaskWords; i += T) s_mask[i / kMaskWords][i % kMaskWords] = 0u;
  const int count = q.c.count;
  constexpr unsigned nA = M2 / CB, nB = M1 / 2 + 1;
  unsigned* doneA = q.ctr + 2;
  unsigned* doneB = q.ctr + 2 + count;
  if (threadIdx.x == 0) {
    const int w = (int)atomicAdd(q.ctr, 1u);
    s_it = w < q.n_items ? __ldg(q.items + w) : make_int2(-1, 0);
  }
  __syncthreads();
  while (true) {
    const int2 it = s_it;
    if (it.x < 0) break;
    const int kind = it.x >> 16, ci = it.x & 0xffff, idx = it.y;
    int2 nxt = make_int2(-1, 0);
    if (threadIdx.x == 0) {
      // the next item is taken now; its index and entry arrive while this one runs
      const int w = (int)atomicAdd(q.ctr, 1u);
      if (w < q.n_items) nxt = __ldg(q.items + w);
      if (kind != kItemA) {
        const int m = kind == kItemB ? 0 : 1;
        const bool cached = ci < 32 * kMaskWords && ((s_mask[m][ci >> 5] >> (ci & 31)) & 1u);
        if (!cached) {
          wait_count((m == 0 ? doneA : doneB) + ci, m == 0 ? nA : nB, q.fault, q.n_polls);
          if (ci < 32 * kMaskWords) s_mask[m][ci >> 5] |= 1u << (ci & 31);
        }
      }
    }
    __syncthreads();
    const ChunkDesc d = q.c.desc[q.c.chunks[ci]];
    if (kind == kItemA) {
      const DstY<> dst{q.c.ybuf + (int64_t)ci * d.M, &q.c.g, idx * CB, M2};
      smem_fft<M1, CB, ColLayout<CB>, T, -1>(
          sm, q.c.g.tw_col, SrcGather<NC, CB>{&q.c, d.off + (int64_t)idx * (2 * CB * M1)}, dst);
    } else if (kind == kItemB) {
      if (threadIdx.x == 0) {
        // this job's d~ (messenger only) and Nbar rows into L2 while the forward row DFTs run
        const int rb = (M1 - idx) & (M1 - 1);
        if (MODE == kRowMessenger) prefetch_l2(q.r.dtab + d.spec + (int64_t)idx * M2, 8 * M2);
        prefetch_l2(q.r.nbar + d.spec + (int64_t)idx * M2, 4 * M2);
        if (rb != idx) {
          if (MODE == kRowMessenger) prefetch_l2(q.r.dtab + d.spec + (int64_t)rb * M2, 8 * M2);
          prefetch_l2(q.r.nbar + d.spec + (int64_t)rb * M2, 4 * M2);
        }
      }
      kernel_body_job<M2, T, MODE>(q.r, sm, tws, red, ci, idx);
    } else {
      constexpr int RUN = 2 * CB, NS = M1 * RUN, ROWL = RUN / 4;
      using Lay = ColLayout<CB>;
      const float* smf = reinterpret_cast<const float*>(sm);
      smem_fft<M1, CB, Lay, T, +1>(sm, q.c.g.tw_col,
                                   SrcY<>{q.c.ybuf + (int64_t)ci * d.M, idx * CB, M2});
      const int64_t tbase = d.off + (int64_t)idx * NS;
#pragma unroll 2
      for (int e4 = threadIdx.x; e4 < NS / 4; e4 += T) {
        const int e = 4 * e4;
        const int so = e + (Lay::kPad ? 2 * ((e / RUN) >> 4) * Lay::kPad : 0);
        scatter4<NC, ROWL>(q.c, tbase + e, *reinterpret_cast<const float4*>(smf + so),
                           e4 & (ROWL - 1));
      }
    }
    // release the intermediate rows written by an A tile or a B job before its count: the
    // barrier orders every thread's stores before thread 0's fence, which (being cumulative)
    // orders them before the count at GPU scope (measured against a fence in every thread:
    // 4.57 -> 4.54 ms per 16 x 2^24-sample batch, 429 -> 425 us per 8 x 2^22)
    __syncthreads();
    if (threadIdx.x == 0) {
      if (kind != kItemC) __threadfence();
      if (kind == kItemA) atomicAdd(doneA + ci, 1u);
      if (kind == kItemB) atomicAdd(doneB + ci, 1u);
      s_it = nxt;
    }
    __syncthreads();
  }
  // the last CTA out clears the counters for the next launch
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(q.ctr + 1, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    for (int i = threadIdx.x; i < 2 + 2 * count; i += T) q.ctr[i] = 0u;
    __threadfence();
  }
}

// The fused path covers the shapes instantiated here, whose column tiles and row-pair jobs
// both take 512 threads and about 64 KB: rows of 4096 points with columns of 512 (chunks of
// 2^22 samples, 16-column tiles), 1024 (2^23, 8 columns) and 2048 points (2^24, 4 columns).
static bool fused_shape(int M1, int M2, bool general) {
  return !general && M2 == 4096 && (M1 == 512 || M1 == 1024 || M1 == 2048);
}

bool fused_eligible(const mm_plan_s* p, const Batch& b) {
  if (b.group < 0 || p->composite || p->h_fused_n == nullptr) return false;
  const Group& g = p->groups[b.group];
  return fused_shape(g.M1, g.M2, g.general) && p->h_fused_n[&b - p->h_batches] > 0;
}

int fused_items_per_chunk(int M1, int M2, bool general) {
  return fused_shape(M1, M2, general) ? 2 * (M2 / col_cb(M1)) + M1 / 2 + 1 : 0;
}

// Item list of a batch of `count` chunks: step s has the A tiles of chunk s, the B jobs of
// chunk s - lagAB and the C tiles of chunk s - lagAB - lagBC, taken round-robin.  Every
// item's prerequisites (all A tiles of its chunk for a B job, all B jobs for a C tile) come
// earlier in the list.  Measured on 8 x 2^22 samples (us per launch): lags 1/1 546, 1/2 490,
// 2/1 518, 2/2 449, 2/3 447, 3/3 447, 4/4 447, 8/8 (all A, then all B, then all C) 449:
// short lags leave items waiting; beyond that the order hardly matters, and the gain over
// three launches (A + B + C = 465 us) is their tails and the gaps between them.  For the
// longer chunks (1024- and 2048-point columns) the column tiles of all chunks run first
// (lagAB = count), then the row jobs and inverse tiles interleaved with lag 3: on 32 x 2^24
// samples in one batch, 8.89 ms per launch against 8.98 with the three phases one after
// the other, 8.93 with the column and row passes interleaved and the inverse tiles last,
// and (per 16-chunk batch) 4.65 against 4.57 with lags 2/3 throughout: the column and
// inverse tiles' map and accumulator accesses do better apart.  Taking the column tiles
// column block by column block across the chunks was slower still (4.75 per 16 chunks).
int fused_build_items(int M1, int M2, int count, int2* out) {
  const bool long_chunks = M1 > 512;
  const int lagAB = long_chunks ? count : 2, lagBC = 3;
  const int nA = M2 / col_cb(M1), nB = M1 / 2 + 1, nC = nA;
  int n = 0;
  for (int s = 0; s < count + lagAB + lagBC; ++s) {
    const int ca = s, cb = s - lagAB, cc = s - lagAB - lagBC;
    const bool ha = ca < count, hb = cb >= 0 && cb < count, hc = cc >= 0 && cc < count;
    const int m = (ha ? nA : 0) > (hb ? nB : 0) ? (ha ? nA : 0) : (hb ? nB : 0);
    const int mm = m > (hc ? nC : 0) ? m : (hc ? nC : 0);
    for (int i = 0; i < mm; ++i) {
      if (ha && i < nA) out[n++] = make_int2(kItemA << 16 | ca, i);
      if (hb && i < nB) out[n++] = make_int2(kItemB << 16 | cb, i);
      if (hc && i < nC) out[n++] = make_int2(kItemC << 16 | cc, i);
    }
  }
  return n;
}

template <int M1, int NC>
static void (*fused_kernel(int mode))(FusedParams) {
  constexpr int CB = col_cb(M1);
  if (mode == kRowMessenger) return k_fused<M1, 4096, CB, 512, NC, kRowMessenger>;
  if (mode == kRowMessengerF) return k_fused<M1, 4096, CB, 512, NC, kRowMessengerF>;
  if (mode == kRowPcgApply) return k_fused<M1, 4096, CB, 512, NC, kRowPcgApply>;
  return nullptr;
}

// a.mode: kRowMessenger, kRowMessengerF or kRowPcgApply.
cudaError_t launch_fused(const mm_plan_s* p, const Batch& b, const RowArgs& a, cudaStream_t st) {
  const int bi = (int)(&b - p->h_batches);
  const Group& g = p->groups[b.group];
  FusedParams q;
  q.c = make_col_params(p, b);
  q.r = make_row_params(p, b, a);
  q.items = p->fused_items + p->h_fused_first[bi];
  q.n_items = p->h_fused_n[bi];
  q.ctr = p->fused_ctr;
  q.fault = p->fault;
  q.n_polls = p->wait_polls;
  // the row jobs' two rows and the (padded) column tile share one buffer
  size_t words = 2 * (size_t)g.M2;
  void (*k)(FusedParams) = nullptr;
  const bool iqu = p->ncomp == 3;
  switch (g.M1) {
    case 512:
      k = iqu ? fused_kernel<512, 3>(a.mode) : fused_kernel<512, 1>(a.mode);
      words = words > (size_t)ColLayout<col_cb(512)>::size(512) ? words : ColLayout<col_cb(512)>::size(512);
      break;
    case 1024:
      k = iqu ? fused_kernel<1024, 3>(a.mode) : fused_kernel<1024, 1>(a.mode);
      words = words > (size_t)ColLayout<col_cb(1024)>::size(1024) ? words : ColLayout<col_cb(1024)>::size(1024);
      break;
    case 2048:
      k = iqu ? fused_kernel<2048, 3>(a.mode) : fused_kernel<2048, 1>(a.mode);
      words = words > (size_t)ColLayout<col_cb(2048)>::size(2048) ? words : ColLayout<col_cb(2048)>::size(2048);
      break;
  }
  if (k == nullptr || g.M2 != 4096) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float2) * words;
  int grid = 0;
  cudaError_t e = persistent_grid(k, 512, smem, q.n_items, &grid);
  if (e != cudaSuccess) return e;
  k<<<grid, 512, smem, st>>>(q);
  return cudaGetLastError();
}

// Check of the bounded wait above: one thread waits for a flag to reach 1; the flag is set
// beforehand (the wait returns at once) or never (the wait runs out and reports it).
static __device__ unsigned g_wait_flag;
static __device__ int g_wait_fault;

__global__ void k_wait_check(int n_polls) {
  if (threadIdx.x == 0) wait_count(&g_wait_flag, 1u, &g_wait_fault, n_polls);
}

}  // namespace mm

extern "C" mm_status mm_fused_item_list(int m1, int m2, int count, int* out, int capacity,
                                        int* n_items) {
  using namespace mm;
  if (!n_items || count < 1 || count > 0xffff || m1 < 2 || m1 > 8192 || (m1 & (m1 - 1)) != 0 ||
      m2 < col_cb(m1) || (m2 % col_cb(m1)) != 0) {
    mm_set_error("mm_fused_item_list: bad argument");
    return MM_ERR_ARG;
  }
  const int per = 2 * (m2 / col_cb(m1)) + m1 / 2 + 1;
  const int64_t total = (int64_t)per * count;
  *n_items = (int)total;
  if (!out) return MM_OK;
  if (capacity < total) {
    mm_set_error("mm_fused_item_list: capacity %d < %lld items", capacity, (long long)total);
    return MM_ERR_ARG;
  }
  std::vector<int2> v((size_t)total);
  const int n = fused_build_items(m1, m2, count, v.data());
  for (int i = 0; i < n; ++i) {
    out[3 * i] = v[i].x >> 16;
    out[3 * i + 1] = v[i].x & 0xffff;
    out[3 * i + 2] = v[i].y;
  }
  return n == total ? MM_OK : MM_ERR_ARG;
}

extern "C" mm_status mm_check_bounded_wait(int n_polls, int flag_set, int* expired, void* stream) {
  using namespace mm;
  if (!expired || n_polls < 1 || n_polls > (1 << 22)) {
    mm_set_error("mm_check_bounded_wait: expired is NULL or n_polls outside [1, 2^22]");
    return MM_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void* flag = nullptr;
  void* fault = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&flag, g_wait_flag);
  if (e == cudaSuccess) e = cudaGetSymbolAddress(&fault, g_wait_fault);
  const unsigned f = flag_set ? 1u : 0u;
  if (e == cudaSuccess) e = cudaMemcpyAsync(flag, &f, sizeof(f), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(fault, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_wait_check<<<1, 32, 0, s>>>(n_polls);
    e = cudaGetLastError();
  }
  int r = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&r, fault, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    mm_set_error("mm_check_bounded_wait: %s", cudaGetErrorString(e));
    return MM_ERR_CUDA;
  }
  *expired = r;
  return MM_OK;
}
