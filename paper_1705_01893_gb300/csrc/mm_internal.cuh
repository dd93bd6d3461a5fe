// Internal declarations of the messenger mapmaker: plan layout, chunk descriptors,
// complex arithmetic and the shared-memory Stockham FFT used by every hot kernel.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/mm.h"

namespace mm {

// ----------------------------------------------------------------------------- layout
// One chunk of the timestream.  Its rfft of length n = 2M is computed as a complex FFT of
// length M = M1 * M2 over z_j = x_{2j} + i x_{2j+1}, done as a four-step transform:
// column FFTs of length M1 (kernel A / C), twiddles w_M^{k1 j2}, row FFTs of length M2
// (kernel B).  Spectra live in "row layout": slot k1*M2 + k2 holds frequency k1 + M1*k2.
// A chunk of odd length n ("complex" chunk, general path only) is transformed as a complex
// FFT of M = n points over z_j = x_j + 0i; its row layout then holds all n frequencies.
struct ChunkDesc {
  int64_t off;       // first sample of the chunk
  int64_t spec;      // first slot of the chunk in the spectrum-sized buffers (M per chunk)
  int64_t nat;       // first bin of the chunk in natural-order rfft arrays (n/2 + 1 per chunk)
  int n, M, M1, M2;
  int grp;           // FFT group
  int cplx;          // 1: odd n, complex transform of M = n points
  double tau;        // messenger variance tau_c (Sec. 4.2)
};

// Chunks of the same length share FFT shapes and twiddle tables and run in one launch.
// Power-of-two lengths use the compile-time kernels; other 5-smooth lengths ("general")
// use runtime mixed-radix Stockham passes with the radix sequences below.
constexpr int kMaxRadices = 16;
struct Group {
  int M, M1, M2, log_lo;   // w_M^e = tw_hi[e >> log_lo] * tw_lo[e & (2^log_lo - 1)]
  int n_chunks;
  int batch;               // chunks per batch
  int general, cplx;       // general path; odd length (complex transform)
  int nr1, nr2;            // general: radix sequences of the M1 and M2 DFTs
  int8_t rad1[kMaxRadices], rad2[kMaxRadices];
  int* chunks;             // device: chunk indices of this group
  float2* tw_col;          // per-pass twiddles of the length-M1 DFT (see tw_offset;
                           // general: [< 2 M1], pass tables of the tuned radix plan)
  float2* tw_row;          // per-pass twiddles of the length-M2 DFT (general: [< 2 M2])
  float2* tw_lo;           // [2^log_lo]          exp(-2 pi i m / M)
  float2* tw_hi;           // [M >> log_lo (+1)]   exp(-2 pi i m 2^log_lo / M)
  float2* tw_pack_a;       // [M1]  exp(-2 pi i m / (2M))     (real-pack twiddle, k1 part)
  float2* tw_pack_b;       // [M2]  exp(-2 pi i m M1 / (2M))  (real-pack twiddle, k2 part)
};

constexpr int kMaxGroups = 128;

// Column / row limits of the general path (shared memory of one CTA: two ping-pong tiles).
constexpr int kGenMaxM1 = 512;
constexpr int kGenMaxM2 = 4096;
// Row jobs of the general path gather pairs of rows (k1, M1 - k1) up to about this many
// elements, so that each Stockham pass has several butterflies per thread.
constexpr int kGenRowElems = 4096;
__host__ __device__ inline int gen_row_pairs(int M1, int M2) {
  const int h = (M1 - 1) / 2;                 // rows 1 .. h pair with M1 - 1 .. M1 - h
  int n = kGenRowElems / (2 * M2);
  if (n < 1) n = 1;
  return h < n ? h : n;
}

// A batch: `count` consecutive chunks of one group whose four-step intermediates share the
// ybuf slot (its size is the plan's intermediate budget, 2 GB by default); batches run one
// after another on the caller's stream.
struct Batch {
  int group;          // -1: a batch of the general path (chunks of any general length)
  int first;          // index into the group's chunk list (general: into the general list)
  int count;
};

// State of the plateau-driven cooling controller (device memory, one per plan).
constexpr int kMaxLevels = 64;
struct AdaptState {
  int level;          // current level, -1 during the lambda = inf step
  int start;          // iterations done when the current level began
  int n_done;         // iterations run, set when the loop ends
  int n_levels, min_per, max_per, max_iter;
  double rel_tol;
  double* chi2;       // [max_iter] chi^2 of each iteration's input map
  double* lambda_out; // [max_iter] lambda of each iteration
  double levels[kMaxLevels];
};

// Schedule of the general path's persistent kernels: tile width, threads and radix order
// (picked per plan by measurement, see mm_autotune).
struct GenTune {
  int col_nb;         // columns per column tile: 8 or 16
  int col_threads;    // 256 or 512
  int row_threads;    // 256, 512 or 1024
  int radix_order;    // 0: radix 8 first, then 4/2, 5, 3; 1: radix 4 instead of 8; 2: 3s and 5s first
};

// Everything a general-path kernel needs about one chunk, in one record (one dependent load
// per work item instead of chunk list -> descriptor -> group).
struct GenChunk {
  ChunkDesc d;
  int c;                   // chunk index in the plan
  int log_lo, nr1, nr2;
  int64_t yoff;            // intermediate offset in the general list
  const float2* tw_col;    // per-pass tables of the M1 DFT for the radix plan rad1
  const float2* tw_row;    // per-pass tables of the M2 DFT for the radix plan rad2
  const float2* tw_lo;
  const float2* tw_hi;
  const float2* pack_a;
  const float2* pack_b;
  int8_t rad1[kMaxRadices], rad2[kMaxRadices];
};

}  // namespace mm

struct mm_plan_s {
  int n_chunks, ncomp, wdtype;
  // composite pointing P = g_a P_a + g_b P_b (App. B); the first component is pix/cosw/sinw
  int composite;
  const int32_t* pix_b;
  const void* cos_b;
  const void* sin_b;
  float gain_a, gain_b;
  int64_t n_pix, n_total, spec_total;
  double rcond_min;
  const int32_t* pix;
  const void* cosw;
  const void* sinw;
  // host copies
  mm::ChunkDesc* h_desc;
  int n_groups;
  mm::Group groups[mm::kMaxGroups];
  int* h_chunk_group;
  mm::Batch* h_batches;
  int n_batches;
  bool noise_set;
  // device regions inside the caller's workspace
  mm::ChunkDesc* d_desc;
  int32_t* hits;
  uint8_t* valid;
  double* W;        // [n_pix][6] (IQU, symmetric upper triangle 00 01 02 11 12 22) or [n_pix]
  double* Minv;     // PCG block preconditioner, same layout
  double* acc;      // [ncomp][n_pix] (planar) FP64 accumulators of P^T T^-1 t
  double* acc12;    // [n_pix][12] set-up scratch: P^T T^-1 P and sum c0 P^T P (6 each)
  void* map4;       // float4 [n_pix] (IQU) or float [n_pix] (T)
  double* bvec;     // [n_pix][ncomp] b = P^T N^-1 d
  float2* dtab;     // [spec_total] d~ in row layout (slot 0: (d~_0, d~_M))
  float* nbar;      // [spec_total] Nbar on the same slots (slot 0: Nbar_0)
  float* nyq;       // [n_chunks] Nbar at the Nyquist bin
  double* c0;       // [n_chunks] (1/n) sum_k w_k / N_k
  float2* ybuf;     // one batch's four-step intermediate (L2-resident between passes)
  size_t ybuf_bytes;
  bool theta_ok;     // noise from (sigma, f_knee, alpha) with tau = sigma^2: theta gradients defined
  // CUDA graph of one messenger iteration (captured on first use of mm_messenger_graph)
  cudaGraphExec_t graph_exec;
  cudaStream_t graph_stream;
  double* lam_table;   // device [lam_cap] schedule
  int lam_cap;
  int* iter;           // device iteration counter
  double** chi2_base;  // device pointer slot: chi^2 output array or NULL
  double* map64;       // device FP64 copy of the current map (graph mode)
  // adaptive cooling: graph with a device-side loop (conditional WHILE node) and its state
  cudaGraphExec_t adapt_exec;
  void* adapt_st;      // device mm::AdaptState followed by the level table
  unsigned* row_queue; // device [2]: the row kernel's job counter and finished-CTA count
                       // (zero between launches: the last CTA of each launch resets both)
  // fused iteration kernel (mm_fused.cu): per-batch item lists, counters, fault flag
  int2* fused_items;   // device, all eligible batches' lists back to back
  int* h_fused_first;  // host [n_batches]: offset of the batch's list (items)
  int* h_fused_n;      // host [n_batches]: items of the batch's list, 0 = not fused
  unsigned* fused_ctr; // device [2 + 2 n_chunks], zero between launches
  int* fault;          // device flag: a bounded wait of a kernel expired
  int wait_polls;      // poll limit of the fused launch's waits (default 2^22, about a second)
  int check_on_return; // 1: the solver calls synchronise and report an expired wait
  double* scal;     // [64] scalars (see kScal*)
  double* params;   // [n_chunks][4] noise parameters (device copy)
  float2* tw_pool;
  // general path: chunk list in plan order and per-chunk prefix sums over it (column tiles,
  // row jobs, intermediate elements), device and host copies; device copy of the groups
  int n_gen;
  int* gen_chunks;
  int64_t* gen_ctile;
  int64_t* gen_rjob;
  int64_t* gen_yoff;
  int64_t* h_gen_ctile;
  int64_t* h_gen_rjob;
  int64_t* h_gen_yoff;
  int* h_gen_chunks;
  mm::GenChunk* gen_rec;   // [n_gen] device records
  int2* gen_ctab;          // column tiles: (general index, first column), capacity gen_ccap
  int4* gen_rtab;          // row jobs: (general index, first row, pairs or 0 for a self-paired row)
  int64_t gen_ccap;
  mm::Group* d_groups;
  mm::GenTune gen_tune;
  int32_t* tpix;    // pointing copied into column-tile order (see k_tile_pointing)
  void* tcos;
  void* tsin;
};

namespace mm {

enum {
  kScalLambdaMax = 0,   // stored as the bit pattern of a non-negative double
  kScalCdd = 1,         // d^T N^-1 d
  kScalTmp = 2,
  kScalCount = 64
};

// ---------------------------------------------------------------------- complex helpers
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return make_float2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) {
  return make_float2(a.x * s, a.y * s);
}
// multiply by -i (DIR < 0) or +i (DIR > 0)
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// Distance between the component planes of the FP64 pixel accumulators ([ncomp][stride]):
// n_pix rounded up to 32 and skewed by 32 more, so that planes are never a power of two
// apart (measured: the 4 M-pixel map step 0.256 -> 0.244 ms, no change at 262 k pixels).
__host__ __device__ __forceinline__ int64_t acc_stride_of(int64_t n_pix, int ncomp) {
  return ncomp == 1 ? n_pix : ((n_pix + 31) / 32) * 32 + 32;
}

// ------------------------------------------------------------------------- butterflies
// In-register DFTs of length 2, 4, 8 with kernel exp(DIR * 2 pi i jk / R).
template <int DIR>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3) {
  float2 t0 = cadd(v0, v2), t1 = csub(v0, v2);
  float2 t2 = cadd(v1, v3), t3 = mul_i<DIR>(csub(v1, v3));
  v0 = cadd(t0, t2);
  v2 = csub(t0, t2);
  v1 = cadd(t1, t3);
  v3 = csub(t1, t3);
}

template <int DIR>
__device__ __forceinline__ void dft8(float2* v) {
  const float h = 0.70710678118654752440f;
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<DIR>(e0, e1, e2, e3);
  dft4<DIR>(o0, o1, o2, o3);
  // o_k *= w8^k, w8 = exp(DIR * i pi / 4)
  o1 = DIR < 0 ? make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x))
               : make_float2(h * (o1.x - o1.y), h * (o1.y + o1.x));
  o2 = mul_i<DIR>(o2);
  o3 = DIR < 0 ? make_float2(h * (o3.y - o3.x), -h * (o3.x + o3.y))
               : make_float2(-h * (o3.x + o3.y), h * (o3.x - o3.y));
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

// v *= exp(DIR * 2 pi i e / 16) for the constant exponents a radix-16 butterfly needs.
template <int DIR, int E>
__device__ __forceinline__ float2 w16(float2 v) {
  constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;
  constexpr float h = 0.70710678118654752440f;
  constexpr float cx = E == 1 ? c1 : E == 2 ? h : E == 3 ? s1 : E == 6 ? -h : E == 9 ? -c1 : 0.f;
  constexpr float sy = E == 1 ? s1 : E == 2 ? h : E == 3 ? c1 : E == 6 ? h : E == 9 ? -s1 : 1.f;
  constexpr float cy = DIR < 0 ? -sy : sy;
  if constexpr (E == 4) return mul_i<DIR>(v);
  return make_float2(v.x * cx - v.y * cy, v.x * cy + v.y * cx);
}

// DFT of 16 points as 4 x 4: DFT4 over the stride-4 subsequences, constant twiddles
// w16^(n1 k1), DFT4 over the contiguous quadruples; the result sits 4x4-transposed in
// registers and is renamed back into natural order.
template <int DIR>
__device__ __forceinline__ void dft16(float2* v) {
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) dft4<DIR>(v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]);
  v[5] = w16<DIR, 1>(v[5]);  v[9] = w16<DIR, 2>(v[9]);   v[13] = w16<DIR, 3>(v[13]);
  v[6] = w16<DIR, 2>(v[6]);  v[10] = w16<DIR, 4>(v[10]); v[14] = w16<DIR, 6>(v[14]);
  v[7] = w16<DIR, 3>(v[7]);  v[11] = w16<DIR, 6>(v[11]); v[15] = w16<DIR, 9>(v[15]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<DIR>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  float2 t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2 + 4 * k1];
}

// DFT of 3 points: y_{1,2} = v0 - (v1 + v2)/2 +- DIR i (sqrt 3 / 2)(v1 - v2).
template <int DIR>
__device__ __forceinline__ void dft3(float2* v) {
  constexpr float h3 = 0.86602540378443864676f;   // sin(2 pi / 3)
  const float2 t1 = cadd(v[1], v[2]);
  const float2 t2 = cscale(mul_i<DIR>(csub(v[1], v[2])), h3);
  const float2 m = make_float2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
  v[0] = cadd(v[0], t1);
  v[1] = cadd(m, t2);
  v[2] = csub(m, t2);
}

// DFT of 5 points from the sums and differences of the symmetric pairs (1, 4) and (2, 3):
// y_{1,4} = v0 + c1 a + c2 b +- DIR i (s1 p + s2 q), y_{2,3} = v0 + c2 a + c1 b +- DIR i (s2 p - s1 q)
// with a = v1 + v4, b = v2 + v3, p = v1 - v4, q = v2 - v3, c_j = cos(2 pi j / 5), s_j = sin(2 pi j / 5).
template <int DIR>
__device__ __forceinline__ void dft5(float2* v) {
  constexpr float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
  constexpr float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
  const float2 a = cadd(v[1], v[4]), b = cadd(v[2], v[3]);
  const float2 p = csub(v[1], v[4]), q = csub(v[2], v[3]);
  const float2 r1 = make_float2(v[0].x + c1 * a.x + c2 * b.x, v[0].y + c1 * a.y + c2 * b.y);
  const float2 r2 = make_float2(v[0].x + c2 * a.x + c1 * b.x, v[0].y + c2 * a.y + c1 * b.y);
  const float2 i1 = mul_i<DIR>(make_float2(s1 * p.x + s2 * q.x, s1 * p.y + s2 * q.y));
  const float2 i2 = mul_i<DIR>(make_float2(s2 * p.x - s1 * q.x, s2 * p.y - s1 * q.y));
  v[0] = cadd(v[0], cadd(a, b));
  v[1] = cadd(r1, i1);
  v[4] = csub(r1, i1);
  v[2] = cadd(r2, i2);
  v[3] = csub(r2, i2);
}

template <int R, int DIR>
__device__ __forceinline__ void dftR(float2* v) {
  if constexpr (R == 2) dft2<DIR>(v[0], v[1]);
  else if constexpr (R == 3) dft3<DIR>(v);
  else if constexpr (R == 4) dft4<DIR>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 5) dft5<DIR>(v);
  else if constexpr (R == 8) dft8<DIR>(v);
  else dft16<DIR>(v);
}

// ----------------------------------------------------------------- shared-memory layouts
// Column layout: NB transforms interleaved, element (b, i) at s[i * NB + b]; with NB >= 16
// consecutive b are consecutive 8-byte words, so every access of a pass is conflict-free.
// Narrower tiles (NB = 8, 4) get one spare block of NB words after every 16 rows: the first
// radix-16 pass stores the rows of a warp's butterflies 16 rows apart, which would
// otherwise fall on the same banks; the spare block shifts each by 2 NB banks.
template <int NB>
struct ColLayout {
  static constexpr int kPad = NB < 16 ? NB : 0;
  __device__ __forceinline__ static int at(int b, int i) {
    return i * NB + b + (kPad ? (i >> 4) * kPad : 0);
  }
  // float2 words of a tile of NB transforms of length L
  __host__ __device__ static constexpr int size(int L) { return L * NB + (kPad ? (L >> 4) * kPad : 0); }
  static constexpr bool kBFast = true;
};
// Row layout: transform b occupies [b*L, (b+1)*L), XOR-swizzled in 16-word groups so the
// strided stores of the first Stockham passes spread over all banks.
template <int L>
struct RowLayout {
  __device__ __forceinline__ static int swz(int idx) { return idx ^ ((idx >> 4) & 15); }
  __device__ __forceinline__ static int at(int b, int i) { return swz(b * L + i); }
  static constexpr bool kBFast = false;
};

// Radix plan of a length-L DFT: ceil(log2(L)/4) passes with radices 2^r as equal as
// possible, larger radices first (4096 = 16.16.16, 2048 = 16.16.8, 512 = 8.8.8).
__host__ __device__ constexpr int pick_radix(int rem) {
  const int m = ilog2(rem);
  const int P = (m + 3) / 4;
  const int r = (m + P - 1) / P;
  return 1 << r;
}
// Offset of the twiddle table of the pass whose input sub-transforms have length Ns; the
// pass (Ns, R) stores w_{Ns R}^{r k} at [r * Ns + k], so lanes with consecutive k read
// consecutive words.
__host__ __device__ constexpr int tw_offset(int L, int Ns) {
  int off = 0, ns = 1;
  while (ns < Ns) {
    const int r = pick_radix(L / ns);
    off += ns * r;
    ns *= r;
  }
  return off;
}
__host__ __device__ constexpr int tw_size(int L) { return tw_offset(L, L); }

// Tag: a pass reads from / writes to the shared-memory buffer itself.
struct SmemIO {};

// One radix-R Stockham pass (auto-sorting): for butterfly j of transform b with k = j mod Ns,
// gather x[j + r L/R], twiddle by w_{Ns R}^{r k}, DFT_R, scatter to (j - k) R + k + q Ns.
// Input comes from shared memory or, for a first pass, from src(b, i); output goes to
// shared memory or, for a last pass, to dst(b, i, value) (where (j - k) R + k = j, so
// consecutive threads write consecutive i).  In place in shared memory through registers.
template <int L, int NB, class Lay, int T, int DIR, int R, int Ns, class Src, class Dst>
__device__ __forceinline__ void fft_pass_io(float2* s, const float2* __restrict__ tw,
                                            const Src& src, const Dst& dst) {
  constexpr bool kSrcSm = std::is_same<Src, SmemIO>::value;
  constexpr bool kDstSm = std::is_same<Dst, SmemIO>::value;
  constexpr int NBF = NB * (L / R);
  constexpr int U = (NBF + T - 1) / T;
  constexpr int TWO = tw_offset(L, Ns);
  float2 v[U][R];
  int jj[U], bb[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int g = threadIdx.x + u * T;
    if (NBF % T != 0 && g >= NBF) continue;
    int b, j;
    if constexpr (Lay::kBFast) { b = g % NB; j = g / NB; }
    else { j = g % (L / R); b = g / (L / R); }
    jj[u] = j; bb[u] = b;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (kSrcSm) v[u][r] = s[Lay::at(b, j + r * (L / R))];
      else v[u][r] = src(b, j + r * (L / R));
    }
    if constexpr (Ns > 1) {
      const int k = j % Ns;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = tw[TWO + r * Ns + k];
        if (DIR > 0) w.y = -w.y;
        v[u][r] = cmul(v[u][r], w);
      }
    }
    dftR<R, DIR>(v[u]);
  }
  if constexpr (kSrcSm && kDstSm) __syncthreads();
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int g = threadIdx.x + u * T;
    if (NBF % T != 0 && g >= NBF) continue;
    const int j = jj[u], b = bb[u];
    const int k = j % Ns;
    const int o = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (kDstSm) s[Lay::at(b, o + r * Ns)] = v[u][r];
      else dst(b, o + r * Ns, v[u][r]);
    }
  }
  if constexpr (kDstSm) __syncthreads();
}

template <int L, int NB, class Lay, int T, int DIR, int Ns, class Src, class Dst>
__device__ __forceinline__ void fft_passes_io(float2* s, const float2* __restrict__ tw,
                                              const Src& src, const Dst& dst) {
  if constexpr (Ns < L) {
    constexpr int R = pick_radix(L / Ns);
    constexpr bool first = Ns == 1, last = Ns * R == L;
    if constexpr (first && last) fft_pass_io<L, NB, Lay, T, DIR, R, Ns, Src, Dst>(s, tw, src, dst);
    else if constexpr (first)
      fft_pass_io<L, NB, Lay, T, DIR, R, Ns, Src, SmemIO>(s, tw, src, SmemIO{});
    else if constexpr (last)
      fft_pass_io<L, NB, Lay, T, DIR, R, Ns, SmemIO, Dst>(s, tw, SmemIO{}, dst);
    else fft_pass_io<L, NB, Lay, T, DIR, R, Ns, SmemIO, SmemIO>(s, tw, SmemIO{}, SmemIO{});
    fft_passes_io<L, NB, Lay, T, DIR, Ns * R>(s, tw, src, dst);
  }
}

// NB unnormalised length-L DFTs (kernel exp(DIR 2 pi i jk / L)), natural order in and out.
// Input from src (or shared memory), output to dst (or shared memory).  tw: the per-pass
// tables (tw_size(L) entries).  A shared-memory destination ends with a __syncthreads; a
// caller that reads from a functor must have finished every earlier use of `s`.
template <int L, int NB, class Lay, int T, int DIR, class Src = SmemIO, class Dst = SmemIO>
__device__ __forceinline__ void smem_fft(float2* s, const float2* __restrict__ tw,
                                         const Src& src = Src{}, const Dst& dst = Dst{}) {
  fft_passes_io<L, NB, Lay, T, DIR, 1>(s, tw, src, dst);
}

// L2 eviction priority of the FP64 pixel accumulators: their reductions carry an
// evict-last policy, so that the accumulators of a large map (100 MB at 4 M IQU pixels)
// keep their lines in L2 against the streams of pointing and intermediate that pass
// through it once per pass (read with evict-first loads).
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// *a += v (relaxed, device scope, performed in L2) with an L2 cache policy.
__device__ __forceinline__ void red_add_f64(double* a, double v, uint64_t pol) {
  asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.f64 [%0], %1, %2;"
               ::"l"(a), "d"(v), "l"(pol) : "memory");
}

// Bulk prefetch of [p, p + bytes) into L2 by the TMA engine (p and bytes multiples of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Bulk prefetch of the 16-byte-aligned interior of [p, p + bytes) (start rounded up, end
// rounded down, so that nothing outside the range is touched), for ranges that need not be
// aligned (rows of general-length chunks).
__device__ __forceinline__ void prefetch_l2_inner(const void* p, size_t bytes) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p), e = a + bytes;
  const uintptr_t a16 = (a + 15) & ~uintptr_t(15), e16 = e & ~uintptr_t(15);
  if (e16 > a16) prefetch_l2(reinterpret_cast<const void*>(a16), (unsigned)(e16 - a16));
}

// Resident CTAs of `kernel` on the whole GPU (opting it in to `smem` bytes of dynamic
// shared memory on first use); cached per kernel.
cudaError_t resident_ctas(const void* kernel, int threads, size_t smem, int* out);

// Grid of a persistent kernel: resident CTAs per SM x SMs, at most `work` CTAs.
template <typename K>
static cudaError_t persistent_grid(K kernel, int threads, size_t smem, int work, int* grid) {
  int resident = 0;
  cudaError_t e = resident_ctas(reinterpret_cast<const void*>(kernel), threads, smem, &resident);
  if (e != cudaSuccess) return e;
  *grid = work < resident ? work : resident;
  return cudaSuccess;
}

// Exact FP32 -> FP64 widening with integer operations only (sign, exponent rebias, mantissa
// shift), keeping the conversion off GB300's narrow FP64 pipe; the FP64 additions then
// happen in the L2 atomic units.  Zero and subnormal inputs give +-0 (|x| < 1.2e-38).
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long ed = e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896u);
  const unsigned long long mag = (ed << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)(e == 0u ? sgn : (sgn | mag)));
}

// w_M^e for 0 <= e < M from the two-level table (FP64-accurate entries, FP32 product).
__device__ __forceinline__ float2 tw_big(const Group& g, int e) {
  return cmul(__ldg(&g.tw_hi[e >> g.log_lo]), __ldg(&g.tw_lo[e & ((1 << g.log_lo) - 1)]));
}

// -------------------------------------------------------------------- kernel launchers
// Modes of the row kernel (B).
enum RowMode {
  kRowSpectrum = 0,   // forward only: store X = rfft(x) into dtab (row layout)
  kRowNatural = 1,    // forward only: store X into a natural-order complex64 array
  kRowMessenger = 2,  // forward, messenger filter (+ chi^2 of the input), inverse
  kRowPcgApply = 3,   // forward, Y = X / N, inverse
  kRowPcgRhs = 4,     // no forward: Y = d~ / N (+ chi^2 of m = 0, i.e. d^T N^-1 d), inverse
  kRowChi2 = 5,       // forward, chi^2 only
  // map-sized form m' = m_d(lambda) + F(lambda) m of the messenger step (Sec. 2.1):
  kRowMessengerF = 6, // forward, Y = Nbar X / (lambda tau + Nbar) (the F part, no d~), chi^2
                      // partial sum_k w_k |X_k|^2 / N_k / n, inverse
  kRowMd = 7,         // no forward: Y = lambda tau d~ / (lambda tau + Nbar) (the m_d part), inverse
  // composite pointing (App. B), general path only:
  kRowResidual = 8,   // forward, Y = (d~ - X) / (n (Nbar / lambda + tau)), chi^2, inverse
  // the messenger step that also keeps its forward spectrum X = (P m)~ in row layout at
  // RowArgs::natural + spec (the adjoint's recomputation; run-time instance only)
  kRowMessengerKeep = 9,
  // forward, chi^2(m, lambda) per Fourier mode, |d~_k - X_k|^2 / (n (Nbar_k + lambda tau)),
  // as float64 at ((double*)RowArgs::natural)[nat + k] in natural order, and the total
  kRowChi2Modes = 10
};

struct RowArgs {
  int mode;
  double lambda;       // cooling parameter (messenger) / N' = N + (lambda-1) tau (chi^2)
  double* chi2;        // device accumulator or nullptr
  float2* natural;     // kRowNatural output (natural order), kRowMessengerKeep output (row layout)
  // Graph mode (lam_table != nullptr): lambda = lam_table[*iter] and the chi^2 slot is
  // chi2_base[0] + *iter when chi2_base[0] is set; the values live in device memory so one
  // captured CUDA graph serves every iteration of a schedule.
  const double* lam_table = nullptr;
  const int* iter = nullptr;
  double* const* chi2_base = nullptr;
};

// Source of the forward column pass.
enum ColSrc { kSrcGather = 0, kSrcTod = 1 };

cudaError_t launch_col_forward(const mm_plan_s* p, const Batch& b, int src, const float* tod,
                               cudaStream_t st);
cudaError_t launch_row(const mm_plan_s* p, const Batch& b, const RowArgs& a, cudaStream_t st);
// One messenger iteration on map_inout (as mm_messenger_iterate) that also keeps each
// chunk's forward spectrum (P m)~ in row layout at keep + ChunkDesc::spec (mm_api.cu).
mm_status messenger_step_keep(mm_plan_s* p, double lambda, double* map_inout, float2* keep,
                              cudaStream_t s);
// Fused A + B + C launch of one batch's messenger iteration (mm_fused.cu).
bool fused_eligible(const mm_plan_s* p, const Batch& b);
int fused_items_per_chunk(int M1, int M2, bool general);
int fused_build_items(int M1, int M2, int count, int2* out);
cudaError_t launch_fused(const mm_plan_s* p, const Batch& b, const RowArgs& a, cudaStream_t st);
cudaError_t launch_col_inverse(const mm_plan_s* p, const Batch& b, cudaStream_t st);
cudaError_t launch_tile_pointing(const mm_plan_s* p, cudaStream_t st);
// General path (mm_gen.cu): the same three stages for a batch of general-length chunks,
// one persistent launch each, with the same intermediate layout and scale conventions.
cudaError_t launch_gen_col_forward(const mm_plan_s* p, const Batch& b, int src, const float* tod,
                                   cudaStream_t st);
cudaError_t launch_gen_row(const mm_plan_s* p, const Batch& b, const RowArgs& a, cudaStream_t st);
cudaError_t launch_gen_col_inverse(const mm_plan_s* p, const Batch& b, cudaStream_t st);
// Copy the general chunks' pointing into column-tile order for the schedule's tile width
// (run whenever that width is set).
cudaError_t launch_gen_tile_pointing(const mm_plan_s* p, cudaStream_t st);
// Forward column pass gathering from `map4` into `ybuf` (either NULL = the plan's own).
cudaError_t launch_col_forward_ex(const mm_plan_s* p, const Batch& b, int src, const float* tod,
                                  const void* map4, float2* ybuf, cudaStream_t st);
// Columns per tile of the column kernels: 16 (runs of 32 samples) up to 512-point columns,
// then 8192 / M1 (8 for 1024, 4 for 2048 points), so that a tile stays at 64 KB and 512
// threads: two CTAs per SM overlap one's loads with the other's DFT passes.
constexpr int kColCB = 16;
__host__ __device__ constexpr int col_cb(int M1) { return M1 <= 512 ? kColCB : 8192 / M1; }
// Threads of the column kernels for column length M1 (16 complex values per thread per pass).
__host__ __device__ constexpr int col_threads(int M1) {
  return M1 * col_cb(M1) / 16 < 64 ? 64
         : (M1 * col_cb(M1) / 16 > 1024 ? 1024 : M1 * col_cb(M1) / 16);
}

}  // namespace mm

// error reporting shared by the ABI translation units
void mm_set_error(const char* fmt, ...);

// NVTX range around an entry point (header-only NVTX 3: a no-op unless a profiler that
// records ranges is attached).
#include <nvtx3/nvToolsExt.h>
struct MmRange {
  explicit MmRange(const char* name) { nvtxRangePushA(name); }
  ~MmRange() { nvtxRangePop(); }
  MmRange(const MmRange&) = delete;
  MmRange& operator=(const MmRange&) = delete;
};
