// Plain FP64 messenger step: one cooperative launch per iteration, everything in double
// precision and with no blocking beyond the textbook algorithm -- the same-GPU baseline the
// FP32 four-step path is measured against.  Per iteration (Sec. 2.1, residual form of the
// messenger update, a + b = 1):
//   x   = d - P m                                    (gather, FP64 weights and map)
//   X   = FFT of the packed complex sequence x_2j + i x_2j+1   (radix-2 Stockham passes
//         through global memory)
//   Y_k = b_k X_k / n,  b_k = Nbar_k / (lambda tau + Nbar_k),  chi^2 += w_k |X_k|^2 / N_k / n
//   t   = d - irfft(Y)
//   m'  = (P^T T^-1 P)^-1 P^T t / tau                (FP64 atomics, per-pixel 3x3 solve)
// Phases are separated by a grid barrier whose waits are bounded: a barrier that does not
// complete within its limit sets an error flag, every thread returns, and the host reports
// MM_ERR_TIMEOUT.
#include <math.h>

#include "mm_internal.cuh"

namespace mm {

struct PlainArgs {
  const ChunkDesc* desc;
  int n_chunks, M, logM;
  const int32_t* pix;
  const void* cosw;
  const void* sinw;
  int half_w, ncomp;
  const float* tod;
  double* map;                 // in: m_i, out: m_{i+1} (float64 [n_pix][ncomp])
  const double* W;
  const uint8_t* valid;
  double* acc;
  int64_t n_pix;
  const float* nbar;           // plan's Nbar table (row layout) and Nyquist values
  const float* nyq;
  int M1, M2;
  const double2* tw;           // exp(-2 pi i m / M), m < M / 2
  const double2* tw2;          // exp(-i pi k / M), k <= M / 2
  double2* buf0;
  double2* buf1;
  double lambda;
  double* chi2;
  unsigned* bar;               // [0] arrival count, [1] generation
  int* err;
};

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Grid-wide barrier with bounded waiting (about 2 s); false once any CTA has timed out.
__device__ bool plain_sync(const PlainArgs& a) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = a.bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(a.bar, 1u) == gridDim.x - 1) {
      a.bar[0] = 0;
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      long long it = 0;
      while (*gen == g) {
        if (++it > 2000000 || *(volatile int*)a.err) {
          atomicExch(a.err, 1);
          break;
        }
        __nanosleep(1000);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)a.err == 0;
}

__device__ __forceinline__ double plain_w(const void* w, int half_w, int64_t s) {
  return half_w ? (double)__half2float(static_cast<const __half*>(w)[s])
                : (double)static_cast<const float*>(w)[s];
}

__device__ __forceinline__ double plain_pm(const PlainArgs& a, int64_t s) {
  const int p = a.pix[s];
  if (p < 0 || !a.valid[p]) return 0.0;
  if (a.ncomp == 1) return a.map[p];
  const double* m = a.map + 3 * (int64_t)p;
  return m[0] + plain_w(a.cosw, a.half_w, s) * m[1] + plain_w(a.sinw, a.half_w, s) * m[2];
}

// One radix-2 Stockham pass over every chunk: out[(j-k)2 + k (+Ns)] = in[j] +- w in[j+M/2].
__device__ void plain_pass(const PlainArgs& a, const double2* in, double2* out, int Ns, int dir) {
  const int half = a.M / 2;
  const int64_t total = (int64_t)a.n_chunks * half;
  const int stride = a.M / (2 * Ns);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t base = (g / half) * a.M;
    const int j = (int)(g % half);
    const int k = j % Ns;
    double2 w = a.tw[k * stride];
    if (dir > 0) w.y = -w.y;
    const double2 v0 = in[base + j];
    const double2 v1 = zmul(in[base + j + half], w);
    const int o = (j - k) * 2 + k;
    out[base + o] = make_double2(v0.x + v1.x, v0.y + v1.y);
    out[base + o + Ns] = make_double2(v0.x - v1.x, v0.y - v1.y);
  }
}

// log2(M) passes; returns the buffer holding the result.
__device__ double2* plain_fft(const PlainArgs& a, int dir, bool* ok) {
  double2* in = a.buf0;
  double2* out = a.buf1;
  for (int Ns = 1; Ns < a.M; Ns *= 2) {
    plain_pass(a, in, out, Ns, dir);
    if (!(*ok = plain_sync(a))) return in;
    double2* t = in; in = out; out = t;
  }
  return in;
}

__device__ __forceinline__ float plain_nbar(const PlainArgs& a, int c, int k) {
  if (k == a.M) return a.nyq[c];
  return a.nbar[a.desc[c].spec + (int64_t)(k % a.M1) * a.M2 + k / a.M1];
}

__global__ void k_plain_iteration(PlainArgs a) {
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int half = a.M / 2;
  bool ok = true;
  // 1. residual x = d - P m, packed z_j = x_2j + i x_2j+1 per chunk
  for (int64_t g = tid; g < (int64_t)a.n_chunks * a.M; g += nthreads) {
    const int c = (int)(g / a.M);
    const int j = (int)(g % a.M);
    const int64_t s = a.desc[c].off + 2ll * j;
    a.buf0[g] = make_double2((double)a.tod[s] - plain_pm(a, s),
                             (double)a.tod[s + 1] - plain_pm(a, s + 1));
  }
  if (!plain_sync(a)) return;
  // 2. forward FFT
  double2* Z = plain_fft(a, -1, &ok);
  if (!ok) return;
  double2* Zo = Z == a.buf0 ? a.buf1 : a.buf0;
  // 3. split X = rfft(x), chi^2, filter Y = b X / n, merge back into packed form
  double x2 = 0.0;
  const bool lam_inf = isinf(a.lambda);
  for (int64_t g = tid; g < (int64_t)a.n_chunks * (half + 1); g += nthreads) {
    const int c = (int)(g / (half + 1));
    const int k = (int)(g % (half + 1));
    const ChunkDesc& d = a.desc[c];
    const double tau = d.tau, n = (double)d.n;
    const double2* z = Z + (int64_t)c * a.M;
    double2* zo = Zo + (int64_t)c * a.M;
    const int kp = (a.M - k) % a.M;
    const double2 Zk = z[k], Zp = z[kp];
    if (k == 0) {
      const double X0 = Zk.x + Zk.y, XM = Zk.x - Zk.y;
      const double n0 = plain_nbar(a, c, 0), nM = plain_nbar(a, c, a.M);
      x2 += (X0 * X0 / (n0 + tau) + XM * XM / (nM + tau)) / n;
      const double b0 = lam_inf ? 0.0 : n0 / (a.lambda * tau + n0);
      const double bM = lam_inf ? 0.0 : nM / (a.lambda * tau + nM);
      const double Y0 = b0 * X0 / n, YM = bM * XM / n;
      zo[0] = make_double2(Y0 + YM, Y0 - YM);
      continue;
    }
    // w = exp(-i pi k / M); E = (Zk + conj Zp)/2, O = -i (Zk - conj Zp)/2
    const double2 w = a.tw2[k];
    const double2 E = make_double2(0.5 * (Zk.x + Zp.x), 0.5 * (Zk.y - Zp.y));
    const double2 O = make_double2(0.5 * (Zk.y + Zp.y), -0.5 * (Zk.x - Zp.x));
    const double2 wO = zmul(w, O);
    const double2 Xk = make_double2(E.x + wO.x, E.y + wO.y);
    const double2 Xp = make_double2(E.x - wO.x, -(E.y - wO.y));
    const double nk = plain_nbar(a, c, k), np = plain_nbar(a, c, a.M - k);
    const bool same = kp == k;
    x2 += 2.0 * (Xk.x * Xk.x + Xk.y * Xk.y) / (nk + tau) / n;
    if (!same) x2 += 2.0 * (Xp.x * Xp.x + Xp.y * Xp.y) / (np + tau) / n;
    const double bk = lam_inf ? 0.0 : nk / (a.lambda * tau + nk);
    const double bp = lam_inf ? 0.0 : np / (a.lambda * tau + np);
    const double2 Yk = make_double2(bk * Xk.x / n, bk * Xk.y / n);
    const double2 Yp = make_double2(bp * Xp.x / n, bp * Xp.y / n);
    // Z'_k = (Yk + conj Yp) + i conj(w) (Yk - conj Yp); Z'_p = (Yp + conj Yk) - i w (Yp - conj Yk)
    const double2 s1 = make_double2(Yk.x + Yp.x, Yk.y - Yp.y);
    const double2 d1 = zmul(make_double2(Yk.x - Yp.x, Yk.y + Yp.y), make_double2(w.x, -w.y));
    zo[k] = make_double2(s1.x - d1.y, s1.y + d1.x);
    if (!same) {
      const double2 s2 = make_double2(Yp.x + Yk.x, Yp.y - Yk.y);
      const double2 d2 = zmul(w, make_double2(Yp.x - Yk.x, Yp.y + Yk.y));
      zo[kp] = make_double2(s2.x + d2.y, s2.y - d2.x);
    }
  }
  if (a.chi2) {
    for (int o = 16; o > 0; o >>= 1) x2 += __shfl_down_sync(0xffffffffu, x2, o);
    if ((threadIdx.x & 31) == 0 && x2 != 0.0) atomicAdd(a.chi2, x2);
  }
  if (!plain_sync(a)) return;
  // 4. inverse FFT of the filtered spectrum (now in Zo)
  PlainArgs b = a;
  b.buf0 = Zo;
  b.buf1 = Z;
  double2* w = plain_fft(b, +1, &ok);
  if (!ok) return;
  // 5. t = d - irfft(Y); P^T t / tau into FP64 accumulators
  for (int64_t g = tid; g < (int64_t)a.n_chunks * a.M; g += nthreads) {
    const int c = (int)(g / a.M);
    const int j = (int)(g % a.M);
    const ChunkDesc& d = a.desc[c];
    const double2 v = w[g];
    for (int h = 0; h < 2; ++h) {
      const int64_t s = d.off + 2ll * j + h;
      const int p = a.pix[s];
      if (p < 0) continue;
      const double t = ((double)a.tod[s] - (h ? v.y : v.x)) / d.tau;
      if (a.ncomp == 1) {
        atomicAdd(a.acc + p, t);
      } else {
        double* ac = a.acc + 3 * (int64_t)p;
        atomicAdd(ac, t);
        atomicAdd(ac + 1, t * plain_w(a.cosw, a.half_w, s));
        atomicAdd(ac + 2, t * plain_w(a.sinw, a.half_w, s));
      }
    }
  }
  if (!plain_sync(a)) return;
  // 6. m' = W acc per pixel; clear acc
  for (int64_t p = tid; p < a.n_pix; p += nthreads) {
    if (a.ncomp == 1) {
      a.map[p] = a.W[p] * a.acc[p];
      a.acc[p] = 0.0;
    } else {
      const double* Wp = a.W + 6 * p;
      double* ac = a.acc + 3 * p;
      const double x0 = ac[0], x1 = ac[1], x2v = ac[2];
      a.map[3 * p + 0] = Wp[0] * x0 + Wp[1] * x1 + Wp[2] * x2v;
      a.map[3 * p + 1] = Wp[1] * x0 + Wp[3] * x1 + Wp[4] * x2v;
      a.map[3 * p + 2] = Wp[2] * x0 + Wp[4] * x1 + Wp[5] * x2v;
      ac[0] = ac[1] = ac[2] = 0.0;
    }
  }
}

__global__ void k_plain_twiddles(double2* tw, double2* tw2, int M) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > M / 2) return;
  double s, c;
  if (m < M / 2) {
    sincospi(-2.0 * (double)m / (double)M, &s, &c);
    tw[m] = make_double2(c, s);
  }
  sincospi(-(double)m / (double)M, &s, &c);
  tw2[m] = make_double2(c, s);
}

}  // namespace mm

using namespace mm;

static size_t plain_up(size_t x) { return (x + 255) & ~size_t(255); }

extern "C" mm_status mm_plain_work_bytes(mm_plan p, size_t* bytes) {
  if (!p || !bytes) { mm_set_error("mm_plain_work_bytes: NULL argument"); return MM_ERR_ARG; }
  if (p->n_groups != 1 || p->groups[0].general) {
    mm_set_error("the plain FP64 step needs all chunks of one power-of-two length");
    return MM_ERR_UNSUPPORTED;
  }
  const int M = p->groups[0].M;
  const size_t cbytes = sizeof(double2) * (size_t)M * p->n_chunks;
  *bytes = 2 * plain_up(cbytes) + plain_up(sizeof(double2) * (M / 2)) +
           plain_up(sizeof(double2) * (M / 2 + 1)) + 256;
  return MM_OK;
}

extern "C" mm_status mm_messenger_plain_fp64(mm_plan p, const float* tod, const double* lambdas,
                                             int n_iter, double* map_inout, double* chi2_out,
                                             void* work, size_t work_bytes, void* stream) {
  MmRange nvtx_range_("mm_messenger_plain_fp64");
  size_t need = 0;
  mm_status st = mm_plain_work_bytes(p, &need);
  if (st != MM_OK) return st;
  if (!tod || !map_inout || !work || (n_iter > 0 && !lambdas) || n_iter < 0) {
    mm_set_error("mm_messenger_plain_fp64: NULL pointer or negative count");
    return MM_ERR_ARG;
  }
  if (!p->noise_set) { mm_set_error("mm_set_noise_psd has not run"); return MM_ERR_STATE; }
  if (((uintptr_t)work & 255) || work_bytes < need) {
    mm_set_error("mm_messenger_plain_fp64: work must be 256-byte aligned and >= %zu bytes", need);
    return MM_ERR_NOMEM;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const Group& G = p->groups[0];
  const int M = G.M;
  const size_t cbytes = plain_up(sizeof(double2) * (size_t)M * p->n_chunks);
  char* w = static_cast<char*>(work);
  PlainArgs a;
  a.desc = p->d_desc;
  a.n_chunks = p->n_chunks;
  a.M = M;
  a.logM = 0;
  while ((1 << a.logM) < M) ++a.logM;
  a.pix = p->pix;
  a.cosw = p->cosw;
  a.sinw = p->sinw;
  a.half_w = p->wdtype == MM_W_F16;
  a.ncomp = p->ncomp;
  a.tod = tod;
  a.map = map_inout;
  a.W = p->W;
  a.valid = p->valid;
  a.acc = p->acc;
  a.n_pix = p->n_pix;
  a.nbar = p->nbar;
  a.nyq = p->nyq;
  a.M1 = G.M1;
  a.M2 = G.M2;
  a.buf0 = reinterpret_cast<double2*>(w);
  a.buf1 = reinterpret_cast<double2*>(w + cbytes);
  a.tw = reinterpret_cast<const double2*>(w + 2 * cbytes);
  a.tw2 = reinterpret_cast<const double2*>(w + 2 * cbytes + plain_up(sizeof(double2) * (M / 2)));
  a.bar = reinterpret_cast<unsigned*>(w + 2 * cbytes + plain_up(sizeof(double2) * (M / 2)) +
                                      plain_up(sizeof(double2) * (M / 2 + 1)));
  a.err = reinterpret_cast<int*>(a.bar + 2);
  cudaError_t e;
  k_plain_twiddles<<<(M / 2 + 256) / 256, 256, 0, s>>>(const_cast<double2*>(a.tw),
                                                        const_cast<double2*>(a.tw2), M);
  if ((e = cudaGetLastError()) != cudaSuccess) {
    mm_set_error("plain twiddles: %s", cudaGetErrorString(e));
    return MM_ERR_CUDA;
  }
  int dev = 0, nsm = 0, occ = 0;
  const int threads = 256;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_plain_iteration, threads, 0)) !=
          cudaSuccess) {
    mm_set_error("plain occupancy: %s", cudaGetErrorString(e));
    return MM_ERR_CUDA;
  }
  const int grid = (occ < 1 ? 1 : occ) * nsm;
  if ((e = cudaMemsetAsync(a.bar, 0, 16, s)) != cudaSuccess) {   // barrier state and error flag
    mm_set_error("memset: %s", cudaGetErrorString(e));
    return MM_ERR_CUDA;
  }
  if (chi2_out && n_iter > 0) {
    if ((e = cudaMemsetAsync(chi2_out, 0, sizeof(double) * n_iter, s)) != cudaSuccess) {
      mm_set_error("memset: %s", cudaGetErrorString(e));
      return MM_ERR_CUDA;
    }
  }
  for (int it = 0; it < n_iter; ++it) {
    if (!(lambdas[it] >= 1.0 || isinf(lambdas[it]))) {
      mm_set_error("lambdas[%d] must be >= 1 or inf", it);
      return MM_ERR_ARG;
    }
    if ((e = cudaMemsetAsync(a.bar, 0, 8, s)) != cudaSuccess) {   // count, generation
      mm_set_error("memset: %s", cudaGetErrorString(e));
      return MM_ERR_CUDA;
    }
    a.lambda = lambdas[it];
    a.chi2 = chi2_out ? chi2_out + it : nullptr;
    void* args[] = {&a};
    if ((e = cudaLaunchCooperativeKernel((const void*)k_plain_iteration, grid, threads, args, 0, s)) !=
        cudaSuccess) {
      mm_set_error("cooperative launch: %s", cudaGetErrorString(e));
      return MM_ERR_CUDA;
    }
  }
  // a barrier that gave up leaves err set: report it (synchronises the stream)
  int err = 0;
  if ((e = cudaMemcpyAsync(&err, a.err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    mm_set_error("plain step: %s", cudaGetErrorString(e));
    return MM_ERR_CUDA;
  }
  if (err) {
    mm_set_error("plain step: a grid barrier timed out");
    return MM_ERR_TIMEOUT;
  }
  return MM_OK;
}
