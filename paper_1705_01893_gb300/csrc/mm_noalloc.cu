// Binned map without any allocation: m = (P^T P)^-1 P^T d per pixel, with its FP64
// accumulators in a fixed, file-scope device array instead of caller- or library-allocated
// memory.  For callers that cannot allocate device memory at all -- code running inside a
// CUDA graph capture, under an allocator that must not grow, or in a host process that
// only receives device pointers from elsewhere -- and still want the binned map.
#include <mutex>

#include "mm_internal.cuh"

namespace {

// Scratch: for every pixel 6 entries of the symmetric 3x3 block P^T P (upper triangle
// 00 01 02 11 12 22) and 3 entries of P^T d (T-only maps use 2 of the 9).  The array lives
// in every GPU that loads the library, until the process exits.
constexpr int64_t kNoallocMaxPix = int64_t(1) << 18;
constexpr int kNoallocPerPix = 9;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocMaxPix * kNoallocPerPix];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

// The device address of the scratch on the current device.  Outside stream capture it is
// looked up on every call (a host-side query once the module is loaded), so a context that
// was reset and re-created, which may load the module at another address, is followed;
// during capture the address of the last lookup on this device is used, which is why the
// first call on a device must come before any capture.
cudaError_t noalloc_scratch(cudaStream_t s, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  } else if (!g_noalloc_ptr[dev]) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

__global__ void k_noalloc_clear(double* s, int64_t len) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    s[i] = 0.0;
}

__global__ void k_noalloc_accum(const int32_t* __restrict__ pix, const void* cosw, const void* sinw,
                                int half_w, const float* __restrict__ tod, int64_t n,
                                int64_t n_pix, int ncomp, double* __restrict__ s) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = pix[i];
  if (p < 0 || p >= n_pix) return;   // excluded sample (or an index outside the map)
  const double d = (double)tod[i];
  double* a = s + (int64_t)p * kNoallocPerPix;
  if (ncomp == 1) {
    atomicAdd(a, 1.0);
    atomicAdd(a + 1, d);
    return;
  }
  double c, w;
  if (half_w) {
    c = __half2float(static_cast<const __half*>(cosw)[i]);
    w = __half2float(static_cast<const __half*>(sinw)[i]);
  } else {
    c = static_cast<const float*>(cosw)[i];
    w = static_cast<const float*>(sinw)[i];
  }
  atomicAdd(a + 0, 1.0);
  atomicAdd(a + 1, c);
  atomicAdd(a + 2, w);
  atomicAdd(a + 3, c * c);
  atomicAdd(a + 4, c * w);
  atomicAdd(a + 5, w * w);
  atomicAdd(a + 6, d);
  atomicAdd(a + 7, c * d);
  atomicAdd(a + 8, w * d);
}

// Extreme eigenvalues of a symmetric 3x3 block (trigonometric closed form, Smith 1961).
__device__ void noalloc_eig(const double* m, double* emin, double* emax) {
  const double a00 = m[0], a01 = m[1], a02 = m[2], a11 = m[3], a12 = m[4], a22 = m[5];
  const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
  const double q = (a00 + a11 + a22) / 3.0;
  const double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
  const double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * p1;
  if (p2 <= 0.0) { *emin = *emax = q; return; }
  const double pp = sqrt(p2 / 6.0);
  const double det = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) +
                     a02 * (a01 * a12 - b11 * a02);
  const double r = fmin(1.0, fmax(-1.0, det / (2.0 * pp * pp * pp)));
  const double phi = acos(r) / 3.0;
  *emax = q + 2.0 * pp * cos(phi);
  *emin = q + 2.0 * pp * cos(phi + 2.0943951023931954923);
}

// Per pixel: keep it iff it has a hit and (IQU) eigmin/eigmax >= rcond_min; solve the block.
__global__ void k_noalloc_solve(const double* __restrict__ s, int64_t n_pix, int ncomp,
                                double rcond_min, double* __restrict__ map) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  const double* a = s + p * kNoallocPerPix;
  if (ncomp == 1) {
    map[p] = a[0] > 0.0 ? a[1] / a[0] : 0.0;
    return;
  }
  double* o = map + 3 * p;
  o[0] = o[1] = o[2] = 0.0;
  if (!(a[0] > 0.0)) return;
  double emin, emax;
  noalloc_eig(a, &emin, &emax);
  if (!(emax > 0.0) || emin / emax < rcond_min) return;
  const double A = a[0], B = a[1], C = a[2], D = a[3], E = a[4], F = a[5];
  const double c00 = D * F - E * E, c01 = C * E - B * F, c02 = B * E - C * D;
  const double det = A * c00 + B * c01 + C * c02;
  if (!(det > 0.0) && !(det < 0.0)) return;
  const double c11 = A * F - C * C, c12 = B * C - A * E, c22 = A * D - B * B;
  const double b0 = a[6], b1 = a[7], b2 = a[8];
  o[0] = (c00 * b0 + c01 * b1 + c02 * b2) / det;
  o[1] = (c01 * b0 + c11 * b1 + c12 * b2) / det;
  o[2] = (c02 * b0 + c12 * b1 + c22 * b2) / det;
}

}  // namespace

extern "C" mm_status mm_binned_map_noalloc(const int32_t* pix, const void* cos2psi,
                                           const void* sin2psi, int weight_dtype,
                                           const float* tod, int64_t n, int64_t n_pix,
                                           int ncomp, double rcond_min, double* map_out,
                                           void* stream) {
  if (!pix || !tod || !map_out || n < 0) {
    mm_set_error("mm_binned_map_noalloc: NULL pointer or negative sample count");
    return MM_ERR_ARG;
  }
  if (ncomp != 1 && ncomp != 3) {
    mm_set_error("mm_binned_map_noalloc: ncomp must be 1 or 3 (got %d)", ncomp);
    return MM_ERR_ARG;
  }
  if ((ncomp == 3) != (cos2psi != nullptr && sin2psi != nullptr)) {
    mm_set_error("mm_binned_map_noalloc: cos2psi/sin2psi must be given iff ncomp == 3");
    return MM_ERR_ARG;
  }
  if (weight_dtype != MM_W_F32 && weight_dtype != MM_W_F16) {
    mm_set_error("mm_binned_map_noalloc: bad weight_dtype %d", weight_dtype);
    return MM_ERR_ARG;
  }
  if (!(rcond_min >= 0.0 && rcond_min <= 1.0)) {   // also rejects NaN
    mm_set_error("mm_binned_map_noalloc: rcond_min must be in [0, 1]");
    return MM_ERR_ARG;
  }
  if (n_pix < 1 || n_pix > kNoallocMaxPix) {
    mm_set_error("mm_binned_map_noalloc: n_pix = %lld outside [1, %lld], the size of its "
                 "fixed scratch", (long long)n_pix, (long long)kNoallocMaxPix);
    return MM_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  cudaError_t e = noalloc_scratch(s, &scratch);
  if (e != cudaSuccess) {
    mm_set_error("mm_binned_map_noalloc: scratch address lookup failed: %s (the first call on "
                 "a device must come before any stream capture)", cudaGetErrorString(e));
    return MM_ERR_CUDA;
  }
  const int64_t len = n_pix * kNoallocPerPix;   // the previous call's contents are cleared
  k_noalloc_clear<<<(unsigned)((len + 255) / 256 < 4096 ? (len + 255) / 256 : 4096), 256, 0, s>>>(
      scratch, len);
  if (n > 0)
    k_noalloc_accum<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        pix, cos2psi, sin2psi, weight_dtype == MM_W_F16, tod, n, n_pix, ncomp, scratch);
  k_noalloc_solve<<<(unsigned)((n_pix + 255) / 256), 256, 0, s>>>(scratch, n_pix, ncomp,
                                                                  rcond_min, map_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    mm_set_error("mm_binned_map_noalloc: launch failed: %s", cudaGetErrorString(e));
    return MM_ERR_CUDA;
  }
  return MM_OK;
}
