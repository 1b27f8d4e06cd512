// Allocation-free direct banded solve.
//
// Some callers cannot call cudaMalloc: cudaMalloc may synchronise the
// device, which latency-critical loops cannot afford, and some host
// programs own all device memory themselves and forbid new driver
// allocations.  sap_band_solve_noalloc serves them: it runs the same
// kernels as sap_factor (P = 1, SaP-D) followed by
// sap_apply_preconditioner, i.e. one banded LU without pivoting (boosted
// pivots) and its two triangular sweeps, but keeps every intermediate
// (factor array, sweep intermediate, partition descriptor, boost
// threshold, counters) in one file-scope device array instead of
// allocating.  Its header words are written by a one-thread kernel, so the
// call copies nothing from host memory.  The array is kScratchBytes large and
// lives on every GPU that loads the library until the process exits.
#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>
#include <mutex>
#include "sap_internal.cuh"

using namespace sap;

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device; host code may not use the symbol itself as an address).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = p;
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// The call's header words, written on the device so that the call copies
// nothing from host memory: the one-block partition descriptor
// {off[0], off[1], fbase, ld, cbase} = {0, N, 0, ld, 0}, the boosted-pivot
// counter, and the wait error word {flag, polls} of the bounded waits.
__global__ void k_noalloc_header(int64_t* desc, int64_t N, int64_t ld, unsigned long long* nb, int* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  desc[0] = 0;
  desc[1] = N;
  desc[2] = 0;
  desc[3] = ld;
  desc[4] = 0;
  *nb = 0ull;
  err[0] = 0;
  err[1] = kDefaultSpin;
}

// Copies the wait error flag into the caller's word (1 = a bounded wait gave up).
__global__ void k_noalloc_status(const int* err, int32_t* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = err[0] != 0 ? 1 : 0;
}

template <typename T>
sap_status_t run(const double* band, int64_t N, int K, const double* b, double* x, int32_t* timeout_dev,
                 cudaStream_t s) {
  const int W = 2 * K + 1;
  const int64_t ld = (N + 31) / 32 * 32;
  // scratch layout: header | factors | chunk matrices (L, U sweeps) | sweep scratch
  const size_t hdr = 256;
  const size_t f_bytes = align256((size_t)ld * W * sizeof(T));
  const size_t c_elems = (size_t)(ld / 32) * (1 + chunk_couplings(K)) * 32 * 32;
  const size_t c_bytes = align256(c_elems * sizeof(T));
  const size_t a_bytes = align256((size_t)(2 * N + 2 * K + 8) * sizeof(double));
  const size_t b_bytes = sizeof(T) == 4 ? align256((size_t)N * W * sizeof(float)) : 0;   // FP32 band copy
  const bool gw = lu_window_global(K, sizeof(T) == 8);                                   // factor window
  const size_t w_bytes = gw ? align256(lu_window_elems(K) * sizeof(T)) : 0;
  if (hdr + f_bytes + 2 * c_bytes + a_bytes + b_bytes + w_bytes > kScratchBytes) return SAP_ERR_INVALID_ARG;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return SAP_ERR_CUDA;
  unsigned char* p = static_cast<unsigned char*>(base);
  int64_t* desc = reinterpret_cast<int64_t*>(p);        // off[2], fbase[1], ld[1], cbase[1]
  double* absmax = reinterpret_cast<double*>(p + 64);
  unsigned long long* nb = reinterpret_cast<unsigned long long*>(p + 128);
  int* err = reinterpret_cast<int*>(p + 192);          // int[2]
  T* F = reinterpret_cast<T*>(p + hdr);
  T* Mlf = reinterpret_cast<T*>(p + hdr + f_bytes);
  T* Mub = reinterpret_cast<T*>(p + hdr + f_bytes + c_bytes);
  double* ascratch = reinterpret_cast<double*>(p + hdr + f_bytes + 2 * c_bytes);
  float* bandf = reinterpret_cast<float*>(p + hdr + f_bytes + 2 * c_bytes + a_bytes);
  T* wlu = gw ? reinterpret_cast<T*>(p + hdr + f_bytes + 2 * c_bytes + a_bytes + b_bytes) : nullptr;
  // descriptor and counters (the previous call's values are overwritten);
  // factor padding columns are read as zeros by the sweeps
  count_launches(1);
  k_noalloc_header<<<1, 32, 0, s>>>(desc, N, ld, nb, err);
  if (cudaGetLastError() != cudaSuccess) return SAP_ERR_CUDA;
  if (cudaMemsetAsync(F, 0, (size_t)ld * W * sizeof(T), s) != cudaSuccess) return SAP_ERR_CUDA;
  Dev d{desc, desc + 2, desc + 3};
  const double eps = sizeof(T) == 8 ? 0x1p-53 : 0x1p-24;
  const T* bandT;
  if (sizeof(T) == 4) {
    if (launch_absmax_cast(band, N, K, absmax, bandf, s) != cudaSuccess) return SAP_ERR_CUDA;
    bandT = reinterpret_cast<const T*>(bandf);
  } else {
    if (launch_absmax(band, N, K, absmax, s) != cudaSuccess) return SAP_ERR_CUDA;
    bandT = reinterpret_cast<const T*>(band);
  }
  if (launch_factor_lu<T>(bandT, N, K, 1, d, absmax, eps, F, nb, wlu, false, err, s) != cudaSuccess) return SAP_ERR_CUDA;
  const int64_t* cbase = desc + 4;
  if (launch_chunk_mats<T>(F, K, 1, d, cbase, (int)(ld / 32), 0, Mlf, s) != cudaSuccess) return SAP_ERR_CUDA;
  if (launch_chunk_mats<T>(F, K, 1, d, cbase, (int)(ld / 32), 1, Mub, s) != cudaSuccess) return SAP_ERR_CUDA;
  Factors<T> f;
  f.F = F;
  f.Mlf = Mlf;
  f.Mub = Mub;
  f.cbase = cbase;
  f.err = err;
  if (launch_apply<T>(band, N, K, 1, d, f, SAP_D, false, b, x, ascratch, s) != cudaSuccess) return SAP_ERR_CUDA;
  if (timeout_dev) {
    count_launches(1);
    k_noalloc_status<<<1, 32, 0, s>>>(err, timeout_dev);
    if (cudaGetLastError() != cudaSuccess) return SAP_ERR_CUDA;
  }
  return SAP_OK;
}

}  // namespace

extern "C" sap_status_t sap_band_solve_noalloc(const double* band_dev, int64_t N, int32_t K, const double* b_dev,
                                               double* x_dev, int32_t precision, int32_t* timeout_dev,
                                               cudaStream_t stream) {
  if (!band_dev || !b_dev || !x_dev || b_dev == x_dev) return SAP_ERR_INVALID_ARG;
  if (N < 2 || K < 1 || K >= N) return SAP_ERR_INVALID_ARG;
  if (precision != SAP_FP64 && precision != SAP_FP32) return SAP_ERR_INVALID_ARG;
  if (K > sap_max_K(precision)) return SAP_ERR_NOT_IMPLEMENTED;
  return precision == SAP_FP64 ? run<double>(band_dev, N, K, b_dev, x_dev, timeout_dev, stream)
                               : run<float>(band_dev, N, K, b_dev, x_dev, timeout_dev, stream);
}
