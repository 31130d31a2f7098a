// Allocation-free volume sum (mwdg_volume_noalloc in include/mwdg.h).
//
// Some callers cannot call cudaMalloc while they run: a host application
// that hands all device memory to its own pool at start-up and forbids
// further allocation, an embedded or real-time flood-warning loop that must
// not risk an allocation failure or its latency mid-run, or a plug-in that
// only receives buffers from its host.  This entry point serves them.  It
// computes the same deterministic FP64 volume sum as mwdg_get_volume, but
// from caller-provided device arrays and without any allocation: the
// per-block partial sums live in a fixed file-scope device array that every
// GPU loading this library holds until the process exits.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "mwdg.h"

namespace {

constexpr int NA_TPB = 256;
constexpr int NA_PER_THREAD = 16;
constexpr long long NA_CHUNK = (long long)NA_TPB * NA_PER_THREAD;  // leaves per block
constexpr int NA_SCRATCH = 16384;                                   // partial sums (128 KB)
constexpr int NA_MAX_DEVICES = 64;

// Scratch shared by every call on a device: per-block partial sums.  Each
// call overwrites the entries it reads, so nothing needs clearing; calls
// whose work overlaps on the GPU race on this array.
static __device__ __align__(256) double g_na_part[NA_SCRATCH];
// set when a leaf's level lies outside 0..L; cleared at the start of each call
static __device__ int g_na_bad;

// device address of g_na_part per device, looked up once per device
double *g_na_ptr[NA_MAX_DEVICES] = {};
std::mutex g_na_mu;

__global__ void k_na_clear() { g_na_bad = 0; }

__global__ void k_na_part(const double *h0, const int32_t *level, long long n, double dx, int L,
                          double *part) {
  __shared__ double sh[NA_TPB];
  const long long base = (long long)blockIdx.x * NA_CHUNK;
  double acc = 0.0;
  for (int q = 0; q < NA_PER_THREAD; q++) {
    long long k = base + (long long)q * NA_TPB + threadIdx.x;
    if (k < n) {
      const int lv = level[k];
      if (lv < 0 || lv > L) {  // not a level of this hierarchy: the call fails
        g_na_bad = 1;
        continue;
      }
      double side = dx * (double)(1LL << (L - lv));
      acc += h0[k] * (side * side);
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = NA_TPB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_na_final(const double *part, int nb, double *out) {
  __shared__ double sh[NA_TPB];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += NA_TPB) acc += part[b];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = NA_TPB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = g_na_bad ? __longlong_as_double(0x7ff8000000000000LL) : sh[0];
}

// once per device, with that device current: the device address of the
// scratch array (a host-side use of the symbol itself would not be it)
mwdg_status scratch_for_current_device(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return MWDG_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    double *ptr = nullptr;
    if (cudaGetSymbolAddress((void **)&ptr, g_na_part) != cudaSuccess || !ptr) return MWDG_ERR_CUDA;
    g_na_ptr[dev] = ptr;
  }
  *out = g_na_ptr[dev];
  return MWDG_OK;
}

}  // namespace

extern "C" mwdg_status mwdg_volume_noalloc(const double *h0, const int32_t *level, int64_t n, double dx,
                                           int32_t L, double *volume, void *cuda_stream) {
  if (!volume || n < 0 || (n > 0 && (!h0 || !level)) || !(dx > 0.0) || L < 0 || L > MWDG_LMAX)
    return MWDG_ERR_ARG;
  if (n > MWDG_VOLUME_NOALLOC_MAX) return MWDG_ERR_CAPACITY;
  // an error left pending by earlier work of the caller or another library
  // is not this call's: it is reported as MWDG_ERR_CUDA and left in place
  // for its owner
  if (cudaPeekAtLastError() != cudaSuccess) return MWDG_ERR_CUDA;
  double *part = nullptr;
  mwdg_status s = scratch_for_current_device(&part);
  if (s != MWDG_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nb = (int)((n + NA_CHUNK - 1) / NA_CHUNK);
  k_na_clear<<<1, 1, 0, st>>>();
  if (nb > 0) k_na_part<<<nb, NA_TPB, 0, st>>>(h0, level, (long long)n, dx, L, part);
  k_na_final<<<1, NA_TPB, 0, st>>>(part, nb, volume);
  if (cudaPeekAtLastError() != cudaSuccess) {
    (void)cudaGetLastError();  // this call's own launch error
    return MWDG_ERR_CUDA;
  }
  // the level check: wait for this call's work and read its flag (into host
  // stack memory; nothing is allocated)
  int bad = 0;
  if (cudaMemcpyFromSymbolAsync(&bad, g_na_bad, sizeof bad, 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    (void)cudaGetLastError();
    return MWDG_ERR_CUDA;
  }
  return bad ? MWDG_ERR_ARG : MWDG_OK;
}

static_assert(MWDG_VOLUME_NOALLOC_MAX <= (long long)NA_SCRATCH * NA_CHUNK, "scratch too small");
