// hope_noalloc.cu -- hope_total_mass_noalloc: the FP64 mass diagnostic for callers
// that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the diagnostic:
// host code embedded in a framework whose device-memory budget is fixed after start-up
// and which owns every allocation, a monitor thread that must never change the
// device's allocation state, or a time-stepping loop that cannot afford the
// device-wide synchronisation an allocation may cause.  This entry point needs no context (creating one
// allocates tables) and no per-call allocation: the per-block partial sums live in the
// file-scope device array below, which every GPU that loads the library holds
// (32 KiB) until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "hope_internal.h"

namespace hope {

constexpr int NOALLOC_MASS_PARTIALS = HOPE_NOALLOC_MASS_PARTIALS;  // 4096 doubles = 32 KiB
constexpr int NOALLOC_MASS_CHUNK = HOPE_NOALLOC_MASS_CHUNK;        // elements per partial
constexpr int NOALLOC_THREADS = 256;

static __device__ __align__(256) double g_noalloc_mass_partials[NOALLOC_MASS_PARTIALS];

// Device address of g_noalloc_mass_partials per device, looked up once per device.
static std::mutex g_noalloc_mutex;
static double *g_noalloc_ptr[256] = {nullptr};

template <typename T>
__global__ void __launch_bounds__(NOALLOC_THREADS)
    k_mass_partial_noalloc(const T *__restrict__ q, long long n, double *__restrict__ partials) {
  __shared__ double red[NOALLOC_THREADS];
  long long b = (long long)blockIdx.x * NOALLOC_MASS_CHUNK;
  long long e = b + NOALLOC_MASS_CHUNK < n ? b + NOALLOC_MASS_CHUNK : n;
  double s = 0.0;
  for (long long t = b + threadIdx.x; t < e; t += NOALLOC_THREADS) s += (double)q[t];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = NOALLOC_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];  // every used slot is written here
}

__global__ void k_mass_final_noalloc(const double *__restrict__ partials, int nparts, double scale,
                                     double *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += partials[b];  // fixed order: reproducible
    *out = s * scale;
  }
}

}  // namespace hope

using namespace hope;

extern "C" int hope_total_mass_noalloc(const void *q_dev, int precision, int N, double *mass_dev,
                                       hope_stream_t stream) {
  if (!q_dev || !mass_dev || (precision != HOPE_FP64 && precision != HOPE_FP32) || N < 1) {
    set_error("hope_total_mass_noalloc: invalid argument");
    return HOPE_EINVAL;
  }
  const long long n = 6LL * N * N;
  const long long nparts = (n + NOALLOC_MASS_CHUNK - 1) / NOALLOC_MASS_CHUNK;
  if (nparts > NOALLOC_MASS_PARTIALS) {
    set_error("hope_total_mass_noalloc: N = " + std::to_string(N) + " needs " + std::to_string(nparts) +
              " partial sums, more than the " + std::to_string(NOALLOC_MASS_PARTIALS) +
              " of the static scratch (largest N is " + std::to_string(HOPE_NOALLOC_MASS_MAX_N) + ")");
    return HOPE_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256) {
    set_error(std::string("hope_total_mass_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return HOPE_ECUDA;
  }
  double *partials = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      // Set-up on the first call on this device (with it current): the host-side name
      // g_noalloc_mass_partials is only a stand-in; the kernel needs the device address.
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_mass_partials);
      if (e != cudaSuccess || !p) {
        set_error(std::string("hope_total_mass_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return HOPE_ECUDA;
      }
      g_noalloc_ptr[dev] = (double *)p;
    }
    partials = g_noalloc_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const double dx = 3.14159265358979323846 / (2.0 * N);
  if (precision == HOPE_FP64)
    k_mass_partial_noalloc<double><<<(unsigned)nparts, NOALLOC_THREADS, 0, st>>>((const double *)q_dev, n,
                                                                                partials);
  else
    k_mass_partial_noalloc<float><<<(unsigned)nparts, NOALLOC_THREADS, 0, st>>>((const float *)q_dev, n,
                                                                               partials);
  k_mass_final_noalloc<<<1, 32, 0, st>>>(partials, (int)nparts, dx * dx, mass_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("hope_total_mass_noalloc: launch: ") + cudaGetErrorString(e));
    return HOPE_ECUDA;
  }
  return HOPE_OK;
}
