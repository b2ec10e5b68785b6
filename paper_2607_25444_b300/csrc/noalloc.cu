// noalloc.cu -- the volume correction of a phase field that the caller owns,
// run without allocating any device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is
// already handed to another allocator's pool, a host that forbids device
// allocation once it is serving, or code that must not risk the implicit
// device synchronisation that cudaFree performs. For them this file keeps
// the reduction scratch of the correction in a fixed array compiled into
// the library (g_noalloc_scratch, 256 KiB, on every GPU that loads the
// library, until the process exits). The caller passes the phase field
// (corrected in place), the occupancy and an optional output; nothing else
// is allocated.
//
// The arithmetic is that of the context's correction: M* = sum of phi over
// fluid nodes, W = sum of chi(phi) with chi = phi (1 - phi) inside
// (eps, 1 - eps), lambda = (M_ref - M*)/W (0 when W = 0), and
// phi += lambda chi(phi) at fluid nodes. Sums are FP64, in a fixed order.
// The update is rounded without bias, as in the context's correction: a
// correction below the FP32 resolution of phi is applied on average instead
// of being rounded away at every call. The rounding key is a call counter
// the library keeps in the scratch array (it starts at zero when the
// library is loaded and advances by one per call on that device).
#include <mutex>

#include "cacl_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_THREAD = 16;
constexpr int NA_NODES_PER_BLOCK = NA_THREADS * NA_PER_THREAD;  // 4096
constexpr int NA_MAX_BLOCKS = 16384;
constexpr int64_t NA_MAX_NODES = (int64_t)NA_MAX_BLOCKS * NA_NODES_PER_BLOCK;
constexpr int NA_FIN_THREADS = 1024;

// [0, MAX): block sums of phi; [MAX, 2 MAX): block sums of chi;
// [2 MAX, 2 MAX + 3): M*, W, lambda of the last call; [2 MAX + 3]: the
// call counter (the rounding key of the unbiased update), as 64-bit bits.
static __device__ __align__(256) double g_noalloc_scratch[2 * NA_MAX_BLOCKS + 8];

std::mutex g_setup_mu;
double* g_scratch_ptr[64] = {};

// Device address of the scratch array on the current device, looked up once
// per device. Host code must not use the symbol's name as an address.
cudaError_t scratch_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

__device__ __forceinline__ float band_weight(float v, float eps) {
  return (v > eps && v < 1.0f - eps) ? v * (1.0f - v) : 0.0f;
}

__global__ void __launch_bounds__(NA_THREADS)
noalloc_partials(const float* __restrict__ phi, const uint8_t* __restrict__ solid,
                 int64_t n, float eps, double* __restrict__ scratch) {
  __shared__ double sm[NA_THREADS], sw[NA_THREADS];
  const int64_t base = (int64_t)blockIdx.x * NA_NODES_PER_BLOCK;
  double m = 0.0, w = 0.0;
  for (int j = 0; j < NA_PER_THREAD; ++j) {
    const int64_t i = base + (int64_t)j * NA_THREADS + threadIdx.x;
    if (i < n && !solid[i]) {
      const float v = phi[i];
      m += (double)v;
      w += (double)band_weight(v, eps);
    }
  }
  sm[threadIdx.x] = m;
  sw[threadIdx.x] = w;
  __syncthreads();
  for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sm[threadIdx.x] += sm[threadIdx.x + s];
      sw[threadIdx.x] += sw[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scratch[blockIdx.x] = sm[0];
    scratch[NA_MAX_BLOCKS + blockIdx.x] = sw[0];
  }
}

__global__ void __launch_bounds__(NA_FIN_THREADS)
noalloc_finalize(double* __restrict__ scratch, int nb, double m_ref,
                 double* __restrict__ out) {
  __shared__ double sm[NA_FIN_THREADS], sw[NA_FIN_THREADS];
  double m = 0.0, w = 0.0;
  for (int i = threadIdx.x; i < nb; i += NA_FIN_THREADS) {
    m += scratch[i];
    w += scratch[NA_MAX_BLOCKS + i];
  }
  sm[threadIdx.x] = m;
  sw[threadIdx.x] = w;
  __syncthreads();
  for (int s = NA_FIN_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sm[threadIdx.x] += sm[threadIdx.x + s];
      sw[threadIdx.x] += sw[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double lam = (sw[0] > 0.0) ? (m_ref - sm[0]) / sw[0] : 0.0;
    scratch[2 * NA_MAX_BLOCKS + 0] = sm[0];
    scratch[2 * NA_MAX_BLOCKS + 1] = sw[0];
    scratch[2 * NA_MAX_BLOCKS + 2] = lam;
    uint64_t* calls = reinterpret_cast<uint64_t*>(scratch + 2 * NA_MAX_BLOCKS + 3);
    *calls += 1;
    if (out) {
      out[0] = sm[0];
      out[1] = sw[0];
      out[2] = lam;
    }
  }
}

__global__ void __launch_bounds__(NA_THREADS)
noalloc_apply(float* __restrict__ phi, const uint8_t* __restrict__ solid,
              int64_t n, float eps, const double* __restrict__ scratch) {
  const float lam = (float)scratch[2 * NA_MAX_BLOCKS + 2];
  const uint32_t key = (uint32_t)*reinterpret_cast<const uint64_t*>(
      scratch + 2 * NA_MAX_BLOCKS + 3);
  const int64_t i = (int64_t)blockIdx.x * NA_THREADS + threadIdx.x;
  if (i >= n || solid[i]) return;
  const float v = phi[i];
  phi[i] = cacl::add_unbiased(v, lam * band_weight(v, eps), key, (uint64_t)i);
}

}  // namespace

extern "C" cacl_status cacl_volume_correct_noalloc(float* phi,
                                                   const uint8_t* solid,
                                                   int64_t n, double m_ref,
                                                   double eps_phi, double* out,
                                                   void* stream) {
  if (!phi || !solid || n < 1) return CACL_ERR_ARG;
  if (!(eps_phi > 0.0 && eps_phi < 0.5)) return CACL_ERR_ARG;
  if (n > NA_MAX_NODES) return CACL_ERR_TOO_LARGE;
  // phi, solid and out must live on the current device: the scratch array
  // used below is that device's copy
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CACL_ERR_CUDA;
  const void* ptrs[3] = {phi, solid, out};
  for (const void* q : ptrs) {
    if (!q) continue;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
      cudaGetLastError();  // clear the error this query recorded
      return CACL_ERR_ARG;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
      return CACL_ERR_ARG;
    if (at.device != dev) return CACL_ERR_ARG;
  }
  double* scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) return CACL_ERR_CUDA;
  // clear a non-sticky error left by earlier unrelated work, so that the
  // check after the launches reports these launches only
  cudaGetLastError();
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = (int)((n + NA_NODES_PER_BLOCK - 1) / NA_NODES_PER_BLOCK);
  const float eps = (float)eps_phi;
  noalloc_partials<<<nb, NA_THREADS, 0, st>>>(phi, solid, n, eps, scratch);
  noalloc_finalize<<<1, NA_FIN_THREADS, 0, st>>>(scratch, nb, m_ref, out);
  const int ne = (int)((n + NA_THREADS - 1) / NA_THREADS);
  noalloc_apply<<<ne, NA_THREADS, 0, st>>>(phi, solid, n, eps, scratch);
  return cudaGetLastError() == cudaSuccess ? CACL_OK : CACL_ERR_CUDA;
}
