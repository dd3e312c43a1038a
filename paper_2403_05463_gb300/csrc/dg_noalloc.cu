// dg_noalloc.cu -- conservation sums that allocate nothing.
//
// dg_conservation keeps a library-owned buffer of per-element partial sums (allocated with the
// mesh) and finishes the sum on the host. The variant here is for callers that must not
// allocate device memory or copy to the host while they run: a serving loop whose memory pool
// has already reserved the device, or a time-critical loop in which a cudaMalloc or cudaFree
// would synchronise the whole device. Its partial sums go to one file-scope device array that
// the module carries from load time, the final sums are reduced on the device in a fixed order,
// and the result lands in caller-owned device memory.
//
// Every call in one process on one device shares that array, whatever mesh it is for: two
// calls whose kernels overlap on the GPU (different streams, or different host threads)
// overwrite each other's partial sums. Nothing in the array has to start at zero: each call
// writes every partial sum (4 per element) before its final reduction reads them.
#include <mutex>

#include "dg_device.cuh"

namespace dgk {

// 4 variables x kNoAllocMaxElems elements, 2 MiB.
static __device__ __align__(256) double g_noalloc_partial[4 * kNoAllocMaxElems];

namespace {

constexpr int kMaxDevices = 64;
constexpr int kSumThreads = 256;

std::mutex g_setup_mutex;
double* g_scratch[kMaxDevices] = {};  // device address of g_noalloc_partial, per device

// Block v sums partial[v][0..ne): each thread a strided run in element order, then a pairwise
// tree in shared memory. The order is fixed, so repeated calls give identical sums.
__global__ void k_conservation_final(const double* __restrict__ partial, int64_t ne, double* out) {
  __shared__ double s[kSumThreads];
  const int v = blockIdx.x, t = threadIdx.x;
  double a = 0.0;
  for (int64_t e = t; e < ne; e += kSumThreads) a += partial[v * ne + e];
  s[t] = a;
  __syncthreads();
  for (int h = kSumThreads / 2; h > 0; h >>= 1) {
    if (t < h) s[t] += s[t + h];
    __syncthreads();
  }
  if (t == 0) out[v] = s[0];
}

}  // namespace

// Set-up, once per device, with that device current: look up the device address of the
// scratch array. The lookup can load this module onto the device, which is why the first call
// on a device belongs before any stream capture.
cudaError_t noalloc_scratch(int device, double** ptr) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch[device]) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_partial);
    if (e != cudaSuccess) return e;
    g_scratch[device] = p;
  }
  *ptr = g_scratch[device];
  return cudaSuccess;
}

cudaError_t launch_conservation_noalloc(const DevMesh& M, const Bucket* buckets, int n_buckets, const double* R,
                                        double* scratch, double* out, cudaStream_t s) {
  if (M.n_elem > kNoAllocMaxElems) return cudaErrorInvalidValue;
  // the per-element weighted sums are those of dg_conservation (one kernel, k_conservation),
  // written to the static scratch instead of the context's buffer
  for (int i = 0; i < n_buckets; ++i) {
    const cudaError_t e = launch_conservation(M, buckets[i], R, 4, scratch, s);
    if (e != cudaSuccess) return e;
  }
  k_conservation_final<<<4, kSumThreads, 0, s>>>(scratch, M.n_elem, out);
  return cudaGetLastError();
}

}  // namespace dgk
