// noalloc.cu -- projection entry point for callers that cannot allocate.
//
// pca_project needs a caller-provided workspace for two small intermediates:
// the FP32 copies of the band means and of the first k eigenvectors that the
// projection kernel streams the cube against.  Some callers have no way to
// provide one: code that runs while a CUDA graph is being captured (where an
// allocation would be recorded or would fail), a plug-in inside a host
// application that owns the device allocator and exposes only tensors, or a
// real-time loop that must never block in an allocator.  pca_project_noalloc
// keeps those intermediates in a fixed array in device memory that belongs
// to this library instead, so it neither allocates nor needs a workspace.
//
// The array holds kNoAllocFloats = 8,448 floats (33,792 bytes: B + B*k for
// 256 bands and 32 components, or fewer bands with more components) and stays
// allocated on every GPU that loads the library until the process exits.  All calls share it, and each call
// rewrites every entry it reads before reading it, so nothing has to start
// at zero -- but two calls whose work overlaps on the GPU (different streams,
// or different host threads) race on it and must be serialised by the caller.
#include <mutex>

#include "common.cuh"

namespace gbpca {
namespace {

constexpr int kNoAllocFloats = 256 + 256 * 32;
constexpr int kMaxDevices = 64;

// File-scope device array.  In host code its name is only a host-side handle
// for the symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
cudaError_t noalloc_scratch(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace gbpca

using namespace gbpca;

extern "C" int pca_project_noalloc(const void* cube, pca_dtype dtype, int64_t N, int B, int k,
                                   const double* mu, const double* eigvecs, float* proj,
                                   void* stream) {
  if (!cube || !mu || !eigvecs || !proj) return PCA_ERR_ARG;
  if (dtype != PCA_F32 && dtype != PCA_BF16 && dtype != PCA_F16) return PCA_ERR_ARG;
  if (N < 1 || B < 2 || B > kMaxB || k < 1 || k > B) return PCA_ERR_ARG;
  if (((uintptr_t)cube) % 16 != 0) return PCA_ERR_ARG;
  if ((int64_t)B + (int64_t)B * k > kNoAllocFloats) return PCA_ERR_ARG;  // beyond the array
  float* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) return PCA_ERR_CUDA;
  float* mu_f = scratch;       // [B]
  float* vk = scratch + B;     // [B][k]
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (launch_narrow_inputs(mu, eigvecs, B, k, mu_f, vk, st) != cudaSuccess) return PCA_ERR_CUDA;
  if (launch_project(cube, dtype, N, B, k, mu_f, vk, proj, st) != cudaSuccess) return PCA_ERR_CUDA;
  return PCA_OK;
}
