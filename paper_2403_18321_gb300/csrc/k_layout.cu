// k_layout.cu -- band-sequential (BSQ) input: the paper's GPU code keeps each
// band contiguous (Sec. 4.2, data initialisation: image[b*PIXELS + n]); the
// fit reads pixel-major cubes (band interleaved by pixel, the manycore layout
// of Sec. 5).  pca_bsq_to_bip transposes one into the other: 32-band x
// 128-pixel tiles staged in shared memory, read along pixels and written along
// bands, so both sides move whole 32-byte sectors, 16 independent loads in
// flight per thread; one read and one write of the cube (HBM-bound).
#include "common.cuh"

namespace gbpca {
namespace {

constexpr int kTb = 32;   // bands per tile
constexpr int kTp = 128;  // pixels per tile

template <typename T>
__global__ void __launch_bounds__(256)
k_bsq_to_bip(const T* __restrict__ bsq, int64_t N, int B, T* __restrict__ bip) {
  __shared__ T tile[kTb][kTp + 1];
  const int64_t p0 = (int64_t)blockIdx.x * kTp;
  const int b0 = blockIdx.y * kTb;
  const int tx = threadIdx.x & 127, ty = threadIdx.x >> 7;  // 128 x 2
#pragma unroll
  for (int b = ty; b < kTb; b += 2) {
    const int64_t p = p0 + tx;
    if (b0 + b < B && p < N) tile[b][tx] = bsq[(int64_t)(b0 + b) * N + p];
  }
  __syncthreads();
  const int lb = threadIdx.x & 31, lp = threadIdx.x >> 5;  // 32 x 8
#pragma unroll
  for (int p = lp; p < kTp; p += 8) {
    const int64_t n = p0 + p;
    if (b0 + lb < B && n < N) bip[n * B + b0 + lb] = tile[lb][p];
  }
}

template <typename T>
cudaError_t bsq_to_bip(const void* bsq, int64_t N, int B, void* bip, cudaStream_t st) {
  const dim3 grid((unsigned)((N + kTp - 1) / kTp), (unsigned)((B + kTb - 1) / kTb));
  k_bsq_to_bip<T><<<grid, 256, 0, st>>>(static_cast<const T*>(bsq), N, B, static_cast<T*>(bip));
  return cudaGetLastError();
}

}  // namespace
}  // namespace gbpca

using namespace gbpca;

extern "C" int pca_bsq_to_bip(const void* bsq, pca_dtype dtype, int64_t N, int B, void* bip,
                              void* stream) {
  if (!bsq || !bip || N < 1 || B < 1 || N > ((int64_t)1 << 40)) return PCA_ERR_ARG;
  if ((N + kTp - 1) / kTp > 0x7fffffff || (B + kTb - 1) / kTb > 65535) return PCA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (dtype) {
    case PCA_F32: e = bsq_to_bip<float>(bsq, N, B, bip, st); break;
    case PCA_BF16:
    case PCA_F16: e = bsq_to_bip<unsigned short>(bsq, N, B, bip, st); break;
    default: return PCA_ERR_ARG;
  }
  return e == cudaSuccess ? PCA_OK : PCA_ERR_CUDA;
}
