// moments.cu -- combination of per-shard band means and covariances, for a
// cube whose pixels are split over several GPUs (or several calls).  Not in
// the paper (it fits one image on one device); the manycore version splits
// the pixels over two I/O halves and adds partial products (Sec. 5), which is
// the same exchange step.
//
// Shard g holds n_g pixels with mean mu_g and covariance C_g (divided by
// n_g - 1; 0 for a one-pixel shard).  The pooled moments follow the pairwise
// rule of Chan, Golub and LeVeque (1979), applied to all shards at once:
//   mu   = sum_g n_g mu_g / n,                               n = sum_g n_g
//   C_ij = sum_g [ (n_g - 1) C_g,ij + n_g (mu_g,i - mu_i)(mu_g,j - mu_j) ] / (n - 1)
// -- exactly the mean and covariance of the union of the shards, with no
// cancellation between large raw moments.  FP64 throughout; shards are added
// in index order, so every caller with the same inputs gets the same bits.
#include "common.cuh"

namespace gbpca {
namespace {

constexpr int kMaxShards = 256;

struct ShardCounts {  // a kernel parameter: no copy, no allocation
  double n[kMaxShards];
};

__global__ void k_combine_mu(const double* __restrict__ mu_parts, int parts, int B,
                             const __grid_constant__ ShardCounts cnt, double inv_n,
                             double* __restrict__ mu) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s = 0.0;
  for (int g = 0; g < parts; ++g) s = fma(cnt.n[g], mu_parts[(size_t)g * B + b], s);
  mu[b] = s * inv_n;
}

__global__ void k_combine_cov(const double* __restrict__ mu_parts,
                              const double* __restrict__ C_parts, int parts, int B,
                              const __grid_constant__ ShardCounts cnt,
                              const double* __restrict__ mu, double inv_nm1,
                              double* __restrict__ C) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= B) return;
  const double mi = mu[i], mj = mu[j];
  double s = 0.0;
  for (int g = 0; g < parts; ++g) {
    const double ng = cnt.n[g];
    const double di = mu_parts[(size_t)g * B + i] - mi, dj = mu_parts[(size_t)g * B + j] - mj;
    s += (ng - 1.0) * C_parts[((size_t)g * B + i) * B + j] + ng * di * dj;
  }
  C[(size_t)i * B + j] = s * inv_nm1;
}

}  // namespace
}  // namespace gbpca

using namespace gbpca;

extern "C" int pca_combine_moments(int parts, const int64_t* n, const double* mu_parts,
                                   const double* C_parts, int B, double* mu, double* C,
                                   void* stream) {
  if (parts < 1 || parts > kMaxShards || !n || !mu_parts || !C_parts || !mu || !C)
    return PCA_ERR_ARG;
  if (B < 1 || B > kMaxB) return PCA_ERR_ARG;
  ShardCounts cnt{};
  double total = 0.0;
  for (int g = 0; g < parts; ++g) {
    if (n[g] < 1) return PCA_ERR_ARG;
    cnt.n[g] = (double)n[g];
    total += (double)n[g];
  }
  if (total < 2.0) return PCA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_combine_mu<<<(B + 127) / 128, 128, 0, st>>>(mu_parts, parts, B, cnt, 1.0 / total, mu);
  k_combine_cov<<<dim3((B + 127) / 128, B), 128, 0, st>>>(mu_parts, C_parts, parts, B, cnt, mu,
                                                         1.0 / (total - 1.0), C);
  return cudaGetLastError() == cudaSuccess ? PCA_OK : PCA_ERR_CUDA;
}
