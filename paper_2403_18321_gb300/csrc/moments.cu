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
//
// The same pooling as one sum (for a single all-reduce over the ranks): with a
// shift s common to all shards, shard g contributes n_g, S1 = n_g (mu_g - s)
// and S2 = (n_g - 1) C_g + n_g (mu_g - s)(mu_g - s)^T (upper triangle); the
// summed vector gives mu = s + S1/n and C = (S2 - S1 S1^T/n)/(n - 1).  With s
// near the cube's mean (the mean of one shard) the subtraction loses no more
// than the spread of the shard means against the pixel spread.
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

// Row i of the packed upper triangle starts at i B - i (i - 1)/2.
__device__ __forceinline__ size_t tri_row(int i, int B) {
  return (size_t)i * B - (size_t)i * (i - 1) / 2;
}

// grid (ceil(B/128), B + 1): rows 0..B-1 write S2 row i, row B writes n and S1
__global__ void k_shifted_sums(double n, const double* __restrict__ mu,
                               const double* __restrict__ C, const double* __restrict__ s, int B,
                               double* __restrict__ sums) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= B) return;
  const double dj = mu[j] - s[j];
  if (i == B) {
    sums[1 + j] = n * dj;
    if (j == 0) sums[0] = n;
    return;
  }
  if (j < i) return;
  const double di = mu[i] - s[i];
  sums[1 + B + tri_row(i, B) + (j - i)] = fma(n * di, dj, (n - 1.0) * C[(size_t)i * B + j]);
}

__global__ void k_moments_from_sums(const double* __restrict__ sums, const double* __restrict__ s,
                                    int B, double* __restrict__ mu, double* __restrict__ C) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= B) return;
  const double n = sums[0];
  const double* S1 = sums + 1;
  if (i == 0) mu[j] = s[j] + S1[j] / n;
  const int a = i < j ? i : j, b = i < j ? j : i;
  const double s2 = sums[1 + B + tri_row(a, B) + (b - a)];
  C[(size_t)i * B + j] = n >= 2.0 ? (s2 - S1[i] * S1[j] / n) / (n - 1.0) : 0.0;
}

}  // namespace
}  // namespace gbpca

using namespace gbpca;

extern "C" int pca_shifted_sums(int64_t n, const double* mu, const double* C, const double* s,
                                int B, double* sums, void* stream) {
  if (n < 1 || !mu || !C || !s || !sums || B < 1 || B > kMaxB) return PCA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_shifted_sums<<<dim3((B + 127) / 128, B + 1), 128, 0, st>>>((double)n, mu, C, s, B, sums);
  return cudaGetLastError() == cudaSuccess ? PCA_OK : PCA_ERR_CUDA;
}

extern "C" int pca_moments_from_sums(const double* sums, const double* s, int B, double* mu,
                                     double* C, void* stream) {
  if (!sums || !s || !mu || !C || B < 1 || B > kMaxB) return PCA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_moments_from_sums<<<dim3((B + 127) / 128, B), 128, 0, st>>>(sums, s, B, mu, C);
  return cudaGetLastError() == cudaSuccess ? PCA_OK : PCA_ERR_CUDA;
}

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
