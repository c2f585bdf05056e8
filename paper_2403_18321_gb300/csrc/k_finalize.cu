// k_finalize.cu -- eigen-pair extraction, descending sort and sign rule
// (Sec. 4.2 stage 4.3), and the narrowing of mu and V_k for the projection
// (k_project.cu).
#include "common.cuh"

namespace gbpca {

namespace {

// Sort and sign rule in two fully parallel passes.
// k_rank_sign: one CTA per eigen-pair j.  Its rank = number of eigenvalues
// that sort before it (larger, or equal and at a lower position) -- no
// comparison sort needed for B <= 256 -- and the sign that makes the entry of
// largest magnitude (lowest row on ties) of column j positive.
__device__ __forceinline__ void rank_sign_pair(int j, const double* __restrict__ lam,
                                               const float2* __restrict__ vc, int B,
                                               int* __restrict__ rank, double* __restrict__ sgn,
                                               double* __restrict__ eigvals) {
  __shared__ int cnt[8];
  __shared__ double bv[8];
  __shared__ int bi[8];
  const int i = threadIdx.x, lane = i & 31, warp = i >> 5;
  const double lj = lam[j];
  int c = 0;
  double v = -1.0;
  int vi = 0x7fffffff;
  if (i < B) {
    const double li = lam[i];
    c = (li > lj) || (li == lj && i < j);
    const float2 x = vc[(size_t)i * B + j];
    v = fabs((double)x.x + (double)x.y);
    vi = i;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_xor_sync(kFull, c, o);
    const double ov = __shfl_xor_sync(kFull, v, o);
    const int oi = __shfl_xor_sync(kFull, vi, o);
    if (ov > v || (ov == v && oi < vi)) { v = ov; vi = oi; }
  }
  if (lane == 0) { cnt[warp] = c; bv[warp] = v; bi[warp] = vi; }
  __syncthreads();
  if (i == 0) {
    int tot = 0;
    double best = -1.0;
    int besti = 0x7fffffff;
    for (int w = 0; w < 8; ++w) {
      tot += cnt[w];
      if (bv[w] > best || (bv[w] == best && bi[w] < besti)) { best = bv[w]; besti = bi[w]; }
    }
    const int r = min(tot, B - 1);
    const float2 x = vc[(size_t)besti * B + j];
    rank[j] = r;
    sgn[j] = ((double)x.x + (double)x.y) < 0.0 ? -1.0 : 1.0;
    eigvals[r] = lj;
  }
}
__global__ void __launch_bounds__(256)
k_rank_sign(const double* __restrict__ lam, const float2* __restrict__ vc, int B,
            int* __restrict__ rank, double* __restrict__ sgn, double* __restrict__ eigvals) {
  rank_sign_pair(blockIdx.x, lam, vc, B, rank, sgn, eigvals);
}

// scatter: one CTA per row i of V writes row i of the sorted, signed eigvecs.
__device__ __forceinline__ void scatter_row(int i, const float2* __restrict__ vc, int B, int k,
                                            const int* __restrict__ rank,
                                            const double* __restrict__ sgn,
                                            double* __restrict__ eigvecs, float* __restrict__ vk) {
  for (int j = threadIdx.x; j < B; j += blockDim.x) {
    const float2 x = vc[(size_t)i * B + j];
    const double v = sgn[j] * ((double)x.x + (double)x.y);
    const int r = rank[j];
    eigvecs[(size_t)i * B + r] = v;
    if (r < k) vk[(size_t)i * k + r] = (float)v;
  }
}
__global__ void __launch_bounds__(256)
k_scatter(const float2* __restrict__ vc, int B, int k, const int* __restrict__ rank,
          const double* __restrict__ sgn, double* __restrict__ eigvecs, float* __restrict__ vk) {
  scatter_row(blockIdx.x, vc, B, k, rank, sgn, eigvecs, vk);
}
__global__ void __launch_bounds__(256)
k_rank_sign_batched(const TileDesc* __restrict__ T, int in_w) {
  const TileDesc& t = T[blockIdx.y];
  if ((int)blockIdx.x >= t.B) return;
  rank_sign_pair(blockIdx.x, t.lam, in_w ? t.w : t.vc, t.B, t.rank, t.sgn, t.eigvals);
}
__global__ void __launch_bounds__(256)
k_scatter_batched(const TileDesc* __restrict__ T, int in_w) {
  const TileDesc& t = T[blockIdx.y];
  if ((int)blockIdx.x >= t.B) return;
  scatter_row(blockIdx.x, in_w ? t.w : t.vc, t.B, t.k, t.rank, t.sgn, t.eigvecs, t.vk);
}
__global__ void k_narrow(const double* __restrict__ mu, const double* __restrict__ V, int B, int k,
                         float* __restrict__ mu_f, float* __restrict__ vk) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * k; e += gridDim.x * blockDim.x) {
    const int i = e / k, j = e - i * k;
    vk[e] = (float)V[(size_t)i * B + j];
  }
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x)
    mu_f[b] = (float)mu[b];
}

}  // namespace

cudaError_t launch_narrow_inputs(const double* mu, const double* eigvecs, int B, int k, float* mu_f,
                                 float* vk, cudaStream_t st) {
  k_narrow<<<(B * k + 255) / 256, 256, 0, st>>>(mu, eigvecs, B, k, mu_f, vk);
  return cudaGetLastError();
}

cudaError_t launch_sort_sign(const double* lam, const float2* vc, int B, int k, double* eigvals,
                             double* eigvecs, float* vk, int* rank, double* sgn, cudaStream_t st) {
  k_rank_sign<<<B, 256, 0, st>>>(lam, vc, B, rank, sgn, eigvals);
  k_scatter<<<B, 256, 0, st>>>(vc, B, k, rank, sgn, eigvecs, vk);
  return cudaGetLastError();
}

cudaError_t launch_sort_sign_batched(const TileDesc* T, int ntiles, int maxB, bool final_in_w,
                                     cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  k_rank_sign_batched<<<dim3(maxB, ntiles), 256, 0, st>>>(T, final_in_w ? 1 : 0);
  k_scatter_batched<<<dim3(maxB, ntiles), 256, 0, st>>>(T, final_in_w ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace gbpca
