// k_refine.cu -- FP64 refinement of the FP32 Jacobi result.
//
// The FP32 sweeps leave eigenvalues and eigenvectors with errors of order
// 2^-24 ||C||.  One refinement iteration is one simultaneous Jacobi-like
// sweep in FP64 over all pairs at once: with S = V^T C V (nearly diagonal)
// and R = I - V^T V, each pair (i, j) is turned by the first-order Jacobi
// angle  E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i)  -- the small-angle
// limit t ~ m/2 = C_ij / (C_jj - C_ii) of Eqs. 3 and 7, corrected for the
// non-orthogonality R -- and V <- V (I + E).  This is the iterative
// refinement of Ogita and Aishima (Japan J. Indust. Appl. Math. 35, 2018),
// which converges quadratically.  Their global cluster threshold (built from
// norms of S - diag and of R) is replaced by a per-pair test on the angle
// itself: pairs whose first-order angle exceeds 1/16 are treated as one
// cluster and only re-orthogonalised (E_ij = R_ij / 2).
//
// GB300 executes FP64 at about 1/58 of its FP32 rate, so only these O(B^3)
// GEMMs (spread over every SM) and the small element-wise steps run in FP64.
#include "common.cuh"

namespace gbpca {

namespace {

constexpr int kT = 16;  // output tile edge; 16x16 tiles spread B<=232 over ~200 CTAs

// D = op(A) Bm (+ X), all n x n row-major FP64.  op(A) = A or A^T.
template <bool kTransA>
__global__ void __launch_bounds__(kT* kT)
k_dgemm(const double* __restrict__ A, const double* __restrict__ Bm,
        const double* __restrict__ X, double* __restrict__ D, int n) {
  __shared__ double as[kT][kT + 1];
  __shared__ double bs[kT][kT + 1];
  const int tx = threadIdx.x % kT, ty = threadIdx.x / kT;
  const int row = blockIdx.y * kT + ty, col = blockIdx.x * kT + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < n; k0 += kT) {
    // as[ty][tx] = op(A)[row][k0 + tx]
    {
      const int r = blockIdx.y * kT + ty, k = k0 + tx;
      double v = 0.0;
      if (r < n && k < n) v = kTransA ? A[(size_t)k * n + r] : A[(size_t)r * n + k];
      as[ty][tx] = v;
    }
    {
      const int k = k0 + ty, c = blockIdx.x * kT + tx;
      bs[ty][tx] = (k < n && c < n) ? Bm[(size_t)k * n + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kT; ++kk) acc = fma(as[ty][kk], bs[kk][tx], acc);
    __syncthreads();
  }
  if (row < n && col < n) {
    if (X) acc += X[(size_t)row * n + col];
    D[(size_t)row * n + col] = acc;
  }
}

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// E_ij and lam~ (written by the diagonal entries).
__global__ void k_refine_E(const double* __restrict__ S, const double* __restrict__ G, int n,
                           double* __restrict__ E, double* __restrict__ lam,
                           DevHeader* __restrict__ hdr, double inv_max_angle) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double rii = 1.0 - G[(size_t)i * n + i], rjj = 1.0 - G[(size_t)j * n + j];
  const double li = S[(size_t)i * n + i] / (1.0 - rii);   // = S_ii / G_ii
  const double lj = S[(size_t)j * n + j] / (1.0 - rjj);
  const double rij = (i == j ? 1.0 : 0.0) - G[(size_t)i * n + j];
  const double num = S[(size_t)i * n + j] + lj * rij;
  const double gap = lj - li;
  // the first-order Jacobi angle where it is small (|t| <= max_angle); a pair
  // whose angle is larger is treated as part of a cluster and only
  // re-orthogonalised
  double e;
  if (i != j && fabs(gap) > inv_max_angle * fabs(num)) e = num / gap;
  else e = 0.5 * rij;
  E[(size_t)i * n + j] = e;
  if (i == j) lam[i] = li;
  atomic_max_pos(&hdr->refine_res, fabs(e));
}

}  // namespace

cudaError_t launch_refine(const double* C, int B, double* vc, double* lam, double* w, double* s,
                          double* g, double* e, DevHeader* hdr, double max_angle, cudaStream_t st) {
  const dim3 grid((B + kT - 1) / kT, (B + kT - 1) / kT);
  k_dgemm<false><<<grid, kT * kT, 0, st>>>(C, vc, nullptr, w, B);   // W = C V
  k_dgemm<true><<<grid, kT * kT, 0, st>>>(vc, w, nullptr, s, B);    // S = V^T W
  k_dgemm<true><<<grid, kT * kT, 0, st>>>(vc, vc, nullptr, g, B);   // G = V^T V
  cudaMemsetAsync(&hdr->refine_res, 0, sizeof(double), st);
  k_refine_E<<<dim3((B + 127) / 128, B), 128, 0, st>>>(s, g, B, e, lam, hdr, 1.0 / max_angle);
  k_dgemm<false><<<grid, kT * kT, 0, st>>>(vc, e, vc, w, B);        // V' = V E + V
  cudaMemcpyAsync(vc, w, sizeof(double) * (size_t)B * B, cudaMemcpyDeviceToDevice, st);
  return cudaGetLastError();
}

}  // namespace gbpca
