// k_compact.cu -- drops the padding slot of the Jacobi result (Sec. 2,
// Eqs. 2-10): when B is odd the solver runs on B' = B + 1 with a zero row
// and column, whose slot is recognised by its row of V (every rotation that
// meets the padding index has a_pq = 0, so it only swaps positions and the
// padding row of V stays a unit vector).
#include "common.cuh"

namespace gbpca {

namespace {

// lam[c], vc[i][c] for the real rows i < B and the real slots (padding slot
// dropped); one CTA per row i.
__device__ __forceinline__ void compact_row(int i, const float* __restrict__ diag32,
                                            const float* __restrict__ v32, int B,
                                            DevHeader* __restrict__ hdr, double* __restrict__ lam,
                                            float2* __restrict__ vc) {
  const int Bp = B + (B & 1);
  __shared__ int s_dummy;
  if (threadIdx.x == 0) s_dummy = -1;
  __syncthreads();
  if (B & 1) {
    const float* last = v32 + (size_t)(Bp - 1) * Bp;
    for (int j = threadIdx.x; j < Bp; j += blockDim.x)
      if (last[j] == 1.f) s_dummy = j;
  }
  __syncthreads();
  const int dmy = s_dummy;
  for (int j = threadIdx.x; j < Bp; j += blockDim.x) {
    if (j == dmy) continue;
    const int c = (dmy >= 0 && j > dmy) ? j - 1 : j;
    if (c >= B) continue;
    vc[(size_t)i * B + c] = make_float2(v32[(size_t)i * Bp + j], 0.f);
    if (i == 0) lam[c] = (double)diag32[j];
  }
  if (i == 0 && threadIdx.x == 0) hdr->dummy_slot = dmy;
}
__global__ void k_compact(const float* __restrict__ diag32, const float* __restrict__ v32, int B,
                          DevHeader* __restrict__ hdr, double* __restrict__ lam,
                          float2* __restrict__ vc) {
  compact_row(blockIdx.x, diag32, v32, B, hdr, lam, vc);
}
__global__ void k_compact_batched(const TileDesc* __restrict__ T) {
  const TileDesc& t = T[blockIdx.y];
  if ((int)blockIdx.x >= t.B) return;
  compact_row(blockIdx.x, t.diag32, t.v32, t.B, t.hdr, t.lam, t.vc);
}

}  // namespace

cudaError_t launch_compact(const float* diag32, const float* v32, int B, DevHeader* hdr,
                           double* lam, float2* vc, cudaStream_t st) {
  k_compact<<<B, 256, 0, st>>>(diag32, v32, B, hdr, lam, vc);
  return cudaGetLastError();
}

cudaError_t launch_compact_batched(const TileDesc* T, int ntiles, int maxB, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  k_compact_batched<<<dim3(maxB, ntiles), 256, 0, st>>>(T);
  return cudaGetLastError();
}

}  // namespace gbpca
