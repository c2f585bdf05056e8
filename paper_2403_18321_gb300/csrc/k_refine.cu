// k_refine.cu -- high-precision refinement of the FP32 Jacobi result.
//
// The FP32 sweeps leave eigenvalues and eigenvectors with errors of order
// 2^-24 ||C||.  One refinement iteration is one simultaneous Jacobi-like
// sweep over all pairs at once: with S = V^T C V (nearly diagonal) and
// R = I - V^T V, each pair (i, j) is turned by the first-order Jacobi angle
//     E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i)
// -- the small-angle limit t ~ m/2 = C_ij / (C_jj - C_ii) of Eqs. 3 and 7,
// corrected for the non-orthogonality R -- and V <- V (I + E).  This is the
// iterative refinement of Ogita and Aishima (Japan J. Indust. Appl. Math. 35,
// 2018), which converges quadratically.  Their global cluster threshold is
// replaced by a per-pair test on the angle itself: a pair whose first-order
// angle exceeds `max_angle` is treated as part of a cluster and only
// re-orthogonalised (E_ij = R_ij / 2).  A first-order update leaves V
// non-orthogonal by O(||E||^2); a closing Newton-Schulz step
// V <- V (3I - V^T V)/2 squares that away (launch_orthonormalize).
//
// Arithmetic: GB300 executes FP64 at about 1/58 of its FP32 rate (1.9 DFMA
// per clock per SM), which would make each B^3 product cost ~20 us at
// B = 224.  The products therefore run in double-float: every matrix is kept
// as an unevaluated sum hi + lo of two FP32 values (48-bit significand), each
// product is formed exactly with one FMA (Dekker/Kahan "TwoProduct"), and the
// running sum is carried with Knuth's "TwoSum" (error-free transformations;
// Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26, 2005).  Only the O(B^2)
// element-wise steps (angles, lambda) use FP64.
#include "common.cuh"

namespace gbpca {

namespace {

constexpr int kT = 16;           // output tile edge per CTA
constexpr int kTh = 64;          // threads per CTA: 8 x 8, each 2 x 2 outputs

__device__ __forceinline__ double df_to_d(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ float2 d_to_df(double d) {
  const float hi = (float)d;
  return make_float2(hi, (float)(d - (double)hi));
}

// acc += a * b in double-float.  The _rn intrinsics keep the compiler from
// contracting the error-free transformations into fused operations.
__device__ __forceinline__ void df_mac(float2& acc, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);           // exact: a.x*b.x = p + e
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);                  // a.y*b.y (2^-48 relative) dropped
  const float s = __fadd_rn(acc.x, p);    // TwoSum(acc.x, p)
  const float z = __fsub_rn(s, acc.x);
  const float t = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(s, z)), __fsub_rn(p, z));
  acc.y = __fadd_rn(acc.y, __fadd_rn(t, e));
  acc.x = s;
}
__device__ __forceinline__ float2 df_norm(float2 v) {  // Fast2Sum renormalisation
  const float s = __fadd_rn(v.x, v.y);
  return make_float2(s, __fsub_rn(v.y, __fsub_rn(s, v.x)));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float z = __fsub_rn(s, a.x);
  const float t = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, z)), __fsub_rn(b.x, z));
  return df_norm(make_float2(s, __fadd_rn(__fadd_rn(t, a.y), b.y)));
}

// D = op(A) Bm (+ X), n x n row-major double-float (float2 = hi, lo).
// CTA = 16 x 16 output tile, 256 threads = 4 K-groups x (8 x 8 threads with
// 2 x 2 outputs each); the K-groups take every fourth 16-wide K chunk and
// their partial sums are added at the end (enough warps per SM to hide the
// dependent chains of the error-free transformations).
template <bool kTransA>
__device__ __forceinline__ void dfgemm_tile(const float2* __restrict__ A,
                                            const float2* __restrict__ Bm,
                                            const float2* __restrict__ X, float2* __restrict__ D,
                                            int n, int r0, int c0) {
  __shared__ float2 as[4][kT][kT + 1];  // as[group][k][row]
  __shared__ float2 bs[4][kT][kT + 1];  // bs[group][k][col]
  __shared__ float2 red[3][kT * kT];
  const int grp = threadIdx.x / kTh, t = threadIdx.x % kTh;
  const int tx = t & 7, ty = t >> 3;
  float2 acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_float2(0.f, 0.f);
  const int nchunks = (n + kT - 1) / kT;
  for (int base = 0; base < nchunks; base += 4) {
    const int ch = base + grp;
    const int k0 = ch * kT;
    if (ch < nchunks) {
      for (int e = t; e < kT * kT; e += kTh) {
        const int a = e / kT, b = e % kT;
        {  // as[k][row] = op(A)[r0 + row][k0 + k]; the index that runs fastest
           // over the threads is the one contiguous in memory
          const int row = kTransA ? b : a, kk = kTransA ? a : b;
          const int r = r0 + row, k = k0 + kk;
          float2 v = make_float2(0.f, 0.f);
          if (r < n && k < n) v = kTransA ? A[(size_t)k * n + r] : A[(size_t)r * n + k];
          as[grp][kk][row] = v;
        }
        {  // bs[k = a][col = b] = Bm[k0 + a][c0 + b]
          const int k = k0 + a, c = c0 + b;
          bs[grp][a][b] = (k < n && c < n) ? Bm[(size_t)k * n + c] : make_float2(0.f, 0.f);
        }
      }
    }
    __syncthreads();
    if (ch < nchunks) {
#pragma unroll 4
      for (int kk = 0; kk < kT; ++kk) {
        const float2 a0 = as[grp][kk][2 * ty], a1 = as[grp][kk][2 * ty + 1];
        const float2 b0 = bs[grp][kk][2 * tx], b1 = bs[grp][kk][2 * tx + 1];
        df_mac(acc[0][0], a0, b0);
        df_mac(acc[0][1], a0, b1);
        df_mac(acc[1][0], a1, b0);
        df_mac(acc[1][1], a1, b1);
      }
    }
    __syncthreads();
  }
  if (grp > 0) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) red[grp - 1][(2 * ty + i) * kT + 2 * tx + j] = df_norm(acc[i][j]);
  }
  __syncthreads();
  if (grp == 0) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int r = r0 + 2 * ty + i, c = c0 + 2 * tx + j;
        float2 v = df_norm(acc[i][j]);
#pragma unroll
        for (int q = 0; q < 3; ++q) v = df_add(v, red[q][(2 * ty + i) * kT + 2 * tx + j]);
        if (r < n && c < n) {
          if (X) v = df_add(v, X[(size_t)r * n + c]);
          D[(size_t)r * n + c] = v;
        }
      }
  }
}

// sym: D is symmetric (V^T W, V^T V) -- only the tiles on or above the
// diagonal are formed, and readers take entry (min(i,j), max(i,j)).
template <bool kTransA>
__global__ void __launch_bounds__(kTh * 4)
k_dfgemm(const float2* __restrict__ A, const float2* __restrict__ Bm,
         const float2* __restrict__ X, float2* __restrict__ D, int n, int sym) {
  if (sym && blockIdx.y > blockIdx.x) return;
  dfgemm_tile<kTransA>(A, Bm, X, D, n, blockIdx.y * kT, blockIdx.x * kT);
}

// The products of one refinement iteration / orthogonalisation step for
// every tile of a batch (tile = blockIdx.z); v is vc, or w when flip.
enum BatchedProduct { kCV = 0, kVtW = 1, kVtV = 2, kVEpV = 3 };
template <bool kTransA>
__global__ void __launch_bounds__(kTh * 4)
k_dfgemm_batched(const TileDesc* __restrict__ T, int product, int flip) {
  const TileDesc& t = T[blockIdx.z];
  const int n = t.B;
  if ((int)blockIdx.y * kT >= n || (int)blockIdx.x * kT >= n) return;
  if ((product == kVtW || product == kVtV) && blockIdx.y > blockIdx.x) return;  // symmetric
  const float2* v = flip ? t.w : t.vc;
  float2* vout = flip ? t.vc : t.w;
  const float2 *A, *Bm, *X = nullptr;
  float2* D;
  switch (product) {
    case kCV: A = t.cdf; Bm = v; D = vout; break;             // W = C V (in vout)
    case kVtW: A = v; Bm = vout; D = t.s; break;              // S = V^T W
    case kVtV: A = v; Bm = v; D = t.g; break;                 // G = V^T V
    default: A = v; Bm = t.e; X = v; D = vout; break;         // V' = V E + V
  }
  dfgemm_tile<kTransA>(A, Bm, X, D, n, blockIdx.y * kT, blockIdx.x * kT);
}

void dfgemm(bool transA, const float2* A, const float2* Bm, const float2* X, float2* D, int n,
            bool sym, cudaStream_t st) {
  const dim3 grid((n + kT - 1) / kT, (n + kT - 1) / kT);
  if (transA) k_dfgemm<true><<<grid, kTh * 4, 0, st>>>(A, Bm, X, D, n, sym ? 1 : 0);
  else k_dfgemm<false><<<grid, kTh * 4, 0, st>>>(A, Bm, X, D, n, sym ? 1 : 0);
}

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// num / den in FP64 without the FP64 divider (slow on this GPU): an FP32
// reciprocal as the seed, one Newton-Raphson step r <- r (2 - den r), the
// quotient q = num r, and one residual correction q <- q + r (num - den q)
// (Markstein's scheme), all in FP64.  Denominators outside the FP32 normal
// range take the plain division.
__device__ __forceinline__ double quotient(double num, double den) {
  const float df = (float)den;
  if (!(fabsf(df) >= 1.17549435e-38f) || !(fabsf(df) <= 3.0e38f)) return num / den;
  double r = (double)__frcp_rn(df);
  r = r * fma(-den, r, 2.0);
  double q = num * r;
  return fma(r, fma(-den, q, num), q);
}

// lam~_i = S_ii / G_ii, once per eigen-pair, and the residual word reset
// before k_refine_E maximises into it.
__device__ __forceinline__ void refine_lam_entry(int i, const float2* __restrict__ S,
                                                 const float2* __restrict__ G, int n,
                                                 double* __restrict__ lam,
                                                 DevHeader* __restrict__ hdr) {
  if (i < n) lam[i] = df_to_d(S[(size_t)i * n + i]) / df_to_d(G[(size_t)i * n + i]);
  if (i == 0) hdr->refine_res = 0.0;
}

// E_ij from the upper triangles of S and G (both symmetric), FP64.
__device__ __forceinline__ void refine_E_row(int i, int j, const float2* __restrict__ S,
                                             const float2* __restrict__ G, int n,
                                             float2* __restrict__ E,
                                             const double* __restrict__ lam,
                                             DevHeader* __restrict__ hdr, double inv_max_angle) {
  double e = 0.0;
  if (j < n) {
    const size_t u = i <= j ? (size_t)i * n + j : (size_t)j * n + i;
    const double li = lam[i], lj = lam[j];
    const double rij = (i == j ? 1.0 : 0.0) - df_to_d(G[u]);
    const double sij = df_to_d(S[u]);
    const double num = sij + lj * rij;
    const double gap = lj - li;
    // classified the same way from (i, j) and (j, i), so that E_ij + E_ji = R_ij;
    // gaps at FP64 rounding level of ||A||_F (e.g. the null space of a
    // rank-deficient covariance) count as clustered too
    const double size = fabs(sij) + fmax(fabs(li), fabs(lj)) * fabs(rij);
    const double floor = 64.0 * 2.220446049250313e-16 * hdr->fro;
    if (i != j && fabs(gap) > inv_max_angle * size && fabs(gap) > floor) e = quotient(num, gap);
    else e = 0.5 * rij;
    E[(size_t)i * n + j] = d_to_df(e);
  }
  // largest |E_ij|: one atomic per warp (one max over all B^2 entries on a
  // single word would serialise)
  double m = fabs(e);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomic_max_pos(&hdr->refine_res, m);
}
__global__ void k_refine_lam(const float2* __restrict__ S, const float2* __restrict__ G, int n,
                             double* __restrict__ lam, DevHeader* __restrict__ hdr) {
  refine_lam_entry(blockIdx.x * blockDim.x + threadIdx.x, S, G, n, lam, hdr);
}
__global__ void k_refine_lam_batched(const TileDesc* __restrict__ T) {
  const TileDesc& t = T[blockIdx.y];
  refine_lam_entry(blockIdx.x * blockDim.x + threadIdx.x, t.s, t.g, t.B, t.lam, t.hdr);
}
__global__ void k_refine_E(const float2* __restrict__ S, const float2* __restrict__ G, int n,
                           float2* __restrict__ E, const double* __restrict__ lam,
                           DevHeader* __restrict__ hdr, double inv_max_angle) {
  refine_E_row(blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x, S, G, n, E, lam, hdr,
               inv_max_angle);
}
__global__ void k_refine_E_batched(const TileDesc* __restrict__ T, double inv_max_angle) {
  const TileDesc& t = T[blockIdx.z];
  if ((int)blockIdx.y >= t.B || (int)blockIdx.x * (int)blockDim.x >= t.B) return;
  refine_E_row(blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x, t.s, t.g, t.B, t.e, t.lam, t.hdr,
               inv_max_angle);
}

// E = (I - G) / 2: one Newton-Schulz step V <- V (3I - V^T V)/2 = V + V E.
__device__ __forceinline__ void ns_E_entry(int i, int j, const float2* __restrict__ G, int n,
                                           float2* __restrict__ E) {
  if (j >= n) return;
  const float2 g = G[i <= j ? (size_t)i * n + j : (size_t)j * n + i];  // upper triangle
  const float2 r = i == j ? df_add(make_float2(1.f, 0.f), make_float2(-g.x, -g.y))
                          : make_float2(-g.x, -g.y);
  E[(size_t)i * n + j] = make_float2(0.5f * r.x, 0.5f * r.y);
}
__global__ void k_ns_E(const float2* __restrict__ G, int n, float2* __restrict__ E) {
  ns_E_entry(blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x, G, n, E);
}
__global__ void k_ns_E_batched(const TileDesc* __restrict__ T) {
  const TileDesc& t = T[blockIdx.z];
  if ((int)blockIdx.y >= t.B) return;
  ns_E_entry(blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x, t.g, t.B, t.e);
}

__global__ void k_to_df(const double* __restrict__ src, float2* __restrict__ dst, int count) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
    dst[e] = d_to_df(src[e]);
}
__global__ void k_to_df_batched(const TileDesc* __restrict__ T) {
  const TileDesc& t = T[blockIdx.y];
  const int count = t.B * t.B;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
    t.cdf[e] = d_to_df(t.C[e]);
}

}  // namespace

cudaError_t launch_to_df(const double* src, float2* dst, int count, cudaStream_t st) {
  k_to_df<<<(count + 255) / 256, 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

cudaError_t launch_orthonormalize(const float2* v, float2* vout, int B, float2* g, float2* e,
                                  cudaStream_t st) {
  dfgemm(true, v, v, nullptr, g, B, true, st);                   // G = V^T V (upper)
  k_ns_E<<<dim3((B + 127) / 128, B), 128, 0, st>>>(g, B, e);
  dfgemm(false, v, e, v, vout, B, false, st);                    // V' = V E + V
  return cudaGetLastError();
}

cudaError_t launch_refine(const float2* C, int B, const float2* v, float2* vout, double* lam,
                          float2* s, float2* g, float2* e, DevHeader* hdr, double max_angle,
                          cudaStream_t st) {
  dfgemm(false, C, v, nullptr, vout, B, false, st);  // W = C V (in vout until the last product)
  dfgemm(true, v, vout, nullptr, s, B, true, st);    // S = V^T W (upper)
  dfgemm(true, v, v, nullptr, g, B, true, st);       // G = V^T V (upper)
  k_refine_lam<<<(B + 127) / 128, 128, 0, st>>>(s, g, B, lam, hdr);
  k_refine_E<<<dim3((B + 127) / 128, B), 128, 0, st>>>(s, g, B, e, lam, hdr, 1.0 / max_angle);
  dfgemm(false, v, e, v, vout, B, false, st);        // V' = V E + V
  return cudaGetLastError();
}

void dfgemm_batched(bool transA, const TileDesc* T, int ntiles, int maxB, int product, bool flip,
                    cudaStream_t st) {
  const dim3 grid((maxB + kT - 1) / kT, (maxB + kT - 1) / kT, ntiles);
  if (transA) k_dfgemm_batched<true><<<grid, kTh * 4, 0, st>>>(T, product, flip ? 1 : 0);
  else k_dfgemm_batched<false><<<grid, kTh * 4, 0, st>>>(T, product, flip ? 1 : 0);
}

cudaError_t launch_to_df_batched(const TileDesc* T, int ntiles, int maxB, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  k_to_df_batched<<<dim3((maxB * maxB + 1023) / 1024, ntiles), 256, 0, st>>>(T);
  return cudaGetLastError();
}

cudaError_t launch_refine_batched(const TileDesc* T, int ntiles, int maxB, bool flip,
                                  double max_angle, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  dfgemm_batched(false, T, ntiles, maxB, kCV, flip, st);
  dfgemm_batched(true, T, ntiles, maxB, kVtW, flip, st);
  dfgemm_batched(true, T, ntiles, maxB, kVtV, flip, st);
  k_refine_lam_batched<<<dim3((maxB + 127) / 128, ntiles), 128, 0, st>>>(T);
  k_refine_E_batched<<<dim3((maxB + 127) / 128, maxB, ntiles), 128, 0, st>>>(T, 1.0 / max_angle);
  dfgemm_batched(false, T, ntiles, maxB, kVEpV, flip, st);
  return cudaGetLastError();
}

cudaError_t launch_orthonormalize_batched(const TileDesc* T, int ntiles, int maxB, bool flip,
                                          cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  dfgemm_batched(true, T, ntiles, maxB, kVtV, flip, st);
  k_ns_E_batched<<<dim3((maxB + 127) / 128, maxB, ntiles), 128, 0, st>>>(T);
  dfgemm_batched(false, T, ntiles, maxB, kVEpV, flip, st);
  return cudaGetLastError();
}

}  // namespace gbpca
