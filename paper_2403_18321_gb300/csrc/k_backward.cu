// k_backward.cu -- adjoint of the PCA projection layer (the backward pass of
// Q = (Y - 1 mu^T) V_k, with an optional gradient of the eigenvalues).  Not in
// the paper; written from first-order perturbation theory of the symmetric
// eigenproblem:
//   dV_k = X^T dQ
//   G    = F o (V^T [dV_k, 0]) + diag(dlam),  F_ij = 1/(lam_j - lam_i) for
//          i != j with |lam_j - lam_i| > gap_eps |lam_1|, else 0
//   S    = sym(V G V^T)
//   dY   = (dQ - 1 mean_n dQ) V_k^T + 2/(N-1) X S.
// Three stages:
//   k_bwd_dv     one streaming pass over cube and dQ (TMA bulk copies of
//                64-pixel chunks): per-CTA partial sums of X^T dQ and of the
//                columns of dQ (FP32), thread = band;
//   k_bwd_reduce / k_bwd_m / k_bwd_s / k_bwd_sym   the B x B algebra in
//                FP64 (the FP32 partials added in FP64);
//   k_bwd_dy     dY as a register-tiled SIMT product [X | dQ'] [S'; V_k^T]
//                over 128-pixel x 64-band tiles, X centred while staged.
#include "tma.cuh"

namespace gbpca {

namespace {

// ------------------------------------------------------------------ k_bwd_dv
constexpr int kDvPx = 64;                 // pixels per chunk
constexpr int kDvWarps = 8;               // thread = band (B <= 256)
constexpr int kDvThreads = kDvWarps * 32 + 32;
constexpr int kDvStages = 3;

struct __align__(8) DvSync {
  uint64_t full[kDvStages];
  uint64_t empty[kDvStages];
  int abort;
};

template <typename In, int KQ>
__global__ void __launch_bounds__(kDvThreads, 1)
k_bwd_dv(const In* __restrict__ cube, const float* __restrict__ dq, int64_t N, int B, int k,
         const double* __restrict__ mu, float* __restrict__ dv_part, float* __restrict__ dqs_part,
         int cube_stage, int dq_stage, DevHeader* __restrict__ hdr) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* cst = smem;                                        // [S][cube_stage]
  float* dqst = reinterpret_cast<float*>(smem + kDvStages * cube_stage);  // [S][dq_stage/4]
  float* mus = dqst + kDvStages * dq_stage / 4;                     // [256]
  DvSync* sy = reinterpret_cast<DvSync*>(mus + 256);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x, g = blockIdx.x;
  const int64_t nch_total = (N + kDvPx - 1) / kDvPx;
  const int64_t c_begin = nch_total * g / G, c_end = nch_total * (g + 1) / G;
  const int nch = (int)(c_end - c_begin);
  for (int b = tid; b < 256; b += kDvThreads) mus[b] = b < B ? (float)mu[b] : 0.f;
  if (tid == 0) {
    for (int s = 0; s < kDvStages; ++s) { mbar_init(&sy->full[s], 1); mbar_init(&sy->empty[s], kDvWarps); }
    sy->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == kDvWarps) {
    if (lane == 0) {
      for (int c = 0; c < nch; ++c) {
        const int s = c % kDvStages;
        if (!mbar_wait(&sy->empty[s], ((c / kDvStages) & 1) ^ 1, &sy->abort)) break;
        const int64_t p0 = (c_begin + c) * kDvPx;
        const int cp = (int)((N - p0) < kDvPx ? (N - p0) : kDvPx);
        const uint32_t cb = (uint32_t)((size_t)cp * B * sizeof(In)) & ~15u;
        const uint32_t db = (uint32_t)((size_t)cp * k * 4) & ~15u;
        mbar_expect_tx(&sy->full[s], cb + db);
        if (cb) bulk_g2s(cst + (size_t)s * cube_stage, cube + p0 * B, cb, &sy->full[s]);
        if (db) bulk_g2s(reinterpret_cast<unsigned char*>(dqst) + (size_t)s * dq_stage, dq + p0 * k, db,
                         &sy->full[s]);
      }
    }
    return;
  }
  const int b = tid;                    // this thread's band
  float4 acc[KQ];
#pragma unroll
  for (int q = 0; q < KQ; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  float csum = 0.f;                     // column sum of dQ (threads j < k)
  const float m = b < B ? mus[b] : 0.f;
  int c = 0;
  for (; c < nch; ++c) {
    const int s = c % kDvStages;
    int ok = 1;
    if (lane == 0) ok = mbar_wait(&sy->full[s], (c / kDvStages) & 1, &sy->abort) ? 1 : 0;
    ok = __shfl_sync(kFull, ok, 0);
    if (!ok) break;
    const int64_t p0 = (c_begin + c) * kDvPx;
    const int cp = (int)((N - p0) < kDvPx ? (N - p0) : kDvPx);
    const In* xs = reinterpret_cast<const In*>(cst + (size_t)s * cube_stage);
    const float* ds = dqst + (size_t)s * dq_stage / 4;
    const int copied_x = (int)((((size_t)cp * B * sizeof(In)) & ~(size_t)15) / sizeof(In));
    const int copied_d = (int)((((size_t)cp * k * 4) & ~(size_t)15) / 4);
    const bool whole = copied_x == cp * B && copied_d == cp * k;
    for (int p = 0; p < cp; ++p) {
      float x = 0.f;
      float dv[KQ * 4];
      if (whole) {
        if (b < B) x = to_f32<In>(xs[p * B + b]) - m;
#pragma unroll
        for (int j = 0; j < KQ * 4; ++j) dv[j] = j < k ? ds[p * k + j] : 0.f;
      } else {
        const int ex = p * B + b;
        if (b < B) x = (ex < copied_x ? to_f32<In>(xs[ex]) : to_f32<In>(cube[p0 * B + ex])) - m;
#pragma unroll
        for (int j = 0; j < KQ * 4; ++j) {
          const int ed = p * k + j;
          dv[j] = j < k ? (ed < copied_d ? ds[ed] : dq[p0 * k + ed]) : 0.f;
        }
      }
#pragma unroll
      for (int q = 0; q < KQ; ++q) {
        acc[q].x = fmaf(x, dv[4 * q], acc[q].x);
        acc[q].y = fmaf(x, dv[4 * q + 1], acc[q].y);
        acc[q].z = fmaf(x, dv[4 * q + 2], acc[q].z);
        acc[q].w = fmaf(x, dv[4 * q + 3], acc[q].w);
      }
      if (tid < k) {
        const int ed = p * k + tid;
        csum += ed < copied_d ? ds[ed] : dq[p0 * k + ed];
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sy->empty[s]);
  }
  if (c < nch && tid == 0 && hdr) set_status(hdr, PCA_ERR_TIMEOUT);
  if (b < B) {
    float* out = dv_part + ((size_t)g * B + b) * k;
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
      const float v[4] = {acc[q].x, acc[q].y, acc[q].z, acc[q].w};
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (4 * q + t < k) out[4 * q + t] = v[t];
    }
  }
  if (tid < k) dqs_part[(size_t)g * k + tid] = csum;
}

// ------------------------------------------------------------------ k_bwd_reduce
// dVk[b][j] = sum over the partials (FP64), FP32 copy of mu; CTA 0 also forms
// the column means of dQ.  One CTA (one warp) per band.
__global__ void k_bwd_reduce(const float* __restrict__ dv_part, const float* __restrict__ dqs_part,
                             int parts, int64_t N, int B, int k, const double* __restrict__ mu,
                             double* __restrict__ dVk, float* __restrict__ mdq,
                             float* __restrict__ mu32) {
  const int b = blockIdx.x, j = threadIdx.x;
  if (j < k) {
    double s = 0.0;
    for (int gg = 0; gg < parts; ++gg) s += (double)dv_part[((size_t)gg * B + b) * k + j];
    dVk[(size_t)b * k + j] = s;
    if (b == 0) {
      double t = 0.0;
      for (int gg = 0; gg < parts; ++gg) t += (double)dqs_part[(size_t)gg * k + j];
      mdq[j] = (float)(t / (double)N);
    }
  }
  if (j == 0) mu32[b] = (float)mu[b];
}

// ------------------------------------------------------------------ k_bwd_m
// G_ij = F_ij (V^T dVk)_ij for j < k (i != j), G_jj = dlam_j; one warp per row i.
__global__ void k_bwd_m(int B, int k, const double* __restrict__ lam, const double* __restrict__ V,
                        const double* __restrict__ dVk, const double* __restrict__ dlam,
                        double gap_eps, double* __restrict__ Gk) {
  const int i = blockIdx.x, j = threadIdx.x;
  if (j >= k) return;
  double m = 0.0;
  for (int bb = 0; bb < B; ++bb) m += V[(size_t)bb * B + i] * dVk[(size_t)bb * k + j];
  double gval;
  if (i == j) {
    gval = dlam ? dlam[i] : 0.0;
  } else {
    const double gap = lam[j] - lam[i];
    gval = fabs(gap) > gap_eps * fabs(lam[0]) ? m / gap : 0.0;
  }
  Gk[(size_t)i * k + j] = gval;
}

// ------------------------------------------------------------------ k_bwd_s
// dA = V G V^T = T V^T with T = V G: T_aj = sum_{i} V_ai G_ij for j < k
// (plus V_aj dlam_j for j >= k), then S' = 2/(N-1) (dA + dA^T)/2 in FP32 and
// V_k in FP32.  One CTA per row a.
__global__ void __launch_bounds__(256)
k_bwd_s(const double* __restrict__ V, const double* __restrict__ Gk, const double* __restrict__ dlam,
        int64_t N, int B, int k, double* __restrict__ dA, float* __restrict__ vk32) {
  __shared__ double T[256];
  const int a = blockIdx.x, tid = threadIdx.x;
  for (int j = tid; j < B; j += 256) {
    double t;
    if (j < k) {
      t = 0.0;
      for (int i = 0; i < B; ++i) t += V[(size_t)a * B + i] * Gk[(size_t)i * k + j];
    } else {
      t = dlam ? V[(size_t)a * B + j] * dlam[j] : 0.0;
    }
    T[j] = t;
    if (j < k) vk32[(size_t)a * k + j] = (float)V[(size_t)a * B + j];
  }
  __syncthreads();
  const int jmax = dlam ? B : k;
  for (int c = tid; c < B; c += 256) {
    double s = 0.0;
    for (int j = 0; j < jmax; ++j) s += T[j] * V[(size_t)c * B + j];
    dA[(size_t)a * B + c] = s;
  }
}

__global__ void k_bwd_sym(const double* __restrict__ dA, int64_t N, int B, float* __restrict__ S32) {
  const int a = blockIdx.y, c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= B) return;
  const double f = 2.0 / (double)(N - 1);
  S32[(size_t)a * B + c] = (float)(f * 0.5 * (dA[(size_t)a * B + c] + dA[(size_t)c * B + a]));
}

// ------------------------------------------------------------------ k_bwd_dy
// dY[n][c] = sum_b x_nb S'_bc + sum_j (dq_nj - mdq_j) V_cj over a 128-pixel x
// 64-band output tile per CTA (256 threads, 8 x 4 outputs each), K staged in
// steps of 16 through shared memory; the band tiles of one pixel block are
// consecutive blocks of the grid, so that they reuse its cube rows from L2.
constexpr int kTM = 128, kTN = 64, kTK = 16;

template <typename In>
__global__ void __launch_bounds__(256)
k_bwd_dy(const In* __restrict__ cube, const float* __restrict__ dq, int64_t N, int B, int k,
         const float* __restrict__ mu32, const float* __restrict__ mdq, const float* __restrict__ S32,
         const float* __restrict__ vk32, float* __restrict__ dY) {
  __shared__ float As[kTK][kTM + 4];
  __shared__ float Bs[kTK][kTN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;          // 16 x 16 threads
  const int nbt = (B + kTN - 1) / kTN;            // band tiles of one pixel block
  const int c0 = (int)(blockIdx.x % nbt) * kTN;
  const int64_t n0 = (int64_t)(blockIdx.x / nbt) * kTM;
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  const int KT = B + k;                            // [X | dQ'] times [S'; V_k^T]
  for (int kk = 0; kk < KT; kk += kTK) {
    // A tile: rows n0.., columns kk.. of [X | dQ']
    for (int e = tid; e < kTK * kTM; e += 256) {
      const int r = e / kTK, q = e % kTK;          // q fastest: consecutive columns
      const int col = kk + q;
      const int64_t n = n0 + r;
      float v = 0.f;
      if (n < N) {
        if (col < B) v = to_f32<In>(cube[n * B + col]) - mu32[col];
        else if (col < KT) v = dq[n * k + (col - B)] - mdq[col - B];
      }
      As[q][r] = v;
    }
    // B tile: rows kk.. of [S'; V_k^T], columns c0..
    for (int e = tid; e < kTK * kTN; e += 256) {
      const int q = e / kTN, cc = e % kTN;
      const int row = kk + q, c = c0 + cc;
      float v = 0.f;
      if (c < B) {
        if (row < B) v = S32[(size_t)row * B + c];
        else if (row < KT) v = vk32[(size_t)c * k + (row - B)];
      }
      Bs[q][cc] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kTK; ++q) {
      float a[8], bv[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[q][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[q][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t n = n0 + ty + 16 * i;
    if (n >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c < B) dY[n * B + c] = acc[i][j];
    }
  }
}

template <typename In, int KQ>
cudaError_t dv_kq(const In* cube, const float* dq, int64_t N, int B, int k, const double* mu,
                  float* dv_part, float* dqs_part, int parts, DevHeader* hdr, cudaStream_t st) {
  const int cube_stage = (int)((((size_t)kDvPx * B * sizeof(In)) + 127) & ~(size_t)127);
  const int dq_stage = (int)((((size_t)kDvPx * k * 4) + 127) & ~(size_t)127);
  const size_t smem = (size_t)kDvStages * (cube_stage + dq_stage) + 256 * 4 + sizeof(DvSync);
  auto kern = k_bwd_dv<In, KQ>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<parts, kDvThreads, smem, st>>>(cube, dq, N, B, k, mu, dv_part, dqs_part, cube_stage,
                                        dq_stage, hdr);
  return cudaGetLastError();
}

template <typename In>
cudaError_t dv_typed(const In* cube, const float* dq, int64_t N, int B, int k, const double* mu,
                     float* dv_part, float* dqs_part, int parts, DevHeader* hdr, cudaStream_t st) {
  switch ((k + 3) / 4) {
    case 1: return dv_kq<In, 1>(cube, dq, N, B, k, mu, dv_part, dqs_part, parts, hdr, st);
    case 2: return dv_kq<In, 2>(cube, dq, N, B, k, mu, dv_part, dqs_part, parts, hdr, st);
    case 3: return dv_kq<In, 3>(cube, dq, N, B, k, mu, dv_part, dqs_part, parts, hdr, st);
    case 4: return dv_kq<In, 4>(cube, dq, N, B, k, mu, dv_part, dqs_part, parts, hdr, st);
    case 5: return dv_kq<In, 5>(cube, dq, N, B, k, mu, dv_part, dqs_part, parts, hdr, st);
    case 6: return dv_kq<In, 6>(cube, dq, N, B, k, mu, dv_part, dqs_part, parts, hdr, st);
    case 7: return dv_kq<In, 7>(cube, dq, N, B, k, mu, dv_part, dqs_part, parts, hdr, st);
    case 8: return dv_kq<In, 8>(cube, dq, N, B, k, mu, dv_part, dqs_part, parts, hdr, st);
  }
  return cudaErrorInvalidValue;
}

template <typename In>
cudaError_t dy_typed(const In* cube, const float* dq, int64_t N, int B, int k, const float* mu32,
                     const float* mdq, const float* S32, const float* vk32, float* dY,
                     cudaStream_t st) {
  const int64_t tiles = (int64_t)((B + kTN - 1) / kTN) * ((N + kTM - 1) / kTM);
  if (tiles > 0x7fffffffll) return cudaErrorInvalidValue;
  k_bwd_dy<In><<<(unsigned)tiles, 256, 0, st>>>(cube, dq, N, B, k, mu32, mdq, S32, vk32, dY);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_backward(const void* cube, pca_dtype dt, int64_t N, int B, int k,
                            const double* mu, const double* lam, const double* V,
                            const float* dq, const double* dlam, double gap_eps, float* dY,
                            const BwdPtrs& w, DevHeader* hdr, cudaStream_t st) {
  cudaError_t e;
  switch (dt) {
    case PCA_F32:
      e = dv_typed((const float*)cube, dq, N, B, k, mu, w.dv_part, w.dqs_part, w.parts, hdr, st);
      break;
    case PCA_BF16:
      e = dv_typed((const __nv_bfloat16*)cube, dq, N, B, k, mu, w.dv_part, w.dqs_part, w.parts, hdr,
                   st);
      break;
    case PCA_F16:
      e = dv_typed((const __half*)cube, dq, N, B, k, mu, w.dv_part, w.dqs_part, w.parts, hdr, st);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  k_bwd_reduce<<<B, 32, 0, st>>>(w.dv_part, w.dqs_part, w.parts, N, B, k, mu, w.dVk, w.mdq, w.mu32);
  k_bwd_m<<<B, 32, 0, st>>>(B, k, lam, V, w.dVk, dlam, gap_eps, w.Gk);
  k_bwd_s<<<B, 256, 0, st>>>(V, w.Gk, dlam, N, B, k, w.dA, w.vk32);
  k_bwd_sym<<<dim3((B + 127) / 128, B), 128, 0, st>>>(w.dA, N, B, w.S32);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  switch (dt) {
    case PCA_F32:
      return dy_typed((const float*)cube, dq, N, B, k, w.mu32, w.mdq, w.S32, w.vk32, dY, st);
    case PCA_BF16:
      return dy_typed((const __nv_bfloat16*)cube, dq, N, B, k, w.mu32, w.mdq, w.S32, w.vk32, dY, st);
    case PCA_F16:
      return dy_typed((const __half*)cube, dq, N, B, k, w.mu32, w.mdq, w.S32, w.vk32, dY, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbpca
