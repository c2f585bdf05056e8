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
//   k_bwd_dv     one streaming pass over cube and dQ per group of 32
//                columns of dQ (TMA bulk copies of
//                64-pixel chunks): per-CTA partial sums of X^T dQ and of the
//                columns of dQ (FP32), thread = band in each of three
//                groups (two for k > 16, where the registers of 800 threads
//                run out) that take alternate pixels, so that several warps
//                per band slice keep shared-memory loads in flight while
//                others compute; their sums are added at the end;
//                the same pass records the largest |x_b| and |dq_j| (the
//                operand scales of the dY product);
//   k_bwd_reduce / k_bwd_m / k_bwd_s / k_bwd_sym   the B x B algebra in
//                FP64 (the FP32 partials added in FP64);
//   dY           the product [X | dQ'] [S'; V_k^T] on the tensor cores
//                (k_bwd_dy_tc.cu).
#include "tma.cuh"

namespace gbpca {

namespace {

// ------------------------------------------------------------------ k_bwd_dv
constexpr int kDvPx = 64;                 // pixels per chunk
// pixel groups (alternate pixels; thread = band within a group, B <= 256):
// three while the registers of 800 threads allow it (k <= 16), else two
__host__ __device__ constexpr int dv_groups(int KQ) { return KQ <= 4 ? 3 : 2; }
__host__ __device__ constexpr int dv_compute(int KQ) { return dv_groups(KQ) * 256; }
__host__ __device__ constexpr int dv_threads(int KQ) { return dv_compute(KQ) + 32; }
constexpr int kDvStages = 3;              // most stages; fewer when shared memory is short

template <int NT>
__device__ __forceinline__ void dv_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}
// AND of a flag over the compute warps (they leave the chunk loop together)
template <int NT>
__device__ __forceinline__ int dv_and(int v) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n"
      " selp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(v), "n"(NT)
      : "memory");
  return r;
}

struct __align__(16) DvSync {
  uint64_t full[kDvStages];
  uint64_t empty[kDvStages];
  int abort;
  int pad[3];
  float4 comb[256];          // the second group's sums, one column quad at a time
  float combv[3][256];       // its xmax (by band), column sums and |dq| maxima
};

// One pass covers dQ columns [j0, j0 + k) (k <= 32) of a dQ whose rows are ld
// floats long; the partials are written at the same column offset.  dQ rows
// are bulk-copied with the cube chunk when the pass covers all columns
// (ld == k), else read straight from dQ.
template <typename In, int KQ>
__global__ void __launch_bounds__(dv_threads(KQ), 1)
k_bwd_dv(const In* __restrict__ cube, const float* __restrict__ dq, int64_t N, int B, int k,
         int j0, int ld, const double* __restrict__ mu, float* __restrict__ dv_part,
         float* __restrict__ dqs_part, float* __restrict__ xmax_part,
         float* __restrict__ dqmax_part, int cube_stage, int dq_stage, int nst,
         DevHeader* __restrict__ hdr) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* cst = smem;                                        // [nst][cube_stage]
  float* dqst = reinterpret_cast<float*>(smem + nst * cube_stage);  // [nst][dq_stage/4]
  float* mus = dqst + nst * dq_stage / 4;                           // [256]
  float4* dqpad = reinterpret_cast<float4*>(mus + 256);              // [2][kDvPx][KQ]
  DvSync* sy = reinterpret_cast<DvSync*>(dqpad + 2 * kDvPx * KQ);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x, g = blockIdx.x;
  const int64_t nch_total = (N + kDvPx - 1) / kDvPx;
  const int64_t c_begin = nch_total * g / G, c_end = nch_total * (g + 1) / G;
  const int nch = (int)(c_end - c_begin);
  constexpr int kGroups = dv_groups(KQ), kComp = dv_compute(KQ), kWarps = kComp / 32;
  for (int b = tid; b < 256; b += dv_threads(KQ)) mus[b] = b < B ? (float)mu[b] : 0.f;
  if (tid == 0) {
    for (int s = 0; s < nst; ++s) { mbar_init(&sy->full[s], 1); mbar_init(&sy->empty[s], kWarps); }
    sy->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == kWarps) {
    if (lane == 0) {
      for (int c = 0; c < nch; ++c) {
        const int s = c % nst;
        if (!mbar_wait(&sy->empty[s], ((c / nst) & 1) ^ 1, &sy->abort)) break;
        const int64_t p0 = (c_begin + c) * kDvPx;
        const int cp = (int)((N - p0) < kDvPx ? (N - p0) : kDvPx);
        const uint32_t cb = (uint32_t)((size_t)cp * B * sizeof(In)) & ~15u;
        const uint32_t db = ld == k ? (uint32_t)((size_t)cp * k * 4) & ~15u : 0u;
        mbar_expect_tx(&sy->full[s], cb + db);
        if (cb) bulk_g2s(cst + (size_t)s * cube_stage, cube + p0 * B, cb, &sy->full[s]);
        if (db) bulk_g2s(reinterpret_cast<unsigned char*>(dqst) + (size_t)s * dq_stage, dq + p0 * k, db,
                         &sy->full[s]);
      }
    }
    return;
  }
  const int grp = tid / 256, b = tid % 256;  // pixel group, this thread's band
  float4 acc[KQ];
#pragma unroll
  for (int q = 0; q < KQ; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  float csum = 0.f;                     // column sum of dQ (threads j < k)
  float xmax = 0.f, dmax = 0.f;         // largest |x_b| and |dq_j| (operand scales of dY)
  const float m = b < B ? mus[b] : 0.f;
  int c = 0;
  for (; c < nch; ++c) {
    const int s = c % nst;
    int ok = 1;
    if (lane == 0) ok = mbar_wait(&sy->full[s], (c / nst) & 1, &sy->abort) ? 1 : 0;
    ok = __shfl_sync(kFull, ok, 0);
    if (!dv_and<kComp>(ok)) break;
    const int64_t p0 = (c_begin + c) * kDvPx;
    const int cp = (int)((N - p0) < kDvPx ? (N - p0) : kDvPx);
    const In* xs = reinterpret_cast<const In*>(cst + (size_t)s * cube_stage);
    const float* ds = dqst + (size_t)s * dq_stage / 4;
    const int copied_x = (int)((((size_t)cp * B * sizeof(In)) & ~(size_t)15) / sizeof(In));
    const int copied_d = ld == k ? (int)((((size_t)cp * k * 4) & ~(size_t)15) / 4) : 0;
    const bool whole = copied_x == cp * B;
    // dQ rows of this chunk padded to 16-byte rows (two buffers by chunk
    // parity), so that every pixel's row is read as KQ vectors
    float4* dqp = dqpad + (size_t)(c & 1) * kDvPx * KQ;
    for (int e = tid; e < cp * KQ * 4; e += kComp) {
      const int pp = e / (KQ * 4), j = e - pp * (KQ * 4);
      const int ed = pp * k + j;
      reinterpret_cast<float*>(dqp)[e] =
          j < k ? (ed < copied_d ? ds[ed] : dq[(p0 + pp) * ld + j0 + j]) : 0.f;
    }
    dv_sync<kComp>();
    for (int p = grp; p < cp; p += kGroups) {
      float x = 0.f;
      float dv[KQ * 4];
      if (whole) {
        if (b < B) x = to_f32<In>(xs[p * B + b]) - m;
      } else {
        const int ex = p * B + b;
        if (b < B) x = (ex < copied_x ? to_f32<In>(xs[ex]) : to_f32<In>(cube[p0 * B + ex])) - m;
      }
#pragma unroll
      for (int q = 0; q < KQ; ++q) {
        const float4 v = dqp[p * KQ + q];
        dv[4 * q] = v.x; dv[4 * q + 1] = v.y; dv[4 * q + 2] = v.z; dv[4 * q + 3] = v.w;
      }
      xmax = fmaxf(xmax, fabsf(x));
#pragma unroll
      for (int q = 0; q < KQ; ++q) {
        acc[q].x = fmaf(x, dv[4 * q], acc[q].x);
        acc[q].y = fmaf(x, dv[4 * q + 1], acc[q].y);
        acc[q].z = fmaf(x, dv[4 * q + 2], acc[q].z);
        acc[q].w = fmaf(x, dv[4 * q + 3], acc[q].w);
      }
      if (b < k) {
        const float d = reinterpret_cast<const float*>(dqp)[p * KQ * 4 + b];
        csum += d;
        dmax = fmaxf(dmax, fabsf(d));
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sy->empty[s]);
  }
  if (c < nch && tid == 0 && hdr) set_status(hdr, PCA_ERR_TIMEOUT);
  // the other groups hand their sums to the first through shared memory, one
  // group and one column quad at a time
  float* out = dv_part + ((size_t)g * B + b) * ld + j0;
#pragma unroll
  for (int q = 0; q < KQ; ++q) {
    for (int h = 1; h < kGroups; ++h) {
      if (grp == h) sy->comb[b] = acc[q];
      dv_sync<kComp>();
      if (grp == 0) {
        const float4 o = sy->comb[b];
        acc[q].x += o.x; acc[q].y += o.y; acc[q].z += o.z; acc[q].w += o.w;
      }
      dv_sync<kComp>();
    }
    if (grp == 0 && b < B) {
      const float v[4] = {acc[q].x, acc[q].y, acc[q].z, acc[q].w};
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (4 * q + t < k) out[4 * q + t] = v[t];
    }
  }
  for (int h = 1; h < kGroups; ++h) {
    if (grp == h) {
      sy->combv[0][b] = xmax;
      sy->combv[1][b] = csum;
      sy->combv[2][b] = dmax;
    }
    dv_sync<kComp>();
    if (grp == 0) {
      xmax = fmaxf(xmax, sy->combv[0][b]);
      csum += sy->combv[1][b];
      dmax = fmaxf(dmax, sy->combv[2][b]);
    }
    dv_sync<kComp>();
  }
  if (grp == 0) {
    if (b < k) {
      dqs_part[(size_t)g * ld + j0 + b] = csum;
      dqmax_part[(size_t)g * ld + j0 + b] = dmax;
    }
    if (b < B) xmax_part[(size_t)g * B + b] = xmax;
  }
}

// ------------------------------------------------------------------ k_bwd_reduce
// dVk[b][j] = sum over the partials (FP64), FP32 copy of mu; the CTAs of band 0
// also form the column means of dQ.  One CTA per band and group of 32 columns:
// warp w adds the partials w, w + 8, ... for every column (lane = column), then
// the eight warp sums.
constexpr int kRedWarps = 8;

__global__ void __launch_bounds__(kRedWarps * 32)
k_bwd_reduce(const float* __restrict__ dv_part, const float* __restrict__ dqs_part, int parts,
             int64_t N, int B, int k, const double* __restrict__ mu, double* __restrict__ dVk,
             float* __restrict__ mdq, float* __restrict__ mu32) {
  __shared__ double red[2][kRedWarps][32];
  const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = 32 * blockIdx.y + lane;
  double s = 0.0, t = 0.0;
  if (j < k) {
    for (int gg = warp; gg < parts; gg += kRedWarps) {
      s += (double)dv_part[((size_t)gg * B + b) * k + j];
      if (b == 0) t += (double)dqs_part[(size_t)gg * k + j];
    }
  }
  red[0][warp][lane] = s;
  red[1][warp][lane] = t;
  __syncthreads();
  if (warp == 0 && j < k) {
    double a = 0.0, c = 0.0;
#pragma unroll
    for (int w = 0; w < kRedWarps; ++w) { a += red[0][w][lane]; c += red[1][w][lane]; }
    dVk[(size_t)b * k + j] = a;
    if (b == 0) mdq[j] = (float)(c / (double)N);
  }
  if (threadIdx.x == 0 && blockIdx.y == 0) mu32[b] = (float)mu[b];
}

// ------------------------------------------------------------------ k_bwd_m
// G_ij = F_ij (V^T dVk)_ij for j < k (i != j), G_jj = dlam_j.  One CTA per
// row i and group of 32 columns; thread = band b, the products summed by
// shuffles and shared memory.
__global__ void __launch_bounds__(256)
k_bwd_m(int B, int k, const double* __restrict__ lam, const double* __restrict__ V,
        const double* __restrict__ dVk, const double* __restrict__ dlam, double gap_eps,
        double* __restrict__ Gk) {
  __shared__ double part[8][32];
  const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int jc = 32 * blockIdx.y, nj = k - jc < 32 ? k - jc : 32;
  const double v = tid < B ? V[(size_t)tid * B + i] : 0.0;
  for (int jj = 0; jj < nj; ++jj) {
    double m = tid < B ? v * dVk[(size_t)tid * k + jc + jj] : 0.0;
    m = warp_sum(m);
    if (lane == 0) part[warp][jj] = m;
  }
  __syncthreads();
  if (tid < nj) {
    const int j = jc + tid;
    double m = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) m += part[w][tid];
    double gval;
    if (i == j) {
      gval = dlam ? dlam[i] : 0.0;
    } else {
      const double gap = lam[j] - lam[i];
      gval = fabs(gap) > gap_eps * fabs(lam[0]) ? m / gap : 0.0;
    }
    Gk[(size_t)i * k + j] = gval;
  }
}

// ------------------------------------------------------------------ k_bwd_s
// dA = V G V^T = T V^T with T = V G: T_aj = sum_i V_ai G_ij for j < k (plus
// V_aj dlam_j for j >= k), and V_k in FP32.  One CTA per row a.
__global__ void __launch_bounds__(256)
k_bwd_s(const double* __restrict__ V, const double* __restrict__ Gk, const double* __restrict__ dlam,
        int64_t N, int B, int k, double* __restrict__ dA, float* __restrict__ vk32) {
  __shared__ double T[256];
  __shared__ double part[8][256];
  const int a = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double vai = tid < B ? V[(size_t)a * B + tid] : 0.0;   // thread = i
  for (int j = 0; j < k; ++j) {
    double t = tid < B ? vai * Gk[(size_t)tid * k + j] : 0.0;
    t = warp_sum(t);
    if (lane == 0) part[warp][j] = t;
  }
  __syncthreads();
  if (tid < B) {
    double t;
    if (tid < k) {
      t = 0.0;
#pragma unroll
      for (int w = 0; w < 8; ++w) t += part[w][tid];
      vk32[(size_t)a * k + tid] = (float)vai;
    } else {
      t = dlam ? vai * dlam[tid] : 0.0;
    }
    T[tid] = t;
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

template <typename In, int KQ>
cudaError_t dv_kq(const In* cube, const float* dq, int64_t N, int B, int k, int j0, int ld,
                  const double* mu, float* dv_part, float* dqs_part, float* xmax_part,
                  float* dqmax_part, int parts, DevHeader* hdr, cudaStream_t st) {
  const int cube_stage = (int)((((size_t)kDvPx * B * sizeof(In)) + 127) & ~(size_t)127);
  const int dq_stage = ld == k ? (int)((((size_t)kDvPx * k * 4) + 127) & ~(size_t)127) : 0;
  // three stages where they fit in the 227 KB a CTA may use (all but the
  // largest FP32 shapes), else two
  auto bytes = [&](int n) {
    return (size_t)n * (cube_stage + dq_stage) + 256 * 4 + (size_t)2 * kDvPx * KQ * 16 + sizeof(DvSync);
  };
  const int nst = bytes(kDvStages) <= (size_t)227 * 1024 ? kDvStages : 2;
  const size_t smem = bytes(nst);
  auto kern = k_bwd_dv<In, KQ>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<parts, dv_threads(KQ), smem, st>>>(cube, dq, N, B, k, j0, ld, mu, dv_part, dqs_part,
                                            xmax_part, dqmax_part, cube_stage, dq_stage, nst, hdr);
  return cudaGetLastError();
}

// X^T dQ in passes of at most 32 columns (the accumulators live in registers)
template <typename In>
cudaError_t dv_typed(const In* cube, const float* dq, int64_t N, int B, int k, const double* mu,
                     const BwdPtrs& w, DevHeader* hdr, cudaStream_t st) {
  for (int j0 = 0; j0 < k; j0 += 32) {
    const int kk = k - j0 < 32 ? k - j0 : 32;
    cudaError_t e = cudaErrorInvalidValue;
    switch ((kk + 3) / 4) {
#define GB_DV_CASE(q) \
      case q: e = dv_kq<In, q>(cube, dq, N, B, kk, j0, k, mu, w.dv_part, w.dqs_part, w.xmax_part, \
                               w.dqmax_part, w.parts, hdr, st); break;
      GB_DV_CASE(1) GB_DV_CASE(2) GB_DV_CASE(3) GB_DV_CASE(4)
      GB_DV_CASE(5) GB_DV_CASE(6) GB_DV_CASE(7) GB_DV_CASE(8)
#undef GB_DV_CASE
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_backward(const void* cube, pca_dtype dt, int64_t N, int B, int k,
                            const double* mu, const double* lam, const double* V,
                            const float* dq, const double* dlam, double gap_eps, float* dY,
                            const BwdPtrs& w, DevHeader* hdr, cudaStream_t st) {
  cudaError_t e;
  switch (dt) {
    case PCA_F32: e = dv_typed((const float*)cube, dq, N, B, k, mu, w, hdr, st); break;
    case PCA_BF16: e = dv_typed((const __nv_bfloat16*)cube, dq, N, B, k, mu, w, hdr, st); break;
    case PCA_F16: e = dv_typed((const __half*)cube, dq, N, B, k, mu, w, hdr, st); break;
    default:
      return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  const int kg = (k + 31) / 32;   // groups of 32 columns
  k_bwd_reduce<<<dim3(B, kg), kRedWarps * 32, 0, st>>>(w.dv_part, w.dqs_part, w.parts, N, B, k,
                                                       mu, w.dVk, w.mdq, w.mu32);
  k_bwd_m<<<dim3(B, kg), 256, 0, st>>>(B, k, lam, V, w.dVk, dlam, gap_eps, w.Gk);
  k_bwd_s<<<B, 256, 0, st>>>(V, w.Gk, dlam, N, B, k, w.dA, w.vk32);
  k_bwd_sym<<<dim3((B + 127) / 128, B), 128, 0, st>>>(w.dA, N, B, w.S32);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // dY on the tensor cores (k_bwd_dy_tc.cu)
  return launch_bwd_dy_tc(cube, dt, dq, N, B, k, w.xmax_part, w.dqmax_part, w.parts, w.mu32,
                          w.mdq, w.S32, w.vk32, w.ascale, w.anshift, w.bop, w.fcol, dY, hdr, st);
}

}  // namespace gbpca
