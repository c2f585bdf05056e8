// k_finalize.cu -- eigen-pair extraction, descending sort and sign rule
// (Sec. 4.2 stage 4.3), and the projection of the centred cube onto the
// first k eigenvectors (Algorithm 1 stages 5-6; Sec. 4.2 stage 5).
#include "common.cuh"

namespace gbpca {

namespace {

// Sort and sign rule in two fully parallel passes.
// k_rank_sign: one CTA per eigen-pair j.  Its rank = number of eigenvalues
// that sort before it (larger, or equal and at a lower position) -- no
// comparison sort needed for B <= 232 -- and the sign that makes the entry of
// largest magnitude (lowest row on ties) of column j positive.
__global__ void __launch_bounds__(256)
k_rank_sign(const double* __restrict__ lam, const float2* __restrict__ vc, int B,
            int* __restrict__ rank, double* __restrict__ sgn, double* __restrict__ eigvals) {
  __shared__ int cnt[8];
  __shared__ double bv[8];
  __shared__ int bi[8];
  const int j = blockIdx.x, i = threadIdx.x, lane = i & 31, warp = i >> 5;
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

// k_scatter: one CTA per row i of V writes row i of the sorted, signed eigvecs.
__global__ void __launch_bounds__(256)
k_scatter(const float2* __restrict__ vc, int B, int k, const int* __restrict__ rank,
          const double* __restrict__ sgn, double* __restrict__ eigvecs, float* __restrict__ vk) {
  const int i = blockIdx.x;
  for (int j = threadIdx.x; j < B; j += blockDim.x) {
    const float2 x = vc[(size_t)i * B + j];
    const double v = sgn[j] * ((double)x.x + (double)x.y);
    const int r = rank[j];
    eigvecs[(size_t)i * B + r] = v;
    if (r < k) vk[(size_t)i * k + r] = (float)v;
  }
}

// Q[n][j] = sum_b (Y_nb - mu_b) V_bj, FP32, one pixel per thread.  V_k and mu
// sit in shared memory; V_k rows are padded to KQ float4 groups so one
// 16-byte load feeds four FMAs.
constexpr int kProjThreads = 256;

template <typename In, int KQ, bool kVec4>
__global__ void __launch_bounds__(kProjThreads)
k_project(const In* __restrict__ cube, int64_t N, int B, int k, const float* __restrict__ mu_f,
          const float* __restrict__ vk, float* __restrict__ proj) {
  extern __shared__ __align__(16) float sm[];
  float4* v4 = reinterpret_cast<float4*>(sm);      // [B][KQ]
  float* mus = sm + (size_t)B * KQ * 4;             // [B]
  for (int e = threadIdx.x; e < B * KQ * 4; e += kProjThreads) {
    const int b = e / (KQ * 4), j = e - b * (KQ * 4);
    sm[e] = j < k ? vk[(size_t)b * k + j] : 0.f;
  }
  for (int b = threadIdx.x; b < B; b += kProjThreads) mus[b] = mu_f[b];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * kProjThreads;
  for (int64_t n = (int64_t)blockIdx.x * kProjThreads + threadIdx.x; n < N; n += stride) {
    float4 acc[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    const In* row = cube + n * (int64_t)B;
    auto accum = [&](float x, int b) {
      x -= mus[b];
#pragma unroll
      for (int q = 0; q < KQ; ++q) {
        const float4 v = v4[b * KQ + q];
        acc[q].x = fmaf(x, v.x, acc[q].x);
        acc[q].y = fmaf(x, v.y, acc[q].y);
        acc[q].z = fmaf(x, v.z, acc[q].z);
        acc[q].w = fmaf(x, v.w, acc[q].w);
      }
    };
    if constexpr (kVec4) {
      // 16 bands per batch: four 16-byte loads in flight per thread before the FMAs
      const float4* r4 = reinterpret_cast<const float4*>(row);
      const int nb4 = B / 4;
      int b4 = 0;
      for (; b4 + 4 <= nb4; b4 += 4) {
        float4 y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) y[u] = __ldg(r4 + b4 + u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          accum(y[u].x, 4 * (b4 + u));
          accum(y[u].y, 4 * (b4 + u) + 1);
          accum(y[u].z, 4 * (b4 + u) + 2);
          accum(y[u].w, 4 * (b4 + u) + 3);
        }
      }
      for (; b4 < nb4; ++b4) {
        const float4 y = __ldg(r4 + b4);
        accum(y.x, 4 * b4);
        accum(y.y, 4 * b4 + 1);
        accum(y.z, 4 * b4 + 2);
        accum(y.w, 4 * b4 + 3);
      }
    } else {
      int b = 0;
      for (; b + 8 <= B; b += 8) {
        float y[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) y[u] = to_f32<In>(row[b + u]);
#pragma unroll
        for (int u = 0; u < 8; ++u) accum(y[u], b + u);
      }
      for (; b < B; ++b) accum(to_f32<In>(row[b]), b);
    }
    float* out = proj + n * (int64_t)k;
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
      const float vals[4] = {acc[q].x, acc[q].y, acc[q].z, acc[q].w};
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (4 * q + t < k) out[4 * q + t] = vals[t];
    }
  }
}

template <typename In, int KQ>
cudaError_t project_kq(const In* cube, int64_t N, int B, int k, const float* mu_f,
                       const float* vk, float* proj, cudaStream_t st, bool vec4) {
  const size_t smem = ((size_t)B * KQ * 4 + B) * sizeof(float);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (N + kProjThreads - 1) / kProjThreads;
  const int blocks = (int)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
  if (vec4) {
    auto kern = k_project<In, KQ, true>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<blocks, kProjThreads, smem, st>>>(cube, N, B, k, mu_f, vk, proj);
  } else {
    auto kern = k_project<In, KQ, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<blocks, kProjThreads, smem, st>>>(cube, N, B, k, mu_f, vk, proj);
  }
  return cudaGetLastError();
}

template <typename In>
cudaError_t project_typed(const In* cube, int64_t N, int B, int k, const float* mu_f,
                          const float* vk, float* proj, cudaStream_t st, bool vec4) {
  const int kq = (k + 3) / 4;
  switch (kq) {
    case 1: return project_kq<In, 1>(cube, N, B, k, mu_f, vk, proj, st, vec4);
    case 2: return project_kq<In, 2>(cube, N, B, k, mu_f, vk, proj, st, vec4);
    case 3: return project_kq<In, 3>(cube, N, B, k, mu_f, vk, proj, st, vec4);
    case 4: return project_kq<In, 4>(cube, N, B, k, mu_f, vk, proj, st, vec4);
    case 5: return project_kq<In, 5>(cube, N, B, k, mu_f, vk, proj, st, vec4);
    case 6: return project_kq<In, 6>(cube, N, B, k, mu_f, vk, proj, st, vec4);
    case 7: return project_kq<In, 7>(cube, N, B, k, mu_f, vk, proj, st, vec4);
    case 8: return project_kq<In, 8>(cube, N, B, k, mu_f, vk, proj, st, vec4);
  }
  return cudaErrorInvalidValue;
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

cudaError_t launch_project(const void* cube, pca_dtype dt, int64_t N, int B, int k,
                           const float* mu_f, const float* vk, float* proj, cudaStream_t st) {
  const bool vec4 = dt == PCA_F32 && (B % 4) == 0 && ((uintptr_t)cube % 16) == 0;
  switch (dt) {
    case PCA_F32: return project_typed((const float*)cube, N, B, k, mu_f, vk, proj, st, vec4);
    case PCA_BF16:
      return project_typed((const __nv_bfloat16*)cube, N, B, k, mu_f, vk, proj, st, false);
    case PCA_F16: return project_typed((const __half*)cube, N, B, k, mu_f, vk, proj, st, false);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbpca
