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

// Q[n][j] = sum_b (Y_nb - mu_b) V_bj, FP32.  Each thread computes two pixels
// so that every 16-byte V_k load from shared memory feeds eight FMAs; V_k
// rows are padded to KQ float4 groups, mu sits beside them.  Rows are read
// 16 bands at a time (four 16-byte loads in flight per pixel).
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
  const int64_t half = (N + 1) / 2;
  const int64_t stride = (int64_t)gridDim.x * kProjThreads;
  for (int64_t n0 = (int64_t)blockIdx.x * kProjThreads + threadIdx.x; n0 < half; n0 += stride) {
    const int64_t n1 = n0 + half;
    const bool two = n1 < N;
    float4 a0[KQ], a1[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) { a0[q] = make_float4(0.f, 0.f, 0.f, 0.f); a1[q] = a0[q]; }
    const In* row0 = cube + n0 * (int64_t)B;
    const In* row1 = cube + (two ? n1 : n0) * (int64_t)B;
    auto accum = [&](float x0, float x1, int b) {
      const float m = mus[b];
      x0 -= m;
      x1 -= m;
#pragma unroll
      for (int q = 0; q < KQ; ++q) {
        const float4 v = v4[b * KQ + q];
        a0[q].x = fmaf(x0, v.x, a0[q].x); a1[q].x = fmaf(x1, v.x, a1[q].x);
        a0[q].y = fmaf(x0, v.y, a0[q].y); a1[q].y = fmaf(x1, v.y, a1[q].y);
        a0[q].z = fmaf(x0, v.z, a0[q].z); a1[q].z = fmaf(x1, v.z, a1[q].z);
        a0[q].w = fmaf(x0, v.w, a0[q].w); a1[q].w = fmaf(x1, v.w, a1[q].w);
      }
    };
    if constexpr (kVec4) {
      const float4* p0 = reinterpret_cast<const float4*>(row0);
      const float4* p1 = reinterpret_cast<const float4*>(row1);
      const int nb4 = B / 4;
      int b4 = 0;
      for (; b4 + 4 <= nb4; b4 += 4) {
        float4 y0[4], y1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { y0[u] = __ldg(p0 + b4 + u); y1[u] = __ldg(p1 + b4 + u); }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          accum(y0[u].x, y1[u].x, 4 * (b4 + u));
          accum(y0[u].y, y1[u].y, 4 * (b4 + u) + 1);
          accum(y0[u].z, y1[u].z, 4 * (b4 + u) + 2);
          accum(y0[u].w, y1[u].w, 4 * (b4 + u) + 3);
        }
      }
      for (; b4 < nb4; ++b4) {
        const float4 y0 = __ldg(p0 + b4), y1 = __ldg(p1 + b4);
        accum(y0.x, y1.x, 4 * b4);
        accum(y0.y, y1.y, 4 * b4 + 1);
        accum(y0.z, y1.z, 4 * b4 + 2);
        accum(y0.w, y1.w, 4 * b4 + 3);
      }
    } else {
      int b = 0;
      for (; b + 8 <= B; b += 8) {
        float y0[8], y1[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) { y0[u] = to_f32<In>(row0[b + u]); y1[u] = to_f32<In>(row1[b + u]); }
#pragma unroll
        for (int u = 0; u < 8; ++u) accum(y0[u], y1[u], b + u);
      }
      for (; b < B; ++b) accum(to_f32<In>(row0[b]), to_f32<In>(row1[b]), b);
    }
    float* out0 = proj + n0 * (int64_t)k;
    float* out1 = proj + n1 * (int64_t)k;
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
      const float v0[4] = {a0[q].x, a0[q].y, a0[q].z, a0[q].w};
      const float v1[4] = {a1[q].x, a1[q].y, a1[q].z, a1[q].w};
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (4 * q + t < k) {
          out0[4 * q + t] = v0[t];
          if (two) out1[4 * q + t] = v1[t];
        }
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
  const int64_t want = ((N + 1) / 2 + kProjThreads - 1) / kProjThreads;
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
