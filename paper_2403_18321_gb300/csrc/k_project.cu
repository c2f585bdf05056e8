// k_project.cu -- projection of the centred cube onto the first k
// eigenvectors, Q = (Y - 1 mu^T) V_k (Algorithm 1 stages 5-6; Sec. 4.2
// stage 5), FP32 arithmetic.
//
// A streaming kernel: one persistent CTA per SM walks a contiguous range of
// 64-pixel chunks.  Warp 8 is the TMA producer; it fills a ring of stages
// with each chunk --
//   tiled:   when a pixel row is a whole number of 16-byte units, as 128-byte
//            wide boxes of a 2-D tensor map with the 128-byte swizzle, so that
//            the eight 16-byte units of a box row land in a different bank
//            group for each of eight consecutive pixels;
//   untiled: otherwise, as one contiguous bulk copy (the odd row stride then
//            spreads consecutive pixels over the banks by itself).
// Warps 0-7 each take one eighth of the bands for the same 64 pixels (two
// pixels per lane), accumulate x * V_k in registers with V_k and mu read as
// broadcasts from shared memory, and the eight partial sums are added through
// shared memory before the chunk's k columns are stored.  Every wait is
// bounded; on time-out the CTA fills the rest of its output range with NaN
// and records PCA_ERR_TIMEOUT when a header is given.
#include "tma.cuh"

namespace gbpca {

namespace {

constexpr int kPc = 64;                  // pixels per chunk
constexpr int kParts = 8;                // compute warps (band parts)
constexpr int kCompute = kParts * 32;
constexpr int kThreadsP = kCompute + 32;
constexpr int kMaxStages = 8;
constexpr int kMaxU = (kMaxB + 4 * kParts - 1) / (4 * kParts);  // 16-byte units per band part

struct __align__(8) ProjSync {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  int abort;
};

__device__ __forceinline__ void named_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kCompute) : "memory");
}
__device__ __forceinline__ int named_and(int v) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n"
      " selp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(v), "n"(kCompute)
      : "memory");
  return r;
}

template <typename In>
__device__ __forceinline__ void unpack16(const uint4& u, float* v);
template <>
__device__ __forceinline__ void unpack16<float>(const uint4& u, float* v) {
  v[0] = __uint_as_float(u.x); v[1] = __uint_as_float(u.y);
  v[2] = __uint_as_float(u.z); v[3] = __uint_as_float(u.w);
}
template <>
__device__ __forceinline__ void unpack16<__nv_bfloat16>(const uint4& u, float* v) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}
template <>
__device__ __forceinline__ void unpack16<__half>(const uint4& u, float* v) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __half2float(__ushort_as_half((unsigned short)(w[i] & 0xffffu)));
    v[2 * i + 1] = __half2float(__ushort_as_half((unsigned short)(w[i] >> 16)));
  }
}

template <int KQ>
__device__ __forceinline__ void fma_band(float x0, float x1, const float4* __restrict__ vrow,
                                         float4* a0, float4* a1) {
#pragma unroll
  for (int q = 0; q < KQ; ++q) {
    const float4 v = vrow[q];
    a0[q].x = fmaf(x0, v.x, a0[q].x); a1[q].x = fmaf(x1, v.x, a1[q].x);
    a0[q].y = fmaf(x0, v.y, a0[q].y); a1[q].y = fmaf(x1, v.y, a1[q].y);
    a0[q].z = fmaf(x0, v.z, a0[q].z); a1[q].z = fmaf(x1, v.z, a1[q].z);
    a0[q].w = fmaf(x0, v.w, a0[q].w); a1[q].w = fmaf(x1, v.w, a1[q].w);
  }
}

struct ProjArgs {
  const void* cube;
  int64_t N;
  int B, k;
  const float* mu_f;
  const float* vk;
  float* proj;
  int stages, stage_bytes;
  DevHeader* hdr;
};

template <typename In, int KQ, bool kTiled>
__global__ void __launch_bounds__(kThreadsP, 1)
k_project(const __grid_constant__ CUtensorMap tmap, const ProjArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned start (the 128-byte swizzle repeats every 1024 bytes);
  // offsetting the array itself keeps every access a shared-memory one
  unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  constexpr int E = 16 / (int)sizeof(In);           // elements per 16-byte unit
  const In* cube = static_cast<const In*>(a.cube);
  const int64_t N = a.N;
  const int B = a.B, k = a.k, S = a.stages;
  const int B8 = (B + 7) & ~7;
  unsigned char* stages = smem;
  float4* vs = reinterpret_cast<float4*>(stages + (size_t)S * a.stage_bytes);  // [B8][KQ]
  float* mus = reinterpret_cast<float*>(vs + (size_t)B8 * KQ);                  // [B8]
  float* red = mus + B8;                                                        // [kParts][kPc][k]
  ProjSync* sy = reinterpret_cast<ProjSync*>(red + (size_t)kParts * kPc * k);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x, g = blockIdx.x;
  const int64_t nch_total = (N + kPc - 1) / kPc;
  const int64_t c_begin = nch_total * g / G, c_end = nch_total * (g + 1) / G;
  const int nch = (int)(c_end - c_begin);

  if (tid == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&sy->full[s], 1); mbar_init(&sy->empty[s], kParts); }
    sy->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // the producer starts streaming at once; the compute warps stage V_k and mu
  // meanwhile and meet at their own barrier
  if (warp < kParts) {
    for (int e = tid; e < B8 * KQ * 4; e += kCompute) {
      const int b = e / (KQ * 4), j = e - b * (KQ * 4);
      reinterpret_cast<float*>(vs)[e] = (b < B && j < k) ? a.vk[(size_t)b * k + j] : 0.f;
    }
    for (int b = tid; b < B8; b += kCompute) mus[b] = b < B ? a.mu_f[b] : 0.f;
    named_sync();
  }

  if (warp == kParts) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      const int nbox = (B * (int)sizeof(In) + 127) / 128;
      for (int c = 0; c < nch; ++c) {
        const int s = c % S;
        if (!mbar_wait(&sy->empty[s], ((c / S) & 1) ^ 1, &sy->abort)) break;
        const int64_t p0 = (c_begin + c) * kPc;
        unsigned char* dst = stages + (size_t)s * a.stage_bytes;
        if constexpr (kTiled) {
          mbar_expect_tx(&sy->full[s], (uint32_t)(nbox * kPc * 128));
          for (int bx = 0; bx < nbox; ++bx)
            tma_load_2d(dst + (size_t)bx * kPc * 128, &tmap, bx * (128 / (int)sizeof(In)), (int)p0,
                        &sy->full[s]);
        } else {
          const int cp = (int)((N - p0) < kPc ? (N - p0) : kPc);
          const uint32_t bytes = (uint32_t)((size_t)cp * B * sizeof(In)) & ~15u;
          mbar_expect_tx(&sy->full[s], bytes);
          if (bytes) bulk_g2s(dst, cube + p0 * B, bytes, &sy->full[s]);
        }
      }
    }
    return;
  }

  // -------------------------------------------------------------- compute
  const int h = warp;
  const int pa = lane, pb = lane + 32;
  int c = 0;
  for (; c < nch; ++c) {
    const int s = c % S;
    int ok = 1;
    if (lane == 0) ok = mbar_wait(&sy->full[s], (c / S) & 1, &sy->abort) ? 1 : 0;
    ok = __shfl_sync(kFull, ok, 0);
    if (!named_and(ok)) break;
    const int64_t p0 = (c_begin + c) * kPc;
    const int cp = (int)((N - p0) < kPc ? (N - p0) : kPc);
    const unsigned char* st = stages + (size_t)s * a.stage_bytes;
    float4 a0[KQ], a1[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) { a0[q] = make_float4(0.f, 0.f, 0.f, 0.f); a1[q] = a0[q]; }
    if constexpr (kTiled) {
      const int G16 = B / E;                       // 16-byte units per pixel row
      for (int u = h; u < G16; u += kParts) {
        const unsigned char* box = st + (size_t)(u >> 3) * kPc * 128;
        const int sw = ((u & 7) ^ (pa & 7)) << 4;    // pb & 7 == pa & 7
        const uint4 r0 = *reinterpret_cast<const uint4*>(box + pa * 128 + sw);
        const uint4 r1 = *reinterpret_cast<const uint4*>(box + pb * 128 + sw);
        float y0[E], y1[E];
        unpack16<In>(r0, y0);
        unpack16<In>(r1, y1);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int b = u * E + e;
          const float m = mus[b];
          fma_band<KQ>(y0[e] - m, y1[e] - m, vs + (size_t)b * KQ, a0, a1);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sy->empty[s]);   // this warp is done with the stage
    } else {
      // bands 4u .. 4u+3 for u = h, h + 8, ...: at most kMaxU groups per part,
      // read four groups at a time; the stage is released after the reads of
      // the last four
      const In* sp = reinterpret_cast<const In*>(st);
      const size_t copied = (((size_t)cp * B * sizeof(In)) & ~(size_t)15) / sizeof(In);
      const bool whole = cp == kPc && copied == (size_t)kPc * B;
      const In* gp = cube + p0 * B;
      const int ng = (B + 3) / 4;
      const int mine = ng > h ? (ng - h + kParts - 1) / kParts : 0;   // groups of this part
      if (mine == 0) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&sy->empty[s]);
      }
      for (int i0 = 0; i0 < mine; i0 += 4) {
        float y0[4][4], y1[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int b = 4 * (h + kParts * (i0 + i)) + e;
            float v0 = 0.f, v1 = 0.f;
            if (i0 + i < mine && b < B) {
              if (whole) {
                v0 = to_f32<In>(sp[pa * B + b]);
                v1 = to_f32<In>(sp[pb * B + b]);
              } else {
                const size_t e0 = (size_t)pa * B + b, e1 = (size_t)pb * B + b;
                if (pa < cp) v0 = e0 < copied ? to_f32<In>(sp[e0]) : to_f32<In>(gp[e0]);
                if (pb < cp) v1 = e1 < copied ? to_f32<In>(sp[e1]) : to_f32<In>(gp[e1]);
              }
            }
            y0[i][e] = v0;
            y1[i][e] = v1;
          }
        }
        if (i0 + 4 >= mine) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&sy->empty[s]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int b = 4 * (h + kParts * (i0 + i)) + e;
            if (i0 + i < mine && b < B) {
              const float m = mus[b];
              fma_band<KQ>(y0[i][e] - m, y1[i][e] - m, vs + (size_t)b * KQ, a0, a1);
            }
          }
        }
      }
    }
    // partial sums of this band part -> shared, then the eight parts are added
    float* rp = red + (size_t)h * kPc * k;
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
      const float v0[4] = {a0[q].x, a0[q].y, a0[q].z, a0[q].w};
      const float v1[4] = {a1[q].x, a1[q].y, a1[q].z, a1[q].w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int j = 4 * q + t;
        if (j < k) { rp[pa * k + j] = v0[t]; rp[pb * k + j] = v1[t]; }
      }
    }
    named_sync();
    float* out = a.proj + p0 * k;
    for (int o = tid; o < cp * k; o += kCompute) {
      float sum = 0.f;
#pragma unroll
      for (int hh = 0; hh < kParts; ++hh) sum += red[(size_t)hh * kPc * k + o];
      out[o] = sum;
    }
    named_sync();
  }
  if (c < nch) {
    // a bounded wait gave up: make the rest of this CTA's range visibly invalid
    const int64_t o0 = (c_begin + c) * kPc * k;
    const int64_t o1 = (c_end * kPc < N ? c_end * kPc : N) * k;
    for (int64_t o = o0 + tid; o < o1; o += kCompute) a.proj[o] = __int_as_float(0x7fc00000);
    if (tid == 0 && a.hdr) set_status(a.hdr, PCA_ERR_TIMEOUT);
  }
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link-time
// dependence on the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

template <typename In> constexpr CUtensorMapDataType tmap_type();
template <> constexpr CUtensorMapDataType tmap_type<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> constexpr CUtensorMapDataType tmap_type<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }
template <> constexpr CUtensorMapDataType tmap_type<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }

template <typename In, int KQ>
cudaError_t project_kq(const In* cube, int64_t N, int B, int k, const float* mu_f, const float* vk,
                       float* proj, DevHeader* hdr, cudaStream_t st) {
  CUtensorMap tmap;
  memset(&tmap, 0, sizeof(tmap));
  bool tiled = (B * sizeof(In)) % 16 == 0 && ((uintptr_t)cube % 16) == 0 && N < (1ll << 31) &&
               encode_fn() != nullptr;
  if (tiled) {
    const cuuint64_t gdim[2] = {(cuuint64_t)B, (cuuint64_t)N};
    const cuuint64_t gstride[1] = {(cuuint64_t)B * sizeof(In)};
    const cuuint32_t box[2] = {(cuuint32_t)(128 / sizeof(In)), (cuuint32_t)kPc};
    const cuuint32_t estr[2] = {1, 1};
    tiled = encode_fn()(&tmap, tmap_type<In>(), 2, const_cast<In*>(cube), gdim, gstride, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  const int B8 = (B + 7) & ~7;
  const int nbox = (B * (int)sizeof(In) + 127) / 128;
  const int stage_bytes = tiled ? nbox * kPc * 128
                                : (int)((((size_t)kPc * B * sizeof(In)) + 1023) & ~(size_t)1023);
  const size_t fixed = (size_t)B8 * KQ * 16 + (size_t)B8 * 4 + (size_t)kParts * kPc * k * 4 +
                       sizeof(ProjSync) + 1024;
  const size_t budget = 227 * 1024;
  int stages = (int)((budget - fixed) / stage_bytes);
  stages = stages > kMaxStages ? kMaxStages : stages;
  if (stages < 2) return cudaErrorInvalidValue;
  const size_t smem = fixed + (size_t)stages * stage_bytes;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nch = (N + kPc - 1) / kPc;
  const int grid = (int)(nch < sms ? nch : sms);
  ProjArgs a{cube, N, B, k, mu_f, vk, proj, stages, stage_bytes, hdr};
  auto kern = tiled ? k_project<In, KQ, true> : k_project<In, KQ, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreadsP, smem, st>>>(tmap, a);
  return cudaGetLastError();
}

template <typename In>
cudaError_t project_typed(const In* cube, int64_t N, int B, int k, const float* mu_f,
                          const float* vk, float* proj, DevHeader* hdr, cudaStream_t st) {
  switch ((k + 3) / 4) {
    case 1: return project_kq<In, 1>(cube, N, B, k, mu_f, vk, proj, hdr, st);
    case 2: return project_kq<In, 2>(cube, N, B, k, mu_f, vk, proj, hdr, st);
    case 3: return project_kq<In, 3>(cube, N, B, k, mu_f, vk, proj, hdr, st);
    case 4: return project_kq<In, 4>(cube, N, B, k, mu_f, vk, proj, hdr, st);
    case 5: return project_kq<In, 5>(cube, N, B, k, mu_f, vk, proj, hdr, st);
    case 6: return project_kq<In, 6>(cube, N, B, k, mu_f, vk, proj, hdr, st);
    case 7: return project_kq<In, 7>(cube, N, B, k, mu_f, vk, proj, hdr, st);
    case 8: return project_kq<In, 8>(cube, N, B, k, mu_f, vk, proj, hdr, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_project(const void* cube, pca_dtype dt, int64_t N, int B, int k,
                           const float* mu_f, const float* vk, float* proj, cudaStream_t st,
                           DevHeader* hdr) {
  if (N < 1) return cudaSuccess;
  switch (dt) {
    case PCA_F32:
      return project_typed((const float*)cube, N, B, k, mu_f, vk, proj, hdr, st);
    case PCA_BF16:
      return project_typed((const __nv_bfloat16*)cube, N, B, k, mu_f, vk, proj, hdr, st);
    case PCA_F16:
      return project_typed((const __half*)cube, N, B, k, mu_f, vk, proj, hdr, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbpca
