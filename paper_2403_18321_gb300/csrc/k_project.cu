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
// shared memory before the chunk's columns are stored.  One pass handles up to
// 32 columns; more components take one pass per group of 32 (the batched form:
// one work item per tile, chunk range and column group).  Every wait is
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
constexpr int kColGroup = 32;            // columns of V_k per pass (registers per thread)

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

// One pass projects columns [j0, j0 + k) of V_k (k <= 32): vk and proj point at
// column j0 of their matrices, whose rows are vk_ld and q_ld floats apart.
struct ProjArgs {
  const void* cube;
  int64_t N;
  int B, k;
  const float* mu_f;
  const float* vk;
  float* proj;
  DevHeader* hdr;
  int vk_ld, q_ld;
  const int* guard;    // single cube: run only when *guard != 0 (nullable)
};

// One work item: chunks [c0, c1) of one cube and its tensor map.
struct PItem {
  ProjArgs a;
  const CUtensorMap* map;
  int64_t c0, c1;
};

__device__ __forceinline__ PItem proj_item(const ProjArgs& one, const CUtensorMap* one_map,
                                           const TileDesc* __restrict__ T,
                                           const CUtensorMap* __restrict__ maps,
                                           const ProjItem* __restrict__ items,
                                           const int* __restrict__ cta_items, int i) {
  PItem it;
  if (T == nullptr) {  // single cube: CTA g takes its share of the chunks
    const int G = gridDim.x, g = blockIdx.x;
    const int64_t nch = (one.N + kPc - 1) / kPc;
    it.a = one;
    it.map = one_map;
    it.c0 = nch * g / G;
    it.c1 = nch * (g + 1) / G;
  } else {
    const ProjItem pi = items[cta_items[blockIdx.x] + i];
    const TileDesc& d = T[pi.tile];
    const int j0 = kColGroup * pi.pad;     // this item's column group
    it.a.cube = d.cube;
    it.a.N = d.N;
    it.a.B = d.B;
    it.a.k = d.k - j0 < kColGroup ? d.k - j0 : kColGroup;
    it.a.mu_f = d.muf;
    it.a.vk = d.vk + j0;
    it.a.proj = d.proj + j0;
    it.a.hdr = d.hdr;
    it.a.vk_ld = d.k;
    it.a.q_ld = d.k;
    it.map = maps != nullptr ? maps + pi.tile : nullptr;
    it.c0 = pi.c0;
    it.c1 = pi.c1;
  }
  return it;
}

// maxB, maxk: the largest bands and components of the items (shared-memory
// sizing); the single-cube form takes its cube as `one` with map `tmap`.
template <typename In, int KQ, bool kTiled>
__global__ void __launch_bounds__(kThreadsP, 1)
k_project(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ ProjArgs one,
          const TileDesc* __restrict__ T, const CUtensorMap* __restrict__ maps,
          const ProjItem* __restrict__ items, const int* __restrict__ cta_items, int maxB,
          int maxk, int S, int stage_bytes) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned start (the 128-byte swizzle repeats every 1024 bytes);
  // offsetting the array itself keeps every access a shared-memory one
  unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  constexpr int E = 16 / (int)sizeof(In);           // elements per 16-byte unit
  const int B8m = (maxB + 7) & ~7;
  unsigned char* stages = smem;
  float4* vs = reinterpret_cast<float4*>(stages + (size_t)S * stage_bytes);  // [B8][KQ]
  float* mus = reinterpret_cast<float*>(vs + (size_t)B8m * KQ);              // [B8]
  float* red = mus + B8m;                                                    // [kParts][kPc][k]
  ProjSync* sy = reinterpret_cast<ProjSync*>(red + (size_t)kParts * kPc * maxk);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nitems = T == nullptr ? 1 : cta_items[blockIdx.x + 1] - cta_items[blockIdx.x];
  if (T == nullptr && one.guard != nullptr && *(volatile const int*)one.guard == 0) return;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&sy->full[s], 1); mbar_init(&sy->empty[s], kParts); }
    sy->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == kParts) {
    // ------------------------------------------------------------ producer
    // streams every item's chunks through one ring, ahead of the compute warps
    if (lane == 0) {
      Ring rq(S);
      bool ok = true;
      for (int i = 0; i < nitems && ok; ++i) {
        const PItem it = proj_item(one, &tmap, T, maps, items, cta_items, i);
        const In* cube = static_cast<const In*>(it.a.cube);
        const int64_t N = it.a.N;
        const int B = it.a.B;
        const int nbox = (B * (int)sizeof(In) + 127) / 128;
        for (int64_t c = it.c0; c < it.c1; ++c, rq.next()) {
          const int s = rq.idx;
          if (!mbar_wait(&sy->empty[s], rq.phase ^ 1u, &sy->abort)) { ok = false; break; }
          const int64_t p0 = c * kPc;
          unsigned char* dst = stages + (size_t)s * stage_bytes;
          if constexpr (kTiled) {
            mbar_expect_tx(&sy->full[s], (uint32_t)(nbox * kPc * 128));
            for (int bx = 0; bx < nbox; ++bx)
              tma_load_2d(dst + (size_t)bx * kPc * 128, it.map, bx * (128 / (int)sizeof(In)),
                          (int)p0, &sy->full[s]);
          } else {
            const int cp = (int)((N - p0) < kPc ? (N - p0) : kPc);
            const uint32_t bytes = (uint32_t)((size_t)cp * B * sizeof(In)) & ~15u;
            mbar_expect_tx(&sy->full[s], bytes);
            if (bytes) bulk_g2s(dst, cube + p0 * B, bytes, &sy->full[s]);
          }
        }
      }
    }
    return;
  }

  // -------------------------------------------------------------- compute
  const int h = warp;
  const int pa = lane, pb = lane + 32;
  Ring rq(S);
  bool stop = false;
  for (int i = 0; i < nitems && !stop; ++i) {
  const PItem it = proj_item(one, &tmap, T, maps, items, cta_items, i);
  const ProjArgs& a = it.a;
  const In* cube = static_cast<const In*>(a.cube);
  const int64_t N = a.N;
  const int B = a.B, k = a.k;
  const int B8 = (B + 7) & ~7;
  // V_k and mu of this item's cube (the producer is already streaming)
  if (i > 0) named_sync();   // every warp is done with the previous item's V_k
  for (int e = tid; e < B8 * KQ * 4; e += kCompute) {
    const int b = e / (KQ * 4), j = e - b * (KQ * 4);
    reinterpret_cast<float*>(vs)[e] = (b < B && j < k) ? a.vk[(size_t)b * a.vk_ld + j] : 0.f;
  }
  for (int b = tid; b < B8; b += kCompute) mus[b] = b < B ? a.mu_f[b] : 0.f;
  named_sync();
  int64_t c = it.c0;
  for (; c < it.c1; ++c, rq.next()) {
    const int s = rq.idx;
    int ok = 1;
    if (lane == 0) ok = mbar_wait(&sy->full[s], rq.phase, &sy->abort) ? 1 : 0;
    ok = __shfl_sync(kFull, ok, 0);
    if (!named_and(ok)) break;
    const int64_t p0 = c * kPc;
    const int cp = (int)((N - p0) < kPc ? (N - p0) : kPc);
    const unsigned char* st = stages + (size_t)s * stage_bytes;
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
      // bands 4u .. 4u+3 for u = h, h + 8, ...: read four groups at a time.
      // The stage is released only after the last values read from it have
      // been used: an arrive right after the loads let the next copy into the
      // stage overwrite values still being read (wrong projections seen on
      // the GPU when B was a multiple of 32).
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
        if (i0 + 4 >= mine) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&sy->empty[s]);
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
    float* out = a.proj + p0 * a.q_ld;
    for (int o = tid; o < cp * k; o += kCompute) {
      float sum = 0.f;
#pragma unroll
      for (int hh = 0; hh < kParts; ++hh) sum += red[(size_t)hh * kPc * k + o];
      const int row = o / k;
      out[(size_t)row * a.q_ld + (o - row * k)] = sum;
    }
    named_sync();
  }
  if (c < it.c1) {
    // a bounded wait gave up: make the rest of this CTA's work visibly invalid
    stop = true;
    for (int j = i; j < nitems; ++j) {
      const PItem rest = proj_item(one, &tmap, T, maps, items, cta_items, j);
      const int64_t c0 = j == i ? c : rest.c0;
      const int64_t kk = rest.a.k;
      const int64_t o0 = c0 * kPc * kk;
      const int64_t o1 = (rest.c1 * kPc < rest.a.N ? rest.c1 * kPc : rest.a.N) * kk;
      for (int64_t o = o0 + tid; o < o1; o += kCompute)
        rest.a.proj[(o / kk) * rest.a.q_ld + o % kk] = __int_as_float(0x7fc00000);
      if (tid == 0 && rest.a.hdr) set_status(rest.a.hdr, PCA_ERR_TIMEOUT);
    }
  }
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

// 2-D map of a cube [N][B] for the swizzled tiled load: boxes of 128 bytes x
// kPc pixels.  False when the rows are not whole 16-byte units or encoding fails.
template <typename In>
bool encode_map(const void* cube, int64_t N, int B, CUtensorMap* map, int box_rows = kPc) {
  memset(map, 0, sizeof(*map));
  if ((B * sizeof(In)) % 16 != 0 || ((uintptr_t)cube % 16) != 0 || N >= (1ll << 31) ||
      encode_fn() == nullptr)
    return false;
  const cuuint64_t gdim[2] = {(cuuint64_t)B, (cuuint64_t)N};
  const cuuint64_t gstride[1] = {(cuuint64_t)B * sizeof(In)};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / sizeof(In)), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return encode_fn()(map, tmap_type<In>(), 2, const_cast<void*>(cube), gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename In, int KQ>
cudaError_t project_launch(bool tiled, const CUtensorMap& tmap, const ProjArgs& one,
                           const TileDesc* T, const CUtensorMap* maps, const ProjItem* items,
                           const int* cta_items, int ctas, int maxB, int maxk, cudaStream_t st) {
  const int B8 = (maxB + 7) & ~7;
  const int nbox = (maxB * (int)sizeof(In) + 127) / 128;
  const int stage_bytes = tiled ? nbox * kPc * 128
                                : (int)((((size_t)kPc * maxB * sizeof(In)) + 1023) & ~(size_t)1023);
  const size_t fixed = (size_t)B8 * KQ * 16 + (size_t)B8 * 4 + (size_t)kParts * kPc * maxk * 4 +
                       sizeof(ProjSync) + 1024;
  const size_t budget = 227 * 1024;
  int stages = (int)((budget - fixed) / stage_bytes);
  stages = stages > kMaxStages ? kMaxStages : stages;
  if (stages < 2) return cudaErrorInvalidValue;
  const size_t smem = fixed + (size_t)stages * stage_bytes;
  auto kern = tiled ? k_project<In, KQ, true> : k_project<In, KQ, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<ctas, kThreadsP, smem, st>>>(tmap, one, T, maps, items, cta_items, maxB, maxk, stages,
                                      stage_bytes);
  return cudaGetLastError();
}

template <typename In>
cudaError_t project_any(bool tiled, const CUtensorMap& tmap, const ProjArgs& one, const TileDesc* T,
                        const CUtensorMap* maps, const ProjItem* items, const int* cta_items,
                        int ctas, int maxB, int maxk, cudaStream_t st) {
  switch ((maxk + 3) / 4) {
#define GB_PROJ_CASE(q) \
    case q: return project_launch<In, q>(tiled, tmap, one, T, maps, items, cta_items, ctas, maxB, maxk, st);
    GB_PROJ_CASE(1) GB_PROJ_CASE(2) GB_PROJ_CASE(3) GB_PROJ_CASE(4)
    GB_PROJ_CASE(5) GB_PROJ_CASE(6) GB_PROJ_CASE(7) GB_PROJ_CASE(8)
#undef GB_PROJ_CASE
  }
  return cudaErrorInvalidValue;
}

template <typename In>
cudaError_t project_typed(const In* cube, int64_t N, int B, int k, const float* mu_f,
                          const float* vk, float* proj, DevHeader* hdr, const int* guard,
                          cudaStream_t st) {
  CUtensorMap tmap;
  const bool tiled = encode_map<In>(cube, N, B, &tmap);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nch = (N + kPc - 1) / kPc;
  const int grid = (int)(nch < sms ? nch : sms);
  // one pass per group of at most kColGroup columns
  for (int j0 = 0; j0 < k; j0 += kColGroup) {
    const int kk = k - j0 < kColGroup ? k - j0 : kColGroup;
    const ProjArgs one{cube, N, B, kk, mu_f, vk + j0, proj + j0, hdr, k, k, guard};
    const cudaError_t e =
        project_any<In>(tiled, tmap, one, nullptr, nullptr, nullptr, nullptr, grid, B, kk, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

bool encode_cube_map(pca_dtype dt, const void* cube, int64_t N, int B, void* map, int box_rows) {
  CUtensorMap* m = static_cast<CUtensorMap*>(map);
  switch (dt) {
    case PCA_F32: return encode_map<float>(cube, N, B, m, box_rows);
    case PCA_BF16: return encode_map<__nv_bfloat16>(cube, N, B, m, box_rows);
    case PCA_F16: return encode_map<__half>(cube, N, B, m, box_rows);
  }
  return false;
}

cudaError_t launch_project_grouped(const TileDesc* T, const void* maps, const ProjItem* items,
                                   const int* cta_items, int ctas, int maxB, int maxk,
                                   pca_dtype dt, cudaStream_t st) {
  if (ctas <= 0) return cudaSuccess;
  CUtensorMap none;
  memset(&none, 0, sizeof(none));
  const ProjArgs one{};
  const CUtensorMap* m = static_cast<const CUtensorMap*>(maps);
  if (maxk > kColGroup) maxk = kColGroup;   // items carry one column group each
  switch (dt) {
    case PCA_F32:
      return project_any<float>(m != nullptr, none, one, T, m, items, cta_items, ctas, maxB, maxk, st);
    case PCA_BF16:
      return project_any<__nv_bfloat16>(m != nullptr, none, one, T, m, items, cta_items, ctas, maxB,
                                        maxk, st);
    case PCA_F16:
      return project_any<__half>(m != nullptr, none, one, T, m, items, cta_items, ctas, maxB, maxk,
                                 st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_project(const void* cube, pca_dtype dt, int64_t N, int B, int k,
                           const float* mu_f, const float* vk, float* proj, cudaStream_t st,
                           DevHeader* hdr, const int* guard) {
  if (N < 1) return cudaSuccess;
  switch (dt) {
    case PCA_F32:
      return project_typed((const float*)cube, N, B, k, mu_f, vk, proj, hdr, guard, st);
    case PCA_BF16:
      return project_typed((const __nv_bfloat16*)cube, N, B, k, mu_f, vk, proj, hdr, guard, st);
    case PCA_F16:
      return project_typed((const __half*)cube, N, B, k, mu_f, vk, proj, hdr, guard, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbpca
