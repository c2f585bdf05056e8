// k_syrk_tc.cu -- covariance partials on the 5th-generation tensor cores
// (tcgen05 + TMEM), the dense contraction of Algorithm 1 stage 3 (Sec. 4.2
// stage 3 forms it with one cuBLAS SGEMM; here it is hand-written).
//
// One persistent CTA per SM walks a contiguous range of 32-pixel chunks:
//   warp 0      TMA producer: cp.async.bulk of each chunk (pixel-major, a
//               contiguous byte range of the cube) into a ring of as many
//               stages (up to 12) as shared memory holds;
//   warps 2-17  converters: x = (y - s) 2^e per band (s = the mean of 32
//               pixels spread through the cube and e a power-of-two scale,
//               both computed by every CTA from the same pixels), split into
//               FP16 hi = fp16(x), lo = fp16(x - hi) -- 22 significant bits
//               of x -- written transposed ([band][pixel], K-major core-
//               matrix layout) into a 2-stage operand ring, and keep the
//               band sums S1 = sum x of the values they converted (FP32 over
//               16 chunks, then FP64);
//   warp 1      MMA issuer (one thread): D += hi hi^T + hi lo^T + lo hi^T
//               for the upper block-triangle (row tile 0: bands 0-127 x all;
//               row tile 1: bands 128-255 x bands 128-255) with FP32
//               accumulation in TMEM;
//   warps 2-5   epilogue: TMEM -> registers -> the CTA's partial slot
//               (packed upper triangle, FP32, still scaled by 2^(e_i+e_j));
//               the converters write S1 (FP64, unscaled).
// A scaled value outside the FP16 range sets hdr->cov_range; the caller then
// recomputes the partials on the SIMT path.  The partials are reduced and
// finalised by k_cov.cu.  Every mbarrier wait is bounded (one second of
// globaltimer); on time-out the CTA records PCA_ERR_TIMEOUT, drains its MMAs,
// frees TMEM and returns.
#include "tma.cuh"

namespace gbpca {

namespace {

constexpr int kKC = 32;                 // pixels per chunk (K of one stage)
constexpr int kMaxStages = 12;          // TMA ring depth: as many stages as shared memory holds
constexpr int kOpStages = 2;            // FP16 operand ring depth
constexpr int kRows = 256;              // operand rows (bands, padded to 16)
constexpr int kConvWarps = 16;
constexpr int kThreads = (2 + kConvWarps) * 32;
constexpr int kOpBytes = kRows * kKC * 2;        // one FP16 operand (hi or lo): 16 KB
constexpr uint32_t kLBO = 128;                   // K-adjacent core matrices
constexpr uint32_t kSBO = (kKC / 8) * 128;       // 8-row groups: 512 B
constexpr int kTmemCols = 512;
constexpr int kProbe = 32;               // pixels of the band probe
constexpr int kS1Flush = 16;             // chunks summed in FP32 before the FP64 add

struct __align__(8) SyncBlock {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t opfull[kOpStages];
  uint64_t opempty[kOpStages];
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// K-major, no swizzle: core matrix = 8 rows x 16 bytes; LBO = K stride, SBO = row-group stride.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((kLBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((kSBO >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// kind::f16 instruction descriptor: D F32, A/B F16 (format 0), both K-major,
// M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_f16(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   su32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_f16x2(float a, float b) {
  uint32_t r;  // low half = a, high half = b
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}
__device__ __forceinline__ void unpack_f16x2(uint32_t v, float& a, float& b) {
  a = __half2float(__ushort_as_half((unsigned short)(v & 0xffffu)));
  b = __half2float(__ushort_as_half((unsigned short)(v >> 16)));
}

template <typename In>
__device__ __forceinline__ float elem(const In* p) { return to_f32<In>(*p); }

// barrier among the converter warps only (the producer and MMA warps are busy)
__device__ __forceinline__ void conv_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kConvWarps * 32) : "memory");
}

template <typename In>
__global__ void __launch_bounds__(kThreads, 1)
k_syrk_tc(const In* __restrict__ cube, int64_t N, int B, float* __restrict__ shift_out,
          int* __restrict__ escale_out, double* __restrict__ s1_part,
          float* __restrict__ s2_part, int s2_elems, DevHeader* __restrict__ hdr, int S) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int R16 = (B + 15) & ~15;     // bands padded to the 16-row MMA granule
  const int stage_bytes_max = kKC * B * (int)sizeof(In);
  const int stage_stride = (stage_bytes_max + 127) & ~127;
  unsigned char* ops = smem;                                        // [kOpStages][hi|lo][kOpBytes]
  unsigned char* stages = smem + kOpStages * 2 * kOpBytes;          // [S][stage_stride]
  float* shs = reinterpret_cast<float*>(stages + S * stage_stride);        // [kRows] shift
  int* sesc = reinterpret_cast<int*>(shs + kRows);                         // [kRows] exponent
  double* psum = reinterpret_cast<double*>(sesc + kRows);                  // [4][kRows]
  float* pmin = reinterpret_cast<float*>(psum + 4 * kRows);                // [2][kRows]
  float* pmax = pmin + 2 * kRows;                                          // [2][kRows]
  SyncBlock* sb = reinterpret_cast<SyncBlock*>(pmax + 2 * kRows);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x, g = blockIdx.x;
  const int64_t nchunk_total = (N + kKC - 1) / kKC;
  const int64_t c_begin = nchunk_total * g / G, c_end = nchunk_total * (g + 1) / G;
  const int nch = (int)(c_end - c_begin);

  const bool two_tiles = B > 128;
  const int N0 = R16;                            // tile 0 columns: bands 0..R16-1
  const int N1 = two_tiles ? (R16 - 128) : 0;     // tile 1 columns: bands 128..R16-1

  // ---- set-up
  for (int i = tid; i < kOpStages * 2 * kOpBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(ops)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&sb->full[s], 1); mbar_init(&sb->empty[s], kConvWarps); }
    for (int s = 0; s < kOpStages; ++s) { mbar_init(&sb->opfull[s], kConvWarps); mbar_init(&sb->opempty[s], 1); }
    mbar_init(&sb->done, 1);
    sb->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&sb->tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = sb->tmem_base;
  int out_of_range = 0;   // a scaled value this thread converted left the FP16 range

  if (warp == 0) {
    // ---------------------------------------------------------- TMA producer
    if (lane == 0) {
      for (int c = 0; c < nch; ++c) {
        const int s = c % S;
        if (!mbar_wait(&sb->empty[s], ((c / S) & 1) ^ 1, &sb->abort)) break;
        const int64_t p0 = (c_begin + c) * kKC;
        const int cp = (int)((N - p0) < kKC ? (N - p0) : kKC);
        const uint32_t bytes = (uint32_t)(cp * B * (int)sizeof(In)) & ~15u;
        mbar_expect_tx(&sb->full[s], bytes);
        if (bytes) bulk_g2s(stages + s * stage_stride, cube + p0 * B, bytes, &sb->full[s]);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t ops_base = su32(ops);
      const uint32_t id0 = idesc_f16(N0), id1 = idesc_f16(N1 > 0 ? N1 : 16);
      bool issued = false;
      for (int c = 0; c < nch; ++c) {
        const int o = c % kOpStages;
        if (!mbar_wait(&sb->opfull[o], (c / kOpStages) & 1, &sb->abort)) break;
        tc_fence_after();
        const uint32_t hi = ops_base + (uint32_t)(o * 2) * kOpBytes;
        const uint32_t lo = hi + kOpBytes;
#pragma unroll
        for (int kk = 0; kk < kKC / 16; ++kk) {
          const uint32_t ko = kk * 2 * kLBO;
          const uint32_t acc0 = (c > 0 || kk > 0) ? 1u : 0u;
          // tile 0: rows 0..127 (A) x rows 0..N0-1 (B)
          mma_f16(tbase, sdesc(hi + ko), sdesc(hi + ko), id0, acc0);
          mma_f16(tbase, sdesc(hi + ko), sdesc(lo + ko), id0, 1u);
          mma_f16(tbase, sdesc(lo + ko), sdesc(hi + ko), id0, 1u);
          if (two_tiles) {
            const uint32_t r128 = (128 / 8) * kSBO;
            const uint32_t t1 = tbase + (uint32_t)N0;
            mma_f16(t1, sdesc(hi + r128 + ko), sdesc(hi + r128 + ko), id1, acc0);
            mma_f16(t1, sdesc(hi + r128 + ko), sdesc(lo + r128 + ko), id1, 1u);
            mma_f16(t1, sdesc(lo + r128 + ko), sdesc(hi + r128 + ko), id1, 1u);
          }
        }
        issued = true;
        mma_commit(&sb->opempty[o]);  // operand stage free once these MMAs finished
      }
      (void)issued;
      mma_commit(&sb->done);          // all MMAs of this CTA finished
    }
  } else {
    // ---------------------------------------------------------- converters
    // Item = (band, 8-pixel group); a thread owns the same items in every
    // chunk (at most two for B <= 256), so their decode happens once.
    const int ct = tid - 64;
    // Band probe (every CTA computes the same values from the same pixels):
    // over S = min(N, 32) pixels spread evenly through the cube, per band b
    //   shift_b = sample mean,  escale_b = 6 - E with max |y - shift_b| <= 2^E,
    // so that the sampled deviations scale into (2^5, 2^6] and a scaled value
    // leaves the FP16 range (65504) only if it lies about a thousand times
    // further from the shift than every sampled one.  A degenerate sample
    // falls back to |shift_b|, then to scale 1.
    {
      const int S = (int)(N < kProbe ? N : kProbe);
      const int b = ct % kRows, half = ct / kRows;     // 512 threads: two halves of the sample
      double sum = 0.0;
      float lo = INFINITY, hi = -INFINITY;
      if (b < B) {
        float y[kProbe / 2];
#pragma unroll
        for (int u = 0; u < kProbe / 2; ++u) {
          const int i = half + 2 * u;
          y[u] = i < S ? elem(cube + ((int64_t)i * N / S) * B + b) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kProbe / 2; ++u) {
          if (half + 2 * u < S) {
            sum += (double)y[u];
            lo = fminf(lo, y[u]);
            hi = fmaxf(hi, y[u]);
          }
        }
      }
      psum[half * kRows + b] = sum;
      pmin[half * kRows + b] = lo;
      pmax[half * kRows + b] = hi;
      conv_sync();
      if (ct < kRows) {
        float m = 0.f;
        int e = 0;
        if (b < B) {
          const double tot = psum[b] + psum[kRows + b];
          lo = fminf(pmin[b], pmin[kRows + b]);
          hi = fmaxf(pmax[b], pmax[kRows + b]);
          m = (float)(tot / (double)S);
          double dev = fmax((double)hi - (double)m, (double)m - (double)lo);
          if (!isfinite(m) || !isfinite(dev)) { m = 0.f; dev = 0.0; }
          if (!(dev > 0.0)) dev = fabs((double)m);
          if (dev > 0.0) {
            int E;
            frexp(dev, &E);
            e = 6 - E;
            e = e < -120 ? -120 : (e > 120 ? 120 : e);
          }
          if (g == 0) { shift_out[b] = m; escale_out[b] = e; }
        }
        shs[b] = m;
        sesc[b] = e;
      }
      conv_sync();
    }
    const int items = B * (kKC / 8);
    int ib[2], ipg[2], ioff[2];
    float ish[2], isc[2], s1f[2] = {0.f, 0.f};
    double s1d[2] = {0.0, 0.0};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int w = ct + u * kConvWarps * 32;
      ipg[u] = w < items ? w / B : -1;
      ib[u] = w < items ? w - ipg[u] * B : 0;
      const int row = ib[u];
      ioff[u] = (row >> 3) * (int)kSBO + (ipg[u] < 0 ? 0 : ipg[u]) * 128 + (row & 7) * 16;
      ish[u] = shs[row];
      isc[u] = ldexpf(1.f, sesc[row]);
    }
    for (int c = 0; c < nch; ++c) {
      const int s = c % S, o = c % kOpStages;
      // one lane per warp polls the barriers (the others would only add
      // shared-memory traffic), then the warp proceeds together
      int ok = 1;
      if (lane == 0) {
        ok = mbar_wait(&sb->full[s], (c / S) & 1, &sb->abort) ? 1 : 0;
        if (ok) ok = mbar_wait(&sb->opempty[o], ((c / kOpStages) & 1) ^ 1, &sb->abort) ? 1 : 0;
      }
      ok = __shfl_sync(kFull, ok, 0);
      if (!ok) break;
      const int64_t p0 = (c_begin + c) * kKC;
      const int cp = (int)((N - p0) < kKC ? (N - p0) : kKC);
      const int copied = (int)(((uint32_t)(cp * B * (int)sizeof(In)) & ~15u) / sizeof(In));
      const bool full = cp == kKC && copied == kKC * B;
      const In* st = reinterpret_cast<const In*>(stages + s * stage_stride);
      const In* gsrc = cube + p0 * B;
      unsigned char* hi = ops + (size_t)(o * 2) * kOpBytes;
      unsigned char* lo = hi + kOpBytes;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int pg = ipg[u], b = ib[u];
        if (pg < 0) continue;
        uint32_t h[4], l[4];
        {
          const float sh = ish[u], sc = isc[u];
          float x[8];
          if (full) {
            const In* src = st + pg * 8 * B + b;
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = (elem(src + i * B) - sh) * sc;
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int p = pg * 8 + i;
              const int e = p * B + b;
              float v = 0.f;
              if (p < cp) v = ((e < copied ? elem(st + e) : elem(gsrc + e)) - sh) * sc;
              x[i] = v;
            }
          }
          // NaN compares false, so it counts as out of range too
#pragma unroll
          for (int i = 0; i < 8; ++i) out_of_range |= !(fabsf(x[i]) <= 65504.f);
          s1f[u] += ((x[0] + x[1]) + (x[2] + x[3])) + ((x[4] + x[5]) + (x[6] + x[7]));
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            h[i] = pack_f16x2(x[2 * i], x[2 * i + 1]);
            float a, bb;
            unpack_f16x2(h[i], a, bb);
            l[i] = pack_f16x2(x[2 * i] - a, x[2 * i + 1] - bb);
          }
        }
        *reinterpret_cast<uint4*>(hi + ioff[u]) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(lo + ioff[u]) = make_uint4(l[0], l[1], l[2], l[3]);
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) { mbar_arrive(&sb->opfull[o]); mbar_arrive(&sb->empty[s]); }
      if ((c + 1) % kS1Flush == 0) {
#pragma unroll
        for (int u = 0; u < 2; ++u) { s1d[u] += (double)s1f[u]; s1f[u] = 0.f; }
      }
    }
    // band sums: the four 8-pixel groups of a band meet in shared memory (the
    // probe's sums are no longer read once the loop has started)
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (ipg[u] >= 0) psum[ipg[u] * kRows + ib[u]] = s1d[u] + (double)s1f[u];
    conv_sync();
    for (int b = ct; b < B; b += kConvWarps * 32)
      s1_part[(size_t)g * B + b] =
          ldexp((psum[b] + psum[kRows + b]) + (psum[2 * kRows + b] + psum[3 * kRows + b]), -sesc[b]);
    // ---------------------------------------------------------- epilogue
    if (warp >= 2 && warp < 6) {
      int okw = 0;
      if (lane == 0) okw = (mbar_wait(&sb->done, 0, &sb->abort) && !*(volatile int*)&sb->abort) ? 1 : 0;
      const bool ok = __shfl_sync(kFull, okw, 0) != 0;
      tc_fence_after();
      const int q = warp & 3;          // TMEM lane quarter this warp may read
      const int r = q * 32 + lane;     // accumulator row
      const uint32_t lane_off = (uint32_t)(q * 32) << 16;
      float* out = s2_part + (size_t)g * s2_elems;
      // tile 0: row r = band r, column j = band j (j < R16)
      for (int j0 = 0; j0 < N0; j0 += 16) {
        float v[16];
        if (ok) tmem_ld16(tbase + lane_off + (uint32_t)j0, v);
        else
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int j = j0 + i;
          if (r < B && r < 128 && j < B && j >= r) out[packed_index(r, j, B)] = v[i];
        }
      }
      if (two_tiles) {
        const int band = 128 + r;
        for (int j0 = 0; j0 < N1; j0 += 16) {
          float v[16];
          if (ok) tmem_ld16(tbase + lane_off + (uint32_t)(N0 + j0), v);
          else
            for (int i = 0; i < 16; ++i) v[i] = 0.f;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int jb = 128 + j0 + i;
            if (band < B && jb < B && jb >= band) out[packed_index(band, jb, B)] = v[i];
          }
        }
      }
      if (!ok && lane == 0) set_status(hdr, PCA_ERR_TIMEOUT);
    }
  }
  tc_fence_before();
  if (__syncthreads_or(out_of_range) && tid == 0) atomicOr(&hdr->cov_range, 1);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "r"(kTmemCols)
                 : "memory");
  }
}

template <typename In>
cudaError_t syrk_tc_typed(const In* cube, int64_t N, int B, float* shift, int* escale,
                          double* s1_part, float* s2_part, int partials, DevHeader* hdr,
                          cudaStream_t st) {
  const int stage_stride = ((kKC * B * (int)sizeof(In)) + 127) & ~127;
  const size_t fixed = 1024 + (size_t)kOpStages * 2 * kOpBytes +
                       kRows * (sizeof(float) + sizeof(int)) +
                       kRows * (4 * sizeof(double) + 4 * sizeof(float)) + sizeof(SyncBlock);
  int S = (int)((227 * 1024 - fixed) / stage_stride);
  S = S > kMaxStages ? kMaxStages : S;
  if (S < 2) return cudaErrorInvalidValue;
  const size_t smem = fixed + (size_t)S * stage_stride;
  auto kern = k_syrk_tc<In>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<partials, kThreads, smem, st>>>(cube, N, B, shift, escale, s1_part, s2_part,
                                         B * (B + 1) / 2, hdr, S);
  return cudaGetLastError();
}

}  // namespace

bool syrk_tc_supported(int B) { return B >= 2 && B <= kMaxB; }

cudaError_t launch_syrk_tc(const void* cube, pca_dtype dt, int64_t N, int B, float* shift,
                           int* escale, double* s1_part, float* s2_part, int partials,
                           DevHeader* hdr, cudaStream_t st) {
  switch (dt) {
    case PCA_F32:
      return syrk_tc_typed((const float*)cube, N, B, shift, escale, s1_part, s2_part, partials, hdr,
                           st);
    case PCA_BF16:
      return syrk_tc_typed((const __nv_bfloat16*)cube, N, B, shift, escale, s1_part, s2_part,
                           partials, hdr, st);
    case PCA_F16:
      return syrk_tc_typed((const __half*)cube, N, B, shift, escale, s1_part, s2_part, partials,
                           hdr, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbpca
