// k_bwd_dy_tc.cu -- the dominant product of the adjoint on the tensor cores:
//   dY[n][c] = sum_b x_nb S'_bc + sum_j dq'_nj V_cj,   x = y - mu, dq' = dq - mean dq,
// i.e. [X | dQ'] [S'; V_k^T] (S' = 2/(N-1) sym(V G V^T), see k_backward.cu).
// Both operands go through the two-term FP16 split of the
// covariance kernel (22 significant bits each; products hi hi + hi lo + lo hi,
// FP32 accumulation in TMEM), with power-of-two scales that keep every value
// inside the FP16 range.  The two terms are two segments of K -- the bands
// [0, B) and, from the next multiple of 32, the k columns of dQ -- each with
// its own TMEM accumulator, so that neither is scaled for the other's range:
//   A (pixels x K): column kk scaled by 2^a_kk from the exact maximum of
//     |x_b| (or |dq'_j|) over the cube, measured by k_bwd_dv;
//   B (K x bands):  row kk by 2^-a_kk (so the products are unscaled) and,
//     per segment, column c by 2^f_c from its largest entry; the epilogue
//     adds the two accumulators times 2^-f_c.  k_bwd_bop writes B once, hi
//     and lo planes already in the shared-memory core-matrix layout of each
//     32-wide K block.
// One persistent CTA per SM walks 128-pixel tiles:
//   warp 0       bulk copies of the K blocks of B and, for FP32 cubes whose
//                rows are whole 16-byte units, 2-D tensor-map loads (128-byte
//                swizzle) of the cube's 128 x 32 band blocks (3-stage rings);
//   warps 2-17   converters: each thread one (pixel row, 8-wide K group) of
//                the A block, read from the staged cube block (else straight
//                from the cube, one block ahead) and, for the dQ block, from
//                dQ; centred, scaled, split, written as K-major core matrices;
//   warp 1       MMA issuer (one thread): M = 128, N = B rounded to 16, two
//                K = 16 steps x three products per block, into the band or
//                the dQ accumulator (TMEM columns 0 and 256);
//   warps 2-9    epilogue: TMEM -> registers -> column scales -> dY rows
//                (two warps per TMEM lane quarter, half the columns each).
// Every wait is bounded (one second); on time-out the CTA records
// PCA_ERR_TIMEOUT, drains its MMAs and frees TMEM.
#include "tc.cuh"

namespace gbpca {

namespace {

constexpr int kM = 128;          // pixels per tile (MMA M)
constexpr int kKB = 32;          // K per block
constexpr int kSt = 3;           // ring depth (A and B in lock-step)
constexpr int kConv = 16;        // converter warps
constexpr int kThr = (2 + kConv) * 32;
constexpr uint32_t kLBO = 128;                 // K-adjacent core matrices
constexpr uint32_t kSBO = (kKB / 8) * 128;     // 8-row groups: 512 B
constexpr int kAPlane = kM * kKB * 2;          // one FP16 plane of an A block: 8 KB
constexpr int kXStage = kM * 128;              // a staged FP32 cube block: 128 rows x 128 B
constexpr int kMaxKdim = 256 + 256;   // bands (rounded to 32) + dQ columns
constexpr int kEpiWarps = 8;     // epilogue warps: two per TMEM lane quarter, each half the columns

struct __align__(8) DySync {
  uint64_t xfull[kSt];
  uint64_t afull[kSt];
  uint64_t bfull[kSt];
  uint64_t sfree[kSt];
  uint64_t done;
  uint64_t tfree;
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};

// The raw values of the 8-wide K group kk0.. of pixel n (0 past the cube, in
// the gap between the band and dQ segments and past K): two 16-byte loads of
// the cube row when the group lies inside the bands and the row offset is a
// whole number of 16-byte units, else element loads.
template <typename In>
__device__ __forceinline__ void load_group(const In* __restrict__ cube, const float* __restrict__ dq,
                                           int64_t n, int64_t N, int B, int B32, int k, int kk0,
                                           float* raw) {
#pragma unroll
  for (int e = 0; e < 8; ++e) raw[e] = 0.f;
  if (n >= N) return;
  if (kk0 + 8 <= B) {
    const In* src = cube + n * B + kk0;
    if constexpr (sizeof(In) == 4) {
      if ((B & 3) == 0) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(src));
        const float4 b = __ldg(reinterpret_cast<const float4*>(src) + 1);
        raw[0] = a.x; raw[1] = a.y; raw[2] = a.z; raw[3] = a.w;
        raw[4] = b.x; raw[5] = b.y; raw[6] = b.z; raw[7] = b.w;
        return;
      }
    } else {
      if ((B & 7) == 0) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(src));
        const In* h = reinterpret_cast<const In*>(&u);
#pragma unroll
        for (int e = 0; e < 8; ++e) raw[e] = to_f32<In>(h[e]);
        return;
      }
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) raw[e] = to_f32<In>(src[e]);
    return;
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int kk = kk0 + e;
    if (kk < B) raw[e] = to_f32<In>(cube[n * B + kk]);
    else if (kk >= B32 && kk - B32 < k) raw[e] = dq[n * k + (kk - B32)];
  }
}

__device__ __forceinline__ void conv_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(kConv * 32) : "memory");
}

template <typename In>
__global__ void __launch_bounds__(kThr, 1)
k_bwd_dy_tc(const __grid_constant__ CUtensorMap xmap, int xtma, const In* __restrict__ cube,
            const float* __restrict__ dq, int64_t N, int B, int k,
            const float* __restrict__ ascale, const float* __restrict__ anshift,
            const unsigned char* __restrict__ bop, const float* __restrict__ fcol,
            float* __restrict__ dY, DevHeader* __restrict__ hdr) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned start (the 128-byte swizzle repeats every 1024 bytes)
  unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  const int R16 = (B + 15) & ~15;
  const int B32 = (B + kKB - 1) & ~(kKB - 1);           // the dQ segment starts here
  const int K = B32 + k, KB = (K + kKB - 1) / kKB, KB1 = B32 / kKB;
  const int bplane = R16 * kKB * 2;                     // one FP16 plane of a B block
  unsigned char* xs = smem;                              // [kSt][kXStage] staged cube blocks
  unsigned char* as = xs + kSt * kXStage;                // [kSt][hi|lo][kAPlane]
  unsigned char* bs = as + kSt * 2 * kAPlane;            // [kSt][hi|lo][bplane]
  float* sc = reinterpret_cast<float*>(bs + (size_t)kSt * 2 * bplane);   // [kMaxKdim]
  float* sh = sc + kMaxKdim;                                                // [kMaxKdim]
  float* fc = sh + kMaxKdim;                                                // [2][256]
  DySync* sy = reinterpret_cast<DySync*>(fc + 512);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (N + kM - 1) / kM;

  for (int i = tid; i < kMaxKdim; i += kThr) {
    sc[i] = i < K ? ascale[i] : 0.f;
    sh[i] = i < K ? anshift[i] : 0.f;
  }
  for (int i = tid; i < 512; i += kThr) fc[i] = (i & 255) < B ? fcol[(i >> 8) * B + (i & 255)] : 0.f;
  if (tid == 0) {
    for (int s = 0; s < kSt; ++s) {
      mbar_init(&sy->xfull[s], 1);
      mbar_init(&sy->afull[s], kConv);
      mbar_init(&sy->bfull[s], 1);
      mbar_init(&sy->sfree[s], 1);
    }
    mbar_init(&sy->done, 1);
    mbar_init(&sy->tfree, kEpiWarps);
    mbar_init(&sy->drain, 1);
    sy->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&sy->tmem_base)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = sy->tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ B blocks
    if (lane == 0) {
      int q = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        for (int kb = 0; kb < KB; ++kb, ++q) {
          const int s = q % kSt;
          if (!mbar_wait(&sy->sfree[s], ((q / kSt) & 1) ^ 1, &sy->abort)) { ok = false; break; }
          if (xtma) {
            if (kb < KB1) {         // the stage's cube block: 32 bands x 128 pixels
              mbar_expect_tx(&sy->xfull[s], (uint32_t)kXStage);
              tma_load_2d(xs + (size_t)s * kXStage, &xmap, kb * kKB, (int)(t * kM), &sy->xfull[s]);
            } else {                // the dQ block stages nothing; the phase still
              mbar_arrive(&sy->xfull[s]);   // advances, in step with the ring position
            }
          }
          mbar_expect_tx(&sy->bfull[s], (uint32_t)(2 * bplane));
          bulk_g2s(bs + (size_t)s * 2 * bplane, bop + (size_t)kb * 2 * bplane, (uint32_t)(2 * bplane),
                   &sy->bfull[s]);
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | ((uint32_t)(R16 >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
      int q = 0, tl = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
        // the accumulators are free once the previous tile's epilogue has read them
        if (tl >= 1 && !mbar_wait(&sy->tfree, (tl - 1) & 1, &sy->abort)) break;
        tc_fence_after();
        for (int kb = 0; kb < KB; ++kb, ++q) {
          const bool seg2 = kb >= KB1;                     // a dQ block
          const uint32_t dt = tbase + (seg2 ? 256u : 0u);
          const int s = q % kSt;
          if (!mbar_wait(&sy->afull[s], (q / kSt) & 1, &sy->abort) ||
              !mbar_wait(&sy->bfull[s], (q / kSt) & 1, &sy->abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ahi = su32(as + (size_t)s * 2 * kAPlane), alo = ahi + kAPlane;
          const uint32_t bhi = su32(bs + (size_t)s * 2 * bplane), blo = bhi + (uint32_t)bplane;
#pragma unroll
          for (int kk = 0; kk < kKB / 16; ++kk) {
            const uint32_t ko = kk * 2 * kLBO;
            const uint32_t acc0 = ((kb != 0 && kb != KB1) || kk > 0) ? 1u : 0u;
            mma_f16(dt, sdesc_kmajor(ahi + ko, kLBO, kSBO), sdesc_kmajor(bhi + ko, kLBO, kSBO), idesc, acc0);
            mma_f16(dt, sdesc_kmajor(ahi + ko, kLBO, kSBO), sdesc_kmajor(blo + ko, kLBO, kSBO), idesc, 1u);
            mma_f16(dt, sdesc_kmajor(alo + ko, kLBO, kSBO), sdesc_kmajor(bhi + ko, kLBO, kSBO), idesc, 1u);
          }
          mma_commit(&sy->sfree[s]);   // A and B stage s free once these MMAs finished
        }
        mma_commit(&sy->done);         // this tile's accumulation finished
      }
    }
  } else {
    // ------------------------------------------------------------ converters
    const int ct = tid - 64;
    // pixel row and 8-wide K group: the 8 lanes of a quarter warp take eight
    // rows of one K group, so that their 16-byte stores fill one core matrix
    // (all 32 banks) and their reads of a swizzled row hit 8 distinct units
    const int r = ((ct >> 5) << 3) | (ct & 7), kg = (ct >> 3) & 3;
    const uint32_t aoff = (uint32_t)((r >> 3) * (int)kSBO + kg * 128 + (r & 7) * 16);
    int q = 0, tl = 0;
    bool ok = true;
    // blocks read straight from memory are loaded one block ahead, while the
    // current one is converted; staged blocks are read from shared memory
    float cur[8];
    if (!xtma)
      load_group<In>(cube, dq, (int64_t)blockIdx.x * kM + r, N, B, B32, k, kg * 8, cur);
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
      for (int kb = 0; kb < KB && ok; ++kb, ++q) {
        const int kk0 = kb * kKB + kg * 8;
        const bool staged = xtma && kb < KB1;
        float nxt[8];
        {
          const bool last = kb + 1 == KB;
          const int64_t tn = last ? t + gridDim.x : t;
          const int kbn = last ? 0 : kb + 1;
          if (!(xtma && kbn < KB1))
            load_group<In>(cube, dq, tn * kM + r, tn < ntiles ? N : 0, B, B32, k,
                           kbn * kKB + kg * 8, nxt);
          else
            for (int e = 0; e < 8; ++e) nxt[e] = 0.f;
        }
        const int s = q % kSt;
        int okw = 1;
        if (lane == 0) {
          okw = mbar_wait(&sy->sfree[s], ((q / kSt) & 1) ^ 1, &sy->abort) ? 1 : 0;
          if (okw && staged) okw = mbar_wait(&sy->xfull[s], (q / kSt) & 1, &sy->abort) ? 1 : 0;
        }
        ok = __shfl_sync(kFull, okw, 0) != 0;
        if (!ok) break;
        if (staged) {   // row r, 16-byte units 2kg and 2kg + 1 of the swizzled block
          const unsigned char* row = xs + (size_t)s * kXStage + r * 128;
          const float4 a = *reinterpret_cast<const float4*>(row + (((2 * kg) ^ (r & 7)) << 4));
          const float4 b = *reinterpret_cast<const float4*>(row + (((2 * kg + 1) ^ (r & 7)) << 4));
          cur[0] = a.x; cur[1] = a.y; cur[2] = a.z; cur[3] = a.w;
          cur[4] = b.x; cur[5] = b.y; cur[6] = b.z; cur[7] = b.w;
        }
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int kk = kk0 + e;
          // outside both segments cur = 0 and sh = 0, so x = 0; rows past N
          // (cur = 0) reach only rows of dY that are not stored
          x[e] = fmaf(cur[e], sc[kk], sh[kk]);
          cur[e] = nxt[e];
        }
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          h[e] = pack_f16x2(x[2 * e], x[2 * e + 1]);
          float a, b2;
          unpack_f16x2(h[e], a, b2);
          l[e] = pack_f16x2(x[2 * e] - a, x[2 * e + 1] - b2);
        }
        unsigned char* ah = as + (size_t)s * 2 * kAPlane;
        *reinterpret_cast<uint4*>(ah + aoff) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(ah + kAPlane + aoff) = make_uint4(l[0], l[1], l[2], l[3]);
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sy->afull[s]);
      }
      // the converters leave the tile loop together (an abandoned wait anywhere)
      conv_bar();
      if (*(volatile int*)&sy->abort) ok = false;
      conv_bar();
      // ---------------------------------------------------------- epilogue
      if (warp < 2 + kEpiWarps) {
        int okw = 0;
        if (lane == 0) okw = (ok && mbar_wait(&sy->done, tl & 1, &sy->abort)) ? 1 : 0;
        const bool got = __shfl_sync(kFull, okw, 0) != 0;
        tc_fence_after();
        const int q4 = warp & 3;                 // TMEM lane quarter of this warp
        const int64_t row = t * kM + q4 * 32 + lane;
        const uint32_t taddr = tbase + ((uint32_t)(q4 * 32) << 16);
        // warps 2-5 the first half of the 16-column groups, warps 6-9 the rest
        const int ng = R16 / 16, gh = (ng + 1) / 2;
        const int g0 = warp < 6 ? 0 : gh, g1 = warp < 6 ? gh : ng;
        if (got) {
          const bool vec = (B & 3) == 0;          // rows of whole 16-byte units
          for (int c0 = 16 * g0; c0 < 16 * g1; c0 += 16) {
            float v1[16], v2[16];
            tmem_ld16x2(taddr + (uint32_t)c0, taddr + 256u + (uint32_t)c0, v1, v2);
#pragma unroll
            for (int e = 0; e < 16; ++e) v1[e] = fmaf(v1[e], fc[c0 + e], v2[e] * fc[256 + c0 + e]);
            if (row < N) {
              float* out = dY + row * B + c0;
              if (vec) {
#pragma unroll
                for (int e = 0; e < 16; e += 4)
                  if (c0 + e < B)
                    *reinterpret_cast<float4*>(out + e) = make_float4(v1[e], v1[e + 1], v1[e + 2], v1[e + 3]);
              } else {
#pragma unroll
                for (int e = 0; e < 16; ++e)
                  if (c0 + e < B) out[e] = v1[e];
              }
            }
          }
        } else if (lane == 0) {
          set_status(hdr, PCA_ERR_TIMEOUT);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sy->tfree);
      }
      if (!ok) break;
    }
  }
  // teardown: every MMA of this CTA has finished before TMEM is released
  if (warp == 1 && lane == 0) {
    mma_commit(&sy->drain);
    const unsigned long long t0 = gtimer();
    while (!mbar_try(&sy->drain, 0) && gtimer() - t0 < kWaitNs) {
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512)
                 : "memory");
  }
}

// ------------------------------------------------------------------ k_bwd_scales
// a_kk from the exact maxima of |x_b| (bands) and |dq_j| (|dq_j - mean| is at
// most twice that): the scaled maximum stays below 2^14.
__device__ __forceinline__ int scale_exp(float m) {
  if (!(m > 0.f) || !isfinite(m)) return 0;
  int E;
  frexpf(m, &E);               // m < 2^E
  const int e = 14 - E;
  return e < -100 ? -100 : (e > 100 ? 100 : e);
}

// Indexed by the K layout: bands kk < B, dQ columns kk = B32 + j (B32 = B
// rounded up to 32); the gap between them is 0.  One warp per entry, the
// lanes taking every 32nd partial maximum.
__global__ void k_bwd_scales(const float* __restrict__ xmax_part, const float* __restrict__ dqmax_part,
                             int parts, int B, int k, const float* __restrict__ mu32,
                             const float* __restrict__ mdq, float* __restrict__ ascale,
                             float* __restrict__ anshift) {
  const int B32 = (B + kKB - 1) & ~(kKB - 1);
  const int kk = blockIdx.x, lane = threadIdx.x;
  float m = 0.f, shift = 0.f;
  if (kk < B) {
    for (int g = lane; g < parts; g += 32) m = fmaxf(m, xmax_part[(size_t)g * B + kk]);
    shift = mu32[kk];
  } else if (kk >= B32) {
    for (int g = lane; g < parts; g += 32) m = fmaxf(m, 2.f * dqmax_part[(size_t)g * k + (kk - B32)]);
    shift = mdq[kk - B32];
  }
  m = warp_max(m);
  if (lane == 0) {
    const float s = ldexpf(1.f, scale_exp(m));
    ascale[kk] = s;
    anshift[kk] = -shift * s;   // exact: s is a power of two
  }
}

// ------------------------------------------------------------------ k_bwd_bop
// B operand, one CTA per output column c (c < B rounded to 16): entries
// S'_kk,c (kk < B) or V_c,j (kk = B32 + j), row-scaled by 2^-a_kk, then, per
// segment, the column scaled so that its largest entry lies below 2^14;
// written as FP16 hi and lo planes of each 32-wide K block in core-matrix
// order.  fcol[s * B + c] = 2^-f of segment s.
__global__ void __launch_bounds__(512)
k_bwd_bop(const float* __restrict__ S32, const float* __restrict__ vk32, int B, int k,
          const float* __restrict__ ascale, unsigned char* __restrict__ bop,
          float* __restrict__ fcol) {
  __shared__ float red[2][16];
  const int c = blockIdx.x, kk = threadIdx.x, lane = kk & 31, warp = kk >> 5;
  const int R16 = (B + 15) & ~15, B32 = (B + kKB - 1) & ~(kKB - 1);
  const int K = B32 + k, KB = (K + kKB - 1) / kKB;
  const bool seg2 = kk >= B32;
  float v = 0.f;
  if (c < B && (kk < B || (seg2 && kk < K))) {
    const float raw = kk < B ? S32[(size_t)kk * B + c] : vk32[(size_t)c * k + (kk - B32)];
    v = raw / ascale[kk];                   // exact: a power of two
  }
  const float m1 = warp_max(seg2 ? 0.f : fabsf(v)), m2 = warp_max(seg2 ? fabsf(v) : 0.f);
  if (lane == 0) { red[0][warp] = m1; red[1][warp] = m2; }
  __syncthreads();
  float m = 0.f;
#pragma unroll
  for (int w = 0; w < 16; ++w) m = fmaxf(m, red[seg2 ? 1 : 0][w]);
  const float f = ldexpf(1.f, scale_exp(m));
  if ((kk == 0 || kk == B32) && c < B) fcol[(seg2 ? B : 0) + c] = 1.f / f;  // exact
  if (kk < KB * kKB) {
    const float x = v * f;
    const __half hi = __float2half_rn(x);
    const __half lo = __float2half_rn(x - __half2float(hi));
    const int kb = kk / kKB, kg = (kk % kKB) / 8, e = kk % 8;
    const size_t plane = (size_t)R16 * kKB * 2;
    const size_t off = (size_t)kb * 2 * plane + (size_t)((c >> 3) * (int)kSBO + kg * 128 + (c & 7) * 16 + e * 2);
    *reinterpret_cast<__half*>(bop + off) = hi;
    *reinterpret_cast<__half*>(bop + off + plane) = lo;
  }
}

template <typename In>
cudaError_t dy_tc_typed(const In* cube, const float* dq, int64_t N, int B, int k,
                        const float* ascale, const float* anshift, const unsigned char* bop,
                        const float* fcol, float* dY, DevHeader* hdr, cudaStream_t st) {
  const int R16 = (B + 15) & ~15;
  // staged cube blocks: FP32 rows of whole 16-byte units (a 32-band block is
  // then one 128-byte box row)
  CUtensorMap xmap;
  const bool xtma = sizeof(In) == 4 && encode_cube_map(PCA_F32, cube, N, B, &xmap, kM);
  if (!xtma) memset(&xmap, 0, sizeof(xmap));
  size_t smem = 1024 + (size_t)kSt * kXStage + (size_t)kSt * 2 * kAPlane +
                (size_t)kSt * 2 * R16 * kKB * 2 + (size_t)(2 * kMaxKdim + 512) * 4 + sizeof(DySync);
  // more than half of an SM's shared memory: one CTA per SM, so that no two
  // CTAs compete for the 512 TMEM columns each allocates
  if (smem < 120 * 1024) smem = 120 * 1024;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = (N + kM - 1) / kM;
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  auto kern = k_bwd_dy_tc<In>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThr, smem, st>>>(xmap, xtma ? 1 : 0, cube, dq, N, B, k, ascale, anshift, bop, fcol,
                                 dY, hdr);
  return cudaGetLastError();
}

}  // namespace

size_t bwd_bop_bytes(int B, int k) {
  const int R16 = (B + 15) & ~15, B32 = (B + kKB - 1) & ~(kKB - 1);
  const int KB = (B32 + k + kKB - 1) / kKB;
  return (size_t)KB * 2 * R16 * kKB * 2;
}

cudaError_t launch_bwd_dy_tc(const void* cube, pca_dtype dt, const float* dq, int64_t N, int B,
                             int k, const float* xmax_part, const float* dqmax_part, int parts,
                             const float* mu32, const float* mdq, const float* S32,
                             const float* vk32, float* ascale, float* anshift, unsigned char* bop,
                             float* fcol, float* dY, DevHeader* hdr, cudaStream_t st) {
  if (((B + kKB - 1) & ~(kKB - 1)) + k > kMaxKdim) return cudaErrorInvalidValue;
  k_bwd_scales<<<((B + kKB - 1) & ~(kKB - 1)) + k, 32, 0, st>>>(xmax_part, dqmax_part, parts, B, k,
                                                                 mu32, mdq, ascale, anshift);
  k_bwd_bop<<<(B + 15) & ~15, 512, 0, st>>>(S32, vk32, B, k, ascale, bop, fcol);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  switch (dt) {
    case PCA_F32:
      return dy_tc_typed((const float*)cube, dq, N, B, k, ascale, anshift, bop, fcol, dY, hdr, st);
    case PCA_BF16:
      return dy_tc_typed((const __nv_bfloat16*)cube, dq, N, B, k, ascale, anshift, bop, fcol, dY,
                         hdr, st);
    case PCA_F16:
      return dy_tc_typed((const __half*)cube, dq, N, B, k, ascale, anshift, bop, fcol, dY, hdr, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbpca
