// k_project_tc.cu -- the projection Q = (Y - 1 mu^T) V_k (Algorithm 1 stages
// 5-6) on the 5th-generation tensor cores, for the mixed-precision form.
//
// Q is a skinny GEMM: M = pixels (128 per tile), K = bands, N = components.
// The cube is pixel-major, so a pixel's bands are the K-contiguous rows of the
// A operand: the converters read 16 consecutive bands of a pixel with vector
// loads and write them, shifted, scaled and split into FP16 hi + lo, as rows of
// K-major core matrices -- no transpose.  V_k is the B operand (K-major, a
// component's bands contiguous), prepared once per fit by two small kernels:
//   k_ptc_bands  per band a shift s_b (the band mean rounded to the input's
//                type, so that y - s_b is exact for 16-bit cubes) and a
//                power-of-two scale 2^e_b (the deviations of 32 sampled
//                pixels scaled into (2^5, 2^6], as in the covariance);
//   k_ptc_vop    per column j the entries v_bj 2^-e_b scaled by 2^f_j into
//                [2^13, 2^14), split into FP16 hi + lo planes in core-matrix
//                order, and the centring correction c_j = sum_b (mu_b - s_b)
//                v_bj (FP64), so that Q_nj = 2^-f_j sum_b x_nb w_bj - c_j with
//                x_nb = (y_nb - s_b) 2^e_b.
// Products x_hi [V_hi | V_lo] (one MMA of 2 N16 columns) and x_lo V_hi (only
// when a chunk has a non-zero lo part: never for 16-bit cubes within 2^11 grid
// steps of the shift), FP32 accumulation in TMEM; the K-steps of a tile rotate
// over up to eight accumulators, so that consecutive MMAs are independent and
// none sums more than a few products; double-buffered by tile.
// One persistent CTA per SM walks its 128-pixel tiles:
//   warp 0       TMA producer: when a pixel row is a whole number of 16-byte
//                units, 128-pixel x 128-byte boxes of a 2-D tensor map
//                (128-byte swizzle; one box per 64-band chunk of a 16-bit
//                cube, two of an FP32 one) into a ring of raw stages -- many
//                chunks in flight, which direct loads by the converters cannot
//                keep up (other cubes: the converters load directly);
//   warps 2-17   converters: per 64-band chunk each thread takes one pixel and
//                16 bands;
//   warp 1       MMA issuer (one thread) and TMEM owner;
//   warps 18-21  epilogue: TMEM -> registers (the chunk accumulators added in
//                FP32) -> column scale and correction -> Q rows.
// At most 128 columns per launch; more components take a second launch.  A
// scaled value outside the FP16 range sets hdr->proj_range and the caller's
// guarded SIMT projection recomputes Q.  Every wait is bounded (one second);
// on time-out the CTA records PCA_ERR_TIMEOUT, drains its MMAs and frees TMEM.
#include <cstddef>
#include <cstring>
#include <type_traits>

#include "tc.cuh"

namespace gbpca {

namespace {

constexpr int kTM = 128;                 // pixels per tile (MMA M)
constexpr int kKC = 64;                  // bands per K-chunk (one operand stage)
constexpr int kMaxSt = 6;                // operand ring depth (as shared memory allows)
constexpr int kMaxRaw = 8;               // raw-chunk ring depth of the TMA path
constexpr int kConvW = 16;               // converter warps
constexpr int kEpiW = 4;                 // epilogue warps (one per TMEM lane quarter)
constexpr int kThr = (2 + kConvW + kEpiW) * 32;
constexpr int kPlane = kTM * kKC * 2;    // one FP16 plane of an A stage: 16 KB
// Operands in the 128-byte swizzled K-major layout: one 64-band chunk is one
// row of 128 bytes per pixel (A) or per column of [V_hi | V_lo] (B).
constexpr int kMaxCols = 128;            // columns of one launch
constexpr int kProbe = 32;

struct __align__(16) PtcSync {
  uint64_t rfull[kMaxRaw];
  uint64_t rempty[kMaxRaw];
  uint64_t opfull[kMaxSt];
  uint64_t opempty[kMaxSt];
  uint64_t tdone[2];   // the MMAs of a tile finished (per TMEM buffer)
  uint64_t tfree[2];   // the epilogue has read a TMEM buffer
  uint64_t drain;
  // per converter warp: a lo part is non-zero; each stage's 16 flags are one
  // 16-byte aligned row (the MMA thread reads a row with one vector load)
  alignas(16) unsigned char lo_nz[kMaxSt][kConvW];
  uint32_t tmem_base;
  int abort;
};

static_assert(offsetof(PtcSync, lo_nz) % 16 == 0 && kConvW == 16,
              "each stage's flags must be one aligned 16-byte row");

template <typename In>
__device__ __forceinline__ float on_grid(float m);
template <>
__device__ __forceinline__ float on_grid<float>(float m) { return m; }
template <>
__device__ __forceinline__ float on_grid<__nv_bfloat16>(float m) {
  return __bfloat162float(__float2bfloat16_rn(m));
}
template <>
__device__ __forceinline__ float on_grid<__half>(float m) {
  return fabsf(m) <= 65504.f ? __half2float(__float2half_rn(m)) : m;
}

// ------------------------------------------------------------------ k_ptc_bands
// Band shifts and scales (one CTA, thread = band): s_b = mu_b on the input's
// grid; e_b from the largest |y - s_b| over 32 pixels spread through the cube.
template <typename In>
__global__ void __launch_bounds__(256)
k_ptc_bands(const In* __restrict__ cube, int64_t N, int B, const double* __restrict__ mu,
            float* __restrict__ shift, int* __restrict__ escale) {
  const int b = threadIdx.x;
  if (b >= B) return;
  const float s = on_grid<In>((float)mu[b]);
  const int Sp = (int)(N < kProbe ? N : kProbe);
  // all sampled loads in flight at once (a loop of dependent loads costs
  // kProbe memory latencies)
  float y[kProbe];
#pragma unroll
  for (int i = 0; i < kProbe; ++i)
    y[i] = i < Sp ? to_f32<In>(cube[((int64_t)i * N / Sp) * B + b]) : s;
  float dev = 0.f;
#pragma unroll
  for (int i = 0; i < kProbe; ++i) dev = fmaxf(dev, fabsf(y[i] - s));
  if (!(dev > 0.f) || !isfinite(dev)) dev = fabsf(s);
  int e = 0;
  if (dev > 0.f && isfinite(dev)) {
    int E;
    frexpf(dev, &E);        // dev < 2^E
    e = 6 - E;
    e = e < -120 ? -120 : (e > 120 ? 120 : e);
  }
  shift[b] = s;
  escale[b] = e;
}

// ------------------------------------------------------------------ k_ptc_vop
// The B operand of one launch, one CTA per column j < N16 (thread = band):
// per 64-band chunk c a block of 2 N16 rows of 128 bytes -- row j = V_hi
// column j, row N16 + j = V_lo column j -- in the 128-byte swizzled K-major
// layout (unit u of row n at u ^ (n mod 8)); the column scale 2^-f_j and the
// correction c_j.
__global__ void __launch_bounds__(256)
k_ptc_vop(const double* __restrict__ V, int B, int j0, int k, const double* __restrict__ mu,
          const float* __restrict__ shift, const int* __restrict__ escale,
          unsigned char* __restrict__ planes, float* __restrict__ colscale,
          float* __restrict__ corr) {
  __shared__ float wmax[8];
  __shared__ double csum[8];
  const int j = blockIdx.x, b = threadIdx.x, lane = b & 31, warp = b >> 5;
  const int B16 = (B + 15) & ~15, N16 = gridDim.x;
  const bool live = b < B && j < k;
  const double v = live ? V[(size_t)b * B + j0 + j] : 0.0;
  const float w = live ? ldexpf((float)v, -escale[b]) : 0.f;
  const double c = live ? (mu[b] - (double)shift[b]) * v : 0.0;
  float m = warp_max(fabsf(w));
  const double cs = warp_sum(c);
  if (lane == 0) { wmax[warp] = m; csum[warp] = cs; }
  __syncthreads();
  m = 0.f;
  double ct = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) { m = fmaxf(m, wmax[i]); ct += csum[i]; }
  int f = 0;
  if (m > 0.f && isfinite(m)) {
    int E;
    frexpf(m, &E);
    f = 14 - E;
    f = f < -100 ? -100 : (f > 100 ? 100 : f);
  }
  if (b == 0) {
    colscale[j] = ldexpf(1.f, -f);
    corr[j] = (float)ct;
  }
  if (b < ((B16 + 63) & ~63)) {   // every band of the chunks (0 past B)
    const float x = ldexpf(w, f);
    const __half hi = __float2half_rn(x);
    const __half lo = __float2half_rn(x - __half2float(hi));
    const int c = b >> 6, u = (b & 63) >> 3;
    unsigned char* blk = planes + (size_t)c * (2 * N16) * 128;
    const int nh = j, nl = N16 + j;
    *reinterpret_cast<__half*>(blk + nh * 128 + ((u ^ (nh & 7)) << 4) + (b & 7) * 2) = hi;
    *reinterpret_cast<__half*>(blk + nl * 128 + ((u ^ (nl & 7)) << 4) + (b & 7) * 2) = lo;
  }
}

// Sixteen raw values (bands b0 .. b0+15 of pixel n; 0 outside the cube).
template <typename In>
__device__ __forceinline__ void load16(const In* __restrict__ cube, int64_t n, int64_t N, int B,
                                       int b0, bool vec, float* r) {
  if (n < N && vec && b0 + 16 <= B) {
    const In* src = cube + n * B + b0;
    if constexpr (sizeof(In) == 4) {
      const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 a = __ldg(s4 + i);
        r[4 * i] = a.x; r[4 * i + 1] = a.y; r[4 * i + 2] = a.z; r[4 * i + 3] = a.w;
      }
    } else {
      const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const uint4 u = __ldg(s4 + i);
        const In* h = reinterpret_cast<const In*>(&u);
#pragma unroll
        for (int e = 0; e < 8; ++e) r[8 * i + e] = to_f32<In>(h[e]);
      }
    }
    return;
  }
#pragma unroll
  for (int e = 0; e < 16; ++e) r[e] = (n < N && b0 + e < B) ? to_f32<In>(cube[n * B + b0 + e]) : 0.f;
}

struct PtcArgs {
  const void* cube;
  int64_t N;
  int B;
  int k;               // columns of this launch
  int N16;             // k rounded up to 16
  int q_ld;            // floats between rows of proj
  float* proj;         // column 0 of this launch
  const float* shift;
  const int* escale;
  const unsigned char* planes;
  const float* colscale;
  const float* corr;
  DevHeader* hdr;
};

// Raw bytes of one 64-band chunk of a tile in the TMA ring: 128 rows of 128
// bytes per box, one box (16-bit) or two (FP32).
template <typename In>
constexpr int raw_chunk_bytes() { return kTM * 128 * (sizeof(In) == 4 ? 2 : 1); }

template <typename In, bool kTiled>
__global__ void __launch_bounds__(kThr, 1)
k_project_tc(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ PtcArgs a, int S,
             int R, int nacc) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  const int B = a.B, N16 = a.N16;
  const int B16 = (B + 15) & ~15;
  const int KC = (B16 + kKC - 1) / kKC;                    // K-chunks per tile
  const int vbytes = KC * 2 * N16 * 128;                   // [V_hi | V_lo], all chunks
  constexpr int kRaw = raw_chunk_bytes<In>();
  unsigned char* raw = smem;                               // [R][kRaw] (TMA path)
  // V: the lo plane right after the hi plane, so that [V_hi | V_lo] is one B
  // operand of 2 N16 rows (one MMA gives both products of a K-step)
  unsigned char* vs = raw + (size_t)R * kRaw;              // [KC][2 N16][128]
  unsigned char* ops = vs + ((vbytes + 1023) & ~1023);     // [S][hi|lo][kPlane]
  float2* cst = reinterpret_cast<float2*>(ops + (size_t)S * 2 * kPlane);  // [256] (2^e, -s 2^e)
  float* cls = reinterpret_cast<float*>(cst + 256);                       // [128] 2^-f
  float* crs = cls + kMaxCols;                                            // [128] c_j
  PtcSync* sy = reinterpret_cast<PtcSync*>((reinterpret_cast<uintptr_t>(crs + kMaxCols) + 15) &
                                            ~static_cast<uintptr_t>(15));

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const In* cube = static_cast<const In*>(a.cube);
  const int64_t N = a.N;
  const int64_t ntiles = (N + kTM - 1) / kTM;
  const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
  const int nt = (int)(t1 - t0);

  // ---- set-up: V planes, zero lo planes, band and column constants, barriers, TMEM
  {
    const uint4* src = reinterpret_cast<const uint4*>(a.planes);
    for (int i = tid; i < vbytes / 16; i += kThr) reinterpret_cast<uint4*>(vs)[i] = src[i];
    // the converters store a lo unit only when it is (or was) non-zero
    for (int i = tid; i < S * (kPlane / 16); i += kThr) {
      const int st = i / (kPlane / 16), u = i - st * (kPlane / 16);
      reinterpret_cast<uint4*>(ops + (size_t)(st * 2 + 1) * kPlane)[u] = make_uint4(0, 0, 0, 0);
    }
  }
  // x = (y - s) 2^e as one FMA: y 2^e is exact (a power of two) and the sum is
  // rounded once, as (y - s) would be before the exact scaling
  // 16-bit cubes read through the tensor map: the raw pairs enter the FMA,
  // the scales as pairs of the input type (FP16: when every band's scale is
  // in FP16's normal range)
  constexpr bool kMix16 = sizeof(In) == 2 && kTiled;
  constexpr bool kBf = std::is_same<In, __nv_bfloat16>::value;
  bool in_range = true;
  for (int b = tid; b < B; b += kThr) in_range &= kBf || (a.escale[b] >= -14 && a.escale[b] <= 15);
  const bool mix_ok = kMix16 && __syncthreads_and(in_range);
  if (mix_ok) {
    // [256] shifts -s 2^e (FP32), then [128] packed scale pairs
    float* shf = reinterpret_cast<float*>(cst);
    uint32_t* scb = reinterpret_cast<uint32_t*>(shf + 256);
    for (int b = tid; b < 256; b += kThr)
      shf[b] = b < B ? -a.shift[b] * ldexpf(1.f, a.escale[b]) : 0.f;
    auto pw = [&](int e) { return kBf ? bf16_pow2(e) : f16_pow2(e); };
    for (int b2 = tid; b2 < 128; b2 += kThr) {
      const int b = 2 * b2;
      scb[b2] = (b < B ? pw(a.escale[b]) : 0u) | ((b + 1 < B ? pw(a.escale[b + 1]) : 0u) << 16);
    }
  } else {
    for (int b = tid; b < 256; b += kThr) {
      const float sc = b < B ? ldexpf(1.f, a.escale[b]) : 0.f;
      cst[b] = make_float2(sc, b < B ? -a.shift[b] * sc : 0.f);
    }
  }
  for (int j = tid; j < kMaxCols; j += kThr) {
    cls[j] = j < a.k ? a.colscale[j] : 0.f;
    crs[j] = j < a.k ? a.corr[j] : 0.f;
  }
  if (tid == 0) {
    for (int s = 0; s < R; ++s) { mbar_init(&sy->rfull[s], 1); mbar_init(&sy->rempty[s], kConvW); }
    for (int s = 0; s < S; ++s) { mbar_init(&sy->opfull[s], kConvW); mbar_init(&sy->opempty[s], 1); }
    for (int i = 0; i < 2; ++i) { mbar_init(&sy->tdone[i], 1); mbar_init(&sy->tfree[i], kEpiW); }
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
  // nacc accumulators of 2 N16 columns per tile buffer, the K-steps of a tile
  // rotating over them (consecutive MMAs do not wait for each other): columns
  // [0, N16) sum x_hi V_hi (+ x_lo V_hi), [N16, 2 N16) sum x_hi V_lo
  const int accw = nacc * 2 * N16;        // TMEM columns of one tile buffer

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (kTiled && lane == 0) {
      Ring rs(R);
      bool go = true;
      for (int i = 0; i < nt && go; ++i) {
        const int y = (int)((t0 + i) * kTM);
        for (int c = 0; c < KC; ++c, rs.next()) {
          if (!mbar_wait(&sy->rempty[rs.idx], rs.phase ^ 1u, &sy->abort)) { go = false; break; }
          unsigned char* dst = raw + (size_t)rs.idx * kRaw;
          mbar_expect_tx(&sy->rfull[rs.idx], (uint32_t)kRaw);
          tma_load_2d(dst, &xmap, c * kKC, y, &sy->rfull[rs.idx]);
          if (sizeof(In) == 4)
            tma_load_2d(dst + kTM * 128, &xmap, c * kKC + 32, y, &sy->rfull[rs.idx]);
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    // The whole warp runs this loop (uniform control flow); lane 0 waits on the
    // barriers and broadcasts the outcome, one elected lane issues each MMA.
    const uint32_t ops_base = su32(ops), vhi = su32(vs);
    const uint32_t id_both = idesc_f16(2 * N16), id_hi = idesc_f16(N16);
    // descriptors of the operand bases; an offset of d bytes adds d >> 4 to
    // the start-address field (every address stays below 256 KB)
    const uint64_t dA = sdesc_sw128(ops_base);
    const uint64_t dV = sdesc_sw128(vhi);   // chunk c: [V_hi | V_lo] at c * 2 N16 * 128
    Ring ro(S);
    bool ok = true;
    for (int i = 0; i < nt && ok; ++i) {
      const int bf = i & 1;
      // the epilogue has read this buffer's previous tile (i - 2)
      if (i >= 2) {
        int w = 1;
        if (lane == 0) w = mbar_wait(&sy->tfree[bf], ((i - 2) >> 1) & 1, &sy->abort) ? 1 : 0;
        if (!__shfl_sync(kFull, w, 0)) break;
      }
      tc_fence_after();
      const uint32_t acc0 = tbase + (uint32_t)(bf * accw);
      int ai = 0, ks = 0;      // rotating accumulator, K-step of the tile
      for (int c = 0; c < KC; ++c, ro.next()) {
        const int o = ro.idx;
        int w = 1;
        if (lane == 0) w = mbar_wait(&sy->opfull[o], ro.phase, &sy->abort) ? 1 : 0;
        if (!__shfl_sync(kFull, w, 0)) { ok = false; break; }
        tc_fence_after();
        uint32_t f0, f1, f2, f3;   // the 16 warps' flags in one 16-byte load
        asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(f0), "=r"(f1), "=r"(f2), "=r"(f3)
                     : "r"(su32(sy->lo_nz[o])));
        const uint32_t nz = (f0 | f1) | (f2 | f3);
        const uint64_t ahi = dA + (uint64_t)((o * 2 * kPlane) >> 4), alo = ahi + (kPlane >> 4);
        const int ksteps = (B16 - c * kKC) < kKC ? (B16 - c * kKC) / 16 : kKC / 16;
        const uint64_t vc = dV + (uint64_t)((c * 2 * N16 * 128) >> 4);
        for (int kk = 0; kk < ksteps; ++kk, ++ks) {
          const uint64_t kofs = (uint64_t)(kk * 32 >> 4);     // 16 K-values = 32 bytes
          const uint32_t acc = acc0 + (uint32_t)(ai * 2 * N16);
          mma_f16_warp(acc, ahi + kofs, vc + kofs, id_both, ks < nacc ? 0u : 1u);
          if (nz) mma_f16_warp(acc, alo + kofs, vc + kofs, id_hi, 1u);
          ai = ai + 1 == nacc ? 0 : ai + 1;
        }
        mma_commit_warp(&sy->opempty[o]);
      }
      if (ok) mma_commit_warp(&sy->tdone[bf]);
    }
    __syncwarp();
  } else if (warp >= 2 && warp < 2 + kConvW) {
    // ------------------------------------------------------------ converters
    const int ct = tid - 64, cw = warp - 2;
    const int pr = ct % kTM, gp = ct / kTM;   // pixel row of the tile; 16-band group of a chunk
    const bool vec = (B * (int)sizeof(In)) % 16 == 0;
    const int Q = nt * KC;
    float cur[16], nxt[16];
    uint32_t raw16[8];       // BF16 path: the 16 values as 8 packed pairs
    // (tile, chunk) of the chunk being converted and of the next one
    int64_t tile = t0, ntile = t0;
    int c = 0, nc = 0;
    auto advance = [&](int64_t& t, int& cc) { if (++cc == KC) { cc = 0; ++t; } };
    if (!kTiled && Q > 0) load16<In>(cube, t0 * kTM + pr, N, B, gp * 16, vec, cur);
    advance(ntile, nc);
    // a value beyond the FP16 range -> fallback.  FP32 cubes track the largest
    // |x|; for 16-bit cubes (whose lo parts are nearly always zero) an
    // infinite lo part is the sign of it, checked where lo is stored
    constexpr bool k16 = sizeof(In) == 2;
    float mx = 0.f;
    int rng = 0;
    uint32_t dirty = 0u;      // bit o: this thread's lo units of operand stage o are non-zero
    Ring ro(S), rs(R > 0 ? R : 1);
    for (int q = 0; q < Q; ++q, ro.next(), rs.next()) {
      const int o = ro.idx;
      if constexpr (kTiled) {
        // bands gp*16 .. +15 of row pr: 16-byte units of the swizzled box row
        const int s = rs.idx;
        int okr = 1;
        if (lane == 0) okr = mbar_wait(&sy->rfull[s], rs.phase, &sy->abort) ? 1 : 0;
        okr = __shfl_sync(kFull, okr, 0);
        if (!okr) break;
        const unsigned char* box = raw + (size_t)s * kRaw;
        constexpr int E = 16 / (int)sizeof(In);          // elements per 16-byte unit
        constexpr int U = 16 / E;                        // units of 16 bands
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int unit = gp * U + u;                   // unit of the chunk (8 per box)
          const unsigned char* bx = box + (size_t)(unit >> 3) * kTM * 128;
          const uint4 v = *reinterpret_cast<const uint4*>(
              bx + pr * 128 + (((unit & 7) ^ (pr & 7)) << 4));
          if constexpr (kMix16) {
            raw16[4 * u] = v.x; raw16[4 * u + 1] = v.y; raw16[4 * u + 2] = v.z; raw16[4 * u + 3] = v.w;
          } else {
            const In* h = reinterpret_cast<const In*>(&v);
#pragma unroll
            for (int e = 0; e < E; ++e) cur[u * E + e] = to_f32<In>(h[e]);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sy->rempty[s]);
      } else {
        if (q + 1 < Q) load16<In>(cube, ntile * kTM + pr, N, B, nc * kKC + gp * 16, vec, nxt);
      }
      const int b0 = c * kKC + gp * 16;
      const bool row = tile * kTM + pr < N;    // rows past the cube stay 0
      float x[16];
      if constexpr (kMix16) {
        if (!mix_ok) {   // FP16 scales out of range: widen the raw values
          const In* h16 = reinterpret_cast<const In*>(raw16);
#pragma unroll
          for (int e = 0; e < 16; ++e) cur[e] = to_f32<In>(h16[e]);
        }
      }
      if (kMix16 && mix_ok) {
        // the 16-bit pairs enter the FMA as they are; constants: 16 shifts and
        // 8 scale pairs (broadcast reads: the lanes of a warp share b0)
        const float* shf = reinterpret_cast<const float*>(cst);
        const uint32_t* scb = reinterpret_cast<const uint32_t*>(shf + 256);
        float sh[16];
        uint32_t sp[8];
#pragma unroll
        for (int e = 0; e < 16; e += 4) {
          const float4 t = *reinterpret_cast<const float4*>(shf + b0 + e);
          sh[e] = t.x; sh[e + 1] = t.y; sh[e + 2] = t.z; sh[e + 3] = t.w;
        }
#pragma unroll
        for (int e = 0; e < 8; e += 4) {
          const uint4 t = *reinterpret_cast<const uint4*>(scb + (b0 >> 1) + e);
          sp[e] = t.x; sp[e + 1] = t.y; sp[e + 2] = t.z; sp[e + 3] = t.w;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          if constexpr (kBf) fma_bf16x2_f32(raw16[e], sp[e], sh[2 * e], sh[2 * e + 1], x[2 * e], x[2 * e + 1]);
          else fma_f16x2_f32(raw16[e], sp[e], sh[2 * e], sh[2 * e + 1], x[2 * e], x[2 * e + 1]);
        }
        if (!(row && b0 + 16 <= B)) {
#pragma unroll
          for (int e = 0; e < 16; ++e) x[e] = row && b0 + e < B ? x[e] : 0.f;
        }
      } else {
        // the 16 bands' constants (broadcast reads: every lane of the warp has the same b0)
        float2 kc[16];
#pragma unroll
        for (int e = 0; e < 16; e += 2) {
          const float4 t = *reinterpret_cast<const float4*>(cst + b0 + e);
          kc[e] = make_float2(t.x, t.y);
          kc[e + 1] = make_float2(t.z, t.w);
        }
        if (row && b0 + 16 <= B) {
#pragma unroll
          for (int e = 0; e < 16; ++e) x[e] = fmaf(cur[e], kc[e].x, kc[e].y);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) x[e] = row && b0 + e < B ? fmaf(cur[e], kc[e].x, kc[e].y) : 0.f;
        }
      }
      uint32_t h[8], l[8];
      uint32_t lo_bits = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        if constexpr (!k16) mx = fmaxf(mx, fmaxf(fabsf(x[2 * e]), fabsf(x[2 * e + 1])));
        h[e] = pack_f16x2(x[2 * e], x[2 * e + 1]);
        float r0, r1;
        if constexpr (kMix16) {
          resid_f16x2(h[e], x[2 * e], x[2 * e + 1], r0, r1);
        } else {
          unpack_f16x2(h[e], r0, r1);
          r0 = x[2 * e] - r0;
          r1 = x[2 * e + 1] - r1;
        }
        l[e] = pack_f16x2(r0, r1);
        lo_bits |= l[e];
      }
      const int any_lo = __any_sync(kFull, lo_bits != 0u);
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&sy->opempty[o], ro.phase ^ 1u, &sy->abort) ? 1 : 0;
      ok = __shfl_sync(kFull, ok, 0);
      if (!ok) break;
      // row pr of the A stage, bands gp*16 .. +15 = core matrices 2gp, 2gp+1
      unsigned char* hi = ops + (size_t)(o * 2) * kPlane;
      unsigned char* lo = hi + kPlane;
      // row pr, units 2 gp and 2 gp + 1, swizzled
      const uint32_t o0 = (uint32_t)pr * 128 + ((uint32_t)((2 * gp) ^ (pr & 7)) << 4);
      const uint32_t o1 = (uint32_t)pr * 128 + ((uint32_t)((2 * gp + 1) ^ (pr & 7)) << 4);
      *reinterpret_cast<uint4*>(hi + o0) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(hi + o1) = make_uint4(h[4], h[5], h[6], h[7]);
      // lo units: stored when non-zero, or to clear what this thread left
      // there before; units that are and stay zero are skipped
      if (lo_bits != 0u || (dirty & (1u << o))) {
        *reinterpret_cast<uint4*>(lo + o0) = make_uint4(l[0], l[1], l[2], l[3]);
        *reinterpret_cast<uint4*>(lo + o1) = make_uint4(l[4], l[5], l[6], l[7]);
        dirty = lo_bits != 0u ? (dirty | (1u << o)) : (dirty & ~(1u << o));
        if constexpr (k16) {
          bool inf = false;
#pragma unroll
          for (int e = 0; e < 8; ++e) inf |= f16x2_has_inf(l[e]);
          rng |= inf ? 1 : 0;
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        sy->lo_nz[o][cw] = (unsigned char)any_lo;   // published by the release of the arrival below
        mbar_arrive(&sy->opfull[o]);
      }
      if constexpr (!kTiled) {
#pragma unroll
        for (int e = 0; e < 16; ++e) cur[e] = nxt[e];
      }
      advance(tile, c);
      advance(ntile, nc);
    }
    const int bad = !(mx <= 65504.f) || rng != 0;
    if (__any_sync(kFull, bad) && lane == 0 && a.hdr) atomicOr(&a.hdr->proj_range, 1);
  } else if (warp >= 2 + kConvW) {
    // ------------------------------------------------------------ epilogue
    const int q4 = warp & 3;
    const int r = q4 * 32 + lane;
    const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
    const int nused = nacc < B16 / 16 ? nacc : B16 / 16;   // accumulators a tile writes
    const bool v4 = (a.q_ld & 3) == 0 && (a.k & 3) == 0 &&
                    (reinterpret_cast<uintptr_t>(a.proj) & 15) == 0;
    bool ok = true;
    for (int i = 0; i < nt; ++i) {
      const int bf = i & 1;
      int okw = 0;
      if (lane == 0) okw = mbar_wait(&sy->tdone[bf], (i >> 1) & 1, &sy->abort) ? 1 : 0;
      ok = __shfl_sync(kFull, okw, 0) != 0;
      if (!ok) break;
      tc_fence_after();
      const int64_t n = (t0 + i) * kTM + r;
      float* out = a.proj + n * a.q_ld;
      for (int j0 = 0; j0 < N16; j0 += 16) {
        float v[16], w[16];
        const uint32_t t = tbase + lane_off + (uint32_t)(bf * accw + j0);
        // both halves of every accumulator (two loads in flight per wait)
        tmem_ld16x2(t, t + (uint32_t)N16, v, w);
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] += w[e];
        for (int ac = 1; ac < nused; ++ac) {
          float x2[16], y2[16];
          const uint32_t ta = t + (uint32_t)(ac * 2 * N16);
          tmem_ld16x2(ta, ta + (uint32_t)N16, x2, y2);
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] += x2[e] + y2[e];
        }
        if (n < N) {
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = v[e] * cls[j0 + e] - crs[j0 + e];
          if (v4 && j0 + 16 <= a.k) {
#pragma unroll
            for (int e = 0; e < 16; e += 4)
              *reinterpret_cast<float4*>(out + j0 + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
          } else {
#pragma unroll
            for (int e = 0; e < 16; ++e)
              if (j0 + e < a.k) out[j0 + e] = v[e];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sy->tfree[bf]);
    }
    if (!ok) {
      // a bounded wait gave up: this CTA's remaining rows are invalid
      for (int64_t n = (t0 * kTM) + r; n < t1 * kTM && n < N; n += kTM)
        for (int j = 0; j < a.k; ++j) a.proj[n * a.q_ld + j] = __int_as_float(0x7fc00000);
      if (lane == 0 && a.hdr) set_status(a.hdr, PCA_ERR_TIMEOUT);
    }
  }
  // teardown: every MMA of this CTA has finished before TMEM is released
  if (warp == 1 && lane == 0) {
    mma_commit(&sy->drain);
    const unsigned long long tw = gtimer();
    while (!mbar_try(&sy->drain, 0) && gtimer() - tw < kWaitNs) {
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

size_t ptc_smem(int B, int N16, int S, int R, int raw_bytes) {
  const int KC = (((B + 15) & ~15) + kKC - 1) / kKC;
  const size_t vplanes = (size_t)((KC * 2 * N16 * 128 + 1023) & ~1023);
  return 1024 + (size_t)R * raw_bytes + vplanes + (size_t)S * 2 * kPlane +
         (256 * 2 + 2 * kMaxCols) * 4 + sizeof(PtcSync) + 16;   // cst[256] float2 + cls + crs
}

template <typename In>
cudaError_t ptc_typed(const PtcArgs& a, cudaStream_t st) {
  // the tensor-map path when the rows are whole 16-byte units
  CUtensorMap xmap;
  bool tiled = encode_cube_map(sizeof(In) == 4 ? PCA_F32 : (std::is_same<In, __half>::value
                                                              ? PCA_F16 : PCA_BF16),
                               a.cube, a.N, a.B, &xmap, kTM);
  const int rb = raw_chunk_bytes<In>();
  const size_t budget = (size_t)227 * 1024;
  auto fits = [&](int s_, int r_) { return ptc_smem(a.B, a.N16, s_, r_, rb) <= budget; };
  // tensor-map path: 3 operand stages if they fit (else 2), then as many raw
  // stages as fit (2..8); when not even 2 + 2 fit, the direct-load path
  const pca_tuning tu = tuning();
  int S = 2, R = 0;
  if (tiled && !fits(2, 2)) tiled = false;
  if (tiled) {
    S = fits(3, 2) ? 3 : 2;
    if (tu.proj_tc_stages >= 2 && tu.proj_tc_stages <= kMaxSt && fits(tu.proj_tc_stages, 2))
      S = tu.proj_tc_stages;
    R = 2;
    while (R < kMaxRaw && fits(S, R + 1) && (tu.proj_tc_raw_stages == 0 || R < tu.proj_tc_raw_stages))
      ++R;
  } else {
    S = kMaxSt;
    while (S > 2 && !fits(S, 0)) --S;
    if (!fits(S, 0)) return cudaErrorInvalidValue;
    memset(&xmap, 0, sizeof(xmap));
  }
  const int B16 = (a.B + 15) & ~15;
  // accumulators of 2 N16 columns per tile buffer (two buffers in 512 columns)
  int nacc = 256 / (2 * a.N16);
  nacc = nacc > B16 / 16 ? B16 / 16 : nacc;
  nacc = nacc < 1 ? 1 : nacc;
  const size_t smem = ptc_smem(a.B, a.N16, S, R, rb);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  sms = sms - tu.stream_sms_reserve > 1 ? sms - tu.stream_sms_reserve : 1;  // SMs left to a concurrent fit
  const int64_t ntiles = (a.N + kTM - 1) / kTM;
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  auto kern = tiled ? k_project_tc<In, true> : k_project_tc<In, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThr, smem, st>>>(xmap, a, S, R, nacc);
  return cudaGetLastError();
}

}  // namespace

size_t project_tc_planes_bytes(int B, int k) {
  const int KC = (((B + 15) & ~15) + kKC - 1) / kKC;
  const int N16 = ((k < kMaxCols ? k : kMaxCols) + 15) & ~15;
  return (size_t)KC * 2 * N16 * 128;
}

cudaError_t launch_project_tc(const void* cube, pca_dtype dt, int64_t N, int B, int k,
                              const double* mu, const double* V, float* proj, float* shift,
                              int* escale, unsigned char* planes, float* colscale, float* corr,
                              DevHeader* hdr, cudaStream_t st) {
  if (N < 1) return cudaSuccess;
  switch (dt) {
    case PCA_F32:
      k_ptc_bands<float><<<1, 256, 0, st>>>((const float*)cube, N, B, mu, shift, escale);
      break;
    case PCA_BF16:
      k_ptc_bands<__nv_bfloat16><<<1, 256, 0, st>>>((const __nv_bfloat16*)cube, N, B, mu, shift,
                                                     escale);
      break;
    case PCA_F16:
      k_ptc_bands<__half><<<1, 256, 0, st>>>((const __half*)cube, N, B, mu, shift, escale);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // one launch per group of at most 128 columns (the V operand in shared memory)
  for (int j0 = 0; j0 < k; j0 += kMaxCols) {
    const int kk = k - j0 < kMaxCols ? k - j0 : kMaxCols;
    const int N16 = (kk + 15) & ~15;
    k_ptc_vop<<<N16, 256, 0, st>>>(V, B, j0, kk, mu, shift, escale, planes, colscale, corr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const PtcArgs a{cube, N, B, kk, N16, k, proj + j0, shift, escale, planes, colscale, corr, hdr};
    switch (dt) {
      case PCA_F32: e = ptc_typed<float>(a, st); break;
      case PCA_BF16: e = ptc_typed<__nv_bfloat16>(a, st); break;
      case PCA_F16: e = ptc_typed<__half>(a, st); break;
      default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace gbpca
