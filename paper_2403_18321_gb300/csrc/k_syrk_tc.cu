// k_syrk_tc.cu -- covariance partials on the 5th-generation tensor cores
// (tcgen05 + TMEM), the dense contraction of Algorithm 1 stage 3 (Sec. 4.2
// stage 3 forms it with one cuBLAS SGEMM; here it is hand-written).
//
// One persistent CTA per SM walks its work items -- for a single cube a
// contiguous range of 32-pixel chunks, for a batch a list of (tile, pixel
// range) items -- in 32-pixel chunks:
//   warp 0      TMA producer: cp.async.bulk of each chunk (pixel-major, a
//               contiguous byte range of the cube) into a ring of as many
//               stages (up to 12) as shared memory holds;
//   warps 2-17  converters: x = (y - s) 2^e per band (s = the mean of 32
//               pixels spread through the cube and e a power-of-two scale,
//               both computed by every CTA from the same pixels), split into
//               FP16 hi = fp16(x), lo = fp16(x - hi) -- 22 significant bits
//               of x -- written in the cube's own [pixel][band] order as
//               MN-major operands with the 128-byte swizzle (16-byte vector
//               loads and stores) into a 3-stage operand ring; a thread owns
//               8 bands of two pixel rows and keeps their constants in
//               registers; a lo unit is stored only when it is non-zero or
//               was non-zero the last time; each warp flags whether any lo of
//               its values is non-zero;
//   warp 1      MMA issuer (one thread): D += hi hi^T + hi lo^T + lo hi^T
//               for the upper block-triangle (row tile 0: bands 0-127 x all;
//               row tile 1: bands 128-255 x bands 128-255) with FP32
//               accumulation in TMEM, and the band sums S1 = (hi + lo)^T 1
//               against a constant operand of ones (N = 16, column 0).  A chunk whose lo parts are all zero
//               gets the first product only: the other two are exactly zero.
//               That is the rule for 16-bit cubes, whose shift is rounded to
//               the input type: y - s then has at most the bits of the
//               input's grid, which a single FP16 holds as long as the
//               pixel's deviation stays within 2^11 grid steps;
//   then, after the item's last chunk, the same 16 warps are the epilogue:
//               TMEM -> registers -> the item's partial slot (packed upper
//               triangle, FP32, still scaled by 2^(e_i+e_j)) and S1 (FP64,
//               unscaled).  S1 shares the covariance entries' accumulation:
//               exact for 16-bit cubes within their runs, FP32 runs otherwise.
// The rings continue across items; the MMAs of an item start once the
// epilogue of the previous one has read the accumulators out of TMEM.
// A scaled value outside the FP16 range sets hdr->cov_range; the caller then
// recomputes the partials on the SIMT path.  The partials are reduced and
// finalised by k_cov.cu.  Every mbarrier wait is bounded (one second of
// globaltimer); on time-out the CTA records PCA_ERR_TIMEOUT, drains its MMAs,
// frees TMEM and returns.
#include <type_traits>

#include "tc.cuh"

namespace gbpca {

namespace {

constexpr int kKC = 32;                 // pixels per chunk (K of one stage)
constexpr int kMaxStages = 12;          // TMA ring depth: as many stages as shared memory holds
constexpr int kOpStages = 3;            // FP16 operand ring depth
constexpr int kRows = 256;              // operand rows (bands, padded to 16)
#ifndef GBPCA_COV_CONV_WARPS
#define GBPCA_COV_CONV_WARPS 16
#endif
constexpr int kConvWarps = GBPCA_COV_CONV_WARPS;   // 8 or 16
constexpr int kThreads = (2 + kConvWarps) * 32;
constexpr int kConvThreads = kConvWarps * 32;
constexpr int kRowsPT = 32 * 32 / kConvThreads;  // pixel rows of a chunk per converter thread
constexpr int kRowStep = 32 / kRowsPT;           // a thread's rows: pr, pr + kRowStep, ...
constexpr int kProbeHalves = kConvThreads / 256; // threads per band in the probe
static_assert(kConvWarps == 8 || kConvWarps == 16, "8 or 16 converter warps");
constexpr int kOpBytes = kRows * kKC * 2;        // one FP16 operand (hi or lo): 16 KB
// Operands in the MN-major layout with the 128-byte swizzle, in the cube's own
// order: per pixel (K) a row of 64 bands (MN) = 128 bytes; 8 pixel rows form a
// 1 KB swizzle atom; the 4 atoms of a 32-pixel chunk make a 4 KB block of 64
// bands; the blocks of bands 0-63, 64-127, ... follow each other.
constexpr uint32_t kMnSBO = 1024;                // next 8 pixels (K)
constexpr uint32_t kMnLBO = (kKC / 8) * 1024;    // next 64 bands (MN): 4 KB
constexpr int kTmemCols = 512;
constexpr int kOnesBytes = 16 * 128;     // B operand of the band sums: 16 rows x 128 bytes
constexpr uint32_t kS1Col = 384;         // TMEM columns of the band sums (tile 0; tile 1 at +16)
constexpr int kProbe = 32;               // pixels of the band probe

struct __align__(8) SyncBlock {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t opfull[kOpStages];
  uint64_t opempty[kOpStages];
  uint64_t done;       // the MMAs of an item finished (one phase per item)
  uint64_t tfree;      // the epilogue has read the item's accumulators out of TMEM
  uint64_t drain;      // every MMA of the CTA finished (teardown)
  int lo_nz[kOpStages][kConvWarps];  // per operand stage and converter warp: a lo part is non-zero
  uint32_t tmem_base;
  int abort;
};

// MN-major 128-byte swizzled operand descriptor of the ring layout
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(kMnLBO >> 4) << 16) |
         ((uint64_t)(kMnSBO >> 4) << 32) | (1ull << 46) | (2ull << 61);
}
// kind::f16 instruction descriptor with both operands MN-major
__device__ __forceinline__ uint32_t idesc_mn(int n) { return idesc_f16(n) | (1u << 15) | (1u << 16); }

// The band sums S1 come out of the tensor cores.  Up to 248 bands, operand row
// ob = 8 G8 (the first 8-band group past the data) holds 1.0 for every pixel,
// so accumulator column ob sums each band's values, hi + lo, like any
// covariance entry; wider cubes have no free row below 256 and take S1 from
// extra MMAs against a separate operand of ones.
__device__ __forceinline__ int ones_band(int B) {
  const int ob = ((B + 7) >> 3) << 3;
  return ob < kRows ? ob : -1;
}
// operand rows (bands, and the ones row) padded to the 16-row MMA granule
__device__ __forceinline__ int mma_rows(int B) {
  const int ob = ones_band(B);
  return ob >= 0 ? (ob + 16) & ~15 : (B + 15) & ~15;
}

template <typename In>
__device__ __forceinline__ float elem(const In* p) { return to_f32<In>(*p); }

// The band shift on the input's own grid (16-bit cubes), so that y - s is exact
// in FP32 and carries no more bits than the input does.
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

// barriers among the converter warps only (the producer and MMA warps are busy)
__device__ __forceinline__ void conv_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kConvWarps * 32) : "memory");
}
__device__ __forceinline__ int conv_or(int v) {  // barrier + OR over the converter threads
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n"
      " selp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(v), "n"(kConvWarps * 32)
      : "memory");
  return r;
}

// One tile as the kernel sees it (the single-cube form passes it by value).
struct TcTile {
  const void* cube;
  int64_t N;
  int B;
  int slots;          // single cube: partial slots, split evenly over the CTAs
  float* shift;       // written by the CTA holding partial slot 0
  int* escale;
  double* s1_part;    // [slots][B]
  float* s2_part;     // [slots][B(B+1)/2]
  DevHeader* hdr;
};

// One work item: pixels [p0, p1) of a tile into partial slot `slot`.
struct TcItem {
  TcTile t;
  int64_t p0, p1;
  int slot;
};

__device__ __forceinline__ TcItem tc_item(const TcTile& one, const TileDesc* __restrict__ T,
                                          const CovItem* __restrict__ items,
                                          const int* __restrict__ cta_items, int i) {
  TcItem it;
  if (T == nullptr) {  // single cube: CTA g takes its share of the slots, slot s
                       // its share of the 32-pixel chunks
    const int G = gridDim.x, g = blockIdx.x;
    const int s = (int)((int64_t)one.slots * g / G) + i;
    const int64_t nchunk = (one.N + kKC - 1) / kKC;
    it.t = one;
    it.p0 = nchunk * s / one.slots * kKC;
    it.p1 = nchunk * (s + 1) / one.slots * kKC;
    if (it.p1 > one.N) it.p1 = one.N;
    it.slot = s;
  } else {
    const CovItem ci = items[cta_items[blockIdx.x] + i];
    const TileDesc& d = T[ci.tile];
    it.t.cube = d.cube;
    it.t.N = d.N;
    it.t.B = d.B;
    it.t.shift = d.shift;
    it.t.escale = d.escale;
    it.t.s1_part = d.s1p;
    it.t.s2_part = static_cast<float*>(d.s2p);
    it.t.hdr = d.hdr;
    it.p0 = ci.p0;
    it.p1 = ci.p1;
    it.slot = ci.slot;
  }
  return it;
}

template <typename In>
__global__ void __launch_bounds__(kThreads, 1)
k_syrk_tc(const __grid_constant__ TcTile one, const TileDesc* __restrict__ T,
          const CovItem* __restrict__ items, const int* __restrict__ cta_items, int S,
          int stage_stride) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* ops = smem;                                        // [kOpStages][hi|lo][kOpBytes]
  unsigned char* ones = smem + kOpStages * 2 * kOpBytes;            // [16][128 B], row 0 = 1.0
  unsigned char* stages = ones + kOnesBytes;                        // [S][stage_stride]
  float* shs = reinterpret_cast<float*>(stages + S * stage_stride);        // [kRows] shift
  int* sesc = reinterpret_cast<int*>(shs + kRows);                         // [kRows] exponent
  double* psum = reinterpret_cast<double*>(sesc + kRows);                  // [2][kRows]
  float* pmin = reinterpret_cast<float*>(psum + 2 * kRows);                // [2][kRows]
  float* pmax = pmin + 2 * kRows;                                          // [2][kRows]
  SyncBlock* sb = reinterpret_cast<SyncBlock*>(pmax + 2 * kRows);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nitems =
      T == nullptr ? (int)((int64_t)one.slots * (blockIdx.x + 1) / gridDim.x -
                           (int64_t)one.slots * blockIdx.x / gridDim.x)
                   : cta_items[blockIdx.x + 1] - cta_items[blockIdx.x];

  // ---- set-up
  for (int i = tid; i < kOpStages * 2 * kOpBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(ops)[i] = make_uint4(0, 0, 0, 0);
  // the ones operand: K-major (pixels contiguous), row 0 = FP16 1.0 for every
  // pixel, rows 1-15 zero (the 128-byte swizzle only permutes 16-byte units
  // inside a row, so it leaves this pattern as it is)
  for (int i = tid; i < kOnesBytes / 16; i += kThreads) {
    const uint32_t w = i < 8 ? 0x3c003c00u : 0u;
    reinterpret_cast<uint4*>(ones)[i] = make_uint4(w, w, w, w);
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&sb->full[s], 1); mbar_init(&sb->empty[s], kConvWarps); }
    for (int s = 0; s < kOpStages; ++s) { mbar_init(&sb->opfull[s], kConvWarps); mbar_init(&sb->opempty[s], 1); }
    mbar_init(&sb->done, 1);
    mbar_init(&sb->tfree, kConvWarps);
    mbar_init(&sb->drain, 1);
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

  if (warp == 0) {
    // ---------------------------------------------------------- TMA producer
    if (lane == 0) {
      Ring rq(S);  // ring position, continued across items
      bool ok = true;
      for (int i = 0; i < nitems && ok; ++i) {
        const TcItem it = tc_item(one, T, items, cta_items, i);
        const In* cube = static_cast<const In*>(it.t.cube);
        const int B = it.t.B;
        for (int64_t p0 = it.p0; p0 < it.p1; p0 += kKC, rq.next()) {
          const int s = rq.idx;
          if (!mbar_wait(&sb->empty[s], rq.phase ^ 1u, &sb->abort)) { ok = false; break; }
          const int cp = (int)((it.p1 - p0) < kKC ? (it.p1 - p0) : kKC);
          const uint32_t bytes = (uint32_t)(cp * B * (int)sizeof(In)) & ~15u;
          mbar_expect_tx(&sb->full[s], bytes);
          if (bytes) bulk_g2s(stages + s * stage_stride, cube + p0 * B, bytes, &sb->full[s]);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    // The whole warp runs this loop (uniform control flow keeps the
    // descriptors in uniform registers); lane 0 waits on the barriers and
    // broadcasts the outcome, one elected lane issues each MMA.
    const uint32_t ops_base = su32(ops);
    const uint64_t d0 = sdesc(ops_base);   // an offset of d bytes adds d >> 4
    const uint64_t d1s = sdesc_sw128(su32(ones));
    // band sums S1 = x^T 1: A = the tile's rows (MN-major), B = the ones (K-major), N = 16
    const uint32_t id_s1 = idesc_f16(16) | (1u << 15);
    Ring ro(kOpStages);  // operand-ring position, continued across items
    bool ok = true;
    for (int i = 0; i < nitems && ok; ++i) {
      const TcItem it = tc_item(one, T, items, cta_items, i);
      const int B = it.t.B;
      const int R16 = mma_rows(B);                  // bands (and the ones row), padded
      const bool s1mma = ones_band(B) < 0;          // S1 from the separate ones operand
      const bool two_tiles = B > 128;
      const int N0 = R16;                           // tile 0 columns: bands 0..R16-1
      const int N1 = two_tiles ? (R16 - 128) : 0;   // tile 1 columns: bands 128..R16-1
      const uint32_t id0 = idesc_mn(N0), id1 = idesc_mn(N1 > 0 ? N1 : 16);
      // the accumulators are free once the previous item's epilogue read them
      if (i > 0) {
        int w = 1;
        if (lane == 0) w = mbar_wait(&sb->tfree, (i - 1) & 1, &sb->abort) ? 1 : 0;
        if (!__shfl_sync(kFull, w, 0)) break;
      }
      tc_fence_after();
      bool first = true;
      const uint32_t t1 = tbase + (uint32_t)N0;
      constexpr uint64_t r128 = (uint64_t)(2 * kMnLBO) >> 4;   // tile 1: bands 128..
      for (int64_t p0 = it.p0; p0 < it.p1; p0 += kKC, ro.next()) {
        const int o = ro.idx;
        int w = 1;
        if (lane == 0) w = mbar_wait(&sb->opfull[o], ro.phase, &sb->abort) ? 1 : 0;
        if (!__shfl_sync(kFull, w, 0)) { ok = false; break; }
        tc_fence_after();
        // the converters' flags (written before their arrivals on opfull)
        int nz = 0;
#pragma unroll
        for (int cw = 0; cw < kConvWarps; ++cw) nz |= ((volatile int*)sb->lo_nz[o])[cw];
        const uint64_t hi = d0 + (uint64_t)(((uint32_t)(o * 2) * kOpBytes) >> 4);
        const uint64_t lo = hi + (uint64_t)(kOpBytes >> 4);
#pragma unroll
        for (int kk = 0; kk < kKC / 16; ++kk) {
          const uint64_t ko = (uint64_t)((kk * 2 * kMnSBO) >> 4);   // pixels 16 kk ..
          const uint32_t acc0 = (!first || kk > 0) ? 1u : 0u;
          // tile 0: rows 0..127 (A) x rows 0..N0-1 (B)
          mma_f16_warp(tbase, hi + ko, hi + ko, id0, acc0);
          if (nz) {
            mma_f16_warp(tbase, hi + ko, lo + ko, id0, 1u);
            mma_f16_warp(tbase, lo + ko, hi + ko, id0, 1u);
          }
          if (two_tiles) {
            mma_f16_warp(t1, hi + r128 + ko, hi + r128 + ko, id1, acc0);
            if (nz) {
              mma_f16_warp(t1, hi + r128 + ko, lo + r128 + ko, id1, 1u);
              mma_f16_warp(t1, lo + r128 + ko, hi + r128 + ko, id1, 1u);
            }
          }
          if (s1mma) {
            // band sums: (hi + lo)^T 1, column 0 of a 16-column accumulator per tile
            mma_f16_warp(tbase + kS1Col, hi + ko, d1s, id_s1, acc0);
            if (nz) mma_f16_warp(tbase + kS1Col, lo + ko, d1s, id_s1, 1u);
            if (two_tiles) {
              mma_f16_warp(tbase + kS1Col + 16, hi + r128 + ko, d1s, id_s1, acc0);
              if (nz) mma_f16_warp(tbase + kS1Col + 16, lo + r128 + ko, d1s, id_s1, 1u);
            }
          }
        }
        first = false;
        mma_commit_warp(&sb->opempty[o]);  // operand stage free once these MMAs finished
      }
      mma_commit_warp(&sb->done);          // this item's MMAs finished
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- converters
    const int ct = tid - 64;
    Ring rs(S), ro(kOpStages);        // ring / operand-ring positions, continued across items
    const void* probed = nullptr;     // the cube (and pixel count) whose shift and
    int64_t probed_n = -1;            // scale are in shs / sesc
    int mapB = -1;                    // the band count of the current unit layout
    int pr = 0, gq = 0;               // this thread's first pixel row and band group
    uint32_t uoff[kRowsPT] = {};      // its units' byte offsets in an operand
    uint32_t dirty = 0;               // bit kRowsPT o + u: lo unit u of operand stage o is non-zero
    for (int i = 0; i < nitems; ++i) {
      const TcItem it = tc_item(one, T, items, cta_items, i);
      const In* cube = static_cast<const In*>(it.t.cube);
      const int64_t N = it.t.N;
      const int B = it.t.B;
      conv_sync();  // the previous item's epilogue is over (every MMA of it finished)
      // Band probe (every CTA computes the same values from the same pixels):
      // over S = min(N, 32) pixels spread evenly through the cube, per band b
      //   shift_b = sample mean,  escale_b = 6 - E with max |y - shift_b| <= 2^E,
      // so that the sampled deviations scale into (2^5, 2^6] and a scaled value
      // leaves the FP16 range (65504) only if it lies about a thousand times
      // further from the shift than every sampled one.  A degenerate sample
      // falls back to |shift_b|, then to scale 1.  Consecutive items of one
      // cube (slots of one tile) reuse the values.
      if (it.t.cube != probed || N != probed_n) {
        probed = it.t.cube;
        probed_n = N;
        const int Sp = (int)(N < kProbe ? N : kProbe);
        const int b = ct % kRows, half = ct / kRows;     // kProbeHalves threads per band
        double sum = 0.0;
        float lo = INFINITY, hi = -INFINITY;
        if (b < B) {
          constexpr int kPer = kProbe / kProbeHalves;
          float y[kPer];
#pragma unroll
          for (int u = 0; u < kPer; ++u) {
            const int pi = half + kProbeHalves * u;
            y[u] = pi < Sp ? elem(cube + ((int64_t)pi * N / Sp) * B + b) : 0.f;
          }
#pragma unroll
          for (int u = 0; u < kPer; ++u) {
            if (half + kProbeHalves * u < Sp) {
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
            double tot = psum[b];
            lo = pmin[b];
            hi = pmax[b];
            if (kProbeHalves > 1) {
              tot += psum[kRows + b];
              lo = fminf(lo, pmin[kRows + b]);
              hi = fmaxf(hi, pmax[kRows + b]);
            }
            m = on_grid<In>((float)(tot / (double)Sp));
            double dev = fmax((double)hi - (double)m, (double)m - (double)lo);
            if (!isfinite(m) || !isfinite(dev)) { m = 0.f; dev = 0.0; }
            if (!(dev > 0.0)) dev = fabs((double)m);
            if (dev > 0.0) {
              int E;
              frexp(dev, &E);
              e = 6 - E;
              e = e < -120 ? -120 : (e > 120 ? 120 : e);
            }
            if (it.slot == 0) { it.t.shift[b] = m; it.t.escale[b] = e; }
          }
          shs[b] = m;
          sesc[b] = e;
        }
        conv_sync();
      }
      // Units: thread ct owns the 8-band group gq of pixel rows pr, pr + kRowStep,
      // ... of every chunk (kRowStep G8 <= kConvThreads; the others only take
      // part in the barriers), so the per-band constants of its bands stay in registers:
      // x = y 2^e - s 2^e in one FMA (y 2^e and s 2^e are exact); bands past B
      // get 0, 0.  Its values are written as one 16-byte row unit of the
      // MN-major operand with the 128-byte swizzle: 64-band blocks 4 KB apart,
      // 8-pixel groups 1 KB apart inside a block, unit gq mod 8 of pixel row p
      // at (gq ^ p) mod 8.
      const int G8 = (B + 7) >> 3;                  // 8-band groups
      if (B != mapB) {
        // A new unit layout: the lo units this thread left non-zero under the
        // old one are cleared first (every MMA of the previous item finished
        // before its epilogue, which the barrier above follows).
        for (int o = 0; o < kOpStages; ++o)
#pragma unroll
          for (int u = 0; u < kRowsPT; ++u)
            if (dirty & (1u << (kRowsPT * o + u)))
              *reinterpret_cast<uint4*>(ops + (size_t)(o * 2 + 1) * kOpBytes + uoff[u]) =
                  make_uint4(0, 0, 0, 0);
        dirty = 0;
        // the ones row of the new layout in the hi plane of every stage (and
        // the old one cleared): unit G8 of each of the 32 pixel rows
        const int ob_old = mapB > 0 ? ones_band(mapB) : -1, ob_new = ones_band(B);
        if (ct < kOpStages * kKC) {
          const int o = ct / kKC, k = ct - o * kKC;
          unsigned char* hp = ops + (size_t)(o * 2) * kOpBytes + (k >> 3) * kMnSBO + (k & 7) * 128;
          if (ob_old >= 0 && ob_old != ob_new) {
            const int gu = ob_old >> 3;
            *reinterpret_cast<uint4*>(hp + (gu >> 3) * kMnLBO + (((gu & 7) ^ (k & 7)) << 4)) =
                make_uint4(0, 0, 0, 0);
          }
          if (ob_new >= 0) {
            const int gu = ob_new >> 3;
            *reinterpret_cast<uint4*>(hp + (gu >> 3) * kMnLBO + (((gu & 7) ^ (k & 7)) << 4)) =
                make_uint4(0x3c00u, 0, 0, 0);   // FP16 1.0 at band ob, 0 at ob+1..ob+7
          }
        }
        mapB = B;
        pr = ct / G8;
        gq = ct - pr * G8;
#pragma unroll
        for (int u = 0; u < kRowsPT; ++u) {
          const int pp = pr < kRowStep ? pr + kRowStep * u : 0;
          uoff[u] = (uint32_t)(gq >> 3) * kMnLBO + (uint32_t)(pp >> 3) * kMnSBO + (pp & 7) * 128 +
                    ((uint32_t)((gq & 7) ^ (pp & 7)) << 4);
        }
      }
      const bool act = pr < kRowStep;
      const int b0 = 8 * gq;
      constexpr bool k16 = sizeof(In) == 2;
      constexpr bool kBf = std::is_same<In, __nv_bfloat16>::value;
      float sc[8], sh[8];
      uint32_t sc16[4];          // 16-bit cubes: the scales as packed pairs of the input type
      bool mixfma = k16;         // FP16 cubes: scales within FP16's normal range
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int b = b0 + e;
        sc[e] = (act && b < B) ? ldexpf(1.f, sesc[b]) : 0.f;
        sh[e] = (act && b < B) ? -shs[b] * sc[e] : 0.f;
        if (!kBf && act && b < B && (sesc[b] < -14 || sesc[b] > 15)) mixfma = false;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int e0 = sesc[b0 + 2 * e & 255], e1 = sesc[b0 + 2 * e + 1 & 255];
        const uint32_t p0 = sc[2 * e] == 0.f ? 0u : (kBf ? bf16_pow2(e0) : f16_pow2(e0));
        const uint32_t p1 = sc[2 * e + 1] == 0.f ? 0u : (kBf ? bf16_pow2(e1) : f16_pow2(e1));
        sc16[e] = p0 | (p1 << 16);
      }
      const bool vec = (B * (int)sizeof(In)) % 16 == 0 && b0 + 8 <= B;
      // a value beyond the FP16 range -> SIMT pass.  FP32 cubes track the
      // largest |x|; for 16-bit cubes (whose lo parts are nearly always zero)
      // an infinite lo part is the sign of it, checked where lo is stored
      float mx = 0.f;
      int rng = 0;
      const int cw = warp - 2;  // converter warp index
      for (int64_t p0 = it.p0; p0 < it.p1; p0 += kKC, rs.next(), ro.next()) {
        const int s = rs.idx, o = ro.idx;
        // one lane per warp polls the barriers (the others would only add
        // shared-memory traffic), then the warp proceeds together
        int ok = 1;
        if (lane == 0) {
          ok = mbar_wait(&sb->full[s], rs.phase, &sb->abort) ? 1 : 0;
          if (ok) ok = mbar_wait(&sb->opempty[o], ro.phase ^ 1u, &sb->abort) ? 1 : 0;
        }
        ok = __shfl_sync(kFull, ok, 0);
        if (!ok) break;
        const int cp = (int)((it.p1 - p0) < kKC ? (it.p1 - p0) : kKC);
        const int copied = (int)(((uint32_t)(cp * B * (int)sizeof(In)) & ~15u) / sizeof(In));
        const bool fast = vec && cp == kKC && copied == kKC * B;
        const In* st = reinterpret_cast<const In*>(stages + s * stage_stride);
        const In* gsrc = cube + p0 * B;
        unsigned char* hi = ops + (size_t)(o * 2) * kOpBytes;
        unsigned char* lo = hi + kOpBytes;
        uint32_t lo_bits = 0;    // OR of this thread's lo parts in this chunk
        // the units of this chunk; FM: the common case (a full chunk of a 16-bit
        // cube whose scales FP16 holds) compiled on its own, without the
        // per-unit tests of the other paths
        auto units = [&](auto FM_) {
          constexpr bool FM = decltype(FM_)::value;
#pragma unroll
          for (int u = 0; u < kRowsPT; ++u) {
            const int pp = pr + kRowStep * u;
            float x[8];
            if (FM || fast) {
              const In* src = st + pp * B + b0;
              if (FM || (k16 && mixfma)) {
                // the 16-bit pairs enter the FMA as they are
                const uint4 v = *reinterpret_cast<const uint4*>(src);
                if constexpr (kBf) {
                  fma_bf16x2_f32(v.x, sc16[0], sh[0], sh[1], x[0], x[1]);
                  fma_bf16x2_f32(v.y, sc16[1], sh[2], sh[3], x[2], x[3]);
                  fma_bf16x2_f32(v.z, sc16[2], sh[4], sh[5], x[4], x[5]);
                  fma_bf16x2_f32(v.w, sc16[3], sh[6], sh[7], x[6], x[7]);
                } else {
                  fma_f16x2_f32(v.x, sc16[0], sh[0], sh[1], x[0], x[1]);
                  fma_f16x2_f32(v.y, sc16[1], sh[2], sh[3], x[2], x[3]);
                  fma_f16x2_f32(v.z, sc16[2], sh[4], sh[5], x[4], x[5]);
                  fma_f16x2_f32(v.w, sc16[3], sh[6], sh[7], x[6], x[7]);
                }
              } else {
                float y[8];
                if constexpr (sizeof(In) == 4) {
                  const float4 a0 = *reinterpret_cast<const float4*>(src);
                  const float4 a1 = *reinterpret_cast<const float4*>(src + 4);
                  y[0] = a0.x; y[1] = a0.y; y[2] = a0.z; y[3] = a0.w;
                  y[4] = a1.x; y[5] = a1.y; y[6] = a1.z; y[7] = a1.w;
                } else {
                  const uint4 v = *reinterpret_cast<const uint4*>(src);
                  const In* h8 = reinterpret_cast<const In*>(&v);
#pragma unroll
                  for (int e = 0; e < 8; ++e) y[e] = to_f32<In>(h8[e]);
                }
#pragma unroll
                for (int e = 0; e < 8; ++e) x[e] = fmaf(y[e], sc[e], sh[e]);
              }
            } else {
              // partial chunk, a ragged pixel row or the last band group: pixels
              // past the chunk and bands past B contribute 0
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int el = pp * B + b0 + e;
                const bool v = pp < cp && b0 + e < B;
                const float y = v ? (el < copied ? elem(st + el) : elem(gsrc + el)) : 0.f;
                if constexpr (std::is_same<In, __nv_bfloat16>::value) {
                  const float c = v ? ldexpf(1.f, sesc[b0 + e]) : 0.f;   // as sc, sh
                  x[e] = v ? fmaf(y, c, -shs[b0 + e] * c) : 0.f;
                } else {
                  x[e] = v ? fmaf(y, sc[e], sh[e]) : 0.f;
                }
              }
            }
            uint32_t h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if constexpr (!k16) mx = fmaxf(mx, fmaxf(fabsf(x[2 * e]), fabsf(x[2 * e + 1])));
              h[e] = pack_f16x2(x[2 * e], x[2 * e + 1]);
              float r0, r1;
              if constexpr (k16) {
                resid_f16x2(h[e], x[2 * e], x[2 * e + 1], r0, r1);
              } else {
                unpack_f16x2(h[e], r0, r1);
                r0 = x[2 * e] - r0;
                r1 = x[2 * e + 1] - r1;
              }
              l[e] = pack_f16x2(r0, r1);
            }
            *reinterpret_cast<uint4*>(hi + uoff[u]) = make_uint4(h[0], h[1], h[2], h[3]);
            // the lo unit is stored when it is non-zero, or to clear what this
            // thread left there before; a unit that is and stays zero is skipped
            const uint32_t lu = (l[0] | l[1]) | (l[2] | l[3]);
            const uint32_t bit = 1u << (kRowsPT * o + u);
            if (lu != 0u || (dirty & bit)) {
              *reinterpret_cast<uint4*>(lo + uoff[u]) = make_uint4(l[0], l[1], l[2], l[3]);
              dirty = lu != 0u ? (dirty | bit) : (dirty & ~bit);
              if constexpr (k16)
                rng |= (f16x2_has_inf(l[0]) | f16x2_has_inf(l[1]) | f16x2_has_inf(l[2]) |
                        f16x2_has_inf(l[3])) ? 1 : 0;
            }
            lo_bits |= lu;
          }
        };
        if (act) {
          if (k16 && fast && mixfma) units(std::integral_constant<bool, true>{});
          else units(std::integral_constant<bool, false>{});
        }
        const int any_lo = __any_sync(kFull, lo_bits != 0u);
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
          sb->lo_nz[o][cw] = any_lo;   // published by the release of the arrival below
          mbar_arrive(&sb->opfull[o]);
          mbar_arrive(&sb->empty[s]);
        }
      }
      // the item's outputs, fetched again (not kept live through the chunk loop)
      const TcItem io = tc_item(one, T, items, cta_items, i);
      // NaN compares false (and gives a NaN lo part, not an infinite one): a
      // non-finite value is reported by the finalisation
      if (__any_sync(kFull, (!(mx <= 65504.f) && mx == mx) || rng != 0) && lane == 0)
        atomicOr(&io.t.hdr->cov_range, 1);
      // barrier, and a uniform decision to stop after an abandoned wait
      const bool aborted = conv_or(*(volatile int*)&sb->abort) != 0;
      // ---------------------------------------------------------- epilogue
      // All converter warps: warp w reads TMEM lane quarter w mod 4 (the
      // quarter it may access) and every fourth 16-column block, from block
      // (w - 2) / 4 on.
      {
        int okw = 0;
        if (lane == 0) okw = (!aborted && mbar_wait(&sb->done, i & 1, &sb->abort) && !*(volatile int*)&sb->abort) ? 1 : 0;
        const bool ok = __shfl_sync(kFull, okw, 0) != 0;
        const bool any = io.p1 > io.p0;   // an empty item leaves the accumulators unwritten
        tc_fence_after();
        const int R16 = mma_rows(B);
        const int N0 = R16, N1 = B > 128 ? R16 - 128 : 0;
        const int ob = ones_band(B);      // accumulator column of the band sums (-1: separate)
        const int q4 = warp & 3;          // TMEM lane quarter this warp may read
        const int part = cw >> 2;         // which blocks of the quarter (kConvWarps / 4 parts)
        const int r = q4 * 32 + lane;     // accumulator row
        const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
        float* out = io.t.s2_part + (size_t)io.slot * (B * (B + 1) / 2);
        const int nb0 = N0 >> 4, nb = nb0 + (N1 >> 4);
        for (int bk = part; bk < nb; bk += kConvWarps / 4) {
          const bool t1 = bk >= nb0;
          const int j0 = (t1 ? bk - nb0 : bk) << 4;       // column within the tile
          float v[16];
          if (ok && any) tmem_ld16(tbase + lane_off + (uint32_t)(t1 ? N0 + j0 : j0), v);
          else
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = 0.f;
          // tile 0: row r = band r, column j = band j; tile 1: bands 128 + r, 128 + j
          const int band = t1 ? 128 + r : r;
          const int jb0 = t1 ? 128 + j0 : j0;
          if (band < B && (t1 || r < 128)) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const int jb = jb0 + k;
              if (jb < B && jb >= band) out[packed_index(band, jb, B)] = v[k];
            }
          }
        }
        // band sums (FP64, unscaled): column ob of the tiles' accumulators, or
        // column 0 of the separate ones accumulators
        if (part == 0) {
          for (int t = 0; t < (B > 128 ? 2 : 1); ++t) {
            const uint32_t col = ob >= 0 ? (uint32_t)(t == 0 ? (ob & ~15) : N0 + ((ob - 128) & ~15))
                                         : kS1Col + 16u * (uint32_t)t;
            const int kk = ob >= 0 ? (ob & 15) : 0;   // the same for both tiles (128 = 0 mod 16)
            float v[16];
            if (ok && any) tmem_ld16(tbase + lane_off + col, v);
            else
#pragma unroll
              for (int k = 0; k < 16; ++k) v[k] = 0.f;
            float sv = v[0];
#pragma unroll
            for (int k = 1; k < 16; ++k) sv = k == kk ? v[k] : sv;
            const int band = 128 * t + r;
            if (band < B) io.t.s1_part[(size_t)io.slot * B + band] = ldexp((double)sv, -sesc[band]);
          }
        }
        if (!ok && lane == 0) set_status(io.t.hdr, PCA_ERR_TIMEOUT);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sb->tfree);
      }
      if (aborted) break;
    }
  }
  // teardown: every MMA of this CTA has finished before TMEM is released
  if (warp == 1 && lane == 0) {
    mma_commit(&sb->drain);
    const unsigned long long t0 = gtimer();
    while (!mbar_try(&sb->drain, 0) && gtimer() - t0 < kWaitNs) {
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// shared memory: operand ring, TMA ring of S stages, probe and sync blocks
size_t tc_fixed_smem() {
  return 1024 + (size_t)kOpStages * 2 * kOpBytes + kOnesBytes + kRows * (sizeof(float) + sizeof(int)) +
         kRows * (2 * sizeof(double) + 4 * sizeof(float)) + sizeof(SyncBlock);
}

template <typename In>
cudaError_t syrk_tc_launch(const TcTile& one, const TileDesc* T, const CovItem* items,
                           const int* cta_items, int ctas, int maxB, cudaStream_t st) {
  const int stage_stride = ((kKC * maxB * (int)sizeof(In)) + 127) & ~127;
  const size_t fixed = tc_fixed_smem();
  int S = (int)((227 * 1024 - fixed) / stage_stride);
  S = S > kMaxStages ? kMaxStages : S;
  if (S < 2) return cudaErrorInvalidValue;
  const size_t smem = fixed + (size_t)S * stage_stride;
  auto kern = k_syrk_tc<In>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<ctas, kThreads, smem, st>>>(one, T, items, cta_items, S, stage_stride);
  return cudaGetLastError();
}

template <typename In>
cudaError_t syrk_tc_typed(const void* cube, int64_t N, int B, float* shift, int* escale,
                          double* s1_part, float* s2_part, int partials, int ctas, DevHeader* hdr,
                          cudaStream_t st) {
  TcTile one{cube, N, B, partials, shift, escale, s1_part, s2_part, hdr};
  return syrk_tc_launch<In>(one, nullptr, nullptr, nullptr, ctas, B, st);
}

}  // namespace

bool syrk_tc_supported(int B) { return B >= 2 && B <= kMaxB; }

cudaError_t launch_syrk_tc(const void* cube, pca_dtype dt, int64_t N, int B, float* shift,
                           int* escale, double* s1_part, float* s2_part, int partials, int ctas,
                           DevHeader* hdr, cudaStream_t st) {
  if (ctas < 1 || ctas > partials) return cudaErrorInvalidValue;
  switch (dt) {
    case PCA_F32:
      return syrk_tc_typed<float>(cube, N, B, shift, escale, s1_part, s2_part, partials, ctas, hdr,
                                  st);
    case PCA_BF16:
      return syrk_tc_typed<__nv_bfloat16>(cube, N, B, shift, escale, s1_part, s2_part, partials,
                                          ctas, hdr, st);
    case PCA_F16:
      return syrk_tc_typed<__half>(cube, N, B, shift, escale, s1_part, s2_part, partials, ctas, hdr,
                                   st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_syrk_tc_grouped(const TileDesc* T, const CovItem* items, const int* cta_items,
                                   int ctas, int maxB, pca_dtype dt, cudaStream_t st) {
  if (ctas <= 0) return cudaSuccess;
  const TcTile none{};
  switch (dt) {
    case PCA_F32: return syrk_tc_launch<float>(none, T, items, cta_items, ctas, maxB, st);
    case PCA_BF16: return syrk_tc_launch<__nv_bfloat16>(none, T, items, cta_items, ctas, maxB, st);
    case PCA_F16: return syrk_tc_launch<__half>(none, T, items, cta_items, ctas, maxB, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbpca
