// k_cov.cu -- band means and covariance (Algorithm 1 stages 2-3; Sec. 4.2
// stages 2 and 3) on SIMT cores, and the reduction of per-CTA partials.
//
// One pass over the cube.  Every partial slot g (a contiguous pixel range)
// accumulates, for x = y - s with s the first pixel of the cube (a per-band
// shift; any fixed s works),
//     S1_g = sum_n x_n            (FP64, per band)
//     S2_g = sum_n x_n x_n^T      (upper triangle, FP32 for P32 / FP64 for P64)
// and the finalisation turns the totals into the paper's quantities:
//     mu = s + S1/N,  C = (S2 - S1 S1^T / N) / (N - 1),
// which equals X^T X/(N-1) with X = Y - 1 mu^T exactly in real arithmetic.
// The shift keeps the summands centred near zero, so the correction term is
// of the order of one band variance (no catastrophic cancellation) and the
// cube is read once instead of twice (separate mean pass + covariance pass).
#include "common.cuh"

namespace gbpca {

namespace {

constexpr int kSyrkThreads = 256;
constexpr int kChunk = 32;  // pixels staged in shared memory per iteration

template <typename In>
__device__ __forceinline__ float ld(const In* p) { return to_f32<In>(*p); }

// One CTA: pixels [n0, n1) of the cube into partial slot g (S1 when grp is
// 0), band-tile group grp.  Each thread owns one TM x TM tile of the upper
// block-triangle of S2.
template <typename In, typename Acc, int TM>
__device__ __forceinline__ void syrk_simt_cta(const In* __restrict__ cube, int B, int64_t n0,
                                              int64_t n1, int g, int grp,
                                              float* __restrict__ shift_out,
                                              double* __restrict__ s1_part,
                                              Acc* __restrict__ s2_part,
                                              int* __restrict__ escale, unsigned char* smem_raw) {
  const int Bt = (B + TM - 1) / TM, ntiles = Bt * (Bt + 1) / 2;
  const int s2_elems = B * (B + 1) / 2;
  const int Bpad = Bt * TM;
  Acc* xs = reinterpret_cast<Acc*>(smem_raw);                   // [kChunk][Bpad]
  float* sh = reinterpret_cast<float*>(xs + kChunk * Bpad);     // [Bpad] shift
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int b = tid; b < Bpad; b += kSyrkThreads) sh[b] = b < B ? ld(cube + b) : 0.f;
  if (g == 0 && grp == 0)
    for (int b = tid; b < B; b += kSyrkThreads) {
      shift_out[b] = ld(cube + b);
      if (escale != nullptr) escale[b] = 0;
    }

  // tile of this thread: enumerate the upper block-triangle row by row
  const int t = grp * kSyrkThreads + tid;
  int ti = -1, tj = -1;
  if (t < ntiles) {
    int rem = t;
    for (int r = 0; r < Bt; ++r) {
      const int len = Bt - r;
      if (rem < len) { ti = r; tj = r + rem; break; }
      rem -= len;
    }
  }
  Acc acc[TM][TM];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc[i][j] = Acc(0);
  double s1 = 0.0;  // band `tid` (block-row 0 of the grid only)
  __syncthreads();

  for (int64_t c0 = n0; c0 < n1; c0 += kChunk) {
    const int cp = (int)((n1 - c0) < kChunk ? (n1 - c0) : kChunk);
    for (int p = warp; p < kChunk; p += kSyrkThreads / 32) {
      const In* row = cube + (c0 + p) * (int64_t)B;
      for (int b = lane; b < Bpad; b += 32)
        xs[p * Bpad + b] = (p < cp && b < B) ? Acc(ld(row + b)) - Acc(sh[b]) : Acc(0);
    }
    __syncthreads();
    if (grp == 0 && tid < B) {
      Acc cs = Acc(0);
      for (int p = 0; p < cp; ++p) cs += xs[p * Bpad + tid];
      s1 += (double)cs;
    }
    if (ti >= 0) {
      const Acc* xa = xs + ti * TM;
      const Acc* xb = xs + tj * TM;
      for (int p = 0; p < cp; ++p) {
        Acc a[TM], bv[TM];
#pragma unroll
        for (int i = 0; i < TM; ++i) { a[i] = xa[p * Bpad + i]; bv[i] = xb[p * Bpad + i]; }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TM; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
      }
    }
    __syncthreads();
  }

  if (grp == 0 && tid < B) s1_part[(size_t)g * B + tid] = s1;
  if (ti >= 0) {
    Acc* out = s2_part + (size_t)g * s2_elems;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int r = ti * TM + i;
#pragma unroll
      for (int j = 0; j < TM; ++j) {
        const int c = tj * TM + j;
        if (r < B && c < B && r <= c) out[packed_index(r, c, B)] = acc[i][j];
      }
    }
  }
}

// Grid: x walks the partial slots g (pixel ranges N g / parts ..), y = band-tile
// group.  The guarded form (the re-computation after an out-of-range
// tensor-core pass) runs on a small grid that returns at once when the flag is
// clear, instead of one CTA per slot.
template <typename In, typename Acc, int TM, bool kGuarded>
__global__ void __launch_bounds__(kSyrkThreads)
k_syrk_simt(const In* __restrict__ cube, int64_t N, int B, int parts, float* __restrict__ shift_out,
            double* __restrict__ s1_part, Acc* __restrict__ s2_part,
            const int* __restrict__ guard, int* __restrict__ escale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if constexpr (kGuarded) {
    if (*(volatile const int*)guard == 0) return;
    for (int g = blockIdx.x; g < parts; g += gridDim.x) {
      syrk_simt_cta<In, Acc, TM>(cube, B, N * g / parts, N * (g + 1) / parts, g, blockIdx.y,
                                 shift_out, s1_part, s2_part, escale, smem_raw);
      __syncthreads();   // the CTA's shared staging is reused by the next slot
    }
  } else {   // one slot per CTA
    const int g = blockIdx.x;
    syrk_simt_cta<In, Acc, TM>(cube, B, N * g / parts, N * (g + 1) / parts, g, blockIdx.y,
                               shift_out, s1_part, s2_part, nullptr, smem_raw);
  }
}

// Grid: x walks the items (item x, x + gridDim.x, ...), y = band-tile group
// (groups beyond an item's tile skip it).  The guarded form runs on a small
// grid whose CTAs first look at every tile's range flag together and return
// when none is set, so that the common case costs a few microseconds, not one
// CTA per item.
template <typename In, typename Acc, int TM, bool kGuarded>
__global__ void __launch_bounds__(kSyrkThreads)
k_syrk_simt_grouped(const TileDesc* __restrict__ T, const CovItem* __restrict__ items, int nitems,
                    int ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if constexpr (kGuarded) {
    int any = 0;
    for (int i = threadIdx.x; i < ntiles; i += kSyrkThreads)
      any |= *(volatile const int*)&T[i].hdr->cov_range;
    if (!__syncthreads_or(any)) return;
    for (int x = blockIdx.x; x < nitems; x += gridDim.x) {
      const CovItem it = items[x];
      const TileDesc& t = T[it.tile];
      const int B = t.B, Bt = (B + TM - 1) / TM;
      if ((int)blockIdx.y * kSyrkThreads >= Bt * (Bt + 1) / 2) continue;
      if (*(volatile const int*)&t.hdr->cov_range == 0) continue;
      syrk_simt_cta<In, Acc, TM>(static_cast<const In*>(t.cube), B, it.p0, it.p1, it.slot,
                                 blockIdx.y, t.shift, t.s1p, static_cast<Acc*>(t.s2p), t.escale,
                                 smem_raw);
      __syncthreads();   // the CTA's shared staging is reused by the next item
    }
  } else {   // one item per CTA
    const CovItem it = items[blockIdx.x];
    const TileDesc& t = T[it.tile];
    const int B = t.B, Bt = (B + TM - 1) / TM;
    if ((int)blockIdx.y * kSyrkThreads >= Bt * (Bt + 1) / 2) return;
    syrk_simt_cta<In, Acc, TM>(static_cast<const In*>(t.cube), B, it.p0, it.p1, it.slot,
                               blockIdx.y, t.shift, t.s1p, static_cast<Acc*>(t.s2p), nullptr,
                               smem_raw);
  }
}

template <typename In>
cudaError_t syrk_simt_typed(const In* cube, int64_t N, int B, bool fp64, float* shift,
                            double* s1_part, void* s2_part, int partials, cudaStream_t st,
                            const int* guard, int* escale) {
  const int gx = guard != nullptr ? std::min(partials, 4 * device_sms()) : partials;
  if (fp64) {
    constexpr int TM = 4;
    const int Bt = (B + TM - 1) / TM, ntiles = Bt * (Bt + 1) / 2;
    const int groups = (ntiles + kSyrkThreads - 1) / kSyrkThreads;
    const size_t smem = (size_t)kChunk * Bt * TM * sizeof(double) + Bt * TM * sizeof(float);
    auto kern = guard != nullptr ? k_syrk_simt<In, double, TM, true> : k_syrk_simt<In, double, TM, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<dim3(gx, groups), kSyrkThreads, smem, st>>>(cube, N, B, partials, shift, s1_part,
                                                       (double*)s2_part, guard, escale);
  } else {
    constexpr int TM = 8;
    const int Bt = (B + TM - 1) / TM, ntiles = Bt * (Bt + 1) / 2;
    const int groups = (ntiles + kSyrkThreads - 1) / kSyrkThreads;
    const size_t smem = (size_t)kChunk * Bt * TM * sizeof(float) + Bt * TM * sizeof(float);
    auto kern = guard != nullptr ? k_syrk_simt<In, float, TM, true> : k_syrk_simt<In, float, TM, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<dim3(gx, groups), kSyrkThreads, smem, st>>>(cube, N, B, partials, shift, s1_part,
                                                       (float*)s2_part, guard, escale);
  }
  return cudaGetLastError();
}

template <typename In>
cudaError_t syrk_simt_grouped_typed(const TileDesc* T, const CovItem* items, int nitems, int maxB,
                                    int ntiles, bool fp64, bool guarded, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  const int gx = guarded ? std::min(nitems, 4 * device_sms()) : nitems;
  if (fp64) {
    constexpr int TM = 4;
    const int Bt = (maxB + TM - 1) / TM, groups = (Bt * (Bt + 1) / 2 + kSyrkThreads - 1) / kSyrkThreads;
    const size_t smem = (size_t)kChunk * Bt * TM * sizeof(double) + Bt * TM * sizeof(float);
    auto kern = guarded ? k_syrk_simt_grouped<In, double, TM, true>
                        : k_syrk_simt_grouped<In, double, TM, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(gx, groups), kSyrkThreads, smem, st>>>(T, items, nitems, ntiles);
  } else {
    constexpr int TM = 8;
    const int Bt = (maxB + TM - 1) / TM, groups = (Bt * (Bt + 1) / 2 + kSyrkThreads - 1) / kSyrkThreads;
    const size_t smem = (size_t)kChunk * Bt * TM * sizeof(float) + Bt * TM * sizeof(float);
    auto kern = guarded ? k_syrk_simt_grouped<In, float, TM, true>
                        : k_syrk_simt_grouped<In, float, TM, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(gx, groups), kSyrkThreads, smem, st>>>(T, items, nitems, ntiles);
  }
  return cudaGetLastError();
}

// d[b] = (sum_g S1_g[b]) / N, one warp per band (FP64 adds spread over SMs).
__device__ __forceinline__ void s1_reduce_band(int b, const double* __restrict__ s1_part,
                                               int partials, int B, int64_t N,
                                               const float* __restrict__ shift,
                                               double* __restrict__ dvec, double* __restrict__ mu,
                                               float* __restrict__ mu_f,
                                               DevHeader* __restrict__ hdr) {
  const int lane = threadIdx.x;
  double s = 0.0;
  for (int g = lane; g < partials; g += 32) s += s1_part[(size_t)g * B + b];
  s = warp_sum(s);
  if (lane == 0) {
    const double d = s / (double)N;
    const double m = (double)shift[b] + d;
    dvec[b] = d;
    mu[b] = m;
    mu_f[b] = (float)m;
    if (!isfinite(m)) { atomicOr(&hdr->nonfinite, 1); set_status(hdr, PCA_ERR_NONFINITE); }
  }
}
__global__ void k_s1_reduce(const double* __restrict__ s1_part, int partials, int B, int64_t N,
                            const float* __restrict__ shift, double* __restrict__ dvec,
                            double* __restrict__ mu, float* __restrict__ mu_f,
                            DevHeader* __restrict__ hdr) {
  s1_reduce_band(blockIdx.x, s1_part, partials, B, N, shift, dvec, mu, mu_f, hdr);
}
__global__ void k_s1_reduce_batched(const TileDesc* __restrict__ T) {
  const TileDesc& t = T[blockIdx.y];
  if ((int)blockIdx.x >= t.B) return;
  s1_reduce_band(blockIdx.x, t.s1p, t.parts, t.B, t.N, t.shift, t.dvec, t.mu, t.muf, t.hdr);
}

// C_ij = (S2_ij - N d_i d_j) / (N - 1), S2 summed over the partials.  One
// CTA per 32 consecutive packed entries: lane = entry (coalesced reads of
// every partial), warp w adds the partials w, w + 8, ...  FP32 partials are
// added as an unevaluated FP32 pair (hi, lo) with error-free TwoSum steps --
// FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU --
// and the eight warp sums are added in FP64 in a fixed order.
constexpr int kFinWarps = 8;

template <typename Acc>
__device__ __forceinline__ void cov_finalize_block(int blk, const Acc* __restrict__ s2_part,
                                                   int partials, int s2_elems, int B, int64_t N,
                                                   const double* __restrict__ dvec,
                                                   double* __restrict__ C,
                                                   DevHeader* __restrict__ hdr,
                                                   const int* __restrict__ escale) {
  __shared__ double part[kFinWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blk * 32 + lane;
  double sum = 0.0;
  if (e < s2_elems) {
    if constexpr (sizeof(Acc) == 4) {
      float hi = 0.f, lo = 0.f;
      for (int g = warp; g < partials; g += kFinWarps) {
        const float v = (float)s2_part[(size_t)g * s2_elems + e];
        const float s = __fadd_rn(hi, v);          // TwoSum(hi, v)
        const float z = __fsub_rn(s, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, z)), __fsub_rn(v, z)));
        hi = s;
      }
      sum = (double)hi + (double)lo;
    } else {
      for (int g = warp; g < partials; g += kFinWarps) sum += (double)s2_part[(size_t)g * s2_elems + e];
    }
  }
  part[warp][lane] = sum;
  __syncthreads();
  if (warp == 0 && e < s2_elems) {
    double S2 = 0.0;
#pragma unroll
    for (int w = 0; w < kFinWarps; ++w) S2 += part[w][lane];
    // (i, j) of packed entry e = j(j+1)/2 + i
    int j = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    while ((int64_t)(j + 1) * (j + 2) / 2 <= e) ++j;
    while ((int64_t)j * (j + 1) / 2 > e) --j;
    const int i = (int)(e - (int64_t)j * (j + 1) / 2);
    if (escale != nullptr) S2 = ldexp(S2, -(escale[i] + escale[j]));  // exact power of two
    const double c = (S2 - (double)N * dvec[i] * dvec[j]) / (double)(N - 1);
    C[(size_t)i * B + j] = c;
    C[(size_t)j * B + i] = c;
    if (!isfinite(c)) { atomicOr(&hdr->nonfinite, 1); set_status(hdr, PCA_ERR_NONFINITE); }
  }
}
template <typename Acc>
__global__ void __launch_bounds__(kFinWarps * 32)
k_cov_finalize(const Acc* __restrict__ s2_part, int partials, int s2_elems, int B, int64_t N,
               const double* __restrict__ dvec, double* __restrict__ C,
               DevHeader* __restrict__ hdr, const int* __restrict__ escale) {
  cov_finalize_block<Acc>(blockIdx.x, s2_part, partials, s2_elems, B, N, dvec, C, hdr, escale);
}
template <typename Acc>
__global__ void __launch_bounds__(kFinWarps * 32)
k_cov_finalize_batched(const TileDesc* __restrict__ T, int escaled) {
  const TileDesc& t = T[blockIdx.y];
  const int s2_elems = t.B * (t.B + 1) / 2;
  if ((int)blockIdx.x * 32 >= s2_elems) return;
  cov_finalize_block<Acc>(blockIdx.x, static_cast<const Acc*>(t.s2p), t.parts, s2_elems, t.B, t.N,
                          t.dvec, t.C, t.hdr, escaled ? t.escale : nullptr);
}

}  // namespace

cudaError_t launch_syrk_simt(const void* cube, pca_dtype dt, int64_t N, int B, bool fp64,
                             float* shift, double* s1_part, void* s2_part, int partials,
                             cudaStream_t st, const int* guard, int* escale) {
  switch (dt) {
    case PCA_F32:
      return syrk_simt_typed((const float*)cube, N, B, fp64, shift, s1_part, s2_part, partials, st,
                             guard, escale);
    case PCA_BF16:
      return syrk_simt_typed((const __nv_bfloat16*)cube, N, B, fp64, shift, s1_part, s2_part,
                             partials, st, guard, escale);
    case PCA_F16:
      return syrk_simt_typed((const __half*)cube, N, B, fp64, shift, s1_part, s2_part, partials, st,
                             guard, escale);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_cov_finalize(const float* shift, const double* s1_part, const void* s2_part,
                                bool fp64_partials, int partials, int64_t N, int B, double* mu,
                                double* C, float* mu_f, double* dvec, DevHeader* hdr,
                                cudaStream_t st, const int* escale) {
  k_s1_reduce<<<B, 32, 0, st>>>(s1_part, partials, B, N, shift, dvec, mu, mu_f, hdr);
  const int s2_elems = B * (B + 1) / 2;
  const int grid = (s2_elems + 31) / 32;
  if (fp64_partials)
    k_cov_finalize<double><<<grid, kFinWarps * 32, 0, st>>>((const double*)s2_part, partials,
                                                            s2_elems, B, N, dvec, C, hdr, escale);
  else
    k_cov_finalize<float><<<grid, kFinWarps * 32, 0, st>>>((const float*)s2_part, partials,
                                                           s2_elems, B, N, dvec, C, hdr, escale);
  return cudaGetLastError();
}

cudaError_t launch_syrk_simt_grouped(const TileDesc* T, const CovItem* items, int nitems,
                                     int maxB, int ntiles, pca_dtype dt, bool fp64, bool guarded,
                                     cudaStream_t st) {
  switch (dt) {
    case PCA_F32:
      return syrk_simt_grouped_typed<float>(T, items, nitems, maxB, ntiles, fp64, guarded, st);
    case PCA_BF16:
      return syrk_simt_grouped_typed<__nv_bfloat16>(T, items, nitems, maxB, ntiles, fp64, guarded,
                                                    st);
    case PCA_F16:
      return syrk_simt_grouped_typed<__half>(T, items, nitems, maxB, ntiles, fp64, guarded, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_cov_finalize_batched(const TileDesc* T, int ntiles, int maxB, bool fp64,
                                        bool escaled, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  k_s1_reduce_batched<<<dim3(maxB, ntiles), 32, 0, st>>>(T);
  const dim3 grid((maxB * (maxB + 1) / 2 + 31) / 32, ntiles);
  if (fp64)
    k_cov_finalize_batched<double><<<grid, kFinWarps * 32, 0, st>>>(T, escaled ? 1 : 0);
  else
    k_cov_finalize_batched<float><<<grid, kFinWarps * 32, 0, st>>>(T, escaled ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace gbpca
