// k_jacobi_cluster.cu -- the cyclic Jacobi eigen-solver (Sec. 2, Eqs. 2-10)
// spread over one thread-block cluster.
//
// The paper zeroes one element per host round trip (Sec. 4.2 stage 4) and
// notes that rotations on disjoint row/column pairs commute (Sec. 2, last
// paragraph).  Here every parallel step applies B'/2 disjoint rotations
// (B' = B rounded up to even, a zero padding index when B is odd), FP32.
//
// Ordering: odd-even.  Even steps rotate the position pairs (0,1),(2,3),...,
// odd steps (1,2),(3,4),...; after each rotation the two positions swap, so
// the rotation actually applied is G = R Pi with R = [[c, s], [-s, c]] the
// Eq. 1/Eq. 6 rotation and Pi the 2x2 swap, G = [[s, c], [c, -s]].  With the
// swap every index pair meets exactly once in B' steps (a valid cyclic
// sweep), and the pairs are always adjacent positions: a step touches only
// 2x2 blocks in place, with no index tables.  V receives the same G
// (V <- V G), so at the end eigenvalue diag(A)[j] belongs to column j of V.
//
// The B' x B' matrix (upper triangle i <= j only) is split by rows over the
// nA CTAs of the cluster, and every CTA also holds a slice of the rows of
// the eigenvector matrix V in registers.
//
//   * CTA r owns the even row pairs [rp[r], rp[r+1]) -- rows
//     [2rp[r], 2rp[r+1]) -- in shared memory, plus one halo row 2rp[r+1]
//     (the next CTA's first row).  Even steps update its own rows; odd steps
//     update the odd row pairs [rp[r], rp[r+1]) -- rows [2rp[r]+1, 2rp[r+1]]
//     -- whose last row is the halo.  The threads that compute a row which
//     changes holder also write it straight into the other holder's copy
//     (distributed shared memory), so a step needs no CTA-local barrier.
//   * Whoever rotates the diagonal block of a pair of the next step writes
//     one record (c, s) + (new a_pp, new a_qq) into every CTA of the
//     cluster, as two 8-byte halves in separate arrays (the rotations read
//     only (c, s)).  Records rotate through four slots by global step number.
//   * V rows live in registers: lane l of a warp holds positions
//     [W l, W l + W) of a row.  Even-step pairs are lane-local; an odd-step
//     pair that straddles two lanes is completed by both lanes from one
//     shuffle each way.
//   * No cluster barrier inside a sweep.  Records and handed-over row
//     values travel as st.async stores that complete on the receiver's
//     mbarrier of the step they feed (one per record slot); each CTA's
//     mbarrier of step s+1 also takes one arrival per local warp (its
//     shared-memory writes of step s), with the byte count of the records
//     and row values it will receive.  A CTA starts step s+1 when that
//     phase completes, so no CTA runs more than one step ahead of another:
//     when a CTA pushes the records of step s+2, every CTA has at least
//     entered step s and reads slots s-1 and s only (four slots suffice),
//     and a handed-over row is written only after its holder sent its own
//     values of that row for the previous step (after its last read).
// Control flow is identical in every CTA (the stop decision is made by CTA 0
// and broadcast), so every CTA reaches every cluster barrier (three per
// sweep, at its start).  Every mbarrier wait is bounded; a CTA that gives up
// stops waiting and the sweep's stop test ends the solve with
// PCA_ERR_TIMEOUT.
#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace gbpca {

namespace {

constexpr int kThreads = 640;
constexpr int kBandWarps = 4;
constexpr int kBulkWarps = kThreads / 32 - kBandWarps;
constexpr int kBulkLanes = kBulkWarps * 32;
constexpr int kMaxItems = 4;      // bulk blocks per lane per parity (checked), default variant
constexpr int kVRows = 2;         // V rows per bulk warp (checked), default variant
constexpr int kWideVRows = 3;     // the same for the fewer-CTA variant
constexpr int kWideItems = 3;
constexpr int kMaxCl = 8;
constexpr int kSlots = 4;
constexpr int kRecs = 128;        // records per slot: 32 lanes x W/2 pairs, W <= 8
constexpr uint32_t kNone = 0xffffffffu;

struct Params {
  const double* C;
  int B;
  float tol32;
  int sweeps_max;
  int relative_stop;
  int nA;
  int rp[kMaxCl + 1];     // even row-pair boundaries of the CTAs, rp[nA] = P
  float* diag32;
  float* v32;
  DevHeader* hdr;
};

__device__ __forceinline__ float rcp_nr(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return fmaf(r, fmaf(-x, r, 1.f), r);
}
__device__ __forceinline__ float rsqrt_nr(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return fmaf(y, fmaf(-0.5f * x * y, y, 0.5f), y);
}
__device__ __forceinline__ float sqrt_est(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Eqs. 2-5: small root t of Eq. 3 as t = sgn(tau)/(|tau| + sqrt(1+tau^2)),
// tau = (aqq - app)/(2 apq); an off-diagonal below 2^-24 sqrt(|app aqq|) is
// dropped without rotating (c = 1, s = 0).  Returns the record of the pair:
// (c, s) and the two diagonal values after the rotation and position swap.
// With d = aqq - app and n = 2 apq the same root is
// t = sgn(tau) |n| / (|d| + sqrt(d^2 + n^2)) (sgn 0 = +1): three dependent
// reciprocal/root steps instead of four (the step's critical path runs
// through this record).  Where d^2 + n^2 could leave the FP32 range (|d| or
// |n| beyond 1e18, or both below 1e-18) the scale-free tau form is taken.
__device__ __forceinline__ float4 pair_record(float app, float aqq, float apq) {
  const float thr = 5.9604645e-08f * sqrt_est(fabsf(app)) * sqrt_est(fabsf(aqq));
  if (!(fabsf(apq) > thr)) return make_float4(1.f, 0.f, aqq, app);
  {
    const float d = aqq - app, n = 2.f * apq;
    const float ad = fabsf(d), an = fabsf(n);
    if (ad < 1e18f && an < 1e18f && (ad > 1e-18f || an > 1e-18f)) {
      const float q = fmaf(d, d, n * n);
      float tt = an * rcp_nr(ad + q * rsqrt_nr(q));
      tt = (d != 0.f && ((d < 0.f) != (n < 0.f))) ? -tt : tt;
      const float c = rsqrt_nr(fmaf(tt, tt, 1.f));
      return make_float4(c, tt * c, fmaf(tt, apq, aqq), fmaf(-tt, apq, app));
    }
  }
  const float tau = (aqq - app) * rcp_nr(2.f * apq);
  const float at = fabsf(tau);
  float tt;
  if (at > 1e18f) {
    tt = 0.5f * rcp_nr(at);
  } else {
    const float u = fmaf(tau, tau, 1.f);
    tt = rcp_nr(at + u * rsqrt_nr(u));
  }
  tt = (tau >= 0.f) ? tt : -tt;
  const float c = rsqrt_nr(fmaf(tt, tt, 1.f));
  return make_float4(c, tt * c, fmaf(tt, apq, aqq), fmaf(-tt, apq, app));
}

// M' = G_I M G_J, G = [[s, c], [c, -s]].
__device__ __forceinline__ void rot_block(float2 csI, float2 csJ, float& m00, float& m01,
                                          float& m10, float& m11) {
  const float cI = csI.x, sI = csI.y, cJ = csJ.x, sJ = csJ.y;
  const float t00 = fmaf(m00, sJ, m01 * cJ), t01 = fmaf(m00, cJ, -m01 * sJ);
  const float t10 = fmaf(m10, sJ, m11 * cJ), t11 = fmaf(m10, cJ, -m11 * sJ);
  m00 = fmaf(sI, t00, cI * t10);
  m01 = fmaf(sI, t01, cI * t11);
  m10 = fmaf(cI, t00, -sI * t10);
  m11 = fmaf(cI, t01, -sI * t11);
}

struct Shared {
  uint64_t mbar[kSlots];  // step s+1 completes on mbar[(s + 1) % kSlots]
  float2 cs[kSlots][kRecs];  // (c, s) of the pairs of a step
  float2 dd[kSlots][kRecs];  // the pairs' two diagonal values after the step
  float dg[kMaxB];        // diagonal at the sweep boundary
  double part_o[kMaxCl], part_d[kMaxCl];
  int part_v[kMaxCl];
  int part_a[kMaxCl];
  int abort;
  uint32_t halo_a, first_a;  // handed-over rows in the neighbours' windows
  uint32_t halo_bytes[2];    // row-value bytes received after even / odd steps
  double wred[2][32];
  int wviol[32];
  int flag;
  int ovf;
  double off_rel, fro;
  int escale;                // the matrix is held scaled by 2^-escale
};

// Record index of pair J = H q + t: row t of a 32-wide table, column q
// XOR t*32/H.  Lane l of a V warp reads its pairs l*H + t (t < H) as H
// loads of 32 distinct columns; 32 consecutive pairs (a bulk warp) fall on
// 32 distinct columns too, so both 8-byte access patterns are free of bank
// conflicts.
template <int H>
__device__ __forceinline__ int rix(int J) {
  const int t = J % H, q = J / H;
  return t * 32 + (q ^ (t * (32 / H)));
}

// Plain remote stores, ordered by the cluster barrier that follows (sweep start).
template <int H>
__device__ __forceinline__ void push_record(cg::cluster_group& cl, Shared* sh, int ncl, int slot,
                                            int J, float4 r) {
  const int i = rix<H>(J);
  for (int q = 0; q < ncl; ++q) {
    Shared* d = cl.map_shared_rank(sh, q);
    d->cs[slot][i] = make_float2(r.x, r.y);
    d->dd[slot][i] = make_float2(r.z, r.w);
  }
}

// Shared-memory address a (this CTA's window) in the window of CTA `rank`.
__device__ __forceinline__ uint32_t mapa(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// Stores into a CTA of the cluster that complete-tx their bytes on that
// CTA's mbarrier `bar` (both addresses in the receiver's window).
__device__ __forceinline__ void st_async(uint32_t a, float x, float y, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(a),
               "f"(x), "f"(y), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void st_async(uint32_t a, float x, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(a),
               "f"(x), "r"(bar)
               : "memory");
}
// A record of the next step into every CTA (slot and mbarrier of that step).
template <int H>
__device__ __forceinline__ void push_record_async(Shared* sh, int ncl, int slot, int J, float4 r) {
  const int i = rix<H>(J);
  const uint32_t a = su32(&sh->cs[slot][i]), b = su32(&sh->dd[slot][i]), bar = su32(&sh->mbar[slot]);
  for (int q = 0; q < ncl; ++q) {
    const uint32_t bq = mapa(bar, q);
    st_async(mapa(a, q), r.x, r.y, bq);
    st_async(mapa(b, q), r.z, r.w, bq);
  }
}
// The whole record of pair J in a slot: (c, s, new a_pp, new a_qq).
template <int H>
__device__ __forceinline__ float4 rec4(const Shared* sh, int slot, int J) {
  const int i = rix<H>(J);
  const float2 a = sh->cs[slot][i], b = sh->dd[slot][i];
  return make_float4(a.x, a.y, b.x, b.y);
}
// Phase wait with cluster-scope acquire (the st.async data of other CTAs).
__device__ __forceinline__ bool mbar_try_cluster(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
static __device__ __noinline__ void mbar_wait_cluster_slow(uint64_t* b, uint32_t parity, int* abort) {
  const unsigned long long t0 = gtimer();
  for (;;) {
    if (*(volatile int*)abort) return;
    if (mbar_try_cluster(b, parity)) return;
    if (gtimer() - t0 > kWaitNs) {
      atomicExch(abort, 1);
      return;
    }
  }
}
__device__ __forceinline__ void mbar_wait_cluster(uint64_t* b, uint32_t parity, int* abort) {
  if (!mbar_try_cluster(b, parity)) mbar_wait_cluster_slow(b, parity, abort);
}

// Diagonal position x after an odd step (records in slot so) preceded by an
// even step (slot se): positions 0 and B'-1 sat out the odd step.
template <int H>
__device__ __forceinline__ float diag_after_odd(const Shared* sh, int so, int se, int x, int Bp) {
  const int P = Bp / 2;
  if (x == 0) return sh->dd[se][rix<H>(0)].x;
  if (x == Bp - 1) return sh->dd[se][rix<H>(P - 1)].y;
  return (x & 1) ? sh->dd[so][rix<H>((x - 1) >> 1)].x : sh->dd[so][rix<H>((x - 2) >> 1)].y;
}

// The parameters of this CTA's matrix, read in place (parameter space or global
// memory) at each use rather than held in registers.
__device__ __forceinline__ const Params& par(const Params& one, const Params* list) {
  return list != nullptr ? list[blockIdx.x / one.nA] : one;
}

// One matrix per cluster: `one` when list is null, else list[cluster index]
// (every entry of a list has the cluster size one.nA).
template <int W, int VR, int MI>
__global__ void __launch_bounds__(kThreads, 1)
k_jacobi_cluster(const __grid_constant__ Params one, const Params* __restrict__ list) {
  constexpr int H = W / 2;                 // pairs per lane in a V row
  extern __shared__ __align__(16) float rows[];
  __shared__ Shared sh;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int B = par(one, list).B, Bp = B + (B & 1), P = Bp / 2;
  const int ncl = par(one, list).nA;
  const double* C = par(one, list).C;
  const bool band = warp < kBandWarps;
  const int bw = warp - kBandWarps;        // bulk warp index
  const int lid = tid - kBandWarps * 32;   // bulk lane index

  // ---- this CTA's rows and V rows
  // (the parameter array is read with constant indices: a dynamic index
  // would copy it to local memory)
  int I_lo = 0, I_hi = 0, prev_lo = 0;
#pragma unroll
  for (int r = 0; r < kMaxCl; ++r) {
    if (r == rank) { I_lo = par(one, list).rp[r]; I_hi = par(one, list).rp[r + 1]; }
    if (r + 1 == rank) prev_lo = par(one, list).rp[r];
  }
  const int R0 = 2 * I_lo;
  const int nrows = 2 * (I_hi - I_lo) + (I_hi < P ? 1 : 0);
  const int V0 = (int)((long)Bp * rank / ncl), V1 = (int)((long)Bp * (rank + 1) / ncl);
  // remote copies a handed-over row goes to: the previous CTA's halo row
  // (after even steps) and the next CTA's first row (after odd steps)
  // (kept in shared memory: they are used by few threads, and registers are full)
  const bool has_prev = rank > 0, has_next = rank + 1 < ncl;
  const int halo_row = 2 * (I_lo - prev_lo);  // in the previous CTA's rows

  // ---- uniform early exit (every CTA reads the same header word)
  if (par(one, list).hdr->nonfinite) {
    if (rank == 0) {
      for (int i = tid; i < Bp; i += kThreads) par(one, list).diag32[i] = 0.f;
      if (tid == 0) { par(one, list).hdr->sweeps = 0; par(one, list).hdr->steps = 0; par(one, list).hdr->tol_used = par(one, list).tol32; }
    }
    for (int e = tid; e < (V1 - V0) * Bp; e += kThreads) {
      const int r = V0 + e / Bp, c = e % Bp;
      par(one, list).v32[(size_t)r * Bp + c] = (r == c) ? 1.f : 0.f;
    }
    return;
  }

  // ---- the matrix is held scaled by 2^-E, with max_i |a_ii| in [2^(E-1), 2^E)
  //      (every CTA reads the whole diagonal and forms the same E): squares
  //      and products of entries then stay inside the FP32 range whatever the
  //      covariance's scale (|a_ij| <= max a_ii for a covariance); the
  //      eigenvalues and the norm are scaled back on output, the rotations
  //      and eigenvectors do not depend on it
  {
    double m = 0.0;
    for (int i = tid; i < B; i += kThreads) m = fmax(m, fabs(C[(size_t)i * B + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
    if (lane == 0) sh.wred[0][warp] = m;
    __syncthreads();
    if (tid == 0) {
      double cm = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) cm = fmax(cm, sh.wred[0][w]);
      int E = 0;
      if (cm > 0.0 && isfinite(cm)) frexp(cm, &E);
      sh.escale = E;
    }
    __syncthreads();
  }
  const int escale = sh.escale;
  const double dscale = ldexp(1.0, -escale);
  // ---- matrix rows, and records that reproduce the initial diagonal as the
  //      state after an odd step (slot 3) preceded by an even step (slot 2)
  for (int e = tid; e < nrows * Bp; e += kThreads) {
    const int i = R0 + e / Bp, j = e % Bp;
    rows[e] = (i < B && j < B) ? (float)(C[(size_t)i * B + j] * dscale) : 0.f;
  }
  auto d0 = [&](int i) { return i < B ? (float)(C[(size_t)i * B + i] * dscale) : 0.f; };
  for (int J = tid; J < P; J += kThreads) {
    sh.cs[2][rix<H>(J)] = sh.cs[3][rix<H>(J)] = make_float2(1.f, 0.f);
    sh.dd[2][rix<H>(J)] = make_float2(d0(2 * J), d0(2 * J + 1));
    sh.dd[3][rix<H>(J)] = make_float2(d0(2 * J + 1), J + 1 < P ? d0(2 * J + 2) : 0.f);
  }
  if (tid == 0) {
    sh.ovf = 0;
    sh.flag = 0;
    sh.abort = 0;
    sh.halo_a = has_prev ? mapa(su32(rows) + 4u * (uint32_t)(halo_row * Bp), rank - 1) : 0u;
    sh.first_a = has_next ? mapa(su32(rows), rank + 1) : 0u;
    // bytes of handed-over row values this CTA receives per step: after an
    // even step the next CTA's first row from column 2 I_hi + 2 on (its
    // blocks J = I_hi + 1 .. P - 1); after an odd step columns 2 I_lo + 1 ..
    // B' - 1 of this CTA's first row, from the previous CTA
    sh.halo_bytes[0] = has_next ? 8u * (uint32_t)max(0, P - 1 - I_hi) : 0u;
    sh.halo_bytes[1] = has_prev ? 4u * (uint32_t)(2 * max(0, P - 1 - I_lo) + 1) : 0u;
    for (int k = 0; k < kSlots; ++k) mbar_init(&sh.mbar[k], kThreads / 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  // ---- V rows in registers: bulk warp bw holds rows V0 + bw + kBulkWarps*k
  float v[VR][W];
  int vrow[VR];
#pragma unroll
  for (int k = 0; k < VR; ++k) {
    vrow[k] = band ? -1 : V0 + bw + kBulkWarps * k;
    if (vrow[k] >= V1) vrow[k] = -1;
#pragma unroll
    for (int c = 0; c < W; ++c) v[k][c] = (vrow[k] >= 0 && vrow[k] == W * lane + c) ? 1.f : 0.f;
  }

  // ---- bulk block lists (blocks (I, J >= I+2) of this CTA's row pairs)
  uint32_t lst[2][MI];
  uint32_t xitem = kNone;   // odd steps: one row-0 or last-column item
  int overflow = 0;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int np = P - e;
#pragma unroll
    for (int t = 0; t < MI; ++t) lst[e][t] = kNone;
    if (!band) {
      const int Ihi = min(I_hi, np - 2);  // rows that hold a block with J >= I + 2
      int total = 0;
      for (int I = I_lo; I < Ihi; ++I) total += np - 2 - I;
      if (total > MI * kBulkLanes) overflow = 1;
#pragma unroll
      for (int t = 0; t < MI; ++t) {
        const int idx = lid + t * kBulkLanes;
        if (idx < total) {
          int rem = idx, I = I_lo;
          while (rem >= np - 2 - I) { rem -= np - 2 - I; ++I; }
          const int J = I + 2 + rem;
          const int off = (2 * I + e - R0) * Bp + 2 * J + e;
          lst[e][t] = ((uint32_t)I << 24) | ((uint32_t)J << 16) | (uint32_t)off;
        }
      }
    }
  }
  if (!band) {
    // odd-step extras: row 0 against odd pairs 1..P-2 (CTA 0), and this CTA's
    // odd pairs against the idle last column (pair P-2 goes to a band thread)
    const int nrow0 = (rank == 0 && P > 2) ? P - 2 : 0;
    const int Ioe = min(I_hi, P - 1);
    const int ncol = Ioe > I_lo ? Ioe - I_lo : 0;
    if (nrow0 + ncol > kBulkLanes) overflow = 1;
    if (lid < nrow0) {
      xitem = (uint32_t)(lid + 1);
    } else if (lid < nrow0 + ncol) {
      const int I = I_lo + (lid - nrow0);
      if (I != P - 2) xitem = (1u << 31) | (uint32_t)I;
    }
  }
  if (V1 - V0 > VR * kBulkWarps || P > 32 * H) overflow = 1;
  overflow = __syncthreads_or(overflow);
  cl.sync();  // every CTA's flags and records are initialised before remote writes
  if (overflow && tid == 0)
    for (int r = 0; r < ncl; ++r) atomicOr(&cl.map_shared_rank(&sh, r)->ovf, 1);
  cl.sync();
  const bool ovf = *(volatile int*)&sh.ovf != 0;
  if (ovf && rank == 0 && tid == 0) set_status(par(one, list).hdr, PCA_ERR_ARG);

  int sweep = 0, status = PCA_OK;
  int gs = 0;                    // global step number; step gs uses record slot gs % 4
  const float tol2 = par(one, list).tol32 * par(one, list).tol32;
  for (; !ovf;) {
    // ---------------- diagonal at the sweep boundary (after the last odd step)
    {
      const int so = (gs + 3) % kSlots, se = (gs + 2) % kSlots;
      for (int x = tid; x < Bp; x += kThreads) sh.dg[x] = diag_after_odd<H>(&sh, so, se, x, Bp);
    }
    __syncthreads();
    // ---------------- stop test over this CTA's own rows, decided by CTA 0
    {
      float so2 = 0.f, sd = 0.f;
      int viol = 0;
      for (int i = R0 + warp; i < 2 * I_hi; i += kThreads / 32) {
        const float* Ai = rows + (i - R0) * Bp;
        const float dii = sh.dg[i];
        if (lane == 0) sd = fmaf(dii, dii, sd);
        const float aii = fabsf(dii);
        for (int j = i + 1 + lane; j < Bp; j += 32) {
          const float a = Ai[j];
          so2 = fmaf(a, a, so2);
          viol |= (a * a > tol2 * aii * fabsf(sh.dg[j])) ? 1 : 0;
        }
      }
      so2 = warp_sum(so2);
      sd = warp_sum(sd);
      viol = __any_sync(kFull, viol);
      if (lane == 0) {
        sh.wred[0][warp] = (double)so2;
        sh.wred[1][warp] = (double)sd;
        sh.wviol[warp] = viol;
      }
      __syncthreads();
      if (warp == 0) {
        constexpr int kWarps = kThreads / 32;
        const bool has = lane < kWarps;
        const double o = warp_sum(has ? sh.wred[0][lane] : 0.0);
        const double d = warp_sum(has ? sh.wred[1][lane] : 0.0);
        const int anyv = __any_sync(kFull, has && sh.wviol[lane]);
        if (lane == 0) {
          Shared* s0 = cl.map_shared_rank(&sh, 0);
          s0->part_o[rank] = o;
          s0->part_d[rank] = d;
          s0->part_v[rank] = anyv;
          s0->part_a[rank] = *(volatile int*)&sh.abort;
        }
      }
    }
    cl.sync();
    if (rank == 0 && tid == 0) {
      double o = 0.0, d = 0.0;
      int anyv = 0, anya = 0;
      for (int r = 0; r < ncl; ++r) {
        o += sh.part_o[r];
        d += sh.part_d[r];
        anyv |= sh.part_v[r];
        anya |= sh.part_a[r];
      }
      const double off = sqrt(2.0 * o), fro = sqrt(2.0 * o + d);
      const bool conv = par(one, list).relative_stop ? !anyv : off <= (double)par(one, list).tol32 * fro;
      int flag = 0;
      if (anya) flag = 3;
      else if (fro == 0.0 || conv) flag = 1;
      else if (sweep >= par(one, list).sweeps_max) flag = 2;
      for (int r = 0; r < ncl; ++r) cl.map_shared_rank(&sh, r)->flag = flag;
      sh.off_rel = fro == 0.0 ? 0.0 : off / fro;
      sh.fro = fro;
    }
    cl.sync();
    const int flag = sh.flag;
    if (flag) {
      status = flag == 1 ? PCA_OK : (flag == 2 ? PCA_ERR_NOCONV : PCA_ERR_TIMEOUT);
      break;
    }

    // ---------------- the first (even) step's pairs: rotate their diagonal blocks
    if (tid < I_hi - I_lo) {
      const int I = I_lo + tid, p = 2 * I;
      float* apq = rows + (p - R0) * Bp + p + 1;
      push_record<H>(cl, &sh, ncl, gs % kSlots, I, pair_record(sh.dg[p], sh.dg[p + 1], *apq));
      *apq = 0.f;
      if (I == I_lo && has_prev) cl.map_shared_rank(rows, rank - 1)[(size_t)halo_row * Bp + p + 1] = 0.f;
    }
    cl.sync();

    auto step_body = [&](auto E_, bool last) {
      constexpr int e = decltype(E_)::value;
      const int np = P - e;
      const int cur = gs % kSlots, nxt = (gs + 1) % kSlots, prv = (gs + 3) % kSlots;
      const uint32_t bar_nxt = su32(&sh.mbar[nxt]);
      // stores into the previous CTA's halo row / the next CTA's first row
      auto to_prev = [&](int col, float x, float y) {
        st_async(sh.halo_a + 4u * col, x, y, mapa(bar_nxt, rank - 1));
      };
      auto to_next = [&](int col, float x) { st_async(sh.first_a + 4u * col, x, mapa(bar_nxt, rank + 1)); };
      const float2* rc = sh.cs[cur];
      if (band) {
        // super-diagonal blocks (I, I+1) of this CTA's row pairs
        const int I = I_lo + tid;
        const int Iend = min(I_hi, np - 1);
        if (I < Iend) {
          const int pI = 2 * I + e;
          float* r0 = rows + (pI - R0) * Bp + pI + 2;
          float* r1 = r0 + Bp;
          float m00, m01, m10, m11;
          if (e == 0) {
            const float2 x = *reinterpret_cast<const float2*>(r0);
            const float2 y = *reinterpret_cast<const float2*>(r1);
            m00 = x.x; m01 = x.y; m10 = y.x; m11 = y.y;
          } else {
            m00 = r0[0]; m01 = r0[1]; m10 = r1[0]; m11 = r1[1];
          }
          const float4 gI = rec4<H>(&sh, cur, I), gJ = rec4<H>(&sh, cur, I + 1);
          rot_block(make_float2(gI.x, gI.y), make_float2(gJ.x, gJ.y), m00, m01, m10, m11);
          if (!last) {  // (q_I, p_{I+1}) is the off-diagonal of a next-step pair
            push_record_async<H>(&sh, ncl, nxt, e == 0 ? I : I + 1, pair_record(gI.w, gJ.z, m10));
            m10 = 0.f;
          }
          if (e == 0) {
            *reinterpret_cast<float2*>(r0) = make_float2(m00, m01);
            *reinterpret_cast<float2*>(r1) = make_float2(m10, m11);
            if (I == I_lo && has_prev) to_prev(pI + 2, m00, m01);
          } else {
            r0[0] = m00; r0[1] = m01; r1[0] = m10; r1[1] = m11;
            if (I == I_hi - 1 && has_next) {
              to_next(pI + 2, m10);
              to_next(pI + 3, m11);
            }
          }
        }
        if (e) {
          // odd-step items whose result is the off-diagonal of a next even
          // pair, each on a thread of its own: (0, 1) -> pair 0 (CTA 0) and
          // (B'-2, B'-1) -> pair P-1 (the CTA that holds odd pair P-2)
          if (tid == kBandWarps * 32 - 1 && rank == 0 && P >= 2) {
            const float4 g = rec4<H>(&sh, cur, 0);
            float* a = rows + 1;                     // (0, 1), (0, 2)
            const float x = a[0], y = a[1];
            float n0 = fmaf(x, g.y, y * g.x);
            const float n1 = fmaf(x, g.x, -y * g.y);
            if (!last) {
              push_record_async<H>(&sh, ncl, nxt, 0, pair_record(sh.dd[prv][rix<H>(0)].x, g.z, n0));
              n0 = 0.f;
            }
            a[0] = n0;
            a[1] = n1;
          }
          if (tid == kBandWarps * 32 - 2 && P >= 2 && I_lo <= P - 2 && P - 2 < I_hi) {
            const float4 g = rec4<H>(&sh, cur, P - 2);
            float* a = rows + (Bp - 3 - R0) * Bp + (Bp - 1);  // (B'-3, L), (B'-2, L)
            const float x = a[0], y = a[Bp];
            const float n0 = fmaf(g.y, x, g.x * y);
            float n1 = fmaf(g.x, x, -g.y * y);
            if (!last) {
              push_record_async<H>(&sh, ncl, nxt, P - 1,
                                   pair_record(g.w, sh.dd[prv][rix<H>(P - 1)].y, n1));
              n1 = 0.f;
            }
            a[0] = n0;
            a[Bp] = n1;
            if (P - 2 == I_hi - 1 && has_next) to_next(Bp - 1, n1);
          }
        }
      } else {
#pragma unroll
        for (int t = 0; t < MI; ++t) {
          const uint32_t w = lst[e][t];
          if (w == kNone) continue;
          const int I = (int)(w >> 24), J = (int)((w >> 16) & 0xff);
          const float2 csI = rc[rix<H>(I)], csJ = rc[rix<H>(J)];
          float* r0 = rows + (w & 0xffff);
          float* r1 = r0 + Bp;
          float m00, m01, m10, m11;
          if (e == 0) {
            const float2 u = *reinterpret_cast<const float2*>(r0);
            const float2 q = *reinterpret_cast<const float2*>(r1);
            m00 = u.x; m01 = u.y; m10 = q.x; m11 = q.y;
          } else {
            m00 = r0[0]; m01 = r0[1]; m10 = r1[0]; m11 = r1[1];
          }
          rot_block(csI, csJ, m00, m01, m10, m11);
          if (e == 0) {
            *reinterpret_cast<float2*>(r0) = make_float2(m00, m01);
            *reinterpret_cast<float2*>(r1) = make_float2(m10, m11);
            if (I == I_lo && has_prev) to_prev(2 * J, m00, m01);
          } else {
            r0[0] = m00; r0[1] = m01; r1[0] = m10; r1[1] = m11;
            if (I == I_hi - 1 && has_next) {
              to_next(2 * J + 1, m10);
              to_next(2 * J + 2, m11);
            }
          }
        }
        if (e && xitem != kNone) {
          if (!(xitem >> 31)) {        // (0, p), (0, q) against column pair w
            const int wp = (int)(xitem & 0xffff);
            const float2 g = rc[rix<H>(wp)];
            float* a = rows + 2 * wp + 1;
            const float x = a[0], y = a[1];
            a[0] = fmaf(x, g.y, y * g.x);
            a[1] = fmaf(x, g.x, -y * g.y);
          } else {                     // (p, L), (q, L) against row pair I
            const int I = (int)(xitem & 0xffff);
            const float2 g = rc[rix<H>(I)];
            float* a = rows + (2 * I + 1 - R0) * Bp + (Bp - 1);
            const float x = a[0], y = a[Bp];
            const float n1 = fmaf(g.x, x, -g.y * y);
            a[0] = fmaf(g.y, x, g.x * y);
            a[Bp] = n1;
            if (I == I_hi - 1 && has_next) to_next(Bp - 1, n1);
          }
        }
      }
      // this warp's shared-memory writes of the step are done: arrive on the
      // next step's mbarrier (warp 0 with the bytes this CTA will receive)
      __syncwarp();
      if (lane == 0) {
        if (warp == 0)
          mbar_expect_tx(&sh.mbar[nxt], (last ? 0u : 16u * (uint32_t)(P - 1 + e)) + sh.halo_bytes[e]);
        else
          mbar_arrive(&sh.mbar[nxt]);
      }
      // V rows: (v_p, v_q) <- (v_p, v_q) G for every pair of this step.  The
      // records of this slot are rewritten only three steps later.
      if (!band && vrow[0] >= 0) {
        const int J0 = H * lane;
        float2 g[H];
#pragma unroll
        for (int t = 0; t < H; ++t) g[t] = rc[rix<H>(H * lane + t)];
        if (e == 0) {
#pragma unroll
          for (int k = 0; k < VR; ++k) {
            if (vrow[k] < 0) continue;
#pragma unroll
            for (int t = 0; t < H; ++t) {
              if (J0 + t < P) {
                const float x = v[k][2 * t], y = v[k][2 * t + 1];
                v[k][2 * t] = fmaf(x, g[t].y, y * g[t].x);
                v[k][2 * t + 1] = fmaf(x, g[t].x, -y * g[t].y);
              }
            }
          }
        } else {
          // pair J0-1 straddles this lane and the previous one
          const float2 gp = lane > 0 ? rc[rix<H>(H * lane - 1)] : make_float2(1.f, 0.f);
#pragma unroll
          for (int k = 0; k < VR; ++k) {
            if (vrow[k] < 0) continue;        // uniform over the warp
            const float yn = __shfl_down_sync(kFull, v[k][0], 1);     // next lane's first
            const float xp = __shfl_up_sync(kFull, v[k][W - 1], 1);   // previous lane's last
            const float xl = v[k][W - 1], y0 = v[k][0];
#pragma unroll
            for (int t = 0; t < H - 1; ++t) {
              if (J0 + t < P - 1) {
                const float x = v[k][2 * t + 1], y = v[k][2 * t + 2];
                v[k][2 * t + 1] = fmaf(x, g[t].y, y * g[t].x);
                v[k][2 * t + 2] = fmaf(x, g[t].x, -y * g[t].y);
              }
            }
            if (J0 + H - 1 < P - 1) v[k][W - 1] = fmaf(xl, g[H - 1].y, yn * g[H - 1].x);
            if (lane > 0 && J0 - 1 < P - 1) v[k][0] = fmaf(xp, gp.x, -y0 * gp.y);
          }
        }
      }
      // steps gs = 4j + 3, 4j, 4j + 1, 4j + 2 complete phase j of slots 0..3
      mbar_wait_cluster(&sh.mbar[nxt], (uint32_t)(gs >> 2) & 1u, &sh.abort);
      ++gs;
    };
    for (int step = 0; step < Bp; step += 2) {
      step_body(std::integral_constant<int, 0>{}, false);
      step_body(std::integral_constant<int, 1>{}, step + 1 == Bp - 1);
    }
    ++sweep;
  }

  if (rank == 0) {
    const int so = (gs + 3) % kSlots, se = (gs + 2) % kSlots;
    for (int x = tid; x < Bp; x += kThreads)
      par(one, list).diag32[x] = ovf ? 0.f : ldexpf(diag_after_odd<H>(&sh, so, se, x, Bp), escale);
    if (tid == 0) {
      par(one, list).hdr->sweeps = sweep;
      par(one, list).hdr->steps = sweep * Bp;
      par(one, list).hdr->tol_used = par(one, list).tol32;
      par(one, list).hdr->off_rel = sh.off_rel;
      par(one, list).hdr->fro = ldexp(sh.fro, escale);
      if (status != PCA_OK) set_status(par(one, list).hdr, status);
    }
  }
#pragma unroll
  for (int k = 0; k < VR; ++k) {
    if (vrow[k] < 0) continue;
#pragma unroll
    for (int c = 0; c < W; ++c) {
      const int pos = W * lane + c;
      if (pos < Bp) par(one, list).v32[(size_t)vrow[k] * Bp + pos] = v[k][c];
    }
  }
  if (status == PCA_ERR_TIMEOUT) {
    // an abandoned wait may leave stores of other CTAs in flight: give them
    // time to land before any CTA of the cluster leaves
    const unsigned long long t0 = gtimer();
    while (gtimer() - t0 < 100000ull) {
    }
  }
  cl.sync();  // no CTA leaves while others may still write its shared memory
}

int v_width(int Bp) { return Bp <= 64 ? 2 : (Bp <= 128 ? 4 : 8); }

}  // namespace

bool jacobi_cluster_shape(int B, int* nA, int* nV) {
  const int Bp = round_even(B);
  *nA = Bp <= 32 ? 1 : (Bp <= 64 ? 2 : (Bp <= 128 ? 4 : 8));
  *nV = 0;
  return true;
}

namespace {

// Parameters of one matrix, and the dynamic shared memory its cluster needs.
size_t make_params(const double* C, int B, float tol32, int sweeps_max, bool relative_stop,
                   float* diag32, float* v32, DevHeader* hdr, int nA, Params* out) {
  const int Bp = round_even(B), P = Bp / 2;
  Params prm{};
  prm.C = C;
  prm.B = B;
  prm.tol32 = tol32;
  prm.sweeps_max = sweeps_max;
  prm.relative_stop = relative_stop ? 1 : 0;
  int nV = 0;
  jacobi_cluster_shape(B, &prm.nA, &nV);
  if (nA > 0) prm.nA = nA;
  if (prm.nA > P) prm.nA = P;
  // rows: balance the blocks (I, J >= I) of the even steps
  const long total = (long)P * (P + 1) / 2;
  prm.rp[0] = 0;
  long acc = 0;
  int I = 0;
  for (int r = 1; r < prm.nA; ++r) {
    const long target = total * r / prm.nA;
    while (I < P && acc + (P - I) <= target) { acc += P - I; ++I; }
    const int lo = prm.rp[r - 1] + 1, hi = P - (prm.nA - r);
    prm.rp[r] = I < lo ? lo : (I > hi ? hi : I);
    I = prm.rp[r];
    acc = 0;
    for (int i = 0; i < I; ++i) acc += P - i;
  }
  prm.rp[prm.nA] = P;
  prm.diag32 = diag32;
  prm.v32 = v32;
  prm.hdr = hdr;
  int maxrows = 0;
  for (int r = 0; r < prm.nA; ++r) {
    const int n = 2 * (prm.rp[r + 1] - prm.rp[r]) + (prm.rp[r + 1] < P ? 1 : 0);
    maxrows = n > maxrows ? n : maxrows;
  }
  *out = prm;
  return (size_t)maxrows * Bp * sizeof(float);
}

// Kernel variant: the default holds kVRows rows of V per bulk warp; clusters
// with fewer CTAs than that needs (the batched form's throughput shapes) hold
// kWideVRows rows and up to kWideItems bulk blocks per lane.
cudaError_t launch_clusters(int w, const Params& one, const Params* list, int count, size_t smem,
                            cudaStream_t st) {
  void (*kern)(const Params, const Params*);
  const bool wide = one.nA < jacobi_min_ctas(one.B);
  switch (w) {
    case 2: kern = wide ? k_jacobi_cluster<2, kWideVRows, kWideItems> : k_jacobi_cluster<2, kVRows, kMaxItems>; break;
    case 4: kern = wide ? k_jacobi_cluster<4, kWideVRows, kWideItems> : k_jacobi_cluster<4, kVRows, kMaxItems>; break;
    default: kern = wide ? k_jacobi_cluster<8, kWideVRows, kWideItems> : k_jacobi_cluster<8, kVRows, kMaxItems>; break;
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(one.nA * count);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = one.nA;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, one, list);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_jacobi_cluster(const double* C, int B, float tol32, int sweeps_max,
                                  bool relative_stop, float* diag32, float* v32, DevHeader* hdr,
                                  cudaStream_t st) {
  Params prm;
  const size_t smem =
      make_params(C, B, tol32, sweeps_max, relative_stop, diag32, v32, hdr, 0, &prm);
  return launch_clusters(v_width(round_even(B)), prm, nullptr, 1, smem, st);
}

int jacobi_width(int B) { return v_width(round_even(B)); }

// Fewest CTAs whose kernel variant holds the matrix: every CTA's rows of V
// and bulk blocks of both parities within the variant's capacity (the same
// counts the kernel checks).
int jacobi_batch_ctas(int B) { return jacobi_ctas_at_least(B, 1); }

int jacobi_ctas_at_least(int B, int n0) {
  const int Bp = round_even(B), P = Bp / 2;
  for (int n = n0 < 1 ? 1 : n0; n <= kMaxCl; ++n) {
    Params prm;
    make_params(nullptr, B, 1.f, 1, true, nullptr, nullptr, nullptr, n, &prm);
    const bool wide = prm.nA < jacobi_min_ctas(B);
    const int vr = wide ? kWideVRows : kVRows, mi = wide ? kWideItems : kMaxItems;
    bool fits = P <= 32 * (v_width(Bp) / 2);
    for (int r = 0; r < prm.nA && fits; ++r) {
      const int V0 = (int)((long)Bp * r / prm.nA), V1 = (int)((long)Bp * (r + 1) / prm.nA);
      if (V1 - V0 > vr * kBulkWarps) fits = false;
      for (int e = 0; e < 2 && fits; ++e) {
        const int np = P - e, hi = std::min(prm.rp[r + 1], np - 2);
        long total = 0;
        for (int I = prm.rp[r]; I < hi; ++I) total += np - 2 - I;
        if (total > (long)mi * kBulkLanes) fits = false;
      }
    }
    if (fits) return prm.nA;
  }
  return jacobi_min_ctas(B);
}

// Fewest CTAs that hold the rows of V in registers: kVRows rows per bulk warp.
int jacobi_min_ctas(int B) {
  const int Bp = round_even(B), per = kVRows * kBulkWarps;
  const int n = (Bp + per - 1) / per;
  return n < 1 ? 1 : (n > kMaxCl ? kMaxCl : n);
}

size_t jacobi_params_bytes() { return sizeof(Params); }

size_t jacobi_fill_params(void* dst, const double* C, int B, float tol32, int sweeps_max,
                          bool relative_stop, float* diag32, float* v32, DevHeader* hdr, int nA) {
  return make_params(C, B, tol32, sweeps_max, relative_stop, diag32, v32, hdr, nA,
                     static_cast<Params*>(dst));
}

int jacobi_params_ctas(const void* params) { return static_cast<const Params*>(params)->nA; }

cudaError_t launch_jacobi_cluster_list(const void* host_first, const void* dev_list, int count,
                                       size_t smem, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const Params& one = *static_cast<const Params*>(host_first);
  return launch_clusters(v_width(round_even(one.B)), one, static_cast<const Params*>(dev_list),
                         count, smem, st);
}

}  // namespace gbpca
