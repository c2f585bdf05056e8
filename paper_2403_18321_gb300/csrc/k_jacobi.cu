// k_jacobi.cu -- cyclic Jacobi eigen-solver of the covariance (Sec. 2,
// Eqs. 2-10), device resident, on one SM.
//
// The paper zeroes one element per host round trip (Sec. 4.2 stage 4) and
// notes that rotations on disjoint row/column pairs commute (Sec. 2, last
// paragraph).  Here every parallel step applies B'/2 disjoint rotations
// (B' = B rounded up to even, a zero padding index when B is odd) with the
// whole matrix A resident in shared memory (FP32, B' x B' row-major, only
// the upper triangle i <= j is ever read or written).
//
// Ordering: odd-even.  Even steps rotate the position pairs (0,1),(2,3),...,
// odd steps (1,2),(3,4),...; after each rotation the two positions swap, so
// the rotation actually applied is G = R Pi with R = [[c, s], [-s, c]] the
// Eq. 1/Eq. 6 rotation and Pi the 2x2 swap, G = [[s, c], [c, -s]].  With the
// swap every index pair meets exactly once in B' steps (a valid cyclic
// sweep), and the pairs are always adjacent positions: a step touches only
// 2x2 blocks in place, with no index tables.  A and V stay consistent
// because V receives the same G (V <- V G): at the end eigenvalue
// diag(A)[j] belongs to column j of V.
//
// Angles (Eqs. 2-5) are computed in FP32; V is not updated here: every
// (c, s) goes to a rotation log that k_vreplay applies to the rows of V
// on other SMs (rows of V evolve independently).
#include "common.cuh"

namespace gbpca {

namespace {

constexpr int kJacThreads = 1024;
constexpr int kBandWarps = 4;   // diagonal band: super-diagonal blocks, next angles, edges

__device__ __forceinline__ float rcp_nr(float x) {  // 1/x: hardware estimate + one Newton step
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return fmaf(r, fmaf(-x, r, 1.f), r);
}
__device__ __forceinline__ float rsqrt_nr(float x) {  // 1/sqrt(x), x > 0: estimate + Newton
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return fmaf(y, fmaf(-0.5f * x * y, y, 0.5f), y);
}
__device__ __forceinline__ float sqrt_est(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Eqs. 2-5 for the pair with diagonal app, aqq and off-diagonal apq: the small
// root t of Eq. 3 in the form t = sgn(tau)/(|tau| + sqrt(1 + tau^2)),
// tau = 1/m = (aqq - app)/(2 apq) (Eq. 7).  An off-diagonal below 2^-24 of
// sqrt(|app aqq|) cannot move either diagonal in FP32 and is set to zero
// without a rotation (c = 1, s = 0).
__device__ __forceinline__ void jacobi_angle(float app, float aqq, float apq, float& c, float& s,
                                             float& t) {
  const float thr = 5.9604645e-08f * sqrt_est(fabsf(app)) * sqrt_est(fabsf(aqq));
  if (!(fabsf(apq) > thr)) { c = 1.f; s = 0.f; t = 0.f; return; }
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
  c = rsqrt_nr(fmaf(tt, tt, 1.f));
  s = tt * c;
  t = tt;
}

// M' = G_I M G_J for the 2x2 block M = [[m00, m01], [m10, m11]], G = [[s, c], [c, -s]].
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

// Rotates the pair (p, q = p+1) whose off-diagonal value is apq (already in a
// register) and whose diagonals sit in A; finishes the diagonal block (rotate,
// then swap the two positions) and publishes (c, s).  Returns nothing; the
// caller stores 0 at (p, q).
__device__ __forceinline__ void pair_rotation(float* A, int Bp, int p, float apq, float2* cs_slot,
                                              float2* log_slot) {
  float* dp = A + p * Bp + p;
  float* dq = dp + Bp + 1;
  const float app = *dp, aqq = *dq;
  float c, s, t;
  jacobi_angle(app, aqq, apq, c, s, t);
  const float2 v = make_float2(c, s);
  *cs_slot = v;
  *log_slot = v;
  // R^T [[app, apq], [apq, aqq]] R = diag(app - t apq, aqq + t apq); then swap
  *dp = fmaf(t, apq, aqq);
  *dq = fmaf(-t, apq, app);
}

// Blocks (I, J) with J >= I + 2 of a step with np pairs, dealt to the bulk
// warps: row I holds np-2-I of them; row f is folded with row np-3-f so that
// every fold holds np-1 blocks; (fold, 32-lane chunk) work items go round-robin
// over the bulk warps.  Every lane packs its blocks once per launch into
// registers: word = I << 24 | J << 16 | shared-memory offset of (p_I, p_J).
constexpr int kBulkWarps = kJacThreads / 32 - kBandWarps;
constexpr int kMaxItems = 9;   // ceil(ceil((116-2)/2) * ceil(115/32) / 28) for B' = 232

__device__ __forceinline__ void build_items(int np, int e, int Bp, uint32_t* items) {
  const int lane = threadIdx.x & 31, bw = (threadIdx.x >> 5) - kBandWarps;
  const int rows = np - 2;
  const int nfold = rows > 0 ? (rows + 1) / 2 : 0;
  const int per = np - 1;
  const int nch = (per + 31) >> 5;
#pragma unroll
  for (int t = 0; t < kMaxItems; ++t) {
    items[t] = 0xffffffffu;
    const int wi = bw + t * kBulkWarps;
    if (rows <= 0 || wi >= nfold * nch) continue;
    const int f = wi / nch;
    const int x = ((wi - f * nch) << 5) + lane;
    const int first = np - 2 - f;
    const int limit = (2 * f + 1 == rows) ? first : per;
    if (x >= limit) continue;
    int I, J;
    if (x < first) { I = f; J = f + 2 + x; }
    else { I = np - 3 - f; J = I + 2 + (x - first); }
    const int off = (2 * I + e) * Bp + 2 * J + e;
    items[t] = ((uint32_t)I << 24) | ((uint32_t)J << 16) | (uint32_t)off;
  }
}

// One parallel step.  Even steps (e = 0) rotate position pairs (2J, 2J+1),
// odd steps (e = 1) the pairs (2J+1, 2J+2) with positions 0 and Bp-1 idle.
// The diagonal blocks of this step were finished (and cur[] filled) before it
// started.  Band warps update the super-diagonal blocks (I, I+1) and, unless
// this is the last step of the sweep, immediately rotate the diagonal block
// of the next step's pair that block completes, filling nxt[]; they also
// handle the idle row 0 / column Bp-1 of odd steps.  The bulk warps update
// every block (I, J) with J >= I + 2 from their packed item lists.
__device__ __forceinline__ void jacobi_step(float* A, int Bp, int P, int e, bool last,
                                            const float2* cur, float2* nxt, float2* log_next,
                                            const uint32_t* items) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const int np = P - e;
  if (warp < kBandWarps) {
    const int b = tid;
    if (b < np - 1) {  // super-diagonal block (I, I+1)
      const int I = b, pI = 2 * I + e;
      float* r0 = A + pI * Bp + pI + 2;
      float* r1 = r0 + Bp;
      float m00, m01, m10, m11;
      if (e == 0) {
        const float2 x = *reinterpret_cast<const float2*>(r0);
        const float2 y = *reinterpret_cast<const float2*>(r1);
        m00 = x.x; m01 = x.y; m10 = y.x; m11 = y.y;
      } else {
        m00 = r0[0]; m01 = r0[1]; m10 = r1[0]; m11 = r1[1];
      }
      rot_block(cur[I], cur[I + 1], m00, m01, m10, m11);
      if (!last) {  // (q_I, p_{I+1}) is the off-diagonal of the next step's pair
        const int J2 = e == 0 ? I : I + 1;
        pair_rotation(A, Bp, pI + 1, m10, nxt + J2, log_next + J2);
        m10 = 0.f;
      }
      if (e == 0) {
        *reinterpret_cast<float2*>(r0) = make_float2(m00, m01);
        *reinterpret_cast<float2*>(r1) = make_float2(m10, m11);
      } else {
        r0[0] = m00; r0[1] = m01; r1[0] = m10; r1[1] = m11;
      }
    }
    if (e) {  // idle row 0 against every pair, every pair against idle column Bp-1
      for (int w = b; w < 2 * np; w += kBandWarps * 32) {
        if (w < np) {
          const float2 g = cur[w];
          float* a = A + 2 * w + 1;  // (0, p), (0, q)
          const float x = a[0], y = a[1];
          float n0 = fmaf(x, g.y, y * g.x);
          const float n1 = fmaf(x, g.x, -y * g.y);
          if (w == 0 && !last) {  // (0, 1) is the off-diagonal of the next even pair 0
            pair_rotation(A, Bp, 0, n0, nxt, log_next);
            n0 = 0.f;
          }
          a[0] = n0;
          a[1] = n1;
        } else {
          const int I = w - np;
          const float2 g = cur[I];
          float* a = A + (2 * I + 1) * Bp + (Bp - 1);  // (p, L), (q, L)
          const float x = a[0], y = a[Bp];
          const float n0 = fmaf(g.y, x, g.x * y);
          float n1 = fmaf(g.x, x, -g.y * y);
          if (I == P - 2 && !last) {  // (Bp-2, Bp-1) is the next even pair P-1
            pair_rotation(A, Bp, Bp - 2, n1, nxt + (P - 1), log_next + (P - 1));
            n1 = 0.f;
          }
          a[0] = n0;
          a[Bp] = n1;
        }
      }
    }
  } else {
#pragma unroll
    for (int t = 0; t < kMaxItems; ++t) {
      const uint32_t w = items[t];
      if (w == 0xffffffffu) continue;
      const float2 csI = cur[w >> 24], csJ = cur[(w >> 16) & 0xff];
      float* r0 = A + (w & 0xffff);
      float* r1 = r0 + Bp;
      float m00, m01, m10, m11;
      if (e == 0) {
        const float2 u = *reinterpret_cast<const float2*>(r0);
        const float2 v = *reinterpret_cast<const float2*>(r1);
        m00 = u.x; m01 = u.y; m10 = v.x; m11 = v.y;
      } else {
        m00 = r0[0]; m01 = r0[1]; m10 = r1[0]; m11 = r1[1];
      }
      rot_block(csI, csJ, m00, m01, m10, m11);
      if (e == 0) {
        *reinterpret_cast<float2*>(r0) = make_float2(m00, m01);
        *reinterpret_cast<float2*>(r1) = make_float2(m10, m11);
      } else {
        r0[0] = m00; r0[1] = m01; r1[0] = m10; r1[1] = m11;
      }
    }
  }
}

__global__ void __launch_bounds__(kJacThreads, 1)
k_jacobi(const double* __restrict__ C, int B, float tol32, int sweeps_max, int relative_stop,
         float2* __restrict__ log, float* __restrict__ diag32, DevHeader* __restrict__ hdr) {
  extern __shared__ __align__(16) float A[];  // [Bp][Bp]
  __shared__ float2 cs[2][kMaxB / 2];
  __shared__ double red[2][32];
  __shared__ int s_flag;
  __shared__ int s_viol[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Bp = B + (B & 1), P = Bp / 2;

  if (hdr->nonfinite) {  // nothing sensible to diagonalise
    for (int i = tid; i < Bp; i += kJacThreads) diag32[i] = 0.f;
    if (tid == 0) { hdr->sweeps = 0; hdr->steps = 0; hdr->tol_used = tol32; }
    return;
  }
  for (int e = tid; e < Bp * Bp; e += kJacThreads) {
    const int i = e / Bp, j = e - i * Bp;
    A[e] = (i < B && j < B) ? (float)C[(size_t)i * B + j] : 0.f;
  }
  uint32_t items0[kMaxItems], items1[kMaxItems];
  {  // the packed lists must hold every block of both parities (true for B' <= 232)
    const int nw0 = ((P - 1) / 2) * ((P - 1 + 31) / 32);
    if (nw0 > kMaxItems * kBulkWarps) {
      if (tid == 0) { set_status(hdr, PCA_ERR_ARG); hdr->sweeps = 0; hdr->steps = 0; }
      return;
    }
  }
  if (warp >= kBandWarps) {
    build_items(P, 0, Bp, items0);
    build_items(P - 1, 1, Bp, items1);
  }
  __syncthreads();

  int sweep = 0, status = PCA_OK;
  for (;;) {
    // stop test (before every sweep).  relative_stop: element-wise, every
    // off-diagonal |a_pq| <= tol * sqrt(|a_pp a_qq|) -- the paper's "all
    // off-diagonal elements below the stop factor", scaled per pair so that
    // small eigenvalues converge to the same relative accuracy as large
    // ones; otherwise off(A) <= tol * ||A||_F (enough when an FP64
    // refinement follows).  off(A)/||A||_F is reported either way.
    float so = 0.f, sd = 0.f;
    int viol = 0;
    const float tol2 = tol32 * tol32;
    for (int i = warp; i < Bp; i += 32) {
      const float* Ai = A + i * Bp;
      const float aii = fabsf(Ai[i]);
      for (int j = i + lane; j < Bp; j += 32) {
        const float a = Ai[j];
        if (j == i) {
          sd = fmaf(a, a, sd);
        } else {
          so = fmaf(a, a, so);
          const float ajj = fabsf(A[j * Bp + j]);
          viol |= (a * a > tol2 * aii * ajj) ? 1 : 0;
        }
      }
    }
    so = warp_sum(so);
    sd = warp_sum(sd);
    viol = __any_sync(kFull, viol);
    if (lane == 0) { red[0][warp] = (double)so; red[1][warp] = (double)sd; s_viol[warp] = viol; }
    __syncthreads();
    if (warp == 0) {
      const double o = warp_sum(red[0][lane]), d = warp_sum(red[1][lane]);
      const int anyv = __any_sync(kFull, s_viol[lane]);
      if (lane == 0) {
        const double off = sqrt(2.0 * o), fro = sqrt(2.0 * o + d);
        int flag = 0;
        const bool conv = relative_stop ? !anyv : off <= (double)tol32 * fro;
        if (fro == 0.0 || conv) flag = 1;
        else if (sweep >= sweeps_max) flag = 2;
        s_flag = flag;
        hdr->off_rel = fro == 0.0 ? 0.0 : off / fro;
        hdr->fro = fro;
      }
    }
    __syncthreads();
    const int flag = s_flag;
    if (flag) { status = flag == 1 ? PCA_OK : PCA_ERR_NOCONV; break; }

    // the first step's pairs (even): rotate their diagonal blocks
    float2* logs = log + (size_t)sweep * Bp * P;
    if (tid < P) {
      float* ap = A + (2 * tid) * Bp + 2 * tid + 1;
      pair_rotation(A, Bp, 2 * tid, *ap, &cs[0][tid], logs + tid);
      *ap = 0.f;
    }
    __syncthreads();
    for (int step = 0; step < Bp; step += 2) {
      jacobi_step(A, Bp, P, 0, false, cs[0], cs[1], logs + (size_t)(step + 1) * P, items0);
      __syncthreads();
      jacobi_step(A, Bp, P, 1, step + 1 == Bp - 1, cs[1], cs[0], logs + (size_t)(step + 2) * P,
                  items1);
      __syncthreads();
    }
    ++sweep;
  }
  for (int i = tid; i < Bp; i += kJacThreads) diag32[i] = A[i * Bp + i];
  if (tid == 0) {
    hdr->sweeps = sweep;
    hdr->steps = sweep * Bp;
    hdr->tol_used = tol32;
    if (status != PCA_OK) set_status(hdr, status);
  }
}

// ------------------------------------------------------------------ V replay
// V <- V G_1 G_2 ... applied to the rows of V = I (B' x B'), one warp per row.
// Lane l holds the position pairs J = l + 32 g (g < NG) as registers (x, y).
// Even steps rotate (x, y) of each pair locally; odd steps rotate (y of pair
// J, x of pair J+1), the neighbour value arriving and returning by shuffles.
constexpr int kReplayWarps = 8;
constexpr int kReplayChunk = 16;  // steps staged in shared memory at a time

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

template <int NG>
__global__ void __launch_bounds__(kReplayWarps * 32)
k_vreplay(const float2* __restrict__ log, int B, const DevHeader* __restrict__ hdr,
          float* __restrict__ v32) {
  extern __shared__ __align__(16) float2 stage[];  // [2][kReplayChunk][P]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Bp = B + (B & 1), P = Bp / 2;
  const int row = blockIdx.x * kReplayWarps + warp;
  const int steps = hdr->steps;

  float x[NG], y[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const int J = lane + 32 * g;
    x[g] = (2 * J == row) ? 1.f : 0.f;
    y[g] = (2 * J + 1 == row) ? 1.f : 0.f;
  }
  const int nchunks = (steps + kReplayChunk - 1) / kReplayChunk;
  auto issue = [&](int ch) {
    const int s0 = ch * kReplayChunk;
    const int ns = min(kReplayChunk, steps - s0);
    float2* dst = stage + (size_t)(ch & 1) * kReplayChunk * P;
    const float2* src = log + (size_t)s0 * P;
    for (int i = tid; i < ns * P; i += kReplayWarps * 32) cp_async8(dst + i, src + i);
    cp_async_commit();
  };
  if (nchunks > 0) issue(0);
  for (int ch = 0; ch < nchunks; ++ch) {
    if (ch + 1 < nchunks) { issue(ch + 1); cp_async_wait1(); } else { cp_async_wait0(); }
    __syncthreads();
    const float2* buf = stage + (size_t)(ch & 1) * kReplayChunk * P;
    const int s0 = ch * kReplayChunk;
    const int ns = min(kReplayChunk, steps - s0);
    for (int si = 0; si < ns; ++si) {
      const int step = s0 + si;  // steps per sweep = Bp (even), so parity = step & 1
      const float2* g2 = buf + si * P;
      if ((step & 1) == 0) {
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          const int J = lane + 32 * g;
          if (J < P) {
            const float2 r = g2[J];
            const float nx = fmaf(x[g], r.y, y[g] * r.x);
            const float ny = fmaf(x[g], r.x, -y[g] * r.y);
            x[g] = nx; y[g] = ny;
          }
        }
      } else {
        float nxn[NG];
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          const float a = __shfl_down_sync(kFull, x[g], 1);
          const float b = __shfl_sync(kFull, x[g + 1 < NG ? g + 1 : g], 0);
          const float nx = lane < 31 ? a : b;
          const int J = lane + 32 * g;
          nxn[g] = nx;
          if (J < P - 1) {
            const float2 r = g2[J];
            const float yy = y[g];
            y[g] = fmaf(yy, r.y, nx * r.x);
            nxn[g] = fmaf(yy, r.x, -nx * r.y);
          }
        }
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          const float up = __shfl_up_sync(kFull, nxn[g], 1);
          const float w = __shfl_sync(kFull, nxn[g > 0 ? g - 1 : 0], 31);
          if (lane > 0) x[g] = up;
          else if (g > 0) x[g] = w;
        }
      }
    }
    __syncthreads();
  }
  if (row < Bp) {
    float* out = v32 + (size_t)row * Bp;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int J = lane + 32 * g;
      if (J < P) { out[2 * J] = x[g]; out[2 * J + 1] = y[g]; }
    }
  }
}

// lam[c], vc[i][c] for the real rows i < B and the real slots (padding slot dropped).
__global__ void k_compact(const float* __restrict__ diag32, const float* __restrict__ v32, int B,
                          DevHeader* __restrict__ hdr, double* __restrict__ lam,
                          float2* __restrict__ vc) {
  const int Bp = B + (B & 1);
  __shared__ int s_dummy;
  if (threadIdx.x == 0) s_dummy = -1;
  __syncthreads();
  if (B & 1) {
    const float* last = v32 + (size_t)(Bp - 1) * Bp;
    for (int j = threadIdx.x; j < Bp; j += blockDim.x)
      if (last[j] == 1.f) s_dummy = j;
  }
  __syncthreads();
  const int dmy = s_dummy;
  const int i = blockIdx.x;  // row of V
  for (int j = threadIdx.x; j < Bp; j += blockDim.x) {
    if (j == dmy) continue;
    const int c = (dmy >= 0 && j > dmy) ? j - 1 : j;
    if (c >= B) continue;
    vc[(size_t)i * B + c] = make_float2(v32[(size_t)i * Bp + j], 0.f);
    if (i == 0) lam[c] = (double)diag32[j];
  }
  if (i == 0 && threadIdx.x == 0) hdr->dummy_slot = dmy;
}

}  // namespace

cudaError_t launch_jacobi(const double* C, int B, float tol32, int sweeps_max, bool relative_stop,
                          float2* log, float* diag32, DevHeader* hdr, cudaStream_t st) {
  const int Bp = round_even(B);
  const size_t smem = (size_t)Bp * Bp * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_jacobi<<<1, kJacThreads, smem, st>>>(C, B, tol32, sweeps_max, relative_stop ? 1 : 0, log,
                                         diag32, hdr);
  return cudaGetLastError();
}

cudaError_t launch_vreplay(const float2* log, int B, const DevHeader* hdr, float* v32,
                           cudaStream_t st) {
  const int Bp = round_even(B), P = Bp / 2;
  const int NG = (P + 31) / 32;
  const int blocks = (Bp + kReplayWarps - 1) / kReplayWarps;
  const size_t smem = (size_t)2 * kReplayChunk * P * sizeof(float2);
  switch (NG) {
    case 1: k_vreplay<1><<<blocks, kReplayWarps * 32, smem, st>>>(log, B, hdr, v32); break;
    case 2: k_vreplay<2><<<blocks, kReplayWarps * 32, smem, st>>>(log, B, hdr, v32); break;
    case 3: k_vreplay<3><<<blocks, kReplayWarps * 32, smem, st>>>(log, B, hdr, v32); break;
    case 4: k_vreplay<4><<<blocks, kReplayWarps * 32, smem, st>>>(log, B, hdr, v32); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_compact(const float* diag32, const float* v32, int B, DevHeader* hdr,
                           double* lam, float2* vc, cudaStream_t st) {
  k_compact<<<B, 256, 0, st>>>(diag32, v32, B, hdr, lam, vc);
  return cudaGetLastError();
}

}  // namespace gbpca
