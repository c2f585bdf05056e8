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

// Eqs. 2-5 for the pair with diagonal app, aqq and off-diagonal apq: the small
// root t of Eq. 3 in the form t = sgn(tau)/(|tau| + sqrt(1 + tau^2)),
// tau = 1/m = (aqq - app)/(2 apq) (Eq. 7).  An off-diagonal below 2^-24 of
// sqrt(|app aqq|) cannot move either diagonal in FP32 and is set to zero
// without a rotation (c = 1, s = 0).
__device__ __forceinline__ void jacobi_angle(float app, float aqq, float apq, float& c, float& s,
                                             float& t) {
  const float thr = 5.9604645e-08f * sqrtf(fabsf(app)) * sqrtf(fabsf(aqq));
  if (!(fabsf(apq) > thr)) { c = 1.f; s = 0.f; t = 0.f; return; }
  const float tau = (aqq - app) / (2.f * apq);
  const float at = fabsf(tau);
  float tt = (at > 1e18f) ? 0.5f / at : 1.f / (at + sqrtf(fmaf(tau, tau, 1.f)));
  tt = (tau >= 0.f) ? tt : -tt;
  c = 1.f / sqrtf(fmaf(tt, tt, 1.f));
  s = tt * c;
  t = tt;
}

// M' = G_I M G_J for the 2x2 block M = [[m00, m01], [m10, m11]].
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

__global__ void __launch_bounds__(kJacThreads, 1)
k_jacobi(const double* __restrict__ C, int B, float tol32, int sweeps_max,
         float2* __restrict__ log, float* __restrict__ diag32, DevHeader* __restrict__ hdr) {
  extern __shared__ __align__(16) float A[];  // [Bp][Bp]
  __shared__ float2 cs[kMaxB / 2];
  __shared__ double red[2][32];
  __shared__ int s_flag;
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
  __syncthreads();

  int sweep = 0, status = PCA_OK;
  for (;;) {
    // stop test (before every sweep): off(A) <= tol * ||A||_F
    float so = 0.f, sd = 0.f;
    for (int i = warp; i < Bp; i += 32) {
      const float* Ai = A + i * Bp;
      for (int j = i + lane; j < Bp; j += 32) {
        const float a = Ai[j];
        if (j == i) sd = fmaf(a, a, sd); else so = fmaf(a, a, so);
      }
    }
    so = warp_sum(so);
    sd = warp_sum(sd);
    if (lane == 0) { red[0][warp] = (double)so; red[1][warp] = (double)sd; }
    __syncthreads();
    if (warp == 0) {
      const double o = warp_sum(red[0][lane]), d = warp_sum(red[1][lane]);
      if (lane == 0) {
        const double off = sqrt(2.0 * o), fro = sqrt(2.0 * o + d);
        int flag = 0;
        if (fro == 0.0 || off <= (double)tol32 * fro) flag = 1;
        else if (sweep >= sweeps_max) flag = 2;
        s_flag = flag;
        hdr->off_rel = fro == 0.0 ? 0.0 : off / fro;
        hdr->fro = fro;
      }
    }
    __syncthreads();
    const int flag = s_flag;
    if (flag) { status = flag == 1 ? PCA_OK : PCA_ERR_NOCONV; break; }

    for (int step = 0; step < Bp; ++step) {
      const int e = step & 1;
      const int np = P - e;  // odd steps leave positions 0 and Bp-1 idle
      // phase A: angles of the np pairs; the diagonal block is finished here
      if (tid < np) {
        const int p = 2 * tid + e, q = p + 1;
        float* Ap = A + p * Bp;
        float* Aq = A + q * Bp;
        const float app = Ap[p], aqq = Aq[q], apq = Ap[q];
        float c, s, t;
        jacobi_angle(app, aqq, apq, c, s, t);
        const float2 v = make_float2(c, s);
        cs[tid] = v;
        log[((size_t)sweep * Bp + step) * P + tid] = v;
        // R^T [[app, apq], [apq, aqq]] R = diag(app - t apq, aqq + t apq); then swap
        Ap[p] = fmaf(t, apq, aqq);
        Aq[q] = fmaf(-t, apq, app);
        Ap[q] = 0.f;
      }
      __syncthreads();
      // phase B: off-diagonal blocks (I < J), folded so that every warp row
      // holds np blocks: row f with row np-2-f.
      const int R = np - 1;
      const int nfold = (R + 1) / 2;
      for (int f = warp; f < nfold; f += 32) {
        const int first = np - 1 - f;                       // blocks in row f
        const int limit = (2 * f + 1 == R) ? first : np;    // middle row when R is odd
        for (int x = lane; x < limit; x += 32) {
          int I, J;
          if (x < first) { I = f; J = f + 1 + x; }
          else { I = np - 2 - f; J = I + 1 + (x - first); }
          const int pI = 2 * I + e, pJ = 2 * J + e;
          float* r0 = A + pI * Bp + pJ;
          float* r1 = r0 + Bp;
          float m00, m01, m10, m11;
          if (e == 0) {
            const float2 a = *reinterpret_cast<const float2*>(r0);
            const float2 b = *reinterpret_cast<const float2*>(r1);
            m00 = a.x; m01 = a.y; m10 = b.x; m11 = b.y;
          } else {
            m00 = r0[0]; m01 = r0[1]; m10 = r1[0]; m11 = r1[1];
          }
          rot_block(cs[I], cs[J], m00, m01, m10, m11);
          if (e == 0) {
            *reinterpret_cast<float2*>(r0) = make_float2(m00, m01);
            *reinterpret_cast<float2*>(r1) = make_float2(m10, m11);
          } else {
            r0[0] = m00; r0[1] = m01; r1[0] = m10; r1[1] = m11;
          }
        }
      }
      if (e) {  // row 0 (idle position) against every pair, every pair against column Bp-1
        for (int w = tid; w < 2 * np; w += kJacThreads) {
          if (w < np) {
            const float2 g = cs[w];
            float* a = A + 2 * w + 1;  // (0, p), (0, q)
            const float x = a[0], y = a[1];
            a[0] = fmaf(x, g.y, y * g.x);
            a[1] = fmaf(x, g.x, -y * g.y);
          } else {
            const int I = w - np;
            const float2 g = cs[I];
            float* a = A + (2 * I + 1) * Bp + (Bp - 1);  // (p, L), (q, L)
            const float x = a[0], y = a[Bp];
            a[0] = fmaf(g.y, x, g.x * y);
            a[Bp] = fmaf(g.x, x, -g.y * y);
          }
        }
      }
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
                          double* __restrict__ vc) {
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
    vc[(size_t)i * B + c] = (double)v32[(size_t)i * Bp + j];
    if (i == 0) lam[c] = (double)diag32[j];
  }
  if (i == 0 && threadIdx.x == 0) hdr->dummy_slot = dmy;
}

}  // namespace

cudaError_t launch_jacobi(const double* C, int B, float tol32, int sweeps_max, float2* log,
                          float* diag32, DevHeader* hdr, cudaStream_t st) {
  const int Bp = round_even(B);
  const size_t smem = (size_t)Bp * Bp * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_jacobi<<<1, kJacThreads, smem, st>>>(C, B, tol32, sweeps_max, log, diag32, hdr);
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
                           double* lam, double* vc, cudaStream_t st) {
  k_compact<<<B, 256, 0, st>>>(diag32, v32, B, hdr, lam, vc);
  return cudaGetLastError();
}

}  // namespace gbpca
