// k_jacobi_cluster.cu -- the cyclic Jacobi eigen-solver (Sec. 2, Eqs. 2-10)
// spread over one thread-block cluster.
//
// Same ordering and arithmetic as k_jacobi.cu (odd-even parallel ordering
// with a position swap after every rotation, G = [[s, c], [c, -s]], FP32,
// B'/2 disjoint rotations per step), but the B' x B' matrix is split by rows
// over nA "A" CTAs and the eigenvector matrix V by rows over nV "V" CTAs of
// the same cluster, so that every step costs each SM only a fraction of the
// shared-memory traffic, and V is rotated in lock-step instead of being
// replayed afterwards.
//
//   * A-CTA r owns the even row pairs [rp[r], rp[r+1]) -- rows
//     [2rp[r], 2rp[r+1]) -- plus one halo row 2rp[r+1] (the next CTA's first
//     row).  Even steps update its own rows; odd steps update the odd row
//     pairs [rp[r], rp[r+1]) -- rows [2rp[r]+1, 2rp[r+1]] -- whose last row
//     is the halo.  After every step the row that changed hands is copied to
//     its other holder through distributed shared memory.
//   * The diagonal lives in a replicated array dg[] in every CTA; whoever
//     rotates a diagonal block writes (c, s) and the two new diagonal values
//     into every CTA of the cluster.
//   * One cluster barrier per step (release/acquire) orders all of it.
// Control flow is identical in every CTA (the stop decision is made by CTA 0
// and broadcast), so every CTA reaches every cluster barrier.
#include <cooperative_groups.h>

#include <type_traits>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace gbpca {

namespace {

constexpr int kThreads = 1024;
constexpr int kBandWarps = 4;
constexpr int kBulkLanes = kThreads - kBandWarps * 32;
constexpr int kMaxItems = 4;      // bulk blocks per lane per parity (checked)
constexpr int kMaxVItems = 8;     // V pair-rotations per thread per parity (checked)
constexpr int kMaxCl = 8;

struct Params {
  const double* C;
  int B;
  float tol32;
  int sweeps_max;
  int relative_stop;
  int nA, nV;
  int rp[kMaxCl + 1];     // even row-pair boundaries of the A-CTAs, rp[nA] = P
  int vr[kMaxCl + 1];     // row boundaries of the V-CTAs, vr[nV] = B'
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
// dropped without rotating (c = 1, s = 0).
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
  float2 cs[2][kMaxB / 2];
  float dg[kMaxB];
  double part_o[kMaxCl], part_d[kMaxCl];
  int part_v[kMaxCl];
  double wred[2][32];
  int wviol[32];
  int flag;
  int ovf;
  double off_rel, fro;
};

// Rotates the diagonal block of pair (p, p+1) whose off-diagonal apq is in a
// register: new (c, s) into cs_next[J] and the rotated-and-swapped diagonal
// into dg[p], dg[p+1] of every CTA of the cluster.
__device__ __forceinline__ void pair_rotation(cg::cluster_group& cl, Shared* sh, int ncl, int p,
                                              float apq, int slot, int J) {
  const float app = sh->dg[p], aqq = sh->dg[p + 1];
  float c, s, t;
  jacobi_angle(app, aqq, apq, c, s, t);
  const float2 v = make_float2(c, s);
  const float np0 = fmaf(t, apq, aqq), np1 = fmaf(-t, apq, app);
  for (int r = 0; r < ncl; ++r) {
    Shared* o = cl.map_shared_rank(sh, r);
    o->cs[slot][J] = v;
    o->dg[p] = np0;
    o->dg[p + 1] = np1;
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_jacobi_cluster(const Params prm) {
  extern __shared__ __align__(16) float rows[];
  __shared__ Shared sh;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int B = prm.B, Bp = B + (B & 1), P = Bp / 2;
  const int ncl = prm.nA + prm.nV;
  const bool isA = rank < prm.nA;
  const double* C = prm.C;

  // ---- uniform early exit (every CTA reads the same header word)
  if (prm.hdr->nonfinite) {
    if (rank == 0) {
      for (int i = tid; i < Bp; i += kThreads) prm.diag32[i] = 0.f;
      if (tid == 0) { prm.hdr->sweeps = 0; prm.hdr->steps = 0; prm.hdr->tol_used = prm.tol32; }
    }
    if (!isA) {
      const int v = rank - prm.nA;
      for (int e = tid; e < (prm.vr[v + 1] - prm.vr[v]) * Bp; e += kThreads) {
        const int r = prm.vr[v] + e / Bp, c = e % Bp;
        prm.v32[(size_t)r * Bp + c] = (r == c) ? 1.f : 0.f;
      }
    }
    return;
  }

  // ---- this CTA's rows
  const int I_lo = isA ? prm.rp[rank] : 0, I_hi = isA ? prm.rp[rank + 1] : 0;
  const int R0 = 2 * I_lo;
  const int nrows = isA ? 2 * (I_hi - I_lo) + (I_hi < P ? 1 : 0) : 0;
  const int v = rank - prm.nA;
  const int V0 = isA ? 0 : prm.vr[v], V1 = isA ? 0 : prm.vr[v + 1];
  const int prev_lo = (isA && rank > 0) ? prm.rp[rank - 1] : 0;  // previous A-CTA's first pair

  for (int i = tid; i < Bp; i += kThreads) sh.dg[i] = i < B ? (float)C[(size_t)i * B + i] : 0.f;
  if (tid == 0) { sh.ovf = 0; sh.flag = 0; }
  if (isA) {
    for (int e = tid; e < nrows * Bp; e += kThreads) {
      const int i = R0 + e / Bp, j = e % Bp;
      rows[e] = (i < B && j < B) ? (float)C[(size_t)i * B + j] : 0.f;
    }
  } else {
    for (int e = tid; e < (V1 - V0) * Bp; e += kThreads) {
      const int i = V0 + e / Bp, j = e % Bp;
      rows[e] = (i == j) ? 1.f : 0.f;
    }
  }
  cl.sync();  // every CTA's flags are initialised before anyone writes them remotely

  // A-CTAs use lst[e][0..kMaxItems), V-CTAs lst[e][0..kMaxVItems)
  uint32_t lst[2][kMaxVItems];
  int overflow = 0;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int np = P - e;
#pragma unroll
    for (int t = 0; t < kMaxVItems; ++t) lst[e][t] = 0xffffffffu;
    if (isA && warp >= kBandWarps) {
      const int lid = tid - kBandWarps * 32;
      const int Ihi = min(I_hi, np - 2);  // rows that hold a block with J >= I + 2
      int total = 0;
      for (int I = I_lo; I < Ihi; ++I) total += np - 2 - I;
      if (total > kMaxItems * kBulkLanes) overflow = 1;
#pragma unroll
      for (int t = 0; t < kMaxItems; ++t) {
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
    if (!isA) {
      const int total = (V1 - V0) * np;
      if (total > kMaxVItems * kThreads) overflow = 1;
#pragma unroll
      for (int t = 0; t < kMaxVItems; ++t) {
        const int idx = tid + t * kThreads;
        if (idx < total) {
          const int lr = idx / np, J = idx - lr * np;
          const int off = lr * Bp + 2 * J + e;
          lst[e][t] = ((uint32_t)J << 16) | (uint32_t)off;
        }
      }
    }
  }
  // the capacities hold for every B <= 232 with the partitions the host builds;
  // a violation is made known to every CTA so that all of them stop together
  overflow = __syncthreads_or(overflow);
  if (overflow && tid == 0)
    for (int r = 0; r < ncl; ++r) atomicOr(&cl.map_shared_rank(&sh, r)->ovf, 1);
  cl.sync();
  const bool ovf = *(volatile int*)&sh.ovf != 0;
  if (ovf && rank == 0 && tid == 0) set_status(prm.hdr, PCA_ERR_ARG);

  int sweep = 0, status = PCA_OK;
  const float tol2 = prm.tol32 * prm.tol32;
  for (; !ovf;) {
    // ---------------- stop test over the A-CTAs' own rows, decided by CTA 0
    if (isA) {
      float so = 0.f, sd = 0.f;
      int viol = 0;
      for (int i = R0 + warp; i < 2 * I_hi; i += kThreads / 32) {
        const float* Ai = rows + (i - R0) * Bp;
        const float dii = sh.dg[i];
        if (lane == 0) sd = fmaf(dii, dii, sd);
        const float aii = fabsf(dii);
        for (int j = i + 1 + lane; j < Bp; j += 32) {
          const float a = Ai[j];
          so = fmaf(a, a, so);
          viol |= (a * a > tol2 * aii * fabsf(sh.dg[j])) ? 1 : 0;
        }
      }
      so = warp_sum(so);
      sd = warp_sum(sd);
      viol = __any_sync(kFull, viol);
      if (lane == 0) { sh.wred[0][warp] = (double)so; sh.wred[1][warp] = (double)sd; sh.wviol[warp] = viol; }
      __syncthreads();
      if (warp == 0) {
        const double o = warp_sum(sh.wred[0][lane]), d = warp_sum(sh.wred[1][lane]);
        const int anyv = __any_sync(kFull, sh.wviol[lane]);
        if (lane == 0) {
          Shared* s0 = cl.map_shared_rank(&sh, 0);
          s0->part_o[rank] = o;
          s0->part_d[rank] = d;
          s0->part_v[rank] = anyv;
        }
      }
    }
    cl.sync();
    if (rank == 0 && tid == 0) {
      double o = 0.0, d = 0.0;
      int anyv = 0;
      for (int r = 0; r < prm.nA; ++r) { o += sh.part_o[r]; d += sh.part_d[r]; anyv |= sh.part_v[r]; }
      const double off = sqrt(2.0 * o), fro = sqrt(2.0 * o + d);
      const bool conv = prm.relative_stop ? !anyv : off <= (double)prm.tol32 * fro;
      int flag = 0;
      if (fro == 0.0 || conv) flag = 1;
      else if (sweep >= prm.sweeps_max) flag = 2;
      for (int r = 0; r < ncl; ++r) cl.map_shared_rank(&sh, r)->flag = flag;
      sh.off_rel = fro == 0.0 ? 0.0 : off / fro;
      sh.fro = fro;
    }
    cl.sync();
    const int flag = sh.flag;
    if (flag) { status = flag == 1 ? PCA_OK : PCA_ERR_NOCONV; break; }

    // ---------------- the first (even) step's pairs: rotate their diagonal blocks
    if (isA && tid < I_hi - I_lo) {
      const int I = I_lo + tid, p = 2 * I;
      float* apq = rows + (p - R0) * Bp + p + 1;
      pair_rotation(cl, &sh, ncl, p, *apq, 0, I);
      *apq = 0.f;
    }
    cl.sync();

    auto step_body = [&](auto E_, bool last) {
      constexpr int e = decltype(E_)::value;
      const int np = P - e;
      const float2* cur = sh.cs[e];
      const int nslot = e ^ 1;
      if (isA) {
        if (warp < kBandWarps) {
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
            rot_block(cur[I], cur[I + 1], m00, m01, m10, m11);
            if (!last) {  // (q_I, p_{I+1}) is the off-diagonal of a next-step pair
              pair_rotation(cl, &sh, ncl, pI + 1, m10, nslot, e == 0 ? I : I + 1);
              m10 = 0.f;
            }
            if (e == 0) {
              *reinterpret_cast<float2*>(r0) = make_float2(m00, m01);
              *reinterpret_cast<float2*>(r1) = make_float2(m10, m11);
            } else {
              r0[0] = m00; r0[1] = m01; r1[0] = m10; r1[1] = m11;
            }
          }
          if (e) {
            // idle row 0 (CTA 0) against every pair; this CTA's odd pairs
            // against the idle column Bp-1
            const int nrow0 = rank == 0 ? np : 0;
            const int Ioe = min(I_hi, np);
            const int ncol = Ioe > I_lo ? Ioe - I_lo : 0;
            for (int w = tid; w < nrow0 + ncol; w += kBandWarps * 32) {
              if (w < nrow0) {
                const float2 g = cur[w];
                float* a = rows + 2 * w + 1;  // (0, p), (0, q)
                const float x = a[0], y = a[1];
                float n0 = fmaf(x, g.y, y * g.x);
                const float n1 = fmaf(x, g.x, -y * g.y);
                if (w == 0 && !last) {  // (0, 1): next even pair 0
                  pair_rotation(cl, &sh, ncl, 0, n0, nslot, 0);
                  n0 = 0.f;
                }
                a[0] = n0;
                a[1] = n1;
              } else {
                const int I = I_lo + (w - nrow0);
                const float2 g = cur[I];
                float* a = rows + (2 * I + 1 - R0) * Bp + (Bp - 1);  // (p, L), (q, L)
                const float x = a[0], y = a[Bp];
                const float n0 = fmaf(g.y, x, g.x * y);
                float n1 = fmaf(g.x, x, -g.y * y);
                if (I == P - 2 && !last) {  // (Bp-2, Bp-1): next even pair P-1
                  pair_rotation(cl, &sh, ncl, Bp - 2, n1, nslot, P - 1);
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
            const uint32_t w = lst[e][t];
            if (w == 0xffffffffu) continue;
            const float2 csI = cur[w >> 24], csJ = cur[(w >> 16) & 0xff];
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
            } else {
              r0[0] = m00; r0[1] = m01; r1[0] = m10; r1[1] = m11;
            }
          }
        }
      } else {
        // V rows: (v_p, v_q) <- (v_p, v_q) G for every pair of this step
#pragma unroll
        for (int t = 0; t < kMaxVItems; ++t) {
          const uint32_t w = lst[e][t];
          if (w == 0xffffffffu) continue;
          const float2 g = cur[w >> 16];
          float* a = rows + (w & 0xffff);
          float x, y;
          if (e == 0) {
            const float2 u = *reinterpret_cast<const float2*>(a);
            x = u.x; y = u.y;
          } else {
            x = a[0]; y = a[1];
          }
          const float nx = fmaf(x, g.y, y * g.x), ny = fmaf(x, g.x, -y * g.y);
          if (e == 0) *reinterpret_cast<float2*>(a) = make_float2(nx, ny);
          else { a[0] = nx; a[1] = ny; }
        }
      }
      __syncthreads();
      // hand over the row that changes holder: after an even step this CTA's
      // first row goes to the previous A-CTA's halo; after an odd step its halo
      // row goes back to the next A-CTA's first row
      if (isA) {
        if (e == 0 && rank > 0) {
          float* dst = cl.map_shared_rank(rows, rank - 1) + (size_t)(2 * (I_lo - prev_lo)) * Bp;
          for (int j = R0 + tid; j < Bp; j += kThreads) dst[j] = rows[j];
        } else if (e == 1 && rank + 1 < prm.nA) {
          const float* src = rows + (size_t)(2 * (I_hi - I_lo)) * Bp;
          float* dst = cl.map_shared_rank(rows, rank + 1);
          for (int j = 2 * I_hi + tid; j < Bp; j += kThreads) dst[j] = src[j];
        }
      }
      cl.sync();
    };
    for (int step = 0; step < Bp; step += 2) {
      step_body(std::integral_constant<int, 0>{}, false);
      step_body(std::integral_constant<int, 1>{}, step + 1 == Bp - 1);
    }
    ++sweep;
  }

  if (rank == 0) {
    for (int i = tid; i < Bp; i += kThreads) prm.diag32[i] = sh.dg[i];
    if (tid == 0) {
      prm.hdr->sweeps = sweep;
      prm.hdr->steps = sweep * Bp;
      prm.hdr->tol_used = prm.tol32;
      prm.hdr->off_rel = sh.off_rel;
      prm.hdr->fro = sh.fro;
      if (status != PCA_OK) set_status(prm.hdr, status);
    }
  }
  if (!isA) {
    for (int e = tid; e < (V1 - V0) * Bp; e += kThreads)
      prm.v32[(size_t)V0 * Bp + e] = rows[e];
  }
  cl.sync();  // no CTA leaves while others may still read its shared memory
}

}  // namespace

bool jacobi_cluster_shape(int B, int* nA, int* nV) {
  const int Bp = round_even(B);
  if (Bp <= 64) { *nA = 1; *nV = 1; }
  else if (Bp <= 128) { *nA = 2; *nV = 2; }
  else { *nA = 4; *nV = 4; }
  return true;
}

cudaError_t launch_jacobi_cluster(const double* C, int B, float tol32, int sweeps_max,
                                  bool relative_stop, float* diag32, float* v32, DevHeader* hdr,
                                  cudaStream_t st) {
  const int Bp = round_even(B), P = Bp / 2;
  Params prm{};
  prm.C = C;
  prm.B = B;
  prm.tol32 = tol32;
  prm.sweeps_max = sweeps_max;
  prm.relative_stop = relative_stop ? 1 : 0;
  jacobi_cluster_shape(B, &prm.nA, &prm.nV);
  if (prm.nA > P) prm.nA = P;
  // A rows: balance the blocks (I, J >= I) of the even steps
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
  for (int r = 0; r <= prm.nV; ++r) prm.vr[r] = (int)((long)Bp * r / prm.nV);
  prm.diag32 = diag32;
  prm.v32 = v32;
  prm.hdr = hdr;

  int maxrows = 0;
  for (int r = 0; r < prm.nA; ++r) {
    const int n = 2 * (prm.rp[r + 1] - prm.rp[r]) + (prm.rp[r + 1] < P ? 1 : 0);
    maxrows = n > maxrows ? n : maxrows;
  }
  for (int r = 0; r < prm.nV; ++r) {
    const int n = prm.vr[r + 1] - prm.vr[r];
    maxrows = n > maxrows ? n : maxrows;
  }
  const size_t smem = (size_t)maxrows * Bp * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_jacobi_cluster,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(prm.nA + prm.nV);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = prm.nA + prm.nV;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_jacobi_cluster, prm);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace gbpca
