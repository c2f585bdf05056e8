/*
 * pca_oracle.c -- plain, slow, FP64 CPU reference of the Jacobi-PCA hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA library: every step below is written out from the paper's
 * statement of the method (Jacobi-based PCA for hyperspectral dimensionality
 * reduction, arXiv 2403.18321) in the paper's order and notation.
 *
 * Notation: Y is the N x B cube, pixel-major (band-interleaved-by-pixel),
 * Y[n*B + b].  X = Y - 1 mu^T.  C = X^T X / (N-1).  C = V diag(lambda) V^T,
 * column j of V (V[i*B + j]) is eigenvector j.  Q = X V[:, :k].
 *
 * Readings of points the paper leaves open (each one is also listed in the
 * design notes of the repository):
 *   - rotation angle: the small root of Eq. 3 written in its cancellation-free
 *     form t = sgn(tau)/(|tau| + sqrt(1+tau^2)), tau = 1/m = (a_qq-a_pp)/(2a_pq),
 *     sgn(0) = +1; a_pq == 0 skips the rotation (c = 1, s = 0).
 *   - stop rule: off(A) <= tol * ||A||_F, tested before every sweep, with
 *     off(A) the Frobenius norm of the off-diagonal part.
 *   - sort: eigenvalues descending, equal values keep the lower original index.
 *   - sign: every eigenvector is flipped so that its entry of largest
 *     magnitude (lowest row on ties) is positive.
 *   - projection: of the centred cube X (the GPU code of Sec. 4.2 projects the
 *     image after the in-place mean subtraction).
 *
 * Parity of every function here is pinned by the CPU tests (closed forms,
 * invariants, planted spectra, LAPACK on the oracle's own covariance, brute
 * force on tiny inputs); none is "parity unpinned".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_NOCONV 2
#define ORC_ERR_NONFINITE 3

/* Number of OpenMP threads the pixel loops may use (1 = serial). */
static int g_threads = 1;

int oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t < 1) t = omp_get_max_threads();
  g_threads = t;
#else
  (void)t;
  g_threads = 1;
#endif
  return g_threads;
}

/*
 * Stage 1 of Algorithm 1 ("band average removal"), first half: the average
 * of every band over all N pixels (Sec. 4.2 stage 2.1 computes it as
 * (1/N) Y^T 1).  Two passes: a plain sum, then a correction pass that adds
 * the mean of the residuals, so the result is the FP64 mean to a few ulps.
 * Returns ORC_ERR_NONFINITE if any input value is NaN or infinite.
 */
int oracle_band_means(const double *Y, long N, int B, double *mu) {
  if (N < 1 || B < 1) return ORC_ERR_ARG;
  for (int b = 0; b < B; ++b) {
    double s = 0.0;
    for (long n = 0; n < N; ++n) {
      double y = Y[n * B + b];
      if (!isfinite(y)) return ORC_ERR_NONFINITE;
      s += y;
    }
    double m = s / (double)N;
    double r = 0.0;
    for (long n = 0; n < N; ++n) r += Y[n * B + b] - m;
    mu[b] = m + r / (double)N;
  }
  return ORC_OK;
}

/*
 * Stage 2 of Algorithm 1: C = X^T X with X = Y - 1 mu^T, then divided by
 * N-1 as the GPU code of Sec. 4.2 (stage 3) does.  Triple loop in FP64:
 * for every pixel n, for every band pair (i, j) with i <= j, add
 * x_ni * x_nj; the lower triangle is the mirror of the upper one.
 * With OpenMP each thread sums a contiguous block of pixels into its own
 * partial matrix and the partials are added in thread order.
 */
int oracle_covariance(const double *Y, long N, int B, const double *mu, double *C) {
  if (N < 2 || B < 1) return ORC_ERR_ARG;
  const size_t BB = (size_t)B * (size_t)B;
  int T = g_threads;
  if ((long)T > N) T = (int)N;
  double *part = (double *)calloc((size_t)T * BB, sizeof(double));
  double *xbuf = (double *)malloc((size_t)T * (size_t)B * sizeof(double));
  if (!part || !xbuf) { free(part); free(xbuf); return ORC_ERR_ARG; }
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(static)
#endif
  for (int t = 0; t < T; ++t) {
    long n0 = N * t / T, n1 = N * (t + 1) / T;
    double *P = part + (size_t)t * BB;
    double *x = xbuf + (size_t)t * B;
    for (long n = n0; n < n1; ++n) {
      for (int b = 0; b < B; ++b) x[b] = Y[n * B + b] - mu[b];
      for (int i = 0; i < B; ++i) {
        double xi = x[i];
        double *Pi = P + (size_t)i * B;
        for (int j = i; j < B; ++j) Pi[j] += xi * x[j];
      }
    }
  }
  const double inv = 1.0 / (double)(N - 1);
  for (int i = 0; i < B; ++i)
    for (int j = i; j < B; ++j) {
      double s = 0.0;
      for (int t = 0; t < T; ++t) s += part[(size_t)t * BB + (size_t)i * B + j];
      C[(size_t)i * B + j] = s * inv;
      C[(size_t)j * B + i] = s * inv;
    }
  free(part);
  free(xbuf);
  return ORC_OK;
}

/*
 * Eqs. 2-5 (generalised by Eq. 7 to the pair (p, q), p < q): the rotation
 * that zeroes a_pq of the symmetric 2x2 block [[a_pp, a_pq], [a_pq, a_qq]]
 * under B = P^T A P with P = [[c, s], [-s, c]] (Eq. 1, Eq. 6).
 * m = 2 a_pq / (a_qq - a_pp) (Eq. 7); t is the root of Eq. 3, evaluated as
 * t = sgn(tau) / (|tau| + sqrt(1 + tau^2)) with tau = 1/m, which is the same
 * number without the cancellation of Eq. 3 at small m and without its
 * division by zero at a_pp == a_qq (tau = 0 gives t = 1, a 45 degree turn).
 * c = 1/sqrt(1+t^2) (Eq. 4), s = t c (Eq. 5).
 */
void oracle_rotation(double app, double aqq, double apq, double *c, double *s) {
  if (apq == 0.0) { *c = 1.0; *s = 0.0; return; }
  double tau = (aqq - app) / (2.0 * apq);
  double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  double cc = 1.0 / sqrt(1.0 + t * t);
  *c = cc;
  *s = t * cc;
}

/*
 * One Jacobi rotation, Eq. 8 restricted to the rows and columns it changes:
 * rows p and q of A are combined first (the "update rows" step of the
 * manycore implementation, Sec. 5 stage 3), then columns p and q (its
 * "update columns" step), and columns p and q of V are combined the same
 * way (Eq. 10: E = P_1 P_2 ... P_K accumulated column-wise).  The zeroed
 * pair is set to exactly 0, which it is in exact arithmetic.
 * Returns 1 if a rotation was applied, 0 if a_pq was already 0.
 */
static int rotate_pair(double *A, double *V, int B, int p, int q) {
  double c, s;
  double apq = A[(size_t)p * B + q];
  if (apq == 0.0) return 0;
  oracle_rotation(A[(size_t)p * B + p], A[(size_t)q * B + q], apq, &c, &s);
  /* rows: A <- P^T A ; (P^T)_{pp}=c, (P^T)_{pq}=-s, (P^T)_{qp}=s, (P^T)_{qq}=c */
  for (int k = 0; k < B; ++k) {
    double apk = A[(size_t)p * B + k], aqk = A[(size_t)q * B + k];
    A[(size_t)p * B + k] = c * apk - s * aqk;
    A[(size_t)q * B + k] = s * apk + c * aqk;
  }
  /* columns: A <- A P ; P_{pp}=c, P_{pq}=s, P_{qp}=-s, P_{qq}=c */
  for (int k = 0; k < B; ++k) {
    double akp = A[(size_t)k * B + p], akq = A[(size_t)k * B + q];
    A[(size_t)k * B + p] = c * akp - s * akq;
    A[(size_t)k * B + q] = s * akp + c * akq;
  }
  A[(size_t)p * B + q] = 0.0;
  A[(size_t)q * B + p] = 0.0;
  /* eigenvectors: V <- V P */
  for (int k = 0; k < B; ++k) {
    double vkp = V[(size_t)k * B + p], vkq = V[(size_t)k * B + q];
    V[(size_t)k * B + p] = c * vkp - s * vkq;
    V[(size_t)k * B + q] = s * vkp + c * vkq;
  }
  return 1;
}

/* Off-diagonal Frobenius norm and full Frobenius norm of A. */
static void norms(const double *A, int B, double *off, double *fro) {
  double so = 0.0, sd = 0.0;
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < B; ++j) {
      double a = A[(size_t)i * B + j];
      if (i == j) sd += a * a; else so += a * a;
    }
  *off = sqrt(so);
  *fro = sqrt(so + sd);
}

#define ORD_ROW_CYCLIC 0
#define ORD_ROUND_ROBIN 1
#define ORD_ODD_EVEN 2
#define ORD_CLASSICAL 3
#define ORD_GREEDY 4

/*
 * Classical pivot (Sec. 4.2 stage 4.1): the off-diagonal element of largest
 * magnitude in the upper triangle, the first in row-major order on ties.
 * Returns 0 when every off-diagonal element is 0.
 */
static int classical_pivot(const double *A, int B, int *pp, int *pq) {
  double best = 0.0;
  int found = 0;
  for (int i = 0; i < B - 1; ++i)
    for (int j = i + 1; j < B; ++j) {
      double a = fabs(A[(size_t)i * B + j]);
      if (a > best) { best = a; *pp = i; *pq = j; found = 1; }
    }
  return found;
}

/*
 * One iteration of the manycore's greedy selection (Sec. 5, Code 5.3.1): scan
 * the upper triangle row by row and take (i, j) when |a_ij| > thr, (i, j) has
 * not been zeroed yet in this sweep, and neither i nor j is already used in
 * this iteration; the taken pairs share no index, so their rotations commute
 * (Sec. 2) and are applied one after the other.  zeroed[B*B] marks the pairs
 * of the sweep; used[B] is scratch.  Returns the number of pairs rotated.
 */
static int greedy_iteration(double *A, double *V, int B, double thr, unsigned char *zeroed,
                            unsigned char *used, long *nrot) {
  memset(used, 0, (size_t)B);
  int taken = 0;
  for (int i = 0; i < B - 1; ++i)
    for (int j = i + 1; j < B; ++j) {
      if (used[i] || used[j] || zeroed[(size_t)i * B + j]) continue;
      if (!(fabs(A[(size_t)i * B + j]) > thr)) continue;
      used[i] = used[j] = 1;
      zeroed[(size_t)i * B + j] = 1;
      *nrot += rotate_pair(A, V, B, i, j);
      ++taken;
    }
  return taken;
}

/*
 * Cyclic Jacobi (Sec. 2, Eqs. 6-10; cyclic ordering chosen in Sec. 2 over
 * the classical largest-element pivot).  A (B x B, symmetric, row-major) is
 * overwritten by the nearly diagonal C_K of Eq. 9; V (B x B) receives
 * E = P_1 ... P_K of Eq. 10, starting from the identity.
 *
 * ordering:
 *   0 row-cyclic: (0,1),(0,2),...,(0,B-1),(1,2),...,(B-2,B-1), the textbook
 *     "row by row" order named in Sec. 2;
 *   1 round-robin (circle method): B'-1 rounds of B'/2 disjoint pairs, B' = B
 *     rounded up to even, index B'-1 a dummy when B is odd; the pairs of a
 *     round touch disjoint rows and columns (Sec. 2, last paragraph), here
 *     applied one after the other;
 *   2 odd-even: B' rounds; even rounds pair positions (0,1),(2,3),...,
 *     odd rounds (1,2),(3,4),...; after each rotation the two indices swap
 *     positions, so every index pair meets exactly once per sweep;
 *   3 classical (the GPU host loop of Sec. 4.2 stage 4.1): every rotation
 *     zeroes the largest off-diagonal element; a "sweep" is B(B-1)/2
 *     rotations (fewer when the matrix is already diagonal);
 *   4 greedy (the manycore's Code 5.3.1): iterations of disjoint pairs chosen
 *     row by row among the elements above thr = tol ||A||_F / sqrt(B(B-1))
 *     not yet zeroed in the sweep; a sweep ends when an iteration finds none.
 *     The per-element threshold is the one at which every element below it
 *     implies the stop test off(A) <= tol ||A||_F.
 * The stop test runs before each sweep: off(A) <= tol * ||A||_F, or
 * ||A||_F == 0.  *sweeps = sweeps run, *off_rel = final off(A)/||A||_F,
 * *rotations = rotations applied.  Returns ORC_ERR_NOCONV if sweeps_max
 * sweeps did not reach the tolerance (A and V then hold the last iterate).
 */
int oracle_jacobi(double *A, int B, double tol, int sweeps_max, int ordering,
                  double *V, int *sweeps, double *off_rel, long *rotations) {
  if (B < 1 || sweeps_max < 0 || !(tol >= 0.0)) return ORC_ERR_ARG;
  for (size_t i = 0; i < (size_t)B * B; ++i)
    if (!isfinite(A[i])) return ORC_ERR_NONFINITE;
  memset(V, 0, sizeof(double) * (size_t)B * B);
  for (int i = 0; i < B; ++i) V[(size_t)i * B + i] = 1.0;
  const int Bp = B + (B & 1);
  int *pos = (int *)malloc(sizeof(int) * (size_t)Bp);
  unsigned char *zeroed = (unsigned char *)malloc((size_t)B * B + 1);
  unsigned char *used = (unsigned char *)malloc((size_t)B + 1);
  if (!pos || !zeroed || !used) { free(pos); free(zeroed); free(used); return ORC_ERR_ARG; }
  long nrot = 0;
  int sw = 0, status = ORC_ERR_NOCONV;
  double off, fro;
  for (;;) {
    norms(A, B, &off, &fro);
    if (fro == 0.0 || off <= tol * fro) { status = ORC_OK; break; }
    if (sw >= sweeps_max) break;
    if (ordering == ORD_ROW_CYCLIC) {
      for (int p = 0; p < B - 1; ++p)
        for (int q = p + 1; q < B; ++q) nrot += rotate_pair(A, V, B, p, q);
    } else if (ordering == ORD_ROUND_ROBIN) {
      for (int r = 0; r < Bp - 1; ++r) {
        for (int s = 0; s < Bp; ++s) pos[s] = (s == 0) ? 0 : ((s - 1 + r) % (Bp - 1)) + 1;
        for (int i = 0; i < Bp / 2; ++i) {
          int a = pos[i], b = pos[Bp - 1 - i];
          int p = a < b ? a : b, q = a < b ? b : a;
          if (q >= B) continue; /* the dummy index */
          nrot += rotate_pair(A, V, B, p, q);
        }
      }
    } else if (ordering == ORD_ODD_EVEN) {
      if (sw == 0)
        for (int s = 0; s < Bp; ++s) pos[s] = s;
      for (int r = 0; r < Bp; ++r) {
        for (int s0 = (r & 1); s0 + 1 < Bp; s0 += 2) {
          int a = pos[s0], b = pos[s0 + 1];
          int p = a < b ? a : b, q = a < b ? b : a;
          if (q < B) nrot += rotate_pair(A, V, B, p, q);
          pos[s0] = b;
          pos[s0 + 1] = a;
        }
      }
    } else if (ordering == ORD_CLASSICAL) {
      const long m = (long)B * (B - 1) / 2;
      for (long r = 0; r < m; ++r) {
        int p = 0, q = 0;
        if (!classical_pivot(A, B, &p, &q)) break;
        nrot += rotate_pair(A, V, B, p, q);
      }
    } else if (ordering == ORD_GREEDY) {
      const double thr = B > 1 ? tol * fro / sqrt((double)B * (B - 1)) : 0.0;
      memset(zeroed, 0, (size_t)B * B);
      while (greedy_iteration(A, V, B, thr, zeroed, used, &nrot) > 0) {
      }
    } else {
      free(pos); free(zeroed); free(used);
      return ORC_ERR_ARG;
    }
    ++sw;
  }
  free(pos);
  free(zeroed);
  free(used);
  *sweeps = sw;
  *off_rel = (fro == 0.0) ? 0.0 : off / fro;
  *rotations = nrot;
  return status;
}

/*
 * The first `steps` steps of an ordering, without any stop test, for the pins
 * of the orderings: a step is one rotation (classical) or one iteration of
 * disjoint pairs (greedy, threshold thr, all in one sweep).  V starts from the
 * identity.  Returns the number of rotations applied (< 0 on bad arguments).
 */
long oracle_jacobi_steps(double *A, int B, int ordering, int steps, double thr, double *V) {
  if (B < 1 || steps < 0 || (ordering != ORD_CLASSICAL && ordering != ORD_GREEDY)) return -1;
  memset(V, 0, sizeof(double) * (size_t)B * B);
  for (int i = 0; i < B; ++i) V[(size_t)i * B + i] = 1.0;
  long nrot = 0;
  if (ordering == ORD_CLASSICAL) {
    for (int s = 0; s < steps; ++s) {
      int p = 0, q = 0;
      if (!classical_pivot(A, B, &p, &q)) break;
      nrot += rotate_pair(A, V, B, p, q);
    }
    return nrot;
  }
  unsigned char *zeroed = (unsigned char *)calloc((size_t)B * B + 1, 1);
  unsigned char *used = (unsigned char *)malloc((size_t)B + 1);
  if (!zeroed || !used) { free(zeroed); free(used); return -1; }
  for (int s = 0; s < steps; ++s)
    if (greedy_iteration(A, V, B, thr, zeroed, used, &nrot) == 0) break;
  free(zeroed);
  free(used);
  return nrot;
}

/*
 * Sec. 4.2 stage 4.3: the eigenvalues are the diagonal of C_K, sorted in
 * descending order, and the eigenvectors (columns of V) follow the same
 * permutation.  Ties keep the lower original index first (insertion sort is
 * stable).  Then the sign rule: each column is negated when its entry of
 * largest magnitude (lowest row on ties) is negative.
 * lam[B] holds diag(C_K) on entry and the sorted eigenvalues on return.
 */
int oracle_sort_sign(int B, double *lam, double *V) {
  int *idx = (int *)malloc(sizeof(int) * (size_t)B);
  double *W = (double *)malloc(sizeof(double) * (size_t)B * B);
  double *l2 = (double *)malloc(sizeof(double) * (size_t)B);
  if (!idx || !W || !l2) { free(idx); free(W); free(l2); return ORC_ERR_ARG; }
  for (int i = 0; i < B; ++i) idx[i] = i;
  for (int i = 1; i < B; ++i) {
    int v = idx[i];
    int j = i - 1;
    while (j >= 0 && lam[idx[j]] < lam[v]) { idx[j + 1] = idx[j]; --j; }
    idx[j + 1] = v;
  }
  for (int j = 0; j < B; ++j) {
    int src = idx[j];
    l2[j] = lam[src];
    for (int i = 0; i < B; ++i) W[(size_t)i * B + j] = V[(size_t)i * B + src];
  }
  for (int j = 0; j < B; ++j) {
    int im = 0;
    double best = fabs(W[j]);
    for (int i = 1; i < B; ++i) {
      double a = fabs(W[(size_t)i * B + j]);
      if (a > best) { best = a; im = i; }
    }
    double sg = W[(size_t)im * B + j] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < B; ++i) V[(size_t)i * B + j] = sg * W[(size_t)i * B + j];
    lam[j] = l2[j];
  }
  free(idx);
  free(W);
  free(l2);
  return ORC_OK;
}

/*
 * Stages 3-4 of Algorithm 1 ("Projection" and "MatrixColumnRemoval"):
 * Q = X V, keeping the first k columns.  Q[n*k + j] = sum_b (Y_nb - mu_b) V_bj.
 */
int oracle_project(const double *Y, long N, int B, const double *mu, const double *V,
                   int k, double *Q) {
  if (N < 1 || B < 1 || k < 1 || k > B) return ORC_ERR_ARG;
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) schedule(static)
#endif
  for (long n = 0; n < N; ++n) {
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int b = 0; b < B; ++b) s += (Y[n * B + b] - mu[b]) * V[(size_t)b * B + j];
      Q[n * k + j] = s;
    }
  }
  return ORC_OK;
}

/*
 * The four stages of Algorithm 1 in order: means, covariance, Jacobi with
 * row-cyclic order (unless `ordering` says otherwise), sort + sign,
 * projection onto the first k eigenvectors.  Q may be NULL (no projection).
 */
int oracle_pca_fit(const double *Y, long N, int B, int k, double tol, int sweeps_max,
                   int ordering, double *mu, double *lam, double *V, double *Q,
                   int *sweeps, double *off_rel, long *rotations) {
  if (N < 2 || B < 1 || k < 1 || k > B || sweeps_max < 0) return ORC_ERR_ARG;
  int st = oracle_band_means(Y, N, B, mu);
  if (st) return st;
  double *C = (double *)malloc(sizeof(double) * (size_t)B * B);
  if (!C) return ORC_ERR_ARG;
  st = oracle_covariance(Y, N, B, mu, C);
  if (st) { free(C); return st; }
  int js = oracle_jacobi(C, B, tol, sweeps_max, ordering, V, sweeps, off_rel, rotations);
  if (js != ORC_OK && js != ORC_ERR_NOCONV) { free(C); return js; }
  for (int i = 0; i < B; ++i) lam[i] = C[(size_t)i * B + i];
  free(C);
  oracle_sort_sign(B, lam, V);
  if (Q) {
    st = oracle_project(Y, N, B, mu, V, k, Q);
    if (st) return st;
  }
  return js;
}

/*
 * Adjoint of the whole path (not in the paper; the backward pass of the PCA
 * projection layer, written from first-order perturbation theory of the
 * symmetric eigenproblem).  Given the forward results mu [B], lam [B]
 * (descending), V [B][B] (column j = eigenvector j) of the cube Y [N][B], the
 * upstream gradient dQ [N][k] of Q = X V_k and, optionally, dlam [B] (NULL =
 * zero), it forms, step by step:
 *   X        = Y - 1 mu^T
 *   dVk      = X^T dQ                                   (B x k)
 *   M        = V^T [dVk, 0]                             (B x B, columns >= k zero)
 *   G_ij     = M_ij / (lam_j - lam_i)  for i != j with |lam_j - lam_i| > gap_eps |lam_1|,
 *              0 for the other off-diagonal entries,  G_ii = dlam_i
 *   dA       = V G V^T,   S = (dA + dA^T) / 2
 *   dY       = (dQ - 1 mean_n(dQ)) V_k^T + 2/(N-1) X S
 * (C = X^T X/(N-1) gives dX = 2 X S/(N-1); the centring maps dX to
 * dX - 1 mean_n(dX), and 1^T X = 0 leaves the second term unchanged.)
 */
int oracle_backward(const double *Y, long N, int B, int k, const double *mu,
                    const double *lam, const double *V, const double *dQ, const double *dlam,
                    double gap_eps, double *dY) {
  if (N < 2 || B < 1 || k < 1 || k > B) return ORC_ERR_ARG;
  const size_t BB = (size_t)B * B;
  double *dVk = (double *)calloc((size_t)B * k, sizeof(double));
  double *M = (double *)calloc(BB, sizeof(double));
  double *G = (double *)calloc(BB, sizeof(double));
  double *T = (double *)calloc(BB, sizeof(double));
  double *S = (double *)calloc(BB, sizeof(double));
  double *mdq = (double *)calloc((size_t)k, sizeof(double));
  if (!dVk || !M || !G || !T || !S || !mdq) {
    free(dVk); free(M); free(G); free(T); free(S); free(mdq);
    return ORC_ERR_ARG;
  }
  /* dVk = X^T dQ and the column means of dQ */
  for (long n = 0; n < N; ++n)
    for (int b = 0; b < B; ++b) {
      const double x = Y[n * B + b] - mu[b];
      for (int j = 0; j < k; ++j) dVk[(size_t)b * k + j] += x * dQ[n * k + j];
    }
  for (long n = 0; n < N; ++n)
    for (int j = 0; j < k; ++j) mdq[j] += dQ[n * k + j];
  for (int j = 0; j < k; ++j) mdq[j] /= (double)N;
  /* M = V^T [dVk, 0] */
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int b = 0; b < B; ++b) s += V[(size_t)b * B + i] * dVk[(size_t)b * k + j];
      M[(size_t)i * B + j] = s;
    }
  /* G = F o M + diag(dlam) */
  const double big = fabs(lam[0]);
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < B; ++j) {
      if (i == j) {
        G[(size_t)i * B + j] = dlam ? dlam[i] : 0.0;
      } else {
        const double gap = lam[j] - lam[i];
        G[(size_t)i * B + j] = fabs(gap) > gap_eps * big ? M[(size_t)i * B + j] / gap : 0.0;
      }
    }
  /* dA = V G V^T (T = V G first), S = (dA + dA^T)/2 */
  for (int a = 0; a < B; ++a)
    for (int j = 0; j < B; ++j) {
      double s = 0.0;
      for (int i = 0; i < B; ++i) s += V[(size_t)a * B + i] * G[(size_t)i * B + j];
      T[(size_t)a * B + j] = s;
    }
  for (int a = 0; a < B; ++a)
    for (int c = 0; c < B; ++c) {
      double s = 0.0;
      for (int j = 0; j < B; ++j) s += T[(size_t)a * B + j] * V[(size_t)c * B + j];
      S[(size_t)a * B + c] += 0.5 * s;
      S[(size_t)c * B + a] += 0.5 * s;
    }
  /* dY */
  const double f = 2.0 / (double)(N - 1);
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) schedule(static)
#endif
  for (long n = 0; n < N; ++n)
    for (int c = 0; c < B; ++c) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += (dQ[n * k + j] - mdq[j]) * V[(size_t)c * B + j];
      double t = 0.0;
      for (int b = 0; b < B; ++b) t += (Y[n * B + b] - mu[b]) * S[(size_t)b * B + c];
      dY[n * B + c] = s + f * t;
    }
  free(dVk); free(M); free(G); free(T); free(S); free(mdq);
  return ORC_OK;
}
