// internal.h -- shared declarations of the sm_103a Jacobi-PCA kernels.
// Not part of the public ABI (include/gbpca.h is).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gbpca.h"

namespace gbpca {

constexpr int kMaxB = 256;          // two 128-row tensor-core tiles; 8 Jacobi CTAs x 32 V rows
constexpr int kMaxPartials = 320;   // per-CTA covariance partial slots
constexpr float kJacobiFloor = 2.384185791015625e-07f;  // 2^-22: FP32 Jacobi stop floor
constexpr float kMixJacobiFloor = 1e-5f;                 // MIX: refinement takes over from here

// Device-side outcome, first 256 bytes of the workspace.
struct DevHeader {
  int status;        // pca_status
  int sweeps;
  int steps;
  int refine_iters;
  int nonfinite;
  int dummy_slot;    // slot of the padding index when B is odd, else -1
  int cov_range;     // tensor-core covariance met a value outside its scaled FP16 range
  int proj_range;    // tensor-core projection met a value outside its scaled FP16 range
  double off_rel;
  double fro;
  double tol_used;
  double refine_res;
  double delta;      // cluster threshold of the last refinement iteration
};

// Offsets (bytes) of every workspace region; all 256-byte aligned.
struct Layout {
  size_t hdr, shift, escale, s1_part, s2_part, dvec, cov, cdf, rank, sgn, diag32, v32, lam, vc, w, s, r, e, vk, muf;
  size_t ptc_shift, ptc_escale, ptc_planes, ptc_colscale, ptc_corr;   // tensor-core projection
  size_t total;
  int partials;      // number of covariance partial slots the SYRK uses
  int tc_ctas;       // MIX: CTAs of the tensor-core pass (partials spread over them)
  int s2_elems;      // packed upper-triangle entries per partial: B(B+1)/2
  int s2_bytes_el;   // 4 (FP32 partials) or 8 (FP64 partials)
};

Layout make_layout(int64_t N, int B, int k, pca_dtype dt, pca_precision prec, int num_sms);

__host__ __device__ inline int round_even(int b) { return b + (b & 1); }
// Packed upper triangle, column by column: entry (i, j), i <= j, of a B x B
// symmetric matrix at j(j+1)/2 + i, so that the rows of one column -- the
// TMEM lanes of the tensor-core epilogue -- are contiguous.
__host__ __device__ inline int64_t packed_index(int i, int j, int B) {  // i <= j
  (void)B;
  return (int64_t)j * (j + 1) / 2 + i;
}

// ---------------------------------------------------------------- precision policy
// FP64 refinement iterations after the FP32 sweeps.  P64 runs five: pairs just
// outside a cluster (first-order angles a little below the cluster bound)
// converge slowly, and on a spectrum with a large cluster (the 16-bit rounding
// floor of a 2048 x 2048 x 224 BF16 cube) three iterations left eigenvector
// residuals of 1e-10 ||C||, five leave 3e-12.
inline int refine_iterations(pca_precision prec) {
  return prec == PCA_PREC_P32 ? 0 : (prec == PCA_PREC_MIX ? 1 : 5);
}
// Lowest stop threshold of the FP32 sweeps.  MIX hands the eigen-pairs to its
// quadratically convergent refinement once off(A) <= 1e-5 ||A||_F: on the
// scene cubes that saves two to three sweeps, and one iteration leaves the
// top-k eigenvalues within 3e-7 relative of the exact C's -- far below the
// error of the tensor-core covariance itself; P32 and P64 sweep to the FP32
// floor.
inline float stop_floor(pca_precision prec) {
  return prec == PCA_PREC_MIX ? kMixJacobiFloor : kJacobiFloor;
}
// Largest first-order angle the refinement applies (pairs above it count as clustered).
inline double refine_max_angle(pca_precision prec) { (void)prec; return 1.0 / 64; }
// Closing Newton-Schulz orthogonalisation steps (P64: one more, for the
// non-orthogonality a large last update leaves, ~1e-3 in the case above).
inline int ortho_steps(pca_precision prec) {
  return prec == PCA_PREC_P32 ? 0 : (prec == PCA_PREC_MIX ? 2 : 3);
}
// MIX stops its FP32 sweeps on the Frobenius test (the refinement resolves what
// the element-wise test would still demand); P32 and P64 use the element-wise test.
inline bool relative_stop(pca_precision prec) { return prec != PCA_PREC_MIX; }

// The current tuning parameters (pca_set_tuning; measured defaults otherwise).
pca_tuning tuning();

// Argument checks shared by the entry points; SMs of the current device.
bool args_ok(const void* cube, pca_dtype dt, int64_t N, int B, int k, double tol,
             int sweeps_max, pca_precision prec);
int device_sms();

// Optional per-stage CUDA-event timing (pca_profile): one record per fit, marks
// 0..8 around the stages covariance, finalisation, Jacobi, (empty), compaction,
// refinement, sort/sign, projection.  Inactive unless profiling is on.
struct StageMark {
  cudaStream_t st;
  int rec;
  explicit StageMark(cudaStream_t s);
  void mark(int i);
};

// ---------------------------------------------------------------- batched form
// One tile of a batch: its input, the caller's outputs and its workspace
// regions.  Device-resident, written once when the batch is planned.
struct TileDesc {
  const void* cube;    // [N][B], 16-byte aligned
  int64_t N;
  int B, k;
  double* mu;          // caller outputs
  double* eigvals;
  double* eigvecs;
  float* proj;         // nullable
  DevHeader* hdr;      // workspace
  float* shift;
  int* escale;
  double* s1p;         // [parts][B]
  void* s2p;           // [parts][B(B+1)/2], FP32 or FP64
  int parts;           // covariance partial slots of this tile
  int pad0;
  double* dvec;
  double* C;
  float2* cdf;
  int* rank;
  double* sgn;
  float* diag32;
  float* v32;
  double* lam;
  float2* vc;
  float2* w;
  float2* s;
  float2* g;
  float2* e;
  float* vk;
  float* muf;
};
// Pixels [p0, p1) of one tile and the partial slot they are summed into.
struct CovItem {
  int tile, slot;
  int64_t p0, p1;
};
// 64-pixel chunks [c0, c1) of one tile, columns [32 pad, 32 pad + 32) of its V_k.
struct ProjItem {
  int tile, pad;
  int64_t c0, c1;
};

// ---------------------------------------------------------------- launchers
// All return cudaError_t of the launch; none synchronises.

// Covariance partials, SIMT: P32 (FP32 accumulate) or P64 (FP64 accumulate).
// shift = first pixel; writes s1_part[G][B] (FP64) and s2_part[G][B(B+1)/2].
// With guard != nullptr every CTA returns at once unless *guard != 0; a run
// then also zeroes escale[B] (the partials it writes are unscaled).
cudaError_t launch_syrk_simt(const void* cube, pca_dtype dt, int64_t N, int B, bool fp64,
                             float* shift, double* s1_part, void* s2_part, int partials,
                             cudaStream_t st, const int* guard = nullptr, int* escale = nullptr);

// Covariance partials on the tensor cores (tcgen05, split-FP16 of the scaled,
// shifted values, three products).  Every CTA derives the per-band shift
// (mean of 32 sampled pixels) and power-of-two scale exponent from the same
// pixels; CTA 0 writes them to shift [B] (FP32) and escale [B] (int).  S1
// partials are unscaled, S2 partials stay scaled by 2^(e_i + e_j).  A value
// outside the FP16 range after scaling sets hdr->cov_range.
cudaError_t launch_syrk_tc(const void* cube, pca_dtype dt, int64_t N, int B, float* shift,
                           int* escale, double* s1_part, float* s2_part, int partials, int ctas,
                           DevHeader* hdr, cudaStream_t st);
// Longest run of 32-pixel chunks one tensor-core partial slot accumulates for a
// cube of this type: the FP32 accumulation in tensor memory loses accuracy in
// proportion to its length (FP32 cubes); 16-bit cubes sum exact products.
int tc_slot_chunks(pca_dtype dt);
bool syrk_tc_supported(int B);

// Sums the partials, applies the shift correction, writes mu (FP64), C (FP64, full
// symmetric) and mu_f (FP32), flags non-finite sums in the header.
// escale (nullable): S2 partials are scaled by 2^(escale[i] + escale[j]).
cudaError_t launch_cov_finalize(const float* shift, const double* s1_part, const void* s2_part,
                                bool fp64_partials, int partials, int64_t N, int B, double* mu,
                                double* C, float* mu_f, double* dvec, DevHeader* hdr,
                                cudaStream_t st, const int* escale = nullptr);

// FP32 odd-even Jacobi on one thread-block cluster (matrix rows split over
// the CTAs, rows of V in registers): writes diag32 [B'] and V32 [B'][B'].
// relative_stop selects the element-wise relative stop test (else
// off(A) <= tol ||A||_F).
cudaError_t launch_jacobi_cluster(const double* C, int B, float tol32, int sweeps_max,
                                  bool relative_stop, float* diag32, float* v32, DevHeader* hdr,
                                  cudaStream_t st);

// CTAs (= SMs) the cluster Jacobi uses for B bands: nA matrix CTAs + nV V CTAs.
bool jacobi_cluster_shape(int B, int* nA, int* nV);

// Drops the padding slot: lam (FP64) [B] and Vc [B][B] in slot order, Vc as
// double-float (hi, lo) pairs.
cudaError_t launch_compact(const float* diag32, const float* v32, int B, DevHeader* hdr,
                           double* lam, float2* vc, cudaStream_t st);

// dst = src as double-float (hi, lo) pairs.
cudaError_t launch_to_df(const double* src, float2* dst, int count, cudaStream_t st);

// One refinement iteration (double-float products, FP64 angles) from V (v)
// to V' (vout; also the scratch for C V); C, s, g, e are B x B double-float.
// max_angle: pairs whose first-order angle exceeds it are only
// re-orthogonalised.
cudaError_t launch_refine(const float2* C, int B, const float2* v, float2* vout, double* lam,
                          float2* s, float2* g, float2* e, DevHeader* hdr, double max_angle,
                          cudaStream_t st);

// One Newton-Schulz orthogonalisation step of V (double-float), v -> vout.
cudaError_t launch_orthonormalize(const float2* v, float2* vout, int B, float2* g, float2* e,
                                  cudaStream_t st);

// Sort descending, sign-normalise, write eigvals/eigvecs (FP64) and V_k (FP32).
// rank [B] (int) and sgn [B] (FP64) are scratch.
cudaError_t launch_sort_sign(const double* lam, const float2* vc, int B, int k, double* eigvals,
                             double* eigvecs, float* vk, int* rank, double* sgn, cudaStream_t st);

// mu_f = (float)mu, vk = (float)eigvecs[:, :k] (eigvecs B x B row-major).
cudaError_t launch_narrow_inputs(const double* mu, const double* eigvecs, int B, int k, float* mu_f,
                                 float* vk, cudaStream_t st);

// Q = (Y - 1 mu^T) V_k, FP32 (TMA-streamed).  hdr (nullable) receives
// PCA_ERR_TIMEOUT if a bounded wait gives up (the output range is then NaN).
// With guard != nullptr every CTA returns at once unless *guard != 0.
cudaError_t launch_project(const void* cube, pca_dtype dt, int64_t N, int B, int k,
                           const float* mu_f, const float* vk, float* proj, cudaStream_t st,
                           DevHeader* hdr = nullptr, const int* guard = nullptr);

// Q = (Y - 1 mu^T) V_k on the tensor cores from mu [B] and V [B][B] (FP64,
// device; the first k columns of V), FP32 accumulation; workspace: shift [256]
// (FP32), escale [256] (int), planes of project_tc_planes_bytes(B, k) bytes,
// colscale [128], corr [128] (FP32).  A scaled value outside the FP16 range
// sets hdr->proj_range (the caller then recomputes Q on the SIMT path).
size_t project_tc_planes_bytes(int B, int k);
cudaError_t launch_project_tc(const void* cube, pca_dtype dt, int64_t N, int B, int k,
                              const double* mu, const double* V, float* proj, float* shift,
                              int* escale, unsigned char* planes, float* colscale, float* corr,
                              DevHeader* hdr, cudaStream_t st);

// Scratch of the backward pass (all device pointers, inside the caller's
// workspace): parts per-CTA partials of X^T dQ [parts][B][k] and of the column
// sums of dQ [parts][k] (FP32); dVk [B][k], Gk [B][k], dA [B][B] (FP64); S'
// [B][B], V_k [B][k], mean dQ [k], mu [B] (FP32).
struct BwdPtrs {
  int parts;
  float* dv_part;
  float* dqs_part;
  double* dVk;
  double* Gk;
  double* dA;
  float* S32;
  float* vk32;
  float* mdq;
  float* mu32;
  float* xmax_part;      // [parts][B] largest |x_b| per CTA
  float* dqmax_part;     // [parts][k] largest |dq_j| per CTA
  float* ascale;         // [B32 + k] power-of-two scales of the A operand of dY (B32 = B
                         // rounded up to 32, where the dQ segment of K starts)
  float* anshift;        // [B32 + k] -shift * scale
  unsigned char* bop;    // B operand of dY: FP16 hi/lo planes per 32-wide K block
  float* fcol;           // [2][B] column scales 2^-f_c of the two K segments
};
// Bytes of the B operand planes of the tensor-core dY product.
size_t bwd_bop_bytes(int B, int k);
// dY = [X | dQ'] [S'; V_k^T] on the tensor cores (with its scale and operand
// preparation kernels).
cudaError_t launch_bwd_dy_tc(const void* cube, pca_dtype dt, const float* dq, int64_t N, int B,
                             int k, const float* xmax_part, const float* dqmax_part, int parts,
                             const float* mu32, const float* mdq, const float* S32,
                             const float* vk32, float* ascale, float* anshift, unsigned char* bop,
                             float* fcol, float* dY, DevHeader* hdr, cudaStream_t st);

// dY = (dQ - 1 mean dQ) V_k^T + 2/(N-1) X S (the adjoint of the projection
// layer; dlam nullable).
cudaError_t launch_backward(const void* cube, pca_dtype dt, int64_t N, int B, int k,
                            const double* mu, const double* lam, const double* V,
                            const float* dq, const double* dlam, double gap_eps, float* dY,
                            const BwdPtrs& w, DevHeader* hdr, cudaStream_t st);

// ---- batched launchers: tile t of T[] is blockIdx.y (or an item's tile)
cudaError_t launch_header_init_batched(TileDesc* T, int ntiles, int refine_iters, float tol32,
                                       cudaStream_t st);
// SIMT partials of every item (grid: items x band-tile groups of the largest B).
// guarded: a tile is skipped unless its hdr->cov_range is set, and a run then
// zeroes its escale; the launch is a small grid that returns at once when no
// tile of the ntiles is flagged.
cudaError_t launch_syrk_simt_grouped(const TileDesc* T, const CovItem* items, int nitems,
                                     int maxB, int ntiles, pca_dtype dt, bool fp64, bool guarded,
                                     cudaStream_t st);
// Tensor-core partials: CTA g walks items [cta_items[g], cta_items[g+1]).
cudaError_t launch_syrk_tc_grouped(const TileDesc* T, const CovItem* items, const int* cta_items,
                                   int ctas, int maxB, pca_dtype dt, cudaStream_t st);
cudaError_t launch_cov_finalize_batched(const TileDesc* T, int ntiles, int maxB, bool fp64,
                                        bool escaled, cudaStream_t st);
// Jacobi parameter lists: matrices of one shape (equal V width and cluster
// size) run in one launch, one cluster each.
int jacobi_width(int B);     // V values per lane of a V row (kernel variant)
int jacobi_min_ctas(int B);  // fewest CTAs per cluster of the default kernel variant
int jacobi_batch_ctas(int B);  // fewest CTAs per cluster of any variant (batched form)
// The fewest CTAs, at least n, whose cluster holds a matrix of B bands (some
// variant fits); n <= 0 gives jacobi_batch_ctas(B).
int jacobi_ctas_at_least(int B, int n);
size_t jacobi_params_bytes();
// Writes the parameters of one matrix to dst (host) for a cluster of nA CTAs
// (0: the latency-oriented default of the single-matrix form); returns the
// dynamic shared memory its cluster needs.
size_t jacobi_fill_params(void* dst, const double* C, int B, float tol32, int sweeps_max,
                          bool relative_stop, float* diag32, float* v32, DevHeader* hdr, int nA);
int jacobi_params_ctas(const void* params);
cudaError_t launch_jacobi_cluster_list(const void* host_first, const void* dev_list, int count,
                                       size_t smem, cudaStream_t st);
cudaError_t launch_compact_batched(const TileDesc* T, int ntiles, int maxB, cudaStream_t st);
cudaError_t launch_to_df_batched(const TileDesc* T, int ntiles, int maxB, cudaStream_t st);
// One refinement iteration / orthogonalisation step of every tile; `flip`
// selects the direction of the V double buffer (false: vc -> w).
cudaError_t launch_refine_batched(const TileDesc* T, int ntiles, int maxB, bool flip,
                                  double max_angle, cudaStream_t st);
cudaError_t launch_orthonormalize_batched(const TileDesc* T, int ntiles, int maxB, bool flip,
                                          cudaStream_t st);
cudaError_t launch_sort_sign_batched(const TileDesc* T, int ntiles, int maxB, bool final_in_w,
                                     cudaStream_t st);
// Streamed projection of every item; maps (nullable, 64-byte aligned, one per
// tile) are 2-D tensor maps of the cubes for the swizzled tiled load.
// Encodes the 2-D tensor map (CUtensorMap, 128 bytes, 64-byte aligned) of a cube
// [N][B]: boxes of 128 bytes of a row x box_rows rows, 128-byte swizzle (the
// tiled projection load uses 64 rows); false when the cube does not qualify
// (rows not a whole number of 16-byte units, base not 16-byte aligned).
bool encode_cube_map(pca_dtype dt, const void* cube, int64_t N, int B, void* map,
                     int box_rows = 64);
cudaError_t launch_project_grouped(const TileDesc* T, const void* maps, const ProjItem* items,
                                   const int* cta_items, int ctas, int maxB, int maxk,
                                   pca_dtype dt, cudaStream_t st);

}  // namespace gbpca
