/*
 * gbpca.h -- C ABI of the GB300 (sm_103a) Jacobi-PCA library.
 *
 * The library computes the four stages of the paper's PCA (Algorithm 1 of
 * "Jacobi-based PCA for hyperspectral dimensionality reduction", arXiv
 * 2403.18321): per-band mean removal, the covariance C = X^T X / (N-1)
 * (Sec. 4.2 stage 3), all eigen-pairs of C by cyclic Jacobi rotations
 * (Sec. 2, Eqs. 2-10) sorted in descending order (Sec. 4.2 stage 4.3), and
 * the projection of the centred cube onto the first k eigenvectors
 * (Algorithm 1, stages 5-6).
 *
 * Conventions shared by every entry point
 *   - The cube is N pixels x B bands, pixel-major ("band interleaved by
 *     pixel"): value (n, b) at cube[n*B + b], element type given by
 *     pca_dtype.  The paper's GPU code stores bands contiguously instead
 *     (Sec. 4.2 data initialisation); this ABI takes the manycore layout of
 *     Sec. 5 (image[i*BANDS + j]).
 *   - Every pointer argument except `info` (and the host-side arrays of the
 *     batched form) is a DEVICE pointer on the current CUDA device,
 *     allocated and owned by the caller.  The library allocates no device
 *     memory; all scratch lives in the caller's workspace of
 *     pca_workspace_size() bytes.  (Only a batch plan allocates, in host
 *     memory, together with its streams and events.)
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All work is enqueued on it; nothing synchronises unless
 *     `info` is non-NULL, in which case the call waits for the stream and
 *     fills *info.
 *   - Errors: argument errors are detected on the host before any launch
 *     and returned as PCA_ERR_ARG / PCA_ERR_WORKSPACE.  A failed launch
 *     returns PCA_ERR_CUDA.  Data-dependent outcomes (non-finite input,
 *     Jacobi not converged) are written to a status word in the workspace;
 *     they are returned only when `info` is given (else read them later
 *     with pca_read_info).  No entry point traps, asserts or hangs on the
 *     device.
 */
#ifndef GBPCA_H
#define GBPCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PCA_OK = 0,
  PCA_ERR_ARG = 1,        /* invalid argument (checked on the host)           */
  PCA_ERR_NOCONV = 2,     /* Jacobi hit sweeps_max; outputs hold the last iterate */
  PCA_ERR_NONFINITE = 3,  /* NaN or Inf in the cube; outputs are undefined      */
  PCA_ERR_TIMEOUT = 4,    /* a bounded device wait gave up                      */
  PCA_ERR_CUDA = 5,       /* a CUDA runtime call failed                          */
  PCA_ERR_WORKSPACE = 6   /* workspace too small or misaligned                   */
} pca_status;

typedef enum { PCA_F32 = 0, PCA_BF16 = 1, PCA_F16 = 2 } pca_dtype;

/*
 * Precision forms.
 *   PCA_PREC_P64: covariance accumulated in FP64 from exact products;
 *     FP32 Jacobi followed by five FP64 refinement iterations and three
 *     orthogonalisation steps (eigen-pairs separated from the rest of the
 *     spectrum by more than about 1e-5 of ||C|| come out FP64-accurate --
 *     eigenvalues below about 1e-3 ||C|| to about 1e-13 ||C|| absolute, the
 *     precision of the double-float products; tighter clusters keep
 *     FP32-level accuracy within the cluster, at least 1e-7 ||C|| absolute).
 *   PCA_PREC_P32: plain FP32 on the GPU (SIMT covariance, FP32 Jacobi, no
 *     refinement).
 *   PCA_PREC_MIX: covariance on the tensor cores from a two-term FP16
 *     split of the cube, shifted by a sampled band mean and scaled per band
 *     by a power of two (three products, FP32 accumulation in tensor
 *     memory), FP32 Jacobi stopped on the Frobenius test at
 *     max(tol, 1e-5), one refinement iteration and two orthogonalisation
 *     steps in double-float/FP64, and the projection on the tensor cores
 *     (the centred cube split the same way, V_k split into FP16 hi + lo,
 *     FP32 accumulation).  The split keeps 22 bits of every value; the
 *     remaining covariance error comes from the tensor cores' FP32
 *     accumulation, and vanishes for BF16/FP16 cubes, whose shifted values
 *     fit one FP16 and whose products and sums are then exact.  A value that
 *     leaves the scaled FP16 range makes the covariance (or the projection)
 *     be recomputed in FP32 on the SIMT cores (pca_info.cov_fallback,
 *     proj_fallback).
 */
typedef enum { PCA_PREC_P64 = 0, PCA_PREC_P32 = 1, PCA_PREC_MIX = 2 } pca_precision;

typedef struct {
  int status;        /* pca_status of the device-side work                    */
  int sweeps;        /* Jacobi sweeps run                                      */
  int refine_iters;  /* FP64 refinement iterations run                         */
  int steps;         /* Jacobi parallel steps run (sweeps x steps per sweep)   */
  double off_rel;    /* off(A)/||A||_F when the FP32 Jacobi stopped            */
  double tol_used;   /* the stop threshold the FP32 Jacobi applied             */
  double refine_res; /* largest |E_ij| of the last refinement correction (0 if none) */
  int cov_fallback;  /* MIX only: 1 if a scaled value left the FP16 range and the
                        covariance was recomputed in FP32 on the SIMT cores     */
  int proj_fallback; /* MIX only: the same for the tensor-core projection       */
} pca_info;

/*
 * Bytes of device workspace pca_fit needs for this problem.  Returns 0 for
 * arguments pca_fit would reject.  The workspace must be 256-byte aligned.
 */
size_t pca_workspace_size(int64_t N, int B, int k, pca_dtype dtype, pca_precision prec);

/*
 * pca_fit -- the whole hot path for one cube (Algorithm 1).
 *
 * cube       [N][B] device array of `dtype`, 16-byte aligned.
 * N          pixels, N >= 2 (C is divided by N-1, Sec. 4.2 stage 3).
 * B          bands, 2 <= B <= 256.
 * k          components to project onto, 1 <= k <= B.
 * tol        Jacobi stop factor (Sec. 2, "until all off-diagonal elements are
 *            smaller than the stop factor").  The FP32 Jacobi applies
 *            tau = max(tol, 2^-22) for P32 and P64, which stop when every
 *            |a_pq| <= tau sqrt(|a_pp a_qq|), and tau = max(tol, 1e-5) for
 *            MIX, which stops when off(A) <= tau ||A||_F (off: Frobenius
 *            norm of the off-diagonal part) and leaves the rest to the
 *            refinement; *info reports tau.  tol > 0.
 * sweeps_max maximum Jacobi sweeps, >= 1.
 * mu         [B] FP64 out: band means (Algorithm 1 stage 2).
 * eigvals    [B] FP64 out: eigenvalues of C, descending; equal values keep
 *            the order of the Jacobi's final diagonal positions.
 * eigvecs    [B][B] FP64 out, row-major: column j is the unit eigenvector
 *            of eigvals[j], its largest-magnitude entry (lowest row on
 *            ties) positive.
 * proj       [N][k] FP32 out: Q = (Y - 1 mu^T) eigvecs[:, :k].  May be NULL
 *            to skip the projection.
 * workspace  device scratch of ws_bytes >= pca_workspace_size(...) bytes.
 * stream     cudaStream_t as void*.
 * info       host pointer or NULL (see the conventions above).
 * Returns PCA_OK when the work was enqueued (and, with info, finished
 * without a data error), else a pca_status.
 */
int pca_fit(const void *cube, pca_dtype dtype, int64_t N, int B, int k, double tol,
            int sweeps_max, pca_precision prec, double *mu, double *eigvals,
            double *eigvecs, float *proj, void *workspace, size_t ws_bytes,
            void *stream, pca_info *info);

/*
 * The stages of pca_fit as separate calls (same conventions, same workspace
 * size as pca_fit for the same N, B, k, dtype, prec).
 *
 * pca_covariance -- Algorithm 1 stages 2-3: mu [B] and C = X^T X/(N-1),
 *   cov [B][B] FP64 row-major (full symmetric).  prec selects the
 *   covariance form (P64: FP64 accumulation; P32: FP32 SIMT; MIX: split-FP16
 *   tensor cores on per-band shifted and power-of-two scaled values).
 * pca_eigh -- Algorithm 1 stage 4 on a given symmetric matrix A [B][B] FP64
 *   (device): cyclic Jacobi (Eqs. 2-10), FP64 refinement (P32: none; MIX: one
 *   iteration and two orthogonalisation steps; P64: five and three),
 *   descending sort and sign rule; eigvals [B],
 *   eigvecs [B][B] as in pca_fit.  The workspace is that of pca_fit with
 *   N = 2 (any N works).
 * pca_project -- Algorithm 1 stages 5-6: proj [N][k] FP32 = (Y - 1 mu^T) V[:, :k]
 *   with mu [B] and eigvecs [B][B] FP64 on the device (narrowed to FP32).
 */
int pca_covariance(const void *cube, pca_dtype dtype, int64_t N, int B, pca_precision prec,
                   double *mu, double *cov, void *workspace, size_t ws_bytes, void *stream,
                   pca_info *info);
int pca_eigh(const double *A, int B, double tol, int sweeps_max, pca_precision prec,
             double *eigvals, double *eigvecs, void *workspace, size_t ws_bytes, void *stream,
             pca_info *info);
int pca_project(const void *cube, pca_dtype dtype, int64_t N, int B, int k, const double *mu,
                const double *eigvecs, float *proj, void *workspace, size_t ws_bytes,
                void *stream);

/*
 * pca_fit_host -- pca_fit of a cube that lives in host memory, with the
 * transfers overlapped with the stages.  (The paper's GPU code copies the
 * whole image before its first stage, Sec. 4.2 stage 1, and its times include
 * that copy.)  The cube is copied to the device in pixel ranges (at most 16,
 * each a multiple of 128 pixels and at least 65,536 pixels); the covariance of
 * a range runs as soon as its copy has landed, the ranges' means and
 * covariances are pooled exactly in FP64 (the rule of pca_combine_moments),
 * then the eigen-decomposition runs as in pca_fit, and the projection of each
 * range is copied back while the next range is projected.  The results equal
 * pca_fit's within its error bounds, not bit for bit (each range has its own
 * shift and accumulation runs).
 *   cube_host  [N][B] of dtype in host memory.  Page-locked memory
 *              (cudaHostAlloc, or torch's pin_memory) lets the copies run
 *              asynchronously; pageable memory works but makes them blocking.
 *   mu [B], eigvals [B], eigvecs [B][B] (FP64) and proj [N][k] (FP32): host
 *              memory, written as pca_fit writes them; proj may be NULL
 *              (no projection).
 *   cube_dev   device buffer of N*B elements of dtype, 16-byte aligned,
 *              receives the cube (its contents afterwards: the cube).
 *   proj_dev   device buffer of N*k floats, 16-byte aligned, receives the
 *              projection before it is copied back (NULL when proj is NULL).
 *   workspace  device, at least pca_fit_host_workspace_size() bytes, 256-byte
 *              aligned.
 * Everything is enqueued on `stream`; an internal copy stream joins it before
 * the call's last operation, so `stream` completes after every copy.  The host
 * buffers must stay valid (and cube_host unchanged) until then.  With info
 * non-NULL the call waits for `stream` and fills it (as pca_fit).  Return
 * codes as pca_fit; PCA_ERR_ARG also for a misaligned proj_dev or a NULL one
 * with proj given.
 */
size_t pca_fit_host_workspace_size(int64_t N, int B, int k, pca_dtype dtype, pca_precision prec);
int pca_fit_host(const void *cube_host, pca_dtype dtype, int64_t N, int B, int k, double tol,
                 int sweeps_max, pca_precision prec, double *mu, double *eigvals, double *eigvecs,
                 float *proj, void *cube_dev, float *proj_dev, void *workspace, size_t ws_bytes,
                 void *stream, pca_info *info);

/*
 * pca_bsq_to_bip -- band-sequential input.  The paper's GPU code stores each
 * band contiguously (Sec. 4.2, data initialisation: value (n, b) at
 * bsq[b*N + n]); every other entry point takes the pixel-major layout.  This
 * writes bip[n*B + b] = bsq[b*N + n] (both device arrays of `dtype`, N x B
 * elements, no alignment requirement, not overlapping), enqueued on `stream`;
 * the result is a cube for pca_fit.  Returns PCA_ERR_ARG for null pointers,
 * N < 1 or B < 1.
 */
int pca_bsq_to_bip(const void *bsq, pca_dtype dtype, int64_t N, int B, void *bip, void *stream);

/*
 * pca_combine_moments -- pooled band means and covariance of a cube whose
 * pixels are split into `parts` shards (one per GPU of a multi-GPU fit, or
 * several calls on one GPU); the exchange step of a pixel-sharded fit, which
 * the paper's manycore version performs over its two I/O halves (Sec. 5).
 * Shard g has n[g] >= 1 pixels (host array), mean mu_parts[g][B] and
 * covariance C_parts[g][B][B] (FP64, device, as pca_covariance returns them;
 * divided by n[g] - 1).  Writes mu [B] and C [B][B] (device) of the union by
 * the rule of Chan, Golub and LeVeque, in FP64, shards added in index order
 * (equal inputs give equal bits on every GPU).  1 <= parts <= 256,
 * 1 <= B <= 256, sum n >= 2, else PCA_ERR_ARG.  No workspace; enqueued on
 * `stream`, no synchronisation.
 */
int pca_combine_moments(int parts, const int64_t *n, const double *mu_parts,
                        const double *C_parts, int B, double *mu, double *C, void *stream);

/*
 * pca_shifted_sums / pca_moments_from_sums -- the same exchange as ONE sum of
 * a vector whose length does not grow with the number of shards, so that a
 * pixel-sharded fit needs a single all-reduce (the manycore version of the
 * paper likewise adds the partial products of its two I/O halves, Sec. 5).
 * Every shard uses the same shift s [B] (e.g. the mean of shard 0, sent to
 * the others first), which keeps the sums free of cancellation.
 *   sums layout (FP64, device, PCA_SUMS_LEN(B) = 1 + B + B(B+1)/2 values):
 *     sums[0]            n, the shard's pixel count (exact up to 2^53)
 *     sums[1 + b]        S1_b  = n (mu_b - s_b)
 *     sums[1 + B + t]    S2_ij = (n - 1) C_ij + n (mu_i - s_i)(mu_j - s_j),
 *                        t running over i <= j row by row (upper triangle)
 *   Summed over the shards these are n, sum (y - s) and sum (y - s)(y - s)^T of
 *   the whole cube.
 * pca_shifted_sums: n >= 1 (host), mu [B], C [B][B] (full symmetric, as
 *   pca_covariance returns them; 0 for a one-pixel shard) and s [B], all FP64
 *   on the device; writes sums.
 * pca_moments_from_sums: from the summed vector and the same s, writes
 *   mu = s + S1/n and C = (S2 - S1 S1^T / n) / (n - 1), full symmetric [B][B]
 *   (C is 0 when the summed n is below 2).
 * Outputs must not overlap the inputs.  1 <= B <= 256 and non-NULL pointers,
 * else PCA_ERR_ARG.  No workspace; enqueued on `stream`, no synchronisation.
 */
#define PCA_SUMS_LEN(B) (1 + (B) + (B) * ((B) + 1) / 2)
int pca_shifted_sums(int64_t n, const double *mu, const double *C, const double *s, int B,
                     double *sums, void *stream);
int pca_moments_from_sums(const double *sums, const double *s, int B, double *mu, double *C,
                          void *stream);

/*
 * pca_project_noalloc -- pca_project for callers that cannot allocate.  (No
 * counterpart in the paper.)  Some callers cannot hand the library a
 * workspace: code running while a CUDA graph is captured, plug-ins whose
 * host owns the device allocator, real-time loops that must not block in an
 * allocator.  This entry point computes the same proj [N][k] as pca_project
 * but keeps its two small intermediates (FP32 copies of mu and of the first
 * k eigenvectors) in a fixed device array that belongs to the library:
 * 256 + 256*32 floats (33,792 bytes), held on every GPU that loads the
 * library until the process exits.  It allocates and frees nothing.
 *   - Arguments as pca_project, without workspace; B*(k+1) above the array
 *     size (8,448 floats: up to 32 components at 256 bands, 131 at 64 bands)
 *     returns PCA_ERR_ARG.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the array.  Every call rewrites what it reads before
 *     reading it, but calls whose GPU work overlaps (other streams, other
 *     host threads) race on it: serialise them.
 *   - There is no workspace, hence no device status word: if a bounded wait
 *     of the projection kernel gives up (PCA_ERR_TIMEOUT in the other entry
 *     points), the rows it had not written are filled with NaN and the call
 *     still returns PCA_OK.  NaN in proj is the only sign of it.
 */
int pca_project_noalloc(const void *cube, pca_dtype dtype, int64_t N, int B, int k,
                        const double *mu, const double *eigvecs, float *proj, void *stream);

/*
 * pca_backward -- adjoint of the projection layer Q = (Y - 1 mu^T) V_k and,
 * optionally, of the eigenvalues (no counterpart in the paper: the backward
 * pass that makes the PCA usable as a differentiable layer).  With the
 * forward results of the same cube it computes, from first-order
 * perturbation theory of the symmetric eigenproblem,
 *     dV_k = X^T dproj,
 *     G    = F o (V^T [dV_k, 0]) + diag(deigvals),
 *            F_ij = 1/(lam_j - lam_i) for i != j with
 *            |lam_j - lam_i| > gap_eps |lam_1|, else 0 (degenerate gaps),
 *     S    = (V G V^T + (V G V^T)^T) / 2,
 *     dcube = (dproj - 1 mean_n dproj) V_k^T + 2/(N-1) X S.
 * cube, dtype, N, B, k  as in pca_fit.
 * mu [B], eigvals [B] (descending), eigvecs [B][B] (column j = vector j):
 *            the forward outputs, FP64, device.
 * dproj      [N][k] FP32 device, 16-byte aligned: gradient of proj.
 * deigvals   [B] FP64 device, or NULL: gradient of eigvals.
 * gap_eps    >= 0, finite.
 * dcube      [N][B] FP32 device out: gradient of the cube.
 * workspace  pca_backward_workspace_size(N, B, k) bytes, 256-byte aligned.
 * info       as in pca_fit (sweeps and refinement fields are 0).
 * Arithmetic: the pass over the cube accumulates in FP32 per CTA and adds the
 * partials in FP64; the B x B algebra is FP64; dcube is formed in FP32.
 */
size_t pca_backward_workspace_size(int64_t N, int B, int k);
int pca_backward(const void *cube, pca_dtype dtype, int64_t N, int B, int k, const double *mu,
                 const double *eigvals, const double *eigvecs, const float *dproj,
                 const double *deigvals, double gap_eps, float *dcube, void *workspace,
                 size_t ws_bytes, void *stream, pca_info *info);

/*
 * Batched form -- many independent cubes ("tiles": the tiles of a large
 * scene, or many scenes) fitted in one go, each tile exactly as pca_fit
 * would fit it (Algorithm 1 per tile; the paper fits one image at a time,
 * the batching is this library's).
 *
 * One persistent covariance launch walks a list of (tile, pixel range)
 * items balanced by bytes over the SMs; the Jacobi runs one thread-block
 * cluster per tile (tiles grouped by cluster shape, the groups on forked
 * streams); every small per-tile stage is one launch over all tiles; one
 * persistent projection launch walks (tile, pixel range) items.
 *
 * pca_tile   cube [N][B] device array of the batch's dtype, 16-byte aligned;
 *            N >= 2, 2 <= B <= 256, 1 <= k <= B; device outputs
 *            mu [B], eigvals [B], eigvecs [B][B] (FP64, as pca_fit) and
 *            proj [N][k] FP32 (NULL: no projection for this tile).
 * All tiles share dtype, precision, tol and sweeps_max (as in pca_fit).
 *
 * pca_batch_workspace_size  bytes of device workspace for these tiles on the
 *     current device (0 if a tile is invalid); 256-byte aligned.
 * pca_batch_create  checks every tile (the index of the first bad one goes
 *     to *bad_tile when not NULL), lays out the workspace, encodes the
 *     tensor maps of the cubes and writes the work lists and per-tile
 *     descriptors into the workspace with one synchronous host-to-device
 *     copy.  The plan lives in host memory and owns a CUDA stream and an
 *     event per Jacobi cluster shape (at most 24) plus one event (no device
 *     memory); the tiles' pointers and the workspace must stay valid for its
 *     life.  Returns PCA_OK, PCA_ERR_ARG,
 *     PCA_ERR_WORKSPACE or PCA_ERR_CUDA.
 * pca_batch_run  enqueues the fit of every tile on `stream`.  It launches
 *     kernels and records events only -- no allocation, copy or
 *     synchronisation -- so it can be captured into a CUDA graph and
 *     replayed (new input values between replays, same addresses and
 *     shapes).  Two runs of one plan must not overlap.
 * pca_batch_read_info  waits for `stream`, fills infos[ntiles] (NULL: not
 *     filled) and returns the status of the first tile that is not PCA_OK
 *     (PCA_OK if none).
 * pca_batch_destroy  releases the plan (its streams finish their work first).
 * pca_fit_batched  create + run + read_info (only when infos != NULL) +
 *     destroy.
 */
typedef struct {
  const void *cube;
  int64_t N;
  int B;
  int k;
  double *mu;
  double *eigvals;
  double *eigvecs;
  float *proj;
} pca_tile;
typedef struct pca_batch pca_batch;
size_t pca_batch_workspace_size(int ntiles, const pca_tile *tiles, pca_dtype dtype,
                                pca_precision prec);
int pca_batch_create(pca_batch **plan, int ntiles, const pca_tile *tiles, pca_dtype dtype,
                     double tol, int sweeps_max, pca_precision prec, void *workspace,
                     size_t ws_bytes, int *bad_tile);
int pca_batch_run(pca_batch *plan, void *stream);
int pca_batch_read_info(pca_batch *plan, void *stream, pca_info *infos);
void pca_batch_destroy(pca_batch *plan);
int pca_fit_batched(int ntiles, const pca_tile *tiles, pca_dtype dtype, double tol, int sweeps_max,
                    pca_precision prec, void *workspace, size_t ws_bytes, void *stream,
                    pca_info *infos);

/*
 * Tuning (no counterpart in the paper): process-wide parameters that trade
 * speed against accuracy (the accumulation run of the tensor-core covariance)
 * or shape the batched form's work split, chosen by the package's autotuner
 * and otherwise left at measured defaults.  They are read when a workspace is
 * sized, when pca_fit enqueues its work and when pca_batch_create plans a
 * batch (a plan keeps what it read); change them before sizing a workspace,
 * or a fit may find its workspace too small (PCA_ERR_WORKSPACE).  Host only.
 *
 * tc_slot_chunks   MIX covariance of FP32 cubes: the longest run of 32-pixel
 *                  chunks that one tensor-memory accumulator sums in FP32
 *                  before it is written out and added in FP64 (1..1024,
 *                  default 4).  The FP32 accumulation error grows linearly with
 *                  the run (measured ||dC||_2 / lambda_1 on the 610x340x103
 *                  scene: 3.0e-7 at 2 chunks, 6.1e-7 at 4, 1.2e-6 at 8, 2.5e-6
 *                  at 16, 8.0e-6 at 64); shorter runs write more partials.  At
 *                  4 chunks every top-10 eigenvalue of the two paper-shaped
 *                  scene cubes is within 1.2e-5 of its own size (2.6e-5 at 8).
 * tc_slot_chunks_batch  the same for the FP32 tiles of the batched form
 *                  (default 8: its tiles' top eigenvalues stay within 1.1e-6
 *                  there, and shorter runs cost it 20% more time).
 * tc_slot_chunks_f16, tc_slot_chunks_bf16  the same for FP16 and BF16 cubes
 *                  (defaults 64 and 1024).  Their shifted values fit one FP16
 *                  each, the products are exact, and so are the FP32 sums while
 *                  they stay below 2^24 units of the product grid: measured on
 *                  the 2048 x 2048 x 224 planted cube against the FP64
 *                  covariance, BF16 (8-bit values) is exact at every run length,
 *                  FP16 (11-bit values) at 64 chunks but not at 256 (3e-7).
 * batch_jacobi_ctas[i]  batched form: CTAs of the Jacobi cluster of a tile
 *                  with 32i < B' <= 32(i+1) bands (B' = B rounded up to even);
 *                  0 = the fewest that hold the matrix (default), otherwise
 *                  raised to the fewest that hold it, at most 8.
 * batch_cov_tc_fixed, batch_proj_fixed  batched form: fixed cost of one
 *                  32-pixel covariance chunk (MIX) / one 64-pixel projection
 *                  chunk, in units of the per-band cost of a chunk; the work
 *                  is split over the CTAs by this cost model (defaults 464 and
 *                  223, measured).
 * batch_cov_simt_fixed  the same for the SIMT covariance (P32, P64), in units
 *                  of one product per pixel (default 13900).
 * batch_simt_items_per_sm  SIMT covariance work items per SM (1..64, default 4).
 * proj_tc_stages, proj_tc_raw_stages  tensor-core projection (MIX): depth of
 *                  the converted-operand ring (2..6) and of the TMA ring of raw
 *                  cube chunks (2..8); 0 = as many as shared memory holds, with
 *                  3 operand stages first (default).
 * stream_sms_reserve  SMs (0..64, default 0) that the single-cube tensor-core
 *                  covariance and projection (MIX) leave free: their persistent
 *                  grids hold one CTA per SM and would otherwise wait for the
 *                  SMs a Jacobi cluster of a second fit, enqueued on another
 *                  stream, holds (8 for more than 128 bands).  Set it when fits
 *                  run two at a time, before sizing their workspaces
 *                  (pca_workspace_size reads it; a smaller workspace gives
 *                  PCA_ERR_WORKSPACE).
 *
 * pca_tuning_defaults fills *t with the defaults.  pca_set_tuning installs *t
 * (NULL: the defaults); PCA_ERR_ARG, and no change, for a value out of range.
 * pca_get_tuning copies the current values.
 */
typedef struct {
  int tc_slot_chunks;
  int tc_slot_chunks_f16;
  int tc_slot_chunks_bf16;
  int batch_jacobi_ctas[8];
  double batch_cov_tc_fixed;
  double batch_proj_fixed;
  double batch_cov_simt_fixed;
  int batch_simt_items_per_sm;
  int proj_tc_stages;
  int proj_tc_raw_stages;
  int tc_slot_chunks_batch;
  int stream_sms_reserve;
} pca_tuning;
void pca_tuning_defaults(pca_tuning *t);
int pca_set_tuning(const pca_tuning *t);
int pca_get_tuning(pca_tuning *t);

/*
 * Waits for `stream` and copies the device-side outcome of the last
 * pca_fit (or pca_backward) that used `workspace` into *info.  Returns
 * info->status.
 */
int pca_read_info(const void *workspace, void *stream, pca_info *info);

/* Static description of a status code. */
const char *pca_status_string(int status);

/* ABI version (major*100 + minor). */
int pca_version(void);

/* ---- instrumentation (no counterpart in the paper; used by the benchmark) */

/* Number of kernels one pca_fit enqueues for this precision form when it
 * projects onto k components (k = 0: no projection). */
int pca_kernel_launches(pca_precision prec, int k);

/* Number of kernels one pca_batch_run of this plan enqueues. */
int pca_batch_kernel_launches(const pca_batch *plan);

/* SMs (CTAs of one cluster) the Jacobi stage occupies for B bands; 0 if B is invalid. */
int pca_jacobi_sms(int B);

/* The shape of the plan pca_batch_create would make for these tiles under the
 * current tuning, without a workspace or a device: counts[0] covariance work
 * items, counts[1] projection work items, counts[2] Jacobi launches (one per
 * cluster shape), counts[3] CTAs of the largest Jacobi cluster.  Returns
 * PCA_ERR_ARG for invalid tiles (no pointer of a tile is read; every tile
 * counts as projected). */
int pca_batch_plan_counts(int ntiles, const pca_tile *tiles, pca_dtype dtype, pca_precision prec,
                          int *counts);

/* CTAs of the batched form's Jacobi cluster for a B-band tile when the tuning
 * asks for `request` (0: the fewest that hold the matrix; else raised to the
 * fewest that hold it, at most 8); 0 if B or request is invalid. */
int pca_batch_jacobi_ctas(int B, int request);

/*
 * Per-stage timing.  pca_profile(1) makes every later pca_fit (and
 * pca_batch_run, one record per run) on the calling host thread record CUDA
 * events on its stream around its eight stages
 * (covariance, covariance finalisation, Jacobi, a fourth slot that is always
 * 0 because the Jacobi kernel rotates V itself, compaction, refinement,
 * sort/sign, projection), up to 256 fits; pca_profile(0) stops.
 * Both reset the record list and return the stage count (8).
 * pca_profile_collect waits for the recorded events and writes, per fit
 * r < max_records, the stage durations in ms to ms[r*8 + i]; returns the
 * number of fits written.  Host memory only; no allocation on the device.
 */
int pca_profile(int enable);
int pca_profile_collect(float *ms, int max_records);

#ifdef __cplusplus
}
#endif

#endif /* GBPCA_H */
