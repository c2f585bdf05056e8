// api.cu -- the C ABI of include/gbpca.h: argument checks, workspace
// layout and the launch sequence of the four PCA stages (Algorithm 1).
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "common.cuh"

namespace gbpca {

namespace {

constexpr int kMaxSweeps = 100;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

__global__ void k_header_init(DevHeader* h, int refine_iters, float tol32) {
  DevHeader z;
  memset(&z, 0, sizeof(z));
  z.refine_iters = refine_iters;
  z.tol_used = tol32;
  z.dummy_slot = -1;
  *h = z;
}

}  // namespace

// FP32 cubes: 4 chunks = 128 pixels per slot by default.  The covariance error
// grows linearly with the slot length (||dC||_2 / lambda_1 on the 103-band scene:
// 6.1e-7 at 4 chunks, half the plain FP32 form's, 1.2e-6 at 8, 8.0e-6 at 64); at
// 4 chunks every top-10 eigenvalue of both paper-shaped scenes is within 2e-5
// of its own size.  16-bit cubes: products and sums
// are exact while the sums stay within FP32's 24 bits -- FP16 64 chunks, BF16
// (8-bit values) 1024 chunks (equal to the FP64 covariance on the planted cube).
int tc_slot_chunks(pca_dtype dt) {
  const pca_tuning t = tuning();
  return dt == PCA_F32 ? t.tc_slot_chunks
                       : (dt == PCA_F16 ? t.tc_slot_chunks_f16 : t.tc_slot_chunks_bf16);
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return 148;
  return sms;
}

bool args_ok(const void* cube, pca_dtype dt, int64_t N, int B, int k, double tol,
             int sweeps_max, pca_precision prec) {
  if (!cube) return false;
  if (dt != PCA_F32 && dt != PCA_BF16 && dt != PCA_F16) return false;
  if (prec != PCA_PREC_P64 && prec != PCA_PREC_P32 && prec != PCA_PREC_MIX) return false;
  if (N < 2 || B < 2 || B > kMaxB || k < 1 || k > B) return false;
  if (!(tol > 0.0) || !std::isfinite(tol)) return false;
  if (sweeps_max < 1 || sweeps_max > kMaxSweeps) return false;
  if (((uintptr_t)cube) % 16 != 0) return false;
  if (prec == PCA_PREC_MIX && !syrk_tc_supported(B)) return false;
  return true;
}

namespace {

// ---- optional per-stage CUDA-event timing (profiling entry points of gbpca.h)
constexpr int kProfStages = 8;  // cov, cov_finalize, jacobi, (empty), compact, refine, sort, project
constexpr int kProfRecords = 256;
struct ProfState {
  bool on = false;
  int nrec = 0;
  cudaEvent_t ev[kProfRecords][kProfStages + 1] = {};
  bool used[kProfRecords][kProfStages + 1] = {};
};
thread_local ProfState g_prof;

}  // namespace

StageMark::StageMark(cudaStream_t s) : st(s), rec(-1) {
  if (g_prof.on && g_prof.nrec < kProfRecords) rec = g_prof.nrec++;
}
void StageMark::mark(int i) {
  if (rec < 0) return;
  cudaEvent_t& e = g_prof.ev[rec][i];
  if (!e) cudaEventCreate(&e);
  cudaEventRecord(e, st);
  g_prof.used[rec][i] = true;
}

namespace {

}  // namespace

Layout make_layout(int64_t N, int B, int k, pca_dtype dt, pca_precision prec, int num_sms) {
  Layout L{};
  const int Bp = round_even(B);
  if (prec == PCA_PREC_MIX) {
    // one persistent CTA per SM, less the SMs left to a concurrent fit's Jacobi
    const int use = std::max(1, num_sms - tuning().stream_sms_reserve);
    L.tc_ctas = (int)std::min<int64_t>(use, std::max<int64_t>(1, (N + 127) / 128));
    // every CTA gets the same number of slots, each at most tc_slot_chunks() long
    const int64_t nchunk = (N + 31) / 32, cap = tc_slot_chunks(dt);
    const int64_t per_cta = (nchunk + L.tc_ctas - 1) / L.tc_ctas;
    L.partials = L.tc_ctas * (int)((per_cta + cap - 1) / cap);
    L.s2_bytes_el = 4;
  } else {
    L.partials = (int)std::min<int64_t>(kMaxPartials, std::max<int64_t>(1, (N + 255) / 256));
    L.s2_bytes_el = prec == PCA_PREC_P64 ? 8 : 4;
  }
  L.s2_elems = B * (B + 1) / 2;
  const size_t BB8 = sizeof(double) * (size_t)B * B;
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o = align256(o + bytes); return at; };
  L.hdr = take(sizeof(DevHeader));
  L.shift = take(sizeof(float) * B);
  L.escale = take(sizeof(int) * B);
  L.s1_part = take(sizeof(double) * (size_t)L.partials * B);
  L.s2_part = take((size_t)L.s2_bytes_el * L.partials * L.s2_elems);
  L.dvec = take(sizeof(double) * B);
  L.cov = take(BB8);
  L.cdf = take(BB8);
  L.rank = take(sizeof(int) * B);
  L.sgn = take(sizeof(double) * B);
  L.diag32 = take(sizeof(float) * Bp);
  L.v32 = take(sizeof(float) * (size_t)Bp * Bp);
  L.lam = take(sizeof(double) * B);
  L.vc = take(BB8);
  L.w = take(BB8);
  L.s = take(BB8);
  L.r = take(BB8);
  L.e = take(BB8);
  L.vk = take(sizeof(float) * (size_t)B * k);
  L.muf = take(sizeof(float) * B);
  L.ptc_shift = take(sizeof(float) * 256);
  L.ptc_escale = take(sizeof(int) * 256);
  L.ptc_planes = take(project_tc_planes_bytes(B, k));
  L.ptc_colscale = take(sizeof(float) * 128);
  L.ptc_corr = take(sizeof(float) * 128);
  L.total = o;
  return L;
}

namespace {

struct BwdLayout {
  size_t hdr, dv_part, dqs_part, dVk, Gk, dA, S32, vk32, mdq, mu32, xmax_part, dqmax_part, ascale,
      anshift, bop, fcol, total;
  int parts;
};

BwdLayout make_bwd_layout(int64_t N, int B, int k, int num_sms) {
  BwdLayout L{};
  L.parts = (int)std::min<int64_t>(num_sms, std::max<int64_t>(1, (N + 63) / 64));
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o = align256(o + bytes); return at; };
  L.hdr = take(sizeof(DevHeader));
  L.dv_part = take(sizeof(float) * (size_t)L.parts * B * k);
  L.dqs_part = take(sizeof(float) * (size_t)L.parts * k);
  L.dVk = take(sizeof(double) * (size_t)B * k);
  L.Gk = take(sizeof(double) * (size_t)B * k);
  L.dA = take(sizeof(double) * (size_t)B * B);
  L.S32 = take(sizeof(float) * (size_t)B * B);
  L.vk32 = take(sizeof(float) * (size_t)B * k);
  L.mdq = take(sizeof(float) * (size_t)k);
  L.mu32 = take(sizeof(float) * (size_t)B);
  L.xmax_part = take(sizeof(float) * (size_t)L.parts * B);
  L.dqmax_part = take(sizeof(float) * (size_t)L.parts * k);
  const int B32 = (B + 31) & ~31;                 // the dQ segment of K starts here
  L.ascale = take(sizeof(float) * (size_t)(B32 + k));
  L.anshift = take(sizeof(float) * (size_t)(B32 + k));
  L.bop = take(bwd_bop_bytes(B, k));
  L.fcol = take(sizeof(float) * (size_t)2 * B);
  L.total = o;
  return L;
}

bool bwd_args_ok(const void* cube, pca_dtype dt, int64_t N, int B, int k, double gap_eps) {
  static const float kDummy[4] = {0.f, 0.f, 0.f, 0.f};
  return args_ok(cube ? cube : kDummy, dt, N, B, k, 1.0, 1, PCA_PREC_P32) && gap_eps >= 0.0 &&
         std::isfinite(gap_eps);
}

}  // namespace

}  // namespace gbpca

using namespace gbpca;

#define GB_CK(x)                                   \
  do {                                             \
    if ((x) != cudaSuccess) return PCA_ERR_CUDA;   \
  } while (0)

extern "C" {

size_t pca_workspace_size(int64_t N, int B, int k, pca_dtype dtype, pca_precision prec) {
  static const float kDummy[4] = {0.f, 0.f, 0.f, 0.f};
  if (!args_ok(kDummy, dtype, N, B, k, 1.0, 1, prec)) return 0;
  return make_layout(N, B, k, dtype, prec, device_sms()).total;
}

int pca_read_info(const void* workspace, void* stream, pca_info* info) {
  if (!workspace || !info) return PCA_ERR_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return PCA_ERR_CUDA;
  DevHeader h;
  if (cudaMemcpy(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PCA_ERR_CUDA;
  info->status = h.status;
  info->sweeps = h.sweeps;
  info->refine_iters = h.refine_iters;
  info->steps = h.steps;
  info->off_rel = h.off_rel;
  info->tol_used = h.tol_used;
  info->refine_res = h.refine_res;
  info->cov_fallback = h.cov_range != 0 ? 1 : 0;
  info->proj_fallback = h.proj_range != 0 ? 1 : 0;
  return info->status;
}

}  // extern "C"

namespace gbpca {
namespace {

struct Ptrs {
  DevHeader* hdr;
  float* shift;
  int* escale;
  double* s1p;
  void* s2p;
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
  float* ptc_shift;
  int* ptc_escale;
  unsigned char* ptc_planes;
  float* ptc_colscale;
  float* ptc_corr;
};

Ptrs carve(void* workspace, const Layout& L) {
  char* ws = static_cast<char*>(workspace);
  Ptrs p;
  p.hdr = reinterpret_cast<DevHeader*>(ws + L.hdr);
  p.shift = reinterpret_cast<float*>(ws + L.shift);
  p.escale = reinterpret_cast<int*>(ws + L.escale);
  p.s1p = reinterpret_cast<double*>(ws + L.s1_part);
  p.s2p = ws + L.s2_part;
  p.dvec = reinterpret_cast<double*>(ws + L.dvec);
  p.C = reinterpret_cast<double*>(ws + L.cov);
  p.cdf = reinterpret_cast<float2*>(ws + L.cdf);
  p.rank = reinterpret_cast<int*>(ws + L.rank);
  p.sgn = reinterpret_cast<double*>(ws + L.sgn);
  p.diag32 = reinterpret_cast<float*>(ws + L.diag32);
  p.v32 = reinterpret_cast<float*>(ws + L.v32);
  p.lam = reinterpret_cast<double*>(ws + L.lam);
  p.vc = reinterpret_cast<float2*>(ws + L.vc);
  p.w = reinterpret_cast<float2*>(ws + L.w);
  p.s = reinterpret_cast<float2*>(ws + L.s);
  p.g = reinterpret_cast<float2*>(ws + L.r);
  p.e = reinterpret_cast<float2*>(ws + L.e);
  p.vk = reinterpret_cast<float*>(ws + L.vk);
  p.muf = reinterpret_cast<float*>(ws + L.muf);
  p.ptc_shift = reinterpret_cast<float*>(ws + L.ptc_shift);
  p.ptc_escale = reinterpret_cast<int*>(ws + L.ptc_escale);
  p.ptc_planes = reinterpret_cast<unsigned char*>(ws + L.ptc_planes);
  p.ptc_colscale = reinterpret_cast<float*>(ws + L.ptc_colscale);
  p.ptc_corr = reinterpret_cast<float*>(ws + L.ptc_corr);
  return p;
}

// stages 2-3 of Algorithm 1: band means and covariance in one pass over the cube
cudaError_t run_cov(const void* cube, pca_dtype dt, int64_t N, int B, pca_precision prec,
                    const Layout& L, const Ptrs& P, double* mu, cudaStream_t st, StageMark& pm) {
  cudaError_t e;
  pm.mark(0);
  if (prec == PCA_PREC_MIX) {
    e = launch_syrk_tc(cube, dt, N, B, P.shift, P.escale, P.s1p, (float*)P.s2p, L.partials,
                       L.tc_ctas, P.hdr, st);
    if (e != cudaSuccess) return e;
    // a value outside the scaled FP16 range: the SIMT form recomputes the partials
    // (its CTAs return at once when the flag is clear)
    e = launch_syrk_simt(cube, dt, N, B, false, P.shift, P.s1p, P.s2p, L.partials, st,
                         &P.hdr->cov_range, P.escale);
  } else {
    e = launch_syrk_simt(cube, dt, N, B, prec == PCA_PREC_P64, P.shift, P.s1p, P.s2p, L.partials, st);
  }
  if (e != cudaSuccess) return e;
  pm.mark(1);
  return launch_cov_finalize(P.shift, P.s1p, P.s2p, L.s2_bytes_el == 8, L.partials, N, B, mu, P.C,
                             P.muf, P.dvec, P.hdr, st, prec == PCA_PREC_MIX ? P.escale : nullptr);
}

// stage 4: Jacobi (rotating V), FP64 refinement, sort and sign rule
cudaError_t run_eigh(const double* A, int B, float tol32, int sweeps_max, pca_precision prec,
                     int k, const Ptrs& P, double* eigvals, double* eigvecs, cudaStream_t st,
                     StageMark& pm) {
  cudaError_t e;
  pm.mark(2);
  if ((e = launch_jacobi_cluster(A, B, tol32, sweeps_max, relative_stop(prec), P.diag32, P.v32,
                                 P.hdr, st)) != cudaSuccess)
    return e;
  pm.mark(3);
  pm.mark(4);
  if ((e = launch_compact(P.diag32, P.v32, B, P.hdr, P.lam, P.vc, st)) != cudaSuccess) return e;
  pm.mark(5);
  const int iters = refine_iterations(prec);
  if (iters > 0 && (e = launch_to_df(A, P.cdf, B * B, st)) != cudaSuccess) return e;
  // V alternates between two buffers, so that no step copies it back
  float2* v = P.vc;
  float2* other = P.w;
  for (int it = 0; it < iters; ++it) {
    if ((e = launch_refine(P.cdf, B, v, other, P.lam, P.s, P.g, P.e, P.hdr, refine_max_angle(prec),
                           st)) != cudaSuccess)
      return e;
    std::swap(v, other);
  }
  for (int it = 0; it < ortho_steps(prec); ++it) {
    if ((e = launch_orthonormalize(v, other, B, P.g, P.e, st)) != cudaSuccess) return e;
    std::swap(v, other);
  }
  pm.mark(6);
  return launch_sort_sign(P.lam, v, B, k, eigvals, eigvecs, P.vk, P.rank, P.sgn, st);
}

}  // namespace
}  // namespace gbpca

extern "C" {

int pca_fit(const void* cube, pca_dtype dt, int64_t N, int B, int k, double tol, int sweeps_max,
            pca_precision prec, double* mu, double* eigvals, double* eigvecs, float* proj,
            void* workspace, size_t ws_bytes, void* stream, pca_info* info) {
  if (!args_ok(cube, dt, N, B, k, tol, sweeps_max, prec)) return PCA_ERR_ARG;
  if (!mu || !eigvals || !eigvecs) return PCA_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace) % 256 != 0) return PCA_ERR_WORKSPACE;
  const Layout L = make_layout(N, B, k, dt, prec, device_sms());
  if (ws_bytes < L.total) return PCA_ERR_WORKSPACE;
  const Ptrs P = carve(workspace, L);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const float tol32 = std::max((float)tol, stop_floor(prec));
  StageMark pm(st);
  k_header_init<<<1, 1, 0, st>>>(P.hdr, refine_iterations(prec), tol32);
  GB_CK(cudaGetLastError());
  GB_CK(run_cov(cube, dt, N, B, prec, L, P, mu, st, pm));
  GB_CK(run_eigh(P.C, B, tol32, sweeps_max, prec, k, P, eigvals, eigvecs, st, pm));
  // stages 5-6: projection onto the first k eigenvectors (MIX: tensor cores, with
  // the FP32 SIMT form as the guarded fallback for values outside their range)
  pm.mark(7);
  if (proj && prec == PCA_PREC_MIX) {
    GB_CK(launch_project_tc(cube, dt, N, B, k, mu, eigvecs, proj, P.ptc_shift, P.ptc_escale,
                            P.ptc_planes, P.ptc_colscale, P.ptc_corr, P.hdr, st));
    GB_CK(launch_project(cube, dt, N, B, k, P.muf, P.vk, proj, st, P.hdr, &P.hdr->proj_range));
  } else if (proj) {
    GB_CK(launch_project(cube, dt, N, B, k, P.muf, P.vk, proj, st, P.hdr));
  }
  pm.mark(8);
  if (info) return pca_read_info(workspace, stream, info);
  return PCA_OK;
}

int pca_covariance(const void* cube, pca_dtype dt, int64_t N, int B, pca_precision prec,
                   double* mu, double* cov, void* workspace, size_t ws_bytes, void* stream,
                   pca_info* info) {
  if (!args_ok(cube, dt, N, B, 1, 1.0, 1, prec) || !mu || !cov) return PCA_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace) % 256 != 0) return PCA_ERR_WORKSPACE;
  const Layout L = make_layout(N, B, 1, dt, prec, device_sms());
  if (ws_bytes < L.total) return PCA_ERR_WORKSPACE;
  const Ptrs P = carve(workspace, L);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  StageMark pm(st);
  k_header_init<<<1, 1, 0, st>>>(P.hdr, 0, 0.f);
  GB_CK(cudaGetLastError());
  GB_CK(run_cov(cube, dt, N, B, prec, L, P, mu, st, pm));
  GB_CK(cudaMemcpyAsync(cov, P.C, sizeof(double) * (size_t)B * B, cudaMemcpyDeviceToDevice, st));
  if (info) return pca_read_info(workspace, stream, info);
  return PCA_OK;
}

int pca_eigh(const double* A, int B, double tol, int sweeps_max, pca_precision prec,
             double* eigvals, double* eigvecs, void* workspace, size_t ws_bytes, void* stream,
             pca_info* info) {
  static const float kDummy[4] = {0.f, 0.f, 0.f, 0.f};
  if (!A || !eigvals || !eigvecs || !args_ok(kDummy, PCA_F32, 2, B, 1, tol, sweeps_max, prec))
    return PCA_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace) % 256 != 0) return PCA_ERR_WORKSPACE;
  const Layout L = make_layout(2, B, 1, PCA_F32, prec, device_sms());
  if (ws_bytes < L.total) return PCA_ERR_WORKSPACE;
  const Ptrs P = carve(workspace, L);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const float tol32 = std::max((float)tol, stop_floor(prec));
  StageMark pm(st);
  k_header_init<<<1, 1, 0, st>>>(P.hdr, refine_iterations(prec), tol32);
  GB_CK(cudaGetLastError());
  GB_CK(run_eigh(A, B, tol32, sweeps_max, prec, 1, P, eigvals, eigvecs, st, pm));
  if (info) return pca_read_info(workspace, stream, info);
  return PCA_OK;
}

int pca_project(const void* cube, pca_dtype dt, int64_t N, int B, int k, const double* mu,
                const double* eigvecs, float* proj, void* workspace, size_t ws_bytes,
                void* stream) {
  if (!args_ok(cube, dt, N, B, k, 1.0, 1, PCA_PREC_P32) || !mu || !eigvecs || !proj)
    return PCA_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace) % 256 != 0) return PCA_ERR_WORKSPACE;
  const Layout L = make_layout(N, B, k, dt, PCA_PREC_P32, device_sms());
  if (ws_bytes < L.total) return PCA_ERR_WORKSPACE;
  const Ptrs P = carve(workspace, L);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GB_CK(launch_narrow_inputs(mu, eigvecs, B, k, P.muf, P.vk, st));
  GB_CK(launch_project(cube, dt, N, B, k, P.muf, P.vk, proj, st, P.hdr));
  return PCA_OK;
}

}  // extern "C"

namespace gbpca {
namespace {

// ---- host-resident cubes: the pixel ranges whose copies overlap the stages
constexpr int kHostRanges = 16;
constexpr int64_t kHostMinRange = 65536;

struct HostLayout {
  int64_t range = 0;     // pixels per range (the last one takes the rest)
  int parts = 0;
  Layout L{};            // the fit's layout, sized for the largest range
  size_t mu_parts = 0, C_parts = 0, mu = 0, ev = 0, V = 0, total = 0;
};

HostLayout make_host_layout(int64_t N, int B, int k, pca_dtype dt, pca_precision prec, int sms) {
  HostLayout H;
  int64_t r = std::max<int64_t>((N + kHostRanges - 1) / kHostRanges, kHostMinRange);
  r = (r + 127) & ~int64_t(127);            // 16-byte aligned range starts
  H.range = std::min(r, N);
  H.parts = (int)((N + H.range - 1) / H.range);
  if (H.parts > 1 && N - (int64_t)(H.parts - 1) * H.range < 2) --H.parts;   // no 1-pixel range
  const int64_t last = N - (int64_t)(H.parts - 1) * H.range;
  H.L = make_layout(std::max(H.range, last), B, k, dt, prec, sms);
  size_t o = align256(H.L.total);
  auto take = [&](size_t bytes) { const size_t at = o; o = align256(o + bytes); return at; };
  H.mu_parts = take(sizeof(double) * (size_t)H.parts * B);
  H.C_parts = take(sizeof(double) * (size_t)H.parts * B * B);
  H.mu = take(sizeof(double) * B);
  H.ev = take(sizeof(double) * B);
  H.V = take(sizeof(double) * (size_t)B * B);
  H.total = o;
  return H;
}

}  // namespace
}  // namespace gbpca

extern "C" {

size_t pca_fit_host_workspace_size(int64_t N, int B, int k, pca_dtype dtype, pca_precision prec) {
  static const float kDummy[4] = {0.f, 0.f, 0.f, 0.f};
  if (!args_ok(kDummy, dtype, N, B, k, 1.0, 1, prec)) return 0;
  return make_host_layout(N, B, k, dtype, prec, device_sms()).total;
}

int pca_fit_host(const void* cube_host, pca_dtype dt, int64_t N, int B, int k, double tol,
                 int sweeps_max, pca_precision prec, double* mu, double* eigvals, double* eigvecs,
                 float* proj, void* cube_dev, float* proj_dev, void* workspace, size_t ws_bytes,
                 void* stream, pca_info* info) {
  if (!cube_host || !args_ok(cube_dev, dt, N, B, k, tol, sweeps_max, prec)) return PCA_ERR_ARG;
  if (!mu || !eigvals || !eigvecs) return PCA_ERR_ARG;
  if (proj && (!proj_dev || ((uintptr_t)proj_dev) % 16 != 0)) return PCA_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace) % 256 != 0) return PCA_ERR_WORKSPACE;
  const HostLayout H = make_host_layout(N, B, k, dt, prec, device_sms());
  if (ws_bytes < H.total) return PCA_ERR_WORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  const Ptrs P = carve(workspace, H.L);
  double* mu_parts = reinterpret_cast<double*>(ws + H.mu_parts);
  double* C_parts = reinterpret_cast<double*>(ws + H.C_parts);
  double* mu_d = reinterpret_cast<double*>(ws + H.mu);
  double* ev_d = reinterpret_cast<double*>(ws + H.ev);
  double* V_d = reinterpret_cast<double*>(ws + H.V);
  const size_t el = dt == PCA_F32 ? 4 : 2;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the copies run on a stream of their own, ordered against `st` by events
  cudaStream_t cs = nullptr;
  GB_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  std::vector<cudaEvent_t> evs;
  auto event = [&](cudaEvent_t* e) {
    const cudaError_t r = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
    if (r == cudaSuccess) evs.push_back(*e);
    return r;
  };
  // the events and the copy stream are released once their work is done
  auto finish = [&](int rc) {
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
    cudaStreamDestroy(cs);
    return rc;
  };
#define GB_HK(x)                                            \
  do {                                                      \
    if ((x) != cudaSuccess) return finish(PCA_ERR_CUDA);    \
  } while (0)
  const float tol32 = std::max((float)tol, stop_floor(prec));
  StageMark pm(st);
  cudaEvent_t start;
  GB_HK(event(&start));
  GB_HK(cudaEventRecord(start, st));          // the copies follow earlier work on `st`
  GB_HK(cudaStreamWaitEvent(cs, start, 0));
  k_header_init<<<1, 1, 0, st>>>(P.hdr, refine_iterations(prec), tol32);
  GB_HK(cudaGetLastError());
  // stages 1-3 per pixel range, each as soon as its bytes are on the device
  std::vector<int64_t> counts((size_t)H.parts);
  for (int c = 0; c < H.parts; ++c) {
    const int64_t p0 = (int64_t)c * H.range;
    const int64_t n = c + 1 < H.parts ? H.range : N - p0;
    counts[(size_t)c] = n;
    const unsigned char* src = static_cast<const unsigned char*>(cube_host) + (size_t)p0 * B * el;
    unsigned char* dst = static_cast<unsigned char*>(cube_dev) + (size_t)p0 * B * el;
    GB_HK(cudaMemcpyAsync(dst, src, (size_t)n * B * el, cudaMemcpyHostToDevice, cs));
    cudaEvent_t in;
    GB_HK(event(&in));
    GB_HK(cudaEventRecord(in, cs));
    GB_HK(cudaStreamWaitEvent(st, in, 0));
    const Layout Lc = make_layout(n, B, k, dt, prec, device_sms());
    Ptrs Pc = carve(workspace, Lc);
    Pc.C = C_parts + (size_t)c * B * B;
    GB_HK(run_cov(dst, dt, n, B, prec, Lc, Pc, mu_parts + (size_t)c * B, st, pm));
  }
  // the ranges' moments pooled exactly (Chan, Golub and LeVeque), then stage 4
  if (pca_combine_moments(H.parts, counts.data(), mu_parts, C_parts, B, mu_d, P.C, st) != PCA_OK)
    return finish(PCA_ERR_CUDA);
  GB_HK(run_eigh(P.C, B, tol32, sweeps_max, prec, k, P, ev_d, V_d, st, pm));
  GB_HK(launch_narrow_inputs(mu_d, V_d, B, k, P.muf, P.vk, st));
  GB_HK(cudaMemcpyAsync(mu, mu_d, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  GB_HK(cudaMemcpyAsync(eigvals, ev_d, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  GB_HK(cudaMemcpyAsync(eigvecs, V_d, sizeof(double) * B * B, cudaMemcpyDeviceToHost, st));
  // stages 5-6 per range, each range's rows copied back while the next is projected
  pm.mark(7);
  if (proj) {
    for (int c = 0; c < H.parts; ++c) {
      const int64_t p0 = (int64_t)c * H.range, n = counts[(size_t)c];
      const unsigned char* cube_c = static_cast<const unsigned char*>(cube_dev) + (size_t)p0 * B * el;
      float* q = proj_dev + (size_t)p0 * k;
      if (prec == PCA_PREC_MIX) {
        GB_HK(launch_project_tc(cube_c, dt, n, B, k, mu_d, V_d, q, P.ptc_shift, P.ptc_escale,
                                P.ptc_planes, P.ptc_colscale, P.ptc_corr, P.hdr, st));
        GB_HK(launch_project(cube_c, dt, n, B, k, P.muf, P.vk, q, st, P.hdr, &P.hdr->proj_range));
      } else {
        GB_HK(launch_project(cube_c, dt, n, B, k, P.muf, P.vk, q, st, P.hdr));
      }
      cudaEvent_t out;
      GB_HK(event(&out));
      GB_HK(cudaEventRecord(out, st));
      GB_HK(cudaStreamWaitEvent(cs, out, 0));
      GB_HK(cudaMemcpyAsync(proj + (size_t)p0 * k, q, sizeof(float) * (size_t)n * k,
                            cudaMemcpyDeviceToHost, cs));
    }
  }
  pm.mark(8);
  cudaEvent_t done;
  GB_HK(event(&done));
  GB_HK(cudaEventRecord(done, cs));
  GB_HK(cudaStreamWaitEvent(st, done, 0));     // `st` completes after the last copy
#undef GB_HK
  const int rc = finish(PCA_OK);
  if (rc == PCA_OK && info) return pca_read_info(workspace, stream, info);
  return rc;
}

const char* pca_status_string(int status) {
  switch (status) {
    case PCA_OK: return "ok";
    case PCA_ERR_ARG: return "invalid argument";
    case PCA_ERR_NOCONV: return "Jacobi did not reach the tolerance within sweeps_max sweeps";
    case PCA_ERR_NONFINITE: return "non-finite value in the cube";
    case PCA_ERR_TIMEOUT: return "a bounded device wait timed out";
    case PCA_ERR_CUDA: return "CUDA runtime error";
    case PCA_ERR_WORKSPACE: return "workspace too small or misaligned";
  }
  return "unknown status";
}

size_t pca_backward_workspace_size(int64_t N, int B, int k) {
  if (!bwd_args_ok(nullptr, PCA_F32, N, B, k, 0.0)) return 0;
  return make_bwd_layout(N, B, k, device_sms()).total;
}

int pca_backward(const void* cube, pca_dtype dt, int64_t N, int B, int k, const double* mu,
                 const double* eigvals, const double* eigvecs, const float* dproj,
                 const double* deigvals, double gap_eps, float* dcube, void* workspace,
                 size_t ws_bytes, void* stream, pca_info* info) {
  if (!bwd_args_ok(cube, dt, N, B, k, gap_eps)) return PCA_ERR_ARG;
  if (!mu || !eigvals || !eigvecs || !dproj || !dcube) return PCA_ERR_ARG;
  if (((uintptr_t)dproj) % 16 != 0) return PCA_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace) % 256 != 0) return PCA_ERR_WORKSPACE;
  const BwdLayout L = make_bwd_layout(N, B, k, device_sms());
  if (ws_bytes < L.total) return PCA_ERR_WORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  BwdPtrs w{};
  w.parts = L.parts;
  w.dv_part = reinterpret_cast<float*>(ws + L.dv_part);
  w.dqs_part = reinterpret_cast<float*>(ws + L.dqs_part);
  w.dVk = reinterpret_cast<double*>(ws + L.dVk);
  w.Gk = reinterpret_cast<double*>(ws + L.Gk);
  w.dA = reinterpret_cast<double*>(ws + L.dA);
  w.S32 = reinterpret_cast<float*>(ws + L.S32);
  w.vk32 = reinterpret_cast<float*>(ws + L.vk32);
  w.mdq = reinterpret_cast<float*>(ws + L.mdq);
  w.mu32 = reinterpret_cast<float*>(ws + L.mu32);
  w.xmax_part = reinterpret_cast<float*>(ws + L.xmax_part);
  w.dqmax_part = reinterpret_cast<float*>(ws + L.dqmax_part);
  w.ascale = reinterpret_cast<float*>(ws + L.ascale);
  w.anshift = reinterpret_cast<float*>(ws + L.anshift);
  w.bop = ws + L.bop;
  w.fcol = reinterpret_cast<float*>(ws + L.fcol);
  DevHeader* hdr = reinterpret_cast<DevHeader*>(ws + L.hdr);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_header_init<<<1, 1, 0, st>>>(hdr, 0, 0.f);
  GB_CK(cudaGetLastError());
  GB_CK(launch_backward(cube, dt, N, B, k, mu, eigvals, eigvecs, dproj, deigvals, gap_eps, dcube, w,
                        hdr, st));
  if (info) return pca_read_info(workspace, stream, info);
  return PCA_OK;
}

int pca_version(void) { return 100; }

int pca_kernel_launches(pca_precision prec, int k) {
  // header init, covariance (MIX: tensor-core pass + guarded SIMT
  // re-computation), band-sum reduce, covariance finalise, Jacobi (with
  // V), compact, 6 per refinement iteration (four products, the eigenvalue
  // and the angle kernels), 1 conversion, 3 per orthogonalisation step,
  // rank/sign + scatter, projection: one SIMT pass per 32 columns (MIX: band
  // constants, then operand preparation + tensor-core pass per 128 columns,
  // and the guarded SIMT passes)
  const int it = refine_iterations(prec);
  const int cov = prec == PCA_PREC_MIX ? 2 : 1;
  int proj = 0;
  if (k > 0) {
    proj = (k + 31) / 32;
    if (prec == PCA_PREC_MIX) proj += 1 + 2 * ((k + 127) / 128);
  }
  return 5 + cov + 6 * it + (it > 0 ? 1 : 0) + 3 * ortho_steps(prec) + 2 + proj;
}

int pca_jacobi_sms(int B) {
  if (B < 2 || B > kMaxB) return 0;
  int nA = 0, nV = 0;
  jacobi_cluster_shape(B, &nA, &nV);
  const int P = round_even(B) / 2;
  return (nA > P ? P : nA) + nV;
}

int pca_batch_jacobi_ctas(int B, int request) {
  if (B < 2 || B > kMaxB || request < 0 || request > 8) return 0;
  return jacobi_ctas_at_least(B, request);
}

int pca_profile(int enable) {
  g_prof.on = enable != 0;
  g_prof.nrec = 0;
  return kProfStages;
}

int pca_profile_collect(float* ms, int max_records) {
  const int n = std::min(g_prof.nrec, max_records);
  for (int r = 0; r < n; ++r) {
    if (g_prof.used[r][kProfStages]) cudaEventSynchronize(g_prof.ev[r][kProfStages]);
    for (int i = 0; i < kProfStages; ++i) {
      float t = 0.f;
      if (g_prof.used[r][i] && g_prof.used[r][i + 1])
        cudaEventElapsedTime(&t, g_prof.ev[r][i], g_prof.ev[r][i + 1]);
      ms[r * kProfStages + i] = t;
    }
  }
  return n;
}

}  // extern "C"
