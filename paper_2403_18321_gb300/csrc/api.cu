// api.cu -- the C ABI of include/gbpca.h: argument checks, workspace
// layout and the launch sequence of the four PCA stages (Algorithm 1).
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace gbpca {

namespace {

constexpr int kMaxSweeps = 100;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return 148;
  return sms;
}

__global__ void k_header_init(DevHeader* h, int refine_iters, float tol32) {
  DevHeader z;
  memset(&z, 0, sizeof(z));
  z.refine_iters = refine_iters;
  z.tol_used = tol32;
  z.dummy_slot = -1;
  *h = z;
}

bool args_ok(const void* cube, pca_dtype dt, int64_t N, int B, int k, double tol,
             int sweeps_max, pca_precision prec) {
  if (!cube) return false;
  if (dt != PCA_F32 && dt != PCA_BF16 && dt != PCA_F16) return false;
  if (prec != PCA_PREC_P64 && prec != PCA_PREC_P32 && prec != PCA_PREC_MIX) return false;
  if (N < 2 || B < 2 || B > kMaxB || k < 1 || k > B || k > kMaxK) return false;
  if (!(tol > 0.0) || !std::isfinite(tol)) return false;
  if (sweeps_max < 1 || sweeps_max > kMaxSweeps) return false;
  if (((uintptr_t)cube) % 16 != 0) return false;
  if (prec == PCA_PREC_MIX && !syrk_tc_supported(B)) return false;
  return true;
}

// ---- optional per-stage CUDA-event timing (profiling entry points of gbpca.h)
constexpr int kProfStages = 8;  // cov, cov_finalize, jacobi, vreplay, compact, refine, sort, project
constexpr int kProfRecords = 256;
struct ProfState {
  bool on = false;
  int nrec = 0;
  cudaEvent_t ev[kProfRecords][kProfStages + 1] = {};
  bool used[kProfRecords][kProfStages + 1] = {};
};
thread_local ProfState g_prof;

struct StageMark {
  cudaStream_t st;
  int rec;
  explicit StageMark(cudaStream_t s) : st(s), rec(-1) {
    if (g_prof.on && g_prof.nrec < kProfRecords) rec = g_prof.nrec++;
  }
  void mark(int i) {
    if (rec < 0) return;
    cudaEvent_t& e = g_prof.ev[rec][i];
    if (!e) cudaEventCreate(&e);
    cudaEventRecord(e, st);
    g_prof.used[rec][i] = true;
  }
};

int refine_iterations(pca_precision prec) {
  return prec == PCA_PREC_P32 ? 0 : (prec == PCA_PREC_MIX ? 1 : 2);
}

}  // namespace

Layout make_layout(int64_t N, int B, int k, pca_dtype dt, pca_precision prec, int num_sms) {
  (void)dt;
  Layout L{};
  const int Bp = round_even(B), P = Bp / 2;
  if (prec == PCA_PREC_MIX) {
    L.partials = (int)std::min<int64_t>(num_sms, std::max<int64_t>(1, (N + 127) / 128));
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
  L.s1_part = take(sizeof(double) * (size_t)L.partials * B);
  L.s2_part = take((size_t)L.s2_bytes_el * L.partials * L.s2_elems);
  L.dvec = take(sizeof(double) * B);
  L.cov = take(BB8);
  L.diag32 = take(sizeof(float) * Bp);
  L.log = take(sizeof(float2) * (size_t)kMaxSweeps * Bp * P);
  L.v32 = take(sizeof(float) * (size_t)Bp * Bp);
  L.lam = take(sizeof(double) * B);
  L.vc = take(BB8);
  L.w = take(BB8);
  L.s = take(BB8);
  L.r = take(BB8);
  L.e = take(BB8);
  L.vk = take(sizeof(float) * (size_t)B * k);
  L.muf = take(sizeof(float) * B);
  L.total = o;
  return L;
}

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
  return info->status;
}

int pca_fit(const void* cube, pca_dtype dt, int64_t N, int B, int k, double tol, int sweeps_max,
            pca_precision prec, double* mu, double* eigvals, double* eigvecs, float* proj,
            void* workspace, size_t ws_bytes, void* stream, pca_info* info) {
  if (!args_ok(cube, dt, N, B, k, tol, sweeps_max, prec)) return PCA_ERR_ARG;
  if (!mu || !eigvals || !eigvecs) return PCA_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace) % 256 != 0) return PCA_ERR_WORKSPACE;
  const Layout L = make_layout(N, B, k, dt, prec, device_sms());
  if (ws_bytes < L.total) return PCA_ERR_WORKSPACE;

  char* ws = static_cast<char*>(workspace);
  DevHeader* hdr = reinterpret_cast<DevHeader*>(ws + L.hdr);
  float* shift = reinterpret_cast<float*>(ws + L.shift);
  double* s1p = reinterpret_cast<double*>(ws + L.s1_part);
  void* s2p = ws + L.s2_part;
  double* dvec = reinterpret_cast<double*>(ws + L.dvec);
  double* C = reinterpret_cast<double*>(ws + L.cov);
  float* diag32 = reinterpret_cast<float*>(ws + L.diag32);
  float2* log = reinterpret_cast<float2*>(ws + L.log);
  float* v32 = reinterpret_cast<float*>(ws + L.v32);
  double* lam = reinterpret_cast<double*>(ws + L.lam);
  double* vc = reinterpret_cast<double*>(ws + L.vc);
  double* w = reinterpret_cast<double*>(ws + L.w);
  double* s = reinterpret_cast<double*>(ws + L.s);
  double* g = reinterpret_cast<double*>(ws + L.r);
  double* e = reinterpret_cast<double*>(ws + L.e);
  float* vk = reinterpret_cast<float*>(ws + L.vk);
  float* muf = reinterpret_cast<float*>(ws + L.muf);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  const int iters = refine_iterations(prec);
  const float tol32 = std::max((float)tol, kJacobiFloor);
  StageMark pm(st);
  k_header_init<<<1, 1, 0, st>>>(hdr, iters, tol32);
  GB_CK(cudaGetLastError());

  // stages 2-3 of Algorithm 1: band means and covariance, one pass
  pm.mark(0);
  if (prec == PCA_PREC_MIX)
    GB_CK(launch_syrk_tc(cube, dt, N, B, shift, s1p, (float*)s2p, L.partials, hdr, st));
  else
    GB_CK(launch_syrk_simt(cube, dt, N, B, prec == PCA_PREC_P64, shift, s1p, s2p, L.partials, st));
  pm.mark(1);
  GB_CK(launch_cov_finalize(shift, s1p, s2p, L.s2_bytes_el == 8, L.partials, N, B, mu, C, muf,
                            dvec, hdr, st));
  // stage 4: eigen-decomposition
  pm.mark(2);
  GB_CK(launch_jacobi(C, B, tol32, sweeps_max, log, diag32, hdr, st));
  pm.mark(3);
  GB_CK(launch_vreplay(log, B, hdr, v32, st));
  pm.mark(4);
  GB_CK(launch_compact(diag32, v32, B, hdr, lam, vc, st));
  pm.mark(5);
  for (int it = 0; it < iters; ++it) GB_CK(launch_refine(C, B, vc, lam, w, s, g, e, hdr, st));
  pm.mark(6);
  GB_CK(launch_sort_sign(lam, vc, B, k, eigvals, eigvecs, vk, hdr, st));
  // stages 5-6: projection onto the first k eigenvectors
  pm.mark(7);
  if (proj) GB_CK(launch_project(cube, dt, N, B, k, muf, vk, proj, st));
  pm.mark(8);

  if (info) return pca_read_info(ws, stream, info);
  return PCA_OK;
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

int pca_version(void) { return 100; }

int pca_kernel_launches(pca_precision prec, int with_projection) {
  // header init, covariance, band-sum reduce, covariance finalise, Jacobi,
  // V replay, compact, 6 per refinement iteration, sort/sign, projection
  return 7 + 6 * refine_iterations(prec) + 1 + (with_projection ? 1 : 0);
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
