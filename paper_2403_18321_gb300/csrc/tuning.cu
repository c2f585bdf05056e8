// tuning.cu -- the process-wide tuning parameters of include/gbpca.h
// (pca_tuning): the accumulation-run length of the tensor-core covariance and
// the work-balance and cluster-shape choices of the batched form.  Host only;
// read when a workspace is sized, a fit is enqueued or a batch is planned.
#include <cmath>
#include <mutex>

#include "internal.h"

namespace gbpca {
namespace {

pca_tuning defaults() {
  pca_tuning t{};
  t.tc_slot_chunks = 4;
  t.tc_slot_chunks_f16 = 64;
  t.tc_slot_chunks_bf16 = 1024;
  t.tc_slot_chunks_batch = 8;
  for (int i = 0; i < 8; ++i) t.batch_jacobi_ctas[i] = 0;
  t.batch_cov_tc_fixed = 464.0;
  t.batch_proj_fixed = 223.0;
  t.batch_cov_simt_fixed = 13900.0;
  t.batch_simt_items_per_sm = 4;
  t.proj_tc_stages = 0;
  t.proj_tc_raw_stages = 0;
  t.stream_sms_reserve = 0;
  return t;
}

std::mutex g_mu;
pca_tuning g_tuning = defaults();

bool valid(const pca_tuning& t) {
  if (t.tc_slot_chunks < 1 || t.tc_slot_chunks > 1024) return false;
  if (t.tc_slot_chunks_batch < 1 || t.tc_slot_chunks_batch > 1024) return false;
  if (t.tc_slot_chunks_f16 < 1 || t.tc_slot_chunks_f16 > 1024) return false;
  if (t.tc_slot_chunks_bf16 < 1 || t.tc_slot_chunks_bf16 > 1024) return false;
  for (int i = 0; i < 8; ++i)
    if (t.batch_jacobi_ctas[i] < 0 || t.batch_jacobi_ctas[i] > 8) return false;
  auto ok = [](double v) { return std::isfinite(v) && v >= 0.0 && v <= 1e9; };
  if (!ok(t.batch_cov_tc_fixed) || !ok(t.batch_proj_fixed) || !ok(t.batch_cov_simt_fixed))
    return false;
  if (t.proj_tc_stages != 0 && (t.proj_tc_stages < 2 || t.proj_tc_stages > 6)) return false;
  if (t.proj_tc_raw_stages != 0 && (t.proj_tc_raw_stages < 2 || t.proj_tc_raw_stages > 8))
    return false;
  if (t.stream_sms_reserve < 0 || t.stream_sms_reserve > 64) return false;
  return t.batch_simt_items_per_sm >= 1 && t.batch_simt_items_per_sm <= 64;
}

}  // namespace

pca_tuning tuning() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_tuning;
}

}  // namespace gbpca

extern "C" {

void pca_tuning_defaults(pca_tuning* t) {
  if (t) *t = gbpca::defaults();
}

int pca_set_tuning(const pca_tuning* t) {
  const pca_tuning v = t ? *t : gbpca::defaults();
  if (!gbpca::valid(v)) return PCA_ERR_ARG;
  std::lock_guard<std::mutex> lk(gbpca::g_mu);
  gbpca::g_tuning = v;
  return PCA_OK;
}

int pca_get_tuning(pca_tuning* t) {
  if (!t) return PCA_ERR_ARG;
  *t = gbpca::tuning();
  return PCA_OK;
}

}  // extern "C"
