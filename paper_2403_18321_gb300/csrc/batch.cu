// batch.cu -- the batched form of include/gbpca.h: many independent cubes
// ("tiles") fitted in one go, each as pca_fit fits one cube (Algorithm 1 per
// tile).
//
// Plan (host, once): per-tile workspace regions; the covariance work list --
// (tile, pixel range) items balanced by bytes over the CTAs of one
// persistent launch, each item with its own partial slot; the projection
// work list, balanced the same way; the Jacobi parameter lists, one per
// cluster shape; the tensor maps of the cubes.  All of it is written into the
// workspace with one copy.
//
// Run (per call, kernels only): header init, covariance partials (tensor
// cores for MIX, with the guarded SIMT recomputation; SIMT for P32/P64),
// finalisation, one Jacobi launch per cluster shape on forked streams,
// compaction, refinement (MIX/P64), sort and sign, projection.  Every small
// stage is one launch over all tiles (tile = blockIdx.y or .z).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace gbpca {
namespace {

constexpr int kCovChunk = 32;    // pixel granularity of covariance items
constexpr int kProjChunk = 64;   // pixel granularity of projection items
constexpr int kProjCols = 32;    // columns of one projection pass

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

__global__ void k_header_init_batched(TileDesc* __restrict__ T, int ntiles, int refine_iters,
                                      float tol32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntiles) return;
  DevHeader z;
  memset(&z, 0, sizeof(z));
  z.refine_iters = refine_iters;
  z.tol_used = tol32;
  z.dummy_slot = -1;
  *T[i].hdr = z;
}

// Cost of one chunk of a tile with B bands, in arbitrary units, fitted to the
// measured times of the streaming kernels on this GPU: a fixed part per chunk
// (barrier round trips, the MMA/epilogue cadence) plus a part per band; the
// SIMT covariance grows with the B^2/2 products per pixel.  The fixed parts
// are tuning parameters (defaults: ~1.16 us + 2.5 ns per band per 32-pixel
// covariance chunk, ~1.07 us + 4.8 ns per band per 64-pixel projection chunk).
enum class Cost { kTensorCov, kSimtCov, kProject };
double chunk_cost(const pca_tuning& tu, Cost c, int B) {
  switch (c) {
    case Cost::kTensorCov: return tu.batch_cov_tc_fixed + B;
    case Cost::kSimtCov: return tu.batch_cov_simt_fixed + (double)B * B;
    case Cost::kProject: return tu.batch_proj_fixed + B;
  }
  return B;
}

// CTAs of the batched Jacobi cluster of a B-band tile under the tuning.
int batch_cluster_ctas(const pca_tuning& tu, int B) {
  const int bucket = (round_even(B) - 1) / 32;
  const int want = tu.batch_jacobi_ctas[bucket < 0 ? 0 : (bucket > 7 ? 7 : bucket)];
  return jacobi_ctas_at_least(B, want);
}

// Splits the tiles' chunks into `ctas` contiguous ranges of equal cost; every
// (tile, range) piece is one item.  Returns the items grouped by CTA and the
// number of items of every tile.
struct Split {
  std::vector<std::vector<CovItem>> per_cta;
  std::vector<int> parts;
};
Split split_chunks(const std::vector<pca_tile>& tiles, int chunk, int ctas, Cost cost,
                   const pca_tuning& tu) {
  Split sp;
  const int n = (int)tiles.size();
  sp.per_cta.assign(ctas, {});
  sp.parts.assign(n, 0);
  long double total = 0;
  for (const pca_tile& t : tiles)
    total += (long double)((t.N + chunk - 1) / chunk) * chunk_cost(tu, cost, t.B);
  long double w0 = 0;  // weight before the current tile
  int g = 0;
  for (int ti = 0; ti < n; ++ti) {
    const int64_t nch = (tiles[ti].N + chunk - 1) / chunk;
    const double wc = chunk_cost(tu, cost, tiles[ti].B);  // cost of one chunk
    int64_t c = 0;
    while (c < nch) {
      int64_t cend = nch;
      if (g < ctas - 1) {
        const long double end = total * (g + 1) / ctas;  // weight at which CTA g stops
        const long double x = (end - w0) / wc;
        cend = x <= 0 ? 0 : std::min<int64_t>(nch, (int64_t)std::ceil((double)x));
        if (cend <= c) { ++g; continue; }
      }
      CovItem it;
      it.tile = ti;
      it.slot = sp.parts[ti]++;
      it.p0 = c * chunk;
      it.p1 = std::min<int64_t>(tiles[ti].N, cend * chunk);
      sp.per_cta[g].push_back(it);
      c = cend;
    }
    w0 += (long double)nch * wc;
  }
  return sp;
}

}  // namespace
}  // namespace gbpca

using namespace gbpca;

struct pca_batch {
  int ntiles = 0;
  pca_dtype dt = PCA_F32;
  pca_precision prec = PCA_PREC_P32;
  float tol32 = 0.f;
  int maxB = 0, maxk = 0;
  TileDesc* T = nullptr;          // device
  DevHeader* hdrs = nullptr;      // device, [ntiles] contiguous
  // covariance items
  CovItem* cov_items = nullptr;
  int* cov_off = nullptr;
  int cov_ctas = 0, cov_nitems = 0;
  // projection items
  ProjItem* proj_items = nullptr;
  int* proj_off = nullptr;
  int proj_ctas = 0;
  void* maps = nullptr;           // device CUtensorMap[ntiles] or null (untiled loads)
  // Jacobi lists, one per cluster shape (V width, CTAs per cluster), each
  // launched on its own stream
  struct Bucket {
    void* list = nullptr;         // device, `count` parameter entries
    int count = 0;
    size_t smem = 0;
    std::vector<unsigned char> first;  // host copy of the first entry (launch shape)
    cudaStream_t stream = nullptr;
    cudaEvent_t join = nullptr;
  };
  std::vector<Bucket> buckets;
  cudaEvent_t fork = nullptr;
};

namespace {

bool tile_ok(const pca_tile& t, pca_dtype dt, pca_precision prec, double tol, int sweeps_max) {
  if (!t.mu || !t.eigvals || !t.eigvecs) return false;
  return args_ok(t.cube, dt, t.N, t.B, t.k, tol, sweeps_max, prec);
}

// Workspace layout of a batch.  With descs != nullptr the per-tile
// descriptors are filled in, pointing into the workspace at `base`.
struct BatchLayout {
  size_t tiles, hdrs, cov_items, cov_off, proj_items, proj_off, maps, lists;
  size_t total;
  Split cov, proj;
};

BatchLayout batch_layout(const std::vector<pca_tile>& tiles, pca_dtype dt, pca_precision prec,
                         int sms, const pca_tuning& tu, std::vector<TileDesc>* descs, char* base) {
  BatchLayout L{};
  const int n = (int)tiles.size();
  const bool mix = prec == PCA_PREC_MIX, p64 = prec == PCA_PREC_P64;
  const bool refine = refine_iterations(prec) > 0;
  const int cov_ctas = mix ? sms : tu.batch_simt_items_per_sm * sms;
  L.cov = split_chunks(tiles, kCovChunk, cov_ctas, mix ? Cost::kTensorCov : Cost::kSimtCov, tu);
  if (mix) {  // bound the tensor-core accumulation: long items become several slots
    const int64_t cap = dt == PCA_F32 ? tu.tc_slot_chunks_batch
                                      : (dt == PCA_F16 ? tu.tc_slot_chunks_f16 : tu.tc_slot_chunks_bf16);
    std::vector<int> slot_of(n, 0);
    for (auto& v : L.cov.per_cta) {
      std::vector<CovItem> split;
      for (const CovItem& it : v) {
        const int64_t c0 = it.p0 / kCovChunk, c1 = (it.p1 + kCovChunk - 1) / kCovChunk;
        const int64_t pieces = (c1 - c0 + cap - 1) / cap;
        for (int64_t q = 0; q < pieces; ++q) {
          CovItem x = it;
          x.p0 = (c0 + (c1 - c0) * q / pieces) * kCovChunk;
          x.p1 = std::min<int64_t>(it.p1, (c0 + (c1 - c0) * (q + 1) / pieces) * kCovChunk);
          x.slot = slot_of[it.tile]++;
          split.push_back(x);
        }
      }
      v.swap(split);
    }
    L.cov.parts = slot_of;
  }
  // one projection "tile" per projected tile and group of 32 columns (the
  // projection kernel's pass width); CovItem.slot carries the column group
  std::vector<pca_tile> ptiles;
  std::vector<int> pmap, gmap;
  for (int i = 0; i < n; ++i)
    if (tiles[i].proj)
      for (int grp = 0; grp * kProjCols < tiles[i].k; ++grp) {
        ptiles.push_back(tiles[i]);
        pmap.push_back(i);
        gmap.push_back(grp);
      }
  L.proj = split_chunks(ptiles, kProjChunk, sms, Cost::kProject, tu);
  for (auto& v : L.proj.per_cta)
    for (auto& it : v) {
      it.slot = gmap[it.tile];
      it.tile = pmap[it.tile];
    }
  int ncov = 0, nproj = 0;
  for (auto& v : L.cov.per_cta) ncov += (int)v.size();
  for (auto& v : L.proj.per_cta) nproj += (int)v.size();
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o = al256(o + bytes); return at; };
  L.tiles = take(sizeof(TileDesc) * n);
  L.hdrs = take(sizeof(DevHeader) * n);
  L.cov_items = take(sizeof(CovItem) * std::max(ncov, 1));
  L.cov_off = take(sizeof(int) * (cov_ctas + 1));
  L.proj_items = take(sizeof(ProjItem) * std::max(nproj, 1));
  L.proj_off = take(sizeof(int) * (sms + 1));
  L.maps = take(128 * (size_t)n);
  L.lists = take(jacobi_params_bytes() * n);
  if (descs) descs->assign(n, TileDesc{});
  for (int i = 0; i < n; ++i) {
    const pca_tile& t = tiles[i];
    const int B = t.B, Bp = round_even(B), k = t.k;
    const int parts = L.cov.parts[i];
    const size_t BB = (size_t)B * B;
    TileDesc d{};
    auto at = [&](size_t off) -> void* { return base ? base + off : nullptr; };
    d.cube = t.cube;
    d.N = t.N;
    d.B = B;
    d.k = k;
    d.mu = t.mu;
    d.eigvals = t.eigvals;
    d.eigvecs = t.eigvecs;
    d.proj = t.proj;
    d.hdr = static_cast<DevHeader*>(at(L.hdrs + sizeof(DevHeader) * i));
    d.parts = parts;
    d.shift = static_cast<float*>(at(take(sizeof(float) * B)));
    d.escale = static_cast<int*>(at(take(sizeof(int) * B)));
    d.s1p = static_cast<double*>(at(take(sizeof(double) * parts * B)));
    d.s2p = at(take((p64 ? 8 : 4) * (size_t)parts * (B * (B + 1) / 2)));
    d.dvec = static_cast<double*>(at(take(sizeof(double) * B)));
    d.C = static_cast<double*>(at(take(sizeof(double) * BB)));
    d.cdf = refine ? static_cast<float2*>(at(take(sizeof(float2) * BB))) : nullptr;
    d.rank = static_cast<int*>(at(take(sizeof(int) * B)));
    d.sgn = static_cast<double*>(at(take(sizeof(double) * B)));
    d.diag32 = static_cast<float*>(at(take(sizeof(float) * Bp)));
    d.v32 = static_cast<float*>(at(take(sizeof(float) * (size_t)Bp * Bp)));
    d.lam = static_cast<double*>(at(take(sizeof(double) * B)));
    d.vc = static_cast<float2*>(at(take(sizeof(float2) * BB)));
    if (refine) {
      d.w = static_cast<float2*>(at(take(sizeof(float2) * BB)));
      d.s = static_cast<float2*>(at(take(sizeof(float2) * BB)));
      d.g = static_cast<float2*>(at(take(sizeof(float2) * BB)));
      d.e = static_cast<float2*>(at(take(sizeof(float2) * BB)));
    }
    d.vk = static_cast<float*>(at(take(sizeof(float) * (size_t)B * k)));
    d.muf = static_cast<float*>(at(take(sizeof(float) * B)));
    if (descs) (*descs)[i] = d;
  }
  L.total = o;
  return L;
}

std::vector<pca_tile> as_vector(int ntiles, const pca_tile* tiles) {
  return std::vector<pca_tile>(tiles, tiles + ntiles);
}

#define GB_CK(x)                                   \
  do {                                             \
    if ((x) != cudaSuccess) return PCA_ERR_CUDA;   \
  } while (0)

}  // namespace

extern "C" {

size_t pca_batch_workspace_size(int ntiles, const pca_tile* tiles, pca_dtype dtype,
                                pca_precision prec) {
  static const float kDummy[4] = {0.f, 0.f, 0.f, 0.f};
  if (ntiles < 1 || !tiles) return 0;
  std::vector<pca_tile> v = as_vector(ntiles, tiles);
  for (pca_tile& t : v) {
    if (!args_ok(kDummy, dtype, t.N, t.B, t.k, 1.0, 1, prec)) return 0;
    t.cube = kDummy;
  }
  return batch_layout(v, dtype, prec, device_sms(), tuning(), nullptr, nullptr).total;
}

int pca_batch_plan_counts(int ntiles, const pca_tile* tiles, pca_dtype dtype, pca_precision prec,
                          int* counts) {
  static const float kDummy[4] = {0.f, 0.f, 0.f, 0.f};
  if (ntiles < 1 || !tiles || !counts) return PCA_ERR_ARG;
  std::vector<pca_tile> v = as_vector(ntiles, tiles);
  for (pca_tile& t : v) {
    if (!args_ok(kDummy, dtype, t.N, t.B, t.k, 1.0, 1, prec)) return PCA_ERR_ARG;
    t.cube = kDummy;
    t.proj = const_cast<float*>(kDummy);   // every tile counted as projected
  }
  const pca_tuning tu = tuning();
  const BatchLayout L = batch_layout(v, dtype, prec, device_sms(), tu, nullptr, nullptr);
  int ncov = 0, nproj = 0;
  for (const auto& c : L.cov.per_cta) ncov += (int)c.size();
  for (const auto& c : L.proj.per_cta) nproj += (int)c.size();
  std::vector<int> shapes;
  int widest = 0;
  for (const pca_tile& t : v) {
    const int n = batch_cluster_ctas(tu, t.B);
    shapes.push_back(jacobi_width(t.B) * 16 + n);
    widest = std::max(widest, n);
  }
  std::sort(shapes.begin(), shapes.end());
  counts[0] = ncov;
  counts[1] = nproj;
  counts[2] = (int)(std::unique(shapes.begin(), shapes.end()) - shapes.begin());
  counts[3] = widest;
  return PCA_OK;
}

int pca_batch_create(pca_batch** plan, int ntiles, const pca_tile* tiles, pca_dtype dtype,
                     double tol, int sweeps_max, pca_precision prec, void* workspace,
                     size_t ws_bytes, int* bad_tile) {
  if (!plan) return PCA_ERR_ARG;
  *plan = nullptr;
  if (ntiles < 1 || !tiles) return PCA_ERR_ARG;
  for (int i = 0; i < ntiles; ++i)
    if (!tile_ok(tiles[i], dtype, prec, tol, sweeps_max)) {
      if (bad_tile) *bad_tile = i;
      return PCA_ERR_ARG;
    }
  if (!workspace || ((uintptr_t)workspace) % 256 != 0) return PCA_ERR_WORKSPACE;
  const std::vector<pca_tile> v = as_vector(ntiles, tiles);
  const int sms = device_sms();
  char* ws = static_cast<char*>(workspace);
  std::vector<TileDesc> descs;
  const pca_tuning tu = tuning();
  const BatchLayout L = batch_layout(v, dtype, prec, sms, tu, &descs, ws);
  if (ws_bytes < L.total) return PCA_ERR_WORKSPACE;

  pca_batch* b = new (std::nothrow) pca_batch;
  if (!b) return PCA_ERR_ARG;
  b->ntiles = ntiles;
  b->dt = dtype;
  b->prec = prec;
  b->tol32 = std::max((float)tol, stop_floor(prec));
  for (const pca_tile& t : v) { b->maxB = std::max(b->maxB, t.B); b->maxk = std::max(b->maxk, t.k); }
  b->T = reinterpret_cast<TileDesc*>(ws + L.tiles);
  b->hdrs = reinterpret_cast<DevHeader*>(ws + L.hdrs);

  // the table region [0, end of the Jacobi lists) is built on the host and copied once
  const size_t table = L.lists + jacobi_params_bytes() * ntiles;
  std::vector<unsigned char> img(table, 0);
  std::memcpy(img.data() + L.tiles, descs.data(), sizeof(TileDesc) * ntiles);
  {  // covariance items, CTA by CTA
    std::vector<CovItem> items;
    std::vector<int> off(1, 0);
    for (const auto& c : L.cov.per_cta) {
      items.insert(items.end(), c.begin(), c.end());
      off.push_back((int)items.size());
    }
    std::memcpy(img.data() + L.cov_items, items.data(), sizeof(CovItem) * items.size());
    std::memcpy(img.data() + L.cov_off, off.data(), sizeof(int) * off.size());
    b->cov_items = reinterpret_cast<CovItem*>(ws + L.cov_items);
    b->cov_off = reinterpret_cast<int*>(ws + L.cov_off);
    b->cov_ctas = (int)L.cov.per_cta.size();
    b->cov_nitems = (int)items.size();
  }
  {  // projection items (64-pixel chunks), CTA by CTA
    std::vector<ProjItem> items;
    std::vector<int> off(1, 0);
    for (const auto& c : L.proj.per_cta) {
      for (const CovItem& it : c) {
        ProjItem p{};
        p.tile = it.tile;
        p.pad = it.slot;               // column group
        p.c0 = it.p0 / kProjChunk;
        p.c1 = (it.p1 + kProjChunk - 1) / kProjChunk;
        items.push_back(p);
      }
      off.push_back((int)items.size());
    }
    std::memcpy(img.data() + L.proj_items, items.data(), sizeof(ProjItem) * items.size());
    std::memcpy(img.data() + L.proj_off, off.data(), sizeof(int) * off.size());
    b->proj_items = reinterpret_cast<ProjItem*>(ws + L.proj_items);
    b->proj_off = reinterpret_cast<int*>(ws + L.proj_off);
    b->proj_ctas = items.empty() ? 0 : (int)L.proj.per_cta.size();
  }
  {  // tensor maps: the tiled load when every projected cube qualifies
    bool all = true;
    for (int i = 0; i < ntiles && all; ++i)
      if (v[i].proj) all = encode_cube_map(dtype, v[i].cube, v[i].N, v[i].B, img.data() + L.maps + 128 * (size_t)i);
    b->maps = all ? ws + L.maps : nullptr;
  }
  {  // Jacobi lists.  Throughput over latency: each matrix gets the fewest
     // CTAs that hold its V (a cluster per matrix; the clusters of one shape
     // share a launch), and within a shape the largest matrices start first.
    std::vector<int> order(ntiles);
    for (int i = 0; i < ntiles; ++i) order[i] = i;
    auto key = [&](int i) { return jacobi_width(v[i].B) * 16 + batch_cluster_ctas(tu, v[i].B); };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
      return key(a) != key(c) ? key(a) > key(c) : v[a].B > v[c].B;
    });
    const size_t pb = jacobi_params_bytes();
    int prev = -1;
    for (int pos = 0; pos < ntiles; ++pos) {
      const int i = order[pos];
      if (key(i) != prev) {
        b->buckets.emplace_back();
        b->buckets.back().list = ws + L.lists + pb * pos;
        prev = key(i);
      }
      pca_batch::Bucket& bu = b->buckets.back();
      unsigned char* dst = img.data() + L.lists + pb * pos;
      const size_t smem = jacobi_fill_params(dst, descs[i].C, v[i].B, b->tol32, sweeps_max,
                                             relative_stop(prec), descs[i].diag32, descs[i].v32,
                                             descs[i].hdr, batch_cluster_ctas(tu, v[i].B));
      bu.smem = std::max(bu.smem, smem);
      if (bu.count == 0) bu.first.assign(dst, dst + pb);
      ++bu.count;
    }
  }
  bool ok = cudaMemcpy(ws, img.data(), table, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (pca_batch::Bucket& bu : b->buckets) {
    if (!ok) break;
    ok = cudaStreamCreateWithFlags(&bu.stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&bu.join, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    pca_batch_destroy(b);
    return PCA_ERR_CUDA;
  }
  *plan = b;
  return PCA_OK;
}

int pca_batch_run(pca_batch* b, void* stream) {
  if (!b) return PCA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = b->ntiles, maxB = b->maxB;
  const pca_precision prec = b->prec;
  const int iters = refine_iterations(prec), ortho = ortho_steps(prec);
  StageMark pm(st);
  k_header_init_batched<<<(n + 127) / 128, 128, 0, st>>>(b->T, n, iters, b->tol32);
  GB_CK(cudaGetLastError());
  // stages 2-3: band means and covariance
  pm.mark(0);
  if (prec == PCA_PREC_MIX) {
    GB_CK(launch_syrk_tc_grouped(b->T, b->cov_items, b->cov_off, b->cov_ctas, maxB, b->dt, st));
    GB_CK(launch_syrk_simt_grouped(b->T, b->cov_items, b->cov_nitems, maxB, n, b->dt, false, true,
                                   st));
  } else {
    GB_CK(launch_syrk_simt_grouped(b->T, b->cov_items, b->cov_nitems, maxB, n, b->dt,
                                   prec == PCA_PREC_P64, false, st));
  }
  pm.mark(1);
  GB_CK(launch_cov_finalize_batched(b->T, n, maxB, prec == PCA_PREC_P64, prec == PCA_PREC_MIX, st));
  // stage 4: one Jacobi launch per cluster shape, side by side
  pm.mark(2);
  GB_CK(cudaEventRecord(b->fork, st));
  for (pca_batch::Bucket& bu : b->buckets) {
    GB_CK(cudaStreamWaitEvent(bu.stream, b->fork, 0));
    GB_CK(launch_jacobi_cluster_list(bu.first.data(), bu.list, bu.count, bu.smem, bu.stream));
    GB_CK(cudaEventRecord(bu.join, bu.stream));
  }
  for (pca_batch::Bucket& bu : b->buckets) GB_CK(cudaStreamWaitEvent(st, bu.join, 0));
  pm.mark(3);
  pm.mark(4);
  GB_CK(launch_compact_batched(b->T, n, maxB, st));
  pm.mark(5);
  bool in_w = false;  // V alternates between vc and w
  if (iters > 0) GB_CK(launch_to_df_batched(b->T, n, maxB, st));
  for (int it = 0; it < iters; ++it, in_w = !in_w)
    GB_CK(launch_refine_batched(b->T, n, maxB, in_w, refine_max_angle(prec), st));
  for (int it = 0; it < ortho; ++it, in_w = !in_w)
    GB_CK(launch_orthonormalize_batched(b->T, n, maxB, in_w, st));
  pm.mark(6);
  GB_CK(launch_sort_sign_batched(b->T, n, maxB, in_w, st));
  // stages 5-6: projection
  pm.mark(7);
  GB_CK(launch_project_grouped(b->T, b->maps, b->proj_items, b->proj_off, b->proj_ctas, maxB,
                               b->maxk, b->dt, st));
  pm.mark(8);
  return PCA_OK;
}

int pca_batch_read_info(pca_batch* b, void* stream, pca_info* infos) {
  if (!b) return PCA_ERR_ARG;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return PCA_ERR_CUDA;
  std::vector<DevHeader> h(b->ntiles);
  if (cudaMemcpy(h.data(), b->hdrs, sizeof(DevHeader) * b->ntiles, cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return PCA_ERR_CUDA;
  int worst = PCA_OK;
  for (int i = 0; i < b->ntiles; ++i) {
    if (worst == PCA_OK && h[i].status != PCA_OK) worst = h[i].status;
    if (!infos) continue;
    pca_info& o = infos[i];
    o.status = h[i].status;
    o.sweeps = h[i].sweeps;
    o.refine_iters = h[i].refine_iters;
    o.steps = h[i].steps;
    o.off_rel = h[i].off_rel;
    o.tol_used = h[i].tol_used;
    o.refine_res = h[i].refine_res;
    o.cov_fallback = h[i].cov_range != 0 ? 1 : 0;
    o.proj_fallback = h[i].proj_range != 0 ? 1 : 0;
  }
  return worst;
}

int pca_batch_kernel_launches(const pca_batch* b) {
  if (!b) return 0;
  const int iters = refine_iterations(b->prec), ortho = ortho_steps(b->prec);
  int n = 1 + (b->prec == PCA_PREC_MIX ? 2 : 1) + 2;  // header, covariance, finalisation
  n += (int)b->buckets.size();
  n += 1;                                              // compaction
  n += (iters > 0 ? 1 : 0) + 6 * iters + 3 * ortho;    // refinement
  n += 2;                                              // rank/sign, scatter
  n += b->proj_ctas > 0 ? 1 : 0;
  return n;
}

void pca_batch_destroy(pca_batch* b) {
  if (!b) return;
  for (pca_batch::Bucket& bu : b->buckets) {
    if (bu.stream) cudaStreamDestroy(bu.stream);
    if (bu.join) cudaEventDestroy(bu.join);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

int pca_fit_batched(int ntiles, const pca_tile* tiles, pca_dtype dtype, double tol, int sweeps_max,
                    pca_precision prec, void* workspace, size_t ws_bytes, void* stream,
                    pca_info* infos) {
  pca_batch* b = nullptr;
  int r = pca_batch_create(&b, ntiles, tiles, dtype, tol, sweeps_max, prec, workspace, ws_bytes,
                           nullptr);
  if (r != PCA_OK) return r;
  r = pca_batch_run(b, stream);
  if (r == PCA_OK && infos) r = pca_batch_read_info(b, stream, infos);
  pca_batch_destroy(b);
  return r;
}

}  // extern "C"
