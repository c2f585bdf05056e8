"""GPU parity of the batched form (pca_batch_* / pca_fit_batched) against the
FP64 oracle, tile by tile.  A batch mixes band counts across all four
Jacobi cluster shapes (B' <= 32, 64, 128, 256), odd band counts (padding
index), pixel counts that leave ragged covariance and projection chunks,
different k, a tile without projection; plus graph capture and replay with
new input values, and the argument checks."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import compare

FORMS = ["p32", "mix", "p64"]

# (rows, cols, bands, endmembers, k): N from 2 pixels up to a few thousand
SHAPES = [(17, 11, 2, 1, 1), (9, 7, 3, 2, 2), (23, 29, 7, 3, 3), (31, 33, 31, 4, 4),
          (40, 41, 33, 5, 5), (37, 41, 64, 4, 4), (61, 34, 103, 10, 10), (50, 51, 128, 5, 5),
          (29, 31, 130, 6, 6), (45, 47, 200, 8, 8), (30, 40, 255, 8, 8), (33, 35, 256, 9, 9),
          (1, 2, 16, 1, 1), (70, 90, 96, 12, 32)]


def _cubes(shapes, seed0=100):
    return [synth.linear_mixing(seed=seed0 + i, rows=r, cols=c, bands=B, endmembers=e, k=k)
            for i, (r, c, B, e, k) in enumerate(shapes)]


def _host(t):
    return t.cpu().numpy().astype(np.float64) if t is not None else None


@pytest.mark.gpu
@pytest.mark.parametrize("form", FORMS)
def test_batch_matches_oracle_tile_by_tile(gbpca_lib, form):
    g = gbpca_lib
    cubes = _cubes(SHAPES)
    dev = [torch.as_tensor(c.Y).cuda() for c in cubes]
    results, status, infos = g.fit_batched(dev, [c.k for c in cubes], tol=1e-10, precision=form)
    assert status == 0, infos
    for c, (mu, ev, V, Q), info in zip(cubes, results, infos):
        assert info["status"] == 0, (c.name, info)
        ref = oracle.pca_fit(c.Y, c.k, tol=1e-14)
        # P64 resolves eigen-pairs to FP64 only outside clusters tighter than
        # about 1e-6 ||C|| (include/gbpca.h); beyond the signal rank (endmembers
        # - 1) the noise eigenvalues form such a cluster, so the FP64 bounds
        # apply to the leading signal components there
        kc = min(c.k, max(1, c.meta["endmembers"] - 1)) if form == "p64" else c.k
        gpu = (_host(mu), _host(ev), _host(V), _host(Q)[:, :kc] if Q is not None else None)
        compare(gpu, ref, kc, form)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_batch_16bit_inputs(gbpca_lib, dtype):
    g = gbpca_lib
    cubes = _cubes(SHAPES[4:10], seed0=300)
    dev = [torch.as_tensor(c.Y).to(dtype).cuda() for c in cubes]
    results, status, _ = g.fit_batched(dev, [c.k for c in cubes], precision="mix")
    assert status == 0
    for c, d, (mu, ev, V, Q) in zip(cubes, dev, results):
        Yq = d.float().cpu().numpy()  # the oracle sees the same rounded values
        ref = oracle.pca_fit(Yq, c.k, tol=1e-14)
        compare((_host(mu), _host(ev), _host(V), _host(Q)), ref, c.k, "mix")


@pytest.mark.gpu
def test_batch_without_projection_and_repeated_runs(gbpca_lib):
    g = gbpca_lib
    cubes = _cubes(SHAPES[5:9], seed0=200)
    dev = [torch.as_tensor(c.Y).cuda() for c in cubes]
    b = g.Batch(dev, [c.k for c in cubes], precision="mix", project=False)
    for _ in range(3):            # the plan is reusable
        b.run()
    status, infos = b.info()
    assert status == 0
    assert all(r[3] is None for r in b.results)
    for c, (mu, ev, V, _) in zip(cubes, b.results):
        ref = oracle.pca_fit(c.Y, c.k, tol=1e-14)
        compare((_host(mu), _host(ev), _host(V), None), ref, c.k, "mix", check_q=False)
    assert b.kernel_launches() > 0
    b.close()


@pytest.mark.gpu
def test_batch_graph_capture_and_replay(gbpca_lib):
    """pca_batch_run launches kernels only: capture it once, change the input
    values in place, replay, and compare with the oracle of the new values."""
    g = gbpca_lib
    shapes = SHAPES[3:11]
    first = _cubes(shapes, seed0=400)
    second = _cubes(shapes, seed0=500)
    dev = [torch.as_tensor(c.Y).cuda() for c in first]
    b = g.Batch(dev, [c.k for c in first], precision="mix")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(stream=s)            # warm-up outside capture (kernel attributes, modules)
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        b.run(stream=s)
    for d, c in zip(dev, second):
        d.copy_(torch.as_tensor(c.Y))
    graph.replay()
    torch.cuda.synchronize()
    status, infos = b.info()
    assert status == 0, infos
    for c, (mu, ev, V, Q) in zip(second, b.results):
        ref = oracle.pca_fit(c.Y, c.k, tol=1e-14)
        compare((_host(mu), _host(ev), _host(V), _host(Q)), ref, c.k, "mix")
    b.close()


@pytest.mark.gpu
@pytest.mark.parametrize("form", ["p32", "mix"])
def test_batch_tile_specs_reduced(gbpca_lib, form):
    """Tiles drawn like the batched workload (log-uniform N, B from the seven
    band counts, 3-15 endmembers, k = 8, tol 1e-8), N scaled down so that the
    oracle finishes quickly."""
    g = gbpca_lib
    specs = synth.tile_batch_specs(seed=3, tiles=24, n_lo=512, n_hi=8192)
    cubes = [synth.tile(s) for s in specs]
    dev = [torch.as_tensor(c.Y).cuda() for c in cubes]
    results, status, infos = g.fit_batched(dev, 8, tol=1e-8, precision=form)
    assert status == 0, [i for i in infos if i["status"]]
    for c, (mu, ev, V, Q) in zip(cubes, results):
        ref = oracle.pca_fit(c.Y, 8, tol=1e-14)
        compare((_host(mu), _host(ev), _host(V), _host(Q)), ref, 8, form)


@pytest.mark.gpu
def test_batch_bad_tile_is_rejected(gbpca_lib):
    g = gbpca_lib
    good = torch.zeros(64, 8, device="cuda")
    bad = torch.zeros(64, 8, device="cuda")
    with pytest.raises(g.PCAError) as e:
        g.Batch([good, bad], [2, 9])          # k > B in tile 1
    assert e.value.status == 1 and "tile 1" in str(e.value)
    with pytest.raises(g.PCAError):
        g.Batch([torch.zeros(64, 257, device="cuda")], 2)


@pytest.mark.gpu
def test_batch_range_guard_recomputes_only_the_flagged_tile(gbpca_lib):
    """A tile with one value far outside its sampled spread leaves the scaled
    FP16 range: that tile (and only that one) is recomputed on the SIMT path,
    and every tile still matches the oracle (the flagged one at P32 accuracy)."""
    g = gbpca_lib
    cubes = _cubes(SHAPES[4:9], seed0=600)
    Ys = [c.Y.copy() for c in cubes]
    assert Ys[2].shape[0] > 1024
    Ys[2][1, 7] = 5e6                          # the data lie in [0, 1]
    dev = [torch.as_tensor(y).cuda() for y in Ys]
    results, status, infos = g.fit_batched(dev, [c.k for c in cubes], precision="mix")
    assert status == 0
    assert [i["cov_fallback"] for i in infos] == [0, 0, 1, 0, 0]
    for t, (c, y, (mu, ev, V, Q)) in enumerate(zip(cubes, Ys, results)):
        ref = oracle.pca_fit(y, c.k, tol=1e-14)
        compare((_host(mu), _host(ev), _host(V), _host(Q)), ref, c.k, "p32" if t == 2 else "mix")


@pytest.mark.gpu
def test_batch_nonfinite_tile_is_reported_alone(gbpca_lib):
    """A NaN in one tile gives that tile PCA_ERR_NONFINITE; the others fit."""
    g = gbpca_lib
    cubes = _cubes(SHAPES[5:8], seed0=700)
    Ys = [c.Y.copy() for c in cubes]
    Ys[1][3, 2] = np.nan
    dev = [torch.as_tensor(y).cuda() for y in Ys]
    for form in ("mix", "p32"):
        results, status, infos = g.fit_batched(dev, [c.k for c in cubes], precision=form)
        assert status == 3
        assert [i["status"] for i in infos] == [0, 3, 0]
        for t in (0, 2):
            ref = oracle.pca_fit(cubes[t].Y, cubes[t].k, tol=1e-14)
            mu, ev, V, Q = results[t]
            compare((_host(mu), _host(ev), _host(V), _host(Q)), ref, cubes[t].k, form)


@pytest.mark.gpu
@pytest.mark.parametrize("form", ["mix", "p32"])
def test_batch_full_size_workload(gbpca_lib, form):
    """The batched workload at full size: 256 tiles (N log-uniform in [4096,
    262144], B from the seven band counts, 3-15 endmembers, k = 8, tol 1e-8;
    15.25 M pixels, 9.9 GB FP32 drawn on the GPU).  Every tile: status, descending
    eigenvalues, orthonormal eigenvectors; four tiles (smallest and largest N, the
    median, the largest B) against the oracle in full."""
    g = gbpca_lib
    specs = synth.tile_batch_specs(seed=3)
    cubes = [synth.tile_device(s, "cuda") for s in specs]
    assert len(cubes) == 256
    results, status, infos = g.fit_batched([c.Y for c in cubes], 8, tol=1e-8, precision=form)
    torch.cuda.synchronize()
    assert status == 0 and all(i["status"] == 0 for i in infos)
    orth_tol = {"mix": 1e-6, "p32": 1e-4}[form]
    for (mu, ev, V, Q) in results:
        lam = ev.cpu().numpy()
        assert np.all(np.diff(lam) <= 0)
        Vh = V.cpu().numpy()
        assert np.abs(Vh.T @ Vh - np.eye(Vh.shape[0])).max() <= orth_tol
    order = np.argsort([c.N for c in cubes])
    sample = {int(order[0]), int(order[len(order) // 2]), int(order[-1]),
              int(np.argmax([c.B for c in cubes]))}
    oracle.set_threads(0)
    for t in sorted(sample):
        c = cubes[t]
        ref = oracle.pca_fit(c.Y.cpu().numpy(), 8, tol=1e-14)
        mu, ev, V, Q = results[t]
        compare((_host(mu), _host(ev), _host(V), _host(Q)), ref, 8, form)


@pytest.mark.gpu
def test_autotuned_batch_keeps_parity(gbpca_lib, tmp_path):
    """The autotuner times its candidates on a small batch, caches the fastest
    parameters, and a batch planned from the cache (other cluster shapes and
    work splits) still matches the oracle tile by tile."""
    from paper_2403_18321_gb300 import tune
    g = gbpca_lib
    cubes = _cubes(SHAPES[3:12], seed0=400)
    dev = [torch.as_tensor(c.Y).cuda() for c in cubes]
    ks = [c.k for c in cubes]
    path = str(tmp_path / "tuning.json")
    res = tune.tune_batch(dev, ks, precision="mix", tol=1e-10, warmup=1, reps=3, path=path)
    assert len(res["trials"]) > 3 and res["ms"] <= res["default_ms"]
    params = tune.lookup(res["key"], path)
    assert params == {k: v for k, v in res["params"].items() if k in tune.SPEED_KEYS}
    # force a non-default shape so that the check covers a tuned plan either way
    params = dict(params, batch_jacobi_ctas=[8] * 8, batch_cov_tc_fixed=232.0)
    b = g.Batch(dev, ks, tol=1e-10, precision="mix", tuning=params)
    b.run()
    status, infos = b.info()
    assert status == 0, infos
    assert g.tuning() == g.tuning_defaults()          # planning restored the defaults
    for c, (mu, ev, V, Q) in zip(cubes, b.results):
        ref = oracle.pca_fit(c.Y, c.k, tol=1e-14)
        compare((_host(mu), _host(ev), _host(V), _host(Q)), ref, c.k, "mix")
    b.close()
