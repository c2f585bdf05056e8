"""The autotuner's cache (CPU): parameters stored under a device key are read
back (speed parameters only), installed in the library while a batch is
planned and restored afterwards, and change the plan the library makes."""
import json

import pytest

import paper_2403_18321_gb300 as g
from paper_2403_18321_gb300 import tune

SHAPES = [(4096, 64, 8), (9000, 128, 8), (20000, 224, 8), (7000, 256, 8), (5000, 160, 8)]


@pytest.fixture
def cache(tmp_path, monkeypatch):
    p = tmp_path / "tuning.json"
    monkeypatch.setenv(tune.CACHE_ENV, str(p))
    yield p
    g.set_tuning(None)


def test_cache_roundtrip_keeps_speed_parameters_only(cache):
    key = tune.cache_key("NVIDIA GB300", 152, 0, 2)
    assert key == "NVIDIA GB300|sm152|f32|mix"
    params = {"batch_jacobi_ctas": [0, 0, 3, 4, 0, 6, 8, 7], "batch_cov_tc_fixed": 232.0,
              "tc_slot_chunks": 8}                  # an accuracy parameter: never cached
    assert tune.store(key, params, {"ms": 21.0}) == str(cache)
    got = tune.lookup(key)
    assert got == {"batch_jacobi_ctas": [0, 0, 3, 4, 0, 6, 8, 7], "batch_cov_tc_fixed": 232.0}
    assert tune.lookup("other|sm1|f32|mix") is None
    d = json.loads(cache.read_text())
    assert d[key]["ms"] == 21.0


def test_applied_installs_and_restores(cache):
    default = g.tuning()
    with tune.applied({"batch_jacobi_ctas": [8] * 8, "batch_proj_fixed": 100.0}):
        t = g.tuning()
        assert t["batch_jacobi_ctas"] == [8] * 8 and t["batch_proj_fixed"] == 100.0
        assert t["tc_slot_chunks"] == default["tc_slot_chunks"]
        assert t["tc_slot_chunks_f16"] == default["tc_slot_chunks_f16"]
        assert t["tc_slot_chunks_bf16"] == default["tc_slot_chunks_bf16"]
        assert t["tc_slot_chunks_batch"] == default["tc_slot_chunks_batch"]
    assert g.tuning() == default


def test_cached_parameters_change_the_plan(cache):
    key = tune.cache_key("NVIDIA GB300", 152, 0, 2)
    base = g.batch_plan_counts(SHAPES, "mix")
    tune.store(key, {"batch_jacobi_ctas": [8] * 8})
    with tune.applied(tune.lookup(key)):
        tuned = g.batch_plan_counts(SHAPES, "mix")
    assert base["widest_cluster"] < 8 and tuned["widest_cluster"] == 8
    assert tuned["jacobi_launches"] < base["jacobi_launches"]
    assert g.batch_plan_counts(SHAPES, "mix") == base        # restored


def test_invalid_tuning_is_rejected_and_leaves_the_old_values():
    before = g.tuning()
    with pytest.raises(g.PCAError):
        g.set_tuning({"batch_jacobi_ctas": [9] * 8})
    with pytest.raises(g.PCAError):
        g.set_tuning({"tc_slot_chunks": 0})
    for bad in (-1, 65):
        with pytest.raises(g.PCAError):
            g.set_tuning({"stream_sms_reserve": bad})
    assert g.tuning() == before


def test_sm_reserve_shrinks_the_streaming_grid_in_the_workspace_plan():
    """stream_sms_reserve takes SMs from the persistent covariance grid: a BF16
    cube of this size gives every CTA one accumulation run (at most 1024 chunks),
    so the grid's CTA count is its count of partial slots, which the workspace
    size reads (host only, no GPU)."""
    assert g.tuning()["stream_sms_reserve"] == 0
    N, B, k = 4_194_304, 224, 20
    base = g.workspace_size(N, B, k, 1, "mix")
    try:
        g.set_tuning({"stream_sms_reserve": 8})
        assert g.tuning()["stream_sms_reserve"] == 8
        reserved = g.workspace_size(N, B, k, 1, "mix")
    finally:
        g.set_tuning(None)
    assert reserved < base
    assert g.workspace_size(N, B, k, 1, "mix") == base


def test_cluster_request_is_raised_to_a_shape_that_holds_the_matrix():
    for B in (64, 128, 224, 256):
        fewest = g.batch_jacobi_ctas(B, 0)
        assert 1 <= fewest <= 8
        assert g.batch_jacobi_ctas(B, 1) == fewest
        assert g.batch_jacobi_ctas(B, 8) == 8
        for n in range(fewest, 9):
            assert g.batch_jacobi_ctas(B, n) == n
