"""GPU side of the pixel-sharded fit: the pooling kernel (pca_combine_moments)
and the shifted-sum exchange (pca_shifted_sums, the sum the all-reduce
forms, pca_moments_from_sums) against the oracle's moments of the whole
cube, and fit_sharded on a one-rank NCCL group against pca_fit.  (More than
one rank needs more than one GPU; the exchange itself is tested on CPU ranks
in test_sharded.py.)"""
import os
import socket

import numpy as np
import pytest
import torch

import oracle
import synth


@pytest.mark.gpu
@pytest.mark.parametrize("bounds", [(0, 700, 702, 1230), (0, 1230), (0, 2, 4, 6, 1230)])
def test_combine_moments_matches_whole_cube(gbpca_lib, bounds):
    g = gbpca_lib
    cube = synth.linear_mixing(seed=78, rows=30, cols=41, bands=37, endmembers=6, k=4)
    Y = torch.from_numpy(cube.Y).cuda()
    mus, Cs, counts = [], [], []
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        mu, C, info = g.covariance(Y[lo:hi].clone(), precision="p64")  # own 16-byte aligned copy
        assert info["status"] == 0
        mus.append(mu)
        Cs.append(C)
        counts.append(hi - lo)
    mu, C = g.combine_moments(counts, torch.stack(mus), torch.stack(Cs))
    torch.cuda.synchronize()
    mu_ref = oracle.band_means(cube.Y)
    C_ref = oracle.covariance(cube.Y)
    assert np.abs(mu.cpu().numpy() - mu_ref).max() <= 1e-13 * np.abs(mu_ref).max()
    assert np.abs(C.cpu().numpy() - C_ref).max() <= 1e-12 * np.abs(C_ref).max()


@pytest.mark.gpu
def test_combine_moments_rejects_bad_counts(gbpca_lib):
    g = gbpca_lib
    mus = torch.zeros(2, 4, dtype=torch.float64, device="cuda")
    Cs = torch.zeros(2, 4, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(g.PCAError):
        g.combine_moments([3, 0], mus, Cs)
    with pytest.raises(g.PCAError):
        g.combine_moments([1], mus[:1], Cs[:1])


@pytest.mark.gpu
@pytest.mark.parametrize("bounds", [(0, 700, 702, 1230), (0, 1230), (0, 2, 4, 6, 1230)])
@pytest.mark.parametrize("offset", [0.0, 1e4])
def test_shifted_sums_match_whole_cube(gbpca_lib, bounds, offset):
    """The shards' shifted sums, added as an all-reduce adds them, give the whole
    cube's moments; a large common offset of every band (10^4, far above the
    pixels' spread) must not cost accuracy, since the shift takes it out first."""
    g = gbpca_lib
    cube = synth.linear_mixing(seed=78, rows=30, cols=41, bands=37, endmembers=6, k=4)
    Yn = (cube.Y + np.float32(offset)).astype(np.float32)
    Y = torch.from_numpy(Yn).cuda()
    parts = []
    s = None
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        mu, C, info = g.covariance(Y[lo:hi].clone(), precision="p64")
        assert info["status"] == 0
        if s is None:
            s = mu.clone()            # the common shift: the first shard's mean
        parts.append(g.shifted_sums(hi - lo, mu, C, s))
    total = torch.stack(parts).sum(0)
    assert total.numel() == g.sums_length(37)
    assert total[0].item() == bounds[-1]
    mu, C = g.moments_from_sums(total, s)
    torch.cuda.synchronize()
    mu_ref = oracle.band_means(Yn)
    C_ref = oracle.covariance(Yn)
    assert np.abs(mu.cpu().numpy() - mu_ref).max() <= 1e-13 * np.abs(mu_ref).max()
    assert np.abs(C.cpu().numpy() - C_ref).max() <= 1e-11 * np.abs(C_ref).max()
    Cn = C.cpu().numpy()
    assert np.array_equal(Cn, Cn.T)


@pytest.mark.gpu
def test_shifted_sums_reject_bad_arguments(gbpca_lib):
    g = gbpca_lib
    mu = torch.zeros(4, dtype=torch.float64, device="cuda")
    C = torch.zeros(4, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(g.PCAError):
        g.shifted_sums(0, mu, C, mu)
    with pytest.raises(ValueError):
        g.moments_from_sums(torch.zeros(5, dtype=torch.float64, device="cuda"), mu)


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.gpu
@pytest.mark.parametrize("form", ["p64", "mix"])
def test_fit_sharded_one_rank_equals_fit(gbpca_lib, form):
    import torch.distributed as dist
    g = gbpca_lib
    cube = synth.linear_mixing(seed=79, rows=40, cols=50, bands=64, endmembers=6, k=5)
    Y = torch.from_numpy(cube.Y).cuda()
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_port()}", rank=0,
                            world_size=1)
    try:
        mu, ev, V, Q, info = g.fit_sharded(Y, 5, precision=form)
        torch.cuda.synchronize()
    finally:
        dist.destroy_process_group()
    assert info["status"] == 0
    mu1, ev1, V1, Q1, _ = g.fit(Y, 5, precision=form)
    l1 = abs(ev1[0].item())
    assert (mu - mu1).abs().max().item() <= 1e-12 * mu1.abs().max().item()
    assert (ev - ev1).abs().max().item() <= 1e-9 * l1
    assert (Q - Q1).abs().max().item() <= 1e-5 * Q1.abs().max().item()
