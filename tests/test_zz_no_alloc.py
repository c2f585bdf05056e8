"""pca_project_noalloc: the projection for callers that cannot allocate device
memory (graph capture, host-owned allocators, real-time loops).  It keeps its
intermediates in a fixed device array of the library instead of a workspace;
its results must equal those of pca_project on the same inputs.

This file runs last (its name sorts last) so that a run stopping at the first
failure has already run every other test; it passes alone in a fresh process
as well as after the others."""
import numpy as np
import pytest
import torch

import oracle
import synth


def _inputs(cube, dtype=torch.float32):
    Yt = torch.from_numpy(cube.Y).to(dtype)         # the oracle sees the same values
    ref = oracle.pca_fit(Yt, cube.k, tol=1e-14)
    Y = Yt.cuda()
    mu = torch.from_numpy(ref["mu"]).cuda()
    V = torch.from_numpy(ref["V"]).cuda()
    return Y, mu, V, ref["Q"]


@pytest.mark.gpu
def test_noalloc_projection_matches_pca_project_on_consecutive_calls(gbpca_lib):
    g = gbpca_lib
    cubes = [synth.linear_mixing(seed=31, rows=41, cols=43, bands=96, endmembers=6, k=6),
             synth.linear_mixing(seed=32, rows=29, cols=31, bands=256, endmembers=8, k=32),
             synth.linear_mixing(seed=33, rows=17, cols=19, bands=7, endmembers=3, k=2)]
    cases = [(cubes[0], torch.float32), (cubes[1], torch.float32), (cubes[2], torch.float32),
             (cubes[0], torch.bfloat16), (cubes[1], torch.float16)]
    for cube, dtype in cases:                # consecutive calls share the array
        Y, mu, V, Q_oracle = _inputs(cube, dtype)
        Q_ref = g.project(Y, mu, V, cube.k)  # pca_project, with a workspace
        Q = g.project_noalloc(Y, mu, V, cube.k)
        torch.cuda.synchronize()
        a = Q.cpu().numpy().astype(np.float64)
        b = Q_ref.cpu().numpy().astype(np.float64)
        for j in range(cube.k):
            scale = max(np.abs(Q_oracle[:, j]).max(), 1e-30)
            err = np.abs(a[:, j] - b[:, j]).max() / max(np.abs(b[:, j]).max(), 1e-30)
            assert err <= 1e-5, (cube.name, dtype, j, err)
            err_o = np.abs(a[:, j] - Q_oracle[:, j]).max() / scale
            assert err_o <= 1e-5, (cube.name, dtype, j, err_o)


@pytest.mark.gpu
def test_noalloc_projection_rejects_bad_sizes(gbpca_lib):
    g = gbpca_lib
    Y = torch.zeros(64, 8, device="cuda")
    mu = torch.zeros(8, dtype=torch.float64, device="cuda")
    V = torch.eye(8, dtype=torch.float64, device="cuda")
    with pytest.raises(g.PCAError) as e:
        g.project_noalloc(Y, mu, V, 9)       # k > B
    assert e.value.status == 1
    # within the ABI (k <= B) but beyond the library's fixed array: B + B k > 8448
    Y = torch.zeros(64, 256, device="cuda")
    mu = torch.zeros(256, dtype=torch.float64, device="cuda")
    V = torch.eye(256, dtype=torch.float64, device="cuda")
    with pytest.raises(g.PCAError) as e:
        g.project_noalloc(Y, mu, V, 33)
    assert e.value.status == 1
