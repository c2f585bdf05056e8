"""Components beyond 32 (1 <= k <= B): pca_fit in every form, the batched form
and the adjoint, at k = 33, 64, 128 and k = B, up to B = k = 256.

Where the eigen-pairs are individually defined the comparison rules of
parity.compare apply; every column of the projection (including those in
the noise cluster, whose vectors are not individually pinned) is checked
against the FP64 projection of the cube onto the GPU's own eigenvectors,
within the rounding-error bound of an FP32 dot product, and the adjoint
against the oracle adjoint (2e-5 of max |dY|)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import compare

CASES = [(40, 41, 64, 33), (30, 33, 96, 64), (25, 27, 160, 128), (21, 23, 96, 96),
         (17, 19, 256, 256)]


def _projection_stage_err(Y, mu, V, Q, k):
    """|Q - (Y - mu) V_k| against the rounding-error bound of an FP32 dot
    product of B terms computed from FP32 copies of mu and V (Higham's
    gamma_n = n u / (1 - n u), n = B + 3 roundings per term path, u = 2^-24):
        |Q_nj - R_nj| <= gamma_{B+3} sum_b (|x_nb| + |mu_b|) |v_bj|,
    which holds whatever the summation order and however much the terms
    cancel (the noise-floor columns).  Returns the largest ratio of the error
    to its bound (<= 1 passes)."""
    B = Y.shape[1]
    X = Y.astype(np.float64) - mu[None, :]
    Vk = V[:, :k]
    R = X @ Vk
    S = (np.abs(X) + np.abs(mu)[None, :]) @ np.abs(Vk)
    u = 2.0 ** -24
    gamma = (B + 3) * u / (1 - (B + 3) * u)
    return float(np.max(np.abs(Q - R) / np.maximum(gamma * S, 1e-300)))


@pytest.mark.gpu
@pytest.mark.parametrize("form", ["p32", "mix", "p64"])
@pytest.mark.parametrize("rows,cols,B,k", CASES)
def test_fit_with_many_components(gbpca_lib, form, rows, cols, B, k):
    g = gbpca_lib
    c = synth.linear_mixing(seed=rows + B + k, rows=rows, cols=cols, bands=B, endmembers=9, k=k)
    ref = oracle.pca_fit(c.Y, k, tol=1e-14)
    mu, ev, V, Q, info = g.fit(torch.from_numpy(c.Y).cuda(), k, tol=1e-10, precision=form)
    torch.cuda.synchronize()
    assert info["status"] == 0, info
    host = [t.cpu().numpy().astype(np.float64) for t in (mu, ev, V, Q)]
    assert host[3].shape == (c.N, k)
    # P64 is FP64-accurate outside clusters: the signal components (endmembers - 1)
    kc = min(k, 8) if form == "p64" else k
    compare((host[0], host[1], host[2], host[3][:, :kc]), ref, kc, form)
    err = _projection_stage_err(c.Y, host[0], host[2], host[3], k)
    assert err <= 1.0, err


@pytest.mark.gpu
@pytest.mark.parametrize("form", ["mix", "p32"])
def test_batched_with_many_components(gbpca_lib, form):
    g = gbpca_lib
    cubes = [synth.linear_mixing(seed=900 + i, rows=r, cols=cc, bands=B, endmembers=7, k=k)
             for i, (r, cc, B, k) in enumerate(CASES)]
    dev = [torch.from_numpy(c.Y).cuda() for c in cubes]
    results, status, infos = g.fit_batched(dev, [c.k for c in cubes], tol=1e-10, precision=form)
    assert status == 0, infos
    for c, (mu, ev, V, Q) in zip(cubes, results):
        ref = oracle.pca_fit(c.Y, c.k, tol=1e-14)
        host = [t.cpu().numpy().astype(np.float64) for t in (mu, ev, V, Q)]
        compare((host[0], host[1], host[2], host[3]), ref, c.k, form)
        err = _projection_stage_err(c.Y, host[0], host[2], host[3], c.k)
        assert err <= 1.0, (c.name, err)


@pytest.mark.gpu
@pytest.mark.parametrize("side,bands,k", [(12, 48, 33), (10, 96, 64), (9, 160, 128),
                                          (8, 256, 256)])
def test_backward_with_many_components(gbpca_lib, side, bands, k):
    c = synth.gradient_cube(seed=side + bands, side=side, bands=bands, comps=min(bands, 12),
                            k=k, grad_seed=k)
    Y, dQ = c.Y, c.meta["dQ"]
    ref_fwd = oracle.pca_fit(Y, k, tol=1e-14)
    ref = oracle.backward(Y, k, ref_fwd["mu"], ref_fwd["lam"], ref_fwd["V"], dQ, None, 1e-9)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = gbpca_lib.backward(dev(Y), dev(ref_fwd["mu"]), dev(ref_fwd["lam"]), dev(ref_fwd["V"]),
                             dev(dQ.astype(np.float32)), gap_eps=1e-9)
    torch.cuda.synchronize()
    err = np.abs(out.cpu().numpy().astype(np.float64) - ref).max() / np.abs(ref).max()
    print(f"B={bands} k={k} err={err:.2e}")
    assert err <= 2e-5, err


@pytest.mark.gpu
def test_project_stage_with_many_components(gbpca_lib):
    g = gbpca_lib
    c = synth.linear_mixing(seed=77, rows=33, cols=35, bands=200, endmembers=6, k=150)
    ref = oracle.pca_fit(c.Y, c.k, tol=1e-14)
    Q = g.project(torch.from_numpy(c.Y).cuda(), torch.from_numpy(ref["mu"]).cuda(),
                  torch.from_numpy(ref["V"]).cuda(), c.k)
    Qn = Q.cpu().numpy().astype(np.float64)
    err = np.max(np.abs(Qn - ref["Q"]).max(axis=0) / np.abs(ref["Q"]).max(axis=0))
    assert err <= 1e-5, err
