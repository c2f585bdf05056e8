"""GPU parity of the adjoint (pca_backward) against the FP64 oracle adjoint,
itself pinned by central differences in test_oracle.py.

The backward pass accumulates X^T dQ in FP32 per CTA (FP64 across CTAs),
does the B x B algebra in FP64 and forms dY in FP32 (K = B + k terms per
entry), so the tolerance is 2e-5 of the largest |dY| entry.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

TOL = 2e-5


def _case(seed, side, bands, k, comps=None):
    c = synth.gradient_cube(seed=seed, side=side, bands=bands, comps=comps or min(bands, k + 2),
                            k=k, grad_seed=seed + 40)
    return c.Y, c.k, c.meta["dQ"]


def _check(gbpca, Y, k, dQ, dlam=None, dtype=torch.float32, gap_eps=1e-9):
    Yt = torch.from_numpy(Y).to(dtype)
    ref_fwd = oracle.pca_fit(Yt, k, tol=1e-14)
    ref = oracle.backward(Yt, k, ref_fwd["mu"], ref_fwd["lam"], ref_fwd["V"], dQ, dlam, gap_eps)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = gbpca.backward(Yt.cuda(), dev(ref_fwd["mu"]), dev(ref_fwd["lam"]), dev(ref_fwd["V"]),
                         dev(dQ.astype(np.float32)), dev(dlam) if dlam is not None else None,
                         gap_eps=gap_eps)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    return err


@pytest.mark.gpu
# (9, 256, 32): the largest B and k of the ABI (two pipeline stages in the
# X^T dQ pass, the widest tensor-core dY product)
@pytest.mark.parametrize("side,bands,k", [(16, 24, 5), (21, 33, 6), (20, 48, 10), (13, 7, 3),
                                          (9, 256, 32)])
def test_backward_matches_oracle(gbpca_lib, side, bands, k):
    Y, k, dQ = _case(side * 3 + bands, side, bands, k)
    err = _check(gbpca_lib, Y, k, dQ)
    print(f"N={Y.shape[0]} B={bands} k={k} err={err:.2e}")
    assert err <= TOL


@pytest.mark.gpu
def test_backward_with_eigenvalue_gradient_and_bf16(gbpca_lib):
    Y, k, dQ = _case(77, 19, 40, 6)
    dl = np.random.default_rng(5).standard_normal(Y.shape[1])
    assert _check(gbpca_lib, Y, k, dQ, dlam=dl) <= TOL
    # only the eigenvalue gradient
    assert _check(gbpca_lib, Y, k, np.zeros_like(dQ), dlam=dl) <= TOL
    # a bf16 cube (the oracle widens the same bf16 values exactly)
    assert _check(gbpca_lib, Y, k, dQ, dtype=torch.bfloat16) <= TOL


@pytest.mark.gpu
def test_backward_full_size_differentiation_workload(gbpca_lib):
    """512 x 512 pixels x 200 bands, k = 10, planted spectrum with relative gaps
    >= 1e-3 among the top 11 and dQ ~ N(0, 1): every entry of dY against the
    oracle adjoint."""
    c = synth.gradient_cube()
    err = _check(gbpca_lib, c.Y, c.k, c.meta["dQ"], gap_eps=1e-6)
    print(f"full-size backward err={err:.2e}")
    assert err <= TOL


@pytest.mark.gpu
def test_autograd_function_uses_the_adjoint(gbpca_lib):
    Y, k, dQ = _case(91, 17, 30, 5)
    cube = torch.from_numpy(Y).cuda().requires_grad_(True)
    Q = gbpca_lib.PCAProjection.apply(cube, k, "p64", 1e-12, 30, 1e-9)
    G = torch.from_numpy(dQ.astype(np.float32)).cuda()
    (Q * G).sum().backward()
    ref_fwd = oracle.pca_fit(Y, k, tol=1e-14)
    ref = oracle.backward(Y, k, ref_fwd["mu"], ref_fwd["lam"], ref_fwd["V"], dQ, None, 1e-9)
    err = np.abs(cube.grad.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 1e-4, err
