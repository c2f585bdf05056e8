"""GPU parity on the precision form: 2048 x 2048 pixels x 224 bands, BF16 and FP16
inputs in [0, 1], planted spectrum s_i = 0.7^(i-1) over 20 components above a
1e-3 floor, k = 20.

Reduced size (256 x 256 pixels): every output against the FP64 oracle.

Full size (4,194,304 pixels; the oracle's triple-loop covariance would take about
1e11 FP64 multiply-adds): properties that hold at any size, evaluated in FP64 on
the host from the same 16-bit values --
  * the band means against the exact FP64 column means;
  * for every returned pair j < k the eigen-residual |C v_j - lam_j v_j| / lam_1
    and the Rayleigh quotient |v_j^T C v_j - lam_j| / lam_1, with the exact
    C = X^T X / (N - 1), X = Y - 1 mu*^T applied in chunked FP64 products (both
    hold inside the noise-floor cluster, where single vectors are not defined:
    rounding the data to 16 bits adds a floor near 1e-5 lam_1, above the planted
    components beyond about the 16th);
  * the orthogonality of V;
  * sampled rows of Q against (y_n - mu) V_k in FP64 from the GPU's own mu and V
    (the projection kernel computes in FP32 in every form).
"""
import functools

import numpy as np
import pytest
import torch

import oracle
import synth
from parity import LAM_ALL_TOL, LAM_TOL, MU_TOL, ORTH_TOL, compare

# eigen-residual and Rayleigh-quotient bounds, relative to lam_1: the eigenvalue
# bounds of each form (the residual of an eigenpair bounds its eigenvalue error)
RES_TOL = {"mix": LAM_TOL["mix"], "p32": LAM_ALL_TOL["p32"], "p64": LAM_TOL["p64"]}
Q_ROW_TOL = 1e-4       # sampled projection rows, relative to max |Q[:, 0]|
CLUSTER_TOL = 1e-6     # P64 pairs inside a cluster (FP32-level accuracy, include/gbpca.h)
# P64 eigenvalues below 1e-3 lam_1: 1e-10 of 1e-3 lam_1 absolute (the refinement's
# double-float products carry about 2^-48 ||C|| per entry)
P64_LAM_FLOOR = 1e-3
CHUNK = 1 << 18


def _separated(lam, k, thr=1e-5):
    """Number of leading pairs separated from both neighbours by more than
    thr * lam_1: the pairs P64 resolves to FP64.  The refinement treats a pair
    whose first-order angle exceeds 1/64 as part of a cluster, i.e. gaps below
    about 64 times the FP32 accuracy of the Jacobi (~4e-6 lam_1); such clusters
    keep FP32-level accuracy (here the 16-bit rounding floor is one)."""
    l1 = abs(lam[0])
    for j in range(k):
        left = lam[j - 1] - lam[j] if j > 0 else np.inf
        if min(left, lam[j] - lam[j + 1]) <= thr * l1:
            return j
    return k


@functools.lru_cache(maxsize=4)
def _cube(side, dtype):
    return synth.planted_spectrum(side=side, dtype=dtype)


def _fit(g, Y16, k, form):
    mu, ev, V, Q, info = g.fit(Y16.cuda(), k, tol=1e-10, sweeps_max=30, precision=form)
    torch.cuda.synchronize()
    return (mu.cpu().numpy(), ev.cpu().numpy(), V.cpu().numpy(),
            Q.cpu().numpy().astype(np.float64)), info


@pytest.mark.gpu
@pytest.mark.parametrize("form", ["mix", "p32", "p64"])
@pytest.mark.parametrize("dtype", ["bf16", "fp16"])
def test_precision_form_reduced_against_oracle(gbpca_lib, dtype, form):
    c = _cube(256, dtype)
    Yq = c.Y.float().numpy()          # the oracle sees the same rounded values
    oracle.set_threads(0)
    ref = oracle.pca_fit(Yq, c.k, tol=1e-14)
    out, info = _fit(gbpca_lib, c.Y, c.k, form)
    assert info["status"] == 0, info
    kc = _separated(ref["lam"], c.k) if form == "p64" else c.k
    assert kc >= 12
    mu, lam, V, Q = out
    m = compare((mu, lam, V, Q[:, :kc]), ref, kc, form,
                lam_floor=P64_LAM_FLOOR if form == "p64" else None)
    print(f"{dtype} {form}: kc {kc} {m}")


def _exact_moments(Y16, V):
    """mu* (FP64 column means) and C V for the columns of V, with C the exact
    covariance of the 16-bit cube (chunked FP64 products)."""
    N, B = Y16.shape
    s = np.zeros(B)
    for n0 in range(0, N, CHUNK):
        s += Y16[n0:n0 + CHUNK].double().numpy().sum(axis=0)
    mu = s / N
    CV = np.zeros((B, V.shape[1]))
    for n0 in range(0, N, CHUNK):
        X = Y16[n0:n0 + CHUNK].double().numpy() - mu[None, :]
        CV += X.T @ (X @ V)
    return mu, CV / (N - 1)


@pytest.mark.gpu
@pytest.mark.parametrize("form,dtype", [("mix", "bf16"), ("mix", "fp16"), ("p32", "bf16"),
                                        ("p64", "bf16")])
def test_precision_form_full_size_properties(gbpca_lib, form, dtype):
    c = _cube(2048, dtype)
    N, B, k = c.N, c.B, c.k
    (mu, lam, V, Q), info = _fit(gbpca_lib, c.Y, k, form)
    assert info["status"] == 0, info
    Vk = V[:, :k]
    mu_ref, CV = _exact_moments(c.Y, Vk)
    l1 = abs(lam[0])
    # band means
    mu_err = np.abs(mu - mu_ref).max() / np.abs(mu_ref).max()
    assert mu_err <= MU_TOL[form], mu_err
    # eigen-residuals and Rayleigh quotients of the returned pairs
    res = np.linalg.norm(CV - Vk * lam[None, :k], axis=0) / l1
    rq = np.abs(np.einsum("bj,bj->j", Vk, CV) - lam[:k]) / l1
    print(f"{dtype} {form}: mu {mu_err:.2e} residual {res.max():.2e} rayleigh {rq.max():.2e} "
          f"sweeps {info['sweeps']} residuals {np.array2string(res, precision=1)}")
    kc = _separated(lam, k) if form == "p64" else k
    assert kc >= 12
    assert res[:kc].max() <= RES_TOL[form], res
    assert rq[:kc].max() <= RES_TOL[form], rq
    if kc < k:
        assert res[kc:].max() <= CLUSTER_TOL, res
        assert rq[kc:].max() <= CLUSTER_TOL, rq
    # descending, and orthonormal
    assert np.all(np.diff(lam) <= 0)
    assert np.abs(V.T @ V - np.eye(B)).max() <= ORTH_TOL[form]
    # sampled projection rows from the GPU's own mu and V
    rows = np.random.default_rng(7).choice(N, 4096, replace=False)
    rows = np.concatenate([rows, [0, N - 1]])
    Xs = c.Y[torch.from_numpy(rows)].double().numpy() - mu[None, :]
    q_err = np.abs(Q[rows] - Xs @ Vk).max() / np.abs(Q[:, 0]).max()
    assert q_err <= Q_ROW_TOL, q_err
