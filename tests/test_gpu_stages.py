"""Stage-by-stage GPU parity through the C ABI (pca_covariance, pca_eigh,
pca_project) against the FP64 oracle, so that each row of the hot path is
checked on its own inputs:

  band means + covariance  (Algorithm 1 stages 2-3)   pca_covariance
  Jacobi + sort + sign     (stage 4, Eqs. 2-10)       pca_eigh on the oracle's C
  projection               (stages 5-6)               pca_project on the oracle's mu, V
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import E_COV, compare, LAM_TOL, ORTH_TOL, rel_gaps, sign_norm

# covariance: max_ij |C - C*| / max_ij |C*|; in the spectral norm relative to
# lambda_1, E_COV (the bound every later comparison builds on)
COV_TOL = {"p64": 1e-13, "p32": 2e-6, "mix": 2e-5}
MU_TOL = {"p64": 1e-13, "p32": 1e-6, "mix": 1e-6}


def cubes_small():
    return [synth.linear_mixing(seed=7, rows=37, cols=41, bands=64, endmembers=5),
            synth.linear_mixing(seed=8, rows=33, cols=31, bands=103, endmembers=6)] + \
        synth.paper_scenes(scale=0.2)


@pytest.mark.gpu
@pytest.mark.parametrize("form,dtype", [("p32", torch.float32), ("mix", torch.float32),
                                        ("p64", torch.float32), ("mix", torch.bfloat16),
                                        ("mix", torch.float16), ("p64", torch.bfloat16)])
def test_covariance_stage(gbpca_lib, form, dtype):
    """16-bit cubes: the oracle sees the same rounded values.  The scene-shaped
    cubes (values up to 8000) spread each band over many binades, so the
    tensor-core runs of 16-bit cubes are not exact there and the MIX bound is
    the same as for FP32 cubes.  (The P32 form is held to its bound on FP32
    cubes: on 16-bit ones its shift, the first pixel, and FP32 sums of
    products with few significant bits give 1.8e-5 element-wise, 2.2e-6 in the
    spectral norm, on the 64-band mixing cube; its eigen-level accuracy on
    16-bit cubes is tested with the precision forms.)"""
    g = gbpca_lib
    for cube in cubes_small():
        Yd = torch.from_numpy(cube.Y).to(dtype)
        Yh = Yd.float().numpy().astype(np.float64)
        Y = Yd.cuda()
        mu, C, info = g.covariance(Y, precision=form)
        torch.cuda.synchronize()
        assert info["status"] == 0
        mu_ref = oracle.band_means(Yh)
        C_ref = oracle.covariance(Yh, mu_ref)
        mu_err = np.abs(mu.cpu().numpy() - mu_ref).max() / np.abs(mu_ref).max()
        cov_err = np.abs(C.cpu().numpy() - C_ref).max() / np.abs(C_ref).max()
        cov_norm = np.linalg.norm(C.cpu().numpy() - C_ref, 2) / np.linalg.norm(C_ref, 2)
        print(f"{cube.name} {form} {dtype} mu_err={mu_err:.3e} cov_err={cov_err:.3e} "
              f"||dC||_2/lam1={cov_norm:.3e}")
        assert mu_err <= MU_TOL[form]
        assert cov_err <= COV_TOL[form]
        assert cov_norm <= E_COV[form], cov_norm
        assert np.array_equal(C.cpu().numpy(), C.cpu().numpy().T)


@pytest.mark.gpu
@pytest.mark.parametrize("form", ["p32", "mix", "p64"])
def test_eigh_stage_on_oracle_covariance(gbpca_lib, form):
    g = gbpca_lib
    for cube in cubes_small():
        C_ref = oracle.covariance(cube.Y)
        ev, V, info = g.eigh(torch.from_numpy(C_ref).cuda(), precision=form)
        torch.cuda.synchronize()
        assert info["status"] == 0, info
        A_k, V_ref, _ = oracle.jacobi(C_ref, tol=1e-15)
        lam_ref, V_ref = oracle.sort_sign(np.diag(A_k), V_ref)
        lam = ev.cpu().numpy()
        Vg = V.cpu().numpy()
        k = cube.k
        gaps = rel_gaps(lam_ref)
        eps = {"p64": 1e-15, "mix": 1e-12, "p32": 1e-6}[form]
        pinned = gaps[:k] >= 1e3 * eps
        rel = np.abs(lam[:k] - lam_ref[:k]) / np.abs(lam_ref[:k])
        print(f"{cube.name} {form} eig_rel_topk={rel[pinned].max():.3e} "
              f"all/l1={np.abs(lam - lam_ref).max() / lam_ref[0]:.3e} "
              f"orth={np.abs(Vg.T @ Vg - np.eye(cube.B)).max():.3e} sweeps={info['sweeps']}")
        tol = {"p64": 1e-10, "mix": 1e-6, "p32": LAM_TOL["p32"]}[form]
        assert rel[pinned].max() <= tol
        assert np.abs(Vg.T @ Vg - np.eye(cube.B)).max() <= {"p64": 1e-11, "mix": 1e-6, "p32": 1e-4}[form]
        # residual of the eigen-equation, relative to ||C||
        res = np.abs(C_ref @ Vg[:, :k] - Vg[:, :k] * lam[None, :k]).max() / lam_ref[0]
        assert res <= {"p64": 1e-12, "mix": 1e-7, "p32": 1e-4}[form]
        assert np.array_equal(sign_norm(Vg), Vg)


@pytest.mark.gpu
def test_eigh_sort_ties_and_diagonal_input(gbpca_lib):
    g = gbpca_lib
    A = np.diag([3.0, 1.0, 3.0, 2.0, 0.5])
    for form in ("p32", "mix", "p64"):
        ev, V, info = g.eigh(torch.from_numpy(A).cuda(), precision=form)
        assert info["sweeps"] == 0
        assert list(ev.cpu().numpy()) == [3.0, 3.0, 2.0, 1.0, 0.5]
        assert np.array_equal(V.cpu().numpy()[:, :2], np.eye(5)[:, [0, 2]])


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("bands", [96, 103, 102, 232, 256])
def test_project_stage(gbpca_lib, dtype, bands):
    """Both load paths of the streamed projection: rows that are a whole number
    of 16-byte units go through the swizzled 2-D tensor map (96, 232, 256
    bands in FP32; 96, 232, 256 in 16-bit), the others through one contiguous copy per
    chunk; 45 x 47 pixels leave a ragged last chunk."""
    g = gbpca_lib
    cube = synth.linear_mixing(seed=11, rows=45, cols=47, bands=bands, endmembers=6, k=6)
    Yt = torch.from_numpy(cube.Y).to(dtype)
    ref = oracle.pca_fit(Yt, cube.k, tol=1e-14)
    Q = g.project(Yt.cuda(), torch.from_numpy(ref["mu"]).cuda(), torch.from_numpy(ref["V"]).cuda(),
                  cube.k)
    Qn = Q.cpu().numpy().astype(np.float64)
    for j in range(cube.k):
        err = np.abs(Qn[:, j] - ref["Q"][:, j]).max() / np.abs(ref["Q"][:, j]).max()
        assert err <= 1e-5, (j, err)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,big", [(torch.bfloat16, 5e6), (torch.float16, 6e4)])
def test_mix_range_guard_16bit_cubes(gbpca_lib, dtype, big):
    """16-bit cubes: the converters see a value beyond the FP16 range through
    its infinite hi and lo parts; the covariance and the projection are then
    recomputed on the SIMT path and match the oracle at P32 accuracy, while
    the same cube without the outlier stays on the tensor cores."""
    g = gbpca_lib
    cube = synth.linear_mixing(seed=21, rows=61, cols=67, bands=48, endmembers=5)
    assert cube.N > 1024          # pixel 1 is then outside the strided sample
    Yd = torch.from_numpy(cube.Y).to(dtype)
    *_, info = g.fit(Yd.cuda(), cube.k, precision="mix")
    assert info["status"] == 0 and info["cov_fallback"] == 0 and info["proj_fallback"] == 0
    Yd[1, 7] = big                # the data lie in [0, 1]
    Yh = Yd.float().numpy().astype(np.float64)
    mu, ev, V, Q, info = g.fit(Yd.cuda(), cube.k, precision="mix")
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["cov_fallback"] == 1 and info["proj_fallback"] == 1, info
    ref = oracle.pca_fit(Yh, cube.k, tol=1e-14)
    compare((mu.cpu().numpy(), ev.cpu().numpy(), V.cpu().numpy(),
             Q.cpu().numpy().astype(np.float64)), ref, cube.k, "p32")


@pytest.mark.gpu
def test_mix_range_guard_recomputes_on_simt(gbpca_lib):
    """MIX scales every band by a power of two taken from a pixel sample; a
    value far outside the sampled spread leaves the FP16 range, which must
    make the covariance be recomputed in FP32 (same result up to P32
    accuracy), while an ordinary cube stays on the tensor-core form."""
    g = gbpca_lib
    cube = synth.linear_mixing(seed=21, rows=61, cols=67, bands=48, endmembers=5)
    assert cube.N > 1024          # pixel 1 is then outside the strided sample
    Y = cube.Y.copy()
    _, _, info = g.covariance(torch.from_numpy(Y).cuda(), precision="mix")
    assert info["status"] == 0 and info["cov_fallback"] == 0
    Y[1, 7] = 5e6                 # the data lie in [0, 1]
    mu, C, info = g.covariance(torch.from_numpy(Y).cuda(), precision="mix")
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["cov_fallback"] == 1
    mu_ref = oracle.band_means(Y)
    C_ref = oracle.covariance(Y, mu_ref)
    assert np.abs(mu.cpu().numpy() - mu_ref).max() / np.abs(mu_ref).max() <= MU_TOL["p32"]
    assert np.abs(C.cpu().numpy() - C_ref).max() / np.abs(C_ref).max() <= COV_TOL["p32"]


@pytest.mark.gpu
def test_mix_fp16_band_with_tiny_spread(gbpca_lib):
    """An FP16 band whose values differ only in the last bits of 0.5 gets a
    power-of-two scale beyond FP16's normal range (2^16 and more): the
    converters then widen those values instead of scaling them in FP16, and
    the fit still matches the oracle."""
    g = gbpca_lib
    cube = synth.linear_mixing(seed=23, rows=41, cols=43, bands=48, endmembers=5)
    Y = cube.Y.copy()
    rng = np.random.default_rng(5)
    Y[:, 9] = 0.5 + 2.0 ** -11 * rng.integers(-1, 2, size=Y.shape[0])   # three FP16 values
    Yd = torch.from_numpy(Y).to(torch.float16)
    Yh = Yd.float().numpy().astype(np.float64)
    mu, ev, V, Q, info = g.fit(Yd.cuda(), cube.k, precision="mix")
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["cov_fallback"] == 0 and info["proj_fallback"] == 0, info
    ref = oracle.pca_fit(Yh, cube.k, tol=1e-14)
    compare((mu.cpu().numpy(), ev.cpu().numpy(), V.cpu().numpy(),
             Q.cpu().numpy().astype(np.float64)), ref, cube.k, "mix")
