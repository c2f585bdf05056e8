"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded cubes.  Sizes span several chunks/tiles with ragged tails, odd
band counts (padding index), the smallest and largest band counts, and the
status paths (non-finite input, non-convergence, bad arguments)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import compare

FORMS = ["p32", "mix", "p64"]


def run(g, Y, k, form, tol=1e-10, sweeps_max=30, project=True):
    Yt = torch.as_tensor(Y).to("cuda")
    mu, ev, V, Q, info = g.fit(Yt, k, tol=tol, sweeps_max=sweeps_max, precision=form,
                               project=project)
    torch.cuda.synchronize()
    out = (mu.cpu().numpy(), ev.cpu().numpy(), V.cpu().numpy(),
           Q.cpu().numpy().astype(np.float64) if Q is not None else None)
    return out, info


def skip_if_unsupported(g, form, B):
    if form == "mix" and g.workspace_size(1000, B, 1, 0, "mix") == 0:
        pytest.skip("tensor-core covariance not available for this B")


@pytest.mark.gpu
@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("shape", [(37, 41, 64, 4), (61, 34, 103, 10), (23, 29, 7, 3),
                                   (50, 51, 128, 5), (17, 11, 2, 1), (9, 7, 3, 2),
                                   (1, 2, 16, 1)])
def test_linear_mixing_small(gbpca_lib, form, shape):
    rows, cols, B, k = shape
    skip_if_unsupported(gbpca_lib, form, B)
    e = max(1, min(5, B - 1))
    cube = synth.linear_mixing(seed=rows * cols + B, rows=rows, cols=cols, bands=B, endmembers=e)
    ref = oracle.pca_fit(cube.Y, k, tol=1e-14)
    out, info = run(gbpca_lib, cube.Y, k, form)
    assert info["status"] == 0, info
    compare(out, ref, k, form)


@pytest.mark.gpu
@pytest.mark.parametrize("form", FORMS)
def test_paper_scene_reduced(gbpca_lib, form):
    for cube in synth.paper_scenes(scale=0.2):
        skip_if_unsupported(gbpca_lib, form, cube.B)
        ref = oracle.pca_fit(cube.Y, cube.k, tol=1e-14)
        out, info = run(gbpca_lib, cube.Y, cube.k, form)
        assert info["status"] == 0, info
        compare(out, ref, cube.k, form)


@pytest.mark.gpu
@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("bands", [232, 255, 256])
def test_max_bands(gbpca_lib, form, bands):
    """Up to the largest band count: both 128-row tensor-core tiles full (256),
    an odd count with the padding index (255), and 8-CTA Jacobi clusters."""
    skip_if_unsupported(gbpca_lib, form, bands)
    cube = synth.linear_mixing(seed=5, rows=30, cols=40, bands=bands, endmembers=8)
    ref = oracle.pca_fit(cube.Y, 8, tol=1e-14)
    out, info = run(gbpca_lib, cube.Y, 8, form)
    assert info["status"] == 0, info
    compare(out, ref, 8, form)


@pytest.mark.gpu
def test_constant_cube_gives_zero_spectrum(gbpca_lib):
    Y = np.full((1000, 16), 3.25, dtype=np.float32)
    for form in ("p32", "p64"):
        (mu, lam, V, Q), info = run(gbpca_lib, Y, 3, form)
        assert info["status"] == 0 and info["sweeps"] == 0
        assert np.all(lam == 0.0) and np.allclose(mu, 3.25)
        assert np.array_equal(V, np.eye(16)) and np.all(Q == 0.0)


@pytest.mark.gpu
def test_nonfinite_cube_is_reported(gbpca_lib):
    Y = synth.linear_mixing(seed=1, rows=20, cols=20, bands=16).Y.copy()
    Y[123, 5] = np.nan
    _, info = run(gbpca_lib, Y, 2, "p32")
    assert info["status"] == 3
    Y[123, 5] = np.inf
    _, info = run(gbpca_lib, Y, 2, "p64")
    assert info["status"] == 3


@pytest.mark.gpu
def test_sweep_limit_reports_noconv_with_last_iterate(gbpca_lib):
    cube = synth.linear_mixing(seed=2, rows=30, cols=30, bands=48, endmembers=5)
    (mu, lam, V, Q), info = run(gbpca_lib, cube.Y, 3, "p32", sweeps_max=1)
    assert info["status"] == 2 and info["sweeps"] == 1
    assert np.abs(V.T @ V - np.eye(48)).max() < 1e-4
    ref = oracle.pca_fit(cube.Y, 3, tol=1e-14)
    assert abs(lam.sum() - ref["lam"].sum()) <= 1e-4 * abs(ref["lam"]).sum()


@pytest.mark.gpu
def test_bad_arguments_are_rejected_on_the_host(gbpca_lib):
    g = gbpca_lib
    lib = g.load()
    Y = torch.zeros(100, 8, device="cuda")
    bad = [dict(k=0), dict(k=9), dict(tol=0.0), dict(tol=float("nan")), dict(sweeps_max=0)]
    for kw in bad:
        args = dict(k=2, tol=1e-10, sweeps_max=30)
        args.update(kw)
        with pytest.raises(g.PCAError) as e:
            g.fit(Y, args["k"], tol=args["tol"], sweeps_max=args["sweeps_max"], precision="p32")
        assert e.value.status == 1
    assert lib.pca_workspace_size(1, 8, 2, 0, 1) == 0          # N < 2
    assert lib.pca_workspace_size(100, 1, 1, 0, 1) == 0        # B < 2
    assert lib.pca_workspace_size(100, 257, 2, 0, 1) == 0      # B too large
    assert lib.pca_workspace_size(100, 256, 2, 0, 1) > 0
    with pytest.raises(g.PCAError):                            # misaligned cube pointer
        g.fit(Y.view(-1)[1:793].view(99, 8), 2, precision="p32")


@pytest.mark.gpu
@pytest.mark.parametrize("form", FORMS)
def test_paper_scenes_full_size(gbpca_lib, form):
    """The benchmarked workload at full size (610x340x103 and 512x217x224), whole
    outputs against the oracle (multi-threaded on the host)."""
    oracle.set_threads(0)
    for cube in synth.paper_scenes(scale=1.0):
        skip_if_unsupported(gbpca_lib, form, cube.B)
        ref = oracle.pca_fit(cube.Y, cube.k, tol=1e-14)
        out, info = run(gbpca_lib, cube.Y, cube.k, form)
        assert info["status"] == 0, info
        compare(out, ref, cube.k, form)


@pytest.mark.gpu
@pytest.mark.parametrize("form", FORMS)
def test_plain_pca_config_exact(gbpca_lib, form):
    """Plain PCA exactly as specified: 100 x 100 pixels x 128 bands, 5 endmembers
    (U[0,1] spectra, Dirichlet(1) abundances, 0.01 Gaussian noise), seed 0, k = 5,
    tol 1e-10, 30 sweeps; whole outputs against the oracle."""
    cube = synth.linear_mixing()
    assert (cube.N, cube.B, cube.k) == (10000, 128, 5)
    ref = oracle.pca_fit(cube.Y, cube.k, tol=1e-14)
    out, info = run(gbpca_lib, cube.Y, cube.k, form, tol=cube.tol, sweeps_max=cube.sweeps_max)
    assert info["status"] == 0, info
    # P64 at FP64 accuracy for the signal components (endmembers - 1 of them);
    # the noise eigenvalues beyond form a cluster (include/gbpca.h)
    kc = min(cube.k, 4) if form == "p64" else cube.k
    mu, lam, V, Q = out
    compare((mu, lam, V, Q[:, :kc]), ref, kc, form)


@pytest.mark.gpu
@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("p2", [-40, 40])
def test_cube_scaled_by_a_power_of_two(gbpca_lib, form, p2):
    """A cube scaled by 2^p2 (values near 1e-12 or 1e12, covariance entries near
    1e-26 or 1e22) fits like the unscaled one: the Jacobi's rotation angles are
    formed from differences and products of covariance entries, whose squares
    would leave the FP32 range at these scales (the scale-free form is taken
    there).  Eigenvalues scale by 2^(2 p2), eigenvectors and the projection's
    parity with the oracle are unchanged."""
    cube = synth.linear_mixing(seed=91, rows=30, cols=40, bands=64, endmembers=5)
    Ys = (cube.Y.astype(np.float64) * 2.0 ** p2).astype(np.float32)
    k = 4
    ref = oracle.pca_fit(Ys.astype(np.float64), k, tol=1e-14)
    out, info = run(gbpca_lib, Ys, k, form)
    assert info["status"] == 0, info
    compare(out, ref, k, form)
