"""Band-sequential input (pca_bsq_to_bip): the conversion against PyTorch's own
transpose, byte for byte, on ragged shapes; and a fit of a BSQ cube equal to
the fit of the same cube in pixel-major order (identical bytes in, identical
bits out), checked against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import compare


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("shape", [(1, 1), (5, 7), (103, 1000), (224, 4161), (256, 64)])
def test_bsq_to_bip_is_the_transpose(gbpca_lib, dtype, shape):
    g = gbpca_lib
    B, N = shape
    gen = torch.Generator(device="cuda").manual_seed(B * 1000 + N)
    bsq = torch.randn(B, N, generator=gen, device="cuda").to(dtype)
    bip = g.bsq_to_bip(bsq)
    torch.cuda.synchronize()
    assert bip.shape == (N, B)
    assert torch.equal(bip.view(torch.int16 if dtype != torch.float32 else torch.int32),
                       bsq.t().contiguous().view(torch.int16 if dtype != torch.float32 else torch.int32))


@pytest.mark.gpu
@pytest.mark.parametrize("form", ["mix", "p32"])
def test_fit_of_bsq_cube_equals_pixel_major_fit(gbpca_lib, form):
    g = gbpca_lib
    cube = synth.paper_scene(5, 61, 37, 103, k=6)
    bip = torch.from_numpy(cube.Y).cuda()
    bsq = bip.t().contiguous()
    a = g.fit(bsq, 6, precision=form, layout="bsq")
    b = g.fit(bip, 6, precision=form)
    torch.cuda.synchronize()
    for x, y in zip(a[:4], b[:4]):
        assert torch.equal(x, y)
    ref = oracle.pca_fit(cube.Y, 6, tol=1e-14)
    compare(tuple(t.cpu().numpy().astype(np.float64) for t in a[:4]), ref, 6, form)
