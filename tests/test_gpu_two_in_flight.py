"""Two device-resident fits in flight on two CUDA streams, as a stream of
scenes is fitted: with or without the SMs the streaming kernels leave to the
other fit's Jacobi (stream_sms_reserve), every fit gives the bits of the same
fit made alone, and those match the FP64 oracle as any MIX fit does."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import compare


@pytest.mark.gpu
@pytest.mark.parametrize("reserve", [0, 8])
def test_two_fits_in_flight(gbpca_lib, reserve):
    g = gbpca_lib
    k, N, B = 8, 48_000, 224
    cubes = []
    for i in range(2):
        c = synth.linear_mixing(seed=60 + i, rows=1, cols=N, bands=B, endmembers=7)
        cubes.append(torch.from_numpy(c.Y).to(torch.bfloat16).cuda())
    prev = g.set_tuning({"stream_sms_reserve": reserve})
    try:
        alone = [g.fit(Y, k, tol=1e-10, precision="mix") for Y in cubes]
        for r in alone:
            assert r[4]["status"] == 0, r[4]
        ws = [g.make_workspace(N, B, k, 1, "mix", cubes[0].device) for _ in range(2)]
        outs = [(torch.empty(B, dtype=torch.float64, device="cuda"),
                 torch.empty(B, dtype=torch.float64, device="cuda"),
                 torch.empty(B, B, dtype=torch.float64, device="cuda"),
                 torch.empty(N, k, dtype=torch.float32, device="cuda")) for _ in range(2)]
        streams = (torch.cuda.Stream(), torch.cuda.Stream())
        for rnd in range(3):
            for i in range(2):
                g.fit(cubes[i], k, tol=1e-10, precision="mix", out=outs[i], workspace=ws[i],
                      sync=False, stream=streams[i])
            for s in streams:
                s.synchronize()
            for i in range(2):
                for a, b in zip(outs[i], alone[i][:4]):
                    assert torch.equal(a, b), (reserve, rnd, i)
    finally:
        g.set_tuning(prev)
    Y0 = cubes[0].float().cpu().numpy().astype(np.float64)
    ref = oracle.pca_fit(Y0, k, tol=1e-14)
    mu, ev, V, Q, _ = alone[0]
    compare((mu.cpu().numpy(), ev.cpu().numpy(), V.cpu().numpy(),
             Q.cpu().numpy().astype(np.float64)), ref, k, "mix")
