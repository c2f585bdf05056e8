"""pca_fit_host (host cube in, host results out, copies overlapped with the
stages in pixel ranges) against the FP64 oracle, through the C ABI: several
ranges with a ragged last one, a last range that would hold one pixel, BF16
input, pageable input memory, and no projection; two calls in flight on two
streams (each with its own buffers) give the results of calls made one by one."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import compare


def _cube(N, B, seed, dtype):
    c = synth.linear_mixing(seed=seed, rows=1, cols=N, bands=B, endmembers=6)
    Y = torch.from_numpy(c.Y).to(dtype)
    return c, Y


@pytest.mark.gpu
@pytest.mark.parametrize("precision,dtype,N,pinned", [
    ("mix", torch.float32, 200_003, True),      # 4 ranges, the last ragged
    ("p32", torch.float32, 65_537, True),       # the 1-pixel tail joins the only range
    ("mix", torch.bfloat16, 140_000, True),
    ("p64", torch.float32, 70_000, False),      # pageable host memory
])
def test_fit_host_against_oracle(gbpca_lib, precision, dtype, N, pinned):
    g = gbpca_lib
    c, Y = _cube(N, 40, 31, dtype)
    Yh = Y.pin_memory() if pinned else Y
    k = 6
    mu, ev, V, Q, info = g.fit_host(Yh, k, tol=1e-12, precision=precision)
    assert info["status"] == 0, info
    ref = oracle.pca_fit(Y.float().numpy().astype(np.float64), k, tol=1e-14)
    m = compare((mu.numpy(), ev.numpy(), V.numpy(), Q.numpy().astype(np.float64)), ref, k,
                precision)
    print(precision, dtype, N, m)
    # the device copy of the cube is the cube
    hb = g.HostFit(N, 40, k, dtype, precision)
    g.fit_host(Yh, k, tol=1e-12, precision=precision, buffers=hb)
    assert torch.equal(hb.cube_dev.cpu(), Y)


@pytest.mark.gpu
def test_fit_host_matches_fit_and_skips_projection(gbpca_lib):
    g = gbpca_lib
    c, Y = _cube(150_000, 64, 32, torch.float32)
    Yh = Y.pin_memory()
    mu, ev, V, Q, info = g.fit_host(Yh, 5, precision="p32", project=False)
    assert Q is None and info["status"] == 0
    mu2, ev2, V2, _, _ = g.fit(Y.cuda(), 5, precision="p32")
    assert np.abs(mu.numpy() - mu2.cpu().numpy()).max() <= 1e-6 * np.abs(mu2.cpu().numpy()).max()
    assert np.abs(ev.numpy()[:5] - ev2.cpu().numpy()[:5]).max() <= 2e-5 * ev2[0].item()


@pytest.mark.gpu
@pytest.mark.parametrize("reserve", [0, 8])
def test_two_fits_in_flight_on_two_streams(gbpca_lib, reserve):
    """Cubes of a stream of scenes: calls alternate between two CUDA streams with
    their own device buffers and host outputs and nothing waits in between, so
    the copies of one call overlap the other's stages.  Every call must give the
    bits a call made on its own gives (also with SMs left to the other call's
    Jacobi, stream_sms_reserve)."""
    g = gbpca_lib
    N, B, k = 150_000, 160, 6
    cubes = [_cube(N, B, 40 + i, torch.bfloat16)[1].pin_memory() for i in range(2)]
    prev = g.set_tuning({**g.tuning(), "stream_sms_reserve": reserve})
    try:
        ref = [g.fit_host(Yh, k, tol=1e-12, precision="mix") for Yh in cubes]
        streams = (torch.cuda.Stream(), torch.cuda.Stream())
        bufs = [g.HostFit(N, B, k, torch.bfloat16, "mix") for _ in range(2)]
        outs = [(torch.empty(B, dtype=torch.float64, pin_memory=True),
                 torch.empty(B, dtype=torch.float64, pin_memory=True),
                 torch.empty(B, B, dtype=torch.float64, pin_memory=True),
                 torch.empty(N, k, dtype=torch.float32, pin_memory=True)) for _ in range(2)]
        for rnd in range(3):
            for i in range(2):
                g.fit_host(cubes[i], k, tol=1e-12, precision="mix", buffers=bufs[i], out=outs[i],
                           sync=False, stream=streams[i])
            for s in streams:
                s.synchronize()
            for i in range(2):
                for a, b in zip(outs[i], ref[i][:4]):
                    assert torch.equal(a, b), (rnd, i)
    finally:
        g.set_tuning(prev)
    Y0 = cubes[0].float().numpy().astype(np.float64)
    compare(tuple(t.numpy().astype(np.float64) for t in ref[0][:4]),
            oracle.pca_fit(Y0, k, tol=1e-14), k, "mix")
