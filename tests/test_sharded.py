"""Pixel-sharded fit (fit_sharded): the exchange of per-rank moments (the
common shift from rank 0, one all-reduce of shifted sums), the pooled
eigen-solve on rank 0 and its broadcast, on CPU ranks (gloo, world sizes 2
and 3, uneven shards including a one-pixel shard).  The stages are the FP64
oracle's here, so every rank must reproduce the oracle's fit of the whole
cube; the GPU kernels of the exchange have their own tests in
test_gpu_sharded.py."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class OracleOps:
    """The stages on the CPU, from the oracle (test scaffolding only)."""

    def moments(self, cube):
        import torch

        import oracle
        Y = cube.numpy()
        mu = oracle.band_means(Y)
        C = oracle.covariance(Y) if Y.shape[0] > 1 else np.zeros((Y.shape[1], Y.shape[1]))
        return torch.from_numpy(mu), torch.from_numpy(C)

    def shifted_sums(self, n, mu, C, s):
        # (n, S1, S2 upper) about the common shift, written out for the CPU ranks
        import torch
        d = mu.numpy() - s.numpy()
        S2 = (n - 1.0) * C.numpy() + n * np.outer(d, d)
        iu = np.triu_indices(len(d))
        return torch.from_numpy(np.concatenate([[float(n)], n * d, S2[iu]]))

    def from_sums(self, sums, s):
        import torch
        v, sv = sums.numpy(), s.numpy()
        B = len(sv)
        n, S1 = v[0], v[1:1 + B]
        S2 = np.zeros((B, B))
        S2[np.triu_indices(B)] = v[1 + B:]
        S2 = S2 + np.triu(S2, 1).T
        return torch.from_numpy(sv + S1 / n), torch.from_numpy((S2 - np.outer(S1, S1) / n) / (n - 1.0))

    def eigh(self, C):
        import torch

        import oracle
        Ak, V, info = oracle.jacobi(C.numpy(), tol=1e-14)
        lam, Vs = oracle.sort_sign(np.diag(Ak).copy(), V)
        return torch.from_numpy(lam), torch.from_numpy(Vs), info

    def project(self, cube, mu, V, k):
        import torch

        import oracle
        return torch.from_numpy(oracle.project(cube.numpy(), mu.numpy(), V.numpy(), k))


def _worker(rank, world, port, bounds, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    import paper_2403_18321_gb300 as g
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cube = synth.linear_mixing(seed=77, rows=30, cols=41, bands=24, endmembers=6, k=4)
    lo, hi = bounds[rank], bounds[rank + 1]
    mine = torch.from_numpy(cube.Y[lo:hi].astype(np.float64))
    mu, ev, V, Q, info = g.fit_sharded(mine, 4, ops=OracleOps())
    q.put((rank, mu.numpy(), ev.numpy(), V.numpy(), Q.numpy(), info is not None))
    dist.destroy_process_group()


@pytest.mark.parametrize("bounds", [(0, 700, 1230), (0, 1, 500, 1230)])
def test_sharded_fit_matches_the_whole_cube(bounds):
    import oracle
    import synth
    world, port = len(bounds) - 1, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, bounds, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=180) for _ in range(world)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cube = synth.linear_mixing(seed=77, rows=30, cols=41, bands=24, endmembers=6, k=4)
    ref = oracle.pca_fit(cube.Y, 4, tol=1e-14)
    lam1 = ref["lam"][0]
    for rank, mu, ev, V, Q, has_info in out:
        assert has_info == (rank == 0)
        assert np.abs(mu - ref["mu"]).max() <= 1e-13 * np.abs(ref["mu"]).max()
        assert np.abs(ev - ref["lam"]).max() <= 1e-11 * lam1
        # the leading (well separated) vectors individually, sign-normalised by both sides
        assert np.abs(V[:, :4] - ref["V"][:, :4]).max() <= 1e-9
        lo, hi = bounds[rank], bounds[rank + 1]
        assert np.abs(Q - ref["Q"][lo:hi]).max() <= 1e-9 * np.abs(ref["Q"]).max()
    # every rank holds the same bits of the eigen-pairs (broadcast from rank 0)
    for _, _, ev, V, _, _ in out[1:]:
        assert np.array_equal(ev, out[0][2]) and np.array_equal(V, out[0][3])
