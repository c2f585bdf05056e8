"""The kernel count that pca_kernel_launches reports (the benchmark's
gpu_launches) against the kernels one pca_fit really enqueues: the fit is
captured into a CUDA graph and its kernel nodes are counted through the
driver API."""
import ctypes

import pytest
import torch

import synth

CU_GRAPH_NODE_TYPE_KERNEL = 0


def _kernel_nodes(graph) -> int:
    cu = ctypes.CDLL("libcuda.so.1")
    h = ctypes.c_void_p(graph.raw_cuda_graph())
    n = ctypes.c_size_t(0)
    assert cu.cuGraphGetNodes(h, None, ctypes.byref(n)) == 0
    nodes = (ctypes.c_void_p * n.value)()
    assert cu.cuGraphGetNodes(h, nodes, ctypes.byref(n)) == 0
    kernels = 0
    for i in range(n.value):
        t = ctypes.c_int(-1)
        assert cu.cuGraphNodeGetType(ctypes.c_void_p(nodes[i]), ctypes.byref(t)) == 0
        kernels += t.value == CU_GRAPH_NODE_TYPE_KERNEL
    return kernels


@pytest.mark.gpu
@pytest.mark.parametrize("precision,k,bands", [("mix", 20, 64), ("mix", 40, 96), ("mix", 0, 64),
                                               ("p32", 10, 64), ("p32", 33, 64), ("p64", 5, 48)])
def test_kernel_launches_match_a_captured_fit(gbpca_lib, precision, k, bands):
    g = gbpca_lib
    if not hasattr(torch.cuda.CUDAGraph, "raw_cuda_graph"):
        pytest.skip("this torch has no CUDAGraph.raw_cuda_graph")
    c = synth.linear_mixing(seed=3, rows=64, cols=64, bands=bands, endmembers=6)
    Y = torch.from_numpy(c.Y).cuda()
    N, B = Y.shape
    dt = 0
    ws = g.make_workspace(N, B, max(k, 1), dt, precision, Y.device)
    outs = (torch.empty(B, dtype=torch.float64, device="cuda"),
            torch.empty(B, dtype=torch.float64, device="cuda"),
            torch.empty(B, B, dtype=torch.float64, device="cuda"),
            torch.empty(N, max(k, 1), dtype=torch.float32, device="cuda") if k > 0 else None)
    kw = dict(precision=precision, out=outs, workspace=ws, project=k > 0)
    g.fit(Y, max(k, 1), **kw)            # first call: one-time set-up outside the capture
    torch.cuda.synchronize()
    try:
        graph = torch.cuda.CUDAGraph(keep_graph=True)   # the raw graph stays readable
    except TypeError:
        pytest.skip("this torch cannot keep the captured graph")
    with torch.cuda.graph(graph):
        g.fit(Y, max(k, 1), sync=False, **kw)
    torch.cuda.synchronize()
    assert _kernel_nodes(graph) == g.kernel_launches(precision, k)
