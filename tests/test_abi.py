"""CPU checks of the C ABI: the library builds, loads, and exports every entry
point include/gbpca.h declares.  No compute call (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbpca.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pca_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pca_fit", "pca_workspace_size", "pca_status_string", "pca_read_info"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2403_18321_gb300 import _build
    lib_path = _build.build()
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in gbpca.h but not exported"


def test_status_strings_and_version_need_no_gpu():
    import paper_2403_18321_gb300 as g
    lib = g.load(build_if_missing=True)
    assert lib.pca_version() >= 100
    for code in range(7):
        assert lib.pca_status_string(code)
    assert lib.pca_status_string(99) == b"unknown status"


def test_binding_names_match_the_abi():
    import paper_2403_18321_gb300 as g
    assert set(g.EXPORTS) <= set(declared_functions())


def test_binding_refuses_cpu_tensors():
    import torch
    import paper_2403_18321_gb300 as g
    with pytest.raises(TypeError):
        g.fit(torch.zeros(10, 4), 2)


def test_batch_workspace_size_is_host_only_and_checks_every_tile():
    """pca_batch_workspace_size lays out a batch on the host: positive for valid
    tiles, 0 as soon as one tile is invalid, growing with the tiles."""
    import paper_2403_18321_gb300 as g
    lib = g.load(build_if_missing=True)

    def tiles(shapes):
        arr = (g.Tile * len(shapes))()
        for i, (N, B, k) in enumerate(shapes):
            arr[i] = g.Tile(None, N, B, k, None, None, None, None)
        return arr

    ok = [(4096, 64, 8), (100, 7, 3), (262144, 256, 8), (2, 2, 1)]
    for prec in (0, 1, 2):
        one = lib.pca_batch_workspace_size(1, tiles(ok[:1]), 0, prec)
        four = lib.pca_batch_workspace_size(4, tiles(ok), 0, prec)
        assert one > 0 and four > one
    assert lib.pca_batch_workspace_size(2, tiles([(4096, 64, 8), (100, 257, 3)]), 0, 1) == 0
    assert lib.pca_batch_workspace_size(2, tiles([(4096, 64, 8), (1, 8, 3)]), 0, 1) == 0
    assert lib.pca_batch_workspace_size(2, tiles([(4096, 64, 8), (100, 8, 9)]), 0, 1) == 0
    assert lib.pca_batch_workspace_size(0, tiles(ok), 0, 1) == 0


def test_workspace_sizes_accept_every_k_up_to_B():
    """1 <= k <= B (Algorithm 1 stages 5-6 project onto any number of
    components); sizes are computed on the host."""
    import paper_2403_18321_gb300 as g
    lib = g.load(build_if_missing=True)
    for prec in (0, 1, 2):
        for B, k in ((256, 256), (224, 33), (103, 103), (2, 2)):
            assert lib.pca_workspace_size(1000, B, k, 0, prec) > 0, (B, k, prec)
        assert lib.pca_workspace_size(1000, 64, 65, 0, prec) == 0
    assert lib.pca_backward_workspace_size(1000, 256, 256) > 0
    assert lib.pca_backward_workspace_size(1000, 256, 257) == 0
