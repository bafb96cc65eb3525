"""The allocation-free bucket sort (dig_sort_by_cell_noalloc) against the
regular one (dig_sort_by_cell, caller-provided scratch), through the C ABI.

The allocation-free entry point is for callers that cannot allocate device
memory: it takes its working memory from a fixed array inside the library.
Both entry points must give bit-identical outputs, also on consecutive calls
that reuse the same fixed array (its previous contents must not leak into the
next result).  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_08195_gb300 import dig  # noqa: E402

MAX_N, MAX_CELLS = 4194304, 1048576  # DIG_NOALLOC_MAX_N / DIG_NOALLOC_MAX_CELLS in include/dig.h


def regular(L, cell, n_cells, stream):
    n = cell.numel()
    nb = C.c_int64(0)
    assert L.dig_sort_scratch_bytes(n, n_cells, C.byref(nb)) == 0
    scratch = torch.empty(nb.value + 256, dtype=torch.uint8, device=cell.device)
    sp = (scratch.data_ptr() + 255) & ~255
    cs = torch.full((n_cells + 1,), -7, dtype=torch.int32, device=cell.device)
    order = torch.full((max(n, 1),), -7, dtype=torch.int32, device=cell.device)
    rc = L.dig_sort_by_cell(C.c_void_p(cell.data_ptr()), n, n_cells, C.c_void_p(cs.data_ptr()),
                            C.c_void_p(order.data_ptr()), C.c_void_p(sp), nb.value, C.c_void_p(stream.cuda_stream))
    assert rc == 0, L.dig_last_error(None)
    stream.synchronize()
    return cs.cpu().numpy(), order.cpu().numpy()[: int(cs[-1].item())]


def noalloc(L, cell, n_cells, stream):
    n = cell.numel()
    cs = torch.full((n_cells + 1,), -7, dtype=torch.int32, device=cell.device)
    order = torch.full((max(n, 1),), -7, dtype=torch.int32, device=cell.device)
    rc = L.dig_sort_by_cell_noalloc(C.c_void_p(cell.data_ptr()), n, n_cells, C.c_void_p(cs.data_ptr()),
                                    C.c_void_p(order.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == 0, L.dig_last_error(None)
    stream.synchronize()
    return cs.cpu().numpy(), order.cpu().numpy()[: int(cs[-1].item())]


def test_noalloc_matches_regular_on_consecutive_calls():
    L = dig.load_library()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(12)
    # first call large (dense counters everywhere), second call smaller with
    # fewer cells: stale counts or orders from the first call would show up
    for n, n_cells in ((MAX_N, 162_000), (300_001, 1296), (MAX_N // 3, MAX_CELLS)):
        cell = torch.from_numpy(rng.integers(-1, n_cells, size=n).astype(np.int32)).cuda()
        cs_r, ord_r = regular(L, cell, n_cells, stream)
        cs_n, ord_n = noalloc(L, cell, n_cells, stream)
        assert np.array_equal(cs_n, cs_r)
        assert np.array_equal(ord_n, ord_r)
        assert cs_r[-1] == int((cell >= 0).sum().item())


def test_noalloc_rejects_sizes_beyond_its_limits():
    L = dig.load_library()
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = C.c_void_p(dummy.data_ptr())
    assert L.dig_sort_by_cell_noalloc(p, MAX_N + 1, 10, p, p, s) == -3
    assert b"limits" in L.dig_last_error(None)
    assert L.dig_sort_by_cell_noalloc(p, 10, MAX_CELLS + 1, p, p, s) == -3
