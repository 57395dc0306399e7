"""sp_export_csr_noalloc against sp_export_csr (collected last on purpose).

Callers that must not allocate device memory mid-run (a serving process that
snapshots a live graph into buffers reserved at start-up, code held to a
fixed footprint) use the allocation-free export.  It must give exactly the
arrays the regular device-side export gives, call after call, and must not
grow the graph's or PyTorch's device memory while it runs.
"""
import numpy as np
import pytest

from paper_2507_11094_gb300 import sp
from paper_2507_11094_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2507_11094_gb300 import build
    build.build()
    sp.load()
    return torch


def _export_pair(torch, g, reverse):
    n, m = g.n, g.m
    dev = torch.device("cuda")
    ref = (torch.full((n + 1,), -7, dtype=torch.int64, device=dev),
           torch.full((max(m, 1),), -7, dtype=torch.int32, device=dev),
           torch.full((max(m, 1),), -7, dtype=torch.int32, device=dev))
    out = (torch.full((n + 1,), -9, dtype=torch.int64, device=dev),
           torch.full((max(m, 1),), -9, dtype=torch.int32, device=dev),
           torch.full((max(m, 1),), -9, dtype=torch.int32, device=dev))
    g.export_csr_device(*ref, reverse=reverse)
    torch.cuda.synchronize()
    held = g.info().device_bytes
    torch_held = torch.cuda.memory_allocated()
    g.export_csr_device(*out, reverse=reverse, noalloc=True)
    torch.cuda.synchronize()
    assert g.info().device_bytes == held
    assert torch.cuda.memory_allocated() == torch_held
    return ref, out


def test_noalloc_export_matches_regular_export_twice(torch_cuda):
    torch = torch_cuda
    W = wl.rmat(scale=14, batch_frac=0.02, seed=3)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        g.sssp_init(W.source)
        g.apply(W.batch(0))
        for reverse in (False, True):          # two calls in a row
            ref, out = _export_pair(torch, g, reverse)
            for a, b in zip(ref, out):
                np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
        g.apply(W.batch(1))
        ref, out = _export_pair(torch, g, False)
        for a, b in zip(ref, out):
            np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
        # and the exported forward store is the generator's edge set
        ro, col, w = W.stream.csr()
        np.testing.assert_array_equal(out[0].cpu().numpy(), ro)
        np.testing.assert_array_equal(out[1].cpu().numpy()[:col.size], col)
        np.testing.assert_array_equal(out[2].cpu().numpy()[:col.size], w)


def test_noalloc_export_above_one_scan_tile(torch_cuda):
    """A graph of more than 2048 x 2048 vertices: the scan of the degrees
    recurses over a second level of partial sums, still inside the fixed
    array; two exports in a row equal the regular export."""
    torch = torch_cuda
    W = wl.grid(2100, 2100, batch_frac=0.001, seed=2)
    assert W.n > 2048 * 2048
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        for reverse in (False, True):
            ref, out = _export_pair(torch, g, reverse)
            for a, b in zip(ref, out):
                np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
        np.testing.assert_array_equal(out[0].cpu().numpy()[-1], W.m)
