"""xtn_tcrdist_filter_noalloc: the TCRdist filter for callers that cannot
allocate device memory -- a process held to a fixed device-memory budget, or
a library running inside a host application whose own allocator owns the
device memory.  Its scratch lives in one fixed device array, so it must give
exactly the rows of xtn_tcrdist_filter, call after call, without the device's
free memory changing.  This file is collected last so a failure here never
hides the other tests."""
import ctypes

import numpy as np
import pytest

import cdr3_synth as gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2403_09010_gb300 as pkg
    from paper_2403_09010_gb300 import native
    pkg.build()
    return native.lib()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _filter(lib, fn, seqs, off, rows, thr, stream):
    out = torch.empty_like(rows)
    n_out = ctypes.c_int64(-1)
    rc = getattr(lib, fn)(_p(seqs), _p(off), off.numel() - 1, _p(rows), rows.shape[0], thr,
                          _p(out), ctypes.byref(n_out), stream)
    return rc, out[: max(n_out.value, 0)].cpu().numpy()


def test_noalloc_matches_allocating_filter_twice(lib):
    from paper_2403_09010_gb300 import native
    import paper_2403_09010_gb300 as xtn
    s, o = gen.workload(gen.TCRDIST_1M, 20_000)
    seqs = torch.from_numpy(s).cuda()
    off = torch.from_numpy(o).cuda()
    rows = xtn.search_self(seqs, off, 2)            # (rows, 3) int32 on the device
    assert rows.shape[0] > 1000
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # first call sets up the device address of the scratch array
    rc, _ = _filter(lib, "xtn_tcrdist_filter_noalloc", seqs, off, rows, 24, stream)
    assert rc == native.XTN_OK
    results = []
    for thr in (24, 9):                              # two calls in a row, different outputs
        rc_ref, want = _filter(lib, "xtn_tcrdist_filter", seqs, off, rows, thr, stream)
        assert rc_ref == native.XTN_OK
        rc, got = _filter(lib, "xtn_tcrdist_filter_noalloc", seqs, off, rows, thr, stream)
        assert rc == native.XTN_OK
        assert got.shape == want.shape and np.array_equal(got, want), thr
        results.append(got.shape[0])
    assert results[0] > results[1] > 0
    # the no-alloc calls alone leave the device's free memory exactly as it was
    outs = [torch.empty_like(rows) for _ in range(2)]
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for out in outs:
        n_out = ctypes.c_int64(-1)
        rc = lib.xtn_tcrdist_filter_noalloc(_p(seqs), _p(off), off.numel() - 1, _p(rows),
                                            rows.shape[0], 24, _p(out), ctypes.byref(n_out),
                                            stream)
        assert rc == native.XTN_OK and n_out.value == results[0]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    assert torch.equal(outs[0][: results[0]], outs[1][: results[0]])


def test_noalloc_rejects_what_it_cannot_hold(lib):
    from paper_2403_09010_gb300 import native
    n_out = ctypes.c_int64(7)
    big = native.XTN_NOALLOC_MAX_SEQS + 1
    off = torch.zeros(big + 1, dtype=torch.int64, device="cuda")
    seqs = torch.zeros(1, dtype=torch.uint8, device="cuda")
    rows = torch.zeros((4, 3), dtype=torch.int32, device="cuda")
    out = torch.empty_like(rows)
    rc = lib.xtn_tcrdist_filter_noalloc(_p(seqs), _p(off), big, _p(rows), 4, 24, _p(out),
                                        ctypes.byref(n_out), None)
    assert rc == native.XTN_ERR_TOO_LARGE and n_out.value == 0
    # host buffers would need device copies: rejected
    h_rows = np.zeros((4, 3), np.uint32)
    off_small = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    rc = lib.xtn_tcrdist_filter_noalloc(_p(seqs), _p(off_small), 1, h_rows.ctypes.data, 4, 24,
                                        _p(out), ctypes.byref(n_out), None)
    assert rc == native.XTN_ERR_INVALID_ARG
