"""Allocation-free column statistics against the context-based path.

rise_column_stats_noalloc serves callers that may not allocate device memory
(a host framework that owns all of it and forbids allocation in its per-frame
callbacks, or a real-time loop where a cudaMalloc could synchronise the device
and stall other streams).  It keeps its column histograms in one fixed device
array shared by every call, so each test here makes two calls in a row: the
second one only comes out right if the first call's counts were cleared.
Both are checked against rise_detect_image (which allocates its scratch in a
context) and against the FP64 oracle's column histograms and exhaustive Otsu
search on the same image: S and the Otsu threshold are integers, so they must
agree exactly.  One test orders two calls on two streams with an event, the
way a caller with several streams keeps them from racing on the shared
array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _image(T, F, seed):
    # noise floor with a slow ripple across frequency, plus bright blocks of
    # varied size and level: columns with and without an Otsu split
    rng = np.random.default_rng(seed)
    base = 60 + 20 * np.sin(np.arange(F) / 37.0)
    q = np.clip(rng.normal(base, 6.0, size=(T, F)), 0, 255)
    for _ in range(40):
        t0, f0 = rng.integers(0, T), rng.integers(0, F)
        q[t0:t0 + rng.integers(2, 400), f0:f0 + rng.integers(2, 300)] += rng.integers(40, 150)
    q = np.clip(q, 0, 255).astype(np.uint8)
    q[:, :7] = 255      # constant columns: no split
    q[:, 8] = 0
    return q


def _via_context(det, img):
    from paper_2603_20481_gb300 import rise
    T, F = img.shape
    det.detect_image(img)
    return det.debug(rise.DBG_COLSTATS, T, F)


def _via_noalloc(img, stream=None):
    import torch
    from paper_2603_20481_gb300 import rise
    F = img.shape[1]
    cols = torch.full((F * rise.COLSTAT_DTYPE.itemsize,), 0xAB, dtype=torch.uint8, device=img.device)
    rc = rise.column_stats_noalloc(img, cols, stream)
    assert rc == rise.RISE_OK, rise.strerror(rc)
    (stream or torch.cuda.current_stream()).synchronize()
    return cols.cpu().numpy().view(rise.COLSTAT_DTYPE)


def _check(got, want, img=None):
    np.testing.assert_array_equal(got["S"], want["S"])
    np.testing.assert_array_equal(got["otsu"], want["otsu"])
    assert not got["Shat"].any() and not got["keep"].any()
    assert not got["eff"].any() and not got["pad"].any()
    if img is not None:
        import oracle
        q = img.cpu().numpy()
        ref = oracle.column_thresholds(oracle.column_hist(q), q.shape[0])
        np.testing.assert_array_equal(got["S"], ref["S"])
        np.testing.assert_array_equal(got["otsu"], ref["otsu"])


@pytest.mark.parametrize("shapes", [
    ((3001, 1024), (3001, 1024)),        # same size twice: every counter reused
    ((70001, 4096), (517, 256)),          # the largest F, then a small ragged image
])
def test_two_calls_in_a_row_match_the_context_path(det, shapes):
    import torch
    for k, (T, F) in enumerate(shapes):
        img = torch.from_numpy(_image(T, F, 40 + k)).cuda()
        _check(_via_noalloc(img), _via_context(det, img), img)


def test_on_a_side_stream(det):
    import torch
    s = torch.cuda.Stream()
    for k in range(2):
        img = torch.from_numpy(_image(2048, 2048, 60 + k)).cuda()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            got = _via_noalloc(img, s)
        _check(got, _via_context(det, img))


def test_two_streams_ordered_by_an_event(det):
    """The first call runs on stream a, the second on stream b after an event
    recorded behind the first: the second call's clear of the shared array
    waits for the first call's counts to be used, so both results are right."""
    import torch
    from paper_2603_20481_gb300 import rise
    imgs = [torch.from_numpy(_image(4099, 1024, 80 + k)).cuda() for k in range(2)]
    torch.cuda.synchronize()
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    outs = [torch.full((1024 * rise.COLSTAT_DTYPE.itemsize,), 0xAB, dtype=torch.uint8, device="cuda")
            for _ in range(2)]
    done = torch.cuda.Event()
    assert rise.column_stats_noalloc(imgs[0], outs[0], a) == rise.RISE_OK
    done.record(a)
    b.wait_event(done)
    assert rise.column_stats_noalloc(imgs[1], outs[1], b) == rise.RISE_OK
    b.synchronize()
    a.synchronize()
    for img, out in zip(imgs, outs):
        _check(out.cpu().numpy().view(rise.COLSTAT_DTYPE), _via_context(det, img), img)


def test_rejects_what_it_cannot_hold(det):
    import torch
    from paper_2603_20481_gb300 import rise
    L = rise.lib()
    cols = torch.zeros(8192 * rise.COLSTAT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    img = torch.zeros((64, 8192), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert rise.column_stats_noalloc(img, cols) == rise.RISE_ESCRATCH
    assert rise.strerror(rise.RISE_ESCRATCH) != "unknown"
    assert L.rise_column_stats_noalloc(ctypes.c_void_p(img.data_ptr()), 0, 256,
                                       ctypes.c_void_p(cols.data_ptr()), stream) == rise.RISE_EINVAL
    assert L.rise_column_stats_noalloc(ctypes.c_void_p(img.data_ptr()), 64, 384,
                                       ctypes.c_void_p(cols.data_ptr()), stream) == rise.RISE_EINVAL
    assert L.rise_column_stats_noalloc(None, 64, 256, ctypes.c_void_p(cols.data_ptr()),
                                       stream) == rise.RISE_EINVAL
    host = np.zeros((64, 256), np.uint8)       # host memory is refused before any launch
    assert L.rise_column_stats_noalloc(ctypes.c_void_p(host.ctypes.data), 64, 256,
                                       ctypes.c_void_p(cols.data_ptr()), stream) == rise.RISE_EINVAL
    assert not cols.any().item()                # nothing was written
