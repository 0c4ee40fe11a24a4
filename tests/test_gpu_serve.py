"""Serving: continuous batching over chunks from many radio streams.

Each chunk's result must not depend on what shares its batch or lane: the
same chunks are served one at a time (one lane, batches of one) and all
interleaved (several lanes, large batches), and every (stream, chunk) result
must be identical.  Every result is also checked against the FP64 oracle on
the samples the stream carries into the chunk followed by the chunk itself,
assembled here on the host (which checks the carry kept on the device): the
server keeps the 8-bit image each result was detected on, that image is
within one level of the oracle's on at most ceil(1e-5 px) + 6 pixels, and the
boxes equal the oracle run on that image, bit for bit.  Window mode is
checked the same way, plot by plot.  Results also equal rise_detect on the
same samples.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_20481_gb300 import synth

pytestmark = pytest.mark.gpu

N, HOP = 2048, 1024


def _oracle_check(x, boxes, img, what):
    """Boxes bit-exact against the oracle on the served image; the image
    within the one-level budget of the oracle's FP64 image of samples x."""
    np.testing.assert_array_equal(boxes, oracle.detect_image(img), err_msg=what)
    _, qr, _ = oracle.detect(x, N, HOP)
    assert img.shape == qr.shape, what
    d = img.astype(np.int16) - qr.astype(np.int16)
    assert np.abs(d).max(initial=0) <= 1, what
    assert np.count_nonzero(d) <= math.ceil(1e-5 * img.size) + 6, what


def _chunks(streams, per_stream, n=61440 + 512):
    # chunk length not a multiple of the hop: the carry length varies
    return {s: [synth.served_chunk(s, k, n=n).iq for k in range(per_stream)] for s in range(streams)}


def _assemble(chunks):
    """Host restatement of the stream carry: (capture, frames, first_frame) per chunk."""
    carry = np.zeros(0, np.complex64)
    out, frame = [], 0
    for ch in chunks:
        x = np.concatenate([carry, ch])
        T = (len(x) - N) // HOP + 1 if len(x) >= N else 0
        out.append((x, T, frame))
        frame += T
        carry = x[T * HOP:]
    return out


def _serve(chunks, order, images=None, **kw):
    """Serves the chunks in `order`; with `images` (a dict) the server keeps
    every result's 8-bit image and they are collected into it."""
    import torch
    from paper_2603_20481_gb300 import rise
    pinned = {s: [torch.from_numpy(c).pin_memory() for c in cs] for s, cs in chunks.items()}
    res = {}
    with rise.Server(N, HOP, max_chunk=max(len(c) for cs in chunks.values() for c in cs),
                     max_streams=max(chunks) + 1, keep_images=images is not None, **kw) as srv:
        for s, k in order:
            while not srv.submit(s, pinned[s][k], tag=1000 * s + k):
                for d, b in srv.poll(timeout_ms=5):
                    res[(d["stream"], d["seq"])] = (d, b)
        srv.drain()
        while len(res) < len(order):
            for d, b in srv.poll(timeout_ms=100):
                res[(d["stream"], d["seq"])] = (d, b)
        if images is not None:
            for key, (d, _) in res.items():
                if d["frames"] > 0:
                    images[key] = srv.result_image(*key)
        stats = srv.stats()
    return res, stats


def test_alone_and_in_the_mix_are_identical(det):
    chunks = _chunks(6, 4)
    seq_order = [(s, k) for s in chunks for k in range(4)]            # one stream after another
    mix_order = [(s, k) for k in range(4) for s in chunks]            # interleaved
    img_a, img_m = {}, {}
    alone, st_a = _serve(chunks, seq_order, img_a, lanes=1, max_batch=1)
    mixed, st_m = _serve(chunks, mix_order, img_m, lanes=3, max_batch=8)
    assert st_a["largest_batch"] == 1 and st_a["completed"] == 24
    assert st_m["completed"] == 24 and st_m["largest_batch"] > 1
    import torch
    for s, cs in chunks.items():
        for k, (x, T, f0) in enumerate(_assemble(cs)):
            da, ba = alone[(s, k)]
            dm, bm = mixed[(s, k)]
            assert da["status"] == dm["status"] == 0
            assert da["tag"] == dm["tag"] == 1000 * s + k
            assert da["frames"] == dm["frames"] == T and da["first_frame"] == dm["first_frame"] == f0
            np.testing.assert_array_equal(img_a[(s, k)], img_m[(s, k)], err_msg=f"stream {s} chunk {k}")
            np.testing.assert_array_equal(ba, bm, err_msg=f"stream {s} chunk {k}")
            _oracle_check(x, bm, img_m[(s, k)], f"stream {s} chunk {k} vs the oracle")
            want = det.detect(torch.from_numpy(x).cuda(), N, HOP)
            np.testing.assert_array_equal(ba, want, err_msg=f"stream {s} chunk {k} vs rise_detect")


def test_export_import_continues_the_stream(det):
    import torch
    from paper_2603_20481_gb300 import rise
    cs = _chunks(1, 3)[0]
    full, _ = _serve({0: cs}, [(0, 0), (0, 1), (0, 2)], lanes=2, max_batch=4)
    pinned = [torch.from_numpy(c).pin_memory() for c in cs]
    with rise.Server(N, HOP, max_chunk=len(cs[0]), max_streams=2) as a:
        a.submit(0, pinned[0])
        a.submit(0, pinned[1])
        a.drain()
        a.poll(timeout_ms=100)
        state = a.export_stream(0)
    with rise.Server(N, HOP, max_chunk=len(cs[0]), max_streams=4) as b:
        b.import_stream(3, state)
        assert b.submit(3, pinned[2])
        b.drain()
        (d, boxes), = b.poll(timeout_ms=1000)
    fd, fb = full[(0, 2)]
    assert d["seq"] == 2 and d["first_frame"] == fd["first_frame"] and d["frames"] == fd["frames"]
    np.testing.assert_array_equal(boxes, fb)
    with pytest.raises(rise.RiseError):
        with rise.Server(4096, 2048, max_chunk=len(cs[0]), max_streams=1) as c:
            c.import_stream(0, state)                 # another FFT size


def test_short_chunks_carry_everything(det):
    import torch
    rng = np.random.default_rng(3)
    long = synth.served_chunk(7, 0, n=40960).iq
    parts = [long[:500], long[500:1300], long[1300:1400], long[1400:]]   # the first three hold no frame
    imgs = {}
    res, _ = _serve({0: parts}, [(0, k) for k in range(4)], imgs, lanes=2, max_batch=2)
    plan = _assemble(parts)
    for k, (x, T, f0) in enumerate(plan):
        d, b = res[(0, k)]
        assert d["frames"] == T and d["first_frame"] == f0
        if T == 0:
            assert len(b) == 0 and (0, k) not in imgs
        else:
            _oracle_check(x, b, imgs[(0, k)], f"chunk {k} vs the oracle")
            np.testing.assert_array_equal(b, det.detect(torch.from_numpy(x).cuda(), N, HOP))
    assert plan[3][0].shape[0] == 40960                     # all earlier samples were carried
    del rng


def test_backpressure_and_bad_arguments():
    import torch
    from paper_2603_20481_gb300 import rise
    x = torch.from_numpy(synth.served_chunk(9, 0, n=8192).iq).pin_memory()
    with rise.Server(N, HOP, max_chunk=8192, max_streams=2, lanes=1, max_batch=1, max_pending=2) as srv:
        accepted = sum(srv.submit(i % 2, x) for i in range(300))
        srv.drain()
        got = 0
        while got < accepted:
            got += len(srv.poll(timeout_ms=100))
        st = srv.stats()
        assert st["submitted"] == accepted and st["completed"] == accepted
        assert st["rejected"] == 300 - accepted > 0
        with pytest.raises(rise.RiseError):
            srv.submit(2, x)                                  # no such stream
        big = torch.zeros(8193, dtype=torch.complex64).pin_memory()
        with pytest.raises(rise.RiseError):
            srv.submit(0, big)                                # longer than max_chunk
    with pytest.raises(rise.RiseError):
        rise.Server(1000, 500, max_chunk=8192, max_streams=1)   # FFT size not a power of two


def _serve_windows(chunks, order, W, images=None, **kw):
    import torch
    from paper_2603_20481_gb300 import rise
    pinned = {s: [torch.from_numpy(c).pin_memory() for c in cs] for s, cs in chunks.items()}
    res = {}
    with rise.Server(N, HOP, max_chunk=max(len(c) for cs in chunks.values() for c in cs),
                     max_streams=max(chunks) + 1, window_frames=W, keep_images=images is not None,
                     **kw) as srv:
        for s, k in order:
            assert srv.submit(s, pinned[s][k], tag=1000 * s + k)
        srv.drain()
        for d, b in srv.poll(timeout_ms=100):
            res[(d["stream"], d["seq"])] = (d, b)
        if images is not None:
            for key in res:
                images[key] = srv.result_image(*key)
    return res


def test_window_mode_plots_match_rise_detect(det):
    """Plots of W frames cut across chunks of uneven length: plot w is
    exactly rise_detect on samples [w W hop, w W hop + (W - 1) hop + N) of
    the stream, alone or served interleaved with other streams."""
    import torch
    W = 37
    rng = np.random.default_rng(11)
    chunks = {}
    for s in range(3):
        full = synth.served_chunk(20 + s, 0, n=180000).iq
        cuts = np.sort(rng.choice(np.arange(1, full.shape[0]), size=6, replace=False))
        chunks[s] = np.split(full, cuts)                       # 7 chunks, uneven
    span = (W - 1) * HOP + N
    for order, kw in (([(s, k) for s in chunks for k in range(7)], dict(lanes=1, max_batch=1)),
                      ([(s, k) for k in range(7) for s in chunks], dict(lanes=3, max_batch=8))):
        imgs = {}
        res = _serve_windows(chunks, order, W, imgs, **kw)
        for s, cs in chunks.items():
            full = np.concatenate(cs)
            n_plots = (full.shape[0] - span) // (W * HOP) + 1
            assert sum(1 for key in res if key[0] == s) == n_plots
            for w in range(n_plots):
                d, b = res[(s, w)]
                assert d["first_frame"] == w * W and d["frames"] == W
                x = full[w * W * HOP: w * W * HOP + span]
                assert imgs[(s, w)].shape == (W, N)
                _oracle_check(x, b, imgs[(s, w)], f"stream {s} plot {w} vs the oracle")
                np.testing.assert_array_equal(b, det.detect(torch.from_numpy(x).cuda(), N, HOP),
                                              err_msg=f"stream {s} plot {w}")


@pytest.mark.parametrize("W", [0, 40])
def test_lanes_do_not_grow_while_serving(W):
    """A lane's buffers are sized for its largest batch when the server is
    made: a burst that fills whole batches (the most chunks, each after the
    longest carry) after a batch of one allocates nothing more, so the
    lane's buffer generation stays where the first batch left it."""
    import torch
    from paper_2603_20481_gb300 import rise
    n = 2 * 40 * HOP + 512 if W else 61440 + 512          # window mode: up to 2 plots a chunk
    pinned = [torch.from_numpy(synth.served_chunk(40 + s, 0, n=n).iq).pin_memory() for s in range(8)]
    with rise.Server(N, HOP, max_chunk=n, max_streams=8, lanes=1, max_batch=8,
                     window_frames=W, max_pending=4096) as srv:
        assert srv.submit(0, pinned[0])
        srv.drain()
        first = srv.stats()
        assert first["batches"] == 1
        for k in range(12):
            for s in range(8):
                assert srv.submit(s, pinned[s])
        srv.drain()
        got = 0
        while True:
            res = srv.poll(timeout_ms=0)
            if not res:
                break
            got += len(res)
            assert all(d["status"] == 0 for d, _ in res)
        st = srv.stats()
    assert st["completed"] == 97 and st["largest_batch"] == 8
    assert st["buffer_generations"] == first["buffer_generations"]
