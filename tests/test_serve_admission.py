"""Host logic of the query server (no GPU): admission oldest request first, batches of one
(resolution, subcarrier count) up to max_batch within the memory budget, moving-receiver
requests alone, the order of the requests left waiting, a head that does not fit blocking
admission until memory frees up; rejection of a request larger than the budget; cancellation of
a waiting request; latency statistics without rejected or cancelled requests."""
import collections

import pytest

from paper_2511_22793_gb300.serve import Request, admit


def _bytes(H, W, K):
    return H * W * K          # a stand-in size: what matters is the arithmetic of the budget


def _q(rid, res=(90, 360), K=1, rx=None):
    return Request(rid=rid, tx=(0.0, 0.0, 0.0), res=res, K=K, rx=rx)


def _ids(qs):
    return [q.rid for q in qs]


def test_batches_same_shape_oldest_first_and_keeps_the_rest_in_order():
    w = collections.deque([_q(0), _q(1, K=64), _q(2), _q(3, res=(45, 180)), _q(4), _q(5)])
    group, left = admit(w, used=0, budget=10 ** 9, max_batch=3, request_bytes=_bytes)
    assert _ids(group) == [0, 2, 4]
    assert _ids(left) == [1, 3, 5]
    assert _ids(w) == [0, 1, 2, 3, 4, 5]          # the caller's queue is not consumed


def test_budget_limits_the_batch_and_blocks_a_head_that_does_not_fit():
    one = _bytes(90, 360, 1)
    w = collections.deque([_q(i) for i in range(5)])
    group, left = admit(w, used=one, budget=3 * one, max_batch=8, request_bytes=_bytes)
    assert _ids(group) == [0, 1] and _ids(left) == [2, 3, 4]
    assert admit(w, used=3 * one - 1, budget=3 * one, max_batch=8, request_bytes=_bytes) is None


def test_moving_receiver_runs_alone_and_is_not_joined():
    w = collections.deque([_q(0, rx=(1.0, 0.0, 0.0)), _q(1), _q(2)])
    group, left = admit(w, used=0, budget=10 ** 9, max_batch=8, request_bytes=_bytes)
    assert _ids(group) == [0] and _ids(left) == [1, 2]
    w = collections.deque([_q(0), _q(1, rx=(1.0, 0.0, 0.0)), _q(2)])
    group, left = admit(w, used=0, budget=10 ** 9, max_batch=8, request_bytes=_bytes)
    assert _ids(group) == [0, 2] and _ids(left) == [1]


def test_draining_a_queue_serves_every_request_once():
    import numpy as np

    rng = np.random.default_rng(0)
    shapes = [((45, 180), 1), ((90, 360), 64), ((180, 720), 256)]
    w = collections.deque()
    for i in range(200):
        res, K = shapes[rng.integers(0, 3)]
        w.append(_q(i, res=res, K=K, rx=(1.0, 2.0, 0.5) if rng.uniform() < 0.1 else None))
    seen = []
    while w:
        group, w = admit(w, used=0, budget=10 ** 12, max_batch=8, request_bytes=_bytes)
        assert 1 <= len(group) <= 8
        assert len({(q.res, q.K) for q in group}) == 1
        assert all(q.rx is None for q in group) or len(group) == 1
        seen += _ids(group)
    assert sorted(seen) == list(range(200))


def _server_state(budget=10 ** 9):
    """The host state Server.submit and Server.cancel work on, without a device."""
    import types

    from paper_2511_22793_gb300.serve import Server

    st = types.SimpleNamespace(budget=budget, waiting=collections.deque(), done=[],
                               geom={(90, 360): None, (45, 180): None, (180, 720): None},
                               slot_geom={(0, 90, 360): None})
    st.request_bytes = lambda H, W, K: _bytes(H, W, K)
    return Server, st


def test_submit_rejects_a_request_larger_than_the_budget():
    Server, st = _server_state(budget=90 * 360 * 64 - 1)
    big, small = _q(0, K=64), _q(1, K=1)
    Server.submit(st, big)
    Server.submit(st, small)
    assert big.rejected and big.t_done > 0 and st.done == [big]
    assert not small.rejected and list(st.waiting) == [small]
    # a resolution the server has no geometry for is rejected too
    odd = _q(2, res=(30, 120))
    Server.submit(st, odd)
    assert odd.rejected and st.done == [big, odd]


def test_cancel_withdraws_only_waiting_requests():
    Server, st = _server_state()
    qs = [_q(i) for i in range(4)]
    for q in qs:
        Server.submit(st, q)
    assert Server.cancel(st, 2) is True
    assert qs[2].cancelled and st.done == [qs[2]] and _ids(st.waiting) == [0, 1, 3]
    assert Server.cancel(st, 2) is False           # no longer waiting
    assert Server.cancel(st, 99) is False          # unknown (or already on the GPU)
    group, left = admit(st.waiting, used=0, budget=10 ** 9, max_batch=8, request_bytes=_bytes)
    assert _ids(group) == [0, 1, 3] and not left


def test_latency_stats_leave_out_rejected_and_cancelled_requests():
    from paper_2511_22793_gb300.serve import latency_stats

    qs = [_q(i) for i in range(4)]
    for i, q in enumerate(qs):
        q.t_arrival, q.t_done = 0.0, 0.001 * (i + 1)
    qs[1].rejected = True
    qs[2].cancelled = True
    st = latency_stats(qs)
    assert st["served"] == 2 and st["rejected"] == 1 and st["cancelled"] == 1
    assert st["p50_ms"] == pytest.approx(2.5)


def test_arena_first_fit_alignment_and_merging():
    from paper_2511_22793_gb300.serve import Arena

    a = Arena(4096, align=256)
    x = a.alloc(100)
    y = a.alloc(300)
    z = a.alloc(256)
    assert (x, y, z) == (0, 256, 768) and a.used == 1024
    assert a.alloc(4096) is None and a.fits(3072) and not a.fits(3073)
    a.free(y)                      # a 512-byte hole between x and z
    assert a.alloc(600) == 1024    # does not fit the hole: first fit goes past it
    assert a.alloc(512) == 256     # fills the hole exactly
    a.free(x)
    a.free(256)
    a.free(z)                      # x, the hole's block and z merge into one free block at 0
    assert a.free_list[0] == (0, 1024)
    a.free(1024)
    assert a.free_list == [(0, 4096)] and a.used == 0 and not a.taken


def test_admission_shrinks_a_batch_to_a_contiguous_block():
    one = _bytes(90, 360, 1)
    w = collections.deque([_q(i) for i in range(6)])
    # budget for six, but the largest contiguous block holds only four
    group, left = admit(w, used=0, budget=10 * one, max_batch=8, request_bytes=_bytes,
                        fits=lambda n: n <= 4 * one)
    assert _ids(group) == [0, 1, 2, 3] and _ids(left) == [4, 5]
    assert admit(w, used=0, budget=10 * one, max_batch=8, request_bytes=_bytes, fits=lambda n: False) is None


def test_arena_random_traffic_never_overlaps():
    import numpy as np

    from paper_2511_22793_gb300.serve import Arena

    rng = np.random.default_rng(3)
    a = Arena(1 << 20, align=256)
    live = {}
    for _ in range(2000):
        if live and rng.uniform() < 0.45:
            off = list(live)[rng.integers(len(live))]
            a.free(off)
            del live[off]
        else:
            n = int(rng.integers(1, 50_000))
            off = a.alloc(n)
            if off is not None:
                assert off % 256 == 0 and off + n <= a.size
                for o, m in live.items():
                    assert off + n <= o or o + m <= off
                live[off] = n
    assert a.used == sum((m + 255) // 256 * 256 for m in live.values())
