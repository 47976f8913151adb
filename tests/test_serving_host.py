"""Host logic of the serving loop and the profiling summariser, on the CPU."""
import math

from paper_2305_18396_gb300 import serving as SV
from paper_2305_18396_gb300.profiling import summarize_launches


def reqs(*ests):
    return [SV.Request(rid=i, model="x", m=1, arrival=float(i), mask_seed=i, est=e) for i, e in enumerate(ests)]


def test_take_batch_work_cap_keeps_arrival_order_and_skips_what_does_not_fit():
    admitted = reqs(1e-3, 0.2e-3, 5e-3, 0.1e-3, 0.3e-3)
    batch, rest = SV.take_batch(admitted, max_batch=8, work_factor=0.25, floor_s=1e-3)
    # cap = max(1 ms, 1.25 ms) = 1.25 ms: 1.0 + 0.2 fits, 5.0 does not, 0.1 would overflow 1.3
    assert [r.rid for r in batch] == [0, 1]
    assert [r.rid for r in rest] == [2, 3, 4]
    # the floor admits several small requests behind a small first one
    batch, rest = SV.take_batch(reqs(0.1e-3, 0.2e-3, 0.3e-3, 0.5e-3), 8, 0.25, 1e-3)
    assert [r.rid for r in batch] == [0, 1, 2] and [r.rid for r in rest] == [3]
    # a long first request takes no company beyond 25% of its own estimate
    batch, rest = SV.take_batch(reqs(8e-3, 1e-3, 1.5e-3, 0.4e-3), 8, 0.25, 1e-3)
    assert [r.rid for r in batch] == [0, 1, 3] and [r.rid for r in rest] == [2]


def test_take_batch_limits_and_no_cap():
    batch, rest = SV.take_batch(reqs(*[1e-4] * 10), max_batch=4, work_factor=None, floor_s=0.0)
    assert len(batch) == 4 and len(rest) == 6
    batch, rest = SV.take_batch(reqs(1.0, 5.0, 9.0), max_batch=8, work_factor=None, floor_s=0.0)
    assert len(batch) == 3 and not rest


def test_launch_allowed_overlap_gate():
    assert SV.launch_allowed([], now=0.0, slots=2, overlap_s=2e-3)
    # one long launch just started: 5 ms left > 2 ms window
    assert not SV.launch_allowed([(0.0, 5e-3)], now=0.0, slots=2, overlap_s=2e-3)
    # the same launch near its end: 1 ms left
    assert SV.launch_allowed([(0.0, 5e-3)], now=4e-3, slots=2, overlap_s=2e-3)
    # estimates that have run out count as zero, but the slots still bound concurrency
    assert SV.launch_allowed([(0.0, 1e-3)], now=5e-3, slots=2, overlap_s=0.0)
    assert not SV.launch_allowed([(0.0, 1e-3), (0.0, 1e-3)], now=5e-3, slots=2, overlap_s=math.inf)


def test_summarize_launches_window_and_units(tmp_path):
    rows = [
        ('"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"'),
        ('"0","k_setup(int)","gpu__time_duration.sum","usecond","5"'),
        ('"1","void k_fwd_multi_t<12>(T)","gpu__time_duration.sum","usecond","10"'),
        ('"2","void (anonymous namespace)::k_mac(int)","gpu__time_duration.sum","msecond","2"'),
        ('"3","at::fill(float)","gpu__time_duration.sum","nsecond","500"'),
        ('"4","void k_fwd_multi_t<12>(T)","gpu__time_duration.sum","usecond","30"'),
        ('"5","k_tail(int)","gpu__time_duration.sum","usecond","7"'),
    ]
    f = tmp_path / "launches.csv"
    f.write_text("\n".join(rows) + "\n")
    agg = summarize_launches(str(f), skip_prefixes=("at::",), first="k_fwd_multi", last="k_fwd_multi")
    assert agg == {"k_fwd_multi_t<12>": [2, 40.0], "k_mac": [1, 2000.0]}
    agg = summarize_launches(str(f), skip_first=5)
    assert agg == {"k_tail": [1, 7.0]}
    agg = summarize_launches(str(f), back=1, first="k_mac")
    assert set(agg) == {"k_fwd_multi_t<12>", "k_mac", "at::fill", "k_tail"}


def test_take_batch_fifo_stops_at_first_misfit():
    admitted = reqs(1e-3, 0.2e-3, 5e-3, 0.1e-3, 0.3e-3)
    batch, rest = SV.take_batch(admitted, max_batch=8, work_factor=0.25, floor_s=1e-3, fifo=True)
    assert [r.rid for r in batch] == [0, 1]
    assert [r.rid for r in rest] == [2, 3, 4]
    batch, rest = SV.take_batch(reqs(0.1e-3, 2e-3, 0.1e-3), 8, 0.25, 1e-3, fifo=True)
    assert [r.rid for r in batch] == [0] and [r.rid for r in rest] == [1, 2]
    batch, rest = SV.take_batch(reqs(0.1e-3, 2e-3, 0.1e-3), 8, 0.25, 1e-3, fifo=False)
    assert [r.rid for r in batch] == [0, 2] and [r.rid for r in rest] == [1]


def test_withdraw_from_queue_or_admitted():
    queue, admitted = reqs(1e-3, 2e-3), reqs(3e-3, 4e-3, 5e-3)
    for r in admitted:
        r.rid += 10
    q, a, r, where = SV.withdraw(queue, admitted, 11)
    assert where == "admitted" and r.rid == 11 and [x.rid for x in a] == [10, 12] and q == queue
    q, a, r, where = SV.withdraw(queue, admitted, 1)
    assert where == "queued" and r.rid == 1 and [x.rid for x in q] == [0] and a == admitted
    assert SV.withdraw(queue, admitted, 99) == (queue, admitted, None, None)


class _Event:
    def __init__(self, done):
        self.done = done

    def query(self):
        return self.done


def _server_state():
    """A Server's host state without a device: two queued, two admitted, one launch in flight."""
    srv = object.__new__(SV.Server)
    srv.queue, srv.admitted = reqs(1e-3, 1e-3), reqs(1e-3, 1e-3)
    for i, r in enumerate(srv.admitted):
        r.rid, r.footprint = 10 + i, 100
    running = reqs(1e-3, 1e-3)
    for i, r in enumerate(running):
        r.rid, r.footprint, r.out = 20 + i, 100, object()
    srv.inflight = [SV._InFlight(0.0, 1e-3, 0, _Event(False), running, None, None)]
    srv.done, srv.cancelled, srv.failed, srv.in_use, srv.keep, srv.ctx = [], [], [], 400, True, None
    return srv


def test_cancel_queued_admitted_and_launched_requests(monkeypatch):
    monkeypatch.setattr(SV.B, "he_device_status", lambda ctx, stream=None: None)  # no device error
    srv = _server_state()
    assert srv.cancel(1) == "queued" and [r.rid for r in srv.queue] == [0] and srv.in_use == 400
    assert srv.cancel(11) == "admitted" and [r.rid for r in srv.admitted] == [10] and srv.in_use == 300
    assert srv.cancel(21) == "in_flight" and srv.cancel(21) is None  # already withdrawn
    assert srv.cancel(99) is None
    assert [r.rid for r in srv.cancelled] == [1, 11]
    srv._poll(1.0)  # launch still running: nothing completes
    assert srv.inflight and not srv.done
    srv.inflight[0].event.done = True
    srv._poll(2.0)  # the launch completes: the cancelled request's output is dropped
    assert not srv.inflight and srv.in_use == 100
    assert [r.rid for r in srv.done] == [20] and srv.done[0].out is not None
    assert [r.rid for r in srv.cancelled] == [1, 11, 21] and srv.cancelled[-1].out is None



def _launch(start, rids, done):
    reqs_ = [SV.Request(rid=i, model="x", m=1, arrival=0.0, mask_seed=i, footprint=10) for i in rids]
    return SV._InFlight(start, 1e-3, 0, _Event(done), reqs_, None, None)


def _bare_server(inflight):
    srv = object.__new__(SV.Server)  # only the completion logic: no device, no streams
    srv.ctx, srv.keep = None, True
    srv.inflight, srv.done, srv.cancelled, srv.failed = inflight, [], [], []
    srv.in_use = sum(r.footprint for f in inflight for r in f.reqs)
    return srv


def test_poll_reports_requests_of_a_launch_with_a_device_error_as_failed(monkeypatch):
    """The bounded wait of a kernel expired (the context's flag is set): the finished launch and
    the one still in flight (either may have set the flag) report failed requests, none done."""
    calls = []

    def status(ctx, stream=None):
        calls.append(stream)
        if len(calls) == 1:
            raise SV.B.HEError(SV.B.HE_ETIMEOUT, "bounded wait expired")

    monkeypatch.setattr(SV.B, "he_device_status", status)
    a, b = _launch(0.0, [0, 1], True), _launch(0.1, [2], False)
    srv = _bare_server([a, b])
    srv._poll(1.0)
    assert [r.rid for r in srv.failed] == [0, 1] and not srv.done and srv.inflight == [b]
    assert all(r.out is None and r.failed for r in a.reqs) and b.failed
    b.event.done = True
    srv._poll(2.0)  # the flag is clear now, but b was in flight when it was set
    assert [r.rid for r in srv.failed] == [0, 1, 2] and not srv.done and srv.in_use == 0
    c = _launch(2.5, [3], True)
    srv.inflight = [c]
    srv.in_use += 10
    srv._poll(3.0)
    assert [r.rid for r in srv.done] == [3] and not c.failed


def test_mark_failed_without_error_marks_nothing():
    a, b = _launch(0.0, [0], True), _launch(0.0, [1], False)
    SV.mark_failed([a], [b], False)
    assert not a.failed and not b.failed
    SV.mark_failed([a], [b], True)
    assert a.failed and b.failed


def test_take_batch_merges_requests_of_the_oldest_matrix_past_the_cap():
    admitted = reqs(1e-3, 5e-3, 4e-3, 0.1e-3)
    admitted[1].model = admitted[2].model = "y"
    admitted[0].model = admitted[3].model = "x"
    batch, rest = SV.take_batch(admitted, 8, 0.25, 1e-3, merge_same_model=True)
    assert [r.rid for r in batch] == [0, 3] and [r.rid for r in rest] == [1, 2]
    big = reqs(1e-3, 9e-3, 9e-3, 9e-3)
    batch, rest = SV.take_batch(big, 3, 0.25, 1e-3, merge_same_model=True)  # same matrix: past the cap, up to max_batch
    assert [r.rid for r in batch] == [0, 1, 2] and [r.rid for r in rest] == [3]
    batch, rest = SV.take_batch(big, 3, 0.25, 1e-3)  # without merging the cap holds
    assert [r.rid for r in batch] == [0] and len(rest) == 3
