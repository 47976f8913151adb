"""Continuous-batching server for private-inference matrix-product requests.

A request is one Pi_MatMul (Algorithm 1, Sec. 3.1.1) of a client's encrypted share
X (m x k) against one of the server's resident weight matrices W (k x n) -- e.g.
the QKV, attention-output or FFN product of a BERT-base or BERT-large layer at the
client's sequence length m.  The server keeps every weight matrix resident in NTT
form; requests arrive over time and are

* admitted in arrival order while the device-memory footprint of the admitted but
  unfinished requests (their output ciphertexts plus the workspace of their launch)
  stays within a budget;
* launched as soon as a launch slot is free: the oldest admitted request, and after it
  the admitted requests that fit a work cap (their estimated device time, summed, at
  most `batch_work_factor` above the oldest's, or `batch_floor_ms`), go into one
  multi-product launch (he_matmul_multi, up to 64 products of any shapes), so requests
  that arrive while others are on the GPU join the next launch and their work overlaps
  on the device with the running one.  The cap keeps a long request from being delayed
  by the requests that arrived after it.  Requests of the oldest's weight matrix join
  regardless of the cap: the launch merges them into one product whose weight stream
  serves all their rows;
* started only while the work still in flight is estimated to end within an overlap
  window (2 ms): short launches overlap the next one, a long launch runs without a
  second one taking SMs at its kernel boundaries (requests arriving meanwhile are
  batched into the launch that follows it);
* run on a stream whose CUDA priority is below that of every launch still in flight
  (the highest when the device is idle): the oldest launch keeps the SMs it can fill,
  later launches take the SMs it leaves idle (its tail, its small grids); each launch
  stream keeps its workspace between launches;
* completed when their launch's event fires (latency = completion - arrival), after
  the context's error flag is read: a kernel whose bounded wait for its data expired
  leaves invalid outputs, and the flag (one per context) cannot tell which launch set
  it, so every launch that may have set it -- the ones that completed and the ones
  still in flight -- is marked failed and its requests are reported as failed, not
  done;
* withdrawn by `Server.cancel` (a client that went away): a queued or admitted request
  leaves at once and frees its share of the budget; one already launched cannot be
  taken back from the GPU, so its output is dropped when its launch completes.

`run_per_request` is the plain path it is compared against: one he_matmul per request,
in arrival order, on one stream.

The timing loop runs on the host clock; all arithmetic runs in the library's kernels.
"""
import heapq
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import binding as B


@dataclass
class Model:
    """One resident weight matrix: encoded weights and its fixed blocking (wire format)."""
    name: str
    k: int
    n: int
    blk: tuple
    pt: torch.Tensor
    ct_pool: torch.Tensor  # input ciphertexts for the largest m (requests use a prefix)
    max_m: int


@dataclass
class Request:
    rid: int
    model: str
    m: int
    arrival: float  # seconds since start
    mask_seed: int
    out: torch.Tensor = None
    launched: float = math.nan
    done: float = math.nan
    footprint: int = 0
    est: float = 0.0  # estimated device seconds inside a multi-product launch
    cancelled: bool = False
    failed: bool = False  # its launch hit a device error: no valid output


# Device-time estimate of one product inside a multi-product launch: a fixed part per
# product plus its plaintext MACs at the rate large BERT-shaped products reach alone at
# the ring dimension (N = 8192 carries three primes and twice the slots per ciphertext).
EST_FIXED_S = 100e-6
EST_MACS_PER_S = {4096: 4.0e11, 8192: 2.0e11}


def est_rate(N):
    return EST_MACS_PER_S.get(N, 4.0e11 * 4096 / max(N, 1))


@dataclass(order=True)
class _InFlight:
    start: float
    est: float = field(compare=False)  # estimated device seconds of the launch
    level: int = field(compare=False)
    event: object = field(compare=False)
    reqs: list = field(compare=False)
    ws: torch.Tensor = field(compare=False)
    stream: object = field(compare=False)
    failed: bool = field(default=False, compare=False)


def mark_failed(finished, inflight, device_error):
    """After reading the context's error flag at the completion of `finished` launches:
    with an error, every launch that may have set it -- those finished and those still
    `inflight` -- is marked failed (the flag is one per context)."""
    if device_error:
        for f in list(finished) + list(inflight):
            f.failed = True


def device_error(ctx, stream):
    """True if a kernel of the context gave up a bounded wait since the last check
    (he_device_status reads and clears the flag; `stream` has completed its work)."""
    try:
        B.he_device_status(ctx, stream)
    except B.HEError as e:
        if e.code == B.HE_ETIMEOUT:
            return True
        raise
    return False


def request_footprint(ctx, model, m, flags):
    """Device bytes a request holds while admitted: outputs + its share of a launch workspace."""
    si = ctx.sizes(m, model.k, model.n, model.blk)
    out = si["out_words_compact"] if flags else si["out_words"]
    ws = si["workspace_bytes_compact"] if flags else si["workspace_bytes"]
    return 8 * out + ws + 512


def priority_levels(n=4):
    """Up to `n` CUDA stream priorities, highest first (lower number = higher priority)."""
    least, greatest = torch.cuda.Stream.priority_range()
    return [p for p in range(greatest, least + 1)][:n] or [0]


def take_batch(admitted, max_batch, work_factor, floor_s, fifo=False, merge_same_model=False):
    """Batch formation: the oldest admitted request plus, in arrival order, the requests
    whose estimated device time keeps the batch within max(floor_s, (1 + work_factor) x
    the oldest's estimate) (no cap with work_factor None), at most max_batch in all.  With
    merge_same_model, requests of the oldest's weight matrix join regardless of the cap:
    the multi-product launch merges them into one product whose weight stream serves all
    their rows, so they add little to the launch.  With fifo the batch ends at the first
    request that does not fit (none is overtaken), else later requests that fit are still
    taken.  Returns (batch, the requests left admitted)."""
    first = admitted[0]
    cap = max(floor_s, first.est * (1.0 + work_factor)) if work_factor is not None else math.inf
    batch, rest, total = [first], [], first.est
    for i, r in enumerate(admitted[1:], 1):
        same = merge_same_model and r.model == first.model
        if len(batch) < max_batch and (same or total + r.est <= cap):
            batch.append(r)
            total += 0.0 if same else r.est
        elif fifo:
            rest = list(admitted[i:])
            break
        else:
            rest.append(r)
    return batch, rest


def launch_allowed(inflight, now, slots, overlap_s):
    """inflight: (start, estimated seconds) of the launches running.  A new launch may start
    when a slot is free and the work in flight is estimated to end within overlap_s: a long
    launch is not slowed by a second one taking SMs at its kernel boundaries, while short
    launches overlap the next."""
    if len(inflight) >= slots:
        return False
    remaining = sum(max(0.0, est - (now - start)) for start, est in inflight)
    return not inflight or remaining <= overlap_s


def withdraw(queue, admitted, rid):
    """Takes request `rid` out of the waiting lists.  Returns (queue, admitted, request,
    where) with where "queued" or "admitted", or (queue, admitted, None, None) when it
    is in neither (launched, finished or unknown)."""
    for where, lst in (("queued", queue), ("admitted", admitted)):
        for i, r in enumerate(lst):
            if r.rid == rid:
                rest = lst[:i] + lst[i + 1:]
                return (rest, admitted, r, where) if where == "queued" else (queue, rest, r, where)
    return queue, admitted, None, None


class Server:
    def __init__(self, ctx, models, flags=B.HE_DROP_C0, hbm_budget=32 << 30, slots=2, max_batch=8,
                 batch_work_factor=0.25, batch_floor_ms=1.0, priorities=True, keep_outputs=True,
                 overlap_ms=2.0, fifo=False, merge_same_model=True):
        self.ctx, self.models, self.flags = ctx, {mm.name: mm for mm in models}, flags
        self.budget, self.max_batch = hbm_budget, min(max_batch, 64)
        self.slots = slots
        self.work_factor, self.floor_s = batch_work_factor, batch_floor_ms * 1e-3
        self.overlap_s = overlap_ms * 1e-3
        self.fifo = fifo
        self.merge = merge_same_model and bool(flags & B.HE_DROP_C0)  # the launch merges compact products only
        self.keep = keep_outputs
        levels = priority_levels() if priorities else [0]
        # a fixed set of streams, `slots` per priority level; buffers are allocated on the
        # stream that builds the server and handed to a launch stream with record_stream, so
        # the caching allocator keeps one pool instead of one per launch stream
        self.streams = [[torch.cuda.Stream(device=ctx.device, priority=p) for _ in range(slots)] for p in levels]
        self.alloc_stream = torch.cuda.current_stream(ctx.device)
        self.queue, self.admitted, self.inflight, self.done, self.cancelled = [], [], [], [], []
        self.failed = []
        self.in_use = 0
        self.launches = 0
        self._sizes = {}  # (matrix, m) -> he_sizes
        self._ws = {}     # launch stream -> workspace, grown as needed (a stream runs one launch at a time)

    def _size(self, mm, m):
        key = (mm.name, m)
        if key not in self._sizes:
            self._sizes[key] = self.ctx.sizes(m, mm.k, mm.n, mm.blk)
        return self._sizes[key]

    def submit(self, req):
        mm = self.models[req.model]
        req.footprint = request_footprint(self.ctx, mm, req.m, self.flags)
        req.est = EST_FIXED_S + req.m * mm.k * mm.n / est_rate(self.ctx.N)
        if req.footprint > self.budget:
            raise ValueError(f"request {req.rid} needs {req.footprint} bytes, more than the whole budget")
        self.queue.append(req)

    def cancel(self, rid):
        """Withdraws request `rid`: "queued" / "admitted" (gone at once; an admitted one
        frees its budget), "in_flight" (launched: its output is dropped when the launch
        completes), or None (finished or unknown)."""
        self.queue, self.admitted, r, where = withdraw(self.queue, self.admitted, rid)
        if r is not None:
            r.cancelled = True
            if where == "admitted":
                self.in_use -= r.footprint
            self.cancelled.append(r)
            return where
        for f in self.inflight:
            for r in f.reqs:
                if r.rid == rid and not r.cancelled:
                    r.cancelled = True
                    return "in_flight"
        return None

    def _admit(self):
        while self.queue and self.in_use + self.queue[0].footprint <= self.budget:
            r = self.queue.pop(0)
            self.in_use += r.footprint
            self.admitted.append(r)

    def _take_batch(self):
        batch, self.admitted = take_batch(self.admitted, self.max_batch, self.work_factor, self.floor_s, self.fifo,
                                          self.merge)
        return batch

    def _may_launch(self, now):
        return bool(self.admitted) and launch_allowed([(f.start, f.est) for f in self.inflight], now, self.slots,
                                                      self.overlap_s)

    def _launch(self, now):
        if not self._may_launch(now):
            return
        batch = self._take_batch()
        # below every launch in flight, so the oldest work keeps priority on the SMs
        level = min(max((f.level for f in self.inflight), default=-1) + 1, len(self.streams) - 1)
        busy = {id(f.stream) for f in self.inflight}
        stream = next(st for st in self.streams[level] if id(st) not in busy)
        items = []
        for r in batch:
            mm = self.models[r.model]
            si = self._size(mm, r.m)
            ow = si["out_words_compact"] if self.flags else si["out_words"]
            r.out = self.ctx.empty(ow)
            r.out.record_stream(stream)
            items.append(dict(ct_in=mm.ct_pool, pt=mm.pt, ct_out=r.out, m=r.m, k=mm.k, n=mm.n, blk=mm.blk,
                              flags=self.flags, mask_seed=r.mask_seed))
            r.launched = now
        if len(batch) == 1:  # one product: its own launch, no descriptor table to build
            r, mm = batch[0], self.models[batch[0].model]
            si = self._size(mm, r.m)
            need = (si["workspace_bytes_compact"] if self.flags else si["workspace_bytes"]) // 8 + 1
        else:
            prods = B.make_products(items)
            need = B.he_multi_workspace_bytes(self.ctx, prods) // 8 + 1
        ws = self._ws.get(id(stream))
        if ws is None or ws.numel() < need:  # the stream's previous launch has completed
            ws = self._ws[id(stream)] = self.ctx.empty(need)
            ws.record_stream(stream)
        stream.wait_stream(self.alloc_stream)  # the buffers' previous users are done
        if len(batch) == 1:
            B.he_matmul(self.ctx, mm.ct_pool, mm.pt, r.m, mm.k, mm.n, mm.blk, r.mask_seed, ct_out=r.out, workspace=ws,
                        flags=self.flags, stream=stream)
        else:
            B.he_matmul_multi(self.ctx, prods, ws, stream=stream)
        ev = torch.cuda.Event()
        ev.record(stream)
        heapq.heappush(self.inflight, _InFlight(now, sum(r.est for r in batch), level, ev, batch, ws, stream))
        self.launches += 1

    def _poll(self, now):
        finished, still = [], []
        for f in self.inflight:
            (finished if f.event.query() else still).append(f)
        self.inflight = still
        if not finished:
            return
        mark_failed(finished, still, device_error(self.ctx, finished[0].stream))
        for f in finished:
            for r in f.reqs:
                r.done = now
                self.in_use -= r.footprint
                if f.failed:
                    r.failed = True
                if not self.keep or r.cancelled or r.failed:
                    r.out = None
                (self.cancelled if r.cancelled else self.failed if r.failed else self.done).append(r)

    def pump(self, now):
        self._poll(now)
        self._admit()
        while self._may_launch(now):
            self._launch(now)

    def idle(self):
        return not (self.queue or self.admitted or self.inflight)


def make_models(ctx, specs, seed=2):
    """specs: (name, k, n, max_m).  Encodes random fixed-point weights and one pool of input
    ciphertexts per matrix (the client's encrypted shares for the largest m)."""
    from . import synthetic as S

    models = []
    sk = B.he_keygen(ctx, 77)
    for i, (name, k, n, max_m) in enumerate(specs):
        blk = ctx.default_blocking(128, k, n)
        W = torch.from_numpy(S.fixed_point_weights((k, n), seed + i).view(np.int64).reshape(-1)).to(ctx.device)
        pt = B.he_encode_weights(ctx, W, k, n, blk)
        X = torch.from_numpy(S.uniform_share((max_m, k), 1000 + i).view(np.int64).reshape(-1)).to(ctx.device)
        ct = B.he_encrypt(ctx, sk, B.he_pack_input(ctx, X, max_m, k, blk), 2000 + i)
        models.append(Model(name, k, n, blk, pt, ct, max_m))
    torch.cuda.synchronize()
    return models


def make_requests(models, count, rate, seed=6, m_lo=8, m_hi=512):
    """Poisson arrivals at `rate` req/s, m log-uniform in [m_lo, m_hi], matrices uniform."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    ms = np.exp(rng.uniform(math.log(m_lo), math.log(m_hi), size=count)).astype(int)
    which = rng.integers(0, len(models), size=count)
    return [Request(i, models[which[i]].name, int(min(ms[i], models[which[i]].max_m)), float(t[i]), 10_000 + i)
            for i in range(count)]


def _stats(reqs, models, wall):
    if not reqs:
        return {"requests": 0, "throughput_req_s": 0.0, "plain_macs_per_s": 0.0, "p50_ms": math.nan,
                "p99_ms": math.nan, "mean_ms": math.nan}
    lat = np.array([(r.done - r.arrival) * 1e3 for r in reqs])
    macs = sum(r.m * models[r.model].k * models[r.model].n for r in reqs)
    return {"requests": len(reqs), "throughput_req_s": len(reqs) / wall, "plain_macs_per_s": macs / wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean())}


def run_served(ctx, models, requests, **kw):
    """Real-time continuous batching over the arrival schedule; returns latency/throughput stats."""
    srv = Server(ctx, models, **kw)
    pending = sorted(requests, key=lambda r: r.arrival)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    i = 0
    while i < len(pending) or not srv.idle():
        now = time.perf_counter() - t0
        while i < len(pending) and pending[i].arrival <= now:
            srv.submit(pending[i])
            i += 1
        srv.pump(now)
        if srv.idle() and i < len(pending):
            time.sleep(max(0.0, min(pending[i].arrival - now, 0.0005)))
    wall = time.perf_counter() - t0
    st = _stats(srv.done, {mm.name: mm for mm in models}, wall)
    st["launches"] = srv.launches
    st["failed"] = len(srv.failed)
    return st, srv.done


def run_per_request(ctx, models, requests, flags=B.HE_DROP_C0, keep_outputs=True):
    """The plain path: one he_matmul per request in arrival order on one stream."""
    by = {mm.name: mm for mm in models}
    pending = sorted(requests, key=lambda r: r.arrival)
    stream = torch.cuda.Stream(device=ctx.device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in pending:
        now = time.perf_counter() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        mm = by[r.model]
        with torch.cuda.stream(stream):
            r.out = B.he_matmul(ctx, mm.ct_pool, mm.pt, r.m, mm.k, mm.n, mm.blk, r.mask_seed, flags=flags,
                                stream=stream)
        stream.synchronize()
        r.done = time.perf_counter() - t0
        r.failed = device_error(ctx, stream)
        if not keep_outputs or r.failed:
            r.out = None
    wall = time.perf_counter() - t0
    ok = [r for r in pending if not r.failed]
    st = _stats(ok, by, wall)
    st["launches"] = len(pending)
    st["failed"] = len(pending) - len(ok)
    return st, ok
