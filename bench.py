"""Benchmark: homomorphic matrix products (Algorithm 1) of one transformer encoder layer.

One step = every linear product of one encoder layer (Sec. 3.1.1): the four fully
connected layers against resident NTT-form weights and, for each head, the two cross
terms of Q K^T and of P V against the server's shares (encoded per step).  The default
(headline) workload is one BERT-large layer at sequence length 512 with BFV N = 8192,
three ~50-bit primes, t = 2^37: 68 server-side Pi_MatMul calls, 7,516,192,768 plain
multiply-accumulates per step.  `--workload bert-base` runs one BERT-base layer at
sequence 128 with N = 4096 and two primes instead (52 calls, 956,301,312 MACs); the
default run also times that layer and reports it under "bert_base_layer".  Input
ciphertexts are encrypted (GPU test client) before timing and stay resident; every
call re-masks with a fresh seed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  value = plain MACs/s over all ranks (each rank
runs its own layer: independent requests, weak scaling).
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "HE-MatMul plaintext MACs/s"
UNIT = "MAC/s"
# selectable with --workload; the default is the headline configuration (the largest that
# fits one GPU)
WORKLOADS = {
    "bert-large-n8192": dict(N=8192, L=3, model="BERT_LARGE", host_depth=3,
                             desc="bert-large layer linear products, seq 512, N=8192, L=3 (QKV, attn-out, FFN1, FFN2 "
                                  "+ 16 heads x 2 cross terms x {QK^T, PV})"),
    "bert-base": dict(N=4096, L=2, model="BERT_BASE", host_depth=6,
                      desc="bert-base layer linear products, seq 128 (QKV, attn-out, FFN1, FFN2 + 12 heads x 2 cross "
                           "terms x {QK^T, PV})"),
}
DEFAULT_WORKLOAD = "bert-large-n8192"

# Blockings (m_b, k_b, n_b) of the products the CPU oracle legs sample, keyed by (N, m, k, n),
# written out so that the oracle legs load no part of the CUDA library (the blocking fixes
# the ciphertexts, not the plain MACs a product computes).
ORACLE_BLOCKINGS = {
    (4096, 128, 64, 128): (32, 8, 16), (4096, 128, 128, 64): (32, 16, 8), (4096, 64, 128, 128): (16, 16, 16),
    (8192, 512, 64, 512): (64, 4, 32), (8192, 512, 512, 64): (64, 32, 4), (8192, 64, 512, 512): (8, 32, 32),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the mixed-request leg (one multi-product launch vs one call per request)")
    ap.add_argument("--serving-rates", default="50,100,400,800,1600,3200",
                    help="Poisson arrival rates (requests/s); the highest saturate the per-request path")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="requests per rate (at most 10 s of arrivals per rate)")
    ap.add_argument("--launch", default="multi", choices=["multi", "groups"],
                    help="multi: the whole layer as one multi-product launch per step; groups: one batched "
                         "launch per product shape")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS),
                    help="bert-large-n8192: the headline, one BERT-large layer at seq 512 with N=8192, L=3; "
                         "bert-base: one BERT-base layer at seq 128 with N=4096, L=2")
    ap.add_argument("--no-bert-base", action="store_true",
                    help="skip the extra BERT-base layer (N=4096) timed beside the headline workload")
    ap.add_argument("--host-depth", type=int, default=None,
                    help="end-to-end leg: host-buffer steps in flight (streams with their own buffers); default 3 "
                         "for the BERT-large layer, 6 for the BERT-base layer")
    ap.add_argument("--graph", type=int, default=1, choices=[0, 1],
                    help="1: replay each step as a captured CUDA graph (multi launch; mask seeds read from device "
                         "memory, fresh every step)")
    ap.add_argument("--blocking", default="tuned", choices=["tuned", "model"],
                    help="tuned: he_autotune_blocking per product at set-up; model: the cost model's choice")
    ap.add_argument("--ntt-radix", default="tuned", choices=["tuned", "3", "4", "5"],
                    help="log2 of the values per thread of the transforms: tuned = he_autotune_ntt_radix at set-up")
    ap.add_argument("--mac-engine", default="auto", choices=["auto", "integer", "tensor", "coset"],
                    help="multiply-accumulate engine (he_set_mac_engine): auto = the coset form where n_b k_b <= N/2, "
                         "else the tensor cores from 32 k-blocks on")
    ap.add_argument("--full-c0", action="store_true",
                    help="return all of c0 instead of only the decoded coefficients (Sec. 3.1.3)")
    return ap.parse_args()


# ------------------------------------------------------------------ distributed plumbing


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "gb300" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.dev = device_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ the layer


class Layer:
    """Device state of one layer's products: resident weights, input ciphertexts, outputs.
    Products that occur once per head run as one same-shape batch (he_matmul_batch)."""

    def __init__(self, B, ctx, prods, rank, want_host, flags, tune=True, multi=True, graph=False, host_depth=6):
        import numpy as np
        import torch

        from paper_2305_18396_gb300 import synthetic as S

        self.B, self.ctx, self.flags = B, ctx, flags
        self.calls = []
        dev = ctx.device
        self.sk = B.he_keygen(ctx, S.SEED_KEY + 1000 * rank)
        max_ws = max_pt = max_hostws = 0
        idx = 0
        for p in prods:
            if tune:  # measured choice among the cost model's best blockings (set-up, untimed)
                blk = ctx.autotune_blocking(p.m, p.k, p.n, p.share_weights, flags, p.count)[0]
            else:
                blk = ctx.default_blocking(p.m, p.k, p.n, p.share_weights)
            si = ctx.sizes(p.m, p.k, p.n, blk)
            ow, wb = B._out_ws(si, flags)
            si = dict(si, out=ow, ws=wb)
            cnt = p.count
            max_ws = max(max_ws, cnt * wb)
            max_hostws = max(max_hostws, cnt * B.matmul_host_workspace_words(ctx, p.m, p.k, p.n, blk, flags))
            seed = 10_000 * (rank + 1) + idx
            Xs = [S.uniform_share((p.m, p.k), seed + b) for b in range(cnt)]
            if p.share_weights:
                Ws = [S.uniform_share((p.k, p.n), seed + 500_000 + b) for b in range(cnt)]
            else:
                Ws = [S.fixed_point_weights((p.k, p.n), seed + 500_000 + b) for b in range(cnt)]
            Xd = torch.from_numpy(np.concatenate([x.reshape(-1) for x in Xs]).view(np.int64)).to(dev)
            Wd = torch.from_numpy(np.concatenate([w.reshape(-1) for w in Ws]).view(np.int64)).to(dev)
            polys = ctx.empty(cnt * si["packed_words"])
            for b in range(cnt):
                B.he_pack_input(ctx, Xd[b * p.m * p.k:(b + 1) * p.m * p.k], p.m, p.k, blk,
                                polys=polys[b * si["packed_words"]:(b + 1) * si["packed_words"]])
            ct_in = B.he_encrypt(ctx, self.sk, polys, seed + 900_000)
            call = dict(p=p, blk=blk, si=si, cnt=cnt, ct_in=ct_in, out=ctx.empty(cnt * si["out"]), idx=idx,
                        tc=ctx.uses_tensor_cores(p.k, blk), coset=ctx.uses_cosets(blk))
            if p.share_weights:
                call["W"] = Wd  # the server's shares, encoded on every step
                max_pt = max(max_pt, cnt * si["pt_words"])
            else:
                call["pt"] = B.he_encode_weights_batch(ctx, Wd, p.k, p.n, blk, cnt)  # resident NTT-form weights
            if want_host:
                call["in_host"] = ct_in.cpu().pin_memory()
                call["out_host"] = torch.empty(cnt * si["out"], dtype=torch.int64).pin_memory()
            self.calls.append(call)
            idx += cnt
        self.ws = ctx.empty(max((max_ws + 7) // 8, 1))
        self.pt_tmp = ctx.empty(max(max_pt, 1))
        # one multi-product launch per step: every product of the layer as one item (the
        # server's per-step shares encoded into a buffer per launch group first)
        self.multi = multi
        if multi:
            items = []
            for c in self.calls:
                p, si, cnt = c["p"], c["si"], c["cnt"]
                if "pt" not in c:
                    c["pt_step"] = ctx.empty(cnt * si["pt_words"])
                pt_all = c.get("pt", c.get("pt_step"))
                for b in range(cnt):
                    items.append(dict(ct_in=c["ct_in"][b * si["in_words"]:(b + 1) * si["in_words"]],
                                      pt=pt_all[b * si["pt_words"]:(b + 1) * si["pt_words"]],
                                      ct_out=c["out"][b * si["out"]:(b + 1) * si["out"]], m=p.m, k=p.k, n=p.n,
                                      blk=c["blk"], flags=flags, mask_seed=0))
            self.items = items
            # at most 64 products per multi-product launch: larger layers run as consecutive
            # launches on one stream, sharing one workspace
            self.prod_chunks = [B.make_products(items[i:i + 64]) for i in range(0, len(items), 64)]
            self.prods = [a for arr in self.prod_chunks for a in arr]
            self.multi_ws = ctx.empty(max(B.he_multi_workspace_bytes(ctx, arr) for arr in self.prod_chunks) // 8 + 1)
            # seed of item b of launch group c on step s: (s << 20) + idx_c + b
            self.seed_offs = np.array([c["idx"] + b for c in self.calls for b in range(c["cnt"])], dtype=np.int64)
        # host-buffer steps of the whole-layer launch through an he_pipe: uploads, kernels and
        # downloads of consecutive steps overlap on the pipe's three streams over `host_depth`
        # staging slots; inputs are shared (read-only), each slot's step downloads into its
        # own pinned output buffers, and the server's per-step shares are encoded on the
        # pipe's compute stream (in order with its launches) into one set of buffers
        self.pipe, self.host_sets, self.host_k = None, [], 0
        if multi and want_host:
            self.pipe = B.Pipe(ctx, depth=host_depth)
            pt_bufs = {}
            for sidx in range(host_depth):
                items = []
                for c in self.calls:
                    p, si, cnt = c["p"], c["si"], c["cnt"]
                    pt_all = c.get("pt")
                    if pt_all is None:
                        if c["idx"] not in pt_bufs:
                            pt_bufs[c["idx"]] = ctx.empty(cnt * si["pt_words"])
                        pt_all = pt_bufs[c["idx"]]
                    out_h = torch.empty(cnt * si["out"], dtype=torch.int64).pin_memory()
                    for b in range(cnt):
                        items.append(dict(ct_in=c["in_host"][b * si["in_words"]:(b + 1) * si["in_words"]],
                                          pt=pt_all[b * si["pt_words"]:(b + 1) * si["pt_words"]],
                                          ct_out=out_h[b * si["out"]:(b + 1) * si["out"]], m=p.m, k=p.k, n=p.n,
                                          blk=c["blk"], flags=flags, mask_seed=0, keep=out_h))
                self.host_sets.append((B.make_products(items), items))
            self.pipe_pt = pt_bufs
            self.pipe_ws = ctx.empty(self.pipe.workspace_bytes(self.host_sets[0][0]) // 8 + 1)
        self.graph, self.graph_kernels = None, 0
        if multi and graph:  # the replayed graph reads every product's mask seed from device memory
            self.seeds_dev = torch.zeros(len(self.prods), dtype=torch.int64, device=dev)
            for i, a in enumerate(self.prods):
                a.flags |= B.HE_SEED_DEVICE
                a.mask_seed = self.seeds_dev.data_ptr() + 8 * i
        self.host_ws = [ctx.empty(max_hostws), ctx.empty(max_hostws)] if want_host else None
        self.host_streams = [torch.cuda.Stream(device=dev) for _ in range(max(2, host_depth))] if want_host else None
        self.enc_done = torch.cuda.Event()
        self.torch = torch
        self.macs = sum(c["p"].m * c["p"].k * c["p"].n * c["cnt"] for c in self.calls)
        self.products = sum(c["cnt"] for c in self.calls)
        torch.cuda.synchronize()

    def _multi_body(self, serial=False):
        """The per-step encodings of the server's shares, one per product shape, run side by
        side on their own streams (their small grids overlap instead of each draining
        alone), joined before the whole-layer launch; a captured graph keeps the fork.
        serial: all on the current stream (the per-kernel timing pass, whose events on one
        stream then time each kernel alone)."""
        B, ctx, torch = self.B, self.ctx, self.torch
        enc = [c for c in self.calls if "pt_step" in c]
        main = torch.cuda.current_stream()
        if not hasattr(self, "enc_streams"):
            self.enc_streams = [torch.cuda.Stream(device=ctx.device) for _ in enc]
        if serial:
            for c in enc:
                p = c["p"]
                B.he_encode_weights_batch(ctx, c["W"], p.k, p.n, c["blk"], c["cnt"], pt=c["pt_step"], stream=main)
            for arr in self.prod_chunks:
                B.he_matmul_multi(ctx, arr, self.multi_ws)
            return
        for c, st in zip(enc, self.enc_streams):
            st.wait_stream(main)
            p = c["p"]
            B.he_encode_weights_batch(ctx, c["W"], p.k, p.n, c["blk"], c["cnt"], pt=c["pt_step"], stream=st)
        for st in self.enc_streams:
            main.wait_stream(st)
        for arr in self.prod_chunks:
            B.he_matmul_multi(ctx, arr, self.multi_ws)

    def capture(self):
        """Capture one step (per-step encodings + the whole-layer launch) as a CUDA graph."""
        torch, B = self.torch, self.B
        self.seeds_dev.copy_(torch.from_numpy(self.seed_offs))
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self._multi_body()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        l0 = B.he_launch_count(self.ctx)
        with torch.cuda.graph(self.graph):
            self._multi_body()
        self.graph_kernels = B.he_launch_count(self.ctx) - l0
        torch.cuda.synchronize()

    def step(self, step_idx, host=False, eager=False):
        B, ctx = self.B, self.ctx
        if self.multi and host:  # enqueue only: the caller waits with self.pipe.wait()
            k = self.host_k
            self.host_k = (k + 1) % len(self.host_sets)
            arr, _ = self.host_sets[k]
            st = self.pipe.compute_stream
            for c in self.calls:
                if c["idx"] in self.pipe_pt:
                    p = c["p"]
                    B.he_encode_weights_batch(ctx, c["W"], p.k, p.n, c["blk"], c["cnt"], pt=self.pipe_pt[c["idx"]],
                                              stream=st)
            seeds = (step_idx << 20) + self.seed_offs
            for i, a in enumerate(arr):
                a.mask_seed = int(seeds[i])
            self.pipe.submit(arr, self.pipe_ws)
            return
        if self.multi and not host:
            seeds = (step_idx << 20) + self.seed_offs
            if self.graph is not None and not eager:
                # this step's seeds into the device words the graph reads, then replay
                self.seeds_dev.copy_(self.torch.from_numpy(seeds).pin_memory(), non_blocking=True)
                self.graph.replay()
                return
            if self.graph is None:
                for i, a in enumerate(self.prods):
                    a.mask_seed = int(seeds[i])
            else:  # eager pass of a graph-mode layer: the products read device seeds
                self.seeds_dev.copy_(self.torch.from_numpy(seeds).pin_memory(), non_blocking=True)
            self._multi_body(serial=eager)
            return
        k = 0
        for c in self.calls:
            p, blk, cnt, si = c["p"], c["blk"], c["cnt"], c["si"]
            pt = c.get("pt")
            if pt is None:
                pt = B.he_encode_weights_batch(ctx, c["W"], p.k, p.n, blk, cnt, pt=self.pt_tmp)
                if host:  # the host-buffer calls below run on two side streams
                    self.enc_done.record()
            seed = (step_idx << 20) | c["idx"]
            if host:
                # host buffers: one C-ABI call per launch group, alternating two streams (each with
                # its own workspace) so one call's transfers overlap the other's kernels
                st = self.host_streams[k % 2]
                if pt is not c.get("pt"):
                    st.wait_event(self.enc_done)
                B.he_matmul_batch_host(ctx, c["in_host"], pt, p.m, p.k, p.n, blk, cnt, seed, c["out_host"],
                                       self.host_ws[k % 2], flags=self.flags | B.HE_ASYNC, stream=st)
                if pt is not c.get("pt"):  # the next per-step encode reuses pt_tmp
                    self.torch.cuda.current_stream().wait_stream(st)
                k += 1
            else:
                B.he_matmul_batch(ctx, c["ct_in"], pt, p.m, p.k, p.n, blk, cnt, seed, c["out"], self.ws,
                                  flags=self.flags)
        if host:
            for st in self.host_streams:
                st.synchronize()

    def algorithmic_bytes(self):
        """Per kernel family: algorithmic HBM bytes of one step (reads + writes, 8-byte words)."""
        tot = {"mac": 0, "mac_tc": 0, "ntt_forward": 0, "intt_mask": 0, "encode_weights": 0, "coset_forward": 0,
               "coset_inverse": 0, "coset_encode": 0}
        for c in self.calls:
            si, p, cnt = c["si"], c["p"], c["cnt"]
            pt_b, in_b = 8 * si["pt_words"], 8 * si["in_words"]
            full_b = 8 * si["out_words"]  # the multiply-accumulate writes both components in full (NTT domain)
            c1_b = full_b // 2
            if c["coset"]:  # 2N words per input and output component in the transform domain
                tot["coset_forward"] += cnt * 3 * in_b
                tot["mac_tc"] += cnt * (pt_b + 2 * in_b + 2 * full_b)
                tot["coset_inverse"] += cnt * (2 * full_b + 8 * si["out"])
                if p.share_weights:
                    tot["coset_encode"] += cnt * (8 * p.k * p.n + pt_b)
                continue
            tot["mac_tc" if c["tc"] else "mac"] += cnt * (pt_b + in_b + full_b)
            tot["ntt_forward"] += cnt * 2 * in_b
            if self.flags:  # c1: read + write; c0: read in full, write the kept coefficients
                tot["intt_mask"] += cnt * 2 * c1_b
                tot["intt_c0_targets"] = tot.get("intt_c0_targets", 0) + cnt * (c1_b + 8 * si["out"] - c1_b)
            else:
                tot["intt_mask"] += cnt * 2 * full_b
            if p.share_weights:
                tot["encode_weights"] += cnt * (8 * p.k * p.n + pt_b)
        tot["intt_c1_c0"] = tot["intt_mask"] + tot.get("intt_c0_targets", 0)  # the whole-layer launch's fused grid
        return tot

    def slot_macs(self, tc=None):
        """Slot-wise modular multiply-accumulates of one step (tc: only the products on the tensor
        cores (True) or on the integer pipe (False)); a coset product performs 2N per pair of
        input and weight blocks and component, twice the N of the NTT domain."""
        L, N = self.ctx.L, self.ctx.N
        return sum(c["cnt"] * c["si"]["nI"] * c["si"]["nJ"] * c["si"]["nLb"] * 2 * L * N * (2 if c["coset"] else 1)
                   for c in self.calls if tc is None or c["tc"] == tc)


def kernel_source_hash():
    """Fingerprint of what sets the multiply-accumulate kernel's DRAM traffic: its
    configuration and body, the headers it includes, the whole-layer launch's kernels (grid
    order), the blocking choice and autotuner (capi.cu) and the workload shapes -- a traffic
    figure recorded for an older fingerprint is stale."""
    csrc = ROOT / "paper_2305_18396_gb300" / "csrc"
    h = hashlib.sha256((csrc / "mac.cuh").read_bytes())
    for f in ("mac_tc.cuh", "mac_tcr.cuh", "coset.cuh", "tcgen05.cuh", "async.cuh", "he_common.cuh", "multi.cu",
              "multi_items.cuh", "coset.cu", "capi.cu"):
        h.update((csrc / f).read_bytes())
    h.update((ROOT / "paper_2305_18396_gb300" / "workloads.py").read_bytes())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, launch, workload=DEFAULT_WORKLOAD):
    """DRAM traffic per launch from the committed ncu summary, if it was taken on this source,
    in this launch mode (per-group launches and the whole-layer launch differ in size) and on
    this workload."""
    for f in (ROOT / "profiles").glob("*.md"):
        txt = f.read_text()
        m = re.search(r"^traffic_kernel:\s*(\S+)\s*$", txt, re.M)
        if not m or m.group(1) != kernel:
            continue
        src = re.search(r"^source_hash:\s*(\S+)\s*$", txt, re.M)
        mode = re.search(r"^traffic_launch:\s*(\S+)\s*$", txt, re.M)
        wl = re.search(r"^traffic_workload:\s*(\S+)\s*$", txt, re.M)
        val = re.search(r"^traffic_bytes_per_launch:\s*([0-9.eE+]+)\s*$", txt, re.M)
        if src and val and mode and wl and src.group(1) == kernel_source_hash() and mode.group(1) == launch \
                and wl.group(1) == workload:
            return float(val.group(1))
    return None


def peaks():
    try:
        return json.loads((ROOT / "MEASURED_PEAKS.json").read_text()), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------------ workload identity


def workload_config(args):
    """The `config` object of the JSON line: what the workload is, identical for the GPU arm
    and the reference arm (how the GPU arm ran it goes under "run")."""
    from paper_2305_18396_gb300 import workloads

    wl = WORKLOADS[args.workload]
    prods = workloads.bert_layer_products(**getattr(workloads, wl["model"]))
    return {"workload": wl["desc"], "N": wl["N"], "L": wl["L"], "log2_t": 37,
            "products_per_step": sum(p.count for p in prods), "plain_macs_per_step": workloads.layer_macs(prods),
            "output": "full ciphertexts" if args.full_c0 else
            "c1 + c0 at the decoded coefficients only (Sec. 3.1.3, HE_DROP_C0)",
            "l2": "inputs larger than L2: one step reads and writes several GB of ciphertexts and weights"}


# ------------------------------------------------------------------ CPU oracle legs


def oracle_sample(workload):
    """The oracle as it stands on a bounded sample of the layer: one head's four attention
    cross products (Q K^T's two cross terms, P V's two), full Pi_MatMul each (encode, NTT,
    multiply-accumulate, inverse NTT, mask).  Imports the oracle and the input generators
    only: nothing of the CUDA library."""
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    import oracle as O
    from paper_2305_18396_gb300 import synthetic as S
    from paper_2305_18396_gb300 import workloads

    wl = WORKLOADS[workload]
    n_poly, l_primes = wl["N"], wl["L"]
    prods = [p for p in workloads.bert_layer_products(distinct_heads=1, **getattr(workloads, wl["model"]))]
    heads = [p for p in prods if p.share_weights]
    heads = heads + [heads[0]]  # qk_x1 has the shape of qk_x0
    P = O.Params(n_poly, l_primes)
    s = O.keygen(P, S.SEED_KEY)
    jobs = []
    for i, p in enumerate(heads):
        blk = ORACLE_BLOCKINGS[(n_poly, p.m, p.k, p.n)]
        X = S.uniform_share((p.m, p.k), 100 + i)
        W = S.uniform_share((p.k, p.n), 200 + i)
        ct = O.encrypt(P, s, O.pack_input(X, blk, n_poly), 300 + i)
        jobs.append((p, blk, ct, W))
    return P, jobs, O


def run_oracle(P, jobs, O, seed):
    macs = 0
    t0 = time.perf_counter()
    for p, blk, ct, W in jobs:
        O.matmul(P, ct, W, p.m, p.k, p.n, blk, seed)
        macs += p.m * p.k * p.n
    return macs, time.perf_counter() - t0


SAMPLE_DESC = "one head's 4 attention cross products ({macs} plain MACs), full Pi_MatMul each on the host cores"


def cpu_baseline(workload, min_s=10.0, max_reps=20):
    """The same sample as the reference arm's step, repeated until at least min_s of CPU work."""
    P, jobs, O = oracle_sample(workload)
    macs, dt, reps = 0, 0.0, 0
    while (dt < min_s and reps < max_reps) or reps == 0:
        m, d = run_oracle(P, jobs, O, 12345 + reps)
        macs, dt, reps = macs + m, dt + d, reps + 1
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": macs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": SAMPLE_DESC.format(macs=macs // reps) + f", {reps} passes in {dt:.1f} s"}


def reference_arm(args, world, rank):
    if rank != 0:
        return
    P, jobs, O = oracle_sample(args.workload)
    for w in range(args.warmup):
        run_oracle(P, jobs, O, w)
    tot_macs, tot_t, per = 0, 0.0, []
    for k in range(args.steps):
        macs, dt = run_oracle(P, jobs, O, 1000 + k)
        tot_macs += macs
        tot_t += dt
        per.append(dt * 1e3)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    v = tot_macs / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "per step: " + SAMPLE_DESC.format(macs=tot_macs // args.steps)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "latency_ms": {"p50": statistics.median(per), "p99": sorted(per)[min(len(per) - 1, int(0.99 * len(per)))]}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving leg


def serving_leg(B, ctx, args):
    """Poisson arrivals of single-product requests (BERT-base and BERT-large layer matrices,
    m log-uniform in [8, 512]): continuous batching vs the plain per-request path."""
    import torch

    from paper_2305_18396_gb300 import serving as SV

    specs = [("base.qkv", 768, 2304, 512), ("base.out", 768, 768, 512), ("base.ffn1", 768, 3072, 512),
             ("base.ffn2", 3072, 768, 512), ("large.qkv", 1024, 3072, 512), ("large.out", 1024, 1024, 512),
             ("large.ffn1", 1024, 4096, 512), ("large.ffn2", 4096, 1024, 512)]
    models = SV.make_models(ctx, specs)
    out = {"requests_per_rate": f"min({args.serving_requests}, 10 s of arrivals), at least 100", "N": ctx.N,
           "mix": "BERT-base/large layer matrices (QKV, out, FFN1, FFN2), m log-uniform in [8, 512], Poisson arrivals",
           "resident_weight_gb": round(sum(m.pt.numel() for m in models) * 8 / 1e9, 2),
           "policy": "up to 2 launches in flight, a second one only while the first is estimated to end within 2 "
                     "ms; each on a stream of lower CUDA priority than those running; a launch "
                     "takes the oldest admitted request plus, in arrival order, requests whose estimated device "
                     "time fits 1.25 x the oldest's (at least 1 ms) and every request of the oldest's weight "
                     "matrix (merged into one product sharing the weight stream), up to 16; admission by a 32 GiB "
                     "device budget for outputs + workspace; outputs released on completion", "rates": {}}
    for rate in [float(x) for x in args.serving_rates.split(",") if x]:
        res = {}
        count = max(100, min(args.serving_requests, int(rate * 10)))  # at most ~10 s of arrivals per path
        for name, fn, kw in (("per_request", SV.run_per_request, {"keep_outputs": False}),
                             ("continuous_batching", SV.run_served,
                              {"slots": 2, "max_batch": 16, "keep_outputs": False})):
            reqs = SV.make_requests(models, count, rate)
            st, _ = fn(ctx, models, reqs, **kw)
            res[name] = {k: (round(v, 3) if isinstance(v, float) else v) for k, v in st.items()}
        out["rates"][str(int(rate))] = res
    del models
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ batched requests (one launch vs one per request)

BATCHED_MATRICES = [("base.qkv", 768, 2304), ("base.ffn2", 3072, 768), ("large.out", 1024, 1024),
                    ("large.ffn1", 1024, 4096)]


def batched_leg(B, ctx, flags, reps=5, count=64):
    """Mixed requests of resident BERT-base / BERT-large layer matrices, sequence lengths
    uniform in [16, 512]: 64 requests at the context's N, device-resident.  Times the whole
    set as he_matmul_multi launches of at most 64 products against one he_matmul call per
    request on the same stream, and checks that every request's output is the same bit for
    bit both ways."""
    import numpy as np
    import torch

    from paper_2305_18396_gb300 import synthetic as S

    rng = np.random.default_rng(31 + ctx.N)
    sk = B.he_keygen(ctx, S.SEED_KEY)
    weights = {}
    for idx, (name, k, n) in enumerate(BATCHED_MATRICES):
        blk = ctx.default_blocking(128, k, n)  # the blocking is fixed per weight matrix
        W = torch.from_numpy(S.fixed_point_weights((k, n), 800 + idx).view(np.int64).reshape(-1)).to(ctx.device)
        weights[name] = (k, n, blk, B.he_encode_weights(ctx, W, k, n, blk))
    items, alone, macs, ws_words = [], [], 0, 1
    for r in range(count):
        name = BATCHED_MATRICES[int(rng.integers(0, len(BATCHED_MATRICES)))][0]
        k, n, blk, pt = weights[name]
        m = int(rng.integers(16, 513))
        X = torch.from_numpy(S.uniform_share((m, k), 8000 + r).view(np.int64).reshape(-1)).to(ctx.device)
        ct = B.he_encrypt(ctx, sk, B.he_pack_input(ctx, X, m, k, blk), 8500 + r)
        del X
        si = ctx.sizes(m, k, n, blk)
        ow, wb = B._out_ws(si, flags)
        ws_words = max(ws_words, (wb + 7) // 8)
        items.append(dict(ct_in=ct, pt=pt, ct_out=ctx.empty(ow), m=m, k=k, n=n, blk=blk, flags=flags,
                          mask_seed=9000 + r))
        alone.append(ctx.empty(ow))
        macs += m * k * n
    chunks = [B.make_products(items[i:i + 64]) for i in range(0, len(items), 64)]
    ws_multi = ctx.empty(max(B.he_multi_workspace_bytes(ctx, arr) for arr in chunks) // 8 + 1)
    ws_one = ctx.empty(ws_words)
    stream = torch.cuda.current_stream()

    def multi():
        for arr in chunks:
            B.he_matmul_multi(ctx, arr, ws_multi)

    def separate():
        for it, out in zip(items, alone):
            B.he_matmul(ctx, it["ct_in"], it["pt"], it["m"], it["k"], it["n"], it["blk"], it["mask_seed"],
                        ct_out=out, workspace=ws_one, flags=flags)

    res = {}
    for name, fn in (("one_launch", multi), ("per_request", separate)):
        for _ in range(2):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"ms": round(ms, 3), "value": macs / (ms / 1e3), "unit": UNIT}
    B.he_device_status(ctx)
    same = all(torch.equal(it["ct_out"], out) for it, out in zip(items, alone))
    ms_ = [it["m"] for it in items]
    out = {"what": f"{count} requests of mixed BERT-base/large layer matrices (QKV, FFN2, large attn-out, large "
                   f"FFN1), m uniform in [16, 512], N={ctx.N}, inputs resident: {len(chunks)} he_matmul_multi "
                   "launch(es) of at most 64 products vs one he_matmul call per request",
           "N": ctx.N, "launches": len(chunks),
           "requests": count, "plain_macs": macs, "m_min": min(ms_), "m_max": max(ms_),
           "speedup": round(res["per_request"]["ms"] / res["one_launch"]["ms"], 3),
           "outputs_identical": bool(same), **res}
    del items, alone, chunks, ws_multi, ws_one, weights
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ server-local share products


def share_products_leg(B, ctx, prods, mad_peak, reps=20):
    """The server's plaintext side of the same layer (Sec. 3.1.1): W<x>_1 + b for the four
    fully connected products and <X>_1 <Y>_1 for every per-head attention product, through
    he_share_matmul, device-resident, timed with events over `reps` passes."""
    import numpy as np
    import torch

    from paper_2305_18396_gb300 import synthetic as S

    calls, macs = [], 0
    for i, p in enumerate(prods):  # the per-head products of one shape run as one batch
        c = p.count
        X = torch.from_numpy(S.uniform_share((c * p.m, p.k), 900 + i).view(np.int64).reshape(-1)).to(ctx.device)
        W = torch.from_numpy(S.uniform_share((c * p.k, p.n), 950 + i).view(np.int64).reshape(-1)).to(ctx.device)
        bias = None if p.share_weights else torch.from_numpy(
            S.uniform_share((c, p.n), 990 + i).view(np.int64).reshape(-1)).to(ctx.device)
        calls.append((p, X, W, bias, ctx.empty(c * p.m * p.n)))
        macs += p.m * p.k * p.n * c
    stream = torch.cuda.current_stream()

    def one_pass():
        for p, X, W, bias, out in calls:
            B.he_share_matmul_batch(ctx, X, W, p.m, p.k, p.n, p.count, bias=bias, out=out)

    for _ in range(3):
        one_pass()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        one_pass()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    rate = macs / (ms / 1e3)
    # two integer multiply-adds per MAC (one 32x32->64, one 32-bit on the packed cross term,
    # t = 2^37), against the measured mad.wide.u32 rate of the integer pipe
    return {"what": "server-local W<x>_1 + b (4 FC products) and <X>_1 <Y>_1 (24 per-head products, 4 batches) "
                    "of the same layer, he_share_matmul_batch, inputs resident", "macs_per_pass": macs,
            "ms_per_pass": round(ms, 4), "value": rate, "unit": "MAC/s",
            "integer_ops_per_mac": 2, "frac_of_integer_peak": round(2 * rate / mad_peak, 4)}


# ------------------------------------------------------------------ GPU arm


def bert_base_leg(B, args, local, flags, steps=20):
    """The BERT-base layer (seq 128, N=4096, L=2) timed beside the headline workload: same
    launch mode (whole layer in one multi-product launch, CUDA-graph replay, tuned blockings
    and radix), device-resident inputs, CUDA events over `steps` steps."""
    import torch

    from paper_2305_18396_gb300 import workloads

    ctx = B.Context(4096, 2, device=local)
    ctx.set_mac_engine({"auto": B.HE_MAC_AUTO, "integer": B.HE_MAC_INTEGER, "tensor": B.HE_MAC_TENSOR, "coset": B.HE_MAC_COSET}[args.mac_engine])
    if args.ntt_radix == "tuned":
        ctx.autotune_ntt_radix()
    else:
        ctx.set_ntt_radix(int(args.ntt_radix))
    prods = workloads.bert_layer_products(**workloads.BERT_BASE)
    use_graph = args.graph and args.launch == "multi"
    layer = Layer(B, ctx, prods, 0, False, flags, tune=args.blocking == "tuned", multi=args.launch == "multi",
                  graph=use_graph)
    if use_graph:
        layer.capture()
    for w in range(3):
        layer.step(w)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(steps):
        layer.step(1000 + k)
    e1.record(stream)
    torch.cuda.synchronize()
    B.he_device_status(ctx)
    ms = e0.elapsed_time(e1) / steps
    out = {"workload": WORKLOADS["bert-base"]["desc"], "N": 4096, "L": 2, "steps": steps,
           "plain_macs_per_step": layer.macs, "ms_per_step": round(ms, 4), "value": layer.macs / (ms / 1e3),
           "unit": UNIT}
    del layer
    ctx.close()
    torch.cuda.empty_cache()
    return out


def gpu_arm(args, world, rank, local):
    import torch

    from paper_2305_18396_gb300 import binding as B
    from paper_2305_18396_gb300 import workloads

    torch.cuda.set_device(local)
    wl = WORKLOADS[args.workload]
    ctx = B.Context(wl["N"], wl["L"], device=local)
    engine = {"auto": B.HE_MAC_AUTO, "integer": B.HE_MAC_INTEGER, "tensor": B.HE_MAC_TENSOR, "coset": B.HE_MAC_COSET}[args.mac_engine]
    ctx.set_mac_engine(engine)  # before any weights are encoded: it fixes their layout
    if args.ntt_radix == "tuned":  # before the blocking tuner, which times whole products at this radix
        radix_ms = {str(r): round(v, 4) for r, v in ctx.autotune_ntt_radix()[1].items()}
    else:
        ctx.set_ntt_radix(int(args.ntt_radix))
        radix_ms = None
    prods = workloads.bert_layer_products(**getattr(workloads, wl["model"]))
    want_host = not args.no_e2e
    flags = B.HE_FLAGS_NONE if args.full_c0 else B.HE_DROP_C0
    use_graph = args.graph and args.launch == "multi"
    host_depth = args.host_depth or wl["host_depth"]
    layer = Layer(B, ctx, prods, rank, want_host, flags, tune=args.blocking == "tuned", multi=args.launch == "multi",
                  graph=use_graph, host_depth=host_depth)
    stream = torch.cuda.current_stream()

    mad_peak, mad_per_sm_clk = B.he_probe_mad_wide(ctx)
    if use_graph:
        layer.capture()
    for w in range(max(args.warmup, 3) if args.warmup else 0):
        layer.step(w)
    torch.cuda.synchronize()

    # headline: K steps, device-resident inputs, CUDA events per step on the launching stream
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = B.he_launch_count(ctx)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(args.steps):
            evs[k][0].record(stream)
            layer.step(1000 + k)
            evs[k][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    launches = B.he_launch_count(ctx) - l0 + layer.graph_kernels * args.steps  # graph replays: captured kernels
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), world, device=f"cuda:{local}")
    per = [a.elapsed_time(b) for a, b in evs]
    ms_per_step = total_ms / args.steps
    value = world * layer.macs * args.steps / (total_ms / 1e3)

    # roofline: per-kernel event timing (separate pass, same steps, every kernel on one stream)
    B.he_profile_enable(ctx, True)
    steps_prof = max(3, min(args.steps, 10))
    for k in range(steps_prof):
        layer.step(5000 + k, eager=True)
    stats = B.he_profile_read(ctx)
    B.he_profile_enable(ctx, False)
    alg = layer.algorithmic_bytes()
    pk, pk_src = peaks()
    dom = max(stats, key=lambda k: stats[k]["total_ms"])
    total_prof_ms = sum(v["total_ms"] for v in stats.values())
    kern = {}
    for name, v in stats.items():
        b = alg.get(name, 0) * steps_prof
        kern[name] = {"launches": v["launches"], "ms": round(v["total_ms"], 3),
                      "share": round(v["total_ms"] / total_prof_ms, 4),
                      "gbs": round(b / (v["total_ms"] / 1e3) / 1e9, 1) if b else None}
    per_launch_s = stats[dom]["total_ms"] / stats[dom]["launches"] / 1e3
    launches_per_step = stats[dom]["launches"] / steps_prof
    bytes_per_launch = alg.get(dom, 0) / launches_per_step
    hbm_gbs = bytes_per_launch / per_launch_s / 1e9
    if dom == "mac_tc":
        # tensor-core multiply-accumulate: 49 digit products (2 flops each) per slot product, bf16
        # on tcgen05, against the measured dense bf16 rate (sustained: the kernel runs inside a
        # long step), and its HBM bytes against the measured copy bandwidth; the bound named is
        # the roof it runs closest to
        tc_peak = 1e12 * pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1700.0))
        flops_per_launch = 2 * 49 * layer.slot_macs(True) / launches_per_step
        tflops = flops_per_launch / per_launch_s
        fr_t, fr_h = tflops / tc_peak, hbm_gbs / pk["hbm_gbs"]
        t_obj = {"achieved": round(tflops / 1e12, 2), "peak": round(tc_peak / 1e12, 1), "unit": "TFLOP/s",
                 "frac": round(fr_t, 4), "peak_source": f"{pk_src}: bf16 dense, sustained",
                 "tcgen05_probe_tflops": round(B.he_probe_tensor(ctx, 0) / 1e12, 1),
                 "flops_per_launch": flops_per_launch}
        h_obj = {"achieved": round(hbm_gbs, 1), "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": round(fr_h, 4),
                 "peak_source": pk_src}
        main, other, bound = (h_obj, t_obj, "hbm") if fr_h >= fr_t else (t_obj, h_obj, "tensor")
        roofline = {"bound": bound, "kernel": dom, **{k: main[k] for k in ("achieved", "peak", "unit", "frac",
                                                                           "peak_source")},
                    ("tensor" if bound == "hbm" else "hbm"): other,
                    "slot_products_per_s": layer.slot_macs(True) * steps_prof / (stats[dom]["total_ms"] / 1e3)}
    elif dom == "mac":
        # integer-pipe bound: three mad.wide.u32 per slot product (Karatsuba), peak measured by
        # he_probe_mad_wide on this GPU (per-SM rate x SMs x clock)
        ops_per_launch = 3 * layer.slot_macs(False) / launches_per_step
        achieved = ops_per_launch / per_launch_s
        roofline = {"bound": "alu", "kernel": dom, "achieved": round(achieved / 1e12, 3),
                    "peak": round(mad_peak / 1e12, 3), "unit": "T mad.wide.u32/s", "frac": round(achieved / mad_peak, 4),
                    "peak_source": f"measured: he_probe_mad_wide, {mad_per_sm_clk:.1f} per SM per clock",
                    "ops_per_launch": ops_per_launch,
                    "hbm": {"achieved": round(hbm_gbs, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                            "frac": round(hbm_gbs / pk["hbm_gbs"], 4), "peak_source": pk_src}}
    else:
        roofline = {"bound": "hbm", "kernel": dom, "achieved": round(hbm_gbs, 1), "peak": pk["hbm_gbs"],
                    "unit": "GB/s", "frac": round(hbm_gbs / pk["hbm_gbs"], 4), "peak_source": pk_src}
    roofline.update({"algorithmic_bytes_per_launch": bytes_per_launch, "traffic": recorded_traffic(dom, args.launch, args.workload),
                     "kernels": kern,
                     "slot_macs_per_s": layer.slot_macs(False) * steps_prof / (stats["mac"]["total_ms"] / 1e3)
                     if "mac" in stats and layer.slot_macs(False) else None})

    # end to end: host buffers through he_matmul_host (H2D + compute + D2H inside the region)
    e2e = None
    if want_host:
        h2d = sum(8 * c["cnt"] * c["si"]["in_words"] for c in layer.calls)
        d2h = sum(8 * c["cnt"] * c["si"]["out"] for c in layer.calls)
        for w in range(max(2, len(layer.host_sets))):  # every slot's buffers once before timing
            layer.step(9000 + w, host=True)
        if layer.pipe is not None:
            layer.pipe.wait()
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ksteps = max(1, min(args.steps, 40))
        for k in range(ksteps):
            layer.step(9100 + k, host=True)
        if layer.pipe is not None:
            layer.pipe.wait()
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, world, device=f"cuda:{local}")
        e2e = {"value": world * layer.macs * ksteps / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "steps_in_flight": len(layer.host_sets) if layer.multi else 2,
               "d2h_bytes_per_step": d2h, "steps": ksteps, "ms_per_step": dt * 1e3 / ksteps}

    share = share_products_leg(B, ctx, prods, mad_peak)
    blks = {}
    for c in layer.calls:
        blks.setdefault(c["p"].name, list(c["blk"]))
    layer_multi, n_calls = layer.multi, len(layer.calls)
    tc_calls = [c for c in layer.calls if ctx.uses_tensor_cores(c["p"].k, c["blk"])]
    batched = batched_leg(B, ctx, flags) if world == 1 and not args.no_batched else None

    serving = None
    if world == 1 and not args.no_serving:
        serving = serving_leg(B, ctx, args)
    base_layer = None
    if world == 1 and args.workload != "bert-base" and not args.no_bert_base:
        del layer
        torch.cuda.empty_cache()
        base_layer = bert_base_leg(B, args, local, flags)
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(args),
        "run": {"blockings_mkn": blks, "blocking_choice": args.blocking, "launch": args.launch,
                "mac_engine": args.mac_engine,
                "tensor_core_products": sum(c["cnt"] for c in tc_calls), 
                "launch_groups_per_step": 1 if layer_multi else n_calls,
                "ntt_values_per_thread": 1 << ctx.ntt_radix, "ntt_radix_choice": args.ntt_radix,
                "ntt_radix_round_trip_ms": radix_ms, "cuda_graph": bool(use_graph),
                "kernel_source_hash": kernel_source_hash(),
                "parallelism": f"replicas x{world} (independent layers, no collective)"},
        "latency_ms": {"p50": statistics.median(per), "p99": sorted(per)[min(len(per) - 1, int(0.99 * len(per)))]},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "serving": serving, "share_products": share,
        "batched_requests": batched, "bert_base_layer": base_layer,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        reference_arm(args, world, rank)
    else:
        gpu_arm(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
