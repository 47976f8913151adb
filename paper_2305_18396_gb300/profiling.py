"""Profiling drivers: small, self-contained invocations of the product for `ncu` captures,
and a reader for the per-launch CSV that `ncu --metrics gpu__time_duration.sum --csv`
writes.

    python -m paper_2305_18396_gb300.profiling case M K N [--repeat R] [--full-c0] [--logn 13 --L 3] [--multi]
    python -m paper_2305_18396_gb300.profiling share M K N [--repeat R]
    python -m paper_2305_18396_gb300.profiling launches launches.csv

`case` runs one Pi_MatMul (Algorithm 1) of an M x K share against a K x N weight matrix
at N=4096, L=2 (or --logn / --L) through the public binding (he_matmul, or with --multi
he_matmul_multi): key generation, packing, encryption and
weight encoding once, then R products (compact output, Sec. 3.1.3, unless --full-c0),
then a device status check.  The products are the launches worth capturing; everything
before them is set-up.

`launches` aggregates an ncu launch list by kernel: launches, total device time, share.
"""
import argparse
import collections
import csv
import re
import sys

import numpy as np


def run_case(m, k, n, repeat=3, compact=True, logN=12, L=2, multi=False, engine=0, blk=None, encodes=1):
    import torch

    from . import binding as B
    from . import synthetic as S

    ctx = B.Context(1 << logN, L)
    ctx.set_mac_engine(engine)
    blk = tuple(blk) if blk else ctx.default_blocking(m, k, n)
    X = torch.from_numpy(S.uniform_share((m, k), 1).view(np.int64).reshape(-1)).to(ctx.device)
    W = torch.from_numpy(S.fixed_point_weights((k, n), 2).view(np.int64).reshape(-1)).to(ctx.device)
    sk = B.he_keygen(ctx, 3)
    ct = B.he_encrypt(ctx, sk, B.he_pack_input(ctx, X, m, k, blk), 4)
    for _ in range(encodes):  # encodes > 1: the weight encoding's own kernel, launched again
        pt = B.he_encode_weights(ctx, W, k, n, blk)
    flags = B.HE_DROP_C0 if compact else 0
    out = None
    if multi:  # through the multi-product launch (one product): the kernels of a whole-layer step
        si = ctx.sizes(m, k, n, blk)
        out = ctx.empty(si["out_words_compact"] if compact else si["out_words"])
        prods = B.make_products([dict(ct_in=ct, pt=pt, ct_out=out, m=m, k=k, n=n, blk=blk, flags=flags,
                                      mask_seed=5)])
        ws = ctx.empty(B.he_multi_workspace_bytes(ctx, prods) // 8 + 1)
        for i in range(repeat):
            B.he_matmul_multi(ctx, prods, ws)
    for i in range(0 if multi else repeat):
        out = B.he_matmul(ctx, ct, pt, m, k, n, blk, 5 + i, ct_out=out, flags=flags)
    torch.cuda.synchronize()
    B.he_device_status(ctx)
    return blk, ctx.sizes(m, k, n, blk)


def run_share_case(m, k, n, repeat=3):
    """he_share_matmul (server-local product, Sec. 3.1.1) of an m x k by k x n share."""
    import torch

    from . import binding as B
    from . import synthetic as S

    ctx = B.Context(4096, 2)
    X = torch.from_numpy(S.uniform_share((m, k), 1).view(np.int64).reshape(-1)).to(ctx.device)
    W = torch.from_numpy(S.uniform_share((k, n), 2).view(np.int64).reshape(-1)).to(ctx.device)
    bias = torch.from_numpy(S.uniform_share((1, n), 3).view(np.int64).reshape(-1)).to(ctx.device)
    out = ctx.empty(m * n)
    for _ in range(repeat):
        B.he_share_matmul(ctx, X, W, m, k, n, bias=bias, out=out)
    torch.cuda.synchronize()
    B.he_device_status(ctx)


def _short(name):
    """Kernel name without return type, parameters and anonymous-namespace prefix."""
    name = name.replace("(anonymous namespace)::", "").replace("void ", "")
    return re.sub(r"^.*?unnamed>::", "", name.split("(")[0]).strip()


def summarize_launches(path, skip_prefixes=(), skip_first=0, metric="gpu__time_duration.sum", first=None, back=0,
                       last=None):
    """Per kernel: (launches, total) of `metric` from an ncu --csv launch list (durations in
    microseconds).  Leaves out the first `skip_first` launches and kernels named by a prefix;
    with `first` / `last` keeps only the window from `back` launches before the first launch
    whose name contains `first` to the last launch whose name contains `last`."""
    rows = []
    hdr = None
    with open(path, newline="") as f:
        for r in csv.reader(f):
            if "Kernel Name" in r:
                hdr = r
                continue
            if not hdr or len(r) != len(hdr):
                continue
            d = dict(zip(hdr, r))
            if d.get("Metric Name") != metric or int(d["ID"]) < skip_first:
                continue
            v, u = float(d["Metric Value"].replace(",", "")), d["Metric Unit"]
            if metric == "gpu__time_duration.sum":
                v = v / 1e3 if u in ("ns", "nsecond") else v * 1e3 if u in ("ms", "msecond") else v
            elif u.endswith("byte"):
                v *= {"Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(u, 1.0)
            rows.append((_short(d["Kernel Name"]), v))
    lo, hi = 0, len(rows)
    if first:
        lo = max(0, next(i for i, (nm, _) in enumerate(rows) if first in nm) - back)
    if last:
        hi = max(i for i, (nm, _) in enumerate(rows) if last in nm) + 1
    agg = collections.defaultdict(lambda: [0, 0.0])
    for name, v in rows[lo:hi]:
        if any(name.startswith(p) for p in skip_prefixes):
            continue
        agg[name][0] += 1
        agg[name][1] += v
    return dict(agg)


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("case")
    c.add_argument("m", type=int)
    c.add_argument("k", type=int)
    c.add_argument("n", type=int)
    c.add_argument("--repeat", type=int, default=3)
    c.add_argument("--full-c0", action="store_true")
    c.add_argument("--logn", type=int, default=12, help="log2 N (12 or 13)")
    c.add_argument("--L", type=int, default=2, help="number of primes")
    c.add_argument("--multi", action="store_true", help="run through he_matmul_multi")
    c.add_argument("--engine", type=int, default=0, help="0 auto, 1 integer, 2 tensor (he_set_mac_engine)")
    c.add_argument("--blocking", help="m_b,k_b,n_b (default: the context's default blocking)")
    c.add_argument("--encodes", type=int, default=1, help="weight encodings before the products")
    sh = sub.add_parser("share")
    sh.add_argument("m", type=int)
    sh.add_argument("k", type=int)
    sh.add_argument("n", type=int)
    sh.add_argument("--repeat", type=int, default=3)
    s = sub.add_parser("launches")
    s.add_argument("csv")
    s.add_argument("--skip", action="append", default=[], help="kernel-name prefix to leave out")
    s.add_argument("--skip-first", type=int, default=0, help="leave out the first launches (set-up)")
    s.add_argument("--metric", default="gpu__time_duration.sum")
    s.add_argument("--first", help="window starts at the first launch whose name contains this")
    s.add_argument("--back", type=int, default=0, help="... and this many launches before it")
    s.add_argument("--last", help="window ends at the last launch whose name contains this")
    a = ap.parse_args(argv)
    if a.cmd == "case":
        blk = [int(v) for v in a.blocking.split(",")] if a.blocking else None
        blk, si = run_case(a.m, a.k, a.n, a.repeat, not a.full_c0, a.logn, a.L, a.multi, a.engine, blk, a.encodes)
        print("ok", blk, si)
    elif a.cmd == "share":
        run_share_case(a.m, a.k, a.n, a.repeat)
        print("ok")
    else:
        agg = summarize_launches(a.csv, tuple(a.skip), a.skip_first, a.metric, a.first, a.back, a.last)
        tot = sum(v[1] for v in agg.values()) or 1.0
        print(f"| kernel | launches | total {a.metric} | per launch | share |\n|---|---|---|---|---|")
        for name, (cnt, x) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
            print(f"| `{name}` | {cnt} | {x:.1f} | {x / cnt:.1f} | {100 * x / tot:.1f}% |")
    return 0


if __name__ == "__main__":
    sys.exit(main())
