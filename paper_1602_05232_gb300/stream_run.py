"""Run the first B minibatches of a benchmark stream with the tuned options.

A fixed, short workload for profilers (the ncu summaries under profiles/ name
this command): the first B minibatches' edges and pairs are copied to the
device first, then each minibatch's Bulk-Update and Bulk-Query run in stream
order on one forest with bench.py's launch options for that workload.

    python -m paper_1602_05232_gb300.stream_run --workload grid --minibatches 24
    python -m paper_1602_05232_gb300.stream_run --workload grid --minibatches 16 \
        --opt big_filter=0 --opt compress_every=4     # an earlier configuration
"""
from __future__ import annotations

import argparse
import sys
from pathlib import Path


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", choices=["grid", "rmat"], default="grid")
    ap.add_argument("--minibatches", type=int, default=16)
    ap.add_argument("--opt", action="append", default=[], metavar="KEY=VALUE",
                    help="launch option over the tuned ones (repeatable)")
    args = ap.parse_args(argv)

    import torch
    sys.path.insert(0, str(Path(__file__).resolve().parents[1]))
    from bench import launch_options
    from paper_1602_05232_gb300 import cc, inputs as I

    s = I.grid_stream(seed=0) if args.workload == "grid" else I.rmat_stream(seed=0)
    B = max(1, min(args.minibatches, s.batches))
    eoff, qoff = s.edge_offsets(), s.query_offsets()
    e = torch.from_numpy(s.edges_range(0, int(eoff[B]))).cuda()
    q = torch.from_numpy(I.uniform_pairs(s.n, int(qoff[B]), s.seed, I.TAG_QUERIES, 0)).cuda()
    o = torch.empty(int(qoff[B]), dtype=torch.uint8, device="cuda")
    opts = launch_options(args.workload)
    for kv in args.opt:
        k, v = kv.split("=", 1)
        if k not in cc.OPTIONS:
            ap.error(f"unknown option {k}")
        opts[k] = int(v)
    f = cc.Forest(s.n, **opts)
    for b in range(B):
        f.bulk_update(e[eoff[b]:eoff[b + 1]])
        f.bulk_query(q[qoff[b]:qoff[b + 1]], out=o[qoff[b]:qoff[b + 1]])
    f.sync()
    torch.cuda.synchronize()
    print(f"{args.workload}: {B} minibatches, {f.components()} components, launches {f.kernel_stats()}")
    f.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
