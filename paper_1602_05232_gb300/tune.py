"""Autotuner for libcc's launch options.

Picks, per workload and device, the options that minimise the time of one
pass over a workload's minibatch stream:
  * plain form: Bulk-Update kernel variant, edges (pairs) per thread, block
    size, how often cc_bulk_update runs the full compression pass, and
    whether Bulk-Query halves paths;
  * batched form: CTA size, edges per thread, the shared-memory graph-size
    cap (which also sets how many CTAs fit on an SM) and the persistent
    grid size.

The search is coordinate descent from a starting point: each parameter in
turn is swept with the others fixed, keeping the best, for a few rounds; the
best few configurations seen are then re-timed and the fastest wins. Every
evaluation is the median of `repeats` passes timed with CUDA events on the
forest's stream, each pass starting from an empty forest (reset not timed).

Results are cached in ``tuned.json`` next to this file, keyed by device name
and workload; ``tuned_options()`` reads them. Run as a module on the GPU to
(re)tune: ``python -m paper_1602_05232_gb300.tune --workload rmat --write``.
"""
from __future__ import annotations

import argparse
import json
import statistics
from pathlib import Path

import numpy as np
import torch

from . import cc
from . import inputs as I

CACHE = Path(__file__).resolve().parent / "tuned.json"

PLAIN_SPACE = {
    "update_variant": [0, 1, 2, 3, 4, 5],
    "edges_per_thread": [1, 2, 4],
    "block": [128, 256, 512, 1024],
    "compress_every": [0, 1, 2, 3, 4, 6, 8, 16],
    "compress_scope": [0, 1],
    "query_halving": [0, 1, 2],
    "l2_persist": [0, 1],
    "query_variant": [0, 1, 2],
    "pdl": [0, 1, 2],
    "query_pairs_per_thread": [0, 1, 2, 4],
    "hook": [0, 1, 2],
    "edge_order": [0, 7, 9],
    "hook_warp": [0, 1],
    "big_filter": [0, 384, 640, 896],
}
# options that only act together: the largest-component filter is built by
# full compression passes, so it does nothing while compression is off
PLAIN_PAIRS = (("big_filter", "compress_every"),)

PLAIN_START = {"update_variant": 0, "edges_per_thread": 2, "block": 256, "compress_every": 1,
               "compress_scope": 0, "query_halving": 0, "l2_persist": 0, "query_variant": 0,
               "pdl": 1, "query_pairs_per_thread": 0, "hook": 0, "edge_order": 0, "hook_warp": 0,
               "big_filter": 0}

SEG_SPACE = {
    "seg_block": [128, 256, 512, 1024],
    "seg_edges_per_thread": [1, 2, 4],
    "seg_smem_cap": [65536, 32768, 16384],
    "seg_max_ctas": [0, 152, 304],
}
SEG_START = {"seg_block": 512, "seg_edges_per_thread": 1, "seg_smem_cap": 65536,
             "seg_max_ctas": 0, "seg_graph": 1}


def device_name() -> str:
    return torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"


def tuned_options(workload: str, device: str | None = None) -> dict | None:
    """Cached best options for `workload` on `device` (default: the current
    CUDA device), or None.

    The result may contain pdl=2 (programmatic dependent launch reading each
    thread's first pairs before waiting for the previous kernel). That is only
    valid when the edge/pair arrays are not written by the kernel launched just
    before on the same stream -- true for the benchmarks' resident streams and
    for inputs copied in, not for edges produced by a caller's own kernel
    right before the call. Such callers set pdl to 1 (or 0)."""
    try:
        d = json.loads(CACHE.read_text())
        return dict(d[device or device_name()][workload]["options"])
    except Exception:
        return None


def _store(workload: str, best: dict, ms: float, table: list) -> None:
    d = json.loads(CACHE.read_text()) if CACHE.exists() else {}
    d.setdefault(device_name(), {})[workload] = {
        "options": best, "ms_per_pass": round(ms, 4),
        "evaluated": [{"options": o, "ms": round(t, 4)} for o, t in sorted(table, key=lambda x: x[1])[:12]],
    }
    CACHE.write_text(json.dumps(d, indent=1, sort_keys=True) + "\n")


def coordinate_descent(space: dict, start, evaluate, rounds: int = 2, finalists: int = 3,
                       log=None, pairs=()) -> tuple[dict, float, list]:
    """Minimise evaluate(options) over the product space by sweeping one
    parameter at a time, from one start point or from each of a list of them
    (sharing the measurements); the best few points seen are timed again and
    the fastest wins. `pairs`: options that only act together (each (a, b) is
    also swept over the product of their values in every round), which single
    moves cannot find from a start where neither is on. Returns (best options,
    time, [(options, time)])."""
    seen: dict[str, float] = {}

    def ev(o):
        key = json.dumps(o, sort_keys=True)
        if key not in seen:
            seen[key] = evaluate(o)
            if log:
                log(o, seen[key])
        return seen[key]

    for s0 in ([start] if isinstance(start, dict) else list(start)):
        best = dict(s0)
        best_t = ev(best)
        for _ in range(rounds):
            improved = False
            for name, values in space.items():
                for v in values:
                    cand = dict(best, **{name: v})
                    t = ev(cand)
                    if t < best_t:
                        best, best_t, improved = cand, t, True
            for a, b in pairs:
                for va in space.get(a, ()):
                    for vb in space.get(b, ()):
                        cand = dict(best, **{a: va, b: vb})
                        t = ev(cand)
                        if t < best_t:
                            best, best_t, improved = cand, t, True
            if not improved:
                break
    table = [(json.loads(k), t) for k, t in seen.items()]
    top = sorted(table, key=lambda x: x[1])[:finalists]
    retimed = [(o, min(t, evaluate(o))) for o, t in top]
    best, best_t = min(retimed, key=lambda x: x[1])
    return best, best_t, table


def starts_for(workload: str, space: dict, default: dict) -> list[dict]:
    """The default start point and, when this device has a stored result for
    the workload, that result too (completed with the defaults for options it
    predates, and only if every value is still in the space): descent from a
    single point can settle in a worse local optimum, and a retune should not
    end up slower than what is stored."""
    starts = [dict(default)]
    cached = tuned_options(workload)
    if cached:
        cand = {k: cached.get(k, default[k]) for k in default}
        if all(cand[k] in space[k] for k in space if k in cand) and cand != starts[0]:
            starts.append(cand)
    return starts


# ------------------------------------------------------------ plain form

class PlainBench:
    """A minibatch stream resident on the device, timed pass by pass."""

    def __init__(self, stream_obj, device="cuda"):
        self.s = stream_obj
        self.d_e = torch.from_numpy(stream_obj.all_edges()).to(device)
        self.d_q = torch.from_numpy(stream_obj.all_queries()).to(device)
        self.d_o = torch.empty(stream_obj.q, dtype=torch.uint8, device=device)
        self.eoff = stream_obj.edge_offsets()
        self.qoff = stream_obj.query_offsets()
        self.cuda_stream = torch.cuda.Stream()
        # every minibatch's views made once: on small minibatches, slicing
        # tensors inside the timed pass would time the host, not the kernels
        self.views = [(self.d_e[self.eoff[i]:self.eoff[i + 1]], self.d_q[self.qoff[i]:self.qoff[i + 1]],
                       self.d_o[self.qoff[i]:self.qoff[i + 1]]) for i in range(stream_obj.batches)]

    def time(self, options: dict, repeats: int = 3) -> float:
        st = self.cuda_stream
        with torch.cuda.stream(st):
            f = cc.Forest(self.s.n, stream=st, **options)
            times = []
            for r in range(repeats + 1):
                f.reset()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                for e, q, o in self.views:
                    f.bulk_update(e)
                    f.bulk_query(q, out=o)
                b.record(st)
                st.synchronize()
                if r:  # the first pass warms up
                    times.append(a.elapsed_time(b))
            f.sync()
            f.close()
        return statistics.median(times)


def canonical_plain(options: dict) -> dict:
    """The same launch with options that cannot act set to their defaults: the
    largest-component filter is built only by full compression passes."""
    o = dict(options)
    if o.get("compress_every", 1) == 0 or o.get("compress_scope", 0) == 1:
        o["big_filter"] = 0
    return o


def tune_plain(stream_obj, space=PLAIN_SPACE, start=PLAIN_START, repeats: int = 3, log=None):
    """start: one option dict or a list of them (see coordinate_descent)."""
    bench = PlainBench(stream_obj)
    best, t, table = coordinate_descent(space, start, lambda o: bench.time(o, repeats), log=log,
                                        pairs=PLAIN_PAIRS)
    return canonical_plain(best), t, table


# ---------------------------------------------------------- batched form

class SegmentedBench:
    def __init__(self, w, device="cuda"):
        self.w = w
        self.d_e, self.d_q, self.ops = [], [], []
        m_all = w.total_edges
        self.out = torch.empty(m_all, dtype=torch.uint8, device=device)
        base = 0
        for g in range(w.G):
            self.d_e.append(torch.from_numpy(w.edges(g)).to(device))
            self.d_q.append(torch.from_numpy(w.queries(g)).to(device))
            for kind, off, k in w.ops(g):
                src = self.d_e[g] if kind == 0 else self.d_q[g]
                self.ops.append((g, kind, src.data_ptr() + 8 * off, k,
                                 self.out.data_ptr() + base + off if kind == 1 else 0))
            base += w.m(g)
        self.ops = np.array(self.ops, dtype=cc.OP_DTYPE)
        self.cuda_stream = torch.cuda.Stream()

    def time(self, options: dict, repeats: int = 5) -> float:
        st = self.cuda_stream
        with torch.cuda.stream(st):
            f = cc.Forest.segmented(self.w.n, stream=st, **options)
            times = []
            for r in range(repeats + 1):
                f.reset()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                f.submit(self.ops)
                b.record(st)
                st.synchronize()
                if r:
                    times.append(a.elapsed_time(b))
            f.sync()
            f.close()
        return statistics.median(times)


def tune_segmented(w, space=SEG_SPACE, start=SEG_START, repeats: int = 5, log=None):
    bench = SegmentedBench(w)
    return coordinate_descent(space, start, lambda o: bench.time(o, repeats), log=log)


WORKLOADS = {
    "rmat": lambda: ("plain", I.rmat_stream()),
    "grid": lambda: ("plain", I.grid_stream()),
    "uniform": lambda: ("plain", I.uniform_stream()),
    "serving": lambda: ("plain", I.rmat_stream(scale=26, m=1 << 28, batch=1 << 20, q=1 << 18)),
    "segmented": lambda: ("segmented", I.segmented_workload()),
    "paper-random": lambda: ("plain", I.paper_stream("random", batch=10_000_000, q=1)),
    "paper-rmat5": lambda: ("plain", I.paper_stream("rmat5", batch=10_000_000, q=1)),
    "paper-rmat16": lambda: ("plain", I.paper_stream("rmat16", batch=10_000_000, q=1)),
    "paper-3dgrid": lambda: ("plain", I.paper_stream("3dgrid", batch=10_000_000, q=1)),
}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description="tune libcc launch options on this GPU")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), action="append", required=True)
    ap.add_argument("--write", action="store_true", help="store the result in tuned.json")
    args = ap.parse_args(argv)
    for wl in args.workload:
        form, obj = WORKLOADS[wl]()
        log = lambda o, t: print(f"  {wl}: {t:9.3f} ms  {o}", flush=True)
        if form == "plain":
            best, t, table = tune_plain(obj, start=starts_for(wl, PLAIN_SPACE, PLAIN_START), log=log)
        else:
            best, t, table = tune_segmented(obj, start=starts_for(wl, SEG_SPACE, SEG_START), log=log)
        print(json.dumps({"workload": wl, "device": device_name(), "best": best,
                          "ms_per_pass": round(t, 4), "evaluated": len(table)}), flush=True)
        if args.write:
            _store(wl, best, t, table)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
