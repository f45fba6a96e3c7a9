"""Benchmark: bulk incremental connectivity on one GB300 (or N replicas).

Headline workload (default ``grid``): one forest on the 8192 x 8192
4-neighbour grid (n = 2^26, a 256 MiB forest, larger than L2), fed its
134,201,344 edges, shuffled, in 32 minibatches of 2^22; after each
Bulk-Update, one Bulk-Query of 2^22 uniform vertex pairs. A STEP is one whole
pass of that stream from the empty graph: a reset of the forest to n
singletons, then every minibatch's Bulk-Update (with the compression policy)
and Bulk-Query in order. Throughput is total edges over total time (Section
5.3, Table 3).

Timing: W untimed passes, then exactly K passes bracketed by a barrier and a
device synchronise, timed with CUDA events on the forest's stream; the max
over ranks is reported. The edge and pair streams (1 GiB each) are larger
than L2 and each is read once per pass.

The same JSON line carries the other forms (``--forms``): the plain form on
the R-MAT n=2^24 and uniform n=2^16 streams (same step definition), the
batched form (1024 segmented graphs, one persistent kernel replayed as a CUDA
graph) against one launch per minibatch, and the served form (continuous
batching over an R-MAT n=2^26, 2^30-edge request trace) against one request
at a time.

``--impl reference`` times the CPU oracle (sequential union-find with path
compression) on a bounded sample of every pass.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
METRIC = ("Bulk-Update edges/s & Bulk-Query queries/s (1 GB300), % HBM roofline; "
          "p50/p99 batch latency")

# Sector-model algorithmic bytes per unit (random 4-byte parent reads cost a
# 32-byte sector): update 8 B edge + 2 x 32 B; query 8 B pair + 1 B answer +
# 2 x 32 B; full compression 4 B read + 4 B write per vertex. With the
# largest-component filter an edge or pair whose endpoints are both marked
# reads two 32-byte bitmap sectors in place of two parent sectors (the same
# bytes in this model; the 1-bit-per-vertex bitmap stays in L2), and a full
# compression also writes the bitmap, 1/8 B per vertex (BITMAP_BYTES).
BYTES_PER_UNIT = {"update": 72.0, "query": 73.0, "compress_all": 8.0,
                  "compress_touched": 72.0, "labels": 12.0, "reset": 4.0,
                  "order": 24.0}  # edge order: the edges read twice and written once
BITMAP_BYTES = 0.125

# Options of the launches this benchmark times, per workload (also used by
# the full-size parity tests, so they check exactly this configuration).
LAUNCH_OPTIONS = {
    "rmat": {"block": 256, "edges_per_thread": 4, "update_variant": 2, "compress_every": 0,
             "compress_scope": 0},
    "uniform": {"block": 256, "edges_per_thread": 2, "update_variant": 0, "compress_every": 0,
                "compress_scope": 0},
    "grid": {"block": 256, "edges_per_thread": 2, "update_variant": 2, "compress_every": 4,
             "compress_scope": 0},
    "hub": {"block": 256, "edges_per_thread": 4, "update_variant": 2, "compress_every": 0},
    "segmented": {"seg_block": 512, "seg_edges_per_thread": 1, "seg_smem_cap": 65536,
                  "seg_graph": 1},
    "serving": {"block": 256, "edges_per_thread": 4, "update_variant": 2, "compress_every": 0,
                "compress_scope": 0},
    "paper-random": {"block": 256, "edges_per_thread": 4, "update_variant": 2, "compress_every": 0},
    "paper-rmat5": {"block": 256, "edges_per_thread": 4, "update_variant": 2, "compress_every": 0},
    "paper-rmat16": {"block": 256, "edges_per_thread": 4, "update_variant": 2, "compress_every": 0},
    "paper-3dgrid": {"block": 256, "edges_per_thread": 2, "update_variant": 2, "compress_every": 2},
}


OPTION_OVERRIDES: dict = {}


def launch_options(workload: str) -> dict:
    """Autotuned options for this device when cached (paper_1602_05232_gb300/
    tuned.json, written by ``python -m paper_1602_05232_gb300.tune``), else
    the built-in defaults above; ``--opt key=value`` overrides either."""
    try:
        from paper_1602_05232_gb300 import tune
        t = tune.tuned_options(workload)
    except Exception:
        t = None
    opts = t if t is not None else dict(LAUNCH_OPTIONS[workload])
    opts.update(OPTION_OVERRIDES)
    return opts


def make_stream(workload: str, seed: int):
    from paper_1602_05232_gb300 import inputs as I
    if workload == "hub":
        return I.hub_stream(seed=seed)
    if workload == "rmat":
        return I.rmat_stream(seed=seed)
    if workload == "uniform":
        return I.uniform_stream(seed=seed)
    if workload == "grid":
        return I.grid_stream(seed=seed)
    raise ValueError(workload)


WORKLOAD_TEXT = {
    "rmat": "R-MAT n=2^24 (a,b,c,d=.57,.19,.19,.05, permuted ids), 2^27 edges in 128 "
            "Bulk-Updates of 2^20, each followed by a Bulk-Query of 2^20 uniform pairs",
    "uniform": "uniform n=2^16, 2^20 edges in 16 Bulk-Updates of 2^16, each followed by "
               "a Bulk-Query of 2^16 uniform pairs",
    "grid": "shuffled 8192x8192 4-neighbour grid (n=2^26, 134,201,344 edges) in 32 "
            "Bulk-Updates of 2^22, each followed by a Bulk-Query of 2^22 uniform pairs",
    "hub": "star at scale: n=2^24, 2^27 edges (hub n-1, uniform vertex) in 128 Bulk-Updates of "
           "2^20, each followed by a Bulk-Query of 2^20 uniform pairs",
    "segmented": "1024 graphs, n log-uniform in [2^8,2^16), m=4n uniform edges, minibatches "
                 "log-uniform in [2^6,2^14), each followed by a Bulk-Query of the same size",
    "serving": "request loop on one R-MAT n=2^26 stream (2^30 edges): Poisson arrivals, "
               "3:1 updates (log-uniform [2^8,2^20] edges) to queries (log-uniform [2^8,2^18] pairs)",
}


# ------------------------------------------------------------ distributed

def dist_env() -> tuple[int, int, int]:
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def dist_init(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend)
    return dist


def dist_barrier(dist) -> None:
    if dist is not None:
        dist.barrier()


def dist_max(dist, x: float, device=None) -> float:
    """Max of a host float over ranks (the timing reduction; no data path)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_sum(dist, x: float, device=None) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------- clocks

CLOCK_FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
                "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
                "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    def __init__(self, device_index: int, period_ms: int = 50):
        self.cmd = ["nvidia-smi", f"--id={device_index}", "--query-gpu=" + ",".join(CLOCK_FIELDS),
                    "--format=csv,noheader,nounits", f"-lms={period_ms}"]
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < len(CLOCK_FIELDS):
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------- peaks

def hbm_peak() -> tuple[float, str]:
    p = ROOT / "MEASURED_PEAKS.json"
    try:
        return float(json.loads(p.read_text())["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(kernel: str, workload: str):
    """(DRAM bytes per launch, what was captured) of `kernel` from the committed
    ncu summary, if it was taken on the current kernel source with the tuned
    options this run uses (no --opt overrides); else (None, None)."""
    if OPTION_OVERRIDES:
        return None, None
    p = ROOT / "profiles" / "ncu_traffic.json"
    try:
        d = json.loads(p.read_text())
        ent = d[workload][kernel]
        import hashlib
        csrc = ROOT / "paper_1602_05232_gb300" / "csrc"
        files = [csrc / "cc_device.cuh", csrc / "cc_kernels.cu", csrc / "cc_internal.cuh"]
        h = hashlib.sha256(b"".join(f.read_bytes() for f in files)).hexdigest()[:16]
        if ent.get("source_hash") != h:
            return None, None
        return ent["bytes_per_launch"], ent.get("kernel")
    except Exception:
        return None, None


# ------------------------------------------------------ batched form (segmented)

def run_segmented(args, rank: int, world: int, local_rank: int, dist) -> dict:
    """Many graphs: a STEP is the whole workload (every graph's minibatch
    stream) from an empty forest, as ONE cc_submit (persistent kernel,
    replayed CUDA graph), against the plain form: the same minibatches as one
    launch each on a plain handle with global ids."""
    import torch
    from paper_1602_05232_gb300 import cc, inputs as I

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = I.segmented_workload(seed=rank)
    off = np.concatenate([[0], np.cumsum(w.n)]).astype(np.int64)
    m_all = int(w.total_edges)
    h_e = np.empty((m_all, 2), dtype=np.int32)
    h_q = np.empty((m_all, 2), dtype=np.int32)
    eoff = np.concatenate([[0], np.cumsum([w.m(g) for g in range(w.G)])]).astype(np.int64)
    for g in range(w.G):
        h_e[eoff[g]:eoff[g + 1]] = w.edges(g)
        h_q[eoff[g]:eoff[g + 1]] = w.queries(g)
    d_e = torch.from_numpy(h_e).to(dev)
    d_q = torch.from_numpy(h_q).to(dev)
    shift = torch.from_numpy(np.repeat(off[:-1], [w.m(g) for g in range(w.G)]).astype(np.int32)).to(dev)
    d_eg = d_e + shift[:, None]          # global ids for the plain form
    d_qg = d_q + shift[:, None]
    out = torch.empty(m_all, dtype=torch.uint8, device=dev)
    seq = []
    for g in range(w.G):
        for kind, o, k in w.ops(g):
            seq.append((g, kind, int(eoff[g]) + o, k))
    ops = np.zeros(len(seq), dtype=cc.OP_DTYPE)
    for i, (g, kind, o, k) in enumerate(seq):
        ops[i] = (g, kind, (d_e if kind == 0 else d_q).data_ptr() + 8 * o, k,
                  out.data_ptr() + o if kind == 1 else 0)
    stream = torch.cuda.Stream(device=dev)
    opts = launch_options("segmented")
    with torch.cuda.stream(stream):
        f = cc.Forest.segmented(w.n, stream=stream, **opts)
        for _ in range(args.warmup):
            f.reset()
            f.submit(ops)
        stream.synchronize()
        f.set_option("profile", 1)
        f.kernel_stats(timing=True)
        l0 = f.kernel_stats()
        dist_barrier(dist)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clk:
            a.record(stream)
            for _ in range(args.steps):
                f.reset()
                f.submit(ops)
            b.record(stream)
            stream.synchronize()
        dist_barrier(dist)
        ks = f.kernel_stats(timing=True)
        l1 = f.kernel_stats()
        f.sync()
        f.close()
        ms = dist_max(dist, a.elapsed_time(b), dev)
        # plain form: one launch per minibatch, same edges with global ids
        fp = cc.Forest(int(off[-1]), stream=stream, **launch_options("uniform"))
        plain_steps = max(1, min(args.steps, 2))

        def plain_pass():
            fp.reset()
            for g, kind, o, k in seq:
                if kind == 0:
                    fp.bulk_update(d_eg[o:o + k])
                else:
                    fp.bulk_query(d_qg[o:o + k], out=out[o:o + k])
        plain_pass()
        stream.synchronize()
        a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a2.record(stream)
        for _ in range(plain_steps):
            plain_pass()
        b2.record(stream)
        stream.synchronize()
        pl = fp.kernel_stats()
        fp.sync()
        fp.close()
    ms_plain = a2.elapsed_time(b2) / plain_steps
    edges_all = dist_sum(dist, float(m_all * args.steps), dev)
    value = edges_all / (ms / 1e3)
    seg_ms = ks["segmented"][1] / max(1, l1["segmented"] - l0["segmented"])
    return {
        "metric": METRIC, "value": round(value, 1), "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "form": "batched",
        "config": {"workload": WORKLOAD_TEXT["segmented"], "graphs": w.G,
                   "vertices": int(off[-1]), "edges": m_all, "queries": m_all,
                   "ops_per_step": len(ops), "options": opts},
        "queries_per_s": round(edges_all / (ms / 1e3), 1),
        "kernel_ms_per_submit": round(seg_ms, 4),
        "gpu_launches": sum(l1[k] - l0[k] for k in l1),
        "plain_form": {"edges_per_s": round(m_all / (ms_plain / 1e3), 1),
                       "ms_per_pass": round(ms_plain, 3),
                       "launches_per_pass": len(seq), "what": "one cc_bulk_update / "
                       "cc_bulk_query launch per minibatch on a plain handle, global ids"},
        "speedup_vs_plain": round(ms_plain / (ms / args.steps), 2),
        "clocks": clk.summary(),
    }


# ------------------------------------------------------------ serving form

class ServingTrace:
    """The served workload: one R-MAT stream of 2^(scale+4) edges (scale 26:
    n = 2^26, 2^30 edges) in pinned host memory, and the request trace over
    it (Poisson arrivals; updates of log-uniform [2^8, 2^20] edges taken from
    the stream in order, queries of log-uniform [2^8, 2^18] uniform pairs, at
    3:1). `views` holds each request's host tensors; `many` the same requests
    as the arrays cc_server_enqueue_many takes."""

    NOMINAL_HZ = 1000.0

    def __init__(self, scale: int = 26, seed: int = 0):
        import torch
        from paper_1602_05232_gb300 import inputs as I
        self.scale = scale
        self.m = 1 << (scale + 4)
        self.stream = I.rmat_stream(scale=scale, m=self.m, batch=self.m, q=1, seed=seed)
        self.n = self.stream.n
        self.h_edges = torch.empty((self.m, 2), dtype=torch.int32, pin_memory=True)
        self.stream.all_edges(out=self.h_edges.numpy())
        self.reqs = I.request_trace(self.m, rate_hz=self.NOMINAL_HZ, seed=seed)
        self.qtot = sum(r.size for r in self.reqs if r.kind == 1)
        self.h_pairs = torch.empty((self.qtot, 2), dtype=torch.int32, pin_memory=True)
        I.uniform_pairs(self.n, self.qtot, seed, I.TAG_QUERIES, 0, out=self.h_pairs.numpy())
        self.h_out = torch.zeros(self.qtot, dtype=torch.uint8, pin_memory=True)
        self.views = []
        for r in self.reqs:
            if r.kind == 0:
                self.views.append((0, self.h_edges[r.offset:r.offset + r.size], None))
            else:
                self.views.append((1, self.h_pairs[r.offset:r.offset + r.size],
                                   self.h_out[r.offset:r.offset + r.size]))
        self.many = (np.array([kind for kind, _, _ in self.views], dtype=np.int32),
                     np.array([d.data_ptr() for _, d, _ in self.views], dtype=np.uint64),
                     np.array([d.shape[0] for _, d, _ in self.views], dtype=np.int64),
                     np.array([o.data_ptr() if o is not None else 0 for _, _, o in self.views],
                              dtype=np.uint64))


def host_memory_state(tensors=()) -> dict:
    """Host-side evidence for run-to-run changes of the served form: kernel
    memory-compaction and huge-page counters (/proc/vmstat), free and huge
    memory (/proc/meminfo), and how the pinned buffers in `tensors` are
    mapped (page size, huge pages) according to /proc/self/smaps."""
    out = {}
    want_vm = ("compact_stall", "compact_fail", "compact_success", "thp_fault_alloc",
               "thp_fault_fallback", "pgmajfault", "numa_hint_faults", "pgmigrate_success")
    try:
        for line in open("/proc/vmstat"):
            k, v = line.split()
            if k in want_vm:
                out[k] = int(v)
    except OSError:
        pass
    want_mi = ("MemFree", "MemAvailable", "AnonHugePages", "HugePages_Total", "HugePages_Free",
               "Hugepagesize", "Mlocked")
    try:
        for line in open("/proc/meminfo"):
            k, _, v = line.partition(":")
            if k in want_mi:
                out[k] = v.strip()
    except OSError:
        pass
    if tensors:
        spans = [(t.data_ptr(), t.data_ptr() + t.numel() * t.element_size()) for t in tensors]
        maps = []
        try:
            cur = None
            for line in open("/proc/self/smaps"):
                head = line.split()
                if "-" in head[0] and len(head) >= 5 and ":" not in head[0]:
                    lo, hi = (int(x, 16) for x in head[0].split("-"))
                    cur = {"lo": lo, "hi": hi} if any(a < hi and lo < b for a, b in spans) else None
                    if cur is not None:
                        maps.append(cur)
                elif cur is not None and head[0] in ("KernelPageSize:", "AnonHugePages:", "Rss:",
                                                     "Locked:"):
                    cur[head[0][:-1]] = " ".join(head[1:])
        except OSError:
            pass
        out["pinned_mappings"] = len(maps)
        out["pinned_GiB"] = round(sum(m["hi"] - m["lo"] for m in maps) / 2**30, 2)
        out["pinned_page_sizes"] = sorted({m.get("KernelPageSize", "?") for m in maps})
        out["pinned_anon_huge_kB"] = sum(int(m.get("AnonHugePages", "0 kB").split()[0]) for m in maps)
    return out


def h2d_rate(h, nbytes: int = 1 << 30, chunk: int = 8 << 20) -> float:
    """GB/s of host->device copies of the first `nbytes` of pinned tensor h."""
    import torch
    src = h.view(torch.uint8).view(-1)[:nbytes]
    dst = torch.empty(src.numel(), dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(st):
        for o in range(0, src.numel(), chunk):
            dst[o:o + chunk].copy_(src[o:o + chunk], non_blocking=True)
    st.synchronize()
    dt = time.perf_counter() - t0
    del dst
    return round(src.numel() / dt / 1e9, 1)


def run_serving(args, rank: int, world: int, local_rank: int, dist) -> dict:
    """Served form: the whole request trace through cc_server (continuous
    batching). Saturation: every request enqueued at once, edges/s from first
    enqueue to drain. Then the trace replayed at 0.5 / 0.8 / 0.95 of that
    capacity with Poisson arrivals for p50/p99 latency from arrival to
    completion. Plain form: the same requests one at a time (copy in, one
    launch, copy out, wait)."""
    import torch
    from paper_1602_05232_gb300 import cc

    torch.cuda.set_device(local_rank)
    scale = args.serve_scale
    tr = ServingTrace(scale, seed=rank)
    s, m, reqs, views, many = tr.stream, tr.m, tr.reqs, tr.views, tr.many
    qtot = tr.qtot
    nominal = tr.NOMINAL_HZ
    opts = launch_options("serving")
    mem_before = host_memory_state((tr.h_edges, tr.h_pairs, tr.h_out))
    h2d_before = h2d_rate(tr.h_edges)
    # Warm-up of the data path: on this host, pinned buffers that were just
    # allocated and filled copy to the device slowly until they have been
    # copied a few times; a server that runs for long copies from warm
    # buffers. Three full copies of the trace, untimed.
    h2d_warm = [h2d_rate(tr.h_edges, nbytes=tr.h_edges.numel() * 4) for _ in range(3)]

    def serve(rate: float | None, at_once: bool = False):
        f = cc.Forest(s.n, **opts)
        with cc.Server(f) as srv:
            gc.disable()                         # no collector pause inside the enqueue loop
            t0 = time.perf_counter()
            if at_once:
                srv.enqueue_many(*many)
            else:
                for r, (kind, d, o) in zip(reqs, views):
                    if rate is not None:
                        due = r.t * nominal / rate
                        while time.perf_counter() - t0 < due:
                            pass
                    srv.enqueue(kind, d, o)
            srv.drain()
            dt = time.perf_counter() - t0
            gc.enable()
            lat = srv.latencies()
            st = srv.stats()
        labels = f.labels()
        f.close()
        return dt, lat, st, labels

    serve(None)                                  # warm-up
    dist_barrier(dist)
    with ClockSampler(local_rank) as clk:
        # saturation: every request is there at the start, handed over in one
        # call; three runs in a row, to show whether the rate holds
        sat_runs = [serve(None, at_once=True) for _ in range(3)]
        dt_sat, lat_sat, st_sat, lab_served = sorted(sat_runs, key=lambda r: r[0])[1]   # the median run
        # the same with one enqueue call per request (the caller's loop is in the time)
        dt_sat1, _, st_sat1, _ = serve(None)
    dist_barrier(dist)
    mem_after = host_memory_state((tr.h_edges, tr.h_pairs, tr.h_out))
    h2d_after = h2d_rate(tr.h_edges)
    cap_edges = m / dt_sat
    cap_rps = len(reqs) / dt_sat
    loads = {}
    for load_frac in (0.5, 0.8, 0.95):
        rate = cap_rps * load_frac
        dt, lat, st, _ = serve(rate)
        loads[str(load_frac)] = {"offered_req_per_s": round(rate, 1),
                                 "p50_ms": round(1e3 * float(np.percentile(lat, 50)), 3),
                                 "p99_ms": round(1e3 * float(np.percentile(lat, 99)), 3),
                                 "edges_per_s": round(m / dt, 1), "groups": st["groups"]}
    # plain form: one request at a time through the plain API
    f = cc.Forest(s.n, **opts)
    dev = torch.device("cuda", local_rank)
    kmax = max(r.size for r in reqs)
    d_in = torch.empty((kmax, 2), dtype=torch.int32, device=dev)
    d_o = torch.empty(kmax, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for kind, d, o in views:
        k = d.shape[0]
        d_in[:k].copy_(d, non_blocking=True)
        if kind == 0:
            f.bulk_update(d_in[:k])
        else:
            f.bulk_query(d_in[:k], out=d_o[:k])
            o.copy_(d_o[:k], non_blocking=True)
        torch.cuda.current_stream().synchronize()
    dt_plain = time.perf_counter() - t0
    same = bool(torch.equal(f.labels(), lab_served))
    f.close()
    value = dist_sum(dist, cap_edges, dev)
    return {
        "metric": METRIC, "value": round(value, 1), "unit": "edges/s", "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": round(1e3 * dt_sat, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "form": "served",
        "config": {"workload": WORKLOAD_TEXT["serving"] if scale == 26 else
                   f"serving trace on R-MAT scale {scale}", "n": s.n, "edges": m,
                   "requests": len(reqs), "query_pairs": qtot, "options": opts},
        "saturation": {"edges_per_s": round(cap_edges, 1), "req_per_s": round(cap_rps, 1),
                       "runs_edges_per_s": [round(m / r[0], 1) for r in sat_runs],
                       "runs_what": "three saturation runs in a row in this process (new forest and "
                                    "server each); the value is the median run",
                       "p50_ms": round(1e3 * float(np.percentile(lat_sat, 50)), 3),
                       "p99_ms": round(1e3 * float(np.percentile(lat_sat, 99)), 3),
                       "groups": st_sat["groups"],
                       "enqueue": "all requests in one cc_server_enqueue_many call",
                       "per_call_enqueue": {"edges_per_s": round(m / dt_sat1, 1),
                                            "groups": st_sat1["groups"],
                                            "what": "one cc_server_enqueue per request from a Python loop"}},
        "latency_at_load": loads,
        "plain_form": {"edges_per_s": round(m / dt_plain, 1), "seconds": round(dt_plain, 3),
                       "what": "each request alone: copy in, one launch, copy out, synchronise"},
        "served_labels_equal_plain": same,
        "host_memory": {"before": mem_before, "after": mem_after},
        "h2d_GBps_of_trace": {"before": h2d_before, "warm_up_copies": h2d_warm,
                              "after_saturation_runs": h2d_after,
                              "what": "pinned host->device copy rate of the trace's edge buffer in 8 MiB "
                                      "copies: its first GiB before anything else, three untimed copies of "
                                      "the whole buffer (the data path's warm-up), and its first GiB after "
                                      "the saturation runs; the served form is bound by these copies"},
        "clocks": clk.summary(),
    }


# ------------------------------------------------- paper-scale streams (Table 3)

# Bulk-Update throughput on 20 cores, M edges/s at b = 500K / 1M / 5M / 10M
# (Table 3), for the graphs these streams stand in for.
PAPER_T20C = {"random": [36.87, 46.02, 60.66, 63.90], "rmat5": [26.08, 34.19, 49.92, 50.37],
              "3dgrid": [27.97, 34.97, 44.27, 45.24], "rmat16": [54.94, 78.10, 143.63, 167.68]}
PAPER_BATCHES = [500_000, 1_000_000, 5_000_000, 10_000_000]


def paper_compress_every(tuned_every: int, batch: int) -> int:
    """The compression interval, in Bulk-Updates, at `batch` edges per update
    when `tuned_every` was tuned at the largest paper batch: about as many
    edges between two compressions. 0 (never) stays 0."""
    if tuned_every <= 0:
        return 0
    return max(1, round(tuned_every * PAPER_BATCHES[-1] / batch))


def run_paper(args, rank: int, world: int, local_rank: int, dist) -> dict:
    """Bulk-Update throughput (total edges / total update time, as in Table 3)
    on a paper-size stream at the paper's four batch sizes, and the number of
    connected components at every tenth of the stream (the Figure 2 curve).
    The options are tuned at the largest batch; at the smaller ones the
    compression interval (counted in Bulk-Updates) is scaled so that about as
    many edges pass between two compressions."""
    import torch
    from paper_1602_05232_gb300 import cc, inputs as I

    name = args.workload.split("-", 1)[1]
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    s0 = I.paper_stream(name, batch=PAPER_BATCHES[-1], seed=rank)
    d_edges = torch.from_numpy(s0.all_edges()).to(dev)
    opts = launch_options(args.workload)
    stream = torch.cuda.Stream(device=dev)
    per_batch = {}
    with torch.cuda.stream(stream):
        f = cc.Forest(s0.n, stream=stream, **opts)
        every = {}
        for b in PAPER_BATCHES:
            cuts = list(range(0, s0.m, b)) + [s0.m]
            every[b] = paper_compress_every(int(opts.get("compress_every", 1)), b)
            f.set_option("compress_every", every[b])

            def one_pass():
                f.reset()
                for i in range(len(cuts) - 1):
                    f.bulk_update(d_edges[cuts[i]:cuts[i + 1]])
            one_pass()
            stream.synchronize()
            times = []
            for _ in range(max(1, min(args.steps, 3))):
                a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                f.reset()
                stream.synchronize()
                a.record(stream)
                for i in range(len(cuts) - 1):
                    f.bulk_update(d_edges[cuts[i]:cuts[i + 1]])
                e.record(stream)
                stream.synchronize()
                times.append(a.elapsed_time(e))
            per_batch[b] = s0.m / (statistics.median(times) / 1e3)
        # component count at every tenth of the stream, b = 10M
        f.set_option("compress_every", every[PAPER_BATCHES[-1]])
        f.reset()
        curve, b = [], PAPER_BATCHES[-1]
        cuts = list(range(0, s0.m, b)) + [s0.m]
        marks = {int(round(s0.m * t / 10)) for t in range(1, 11)}
        done = 0
        for i in range(len(cuts) - 1):
            f.bulk_update(d_edges[cuts[i]:cuts[i + 1]])
            done = cuts[i + 1]
            if any(cuts[i] < mk <= done for mk in marks):
                curve.append([round(100.0 * done / s0.m, 1), f.components()])
        f.sync()
        f.close()
    t20 = PAPER_T20C[name]
    return {
        "metric": "Bulk-Update edges/s (Table 3 shape: total edges / total update time)",
        "value": round(per_batch[PAPER_BATCHES[-1]], 1), "unit": "edges/s", "n_gpus": world,
        "higher_is_better": True, "dtype": "int32", "data": "synthetic",
        "config": {"workload": s0.name, "n": s0.n, "m": s0.m, "options": opts,
                   "stands_in_for": name},
        "bulk_update_edges_per_s": {str(b): round(v, 1) for b, v in per_batch.items()},
        "compress_every_per_batch": {str(b): v for b, v in every.items()},
        "paper_T20c_edges_per_s": {str(b): t * 1e6 for b, t in zip(PAPER_BATCHES, t20)},
        "ratio_to_paper_20c": {str(b): round(per_batch[b] / (t * 1e6), 1)
                               for b, t in zip(PAPER_BATCHES, t20)},
        "components_curve": curve,
    }


# --------------------------------------------------------------- GPU arm

def run_gpu(args, rank: int, world: int, local_rank: int, dist, workload: str | None = None,
            steps: int | None = None, warmup: int | None = None, e2e: bool = True,
            cpu: bool = True) -> dict | None:
    """Plain form on one minibatch stream. A STEP is one whole pass of the
    stream from the empty graph: a reset of the forest to n singletons, then
    every minibatch's Bulk-Update (with the compression policy) and
    Bulk-Query in stream order. Throughput is total edges over total time, as
    in Section 5.3; latency is per minibatch (update + query) and per pass."""
    import torch
    from paper_1602_05232_gb300 import cc

    workload = workload or args.workload
    K = args.steps if steps is None else steps
    W = args.warmup if warmup is None else warmup
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    s = make_stream(workload, seed=rank)
    B = s.batches
    # whole stream in pinned host memory, then resident in HBM
    h_edges = torch.empty((s.m, 2), dtype=torch.int32, pin_memory=True)
    h_pairs = torch.empty((s.q, 2), dtype=torch.int32, pin_memory=True)
    s.all_edges(out=h_edges.numpy())
    s.all_queries(out=h_pairs.numpy())
    eoff, qoff = s.edge_offsets(), s.query_offsets()
    d_edges = h_edges.to(dev)
    d_pairs = h_pairs.to(dev)
    d_out = torch.empty(s.q, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    opts = launch_options(workload)
    # every minibatch's views, made once (no slicing inside the timed regions)
    views = [(d_edges[eoff[b]:eoff[b + 1]], d_pairs[qoff[b]:qoff[b + 1]], d_out[qoff[b]:qoff[b + 1]])
             for b in range(B)]

    with torch.cuda.stream(stream):
        f = cc.Forest(s.n, stream=stream, **opts)

    def one_pass(ev: list | None = None) -> None:
        f.reset()
        for b, (e, q, o) in enumerate(views):
            f.bulk_update(e)
            f.bulk_query(q, out=o)
            if ev is not None:
                ev[b].record(stream)

    for _ in range(W):
        one_pass()
    stream.synchronize()

    def region(batch_events: bool, profile: bool):
        """K passes, timed on the forest's stream."""
        f.set_option("profile", 1 if profile else 0)
        stream.synchronize()
        f.kernel_stats(timing=profile)    # clears the timing sums
        l0 = f.kernel_stats()
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        bev = [[torch.cuda.Event(enable_timing=True) for _ in range(B)] for _ in range(K)] \
            if batch_events else None
        pev = [torch.cuda.Event(enable_timing=True) for _ in range(K)] if batch_events else None
        dist_barrier(dist)
        torch.cuda.synchronize(dev)
        start.record(stream)
        for i in range(K):
            one_pass(bev[i] if bev else None)
            if pev:
                pev[i].record(stream)
        stop.record(stream)
        torch.cuda.synchronize(dev)
        dist_barrier(dist)
        ks = f.kernel_stats(timing=profile) if profile else None
        l1 = f.kernel_stats()
        f.set_option("profile", 0)
        batch_ms = pass_ms = None
        if batch_events:
            batch_ms, pass_ms, prev = [], [], start
            for i in range(K):
                # a pass's first minibatch also carries that pass's reset
                for b in range(B):
                    batch_ms.append(prev.elapsed_time(bev[i][b]))
                    prev = bev[i][b]
                pass_ms.append((start if i == 0 else pev[i - 1]).elapsed_time(pev[i]))
                prev = pev[i]
        return start.elapsed_time(stop), batch_ms, pass_ms, ks, l0, l1

    # (A) the value: nothing but the K passes between two events
    with ClockSampler(local_rank) as clk:
        total_ms, _, _, _, la0, la1 = region(False, False)
        # (B) an event after every minibatch, for the latency distributions
        _, batch_ms, pass_ms, _, _, _ = region(True, False)
        # (C) libcc's per-kernel events, for the roofline
        _, _, _, kstats, launches0, launches1 = region(False, True)
    gpu_launches = sum(la1[k] - la0[k] for k in la1)
    depth_max, depth_mean = f.depth()
    f.sync()
    expect = d_out.cpu() if e2e else None       # the last pass's answers, for the e2e check
    gather = gather_ceiling(f, views)

    total_ms_max = dist_max(dist, total_ms, dev)
    edges_all = dist_sum(dist, float(K * s.m), dev)
    pairs_all = dist_sum(dist, float(K * s.q), dev)
    value = edges_all / (total_ms_max / 1e3)

    # per-kernel breakdown and the roofline of the dominant kernel
    peak, peak_kind = hbm_peak()
    units = {"update": K * s.m, "query": K * s.q,
             "compress_all": s.n * (launches1["compress_all"] - launches0["compress_all"]),
             "compress_touched": K * s.m,
             "reset": s.n * (launches1["reset"] - launches0["reset"]),
             "order": K * s.m}
    bpu = dict(BYTES_PER_UNIT)
    if opts.get("big_filter", 0) and opts.get("compress_every", 1) and not opts.get("compress_scope", 0):
        bpu["compress_all"] += BITMAP_BYTES
    kernels = {}
    for k, (_, ms) in kstats.items():
        cnt = launches1[k] - launches0[k]
        if cnt and ms > 0:
            gb = bpu.get(k, 0.0) * units.get(k, 0) / 1e9
            kernels[k] = {"launches": cnt, "ms_total": round(ms, 4), "us_avg": round(1e3 * ms / cnt, 3),
                          "share": None, "GBps_algorithmic": round(gb / (ms / 1e3), 1) if gb else None}
    tot_k = sum(v["ms_total"] for v in kernels.values()) or 1.0
    for v in kernels.values():
        v["share"] = round(v["ms_total"] / tot_k, 4)
    dom = max((k for k in kernels if k in units), key=lambda k: kernels[k]["ms_total"])
    dk = kernels[dom]
    per_launch_units = units[dom] / dk["launches"]
    achieved = bpu[dom] * per_launch_units / (dk["us_avg"] * 1e-6) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "peak_source": f"of {peak_kind}",
                "bytes_per_unit": bpu[dom],
                "units_per_launch": per_launch_units,
                "traffic": None,
                "timing_basis": "per-kernel events, PDL serialised",
                "in_step_share": round(dk["ms_total"] / total_ms, 4),
                "in_step_share_what": "the dominant kernel's summed event time over the same K "
                                      "passes / the pass time of the value's region"}
    if opts.get("big_filter", 0) and dom in ("update", "query"):
        roofline["filter"] = ("largest-component bitmap on: an edge or pair with both endpoints marked "
                              "reads two L2-resident bitmap sectors in place of two parent sectors "
                              "(the same sector-model bytes)")
    roofline["traffic"], traffic_kernel = ncu_traffic(dom, workload)
    if roofline["traffic"]:
        roofline["traffic_kernel"] = traffic_kernel
        # the measured DRAM bytes of the same kernel over the same launch time
        roofline["traffic_GBps"] = round(roofline["traffic"] / (dk["us_avg"] * 1e-6) / 1e9, 1)
        roofline["traffic_frac"] = round(roofline["traffic_GBps"] / peak, 4)
    if gather:
        gather["frac_of_peak"] = round(gather["GBps"] / peak, 4)
        gather["dominant_kernel_frac_of_this"] = round(achieved / gather["GBps"], 4)
        roofline["gather_ceiling"] = gather

    upd_ms = sum(kstats[k][1] for k in ("update", "compress_all", "compress_touched"))
    qry_ms = kstats["query"][1]
    e2e_out = run_e2e(args, s, h_edges, h_pairs, eoff, qoff, dev, dist, workload, K, W, expect) if e2e else None

    f.close()
    del views, d_edges, d_pairs, d_out
    torch.cuda.empty_cache()

    cpu_out = None
    if cpu and rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_out = cpu_baseline(s, h_edges.numpy(), h_pairs.numpy(), eoff, qoff, args.cpu_seconds)

    def pct(xs, q):
        xs = sorted(xs)
        return round(xs[min(len(xs) - 1, int(q * len(xs)))], 4)

    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "edges/s", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": round(total_ms_max / K, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded R-MAT / uniform / grid generators; no dataset)",
        "config": {"workload": WORKLOAD_TEXT.get(workload, s.name), "n": s.n, "edges_per_pass": s.m,
                   "queries_per_pass": s.q, "minibatches_per_pass": B,
                   "batch": int(eoff[1]), "query_batch": int(qoff[1]),
                   "step": "one whole pass of the stream from the empty graph (reset, then every "
                           "minibatch's Bulk-Update and Bulk-Query in order)",
                   "form": "plain (one launch per bulk operation)", "options": opts,
                   "l2": f"inputs larger than L2: {8 * s.m / 2**30:.2f} GiB of edges and "
                         f"{8 * s.q / 2**30:.2f} GiB of pairs, each read once per pass",
                   "parallelism": f"replicas x{world} (independent streams, no collective)"},
        "queries_per_s": round(pairs_all / (total_ms_max / 1e3), 1),
        "update_edges_per_s_kernels": round(K * s.m / (upd_ms / 1e3), 1) if upd_ms else None,
        "query_per_s_kernel": round(K * s.q / (qry_ms / 1e3), 1) if qry_ms else None,
        "latency_ms": {"batch_p50": pct(batch_ms, 0.5), "batch_p99": pct(batch_ms, 0.99),
                       "pass_p50": pct(pass_ms, 0.5), "pass_p99": pct(pass_ms, 0.99),
                       "what": "device time of one minibatch (Bulk-Update + its compression + "
                               "Bulk-Query; the first of a pass also its reset) and of one pass, "
                               "from a second run of the K passes with an event after each minibatch"},
        "timing": "value from K passes between two events with nothing else recorded; latency "
                  "and the per-kernel times (roofline) from two more runs of the same K passes",
        "forest_depth": {"max": depth_max, "mean": round(depth_mean, 4),
                         "what": "distance from a vertex to its root after the timed passes"},
        "roofline": roofline, "kernels": kernels, "gpu_launches": gpu_launches,
        "clocks": clk.summary(), "e2e": e2e_out, "cpu_baseline": cpu_out,
    }
    return out


def gather_ceiling(f, views, reps: int = 20) -> dict | None:
    """Context for the roofline: the query launch shape doing nothing but its
    gathers. After a full compression every vertex points at its root, so a
    query is decided by parent[u] == parent[v]: one streamed pair and two
    random 4-byte reads, the minimum any update or query of this layout pays.
    Timed with libcc's per-kernel events, like the kernels of the timed
    regions, and run after them (it changes the forest)."""
    if f.kernel_stats().get("query") is None:
        return None
    big = f.get_option("big_filter")
    f.set_option("big_filter", 0)               # every pair reads the forest
    f.compress()                                # flat forest: parent equality decides
    bulk_find = f.get_option("bulk_find")
    f.set_option("bulk_find", 0)                # the plain query launch shape, whatever the options
    f.set_option("profile", 1)
    f.sync()
    f.kernel_stats(timing=True)                 # clears the timing sums
    n0 = f.kernel_stats()["query"]
    pairs = 0
    for r in range(reps):
        _, q, o = views[r % len(views)]
        f.bulk_query(q, out=o)
        pairs += q.shape[0]
    f.sync()
    launches, ms = f.kernel_stats(timing=True)["query"]
    f.set_option("profile", 0)
    f.set_option("bulk_find", bulk_find)
    f.set_option("big_filter", big)
    launches -= n0
    if launches <= 0 or ms <= 0:
        return None
    us = 1e3 * ms / launches
    gbps = BYTES_PER_UNIT["query"] * (pairs / launches) / (us * 1e-6) / 1e9
    return {"kernel": "query on a flattened forest (parent equality only)", "us_per_launch": round(us, 3),
            "GBps": round(gbps, 1), "launches": launches,
            "what": "the same sector-model bytes per pair (73 B) moved by pure random gathers: the "
                    "practical ceiling of this access pattern on this GPU, beside the copy-bandwidth peak"}


def run_e2e(args, s, h_edges, h_pairs, eoff, qoff, dev, dist, workload: str, K: int, W: int,
            expect=None) -> dict:
    """Same metric through the public API from HOST buffers (pinned), with the
    host<->device traffic of every pass inside the timed region: each pass
    resets the forest, and its edges and pairs go to the device and its
    answers come back. Two ways:
      zero_copy  the bulk calls get the host pointers themselves; the kernels
                 read the edges and pairs and write the answers over the host
                 link (NVLink-C2C on Grace-Blackwell);
      pipelined  the inputs are copied to device buffers on a copy stream,
                 G consecutive minibatches per copy (two buffers, the next
                 group's copy overlapping this group's kernels, also across
                 the boundary between two passes), and the answers copied
                 back, G = 1, 2, 4.
    The better of the two is the e2e value; both are reported. Each way's
    answers of its last pass are compared with `expect` (the device-resident
    run's), and a difference is an error."""
    import torch
    from paper_1602_05232_gb300 import cc

    B = s.batches
    opts = launch_options(workload)
    h_o = torch.empty(s.q, dtype=torch.uint8, pin_memory=True)
    stream = torch.cuda.Stream(device=dev)
    results = {}
    h2d = 8 * s.m + 8 * s.q                       # per pass (= per step)
    d2h = s.q

    def timed(run_pass):
        with torch.cuda.stream(stream):
            f = cc.Forest(s.n, stream=stream, **opts)
            for _ in range(max(1, min(W, 2))):
                run_pass(f)
            if getattr(run_pass, "finish", None):
                run_pass.finish()
            stream.synchronize()
            dist_barrier(dist)
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(K):
                run_pass(f)
            finish = getattr(run_pass, "finish", None)
            if finish:
                finish()                          # the last answers are on the host
            b_.record(stream)
            stream.synchronize()
            dist_barrier(dist)
            f.sync()
            f.close()
        return dist_max(dist, a.elapsed_time(b_), dev)

    def check(name: str) -> None:
        if expect is not None and not torch.equal(h_o, expect):
            bad = int((h_o != expect).sum())
            raise RuntimeError(f"e2e {name}: {bad} answers differ from the device-resident run")
        h_o.zero_()

    zero_copy_ok = cc.device_can_read(h_edges) and cc.device_can_read(h_o)
    if zero_copy_ok:
        zviews = [(h_edges[eoff[b]:eoff[b + 1]], h_pairs[qoff[b]:qoff[b + 1]], h_o[qoff[b]:qoff[b + 1]])
                  for b in range(B)]

        def zc(f):
            f.reset()
            for e, q, o in zviews:
                f.bulk_update(e)
                f.bulk_query(q, out=o)
        results["zero_copy"] = timed(zc)
        check("zero_copy")

    copy_in = torch.cuda.Stream(device=dev)
    copy_out = torch.cuda.Stream(device=dev)

    def make_piped(G: int):
        """A pass in groups of G consecutive minibatches: one host->device copy
        of the group's edges and one of its pairs (contiguous ranges of the
        pinned stream), one device->host copy of its answers, two device
        buffers so that a group's copies overlap the previous group's kernels.
        Every minibatch is still one cc_bulk_update + one cc_bulk_query call.
        All tensor views are made before the timed region."""
        groups = [list(range(g, min(g + G, B))) for g in range(0, B, G)]
        ke = max(int(eoff[grp[-1] + 1] - eoff[grp[0]]) for grp in groups)
        kq = max(int(qoff[grp[-1] + 1] - qoff[grp[0]]) for grp in groups)
        d_e = [torch.empty((ke, 2), dtype=torch.int32, device=dev) for _ in range(2)]
        d_q = [torch.empty((kq, 2), dtype=torch.int32, device=dev) for _ in range(2)]
        d_o = [torch.empty(kq, dtype=torch.uint8, device=dev) for _ in range(2)]
        plan = []
        for gi, grp in enumerate(groups):
            j = gi % 2
            b0, b1 = grp[0], grp[-1] + 1
            ne, nq = int(eoff[b1] - eoff[b0]), int(qoff[b1] - qoff[b0])
            calls = []
            for b in grp:
                e_lo, e_hi = int(eoff[b] - eoff[b0]), int(eoff[b + 1] - eoff[b0])
                q_lo, q_hi = int(qoff[b] - qoff[b0]), int(qoff[b + 1] - qoff[b0])
                calls.append((d_e[j][e_lo:e_hi], d_q[j][q_lo:q_hi], d_o[j][q_lo:q_hi]))
            plan.append((j, h_edges[eoff[b0]:eoff[b1]], d_e[j][:ne], h_pairs[qoff[b0]:qoff[b1]], d_q[j][:nq],
                         h_o[qoff[b0]:qoff[b1]], d_o[j][:nq], calls))
        done_ev = [torch.cuda.Event(), torch.cuda.Event()]
        ready_ev = [torch.cuda.Event(), torch.cuda.Event()]
        out_ev = [torch.cuda.Event(), torch.cuda.Event()]
        started = [False]

        def piped(f):
            # Buffer j's events carry over from the previous pass: the first
            # copy of this pass waits only for that buffer's last kernels, so it
            # overlaps the previous pass's last group (its answers still come
            # back before the kernels that reuse the buffer).
            if not started[0]:
                for e in done_ev + out_ev:
                    e.record(stream)
                started[0] = True

            def issue_copy(gi):
                j, he, de, hq, dq = plan[gi][:5]
                copy_in.wait_event(done_ev[j])      # buffer j free (its kernels done)
                with torch.cuda.stream(copy_in):
                    de.copy_(he, non_blocking=True)
                    dq.copy_(hq, non_blocking=True)
                ready_ev[j].record(copy_in)

            f.reset()
            issue_copy(0)
            for gi, (j, he, de, hq, dq, ho, do, calls) in enumerate(plan):
                if gi + 1 < len(plan):
                    issue_copy(gi + 1)
                stream.wait_event(ready_ev[j])
                stream.wait_event(out_ev[j])        # the answers that used buffer j are out
                for ce, cq, co in calls:
                    f.bulk_update(ce)
                    f.bulk_query(cq, out=co)
                done_ev[j].record(stream)
                copy_out.wait_event(done_ev[j])
                with torch.cuda.stream(copy_out):
                    ho.copy_(do, non_blocking=True)
                out_ev[j].record(copy_out)

        def finish():
            stream.wait_event(out_ev[0])
            stream.wait_event(out_ev[1])

        piped.finish = finish
        return piped

    for G in (1, 2, 4):
        results[f"pipelined_g{G}"] = timed(make_piped(G))
        check(f"pipelined_g{G}")
    edges_all = dist_sum(dist, float(K * s.m), dev)
    best = min(results, key=results.get)
    return {"value": round(edges_all / (results[best] / 1e3), 1), "unit": "edges/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": K, "variant": best,
            "variants": {k: round(edges_all / (v / 1e3), 1) for k, v in results.items()},
            "what": "pinned host buffers through cc_bulk_update/cc_bulk_query, one whole pass per "
                    "step; zero_copy: the kernels read/write host memory directly; pipelined_gG: "
                    "copies on two copy streams overlapping the kernels (and the next pass's first "
                    "copy overlapping this pass's last kernels), G minibatches per copy (one update "
                    "and one query call per minibatch); every way's answers equal the device-resident "
                    "run's",
            "answers_checked": expect is not None}


# ------------------------------------------------------------ CPU oracle

def cpu_baseline(s, edges: np.ndarray, pairs: np.ndarray, eoff, qoff, seconds: float) -> dict:
    """The oracle (single-threaded sequential union-find) on the host: the
    stream's minibatches in order from the empty graph until `seconds` of
    oracle time have been spent."""
    import oracle
    uf = oracle.OracleUF(s.n)
    t_total, e_done, q_done, b = 0.0, 0, 0, 0
    while b < s.batches and t_total < seconds:
        e = edges[eoff[b]:eoff[b + 1]]
        q = pairs[qoff[b]:qoff[b + 1]]
        t0 = time.perf_counter()
        uf.bulk_update(e)
        uf.bulk_query(q)
        t_total += time.perf_counter() - t0
        e_done += len(e)
        q_done += len(q)
        b += 1
    ncpu = os.cpu_count()
    return {"value": round(e_done / t_total, 1), "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": f"first {b} of {s.batches} minibatches ({e_done} edges + {q_done} query "
                      f"pairs) from the empty graph, {t_total:.1f} s on one host core",
            "host_cores_available": ncpu, "host": host_info(),
            "note": f"the oracle (a sequential union-find) uses 1 of {ncpu} host cores"}


def host_info() -> dict:
    """CPU model (from /proc/cpuinfo) and the process's CPU affinity."""
    model = None
    try:
        keys = {}
        for line in open("/proc/cpuinfo"):
            k, _, v = line.partition(":")
            k, v = k.strip(), v.strip()
            if k in ("model name", "CPU implementer", "CPU part") and k not in keys:
                keys[k] = v
        model = keys.get("model name") or (
            f"implementer {keys.get('CPU implementer')} part {keys.get('CPU part')}" if keys else None)
    except OSError:
        pass
    try:
        aff = sorted(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        aff = []
    return {"cpu_model": model, "affinity_cpus": len(aff),
            "affinity": f"{aff[0]}-{aff[-1]}" if aff and aff == list(range(aff[0], aff[-1] + 1)) else aff}


def run_reference(args, rank: int, world: int) -> dict | None:
    """--impl reference: the CPU oracle, as it stands, on a bounded sample of
    every step. A step is one pass of the workload's stream from the empty
    graph, as in the GPU arm, over the first 1/frac of every minibatch's
    edges and pairs."""
    if rank != 0:
        return None
    import oracle
    s = make_stream(args.workload, seed=0)
    B = s.batches
    frac = args.ref_fraction
    eoff, qoff = s.edge_offsets(), s.query_offsets()
    sample = []
    for b in range(B):
        ke = max(1, int(eoff[b + 1] - eoff[b]) // frac)
        kq = max(1, int(qoff[b + 1] - qoff[b]) // frac)
        sample.append((s.edges_range(int(eoff[b]), int(eoff[b]) + ke), uniform_slice(s, b, kq)))
    edges_per_pass = sum(len(e) for e, _ in sample)
    pairs_per_pass = sum(len(q) for _, q in sample)

    def one_pass():
        uf = oracle.OracleUF(s.n)
        for e, q in sample:
            uf.bulk_update(e)
            uf.bulk_query(q)

    for _ in range(args.warmup):
        one_pass()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_pass()
    dt = time.perf_counter() - t0
    v = args.steps * edges_per_pass / dt
    return {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "edges/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * dt / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "queries_per_s": round(args.steps * pairs_per_pass / dt, 1),
            "config": {"workload": WORKLOAD_TEXT[args.workload],
                       "step": "one pass of the stream from the empty graph",
                       "sample": f"each pass applies the first 1/{frac} of every minibatch's edges "
                                 f"and queries the first 1/{frac} of its pairs ({edges_per_pass} "
                                 f"edges + {pairs_per_pass} pairs per pass)"},
            "cpu_baseline": {"value": round(v, 1), "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": f"1/{frac} of every minibatch, {args.steps} passes",
                             "host_cores_available": os.cpu_count(), "host": host_info()},
            "e2e": {"value": round(v, 1), "unit": "edges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def uniform_slice(s, b: int, kq: int) -> np.ndarray:
    from paper_1602_05232_gb300 import inputs as I
    return I.uniform_pairs(s.n, kq, s.seed, I.TAG_QUERIES, int(s.query_offsets()[b]))


HEADLINE = "grid"
FORMS = ("rmat", "uniform", "segmented", "serving")
DROP_IN_FORMS = ("metric", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "dtype", "data",
                 "e2e", "cpu_baseline", "warmup")


def form_summary(d: dict) -> dict:
    return {k: v for k, v in d.items() if k not in DROP_IN_FORMS}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20,
                    help="timed steps; a step of a plain workload is one whole pass of its stream")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", choices=sorted(LAUNCH_OPTIONS) + [
        "paper-random", "paper-rmat5", "paper-rmat16", "paper-3dgrid"], default=HEADLINE)
    ap.add_argument("--forms", default="all",
                    help="with the headline workload: the other forms to run and report in the same "
                         "line, a comma list of " + ",".join(FORMS) + ", or 'all' or 'none'")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-fraction", type=int, default=64)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--opt", action="append", default=[], metavar="KEY=VALUE",
                    help="override a libcc launch option (e.g. update_schedule=1)")
    ap.add_argument("--serve-scale", type=int, default=26,
                    help="R-MAT scale of the serving trace (2^(scale+4) edges)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    for kv in args.opt:
        k, v = kv.split("=", 1)
        OPTION_OVERRIDES[k] = int(v)
    forms = [] if args.forms == "none" else list(FORMS) if args.forms == "all" else \
        [x for x in args.forms.split(",") if x]
    for x in forms:
        if x not in FORMS:
            ap.error(f"--forms: unknown form {x}")
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        dist = dist_init(world, "nccl")
        if args.workload == "segmented":
            out = run_segmented(args, rank, world, local_rank, dist)
        elif args.workload == "serving":
            out = run_serving(args, rank, world, local_rank, dist)
        elif args.workload.startswith("paper-"):
            out = run_paper(args, rank, world, local_rank, dist)
        else:
            sub = {}
            # Under torchrun (N > 1) every rank is a replica of the headline
            # only: the other forms are single-GPU comparisons.
            with_forms = args.workload == HEADLINE and forms and world == 1
            # The served form goes first: its copies from pinned host memory
            # run fastest before the process has pinned and copied other
            # streams (the plain forms time device-resident inputs).
            if with_forms and "serving" in forms:
                sub["serving"] = form_summary(run_serving(args, rank, world, local_rank, dist))
            out = run_gpu(args, rank, world, local_rank, dist, e2e=not args.no_e2e)
            if with_forms:
                for x in forms:
                    if x in ("rmat", "uniform"):
                        d = run_gpu(args, rank, world, local_rank, dist, workload=x, e2e=False, cpu=False)
                    elif x == "segmented":
                        d = run_segmented(args, rank, world, local_rank, dist)
                    else:
                        continue
                    if d is not None:
                        sub[x] = form_summary(d)
                if out is not None:
                    out["forms"] = sub
                    out["forms_what"] = (
                        "the other configurations in the same run: rmat (plain, R-MAT n=2^24), "
                        "uniform (plain, n=2^16), segmented (batched form: 1024 graphs in one "
                        "persistent kernel replayed as a CUDA graph, against one launch per "
                        "minibatch), serving (served form on R-MAT n=2^26, 2^30 edges: saturation "
                        "and p50/p99 request latency at 0.5/0.8/0.95 load, against one request at "
                        "a time)")
        if dist is not None:
            dist.destroy_process_group()
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
