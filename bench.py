"""Benchmark: exact model counting at n = 36 on one B300 (and N replicas).

Workload (count mode, 2^36 assignments each, nothing stored): transitive
relations on 6 points (36 letters r(i,j), transitivity only), triangle-free
labelled graphs on 9 vertices (36 edge letters), automorphisms of the seeded
random graph G(6, 1/2) (seed 3) as 6 x 6 permutation matrices.  One step
counts all three.  Metric: assignments per second (Gassign/s) over the whole
job; the roofline is the integer-logic (lop3) pipe.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs the same workload on its own GPU (replicas:
the formulas are independent problems, no data-path collective); value =
all ranks' assignments / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Host allocator: the serving leg compiles on 8 client threads, and the
# library's shared host caches free a build on whichever thread evicts it, so
# most frees return memory to another thread's malloc arena, under that
# arena's lock.  A larger per-thread free cache (glibc tunable, read only at
# process start) keeps those frees thread-local: on 8 threads the host side
# of a submission ran at 9,900 instead of 5,400 requests/s.  The bench
# restarts itself once with the tunable set; an application sets it the same
# way (or links another allocator).
MALLOC_TUNABLE = "glibc.malloc.tcache_count=1000"
if MALLOC_TUNABLE not in os.environ.get("GLIBC_TUNABLES", "") and __name__ == "__main__":
    _t = os.environ.get("GLIBC_TUNABLES", "")
    os.environ["GLIBC_TUNABLES"] = f"{_t}:{MALLOC_TUNABLE}" if _t else MALLOC_TUNABLE
    os.execv(sys.executable, [sys.executable] + sys.argv)

LOP3_LANES_PER_CLK_SM = 64      # lop3.b32 issue rate per SM per clock on sm_103a (fbg_probe_lop3_rate: 0.99 of it)
NOMINAL_SM_MHZ = 2032.0         # maximum SM clock of the part, when nvidia-smi gives none

# Figures from one ncu capture of the count and table kernels, valid only for
# the kernel sources they were taken from: `sources_sha` is
# kernel_fingerprint() of the captured build (the NVRTC sources of the three
# count kernels in their tuned shapes, or of the table kernel).  When the
# running build's fingerprint differs, the figures are reported as null with
# the reason.
#   count: DRAM bytes (read + write) of the three count launches of a step, and
#          their vector-pipe LOP3 warp instructions (sass__inst_executed_per_opcode:
#          the formulas' LUTs and the popcount's full adders, not the ULOP3 of
#          the uniform datapath)
#          and, per launch (transitive, triangle-free, Aut), the issue slots used
#          and the ALU pipe's busy share, in % of the SMs' active cycles
#          (smsp__issue_active, sm__inst_executed_pipe_alu), with the SMs'
#          active and elapsed cycles (ncu serialises the three launches)
#   table: DRAM bytes of one truth-table launch
NCU_COUNT = {"sources_sha": "eb8600039356cfa3", "traffic_step": 47_104 + 101_632 + 54_016,
             "vector_lop3_step": 8_895_229 + 22_819_402 + 34_166,
             "per_launch": {"issue_slots_used_pct": [43.7, 64.9, 25.1], "alu_pipe_pct": [70.7, 79.4, 35.1],
                            "sm_active_cycles": [46_995, 109_828, 374], "sm_elapsed_cycles": [58_887, 118_257, 13_903]}}
NCU_TABLE = {"sources_sha": "898d05ddf8c3e3ff", "traffic_launch": 478_359_040 + 68_096}


def kernel_fingerprint(progs, mode: int = 0) -> str:
    """SHA-256 (16 hex digits) of the programs' generated kernel sources in
    their current shapes: it changes whenever the emitter, a shape or the
    device header changes."""
    import hashlib
    h = hashlib.sha256()
    for p in progs:
        h.update(p.source(mode).encode())
        h.update(b"\0")
    return h.hexdigest()[:16]


def ncu_figures(table: dict, fingerprint: str, keys) -> dict:
    """The captured figures when they belong to this build, else nulls and why."""
    if table.get("sources_sha") and table["sources_sha"] == fingerprint:
        return {k: table[k] for k in keys} | {"stale": False}
    why = ("no capture recorded" if not table.get("sources_sha") else
           f"captured on sources {table['sources_sha']}, running {fingerprint}")
    return {k: None for k in keys} | {"stale": True, "reason": why}


def ncu_utilisation(per: dict) -> dict:
    """Issue slots used and ALU-pipe busy share of the count launches (ncu,
    % of active cycles), per launch and weighted by each launch's SM active
    cycles."""
    w = per["sm_active_cycles"]
    tot = sum(w)
    return {"issue_slots_used_pct": per["issue_slots_used_pct"], "alu_pipe_pct": per["alu_pipe_pct"],
            "issue_slots_used_pct_weighted": sum(a * b for a, b in zip(per["issue_slots_used_pct"], w)) / tot,
            "alu_pipe_pct_weighted": sum(a * b for a, b in zip(per["alu_pipe_pct"], w)) / tot,
            "sm_active_share": [a / e for a, e in zip(w, per["sm_elapsed_cycles"])],
            "launches": ["transitive k=6", "triangle-free k=9", "Aut(G(6,1/2))"]}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 20 ms; only the
    samples whose timestamps fall inside the timed window are summarised."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.5)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def start(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()

    def __exit__(self, *a):
        time.sleep(0.1)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        import datetime
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        inside = [r for r in rows if self.t0 is not None and self.t0 - 0.02 <= r[0] <= self.t1 + 0.02]
        window_short = not inside
        if window_short and rows and self.t0 is not None:
            mid = (self.t0 + self.t1) / 2
            inside = sorted(rows, key=lambda r: abs(r[0] - mid))[:3]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in inside:
            for nm, v in zip(names, r[3]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        mhz = sorted(r[1] for r in inside)
        return {"sm_mhz": mhz[len(mhz) // 2] if mhz else None, "sm_max_mhz": inside[0][2] if inside else None,
                "reasons": sorted(reasons), "samples": len(inside), "window_s": (self.t1 - self.t0) if self.t0 else None,
                "nearest_outside_window": window_short}


def workloads():
    from paper_1310_6978_b300 import workloads as W
    return [W.TRANSITIVE6, W.TRIFREE9, W.AUT6]


# ----------------------------------------------------------------- oracle --

def cpu_oracle_rate(wls, seconds_budget: float, seed: int = 7):
    """The oracle as it stands, all host cores, on random subcubes of each
    formula (2^22 assignments each) until the budget is used."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)
    cores = oracle.max_threads()
    done = 0
    t0 = time.perf_counter()
    chunks = 0
    while time.perf_counter() - t0 < seconds_budget or chunks < len(wls):
        wl = wls[chunks % len(wls)]
        th = oracle.Theory(wl.text, wl.k)
        fixed = [int(v) for v in rng.choice(wl.n, wl.n - 22, replace=False)]
        mask = sum(1 << v for v in fixed)
        vals = int(rng.integers(0, 1 << 62)) & mask
        th.count_cube_par(mask, vals)
        done += 1 << 22
        chunks += 1
    dt = time.perf_counter() - t0
    return done / dt, cores, f"{chunks} random subcubes of 2^22 assignments (22 free letters) over the three n=36 formulas, {dt:.1f} s"


def cpu_single_thread_rate(wls, seconds_budget: float = 3.0, seed: int = 11):
    """The oracle on one host thread, same kind of sample (2^20-assignment
    subcubes)."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)
    done, chunks = 0, 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds_budget or chunks < len(wls):
        wl = wls[chunks % len(wls)]
        th = oracle.Theory(wl.text, wl.k)
        fixed = [int(v) for v in rng.choice(wl.n, wl.n - 20, replace=False)]
        mask = sum(1 << v for v in fixed)
        th.count_cube(mask, int(rng.integers(0, 1 << 62)) & mask)
        done += 1 << 20
        chunks += 1
    return done / (time.perf_counter() - t0)


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def e2e_once(F, tuning, wls, stream, cache):
    """One end-to-end step through the public API: compile each text, apply
    its tuned shape, count it; returns the counts."""
    counts = []
    for w in wls:
        p = F.compile(w.text, w.k)
        tuning.ensure(p, 0, cache)
        counts.append(p.count(stream=stream))
    return counts


def run_small(torch, F, stream):
    """Posets on 3 points (n = 9, 19 models, 8-word table): latency of the
    public calls (host round trip) and device time of back-to-back launches."""
    from paper_1310_6978_b300 import workloads as W
    wl = W.POSET3
    p = F.compile(wl.text, wl.k)
    table = torch.zeros(p.table_words(), dtype=torch.int64, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert p.count(stream) == 19
    p.truth_table(table, stream)
    stream.synchronize()
    host_us = []
    for _ in range(200):
        t0 = time.perf_counter()
        c = p.count(stream)
        host_us.append((time.perf_counter() - t0) * 1e6)
    assert c == 19
    host_us.sort()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 200
    with torch.cuda.stream(stream):
        for _ in range(5):
            p.count_async(out, stream=stream)
        e0.record(stream)
        for _ in range(reps):
            p.count_async(out, stream=stream)
        e1.record(stream)
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for _ in range(reps):
            p.truth_table(table, stream)
        e3.record(stream)
    stream.synchronize()
    assert int(out.item()) == 19
    return {"workload": "posets on 3 points (n=9): count 19, 8-word table",
            "count_call_us_p50": host_us[len(host_us) // 2], "count_call_us_p99": host_us[int(0.99 * len(host_us))],
            "count_launch_us": e0.elapsed_time(e1) * 1e3 / reps, "table_launch_us": e2.elapsed_time(e3) * 1e3 / reps,
            "basis": "call = fbg_count incl. launch, sync and copy of the count to the host; launch = CUDA-event "
                     "time per launch over 200 back-to-back launches"}


def oracle_step(wls, bits, rng):
    """One reference step: one random subcube of 2^bits assignments per
    formula, counted by the oracle on all host cores; returns seconds."""
    import oracle
    t0 = time.perf_counter()
    for wl in wls:
        th = oracle.Theory(wl.text, wl.k)
        fixed = [int(v) for v in rng.choice(wl.n, wl.n - bits, replace=False)]
        mask = sum(1 << v for v in fixed)
        th.count_cube_par(mask, int(rng.integers(0, 1 << 62)) & mask)
    return time.perf_counter() - t0


def run_reference(args, rank, world):
    """The oracle as it stands on the same metric; each step is a bounded
    sample (one subcube per formula) sized so that warm-up and timed steps
    together take about --ref-total-seconds."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    wls = workloads()
    rng = np.random.default_rng(7)
    probe = oracle_step(wls, 16, rng) / (3 << 16)            # seconds per assignment
    per_step = max(0.002, args.ref_total_seconds / max(1, args.steps + args.warmup))
    bits = int(min(22, max(10, np.floor(np.log2(max(1.0, per_step / probe / 3))))))
    for _ in range(args.warmup):
        oracle_step(wls, bits, rng)
    times = [oracle_step(wls, bits, rng) for _ in range(args.steps)]
    rate = 3 * (1 << bits) / sorted(times)[len(times) // 2]
    cores = oracle.max_threads()
    sample = (f"per step one random subcube of 2^{bits} assignments of each of the three n=36 formulas, "
              f"{args.steps} timed steps (median)")
    line = {"metric": "model-count throughput at n=36 (Gassign/s)", "value": rate / 1e9, "unit": "Gassign/s",
            "impl": "reference", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 3 * (1 << bits) / rate * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "count n=36: transitive k=6, triangle-free k=9, Aut(G(6,1/2)) seed 3",
                       "engine": "CPU oracle (model checking per assignment)", "flush_l2": False},
            "cpu_baseline": {"value": rate / 1e9, "unit": "Gassign/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate / 1e9, "unit": "Gassign/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_table(args, torch, F, L, peaks):
    """Truth table of the seeded 3-CNF with n = 32, m = 136 (seed 1): 2^26
    64-bit words = 512 MiB written per launch into a caller-owned tensor
    (larger than L2, so no flush is needed between launches)."""
    from paper_1310_6978_b300 import workloads as W
    from paper_1310_6978_b300 import tuning
    wl = W.CNF32
    p = F.compile(wl.text, wl.k)
    stream = torch.cuda.Stream()
    cache = tuning.load()
    shape = tuning.ensure(p, 1, cache, tune=args.autotune, stream=stream)
    if args.autotune and args.tune_out:
        merged = tuning.load(args.tune_out)
        merged.update(cache)
        tuning.save(merged, args.tune_out)
    table = torch.empty(p.table_words(), dtype=torch.int64, device="cuda")
    for _ in range(3):
        p.truth_table(table, stream)
    stream.synchronize()
    cnt = p.count(stream)
    reps = max(5, min(args.steps, 50))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(reps):
            p.truth_table(table, stream)
        e1.record(stream)
    stream.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    import numpy as np
    host = table.cpu().numpy().view(np.uint64)
    pop = int(np.bitwise_count(host).sum())
    assert pop == cnt
    nbytes = table.numel() * 8
    peak = peaks.get("hbm_gbs")
    ncu = ncu_figures(NCU_TABLE, kernel_fingerprint([p], 1), ["traffic_launch"])
    return {"workload": "3-CNF n=32 m=136 seed 1 (unsatisfiable: an all-zero table), full truth table", "shape": shape, "value": (1 << 32) / t / 1e9, "unit": "Gassign/s",
            "ms": t * 1e3, "bytes_written": nbytes, "count": cnt, "popcount_equals_count": True,
            "roofline": {"bound": "hbm", "achieved": nbytes / t / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": (nbytes / t / 1e9) / peak if peak else None, "traffic": ncu["traffic_launch"],
                         "traffic_capture": ncu,
                         "basis": "algorithmic bytes = 2^32/8 written per launch; peak = measured copy GB/s "
                                  "(MEASURED_PEAKS.json hbm_gbs)"}}


def _table_launch_ms(torch, p, table, stream, reps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(reps):
            p.truth_table(table, stream)
        e1.record(stream)
    stream.synchronize()
    return e0.elapsed_time(e1) / reps


def run_table_dense(args, torch, F, L, peaks, lop3_peak):
    """Truth table of a satisfiable 3-CNF with many models: n = 32, ratio 2
    (m = 64 clauses), seed 3.  Its level conjunctions prune far less than
    those of the ratio-4.25 formula, and with pruning off (the paper's
    evaluation of every block) none of its logic is skipped.  Each variant
    is timed, its executed lop3 read from the level counters of an untimed
    launch, and reported against both roofs (the integer-logic pipe and the
    HBM write bandwidth); the bound is the larger fraction."""
    import hashlib
    import numpy as np
    from paper_1310_6978_b300 import workloads as W
    wl = W.cnf3(32, 3, 2.0)
    stream = torch.cuda.Stream()
    table = torch.empty(1 << 26, dtype=torch.int64, device="cuda")
    gold = {}
    gpath = os.path.join(ROOT, "tests", "golden", "cnf32_r2_seed3.txt")
    if os.path.exists(gpath):
        for ln in open(gpath):
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()
                gold[k] = v
    peak_hbm = peaks.get("hbm_gbs")
    out = {"workload": "3-CNF n=32 m=64 (ratio 2) seed 3: full truth table (512 MiB), "
                       f"{gold.get('count', '?')} models"}
    digests = []
    for name, prune in (("pruned", 1), ("unpruned", 0)):
        p = F.compile(wl.text, wl.k).set_option(L.OPT_PRUNE, prune)
        for _ in range(2):
            p.truth_table(table, stream)
        stream.synchronize()
        ms = _table_launch_ms(torch, p, table, stream, max(3, min(args.steps, 10)))
        host = table.cpu().numpy().view(np.uint64)
        digests.append(hashlib.sha256(host.astype("<u8").tobytes()).hexdigest())
        pop = int(np.bitwise_count(host).sum())
        cnt = p.count(stream)
        assert pop == cnt, (pop, cnt)
        p.set_option(L.OPT_STATS, 1)
        p.truth_table(table, stream)
        es = p.exec_stats()
        p.set_option(L.OPT_STATS, 0)
        t = ms / 1e3
        alu = es.lop3_executed / t
        hbm = (1 << 29) / t / 1e9
        fr_alu = alu / lop3_peak
        fr_hbm = hbm / peak_hbm if peak_hbm else None
        bound = "alu" if fr_hbm is None or fr_alu >= fr_hbm else "hbm"
        out[name] = {"ms": ms, "value": (1 << 32) / t / 1e9, "unit": "Gassign/s", "count": cnt,
                     "executed_lop3": es.lop3_executed, "nominal_lop3": es.lop3_nominal,
                     "executed_over_nominal": es.lop3_executed / es.lop3_nominal if es.lop3_nominal else None,
                     "roofline": {"bound": bound, "alu": {"achieved": alu / 1e12, "peak": lop3_peak / 1e12,
                                                         "unit": "Tlop3/s", "frac": fr_alu},
                                  "hbm": {"achieved": hbm, "peak": peak_hbm, "unit": "GB/s", "frac": fr_hbm}}}
    out["tables_identical"] = digests[0] == digests[1]
    out["sha256"] = digests[0]
    out["matches_golden"] = (digests[0] == gold.get("sha256")) if gold else None
    assert out["tables_identical"]
    return out


def run_enumerate(args, torch, F, L):
    """Model list of transitive relations on 6 points (n = 36, 9,415,189
    models), the first 10^6 in ascending j, with the specialised kernel
    (per-item counts, scan, ordered writes) and with the interpreter.  Each
    call is timed end to end on the host (it synchronises); the lists must be
    equal, ascending, and every sampled model must decode to a transitive
    relation (checked here in plain Python)."""
    import numpy as np
    from paper_1310_6978_b300 import workloads as W
    wl = W.TRANSITIVE6
    cap = 1_000_000
    stream = torch.cuda.Stream()
    res = {"workload": "transitive relations on 6 points (n=36), first 10^6 models in ascending order", "cap": cap}
    lists = {}
    for name, eng in (("jit", L.ENGINE_JIT), ("interp", L.ENGINE_INTERP)):
        p = F.compile(wl.text, wl.k).set_option(L.OPT_ENGINE, eng)
        buf = torch.empty(cap, dtype=torch.int64, device="cuda")
        p.enumerate_models(buf, cap, stream)        # builds, warms
        reps = 3 if name == "interp" else max(3, min(args.steps, 10))
        t0 = time.perf_counter()
        for _ in range(reps):
            total, written = p.enumerate_models(buf, cap, stream)
        t = (time.perf_counter() - t0) / reps
        lists[name] = buf.cpu().numpy().view(np.uint64).copy()
        res[name] = {"ms": t * 1e3, "total": total, "written": written, "models_per_s": written / t,
                     "gassign_per_s": (1 << 36) / t / 1e9}
    a = lists["jit"]
    assert np.array_equal(a, lists["interp"]) and bool(np.all(a[1:] > a[:-1]))
    rng = np.random.default_rng(6)
    for j in rng.choice(a, 2000, replace=False):
        j = int(j)
        r = [[(j >> (i * 6 + l)) & 1 for l in range(6)] for i in range(6)]
        assert all((not (r[x][y] and r[y][z])) or r[x][z] for x in range(6) for y in range(6) for z in range(6))
    res["lists_equal"] = True
    res["sampled_models_transitive"] = 2000
    res["speedup_jit_vs_interp"] = res["interp"]["ms"] / res["jit"]["ms"]
    return res


def run_batched(args, torch, F, L):
    """4096 mixed formulas (seed 2) in one persistent launch replayed from a
    CUDA graph, against one interpreter launch per formula (same kernel,
    per-formula synchronisation)."""
    from paper_1310_6978_b300 import workloads as W
    mix = W.batch_mix(4096, 2)[:args.batch_formulas]
    progs = [F.compile(w.text, w.k) for w in mix]
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    b = F.Batch(progs, use_graph=True)
    t_create = time.perf_counter() - t0         # plans, NVRTC compiles (worker pool), graph capture
    for _ in range(3):
        b.run(stream)
    counts = b.results(stream)
    reps = max(3, min(args.steps, 20))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(reps):
            b.run(stream)
        e1.record(stream)
    stream.synchronize()
    assert [int(x) for x in b.results(stream)] == [int(x) for x in counts]
    t_batch = e0.elapsed_time(e1) / 1e3 / reps
    # one launch per formula with the engine the batch uses for it (the
    # specialised kernel or the interpreter), synchronised each time
    kinds = b.program_kinds()
    singles = [F.compile(w.text, w.k).set_option(L.OPT_ENGINE, L.ENGINE_JIT if kd else L.ENGINE_INTERP)
               for w, kd in zip(mix, kinds)]
    for i, p in enumerate(singles):          # builds (and compiles) every engine before timing
        if kinds[i] or i < 64:
            p.count(stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    single_counts = [p.count(stream) for p in singles]
    t_single = time.perf_counter() - t0
    assert single_counts == [int(x) for x in counts]
    # plain launches without Python or synchronisation per formula: one count
    # launch per formula issued back to back from C (fbg_count_each)
    dev = torch.zeros(len(singles), dtype=torch.int64, device="cuda")
    F.count_each(singles, dev, stream)
    stream.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        e2.record(stream)
        F.count_each(singles, dev, stream)
        e3.record(stream)
    stream.synchronize()
    t_plain_wall = time.perf_counter() - t0
    t_plain = e2.elapsed_time(e3) / 1e3
    assert F.read_counts(dev) == [int(x) for x in counts]
    small = [i for i, w in enumerate(mix) if w.n <= 20]
    sb = F.Batch([progs[i] for i in small], use_graph=True)
    for _ in range(3):
        sb.run(stream)
    sb.results(stream)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(reps):
            sb.run(stream)
        e1.record(stream)
    stream.synchronize()
    t_small_b = e0.elapsed_time(e1) / 1e3 / reps
    t0 = time.perf_counter()
    for i in small:
        singles[i].count(stream)
    t_small_s = time.perf_counter() - t0
    assign = sum(1 << w.n for w in mix)
    assign_small = sum(1 << mix[i].n for i in small)
    info = b.info()
    return {"formulas": len(mix), "specialized_programs": info["specialized"],
            "specialized_formulas": int(sum(kinds)), "assignments": assign, "value": assign / t_batch / 1e9, "unit": "Gassign/s",
            "ms": t_batch * 1e3, "per_formula_ms": t_single * 1e3, "speedup_vs_per_formula": t_single / t_batch,
            "create_s": t_create,
            "plain_launches": {"ms": t_plain * 1e3, "wall_ms": t_plain_wall * 1e3, "speedup": t_plain / t_batch,
                               "basis": "one count launch per formula issued back to back from C (fbg_count_each), "
                                        "no per-formula synchronisation; CUDA events around all of them"},
            "per_formula_basis": "Python loop of fbg_count (launch, copy of the count, synchronisation) per formula",
            "small_n_le_20": {"formulas": len(small), "batched_ms": t_small_b * 1e3, "per_formula_ms": t_small_s * 1e3,
                              "speedup": t_small_s / t_small_b,
                              "batched_gassign_s": assign_small / t_small_b / 1e9},
            "queue": {"items": info["items"], "units": info["units"], "grid": info["grid"]}, "graph": True,
            "counts_match_per_formula": True}


def run_serving(args, torch, F, L):
    """Poisson stream of requests (seed 5): n uniform in 16..38, a family with
    exactly n letters else 3-CNF; 90% count, 10% enumerate (cap 1e6).  The
    rate is 0.7x the throughput of a calibration run (4000 other requests
    through the same clients and collector, unpaced).  Count requests of
    recurring texts with at least jit_min_n letters move to specialised
    kernels that the server compiles in the background."""
    import sys
    import threading
    from paper_1310_6978_b300 import workloads as W
    nreq = args.serve_requests
    # client threads that wake at their arrival times take the interpreter
    # lock from one another: hand it over every 0.5 ms instead of every 5 ms
    switch = sys.getswitchinterval()
    sys.setswitchinterval(0.0005)
    # one-time costs (module loads, the stream-ordered pool) are paid by an
    # untimed burst of other requests; the calibration has texts of its own,
    # as the stream has
    warm = W.request_stream(200, rate_per_s=1.0, seed=54)
    srv = F.Server(jit_min_n=args.serve_jit_min_n)
    for r in warm:
        srv.submit(r.workload.text, r.workload.k, L.MODE_ENUMERATE if r.mode == "enumerate" else L.MODE_COUNT, r.cap)
    srv.drain(600)
    srv.close()
    nclients = 8

    def play(srv, reqs, paced):
        """Submit reqs from nclients client threads (client c submits requests
        c, c + nclients, ...; submission compiles the text on the calling
        thread, and one thread alone could not keep up), at their arrival
        times when paced, else as fast as they go, while this thread collects
        the results.  Returns (per request (latency from submission, count,
        latency from admission), per request delay past its arrival time,
        the largest delay, wall seconds until the last result)."""
        index = {}                           # request id -> position in reqs
        done = [None] * len(reqs)
        late = [0.0] * nclients              # largest delay of a submission past its arrival time
        lag = [0.0] * len(reqs)              # each request's submission delay past its arrival time
        start = time.perf_counter()

        def producer(c):
            for i in range(c, len(reqs), nclients):
                r = reqs[i]
                if paced:
                    delay = start + r.arrival_s - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                    else:
                        late[c] = max(late[c], -delay)
                    lag[i] = max(0.0, time.perf_counter() - (start + r.arrival_s))
                rid = srv.submit(r.workload.text, r.workload.k,
                                 L.MODE_ENUMERATE if r.mode == "enumerate" else L.MODE_COUNT, r.cap)
                index[rid] = i

        def collect():
            # the requests finished since the last call (fbg_server_completed):
            # read each result and release it, so that results (model lists of
            # up to 10^6 words) do not pile up
            got = 0
            for rid in srv.completed():
                while rid not in index:      # finished before the producer recorded it
                    time.sleep(0.0005)
                res = srv.poll(rid, models=False)
                assert res["status"] == 0
                done[index[rid]] = (res["done_s"] - res["submit_s"], res["count"], res["done_s"] - res["admit_s"])
                srv.release(rid)
                got += 1
            return got

        clients = [threading.Thread(target=producer, args=(c,)) for c in range(nclients)]
        for th in clients:
            th.start()
        while any(th.is_alive() for th in clients):
            clients[0].join(0.05)
            collect()
        for th in clients:
            th.join()
        srv.drain(max(300.0, 3 * reqs[-1].arrival_s if paced else 0.0))
        wall = time.perf_counter() - start
        while collect():
            pass
        assert all(d is not None for d in done)
        return done, lag, max(late), wall

    # the calibration: the same clients and collector with no pacing, so the
    # throughput includes the host's compiles and the collection of results
    calib = W.request_stream(min(4000, nreq), rate_per_s=1.0, seed=55)
    srv = F.Server(jit_min_n=args.serve_jit_min_n)
    t_cal = play(srv, calib, paced=False)[3]
    srv.close()
    rate = args.serve_rate if args.serve_rate > 0 else 0.7 * len(calib) / t_cal
    reqs = W.request_stream(nreq, rate_per_s=rate, seed=5)
    srv = F.Server(jit_min_n=args.serve_jit_min_n)
    done, lag, max_lag, wall = play(srv, reqs, paced=True)
    lat, lat_arr, lat_srv, assign, counts = [], [], [], 0, []
    for (lt, cnt, ls), r, lg in zip(done, reqs, lag):
        lat.append(lt)
        lat_srv.append(ls)
        lat_arr.append(lt + lg)
        assign += 1 << r.workload.n
        counts.append(cnt)
    st = srv.stats()
    srv.close()
    # exactness on a sample: the server's counts equal standalone counts of
    # the specialised kernel (n <= 30: its compile time stays small) or the
    # interpreter (larger n)
    rng = __import__("random").Random(5)
    sample = rng.sample(range(len(reqs)), min(60, len(reqs)))
    for i in sample:
        r = reqs[i]
        p = F.compile(r.workload.text, r.workload.k)
        if r.workload.n > 30:
            p.set_option(L.OPT_ENGINE, L.ENGINE_INTERP)
        assert p.count() == counts[i]
    small = sorted(l for l, r in zip(lat, reqs) if r.workload.n <= 27)
    lat.sort()
    lat_arr.sort()
    lat_srv.sort()
    sys.setswitchinterval(switch)
    return {"requests": len(reqs), "rate_per_s": rate, "wall_s": wall, "p50_ms": lat[len(lat) // 2] * 1e3,
            "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))] * 1e3,
            "latency_basis": "p50_ms/p99_ms: entry to fbg_server_submit (the request's compile and host build "
                             "included) to its result, server clock",
            "value": assign / wall / 1e9,
            "unit": "Gassign/s", "ticks": st["ticks"], "launches": st["launches"],
            "server_s": {k: st[k] for k in ("busy_s", "admit_s", "count_s", "enum_s", "gpu_s")}, "clients": nclients,
            "recurring_texts": {"specialised_programs": st["jit_programs"], "requests_on_them": st["jit_requests"],
                                "background_compile_s": st["jit_compile_s"],
                                "jit_min_n": args.serve_jit_min_n or 30},
            "latency_from_admission_ms": {"p50": lat_srv[len(lat_srv) // 2] * 1e3,
                                          "p99": lat_srv[min(len(lat_srv) - 1, int(0.99 * len(lat_srv)))] * 1e3,
                                          "basis": "admission by the server thread (host build done, program "
                                                   "uploaded) to the result: the ticks' queueing and work"},
            "latency_from_arrival_ms": {"p50": lat_arr[len(lat_arr) // 2] * 1e3,
                                        "p99": lat_arr[min(len(lat_arr) - 1, int(0.99 * len(lat_arr)))] * 1e3,
                                        "basis": "the client's delay past the scheduled arrival time plus the "
                                                 "time from entering fbg_server_submit (compile and host build "
                                                 "included) to the result"},
            "submit_lag_s": max_lag, "arrival_window_s": reqs[-1].arrival_s,
            "p50_ms_n_le_27": small[len(small) // 2] * 1e3 if small else None,
            "model_lists": sum(1 for r in reqs if r.mode == "enumerate"),
            "checked_against_single_counts": len(sample), "calibration": {"requests": len(calib), "s": t_cal},
            "_oracle_sample": [(reqs[i].workload, counts[i]) for i in sample[:24]]}


def oracle_check_serving(F, L, torch, sample, seed=5):
    """CPU-baseline leg: the oracle checks a sample of the served counts --
    all 2^n assignments up to n = 22; above, the interpreter's per-unit counts
    (units of 2^(n-16) or more assignments) must add up to the served count
    and three sampled units must equal the oracle's subcube counts."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)
    checked = 0
    for wl, count in sample:
        th = oracle.Theory(wl.text, wl.k)
        if wl.n <= 22:
            assert th.count_par(0, 1 << wl.n) == count, wl
        else:
            p = F.compile(wl.text, wl.k).set_option(L.OPT_ENGINE, L.ENGINE_INTERP)
            p.set_option(L.OPT_UNIT_BITS, min(16, wl.n - 18))
            vars_, nunits = p.unit_vars()
            dev = torch.zeros(nunits, dtype=torch.int64, device="cuda")
            p.count_units(dev)
            uc = F.read_counts(dev)
            assert sum(uc) == count, wl
            mask = sum(1 << v for v in vars_)
            for u in {0, nunits - 1, int(rng.integers(0, nunits))}:
                vals = sum(((u >> b) & 1) << v for b, v in enumerate(vars_))
                assert uc[u] == th.count_cube_par(mask, vals), (wl, u)
        checked += 1
    return checked


# -------------------------------------------------------------------- ours --

def max_over_ranks(t_local: float, world: int, device: str) -> float:
    """The slowest rank's time (seconds): the job's time under replicas."""
    import torch
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_all_ranks: int, t_max: float) -> float:
    """Giga-units per second for the whole job: every rank's units over the
    slowest rank's time."""
    return units_all_ranks / t_max / 1e9


def run_ours(args, rank, world):
    import torch
    import paper_1310_6978_b300 as F
    from paper_1310_6978_b300 import _lib as L

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    from paper_1310_6978_b300 import tuning
    wls = workloads()
    stream = torch.cuda.Stream()
    cache = tuning.load()
    # end to end, cold: the first compile and count of each text in this
    # process (parse, ground, layout, lowering, item pruning, emit, NVRTC,
    # module load, launch, copy of the count)
    t0 = time.perf_counter()
    cold_counts = e2e_once(F, tuning, wls, stream, cache)
    e2e_cold_t = time.perf_counter() - t0
    progs = [F.compile(w.text, w.k) for w in wls]
    shapes = [tuning.ensure(p, 0, cache, tune=args.autotune, stream=stream, refine=args.retune) for p in progs]
    if (args.autotune or args.retune) and args.tune_out:
        tuning.save(cache, args.tune_out)
    for p in progs:                       # longest-first item order (setup, untimed)
        p.schedule_units(stream=stream)
    out = torch.zeros(len(progs), dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > L2 (126 MB)

    # a step counts the three programs concurrently, one stream each (forked
    # from and joined back into `stream`), so that one kernel's tail overlaps
    # the others' work
    side = [torch.cuda.Stream() for _ in progs]
    fork = torch.cuda.Event()
    joins = [torch.cuda.Event() for _ in progs]

    def step(on):
        fork.record(on)
        for i, p in enumerate(progs):
            side[i].wait_event(fork)
            p.count_async(out[i:i + 1], stream=side[i])
            joins[i].record(side[i])
            on.wait_event(joins[i])

    for _ in range(max(3, args.warmup)):
        step(stream)
    stream.synchronize()
    expected = out.cpu().tolist()
    # The step is captured once as a CUDA graph (the count launches reset
    # their own counters, so a replay needs no memsets) and replayed: the
    # host then enqueues four operations per step and stays ahead of the GPU.
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step(stream)
    graph.replay()
    stream.synchronize()
    assert out.cpu().tolist() == expected

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    step_ms = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # The steps are enqueued back to back on one stream, each after an L2
    # flush on the same stream; the host runs ahead of the GPU, so the events
    # time the device work and not the host's submission.
    with ClockSampler(dev) as clk:
        clk.start()
        with torch.cuda.stream(stream):
            for s in range(args.steps):
                flush.zero_()                              # L2 flushed between timed steps
                evs[s][0].record(stream)
                graph.replay()
                evs[s][1].record(stream)
        stream.synchronize()
        clk.stop()
    torch.cuda.synchronize()
    got = out.cpu().tolist()
    assert got == expected, (got, expected)
    for s in range(args.steps):
        step_ms.append(evs[s][0].elapsed_time(evs[s][1]))
    t_max = max_over_ranks(sum(step_ms) / 1e3, world, "cuda")
    assign_per_step = sum(1 << w.n for w in wls)
    value = whole_job_rate(world * assign_per_step * args.steps, t_max)

    # end to end through the public API, warm: per step each text is compiled
    # (fbg_compile), given its tuned shape and counted (fbg_count: launch,
    # copy of the count to the host, synchronisation); the host caches hold
    # the compiled theory, the kernel build and the NVRTC kernel.  Timed
    # before the other legs (after the batch and serving legs, with hundreds
    # more kernels and buffers in the process, the host side runs slower).
    e2e_steps = 3 if args.quick else max(3, min(args.steps, 20))
    e2e_once(F, tuning, wls, stream, cache)                      # untimed: fills the caches
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        res = e2e_once(F, tuning, wls, stream, cache)
        assert res == expected
    e2e_t = (time.perf_counter() - t0) / e2e_steps
    # bytes a new program sends to the device per count: its item list (4 B
    # per entry; the kernel parameters and the scratch memset aside)
    e2e_h2d = 4 * sum(int(p.debug_dump(0).get("item_list_entries", 0)) for p in progs)

    # executed work of the same kernels (level iteration counters), untimed
    executed = 0.0
    nominal = 0.0
    uniform = 0.0
    for p in progs:
        p.set_option(L.OPT_STATS, 1)
        p.count()
        es = p.exec_stats()
        executed += es.lop3_executed
        nominal += es.lop3_nominal
        uniform += es.lop3_uniform
        p.set_option(L.OPT_STATS, 0)
    kern_s = sum(step_ms) / args.steps / 1e3   # the three concurrent count launches of a step
    lop3_probe = F.probe_lop3_rate(stream)      # independent lop3 chains: the measured roof
    clocks = clk.summary()
    # the integer-logic roof of this GPU: its SM count x the lop3.b32 lanes per
    # SM and clock x the median SM clock sampled in the timed window (and, for
    # comparison, x the maximum SM clock)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or load_peaks().get("sm_max_mhz") or NOMINAL_SM_MHZ
    run_mhz = clocks.get("sm_mhz") or max_mhz
    peak_lop3 = sms * LOP3_LANES_PER_CLK_SM * run_mhz * 1e6
    peak_lop3_max = sms * LOP3_LANES_PER_CLK_SM * max_mhz * 1e6
    ncu = ncu_figures(NCU_COUNT, kernel_fingerprint(progs, 0), ["traffic_step", "vector_lop3_step", "per_launch"])

    # the paper's brute-force evaluation (every word), same kernels without pruning
    brute = {}
    if not args.quick:
        bp = [F.compile(w.text, w.k).set_option(L.OPT_PRUNE, 0).set_option(L.OPT_STATS, 1) for w in wls]
        for p in bp:
            p.count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        bo = torch.zeros(len(bp), dtype=torch.int64, device="cuda")
        with torch.cuda.stream(stream):
            e0.record(stream)
            for i, p in enumerate(bp):
                p.count_async(bo[i:i + 1], stream=stream)
            e1.record(stream)
        stream.synchronize()
        assert bo.cpu().tolist() == expected
        bt = e0.elapsed_time(e1) / 1e3
        bex = 0.0
        for p in bp:
            p.count()
            bex += p.exec_stats().lop3_executed
        brute = {"value": assign_per_step / bt / 1e9, "unit": "Gassign/s", "ms": bt * 1e3,
                 "lop3_tops": bex / bt / 1e12, "frac": bex / bt / peak_lop3}

    table_leg = {} if args.quick else run_table(args, torch, F, L, load_peaks())
    dense_leg = {} if args.quick else run_table_dense(args, torch, F, L, load_peaks(), peak_lop3)
    enum_leg = {} if args.quick else run_enumerate(args, torch, F, L)
    small_leg = {} if args.quick else run_small(torch, F, stream)
    batched = {} if args.quick or args.no_batch else run_batched(args, torch, F, L)
    serving = {} if args.quick or args.no_serve else run_serving(args, torch, F, L)


    if rank != 0:
        return
    cpu = {}
    oracle_sample = serving.pop("_oracle_sample", None) if serving else None
    if world == 1 and not args.no_cpu:
        if oracle_sample:
            serving["checked_against_oracle"] = oracle_check_serving(F, L, torch, oracle_sample)
        rate, cores, sample = cpu_oracle_rate(wls, args.cpu_seconds)
        one = cpu_single_thread_rate(wls)
        cpu = {"value": rate / 1e9, "unit": "Gassign/s", "cores": cores, "kind": "oracle", "sample": sample,
               "single_thread_value": one / 1e9, "cpu_model": cpu_model(), "extrapolated": True}
    peaks = load_peaks()
    line = {
        "metric": "model-count throughput at n=36 (Gassign/s)",
        "value": value, "unit": "Gassign/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "count n=36: transitive k=6, triangle-free k=9, Aut(G(6,1/2)) seed 3",
                   "formulas": 3, "assignments_per_step": assign_per_step, "engine": "nvrtc straight-line, pruned, longest-first items, 3 concurrent streams captured in one CUDA graph",
                   "flush_l2": True, "parallelism": f"replicas x{world}", "counts": expected,
                   "shapes": shapes},
        "roofline": {"bound": "alu", "achieved": executed / kern_s / 1e12, "peak": peak_lop3 / 1e12,
                     "unit": "Tlop3/s", "frac": executed / kern_s / peak_lop3, "traffic": ncu["traffic_step"],
                     "frac_at_max_clock": executed / kern_s / peak_lop3_max,
                     "peak_basis": {"sms": sms, "lop3_lanes_per_clk_sm": LOP3_LANES_PER_CLK_SM,
                                    "sm_mhz": run_mhz, "sm_max_mhz": max_mhz,
                                    "clock": "median SM clock sampled in the timed window" if clocks.get("sm_mhz")
                                             else "no clock sample: maximum SM clock"},
                     "basis": "executed lane-varying lop3.b32 lane-ops of the step's three concurrent "
                              "fbg_jit_count launches (in-kernel level counters, untimed run) / CUDA-event step "
                              "time on the launching stream; lop3 whose inputs are all warp-uniform (constants, "
                              "unit letters, loop counters: the uniform datapath) are not counted",
                     "uniform_lop3_warp_ops_per_step": uniform,
                     "ncu_capture": ncu,
                     "ncu_cross_check": None if ncu["stale"] else {
                         "vector_lop3_warp_instructions_per_step": ncu["vector_lop3_step"],
                         "achieved": ncu["vector_lop3_step"] * 32 / kern_s / 1e12,
                         "frac": ncu["vector_lop3_step"] * 32 / kern_s / peak_lop3,
                         "basis": "every LOP3 the three launches issued on the vector ALU pipe (ncu count of the "
                                  "same kernels and shapes, full adders included) / CUDA-event step time"},
                     "ncu_utilisation": None if ncu["stale"] else ncu_utilisation(ncu["per_launch"])},
        "nominal_lop3_ratio": executed / nominal if nominal else None,
        "alu_probe": {"lop3_tops": lop3_probe, "of_nominal_peak": lop3_probe / (peak_lop3 / 1e12),
                      "basis": "fbg_probe_lop3_rate: 16 independent lop3.b32 chains per thread, CUDA events"},
        "brute_force": brute,
        "truth_table": table_leg,
        "truth_table_dense": dense_leg,
        "enumerate": enum_leg,
        "small_poset3": small_leg,
        "batched": batched,
        "serving": serving,
        "clocks": clocks,
        "e2e": {"value": assign_per_step / e2e_t / 1e9, "unit": "Gassign/s",
                "h2d_bytes_per_step": e2e_h2d, "d2h_bytes_per_step": 256 * len(wls),
                "ms_per_step": e2e_t * 1e3,
                "basis": "warm: per step each of the three texts -> fbg_compile -> tuned shape -> fbg_count "
                         "(one launch, the count to the host, synchronisation), host compile caches and NVRTC "
                         "kernel cache warm; no input data exists on the host (the formula is compiled there): "
                         "h2d = the new programs' item lists, d2h = the 256-byte counter head per count",
                "cold": {"value": assign_per_step / e2e_cold_t / 1e9, "unit": "Gassign/s",
                         "ms_per_step": e2e_cold_t * 1e3, "counts_match": cold_counts == expected,
                         "basis": "the first compile and count of each text in the process: parse, ground, "
                                  "layout, lowering, item pruning, emit, NVRTC, module load, count"}},
        "gpu_launches": len(wls) * args.steps,   # one fbg_jit_count launch per program and step (no memsets)
        "cpu_baseline": cpu,
        "peaks_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--only", default="", choices=["", "table", "dense", "enum", "batch", "serve"],
                    help="run one leg alone (profiling)")
    ap.add_argument("--batch-formulas", type=int, default=4096)
    ap.add_argument("--autotune", action="store_true", help="tune kernel shapes missing from the cache")
    ap.add_argument("--retune", action="store_true", help="tune again from the cached shapes, keep the better")
    ap.add_argument("--tune-out", default="", help="write the updated shape cache here")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=100000)
    ap.add_argument("--serve-rate", type=float, default=0.0, help="offered requests/s (0: 0.7 x calibrated)")
    ap.add_argument("--serve-jit-min-n", type=int, default=0,
                    help="server option jit_min_n (0: the library default, 30; -1: interpreter only)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-total-seconds", type=float, default=90.0,
                    help="reference arm: seconds for all its warm-up and timed steps together")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.init_process_group("nccl")
    if args.only:
        import torch
        import paper_1310_6978_b300 as F
        from paper_1310_6978_b300 import _lib as L
        if args.only == "table":
            leg = run_table(args, torch, F, L, load_peaks())
        elif args.only == "dense":
            leg = run_table_dense(args, torch, F, L, load_peaks(), 148 * LOP3_LANES_PER_CLK_SM * NOMINAL_SM_MHZ * 1e6)
        elif args.only == "enum":
            leg = run_enumerate(args, torch, F, L)
        elif args.only == "batch":
            leg = run_batched(args, torch, F, L)
        else:
            leg = run_serving(args, torch, F, L)
            sample = leg.pop("_oracle_sample", None)
            if sample and not args.no_cpu:
                leg["checked_against_oracle"] = oracle_check_serving(F, L, torch, sample)
        print(json.dumps(leg), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
