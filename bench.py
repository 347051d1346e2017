"""Benchmark: input GB/s of the speculative chunked DFA membership test on GB300.

Default workload (N=1): the regex-shaped test - a 512-state DFA over bytes
folded to 32 classes (gamma in 0.02-0.47), matched against 1 GiB of seeded
Zipf(1.1) printable text with 0.1% planted accepted words, by Algorithm 3 with
one reverse-lookahead symbol and the chunk starts of Eqs. (6)-(7).  One step is
one whole membership test (planning kernels + match kernel, i.e. every step of
the hot path) on device-resident input.  The input is larger than L2, so every
step streams it from HBM.  Every answer the line reports (a timed step, the
end-to-end call, every extra leg) is checked against the CPU oracle
(Algorithm 1) on the same full input.

The same line carries, each with its own clock record:
  lookahead / algorithm2 / model_vs_measured   r = 2, 4 (Eq. 13), r = 0
        (Algorithm 2) and the time model of Eqs. 14-18 beside the measurements;
  placement   Sec. 4.2's boundary placement, an optimization the paper
        suggests and sets aside (opt-in, --boundary-window; not the headline);
  configs     the other workloads: the plain 16-state DFA (4 MiB, 1024
        chunks), the protein-shaped 1288-state DFA on 10 GB, the batched mix
        (64 DFAs, 4096 tests, 21.7 GB, one graph-replayed launch against one
        call per test) and the serving loop on that mix (Poisson arrivals,
        40 GB budget, 20k req/s and 0.25-1.0x of batched capacity).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload regex|plain|protein|batch|serve]
                    [--impl ours|reference] [--no-configs] [--no-mix] [--no-cpu]

Under torchrun (N > 1) every rank matches its own independent string (seed +
rank): the tests shard with no collective on the data path (weak scaling);
value = all ranks' bytes / the slowest rank's time; the extra configs run at
N = 1 only.  --impl reference times the CPU oracle (Algorithm 1 in C) on the
host cores instead.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import gc
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "input GB/s per GB300 (batched vs plain GPU path), % of HBM peak; p50/p99 latency"
L2_BYTES = 129 << 20
OUTSIDE = ("Sec. 4.2 boundary placement: an optimization the paper suggests and sets aside; "
           "opt-in here, outside the contracted method, not the headline")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


def _workload(name: str, seed: int, nbytes: int = 0):
    import gen
    if name == "plain":
        return gen.plain_workload(seed, nbytes or (4 << 20))
    if name == "protein":
        return gen.protein_workload(seed, nbytes or 10 * 10**9)
    return gen.regex_workload(seed, nbytes or (1 << 30))


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.15)
        return self

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.file.name)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                   "reasons": sorted(reasons), "samples": len(sm)}
        return out


def lookups_per_launch(dm, d, dev, n: int, num_chunks: int = 0, lookahead: int = 1,
                       boundary_window: int = 0) -> tuple:
    """Algorithmic work of one launch (the second term of Eq. 16):
    W = L_0 + sum_{k>=1} L_k |I_k|.  |I_k| comes from the planning kernels
    (dfa_plan_sets), the chunk lengths from the chunk starts the launch uses
    (dfa_plan_starts: Eqs. 6-7, or the Sec. 4.2 placement)."""
    sizes = d.plan_sets(dev, num_chunks=num_chunks, lookahead=lookahead,
                        boundary_window=boundary_window).astype(np.int64)
    P = len(sizes)
    lens = np.diff(d.plan_starts(dev, num_chunks=num_chunks, lookahead=lookahead,
                                 boundary_window=boundary_window).astype(np.int64))
    assert len(lens) == P and int(lens.sum()) == n
    W = int((lens * sizes).sum())
    return W, float(sizes[1:].mean()) if P > 1 else 1.0


def device_code_sha(text: bytes = None) -> str:
    """sha256 prefix of the kernels' device code: dfa_kernels.cu above its host-side
    section (launch helpers below it do not change what a launch reads or writes),
    with comments and blank space dropped (they do not either)."""
    import re
    if text is None:
        src = os.path.join(ROOT, "paper_1210_5093_gb300", "csrc", "dfa_kernels.cu")
        text = open(src, "rb").read()
    cut = text.find(b"// ------------------------------------------------------------ host side")
    code = (text[:cut] if cut >= 0 else text).decode()
    code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
    code = re.sub(r"//[^\n]*", " ", code)
    code = " ".join(code.split())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def _traffic_record(workload: str, window: int = 0):
    """DRAM bytes per match-kernel launch from the committed ncu summary of this
    workload and placement window, valid only while the kernels' device code is
    unchanged."""
    sha = device_code_sha()
    name = workload + ("_w%d" % window if window else "")
    p = os.path.join(ROOT, "profiles", "k_match_%s_traffic.json" % name)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    if rec.get("kernel_source_sha") != sha:
        return None
    return rec.get("dram_bytes_per_launch")


# ------------------------------------------------------------------ the oracle

def oracle_answer(spec, data) -> tuple:
    """Algorithm 1 on the whole input (the oracle, one core); returns
    ((status, final, accept), seconds)."""
    import oracle
    od = oracle.Dfa.from_spec(spec)
    t = time.perf_counter()
    ans = od.run(data)
    return ans, time.perf_counter() - t


def oracle_answers_all_cores(specs, picks, datas):
    """Algorithm 1 on every test, one string per host thread on all host cores
    (the C oracle releases the interpreter lock).  Returns (answers, seconds,
    threads)."""
    import oracle
    ods = [oracle.Dfa.from_spec(s) for s in specs]
    threads = os.cpu_count() or 1
    order = sorted(range(len(datas)), key=lambda i: -len(datas[i]))   # longest first
    out = [None] * len(datas)

    def one(i):
        out[i] = ods[picks[i]].run(datas[i])
    t = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        list(ex.map(one, order))
    return out, time.perf_counter() - t, threads


def _as_answer(res) -> tuple:
    """(final, accept, status) from results_from -> the oracle's (status, final, accept)."""
    fs, acc, st = res
    return (st, None, None) if st != 0 else (0, fs, acc)


def run_reference(args, rank: int, world: int):
    """The oracle (Algorithm 1, plain C, one core) timed on the host."""
    if rank != 0:
        return
    w = _workload(args.workload if args.workload in ("regex", "plain", "protein") else "regex",
                  args.seed, args.bytes)
    import oracle
    od = oracle.Dfa.from_spec(w.spec)
    sample = min(len(w.data), 64 << 20)
    x = w.data[:sample]
    for _ in range(args.warmup):
        od.run(x)
    t = time.perf_counter()
    for _ in range(args.steps):
        od.run(x)
    el = time.perf_counter() - t
    gbs = sample * args.steps / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(gbs, 4), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": _dtype(w.spec), "data": "synthetic",
        "config": {"workload": w.name, "sample_bytes": sample},
        "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "first %d MiB of the %s input, Algorithm 1 in C on one core"
                                   % (sample >> 20, w.name)},
        "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU legs

class L2Flush:
    """Writes a buffer larger than L2 between timed steps of inputs that fit in L2."""

    def __init__(self, torch, nbytes: int = 2 * L2_BYTES):
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")

    def __call__(self):
        self.buf.zero_()


def single_leg(dm, torch, d, dev, n, stream, reps, r=1, win=0, num_chunks=0, tune=True,
               flush=None, tune_len=1 << 30, min_s=0.4, expect=None):
    """`reps` (at least; more until `min_s` of timed region) single-test steps of
    one configuration on a device-resident input: whole step and match kernel
    alone, CUDA events on the launching stream, clocks sampled meanwhile.
    Flushes L2 between steps when `flush` is given.  Checks the answer."""
    tr = None
    if tune and not num_chunks:
        t, _ = d.autotune(dev[:tune_len], lookahead=r, boundary_window=win)
        tr = {"states_per_thread": t.states_per_thread, "tiles_per_cta": t.tiles_per_cta,
              "ctas_per_sm": t.ctas_per_sm, "grid_waves": max(1, t.grid_waves)}
    ws = torch.empty(d.workspace_size(n, num_chunks=num_chunks, lookahead=r, boundary_window=win),
                     dtype=torch.uint8, device="cuda")
    out = torch.zeros(12, dtype=torch.uint8, device="cuda")

    def launch(ev=None):
        d.match_async(dev, out, ws, stream=stream, num_chunks=num_chunks, lookahead=r,
                      boundary_window=win, events=ev)
    with torch.cuda.stream(stream):
        for _ in range(3):
            if flush:
                flush()
            launch()
    torch.cuda.synchronize()
    res = dm.results_from(out)[0]
    if expect is not None:
        assert _as_answer(res) == expect, ("answer differs from the oracle", res, expect)
    clk = Clocks(torch.cuda.current_device()).start()
    kms, sms = [], []
    t_start = time.perf_counter()
    while len(kms) < reps or time.perf_counter() - t_start < min_s:
        batch = max(1, reps)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(batch)] for _ in range(4)]
        for e in sum(ev, []):
            e.record(stream)    # creates the events; the library re-records them around k_match
        with torch.cuda.stream(stream):
            for i in range(batch):
                if flush:
                    flush()
                ev[2][i].record(stream)
                launch((ev[0][i], ev[1][i]))
                ev[3][i].record(stream)
        torch.cuda.synchronize()
        kms += [a.elapsed_time(b) for a, b in zip(ev[0], ev[1])]
        sms += [a.elapsed_time(b) for a, b in zip(ev[2], ev[3])]
        if len(kms) > 20000:
            break
    clocks = clk.stop()
    assert dm.results_from(out)[0] == res, "the answer changed between steps"
    km, sm = statistics.median(kms), statistics.median(sms)
    return {"gbs": round(n / sm / 1e6, 3), "step_ms": round(sm, 4), "kernel_ms": round(km, 4),
            "kernel_gbs": round(n / km / 1e6, 3), "steps_timed": len(kms), "lookahead": r,
            "boundary_window": win, "tuning": tr, "clocks": clocks,
            "l2": ("flushed between steps (%d MiB written)" % (flush.buf.numel() >> 20)) if flush
            else "input larger than L2, not flushed",
            "result": {"final_state": res[0], "accept": res[1], "status": res[2]},
            "oracle_match": expect is not None}, km


def with_work(leg, dm, d, dev, n, lookup_peak, num_chunks=0):
    """Adds the leg's algorithmic work and its fraction of the lookup roof."""
    W, mI = lookups_per_launch(dm, d, dev, n, num_chunks, leg["lookahead"], leg["boundary_window"])
    leg["lookups_per_byte"] = round(W / n, 3)
    leg["mean_set"] = round(mI, 3)
    leg["lookup_roof_frac"] = round(W / (leg["kernel_ms"] / 1e3) / lookup_peak, 4)
    return W


def _mixed_strings(spec, seed: int, count: int, lo: int, hi: int):
    """Strings for the batched/serving legs: lengths log-uniform in [lo, hi]."""
    import gen
    lens = gen.batch_lengths(seed, count, lo, hi)
    return [gen.batch_text(seed * 1000003 + i, spec, int(n)) for i, n in enumerate(lens)]


def batched_leg(dm, torch, dfas, tens, reps: int = 5, window: int = 0):
    """One persistent graph-replayed launch over all tests vs the plain path
    (one dfa_match_async per string, back to back on one stream).  Device-resident;
    clocks sampled over the batched timed region."""
    total = sum(t.numel() for t in tens)
    stream = torch.cuda.Stream()
    out = torch.zeros(12 * len(tens), dtype=torch.uint8, device="cuda")
    b = dm.Batch(dfas, tens, boundary_window=window)
    with torch.cuda.stream(stream):
        for _ in range(2):
            b.launch(out, stream=stream, graph=True)
    torch.cuda.synchronize()
    res_b = dm.results_from(out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = Clocks(torch.cuda.current_device()).start()
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(reps):
            b.launch(out, stream=stream, graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    t_batch = e0.elapsed_time(e1) / 1e3 / reps
    assert dm.results_from(out) == res_b, "graph replays disagree"
    # plain path: per-string launches with one reusable workspace
    wsz = max(d.workspace_size(t.numel(), boundary_window=window) for d, t in zip(dfas, tens))
    ws = torch.empty(wsz, dtype=torch.uint8, device="cuda")
    outs = torch.zeros(12 * len(tens), dtype=torch.uint8, device="cuda")

    def plain():
        for i, (d, t) in enumerate(zip(dfas, tens)):
            d.match_async(t, outs[12 * i:12 * i + 12], ws, stream=stream, boundary_window=window)
    with torch.cuda.stream(stream):
        plain()
    torch.cuda.synchronize()
    res_p = dm.results_from(outs)
    preps = max(1, reps // 2)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(preps):
            plain()
    e1.record(stream)
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3 / preps
    kernels = b.num_kernels()
    b.close()
    del ws, outs, out
    return {"tests": len(tens), "bytes": total, "gbs": round(total / t_batch / 1e9, 3),
            "ms": round(t_batch * 1e3, 3), "reps": reps, "plain_gbs": round(total / t_plain / 1e9, 3),
            "plain_ms": round(t_plain * 1e3, 3), "speedup_vs_plain": round(t_plain / t_batch, 3),
            "launches": kernels, "plain_launches": 6 * len(tens), "clocks": clocks}, res_b, res_p


def serving_leg(dm, torch, dfas, pinned, rate_gbs: float, seconds: float = 2.0,
                budget: int = 2 << 30, inflight: int = 8, seed: int = 5, window: int = 0):
    """Poisson arrivals at `rate_gbs` of offered load drawn from the given tests
    (pinned host buffers); reports achieved GB/s and arrival->result latency."""
    import gen
    mean_bytes = sum(x.numel() for x in pinned) / len(pinned)
    lam = rate_gbs * 1e9 / mean_bytes                       # requests per second
    n = max(20, int(lam * seconds))
    gaps = -np.log(1.0 - gen.unit(gen.draws(gen.key(seed, 99), n))) / lam
    picks = gen.below(gen.draws(gen.key(seed, 98), n), len(pinned)).astype(np.int64)
    srv = dm.Server(budget, max_inflight=inflight, boundary_window=window)
    clk = Clocks(torch.cuda.current_device()).start()
    gc.disable()   # arrivals keep their schedule: no interpreter collection meanwhile
    t0 = time.perf_counter()
    t_next = t0
    sub = {}
    for i in range(n):
        t_next += gaps[i]
        while time.perf_counter() < t_next:
            pass
        sub[srv.submit(dfas[picks[i]], pinned[picks[i]])] = int(picks[i])
    srv.drain(600.0)
    gc.enable()
    clocks = clk.stop()
    done = srv.poll(n + 16)
    st = srv.stats()
    srv.close()
    lat = sorted((c[5] - c[4]) * 1e3 for c in done)
    t_first = min(c[4] for c in done)
    t_last = max(c[5] for c in done)
    nbytes = sum(pinned[sub[c[0]]].numel() for c in done)
    return {"requests": len(done), "offered_gbs": round(rate_gbs, 3),
            "offered_req_s": round(lam, 1), "achieved_gbs": round(nbytes / (t_last - t_first) / 1e9, 3),
            "p50_ms": round(lat[len(lat) // 2], 3),
            "p99_ms": round(lat[min(len(lat) - 1, int(0.99 * len(lat)))], 3),
            "launches": int(st.launches), "mean_batch_bytes": int(nbytes / max(1, int(st.launches))),
            "max_concurrent_batches": int(st.max_concurrent),
            "budget_bytes": budget, "clocks": clocks}, done, sub


def rank_seed(base: int, rank: int) -> int:
    """Each rank matches its own independent test: the work shards by test,
    with no collective on the data path (weak scaling)."""
    return base + rank


def reduce_job(dist, device, bytes_per_rank: int, steps: int, elapsed_ms: float, world: int):
    """Whole-job throughput: all ranks' bytes over the slowest rank's time
    (max over ranks of the timed region).  Returns (GB/s, max elapsed ms)."""
    import torch
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return bytes_per_rank * world * steps / (ms_max / 1e3) / 1e9, ms_max


def _dtype(spec) -> str:
    return "u8" if spec.num_states + 1 <= 256 else "u16"


def _free(torch):
    import gc
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


# ------------------------------------------------------------------ configs

def plain16_config(args, dm, torch, lookup_peak):
    """The plain 16-state DFA: 4 MiB of uniform bytes in 1024 chunks (latency-bound
    by design: about 10 chains of 4 KiB per chunk).  The input fits in L2, so L2 is
    flushed between the timed steps."""
    import gen
    w = gen.plain_workload(1, 4 << 20)
    d = dm.Dfa.from_spec(w.spec)
    dev = torch.from_numpy(w.data).cuda()
    expect, t_or = oracle_answer(w.spec, w.data)
    stream = torch.cuda.Stream()
    leg, _ = single_leg(dm, torch, d, dev, len(w.data), stream, max(args.steps, 200),
                        num_chunks=w.num_chunks, flush=L2Flush(torch), expect=expect)
    with_work(leg, dm, d, dev, len(w.data), lookup_peak, w.num_chunks)
    leg.update(workload=w.name, chunks=w.num_chunks, states=w.spec.num_states,
               classes=int(d.info().num_classes),
               cpu_baseline={"value": round(len(w.data) / t_or / 1e9, 4), "unit": "GB/s",
                             "cores": 1, "kind": "oracle",
                             "sample": "the whole 4 MiB input, Algorithm 1 (C, one core)"})
    d.close()
    return leg


def protein_config(args, dm, torch, lookup_peak, nbytes: int = 10 * 10**9):
    """The protein-shaped 1288-state DFA over 20 amino-acid letters on 10 GB,
    starts of Eqs. 6-7, r = 1, autotuned on its first GiB."""
    w = _workload("protein", 3, nbytes)
    d = dm.Dfa.from_spec(w.spec)
    n = len(w.data)
    dev = torch.from_numpy(w.data).cuda()
    stream = torch.cuda.Stream()
    leg, _ = single_leg(dm, torch, d, dev, n, stream, max(3, min(args.steps, 10)))
    with_work(leg, dm, d, dev, n, lookup_peak)
    expect, t_or = oracle_answer(w.spec, w.data)
    got = (leg["result"]["status"], leg["result"]["final_state"], leg["result"]["accept"])
    assert _as_answer((got[1], got[2], got[0])) == expect, ("protein answer differs", got, expect)
    leg["oracle_match"] = True
    leg.update(workload=w.name, input_bytes=n, states=w.spec.num_states,
               classes=int(d.info().num_classes), i_max=int(d.info().i_max),
               cpu_baseline={"value": round(n / t_or / 1e9, 4), "unit": "GB/s", "cores": 1,
                             "kind": "oracle",
                             "sample": "the whole %d GB input, Algorithm 1 (C, one core); the "
                                       "same run checks the answer" % (n // 10**9)})
    del dev
    d.close()
    _free(torch)
    return leg


def batch_inputs(args):
    """The batched mix: 64 DFAs (|Q| log-uniform 8-1288, byte folded/unfolded and
    20-letter alphabets, gamma_max 0.02-0.47), `tests` tests with lengths
    log-uniform 256 B - 64 MiB."""
    import gen
    specs = gen.batch_dfas(args.seed, 64)
    lens = gen.batch_lengths(args.seed, args.tests, 256, args.max_len)
    picks = gen.batch_picks(args.seed, args.tests, len(specs))
    datas = [gen.batch_text(args.seed * 1000003 + i, specs[picks[i]], int(lens[i]))
             for i in range(args.tests)]
    return specs, picks, datas


def group_config(args, dm, torch, lookup_peak, n: int = 1 << 30, reps: int = 5, tuning=None,
                 check: bool = True, compare: bool = True):
    """Several DFAs on one input, the input staged once for all of them (Sec. 5):
    8 protein-shaped DFAs (|Q| 16-480 over the 20 amino-acid letters) on n bytes
    of protein text, as one group launch (tuned on the input first, or with the
    given (K, CTAs per SM)), against one batched launch of the same 8 tests and
    one launch per DFA.  GB/s count the input bytes once per DFA (every DFA
    reads the whole input)."""
    import gen
    specs = gen.protein_group_dfas(7)
    dfas = [dm.Dfa.from_spec(s) for s in specs]
    g = dm.Group(dfas)
    data = gen.protein_text(3, n)
    dev = torch.from_numpy(data).cuda()
    expect = None
    if check:
        expect, t_or, thr = oracle_answers_all_cores(specs, list(range(len(specs))),
                                                     [data] * len(specs))
    stream = torch.cuda.Stream()
    if tuning:
        K, cps = tuning
    else:
        K, cps, _ = g.autotune(dev, stream=stream)
    info = g.info()
    ws = torch.empty(g.workspace_size(n, states_per_thread=K, ctas_per_sm=cps), dtype=torch.uint8,
                     device="cuda")
    out = torch.zeros(12 * g.count, dtype=torch.uint8, device="cuda")
    work = torch.zeros(1, dtype=torch.int64, device="cuda")
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(reps)] for _ in range(4)]
    for e in sum(ev, []):
        e.record(stream)    # creates the events; the library re-records the first two kinds
    stream.wait_stream(torch.cuda.current_stream())
    kw = {"states_per_thread": K, "ctas_per_sm": cps}
    with torch.cuda.stream(stream):
        for _ in range(3):
            g.match_async(dev, out, ws, stream=stream, work=work, **kw)
    torch.cuda.synchronize()
    res = dm.results_from(out)
    assert expect is None or [_as_answer(r) for r in res] == expect, \
        "group answers differ from the oracle"
    W = int(work.item())
    clk = Clocks(torch.cuda.current_device()).start()
    with torch.cuda.stream(stream):
        for i in range(reps):
            ev[2][i].record(stream)
            g.match_async(dev, out, ws, stream=stream, events=(ev[0][i], ev[1][i]), **kw)
            ev[3][i].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    assert dm.results_from(out) == res, "the answers changed between steps"
    km = statistics.median(a.elapsed_time(b) for a, b in zip(ev[0], ev[1]))
    sm_ = statistics.median(a.elapsed_time(b) for a, b in zip(ev[2], ev[3]))
    # end to end through dfa_group_match on a pinned host buffer: the H2D copy of
    # the input, both kernels and the results read back, per call
    pinned = torch.from_numpy(data).pin_memory()
    for _ in range(2):
        g.match(pinned, **kw)
    e2e_calls, e2e_res = [], []
    for _ in range(max(3, reps)):
        te = time.perf_counter()
        e2e_res.append(g.match(pinned, **kw))
        e2e_calls.append(time.perf_counter() - te)
    assert expect is None or all(r == expect for r in e2e_res), \
        "end-to-end group answers differ from the oracle"
    del pinned
    e2e_s = statistics.median(e2e_calls)
    total = n * len(specs)
    leg = {"workload": "protein_group_%ddfa_%s" % (len(specs), gen._size_name(n)),
           "states": [s.num_states for s in specs], "input_bytes": n,
           "joint_classes": int(info.joint_classes), "table_bytes": int(info.table_bytes),
           "state_bytes": int(info.state_bytes),
           "tuning": {"states_per_thread": K, "ctas_per_sm": cps, "fixed": bool(tuning)},
           "chunks": g.plan_chunks(n, **kw),
           "gbs": round(total / sm_ / 1e6, 3), "input_gbs": round(n / sm_ / 1e6, 3),
           "step_ms": round(sm_, 4), "kernel_ms": round(km, 4), "steps_timed": reps,
           "lookups_per_byte": round(W / n, 3),
           "lookup_roof_frac": round(W / (km / 1e3) / lookup_peak, 4),
           "launches": 2, "clocks": clocks,
           "l2": "input larger than L2, not flushed" if n > L2_BYTES else "input fits in L2",
           "e2e": {"value": round(total / e2e_s / 1e9, 3), "unit": "GB/s",
                   "h2d_bytes_per_step": n, "d2h_bytes_per_step": 12 * len(specs),
                   "api": "dfa_group_match (pinned host buffer, copied in segments while "
                          "earlier segments are matched)",
                   "calls": len(e2e_calls), "statistic": "median call time",
                   "call_ms": [round(x * 1e3, 2) for x in e2e_calls]}}
    if compare:
        bl, res_b, res_p = batched_leg(dm, torch, dfas, [dev] * len(dfas), reps=reps)
        assert expect is None or [_as_answer(r) for r in res_b] == expect == \
            [_as_answer(r) for r in res_p], "batched or per-DFA answers differ from the oracle"
        leg.update(batched={"gbs": bl["gbs"], "ms": bl["ms"], "launches": bl["launches"]},
                   per_dfa={"gbs": bl["plain_gbs"], "ms": bl["plain_ms"],
                            "launches": bl["plain_launches"]},
                   speedup_vs_batched=round(bl["ms"] / sm_, 3),
                   speedup_vs_per_dfa=round(bl["plain_ms"] / sm_, 3))
    if check:
        leg["oracle_match"] = "all %d DFAs (group%s)" % (
            len(specs), ", batched and per-DFA launches" if compare else "")
        leg["cpu_baseline"] = {"value": round(total / t_or / 1e9, 4), "unit": "GB/s", "cores": thr,
                               "kind": "oracle",
                               "sample": "every DFA on the whole input, Algorithm 1 (C), one DFA "
                                         "per host thread; the same run checks every answer"}
    g.close()
    for d in dfas:
        d.close()
    del dev, ws, out, work
    return leg


def batch_config(args, dm, torch):
    """One persistent graph-replayed launch over the batched mix against the
    plain path (one call per test); every answer checked against the oracle,
    which runs one string per host thread on all host cores (the CPU baseline
    of this config)."""
    import gen
    t_setup = time.perf_counter()
    specs, picks, datas = batch_inputs(args)
    dfas = [dm.Dfa.from_spec(s) for s in specs]
    if not args.no_tune:
        for k, (s, d) in enumerate(zip(specs, dfas)):
            sample = torch.from_numpy(gen.batch_text(7 + k, s, 16 << 20)).cuda()
            d.autotune(sample, boundary_window=args.boundary_window)
            del sample
    tens = [torch.from_numpy(x).cuda() for x in datas]
    setup_s = time.perf_counter() - t_setup
    bl, res_b, res_p = batched_leg(dm, torch, [dfas[p] for p in picks], tens, reps=max(3, args.steps // 4),
                                   window=args.boundary_window)
    expect, t_or, threads = oracle_answers_all_cores(specs, picks, datas)
    bad = [i for i in range(len(datas)) if _as_answer(res_b[i]) != expect[i]
           or _as_answer(res_p[i]) != expect[i]]
    assert not bad, ("batched answers differ from the oracle", bad[:8])
    total = sum(len(x) for x in datas)
    bl.update(workload="batched_64dfa_%dtests" % len(datas), input_bytes=total,
              max_len=args.max_len, autotuned=not args.no_tune,
              boundary_window=args.boundary_window, oracle_match="all %d tests" % len(datas),
              setup_s=round(setup_s, 1),
              cpu_baseline={"value": round(total / t_or / 1e9, 4), "unit": "GB/s", "cores": threads,
                            "kind": "oracle", "cpu": _cpu_model(),
                            "sample": "every test of the mix, Algorithm 1 (C), one string per "
                                      "thread on %d host threads; the same run checks every answer"
                                      % threads})
    del tens
    _free(torch)
    return bl, (specs, dfas, picks, datas, expect, res_b)


def serve_config(args, dm, torch, batch_state, capacity_gbs):
    """The serving loop over the batched mix: Poisson arrivals from pinned host
    buffers at 20k requests/s and at 0.25-1.0x of the batched capacity, a 40 GB
    admission budget; every served answer checked against the oracle."""
    specs, dfas, picks, datas, expect, _ = batch_state
    pinned = [torch.from_numpy(x).pin_memory() for x in datas]
    dd = [dfas[p] for p in picks]
    mean = sum(len(x) for x in datas) / len(datas)
    rates = [("20k_req_s", 20000 * mean / 1e9)] + [("%.2fx" % f, f * capacity_gbs)
                                                   for f in (0.25, 0.5, 0.75, 1.0)]
    out = {}
    for i, (name, gbs) in enumerate(rates):
        sv, done, sub = serving_leg(dm, torch, dd, pinned, gbs, seconds=args.serve_seconds,
                                    budget=args.budget, inflight=args.inflight, seed=i + 1,
                                    window=args.boundary_window)
        for c in done:
            assert (c[3], c[1], c[2]) == expect[sub[c[0]]] or (
                c[3] != 0 and c[3] == expect[sub[c[0]]][0]), "served result differs from the oracle"
        sv["oracle_match"] = True
        out[name] = sv
    del pinned
    return {"workload": "serving_batched_mix", "pool_tests": len(datas),
            "budget_bytes": args.budget, "mean_request_bytes": int(mean),
            "inflight": args.inflight, "boundary_window": args.boundary_window,
            "batched_capacity_gbs": capacity_gbs, "points": out,
            "cpu_baseline": "as batched_cfg4 (the same requests)"}


# ------------------------------------------------------------------ main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="regex",
                    choices=["regex", "plain", "protein", "batch", "serve", "group"])
    ap.add_argument("--tests", type=int, default=4096, help="batch/serve: number of tests")
    ap.add_argument("--max-len", type=int, default=64 << 20, help="batch/serve: longest test")
    ap.add_argument("--budget", type=int, default=40 << 30, help="serve: admission budget (bytes)")
    ap.add_argument("--inflight", type=int, default=8, help="serve: batches in flight (streams)")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--bytes", type=int, default=0, help="input size override (small profiling cases)")
    ap.add_argument("--protein-bytes", type=int, default=10 * 10**9,
                    help="input size of the protein config leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle checks and CPU baselines")
    ap.add_argument("--no-mix", action="store_true", help="skip the extra legs of the headline test")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (library defaults)")
    ap.add_argument("--boundary-window", type=int, default=0,
                    help="Sec. 4.2 boundary placement window in bytes for the headline "
                         "(0: the starts of Eqs. 6-7, the paper's partition)")
    ap.add_argument("--lookahead", type=int, default=1,
                    help="reverse-lookahead symbols r of the headline test (profiling runs; "
                         "1 = Algorithm 3 as contracted, 2-8 = the sets of Eq. 13; the extra "
                         "legs and configs are skipped when r != 1)")
    ap.add_argument("--tuning", default="",
                    help="K,tiles_per_cta,ctas_per_sm[,grid_waves] instead of the autotuner "
                         "(profiling runs; for --workload group: K,ctas_per_sm)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1210_5093_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    import paper_1210_5093_gb300 as dm

    hbm_peak, sm_max_mhz, peak_src = _peaks()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    lookup_peak = nsm * 32 * sm_max_mhz * 1e6           # 32 shared-memory lanes per clock per SM

    if args.workload == "group":
        # several DFAs on one input with one shared stage, alone (profiling runs):
        # --bytes sets the input size, --tuning K,C fixes the tuning
        if rank == 0:
            tu = tuple(int(x) for x in args.tuning.split(",")[:2]) if args.tuning else None
            leg = group_config(args, dm, torch, lookup_peak, n=args.bytes or (1 << 30),
                               reps=max(1, args.steps), tuning=tu, check=not args.no_cpu,
                               compare=not args.no_mix)
            line = {"metric": METRIC, "value": leg["gbs"], "unit": "GB/s", "n_gpus": 1,
                    "steps": leg["steps_timed"], "warmup": 3, "ms_per_step": leg["step_ms"],
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                    "dtype": "u16", "data": "synthetic", "config": {"workload": leg["workload"]},
                    "group": leg}
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    if args.workload in ("batch", "serve"):
        if rank == 0:
            bl, state = batch_config(args, dm, torch)
            line = {"metric": METRIC, "value": bl["gbs"], "unit": "GB/s", "n_gpus": 1,
                    "steps": bl["reps"], "warmup": 2, "ms_per_step": bl["ms"],
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                    "dtype": "u16", "data": "synthetic",
                    "config": {"workload": bl["workload"]}, "batched": bl}
            if args.workload == "serve":
                line["serving"] = serve_config(args, dm, torch, state, bl["gbs"])
                line["value"] = line["serving"]["points"]["20k_req_s"]["achieved_gbs"]
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    w = _workload(args.workload, rank_seed(args.seed, rank), args.bytes)
    d = dm.Dfa.from_spec(w.spec)
    n = len(w.data)
    dev = torch.from_numpy(w.data).cuda()
    tuning = None
    bw = args.boundary_window
    la = args.lookahead
    if la != 1:
        args.no_mix = args.no_configs = True
    if args.tuning:
        k, tpc, cps, *gw = (int(x) for x in args.tuning.split(","))
        d.set_tuning(states_per_thread=k, tiles_per_cta=tpc, ctas_per_sm=cps, boundary_window=bw,
                     grid_waves=gw[0] if gw else 0, lookahead=la)
        tuning = {"states_per_thread": k, "tiles_per_cta": tpc, "ctas_per_sm": cps,
                  "grid_waves": gw[0] if gw else 1, "fixed": True}
    elif not w.num_chunks and not args.no_tune:
        # the library's per-DFA tuner (on at most 1 GiB), before any timing
        t, _ = d.autotune(dev[: 1 << 30], boundary_window=bw, lookahead=la)
        tuning = {"states_per_thread": t.states_per_thread, "tiles_per_cta": t.tiles_per_cta,
                  "ctas_per_sm": t.ctas_per_sm, "grid_waves": max(1, t.grid_waves)}
    P = d.plan_chunks(n, num_chunks=w.num_chunks, boundary_window=bw, lookahead=la)
    ws = torch.empty(d.workspace_size(n, num_chunks=w.num_chunks, boundary_window=bw, lookahead=la),
                     dtype=torch.uint8, device="cuda")
    out = torch.zeros(12, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    flush = L2Flush(torch) if n <= L2_BYTES else None
    kb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ke = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    se = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for e in kb + ke:
        e.record(stream)  # creates the events; the library re-records them around k_match

    def step(i=None, timed=False):
        ev = (kb[i], ke[i]) if timed else None
        if flush:
            flush()
        if timed:
            sb[i].record(stream)
        d.match_async(dev, out, ws, stream=stream, num_chunks=w.num_chunks, events=ev,
                      boundary_window=bw, lookahead=la)
        if timed:
            se[i].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()

    clocks = Clocks(local).start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            step(i, timed=True)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    # with L2 flushes between steps the steps alone are summed (the flushes are not work)
    ms = sum(a.elapsed_time(b) for a, b in zip(sb, se)) if flush else t0.elapsed_time(t1)
    k_ms = [a.elapsed_time(b) for a, b in zip(kb, ke)]
    gbs, ms_max = reduce_job(dist, "cuda", len(w.data), args.steps, ms, world)
    res_timed = dm.results_from(out)[0]

    # end to end through the public API with a pinned host buffer: H2D copy,
    # every kernel and the 12-byte result read back, per step
    pinned = torch.from_numpy(w.data).pin_memory()
    e2e_steps = max(3, min(10, args.steps))
    for _ in range(2):
        d.match(pinned, boundary_window=bw, lookahead=la)
    torch.cuda.synchronize()
    e2e_res = set()
    e2e_calls = []
    gc.disable()   # no interpreter collection inside a timed call
    for _ in range(e2e_steps):
        te = time.perf_counter()
        e2e_res.add(d.match(pinned, boundary_window=bw, lookahead=la))
        e2e_calls.append(time.perf_counter() - te)
    gc.enable()
    e2e_s = statistics.median(e2e_calls)   # per call: copies, kernels and the result read
    # context: this box's plain host-to-device copy rate (the pipelined host
    # path cannot run faster than the copies that feed it)
    h2d_buf = torch.empty(n, dtype=torch.uint8, device="cuda")
    h2d_buf.copy_(pinned, non_blocking=True)
    torch.cuda.synchronize()
    th = time.perf_counter()
    for _ in range(3):
        h2d_buf.copy_(pinned, non_blocking=True)
    torch.cuda.synchronize()
    h2d_gbs = 3 * n / (time.perf_counter() - th) / 1e9
    del h2d_buf, pinned
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    # parity of what was timed: the oracle (Algorithm 1) on the whole input
    expect, t_oracle = (None, None) if args.no_cpu else oracle_answer(w.spec, w.data)
    if expect is not None:
        assert _as_answer(res_timed) == expect, ("timed step differs from the oracle", res_timed, expect)
        assert e2e_res == {expect}, ("end-to-end answer differs from the oracle", e2e_res, expect)

    if rank == 0:
        W, mean_I = lookups_per_launch(dm, d, dev, n, w.num_chunks, la, bw)
        k_avg_s = statistics.mean(k_ms) / 1e3
        achieved = W / k_avg_s
        info = d.info()
        traffic = _traffic_record(w.name, bw) if la == 1 else None
        fs, acc, st = res_timed
        line = {
            "metric": METRIC, "value": round(gbs, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": _dtype(w.spec), "data": "synthetic",
            "config": {"workload": w.name, "states": w.spec.num_states,
                       "classes": int(info.num_classes), "input_bytes": n, "chunks": int(P),
                       "lookahead": la,
                       "algorithm": ("Algorithm 3, one reverse-lookahead symbol" if la == 1 else
                                     "Algorithm 3 with the %d-symbol sets of Eq. 13" % la
                                     if la > 1 else "Algorithm 2 (every chunk from all of Q)"),
                       "i_max": int(info.i_max), "gamma": round(info.gamma, 4),
                       "chunk_starts": ("Sec. 4.2 placement within %d bytes of Eqs. 6-7 (%s)"
                                        % (bw, OUTSIDE) if bw else "Eqs. 6-7"),
                       "boundary_window": bw, "mean_set": round(mean_I, 3),
                       "tuning": tuning,
                       "l2": "input (%d MiB) larger than L2 (129 MB); no flush needed" % (n >> 20)
                       if n > L2_BYTES else "L2 flushed between steps (input smaller than L2)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "hbm_frac": round(gbs / world / hbm_peak, 5),
            "lookups_per_byte": round(W / n, 3),
            "roofline": {"bound": "smem", "achieved": round(achieved / 1e9, 2),
                         "peak": round(lookup_peak / 1e9, 1), "unit": "Glookup/s",
                         "frac": round(achieved / lookup_peak, 4), "traffic": traffic,
                         "kernel": "k_match", "kernel_ms": round(k_avg_s * 1e3, 4),
                         "peak_source": "%d SMs x 32 lanes/clk x %.0f MHz (%s clock)"
                                        % (nsm, sm_max_mhz, peak_src)},
            "roofline_hbm": {"bound": "hbm", "achieved": round(n / k_avg_s / 1e9, 2),
                             "peak": hbm_peak, "unit": "GB/s",
                             "frac": round(n / k_avg_s / 1e9 / hbm_peak, 5),
                             "peak_source": peak_src},
            "e2e": {"value": round(n * world / e2e_s / 1e9, 3), "unit": "GB/s",
                    "h2d_bytes_per_step": n, "d2h_bytes_per_step": 12,
                    "api": "dfa_match (pinned host buffer)", "h2d_copy_gbs": round(h2d_gbs, 1),
                    "calls": e2e_steps, "statistic": "median call time",
                    "call_ms": [round(x * 1e3, 2) for x in e2e_calls]},
            "gpu_launches": d.num_kernels(n, num_chunks=w.num_chunks, boundary_window=bw,
                                          lookahead=la) * args.steps,
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                       "reasons": clk["reasons"], "samples": clk["samples"]},
            "result": {"final_state": fs, "accept": acc, "status": st},
            "parity": ({"oracle": "Algorithm 1 (C) on the whole input",
                        "timed_step": "equal", "e2e": "equal (%d calls)" % e2e_steps}
                       if expect is not None else None),
        }
        if expect is not None:
            line["cpu_baseline"] = {"value": round(n / t_oracle / 1e9, 4), "unit": "GB/s",
                                    "cores": 1, "kind": "oracle",
                                    "sample": "the whole %d MiB input, one run of Algorithm 1 (C, "
                                              "one core); the same run checks the answers"
                                              % (n >> 20)}
        if world == 1:
            # measured lookup roofs: the unit of work alone on this DFA's table
            # (shared memory) and on a 256-class, 1288-state table read through L2
            import gen
            l2d = dm.Dfa.from_spec(gen.class_dfa(81, 1288, 256, 0.02, 0.3, 12, "byte"))
            r_smem = dm.probe_lookup_rate(d, 4096, stream)
            r_l2 = dm.probe_lookup_rate(l2d, 1024, stream)
            l2d.close()
            line["lookup_probe"] = {
                "smem_glookup_s": round(r_smem / 1e9, 1),
                "smem_vs_derived_peak": round(r_smem / lookup_peak, 4),
                "l2_glookup_s": round(r_l2 / 1e9, 1),
                "what": "dfa_probe_lookup_rate: 8 dependent chains per thread on the DFA's own "
                        "table (%s table in shared memory) and on a 659 KB table read through "
                        "L2 (256 classes x 1288 states), full-GPU launch, no staging" % w.name}
            line["roofline"]["frac_of_probe"] = round(achieved / r_smem, 4)
        if not args.no_mix and args.workload in ("regex", "protein") and world == 1:
            tune = not args.tuning and not args.no_tune
            legs = {}
            for r in (2, 4):   # r-symbol reverse lookahead (Eq. 13): smaller sets
                legs[r], _ = single_leg(dm, torch, d, dev, n, stream, 5, r=r, tune=tune,
                                        expect=expect)
                with_work(legs[r], dm, d, dev, n, lookup_peak)
            line["lookahead"] = {"r%d" % r: legs[r] for r in (2, 4)}
            # Algorithm 2 (every chunk from all of Q) on a prefix of the input
            n0 = min(n, 256 << 20)
            pre = dev[:n0]
            e0 = None if expect is None else oracle_answer(w.spec, w.data[:n0])[0]
            a2, _ = single_leg(dm, torch, d, pre, n0, stream, 3, r=0, tune=tune,
                               tune_len=n0, expect=e0)
            W0 = with_work(a2, dm, d, pre, n0, lookup_peak)
            a2["input_bytes"] = n0
            line["algorithm2"] = a2
            # the time model of Eqs. 14-18 beside the measurements (per input byte)
            head = {"kernel_ms": round(k_avg_s * 1e3, 4), "lookups_per_byte": W / n,
                    "mean_set": mean_I, "lookahead": 1}
            per_byte = {0: (a2["kernel_ms"] / n0, W0 / n0), 1: (head["kernel_ms"] / n, W / n)}
            for r in (2, 4):
                per_byte[r] = (legs[r]["kernel_ms"] / n, legs[r]["lookups_per_byte"])
            q_all = w.spec.num_states + 1 - int(info.num_excluded)
            mv = {}
            for r, (t_b, wpb) in sorted(per_byte.items()):
                mv["r%d" % r] = {
                    "m_static": q_all if r == 0 else (int(info.i_max) if r == 1 else None),
                    "lookups_per_byte": round(wpb, 3),
                    "pred_speedup_vs_alg2_static": (round(q_all / int(info.i_max), 3) if r == 1
                                                    else (1.0 if r == 0 else None)),
                    "pred_speedup_vs_alg2_sets": round(per_byte[0][1] / wpb, 3),
                    "measured_speedup_vs_alg2": round(per_byte[0][0] / t_b, 3),
                    "pred_kernel_ms_per_gib_at_roof": round(wpb * (1 << 30) / lookup_peak * 1e3, 3),
                    "measured_kernel_ms_per_gib": round(t_b * (1 << 30), 3),
                }
            line["model_vs_measured"] = {
                "model": "Eqs. 14-16: with P >> m the time is proportional to n*m, m = |Q| "
                         "(Algorithm 2) or the lookahead set size (Algorithm 3, Eq. 13); Eq. 18 "
                         "over Eq. 15 gives the speedup |Q|/I_max (static sets) or the work "
                         "ratio with the chunks' actual sets; the roof time is lookups / "
                         "(SMs x 32 x clock)",
                "legs": mv}
            # several DFAs on one input (Sec. 5: one symbol-index input run by
            # several DFAs): one batched launch against one launch per DFA
            if args.workload == "regex":
                import gen
                specs = [w.spec] + [sp for sp in gen.batch_dfas(21, 16)
                                    if sp.byte_to_symbol is None][:7]
                many = [dm.Dfa.from_spec(sp) for sp in specs]
                n1 = min(n, 256 << 20)
                bl1, res1, resp1 = batched_leg(dm, torch, many, [dev[:n1]] * len(many), reps=5)
                exp1, t1s, thr1 = oracle_answers_all_cores(specs, list(range(len(specs))),
                                                           [w.data[:n1]] * len(specs))
                assert [_as_answer(r) for r in res1] == exp1 == [_as_answer(r) for r in resp1], \
                    "several-DFA answers differ from the oracle"
                bl1.update(workload="%d DFAs (regex512 and %d byte DFAs of the batched mix, |Q| %s) "
                                    "on the first %d MiB of the input"
                                    % (len(specs), len(specs) - 1,
                                       sorted(sp.num_states for sp in specs), n1 >> 20),
                           oracle_match="all %d tests" % len(specs))
                line["several_dfas_one_input"] = bl1
                for x in many:
                    x.close()
            # Sec. 4.2 placement (opt-in; not the contracted method)
            if bw == 0:
                pl = {}
                for r in (1, 4):
                    pl["r%d" % r], _ = single_leg(dm, torch, d, dev, n, stream, 5, r=r, win=256,
                                                  tune=tune, expect=expect)
                    with_work(pl["r%d" % r], dm, d, dev, n, lookup_peak)
                line["placement"] = {"note": OUTSIDE, **pl}
            else:
                e67, _ = single_leg(dm, torch, d, dev, n, stream, 5, tune=tune, expect=expect)
                with_work(e67, dm, d, dev, n, lookup_peak)
                line["eqs_6_7"] = {"r1": e67}
        del dev, ws, out
        d.close()
        _free(torch)
        if not args.no_configs and args.workload == "regex" and world == 1:
            cfg = {}
            cfg["plain16_4MiB"] = plain16_config(args, dm, torch, lookup_peak)
            _free(torch)
            cfg["protein1288_%s" % ("10GB" if args.protein_bytes == 10 * 10**9
                                    else "%dB" % args.protein_bytes)] = \
                protein_config(args, dm, torch, lookup_peak, args.protein_bytes)
            _free(torch)
            grp = group_config(args, dm, torch, lookup_peak)
            cfg[grp["workload"]] = grp
            _free(torch)
            bl, state = batch_config(args, dm, torch)
            cfg["batched_cfg4"] = bl
            cfg["serving_cfg5"] = serve_config(args, dm, torch, state, bl["gbs"])
            line["configs"] = cfg
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
