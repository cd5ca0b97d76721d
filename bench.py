"""Benchmark: text GB/s of exact multiple pattern matching (MAG) on GB300.

One step = one search over the whole text: the fused encode + AOSO Shift-Or
scan, verification, the occurrence count and the sort of the occurrence
list.  The default workload is uniform DNA at 1 GiB with r = 100 patterns of
length m = 16, half planted (the 1 MiB DNA configuration's distribution and
pattern shape at a text larger than the 129 MB L2, so no flush is needed
between steps); the filter's parameters come from the autotuner, which
times MAG's non-overlapping q-grams and Section 2's overlapping ones.

The default run (one GPU) adds the other configurations to the same line
under "other_configs", each in a bounded form: the 1 MiB DNA search as
stated (L2 flushed before every search), the protein-like workload, the
large pattern sets, the batch of 4096 texts (batched + learned against the
plain per-request form) and the cost model's regret timed live.

Prints one JSON line.  --impl reference times the oracle (textbook
Aho-Corasick in C, threaded) on the host cores instead.
Multi-GPU: launched under torchrun, every rank searches its own text
(weak scaling); rank 0 prints the aggregate.
"""
import argparse
import json
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "text GB/s scanned (bit-exact), % of HBM peak; batched+learned vs plain form"

WORKLOADS = {
    # name: (generator, sigma, description)
    "protein-256MiB": ("config2", 20,
                       "protein-like text 256 MiB, 20 symbols Zipf s=0.8, r=1000, m=32, "
                       "half planted"),
    "dna-1GiB": ("config1_scaled", 4,
                 "uniform DNA text 1 GiB, r=100, m=16, half planted (config-1 shape at scale)"),
    "dna-1MiB": ("config1", 4, "uniform DNA text 1 MiB, r=100, m=16, half planted"),
    # the same at 256 MiB: still larger than L2, small enough for a full
    # profiler capture of the scan
    "dna-256MiB": ("config1_scaled", 4, "uniform DNA text 256 MiB, r=100, m=16, half planted",
                   {"n": 1 << 28}),
    "protein-256MiB-varlen": ("config2_varlen", 20,
                              "protein-like text 256 MiB, r=1000 patterns of lengths 16..64, "
                              "half planted (filter on the 16-byte prefixes)"),
    # large pattern sets on uniform DNA: the verification-heavy regime
    "dna-1GiB-r100k": ("config3", 4, "uniform DNA text 1 GiB, r=100,000, m=32, 10% planted"),
    "dna-1GiB-r10k-m16": ("config3", 4, "uniform DNA text 1 GiB, r=10,000, m=16, 10% planted",
                          {"r": 10_000, "m": 16}),
    "dna-1GiB-r10k-m64": ("config3", 4, "uniform DNA text 1 GiB, r=10,000, m=64, 10% planted",
                          {"r": 10_000, "m": 64}),
}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """SM clocks and clock-event (throttle) reasons of the benchmarked GPU,
    read through NVML every 5 ms on a background thread while the timed
    region runs (nvidia-smi's 200 ms period is longer than a short region)."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_index, period=0.005):
        import threading
        self.period = period
        self.samples = []
        self.max_mhz = None
        self.handle = None
        self._stop = threading.Event()
        self._thread = None
        try:
            import ctypes
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            bus = None
            try:
                import torch
                pr = torch.cuda.get_device_properties(torch_index)
                bus = "%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
            except Exception:
                bus = None
            ok = bus is not None and nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(),
                                                                         ctypes.byref(h)) == 0
            if not ok and nv.nvmlDeviceGetHandleByIndex_v2(torch_index, ctypes.byref(h)) != 0:
                return
            self.nv, self.handle, self.ct = nv, h, ctypes
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = mx.value
        except Exception:
            self.handle = None

    def sample(self):
        ct = self.ct
        mhz, reasons = ct.c_uint(), ct.c_ulonglong()
        if self.nv.nvmlDeviceGetClockInfo(self.handle, 1, ct.byref(mhz)) != 0:
            return
        if self.nv.nvmlDeviceGetCurrentClocksEventReasons(self.handle, ct.byref(reasons)) != 0:
            self.nv.nvmlDeviceGetCurrentClocksThrottleReasons(self.handle, ct.byref(reasons))
        self.samples.append((mhz.value, reasons.value))

    def _run(self):
        while not self._stop.is_set():
            self.sample()
            self._stop.wait(self.period)

    def __enter__(self):
        if self.handle is not None:
            import threading
            self.sample()
            self._thread = threading.Thread(target=self._run, daemon=True)
            self._thread.start()
        return self

    def __exit__(self, *a):
        if self._thread is not None:
            self._stop.set()
            self._thread.join()
            self.sample()

    def summary(self):
        if not self.samples:
            return None
        reasons = set()
        for _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(m for m, _ in self.samples),
                "sm_max_mhz": self.max_mhz, "reasons": sorted(reasons),
                "samples": len(self.samples), "source": "nvml"}


def make_case(name):
    from paper_1405_5483_gb300 import workloads as W
    gen, sigma, desc = WORKLOADS[name][:3]
    kwargs = WORKLOADS[name][3] if len(WORKLOADS[name]) > 3 else {}
    return getattr(W, gen)(**kwargs), sigma, desc


def cpu_baseline(case, sample_bytes):
    """The oracle (Aho-Corasick, C, all host cores) on the first sample_bytes."""
    from oracle import native
    threads = os.cpu_count() or 1
    n = min(case.n, sample_bytes)
    T = np.ascontiguousarray(case.T[:n])
    ac = native.AhoCorasick(case.P)
    t0 = time.perf_counter()
    pos, _ = ac.search(T, threads=threads)
    dt = time.perf_counter() - t0
    ac.close()
    return {"value": n / dt / 1e9, "unit": "GB/s", "cores": threads, "kind": "oracle",
            "sample": "first %d MiB of the text, all %d patterns, Aho-Corasick over %d threads "
                      "(%.2f s, %d occurrences)" % (n >> 20, case.r, threads, dt, pos.size)}


class OracleBatchSample:
    """The oracle on the batch workload: one Aho-Corasick automaton per
    pattern set, each text searched with its set's automaton, over the first
    texts (in text order) up to `budget` bytes."""

    def __init__(self, b, budget):
        from oracle import native
        self.b = b
        self.threads = os.cpu_count() or 1
        self.picked, self.total = [], 0
        for t, T in enumerate(b.texts):
            if self.total >= budget:
                break
            self.picked.append(t)
            self.total += T.size
        sets = sorted(set(int(b.set_of_text[t]) for t in self.picked))
        self.acs = {s: native.AhoCorasick(b.sets[s]) for s in sets}

    def step(self):
        z = 0
        for t in self.picked:
            pos, _ = self.acs[int(self.b.set_of_text[t])].search(self.b.texts[t],
                                                                  threads=self.threads)
            z += pos.size
        return z

    def describe(self):
        return ("the first %d texts (%d MiB), each with its set's Aho-Corasick automaton over "
                "%d threads" % (len(self.picked), self.total >> 20, self.threads))

    def close(self):
        for ac in self.acs.values():
            ac.close()


def run_reference_batch(args):
    """The oracle on the batch workload over a bounded sample of the texts
    per step."""
    from paper_1405_5483_gb300 import workloads as W
    b = W.config4()
    budget = max(4 << 20, min(args.ref_sample_mib << 20, (2 << 30) // max(1, args.steps)))
    o = OracleBatchSample(b, budget)
    for _ in range(args.warmup):
        o.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step()
    dt = time.perf_counter() - t0
    value = o.total * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "batch-4096", "texts": len(o.picked), "bytes": o.total},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": o.threads, "kind": "oracle",
                         "sample": o.describe()},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    o.close()
    print(json.dumps(line))


def run_reference(args, rank):
    if rank != 0:
        return
    if args.workload == "batch-4096":
        return run_reference_batch(args)
    case, sigma, desc = make_case(args.workload)
    # per-step sample: at most 64 MiB, and about 2 GiB over all steps, so
    # that the whole run stays within a few minutes on the host cores
    sample = max(4 << 20, min(args.ref_sample_mib << 20, (2 << 30) // max(1, args.steps)))
    from oracle import native
    threads = os.cpu_count() or 1
    ac = native.AhoCorasick(case.P)
    n = min(case.n, sample)
    T = np.ascontiguousarray(case.T[:n])
    for _ in range(args.warmup):
        ac.search(T, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ac.search(T, threads=threads)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n": n, "r": case.r,
                   "m": case.m},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": "first %d MiB of the text per step, Aho-Corasick over %d "
                                   "threads" % (n >> 20, threads)},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_batch(args, rank, steps=None, fast=False):
    """Config 4: 4096 texts (1 KiB - 4 MiB, printable Zipf text) against 64
    pattern sets.  Plain form: one mpm_search per text, each set's
    parameters tuned by the autotuner on a sample of its texts.  Batched
    forms: one persistent launch replayed from a CUDA graph, with each set's
    parameters proposed by the learned cost model (the headline) or picked by
    the exhaustive autotuner timing the batched kernel on a sample of the
    set's texts.  All forms produce the same occurrences, checked.  Returns
    the JSON line (fast: smaller tuning budgets)."""
    import torch
    import paper_1405_5483_gb300 as mpm
    from paper_1405_5483_gb300 import _native as mpm_native
    from paper_1405_5483_gb300 import cost_model as CM
    from paper_1405_5483_gb300 import workloads as W
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    b = W.config4()
    gen_s = time.perf_counter() - t0
    # all texts in one device buffer (each at a 256-byte boundary), so that
    # the end-to-end run moves them with one host-to-device copy
    offs = np.zeros(len(b.texts) + 1, np.int64)
    for i, t in enumerate(b.texts):
        offs[i + 1] = (offs[i] + t.size + 255) & ~255
    flat = np.zeros(int(offs[-1]), np.uint8)
    for i, t in enumerate(b.texts):
        flat[offs[i]: offs[i] + t.size] = t
    dflat = torch.from_numpy(flat).to(dev)
    texts = [dflat[int(offs[i]): int(offs[i]) + t.size] for i, t in enumerate(b.texts)]
    total = b.total_bytes
    steps = max(1, steps or args.steps)
    # plain per-request form: each set's parameters tuned (mpm_search timed)
    # on up to 16 MiB of its texts (--no-tune: the automatic parameters)
    t0 = time.perf_counter()
    plain = []
    for sidx, P in enumerate(b.sets):
        mine = [texts[t] for t in np.flatnonzero(b.set_of_text == sidx)]
        sample = torch.cat(mine)[: 16 << 20] if mine else texts[0]
        best = {}
        if not args.no_tune:
            try:
                best, _ = mpm.autotune(P, b.sigma, sample, kernels=3, overlap=1,
                                       max_sets=8 if fast else 24, reps=2)
            except mpm.MpmError:
                best = {}
        plain.append(mpm.Matcher(P, sigma=b.sigma, **best))
    plain_tune_s = time.perf_counter() - t0
    cap = 1 << 20
    out_pos = torch.empty(cap, dtype=torch.int32, device=dev)
    out_pid = torch.empty(cap, dtype=torch.int32, device=dev)

    def plain_pass(collect=False):
        res = []
        for t, T in enumerate(texts):
            z = plain[b.set_of_text[t]].search_into(T, out_pos, out_pid)
            if collect and z:
                res.append(np.stack([np.full(z, t, np.uint32),
                                     out_pos[:z].cpu().numpy().view(np.uint32),
                                     out_pid[:z].cpu().numpy().view(np.uint32)], axis=1))
        return np.concatenate(res) if res else np.zeros((0, 3), np.uint32)

    def build(params):
        return mpm.Batch([CM.batch_matcher(P, b.sigma, p) for P, p in zip(b.sets, params)],
                         texts, b.set_of_text)

    def timed(B, label):
        for _ in range(max(3, args.warmup)):
            B.run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(label)
        e0.record()
        for _ in range(steps):
            B.run()
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        return e0.elapsed_time(e1) / steps

    def result(B):
        return np.stack([x.cpu().numpy().view(np.uint32) for x in B.run()], axis=1)

    want = plain_pass(collect=True)
    # batched + learned: the committed cost model proposes each set's parameters
    t0 = time.perf_counter()
    model = CM.Model.load()
    # mask tables that the batched kernel keeps in shared memory
    learned = CM.learned_batch_params(b, model, mpm_native.BATCH_SMEM_TABLE_BYTES)
    learn_s = time.perf_counter() - t0
    # the same parameters through the precompiled kernel (run-time q, k and
    # mapping), for comparison with the kernel compiled for the batch
    BG = mpm.Batch([CM.batch_matcher(P, b.sigma, p) for P, p in zip(b.sets, learned)],
                   texts, b.set_of_text, generic=True)
    exact_generic = bool(np.array_equal(result(BG), want))
    generic_ms = timed(BG, "batch_generic")
    BG.close()
    t0 = time.perf_counter()
    BL = build(learned)
    compile_s = time.perf_counter() - t0
    exact_learned = bool(np.array_equal(result(BL), want)) and exact_generic
    with ClockSampler(dev.index) as clk:
        learned_ms = timed(BL, "batch_timed")
    st = BL.stats
    launches = int(st["launches"]) * steps
    # the scan kernel alone: events on either side of it inside the graph
    scans = []
    for _ in range(10):
        BL.run()
        scans.append(BL.stats["scan_ms"])
    scan_ms = statistics.median(scans)
    BL.close()
    # batched + tuned: the exhaustive tuner on a sample of each set's texts
    t0 = time.perf_counter()
    tuned = []
    for sidx, P in enumerate(b.sets if not args.no_tune else []):
        mine = [texts[t] for t in np.flatnonzero(b.set_of_text == sidx)]
        sample = torch.cat(mine)[: 16 << 20] if mine else texts[0]
        try:
            best, _ = mpm.autotune(P, b.sigma, sample, kernels=8, max_positions=32,
                                   max_sets=12 if fast else 24, reps=2,
                                   max_table_kib=mpm_native.BATCH_SMEM_TABLE_BYTES >> 10)
        except mpm.MpmError:
            best = {}
        tuned.append(best)
    tune_s = time.perf_counter() - t0
    exact_tuned, tuned_ms = True, None
    if tuned:
        BT = build(tuned)
        exact_tuned = bool(np.array_equal(result(BT), want))
        tuned_ms = timed(BT, "batch_tuned")
        BT.close()

    plain_steps = max(1, min(3, steps))
    plain_pass()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(plain_steps):
        plain_pass()
    e1.record()
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / plain_steps

    # end to end: the texts from pinned host memory (one copy), the batched
    # run with the learned parameters, and its occurrence triples read back
    # to the host
    hflat = torch.empty(flat.size, dtype=torch.uint8, pin_memory=True)
    hflat.numpy()[:] = flat
    BL = build(learned)
    BL.run()
    e2e_steps = max(2, min(steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        dflat.copy_(hflat, non_blocking=True)
        torch.cuda.synchronize()  # the batch runs on its own stream
        got = [x.cpu() for x in BL.run()]
    e2e_s = time.perf_counter() - t0
    e2e_z = int(got[0].numel())
    BL.close()
    del hflat
    value = total / (learned_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    cpu = None
    if not args.no_cpu_baseline and not fast:
        o = OracleBatchSample(b, args.cpu_sample_mib << 20)
        t0 = time.perf_counter()
        oz = o.step()
        dt = time.perf_counter() - t0
        cpu = {"value": o.total / dt / 1e9, "unit": "GB/s", "cores": o.threads,
               "kind": "oracle", "sample": o.describe() + " (%.2f s, %d occurrences)" % (dt, oz)}
        o.close()
    # the dominant kernel (mpm_batch_jit, the kernel compiled for the batch,
    # or batch_scan_kernel when it could not be): algorithmic bytes per
    # launch = every text byte once (candidate records stay in shared memory;
    # the occurrence records it writes are a few hundred KB)
    achieved = total / (scan_ms * 1e-3) / 1e9 if scan_ms > 0 else None
    kname = "mpm_batch_jit" if st["variants"] else "batch_scan_kernel"
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": 1, "steps": steps,
        "warmup": max(3, args.warmup), "ms_per_step": learned_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "batch-4096", "texts": len(texts), "sets": len(b.sets),
                   "bytes": total, "form": "batched (one persistent launch, CUDA graph) of the "
                   "kernel compiled for the batch's %d parameter sets, parameters per set from "
                   "the learned cost model (mask tables that fit shared memory)" % st["variants"],
                   "l2": "inputs larger than L2 (no flush)"},
        "hbm_frac_of_%s_peak" % peak_kind: value / peak,
        "plain_per_request": {"value": total / (plain_ms * 1e-3) / 1e9, "unit": "GB/s",
                              "ms_per_step": plain_ms,
                              "form": "one mpm_search per text, each set's parameters "
                                      + ("automatic" if args.no_tune else
                                         "from the autotuner (mpm_search timed on up to 16 "
                                         "MiB of its texts)")},
        "batched_tuned": None if tuned_ms is None else {
            "value": total / (tuned_ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": tuned_ms,
            "form": "batched, parameters from the exhaustive autotuner (the compiled batched "
                    "kernel timed on 16 MiB of each set's texts)"},
        "batched_precompiled_kernel": {"value": total / (generic_ms * 1e-3) / 1e9, "unit": "GB/s",
                                       "ms_per_step": generic_ms,
                                       "form": "the learned parameters through the precompiled "
                                               "batched kernel (run-time q, k and mapping)"},
        "batched_over_plain": plain_ms / learned_ms,
        "learned_over_tuned": None if tuned_ms is None else tuned_ms / learned_ms,
        "bit_exact_vs_plain": exact_learned and exact_tuned, "occurrences": int(st["z"]),
        "candidates_per_step": int(st["candidates"]),
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None,
                     "traffic": recorded_traffic("batch-4096", {}, kname,
                                                 batch_kernel_rev(kname)),
                     "kernel": kname, "peak_kind": peak_kind, "scan_ms": scan_ms},
        "e2e": {"value": total * e2e_steps / e2e_s / 1e9, "unit": "GB/s",
                "h2d_bytes_per_step": int(flat.size),
                "d2h_bytes_per_step": 16 + 12 * e2e_z},
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "setup_seconds": {"generate": round(gen_s, 1), "learned_choice": round(learn_s, 1),
                          "compile_batch_kernel": round(compile_s, 1),
                          "tune": round(tune_s, 1), "tune_plain": round(plain_tune_s, 1)},
    }
    for mm in plain:
        mm.close()
    del dflat, texts
    torch.cuda.empty_cache()
    return line


def search_line(args, name, dev, world=1, params=None, tune_sets=None, steps=None,
                e2e=True, cpu=True):
    """One workload through the single-text API (mpm_build, mpm_search_async /
    mpm_search): parameters from the autotuner (both q-gram families) unless
    given, pipelined searches timed back to back (a text that fits in L2:
    each search after an L2 flush), the synchronous form beside them, the end
    to end run from pinned host memory and the oracle's CPU baseline.
    Returns the JSON line's keys; every rank returns its own timings, the
    maximum over ranks is taken here."""
    import torch
    import torch.distributed as dist
    import paper_1405_5483_gb300 as mpm

    case, sigma, desc = make_case(name)
    T = torch.from_numpy(case.T).to(dev)
    tuning = None
    if params is None:
        params = {}
        if args.params:
            params = parse_params(args.params)
        elif not args.no_tune:
            # exhaustive autotuner on a sample of the text; not timed, like the build
            sample = T[: min(case.n, args.tune_sample_mib << 20)]
            t0 = time.perf_counter()
            # patterns of different lengths: the filter's parameters are tuned on
            # their common-length prefixes
            params, sets = mpm.autotune(case.prefix_matrix(), sigma, sample, kernels=3,
                                        max_sets=tune_sets or args.tune_sets, overlap=1)
            tuning = {"sample_bytes": int(sample.numel()), "sets_timed": len(sets),
                      "seconds": round(time.perf_counter() - t0, 2)}
    m = mpm.Matcher(case.P, sigma=sigma, **params)
    m.set_timing(True)
    cap = max(1 << 16, 8 * case.r)
    out_pos = torch.empty(cap, dtype=torch.int32, device=dev)
    out_pid = torch.empty(cap, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    # one synchronous search sizes the handle's buffers and gives the count
    z = m.search_into(T, out_pos, out_pid)
    steps = max(1, steps or args.steps)
    status = torch.zeros((steps, 4), dtype=torch.int32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # a text that fits in L2 would be timed warm: then L2 is flushed (a write
    # of twice its size) before every timed search, outside the search's events
    l2 = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or 129 * 10**6)
    flush = torch.empty(2 * l2, dtype=torch.uint8, device=dev) if case.n < l2 else None

    def timed_flushed(k, search):
        """k searches, each after an L2 flush, each timed alone; the sum."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k)]
        barrier()
        for i, (a, b) in enumerate(evs):
            flush.zero_()
            a.record(stream)
            search(i)
            b.record(stream)
        barrier()
        return sum(a.elapsed_time(b) for a, b in evs)

    def pipelined_step(i):
        m.search_async(T, out_pos, out_pid, status[i])
        m.join()  # its closing sort belongs to the step

    def timed_pipelined():
        """Searches issued back to back (mpm_search_async), each writing its
        own status row; the stream never waits for the host."""
        for _ in range(max(3, args.warmup)):
            m.search_async(T, out_pos, out_pid, status[0])
        m.sync()
        m.reset_stats()
        if flush is not None:
            with ClockSampler(dev.index) as clk:
                ms = timed_flushed(steps, pipelined_step)
            m.sync()
            return ms, clk
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev.index) as clk:
            barrier()
            ev0.record(stream)
            for i in range(steps):
                m.search_async(T, out_pos, out_pid, status[i])
            m.join()  # the last searches' closing sorts belong to the timed region
            ev1.record(stream)
            barrier()
        m.sync()
        return ev0.elapsed_time(ev1), clk

    def timed_sync(k):
        """The same searches, one synchronous mpm_search call each."""
        for _ in range(max(3, args.warmup)):
            m.search_into(T, out_pos, out_pid)
        if flush is not None:
            return timed_flushed(k, lambda i: m.search_into(T, out_pos, out_pid))
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        for _ in range(k):
            m.search_into(T, out_pos, out_pid)
        ev1.record(stream)
        barrier()
        return ev0.elapsed_time(ev1)

    elapsed_ms, clk = timed_pipelined()
    st = m.stats
    rows = status.cpu().numpy()
    pipelined_ok = bool(np.all(rows[:, 3] == 1) and np.all(rows[:, 1] == z) and
                        np.all(rows[:, 2] == 0))
    scan_avg = st["ms_scan"] / steps
    verify_avg = st["ms_verify"] / steps
    launches = int(st["launches"])
    candidates = int(rows[:, 0].mean())
    sync_steps = min(steps, 100)
    sync_ms = timed_sync(sync_steps)
    if not pipelined_ok:
        # a search the pipelined call does not finish by itself: the
        # synchronous form is the step
        with ClockSampler(dev.index) as clk:
            elapsed_ms = timed_sync(steps)
        st = m.stats
        scan_avg, verify_avg = st["ms_scan"], st["ms_verify"]
        launches = int(st["launches"]) * steps
        candidates = int(st["candidates"])
    if world > 1:
        t = torch.tensor([elapsed_ms, sync_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms, sync_ms = float(t[0].item()), float(t[1].item())
    value = case.n * steps * world / (elapsed_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()

    e2e_line = None
    if e2e:
        # end to end through the public API with host buffers: pinned host
        # text, host outputs, copies inside the timed region
        hT = torch.from_numpy(case.T).pin_memory()
        hpos = np.empty(cap, np.uint32)
        hpid = np.empty(cap, np.uint32)
        e2e_steps = max(2, min(args.steps, 5))
        m.search_into(hT, hpos, hpid)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ze = m.search_into(hT, hpos, hpid)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_line = {"value": case.n * e2e_steps * world / e2e_s / 1e9, "unit": "GB/s",
                    "h2d_bytes_per_step": case.n, "d2h_bytes_per_step": 16 + 8 * ze}
        del hT

    # the dominant kernel: the scan.  Algorithmic bytes per launch = the
    # text read once plus, when the scan writes candidate records to HBM (the
    # split and generic kernels), 8 bytes per record.
    p = m.params
    fused = bool(p["kernel"] == mpm.KERNEL_SPECIALISED)
    algo_bytes = case.n + (0 if fused else 8 * candidates)
    achieved = algo_bytes / (scan_avg * 1e-3) / 1e9
    if st["specialised"]:
        kname = "mpm_scan_jit (specialised%s)" % (", overlapping q-grams" if p["overlap"] else "")
    else:
        kname = ("scan_overlap_kernel (generic, overlapping q-grams)" if p["overlap"]
                 else "scan_tma_kernel (generic)")
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
        "steps": steps, "warmup": max(3, args.warmup),
        "ms_per_step": elapsed_ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": name, "description": desc, "n": case.n,
                   "r": case.r, "m": case.m, "params": p, "tuning": tuning,
                   "l2": ("inputs larger than L2 (no flush)" if flush is None else
                          "text smaller than L2: L2 flushed (a %d-byte write) before "
                          "every timed search, outside its events" % (2 * l2)),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "hbm_frac_of_%s_peak" % peak_kind: value / peak,
        "form": ("pipelined: mpm_search_async back to back, every step's status checked "
                 "(complete, z as the synchronous search)" if pipelined_ok else
                 "synchronous mpm_search per step"),
        "sync_per_call": {"value": case.n * sync_steps * world / (sync_ms * 1e-3) / 1e9,
                          "unit": "GB/s", "ms_per_step": sync_ms / sync_steps,
                          "form": "one synchronous mpm_search per step"},
        "occurrences": z,
        "candidates_per_step": candidates,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(name, p),
                     "kernel": kname, "peak_kind": peak_kind, "scan_ms": scan_avg,
                     "verify_ms": verify_avg},
        "e2e": e2e_line,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "cpu_baseline": None,
    }
    if cpu and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(case, args.cpu_sample_mib << 20)
    m.close()
    del T, out_pos, out_pid, status, flush
    torch.cuda.empty_cache()
    return line


def run_regret(args, dev, nsets=50):
    """Config 5 measured live: for each of the first nsets held-out pattern
    sets of the cost model's data (config-4-shaped, never trained on), every
    point of the model's grid is timed with the batched kernel (the
    autotuner's grid mode: the whole GPU busy, the set's text repeated to at
    least 128 MiB, median device time); the model's choice is the grid point
    of least predicted time, its regret t(choice) / t(best) - 1 in the same
    timing; the library's default parameters are timed the same way."""
    import torch
    import paper_1405_5483_gb300 as mpm
    from paper_1405_5483_gb300 import cost_model as CM
    from paper_1405_5483_gb300 import workloads as W
    model = CM.Model.load()
    regrets, gains, points = [], [], 0
    t0 = time.perf_counter()
    for idx in list(CM.HELDOUT_SETS)[:nsets]:
        case = W.config5_set(idx)
        T = torch.from_numpy(case.T).to(dev)
        ent = CM.entropy_bits(case.T)
        _, entries = mpm.autotune(case.P, case.sigma, T, kernels=8, grid=1, max_positions=32,
                                  reps=3)
        ok = [e for e in entries if e["status"] == 0 and e["ms"] > 0]
        if not ok:
            continue
        points += len(ok)
        ms = np.array([e["ms"] for e in ok])
        pred = model.predict(CM.features(case.sigma, ent, case.m, case.r, case.n,
                                         [e["params"] for e in ok]))
        pick = float(ms[int(np.argmin(pred))])
        regrets.append(pick / float(ms.min()) - 1.0)
        dp = CM.default_params(case.P, case.sigma)
        if dp:
            gains.append(CM.time_batched(case.P, case.sigma, T, dp, reps=3) / pick)
        del T
    regrets = np.array(regrets)
    return {
        "sets": int(regrets.size), "grid_points_timed": points,
        "mean_regret": float(regrets.mean()) if regrets.size else None,
        "median_regret": float(np.median(regrets)) if regrets.size else None,
        "p90_regret": float(np.quantile(regrets, 0.9)) if regrets.size else None,
        "geomean_speedup_over_default":
            float(np.exp(np.mean(np.log(gains)))) if gains else None,
        "form": "held-out cost-model sets %d.. (config-4 shape), every grid point timed live "
                "with the batched kernel; regret of the model's least-predicted point "
                "against the best timed point" % CM.HELDOUT_SETS.start,
        "target": "mean regret <= 0.05",
        "timing_seconds": round(time.perf_counter() - t0, 1),
    }


# The configurations measured, each in a bounded form, beside the headline
# workload in the default run (one GPU): config 1 as stated, the protein
# workload, the large pattern sets, the batch and the cost model's regret.
OTHER_CONFIGS = ("dna-1MiB", "protein-256MiB", "dna-1GiB-r100k", "dna-1GiB-r10k-m16",
                 "dna-1GiB-r10k-m64", "batch-4096", "learned-regret")


def summary_of(line):
    """The keys of a workload's line that the default run repeats for it."""
    keep = ("value", "unit", "ms_per_step", "steps", "hbm_frac_of_measured_peak",
            "hbm_frac_of_fallback_peak", "form", "occurrences", "candidates_per_step",
            "roofline", "sync_per_call", "plain_per_request", "batched_tuned",
            "batched_over_plain", "learned_over_tuned", "bit_exact_vs_plain", "clocks",
            "batched_precompiled_kernel",
            "gpu_launches", "setup_seconds")
    out = {k: line[k] for k in keep if k in line}
    out["config"] = line.get("config")
    return out


def other_configs(args, dev):
    """The other configurations, each timed as its own workload with fewer
    steps and a smaller tuning budget; a failure is recorded, not raised."""
    import torch
    sub = argparse.Namespace(**vars(args))
    sub.params = ""
    out = {}
    for name in OTHER_CONFIGS:
        t0 = time.perf_counter()
        try:
            if name == "batch-4096":
                res = summary_of(run_batch(sub, 0, steps=min(args.steps, 10), fast=True))
            elif name == "learned-regret":
                res = run_regret(sub, dev, nsets=args.regret_sets)
            else:
                res = summary_of(search_line(sub, name, dev, tune_sets=16,
                                             steps=min(args.steps, 20), e2e=False, cpu=False))
        except Exception as e:  # recorded in the line
            res = {"error": ("%s: %s" % (type(e).__name__, e))[:400]}
        res["seconds"] = round(time.perf_counter() - t0, 1)
        out[name] = res
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dna-1GiB",
                    choices=sorted(WORKLOADS) + ["batch-4096"])
    ap.add_argument("--main-only", action="store_true",
                    help="skip the other configurations of the default run")
    ap.add_argument("--cpu-sample-mib", type=int, default=256)
    ap.add_argument("--ref-sample-mib", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--tune-sample-mib", type=int, default=256)
    ap.add_argument("--params", default="", help="JSON filter parameters; skips tuning")
    ap.add_argument("--tune-sets", type=int, default=48)
    ap.add_argument("--regret-sets", type=int, default=50)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "batch-4096":
        line = run_batch(args, rank)
        if rank == 0:
            print(json.dumps(line))
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    line = search_line(args, args.workload, dev, world=world)
    default_run = (args.workload == "dna-1GiB" and not args.params and not args.main_only)
    if rank == 0 and world == 1 and default_run:
        line["other_configs"] = other_configs(args, dev)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def parse_params(text):
    """Filter parameters from JSON or from a list like q=5,sigma_r=65536,k=1."""
    text = text.strip()
    if text.startswith("{"):
        return json.loads(text)
    out = {}
    for item in filter(None, text.split(",")):
        k, v = item.split("=", 1)
        out[k.strip()] = int(v)
    return out


def source_rev(files):
    """A hash of kernel sources, to tie DRAM counters recorded under
    profiles/ to the code that made them."""
    import hashlib
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_1405_5483_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def kernel_rev():
    """The specialised scan kernel's source and launch geometry."""
    return source_rev(("keyhash.h", "multiword.h", "scan_jit_args.h", "ptx_common.cuh",
                       "window_check.cuh", "jit_types.h", "scan_stage.cuh", "scan_jit.cuh",
                       "jit.cpp"))


def batch_kernel_rev(kernel="batch_scan_kernel"):
    """A batched kernel's source and its host side (units, launch)."""
    if kernel == "mpm_batch_jit":
        return source_rev(("batch.cu", "batch_args.h", "batch_lane.cuh", "batch_jit.cuh",
                           "scan_stage.cuh", "jit_types.h", "jit.cpp", "window_check.cuh",
                           "keyhash.h", "ptx_common.cuh", "multiword.h"))
    return source_rev(("batch.cu", "batch_args.h", "stepper.cuh", "multiword.h",
                       "device_common.cuh", "window_check.cuh", "keyhash.h"))


def recorded_traffic(workload, params, profile="mpm_scan_jit", rev=None):
    """DRAM bytes per launch of the dominant kernel from the ncu summary of
    this workload, when it was taken on the current kernel with these
    parameters.  The summary lists `kernel_rev` once and one `record` line
    (JSON with params and traffic_bytes_per_launch) per captured parameter
    set."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (profile, workload))
    if not os.path.exists(path):
        return None
    found, records = None, []
    for line in open(path):
        if not line.startswith("- `"):
            continue
        key, rest = line[3:].split("`", 1)
        val = rest.split(":", 1)[1].strip().strip("`") if ":" in rest else ""
        if key == "kernel_rev":
            found = val
        elif key == "record":
            try:
                records.append(json.loads(val))
            except ValueError:
                pass
    if found != (rev if rev is not None else kernel_rev()):
        return None
    for rec in records:
        if all(params.get(k) == v for k, v in rec.get("params", {}).items()):
            try:
                return int(rec["traffic_bytes_per_launch"])
            except (KeyError, ValueError, TypeError):
                return None
    return None


if __name__ == "__main__":
    main()
