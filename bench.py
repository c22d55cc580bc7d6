#!/usr/bin/env python
"""Benchmark of the CV-QKD slice-reconciliation hot path on B300.

Workload (the block-size sweep): one long block of 2^27 Gaussian quadrature
pairs at SNR 3 and at SNR 15 (x ~ N(0,1), y = x + N(0, 1/SNR)), Bob's 5-slice
Gray quantiser on [-4 sigma_y, 4 sigma_y], the block subdivided into
sub-blocks of n = 2^12 .. 2^20 (F = 2^27 / n frames per slice), one seeded
left-regular dv = 3 code per (SNR, n, slice) at 0.95 x the slice's
conditional capacity rounded to 1/64 (slices with rate 0 are disclosed),
syndrome-based FP32 sum-product with flooding schedule, at most 100
iterations, per-frame early stop.  One step = the whole reverse
reconciliation of every (SNR, n) point: quantise + syndromes (Bob), then per
slice the LLR from x and the already reconciled lower slices and the decode
of all sub-blocks (Alice).

value = reconciled key bits / s: bits of decoded (non-disclosed) slices in
sub-blocks whose decoded word equals Bob's, summed over all points and ranks,
divided by the device time of the step (inputs resident in HBM).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

N_SAMPLES = 1 << 27
SNRS = (3.0, 15.0)
DATA_SEED = {3.0: 2, 15.0: 3}
LOGNS = (12, 14, 16, 18, 20)
M_SLICES = 5
MAX_ITER = 100
WORKLOAD = ("block-size sweep: 2^27 samples at SNR 3 and 15, 5 Gray slices, sub-blocks n = 2^12..2^20, "
            "dv=3 codes at 0.95 x slice capacity, FP32 sum-product flooding, <= 100 iterations, early stop")
RATES_BACKOFF = ("dv=3 codes at the Sec. V-B back-off rates (per SNR, n and slice: start 0.95 x slice capacity, "
                 "minus 3/64 while > 1 of 32 trial frames fail; below 0.10: disclosed; table in sweep_rates.json)")


def sweep_workload(rate_rule):
    """The sweep's workload line for the rate rule in use (reconciled bits at a fixed
    FER target with the back-off rates)."""
    return WORKLOAD if rate_rule != "backoff" else WORKLOAD.replace("dv=3 codes at 0.95 x slice capacity",
                                                                      RATES_BACKOFF)


# iterations after which the FP32 flooding decoders re-pack their decoding
# frames (the library's fixed schedule)
REPACK_AT = (16, 32, 64)


def block_work(t, sched, B=32):
    """Frame-iterations that 32-frame blocks occupy for frames taking t[f] check
    passes, re-packed densely (in their order) after each iteration in sched."""
    work, cur = 0, np.asarray(t)
    for it in range(1, int(cur.max()) + 1 if cur.size else 1):
        if it - 1 in sched:
            cur = cur[cur >= it]
        pad = (-cur.size) % B
        tb = np.concatenate([cur, np.zeros(pad, dtype=cur.dtype)]).reshape(-1, B)
        work += int((tb >= it).any(axis=1).sum()) * B
    return work


def code_seed(logn, j):
    return 2000 + 100 * logn + j


def rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ------------------------------------------------------------------ set-up
def slice_rates(snr, capacity_fn):
    """Capacities and 0.95 x capacity rates of the sweep's slices (library calls)."""
    import paper_2108_08418_b300 as q
    lo, hi = q.qkdrec_quantiser_range(snr)
    caps = [capacity_fn(snr, M_SLICES, j, lo, hi) for j in range(M_SLICES)]
    return caps, [q.qkdrec_code_rate(c) for c in caps]


def _make_code(args):
    logn, j, rate, by_rate = args
    n = 1 << logn
    M = synth.checks_for_rate(n, rate)
    seed = uneven_code_seed(n, rate) if by_rate else code_seed(logn, j)
    rp, ci, res = synth.make_regular_code(seed, n, M)
    return (logn, j, rate), (rp, ci, res, seed)


def build_codes(jobs, workers, by_rate=False):
    """Construct the parity-check matrices in a spawn pool (before any CUDA use)."""
    import multiprocessing as mp
    out = {}
    jobs = [(*jb, by_rate) for jb in sorted(jobs, key=lambda t: -t[0])]
    if workers <= 1:
        for jb in jobs:
            k, v = _make_code(jb)
            out[k] = v
        return out
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        for k, v in pool.imap_unordered(_make_code, jobs):
            out[k] = v
    return out


# ------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------ CPU (oracle)
def _oracle_frame(task):
    """Full reverse reconciliation of one sub-block by the FP64 oracle."""
    import oracle
    snr, logn, frame, rates, codes = task
    n = 1 << logn
    x, y = synth.gaussian_pair(DATA_SEED[snr], (frame + 1) * n, snr)
    x, y = x[frame * n:], y[frame * n:]
    lo, hi = oracle.quantiser_range(snr)
    sn = snr ** -0.5
    t0 = time.perf_counter()
    _, bits = oracle.quantise(y, M_SLICES, lo, hi)
    alice = np.zeros_like(bits)
    good = 0
    for j in range(M_SLICES):
        if rates[j] <= 0:
            alice[j] = bits[j]
            continue
        rp, ci = codes[j]
        s = oracle.syndrome(rp, ci, bits[j][None])
        llr = oracle.slice_llr(x, alice[:j] if j else None, j, M_SLICES, lo, hi, sn)
        out = oracle.decode(rp, ci, llr[None], s, "sp_flood", max_iter=MAX_ITER)
        alice[j] = out["bits"][0]
        good += n * int(np.array_equal(out["bits"][0], bits[j]))
    return good, time.perf_counter() - t0


def load_sweep_rates():
    try:
        t = json.load(open(SWEEP_RATES))
    except OSError:
        raise SystemExit(f"{SWEEP_RATES} missing: run python bench.py --calibrate")
    return {(float(r[0]), int(r[1]), int(r[2])): float(r[3]) for r in t["rates"]}


def oracle_sample(step, budget_frames, cores, rate_of=None):
    """A bounded sample of the sweep: `budget_frames` sub-blocks of n = 2^12 per SNR
    (frames step*budget .. ), each reconciled over all 5 slices by the oracle
    (rates: 0.95 x capacity, or the back-off table `rate_of`)."""
    import multiprocessing as mp
    import oracle
    tasks = []
    for snr in SNRS:
        if rate_of is None:
            # the oracle's own capacities and rate rule (no library call on this leg)
            rates = [oracle.code_rate(oracle.slice_capacity(snr, M_SLICES, j)) for j in range(M_SLICES)]
        else:
            rates = [rate_of[(snr, 12, j)] for j in range(M_SLICES)]
        codes = {}
        for j in range(M_SLICES):
            if rates[j] > 0:
                M = synth.checks_for_rate(1 << 12, rates[j])
                seed = code_seed(12, j) if rate_of is None else uneven_code_seed(1 << 12, rates[j])
                rp, ci, _ = synth.make_regular_code(seed, 1 << 12, M)
                codes[j] = (rp, ci)
        for f in range(budget_frames):
            tasks.append((snr, 12, step * budget_frames + f, rates, codes))
    t0 = time.perf_counter()
    if cores > 1:
        with mp.get_context("spawn").Pool(min(cores, len(tasks))) as pool:
            res = pool.map(_oracle_frame, tasks)
    else:
        res = [_oracle_frame(t) for t in tasks]
    wall = time.perf_counter() - t0
    good = sum(r[0] for r in res)
    return good, wall, len(tasks)


# ---------------------------------------------------------- uneven batch
UNEVEN_FRAMES = 4096
UNEVEN_LENGTHS = (4096, 16384, 65536)
UNEVEN_SNR = (2.0, 15.0)
UNEVEN_SNR_STEP = 0.1
UNEVEN_MAX_ITER = 50
UNEVEN_SEED = 11
UNEVEN_SNR_BIN = 1.0            # rates are set per (n, slice, SNR bin [2,3), [3,4), ..., [14,15])
UNEVEN_RATES = os.path.join(ROOT, "uneven_rates.json")
SWEEP_RATES = os.path.join(ROOT, "sweep_rates.json")
UNEVEN_WORKLOAD = ("uneven batch: 4096 frames, n in {4096, 16384, 65536}, SNR uniform on the 0.1 grid of 2..15, "
                   "5 Gray slices, per (n, slice, SNR bin of width 1) rate from the Sec. V-B back-off (start 0.95 x "
                   "capacity at the bin's lowest SNR, minus 3/64 while > 1 of 32 trial frames fail; below 0.10: "
                   "disclosed; table in uneven_rates.json), dv=3 codes per (n, rate), layered offset min-sum FP32 "
                   "(offset 0.5), "
                   "<= 50 iterations, early stop, the frames in parts decoded on their own streams, whole step "
                   "replayed as one CUDA graph")


def _capacity_row(snr):
    import paper_2108_08418_b300 as q
    lo, hi = q.quantiser_range(snr)
    return snr, [q.qkdrec_slice_capacity(snr, M_SLICES, j, lo, hi) for j in range(M_SLICES)]


def uneven_start_rate(capacity):
    """First rate the back-off tries: 0.95 x capacity on the 1/64 grid (the library's
    rate rule), at most 60/64."""
    import paper_2108_08418_b300 as q
    return min(q.qkdrec_code_rate(capacity), 60 / 64)


def uneven_bin(snr):
    k = int((UNEVEN_SNR[1] - UNEVEN_SNR[0]) / UNEVEN_SNR_BIN)
    return np.minimum(((np.asarray(snr) - UNEVEN_SNR[0]) / UNEVEN_SNR_BIN + 1e-9).astype(np.int64), k - 1)


def uneven_bin_low(b):
    return UNEVEN_SNR[0] + UNEVEN_SNR_BIN * int(b)


def load_uneven_rates():
    try:
        t = json.load(open(UNEVEN_RATES))
    except OSError:
        raise SystemExit(f"{UNEVEN_RATES} missing: run python bench.py --workload uneven --calibrate")
    return {(int(r[0]), int(r[1]), int(r[2])): float(r[3]) for r in t["rates"]}


def uneven_code_seed(n, rate):
    return 9_000_000 + 1000 * int(n).bit_length() + int(round(rate * 64))


def _make_code_nr(key):
    n, rate = key
    rp, ci, res = synth.make_regular_code(uneven_code_seed(n, rate), n, synth.checks_for_rate(n, rate))
    return key, (rp, ci, res)


def _pool_map(fn, items, workers):
    import multiprocessing as mp
    if workers <= 1:
        return [fn(i) for i in items]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(fn, items)


def uneven_setup(seed, workers, rule="backoff"):
    """Frames (sorted by (n, SNR)), per-(slice, frame) rates and the CSR codes (host only).
    rule "backoff": the committed back-off table per (n, slice, SNR bin);
    rule "capacity": 0.95 x capacity at the frame's SNR, 1/64 grid, at most 60/64,
    below 0.10 disclosed."""
    n, snr = synth.uneven_frames(seed, UNEVEN_FRAMES, UNEVEN_LENGTHS, UNEVEN_SNR, UNEVEN_SNR_STEP)
    order = np.lexsort((snr, n))
    n, snr = n[order], snr[order]
    if rule == "backoff":
        table = load_uneven_rates()
        bins = uneven_bin(snr)
        rates = np.array([[table[(int(n[f]), int(bins[f]), j)] for f in range(n.size)] for j in range(M_SLICES)])
    else:
        caps = dict(_pool_map(_capacity_row, sorted(set(snr.tolist())), workers))
        start = np.array([[uneven_start_rate(caps[s_][j]) for s_ in snr.tolist()] for j in range(M_SLICES)])
        rates = np.where(start >= 0.10, start, 0.0)
    keys = sorted({(int(n[f]), float(rates[j, f])) for j in range(M_SLICES) for f in range(n.size)
                   if rates[j, f] > 0}, key=lambda k: -k[0])
    codes = dict(_pool_map(_make_code_nr, keys, workers))
    return n, snr, rates, codes


def _trial_sample(point):
    n, snr, j = point
    b = int(uneven_bin(snr))
    x, y = synth.gaussian_pair(600_000 + 100 * b + int(n).bit_length(), 32 * n, snr)
    return x, y


def _sweep_trial_sample(point):
    n, snr, j = point
    return synth.gaussian_pair(700_000 + 100 * int(n).bit_length() + int(snr), 32 * n, snr)


def run_calibrate(args):
    """Sec. V-B back-off on 32 trial frames per point; writes the rate table.
    uneven: every (n, slice, SNR bin), trial frames at the bin's lowest SNR;
    sweep: every (SNR, n, slice) of the block-size sweep."""
    cores = len(os.sched_getaffinity(0))
    workers = max(1, min(cores, 16))
    import paper_2108_08418_b300 as q
    from paper_2108_08418_b300 import build as qbuild
    qbuild.build()
    if args.workload == "sweep":
        points = [(1 << ln, snr, j) for snr in SNRS for ln in LOGNS for j in range(M_SLICES)]
        rates0 = {snr: slice_rates(snr, q.qkdrec_slice_capacity)[1] for snr in SNRS}
        start = {p: rates0[p[1]][p[2]] for p in points}
        sample, lows = _sweep_trial_sample, None
    else:
        nbins = int((UNEVEN_SNR[1] - UNEVEN_SNR[0]) / UNEVEN_SNR_BIN)
        lows = [uneven_bin_low(b) for b in range(nbins)]
        caps = dict(_pool_map(_capacity_row, lows, workers))
        points = [(n, s, j) for n in UNEVEN_LENGTHS for s in lows for j in range(M_SLICES)]
        start = {p: uneven_start_rate(caps[p[1]][p[2]]) for p in points}
        sample = _trial_sample
    import torch
    from paper_2108_08418_b300.uneven import backoff_rates
    torch.cuda.set_device(0)
    cache = {}

    def codes_for(keys):
        new = sorted(k for k in keys if k not in cache)
        for k, v in _pool_map(_make_code_nr, new, workers):
            cache[k] = q.Code(k[0], v[0], v[1], seed=uneven_code_seed(*k))
        return cache

    t0 = time.time()
    got = backoff_rates(points, start, codes_for, sample, trial_frames=32, max_fail=1, step=3 / 64,
                        min_rate=0.10, m_slices=M_SLICES, max_iter=UNEVEN_MAX_ITER, offset=0.5)
    if args.workload == "sweep":
        rows = [[p[1], p[0].bit_length() - 1, p[2], got[p][0], got[p][1], start[p]] for p in points]
        out = {"procedure": "Sec. V-B back-off: start at the sweep's rate (0.95 x slice capacity, 1/64 grid, "
                            "<= 63/64); 32 trial frames (seed 700000 + 100 bitlength(n) + SNR), Bob's lower "
                            "slices; layered offset min-sum <= 50 iterations; lower the rate by 3/64 while more "
                            "than 1 frame fails; below 0.10 the slice is disclosed (rate 0)",
               "command": "python bench.py --calibrate",
               "columns": ["snr", "log2_n", "slice", "rate", "trial_frame_errors", "start_rate"]}
    else:
        rows = [[p[0], int(uneven_bin(p[1])), p[2], got[p][0], got[p][1], start[p]] for p in points]
        out = {"procedure": "Sec. V-B back-off: start at 0.95 x slice capacity (1/64 grid, <= 60/64) at the "
                            "bin's lowest SNR; 32 trial frames (seed 600000 + 100 bin + bitlength(n)), Bob's "
                            "lower slices; layered offset min-sum <= 50 iterations; lower the rate by 3/64 while "
                            "more than 1 frame fails; below 0.10 the slice is disclosed (rate 0)",
               "command": "python bench.py --workload uneven --calibrate",
               "columns": ["n", "snr_bin", "slice", "rate", "trial_frame_errors", "start_rate"],
               "snr_bins": [[lo, lo + UNEVEN_SNR_BIN] for lo in lows]}
    out.update({"seconds": round(time.time() - t0, 1), "rates": rows})
    with open(args.rates_out or (SWEEP_RATES if args.workload == "sweep" else UNEVEN_RATES), "w") as fh:
        json.dump(out, fh, indent=0)
    print(json.dumps({"calibrated_points": len(rows), "seconds": out["seconds"],
                      "disclosed": sum(1 for r in rows if r[3] == 0.0)}), flush=True)


def _oracle_uneven_frame(task):
    """Reverse reconciliation of one frame of the uneven batch by the FP64 oracle."""
    import oracle
    x, y, snr, rates, csr, algo, max_iter = task
    lo, hi = oracle.quantiser_range(snr)
    t0 = time.perf_counter()
    _, bits = oracle.quantise(y, M_SLICES, lo, hi)
    alice = np.zeros_like(bits)
    good = 0
    for j in range(M_SLICES):
        if rates[j] <= 0:
            alice[j] = bits[j]
            continue
        rp, ci = csr[j]
        s = oracle.syndrome(rp, ci, bits[j][None])
        llr = oracle.slice_llr(x.astype(np.float64), alice[:j] if j else None, j, M_SLICES, lo, hi, snr ** -0.5)
        out = oracle.decode(rp, ci, llr[None], s, algo, max_iter=max_iter, offset=0.5)
        alice[j] = out["bits"][0]
        good += y.size * int(np.array_equal(out["bits"][0], bits[j]))
    return good, time.perf_counter() - t0


def oracle_uneven_sample(step, per_step, cores, setup=None, algo="oms_layered", max_iter=UNEVEN_MAX_ITER):
    """A bounded sample of the uneven batch: `per_step` frames of n = 4096 (spread over
    the SNR range), each reconciled over all 5 slices by the oracle."""
    n, snr, rates, codes = setup or uneven_setup(UNEVEN_SEED, max(1, min(cores, 16)))
    x, y = synth.gaussian_frames(UNEVEN_SEED, n, snr)
    off = np.concatenate([[0], np.cumsum(n)])
    small = np.flatnonzero(n == UNEVEN_LENGTHS[0])
    pick = small[(np.arange(per_step) * 97 + step * per_step * 97) % small.size]
    tasks = []
    for f in pick:
        csr = {j: codes[(int(n[f]), float(rates[j, f]))][:2] for j in range(M_SLICES) if rates[j, f] > 0}
        tasks.append((x[off[f]:off[f + 1]], y[off[f]:off[f + 1]], float(snr[f]), rates[:, f].copy(), csr, algo,
                      max_iter))
    t0 = time.perf_counter()
    res = _pool_map(_oracle_uneven_frame, tasks, min(cores, len(tasks)))
    wall = time.perf_counter() - t0
    return sum(r[0] for r in res), wall, len(tasks)


def run_uneven(args):
    rank, world, local = rank_env()
    cores = len(os.sched_getaffinity(0))
    import paper_2108_08418_b300 as q
    from paper_2108_08418_b300 import build as qbuild
    qbuild.build()
    t_setup = time.time()
    seed = UNEVEN_SEED + 1000 * rank
    n, snr, rates, codes_h = uneven_setup(seed, max(1, min(cores, 16)), args.rate_rule)
    plain = args.uneven_decoder == "sp_f32"
    algo, max_iter = ("sp_flood", MAX_ITER) if plain else ("oms_layered", UNEVEN_MAX_ITER)
    algo_text = (f"sum-product flooding <= {max_iter} iterations" if plain
                 else f"layered offset min-sum <= {max_iter} iterations")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        per = 3 * max(1, min(cores, 8))
        good, wall, nfr = oracle_uneven_sample(0, per, cores, (n, snr, rates, codes_h), algo, max_iter)
        cpu = {"value": good / wall, "unit": "bit/s", "cores": min(cores, nfr), "kind": "oracle",
               "sample": f"{nfr} frames of n=4096 of the batch, each reconciled over all 5 slices (FP64 quantiser, "
                         f"LLR, syndrome, {algo_text}), one process per frame", "wall_s": wall}

    import torch
    import torch.distributed as dist
    from paper_2108_08418_b300.uneven import UnevenBatch
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    codes = {k: q.Code(k[0], v[0], v[1], seed=uneven_code_seed(*k)) for k, v in codes_h.items()}
    residual = max(v[2] for v in codes_h.values())
    x, y = synth.gaussian_frames(seed, n, snr)
    hx, hy = torch.from_numpy(x).pin_memory(), torch.from_numpy(y).pin_memory()
    decoder = q.DecodeOpts(algo="sp_flood", prec="f32", max_iter=MAX_ITER, early_stop=True) if plain else None
    ub = UnevenBatch(n, snr, rates, codes, M_SLICES, max_iter=UNEVEN_MAX_ITER, device=dev, decoder=decoder,
                     parts=args.uneven_parts)
    ub.x.copy_(hx)
    ub.y.copy_(hy)
    tunings = ub.autotune(max_iter=10)
    ub.capture()
    setup_s = time.time() - t_setup
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ub.replay()
    barrier()
    sampler = ClockSampler(smi_index(torch, dev, local))
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ub.replay()
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    good_bits, raw_bits = ub.reconciled_bits(), ub.decoded_bits()
    ok = ub.frame_ok().cpu().numpy()
    dec = rates > 0
    fer = {}
    for ln in UNEVEN_LENGTHS:
        sel = n == ln
        fer[f"n{ln}"] = [round(float(1 - ok[j, sel & dec[j]].mean()), 4) if (sel & dec[j]).any() else None
                         for j in range(M_SLICES)]
    iters = ub.iters.cpu().numpy()
    mean_iters = [round(float(iters[j, dec[j]].mean()), 2) if dec[j].any() else None for j in range(M_SLICES)]

    # per-kernel durations: the same step run eagerly with the profiling hooks
    q.qkdrec_profile_begin()
    for _ in range(args.steps):
        ub.step(overlap=False)
    barrier()
    stats = q.qkdrec_profile_end()

    # end to end: pinned host x, y -> device, graph replay, Alice's reconciled slices
    # (packed 8 per byte), flags and iteration counts back to pinned host memory
    t_e2e = None
    pk = torch.empty((ub.m, ub.count // 8), dtype=torch.uint8, device=dev)
    hpk = torch.empty(pk.shape, dtype=torch.uint8).pin_memory()
    hconv = torch.empty(ub.conv.shape, dtype=ub.conv.dtype).pin_memory()
    hits = torch.empty(ub.iters.shape, dtype=ub.iters.dtype).pin_memory()
    h2d = hx.numel() * 4 + hy.numel() * 4
    d2h = hpk.numel() + hconv.numel() + hits.numel() * 4
    e2e_same = None
    if not args.no_e2e:
        # inputs double-buffered: step k+1's x, y travel from pinned host memory into
        # a staging buffer on a copy stream while step k decodes; each step moves its
        # staged inputs into place (a device copy), replays, and reads its results
        # back before the next step starts
        stage = [(torch.empty_like(ub.x), torch.empty_like(ub.y)) for _ in range(2)]
        copy_st = torch.cuda.Stream(dev)
        staged = [torch.cuda.Event() for _ in range(2)]

        def fetch(b):
            copy_st.wait_stream(stream)
            with torch.cuda.stream(copy_st):
                stage[b][0].copy_(hx, non_blocking=True)
                stage[b][1].copy_(hy, non_blocking=True)
                staged[b].record(copy_st)

        barrier()
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        fetch(0)
        for k in range(args.steps):
            stream.wait_event(staged[k % 2])
            ub.x.copy_(stage[k % 2][0])
            ub.y.copy_(stage[k % 2][1])
            if k + 1 < args.steps:
                fetch((k + 1) % 2)
            ub.replay()
            for j in range(ub.m):
                q.qkdrec_pack_bits(ub.alice[j], out=pk[j])
            hpk.copy_(pk, non_blocking=True)
            hconv.copy_(ub.conv, non_blocking=True)
            hits.copy_(ub.iters, non_blocking=True)
            stream.synchronize()
        e3.record(stream)
        barrier()
        t_e2e = e2.elapsed_time(e3)
        e2e_same = bool(torch.equal(hpk.to(dev), torch.stack([q.qkdrec_pack_bits(ub.alice[j]) for j in range(ub.m)])))

    (good_bits, raw_bits), (ms, t_e2e_max) = reduce_over_ranks([good_bits, raw_bits], [ms, t_e2e or 0.0], dev,
                                                                world)
    ms_step = ms / args.steps
    roof, kernels, launches = roofline(stats, args.steps)
    if rank != 0:
        return
    line = {
        "metric": "reconciled key bits/s", "value": good_bits / (ms_step / 1e3), "unit": "bit/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded Philox Gaussian quadratures and seeded regular dv=3 LDPC codes",
        "config": {"workload": UNEVEN_WORKLOAD if not plain else UNEVEN_WORKLOAD.replace(
                       "layered offset min-sum FP32 (offset 0.5), <= 50 iterations",
                       f"FP32 sum-product flooding, <= {MAX_ITER} iterations, one batch-decoder call per group"),
                   "frames": int(n.size), "samples": int(n.sum()),
                   "groups_per_slice": [len(g) for g in ub.groups], "parts": ub.parts, "algo": algo, "prec": "f32",
                   "max_iter": max_iter, "tuning_per_part_and_slice": [t[0] for t in tunings],
                   "rate_rule": args.rate_rule,
                   "l2": "inputs larger than L2 (x, y 470 MB each; plan workspace "
                         f"{ub.ws.numel() / 2**30:.2f} GiB)",
                   "raw_decoded_bits_per_s": raw_bits / (ms_step / 1e3), "fer_per_slice": fer,
                   "mean_iters_per_slice": mean_iters, "code_residual_4cycles": residual,
                   "kernel_times": "per-kernel figures from the same step run eagerly with the profiling hooks, its "
                                   "parts and syndromes in order on one stream",
                   "dominant_kernel_gbs_over_step": (roof["achieved"] * roof["avg_launch_ms"] * roof["launches"]
                                                     / args.steps / ms_step if roof else None),
                   "setup_s": round(setup_s, 1)},
        "roofline": roof,
        "kernels": kernels,
        "cpu_baseline": cpu,
        "e2e": ({"value": good_bits / (t_e2e_max / args.steps / 1e3), "unit": "bit/s",
                 "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                 "ms_per_step": t_e2e_max / args.steps,
                 "api": "the uneven step's graph replayed with x, y copied from pinned host memory (the next "
                        "step's copy overlapping this step's decode, double-buffered); Alice's slices packed 8 per "
                        "byte, flags and iteration counts copied back to pinned host memory every step",
                 "same_result_as_device_run": e2e_same} if t_e2e else None),
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def reduce_over_ranks(sums, maxes, dev, world):
    """Whole-job figures: counters summed over ranks, times maxed over ranks (every
    rank calls this; one rank returns its own values)."""
    import torch
    import torch.distributed as dist
    tot = torch.tensor([float(v) for v in sums], dtype=torch.float64, device=dev)
    tmax = torch.tensor([float(v) for v in maxes], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    return [float(v) for v in tot], [float(v) for v in tmax]


def smi_index(torch, dev, local):
    props = torch.cuda.get_device_properties(dev)
    bus = getattr(props, "pci_bus_id", None)
    return (f"{getattr(props, 'pci_domain_id', 0):08x}:{bus:02x}:{getattr(props, 'pci_device_id', 0):02x}.0"
            if bus is not None else str(local))


def roofline(stats, steps):
    """Roofline of the dominant kernel class, per-kernel table and our launches per step."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak, peak_src = (peaks["hbm_gbs"], "measured") if "hbm_gbs" in peaks else (6400.0, "fallback")
    dname, d = max(stats.items(), key=lambda kv: kv[1]["ms"])
    achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": dname, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": peak_src,
            "traffic": load_traffic(dname, d), "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
            "avg_launch_ms": d["ms"] / d["launches"], "launches": d["launches"],
            "share": round(d["ms"] / sum(v["ms"] for v in stats.values()), 4)}
    kernels = {k: {"launches": v["launches"], "ms_per_step": round(v["ms"] / steps, 3),
                   "GB/s": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 else None}
               for k, v in sorted(stats.items(), key=lambda kv: -kv[1]["ms"])}
    launches = int(sum(v["launches"] for v in stats.values()) / steps)
    return roof, kernels, launches


# ------------------------------------------------ differentiable weighted min-sum
WOMS_N, WOMS_F, WOMS_T, WOMS_K, WOMS_SNR, WOMS_SLICE = 16384, 1024, 20, 5, 3.0, 4
WOMS_WORKLOAD = ("weighted offset min-sum training: 1024 frames of n=16384, slice 4 (capacity 0.545) of the 5-slice "
                 "Gray quantiser at "
                 "SNR 3, rate-1/2 (dv=3, dc=6) code, 20 unrolled flooding iterations, alpha/beta [20][2], "
                 "checkpoints every 5, BCE loss, Adam; one step = forward + adjoint + update")


def _oracle_woms_task(task):
    """Loss and FP64 reverse-mode gradient of the unrolled weighted min-sum for a
    few frames by the oracle; returns the wall time."""
    import oracle
    rp, ci, llr, synd, tgt, a, b = task
    t0 = time.perf_counter()
    oracle.woms(rp, ci, llr, synd, tgt, a, b)
    return time.perf_counter() - t0


def oracle_woms_sample(step, cores, per_proc=12):
    """A bounded sample of one training step: `per_proc` frames per host process
    (frames step*k .. of the training batch, k = processes x per_proc), inputs
    from the oracle's own quantiser, slice LLRs and syndromes; weights at their
    initial values.  Returns (frames, wall seconds, processes)."""
    import oracle
    procs = max(1, min(cores, 8))
    k = procs * per_proc
    f0 = (step * k) % WOMS_F
    rp, ci, _ = synth.make_regular_code(5000, WOMS_N, synth.checks_for_rate(WOMS_N, 0.5))
    x, y = synth.gaussian_pair(5, (f0 + k) * WOMS_N, WOMS_SNR)
    x, y = x[f0 * WOMS_N:], y[f0 * WOMS_N:]
    lo, hi = oracle.quantiser_range(WOMS_SNR)
    _, bits = oracle.quantise(y, M_SLICES, lo, hi)
    j = WOMS_SLICE
    llr = oracle.slice_llr(x.astype(np.float64), bits[:j], j, M_SLICES, lo, hi, WOMS_SNR ** -0.5).reshape(k, WOMS_N)
    tgt = bits[j].reshape(k, WOMS_N)
    synd = oracle.syndrome(rp, ci, tgt)
    a, b = np.ones((WOMS_T, 2)), np.full((WOMS_T, 2), 0.5)
    tasks = [(rp, ci, llr[i:i + per_proc], synd[i:i + per_proc], tgt[i:i + per_proc], a, b)
             for i in range(0, k, per_proc)]
    t0 = time.perf_counter()
    _pool_map(_oracle_woms_task, tasks, procs)
    return k, time.perf_counter() - t0, procs


def woms_frames(q, torch, code, seed, dev):
    """Slice LLRs (Bob's lower slices reconciled), Bob's slice bits and syndromes."""
    x, y = synth.gaussian_pair(seed, WOMS_F * WOMS_N, WOMS_SNR)
    lo, hi = q.quantiser_range(WOMS_SNR)
    _, bits = q.qkdrec_quantise_slices(torch.from_numpy(y).to(dev), M_SLICES, lo, hi, want_idx=False)
    j = WOMS_SLICE
    target = bits[j].reshape(WOMS_F, WOMS_N).contiguous()
    llr = q.qkdrec_slice_llr(torch.from_numpy(x).to(dev), M_SLICES, j, lo, hi, WOMS_SNR ** -0.5, bits[:j])
    return llr.reshape(WOMS_F, WOMS_N), q.qkdrec_syndrome(code, target), target


def run_woms(args):
    rank, world, local = rank_env()
    cores = len(os.sched_getaffinity(0))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # before CUDA is touched (spawn pool)
        nfr, wall, procs = oracle_woms_sample(0, cores)
        cpu = {"value": nfr / (WOMS_F * wall), "unit": "step/s", "cores": procs, "kind": "oracle",
               "sample": f"{nfr} of the {WOMS_F} frames of one step: FP64 forward and reverse-mode gradient "
                         f"({WOMS_T} iterations), {procs} processes; steps/s = frames / ({WOMS_F} x wall)",
               "wall_s": wall}
    import paper_2108_08418_b300 as q
    from paper_2108_08418_b300 import build as qbuild
    from paper_2108_08418_b300.woms import woms_loss
    qbuild.build()
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rp, ci, res = synth.make_regular_code(5000, WOMS_N, synth.checks_for_rate(WOMS_N, 0.5))
    code = q.Code(WOMS_N, rp, ci, seed=5000)
    llr, synd, target = woms_frames(q, torch, code, 5 + 1000 * rank, dev)
    ev_llr, ev_synd, ev_target = woms_frames(q, torch, code, 6 + 1000 * rank, dev)
    alpha = torch.ones((WOMS_T, 2), device=dev, requires_grad=True)
    beta = torch.full((WOMS_T, 2), 0.5, device=dev, requires_grad=True)
    opt = torch.optim.Adam([alpha, beta], lr=0.02)

    def fer(a, b):
        ws = torch.empty(q.qkdrec_woms_workspace_size(code, WOMS_F, WOMS_T, WOMS_K), dtype=torch.uint8, device=dev)
        _, post = q.qkdrec_woms_forward(code, ev_llr, ev_synd, ev_target, a.detach().contiguous(),
                                        b.detach().contiguous(), WOMS_K, ws, want_post=True)
        return float(((post < 0).to(torch.uint8) != ev_target).any(dim=1).float().mean())

    fer_init = fer(alpha, beta)
    sp = q.qkdrec_decode_batch(code, ev_llr, ev_synd, q.DecodeOpts(algo="sp_flood", max_iter=WOMS_T, early_stop=False))
    fer_sp = float((sp["bits"] != ev_target).any(dim=1).float().mean())
    losses = []

    def step():
        opt.zero_grad()
        loss = woms_loss(code, llr, synd, target, alpha, beta, WOMS_K)
        loss.backward()
        opt.step()
        return loss.detach()

    for _ in range(args.warmup):
        losses.append(float(step()))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    sampler = ClockSampler(smi_index(torch, dev, local))
    sampler.start()
    q.qkdrec_profile_begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    timed = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    stats = q.qkdrec_profile_end()
    clocks = sampler.stop()
    losses += [float(v) for v in timed]
    ms = e0.elapsed_time(e1) / args.steps
    # check edge-updates of one step: the forward, its recomputation and the adjoint
    upd_units = sum(stats.get(k, {}).get("units", 0) for k in ("woms_check_fwd", "woms_check_bwd")) / args.steps
    roof, kernels, launches = roofline(stats, args.steps)
    # a short training run after the timed steps, then the FER of the trained weights
    for _ in range(max(0, args.train_steps - args.warmup - args.steps)):
        losses.append(float(step()))
    fer_trained = fer(alpha, beta)

    # end to end: each step's frames from pinned host memory, the loss read back
    e2e = None
    if not args.no_e2e:
        hl, hs, ht = llr.cpu().pin_memory(), synd.cpu().pin_memory(), target.cpu().pin_memory()
        h2d = hl.numel() * 4 + hs.numel() + ht.numel()
        torch.cuda.synchronize()
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for _ in range(args.steps):
            llr.copy_(hl, non_blocking=True)
            synd.copy_(hs, non_blocking=True)
            target.copy_(ht, non_blocking=True)
            losses.append(float(step()))
        e3.record(stream)
        torch.cuda.synchronize()
        e2e = {"value": 1e3 / (e2.elapsed_time(e3) / args.steps), "unit": "step/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 4}
    if rank != 0:
        return
    line = {
        "metric": "weighted min-sum training steps/s", "value": 1e3 / ms, "unit": "step/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded Philox Gaussian quadratures and a seeded regular (3,6) LDPC code",
        "config": {"workload": WOMS_WORKLOAD, "frames": WOMS_F, "n": WOMS_N, "iterations": WOMS_T,
                   "ckpt_every": WOMS_K, "check_edge_updates_per_s": upd_units / (ms / 1e3),
                   "loss_first": losses[0], "loss_last": losses[-1], "train_steps": len(losses),
                   "fer_eval": {"woms_initial": fer_init, "woms_trained": fer_trained, "sum_product_20it": fer_sp},
                   "l2": "messages 201 MB per copy, checkpoints 805 MB: larger than L2"},
        "roofline": roof, "kernels": kernels, "cpu_baseline": cpu,
        "e2e": e2e, "gpu_launches": launches * args.steps, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
# --decoder: the block-size sweep decoded with another form (the precision study)
DECODERS = {"sp_f32": ("sp_flood", "f32"), "sp_f16": ("sp_flood", "f16"), "oms_f32": ("oms_flood", "f32"),
            "oms_f16": ("oms_flood", "f16"), "oms_i8": ("oms_flood", "i8"), "layered_f32": ("oms_layered", "f32"),
            "layered_f16": ("oms_layered", "f16"), "layered_i8": ("oms_layered", "i8")}


def run_ours(args):
    rank, world, local = rank_env()
    cores = len(os.sched_getaffinity(0))
    # the codes are built before CUDA is touched (spawn pool)
    import paper_2108_08418_b300 as q
    from paper_2108_08418_b300 import build as qbuild
    qbuild.build()
    if args.rate_rule == "backoff":
        # the sweep's frames at the Sec. V-B back-off rates (table written by --calibrate)
        rate_of = load_sweep_rates()
    else:
        base = {snr: slice_rates(snr, q.qkdrec_slice_capacity)[1] for snr in SNRS}
        rate_of = {(snr, ln, j): base[snr][j] for snr in SNRS for ln in LOGNS for j in range(M_SLICES)}
    jobs = {(ln, j, r) for (snr, ln, j), r in rate_of.items() if r > 0}
    t_setup = time.time()
    codes_h = build_codes(jobs, max(1, min(cores, 16)), args.rate_rule == "backoff")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # frames at the back-off rates converge in a few iterations: twice the sub-blocks
        # keep the sample at 10-30 s of host CPU work
        per = max(1, min(cores, 8) // 2) * (2 if args.rate_rule == "backoff" else 1)
        good, wall, nfr = oracle_sample(0, per, cores, rate_of if args.rate_rule == "backoff" else None)
        cpu = {"value": good / wall, "unit": "bit/s", "cores": min(cores, nfr), "kind": "oracle",
               "sample": f"{nfr} sub-blocks of n=4096 ({nfr // 2} per SNR), each reconciled over all 5 slices "
                         f"(FP64 quantiser, LLR, syndrome, sum-product <= 100 iterations), one process per sub-block",
               "wall_s": wall}

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    codes = {k: q.Code(1 << k[0], v[0], v[1], seed=v[3]) for k, v in codes_h.items()}
    residual = max(v[2] for v in codes_h.values())

    # data: rank r reconciles its own block (weak scaling)
    host_x, host_y, dx, dy = {}, {}, {}, {}
    for snr in SNRS:
        x, y = synth.gaussian_pair(DATA_SEED[snr] + 1000 * rank, N_SAMPLES, snr)
        host_x[snr] = torch.from_numpy(x).pin_memory()
        host_y[snr] = torch.from_numpy(y).pin_memory()
        dx[snr] = host_x[snr].to(dev)
        dy[snr] = host_y[snr].to(dev)
    algo, prec = DECODERS[args.decoder]
    # low-precision forms re-decode the frames they leave unsatisfied in FP32
    opts = q.DecodeOpts(algo=algo, prec=prec, max_iter=MAX_ITER, early_stop=True,
                        fallback_f32=(args.fallback if prec != "f32" else False))
    plain = q.DecodeOpts(algo="sp_flood", prec="f32", max_iter=MAX_ITER, early_stop=True)
    lo_hi = {snr: q.quantiser_range(snr) for snr in SNRS}
    # per point (SNR, n): Alice's reconciled slices packed 8 to a byte, flags, iterations
    alice_pk = {(snr, ln): torch.empty((M_SLICES, N_SAMPLES // 8), dtype=torch.uint8, device=dev)
                for snr in SNRS for ln in LOGNS}
    conv_pt = {(snr, ln): torch.empty((M_SLICES, N_SAMPLES >> ln), dtype=torch.uint8, device=dev)
               for snr in SNRS for ln in LOGNS}
    its_pt = {(snr, ln): torch.empty((M_SLICES, N_SAMPLES >> ln), dtype=torch.int32, device=dev)
              for snr in SNRS for ln in LOGNS}
    iters = {(snr, ln, j): its_pt[(snr, ln)][j] for snr in SNRS for ln in LOGNS for j in range(M_SLICES)}
    conv = {(snr, ln, j): conv_pt[(snr, ln)][j] for snr in SNRS for ln in LOGNS for j in range(M_SLICES)}

    def slice_codes(snr, ln):
        return [codes[(ln, j, rate_of[(snr, ln, j)])] if rate_of[(snr, ln, j)] > 0 else None
                for j in range(M_SLICES)]

    def points(snr, outs):
        return [dict(n=1 << ln, codes=slice_codes(snr, ln), alice_packed=outs[0][(snr, ln)],
                     converged=outs[1][(snr, ln)], iters=outs[2][(snr, ln)]) for ln in LOGNS]

    dev_outs = (alice_pk, conv_pt, its_pt)
    # every sub-block length of a block decodes at once (one workspace slot and side
    # stream each); the per-kernel profile runs them one after another (one slot), so
    # that each kernel's event time is its own
    rws = torch.empty(max(q.qkdrec_reconcile_workspace_size(N_SAMPLES, M_SLICES, o, points(snr, dev_outs))
                          for snr in SNRS for o in (opts, plain)), dtype=torch.uint8, device=dev)
    rws1 = rws[:max(q.qkdrec_reconcile_workspace_size_limited(N_SAMPLES, M_SLICES, o, points(snr, dev_outs), 1)
                    for snr in SNRS for o in (opts, plain))]
    # the two blocks (SNRs) overlap as well: the second runs on its own stream and
    # workspace, each of its sub-block lengths following the first block's on the
    # same side stream
    rws_b = torch.empty_like(rws) if not args.soft_chain else None
    side = torch.cuda.Stream(dev)
    if args.soft_chain:
        # soft chaining (slice j's LLRs from the lower slices' decoder posteriors) runs
        # through the single-step calls
        ws = torch.empty(max(q.qkdrec_decode_workspace_size(c, N_SAMPLES >> k[0], opts) for k, c in codes.items()),
                         dtype=torch.uint8, device=dev)
        alice = torch.empty((M_SLICES, N_SAMPLES), dtype=torch.uint8, device=dev)
        llr = torch.empty(N_SAMPLES, dtype=torch.float32, device=dev)
        post = torch.empty((M_SLICES, N_SAMPLES), dtype=torch.float32, device=dev)
    setup_s = time.time() - t_setup

    def step_soft(xs, ys, opts, outs):
        for snr in SNRS:
            lo, hi = lo_hi[snr]
            sn = snr ** -0.5
            x_s = xs[snr] if xs[snr].is_cuda else xs[snr].to(dev, non_blocking=True)
            y_s = ys[snr] if ys[snr].is_cuda else ys[snr].to(dev, non_blocking=True)
            _, bits = q.qkdrec_quantise_slices(y_s, M_SLICES, lo, hi, want_idx=False)
            for ln in LOGNS:
                n, F = 1 << ln, N_SAMPLES >> ln
                for j in range(M_SLICES):
                    r = rate_of[(snr, ln, j)]
                    if r <= 0:
                        alice[j].copy_(bits[j])          # disclosed slice: Bob's bits in the clear
                        q.qkdrec_bits_to_llr(bits[j], out=post[j])
                        conv_pt[(snr, ln)][j].fill_(1)
                        its_pt[(snr, ln)][j].zero_()
                        continue
                    c = codes[(ln, j, r)]
                    synd = q.qkdrec_syndrome(c, bits[j].view(F, n))
                    q.qkdrec_slice_llr_soft(x_s, M_SLICES, j, lo, hi, sn, post[:j] if j else None, out=llr)
                    q.qkdrec_decode_batch(c, llr.view(F, n), synd, opts, workspace=ws,
                                          out=dict(bits=alice[j].view(F, n), iters=its_pt[(snr, ln)][j],
                                                   converged=conv_pt[(snr, ln)][j], post=post[j].view(F, n)))
                for j in range(M_SLICES):
                    q.qkdrec_pack_bits(alice[j], out=alice_pk[(snr, ln)][j])
                if outs is not dev_outs:
                    for k in range(3):
                        outs[k][(snr, ln)].copy_(dev_outs[k][(snr, ln)], non_blocking=True)

    def step(xs, ys, opts=opts, outs=dev_outs, ws=rws, overlap=True):
        """One reverse reconciliation of both blocks at every sub-block length."""
        if args.soft_chain:
            step_soft(xs, ys, opts, outs)
            return
        main = torch.cuda.current_stream(dev)
        if overlap:
            side.wait_stream(main)
        for i, snr in enumerate(SNRS):
            lo, hi = lo_hi[snr]
            with torch.cuda.stream(side if overlap and i % 2 else main):
                q.qkdrec_reconcile(xs[snr], ys[snr], M_SLICES, lo, hi, snr ** -0.5, opts, points(snr, outs),
                                   workspace=rws_b if overlap and i % 2 else ws, device=dev)
        if overlap:
            main.wait_stream(side)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(dx, dy)
    barrier()
    # the step has no host synchronisation and allocates nothing, so it is captured
    # once as a CUDA graph and replayed (the soft-chained form runs eagerly)
    graph = None
    if not args.soft_chain:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, capture_error_mode="relaxed"):
            step(dx, dy)
        graph.replay()
        barrier()
    sampler = ClockSampler(smi_index(torch, dev, local))
    sampler.start()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        if graph is not None:
            graph.replay()
        else:
            step(dx, dy)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    # per-kernel figures: the same steps run eagerly with every library launch
    # bracketed by CUDA events on its stream (events inside a replayed graph do not time)
    q.qkdrec_profile_begin()
    e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e4.record(stream)
    for _ in range(args.steps):
        step(dx, dy, ws=rws1, overlap=False)
    e5.record(stream)
    barrier()
    stats = q.qkdrec_profile_end()
    ms_profiled = e4.elapsed_time(e5)
    clocks = sampler.stop()

    # correctness of the last step: sub-blocks whose decoded word equals Bob's
    # (Bob's slices packed the same way, outside the timed region)
    bob_pk = {}
    for snr in SNRS:
        lo, hi = lo_hi[snr]
        _, bits = q.qkdrec_quantise_slices(dy[snr], M_SLICES, lo, hi, want_idx=False)
        bob_pk[snr] = torch.stack([q.qkdrec_pack_bits(bits[j]) for j in range(M_SLICES)])
        del bits

    def frame_bad(snr, ln, j, packed):
        n, F = 1 << ln, N_SAMPLES >> ln
        return (packed[(snr, ln)][j].view(F, n // 8) != bob_pk[snr][j].view(F, n // 8)).any(dim=1)

    def frame_errors(snr, ln, j, packed):
        return int(frame_bad(snr, ln, j, packed).sum())

    good_bits, raw_bits, fer, mean_iters = 0, 0, {}, {}
    edge_updates = sum(v["units"] for k, v in stats.items() if k.startswith(("check_flood", "layer_oms"))) / args.steps
    for snr in SNRS:
        for ln in LOGNS:
            n, F = 1 << ln, N_SAMPLES >> ln
            errs, its = [], []
            for j in range(M_SLICES):
                if rate_of[(snr, ln, j)] <= 0:
                    continue
                nbad = frame_errors(snr, ln, j, alice_pk)
                good_bits += n * (F - nbad)
                raw_bits += N_SAMPLES
                errs.append(round(nbad / F, 4))
                its.append(round(float(iters[(snr, ln, j)].float().mean().item()), 2))
            fer[f"snr{int(snr)}_n2^{ln}"] = errs
            mean_iters[f"snr{int(snr)}_n2^{ln}"] = its
    # the paper's reconciliation efficiency of each point's rates (Eq. beta, disclosed
    # slices at rate 0), and the net key it leaves: (Pi(M(Y)) - m + sum R_j) bits per
    # sample of every sub-block whose slices all reconciled, per second
    beta_pt, net_bits = {}, 0.0
    for snr in SNRS:
        lo, hi = lo_hi[snr]
        for ln in LOGNS:
            n, F = 1 << ln, N_SAMPLES >> ln
            rates = [rate_of[(snr, ln, j)] for j in range(M_SLICES)]
            beta, H = q.qkdrec_reconciliation_efficiency(snr, M_SLICES, lo, hi, rates)
            beta_pt[f"snr{int(snr)}_n2^{ln}"] = round(beta, 4)
            bad = torch.zeros(F, dtype=torch.bool, device=dev)
            for j in range(M_SLICES):
                if rates[j] > 0:
                    bad |= frame_bad(snr, ln, j, alice_pk)
            net_bits += (H - M_SLICES + sum(rates)) * n * (F - int(bad.sum()))
    # Sec. IV-B's optimum sub-block length with this decoder's measured inputs:
    # c_h (time per arithmetic operation, Eq. DeltaT) and D_j (mean iterations of
    # each decoded slice of the largest sub-blocks at SNR 3; 3 edges per sample for
    # the dv = 3 codes, 0 for a disclosed slice), at the paper's standard settings
    nr_opt = None
    if edge_updates:
        c_h = (ms / args.steps / 1e3) / (7 * edge_updates)
        ln_big = max(LOGNS)
        g_j = [3.0 if rate_of[(3.0, ln_big, j)] > 0 else 0.0 for j in range(M_SLICES)]
        d_j = [float(iters[(3.0, ln_big, j)].float().mean()) if g_j[j] else 0.0 for j in range(M_SLICES)]
        nr_opt = {}
        for form, name in ((0, "awgn_dispersion"), (1, "printed_dispersion")):
            r = q.qkdrec_nr_optimise(g_j, d_j, c_h=c_h, dispersion_form=form)
            nr_opt[name] = {"nr_opt": r["nr_opt"], "key_rate_bits_per_s": r["key_rate_opt"],
                            "at_boundary": bool(r["at_boundary"])}
        nr_opt["inputs"] = {"c_h_s": c_h, "D_j": [round(v, 2) for v in d_j], "edges_per_sample": g_j,
                            "settings": "the paper's standard CV-QKD settings (N = 1e9, m = 5, eps = 2.5e-10, "
                                        "V_A = 5, T = 0.9, xi_ch = 0.0186, xi_d = 0.0133)"}
        nr_opt["paper"] = {"nr_opt": 3.6e7, "key_rate_bits_per_s": 4.3e5, "c_h_s": 3.2e-9, "hardware": "GTX 1060"}
    # how full the decoders' 32-frame blocks stay: frame-iterations done over the
    # frame-iterations the blocks occupy (a block runs until its last frame stops),
    # from the per-frame iteration counts; with the FP32 flooding decoders' re-packing
    # of the decoding frames after iterations REPACK_AT, and without it
    occ = {}
    repacks = prec == "f32" and algo != "oms_layered"
    for name, sched in (("with_repacking", REPACK_AT if repacks else ()), ("without_repacking", ())):
        num = den = 0.0
        for (snr, ln, j), it in iters.items():
            if rate_of[(snr, ln, j)] <= 0:
                continue
            e = codes[(ln, j, rate_of[(snr, ln, j)])].E
            t_f = it.cpu().numpy().astype(np.int64) + 1
            num += float(t_f.sum()) * e
            den += block_work(t_f, sched) * e
        occ[name] = num / den if den else None

    # per-result error against the FP64 oracle on a sample of sub-blocks, and (for the
    # low-precision forms) the FER of the plain FP32 sum-product form on the same block
    err_oracle = None if args.soft_chain or world > 1 else error_vs_oracle(
        q, torch, dev, codes, codes_h, rate_of, host_x, host_y, opts)
    fer_plain = None
    if args.decoder != "sp_f32" and not args.soft_chain:
        step(dx, dy, plain)
        fer_plain = {f"snr{int(snr)}_n2^{ln}": [round(frame_errors(snr, ln, j, alice_pk) / (N_SAMPLES >> ln), 4)
                                                 for j in range(M_SLICES) if rate_of[(snr, ln, j)] > 0]
                     for snr in SNRS for ln in LOGNS}

    # end to end through the public API: the same call with HOST buffers -- x, y read
    # from pinned host memory and Alice's packed slices, flags and iteration counts of
    # every point written back to pinned host memory, inside the timed region
    t_e2e = None
    host_outs = tuple({k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in d.items()}
                      for d in dev_outs)
    h2d = sum(host_x[s].numel() * 4 + host_y[s].numel() * 4 for s in SNRS)
    d2h = sum(t.numel() * t.element_size() for d in host_outs for t in d.values())
    if not args.no_e2e:
        barrier()
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for _ in range(args.steps):
            step(host_x, host_y, opts, host_outs)
            torch.cuda.current_stream(dev).synchronize()
        e3.record(stream)
        barrier()
        t_e2e = e2.elapsed_time(e3)
        # the host copies hold the same result as the device-timed run
        e2e_same = all(torch.equal(host_outs[0][k].to(dev), alice_pk[k]) for k in alice_pk)
    else:
        e2e_same = None

    # aggregate over ranks
    (good_bits, raw_bits), (ms, t_e2e_max) = reduce_over_ranks([good_bits, raw_bits], [ms, t_e2e or 0.0], dev,
                                                                world)
    ms_step = ms / args.steps
    value = good_bits / (ms_step / 1e3)

    roof, kernels, launches = roofline(stats, args.steps)
    if rank != 0:
        return
    line = {
        "metric": "reconciled key bits/s", "value": value, "unit": "bit/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"f32": "f32", "f16": "f16+f32", "i8": "i8"}[prec],
        "data": "synthetic: seeded Philox Gaussian quadratures and seeded regular dv=3 LDPC codes",
        "config": {"workload": sweep_workload(args.rate_rule) if args.decoder == "sp_f32" else
                   sweep_workload(args.rate_rule).replace("FP32 sum-product flooding", f"decoder {args.decoder} (failed frames re-decoded "
                                                                 f"in FP32, {args.fallback} algorithm)"
                                    if opts.fallback_f32 else args.decoder),
                   "samples_per_snr": N_SAMPLES, "snr": list(SNRS),
                   "lower_slices": "soft (decoder posteriors)" if args.soft_chain else "hard (decoded bits)",
                   "sub_block_log2": list(LOGNS), "slices": M_SLICES, "algo": algo, "prec": prec,
                   "fallback_f32": opts.fallback_f32,
                   "max_iter": MAX_ITER, "rate_rule": args.rate_rule if args.rate_rule == "backoff" else "0.95 x capacity",
                   "rates": {f"snr{int(s)}_n2^{ln}": [rate_of[(s, ln, j)] for j in range(M_SLICES)]
                             for s in SNRS for ln in LOGNS},
                   "l2": "inputs larger than L2 (x, y 512 MiB each per SNR; edge messages up to 1.5 GiB)",
                   "raw_decoded_bits_per_s": raw_bits / (ms_step / 1e3),
                   "edge_updates_per_s": edge_updates * world / (ms_step / 1e3),
                   # Sec. III-C: E_j = 7G operations per iteration, so the time per operation is
                   # the step time over 7 x the edge-updates executed (the paper's GPU: 3.2e-9 s)
                   "equivalent_c_h_s": (ms_step / 1e3) / (7 * edge_updates * world) if edge_updates else None,
                   "fer_per_slice": fer, "mean_iters_per_slice": mean_iters,
                   "fer_plain_sp_f32_per_slice": fer_plain,
                   "frame_block_occupancy": occ,
                   "beta_per_point": beta_pt,
                   "nr_optimum": nr_opt,
                   "net_key_bits_per_s": net_bits * world / (ms_step / 1e3),
                   "net_key_note": ("(Pi(M(Y)) - m + sum_j R_j) x samples of sub-blocks with every slice reconciled, "
                                    "over the device step time (Eq. beta's numerator; before parameter estimation "
                                    "and privacy amplification)"),
                   "rate_tables_note": ("the back-off rates were calibrated with layered offset min-sum trials "
                                        "(<= 50 iterations); the line decodes with the form named in 'algo'")
                   if args.rate_rule == "backoff" else None,
                   "error_vs_oracle": err_oracle,
                   "code_residual_4cycles": residual, "setup_s": round(setup_s, 1),
                   "timing": ("step captured once as a CUDA graph and replayed, the five sub-block lengths of "
                              "a block decoding concurrently (one side stream each) and the two blocks "
                              "overlapping; kernel figures from the same steps run eagerly with per-launch "
                              "events, blocks and lengths one after another" if graph is not None else "eager"),
                   "workspace_gib": round((rws.numel() + (rws_b.numel() if rws_b is not None else 0)) / 2**30, 1),
                   "profiled_ms_per_step": ms_profiled / args.steps},
        "roofline": roof,
        "kernels": kernels,
        "cpu_baseline": cpu,
        "e2e": ({"value": good_bits / (t_e2e_max / args.steps / 1e3), "unit": "bit/s",
                 "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                 "ms_per_step": t_e2e_max / args.steps,
                 "api": "qkdrec_reconcile with host x, y and host outputs (Alice's slices packed 8 per byte, "
                        "converged flags, iteration counts of every point)",
                 "same_result_as_device_run": e2e_same} if t_e2e else None),
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def error_vs_oracle(q, torch, dev, codes, codes_h, rate_of, host_x, host_y, opts, frames=8, iters=4):
    """Per-result error of the decoder form against the FP64 oracle on a sample:
    the first `frames` sub-blocks of n = 2^12 of every decoded slice at both SNRs,
    with Bob's lower slices as the reconciled ones.  Each side computes its own
    inputs (GPU: quantiser, slice LLR and syndrome kernels; oracle: its own FP64
    quantiser, LLRs and syndromes from the same synthetic x, y).
      llr_*         channel LLRs, |gpu - oracle|
      post*_        posteriors after `iters` iterations without stopping test, same
                    algorithm (FP64 on the oracle side), relative |gpu - oracle| /
                    max(|oracle|, 1), and the fraction of hard decisions that differ
      decoded_*     full decodes as in the bench (stopping test, <= MAX_ITER, the
                    FP32 re-decode of failed frames): decoded bits and frames that
                    differ from the oracle's FP64 decode of the same algorithm."""
    import oracle
    ln, n = 12, 1 << 12
    cnt = frames * n
    algo = opts.algo
    o_alg = ("i" + algo) if opts.prec == "i8" else algo
    fixed = q.DecodeOpts(algo=algo, prec=opts.prec, max_iter=iters, early_stop=False)
    acc = dict(llr_max_abs=0.0, llr_mean_abs=[], post_max_rel=0.0, post_mean_rel=[], bits_differ=[],
               decoded_bits_differ=[], decoded_frames_differ=[])
    for snr in SNRS:
        lo, hi = oracle.quantiser_range(snr)
        sn = snr ** -0.5
        x = host_x[snr][:cnt].numpy()
        y = host_y[snr][:cnt].numpy()
        _, bob_o = oracle.quantise(y, M_SLICES, lo, hi)
        xd = torch.from_numpy(x).to(dev)
        _, bob_g = q.qkdrec_quantise_slices(torch.from_numpy(y).to(dev), M_SLICES, lo, hi, want_idx=False)
        for j in range(M_SLICES):
            r = rate_of[(snr, ln, j)]
            if r <= 0:
                continue
            rp, ci = codes_h[(ln, j, r)][:2]
            c = codes[(ln, j, r)]
            llr_g = q.qkdrec_slice_llr(xd, M_SLICES, j, lo, hi, sn, bob_g[:j] if j else None)
            llr_o = oracle.slice_llr(x, bob_o[:j] if j else None, j, M_SLICES, lo, hi, sn)
            d = np.abs(llr_g.cpu().numpy().astype(np.float64) - llr_o)
            acc["llr_max_abs"] = max(acc["llr_max_abs"], float(d.max()))
            acc["llr_mean_abs"].append(float(d.mean()))
            syn_g = q.qkdrec_syndrome(c, bob_g[j].view(frames, n))
            syn_o = oracle.syndrome(rp, ci, bob_o[j].reshape(frames, n))
            g4 = q.qkdrec_decode_batch(c, llr_g.view(frames, n), syn_g, fixed, want_post=True)
            o4 = oracle.decode(rp, ci, llr_o.reshape(frames, n), syn_o, o_alg, max_iter=iters, early_stop=False)
            rel = np.abs(g4["post"].cpu().numpy() - o4["post"]) / np.maximum(np.abs(o4["post"]), 1.0)
            acc["post_max_rel"] = max(acc["post_max_rel"], float(rel.max()))
            acc["post_mean_rel"].append(float(rel.mean()))
            acc["bits_differ"].append(float(np.mean(g4["bits"].cpu().numpy() != o4["bits"])))
            gf = q.qkdrec_decode_batch(c, llr_g.view(frames, n), syn_g, opts)
            of = oracle.decode(rp, ci, llr_o.reshape(frames, n), syn_o, o_alg, max_iter=MAX_ITER)
            if opts.fallback_f32:
                # the oracle re-decodes its failed frames with the same FP32 rule
                o2 = "sp_flood" if opts.fallback_f32 == "sp" else algo
                bad = ~of["converged"].astype(bool)
                if bad.any():
                    redo = oracle.decode(rp, ci, llr_o.reshape(frames, n)[bad], syn_o[bad], o2, max_iter=MAX_ITER)
                    of["bits"][bad] = redo["bits"]
            gb = gf["bits"].cpu().numpy()
            acc["decoded_bits_differ"].append(float(np.mean(gb != of["bits"])))
            acc["decoded_frames_differ"].append(float(np.mean(np.any(gb != of["bits"], axis=1))))
    mean = lambda v: float(np.mean(v)) if v else 0.0
    return {"sample": f"{frames} sub-blocks of n={n} per decoded slice at SNR 3 and 15, Bob's lower slices",
            "iterations": iters, "llr_max_abs": acc["llr_max_abs"], "llr_mean_abs": mean(acc["llr_mean_abs"]),
            "post_max_rel": acc["post_max_rel"], "post_mean_rel": mean(acc["post_mean_rel"]),
            "bits_differ": mean(acc["bits_differ"]), "decoded_bits_differ": mean(acc["decoded_bits_differ"]),
            "decoded_frames_differ": mean(acc["decoded_frames_differ"])}


def source_region_sha(path, start, end):
    """SHA-256 prefix of the source text from the line holding `start` up to the
    line holding `end` (the kernel and the device helpers it compiles from)."""
    import hashlib
    text = open(path).read()
    i = text.index(start)
    j = text.index(end, i)
    return hashlib.sha256(text[i:j].encode()).hexdigest()[:16]


def load_traffic(kernel, d):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled by the
    units this run's launches processed; None if no capture matches the current
    source of that kernel."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        t = json.load(open(path))[kernel]
        src = os.path.join(ROOT, "paper_2108_08418_b300", "csrc", t["source"])
        sha = source_region_sha(src, *t["region"])
    except (OSError, ValueError, KeyError):
        return None
    if sha != t.get("source_sha"):
        return None
    return t["dram_bytes_per_unit"] * d["units"] / d["launches"]


# ----------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    if args.workload == "uneven":
        run_reference_uneven(args, world, cores)
        return
    if args.workload == "woms":
        run_reference_woms(args, world, cores)
        return
    per_snr = max(1, min(cores, 8) // 2)
    rate_of = load_sweep_rates() if args.rate_rule == "backoff" else None
    for w in range(args.warmup):
        oracle_sample(w, per_snr, cores, rate_of)
    goods, walls, nfr = 0, 0.0, 0
    for s in range(args.steps):
        g, wall, n = oracle_sample(args.warmup + s, per_snr, cores, rate_of)
        goods += g
        walls += wall
        nfr = n
    value = goods / walls
    line = {
        "impl": "reference", "metric": "reconciled key bits/s", "value": value, "unit": "bit/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": walls / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded Philox Gaussian quadratures and seeded regular dv=3 LDPC codes",
        "config": {"workload": sweep_workload(args.rate_rule), "sample": "per step: sub-blocks of n=4096 at SNR 3 and 15"},
        "cpu_baseline": {"value": value, "unit": "bit/s", "cores": min(cores, nfr), "kind": "oracle",
                         "sample": f"{nfr} sub-blocks of n=4096 per step, each reconciled over all 5 slices"},
        "e2e": {"value": value, "unit": "bit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_woms(args, world, cores):
    for w in range(args.warmup):
        oracle_woms_sample(w, cores)
    frames, walls, procs = 0, 0.0, 1
    for s in range(args.steps):
        k, wall, procs = oracle_woms_sample(args.warmup + s, cores)
        frames += k
        walls += wall
    value = frames / (WOMS_F * walls)
    line = {
        "impl": "reference", "metric": "weighted min-sum training steps/s", "value": value, "unit": "step/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded Philox Gaussian quadratures and a seeded regular (3,6) LDPC code",
        "config": {"workload": WOMS_WORKLOAD, "sample": f"per step: {frames // max(args.steps, 1)} of the {WOMS_F} "
                                                        f"frames, forward and gradient (no optimiser update)"},
        "cpu_baseline": {"value": value, "unit": "step/s", "cores": procs, "kind": "oracle",
                         "sample": f"{frames // max(args.steps, 1)} frames per step, {procs} processes"},
        "e2e": {"value": value, "unit": "step/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_uneven(args, world, cores):
    setup = uneven_setup(UNEVEN_SEED, max(1, min(cores, 16)), args.rate_rule)
    per = 3 * max(1, min(cores, 8))
    algo, max_iter = ("sp_flood", MAX_ITER) if args.uneven_decoder == "sp_f32" else ("oms_layered", UNEVEN_MAX_ITER)
    for w in range(args.warmup):
        oracle_uneven_sample(w, per, cores, setup, algo, max_iter)
    goods, walls, nfr = 0, 0.0, 0
    for s in range(args.steps):
        g, wall, nfr = oracle_uneven_sample(args.warmup + s, per, cores, setup, algo, max_iter)
        goods += g
        walls += wall
    value = goods / walls
    line = {
        "impl": "reference", "metric": "reconciled key bits/s", "value": value, "unit": "bit/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": walls / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded Philox Gaussian quadratures and seeded regular dv=3 LDPC codes",
        "config": {"workload": UNEVEN_WORKLOAD, "sample": f"per step: {nfr} frames of n=4096 of the batch"},
        "cpu_baseline": {"value": value, "unit": "bit/s", "cores": min(cores, nfr), "kind": "oracle",
                         "sample": f"{nfr} frames of n=4096 per step, each reconciled over all 5 slices"},
        "e2e": {"value": value, "unit": "bit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- profiling case
CASES = {
    # the slice LLR kernel on 2^24 samples of the sweep's data (SNR 3, slice 2, Bob's
    # lower slices): the small case for ncu
    "slice_llr": dict(llr=(3.0, 2), count=1 << 24),
    # the same kernel on the top slice at SNR 15 (two candidates per sample)
    "slice_llr_j4": dict(llr=(15.0, 4), count=1 << 24),
    # one slice decode of the sweep at n = 2^16 and 512 frames (edge messages 400 MB,
    # larger than L2; ~1 GB on the device): the small case for ncu --set full
    "decode_sp_f32": dict(logn=16, frames=512, rate=0.84375, algo="sp_flood", prec="f32", iters=5),
    "decode_oms_f32": dict(logn=16, frames=512, rate=0.84375, algo="oms_flood", prec="f32", iters=5),
    "decode_layered_f32": dict(logn=16, frames=512, rate=0.84375, algo="oms_layered", prec="f32", iters=5),
    "decode_oms_i8": dict(logn=16, frames=512, rate=0.84375, algo="oms_flood", prec="i8", iters=5),
    "decode_oms_f16": dict(logn=16, frames=512, rate=0.84375, algo="oms_flood", prec="f16", iters=5),
    # the plan decoder on a small uneven batch: 96 frames of n = 2^16, 192 of 2^14, 384 of 2^12
    # (rate 0.84375; ~0.9 GB on the device)
    # layered min-sum of a quasi-cyclic code (Z = 2^13, 3 x 8 base matrix: n = 2^16, rate 0.625),
    # 512 frames, 5 iterations: with the TMA-staged path, and the same matrix without the structure
    "decode_layered_qc_f32": dict(qc=(8192, 8), frames=512, iters=5, attach=True),
    "decode_layered_qcplain_f32": dict(qc=(8192, 8), frames=512, iters=5, attach=False),
    "plan_layered": dict(groups=((16, 96), (14, 192), (12, 384)), rate=0.84375, iters=5,
                         tuning=dict(frames_per_tile=8, threads_per_cta=1024, stage_depth=4, ctas_per_tile=8)),
    "plan_layered_cta": dict(groups=((16, 96), (14, 192), (12, 384)), rate=0.84375, iters=5,
                             tuning=dict(frames_per_tile=8, threads_per_cta=1024, stage_depth=4, ctas_per_tile=1)),
    "plan_layered_ft32": dict(groups=((16, 96), (14, 192), (12, 384)), rate=0.84375, iters=5,
                              tuning=dict(frames_per_tile=32, threads_per_cta=512, stage_depth=8, ctas_per_tile=8)),
    # the shape the autotuner picks on the uneven batch: 4 frames per lane, 2 tiles per item
    "plan_layered_v4": dict(groups=((16, 96), (14, 192), (12, 384)), rate=0.84375, iters=5,
                            tuning=dict(frames_per_tile=32, threads_per_cta=512, stage_depth=4, ctas_per_tile=8,
                                        tiles_per_item=2, frames_per_lane=4, sparse_frames=4)),
}


def run_qc_case(args, c):
    import torch
    import paper_2108_08418_b300 as q
    Z, nb = c["qc"]
    n, F = Z * nb, c["frames"]
    rp, ci, S, _ = synth.make_qc_code(4242, Z, nb)
    code = q.Code(n, rp, ci)
    if c["attach"]:
        code.set_qc(Z, 3, nb, S)
    g = synth.philox(79)
    b = g.integers(0, 2, size=(F, n)).astype(np.uint8)
    llr = ((2 / 0.6 ** 2) * ((1.0 - 2.0 * b) + 0.6 * g.standard_normal((F, n)))).astype(np.float32)
    bd, ld = torch.from_numpy(b).cuda(), torch.from_numpy(llr).cuda()
    synd = q.qkdrec_syndrome(code, bd)
    opts = q.DecodeOpts(algo="oms_layered", prec="f32", max_iter=c["iters"], early_stop=False)
    ws = q.workspace_for(code, F, opts, "cuda")
    q.qkdrec_profile_begin()
    for _ in range(args.warmup + args.steps):
        q.qkdrec_decode_batch(code, ld, synd, opts, workspace=ws)
    torch.cuda.synchronize()
    st = q.qkdrec_profile_end()
    k = "layer_qc_tma" if c["attach"] else "layer_oms_f32"
    print(f"case {args.case}: n={n} F={F} {k}: {st[k]['ms'] / st[k]['launches']:.4f} ms/launch, "
          f"{st[k]['bytes'] / st[k]['ms'] / 1e6:.1f} GB/s; timeouts {q.qkdrec_qc_timeouts()}", flush=True)


def run_plan_case(args, c):
    import torch
    import paper_2108_08418_b300 as q
    g = synth.philox(78)
    groups = []
    for logn, F in c["groups"]:
        n = 1 << logn
        rp, ci, _ = synth.make_regular_code(code_seed(logn, 3), n, synth.checks_for_rate(n, c["rate"]))
        code = q.Code(n, rp, ci)
        b = g.integers(0, 2, size=(F, n)).astype(np.uint8)
        llr = ((2 / 0.52 ** 2) * ((1.0 - 2.0 * b) + 0.52 * g.standard_normal((F, n)))).astype(np.float32)
        bd = torch.from_numpy(b).cuda()
        groups.append(dict(code=code, llr=torch.from_numpy(llr).cuda(), synd=q.qkdrec_syndrome(code, bd),
                           bits=torch.empty_like(bd), iters=torch.empty(F, dtype=torch.int32, device="cuda"),
                           conv=torch.empty(F, dtype=torch.uint8, device="cuda")))
    opts = q.DecodeOpts(algo="oms_layered", prec="f32", max_iter=c["iters"], early_stop=False)
    plan = q.Plan(groups, opts, c["tuning"])
    ws = plan.workspace()
    for _ in range(args.warmup + args.steps):
        plan.launch(ws)
    torch.cuda.synchronize()
    print(f"case {args.case}: frames={sum(F for _, F in c['groups'])} "
          f"edge-frames/launch={sum(gr['code'].E * gr['llr'].shape[0] for gr in groups)}", flush=True)


def run_case(args):
    """Run one small fixed decode W + K times (no timing output): the command ncu captures."""
    import torch
    import paper_2108_08418_b300 as q
    from paper_2108_08418_b300 import build as qbuild
    qbuild.build()
    c = CASES[args.case]
    if "llr" in c:
        snr, j = c["llr"]
        lo, hi = q.qkdrec_quantiser_range(snr)
        x, y = synth.gaussian_pair(DATA_SEED[snr], c["count"], snr)
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        _, bits = q.qkdrec_quantise_slices(yd, M_SLICES, lo, hi, want_idx=False)
        out = torch.empty_like(xd)
        for _ in range(args.warmup + args.steps):
            q.qkdrec_slice_llr(xd, M_SLICES, j, lo, hi, snr ** -0.5, bits[:j] if j else None, out=out)
        torch.cuda.synchronize()
        print(f"case {args.case}: {c['count']} samples, slice {j} at SNR {snr}", flush=True)
        return
    if "groups" in c:
        run_plan_case(args, c)
        return
    if "qc" in c:
        run_qc_case(args, c)
        return
    n, F = 1 << c["logn"], c["frames"]
    M = synth.checks_for_rate(n, c["rate"])
    rp, ci, _ = synth.make_regular_code(code_seed(c["logn"], 3), n, M)
    code = q.Code(n, rp, ci)
    g = synth.philox(77)
    b = g.integers(0, 2, size=(F, n)).astype(np.uint8)
    llr = ((2 / 0.52 ** 2) * ((1.0 - 2.0 * b) + 0.52 * g.standard_normal((F, n)))).astype(np.float32)
    bd, ld = torch.from_numpy(b).cuda(), torch.from_numpy(llr).cuda()
    synd = q.qkdrec_syndrome(code, bd)
    opts = q.DecodeOpts(algo=c["algo"], prec=c["prec"], max_iter=c["iters"], early_stop=False)
    ws = q.workspace_for(code, F, opts, "cuda")
    for _ in range(args.warmup + args.steps):
        q.qkdrec_decode_batch(code, ld, synd, opts, workspace=ws)
    torch.cuda.synchronize()
    print(f"case {args.case}: n={n} F={F} edges/launch={code.E * F}", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end loop")
    ap.add_argument("--case", choices=sorted(CASES), help="run one small fixed decode (for ncu)")
    ap.add_argument("--workload", choices=["sweep", "uneven", "woms"], default="sweep",
                    help="sweep: the block-size sweep (default); uneven: the one-graph uneven batch; "
                         "woms: training of the weighted min-sum decoder")
    ap.add_argument("--train-steps", type=int, default=60, help="woms: training steps before the FER check")
    ap.add_argument("--calibrate", action="store_true",
                    help="run the rate back-off of the workload and write its table (sweep_rates.json, "
                         "uneven_rates.json)")
    ap.add_argument("--rates-out", help="where --calibrate writes the table (default: uneven_rates.json)")
    ap.add_argument("--decoder", choices=sorted(DECODERS), default="sp_f32",
                    help="sweep workload: decoder form (default FP32 sum-product; others re-decode failures in FP32)")
    ap.add_argument("--soft-chain", action="store_true",
                    help="sweep: slice LLRs from the lower slices' decoder posteriors (soft) instead of their bits")
    ap.add_argument("--uneven-parts", type=int, default=2,
                    help="uneven workload: parts of the batch decoded on their own streams")
    ap.add_argument("--uneven-decoder", choices=["plan", "sp_f32"], default="plan",
                    help="uneven workload: one persistent layered min-sum plan launch per slice (default) or the "
                         "plain FP32 sum-product batch decoder on every group")
    ap.add_argument("--fallback", choices=["sp", "same"], default="sp",
                    help="low-precision decoders: re-decode failed frames with FP32 sum-product (default) or "
                         "with the same algorithm in FP32")
    ap.add_argument("--rate-rule", choices=["backoff", "capacity"], default="backoff",
                    help="rates: the Sec. V-B back-off table, i.e. reconciled bits at a fixed FER target "
                         "(default), or 0.95 x slice capacity")
    args = ap.parse_args()
    if args.case:
        run_case(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.calibrate:
        run_calibrate(args)
    elif args.workload == "uneven":
        run_uneven(args)
    elif args.workload == "woms":
        run_woms(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
