#!/usr/bin/env python
"""Benchmark of the exact Skolem/Langford count on GB300.

Default workload (one "step"): the mid-size exact counts S(n) and L(n) for
n = 16..20, one launch per job, residues modulo three 62-bit primes and the
CRT on the host -- 2 * sum_{n=16..20} 2^{2n-1} = 1.46e12 +-1 terms.
Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (Algorithm 1 written out plainly, C,
all host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("±1-terms/s and INT32 peak fraction for exact S(n),L(n); "
          "PT error vs time, learned/plain")
JOBS = [(0, n) for n in range(16, 21)] + [(1, n) for n in range(16, 21)]
WORKLOAD = "exact S(n), L(n), n=16..20 (2^31..2^39 terms each), one launch per job, 3 x 62-bit moduli + CRT"


def terms_per_step():
    return sum(1 << (2 * n - 1) for _, n in JOBS)


def groups(delta, n):
    """The kernel's grouping of c_1..c_n into int32 products (bound < 2^31)."""
    g, prod = 0, 1
    for k in range(1, n + 1):
        L = max(2 * n - k - delta, 1)
        if k == 1 or prod * L > 2147483647:
            g += 1
            prod = 1
        prod *= L
    return g


def group_bits(delta, n):
    """Bit lengths of the products of the bounds L_k = 2n - k - delta over the
    groups 0..j (the kernel sizes its limbs from these)."""
    bits, prod, g_prev, k0 = [], 1, None, 1
    g, gp = 0, 1
    starts = []
    for k in range(1, n + 1):
        L = max(2 * n - k - delta, 1)
        if k == 1 or gp * L > 2147483647:
            starts.append(k)
            gp = 1
        gp *= L
    starts.append(n + 1)
    for j in range(len(starts) - 1):
        for k in range(starts[j], starts[j + 1]):
            prod *= max(2 * n - k - delta, 1)
        bits.append(prod.bit_length())
    return bits


def alg_ops_per_term(variant, n, nprimes=3):
    """32-bit integer operations one term of Lemma 2.1 needs, whatever form
    the kernel takes: n correlation updates (one add each); the exact product
    of the n factors -- n - g int32 multiplies inside the g int32 groups
    (bound < 2^31 each, greedy), then, per further group, one 32x32->64
    multiply per 32-bit word of the running product (counted as two
    operations: it yields two words); and one add per 32-bit word of the
    signed accumulate.  The moduli enter once per work item, not per term."""
    delta = 1 if variant == 1 else 0
    bits = group_bits(delta, n)
    g = len(bits)
    words = [max(1, (b + 31) // 32) for b in bits]
    wide = sum(words[:-1])
    acc = (bits[-1] + 1 + 31) // 32
    return n + (n - g) + 2 * wide + acc


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle

def oracle_sample(seconds_target=12.0):
    """The oracle as it stands (plain Algorithm 1 summand per assignment,
    reduced mod each prime), on all host cores: work items of S(20) / L(20)
    with 2^12 terms each, three moduli.  Returns (terms/s, cores, sample,
    seconds of the timed sample)."""
    import concurrent.futures as cf
    import oracle
    p = [4611686018427387847, 4611686018427387817, 4611686018427387787]
    cores = os.cpu_count() or 1
    m = 12
    t0 = time.perf_counter()
    oracle.partial_sum_mod(0, 20, m, 0, p[0])        # builds + warms the library
    one = time.perf_counter() - t0
    per_core = max(1, int(seconds_target / max(one * 3, 1e-3)))
    items = [(v, q) for q in range(per_core * cores) for v in (0, 1)][:per_core * cores]

    def work(vq):
        v, q = vq
        for pi in p:
            oracle.partial_sum_mod(v, 20, m, q * 977 % (1 << 27), pi)
        return 1

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(work, items))
    dt = time.perf_counter() - t0
    terms = len(items) * (1 << m)
    return (terms / dt, cores,
            f"{len(items)} work items of S(20)/L(20), 2^{m} terms each, 3 moduli, {dt:.1f} s", dt)


# ------------------------------------------------------------------ main

def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def reduce_max_over_ranks(values, device):
    """Maximum over the ranks of each of a few floats (the slowest rank's
    time); the values unchanged with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def job_throughput(world, steps, units_per_step, seconds):
    """Units processed by all ranks (one replica of the workload each) per
    second of the slowest rank."""
    return world * steps * units_per_step / seconds


def source_hash():
    h = hashlib.sha256()
    for f in ("sk_exact.cuh", "sk_exact_launch.cuh"):
        with open(os.path.join(ROOT, "paper_1507_00315_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """dram bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "exact_kernel_traffic.json")
    try:
        d = json.load(open(p))
        if d.get("source_hash") == source_hash():
            return d["dram_bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        pass
    return None


def recorded_imad_busy():
    p = os.path.join(ROOT, "profiles", "exact_kernel_traffic.json")
    try:
        d = json.load(open(p))
        if d.get("source_hash") == source_hash():
            return d.get("fmaheavy_busy_frac")
    except (OSError, ValueError, KeyError):
        pass
    return None


def run_extra(args, world, rank, local):
    """Extra workloads, one JSON line each: --config batch (all three
    problems, n = 4..nmax, one persistent graph-captured launch vs one launch
    per job), --config large (S(24), L(24), four moduli, checkpointed),
    --config pt (tempering error vs GPU time, plain and learned proposal) and
    --config pt-large (tempering at the orders of Tables 7 / 8 above 24)."""
    import torch
    import paper_1507_00315_gb300 as sk
    torch.cuda.set_device(local)
    sh = torch.cuda.current_stream().cuda_stream
    if args.config == "batch":
        line = run_batch_bench(args, sk, sh)
    elif args.config == "slices":
        line = run_slices_bench(args, sk, sh)
    elif args.config == "ie":
        line = run_ie_bench(args, sk, sh)
    elif args.config == "symmetry":
        line = run_symmetry_bench(args, sk, sh)
    elif args.config == "pt":
        line = run_pt_bench(args, sk, sh)
    elif args.config == "pt-large":
        line = run_pt_large_bench(args, sk, sh)
    elif args.config == "pt-bias":
        line = run_pt_bias_bench(args, sk, sh)
    elif args.config == "pt-gain":
        line = run_pt_gain_bench(args, sk, sh)
    elif args.config == "train":
        line = run_train_bench(args, sk, sh)
    else:
        import tempfile
        res = {}
        names = {sk.SYMMETRY_NEGATION: "", sk.SYMMETRY_NEGATION_EVEN: " lemma 2.4",
                 sk.SYMMETRY_REVERSAL: " lemma 2.3", sk.SYMMETRY_REVERSAL_EVEN: " lemmas 2.3 + 2.4"}
        want = {(0, 24): EXACT_S[24], (1, 24): EXACT_L[24]}
        for sym in args.symmetries:
            for v, n in ((0, 24), (1, 24)):
                path = os.path.join(args.ckpt_dir or tempfile.gettempdir(),
                                    f"sk_ckpt_{v}_{n}_s{sym}.txt")
                c, rep = sk.count_ex(v, n, nprimes=4, checkpoint=path, stream=sh, symmetry=sym)
                key = f"{'SL'[v]}({n})" + names[sym]
                res[key] = {"count": str(c), "equals_paper": c == want[(v, n)],
                            "kernel_s": rep["kernel_ms"] / 1e3,
                            "wall_s": rep["wall_ms"] / 1e3, "chunks": rep["chunks_total"],
                            "resumed": rep["chunks_resumed"], "terms": rep["terms"],
                            "walk_bits": rep["walk_bits"],
                            "terms_per_s": rep["terms"] / max(rep["kernel_ms"], 1e-9) * 1e3}
        line = {"metric": "exact S(24), L(24): terms/s, checkpointed, 4 moduli",
                "config": {"workload": "S(24), L(24): 2^47 terms each with Lemma 2.2 alone, 2^46 "
                                       "with Lemma 2.4, (1/2 + 2^-9) 2^47 with Lemma 2.3; 3 moduli + "
                                       "check modulus",
                           "symmetries": [names[s].strip() or "lemma 2.2" for s in args.symmetries]},
                "unit": "terms/s", "results": res}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_batch_bench(args, sk, sh):
    """The batched sweep: {Skolem, Langford, hooked} x n = 4..nmax, 3 moduli,
    as one persistent graph-captured launch and as one launch per job
    (largest job first, same stream), each timed over `steps` (at least 5)
    separate calls after one warm-up call, reported as median, minimum and
    maximum of the device time between events around the whole sweep; the
    autotuned persistent run (walk width and block size per job) beside them.
    Every mode must give the same counts."""
    import statistics as stt
    jobs = [(v, n) for v in (0, 1, 2) for n in range(4, args.nmax + 1)]
    reps = max(5, args.steps)
    modes = [("per_job", {"mode": sk.BATCH_PER_JOB}), ("persistent_graph", {})]
    if not args.no_autotune:
        modes.append(("persistent_graph_autotuned", {"autotune": True}))
    out, counts = {}, None
    for name, kw in modes:
        times, rep = [], None
        for i in range(reps + 1):
            c, st, rep = sk.count_batch(jobs, repeats=1, stream=sh, **kw)
            assert counts is None or c == counts, name
            counts = c
            if i:                                   # the first call warms up
                times.append(rep["kernel_ms"])
        med = stt.median(times)
        out[name] = {"kernel_ms_median": med, "kernel_ms_min": min(times),
                     "kernel_ms_max": max(times), "repeats": reps,
                     "spread_frac": (max(times) - min(times)) / med,
                     "terms_per_s_median": rep["terms"] / (med / 1e3), "launches": rep["launches"],
                     "block_threads": rep["block_threads"], "grid": rep["grid"]}
    pj, pg = out["per_job"], out["persistent_graph"]
    return {"metric": "batched sweep terms/s, persistent graph launch vs one launch per job",
            "config": {"workload": f"{{Skolem, Langford, hooked}} x n=4..{args.nmax}, 3 moduli",
                       "jobs": len(jobs), "terms": sum(1 << (2 * n - 1) for _, n in jobs)},
            "unit": "terms/s", "results": out,
            "speedup_persistent_vs_per_job_median": pj["kernel_ms_median"] / pg["kernel_ms_median"],
            # beyond the spread: the slowest persistent run beats the fastest per-job run
            "persistent_beats_per_job_beyond_spread": pg["kernel_ms_max"] < pj["kernel_ms_min"]}


def run_symmetry_bench(args, sk, sh):
    """What the extra symmetries buy on the mid-size workload: every job with
    Lemma 2.2 alone (2^{2n-1} terms), with Lemma 2.4 on top (half of them,
    in the existence classes; none outside), with Lemma 2.3 on top (the
    mirrored walk, about half) and with both (about a quarter in the
    existence classes), best of `steps` runs each.  The counts must
    agree.  Reported per job: kernel time, terms evaluated, and the
    equivalent rate 2^{2n-1} / time (the plain half-sum's terms per second of
    the run that skips some of them)."""
    modes = (("lemma_2_2", sk.SYMMETRY_NEGATION), ("lemma_2_4", sk.SYMMETRY_NEGATION_EVEN),
             ("lemma_2_3", sk.SYMMETRY_REVERSAL), ("lemma_2_3_and_2_4", sk.SYMMETRY_REVERSAL_EVEN))
    out, tot = {}, {name: 0.0 for name, _ in modes}
    for v, n in JOBS:
        row, c0 = {}, None
        for name, sym in modes:
            best = None
            for _ in range(max(1, args.steps)):
                c, rep = sk.count_ex(v, n, stream=sh, symmetry=sym)
                assert c0 is None or c == c0, (v, n, name)
                c0 = c
                best = rep["kernel_ms"] if best is None else min(best, rep["kernel_ms"])
            row[name] = {"kernel_ms": best, "terms_evaluated": rep["terms"],
                         "walk_bits": rep["walk_bits"], "symmetry_used": rep["symmetry"],
                         # no terms: the sum vanishes by Lemma 2.4's sign, nothing ran
                         "equivalent_terms_per_s": ((1 << (2 * n - 1)) / best * 1e3
                                                    if rep["terms"] else None)}
            tot[name] += best
        out[f"{'SL'[v]}({n})"] = row
    return {"metric": "exact count time with Lemma 2.2 alone, + Lemma 2.4, + Lemma 2.3",
            "unit": "ms", "config": {"workload": WORKLOAD},
            "results": out, "total_kernel_ms": tot,
            "speedup_vs_lemma_2_2": {k: tot["lemma_2_2"] / v for k, v in tot.items() if v > 0}}


def run_ie_bench(args, sk, sh):
    """The inclusion-exclusion count (Sec. 2, third approach) beside the
    algebraic count of Lemma 2.1 on the mid-size workload: each job counted
    both ways (the counts must agree bit for bit), best of `steps` runs of
    each.  Inclusion-exclusion sums 2^{2n} terms, the algebraic count 2^{2n-1}
    (Lemma 2.2); both walks do the same work per term (n correlation updates,
    the exact product, one signed accumulate)."""
    peak = sk.int32_peak(1)[0]
    out = {}
    for v, n in JOBS:
        row = {}
        for name, fn in (("algebraic", sk.count_ex), ("inclusion_exclusion",
                                                      sk.count_inclusion_exclusion)):
            best, c0 = None, None
            for _ in range(max(1, args.steps)):
                c, rep = fn(v, n, stream=sh)
                assert c0 is None or c == c0
                c0 = c
                best = rep["kernel_ms"] if best is None else min(best, rep["kernel_ms"])
            rate = rep["terms"] / (best / 1e3)
            row[name] = {"count": str(c0), "terms": rep["terms"], "kernel_ms": best,
                         "terms_per_s": rate,
                         "int32_frac": alg_ops_per_term(v, n) * rate / peak}
        assert row["algebraic"]["count"] == row["inclusion_exclusion"]["count"], (v, n, row)
        row["time_ratio_ie_vs_algebraic"] = (row["inclusion_exclusion"]["kernel_ms"] /
                                             row["algebraic"]["kernel_ms"])
        out[f"{'SL'[v]}({n})"] = row
    return {"metric": "exact count terms/s: inclusion-exclusion vs the algebraic method",
            "unit": "terms/s",
            "config": {"workload": WORKLOAD.replace("one launch per job", "each job both ways"),
                       "int32_peak_tops": peak / 1e12,
                       "peak_source": "measured: sk_int32_peak mode 1, same run"},
            "results": out}


SLICE_CASES = [(0, 21), (1, 23), (0, 24), (1, 24), (0, 25), (1, 27), (0, 28), (1, 28), (0, 29),
               (2, 30), (1, 31)]


def run_slices_bench(args, sk, sh):
    """Timed slices of the large exact counts: the first 2^slice_bits terms
    (one checkpoint chunk) of S(21) .. S(29), L(23) .. L(31) and hooked
    Skolem n = 30, four moduli, Lemma 2.4 on where it applies.  The walk
    width is the plan's, capped so that a slice holds at least 2^17 work items
    (the GPU holds ~78k threads; at n = 31 the plan walks 2^31 terms per item,
    which a slice could not spread over the GPU).  A full count's time is
    projected from the slice's rate (every work item walks the same Gray
    schedule, so the rate does not depend on which items are timed)."""
    import tempfile
    peak = sk.int32_peak(1)[0]
    out = {}
    d = args.ckpt_dir or tempfile.mkdtemp(prefix="sk_slices_")
    for v, n in SLICE_CASES[:args.pt_cases + 2]:
        sym = sk.SYMMETRY_NEGATION_EVEN
        path = os.path.join(d, f"slice_{v}_{n}.ckpt")
        if os.path.exists(path):
            os.remove(path)
        plan = sk.count_plan(v, n, nprimes=4, checkpoint=path, symmetry=sym)
        m = min(plan["walk_bits"], max(plan["inner_bits"], args.slice_bits - 17))
        plan = sk.count_plan(v, n, nprimes=4, checkpoint=path, symmetry=sym, walk_bits=m)
        chunk = 1 << max(0, args.slice_bits - m)
        best = None
        for rep_i in range(2):                  # first call warms the kernel up
            if os.path.exists(path):
                os.remove(path)
            c, rep = sk.count_ex(v, n, nprimes=4, checkpoint=path, chunk_items=chunk,
                                 max_chunks=1, symmetry=sym, stream=sh, walk_bits=m)
            # one chunk; a slice as large as the count is the whole count
            assert rep["chunks_done"] == 1 and (c is None) == (rep["chunks_total"] > 1), rep
            best = rep["kernel_ms"] if best is None else min(best, rep["kernel_ms"])
        os.remove(path)
        terms = chunk << m
        rate = terms / (best / 1e3)
        ops = alg_ops_per_term(v, n)
        out[f"{'SLH'[v]}({n})"] = {
            "terms_total": plan["terms"], "walk_bits": m, "items_total": plan["items"],
            "slice_terms": terms, "slice_ms": best, "terms_per_s": rate,
            "ops_per_term": ops, "int32_frac": ops * rate / peak,
            "projected_hours_full_count": plan["terms"] / rate / 3600.0}
    return {"metric": "exact count slices beyond the mid-size workload: terms/s and projected time",
            "unit": "terms/s",
            "config": {"workload": f"first 2^{args.slice_bits} terms of each count, 4 moduli, "
                                   "Lemma 2.2 + 2.4, the planner's walk width",
                       "int32_peak_tops": peak / 1e12,
                       "peak_source": "measured: sk_int32_peak mode 1, same run"},
            "results": out}


# 32-bit integer operations of one Metropolis iteration of one chain in
# Algorithm 2 (plain proposal): one Philox-4x32-10 block (10 rounds of two
# 32x32->64 products, counted as two operations each, two three-input xors
# and two key additions: 80); the move (pair and slot by two multiply-highs,
# the skip of the current slot, four occupancy updates with their empty-bin
# tests, the energy change, the threshold test, the slot write: 18); the
# histogram count (3); the exchange decision, made for half of the rungs per
# iteration (energy difference, threshold test, the swap: 2).  The count is a
# property of the algorithm, not of the kernel's form.
PT_OPS_PER_LANE_ITERATION = 80 + 18 + 3 + 2

EXACT_S = {16: 700078384, 20: 5717789399488, 24: 102388058845620672,
           25: 1317281759888482688, 28: 3532373626038214732032,
           29: 52717585747603598276736}                        # Table 7, exact column
EXACT_L = {16: 326721800, 20: 2636337861200, 24: 46845158056515936,
           27: 111683611098764903232, 28: 1607383260609382393152}  # Table 8, exact column
# the paper's own tempering estimates (Tables 7 / 8, approximate column)
PAPER_PT_S = {25: 1.317e18, 28: 3.523e21, 29: 5.294e22, 32: 2.213e26, 33: 3.614e27,
              64: 4.1e70}                                  # S(64): the closing section
PAPER_PT_L = {27: 1.115e20, 28: 1.603e21, 31: 5.381e24, 32: 8.812e25}


def run_pt_bench(args, sk, sh):
    """Tempering: relative error against the exact counts (Tables 7 / 8)
    versus GPU time, plain proposal and learned proposal (network trained on
    plain-tempering samples), 32 temperatures x 4096 ladders."""
    import numpy as np
    cases = [(0, 16), (1, 16), (0, 20), (1, 20), (0, 24), (1, 24)][:args.pt_cases]
    out = {}
    for v, n in cases:
        exact = (EXACT_S if v == 0 else EXACT_L)[n]
        rows = []
        for budget in sorted(set(args.pt_budgets) | set(args.pt_learned_budgets)):
            est, rep = sk.pt_estimate(v, n, budget, ladders=4096, seed=budget, stream=sh)
            rows.append({"proposal": "plain", "iterations": budget, "estimate": est,
                         "rel_error": est / exact - 1, "rel_stderr": rep["rel_stderr"],
                         "gpu_ms": rep["kernel_ms"], "tune_ms": rep["tune_ms"]})
        # training set: final states of independent plain runs on the tuned ladder
        beta = sk.tune_ladder(v, n, 32, 32.0, 0)
        states, seed = [], 100
        while sum(len(x) for x in states) < args.pt_samples:
            r = sk.pt_run(v, n, beta, 4096, 1000, 0, seed, want_final=True)
            states.append(r["final_slots"].reshape(-1, n))
            seed += 1
        states = np.concatenate(states)[:args.pt_samples]
        model = sk.Mlp(v, n, 131072, seed=1)
        loss, train_ms = model.train(states, epochs=1, batch=4096, lr=1e-3, beta_star=2.0, seed=1)
        for budget in args.pt_learned_budgets:
            est, rep = sk.pt_estimate(v, n, budget, ladders=4096, seed=budget, beta=beta,
                                      model=model, stream=sh)
            rows.append({"proposal": "learned", "iterations": budget, "estimate": est,
                         "rel_error": est / exact - 1, "gpu_ms": rep["kernel_ms"],
                         "train_ms": train_ms, "train_loss": loss,
                         "train_samples": int(states.shape[0])})
        model.close()
        out[f"{'SL'[v]}({n})"] = rows
    summary = {}
    for case, rows in out.items():
        for prop in ("plain", "learned"):
            ok = [r for r in rows if r["proposal"] == prop and abs(r["rel_error"]) < 0.01]
            summary[f"{case} {prop}: GPU ms to |error| < 1%"] = min((r["gpu_ms"] for r in ok), default=None)
    # roofline of the plain tempering kernel: its longest run
    case, big = max(((c, r) for c, rows in out.items() for r in rows if r["proposal"] == "plain"),
                    key=lambda x: x[1]["gpu_ms"])
    rate = 4096 * 32 * big["iterations"] / (big["gpu_ms"] * 1e-3)
    peak = sk.int32_peak(1)[0] / 1e12
    achieved = PT_OPS_PER_LANE_ITERATION * rate / 1e12
    roofline = {"bound": "alu", "kernel": f"pt_kernel ({case}, {big['iterations']} iterations)",
                "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": None, "ops_per_lane_iteration": PT_OPS_PER_LANE_ITERATION,
                "lane_iterations_per_s": rate,
                "peak_source": "measured: sk_int32_peak mode 1 (multiply-add / lop3 mix), same run"}
    return {"metric": "PT relative error vs GPU time, learned vs plain proposal",
            "summary": summary, "roofline": roofline,
            "config": {"workload": "32 temperatures x 4096 ladders, Skolem / Langford n=16..24",
                       "training": f"{args.pt_samples} plain-PT states, 1 epoch, Adam 1e-3"},
            "unit": "relative error", "results": out}


def run_pt_large_bench(args, sk, sh):
    """Plain tempering beyond the exact workloads: the orders of Tables 7 / 8
    above 24, errors against the exact counts where the paper has them and
    the estimate beside the paper's own tempering estimate."""
    cases = [(0, 25), (0, 28), (0, 29), (1, 27), (1, 28), (0, 32), (0, 33), (1, 31), (1, 32),
             (0, 64)]
    if args.pt_only:
        cases = [c for c in cases if f"{c[0]},{c[1]}" in args.pt_only]
    out = {}
    for v, n in cases[:args.pt_cases]:
        exact = (EXACT_S if v == 0 else EXACT_L).get(n)
        paper = (PAPER_PT_S if v == 0 else PAPER_PT_L)[n]
        rows = []
        for budget in args.pt_budgets:
            est, rep = sk.pt_estimate(v, n, budget, rungs=args.pt_rungs, ladders=4096, seed=budget,
                                      stream=sh, round_trips=True)
            rows.append({"iterations": budget, "rungs": rep["rungs"], "estimate": est,
                         "round_trips_per_configuration": rep["round_trips"] / (4096 * rep["rungs"]),
                         "rel_error": (est / exact - 1) if exact else None,
                         "paper_estimate": paper,
                         "paper_rel_error": (paper / exact - 1) if exact else None,
                         "vs_paper_estimate": est / paper - 1, "rel_stderr": rep["rel_stderr"],
                         "gpu_ms": rep["kernel_ms"]})
        out[f"{'SL'[v]}({n})"] = rows
    return {"metric": "PT estimates beyond n = 24 (Tables 7 / 8)", "unit": "relative error",
            "config": {"workload": f"{args.pt_rungs} temperatures x 4096 ladders, Skolem "
                                   "n=25..33 and 64, Langford n=27..32"},
            "results": out}


EXACT_S12, EXACT_L12 = 227968, 108144                  # Tables 7 / 8


def run_train_bench(args, sk, sh):
    """Training of the proposal network: one epoch of Adam over 2^20 plain-
    tempering states (minibatch 4096, 256 steps) for S(20), with the forward
    and backward GEMMs on tcgen05 and on mma.sync; device time per step
    (sk_mlp_train's CUDA events), best of `steps` epochs after one warm-up
    epoch.  Both start from the same weights."""
    import numpy as np
    v, n = 0, 20
    beta = sk.tune_ladder(v, n, 32, 32.0, 0)
    states = np.concatenate([
        sk.pt_run(v, n, beta, 4096, 500, 0, 300 + s, want_final=True)["final_slots"].reshape(-1, n)
        for s in range(8)])[:1 << 20]
    out = {}
    for name, tc in (("tcgen05", True), ("mma_sync", False)):
        model = sk.Mlp(v, n, 4096, seed=1)
        model.set_gemm(tc)
        model.train(states, epochs=1, batch=4096, lr=1e-3, beta_star=2.0, seed=1)
        best = None
        for _ in range(max(1, args.steps)):
            loss, ms = model.train(states, epochs=1, batch=4096, lr=1e-3, beta_star=2.0, seed=2)
            best = ms if best is None else min(best, ms)
        model.check()
        model.close()
        steps = states.shape[0] // 4096
        out[name] = {"ms_per_epoch": best, "ms_per_step": best / steps, "steps": steps,
                     "final_loss": loss}
    return {"metric": "proposal-network training step time, tcgen05 vs mma.sync GEMMs",
            "unit": "ms", "config": {"workload": "S(20) network (40 -> 256 -> 256 -> 590 moves), "
                                                 "minibatch 4096, 2^20 plain-PT states"},
            "results": out,
            "speedup_tcgen05": out["mma_sync"]["ms_per_step"] / out["tcgen05"]["ms_per_step"]}


def run_pt_gain_bench(args, sk, sh):
    """What the trained proposal network gains per iteration and what it
    costs in GPU time: plain and learned chains at equal iterations on
    S(12), L(12) and S(16), the pilot-tuned 32-rung ladder, 512 ladders, 10 %
    burn-in, six seeds per point (mean relative error and its standard
    error over the seeds, mean move acceptance at the middle rung, GPU time
    of the chains).  The network is trained on 262144 final states of plain
    runs on the same ladder (5 epochs, minibatch 4096, Adam 1e-3,
    beta* = 2)."""
    import numpy as np
    cases = [(0, 12, EXACT_S12), (1, 12, EXACT_L12), (0, 16, EXACT_S[16])]
    budgets = (400, 800, 1600, 3200)
    L, seeds = 512, 6
    out = {}
    for v, n, exact in cases[:args.pt_cases]:
        beta = sk.tune_ladder(v, n, 32, 32.0, 0)
        states = np.concatenate([
            sk.pt_run(v, n, beta, 1024, 1000, 0, 100 + s, want_final=True)["final_slots"].reshape(-1, n)
            for s in range(8)])
        model = sk.Mlp(v, n, L * 32, seed=1)
        loss, train_ms = model.train(states, epochs=5, batch=4096, lr=1e-3, beta_star=2.0, seed=1)
        rows = []
        for iters in budgets:
            row = {"iterations": iters}
            for name, mdl in (("plain", None), ("learned", model)):
                errs, acc, ms = [], [], 0.0
                for s in range(seeds):
                    est, rep = sk.pt_estimate(v, n, iters, ladders=L, seed=1000 + s, beta=beta,
                                              model=mdl, stream=sh)
                    errs.append(est / exact - 1)
                    acc.append(rep["acc_move"][16])
                    ms += rep["kernel_ms"]
                row[name] = {"rel_error": float(np.mean(errs)),
                             "se": float(np.std(errs, ddof=1) / np.sqrt(seeds)),
                             "acc_move_mid": float(np.mean(acc)), "gpu_ms_per_run": ms / seeds}
            rows.append(row)
        model.close()
        out[f"{'SL'[v]}({n})"] = {"train_loss": loss, "train_ms": train_ms, "rows": rows}
    return {"metric": "PT error at equal iterations and GPU time, learned vs plain proposal",
            "unit": "relative error",
            "config": {"workload": "32 temperatures x 512 ladders, S(12), L(12), S(16), 6 seeds",
                       "training": "262144 plain-PT states, 5 epochs, Adam 1e-3"},
            "results": out}


def run_pt_bias_bench(args, sk, sh):
    """Is there a bias of the tempering estimate at the largest orders?  The
    orders of Tables 7 / 8 from 27 up, each estimated with the pilot-tuned
    32-rung ladder topped at beta_max = 32, 48 and 64, and with beta_max = 32
    and four times the iterations; per run the estimate and its standard
    error (16 groups of 256 ladders), the smallest exchange acceptance of
    the ladder, P(E = 0) at the top rung (the last ratio of Algorithm 2) and
    the round trips of configurations between the ends of the ladder.
    Then 64 rungs topped at beta_max = 32 (two warps a ladder): the same
    top temperature with twice the rungs, closer neighbours and higher
    exchange acceptance.  With --pt-rungs 64 only the 64-rung ladder runs,
    for the base and four times the iterations."""
    cases = [(0, 28), (0, 29), (1, 27), (1, 28), (0, 32), (0, 33), (1, 31), (1, 32), (0, 64)]
    if args.pt_only:
        cases = [c for c in cases if f"{c[0]},{c[1]}" in args.pt_only]
    base = args.pt_budgets[0]
    variants = [(32.0, base, 32), (48.0, base, 32), (64.0, base, 32), (32.0, 4 * base, 32),
                (32.0, base, 64)]
    if args.pt_rungs == 64:
        variants = [(32.0, base, 64), (32.0, 4 * base, 64)]
    out = {}
    for v, n in cases[:args.pt_cases]:
        exact = (EXACT_S if v == 0 else EXACT_L).get(n)
        paper = (PAPER_PT_S if v == 0 else PAPER_PT_L)[n]
        rows = []
        for bmax, budget, rungs in variants:
            est, rep = sk.pt_estimate(v, n, budget, rungs=rungs, ladders=4096, seed=7,
                                      beta_max=bmax, stream=sh, round_trips=True)
            M = rep["rungs"]
            rows.append({"beta_max": bmax, "iterations": budget, "rungs": M, "estimate": est,
                         "round_trips": rep["round_trips"],
                         "round_trips_per_configuration": rep["round_trips"] / (4096 * M),
                         "rel_stderr": rep["rel_stderr"],
                         "rel_error": (est / exact - 1) if exact else None,
                         "z_vs_exact": ((est / exact - 1) / rep["rel_stderr"]) if exact else None,
                         "vs_paper_estimate": est / paper - 1,
                         "min_exchange_acceptance": min(rep["acc_swap"][:M - 1]),
                         "p_top_E0": rep["ratio"][M - 1], "beta": rep["beta"],
                         "gpu_ms": rep["kernel_ms"]})
        out[f"{'SL'[v]}({n})"] = rows
    return {"metric": "PT estimates at n = 27..33 across ladders (beta_max) and run lengths",
            "unit": "relative error",
            "config": {"workload": "32 and 64 temperatures x 4096 ladders, Skolem "
                                   "n=28,29,32,33,64, Langford n=27,28,31,32"},
            "results": out}


def run_reference(args, world, rank):
    if rank != 0:
        return
    vals, secs = [], []
    cores = sample = None
    for i in range(args.warmup + args.steps):
        v, cores, sample, dt = oracle_sample(seconds_target=8.0)
        if i >= args.warmup:
            vals.append(v)
            secs.append(dt)
    value = statistics.mean(vals)
    # a step is a bounded sample of the workload: its measured time, not the
    # workload's time at this rate
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "terms/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(secs) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": "a bounded sample of the workload: " + sample},
            "cpu_baseline": {"value": value, "unit": "terms/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "terms/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch
    import paper_1507_00315_gb300 as sk
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    want = {}

    def step(record):
        kms = []
        for v, n in JOBS:
            c, rep = sk.count_ex(v, n, stream=sh)
            if (v, n) in want:
                assert c == want[(v, n)], (v, n, c, want[(v, n)])
            else:
                want[(v, n)] = c
            kms.append(((v, n), rep["kernel_ms"], rep))
        flush.zero_()                               # L2 flushed between steps
        return kms

    for _ in range(args.warmup):
        step(False)
    peak_mix, _ = sk.int32_peak(1)
    peak_mad, _ = sk.int32_peak(0)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    e0.record(stream)
    per_launch = []
    for _ in range(args.steps):
        per_launch += step(True)
    e1.record(stream)
    torch.cuda.synchronize()
    w1 = time.perf_counter()
    clk = clocks.stop()
    dev_s = e0.elapsed_time(e1) / 1e3
    wall_s = w1 - w0
    dev_s, wall_s = reduce_max_over_ranks([dev_s, wall_s], "cuda")
    if rank != 0:
        return
    tps = terms_per_step()
    value = job_throughput(world, args.steps, tps, dev_s)
    e2e = job_throughput(world, args.steps, tps, wall_s)
    # roofline of the dominant kernel: the largest launch (S(20))
    dom = [x for x in per_launch if x[0] == (0, 20)]
    dom_ms = statistics.mean(x[1] for x in dom)
    ops = alg_ops_per_term(0, 20) * (1 << 39)
    achieved = ops / (dom_ms / 1e3) / 1e12
    peak = peak_mix / 1e12
    all_ops = sum(alg_ops_per_term(v, n) * (1 << (2 * n - 1)) for (v, n), _, _ in per_launch)
    all_ms = sum(x[1] for x in per_launch)
    line = {
        "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_s / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "jobs": [f"{'SL'[v]}({n})" for v, n in JOBS],
                   "moduli": 3, "l2": "flushed between steps (512 MiB write)",
                   "walk_bits": {f"{'SL'[v]}({n})": r["walk_bits"] for (v, n), _, r in per_launch[:len(JOBS)]},
                   "block_threads": 256, "parallelism": f"{world} replica(s), one GPU each"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(),
                     "kernel": "limb_kernel<0,20> (S(20), 2^39 terms)",
                     "ops_per_term": alg_ops_per_term(0, 20),
                     "peak_source": "measured: sk_int32_peak mode 1 (multiply-add / lop3 mix), same run",
                     "imad_pipe_busy_ncu": recorded_imad_busy(),
                     "int32_mad_peak_tops": peak_mad / 1e12,
                     "all_launches_frac": (all_ops / (all_ms / 1e3) / 1e12) / peak},
        "e2e": {"value": e2e, "unit": "terms/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 48 * len(JOBS)},
        "gpu_launches": args.steps * len(JOBS),
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        v, cores, sample, _ = oracle_sample()
        line["cpu_baseline"] = {"value": v, "unit": "terms/s", "cores": cores, "kind": "oracle",
                                "sample": sample}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pt-budgets", type=int, nargs="+", default=[2000, 8000, 32000])
    ap.add_argument("--pt-learned-budgets", type=int, nargs="+", default=[200, 800])
    ap.add_argument("--pt-samples", type=int, default=10_000_000)
    ap.add_argument("--pt-cases", type=int, default=10, help="first cases of --config pt / pt-large")
    ap.add_argument("--pt-rungs", type=int, default=32,
                    help="temperatures a ladder, --config pt-large (pt-bias: 64 -> 64-rung rows only)")
    ap.add_argument("--pt-only", nargs="+", default=None,
                    help="--config pt-large / pt-bias: only these cases, as variant,n (e.g. 0,64)")
    ap.add_argument("--slice-bits", type=int, default=40, help="terms per slice of --config slices (log2)")
    ap.add_argument("--config", default="mid",
                    choices=["mid", "batch", "large", "slices", "ie", "symmetry", "pt", "pt-large",
                             "pt-bias", "pt-gain", "train"],
                    help="mid: the headline workload; the others: extra measurements")
    ap.add_argument("--nmax", type=int, default=22, help="largest n of --config batch")
    ap.add_argument("--no-autotune", action="store_true", help="--config batch without the tuned run")
    ap.add_argument("--ckpt-dir", default=None, help="checkpoint directory of --config large")
    ap.add_argument("--symmetries", type=int, nargs="+", default=[0, 1],
                    help="--config large: SK_SYMMETRY_* options to run (0: Lemma 2.2, 1: + 2.4, "
                         "2: + 2.3, 3: + 2.3 + 2.4)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        # rank 0 alone times the oracle; other ranks exit without work
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
        return
    world, rank, local = dist_setup(args.gpus)
    if args.config != "mid":
        run_extra(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
