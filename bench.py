"""Benchmark of the GB300 per-day GradABM step (forward + MSE + hand-written backward).

Workload: 1,000,000 agents on the four-interaction-type synthetic contact graph
(households, schools, workplaces, random contacts; ~22.4M directed edges),
60 days, R = 2.5, 20 seed infections, MSE on daily deaths against a seeded
synthetic curve, gradients for R_t, m_t and S_a.  One step = one forward over
the horizon + the loss + the reverse sweep, all in the library's kernels.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (on a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "agent-days/s fwd and fwd+bwd at 1M agents; HBM GB/s fraction; batched vs plain"
N_AGENTS = 1_000_000
DAYS = 60
R0 = 2.5
MORTALITY = 0.01
N_SEED = 20
TAU_EI, TAU_IR = 4, 7
# batched ensemble: parameter sets sharing one contact graph
BATCH_AGENTS = 500_000
BATCH_SETS = 64
BATCH_DAYS = 45


def max_over_ranks(ms: float, dist=None, device="cpu") -> float:
    """Whole-job time of a timed region: the maximum over ranks (each rank's own CUDA-event
    time); the plain value with one rank."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms_per_step_max: float) -> float:
    """Units all ranks processed per second (weak scaling: every rank runs the full workload)."""
    return world * units_per_rank / (ms_per_step_max / 1e3)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _kernel_source_sha(names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2207_09714_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel: str, sha: str, workload: str):
    """Per-launch DRAM bytes of ``kernel`` from the committed ncu summary, if it was taken
    on the current kernel source and this workload; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
        if kv.get("kernel") == kernel and kv.get("src_sha") == sha and kv.get("workload") == workload:
            return float(kv["bytes_per_launch"])
    return None


# a kernel's sources and capi.cu, which builds the device layout its traffic depends on
_SRC = {"k_fwd_day": ["forward.cu", "rowsum.cuh", "gabm_internal.cuh", "capi.cu"],
        "k_bwd_day": ["backward.cu", "rowsum.cuh", "gabm_internal.cuh", "capi.cu"],
        "k_fwd_day_b": ["batched.cu", "batched_common.cuh", "rowsum.cuh", "gabm_internal.cuh", "capi.cu"],
        "k_bwd_day_b": ["batched_bwd.cu", "batched_common.cuh", "rowsum.cuh", "gabm_internal.cuh", "capi.cu"]}


def dram_rate(kernel: str, workload: str, ms_per_launch: float, peak: float):
    """The ncu-measured DRAM bytes per launch of ``kernel`` on ``workload`` (profiles/
    ncu_traffic.txt, current source only) and the rate and fraction of the peak they
    give at the live per-launch duration; None without a matching capture."""
    tr = _ncu_traffic(kernel, _kernel_source_sha(_SRC[kernel]), workload)
    if tr is None or not ms_per_launch:
        return None
    gbs = tr / (ms_per_launch / 1e3) / 1e9
    return {"traffic_bytes_per_launch": tr, "dram_gbs": gbs, "dram_frac": gbs / peak}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms while running.  Entering
    waits until the sampler is up, so its samples cover the region it brackets."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)
        except (OSError, FileNotFoundError):
            self.proc = None
        self.t0 = time.time()
        return self

    def __exit__(self, *exc):
        self.t1 = time.time()
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def _within(self, stamp):
        try:
            whole, _, frac = stamp.partition(".")
            t = time.mktime(time.strptime(whole, "%Y/%m/%d %H:%M:%S")) + float("0." + (frac or "0"))
        except (ValueError, IndexError):
            return None
        return self.t0 - 0.05 <= t <= self.t1 + 0.05

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = [[x.strip() for x in l.split(",")] for l in getattr(self, "lines", [])]
        stamped = [(self._within(p[0]), p) for p in lines]
        if any(w is not None for w, _ in stamped):    # keep the samples inside the bracketed region
            lines = [p for w, p in stamped if w]
        for p in lines:
            p = p[1:]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def frontier_counts(pop, E, T, L):
    """Per day t of the trajectory fixed by the final exposure days E (caller order): the
    susceptible rows with an in-neighbour infectious on day t (the rows the forward sums),
    their entries, and the out-entries of the rows infectious on day t + 1 (the flags the
    day's launch pushes for tomorrow)."""
    E = np.asarray(E).astype(np.int64)
    NEVER = 32767
    deg = np.diff(pop.rowptr.astype(np.int64))
    col = pop.col.astype(np.int64)
    rows = np.repeat(np.arange(pop.n, dtype=np.int64), deg)
    sf_rows = np.zeros(T)
    sf_nnz = np.zeros(T)
    push = np.zeros(T)
    for t in range(T):
        inf = (E != NEVER) & (t - E >= 1) & (t - E < L)
        flag = np.zeros(pop.n, bool)
        flag[rows[inf[col]]] = True
        sf = flag & (E >= t)
        sf_rows[t] = sf.sum()
        sf_nnz[t] = deg[sf].sum()
        inf1 = (E != NEVER) & (t + 1 - E >= 1) & (t + 1 - E < L)
        push[t] = deg[inf1].sum()
    return sf_rows, sf_nnz, push


def trajectory_bytes(E, deg, T, L, n_rows, policy_store, frontier=None):
    """Algorithmic (compulsory) HBM bytes of every forward and backward day launch, from
    the final exposure days E (which determine each day's state).  With ``frontier`` (from
    frontier_counts) the forward reads only the entries of susceptible rows with an
    infectious in-neighbour, plus every row's state, flag and length and the pushes of
    tomorrow's flags; without it, every susceptible row's entries."""
    E = E.astype(np.int64)
    NEVER = 32767
    seed = (E != NEVER) & (E < 0)
    live = ~seed
    never = E == NEVER
    Ec = np.where(never, T, E)          # never infected counts as susceptible every day
    Ec = np.where(seed, -1, Ec)
    # rows susceptible on day t: Ec >= t ; edges of those rows
    hist_n = np.bincount(np.clip(Ec[live], 0, T), minlength=T + 1)
    hist_e = np.bincount(np.clip(Ec[live], 0, T), weights=deg[live], minlength=T + 1)
    S_cnt = np.cumsum(hist_n[::-1])[::-1][:T]
    S_nnz = np.cumsum(hist_e[::-1])[::-1][:T]
    new = np.bincount(E[live & ~never], minlength=T)[:T]
    n_never = int(np.count_nonzero(live & never))
    if frontier is None:
        fwd = 8.0 * S_nnz + 4.0 * S_cnt + 1.0 * S_cnt + 2.0 * n_rows + 2.0 * new
    else:
        sf_rows, sf_nnz, push = frontier
        # entries (col + w) and age + caller id of the summed rows; state, flag read and
        # clear, row length of every row; tomorrow's flags: out-entries read, one byte each
        fwd = 8.0 * sf_nnz + 5.0 * sf_rows + 8.0 * n_rows + 2.0 * new + 5.0 * push
    if policy_store:
        fwd += 4.0 * S_cnt
    # backward: rows needing the transpose gather on day t are live with Ec >= t + 2 - L
    def ge(thr):
        thr = np.clip(thr, 0, T)
        return S_cnt_full[thr], S_nnz_full[thr]
    S_cnt_full = np.concatenate([np.cumsum(hist_n[::-1])[::-1], [0]])
    S_nnz_full = np.concatenate([np.cumsum(hist_e[::-1])[::-1], [0]])
    bwd = np.zeros(T)
    for t in range(T):
        nS, eS = S_cnt[t], S_nnz[t]
        # the last reverse day has no gx(t+1) to gather
        nA, eA = ge(max(t + 2 - L, 0)) if t + 1 < T else (0, 0.0)
        ring_reads = max(0, min(L - 1, T - 1 - t) - 1)      # slots k = 2..L-1 inside the horizon
        # entries (col + w) of the gathering rows; state and row length of every row; age
        # of the susceptible rows
        b = 8.0 * eA + 6.0 * n_rows + 1.0 * nS
        b += 4.0 * ring_reads * nS + (4.0 * nA if t + 1 < T else 0.0)   # ring reads and write
        # A read by the susceptible rows exposed later (not today, not never), written by
        # today's exposures; r written by every susceptible row
        b += 4.0 * (nS - n_never - new[t]) + 4.0 * new[t] + 4.0 * nS
        if policy_store:
            b += 4.0 * nS
        b += 72.0 * (n_rows // 32)                                   # per-tile partial sums
        bwd[t] = b
    return fwd, bwd, S_cnt, S_nnz


def batched_trajectory_bytes(E, deg, T, L, n, B, l2_bytes):
    """Algorithmic HBM bytes of the batched day launches (B sets sharing one graph) from the
    final exposure days E [B, n] of every set: rows are read once for all sets, per-set
    state once per set.  The backward's coefficient gather costs nothing per edge when
    the array fits in half of L2, else its B values per edge (every entry of a row that
    needs the transpose gather reads them).  The forward's exposure-day gathers are not
    charged: they are made for the marked neighbours only (infectious in some set), a
    data-dependent share of the entries, and their DRAM cost is what ncu measures."""
    E = E.astype(np.int64)
    NEVER = 32767
    seed = (E != NEVER) & (E < 0)
    Ec = np.where(E == NEVER, T, E)
    Ec = np.where(seed, -1, Ec)                      # [B, n] last susceptible day (>= t: S on day t)
    last_any = Ec.max(axis=0)                        # a row is read while some set is susceptible
    hist_r = np.bincount(np.clip(last_any[last_any >= 0], 0, T), minlength=T + 1)
    hist_e = np.bincount(np.clip(last_any[last_any >= 0], 0, T), weights=deg[last_any >= 0], minlength=T + 1)
    rows_t = np.cumsum(hist_r[::-1])[::-1]
    nnz_t = np.cumsum(hist_e[::-1])[::-1]
    flat = Ec[Ec >= 0]
    hist_s = np.bincount(np.clip(flat, 0, T), minlength=T + 1)
    S_t = np.cumsum(hist_s[::-1])[::-1]              # sum over sets of susceptible agents on day t
    new = np.bincount(E[(E != NEVER) & (E >= 0)], minlength=T)[:T]
    gath_f = 0.0
    gath_b = 0.0 if n * B * 4 <= l2_bytes / 2 else 4.0 * B
    fwd = np.zeros(T)
    bwd = np.zeros(T)
    for t in range(T):
        fwd[t] = (8.0 * nnz_t[t] + 8.0 * rows_t[t] + 2.0 * n * B + n + 2.0 * new[t] + 4.0 * S_t[t]
                  + gath_f * nnz_t[t])
        ring_reads = max(0, min(L - 1, T - 1 - t) - 1)
        thr = min(T, max(t + 2 - L, 0))
        b = 4.0 * S_t[t] + 2.0 * n * B + n + S_t[t] * (4.0 * ring_reads + 4.0 + 4.0)
        if t + 1 < T:
            b += 8.0 * nnz_t[thr] + 8.0 * rows_t[thr] + 4.0 * n * B + gath_b * nnz_t[thr]
        bwd[t] = b
    return fwd, bwd


def bench_batched(args, stream, peak, peak_kind):
    """B parameter sets on one shared graph, forward + MSE + backward per set: the
    batched kernels (one launch per day phase, day loops replayed as CUDA graphs,
    schedule from the autotuner) next to the plain path (one set at a time through
    the autograd Function, eager launches)."""
    import torch
    from paper_2207_09714_gb300 import capi, synth
    from paper_2207_09714_gb300.autograd import GabmFunction
    B, T = BATCH_SETS, args.batched_days
    pop = synth.population_typed(args.batched_agents, seed=0)
    c = synth.infectiousness_table(TAU_EI, TAU_IR)
    rng = np.random.default_rng(0)
    R_np = np.repeat(rng.uniform(1.5, 4.0, (B, 1)), T, axis=1).astype(np.float32)
    m_np = np.repeat(rng.uniform(0.005, 0.05, (B, 1)), T, axis=1).astype(np.float32)
    R = torch.from_numpy(R_np).cuda()
    m = torch.from_numpy(m_np).cuda()
    S = torch.from_numpy(np.tile(synth.SUSCEPTIBILITY, (B, 1)).astype(np.float32)).cuda()
    y = torch.from_numpy(np.stack([synth.target_curve(T, pop.n, seed=b) for b in range(B)])).cuda()
    seeds = [N_SEED] * B
    with torch.cuda.stream(stream):
        ctx = capi.gabm_create([pop], capi.ModelDesc(TAU_EI, TAU_IR, c, seed=0), sets_per_graph=B, stream=stream)
    D = torch.empty((B, T), dtype=torch.float64, device="cuda")
    loss = torch.empty((B,), dtype=torch.float64, device="cuda")
    gD = torch.empty((B, T), dtype=torch.float64, device="cuda")
    dR = torch.empty((B, T), dtype=torch.float64, device="cuda")
    dm = torch.empty((B, T), dtype=torch.float64, device="cuda")
    dS = torch.empty((B, 9), dtype=torch.float64, device="cuda")

    def step():
        capi.gabm_forward(ctx, T, R, m, S, seeds, D=D)
        capi.gabm_mse_loss(ctx, y, loss=loss, gD=gD)
        capi.gabm_backward(ctx, gD, dR=dR, dm=dm, dS_age=dS)

    step()
    if args.batched_schedule:   # a fixed schedule (profiling runs): no autotuner launches
        spl_f, spl_b, smem, chunk = (int(x) for x in args.batched_schedule.split(","))
        capi.gabm_set_schedule(ctx, spl_f, spl_b, smem, chunk)
        schedule = capi.gabm_get_schedule(ctx)
    else:
        schedule = capi.gabm_autotune(ctx, 1)
    steps = max(args.steps // 2, 2)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = capi.gabm_launch_count(ctx)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = capi.gabm_launch_count(ctx) - l0
    ms = e0.elapsed_time(e1) / steps
    # per-kernel durations (events around each day launch: eager launches)
    capi.gabm_set_profiling(ctx, True)
    step()
    f_ms, f_n = capi.gabm_get_profile(ctx, 0)
    b_ms, b_n = capi.gabm_get_profile(ctx, 1)
    capi.gabm_set_profiling(ctx, False)
    E = capi.gabm_get_state(ctx)
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    fwd_b, bwd_b = batched_trajectory_bytes(E, pop.degrees().astype(np.float64), T, TAU_EI + TAU_IR, pop.n, B, l2)
    f_gbs = fwd_b.sum() / (f_ms / 1e3) / 1e9
    b_gbs = bwd_b.sum() / (b_ms / 1e3) / 1e9
    both_gbs = (fwd_b.sum() + bwd_b.sum()) / ((f_ms + b_ms) / 1e3) / 1e9
    counts = capi.gabm_forward(ctx, T, R, m, S, seeds, want_counts=True)[1]
    torch.cuda.synchronize()   # the ctx works on its own stream
    counts = counts.cpu().numpy()
    attack = 1.0 - counts[:, -1, 0] / pop.n
    del ctx
    units = B * pop.n * T
    dom = "k_bwd_day_b" if b_ms >= f_ms else "k_fwd_day_b"
    src = ["batched_bwd.cu" if dom == "k_bwd_day_b" else "batched.cu", "batched_common.cuh", "rowsum.cuh",
           "gabm_internal.cuh"]
    wl = f"typed{pop.n // 1000}k_B{B}_T{T}_store"
    traffic = _ncu_traffic(dom, _kernel_source_sha(src), wl)
    f_dr = dram_rate("k_fwd_day_b", wl, f_ms / f_n, peak)
    b_dr = dram_rate("k_bwd_day_b", wl, b_ms / b_n, peak)
    result = {
        "workload": f"one shared {pop.n}-agent typed contact graph, {B} parameter sets (R ~ U[1.5, 4.0], "
                    f"m ~ U[0.005, 0.05]), {T} days, forward + MSE + backward of every set",
        "n_agents": pop.n, "nnz": pop.nnz, "sets": B, "days": T,
        "value": units / (ms / 1e3), "unit": "agent-days/s", "ms_per_step": ms, "steps": steps,
        "schedule": schedule, "attack_rate_range": [float(attack.min()), float(attack.max())],
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": dom,
                     "achieved": b_gbs if dom == "k_bwd_day_b" else f_gbs, "peak": peak, "unit": "GB/s",
                     "frac": (b_gbs if dom == "k_bwd_day_b" else f_gbs) / peak, "peak_source": peak_kind,
                     "traffic": traffic,
                     "fwd_day": {"achieved": f_gbs, "launches": f_n, "ms_total": f_ms,
                                 "alg_bytes_per_launch": fwd_b.sum() / T},
                     "bwd_day": {"achieved": b_gbs, "launches": b_n, "ms_total": b_ms,
                                 "alg_bytes_per_launch": bwd_b.sum() / T},
                     "fwd_plus_bwd_frac": both_gbs / peak},
    }
    result["roofline"]["fwd_day"]["dram"] = f_dr
    result["roofline"]["bwd_day"]["dram"] = b_dr
    if f_dr and b_dr:
        tot = f_dr["traffic_bytes_per_launch"] * f_n + b_dr["traffic_bytes_per_launch"] * b_n
        result["roofline"]["fwd_plus_bwd_dram_frac"] = tot / ((f_ms + b_ms) / 1e3) / 1e9 / peak
    if args.no_plain:
        return result

    # plain: one parameter set at a time through the autograd Function, eager launches
    os.environ["GABM_CUDA_GRAPHS"] = "0"
    try:
        with torch.cuda.stream(stream):
            pctx = capi.gabm_create([pop], capi.ModelDesc(TAU_EI, TAU_IR, c, seed=0), stream=stream)
    finally:
        del os.environ["GABM_CUDA_GRAPHS"]

    def plain_step():
        with torch.cuda.stream(stream):
            for b in range(B):
                Rb = R[b:b + 1].clone().requires_grad_(True)
                mb = m[b:b + 1].clone().requires_grad_(True)
                Sb = S[b:b + 1].clone().requires_grad_(True)
                Db = GabmFunction.apply(pctx, Rb, mb, Sb, [N_SEED])
                ((Db - y[b:b + 1]) ** 2).mean().backward()

    plain_step()
    torch.cuda.synchronize()
    e0.record(stream)
    plain_step()
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    result["plain"] = {"value": units / (plain_ms / 1e3), "ms_per_step": plain_ms,
                       "path": "one set at a time: GabmFunction (torch.autograd) over the single-set kernels, "
                               "eager launches, no CUDA graph"}
    result["speedup_vs_plain"] = plain_ms / ms
    return result


def workload_config(pop, policy: str) -> dict:
    """The bench workload's config (both arms)."""
    return {"workload": f"1M-agent typed contact graph (households, schools, workplaces, random), "
                        f"{DAYS} days, forward + MSE + hand-written backward",
            "n_agents": pop.n, "nnz": pop.nnz, "days": DAYS, "instances_per_gpu": 1,
            "lambda_policy": policy, "R": R0, "n_seed": N_SEED,
            "l2": f"inputs larger than L2 (edge arrays {pop.nnz * 8 / 1e6:.0f} MB > 129 MB), no flush"}


def run_reference(args, world, rank):
    """The FP64 CPU oracle as it stands (OpenMP over the host cores) on the same workload
    and config as the GPU arm: each step is one forward + MSE + backward of the 1M-agent,
    60-day workload (about 6 s on 16 cores).  Warm-up is capped at one step: the oracle has
    no caches or compilation to warm, and each step is a full workload."""
    if rank != 0:
        return
    import oracle as O
    from paper_2207_09714_gb300 import synth
    pop = synth.population_typed(N_AGENTS, seed=0)
    c = synth.infectiousness_table(TAU_EI, TAU_IR)
    R = np.full(DAYS, R0, np.float32)
    m = np.full(DAYS, MORTALITY, np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    y = synth.target_curve(DAYS, pop.n)
    md = O.Model(TAU_EI, TAU_IR, c, seed=0)
    O.build()

    def step():
        f = O.forward_hard(pop, md, R, m, S, n_seed=N_SEED)
        _, gD = O.mse(f["D"], y)
        O.backward_hard(pop, md, R, m, S, f["e_final"], gD)

    warm = min(args.warmup, 1)
    for _ in range(warm):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    value = pop.n * DAYS / dt
    sample = (f"each step the full workload: {pop.n} agents, {pop.nnz} directed edges, {DAYS} days, forward + MSE "
              f"+ backward, FP64, {dt:.1f} s per step on {O.num_threads()} threads ({_cpu_model()})")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "agent-days/s", "n_gpus": world,
        "steps": args.steps, "warmup": warm, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(pop, args.policy),
        "cpu_baseline": {"value": value, "unit": "agent-days/s", "cores": O.num_threads(), "kind": "oracle",
                         "sample": sample, "cpu_model": _cpu_model(), "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": "agent-days/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(pop, c, y):
    """The FP64 oracle on the host cores: one forward + MSE + backward of the same
    1M-agent, 60-day workload (about 10 s of CPU work)."""
    import oracle as O
    from paper_2207_09714_gb300 import synth
    R = np.full(DAYS, R0, np.float32)
    m = np.full(DAYS, MORTALITY, np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    md = O.Model(TAU_EI, TAU_IR, c, seed=0)
    O.build()
    t0 = time.perf_counter()
    f = O.forward_hard(pop, md, R, m, S, n_seed=N_SEED)
    _, gD = O.mse(f["D"], y)
    O.backward_hard(pop, md, R, m, S, f["e_final"], gD)
    dt = time.perf_counter() - t0
    return {"value": pop.n * DAYS / dt, "unit": "agent-days/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"one forward + MSE + backward of the full workload ({pop.n} agents, {pop.nnz} directed "
                      f"edges, {DAYS} days), FP64, {dt:.1f} s",
            "cpu_model": _cpu_model(), "nproc": os.cpu_count()}


def bench_twohop(stream, dist, steps=5, n=1_000_000):
    """The agent-location workload (GradABM-JUNE, Sec. 6): one forward + MSE + backward
    step over 60 days on a synthetic agent-location graph of n agents (households,
    schools of 100-400, workplaces of 5-60, shared venues), computed in two hops over the
    attendance entries.  Reports the pair count the two hops avoid forming."""
    import torch
    from paper_2207_09714_gb300 import capi, synth

    bip = synth.population_bipartite(n, seed=0)
    sizes = np.bincount(bip.loc.astype(np.int64), minlength=bip.n_loc).astype(np.int64)
    pairs = int((sizes * (sizes - 1)).sum())
    with torch.cuda.stream(stream):
        ctx = capi.gabm_create_bipartite(bip, capi.ModelDesc(TAU_EI, TAU_IR, synth.infectiousness_table(TAU_EI, TAU_IR),
                                                             seed=0), stream=stream)
        R = torch.full((1, DAYS), R0, dtype=torch.float32, device="cuda")
        m = torch.full((1, DAYS), MORTALITY, dtype=torch.float32, device="cuda")
        S = torch.from_numpy(synth.SUSCEPTIBILITY[None, :].copy()).cuda()
        y = torch.from_numpy(synth.target_curve(DAYS, n)[None, :]).cuda()

        def step():
            capi.gabm_forward(ctx, DAYS, R, m, S, [N_SEED])
            _, gD = capi.gabm_mse_loss(ctx, y)
            capi.gabm_backward(ctx, gD)

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda") / steps
    return {"workload": f"agent-location graph, {n} agents, {bip.n_loc} locations, {DAYS} days, "
                        f"forward + MSE + backward in two hops", "n_agents": n, "attendances": bip.nnz,
            "pair_entries_avoided": pairs, "ms_per_step": ms, "steps": steps,
            "value": n * DAYS / (ms / 1e3), "unit": "agent-days/s"}


TAU_IM = 10   # I->M days of the sampled R/M split workload (the paper gives no value)
# I-stage duration pmf of the stochastic-duration workload (1..9 days; mean 5.7)
P_IR = np.array([0.02, 0.05, 0.13, 0.2, 0.2, 0.15, 0.12, 0.08, 0.05], np.float32)
TAU_RS = 10   # days in RM before S again in the SIRS-reinfection workload (the paper gives no value)


def bench_progression_variant(pop, stream, S, y_np, dist, peak, peak_kind, variant, steps=5):
    """A progression variant on the bench graph and parameters: ``rm_split`` (tau_IM > 0,
    fates drawn at I entry, deaths counted) or ``durations`` (per-agent I-stage durations
    from P_IR).  One forward + MSE + backward step, then the same steps with events around
    every day launch for the per-kernel rates (the algorithmic bytes of the base model's
    day kernels with the longest window L)."""
    import torch
    from paper_2207_09714_gb300 import capi, synth

    if variant == "rm_split":
        L = TAU_EI + max(TAU_IR, TAU_IM)
        md = capi.ModelDesc(TAU_EI, TAU_IR, synth.infectiousness_table(TAU_EI, max(TAU_IR, TAU_IM)), seed=0,
                            tau_IM=TAU_IM)
        what = f"sampled R/M split: tau_EI {TAU_EI}, tau_IR {TAU_IR}, tau_IM {TAU_IM}"
    elif variant == "durations":
        L = TAU_EI + P_IR.size
        md = capi.ModelDesc(TAU_EI, P_IR.size, synth.infectiousness_table(TAU_EI, P_IR.size), seed=0, p_IR=P_IR)
        what = f"stochastic I-stage durations: tau_EI {TAU_EI}, I days ~ pmf {P_IR.round(2).tolist()} over 1..{P_IR.size}"
    else:
        L = TAU_EI + TAU_IR
        md = capi.ModelDesc(TAU_EI, TAU_IR, synth.infectiousness_table(TAU_EI, TAU_IR), seed=0, tau_RS=TAU_RS)
        what = f"SIRS reinfection: tau_EI {TAU_EI}, tau_IR {TAU_IR}, back to S after tau_RS {TAU_RS}"
    with torch.cuda.stream(stream):
        ctx = capi.gabm_create([pop], md, stream=stream)
        R = torch.full((1, DAYS), R0, dtype=torch.float32, device="cuda")
        m = torch.full((1, DAYS), MORTALITY, dtype=torch.float32, device="cuda")
        y = torch.from_numpy(y_np).cuda()

        def step():
            capi.gabm_forward(ctx, DAYS, R, m, S, [N_SEED])
            _, gD = capi.gabm_mse_loss(ctx, y)
            capi.gabm_backward(ctx, gD)

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda") / steps
        capi.gabm_set_profiling(ctx, True)
        for _ in range(steps):
            step()
        torch.cuda.synchronize()
        f_ms, f_n = capi.gabm_get_profile(ctx, 0)
        b_ms, b_n = capi.gabm_get_profile(ctx, 1)
        capi.gabm_set_profiling(ctx, False)
        E = capi.gabm_get_state(ctx)[0]
        D = capi.gabm_forward(ctx, DAYS, R, m, S, [N_SEED])[0].cpu().numpy()[0]
    out = {"workload": f"{what}, on the bench graph, m = {MORTALITY}, {DAYS} days, forward + MSE + backward",
           "ms_per_step": ms, "steps": steps, "value": pop.n * DAYS / (ms / 1e3), "unit": "agent-days/s",
           "deaths": float(D.sum())}
    if variant == "sirs":
        # the final state does not fix who was susceptible on each day under reinfection,
        # so the base model's byte count does not apply; launch times only
        out.update({"fwd_day": {"avg_launch_ms": f_ms / f_n}, "bwd_day": {"avg_launch_ms": b_ms / b_n},
                    "agents_last_exposed_after_day_0_share": float(np.mean((E >= 0) & (E != 32767)))})
        return out
    n_rows = ((pop.n + 31) // 32) * 32
    fwd_b, bwd_b, _, _ = trajectory_bytes(E, pop.degrees().astype(np.float64), DAYS, L, n_rows, True,
                                          frontier=frontier_counts(pop, E, DAYS, L))
    f_gbs = fwd_b.sum() * steps / (f_ms / 1e3) / 1e9
    b_gbs = bwd_b.sum() * steps / (b_ms / 1e3) / 1e9
    return {"workload": f"{what}, on the bench graph, m = {MORTALITY}, {DAYS} days, forward + MSE + backward",
            "ms_per_step": ms, "steps": steps, "value": pop.n * DAYS / (ms / 1e3), "unit": "agent-days/s",
            "deaths": float(D.sum()),
            "fwd_day": {"avg_launch_ms": f_ms / f_n, "achieved_gbs": f_gbs, "frac": f_gbs / peak},
            "bwd_day": {"avg_launch_ms": b_ms / b_n, "achieved_gbs": b_gbs, "frac": b_gbs / peak},
            "peak": peak, "peak_source": peak_kind}


def bench_calibration(ctx, stream, S, y_np, dist, steps=5):
    """One Adam step of the calibration workload on the bench graph: weekly-tied R and m,
    the stage factors and profile of the infectiousness table, MSE on cumulative deaths.
    A step is the forward, the adjoint including dL/dc, the torch parameter maps and the
    update; the table changes every step, so both day loops are re-captured each step."""
    import torch
    from paper_2207_09714_gb300 import calibrate

    with torch.cuda.stream(stream):
        p = calibrate.WeeklyParams(1, DAYS, R0=R0, m0=MORTALITY)
        opt = torch.optim.Adam(p.parameters(), lr=0.02)
        y_cum = torch.cumsum(torch.from_numpy(y_np).cuda(), dim=-1)
        losses = []

        def cstep():
            opt.zero_grad()
            R, m, c = p()
            D = calibrate.TableFunction.apply(ctx, R, m, S, c, [N_SEED])
            loss = calibrate.cumulative_mse(D, y_cum)
            loss.backward()
            opt.step()
            losses.append(loss.detach())

        def timed(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return max_over_ranks(e0.elapsed_time(e1), dist, "cuda") / steps

        ms = timed(cstep)
        first_last = [float(losses[0]), float(losses[-1])]
        # DC-GradABM: the weekly parameters from CalibNN over synthetic features
        torch.manual_seed(0)
        x = torch.as_tensor(calibrate.synthetic_features(np.full((1, DAYS), R0), t_N=DAYS, F=5, seed=0),
                            device="cuda")
        net = calibrate.DeepCalibration(5, DAYS, hidden=32).cuda()
        opt_dc = torch.optim.Adam([q for q in net.parameters() if q.requires_grad], lr=0.004)

        def dcstep():
            opt_dc.zero_grad()
            R, m, c = net(x)
            calibrate.cumulative_mse(calibrate.TableFunction.apply(ctx, R, m, S, c, [N_SEED]), y_cum).backward()
            opt_dc.step()

        ms_dc = timed(dcstep)
    return {"workload": f"calibration on the same graph: {DAYS} days, weekly-tied R and m, T_E, T_I and "
                        f"the infectiousness profile; MSE on cumulative deaths; Adam",
            "ms_per_step": ms, "steps": steps, "loss_first_last": first_last,
            "dc_calibnn_ms_per_step": ms_dc}


# ---- the other configurations of the workload family -------------------------------
CFG0_AGENTS, CFG0_DAYS = 10_000, 30
CFG3_COUNTIES, CFG3_DAYS = 32, 90
CFG4_AGENTS, CFG4_DAYS = 8_000_000, 120
B1M_SETS, B1M_DAYS = 64, 60
ORACLE_SAMPLE_DAYS = 8


def _gen_population(kind, arg):
    """Worker of the generator pool (spawned processes): one synthetic population."""
    from paper_2207_09714_gb300 import synth
    if kind == "powerlaw":
        return synth.population_typed(arg, seed=0, powerlaw=True)
    g, n = arg
    return synth.county(g, n, seed=0)


class Populations:
    """The large populations of configs 3 and 4, generated by a pool of spawned processes
    while the GPU sections before them run."""

    def __init__(self, workers: int):
        import multiprocessing as mp
        from paper_2207_09714_gb300 import synth
        self.sizes = synth.uneven_county_sizes(CFG3_COUNTIES, seed=0)
        self.pool = mp.get_context("spawn").Pool(processes=workers)
        self.big = self.pool.apply_async(_gen_population, ("powerlaw", CFG4_AGENTS))
        order = sorted(range(len(self.sizes)), key=lambda g: -self.sizes[g])
        self.counties = {g: self.pool.apply_async(_gen_population, ("county", (g, self.sizes[g]))) for g in order}

    def powerlaw(self):
        return self.big.get()

    def county_list(self):
        return [self.counties[g].get() for g in range(len(self.sizes))]

    def close(self):
        self.pool.close()
        self.pool.join()


def _padded_rows(pops):
    return sum(((p.n + 31) // 32) * 32 for p in pops)


def workload_bytes(pops, E, B, T, L, store, l2_bytes):
    """Algorithmic bytes per forward and backward day launch of a ctx over ``pops`` (one
    set per graph, or B sets on one graph) from its final state E [B, n_total], and the
    paper-style full-pull count (every row, every day)."""
    deg = np.concatenate([p.degrees().astype(np.float64) for p in pops])
    NEVER = 32767
    if B == 1:
        n_rows = _padded_rows(pops)
        off = np.concatenate([[0], np.cumsum([p.n for p in pops])])
        parts = [frontier_counts(p, E[0][off[g]:off[g + 1]], T, L) for g, p in enumerate(pops)]
        frontier = tuple(sum(pt[k] for pt in parts) for k in range(3))
        fwd, bwd, _, _ = trajectory_bytes(E[0], deg, T, L, n_rows, store, frontier=frontier)
        ffwd, fbwd, _, _ = trajectory_bytes(np.full(deg.size, NEVER, np.int16), deg, T, L, n_rows, store)
    else:
        n = pops[0].n
        fwd, bwd = batched_trajectory_bytes(E, deg, T, L, n, B, l2_bytes)
        ffwd, fbwd = batched_trajectory_bytes(np.full((B, n), NEVER, np.int16), deg, T, L, n, B, l2_bytes)
    return fwd, bwd, ffwd, fbwd


def bench_workload(name, what, pops, B, T, R_np, m_np, S_np, n_seed, y_np, policy, stream, peak, peak_kind,
                   fwd_only=False, steps=3, warmup=3, autotune=True):
    """One configuration through the library: the ctx, a warm-up, the autotuner, then
    ``steps`` timed steps (forward, or forward + MSE + backward) with CUDA events on the ctx
    stream (day loops replayed as CUDA graphs), one profiled step with events around every
    day launch for the per-kernel rates, algorithmic and full-pull bytes, peak HBM."""
    import torch
    from paper_2207_09714_gb300 import capi, synth
    c = synth.infectiousness_table(TAU_EI, TAU_IR)
    L = TAU_EI + TAU_IR
    I = len(pops) * B
    with torch.cuda.stream(stream):
        ctx = capi.gabm_create(pops, capi.ModelDesc(TAU_EI, TAU_IR, c, seed=0, lambda_policy=policy),
                               sets_per_graph=B, stream=stream)
    R = torch.from_numpy(np.ascontiguousarray(R_np, np.float32)).cuda()
    m = torch.from_numpy(np.ascontiguousarray(m_np, np.float32)).cuda()
    S = torch.from_numpy(np.ascontiguousarray(S_np, np.float32)).cuda()
    y = torch.from_numpy(np.ascontiguousarray(y_np, np.float64)).cuda()
    D = torch.empty((I, T), dtype=torch.float64, device="cuda")
    loss = torch.empty((I,), dtype=torch.float64, device="cuda")
    gD = torch.empty((I, T), dtype=torch.float64, device="cuda")
    dR = torch.empty((I, T), dtype=torch.float64, device="cuda")
    dm = torch.empty((I, T), dtype=torch.float64, device="cuda")
    dS = torch.empty((I, 9), dtype=torch.float64, device="cuda")

    def step():
        capi.gabm_forward(ctx, T, R, m, S, n_seed, D=D)
        if not fwd_only:
            capi.gabm_mse_loss(ctx, y, loss=loss, gD=gD)
            capi.gabm_backward(ctx, gD, dR=dR, dm=dm, dS_age=dS)

    step()
    schedule = capi.gabm_autotune(ctx, 1) if autotune else capi.gabm_get_schedule(ctx)
    for _ in range(max(warmup, 3)):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = capi.gabm_launch_count(ctx)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = capi.gabm_launch_count(ctx) - l0
    ms = e0.elapsed_time(e1) / steps
    capi.gabm_set_profiling(ctx, True)
    step()
    torch.cuda.synchronize()
    f_ms, f_n = capi.gabm_get_profile(ctx, 0)
    b_ms, b_n = capi.gabm_get_profile(ctx, 1)
    capi.gabm_set_profiling(ctx, False)
    E = capi.gabm_get_state(ctx)
    counts = capi.gabm_forward(ctx, T, R, m, S, n_seed, want_counts=True)[1]
    torch.cuda.synchronize()
    counts = counts.cpu().numpy()
    _, peak_mem = capi.gabm_mem_stats(ctx)
    del ctx
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    fwd_b, bwd_b, ffwd_b, fbwd_b = workload_bytes(pops, E, B, T, L, policy == capi.GABM_STORE_LAMBDA, l2)
    n_tot = sum(p.n for p in pops)
    nnz_tot = sum(p.nnz for p in pops)
    units = B * n_tot * T
    f_gbs = fwd_b.sum() / (f_ms / 1e3) / 1e9
    out = {"workload": what, "n_agents": n_tot, "nnz": nnz_tot, "graphs": len(pops), "sets_per_graph": B,
           "days": T, "lambda_policy": "store" if policy == capi.GABM_STORE_LAMBDA else "recompute",
           "step": "forward" if fwd_only else "forward + MSE + backward",
           "ms_per_step": ms, "steps": steps, "value": units / (ms / 1e3), "unit": "agent-days/s",
           "edge_updates_per_s": B * nnz_tot * T / (ms / 1e3), "gpu_launches": launches,
           "schedule": schedule, "peak_hbm_bytes": peak_mem,
           "attack_rate_range": [float(1.0 - (counts[:, -1, 0] / np.repeat([p.n for p in pops], B)).max()),
                                 float(1.0 - (counts[:, -1, 0] / np.repeat([p.n for p in pops], B)).min())],
           "fwd_day": {"launches": f_n, "avg_launch_ms": f_ms / f_n, "alg_bytes_per_launch": fwd_b.sum() / T,
                       "achieved_gbs": f_gbs, "frac": f_gbs / peak}}
    full = ffwd_b.sum() if fwd_only else ffwd_b.sum() + fbwd_b.sum()
    alg = fwd_b.sum() if fwd_only else fwd_b.sum() + bwd_b.sum()
    kern_ms = f_ms if fwd_only else f_ms + b_ms
    if not fwd_only:
        b_gbs = bwd_b.sum() / (b_ms / 1e3) / 1e9
        out["bwd_day"] = {"launches": b_n, "avg_launch_ms": b_ms / b_n, "alg_bytes_per_launch": bwd_b.sum() / T,
                          "achieved_gbs": b_gbs, "frac": b_gbs / peak}
    out["day_kernels"] = {"alg_bytes_per_step": alg, "ms_per_step": kern_ms,
                          "achieved_gbs": alg / (kern_ms / 1e3) / 1e9, "frac": alg / (kern_ms / 1e3) / 1e9 / peak,
                          "peak": peak, "peak_source": peak_kind}
    if B > 1 and len(pops) == 1 and policy == capi.GABM_STORE_LAMBDA:
        wl = f"typed{pops[0].n // 1000}k_B{B}_T{T}_store".replace("1000k", "1M")
        f_dr = dram_rate("k_fwd_day_b", wl, f_ms / f_n, peak)
        b_dr = None if fwd_only else dram_rate("k_bwd_day_b", wl, b_ms / b_n, peak)
        out["fwd_day"]["dram"] = f_dr
        if not fwd_only:
            out["bwd_day"]["dram"] = b_dr
        if f_dr and b_dr:
            tot = f_dr["traffic_bytes_per_launch"] * f_n + b_dr["traffic_bytes_per_launch"] * b_n
            out["day_kernels"]["dram_frac"] = tot / (kern_ms / 1e3) / 1e9 / peak
    out["full_pull"] = {"bytes_per_step": full, "gbs_at_step_time": full / (ms / 1e3) / 1e9,
                        "note": "paper-style count: every row's edges and state on every day"}
    return out


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample(pops, B, T, days, R_np, m_np, S_np, n_seed, y_np, fwd_only, insts=None):
    """The FP64 oracle (OpenMP over the host cores) on a bounded sample of a configuration:
    the first ``days`` days of the instances ``insts`` (all by default), forward (+ MSE +
    backward over those days).  Returns agent-days/s of the sample and its description."""
    import oracle as O
    from paper_2207_09714_gb300 import synth
    md = O.Model(TAU_EI, TAU_IR, synth.infectiousness_table(TAU_EI, TAU_IR), seed=0)
    insts = list(range(len(pops) * B)) if insts is None else insts
    O.build()
    units = 0
    t0 = time.perf_counter()
    for i in insts:
        pop = pops[i // B]
        f = O.forward_hard(pop, md, R_np[i, :days], m_np[i, :days], S_np[i], n_seed=n_seed[i], inst=i)
        if not fwd_only:
            _, gD = O.mse(f["D"], y_np[i, :days])
            O.backward_hard(pop, md, R_np[i, :days], m_np[i, :days], S_np[i], f["e_final"], gD, inst=i)
        units += pop.n * days
    dt = time.perf_counter() - t0
    return {"value": units / dt, "unit": "agent-days/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{len(insts)} of {len(pops) * B} instances, days 0..{days - 1} of {T}, "
                      f"{'forward' if fwd_only else 'forward + MSE + backward'}, FP64, {dt:.1f} s"
                      + ("" if days == T else "; throughput of the first days, not extrapolated")}


def _single_thread_oracle_cmd():
    """Command of a child process that times the oracle single-threaded on the full main
    workload (one forward + MSE + backward of 1M agents over 60 days) and prints JSON."""
    code = (
        "import json,time,numpy as np,oracle as O;"
        "from paper_2207_09714_gb300 import synth;"
        f"pop=synth.population_typed({N_AGENTS},seed=0);"
        f"c=synth.infectiousness_table({TAU_EI},{TAU_IR});md=O.Model({TAU_EI},{TAU_IR},c,seed=0);"
        f"R=np.full({DAYS},{R0},np.float32);m=np.full({DAYS},{MORTALITY},np.float32);"
        "S=synth.SUSCEPTIBILITY.astype(np.float32);"
        f"y=synth.target_curve({DAYS},pop.n);O.build();t0=time.perf_counter();"
        f"f=O.forward_hard(pop,md,R,m,S,n_seed={N_SEED});_,gD=O.mse(f['D'],y);"
        "O.backward_hard(pop,md,R,m,S,f['e_final'],gD);dt=time.perf_counter()-t0;"
        f"print(json.dumps({{'seconds':dt,'threads':O.num_threads(),'value':pop.n*{DAYS}/dt}}))")
    return [sys.executable, "-c", code]


CONFIG_KEYS = {"c0": "c0_10k_forward_30d", "b1m": "batched_1M_x64_60d", "c3": "c3_32_counties_90d",
               "c4": "c4_8M_powerlaw_120d"}


def run_configs(args, gen, pop1m, stream, peak, peak_kind, only=None):
    """The other configurations, each in its own key (a failure is reported there):
    10k agents forward only (30 days); 1M agents x 64 parameter sets (60 days); 32 uneven
    counties (90 days); 8M agents with power-law contacts (120 days, recompute policy).
    The single-threaded oracle runs in a child process meanwhile (after the generator
    pool has finished, so that nothing else loads the host), and the OpenMP oracle on a
    bounded sample of each configuration after the GPU sections."""
    from paper_2207_09714_gb300 import capi, synth
    out = {}
    samples = {}
    rng = np.random.default_rng(0)

    def guarded(key, fn):
        if only is not None and CONFIG_KEYS[only] != key:
            return
        try:
            out[key] = fn()
        except Exception as exc:   # reported, the other sections still run
            out[key] = {"error": f"{type(exc).__name__}: {exc}"}

    # config 0: 10k agents, households + random contacts, forward only
    p0 = synth.population_small(CFG0_AGENTS, seed=0)
    R0v = np.full((1, CFG0_DAYS), R0, np.float32)
    m0v = np.full((1, CFG0_DAYS), MORTALITY, np.float32)
    S0v = synth.SUSCEPTIBILITY[None, :].astype(np.float32)
    y0 = synth.target_curve(CFG0_DAYS, p0.n)[None, :]
    guarded("c0_10k_forward_30d", lambda: bench_workload(
        "c0", f"{p0.n} agents, households U{{1..6}} + random contacts (mean degree 10), {CFG0_DAYS} days, forward only",
        [p0], 1, CFG0_DAYS, R0v, m0v, S0v, [N_SEED], y0, capi.GABM_STORE_LAMBDA, stream, peak, peak_kind,
        fwd_only=True, steps=20))

    # 1M agents x 64 parameter sets, 60 days (the main graph, the ensemble's parameter ranges)
    Rb = np.repeat(rng.uniform(1.5, 4.0, (B1M_SETS, 1)), B1M_DAYS, axis=1).astype(np.float32)
    mb = np.repeat(rng.uniform(0.005, 0.05, (B1M_SETS, 1)), B1M_DAYS, axis=1).astype(np.float32)
    Sb = np.tile(synth.SUSCEPTIBILITY, (B1M_SETS, 1)).astype(np.float32)
    yb = np.stack([synth.target_curve(B1M_DAYS, N_AGENTS, seed=b) for b in range(B1M_SETS)])
    guarded("batched_1M_x64_60d", lambda: bench_workload(
        "b1m", f"one shared {pop1m.n}-agent typed contact graph, {B1M_SETS} parameter sets (R ~ U[1.5, 4.0], "
               f"m ~ U[0.005, 0.05]), {B1M_DAYS} days, forward + MSE + backward of every set",
        [pop1m], B1M_SETS, B1M_DAYS, Rb, mb, Sb, [N_SEED] * B1M_SETS, yb, capi.GABM_STORE_LAMBDA, stream, peak,
        peak_kind, steps=3))

    if only in ("c0", "b1m"):
        return out
    if gen is not None:
        counties = gen.county_list() if only in (None, "c3") else []
        p4 = gen.powerlaw() if only in (None, "c4") else None
        gen.close()
    else:
        counties = ([synth.county(g, n) for g, n in enumerate(synth.uneven_county_sizes(CFG3_COUNTIES, seed=0))]
                    if only in (None, "c3") else [])
        p4 = synth.population_typed(CFG4_AGENTS, seed=0, powerlaw=True) if only in (None, "c4") else None
    single = None
    if not args.no_cpu_baseline and only is None:
        single = subprocess.Popen(_single_thread_oracle_cmd(), stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                  text=True, cwd=ROOT, env=dict(os.environ, OMP_NUM_THREADS="1"))

    # config 3: 32 uneven counties, each with its own parameters, 90 days
    G = max(len(counties), 1)
    R3 = (rng.uniform(1.8, 3.2, (G, 1)) * rng.uniform(0.9, 1.1, (G, CFG3_DAYS))).astype(np.float32)
    m3 = np.repeat(rng.uniform(0.005, 0.05, (G, 1)), CFG3_DAYS, axis=1).astype(np.float32)
    S3 = (synth.SUSCEPTIBILITY[None, :] * rng.uniform(0.8, 1.2, (G, 9))).astype(np.float32)
    y3 = (np.stack([synth.target_curve(CFG3_DAYS, p.n, seed=g) for g, p in enumerate(counties)]) if counties
          else np.zeros((1, CFG3_DAYS)))
    guarded("c3_32_counties_90d", lambda: bench_workload(
        "c3", f"{G} county graphs of the typed generator, agent counts log-uniform in [5e4, 2e6] "
              f"(sum {sum(p.n for p in counties)}), own parameters each, {CFG3_DAYS} days, autotuned, "
              f"forward + MSE + backward", counties, 1, CFG3_DAYS, R3, m3, S3, [N_SEED] * G, y3,
        capi.GABM_STORE_LAMBDA, stream, peak, peak_kind, steps=3))

    # config 4: 8M agents, power-law random contacts, 120 days, recompute policy
    R4 = np.full((1, CFG4_DAYS), R0, np.float32)
    m4 = np.full((1, CFG4_DAYS), MORTALITY, np.float32)
    S4 = synth.SUSCEPTIBILITY[None, :].astype(np.float32)
    y4 = synth.target_curve(CFG4_DAYS, p4.n if p4 is not None else CFG4_AGENTS)[None, :]
    guarded("c4_8M_powerlaw_120d", lambda: bench_workload(
        "c4", f"{p4.n} agents, typed generator with Chung-Lu power-law contacts (exponent 2.5, degrees up to "
              f"2000), {CFG4_DAYS} days, recompute policy (lambda recomputed from the final exposure days), "
              f"forward + MSE + backward", [p4], 1, CFG4_DAYS, R4, m4, S4, [N_SEED], y4, capi.GABM_RECOMPUTE,
        stream, peak, peak_kind, steps=3))

    if single is not None:
        try:
            so, _ = single.communicate(timeout=900)
            st = json.loads(so.strip().splitlines()[-1])
            out["_single_thread"] = {"value": st["value"], "unit": "agent-days/s", "cores": st["threads"],
                                     "kind": "oracle",
                                     "sample": f"one forward + MSE + backward of the full main workload, one thread, "
                                               f"{st['seconds']:.1f} s (child process, run while the GPU sections "
                                               f"ran)"}
        except Exception as exc:
            single.kill()
            out["_single_thread"] = {"error": f"{type(exc).__name__}: {exc}"}
        try:   # the OpenMP oracle on bounded samples of each configuration
            samples["c0_10k_forward_30d"] = oracle_sample([p0], 1, CFG0_DAYS, CFG0_DAYS, R0v, m0v, S0v, [N_SEED],
                                                          y0, True)
            samples["batched_1M_x64_60d"] = oracle_sample([pop1m], B1M_SETS, B1M_DAYS, B1M_DAYS, Rb, mb, Sb,
                                                          [N_SEED] * B1M_SETS, yb, False, insts=[0])
            samples["c3_32_counties_90d"] = oracle_sample(counties, 1, CFG3_DAYS, ORACLE_SAMPLE_DAYS, R3, m3, S3,
                                                          [N_SEED] * G, y3, False)
            samples["c4_8M_powerlaw_120d"] = oracle_sample([p4], 1, CFG4_DAYS, ORACLE_SAMPLE_DAYS, R4, m4, S4,
                                                           [N_SEED], y4, False)
        except Exception as exc:
            samples["error"] = f"{type(exc).__name__}: {exc}"
        out["_oracle_samples"] = samples
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--policy", default="store", choices=["store", "recompute"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched ensemble; its result is the printed line")
    ap.add_argument("--no-plain", action="store_true", help="skip the per-set plain comparator")
    ap.add_argument("--batched-agents", type=int, default=BATCH_AGENTS,
                    help="agents of the batched ensemble's graph (smaller cases for profiling)")
    ap.add_argument("--batched-days", type=int, default=BATCH_DAYS, help="days of the batched ensemble")
    ap.add_argument("--batched-schedule", default="",
                    help="fwd_sets_per_lane,bwd_sets_per_lane,fwd_smem_bitmap,bwd_sets_per_launch for the "
                         "batched ensemble instead of the autotuner's choice")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations (10k forward, 1M x 64 sets, 32 counties, 8M power-law)")
    ap.add_argument("--only", choices=sorted(CONFIG_KEYS),
                    help="run only this configuration (c0: 10k forward, b1m: 1M x 64 sets, c3: 32 counties, "
                         "c4: 8M power-law) and print its result as the JSON line")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, world, rank)
        return

    extra = world == 1 and not args.no_configs and not args.batched_only
    gen = Populations(workers=max(1, min(8, (os.cpu_count() or 2) // 2))) if extra else None

    import torch
    from paper_2207_09714_gb300 import build as gbuild
    from paper_2207_09714_gb300 import capi, synth

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    gbuild.build()
    if args.only:
        stream = torch.cuda.Stream()
        peak, peak_kind = _peaks()
        pop1m = synth.population_typed(N_AGENTS, seed=0) if args.only == "b1m" else None
        with ClockSampler(local) as clk:
            res = run_configs(args, None, pop1m, stream, peak, peak_kind, only=args.only)[CONFIG_KEYS[args.only]]
        if rank == 0:
            print(json.dumps({"only": CONFIG_KEYS[args.only], "clocks": clk.summary(), **res}), flush=True)
        return
    if args.batched_only:
        stream = torch.cuda.Stream()
        peak, peak_kind = _peaks()
        with ClockSampler(local) as clk:
            b = bench_batched(args, stream, peak, peak_kind)
        if rank == 0:
            line = {"metric": METRIC, "value": b["value"], "unit": "agent-days/s", "n_gpus": world,
                    "steps": b["steps"], "warmup": max(args.warmup, 3), "ms_per_step": b["ms_per_step"],
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                    "data": "synthetic", "config": {"workload": b["workload"]}, "roofline": b["roofline"],
                    "gpu_launches": b["gpu_launches"], "clocks": clk.summary(), "batched": b}
            print(json.dumps(line), flush=True)
        return

    pop = synth.population_typed(N_AGENTS, seed=0)
    c = synth.infectiousness_table(TAU_EI, TAU_IR)
    policy = capi.GABM_STORE_LAMBDA if args.policy == "store" else capi.GABM_RECOMPUTE
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = capi.gabm_create([pop], capi.ModelDesc(TAU_EI, TAU_IR, c, seed=rank, lambda_policy=policy),
                               stream=stream)
    R = torch.full((1, DAYS), R0, dtype=torch.float32, device="cuda")
    m = torch.full((1, DAYS), MORTALITY, dtype=torch.float32, device="cuda")
    S = torch.from_numpy(synth.SUSCEPTIBILITY[None, :].copy()).cuda()
    y_np = synth.target_curve(DAYS, pop.n)[None, :]
    y = torch.from_numpy(y_np).cuda()
    D = torch.empty((1, DAYS), dtype=torch.float64, device="cuda")
    loss = torch.empty((1,), dtype=torch.float64, device="cuda")
    gD = torch.empty((1, DAYS), dtype=torch.float64, device="cuda")
    dR = torch.empty((1, DAYS), dtype=torch.float64, device="cuda")
    dm = torch.empty((1, DAYS), dtype=torch.float64, device="cuda")
    dS = torch.empty((1, 9), dtype=torch.float64, device="cuda")

    def step(ev_mid=None):
        capi.gabm_forward(ctx, DAYS, R, m, S, [N_SEED], D=D)
        if ev_mid is not None:
            ev_mid.record(stream)
        capi.gabm_mse_loss(ctx, y, loss=loss, gD=gD)
        capi.gabm_backward(ctx, gD, dR=dR, dm=dm, dS_age=dS)

    torch.cuda.synchronize()
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # ---- timed region (device-resident inputs; day loops replayed as CUDA graphs) ----
    launches0 = capi.gabm_launch_count(ctx)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            starts[k].record(stream)
            step(mids[k])
            ends[k].record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = capi.gabm_launch_count(ctx) - launches0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    fwd_ms = [s.elapsed_time(e) for s, e in zip(starts, mids)]
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    ms_per_step = total_ms / args.steps
    units = world * pop.n * DAYS
    value = job_throughput(pop.n * DAYS, world, ms_per_step)
    fwd_value = world * pop.n * DAYS / (statistics.median(fwd_ms) / 1e3)

    # ---- the same steps again with CUDA events around every day launch (eager launches):
    # per-kernel durations for the roofline ----
    capi.gabm_set_profiling(ctx, True)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for k in range(args.steps):
        step()
    p1.record(stream)
    torch.cuda.synchronize()
    ms_per_step_profiled = p0.elapsed_time(p1) / args.steps
    fwd_ms_k, fwd_n = capi.gabm_get_profile(ctx, 0)
    bwd_ms_k, bwd_n = capi.gabm_get_profile(ctx, 1)
    capi.gabm_set_profiling(ctx, False)

    # ---- algorithmic bytes of the day kernels, from this trajectory ----
    E = capi.gabm_get_state(ctx)[0]
    deg = pop.degrees().astype(np.float64)
    n_rows = ((pop.n + 31) // 32) * 32
    frontier = frontier_counts(pop, E, DAYS, TAU_EI + TAU_IR)
    fwd_b, bwd_b, S_cnt, S_nnz = trajectory_bytes(E, deg, DAYS, TAU_EI + TAU_IR, n_rows,
                                                  policy == capi.GABM_STORE_LAMBDA, frontier=frontier)
    fwd_gbs = fwd_b.sum() * args.steps / (fwd_ms_k / 1e3) / 1e9 if fwd_ms_k > 0 else None
    bwd_gbs = bwd_b.sum() * args.steps / (bwd_ms_k / 1e3) / 1e9 if bwd_ms_k > 0 else None
    peak, peak_kind = _peaks()
    dominant = "k_bwd_day" if bwd_ms_k >= fwd_ms_k else "k_fwd_day"
    src = ["backward.cu", "rowsum.cuh", "gabm_internal.cuh"] if dominant == "k_bwd_day" else \
          ["forward.cu", "rowsum.cuh", "gabm_internal.cuh"]
    workload_tag = f"typed1M_T{DAYS}_{args.policy}"
    traffic = _ncu_traffic(dominant, _kernel_source_sha(src), workload_tag)
    fwd_dr = dram_rate("k_fwd_day", workload_tag, fwd_ms_k / fwd_n if fwd_n else 0.0, peak)
    bwd_dr = dram_rate("k_bwd_day", workload_tag, bwd_ms_k / bwd_n if bwd_n else 0.0, peak)
    dom_gbs = bwd_gbs if dominant == "k_bwd_day" else fwd_gbs
    dom_bytes = (bwd_b.sum() if dominant == "k_bwd_day" else fwd_b.sum()) / DAYS
    dom_ms = (bwd_ms_k / bwd_n) if dominant == "k_bwd_day" else (fwd_ms_k / fwd_n)

    # ---- end to end through the C ABI with pinned host buffers ----
    Rh = torch.full((1, DAYS), R0, dtype=torch.float32).pin_memory()
    mh = torch.full((1, DAYS), MORTALITY, dtype=torch.float32).pin_memory()
    Sh = torch.from_numpy(synth.SUSCEPTIBILITY[None, :].copy()).pin_memory()
    yh = torch.from_numpy(y_np.copy()).pin_memory()
    Dh = torch.empty((1, DAYS), dtype=torch.float64).pin_memory()
    lh = torch.empty((1,), dtype=torch.float64).pin_memory()
    gDh = torch.empty((1, DAYS), dtype=torch.float64).pin_memory()
    dRh = torch.empty((1, DAYS), dtype=torch.float64).pin_memory()
    dmh = torch.empty((1, DAYS), dtype=torch.float64).pin_memory()
    dSh = torch.empty((1, 9), dtype=torch.float64).pin_memory()

    def e2e_step():
        capi.gabm_forward(ctx, DAYS, Rh, mh, Sh, [N_SEED], D=Dh)
        capi.gabm_mse_loss(ctx, yh, loss=lh, gD=gDh)
        capi.gabm_backward(ctx, gDh, dR=dRh, dm=dmh, dS_age=dSh)

    e2e_step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    e2e_value = job_throughput(pop.n * DAYS, world, e2e_ms / args.steps)
    h2d = (Rh.numel() * 4 + mh.numel() * 4 + Sh.numel() * 4 + yh.numel() * 8 + gDh.numel() * 8)
    d2h = (Dh.numel() * 8 + lh.numel() * 8 + gDh.numel() * 8 + dRh.numel() * 8 + dmh.numel() * 8 + dSh.numel() * 8)

    cur, peak_mem = capi.gabm_mem_stats(ctx)
    calib = bench_calibration(ctx, stream, S, y_np, dist)
    del ctx
    twohop = bench_twohop(stream, dist)
    rm_split = bench_progression_variant(pop, stream, S, y_np, dist, peak, peak_kind, "rm_split")
    durations = bench_progression_variant(pop, stream, S, y_np, dist, peak, peak_kind, "durations")
    batched = None
    if not args.no_batched:
        batched = bench_batched(args, stream, peak, peak_kind)
    try:   # a failure here is reported in its own key
        sirs = bench_progression_variant(pop, stream, S, y_np, dist, peak, peak_kind, "sirs")
    except Exception as exc:
        sirs = {"error": f"{type(exc).__name__}: {exc}"}
    configs = run_configs(args, gen, pop, stream, peak, peak_kind) if extra else None
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(pop, c, y_np[0])
        if configs is not None:
            cpu["single_thread"] = configs.pop("_single_thread", None)
            cpu["per_config"] = configs.pop("_oracle_samples", None)
    if configs is not None:
        configs.pop("_single_thread", None)
        configs.pop("_oracle_samples", None)
    full_fwd, full_bwd = (trajectory_bytes(np.full(pop.n, 32767, np.int16), deg, DAYS, TAU_EI + TAU_IR, n_rows,
                                           policy == capi.GABM_STORE_LAMBDA)[:2])
    line = {
        "metric": METRIC, "value": value, "unit": "agent-days/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(pop, args.policy),
        "fwd_agent_days_per_s": fwd_value,
        "ms_per_step_profiled": ms_per_step_profiled,
        "edge_updates_per_s": world * pop.nnz * DAYS / (ms_per_step / 1e3),
        "sus_edges_per_day_mean": float(S_nnz.mean()),
        "summed_edges_per_day_mean": float(frontier[1].mean()),
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": dom_gbs, "peak": peak, "unit": "GB/s",
                     "frac": (dom_gbs / peak) if dom_gbs else None, "traffic": traffic,
                     "peak_source": peak_kind,
                     "alg_bytes_per_launch": dom_bytes, "avg_launch_ms": dom_ms,
                     "dram_frac": (bwd_dr if dominant == "k_bwd_day" else fwd_dr or {}).get("dram_frac")
                     if (bwd_dr if dominant == "k_bwd_day" else fwd_dr) else None,
                     "fwd_day": {"achieved": fwd_gbs, "launches": fwd_n, "ms_total": fwd_ms_k, "dram": fwd_dr},
                     "bwd_day": {"achieved": bwd_gbs, "launches": bwd_n, "ms_total": bwd_ms_k, "dram": bwd_dr}},
        "e2e": {"value": e2e_value, "unit": "agent-days/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "peak_hbm_bytes": peak_mem,
        "cpu_baseline": cpu,
        "calibration": calib,
        "agent_location": twohop,
        "rm_split": rm_split,
        "stochastic_durations": durations,
        "sirs_reinfection": sirs,
        "batched": batched,
        "full_pull": {"bytes_per_step": float(full_fwd.sum() + full_bwd.sum()),
                      "gbs_at_step_time": float(full_fwd.sum() + full_bwd.sum()) / (ms_per_step / 1e3) / 1e9,
                      "frac": float(full_fwd.sum() + full_bwd.sum()) / (ms_per_step / 1e3) / 1e9 / peak,
                      "note": "paper-style count: every row's edges and state on every day, forward and backward"},
        "configs": configs,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
