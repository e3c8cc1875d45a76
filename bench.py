"""Benchmark of the adaptive-multigrid hot path on one GB300 (or N replicas).

One step is one pass of the whole hot path on the production-shaped
3-level workload (fine 32^3x64 Wilson-clover, 4^4 then 2^4 aggregates,
24 then 32 null vectors, FP32 levels, FP64 outer GCR):

    setup level 0 (MR sweeps on M x = 0, FP64 block Gram-Schmidt)
    -> Galerkin build of level 1 -> setup level 1 -> Galerkin build of level 2
    -> K-cycle GCR solve of M x = b to 1e-10.

value = coarse-apply throughput (algorithmic bytes / kernel time) of every
level-1 coarse apply inside the timed steps, timed by CUDA events that the
library records on the launching stream.  The level-1 links are 1.36 GB, so
inputs are larger than the 129 MB L2 and no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--form fp32|bf16|fp16]
    python bench.py --impl reference   # the CPU oracle timed on a bounded sample

Under torchrun with N > 1 every rank runs its own replica (the method's
lattice is not split across GPUs here: "replicas only"), a barrier brackets
the timed region and the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as syn  # noqa: E402

WORKLOAD = "c2_32^3x64_3lvl_fp32"
METRIC = "coarse_apply GB/s (% HBM peak); MG-GCR s/solve at 1e-10, plain vs tuned forms"


# DRAM traffic per launch of the level-1 coarse apply from one ncu capture,
# valid only for the kernel source it was taken on; reported as null once
# that source changes.
NCU_TRAFFIC = {
    # dram__bytes_read.sum + dram__bytes_write.sum of one launch; "src" is the
    # digest of the k_coarse_stream function text the capture was taken on
    "fp32": {"bytes": 1.362160e9 + 4.048384e6, "src": "fb66ef864905ed61"},
    "bf16": {"bytes": 0.682689e9 + 3.623936e6, "src": "fb66ef864905ed61"},
}


def kernel_digest(path, name):
    """sha256[:16] of a kernel's source text: from the line that opens its
    parameter list to the closing brace at column 0."""
    import hashlib
    with open(path) as fh:
        lines = fh.read().split("\n")
    start = next(i for i, ln in enumerate(lines) if ln.strip().startswith(name + "("))
    end = next(i for i in range(start, len(lines)) if lines[i] == "}")
    return hashlib.sha256("\n".join(lines[start:end + 1]).encode()).hexdigest()[:16]


def coarse_traffic(form):
    rec = NCU_TRAFFIC.get(form)
    if rec is None:
        return None
    src = os.path.join(ROOT, "paper_1612_07873_gb300", "csrc", "coarse.cu")
    return rec["bytes"] if kernel_digest(src, "k_coarse_stream") == rec["src"] else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, path: str = ""):
        import tempfile
        self.index = index
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), f"gbmg_clocks_rank{index}.csv")

    def start(self):
        try:
            if os.path.dirname(self.path):
                os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle leg
def _limit_threads():
    try:
        from threadpoolctl import threadpool_limits
        return threadpool_limits(1)
    except Exception:
        return None


def _oracle_apply_worker(job):
    """One process of the CPU baseline: the FP64 oracle's Eq. (3) on its
    own chunk of coarse sites, repeated for `budget_s` seconds (one thread)."""
    import sys
    sys.path.insert(0, ROOT)
    from oracle import dirac, lattice as lat
    n, cdims, lo, hi, budget_s = job
    _limit_threads()
    vol = lat.volume(cdims)
    rng = np.random.default_rng(1000 + lo)
    sel = np.arange(lo, hi)
    blocks = rng.standard_normal((hi - lo, 9, n, n)) + 1j * rng.standard_normal((hi - lo, 9, n, n))
    g = np.random.default_rng(5)
    psi = g.standard_normal((vol, n)) + 1j * g.standard_normal((vol, n))
    reps, t0 = 0, time.perf_counter()
    while True:
        dirac.apply_at(blocks, psi, cdims, sel)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return reps, el, (hi - lo) * (9 * n * n * 16 + 2 * n * 16)


def oracle_coarse_apply_sample(n=48, cdims=(8, 8, 8, 16), budget_s=12.0, cores=None):
    """The FP64 oracle stencil apply (Eq. 3) on the whole level-1 lattice,
    its sites split into one chunk per host core, each chunk applied by its
    own process (one thread each) for about budget_s seconds; returns the
    summed GB/s of FP64 algorithmic bytes (links + spinor in and out).  The
    processes are spawned: forked children of a CUDA process can hang."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from oracle import lattice as lat
    cores = cores or (os.cpu_count() or 1)
    vol = lat.volume(cdims)
    edges = np.linspace(0, vol, cores + 1).astype(int)
    jobs = [(n, tuple(cdims), int(edges[i]), int(edges[i + 1]), budget_s) for i in range(cores)]
    with cf.ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_apply_worker, jobs))
    gbs = sum(b * r / el for r, el, b in res) / 1e9
    reps = sum(r for r, _, _ in res)
    return dict(value=gbs, unit="GB/s", cores=cores, kind="oracle",
                sample=f"FP64 numpy Eq. (3) apply on all {vol} sites of the {tuple(cdims)} n={n} "
                       f"level-1 lattice, split over {cores} processes (one per host core, one "
                       f"thread each), {reps} chunk applies in about {budget_s:.0f} s each; GB/s "
                       f"of FP64 algorithmic bytes (links + in/out spinor) summed over processes")


def reference_main(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    samples = []
    for _ in range(args.warmup):
        oracle_coarse_apply_sample(budget_s=1.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        samples.append(oracle_coarse_apply_sample(budget_s=max(2.0, 20.0 / args.steps)))
    el = time.perf_counter() - t0
    v = statistics.median(s["value"] for s in samples)
    base = dict(samples[-1])
    base["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "oracle-fp64", "l2": "host"},
            "cpu_baseline": base,
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- multi-rank
def aggregate_ranks(ms_total, kernel_ms, kernel_bytes, device):
    """Replicas: the step time and the kernel time of the job are the maxima
    over ranks, the bytes moved are summed (whole-job throughput)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_total, kernel_ms, kernel_bytes], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(mx[1]), float(sm[2])


# ---------------------------------------------------------------- learned setup
LEARNED_EVAL_SEEDS = (2000, 2001, 2002)


def _stats(vals):
    return {"per_field": vals, "mean": float(np.mean(vals)), "min": min(vals), "max": max(vals)}


def run_learned(args, gb, torch, dev):
    """The learned setup (an addition; the paper draws x0 at random) against
    its controls.  Training: the plain setup's block-orthonormal null
    vectors (Gaussian starts, 10 MR sweeps, m = -0.90) of `ntrain` seeded
    16^4 fields with eps ~ U[0.3, 0.6] (seeds 1000 + i), `epochs` passes of
    Adam, one step per field; held-out loss on four more 16^4 fields (eps
    0.45) after 0, 25, 50, 100, 200 fields of the first pass.  Evaluation:
    three held-out fields of the production shape (32^3x64, eps 0.55, seeds
    2000..2002) at m = -0.90 (near critical for these fields), 3-level MG to
    1e-10 after a setup of k sweeps from
      trained    -- the network's proposals (k = 0, 2, 5),
      untrained  -- the same network with its initial parameters (same seed),
      free_field -- low-momentum plane waves (synthetic.free_field_starts),
      gaussian   -- the plain setup's Gaussian starts (k = 0, 2, 5, 10).
    Outer iterations and s/solve are reported per field with mean, min, max."""
    from paper_1612_07873_gb300 import learned
    mass, nv, tdims, tblock = -0.90, 24, (16, 16, 16, 16), (4, 4, 4, 4)
    ntrain, epochs, lr = args.learned_ntrain, args.learned_epochs, 2e-3
    t0 = time.perf_counter()
    seeds = [1000 + i for i in range(ntrain)]
    eps = [0.3 + 0.3 * np.random.default_rng(sd).random() for sd in seeds]
    fields = syn.gauge_fields(tdims, eps, seeds)
    hseeds = [1900 + i for i in range(4)]
    hfields = syn.gauge_fields(tdims, [0.45] * len(hseeds), hseeds)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()

    def target(U, sd):
        Ud = torch.from_numpy(U).to(dev)
        return (tdims, Ud, learned.plain_vectors(Ud, tdims, tblock, nv, mass, 1.0, 10, sd + 4000))
    samples = [target(U, sd) for U, sd in zip(fields, seeds)]
    held = [target(U, sd) for U, sd in zip(hfields, hseeds)]
    del fields, hfields
    torch.cuda.synchronize()
    t_targets = time.perf_counter() - t0

    P = learned.Proposer(nv, seed=3)
    P0 = learned.Proposer(nv, seed=3)  # the untrained control: the same initial parameters

    def heldout(net):
        return float(np.mean([net.loss(d, tblock, U, T) for d, U, T in held]))
    loss_untrained = heldout(P0)
    curve = [{"fields_seen": 0, "heldout_loss": loss_untrained}]
    marks = {25, 50, 100, 200, ntrain}
    hist, t_train, steps = [], 0.0, 0
    for ep in range(epochs):
        tot = 0.0
        for k, (d, U, T) in enumerate(samples):
            ts = time.perf_counter()
            tot += P.step(d, tblock, U, T, lr)
            t_train += time.perf_counter() - ts
            steps += 1
            if ep == 0 and (k + 1) in marks:
                curve.append({"fields_seen": k + 1, "heldout_loss": heldout(P)})
        hist.append(tot / len(samples))
    loss_trained = heldout(P)
    del samples, held

    w = syn.WORKLOADS[WORKLOAD]
    dims = w["dims"]
    vol = syn.volume(dims)
    b = torch.from_numpy(syn.gaussian_field((vol, 12), 5, stream=99)).to(dev)
    p3 = gb.default_params(dims=dims, block=w["block"], nvec=w["nvec"], mass=mass, csw=1.0,
                           nlevels=3, prec_fine=1, prec_coarse=1, seed=9000)
    ff = torch.from_numpy(syn.free_field_starts(dims, nv)).to(dev)
    plan = {"trained": (0, 2, 5), "untrained": (0, 2, 5), "free_field": (0, 2, 5),
            "gaussian": (0, 2, 5, 10)}
    res = {name: {k: {"iters": [], "s": [], "res": []} for k in ks} for name, ks in plan.items()}
    for fs in LEARNED_EVAL_SEEDS:
        Ue = torch.from_numpy(syn.gauge_field(dims, 0.55, fs)).to(dev)
        starts = {"trained": P.propose(dims, Ue), "untrained": P0.propose(dims, Ue),
                  "free_field": ff, "gaussian": None}
        for name, ks in plan.items():
            for k in ks:
                st = learned.mg_iterations(p3, Ue, starts[name], k, b)
                r = res[name][k]
                r["iters"].append(st["iters"] if st["status"] == 0 else -1)
                r["s"].append(st["seconds"])
                r["res"].append(st["true_residual"])
        del starts, Ue
    P.close()
    P0.close()
    rows = {name: {str(k): {"outer_iters": _stats(r["iters"]),
                            "s_per_solve": _stats([round(v, 4) for v in r["s"]]),
                            "max_true_residual": max(r["res"])}
                   for k, r in ks.items()} for name, ks in res.items()}
    plain = np.mean(res["gaussian"][10]["iters"])
    saved = [10 - k for k in plan["trained"] if np.mean(res["trained"][k]["iters"]) <= plain]
    return {"mass": mass, "train_fields": ntrain, "train_eps": [0.3, 0.6],
            "train_lattice": list(tdims), "epochs": epochs, "adam_lr": lr,
            "targets": "plain setup: Gaussian starts, 10 MR sweeps, block-orthonormalised",
            "fields_gen_s": t_gen, "targets_s": t_targets, "train_s": t_train,
            "train_ms_per_step": 1e3 * t_train / max(steps, 1),
            "loss_per_epoch": hist,
            "heldout_loss": {"untrained": loss_untrained, "trained": loss_trained},
            "heldout_loss_vs_fields_seen": curve,
            "eval_lattice": list(dims), "eval_eps": 0.55, "eval_seeds": list(LEARNED_EVAL_SEEDS),
            "rows": rows, "setup_sweeps_saved": max(saved) if saved else 0}


def run_precision(args, gb, torch, dev):
    """Config 3, the precision forms of the small 2-level workload (8^4,
    2^4 aggregates, 24 vectors, m = -0.2): the FP64 oracle builds its
    hierarchy (10 MR sweeps from the seeded x0, block QR, Galerkin; timed:
    the oracle's s/build on one core) and solves b to 1e-10 (s/solve).  The
    GPU then takes the oracle's block-orthonormal null vectors, builds its
    own Galerkin operator and stores it as FP64, FP32, BF16, FP16 or int16
    (the fine operator FP64 for the first form, FP32 for the others), and
    each level's apply is compared with the oracle's on a Gaussian vector
    (relative L2); the MG-GCR solve of the same b gives the outer and
    per-level iteration counts."""
    from oracle import dirac, solvers
    w = syn.WORKLOADS["c1_8^4_2lvl_fp64"]
    dims, block, nv = w["dims"], w["block"][0], w["nvec"][0]
    vol = syn.volume(dims)
    U = syn.gauge_field(dims, w["eps"], w["seed"])
    x0 = syn.gaussian_field((nv, vol, 12), w["seed"], stream=10)
    b = syn.gaussian_field((vol, 12), w["seed"], stream=99)
    lim = _limit_threads()
    t0 = time.perf_counter()
    op = dirac.wilson_clover_op(U, dims, w["mass"], w["csw"], True)
    hier = solvers.MultigridHierarchy.build(op, [x0], w["sweeps"], [block])
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    ref = hier.solve(b, 1e-10, 100)
    t_solve = time.perf_counter() - t0
    cop = hier.ops[1]
    v0 = syn.gaussian_field((vol, 12), 31)
    v1 = syn.gaussian_field((cop.vol, cop.nd), 32)
    want = [op.apply(v0), cop.apply(v1)]
    if lim is not None and hasattr(lim, "unregister"):
        lim.unregister()
    Ud = torch.from_numpy(U).to(dev)
    Qd = torch.from_numpy(hier.Qs[0]).to(dev)
    bd = torch.from_numpy(b).to(dev)
    forms = {}
    for name, pf, pc in (("fp64", 0, 0), ("fp32", 1, 1), ("bf16", 1, 2), ("fp16", 1, 3),
                         ("int16", 1, 4)):
        p = gb.default_params(dims=dims, block=[block], nvec=[nv], mass=w["mass"], csw=w["csw"],
                              nlevels=2, prec_fine=pf, prec_coarse=pc, setup_sweeps=w["sweeps"],
                              t_antiperiodic=w["antiperiodic"])
        mg = gb.Multigrid(p, Ud)
        gb.mg_set_nullvecs(mg.ctx, 0, Qd)
        gb.mg_build_coarse(mg.ctx, 0)
        errs = []
        for lv, v, ref_y in ((0, v0, want[0]), (1, v1, want[1])):
            dt = mg.levels[lv]["dtype"]
            x = torch.from_numpy(v).to(dev, dt)
            y = torch.empty_like(x)
            gb.mg_apply(mg.ctx, lv, y, x)
            got = y.cpu().numpy().astype(np.complex128)
            errs.append(float(np.linalg.norm(got - ref_y) / np.linalg.norm(ref_y)))
        xs = torch.zeros_like(bd)
        st = gb.mg_gcr_solve(mg.ctx, xs, bd, 1e-10, 200)
        forms[name] = {"fine": "fp64" if pf == 0 else "fp32", "links": name,
                       "apply_rel_l2_vs_oracle": {"level0": errs[0], "level1": errs[1]},
                       "outer_iters": st["iters"], "level_iters": st["level_iters"],
                       "true_residual": st["true_residual"]}
        mg.close()
    return {"workload": "c1_8^4_2lvl_fp64 (fine 8^4, 2^4 aggregates, 24 vectors, m = -0.2)",
            "oracle": {"outer_iters": ref.iters, "true_residual": ref.true_residual,
                       "s_per_build": t_build, "s_per_solve": t_solve, "cores": 1},
            "forms": forms}


def precision_main(args):
    """Only the config-3 precision study (see run_precision); one JSON line."""
    import torch

    import paper_1612_07873_gb300 as gb
    out = run_precision(args, gb, torch, torch.device("cuda"))
    print(json.dumps({"mode": "precision", "precision": out}), flush=True)
    return 0


def learned_main(args):
    """Only the learned-setup study (see run_learned); one JSON line."""
    import torch

    import paper_1612_07873_gb300 as gb
    out = run_learned(args, gb, torch, torch.device("cuda"))
    print(json.dumps({"mode": "learned", "learned_setup": out}), flush=True)
    return 0


# ---------------------------------------------------------------- forms
FORMS = (
    # (name, coarse link store, link slots, RHS per call, red-black, fine smoother)
    ("fp32", 1, 9, 1, 0, 1),
    ("bf16", 2, 9, 1, 0, 1), ("fp16", 3, 9, 1, 0, 1), ("int16", 4, 9, 1, 0, 1),
    ("fp32_5blocks", 1, 5, 1, 0, 1), ("bf16_5blocks", 2, 5, 1, 0, 1),
    ("fp32_mrhs8", 1, 9, 8, 0, 1), ("bf16_mrhs8", 2, 9, 8, 0, 1),
    ("fp32_redblack", 1, 9, 1, 1, 1), ("bf16_redblack", 2, 9, 1, 1, 1),
    ("bf16_redblack_mrhs8", 2, 9, 8, 1, 1),
    ("fp32_smoother16", 1, 9, 1, 0, 2), ("bf16_smoother16", 2, 9, 1, 0, 2),
    ("bf16_smoother16_mrhs8", 2, 9, 8, 0, 2))


def run_forms(args, gb, torch, ev, stream, dev, w, dims, blocks, nvecs, mass, gauge_dev, b, rank):
    """s/solve to 1e-10 of every form at one mass: setup of both levels
    (timed apart), then the median of 3 solves (1 RHS per call) or 2 calls
    (8 RHS per call: the workload's b and 7 seeded Gaussian ones; s/solve =
    seconds per call / 8), after one warm-up solve."""
    out = {}
    for fname, pc, slots, nr, rbp, ps in FORMS:
        pf = gb.default_params(dims=dims, block=blocks, nvec=nvecs, mass=mass,
                               csw=w["csw"], nlevels=3, prec_fine=1, prec_coarse=pc,
                               setup_sweeps=w["sweeps"], t_antiperiodic=w["antiperiodic"],
                               seed=w["seed"] + 1000 * rank, link_slots=slots,
                               red_black=rbp, prec_smoother=ps)
        mf = gb.Multigrid(pf, gauge_dev)
        t0, t1 = ev(), ev()
        t0.record(stream)
        gb.mg_setup_nullvecs(mf.ctx, 0, None)
        gb.mg_build_coarse(mf.ctx, 0)
        gb.mg_setup_nullvecs(mf.ctx, 1, None)
        gb.mg_build_coarse(mf.ctx, 1)
        t1.record(stream)
        if nr == 1:
            xs = torch.zeros_like(b)
            gb.mg_gcr_solve(mf.ctx, xs, b, 1e-10, 500)  # warm-up
            sts = [gb.mg_gcr_solve(mf.ctx, xs, b, 1e-10, 500) for _ in range(3)]
            torch.cuda.synchronize()
            out[fname] = {
                "s_per_solve_median": statistics.median(st["seconds"] for st in sts),
                "outer_iters": [st["iters"] for st in sts],
                "level_iters": sts[-1]["level_iters"],
                "true_residual": max(st["true_residual"] for st in sts),
                "setup_ms": t0.elapsed_time(t1)}
        else:
            g = torch.Generator(device=dev).manual_seed(w["seed"] + 77)
            bm = torch.randn((nr,) + tuple(b.shape), dtype=torch.complex128, device=dev,
                             generator=g)
            bm[0].copy_(b)
            xm = torch.zeros_like(bm)
            gb.mg_gcr_solve_multi(mf.ctx, xm, bm, nr, 1e-10, 500)  # warm-up
            calls = [gb.mg_gcr_solve_multi(mf.ctx, xm, bm, nr, 1e-10, 500) for _ in range(2)]
            torch.cuda.synchronize()
            out[fname] = {
                "s_per_solve_median": statistics.median(c[0]["seconds"] for c in calls) / nr,
                "nrhs": nr,
                "s_per_call_median": statistics.median(c[0]["seconds"] for c in calls),
                "outer_iters": [[st["iters"] for st in c] for c in calls],
                "true_residual": max(st["true_residual"] for c in calls for st in c),
                "setup_ms": t0.elapsed_time(t1)}
            del bm, xm
        mf.close()
    base = out["fp32"]["s_per_solve_median"]
    for v in out.values():
        v["speedup_vs_fp32"] = base / v["s_per_solve_median"]
    return out


# ---------------------------------------------------------------- GPU leg
def gpu_main(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = syn.WORKLOADS[WORKLOAD]
    dims, blocks, nvecs = w["dims"], w["block"], w["nvec"]
    if args.fine:  # smaller fine lattice of the same shape family (profiling runs)
        dims = tuple(int(v) for v in args.fine.split(","))
    form = args.form
    prec_coarse = {"fp32": 1, "bf16": 2, "fp16": 3, "int16": 4}[form]
    t_gen = time.perf_counter()
    U = syn.gauge_field(dims, w["eps"], w["seed"])
    vol = syn.volume(dims)
    b_host = syn.gaussian_field((vol, 12), w["seed"], stream=99)
    t_gen = time.perf_counter() - t_gen

    import paper_1612_07873_gb300 as gb
    p = gb.default_params(dims=dims, block=blocks, nvec=nvecs, mass=w["mass"], csw=w["csw"],
                          nlevels=3, prec_fine=1, prec_coarse=prec_coarse,
                          setup_sweeps=w["sweeps"], t_antiperiodic=w["antiperiodic"],
                          seed=w["seed"] + 1000 * rank)
    gauge_dev = torch.from_numpy(U).to(dev)
    mg = gb.Multigrid(p, gauge_dev)
    del U
    ctx = mg.ctx
    b = torch.from_numpy(b_host).to(dev)
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()
    l1 = mg.levels[1]
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(record):
        es = [ev() for _ in range(6)]
        es[0].record(stream)
        gb.mg_setup_nullvecs(ctx, 0, None)
        es[1].record(stream)
        gb.mg_build_coarse(ctx, 0)
        es[2].record(stream)
        gb.mg_setup_nullvecs(ctx, 1, None)
        es[3].record(stream)
        gb.mg_build_coarse(ctx, 1)
        es[4].record(stream)
        st = gb.mg_gcr_solve(ctx, x, b, 1e-10, 500)
        es[5].record(stream)
        return es, st

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    gb.mg_profile_reset(ctx)
    gb.mg_profile_enable(ctx, True)
    clocks = ClockSampler(local, args.clocks_csv.replace("{rank}", str(rank)))
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = gb.mg_launch_count(ctx)
    if args.profile_range:  # only the timed steps are seen by a profiler started off
        torch.cuda.cudart().cudaProfilerStart()
    t_start, t_stop = ev(), ev()
    t_start.record(stream)
    phases, stats = [], []
    for _ in range(args.steps):
        es, st = step(True)
        phases.append(es)
        stats.append(st)
    t_stop.record(stream)
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.cudart().cudaProfilerStop()
    if world > 1:
        dist.barrier()
    launches = gb.mg_launch_count(ctx) - launches0
    clk = clocks.stop()
    gb.mg_profile_enable(ctx, False)
    ms_total = t_start.elapsed_time(t_stop)
    ph = np.array([[es[i].elapsed_time(es[i + 1]) for i in range(5)] for es in phases])
    kern = {k: gb.mg_profile_query(ctx, k, -1) for k in
            ("coarse_apply", "coarse_apply_multi", "wilson_clover", "galerkin", "block_orth",
             "restrict", "prolong")}
    ca = gb.mg_profile_query(ctx, "coarse_apply", 1)
    ca_ms = ca["ms"]
    ca_bytes = ca["bytes"]

    # whole-job aggregation over ranks: bytes summed, time = max over ranks
    if world > 1:
        ms_total, ca_ms, ca_bytes = aggregate_ranks(ms_total, ca_ms, ca_bytes, dev)
    gbs = ca_bytes / (ca_ms * 1e-3) / 1e9 if ca_ms > 0 else 0.0
    per_launch_bytes = ca["bytes"] / max(ca["launches"], 1)
    per_launch_ms = ca["ms"] / max(ca["launches"], 1)

    # e2e: the level-1 coarse apply through the C ABI with host buffers.
    # Every step copies its input from pinned host memory, applies the
    # operator and copies its result back; with two device buffers and the
    # copies on streams of their own, step k+1's input copy and step k-1's
    # result copy run while step k's apply does.
    n1 = l1["ndof"]
    xh = torch.randn((l1["volume"], n1), dtype=torch.complex64).pin_memory()
    yh = [torch.empty_like(xh).pin_memory() for _ in range(2)]
    xd = [torch.empty_like(xh, device=dev) for _ in range(2)]
    yd = [torch.empty_like(xd[0]) for _ in range(2)]
    s_in, s_op, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    in_done = [ev(), ev()]
    op_done = [ev(), ev()]
    out_done = [ev(), ev()]

    def e2e_steps(count):
        for k in range(count):
            b = k % 2
            if k >= 2:  # step k-2's apply has read xd[b], its result copy yd[b]
                s_in.wait_event(op_done[b])
                s_op.wait_event(out_done[b])
            with torch.cuda.stream(s_in):
                xd[b].copy_(xh, non_blocking=True)
            in_done[b].record(s_in)
            s_op.wait_event(in_done[b])
            gb.mg_coarse_apply(ctx, 1, yd[b], xd[b], stream=s_op)
            op_done[b].record(s_op)
            s_out.wait_event(op_done[b])
            with torch.cuda.stream(s_out):
                yh[b].copy_(yd[b], non_blocking=True)
            out_done[b].record(s_out)

    e2e_steps(4)
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    reps = 20
    e0.record(s_in)
    e2e_steps(reps)
    e1.record(s_out)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / reps
    e2e = {"value": per_launch_bytes / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": xh.numel() * xh.element_size(),
           "d2h_bytes_per_step": yh[0].numel() * yh[0].element_size(),
           "ms_per_apply": e2e_ms,
           "overlap": "two device buffers; step k+1's input copy and step k-1's result "
                      "copy on their own streams during step k's apply"}

    # the tuned forms of the same problem: same gauge field, seeds and solver;
    # setup untimed, s/solve over several solves; at the workload's mass and
    # at the near-critical mass of these fields
    forms = {}
    if args.forms:
        mg.close()
        for fmass in [float(v) for v in args.forms_mass.split(",") if v.strip()]:
            forms[f"m={fmass:+.2f}"] = run_forms(args, gb, torch, ev, stream, dev, w, dims, blocks,
                                                 nvecs, fmass, gauge_dev, b, rank)
    learned_setup = run_learned(args, gb, torch, dev) if args.learned else None
    precision = run_precision(args, gb, torch, dev) if args.precision else None
    peak, peak_kind = peaks()
    fma = {"fp32_tflops": gb.mg_fma_peak(gb.F32), "fp64_tflops": gb.mg_fma_peak(gb.F64),
           "how": "mg_fma_peak: independent FMA chains on every SM, CUDA events"}
    solve_s = [s["seconds"] for s in stats]
    line = {
        "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if form == "fp32" else form,
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "fine": list(dims), "levels": 3,
                   "blocks": [list(b_) for b_ in blocks], "nvec": nvecs, "form": form,
                   "coarse_apply_lattice": list(l1["dims"]), "coarse_apply_ndof": n1,
                   "l2": "inputs larger than L2 (level-1 links 1.36 GB)",
                   "parallelism": "replicas" if world > 1 else "single-gpu"},
        "roofline": {"bound": "hbm", "achieved": per_launch_bytes / (per_launch_ms * 1e-3) / 1e9,
                     "peak": peak, "unit": "GB/s",
                     "frac": per_launch_bytes / (per_launch_ms * 1e-3) / 1e9 / peak,
                     "traffic": coarse_traffic(form), "kernel": "k_coarse_stream (level 1, n=48)",
                     "peak_kind": peak_kind},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "solve": {"s_per_solve_median": statistics.median(solve_s),
                  "outer_iters": [s["iters"] for s in stats],
                  "level_iters": stats[-1]["level_iters"],
                  "true_residual": max(s["true_residual"] for s in stats),
                  "forms": forms},
        "learned_setup": learned_setup,
        "precision": precision,
        "measured_fma_peaks": fma,
        "phases_ms_median": dict(zip(["setup_l0", "build_l1", "setup_l1", "build_l2", "solve"],
                                     [float(v) for v in np.median(ph, axis=0)])),
        "kernels": {k: {"launches": v["launches"], "ms": v["ms"],
                        "gbs": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else 0.0}
                    for k, v in kern.items()},
        "input_gen_s": t_gen,
    }
    if rank == 0 and world == 1:
        try:
            line["cpu_baseline"] = oracle_coarse_apply_sample()
            if precision is not None:
                o = precision["oracle"]
                line["cpu_baseline"]["oracle_small_workload"] = {
                    "workload": "c1_8^4_2lvl_fp64", "s_per_build": o["s_per_build"],
                    "s_per_solve": o["s_per_solve"], "outer_iters": o["outer_iters"],
                    "cores": o["cores"]}
        except Exception as e:  # the baseline must not sink the GPU line
            line["cpu_baseline"] = {"error": str(e)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if mg.ctx is not None:
        mg.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def coarse_apply_main(args):
    """Only the level-1 coarse apply (8^3x16 lattice, n = 48, or the coarse
    lattice of --fine with 2^4 aggregates) with random links: `steps` timed
    applies, each on the same 1.36 GB (FP32) link set."""
    import torch

    import paper_1612_07873_gb300 as gb
    prec = {"fp32": 1, "bf16": 2, "fp16": 3, "int16": 4}[args.form]
    fine = tuple(int(v) for v in args.fine.split(",")) if args.fine else (16, 16, 16, 32)
    U = syn.gauge_field(fine, 0.0, 1)
    p = gb.default_params(dims=fine, block=[(2, 2, 2, 2)], nvec=[args.nvec], nlevels=2,
                          prec_fine=1, prec_coarse=prec, link_slots=args.slots)
    mg = gb.Multigrid(p, torch.from_numpy(U).cuda())
    l1 = mg.levels[1]
    vol, n = l1["volume"], l1["ndof"]
    g = torch.Generator(device="cuda").manual_seed(3)
    links = torch.randn((vol, 9, n, n), dtype=torch.complex128, device="cuda", generator=g)
    gb.mg_set_coarse_links(mg.ctx, 1, links)
    del links
    torch.cuda.empty_cache()  # the FP64 link copy is not needed on the device
    nrhs = args.nrhs
    if args.launch_choice >= 0 and nrhs > 1:  # pin the autotuner's launch shape
        gb.mg_tune_set(f"mma2/{args.form}/n{n}/r{nrhs}/v{vol}/b1", args.launch_choice)
    shape = (vol, n) if nrhs == 1 else (vol, n, nrhs)
    x = torch.randn(shape, dtype=torch.complex64, device="cuda", generator=g)
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        gb.mg_coarse_apply(mg.ctx, 1, y, x, nrhs=nrhs)
    torch.cuda.synchronize()
    gb.mg_profile_reset(mg.ctx)
    gb.mg_profile_enable(mg.ctx, True)
    for _ in range(args.steps):
        gb.mg_coarse_apply(mg.ctx, 1, y, x, nrhs=nrhs)
    gb.mg_device_status(mg.ctx)
    q = gb.mg_profile_query(mg.ctx, "coarse_apply" if nrhs == 1 else "coarse_apply_multi", 1)
    peak, kind = peaks()
    gbs = q["bytes"] / (q["ms"] * 1e-3) / 1e9
    tflops = q["flops"] / (q["ms"] * 1e-3) / 1e12
    choice = gb.mg_tune_get(f"mma2/{args.form}/n{n}/r{nrhs}/v{vol}/b1") if nrhs > 1 else None
    print(json.dumps({"mode": "coarse-apply", "form": args.form, "slots": args.slots,
                      "launch_choice": choice,
                      "lattice": list(l1["dims"]),
                      "ndof": n, "nrhs": nrhs, "launches": q["launches"],
                      "us_per_apply": 1e3 * q["ms"] / q["launches"],
                      "gbs": gbs, "frac": gbs / peak, "peak": peak, "peak_kind": kind,
                      "tflops": tflops, "bytes_per_apply": q["bytes"] / q["launches"]}), flush=True)
    mg.close()
    return 0


def mma_sweep_main(args):
    """Config-4 sweep of the multi-RHS coarse apply (BF16 links, FP32
    accumulation) on the two coarse lattices of the production workload,
    8^3x16 (n = 48) and 4^3x8 (n = 64), with Gaussian links: nrhs = 1 (the
    single-RHS stream) and 8, 16, 32, 64 (tensor cores, autotuned launch
    shape).  Every timed apply follows a write of 512 MB (L2 flushed), timed
    alone by the library's CUDA events; the same applies back to back give
    the L2-warm figure.  GB/s of algorithmic bytes (links + x read + y
    written) and the fraction of the measured HBM copy peak."""
    import torch

    import paper_1612_07873_gb300 as gb
    peak, kind = peaks()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    rows = []
    for cdims, nv in (((8, 8, 8, 16), 24), ((4, 4, 4, 8), 32)):
        fine = tuple(2 * c for c in cdims)
        U = torch.from_numpy(syn.gauge_field(fine, 0.0, 1)).cuda()
        p = gb.default_params(dims=fine, block=[(2, 2, 2, 2)], nvec=[nv], nlevels=2,
                              prec_fine=1, prec_coarse=2)
        mg = gb.Multigrid(p, U)
        l1 = mg.levels[1]
        vol, n = l1["volume"], l1["ndof"]
        g = torch.Generator(device="cuda").manual_seed(3)
        links = torch.randn((vol, 9, n, n), dtype=torch.complex128, device="cuda", generator=g)
        gb.mg_set_coarse_links(mg.ctx, 1, links)
        del links
        for nrhs in (1, 8, 16, 32, 64):
            shape = (vol, n) if nrhs == 1 else (vol, n, nrhs)
            x = torch.randn(shape, dtype=torch.complex64, device="cuda", generator=g)
            y = torch.empty_like(x)
            for _ in range(max(args.warmup, 2)):
                gb.mg_coarse_apply(mg.ctx, 1, y, x, nrhs=nrhs)
            name = "coarse_apply" if nrhs == 1 else "coarse_apply_multi"
            out = {"lattice": list(cdims), "ndof": n, "nrhs": nrhs}
            for mode in ("flushed", "warm"):
                torch.cuda.synchronize()
                gb.mg_profile_reset(mg.ctx)
                gb.mg_profile_enable(mg.ctx, True)
                for _ in range(args.steps):
                    if mode == "flushed":
                        flush.fill_(1)
                    gb.mg_coarse_apply(mg.ctx, 1, y, x, nrhs=nrhs)
                gb.mg_device_status(mg.ctx)
                q = gb.mg_profile_query(mg.ctx, name, 1)
                gb.mg_profile_enable(mg.ctx, False)
                us = 1e3 * q["ms"] / q["launches"]
                gbs = q["bytes"] / q["launches"] / (us * 1e-6) / 1e9
                out[mode] = {"us": us, "gbs": gbs, "frac": gbs / peak,
                             "tflops": q["flops"] / q["launches"] / (us * 1e-6) / 1e12}
                out["bytes"] = q["bytes"] / q["launches"]
            if nrhs > 1:
                key = f"mma2/bf16/n{n}/r{nrhs}/v{vol}/b1"
                out["launch_choice"] = gb.mg_tune_get(key)
                out["tuner_candidates_us"] = {str(c): 1e3 * t for c, t in gb.mg_tune_report(key)}
            rows.append(out)
            del x, y
        mg.close()
    print(json.dumps({"mode": "mma-sweep", "peak_gbs": peak, "peak_kind": kind,
                      "choice_code": "100000 PC + 10000 IL + 1000 cps + 100 KH + 10 SL + SA: "
                                     "pipelined kernel (PC 1: operand pre-converted by a "
                                     "streaming pass; IL 1: interleaved rows, register epilogue; 0: "
                                     "split rows, staged epilogue), cps CTAs per SM, KH half "
                                     "slots per stage, SL/SA load/operand ring depths; "
                                     "q <= 8: register-staged kernel, q CTAs per SM",
                      "rows": rows}), flush=True)
    return 0


def wilson_policies_main(args):
    """Every launch policy of the FP32 fine operator, pinned in turn through
    mg_tune_set, on the 32^3x64 workload lattice for 1, 8 and 24 vectors
    (mg_wilson_clover_apply_multi); microseconds per vector by CUDA events.
    Policies 10 and 11 read 8-real links; the line carries the 8-real
    form's reconstruction error on this field."""
    import torch

    import paper_1612_07873_gb300 as gb
    w = syn.WORKLOADS[WORKLOAD]
    dims = w["dims"]
    vol = syn.volume(dims)
    U = torch.from_numpy(syn.gauge_field(dims, w["eps"], w["seed"])).cuda()
    p = gb.default_params(dims=dims, block=w["block"], nvec=w["nvec"], mass=w["mass"],
                          csw=w["csw"], nlevels=3, prec_fine=1, prec_coarse=1)
    mg = gb.Multigrid(p, U)
    comp = gb.mg_gauge_compression(mg.ctx)
    rows = []
    for nvec in (1, 8, 24):
        g = torch.Generator(device="cuda").manual_seed(nvec)
        x = torch.randn((nvec, vol, 12), dtype=torch.complex64, device="cuda", generator=g)
        y = torch.empty_like(x)
        key = f"wilson/v{vol}/n{nvec}/c1"
        gb.mg_tune_set(key, -1)
        gb.mg_wilson_clover_apply_multi(mg.ctx, y, x, nvec)
        torch.cuda.synchronize()
        pick = gb.mg_tune_get(key)
        for pol in range(14):
            if (6 <= pol < 10 and nvec == 1) or (pol == 6 and nvec % 2) or (pol == 7 and nvec % 4) \
                    or (pol in (8, 9) and nvec < 4) or (pol in (10, 11) and not comp["eight_real"]) \
                    or (pol >= 12 and not comp["two_row"]):
                continue
            gb.mg_tune_set(key, pol)
            for _ in range(args.warmup):
                gb.mg_wilson_clover_apply_multi(mg.ctx, y, x, nvec)
            torch.cuda.synchronize()
            gb.mg_profile_reset(mg.ctx)
            gb.mg_profile_enable(mg.ctx, True)
            for _ in range(args.steps):
                gb.mg_wilson_clover_apply_multi(mg.ctx, y, x, nvec)
            q = gb.mg_profile_query(mg.ctx, "wilson_clover", 0)
            gb.mg_profile_enable(mg.ctx, False)
            us = 1e3 * q["ms"] / q["launches"]
            rows.append({"nvec": nvec, "policy": pol, "us_per_vector": us / nvec,
                         "tuner_pick": pol == pick,
                         "gbs_algorithmic": q["bytes"] / q["launches"] / (us * 1e-6) / 1e9})
        gb.mg_tune_set(key, -1)
    mg.close()
    print(json.dumps({"mode": "wilson-policies", "lattice": list(dims), "compression": comp,
                      "rows": rows}), flush=True)
    return 0


def solve_breakdown_main(args):
    """Per-kernel device time of one MG-GCR solve on the 32^3x64 workload
    (setup untimed), for the plain FP32 form and the 16-bit fine smoother
    form: every kernel launch of the solve recorded by the CUDA activity
    tracer (torch.profiler, not serialised, warm caches), summed per kernel.
    Prints one JSON line per form: wall time of the solve, summed kernel
    time, the span from first to last launch, and the kernels by share."""
    import torch
    from torch.profiler import ProfilerActivity, profile

    import paper_1612_07873_gb300 as gb
    w = syn.WORKLOADS[WORKLOAD]
    dims = tuple(w["dims"])
    vol = syn.volume(dims)
    U = torch.from_numpy(syn.gauge_field(dims, w["eps"], w["seed"])).cuda()
    b = torch.from_numpy(syn.gaussian_field((vol, 12), w["seed"], stream=99)).cuda()
    with profile(activities=[ProfilerActivity.CUDA]):  # the tracer's first session
        torch.zeros(1, device="cuda").add_(1)           # can come back empty
        torch.cuda.synchronize()
    for name, pc, ps in (("fp32", 1, 1), ("bf16_smoother16", 2, 2)):
        p = gb.default_params(dims=dims, block=w["block"], nvec=w["nvec"], mass=w["mass"],
                              csw=w["csw"], nlevels=3, prec_fine=1, prec_coarse=pc,
                              setup_sweeps=w["sweeps"], t_antiperiodic=w["antiperiodic"],
                              seed=w["seed"], prec_smoother=ps)
        mg = gb.Multigrid(p, U)
        for lv in range(2):
            gb.mg_setup_nullvecs(mg.ctx, lv, None)
            gb.mg_build_coarse(mg.ctx, lv)
        x = torch.zeros_like(b)
        for _ in range(max(args.warmup, 1)):
            gb.mg_gcr_solve(mg.ctx, x, b, 1e-10, 500)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = gb.mg_gcr_solve(mg.ctx, x, b, 1e-10, 500)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            gb.mg_gcr_solve(mg.ctx, x, b, 1e-10, 500)
            torch.cuda.synchronize()
        agg, busy, t_lo, t_hi = {}, 0.0, None, None
        for e in prof.events():
            if e.device_type != torch.autograd.DeviceType.CUDA:
                continue
            d = getattr(e, "device_time", None)
            d = e.cuda_time if d is None else d
            key = e.name.replace("(anonymous namespace)::", "")
            key = key.split("(")[0].replace("void ", "")
            a = agg.setdefault(key, [0, 0.0])
            a[0] += 1
            a[1] += d
            busy += d
            t_lo = e.time_range.start if t_lo is None else min(t_lo, e.time_range.start)
            t_hi = e.time_range.end if t_hi is None else max(t_hi, e.time_range.end)
        rows = [{"kernel": k, "launches": n, "ms": t / 1e3, "us_per_launch": t / n,
                 "share": t / busy if busy else 0.0}
                for k, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1])]
        print(json.dumps({"mode": "solve-breakdown", "form": name, "lattice": list(dims),
                          "iters": st["iters"], "wall_ms": wall * 1e3,
                          "kernel_ms": busy / 1e3,
                          "span_ms": (t_hi - t_lo) / 1e3 if rows else 0.0,
                          "kernels": rows}), flush=True)
        mg.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbmg", choices=["gbmg", "reference"])
    ap.add_argument("--form", default="fp32", choices=["fp32", "bf16", "fp16", "int16"])
    ap.add_argument("--mode", default="pipeline",
                    choices=["pipeline", "coarse-apply", "wilson-policies", "solve-breakdown",
                             "learned", "mma-sweep", "precision"])
    ap.add_argument("--fine", default="", help="override the fine extents, e.g. 16,16,16,32")
    ap.add_argument("--nrhs", type=int, default=1, help="right-hand sides (coarse-apply mode)")
    ap.add_argument("--launch-choice", type=int, default=-1,
                    help="pin the tensor-core apply's launch shape (coarse-apply mode, "
                         "nrhs > 1; see mg_tune_report)")
    ap.add_argument("--nvec", type=int, default=24,
                    help="null vectors, n = 2 nvec coarse dofs (coarse-apply mode)")
    ap.add_argument("--slots", type=int, default=9, choices=[5, 9],
                    help="coarse link blocks stored (coarse-apply mode)")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off)")
    ap.add_argument("--no-learned", dest="learned", action="store_false",
                    help="skip training / evaluating the learned setup")
    ap.add_argument("--learned-ntrain", type=int, default=200)
    ap.add_argument("--learned-epochs", type=int, default=4)
    ap.add_argument("--no-forms", dest="forms", action="store_false",
                    help="skip the tuned forms' s/solve")
    ap.add_argument("--forms-mass", default="-0.40,-0.90",
                    help="masses at which the forms table is measured")
    ap.add_argument("--no-precision", dest="precision", action="store_false",
                    help="skip the precision study of the small workload")
    ap.add_argument("--clocks-csv", default="",
                    help="where the nvidia-smi clock samples of the timed region go "
                         "('{rank}' is replaced; default: the temp directory)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_main(args)
    if args.mode == "coarse-apply":
        return coarse_apply_main(args)
    if args.mode == "wilson-policies":
        return wilson_policies_main(args)
    if args.mode == "solve-breakdown":
        return solve_breakdown_main(args)
    if args.mode == "learned":
        return learned_main(args)
    if args.mode == "mma-sweep":
        return mma_sweep_main(args)
    if args.mode == "precision":
        return precision_main(args)
    return gpu_main(args)


if __name__ == "__main__":
    sys.exit(main())
