"""Benchmark: forward + adjoint lattice updates per second (MLUPS) of the LKS / ALKS
gradient on one GB300, plus roofline, end-to-end and CPU-oracle figures.

One step = one full gradient of the workload (LKS forward march, ALKS adjoint march,
sensitivity).  Default workload: the 192^3 D3Q19 duct, Re = 50, 1000 forward + 1000
adjoint steps, FP32, objective dissipation + static pressure drop (the largest
single-GPU configuration of the paper-derived set, 7.08 M nodes, working set far
larger than L2).  The same line carries, under "also", the 512 x 256 channel
(config2, L2-resident) and the 8192^2 channel (67 M nodes) measured the same way,
and on one GPU config3 (plain FP32 against K = 100 BF16 checkpoints) and config5
(the 64-design batch against the plain form design by design) in brief.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload config4|config2|roofline8192|config1|config3|config5]

config3 runs the checkpoint study (plain FP32 trajectory against checkpoints every
K steps with FP32 / BF16 / FP16 snapshots); config5 runs the batched form (64
designs of unequal size, one persistent launch per step, one CUDA graph per
gradient) against the plain FP32 form design by design.

Under torchrun every rank runs an independent replica (designs are independent;
no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import inputs  # noqa: E402

# Algorithmic bytes per node of one launch (FP32 fields, read once + written once;
# gradients recomputed from the halo; gamma read once).
BYTES_FWD = 4 * (3 + 3 + 1)            # drho,u,v in; drho,u,v out; gamma
BYTES_ADJ_STEADY = 4 * (6 + 6 + 2 + 1)  # 6 adjoint fields in + out; u,v; gamma
# Unsteady checkpointed gradient, per node and level: forward (28), recomputed
# forward storing the level's u, v (28 + 8), adjoint reading both levels' u, v with
# the FP32 sensitivity read-modify-write (4 * (6 + 6 + 4 + 1) + 8 = 76).
BYTES_CKPT_LEVEL = BYTES_FWD + (BYTES_FWD + 8) + (4 * (6 + 6 + 4 + 1) + 8)
# D3Q19: drho,u,v,w in + out and gamma; steady adjoint: 10 fields in + out, u,v,w, gamma.
BYTES_FWD_3D = 4 * (4 + 4 + 1)
BYTES_ADJ_3D = 4 * (10 + 10 + 3 + 1)

METRIC = "forward+adjoint MLUPS & % HBM peak; s per gradient vs plain FP32 at 1e-3 rel"

# DRAM bytes (read + write) per node of one launch of the step kernels, from ncu
# captures of the kernels as they stand; None where no capture of the current kernel
# exists.  Multiplied by the nodes of a launch they give roofline.traffic.
TRAFFIC_BYTES_PER_NODE = {
    "adj3c_kernel": 747.7e6 / 7077888,   # the 192^3 duct, 4 + 4 steps
    "fwd3p_kernel": 218.5e6 / 7077888,
    "adj_col_kernel<true>": 4.2666e9 / 67108864,  # the 8192^2 channel, 4 + 4 steps
    "fwd_col2_kernel<10>": 425.4e6 / 16777216,  # the 4096^2 channel, 4 + 4 steps
}


def workload(name: str):
    if name == "config2":
        return inputs.config2(), "config2: 512x256 steady channel, Re=100, 20000+20000 steps, FP32"
    if name == "config1":
        return inputs.config1(), "config1: 64x64 steady channel, Re=10, 5000+5000 steps, FP32"
    if name == "config4":
        pb = inputs.config4()
        return pb, (f"config4: 192^3 steady D3Q19 duct, Re=50 (nu=0.191), {pb.n_steps}+{pb.n_adj} steps, "
                    "FP32, objective = dissipation + static pressure drop (unit weights)")
    if name.startswith("roofline"):
        n = int(name[len("roofline"):])
        pb = inputs.roofline2d(n)
        return pb, f"{name}: {n}x{n} steady channel, {pb.n_steps}+{pb.n_adj} steps, FP32"
    raise SystemExit(f"unknown workload {name}")


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """Slowest rank's time: every rank contributes its own timed milliseconds and
    all receive the maximum (the whole job ends when its slowest replica does)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_mlups(world: int, updates_per_replica_step: float, steps: int, max_ms: float) -> float:
    """Whole-job throughput of `world` independent replicas (weak scaling): the
    updates all ranks did, over the slowest rank's time."""
    return world * updates_per_replica_step * steps / (max_ms * 1e-3) / 1e6


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_steps_for(pb, seconds: float) -> int:
    """Forward (and as many adjoint) steps of the FP64 oracle on the full lattice that
    take about `seconds` on the host cores, from a short timed calibration run."""
    from oracle import oracle as O
    O.build()
    g = pb.gamma()
    n = 2
    t0 = time.perf_counter()
    if hasattr(pb, "nz"):
        st, _, _, _ = O.forward3(pb, g, n)
        O.steady_adjoint3(pb, g, st, n)
    else:
        st, _, _, _ = O.forward(pb, g, n)
        O.steady_adjoint(pb, g, st, n)
    per_pair = (time.perf_counter() - t0) / n
    return int(max(2, min(pb.n_steps, seconds / max(per_pair, 1e-9))))


def cpu_baseline(pb, n_fwd: int, n_adj: int):
    """The FP64 oracle on the host cores, on a bounded sample of the workload: the
    full lattice for n_fwd forward + n_adj adjoint steps (steady iteration)."""
    from oracle import oracle as O
    O.build()
    g = pb.gamma()
    t0 = time.perf_counter()
    if hasattr(pb, "nz"):
        st, _, _, _ = O.forward3(pb, g, n_fwd)
        O.steady_adjoint3(pb, g, st, n_adj)
    else:
        st, _, _, _ = O.forward(pb, g, n_fwd)
        O.steady_adjoint(pb, g, st, n_adj)
    dt = time.perf_counter() - t0
    mlups = pb.n_nodes * (n_fwd + n_adj) / dt / 1e6
    return {"value": mlups, "unit": "MLUPS", "cores": O.get_threads(), "kind": "oracle",
            "sample": f"{pb.nx}x{pb.ny}{'x%d' % pb.nz if hasattr(pb, 'nz') else ''} lattice, "
                      f"{n_fwd} forward + {n_adj} adjoint steps (of "
                      f"{pb.n_steps}+{pb.n_adj}), FP64, {dt:.1f} s"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pb, desc = workload(args.workload)
    n_f = n_a = oracle_steps_for(pb, 3.0)  # each timed step: about 3 s of host work
    from oracle import oracle as O
    O.build()
    g = pb.gamma()
    three_d = hasattr(pb, "nz")
    fwd = O.forward3 if three_d else O.forward
    adj = O.steady_adjoint3 if three_d else O.steady_adjoint
    for _ in range(args.warmup):
        st, _, _, _ = fwd(pb, g, 2)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        st, _, _, _ = fwd(pb, g, n_f)
        adj(pb, g, st, n_a)
        times.append(time.perf_counter() - t0)
    dt = sum(times)
    value = pb.n_nodes * (n_f + n_a) * args.steps / dt / 1e6
    cb = {"value": value, "unit": "MLUPS", "cores": O.get_threads(), "kind": "oracle",
          "sample": f"each step: {pb.nx}x{pb.ny}{'x%d' % pb.nz if three_d else ''} lattice, "
                    f"{n_f} forward + {n_a} adjoint steps from rest (FP64)"}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "l2": "n/a (CPU)"},
        "cpu_baseline": cb, "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                                     "d2h_bytes_per_step": 0}}))


def run_checkpoint_study(args):
    """Unsteady thermal config3 (1024x512, 20000 steps): the plain FP32 form (every
    level of u, v, T kept) against recomputation checkpoints every K steps with
    FP32 / BF16 / FP16 snapshots; seconds per gradient, device memory and gradient
    error relative to the plain form.  One JSON line, metric of the checkpointed
    BF16 form with K = 100."""
    import torch
    from paper_2411_03090_gb300 import LKS

    pb = inputs.config3()
    if args.steps_override:
        pb = pb.with_(n_steps=args.steps_override)
    dev = torch.device("cuda", 0)
    gamma = torch.from_numpy(pb.gamma()).to(dev, torch.float32)
    N = pb.n_nodes
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(s, reps):
        s.gradient(gamma)  # warm-up
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
            J, g = s.gradient(gamma)
            e1.record(s.stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        return min(ts), J.item(), g.double()

    reps = max(1, min(args.steps, 2))
    rows = []
    clocks = ClockSampler(0)  # sampled over the whole study
    clocks.start()
    plain = LKS(pb, real="f32", checkpoint_every=0, device=dev)
    t_plain, J_plain, g_plain = timed(plain, reps)
    ws_plain = plain.workspace.numel()
    rows.append({"form": "plain FP32 trajectory", "K": 0, "snapshot": "-", "s_per_gradient": t_plain,
                 "workspace_GB": ws_plain / 1e9, "grad_rel_err_vs_plain": 0.0, "J": J_plain})
    del plain
    torch.cuda.empty_cache()
    norm = torch.linalg.vector_norm(g_plain).item()
    variants = [(K, snap, "f32") for K in (16, 100, 500, 2000) for snap in ("f32", "bf16", "f16")]
    variants += [(0, "-", "bf16"), (2000, "bf16", "bf16"), (500, "bf16", "bf16")]  # 16-bit stored levels
    for K, snap, seg in variants:
        s = LKS(pb, real="f32", checkpoint_every=K, snapshot=snap if K else "f32", segment=seg, device=dev)
        t, J, g = timed(s, reps)
        err = torch.linalg.vector_norm(g - g_plain).item() / norm
        rows.append({"form": "checkpointed" if K else "plain", "K": K, "snapshot": snap, "levels": seg,
                     "s_per_gradient": t, "workspace_GB": s.workspace.numel() / 1e9,
                     "grad_rel_err_vs_plain": err, "J": J})
        del s
        torch.cuda.empty_cache()
    clk = clocks.stop()
    head = [r for r in rows if r["K"] == 100 and r["snapshot"] == "bf16" and r.get("levels", "f32") == "f32"][0]

    # Gradient error against the FP64 oracle on a truncated horizon (the oracle keeps
    # every level in host memory): the first `oracle_levels` steps of the same problem.
    vs_oracle = []
    if args.oracle_levels > 0:
        from oracle import oracle as O
        pt = pb.with_(n_steps=args.oracle_levels, n_adj=args.oracle_levels)
        g64 = pt.gamma()
        t0 = time.perf_counter()
        ref = O.unsteady_gradient(pt, g64)
        t_or = time.perf_counter() - t0
        rnorm = float(np.linalg.norm(ref["dJdgamma"]))
        for K, snap, seg in ((0, "-", "f32"), (20, "f32", "f32"), (20, "bf16", "f32"), (20, "f16", "f32"),
                             (100, "bf16", "f32"), (100, "f16", "f32"), (0, "-", "bf16"), (20, "bf16", "bf16"),
                             (20, "f16", "f16")):
            s = LKS(pt, real="f32", checkpoint_every=K, snapshot=snap if K else "f32", segment=seg, device=dev)
            J, gg = s.gradient(gamma)
            err = float(np.linalg.norm(gg.double().cpu().numpy() - ref["dJdgamma"])) / rnorm
            vs_oracle.append({"K": K, "snapshot": snap, "levels": seg, "grad_rel_err_vs_oracle": err,
                              "J_rel_err_vs_oracle": abs(J.item() - ref["J"]) / abs(ref["J"])})
            del s
            torch.cuda.empty_cache()
        vs_oracle.append({"oracle_levels": args.oracle_levels, "oracle_seconds": t_or})
    print(json.dumps({
        "metric": METRIC, "value": N * 2 * pb.n_steps / head["s_per_gradient"] / 1e6, "unit": "MLUPS",
        "n_gpus": 1, "steps": reps, "warmup": 1, "ms_per_step": head["s_per_gradient"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"config3: 1024x512 unsteady thermal channel, Re=200, Pr=0.71, pulsed inlet, "
                               f"{pb.n_steps} steps; headline = checkpoints every 100 steps, BF16 snapshots",
                   "updates_counted": "forward + adjoint levels (recomputation not counted)",
                   "l2": "flushed before each timed gradient"},
        "checkpoint_study": rows,
        "vs_oracle_truncated_horizon": vs_oracle,
        "speedup_vs_plain": t_plain / head["s_per_gradient"],
        "memory_ratio_vs_plain": head["workspace_GB"] / (ws_plain / 1e9),
        "clocks": clk}))


def run_fd_study(args):
    """Config2's gradient check: the FP64 instance on the 512x256 channel (Re = 100),
    both marches run to a small relative step change (tolerance marches), then
    central differences of J with step 1e-4 (Eq. sensfdm) on 32 design nodes drawn
    with seed 22 from the nodes at least 3 from an edge and 5 from the inlet and
    outlet strips, each perturbed march warm-started from the converged state.
    Reports the cosine between the ALKS gradient and the differences and the
    per-node ratios (Sec. 2.6 made numeric)."""
    import torch
    from paper_2411_03090_gb300 import LKS

    pb = inputs.config2().with_(n_steps=2000, n_adj=2000)
    dev = torch.device("cuda", 0)
    g = pb.gamma()
    gt = torch.from_numpy(g).to(dev)
    tol, cap = args.fd_tol, args.fd_max_steps
    t0 = time.perf_counter()
    from paper_2411_03090_gb300 import LKSError
    s = LKS(pb, real="f64", device=dev, tol=tol, max_steps=cap, warm_start=True)
    converged = {}
    for name, call in (("forward", lambda: s.lks_forward(gt)), ("adjoint", s.alks_adjoint)):
        try:  # a march that stops at the step limit leaves its last state in place
            call()
            converged[name] = True
        except LKSError as e:
            if e.status != 5:
                raise
            converged[name] = False
    grad = s.lks_sensitivity()
    q = s.query()
    base_steps, adj_steps, fchg, achg = q.forward_steps, q.adjoint_steps, q.fwd_change, q.adj_change
    grad = grad.cpu().numpy()
    base = [x.clone() for x in s.get_state()]
    # Perturbed marches: a fixed number of steps from the converged base state, the
    # same for +eps and -eps, so that whatever drift remains in the base state
    # cancels in the central difference.
    M = args.fd_steps
    s = LKS(pb.with_(n_steps=M), real="f64", device=dev, warm_start=True)
    rng = np.random.default_rng(22)
    cand = [(j, i) for j in range(3, pb.ny - 3) for i in range(pb.strip + 5, pb.nx - pb.strip - 5)]
    nodes = [cand[k] for k in rng.choice(len(cand), 32, replace=False)]
    eps = 1e-4
    rows, steps = [], []
    for (j, i) in nodes:
        Js = []
        for sg in (1.0, -1.0):
            gp = g.copy()
            gp[j, i] += sg * eps
            s.set_state(gt, base[0], base[1], base[2])
            Js.append(s.lks_forward(torch.from_numpy(gp).to(dev)).item())
            steps.append(M)
        fd = (Js[0] - Js[1]) / (2 * eps)
        rows.append({"node": [int(i), int(j)], "alks": float(grad[j, i]), "fd": fd,
                     "ratio": float(grad[j, i] / fd) if fd != 0 else None})
    a = np.array([r["alks"] for r in rows])
    b = np.array([r["fd"] for r in rows])
    ratios = np.array([r["ratio"] for r in rows if r["ratio"] is not None])
    print(json.dumps({
        "study": "config2 gradient vs central differences (FP64 GPU instance)",
        "lattice": f"{pb.nx}x{pb.ny}", "eps": eps, "tol": tol, "forward_steps_base": int(base_steps),
        "forward_change_base": fchg, "adjoint_steps": int(adj_steps), "adjoint_change": achg,
        "converged": converged,
        "perturbed_steps": M,
        "cosine": float(a @ b / np.linalg.norm(a) / np.linalg.norm(b)),
        "rel_l2_alks_vs_fd": float(np.linalg.norm(a - b) / np.linalg.norm(b)),
        "ratio_median": float(np.median(ratios)), "ratio_p10": float(np.percentile(ratios, 10)),
        "ratio_p90": float(np.percentile(ratios, 90)), "seconds": time.perf_counter() - t0, "nodes": rows}))


def run_batch_study(args):
    """Batched config5: 64 unsteady designs (128x64 .. 512x256, 5000 steps) in one
    persistent launch per step, the gradient of all of them one CUDA graph launch,
    BF16 checkpoints at the memory-optimal spacing, autotuned tile shape.  Compared
    with the plain FP32 form (full u, v trajectory, per-step launches) run design by
    design on the same GPU: seconds per batch of gradients, device memory and the
    gradient error between the two."""
    import torch
    from paper_2411_03090_gb300 import LKS, LKSBatch

    pbs = inputs.config5()
    if args.steps_override:
        pbs = [p.with_(n_steps=args.steps_override, n_adj=args.steps_override) for p in pbs]
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n_steps = pbs[0].n_steps
    N = sum(p.n_nodes for p in pbs)
    gam_np = [p.gamma().astype(np.float32) for p in pbs]
    gam = [torch.from_numpy(g).to(dev) for g in gam_np]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    b = LKSBatch(pbs, snapshot="bf16", device=dev, tile_config=args.tile_config, fwd_column=args.fwd_column,
                 adj_column=args.adj_column)
    create_s = time.perf_counter() - t0
    st = b.query()
    for _ in range(max(args.warmup, 3)):
        b.gradient(gam)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        J, G = b.gradient(gam)
        e1.record(b.stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
    clk = clocks.stop()
    st = b.query()
    if st.device_status != 0:
        raise SystemExit(f"device status {st.device_status}")
    t_batch = sum(times) / len(times)
    Jb = J.cpu().numpy().copy()
    Gb = [g.double().cpu().numpy() for g in G]

    # end to end: gamma from pinned host buffers, J and gradients back to pinned host
    e2e_val = None
    if not args.no_e2e:
        gh = [torch.from_numpy(g).pin_memory() for g in gam_np]
        oh = [torch.empty(p.ny, p.nx, dtype=torch.float32).pin_memory() for p in pbs]
        Jh = torch.empty(len(pbs), dtype=torch.float64).pin_memory()
        dg = [torch.empty(p.ny, p.nx, dtype=torch.float32, device=dev) for p in pbs]
        ts = []
        for _ in range(2):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            with torch.cuda.stream(b.stream):
                for d, h in zip(dg, gh):
                    d.copy_(h, non_blocking=True)
            J2, G2 = b.gradient(dg)
            with torch.cuda.stream(b.stream):
                for o, g in zip(oh, G2):
                    o.copy_(g, non_blocking=True)
                Jh.copy_(J2, non_blocking=True)
            b.stream.synchronize()
            ts.append(time.perf_counter() - t1)
        e2e_val = N * 2 * n_steps / min(ts) / 1e6

    # the plain FP32 form, design by design
    t_plain, errs, peak_ws, sum_ws = 0.0, [], 0, 0
    if not args.no_plain:
        for k, p in enumerate(pbs):
            s = LKS(p, real="f32", checkpoint_every=0, device=dev)
            peak_ws = max(peak_ws, s.workspace.numel())
            sum_ws += s.workspace.numel()
            s.gradient(gam[k])
            torch.cuda.synchronize()
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
            _, gp = s.gradient(gam[k])
            e1.record(s.stream)
            torch.cuda.synchronize()
            t_plain += e0.elapsed_time(e1) * 1e-3
            gp = gp.double().cpu().numpy()
            errs.append(float(np.linalg.norm(Gb[k] - gp) / np.linalg.norm(gp)))
            del s
            torch.cuda.empty_cache()
    hbm, peak_kind = peaks()
    gbs = BYTES_CKPT_LEVEL * N * n_steps / t_batch / 1e9
    value = N * 2 * n_steps / t_batch / 1e6
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_batch * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"config5: {len(pbs)} unsteady designs 128x64..512x256 (seed 5), Re 20-200, "
                               f"{n_steps} steps, BF16 checkpoints, one graph launch per batch of gradients",
                   "nodes": N, "updates_counted": "forward + adjoint levels (recomputation not counted)",
                   "l2": "flushed before each timed gradient (256 MB write); arena > L2",
                   "tile_shape": list(__import__("paper_2411_03090_gb300").lks.TILE_SHAPES[st.tile_config]),
                   "autotune_us_per_level": [round(x, 1) for x in st.tune_us],
                   "forward_kernel": "warp-column (60x40 tiles)" if st.fwd_column else "TMA-staged tiles",
                   "autotune_forward_us": {"tma": round(st.tune_fwd_us[st.tile_config], 1),
                                           "column": round(st.tune_col_us, 1)},
                   "adjoint_kernel": "warp-column (28x32 tiles)" if st.adj_column else "TMA-staged tiles",
                   "autotune_adjoint_us": {"tma": round(st.tune_us[st.tile_config] - 2 * st.tune_fwd_us[st.tile_config], 1),
                                           "column": round(st.tune_acol_us, 1)},
                   "checkpoint_every": st.checkpoint_every, "arena": [st.arena_w, st.arena_h],
                   "tiles": st.ntiles, "create_s": create_s},
        "roofline": {"bound": "hbm",
                     "kernel": "whole gradient (graph: %s forward, %s adjoint, batched)" % (
                         "fwd_col2_kernel" if st.fwd_column else "fwd_tma_kernel",
                         "adj_col_kernel" if st.adj_column else "adj_tma_kernel"),
                     "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": None,
                     "peak_kind": peak_kind, "algorithmic_bytes_per_node_level": BYTES_CKPT_LEVEL},
        "batch_vs_plain": {"s_per_batch_gradient": t_batch, "plain_fp32_s_design_by_design": t_plain or None,
                           "speedup": (t_plain / t_batch) if t_plain else None,
                           "batch_workspace_GB": st.workspace_bytes / 1e9,
                           "plain_workspace_GB_all_designs": sum_ws / 1e9 or None,
                           "plain_workspace_GB_largest_design": peak_ws / 1e9 or None,
                           "grad_rel_err_vs_plain_max": max(errs) if errs else None,
                           "grad_rel_err_vs_plain_median": float(np.median(errs)) if errs else None},
        "e2e": {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": 4 * N,
                "d2h_bytes_per_step": 4 * N + 8 * len(pbs)},
        "gpu_launches": int(st.kernel_launches),
        "clocks": clk,
    }))


def also_config3(dev, flush):
    """Config3 in brief for the default line: the plain FP32 form against checkpoints
    every 100 steps with BF16 snapshots (the recompute overlapped with the adjoint),
    one warm-up and one timed gradient each, L2 flushed before the timed one."""
    import torch
    from paper_2411_03090_gb300 import LKS

    pb = inputs.config3()
    gamma = torch.from_numpy(pb.gamma()).to(dev, torch.float32)
    rows, g_plain = {}, None
    for name, K, snap in (("plain_fp32", 0, "f32"), ("checkpointed_K100_bf16", 100, "bf16")):
        s = LKS(pb, real="f32", checkpoint_every=K, snapshot=snap, device=dev)
        s.gradient(gamma)
        torch.cuda.synchronize()
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        J, g = s.gradient(gamma)
        e1.record(s.stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        g = g.double()
        rows[name] = {"s_per_gradient": t, "MLUPS": pb.n_nodes * 2 * pb.n_steps / t / 1e6,
                      "workspace_GB": s.workspace.numel() / 1e9, "J": J.item()}
        if g_plain is None:
            g_plain = g
        else:
            rows[name]["grad_rel_err_vs_plain"] = (torch.linalg.vector_norm(g - g_plain)
                                                   / torch.linalg.vector_norm(g_plain)).item()
        del s, g
        torch.cuda.empty_cache()
    return {"workload": f"config3: 1024x512 unsteady thermal channel, {pb.n_steps} + {pb.n_adj} steps", **rows,
            "updates_counted": "forward + adjoint levels (recomputation not counted)"}


def also_config5(dev, flush):
    """Config5 in brief for the default line: the 64-design batch (one graph launch
    per batch of gradients, BF16 checkpoints, autotuned kernels) against the plain
    FP32 form run design by design, one timed pass each after a warm-up."""
    import torch
    from paper_2411_03090_gb300 import LKS, LKSBatch

    pbs = inputs.config5()
    N, n_steps = sum(p.n_nodes for p in pbs), pbs[0].n_steps
    gam = [torch.from_numpy(p.gamma().astype(np.float32)).to(dev) for p in pbs]
    b = LKSBatch(pbs, snapshot="bf16", device=dev)
    b.gradient(gam)
    torch.cuda.synchronize()
    flush.fill_(1.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    _, G = b.gradient(gam)
    e1.record(b.stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) * 1e-3
    st = b.query()
    if st.device_status != 0:
        raise RuntimeError(f"device status {st.device_status}")
    Gb = [g.double() for g in G]
    ws_batch = st.workspace_bytes / 1e9
    del b, G
    torch.cuda.empty_cache()
    t_plain, errs, ws_plain = 0.0, [], 0
    for k, p in enumerate(pbs):
        s = LKS(p, real="f32", checkpoint_every=0, device=dev)
        ws_plain += s.workspace.numel()
        s.gradient(gam[k])
        torch.cuda.synchronize()
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        _, gp = s.gradient(gam[k])
        e1.record(s.stream)
        torch.cuda.synchronize()
        t_plain += e0.elapsed_time(e1) * 1e-3
        gp = gp.double()
        errs.append((torch.linalg.vector_norm(Gb[k] - gp) / torch.linalg.vector_norm(gp)).item())
        del s
        torch.cuda.empty_cache()
    return {"workload": f"config5: {len(pbs)} unsteady designs 128x64..512x256, {n_steps} + {n_steps} steps",
            "batched_s_per_batch_gradient": t_batch, "batched_MLUPS": N * 2 * n_steps / t_batch / 1e6,
            "batched_workspace_GB": ws_batch, "plain_fp32_s_design_by_design": t_plain,
            "plain_workspace_GB_all_designs": ws_plain / 1e9, "speedup": t_plain / t_batch,
            "grad_rel_err_vs_plain_max": max(errs)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="config4")
    ap.add_argument("--oracle-levels", type=int, default=200,
                    help="config3: levels of the truncated horizon compared with the FP64 oracle (0: none)")
    ap.add_argument("--fd-max-steps", type=int, default=1500000,
                    help="config2fd: step limit of the base tolerance marches")
    ap.add_argument("--fd-tol", type=float, default=1e-12,
                    help="config2fd: relative step change the base marches run to")
    ap.add_argument("--fd-steps", type=int, default=30000,
                    help="config2fd: steps of each perturbed march from the converged base state")
    ap.add_argument("--no-also", action="store_true",
                    help="config4: skip the config2, 8192^2, config3 and config5 figures carried on the same line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--steps-override", type=int, default=0)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--res-steps", type=int, default=0,
                    help="resident marches: steps per exchange of tile bands (0: automatic)")
    ap.add_argument("--tile-config", type=int, default=-1,
                    help="config5: TMA tile shape (-1: autotuned at create)")
    ap.add_argument("--fwd-column", type=int, default=-1,
                    help="config5: forward kernel (-1: autotuned, 0: TMA-staged, 1: warp-column)")
    ap.add_argument("--adj-column", type=int, default=-1,
                    help="config5: adjoint kernel (-1: autotuned, 0: TMA-staged, 1: warp-column)")
    ap.add_argument("--exec-path", default="auto", choices=["auto", "step", "resident", "column"],
                    help="config1/2/4: how the marches run (the library's exec_path)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "config3":
        run_checkpoint_study(args)
        return
    if args.workload == "config5":
        run_batch_study(args)
        return
    if args.workload == "config2fd":
        run_fd_study(args)
        return

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    pb, desc = workload(args.workload)
    if args.steps_override:
        pb = pb.with_(n_steps=args.steps_override, n_adj=args.steps_override)
        desc += f" (shortened to {args.steps_override}+{args.steps_override} steps)"
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    clocks = ClockSampler(local)
    m = measure(pb, args, dev, flush, args.steps, max(args.warmup, 3), world, clocks=clocks, e2e=not args.no_e2e)
    total_ms = m["total_ms"]
    value = job_mlups(world, m["updates_per_step"], args.steps, total_ms)
    e2e_val = m["e2e_single"] * world if m["e2e_single"] is not None else None

    also = {}
    if args.workload == "config4" and not args.steps_override and not args.no_also:
        for name in ("config2", "roofline8192"):
            pb2, desc2 = workload(name)
            m2 = measure(pb2, args, dev, flush, 2, 1, 1, e2e=False)
            also[name] = {"workload": desc2, "value": m2["updates_per_step"] * 2 / (m2["total_ms"] * 1e-3) / 1e6,
                          "unit": "MLUPS", "s_per_gradient": m2["total_ms"] / 2 / 1e3, "roofline": m2["roofline"]}
            if name == "config2":
                also[name]["roofline"]["note"] = ("working set (0.5 MB per field) resident in L2 and shared "
                                                  "memory: the fraction is of HBM, but the traffic is on chip")
        if world == 1:  # the checkpointed and batched forms, once, on the single-GPU line
            for name, fn in (("config3", also_config3), ("config5", also_config5)):
                try:
                    also[name] = fn(dev, flush)
                except Exception as e:  # reported on the line, never silently dropped
                    also[name] = {"error": f"{type(e).__name__}: {e}"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    N = pb.n_nodes
    three_d = hasattr(pb, "nz")
    st = m["stats"]
    out = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc,
                   "lattice": f"{pb.nx}x{pb.ny}" + (f"x{pb.nz}" if three_d else ""), "forward_steps": pb.n_steps,
                   "adjoint_steps": pb.n_adj, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world}", "s_per_gradient": total_ms / args.steps / 1e3,
                   **({"resident_steps_per_exchange": [st.res_steps_fwd, st.res_steps_adj]}
                      if st.fwd_path == 2 or st.adj_path == 2 else {})},
        "roofline": m["roofline"],
        "e2e": {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": 4 * N,
                "d2h_bytes_per_step": 4 * N + 8 + 4},
        "gpu_launches": int(m["launches"]),
        "clocks": m["clocks"],
    }
    if also:
        out["also"] = also
    if not args.no_cpu_baseline:
        try:
            n_cb = oracle_steps_for(pb, 15.0)  # a bounded sample: 10-15 s of host work (the 2-step calibration runs long)
            out["cpu_baseline"] = cpu_baseline(pb, n_cb, n_cb)
        except Exception as e:  # the oracle is a reported baseline, not the product
            out["cpu_baseline"] = {"value": None, "unit": "MLUPS", "kind": "oracle", "error": str(e)}
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def measure(pb, args, dev, flush, steps, warmup, world, clocks=None, e2e=True):
    """Times `steps` gradients of one steady problem (after `warmup` untimed ones)
    with CUDA events on the library's stream: the whole gradient, the forward march
    and the adjoint march.  Returns the slowest rank's total milliseconds, the
    roofline of the adjoint and forward step kernels, the kernels launched in the
    timed region and, when asked, the end-to-end rate through lks_gradient_host."""
    import torch
    from paper_2411_03090_gb300 import LKS

    g_np = pb.gamma()
    gamma = torch.from_numpy(g_np).to(dev, torch.float32)
    s = LKS(pb, real="f32", device=dev, res_steps=args.res_steps, path=args.exec_path)
    stream = s.stream
    N = pb.n_nodes

    def one_gradient(ev=None):
        J = s.lks_forward(gamma)
        if ev is not None:
            ev[1].record(stream)
        s.alks_adjoint()
        if ev is not None:
            ev[2].record(stream)
        g = s.lks_sensitivity()
        return J, g

    for _ in range(max(warmup, 1)):
        one_gradient()
    torch.cuda.synchronize()

    launches0 = s.query().kernel_launches
    if clocks is not None:
        clocks.start()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, fwd_ms, adj_ms = [], [], []
    for _ in range(steps):
        flush.fill_(1.0)  # evict the previous gradient's working set from L2
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        one_gradient(ev)
        ev[3].record(stream)
        torch.cuda.synchronize()
        step_ms.append(ev[0].elapsed_time(ev[3]))
        fwd_ms.append(ev[0].elapsed_time(ev[1]))
        adj_ms.append(ev[1].elapsed_time(ev[2]))
    torch.cuda.synchronize()
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    clk = clocks.stop() if clocks is not None else None
    st = s.query()
    launches = st.kernel_launches - launches0

    # Dominant kernel (adjoint step): algorithmic bytes per launch / mean duration.
    hbm, peak_kind = peaks()
    adj_launch_s = (sum(adj_ms) / len(adj_ms)) * 1e-3 / pb.n_adj
    fwd_launch_s = (sum(fwd_ms) / len(fwd_ms)) * 1e-3 / pb.n_steps
    three_d = hasattr(pb, "nz")
    b_adj = BYTES_ADJ_3D if three_d else BYTES_ADJ_STEADY
    b_fwd = BYTES_FWD_3D if three_d else BYTES_FWD
    adj_gbs = b_adj * N / adj_launch_s / 1e9
    fwd_gbs = b_fwd * N / fwd_launch_s / 1e9
    step_names = (("adj_tma_kernel<false,true,false>", "fwd_tma_kernel<false,false>") if pb.nx % 4 == 0 else
                  ("adj_step_kernel<float,false>", "fwd_step_kernel<float,false>"))
    kname = {1: step_names, 2: ("adj_resident_kernel<float>", "fwd_resident_kernel<float,false>"),
             3: ("adj_col_kernel<true>", "fwd_col2_kernel<10>")}
    adj_k = kname.get(st.adj_path, kname[1])[0]
    fwd_k = kname.get(st.fwd_path, kname[1])[1]
    if three_d:
        tma3 = pb.nx % 4 == 0
        adj_k = ("adj3c_kernel" if st.adj_path == 3 else "adj3t_kernel") if tma3 else "adj3_kernel<float>"
        fwd_k = ("fwd3p_kernel" if st.fwd_path == 3 else "fwd3t_kernel") if tma3 else "fwd3_kernel<float>"

    def traffic(k):
        b = TRAFFIC_BYTES_PER_NODE.get(k)
        return None if b is None else b * N

    roofline = {"bound": "hbm", "kernel": adj_k, "achieved": adj_gbs, "peak": hbm,
                "unit": "GB/s", "frac": adj_gbs / hbm, "traffic": traffic(adj_k), "peak_kind": peak_kind,
                "algorithmic_bytes_per_node": b_adj, "mean_step_us": adj_launch_s * 1e6,
                "forward": {"kernel": fwd_k, "achieved": fwd_gbs, "frac": fwd_gbs / hbm,
                            "traffic": traffic(fwd_k), "algorithmic_bytes_per_node": b_fwd,
                            "mean_step_us": fwd_launch_s * 1e6}}

    # End to end through the C ABI with host buffers (pinned), copies inside.
    e2e_val = None
    if e2e:
        g_host = torch.from_numpy(g_np.astype(np.float32)).pin_memory().numpy()
        grad_host = torch.empty(*g_np.shape, dtype=torch.float32).pin_memory().numpy()
        s.gradient_host(g_host, grad_host)
        e2e_t = []
        for _ in range(max(2, min(steps, 3))):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.gradient_host(g_host, grad_host)
            e2e_t.append(time.perf_counter() - t0)
        e2e_val = N * (pb.n_steps + pb.n_adj) / (sum(e2e_t) / len(e2e_t)) / 1e6
    out = {"total_ms": total_ms, "updates_per_step": N * (pb.n_steps + pb.n_adj), "roofline": roofline,
           "launches": launches, "clocks": clk, "stats": st, "e2e_single": e2e_val}
    del s
    torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    main()
