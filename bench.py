"""Benchmark of the BDD Lagrange-dual hot path (DOGE-Train's Alg. 1 on GB300).

One step = one dual iteration of generalized min-marginal averaging over the
whole instance: forward sweep, S reduction, backward sweep (with the
subproblem energies), S reduction and the FP64 per-instance lower bound.
Metric: BDD-arc updates per second (2 sweeps x 2 arcs per node per
iteration), with the HBM roofline of the sweep kernel beside it.

Default workload: the tracking-like flow instance (500 frames x 2,000
detections, ~6M variables, ~3M constraints), the largest single-GPU
configuration.  Inputs are seeded synthetic data (the paper's datasets are
not available).

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Multi-GPU: every rank solves its own copy of the instance (independent
problems, no collective); value = arc updates of all ranks / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "BDD-arc updates/s per dual iteration (forward+backward sweep)"
UNIT = "arc-updates/s"
WORKLOADS = {
    "tracking_500x2000": lambda: workloads.tracking(),
    "tracking_200x2000": lambda: workloads.tracking(frames=200),
    "matching_quadratic_200": lambda: workloads.matching_quadratic(),
    "independent_set_10k": lambda: workloads.independent_set(),
    "assignment_2000x300": lambda: workloads.assignment(),
}



# layout knobs the tuner tries: locality chunks (rows) and footprint ratios
# (percent) of the launch groups
TUNE_CHUNKS = (16384, 32768)
TUNE_RATIOS = (85, 88, 90, 92)

def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "of measured"
    except Exception:
        return 6800.0, "of fallback"


def _profile_traffic(kernel_key: str, src_sha: str):
    """DRAM bytes per launch recorded by an ncu capture (profiles/*.md), or
    None when absent or taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", f"{kernel_key}.md")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("source_sha") != src_sha:
        return None
    try:
        return float(kv["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


def _kernel_source_sha():
    h = hashlib.sha256()
    for f in ("kernels_sweep.cu", "sweep.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2205_11638_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # the timed region starts only once the sampler is producing lines
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
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
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(local_ms: float, units_per_rank: float, world_size: int, all_reduce_max=None):
    """Whole-job throughput: every rank processes units_per_rank in its own
    time; the job takes the slowest rank's time.  all_reduce_max(x) returns
    the maximum of x over ranks (None for one rank)."""
    t = all_reduce_max(local_ms) if (all_reduce_max and world_size > 1) else local_ms
    return units_per_rank * world_size / (t * 1e-3), t


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    # one oracle iteration per step.  The tracking instance itself when the
    # run is short enough (about 2 s per iteration of the 500-frame instance
    # on one core, plus ~20 s to build its BDDs): up to 40 iterations in all;
    # otherwise a slice of the same generator sized so that the whole run
    # stays within about a minute (about 3 ms per frame and iteration).  The
    # other workloads are small enough to run whole.
    if args.workload == "tracking_500x2000" and args.steps + args.warmup > 40:
        frames = int(max(3, min(50, 12000 // max(1, args.steps + args.warmup))))
        prob = workloads.tracking(frames=frames, dets=2000)
        what = f"tracking {frames} frames x 2000 detections"
    else:
        prob = WORKLOADS[args.workload]()
        what = f"{args.workload} (the whole instance)"
    O = oracle.Oracle(prob)
    lam, M = O.init_lambda()
    arcs = 4 * O.num_nodes
    for _ in range(args.warmup):
        lam, M = O.iterate(lam, M, 0.5, None, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        lam, M = O.iterate(lam, M, 0.5, None, 1)
    dt = time.perf_counter() - t0
    val = arcs * args.steps / dt
    sample = f"{what} ({O.num_slots} slots), one oracle iteration per step"
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "sample": sample},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def _matching_adjoint_measurement(solver, torch, iters=20, ck=10, reps=5):
    """The matching instance with linearised quadratic terms (200 x 200, 10
    candidates, 20,000 pairs) and per-slot parameters (omega = sigmoid of
    random logits, alpha = softmax of random logits over each variable's
    rows): forward + adjoint of the final lower bound through 20 unrolled
    iterations, in ms (mean of `reps` after one warm-up)."""
    import numpy as np
    prob = workloads.matching_quadratic()
    A = solver.plan(prob).bind()
    col, n = prob["col"], prob["n"]
    rng = np.random.default_rng(3)
    z = np.exp(rng.normal(size=len(col)))
    s = np.zeros(n)
    np.add.at(s, col, z)
    alpha = A.from_csr(z / s[col])
    omega = A.from_csr(1.0 / (1.0 + np.exp(-rng.normal(size=len(col)))))
    lam0, M0 = A.init_lambda()
    ws = torch.empty(A.backward_workspace_bytes(iters, ck), dtype=torch.uint8, device=A.device)
    outs = [A.zeros() for _ in range(4)]
    gl, gM = A.zeros(), A.zeros()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    f_ms = b_ms = 0.0
    for rep in range(reps + 1):
        lam, M = lam0.clone(), M0.clone()
        torch.cuda.synchronize()
        ev[0].record()
        A.iterate_checkpointed(lam, M, omega, alpha, iters=iters, ckpt_every=ck, workspace=ws)
        A.lb_seed_into(lam, M, gl, gM)
        ev[1].record()
        A.backward_checkpointed(omega, alpha, iters, ck, gl, gM, ws, outs)
        ev[2].record()
        torch.cuda.synchronize()
        if rep > 0:
            f_ms += ev[0].elapsed_time(ev[1]) / reps
            b_ms += ev[1].elapsed_time(ev[2]) / reps
    # the same step captured once as a CUDA graph and replayed (what a
    # training loop over fixed shapes would do)
    def step():
        lam.copy_(lam0)
        M.copy_(M0)
        A.iterate_checkpointed(lam, M, omega, alpha, iters=iters, ckpt_every=ck, workspace=ws)
        A.lb_seed_into(lam, M, gl, gM)
        A.backward_checkpointed(omega, alpha, iters, ck, gl, gM, ws, outs)

    lam, M = lam0.clone(), M0.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    graph.replay()
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(reps):
        graph.replay()
    ev[1].record()
    torch.cuda.synchronize()
    g_ms = ev[0].elapsed_time(ev[1]) / reps
    # what the oracle leg compares: the inputs (CSR order) and the gradients
    # of the last replay
    keep = {"prob": prob, "lam0": A.to_csr(lam0).double().cpu().numpy(), "M0": A.to_csr(M0).double().cpu().numpy(),
            "omega": A.to_csr(omega).double().cpu().numpy(), "alpha": A.to_csr(alpha).double().cpu().numpy(),
            "grads": [A.to_csr(o).double().cpu().numpy() for o in outs], "iters": iters}
    return {"workload": "matching_quadratic_200", "N_lambda": int(A.stats.sizes.num_lambda),
            "unrolled_iterations": iters, "checkpoint_every": ck, "parameters": "per-slot omega, alpha",
            "forward_ms": f_ms, "backward_ms": b_ms, "fwd_adjoint_ms": f_ms + b_ms,
            "fwd_adjoint_graph_replay_ms": g_ms, "loss": "lower bound (eq. 3 plus unary term)"}, keep


def _batched_measurement(args, solver, torch, iters=50, ck=10):
    """64 uneven instances (independent set, set cover, matching) in one arena,
    ``iters`` iterations captured in one CUDA graph with per-instance FP64
    bounds, against the same instances solved one arena per instance with
    plain dg_iterate calls; then fwd + adjoint of the whole batch against
    fwd + adjoint per instance."""
    prob, kinds = workloads.batched_mix(num=64)
    A = solver.plan(prob).bind()
    stream = torch.cuda.Stream()
    lam0, M0 = A.init_lambda()
    lam, M = lam0.clone(), M0.clone()
    lb = torch.zeros(A.num_inst, dtype=torch.float64, device=A.device)
    with torch.cuda.stream(stream):
        g = A.graph(lam, M, iters=iters, lb_out=lb, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        for r in range(reps + 1):
            lam.copy_(lam0)
            M.copy_(M0)
            if r == 1:
                e0.record(stream)
            g.replay(stream)
        e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / reps
    lb_batch = lb.cpu().numpy().copy()
    # one arena per instance
    irp, ivp = prob["inst_row_ptr"], prob["inst_var_ptr"]
    singles = []
    for k in range(len(irp) - 1):
        r0, r1, v0, v1 = int(irp[k]), int(irp[k + 1]), int(ivp[k]), int(ivp[k + 1])
        b0, b1 = int(prob["row_ptr"][r0]), int(prob["row_ptr"][r1])
        sub = dict(n=v1 - v0, row_ptr=prob["row_ptr"][r0:r1 + 1] - b0, col=prob["col"][b0:b1] - v0,
                   coef=prob["coef"][b0:b1], sense=prob["sense"][r0:r1], rhs=prob["rhs"][r0:r1], c=prob["c"][v0:v1])
        singles.append(solver.plan(sub).bind())
    states = [S.init_lambda() for S in singles]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lbs = []
    for rep in range(2):
        work = [(l.clone(), m.clone()) for (l, m) in states]
        torch.cuda.synchronize()
        e0.record()
        lbs = [S.iterate(l, m, iters=iters, lb=True) for S, (l, m) in zip(singles, work)]
        e1.record()
        torch.cuda.synchronize()
    t_single = e0.elapsed_time(e1)
    lb_single = np.array([float(x[0]) for x in lbs])
    rel = float(np.max(np.abs(lb_single - lb_batch) / np.maximum(1.0, np.abs(lb_single))))
    # fwd + adjoint (lower-bound loss) on the batch vs per instance
    def fwd_adj(S, l0, m0):
        l, m = l0.clone(), m0.clone()
        ws, _ = S.iterate_checkpointed(l, m, iters=iters, ckpt_every=ck)
        gl, gM = S.lb_seed(l, m)
        return S.backward_checkpointed(None, None, iters, ck, gl, gM, ws)
    fwd_adj(A, lam0, M0)
    torch.cuda.synchronize()
    e0.record()
    fwd_adj(A, lam0, M0)
    e1.record()
    torch.cuda.synchronize()
    t_batch_adj = e0.elapsed_time(e1)
    e0.record()
    for S, (l, m) in zip(singles, states):
        fwd_adj(S, l, m)
    e1.record()
    torch.cuda.synchronize()
    t_single_adj = e0.elapsed_time(e1)
    # the batch's forward + adjoint captured once as a CUDA graph and replayed
    ws = torch.empty(A.backward_workspace_bytes(iters, ck), dtype=torch.uint8, device=A.device)
    gl, gM = A.zeros(), A.zeros()
    outs = [A.zeros() for _ in range(4)]
    lam_w, M_w = lam0.clone(), M0.clone()

    def batch_step():
        lam_w.copy_(lam0)
        M_w.copy_(M0)
        A.iterate_checkpointed(lam_w, M_w, iters=iters, ckpt_every=ck, workspace=ws)
        A.lb_seed_into(lam_w, M_w, gl, gM)
        A.backward_checkpointed(None, None, iters, ck, gl, gM, ws, outs)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        batch_step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch_step()
    graph.replay()
    torch.cuda.synchronize()
    e0.record()
    graph.replay()
    e1.record()
    torch.cuda.synchronize()
    t_batch_adj_graph = e0.elapsed_time(e1)
    return {"instances": int(A.num_inst), "kinds": {"independent_set": int((kinds == 0).sum()),
            "set_cover": int((kinds == 1).sum()), "matching": int((kinds == 2).sum())},
            "N_lambda": int(A.stats.sizes.num_lambda), "iterations": iters,
            "batched_graph_ms": t_batch, "one_instance_per_launch_ms": t_single,
            "speedup_plain": t_single / t_batch, "max_rel_bound_difference_batched_vs_single": rel,
            "batched_fwd_adjoint_ms": t_batch_adj, "batched_fwd_adjoint_graph_replay_ms": t_batch_adj_graph,
            "one_instance_per_launch_fwd_adjoint_ms": t_single_adj,
            "speedup_fwd_adjoint": t_single_adj / t_batch_adj, "checkpoint_every": ck}, \
        {"prob": prob, "lb": lb_batch, "iters": iters}


def _independent_set_measurement(solver, torch, iters=200, reps=5):
    """Independent set on G(n = 10,000, p = 8/(n-1)) (about 40,000 two-variable
    rows), plain method, 200 iterations per CUDA-graph replay: arc updates per
    second.  Arena and state (~3 MB) stay in L2, so the byte rate is an L2
    rate, not an HBM one."""
    prob = workloads.independent_set()
    A = solver.plan(prob).bind()
    lam0, M0 = A.init_lambda()
    lam, M = lam0.clone(), M0.clone()
    lb = torch.zeros(1, dtype=torch.float64, device=A.device)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = A.graph(lam, M, iters=iters, lb_out=lb, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for r in range(reps + 2):
            lam.copy_(lam0)
            M.copy_(M0)
            e0.record(stream)
            g.replay(stream)
            e1.record(stream)
            e1.synchronize()
            if r >= 2:
                ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms)
    st = A.stats
    arcs = 4 * st.sizes.num_nodes * iters
    return {"workload": "independent_set_10k", "n_vars": int(st.sizes.n), "constraints": int(st.sizes.m),
            "N_lambda": int(st.sizes.num_lambda), "N_v": int(st.sizes.num_nodes), "iterations": iters,
            "value": arcs / (t * 1e-3), "unit": UNIT, "ms_per_iteration": t / iters,
            "algorithmic_bytes_per_iteration": st.bytes_per_iter,
            "algorithmic_GBps": st.bytes_per_iter * iters / (t * 1e-3) / 1e9,
            "memory_level": "L2 (arena + state below the 126 MB L2; not an HBM roofline)",
            "timing": "median of 5 CUDA-graph replays of 200 iterations"}, \
        {"prob": prob, "lb": float(lb[0]), "iters": iters}


def _long_rows_measurement(solver, torch, iters=50, reps=3):
    """Sparse assignment with long rows (2,000 x 2,000, 300 candidates per
    left node: 4,000 rows of about 300 variables, every BDD beyond a tile
    lane, every level two nodes wide): the plain sweeps of narrow long BDDs,
    several to a warp.  Arc updates per second over a CUDA-graph replay of
    50 iterations, and the roofline of the long-BDD sweep kernel from its
    own CUDA-event time."""
    prob = workloads.assignment()
    A = solver.plan(prob).bind()
    st = A.stats
    lam0, M0 = A.init_lambda()
    lam, M = lam0.clone(), M0.clone()
    lb = torch.zeros(1, dtype=torch.float64, device=A.device)
    stream = torch.cuda.Stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with torch.cuda.stream(stream):
        g = A.graph(lam, M, iters=iters, lb_out=lb, stream=stream)
        ms = []
        for r in range(reps + 1):
            lam.copy_(lam0)
            M.copy_(M0)
            ev[0].record(stream)
            g.replay(stream)
            ev[1].record(stream)
            ev[1].synchronize()
            if r > 0:
                ms.append(ev[0].elapsed_time(ev[1]))
        # one forward and one backward sweep timed on their own
        sw = []
        for r in range(4):
            ev[0].record(stream)
            A.sweep(lam, M, forward=True, stream=stream, costs_in=r > 0, costs_out=True)
            ev[1].record(stream)
            A.sum_M(M, stream=stream)
            ev[2].record(stream)
            A.sweep(lam, M, forward=False, stream=stream, costs_in=True, costs_out=True)
            ev[3].record(stream)
            ev[3].synchronize()
            if r > 0:
                sw += [ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])]
    t = statistics.median(ms)
    sweep_ms = statistics.mean(sw)
    Nv, Nl = st.sizes.num_nodes, st.sizes.num_lambda
    sweep_bytes = 16.0 * Nv + 16.0 * Nl
    peak, peak_src = _peaks()
    achieved = sweep_bytes / (sweep_ms * 1e-3) / 1e9
    return {"workload": "assignment_2000x300", "n_vars": int(st.sizes.n), "constraints": int(st.sizes.m),
            "N_lambda": int(Nl), "N_v": int(Nv), "long_bdds": int(st.sizes.num_long_bdds),
            "long_nodes": int(st.sizes.num_long_nodes), "iterations": iters,
            "value": 4 * Nv * iters / (t * 1e-3), "unit": UNIT, "ms_per_iteration": t / iters,
            "roofline": {"bound": "hbm", "kernel": "k_long_narrow (forward and backward; long BDDs of narrow levels, several to a warp)",
                         "algorithmic_bytes_per_launch": sweep_bytes, "avg_launch_ms": sweep_ms,
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": peak_src},
            "timing": "median of 3 CUDA-graph replays of 50 iterations; sweeps: mean of 3 forward + 3 backward"}, \
        {"iters": iters}


def _e2e_steps(A, lam, M, steps, stream, torch, chunks=4):
    """End-to-end steps with host-resident state: each step uploads (lambda, M)
    from pinned host memory, runs forward sweep, S reduction, backward sweep,
    S reduction and bound through the public calls, and downloads (lambda, M,
    bound).  The copies run on their own streams in chunks, ordered only by
    what they depend on: a chunk's upload waits for the previous step's
    download of that chunk and for the previous step's last read of the
    device state; the first S reduction waits for M only, the sweeps for
    lambda too; the downloads start when the backward sweep has written the
    state.  Returns (ms of all steps, ms of the same steps with every copy
    serialised on the compute stream)."""
    h = [M.detach().cpu().pin_memory(), lam.detach().cpu().pin_memory()]
    d = [torch.empty_like(M), torch.empty_like(lam)]
    h_lb = torch.zeros(A.num_inst, dtype=torch.float64).pin_memory()
    lb_out = torch.zeros(A.num_inst, dtype=torch.float64, device=A.device)
    NS = A.num_slots
    cut = [NS * c // chunks // 64 * 64 for c in range(chunks)] + [NS]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    Ev = torch.cuda.Event
    e0, e1 = Ev(enable_timing=True), Ev(enable_timing=True)
    # events made once and re-recorded every step (a wait uses the latest record)
    ev_up = [Ev(), Ev()]
    ev_down = [[Ev() for _ in range(chunks)] for _ in range(2)]
    ev_final, ev_done = Ev(), Ev()
    hv = [[x[cut[c]:cut[c + 1]] for c in range(chunks)] for x in h]
    dv = [[x[cut[c]:cut[c + 1]] for c in range(chunks)] for x in d]

    def run(overlap):
        s_up = up if overlap else stream
        s_down = down if overlap else stream
        torch.cuda.synchronize()
        t_host = time.perf_counter()
        e0.record(stream)
        for k in range(steps):
            if overlap and k > 0:
                up.wait_event(ev_done)
            for j in range(2):  # M, then lambda
                for c in range(chunks):
                    if overlap and k > 0:
                        up.wait_event(ev_down[j][c])
                    with torch.cuda.stream(s_up):
                        dv[j][c].copy_(hv[j][c], non_blocking=True)
                ev_up[j].record(s_up)
            stream.wait_event(ev_up[0])
            A.sum_M(d[0], stream=stream)
            stream.wait_event(ev_up[1])
            A.sweep(d[1], d[0], forward=True, stream=stream, costs_out=True)
            A.sum_M(d[0], stream=stream)
            A.sweep(d[1], d[0], forward=False, energy=True, stream=stream, costs_in=True)
            ev_final.record(stream)
            s_down.wait_event(ev_final)
            for j in range(2):
                for c in range(chunks):
                    with torch.cuda.stream(s_down):
                        hv[j][c].copy_(dv[j][c], non_blocking=True)
                    ev_down[j][c].record(s_down)
            A.sum_M(d[0], stream=stream)
            A.bound_from_energies(lb_out, stream=stream)
            h_lb.copy_(lb_out, non_blocking=True)
            ev_done.record(stream)
        stream.wait_stream(down)
        stream.wait_stream(up)
        e1.record(stream)
        t_host = time.perf_counter() - t_host
        torch.cuda.synchronize()
        run.host_ms = t_host * 1e3
        return e0.elapsed_time(e1)

    with torch.cuda.stream(stream):
        run(True)  # warm-up of the streams and events
        serial = run(False)
        overlapped = run(True)
    return overlapped, serial, run.host_ms


def _err_stats(g, w):
    rel = float(np.linalg.norm(g - w) / max(1e-12, np.linalg.norm(w)))
    return {"rel_l2": rel, "frac_within_1e-4": float(np.mean(np.abs(g - w) <= 1e-4)),
            "max_abs": float(np.abs(g - w).max())}


def _oracle_leg(args, A, prob, solver, torch, keep):
    """The CPU-baseline leg: the FP64 oracle timed on the host (single thread
    as the checker, and its OpenMP build on all cores), and every figure of
    the GPU run compared with the oracle on the same seeded inputs.  Nothing
    here is timed on the GPU."""
    import oracle
    par = {"tolerances": {"lambda_M_after_1_iteration": "max abs <= 1e-5 * max|c|",
                          "bound": "relative <= 1e-5",
                          "gradients": "rel. L2 < 1e-3 and >= 99% within 1e-4 (long unrolls)"}}
    # (a) the benchmark instance itself, one iteration from the initial split
    cmax = float(np.abs(prob["c"]).max())
    lam, M = A.init_lambda()
    lb1 = float(A.iterate(lam, M, iters=1, lb=True)[0])
    t0 = time.perf_counter()
    O = oracle.Oracle(prob)
    ol, oM = O.init_lambda()
    ol, oM = O.iterate(ol, oM, 0.5, None, 1)
    olb1 = O.lower_bound(ol, oM)
    el = float(np.abs(A.to_csr(lam).double().cpu().numpy() - ol).max())
    eM = float(np.abs(A.to_csr(M).double().cpu().numpy() - oM).max())
    # the FP64 summation of the bound: the GPU's bound against the exactly
    # rounded sum (math.fsum) of its own float32 terms E^j and min(0, S_i)
    import math
    lbE, E = A.lower_bound(lam, M, energies=True)
    Sf = np.zeros(prob["n"], np.float32)
    np.add.at(Sf, prob["col"], A.to_csr(M).cpu().numpy().astype(np.float32))
    covered = np.bincount(prob["col"], minlength=prob["n"]) > 0
    exact = math.fsum(E.cpu().numpy().astype(np.float64).tolist() +
                      np.minimum(0.0, Sf.astype(np.float64)).tolist() +
                      np.minimum(0.0, prob["c"][~covered]).tolist())
    par[args.workload] = {"lambda_max_abs_err_over_max_c": el / cmax, "M_max_abs_err_over_max_c": eM / cmax,
                          "bound_after_1_iteration": lb1, "bound_rel_err": abs(lb1 - olb1) / max(1.0, abs(olb1)),
                          "bound_fp64_sum_rel_err_vs_exact_sum_of_its_terms": abs(float(lbE[0]) - exact) / abs(exact),
                          "iterations": 1, "oracle_s": time.perf_counter() - t0}
    del O, ol, oM
    # (b) 50-frame slice of the same generator: bound after 100 iterations;
    #     the single-threaded oracle's run is the CPU baseline
    frames, its = 50, 100
    sl = workloads.tracking(frames=frames, dets=2000)
    B = solver.plan(sl).bind()
    bl, bM = B.init_lambda()
    glb = float(B.iterate(bl, bM, iters=its, lb=True)[0])
    O = oracle.Oracle(sl)
    ol0, oM0 = O.init_lambda()
    t0 = time.perf_counter()
    ol, oM = O.iterate(ol0, oM0, 0.5, None, its)
    dt = time.perf_counter() - t0
    olb = O.lower_bound(ol, oM)
    arcs = 4 * O.num_nodes
    sample = f"tracking {frames} frames x 2000 detections ({O.num_slots} slots, {O.num_nodes} nodes), {its} iterations"
    cpu = {"value": arcs * its / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"{sample} in {dt:.1f} s"}
    par["tracking_50x2000_slice"] = {"bound_after_100_iterations": glb, "bound_rel_err": abs(glb - olb) / abs(olb),
                                     "iterations": its}
    cpu_all = None
    try:
        P = oracle.Oracle(sl, openmp=True)
        t0 = time.perf_counter()
        pl, pM = P.iterate(ol0, oM0, 0.5, None, its)
        dta = time.perf_counter() - t0
        cpu_all = {"value": arcs * its / dta, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle (OpenMP over BDDs)",
                   "sample": f"{sample} in {dta:.1f} s", "bit_identical_to_single_thread":
                       bool(np.array_equal(pl, ol) and np.array_equal(pM, oM))}
        del P
    except Exception as e:  # noqa: BLE001 -- no OpenMP runtime: report why
        cpu_all = {"unavailable": f"{type(e).__name__}: {e}"}
    del O
    # (c) the 64-instance batch: per-instance bounds of the timed replay
    if "batched" in keep:
        kb = keep["batched"]
        O = oracle.Oracle(kb["prob"])
        ol, oM = O.init_lambda()
        ol, oM = O.iterate(ol, oM, 0.5, None, kb["iters"])
        want = O.lower_bound(ol, oM, per_instance=True)[1]
        rel = np.abs(kb["lb"] - want) / np.maximum(1.0, np.abs(want))
        par["batched_64"] = {"max_bound_rel_err": float(rel.max()), "iterations": kb["iters"]}
        del O
    # (d) the independent-set line
    if "independent_set" in keep:
        ki = keep["independent_set"]
        O = oracle.Oracle(ki["prob"])
        ol, oM = O.init_lambda()
        ol, oM = O.iterate(ol, oM, 0.5, None, ki["iters"])
        w = O.lower_bound(ol, oM)
        par["independent_set_10k"] = {"bound_rel_err": abs(ki["lb"] - w) / max(1.0, abs(w)),
                                      "iterations": ki["iters"]}
    # (d2) the long-row line: the oracle's builder needs ~40 s for the 4,000
    #      rows of 300 variables, so a 600 x 600 slice of the same generator
    #      (1,200 rows of about 300 variables) stands for it: lambda after one
    #      iteration and the bound after the line's 50
    if "long_rows" in keep:
        its = keep["long_rows"]["iters"]
        sl = workloads.assignment(L=600, R=600, cand=300)
        B = solver.plan(sl).bind()
        bl, bM = B.init_lambda()
        B.iterate(bl, bM, iters=1)
        l1 = B.to_csr(bl).double().cpu().numpy()
        glb = float(B.iterate(bl, bM, iters=its - 1, lb=True)[0])
        O = oracle.Oracle(sl)
        ol, oM = O.init_lambda()
        ol, oM = O.iterate(ol, oM, 0.5, None, 1)
        el = float(np.abs(l1 - ol).max()) / float(np.abs(sl["c"]).max())
        ol, oM = O.iterate(ol, oM, 0.5, None, its - 1)
        w = O.lower_bound(ol, oM)
        par["assignment_600x300_slice"] = {"lambda_max_abs_err_over_max_c": el, "bound_rel_err": abs(glb - w) / abs(w),
                                           "iterations": its}
        del O, B
    # (e) the matching adjoint: gradients against the oracle's Alg. 2, and the
    #     oracle's own forward + adjoint time on one core
    cpu_matching = None
    if "matching" in keep:
        km = keep["matching"]
        O = oracle.Oracle(km["prob"])
        t0 = time.perf_counter()
        lT, MT = O.iterate(km["lam0"], km["M0"], km["omega"], km["alpha"], km["iters"])
        sl_, sM_ = O.lb_seed(lT, MT)
        want = O.backward(km["lam0"], km["M0"], km["omega"], km["alpha"], km["iters"], sl_, sM_)
        dtm = time.perf_counter() - t0
        par["adjoint_matching"] = {nm: _err_stats(g, w) for nm, g, w in
                                   zip(("g_lambda0", "g_M0", "g_omega", "g_alpha"), km["grads"], want)}
        cpu_matching = {"fwd_adjoint_ms": dtm * 1e3, "cores": 1, "kind": "oracle",
                        "sample": f"matching_quadratic_200, {km['iters']} unrolled iterations, forward + Alg. 2"}
    # (f) the tracking adjoint: the full instance's 100-iteration adjoint is
    #     beyond the oracle's memory (it keeps every sweep); a 12 x 300 slice
    #     with the same checkpointing (two segments) stands for it
    if "adjoint" in keep:
        tr = workloads.tracking(frames=12, dets=300, seed=77)
        C = solver.plan(tr).bind()
        T, ck = 10, 5
        l0, m0 = C.init_lambda()
        lw, mw = l0.clone(), m0.clone()
        wsb, _ = C.iterate_checkpointed(lw, mw, iters=T, ckpt_every=ck)
        gl, gM = C.lb_seed(lw, mw)
        outs = C.backward_checkpointed(None, None, T, ck, gl, gM, wsb)
        O = oracle.Oracle(tr)
        ol, oM = O.init_lambda()
        ol = np.float32(ol).astype(np.float64)
        lT, MT = O.iterate(ol, oM, 0.5, None, T)
        s1, s2 = O.lb_seed(lT, MT)
        want = O.backward(ol, oM, 0.5, None, T, s1, s2)
        par["adjoint_tracking_12x300_slice"] = {
            nm: _err_stats(C.to_csr(g).double().cpu().numpy(), w)
            for nm, g, w in zip(("g_lambda0", "g_M0"), outs[:2], want[:2])}
        par["adjoint_tracking_12x300_slice"].update({"unrolled_iterations": T, "checkpoint_every": ck})
    return cpu, cpu_all, cpu_matching, par


def run_ours(args):
    import torch

    from paper_2205_11638_gb300 import build, solver

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    prob = WORKLOADS[args.workload]()
    t0 = time.perf_counter()
    plan = solver.plan(prob, block_threads=args.threads, tile_nodes=args.tile_nodes, tile_slots=args.tile_slots)
    A = plan.bind()
    plan_s = time.perf_counter() - t0
    tuned_ms = None
    layout = None
    if not args.no_tune:
        # untimed set-up: the locality chunk and the launch groups' footprint
        # ratio (layout knobs: how rows are ordered into tiles and tiles into
        # launches, never the arithmetic) chosen among a few by timing whole
        # sweep pairs, then the launch shapes
        from paper_2205_11638_gb300 import autotune
        t1 = time.perf_counter()
        del A, plan
        layout, A = autotune.tune(prob, reps=3, chunks=TUNE_CHUNKS, ratios=TUNE_RATIOS, use_cache=False,
                                  block_threads=args.threads, tile_nodes=args.tile_nodes,
                                  tile_slots=args.tile_slots)
        tuned_ms = autotune.tune_launch(A, reps=3)
        layout = dict(layout, tuning_s=round(time.perf_counter() - t1, 1))
    st = A.stats
    Nv, Nl, n = st.sizes.num_nodes, st.sizes.num_lambda, st.sizes.n
    arcs_per_iter = 4 * Nv
    stream = torch.cuda.current_stream()
    lam, M = A.init_lambda()
    lb_out = torch.zeros(A.num_inst, dtype=torch.float64, device=A.device)

    # the steps run as dg_iterate does: every sweep takes the path costs the
    # sweep before it left (except the very first)
    handed = [False]

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        A.sweep(lam, M, forward=True, costs_in=handed[0], costs_out=True)
        if ev is not None:
            ev[1].record(stream)
        A.sum_M(M)
        if ev is not None:
            ev[2].record(stream)
        A.sweep(lam, M, forward=False, energy=True, costs_in=True, costs_out=True)
        if ev is not None:
            ev[3].record(stream)
        A.sum_M(M)
        A.bound_from_energies(lb_out)
        if ev is not None:
            ev[4].record(stream)
        handed[0] = True

    A.sum_M(M)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    for k in range(args.steps):
        step(evs[k])
    torch.cuda.synchronize()
    clk = clocks.stop()
    if ws > 1:
        dist.barrier()
    t_fwd = [e[0].elapsed_time(e[1]) for e in evs]
    t_red = [e[1].elapsed_time(e[2]) for e in evs]
    t_bwd = [e[2].elapsed_time(e[3]) for e in evs]
    t_tail = [e[3].elapsed_time(e[4]) for e in evs]
    total_ms = evs[0][0].elapsed_time(evs[-1][4])

    def _max(x):
        t = torch.tensor([x], device=A.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t[0])

    value, total_ms = aggregate(total_ms, arcs_per_iter * args.steps, ws, _max if ws > 1 else None)
    ms_per_step = total_ms / args.steps

    # roofline of the dominant kernel (the sweep; forward and backward have
    # the same algorithmic bytes): 16 B per node + 16 B per slot per sweep
    sweep_bytes = 16.0 * Nv + 16.0 * Nl
    sweep_ms = statistics.mean(t_fwd + t_bwd)
    peak, peak_src = _peaks()
    achieved = sweep_bytes / (sweep_ms * 1e-3) / 1e9
    src_sha = _kernel_source_sha()
    traffic = _profile_traffic(f"sweep_{args.workload}", src_sha)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_source": peak_src, "kernel": "k_sweep (forward and backward)",
            "algorithmic_bytes_per_launch": sweep_bytes, "avg_launch_ms": sweep_ms,
            "iteration_algorithmic_bytes": st.bytes_per_iter,
            "iteration_frac": st.bytes_per_iter / (ms_per_step * 1e-3) / 1e9 / peak,
            "dram_traffic_frac": (traffic / (sweep_ms * 1e-3) / 1e9 / peak) if traffic else None,
            "kernel_source_sha": src_sha}
    shares = {"k_sweep_fwd": sum(t_fwd), "k_reduce_S": sum(t_red) + 0.0, "k_sweep_bwd": sum(t_bwd),
              "k_reduce_S+k_lb": sum(t_tail)}
    tot = sum(shares.values())
    shares = {k: v / tot for k, v in shares.items()}

    # end to end through the public API with host buffers: every step copies
    # (lambda, M) from pinned host memory, runs one iteration with its bound
    # and reads (lambda, M, bound) back
    e2e = None
    if not args.no_e2e:
        ke = min(args.steps, 10)
        e_ms, serial_ms, host_ms = _e2e_steps(A, lam, M, ke, stream, torch)
        if ws > 1:
            t = torch.tensor([e_ms], device=A.device)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_ms = float(t[0])
        nb = 2 * A.num_slots * 4
        e2e = {"value": arcs_per_iter * ke * ws / (e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb + 8 * A.num_inst,
               "ms_per_step": e_ms / ke, "steps": ke,
               "copies": "state in 4 chunks per vector: each step's upload of a chunk follows the previous step's download of "
                         "it (the host link runs both directions at once), M before lambda (the first S reduction "
                         "needs only M), downloads overlap the last S reduction and the bound",
               "ms_per_step_copies_not_overlapped": serial_ms / ke, "host_enqueue_ms_per_step": host_ms / ke}

    # fwd + adjoint of an unrolled solve (Alg. 1 forward, Alg. 2 backward) on
    # the same instance: with a checkpoint every 10 iterations (segments
    # recomputed as recording sweeps; the forward records the last one), and
    # with one segment (the forward records every sweep: the argmin records
    # of all 2T sweeps stay in HBM and nothing is recomputed).  The headline
    # is the one-segment run when its workspace takes at most half of the
    # free device memory (46.6 GB of the GB300's 280 GB for 100 iterations of
    # the tracking instance), else the checkpointed one; both are reported.
    adjoint = None
    if not args.no_adjoint:
        T = args.adjoint_iters
        free_bytes = torch.cuda.mem_get_info()[0]
        lam0, M0 = A.init_lambda()
        gl = torch.empty_like(lam0)
        gM = torch.empty_like(M0)
        lamw, Mw = lam0.clone(), M0.clone()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        runs = {}
        for ck in (10, T):
            ws_bytes = A.backward_workspace_bytes(T, ck)
            wsb = torch.empty(ws_bytes, dtype=torch.uint8, device=A.device)
            outs = [torch.empty_like(lam0) for _ in range(4)]
            for rep in range(2):  # first repetition warms up
                lamw.copy_(lam0)
                Mw.copy_(M0)
                torch.cuda.synchronize()
                ev[0].record(stream)
                # forward keeping the checkpoints, loss seed, Alg. 2 from the checkpoints
                A.iterate_checkpointed(lamw, Mw, iters=T, ckpt_every=ck, workspace=wsb)
                A.lb_seed_into(lamw, Mw, gl, gM)
                ev[1].record(stream)
                A.backward_checkpointed(None, None, T, ck, gl, gM, wsb, outs)
                ev[2].record(stream)
                torch.cuda.synchronize()
            f_ms, b_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
            runs[ck] = ({"unrolled_iterations": T, "checkpoint_every": ck, "forward_ms": f_ms, "backward_ms": b_ms,
                         "backward_ms_per_unrolled_iteration": b_ms / T,
                         "fwd_adjoint_ms_per_unrolled_step": (f_ms + b_ms) / T, "workspace_bytes": ws_bytes,
                         "loss": "lower bound (eq. 3 plus unary term)"}, outs)
            del wsb
        one_segment = runs[T][0]["workspace_bytes"] <= 0.5 * free_bytes
        adjoint = dict(runs[T][0] if one_segment else runs[10][0])
        adjoint["interval_choice"] = ("one segment: every sweep's argmin records kept in HBM, nothing recomputed "
                                      "(workspace at most half of the free device memory)" if one_segment else
                                      "a checkpoint every 10 iterations (one segment's workspace would exceed half "
                                      "of the free device memory)")
        adjoint["checkpoint_every_10"] = runs[10][0]
        adjoint["records_in_hbm"] = runs[T][0]
        adjoint["gradients_bit_identical_across_intervals"] = bool(
            all(torch.equal(x, y) for x, y in zip(runs[10][1], runs[T][1])))
        del runs

    keep = {}
    if adjoint is not None:
        keep["adjoint"] = True
    batched = None
    if not args.no_batched:
        batched, keep["batched"] = _batched_measurement(args, solver, torch)
    matching_adjoint = None
    if not args.no_adjoint and not args.no_matching:
        matching_adjoint, keep["matching"] = _matching_adjoint_measurement(solver, torch)
    independent_set = None
    if not args.no_is:
        independent_set, keep["independent_set"] = _independent_set_measurement(solver, torch)
    long_rows = None
    if not args.no_long:
        long_rows, keep["long_rows"] = _long_rows_measurement(solver, torch)

    cpu = cpu_all = parity = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu, cpu_all, cpu_matching, parity = _oracle_leg(args, A, prob, solver, torch, keep)
        if matching_adjoint is not None and cpu_matching is not None:
            matching_adjoint["cpu_oracle"] = cpu_matching

    # 2 sweeps x launch groups, 2 S reductions, lb partial, lb final
    launches_per_step = 2 * int(st.sizes.num_launch_groups) + 4
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": args.workload, "n_vars": int(n), "constraints": int(st.sizes.m),
                      "N_lambda": int(Nl), "N_v": int(Nv), "arcs_per_iteration": int(arcs_per_iter),
                      "tiles": int(st.sizes.num_tiles), "launch_groups_per_sweep": int(st.sizes.num_launch_groups),
                      "block_threads": args.threads or 128,
                      "autotuned_sweep_pair_ms": tuned_ms, "layout": layout,
                      "l2": f"inputs larger than L2 (arena {st.sizes.arena_bytes / 1e6:.0f} MB + state "
                            f"{8 * A.num_slots / 1e6:.0f} MB)", "plan_bind_s": round(plan_s, 2),
                      "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
           "roofline": roof, "kernel_shares": shares, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
           "cpu_baseline_all_cores": cpu_all, "parity": parity,
           "adjoint": adjoint, "adjoint_matching": matching_adjoint, "batched": batched,
           "independent_set_10k": independent_set, "long_rows": long_rows,
           "gpu_launches": launches_per_step * args.steps}
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tracking_500x2000", choices=sorted(WORKLOADS))
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--tile-nodes", type=int, default=0)
    ap.add_argument("--tile-slots", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-is", action="store_true")
    ap.add_argument("--no-long", action="store_true")
    ap.add_argument("--no-matching", action="store_true")
    ap.add_argument("--adjoint-iters", type=int, default=100)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
