#!/usr/bin/env python
"""Implicit FE steps/s on GB300: the 350k-DOF Mooney-Rivlin tet beam.

One step = element force/tangent -> gather assembly of A and b -> lagged
LDL^T (A_s snapshot every 5 steps, factored on the side stream, first used k
steps later) -> PCG with FP64 residual refinement to ||r|| <= 1e-8 ||b|| ->
backward Euler.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank steps its own replica of the beam (the path does
not shard: replicas only); rank 0 prints one JSON line.  `value` is
the whole-job steps/s with the per-step loads already resident in HBM;
`e2e` is the same metric through the C ABI with host buffers (host->device
copy of p_t and device->host read of q, v inside the timed region).
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

WORKLOAD = "tet30x30x120-mr"
METRIC = "implicit steps/s (assembly+PCG to 1e-8) at 350k DOF, %HBM roofline; adjoint grads/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _bf16_peak():
    """Dense BF16 tensor peak: the measured sustained bf16 GEMM rate (the
    factor runs inside a long step)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["bf16_tflops_sustained"]), \
            "measured bf16 sustained %.1f TFLOP/s" % float(pk["bf16_tflops_sustained"])
    except Exception:
        return 1700.0, "fallback bf16 sustained 1700 TFLOP/s"


def _tf32_peak():
    """Dense TF32 tensor peak: the measured sustained bf16 GEMM rate (the factor
    runs inside a long step) times the nominal TF32/bf16 ratio 1.1/2.25."""
    ratio = 1.1 / 2.25
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["bf16_tflops_sustained"]) * ratio, \
            "measured bf16 sustained %.1f TFLOP/s x nominal TF32/bf16 1.1/2.25" % float(pk["bf16_tflops_sustained"])
    except Exception:
        return 1700.0 * ratio, "fallback bf16 sustained 1700 TFLOP/s x nominal TF32/bf16 1.1/2.25"


MATERIAL_NAMES = {0: "Saint Venant-Kirchhoff", 1: "neo-Hookean", 2: "Mooney-Rivlin"}

def _source_sha(name):
    """First 16 hex digits of the SHA-256 of a CUDA source file of the package."""
    import hashlib
    path = os.path.join(ROOT, "paper_2306_05893_gb300", "csrc", name)
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _profile_traffic(workload):
    """DRAM bytes per launch from the committed ncu summaries: every line
    'bench-traffic: {json}' under profiles/ names a kernel, the workload it
    is scaled to, the bytes per launch, the capture date and the SHA of the
    source file the kernel was built from.  An entry counts only while that
    source is unchanged (a changed kernel has no traffic figure until it is
    captured again)."""
    out = {}
    pdir = os.path.join(ROOT, "profiles")
    for fn in sorted(os.listdir(pdir)) if os.path.isdir(pdir) else []:
        if not fn.endswith(".md"):
            continue
        with open(os.path.join(pdir, fn)) as f:
            for line in f:
                if not line.startswith("bench-traffic:"):
                    continue
                try:
                    e = json.loads(line.split(":", 1)[1])
                except ValueError:
                    continue
                if e.get("workload") != workload:
                    continue
                try:
                    if _source_sha(e["source"]) != e["source_sha16"]:
                        continue
                except OSError:
                    continue
                e["profile"] = "profiles/" + fn
                out[e["kernel"]] = e
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

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
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1", "0x1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- oracle arm

def oracle_step(wl, t=0, q=None, v=None):
    """One full step of the FP64 oracle, as it stands, on the whole workload:
    element force and tangent, triplet assembly, A and b, then its Jacobi CG
    solve (cg_solve) to the workload's tolerance ||b - A a|| <= tol ||b||
    and backward Euler: the CPU analogue of fast assembly + CG.  (The
    oracle's direct solve does not finish in minutes at 350k DOF.)  The
    model's setup (mass, rest data) is not timed.  Returns (seconds, CG
    iterations, threads used = CPU time / wall time, q+, v+)."""
    from oracle import fe_oracle as O
    om = O.Model.from_workload(wl)
    if q is None:
        q = wl.mesh.X.reshape(-1).copy()
        v = np.zeros_like(q)
    t0, c0 = time.perf_counter(), time.process_time()
    q1, v1, _, its = om.step_cg(q, v, wl.p(t).reshape(-1), wl.tol)
    el = time.perf_counter() - t0
    return el, its, (time.process_time() - c0) / el, q1, v1


def cpu_baseline(wl):
    el, its, thr, _, _ = oracle_step(wl)
    return {"value": 1.0 / el, "unit": "steps/s", "cores": max(1, int(round(thr))), "kind": "oracle",
            "sample": f"one full FP64 oracle step of {wl.name} (all {wl.mesh.n_elems} elements, "
                      f"{3 * wl.mesh.n_nodes} DOF): element force+tangent, triplet assembly, Jacobi CG "
                      f"to {wl.tol:g} ({its} iterations), integration; measured, not extrapolated; "
                      f"{el:.1f} s wall, {thr:.2f} threads busy on average"}


def run_reference(args, rank):
    """The oracle arm: full oracle steps of the workload, at most 2 (each
    about a minute of host CPU), timed one after the other from the rest
    state; `steps` is the number actually run."""
    if rank != 0:
        return
    import fe_inputs as fi
    wl = fi.workload(WORKLOAD)
    steps = max(1, min(args.steps, 2))
    q = v = None
    times, its, thr = [], [], []
    for t in range(steps):
        el, it, th, q, v = oracle_step(wl, t, q, v)
        times.append(el)
        its.append(it)
        thr.append(th)
    tot = sum(times)
    value = steps / tot
    cores = max(1, int(round(float(np.mean(thr)))))
    out = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
           "steps": steps, "warmup": 0, "ms_per_step": 1e3 * tot / steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "precision": "fp64 oracle (Jacobi CG to the workload tolerance)",
                      "cg_iterations": its},
           "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cores, "kind": "oracle",
                            "sample": f"{steps} full oracle steps of {WORKLOAD} from rest "
                                      f"({', '.join('%.1f s' % x for x in times)}); CG iterations {its}"},
           "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------- side metrics

def measure_adjoint(fe, torch, T=20):
    """grads/s of the adjoint workload: hex 20x20x80 neo-Hookean beam with a
    per-element log-normal Young's modulus (median 1e4, sigma 0.3, seed 11),
    L = 1/2 ||q_T - q*||^2 after T steps; one gradient = forward rollout with
    checkpoints + reverse adjoint sweep.  Measured in the mixed path (2
    gradients) and in FP64 (1 gradient), after one untimed gradient each."""
    import fe_inputs as fi
    mesh = fi.hex_beam(20, 20, 80, jitter=0.1, seed=1)
    nu = 3.1e4 / (2 * (3.1e4 + 3.4e3))
    base = np.array([*fi.lame_from_young(1.0, nu), 0.0])
    E = fi.lognormal_modulus(mesh.n_elems, seed=11)
    trac = fi.end_traction(mesh, (50.0, 0.0, 0.0)).reshape(-1)
    q0 = mesh.X.reshape(-1).copy()
    qt = q0 + 1e-4
    out = {"unit": "grads/s", "workload": "hex20x20x80-nh per-element E, T=20", "n_dof": 3 * mesh.n_nodes}
    for prec, reps in ((1, 2), (0, 1)):
        ctx = fe.FEContext(mesh.elem_type, mesh.X, mesh.conn, mesh.fixed_nodes, fi.NEOHOOKE, 1000.0,
                           E[:, None] * base[None, :], 0.01, 0.1, 0.01, precision=prec, refactor_every=5,
                           keep_checkpoints=1)
        q = np.empty(ctx.n)
        v = np.empty(ctx.n)

        def one():
            ctx.set_state(q0, np.zeros_like(q0))
            ctx.clear_checkpoints()
            for _ in range(T):
                ctx.step(trac, q, v)
            ds, _ = ctx.adjoint(q - qt, with_dp=False)
            return ds

        one()  # warm-up (factor buffers, first-call setup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            one()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        ctx.close()
        key = "mixed" if prec else "fp64"
        out[key] = {"value": reps / el, "s_per_grad": el / reps, "grads_timed": reps}
    out["value"] = out["mixed"]["value"]
    out["precision"] = "mixed (fp64 alongside)"
    return out


def run_contact(args, world, rank, local, torch, dist):
    """Contact workload (NEXT-3): the 107,163-DOF Mooney-Rivlin tet beam
    (tet20x20x80-mr) with its free end moving down onto a rigid floor 2 mm
    below its bottom face; 63 frictionless contacts (the bottom-face nodes
    of the last three node layers at the free end), exact factor every step
    (refactor_every = 1: the compliance is built with A^{-1}).  Replicas
    only for N > 1 (no data-path collective)."""
    import fe_inputs as fi
    import paper_2306_05893_gb300 as fe
    wl = fi.workload("tet20x20x80-mr")
    mesh = wl.mesh
    ctx = fe.FEContext.from_workload(wl, refactor_every=1, profile_stages=1,
                                     precond_fp16=args.precond_fp16)
    n = ctx.n
    q0 = mesh.X.reshape(-1).copy()
    v0 = np.zeros_like(q0)
    v0.reshape(-1, 3)[:, 2] = -0.5 * mesh.X[:, 0] / mesh.X[:, 0].max()
    fixed = (3 * mesh.fixed_nodes[:, None] + np.arange(3)).reshape(-1)
    v0[fixed] = 0.0
    xmax = mesh.X[:, 0].max()
    nodes = np.nonzero((mesh.X[:, 2] == 0.0) & (mesh.X[:, 0] >= xmax - 2 * 0.01 - 1e-12))[0].astype(np.int32)
    ctx.set_state(q0, v0)
    ctx.set_contacts(nodes, np.tile([0.0, 0.0, 1.0], (len(nodes), 1)), np.full(len(nodes), -0.002))
    q = np.empty(n)
    p = [wl.p(t).reshape(-1) for t in range(args.warmup + args.steps)]
    for t in range(args.warmup):
        ctx.step(p[t], q, None)
    ctx.reset_stage_times()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    active = []
    for t in range(args.steps):
        ctx.step(p[args.warmup + t], q, None)
        active.append(int((ctx.contact_forces() > 0).sum()))
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    if world > 1:
        tt = torch.tensor([el], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        el = float(tt.item())
    stage_ms, stage_calls, _ = ctx.stage_times()
    gap = q.reshape(-1, 3)[nodes, 2] + 0.002
    ctx.close()
    out = {"metric": "implicit steps/s with frictionless contacts (free motion + compliance + PGS + correction)",
           "value": world * args.steps / el, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "contact: tet20x20x80-mr onto a floor, 63 contacts, R = 1",
                      "n_dof": n, "contacts": int(len(nodes)), "mean_active": float(np.mean(active)),
                      "min_gap_m": float(gap.min()),
                      "parallelism": "replicas" if world > 1 else "single"},
           "stages_ms_per_step": {k: v / args.steps for k, v in stage_ms.items()},
           "contact_ms_per_step": stage_ms["contact"] / args.steps}
    if rank == 0:
        print(json.dumps(out), flush=True)


def _batch_context(fe, fi, members, graph):
    """The batched workload's context: the given members of the 64 uneven tet
    beams (seed 7), mixed precision, R = 5, tol 1e-8; the solve as one graph
    with device-side loops (graph = 1) or host-driven."""
    return fe.FEBatch([(m.mesh.elem_type, m.mesh.X, m.mesh.conn, m.mesh.fixed_nodes, m.model, m.params)
                       for m in members], 0.01, 0.1, 0.01, 1000.0, precision=1, refactor_every=5, tol=1e-8,
                      use_graph=graph)


def measure_batch(fe, torch, steps=10, warmup=3, graph=1):
    """Aggregate DOF*steps/s of the batched workload on this GPU: all 64
    members in one context, loads in HBM, CUDA events around the steps."""
    import fe_inputs as fi
    mem = fi.batch_workload(64, seed=7)
    b = _batch_context(fe, fi, mem, graph)
    pn = np.concatenate([mem[k].load.reshape(-1) for k in b.member])   # stored member order
    qn = np.empty(b.n)
    for _ in range(warmup):
        b.step(pn)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    its = []
    for _ in range(steps):
        its.append(b.step(pn, qn).iters)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    ndof = b.n
    b.close()
    return {"value": ndof * steps / (ms / 1e3), "unit": "DOF*steps/s", "steps_per_s": steps / (ms / 1e3),
            "ms_per_step": ms / steps, "steps": steps, "warmup": warmup, "members": len(mem), "total_dof": ndof,
            "max_pcg_iters": its, "solve": "one graph per step (device-side convergence)" if graph else "host-driven",
            "workload": "batch64-tet (seed 7, 2k-40k DOF each, a tenth of gravity: under full gravity the most "
                        "slender, softest members fold through themselves within 25 steps), mixed, R = 5, tol 1e-8",
            "timer": "CUDA events around the steps (host load and state buffers)"}


def run_batch(args, world, rank, local, torch, dist):
    """Batched workload: 64 uneven tet beams (seed 7) stepped together; members
    sharded over ranks by DOF (no collective on the data path)."""
    import fe_inputs as fi
    import paper_2306_05893_gb300 as fe
    from paper_2306_05893_gb300.sharding import shard_members
    mem = fi.batch_workload(64, seed=7)
    mine = shard_members([3 * m.mesh.n_nodes for m in mem], world)[rank]
    b = _batch_context(fe, fi, [mem[k] for k in mine], args.graph)
    # loads concatenated in the batch's stored member order
    p = np.concatenate([mem[mine[k]].load.reshape(-1) for k in b.member])
    q = np.empty(b.n)
    v = np.empty(b.n)
    for _ in range(args.warmup):
        b.step(p, q, v)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        b.step(p, q, v)
    ev1.record()
    torch.cuda.synchronize()
    el = ev0.elapsed_time(ev1) / 1e3
    if world > 1:
        tt = torch.tensor([el], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        el = float(tt.item())
    ndof_all = sum(3 * m.mesh.n_nodes for m in mem) if world == 1 else None
    dofs_mine = b.n
    if world > 1:
        t = torch.tensor([float(dofs_mine)], device="cuda")
        dist.all_reduce(t)
        ndof_all = float(t.item())
    out = {"metric": "aggregate DOF*steps/s, batched tet beams", "value": ndof_all * args.steps / el,
           "unit": "DOF*steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "batch64-tet (seed 7, 2k-40k DOF each)", "members": len(mem),
                      "total_dof": ndof_all, "steps_per_s_per_beam": args.steps / el,
                      "solve": "one graph per step" if args.graph else "host-driven",
                      "parallelism": f"members sharded over {world} ranks" if world > 1 else "single"}}
    b.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


# --------------------------------------------------------------------- ours

def _ctx_for(fe, wl, args, **kw):
    """The workload's context with the bench's options (kw overrides them)."""
    opts = dict(nd_leaf_nodes=args.nd_leaf, use_graph=1 if args.graph else 0,
                factor_tf32=1 if args.factor_tf32 else 0,
                precond_fp16=args.precond_fp16 if wl.precision else 0,
                factor_lag=args.lag, element_fp64=1 if args.element_fp64 else 0,
                warm_start=args.warm, apply_sm_share=args.apply_share,
                update_bf16=args.update_bf16 if wl.precision else 0)
    if args.inner_tol:
        opts["inner_tol"] = args.inner_tol
    opts.update(kw)
    return fe.FEContext.from_workload(wl, **opts)


def oracle_position_error(fe, args, **kw):
    """Positions after 10 steps from rest of the bench workload in the given
    configuration against the FP64 oracle's rollout of the same steps
    (tests/golden/tet30x30x120_mr_rollout.json, written by the oracle), on the
    stored DOF sample, relative to the oracle's displacement there."""
    import fe_inputs as fi
    path = os.path.join(ROOT, "tests", "golden", "tet30x30x120_mr_rollout.json")
    with open(path) as f:
        g = json.load(f)
    wl = fi.workload(g["workload"])
    ctx = _ctx_for(fe, wl, args, use_graph=0, **kw)
    q = np.empty(ctx.n)
    for t in range(g["steps"]):
        ctx.step(wl.p(t).reshape(-1), q, None)
    ctx.close()
    S = np.asarray(g["dofs"])
    X = wl.mesh.X.reshape(-1)[S]
    qo = np.asarray(g["q"])
    return float(np.linalg.norm(q[S] - qo) / np.linalg.norm(qo - X))


def measure_variant(fe, torch, wl_name, args, steps, warmup, **kw):
    """steps/s of one more configuration (same timing as the headline: loads
    in HBM, CUDA events around the steps on the caller's stream)."""
    import fe_inputs as fi
    wl = fi.workload(wl_name)
    if "precision" in kw:
        wl.precision = kw.pop("precision")
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(priority=-1)
    ctx = _ctx_for(fe, wl, args, device_ptrs=1, stream=stream.cuda_stream, **kw)
    loads = torch.tensor(np.stack([wl.p(t).reshape(-1) for t in range(warmup + steps)]), dtype=torch.float64,
                         device=dev)
    q = torch.empty(ctx.n, dtype=torch.float64, device=dev)
    its = []
    with torch.cuda.stream(stream):
        for t in range(warmup):
            ctx.step(loads[t], q, None)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for t in range(warmup, warmup + steps):
            its.append(ctx.step(loads[t], q, None).iters)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    ctx.close()
    return {"value": steps / (ms / 1e3), "unit": "steps/s", "ms_per_step": ms / steps, "steps": steps,
            "warmup": warmup, "mean_pcg_iters": float(np.mean(its)), "workload": wl_name,
            "precision": "mixed" if wl.precision else "fp64",
            "element_fp64": bool(kw.get("element_fp64", 0))}


def _streaming_rooflines(wl, info, stage_ms, stage_calls, hbm, peak_kind, args, traffic):
    """Achieved HBM bandwidth of the streaming kernels from their algorithmic
    bytes per launch (the units each launch processes times the bytes per
    unit) and their average live launch time (CUDA events on the stream that
    runs them)."""
    n, nnz, E = info["n"], info["nnz"], wl.mesh.n_elems
    npe = 4 if wl.mesh.elem_type == 0 else 8
    mixed = bool(wl.precision)
    kb = 4 if (mixed and not args.element_fp64) else 8     # stored tangent entry
    ab = 4 if mixed else 8                                 # inner matrix / vector entry
    kept, nblk = info["ntrip_kept"], info["n_blocks"]
    nodes = wl.mesh.n_nodes
    rest = (10 if npe == 4 else 200) * 8
    df_force = mixed and not args.element_fp64
    bytes_ = {
        # per element: K_e and f_e out (f_e as FP64 or as float pairs, 8 B
        # either way), rest data + 3 parameters (doubles or float pairs) +
        # connectivity in; per node: q and X, or the float pairs of q - X
        "element": E * ((3 * npe) ** 2 * kb + 3 * npe * 8 + rest + 24 + 4 * npe) + nodes * (24 if df_force else 48),
        # per gathered triplet its K_e value; per block its source list entry
        # (kept / 9 of them), bsrc_ptr, column and mass; per slot A (and its
        # float-pair copy in the mixed path); per element its forces and
        # incidence; per row rowptr and v, p, b
        "assembly": kept * kb + (kept // 9) * 4 + nblk * 16 + nnz * (ab + (8 if mixed else 0))
        + E * (3 * npe * 8 + 4 * npe) + n * (4 + 24) + nodes * 8,
        "spmv": nnz * (ab + 4) + (n + 1) * 4 + 2 * n * ab,
        "residual": nnz * (8 + 4) + (n + 1) * 4 + 3 * n * 8,
    }
    yb = 2 if (mixed and args.precond_fp16) else ab
    bytes_["apply"] = 2 * info["y_nnz"] * yb + 6 * info["n_free"] * ab + 2 * n * ab
    # the SpMV and the residual run the variant the per-context autotuner
    # chose (node-block or CSR); their bytes are the CSR product's
    kern = {"element": "tet_kernel" if npe == 4 else "hex_kernel", "assembly": "assemble_block_kernel",
            "spmv": "bspmv_kernel / spmv_dot_kernel",
            "residual": ("bres_df_kernel / residual_df_kernel" if mixed else "bspmv_kernel / residual_kernel"),
            "apply": "fwd_kernel + bwd_kernel"}
    out = {}
    for k, b in bytes_.items():
        calls = stage_calls.get(k, 0)
        if not calls:
            continue
        ms = stage_ms[k] / calls
        gbs = b / (ms / 1e3) / 1e9 if ms > 0 else None
        tr = traffic.get(kern[k])
        out[k] = {"kernel": kern[k], "bytes_per_launch": int(b), "avg_ms": ms, "achieved": gbs, "peak": hbm,
                  "peak_kind": peak_kind, "unit": "GB/s", "frac": gbs / hbm if gbs else None,
                  "traffic": tr["bytes_per_launch"] if tr else None,
                  "traffic_source": f"{tr['profile']} ({tr['date']})" if tr else None}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP64-tangent and hex mixed-vs-FP64 measurements")
    ap.add_argument("--lag", type=int, default=1,
                    help="factor_lag k: the factor of A_s first preconditions step s+k")
    ap.add_argument("--element-fp64", action="store_true",
                    help="mixed precision with FP64 element tangents (the FP64 system exactly)")
    ap.add_argument("--factor-tf32", action="store_true",
                    help="mixed precision: plain TF32 products in the factor's trailing updates")
    ap.add_argument("--precond-fp16", type=int, default=1, choices=[0, 1],
                    help="mixed precision: the preconditioner applies a binary16 copy of Y")
    ap.add_argument("--graph", type=int, default=1, choices=[0, 1],
                    help="1: each step's solve and integration as one CUDA graph with device-side loops "
                         "(fe_options.use_graph); 0: host-driven PCG")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="mixed precision: the inner FP32 PCG's tolerance per refinement sweep "
                         "(fe_options.inner_tol; 0: the library default 1e-4)")
    ap.add_argument("--update-bf16", type=int, choices=[0, 1], default=1,
                    help="mixed precision: the superpanels' deferred factor updates with BF16 "
                         "operands on the tensor cores (fe_options.update_bf16)")
    ap.add_argument("--apply-share", type=float, default=0.5,
                    help="fraction of the application's CTA slots left to an in-flight factorisation")
    ap.add_argument("--warm", type=int, default=0, choices=[0, 1],
                    help="1: each step's PCG starts from the previous step's acceleration (fe_options.warm_start)")
    ap.add_argument("--nd-leaf", type=int, default=0,
                    help="nested-dissection leaf size in nodes (0: the library default)")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default=None,
                    help="override the workload's precision (default: the workload's own)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    args.warmup = max(3, args.warmup)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2306_05893_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    import fe_inputs as fi
    import paper_2306_05893_gb300 as fe

    if args.workload == "batch64":
        return run_batch(args, world, rank, local, torch, dist)
    if args.workload == "contact":
        return run_contact(args, world, rank, local, torch, dist)
    wl = fi.workload(args.workload)
    if args.precision is not None:
        wl.precision = 1 if args.precision == "mixed" else 0
    args.lag = max(1, min(args.lag, wl.refactor_every))
    K, W = args.steps, args.warmup
    stream = torch.cuda.Stream(priority=-1)  # above the library's background factor stream
    dev = torch.device("cuda", local)
    ctx = _ctx_for(fe, wl, args, device_ptrs=1, stream=stream.cuda_stream, profile_stages=1)
    info = ctx.info()
    n = ctx.n
    loads = torch.tensor(np.stack([wl.p(t).reshape(-1) for t in range(W + K)]), dtype=torch.float64,
                         device=dev)
    q_out = torch.empty(n, dtype=torch.float64, device=dev)
    v_out = torch.empty(n, dtype=torch.float64, device=dev)
    iters, ages, refs = [], [], []
    with torch.cuda.stream(stream):
        for t in range(W):
            ctx.step(loads[t], q_out, v_out)
        torch.cuda.synchronize()
        ctx.reset_stage_times()
        sampler = ClockSampler(local)
        sampler.start()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for t in range(W, W + K):
            si = ctx.step(loads[t], q_out, v_out)
            iters.append(si.iters)
            ages.append(si.factor_age)
            refs.append(si.refinements)
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    stage_ms, stage_calls, launches = ctx.stage_times()
    update_flops = ctx.update_flops()
    update_bf16_flops = ctx.update_bf16_flops()
    update_bf16_tiles = ctx.update_bf16_tiles()
    main_sum = sum(stage_ms[k] for k in ("element", "assembly", "apply", "spmv", "vector", "residual",
                                         "integrate", "pcg_graph")) / K
    timed_stages = {k: v / K for k, v in stage_ms.items()}
    if world > 1:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    value = world * K / (ms / 1e3)
    disp = float((q_out - torch.tensor(wl.mesh.X.reshape(-1), device=dev)).abs().max())
    ctx.close()
    del loads

    # end to end through the C ABI with host buffers: the same steps W .. W+K-1
    # after the same warm-up, with the same stage instrumentation
    e2e = None
    if not args.no_e2e:
        ctx2 = _ctx_for(fe, wl, args, device_ptrs=0, profile_stages=1)
        qh = np.empty(n)
        vh = np.empty(n)
        its2 = []
        for t in range(W):
            ctx2.step(wl.p(t).reshape(-1), qh, vh)
        host_loads = [np.ascontiguousarray(wl.p(t).reshape(-1)) for t in range(W, W + K)]
        torch.cuda.synchronize()
        ctx2.reset_stage_times()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for pl in host_loads:
            its2.append(ctx2.step(pl, qh, vh))
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        ctx2.close()
        scal_reads = sum(i.iters + i.refinements + 1 for i in its2) / len(its2)
        if world > 1:
            tt = torch.tensor([el], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            el = float(tt.item())
        e2e = {"value": world * K / el, "unit": "steps/s", "steps": K, "timer": "host clock",
               "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": int(16 * n + 144 * scal_reads)}

    # roofline of the dominant kernel by share of the launch list: the
    # factor's trailing-update launches (tensor cores, 3xTF32)
    hbm, peak_kind = _peaks()
    tf32_peak, tf32_src = _tf32_peak()
    traffic = _profile_traffic(args.workload)
    upd_calls = max(1, stage_calls["factor_update"])
    upd_ms = stage_ms["factor_update"] / upd_calls
    upd_flops = update_flops / upd_calls
    upd_tflops = upd_flops / (upd_ms / 1e3) / 1e12 if upd_ms > 0 else 0.0
    tr = traffic.get("front_update_tc_kernel")
    tc_roof = {"bound": "tensor",
               "kernel": "front_update_tc_kernel (factor trailing updates, tcgen05 kind::tf32, "
                         + ("TF32" if args.factor_tf32 else "3xTF32") + ")",
               "achieved": upd_tflops, "peak": tf32_peak, "unit": "TFLOP/s", "frac": upd_tflops / tf32_peak,
               "traffic": tr["bytes_per_launch"] if tr else None,
               "traffic_source": f"{tr['profile']} ({tr['date']})" if tr else None,
               "flops_per_launch": upd_flops, "avg_ms": upd_ms, "launches": upd_calls,
               "peak_source": tf32_src,
               "note": "achieved counts algorithmic flops; 3xTF32 issues 3 TF32 MMAs per product, "
                       "so frac <= 1/3; the update launches run on the low-priority factor stream"}
    if wl.precision and args.update_bf16:
        # the superpanels' deferred updates (the bulk of the factor's flops) in
        # the BF16 kernel; the remaining (eager, in-superpanel) updates above
        bf_peak, bf_src = _bf16_peak()
        bcalls = max(1, stage_calls["factor_update_bf16"])
        bms = stage_ms["factor_update_bf16"] / bcalls
        bflops = update_bf16_flops / bcalls
        btf = bflops / (bms / 1e3) / 1e12 if bms > 0 else 0.0
        tb = traffic.get("front_update_bf16_kernel")
        tc_roof["kernel"] = "front_update_tc_kernel (eager in-superpanel updates, tcgen05 kind::tf32, " + \
            ("TF32" if args.factor_tf32 else "3xTF32") + ")"
        roofline = {"bound": "tensor",
                    "kernel": "front_update_bf16_kernel (superpanel trailing updates, TMA + tcgen05 kind::f16, "
                              "BF16 operands, FP32 accumulation)",
                    "achieved": btf, "peak": bf_peak, "unit": "TFLOP/s", "frac": btf / bf_peak,
                    "traffic": tb["bytes_per_launch"] if tb else None,
                    "traffic_source": f"{tb['profile']} ({tb['date']})" if tb else None,
                    "flops_per_launch": bflops, "avg_ms": bms, "launches": bcalls,
                    "peak_source": bf_src,
                    "note": "achieved counts algorithmic flops (lower triangle of the Schur updates plus the "
                            "apply-operator updates); launched on the low-priority factor stream, timed live "
                            "with CUDA events there",
                    "eager_updates": tc_roof}
        # the same launches against HBM: each output tile of F or Y is read
        # and written once by its reduce-add (the BF16 operands come from L2)
        tbytes = update_bf16_tiles / bcalls * 128 * 128 * 4 * 2
        tgbs = tbytes / (bms / 1e3) / 1e9 if bms > 0 else 0.0
        roofline["hbm_view"] = {"bytes_per_launch": int(tbytes), "achieved": tgbs, "peak": hbm, "unit": "GB/s",
                                "frac": tgbs / hbm,
                                "note": "output-tile read-modify-write only (128 KB per 128x128 FP32 tile)"}
    elif wl.precision:
        roofline = tc_roof
    else:
        roofline = {"bound": "alu", "kernel": "front_update_kernel<double> (factor trailing updates, FP64)",
                    "achieved": upd_tflops, "peak": 1.25, "unit": "TFLOP/s", "frac": upd_tflops / 1.25,
                    "traffic": None, "flops_per_launch": upd_flops, "avg_ms": upd_ms, "launches": upd_calls,
                    "peak_source": "nominal GB300 FP64 rate (no measured FP64 peak on this pool)"}
    breakdown_note = "stage times of the timed run"
    if args.graph:
        # inside the step graph the solve's kernels are one timed stage; their
        # individual times come from a host-driven run of the same steps
        # (same kernels and order, not timed for the headline)
        ctx3 = _ctx_for(fe, wl, args, device_ptrs=1, stream=stream.cuda_stream, profile_stages=1, use_graph=0)
        loads3 = torch.tensor(np.stack([wl.p(t).reshape(-1) for t in range(W + K)]), dtype=torch.float64,
                              device=dev)
        with torch.cuda.stream(stream):
            for t in range(W):
                ctx3.step(loads3[t], q_out, v_out)
            torch.cuda.synchronize()
            ctx3.reset_stage_times()
            for t in range(W, W + K):
                ctx3.step(loads3[t], q_out, v_out)
            torch.cuda.synchronize()
        bd_ms, bd_calls, _ = ctx3.stage_times()
        ctx3.close()
        del loads3
        for k in ("apply", "spmv", "vector", "residual", "integrate"):
            stage_ms[k], stage_calls[k] = bd_ms[k], bd_calls[k]
        breakdown_note = ("element, assembly and factor stages from the timed (graph) run; apply, spmv, vector, "
                          "residual and integrate from a host-driven run of the same steps")
    streaming = _streaming_rooflines(wl, info, stage_ms, stage_calls, hbm, peak_kind, args, traffic)
    # the dominant kernel by share of the serialised launch list: with the BF16
    # factor updates the preconditioner application (one forward and one
    # backward launch per PCG iteration), HBM-bound; the factor's tensor-core
    # kernel follows as roofline_tensor
    roofline_tensor = roofline
    if wl.precision and args.update_bf16 and "apply" in streaming:
        a = streaming["apply"]
        roofline = {"bound": "hbm", "kernel": "fwd_kernel + bwd_kernel (one preconditioner application)",
                    "achieved": a["achieved"], "peak": a["peak"], "unit": "GB/s", "frac": a["frac"],
                    "traffic": a["traffic"], "traffic_source": a["traffic_source"],
                    "bytes_per_launch": a["bytes_per_launch"], "avg_ms": a["avg_ms"],
                    "launches": stage_calls.get("apply", 0),
                    "peak_source": "measured copy bandwidth (%s)" % peak_kind,
                    "dominant_by": "share of the serialised launch list (profiles/launches_tet30x30x120-mr.md)",
                    "note": "algorithmic bytes: both sweeps read every stored entry of the binary16 apply "
                            "operators once, plus the vectors; timed with CUDA events on the main stream in a "
                            "host-driven run of the same steps (inside the step graph the application runs in "
                            "device-side loops)"}
    out = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if wl.precision else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n_dof": n, "elements": wl.mesh.n_elems,
                   "nnz": info["nnz"], "material": MATERIAL_NAMES[wl.model],
                   "precision": "mixed" if wl.precision else "fp64",
                   "element_fp64": bool(args.element_fp64),
                   "refactor_every": wl.refactor_every, "factor_lag": args.lag, "tol": wl.tol,
                   "l2": "inputs larger than L2 (apply operators %.2f GB)" % (info["y_nnz"] * 4 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single", "nd_leaf_nodes": args.nd_leaf or 64,
                   "pcg_graph": bool(args.graph), "warm_start": bool(args.warm),
                   "apply_sm_share": args.apply_share,
                   "update_bf16": bool(args.update_bf16),
                   "inner_tol": args.inner_tol or 1e-4,
                   "factor_tf32": bool(args.factor_tf32),
                   "precond_fp16": bool(wl.precision and args.precond_fp16),
                   "mean_pcg_iters": float(np.mean(iters)), "pcg_iters": iters, "factor_ages": ages,
                   "refinements": refs, "max_displacement_m": disp},
        "roofline": roofline,
        "roofline_tensor": roofline_tensor,
        "roofline_streaming": streaming,
        "stage_breakdown": breakdown_note,
        "stages_ms_per_step": timed_stages,
        "main_stream_stage_sum_ms": main_sum,
        "stage_calls": stage_calls,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "e2e": e2e,
    }
    if rank == 0 and not args.no_variants and args.workload == WORKLOAD and wl.precision and not args.element_fp64:
        # the same workload with FP64 element tangents: the configuration whose
        # positions follow the FP64 oracle to 1e-8; both configurations' error
        # after 10 steps against the oracle's stored rollout is measured here
        out["oracle_matching"] = measure_variant(fe, torch, WORKLOAD, args, K, W, element_fp64=1)
        out["oracle_matching"]["position_error_10_steps"] = oracle_position_error(fe, args, element_fp64=1)
        out["config"]["position_error_10_steps"] = oracle_position_error(fe, args)
        # the hex beam (107,163 DOF, neo-Hookean): mixed with FP64 tangents vs
        # FP64, both refined to 1e-8 on the FP64 system (equal accuracy)
        mixed = measure_variant(fe, torch, "hex20x20x80-nh", args, 20, 5, precision=1, element_fp64=1)
        fp64 = measure_variant(fe, torch, "hex20x20x80-nh", args, 10, 3, precision=0)
        out["mixed_vs_fp64_hex20x20x80"] = {"mixed_fp64_tangents": mixed, "fp64": fp64,
                                            "speedup": mixed["value"] / fp64["value"]}
    if rank == 0 and not args.no_adjoint and args.workload == WORKLOAD:
        out["adjoint"] = measure_adjoint(fe, torch)
    if rank == 0 and not args.no_batch and args.workload == WORKLOAD:
        out["batch"] = measure_batch(fe, torch, graph=args.graph)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
