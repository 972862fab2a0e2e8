"""Benchmark: incremental elastoplastic load path on one GB300 through the C ABI.

A step is one whole load path of the workload from the virgin state (ep_reset,
then every load step: semismooth Newton to the relative residual tolerance --
each iteration fused return mapping + tangent assembly + internal forces,
residual and norms, preconditioned Krylov solve, update -- and the state
commit).  The default workload is the P2 plane-strain Drucker-Prager column
(256 x 256 cells, 917 504 points, 40 load steps to 0.98 of the limit
traction), so every path crosses the elastic, the spreading-plastic and the
nearly-singular fully plastic range: at the last step the nonassociated
tangent is indefinite on local plastic-flow modes, GMRES with the V-cycle
stalls, and the solver switches to its sparse LU (one factorisation per
Newton iteration).  W warm-up paths, then K timed paths in each precision,
CUDA events around each path on the context's stream.

value = integration points assembled per second over the timed region
        (n_int x assemblies / elapsed): the rate at which the solver drives
        every integration point through return mapping + tangent assembly,
        Krylov and update included, for the primary precision.  Both
        precisions are timed on the same path: fp64 and mixed (FP32 tangent
        and inner Krylov while they contract well, FP64 return mapping,
        residual and update); with --precision auto (default) the faster is
        the primary and the other is reported under "compare".  load_path_s
        is the median of the K measured path times.
roofline: the kernel with the largest share of the step among the assembly,
        the SpMV of the Krylov solves, the AMG level-0 Chebyshev step and the
        sparse LU's factorisation and solve (CUDA events around every
        assembly, SpMV, factorisation and solve and around a sample of the
        smoothing sweeps, in one instrumented path after the timed region),
        algorithmic bytes (FLOPs for the factorisation) per launch over the
        average launch time; all of them under roofline_kernels.
e2e:    the same metric through the C ABI with host buffers: each path takes
        its load factors from the host and reads u and sigma back to host
        buffers.

--impl reference times the CPU oracle (numpy/scipy, FP64) on a reduced copy
of the workload instead; it is a deliberately slow baseline, not the target.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tangent assembly Gpts/s & load-path time at 1e-10 resid: mixed vs FP64 GPU"
UNIT = "Gpts/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# FP64 FMA pipe of a GB300: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 FMA of a GB300: 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FMAs per row of one training pass of the warm-start network (forward 16*128 + 128*128 + 128*4; backward
# dW3 + dH2 + dW2 + dH1 + dW1)
MLP_FMA_FWD = 16 * 128 + 128 * 128 + 128 * 4
MLP_FMA_TRAIN = MLP_FMA_FWD + 512 + 512 + 128 * 128 + 128 * 128 + 16 * 128


def _workload(name: str, full: bool = True, n: int = 0):
    from synthetic import problems as P
    if n:
        if name == "l_shape_vm":
            return P.l_shape_vm("Q2", m=n)
        return {"p2_plane_dp": P.p2_plane_dp, "p1_plane_vm": P.p1_plane_vm, "q1_cube_vm": P.q1_cube_vm,
                "p2_tet_strip_dp": P.p2_tet_strip_dp}[name](n=n)
    if name == "p2_plane_dp":
        return P.p2_plane_dp() if full else P.p2_plane_dp(n=64)
    if name == "p1_plane_vm":
        return P.p1_plane_vm()
    if name == "q1_cube_vm":
        return P.q1_cube_vm() if full else P.q1_cube_vm(n=16)
    if name == "p2_tet_strip_dp":
        return P.p2_tet_strip_dp() if full else P.p2_tet_strip_dp(n=12)
    if name == "l_shape_vm":
        return P.l_shape_vm("Q2", m=40) if full else P.l_shape_vm("Q2", m=10)
    raise SystemExit(f"unknown workload {name}")


def _workload_config(name, prob, extra=None):
    m = prob.mesh
    cfg = {"workload": f"{name}: {m.elem_type} {m.dim}D {'x'.join(map(str, m.shape))} cells, "
                       f"{m.n_elem} elements, {prob.n_dof} DOFs, {len(prob.zeta)} load steps",
           "n_int": None, "newton_rtol": prob.newton_rtol,
           "l2": "inputs larger than L2 (129 MB): K alone is " + f"{m.n_nodes} node rows"}
    if extra:
        cfg.update(extra)
    return cfg


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM bytes of the FP64 plane SpMV (k_spmv<2, 2, double>) per 2x2 block, from one ncu capture of
# the current kernel on the 320 x 320 P2 column (dram__bytes_read.sum + dram__bytes_write.sum =
# 209 646 080 + 8 653 568 B for 4 715 521 blocks; profiles/k_spmv_fp64_p2_plane_dp_n320.md);
# the traffic grows with the blocks, so the bench scales it to the run's pattern.
SPMV64_2D_DRAM_BYTES_PER_BLOCK = (209646080 + 8653568) / 4715521
# DRAM bytes of a level-0 Chebyshev step that reads the matrix (k_cheb<2, 4, float>), per 2x2 block,
# from one ncu capture on the 320 x 320 P2 column (mean of two launches: 113 237 248 + 3 748 352 and
# 109 949 952 + 3 864 320 B for 4 715 521 blocks; profiles/k_cheb_level0_p2_plane_dp_n320.md).
CHEB0_2D_DRAM_BYTES_PER_BLOCK = (113237248 + 3748352 + 109949952 + 3864320) / 2 / 4715521


def _spmv_bytes(info, dim, vb=8):
    """Algorithmic bytes of one masked block-CSR SpMV with vb-byte values and vectors: values +
    column indices + row pointers + x read once + y written once + free mask."""
    nnzb, n_rows = info.nnz_blocks, info.n_nodes
    n = n_rows * dim
    return nnzb * (dim * dim * vb + 4) + (n_rows + 1) * 4 + n * vb * 2 + n


def _cheb0_bytes(info, dim, deg=2):
    """Algorithmic bytes per launch of the level-0 Chebyshev steps of the AMG V-cycle (k_cheb, FP32),
    averaged over the timed sweep (the pre-smoothing: `deg` steps from zero).  Step 0 starts from
    x = 0 and reads no matrix: block-Jacobi inverse, free mask and b read, d and x written.  Every
    later step reads the matrix (values, column indices, row pointers), the inverse, the mask, and
    b, x_in, d, and writes d and x_out, each once."""
    nnzb, n_rows = info.nnz_blocks, info.n_nodes
    n = n_rows * dim
    step0 = n_rows * dim * dim * 4 + n + 3 * 4 * n
    later = nnzb * (dim * dim * 4 + 4) + (n_rows + 1) * 4 + n_rows * dim * dim * 4 + n + 5 * 4 * n
    return (step0 + (deg - 1) * later) / deg


def _assembly_bytes(info, dim, n_p, n_comp, kb=8, pe=1.0):
    """Algorithmic bytes of one fused assembly launch in the split form of eq. (K-split), with
    kb-byte K values and a fraction pe of the elements plastic: cached gradients and weights,
    connectivity, displacement gather, state read, F read and written once; for the plastic
    elements the slot map and their share of the K blocks read and written once (the reset of those
    blocks to K_elast is a separate launch).  pe = 1 gives the full form's bytes."""
    n_int, n_e = info.n_int, info.n_elem
    return (n_int * (n_p * dim + 1) * 8 + n_e * n_p * 4 + n_e * n_p * dim * 8 + n_int * (n_comp + 1) * 8
            + info.n_nodes * dim * 8 * 2 + pe * (n_e * n_p * n_p * 4 + info.nnz_blocks * dim * dim * kb * 2))


def _tangent_flops_per_point(dim, n_p, sym):
    """FP64 FLOPs of the local tangent per plastic point: H_p = (wD) G_p for every node p
    (NS rows x dim columns, 2 or 3 FMAs each) and the K_pq blocks (dim x dim, 2 or 3 FMAs each)."""
    ns = 3 if dim == 2 else 6
    fm = 2 if dim == 2 else 3
    h = n_p * ns * dim * fm * 2
    nb = n_p * (n_p + 1) // 2 if sym else n_p * n_p
    return h + nb * dim * dim * fm * 2


def _return_map_flops(model):
    """FP64 FLOPs of the return mapping per point (trial state, yield test, correction), counted
    from the closed forms of Section 2 (no division; one reciprocal square root counted as 10)."""
    return {0: 30, 1: 110, 2: 100, 3: 120}.get(model, 120)


def _base_flops_per_point(dim, n_p):
    """FP64 FLOPs spent on every point: strain (G_p u_p per node), wD and w sigma, F_p = G_p^T (w sigma)."""
    ns = 3 if dim == 2 else 6
    fm = 2 if dim == 2 else 3
    strain = n_p * ns * fm * 2 // 2
    force = n_p * dim * fm * 2
    return strain + force + 2 * ns * ns + 2 * ns


def run_reference(args):
    """The CPU oracle, as it stands, on a bounded sample of the workload: a reduced copy of its
    mesh with the same material, boundary conditions and load path (the line names the workload;
    cpu_baseline.sample names the sample)."""
    from oracle.newton import OracleSolver
    full = _workload(args.workload, full=True, n=args.n)
    prob = _workload(args.workload, full=False)
    s = OracleSolver(prob)
    n_path = len(prob.zeta)
    for j in range(args.warmup):
        s.solve_step(float(prob.zeta[j % n_path]), tol=prob.newton_rtol)
    s = OracleSolver(prob)
    t0 = time.perf_counter()
    assemblies = 0
    for j in range(args.steps):
        if j > 0 and j % n_path == 0:
            s = OracleSolver(prob)
        r = s.solve_step(float(prob.zeta[j % n_path]), tol=prob.newton_rtol)
        assemblies += r.newton_its + 1
    dt = time.perf_counter() - t0
    n_int = s.geom.n_int
    value = n_int * assemblies / dt / 1e9
    sample = (f"oracle on a reduced copy ({prob.mesh.elem_type} {prob.mesh.dim}D "
              f"{'x'.join(map(str, prob.mesh.shape))}, {n_int} points), {args.steps} load steps, splu solves")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _workload_config(args.workload, full, {"n_int": full.mesh.n_elem * (n_int // prob.mesh.n_elem)}),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": _cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _cores():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        blas = max((i.get("num_threads", 1) for i in info), default=1)
    except Exception:
        blas = 1
    return int(blas)


def cpu_baseline(args, budget_s=15.0):
    """Oracle IP-assembly throughput on a bounded sample: reduced copy, as many load steps as fit."""
    from oracle.newton import OracleSolver
    prob = _workload(args.workload, full=False)
    s = OracleSolver(prob)
    t0 = time.perf_counter()
    assemblies, steps = 0, 0
    for z in prob.zeta:
        r = s.solve_step(float(z), tol=prob.newton_rtol)
        assemblies += r.newton_its + 1
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": s.geom.n_int * assemblies / dt / 1e9, "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "sample": f"first {steps} load steps of a reduced copy ({prob.mesh.elem_type} "
                      f"{'x'.join(map(str, prob.mesh.shape))}, {s.geom.n_int} points), splu solves, "
                      f"{dt:.1f} s"}


def max_over_ranks(ms: float, world: int, device: str = "cuda") -> float:
    """Replicas (the path does not shard): every rank solves its own copy; the job's time is the
    slowest rank's.  The only collective is this timing reduction."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms


def job_value(world: int, n_int: int, assemblies: int, ms: float) -> float:
    """Whole-job throughput in Gpts/s: the points all ranks assembled over the job's time."""
    return world * n_int * assemblies / (ms / 1e3) / 1e9


def run_batch(args):
    """The batched sweep: problems of uneven size and material (seeded), one context per element
    type, the three batches solved concurrently on three streams, against the same problems solved
    one context after another.  Context creation (and the AMG setup) is outside the timed region."""
    import threading
    import torch
    import paper_1805_04155_gb300.ep as ep
    from synthetic import batch_problems
    hi = args.n if args.n else 48
    groups = batch_problems(seed=1805, n_problems=args.batch, sizes=(16, hi), n_steps=10)
    fams = sorted(groups)
    streams = {f: torch.cuda.Stream() for f in fams}
    ctxs = {f: ep.Context.from_batch(groups[f], stream=streams[f]) for f in fams}
    t_setup0 = time.perf_counter()
    singles = [] if args.no_one_by_one else [(pb, ep.Context.from_problem(pb)) for f in fams for pb in groups[f]]
    opts = ep.default_opts(newton_rtol=1e-10, krylov_graphs=0 if args.no_graphs else 1)
    zeta = groups[fams[0]][0].zeta

    def reset(ctx):
        for fld in (ep.EP_U, ep.EP_PLASTIC_STRAIN, ep.EP_HARDENING, ep.EP_STRESS, ep.EP_PLASTIC_FLAG):
            shape, dt = ctx.field_shape(fld)
            ctx.set(fld, np.zeros(shape, dtype=dt))

    # warm-up (builds every AMG hierarchy), then back to the virgin state
    for c in list(ctxs.values()) + [c for _, c in singles]:
        c.solve_load_path(zeta[:1], opts)
        reset(c)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup0
    results = {}

    def solve(f):
        results[f] = ctxs[f].solve_load_path(zeta, opts)

    t0 = time.perf_counter()
    th = [threading.Thread(target=solve, args=(f,)) for f in fams]
    for t in th:
        t.start()
    for t in th:
        t.join()
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    # the same sweep in mixed precision (FP32 tangent and inner Krylov, FP64 residual), batched
    mopts = ep.default_opts(newton_rtol=opts.newton_rtol, precision=ep.EP_MIXED, krylov_graphs=opts.krylov_graphs)
    for c in ctxs.values():
        reset(c)                             # the FP64 sweep left the contexts at the end of the path
        c.solve_load_path(zeta[:1], mopts)   # FP32 buffers on first use, outside the timed region
        reset(c)
    torch.cuda.synchronize()
    results_m = {}

    def solve_m(f):
        results_m[f] = ctxs[f].solve_load_path(zeta, mopts)

    t0 = time.perf_counter()
    th = [threading.Thread(target=solve_m, args=(f,)) for f in fams]
    for t in th:
        t.start()
    for t in th:
        t.join()
    torch.cuda.synchronize()
    t_batch_mixed = time.perf_counter() - t0
    t0 = time.perf_counter()
    reps_single = [c.solve_load_path(zeta, opts) for _, c in singles]
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    n_int = sum(ctxs[f].info.n_int for f in fams)
    assemblies = sum(r.n_assemble * ctxs[f].info.n_int for f in fams for r in results[f])
    line = {"metric": "batched sweep: integration points assembled per second (load paths of all problems)",
            "value": assemblies / t_batch / 1e9, "unit": "Gpts/s", "n_gpus": 1, "steps": len(zeta),
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.batch} problems, sizes 16..{hi} elements per side, "
                                   f"{', '.join(f'{len(groups[f])} {f}' for f in fams)}; E, nu, Y, H x U(0.7, 1.3)",
                       "n_int": n_int, "dofs": int(sum(ctxs[f].n_dof for f in fams))},
            "krylov_iterations": "direct launches" if args.no_graphs else "replayed from CUDA graphs",
            "batched_s": t_batch, "one_by_one_s": t_single if singles else None,
            "speedup": t_single / t_batch if singles else None, "setup_s": t_setup,
            "per_family": {f: {"problems": len(groups[f]), "dofs": int(ctxs[f].n_dof), "n_int": int(ctxs[f].info.n_int),
                               "newton_its": int(sum(r.newton_its for r in results[f])),
                               "krylov_its": int(sum(r.krylov_its for r in results[f])),
                               "solve_ms": float(sum(r.t_step_ms for r in results[f]))} for f in fams},
            "max_rel_resid": max(r.rel_resid for f in fams for r in results[f]),
            "mixed_batched_s": t_batch_mixed,
            "mixed_max_rel_resid": max(r.rel_resid for f in fams for r in results_m[f]),
            "mixed_newton_its": {f: int(sum(r.newton_its for r in results_m[f])) for f in fams},
            "newton_its": {f: int(sum(r.newton_its for r in results[f])) for f in fams},
            "one_by_one_newton_its": int(sum(r.newton_its for rs in reps_single for r in rs)) if singles else None}
    if args.learned:
        line["learned"] = learned_start_batch(args, ep, ctxs, groups, fams, zeta, opts, reset, results)
        # the combined form (mixed precision, batched, learned start) against the plain
        # FP64 GPU form (batched, extrapolated start) on time to solution at the same tolerance
        line["combined_vs_fp64"] = {"fp64_batched_s": t_batch, "mixed_batched_s": t_batch_mixed,
                                    "fp64_learned_batched_s": line["learned"]["batched_s"],
                                    "mixed_learned_batched_s": line["learned"]["mixed_batched_s"],
                                    "one_by_one_fp64_s": t_single if singles else None,
                                    "tolerance": opts.newton_rtol}
    for c in ctxs.values():
        c.close()
    for _, c in singles:
        c.close()
    print(json.dumps(line))


def learned_start_batch(args, ep, ctxs, groups, fams, zeta, opts, reset, results):
    """Learned warm start on the batched sweep: record (inputs, targets) rows along the load paths of
    a training batch drawn from other seeds (same families, sizes 16..32), train one network on them
    (full-batch Adam, the families' rows in turn), then solve the sweep again from the learned start
    and compare its Newton iterations and time with the extrapolated start timed above."""
    import threading
    import torch
    from synthetic import batch_problems
    from synthetic.random_states import mlp_init
    n_train = max(4, args.batch // 4)
    train = batch_problems(seed=10000, n_problems=n_train, sizes=(16, 32), n_steps=len(zeta))
    t0 = time.perf_counter()
    rec = {}
    for f in sorted(train):
        c = ep.Context.from_batch(train[f])
        c.ws_record(sum(pb.mesh.n_nodes for pb in train[f]) * len(zeta))
        c.solve_load_path(zeta, ep.default_opts(newton_rtol=1e-10, warm_start=1))
        rec[f] = c
    t_record = time.perf_counter() - t0
    net = ep.MLP(mlp_init(0))
    rows = {f: c.ws_samples_ptr() for f, c in rec.items()}
    t0 = time.perf_counter()
    loss0 = {f: net.grad(x, t, n_rows=n)[0] for f, (x, t, n) in rows.items() if n}
    for it in range(args.learned_steps):
        for f, (x, t, n) in rows.items():
            if n:
                net.train_step(x, t, 2e-3, n_rows=n, want_loss=False)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    loss1 = {f: net.grad(x, t, n_rows=n)[0] for f, (x, t, n) in rows.items() if n}
    n_rows = int(sum(n for _, _, n in rows.values()))
    train_tflops = args.learned_steps * n_rows * 2 * MLP_FMA_TRAIN / t_train / 1e12
    for c in rec.values():
        c.close()
    def timed_learned(prec):
        lopts = ep.default_opts(newton_rtol=opts.newton_rtol, warm_start=2, precision=prec,
                                krylov_graphs=opts.krylov_graphs)
        for f in fams:
            reset(ctxs[f])
            ctxs[f].ws_attach(net)
        torch.cuda.synchronize()
        res = {}

        def solve(f):
            res[f] = ctxs[f].solve_load_path(zeta, lopts)

        t0 = time.perf_counter()
        th = [threading.Thread(target=solve, args=(f,)) for f in fams]
        for t in th:
            t.start()
        for t in th:
            t.join()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, res

    t_learned, res = timed_learned(ep.EP_FP64)
    t_learned_mixed, res_mixed = timed_learned(ep.EP_MIXED)
    for f in fams:
        ctxs[f].ws_attach(None)
    net.close()
    return {"training": f"{n_train} problems (seed 10000), sizes 16..32, {n_rows} rows, "
                        f"{args.learned_steps} Adam steps per family at lr 2e-3",
            "record_s": t_record, "train_s": t_train,
            "train_tflops_wall": train_tflops, "train_frac_of_fp32_fma_peak": train_tflops / FP32_PEAK_TFLOPS,
            "loss": {f: [loss0[f], loss1[f]] for f in loss0},
            "batched_s": t_learned, "mixed_batched_s": t_learned_mixed,
            "mixed_newton_its": {f: int(sum(r.newton_its for r in res_mixed[f])) for f in fams},
            "newton_its": {f: int(sum(r.newton_its for r in res[f])) for f in fams},
            "extrapolated_newton_its": {f: int(sum(r.newton_its for r in results[f])) for f in fams},
            "problems_on_learned_start": {f: [int(r.n_learned) for r in res[f]] for f in fams},
            "max_rel_resid": max(r.rel_resid for f in fams for r in res[f])}


def run_mlp(args):
    """Training throughput of the warm-start network alone: Adam steps over n seeded synthetic rows
    (2^21 by default: 168 MB of inputs and targets, more than L2), timed with CUDA events on the
    network's stream.  Roofline: FP32 FMA (the layers are dense FP32 loops over shared memory)."""
    import torch
    import paper_1805_04155_gb300.ep as ep
    from synthetic.random_states import mlp_init, mlp_rows
    n = args.n if args.n else 1 << 21
    X, T = mlp_rows(n, seed=1805)
    Xd = torch.from_numpy(X).cuda()
    Td = torch.from_numpy(T).cuda()
    stream = torch.cuda.current_stream()
    net = ep.MLP(mlp_init(0), stream=stream)
    for _ in range(args.warmup):
        net.train_step(Xd, Td, 1e-3, want_loss=False)
    torch.cuda.synchronize()
    clocks = Clocks()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        net.train_step(Xd, Td, 1e-3, want_loss=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    loss = net.train_step(Xd, Td, 1e-3)
    tflops = n * 2 * MLP_FMA_TRAIN / (ms / 1e3) / 1e12
    net.close()
    line = {"metric": "warm-start network training: rows per second (forward + backward + Adam)",
            "value": n / (ms / 1e3), "unit": "rows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "dtype": "f32 (bf16 weights)", "data": "synthetic",
            "config": {"workload": f"{n} rows of 16 inputs / 4 targets, 16-128-128-4 network",
                       "l2": "inputs larger than L2"},
            "roofline": {"bound": "alu", "achieved": tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": tflops / FP32_PEAK_TFLOPS, "traffic": None,
                         "kernel": "k_mlp<train> + k_mlp_update (one Adam step)",
                         "flops_per_row": 2 * MLP_FMA_TRAIN,
                         "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 x 2.07 GHz (derived)"},
            "loss_after": loss, "clocks": clk}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="p2_plane_dp")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=0, help="cells per side (0: the workload's full size)")
    ap.add_argument("--precision", default="auto", choices=["auto", "mixed", "fp64"],
                    help="primary precision; auto: time both, report the faster as the primary")
    ap.add_argument("--no-compare", action="store_true", help="time the primary precision only (auto: mixed)")
    ap.add_argument("--batch", type=int, default=64, help="problems of the batched sweep (--workload batch)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch the Krylov iterations directly instead of replaying CUDA graphs (same kernels; "
                         "for kernel profilers that cannot follow graph-replayed launches)")
    ap.add_argument("--no-one-by-one", action="store_true",
                    help="--workload batch: skip the one-context-per-problem comparison (large sweeps)")
    ap.add_argument("--learned", action="store_true",
                    help="--workload batch: also train the warm-start network and solve from the learned start")
    ap.add_argument("--learned-steps", type=int, default=300, help="Adam steps per family of the warm-start network")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1805_04155_gb300 import build as B
    B.build()
    import paper_1805_04155_gb300.ep as ep

    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "mlp":
        run_mlp(args)
        return
    run_path(args, ep, local, world, rank)
    if world > 1:
        torch.distributed.destroy_process_group()


def _roof_hbm(name, launches, total_ms, bytes_per_launch, peaks, peaks_kind, step_ms, **extra):
    """Roofline entry of an HBM-bound kernel: algorithmic bytes per launch / average launch time."""
    dur = total_ms / launches / 1e3
    gbs = bytes_per_launch / dur / 1e9
    out = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": gbs / peaks["hbm_gbs"], "traffic": None, "kernel": name, "launches": launches,
           "avg_us": dur * 1e6, "bytes_per_launch": bytes_per_launch,
           "peak_source": f"{peaks_kind} (MEASURED_PEAKS.json hbm_gbs)", "share_of_step": total_ms / step_ms}
    out.update(extra)
    return out


def run_path(args, ep, local, world, rank):
    """The workload's whole load path from the virgin state, timed as one step (see the module
    docstring); both precisions, the end-to-end arm, the roofline of the step's kernels."""
    import torch
    prob = _workload(args.workload, n=args.n)
    stream = torch.cuda.current_stream()
    ctx = ep.Context.from_problem(prob, device=local, stream=stream)
    info = ctx.info
    n_path = len(prob.zeta)
    zeta = np.ascontiguousarray(prob.zeta, dtype=np.float64)
    prec_of = {"mixed": ep.EP_MIXED, "fp64": ep.EP_FP64}

    def opts_for(prec, profile=0):
        return ep.default_opts(newton_rtol=prob.newton_rtol, profile=profile, precision=prec_of[prec],
                               krylov_graphs=0 if args.no_graphs else 1)

    u_host = np.empty(ctx.n_dof)
    s_host = np.empty(ctx.field_shape(ep.EP_STRESS)[0])

    def path(opts, e2e):
        ctx.reset()
        reps = ctx.solve_load_path(zeta, opts)
        if e2e:
            ctx.get(ep.EP_U, out=u_host)
            ctx.get(ep.EP_STRESS, out=s_host)
        return reps

    def timed(prec, e2e: bool, steps: int):
        opts = opts_for(prec)
        reps = []
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        t_wall0 = time.perf_counter()
        evs[0].record(stream)
        for j in range(steps):
            reps.append(path(opts, e2e))
            evs[j + 1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall0
        torch.cuda.nvtx.range_pop()
        if world > 1:
            torch.distributed.barrier()
        per = [evs[j].elapsed_time(evs[j + 1]) for j in range(steps)]
        return evs[0].elapsed_time(evs[-1]), wall, per, reps

    if args.no_compare:
        precs = ["mixed" if args.precision == "auto" else args.precision]
    else:
        precs = ["mixed", "fp64"] if args.precision in ("auto", "mixed") else ["fp64", "mixed"]
    for p_ in precs:                      # warm-up: W whole paths in each precision
        for _ in range(args.warmup):
            path(opts_for(p_), False)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    runs = {}
    for p_ in precs:
        ms_p, wall_p, per_p, reps_p = timed(p_, False, args.steps)
        runs[p_] = (max_over_ranks(ms_p, world), wall_p, per_p, reps_p, ctx.get(ep.EP_U))
    clk = clocks.stop()
    # primary: the precision with the shorter median load-path time (time to solution)
    prec = args.precision if args.precision != "auto" else min(runs, key=lambda k: statistics.median(runs[k][2]))
    ms, wall, per, reps_paths, u_primary = runs[prec]
    reps = [r for rp in reps_paths for r in rp]
    assemblies = sum(r.n_assemble for r in reps)
    n_int = info.n_int
    value = job_value(world, n_int, assemblies, ms)

    def path_summary(prec_, ms_, per_, reps_paths_):
        rr = [r for rp in reps_paths_ for r in rp]
        a_ = sum(r.n_assemble for r in rr)
        last = reps_paths_[-1]
        return {"precision": prec_, "value": job_value(world, n_int, a_, ms_), "unit": UNIT,
                "load_path_s_median": statistics.median(per_) / 1e3, "load_path_s_min": min(per_) / 1e3,
                "paths": len(per_), "newton_its_per_path": int(sum(r.newton_its for r in last)),
                "newton_its_fp32_per_path": int(sum(r.newton_its_fp32 for r in last)),
                "krylov_its_per_path": int(sum(r.krylov_its for r in last)),
                "assemblies_per_path": int(sum(r.n_assemble for r in last)),
                "n_plastic_final": int(last[-1].n_plastic),
                "sparse_lu_steps_per_path": int(sum(r.direct for r in last)),
                "sparse_lu_factorisations_per_path": int(sum(r.n_direct_factor for r in last)),
                "max_rel_resid": max(r.rel_resid for r in rr)}

    compare = None
    others = [p_ for p_ in precs if p_ != prec]
    if others:
        other = others[0]
        ms_o, _, per_o, reps_o, u_o = runs[other]
        compare = path_summary(other, ms_o, per_o, reps_o)
        compare["u_rel_diff"] = float(np.linalg.norm(u_primary - u_o) / max(np.linalg.norm(u_o), 1e-300))

    e2e = None
    if not args.no_e2e:
        ms_e2e, _, _, reps_e2e = timed(prec, True, args.steps)
        ms_e2e = max_over_ranks(ms_e2e, world)
        a2 = sum(r.n_assemble for rp in reps_e2e for r in rp)
        e2e = {"value": job_value(world, n_int, a2, ms_e2e), "unit": UNIT,
               "h2d_bytes_per_step": int(zeta.nbytes), "d2h_bytes_per_step": int(u_host.nbytes + s_host.nbytes),
               "what": "per step: the load factors enter from the host, u and sigma of the path's end are "
                       "read back to host buffers"}

    # roofline of the step's kernels: one instrumented path of the primary precision right after the
    # timed region (CUDA events on the context's stream around every assembly and SpMV launch and
    # around a sample of the AMG level-0 Chebyshev sweeps; the instrumented path launches the Krylov
    # iterations directly, the timed ones replay them from CUDA graphs)
    torch.cuda.synchronize()
    reps_prof = path(opts_for(prec, 1), False)
    torch.cuda.synchronize()
    dim = info.dim
    f32 = prec == "mixed"
    kb = 4 if f32 else 8
    peaks, peaks_kind = _peaks()
    t_spmv = sum(r.t_spmv_kernel_ms for r in reps_prof)
    n_spmv = sum(r.n_spmv for r in reps_prof)
    t_asmk = sum(r.t_assemble_kernel_ms for r in reps_prof)
    n_sm0 = sum(r.n_smooth0 for r in reps_prof)
    t_sm0 = sum(r.t_smooth0_kernel_ms for r in reps_prof)
    sym = prob.material.model != 3
    plastic_assembled = sum(r.n_plastic_assembled for r in reps_prof)
    pe_assembled = sum(r.n_plastic_elem_assembled for r in reps_prof)
    krylov_its = sum(r.krylov_its for r in reps_prof)
    asm_prof = sum(r.n_assemble for r in reps_prof)
    ms_prof_path = statistics.median(per)   # shares against the timed path's median length
    cands = {}
    if n_spmv:
        # the FP64 operator of the Krylov solves: the mixed path's FP64-tangent iterations use it too
        cands["spmv"] = _roof_hbm(f"k_spmv (masked block-CSR)", n_spmv, t_spmv,
                                  _spmv_bytes(info, dim, 8), peaks, peaks_kind, ms_prof_path)
        if dim == 2:
            cands["spmv"]["traffic"] = SPMV64_2D_DRAM_BYTES_PER_BLOCK * info.nnz_blocks
            cands["spmv"]["traffic_source"] = "ncu capture at 320x320 cells, scaled by blocks"
    if asm_prof:
        pf = plastic_assembled / max(1, asm_prof * n_int)
        pe = pe_assembled / max(1, asm_prof * info.n_elem)
        by = _assembly_bytes(info, dim, info.n_p, info.n_comp, kb, pe)
        dur = t_asmk / asm_prof / 1e3
        tan = plastic_assembled * _tangent_flops_per_point(dim, info.n_p, sym) / asm_prof
        base = n_int * (_base_flops_per_point(dim, info.n_p) + _return_map_flops(prob.material.model))
        fp64_flops = base + (0 if f32 else tan)
        cands["assembly"] = _roof_hbm(
            f"k_assemble (fused, tangent {'FP32' if f32 else 'FP64'})", asm_prof, t_asmk, by, peaks, peaks_kind,
            ms_prof_path,
            plastic_fraction=pf, plastic_element_fraction=pe, fp64_flops_per_launch=fp64_flops,
            fp64_tflops=fp64_flops / dur / 1e12, fp64_frac=fp64_flops / dur / 1e12 / FP64_PEAK_TFLOPS,
            fp64_peak_source="FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2.07 GHz (derived)",
            assembled_gpts_s=n_int / dur / 1e9)
    if n_sm0:
        # sampled launches; the step's total is estimated as (Krylov iterations + solves) x the
        # level-0 Chebyshev steps per V-cycle (2 pre + 2 post)
        avg = t_sm0 / n_sm0
        est_n = 4 * krylov_its
        cands["amg_smooth0"] = _roof_hbm("k_cheb (AMG level-0 Chebyshev step, FP32)", n_sm0, t_sm0,
                                         _cheb0_bytes(info, dim), peaks, peaks_kind, ms_prof_path,
                                         share_of_step=avg * est_n / ms_prof_path, launches_sampled=n_sm0,
                                         launches_estimated=est_n)
        if dim == 2:
            # the timed sweep averages a zero-start step (no matrix: its algorithmic bytes) and a
            # matrix step (the capture's DRAM bytes per block, scaled to the run's blocks)
            n_rows = info.n_nodes
            step0 = n_rows * 16 + n_rows * 2 * 13
            cands["amg_smooth0"]["traffic"] = (step0 + CHEB0_2D_DRAM_BYTES_PER_BLOCK * info.nnz_blocks) / 2
            cands["amg_smooth0"]["traffic_source"] = ("matrix step: ncu capture at 320x320 cells scaled by blocks; "
                                                      "zero-start step: algorithmic bytes")
    # the sparse LU of the steps near the limit load (the Newton loop switches to it where the V-cycle
    # stalls): one factorisation per Newton iteration (FP32 FMA bound: the fronts' rank-32 updates),
    # a forward and a backward solve per GMRES iteration (reads the factors' pivot rows and columns)
    n_df = sum(r.n_direct_factor for r in reps_prof)
    if n_df:
        t_df = sum(r.t_direct_factor_ms for r in reps_prof)
        flop = max(r.direct_factor_flop for r in reps_prof)
        dur = t_df / n_df / 1e3
        tf = flop / dur / 1e12
        f64_fronts = os.environ.get("EP_DIRECT_FP32", "0") != "1"
        peak = FP64_PEAK_TFLOPS if f64_fronts else FP32_PEAK_TFLOPS
        cands["sparse_lu_factor"] = {
            "bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
            "traffic": None, "kernel": "sparse LU factorisation (k_df_scatter, k_df_diag, k_df_panel, k_df_update, "
                                       f"k_df_extend over the levels; {'FP64' if f64_fronts else 'FP32'} fronts)",
            "launches": n_df, "what_is_a_launch": "one factorisation (all levels)", "avg_us": dur * 1e6,
            "flop_per_launch": flop,
            "peak_source": ("FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz (derived)" if f64_fronts
                            else "FP32 FMA: 152 SMs x 128 lanes x 2 x 2.07 GHz (derived)"),
            "share_of_step": t_df / ms_prof_path}
    n_ds = sum(r.n_direct_solve for r in reps_prof)
    if n_ds:
        t_ds = sum(r.t_direct_solve_ms for r in reps_prof)
        cands["sparse_lu_solve"] = _roof_hbm("sparse LU solve (k_ds_fwd, k_ds_bwd over the levels)", n_ds, t_ds,
                                             max(r.direct_solve_bytes for r in reps_prof), peaks, peaks_kind,
                                             ms_prof_path, what_is_a_launch="one forward and backward solve")
    dominant = max(cands.values(), key=lambda r: r["share_of_step"]) if cands else None
    for c_ in cands.values():
        c_["timing"] = "instrumented path after the timed region (CUDA events on the launching stream)"
    xs = [r.n_plastic_assembled / r.n_assemble for r in reps_prof if r.n_assemble]
    ys = [1e3 * r.t_assemble_kernel_ms / r.n_assemble for r in reps_prof if r.n_assemble]
    asm_fit = None
    if len(set(np.round(xs, 6))) >= 2:
        A = np.vstack([np.ones(len(xs)), xs]).T
        (b0, b1), *_ = np.linalg.lstsq(A, np.array(ys), rcond=None)
        pred = b0 + b1 * np.array(xs)
        ss = float(np.sum((np.array(ys) - np.mean(ys)) ** 2))
        asm_fit = {"us_no_plastic": float(b0), "us_per_1k_plastic": float(b1 * 1e3),
                   "us_all_plastic_extrapolated": float(b0 + b1 * n_int),
                   "r2": 1.0 - float(np.sum((np.array(ys) - pred) ** 2)) / ss if ss > 0 else None,
                   "points": len(xs)}
    primary = path_summary(prec, ms, per, reps_paths)
    if primary["n_plastic_final"] == 0 and prob.material.model != 0:
        raise SystemExit("bench: the timed load path never left the elastic range")

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if f32 else "f64", "data": "synthetic",
            "config": _workload_config(args.workload, prob, {
                "n_int": n_int, "step": f"one whole load path ({n_path} load steps from the virgin state)",
                "parallelism": "replicas" if world > 1 else "single GPU", "precision": prec,
                "krylov": "GMRES(30)" if prob.material.model == 3 and prob.material.psi != prob.material.phi
                else "CG", "precond": "smoothed-aggregation AMG, FP32 V-cycle, Galerkin from the tangent; "
                                      "sparse LU where GMRES stalls with it (near the limit load)",
                "split_elastic_cache": True,
                "krylov_iterations": "direct launches" if args.no_graphs else "replayed from CUDA graphs"}),
            "roofline": dominant, "roofline_kernels": cands,
            "clocks": clk, "gpu_launches": int(sum(r.launches for r in reps)),
            "load_path_s": primary["load_path_s_median"], "primary": primary,
            "newton_its": primary["newton_its_per_path"], "krylov_its": primary["krylov_its_per_path"],
            "n_plastic_final": primary["n_plastic_final"], "max_rel_resid": primary["max_rel_resid"],
            "wall_s": wall}
    if asm_fit:
        line["assembly_vs_plastic"] = asm_fit
    if compare:
        line["compare"] = compare
    if e2e:
        line["e2e"] = e2e
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args)
    ctx.close()
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
