#!/usr/bin/env python
"""Benchmark of the W-draw hot path: Gibbs sweeps of the spatial fMRI GLM sampler.

One step = one full Gibbs sweep (Section 3.2) on the 3D whole-brain workload
(64x64x33 lattice, ellipsoid mask of ~50k voxels, T=300, K=6, AR(3), 6-neighbour UGL prior,
FP64 PCG with block-Jacobi preconditioner to relative residual 1e-8): perturbed right-hand
side + PCG solve for W (Algorithm 2), the A draw, lambda, alpha and beta draws, with the
chain state resident on the GPU. Each sweep yields one posterior W draw, so the metric is
W-draws/s.

Timing: W untimed warm-up sweeps (also burn-in), then K timed sweeps, each bracketed by CUDA
events on the library's stream, with a 256 MB buffer written between sweeps to flush L2
(the resident working set, ~100 MB, would otherwise stay in the 126 MB L2). Under torchrun
every rank runs its own independent chain (replicas: the path does not shard), the time is
the max over ranks and the value the sum of draws over ranks.

Also reported on the same line: the roofline of the dominant kernel (the W PCG solve, timed
with CUDA events inside the library), the FP64 oracle timed on this host's cores on a
bounded slab of the same workload (cpu_baseline), and an end-to-end figure through the
C ABI with host buffers (upload of X and Y, statistics, the sweeps, and a copy of every W
draw back to host memory).

--impl reference times the FP64 CPU oracle (exact sparse-LU solves in place of PCG) on the
same workload, one bounded slab per step, and prints the same JSON line with impl=reference.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "posterior W-draws/s + HBM-roofline fraction, 3D K=6; p50/p99 batched solve"
UNIT = "W-draws/s"
def workload_name(args):
    pc = {"reduced": "rbreduced", "ssor": "ssor", "bj": "blockjacobi"}[getattr(args, "precond", "reduced")]
    return f"wholebrain3d_64x64x33_ellipsoid_N49928_T300_K6_AR3_fp64_{pc}_delta1e-8"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured", d
    return 6800.0, "fallback", {}


# FP64 non-tensor peak of GB300: 152 SMs x 4 FP64 flops (2 DFMA) per clock x 2070 MHz.
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12


def pcg_flops_per_voxel_iter(K, mode="bj"):
    """FP64 flops of one Chronopoulos-Gear PCG iteration per voxel: four axpys (p, s, x, r)
    8K, block-Jacobi triangular solves 2K^2 + 2K, block product 2K^2, stencil with up to six
    neighbours 6K + 3K, three inner products 6K. Red-black SSOR ("ssor") adds the omega
    scaling K and its two colour phases, each over half of the voxels: neighbour sum 6K,
    right-hand side 2K (black) or K (red), triangular solves 2K^2, update K (black) or 3K
    (red). The reduced red-black system ("reduced", pipelined CG on the split-preconditioned
    system for K <= 6) works per pair of voxels: the black voxel's six axpys 12K (z, s, p, x,
    r, w), three triangular products K(K+1) each (L_b r for the residual norm, L_b^-T w,
    L_b^-1 of the neighbour sum), neighbour sum, scaling and difference 8K, inner products 6K;
    the red voxel's neighbour sum and scaling 7K and block-inverse product 2K^2. For K > 6 the
    unpipelined preconditioned form: per pair two block-inverse products and one block
    product 6K^2 and 30K."""
    base = 4 * K * K + 25 * K
    if mode == "reduced":
        if K <= 6:
            return (5 * K * K + 36 * K) / 2
        return (6 * K * K + 30 * K) / 2
    if mode != "ssor":
        return base
    return base + K + ((6 * K + 2 * K + 2 * K * K + K) + (6 * K + K + 2 * K * K + 3 * K)) / 2


def pcg_bytes_per_voxel_iter(K, w=8):
    """Algorithmic bytes of one PCG iteration per voxel: 11 vector passes of K words plus the
    data block and the preconditioner factor (K(K+1)/2 words each)."""
    return w * (11 * K + 2 * (K * (K + 1) // 2))


# DRAM bytes (read + write) of one W-solve launch on the whole-brain workload, from an ncu
# capture of the current kernel version (--set full, one launch), or None when the kernel has
# changed since its last capture. "reduced": the lane-pair kernel k_pcg_rbp2<6> (the default
# at K = 6: 25.37 MB read + 0.56 MB written); "reduced_one_lane": k_pcg_rbp<6> (--pcg-lanes 1:
# 25.45 MB read + 0.60 MB written). Both are the first touch of the blocks, factors, b and x;
# the iterations run from L2.
NCU_TRAFFIC_W = {"reduced": 25.92e6, "reduced_one_lane": 26.04e6, "ssor": None}


def precond_options(args):
    """Options of the headline FP64 chain's preconditioner (--precond)."""
    from paper_1606_00980_gb300 import bfmri
    if args.precond == "reduced":
        return {"precond": bfmri.PRECOND_RB_REDUCED, "pcg_lanes": args.pcg_lanes}
    if args.precond == "ssor":
        return {"precond": bfmri.PRECOND_SSOR, "ssor_omega": 1.0}
    return {"precond": bfmri.PRECOND_BLOCK_JACOBI}


def run_graph_compare(args, w, flush, stream, sweeps=20):
    """The headline chain without per-launch timing, sweeps launched directly and replayed from
    a captured CUDA graph (use_graph): ms per sweep each way, timed like the headline."""
    import torch

    from paper_1606_00980_gb300.bfmri import Model
    out = {}
    for name, g in (("direct", 0), ("captured", 1)):
        m = Model.from_workload(w, delta=1e-8, seed=2024, use_graph=g, **precond_options(args))
        m.precompute_stats()
        m.gibbs_sweep(args.warmup, 0, info=False)
        torch.cuda.synchronize()
        times, captured = [], 0
        for s in range(sweeps):
            flush.random_(0, 255)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            inf = m.gibbs_sweep(1, args.warmup + s, info=True)
            e1.record(stream)
            times.append((e0, e1))
            captured += inf.captured
        torch.cuda.synchronize()
        m.close()
        ms = sum(a.elapsed_time(b) for a, b in times) / sweeps
        out[name] = {"ms_per_sweep": ms, "W_draws_per_s": 1e3 / ms, "captured_sweeps": captured}
    return out


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = []
        reasons = set()
        smax = None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if "Active" in v and "Not" not in v:
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------------------

def oracle_sweep_time(w, z0, z1, seed=1, counter=0):
    """Seconds for one oracle Gibbs sweep on the slab z0 <= z < z1, and the slab's N."""
    from oracle import gibbs
    from oracle.lattice import Lattice
    from paper_1606_00980_gb300 import synth
    s = synth.zslab(w, z0, z1)
    lat = Lattice(s.mask, s.neighbourhood)
    st = gibbs.default_state(s.K, s.P, s.N)
    st["W"] = s.W_true.copy()
    st["A"] = s.A_true.copy()
    t = time.perf_counter()
    gibbs.gibbs_sweep(lat, s.Y, s.X, st, seed=seed, counter=counter)
    return time.perf_counter() - t, s.N


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info()]
        return max(n) if n else 1
    except Exception:
        return 1


def oracle_draw_time(w):
    """Seconds for one exact oracle W draw of workload w: the precision B~ factored in
    nested-dissection order (linalg.factor_nd) and the two solves of Algorithm 2 (the
    perturbed draw and the conditional mean), from the true A and the prior means of lambda
    and alpha."""
    import numpy as np

    from oracle import gibbs, linalg, model, philox
    from oracle.lattice import Lattice
    lat = Lattice(w.mask, w.neighbourhood)
    st = gibbs.default_state(w.K, w.P, w.N)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, w.A_true, st["lam"], w.eps)
    t = time.perf_counter()
    B = model.precision(lat, Bd, st["alpha"])
    pert, _, _ = model.perturbation(lat, Bd, st["alpha"], 1, 0, philox.TAG_W)
    x, y, z = lat.coords()
    f = linalg.factor_nd(B, np.stack([x, y, z], 1), w.K)
    b = model.kmajor(bw)
    f.solve(b + pert)
    f.solve(b)
    return time.perf_counter() - t


ORACLE_DRAW_CASES = {"slice2d": lambda s: s.slice2d(),
                     "replica3000": lambda s: s.request_workload(seed=5, N_target=3000, K=6, T=60, P=3)}


def oracle_child(kind):
    """Child process of the CPU timings (its BLAS thread count is fixed by the environment
    the parent sets): prints one JSON object."""
    from paper_1606_00980_gb300 import synth
    if kind == "slab":
        w = synth.wholebrain3d()
        zc = w.dims[2] // 2
        t, n_s = oracle_sweep_time(w, zc - 1, zc + 1)
        print(json.dumps({"t": t, "n": n_s, "N": w.N, "z0": zc - 1, "z1": zc}))
    else:
        w = ORACLE_DRAW_CASES[kind](synth)
        print(json.dumps({"t": oracle_draw_time(w), "n": w.N, "name": w.name}))


def oracle_timed(kind, threads):
    """Runs oracle_child(kind) in a fresh process with `threads` BLAS/OpenMP threads."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[v] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-child", kind],
                       env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(f"oracle timing {kind} failed: {r.stderr[-500:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(args, w):
    """The oracle on this host's cores. The exact oracle is infeasible at the whole-brain size
    (a sparse factorisation of B~ with 299,568 unknowns: SuperLU ran for 13 minutes on an
    8-core x86 host without finishing), so the value is one oracle Gibbs sweep on two central
    slices on one core, scaled to the whole volume by the voxel ratio: an upper bound of the
    oracle's whole-volume throughput, since its factorisation grows faster than linearly in
    N. Beside it, the measured per-draw cost (nested-dissection factorisation + two solves) of
    the 2D slice workload and of a 3,000-voxel replica of the whole-brain model (K = 6,
    P = 3, T = 60), on one core and on all cores."""
    cores = os.cpu_count() or 1
    slab = oracle_timed("slab", 1)
    per_draw = {}
    for kind in ORACLE_DRAW_CASES:
        one = oracle_timed(kind, 1)
        allc = oracle_timed(kind, cores)
        per_draw[one["name"]] = {"N": one["n"], "one_core_s": one["t"], "all_cores_s": allc["t"],
                                 "all_cores": cores}
    return {"value": (slab["n"] / slab["N"]) / slab["t"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one oracle Gibbs sweep on slices z={slab['z0']}..{slab['z1']} ({slab['n']} "
                      f"of {slab['N']} voxels, {slab['t']:.1f} s on one core), scaled to the whole "
                      f"volume by the voxel ratio (an upper bound: the exact oracle is infeasible "
                      f"at this size)",
            "exact_oracle_whole_brain": "infeasible at this size (299,568 unknowns)",
            "per_draw_exact": per_draw}


def run_reference(args, world, rank):
    """The FP64 oracle on the host cores: one 1-slice slab of the workload per step; the
    value is scaled to whole-volume W-draws/s by the voxel ratio (optimistic for the oracle:
    its sparse factorisation grows faster than linearly in N)."""
    if rank != 0:
        return
    from paper_1606_00980_gb300 import synth
    w = synth.wholebrain3d()
    zc = w.dims[2] // 2
    for i in range(args.warmup):
        oracle_sweep_time(w, zc, zc + 1, counter=i)
    tot, n_s = 0.0, 0
    for i in range(args.steps):
        t, n_s = oracle_sweep_time(w, zc, zc + 1, counter=1000 + i)
        tot += t
    per_step = tot / max(args.steps, 1)
    value = (n_s / w.N) / per_step
    sample = (f"one Gibbs sweep per step on the z={zc} slice ({n_s} of {w.N} voxels) of the "
              f"same workload; value scaled to the whole volume by the voxel ratio")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(args), "l2": "host run"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# GPU path
# ---------------------------------------------------------------------------------------

def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    from paper_1606_00980_gb300 import synth
    from paper_1606_00980_gb300.bfmri import Model

    w = synth.wholebrain3d()
    K, P, N, T = w.K, w.P, w.N, w.T
    # timed region: CUDA events around every sweep and around every PCG launch (profile 2:
    # solver launches only, which keeps the event overhead out of the other kernels)
    m = Model.from_workload(w, delta=1e-8, seed=2024, stream_id=rank, profile=2,
                            **precond_options(args))
    m.precompute_stats()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    counter = 0
    for _ in range(args.warmup):
        m.gibbs_sweep(1, counter, info=False)
        counter += 1
    torch.cuda.synchronize()
    m.reset_timing()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    times = []
    # sweeps are enqueued without a host wait (their errors and PCG counts are read once,
    # after the loop), so host-side jitter between launches does not idle the GPU inside
    # the timed events
    for s in range(args.steps):
        flush.random_(0, 255)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m.gibbs_sweep(1, counter, info=False)
        e1.record(stream)
        counter += 1
        times.append((e0, e1))
    span = m.synchronize()
    it_w, it_a = span.pcg_iterations_W, span.pcg_iterations_A
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    local_s = sum(a.elapsed_time(b) for a, b in times) / 1e3
    total_s = max_over_ranks(world, local_s)
    tim = m.timing()
    value = world * args.steps / total_s

    # roofline of the dominant kernel: the W PCG solve
    pw = tim["pcg_W"]
    launches = max(pw["launches"], 1)
    dur_s = pw["ms"] / 1e3 / launches
    iters_per_launch = it_w / launches
    flops = N * (iters_per_launch * pcg_flops_per_voxel_iter(K, args.precond) +
                 2 * pcg_flops_per_voxel_iter(K, args.precond))
    bytes_ = N * iters_per_launch * pcg_bytes_per_voxel_iter(K)
    hbm_peak, hbm_src, _ = peaks()
    achieved_tf = flops / dur_s / 1e12
    achieved_gbs = bytes_ / dur_s / 1e9
    # per-kernel breakdown: the same chain (same seed and draw counters) run again with every
    # launch timed (profile 1), over the same sweeps as the timed region
    m.close()
    mp = Model.from_workload(w, delta=1e-8, seed=2024, stream_id=rank, profile=1,
                             **precond_options(args))
    mp.precompute_stats()
    mp.gibbs_sweep(args.warmup, 0, info=False)
    torch.cuda.synchronize()
    mp.reset_timing()
    n_prof = args.steps
    mp.gibbs_sweep(n_prof, args.warmup, info=False)
    torch.cuda.synchronize()
    tim_p = mp.timing()
    mp.close()
    total_ms = sum(v["ms"] for v in tim_p.values()) / n_prof * args.steps
    # kernels per timed launch group: edge terms + assembly (W, A), quadratic form + draw (hyper)
    per_group = {"assemble_W": 2, "assemble_A": 2, "hyper": 2}
    n_launch = sum(v["launches"] * per_group.get(k, 1) for k, v in tim_p.items()) / n_prof * args.steps
    pairs = args.pcg_lanes == 2 or (args.pcg_lanes == 0 and K == 6)
    kname = {"reduced": ((f"k_pcg_rbp2<{K}> (W solve, pipelined CG on the red-black reduced system, "
                          "lane pairs)" if pairs else
                          f"k_pcg_rbp<{K}, false> (W solve, pipelined CG on the red-black reduced system)")
                         if K <= 6 else f"k_pcg_rb<{K}> (W solve, red-black reduced system)"),
             "ssor": f"k_pcg_res<{K}> (W solve, SSOR)",
             "bj": f"k_pcg_res<{K}> (W solve, block-Jacobi)"}[args.precond]
    roof = {"kernel": kname,
            "bound": "alu", "achieved": achieved_tf,
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved_tf / FP64_PEAK_TFLOPS,
            "traffic": NCU_TRAFFIC_W.get("reduced_one_lane" if args.precond == "reduced" and not pairs
                                         else args.precond),
            "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz",
            "hbm_view": {"achieved_gbs": achieved_gbs, "peak_gbs": hbm_peak,
                         "frac": achieved_gbs / hbm_peak, "peak_source": f"{hbm_src} (MEASURED_PEAKS.json)"},
            "iterations_per_launch": iters_per_launch, "avg_launch_ms": dur_s * 1e3,
            "share_of_step": pw["ms"] / total_ms if total_ms > 0 else None}

    # Auxiliary legs. Each runs inside run_leg: a leg that raises is recorded as
    # {"error": ...} in the line (and makes the exit status non-zero) instead of taking the
    # headline, roofline, cpu_baseline and e2e figures down with it. The serving leg, the
    # only one with several host threads launching at once, runs last.
    errors = {}
    main_rank = rank == 0
    mixed = run_leg(errors, "mixed_precision", run_mixed, args, w, flush, stream) if not args.no_mixed else None
    summ = run_leg(errors, "summaries", run_summaries, args, w) if (main_rank and not args.no_summaries) else None
    conv = run_leg(errors, "convergence", run_convergence, args) if (main_rank and not args.no_convergence) else None
    chains = run_leg(errors, "grouped_chains", run_chains, args, w, flush, stream, value) if not args.no_chains else None
    precs = run_leg(errors, "preconditioners", run_precond_compare, args, w) if (main_rank and not args.no_precond) else None
    mgc = run_leg(errors, "multigrid_chain", run_multigrid_chain, args, w) if (main_rank and not args.no_precond) else None
    priors = run_leg(errors, "prior_variants", run_prior_variants, args, w) if (main_rank and not args.no_priors) else None
    graphs = run_leg(errors, "captured_sweeps", run_graph_compare, args, w, flush, stream) if (main_rank and not args.no_graph) else None
    del flush
    # end to end through the C ABI with host buffers
    e2e = run_leg(errors, "e2e", run_e2e, args, w) if main_rank else None
    batched = run_leg(errors, "batched_probes", run_batched, args) if (main_rank and not args.no_batched) else None
    cpu = None
    if main_rank and world == 1 and not args.no_cpu_baseline:
        cpu = run_leg(errors, "cpu_baseline", cpu_baseline, args, w)
    stats_k = run_leg(errors, "stats_kernels", run_stats_kernels, args) if (main_rank and not args.no_stats) else None
    serving = run_leg(errors, "serving", run_serving, args, value * N) if (main_rank and not args.no_serving) else None
    if main_rank:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_name(args), "N": N, "T": T, "K": K, "P": P,
                           "parallelism": f"replicas{world}", "l2": "flushed between steps (256 MB write)",
                           "pcg_iterations_W_per_sweep": it_w / args.steps,
                           "pcg_iterations_A_per_sweep": it_a / args.steps,
                           "pcg_iterations_per_s": (it_w + it_a) / total_s},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "voxel_draws_per_s": value * N,
                "mixed_precision": mixed, "summaries": summ, "convergence": conv,
                "grouped_chains": chains,
                "preconditioners": precs, "multigrid_chain": mgc, "prior_variants": priors,
                "captured_sweeps": graphs, "serving": serving, "batched_probes": batched,
                "stats_kernels": stats_k,
                "gpu_launches": int(n_launch),
                "kernel_ms_per_step": {k: v["ms"] / n_prof for k, v in tim_p.items() if v["launches"]},
                "kernel_ms_per_step_note": "the same chain and sweeps rerun with every launch "
                                           "timed; the timed region times only the solver launches"}
        if errors:
            line["errors"] = errors
        print(json.dumps(line), flush=True)
    return 1 if errors else 0


def run_leg(errors, name, fn, *a, **kw):
    """Runs one auxiliary measurement; on an exception records it under errors[name] and
    returns {"error": ...} so that the JSON line still carries every other figure."""
    try:
        return fn(*a, **kw)
    except Exception as e:           # noqa: BLE001 - recorded in the JSON line, not hidden
        import traceback
        traceback.print_exc(file=sys.stderr)
        errors[name] = f"{type(e).__name__}: {e}"
        return {"error": errors[name]}


def bench_contrasts(K):
    """Three contrasts (first regressor, first minus second, a linear ramp) and thresholds."""
    import numpy as np
    C = np.zeros((3, K))
    C[0, 0] = 1.0
    C[1, 0], C[1, 1 % K] = 1.0, -1.0
    C[2] = np.linspace(0.5, -0.5, K)
    return C, np.array([0.5, 0.0, 0.1])


def run_summaries(args, w, sweeps=20):
    """Posterior summaries on the headline workload: the chain accumulation added to every
    sweep (3 contrast PPMs, a joint-PPM set of 1000 voxels, moments of W; one
    k_chain_accumulate launch per sweep) and the log joint posterior (Eq.
    UnnormalisedJointPosterior), each timed with CUDA events around its launches (profile 1).
    Bytes per accumulation: per voxel W, the reference sample, S1 and S2 read and written
    (8 B words), the counts read and written (4 B), the set flag (1 B)."""
    import numpy as np

    from paper_1606_00980_gb300.bfmri import Model
    m = Model.from_workload(w, delta=1e-8, seed=2024, profile=1, **precond_options(args))
    m.precompute_stats()
    m.gibbs_sweep(3, 0)
    C, g = bench_contrasts(w.K)
    E = np.random.default_rng(5).choice(w.N, 1000, replace=False)
    m.summary_begin(C, g, joint_set=E)
    m.reset_timing()
    m.gibbs_sweep(sweeps, 3)
    tim = m.timing()
    acc = tim["summary"]
    sweep_ms = sum(v["ms"] for v in tim.values()) / sweeps
    got = m.summary_get()
    m.reset_timing()
    for _ in range(10):
        lj = m.log_joint()
    t_lj = m.timing()["summary"]["ms"] / 10
    m.close()
    K, N, nc = w.K, w.N, len(g)
    bytes_acc = N * (8 * (K + K + 2 * K + 2 * (K * (K + 1) // 2)) + 4 * 2 * nc + 1)
    acc_s = acc["ms"] / max(acc["launches"], 1) / 1e3
    hbm_peak, hbm_src, _ = peaks()
    return {"samples": got["n"], "contrasts": nc, "joint_set_voxels": len(E),
            "accumulate_us": acc_s * 1e6, "share_of_sweep": acc["ms"] / sweeps / sweep_ms,
            "accumulate_hbm": {"achieved_gbs": bytes_acc / acc_s / 1e9, "peak_gbs": hbm_peak,
                               "frac": bytes_acc / acc_s / 1e9 / hbm_peak, "bytes": bytes_acc},
            "joint_ppm": (got["joint_count"] / got["n"]).tolist(),
            "log_joint_us": t_lj * 1e3, "log_joint": lj["total"]}


def time_to_within(values, times, tol=0.01):
    """Time at the first record after which every later record stays within tol of the final
    value in every component (relative); values (n_records, D)."""
    import numpy as np
    v = np.asarray(values)
    final = v[-1]
    ok = np.all(np.abs(v / final - 1.0) <= tol, axis=1)
    for i in range(len(ok)):
        if ok[i:].all():
            return float(times[i])
    return float(times[-1])


def library_prior_rows(args):
    """Draws of the simulation's UGL-prior rows as the paper's simulation makes them: the
    library's W and A draws (Algorithm 2) on the whole 53 x 63 x 46 block with no data term
    (lambda = 1e-200, so B_data and the data part of the right-hand side vanish to within
    1e-190 of the prior terms) from a zero start; PCG then solves the consistent singular
    system alpha G'G w = sqrt(alpha) G'z, whose edge increments are those of a prior draw.
    One draw per seed, kept for the sizes that follow."""
    import numpy as np

    from paper_1606_00980_gb300.bfmri import Model
    cache = {}

    def draw(block_xyz, alphas, beta, seed):
        if seed in cache:
            return cache[seed]
        nx, ny, nz = block_xyz
        n = nx * ny * nz
        K, P, T = len(alphas), 1, 8
        rng = np.random.default_rng(seed + 7)
        m = Model((nx, ny, nz, 6), np.ones((nz, ny, nx), np.uint8), rng.standard_normal((T, K)),
                  rng.standard_normal((T, n)), K, P, delta=1e-8, seed=seed, max_iter=20000,
                  **precond_options(args))
        m.precompute_stats()
        m.set_state(W=np.zeros((K, n)), A=np.zeros((P, n)), lam=np.full(n, 1e-200),
                    alpha=np.asarray(alphas, float), beta=np.array([float(beta)]))
        W, _ = m.sample_W(counter=1)
        A, _ = m.sample_A(counter=2)
        m.close()
        cache[seed] = (W, A[0])
        return cache[seed]
    return draw


def run_convergence(args, sizes=(1000, 10000, 100000)):
    """The paper's simulation study on GB300 (Appendix D data at N = 1e3, 1e4, 1e5; K = 5,
    P = 1, T = 351; Section 4's metric): processing time until the posterior mean of alpha is
    within 1 % of its final value. SVB: 50 iterations (N_s = 5 for the first 10, then 100,
    prior means as start values), once as the plain VB fixed-point iteration and once with the
    Appendix C extrapolation every other iteration; final = the last iteration's E[alpha]
    (with the extrapolation the iterates can settle into a cycle, which the per-iteration
    deviations show). MCMC: 1000 burn-in sweeps,
    then 4000 sweeps thinned by 5; the cumulative mean of the kept alpha draws against its
    final value. Device time by CUDA events around each step (statistics included); delta
    1e-8, the --precond solver."""
    import numpy as np
    import torch

    from paper_1606_00980_gb300 import synth
    from paper_1606_00980_gb300.bfmri import Model
    out = []
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    prior_rows = library_prior_rows(args)
    for N in sizes:
        w = synth.paper_simulation(N, seed=21, prior_rows=prior_rows)
        # SVB, with and without the Appendix C extrapolation (trick 1)
        svb = {}
        for name, extrap in (("svb_plain", False), ("svb_extrapolated", True)):
            m = Model.from_workload(w, delta=1e-8, seed=31, **precond_options(args))
            _, t_stats = timed(m.precompute_stats)
            t, times, alphas = t_stats, [], []
            for it in range(50):
                ns = 5 if it < 10 else 100
                # the fixed random numbers of Section 3.3: one draw counter for every iteration
                (avb, _, _), dt = timed(lambda: m.spvb_step(ns, 7, extrapolate=extrap))
                t += dt
                times.append(t)
                alphas.append(np.array(avb))
            m.close()
            dev = [round(float(np.max(np.abs(a / alphas[-1] - 1.0))), 4) for a in alphas]
            svb[name] = {"time_to_1pct_s": time_to_within(alphas, times), "total_s": times[-1],
                         "iteration_ms_Ns100": (times[-1] - times[-2]) * 1e3,
                         "alpha_final": alphas[-1].tolist(), "max_rel_dev_from_final": dev}
        # MCMC
        m = Model.from_workload(w, delta=1e-8, seed=32, **precond_options(args))
        _, t_stats = timed(m.precompute_stats)
        t = t_stats
        _, dt = timed(lambda: m.gibbs_sweep(1000, 0, info=False))
        t += dt
        times_m, cum = [], []
        acc = np.zeros(w.K)
        for j in range(800):
            _, dt = timed(lambda: m.gibbs_sweep(5, 1000 + 5 * j, info=False))
            t += dt
            acc += m.get_state()["alpha"]
            times_m.append(t)
            cum.append(acc / (j + 1))
        m.synchronize()
        m.close()
        mcmc_conv = time_to_within(cum, times_m)
        out.append({"N": N, **svb,
                    "mcmc": {"time_to_1pct_s": mcmc_conv, "total_s": times_m[-1],
                             "ms_per_sweep": (times_m[-1] - times_m[0]) / (5 * 799) * 1e3,
                             "alpha_final": cum[-1].tolist()}})
    return {"workload": "paper simulation (Appendix D), K5 P1 T351, N = 1e3 / 1e4 / 1e5",
            "prior_rows": "W task rows and the AR row drawn by the library's PCG from a zero "
                          "start with no data term, on the 53x63x46 block",
            "metric": "device seconds until E[alpha] is within 1 % of its final value",
            "precond": args.precond, "sizes": out}


def run_mixed(args, w, flush, stream):
    """Sweeps/s of the same workload with the FP32-inner / FP64-refinement solver at the same
    delta (1e-8), timed like the headline."""
    import torch

    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model
    m = Model.from_workload(w, delta=1e-8, seed=2024, precision=bfmri.PREC_MIXED, inner_tol=1e-6,
                            profile=2, **precond_options(args))
    m.precompute_stats()
    counter = 0
    for _ in range(args.warmup):
        m.gibbs_sweep(1, counter, info=False)
        counter += 1
    torch.cuda.synchronize()
    m.reset_timing()
    times = []
    it_w = ref_w = 0
    for s in range(args.steps):
        flush.random_(0, 255)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inf = m.gibbs_sweep(1, counter, info=True)
        e1.record(stream)
        counter += 1
        times.append((e0, e1))
        it_w += inf.pcg_iterations_W
    torch.cuda.synchronize()
    tot = sum(a.elapsed_time(b) for a, b in times) / 1e3
    tim = m.timing()
    # accuracy of one mixed-precision draw against the FP64 draw of the same system and random
    # numbers (FP64 solved to 1e-12; the parity tests bound that within 1e-8 of the exact draw)
    st = m.get_state()
    W_mixed, _ = m.sample_W(counter + 1)
    m.close()
    m64 = Model.from_workload(w, delta=1e-12, seed=2024, **precond_options(args))
    m64.precompute_stats()
    m64.set_state(W=st["W"], A=st["A"], lam=st["lam"], alpha=st["alpha"], beta=st["beta"])
    W64, _ = m64.sample_W(counter + 1)
    m64.close()
    import numpy as np
    err = float(np.linalg.norm(W_mixed - W64) / np.linalg.norm(W64))
    return {"value": args.steps / tot, "unit": UNIT, "ms_per_step": tot / args.steps * 1e3,
            "draw_rel_l2_vs_fp64": err,
            "delta": 1e-8, "inner_tol": 1e-6, "precond": args.precond,
            "inner_iterations_W_per_sweep": it_w / args.steps,
            "kernel_ms_per_step": {k: v["ms"] / args.steps for k, v in tim.items() if v["launches"]}}


def run_chains(args, w, flush, stream, single_value, n_chains=8):
    """n_chains independent chains of the headline workload (seeds 3000 + c), FP64 and
    delta 1e-8 as the headline, advanced by bfmri_gibbs_sweep_group: per sweep step every
    chain's W (then A) system is solved by one multi-RHS launch with a matrix per chain.
    Timed like the headline (CUDA events on the library's stream, L2 flushed between group
    sweeps); value = W-draws/s over all chains."""
    import torch

    from paper_1606_00980_gb300.bfmri import Model, gibbs_sweep_group
    models = []
    for c in range(n_chains):
        m = Model.from_workload(w, delta=1e-8, seed=3000 + c, **precond_options(args))
        m.precompute_stats()
        models.append(m)
    counter = 0
    for _ in range(args.warmup):
        gibbs_sweep_group(models, 1, counter)
        counter += 1
    torch.cuda.synchronize()
    times = []
    it_w = it_a = 0
    for _ in range(args.steps):
        flush.random_(0, 255)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = gibbs_sweep_group(models, 1, counter)
        e1.record(stream)
        counter += 1
        times.append((e0, e1))
        it_w += sum(i.pcg_iterations_W for i in infos)
        it_a += sum(i.pcg_iterations_A for i in infos)
    torch.cuda.synchronize()
    tot = sum(a.elapsed_time(b) for a, b in times) / 1e3

    # the same group in one multi-sweep call, by direct launches and replayed from the CUDA
    # graph of one group sweep (use_graph on the first chain; captured by the untimed call)
    def multi(ms):
        gibbs_sweep_group(ms, 2, 1000)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gibbs_sweep_group(ms, args.steps, 1002)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps
    direct_ms = multi(models)
    for m in models:
        m.close()
    models = []
    for c in range(n_chains):
        m = Model.from_workload(w, delta=1e-8, seed=3000 + c, use_graph=1, **precond_options(args))
        m.precompute_stats()
        models.append(m)
    captured_ms = multi(models)
    for m in models:
        m.close()
    value = n_chains * args.steps / tot
    return {"chains": n_chains, "value": value, "unit": UNIT,
            "ms_per_group_sweep": tot / args.steps * 1e3,
            "pcg_iterations_W_per_chain_sweep": it_w / (n_chains * args.steps),
            "pcg_iterations_A_per_chain_sweep": it_a / (n_chains * args.steps),
            "vs_single_chain": value / single_value if single_value else None,
            "multi_sweep_call_ms_per_sweep": {"direct": direct_ms, "captured_graph": captured_ms},
            "precond": args.precond, "delta": 1e-8, "dtype": "f64"}


def run_precond_compare(args, w, n_draws=10):
    """W and A solves of the headline workload with each preconditioner (after 3 sweeps from
    the prior means, same state and random numbers for all), and with the L'L prior of W:
    PCG iterations and solve time per draw (CUDA events around every launch)."""
    import torch

    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model
    cases = [("block_jacobi_resident", dict(precond=bfmri.PRECOND_BLOCK_JACOBI)),
             ("block_jacobi_streaming", dict(precond=bfmri.PRECOND_BLOCK_JACOBI,
                                             pcg_variant=bfmri.PCG_STREAMING)),
             ("ssor_omega1.0_resident", dict(precond=bfmri.PRECOND_SSOR, ssor_omega=1.0)),
             ("rb_reduced_resident", dict(precond=bfmri.PRECOND_RB_REDUCED)),
             ("ssor_omega1.0_streaming", dict(precond=bfmri.PRECOND_SSOR, ssor_omega=1.0,
                                              pcg_variant=bfmri.PCG_STREAMING)),
             ("ssor_omega1.2_resident", dict(precond=bfmri.PRECOND_SSOR, ssor_omega=1.2)),
             ("mixed_block_jacobi_resident", dict(precond=bfmri.PRECOND_BLOCK_JACOBI,
                                                  precision=bfmri.PREC_MIXED)),
             ("mixed_ssor_omega1.0_resident", dict(precond=bfmri.PRECOND_SSOR, ssor_omega=1.0,
                                                   precision=bfmri.PREC_MIXED)),
             ("mixed_rb_reduced_resident", dict(precond=bfmri.PRECOND_RB_REDUCED,
                                                precision=bfmri.PREC_MIXED)),
             ("multigrid", dict(precond=bfmri.PRECOND_MULTIGRID)),
             # the L'L prior of W (25-point stencil, two-pass streaming PCG): another model,
             # so its chain state and iteration counts are its own
             ("ltl_prior_block_jacobi_streaming", dict(precond=bfmri.PRECOND_BLOCK_JACOBI,
                                                       w_prior=bfmri.PRIOR_LTL))]
    out = {}
    for name, opts in cases:
        m = Model.from_workload(w, delta=1e-8, seed=2024, profile=1, **opts)
        m.precompute_stats()
        m.gibbs_sweep(3, 0, info=False)
        torch.cuda.synchronize()
        m.reset_timing()
        for i in range(n_draws):
            m.sample_W(100 + i, out=False)
            m.sample_A(100 + i, out=False)
        torch.cuda.synchronize()
        t = m.timing()
        m.close()
        out[name] = {"W_iterations_per_draw": t["pcg_W"]["pcg_iterations"] / n_draws,
                     "W_solve_ms_per_draw": t["pcg_W"]["ms"] / n_draws,
                     "A_iterations_per_draw": t["pcg_A"]["pcg_iterations"] / n_draws,
                     "A_solve_ms_per_draw": t["pcg_A"]["ms"] / n_draws}
    return out


def run_prior_variants(args, w, sweeps=20, warm=3):
    """Whole Gibbs sweeps of the headline workload under each prior of W on the FP64
    streaming solver with block-Jacobi (delta 1e-8, seed 2024, from the prior means): the
    graph Laplacian (the baseline of this comparison), per-edge BF16 factors (k / 16 drawn
    uniformly from 8..24), the anisotropic prior with its exchange step for the alphas, and
    the L'L prior; the graph Laplacian and the per-edge factors once more with the resident
    reduced red-black solver (the headline's solver family; one lane per voxel for per-edge
    factors), the anisotropic prior with the register-resident block-Jacobi kernel and with
    the resident reduced red-black solver, and the L'L prior on the resident block-Jacobi
    kernel. Per sweep: milliseconds (CUDA events around every launch), W PCG
    iterations, and for the anisotropic prior the exchange step's time (auxiliary solve
    included), auxiliary PCG iterations and acceptance rate."""
    import numpy as np
    import torch

    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model
    nx, ny, nz = w.dims
    fac = np.random.default_rng(99).integers(8, 25, size=(3, nz, ny, nx)) / 16.0
    cases = [("graph_laplacian", {}, None), ("per_edge_factors", {}, fac),
             ("graph_laplacian_reduced", dict(pcg_variant=bfmri.PCG_AUTO, precond=bfmri.PRECOND_RB_REDUCED), None),
             ("per_edge_factors_reduced", dict(pcg_variant=bfmri.PCG_AUTO, precond=bfmri.PRECOND_RB_REDUCED), fac),
             ("anisotropic", dict(w_prior=bfmri.PRIOR_ANISO), None),
             ("anisotropic_resident", dict(w_prior=bfmri.PRIOR_ANISO, pcg_variant=bfmri.PCG_AUTO), None),
             ("anisotropic_reduced", dict(w_prior=bfmri.PRIOR_ANISO, pcg_variant=bfmri.PCG_AUTO,
                                          precond=bfmri.PRECOND_RB_REDUCED), None),
             ("ltl", dict(w_prior=bfmri.PRIOR_LTL), None),
             ("ltl_resident", dict(w_prior=bfmri.PRIOR_LTL, pcg_variant=bfmri.PCG_AUTO), None)]
    if args is not None and getattr(args, "prior_cases", "all") != "all":
        keep = set(args.prior_cases.split(","))
        cases = [c for c in cases if c[0] in keep]
    out = {}
    for name, opts, f in cases:
        opts = dict(dict(pcg_variant=bfmri.PCG_STREAMING), **opts)
        opts = dict(dict(precond=bfmri.PRECOND_BLOCK_JACOBI), **opts)
        m = Model.from_workload(w, delta=1e-8, seed=2024, profile=1, **opts)
        if f is not None:
            m.set_edge_factors(f)
        m.precompute_stats()
        m.gibbs_sweep(warm, 0, info=False)
        m.synchronize()
        acc0 = m.get_alpha_dirs()[1] if name.startswith("anisotropic") else None
        m.reset_timing()
        m.gibbs_sweep(sweeps, warm, info=False)
        m.synchronize()
        torch.cuda.synchronize()
        t = m.timing()
        row = {"ms_per_sweep": sum(v["ms"] for v in t.values()) / sweeps,
               "W_solve_ms_per_sweep": t["pcg_W"]["ms"] / sweeps,
               "W_iterations_per_sweep": t["pcg_W"]["pcg_iterations"] / sweeps,
               "hyper_ms_per_sweep": t["hyper"]["ms"] / sweeps}
        if name.startswith("anisotropic"):
            a3, acc = m.get_alpha_dirs()
            row.update({"exchange_aux_iterations_per_sweep": t["hyper"]["pcg_iterations"] / sweeps,
                        "acceptance_rate": float(np.mean(acc - acc0)) / sweeps,
                        "alpha_dirs_mean": a3.mean(axis=0).tolist(),
                        "aniso_step": 1.0 / np.sqrt(w.N)})
        m.close()
        out[name] = row
    return out


def run_multigrid_chain(args, w, sweeps=200, windows=((5, 25), (25, 50), (50, 100), (100, 200))):
    """The headline chain (same seed, delta 1e-8, FP64) with the reduced red-black solver and
    with the multigrid V-cycle preconditioner, 200 sweeps each: per window of sweeps, W and A
    PCG iterations and solve time per draw (CUDA events around every solver launch). The
    chains' states differ (different rounding), the windows compare like with like."""
    import torch

    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model
    windows = tuple((a, b) for a, b in windows if b <= sweeps) or ((min(2, sweeps - 1), sweeps),)
    out = {}
    for name, pc in (("rb_reduced", bfmri.PRECOND_RB_REDUCED), ("multigrid", bfmri.PRECOND_MULTIGRID)):
        m = Model.from_workload(w, delta=1e-8, seed=2024, profile=2, precond=pc)
        m.precompute_stats()
        rows = {}
        done = 0
        for (a, b) in windows:
            if done < a:
                m.gibbs_sweep(a - done, done, info=False)
                m.synchronize()
            m.reset_timing()
            m.gibbs_sweep(b - a, a, info=False)
            m.synchronize()
            torch.cuda.synchronize()
            t = m.timing()
            n = b - a
            rows[f"{a}-{b}"] = {"W_iterations": t["pcg_W"]["pcg_iterations"] / n,
                                "W_ms": t["pcg_W"]["ms"] / n,
                                "A_iterations": t["pcg_A"]["pcg_iterations"] / n,
                                "A_ms": t["pcg_A"]["ms"] / n}
            done = b
        m.close()
        out[name] = rows
    return out


def mrhs_bytes_per_voxel_iter_rhs(D, S, w=4):
    """Bytes one multi-RHS iteration must move per voxel and right-hand side: the local phase
    reads u, w, p, s, x, r and writes p, s, x, r, u (11 D words, with r'u and r'r formed from
    the updated values), the product phase reads u and writes w (2 D words); the block and
    the preconditioner factor (D(D+1)/2 words each) are shared by the S right-hand sides."""
    return w * (13 * D) + w * 2 * (D * (D + 1) // 2) / S


def run_batched_chains(args, w, n_chains=8, sweeps=3):
    """8 independent FP64 chains of the 96x96x60 workload (seeds 5000 + c, delta 1e-8, the
    --precond preconditioner) advanced by bfmri_gibbs_sweep_group after 2 warm-up sweeps:
    W-draws/s over the chains, and the HBM view of the grouped W solve (one k_mrhs<8, double>
    launch per sweep; per voxel, iteration and chain 13 K FP64 vector words plus the chain's
    own block and factor, K(K+1)/2 words each; SSOR adds its two colour phases, 4 K words
    and one more factor read; the reduced red-black system moves 8 K words and one factor
    per voxel)."""
    import torch

    from paper_1606_00980_gb300.bfmri import Model, gibbs_sweep_group
    models = []
    for c in range(n_chains):
        m = Model.from_workload(w, delta=1e-8, seed=5000 + c, profile=1 if c == 0 else 0,
                                **precond_options(args))
        m.precompute_stats()
        models.append(m)
    gibbs_sweep_group(models, 2, 0)
    torch.cuda.synchronize()
    models[0].reset_timing()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = gibbs_sweep_group(models, sweeps, 2)
    e1.record(stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3
    tim = models[0].timing()
    with_probes = run_chains_with_probes(models, stream)
    for m in models:
        m.close()
    it_w = sum(i.pcg_iterations_W for i in infos)
    K = w.K
    F = K * (K + 1) // 2
    # words per voxel, iteration and chain: block-Jacobi 13 K + 2 F; SSOR adds its colour
    # phases (4 K + F); the reduced system moves 11 K + F per black voxel (local update and
    # factor) and 5 K + F per voxel pair in the red phase and the black product: 8 K + F
    words = {"bj": 13 * K + 2 * F, "ssor": 17 * K + 3 * F, "reduced": 8 * K + F}[args.precond]
    bytes_w = it_w * w.N * 8 * words
    solve_s = tim["pcg_W"]["ms"] / 1e3
    hbm_peak, hbm_src, _ = peaks()
    return {"chains": n_chains, "W_draws_per_s": n_chains * sweeps / dt,
            "ms_per_group_sweep": dt / sweeps * 1e3,
            "pcg_iterations_W_per_chain_sweep": it_w / (n_chains * sweeps),
            "W_solve_ms_per_group_sweep": solve_s / sweeps * 1e3,
            "W_solve_hbm": {"achieved_gbs": bytes_w / solve_s / 1e9, "peak_gbs": hbm_peak,
                            "frac": bytes_w / solve_s / 1e9 / hbm_peak},
            "precond": args.precond, "dtype": "f64", "delta": 1e-8,
            "with_probes": with_probes}


def run_chains_with_probes(models, stream, n_probes=64):
    """The grouped chains' W step with n_probes FP64 log-det probes of chain 0's W system in
    the same cooperative launch (bfmri_gibbs_sweep_group_probes: 8 matrices x 1 right-hand
    side beside 1 matrix x 64 probes; block-Jacobi for every right-hand side, which the
    probes' Lanczos quadrature needs), against the same work as two calls (one grouped sweep
    with the chains' own preconditioner, then bfmri_logdet_probe). CUDA events around each;
    the first combined call (workspace allocation) is not timed."""
    import torch

    from paper_1606_00980_gb300.bfmri import gibbs_sweep_group, gibbs_sweep_group_probes
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    gibbs_sweep_group_probes(models, 100, models[0], n_probes, 3000, probe_counter=1)
    torch.cuda.synchronize()
    models[0].reset_timing()
    e0.record(stream)
    infos, logdet, se, per = gibbs_sweep_group_probes(models, 101, models[0], n_probes, 3000,
                                                      probe_counter=2)
    e1.record(stream)
    torch.cuda.synchronize()
    combined_ms = e0.elapsed_time(e1)
    tim = models[0].timing()
    e0.record(stream)
    gibbs_sweep_group(models, 1, 102)
    res = models[0].logdet_probe(0, n_probes, 3000, counter=3)
    e1.record(stream)
    torch.cuda.synchronize()
    separate_ms = e0.elapsed_time(e1)
    return {"chains": len(models), "probes": n_probes, "right_hand_sides_in_launch": len(models) + n_probes,
            "combined_sweep_ms": combined_ms, "combined_W_launch_ms": tim["pcg_W"]["ms"],
            "separate_sweep_and_probe_ms": separate_ms,
            "pcg_iterations_W_per_chain": sum(i.pcg_iterations_W for i in infos) / len(models),
            "logdet": logdet, "stderr": se, "logdet_separate_call": res["logdet"],
            "dtype": "f64"}


def run_batched(args):
    """Batched probes: the 96x96x60 lattice (ellipsoid, ~250k voxels, K = 8, AR(3), T = 300),
    64 Rademacher probes for log det B~ solved together by the FP32-storage multi-RHS PCG
    (FP64 scalars and sums) to relative residual 1e-5, after 3 mixed-precision Gibbs sweeps
    from the prior means. Reports the probe solve's achieved HBM bandwidth."""
    import torch

    from paper_1606_00980_gb300 import bfmri, synth
    from paper_1606_00980_gb300.bfmri import Model
    if args.batched_lattice == "96x96x60":
        w = synth.batch3d()
    else:   # a smaller lattice of the same shape (profiling captures)
        nx, ny, nz = (int(v) for v in args.batched_lattice.split("x"))
        w = synth.wholebrain3d(seed=4, K=8, dims=(nx, ny, nz),
                               axes=(0.476 * nx, 0.476 * ny, 0.4767 * nz), T=300)
    m = Model.from_workload(w, delta=1e-5, precision=bfmri.PREC_MIXED, seed=4242, profile=1)
    m.precompute_stats()
    m.gibbs_sweep(3, 0)
    S = args.probes
    # warm-up (workspace allocation; the autotuner times the right-hand-side tiles 1, 2, 4
    # on this first call of the shape and keeps the fastest)
    m.logdet_probe(0, S, 3000, counter=1)
    tile, tile_ms = m.probe_tuning()
    m.reset_timing()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = m.logdet_probe(0, S, 3000, counter=2)
    wall = time.perf_counter() - t0
    tim = m.timing()
    m.close()
    solve_s = tim["other"]["ms"] / 1e3
    iters = int(res["iterations"].sum())
    svb = None
    if not args.no_svb:
        # one spatial-VB iteration (N_s = 100 samples of W and A, FP64 multi-RHS solves with the
        # fixed random numbers of Section 3.3, the --precond preconditioner), after a first
        # iteration that creates the samples
        ms = Model.from_workload(w, delta=1e-8, seed=4243, profile=1, **precond_options(args))
        ms.precompute_stats()
        ms.gibbs_sweep(3, 0)
        ms.spvb_step(100, 7)
        torch.cuda.synchronize()
        ms.reset_timing()
        t1 = time.perf_counter()
        _, _, info = ms.spvb_step(100, 7)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t1
        tsv = ms.timing()
        # Section 3.3 summaries of the 100 samples: moments and Gaussian contrast PPMs (one
        # k_svb_summary launch streams the samples once)
        Cs, gs = bench_contrasts(w.K)
        ms.svb_summary(Cs, gs)
        ms.reset_timing()
        ms.svb_summary(Cs, gs)
        t_sum = ms.timing()["summary"]["ms"]
        ms.close()
        K = w.K
        sum_bytes = 100 * K * w.N * 8 + (K + K * (K + 1) // 2 + len(gs)) * w.N * 8
        # FP64 work: per sample and voxel K subtractions, K additions and K(K+1)/2 FMAs
        sum_flops = 99 * w.N * (2 * K + K * (K + 1))
        hbm_peak, _, _ = peaks()
        svb = {"samples": 100, "precond": args.precond, "iteration_ms": dt * 1e3,
               "pcg_iterations_W_total": int(info.pcg_iterations_W),
               "pcg_iterations_A_total": int(info.pcg_iterations_A),
               "W_solve_ms": tsv["pcg_W"]["ms"], "A_solve_ms": tsv["pcg_A"]["ms"],
               "max_rel_residual_W": info.max_rel_residual_W,
               "summary": {"contrasts": len(gs), "ms": t_sum, "bound": "alu",
                           "fp64": {"achieved_tflops": sum_flops / (t_sum / 1e3) / 1e12,
                                    "peak_tflops": FP64_PEAK_TFLOPS,
                                    "frac": sum_flops / (t_sum / 1e3) / 1e12 / FP64_PEAK_TFLOPS},
                           "hbm": {"achieved_gbs": sum_bytes / (t_sum / 1e3) / 1e9,
                                   "peak_gbs": hbm_peak,
                                   "frac": sum_bytes / (t_sum / 1e3) / 1e9 / hbm_peak},
                           "bytes": sum_bytes}}
    bytes_ = iters * w.N * mrhs_bytes_per_voxel_iter_rhs(w.K, S)
    hbm_peak, hbm_src, _ = peaks()
    gbs = bytes_ / solve_s / 1e9
    # the minimum of the two-pass fused PCG form (11 vector passes; this solver's
    # Chronopoulos-Gear form moves 13)
    bytes11 = iters * w.N * (4 * 11 * w.K + 4 * 2 * (w.K * (w.K + 1) // 2) / S)
    gbs11 = bytes11 / solve_s / 1e9
    return {"workload": f"batch3d_96x96x60_ellipsoid_N{w.N}_K{w.K}_T{w.T}_AR3",
            "probes": S, "logdet": res["logdet"], "stderr": res["stderr"],
            "probe_iterations_mean": float(res["iterations"].mean()),
            "probe_iterations_max": int(res["iterations"].max()),
            "solve_ms": solve_s * 1e3, "call_ms": wall * 1e3, "svb_iteration": svb,
            "autotune": {"rhs_tile": tile, "candidate_ms": {"1": tile_ms[0], "2": tile_ms[1],
                                                            "4": tile_ms[2]}},
            "hbm_11_vector_passes": {"achieved_gbs": gbs11, "frac": gbs11 / hbm_peak},
            "chains": None if args.no_svb else run_batched_chains(args, w),
            "roofline": {"kernel": (f"k_mrhs_tile<{w.K}, {tile}>" if tile > 1 else f"k_mrhs<{w.K}, float>"),
                         "bound": "hbm", "achieved": gbs,
                         "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                         "traffic": None, "peak_source": f"{hbm_src} (MEASURED_PEAKS.json)",
                         "bytes_per_voxel_iter_rhs": mrhs_bytes_per_voxel_iter_rhs(w.K, S)}}


def stats_case_serving_max(seed=77):
    """The largest serving request's statistics shape: an ellipsoid of ~300k voxels,
    T = 600, K = 10, P = 3, FP32 series (random values: the cost does not depend on them)."""
    import numpy as np

    from paper_1606_00980_gb300 import synth
    rng = np.random.default_rng(seed)
    w = synth.request_workload(seed=seed, N_target=20000, K=10, T=600, P=3)
    a = (3.0 * 300000 / (2.0 * np.pi)) ** (1.0 / 3.0)
    nx = ny = int(np.ceil(2 * a + 2))
    nz = int(np.ceil(a + 2))
    mask = synth.ellipsoid_mask(nx, ny, nz, a, a, a / 2.0)
    N = int(mask.sum())
    Y = (100.0 + rng.standard_normal((w.T, N))).astype(np.float32)
    return (nx, ny, nz, 6), mask, w.X, Y, w.K, w.P


def run_stats_kernels(args):
    """Sufficient statistics of FP32 series (Appendix A's pre-computed lagged products): the
    FP64 CUDA-core kernel against the tensor-core kernel (exact BF16 digit products), on the
    whole-brain workload with its series rounded to FP32 and on the largest serving shape
    (~300k voxels, T = 600, K = 10, P = 3). CUDA events around the statistics launch;
    the two results are compared element by element. Tensor work: per 128 voxels and 16 time
    steps, 36 digit-pair MMAs of 128 x N x 16 (N = 8 x (2P + 1) rounded up to 16)."""
    import numpy as np

    from paper_1606_00980_gb300 import bfmri, synth
    from paper_1606_00980_gb300.bfmri import Model
    wb = synth.wholebrain3d()
    nx, ny, nz = wb.dims
    cases = {}
    if args.stats_case in ("all", "wholebrain3d"):
        cases["wholebrain3d_fp32"] = ((nx, ny, nz, 6), wb.mask, wb.X, wb.Y.astype(np.float32), wb.K, wb.P)
    if args.stats_case in ("all", "serving_max"):
        cases["serving_max_N300k_T600_K10_P3"] = stats_case_serving_max()
    out = {}
    for name, (lat, mask, X, Y, K, P) in cases.items():
        res, stats = {}, {}
        for kname, kern in (("fp64_cuda_cores", bfmri.STATS_FP64), ("tensor_cores", bfmri.STATS_TENSOR)):
            times = []
            for rep in range(3):
                m = Model(lat, mask, X, Y, K, P, profile=1, stats_kernel=kern)
                m.precompute_stats()
                times.append(m.timing()["stats"]["ms"])
                if rep == 0:
                    stats[kname] = m.get_stats()
                m.close()
            res[kname] = {"ms": float(np.median(times)), "ms_all": times}
        N, T = Y.shape[1], Y.shape[0]
        Tw = T - 2 * P
        ref = stats["fp64_cuda_cores"]
        diff = float(np.max(np.abs(stats["tensor_cores"] - ref)) / np.abs(ref).max())
        nmma = {0: 16, 1: 32, 2: 48, 3: 64}[P] * ((K + 7) // 8)
        mma_flops = 36.0 * 2 * 128 * nmma * 16 * np.ceil(N / 128) * np.ceil(Tw / 16)
        t_tc = res["tensor_cores"]["ms"] / 1e3
        out[name] = {"N": N, "T": T, "K": K, "P": P, **res,
                     "speedup": res["fp64_cuda_cores"]["ms"] / res["tensor_cores"]["ms"],
                     "max_rel_diff_vs_fp64_kernel": diff,
                     "tensor_mma_tflops": mma_flops / t_tc / 1e12,
                     "fp64_equivalent_tflops": 2.0 * K * (2 * P + 1) * Tw * N / t_tc / 1e12,
                     "y_read_gbs": 2 * 4.0 * N * T / t_tc / 1e9}
    return out


def run_serving(args, fp64_single_voxel_draws=None):
    """Serving workload: a Poisson stream of requests, each a synthetic subject (ellipsoid mask
    of 5k-300k voxels, log-uniform; K in {4,6,8,10}; T in {150,300,600}; AR(1)-AR(3)), each
    running create + statistics + 8 mixed-precision Gibbs sweeps at delta = 1e-8 (the --precond
    preconditioner) with its state
    resident on the device, admitted into 4 slots under a 64 GB device-memory budget. The
    distinct subjects are a pool of 8 that spans those ranges (generating hundreds of distinct
    subjects on the host would dominate the run); requests draw from it uniformly in log N.
    Latency = submission -> result readable on the host."""
    import numpy as np

    from paper_1606_00980_gb300 import bfmri, synth
    rng = np.random.default_rng(11)
    Ks, Ts = [4, 6, 8, 10], [150, 300, 600]
    pool = []
    for i, n_target in enumerate(np.geomspace(5000, 300000, 8)):
        T = Ts[i % 3] if n_target < 150000 else 150
        w = synth.request_workload(seed=300 + i, N_target=int(n_target), K=Ks[i % 4], T=T,
                                   P=1 + i % 3)
        w.Y = w.Y.astype(np.float32)
        pool.append(w)
    slots, sm_budget, budget = 4, 38, 64 << 30
    opts = dict(precision=bfmri.PREC_MIXED, delta=1e-8, inner_tol=1e-6, **precond_options(args))
    # capacity pilot: every pool member alone (service time), then a saturating burst of
    # 4 x the pool through all slots (sustained requests/s)
    # every server is closed in a finally block: closing waits for the requests in flight,
    # so an exception never leaves slot kernels running while the process exits
    with bfmri.Server(budget, slots, sm_budget) as srv:
        pilot = []
        for i, w in enumerate(pool):
            t = srv.submit(w, 8, first_counter=0, seed=1000 + i, **opts)
            r = srv.poll(t)
            pilot.append(r["end_s"] - r["start_s"])
        mean_service = float(np.mean(pilot))
        t0 = time.perf_counter()
        burst = [srv.submit(pool[i % len(pool)], 8, first_counter=i, seed=2000 + i, **opts)
                 for i in range(4 * len(pool))]
        for t in burst:
            srv.poll(t)
        capacity = 4 * len(pool) / (time.perf_counter() - t0)
    rate = 0.8 * capacity                      # offered load 0.8 of the measured capacity
    n_req = args.serving_requests
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    picks = rng.integers(0, len(pool), n_req)
    with bfmri.Server(budget, slots, sm_budget) as srv:
        t0 = time.perf_counter()
        tickets = []
        for i in range(n_req):
            delay = arrivals[i] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(pool[picks[i]], 8, first_counter=17 * i, seed=5000 + i, **opts))
        results = [srv.poll(t) for t in tickets]
        makespan = time.perf_counter() - t0
        st = srv.stats()
    lat = np.array([r["end_s"] - r["submit_s"] for r in results]) * 1e3
    return {"requests": n_req, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "draws_per_s": 8 * n_req / makespan, "unit": UNIT, "makespan_s": makespan,
            "voxel_draws_per_s": 8 * float(sum(pool[j].N for j in picks)) / makespan,
            "capacity_draws_per_s": 8 * capacity,
            "capacity_voxel_draws_per_s": 8 * capacity * float(np.mean([w.N for w in pool])),
            "note": "draws/s follow the offered load (0.8 of capacity); the requests average "
                    "more voxels than the headline workload, so voxel-draws/s compare them",
            "offered_rate_per_s": rate, "capacity_per_s": capacity,
            "mean_service_ms_alone": mean_service * 1e3,
            "slots": slots, "sm_budget_per_slot": sm_budget, "budget_bytes": budget,
            "peak_in_flight": st["peak_running"], "peak_bytes": st["peak_bytes"],
            "pool_N": [int(w.N) for w in pool], "pool_K": [int(w.K) for w in pool],
            "pool_T": [int(w.T) for w in pool], "pool_P": [int(w.P) for w in pool],
            "work_per_request": "create + stats + 8 mixed-precision Gibbs sweeps (delta 1e-8)",
            "fp64_single_chain_voxel_draws_per_s": fp64_single_voxel_draws,
            "capacity_vs_fp64_single_chain": (8 * capacity * float(np.mean([w.N for w in pool]))
                                              / fp64_single_voxel_draws) if fp64_single_voxel_draws else None}


def run_e2e(args, w):
    """create (X, Y and the mask in pinned host memory, copied to the device inside the timed
    region) + statistics + S sweeps, each draw copied to pinned host memory."""
    import dataclasses

    import numpy as np
    import torch

    from paper_1606_00980_gb300.bfmri import Model
    S = max(args.steps, 1)
    Wh = torch.empty((w.K, w.N), dtype=torch.float64, pin_memory=True).numpy()

    def pinned(a):
        p = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True).numpy()
        p[...] = a
        return p
    w = dataclasses.replace(w, Y=pinned(w.Y), X=pinned(w.X), mask=pinned(w.mask))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m = Model.from_workload(w, delta=1e-8, seed=77, **precond_options(args))
    m.precompute_stats()
    for s in range(S):
        m.gibbs_sweep(1, s, info=False)
        m.get_W(out=Wh)                      # the sweep's draw, into pinned host memory
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    m.close()
    h2d = w.Y.nbytes + w.X.nbytes + w.mask.nbytes
    return {"value": S / dt, "unit": UNIT, "h2d_bytes_per_step": h2d // S,
            "d2h_bytes_per_step": w.K * w.N * 8,
            "what": f"create + statistics from pinned host buffers, then {S} sweeps, each W "
                    f"draw copied to pinned host memory"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--probes", type=int, default=64)
    ap.add_argument("--batched-lattice", default="96x96x60",
                    help="lattice of the batched-probe workload (e.g. 64x64x40 for a capture)")
    ap.add_argument("--no-svb", action="store_true")
    ap.add_argument("--no-chains", action="store_true")
    ap.add_argument("--no-precond", action="store_true")
    ap.add_argument("--no-priors", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-summaries", action="store_true")
    ap.add_argument("--no-convergence", action="store_true",
                    help="skip the paper's simulation study (time to 1 %% convergence of "
                         "E[alpha] for SVB and MCMC at N = 1e3, 1e4, 1e5), which runs by default")
    ap.add_argument("--precond", choices=["reduced", "ssor", "bj"], default="reduced",
                    help="preconditioner of the headline chain and of its mixed-precision twin "
                         "(the multi-RHS solves use block-Jacobi)")
    ap.add_argument("--only-batched", action="store_true",
                    help="run only the batched-probe measurement (profiling entry point)")
    ap.add_argument("--serving-requests", type=int, default=96)
    ap.add_argument("--no-stats", action="store_true")
    ap.add_argument("--only-multigrid", action="store_true",
                    help="run only the multigrid-vs-reduced chain comparison")
    ap.add_argument("--pcg-lanes", type=int, default=0, choices=[0, 1, 2],
                    help="lanes per voxel of the resident reduced solver (0: the library's "
                         "default, lane pairs; 1: one lane per voxel)")
    ap.add_argument("--multigrid-sweeps", type=int, default=200,
                    help="sweeps of each chain of the multigrid comparison (profiling: a few)")
    ap.add_argument("--stats-case", default="all", choices=["all", "wholebrain3d", "serving_max"])
    ap.add_argument("--only-stats", action="store_true",
                    help="run only the statistics-kernel comparison (profiling entry point)")
    ap.add_argument("--only-priors", action="store_true",
                    help="run only the prior-variant sweeps (profiling entry point)")
    ap.add_argument("--prior-sweeps", type=int, default=20,
                    help="timed sweeps per prior variant (profiling: a few)")
    ap.add_argument("--prior-cases", default="all",
                    help="comma-separated prior-variant cases to run (default all)")
    ap.add_argument("--oracle-child", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_child:
        oracle_child(args.oracle_child)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    world, rank, local = dist_setup(args)
    rc = 0
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.only_multigrid:
        if rank == 0:
            from paper_1606_00980_gb300 import synth
            print(json.dumps(run_multigrid_chain(args, synth.wholebrain3d(),
                                                 sweeps=max(args.multigrid_sweeps, 2))), flush=True)
    elif args.only_stats:
        if rank == 0:
            print(json.dumps(run_stats_kernels(args)), flush=True)
    elif args.only_batched:
        if rank == 0:
            print(json.dumps(run_batched(args)), flush=True)
    elif args.only_priors:
        if rank == 0:
            from paper_1606_00980_gb300 import synth
            print(json.dumps(run_prior_variants(args, synth.wholebrain3d(),
                                                sweeps=max(args.prior_sweeps, 1))), flush=True)
    else:
        rc = run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rc:
        sys.exit(rc)


if __name__ == "__main__":
    main()
