#!/usr/bin/env python
"""Benchmark of the coupled LBM-PIBM-DEM step on the 2D sedimentation workload
(D2Q9 2048 x 2048 with walls, tau 0.6, 500,000 particles with diameters uniform in
[0.3, 0.8] lu and density ratio 2.5 in the top 60 %, 4-point delta).

Prints one JSON line. ``value`` is whole-job MLUPS (lattice-cell updates per
second, coupled step, all ranks); particle updates per second ride along. Inputs
are resident in HBM when the timed region starts and the two population buffers
(2 x 151 MB in FP32, 2 x 302 MB in FP64) exceed the 129 MB L2, so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle (test infrastructure) on a bounded
sample of the same workload on the host cores.
"""
import argparse
import glob
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")
# FP64 peak of the GB300 CUDA cores: nominal 1.25 TFLOP/s, i.e. about 2 FP64 FMA
# per clock per SM (152 SMs at 2.07 GHz); the FP64 paths are bounded by it.
FP64_PEAK_TFLOPS = 1.25
WORKLOAD_DESC = ("2D sedimentation: D2Q9 2048x2048 walls, tau 0.6, 500k particles "
                 "d~U[0.3,0.8] lu, rho_p/rho_f 2.5, top 60%, gravity 1e-5, 4-point delta, "
                 "linear spring-dashpot kn 1e-2 e 0.9")


def _peaks():
    try:
        with open(PEAKS_FILE) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _src_hash(source):
    """Hash of the source files that define a kernel (csrc/<source>, or a list of
    such names hashed in order)."""
    h = hashlib.sha256()
    for name in ([source] if isinstance(source, str) else source):
        with open(os.path.join(ROOT, "paper_1407_6704_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, only if the source
    file of the kernel is unchanged since it was captured."""
    try:
        with open(TRAFFIC_FILE) as fh:
            t = json.load(fh)
        ent = t.get(kernel)
        if (ent and ent.get("workload") == workload
                and ent.get("source_sha") == _src_hash(ent["source"])):
            return float(ent["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.dev = device_id
        self.proc = None
        self.tmp = None

    def __enter__(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)], stdout=self.tmp, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.tmp:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.tmp.flush()
        with open(self.tmp.name) as fh:
            rows = [r.strip().split(",") for r in fh if r.strip()]
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for nm, v in zip(names, r[4:8]):
                    if v.strip().lower() in ("active", "1"):
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def collide_bytes_per_cell(q, precision):
    # read and write every population once, in the storage type
    return 2 * q * {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}[precision]


def particle_bytes(d):
    # algorithmic bytes per particle, FP64: read X, U, d_p and write X', U':
    # (4 d + 1) * 8; moment, force and tap traffic count as overhead against it
    return (4 * d + 1) * 8


def stencil_cell_bytes(q, d, precision):
    # context only, not the roofline's figure: per lattice cell inside some
    # particle's delta stencil, the Q populations an interpolation of the
    # populations reads and the d force components the spreading writes
    s = 8 if precision == "fp64" else 4
    return q * s + d * s


def stencil_cells(X, n, width):
    """Number of distinct lattice cells covered by the particles' width-point
    delta stencils (walls drop the outside nodes)."""
    import numpy as np
    n = np.asarray(n[:X.shape[1]])
    first = np.floor(X - 0.5).astype(np.int64) - (1 if width == 4 else 0)
    ids = None
    for offs in np.ndindex(*([width] * X.shape[1])):
        c = first + np.asarray(offs)
        ok = np.all((c >= 0) & (c < n), axis=1)
        flat = np.zeros(len(X), dtype=np.int64)
        stride = 1
        for k in range(X.shape[1]):
            flat += c[:, k] * stride
            stride *= int(n[k])
        flat = flat[ok]
        ids = flat if ids is None else np.concatenate([ids, flat])
    return int(np.unique(ids).size)


FP64_OPS_FILE = os.path.join(ROOT, "profiles", "fp64_collide_ops.json")


def collide_fp64_ops(q):
    """FP64 flops per cell of the fused collision (FMA = 2) and the ceiling of
    its instruction mix on the FP64 pipe (2 instructions per clock per SM): from
    the committed ncu instruction counts for D2Q9, else an estimate from the
    kernel's arithmetic scaled by q (marked as such)."""
    try:
        with open(FP64_OPS_FILE) as fh:
            ent = json.load(fh)["d2q9"]
        pc = ent["per_cell"]
        fl, ins, src = pc["flops"], pc["instructions"], "ncu instruction counts"
    except Exception:
        fl, ins, src = 136, 95, "estimate"
    if q != 9:
        fl, ins, src = fl * q / 9.0, ins * q / 9.0, "D2Q9 counts scaled by q/9 (estimate)"
    ceiling = 2.0 * (fl / ins) * 152 * 2.07e9 / 1e12
    return fl, ceiling, src


def warmup_steps(args):
    """W rounded up to a whole number of step graphs (graph_length: the rebuild
    period if even, else twice it)."""
    r = max(int(args.rebin), 1)
    glen = r if r % 2 == 0 else 2 * r
    return -(-int(args.warmup) // glen) * glen


def max_over_ranks(v, dist, device="cuda"):
    """This rank's v -> the maximum over all ranks (v itself in a single process)."""
    if dist is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, units, ms):
    """Whole-job throughput: the units every rank processed in one step over the
    slowest rank's time per step (ms)."""
    return world * units / (ms * 1e-3)


def replica_seed(seed, rank):
    """Each rank sediments its own independent instance (replicas, no exchange)."""
    return seed + 1000 * rank


def run_gpu(args, rank, world):
    import torch
    from paper_1407_6704_gb300 import build
    from paper_1407_6704_gb300.inputs import preset, workload_particles
    from paper_1407_6704_gb300.pibm import Pibm

    build.build()
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = preset(args.workload)
    w.seed = replica_seed(w.seed, rank)
    X, dia, rr = workload_particles(w)
    n_stencil = stencil_cells(X, w.n, w.delta_width)
    peak_gbs, peak_src = _peaks()
    props = torch.cuda.get_device_properties(local)
    dev_id = str(getattr(props, "uuid", local))
    if dev_id and not dev_id.startswith("GPU-") and "-" in dev_id:
        dev_id = "GPU-" + dev_id

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def rank_max(v):
        return max_over_ranks(v, dist)

    results = {}
    clocks = None
    for prec in [args.precision] + [p for p in ("fp64", "fp32") if p != args.precision]:
        sim = Pibm.from_workload(w, precision=prec, particles=(X, dia, rr),
                                 rebin_every=args.rebin)
        stream = sim.stream
        # at least W warm-up steps, rounded up to whole step graphs (one or two
        # cell-list rebuild periods), so that the timed steps replay the graphs from
        # the start of a period instead of launching kernel by kernel up to it
        sim.step(warmup_steps(args))
        n_launch0 = sim.launch_count
        # timed region: K steps through pibm_step (CUDA graphs of one or two cell-list
        # rebuild periods), CUDA events on the handle's stream, barrier + synchronise
        # on both sides
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        sampler = ClockSampler(dev_id) if prec == args.precision else None
        if sampler:
            sampler.__enter__()
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        barrier()
        if sampler:
            sampler.__exit__(None, None, None)
            clocks = sampler.summary()
        ms_graph = rank_max(e0.elapsed_time(e1) / args.steps)
        launches = sim.launch_count - n_launch0
        # second region: the same steps launched phase by phase with CUDA events
        # between the phases (per-kernel durations for the roofline)
        barrier()
        ph = sim.profile_steps(args.steps)
        barrier()
        st = sim.status()
        kps = sim.kernels_per_step
        sim.close()
        results[prec] = dict(ms=ms_graph, ms_phased=rank_max(ph["total"] / args.steps),
                             phases={k: v / args.steps for k, v in ph.items()}, status=st,
                             kps=kps, launches=launches)
        if not args.both:
            break

    # end to end through the public API with pinned host buffers: create (host ->
    # device upload of the particle set; populations start at rest on the device), K
    # steps, read positions and velocities back to the host
    prec = args.precision

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        return t

    Xp, dp, rp = pinned(X), pinned(dia), pinned(rr)
    outp = {nm: torch.empty(X.shape, dtype=torch.float64, pin_memory=True).numpy()
            for nm in ("x", "u")}
    barrier()
    t0 = time.perf_counter()
    sim = Pibm.from_workload(w, precision=prec, particles=(Xp.numpy(), dp.numpy(), rp.numpy()),
                             rebin_every=args.rebin)
    sim.step(args.steps)
    out = sim.read("x", "u", out=outp)
    sim.close()
    torch.cuda.synchronize()
    e2e_s = rank_max(time.perf_counter() - t0)
    h2d = X.nbytes + dia.nbytes + rr.nbytes
    d2h = out["x"].nbytes + out["u"].nbytes

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None

    r = results[prec]
    cells = w.ncell
    mlups = aggregate_rate(world, cells, r["ms"]) / 1e6
    pups = aggregate_rate(world, w.n_particles, r["ms"])
    # dominant kernel roofline
    ph = r["phases"]
    algo_cell = collide_bytes_per_cell(w.q, prec)
    kern = {
        "collide_stream": dict(kernel="k_collide_stream", ms=ph["collide_stream"],
                               bytes=cells * algo_cell),
        "couple": dict(kernel="k_moments + k_couple", ms=ph["couple"],
                       bytes=w.n_particles * particle_bytes(w.d), stencil_cells=n_stencil,
                       bytes_with_stencil_cells=w.n_particles * particle_bytes(w.d)
                       + n_stencil * stencil_cell_bytes(w.q, w.d, prec)),
        "contacts": dict(kernel="k_contacts", ms=ph["contacts"], bytes=None),
        "bin": dict(kernel="k_bin_* + k_scan_*", ms=ph["bin"], bytes=None),
    }
    for k, v in kern.items():
        v["share"] = v["ms"] / max(ph["total"], 1e-12)  # of the phase-by-phase step
        if v["bytes"]:
            v["achieved_gbs"] = v["bytes"] / (v["ms"] * 1e-3) / 1e9
            v["frac_hbm"] = v["achieved_gbs"] / peak_gbs
        if v.get("bytes_with_stencil_cells"):
            v["achieved_gbs_with_stencil_cells"] = v["bytes_with_stencil_cells"] / (v["ms"] * 1e-3) / 1e9
    dom = max(kern, key=lambda k: kern[k]["ms"])
    if prec == "fp64" and dom == "collide_stream":
        fpc, ceil_, src = collide_fp64_ops(w.q)
        ach = cells * fpc / (ph["collide_stream"] * 1e-3) / 1e12
        roof = {"kernel": "k_collide_stream", "bound": "alu", "achieved": ach,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                "traffic": _traffic("k_collide_stream", f"{args.workload}-{prec}"),
                "peak_source": "nominal FP64 rate (2 FMA/clk/SM x 152 SMs x 2.07 GHz)",
                "flops_per_cell": fpc, "flops_source": src,
                "mix_ceiling_tflops": ceil_, "frac_of_mix_ceiling": ach / ceil_}
    else:
        kk = dom if kern[dom]["bytes"] else "collide_stream"
        ach = kern[kk]["achieved_gbs"]
        name = kern[kk]["kernel"]
        roof = {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak_gbs,
                "unit": "GB/s", "frac": ach / peak_gbs,
                "traffic": _traffic(name, f"{args.workload}-{prec}"),
                "algorithmic_bytes": kern[kk]["bytes"],
                "peak_source": f"{peak_src} copy bandwidth"}
    step_bytes = cells * algo_cell + w.n_particles * particle_bytes(w.d)
    step_roof = {"algorithmic_bytes": step_bytes,
                 "achieved_gbs": step_bytes / (r["ms"] * 1e-3) / 1e9}
    step_roof["frac"] = step_roof["achieved_gbs"] / peak_gbs

    line = {
        "metric": "coupled-step MLUPS (lattice updates/s of the full LBM-PIBM-DEM step)",
        "value": mlups,
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r["ms"],
        "ms_per_step_phased": r["ms_phased"],
        "particle_updates_per_s": pups,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64"}[prec],
        "data": "synthetic (seeded uniform non-overlapping particles, fluid at rest)",
        "config": {"workload": WORKLOAD_DESC, "lattice": "D2Q9", "n": list(w.n),
                   "particles": w.n_particles, "precision": prec,
                   "particle_state": "f64",
                   "particle_update": "f64 (U' - U and g formed in FP64; the FP32-formed "
                                      "update is timed under variants.particle_update_fp32)",
                   "parallelism": f"replicas x{world}",
                   "cell_list_rebuild_every": args.rebin,
                   "warmup_steps_run": warmup_steps(args),
                   "overlap": "auto: on for this 2D lattice (contacts and the particle-free "
                              "tiles' collision on a second stream)",
                   "l2": "inputs larger than L2 (population buffers 2x151 MB f32 / 2x302 MB f64)"},
        "phases_ms_per_step": ph,
        "kernels": kern,
        "roofline": roof,
        "step_roofline": step_roof,
        "clocks": clocks,
        "e2e": {"value": world * cells * args.steps / e2e_s / 1e6, "unit": "MLUPS",
                "seconds": e2e_s, "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": d2h / args.steps,
                "note": "create from pinned host arrays + K steps + read X, U into pinned host arrays"},
        "gpu_launches": r["launches"],
        "status": r["status"],
    }
    for p, rr_ in results.items():
        if p == prec:
            continue
        line[p] = {"ms_per_step": rr_["ms"], "ms_per_step_phased": rr_["ms_phased"],
                   "value": world * cells / (rr_["ms"] * 1e-3) / 1e6, "unit": "MLUPS",
                   "phases_ms_per_step": rr_["phases"], "status": rr_["status"]}
        if p == "fp64":
            fpc, ceil_, src = collide_fp64_ops(w.q)
            a = cells * fpc / (rr_["phases"]["collide_stream"] * 1e-3) / 1e12
            line[p]["collide_roofline"] = {"bound": "alu", "achieved": a,
                                           "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                           "frac": a / FP64_PEAK_TFLOPS,
                                           "flops_per_cell": fpc, "flops_source": src,
                                           "mix_ceiling_tflops": ceil_,
                                           "frac_of_mix_ceiling": a / ceil_}
    # the secondary measurements and the CPU baseline belong to the single-GPU run;
    # a multi-rank (scaling) run reports its replicas' throughput only
    solo = world == 1
    if solo and args.rebin > 1:
        line["every_step_rebuild"] = every_step_bench(args, w, X, dia, rr)
    if solo and args.ensemble:
        line["ensemble"] = ensemble_bench(args)
    if solo and args.adjoint:
        line["adjoint"] = adjoint_bench()
    if solo and args.mixed:
        line["mixed_precision_3d"] = mixed_precision_bench(args)
    if solo and args.variants:
        line["variants"] = variants_bench(args, w, X, dia, rr)
    if solo and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, w)
    if dist is not None:
        dist.destroy_process_group()
    return line


def ensemble_bench(args, k=None):
    """The batched ensemble (64 independent 2D instances, 64^2..512^2, FP32), K
    steps each way:
    - persistent: one cooperative kernel launch per 10 steps of all members
      (replayed from a CUDA graph), launch shape autotuned on real steps first;
      also with the default shape, and with every member keeping its cell list
      for 10 steps;
    - branches: one graph launch per two steps, one branch of ordinary step
      kernels per member;
    - one by one: each member stepped in turn through its own graphs, after each
      member's stream-collide block shape is autotuned."""
    import torch
    from paper_1407_6704_gb300.inputs import ensemble_workloads
    from paper_1407_6704_gb300.pibm import Ensemble, Pibm

    ws = ensemble_workloads()
    k = k or min(max(args.steps, 20), 400)
    cells = sum(w.ncell for w, _ in ws)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(step, stream):
        torch.cuda.synchronize()
        e0.record(stream)
        step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    sims = [Pibm.from_workload(w, precision="fp32", particles=p) for w, p in ws]
    for s in sims:
        s.autotune()
        s.step(args.warmup)

    def one_by_one(n):
        for s in sims:
            s.step(n)

    ms_seq = timed(one_by_one, torch.cuda.current_stream())
    ens = Ensemble(sims)
    out = {"persistent_info": ens.info()}
    ens.set_mode(False)
    ens.step(args.warmup + (args.warmup % 2))
    ms_branch = timed(ens.step, ens.stream)
    ens.set_mode(True)
    ens.step(max(args.warmup, 10))
    ms_default = timed(ens.step, ens.stream)
    l0 = ens.launch_count()
    choice = ens.autotune(steps_per_candidate=10)
    ens.step(10)
    l1 = ens.launch_count()
    ms_ens = timed(ens.step, ens.stream)
    launches = ens.launch_count() - l1
    status = ens.status()
    ens.close()
    for s in sims:
        s.close()
    # every member keeping its cell list for 10 steps (persistent only)
    sims = [Pibm.from_workload(w, precision="fp32", particles=p, rebin_every=10) for w, p in ws]
    ens = Ensemble(sims)
    ens.configure(choice["ctas_per_sm"], choice["cells_per_item"])
    ens.step(max(args.warmup, 10))
    ms_kept = timed(ens.step, ens.stream)
    status_kept = ens.status()
    ens.close()
    for s in sims:
        s.close()
    mlups = lambda ms: cells / (ms * 1e-3) / 1e6  # noqa: E731
    out.update({
        "workload": "64 independent 2D D2Q9 sedimentation instances, sides 64..512 "
                    "log-uniform, 100..20k particles, tau 0.55..1.0, ratio 1.5..3.0, "
                    "d 0.5, 2-point delta, FP32, cell list rebuilt every step",
        "cells": cells, "particles": sum(w.n_particles for w, _ in ws), "steps": k,
        "mode": "persistent", "autotuned": choice, "launches_in_timed_region": launches,
        "autotune_launches": l1 - l0,
        "ms_per_step": ms_ens, "value": mlups(ms_ens), "unit": "MLUPS",
        "persistent_default_shape_ms_per_step": ms_default,
        "persistent_default_shape_value": mlups(ms_default),
        "branches_ms_per_step": ms_branch, "branches_value": mlups(ms_branch),
        "members_one_by_one_ms_per_step": ms_seq, "members_one_by_one_value": mlups(ms_seq),
        "persistent_cell_list_kept_10_ms_per_step": ms_kept,
        "persistent_cell_list_kept_10_value": mlups(ms_kept),
        "status": status, "status_kept": status_kept})
    return out


def every_step_bench(args, w, X, dia, rr):
    """The headline configuration with the cell list rebuilt every step, for
    comparison (same physics; the rebuild period only changes the work)."""
    import torch
    from paper_1407_6704_gb300.pibm import Pibm

    sim = Pibm.from_workload(w, precision=args.precision, particles=(X, dia, rr), rebin_every=1)
    sim.step(args.warmup)
    k = min(args.steps, 1000)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(sim.stream)
    sim.step(k)
    e1.record(sim.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / k
    st = sim.status()
    sim.close()
    return {"steps": k, "ms_per_step": ms, "value": w.ncell / (ms * 1e-3) / 1e6,
            "unit": "MLUPS", "status": st}


def _timed_steps(sim, warmup, steps):
    import torch

    sim.step(warmup)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(sim.stream)
    sim.step(steps)
    e1.record(sim.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def variants_bench(args, w, X, dia, rr, steps=200):
    """The paper's variants on the headline workload (c2, FP32 storage): the
    particle update formed in FP32 (the headline forms it in FP64), the
    4-point Lagrange interpolant (Eq. 5), the Hertz normal contact (Eq. 15, E = 0.1,
    nu = 0.3 in lattice units), and Hertz with 4 DEM sub-steps per fluid step (with
    the every-step cell list that sub-cycling needs). A variant that fails reports
    its error instead of a time."""
    import torch
    from paper_1407_6704_gb300.pibm import Pibm

    specs = {
        # the headline configuration with the particle update formed in FP32
        "particle_update_fp32": dict(particle_update="fp32", rebin_every=args.rebin),
        "lagrange4": dict(interp="lagrange4", rebin_every=args.rebin),
        "hertz": dict(contact="hertz", young=0.1, poisson=0.3, rebin_every=args.rebin),
        "hertz_substeps4": dict(contact="hertz", young=0.1, poisson=0.3, substeps=4,
                                rebin_every=1),
    }
    out = {"workload": WORKLOAD_DESC, "precision": "fp32", "steps": steps}
    for name, kw in specs.items():
        try:
            sim = Pibm.from_workload(w, precision="fp32", particles=(X, dia, rr), **kw)
            ms = _timed_steps(sim, 2 * max(kw["rebin_every"], 2), steps)
            out[name] = {"ms_per_step": ms, "value": w.ncell / (ms * 1e-3) / 1e6,
                         "unit": "MLUPS", "status": sim.status()}
            sim.close()
        except Exception as e:  # reported, not fatal to the benchmark line
            out[name] = {"error": str(e)[:200]}
        torch.cuda.empty_cache()
    return out


def mixed_precision_bench(args, steps=40):
    """The 3D workload of the mixed-precision storage modes: D3Q19 256^3, walls,
    tau 0.55, 4M particles (d 0.6, density ratio 2) in the top half, cell list
    rebuilt every 10 steps, with FP32, FP16 and BF16 population storage
    (particles FP64 throughout). Per mode: the step time through graphs, the
    phase-by-phase split, and the collision against its 2 Q s bytes per cell."""
    import torch
    from paper_1407_6704_gb300.inputs import preset, workload_particles
    from paper_1407_6704_gb300.pibm import Pibm

    w = preset("c3")
    X, dia, rr = workload_particles(w)
    peak_gbs, peak_src = _peaks()
    out = {"workload": "D3Q19 256^3 walls, tau 0.55, 4M particles d 0.6 ratio 2 in the top half, "
                       "4-point delta", "cells": w.ncell, "particles": w.n_particles,
           "steps": steps, "cell_list_rebuild_every": args.rebin}
    for prec in ("fp32", "fp16", "bf16"):
        sim = Pibm.from_workload(w, precision=prec, particles=(X, dia, rr), rebin_every=args.rebin)
        sim.step(2 * args.rebin)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(sim.stream)
        sim.step(steps)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        k = 10
        ph = {key: v / k for key, v in sim.profile_steps(k).items()}
        gbs = w.ncell * collide_bytes_per_cell(w.q, prec) / (ph["collide_stream"] * 1e-3) / 1e9
        out[prec] = {"ms_per_step": ms, "value": w.ncell / (ms * 1e-3) / 1e6, "unit": "MLUPS",
                     "phases_ms_per_step": ph,
                     "collide_bytes_per_cell": collide_bytes_per_cell(w.q, prec),
                     "collide_gbs": gbs, "collide_frac": gbs / peak_gbs,
                     "status": sim.status()}
        sim.close()
        torch.cuda.empty_cache()
    # the paper's own 3D velocity set on the same workload, FP32 storage
    try:
        sim = Pibm("d3q15", w.n, w.periodic, w.tau, gravity=w.gravity, delta_width=w.delta_width,
                   precision="fp32", kn=w.kn, restitution=w.restitution, x0=X, diameter=dia,
                   density_ratio=rr, rebin_every=args.rebin)
        ms = _timed_steps(sim, 2 * args.rebin, steps)
        out["d3q15_fp32"] = {"ms_per_step": ms, "value": w.ncell / (ms * 1e-3) / 1e6,
                             "unit": "MLUPS", "status": sim.status()}
        sim.close()
    except Exception as e:  # reported, not fatal to the benchmark line
        out["d3q15_fp32"] = {"error": str(e)[:200]}
    torch.cuda.empty_cache()
    out["peak_source"] = f"{peak_src} copy bandwidth"
    return out


def adjoint_bench(steps=500, K=50):
    """The differentiable configuration: D3Q19 96^3, 20k particles, FP64, the
    gradient of the mean settling velocity after 500 steps with respect to tau,
    the density ratios and the initial positions (checkpoints every 50 steps),
    timed against the forward run alone (wall clock around each call)."""
    import torch
    from paper_1407_6704_gb300.inputs import preset, workload_particles
    from paper_1407_6704_gb300.pibm import settling_gradient

    w = preset("c5")
    X, dia, rr = workload_particles(w)
    kw = dict(gravity=w.gravity, delta_width=w.delta_width, kn=w.kn, restitution=w.restitution,
              x0=X, diameter=dia, density_ratio=rr)
    settling_gradient("d3q19", w.n, w.periodic, w.tau, 20, checkpoint_every=10, **kw)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = settling_gradient("d3q19", w.n, w.periodic, w.tau, steps, checkpoint_every=K, **kw)
    t1 = time.perf_counter()
    f = settling_gradient("d3q19", w.n, w.periodic, w.tau, steps, grads=False, **kw)
    t2 = time.perf_counter()
    return {"workload": "D3Q19 96^3 walls, tau 0.7, 20k particles d 0.5 ratio 2, FP64, 500 steps",
            "checkpoint_every": K, "loss": g["loss"], "dloss_dtau": g["dtau"],
            "gradient_s": t1 - t0, "forward_s": t2 - t1,
            "gradient_over_forward": (t1 - t0) / (t2 - t1),
            "loss_matches_forward": g["loss"] == f["loss"]}


def cpu_sample(w, side=256):
    """A side x side patch of the workload with the same particle density."""
    from paper_1407_6704_gb300.inputs import sample_particles
    frac = (side * side) / float(w.ncell)
    npart = int(round(w.n_particles * frac))
    X, dia, rr = sample_particles((side, side), npart, w.diameter, w.density_ratio, w.band,
                                  w.seed)
    return (side, side), X, dia, rr


def cpu_info():
    """(logical cores, CPU model) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return os.cpu_count() or 1, model or "unknown"


def _timed_oracle(o, budget_s, max_steps=None):
    """Steps of the oracle o for about budget_s seconds: (steps, seconds)."""
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s and (max_steps is None or steps < max_steps):
        o.step(1)
        steps += 1
    return steps, time.perf_counter() - t0


def cpu_baseline(args, w, budget_s=8.0):
    """The oracle (test infrastructure, FP64, brute-force contacts) timed on this
    host's cores on bounded samples of the workloads: the serial build and the
    OpenMP build (cell loops and per-particle updates on every core, the spreading
    serial; bitwise equal results). The headline figure is the OpenMP build on a
    256^2 patch of the benchmark workload with its particle density. The full-size
    lattices of the 2048^2 and 256^3 workloads are timed for the fluid step alone:
    with particles, the brute-force contact search alone would test N^2 pairs per
    step (2.5e11 and 1.6e13); their particle phase is projected from the per-pair
    cost measured here."""
    from oracle.oracle import Oracle
    from paper_1407_6704_gb300.inputs import preset, sample_particles

    nproc, model = cpu_info()
    legs = {}
    n, X, dia, rr = cpu_sample(w)
    kw = dict(delta_width=w.delta_width, gravity=w.gravity, kn=w.kn, restitution=w.restitution,
              x0=X, diameter=dia, density_ratio=rr)
    for par in (False, True):
        o = Oracle(w.q, n, w.periodic, w.tau, parallel=par, **kw)
        o.step(1)
        steps, dt = _timed_oracle(o, budget_s)
        legs["patch_" + ("openmp" if par else "serial")] = {
            "threads": nproc if par else 1, "steps": steps, "seconds": dt,
            "mlups": n[0] * n[1] * steps / dt / 1e6,
            "particle_updates_per_s": len(X) * steps / dt}
    # the per-pair cost of the brute-force contact search: the patch with and
    # without its particles (OpenMP)
    o = Oracle(w.q, n, w.periodic, w.tau, parallel=True, delta_width=w.delta_width)
    o.step(1)
    steps, dt_fluid = _timed_oracle(o, 2.0)
    sec_fluid = dt_fluid / steps
    sec_with = 1.0 / (legs["patch_openmp"]["mlups"] * 1e6 / (n[0] * n[1]))
    pair_s = max(sec_with - sec_fluid, 0.0) / float(len(X)) ** 2
    # the 128^2 workload in full: 200 particles, 2-point kernel, 1000 steps
    c1 = preset("c1")
    X1, d1, r1 = sample_particles(c1.n, c1.n_particles, c1.diameter, c1.density_ratio, c1.band,
                                  c1.seed)
    o = Oracle(c1.q, c1.n, c1.periodic, c1.tau, parallel=True, delta_width=c1.delta_width,
               gravity=c1.gravity, kn=c1.kn, restitution=c1.restitution, x0=X1, diameter=d1,
               density_ratio=r1)
    t0 = time.perf_counter()
    o.step(c1.steps)
    dt = time.perf_counter() - t0
    legs["c1_full_1000_steps"] = {"threads": nproc, "seconds": dt,
                                  "mlups": c1.ncell * c1.steps / dt / 1e6}
    # full-size lattices, fluid step alone, and the projected particle phase
    for name in ("c2", "c3"):
        wf = preset(name)
        o = Oracle(wf.q, wf.n, wf.periodic, wf.tau, parallel=True, delta_width=wf.delta_width)
        steps, dt = _timed_oracle(o, 1.0, max_steps=2)
        fl = dt / steps
        proj = fl + pair_s * float(wf.n_particles) ** 2
        legs[name + "_full_size"] = {
            "threads": nproc, "cells": wf.ncell, "particles": wf.n_particles,
            "fluid_step_seconds": fl, "fluid_mlups": wf.ncell / fl / 1e6,
            "projected_step_seconds_with_particles": proj,
            "projected_mlups_with_particles": wf.ncell / proj / 1e6}
        del o
    # the 64^3 slice of the 256^3 workload (62,500 particles), OpenMP, 2 steps
    ws = preset("c3s")
    Xs, ds, rs = sample_particles(ws.n, ws.n_particles, ws.diameter, ws.density_ratio, ws.band,
                                  ws.seed)
    o = Oracle(ws.q, ws.n, ws.periodic, ws.tau, parallel=True, delta_width=ws.delta_width,
               gravity=ws.gravity, kn=ws.kn, restitution=ws.restitution, x0=Xs, diameter=ds,
               density_ratio=rs)
    steps, dt = _timed_oracle(o, 1.0, max_steps=2)
    legs["c3_slice_64cubed"] = {"threads": nproc, "steps": steps, "seconds": dt,
                                "mlups": ws.ncell * steps / dt / 1e6,
                                "particle_updates_per_s": ws.n_particles * steps / dt}
    head = legs["patch_openmp"]
    return {"value": head["mlups"], "unit": "MLUPS", "cores": nproc, "kind": "oracle",
            "sample": f"{n[0]}x{n[1]} patch of the workload with the same particle density "
                      f"({len(X)} particles), OpenMP build on all {nproc} cores, "
                      f"{head['steps']} steps in {head['seconds']:.1f} s",
            "particle_updates_per_s": head["particle_updates_per_s"],
            "nproc": nproc, "cpu_model": model, "pair_test_seconds": pair_s, "legs": legs}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_1407_6704_gb300.inputs import preset
    w = preset(args.workload)
    from oracle.oracle import Oracle
    # keep the whole reference run within a few minutes: the oracle's brute-force
    # contacts make a step cost grow with the square of the patch's particle count
    total = args.steps + max(args.warmup, 0)
    side = 256 if total <= 200 else (128 if total <= 4000 else 64)
    n, X, dia, rr = cpu_sample(w, side)
    nproc, model = cpu_info()
    o = Oracle(w.q, n, w.periodic, w.tau, delta_width=w.delta_width, gravity=w.gravity,
               kn=w.kn, restitution=w.restitution, x0=X, diameter=dia, density_ratio=rr,
               parallel=True)
    o.step(max(args.warmup, 0))
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    cells = n[0] * n[1]
    v = cells * args.steps / dt / 1e6
    return {"impl": "reference", "metric": "coupled-step MLUPS (lattice updates/s of the full "
            "LBM-PIBM-DEM step)", "value": v, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_DESC, "lattice": "D2Q9",
                                            "n": list(n), "particles": len(X)},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": nproc, "kind": "oracle",
                             "cpu_model": model,
                             "sample": f"{n[0]}x{n[1]} patch with the workload's particle "
                                       f"density ({len(X)} particles), OpenMP build of the "
                                       f"oracle on all {nproc} cores"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_profile_only(args):
    """A few steps launched phase by phase (the driver for ncu captures)."""
    import torch
    from paper_1407_6704_gb300 import build
    from paper_1407_6704_gb300.inputs import preset, workload_particles
    from paper_1407_6704_gb300.pibm import Pibm

    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    if args.workload == "ensemble":
        # the 64-member ensemble through the persistent kernel (10 steps a launch)
        from paper_1407_6704_gb300.inputs import ensemble_workloads
        from paper_1407_6704_gb300.pibm import Ensemble
        sims = [Pibm.from_workload(w, precision="fp32", particles=p, rebin_every=args.rebin)
                for w, p in ensemble_workloads()]
        ens = Ensemble(sims)
        ens.step(args.warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ens.stream)
        ens.step(args.steps)
        e1.record(ens.stream)
        torch.cuda.synchronize()
        print(json.dumps({"workload": "ensemble", "info": ens.info(),
                          "ms_per_step": e0.elapsed_time(e1) / args.steps,
                          "status": ens.status()}))
        ens.close()
        for s_ in sims:
            s_.close()
        return
    w = preset(args.workload)
    X, dia, rr = workload_particles(w)
    sim = Pibm.from_workload(w, precision=args.precision, particles=(X, dia, rr),
                             rebin_every=args.rebin)
    if args.graph:
        # the timed path: steps through pibm_step (graphs, overlap as configured)
        sim.step(args.warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.step(args.steps)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        print(json.dumps({"workload": args.workload, "precision": args.precision,
                          "ms_per_step": e0.elapsed_time(e1) / args.steps,
                          "kernels_per_rebuild_step": sim.kernels_per_step,
                          "status": sim.status()}))
        sim.close()
        return
    sim.profile_steps(args.warmup)
    ph = sim.profile_steps(args.steps)
    print(json.dumps({"workload": args.workload, "precision": args.precision,
                      "phases_ms_per_step": {k: v / args.steps for k, v in ph.items()},
                      "status": sim.status()}))
    sim.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--precision", choices=["fp32", "fp64", "fp16", "bf16"], default="fp32")
    ap.add_argument("--both", type=int, default=1, help="also time the other precision")
    ap.add_argument("--rebin", type=int, default=10,
                    help="cell-list rebuild period in steps (skin-checked on the device)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ensemble", type=int, default=1, help="also time the 64-member ensemble")
    ap.add_argument("--adjoint", type=int, default=1,
                    help="also time the 500-step gradient of the 96^3 FP64 configuration")
    ap.add_argument("--mixed", type=int, default=1,
                    help="also time the 256^3 3D workload in FP32, FP16 and BF16 storage")
    ap.add_argument("--variants", type=int, default=1,
                    help="also time the Lagrange, Hertz and sub-cycled variants on the workload")
    ap.add_argument("--profile-only", action="store_true",
                    help="only run --steps phase-by-phase steps (ncu driver); prints phase times")
    ap.add_argument("--graph", action="store_true",
                    help="with --profile-only: run the steps through pibm_step (graphs) instead")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.gpus != world and world > 1:
        ap.error("--gpus must equal WORLD_SIZE under torchrun")
    if args.profile_only:
        run_profile_only(args)
        return
    line = run_reference(args, rank, world) if args.impl == "reference" else \
        run_gpu(args, rank, world)
    if line is not None and rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
