#!/usr/bin/env python3
"""Particle-pushes/s of the RelSIM step on the 2D relativistic double Harris
sheet, 1024 x 512 cells, 64 particles per cell per species (67.1M particles),
FP32 form; with the HBM roofline of the dominant kernel, the FP64 form on the
same GPU, an end-to-end figure through host buffers, and the FP64 CPU oracle
timed on a bounded sample as a reported baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one pass of the whole hot path: deposit of the predicted current
and mass matrices, the GMRES field solve with the field update, the push
with the cell re-sort, and the energy ledger. Inputs stay resident in HBM
for the headline value; they are far larger than L2 (1.6 GB of particles),
so no L2 flush is needed between steps. With N > 1 (torchrun) every rank runs
an independent replica (the workload is one periodic domain; the path is
not sharded), and the value is the total over ranks.
"""
from __future__ import annotations

import argparse
import csv
import ctypes
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-pushes/s incl. mass-matrix build, % HBM roofline, FP32 vs FP64 form"
UNIT = "particle-pushes/s"

WORKLOAD = {
    "workload": "2D relativistic double Harris sheet, pair plasma, 1024x512 cells (dx=dy=1 d_e), "
                "64 ppc per species (67,108,864 particles), sigma=10, theta_T=0.3, delta=1 d_e, "
                "dt=1/omega_pe, theta=0.5, 1% B_y perturbation, seed 0",
    "nx": 1024, "ny": 512, "ppc_per_species": 64, "particles": 67108864,
    "form": "FP32 particles/fields/mass matrix, GMRES vectors as double-float pairs (FP32 arithmetic, ~48-bit values), FP64 ledger",
    "gmres_tol": 1e-6, "gmres_restart": 30,
    "l2": "inputs larger than L2 (1.6 GB of particle data per step), no flush",
}


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


SMALL = {"nx": 512, "ny": 256, "ppc_per_species": 64, "particles": 16777216}


def harris_config(seed=0, small=False):
    from relsim_inputs import HarrisConfig
    nx, ny = (SMALL["nx"], SMALL["ny"]) if small else (1024, 512)
    return HarrisConfig(nx=nx, ny=ny, ppc=64, theta_T=0.3, delta=1.0, sigma=10.0, pert=0.01,
                        dt=1.0, theta=0.5, seed=seed)


def workload_config(small):
    w = dict(WORKLOAD)
    if small:
        w.update(SMALL)
        w["workload"] = w["workload"].replace("1024x512", "512x256").replace("67,108,864", "16,777,216")
        w["profiling_case"] = "reduced grid for profiler captures (not the headline workload)"
    return w


def subsample(state, every):
    """Every `every`-th particle of each species, weights scaled to keep the
    charge and current densities (the bounded CPU-baseline sample)."""
    import numpy as np
    out = dict(state)
    sp = []
    for s in state["species"]:
        d = {k: (v[::every] if isinstance(v, np.ndarray) else v) for k, v in s.items()}
        d["w"] = d["w"] * every
        sp.append(d)
    out["species"] = sp
    return out


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.f.read())) if len(r) >= 9]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def max_over_ranks(x, dist):
    """The largest x over all ranks (NCCL reduces a CUDA tensor, gloo a CPU one)."""
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def traffic_record(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    rec = d.get(kernel)
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2509_11100_gb300", "csrc", rec["source"])
    if kernel_source_hash(src) != rec.get("kernels_sha256_16"):
        return None
    return rec["dram_bytes_per_launch"]


def kernel_source_hash(path):
    """sha256[:16] of a source file's device code: the text before the end of
    its first anonymous namespace, where the kernels and their device helpers
    live (the host launchers that follow do not change what a kernel moves)."""
    text = open(path, "rb").read()
    end = text.find(b"}  // namespace\n")
    return hashlib.sha256(text[:end if end >= 0 else len(text)]).hexdigest()[:16]


def algorithmic_bytes(slot, n_particles, n_per_species, ncell, esz):
    """Bytes a launch of the slot must move (what its job reads and writes)."""
    if slot == "deposit":       # read offsets, u, w; write M (45) + Jhat (3) per node
        return n_particles * 6 * esz + ncell * 48 * esz
    if slot == "push":          # per species: read + write the particle record; runs per cell
        return n_per_species * 12 * esz + ncell * 18 * 4
    if slot == "permute":       # per species: read + write the particle record; run tables
        return n_per_species * 12 * esz + ncell * 19 * 4
    if slot == "gmres_apply":   # M, v (FP64 in), Av (FP64 out)
        return ncell * (45 * esz + 24 + 24)
    if slot == "field_update":
        return ncell * (24 + 45 * esz + 3 * esz * 6)
    return None


def run_ours(args):
    import numpy as np
    import torch
    import paper_2509_11100_gb300 as rs
    from relsim_inputs import make_harris

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    hc = harris_config(seed=rank, small=args.workload == "small")
    t0 = time.time()
    state = make_harris(hc)
    t_gen = time.time() - t0
    n_per = [len(s["w"]) for s in state["species"]]
    N = sum(n_per)
    ncell = hc.nx * hc.ny

    cfg = rs.make_config(hc.nx, hc.ny, dt=hc.dt, theta_implicit=hc.theta, precision=32,
                         gmres_tol=WORKLOAD["gmres_tol"], gmres_restart=WORKLOAD["gmres_restart"],
                         gamma_pred=args.gamma_pred)
    sim = rs.Simulation(cfg)
    sim.load_state(state)
    tuning = sim.autotune() if not args.no_autotune else None
    for _ in range(args.warmup):
        sim.step(ledger=True)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = rs.relsim_kernel_launches()
    ev0.record(stream)
    ledgers = []
    iters = []
    for _ in range(args.steps):
        led, status = sim.step(ledger=True)
        ledgers.append(led)
        iters.append(led["gmres_iters"])
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = rs.relsim_kernel_launches() - launches0
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    graph = sim.graph_info()
    # per-kernel device times: a further pass with event profiling, which
    # drives the same kernels from the host (event pairs around each group)
    kp = max(1, min(args.steps, 20))
    sim.profile(True)
    sim.profile_read(reset=True)
    for _ in range(kp):
        sim.step(ledger=True)
    prof = sim.profile_read(reset=True)
    sim.profile(False)
    if dist is not None:
        ms = max_over_ranks(ms, dist)
    value = world * N / (ms / 1e3)

    # per-kernel times, dominant kernel roofline
    esz = 4
    per_kernel = {k: {"ms_per_step": v[0] / kp, "groups": v[1], "kernels": v[2]}
                  for k, v in prof.items() if v[1] > 0}
    # each kernel group's algorithmic bytes per step over its time: the HBM
    # roofline fraction of every slot that has a byte count
    peak_gbs, _ = measured_peaks()
    for k, v in per_kernel.items():
        if k in ("push", "permute"):
            ab = sum(algorithmic_bytes(k, 0, n, ncell, 4) for n in n_per)
        elif k == "gmres_apply":
            ab = algorithmic_bytes(k, 0, 0, ncell, 4) * v["kernels"] / kp
        else:
            ab = algorithmic_bytes(k, N, 0, ncell, 4)
        if ab:
            gbs = ab / (v["ms_per_step"] / 1e3) / 1e9
            v.update({"algorithmic_bytes_per_step": ab, "achieved_gbs": gbs, "frac": gbs / peak_gbs})
    step_kernel_ms = sum(v["ms_per_step"] for v in per_kernel.values())
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms_per_step"])
    peak, peak_kind = measured_peaks()
    groups_per_step = per_kernel[dom]["groups"] / kp
    launch_ms = per_kernel[dom]["ms_per_step"] / groups_per_step
    ab = algorithmic_bytes(dom, N, n_per[0], ncell, esz)
    achieved = ab / (launch_ms / 1e3) / 1e9 if ab else None
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "peak_source": peak_kind,
                # counters of the kernel variant this run launched
                "traffic": traffic_record(dom + ("_pred" if args.gamma_pred else "")),
                "algorithmic_bytes_per_launch": ab,
                "launch_ms": launch_ms}
    # the mover + mass-matrix kernels together (deposit, push passes, sort tables)
    mover = ("deposit", "push", "sort_tables", "permute")
    mover_ms = sum(per_kernel[k]["ms_per_step"] for k in mover if k in per_kernel)
    mover_bytes = (algorithmic_bytes("deposit", N, 0, ncell, esz)
                   + sum(algorithmic_bytes("push", 0, n, ncell, esz)
                         + algorithmic_bytes("permute", 0, n, ncell, esz) for n in n_per))
    mover_gbs = mover_bytes / (mover_ms / 1e3) / 1e9
    last = ledgers[-1]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(args.workload == "small"),
                       parallelism=f"replicas{world}" if world > 1 else "single",
                       gamma_bar="gamma(u^n + beta E^n(x)) (predicted)" if args.gamma_pred else "gamma(u^n)"),
        "roofline": roofline,
        "mover_mass_matrix": {"value": N / (mover_ms / 1e3), "unit": UNIT, "ms_per_step": mover_ms,
                              "achieved_gbs": mover_gbs, "frac": mover_gbs / peak,
                              "kernels": list(mover)},
        "per_kernel": per_kernel,
        "per_kernel_pass": f"{kp} further steps with event profiling (host-driven route, same kernels)",
        "kernel_ms_per_step": step_kernel_ms,
        "step_graph": {"graph_steps": graph["graph_steps"], "disabled": graph["disabled"],
                       "why": graph["why"] or None},
        "autotune": tuning,
        "gpu_launches": int(launches),
        "gmres_iters_per_step": statistics.mean(iters),
        "ledger": {"residual_rel": abs(last["residual"]) / last["total"],
                   "mismatch_rel": abs(last["mismatch"]) / last["total"],
                   "gmres_relres": last["gmres_relres"]},
        "clocks": clk,
        "input_generation_s": t_gen,
    }

    # the particle spectrum of the final state (a diagnostic, not part of the
    # step): 256 log bins of gamma - 1 over [1e-2, 1e4], both species
    edges = np.geomspace(1e-2, 1e4, 257)
    sim.spectrum(0, edges, 0)
    sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sa.record(stream)
    spec = [sim.spectrum(s, edges, 0, device=True) for s in range(len(n_per))]
    sb.record(stream)
    torch.cuda.synchronize()
    cnt = sum(c.cpu().numpy() for _, c in spec)
    out["spectrum"] = {"bins": 256, "variable": "gamma-1", "range": [1e-2, 1e4], "ms": sa.elapsed_time(sb),
                       "particles_binned": int(cnt.sum()),
                       "peak_bin_gamma_minus_1": float(np.sqrt(edges[:-1] * edges[1:])[int(np.argmax(cnt[1:-1]))])}

    # end to end through the C ABI with host buffers: every step loads the
    # state from pinned host memory, steps, and reads the ledger back
    if not args.no_e2e:
        pinned = []
        for s in state["species"]:
            x = torch.from_numpy(np.stack([s["x"], s["y"]], axis=1)).pin_memory()
            u = torch.from_numpy(np.stack([s["ux"], s["uy"], s["uz"]], axis=1)).pin_memory()
            w = torch.from_numpy(np.ascontiguousarray(s["w"])).pin_memory()
            pinned.append((x, u, w))
        E = torch.from_numpy(np.ascontiguousarray(state["E"])).pin_memory()
        B = torch.from_numpy(np.ascontiguousarray(state["B"])).pin_memory()
        h2d = sum(x.numel() * 8 + u.numel() * 8 + w.numel() * 8 for x, u, w in pinned)
        h2d += (E.numel() + B.numel()) * 8
        d2h = ctypes.sizeof(rs.relsim_energy)

        def e2e_step():
            for s, (x, u, w) in enumerate(pinned):
                sim.load_species(s, x, u, w)
            sim.set_fields(E, B)
            led, _ = sim.step(ledger=True)
            return led

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        ke = max(1, min(args.steps, 5))
        t1 = time.perf_counter()
        for _ in range(ke):
            e2e_step()
        torch.cuda.synchronize()
        te_serial = (time.perf_counter() - t1) / ke
        # pipelined: two contexts on streams of their own, each step's inputs
        # copied host -> device (copy engine, pinned memory) into one of two
        # device buffers while the other context steps on the previous ones;
        # every step still copies its full inputs and reads its ledger back
        cstream = [torch.cuda.Stream(), torch.cuda.Stream()]
        sstream = [torch.cuda.Stream(), torch.cuda.Stream()]
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        sims = [rs.Simulation(cfg, stream=sstream[0].cuda_stream), rs.Simulation(cfg, stream=sstream[1].cuda_stream)]

        def pipelined(flat, load):
            """Seconds per step of the two-context pipeline; load(sim, device
            buffers) hands one step's inputs to a context."""
            dbuf = [[torch.empty(t.shape, dtype=t.dtype, device="cuda") for t in flat] for _ in range(2)]

            def copy_in(k):
                with torch.cuda.stream(cstream[k]):
                    for d, h in zip(dbuf[k], flat):
                        d.copy_(h, non_blocking=True)
                    ready[k].record(cstream[k])

            def run(k):
                sstream[k].wait_event(ready[k])
                with torch.cuda.stream(sstream[k]):
                    load(sims[k], dbuf[k])
                    led, _ = sims[k].step(ledger=True)
                # the buffer may be refilled once this step has read it
                cstream[k].wait_stream(sstream[k])
                return led

            copy_in(0)
            copy_in(1)
            run(0)
            run(1)   # warm-up: sizes both contexts
            torch.cuda.synchronize()
            barrier()
            copy_in(0)
            t1 = time.perf_counter()
            for t in range(2 * ke):
                if t + 1 < 2 * ke:
                    copy_in((t + 1) % 2)   # the next step's inputs while this one runs
                run(t % 2)
            torch.cuda.synchronize()
            te = (time.perf_counter() - t1) / (2 * ke)
            del dbuf
            return max_over_ranks(te, dist) if dist is not None else te

        nsp = len(pinned)

        def load_record(sm, d):
            for s_ in range(nsp):
                sm.load_species(s_, d[3 * s_], d[3 * s_ + 1], d[3 * s_ + 2])
            sm.set_fields(d[-2], d[-1])

        te_rec = pipelined([t for trio in pinned for t in trio] + [E, B], load_record)
        del pinned
        # the same inputs in the library's own form (cell start table, FP32
        # offsets, momenta and weights: 24 bytes a particle against the FP64
        # record's 48), read out once from a context that loaded the record
        sims[0].load_state(state)
        native = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in sims[0].particles_native(s_)]
                  for s_ in range(nsp)]
        flat_n = [t for quad in native for t in quad] + [E, B]
        h2d_n = sum(t.numel() * t.element_size() for t in flat_n)

        def load_native(sm, d):
            for s_ in range(nsp):
                sm.load_species_native(s_, *d[4 * s_:4 * s_ + 4])
            sm.set_fields(d[-2], d[-1])

        te = pipelined(flat_n, load_native)
        for sm in sims:
            sm.close()
        if dist is not None:
            te_serial = max_over_ranks(te_serial, dist)
        # the headline end-to-end figure goes through the boundary's FP64
        # record (relsim_load_particles: absolute FP64 positions, converted
        # and sorted inside the library); the library's own form follows
        out["e2e"] = {"value": world * N / te_rec, "unit": UNIT, "ms_per_step": te_rec * 1e3,
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                      "steps": 2 * ke,
                      "mode": "pipelined: two contexts, each step's inputs (the FP64 particle record of the "
                              "C ABI: absolute positions, momenta, weights; FP64 E and B) copied from pinned "
                              "host memory while the other context steps, loaded by relsim_load_particles "
                              "(conversion and cell sort on the device) and relsim_set_fields, then "
                              "relsim_step and the ledger read back",
                      "native_form": {"value": world * N / te, "ms_per_step": te * 1e3,
                                      "h2d_bytes_per_step": int(h2d_n), "steps": 2 * ke,
                                      "mode": "the same pipeline with the particles in the library's own form "
                                              "(cell start table, FP32 offsets, momenta, weights: 24 bytes a "
                                              "particle), loaded by relsim_load_particles_native"},
                      "serial": {"value": world * N / te_serial, "ms_per_step": te_serial * 1e3, "steps": ke,
                                 "h2d_bytes_per_step": int(h2d),
                                 "mode": "one context, FP64 record, copy and step in turn"}}
        del native
    sim.close()
    del sim

    # the FP64 form on the same GPU and workload
    if not args.no_fp64:
        cfg64 = rs.make_config(hc.nx, hc.ny, dt=hc.dt, theta_implicit=hc.theta, precision=64,
                               gmres_tol=1e-10, gmres_restart=WORKLOAD["gmres_restart"], gamma_pred=args.gamma_pred)
        s64 = rs.Simulation(cfg64)
        s64.load_state(state)
        s64.step()
        torch.cuda.synchronize()
        k64 = max(1, min(args.steps, 3))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k64):
            led64, _ = s64.step(ledger=True)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b) / k64
        out["fp64_form"] = {"value": N / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                            "steps": k64, "gmres_tol": 1e-10,
                            "ledger_residual_rel": abs(led64["residual"]) / led64["total"],
                            "speedup_fp32_over_fp64": ms64 / ms}
        s64.close()

    # the FP64 CPU oracle, as it stands, on a bounded sample of the workload
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_baseline(state, hc, steps=2, gamma_pred=args.gamma_pred)

    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def oracle_baseline(state, hc, steps=2, every=8, gamma_pred=0):
    """Time the FP64 CPU oracle on the workload's grid with every 8th particle
    of each cell (8 ppc per species, 8.4M particles, weights x8)."""
    import oracle
    sample = subsample(state, every)
    c = oracle.make_config(hc.nx, hc.ny, dt=hc.dt, theta=hc.theta, gmres_tol=1e-12, gmres_restart=50,
                           gamma_pred=gamma_pred)
    P = oracle.Particles(sample["species"])
    n = int(P.off[-1])
    E, B = sample["E"], sample["B"]
    t0 = time.perf_counter()
    for _ in range(steps):
        E, B, led, _ = oracle.step(c, P, E, B)
    dt = time.perf_counter() - t0
    return {"value": n * steps / dt, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"same 1024x512 grid and fields, every {every}th particle of each cell "
                      f"({n} particles, weights x{every}), {steps} full oracle steps "
                      f"(deposit, GMRES tol 1e-12, push), single thread, FP64",
            "seconds": dt}


def run_reference(args):
    rank, world, local = rank_info()
    if rank != 0:
        return
    from relsim_inputs import make_harris
    import oracle
    # the same 1024x512 grid and fields as the GPU arm, a bounded particle
    # sample per step: every 8th particle of each cell (the cpu_baseline
    # sample, ~3 s per oracle step on one core) while steps + warmup <= 40,
    # a sparser sample beyond so the whole run stays within a few minutes
    hc = harris_config(seed=0, small=args.workload == "small")
    state = make_harris(hc)
    every = 8 if args.steps + args.warmup <= 40 else 8 * ((args.steps + args.warmup + 39) // 40)
    sample = subsample(state, every)
    c = oracle.make_config(hc.nx, hc.ny, dt=hc.dt, theta=hc.theta, gmres_tol=1e-12, gmres_restart=50,
                           gamma_pred=args.gamma_pred)
    P = oracle.Particles(sample["species"])
    n = int(P.off[-1])
    E, B = sample["E"], sample["B"]
    for _ in range(args.warmup):
        E, B, led, _ = oracle.step(c, P, E, B)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        E, B, led, _ = oracle.step(c, P, E, B)
    dt = (time.perf_counter() - t0) / args.steps
    value = n / dt
    grid = f"{hc.nx}x{hc.ny}"
    sample_desc = (f"the double Harris sheet of the workload on its {grid} grid, every {every}th particle of "
                   f"each cell ({n} particles, weights x{every}); one full FP64 oracle step (deposit, GMRES "
                   f"tol 1e-12, push) per timed step, single thread")
    cfg = dict(workload_config(args.workload == "small"), parallelism="host cores (oracle)",
               form="FP64 CPU oracle (plain C, single thread): particles, fields, mass matrix and GMRES in FP64",
               gamma_bar="gamma(u^n + beta E^n(x)) (predicted)" if args.gamma_pred else "gamma(u^n)")
    cfg.pop("gmres_tol", None)
    cfg["gmres"] = "tol 1e-12, restart 50"
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"kind": "oracle", "cores": 1, "host_cores": os.cpu_count(), "sample": sample_desc,
                         "value": value, "unit": UNIT},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# Fourier modes of B_y recorded per instance and step in the scan (m = 0 ..
# SCAN_MODES-1): the per-mode growth rates and the dispersion fit
SCAN_MODES = 17
SCAN = {
    "workload": "batched linear tearing scan: 48 independent 2D pair-plasma double Harris sheets, "
                "L_x from {128,192,256,384,512,768} cells (L_y = L_x/2), delta from {0.5,1,2} d_e, "
                "sigma from {1,10,40} (SplitMix64 draws from seed 0), theta_T=0.3, 32 ppc per species, "
                "0.1% B_y perturbation, dt=0.5/omega_pe, theta=0.5",
    "form": "FP32 particles/fields/mass matrix, GMRES vectors as double-float pairs (FP32 arithmetic, ~48-bit values), FP64 ledger",
    "gmres_tol": 1e-6, "gmres_restart": 30,
    "l2": "inputs larger than L2 (about 8 GB of particle data per step), no flush",
}


def lpt_shard(sizes, world):
    """Instances per rank: largest first onto the least-loaded rank."""
    load = [0] * world
    owner = [0] * len(sizes)
    for i in sorted(range(len(sizes)), key=lambda k: -sizes[k]):
        r = min(range(world), key=lambda q: load[q])
        owner[i] = r
        load[r] += sizes[i]
    return owner


def run_scan(args):
    """The 48-instance tearing scan, advanced by the library's batch runner
    (one context and stream per instance, host worker threads); instances
    are sharded whole across ranks (no exchange)."""
    import numpy as np
    import torch
    import paper_2509_11100_gb300 as rs
    from relsim_inputs import make_harris, tearing_scan

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    insts = tearing_scan(48, seed=0)
    sizes = [2 * hc.nx * hc.ny * hc.ppc for hc in insts]
    owner = lpt_shard(sizes, world)
    mine = [i for i in range(len(insts)) if owner[i] == rank]
    t0 = time.time()
    streams, sims = [], []
    for i in mine:
        hc = insts[i]
        st = make_harris(hc)
        stream = torch.cuda.Stream()
        sim = rs.Simulation(rs.make_config(hc.nx, hc.ny, dt=hc.dt, theta_implicit=hc.theta, precision=32,
                                           gmres_tol=SCAN["gmres_tol"], gmres_restart=SCAN["gmres_restart"],
                                           gamma_pred=args.gamma_pred),
                            stream=stream.cuda_stream)
        sim.load_state(st)
        del st
        if not args.no_autotune:
            sim.autotune()
        streams.append(stream)
        sims.append(sim)
    torch.cuda.synchronize()
    t_setup = time.time() - t0
    N = sum(sizes[i] for i in mine)
    batch = rs.Batch(sims, nworkers=args.workers, shared=args.scan_launch == "shared", groups=args.scan_groups)
    batch.run(args.warmup)
    torch.cuda.synchronize()

    # device span: every instance stream waits on ev0; the default stream
    # waits on every instance stream before ev1
    clocks = ClockSampler(local)
    dflt = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = rs.relsim_kernel_launches()
    ev0.record(dflt)
    for st in streams:
        st.wait_event(ev0)
    t1 = time.perf_counter()
    modes, status, iters = batch.run(args.steps, component=1, nmodes=SCAN_MODES)
    wall = time.perf_counter() - t1
    for st in streams:
        e = torch.cuda.Event()
        e.record(st)
        dflt.wait_event(e)
    ev1.record(dflt)
    torch.cuda.synchronize()
    launches = rs.relsim_kernel_launches() - launches0
    path = batch.last_path
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist is not None:
        ms = max_over_ranks(ms, dist)
    total = sum(sizes)
    value = total / (ms / 1e3) if world > 1 else N / (ms / 1e3)
    batch.close()
    for sim in sims:
        sim.close()

    # per instance: the m = 1 B_y mode's energy growth rate over its best
    # 40-step window (the field amplitude grows at half of it), and the
    # per-mode amplitude rates of modes 1 .. SCAN_MODES-1 over one fixed
    # window (steps steps/10 .. 6 steps/10) with their dispersion fit
    # (Sec. 3.1, Fig. 1 b, d: rate = A x b (1 - x^2 b^2), x = k delta)
    rows = []
    win = min(40, args.steps)
    dfirst, dwin = args.steps // 10, args.steps // 2
    for k, i in enumerate(mine):
        hc = insts[i]
        try:
            rate, first = rs.relsim_growth_fit(modes[k, :, 1], hc.dt, win) if win >= 2 else (None, None)
        except rs.RelsimError:
            rate, first = None, None
        disp = None
        if dwin >= 2:
            try:
                rates, A, b = rs.relsim_dispersion_fit(modes[k], hc.dt, dfirst, dwin, hc.nx * hc.dx, hc.delta)
                x = 2 * np.pi * np.arange(SCAN_MODES) * hc.delta / (hc.nx * hc.dx)
                fin = np.isfinite(rates)
                disp = {"window_steps": [dfirst + 1, dfirst + dwin], "ka": [round(float(v), 5) for v in x[1:]],
                        "amplitude_rates": [None if not np.isfinite(v) else float(v) for v in rates[1:]],
                        "fastest_ka": float(x[fin][np.argmax(rates[fin])]) if fin.any() else None,
                        "fit_A": A, "fit_b": b, "fit_peak_ka": 1.0 / (np.sqrt(3.0) * b),
                        "fit_zero_ka": 1.0 / b}
            except rs.RelsimError:
                disp = None
        rows.append({"index": i, "nx": hc.nx, "ny": hc.ny, "delta": hc.delta, "sigma": hc.sigma,
                     "particles": sizes[i], "status": int(status[k]),
                     "gmres_iters_mean": float(np.mean(iters[k])) if args.steps else None,
                     "m1_energy_growth_rate": rate, "fit_window_first_step": first, "dispersion": disp})
    # algorithmic bytes of the particle passes and mass-matrix flush per step
    esz = 4
    mover = 0
    for i in mine:
        hc = insts[i]
        n, ncell = sizes[i], hc.nx * hc.ny
        mover += algorithmic_bytes("deposit", n, 0, ncell, esz)
        mover += 2 * (algorithmic_bytes("push", 0, n // 2, ncell, esz)
                      + algorithmic_bytes("permute", 0, n // 2, ncell, esz))
    peak, peak_kind = measured_peaks()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": dict(SCAN, instances=len(insts), instances_here=len(mine), particles_total=total,
                       gamma_bar="gamma(u^n + beta E^n(x)) (predicted)" if args.gamma_pred else "gamma(u^n)",
                       particles_here=N, workers=args.workers,
                       launch={"shared": f"shared launches: {args.scan_groups} groups of instances, each group's "
                                         "step one graph (one deposit, push and re-sort launch per species over "
                                         "the group's instances, their solves as branches) on its own stream",
                               "graphs": "one step graph per instance on its own stream",
                               "host": "host-driven steps by worker threads"}.get(path, path),
                       parallelism=f"instances sharded over {world} ranks" if world > 1 else "single"),
        "step_effective": {"mover_bytes_per_step": mover, "gbs": mover / (ms / 1e3) / 1e9,
                           "frac_of_peak": mover / (ms / 1e3) / 1e9 / peak, "peak": peak,
                           "peak_source": peak_kind,
                           "note": "particle passes + mass-matrix flush bytes over the whole step's span "
                                   "(GMRES and host waits included)"},
        "host_wall_ms_per_step": wall * 1e3 / max(1, args.steps),
        "gpu_launches": int(launches),
        "clocks": clk,
        "setup_s": t_setup,
        "instances": rows,
    }
    if args.scan_reference and rank == 0:
        out["single_instance_reference"] = scan_single_reference(rs, torch)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_quad(args):
    """The 1024x512 double Harris sheet (64 ppc per species, 67,108,864
    particles) with quadratic (TSC) shapes: the same timing as the headline
    line, its own JSON line."""
    import numpy as np
    import torch
    import paper_2509_11100_gb300 as rs
    from relsim_inputs import make_harris

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    hc = harris_config(seed=rank, small=args.workload == "c1qsmall")
    st = make_harris(hc)
    N = sum(len(sp["w"]) for sp in st["species"])
    cfg = rs.make_config(hc.nx, hc.ny, dt=hc.dt, theta_implicit=hc.theta, precision=32, shape=2,
                         gmres_tol=WORKLOAD["gmres_tol"], gmres_restart=WORKLOAD["gmres_restart"])
    sim = rs.Simulation(cfg)
    sim.load_state(st)
    tuning = sim.autotune() if not args.no_autotune else None
    for _ in range(args.warmup):
        sim.step(ledger=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    time.sleep(0.3)
    ev0.record(stream)
    leds = [sim.step(ledger=True)[0] for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    kp = max(1, min(args.steps, 5))
    sim.profile(True)
    sim.profile_read(reset=True)
    for _ in range(kp):
        sim.step(ledger=True)
    prof = sim.profile_read(reset=True)
    sim.close()
    per_kernel = {k: {"ms_per_step": v[0] / kp, "launches_per_step": v[2] / kp} for k, v in prof.items() if v[1] > 0}
    last = leds[-1]
    out = {"metric": METRIC, "value": N / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"2D relativistic double Harris sheet as the headline line ({hc.nx}x{hc.ny}, 64 "
                                  f"ppc per species, {N:,} particles) with quadratic (TSC) shape functions",
                      "form": "FP32 particles/fields/mass matrix, FP64 GMRES basis and ledger",
                      "gamma_bar": "gamma(u^n) (the quadratic shapes cover the base scheme)",
                      "l2": "inputs larger than L2, no flush"},
           "per_kernel": per_kernel, "gmres_iters_per_step": float(np.mean([l["gmres_iters"] for l in leds])),
           "ledger": {"residual_rel": abs(last["residual"]) / last["total"],
                      "mismatch_rel": abs(last["mismatch"]) / last["total"]},
           "autotune": tuning, "clocks": clk}
    print(json.dumps(out), flush=True)


def run_window(args):
    """The differentiable window on a 256x128 double Harris sheet (32 ppc per
    species, sigma 10, theta_T 0.3): 20 steps with a checkpoint every 5, the
    loss the k_x = 2 pi/L_x B_y mode energy after the window, its gradient
    with respect to the initial fields and particles by the chained step
    adjoints. Times the forward and the backward pass (host orchestration
    and state transfers included)."""
    import numpy as np
    import torch
    import paper_2509_11100_gb300 as rs
    from paper_2509_11100_gb300.window import ModeEnergyWindow
    from relsim_inputs import HarrisConfig, make_harris

    torch.cuda.set_device(rank_info()[2])
    hc = HarrisConfig(nx=256, ny=128, ppc=32, theta_T=0.3, delta=1.0, sigma=10.0, pert=0.01, dt=0.5)
    st = make_harris(hc)
    N = sum(len(s["w"]) for s in st["species"])
    steps = 20
    cfg = rs.make_config(hc.nx, hc.ny, dt=hc.dt, precision=32, gmres_tol=1e-7, gmres_restart=60,
                         gamma_pred=args.gamma_pred)
    win = ModeEnergyWindow(cfg, steps, checkpoint_every=5)
    win.forward(st)   # warm-up (allocations, graph captures)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L = win.forward(st)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    g = win.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    win.close()
    out = {"metric": "differentiable window: forward and backward time", "workload":
           "2D double Harris sheet 256x128, 32 ppc per species (2,097,152 particles), 20 RelSIM steps, "
           "checkpoint every 5, loss = B_y k_x=1 mode energy after the window, FP32 form",
           "gamma_bar": "gamma(u^n + beta E^n(x)) (predicted)" if args.gamma_pred else "gamma(u^n)",
           "particles": N, "steps": steps, "loss": L, "forward_s": t1 - t0, "backward_s": t2 - t1,
           "backward_over_forward": (t2 - t1) / (t1 - t0),
           "grad_norms": {"E": float(np.linalg.norm(g["E"])), "B": float(np.linalg.norm(g["B"])),
                          "u": float(sum(np.linalg.norm(p[0]) for p in g["particles"])),
                          "x": float(sum(np.linalg.norm(p[1]) for p in g["particles"]))},
           "n_gpus": 1, "data": "synthetic"}
    print(json.dumps(out), flush=True)


def run_3d(args):
    """The 3D double Harris sheet (256 x 128 x 128 cells, 16 particles per
    cell per species, 134,217,728 particles; trilinear shapes, 27-node
    stencil), FP32 form timed over the steps, the FP64 form over a few, the
    per-kernel times from an event-profiled pass. Its own JSON line."""
    import numpy as np
    import torch
    import paper_2509_11100_gb300 as rs
    from relsim_inputs import HarrisConfig3, make_harris3

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    small = args.workload == "c2small"
    hc = HarrisConfig3(nx=64 if small else 256, ny=32 if small else 128, nz=32 if small else 128, ppc=16,
                       dt=0.5, seed=rank)
    t0 = time.time()
    st = make_harris3(hc)
    t_gen = time.time() - t0
    N = sum(len(sp["w"]) for sp in st["species"])
    nn = hc.nx * hc.ny * hc.nz

    def sim_for(prec):
        cfg = rs.make_config(hc.nx, hc.ny, nz=hc.nz, dt=hc.dt, theta_implicit=hc.theta, precision=prec,
                             gmres_tol=1e-6 if prec == 32 else 1e-10, gmres_restart=30)
        sim = rs.Simulation(cfg)
        sim.load_state(st)
        return sim

    sim = sim_for(32)
    tuning = sim.autotune() if not args.no_autotune else None
    for _ in range(args.warmup):
        sim.step(ledger=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    time.sleep(0.3)
    launches0 = rs.relsim_kernel_launches()
    ev0.record(stream)
    leds = []
    for _ in range(args.steps):
        led, status = sim.step(ledger=True)
        leds.append(led)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = rs.relsim_kernel_launches() - launches0
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    kp = max(1, min(args.steps, 5))
    sim.profile(True)
    sim.profile_read(reset=True)
    for _ in range(kp):
        sim.step(ledger=True)
    prof = sim.profile_read(reset=True)
    sim.profile(False)
    per_kernel = {k: {"ms_per_step": v[0] / kp, "launches_per_step": v[2] / kp} for k, v in prof.items() if v[1] > 0}
    peak, peak_kind = measured_peaks()
    # algorithmic bytes (FP32 form): the deposit reads the 28-byte particle
    # record and writes M (126 values) and Jhat (3) per node; the push and
    # re-sort read and write the record, the keys and the permutation
    # (28 + 28 + 4 + 4 (+ 8 for the radix passes' pairs) bytes per particle)
    algo = {"deposit": N * 28 + nn * (126 + 3) * 4, "general_sort": N * (28 + 28 + 4 + 4 + 8)}
    for k, ab in algo.items():
        if k in per_kernel:
            gbs = ab / (per_kernel[k]["ms_per_step"] / 1e3) / 1e9
            per_kernel[k].update({"algorithmic_bytes_per_step": ab, "achieved_gbs": gbs, "frac": gbs / peak})
    sim.close()
    fp64 = None
    if not args.no_fp64:
        s64 = sim_for(64)
        s64.step(ledger=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k64 = 2
        e0.record(stream)
        for _ in range(k64):
            l64, _ = s64.step(ledger=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / k64
        fp64 = {"value": N / (ms64 / 1e3), "unit": "particle-pushes/s", "ms_per_step": ms64, "steps": k64,
                "ledger_residual_rel": abs(l64["residual"]) / l64["total"], "speedup_fp32_over_fp64": ms64 / ms}
        s64.close()
    cpu = None
    if not args.no_cpu_baseline:
        # the 3D oracle as it stands on one core, on the same sheet at 64x32x32
        # (16 ppc per species, 2,097,152 particles): one full step
        from oracle.three import Particles3, make_config3, step3
        sc = HarrisConfig3(nx=64, ny=32, nz=32, ppc=16, dt=0.5, seed=rank)
        ss = make_harris3(sc)
        c3 = make_config3(sc.nx, sc.ny, sc.nz, dt=sc.dt, theta=sc.theta, gmres_tol=1e-12, gmres_restart=50)
        P3 = Particles3(ss["species"])
        t0 = time.perf_counter()
        step3(c3, P3, ss["E"], ss["B"])
        dtc = time.perf_counter() - t0
        n3 = int(P3.off[-1])
        cpu = {"value": n3 / dtc, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the same 3D sheet on 64x32x32 cells ({n3} particles), one full oracle step "
                         "(deposit, GMRES tol 1e-12, push), single thread, FP64", "seconds": dtc}
    last = leds[-1]
    out = {"metric": METRIC, "value": N / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"3D relativistic double Harris sheet, pair plasma, {hc.nx}x{hc.ny}x{hc.nz} cells "
                                  f"(dx=dy=dz=1 d_e), 16 ppc per species ({N:,} particles), sigma=10, theta_T=0.3, "
                                  "delta=1 d_e, dt=0.5/omega_pe, theta=0.5, 1% B_y perturbation in x-z modes 1-4, "
                                  "trilinear shapes (27-node stencil), seed 0",
                      "form": "FP32 particles/fields/mass matrix, FP64 GMRES basis and ledger",
                      "gamma_bar": "gamma(u^n) (the 3D form covers the base scheme)",
                      "l2": "inputs larger than L2 (3.8 GB of particle data per step), no flush"},
           "per_kernel": per_kernel, "per_kernel_pass": f"{kp} further steps with event profiling",
           "gpu_launches": launches, "gmres_iters_per_step": float(np.mean([l["gmres_iters"] for l in leds])),
           "ledger": {"residual_rel": abs(last["residual"]) / last["total"],
                      "mismatch_rel": abs(last["mismatch"]) / last["total"]},
           "fp64_form": fp64, "cpu_baseline": cpu, "autotune": tuning, "clocks": clk, "input_generation_s": t_gen}
    print(json.dumps(out), flush=True)


def scan_single_reference(rs, torch, sizes=((1024, 512), (768, 384), (128, 64)), steps=20):
    """Single instances with the scan's parameters (32 ppc per species,
    dt = 0.5, delta 1, sigma 10, 0.1% perturbation), graph steps, for scale."""
    from relsim_inputs import HarrisConfig, make_harris
    res = []
    for nx, ny in sizes:
        hc = HarrisConfig(nx=nx, ny=ny, ppc=32, dt=0.5, delta=1.0, sigma=10.0, pert=1e-3, theta_T=0.3)
        st = make_harris(hc)
        n = sum(len(s["w"]) for s in st["species"])
        sim = rs.Simulation(rs.make_config(nx, ny, dt=hc.dt, theta_implicit=hc.theta, precision=32,
                                           gmres_tol=SCAN["gmres_tol"], gmres_restart=SCAN["gmres_restart"]))
        sim.load_state(st)
        for _ in range(3):
            sim.step(ledger=False)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            sim.step(ledger=True)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        res.append({"nx": nx, "ny": ny, "particles": n, "ms_per_step": ms, "value": n / (ms / 1e3),
                    "unit": UNIT, "steps": steps})
        sim.close()
    return res


def run_long(args):
    """The headline sheet (1024x512, 67.1M particles, FP32 form) run for
    --long-steps steps (2000 by default) as one job: the throughput over the
    whole run, the total energy's drift against the first step's (the
    ledger's total every step), the m = 1 B_y mode energy every 10 steps
    with its best growth rate over 40 samples (the tearing diagnostic), and
    the spectrum of gamma - 1 (256 log bins over [1e-2, 1e4]) at the start
    and at the end."""
    import numpy as np
    import torch
    import paper_2509_11100_gb300 as rs
    from relsim_inputs import make_harris

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    hc = harris_config(seed=rank)
    state = make_harris(hc)
    N = sum(len(sp["w"]) for sp in state["species"])
    cfg = rs.make_config(hc.nx, hc.ny, dt=hc.dt, theta_implicit=hc.theta, precision=32,
                         gmres_tol=WORKLOAD["gmres_tol"], gmres_restart=WORKLOAD["gmres_restart"],
                         gamma_pred=args.gamma_pred)
    sim = rs.Simulation(cfg)
    sim.load_state(state)
    del state
    tuning = sim.autotune() if not args.no_autotune else None
    edges = np.geomspace(1e-2, 1e4, 257)

    def spectrum():
        cnt = sum(sim.spectrum(s, edges, 0)[1] for s in range(2))
        inner = np.asarray(cnt[1:-1], dtype=np.float64)
        mid = np.sqrt(edges[:-1] * edges[1:])
        return {"peak_bin_gamma_minus_1": float(mid[int(np.argmax(inner))]),
                "above_10": float(inner[mid > 10].sum() / max(inner.sum(), 1)),
                "above_100": float(inner[mid > 100].sum() / max(inner.sum(), 1)),
                "max_bin_gamma_minus_1": float(mid[np.nonzero(inner)[0].max()]) if inner.any() else None}

    spec0 = spectrum()
    nsteps = args.long_steps
    totals, modes, iters, fails = [], [], [], 0
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for n in range(nsteps):
        led, code = sim.step(ledger=True)
        fails += code != 0
        totals.append(led["total"])
        iters.append(led["gmres_iters"])
        if n % 10 == 0:
            modes.append(float(sim.field_modes(1, 2)[1]))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    # the same steps without the ledger read and the mode diagnostic: the
    # solver's cost alone at the end of the run
    nq = min(100, nsteps)
    torch.cuda.synchronize()
    tq = time.perf_counter()
    for _ in range(nq):
        sim.step(ledger=False)
    torch.cuda.synchronize()
    wall_q = (time.perf_counter() - tq) / max(1, nq)
    rate, first = rs.relsim_growth_fit(np.asarray(modes), 10 * hc.dt, 40)
    tot = np.asarray(totals)
    out = {"metric": METRIC, "value": N * nsteps / wall, "unit": UNIT, "n_gpus": 1, "steps": nsteps,
           "warmup": 0, "ms_per_step": 1e3 * wall / nsteps, "higher_is_better": True, "dtype": "f32",
           "data": "synthetic",
           "config": dict(WORKLOAD, run="one long run, host wall clock over all steps including the per-step "
                                        "ledger read back and the mode diagnostic every 10 steps",
                          gamma_bar="gamma(u^n + beta E^n(x)) (predicted)" if args.gamma_pred
                          else "gamma(u^n)"),
           "energy": {"max_rel_drift": float(np.abs(tot - tot[0]).max() / abs(tot[0])),
                      "final_rel_drift": float((tot[-1] - tot[0]) / abs(tot[0])),
                      "drift_at": {str(k): float((tot[k - 1] - tot[0]) / abs(tot[0]))
                                   for k in (200, 500, 1000, 2000) if k <= len(tot)}},
           "gmres_iters_per_step": float(np.mean(iters)), "steps_not_converged": int(fails),
           "ms_per_step_no_ledger_at_end": {"ms_per_step": 1e3 * wall_q, "steps": nq,
                                            "note": "steps after the run, without the per-step ledger read "
                                                    "and the mode diagnostic"},
           "tearing_m1": {"energy_first": modes[0], "energy_last": modes[-1], "growth_rate": rate,
                          "fit_first_step": 10 * first + 1,
                          "sampled_after_steps": "1, 11, 21, ... (every 10 steps)", "samples": len(modes)},
           "spectrum_start": spec0, "spectrum_end": spectrum(), "autotune": tuning, "clocks": clk}
    sim.close()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes (no autotuner pass after the load)")
    ap.add_argument("--long-steps", type=int, default=2000, help="long: the number of steps of the run")
    ap.add_argument("--gamma-bar", choices=["pred", "un"], default="pred",
                    help="the Lorentz factor in alpha, Jhat, M and the push: pred (default) the predicted "
                         "gamma(u^n + beta E^n(x)), whose runs keep the energy balance over long runs; un: "
                         "gamma(u^n) (headline, scan and long workloads, and the reference arm)")
    ap.add_argument("--workload", choices=["c1", "small", "scan", "window", "c2", "c2small", "c1q", "c1qsmall",
                                           "long"], default="c1",
                    help="small: 512x256 cells for profiler captures; scan: the 48-instance batched "
                         "tearing scan (run with --steps 400 for its full length); window: the "
                         "differentiable 20-step window on 256x128; c2: the 3D sheet on 256x128x128 "
                         "(c2small: 64x32x32); c1q: the headline sheet with quadratic shapes; long: the "
                         "headline sheet for --long-steps steps (energy drift, tearing mode, spectrum)")
    ap.add_argument("--workers", type=int, default=8, help="host worker threads of the scan's batch runner")
    ap.add_argument("--scan-launch", choices=["shared", "instances"], default="instances",
                    help="scan: one step graph per instance on its own stream (default, the faster as measured) "
                         "or shared launches over groups of instances")
    ap.add_argument("--scan-groups", type=int, default=4,
                    help="scan: instance groups of the shared launches (each group on its own stream)")
    ap.add_argument("--scan-reference", action="store_true",
                    help="scan: also time single 1024x512, 768x384 and 128x64 instances with its parameters")
    args = ap.parse_args()
    args.gamma_pred = 1 if args.gamma_bar == "pred" else 0
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "scan":
        run_scan(args)
    elif args.workload == "window":
        run_window(args)
    elif args.workload in ("c2", "c2small"):
        run_3d(args)
    elif args.workload in ("c1q", "c1qsmall"):
        run_quad(args)
    elif args.workload == "long":
        run_long(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
