#!/usr/bin/env python
"""Benchmark of the SPH hot path on one GB300: density (with the smoothing-length
iteration) + hydro forces, grouped neighbour search (Neighbour Recycling) against the
per-particle search, in active particles per second.

One step = the whole hot path on one particle set: Peano-Hilbert keys and radix sort,
octree build, density with the h iteration, hydro forces -- every stage a kernel of
libsphgrp.so, called through its C ABI.

Workload (default): 2^24 particles, half uniform and half in 256 Plummer spheres (seeded
synthetic stand-in for a cosmological box), velocities N(0, 0.1^2), u log-normal,
N_ngb = 64 +- 2, all particles active.  The step's initial smoothing lengths are the
converged ones of a set-up pass scattered by a seeded log-normal factor (5%), the
change of h over one timestep, so that every step re-converges h (a few passes).

Output: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle instead
(the only reference implementation of this method), on a bounded sample.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SPH density+hydro active particles/s: grouped vs per-particle search, 1 GB300"
UNIT = "active particles/s"

# algorithmic bytes per unit (candidate, member, node) of the two search kernels
B_CAND = {"density": 32, "hydro": 64}
B_MEMBER = {"density": 32 + 16, "hydro": 64 + 16}
B_NODE = 48
# the backward's three pair loops and the velocity-derivative loop: (bytes per staged
# candidate, bytes per member)
B_BWD = {"density_sums": (32, 48), "hydro_adjoint": (80, 136), "density_adjoint": (48, 72)}
B_VEL = (48, 92)


def launch_gbs(e: dict, b_cand: int, b_member: int) -> float:
    """Algorithmic GB/s of one logged search launch (candidates, members, nodes tested)."""
    return (e["candidates"] * b_cand + e["members"] * b_member + e["nodes"] * B_NODE) / (e["ms"] / 1e3) / 1e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--active", type=float, default=1.0)
    ap.add_argument("--group", type=int, default=16)
    ap.add_argument("--h-scatter", type=float, default=0.05)
    ap.add_argument("--iteration", choices=["passes", "recycle", "in-group"], default="passes",
                    help="smoothing-length iteration of the grouped density")
    ap.add_argument("--cpu-n", type=int, default=1 << 19, help="oracle sample size")
    ap.add_argument("--no-individual", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--backward-n", type=int, default=1 << 21, help="particles of the backward workload")
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--batch-boxes", type=int, default=96, help="boxes of the batched workload")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-small", action="store_true", help="skip the uniform 32768 and the group-size sweep legs")
    ap.add_argument("--no-halo", action="store_true", help="skip the domain-decomposition halo leg")
    ap.add_argument("--profile-pass", action="store_true",
                    help="after set-up run one grouped and one per-particle density+hydro pass inside "
                         "the NVTX range 'pass' (for ncu --nvtx-include pass/) and exit")
    return ap.parse_args()


def workload_name(a) -> str:
    return (f"clustered N={a.n} (half uniform, half in 256 Plummer spheres), density+hydro, "
            f"{a.active:.0%} active, Nngb=64+-2")


# ----------------------------------------------------------------------------- CPU oracle

class CpuSample:
    """The FP64 oracle on a smaller set of the same recipe (all active).  Set-up
    (untimed): cold smoothing-length iteration.  One timed run: keys, order, density
    with the h iteration from the scattered h, hydro."""

    def __init__(self, n: int, h_scatter: float, seed_salt: int = 0):
        import oracle
        import sphgen

        self.oracle = oracle
        self.n = n
        self.h_scatter = h_scatter
        d = sphgen.make("clustered", n, config=3, seed_salt=seed_salt)
        self.pos = d["pos"]
        self.m = d["m"].astype(np.float32).astype(np.float64)
        self.vel = d["vel"].astype(np.float32).astype(np.float64)
        self.u = d["u"].astype(np.float32).astype(np.float64)
        hc, _ = oracle.density_iterate(self.pos, self.m, np.full(n, d["h0"]))
        rng = np.random.default_rng(77 + seed_salt)
        self.h0 = hc * np.exp(h_scatter * rng.standard_normal(n))

    def run(self) -> float:
        o = self.oracle
        t0 = time.perf_counter()
        keys = o.hilbert_keys(self.pos)
        o.stable_order(keys)
        h, dens = o.density_iterate(self.pos, self.m, self.h0)
        o.hydro(self.pos, self.vel, self.m, h, dens["rho"], dens["f"], self.u)
        return time.perf_counter() - t0

    def per_pass(self, g: int) -> dict:
        """One density pass and one hydro pass at converged h, per-particle and grouped
        (the oracle's Sec. 2.1 form: g consecutive particles along the curve per walk,
        centred on the group's first particle), with the speedups of grouping."""
        o = self.oracle
        h, dens = o.density_iterate(self.pos, self.m, self.h0)
        args = (self.pos, self.vel, self.m, h, dens["rho"], dens["f"], self.u)
        t = {}
        for form, dfn, hfn in (("per_particle", lambda: o.density(self.pos, self.m, h), lambda: o.hydro(*args)),
                               ("grouped", lambda: o.density_grouped(self.pos, self.m, h, g),
                                lambda: o.hydro_grouped(*args, g))):
            t0 = time.perf_counter()
            dfn()
            t1 = time.perf_counter()
            hfn()
            t[form] = {"density_s": t1 - t0, "hydro_s": time.perf_counter() - t1}
        i, gr = t["per_particle"], t["grouped"]
        return {"g": g, **t, "speedup": {"density": i["density_s"] / gr["density_s"],
                                          "hydro": i["hydro_s"] / gr["hydro_s"],
                                          "total": (i["density_s"] + i["hydro_s"]) /
                                                   (gr["density_s"] + gr["hydro_s"])}}

    def describe(self, seconds: float, value: float) -> dict:
        return {"value": value, "unit": UNIT, "cores": self.oracle.threads(), "kind": "oracle",
                "sample": f"clustered N={self.n} of the same recipe, all active: keys, order, density "
                          f"with h iteration from {self.h_scatter:.0%}-scattered h, hydro "
                          f"({seconds:.1f} s per run)"}


def cpu_sample(n: int, h_scatter: float) -> dict:
    S = CpuSample(n, h_scatter)
    t = S.run()
    out = S.describe(t, n / t)
    out["grouped_form"] = guarded(S.per_pass, 8)
    return out


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    S = CpuSample(a.cpu_n, a.h_scatter)
    for _ in range(max(0, min(a.warmup, 1))):
        S.run()
    ts = [S.run() for _ in range(a.steps)]
    t = float(np.mean(ts))
    v = a.cpu_n / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "oracle_sample_n": a.cpu_n},
            "cpu_baseline": S.describe(t, v),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict | None:
        if not self.path or not os.path.exists(self.path):
            return None
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
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm

class Problem:
    def __init__(self, a, rank: int):
        import torch

        import paper_1810_09898_gb300 as sg
        import sphgen

        self.torch, self.sg, self.a = torch, sg, a
        dev = torch.device("cuda", torch.cuda.current_device())
        self.dev = dev
        n = a.n
        d = sphgen.make("clustered", n, config=3, seed_salt=rank)
        self.n = n
        self.host = {
            "pos": torch.from_numpy(d["pos"]).pin_memory(),
            "m": torch.from_numpy(d["m"].astype(np.float32)).pin_memory(),
            "vel": torch.from_numpy(d["vel"].astype(np.float32)).pin_memory(),
            "u": torch.from_numpy(d["u"].astype(np.float32)).pin_memory(),
        }
        self.pos = self.host["pos"].to(dev)
        self.m = self.host["m"].to(dev)
        self.vel = self.host["vel"].to(dev)
        self.u = self.host["u"].to(dev)
        self.ctx = sg.Context(n, iteration={"in-group": sg.ITER_IN_GROUP, "passes": sg.ITER_PASSES,
                                            "recycle": sg.ITER_RECYCLE}[a.iteration])
        self.perm = torch.empty(n, dtype=torch.int32, device=dev)
        f32 = dict(dtype=torch.float32, device=dev)
        self.rho = torch.zeros(n, **f32)
        self.drho = torch.zeros(n, **f32)
        self.f = torch.zeros(n, **f32)
        self.nn = torch.zeros(n, dtype=torch.int32, device=dev)
        self.nnh = torch.zeros(n, dtype=torch.int32, device=dev)
        self.acc = torch.zeros((n, 3), **f32)
        self.dudt = torch.zeros(n, **f32)
        self.h = torch.empty(n, dtype=torch.float64, device=dev)
        # set-up: order, tree, converged h from the uniform-density guess (cold start)
        self.ctx.sfc_keys_sort(self.pos, None, self.perm)
        self.ctx.tree_build(self.pos, self.m)
        all_act = torch.arange(n, dtype=torch.int32, device=dev)
        self.h.fill_(d["h0"])
        t0 = time.perf_counter()
        self.ctx.density(all_act, self.h, 1, sg.GROUPED, 16, self.rho, self.drho, self.f, self.nn)
        torch.cuda.synchronize()
        self.cold_s = time.perf_counter() - t0
        self.cold_stats = self.ctx.stats()
        # active set: runs along the key order (all particles at 100%)
        if a.active >= 1.0:
            act = np.arange(n, dtype=np.int32)
        else:
            mask = sphgen.active_rank_mask(n, a.active, 32.0, np.random.default_rng(1000 + rank))
            act = np.sort(self.perm.cpu().numpy()[np.flatnonzero(mask)]).astype(np.int32)
        self.n_act = len(act)
        self.act = torch.from_numpy(act).to(dev)
        self.host["act"] = torch.from_numpy(act).pin_memory()
        rng = np.random.default_rng(77 + rank)
        hc = self.h.cpu().numpy()
        hi = hc.copy()
        hi[act] = hc[act] * np.exp(a.h_scatter * rng.standard_normal(len(act)))
        self.h_init = torch.from_numpy(hi).to(dev)
        self.host["h_init"] = torch.from_numpy(hi).pin_memory()
        self.side = torch.cuda.Stream(device=dev)
        self.out_host = {
            "acc": torch.empty((n, 3), dtype=torch.float32).pin_memory(),
            "dudt": torch.empty(n, dtype=torch.float32).pin_memory(),
            "rho": torch.empty(n, dtype=torch.float32).pin_memory(),
            "h": torch.empty(n, dtype=torch.float64).pin_memory(),
        }

    def step(self, mode: int, g: int, collect: list | None = None):
        c = self.ctx
        c.sfc_keys_sort(self.pos, None, self.perm)
        c.tree_build(self.pos, self.m)
        self.h.copy_(self.h_init)
        c.density(self.act, self.h, 1, mode, g, self.rho, self.drho, self.f, self.nn)
        sd = c.stats() if collect is not None else None
        passes = None
        if collect is not None:
            try:   # host-side record of the call's search launches (no device work)
                passes = [{"members": e["members"], "ms": e["ms"]} for e in c.launch_log()]
            except Exception:  # noqa: BLE001 - the per-pass record is optional
                passes = None
        c.hydro_force(self.act, self.h, self.rho, self.f, self.vel, self.u, mode, g, self.acc, self.dudt,
                      self.nnh)
        if collect is not None:
            collect.append({"density": sd, "hydro": c.stats(), "density_passes": passes})

    def step_e2e(self, g: int):
        """The same step from host buffers: inputs copied in, results copied out.  Only
        the positions go up before the keys; the other inputs follow on a second stream in
        the order they are needed (m for the tree, the active list and h for the density,
        v and u for the hydro loop) while keys, sort, tree and density run, and rho and h
        come back on it while hydro runs; the step ends when both streams are done."""
        torch, c = self.torch, self.ctx
        H, O = self.host, self.out_host
        main = torch.cuda.current_stream()
        side = self.side
        self.pos.copy_(H["pos"], non_blocking=True)
        side.wait_stream(main)   # the other inputs start after the positions
        with torch.cuda.stream(side):
            self.m.copy_(H["m"], non_blocking=True)
            tree_in = side.record_event()
            self.act.copy_(H["act"], non_blocking=True)
            self.h.copy_(H["h_init"], non_blocking=True)
            density_in = side.record_event()
            self.vel.copy_(H["vel"], non_blocking=True)
            self.u.copy_(H["u"], non_blocking=True)
            hydro_in = side.record_event()
        c.sfc_keys_sort(self.pos, None, self.perm)
        main.wait_event(tree_in)
        c.tree_build(self.pos, self.m)
        main.wait_event(density_in)
        c.density(self.act, self.h, 1, self.sg.GROUPED, g, self.rho, self.drho, self.f, self.nn)
        side.wait_event(main.record_event())
        with torch.cuda.stream(side):
            O["rho"].copy_(self.rho, non_blocking=True)
            O["h"].copy_(self.h, non_blocking=True)
        main.wait_event(hydro_in)
        c.hydro_force(self.act, self.h, self.rho, self.f, self.vel, self.u, self.sg.GROUPED, g, self.acc,
                      self.dudt, self.nnh)
        O["acc"].copy_(self.acc, non_blocking=True)
        O["dudt"].copy_(self.dudt, non_blocking=True)
        main.synchronize()
        side.synchronize()

    def io_bytes(self):
        n = self.n
        h2d = n * (24 + 4 + 12 + 4 + 8) + 4 * self.n_act
        d2h = n * (12 + 4 + 4 + 8)
        return h2d, d2h


def max_over_ranks(value: float, dist, device) -> float:
    """The largest value over all ranks (every rank gets it); the value itself at N = 1."""
    if not dist:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(world: int, units_per_rank: int, ms_per_step: float) -> float:
    """Whole-job throughput of N replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / (ms_per_step / 1e3)


def timed(P, fn, steps, warmup, dist):
    torch = P.torch
    for _ in range(warmup):
        fn(None)
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    collect = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = P.sg.kernel_launches()
    ev0.record(stream)
    for _ in range(steps):
        fn(collect)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = P.sg.kernel_launches() - l0
    if dist:
        dist.barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, P.dev)
    return ms, collect, launches


def roofline(collect, peak_gbs, clocks=None, form: str = "grouped"):
    """Dominant search kernel: algorithmic bytes per launch / event time per launch.
    form selects the DRAM record of the captured kernels ("grouped" or "individual")."""
    agg = {}
    for rec in collect:
        for k in ("density", "hydro"):
            s = rec[k]
            A = agg.setdefault(k, {"ms": 0.0, "launches": 0, "bytes": 0.0, "cand": 0, "tests": 0, "pairs": 0,
                                   "members": 0, "walks": 0, "nodes": 0})
            A["ms"] += s["search_ms"]
            A["launches"] += s["search_launches"]
            A["bytes"] += s["candidates"] * B_CAND[k] + s["members"] * B_MEMBER[k] + s["nodes_tested"] * B_NODE
            A["cand"] += s["candidates"]
            A["tests"] += s["pair_tests"]
            A["pairs"] += s["pairs"]
            A["members"] += s["members"]
            A["walks"] += s["walks"]
            A["nodes"] += s["nodes_tested"]
    dom = max(agg, key=lambda k: agg[k]["ms"])
    A = agg[dom]
    per_launch_bytes = A["bytes"] / max(1, A["launches"])
    per_launch_s = A["ms"] / max(1, A["launches"]) / 1e3
    achieved = per_launch_bytes / per_launch_s / 1e9
    detail = {k: {"ms_per_step": v["ms"] / max(1, len(collect)), "launches_per_step": v["launches"] / max(1, len(collect)),
                  "candidates_per_member": v["cand"] / max(1, v["members"]),
                  "pair_tests_per_member": v["tests"] / max(1, v["members"]),
                  "pairs_per_member": v["pairs"] / max(1, v["members"]),
                  "members_per_walk": v["members"] / max(1, v["walks"]),
                  "nodes_per_walk": v["nodes"] / max(1, v["walks"])} for k, v in agg.items()}
    traffic = measured_traffic(("indiv_" if form == "individual" else "") + dom, A["members"] / max(1, A["launches"]))
    # the FP32 side of the same launches: ~10 flop per member x candidate test (the
    # difference, r^2, the threshold) and ~25 per true pair (kernel and sums), against
    # 152 SMs x 128 lanes x 2 flop x the sampled SM clock
    flops = (10.0 * A["tests"] + 25.0 * A["pairs"]) / max(1, A["launches"])
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    alu = {"achieved_tflops": flops / per_launch_s / 1e12, "peak_tflops": alu_peak,
           "frac": flops / per_launch_s / 1e12 / alu_peak,
           "peak_source": "152 SMs x 128 FP32 lanes x 2 x sampled SM clock (derived)"}
    # the smoothing-length iteration's density launches of the last step: active members
    # and device time of every pass
    last = collect[-1].get("density_passes") if collect else None
    if last and "density" in detail:
        detail["density"]["passes_of_last_step"] = last
    kernel = f"k_indiv ({dom})" if form == "individual" else f"k_group ({dom})"
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak_gbs,
            "unit": "GB/s", "frac": achieved / peak_gbs, "traffic": traffic,
            "bytes_per_launch": per_launch_bytes, "launch_ms": per_launch_s * 1e3, "alu": alu,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}, detail


def measured_traffic(kind: str, members_per_launch: float):
    """DRAM bytes per launch from the last ncu capture of the search kernel (recorded per
    member in profiles/traffic.json), scaled to the units one launch processes; None when
    the kernel source changed since the capture."""
    import hashlib

    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        src = open(os.path.join(ROOT, rec["kernel_source"]), "rb").read()
    except (OSError, KeyError, ValueError):
        return None
    if hashlib.sha256(src).hexdigest()[:16] != rec.get("kernel_source_sha256_16"):
        return None
    per = rec.get(f"{kind}_dram_bytes_per_member")
    return None if per is None else per * members_per_launch


def guarded(fn, *args):
    """Runs an optional leg of the bench; a failure is reported in its place instead of
    losing the main line."""
    try:
        return fn(*args)
    except Exception as e:  # noqa: BLE001 - any failure of an optional leg is reported
        import traceback

        return {"error": f"{type(e).__name__}: {e}", "where": traceback.format_exc().splitlines()[-7:-1]}


def per_pass(P, mode: int, g: int, reps: int = 5) -> dict:
    """Per-pass metric at converged h: one density pass (no iteration) and one hydro pass
    over the active particles, N_act / (t_density + t_hydro), CUDA events per pass."""
    torch = P.torch
    c = P.ctx
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    td, th = [], []
    for rep in range(reps + 1):
        ev[0].record(stream)
        c.density(P.act, P.h, 0, mode, g, P.rho, P.drho, P.f, P.nn)
        ev[1].record(stream)
        c.hydro_force(P.act, P.h, P.rho, P.f, P.vel, P.u, mode, g, P.acc, P.dudt, P.nnh)
        ev[2].record(stream)
        torch.cuda.synchronize()
        if rep:
            td.append(ev[0].elapsed_time(ev[1]))
            th.append(ev[1].elapsed_time(ev[2]))
    d, h = float(np.median(td)), float(np.median(th))
    return {"density_ms": d, "hydro_ms": h, "value": P.n_act / ((d + h) / 1e3), "unit": UNIT}


def _median_ms(torch, fn, reps: int) -> float:
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    t = []
    for rep in range(reps + 1):
        ev[0].record(stream)
        fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        if rep:
            t.append(ev[0].elapsed_time(ev[1]))
    return float(np.median(t))


def velocity_pass(P, g: int, reps: int = 5) -> dict:
    """At converged h over the active particles, CUDA events per call: one grouped
    velocity divergence + curl pass (its own walk over the density sets); the density pass
    alone and the density pass with div/curl summed in the same loop (fused); one hydro
    pass with the Balsara-limited viscosity fed those div/curl."""
    torch = P.torch
    n = P.n
    c = P.ctx
    divv = torch.zeros(n, dtype=torch.float32, device=P.dev)
    curl = torch.zeros((n, 3), dtype=torch.float32, device=P.dev)
    ms = _median_ms(torch, lambda: c.velocity_derivs(P.act, P.h, P.rho, P.vel, g, divv, curl), reps)
    gbs = launch_gbs(c.launch_log()[0], *B_VEL)
    h = P.h.clone()
    rho, drho, f = (torch.zeros(n, dtype=torch.float32, device=P.dev) for _ in range(3))
    nn = torch.zeros(n, dtype=torch.int32, device=P.dev)
    ms_d = _median_ms(torch, lambda: c.density(P.act, h, 0, P.sg.GROUPED, g, rho, drho, f, nn), reps)
    ms_f = _median_ms(torch, lambda: c.density_derivs(P.act, h, 0, g, P.vel, rho, drho, f, nn, divv, curl), reps)
    acc = torch.zeros((n, 3), dtype=torch.float32, device=P.dev)
    dudt = torch.zeros(n, dtype=torch.float32, device=P.dev)
    ms_h = _median_ms(torch, lambda: c.hydro_force(P.act, P.h, P.rho, P.f, P.vel, P.u, P.sg.GROUPED, g, acc, dudt),
                      reps)
    ms_b = _median_ms(torch, lambda: c.hydro_force(P.act, P.h, P.rho, P.f, P.vel, P.u, P.sg.GROUPED, g, acc, dudt,
                                                   divv=divv, curlv=curl), reps)
    peak = measured_peak_hbm()
    return {"ms": ms, "value": P.n_act / (ms / 1e3), "unit": UNIT, "group_size": g,
            "roofline": {"achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak},
            "fused_in_density": {"density_ms": ms_d, "density_with_derivs_ms": ms_f,
                                 "extra_ms": ms_f - ms_d, "separate_walk_ms": ms},
            "hydro_balsara": {"plain_ms": ms_h, "limited_ms": ms_b}}


def active_leg(P, frac: float, g: int, steps: int, warmup: int, dist, rank: int) -> dict:
    """The same step with a fraction of the particles active in key-order runs (mean
    length 32); inactive particles keep their converged h, rho and f."""
    import sphgen

    torch, sg = P.torch, P.sg
    keep = (P.act, P.h_init, P.n_act)
    mask = sphgen.active_rank_mask(P.n, frac, 32.0, np.random.default_rng(2000 + rank))
    act = np.sort(P.perm.cpu().numpy()[np.flatnonzero(mask)]).astype(np.int32)
    P.act = torch.from_numpy(act).to(P.dev)
    P.n_act = len(act)
    h = P.h.clone()
    rng = np.random.default_rng(3000 + rank)
    scat = torch.from_numpy(np.exp(P.a.h_scatter * rng.standard_normal(len(act)))).to(P.dev)
    h[P.act.long()] *= scat
    P.h_init = h
    out = {"fraction": frac, "n_active": P.n_act}
    try:
        # the group size is the method's tuning knob (Sec. 3.2 finds its optimum numerically):
        # one timed step at each candidate size (after two untimed ones) picks the size this
        # active set runs fastest at
        trial = {}
        for gs in sorted({8, 16, 32, g}):
            for _ in range(2):
                P.step(sg.GROUPED, gs)
            trial[gs], _, _ = timed(P, lambda cl, gs=gs: P.step(sg.GROUPED, gs, cl), 1, 0, dist)
        g_best = min(trial, key=trial.get)
        out["group_size"] = g_best
        out["group_size_trial_ms"] = {str(k): v for k, v in trial.items()}
        for name, mode, gs in (("grouped", sg.GROUPED, g_best), ("individual", sg.INDIVIDUAL, 1)):
            ms, _, _ = timed(P, lambda cl: P.step(mode, gs, cl), steps, warmup, dist)
            out[name] = {"ms_per_step": ms / steps, "value": P.n_act / (ms / steps / 1e3)}
        out["speedup_grouped"] = out["individual"]["ms_per_step"] / out["grouped"]["ms_per_step"]
    finally:
        P.act, P.h_init, P.n_act = keep
    return out


def backward_leg(a, rank: int, steps: int, warmup: int):
    """Forward + backward step on the clustered 2^21-particle workload: keys, sort,
    tree, density at converged h, hydro forces, then the adjoint of
    L = sum w.a + sum s rho (three grouped pair loops and the per-particle chain)."""
    import torch

    import paper_1810_09898_gb300 as sg
    import sphgen

    dev = torch.device("cuda", torch.cuda.current_device())
    n = a.backward_n
    d = sphgen.make("clustered", n, config=4, seed_salt=rank)
    f32 = dict(dtype=torch.float32, device=dev)
    pos = torch.from_numpy(d["pos"]).to(dev)
    m = torch.from_numpy(d["m"].astype(np.float32)).to(dev)
    vel = torch.from_numpy(d["vel"].astype(np.float32)).to(dev)
    u = torch.from_numpy(d["u"].astype(np.float32)).to(dev)
    rng = np.random.default_rng(sphgen.SEED_BASE + 4 + rank)
    w = torch.from_numpy(rng.standard_normal((n, 3)).astype(np.float32)).to(dev)
    s = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(dev)
    ctx = sg.Context(n, nngb_tol=1e-3)
    act = torch.arange(n, dtype=torch.int32, device=dev)
    h = torch.full((n,), d["h0"], dtype=torch.float64, device=dev)
    rho, drho, fg = (torch.zeros(n, **f32) for _ in range(3))
    nn = torch.zeros(n, dtype=torch.int32, device=dev)
    acc, dudt = torch.zeros((n, 3), **f32), torch.zeros(n, **f32)
    gx, gv = torch.zeros((n, 3), **f32), torch.zeros((n, 3), **f32)
    gm = torch.zeros(n, **f32)
    ctx.sfc_keys_sort(pos)
    ctx.tree_build(pos, m)
    try:  # h close to the exact relation (4 pi/3) h^3 rho = 64 m
        ctx.density(act, h, 1, sg.GROUPED, 16, rho, drho, fg, nn)
    except sg.SphgrpError as e:
        if e.code != -3:
            raise
    g = a.group
    bw = {"ms": 0.0, "search_ms": 0.0, "launches": [0.0, 0.0, 0.0], "gbs": [0.0, 0.0, 0.0]}
    names = ("density_sums", "hydro_adjoint", "density_adjoint")

    def step(collect):
        ctx.sfc_keys_sort(pos)
        ctx.tree_build(pos, m)
        ctx.density(act, h, 0, sg.GROUPED, g, rho, drho, fg, nn)
        ctx.hydro_force(act, h, rho, fg, vel, u, sg.GROUPED, g, acc, dudt)
        ctx.backward(h, vel, u, w, s, g, gx, gv, gm)
        if collect is not None:
            log = ctx.launch_log()
            bw["search_ms"] += sum(e["ms"] for e in log)
            for k, e in enumerate(log[:3]):
                bw["launches"][k] += e["ms"]
                bw["gbs"][k] += launch_gbs(e, *B_BWD[names[k]])

    for _ in range(warmup):
        step(None)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        step(bw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # the backward call alone
    for _ in range(2):
        ctx.backward(h, vel, u, w, s, g, gx, gv, gm)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        ctx.backward(h, vel, u, w, s, g, gx, gv, gm)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) / steps
    ctx.close()
    peak = measured_peak_hbm()
    return {"workload": f"clustered N={n} (2^{n.bit_length() - 1}), all active, group {g}, "
                        "L = sum w.a + sum s rho, w and s standard normal",
            "value": n / (ms / 1e3), "unit": "particles/s (forward + backward step)", "ms_per_step": ms,
            "backward_value": n / (ms_b / 1e3), "backward_ms": ms_b,
            "backward_search_ms": {k: v / steps for k, v in zip(names, bw["launches"])},
            "backward_roofline": {k: {"achieved_gbs": v / steps, "peak_gbs": peak, "frac": v / steps / peak}
                                  for k, v in zip(names, bw["gbs"])}}


def batch_leg(a, rank: int, steps: int, warmup: int):
    """Batched solve: 96 independent periodic boxes, N per box log-uniform in
    [1e4, 2e6], uniform or clustered by a coin flip, active fraction uniform in
    [1%, 100%].  Set-up: one all-active step (converged h, rho, f of every particle)
    and the per-class autotuner.  A step restores the active particles' h to the
    converged h x exp(0.05 N(0,1)) and runs keys, sort, forest, density with the h
    iteration and hydro (and the backward) for all boxes in one call."""
    import torch

    import paper_1810_09898_gb300 as sg
    import sphgen

    dev = torch.device("cuda", torch.cuda.current_device())
    gen = sphgen.batch(a.batch_boxes, 10_000, 2_000_000, config=5, seed_salt=rank)
    n = int(gen["box_off"][-1])
    f32 = dict(dtype=torch.float32, device=dev)
    t = lambda x, dt=None: torch.from_numpy(np.ascontiguousarray(x)).to(dev, dtype=dt)  # noqa: E731
    io = {"pos": t(gen["pos"]), "m": t(gen["m"], torch.float32), "vel": t(gen["vel"], torch.float32),
          "u": t(gen["u"], torch.float32), "h": t(gen["h0"]), "active": None,
          "rho": torch.zeros(n, **f32), "drhodh": torch.zeros(n, **f32), "fgrad": torch.ones(n, **f32),
          "nngb": torch.zeros(n, dtype=torch.int32, device=dev), "acc": torch.zeros((n, 3), **f32),
          "dudt": torch.zeros(n, **f32)}
    B = sg.Batch(gen["box_off"], gen["box_class"])
    B.run(io)   # all active, cold start
    torch.cuda.synchronize()
    act = t(gen["active"].astype(np.uint8))
    io["active"] = act
    rng = np.random.default_rng(177 + rank)
    hc = io["h"].cpu().numpy()
    hi = np.where(gen["active"], hc * np.exp(0.05 * rng.standard_normal(n)), hc)
    h_init = t(hi)
    io["h"].copy_(h_init)
    t0 = time.perf_counter()
    B.tune(io)
    tune_s = time.perf_counter() - t0
    tuned = {("uniform" if c == 0 else "clustered"): B.get_config(c) for c in (0, 1)}
    for cfg in tuned.values():   # the class's own throughput: one density + hydro pass
        cfg["pass_active_per_s"] = cfg["tuned_members"] / (cfg["tuned_pass_ms"] / 1e3) if cfg["tuned_pass_ms"] else None
    rng2 = np.random.default_rng(277 + rank)
    io["g_acc"] = t(rng2.standard_normal((n, 3)), torch.float32)
    io["g_rho"] = t(rng2.standard_normal(n), torch.float32)
    io["g_pos"], io["g_vel"] = torch.zeros((n, 3), **f32), torch.zeros((n, 3), **f32)
    io["g_m"] = torch.zeros(n, **f32)
    n_act = int(gen["active"].sum())
    stream = torch.cuda.current_stream()

    def run(graph, backward):
        io["h"].copy_(h_init)
        B.run(io, backward=backward, graph=graph)

    def time_it(graph, backward):
        for _ in range(warmup):
            run(graph, backward)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        l0 = sg.kernel_launches()
        e0.record(stream)
        for _ in range(steps):
            run(graph, backward)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, (sg.kernel_launches() - l0) / steps, B.stats()

    ms_e, k_e, _ = time_it(False, False)
    ms_g, k_g, st = time_it(True, False)
    ms_b, k_b, stb = time_it(True, True)
    B.close()
    # the same forward step as one call per box through the single-box entry points
    ctxs = []
    off = gen["box_off"]
    views = []
    for k in range(len(off) - 1):
        lo, hi_ = int(off[k]), int(off[k + 1])
        ctxs.append(sg.Context(hi_ - lo))
        views.append((lo, hi_, torch.nonzero(act[lo:hi_]).flatten().to(torch.int32)))

    def per_box():
        io["h"].copy_(h_init)
        for c, (lo, hi_, ak) in zip(ctxs, views):
            pos = io["pos"][lo:hi_]
            c.sfc_keys_sort(pos)
            c.tree_build(pos, io["m"][lo:hi_])
            c.density(ak, io["h"][lo:hi_], 1, sg.GROUPED, 16, io["rho"][lo:hi_], io["drhodh"][lo:hi_],
                      io["fgrad"][lo:hi_], io["nngb"][lo:hi_])
            c.hydro_force(ak, io["h"][lo:hi_], io["rho"][lo:hi_], io["fgrad"][lo:hi_], io["vel"][lo:hi_],
                          io["u"][lo:hi_], sg.GROUPED, 16, io["acc"][lo:hi_], io["dudt"][lo:hi_])

    per_box()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(2):
        per_box()
    torch.cuda.synchronize()
    ms_p = (time.perf_counter() - t0) / 2 * 1e3
    for c in ctxs:
        c.close()
    return {"workload": f"{a.batch_boxes} periodic boxes, N per box log-uniform in [1e4, 2e6] (total {n}), "
                        "uniform or clustered by coin flip, active fraction uniform in [1%, 100%] "
                        f"({n_act} active), Nngb=64+-2, h restored to converged x exp(0.05 N(0,1)) per step",
            "n_total": n, "n_active": n_act, "unit": "active particles/s",
            "forward_eager": {"ms_per_step": ms_e, "value": n_act / (ms_e / 1e3), "kernels_per_step": k_e},
            "forward_graph": {"ms_per_step": ms_g, "value": n_act / (ms_g / 1e3), "kernels_per_step": k_g,
                              "groups": st["walks"] // 2, "pairs_per_active": st["pairs"] / max(1, 2 * n_act)},
            "forward_backward_graph": {"ms_per_step": ms_b, "value": n_act / (ms_b / 1e3),
                                       "backward_particles": n, "kernels_per_step": k_b},
            "per_box_calls": {"ms_per_step": ms_p, "value": n_act / (ms_p / 1e3),
                              "note": "one single-box call sequence per box (keys, tree, density, hydro), host-timed"},
            "tuned": tuned, "tune_seconds": tune_s}


def small_configs_leg(a, rank: int, reps: int = 3) -> dict:
    """The two smaller workloads, timed beside the main one (CUDA events, median of
    reps calls after one warm-up):
    * uniform N = 32768, all active, h iterated from the uniform-density guess: one density
      call (keys, sort and tree excluded), per-particle form and grouped (g = 16);
    * clustered N = 2^21, 20% active in key-order runs (mean 32), converged h: one density
      pass and one hydro pass for every group size of the sweep and the per-particle form."""
    import torch

    import paper_1810_09898_gb300 as sg
    import sphgen

    dev = torch.device("cuda", torch.cuda.current_device())
    f32 = dict(dtype=torch.float32, device=dev)
    out = {}
    # uniform 32768
    n = 32768
    d = sphgen.make("uniform", n, config=1, seed_salt=rank)
    pos = torch.from_numpy(d["pos"]).to(dev)
    m = torch.from_numpy(d["m"].astype(np.float32)).to(dev)
    c = sg.Context(n)
    c.sfc_keys_sort(pos)
    c.tree_build(pos, m)
    act = torch.arange(n, dtype=torch.int32, device=dev)
    h = torch.empty(n, dtype=torch.float64, device=dev)
    rho, drho, fg = (torch.zeros(n, **f32) for _ in range(3))
    nn = torch.zeros(n, dtype=torch.int32, device=dev)
    u1 = {"workload": "uniform N=32768, all active, h iterated from (3*64/(4 pi N))^(1/3)", "unit": UNIT}
    for name, mode, g in (("individual", sg.INDIVIDUAL, 1), ("grouped", sg.GROUPED, 16)):
        def call():
            h.fill_(d["h0"])
            c.density(act, h, 1, mode, g, rho, drho, fg, nn)
        ms = _median_ms(torch, call, reps)
        u1[name] = {"ms": ms, "value": n / (ms / 1e3), "iterations": c.stats()["iterations"]}
    c.close()
    out["uniform_32768"] = u1
    # clustered 2^21, 20% active, group-size sweep
    n = 1 << 21
    d = sphgen.make("clustered", n, config=2, seed_salt=rank)
    pos = torch.from_numpy(d["pos"]).to(dev)
    m = torch.from_numpy(d["m"].astype(np.float32)).to(dev)
    vel = torch.from_numpy(d["vel"].astype(np.float32)).to(dev)
    u = torch.from_numpy(d["u"].astype(np.float32)).to(dev)
    c = sg.Context(n)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    c.sfc_keys_sort(pos, None, perm)
    c.tree_build(pos, m)
    allact = torch.arange(n, dtype=torch.int32, device=dev)
    h = torch.full((n,), d["h0"], dtype=torch.float64, device=dev)
    rho, drho, fg = (torch.zeros(n, **f32) for _ in range(3))
    nn = torch.zeros(n, dtype=torch.int32, device=dev)
    c.density(allact, h, 1, sg.GROUPED, 16, rho, drho, fg, nn)
    mask = sphgen.active_rank_mask(n, 0.2, 32.0, np.random.default_rng(1000 + rank))
    act = torch.from_numpy(np.sort(perm.cpu().numpy()[np.flatnonzero(mask)]).astype(np.int32)).to(dev)
    na = int(act.shape[0])
    acc, dudt = torch.zeros((n, 3), **f32), torch.zeros(n, **f32)
    sweep = {"workload": f"clustered N={n}, 20% active in key-order runs (mean 32), converged h; one density and "
                         "one hydro pass", "n_active": na, "unit": UNIT}
    for g in (0, 1, 4, 8, 16, 32, 64, 128):
        mode, gs = (sg.INDIVIDUAL, 1) if g == 0 else (sg.GROUPED, g)
        md = _median_ms(torch, lambda: c.density(act, h, 0, mode, gs, rho, drho, fg, nn), reps)
        st = c.stats()
        mh = _median_ms(torch, lambda: c.hydro_force(act, h, rho, fg, vel, u, mode, gs, acc, dudt), reps)
        sweep["individual" if g == 0 else f"g{g}"] = {
            "density_ms": md, "hydro_ms": mh, "value": na / ((md + mh) / 1e3),
            "members_per_walk": st["members"] / max(1, st["walks"]),
            "candidates_per_member": st["candidates"] / max(1, st["members"])}
    best = max((k for k in sweep if k.startswith("g")), key=lambda k: sweep[k]["value"])
    sweep["best"] = best
    sweep["speedup_best_vs_individual"] = sweep[best]["value"] / sweep["individual"]["value"]
    c.close()
    out["clustered_2M_20pct_sweep"] = sweep
    return out


def halo_leg(a, rank: int, world: int = 8) -> dict:
    """The particle set split into `world` key-range domains (Sec. 1.2), on this one GPU:
    how many particles the halo import moves (each domain's particles that another domain's
    boxes reach, density and hydro), the time of the per-domain box and halo-selection
    kernels, and the export volume of the paper's two-phase scheme (Sec. 2.3): a group
    whose walk superset holds particles of another domain exports all its members there,
    per group size g (g = 1: the per-particle walk)."""
    import torch

    import paper_1810_09898_gb300 as sg
    import sphgen
    from paper_1810_09898_gb300.domain import LibOps

    dev = torch.device("cuda", torch.cuda.current_device())
    n = 1 << 21
    d = sphgen.make("clustered", n, config=2, seed_salt=rank)
    pos = torch.from_numpy(d["pos"]).to(dev)
    m = torch.from_numpy(d["m"].astype(np.float32)).to(dev)
    c = sg.Context(n)
    keys = torch.empty(n, dtype=torch.int64, device=dev)
    c.sfc_keys_sort(pos, keys)
    c.tree_build(pos, m)
    act = torch.arange(n, dtype=torch.int32, device=dev)
    h = torch.full((n,), d["h0"], dtype=torch.float64, device=dev)
    f32 = dict(dtype=torch.float32, device=dev)
    rho, drho, fg = (torch.zeros(n, **f32) for _ in range(3))
    nn = torch.zeros(n, dtype=torch.int32, device=dev)
    c.density(act, h, 1, sg.GROUPED, 16, rho, drho, fg, nn)
    split = keys[[n * j // world for j in range(1, world)]].contiguous()
    lib = LibOps()
    mask = lib.owner_mask(pos, split)
    owner = sum(w * ((mask >> w) & 1) for w in range(world))   # the set bit's index
    doms = [torch.nonzero(owner == r).flatten() for r in range(world)]
    out = {"workload": f"clustered N={n}, converged h, {world} key-range domains"}
    for level in (3, 4):
        boxes, ranks = [], []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r in range(world):
            b = lib.boxes(pos[doms[r]].contiguous(), m[doms[r]].contiguous(), h[doms[r]].contiguous(), level)
            boxes.append(b)
            ranks.append(torch.full((b.shape[0],), r, dtype=torch.int32, device=dev))
        B, R = torch.cat(boxes).contiguous(), torch.cat(ranks).contiguous()
        rec = {"boxes": int(B.shape[0])}
        for kind, name in ((0, "density"), (1, "hydro")):
            ghosts = 0
            for r in range(world):
                mk = lib.halo_mask(pos[doms[r]].contiguous(), m[doms[r]].contiguous(), h[doms[r]].contiguous(), kind,
                                   1.0, B, R, r, world)
                ghosts += int(sum(((mk >> w) & 1).sum().item() for w in range(world)))
            rec[f"import_{name}_per_particle"] = ghosts / n
        torch.cuda.synchronize()
        rec["boxes_and_selection_s"] = time.perf_counter() - t0
        out[f"level{level}"] = rec
    lib.close()
    # the export volume of the two-phase scheme, per group size
    exp = {}
    for g in (1, 4, 8, 16, 32, 64):
        goff = torch.empty(n + 1, dtype=torch.int64, device=dev)
        ng, total = c.group_supersets(act, h, 0, g, goff)
        gfirst = torch.empty(n + 1, dtype=torch.int32, device=dev)
        mem = torch.empty(n, dtype=torch.int32, device=dev)
        cand = torch.empty(total, dtype=torch.int32, device=dev)
        c.group_supersets(act, h, 0, g, goff, gfirst, mem, cand, cap=total)
        cg = torch.repeat_interleave(torch.arange(ng, device=dev), (goff[1:ng + 1] - goff[:ng]))
        present = torch.zeros(ng * world, dtype=torch.int64, device=dev)
        present[cg * world + owner[cand.long()]] = 1
        present = present.view(ng, world)
        mg = torch.repeat_interleave(torch.arange(ng, device=dev), (gfirst[1:ng + 1] - gfirst[:ng]).long())
        other = present.sum(1)[mg] - present[mg, owner[mem.long()]]
        exp[f"g{g}"] = int(other.sum().item()) / n
        del cand, goff
    out["export_per_particle"] = exp
    out["export_g16_over_g1"] = exp["g16"] / max(exp["g1"], 1e-30)
    c.close()
    return out


def measured_peak_hbm() -> float:
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def run_ours(a):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as tdist

        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)
    P = Problem(a, rank)
    sg = P.sg
    g = a.group
    if a.profile_pass:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("pass")
        for mode, gs in ((sg.GROUPED, g), (sg.INDIVIDUAL, 1)):
            P.ctx.density(P.act, P.h, 0, mode, gs, P.rho, P.drho, P.f, P.nn)
            P.ctx.hydro_force(P.act, P.h, P.rho, P.f, P.vel, P.u, mode, gs, P.acc, P.dudt, P.nnh)
        divv = torch.empty(P.n, dtype=torch.float32, device=P.dev)
        curl = torch.empty((P.n, 3), dtype=torch.float32, device=P.dev)
        P.ctx.velocity_derivs(P.act, P.h, P.rho, P.vel, g, divv, curl)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        print(json.dumps({"profile_pass": "done", "n": P.n}))
        return
    steps, warmup = a.steps, max(3, a.warmup)

    with ClockSampler(torch.cuda.current_device()) as clk:
        ms_g, col_g, launches = timed(P, lambda c: P.step(sg.GROUPED, g, c), steps, warmup, dist)
    clocks = clk.summary()
    ms_i = None
    col_i = []
    if not a.no_individual:
        ms_i, col_i, _ = timed(P, lambda c: P.step(sg.INDIVIDUAL, 1, c), steps, warmup, dist)
    passes = {"grouped": guarded(per_pass, P, sg.GROUPED, g)}
    if not a.no_individual:
        passes["individual"] = guarded(per_pass, P, sg.INDIVIDUAL, 1)
        if "value" in passes["grouped"] and "value" in passes["individual"]:
            passes["speedup_grouped"] = passes["grouped"]["value"] / passes["individual"]["value"]
    vel_derivs = guarded(velocity_pass, P, g)
    low_active = None
    if a.active >= 1.0 and not a.no_individual:
        low_active = guarded(active_leg, P, 0.1, g, steps, warmup, dist, rank)
    e2e = None
    if not a.no_e2e:
        for _ in range(2):
            P.step_e2e(g)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            P.step_e2e(g)
        t_e2e = max_over_ranks((time.perf_counter() - t0) / steps, dist, P.dev)
        h2d, d2h = P.io_bytes()
        e2e = {"value": replicas_value(world, P.n_act, 1e3 * t_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * t_e2e}
    back = None
    if not a.no_backward:
        back = guarded(backward_leg, a, rank, steps, warmup)
    batch = None
    if not a.no_batch:
        batch = guarded(batch_leg, a, rank, steps, warmup)
    small = None if a.no_small else guarded(small_configs_leg, a, rank)
    halo = None if a.no_halo else guarded(halo_leg, a, rank)
    peak = measured_peak_hbm()
    roof, detail = roofline(col_g, peak, clocks)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = cpu_sample(a.cpu_n, a.h_scatter)
        cpu.pop("seconds", None)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    ms_step = ms_g / steps
    value = replicas_value(world, P.n_act, ms_step)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(a), "n": P.n, "n_active": P.n_act, "group_size": g,
                   "form": "grouped", "positions": "f64 (fixed-point + f32 offsets on device)",
                   "h_init": f"converged h x exp({a.h_scatter} N(0,1)) per step",
                   "l2": "inputs larger than L2 (no flush needed)", "parallelism": f"replicas x{world}"},
        "individual": None if ms_i is None else {
            "value": replicas_value(world, P.n_act, ms_i / steps), "ms_per_step": ms_i / steps,
            "speedup_grouped": (ms_i / steps) / ms_step},
        "roofline": roof,
        "search_detail": detail,
        "cold_start": {"seconds": P.cold_s, "iterations": P.cold_stats["iterations"]},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "per_pass_converged_h": passes,
        "velocity_derivs": vel_derivs,
        "active_10pct": low_active,
        "backward": back,
        "batch": batch,
        "small_configs": small,
        "domain_halo": halo,
    }
    if ms_i is not None:
        ri, di = roofline(col_i, peak, clocks, form="individual")
        line["individual"]["roofline"] = ri
        line["individual"]["search_detail"] = di
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
