#!/usr/bin/env python3
"""Benchmark of the multirange Shan-Chen lattice Boltzmann step on GB300.

One "step" is one pass of the whole hot path over the lattice: density and pseudopotential,
two-belt + cross + body force, shifted-velocity BGK collision, streaming with walls, and the
observables of the collided state (mass, momentum, profiles, pressure tensor, surface tension,
wall stress, fluidity) reduced in FP64 -- i.e. lbm_step with sampling every step.

Default workload: the two-component A/B emulsion on a 1024 x 1024 periodic lattice, FP32
populations stored as deviations, FP64 reductions (disk packing at fraction 0.8, radii
12 +- 3, G_AA = (-9.0, 8.1), G_BB = (-8.0, 7.1), G_AB = 0.405, rho0 = 0.83).

Metric: MLUPS (million lattice-site updates per second, whole job).  Default L2 handling: four
lattices of the workload are stepped in turn (each step's input comes from DRAM); --l2 flush
writes and reads a buffer larger than L2 between steps.  The timed region is bracketed by CUDA
events on the library's stream.  Roofline: the step kernel's average launch duration over the
timed region (one launch per step); a second pass with events around every launch
(lbm_profile) gives its serialised duration.  --workload adjoint_256 measures gradients of a run
(forward, recompute, adjoint) instead.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
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

BYTES_PER_SITE = {("fp32", 2): 144, ("fp64", 2): 288, ("fp32", 1): 72, ("fp64", 1): 144}
# The FP64 step (two species, observables every step) is bound by the FP64 pipe: FP64 flops per
# site-update counted by ncu (242 DFMA, 244 DADD, 119 DMUL; profiles/k_pull_emulsion_1024_fp64.md)
# against 2 DFMA per SM per cycle x 152 SMs x 2 flops x 2.07 GHz
FP64_FLOPS_PER_SITE = 847
FP64_INSTR_PER_SITE = 605  # the same counts as instructions: each occupies the FP64 pipe once
FP64_PEAK_TFLOPS = 304 * 2 * 2.07e9 / 1e12
L2_FLUSH_BYTES = 256 << 20
L2_BYTES = 126 << 20          # L2 of a GB300 (nvidia-smi / device properties: 126.5 MiB)
ROTATE_BYTES = 512 << 20      # working set of the rotated lattices, well above L2
E2E_RUN = 32                  # steps per lbm_step_read call of the end-to-end measurement


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 2000 lattice steps; 5 gradients for adjoint_256; for the reference "
                         "arm 20 oracle steps, 2 oracle gradients)")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="emulsion_1024")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--rows-per-warp", type=int, default=0)
    ap.add_argument("--kernel", choices=["pull", "fused", "twopass", "sweep"], default="pull")
    ap.add_argument("--tile-rows", type=int, default=0, help="FUSED kernel tile height (8 or 16; 0 = auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=500)
    ap.add_argument("--clocks-csv", default=None, help="keep the raw nvidia-smi clock samples in this file")
    ap.add_argument("--l2", choices=["rotate", "flush", "none"], default="rotate",
                    help="rotate: step several lattices of the workload in turn, so that each step's input "
                         "was evicted from L2 by the others' traffic (no flush); flush: one lattice, a 256 MiB "
                         "write then a 256 MiB read between timed steps; none: one lattice stepped back to back "
                         "(a step's input is what the step before wrote)")
    ap.add_argument("--autotune", type=int, default=0, metavar="STEPS",
                    help="before timing, let the library pick the pull kernel's tile width and pipeline depth by "
                         "timing STEPS steps of each (lbm_autotune_tiles; 0 = the default shape)")
    ap.add_argument("--graph", type=int, default=1,
                    help="1: the timed region replays the captured step launches as one CUDA graph (the rotating "
                         "lattices only); 0: one library call per step inside the region")
    ap.add_argument("--observe-every", type=int, default=1,
                    help="sample the observables every k steps (1 = every step, the full hot path; "
                         "0 = never, for analysis only)")
    return ap.parse_args()


def _dist():
    from paper_1402_6019_gb300 import replicas

    r = replicas.from_env()
    return r.rank, r.world, r.local


class _Nvml:
    """Read-only NVML queries through ctypes (SM clock, its maximum, power, clock event reasons);
    nothing is set."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake"}

    def __init__(self, index, pci_bus_id=None):
        import ctypes

        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        ok = False
        if pci_bus_id:
            ok = self.lib.nvmlDeviceGetHandleByPciBusId_v2(pci_bus_id.encode(), ctypes.byref(self.h)) == 0
        if not ok and self.lib.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        self.max_mhz = float(mx.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0 else None

    def sample(self):
        ct = self.ct
        clk, pw, rs = ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(clk)) != 0:  # NVML_CLOCK_SM
            return None
        self.lib.nvmlDeviceGetPowerUsage(self.h, ct.byref(pw))
        self.reasons_fn(self.h, ct.byref(rs))
        return (time.perf_counter(), float(clk.value), pw.value / 1000.0, int(rs.value))


class Clocks:
    """SM clocks and clock event reasons during the timed region: NVML read every 5 ms by a thread,
    plus one read right before and one right after the region (so a region shorter than the
    period still carries clocks and reasons); nvidia-smi sampling every 50 ms where NVML cannot be
    loaded.
    Read-only: no clock, power or other setting is changed."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    # where the raw nvidia-smi samples go (--clocks-csv); by default a temporary file
    csv_path = None

    def __init__(self, index, pci_bus_id=None):
        self.index = index
        self.proc = None
        self.nvml = None
        self.samples = []
        self.edges = []
        try:
            self.nvml = _Nvml(index, pci_bus_id)
        except (OSError, AttributeError):
            self.nvml = None
        self.path = Clocks.csv_path or os.path.join(tempfile.gettempdir(), f"lbm_clocks_{os.getpid()}.csv")

    # polling interval: NVML reads every millisecond slowed a 20-step region by about 2 %
    # (measured); every 5 ms they do not show, and short regions keep the reads at their edges
    PERIOD_S = 0.005

    def _poll(self):
        while not self.stop.wait(self.PERIOD_S):
            smp = self.nvml.sample()
            if smp:
                self.samples.append(smp)

    def __enter__(self):
        if self.nvml:
            import threading

            self.edges.append(self.nvml.sample())
            self.stop = threading.Event()
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            return self
        try:
            if os.path.dirname(self.path):
                os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.nvml:
            self.stop.set()
            self.thread.join(timeout=5)
            self.edges.append(self.nvml.sample())
            return
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.nvml:
            rows = [r for r in self.samples if r]
            edges = [r for r in self.edges if r]
            allr = rows or edges
            if not allr:
                return None
            reasons = sorted({name for r in allr + edges for bit, name in _Nvml.REASONS.items() if r[3] & bit})
            return {"sm_mhz": float(np.median([r[1] for r in allr])), "sm_max_mhz": self.nvml.max_mhz,
                    "reasons": reasons, "samples": len(rows),
                    "sm_mhz_before_after": [r[1] for r in edges], "power_w_max": max(r[2] for r in allr),
                    "source": "NVML every 5 ms during the timed region, and once right before and after it"}
        if not self.proc:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    pass
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": rows[0][1],
                "reasons": reasons, "samples": len(rows), "source": "nvidia-smi every 50 ms"}


def _pci_bus_id(local):
    try:
        import torch

        p = torch.cuda.get_device_properties(local)
        return f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
    except Exception:
        return None


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _traffic(kernel_src_hash, workload, precision, kernel):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, or None when
    the summary is for another source of the kernel, another kernel or another workload."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    e = d.get(f"{workload}/{precision}/{kernel}")
    if not e or e.get("kernel_source_sha1") != kernel_src_hash:
        return None
    return e.get("dram_bytes_per_launch")


_CORE = ("lbm_core.cuh", "lbm_pair.cuh", "lbm_reduce.cuh")
KERNEL_SOURCE = {"pull": ("lbm_pull.cu",) + _CORE, "fused": ("lbm_tile.cu",) + _CORE,
                 "twopass": ("lbm_twopass.cu",) + _CORE, "sweep": ("lbm_fused.cu",) + _CORE,
                 "k3_step": ("lbm3d.cu",), "k3_density": ("lbm3d.cu",)}


def kernel_source_hash(kernel):
    """SHA-1 of the sources a kernel is compiled from: a committed DRAM-traffic figure holds
    only for the source it was captured on."""
    h = hashlib.sha1()
    for f in KERNEL_SOURCE[kernel]:
        h.update(open(os.path.join(ROOT, "paper_1402_6019_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def oracle_sample(w, n=256):
    """The oracle's bounded sample of a workload: an n x n cut (of the tallest channel of a
    batch, with its drive) as (rho, n_species, z_boundary, params)."""
    if "instances" in w:
        i = int(np.argmax(w["instances"]))
        z0 = int(np.sum(w["instances"][:i]))
        rho = w["rho"][:, z0:z0 + min(n, w["instances"][i]), :n]
        return np.ascontiguousarray(rho), dict(w["params"], **w["drives"][i])
    return np.ascontiguousarray(w["rho"][:, :n, :n]), dict(w["params"])


def cpu_baseline(w, seconds=12.0, lib_run=None, tol=1e-4, err_steps=1000):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of the workload:
    whole oracle steps (step + observables, like the GPU step) on a 256 x 256 lattice cut from
    the same workload, until `seconds` of wall time have passed.

    With `lib_run`, the same oracle run then goes on (untimed, without observables) to
    `err_steps` steps, and the library's run of the same cut over as many steps (observables every
    step) is compared with it: the state (rho, u) and every observable, each as its largest error
    relative to the oracle's largest value, and as a fraction of the bound the state contract
    `tol` allows it (paper_1402_6019_gb300.accuracy)."""
    import oracle

    oracle.build()
    n = 256
    rho, prm = oracle_sample(w, n)
    cz, cx = rho.shape[1], rho.shape[2]  # the cut (smaller than n x n when the lattice is)
    ref = oracle.RefLattice(cx, cz, w["n_species"], w["z_boundary"], **prm)
    ref.set_fields(rho)
    t0 = time.perf_counter()
    k = 0
    while True:
        ref.step(1)
        ref.observables()
        k += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": round(cx * cz * k / dt / 1e6, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
           "sample": f"{k} oracle steps (step + observables) on a {cx}x{cz} cut of the workload, "
                     f"{dt:.1f} s wall, OpenMP threads={cores}"}
    if lib_run is None:
        return out, None
    from paper_1402_6019_gb300 import accuracy

    steps = max(err_steps, k)
    ref.step(steps - k)
    r_rho, r_u, _ = ref.fields()
    r_obs = ref.observables()
    g_rho, g_u, g_obs = lib_run(rho, prm, steps)
    rel = lambda a, b: float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
    errs = accuracy.observable_errors(g_obs, r_obs, ref.scales(), tol, cx, float(np.sum(r_obs["mass"])))
    errors = {"vs": "FP64 oracle", "sample": f"{cx}x{cz} cut of the workload, {steps} steps, "
                                             "observables every step (the library's launch configuration)",
              "tol": tol, "rho": rel(g_rho, r_rho), "u": rel(g_u, r_u),
              "observables": {k_: {"rel": float(f"{e[2]:.3g}"),
                                   "of_bound": float(f"{e[0] / e[1]:.3g}") if 0 < e[1] < float("inf") else None,
                                   "entries": e[3]} for k_, e in errs.items()},
              "rel": "largest |library - oracle| / largest |oracle| of each quantity (momentum: over total "
                     "mass x max |u|, its own value being near zero)",
              "entries": "entries compared (fluid_z: rows where |S_xz| exceeds twice its bound, the ratio being "
                         "undetermined elsewhere)",
              "of_bound": "largest error / the bound the state contract allows (tol x the magnitude of the "
                          "terms the observable is formed from)",
              "within_bounds": not accuracy.check(errs) and rel(g_rho, r_rho) <= tol and rel(g_u, r_u) <= tol}
    return out, errors


def run_reference(a, w):
    """--impl reference: the FP64 oracle timed on the host cores on a bounded sample of the
    workload (a 256 x 256 cut): W warm-up steps then K timed steps, each = oracle step +
    observables, MLUPS over the sample's sites."""
    import oracle

    rank, world, _ = _dist()
    if rank != 0:
        return
    oracle.build()
    n = 256
    rho, prm = oracle_sample(w, n)
    cz, cx = rho.shape[1], rho.shape[2]
    ref = oracle.RefLattice(cx, cz, w["n_species"], w["z_boundary"], **prm)
    ref.set_fields(rho)
    for _ in range(a.warmup):
        ref.step(1)
        ref.observables()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        ref.step(1)
        ref.observables()
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    value = cx * cz * a.steps / dt / 1e6
    sample = f"{a.steps} timed oracle steps (step + observables) on a {cx}x{cz} cut of {a.workload}"
    print(json.dumps({
        "impl": "reference", "metric": "MLUPS", "value": round(value, 4), "unit": "MLUPS",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(dt / a.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": a.workload, "sample": f"{cx}x{cz}"},
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# adjoint kernels: values read and written per site and species (states, lam, intermediate
# fields of the site; neighbour values come from cache): k_adj_moments reads f (9) and writes
# rho, j, psi (4); k_adj_local reads f and lam_{n+1} (18) and rho, j, psi (4), and writes
# psi dF, rho dF (4), the site's own dJ/drho, dJ/dj and psi' (4); k_adj_final reads lam_{n+1}
# (9) and those 8 fields and writes lam_n (9)
ADJ_VALUES = {"moments": 13, "local": 30, "final": 26}


def adjoint_sample(w, n=64, steps=20):
    """The oracle's bounded sample of the calibration workload: an n x n cut, `steps` steps."""
    rho = np.ascontiguousarray(w["rho"][:, :n, :n])
    return rho, w["target_u"][:n].copy(), w["target_rho"][:n].copy(), steps


def cpu_baseline_adjoint(w, seconds=12.0):
    """The oracle's run gradient (forward storing every state, adjoint step by step) on a bounded
    sample of the calibration workload, repeated until `seconds` have passed."""
    import oracle

    oracle.build()
    rho, tu, tr, steps = adjoint_sample(w)
    n = rho.shape[1]
    t0 = time.perf_counter()
    k = 0
    while True:
        oracle.rollout_gradient(n, n, w["n_species"], rho, steps, tu, tr, **w["params"])
        k += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": round(n * n * steps * k / dt / 1e6, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{k} oracle run gradients ({steps} steps forward + {steps} adjoint steps) on a {n}x{n} cut "
                      f"of the workload, {dt:.1f} s wall, OpenMP threads={cores} (forward steps; the adjoint is "
                      "single-threaded)"}


def run_reference_adjoint(a, w):
    import oracle

    rank, world, _ = _dist()
    if rank != 0:
        return
    oracle.build()
    rho, tu, tr, steps = adjoint_sample(w)
    n = rho.shape[1]
    for _ in range(a.warmup):
        oracle.rollout_gradient(n, n, w["n_species"], rho, steps, tu, tr, **w["params"])
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle.rollout_gradient(n, n, w["n_species"], rho, steps, tu, tr, **w["params"])
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    value = n * n * steps * a.steps / dt / 1e6
    sample = f"{a.steps} timed oracle run gradients of {steps} steps on a {n}x{n} cut of {a.workload}"
    print(json.dumps({
        "impl": "reference", "metric": "MLUPS", "value": round(value, 4), "unit": "MLUPS",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(dt / a.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": a.workload, "sample": f"{n}x{n}, {steps} steps"},
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_adjoint(a, w):
    """The calibration workload: one bench step = one whole gradient of the run (forward with a
    snapshot every `checkpoint` steps, objective, then per segment restore + recorded recompute
    + adjoint sweep, and the initial-density gradient).  MLUPS = differentiated site-steps per
    second."""
    import torch

    from paper_1402_6019_gb300 import adjoint as A
    from paper_1402_6019_gb300 import lbm as L
    from paper_1402_6019_gb300 import replicas

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_

        dist_.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    nx, nz, ns, run_steps, ck = w["nx"], w["nz"], w["n_species"], w["steps"], w["checkpoint"]
    sites = nx * nz
    prec = L.LBM_FP32 if a.precision == "fp32" else L.LBM_FP64
    esize = 4 if a.precision == "fp32" else 8
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)  # torch's work and the library's share one stream
    lat = L.Lattice(nx, nz, ns, prec, L.LBM_PERIODIC, device=local, stream=stream.cuda_stream, **w["params"])
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    rho, tu, tr = dev(w["rho"]), dev(w["target_u"]), dev(w["target_rho"])
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    flush_src = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def gradient():
        return A.rollout_gradient(lat, rho, run_steps, tu, tr, checkpoint=ck)

    for _ in range(a.warmup):
        gradient()
    barrier()

    def timed(profile):
        if profile:
            L.lbm_profile(lat.h, True)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
        for k in range(a.steps):
            flush.fill_(float(k))  # no data of the previous gradient left in L2
            flush_src.sum()
            starts[k].record(stream)
            gradient()
            ends[k].record(stream)
        barrier()
        return float(sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)))

    launches0 = lat.launches
    with Clocks(local, _pci_bus_id(local)) as clk:
        grad_ms = timed(False)
    launches = lat.launches - launches0
    # the same gradients again with every step-kernel and adjoint-kernel launch bracketed by
    # events (which also runs the steps one by one instead of in graphs): the kernel durations
    prof_ms = timed(True)
    step_ms, step_n = L.lbm_profile_read(lat.h)
    adj_ms, adj_n = L.lbm_profile_read_adjoint(lat.h)
    L.lbm_profile(lat.h, False)
    grad_s, job = replicas.aggregate(grad_ms * 1e-3, sites * run_steps * a.steps, dist=dist, device="cuda")
    ms_per_grad = grad_s * 1e3 / a.steps
    value = job / grad_s / 1e6

    # the dominant kernel of the gradient: the step kernel (forward and recompute) or one of the
    # three adjoint kernels, by summed event time
    kernels = {"lbm::k_pull<T, 2, M_WRITE>": (step_ms, step_n, 2 * 9 * ns * esize)}
    for name, ms in zip(("moments", "local", "final"), adj_ms):
        kernels[f"lbm::k_adj_{name}<T, {ns}>"] = (ms, adj_n, ADJ_VALUES[name] * ns * esize)
    top = max(kernels, key=lambda k: kernels[k][0])
    ms, n, bps = kernels[top]
    avg = ms / max(n, 1)
    achieved = bps * sites / (avg * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None, "peak_source": peak_kind, "kernel": top,
                "kernel_ms": round(avg, 5), "algorithmic_bytes_per_site": bps,
                "share_of_gradient": round(ms / max(prof_ms, 1e-9), 3),
                "kernels_ms_per_gradient": {k: round(v[0] / a.steps, 3) for k, v in kernels.items()},
                "timing": "kernel durations from CUDA events around every launch in a second, profiled "
                          f"pass over the same {a.steps} gradients ({prof_ms / a.steps:.2f} ms per gradient "
                          "with the events)"}

    # end to end through the public API with host buffers: the initial densities uploaded from
    # pinned host memory, the gradients (densities and parameters) and J read back
    rho_pin = torch.from_numpy(np.ascontiguousarray(w["rho"])).pin_memory()
    barrier()
    t0 = time.perf_counter()
    e2e_n = max(1, min(a.steps, 3))
    for _ in range(e2e_n):
        r = rho_pin.to("cuda", non_blocking=True)
        J, g_rho, grad = A.rollout_gradient(lat, r, run_steps, tu, tr, checkpoint=ck)
        g_host, th_host = g_rho.cpu(), grad.cpu()
    barrier()
    dt, e2e_job = replicas.aggregate(time.perf_counter() - t0, sites * run_steps * e2e_n, dist=dist, device="cuda")
    e2e = {"value": round(e2e_job / dt / 1e6, 2), "unit": "MLUPS", "h2d_bytes_per_step": int(rho_pin.numel() * 8),
           "d2h_bytes_per_step": int(g_host.numel() * 8 + th_host.numel() * 8 + 8), "steps": e2e_n}
    if rank != 0:
        return
    line = {
        "metric": "MLUPS", "value": round(value, 2), "unit": "MLUPS", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(ms_per_grad, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if a.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": a.workload, "nx": nx, "nz": nz, "n_species": ns, "precision": a.precision,
                   "run_steps": run_steps, "checkpoint": ck,
                   "step": "one gradient: forward with snapshots, objective, recompute + adjoint per segment",
                   "unit": "differentiated site-steps per second",
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "a 256 MiB write then a 256 MiB read between timed gradients"},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_adjoint(w)
    print(json.dumps(line))


# the 3-D step (D3Q19, two species): the method reads and writes each population once (304 B per
# site-update in FP32); the collide pass k3_step itself reads the site's populations and the
# psi / rho pairs and writes the pushed populations (152 + 16 + 152 = 320 B), the density pass
# reads the populations and writes the pairs (168 B)
BYTES3 = {"fp32": {"step": 304, "k3_step": 320, "k3_density": 168},
          "fp64": {"step": 608, "k3_step": 640, "k3_density": 336}}


def oracle3_run(w, n, steps):
    """The 3-D oracle on an n^3 cut of the workload: (RefLattice3D after `steps` steps, seconds)."""
    from oracle import ref3d

    ref3d.build()
    rho = np.ascontiguousarray(w["rho"][:, :n, :n, :n])
    keys = ("tau", "G1", "G2", "G_AB", "rho0", "weight_norm", "body_force", "psi_form", "wall_u")
    ref = ref3d.RefLattice3D(n, n, n, w["n_species"], zbc=w["z_boundary"],
                             **{k: w["params"][k] for k in keys if k in w["params"]})
    ref.set_fields(rho)
    t0 = time.perf_counter()
    ref.step(steps)
    return ref, time.perf_counter() - t0, rho


def run_reference_3d(a, w):
    rank, world, _ = _dist()
    if rank != 0:
        return
    n = 32
    oracle3_run(w, n, a.warmup)
    _, dt, _ = oracle3_run(w, n, a.steps)
    value = n ** 3 * a.steps / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = f"{a.steps} timed 3-D oracle steps on a {n}^3 cut of {a.workload}, OpenMP threads={cores}"
    print(json.dumps({
        "impl": "reference", "metric": "MLUPS", "value": round(value, 4), "unit": "MLUPS",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(dt / a.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": a.workload, "sample": f"{n}^3"},
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_3d(a, w):
    """The three-dimensional extension: one bench step = lbm3_step(1), a density pass and a collide
    pass over the whole lattice (128^3 x 2 species: 318 MB of populations per copy, well above
    L2, so every step reads its input from HBM)."""
    import torch

    from paper_1402_6019_gb300 import lbm as L
    from paper_1402_6019_gb300 import replicas

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_

        dist_.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    nx, ny, nz, ns = w["nx"], w["ny"], w["nz"], w["n_species"]
    sites = nx * ny * nz
    prec = L.LBM_FP32 if a.precision == "fp32" else L.LBM_FP64
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    lat = L.Lattice3(nx, ny, nz, ns, prec, w["z_boundary"], device=local, stream=stream.cuda_stream, **w["params"])
    lat.set_fields(w["rho"])
    # the collide pass's tile shape, picked by the library's autotuner on this lattice (untimed)
    shape, tune_ms = lat.autotune(max(a.autotune, 10))
    lat.step(a.warmup)
    lat.synchronize()
    barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local, _pci_bus_id(local)) as clk:
        t0.record(stream)
        lat.step(a.steps)
        t1.record(stream)
        barrier()
    step_ms = float(t0.elapsed_time(t1))
    lat.synchronize()
    # the same number of steps with events around each of the two kernels
    lat.profile(True)
    lat.step(a.steps)
    d_ms, c_ms, nstep = lat.profile_read()
    lat.profile(False)
    step_s, job_sites = replicas.aggregate(step_ms * 1e-3, sites, dist=dist, device="cuda")
    ms_per_step = step_s * 1e3 / a.steps
    value = job_sites / (ms_per_step * 1e-3) / 1e6
    peak, peak_kind = _peaks()
    B = BYTES3[a.precision]
    kd, kc = d_ms / max(nstep, 1), c_ms / max(nstep, 1)
    top, kms = ("k3_step", kc) if kc >= kd else ("k3_density", kd)
    achieved = B[top] * sites / (kms * 1e-3) / 1e9
    traffic = _traffic(kernel_source_hash(top), a.workload, a.precision, top)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": traffic,
                "peak_source": peak_kind,
                "kernel": f"lbm3::{top}<T, ...>", "kernel_ms": round(kms, 5),
                "algorithmic_bytes_per_site": B[top],
                "kernels_ms": {"k3_density": round(kd, 5), "k3_step": round(kc, 5)},
                "step_frac": round(B["step"] * value * 1e6 / 1e9 / peak, 4),
                "step_bytes_per_site": B["step"],
                "timing": "kernel durations from CUDA events around each kernel in a second pass over the same "
                          "number of steps; step_frac = the method's bytes per site-update x MLUPS / peak"}
    # end to end: densities uploaded from pinned host memory, then the steps in runs of E2E_RUN,
    # each step's totals (mass, momentum) written into pinned host memory by the library
    # (lbm3_step_totals), two runs in flight while the oldest run's records are read
    e2e = None
    if a.e2e_steps > 0:
        rho_pin = torch.from_numpy(np.ascontiguousarray(w["rho"])).pin_memory()
        nsteps = a.e2e_steps
        bufs = [torch.zeros((E2E_RUN, 5), dtype=torch.float64).pin_memory() for _ in range(3)]
        barrier()
        tt = time.perf_counter()
        lat.set_fields(rho_pin.numpy())
        pending, left, k, last = [], nsteps, 0, None
        while left > 0:
            n = min(E2E_RUN, left)
            buf = bufs[k % 3]
            k += 1
            pending.append((lat.step_totals(n, buf), buf, n))
            left -= n
            if len(pending) > 2:
                t, buf, n = pending.pop(0)
                lat.wait(t)
                last = buf[:n].numpy().copy()
        for t, buf, n in pending:
            lat.wait(t)
            last = buf[:n].numpy().copy()
        lat.synchronize()
        barrier()
        dt, e2e_sites = replicas.aggregate(time.perf_counter() - tt, sites * nsteps, dist=dist, device="cuda")
        e2e = {"value": round(e2e_sites / dt / 1e6, 2), "unit": "MLUPS",
               "h2d_bytes_per_step": int(rho_pin.numel() * 8 // nsteps), "d2h_bytes_per_step": 40,
               "steps": nsteps, "read": f"the densities uploaded from pinned host memory once, then runs of "
                                        f"{E2E_RUN} steps by lbm3_step_totals, every step's mass and momentum "
                                        f"written into pinned host memory; two runs in flight while the oldest "
                                        f"run's records are read (last total mass {float(last[-1][:ns].sum()):.6e})"}
    if rank != 0:
        return
    line = {
        "metric": "MLUPS", "value": round(value, 2), "unit": "MLUPS", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if a.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": a.workload, "nx": nx, "ny": ny, "nz": nz, "n_species": ns, "precision": a.precision,
                   "lattice": "D3Q19", "parallelism": f"replicas{world}" if world > 1 else "single",
                   "tile_shape": ["32x4x2", "32x2x4", "32x8x1", "32x4x4"][shape],
                   "autotune_ms_per_step": [round(t, 5) for t in tune_ms],
                   "l2": f"one lattice of {2 * 19 * ns * sites * (4 if a.precision == 'fp32' else 8) / 2**20:.0f} "
                         f"MiB of populations (both copies) > {L2_BYTES / 2**20:.0f} MiB L2; no flush"},
        "roofline": roofline, "e2e": e2e, "gpu_launches": 2 * a.steps, "clocks": clk.summary(),
    }
    if world == 1 and not a.no_cpu_baseline:
        n = 32
        ref, dt, rho = oracle3_run(w, n, 20)
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        line["cpu_baseline"] = {"value": round(n ** 3 * 20 / dt / 1e6, 4), "unit": "MLUPS", "cores": cores,
                                "kind": "oracle", "sample": f"20 steps of the 3-D oracle on a {n}^3 cut of the "
                                                            f"workload, {dt:.1f} s, OpenMP threads={cores}"}
        g = L.Lattice3(n, n, n, ns, prec, w["z_boundary"], device=local, stream=stream.cuda_stream, **w["params"])
        g.set_fields(rho)
        g.step(20)
        r_rho, r_u, _ = ref.fields()
        g_rho, g_u, _ = g.fields(populations=False)
        rel = lambda x, y: float(np.abs(x - y).max() / max(np.abs(y).max(), 1e-300))
        line["errors"] = {"vs": "FP64 3-D oracle", "sample": f"{n}^3 cut, 20 steps", "rho": rel(g_rho, r_rho),
                          "u": rel(g_u, r_u)}
    print(json.dumps(line))


def main():
    a = _args()
    Clocks.csv_path = a.clocks_csv
    from paper_1402_6019_gb300 import workloads as W

    from paper_1402_6019_gb300 import replicas

    rank, world, local = _dist()
    w = W.workload(a.workload, seed=replicas.replica_seed(1402, replicas.from_env()))
    if a.steps is None:
        a.steps = {("ours", False): 2000, ("ours", True): 5, ("reference", False): 20,
                   ("reference", True): 2}[(a.impl, "target_u" in w)]
    if "target_u" in w:  # the calibration workload: gradients of a run
        return run_reference_adjoint(a, w) if a.impl == "reference" else run_adjoint(a, w)
    if w.get("dim") == 3:  # the three-dimensional extension
        return run_reference_3d(a, w) if a.impl == "reference" else run_3d(a, w)
    if a.impl == "reference":
        return run_reference(a, w)

    import torch

    from paper_1402_6019_gb300 import lbm as L

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_

        dist_.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    nx, nz, ns = w["nx"], w["nz"], w["n_species"]
    sites = nx * nz
    prec = L.LBM_FP32 if a.precision == "fp32" else L.LBM_FP64
    # a non-default stream: the library runs on it, and the events below are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    kern = {"pull": L.LBM_KERNEL_PULL, "fused": L.LBM_KERNEL_FUSED, "twopass": L.LBM_KERNEL_TWO_PASS,
            "sweep": L.LBM_KERNEL_SWEEP}[a.kernel]
    def make_lattice():
        lt = L.Lattice(nx, nz, ns, prec, w["z_boundary"], kernel=kern, device=local,
                       stream=stream.cuda_stream, rows_per_warp=a.rows_per_warp, tile_rows=a.tile_rows,
                       instances=w.get("instances"), **w["params"])
        for i, d in enumerate(w.get("drives", [])):
            lt.set_instance_drive(i, d["body_force"], d["wall_u"])
        lt.set_fields(w["rho"])
        lt.set_observe(a.observe_every)  # 1: every step reduces the observables of the state it collides
        return lt

    esize = 4 if a.precision == "fp32" else 8
    lattice_bytes = 2 * 9 * ns * sites * esize  # both population buffers
    n_rot = 1 if a.l2 in ("flush", "none") else max(1, min(8, -(-ROTATE_BYTES // lattice_bytes)))
    lats = [make_lattice() for _ in range(n_rot)]
    lat = lats[0]
    depth = None
    tune_ms = None
    if a.autotune > 0 and a.kernel == "pull":
        for lt in lats:
            (width, depth), tune_ms = lt.autotune_tiles(a.autotune)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda") if a.l2 == "flush" else None
    flush_src = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda") if a.l2 == "flush" else None

    def l2_flush(k):
        # write a buffer larger than L2, then read another one, so that the step starts with none
        # of its data in L2 and no foreign dirty lines to write back
        flush.fill_(float(k))
        flush_src.sum()

    for k in range(a.warmup):
        for lt in lats:
            if flush is not None:
                l2_flush(k)
            lt.step(1)
    for lt in lats:
        lt.synchronize()

    timing_mode = {"graph": None}

    def graph_events():
        """Timing events that a graph capture records as nodes of the graph, or None where this
        PyTorch has none."""
        try:
            return (torch.cuda.Event(enable_timing=True, external=True),
                    torch.cuda.Event(enable_timing=True, external=True))
        except TypeError:
            return None

    def capture():
        """The step launches of the timed region, captured (untimed) into one CUDA graph that the
        region replays once, so the host's launch rate cannot starve the GPU; None when refused.
        The graph's first and last nodes record timing events: the device time of exactly the K
        steps, without the host's submission of the replay to a stream that the synchronisation
        before the region left idle."""
        ev = graph_events()
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                if ev:
                    ev[0].record(stream)
                for k in range(a.steps):
                    lats[k % n_rot].step(1)
                if ev:
                    ev[1].record(stream)
            timing_mode["graph"] = True
            timing_mode["events"] = ev
            return g
        except Exception as ex:
            timing_mode["graph"] = f"graph capture failed ({type(ex).__name__}); one library call per step"
            timing_mode["events"] = None
            for lt in lats:
                lt.synchronize()
            return None

    def timed(graph=None):
        if flush is not None:
            starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
            ends = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
            for k in range(a.steps):
                l2_flush(k)
                starts[k].record(stream)
                lat.step(1)
                ends[k].record(stream)
            barrier()
            return float(sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)))
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        if graph is not None:
            graph.replay()
        else:
            for k in range(a.steps):
                lats[k % n_rot].step(1)
        t1.record(stream)
        barrier()
        outer = float(t0.elapsed_time(t1))
        ev = timing_mode.get("events") if graph is not None else None
        if ev:
            timing_mode["outer_ms"] = outer
            return float(ev[0].elapsed_time(ev[1]))
        return outer

    def upload(g):
        """The captured graph's launch data uploaded to the device before the timed region
        (cuGraphUpload), so that its one replay does not pay for it; False where that is not
        available (the replay then uploads it)."""
        try:
            import ctypes

            cu = ctypes.CDLL("libcuda.so.1")
            rc = cu.cuGraphUpload(ctypes.c_void_p(g.raw_cuda_graph_exec()), ctypes.c_void_p(stream.cuda_stream))
            torch.cuda.synchronize()
            return rc == 0
        except Exception:
            return False

    launches0 = sum(lt.launches for lt in lats)
    graph = capture() if a.graph and flush is None else None
    uploaded = upload(graph) if graph is not None else False
    barrier()
    with Clocks(local, _pci_bus_id(local)) as clk:
        step_ms = timed(graph)
    launches = sum(lt.launches for lt in lats) - launches0
    # the same steps again with CUDA events around every step-kernel launch (which serialises the
    # launches: no overlap of a launch with the previous kernel's drain): the kernel's duration
    for lt in lats:
        L.lbm_profile(lt.h, True)
    prof_ms = timed()
    kern_ms, kern_n = 0.0, 0
    for lt in lats:
        km, kn = L.lbm_profile_read(lt.h)
        kern_ms, kern_n = kern_ms + km, kern_n + kn
        L.lbm_profile(lt.h, False)
        lt.synchronize()
    # whole job: the slowest rank's time, every rank's sites
    step_s, job_sites = replicas.aggregate(step_ms * 1e-3, sites, dist=dist, device="cuda")
    ms_per_step = step_s * 1e3 / a.steps
    value = job_sites / (ms_per_step * 1e-3) / 1e6

    # roofline of the dominant kernel (the step kernel).  When every step is one launch of it (the
    # pull kernel folds each step's reduction into the next launch), its average launch duration
    # is the timed region over the launches, as the launches overlap (programmatic dependent
    # launch); otherwise the event-bracketed durations of the second pass
    bps = BYTES_PER_SITE[(a.precision, ns)]
    kern_ser_ms = kern_ms / max(kern_n, 1)
    one_launch = launches == a.steps
    kern_avg_ms = step_ms / a.steps if one_launch else kern_ser_ms
    achieved = bps * sites / (kern_avg_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    # the committed records are of the build that observes every step; without observables (or
    # observing every k-th step) another build runs, whose traffic has no record
    traffic = _traffic(kernel_source_hash(a.kernel), a.workload, a.precision,
                       (a.kernel if a.tile_rows in (0, 8) else f"{a.kernel}{a.tile_rows}")
                       + ("" if a.observe_every == 1 else f"/observe_every_{a.observe_every}"))
    if a.precision == "fp64" and ns == 2 and a.observe_every == 1 and a.kernel == "pull":
        tf = FP64_FLOPS_PER_SITE * sites / (kern_avg_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": round(tf, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                    "unit": "TFLOP/s", "frac": round(tf / FP64_PEAK_TFLOPS, 4), "traffic": None,
                    "peak_source": "FP64 pipe: 2 DFMA per SM per cycle (ncu peak), 152 SMs, 2.07 GHz",
                    "flops_per_site": FP64_FLOPS_PER_SITE, "hbm_frac": round(achieved / peak, 4),
                    "fp64_pipe_frac": round(FP64_INSTR_PER_SITE * sites / (kern_avg_ms * 1e-3) /
                                            (FP64_PEAK_TFLOPS / 2 * 1e12), 4),
                    "kernel": "lbm::k_pull<double, 2, M_WRITE|M_OBS>", "kernel_ms": round(kern_avg_ms, 5),
                    "kernel_ms_serialised": round(kern_ser_ms, 5)}
    else:
        roofline = None
    roofline = roofline or {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": peak_kind,
                "kernel": {"pull": "lbm::k_pull<T, 2, M_WRITE|M_OBS>" if a.observe_every else "lbm::k_pull<T, 2, M_WRITE>",
                           "fused": "lbm::k_tile<T, 2, M_WRITE|M_OBS>",
                           "twopass": "lbm::k_density + lbm::k_twopass<T, 2, M_WRITE|M_OBS>",
                           "sweep": "lbm::k_fused<T, 2, M_WRITE|M_OBS>"}[a.kernel],
                "kernel_ms": round(kern_avg_ms, 5),
                "kernel_ms_serialised": round(kern_ser_ms, 5),
                "algorithmic_bytes_per_site": bps,
                "timing": ("average launch duration over the timed region (one step-kernel launch per step, "
                           "CUDA events on the library's stream)" if one_launch else
                           "kernel duration from CUDA events around every launch in a second pass") +
                          f"; kernel_ms_serialised: events around every launch in a second pass over the same "
                          f"{a.steps} steps, which serialises the launches ({prof_ms / a.steps * 1e3:.2f} us per step)"}

    # end to end through the public API with host buffers: upload the fields from pinned host
    # memory, then run the steps in runs of E2E_RUN with every step's observables copied back into
    # pinned host memory (lbm_step_read: one library call per run), each run's records unpacked on
    # the host while the next run executes
    e2e = None
    if a.e2e_steps > 0:
        rho_pin = torch.from_numpy(np.ascontiguousarray(w["rho"])).pin_memory()
        rho_np = rho_pin.numpy()
        series = lat.series(chunk=E2E_RUN, depth=3)
        reader = lat.reader(depth=1)
        barrier()
        t0 = time.perf_counter()
        lat.set_fields(rho_np)
        lat.set_observe(1)
        pending, left = [], a.e2e_steps
        while left > 0:
            n = min(E2E_RUN, left)
            pending.append(series.run(n))  # each record: the step before's sample (its reduction runs in the next launch)
            left -= n
            if len(pending) > 2:  # two runs in flight while the oldest is unpacked
                series.results(pending.pop(0))
        for ticket in pending:
            series.results(ticket)
        reader.result(reader.enqueue(averages=True, reset=True))  # the last step's
        barrier()
        dt, e2e_sites = replicas.aggregate(time.perf_counter() - t0, sites * a.e2e_steps, dist=dist,
                                           device="cuda")
        e2e = {"value": round(e2e_sites / dt / 1e6, 2), "unit": "MLUPS",
               "h2d_bytes_per_step": int(rho_np.nbytes // a.e2e_steps),
               "d2h_bytes_per_step": int(L.load().lbm_observables_bytes(lat.h)), "steps": a.e2e_steps,
               "read": f"every step's observables (time sums of one sample) copied into pinned host memory "
                       f"by lbm_step_read in runs of {E2E_RUN} steps, each run's records unpacked on the "
                       f"host while the next two runs execute"}

    if rank != 0:
        return
    line = {
        "metric": "MLUPS", "value": round(value, 2), "unit": "MLUPS", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if a.precision == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": a.workload, "nx": nx, "nz": nz, "n_species": ns,
                   "precision": a.precision, "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": ((f"{n_rot} lattices of the workload stepped in turn, back to back " if n_rot > 1 else
                           "one lattice ") +
                          f"({n_rot * lattice_bytes / 2**20:.0f} MiB of populations > {L2_BYTES / 2**20:.0f} MiB L2); "
                          "no flush" if flush is None else
                          "one lattice; a 256 MiB write then a 256 MiB read between timed steps"),
                   "observables": ("every step" if a.observe_every == 1 else
                                   "never" if a.observe_every == 0 else f"every {a.observe_every} steps"),
                   "graph_uploaded_before_timing": uploaded,
                   "timed_launches": ("one CUDA graph replay of the captured step launches"
                                      if timing_mode["graph"] is True else timing_mode["graph"] or
                                      "one library call per step"),
                   **({"timed_region": "events recorded by the graph's first and last nodes (the K steps "
                                       "on the device); the events around the replay on the stream: "
                                       f"{timing_mode['outer_ms']:.4f} ms"}
                      if timing_mode.get("outer_ms") is not None else {}),
                   "rows_per_warp": lat.desc.rows_per_warp, "tile_rows": lat.desc.tile_rows, "kernel": a.kernel,
                   **({"instances": len(w["instances"])} if "instances" in w else {}),
                   **({"tile": f"{width}x8", "pipeline_depth": depth,
                       "autotune_ms_per_step": {"32x8 depth 1": round(tune_ms[0], 5), "32x8 depth 2": round(tune_ms[1], 5),
                                                "64x8 depth 1": round(tune_ms[2], 5), "64x8 depth 2": round(tune_ms[3], 5)}}
                      if depth is not None else {})},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if world == 1 and not a.no_cpu_baseline:
        def lib_run(rho_cut, prm, steps):
            lt = L.Lattice(rho_cut.shape[2], rho_cut.shape[1], ns, prec, w["z_boundary"], device=local,
                           stream=stream.cuda_stream, **prm)
            lt.set_fields(rho_cut)
            lt.set_observe(1)
            lt.step(steps)
            g_rho, g_u, _ = lt.fields(populations=False)
            return g_rho, g_u, lt.observables()

        line["cpu_baseline"], errors = cpu_baseline(w, lib_run=lib_run, tol=1e-4 if a.precision == "fp32" else 1e-12)
        line["errors"] = errors
    print(json.dumps(line))


if __name__ == "__main__":
    main()
