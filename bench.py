"""Throughput of the DG elastic-wave hot path on the large workload.

One bench step = one LSRK(5,4) step (five fused stage launches through the C
ABI's dgw_stage, ping-ponging two state buffers; the fifth through
dgw_stage_energy, which also returns the energy of the new state), over the
64^3-element, N=4 curvilinear mesh with the smooth random medium.
Metric: DOF-stage-updates/s = nel * Np * 9 * 5 * steps / time.

Default run: the FP64 path (every operation in FP64) is the headline line;
the mixed path (FP32 volume/flux/lift, FP64 Runge-Kutta registers and
energy) is reported in ``variants.mixed``.  Further sections of the same
line: ``cpu_baseline`` (the oracle on a bounded sample), ``serving``
(continuous batching against one-at-a-time solves), ``adjoint`` (gradient
cost), ``friedrichs`` (transport and shallow-water throughput) and ``ihdg``
(the iHDG-II iteration).  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead.

Multi-GPU (torchrun): the path is replicated, one independent solve per rank
("replicas only": no data-path collective); value = all ranks' updates / the
slowest rank's time.
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")     # the CPU baseline is single-threaded

import argparse
import ctypes
import json
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "DOF-stage-updates/s on 1 GB300 (FP64 vs mixed) + %HBM roofline; served p99 ms"
UNIT = "DOF-stage-updates/s"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_traffic(precision, key=None):
    """DRAM bytes per stage launch from the committed ncu summary (or another of
    its keys), or None when the stage-kernel sources changed since that capture."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1711_01175_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("dgw_stage.cuh", "dgw_internal.cuh", "dgw_stage_fp64.cu", "dgw_stage_mixed.cu", "dgw_stage_mixed_tc.cu"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    path = os.path.join(ROOT, "profiles", "stage_kernel_traffic.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()[:2]
            vals[k] = v
    if vals.get("source_sha256") != h.hexdigest()[:16]:
        return None
    v = vals.get(key or f"{precision}_bytes_per_launch")
    return float(v) if v is not None else None


# FP64 peak: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz (nominal 1.26 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def algorithmic_bytes_per_dof(N, real_bytes, first_stage=False):
    """Minimum HBM traffic of one fused stage per DOF: u in and u out (FP64),
    the register res out and -- except in the first stage, where a_0 = 0 --
    res in (FP64): 32 B (24 B); 10 geometry values per node (Ja, 1/J); 4 face
    values (n, sJ) per node of the three faces an element owns."""
    n = N + 1
    Np = n ** 3
    state = 24.0 if first_stage else 32.0
    return state + 10.0 * real_bytes / 9.0 + 3 * n * n * 4 * real_bytes / (9.0 * Np)


def step_bytes_per_dof(N, real_bytes):
    """Algorithmic bytes of the five stages of one LSRK step, per DOF."""
    return (algorithmic_bytes_per_dof(N, real_bytes, True)
            + 4 * algorithmic_bytes_per_dof(N, real_bytes, False))


def algorithmic_flops_per_element(N):
    """FP64 flops of one fused stage per element as the kernel's arithmetic is
    written.  Volume term per node and direction: N <= 5, for each line node b
    the summed metric D_ab (m_a + m_b) (3 adds, 3 multiplies) and
    A(D_ab (m_a + m_b)) u_b accumulated (18 FMA = 36 flops); N >= 6 (the staged
    form), A(m)u (27), two length-(N+1) contractions of 9 fields (36(N+1)),
    A(m) du (27) and two 9-wide accumulations (18).  Volume scale (10), Q^{-1}
    (14) and the LSRK update (45) per node; per face node the flux difference
    (jump 9, A(m) 27, |A(m)| 42, scaling 27) and its lift (9)."""
    n = N + 1
    Np, nf = n ** 3, n * n
    volume = 3 * (27 + 36 * n + 27 + 18) if N >= 6 else 3 * n * (3 + 3 + 36)
    per_node = volume + 10 + 14 + 45
    per_face_node = 9 + 27 + 42 + 27 + 9
    return Np * per_node + 6 * nf * per_face_node


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) < 9:
                continue
            for nm, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def workload_config(name, E=None):
    if name == "precision":
        return wl.precision_config(E=E or 48)
    return wl.large_config(E=E or 64)


def build_workload(name, E=None):
    cfg = workload_config(name, E)
    N = cfg.N
    from paper_1711_01175_gb300 import reference_nodes
    r, _ = reference_nodes(N)
    data = cfg.build(r)
    return cfg, data


def setup_solver(precision, cfg, data):
    from paper_1711_01175_gb300 import Solver
    m = data["mesh"]
    s = Solver(cfg.N, tau=cfg.tau, precision=precision, cfl=cfg.cfl)
    s.upload_mesh(data["x"], m.etoe, m.etof, m.orient, m.bc)
    s.upload_material(data["rho"], data["lam"], data["mu"])
    return s


def whole_job_rate(local_ms, local_units, device=None):
    """Whole-job throughput of a replicated run: the units every rank processed
    divided by the slowest rank's time (MAX all-reduce of the time, SUM of the
    units; a single process returns its own figures).  Returns (units/s, max ms)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    max_ms = float(t.item())
    return float(u.item()) / (max_ms * 1e-3), max_ms


def energy_reduction_launches(stage_ctas):
    """Kernels of the fused energy's final reduction (one block up to 2048 partials, two levels above)."""
    return 1 if stage_ctas <= 8 * 256 else 2


def fp64_probe(device):
    """The device's measured FP64 FMA rate (dgw_probe_fp64_rate), with the SM
    clocks sampled while it runs."""
    from paper_1711_01175_gb300 import capi
    clk = Clocks(device.index or 0)
    clk.start()
    best = 0.0
    for _ in range(3):
        st, tf = capi.dgw_probe_fp64_rate(device.index or 0)
        capi.check(st)
        best = max(best, tf)
    return {"tflops": best, "clocks": clk.stop()}


def run_variant(precision, cfg, data, steps, warmup, device, stream, clocks=None):
    """Device-resident timing: K steps of 5 stage launches + 1 energy launch pair."""
    import torch
    from paper_1711_01175_gb300 import capi
    s = setup_solver(precision, cfg, data)
    nel, Np = data["mesh"].nel, (cfg.N + 1) ** 3
    dt = s.dt_cfl()
    with torch.cuda.stream(stream):
        ua = torch.from_numpy(data["u0"]).to(device)
        ub = torch.empty_like(ua)
        res = torch.zeros_like(ua)
    h = capi._P(stream.cuda_stream)
    ctx = s._ctx
    lib = capi.load()
    energies = []

    energy = capi._D()

    def one_step(record=None):
        nonlocal ua, ub
        if record is not None:
            record[0].record(stream)
        for st in range(4):
            capi.check(lib.dgw_stage(ctx, ua.data_ptr(), ub.data_ptr(), res.data_ptr(), st, 0.0, dt, h), ctx)
            ua, ub = ub, ua
        # last stage with the energy of the new state fused into the same kernel
        capi.check(lib.dgw_stage_energy(ctx, ua.data_ptr(), ub.data_ptr(), res.data_ptr(), 4, 0.0, dt,
                                        ctypes.byref(energy), h), ctx)
        ua, ub = ub, ua
        if record is not None:
            record[1].record(stream)
        energies.append(energy.value)

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize(device)
    if torch.distributed.is_initialized():
        torch.distributed.barrier()
    torch.cuda.synchronize(device)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    if clocks:
        clocks.start()
    t0.record(stream)
    for k in range(steps):
        one_step(ev[k])
    t1.record(stream)
    torch.cuda.synchronize(device)
    if torch.distributed.is_initialized():
        torch.distributed.barrier()
    torch.cuda.synchronize(device)
    clk = clocks.stop() if clocks else None
    total_ms = t0.elapsed_time(t1)
    stage_ms = sum(a.elapsed_time(b) for a, b in ev) / (5 * steps)
    dof = nel * Np * 9
    out = {
        "total_ms": total_ms, "ms_per_step": total_ms / steps, "stage_ms": stage_ms,
        "dof": dof, "nel": nel, "Np": Np, "energy_first": energies[0], "energy_last": energies[-1],
        "clocks": clk,
    }
    del ua, ub, res
    s.close()
    torch.cuda.empty_cache()
    return out


VARIANT_DTYPE = {"fp64": "f64", "mixed": "f32/f64", "mixed_tc": "f16x2(tensor)/f32/f64",
                 "mixed_tc_bf16": "bf16x2(tensor)/f32/f64"}
VOLUME_FORM = {"mixed": "FP32 CUDA cores",
               "mixed_tc": "D contractions on tensor cores, FP16 hi/lo (per-row 2^k scale), FP32 accumulate",
               "mixed_tc_bf16": "D contractions on tensor cores, BF16 hi/lo, FP32 accumulate"}


def mixed_roofline(prec, N, r, hbm_peak, peak_kind, cfg):
    """HBM roofline of a mixed-path stage kernel: the algorithmic bytes of the
    step's five launches (stage 0 reads no register) over the CUDA-event stage
    time, against the copy bandwidth."""
    nbytes = step_bytes_per_dof(N, 4) * r["dof"] / 5.0      # average per launch
    ach = nbytes / (r["stage_ms"] * 1e-3) / 1e9
    vol = {"mixed": "", "mixed_tc": ",TcFp16", "mixed_tc_bf16": ",TcBf16"}[prec]
    return {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
            "traffic": measured_traffic(prec) if cfg.name == "large-64^3-N4" else None,
            "kernel": f"stage_kernel<{N},float,LSRK{vol}>",
            "note": f"algorithmic bytes {step_bytes_per_dof(N, 4) / 5:.2f} B/DOF per launch "
                    f"(stage 0: {algorithmic_bytes_per_dof(N, 4, True):.2f}, stages 1-4: "
                    f"{algorithmic_bytes_per_dof(N, 4):.2f}); peak {peak_kind} copy bandwidth; volume term: "
                    f"{VOLUME_FORM[prec]}"}


def run_ab_precision(args, device, stream, hbm_peak, peak_kind):
    """A/B of the volume forms on the precision workload (48^3, N=7): FP64,
    mixed with the FP32 CUDA-core volume term, and the two tensor-core forms,
    each timed over the same LSRK steps as the headline (device-resident
    inputs, CUDA events)."""
    cfg, data = build_workload("precision")
    out = {"workload": workload_name(cfg), "dof": data["mesh"].nel * (cfg.N + 1) ** 3 * 9}
    for prec in ("fp64", "mixed", "mixed_tc", "mixed_tc_bf16"):
        k = max(2, args.ab_steps // 4) if prec == "fp64" else args.ab_steps
        r = run_variant(prec, cfg, data, k, args.warmup, device, stream, Clocks(device.index or 0))
        v = {"value": r["dof"] * 5 * k / (r["total_ms"] * 1e-3), "steps": k, "ms_per_step": r["total_ms"] / k,
             "stage_ms": r["stage_ms"], "dtype": VARIANT_DTYPE[prec], "clocks": r["clocks"]}
        if prec == "fp64":
            flops = algorithmic_flops_per_element(cfg.N) * r["nel"]
            v["roofline"] = {"bound": "alu", "achieved": flops / (r["stage_ms"] * 1e-3) / 1e12,
                             "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s"}
            v["roofline"]["frac"] = v["roofline"]["achieved"] / FP64_PEAK_TFLOPS
        else:
            v["roofline"] = mixed_roofline(prec, cfg.N, r, hbm_peak, peak_kind, cfg)
        out[prec] = v
    best = max(("mixed", "mixed_tc", "mixed_tc_bf16"), key=lambda q: out[q]["value"])
    out["fastest_mixed_form"] = best
    return out


def run_precision_recipe(T, device):
    """The precision recipe at full size (48^3, N=7): FP64, the FP32 CUDA-core
    mixed form and the tensor-core FP16 hi/lo mixed form advanced from the
    Gaussian pulse to time T with the same steps (dt = T / ceil(T / dt_cfl));
    the FP64 state is the reference (the parity tests hold it to the oracle at
    1e-12 per stage).  Relative L2 error of each mixed state at T, the energy
    drift |E_mixed(T) - E_fp64(T)| / E(0), and the wall time of each run."""
    import math
    import torch
    cfg, data = build_workload("precision")
    out = {"workload": workload_name(cfg), "T": T}
    states, energies = {}, {}
    for prec in ("fp64", "mixed", "mixed_tc"):
        s = setup_solver(prec, cfg, data)
        if prec == "fp64":
            nsteps = math.ceil(T / s.dt_cfl())
            dt = T / nsteps
            out.update(steps=nsteps, dt=dt)
        u = torch.from_numpy(data["u0"]).to(device)
        res = torch.zeros_like(u)
        e0 = s.energy(u)
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        s.step(u, res, dt, nsteps)
        torch.cuda.synchronize(device)
        wall = time.perf_counter() - t0
        energies[prec] = (e0, s.energy(u))
        states[prec] = u.cpu().numpy()
        out[prec] = {"wall_s": wall, "E_T_over_E0": energies[prec][1] / e0}
        s.close()
        del u, res
        torch.cuda.empty_cache()
    ref = states["fp64"]
    for prec in ("mixed", "mixed_tc"):
        out[prec]["rel_l2_vs_fp64"] = float(np.linalg.norm(states[prec] - ref) / np.linalg.norm(ref))
        out[prec]["energy_drift"] = abs(energies[prec][1] - energies["fp64"][1]) / energies["fp64"][0]
    return out


def run_e2e(precision, cfg, data, steps, warmup, device, stream):
    """Through the public call with a pinned host state: dgw_step_energy(host u,
    res = NULL, 1 step) copies u in, runs the five stages (the last one also
    accumulating the energy), copies u back and returns the energy.  The LSRK
    register stays on the device (the first stage does not read it)."""
    import torch
    s = setup_solver(precision, cfg, data)
    dt = s.dt_cfl()
    u = torch.from_numpy(data["u0"]).pin_memory()
    nbytes = u.numel() * 8
    with torch.cuda.stream(stream):
        for _ in range(max(1, min(warmup, 2))):
            s.step_energy(u, None, dt, 1, stream=stream)
        torch.cuda.synchronize(device)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            s.step_energy(u, None, dt, 1, stream=stream)
        t1.record(stream)
        torch.cuda.synchronize(device)
    ms = t0.elapsed_time(t1)
    s.close()
    return {"ms": ms, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 8}


def cpu_oracle_sample(cfg, data, target_s=12.0, nel_sample=512):
    """The oracle, as it stands, on a bounded sample: LSRK stages of the large
    workload computed for a contiguous block of elements (single thread)."""
    import oracle
    m = data["mesh"]
    r, _ = oracle.gll(cfg.N)
    x = wl.warped_node_coords(m, r, cfg.amplitude)
    op = oracle.ElasticDG(cfg.N, x, m.etoe, m.etof, m.orient, m.bc, data["rho"], data["lam"], data["mu"], cfg.tau)
    dt = oracle.cfl_dt(cfg.cfl, oracle.h_min_corner_edges(x, cfg.N), op.c_max(), cfg.N)
    elems = np.arange(min(nel_sample, m.nel))
    u = data["u0"]
    res = np.zeros_like(u)
    op.lsrk_stage(u, res, 0, dt, elems)          # geometry of the sample (set-up, untimed)
    stages = 0
    t0 = time.perf_counter()
    while True:
        for s_ in range(5):
            op.lsrk_stage(u, res, s_, dt, elems)
            stages += 1
        if time.perf_counter() - t0 > target_s:
            break
    el = time.perf_counter() - t0
    Np = (cfg.N + 1) ** 3
    return {"value": len(elems) * Np * 9 * stages / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{stages} LSRK stages on {len(elems)} of {m.nel} elements of {cfg.name} "
                      f"(numpy FP64, 1 thread), {el:.1f} s"}


def _oracle_worker(args):
    """One process of the all-cores oracle leg: attach the shared workload
    arrays, build the oracle and time LSRK stages on its own block of elements
    (the loops of all workers start at one barrier)."""
    name, E, paths, mesh_arrays, mat, elems, target_s, barrier = args
    import oracle
    cfg = workload_config(name, E)
    x, u = (np.load(p, mmap_mode="r") for p in paths)
    etoe, etof, orient, bc = mesh_arrays
    op = oracle.ElasticDG(cfg.N, x, etoe, etof, orient, bc, *mat, cfg.tau)
    dt = oracle.cfl_dt(cfg.cfl, oracle.h_min_corner_edges(x, cfg.N), op.c_max(), cfg.N)
    res = np.zeros_like(u)                   # pages stay untouched outside the block
    op.lsrk_stage(u, res, 0, dt, elems)      # geometry of the block (set-up, untimed)
    barrier.wait()
    stages = 0
    t0 = time.perf_counter()
    while True:
        for s_ in range(5):
            op.lsrk_stage(u, res, s_, dt, elems)
            stages += 1
        if time.perf_counter() - t0 > target_s:
            break
    el = time.perf_counter() - t0
    return stages, len(elems), el


def cpu_oracle_all_cores(cfg, data, target_s=12.0, nel_block=256):
    """The oracle, as it stands, on every host core: one spawned process per core,
    each timing LSRK stages on its own block of elements of the same workload
    (node coordinates and state memory-mapped from one file each, not copied).
    Throughput = the sum of the processes' rates over their common timed
    interval."""
    import multiprocessing as mp
    import shutil
    import oracle
    cores = os.cpu_count() or 1
    m = data["mesh"]
    r, _ = oracle.gll(cfg.N)
    x = wl.warped_node_coords(m, r, cfg.amplitude)
    tmp = tempfile.mkdtemp(prefix="dgw_oracle_")
    try:
        paths = []
        for nm, a in (("x", x), ("u0", data["u0"])):
            paths.append(os.path.join(tmp, nm + ".npy"))
            np.save(paths[-1], a)
        del x
        ctx = mp.get_context("spawn")
        with ctx.Manager() as mgr:
            barrier = mgr.Barrier(cores)
            jobs = [(cfg.name.split("-")[0], cfg.E, paths, (m.etoe, m.etof, m.orient, m.bc),
                     (data["rho"], data["lam"], data["mu"]),
                     np.arange(k * nel_block, (k + 1) * nel_block) % m.nel, target_s, barrier) for k in range(cores)]
            with ctx.Pool(cores) as pool:
                outs = pool.map(_oracle_worker, jobs)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    Np = (cfg.N + 1) ** 3
    value = sum(st * ne * Np * 9 / el for st, ne, el in outs)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes x {nel_block} elements of {m.nel} ({cfg.name}), "
                      f"{min(o[0] for o in outs)}-{max(o[0] for o in outs)} LSRK stages each in "
                      f"{max(o[2] for o in outs):.1f} s (numpy FP64, 1 thread per process)",
            "cpu_model": _cpu_model()}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    key, val = line.split(":", 1)
                    return val.strip() if key.lower().startswith("model") else f"{key.strip()} {val.strip()}"
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def workload_name(cfg):
    """The workload as both arms name it in config.workload."""
    return (cfg.name + f" ({cfg.E}^3 hex, N={cfg.N}, warp {cfg.amplitude}, smooth random medium, free surface top, "
            "absorbing bottom, x/y periodic)")


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg, data = build_workload_oracle(args.workload, args.elements)
    N = cfg.N
    per_step = []
    total_units = 0
    import oracle
    m = data["mesh"]
    r, _ = oracle.gll(N)
    x = wl.warped_node_coords(m, r, cfg.amplitude)
    op = oracle.ElasticDG(N, x, m.etoe, m.etof, m.orient, m.bc, data["rho"], data["lam"], data["mu"], cfg.tau)
    dt = oracle.cfl_dt(cfg.cfl, oracle.h_min_corner_edges(x, N), op.c_max(), N)
    elems = np.arange(args.ref_sample)
    u, res = data["u0"], np.zeros_like(data["u0"])
    Np = (N + 1) ** 3
    op.lsrk_stage(u, res, 0, dt, elems)          # geometry of the sample (set-up, untimed)
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for s_ in range(5):
            op.lsrk_stage(u, res, s_, dt, elems)
        el = time.perf_counter() - t0
        if k >= args.warmup:
            per_step.append(el)
            total_units += len(elems) * Np * 9 * 5
    tt = sum(per_step)
    value = total_units / tt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(cfg), "precision": "fp64", "elements": m.nel,
                       "dof": m.nel * Np * 9, "sample_elements": len(elems),
                       "parallelism": "rank 0 only (the oracle on host cores)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"one LSRK step (5 stages) per bench step on {len(elems)} of "
                                       f"{m.nel} elements (numpy FP64, 1 thread)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Served latency: one seeded request stream through continuous batching and
    through one-at-a-time plain solves (mixed path), at each arrival rate of
    --serve-rates (Poisson arrivals; the same requests at every rate, arrival
    times scaled).  Request payloads (mesh, medium, point force) are prepared
    before the clock starts, as a client would send them.  The device's
    capacity for the stream is estimated from the one-at-a-time run at the
    highest rate (busy the whole time): rates below it measure batching
    latency, rates above it measure queueing."""
    from paper_1711_01175_gb300 import serving, reference_nodes
    rates = [float(v) for v in str(args.serve_rates).split(",") if v.strip()]
    base = wl.make_requests(args.serve_requests, seed=7, rate=1.0, E_range=(8, args.serve_max_E), N_choices=(3, 4, 5),
                            steps_range=(args.serve_min_steps, args.serve_max_steps))
    t_build = time.perf_counter()
    for r in base:
        r.payload = r.build(reference_nodes(r.N)[0])
    t_build = time.perf_counter() - t_build
    warm = wl.make_requests(3, seed=8, rate=1000.0, E_range=(2, 3), N_choices=(3, 4, 5), steps_range=(2, 4))
    for r in warm:
        r.payload = r.build(reference_nodes(r.N)[0])
    serving.continuous_batching(warm, precision="mixed")
    serving.one_at_a_time(warm, precision="mixed")
    dof_stages = sum(r.E ** 3 * (r.N + 1) ** 3 * 9 * 5 * r.steps for r in base)
    sweep = []
    for rate in rates:
        arrivals = [r.arrival for r in base]
        for r, a in zip(base, arrivals):
            r.arrival = a / rate
        res_b, wall_b = serving.continuous_batching(base, precision="mixed", memory_budget=args.serve_memory_gb * 1e9)
        res_s, wall_s = serving.one_at_a_time(base, precision="mixed")
        for r, a in zip(base, arrivals):
            r.arrival = a
        b, s1 = serving.summarize(res_b, wall_b), serving.summarize(res_s, wall_s)
        b["dof_stage_updates_per_s"] = dof_stages / wall_b
        s1["dof_stage_updates_per_s"] = dof_stages / wall_s
        sweep.append({"rate_per_s": rate, "continuous_batching": b, "one_at_a_time": s1})
    busiest = max(sweep, key=lambda x: x["rate_per_s"])
    capacity = busiest["one_at_a_time"]["solves_per_s"]
    for x in sweep:
        x["load_vs_one_at_a_time_capacity"] = x["rate_per_s"] / capacity
    below = [x for x in sweep if x["rate_per_s"] < capacity]
    head = min(below, key=lambda x: x["rate_per_s"]) if below else min(sweep, key=lambda x: x["rate_per_s"])
    return {"requests": len(base), "mesh_E": [8, args.serve_max_E], "N": [3, 4, 5],
            "steps": [args.serve_min_steps, args.serve_max_steps], "precision": "mixed",
            "memory_budget_gb": args.serve_memory_gb, "payload_build_s": t_build,
            "one_at_a_time_capacity_solves_per_s": capacity, "rates": sweep,
            "p99_ms": head["continuous_batching"]["p99_ms"], "p50_ms": head["continuous_batching"]["p50_ms"],
            "headline_rate_per_s": head["rate_per_s"]}


def run_adjoint(args):
    """Gradient of a receiver misfit w.r.t. the per-element medium by the
    hand-written adjoint (FP64): forward with checkpoints, then the backward
    sweep; reports the time of each and their ratio.  The experiment: a Ricker
    point force at the centre element (peak frequency 3 / window, centred at
    1.2 / f0 so that it starts from rest), receivers at random points of the
    elements within two faces of the source element (what the window's waves
    reach at CFL 0.5), data recorded in the same experiment with the medium
    perturbed by 5 % seeded noise (untimed), L2 misfit.  Defaults: the adjoint
    recipe (32^3, N=4, 500 steps, 32 receivers, checkpoints every 50)."""
    import torch
    from paper_1711_01175_gb300 import Solver, reference_nodes
    from paper_1711_01175_gb300.adjoint import receiver_traces
    E, N, nsteps, nrec, every = args.adj_E, 4, args.adj_steps, args.adj_receivers, args.adj_checkpoint
    mesh = wl.structured_hex_mesh(E, (True, True, False), {4: wl.BC_ABSORBING, 5: wl.BC_FREE_SURFACE}, "morton")
    r, _ = reference_nodes(N)
    x = wl.warped_node_coords(mesh, r, 0.1)
    rho, lam, mu = wl.smooth_random_material(mesh, 5)
    s = Solver(N)
    s.upload_mesh(x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
    s.upload_material(rho, lam, mu)
    dt = s.dt_cfl()
    centre = int(np.nonzero(np.all(mesh.cell == E // 2, axis=1))[0][0])
    f0 = 3.0 / (nsteps * dt)
    s.set_point_force(centre, [0.1, -0.2, 0.3], [0.0, 0.0, 1.0], f0, 1.2 / f0)
    rng = np.random.default_rng(9)
    near = [centre] + [int(e) for e in mesh.etoe[centre] if e >= 0]
    around = np.unique(np.concatenate([mesh.etoe[e] for e in near]))
    around = around[around >= 0]              # within two faces of the source
    s.set_receivers(rng.choice(around, nrec), rng.uniform(-0.9, 0.9, (nrec, 3)))
    u0 = torch.zeros((9, mesh.nel, (N + 1) ** 3), dtype=torch.float64, device="cuda")
    base = np.stack([rho, lam, mu])
    perturbed = base * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, base.shape))
    with torch.no_grad():
        data = receiver_traces(torch.tensor(perturbed), s, u0, dt, nsteps, checkpoint_every=nsteps).clone()
    m = torch.tensor(base, requires_grad=True)
    # warm-up: two steps forward and back (first launches, workspace allocation)
    w = receiver_traces(m, s, u0, dt, 2, checkpoint_every=every)
    torch.sum(w * w).backward()
    m.grad = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tr = receiver_traces(m, s, u0, dt, nsteps, checkpoint_every=every)
    J = 0.5 * dt * torch.sum((tr - data) ** 2)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    J.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    g = m.grad.numpy()
    s.close()
    g2 = g * g
    return {"mesh": f"{E}^3", "N": N, "steps": nsteps, "receivers": nrec, "checkpoint_every": every,
            "dt": dt, "source_f0": f0, "data": "same experiment, medium x (1 + 0.05 U(-1, 1)), seeded",
            "forward_s": t1 - t0, "backward_s": t2 - t1, "backward_over_forward": (t2 - t1) / (t1 - t0),
            "misfit": float(J.detach()), "trace_rms": float(torch.sqrt(torch.mean(tr.detach() ** 2))),
            "gradient_norm": float(np.linalg.norm(g)),
            "gradient_share_source_and_neighbours": float(g2[:, near].sum() / g2.sum()),
            "gradient_share_within_two_faces": float(g2[:, around].sum() / g2.sum()),
            "adjoint_scratch": ("stage inputs only, operator recomputed in the gradient terms (3 + 5 K states)"
                                if os.environ.get("DGW_ADJOINT_LOW_MEMORY") == "1" else
                                "stage inputs and stage operator outputs (3 + 10 K states, K = checkpoint interval)"),
            "precision": "fp64"}


def friedrichs_flops_per_node(system, N):
    """FP64 flops of one stage per node as the generic kernel's arithmetic is
    written (n = N + 1; 6 n^2 / n^3 face items per node):
    transport   volume 3 (A(m)u 6 + two length-n contractions accumulated 4n +
                A(m) du 6 + 1), face item 18, RK update, lift and fused energy 9;
    shallow water  volume 3 (5 + 12n + 5 + 3), face item 25, update 22."""
    n = N + 1
    per_face = 6.0 * n * n / n ** 3
    if system == "transport":
        return 3 * (13 + 4 * n) + per_face * 18 + 9
    return 3 * (13 + 12 * n) + per_face * 25 + 22


def run_friedrichs(args, hbm_peak, peak_kind):
    """The generic Friedrichs systems (FP64): transport (beta = (0.2, 0.2, 0.2),
    the velocity of the paper's 3-D transport test) on the 64^3, N=4 warped
    periodic mesh, and the shallow-water standing wave with walls on a
    512 x 512 x 1, N=4 mesh.  K steps of dgw_step timed with CUDA events
    (inputs larger than L2); algorithmic bytes per DOF and stage: the FP64 state
    (u and res in and out, 32 B; 24 B in stage 0) plus 10 FP64 geometry values
    per node shared by the m fields."""
    import torch
    from paper_1711_01175_gb300 import Solver, reference_nodes
    N = 4
    r, _ = reference_nodes(N)
    out = {}
    cases = [("transport", wl.structured_hex_mesh(args.fr_E, order="morton"), 0.1),
             ("shallow_water", wl.structured_hex_mesh((8 * args.fr_E, 8 * args.fr_E, 1), (False, False, True),
                                                     {0: wl.BC_WALL, 1: wl.BC_WALL, 2: wl.BC_WALL, 3: wl.BC_WALL},
                                                     order="morton"), 0.0)]
    stream = torch.cuda.Stream()
    for system, mesh, amp in cases:
        x = wl.warped_node_coords(mesh, r, amp)
        s = Solver(N, system=system, beta=(0.2, 0.2, 0.2))
        s.upload_mesh(x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
        u0 = wl.transport_periodic(x, (0.2, 0.2, 0.2)) if system == "transport" else wl.shallow_water_standing_wave(x)
        m = u0.shape[0]
        dt = s.dt_cfl()
        with torch.cuda.stream(stream):
            u = torch.from_numpy(u0).cuda()
            res = torch.zeros_like(u)
            s.step(u, res, dt, args.warmup, stream=stream)
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            s.step(u, res, dt, args.fr_steps, stream=stream)
            t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        e = s.energy(u)
        nodes = mesh.nel * (N + 1) ** 3
        dof_stages = nodes * m * 5 * args.fr_steps
        bytes_step = nodes * (m * (24 + 4 * 32) + 5 * 80)
        gbs = bytes_step * args.fr_steps / (ms * 1e-3) / 1e9
        tf = friedrichs_flops_per_node(system, N) * nodes * 5 * args.fr_steps / (ms * 1e-3) / 1e12
        out[system] = {"mesh": "x".join(str(v) for v in mesh.E), "N": N, "m": m, "dof": nodes * m,
                       "steps": args.fr_steps, "ms_per_step": ms / args.fr_steps,
                       "value": dof_stages / (ms * 1e-3), "unit": UNIT, "dtype": "f64",
                       "roofline": {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                    "frac": tf / FP64_PEAK_TFLOPS,
                                    "note": f"FP64 flops as written ({friedrichs_flops_per_node(system, N):.0f} per "
                                            f"node and stage) / CUDA-event time; HBM: {gbs:.0f} GB/s = "
                                            f"{gbs / hbm_peak:.3f} of {peak_kind} copy bandwidth at "
                                            f"{bytes_step / (5 * nodes * m):.1f} algorithmic B/DOF per stage"},
                       "energy_end": e}
        s.close()
        del u, res
    return out


def run_ihdg(args):
    """iHDG-II for transport (the paper's Section 3 and Section 6.1):
    * steady: beta = (1, 0.7, 0.4) on the undeformed E^3 mesh (E = 16, the
      largest 3-D case of the paper's iteration table), N = 4, manufactured
      u^e = prod sin(pi x_i); set-up time, iterations to the 1e-10 criterion,
      solve time, time per iteration (two launches and the stopping test's host
      round trip) and the iteration kernel's FP64 rate (2 Np^2 flops per element
      for the local inverse);
    * locally implicit: implicit Euler steps of the periodic transport test
      (beta = (0.2, 0.2, 0.2)) at CFL 1, 2 and 5: iterations per step."""
    import torch
    from paper_1711_01175_gb300 import Solver, reference_nodes
    N, E = 4, args.ihdg_E
    r, _ = reference_nodes(N)
    mesh = wl.structured_hex_mesh(E, (False, False, False), order="morton")
    x = wl.warped_node_coords(mesh, r, 0.0)
    beta = np.array([1.0, 0.7, 0.4])
    X = np.pi * x
    sn, cs = np.sin(X), np.cos(X)
    ue = np.prod(sn, axis=-1)[None]
    grad = np.pi * np.stack([cs[..., 0] * sn[..., 1] * sn[..., 2], sn[..., 0] * cs[..., 1] * sn[..., 2],
                             sn[..., 0] * sn[..., 1] * cs[..., 2]], axis=-1)
    f = torch.from_numpy((grad @ beta)[None]).cuda()
    s = Solver(N, system="transport", beta=beta)
    s.upload_mesh(x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.ihdg_setup(0.0)
    setup_s = time.perf_counter() - t0
    u = torch.zeros_like(f)
    s.ihdg_solve(u, f=f, tol=0.0, max_iter=2)            # warm-up
    u.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its, change = s.ihdg_solve(u, f=f, tol=1e-10, max_iter=20 * E)
    solve_s = time.perf_counter() - t0
    err = float(np.linalg.norm(u.cpu().numpy() - ue) / np.linalg.norm(ue))
    Np = (N + 1) ** 3
    flops = 2.0 * Np * Np * mesh.nel * its
    table = {}
    with open(os.path.join(ROOT, "tests", "golden", "ihdg_transport_iterations.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                e_, p_, k_ = (int(v) for v in line.split())
                table[(e_, p_)] = k_
    table_sw = {}
    with open(os.path.join(ROOT, "tests", "golden", "ihdg_shallow_water_iterations.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                n_, p_, a_, b_ = (int(v) for v in line.split())
                table_sw[(n_, p_)] = (a_, b_)
    steady = {"mesh": f"{E}^3", "N": N, "iterations": its, "element_layers_plus_one": 3 * E - 1,
              "paper_table_iterations": table.get((E, N)),
              "last_change": change, "setup_s": setup_s, "solve_ms": solve_s * 1e3,
              "ms_per_iteration": solve_s * 1e3 / its, "rel_l2_error_vs_exact": err,
              "matvec_fp64_tflops": flops / solve_s / 1e12,
              "matvec_frac_of_fp64_peak": flops / solve_s / 1e12 / FP64_PEAK_TFLOPS,
              "inverse_bytes": Np * Np * 8 * mesh.nel}
    s.close()
    del u, f
    # locally implicit Euler steps
    Ei = args.ihdg_implicit_E
    mesh = wl.structured_hex_mesh(Ei, order="morton")
    x = wl.warped_node_coords(mesh, r, 0.05)
    b2 = (0.2, 0.2, 0.2)
    implicit = []
    for cfl in (1.0, 2.0, 5.0):
        s = Solver(N, system="transport", beta=b2, cfl=cfl)
        s.upload_mesh(x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
        dt = s.dt_cfl()
        s.ihdg_setup(1.0 / dt)
        um = torch.from_numpy(wl.transport_periodic(x, b2)).cuda()
        u = um.clone()
        counts = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.ihdg_steps):
            k, _ = s.ihdg_solve(u, u_prev=um, tol=1e-10, max_iter=500)
            counts.append(k)
            um.copy_(u)
        wall = time.perf_counter() - t0
        implicit.append({"cfl": cfl, "dt": dt, "steps": args.ihdg_steps, "iterations_per_step": counts,
                         "ms_per_step": wall * 1e3 / args.ihdg_steps})
        s.close()
    # shallow water, Crank-Nicolson (the paper's Section 6.2 table: 32 x 32 elements, p = 2)
    Ns, Es = 2, 32
    rs, _ = reference_nodes(Ns)
    mesh = wl.structured_hex_mesh((Es, Es, 1), (False, False, True),
                                  {0: wl.BC_WALL, 1: wl.BC_WALL, 2: wl.BC_WALL, 3: wl.BC_WALL})
    x = wl.warped_node_coords(mesh, rs, 0.0)
    sw = Solver(Ns, system="shallow_water")
    sw.upload_mesh(x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
    um = torch.from_numpy(wl.shallow_water_standing_wave(x)).cuda()
    fl = torch.empty_like(um)
    sw.rhs(um, fl)
    cn = []
    for dt in (0.1, 0.01):
        sw.ihdg_setup(2.0 / dt)
        u = um.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k, ch = sw.ihdg_solve(u, u_prev=um, f=fl, tol=1e-10, max_iter=1000)
        cn.append({"dt": dt, "iterations": k, "paper_table_iterations": table_sw.get((Es * Es, Ns), (None, None))[
            0 if dt == 0.1 else 1], "solve_ms": (time.perf_counter() - t0) * 1e3})
    sw.close()
    elastic = run_ihdg_elastic(args) if args.ihdg_elastic_E > 0 else None
    return {"steady": steady, "locally_implicit": {"mesh": f"{Ei}^3", "N": N, "beta": list(b2), "runs": implicit},
            "shallow_water_crank_nicolson": {"mesh": f"{Es}x{Es}", "N": Ns, "first_step": cn},
            "elastic_locally_implicit": elastic, "precision": "fp64"}


def run_ihdg_elastic(args):
    """iHDG-II on the elastic system: implicit Euler steps of the large
    workload's recipe (heterogeneous medium, warped mesh, free surface and
    absorbing faces, Gaussian stress pulse) at E^3 elements and N = 2, FP64 and
    upwind, at CFL 1, 2 and 5: set-up time, iterations per step (1e-10
    criterion), time per step, and the HBM rate of the local solves (the
    inverses, nel (9 Np)^2 doubles, are read once per iteration)."""
    import torch
    from paper_1711_01175_gb300 import Solver, reference_nodes
    N, E = 2, args.ihdg_elastic_E
    w = wl.large_config(E=E, N=N).build(reference_nodes(N)[0])
    mesh = w["mesh"]
    nb = 9 * (N + 1) ** 3
    inv_bytes = float(nb) * nb * 8 * mesh.nel
    runs = []
    for cfl in (1.0, 2.0, 5.0):
        s = Solver(N, cfl=cfl)
        s.upload_mesh(w["x"], mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
        s.upload_material(w["rho"], w["lam"], w["mu"])
        dt = s.dt_cfl()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.ihdg_setup(1.0 / dt)
        setup_s = time.perf_counter() - t0
        um = torch.from_numpy(w["u0"]).cuda()
        u = um.clone()
        s.ihdg_solve(u, u_prev=um, tol=0.0, max_iter=2)          # warm-up
        u.copy_(um)
        counts = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.ihdg_steps):
            k, _ = s.ihdg_solve(u, u_prev=um, tol=1e-10, max_iter=1000)
            counts.append(k)
            um.copy_(u)
        wall = time.perf_counter() - t0
        its = sum(counts)
        runs.append({"cfl": cfl, "dt": dt, "setup_s": setup_s, "steps": args.ihdg_steps,
                     "iterations_per_step": counts, "ms_per_step": wall * 1e3 / args.ihdg_steps,
                     "ms_per_iteration": wall * 1e3 / its,
                     "local_solve_hbm_gbs": inv_bytes * its / wall / 1e9})
        s.close()
        del u, um
    return {"mesh": f"{E}^3", "N": N, "workload": "large recipe (seed 1 medium, warp 0.1, Gaussian pulse)",
            "block_rows": nb, "inverse_bytes": inv_bytes, "runs": runs}


def build_workload_oracle(name, E=None):
    import oracle
    cfg = workload_config(name, E)
    r, _ = oracle.gll(cfg.N)
    return cfg, cfg.build(r)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="all", choices=["all", "both", "fp64", "mixed", "mixed_tc", "mixed_tc_bf16"],
                    help="all: FP64 headline plus the mixed CUDA-core and tensor-core variants; both: FP64 and mixed")
    ap.add_argument("--workload", default="large", choices=["large", "precision"],
                    help="large: 64^3, N=4 (the metric's workload); precision: 48^3, N=7")
    ap.add_argument("--elements", type=int, default=None, help="elements per axis (default: the workload's)")
    ap.add_argument("--mixed-steps", type=int, default=None, help="steps for the mixed variants (default 4x)")
    ap.add_argument("--no-ab", action="store_true",
                    help="skip the A/B of the volume forms on the 48^3, N=7 precision workload")
    ap.add_argument("--ab-steps", type=int, default=8, help="steps per variant of that A/B")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=256, help="elements per reference-arm step")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-friedrichs", action="store_true", help="skip the transport / shallow-water section")
    ap.add_argument("--no-ihdg", action="store_true", help="skip the iHDG-II section")
    ap.add_argument("--ihdg-E", type=int, default=16)
    ap.add_argument("--ihdg-implicit-E", type=int, default=16)
    ap.add_argument("--ihdg-steps", type=int, default=5)
    ap.add_argument("--fr-E", type=int, default=64, help="transport mesh edge (shallow water: 8x this, one layer)")
    ap.add_argument("--ihdg-elastic-E", type=int, default=16,
                    help="elastic iHDG-II mesh edge (N = 2; 0 skips the elastic part)")
    ap.add_argument("--fr-steps", type=int, default=20)
    ap.add_argument("--adj-E", type=int, default=32, help="adjoint mesh edge (the recipe: 32)")
    ap.add_argument("--adj-steps", type=int, default=500, help="(the recipe: 500)")
    ap.add_argument("--adj-receivers", type=int, default=32, help="(the recipe: 32)")
    ap.add_argument("--adj-checkpoint", type=int, default=50, help="(the recipe: 50)")
    ap.add_argument("--serve-requests", type=int, default=160,
                    help="requests of the served-latency run (the full recipe: 2000)")
    ap.add_argument("--serve-rates", default="20,40,80",
                    help="Poisson arrival rates per second, comma separated (the full recipe: about 0.7 solves/s of capacity)")
    ap.add_argument("--serve-recipe", action="store_true",
                    help="the serving recipe's distributions: meshes 8^3..48^3, 200-2000 steps (with --serve-requests, "
                         "--serve-rates)")
    ap.add_argument("--serving-only", action="store_true", help="print a line with the serving section only")
    ap.add_argument("--precision-recipe-T", type=float, default=None,
                    help="print a line with the precision recipe (48^3, N=7) advanced to this time only")
    ap.add_argument("--serve-max-E", type=int, default=20, help="largest mesh edge (the full recipe: 48)")
    ap.add_argument("--serve-min-steps", type=int, default=40, help="(the full recipe: 200)")
    ap.add_argument("--serve-max-steps", type=int, default=120, help="(the full recipe: 2000)")
    ap.add_argument("--serve-memory-gb", type=float, default=40.0, help="device memory the server may hold")
    args = ap.parse_args()
    if args.serve_recipe:
        args.serve_max_E, args.serve_min_steps, args.serve_max_steps = 48, 200, 2000
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    stream = torch.cuda.Stream(device)

    import __graft_entry__ as g
    if rank == 0:
        g.build()
    if world > 1:
        torch.distributed.barrier()
    g.build()

    if args.precision_recipe_T is not None:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "unit": UNIT, "data": "synthetic (seeded medium, Gaussian pulse)",
                              "precision_recipe": run_precision_recipe(args.precision_recipe_T, device)}), flush=True)
        return
    if args.serving_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "unit": UNIT, "data": "synthetic (seeded request stream)",
                              "serving": run_serving(args)}), flush=True)
        return
    cfg, data = build_workload(args.workload, args.elements)
    hbm_peak, peak_kind = peaks()
    variants = {"all": ["fp64", "mixed", "mixed_tc", "mixed_tc_bf16"], "both": ["fp64", "mixed"]}.get(
        args.precision, [args.precision])
    results = {}
    for prec in variants:
        k = args.steps if prec == "fp64" else (args.mixed_steps or 4 * args.steps)
        clk = Clocks(local)
        r = run_variant(prec, cfg, data, k, args.warmup, device, stream, clk)
        r["steps"] = k
        r["value"], r["max_ms"] = whole_job_rate(r["total_ms"], r["dof"] * 5 * k, device)
        if not args.no_e2e and prec != "mixed_tc_bf16":
            e = run_e2e(prec, cfg, data, max(2, k // 4), args.warmup, device, stream)
            r["e2e"] = {"value": r["dof"] * 5 * max(2, k // 4) / (e["ms"] * 1e-3) * world, "unit": UNIT,
                        "h2d_bytes_per_step": e["h2d_bytes_per_step"],
                        "d2h_bytes_per_step": e["d2h_bytes_per_step"]}
        # five stage launches + the final reduction of the fused energy's per-CTA partials
        epb = {1: 16, 2: 9, 3: 4}.get(cfg.N, 1)
        launches_per_step = 5 + energy_reduction_launches((r["nel"] + epb - 1) // epb)
        r["gpu_launches"] = launches_per_step * k
        N = cfg.N
        if prec == "fp64":
            flops = algorithmic_flops_per_element(N) * r["nel"]
            ach = flops / (r["stage_ms"] * 1e-3) / 1e12
            probe = fp64_probe(device)
            busy = measured_traffic("fp64", "fp64_pipe_busy_pct") if cfg.name == "large-64^3-N4" else None
            r["roofline"] = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": ach / FP64_PEAK_TFLOPS,
                             "traffic": measured_traffic("fp64") if cfg.name == "large-64^3-N4" else None,
                             "kernel": f"stage_kernel<{N},double,LSRK>",
                             "peak_measured": probe["tflops"], "frac_of_measured": ach / probe["tflops"],
                             "fp64_pipe_busy_ncu": None if busy is None else busy / 100.0,
                             "note": "FP64 flops as written per launch / CUDA-event stage time; peak derived "
                                     "from 152 SMs x 2 DFMA/clk x 2.07 GHz (nominal); peak_measured: "
                                     "dgw_probe_fp64_rate (independent DFMA chains on every SM) in this run, "
                                     f"SM clock median {probe['clocks']['sm_mhz']} MHz during the probe; "
                                     "fp64_pipe_busy_ncu: sm__pipe_fp64_cycles_active of the committed ncu capture "
                                     "(the figure of merit of a kernel bound by its FP64 pipe)"}
        else:
            r["roofline"] = mixed_roofline(prec, N, r, hbm_peak, peak_kind, cfg)
        results[prec] = r

    if rank != 0:
        torch.distributed.destroy_process_group() if world > 1 else None
        return
    head_prec = "fp64" if "fp64" in results else next(iter(results))
    head = results[head_prec]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": head["steps"],
        "warmup": args.warmup, "ms_per_step": head["max_ms"] / head["steps"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": VARIANT_DTYPE[head_prec],
        "data": "synthetic (seeded mesh, medium and Gaussian pulse of the large workload)",
        "config": {"workload": workload_name(cfg), "precision": head_prec, "elements": head["nel"],
                   "dof": head["dof"], "step": "one LSRK(5,4) step: 5 fused stage launches, the last one also accumulating the energy of the new state",
                   "l2": f"inputs larger than L2 (state {head['dof'] * 8 / 1e9:.2f} GB per buffer)",
                   "parallelism": f"replicas x{world}"},
        "roofline": head["roofline"],
        "clocks": head["clocks"],
        "gpu_launches": head["gpu_launches"],
    }
    if "e2e" in head:
        line["e2e"] = head["e2e"]
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample(cfg, data)
        line["cpu_baseline"]["cpu_model"] = _cpu_model()
        line["cpu_baseline_all_cores"] = cpu_oracle_all_cores(cfg, data)
    if world == 1 and not args.no_serving:
        line["serving"] = run_serving(args)
    if world == 1 and not args.no_adjoint:
        line["adjoint"] = run_adjoint(args)
    if world == 1 and not args.no_friedrichs:
        hbm_peak_f, peak_kind_f = peaks()
        line["friedrichs"] = run_friedrichs(args, hbm_peak_f, peak_kind_f)
    if world == 1 and not args.no_ihdg:
        line["ihdg"] = run_ihdg(args)
    if len(results) > 1:
        line["variants"] = {}
        for prec, m in results.items():
            if prec == head_prec:
                continue
            line["variants"][prec] = {"value": m["value"], "dtype": VARIANT_DTYPE[prec], "steps": m["steps"],
                                      "ms_per_step": m["max_ms"] / m["steps"], "roofline": m["roofline"],
                                      "clocks": m["clocks"], "e2e": m.get("e2e"),
                                      "gpu_launches": m["gpu_launches"]}
    if world == 1 and not args.no_ab and args.workload == "large" and args.precision == "all":
        line["ab_precision_workload"] = run_ab_precision(args, device, stream, hbm_peak, peak_kind)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
