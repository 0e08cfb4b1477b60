"""Benchmark of the ternary ELBM step on GB300.

Headline workload: the D3Q27 192x192x128 lubricated substrate (a liquid-1
drop above a liquid-2 film on a wall, force wetting), 4.72 M nodes, 2.1 GB of
populations: the largest single-GPU configuration, far larger than L2.  One
benchmark step = one full time step of the lattice (moments pass, ghost
layer, stencils, force, ELBM + LBGK collision, streaming with bounce-back),
timed with CUDA events on the lattice's stream.  The D2Q9 1024x64 capillary
channel (9.4 MB, L2-resident) is reported as a sub-key, timed with a 256 MB
buffer written before every step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs one replica (weak scaling, no collective on
the data path); rank 0 prints one JSON line with the max time over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
L2_FLUSH_BYTES = 256 << 20


def kernel_source_hash():
    """sha256 over the device-code sources (csrc/*.cuh, *.h and the per-lattice
    kernel units; not the host-side tlb_api.cu), in name order."""
    import glob
    import hashlib

    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_1904_06881_gb300", "csrc", "*"))):
        if f.endswith((".cu", ".cuh", ".h")) and os.path.basename(f) != "tlb_api.cu":
            h.update(os.path.basename(f).encode())
            with open(f, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


def _counters():
    """The committed ncu counters of the step kernels (profiles/traffic.json),
    or {} when the kernel sources changed since they were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
    except Exception:
        return {}
    return t if t.get("source_sha256") == kernel_source_hash() else {}


def measured_traffic(workload_name):
    """DRAM bytes per launch of the step kernel from the committed ncu capture,
    or None when the kernel sources changed since it was taken."""
    return _counters().get("traffic_bytes_per_launch", {}).get(workload_name)


def measured_instructions(workload_name):
    """Warp instructions executed per launch of the step kernel (ncu
    smsp__inst_executed.sum), or None as for the traffic."""
    return _counters().get("warp_instructions_per_launch", {}).get(workload_name)


# instruction issue: 4 warp schedulers per SM, one instruction each per cycle
ISSUE_PER_SM_PER_CLOCK = 4


def hbm_peak():
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class ClockSampler:
    """nvidia-smi SM clock / throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[3 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def max_over_ranks(value, device=None):
    """The largest value over the ranks of the default process group (the
    job's time is the slowest replica's); identity without a process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload():
    """The headline lattice: D3Q27 192x192x128 lubricated substrate."""
    from paper_1904_06881_gb300 import workloads as W

    return W.c2_lubricated(kw_rho=0.02)


def oracle_sample(wl, n=48):
    """A bounded sample of a D3Q27 workload for the host oracle: the full depth
    (both walls, the film, the drop) of an n x n column through the lattice
    centre; 2D workloads are taken whole."""
    if wl["lattice"] == 0:
        return wl
    nx, ny = wl["nx"], wl["ny"]
    x0, y0 = (nx - n) // 2, (ny - n) // 2
    out = dict(wl)
    for k in ("mask", "rho", "phi"):
        out[k] = np.ascontiguousarray(wl[k][:, y0:y0 + n, x0:x0 + n])
    out["nx"], out["ny"] = n, n
    out["name"] = wl["name"] + " (%dx%d column through the centre, full depth)" % (n, n)
    return out


def density_ratio(wl):
    return round(wl["params"]["rho_l"] / wl["params"]["rho_g"], 3)


def algorithmic_bytes(Q, N):
    """Per launch of the fused step kernel, per node: read f, g (Q floats
    each), write f, g, read the node flag (1 byte); the D3Q27 kernel also
    reads rho, phi (2 floats) from the moments pass (the D2Q9 kernel sums
    them from the populations it reads)."""
    return N * (16 * Q + (1 if Q == 9 else 9))


def measure(lat, stream, steps, warmup, flush=None, kernel_steps=None):
    """Per-step time of whole steps (tlb_step: one launch for D2Q9, a CUDA
    graph of the two launches for D3Q27) and the average duration of the fused
    step kernel alone (launched
    through tlb_step_phase; phase 0, the D3Q27 moments pass, is outside the
    kernel's events), both with CUDA events on the lattice's stream.
    With `flush`, a buffer larger than L2 is written before every timed step."""
    import torch

    from paper_1904_06881_gb300 import tlb

    kernel_steps = kernel_steps or steps
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            if flush is not None:
                flush.fill_(1.0)
            tlb.tlb_step(lat.h, 1)
        stream.synchronize()
        tlb.tlb_sync(lat.h)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        launches0 = lat.launches
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            if flush is not None:
                flush.fill_(float(k))
            ev[k][0].record(stream)
            tlb.tlb_step(lat.h, 1)
            ev[k][1].record(stream)
        stream.synchronize()
        wall = time.perf_counter() - t0
        launches = lat.launches - launches0
        evk = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(kernel_steps)]
        for k in range(kernel_steps):
            if flush is not None:
                flush.fill_(float(k))
            tlb.tlb_step_phase(lat.h, 0)
            tlb.tlb_step_phase(lat.h, 1)
            evk[k][0].record(stream)
            tlb.tlb_step_phase(lat.h, 2)
            evk[k][1].record(stream)
        stream.synchronize()
        tlb.tlb_sync(lat.h)
    step_ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    kern_ms = sum(a.elapsed_time(b) for a, b in evk) / kernel_steps
    return step_ms, kern_ms, launches, wall


def issue_roofline(workload_name, kern_ms, sm_mhz, n_sm=152):
    """Instruction issue against the SMs' ceiling (152 SMs x 4 warp
    instructions per clock at the sampled SM clock): the bound the step
    kernels meet before HBM, from the committed instruction count."""
    inst = measured_instructions(workload_name)
    if not inst or not sm_mhz:
        return None
    achieved = inst / (kern_ms * 1e-3) / 1e9
    peak = n_sm * ISSUE_PER_SM_PER_CLOCK * sm_mhz * 1e6 / 1e9
    return {"achieved": round(achieved, 1), "peak": round(peak, 1), "unit": "G warp-instructions/s",
            "frac": round(achieved / peak, 4), "warp_instructions_per_launch": inst,
            "peak_source": "152 SMs x 4 schedulers x sampled SM clock"}


def roofline(Q, N, kern_ms, peak, peak_kind, kernel_name, workload_name):
    achieved = algorithmic_bytes(Q, N) / (kern_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": kernel_name, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": peak_kind + " hbm_gbs of MEASURED_PEAKS.json",
            "traffic": measured_traffic(workload_name), "kernel_ms": round(kern_ms, 5),
            "algorithmic_bytes_per_launch": algorithmic_bytes(Q, N)}


def _lattice_desc(wl):
    names = {0: "force", 1: "geometric extrapolation", 2: "geometric interpolation"}
    return {"workload": wl["name"], "lattice": "D2Q9" if wl["lattice"] == 0 else "D3Q27", "nx": wl["nx"],
            "ny": wl["ny"], "nz": wl["nz"], "wetting": names[wl["params"]["wetting"]],
            "density_ratio": density_ratio(wl)}


def run_ours(args):
    import torch

    from paper_1904_06881_gb300 import tlb
    from paper_1904_06881_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    peak, peak_kind = hbm_peak()
    wl = workload()
    stream = torch.cuda.Stream()
    lat = tlb.lattice_from_workload(wl)
    tlb.tlb_set_stream(lat.h, stream.cuda_stream)
    N, Q = lat.N, lat.Q
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        step_ms, kern_ms, launches, wall = measure(lat, stream, args.steps, args.warmup, flush=None)
    if world > 1:
        step_ms = max_over_ranks(step_ms, device="cuda")
    value = world * N / (step_ms * 1e-3) / 1e6
    cfg = _lattice_desc(wl)
    cfg.update({"kappa_w": wl["params"]["kw_rho"],
                "l2": "state 2.1 GB, larger than the 126 MB L2; no flush needed",
                "parallelism": "replicas" if world > 1 else "single GPU"})
    fluid = int((wl["mask"] == 0).sum())
    result = {
        "metric": "MLUPS", "value": round(value, 2), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 5), "higher_is_better": True,
        "fluid_mlups": round(world * fluid / (step_ms * 1e-3) / 1e6, 2),
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": cfg,
        "roofline": roofline(Q, N, kern_ms, peak, peak_kind,
                             "step_batch_kernel<D3Q27> (ghost layer, stencils, force, collision, stream)",
                             wl["name"]),
        "whole_step": {"bytes_per_node": algorithmic_bytes(Q, 1) + 8 * Q + 9,
                       "note": "moments pass (read f, g, flag; write rho, phi) + step kernel",
                       "frac_of_peak": round((algorithmic_bytes(Q, 1) + 8 * Q + 9) * N / (step_ms * 1e-3) / 1e9
                                             / peak, 4),
                       "frac_of_peak_16Q": round(16 * Q * N / (step_ms * 1e-3) / 1e9 / peak, 4)},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "host_wall_s": round(wall, 4),
    }
    result["roofline"]["issue"] = issue_roofline(wl["name"], kern_ms, result["clocks"].get("sm_mhz"))
    if rank == 0:
        result["e2e"] = e2e_run(wl, tlb)
    if not args.no_large:
        # reduced-precision g (rest population FP32, moving populations FP16)
        wl16 = dict(wl)
        wl16["params"] = dict(wl["params"], g_fp16=1)
        l16 = tlb.lattice_from_workload(wl16)
        tlb.tlb_set_stream(l16.h, stream.cuda_stream)
        hms, hkms, _, _ = measure(l16, stream, max(args.steps // 4, 10), 3, flush=None)
        # same number of steps from the same initial state in both formats
        n32, n16 = lat.steps_done, l16.steps_done
        if n16 < n32:
            l16.step(n32 - n16)
        elif n32 < n16:
            lat.step(n16 - n32)
        f32, f16 = lat.fields(), l16.fields()
        fl = wl["mask"] == 0
        d = lat.derived
        result["fp16_g"] = {
            "workload": wl["name"] + " (g: g_0 FP32, moving populations FP16)",
            "value": round(world * l16.N / (hms * 1e-3) / 1e6, 2), "unit": "MLUPS", "ms_per_step": round(hms, 4),
            "kernel_ms": round(hkms, 5),
            "roofline_frac_12Q": round((12 * Q + 9) * N / (hkms * 1e-3) / 1e9 / peak, 4),
            "normwise_diff_vs_fp32_after_steps": {
                "steps": int(max(n32, n16)),
                "rho": float(np.abs(f32["rho"] - f16["rho"])[fl].max() / (d["rho_l"] - d["rho_g"])),
                "phi": float(np.abs(f32["phi"] - f16["phi"])[fl].max() / wl["params"]["chi"])}}
        l16.close()
    lat.close()
    # the D2Q9 1024x64 capillary channel: 9.4 MB of state, L2-resident, so a
    # 256 MB buffer is written before every timed step
    c1 = W.c1_capillary()
    l1 = tlb.lattice_from_workload(c1)
    tlb.tlb_set_stream(l1.h, stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    with ClockSampler(local) as clk1:
        ms1, kms1, la1, _ = measure(l1, stream, args.steps, args.warmup, flush=flush)
    d1 = _lattice_desc(c1)
    d1.update({"value": round(world * l1.N / (ms1 * 1e-3) / 1e6, 2), "unit": "MLUPS", "ms_per_step": round(ms1, 5),
               "gpu_launches": int(la1), "clocks": clk1.summary(), "angles_deg": [30, 60, 120],
               "l2": "256 MB buffer written before every timed step; steps timed alone",
               "roofline": roofline(l1.Q, l1.N, kms1, peak, peak_kind,
                                    "step_batch_kernel<D2Q9> (moments, ghost layer, stencils, force, collision, "
                                    "stream)", c1["name"])})
    result["c1_capillary"] = d1
    l1.close()
    del flush
    if not args.no_large:
        # the large periodic lattices (no walls)
        result["big_lattices"] = []
        for bw in (W.big_periodic_drop_2d(4096), W.big_periodic_drop_3d(256)):
            bl = tlb.lattice_from_workload(bw)
            tlb.tlb_set_stream(bl.h, stream.cuda_stream)
            del bw["rho"], bw["phi"]
            bms, bkms, blaunch, _ = measure(bl, stream, 10, 3, flush=None)
            result["big_lattices"].append({
                "workload": bw["name"], "value": round(world * bl.N / (bms * 1e-3) / 1e6, 2), "unit": "MLUPS",
                "ms_per_step": round(bms, 4), "gpu_launches": int(blaunch), "l2": "state larger than L2; no flush",
                "roofline": roofline(bl.Q, bl.N, bkms, peak, peak_kind, "step_batch_kernel", bw["name"])})
            bl.close()
    if rank == 0 and not args.no_batch:
        result["batched"] = batched_sweep()
        result["served"] = served_mix()
        result["tension_sweep"] = tension_sweep()
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(wl, seconds=args.cpu_seconds)
    if world > 1:
        torch.distributed.destroy_process_group()
    return result if rank == 0 else None


def e2e_run(wl, tlb, nsteps=1000, reps=2):
    """MLUPS of whole jobs through the public C ABI: tlb_init_fields from host
    arrays, nsteps steps, tlb_get_fields back to host arrays."""
    lat = tlb.Lattice(wl["lattice"], wl["nx"], wl["ny"], wl["nz"], **wl["params"])
    lat.set_solid(wl["mask"])
    rho = np.ascontiguousarray(wl["rho"], dtype=np.float64)
    phi = np.ascontiguousarray(wl["phi"], dtype=np.float64)
    lat.init_fields(rho, phi)
    lat.step(10)
    lat.fields()
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        lat.init_fields(rho, phi)
        lat.step(nsteps)
        f = lat.fields()
        times.append(time.perf_counter() - t0)
        assert np.isfinite(f["rho"]).all()
    t = min(times)
    N = lat.N
    h2d = 2 * N * 8
    d2h = (2 + lat.D + 3) * N * 8
    return {"value": round(N * nsteps / t / 1e6, 2), "unit": "MLUPS", "h2d_bytes_per_step": round(h2d / nsteps, 1),
            "d2h_bytes_per_step": round(d2h / nsteps, 1),
            "job": "tlb_init_fields (host FP64) + %d steps + tlb_get_fields (host FP64)" % nsteps}


def batched_sweep(steps=5000, seq_steps=100):
    """The contact-angle sweep (512 D2Q9 lattices, 64^2-512^2, 43.8 M nodes):
    one sequential pass, every lattice advanced `seq_steps` by tlb_step one
    after another (steps 3 .. seq_steps + 2), then the whole sweep's `steps`
    (the configuration's 5000) by one resident batch (tlb_batch_*: the launch
    configuration chosen by the autotuner, CUDA-graph replays)."""
    import torch

    from paper_1904_06881_gb300 import tlb
    from paper_1904_06881_gb300 import workloads as W

    items = W.c3_sweep()
    lats = [tlb.lattice_from_workload(W.c3_lattice(it)) for it in items]
    nodes = sum(l.N for l in lats)
    t0 = time.perf_counter()
    batch = tlb.Batch(lats)
    cfg = batch.tune(reps=2)
    t_tune = time.perf_counter() - t0
    batch.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for l in lats:
        l.step(seq_steps)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    batch.step(steps)
    e1.record()
    torch.cuda.synchronize()
    tb = e0.elapsed_time(e1) * 1e-3
    diverged = 0
    for l in lats:
        try:
            l.sync()
        except tlb.TlbError:
            diverged += 1
    names = {0: "lattice-major", 1: "interleaved", 2: "largest first"}
    res = {"workload": "c3 sweep: %d D2Q9 lattices, %d nodes" % (len(lats), nodes),
           "batched_mlups": round(nodes * steps / tb / 1e6, 1),
           "sequential_mlups": round(nodes * seq_steps / ts / 1e6, 1),
           "speedup": round((ts / seq_steps) / (tb / steps), 3), "steps": steps, "sequential_steps": seq_steps,
           "batched_s": round(tb, 3), "diverged_lattices": diverged,
           "tuned": {"variant": cfg["variant"], "tile_order": names[cfg["tile_order"]],
                     "graph_depth": cfg["graph_depth"], "us_per_step": round(cfg["us_per_step"], 2),
                     "tuning_s": round(t_tune, 3)},
           "roofline_frac": round(algorithmic_bytes(9, nodes) / (tb / steps) / 1e9 / hbm_peak()[0], 4),
           "l2": "state %.1f GB, larger than L2" % (sum(l.device_bytes for l in lats) / 1e9)}
    batch.close()
    for l in lats:
        l.close()
    return res


def tension_sweep(grid=4, L=96, R=24.0, steps=3000):
    """Surface-tension characterisation (Sec. III, Table 2): a grid x grid
    map of subspace 6, three bubble lattices per point (one per interface
    pair), all advanced by one batch; then gamma, Neumann angles and D_k per
    point.  Reports the batch's stepping throughput and the whole sweep's
    wall time (creation, stepping, measurement)."""
    from paper_1904_06881_gb300 import tension as T

    t0 = time.perf_counter()
    res, t = T.sweep(T.grid(6, grid), L=L, R=R, steps=steps)
    wall = time.perf_counter() - t0
    ok = sum(1 for r in res if not r["failed"] and all(np.isfinite(r["theta"])))
    return {"workload": "subspace 6 map, %d points x 3 bubbles (%d^2, R %.0f), %d steps" % (len(res), L, R, steps),
            "lattices": t["lattices"], "nodes": t["nodes"], "batch_mlups": round(t["mlups"], 1),
            "sweep_wall_s": round(wall, 3), "points_with_neumann_angles": ok,
            "example": {"lam": res[0]["point"]["lam"], "kappa": res[0]["point"]["kappa"],
                        "gamma": {k: round(v, 5) for k, v in res[0]["gamma"].items()},
                        "theta_deg": [round(v, 2) for v in res[0]["theta"]]}}


def _serve(reqs, budget_gb, max_active, steps_per_round, arrivals, policy=0, max_wait_s=0.0):
    """Run the request list through the continuous-batching server: with
    `arrivals` each request is submitted at its Poisson arrival time, else all
    at once (a saturated server).  Time from submission to result per request
    and aggregate MLUPS over the makespan."""
    from paper_1904_06881_gb300 import tlb

    srv = tlb.Server(int(budget_gb * (1 << 30)), max_active=max_active, steps_per_round=steps_per_round,
                     policy=policy, max_wait_s=max_wait_s)
    t_start = time.perf_counter()
    pending = list(range(len(reqs)))
    tickets, lat, failed = {}, {}, {}
    while len(lat) + len(failed) < len(reqs):
        now = time.perf_counter() - t_start
        while pending and (not arrivals or reqs[pending[0]][0] <= now):
            k = pending.pop(0)
            _, wl, n = reqs[k]
            tickets[k] = srv.submit(wl["lattice"], wl["nx"], wl["ny"], wl["nz"], wl["mask"], wl["rho"], wl["phi"], n,
                                    **wl["params"])
        srv.pump()
        for k, t in list(tickets.items()):
            if k in lat or k in failed:
                continue
            r = srv.poll(t)
            if r["state"] == tlb.REQ_DONE:
                lat[k] = r["done_s"] - r["submit_s"]
            elif r["state"] == tlb.REQ_FAILED:
                failed[k] = tlb.ERRORS.get(r["status"], r["status"])
        if len(lat) + len(failed) == len(tickets) and pending:
            time.sleep(max(0.0, reqs[pending[0]][0] - (time.perf_counter() - t_start)))
    makespan = time.perf_counter() - t_start
    srv.close()
    work = sum(reqs[k][1]["nx"] * reqs[k][1]["ny"] * reqs[k][1]["nz"] * reqs[k][2] for k in lat)
    lats = np.array([lat[k] for k in sorted(lat)]) if lat else np.zeros(1)
    return {"completed": len(lat), "failed": {str(k): v for k, v in failed.items()},
            "p50_s": round(float(np.percentile(lats, 50)), 4), "p99_s": round(float(np.percentile(lats, 99)), 4),
            "aggregate_mlups": round(work / makespan / 1e6, 1), "makespan_s": round(makespan, 3),
            "node_steps": work}, sorted(lat)


def served_mix(budget_gb=48.0, max_active=64, steps_per_round=100):
    """The served mix (workloads.c4_requests: 256 requests of drops, channels,
    lubricated substrates, lenses and drop trains, 64^2-1024^2 and 96^3-192^3,
    liquid-gas and liquid-liquid) through the continuous-batching server:
    with Poisson arrivals (20/s) admitted in arrival order, the same arrivals
    admitted least-work first (requests older than 10 s first), and every
    request submitted at the start (saturated), against the same requests run
    one after another alone through tlb_step (the same kernels, so the same
    results)."""
    import torch

    from paper_1904_06881_gb300 import tlb
    from paper_1904_06881_gb300 import workloads as W

    reqs = W.c4_requests()
    poisson, done = _serve(reqs, budget_gb, max_active, steps_per_round, arrivals=True)
    shortest, _ = _serve(reqs, budget_gb, max_active, steps_per_round, arrivals=True, policy=tlb.SCHED_SHORTEST,
                         max_wait_s=10.0)
    saturated, _ = _serve(reqs, budget_gb, max_active, steps_per_round, arrivals=False)
    t0 = time.perf_counter()
    for k in done:
        _, wl, n = reqs[k]
        l = tlb.lattice_from_workload(wl)
        l.step(n)
        l.sync()
        l.close()
    torch.cuda.synchronize()
    tseq = time.perf_counter() - t0
    work = poisson["node_steps"]
    return {"workload": "c4 served mix: %d requests (%.1f G node-steps), Poisson 20/s over %.1f s"
                        % (len(reqs), sum(w["nx"] * w["ny"] * w["nz"] * n for _, w, n in reqs) / 1e9, reqs[-1][0]),
            "poisson": poisson, "poisson_shortest_first": shortest, "saturated": saturated,
            "sequential_alone_mlups": round(work / tseq / 1e6, 1), "sequential_alone_s": round(tseq, 3),
            "server": {"budget_gb": budget_gb, "max_active": max_active, "steps_per_round": steps_per_round,
                       "admission": "arrival order; poisson_shortest_first: least work first, requests older "
                                    "than 10 s first"}}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu part", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.processor() or platform.machine()


def oracle_rate(wl, threads, seconds):
    """MLUPS of the FP64 oracle as it stands on `wl`, with `threads` host
    threads, over at least one step and about `seconds` of stepping."""
    import oracle

    oracle.threads(threads)
    o = oracle.from_workload(wl)
    o.step(1)
    n, t0 = 0, time.perf_counter()
    while n == 0 or time.perf_counter() - t0 < seconds:
        o.step(1)
        n += 1
    dt = time.perf_counter() - t0
    N = wl["nx"] * wl["ny"] * wl["nz"]
    return N * n / dt / 1e6, n, dt


def cpu_baseline(wl, seconds=4.0):
    """The FP64 oracle as it stands, on this host's cores: the headline's
    bounded sample (a column of the D3Q27 lattice) at all cores, plus the
    D2Q9 drop and channel lattices whole, each at one thread and at all cores."""
    from paper_1904_06881_gb300 import workloads as W

    cores = os.cpu_count()
    detail = []
    head = None
    for w in (W.c0_sessile_drop(), W.c1_capillary(), oracle_sample(wl)):
        for th in (1, cores):
            v, n, dt = oracle_rate(w, th, seconds)
            detail.append({"workload": w["name"], "threads": th, "MLUPS": round(v, 4), "steps": n,
                           "seconds": round(dt, 2)})
            if w["lattice"] == 1 and th == cores:
                head = (v, n, dt, w["name"])
    v, n, dt, name = head
    return {"value": round(v, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": "%d full time steps of %s in %.1f s" % (n, name, dt),
            "cpu_model": _cpu_model(), "nproc": cores, "detail": detail}


def run_only(args):
    """One lattice, timed as in the full run; for profiling under ncu."""
    import torch

    from paper_1904_06881_gb300 import tlb
    from paper_1904_06881_gb300 import workloads as W

    if args.only == "c1":
        wl = W.c1_capillary()
    elif args.only == "c2_96":
        # the c2 geometry at 96 x 96 x 128 (0.6 GB on the device, still larger
        # than L2): the case the detailed ncu captures are taken on
        wl = W.c2_lubricated(nx=96, ny=96, nz=128, kw_rho=0.02)
    elif args.only == "d2q9_2048":
        # a large periodic D2Q9 lattice at a quarter of the bench's 4096^2
        # (0.6 GB on the device, larger than L2)
        wl = W.big_periodic_drop_2d(2048)
    else:
        wl = workload()
    stream = torch.cuda.Stream()
    lat = tlb.lattice_from_workload(wl)
    tlb.tlb_set_stream(lat.h, stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda") if args.only == "c1" else None
    step_ms, kern_ms, launches, _ = measure(lat, stream, args.steps, args.warmup, flush=flush)
    return {"workload": wl["name"], "value": round(lat.N / (step_ms * 1e-3) / 1e6, 2), "unit": "MLUPS",
            "ms_per_step": round(step_ms, 5), "kernel_ms": round(kern_ms, 5), "gpu_launches": int(launches),
            "note": "profiling run; not a benchmark line"}


def run_noalloc(args):
    """The allocation-free entry point (tlb_step_noalloc: the step kernel of
    tlb_step over its own tile table, one launch per D2Q9 step) against a
    context's step on the same lattice, the D2Q9 1024x64 capillary channel
    (65,536 nodes, L2-resident for both), device time per step by CUDA events
    on one stream; and the host time of one call when the previous call left
    the same geometry."""
    import torch

    from paper_1904_06881_gb300 import tlb
    from paper_1904_06881_gb300 import workloads as W

    wl = W.c1_capillary()
    stream = torch.cuda.Stream()
    lat = tlb.lattice_from_workload(wl)
    tlb.tlb_set_stream(lat.h, stream.cuda_stream)
    c, w = tlb.tlb_lattice_directions(wl["lattice"])
    f0, g0 = lat.populations()
    dev = torch.device("cuda")
    f = torch.tensor((f0 - w[:, None]).astype(np.float32), device=dev)
    g = torch.tensor(g0.astype(np.float32), device=dev)
    f_tmp, g_tmp = torch.empty_like(f), torch.empty_like(g)
    p = tlb.make_params(wl["lattice"], wl["nx"], wl["ny"], wl["nz"], **wl["params"])
    K = 2 * max(1, (args.steps + 1) // 2)          # even: the result ends in f, g without a copy

    def noalloc(n):
        tlb.tlb_step_noalloc(p, wl["mask"], f.data_ptr(), f_tmp.data_ptr(), g.data_ptr(), g_tmp.data_ptr(), n,
                             stream.cuda_stream)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn(K)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / K

    noalloc(2 * args.warmup)
    lat.step(args.warmup)
    torch.cuda.synchronize()
    na_ms = min(timed(noalloc) for _ in range(3))
    ctx_ms = min(timed(lat.step) for _ in range(3))
    torch.cuda.synchronize()
    calls = 50
    t0 = time.perf_counter()
    for _ in range(calls):
        noalloc(2)
    host_us = (time.perf_counter() - t0) / calls * 1e6
    torch.cuda.synchronize()
    lat.close()
    N = wl["nx"] * wl["ny"] * wl["nz"]
    return {"workload": wl["name"], "steps_per_timing": K,
            "noalloc": {"ms_per_step": round(na_ms, 5), "MLUPS": round(N / (na_ms * 1e-3) / 1e6, 1),
                        "launches_per_step": 1},
            "context": {"ms_per_step": round(ctx_ms, 5), "MLUPS": round(N / (ctx_ms * 1e-3) / 1e6, 1)},
            "noalloc_host_us_per_call_2_steps": round(host_us, 1),
            "note": "entry-point comparison; not a benchmark line"}


def run_reference(args):
    """The oracle (the reference arm: the paper has no code) on the host cores,
    on the headline workload's bounded sample: one oracle time step of a
    48 x 48 x 128 column of the D3Q27 lattice per bench step."""
    rank, world, local = dist_env()
    if rank != 0:
        return None
    wl = oracle_sample(workload())
    import oracle

    cores = os.cpu_count()
    oracle.threads(cores)
    o = oracle.from_workload(wl)
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    dt = time.perf_counter() - t0
    N = wl["nx"] * wl["ny"] * wl["nz"]
    value = N * args.steps / dt / 1e6
    cfg = _lattice_desc(workload())
    cfg["sample"] = wl["name"]
    return {"impl": "reference", "metric": "MLUPS", "value": round(value, 4), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": "%d full time steps of %s on the host cores" % (args.steps, wl["name"]),
                             "cpu_model": _cpu_model()},
            "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=4.0, help="seconds per oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the reduced-precision run and the large periodic lattices")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched sweep and the served mix")
    ap.add_argument("--only", choices=["c1", "c2", "c2_96", "d2q9_2048", "noalloc"],
                    help="time one lattice only (profiling runs): no e2e, no CPU baseline")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.only == "noalloc":
        res = run_noalloc(args)
    elif args.only:
        res = run_only(args)
    else:
        res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
