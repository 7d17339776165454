#!/usr/bin/env python3
"""Throughput of the full total-Lagrangian vectorial LBM step on one B300.

Workload (default): the 3D D3Q6x12 FP32 thick spherical shell on a 256^3 box
(R_i = 0.4, R_o = 0.9 of the half-width, mu = 1, lambda = 5, internal nominal
pressure with the sin^2 ramp, outer surface traction-free, c = 10, omega = 1.8,
gamma = 10, compatibility projection every 20 steps): 5,841,344 active nodes,
299,448 Neumann cut links.  A step is one pass of Algorithm 1 over the whole body:
fused pull gather + cut-link closure + recovery + collision, per-link boundary
sources (LSQ + Newton), and on every 20th step the two projection solves with the
population repair.  Timed steps include their share of projection steps (K is a
multiple of 20 by default).

Printed: one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on the
host cores instead (a bounded 64^3 copy of the same workload).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and HBM GB/s (% of peak), FP32 vs FP64 at stated L2 error; adjoint/forward time"
UNIT = "MLUPS"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="box nodes per axis of the shell workload")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-bf16", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-errors", action="store_true", help="skip the FP32/FP64 errors against the oracle")
    ap.add_argument("--no-batch", action="store_true", help="skip the packed 2D multi-specimen measurement")
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--batch-specimens", type=int, default=96, help="specimens of the packed 2D batch")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the reverse-mode measurement")
    ap.add_argument("--adj-n", type=int, default=128)
    ap.add_argument("--adj-steps", type=int, default=3000)
    ap.add_argument("--adj-every", type=int, default=100)
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM traffic of the fused kernel from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum
# of one launch) on the 128^3 copy of the workload, stored with the SHA-256 of the kernel sources it
# was measured on and reported only while those sources are unchanged (null otherwise).  Each
# 32-node window of the launch stages and stores whole boxes, so the traffic is scaled to the
# timed box by its number of windows (segments).
KERNEL_SOURCES = ["paper_2606_20646_b300/csrc/lbm_tma.cuh", "paper_2606_20646_b300/csrc/lbm_kernels.cuh",
                  "paper_2606_20646_b300/csrc/lbm_device.cuh"]
TRAFFIC_CAPTURE = {"sources_sha256": "2e5642890a287691ab0a67aeee019f2e73c0b5c4ee76206a35ff6ce29f67fa20",
                   "bytes_per_launch": 375150336 + 265185152, "windows": 30112,
                   "summary": "profiles/k_stream_collide_tma_shell_3d.md"}
# the same for the BF16-storage fused kernel (two windows per warp)
BF16_TRAFFIC_CAPTURE = {"sources_sha256": "2e5642890a287691ab0a67aeee019f2e73c0b5c4ee76206a35ff6ce29f67fa20",
                        "bytes_per_launch": 218193408 + 133783296, "windows": 30112,
                        "summary": "profiles/k_stream_collide_tma_bf16_shell_3d.md"}
# the same for the reverse step on the clamped cube (128^3, the timed size itself)
ADJ_SOURCES = ["paper_2606_20646_b300/csrc/lbm_adjoint.cuh", "paper_2606_20646_b300/csrc/lbm_tma.cuh",
               "paper_2606_20646_b300/csrc/lbm_kernels.cuh"]
ADJ_TRAFFIC_CAPTURE = {"sources_sha256": "1f155594c04ba11848b4cd93e824e9713aa5740703e15a8ba72426b1ee6c3a97",
                       "bytes_per_launch": 741957632 + 576005973, "windows": None,
                       "summary": "profiles/k_adj_step_tma_inclusion_cube.md"}


def kernel_sources_hash(sources=KERNEL_SOURCES):
    import hashlib
    h = hashlib.sha256()
    for rel in sources:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def captured_traffic(windows, cap=TRAFFIC_CAPTURE, sources=KERNEL_SOURCES):
    """Captured bytes per launch, scaled from the captured launch's windows to `windows` (None: the
    capture ran the timed size itself); None when there is no capture of the current sources."""
    if not cap or cap.get("sources_sha256") != kernel_sources_hash(sources):
        return None
    if cap.get("windows") is None:
        return cap["bytes_per_launch"]
    return int(round(cap["bytes_per_launch"] * windows / cap["windows"]))


def bytes_per_node(D, real_size):
    """Algorithmic HBM bytes per active node of the fused collide-stream kernel as this build moves
    them: every population component read once and written once, u* read and written (8 bytes per
    component in both forms: an FP64 plane, or an FP32 hi/lo pair), one flag byte."""
    K, Q = D + D * D, 2 * D
    return 2 * Q * K * real_size + 2 * D * 8 + 1


def method_bytes_per_node(D, real_size):
    """The method's algorithmic bytes per active node and step (the coverage contract's figure):
    every population component read and written once, u* read and written in the population
    precision, one flag byte -- 601 B in 3D FP32.  The build's FP32 u* pairs add 2 D 4 bytes."""
    K, Q = D + D * D, 2 * D
    return 2 * Q * K * real_size + 2 * D * real_size + 1


def link_bytes(D, real_size, n_cut, lsq_entries):
    """Algorithmic bytes of one launch of the link kernel: per cut link its geometry (node,
    direction, BC index, stencil size: 16 B; eta, N_b, tangents: 8 (1 + D + 2 D) B), the kept pair
    read (2 K values), the reconstruction written (K values) and the Newton state read and written
    (2 D values); per Neumann stencil entry its index and D - 1 weights."""
    K = D + D * D
    per_link = 16 + 8 * (1 + 3 * D) + (3 * K + 2 * D) * real_size
    return n_cut * per_link + lsq_entries * (4 + (D - 1) * real_size)


def jacobi_bytes_per_node(D, real_size, sweeps_per_launch=1):
    """Algorithmic HBM bytes per active node and sweep of the damped-Jacobi sweeps: per launch the
    node's correction vector read and written (D values padded to 2 or 4), its residual vector (4
    values: r and the sweep weight) and its flag byte, shared by the sweeps of the launch (two with
    the two-sweep kernel, whose first sweep stays in shared memory); neighbour reads hit in cache.
    The FP32 forms' 3D sweeps and 2D two-sweep launches load no flag byte: the node's cut bits ride
    in a spare slot of d (3D) or of the residual (2D)."""
    dv = 4 if D == 3 else 2
    flag = 1 if real_size == 8 or (D == 2 and sweeps_per_launch == 1) else 0
    return (2 * dv * real_size + 4 * real_size + flag) / sweeps_per_launch


def adjoint_bytes_per_node(D, real_size):
    """Algorithmic HBM bytes per active node of one reverse step: the next step's gbar read once
    and this step's written once (Q*K values each), the recorded F (D*D values) and dL/du* (D
    values) read, dL/dmu (FP64) read and written, one flag byte.  Cut links add their coefficient
    and side rows (below 0.3 % of the nodes' bytes on a clamped cube)."""
    K, Q = D + D * D, 2 * D
    return 2 * Q * K * real_size + D * D * real_size + D * real_size + 2 * 8 + 1


def recompute_bytes_per_node(D, real_size):
    """The forward step of the backward's recomputation: the fused kernel's bytes plus the D*D
    recorded F values written."""
    return bytes_per_node(D, real_size) + D * D * real_size


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(n=64, steps=None, warmup=0, budget_s=15.0, threads=1):
    """FP64 oracle on an n^3 copy of the shell workload on `threads` host threads (0: all)."""
    import oracle
    from paper_2606_20646_b300 import inputs as I
    oracle.set_threads(threads if threads > 0 else (os.cpu_count() or 1))
    p = I.shell_3d(n)
    o = oracle.Oracle(p).set_initial()
    if warmup:
        o.step(warmup)
    nact = o.counts()["n_active"]
    if steps is None:
        # calibrate on one projection cycle (20 steps, one of them a projection step), so that the
        # per-step estimate carries the projection's amortised share
        t0 = time.perf_counter()
        o.step(20)
        dt = time.perf_counter() - t0
        steps = max(20, int(budget_s / max(dt / 20, 1e-6)) // 20 * 20)
    t0 = time.perf_counter()
    o.step(steps)
    el = time.perf_counter() - t0
    return nact * steps / el / 1e6, steps, el, nact


def oracle_errors(n, steps, dev):
    """Relative L2 errors of the FP32 and FP64 forms against the FP64 oracle on an n^3 copy of the
    shell workload after `steps` steps (v, F, F - I, u over the active nodes); the oracle runs on
    all host threads."""
    import numpy as np
    import oracle
    from paper_2606_20646_b300 import inputs as I, lbm
    oracle.set_threads(os.cpu_count() or 1)
    p = I.shell_3d(n)
    o = oracle.Oracle(p).set_initial()
    o.step(steps)
    ref = o.fields()
    act = o.active_mask()
    eye = np.eye(3).reshape(9, 1)
    out = {"workload": f"shell_3d_{n} after {steps} steps (t = {steps * p.dt:.3f})"}
    for prec in ("fp32", "fp64"):
        sim = lbm.Simulation(p, precision=prec, device=dev)
        sim.set_initial().step(steps)
        g = [t.cpu().numpy() for t in sim.fields()]
        sim.close()
        e = {nm: float(np.linalg.norm(a[:, act] - b[:, act]) / np.linalg.norm(b[:, act]))
             for nm, a, b in zip("vFu", g, ref)}
        e["F_minus_I"] = float(np.linalg.norm(g[1][:, act] - ref[1][:, act]) / np.linalg.norm(ref[1][:, act] - eye))
        out[prec] = e
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return
    t0 = time.time()
    cores = os.cpu_count() or 1
    mlups, steps, el, nact = oracle_sample(n=64, steps=args.steps, warmup=args.warmup, threads=cores)
    sample = (f"FP64 C oracle (lbm_oracle.c, {cores} host threads) on the 64^3 copy of the shell workload "
              f"({nact} active nodes), {args.warmup} untimed + {steps} timed steps incl. projection steps")
    line = {"impl": "reference", "metric": METRIC, "value": round(mlups, 4), "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": round(1e3 * el / steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"shell_3d_{args.n} (64^3 copy on the host)"},
            "cpu_baseline": {"value": round(mlups, 4), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(mlups, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(time.time() - t0, 1)}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch
    from paper_2606_20646_b300 import build as b
    b.build()
    from paper_2606_20646_b300 import inputs as I
    from paper_2606_20646_b300 import lbm

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    peak, peak_kind = measured_peaks()
    K, W = args.steps, args.warmup
    p = I.shell_3d(args.n)

    def timed(sim, steps, with_timing):
        stream = sim.stream
        torch.cuda.synchronize()
        barrier(world)
        if with_timing:
            sim.enable_timing(True)
        l0 = sim.info()["launches"]
        clk = Clocks(torch.cuda.current_device()) if with_timing else None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier(world)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = e0.elapsed_time(e1)
        clocks = clk.stop() if clk else None
        launches = sim.info()["launches"] - l0
        kt = sim.kernel_times() if with_timing else None
        return ms, launches, kt, clocks

    # ---- main measurement: FP32, populations resident in HBM --------------------------------
    sim = lbm.Simulation(p, precision="fp32", device=dev)
    sim.set_initial()
    sim.step(W)
    st_warm = sim.sync(raise_on_status=False)
    if st_warm:
        raise SystemExit(f"device status {st_warm} after warm-up; not timing a failing step")
    # tile shapes by the library's autotuner (timed from the warm state, which it restores)
    tuning = sim.autotune(steps=20) if not args.no_autotune else sim.get_tuning()
    ms, launches, kt, clocks = timed(sim, K, True)
    st = sim.sync(raise_on_status=False)
    info = sim.info()
    nact = info["n_active"]
    ms = max_over_ranks(ms, world)
    value = world * nact * K / (ms / 1e3) / 1e6
    avg_sc = kt["stream_collide_ms"] / max(kt["stream_collide_launches"], 1)
    bpn = method_bytes_per_node(3, 4)          # the method's 601 B per node
    achieved = nact * bpn / (avg_sc / 1e3) / 1e9
    achieved_moved = nact * bytes_per_node(3, 4) / (avg_sc / 1e3) / 1e9
    share = {"stream_collide": kt["stream_collide_ms"] / ms, "cutlink": kt["cutlink_ms"] / ms,
             "projection": kt["projection_ms"] / ms, "jacobi (within projection)": kt["jacobi_ms"] / ms}
    avg_jac = kt["jacobi_ms"] / max(kt["jacobi_launches"], 1)
    jsw = tuning.get("jacobi_sweeps", 1) or 1
    jacobi = {"avg_sweep_us": round(avg_jac * 1e3, 2), "sweeps": kt["jacobi_launches"], "sweeps_per_launch": jsw,
              "bytes_per_node_sweep": jacobi_bytes_per_node(3, 4, jsw),
              "GBps": round(nact * jacobi_bytes_per_node(3, 4, jsw) / (avg_jac / 1e3) / 1e9, 1) if avg_jac > 0 else None}
    avg_cut = kt["cutlink_ms"] / max(kt["cutlink_launches"], 1)
    lb = link_bytes(3, 4, info["n_cut"], info["lsq_entries"])
    links = {"kernel": "k_links_f32<3>", "avg_launch_ms": round(avg_cut, 4), "bytes_per_launch": lb,
             "achieved_GBps": round(lb / (avg_cut / 1e3) / 1e9, 1) if avg_cut > 0 else None,
             "frac": round(lb / (avg_cut / 1e3) / 1e9 / peak, 4) if avg_cut > 0 else None}
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": captured_traffic(info["n_segments"]),
                "kernel": "k_stream_collide_tma<3>", "bytes_per_launch": nact * bpn,
                "bytes_per_node": bpn, "avg_launch_ms": round(avg_sc, 4), "peak_kind": peak_kind,
                "frac_of_bytes_moved": round(achieved_moved / peak, 4),
                "bytes_per_node_moved": bytes_per_node(3, 4),
                "note": "frac counts the method's 601 B per active node; frac_of_bytes_moved counts the "
                        "625 B this build moves (u* as FP32 hi/lo pairs); traffic is the ncu DRAM bytes of "
                        "one launch on the 128^3 copy, scaled by windows"}
    del sim
    torch.cuda.empty_cache()

    # ---- FP64 form on the same workload --------------------------------------------------------
    fp64 = None
    if not args.no_fp64:
        sim = lbm.Simulation(p, precision="fp64", device=dev)
        sim.set_initial()
        sim.step(W)
        K64 = max(20, K // 2)
        ms64, _, kt64, _ = timed(sim, K64, True)
        avg64 = kt64["stream_collide_ms"] / max(kt64["stream_collide_launches"], 1)
        fp64 = {"value": round(nact * K64 / (ms64 / 1e3) / 1e6, 2), "steps": K64,
                "stream_collide_GBps": round(nact * bytes_per_node(3, 8) / (avg64 / 1e3) / 1e9, 1),
                "device_status": sim.sync(raise_on_status=False)}
        del sim
        torch.cuda.empty_cache()

    # ---- BF16 population storage on the same workload; its error at t = 1 on the 128^3 copy --------
    bf16 = None
    if not args.no_bf16:
        sim = lbm.Simulation(p, precision="bf16s", device=dev)
        sim.set_initial()
        sim.step(W)
        tune_b = sim.autotune(steps=20) if not args.no_autotune else sim.get_tuning()
        msb, _, ktb, _ = timed(sim, K, True)
        avgb = ktb["stream_collide_ms"] / max(ktb["stream_collide_launches"], 1)
        bpn = bytes_per_node(3, 2)
        gbb = nact * bpn / (avgb / 1e3) / 1e9
        stb = sim.sync(raise_on_status=False)
        del sim
        torch.cuda.empty_cache()
        pe, ne = I.shell_3d(128), 640
        res = {}
        for prec in ("fp64", "bf16s"):
            s2 = lbm.Simulation(pe, precision=prec, device=dev)
            s2.set_initial().step(ne)
            res[prec] = [t.double() for t in s2.fields()]
            acte = torch.as_tensor(s2.active_mask(), device=dev)
            s2.close()
        eye = torch.eye(3, dtype=torch.float64, device=dev).reshape(9, 1, 1, 1)

        def rel(a, b):
            return float(torch.linalg.norm((a - b)[:, acte]) / torch.linalg.norm(b[:, acte]))

        (vb, Fb, ub), (vd, Fd, ud) = res["bf16s"], res["fp64"]
        bf16 = {"value": round(nact * K / (msb / 1e3) / 1e6, 2), "unit": UNIT, "steps": K,
                "ms_per_step": round(msb / K, 4), "dtype": "bf16 storage, f32 arithmetic",
                "stream_collide_ms": round(avgb, 4), "bytes_per_node": bpn,
                "stream_collide_GBps": round(gbb, 1), "frac": round(gbb / peak, 4), "peak_kind": peak_kind,
                "traffic": captured_traffic(info["n_segments"], BF16_TRAFFIC_CAPTURE) if tune_b["windows_per_warp"] == 2 else None,
                "error_vs_fp64": {"workload": "shell_3d_128 at t = 1 (640 steps)", "v": rel(vb, vd),
                                  "F_minus_I": rel(Fb - eye, Fd - eye), "u": rel(ub, ud)},
                "tuning": tune_b, "device_status": stb}
        del res
        torch.cuda.empty_cache()

    # ---- end to end through the C ABI with host buffers ---------------------------------------
    e2e = None
    if not args.no_e2e:
        sim = lbm.Simulation(p, precision="fp32", device=dev, host_staging=True)
        hv = torch.from_numpy(p.v0).pin_memory()
        hF = torch.from_numpy(p.F0).pin_memory()
        hu = torch.from_numpy(p.u0).pin_memory()
        outs = tuple(torch.empty(t.shape, dtype=torch.float64).pin_memory() for t in (hv, hF, hu))
        sim.set_initial(hv, hF, hu)
        sim.step(W)
        sim.fields(out=outs)
        sim.sync(raise_on_status=False)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        sim.set_initial(hv, hF, hu)
        sim.step(K)
        sim.fields(out=outs)
        sim.sync(raise_on_status=False)
        el = max_over_ranks(time.perf_counter() - t0, world)
        h2d = sum(t.numel() * 8 for t in (hv, hF, hu))
        d2h = sum(t.numel() * 8 for t in outs)
        e2e = {"value": round(world * nact * K / el / 1e6, 2), "unit": UNIT,
               "h2d_bytes_per_step": h2d // K, "d2h_bytes_per_step": d2h // K,
               "note": "timed: upload of v0, F0, u0 from pinned host memory, K steps, download of v, F, u"}
        del sim
        torch.cuda.empty_cache()

    # ---- many 2D specimens packed into one body, 1000 steps as one CUDA graph -------------------
    batch = None
    if not args.no_batch:
        packed, specs = I.batch_2d(n_spec=args.batch_specimens, steps=args.batch_steps)
        sim = lbm.Simulation(packed, precision="fp32", device=dev)
        inf_b = sim.info()
        sim.set_initial()
        sim.step(W)
        st_b = sim.sync(raise_on_status=False)
        tune_g = sim.autotune(steps=20) if not args.no_autotune else sim.get_tuning()
        Kb = args.batch_steps
        stream = sim.stream
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        sim.step_graph(Kb)          # stream capture and instantiation on the host, then one launch
        e1.record(stream)
        torch.cuda.synchronize()
        wall = max_over_ranks(time.perf_counter() - t0, world)
        ms_g = max_over_ranks(e0.elapsed_time(e1), world)
        st_b = st_b or sim.sync(raise_on_status=False)
        # the same steps launched one by one, for the launch overhead the graph removes
        e0.record(stream)
        sim.step(Kb // 4)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_s = max_over_ranks(e0.elapsed_time(e1), world) * 4
        nb = inf_b["n_active"]
        batch = {"workload": f"{len(specs)} 2D D2Q4x6 FP32 specimens, sides U{{64..768}}, 1-5 elliptic holes, "
                             f"per-specimen mu and lambda, packed in a {packed.n[0]}x{packed.n[1]} box; "
                             "left edge clamped, right edge translated, holes traction-free",
                 "n_active": nb, "n_cut_links": inf_b["n_cut"], "steps": Kb,
                 "value": round(world * nb * Kb / (ms_g / 1e3) / 1e6, 2) if st_b == 0 else None, "unit": UNIT,
                 "graph_ms": round(ms_g, 2), "graph_wall_s": round(wall, 3),
                 "note": "value over graph_ms: CUDA events around lbm_step_graph, host capture and instantiation included",
                 "stepwise_ms_per_step": round(ms_s / Kb, 4), "graph_ms_per_step": round(ms_g / Kb, 4),
                 "tuning": tune_g, "device_status": st_b}
        del sim
        torch.cuda.empty_cache()

    # ---- reverse mode: dL/dmu and dL/db of a displacement misfit (clamped cube, inclusion) ------
    adj = None
    if not args.no_adjoint:
        from paper_2606_20646_b300 import adjoint as A
        pa = I.inclusion_cube(args.adj_n, args.adj_steps)
        Ka, every = args.adj_steps, args.adj_every
        sim = lbm.Simulation(pa, precision="fp32", device=dev, adjoint=True)
        nact_a = sim.info()["n_active"]
        stream = sim.stream
        ev = lambda: torch.cuda.Event(enable_timing=True)
        # the target displacement (target modulus), then the plain forward time
        sim.set_mu_field(pa.meta["mu_target"]).set_initial()
        sim.step(Ka)
        u_tgt = sim.fields()[2].clone()
        act_t = torch.as_tensor(sim.active_mask(), device=dev)
        sim.set_initial()
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        sim.step(Ka)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_plain = max_over_ranks(e0.elapsed_time(e1), world)

        def run(steps):
            mu = torch.ones(pa.box_shape, dtype=torch.float64, device=dev, requires_grad=True)
            b = torch.tensor(pa.options.body_force, dtype=torch.float64, requires_grad=True)
            e0, e1, e2 = ev(), ev(), ev()
            e0.record(stream)
            u = A.displacement(mu, b, sim, steps, every)
            e1.record(stream)
            loss = 0.5 * (((u - u_tgt) ** 2) * act_t).sum()
            loss.backward()
            e2.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1), e1.elapsed_time(e2), float(loss.detach()), mu.grad, b.grad

        for _ in range(max(W, 3)):   # warm-up sweeps (and the recorded-F ring) of one segment
            run(every)
        ms_fwd, ms_bwd, loss, gmu, gb = run(Ka)
        ms_fwd, ms_bwd = max_over_ranks(ms_fwd, world), max_over_ranks(ms_bwd, world)
        # the backward's two kernels alone: `every` recomputed steps recording F (one fused launch
        # each), then the reverse steps over them (one k_adj_step_tma launch each)
        ring = A._ring(sim, every)
        seed = ((sim.fields()[2] - u_tgt) * act_t).contiguous()
        e0, e1, e2, e3 = ev(), ev(), ev(), ev()
        e0.record(stream)
        for i in range(every):
            sim.step_moments(ring[i])
        e1.record(stream)
        sim.adjoint_begin(seed)
        e2.record(stream)
        for i in reversed(range(every)):
            sim.adjoint_step(ring[i])
        e3.record(stream)
        torch.cuda.synchronize()
        ms_rec = max_over_ranks(e0.elapsed_time(e1), world) / every
        ms_rev = max_over_ranks(e2.elapsed_time(e3), world) / every
        st_adj = sim.sync(raise_on_status=False)
        brev, brec = adjoint_bytes_per_node(3, 4), recompute_bytes_per_node(3, 4)
        gb_rev = nact_a * brev / (ms_rev / 1e3) / 1e9
        gb_rec = nact_a * brec / (ms_rec / 1e3) / 1e9
        kernels = {"reverse": {"kernel": "k_adj_step_tma<3>", "ms_per_launch": round(ms_rev, 4),
                               "bytes_per_node": brev, "achieved_GBps": round(gb_rev, 1),
                               "frac": round(gb_rev / peak, 4),
                               "traffic": captured_traffic(None, ADJ_TRAFFIC_CAPTURE, ADJ_SOURCES) if args.adj_n == 128 else None},
                   "recompute": {"kernel": "k_stream_collide_tma<3> recording F", "ms_per_launch": round(ms_rec, 4),
                                 "bytes_per_node": brec, "achieved_GBps": round(gb_rec, 1),
                                 "frac": round(gb_rec / peak, 4)},
                   "peak": peak, "peak_kind": peak_kind,
                   "note": f"CUDA events around {every} launches of each on the solver's stream"}
        del sim
        torch.cuda.empty_cache()
        # the FP64 form's reverse mode (the one held to central differences at 1e-4 on this workload),
        # over a shorter run: its backward time against its plain forward
        fp64_adj = None
        if not args.no_fp64:
            K64 = min(Ka, 3 * every)
            s64 = lbm.Simulation(pa, precision="fp64", device=dev, adjoint=True)
            s64.set_mu_field(pa.meta["mu_target"]).set_initial()
            s64.step(K64)
            u64_t = s64.fields()[2].clone()
            s64.set_mu_field(torch.ones(pa.box_shape, dtype=torch.float64, device=dev)).set_initial()
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record(s64.stream)
            s64.step(K64)
            e1.record(s64.stream)
            torch.cuda.synchronize()
            ms64_plain = e0.elapsed_time(e1)
            mu = torch.ones(pa.box_shape, dtype=torch.float64, device=dev, requires_grad=True)
            b = torch.tensor(pa.options.body_force, dtype=torch.float64, requires_grad=True)
            e0, e1, e2 = ev(), ev(), ev()
            e0.record(s64.stream)
            u = A.displacement(mu, b, s64, K64, every)
            e1.record(s64.stream)
            (0.5 * (((u - u64_t) ** 2) * act_t).sum()).backward()
            e2.record(s64.stream)
            torch.cuda.synchronize()
            fp64_adj = {"steps": K64, "forward_ms": round(ms64_plain, 2), "backward_ms": round(e1.elapsed_time(e2), 2),
                        "adjoint_over_forward": round(e1.elapsed_time(e2) / ms64_plain, 3),
                        "device_status": s64.sync(raise_on_status=False)}
            del s64
            torch.cuda.empty_cache()
        adj = {"workload": f"inclusion_cube_{args.adj_n}: D3Q6x12 FP32, clamped unit cube, target mu 2 inside "
                           "r = 0.25, parameter mu field (start 1) and body force, loss 1/2 |u(T) - u_target|^2",
               "n_active": nact_a, "steps": Ka, "checkpoint_every": every,
               "forward_MLUPS": round(nact_a * Ka / (ms_plain / 1e3) / 1e6, 2),
               "forward_ms": round(ms_plain, 2), "forward_with_saves_ms": round(ms_fwd, 2),
               "backward_ms": round(ms_bwd, 2), "adjoint_over_forward": round(ms_bwd / ms_plain, 3),
               "loss": loss, "grad_mu_norm": float(gmu.norm()), "grad_b": [float(x) for x in gb],
               "kernels": kernels, "fp64": fp64_adj,
               "device_status": st_adj,
               "note": "backward = recomputation from saved states recording F, then the reverse steps; "
                       "ratio over the plain forward of the same steps"}

    # ---- errors of the FP32 and FP64 forms against the oracle (64^3 copy, t = 1) -----------------
    errors = None
    if rank == 0 and not args.no_errors:
        errors = oracle_errors(64, 320, dev)
        torch.cuda.empty_cache()

    # ---- CPU baseline: the oracle on the host cores (rank 0, N = 1) ---------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        mlups, steps, el, nact64 = oracle_sample(n=64, budget_s=15.0, threads=cores)
        m1, s1, el1, _ = oracle_sample(n=64, steps=20, threads=1)
        cpu = {"value": round(mlups, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"FP64 C oracle, {cores} host threads (OpenMP over nodes and links), 64^3 copy of the "
                         f"shell ({nact64} active nodes), {steps} steps incl. projection steps, {el:.1f} s",
               "one_thread": {"value": round(m1, 4), "steps": s1, "seconds": round(el1, 1)}}

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": round(ms / K, 4), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"shell_3d_{args.n}: D3Q6x12 FP32 thick spherical shell, {args.n}^3 box, "
                                       "R_i=0.4 R_o=0.9, mu=1 lambda=5, internal pressure sin^2 ramp, "
                                       "projection every 20 steps",
                           "n_active": nact, "n_cut_links": info["n_cut"], "lsq_entries": info["lsq_entries"],
                           "n_windows": info["n_segments"],
                           "l2": "no flush: populations (2 x 4.8 GB) are far larger than the 126 MB L2",
                           "parallelism": f"replicas x{world}", "tuning": tuning},
                "roofline": roofline, "kernel_share_of_step": {k: round(v, 4) for k, v in share.items()},
                "jacobi": jacobi, "links": links, "errors_vs_oracle": errors,
                "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "fp64": fp64, "bf16": bf16, "batch_2d": batch,
                "adjoint": adj,
                "cpu_baseline": cpu, "device_status": st}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
