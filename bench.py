"""Benchmark of the fused monodomain step on GB300.

Workload: the 3D Barkley slab, 256 x 256 x 64 nodes, fibre angle rotating
linearly by 120 degrees through z, D_par = 1, D_perp = 0.25, h = 0.3,
dt = 0.005, 19-point anisotropic stencil, FP32 state, 8 seeded point stimuli.
One benchmark step is one explicit time step of the whole grid: stencil +
reaction + activation map + tissue total of V, all in one kernel launch.

  python bench.py [--gpus N --steps K --warmup W] [--impl bbx|reference]

value:  cell-updates/s with the state resident in HBM, device-timed with CUDA
        events around each step's launch; L2 is flushed between timed steps
        (a 256 MiB write, then a 256 MiB read so no dirty line of the flush is
        left for the step to write back), outside the events.
e2e:    the same metric through the C ABI with host buffers: every step
        writes u and v from pinned host memory, steps, and reads u and v back.
Under torchrun the slab is N times as high (64 N planes) and cut into N
z-slabs, one per rank (the paper's domain decomposition): every step each
rank exchanges its one-plane V halo with its neighbours (NCCL send/recv)
and steps its slab; weak scaling, value = all ranks' cells / slowest rank.
The batch of tissues is split over the ranks (independent units).
--impl reference times the FP64 CPU oracle on all host cores instead.
cpu_baseline: the same oracle on all host cores (OpenMP over the node loops)
and on one thread, on bounded samples of the slab.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD_DESC = ("3D Barkley slab 256x256x64, fibre angle rotating 120 deg through z, D_par=1 D_perp=0.25, "
                 "h=0.3, dt=0.005, a=0.75 b=0.02 eps=0.02, 19-point stencil, 8 seeded point stimuli")
METRIC = "cell-updates/s"


def kernel_source_hash():
    """Hash of the step kernel's sources (the device header and the per-model
    instantiations): DRAM counters taken on other sources do not apply."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1605_06015_gb300", "csrc")
    for p in sorted(glob.glob(os.path.join(csrc, "bbx_device.cuh")) + glob.glob(os.path.join(csrc, "step_*.cu"))):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def load_traffic(workload):
    """DRAM bytes per launch of the step kernel from a committed ncu summary,
    valid only while the kernel sources are unchanged."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("kernel_source_hash") == kernel_source_hash() and d.get("workload") == workload:
            return float(d["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
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
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cores():
    """Host cores this process may run on (the GPU machine's Grace cores)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_rate(w, steps, nz_sample=None, threads=1):
    """Oracle (FP64 CPU) cell-updates/s on a bounded sample: `steps` steps in
    one call on the first nz_sample planes of the slab, its node loops on
    `threads` OpenMP threads (bit-identical results for any count)."""
    import oracle
    from paper_1605_06015_gb300 import workloads as wl
    if nz_sample is not None and nz_sample < w.nz:
        w = wl.barkley_slab(w.nx, w.ny, nz_sample)
    used = oracle.set_threads(threads)
    try:
        og = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
        st = w.initial_state(oracle.rest_state(w.model, w.params))
        sim = oracle.Sim(og, w.model, par=w.params, state=st)
        t0 = time.perf_counter()
        sim.step(w.dt, steps)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    return w.n_active() * steps / dt, dt, w, used


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws == 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, local, dist


def max_over_ranks(x, dist, dev=None):
    """The largest of the ranks' values of x (x itself on one rank): timings
    are combined by taking the slowest rank."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, steps, ws, seconds):
    """Units all ranks processed per second of the slowest rank."""
    return units_per_rank * steps * ws / seconds


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on all host cores
    (OpenMP node loops), one oracle call of one step of the full slab per
    benchmark step (the call builds the stencil weights, then steps)."""
    rank, ws, local, dist = dist_setup()
    if rank != 0:
        return 0
    from paper_1605_06015_gb300 import workloads as wl
    w = wl.barkley_slab()
    cores = host_cores()
    times = []
    used = 1
    for i in range(args.warmup + args.steps):
        rate, dt, _, used = oracle_rate(w, 1, threads=cores)
        if i >= args.warmup:
            times.append(dt)
    T = sum(times)
    value = w.n_active() * args.steps / T
    sample = "one oracle call of 1 step of the full 256x256x64 slab per benchmark step, %d threads" % used
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD_DESC, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": used, "kind": "oracle",
                             "sample": sample, "nproc": cores},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_e2e(G, w, st0, S, args, dist, dev, ws, n_tissue, step_fn=None):
    """Steps through the C ABI with host buffers: every step takes a new
    whole state from pinned host memory while the previous step's result goes
    back to pinned host memory, then steps once; the last step's result is
    read after the loop, inside the timed region.  The exchange is
    bbx_exchange_state_async (each step's two copies overlap each other and
    the neighbouring steps; one wait at the end), or bbx_exchange_state where
    the grid's rows are padded."""
    import torch
    from paper_1605_06015_gb300 import bbx
    step = step_fn or (lambda: G.step(w.dt, 1))
    pin_in = torch.from_numpy(st0[:S].copy()).pin_memory()
    pin_out = torch.empty(pin_in.shape, dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    mode = "async"
    try:
        G.exchange_state_async(pin_in, pin_out)
        G.exchange_wait()
    except bbx.BbxError as e:
        if e.code != bbx.BBX_ERR_UNSUPPORTED:
            raise
        mode = "sync"
    exchange = G.exchange_state_async if mode == "async" else G.exchange_state
    for _ in range(2):
        exchange(pin_in, pin_out)
        step()
    G.exchange_wait()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0 = time.perf_counter()
    for _ in range(e2e_steps):
        exchange(pin_in, pin_out)
        step()
    G.exchange_wait()
    G.read_all(out=pin_out)
    torch.cuda.synchronize()
    e_wall = time.perf_counter() - e0
    e_wall = max_over_ranks(e_wall, dist, dev)
    e2e_value = whole_job_rate(n_tissue, e2e_steps, ws, e_wall)
    bytes_io = S * w.n_cells * 4
    return {"value": e2e_value, "unit": "cell-updates/s", "h2d_bytes_per_step": bytes_io,
            "d2h_bytes_per_step": bytes_io, "steps": e2e_steps, "exchange": mode}

def initial_state(G, w):
    """The workload's initial condition on top of the library's own rest
    state (every node holds it right after bbx_set_ionic_model)."""
    import numpy as np
    rest = [float(G.read_state(v).reshape(-1)[0]) for v in range(G.get_info()["nvars"])]
    return w.initial_state(rest).astype(np.float32)


def partition_tissues(cells, n_ranks):
    """Split independent tissues (their node counts) over ranks, largest
    first to the least loaded rank; returns each rank's tissue indices.  The
    tissues are independent units of work, so no data crosses ranks."""
    load = [0] * n_ranks
    out = [[] for _ in range(n_ranks)]
    for i in sorted(range(len(cells)), key=lambda k: (-cells[k], k)):
        r = min(range(n_ranks), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += cells[i]
    return [sorted(o) for o in out]


def run_batched(args, dev, stream, dist=None, n_ranks=1):
    """The batch of 256 independent tissues (192 FHN sheets with sides in
    64..512, 64 Barkley blocks with sides in 64..128, parameters swept by
    +-20%): cell-updates/s of batched, graph-replayed steps against the same
    grids stepped one launch per grid."""
    import numpy as np
    import torch
    from paper_1605_06015_gb300 import bbx
    from paper_1605_06015_gb300 import workloads as wl
    ws_all = wl.tissue_batch(n2d=args.batch_2d, n3d=args.batch_3d)
    rank = dist.get_rank() if dist else 0
    share = partition_tissues([w.n_cells for w in ws_all], n_ranks)[rank]
    ws = [ws_all[i] for i in share]  # this rank's tissues
    cells_all = sum(w.n_cells for w in ws_all)
    grids = []
    for w in ws:
        G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask, stream=stream)
        G.set_fibres(None, w.D_par, w.D_par)
        G.set_ionic_model(w.model, w.params)
        G.set_threshold(w.theta)
        G.set_timestep(w.dt)
        G.write_all(initial_state(G, w))
        grids.append(G)
    cells = sum(w.n_cells for w in ws)
    B = bbx.Batch(grids)
    B.autotune()
    K = args.batch_steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    B.step(16)  # warm-up and graph capture
    torch.cuda.synchronize()
    e0.record(stream)
    B.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    B.sync()
    t_batch = max_over_ranks(e0.elapsed_time(e1) * 1e-3, dist, dev)
    for G, w in zip(grids, ws):
        G.step(w.dt, 2)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(K):
        for G, w in zip(grids, ws):
            G.step(w.dt, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    t_solo = max_over_ranks(e0.elapsed_time(e1) * 1e-3, dist, dev)
    info = B.info()
    B.close()
    for G in grids:
        G.close()
    return {"workload": "%d 2D FHN sheets (sides 64..512) + %d 3D Barkley blocks (sides 64..128), D and model "
                        "parameters swept +-20%%, isotropic" % (args.batch_2d, args.batch_3d),
            "cells": cells_all, "cells_this_rank": cells, "tissues_this_rank": len(ws),
            "partition": "tissues split over %d rank(s), largest first to the least loaded" % n_ranks,
            "steps": K, "value": cells_all * K / t_batch, "unit": "cell-updates/s",
            "one_launch_per_grid_value": cells_all * K / t_solo,
            "speedup_vs_one_launch_per_grid": t_solo / t_batch,
            "groups": info["n_groups"], "tile_y": info["tile_y"], "graph_steps_per_replay": 16}


def run_surrogate(args, dev, stream, dist=None, n_ranks=1):
    """The 256x256x64 rotating-fibre slab with Beeler-Reuter physics and the
    reaction surrogate: 10^7 (state, one-step reaction increment) pairs sampled
    from a plain run, the network trained on the GPU, then the same number of
    steps from the same initial state with the exact model and with the
    surrogate (exact model in the upstroke and outside the envelope):
    cell-updates/s of each and the difference of their activation maps.  The
    state (8 variables, two buffers, 268 MB) is larger than L2."""
    import numpy as np
    import torch
    from paper_1605_06015_gb300 import bbx
    from paper_1605_06015_gb300 import workloads as wl
    w = wl.br_slab(256, 256, 64)

    st0 = []

    def grid():
        G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask, stream=stream)
        G.set_fibres(w.fibres, w.D_par, w.D_perp)
        G.set_ionic_model(w.model, w.params)
        G.set_threshold(w.theta)
        G.set_timestep(w.dt)
        if not st0:
            st0.append(initial_state(G, w))  # on the rest state the grid starts from
        G.write_all(st0[0])
        return G

    n_pairs, chunks, traj = args.surrogate_pairs, 50, args.surrogate_traj_steps
    per = n_pairs // chunks
    X = torch.empty((per * chunks, 8), dtype=torch.float32, device=dev)
    T = torch.empty_like(X)
    G = grid()
    for k in range(chunks):
        bbx.bbx_sample_reaction_pairs(G.g, per, 5000 + k, X[k * per:(k + 1) * per], T[k * per:(k + 1) * per])
        G.step(w.dt, traj // chunks)
    G.close()
    m = bbx.bbx_mlp_create(11, stream=stream)
    bbx.bbx_mlp_fit_normalization(m, X, T, X.shape[0])
    l0 = bbx.bbx_mlp_train(m, X, T, X.shape[0], 4096, 1, 1e-3, seed=12)
    t0 = time.perf_counter()
    l1 = bbx.bbx_mlp_train(m, X, T, X.shape[0], 4096, args.surrogate_train_steps, 1e-3, seed=13)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del X, T
    K = args.surrogate_steps
    res = {}
    acts = {}
    v_ups = [float(v) for v in args.v_upstroke.split(",")]
    for name in ["exact"] + ["surrogate@%g" % v for v in v_ups]:
        G = grid()
        if name != "exact":
            bbx.bbx_set_surrogate(G.g, m, float(name.split("@")[1]))
        G.autotune(w.dt)
        G.write_all(st0[0])
        G.write_activation(np.full(w.shape, bbx.BBX_ACT_NONE, dtype=np.int32))
        G.set_time(0.0, 0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.step(w.dt, K)
        e1.record(stream)
        torch.cuda.synchronize()
        secs = max_over_ranks(e0.elapsed_time(e1) * 1e-3, dist, dev)
        res[name] = whole_job_rate(w.n_cells, K, n_ranks, secs)
        acts[name] = G.read_activation().astype(np.int64)
        G.close()
    bbx.bbx_mlp_destroy(m)
    a = acts["exact"]
    runs = []
    for v in v_ups:
        name = "surrogate@%g" % v
        b = acts[name]
        both = (a != bbx.BBX_ACT_NONE) & (b != bbx.BBX_ACT_NONE)
        diff = np.abs(a - b)[both]
        runs.append({"v_upstroke_mV": v, "value": res[name], "over_exact": res[name] / res["exact"],
                     "activated": int((b != bbx.BBX_ACT_NONE).sum()),
                     "activation_max_abs_diff_steps": int(diff.max()) if diff.size else None,
                     "activation_frac_within_1_step": float((diff <= 1).mean()) if diff.size else None})
    return {"workload": "BR slab 256x256x64 (rotating fibres, D_par=0.1 D_perp=0.025, h=0.2, dt=0.02), "
                        "MLP 8-64-64-8 BF16/FP32, exact model where V >= v_upstroke or outside the envelope",
            "training_pairs": per * chunks, "trajectory_steps": traj, "train_steps": args.surrogate_train_steps,
            "train_batch": 4096, "loss_first": l0, "loss_last": l1, "train_s": t_train, "steps": K,
            "exact_value": res["exact"], "unit": "cell-updates/s",
            "activated_exact": int((a != bbx.BBX_ACT_NONE).sum()), "surrogate_runs": runs}


def run_configs(args, dev, stream, dist=None, n_ranks=1):
    """The other workload shapes, each timed by differencing two back-to-back
    runs of N1 and N2 steps (fixed launch costs cancel): cell-updates/s and
    the fraction of the measured HBM bandwidth the algorithmic bytes imply.
    The 200x200 sheet is L2-resident (latency-bound); the 16384^2 sheet, the
    512x512x256 slab and the 512^3 shell are larger than L2."""
    import numpy as np
    import torch
    from paper_1605_06015_gb300 import bbx
    from paper_1605_06015_gb300 import workloads as wl
    peak, _ = load_peaks()
    makers = {
        "fhn_200": (lambda: wl.fhn_sheet(200, 200), (100, 1100),
                    "2D FitzHugh-Nagumo 200x200, h=0.5, dt=0.01, D=1, 5-point, cross-field IC"),
        "fhn_16384": (lambda: wl.fhn_sheet(16384, 16384), (2, 12),
                      "2D FitzHugh-Nagumo 16384x16384, same physics (roofline figure)"),
        "barkley_512x512x256": (lambda: wl.barkley_slab(512, 512, 256), (2, 22),
                                "3D Barkley slab 512x512x256, rotating fibres, 19-point"),
        "br_shell_512": (lambda: wl.br_shell(512), (2, 22),
                         "Beeler-Reuter ellipsoidal shell in 512^3 (14 % tissue), helical fibres, masked 19-point"),
        "br_256x256x64": (lambda: wl.br_slab(256, 256, 64), (2, 22),
                          "Beeler-Reuter slab 256x256x64, rotating fibres, 19-point, Rush-Larsen gates"),
        "br_mrl_256x256x64": (lambda: wl.br_mrl_slab(256, 256, 64), (2, 22),
                              "the same slab with the sodium activation as a 4-state Markov chain, "
                              "matrix Rush-Larsen with T(V) tabulated"),
        "br_fca_256x256x64": (lambda: wl.br_fca_slab(256, 256, 64), (2, 22),
                              "the same slab with the slow inward current's inactivation as a voltage gate and "
                              "a calcium gate (4-state chain, A(V, Ca) split into univariate parts)"),
        "br_fca_256x256x64_onfly": (lambda: wl.br_fca_slab(256, 256, 64, onfly=True), (2, 22),
                                    "the calcium-gated slab with the channel by exp(dt A(V, Ca)) of the whole "
                                    "generator at run time (no table, no splitting)"),
        "br_shell_256": (lambda: wl.br_shell(256), (2, 22),
                         "Beeler-Reuter shell in 256^3 (profiling size, not in the default list)"),
        "br_256x256x64_tab": (lambda: wl.br_slab(256, 256, 64), (2, 22),
                              "Beeler-Reuter slab 256x256x64, Rush-Larsen coefficients tabulated in V"),
        "br_shell_512_tab": (lambda: wl.br_shell(512), (2, 22),
                             "Beeler-Reuter shell in 512^3, Rush-Larsen coefficients tabulated in V"),
        "br_shell_512_u16": (lambda: wl.br_shell(512), (2, 22),
                             "Beeler-Reuter shell in 512^3, the six gates stored as 16-bit fixed point"),
        "br_shell_512_f16": (lambda: wl.br_shell(512), (2, 22),
                             "Beeler-Reuter shell in 512^3, the six gates stored as binary16"),
        "br_256x256x64_u16": (lambda: wl.br_slab(256, 256, 64), (2, 22),
                              "Beeler-Reuter slab 256x256x64, the six gates stored as 16-bit fixed point"),
        "br_shell_512_tab_u16": (lambda: wl.br_shell(512), (2, 22),
                                 "Beeler-Reuter shell in 512^3, Rush-Larsen coefficients tabulated, the six gates "
                                 "stored as 16-bit fixed point (not in the default list)"),
        "br_256x256x64_tab_u16": (lambda: wl.br_slab(256, 256, 64), (2, 22),
                                  "Beeler-Reuter slab 256x256x64, Rush-Larsen coefficients tabulated, the six gates "
                                  "stored as 16-bit fixed point (not in the default list)"),
    }
    out = {}
    for name in args.configs.split(","):
        if not name:
            continue
        make, (n1, n2), desc = makers[name]
        w = make()
        G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask, stream=stream)
        G.set_fibres(w.fibres, w.D_par, w.D_perp)
        G.set_ionic_model(w.model, w.params)
        G.set_threshold(w.theta)
        G.set_timestep(w.dt)
        if name.endswith("_tab") or "_tab_" in name:
            G.set_tabulation(True)
        st = initial_state(G, w)
        gates = {"_u16": bbx.BBX_GATES_UNORM16, "_f16": bbx.BBX_GATES_FP16}.get(name[-4:], bbx.BBX_GATES_FP32)
        if gates != bbx.BBX_GATES_FP32:
            G.set_gate_storage(gates)
        if args.config_tile:
            G.set_tiling(*(int(v) for v in args.config_tile.split(",")))
        else:
            G.autotune(w.dt)
        G.write_all(st)
        del st
        resident = False
        if name == "fhn_200":
            G.set_resident(True)  # the whole sheet in the shared memory of one CTA cluster
            resident = True
        info = G.get_info()
        cells = info["n_tissue"]
        S = info["nvars"]
        state_bytes = S * 4 if gates == bbx.BBX_GATES_FP32 else 2 * 4 + 6 * 2  # V, Ca + six 16-bit gates
        b_alg = 2 * state_bytes + (12 if info["anisotropic"] else 0) + (1 if info["masked"] else 0)
        G.step(w.dt, 2)
        secs = []
        for n in (n1, n2):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G.step(w.dt, n)
            e1.record(stream)
            torch.cuda.synchronize()
            secs.append(max_over_ranks(e0.elapsed_time(e1) * 1e-3, dist, dev))
        G.step_total()  # synchronising call: reports any device error of the runs
        rate = whole_job_rate(cells, n2 - n1, n_ranks, secs[1] - secs[0])
        out[name] = {"workload": desc, "active_cells": cells, "steps": [n1, n2], "value": rate,
                     "unit": "cell-updates/s", "ms_per_step": 1e3 * (secs[1] - secs[0]) / (n2 - n1),
                     "bytes_per_cell": b_alg, "roofline_frac": rate * b_alg / (peak * 1e9),
                     "tile": [info["tile_x"], info["tile_y"], info["tile_z"]], "resident": resident}
        G.close()
        del w
    return out


def run_output(args, dev, stream, G, w, n_tissue):
    """The headless output kernels, device-timed, L2 flushed (write, then read)
    before each call:
    on the bench slab the sample script's colour map as a byte frame (red = u,
    green = v: two float layers read, three bytes written per node), and the
    phase singularities of (u, v) (8 B per node) on the same slab started from
    a cross-field condition (u = 1 where x < nx/2, v = 0.5 where y < ny/2,
    every z) and stepped until the broken front has curled into a scroll wave
    whose filament crosses every z cross-section."""
    import numpy as np
    import torch
    from paper_1605_06015_gb300 import bbx
    peak, _ = load_peaks()
    frame = torch.empty(3 * w.n_cells, dtype=torch.uint8, device=dev)
    xyz = torch.empty(3 * 65536, dtype=torch.float32, device=dev)
    # L2 flush before each call as in the step timing: a 256 MiB write, then a
    # 256 MiB read, so that no dirty line of the flush is left for the timed
    # kernel to write back
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flush_rd = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)
    # the scroll-wave state
    S = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask, stream=stream)
    S.set_fibres(w.fibres, w.D_par, w.D_perp)
    S.set_ionic_model(w.model, w.params)
    st = np.zeros((2,) + w.shape, np.float32)
    st[0, :, :, : w.nx // 2] = 1.0
    st[1, :, : w.ny // 2, :] = 0.5
    S.write_all(st)
    S.step(w.dt, args.scroll_steps)
    layers = (0, 1, -1)
    res = {}
    for name, grid in (("ppm_frame", G), ("phase_singularities", S)):
        ts, found = [], 0
        for i in range(12):
            # the flush is still running when the call is enqueued, so the
            # events see the device time of the call, not the host's latency
            # (the singularity call still waits for its 4-byte count)
            flush.fill_(float(i))
            torch.sum(flush_rd, dim=0, out=sink)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if name == "ppm_frame":
                grid.ppm_frame(layers, (0.0, 0.0, 0.0), (1.0, 0.8, 1.0), frame)
            else:
                found = grid.phase_singularities(0, 0.5, 1, 0.3, xyz, 65536)
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= 2:
                ts.append(e0.elapsed_time(e1) * 1e-3)
        sec = sum(ts) / len(ts)
        if name == "ppm_frame":
            b = 4 * sum(1 for c in layers if c >= 0) + 3 + (1 if w.mask is not None else 0)
        else:
            b = 8 + (1 if w.mask is not None else 0)
        res[name] = {"us_per_call": sec * 1e6, "bytes_per_node": b, "GB_s": b * w.n_cells / sec / 1e9,
                     "roofline_frac": b * w.n_cells / sec / 1e9 / peak}
        if name != "ppm_frame":
            res[name]["points"] = found
            res[name]["state"] = "scroll wave: cross-field start, %d steps" % args.scroll_steps
        else:
            res[name]["layers"] = list(layers)
    S.close()
    return res


def run_bbx(args):
    import numpy as np
    import torch
    rank, ws, local, dist = dist_setup()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1605_06015_gb300 import bbx
    from paper_1605_06015_gb300 import workloads as wl

    stream = torch.cuda.current_stream()
    slab = None
    if ws == 1:
        w = wl.barkley_slab()
        G = bbx.Grid(w.nx, w.ny, w.nz, w.h, w.mask, stream=stream)
        G.set_fibres(w.fibres, w.D_par, w.D_perp)
        G.set_ionic_model(w.model, w.params)
        G.set_threshold(w.theta)
        st0 = initial_state(G, w)
        G.write_all(st0)
    else:
        # N ranks: the slab 64 N planes high, cut into N z-slabs of 64 planes
        # (the paper's domain decomposition), each rank's halo planes
        # refreshed from its neighbours by NCCL sends and receives every step
        from paper_1605_06015_gb300 import slabs
        w = wl.barkley_slab(256, 256, 64 * ws)
        slab = slabs.SlabGrid(w, ws, rank, stream=stream, device=dev)
        G = slab.G
        rest = [float(G.read_state(v).reshape(-1)[0]) for v in range(G.get_info()["nvars"])]
        st_global = w.initial_state(rest).astype(np.float32)
        slab.write_global_state(st_global)
        st0 = np.ascontiguousarray(st_global[:, slab.a:slab.b])
        del st_global
    if args.tile:
        ty, tz = (int(v) for v in args.tile.split(","))
        G.set_tiling(ty, tz)
        tune_ms = None
    else:
        tune_ms = G.autotune(w.dt)
    info = G.get_info()
    n_tissue = info["n_tissue"]
    S = info["nvars"]
    B_alg = 2 * S * 4 + (12 if info["anisotropic"] else 0) + (1 if info["masked"] else 0)

    # L2 (129 MB) flush between timed steps: write a 256 MiB buffer, then read
    # another 256 MiB buffer so the flush's dirty lines are written back
    # before the timed step starts (both outside the events)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flush_rd = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)

    def flush_l2(val):
        flush.fill_(val)
        torch.sum(flush_rd, dim=0, out=sink)

    def one_step():
        if slab is not None:
            slab.exchange(dist, rank, ws)
        G.step(w.dt, 1)

    for _ in range(args.warmup):
        flush_l2(1.0)
        one_step()
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush_l2(float(i))
        starts[i].record(stream)
        one_step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    dev_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    total_v = G.step_total()
    dev_ms = max_over_ranks(dev_ms, dist, dev)
    ms_step = dev_ms / args.steps
    value = whole_job_rate(n_tissue, args.steps, ws, dev_ms * 1e-3)

    # A/B on the same grid: the flushed step with the W-tilde sums loaded
    # although they all vanish (the library skips them by default)
    wsum_loaded = None
    if ws == 1 and info["wsum_skipped"]:
        G.set_wsum_elision(False)
        for _ in range(args.warmup):
            flush_l2(1.0)
            one_step()
        ab = []
        for i in range(args.steps):
            flush_l2(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_step()
            e1.record(stream)
            ab.append((e0, e1))
        torch.cuda.synchronize()
        ab_ms = sum(a.elapsed_time(b) for a, b in ab) / args.steps
        G.set_wsum_elision(True)
        G.step_total()  # synchronising call: reports any device error of the runs
        wsum_loaded = {"ms_per_step": ab_ms, "value": n_tissue / (ab_ms * 1e-3), "unit": "cell-updates/s",
                       "note": "same grid and timing with the vanishing W-tilde sums (12 B per node) loaded"}

    e2e = None if args.no_e2e else run_e2e(G, w, st0, S, args, dist, dev, ws, n_tissue, one_step)


    batched = None
    if not args.no_batched:
        batched = run_batched(args, dev, stream, dist, ws)
    output = run_output(args, dev, stream, G, w, n_tissue)
    configs = None
    if args.configs:
        configs = run_configs(args, dev, stream, dist, ws)
    surrogate = None
    if not args.no_surrogate:
        surrogate = run_surrogate(args, dev, stream, dist, ws)
    peak, peak_kind = load_peaks()
    achieved = B_alg * n_tissue / (ms_step * 1e-3) / 1e9
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = host_cores()
        rate1, secs1, _, _ = oracle_rate(w, args.cpu_steps, threads=1)
        ratep, secsp, _, used = oracle_rate(w, args.cpu_steps_parallel, threads=cores)
        cpu = {"value": ratep, "unit": "cell-updates/s", "cores": used, "kind": "oracle", "nproc": cores,
               "sample": "%d steps of the full 256x256x64 slab in one oracle call on %d threads (%.1f s, "
                         "weights built once per call)" % (args.cpu_steps_parallel, used, secsp),
               "single_thread": {"value": rate1, "unit": "cell-updates/s", "cores": 1,
                                 "sample": "%d steps of the full slab in one oracle call on 1 thread (%.1f s)"
                                           % (args.cpu_steps, secs1)}}
    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD_DESC, "active_cells": n_tissue, "l2": "flushed between timed steps "
                   "(256 MiB write then 256 MiB read, outside the events)", "tile": [info["tile_x"], info["tile_y"], info["tile_z"]],
                   "parallelism": ("z-slabs of a 256x256x%d slab, one per rank, one-plane V halo exchanged by NCCL "
                                   "send/recv every step (inside the timed region)" % (64 * ws)) if ws > 1
                                  else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": load_traffic("barkley_slab_256x256x64"), "peak_kind": peak_kind,
                     "bytes_per_cell": B_alg, "wsum_skipped": bool(info["wsum_skipped"]),
                     "wsum_loaded": wsum_loaded},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "batched": batched,
        "surrogate": surrogate,
        "configs": configs,
        "output_kernels": output,
        "gpu_launches": args.steps,
        "clocks": clk,
        "tissue_total_V": total_v,
        "autotune_ms_per_step": tune_ms,
        "wall_s_timed": wall,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if slab is not None:
        slab.close()
    else:
        G.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="bbx", choices=["bbx", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=20)
    ap.add_argument("--cpu-steps-parallel", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-2d", type=int, default=192)
    ap.add_argument("--batch-3d", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=48)
    ap.add_argument("--tile", default=None, help="TY,TZ brick shape instead of autotuning")
    ap.add_argument("--config-tile", default=None, help="TY,TZ brick shape of the --configs workloads instead of autotuning")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--configs", default="fhn_200,fhn_16384,barkley_512x512x256,br_shell_512,br_256x256x64,"
                            "br_mrl_256x256x64,br_fca_256x256x64,br_fca_256x256x64_onfly,"
                            "br_256x256x64_tab,br_shell_512_tab,br_shell_512_u16,br_shell_512_f16,br_256x256x64_u16",
                    help="comma-separated other workloads to time by differencing ('' for none)")
    ap.add_argument("--scroll-steps", type=int, default=2000)
    ap.add_argument("--surrogate-pairs", type=int, default=10_000_000)
    ap.add_argument("--surrogate-traj-steps", type=int, default=6000)
    ap.add_argument("--surrogate-train-steps", type=int, default=4000)
    ap.add_argument("--surrogate-steps", type=int, default=3000)
    ap.add_argument("--v-upstroke", default="-60,-75", help="comma-separated upstroke thresholds (mV)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_bbx(args)


if __name__ == "__main__":
    sys.exit(main())
