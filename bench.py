"""Benchmark of the fused stream-and-collide sweep: supersonic Taylor-Green vortex at 256^3.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 256]

One bench step = one pass of the whole hot path over one batch of synthetic input: the
Taylor-Green initial field (M0 = 1.25, Re = 1600, Pr = 0.71, Sutherland, regularized collision
with the compression sensor, FP32 populations) is turned into populations on the device
(init kernel), then advanced by 50 time steps = 49 plain sweeps + 1 diagnostic sweep with FP64
reductions (+ its fixed-order finalize).  Every step restarts from the initial field, so each
timed step does the same work on the same flow.  MLUP/s = 50 * N / step time.

`value` is device-timed with the inputs resident in HBM; `e2e` is the same metric through the
public C ABI with host (pinned) buffers: every step uploads the host FP64 fields
(grlb_stage_primitive, overlapped with the previous step's sweeps on a copy stream),
initialises from them (grlb_init_from_stage), runs the 50 sweeps and reads the diagnostics back.
Working set 4.7 GB >> 126 MB L2, so no L2 flush.

N > 1 (torchrun): every rank runs its own replica domain (weak scaling, no collective on the
data path); barrier + max-over-ranks time.

--impl reference times the FP64 CPU oracle on the machine's host cores on a bounded slab of the
same workload (one oracle sweep of 256 x 256 x 16 cells per step).
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SWEEPS_PER_STEP = 50
# collision readings: name -> (grlb_collision, kernel label)
COLLISIONS = {"rlb": (1, "RLB"), "gated": (2, "RLB_GATED"), "bgk": (0, "BGK")}
BYTES_PER_LUP = {0: 280, 1: 140, 2: 140}
# moment storage (regularized collision): 20 FP32 values per cell read and written
BYTES_PER_LUP_MOMENTS = 160
KERNEL_SOURCES = ["paper_2609_16361_b300/csrc/grlb_device.cuh", "paper_2609_16361_b300/csrc/grlb_check.cuh",
                  "paper_2609_16361_b300/csrc/grlb_kernels.cu"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max_over_ranks(values, ws, device):
    """Element-wise maximum of per-rank values (timings) over all ranks; the identity at N = 1."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_mlups(ws, cells_per_rank, sweeps, seconds):
    """Whole-job throughput: the cell updates of all ranks over the slowest rank's time."""
    return ws * cells_per_rank * sweeps / seconds / 1e6


def code_lines(text):
    """The code of a CUDA source: `//` comments, trailing blanks and empty lines dropped (the
    kernel sources hold no block comments and no `//` inside string literals)."""
    out = []
    for line in text.splitlines():
        line = line.split("//", 1)[0].rstrip()
        if line:
            out.append(line)
    return "\n".join(out)


def kernel_source_sha(sources=None, read=None):
    """Key of the counter records: a hash of the kernel sources' code, so a record stays valid
    across comment edits and is dropped by any change to the code.  `read(path)` returns a
    file's text (default: the working tree)."""
    h = hashlib.sha256()
    for p in KERNEL_SOURCES if sources is None else sources:
        text = read(p) if read else open(os.path.join(ROOT, p), encoding="utf-8").read()
        h.update(code_lines(text).encode())
        h.update(b"\0")
    return h.hexdigest()[:16]


# the spectral post-processing's five kernels and the sweep header they include
SPECTRAL_SOURCES = ["paper_2609_16361_b300/csrc/grlb_device.cuh", "paper_2609_16361_b300/csrc/grlb_check.cuh",
                    "paper_2609_16361_b300/csrc/grlb_spectral.cu"]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def instructions_per_cell(storage):
    """Warp instructions per cell of the plain sweep (ncu smsp__inst_executed.sum / cells),
    recorded in the traffic file for the current kernel source; None when stale or absent."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    rec = json.load(open(TRAFFIC_FILE)).get(f"inst_{storage}")
    if rec and rec.get("source_sha") == kernel_source_sha():
        return float(rec["warp_inst_per_cell"])
    return None


def ffma_issue_rate(stream, iters=2048, reps=5):
    """FFMA warp instructions per second of the device (grlb_ffma_probe, 8 CTAs of 256
    threads per SM, median of `reps` event-timed launches after 3 warm-up launches): the
    instruction-issue ceiling of a kernel whose arithmetic is FP32."""
    import torch
    from paper_2609_16361_b300 import capi
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    ctas = 8 * sms
    sink = torch.zeros(ctas * 256, device="cuda")
    torch.cuda.synchronize()
    for _ in range(3):
        capi.grlb_ffma_probe(ctas, iters, sink.data_ptr(), stream.cuda_stream)
    times = []
    count = 0.0
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        count = capi.grlb_ffma_probe(ctas, iters, sink.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return count / statistics.median(times)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------
def cpu_oracle_sample(n, steps, slab=16, min_seconds=0.0):
    """Time sweeps of the FP64 oracle on an n x n x slab piece of the n^3 workload: `steps`
    sweeps, continued until at least `min_seconds` of CPU work has been timed."""
    import oracle
    from paper_2609_16361_b300 import inputs
    c = inputs.tgv3d(n, nxyz=(n, n, slab))
    o = oracle.Oracle(c.params)
    o.init_primitive(c.rho, c.u, c.p)
    t0 = time.perf_counter()
    o.step(steps)
    while time.perf_counter() - t0 < min_seconds and steps < 400:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    cells = c.params.ncells
    return {"value": cells * steps / dt / 1e6, "unit": "MLUP/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{steps} FP64 oracle sweep(s) of a {n}x{n}x{slab} slab of the {n}^3 "
                      f"Taylor-Green workload (same per-cell parameters)"}, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n = args.n
    for _ in range(args.warmup):
        cpu_oracle_sample(n, 1)
    times = []
    base = None
    for _ in range(args.steps):
        base, dt = cpu_oracle_sample(n, 1)
        times.append(dt)
    cells = n * n * 16
    total = sum(times)
    value = cells * len(times) / total / 1e6
    base["value"] = value
    line = {"impl": "reference", "metric": "MLUP/s", "value": value, "unit": "MLUP/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"tgv{n}_f32_rlb (oracle: FP64, bounded slab)",
                       "grid": [n, n, 16], "sweeps_per_step": 1},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "MLUP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2609_16361_b300 import capi, inputs

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}), flush=True)
        return 1
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    n = args.n
    storage = {"f32": 0, "f16": 1, "bf16": 2}[args.storage]
    coll, coll_label = COLLISIONS[args.collision]
    case = inputs.tgv3d(n, storage=storage, collision=coll)
    moments = args.state == "moments" or (args.state == "auto" and storage == 0 and args.collision == "rlb")
    if moments:
        if storage != 0 or args.collision != "rlb":
            print(json.dumps({"error": "--state moments needs --storage f32 --collision rlb"}), flush=True)
            return 1
        case = dataclasses.replace(case, params=case.params.replace(streaming=2))
    N = case.params.ncells
    dev = torch.device("cuda", local)
    rho_d = torch.from_numpy(case.rho).to(dev)
    u_d = torch.from_numpy(case.u).to(dev).contiguous()
    p_d = torch.from_numpy(case.p).to(dev)
    dom = capi.Domain(case.params, stream=stream.cuda_stream)
    h = dom.h

    def one_step(ev=None):
        capi.grlb_init_primitive_device(h, rho_d.data_ptr(), u_d.data_ptr(), p_d.data_ptr())
        if ev is not None:
            ev[0].record(stream)
        capi.grlb_step(h, SWEEPS_PER_STEP - 1)
        if ev is not None:
            ev[1].record(stream)
        capi.grlb_step_diag(h)

    def barrier():
        if ws > 1:
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
        stream.synchronize()
        barrier()
        torch.cuda.synchronize()
        kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            t0.record(stream)
            for k in range(args.steps):
                one_step(kev[k])
            t1.record(stream)
            stream.synchronize()
        torch.cuda.synchronize()
        barrier()
        ms = t0.elapsed_time(t1)
        sweep_ms = [a.elapsed_time(b) / (SWEEPS_PER_STEP - 1) for a, b in kev]
        diag = dom.diag()
        clocks = clk.summary()

        # ---- end to end through the public C ABI with pinned host buffers ---------------
        rho_h = torch.from_numpy(case.rho).pin_memory()
        u_h = torch.from_numpy(case.u).pin_memory()
        p_h = torch.from_numpy(case.p).pin_memory()
        rho_np, u_np, p_np = rho_h.numpy(), u_h.numpy(), p_h.numpy()
        # a pipelined job of as many steps as the timed region: the first upload has no sweeps
        # to hide behind, later ones do
        e2e_steps = max(2, args.steps)

        # pipelined: the upload of step k+1's fields (copy stream) overlaps step k's sweeps
        def e2e_run(nsteps):
            capi.grlb_stage_primitive(h, rho_np, u_np, p_np)
            for k in range(nsteps):
                capi.grlb_init_from_stage(h)
                if k + 1 < nsteps:
                    capi.grlb_stage_primitive(h, rho_np, u_np, p_np)
                capi.grlb_step(h, SWEEPS_PER_STEP - 1)
                capi.grlb_step_diag(h)
                capi.grlb_diag_read(h)

        e2e_run(1)
        barrier()
        torch.cuda.synchronize()
        te0 = time.perf_counter()
        e2e_run(e2e_steps)
        torch.cuda.synchronize()
        te = time.perf_counter() - te0
        barrier()

        # ---- diagnostics of the same flow after a Chapman-Enskog start (outside the timed
        # region): with omega -> 2 the equilibrium start of the timed steps leaves a
        # non-equilibrium part that flips sign every step, so the cell-local dissipation of
        # their diagnostic sweep is not the flow's; this start carries the gradients from step 0
        capi.grlb_set_init_mode(h, 1)
        capi.grlb_init_primitive_device(h, rho_d.data_ptr(), u_d.data_ptr(), p_d.data_ptr())
        capi.grlb_step(h, SWEEPS_PER_STEP - 1)
        capi.grlb_step_diag(h)
        ce_diag = dom.diag(allow_nonfinite=True)
        _, ce_spec = dom.spectral(nbins=0) if ce_diag["n_nan"] == 0 else (None, None)
        capi.grlb_set_init_mode(h, 0)
        stream.synchronize()

    # max over ranks
    ms, te, sweep_med = reduce_max_over_ranks([ms, te, float(np.median(sweep_ms))], ws, dev)
    ms_per_step = ms / args.steps
    lups = job_mlups(ws, N, SWEEPS_PER_STEP * args.steps, ms / 1e3) * 1e6
    e2e_lups = job_mlups(ws, N, SWEEPS_PER_STEP * e2e_steps, te) * 1e6

    peak, peak_src = measured_peaks()
    bpl = BYTES_PER_LUP_MOMENTS if moments else BYTES_PER_LUP[storage]
    skey = "_moments" if moments else ""
    achieved = bpl * N / (sweep_med / 1e3) / 1e9
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        t = json.load(open(TRAFFIC_FILE))
        rec = t.get(f"tgv{n}_{args.storage}" + ("" if args.collision == "rlb" else f"_{args.collision}") + skey)
        if rec and rec.get("source_sha") == kernel_source_sha():
            traffic = rec.get("dram_bytes_per_launch")

    issue = None
    rate = ffma_issue_rate(stream)
    ipc = instructions_per_cell(args.storage + skey)
    if ipc is not None:
        ach = ipc * N / (sweep_med / 1e3)
        issue = {"bound": "issue", "achieved": ach, "peak": rate, "unit": "warp-inst/s",
                 "frac": ach / rate, "warp_inst_per_cell": ipc,
                 "peak_source": "FFMA probe measured in this run (grlb_ffma_probe)",
                 "inst_source": "ncu smsp__inst_executed.sum of the same kernel source"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, _ = cpu_oracle_sample(n, 1, min_seconds=10.0)

    if rank == 0:
        line = {
            "metric": "MLUP/s", "value": lups / 1e6, "unit": "MLUP/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f32", 1: "f16-storage/f32", 2: "bf16-storage/f32"}[storage],
            "data": "synthetic",
            "config": {"workload": f"tgv{n}_{args.storage}_{args.collision}", "grid": [n, n, n],
                       "mach": 1.25, "re": 1600, "sweeps_per_step": SWEEPS_PER_STEP,
                       "step": "init kernel + 49 sweeps + 1 diagnostic sweep (FP64 reductions)",
                       "parallelism": f"replicas{ws}",
                       "state": ("moments: Q_k, J*_k of the regularized outgoing set, 20 FP32 per cell"
                                 if moments else "populations: 35 per cell"),
                       "l2": f"inputs larger than L2 ({bpl * N / 1e9:.1f} GB of state), no flush"},
            "e2e": {"value": e2e_lups / 1e6, "unit": "MLUP/s",
                    "h2d_bytes_per_step": 5 * N * 8, "d2h_bytes_per_step": 8 * 13},
            # per step: init + 49 plain sweeps + diagnostic sweep + 2 finalize stages
            "gpu_launches": args.steps * (SWEEPS_PER_STEP + 3),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": f"sweep_kernel<{args.storage},{coll_label}{',moments' if moments else ''}> (plain sweep)",
                         "bytes_per_launch": bpl * N, "bytes_per_lup": bpl, "launch_ms_median": sweep_med,
                         "peak_source": f"{peak_src} hbm_gbs",
                         **({"note": "moment storage: 160 B per cell update (the 20 FP32 moments of "
                                     "the regularized outgoing set read and written) in place of the "
                                     "280 B of 35 populations; results bit for bit the same"}
                            if moments else {})},
            "issue_ceiling": issue,
            "ffma_probe": {"warp_inst_per_s": rate, "fp32_tflops": 64.0 * rate / 1e12},
            "clocks": clocks,
            "cpu_baseline": cpu,
            "diag_timed_step": {"n_nan": diag["n_nan"], "n_sensor": diag["n_sensor"],
                                "ke": diag["ke"], "step": diag["step"],
                                "note": "equilibrium start: cell-local dissipation alternates "
                                        "with the non-equilibrium part at omega -> 2"},
            "diag_ce_start": diag_record(ce_diag, ce_spec, case),
        }
        if rank == 0 and not args.no_legs:
            line["batched"] = batched_leg(args)
            line["served"] = served_leg(args)
        print(json.dumps(line), flush=True)
    dom.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_zslab(args):
    """One periodic domain split along z over the ranks (one device each): every rank owns one
    z-period of the n^3 Taylor-Green vortex, so N ranks advance an n x n x (n N) domain (weak
    scaling), exchanging the ghost slices of their slabs with their neighbours before every
    sweep (decomp.SlabRank: pack kernel, NCCL send / receive, unpack kernel).  A bench step =
    initialisation from device-resident fields + 50 exchange-and-sweep iterations; value =
    the interior cell updates of all ranks over the slowest rank's time."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2609_16361_b300 import decomp, inputs
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = args.n
    moments = args.state != "populations"
    whole = inputs.tgv3d(n)
    if moments:
        whole = dataclasses.replace(whole, params=whole.params.replace(streaming=2))
    part = decomp.slab_case(whole, 0, n)   # this rank's period, ghost planes wrapped
    stream = torch.cuda.Stream()
    r = decomp.SlabRank(None, rank, ws, stream=stream, part=part)
    dev = torch.device("cuda", local)
    rho_d = torch.from_numpy(part.rho).to(dev)
    u_d = torch.from_numpy(part.u).to(dev).contiguous()
    p_d = torch.from_numpy(part.p).to(dev)

    def one_step():
        r.init_device(rho_d, u_d, p_d)
        r.step(SWEEPS_PER_STEP)

    for _ in range(args.warmup):
        one_step()
    stream.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            one_step()
        e1.record(stream)
        e1.synchronize()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = reduce_max_over_ranks([e0.elapsed_time(e1)], ws, dev)[0]
    cells = n ** 3
    Q = r.conserved_interior()
    finite = bool(np.isfinite(Q).all())
    r.close()
    if rank == 0:
        line = {"metric": "MLUP/s", "value": job_mlups(ws, cells, SWEEPS_PER_STEP * args.steps, ms / 1e3),
                "unit": "MLUP/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"tgv{n}_f32_rlb z-period per rank: {n}x{n}x{n * ws} periodic domain",
                           "parallelism": f"zslab{ws}", "sweeps_per_step": SWEEPS_PER_STEP,
                           "step": "init kernel + 50 x (ghost pack, NCCL send/recv to both z "
                                   "neighbours, unpack, sweep)",
                           "halo_bytes_per_sweep_per_rank": 2 * (10 if moments else 5) * n * n * 4,
                           "state": "moments" if moments else "populations",
                           "l2": "inputs larger than L2, no flush"},
                "gpu_launches": args.steps * (1 + 3 * SWEEPS_PER_STEP),
                "clocks": clk.summary(), "finite_after_run": finite}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def diag_record(g, spec, case):
    """FP64 diagnostics of a diagnostic sweep in physical units (volume averages normalised by
    rho0 V0^2 and rho0 V0^3 / L0), with the spectral dissipation of the same state."""
    prm = case.params
    N = prm.ncells
    s = prm.dt / prm.dx
    unit = prm.dx ** 2 / prm.dt ** 3 / N
    out = {"step": g["step"], "t_c": g["step"] * prm.dt, "n_nan": g["n_nan"],
           "n_sensor": g["n_sensor"], "n_floor": g["n_floor"], "E_k": g["ke"] / (s * s) / N,
           "eps_s": g["eps_s"] * unit, "eps_d": g["eps_d"] * unit}
    if spec is not None:
        out["eps_s_spectral"] = spec["eps_s"] * unit
        out["eps_d_spectral"] = spec["eps_d"] * unit
        out["eps_s_cell_over_spectral"] = out["eps_s"] / out["eps_s_spectral"]
    return out


def batched_leg(args, steps=200):
    """Short batched leg of the default line: the 64-domain seed-0 mix (48 Becker tubes + 16
    Taylor-Green boxes), `steps` steps in one batch (default schedule: concurrent single-domain
    sweeps replayed from CUDA graphs) against the same domains advanced one after another with
    one launch per sweep (legacy stream: grlb_step replays no graph there)."""
    import torch
    from paper_2609_16361_b300 import capi, inputs
    stream = torch.cuda.Stream()
    st = stream.cuda_stream
    cases = inputs.batched_mix(0)
    cells = sum(c.params.ncells for c in cases)
    moments = args.state != "populations"  # every domain of the mix is FP32, regularized
    doms = [capi.Domain(c.params.replace(streaming=2 if moments else 0), stream=st) for c in cases]
    for d, c in zip(doms, cases):
        d.init(c.rho, c.u, c.p)
    b = capi.grlb_batch_create([d.h for d in doms], use_graph=1)
    capi.grlb_batch_set_stream(b, st)
    capi.grlb_batch_step(b, 20)   # warm-up; also captures the step graphs (>= 16 steps)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    capi.grlb_batch_step(b, steps)
    e1.record(stream)
    e1.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    capi.grlb_batch_destroy(b)
    legacy = torch.cuda.default_stream()
    for d, c in zip(doms, cases):
        capi.grlb_set_stream(d.h, legacy.cuda_stream)
        d.init(c.rho, c.u, c.p)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(legacy)
    for d in doms:
        d.step(steps)
    e1.record(legacy)
    e1.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3
    for d in doms:
        d.close()
    mb, mp = cells * steps / t_batch / 1e6, cells * steps / t_plain / 1e6
    return {"metric": "batched MLUP/s", "value": mb, "unit": "MLUP/s",
            "sequential_plain_mlups": mp, "vs_sequential_plain": mb / mp,
            "workload": "64 uneven domains (48 Becker 128-2048 x 4 x 4, 16 Taylor-Green 32^3-96^3 "
                        "Re 100), seed 0", "cells": cells, "steps": steps,
            "state": "moments" if moments else "populations"}


def served_leg(args, n_requests=40, rate=20.0):
    """Short serving leg of the default line: the seed-0 trace of `n_requests` Poisson
    arrivals at `rate`/s served with continuous batching, against the same trace served first
    in, first out, one domain at a time through grlb_step."""
    from paper_2609_16361_b300 import inputs, serve
    trace = inputs.serving_trace(0, n_requests=n_requests, rate=rate)
    moments = args.state != "populations"  # FP32 requests as moments, FP16 ones as populations
    res = serve.Server(hbm_budget=150e9, chunk=200, moments=moments).run(trace, realtime=True)
    sb = serve.summarize(res)
    sp = serve.summarize(serve.serial_plain(trace, realtime=True, moments=moments))
    keep = ("solves_per_s", "p50_latency_s", "p99_latency_s", "mean_latency_s", "mlups", "failed")
    return {"metric": "served solves/s", "value": sb["solves_per_s"], "unit": "solves/s",
            **{k: sb[k] for k in keep if k != "solves_per_s"},
            "serial_plain": {k: sp[k] for k in keep},
            "vs_serial_plain": sb["solves_per_s"] / sp["solves_per_s"],
            "p99_vs_serial_plain": sb["p99_latency_s"] / sp["p99_latency_s"],
            "workload": f"Poisson {rate:g}/s, {n_requests} requests (Sod / Becker tubes, Taylor-Green "
                        "64^3-192^3 Re 100, FP32 or FP16, 500-5000 steps), seed 0, 150 GB budget",
            "state": "FP32 requests as moments" if moments else "populations"}


# ----------------------------------------------------------------------------------------
def run_batch(args):
    """64 uneven domains (48 Becker tubes + 16 Taylor-Green boxes, seed 0), 1000 steps each,
    under the three batch schedules (concurrent single-domain sweeps -- the value --; one
    launch per step with constant-table records, autotuned or default tiles; the same with
    device-memory records and no graph), the tube class alone under each, against 64
    sequential single-domain runs through grlb_step -- one launch per sweep (the domains on the
    legacy default stream, where grlb_step replays no graph: the baseline `vs_sequential_plain`
    divides by) and, for reference, on a stream of their own, where grlb_step replays the small
    domains' sweeps from CUDA graphs."""
    import torch
    from paper_2609_16361_b300 import autotune, capi, inputs
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    st = stream.cuda_stream
    cases = inputs.batched_mix(0)
    cells = sum(c.params.ncells for c in cases)
    steps = args.batch_steps
    table = autotune.tune(cases, steps=20, stream=stream)
    doms = []
    for c in cases:
        d = capi.Domain(c.params, stream=st)
        d.init(c.rho, c.u, c.p)
        doms.append(d)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = {}
    S = capi
    for label, sched, use_graph, plan in (
            ("batched_concurrent", S.SCHED_CONCURRENT, 1, None),
            ("batched_table_const_graph_tuned", S.SCHED_TABLE_CONST, 1, autotune.plan(cases, table)),
            ("batched_table_const_graph_default", S.SCHED_TABLE_CONST, 1, None),
            ("batched_table_nograph_default", S.SCHED_TABLE, 0, None)):
        for d, c in zip(doms, cases):
            d.init(c.rho, c.u, c.p)
        b = capi.grlb_batch_create([d.h for d in doms], use_graph=use_graph, schedule=sched)
        capi.grlb_batch_set_stream(b, st)
        if plan:
            capi.grlb_batch_set_tile_x(b, plan)
        capi.grlb_batch_step(b, 20)   # warm-up; also captures the step graphs (>= 16 steps)
        stream.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        capi.grlb_batch_step(b, steps)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        capi.grlb_batch_destroy(b)
        out[label] = {"mlups": cells * steps / t / 1e6, "seconds": t}
    # the tube class alone (48 Becker tubes, all in the batched kernel): the two ways of
    # reading the domain records, against the HBM roofline (280 B per cell update)
    tubes = [i for i, c in enumerate(cases) if c.params.name.startswith("becker")]
    tcells = sum(cases[i].params.ncells for i in tubes)
    peak, _ = measured_peaks()
    for label, mode in (("tubes_concurrent", S.SCHED_CONCURRENT), ("tubes_table_const", S.SCHED_TABLE_CONST),
                        ("tubes_table", S.SCHED_TABLE)):
        for i in tubes:
            doms[i].init(cases[i].rho, cases[i].u, cases[i].p)
        b = capi.grlb_batch_create([doms[i].h for i in tubes], use_graph=1, schedule=mode)
        capi.grlb_batch_set_stream(b, st)
        capi.grlb_batch_step(b, 20)   # warm-up; also captures the step graphs (>= 16 steps)
        stream.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        capi.grlb_batch_step(b, steps)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        capi.grlb_batch_destroy(b)
        gbs = 280 * tcells * steps / t / 1e9
        out[label] = {"mlups": tcells * steps / t / 1e6, "seconds": t, "cells": tcells,
                      "achieved_gbs": gbs, "roofline_frac": gbs / peak}
    legacy = torch.cuda.default_stream()
    for label, s_run in (("sequential_plain", legacy), ("sequential_graph_replay", stream)):
        for d, c in zip(doms, cases):
            capi.grlb_set_stream(d.h, s_run.cuda_stream)
            d.init(c.rho, c.u, c.p)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(s_run)
        for d in doms:
            d.step(steps)
        e1.record(s_run)
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        out[label] = {"mlups": cells * steps / t / 1e6, "seconds": t}
    diag_ok = True
    for d in doms:
        d.step_diag()
        diag_ok &= d.diag(allow_nonfinite=True)["n_nan"] == 0
    for d in doms:
        d.close()
    best = out["batched_concurrent"]["mlups"]
    line = {"metric": "batched MLUP/s (64 uneven domains, 1000 steps each)", "value": best,
            "unit": "MLUP/s", "n_gpus": 1, "higher_is_better": True,
            "vs_sequential_plain": best / out["sequential_plain"]["mlups"],
            "vs_sequential_graph_replay": best / out["sequential_graph_replay"]["mlups"],
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "48 Becker tubes (128-2048 x 4 x 4, M 1.5-5) + 16 Taylor-Green "
                                   "boxes (32^3-96^3, M 0.5-1.25, Re 100), seed 0",
                       "cells": cells, "steps": steps},
            "variants": out, "autotune": table, "finite_after_run": bool(diag_ok)}
    print(json.dumps(line), flush=True)
    return 0


def run_batch_tubes(args):
    """The tube class of the batched workload alone: the 48 Becker tubes of the seed-0 mix
    (128-2048 x 4 x 4 cells, all below solo_min_cells), one batch under --schedule,
    --batch-steps steps (CUDA graphs), against the HBM roofline (280 B per cell update)."""
    import torch
    from paper_2609_16361_b300 import capi, inputs
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    st = stream.cuda_stream
    cases = [c for c in inputs.batched_mix(0) if c.params.name.startswith("becker")]
    cells = sum(c.params.ncells for c in cases)
    doms = [capi.Domain(c.params, stream=st) for c in cases]
    for d, c in zip(doms, cases):
        d.init(c.rho, c.u, c.p)
    sched = {"concurrent": capi.SCHED_CONCURRENT, "table_const": capi.SCHED_TABLE_CONST,
             "table": capi.SCHED_TABLE}[args.schedule]
    b = capi.grlb_batch_create([d.h for d in doms], use_graph=1, schedule=sched, max_lanes=args.max_lanes)
    capi.grlb_batch_set_stream(b, st)
    capi.grlb_batch_step(b, 20)   # warm-up; also captures the step graphs (>= 16 steps)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    capi.grlb_batch_step(b, args.batch_steps)
    e1.record(stream)
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    capi.grlb_batch_destroy(b)
    for d in doms:
        d.close()
    peak, src = measured_peaks()
    gbs = 280 * cells * args.batch_steps / t / 1e9
    line = {"metric": "batched MLUP/s (48 Becker tubes)", "value": cells * args.batch_steps / t / 1e6,
            "unit": "MLUP/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "48 Becker tubes 128-2048 x 4 x 4 (M 1.5-5), seed 0", "cells": cells,
                       "steps": args.batch_steps, "schedule": args.schedule, "max_lanes": args.max_lanes},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "peak_source": f"{src} hbm_gbs", "bytes_per_cell": 280}}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Poisson trace (seed 0, --rate requests/s, default 20): continuous-batching server against
    the same trace served first-in first-out one domain at a time with plain launches."""
    import torch
    from paper_2609_16361_b300 import autotune, inputs, serve
    torch.cuda.set_device(0)
    trace = inputs.serving_trace(0, n_requests=args.requests, rate=args.rate)
    table = autotune.tune([r.case for r in trace[:12]], steps=10)
    srv = serve.Server(hbm_budget=150e9, chunk=200, tile_table=table)
    res = srv.run(trace, realtime=True)
    s_batched = serve.summarize(res)
    base = serve.serial_plain(trace, realtime=True)
    s_plain = serve.summarize(base)
    # the same trace with one population buffer for large requests (half their memory)
    srv1 = serve.Server(hbm_budget=150e9, chunk=200, tile_table=table, one_buffer_large=True)
    s_one = serve.summarize(srv1.run(trace, realtime=True))
    s_one["peak_hbm_bytes"] = srv1.peak_bytes
    same = sum(a.digest == b.digest for a, b in zip(res, base))
    line = {"metric": "served solves/s (continuous batching)", "value": s_batched["solves_per_s"],
            "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "p50_latency_s": s_batched["p50_latency_s"], "p99_latency_s": s_batched["p99_latency_s"],
            "baseline_serial_plain": s_plain,
            "batched": s_batched, "batched_one_buffer_large": s_one, "peak_resident": srv.peak_resident,
            "peak_hbm_bytes": srv.peak_bytes, "dtype": "f32/f16 storage, f32 arithmetic",
            "data": "synthetic",
            "config": {"workload": f"Poisson {args.rate:g}/s; Sod / Becker tubes, Taylor-Green "
                                   "64^3-192^3 (Re 100), FP32 or FP16, 500-5000 steps; seed 0",
                       "requests": args.requests, "hbm_budget_bytes": 150e9, "chunk": 200,
                       "lookahead_chunks": 12},
            "bitwise_equal_to_plain": same}
    print(json.dumps(line), flush=True)
    return 0


def run_precision(args):
    """Storage precision modes side by side: FP32, FP16 and BF16 shifted populations (FP32
    arithmetic).  Accuracy against the FP64 oracle, relative L-inf / L1 of rho, u, T:
    Taylor-Green 64^3 after 100 steps, the Sod tube (400 cells, 1000 steps), and the supersonic
    Taylor-Green vortex at --prec-n^3 after --prec-steps steps (the precision study of the
    storage modes; the collision of --collision, Chapman-Enskog start).  Speed: the plain sweep at 256^3 (CUDA
    events, 40 sweeps after warm-up) against the HBM roofline of each mode."""
    import numpy as np
    import torch
    import oracle
    from paper_2609_16361_b300 import capi, inputs
    torch.cuda.set_device(0)
    names = {0: "f32", 1: "f16", 2: "bf16"}

    def prim(Q, gamma):
        rho = Q[0]
        u = Q[1:4] / rho
        p = (gamma - 1) * (Q[4] - 0.5 * rho * (u * u).sum(0))
        return rho, u, p / rho

    def errs(a, b):
        out = {}
        for nm, x, y in zip(("rho", "u", "T"), a, b):
            out[nm] = {"linf": float(np.abs(x - y).max() / np.abs(y).max()),
                       "l1": float(np.abs(x - y).sum() / np.abs(y).sum())}
        return out

    cases = {"tgv64_100": (lambda st: inputs.tgv3d(64, storage=st), 100),
             "sod400_1000": (lambda st: inputs.sod(400, storage=st), 1000)}
    acc = {}
    for cname, (mk, nsteps) in cases.items():
        ref = mk(0)
        o = oracle.Oracle(ref.params)
        o.init_primitive(ref.rho, ref.u, ref.p)
        o.step(nsteps)
        R = prim(o.conserved(), ref.params.gamma)
        for st in (0, 1, 2):
            c = mk(st)
            d = capi.Domain(c.params)
            d.init(c.rho, c.u, c.p)
            d.step(nsteps)
            acc.setdefault(names[st], {})[cname] = errs(prim(d.conserved(), c.params.gamma), R)
            d.close()
    # Storage modes against the FP64 oracle on a long run: the supersonic Taylor-Green vortex at
    # --prec-n^3 (default 128^3: the largest size the oracle finishes in ~15 min on the host
    # cores) after --prec-steps steps (default 2000) in each storage mode.  The oracle runs in
    # a thread (its C stepper releases the GIL) while the device runs the three modes.
    long_steps = args.prec_steps
    pn = args.prec_n
    coll = COLLISIONS[args.collision][0]
    def mk_long(st):
        c = inputs.tgv3d(pn, re=args.prec_re, storage=st, collision=coll)
        if args.omega_min is not None:
            c.params = c.params.replace(omega_min=args.omega_min)
        return c

    ref = mk_long(0)
    orc = {}

    # snapshots along the run: the storage error first, then, once the under-resolved vortex
    # turns chaotic (t_c ~ 5-10), the divergence every pair of runs shows whatever the precision
    marks = sorted({m for m in (long_steps // 8, long_steps // 4, long_steps // 2) if m > 0} | {long_steps})

    def oracle_run():
        try:
            o = oracle.Oracle(ref.params)
            o.init_primitive(ref.rho, ref.u, ref.p, ce_init=True)
            t0 = time.perf_counter()
            done = 0
            for m in marks:
                o.step(m - done)
                done = m
                orc[m] = o.conserved()
            orc["seconds"] = time.perf_counter() - t0
        except RuntimeError as e:   # a non-finite state makes the reconstruction singular
            orc["error"] = str(e)

    def ke_mean(Q):
        return float((0.5 * (Q[1:4] ** 2).sum(0) / Q[0]).mean())

    th = threading.Thread(target=oracle_run)
    th.start()
    snaps = {}
    for st in (0, 1, 2):
        c = mk_long(st)
        d = capi.Domain(c.params)
        d.init(c.rho, c.u, c.p, ce_init=True)
        done = 0
        for m in marks:
            d.step(m - done)
            done = m
            snaps[(st, m)] = d.conserved()
        d.close()
    finite = {names[st]: bool(np.isfinite(snaps[(st, long_steps)]).all()) for st in (0, 1, 2)}
    th.join()
    for m in marks:
        key = f"tgv{pn}_re{args.prec_re:g}_{args.collision}_{m}_vs_oracle"
        if m in orc and np.isfinite(orc[m]).all():
            R = prim(orc[m], ref.params.gamma)
            for st in (0, 1, 2):
                e = errs(prim(snaps[(st, m)], ref.params.gamma), R)
                e["E_k_rel"] = abs(ke_mean(snaps[(st, m)]) / ke_mean(orc[m]) - 1.0)
                acc.setdefault(names[st], {})[key] = e
        for st in (1, 2):
            e = errs(prim(snaps[(st, m)], ref.params.gamma), prim(snaps[(0, m)], ref.params.gamma))
            e["E_k_rel"] = abs(ke_mean(snaps[(st, m)]) / ke_mean(snaps[(0, m)]) - 1.0)
            acc.setdefault(names[st], {})[f"tgv{pn}_re{args.prec_re:g}_{m}_vs_f32"] = e
    del snaps
    speed = {}
    peak, src = measured_peaks()
    for st in (0, 1, 2):
        c = inputs.tgv3d(args.n, storage=st)
        d = capi.Domain(c.params)
        d.init(c.rho, c.u, c.p)
        d.step(5)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        d.step(40)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / 40
        N = c.params.ncells
        gbs = BYTES_PER_LUP[st] * N / (ms / 1e3) / 1e9
        speed[names[st]] = {"ms_per_sweep": ms, "mlups": N / (ms / 1e3) / 1e6,
                            "bytes_per_lup": BYTES_PER_LUP[st], "achieved_gbs": gbs,
                            "roofline_frac": gbs / peak}
        d.close()
    line = {"metric": "precision modes: error vs FP64 oracle and sweep MLUP/s", "unit": "MLUP/s",
            "value": speed["f16"]["mlups"], "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32 / f16 / bf16 storage, f32 arithmetic", "data": "synthetic",
            "config": {"workload": f"tgv{args.n} sweep speed; tgv64 x100 and sod400 x1000 accuracy "
                                   f"vs the FP64 oracle; tgv{pn} Re {args.prec_re:g} ({args.collision} "
                                   f"collision, omega_min {ref.params.omega_min:g}, Chapman-Enskog "
                                   f"start) x{long_steps} vs the FP64 oracle",
                       "peak_gbs": peak, "peak_source": src,
                       "oracle_seconds": orc.get("seconds"), "oracle_threads": oracle.num_threads(),
                       "oracle_error": orc.get("error")},
            "finite_after_long_run": finite, "accuracy": acc, "speed": speed}
    print(json.dumps(line), flush=True)
    return 0


def run_tgv_series(args):
    """Supersonic Taylor-Green at n^3 (M0 1.25, Re 1600, Sutherland, RLB + sensor, FP32) for up
    to --run-steps steps with FP64 diagnostics every 50 steps: volume-averaged kinetic energy
    and solenoidal / dilatational dissipation (normalised by rho0 V0^2 and rho0 V0^3 / L0) in
    convective time t_c, until the run ends or the state stops being finite."""
    import torch
    from paper_2609_16361_b300 import capi, inputs
    torch.cuda.set_device(0)
    c = inputs.tgv3d(args.n, collision=COLLISIONS[args.collision][0])
    if args.omega_min is not None:
        c.params = c.params.replace(omega_min=args.omega_min)
    prm = c.params
    N = prm.ncells
    d = capi.Domain(prm)
    d.init(c.rho, c.u, c.p, ce_init=args.ce_init)
    s = prm.dt / prm.dx
    series = []
    first_bad = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step = 0
    while step < args.run_steps:
        d.step(49)
        d.step_diag()
        g = d.diag(allow_nonfinite=True)
        step = g["step"]
        ke = g["ke"] / (s * s) / N
        eps_s = g["eps_s"] * prm.dx ** 2 / prm.dt ** 3 / N
        eps_d = g["eps_d"] * prm.dx ** 2 / prm.dt ** 3 / N
        rec = {"step": step, "t_c": step * prm.dt, "E_k": ke, "eps_s": eps_s,
               "eps_d": eps_d, "n_sensor": g["n_sensor"], "n_floor": g["n_floor"],
               "n_nan": g["n_nan"]}
        if g["n_nan"] == 0 and math.isfinite(ke):
            # the same channels with spectral derivatives (Sec. 3.4), and the spectrum
            spec, sp = d.spectral()
            rec["eps_s_spectral"] = sp["eps_s"] * prm.dx ** 2 / prm.dt ** 3 / N
            rec["eps_d_spectral"] = sp["eps_d"] * prm.dx ** 2 / prm.dt ** 3 / N
            if step % 200 == 0:
                rec["spectrum"] = [float(v) / (s * s) for v in spec]
        series.append(rec)
        if g["n_nan"] > 0 or not math.isfinite(ke):
            first_bad = step
            break
    wall = time.perf_counter() - t0
    d.close()
    line = {"metric": "Taylor-Green run with FP64 diagnostics every 50 steps", "unit": "MLUP/s",
            "value": N * step / wall / 1e6, "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"tgv{args.n}_f32_{args.collision}", "steps_requested": args.run_steps,
                       "omega": prm.omega_mom, "fmu": c.meta["fmu"], "omega_min": prm.omega_min,
                       "start": "chapman-enskog" if args.ce_init else "equilibrium"},
            "spectral": "eps_*_spectral: spectral derivatives of u = m / rho on the state the "
                        "step landed on; spectrum: shell sums of 1/2 |u^|^2 / N^2 in units of V0^2, "
                        "every 200 steps",
            "steps_run": step, "first_nonfinite_step": first_bad, "wall_s": wall,
            "series": series}
    print(json.dumps(line), flush=True)
    return 0


def run_tgv_map(args):
    """Stability map of the supersonic Taylor-Green vortex (M0 1.25, Re 1600, Sutherland, FP32,
    Chapman-Enskog start) over the collision reading, the background damping f_mu and the
    sensor floor rate omega_min: each run goes up to --run-steps steps with FP64 diagnostics
    every 50 steps and reports how far it stays finite (step, t_c) and its kinetic energy at
    t_c 2, 4, 8, 12, 16, 20.  The paper's setting (Tab. run_params, Sec. 3.4) is f_mu of the
    resolution (0.9 at 128^3) with omega_min 1.987."""
    import torch
    from paper_2609_16361_b300 import capi, inputs
    torch.cuda.set_device(0)
    n = args.n
    rows = []
    marks = (2.0, 4.0, 8.0, 12.0, 16.0, 20.0)
    base_fmu = inputs.fmu_for_resolution(n)
    for coll in ("rlb", "gated"):
        for fmu_scale in (1.0, 2.0, 4.0):
            for om_min in (1.987, 1.95, 1.9, 1.8, 1.5):
                c = inputs.tgv3d(n, collision=COLLISIONS[coll][0], fmu=base_fmu * fmu_scale)
                prm = c.params.replace(omega_min=om_min)
                d = capi.Domain(prm)
                d.init(c.rho, c.u, c.p, ce_init=True)
                s = prm.dt / prm.dx
                step, last_ok, ek_at, sensor_max = 0, 0, {}, 0
                while step < args.run_steps:
                    d.step(49)
                    d.step_diag()
                    g = d.diag(allow_nonfinite=True)
                    step = g["step"]
                    ke = g["ke"] / (s * s) / prm.ncells
                    if g["n_nan"] > 0 or not math.isfinite(ke):
                        break
                    last_ok = step
                    sensor_max = max(sensor_max, g["n_sensor"])
                    tc = step * prm.dt
                    for m in marks:
                        if m not in ek_at and tc >= m:
                            ek_at[m] = ke
                d.close()
                rows.append({"collision": coll, "fmu": base_fmu * fmu_scale, "omega": prm.omega_mom,
                             "omega_min": om_min, "last_finite_step": last_ok,
                             "last_finite_t_c": last_ok * prm.dt, "finite_to_end": last_ok >= args.run_steps,
                             "E_k_at_t_c": {f"{m:g}": v for m, v in ek_at.items()},
                             "max_sensor_cells": sensor_max})
    line = {"metric": "Taylor-Green stability map (steps finite)", "unit": "steps",
            "value": max(r["last_finite_step"] for r in rows), "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"tgv{n} M0 1.25 Re 1600, collision x f_mu x omega_min",
                       "steps_requested": args.run_steps, "paper_setting": {"fmu": base_fmu, "omega_min": 1.987}},
            "runs": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_spectral(args):
    """Spectral post-processing (grlb_spectral_diag) of the n^3 Taylor-Green state after 50
    steps: time per call (CUDA events on the domain's stream, 3 warm-up calls, median of 5),
    against the traffic of its five kernels, 372 B per cell (K1 prep + forward x: 140 + 28;
    forward y: 48; forward z + modes + inverse z: 24 + 32; inverse y: 64; inverse x +
    dissipation: 32 + 4), and the spectral against the cell-local (reconstructed-gradient)
    dissipation."""
    import torch
    from paper_2609_16361_b300 import capi, inputs
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    n = args.n
    c = inputs.tgv3d(n)
    prm = c.params
    N = prm.ncells
    d = capi.Domain(prm, stream=stream.cuda_stream)
    d.init(c.rho, c.u, c.p)
    d.step(49)
    d.step_diag()
    g = d.diag()
    for _ in range(3):
        d.spectral()
    times = []
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        spec, sp = d.spectral()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    # one 50-step Taylor-Green step for scale
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    d.step(49)
    d.step_diag()
    e1.record(stream)
    e1.synchronize()
    step_ms = e0.elapsed_time(e1)
    d.close()
    peak, src = measured_peaks()
    bpc = 372
    ach = bpc * N / (ms / 1e3) / 1e9
    # DRAM bytes of the five kernels of one call (ncu), while the kernel source is unchanged
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        rec = json.load(open(TRAFFIC_FILE)).get(f"spectral_tgv{n}_f32")
        if rec and rec.get("source_sha") == kernel_source_sha(SPECTRAL_SOURCES):
            traffic = rec.get("dram_bytes_per_call")
    line = {"metric": "spectral diagnostics time per call", "value": ms, "unit": "ms",
            "n_gpus": 1, "higher_is_better": False, "dtype": "f32 (FFT), f64 (sums)",
            "data": "synthetic",
            "config": {"workload": f"tgv{n}_f32 state after 50 steps", "grid": [n, n, n],
                       "shells": len(spec)},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "traffic": traffic, "bytes_per_call": bpc * N,
                         "peak_source": f"{src} hbm_gbs",
                         "note": "whole call, including its two host synchronisations"},
            "share_of_50_step_step": ms / step_ms,
            "eps_s": {"spectral": sp["eps_s"], "cell_local": g["eps_s"]},
            "eps_d": {"spectral": sp["eps_d"], "cell_local": g["eps_d"]},
            # K1 prep + forward x, forward y, forward z + modes + inverse z, inverse y,
            # inverse x + dissipation
            "gpu_launches_per_call": 5}
    print(json.dumps(line), flush=True)
    return 0


def run_slabs(args):
    """z-slab decomposition on one device: the n^3 Taylor-Green domain (FP32, RLB + sensor) as
    2 and 4 z-slabs with one ghost plane on each side, the ghost exchange (grlb_halo_exchange_z)
    before every step, against the undivided domain; MLUP/s of interior cells over --steps x 50
    sweeps (CUDA events, 3 warm-up steps)."""
    import torch
    from paper_2609_16361_b300 import capi, decomp, inputs
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    n = args.n
    c = inputs.tgv3d(n)
    N = c.params.ncells
    sweeps = SWEEPS_PER_STEP * args.steps

    def timed(step):
        for _ in range(3):
            step(SWEEPS_PER_STEP)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(sweeps)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3

    out = {}
    d = capi.Domain(c.params, stream=stream.cuda_stream)
    d.init(c.rho, c.u, c.p)
    out["undivided"] = N * sweeps / timed(d.step) / 1e6
    d.close()
    for S in (2, 4):
        s = decomp.SlabSet(c, decomp.slab_sizes(n, S), stream=stream.cuda_stream)
        s.init()
        out[f"slabs{S}"] = N * sweeps / timed(s.step) / 1e6
        s.close()
    line = {"metric": "MLUP/s (interior cells) of the z-slab decomposition on one device",
            "value": out["slabs2"], "unit": "MLUP/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"tgv{n}_f32_rlb_sensor as z-slabs", "steps": args.steps,
                       "sweeps_per_step": SWEEPS_PER_STEP},
            "variants": out, "slabs2_vs_undivided": out["slabs2"] / out["undivided"],
            "slabs4_vs_undivided": out["slabs4"] / out["undivided"]}
    print(json.dumps(line), flush=True)
    return 0


def run_cases(args):
    """Sweep throughput per input kind (FP32, one GPU, CUDA events after warm-up): the Sod tube
    (400 x 1 x 1, 1000 steps) and a Becker tube (2048 x 4 x 4, 1000 steps) of the paper's
    sizes, which are too small to fill the device and are reported per step as well; the same
    tube physics at the Taylor-Green cell count (Sod 262144 x 8 x 8 with the transverse fields
    replicated, Becker 262144 x 8 x 8, M 3; 200 sweeps each); and the supersonic Taylor-Green
    vortex at 256^3 (200 sweeps)."""
    import numpy as np
    import torch
    from paper_2609_16361_b300 import capi, inputs
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    peak, src = measured_peaks()

    def widen(case, ny, nz):
        prm = case.params.replace(ny=ny, nz=nz)
        rep = ny * nz
        return inputs.Case(prm, np.tile(case.rho, rep), np.stack([np.tile(case.u[k], rep) for k in range(3)]),
                           np.tile(case.p, rep), case.meta)

    big_sod_steps = 200
    om = inputs.becker_tied_omega(8.0)  # the dt-tied relaxation at 8 cells per front
    cases = {
        "sod_400x1x1": (inputs.sod(400), 1000),
        "becker_2048x4x4_M3": (inputs.becker(2048, mach=3.0, ny=4, nz=4, cfl_max=0.1, omega=om), 1000),
        "sod_262144x8x8": (widen(inputs.sod(262144, steps=big_sod_steps, t_end=0.08 * big_sod_steps / 262144), 8, 8),
                           big_sod_steps),
        "becker_262144x8x8_M3": (inputs.becker(262144, mach=3.0, ny=8, nz=8, cfl_max=0.1, omega=om), 200),
        "tgv_256^3": (inputs.tgv3d(args.n), 200),
    }
    out = {}
    for name, (c, sweeps) in cases.items():
        d = capi.Domain(c.params, stream=stream.cuda_stream)
        d.init(c.rho, c.u, c.p)
        d.step(10)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d.step(sweeps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / sweeps
        N = c.params.ncells
        gbs = BYTES_PER_LUP[0] * N / (ms / 1e3) / 1e9
        d.step_diag()
        g = d.diag()
        out[name] = {"cells": N, "sweeps": sweeps, "us_per_sweep": 1e3 * ms, "mlups": N / (ms / 1e3) / 1e6,
                     "achieved_gbs": gbs, "roofline_frac": gbs / peak, "n_nan": g["n_nan"]}
        d.close()
    line = {"metric": "sweep MLUP/s per input kind (FP32)", "value": out["becker_262144x8x8_M3"]["mlups"],
            "unit": "MLUP/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "Sod / Becker tubes at the paper's sizes and at 16.8 M cells; Taylor-Green "
                                   f"{args.n}^3", "peak_gbs": peak, "peak_source": src},
            "cases": out}
    print(json.dumps(line), flush=True)
    return 0


def run_capacity(args):
    """Largest grids on one device: the Taylor-Green workload at 1024^3 with FP16 populations in
    one buffer (AA pattern, 75 GB), at 768^3 with FP32 populations in one buffer (63 GB), and at
    1024^3 in FP32 with the state as moments (two buffers of 20 values per cell, 172 GB) -- the
    paper runs 512^3 (19 GB) on a two-GPU node.  The initial fields are generated on the device
    plane by plane and freed after the init kernel; a few sweeps are timed and the diagnostics
    checked finite.  A run whose state and fields do not fit the free device memory is skipped."""
    import torch
    from paper_2609_16361_b300 import capi, inputs
    torch.cuda.set_device(0)
    runs = []
    for n, storage, streaming in ((1024, "f16", 1), (768, "f32", 1), (1024, "f32", 2)):
        st = {"f32": 0, "f16": 1, "bf16": 2}[storage]
        prm = inputs.tgv3d(n, storage=st, nxyz=(1, 1, 1)).params.replace(nx=n, ny=n, nz=n, streaming=streaming)
        need = capi.grlb_bytes_for(prm)
        torch.cuda.empty_cache()
        capi.grlb_trim_pool()  # the previous run's domain went back to the library's pool
        free, _ = torch.cuda.mem_get_info()
        fields = 5 * 8 * n ** 3
        label = "one buffer (AA)" if streaming == 1 else "moments, two buffers"
        if need + fields + (2 << 30) > free:
            runs.append({"grid": [n, n, n], "storage": storage, "streaming": label, "device_bytes": need,
                         "skipped": f"needs {(need + fields) / 1e9:.0f} GB, {free / 1e9:.0f} GB free"})
            continue
        dom = capi.Domain(prm)
        _, rho, u, p = inputs.tgv3d_device(n, storage=st)
        capi.grlb_init_primitive_device(dom.h, rho.data_ptr(), u.data_ptr(), p.data_ptr())
        torch.cuda.synchronize()
        del rho, u, p
        torch.cuda.empty_cache()
        dom.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dom.step(10)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / 10
        dom.step_diag()
        g = dom.diag()
        N = n ** 3
        bpl = BYTES_PER_LUP_MOMENTS if streaming == 2 else BYTES_PER_LUP[st]
        runs.append({"grid": [n, n, n], "storage": storage, "streaming": label,
                     "device_bytes": need, "ms_per_sweep": ms, "mlups": N / (ms / 1e3) / 1e6,
                     "achieved_gbs": bpl * N / (ms / 1e3) / 1e9,
                     "finite": g["n_nan"] == 0, "mass_total": g["totals"][0]})
        dom.close()
        torch.cuda.empty_cache()
    line = {"metric": "largest Taylor-Green grids on one B300 (MLUP/s of the 1024^3 FP16 run)",
            "value": runs[0].get("mlups"), "unit": "MLUP/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "f16 / f32 storage, f32 arithmetic", "data": "synthetic",
            "config": {"workload": "tgv 1024^3 f16 and 768^3 f32 with one population buffer, "
                                   "1024^3 f32 as moments"},
            "runs": runs}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--state", default="auto", choices=["auto", "populations", "moments"],
                    help="tgv (and the batched / served legs of its line): keep the state as 35 "
                         "populations or as the 20 moments of the regularized outgoing set (FP32, "
                         "--collision rlb; bitwise the same results); auto: moments where they "
                         "apply")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--parallelism", default="replicas", choices=["replicas", "zslab"],
                    help="N > 1: independent replica domains, or one domain split along z over the ranks")
    ap.add_argument("--no-legs", action="store_true",
                    help="leave the batched and served legs out of the default line")
    ap.add_argument("--workload", default="tgv", choices=["tgv", "batch", "serve", "precision", "tgv-series",
                             "tgv-map", "batch-tubes", "capacity", "spectral", "slabs", "cases"])
    ap.add_argument("--max-lanes", type=int, default=0, help="batch-tubes: streams of the table schedule (0 = 2)")
    ap.add_argument("--schedule", default="concurrent", choices=["concurrent", "table_const", "table"],
                    help="batch-tubes: concurrent single-domain sweeps, or one launch per step with "
                         "constant-table / device-memory records")
    ap.add_argument("--run-steps", type=int, default=5000)
    ap.add_argument("--prec-n", type=int, default=128, help="precision: grid of the long comparison")
    ap.add_argument("--prec-steps", type=int, default=2000, help="precision: steps of the long comparison")
    ap.add_argument("--prec-re", type=float, default=1600.0, help="precision: Reynolds number of the long run")
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--rate", type=float, default=20.0, help="serving: mean arrivals per second")
    ap.add_argument("--ce-init", action="store_true", help="tgv-series: Chapman-Enskog start")
    ap.add_argument("--omega-min", type=float, default=None,
                    help="Taylor-Green workloads: sensor floor rate (default: the paper's 1.987)")
    ap.add_argument("--collision", default="rlb", choices=list(COLLISIONS),
                    help="rlb: regularized collision in every cell (Alg. 1); gated: regularized "
                         "where the sensor fires, BGK elsewhere; bgk")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "tgv-series":
        return run_tgv_series(args)
    if args.workload == "tgv-map":
        return run_tgv_map(args)
    if args.workload == "batch-tubes":
        return run_batch_tubes(args)
    if args.workload == "spectral":
        return run_spectral(args)
    if args.workload == "slabs":
        return run_slabs(args)
    if args.workload == "cases":
        return run_cases(args)
    if args.workload == "capacity":
        return run_capacity(args)
    if args.parallelism == "zslab":
        return run_zslab(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
