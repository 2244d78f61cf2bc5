"""Benchmark of the TGV hot path on B300: grid-point-steps/s per precision mode.

Workload (default): the 256^3 Taylor-Green precision sweep - periodic
[0, 2pi]^3, M = 0.1, Re = 1600, Pr = 0.71, gamma = 1.4, 4th-order central
differences with the Blaisdell split, low-storage RK3, dt = 0.00125 (the
stable step at 256^3), kinetic energy and enstrophy reduced in FP64 every 10
steps.  One bench step = one RK3 time step (three fused stage launches) plus
its share of the diagnostics.  The headline `value` is the paper's HPSP mode
(Sec. 3.1: Q stored in FP32, the RK increment Qt in FP16, FP32 arithmetic),
the fastest mode that meets the method's dissipation-rate accuracy target
(the modes that store Q itself in 16 bits do not, like the paper's HP);
every other mode of the sweep is timed in the same run and reported under
"modes" next to FP64.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) the same box is split into z-slabs, one per rank, with
the ghost planes exchanged (NCCL point-to-point) before every RK stage
(strong scaling); value = the box's point-steps / max time over ranks.  The
replica figure (one independent box per rank, weak scaling) is reported
beside it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TGV grid-point-steps/s per precision mode vs FP64 on same B300; % of HBM peak"
UNIT = "grid-point-steps/s"
N_DEFAULT = 256
DT_DEFAULT = 0.00125
SWEEP_RUNS = 5  # timed runs per sweep mode; the median is reported
DIAG_EVERY = 10
HEADLINE = "hpsp"
SWEEP = ("fp64", "spdp", "fp32s_fp64c", "fp32", "bf16_fp32", "fp16_fp32", "fp16", "hpsp")
OFFSET_MODES = ("bf16_fp32", "fp16_fp32", "fp16")
STAGE_SRC = os.path.join(ROOT, "paper_2505_20911_b300", "csrc", "tgv_stage.cuh")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--no-sweep", action="store_true", help="headline mode only")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--accuracy", action="store_true",
                    help="precision sweep accuracy report (--n, --accuracy-steps) against "
                         "the FP64 GPU path; prints one JSON object")
    ap.add_argument("--accuracy-steps", type=int, default=None,
                    help="default: 2000 (tgv), 8000 = t 20 (tgsym)")
    ap.add_argument("--accuracy-modes", default=None,
                    help="comma-separated subset of the sweep's modes (default: all)")
    ap.add_argument("--accuracy-dt", type=float, default=None, help="override dt")
    ap.add_argument("--accuracy-mach", type=float, default=None, help="override the Mach number")
    ap.add_argument("--accuracy-t-end", type=float, default=None,
                    help="run to this time (steps = t_end / dt) instead of --accuracy-steps")
    ap.add_argument("--accuracy-workload", default="tgv", choices=["tgv", "tgsym"],
                    help="tgv: periodic 2 pi box, M 0.1, Re 1600, dt 0.00125 at 256^3; tgsym: "
                         "the symmetric pi box of Sec. 4.1/4.3, M 0.5, Re 800, dt 0.0025")
    ap.add_argument("--probe-peaks", action="store_true",
                    help="measure the FMA pipe in its three arithmetic forms (scalar FP32, "
                         "paired FP32, packed FP16) with the library's probe; prints one JSON")
    ap.add_argument("--profile-case", default=None, metavar="MODE",
                    help="run 2 warm-up RK3 steps and 1 more step of MODE at --n, then exit "
                         "(the small case an ncu capture of the stage kernel uses)")
    return ap.parse_args()


def profile_case(args):
    """Launches: 1 init, 6 warm-up stage launches, then 3 stage launches."""
    import torch
    import paper_2505_20911_b300 as tgv
    cfg = mode_config(tgv, args.n, args.profile_case)
    qa = tgv.empty_state(cfg)
    qb = torch.empty_like(qa)
    qt = tgv.empty_qt(cfg)
    tgv.tgv_init(cfg, qa)
    dt = DT_DEFAULT * 256.0 / args.n
    tgv.rk_step(cfg, qa, qb, qt, dt, 2)
    tgv.rk_step(cfg, qa, qb, qt, dt, 1)
    torch.cuda.synchronize()


def accuracy_sweep(args):
    """Every mode of the sweep at --n for --accuracy-steps steps, K and
    enstrophy logged every 10 steps in FP64, against the FP64 GPU path (which
    the tests pin to the FP64 oracle).  Workloads: the periodic TGV (dt =
    0.00125 scaled to the grid) or the symmetric TGSym box at the paper's
    M = 0.5, Re = 800, dt = 0.0025 (to t = 20 by default, the paper's full
    run).  Errors: field relative L2 at the end (rho, momentum vector, rho E),
    the dissipation rate -dK/dt from central differences of K (max error / max
    |ref|), the solenoidal dissipation eps^S(t) (max error / max ref), and the
    paper's measure of Sec. 4.2: the mean absolute difference of the
    dissipation at every 0.5 time units, absolute and relative to the mean
    reference value there, for eps^S and -dK/dt."""
    import torch
    import paper_2505_20911_b300 as tgv
    sym = args.accuracy_workload == "tgsym"
    n = args.n
    dt = args.accuracy_dt or (0.0025 if sym else DT_DEFAULT * 256.0 / n)
    if args.accuracy_t_end:
        steps = int(round(args.accuracy_t_end / dt))
    else:
        steps = args.accuracy_steps or (8000 if sym else 2000)
    mach = args.accuracy_mach or (0.5 if sym else 0.1)
    nrec = steps // DIAG_EVERY + 1

    def run(mode, encoding=None):
        cfg = mode_config(tgv, n, mode)
        if sym:
            cfg = cfg.with_(length=math.pi, symmetric=True, re=800.0)
        cfg = cfg.with_(mach=mach)
        if encoding:
            cfg = cfg.with_(encoding=encoding)
        qa = tgv.empty_state(cfg)
        qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
        tgv.tgv_init(cfg, qa)
        diag = torch.empty(nrec, tgv.TGV_DIAG_COUNT, dtype=torch.float64, device="cuda")
        t0 = time.perf_counter()
        par = tgv.rk_step(cfg, qa, qb, qt, dt, steps, DIAG_EVERY, diag, tgv.empty_workspace(cfg))
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        q = (qb if par else qa).double()
        if cfg.encoding == "offset":
            q[0] += 1.0
            q[4] += 1.0 / (cfg.gamma * (cfg.gamma - 1.0) * cfg.mach ** 2)
        d = diag.cpu()
        del qa, qb, qt
        torch.cuda.empty_cache()
        return q, d[:, 0].tolist(), d[:, 3].tolist(), el

    q_ref, K_ref, E_ref, el_ref = run("fp64")
    diss = lambda K: [-(K[i + 1] - K[i - 1]) / (2 * DIAG_EVERY * dt) for i in range(1, len(K) - 1)]
    d_ref = diss(K_ref)
    per = max(1, int(round(0.5 / (DIAG_EVERY * dt))))
    at = lambda a: a[per - 1::per]       # -dK/dt samples at t = 0.5, 1, ... (index shift 1)
    out = {"workload": args.accuracy_workload, "n": n, "steps": steps, "dt": dt, "mach": mach,
           "t_end": steps * dt, "reference": "fp64 GPU", "reference_seconds": el_ref,
           "modes": {}}
    # the FP64-compute mode costs a second FP64 run; the paper's TGSym study has no such mode
    skip = ("fp64", "fp32s_fp64c") if sym else ("fp64",)
    cases = [(m, None) for m in SWEEP if m not in skip] + [("fp16_fp32", "plain")]
    if args.accuracy_modes:
        keep = set(args.accuracy_modes.split(","))
        cases = [(m, e) for m, e in cases if m in keep]
    for mode, enc in cases:
        q, K, E, el = run(mode, enc)
        nrm = lambda a: float(torch.linalg.vector_norm(a))
        rec = {
            "rho": nrm(q[0] - q_ref[0]) / nrm(q_ref[0]),
            "momentum": nrm(q[1:4] - q_ref[1:4]) / nrm(q_ref[1:4]),
            "rhoE": nrm(q[4] - q_ref[4]) / nrm(q_ref[4]),
            "dKdt": max(abs(a - b) for a, b in zip(diss(K), d_ref)) / max(abs(b) for b in d_ref),
            "epsS": max(abs(a - b) for a, b in zip(E, E_ref)) / max(abs(b) for b in E_ref),
            "epsS_mean_abs_at_0.5": (sum(abs(E[i] - E_ref[i]) for i in range(0, nrec, per))
                                     / sum(abs(E_ref[i]) for i in range(0, nrec, per))),
            "epsS_mean_abs_diff_at_0.5": (sum(abs(E[i] - E_ref[i]) for i in range(0, nrec, per))
                                          / len(range(0, nrec, per))),
            "dKdt_mean_abs_diff_at_0.5": (sum(abs(a - b) for a, b in zip(at(diss(K)), at(d_ref)))
                                          / max(1, len(at(d_ref)))),
            "dKdt_mean_abs_at_0.5": (sum(abs(a - b) for a, b in zip(at(diss(K)), at(d_ref)))
                                     / max(1e-300, sum(abs(b) for b in at(d_ref)))),
            "seconds": el,
        }
        out["modes"][mode + ("" if enc is None else f"[{enc}]")] = rec
        del q
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        # nvidia-smi's start-up (driver and NVML initialisation) must not
        # overlap the timed region: wait for its first sample
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < 10.0:
            time.sleep(0.05)
        time.sleep(0.2)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
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
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- our GPU arm
def alg_bytes_per_point_step(cfg, torch):
    s = torch.tensor([], dtype=cfg.q_dtype).element_size()
    st = torch.tensor([], dtype=cfg.qt_dtype).element_size()
    # per step: Q read+written by all 3 stages (30 s), Qt written by stages 1-2
    # and read by stages 2-3 (20 st)
    return 30 * s + 20 * st


def mode_config(tgv, n, mode):
    return tgv.Config(n=n, mode=mode, encoding="offset" if mode in OFFSET_MODES else "plain")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def stage_source_sha():
    """First 16 hex digits of the SHA-256 of the stage kernel's source with its
    comments and blank lines removed (a comment edit keeps a capture valid)."""
    src = open(STAGE_SRC).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    code = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def profile_traffic(mode, n):
    """dram read+write bytes per stage launch from the committed ncu summary,
    if the stage kernel source is unchanged since the capture; else None."""
    path = os.path.join(ROOT, "profiles", f"stage_kernel_{mode}_{n}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    sha = stage_source_sha()
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("stage_source_sha256_16") != sha:
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def profile_instr_per_point(mode, n):
    """Mean thread instructions per grid point and stage launch from the committed
    ncu summary (if the stage kernel source is unchanged since the capture)."""
    path = os.path.join(ROOT, "profiles", f"stage_kernel_{mode}_{n}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    if profile_traffic(mode, n) is None:  # stale or missing capture
        return None
    for line in text.splitlines():
        if line.startswith("| thread instructions per grid point"):
            cells = [c.strip() for c in line.strip().strip("|").split("|")[1:]]
            try:
                vals = [float(c) for c in cells if c]
                return sum(vals) / len(vals)
            except ValueError:
                return None
    return None


def op_tally_flops(split: str = "blaisdell"):
    """Flops per grid point and RK stage counted from the oracle's formulas
    (the committed summary written by tests/op_tally.py), or None."""
    try:
        text = open(os.path.join(ROOT, "profiles", "op_tally.md")).read()
    except OSError:
        return None
    m = re.search(rf"flops_per_point_stage_{split}: `(\d+)`", text)
    return float(m.group(1)) if m else None


def fp32_peak_tflops(sms: int, sm_mhz: float) -> float:
    """FP32 peak from the unit counts and clock: SMs x 128 FP32 lanes x 2 flops
    (one fused multiply-add) per cycle at the given SM clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def reduce_max(v: float, dist, device) -> float:
    """Max of a per-rank scalar over all ranks (the timing rule: the slowest
    rank's time); identity without a process group."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(points_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Weak-scaling aggregate: all ranks' point-steps over the slowest rank's time."""
    return world * points_per_rank * steps / (max_ms * 1e-3)


def run_ours(args, rank, world, local):
    import torch
    import paper_2505_20911_b300 as tgv

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import datetime
        import torch.distributed as dist
        # a short timeout: a mismatched exchange ends in an error, not a hang
        dist.init_process_group("nccl", device_id=dev, timeout=datetime.timedelta(seconds=120))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        return reduce_max(v, dist, dev)

    n, dt, K, W = args.n, DT_DEFAULT * (256.0 / args.n), args.steps, max(args.warmup, 3)
    stream = torch.cuda.current_stream()

    def setup(mode):
        cfg = mode_config(tgv, n, mode)
        qa = tgv.empty_state(cfg, dev)
        qb = torch.empty_like(qa)
        qt = tgv.empty_qt(cfg, dev)
        ws = tgv.empty_workspace(cfg, dev)
        tgv.tgv_init(cfg, qa)
        return cfg, qa, qb, qt, ws

    def timed_steps(cfg, qa, qb, qt, ws, steps, diag_every):
        nrec = steps // diag_every + 1 if diag_every else 0
        diag = torch.empty(max(nrec, 1), tgv.TGV_DIAG_COUNT, dtype=torch.float64, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        par = tgv.rk_step(cfg, qa, qb, qt, dt, steps, diag_every, diag if nrec else None, ws,
                          stream)
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1), par, diag, nrec

    # ---- headline mode: warm-up, then the timed region with clock sampling
    cfg, qa, qb, qt, ws = setup(HEADLINE)
    tgv.rk_step(cfg, qa, qb, qt, dt, W, DIAG_EVERY, torch.empty(W // DIAG_EVERY + 1,
                tgv.TGV_DIAG_COUNT, dtype=torch.float64, device=dev), ws, stream)
    # every kernel of the timed region has run once before it (the standalone
    # diagnostics of the last state runs only when K is a multiple of 10)
    tgv.diagnostics_reduce(cfg, qa, torch.empty(tgv.TGV_DIAG_COUNT, dtype=torch.float64,
                                                device=dev), ws, stream)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms, par, diag, nrec = timed_steps(cfg, qa, qb, qt, ws, K, DIAG_EVERY)
    ms = max_over_ranks(ms)
    ms_step = ms / K
    value = whole_job_value(n ** 3, K, world, ms)
    replicas = None
    slab_run = None
    if world > 1:
        # the method's parallel strategy: one n^3 box in z-slabs over the
        # ranks (strong scaling), ghosts exchanged before every stage; the
        # replica figure above is kept beside it
        replicas = {"value": value, "ms_per_step": ms / K, "scaling": "weak",
                    "what": f"one independent {n}^3 box per rank, no data-path collective"}
        try:
            slab_run = run_slab(tgv, torch, dist, rank, world, dev, n, dt, K, W, barrier,
                                max_over_ranks)
            value, ms = slab_run["value"], slab_run["ms"]
        except Exception as exc:  # report, do not hide: the line then carries the replicas
            slab_run = {"error": repr(exc)}
    diag_last = diag[nrec - 1].cpu().tolist()
    # 3 stage launches per step (the first of each logged step fuses the
    # diagnostics), one final-reduction launch per logged step, and the
    # standalone two-pass reduction of the last state when K % 10 == 0
    launches = 3 * K + (K + DIAG_EVERY - 1) // DIAG_EVERY + (2 if K % DIAG_EVERY == 0 else 0)

    # ---- roofline of the dominant kernel (the fused stage), on the same stream
    # the timed region's stage kernels (rk_step's three stages, without the
    # diagnostics), launched back to back on the bench stream: the event time
    # over 3 * reps launches is their average duration
    reps = max(10, min(K, 60))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    tgv.rk_step(cfg, qa, qb, qt, dt, reps, 0, None, ws, stream)
    e1.record(stream)
    barrier()
    stage_ms = e0.elapsed_time(e1) / (3 * reps)
    bpp = alg_bytes_per_point_step(cfg, torch)
    alg_bytes_launch = bpp / 3.0 * n ** 3
    peaks, peak_kind = measured_peaks()
    achieved = alg_bytes_launch / (stage_ms * 1e-3) / 1e9
    traffic = profile_traffic(HEADLINE, n)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                "traffic": traffic,
                "traffic_note": (f"ncu dram read+write per launch from profiles/stage_kernel_"
                                 f"{HEADLINE}_{n}.md, captured on this stage kernel source")
                                if traffic is not None else
                                (f"null: profiles/stage_kernel_{HEADLINE}_{n}.md is missing or was "
                                 f"captured on another version of the stage kernel source"),
                "peak_kind": f"{peak_kind} hbm_gbs",
                "kernel": "stage_kernel (fused RHS + RK stage; rk_step's three stages, mean launch)",
                "stage_ms": round(stage_ms, 4),
                "alg_bytes_per_launch": alg_bytes_launch}
    # the arithmetic ceiling: the oracle-counted flops of one stage at this
    # run's stage time against the FP32 peak of the unit counts and clock
    flops_pp = op_tally_flops(cfg.split)
    roof_alu = None
    if flops_pp is not None:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_alu = fp32_peak_tflops(sms, peaks.get("sm_max_mhz", 2032.0))
        ach_alu = flops_pp * n ** 3 / (stage_ms * 1e-3) / 1e12
        ffma2 = tgv.probe_fma_tflops("ffma2")
        roof_alu = {"bound": "alu", "achieved": round(ach_alu, 2), "peak": round(peak_alu, 2),
                    "unit": "TFLOP/s", "frac": round(ach_alu / peak_alu, 4),
                    "peak_measured_ffma2": round(ffma2, 2),
                    "frac_of_measured": round(ach_alu / ffma2, 4),
                    "flops_per_point_stage": flops_pp,
                    "flops_source": "profiles/op_tally.md: the oracle's formulas, each distinct "
                                    "operation counted once (tests/op_tally.py)",
                    "peak_kind": f"derived: {sms} SMs x 128 FP32 lanes x 2 flops (FMA) x "
                                 f"{peaks.get('sm_max_mhz', 2032.0):.0f} MHz"}
    # the ceiling the FP16-storage stage actually meets: instruction issue (148 SMs x
    # 4 schedulers x one warp instruction of 32 threads per clock at 2032 MHz)
    ipp = profile_instr_per_point(HEADLINE, n)
    issue_roof = None
    if ipp is not None:
        peak_issue = 148 * 4 * 32 * 2.032e9 / 1e9
        ach_issue = ipp * n ** 3 / (stage_ms * 1e-3) / 1e9
        issue_roof = {"bound": "issue", "achieved": round(ach_issue, 1), "peak": round(peak_issue, 1),
                      "unit": "G thread-instructions/s", "frac": round(ach_issue / peak_issue, 4),
                      "instr_per_point": round(ipp, 1),
                      "source": "thread instructions per point from the committed ncu summary, "
                                "time from this run; peak from the unit counts at the maximum "
                                "SM clock"}
    del qa, qb, qt
    torch.cuda.empty_cache()

    # ---- e2e through the public host-buffer calls: every step's H2D of Q and
    # D2H of Q + diagnostics inside the timed region, from pinned host memory.
    # Headline: the pipelined call (tgv_run_host_stream, copies overlapped with
    # the steps of another state on a second stream); also the single call.
    e2e = None
    try:
        cfg = mode_config(tgv, n, HEADLINE)
        qdev = tgv.empty_state(cfg, dev)
        tgv.tgv_init(cfg, qdev)
        count, steps_per_call = 8, DIAG_EVERY
        nrec = steps_per_call // DIAG_EVERY + 1
        qh_in = [qdev.cpu().pin_memory() for _ in range(count)]
        qh_out = qh_in  # each state comes back into its own host buffer
        del qdev
        dh = torch.empty(count * nrec * tgv.TGV_DIAG_COUNT, dtype=torch.float64).pin_memory()
        qbytes = tgv.tgv_state_bytes(cfg)
        per_step = {"h2d_bytes_per_step": qbytes / steps_per_call,
                    "d2h_bytes_per_step": (qbytes + nrec * tgv.TGV_DIAG_COUNT * 8) / steps_per_call}
        # single call: one state per call, copies and steps in sequence
        wsb = tgv.tgv_run_host_workspace_bytes(cfg, steps_per_call, DIAG_EVERY)
        dws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        d1 = dh[:nrec * tgv.TGV_DIAG_COUNT]
        tgv.tgv_run_host(cfg, qh_in[0], qh_out[0], dt, steps_per_call, DIAG_EVERY, d1, dws, stream)
        barrier()
        t0 = time.perf_counter()
        for i in range(count):
            tgv.tgv_run_host(cfg, qh_in[i], qh_out[i], dt, steps_per_call, DIAG_EVERY, d1, dws,
                             stream)
        barrier()
        el1 = max_over_ranks(time.perf_counter() - t0)
        del dws
        # pipelined call
        wsb = tgv.tgv_run_host_stream_workspace_bytes(cfg, steps_per_call, DIAG_EVERY)
        dws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        copy_stream = torch.cuda.Stream(device=dev)
        tgv.tgv_run_host_stream(cfg, qh_in[:2], qh_out[:2], dt, steps_per_call, DIAG_EVERY, dh,
                                dws, stream, copy_stream)
        barrier()
        t0 = time.perf_counter()
        tgv.tgv_run_host_stream(cfg, qh_in, qh_out, dt, steps_per_call, DIAG_EVERY, dh, dws,
                                stream, copy_stream)
        barrier()
        el = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": world * n ** 3 * steps_per_call * count / el, "unit": UNIT, **per_step,
               "call": f"tgv_run_host_stream: {count} states from pinned host memory, each H2D "
                       f"of Q, {steps_per_call} RK3 steps with FP64 diagnostics, D2H of Q and "
                       f"diagnostics; copies on a second stream overlap the other state's steps",
               "single_call": {"value": world * n ** 3 * steps_per_call * count / el1,
                               "call": "tgv_run_host: one state per call, copies and steps in "
                                       "sequence"}}
        del dws
        torch.cuda.empty_cache()
    except Exception as exc:  # report, do not hide
        e2e = {"value": None, "unit": UNIT, "error": repr(exc)}

    # ---- the rest of the precision sweep, each next to FP64
    modes = {}
    if not args.no_sweep and world == 1:
        for mode in SWEEP:
            c, a, b, t, w = setup(mode)
            steps = 4 if c.compute_dtype == torch.float64 and mode != "spdp" else 20
            tgv.rk_step(c, a, b, t, dt, 2, 0, None, None, stream)
            # the median of five timed runs (the paper averages five runs)
            runs = []
            for _ in range(SWEEP_RUNS):
                r_ms, _, _, _ = timed_steps(c, a, b, t, w, steps, DIAG_EVERY if steps >= 10 else 0)
                runs.append(max_over_ranks(r_ms))
            m_ms = statistics.median(runs)
            v = world * n ** 3 * steps / (m_ms * 1e-3)
            bpp_m = alg_bytes_per_point_step(c, torch)
            modes[mode] = {"value": v, "ms_per_step": m_ms / steps, "steps": steps,
                           "runs": SWEEP_RUNS, "spread": (max(runs) - min(runs)) / m_ms,
                           "alg_GBs": bpp_m * v / world / 1e9,
                           "hbm_frac": bpp_m * v / world / 1e9 / peaks["hbm_gbs"],
                           "bytes_per_point_step": bpp_m}
            del a, b, t, w
            torch.cuda.empty_cache()
        for mode in modes:
            modes[mode]["vs_fp64"] = modes[mode]["value"] / modes["fp64"]["value"]

    extra = {} if (args.no_sweep or world > 1) else extra_workloads(args, tgv, torch, dev, stream,
                                                                   peaks)

    if dist is not None:
        dist.destroy_process_group()
    return {
        "value": value, "ms_per_step": ms / K, "replicas": replicas, "slab": slab_run,
        "roofline": roofline,
        "roofline_issue": issue_roof, "roofline_alu": roof_alu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clk.summary(), "modes": modes,
        "diag_last": dict(zip(tgv.DIAG_NAMES, diag_last)), "dt": dt, **extra,
    }


def run_slab(tgv, torch, dist, rank, world, dev, n, dt, K, W, barrier, max_over_ranks):
    """One n^3 box of the headline mode split into z-slabs, one per rank: every
    RK stage exchanges two ghost planes per field with each neighbour (NCCL
    point-to-point) and runs the slab stage kernel; diagnostics every 10
    steps, all-reduced.  Time: K steps, max over ranks."""
    from paper_2505_20911_b300 import slab
    cfg = mode_config(tgv, n, HEADLINE)
    z0, nz = slab.slab_bounds(n, world, rank)
    dom = slab.SlabDomain(cfg, [(z0, nz)], rank, world, dist, dev)
    dom.init()
    diag = torch.empty(tgv.TGV_DIAG_COUNT, dtype=torch.float64, device=dev)

    def steps(count):
        for m in range(count):
            if m % DIAG_EVERY == 0:
                dom.step(dt, 1, diag=diag)
                dist.all_reduce(diag)
            else:
                dom.step(dt, 1)

    steps(W)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record()
    steps(K)
    e1.record()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    halo_bytes = 2 * 2 * 5 * n * n * torch.tensor([], dtype=cfg.q_dtype).element_size()
    return {"value": n ** 3 * K / (ms * 1e-3), "ms": ms, "ms_per_step": ms / K,
            "scaling": "strong", "planes_per_rank": nz,
            "halo_bytes_per_stage_per_rank": halo_bytes,
            "what": f"one {n}^3 box in z-slabs over {world} ranks, 2 ghost planes per field "
                    f"exchanged with each neighbour before every RK stage (NCCL), diagnostics "
                    f"all-reduced every {DIAG_EVERY} steps",
            "K": dict(zip(tgv.DIAG_NAMES, diag.cpu().tolist()))["K"]}


def extra_workloads(args, tgv, torch, dev, stream, peaks):
    """The other configurations' throughput (each timed with CUDA events):
    512^3 half-single vs single (dt = 0.000625), the 64^3 adjoint (FP64 and
    FP32-forward / FP64-adjoint, 200 steps, checkpoint every 20) and the
    48-instance ensemble (FP32, 500 steps) against the sum of solo runs."""
    out = {}

    def ev_time(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # 512^3 (config: FP16 storage / FP32 compute against FP32 / FP32)
    big = {}
    for mode in ("fp16_fp32", "fp32"):
        cfg = mode_config(tgv, 512, mode)
        qa = tgv.empty_state(cfg, dev)
        qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg, dev)
        tgv.tgv_init(cfg, qa)
        tgv.rk_step(cfg, qa, qb, qt, 0.000625, 3, 0, None, None, stream)
        steps = 10
        ms = ev_time(lambda: tgv.rk_step(cfg, qa, qb, qt, 0.000625, steps, 0, None, None, stream))
        v = 512 ** 3 * steps / (ms * 1e-3)
        bpp = alg_bytes_per_point_step(cfg, torch)
        big[mode] = {"value": v, "ms_per_step": ms / steps, "alg_GBs": bpp * v / 1e9,
                     "hbm_frac": bpp * v / 1e9 / peaks["hbm_gbs"]}
        del qa, qb, qt
        torch.cuda.empty_cache()
    big["fp16_vs_fp32"] = big["fp16_fp32"]["value"] / big["fp32"]["value"]
    out["n512"] = big

    # the paper's own workload: TGSym 256^3 (pi^3 box with mirror planes),
    # M = 0.5, Re = 800, dt = 0.0025; ms per iteration (one RK3 step) per mode,
    # beside the paper's A100 Storesome times (context, other hardware)
    paper_ms = {"fp64": 50.31, "spdp": 37.60, "fp32": 25.00, "hpsp": 22.13, "fp16": 18.67}
    tgs = {}
    for mode in ("fp64", "spdp", "fp32", "hpsp", "fp16_fp32", "fp16"):
        cfg = tgv.Config(n=256, mode=mode, length=math.pi, symmetric=True, mach=0.5, re=800.0,
                         encoding="offset" if mode in OFFSET_MODES else "plain")
        qa = tgv.empty_state(cfg, dev)
        qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg, dev)
        tgv.tgv_init(cfg, qa)
        tgv.rk_step(cfg, qa, qb, qt, 0.0025, 2, 0, None, None, stream)
        steps = 4 if mode == "fp64" else 20
        ms = ev_time(lambda: tgv.rk_step(cfg, qa, qb, qt, 0.0025, steps, 0, None, None, stream))
        rec = {"ms_per_iteration": ms / steps, "value": 256 ** 3 * steps / (ms * 1e-3)}
        if mode in paper_ms:
            rec["paper_a100_storesome_ms"] = paper_ms[mode]
            rec["speedup_vs_paper_a100"] = paper_ms[mode] / rec["ms_per_iteration"]
        tgs[mode] = rec
        del qa, qb, qt
        torch.cuda.empty_cache()
    out["tgsym_256"] = tgs

    # small grids are launch-bound: 32^3 FP32 per step, direct launches against
    # a CUDA graph of 10 rk_step steps captured by the caller
    cfg = tgv.Config(n=32, mode="fp32")
    qa = tgv.empty_state(cfg)
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    tgv.tgv_init(cfg, qa)
    dt32 = 0.5 * tgv.tgv_dt_max(cfg)
    tgv.rk_step(cfg, qa, qb, qt, dt32, 4, 0, None, None, stream)
    direct_ms = ev_time(lambda: tgv.rk_step(cfg, qa, qb, qt, dt32, 100, 0, None, None, stream)) / 100
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        tgv.rk_step(cfg, qa, qb, qt, dt32, 10, 0, None, None, side)
    graph_ms = ev_time(lambda: [graph.replay() for _ in range(10)]) / 100
    out["graph_32"] = {"direct_ms_per_step": direct_ms, "graph_ms_per_step": graph_ms,
                       "speedup": direct_ms / graph_ms}
    del qa, qb, qt, graph

    # the z-slab decomposition's own cost on one GPU: the headline 256^3 box as
    # P slabs on this device (ghost planes exchanged by device copies before
    # every stage, the P slab-stage launches of a stage one after another)
    # against the whole box, 20 steps each.  With P ranks each would run one
    # slab, so (total - exchange) / P estimates a rank's kernel time per step
    # (transfers not included) and whole / (total - exchange) the strong-scaling
    # efficiency of the kernels alone.
    from paper_2505_20911_b300 import slab
    cfg = mode_config(tgv, 256, HEADLINE)
    dt256 = DT_DEFAULT
    local = {}
    qa = tgv.empty_state(cfg)
    qb, qt = torch.empty_like(qa), tgv.empty_qt(cfg)
    tgv.tgv_init(cfg, qa)
    tgv.rk_step(cfg, qa, qb, qt, dt256, 3, 0, None, None, stream)
    local["whole_box_ms_per_step"] = ev_time(
        lambda: tgv.rk_step(cfg, qa, qb, qt, dt256, 20, 0, None, None, stream)) / 20
    del qa, qb, qt
    for nslab in (2, 4, 8):
        dom = slab.SlabDomain(cfg, [slab.slab_bounds(256, nslab, r) for r in range(nslab)])
        dom.init(stream)
        dom.step(dt256, 3, stream=stream)
        tot = ev_time(lambda: dom.step(dt256, 20, stream=stream)) / 20
        exch = ev_time(lambda: [dom.exchange(stream) for _ in range(60)]) / 20
        local[f"slabs_{nslab}"] = {"ms_per_step": tot, "exchange_ms_per_step": exch,
                                   "per_rank_kernel_ms_per_step": (tot - exch) / nslab,
                                   "kernel_efficiency": local["whole_box_ms_per_step"] / (tot - exch)}
        del dom
    torch.cuda.empty_cache()
    out["slab_local_256"] = local

    # adjoint: 64^3, 200 steps, checkpoint every 20
    adj = {}
    for mode in ("fp64", "fp32"):
        cfg = tgv.Config(n=64, mode=mode)
        q0 = tgv.empty_state(cfg, dev)
        tgv.tgv_init(cfg, q0)
        g = torch.empty((3, 64, 64, 64), dtype=torch.float64, device=dev)
        j = torch.empty(1, dtype=torch.float64, device=dev)
        ws = torch.empty(tgv.tgv_grad_workspace_bytes(cfg, 200, 20), dtype=torch.uint8, device=dev)
        tgv.tgv_grad_final_ke(cfg, q0, 0.004, 200, 20, g, j, ws, stream)
        ms = ev_time(lambda: tgv.tgv_grad_final_ke(cfg, q0, 0.004, 200, 20, g, j, ws, stream))
        qa, qb, qt = q0.clone(), torch.empty_like(q0), tgv.empty_qt(cfg, dev)
        fwd = ev_time(lambda: tgv.rk_step(cfg, qa, qb, qt, 0.004, 200, 0, None, None, stream))
        adj["fp64" if mode == "fp64" else "fp32_fwd_fp64_adj"] = {
            "grad_ms": ms, "forward_ms": fwd, "grad_over_forward": ms / fwd, "J": float(j[0])}
        del q0, g, ws, qa, qb, qt
        torch.cuda.empty_cache()
    out["adjoint_64"] = adj

    # ensemble: 48 instances, FP32, 500 steps, one graph of 10 steps replayed
    cfgs, dts = tgv.ensemble_instances()
    bufs = []
    for c in cfgs:
        q = tgv.empty_state(c, dev)
        tgv.tgv_init(c, q)
        bufs.append((q, torch.empty_like(q), tgv.empty_qt(c, dev)))
    ens = tgv.Ensemble(cfgs, [b[0] for b in bufs], [b[1] for b in bufs], [b[2] for b in bufs],
                       dts, steps_per_graph=10, stream=stream)
    info = ens.info()
    ens.run(1, stream)
    ms = ev_time(lambda: ens.run(50, stream))
    pts = sum(c.n ** 3 for c in cfgs)
    solo = 0.0
    for c, d, b in zip(cfgs, dts, bufs):
        cc = c.with_(tile=info["tile"], zchunk=min(c.n, info["zchunk_target"]))
        solo += ev_time(lambda: tgv.rk_step(cc, b[0], b[1], b[2], d, 500, 0, None, None, stream))
    ens.close()
    out["ensemble_48"] = {"value": pts * 500 / (ms * 1e-3), "unit": UNIT, "ms": ms,
                          "points": pts, "steps": 500, "solo_sum_ms": solo,
                          "speedup_vs_solo_sum": solo / ms, **info}
    del bufs
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------ CPU oracle legs
def oracle_sample(n_sample, steps=1, dt=None):
    """Time `steps` RK3 steps of the FP64 oracle on an n_sample^3 TGV."""
    import oracle
    flow = oracle.Flow(n=n_sample)
    q = oracle.initial_condition(flow)
    dt = dt if dt is not None else DT_DEFAULT * 256.0 / n_sample
    t0 = time.perf_counter()
    for _ in range(steps):
        q = oracle.rk3_step(flow, q, dt)
    el = time.perf_counter() - t0
    return n_sample ** 3 * steps / el, el


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(n):
    """The oracle as it stands on the host cores: one RK substep (a third of a
    step) on the full n^3 grid with all threads (the line's value), the
    32^3 x 100-step run of the small configuration in full, with all threads
    and on one thread."""
    import torch
    import oracle
    threads = torch.get_num_threads()
    flow = oracle.Flow(n=n)
    q = oracle.initial_condition(flow)
    qt = torch.zeros_like(q)
    t0 = time.perf_counter()
    oracle.rk_substep(flow, q, qt, 0, DT_DEFAULT * 256.0 / n)
    el = time.perf_counter() - t0
    small, _ = oracle_sample(32, 100, dt=0.004)
    torch.set_num_threads(1)
    try:
        single, el1 = oracle_sample(32, 100, dt=0.004)
    finally:
        torch.set_num_threads(threads)
    return {"value": n ** 3 / (3.0 * el), "unit": UNIT, "cores": threads, "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "sample": f"1 RK substep (1/3 step) of the FP64 oracle on the full {n}^3 TGV grid, "
                      f"{el:.1f} s on {threads} host threads, scaled to point-steps/s",
            "tgv32_100_steps_all_core": {"value": small, "unit": UNIT, "threads": threads,
                                         "sample": "32^3 TGV, dt 0.004, 100 RK3 steps in full"},
            "tgv32_single_thread": {"value": single, "unit": UNIT, "threads": 1,
                                    "seconds": el1,
                                    "sample": "32^3 TGV, dt 0.004, 100 RK3 steps in full on one thread"}}


def run_reference(args, rank, world):
    """The oracle (plain FP64 PyTorch CPU code) on the same metric and config;
    each step is one RK3 step on an n_s^3 TGV sized so K+W steps fit ~150 s."""
    import torch
    if rank != 0:
        return None
    K, W = args.steps, max(args.warmup, 3)
    # calibrate the per-point cost on a small grid, then size the sample
    rate, _ = oracle_sample(24, 1)
    budget = 150.0 / (K + W)
    n_s = 16
    for cand in (16, 24, 32, 48, 64, 96, 128, 192, 256):
        if cand ** 3 / rate <= budget:
            n_s = cand
    import oracle
    flow = oracle.Flow(n=n_s)
    q = oracle.initial_condition(flow)
    dt = DT_DEFAULT * 256.0 / n_s
    for _ in range(W):
        q = oracle.rk3_step(flow, q, dt)
    t0 = time.perf_counter()
    for _ in range(K):
        q = oracle.rk3_step(flow, q, dt)
    el = time.perf_counter() - t0
    value = n_s ** 3 * K / el
    cores = torch.get_num_threads()
    sample = f"{K} RK3 steps of the FP64 oracle on a {n_s}^3 TGV (same physics), {cores} threads"
    return {"value": value, "ms_per_step": el * 1e3 / K, "sample": sample, "cores": cores}


def probe_peaks():
    import torch
    import paper_2505_20911_b300 as tgv
    out = {k: tgv.probe_fma_tflops(k) for k in ("ffma", "ffma2", "hfma2")}
    props = torch.cuda.get_device_properties(0)
    peaks, _ = measured_peaks()
    out["derived_fp32_fma_peak"] = fp32_peak_tflops(props.multi_processor_count,
                                                    peaks.get("sm_max_mhz", 2032.0))
    out["unit"] = "TFLOP/s"
    return out


def main():
    args = parse()
    if args.probe_peaks:
        print(json.dumps(probe_peaks()), flush=True)
        return
    if args.profile_case:
        profile_case(args)
        return
    if args.accuracy:
        accuracy_sweep(args)
        return
    rank, world, local = dist_env()
    base = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "data": "synthetic (analytic Taylor-Green initial field)"}
    config = {"workload": f"TGV {args.n}^3 precision sweep (headline: HPSP, Q FP32 / Qt FP16 "
                          f"storage, FP32 compute)",
              "n": args.n, "M": 0.1, "Re": 1600.0, "Pr": 0.71, "gamma": 1.4,
              "dt": DT_DEFAULT * 256.0 / args.n, "diag_every": DIAG_EVERY,
              "split": "blaisdell", "l2": "inputs larger than L2: Q in, Q out and Qt of the "
                                          "headline mode are each above 126 MB at 256^3",
              "parallelism": "one GPU" if world == 1 else f"z-slabs x{world} (one box)"}
    if args.impl == "reference":
        ref = run_reference(args, rank, world)
        if rank == 0:
            line = dict(base, impl="reference", value=ref["value"],
                        ms_per_step=ref["ms_per_step"], dtype="f64", config=config,
                        cpu_baseline={"value": ref["value"], "unit": UNIT, "cores": ref["cores"],
                                      "kind": "oracle", "sample": ref["sample"]},
                        e2e={"value": ref["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                             "d2h_bytes_per_step": 0})
            print(json.dumps(line), flush=True)
        return
    res = run_ours(args, rank, world, local)
    if rank != 0:
        return
    line = dict(base, value=res["value"], ms_per_step=res["ms_per_step"], dtype="f32",
                config=config, roofline=res["roofline"], roofline_issue=res["roofline_issue"],
                roofline_alu=res["roofline_alu"],
                e2e=res["e2e"], gpu_launches=res["gpu_launches"], clocks=res["clocks"], modes=res["modes"],
                diag_last=res["diag_last"])
    for key in ("replicas", "slab", "n512", "tgsym_256", "graph_32", "slab_local_256", "adjoint_64",
                "ensemble_48"):
        if res.get(key) is not None:
            line[key] = res[key]
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.n)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
