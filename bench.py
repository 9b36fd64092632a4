"""Benchmark: cell-updates per second of the SSP-RK3 step on one GB300.

Workload (default): decaying relativistic Alfvenic turbulence on a periodic 768^3
grid of a (2 pi)^3 box -- rho0 = 1, B0 along z with sigma0 = B0^2/rho0 = 10,
beta0 = 1, random-phase modes with 1 <= |k| <= 4, mean |dB|/B0 = 0.5, largest
Lorentz factor 5, seeded -- with UCT and high-order INT/DER on, MP5, SSP-RK3 and
CFL 0.4.  One "step" is one full SSP-RK3 step (three substeps of the whole
right-hand side) over all cells; value = cells * steps / time of the FP64 path.
The same line carries the mixed path and the mixed path with the learned Newton
guess on the same workload and step count (rate, Newton iterations, fallback
rate, L1 distance to the FP64 state), the end-to-end rate through the C ABI with
host buffers, the roofline of the dominant kernel and the oracle on the host.

The state (about 200 GB in FP64) is far larger than the 129 MB L2, so no flush is
needed between timed steps.  Prints one JSON line.
"""
import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("cell-updates/s per GB300 (FP64 vs mixed+learned C2P) at stated L1 error; "
          "% HBM peak")
UNIT = "cell-updates/s"
SEED = 2401_03008

# Algorithmic per-unit costs of each kernel kind: one unit is one cell, face or edge
# of the launch.  Bytes: each array element read or written once (stencil
# neighbours come from cache).  FLOPs: FP64 (or FP32 for the mixed path's FP32
# kernels) floating-point operations the kernel performs per unit, an FMA counted
# as 2, as counted by ncu (sass thread instructions, add/mul/fma) on the 192^3
# turbulence and read from profiles/flops_per_unit.json.
R64, R32 = 8, 4


def bytes_per_unit(kind, r):
    return {
        "int_c2p": 5 * 8 + 3 * 8 + 8 + 8 * r + 8,
        "flux_x": 8 * r + 8 + 5 * r + 6 * r, "flux_y": 8 * r + 8 + 5 * r + 6 * r,
        "flux_z": 8 * r + 8 + 5 * r + 6 * r,
        "der_x": 5 * r + 5 * r, "der_y": 5 * r + 10 * r, "der_z": 5 * r + 10 * r,
        "uct_x": 8 * r + 16 + r, "uct_y": 8 * r + 16 + r, "uct_z": 8 * r + 16 + r,
        "rk_curl": 5 * r + 3 * r + 3 * 64,
        # mixed path: the inversion fused with the x sweep (U, B faces, W in and out,
        # the normal field; primitives, rhs and UCT face data out) and the fused y/z
        # sweeps (primitives and the normal field in, rhs read and written, face data)
        "c2p_sweep_x": 5 * 8 + 3 * 8 + 2 * 8 + r + 8 * r + 5 * r + 6 * r,
        "sweep_y": 8 * r + r + 10 * r + 6 * r, "sweep_z": 8 * r + r + 10 * r + 6 * r,
    }.get(kind)


# kernels bound by the FP64 pipe on the mixed path (the inversion and the RK
# accumulation stay FP64); every kernel of the FP64 path is
FP64_BOUND = ("int_c2p", "c2p_sweep_x", "rk_curl")


FLOPS_PER_UNIT = {}  # filled from the ncu counts (profiles/), kernel -> flops per unit


def load_flops_table():
    p = os.path.join(ROOT, "profiles", "flops_per_unit.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device=0):
        self.samples = []
        self.proc = None
        self.device = device

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.samples.append(parts)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _cpu_model():
    """the host CPU's model name and core count (for the oracle timings)"""
    name = platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return "%s, %d cores" % (name, os.cpu_count() or 1)


def job_rate(ms, units_per_rank, world, device="cuda"):
    """The slowest rank's timed milliseconds (max over the process group) and the
    whole-job rate: the units all ranks processed over that time.  Replicas share
    no data; this reduction is the only collective of the run."""
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    return ms, world * units_per_rank / (ms * 1e-3)


def workload_state(n, wave, uct=1):
    """The Alfven-wave workloads (host arrays): (wave, (prim5, bface, apot))."""
    from paper_2401_03008_gb300 import workloads as wl
    m = {"oblique": (1, 1, 1), "x": (1, 0, 0)}[wave]
    c = wl.CPA(n, n, n, m=m)
    if not uct:
        return c, (c.prim5(), c.bcell(), None)
    return c, (c.prim5(), c.bface_background(), c.apot())


def turbulence_state(n, lorentz_max, seed=SEED, device=None):
    """The decaying-turbulence workload on an n^3 grid: (prim5, bface, apot), numpy
    arrays, or float64 tensors generated on ``device`` (the 768^3 synthesis would
    take minutes on the host)."""
    from paper_2401_03008_gb300 import workloads as wl
    tb = wl.Turbulence(n, seed=seed, lorentz_max=lorentz_max, device=device)
    st = (tb.prim5(), tb.bface_background(), tb.apot())
    tb.release()
    return st


TURB_L = (2 * math.pi,) * 3


def state_for(args, n, device=None):
    """(box, (prim5, bface, apot)) of the selected workload on an n^3 grid."""
    if args.workload == "turbulence":
        return TURB_L, turbulence_state(n, args.lorentz_max, device=device)
    _, st = workload_state(n, args.wave, args.uct)
    return (1.0, 1.0, 1.0), st


def workload_name(args, n):
    if args.workload == "turbulence":
        return ("decaying relativistic Alfvenic turbulence, %d^3 periodic (2 pi)^3 box, "
                "sigma0 = 10, beta0 = 1, mean |dB|/B0 = 0.5, max Lorentz factor %g, "
                "1 <= |k| <= 4, seed %d; UCT on, HO on, MP5, CFL 0.4, SSP-RK3"
                % (n, args.lorentz_max, SEED))
    return ("relativistic circularly polarised Alfven wave, k along %s, %d^3 periodic, "
            "UCT %s, HO %s, %s, CFL 0.4, SSP-RK%d"
            % ({"oblique": "(1,1,1)", "x": "x"}[args.wave], n,
               "on" if args.uct else "off", "on" if args.ho else "off",
               "MP5" if args.rec == "mp5" else "linear (MC)", args.rk))


def workload_config(args):
    bpc = 448 if args.precision == "fp64" else 304
    return {"workload": workload_name(args, args.n), "cells": args.n ** 3,
            "precision": args.precision,
            "l2_flush": "not needed: state of ~%.0f GB >> 129 MB L2" % (args.n ** 3 * bpc / 1e9),
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


def _oracle_sample(args, ns):
    """An oracle grid with the ns^3 sample of the workload."""
    from oracle import oracle as orc
    L, st = state_for(args, ns)
    g = orc.Grid(ns, ns, ns, *L, nthreads=os.cpu_count() or 1, uct=args.uct, ho=args.ho,
                 rec=1 if args.rec == "linear" else 0, rk=args.rk)
    g.set_state(*st)
    return g, st


def _oracle_steps_from_start(args, ns, steps):
    """Seconds of oracle work for `steps` SSP-RK3 steps of the ns^3 sample, each taken
    from the sample's initial state (the reset is outside the timed region), so every
    timed step is the same bounded piece of the workload."""
    g, st = _oracle_sample(args, ns)
    el = 0.0
    for _ in range(steps):
        g.set_state(*st)
        t0 = time.perf_counter()
        bad = g.step(1)
        el += time.perf_counter() - t0
        if bad:
            raise RuntimeError("the oracle's inversion failed on the %d^3 sample (too coarse "
                               "for this workload); choose a larger sample" % ns)
    return el


def run_reference(args, world, rank):
    """The oracle (plain FP64 C, all host cores) on a bounded sample of the same
    workload: one SSP-RK3 step of the --ref-n^3 grid per timed step."""
    if rank != 0:
        return
    nthreads = os.cpu_count() or 1
    ns = args.ref_n
    _oracle_steps_from_start(args, ns, args.warmup)
    el = _oracle_steps_from_start(args, ns, args.steps)
    value = ns ** 3 * args.steps / el
    sample = ("%d^3 grid of the same workload, %d SSP-RK3 steps, each from its initial "
              "state (oracle, %s)" % (ns, args.steps, _cpu_model()))
    cfg = workload_config(args)
    cfg.update({"sample": sample, "cells": ns ** 3})
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def cpu_baseline(args):
    nthreads = os.cpu_count() or 1
    ns, steps = args.cpu_n, args.cpu_steps
    el = _oracle_steps_from_start(args, ns, steps)
    return {"value": ns ** 3 * steps / el, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": "%d^3 grid of the same workload, %d SSP-RK3 steps each from its initial "
                      "state, %.1f s on %s" % (ns, steps, el, _cpu_model())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="turbulence", choices=["turbulence", "wave"])
    ap.add_argument("--n", type=int, default=768)
    ap.add_argument("--lorentz-max", type=float, default=5.0)
    ap.add_argument("--wave", default="oblique", choices=["oblique", "x"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--guess", default="prev", choices=["prev", "cold", "mlp"])
    ap.add_argument("--uct", type=int, default=1, help="0: cell-centred field, no UCT")
    ap.add_argument("--ho", type=int, default=1, help="0: two-point INT and DER")
    ap.add_argument("--rec", default="mp5", choices=["mp5", "linear"])
    ap.add_argument("--rk", type=int, default=3, choices=[2, 3])
    ap.add_argument("--sweeps", default="auto", choices=["auto", "fused", "separate"],
                    help="the mixed path's y/z sweep kernels")
    ap.add_argument("--ref-n", type=int, default=64)
    ap.add_argument("--cpu-n", type=int, default=128)   # about 10 s of oracle work
    ap.add_argument("--cpu-steps", type=int, default=6)
    ap.add_argument("--prof-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--variants", type=int, default=1, help="also time mixed and mixed+learned")
    ap.add_argument("--train-n", type=int, default=128)
    ap.add_argument("--train-steps", type=int, default=12)
    ap.add_argument("--config", type=int, default=0,
                    help="1..5: benchmark-plan configurations; 6: the 2.5-D turbulence run of "
                         "Sec. 5; 7: 2 x 2 x 2 blocks with the wide halo against one grid; "
                         "8: time to accuracy of the FP64 and mixed paths on the Alfven wave")
    ap.add_argument("--config-steps", type=int, default=20)
    ap.add_argument("--config-runs", default="",
                    help="configs 4-5: comma list of precision_guess runs to keep "
                         "(e.g. mixed_prev,mixed_mlp); default all")
    ap.add_argument("--config5-n", type=int, default=768)
    ap.add_argument("--config5-steps", type=int, default=200)
    ap.add_argument("--config5-lorentz-max", type=float, default=3.5,
                    help="largest initial Lorentz factor of the 200-step run (the scheme has "
                         "no floors; from 4 up the run ends in a failed inversion first)")
    ap.add_argument("--config6-n", type=int, default=4096)
    ap.add_argument("--config6-t", type=float, default=20.0)
    ap.add_argument("--config6-out", default="", help="write the spectra (.npz) here")
    args = ap.parse_args()
    if args.workload == "turbulence":
        args.uct, args.ho, args.rec, args.rk = 1, 1, "mp5", 3
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.config:
        return run_config(args)

    import torch
    from paper_2401_03008_gb300 import echo

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    n = args.n
    dev = "cuda:%d" % local
    stream = torch.cuda.Stream()  # the library launches on it; the events are recorded on it
    L, st = state_for(args, n, device=dev)
    s = echo.Solver(n, n, n, L=L, precision=args.precision, device=local, guess=args.guess,
                    stream=stream.cuda_stream, uct=args.uct, ho=args.ho, rec=args.rec,
                    rk_order=args.rk, sweeps=args.sweeps)
    weights, train_info = None, None
    if args.guess == "mlp":
        weights, train_info = train_guess(args)
        s.mlp_load(weights)
    s.set_state(*st)
    del st
    torch.cuda.empty_cache()
    s.step(args.warmup)
    torch.cuda.synchronize()
    barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = s.launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    done, t = s.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    launches = s.launches - l0
    clocks = clk.stop()
    assert done == args.steps
    ms, value = job_rate(ms, n ** 3 * args.steps, world)
    diag = s.diagnostics()
    # the state after warm-up + timed steps: the variants are compared with it
    ref = s.primitives(device=True) if args.variants else None

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.precision == "fp64" else "f32+f64",
           "data": ("synthetic (seeded random-phase turbulence, generated on the GPU)"
                    if args.workload == "turbulence" else "synthetic (analytic Alfven wave)"),
           "config": workload_config(args),
           "gpu_launches": launches, "clocks": clocks,
           "diag": {"t": diag["t"], "divb_max": diag["divb_max"],
                    "newton_it_mean": diag["newton_it_mean"],
                    "c2p_fallbacks": diag["c2p_fallbacks"],
                    "c2p_failures": diag["c2p_failures"]}}
    if train_info:
        out["training"] = train_info
    if args.prof_steps > 0:
        out.update(roofline_and_profile(args, s, n))
    if not args.no_e2e:
        out["e2e"] = end_to_end(args, s, n, world)
    s.close()
    del s
    torch.cuda.empty_cache()
    if ref is not None:
        out["variants"] = variants(args, n, ref, stream, dev)
        del ref
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def roofline_and_profile(args, s, n):
    """Per-kernel device time over a profiled pass (CUDA events recorded by the
    library on its launching stream) and the roofline of the dominant kernel."""
    import json as _json
    s.profile(True)
    s.profile_read(reset=True)
    s.step(args.prof_steps)
    prof = s.profile_read(reset=True)
    s.profile(False)
    tot = sum(v[1] for v in prof.values())
    top = max(prof, key=lambda k: prof[k][1])
    cnt, kms = prof[top]
    per_launch_s = kms / cnt * 1e-3

    # roofline of the dominant kernel
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = _json.load(open(pk))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    fp = "fp64" if args.precision == "fp64" or top in FP64_BOUND else "fp32"
    alu_peak = s.probe_fma_peak(fp)
    r = R64 if args.precision == "fp64" else R32
    units = n ** 3
    flops_tab = load_flops_table().get(args.precision, {})
    fpu = flops_tab.get(top)
    bpu = bytes_per_unit(top, r)
    t_alu = fpu * units / alu_peak if fpu else 0.0
    t_hbm = bpu * units / (hbm_peak * 1e9) if bpu else 0.0
    if fpu and t_alu >= t_hbm:
        achieved = fpu * units / per_launch_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak / 1e12,
                "unit": "TFLOP/s", "frac": achieved / (alu_peak / 1e12),
                "peak_source": "measured FMA-chain probe (%s vector)" %
                               ("FP64" if fp == "fp64" else "FP32")}
    else:
        achieved = bpu * units / per_launch_s / 1e9 if bpu else None
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak if achieved else None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s"}
    roof.update({"kernel": top, "traffic": None, "launch_ms": per_launch_s * 1e3,
                 "share": kms / tot, "hbm_gbs_algorithmic": (bpu * units / per_launch_s / 1e9
                                                             if bpu else None)})
    tr = os.path.join(ROOT, "profiles", "traffic_per_unit.json")
    if os.path.exists(tr):
        tab = _json.load(open(tr))
        tt = tab.get(args.workload, {}).get(args.precision, {}).get(top)
        if tt:
            # measured DRAM bytes per unit (ncu on a smaller grid of the same workload,
            # every array far larger than L2) times the units of one launch
            roof["traffic"] = tt * units
            roof["traffic_source"] = ("ncu dram__bytes_read + dram__bytes_write per unit on "
                                      "the 192^3 grid of the workload, times the launch's units")

    fp64_peak = s.probe_fma_peak("fp64")
    fp32_peak = s.probe_fma_peak("fp32")
    return {"roofline": roof, "kernel_ms_per_step":
            {k: v[1] / args.prof_steps for k, v in sorted(prof.items())},
            "measured_vector_peaks_tflops": {"fp64": fp64_peak / 1e12, "fp32": fp32_peak / 1e12}}


def l1_rel(p, ref):
    """L1 distance per primitive, normalised by the field scale (max |.| of rho, of
    the three velocity components together, of p, of the three field components)."""
    import numpy as np
    out = []
    for grp in ([0], [1, 2, 3], [4], [5, 6, 7]):
        scale = float(np.max(np.abs(ref[grp])))
        for v in grp:
            out.append(float(np.mean(np.abs(p[v] - ref[v]))) / scale)
    return out


def harvest_and_train(n_h, steps, stride, make_state, L, seed, epochs=4, cap=None):
    """Learned guess trained on states the solver produced: harvest (features, W/U)
    from a run of the same workload family, train on the GPU."""
    import torch
    from paper_2401_03008_gb300 import echo
    from paper_2401_03008_gb300 import workloads as wl
    cap = cap or steps * 3 * n_h ** 3 // stride + 1
    h = echo.Solver(n_h, n_h, n_h, L=L)
    h.set_state(*make_state(n_h))
    feats = torch.empty((cap, 5), dtype=torch.float32, device="cuda")
    target = torch.empty(cap, dtype=torch.float32, device="cuda")
    cnt = h.mlp_harvest(steps, stride, feats, target)
    h.close()
    t0 = time.perf_counter()
    w, hist = echo.mlp_train(feats[:cnt].contiguous(), target[:cnt].contiguous(), wl.mlp_init(seed),
                             epochs=epochs, batch=4096, lr=3e-3, lr_decay=0.6)
    torch.cuda.synchronize()
    return w, {"states": int(cnt), "epochs": epochs, "train_s": time.perf_counter() - t0,
               "loss_first": float(hist[0]), "loss_last": float(hist[-1])}


def train_guess(args):
    """The network of the learned guess for the selected workload: about 1e7 states
    harvested (every 8th cell after every inversion of --train-steps steps) from a
    --train-n^3 run of another seed of the same workload, trained on the GPU."""
    if args.workload == "turbulence":
        mk = lambda m: turbulence_state(m, args.lorentz_max, seed=SEED + 1)
        return harvest_and_train(args.train_n, args.train_steps, 8, mk, TURB_L, SEED + 2,
                                 cap=10_000_000)
    mk = lambda m: workload_state(m, args.wave)[1]
    return harvest_and_train(64, 8, 4, mk, (1.0, 1.0, 1.0), SEED + 2)


def l1_rel_device(sol, ref):
    """L1 distance per primitive between a solver's state and a reference [8][...]
    (device tensor) by echo_l1_error, normalised by the field scale as l1_rel does."""
    import torch
    l1 = sol.l1_error(ref)
    out = []
    for grp in ([0], [1, 2, 3], [4], [5, 6, 7]):
        scale = float(torch.max(torch.abs(ref[grp])))
        out += [float(l1[v]) / scale for v in grp]
    return out


def run_variant(args, n, precision, guess, stream, dev, ref=None, weights=None):
    """One precision/guess variant of the headline run: same workload, warm-up and
    timed steps; rate, Newton statistics and (with ref) the L1 distance to it."""
    import torch
    from paper_2401_03008_gb300 import echo
    L, st = state_for(args, n, device=dev)
    v = echo.Solver(n, n, n, L=L, precision=precision, guess=guess, stream=stream.cuda_stream,
                    uct=args.uct, ho=args.ho, rec=args.rec, rk_order=args.rk, sweeps=args.sweeps)
    if weights is not None:
        v.mlp_load(weights)
    v.set_state(*st)
    del st
    torch.cuda.empty_cache()
    v.step(args.warmup)
    v.diagnostics(reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    v.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    d = v.diagnostics()
    r = {"value": n ** 3 * args.steps / (ms * 1e-3), "ms_per_step": ms / args.steps,
         "newton_it_fp64": d["newton_it_mean"], "newton_it_fp32": d["newton_it32_mean"],
         "c2p_fallback_rate": d["c2p_fallbacks"] / max(d["c2p_calls"], 1),
         "c2p_failures": d["c2p_failures"]}
    if ref is not None:
        r["l1_vs_fp64"] = l1_rel_device(v, ref)
    v.close()
    del v
    torch.cuda.empty_cache()
    return r


def variants(args, n, ref, stream, dev):
    """The mixed path, and the mixed path with the learned guess, on the same workload
    and step count as the headline, with their L1 distance (per primitive, over the
    field scale) to the FP64 state."""
    out = {"mixed": run_variant(args, n, "mixed", "prev", stream, dev, ref)}
    w, info = train_guess(args)
    r = run_variant(args, n, "mixed", "mlp", stream, dev, ref, w)
    r["training"] = info
    out["mixed_mlp"] = r
    out["l1_tolerance"] = ("L1(mixed - FP64) <= 1e-6 of each field's scale (the mixed path's "
                           "stated bound)")
    return out


def run_config_variant(args, n, precision, guess, steps, stream, dev, ref=None, weights=None,
                       keep=False):
    """A turbulence run of the benchmark plan: one warm-up step, then `steps` timed
    steps; rate, Newton statistics, L1 distance to ref (when given); the primitives
    on the device when keep."""
    import torch
    from paper_2401_03008_gb300 import echo
    L, st = state_for(args, n, device=dev)
    v = echo.Solver(n, n, n, L=L, precision=precision, guess=guess, stream=stream.cuda_stream)
    if weights is not None:
        v.mlp_load(weights)
    v.set_state(*st)
    del st
    torch.cuda.empty_cache()
    v.step(1)
    v.diagnostics(reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    try:
        done, t = v.step(steps)
        failed = None
    except echo.EchoError as e:
        done, t, failed = None, None, str(e)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    d = v.diagnostics()
    r = {"ms_per_step": ms / steps, "cell_updates_per_s": n ** 3 * steps / (ms * 1e-3),
         "t": d["t"], "newton_it_fp64": d["newton_it_mean"],
         "newton_it_fp32": d["newton_it32_mean"],
         "c2p_fallback_rate": d["c2p_fallbacks"] / max(d["c2p_calls"], 1),
         "c2p_failures": d["c2p_failures"], "divb_max": d["divb_max"]}
    if failed:
        r["failed"] = failed
    if ref is not None:
        r["l1_vs_fp64"] = l1_rel_device(v, ref)
    p = v.primitives(device=True) if keep else None
    v.close()
    del v
    torch.cuda.empty_cache()
    return r, p


def run_config(args):
    """The five configurations of the benchmark plan, one JSON line each (for the
    design notes; the default run is the headline line)."""
    import numpy as np
    import torch
    from paper_2401_03008_gb300 import echo
    from paper_2401_03008_gb300 import workloads as wl
    stream = torch.cuda.Stream()  # the library launches on it; the events are recorded on it
    sp = stream.cuda_stream

    def timed(sol, steps, t_end=math.inf):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        done, t = sol.step(steps, t_end)
        e1.record(stream)
        torch.cuda.synchronize()
        return done, t, e0.elapsed_time(e1)

    out = {"config": args.config}
    if args.config == 6:
        out.update(run_turbulence_2d(args, timed, sp))
    elif args.config == 7:
        out.update(run_blocks(args, timed, sp))
    elif args.config == 1:
        from oracle import oracle as orc
        n = 32
        c = wl.CPA(n, n, n, m=(1, 0, 0))
        st = (c.prim5(), c.bface_background(), c.apot())
        s = echo.Solver(n, n, n, stream=sp)
        s.set_state(*st)
        done, t, ms = timed(s, 20)
        g = orc.Grid(n, n, n, nthreads=os.cpu_count())
        g.set_state(*st)
        t0 = time.perf_counter()
        g.step(20)
        el = time.perf_counter() - t0
        # the oracle on one core as well (the same 20 steps)
        g1 = orc.Grid(n, n, n, nthreads=1)
        g1.set_state(*st)
        t0 = time.perf_counter()
        g1.step(20)
        el1 = time.perf_counter() - t0
        p, ref = s.primitives(), g.primitives()
        rel = []
        for grp in ([0], [1, 2, 3], [4], [5, 6, 7]):
            sc = np.max(np.abs(ref[grp]))
            rel += [float(np.max(np.abs(p[v] - ref[v])) / sc) for v in grp]
        out.update({"workload": "Alfven wave along x, 32^3, FP64, 20 steps", "steps": done,
                    "t": t, "gpu_cell_updates_per_s": n ** 3 * 20 / (ms * 1e-3),
                    "oracle_cell_updates_per_s": n ** 3 * 20 / el, "oracle_threads": os.cpu_count(),
                    "oracle_one_core_cell_updates_per_s": n ** 3 * 20 / el1,
                    "host_cpu": _cpu_model(),
                    "max_rel_diff_vs_oracle": rel,
                    "l1_vs_exact": list(map(float, s.l1_error(c.exact_prim8(t))))})
    elif args.config in (2, 3):
        n = 256 if args.config == 2 else 512
        c = wl.CPA(n, n, n, m=(1, 1, 1))
        st = (c.prim5(), c.bface_background(), c.apot())
        res = {}
        precs = ["fp64"] if args.config == 2 else ["fp64", "mixed"]
        prims = {}
        for prec in precs:
            s = echo.Solver(n, n, n, precision=prec, stream=sp)
            s.set_state(*st)
            if args.config == 2:
                done, t, ms = timed(s, 100000, c.period)
            else:
                done, t, ms = timed(s, args.config_steps)
            d = s.diagnostics()
            ex = c.exact_prim8(t)
            res[prec] = {"steps": done, "t": t, "cell_updates_per_s": n ** 3 * done / (ms * 1e-3),
                         "ms_per_step": ms / done, "l1_vs_exact": list(map(float, s.l1_error(ex))),
                         "divb_max": d["divb_max"], "newton_it_fp64": d["newton_it_mean"],
                         "newton_it_fp32": d["newton_it32_mean"], "c2p_failures": d["c2p_failures"]}
            prims[prec] = s.primitives()
            s.close()
        if args.config == 3:
            res["mixed"]["l1_vs_fp64"] = l1_rel(prims["mixed"], prims["fp64"])
        out.update({"workload": "Alfven wave along (1,1,1), %d^3" % n
                    + (", one period" if args.config == 2 else ", %d steps" % args.config_steps),
                    "period": c.period, "results": res})
    elif args.config == 8:
        out.update(run_time_to_accuracy(args, timed, sp))
    else:
        n = 512 if args.config == 4 else args.config5_n
        dev = "cuda:%d" % torch.cuda.current_device()
        args.workload = "turbulence"
        if args.config == 5:
            args.lorentz_max = args.config5_lorentz_max
        w, info = train_guess(args)
        res = {"training": info}
        runs = ([("fp64", "prev"), ("fp64", "cold"), ("fp64", "mlp"), ("mixed", "prev"),
                 ("mixed", "cold"), ("mixed", "mlp")] if args.config == 4 else
                [("fp64", "prev"), ("mixed", "prev"), ("mixed", "mlp")])
        if args.config_runs:
            keep_runs = set(args.config_runs.split(","))
            runs = [r for r in runs if "%s_%s" % r in keep_runs]
        ref, ref_steps = None, None
        for prec, guess in runs:
            steps = args.config_steps if args.config == 4 else args.config5_steps
            keep = prec == "fp64" and guess == "prev"
            r, p = run_config_variant(args, n, prec, guess, steps, stream, dev,
                                      ref if steps == ref_steps else None,
                                      w if guess == "mlp" else None, keep)
            if keep:
                ref, ref_steps = p, steps
            r["steps"] = steps
            res["%s_%s" % (prec, guess)] = r
        out.update({"workload": workload_name(args, n), "results": res})
    print(json.dumps(out))


def run_time_to_accuracy(args, timed, sp):
    """The Alfven wave along (1,1,1) (Sec. 4) for one full period on several grids in
    both paths: steps, GPU seconds, rate and the L1 error of every primitive against
    the exact solution (each over its field scale), so that each path's cost can be
    read off at equal accuracy.  FP64 on 64^3..256^3, mixed on 128^3..512^3."""
    from paper_2401_03008_gb300 import echo
    from paper_2401_03008_gb300 import workloads as wl
    import numpy as np
    runs = [("fp64", 64), ("fp64", 128), ("fp64", 256), ("mixed", 128), ("mixed", 256),
            ("mixed", 512)]
    res = []
    for prec, n in runs:
        c = wl.CPA(n, n, n, m=(1, 1, 1))
        s = echo.Solver(n, n, n, precision=prec, stream=sp)
        s.set_state(c.prim5(), c.bface_background(), c.apot())
        done, t, ms = timed(s, 1 << 30, c.period)
        ex = c.exact_prim8(t)
        l1 = s.l1_error(ex)
        scale = [1.0, c.vA * c.eta, 1.0, math.sqrt(1 + c.eta ** 2) * c.B0]
        grp = [0, 1, 1, 1, 2, 3, 3, 3]
        rel = [float(l1[v]) / scale[grp[v]] for v in range(8)]
        d = s.diagnostics()
        res.append({"path": prec, "n": n, "steps": done, "t": t, "gpu_s": ms * 1e-3,
                    "cell_updates_per_s": n ** 3 * done / (ms * 1e-3),
                    "l1_vs_exact_rel": rel, "l1_max_rel": max(rel), "divb_max": d["divb_max"]})
        s.close()
    return {"workload": "Alfven wave along (1,1,1), one period (T = %.7f), CFL 0.4" % c.period,
            "results": res}


def run_turbulence_2d(args, timed, sp):
    """Decaying 2.5-D Alfvenic turbulence (Sec. 5): n^2 x 1 cells of a (2 pi)^2 box,
    sigma0 = 100, beta0 = 1, eta_rms = 0.25, modes |k| <= 4, UCT = HO = on, run to
    t_end.  Every time unit: mean |dv_perp|/v_A, mean |dB_perp|/B0 and the rms of the
    current J_z; at t = 0 and t_end the isotropised spectra of the perpendicular and
    parallel components of v and B, with power-law slopes over ranges of k_perp."""
    import numpy as np
    import torch
    from paper_2401_03008_gb300 import echo
    from paper_2401_03008_gb300 import spectra
    from paper_2401_03008_gb300 import workloads as wl
    n, seed = args.config6_n, 2401_03008
    tb = wl.Turbulence2D(n, seed=seed)
    s = echo.Solver(n, n, 1, L=tb.L, precision=args.precision, guess=args.guess, ho=args.ho,
                    uct=args.uct, rec=args.rec, rk_order=args.rk, stream=sp)
    if args.uct:
        s.set_state(tb.prim5(), tb.bface_background(), tb.apot())
    else:
        s.set_state(tb.prim5(), tb.bcell())
    h = 2 * np.pi / n
    prim = torch.empty((8, 1, n, n), dtype=torch.float64, device="cuda")

    def sample(t):
        s.primitives(prim)
        v, B = prim[1:3, 0], prim[5:7, 0]
        J = ((torch.roll(B[1], -1, 1) - torch.roll(B[1], 1, 1))
             - (torch.roll(B[0], -1, 0) - torch.roll(B[0], 1, 0))) / (2 * h)
        return {"t": t, "dv_over_vA": float(torch.sqrt((v * v).sum(0)).mean()) / tb.vA,
                "dB_over_B0": float(torch.sqrt((B * B).sum(0)).mean()) / tb.B0,
                "J_rms": float(torch.sqrt((J * J).mean()))}

    def spec():
        p = prim.cpu().numpy()[:, 0]
        k, ev = spectra.shell_spectrum([p[1], p[2]])
        _, eb = spectra.shell_spectrum([p[5], p[6]])
        _, evz = spectra.shell_spectrum([p[3]])
        _, ebz = spectra.shell_spectrum([p[7]])
        return k, {"v_perp": ev, "B_perp": eb, "v_par": evz, "B_par": ebz}

    series = [sample(0.0)]
    k, spec0 = spec()
    total_ms, steps, t, tk = 0.0, 0, 0.0, 0
    while t < args.config6_t:
        tk = min(tk + 1.0, args.config6_t)
        done, t, ms = timed(s, 1 << 30, tk)
        total_ms += ms
        steps += done
        series.append(sample(t))
    k, spec1 = spec()
    d = s.diagnostics()
    ranges = [(8, 64), (16, 128), (32, 256), (64, 512)]
    slopes = {name: {"%d-%d" % r: spectra.slope(k, e, *r) for r in ranges if r[1] <= n // 4}
              for name, e in spec1.items()}
    edges = np.unique(np.round(np.geomspace(1, n // 2, 40)).astype(int))
    binned = {name: [float(e[lo:hi].mean()) for lo, hi in zip(edges[:-1], edges[1:])]
              for name, e in spec1.items()}
    if args.config6_out:
        np.savez(args.config6_out, k=k, **{"t0_" + a: b for a, b in spec0.items()},
                 **{"t1_" + a: b for a, b in spec1.items()})
    return {"workload": "2.5-D decaying Alfvenic turbulence, %d^2 x 1, sigma0 = 100, beta0 = 1, "
                        "eta_rms = 0.25, |k| <= 4, seed %d" % (n, seed),
            "precision": args.precision, "uct": args.uct, "ho": args.ho, "rec": args.rec,
            "rk_order": args.rk, "t_end": t, "steps": steps, "gpu_seconds": total_ms * 1e-3,
            "gpu_seconds_per_time_unit": total_ms * 1e-3 / t,
            "cell_updates_per_s": n * n * steps / (total_ms * 1e-3),
            "divb_max": d["divb_max"], "newton_it_fp64": d["newton_it_mean"],
            "c2p_fallbacks": d["c2p_fallbacks"], "c2p_failures": d["c2p_failures"],
            "series": series, "slopes_t_end": slopes,
            "spectra_t_end_binned": {"k_edges": edges.tolist(), **binned}}


def run_blocks(args, timed, sp):
    """The grid split into 2 x 2 x 2 blocks with the wide halo (one exchange per
    substep), all on this GPU, against the undecomposed grid: rate and identity of
    the state after the same steps."""
    import numpy as np
    from paper_2401_03008_gb300 import echo
    n = args.n
    _, st = workload_state(n, args.wave)
    res = {}
    for prec in ("fp64", "mixed"):
        kw = dict(precision=prec, stream=sp)
        s = echo.Solver(n, n, n, **kw)
        s.set_state(*st)
        s.step(1)
        _, _, ms_s = timed(s, args.config_steps)
        d = echo.Decomp(n, n, n, (2, 2, 2), **kw)
        d.set_state(*st)
        d.step(1)
        _, _, ms_d = timed(d, args.config_steps)
        a, b = s.get_state(), d.get_state()
        same = all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3])) and a[3:] == b[3:]
        npad = (n // 2 + 2 * d.halo)
        res[prec] = {"halo": d.halo, "padded_block": npad,
                     "padded_volume_ratio": 8 * npad ** 3 / n ** 3,
                     "single_grid_cell_updates_per_s": n ** 3 * args.config_steps / (ms_s * 1e-3),
                     "blocks_cell_updates_per_s": n ** 3 * args.config_steps / (ms_d * 1e-3),
                     "state_bit_identical": bool(same)}
        s.close()
        d.close()
    return {"workload": "Alfven wave along (1,1,1), %d^3, 2 x 2 x 2 blocks with the minimum "
                        "wide halo, %d steps" % (n, args.config_steps), "results": res}


def end_to_end(args, s, n, world):
    """The same metric through the C ABI with host buffers: every step uploads the
    state from pinned host memory (echo_set_conserved), advances one step and reads
    the state back (echo_get_state)."""
    import torch
    pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    cons, bf, w = pin((5, n, n, n)), pin((3, n, n, n)), pin((n, n, n))
    _, _, _, t0s, st0 = s.get_state(cons, bf, w)
    ke = 2
    torch.cuda.synchronize()
    q0 = time.perf_counter()
    for _ in range(ke):
        s.set_conserved(cons, bf, w, t0s, st0)
        s.step(1)
        _, _, _, t0s, st0 = s.get_state(cons, bf, w)
    el = time.perf_counter() - q0
    _, value = job_rate(el * 1e3, n ** 3 * ke, world)  # the slowest rank's time
    by = cons.nbytes + bf.nbytes + w.nbytes
    del cons, bf, w
    return {"value": value, "unit": UNIT, "h2d_bytes_per_step": by,
            "d2h_bytes_per_step": by, "steps": ke}


if __name__ == "__main__":
    main()
