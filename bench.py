"""Benchmark: DOF-updates/s per RK stage of the DG operator on the P4 512x512
planet-disc workload (locally isothermal Keplerian disc, q = 3e-5, damping
zones r < 0.4 and r > 2.1, SSP(3,3), torque on the planet every step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One timed step = one full RK step of the hot path (3 fused stage kernels, the
last with damping and CFL, then the torque pass and the finish kernel) on
device-resident inputs.  The state
buffers (157 MB each, 3 of them) are larger than the 129 MB L2, so no flush is
needed between steps.  DOF = nx * ny * (p+1)^2 per stage (Sec. 3.1).
For N > 1 (torchrun) every rank advances an independent replica (no data-path
collective); value = DOF-updates of all ranks / max-over-ranks time.
`--impl reference` times the FP64 CPU oracle (the reference arm of this
project) on this host's cores: K steps of the full mesh, or of the same disc on
a coarser mesh where K full steps would take more than two minutes.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s per RK stage, P4 512² disc: FP32-TC vs FP64 at stated error"
UNIT = "DOF/s"
WORKLOAD = "planet-disc P4 512x512 (q=3e-5, damping 0.4/2.1, SSP(3,3), torque every step)"
# algorithmic work per element per RK stage, P4, 3 variables, FP64 (sum-factorised
# contractions + pointwise flux, gravity and Riemann terms; u^n and u^(s) read,
# u^(s+1) written on average over the 3 SSP(3,3) stages)
FLOP_PER_ELEM_STAGE = 10.0e3
BYTES_PER_ELEM_STAGE_FP64 = 1600.0
# precision form, algorithmic bytes: the FP32 state of 75 floats = 300 B per
# element, read u^(s) (and u^n in stages 2 and 3) and written u^(s+1):
# (2 + 3 + 3) / 3 x 300 = 800 B per element and stage launch, half the FP64
# figure.  The background residual R_b, the background averages and the
# damping offsets are static data of this design, not algorithmic bytes:
# a stage also reads R_b (300 B per element) in the tiles that keep it, the
# last stage the background averages (12 B) and, in the tiles that touch a
# damping zone, the damping offsets (300 B); design_bytes() counts them from
# the handle's own tile counts.
BYTES_PER_ELEM_STAGE_PREC = 800.0


def design_bytes(ntiles, rb_tiles, zone_tiles):
    """Bytes per element and stage launch of the precision-form stage kernel
    with its static data (see above), averaged over the three stages."""
    return (BYTES_PER_ELEM_STAGE_PREC + 300.0 * rb_tiles / ntiles
            + (12.0 + 300.0 * zone_tiles / ntiles) / 3.0)


BYTES_PER_ELEM_TORQUE_PREC = 300.0
# DRAM bytes (read + write) per stage launch of k_stage32<4> at 512^2, the mean
# over the three stages of one step from one ncu capture of the current kernel
# (135.5, 227.3 and 294.7 MB)
TRAFFIC_PER_STAGE_PREC = 219.2e6
# FP64 peak of GB300 derived from unit counts and clock: 2 FP64 FMA / clk / SM
# x 152 SMs x 2 flop x 2.07 GHz = 1.26 TFLOP/s
FP64_PEAK_TFLOPS = 2 * 152 * 2 * 2.07e9 / 1e12


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x, pg, device="cuda"):
    """The largest of the ranks' values of x (x itself with one rank): the
    whole job's time is the slowest rank's."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds):
    """Whole-job throughput of `world` replicas that each process
    `units_per_rank` in `seconds` (the slowest rank's time)."""
    return world * units_per_rank / seconds


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline_sample(cfg, seconds=15.0):
    """FP64 oracle on this host's cores over a bounded sample of the same
    workload: whole steps of the full mesh until ~`seconds` of CPU work."""
    import oracle

    o = oracle.Oracle(cfg)
    n_el = cfg["mesh"]["nx"] * cfg["mesh"]["ny"]
    dof = n_el * (cfg["order"] + 1) ** 2
    t0 = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t0
    nsteps = max(1, min(50, int(seconds / max(one, 1e-3))))
    t0 = time.perf_counter()
    o.step(nsteps)
    el = time.perf_counter() - t0
    cores = oracle.nthreads()
    # the same oracle on one core: one step of the full mesh
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        o.step(1)
        el1 = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    return {"value": dof * 3 * nsteps / el, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": "%d SSP(3,3) steps (%d stages) of the full %dx%d P%d workload, FP64, "
                      "OpenMP over elements" % (nsteps, 3 * nsteps, cfg["mesh"]["nx"],
                                                cfg["mesh"]["ny"], cfg["order"]),
            "one_core": {"value": dof * 3 / el1, "unit": UNIT, "cores": 1,
                         "sample": "1 SSP(3,3) step (3 stages) of the same workload"}}


def reference_sample(cfg, steps, t_step, budget_s=120.0):
    """The workload the reference arm times: the full mesh while `steps` steps
    of it fit in `budget_s` (one step took `t_step` s), otherwise the same disc
    on a coarser mesh, the element count scaled to fit (even sides, at least
    64 unless the mesh is smaller), so that the run stays within a few
    minutes; returns (cfg, note)."""
    import copy

    n = cfg["mesh"]["nx"]
    if steps * t_step <= budget_s:
        return cfg, "the full %dx%d mesh" % (n, cfg["mesh"]["ny"])
    frac = budget_s / (steps * t_step)
    ns = max(int(n * frac ** 0.5) // 2 * 2, min(n, 64))
    if ns >= n:
        return cfg, "the full %dx%d mesh" % (n, cfg["mesh"]["ny"])
    small = copy.deepcopy(cfg)
    small["mesh"]["nx"] = small["mesh"]["ny"] = ns
    return small, "the same disc on a %dx%d mesh (the full %dx%d mesh would take %.0f s)" % (
        ns, ns, n, cfg["mesh"]["ny"], steps * t_step)


def run_reference(args, cfg, budget_s=120.0):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    o = oracle.Oracle(cfg)
    t0 = time.perf_counter()
    o.step(1)
    t_step = time.perf_counter() - t0
    cfg_s, note = reference_sample(cfg, args.steps, t_step, budget_s)
    if cfg_s is not cfg:
        o = oracle.Oracle(cfg_s)
    n_el = cfg_s["mesh"]["nx"] * cfg_s["mesh"]["ny"]
    dof = n_el * (cfg_s["order"] + 1) ** 2
    o.step(max(args.warmup, 0))
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    value = dof * 3 * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "impl": "FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.nthreads(), "kind": "oracle",
                         "sample": "%d SSP(3,3) steps per timed run, each over %s" % (args.steps, note)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def timed_run(dg, torch, cfg, steps, warmup, local, pg):
    """Advance one handle `warmup` untimed steps, then time `steps` steps with CUDA
    events on its stream (barrier + synchronize on both sides) and the stage
    kernels with dg_set_timing; returns (handle, ms, mean stage seconds, clocks)."""
    disc = dg.Disc(cfg)
    stream = torch.cuda.current_stream()
    disc.step(warmup)
    disc.sync()
    disc.set_timing(True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        ev0.record(stream)
        disc.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms = ev0.elapsed_time(ev1)
    stage_ms, nstage = disc.timing()
    disc.set_timing(False)
    disc.sync()
    ms = max_over_ranks(ms, pg)
    return disc, ms, stage_ms / max(nstage, 1) / 1e3, clk.summary()


def error_vs_fp64(dg, cfg, cfg32, nsteps):
    """Precision form against the FP64 operator from the same initial state:
    relative L2 of Sigma, of Sigma - Sigma_bg and of the torque series."""
    bg = dict(cfg, disc=dict(cfg["disc"], noise_amp=0.0))
    with dg.Disc(bg) as b:
        sig_bg = b.fetch()[0]
    with dg.Disc(cfg) as a, dg.Disc(cfg32) as p:
        a.step(nsteps)
        p.step(nsteps)
        ua, up = a.fetch(), p.fetch()
        ta, tp = a.torque_series(), p.torque_series()
    rel = lambda x, y: float(np.linalg.norm(x - y) / np.linalg.norm(y))
    return {"steps": nsteps, "rel_l2_sigma": rel(up[0], ua[0]),
            "rel_l2_sigma_minus_bg": rel(up[0] - sig_bg, ua[0] - sig_bg),
            "rel_l2_momentum": max(rel(up[1], ua[1]), rel(up[2], ua[2])),
            "rel_l2_torque_series": rel(tp, ta),
            "bounds": {"sigma": 1e-5, "torque": 1e-6},
            "torque_form": "node terms and their per-element sums in float-float (~2^-44 relative), the "
                           "reduction over elements and tiles in FP64: the one part of the torque not in "
                           "FP64; an all-FP64 pass is estimated at ~0.16 ms per step against the "
                           "float-float pass's ~0.04 ms"}


def batched_run(dg, torch, steps=10, tune_steps=3):
    """The batched workload: 48 independent discs (sizes 128-512^2, degrees
    2-4, seeded planet masses) advanced by per-instance launches in turn and by
    the batched form (tuned schedule); aggregate DOF-updates/s per stage."""
    from paper_1805_01443_gb300 import inputs
    cfgs = inputs.batch_discs()
    discs = [dg.Disc(c) for c in cfgs]
    dof = sum(c["mesh"]["nx"] * c["mesh"]["ny"] * (c["order"] + 1) ** 2 for c in cfgs)
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn(1)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn(steps)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / steps

    seq_ms = timed(lambda k: [d.step(k) for d in discs])
    with dg.Batch(discs) as bt:
        tuned = bt.tune(steps=tune_steps)
        bat_ms = timed(bt.step)
        bt.sync()
    for d in discs:
        d.sync()
        d.close()
    return {"value": dof * 3 / (bat_ms / 1e3), "unit": UNIT, "ms_per_step": bat_ms,
            "sequential": {"value": dof * 3 / (seq_ms / 1e3), "ms_per_step": seq_ms,
                           "how": "per-instance dg_step launches in turn on one stream"},
            "speedup_vs_sequential": seq_ms / bat_ms, "steps": steps,
            "schedule": {"policy": dg.Batch.POLICIES[tuned["policy"]],
                         "launches": ["one CTA per tile per stage", "persistent CTAs per stage",
                                      "one persistent launch per step",
                                      "one persistent launch per step, round-robin items"][tuned["dynamic"]],
                         "ctas_per_sm": tuned["ctas_per_sm"], "tiles_per_item": tuned["tiles_per_item"]},
            "gpu_launches_per_step": 1 if tuned["dynamic"] >= 2 else 5,
            "config": {"workload": "48 planet discs, sizes 128/256/384/512^2 and degrees 2/3/4 "
                                   "cycling, q = 10^U(-6,-4), seeds 100-147, precision form",
                       "instances": len(cfgs), "dof_per_stage": dof}}


def indicator_run():
    """The learned troubled-cell indicator on the shock-ring disc (adiabatic,
    pressure ring x10 at r = 1.5, q = 1e-3, P3 1024^2): labels from the TVB
    test on the method's own run (seed 5), training with libdg's kernels,
    miss / false-flag rates on a held-out run (seed 6) and the induced density
    error of a network-limited run against the TVB-limited one, next to the
    run without troubled-cell limiting (seed 7)."""
    from paper_1805_01443_gb300 import indicator, inputs
    rec = indicator.evaluate(inputs.shock_ring(1024, 3, seed=5), inputs.shock_ring(1024, 3, seed=6),
                             inputs.shock_ring(1024, 3, seed=7))
    rec["config"] = {"workload": "shock-ring disc P3 1024x1024, gamma 1.4, q 1e-3, TVB M = 50, "
                                 "positivity limiter; MLP 320-64-64-1 GELU, BF16 weights, FP32 accumulate"}
    return rec


def indicator_pass(n, reps, warmup):
    """The learned indicator's limit pass alone (the profiling case of its
    inference kernel): mean ms per pass on the n^2 P3 shock-ring disc."""
    import torch  # noqa: F401
    from paper_1805_01443_gb300 import indicator
    ms = indicator.limit_pass_ms(n=n, order=3, reps=reps, warmup=warmup)
    print(json.dumps({"workload": "limit pass, learned indicator, P3 %d^2 shock ring" % n,
                      "elements": n * n, "ms_per_pass": ms}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--form", default="prec", choices=["prec", "fp64"],
                    help="prec: the precision form is the headline, FP64 alongside")
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--err-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--n", type=int, default=512, help="mesh size (profiling cases only)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 48-disc batched workload")
    ap.add_argument("--no-indicator", action="store_true", help="skip the learned-indicator workload")
    ap.add_argument("--indicator-pass", type=int, default=0, metavar="N",
                    help="profiling case: time `--steps` limit passes of the learned indicator on the "
                         "N^2 P3 shock-ring disc, print one JSON line and exit")
    args = ap.parse_args()
    if args.indicator_pass > 0:
        return indicator_pass(args.indicator_pass, args.steps, args.warmup)

    import copy

    from paper_1805_01443_gb300 import inputs

    world, rank, local = dist_env()
    cfg = inputs.disc_planet_512(n=args.n, seed=3 + rank)
    if args.impl == "reference":
        return run_reference(args, cfg)

    import torch

    from paper_1805_01443_gb300 import dg

    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        pg = tdist
    dg.lib()
    n_el = cfg["mesh"]["nx"] * cfg["mesh"]["ny"]
    dof = n_el * (cfg["order"] + 1) ** 2
    stages_per_step = 3
    peaks = load_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    cfg32 = copy.deepcopy(cfg)
    cfg32["disc"]["prec"] = 1
    head_cfg = cfg32 if args.form == "prec" else cfg

    # headline form
    disc, ms, stage_s, clocks = timed_run(dg, torch, head_cfg, args.steps, args.warmup, local, pg)
    tiles = disc.prec_tiles() if args.form == "prec" else None
    dbytes = design_bytes(*tiles) if tiles else None
    value = job_rate(world, dof * stages_per_step * args.steps, ms / 1e3)

    # end to end through the C ABI with host buffers: every step uploads the
    # state from pinned host memory, advances one step and reads the torque
    # back; the upload of step k+1 runs on the handle's copy stream while
    # step k computes, the torque read is queued behind the step
    # (dg_torque_async), and the timed region ends after the last read has
    # landed.  The precision form's state is its FP32 perturbation, uploaded
    # with dg_set_delta_async; the FP64 state upload (dg_set_state_async) is
    # reported beside it.
    t_now, _, st = disc.get_time()
    n_e2e = max(args.e2e_steps, 1)

    def e2e_run(host, upload):
        tq = torch.empty(n_e2e, dtype=torch.float64, pin_memory=True).numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        upload(host, t_now, st)
        for k in range(n_e2e):
            disc.step(1)
            disc.torque_async(tq, k)
            if k + 1 < n_e2e:
                upload(host, t_now, st)
        disc.sync()
        secs = (time.perf_counter() - t0) / n_e2e
        if not (np.all(np.isfinite(tq)) and np.all(tq == tq[0])):
            raise RuntimeError("end-to-end steps from the same uploaded state disagree")
        secs = max_over_ranks(secs, pg)
        return {"value": job_rate(world, dof * stages_per_step, secs), "unit": UNIT,
                "h2d_bytes_per_step": int(host.nbytes), "d2h_bytes_per_step": 8}

    host = torch.empty(disc.shape, dtype=torch.float64, pin_memory=True).numpy()
    disc.fetch(host)
    e2e_state = e2e_run(host, disc.set_state_async)
    if args.form == "prec":
        hd = torch.empty(disc.shape, dtype=torch.float32, pin_memory=True).numpy()
        disc.fetch_delta(hd)
        e2e = e2e_run(hd, disc.set_delta_async)
        e2e["upload"] = "FP32 perturbation delta = u - u_b (dg_set_delta_async)"
        e2e["fp64_state_upload"] = e2e_state
    else:
        e2e = e2e_state
    disc.close()

    def fp64_roofline(stage64):
        tf = FLOP_PER_ELEM_STAGE * n_el / stage64 / 1e12
        gbs = BYTES_PER_ELEM_STAGE_FP64 * n_el / stage64 / 1e9
        return {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tf / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": "k_stage<4,0> (FP64 fused RK stage)",
                "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2.07 GHz",
                "hbm_achieved_gbs": gbs, "hbm_frac": gbs / hbm_peak,
                "hbm_peak_source": hbm_src, "stage_us": stage64 * 1e6}

    if args.form == "prec":
        gbs = BYTES_PER_ELEM_STAGE_PREC * n_el / stage_s / 1e9
        roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": gbs / hbm_peak,
                    "traffic": TRAFFIC_PER_STAGE_PREC if (n_el == 512 * 512 and cfg["order"] == 4) else None,
                    "kernel": "k_stage32<4> (precision-form fused RK stage)",
                    "peak_source": hbm_src, "stage_us": stage_s * 1e6,
                    "algorithmic_bytes_per_element": BYTES_PER_ELEM_STAGE_PREC,
                    "design_bytes_per_element": dbytes,
                    "design_achieved": dbytes * n_el / stage_s / 1e9,
                    "tiles": {"all": tiles[0], "keeping_R_b": tiles[1], "damping": tiles[2]}}
        d64, ms64, stage64, clocks64 = timed_run(dg, torch, cfg, args.fp64_steps, 2, local, pg)
        d64.close()
        fp64 = {"value": world * dof * stages_per_step * args.fp64_steps / (ms64 / 1e3),
                "unit": UNIT, "steps": args.fp64_steps, "ms_per_step": ms64 / args.fp64_steps,
                "dtype": "f64", "roofline": fp64_roofline(stage64), "clocks": clocks64}
        err = error_vs_fp64(dg, cfg, cfg32, args.err_steps) if args.err_steps > 0 else None
        dtype = "f32"
        form = ("precision form: FP32 operator on the perturbation about the projected "
                "equilibrium; FP64 background residual, torque reduction and sums")
    else:
        roofline = fp64_roofline(stage_s)
        fp64, err, dtype, form = None, None, "f64", "FP64 operator"

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": form, "elements": n_el,
                   "dof_per_stage": dof, "stages_per_step": stages_per_step,
                   "l2": "inputs larger than L2 (state buffers of %.0f MB FP64 / %.0f MB FP32)"
                         % (host.nbytes / 1e6, host.nbytes / 2e6),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline,
        "e2e": e2e,
        # per step: 3 stage kernels, the torque pass and the finish; one
        # planet-position launch per call
        "gpu_launches": 5 * args.steps + 1,
        "clocks": clocks,
    }
    if fp64 is not None:
        line["fp64"] = fp64
    if err is not None:
        line["error_vs_fp64"] = err
    if args.form == "prec" and world == 1 and not args.no_batched:
        line["batched"] = batched_run(dg, torch)
    if args.form == "prec" and world == 1 and not args.no_indicator:
        line["indicator"] = indicator_run()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(cfg)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
