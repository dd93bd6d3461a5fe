"""Benchmark of the GB300 messenger-field mapmaker.

One step = one cooled messenger iteration (Sec. 2.1) over the whole workload: pointing
gather + column FFTs, row FFTs with the Fourier-diagonal filter and chi^2, inverse FFTs +
FP64 binning, and the per-pixel 3x3 map solve.  Workload: 512x512 IQU map, 8 detectors x
2^22 samples at 200 Hz (33.5 M samples), FP32 cos/sin weights, per-detector 1/f noise,
lambda cycling through a 10 x 10 cooling schedule.  Inputs per step (pointing 403 MB,
data spectrum 134 MB, noise table 67 MB) exceed the 129 MB L2, so no flush is needed.

``--impl reference`` times the FP64 CPU oracle on the same workload instead (a bounded
sample: one of the eight detector chunks per step, scaled by eight).

With ``--gpus N`` under torchrun each rank runs an independent replica on its own GPU
(the solver is single-GPU); value = total iterations of all ranks / max rank time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "messenger iters/s"
UNIT = "iter/s"
WORKLOAD = "iqu512_8det_2^22"


def workload_config(s):
    n = int(s["offsets"][-1])
    return {"workload": WORKLOAD, "map": "512x512 IQU", "detectors": len(s["offsets"]) - 1,
            "samples_per_detector": int(s["offsets"][1] - s["offsets"][0]), "n_samples": n,
            "weights": "fp32 cos2psi/sin2psi", "schedule": "10 levels x 10 iterations, cycled",
            "l2": "inputs larger than L2 (>600 MB read per step), no flush",
            "parallelism": "replicas"}


def bytes_per_stage(n, npix, ncomp, wbytes):
    """Algorithmic HBM bytes of each kernel per launch (see the design notes)."""
    blk = 6 if ncomp == 3 else 1
    mapb = 16 if ncomp == 3 else 4
    return {
        "gather_fft": n * (4 + wbytes) + 4 * n + mapb * npix,
        "filter": 14 * n,
        "ifft_bin": 4 * n + n * (4 + wbytes) + 8 * ncomp * npix,
        "map": npix * (16 * ncomp + 8 * blk + mapb),
    }


def b_strict(n, npix, ncomp, wbytes):
    return n * (2 * (4 + wbytes) + 4) + npix * (104 if ncomp == 3 else 24)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id: str):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", dev_id, f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[4 + i]
                          and "Not" not in r[4 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def _multi_rank():
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def fence(dev):
    """Barrier + device synchronize: every rank enters (or leaves) a timed region together."""
    import torch
    if dev.type == "cuda":
        torch.cuda.synchronize(dev)
    if _multi_rank():
        torch.distributed.barrier()
    if dev.type == "cuda":
        torch.cuda.synchronize(dev)


def max_over_ranks(x, dev):
    """The largest of every rank's value of x (the slowest replica sets the job's time)."""
    if not _multi_rank():
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(ms_per_step_local, world, dev):
    """(whole-job iterations/s, ms per step): every rank runs its own replica, so the job
    completes world iterations per step in the slowest rank's time."""
    ms = max_over_ranks(ms_per_step_local, dev)
    return world / (ms / 1e3), ms


# ----------------------------------------------------------------------- CPU oracle
def time_oracle(s, steps, warmup, one_chunk=True):
    """Time the FP64 oracle's messenger step on the host (chunk 0 only when one_chunk,
    scaled by the chunk count)."""
    import oracle.messenger as O
    sub = s
    scale = 1.0
    if one_chunk:
        c = 0
        a, b = int(s["offsets"][c]), int(s["offsets"][c + 1])
        sub = dict(s)
        sub["pix"], sub["tod"] = s["pix"][a:b], s["tod"][a:b]
        sub["cos"] = None if s["cos"] is None else s["cos"][a:b]
        sub["sin"] = None if s["sin"] is None else s["sin"][a:b]
        sub["offsets"] = np.array([0, b - a], dtype=np.int64)
        sub["params"] = s["params"][c:c + 1]
        scale = float(len(s["offsets"]) - 1)
    prob = O.problem_from_synth(sub)
    lam = O.cooling_schedule(O.lambda_max(prob), 10, 10)
    m = np.zeros((sub["npix"], sub["ncomp"]))
    for i in range(warmup):
        m, _ = O.messenger_step(prob, m, lam[i % len(lam)])
    t0 = time.perf_counter()
    for i in range(steps):
        m, _ = O.messenger_step(prob, m, lam[(warmup + i) % len(lam)])
    dt = (time.perf_counter() - t0) / steps * scale
    return 1.0 / dt, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1705_01893_gb300 import synth
    s = synth.config_iqu_512()
    v, dt = time_oracle(s, args.steps, args.warmup, one_chunk=True)
    sample = "chunk 0 of 8 (2^22 samples) per step, time x8; numpy FP64, 1 thread"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(s),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1705_01893_gb300 import binding, build, synth
    if local == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    binding.load()

    s = synth.config_iqu_512()
    n, npix, nc = int(s["offsets"][-1]), s["npix"], s["ncomp"]
    plan = binding.plan_from_synth(s, dev)
    sched = binding.cooling_schedule(plan.lambda_max(), 10, 10)
    m = torch.zeros(npix, nc, dtype=torch.float64, device=dev)
    chi = torch.zeros(max(args.steps, 1) + args.warmup, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    B = binding

    nb = plan.n_batches()

    def step(i, ev=None):
        """One messenger iteration; ev[b][0..3] bracket batch b's three kernels, ev[nb][0..1]
        the map step, all on the launching stream."""
        lam = float(sched[i % len(sched)])
        for b in range(nb):
            if ev is not None:
                ev[b][0].record(stream)
            plan.stage(B.MM_STAGE_GATHER_FFT, b)
            if ev is not None:
                ev[b][1].record(stream)
            plan.stage(B.MM_STAGE_FILTER, b, lam, chi2_slot=chi[i:i + 1])
            if ev is not None:
                ev[b][2].record(stream)
            plan.stage(B.MM_STAGE_IFFT_BIN, b)
            if ev is not None:
                ev[b][3].record(stream)
        if ev is not None:
            ev[nb][0].record(stream)
        plan.stage(B.MM_STAGE_MAP)
        if ev is not None:
            ev[nb][1].record(stream)

    plan.stage(B.MM_STAGE_LOAD, map_inout=m)
    for i in range(args.warmup):
        step(i)
    fence(dev)

    uuid = str(getattr(torch.cuda.get_device_properties(dev), "uuid", local))
    sampler = ClockSampler(("GPU-" + uuid) if "-" in uuid and not uuid.startswith("GPU") else uuid)
    time.sleep(0.3)
    evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(nb + 1)]
           for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(args.warmup + k, evs[k])
    t_end.record(stream)
    fence(dev)
    total_ms = t_start.elapsed_time(t_end)
    stage_names = ["gather_fft", "filter", "ifft_bin"]
    # per-launch durations of each kernel kind (one launch per batch per iteration)
    stage_ms = {nm: [evs[k][b][j].elapsed_time(evs[k][b][j + 1]) for k in range(args.steps)
                     for b in range(nb)] for j, nm in enumerate(stage_names)}
    stage_ms["map"] = [evs[k][nb][0].elapsed_time(evs[k][nb][1]) for k in range(args.steps)]
    _, stage_ms_step = job_rate(total_ms / args.steps, world, dev)

    # the same iterations replayed as one captured CUDA graph per iteration
    mg = m.clone()
    lam_g = np.array([float(sched[(args.warmup + k) % len(sched)]) for k in range(args.steps)])
    plan.messenger_graph(mg, lam_g[:2])
    fence(dev)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    plan.messenger_graph(mg, lam_g)
    g1.record(stream)
    fence(dev)
    clocks = sampler.stop()
    value, ms_step = job_rate(g0.elapsed_time(g1) / args.steps, world, dev)

    # the plain FP64 single-launch-per-iteration step on the same GPU (comparison bar)
    plain_ms = None
    if not args.no_plain:
        mp = m.clone()
        lam_p = np.array([float(sched[k % len(sched)]) for k in range(5)])
        plan.messenger_plain_fp64(mp, lam_p[:1])
        torch.cuda.synchronize(dev)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        plan.messenger_plain_fp64(mp, lam_p)
        p1.record(stream)
        torch.cuda.synchronize(dev)
        plain_ms = p0.elapsed_time(p1) / len(lam_p)

    # cuFFT (through torch.fft, a library call timed only as a comparison) against this
    # library's rfft of the same chunks (column + row kernels, natural-order output)
    fft_cmp = None
    if not args.no_plain:
        tod_dev = plan.tod.view(len(s["offsets"]) - 1, -1)
        spec = torch.empty(tod_dev.shape[0] * (tod_dev.shape[1] // 2 + 1), 2, dtype=torch.float32,
                           device=dev)
        for _ in range(3):
            torch.fft.rfft(tod_dev, dim=1)
            plan.rfft(plan.tod, spec)
        f0, f1, f2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        reps = 10
        f0.record(stream)
        for _ in range(reps):
            torch.fft.rfft(tod_dev, dim=1)
        f1.record(stream)
        for _ in range(reps):
            plan.rfft(plan.tod, spec)
        f2.record(stream)
        torch.cuda.synchronize(dev)
        fft_cmp = {"cufft_rfft_ms": f0.elapsed_time(f1) / reps, "mm_rfft_ms": f1.elapsed_time(f2) / reps,
                   "what": "rfft of 8 x 2^22 float32 samples, complex64 out"}

    # end to end through the public call, host buffers: map in (pinned), one iteration,
    # map and chi^2 out, synchronised every step
    m_host = torch.zeros(npix, nc, dtype=torch.float64).pin_memory()
    m_back = torch.empty_like(m_host).pin_memory()
    c_back = torch.empty(1, dtype=torch.float64).pin_memory()
    m_dev = torch.empty(npix, nc, dtype=torch.float64, device=dev)
    c_dev = torch.zeros(1, dtype=torch.float64, device=dev)
    m_host.copy_(m.cpu())
    e2e_steps = max(3, min(args.steps, 20))
    for i in range(2):
        m_dev.copy_(m_host, non_blocking=True)
        plan.messenger(m_dev, [float(sched[i % len(sched)])], c_dev)
        m_back.copy_(m_dev, non_blocking=True)
        c_back.copy_(c_dev, non_blocking=True)
        torch.cuda.synchronize(dev)
    fence(dev)
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        m_dev.copy_(m_back if i else m_host, non_blocking=True)
        plan.messenger(m_dev, [float(sched[i % len(sched)])], c_dev)
        m_back.copy_(m_dev, non_blocking=True)
        c_back.copy_(c_dev, non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    fence(dev)
    e2e_rate, _ = job_rate(e2e_s * 1e3, world, dev)
    e2e = {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": 8 * npix * nc,
           "d2h_bytes_per_step": 8 * npix * nc + 8}

    tol = time_to_tolerance(plan, s, dev, stream, args) if not args.no_tolerance else None

    if rank != 0:
        return
    wbytes = 8 if s["cos"] is not None and s["cos"].dtype == np.float32 else (4 if nc == 3 else 0)
    # algorithmic bytes of one launch: the three FFT kernels process one batch
    per_batch = bytes_per_stage(n // nb, npix, nc, wbytes)
    full = bytes_per_stage(n, npix, nc, wbytes)
    bps = {k: (per_batch[k] if k != "map" else full[k]) for k in full}
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    avg = {k: sum(v) / len(v) for k, v in stage_ms.items()}
    dom = max(avg, key=lambda k: avg[k])
    achieved = bps[dom] / (avg[dom] * 1e-3) / 1e9
    iter_bytes = sum(full.values())
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        traffic = json.load(open(prof)).get(dom)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(s),
        "tod_gsamples_per_s": n * value / 1e9,
        "iteration_hbm": {"bytes_pass": iter_bytes, "bytes_strict": b_strict(n, npix, nc, wbytes),
                          "frac_pass": iter_bytes / (ms_step * 1e-3) / 1e9 / hbm,
                          "frac_strict": b_strict(n, npix, nc, wbytes) / (ms_step * 1e-3) / 1e9 / hbm,
                          "peak_gbs": hbm, "peak": peak_src},
        "batches": nb,
        "timing": "value/ms_per_step: K iterations replayed as one CUDA graph each (events on "
                  "the launching stream); roofline/stage_ms_per_launch: K iterations launched "
                  "stage by stage with events between the kernels",
        "stage_loop_ms_per_step": stage_ms_step,
        "fp64_plain_ms_per_step": plain_ms,
        "fft_vs_cufft": fft_cmp,
        "speedup_vs_fp64_plain": None if plain_ms is None else plain_ms / ms_step,
        "stage_ms_per_launch": {k: round(v, 5) for k, v in avg.items()},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                     "bytes_per_launch": bps[dom], "peak_source": peak_src},
        "e2e": e2e,
        "gpu_launches": args.steps * (3 * nb + 1),   # per timed region
        "time_to_chi2_tol": tol,
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        v, dt = time_oracle(s, 1, 0, one_chunk=False)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "1 full iteration of the 8 x 2^22 workload, numpy FP64, 1 thread"}
    print(json.dumps(line), flush=True)


def time_to_tolerance(plan, s, dev, stream, args):
    """Iterations and device time for the cooled messenger (10 levels x 10, then lambda = 1)
    and for PCG (the paper's comparison solver, on the same kernels) to bring chi^2 within
    1e-3 and 1e-4 (relative) of chi2_*, the lowest chi^2 either reaches in a long run."""
    import torch
    from paper_1705_01893_gb300 import binding
    npix, nc = s["npix"], s["ncomp"]
    lam_max = plan.lambda_max()
    total = 1 + 100 + args.tol_iters
    runs = {}
    for label, (lv, it) in (("10x10", (10, 10)), ("8x5", (8, 5))):
        cool = binding.cooling_schedule(lam_max, lv, it)
        lam_m = np.concatenate([cool, np.ones(total - len(cool))])
        m = torch.zeros(npix, nc, dtype=torch.float64, device=dev)
        chi = torch.zeros(len(lam_m), dtype=torch.float64, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.messenger(m, lam_m, chi)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        runs[label] = (chi.cpu().numpy(), e0.elapsed_time(e1) / len(lam_m))
    ms_m = runs["10x10"][1]
    n_pcg = total
    x = torch.zeros(npix, nc, dtype=torch.float64, device=dev)
    chi_p = torch.zeros(n_pcg, dtype=torch.float64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.pcg(x, n_pcg, restart=True, chi2_out=chi_p)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_p = e0.elapsed_time(e1) / n_pcg
    cp = chi_p.cpu().numpy()
    star = float(min(min(r[0].min() for r in runs.values()), cp.min()))

    def reach(ch, tol_rel):
        ok = np.flatnonzero((ch - star) / star <= tol_rel)
        return int(ok[0]) if ok.size else None

    out = {"chi2_star": star, "n_samples": int(s["offsets"][-1]), "iterations_run": total,
           "pcg": {"preconditioner": "3x3 pixel-block Jacobi", "ms_per_iter": ms_p,
                   "final_rel": float((cp[-1] - star) / star)}}
    series = [("pcg", cp, ms_p)]
    for label, (ch, ms) in runs.items():
        key = "messenger_" + label
        out[key] = {"schedule": "1 x inf, %s geometric to 1, then lambda = 1" % label,
                    "ms_per_iter": ms, "final_rel": float((ch[-1] - star) / star)}
        series.append((key, ch, ms))
    for name, ch, ms in series:
        for t in (1e-3, 1e-4):
            it = reach(ch, t)
            out[name]["iters_%g" % t] = it
            out[name]["ms_%g" % t] = None if it is None else it * ms
    return out


def plan_groups(s):
    lens = np.diff(s["offsets"])
    return sorted(set(int(x) for x in lens))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tolerance", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--tol-iters", type=int, default=400,
                    help="lambda = 1 iterations after the cooling schedule (and PCG length)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
