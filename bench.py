#!/usr/bin/env python
"""Throughput of the stacking hot path on one GB300 (or N independent replicas).

One step = the whole hot path over one batch: matched-filter planes of every
exposure (load_exposures), propagate/project/gather/stack of every orbit
against every exposure (stack_orbits), and the candidate stage: every orbit
with stacked SNR >= 5 ranked (count_candidates, topk_candidates),
near-duplicates dropped (dedup_candidates) and, for the chosen form, the
list vetted by the CNN (vet) and by outlier trimming (trim_candidates).
Workload: the MBA-scale synthetic survey (200 exposures of 4096 x 4096 over
30 nights, 1,000 injected main-belt asteroids, 16.4 M candidate orbits),
inputs resident in HBM (13-27 GB of planes, far larger than L2).  ``value``
is orbit x exposure samples/s of the chosen form (BF16 planes, persistent
work queue, CUDA graph, autotuned tiles, CNN vetting); the plain form (FP32
planes, one thread per orbit, SNR threshold) is measured in the same run,
and the batched uneven workload as a sub-record.

With ``--impl reference`` the same metric is measured for the FP64 CPU
oracle on the host cores, on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "orbit×exposure samples/s and vetted candidates/s at fixed recall, plain vs chosen"
UNIT = "samples/s"
# The stack kernel's bound is the FP64 pipe.  From unit counts it issues 2
# thread-instructions per SM per clock (152 SMs, 2.07 GHz), 629.3 G/s; the
# roofline's denominator is the rate measured at run time
# (ndt_measure_fp64_rate), reported beside this derived figure.  The fraction
# is the FP64-pipe time the launch needs (instructions per computed sample x
# computed samples / that rate) over its measured time.
FP64_PIPE_PEAK_GIPS = 152 * 2 * 2.07
# FP64 work per computed (orbit, exposure) sample of each stack kernel form,
# from ncu thread-instruction counters (smsp__sass_thread_inst_executed_op_
# {dfma,dmul,dadd}_pred_on.sum) over the samples whose FP64 work ran in the
# captured launch (samples minus those the off-chip and block tests removed):
# (DFMA, DMUL, DADD) per computed sample; flops = 2 DFMA + DMUL + DADD.
# MBA: the workload at 512 orbits per family and 1024 x 1024 images (1.024e8
# samples; chosen 8.637e7 computed); batched: 128 families and 512 x 512
# images (chosen 2.022e8 computed samples; its FP64-state figure, 2.037e8,
# predates the block test).
FP64_MIX = {("mba", "chosen"): (0.119, 0.059, 0.012),
            ("batched", "chosen"): (2.692, 1.458, 0.314),
            ("mba", "chosen_fp64_state"): (23.71, 13.38, 1.98),
            ("mba", "plain"): (22.95, 11.94, 1.98),
            ("mba", "plain_fp64"): (67.95, 42.96, 7.98),
            ("batched", "chosen_fp64_state"): (32.06, 18.23, 2.04)}
# The double-float state forms spend few FP64 instructions per sample and
# are bound by instruction issue: one warp instruction per clock per
# scheduler, 4 schedulers per SM, 152 SMs at 2.07 GHz = 1258.6 G warp-
# instructions/s.  Their roofline: warp instructions issued per computed
# sample (ncu smsp__inst_executed.sum over the computed samples of the
# captured launch, same small cases as above) x computed samples over the
# kernel's CUDA-event time, against that peak.
ISSUE_PEAK_G = 152 * 4 * 2.07
ISSUE_PER_SAMPLE = {("mba", "chosen"): 33.55, ("batched", "chosen"): 43.83}
# DRAM bytes (read + write) of one stack launch on the small MBA case above
# (200 exposures of 1024 x 1024, 512 orbits per family; BF16 planes 0.84 GB,
# FP32 1.68 GB, both larger than L2), ncu dram__bytes_read.sum +
# dram__bytes_write.sum, with that case's algorithmic bytes (plane pairs of
# the on-chip samples).  Family members read the same pixels, so traffic
# grows more slowly than the orbit count: it is not scaled to the full
# launch, whose own traffic stays null.
TRAFFIC_SMALL_CASE = {("mba", "chosen"): (168937472, 343890136),
                      ("mba", "chosen_fp64_state"): (142358272, 343890136),
                      ("mba", "plain"): (178343680, 687780272),
                      ("mba", "plain_fp64"): (177772544, 687780272)}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["mba", "batched", "sparse"], default="mba",
                   help="mba: the MBA-scale survey (default); batched: uneven orbit families; "
                        "sparse: 20,000 small exposures, each orbit on well under 1 % of them")
    p.add_argument("--n-fam", type=int, default=4096, help="families of the batched workload")
    p.add_argument("--fam-size", type=int, default=16384, help="orbits per family")
    p.add_argument("--n-true", type=int, default=1000)
    p.add_argument("--size", type=int, default=None,
                   help="image side (default 4096 for mba, 2048 for batched)")
    p.add_argument("--n-exp", type=int, default=200)
    p.add_argument("--plane", default="bf16", choices=["f32", "bf16", "f16"])
    p.add_argument("--forms", default="chosen,chosen_fp64_state,plain,plain_fp64",
                   help="chosen (BF16, persistent, graph, vetting), plain (FP32 planes, one thread "
                        "per orbit), plain_fp64 (plain with FP64 light time and TAN projection)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--tiles", default=None, help="fixed OT,ET for the persistent form (no autotune)")
    p.add_argument("--no-vet", action="store_true", help="skip the CNN vetting stage")
    p.add_argument("--no-noise", action="store_true", help="skip the iterative-MAD noise timing")
    p.add_argument("--no-batched", action="store_true",
                   help="skip the batched uneven workload's sub-record (MBA runs only)")
    p.add_argument("--no-sparse", action="store_true",
                   help="skip the sparse-regime sub-record (MBA runs only)")
    p.add_argument("--vet-skies", type=int, default=12, help="vetting skies used for training")
    p.add_argument("--vet-train-stamps", type=int, default=200_000,
                   help="stamps in the vetting network's training set (vetting skies, then MBA-like "
                        "survey skies until the count is reached)")
    p.add_argument("--vet-batch", type=int, default=1 << 20,
                   help="candidates of the separately timed vetting pass (0: skip)")
    a = p.parse_args()
    if a.size is None:
        a.size = 2048 if a.workload == "batched" else 4096
    return a


# ----------------------------------------------------------------- clocks ----

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------- workload ----

def make_workload(args, rank, device):
    import torch
    from paper_2503_08854_gb300 import ndt, synth
    stream = torch.cuda.Stream(device=device)
    if args.workload == "batched":
        sky = synth.batched_sky(n_fam=args.n_fam, fam_size=args.fam_size, seed=4 + rank,
                                size=args.size, scale_arcsec=60.0 * 2048 / args.size)
        imgs = synth.noise_images_torch(sky.ex, sky.seed, device)
        sky.fam_dev = tuple(torch.from_numpy(np.ascontiguousarray(x)).to(device)
                            for x in sky.families)
        states = torch.from_numpy(np.ascontiguousarray(sky.states.T)).to(device)
        torch.cuda.synchronize(device)
        return sky, stream, imgs, states
    if args.workload == "sparse":
        sky = synth.sparse_sky(seed=7 + rank)
        sky.fam_dev = None
        # the orbits are seen around opposition, near t0: duplicates are judged there
        sky.dedup_window = (sky.t0 - 20.0, sky.t0 + 20.0)
        imgs = synth.noise_images_torch(sky.ex, sky.seed, device)
        ctx = ndt.create(device.index, stream)
        try:
            ndt.load_exposures(ctx, sky.ex, imgs, plane_dtype="f32")
            st = torch.from_numpy(np.ascontiguousarray(sky.inj_states.T)).to(device)
            xy = torch.empty(len(sky.inj_states) * sky.ex.n * 2, dtype=torch.float64, device=device)
            torch.cuda.synchronize(device)
            ndt.predict_positions(ctx, st, sky.t0, len(sky.inj_states), xy)
        finally:
            ndt.destroy(ctx)
        xy = xy.view(len(sky.inj_states), sky.ex.n, 2)
        W = float(sky.ex.width[0])
        far = (xy[..., 0] < -20) | (xy[..., 0] > W + 20) | (xy[..., 1] < -20) | (xy[..., 1] > W + 20)
        xy[far] = float("nan")                 # render only where a source is near the chip
        synth.render_sources_torch(imgs, xy, sky.inj_flux, sky.ex.sigma)
        states = torch.from_numpy(np.ascontiguousarray(sky.states.T)).to(device)
        torch.cuda.synchronize(device)
        return sky, stream, imgs, states
    sky = synth.mba_sky(n_exp=args.n_exp, size=args.size, n_true=args.n_true,
                        fam_size=args.fam_size, seed=2 + rank,
                        scale_arcsec=10.5 * 4096 / args.size)
    sky.fam_dev = None
    imgs = synth.noise_images_torch(sky.ex, sky.seed, device)
    # injected sources at positions from the library's own position kernel
    ctx = ndt.create(device.index, stream)
    try:
        torch.cuda.synchronize(device)
        ndt.load_exposures(ctx, sky.ex, imgs, plane_dtype="f32")
        st = torch.from_numpy(np.ascontiguousarray(sky.inj_states.T)).to(device)
        xy = torch.empty(len(sky.inj_states) * sky.ex.n * 2, dtype=torch.float64, device=device)
        torch.cuda.synchronize(device)
        ndt.predict_positions(ctx, st, sky.t0, len(sky.inj_states), xy)
    finally:
        ndt.destroy(ctx)
    synth.render_sources_torch(imgs, xy.view(len(sky.inj_states), sky.ex.n, 2), sky.inj_flux,
                               sky.ex.sigma)
    states = torch.from_numpy(np.ascontiguousarray(sky.states.T)).to(device)
    torch.cuda.synchronize(device)
    return sky, stream, imgs, states


class Form:
    def __init__(self, name, plane, mode, graph, block=True, geom64=False, df=False):
        self.name, self.plane, self.mode, self.graph, self.block = name, plane, mode, graph, block
        self.geom64, self.df = geom64, df


NU_MIN = 5.0        # detection threshold of the candidate list (stacked SNR)
DEDUP_PX = 3.0      # duplicate radius at the reference exposures (px)
DEDUP_REFS = 3      # reference exposures of the duplicate test
MATCH_PX = 2.0      # a list entry matches its asteroid within this RMS track distance (px)
FIXED_RECALL = 0.9  # the recall at which false-positive rates are compared


class Candidates:
    """The candidate stage of one context: every orbit of the stack with
    nu >= NU_MIN, ranked (ndt_count_candidates + ndt_topk_candidates),
    near-duplicates dropped (ndt_dedup_candidates), and for the chosen form
    the list vetted by the CNN (ndt_vet) and by outlier trimming
    (ndt_trim_candidates)."""

    def __init__(self, n, device, vet_params=None, window=None):
        import torch
        self.window = window
        self.idx = torch.empty(n, dtype=torch.int64, device=device)
        self.keep = torch.empty(n, dtype=torch.int64, device=device)
        self.vet_params = vet_params
        if vet_params is not None:
            self.scores = torch.empty(n, device=device)
            self.trim = torch.empty(n, device=device)
        self.m = self.nk = 0

    def run(self, ctx, states, t0, n):
        from paper_2503_08854_gb300 import ndt
        self.m = ndt.count_candidates(ctx, NU_MIN)
        ndt.topk_candidates(ctx, self.m, self.idx)
        self.nk = ndt.dedup_candidates(ctx, states, t0, n, self.idx, self.m, self.keep,
                                       radius_px=DEDUP_PX, n_ref=DEDUP_REFS, window=self.window)
        if self.vet_params is not None and self.nk > 0:
            lst = self.keep[:self.nk]
            ndt.vet(ctx, self.vet_params, states, t0, n, lst, self.scores[:self.nk])
            ndt.trim_candidates(ctx, states, t0, n, lst, self.trim[:self.nk])
        return self.nk


def run_steps(ctx, stream, sky, imgs, states, n_steps, plane, cand):
    """Device-resident steps; per-step device time from CUDA events on the
    library's stream (the whole step and its candidate stage), plus the
    stack kernel's own event time."""
    import torch
    from paper_2503_08854_gb300 import ndt
    n = states.shape[1]
    step_ms, stack_ms, cand_ms = [], [], []
    for _ in range(n_steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ndt.load_exposures(ctx, sky.ex, imgs, plane_dtype=plane)
        ndt.stack_orbits(ctx, states, sky.t0, n, families=sky.fam_dev)
        e2.record(stream)
        cand.run(ctx, states, sky.t0, n)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        cand_ms.append(e2.elapsed_time(e1))
        stack_ms.append(ndt.get_stats(ctx)["last_stack_ms"])
    return step_ms, stack_ms, cand_ms


def train_vetter(device, seed=5, n_train_sky=12, n_test_sky=3, train_stamps=200_000, max_survey_skies=24):
    """Untimed setup: synthesise vetting stamps with the library and train the
    CNN with the library's forward/backward/Adam kernels.  Two sources:
    vetting skies (injected asteroids vs random orbits, single-exposure
    artefacts and noise peaks, 10 exposures of 1024^2) and MBA-like survey
    skies (the MBA workload's cadence, chips, PSF and noise; positives are
    orbits tracking an injected asteroid within MATCH_PX, negatives orbits
    that share only part of its path, and noise peaks) until the training
    set holds ``train_stamps`` stamps in all.  The false-positive rate at 90 % recall
    is measured on held-out vetting skies here and on the MBA survey's own
    candidate list in the benchmark."""
    import torch
    from paper_2503_08854_gb300 import ndt, vetting
    stream = torch.cuda.Stream(device=device)
    ctx = ndt.create(device.index, stream)
    try:
        t = time.perf_counter()
        xs, ys = [], []
        x, y, kind, _ = vetting.make_set(ctx, seed, device, n_sky=n_train_sky)
        xs.append(x); ys.append(y)
        n_vet, n_survey, skies = int(x.shape[0]), 0, 0
        while n_vet + n_survey < train_stamps and skies < max_survey_skies:
            x, y, _, _ = vetting.make_survey_set(ctx, seed * 100 + skies, device)
            xs.append(x); ys.append(y)
            n_survey += x.shape[0]
            skies += 1
        x, y = torch.cat(xs), torch.cat(ys)
        xt, yt, kt, st, tt = vetting.make_set(ctx, seed + 1, device, n_sky=n_test_sky, trimmed=True)
        torch.cuda.synchronize(device)
        t_data = time.perf_counter() - t
        p = vetting.init_params(seed, device)
        t = time.perf_counter()
        losses = vetting.train(ctx, p, x, y, epochs=4, batch=256, lr=2e-3)
        t_train = time.perf_counter() - t
        z = vetting.logits(ctx, p, xt).cpu().numpy()
    finally:
        ndt.destroy(ctx)
    pos = kt == 0
    fpr_cnn, _ = vetting.fpr_at_recall(z[pos], z[~pos], 0.9)
    fpr_snr, _ = vetting.fpr_at_recall(st[pos], st[~pos], 0.9)
    fpr_trim, _ = vetting.fpr_at_recall(tt[pos], tt[~pos], 0.9)
    info = {"train_stamps": int(x.shape[0]), "survey_stamps": int(n_survey), "survey_skies": skies,
            "test_stamps": int(xt.shape[0]), "train_steps": len(losses), "train_s": round(t_train, 2),
            "train_stamps_per_s": len(losses) * 256 / t_train, "data_s": round(t_data, 2),
            "final_loss": float(np.mean(losses[-5:])),
            "fpr_at_90pct_recall_vetting_skies": {"cnn": fpr_cnn, "snr_threshold": fpr_snr,
                                                  "trimmed_snr_threshold": fpr_trim},
            "workload": "vetting skies (10 exposures 1024^2; 400 injected asteroids of stacked "
                        "SNR 3-10, 400 random orbits, 400 one-exposure artefacts, 400 noise peaks "
                        "each) and MBA-like survey skies (200 exposures 4096^2, 1000 asteroids of "
                        "per-image SNR 0.3-3 with 512 orbits each)"}
    return p, info


def list_quality(ctx, cand, sky, states, snr_all, device):
    """Untimed: recall of the candidate list and false-positive rates at
    FIXED_RECALL of its scorers.  An entry matches the asteroid of its family
    when its predicted track stays within MATCH_PX (RMS over the exposures
    where the asteroid is on the chip); recall = asteroids with a matching
    entry; the FPR of a scorer is the fraction of non-matching entries that
    pass the threshold keeping FIXED_RECALL of the asteroids."""
    from paper_2503_08854_gb300 import vetting
    nk = cand.nk
    n_obj = len(sky.inj_states)
    if nk == 0 or not np.any(sky.inj_flux > 0):
        return {"list": nk, "above_threshold": cand.m}
    lst = cand.keep[:nk].cpu().numpy()
    rms = vetting.track_rms(ctx, sky, lst, device)
    match = rms < MATCH_PX
    obj = lst // sky.meta["fam_size"]
    out = {"list": int(nk), "above_threshold": int(cand.m), "matching": int(match.sum()),
           "recall": float(len(np.unique(obj[match])) / n_obj),
           "recall_def": f"injected asteroids with a list entry tracking them within {MATCH_PX} px RMS",
           "fixed_recall": FIXED_RECALL, "fpr_at_fixed_recall": {}, "thresholds": {}}
    scorers = {"snr_threshold": snr_all[cand.keep[:nk]].cpu().numpy()}
    if cand.vet_params is not None:
        scorers["cnn"] = cand.scores[:nk].cpu().numpy()
        scorers["trimmed_snr_threshold"] = cand.trim[:nk].cpu().numpy()
    for name, sc in scorers.items():
        fpr, thr = vetting.fpr_at_object_recall(sc, match, obj, n_obj, FIXED_RECALL)
        out["fpr_at_fixed_recall"][name] = fpr
        out["thresholds"][name] = thr
    return out


def bench_form(args, form, sky, stream, imgs, states, device, barrier, vet_params=None):
    import torch
    from paper_2503_08854_gb300 import ndt
    n = states.shape[1]
    ctx = ndt.create(device.index, stream)
    try:
        ndt.set_block_test(ctx, form.block)
        ndt.set_fp64_geometry(ctx, form.geom64)
        ndt.set_df_state(ctx, form.df)
        tiles = None
        if form.mode == "persistent":
            if args.tiles:
                ot, et = (int(x) for x in args.tiles.split(","))
                tiles = {"orbit_tile": ot, "exp_tile": et, "sweep_ms": None}
            else:
                ndt.load_exposures(ctx, sky.ex, imgs, plane_dtype=form.plane)
                times = np.zeros(9, np.float32)
                ndt.autotune(ctx, states, sky.t0, n, families=sky.fam_dev, times_ms=times)
                st = ndt.get_stats(ctx)
                ot, et = st["orbit_tile"], st["exp_tile"]
                tiles = {"orbit_tile": ot, "exp_tile": et,
                         "sweep_ms": [round(float(t), 2) for t in times]}
            ndt.set_launch(ctx, ndt.LAUNCH_PERSISTENT, ot, et, use_graph=form.graph)
        cand = Candidates(n, device, vet_params if form.name == "chosen" else None,
                          getattr(sky, "dedup_window", None))
        run_steps(ctx, stream, sky, imgs, states, args.warmup, form.plane, cand)
        launches0 = ndt.get_stats(ctx)["kernel_launches"]
        barrier()
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        # NVTX range "timed_<form>": lets a profiler select exactly these launches
        torch.cuda.nvtx.range_push(f"timed_{form.name}")
        step_ms, stack_ms, cand_ms = run_steps(ctx, stream, sky, imgs, states, args.steps, form.plane,
                                               cand)
        torch.cuda.synchronize(device)
        torch.cuda.nvtx.range_pop()
        wall = time.perf_counter() - t0
        stats = ndt.get_stats(ctx)
        launches = stats["kernel_launches"] - launches0
        snr_all = torch.empty(n, device=device)     # untimed: one more stack for the list's nu
        ndt.stack_orbits(ctx, states, sky.t0, n, families=sky.fam_dev, snr=snr_all)
        ndt.synchronize(ctx)
        quality = list_quality(ctx, cand, sky, states, snr_all, device)
        out = dict(step_ms=step_ms, stack_ms=stack_ms, cand_ms=cand_ms,
                   wall_s=wall, launches=launches, skipped=stats["offchip_skipped"],
                   valid=stats["valid_samples"], samples=stats["samples"], quality=quality,
                   blocked=stats["block_skipped"],
                   planes_ms=stats["last_planes_ms"], topk_ms=stats["last_topk_ms"], tiles=tiles)
        if cand.vet_params is not None and args.vet_batch > 0:
            out["vet_batch"] = vet_batch_rate(args, ctx, stream, sky, states, vet_params, device)
        e2e = None
        if not args.no_e2e and form.name == "chosen":
            e2e = bench_e2e(args, ctx, stream, sky, imgs, states, cand, form, barrier, device)
        return out, e2e
    finally:
        ndt.destroy(ctx)


def hbm_peak_gbs():
    """Measured copy bandwidth of this machine's GPUs (MEASURED_PEAKS.json beside
    this file), else the 6.8 TB/s fallback of an earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def vet_batch_rate(args, ctx, stream, sky, states, vet_params, device):
    """Vetting throughput at the learned-vetting workload's scale: the top
    ``--vet-batch`` candidates of the stacked batch (ranked once, untimed)
    get stamps and CNN scores; CUDA events time that call alone."""
    import torch
    from paper_2503_08854_gb300 import ndt
    n = states.shape[1]
    m = min(args.vet_batch, n)
    idx = torch.empty(m, dtype=torch.int64, device=device)
    ndt.topk_candidates(ctx, m, idx)
    scores = torch.empty(m, device=device)
    ndt.vet(ctx, vet_params, states, sky.t0, n, idx, scores)     # warm-up
    ms = []
    for _ in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ndt.vet(ctx, vet_params, states, sky.t0, n, idx, scores)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.mean(ms)
    # the stamps alone (track positions + gathers), and their gather bytes:
    # 441 plane pairs (4 B each, BF16) per in-bounds exposure of a candidate
    stamps = torch.empty((m, 2, 21, 21), dtype=torch.int16, device=device)
    ndt.stamps(ctx, states, sky.t0, n, idx, stamps_bf16=stamps)                # warm-up
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ndt.stamps(ctx, states, sky.t0, n, idx, stamps_bf16=stamps)
    e1.record(stream)
    e1.synchronize()
    t_st = e0.elapsed_time(e1)
    del stamps
    nobs = torch.empty(n, dtype=torch.int32, device=device)
    ndt.stack_orbits(ctx, states, sky.t0, n, families=sky.fam_dev, nobs=nobs)
    ndt.synchronize(ctx)                       # nobs is read on torch's stream
    pairs = int(nobs[idx].to(torch.int64).sum().item())
    gather = pairs * 441 * 4
    peak = hbm_peak_gbs()
    return {"candidates": m, "ms": t, "vetted_candidates_per_s": m / (t / 1e3),
            "exposures": int(sky.ex.n),
            "stamps": {"ms": t_st, "in_bounds_pairs": pairs, "gather_bytes": gather,
                       "gather_gbs": gather / (t_st / 1e3) / 1e9, "hbm_peak_gbs": peak,
                       "frac_of_hbm": gather / (t_st / 1e3) / 1e9 / peak,
                       "note": "gathers of the candidates' 21 x 21 windows; near-duplicate candidates "
                               "share windows, so most hit L2 (latency-bound, not HBM-bound)"}}


def noise_rate(device, stream, imgs):
    """Iterative-MAD noise estimate of every image (ndt_noise_mad), timed
    with CUDA events; its roofline is the HBM read rate (each selection
    pass streams the image once; the library counts the bytes)."""
    import torch
    from paper_2503_08854_gb300 import ndt
    ctx = ndt.create(device.index, stream)
    try:
        views = [imgs[j] for j in range(imgs.shape[0])]
        ndt.noise_mad(ctx, views)                                   # warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        med, sig, rnd = ndt.noise_mad(ctx, views)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        read = float(ndt.get_stats(ctx)["noise_bytes_read"])
    finally:
        ndt.destroy(ctx)
    return {"images": len(views), "ms": ms, "rounds_max": int(rnd.max()), "rounds_mean": float(rnd.mean()),
            "read_bytes": read, "passes_per_image": read / (4.0 * views[0].numel() * len(views)),
            "read_gbps": read / (ms / 1e3) / 1e9}


def bench_e2e(args, ctx, stream, sky, imgs, states, cand_dev, form, barrier, device):
    """Same steps through the public API from pinned HOST buffers.  Every step
    copies its images (ndt_load_exposures from host memory) and its orbit
    states (one copy to the device, then used by every call) from pinned
    host memory, runs the stack and the candidate stage, and reads the
    candidate list (and for the chosen form its CNN scores and trimmed nu)
    back to pinned host memory, all inside the timed region.  Steps alternate
    between two new contexts with the form's launch configuration, each on
    its own stream, as a survey pipeline would: while one context stacks step
    i, the other loads step i+1's images, so the host-to-device copies
    overlap the stack kernel."""
    import torch
    from paper_2503_08854_gb300 import ndt
    n = states.shape[1]
    st = ndt.get_stats(ctx)
    streams = [torch.cuda.Stream(device=device) for _ in range(2)]
    ctxs = [ndt.create(device.index, s) for s in streams]
    vet_params = cand_dev.vet_params
    try:
        for c in ctxs:
            ndt.set_block_test(c, form.block)
            ndt.set_fp64_geometry(c, form.geom64)
            ndt.set_df_state(c, form.df)
            if form.mode == "persistent":
                ndt.set_launch(c, ndt.LAUNCH_PERSISTENT, st["orbit_tile"], st["exp_tile"], use_graph=form.graph)
        cands = [Candidates(n, device, vet_params, cand_dev.window) for _ in range(2)]
        st_dev = [torch.empty_like(states) for _ in range(2)]
        ref_list = cand_dev.keep[:cand_dev.nk].cpu().numpy()     # the device-input steps' list
        h_imgs = torch.empty(imgs.shape, dtype=imgs.dtype, pin_memory=True)
        h_imgs.copy_(imgs)
        h_states = torch.empty(states.shape, dtype=states.dtype, pin_memory=True)
        h_states.copy_(states)
        torch.cuda.synchronize(device)
        # untimed: the host link's rate for this very buffer, for context
        scratch = torch.empty_like(imgs)
        link = []
        for _ in range(3):
            t = time.perf_counter()
            scratch.copy_(h_imgs, non_blocking=True)
            torch.cuda.synchronize(device)
            link.append(time.perf_counter() - t)
        del scratch
        torch.cuda.empty_cache()
        link_gbs = h_imgs.numel() * 4 / min(link) / 1e9
        h_out = [torch.empty(n, dtype=torch.int64, pin_memory=True) for _ in range(2)]
        h_sc = [torch.empty((2, n), dtype=torch.float32, pin_memory=True) for _ in range(2)]
        np_imgs = h_imgs.numpy()
        stack_ms, d2h = [], []

        def run(n_steps):
            with torch.cuda.stream(streams[0]):
                st_dev[0].copy_(h_states, non_blocking=True)
            ndt.load_exposures(ctxs[0], sky.ex, np_imgs, plane_dtype=form.plane)
            for i in range(n_steps):
                b = i % 2
                c, cd = ctxs[b], cands[b]
                ndt.stack_orbits(c, st_dev[b], sky.t0, n, families=sky.families)   # returns at once
                if i + 1 < n_steps:                                               # overlaps the stack
                    with torch.cuda.stream(streams[1 - b]):
                        st_dev[1 - b].copy_(h_states, non_blocking=True)
                    ndt.load_exposures(ctxs[1 - b], sky.ex, np_imgs, plane_dtype=form.plane)
                nk = cd.run(c, st_dev[b], sky.t0, n)
                with torch.cuda.stream(streams[b]):
                    h_out[b][:nk].copy_(cd.keep[:nk], non_blocking=True)
                    nb = 8 * nk
                    if vet_params is not None:
                        h_sc[b][0, :nk].copy_(cd.scores[:nk], non_blocking=True)
                        h_sc[b][1, :nk].copy_(cd.trim[:nk], non_blocking=True)
                        nb += 8 * nk
                streams[b].synchronize()
                d2h.append(nb)
                stack_ms.append(ndt.get_stats(c)["last_stack_ms"])   # c's stream is idle here
            return (n_steps - 1) % 2

        run(max(1, args.warmup))
        barrier()
        torch.cuda.synchronize(device)
        stack_ms.clear()
        d2h.clear()
        t0 = time.perf_counter()
        last = run(args.steps)
        torch.cuda.synchronize(device)
        dt = (time.perf_counter() - t0) / args.steps
        got = np.array(h_out[last][:cands[last].nk].numpy())
    finally:
        for c in ctxs:
            ndt.destroy(c)
    h2d = int(h_imgs.numel() * 4 + h_states.numel() * 8)
    same = {"equal": bool(len(got) == len(ref_list) and np.array_equal(got, ref_list)),
            "list": int(len(got)), "device_list": int(len(ref_list))}
    return dict(s_per_step=dt, h2d=h2d, d2h=int(statistics.mean(d2h)), link_gbs=link_gbs,
                list_equals_device=same, stack_ms=statistics.mean(stack_ms), stack_ms_max=max(stack_ms))


# ------------------------------------------------------------ cpu oracle ----

def cpu_oracle_rate(sky, host_imgs, seconds, rng_seed=0):
    """The FP64 oracle as it stands, on a bounded random sample of the orbits of
    the same workload against all exposures, planes evaluated at the gathered
    pixels from the same images.  Returns (samples/s, threads, description)."""
    import oracle as O
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(rng_seed)
    n_exp = sky.ex.n
    imgs = [host_imgs[j] for j in range(n_exp)]
    m = 64
    elapsed = 0.0
    while True:
        sel = np.sort(rng.choice(len(sky.states), m, replace=False))
        t = time.perf_counter()
        O.stack(sky.states[sel], sky.t0, sky.ex, images=imgs, nthreads=threads)
        elapsed = time.perf_counter() - t
        cap = min(2_000_000, len(sky.states))
        if elapsed >= 0.15 * seconds or m >= cap:
            break
        m = int(min(m * max(2.0, 0.3 * seconds / max(elapsed, 1e-3)), cap))
    rate = m * n_exp / elapsed
    return rate, threads, f"{m} random orbits x {n_exp} exposures ({m * n_exp} samples, {elapsed:.1f} s)"


def reference_arm(args):
    """--impl reference: the oracle, on the host cores, steps of a bounded
    sample of the same workload (random orbits against their exposures)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_2503_08854_gb300 import synth
    if args.workload == "batched":
        sky = synth.batched_sky(n_fam=args.n_fam, fam_size=args.fam_size, seed=4, size=args.size,
                                scale_arcsec=60.0 * 2048 / args.size)
    else:
        sky = synth.mba_sky(n_exp=args.n_exp, size=args.size, n_true=args.n_true,
                            fam_size=args.fam_size, seed=2, scale_arcsec=10.5 * 4096 / args.size)
    imgs = synth.noise_images(sky.ex, sky.seed)   # numpy noise: the rate does not depend on values
    threads = os.cpu_count() or 1
    per_step = min(2000, len(sky.states))
    rng = np.random.default_rng(1)

    def step():
        sel = np.sort(rng.choice(len(sky.states), per_step, replace=False))
        fams = None
        n_samples = per_step * sky.ex.n
        if sky.families is not None:
            fo, fe, fi = sky.families
            f_of = np.searchsorted(fo, sel, side="right") - 1
            lists = [fi[fe[f]:fe[f + 1]] for f in f_of]
            mfe = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int64)
            fams = (np.arange(per_step + 1, dtype=np.int64), mfe, np.concatenate(lists))
            n_samples = int(mfe[-1])
        O.stack(sky.states[sel], sky.t0, sky.ex, images=list(imgs), families=fams, nthreads=threads)
        return n_samples

    for _ in range(args.warmup):
        step()
    total = 0
    t = time.perf_counter()
    for _ in range(args.steps):
        total += step()
    dt = (time.perf_counter() - t) / args.steps
    v = total / args.steps / dt
    states_t = np.empty((6, len(sky.states)))                  # shape only, for the name
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args, sky, states_t), "form": "oracle, FP64, host cores",
                       "sample": f"{per_step} random orbits per step against their exposures"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} random orbits per step against their exposures"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def workload_name(args, sky, states):
    n = states.shape[1]
    if args.workload == "batched":
        fo, fe, _ = sky.families
        return (f"batched uneven families: {len(fo) - 1} families x {args.fam_size} orbits "
                f"(NEO/MBA/KBO), {int((fe[1:] - fe[:-1]).min())}-{int((fe[1:] - fe[:-1]).max())} "
                f"of {sky.ex.n} exposures {int(sky.ex.width[0])}^2 each, candidates nu >= {NU_MIN} "
                f"deduplicated")
    return (f"MBA-scale survey: {sky.ex.n} exposures {args.size}x{args.size}, {n} candidate "
            f"orbits ({args.n_true} families), all orbits x all exposures, candidates nu >= {NU_MIN} "
            f"deduplicated and vetted")


# ------------------------------------------------------------------- main ----

def fp64_rates(device):
    """Measured FP64 issue rates (G thread-instructions/s) of this GPU."""
    from paper_2503_08854_gb300 import ndt
    return {op: max(ndt.measure_fp64_rate(device.index, op) for _ in range(2)) / 1e9
            for op in ("dfma", "dmul", "dadd")}


def stack_roofline(workload, form, plane, res, rates):
    """Roofline of a stack kernel form.  FP64 state: FP64-pipe thread
    instructions per computed sample (ncu, FP64_MIX) x computed samples over
    the kernel's CUDA-event time, against the measured DFMA issue rate; the
    mix weighted by the measured DFMA/DMUL/DADD rates gives the bound the mix
    itself allows.  Double-float state: warp instructions issued per computed
    sample (ISSUE_PER_SAMPLE) against the issue peak, with the FP64 pipe's
    share beside it when its mix was measured."""
    mix = FP64_MIX.get((workload, form))
    issue = ISSUE_PER_SAMPLE.get((workload, form))
    if mix is None and issue is None:
        return None
    samples = res["samples"]
    stack_s = statistics.mean(res["stack_ms"]) / 1e3
    computed = samples - res["skipped"]        # the walk runs only for these
    out = {"bound": "alu", "traffic": None, "fp64_samples_per_launch": computed,
           "algorithmic_bytes_per_launch": (8 if plane == "f32" else 4) * res["valid"]}
    small = TRAFFIC_SMALL_CASE.get((workload, form))
    out["traffic_small_case"] = None if small is None else {
        "bytes_per_launch": small[0], "algorithmic_bytes_per_launch": small[1],
        "workload": "200 exposures 1024x1024, 512,000 orbits (1000 families)",
        "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum"}
    fp64 = None
    if mix is not None:
        n_fma, n_mul, n_add = mix
        inst = n_fma + n_mul + n_add
        gips = inst * computed / stack_s / 1e9
        mix_ns = n_fma / rates["dfma"] + n_mul / rates["dmul"] + n_add / rates["dadd"]
        peak_mix = inst / mix_ns
        fp64 = {"achieved": gips, "peak": rates["dfma"], "unit": "G FP64-pipe thread-instructions/s",
                "frac": gips / rates["dfma"],
                "peak_source": "measured: DFMA chains at full occupancy (ndt_measure_fp64_rate)",
                "peak_derived_from_unit_counts": FP64_PIPE_PEAK_GIPS,
                "fp64_rates_measured_gips": rates,
                "peak_for_this_mix": peak_mix, "frac_of_mix_peak": gips / peak_mix,
                "fp64_inst_per_sample": inst, "fp64_mix_per_sample": mix,
                "fp64_tflops": (2 * n_fma + n_mul + n_add) * computed / stack_s / 1e12}
    if issue is None:
        out.update(fp64)
        out["kernel"] = f"stack kernel, {form} form (FP64 pipe)"
        return out
    g = issue * computed / stack_s / 1e9
    out.update({"achieved": g, "peak": ISSUE_PEAK_G, "unit": "G warp-instructions issued/s",
                "frac": g / ISSUE_PEAK_G, "kernel": f"stack kernel, {form} form (instruction issue)",
                "peak_source": "unit counts: 1 warp instruction/clock x 4 schedulers x 152 SMs x 2.07 GHz",
                "warp_inst_per_sample": issue, "fp64_pipe": fp64})
    return out


def form_record(res):
    s = statistics.mean(res["step_ms"]) / 1e3
    q = res["quality"]
    return {"samples_per_s": res["samples"] / s, "ms_per_step": s * 1e3,
            "stack_ms": statistics.mean(res["stack_ms"]), "planes_ms": res["planes_ms"],
            "candidate_stage_ms": statistics.mean(res["cand_ms"]), "topk_ms": res["topk_ms"],
            "candidates_per_s": q["list"] / s, "candidates": q,
            "valid_fraction": res["valid"] / max(res["samples"], 1),
            "offchip_skipped_fraction": res["skipped"] / max(res["samples"], 1),
            "block_skipped_fraction": res["blocked"] / max(res["samples"], 1),
            "fp64_step_fraction": (res["samples"] - res["skipped"]) / max(res["samples"], 1),
            "pairs_rejected_per_s": res["skipped"] / s,
            "tiles": res["tiles"]}


def e2e_record(e2e, samples, world, max_over_ranks):
    return {"value": samples * world / max_over_ranks(e2e["s_per_step"]), "unit": UNIT,
            "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
            "ms_per_step": e2e["s_per_step"] * 1e3,
            "pipelined": "2 contexts: step i+1's host-to-device copies overlap step i's stack",
            "h2d_link_gbs_untimed": e2e["link_gbs"],
            "stack_ms_mean": e2e["stack_ms"], "stack_ms_max": e2e["stack_ms_max"],
            "candidate_list_equals_device": e2e["list_equals_device"]}


def form_dtype(form):
    """The arithmetic the form's path computes in (not a precision claim)."""
    state = ("df32 state (FP32 pairs; f64 for rare long steps)" if form.df else "f64 state")
    geom = "f64 light time and TAN" if form.geom64 else "df32 light time and TAN"
    return f"{state}; {geom}; {form.plane} planes; f32 sums"


def batched_subrecord(args, rank, device, barrier, world, max_over_ranks, rates):
    """The batched uneven workload (4,096 families x 16,384 orbits, 20-400 of
    400 exposures of 2048^2, BF16 planes) measured in the same run: both forms
    and the chosen form's e2e, fewer steps than the headline."""
    import copy
    import torch
    b = copy.copy(args)
    b.workload, b.size, b.no_vet = "batched", 2048, True
    b.steps, b.warmup = min(args.steps, 5), 3
    sky, stream, imgs, states = make_workload(b, rank, device)
    forms = {"chosen": Form("chosen", b.plane, "persistent", True, df=True),
             "plain": Form("plain", "f32", "plain", False)}
    out = {"workload": workload_name(b, sky, states), "steps": b.steps, "warmup": b.warmup}
    res = {}
    for name in ("chosen", "plain"):
        r, e = bench_form(b, forms[name], sky, stream, imgs, states, device, barrier, None)
        res[name] = r
        out[name] = form_record(r)
        if e is not None:
            out["e2e"] = e2e_record(e, r["samples"], world, max_over_ranks)
    r = res["chosen"]
    out["value"] = r["samples"] * world / max_over_ranks(statistics.mean(r["step_ms"]) / 1e3)
    out["unit"] = UNIT
    out["roofline"] = stack_roofline("batched", "chosen", b.plane, r, rates)
    del imgs, states
    torch.cuda.empty_cache()
    return out


def sparse_subrecord(args, rank, device, barrier, world, max_over_ranks, vet_params):
    """The sparse regime (20,000 exposures of 512^2 over a year, 1M orbits,
    each orbit on well under 1 % of the exposures) measured in the same run:
    the chosen form with and without the block cone test, and the plain
    form; fewer steps than the headline."""
    import copy
    import torch
    b = copy.copy(args)
    b.workload, b.no_vet = "sparse", vet_params is None
    b.steps, b.warmup, b.tiles = min(args.steps, 3), 3, "128,16"
    b.no_e2e, b.vet_batch = True, 0
    sky, stream, imgs, states = make_workload(b, rank, device)
    forms = [Form("chosen", b.plane, "persistent", True, block=True, df=True),
             Form("chosen_without_block_test", b.plane, "persistent", True, block=False, df=True),
             Form("plain", "f32", "plain", False)]
    n = states.shape[1]
    out = {"workload": (f"sparse survey: {sky.ex.n} exposures {int(sky.ex.width[0])}^2 over a year, "
                        f"{n} orbits ({sky.meta['n_fam']} families), {len(sky.inj_states)} injected, "
                        f"all orbits x all exposures"),
           "steps": b.steps, "warmup": b.warmup, "tiles": b.tiles}
    for f in forms:
        r, _ = bench_form(b, f, sky, stream, imgs, states, device, barrier,
                          vet_params if f.name == "chosen" else None)
        out[f.name] = form_record(r)
    out["shuffled_orbits"] = footprint_record(b, sky, imgs, states, device)
    r = out["chosen"]
    out["value"] = r["samples_per_s"] * world
    out["unit"] = UNIT
    del imgs, states
    torch.cuda.empty_cache()
    return out


def footprint_record(b, sky, imgs, states, device, steps=3):
    """The sparse survey's orbits in a random order (families interleaved,
    no family arrays), chosen form, with and without the footprint order
    (ndt_set_footprint_sort): the stack_orbits call's time with CUDA events
    on the context's stream (the ordering kernels included), the stack
    kernel's own time and what the off-chip and block tests skipped."""
    import torch
    from paper_2503_08854_gb300 import ndt
    n = states.shape[1]
    gen = torch.Generator()
    gen.manual_seed(17)
    shuffled = states[:, torch.randperm(n, generator=gen).to(states.device)].contiguous()
    stream = torch.cuda.Stream(device=device)
    ctx = ndt.create(device.index, stream)
    res = {"orbits": n, "order": "seeded random permutation of the survey's family-grouped orbits"}
    try:
        ndt.load_exposures(ctx, sky.ex, imgs, plane_dtype=b.plane)
        ot, et = (int(x) for x in b.tiles.split(","))
        ndt.set_launch(ctx, ndt.LAUNCH_PERSISTENT, ot, et, use_graph=True)
        for name, on in (("unordered", False), ("footprint_ordered", True)):
            ndt.set_footprint_sort(ctx, on)
            for _ in range(2):
                ndt.stack_orbits(ctx, shuffled, sky.t0, n)               # warm-up
            ms = []
            for _ in range(steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ndt.stack_orbits(ctx, shuffled, sky.t0, n)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            st = ndt.get_stats(ctx)
            t = statistics.mean(ms)
            res[name] = {"call_ms": t, "stack_kernel_ms": st["last_stack_ms"],
                         "stack_pairs_per_s": st["samples"] / (t / 1e3),
                         "offchip_skipped_fraction": st["offchip_skipped"] / max(st["samples"], 1),
                         "block_skipped_fraction": st["block_skipped"] / max(st["samples"], 1)}
    finally:
        ndt.destroy(ctx)
    return res


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    from paper_2503_08854_gb300 import __name__ as _pkg  # noqa: F401
    import __graft_entry__
    __graft_entry__.build()
    rates = fp64_rates(device)
    vet_params, vet_info = None, None
    if args.workload == "batched":
        args.no_vet = True      # no injected sources to vet in the batched workload
    if "chosen" in args.forms.split(",") and not args.no_vet:
        vet_params, vet_info = train_vetter(device, n_train_sky=args.vet_skies,
                                            n_test_sky=max(1, args.vet_skies // 4),
                                            train_stamps=args.vet_train_stamps)
    sky, stream, imgs, states = make_workload(args, rank, device)
    forms = {"plain": Form("plain", "f32", "plain", False),
             "plain_fp64": Form("plain_fp64", "f32", "plain", False, geom64=True),
             "chosen": Form("chosen", args.plane, "persistent", True, df=True),
             "chosen_fp64_state": Form("chosen_fp64_state", args.plane, "persistent", True)}
    results, e2e = {}, None
    clocks = ClockSampler(local)
    clocks.start()
    for name in args.forms.split(","):
        res, e = bench_form(args, forms[name], sky, stream, imgs, states, device, barrier,
                            vet_params)
        results[name] = res
        if e is not None:
            e2e = e
    head = "chosen" if "chosen" in results else list(results)[0]
    r = results[head]
    samples = r["samples"]
    step_s = max_over_ranks(statistics.mean(r["step_ms"]) / 1e3)
    value = samples * world / step_s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": form_dtype(forms[head]), "data": "synthetic",
        "config": {"workload": workload_name(args, sky, states),
                   "form": head, "planes": forms[head].plane,
                   "launch": forms[head].mode + ("+graph" if forms[head].graph else ""),
                   "tiles": r["tiles"], "l2": "inputs larger than L2 (planes >= 13 GB)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "valid_samples_per_s": r["valid"] * world / step_s,
        "candidates_per_s": r["quality"]["list"] * world / step_s,
        "candidates_def": (f"vetted list per step: orbits with nu >= {NU_MIN}, ranked, near-duplicates "
                           f"within {DEDUP_PX} px at {DEDUP_REFS} reference exposures dropped"
                           + (", CNN-scored and trimmed" if vet_params is not None else "")),
        "recall": r["quality"].get("recall"),
        "recall_def": r["quality"].get("recall_def"),
        "fpr_at_fixed_recall": r["quality"].get("fpr_at_fixed_recall"),
        "gpu_launches": int(r["launches"]),
    }
    if vet_info is not None:
        if r.get("vet_batch"):
            vet_info["batch"] = r["vet_batch"]
        line["vetting"] = vet_info
    for name, res in results.items():
        line[name] = form_record(res)
        line[name]["roofline"] = stack_roofline(args.workload, name, forms[name].plane, res, rates)
    line["roofline"] = line[head]["roofline"] or {"bound": "alu", "achieved": None, "peak": ISSUE_PEAK_G,
                                                  "unit": "G warp-instructions issued/s", "frac": None,
                                                  "traffic": None}
    if e2e is not None:
        line["e2e"] = e2e_record(e2e, samples, world, max_over_ranks)
    if rank == 0 and args.workload == "mba" and not args.no_noise:
        line["noise_estimate"] = noise_rate(device, stream, imgs)
    host = imgs.cpu().numpy() if rank == 0 and not args.no_cpu else None
    if args.workload == "mba" and not args.no_batched:
        del imgs, states
        torch.cuda.empty_cache()
        line["batched"] = batched_subrecord(args, rank, device, barrier, world, max_over_ranks,
                                            rates)
    if args.workload == "mba" and not args.no_sparse:
        torch.cuda.empty_cache()
        line["sparse"] = sparse_subrecord(args, rank, device, barrier, world, max_over_ranks, vet_params)
    line["clocks"] = clocks.stop()
    if host is not None:
        rate, cores, desc = cpu_oracle_rate(sky, host, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": desc}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
