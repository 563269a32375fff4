"""Benchmark: probe update + 1080p query on the procedural-city workload.

One step = one full pass of the hot path over one frame: per-frame ray
pattern, classification of uninitialised probes, active-probe compaction,
trace + shade of every active probe's rays, blend with border copy and state
advance, then the irradiance query of every pixel of a 1920x1080 G-buffer.

Workload: 32x16x32 probes (16,384) at 2 m over a seeded city of 16,384 box
buildings (196,610 triangles), 256 rays per probe, hysteresis 0.97, per-frame
random rotation, multi-bounce, probe state machine on; the G-buffer comes
from a seeded pinhole camera raycast into the same scene.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead (the CPU baseline arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "probe-update ms/frame & Grays/s at 16k probes; query ms at 1080p vs FP32 plain"
WORKLOAD = ("city 32x16x32 probes @ 2 m, 196,610 tris, 256 rays/probe, hysteresis 0.97, "
            "multi-bounce, state machine on, 1920x1080 G-buffer query")
# FP32 lane operations counted per unit of work of the trace passes: a
# child-box slab test is 25, a 4-wide node visit tests four boxes and orders
# them nearest first with 5 compare-exchanges of 5 operations (closest-hit
# and shadow rays alike); a watertight triangle test is 30.
OPS_PER_WIDE_NODE = 4 * 25 + 5 * 5
OPS_PER_TRI = 30
L2_FLUSH_BYTES = 256 << 20
TC_BLEND_DOC = {
    "tf32": "tcgen05 tensor cores: TF32 irradiance, FP32-accurate distance moments (B-side hi/lo split)",
    "bf16": "tcgen05 tensor cores: BF16 irradiance, FP32-accurate distance moments",
    "tf32x3": "tcgen05 tensor cores, FP32-accurate: weights and values split hi + lo in TF32, three products",
}
# DRAM bytes (read + write) of one k_trace_primary launch on this workload,
# from the ncu capture in profiles/trace_passes_city.md; set to None whenever
# the kernel changes until it is captured again
PRIMARY_TRAFFIC_BYTES = 7_106_560 + 3_401_728   # DRAM read + write of one k_trace_primary launch (ncu)
# The traversal's cache roofline: bytes one 4-wide node visit reads (the six
# slab planes and the child references, 7 of the node's 8 float4) and one
# triangle test reads (3 float4), against the L2 read rate measured in the
# same run over L2-resident buffers of these sizes
BYTES_PER_WIDE_NODE = 7 * 16
BYTES_PER_TRI = 3 * 16
L2_PROBE_BYTES = (16 << 20, 32 << 20)
# L2 bytes (lts__t_bytes) of one k_trace_primary launch on this workload,
# from the same ncu capture rules as PRIMARY_TRAFFIC_BYTES
PRIMARY_L2_BYTES = 420_674_752
# Warp instructions of one launch (smsp__inst_executed.sum, ncu) of the
# primary pass and of the 1080p query on this workload: their issue rate
# against the SMs' peak (four schedulers each issuing one warp instruction
# per clock) is the bound these issue-limited kernels meet first; set to
# None whenever the kernel changes until it is captured again
PRIMARY_WARP_INSTR = 109_074_897
QUERY_WARP_INSTR = 65_615_503


def workload_config(desc, n_pix):
    """The workload and timing protocol both arms report (identical in the
    GPU arm's line and the reference arm's)."""
    return {"workload": WORKLOAD, "probes": desc.n_probes, "rays_per_probe": desc.rays_per_probe,
            "query_pixels": n_pix, "l2": "flushed between timed steps (256 MiB write outside the events)"}


def l2_read_rate(g, torch, stream, passes=16, reps=5):
    """L2 read rate (GB/s): the largest over L2_PROBE_BYTES of bytes x passes
    / event time of ddgi_measure_l2_read, after one untimed call that makes
    the buffer resident."""
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    best = 0.0
    with torch.cuda.stream(stream):
        for nbytes in L2_PROBE_BYTES:
            buf = torch.randint(-(1 << 31), (1 << 31) - 1, (nbytes // 4,), dtype=torch.int32, device="cuda")
            g.measure_l2_read(buf, 2, sink, stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                g.measure_l2_read(buf, passes, sink, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            best = max(best, nbytes * passes * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9)
            del buf
    return best


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        self.window = None
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
            # the timed region starts only once the sampler is producing rows
            t0 = time.perf_counter()
            while self._rows() == 0 and time.perf_counter() - t0 < 10.0:
                time.sleep(0.05)
        except Exception:
            self.proc = None
        return self

    def _rows(self):
        try:
            with open(self.file.name) as f:
                return sum(1 for _ in f)
        except OSError:
            return 0

    def mark(self):
        """Row count now: call at the start and at the end of the timed region."""
        return self._rows()

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        if self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        where = "whole run"
        if self.window is not None:
            a, b = self.window
            inside = rows[a:b]
            # a timed region shorter than the sampling period: the first row after it
            rows, where = (inside, "timed region") if inside else (rows[b:b + 1], "first sample after the timed region")
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "window": where}


def make_workload():
    sc = synth.city_scene()
    return sc, synth.city_volume(), synth.city_lights(), synth.city_camera()


# ----------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload
# ----------------------------------------------------------------------------

def oracle_step_estimate(sc, desc, L, n_active, R, n_pixels, subset, n_query_sample, frame=5):
    """Time the oracle's update of the active probes in `subset` and its query
    of `n_query_sample` surface points; extrapolate to one full step."""
    import oracle
    h = oracle.SceneHandle(sc)
    st, irr, dist = oracle.new_state(desc)
    st[:] = oracle.VIGILANT       # steady-state frame: every sampled probe traces
    n_probe_sample = len(subset)
    t0 = time.perf_counter()
    oracle.update(h, L, desc, frame, st, irr, dist, subset=subset)
    t_upd = time.perf_counter() - t0
    pts, nrm = synth.surface_points(sc, n_query_sample, seed=3002)
    t0 = time.perf_counter()
    oracle.query(desc, st, irr, dist, pts, nrm, np.array([0.0, 12.0, -28.0]))
    t_q = time.perf_counter() - t0
    t_step = t_upd * (n_active / n_probe_sample) + t_q * (n_pixels / n_query_sample)
    return t_step, t_upd, t_q


def oracle_active_count(sc, desc, n_sample=128, seed=11):
    """The oracle's own estimate of the active-probe count: classify a random
    probe sample at frame 0 and scale the newly-vigilant fraction.  Returns the
    estimate and the sampled probes found active."""
    import oracle
    st = np.zeros(desc.n_probes, dtype=np.uint8)
    ids = np.sort(np.random.default_rng(seed).choice(desc.n_probes, n_sample, replace=False))
    oracle.classify(oracle.SceneHandle(sc), desc, 0, ids, st)
    act = ids[st[ids] == oracle.NEWLY_VIGILANT]
    return max(1, int(round(len(act) / n_sample * desc.n_probes))), act


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, timed on the host cores on a
    bounded sample per step, extrapolated to the same metric and unit."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sc, desc, L, cam = make_workload()
    n_active, act = oracle_active_count(sc, desc)
    R = desc.rays_per_probe
    n_pix = cam.width * cam.height
    n_qs = 4096
    n_ps = min(len(act), 16)
    times = []
    for k in range(args.warmup + args.steps):
        t_step, _, _ = oracle_step_estimate(sc, desc, L, n_active, R, n_pix, act[:n_ps], n_qs,
                                            frame=k)
        if k >= args.warmup:
            times.append(t_step)
    ms = 1e3 * float(np.mean(times))
    value = n_active * R / (ms * 1e-3) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Grays/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(desc, n_pix),
        "active_probes": n_active, "parallelism": "host cores (FP64 oracle)",
        "cpu_baseline": {"value": value, "unit": "Grays/s", "cores": cores(), "kind": "oracle",
                         "sample": f"{n_ps} active probes (one update) + {n_qs} query points per "
                                   f"step, extrapolated to {n_active} active probes (oracle's own "
                                   f"estimate from 128 classified probes) x {R} rays + {n_pix} pixels"},
        "e2e": {"value": value, "unit": "Grays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2009_10796_gb300 as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    sc, desc, L, cam = make_workload()
    scene = g.Scene.from_arrays(sc)
    vol = g.Volume(desc)
    pos, nrm = scene.raycast_gbuffer(cam.position, cam.forward, cam.up, cam.vfov_deg, cam.width,
                                     cam.height, device=dev)
    n_pix = pos.shape[0]
    out = torch.empty_like(pos)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    camera = cam.position

    # several GPUs (torchrun): the update is sharded by z-slabs of probes,
    # the updated slabs all-gathered into every GPU's own atlases (NCCL, one
    # collective per buffer, persistent buffers), the query sharded by pixels
    # over the replicated atlases; --replicas runs independent copies instead
    sharded = world > 1 and not args.replicas
    if sharded:
        from paper_2009_10796_gb300 import shard
        ranges = shard.slabs(desc.counts, world)
        slab = ranges[rank]
        info = vol.info
        nb = [info.irr_bytes // desc.n_probes, info.dist_bytes // desc.n_probes, 1]
        bufs = [torch.empty(info.irr_bytes, dtype=torch.uint8, device=dev),
                torch.empty(info.dist_bytes, dtype=torch.uint8, device=dev),
                torch.empty(desc.n_probes, dtype=torch.uint8, device=dev)]
        exchange = shard.SlabExchange(nb, ranges, rank, dev)
        cut = [4 * ((n_pix * r // world) // 4) for r in range(world)] + [n_pix]   # 16-byte aligned pixel shards
        pix = slice(cut[rank], cut[rank + 1])
    else:
        pix = slice(0, n_pix)
    pos_q, nrm_q, out_q = pos[pix], nrm[pix], out[pix]

    def update(frame, precision=g.BLEND_FP32):
        if not sharded:
            vol.update(scene, L, frame, precision=precision, stream=stream)
            return
        vol.update_range(scene, L, frame, slab[0], slab[1], precision=precision, stream=stream)
        for k, b in enumerate(bufs):
            vol.copy_buffer(k, b, stream=stream)
        exchange(bufs)
        for k, b in enumerate(bufs):
            vol.set_buffer(k, b, stream=stream)

    def step(frame):
        update(frame)
        vol.query(pos_q, nrm_q, camera, out_q, stream=stream)

    frame = 0
    for _ in range(args.warmup):
        step(frame)
        frame += 1
    torch.cuda.synchronize()
    vol.poll_status()
    states_now = vol.states()
    n_active = int((states_now == g.STATE_VIGILANT).sum().item())
    # this GPU's share (the slab it traces and blends, sharded; else all)
    lo_p, hi_p = slab if sharded else (0, desc.n_probes)
    n_active_local = int((states_now[lo_p:hi_p] == g.STATE_VIGILANT).sum().item())
    R = desc.rays_per_probe
    stats = vol.trace_stats(scene, L)

    def timed_steps(precision, stages):
        # device-timed steps; L2 flushed between steps outside the events.
        # stages=False: events at the step boundaries only (the headline
        # pass); stages=True: per-stage events inside the update and around
        # the query as well (they cost about 20 us per step, so the headline
        # pass runs without them)
        nonlocal frame
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        qev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        vol.read_timings()
        vol.enable_timing(stages)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            update(frame, precision)
            if stages:
                qev[k][0].record(stream)
            vol.query(pos_q, nrm_q, camera, out_q, stream=stream)
            if stages:
                qev[k][1].record(stream)
            evs[k][1].record(stream)
            frame += 1
        torch.cuda.synchronize()
        wall_s = time.perf_counter() - wall0
        if world > 1:
            dist.barrier()
        tm = vol.read_timings()
        vol.enable_timing(False)
        q = [a.elapsed_time(b) for a, b in qev] if stages else None
        return [a.elapsed_time(b) for a, b in evs], q, tm, wall_s

    with ClockSampler(local) as clk:
        m0 = clk.mark()
        step_ms, _, _, wall = timed_steps(g.BLEND_FP32, False)
        time.sleep(0.15)    # one sampling period, so a row taken during the region has landed
        clk.window = (m0, clk.mark())
        # the same steps again with per-stage events: stage times, the query's
        # time and the primary pass's launch duration for the roofline
        _, query_ms, timings, _ = timed_steps(g.BLEND_FP32, True)
        # the same step with the blend on tensor cores, per precision
        mixed = {}
        if not args.no_mixed:
            for name, prec in (("tf32", g.BLEND_TF32), ("bf16", g.BLEND_BF16), ("tf32x3", g.BLEND_TF32X3)):
                m_step, _, _, _ = timed_steps(prec, False)
                _, m_query, m_tm, _ = timed_steps(prec, True)
                mixed[name] = (m_step, m_query, m_tm)
    ms = float(np.mean(step_ms))
    t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    rays_per_step = n_active * R
    # rays of the whole job per step: N replicas each trace the volume; N
    # shards together trace it once
    job_rays = (1 if sharded else world) * rays_per_step
    value = job_rays / (ms_max * 1e-3) / 1e9

    # end to end through the C-ABI frame call with host buffers: pinned
    # G-buffer copied in (alongside the probe update), irradiance copied out
    # (chunked behind the query), every step
    pos_h = pos_q.cpu().pin_memory()
    nrm_h = nrm_q.cpu().pin_memory()
    out_h = torch.empty_like(pos_h).pin_memory()
    if not sharded:
        vol.frame_host(scene, L, frame, pos_h, nrm_h, camera, out_h, stream=stream)   # staging allocation
        frame += 1
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    eev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for k in range(args.steps):   # L2 flushed between steps outside the events
        flush.fill_(float(k))
        eev[k][0].record(stream)
        if sharded:   # the rank's pixel shard in from host memory, its irradiance back out
            pos_q.copy_(pos_h, non_blocking=True)
            nrm_q.copy_(nrm_h, non_blocking=True)
            step(frame)
            out_h.copy_(out_q, non_blocking=True)
        else:
            vol.frame_host(scene, L, frame, pos_h, nrm_h, camera, out_h, stream=stream)
        eev[k][1].record(stream)
        frame += 1
    torch.cuda.synchronize()
    e2e_ms = float(np.mean([a.elapsed_time(b) for a, b in eev]))
    t = torch.tensor([e2e_ms], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_value = job_rays / (float(t.item()) * 1e-3) / 1e9
    vol.poll_status()

    # roofline of the dominant kernel, the primary trace pass: its counted FP32
    # lane operations per launch / its event-timed duration on the update
    # stream; peak = lanes x max SM clock (one operation per lane per clock)
    pk, pk_kind = peaks()
    trace_ms, trace_n = timings["trace_shade"]
    trace_ms_avg = trace_ms / max(trace_n, 1)
    prim_ms = timings["trace_primary"][0] / max(timings["trace_primary"][1], 1)
    shadow_ms = timings["trace_shadow"][0] / max(timings["trace_shadow"][1], 1)
    prim_ops = OPS_PER_WIDE_NODE * stats["nodes"] + OPS_PER_TRI * stats["tris"]
    shadow_ops = OPS_PER_WIDE_NODE * stats["shadow_nodes"] + OPS_PER_TRI * stats["shadow_tris"]
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tops = sm_count * 128 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = prim_ops / (prim_ms * 1e-3) / 1e12
    shadow_achieved = shadow_ops / (shadow_ms * 1e-3) / 1e12
    prim_l2_bytes = BYTES_PER_WIDE_NODE * stats["nodes"] + BYTES_PER_TRI * stats["tris"]
    issue_peak = sm_count * 4 * pk.get("sm_max_mhz", 2070.0) * 1e6   # warp instructions per second

    def issue(instr, launch_ms):
        if not instr:
            return None
        rate = instr / (launch_ms * 1e-3)
        return {"bound": "issue", "achieved": rate / 1e12, "peak": issue_peak / 1e12,
                "unit": "T warp-instr/s", "frac": rate / issue_peak, "instructions_per_launch": instr}
    l2_peak = l2_read_rate(g, torch, stream)
    blend_ms = timings["blend"][0] / max(timings["blend"][1], 1)
    blend_bytes = n_active_local * (R * 16 + 2000 + 2816)      # records in, old interior in, tiles out
    blend_flop = 2 * n_active_local * R * (desc.irr_n ** 2 * 3 + desc.dist_n ** 2 * 2)
    q_ms = float(np.mean(query_ms))
    q_bytes = pos_q.shape[0] * 36                         # positions + normals in, irradiance out
    hbm = pk.get("hbm_gbs", 6800.0)

    # second-order glossy lookups (Sec. 4.4) at the G-buffer points, the camera
    # rays standing in for the reflection rays that reached them
    gdirs = pos - torch.tensor(np.asarray(camera, np.float32), device=dev)
    gdirs = gdirs / gdirs.norm(dim=1, keepdim=True).clamp_min(1e-12)
    gout = torch.empty_like(pos)
    for _ in range(args.warmup):
        vol.query_glossy(pos, nrm, gdirs, gout, stream=stream)
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        gev[k][0].record(stream)
        vol.query_glossy(pos, nrm, gdirs, gout, stream=stream)
        gev[k][1].record(stream)
    torch.cuda.synchronize()
    glossy_ms = float(np.mean([a.elapsed_time(b) for a, b in gev]))

    precision = None if args.no_mixed else run_precision(args, g, torch, stream, scene, L, sc, pos, nrm, camera,
                                                         flush)
    paper_res = None if args.no_paper_res else run_paper_resolution(args, g, torch, stream, scene, L, pos, nrm,
                                                                     camera, flush)
    optimizer = None if args.no_paper_res else run_optimizer(args, g, torch, stream, scene, L)
    dynamic = None
    if not args.no_paper_res:
        dynamic = run_dynamic(args, g, torch, stream, scene, L, pos, nrm, camera, flush)
        # the same with the optional converge pass: 4 batches of R rays for every probe woken
        dynamic["converge_pass"] = run_dynamic(args, g, torch, stream, scene, L, pos, nrm, camera, flush,
                                               converge=4)
    cascade = None if args.no_cascade else run_cascade(args, g, torch, stream)
    diff = None if args.no_diff else run_diff(args, g, torch, stream)

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        n_act_cpu, act = oracle_active_count(sc, desc)
        t_step, t_upd, t_q = oracle_step_estimate(sc, desc, L, n_act_cpu, R, n_pix, act, 16384)
        cpu = {"value": n_act_cpu * R / t_step / 1e9, "unit": "Grays/s", "cores": cores(),
               "kind": "oracle",
               "sample": f"{len(act)} active probes x {R} rays (one update, {t_upd:.1f} s) + 16384 "
                         f"query points "
                         f"({t_q:.2f} s), extrapolated to {n_act_cpu} active probes (oracle's own "
                         f"estimate) + {n_pix} pixels"}
    # steady-state frame: frame setup in two launches (directions and counter
    # clear on the update stream, texel weights on a side stream), 3 trace
    # passes, blend, query (the active list is kept and classification skipped
    # once no probe is uninitialised): 7 launches, as the ncu launch list shows
    launches_per_step = 7
    line = {
        "metric": METRIC, "value": value, "unit": "Grays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(desc, n_pix),
        "active_probes": n_active,
        "timing": "value: CUDA events at the step boundaries only; stage_ms, query and the "
                  "roofline launch times: a second pass of the same steps with per-stage "
                  "events on the update stream",
        "parallelism": ("sharded: z-slabs of probes, NCCL all-gather of the updated slabs, "
                        "pixel-sharded query" if sharded else ("replicas" if world > 1 else "single GPU")),
        "update_ms_per_frame": ms - q_ms, "query_ms_1080p": q_ms, "glossy_query_ms_1080p": glossy_ms,
        "trace_grays_per_s": n_active_local * R / (trace_ms_avg * 1e-3) / 1e9,
        "stage_ms": {k: v[0] / max(v[1], 1) for k, v in timings.items()},
        "wall_ms_per_step": 1e3 * wall / args.steps,
        "trace_work_per_ray": {"wide_nodes": stats["nodes"] / max(stats["rays"], 1),
                               "tris": stats["tris"] / max(stats["rays"], 1),
                               "shadow_rays": stats["shadow_rays"] / max(stats["rays"], 1),
                               "queries": stats["queries"] / max(stats["rays"], 1)},
        "roofline": {"bound": "alu", "kernel": "k_trace_primary", "achieved": achieved,
                     "peak": peak_tops, "unit": "TFLOP/s", "frac": achieved / peak_tops,
                     "traffic": PRIMARY_TRAFFIC_BYTES,
                     "peak_kind": f"FP32 lanes x max SM clock ({pk_kind} clock)",
                     "ops_per_launch": prim_ops, "launch_ms": prim_ms,
                     "l2": {"bound": "l2", "achieved": prim_l2_bytes / (prim_ms * 1e-3) / 1e9, "peak": l2_peak,
                            "unit": "GB/s", "frac": prim_l2_bytes / (prim_ms * 1e-3) / 1e9 / l2_peak,
                            "traffic": PRIMARY_L2_BYTES, "bytes_per_launch": prim_l2_bytes,
                            "traffic_frac": (PRIMARY_L2_BYTES / (prim_ms * 1e-3) / 1e9 / l2_peak
                                             if PRIMARY_L2_BYTES else None),
                            "peak_kind": "measured in this run: ddgi_measure_l2_read, L1-bypassing 16-byte "
                                         "loads over an L2-resident buffer",
                            "bytes_kind": "node visits x 112 B + triangle tests x 48 B (counting build); "
                                          "traffic: lts__t_bytes of one launch (ncu), most node bytes "
                                          "being L1 hits"},
                     "issue": issue(PRIMARY_WARP_INSTR, prim_ms)},
        "roofline_shadow": {"bound": "alu", "kernel": "k_trace_shadow", "achieved": shadow_achieved,
                            "peak": peak_tops, "unit": "TFLOP/s", "frac": shadow_achieved / peak_tops,
                            "launch_ms": shadow_ms},
        "roofline_blend": {"bound": "hbm", "achieved": blend_bytes / (blend_ms * 1e-3) / 1e9,
                           "peak": hbm, "unit": "GB/s",
                           "frac": blend_bytes / (blend_ms * 1e-3) / 1e9 / hbm,
                           # the FP32 multiply-adds of the contraction, R x (36 x 3 + 196 x 2) per
                           # probe, against 152 SMs x 128 lanes x 2 FLOP x the maximum SM clock
                           "fp32": {"achieved": blend_flop / (blend_ms * 1e-3) / 1e12, "peak": 2 * peak_tops,
                                    "unit": "TFLOP/s", "frac": blend_flop / (blend_ms * 1e-3) / 1e12 / (2 * peak_tops)}},
        "roofline_query": {"bound": "hbm", "achieved": q_bytes / (q_ms * 1e-3) / 1e9, "peak": hbm,
                           "unit": "GB/s", "frac": q_bytes / (q_ms * 1e-3) / 1e9 / hbm,
                           "issue": issue(QUERY_WARP_INSTR, q_ms)},
        "tensor_blend": {name: {
            "blend": TC_BLEND_DOC[name],
            "ms_per_step": float(np.mean(m[0])),
            "value": rays_per_step / (float(np.mean(m[0])) * 1e-3) / 1e9,
            "blend_ms": m[2]["blend"][0] / max(m[2]["blend"][1], 1),
            "blend_hbm_frac": blend_bytes / (m[2]["blend"][0] / max(m[2]["blend"][1], 1) * 1e-3) / 1e9 / hbm,
            "frame_setup_ms": m[2]["frame_setup"][0] / max(m[2]["frame_setup"][1], 1)}
            for name, m in mixed.items()},
        "precision_forms": precision,
        "paper_resolution": paper_res,
        "position_optimizer": optimizer,
        "dynamic_objects": dynamic,
        "cascade_batched": cascade,
        "differentiation": diff,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "Grays/s", "h2d_bytes_per_step": 2 * pos_q.shape[0] * 12,
                "d2h_bytes_per_step": pos_q.shape[0] * 12},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_cascade(args, g, torch, stream):
    """Batched cascades: 4 tracking volumes of 32^3 probes at 1/2/4/8 m over a
    1M-triangle terrain with buildings, 288 rays per probe, the camera moving
    0.6 m per frame; every frame is one captured launch sequence over all
    volumes (CUDA graph), launch shapes from the autotuner."""
    sc = synth.terrain_scene()
    L = synth.city_lights()
    descs = synth.terrain_cascades()
    scene = g.Scene.from_arrays(sc)
    C = g.Cascade(descs)
    cache = os.path.join(ROOT, "_build", "autotune.json")
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    from_cache = C.autotune(scene, L, 0, synth.terrain_camera_path(0), cache_path=cache)
    frame = 1
    for _ in range(args.warmup):
        C.update(scene, L, frame, synth.terrain_camera_path(frame), use_graph=True, stream=stream)
        frame += 1
    torch.cuda.synchronize()
    active = [int((C.states(k) == g.STATE_VIGILANT).sum().item()) for k in range(C.n)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        C.update(scene, L, frame, synth.terrain_camera_path(frame), use_graph=True, stream=stream)
        frame += 1
    e1.record(stream)
    torch.cuda.synchronize()
    C.poll_status()
    ms = e0.elapsed_time(e1) / args.steps
    rays = sum(active) * descs[0].rays_per_probe
    forms = run_cascade_forms(args, g, torch, stream, scene, L, descs, C.tuning())
    return {"workload": "terrain + buildings, 1,048,568 tris; 4 tracking cascades of 32^3 probes at 1/2/4/8 m; "
                        "288 rays/probe; camera 0.6 m/frame",
            "ms_per_frame": ms, "grays_per_s": rays / (ms * 1e-3) / 1e9, "active_probes": active,
            "graph": True, "tuning": {"trace_blocks_per_sm": C.tuning()[0], "blend_probes_per_cta": C.tuning()[1],
                                      "from_cache": from_cache},
            "forms": forms}


def _rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.maximum(np.abs(ref), 1e-3 * max(np.abs(ref).max(), 1e-30))
    return np.abs(got - ref) / scale


def _decoded_irr(g, V):
    """Stored irradiance texels as float64 [P, n+2, n+2, 3], any storage format."""
    a = V.irr_atlas().cpu().numpy()
    if V.desc.irr_format != g.IRR_RGB9E5:
        return a.astype(np.float64)
    w = a.astype(np.int64)
    sc = np.exp2((w >> 27) - 24.0)
    return np.stack([(w & 511) * sc, ((w >> 9) & 511) * sc, ((w >> 18) & 511) * sc], -1)


# precision configurations of the city step: irradiance and distance storage
# formats, blend arithmetic
PRECISION_FORMS = {
    "fp32": ("IRR_FP32", "DIST_FP32", "BLEND_FP32"),
    "fp16_atlases": ("IRR_FP16", "DIST_FP16", "BLEND_FP32"),
    "rgb9e5_irradiance": ("IRR_RGB9E5", "DIST_FP32", "BLEND_FP32"),
    "tf32_blend": ("IRR_FP32", "DIST_FP32", "BLEND_TF32"),
    "bf16_blend": ("IRR_FP32", "DIST_FP32", "BLEND_BF16"),
    "tf32x3_blend": ("IRR_FP32", "DIST_FP32", "BLEND_TF32X3"),
    "mixed_tf32_fp16": ("IRR_FP16", "DIST_FP32", "BLEND_TF32"),
    "mixed_bf16_rgb9e5": ("IRR_RGB9E5", "DIST_FP32", "BLEND_BF16"),
}


def run_precision(args, g, torch, stream, scene, L, sc, pos, nrm, camera, flush):
    """The city step (update + 1080p query) in each precision configuration:
    ms per step, blend and query times, the blend's HBM fraction (algorithmic
    bytes at the stored texel sizes), and the texel error against the FP64
    oracle at frame 0 (the oracle's one-step update of 12 seeded active
    probes; max relative error in the stored, gamma-encoded domain)."""
    import oracle
    desc = synth.city_volume()
    R = desc.rays_per_probe
    ref = g.Volume(desc)
    ref.update(scene, L, 0, stream=stream)
    torch.cuda.synchronize()
    act = np.nonzero(ref.states().cpu().numpy() == g.STATE_VIGILANT)[0]
    sample = np.sort(np.random.default_rng(77).choice(act, 12, replace=False))
    st, irr, dist = oracle.new_state(desc)
    oracle.update(oracle.SceneHandle(sc), L, desc, 0, st, irr, dist, subset=sample)
    pk, _ = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    ti, td = desc.irr_n ** 2, desc.dist_n ** 2
    tile_i, tile_d = (desc.irr_n + 2) ** 2, (desc.dist_n + 2) ** 2
    out = {}
    for name, (fi, fd, fb) in PRECISION_FORMS.items():
        prec = getattr(g, fb)
        V = g.Volume(desc, irr_format=getattr(g, fi), dist_format=getattr(g, fd))
        V.update(scene, L, 0, precision=prec, stream=stream)
        torch.cuda.synchronize()
        ei = float(_rel_err(_decoded_irr(g, V)[sample], irr[sample]).max())
        ed = float(_rel_err(V.dist_atlas().cpu().numpy()[sample], dist[sample]).max())
        res = torch.empty_like(pos)
        frame = 1
        for _ in range(args.warmup):
            V.update(scene, L, frame, precision=prec, stream=stream)
            V.query(pos, nrm, camera, res, stream=stream)
            frame += 1
        torch.cuda.synchronize()
        n_active = int((V.states() == g.STATE_VIGILANT).sum().item())
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        V.read_timings()
        V.enable_timing(True)
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            V.update(scene, L, frame, precision=prec, stream=stream)
            V.query(pos, nrm, camera, res, stream=stream)
            ev[k][1].record(stream)
            frame += 1
        torch.cuda.synchronize()
        tm = V.read_timings()
        V.enable_timing(False)
        V.poll_status()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        blend_ms = tm["blend"][0] / max(tm["blend"][1], 1)
        ib = {"IRR_FP32": 12, "IRR_FP16": 8, "IRR_RGB9E5": 4}[fi]    # algorithmic bytes per texel
        db = {"DIST_FP32": 8, "DIST_FP16": 4}[fd]
        blend_bytes = n_active * (R * 16 + ti * ib + td * db + tile_i * ib + tile_d * db)
        out[name] = {"irr_format": fi, "dist_format": fd, "blend": fb, "ms_per_step": ms,
                     "value": n_active * R / (ms * 1e-3) / 1e9, "blend_ms": blend_ms,
                     "blend_hbm_frac": blend_bytes / (blend_ms * 1e-3) / 1e9 / hbm,
                     "texel_max_rel_err_vs_oracle": {"irradiance": ei, "distance": ed},
                     "oracle_sample": "12 seeded active probes, frame 0, one-step FP64 update"}
    return out


def run_cascade_forms(args, g, torch, stream, scene, L, descs, tuning):
    """The batched cascade frame in other forms, for the batching and
    precision gains: TF32 and BF16 tensor-core blends (graph), the same
    launch sequence eager (no graph), and unbatched: each volume its own
    one-volume cascade with its own launch sequence (graph; hit shading then
    samples that volume only)."""
    out = {}

    def timed(cascades, precision, use_graph):
        frame = 1
        for _ in range(args.warmup):
            for C in cascades:
                C.update(scene, L, frame, synth.terrain_camera_path(frame), precision=precision, use_graph=use_graph,
                         stream=stream)
            frame += 1
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            for C in cascades:
                C.update(scene, L, frame, synth.terrain_camera_path(frame), precision=precision, use_graph=use_graph,
                         stream=stream)
            frame += 1
        e1.record(stream)
        torch.cuda.synchronize()
        for C in cascades:
            C.poll_status()
        active = sum(int((C.states(k) == g.STATE_VIGILANT).sum().item()) for C in cascades for k in range(C.n))
        ms = e0.elapsed_time(e1) / args.steps
        return {"ms_per_frame": ms, "grays_per_s": active * descs[0].rays_per_probe / (ms * 1e-3) / 1e9,
                "active_probes": active}

    for name, prec in (("tf32_blend", g.BLEND_TF32), ("bf16_blend", g.BLEND_BF16), ("tf32x3_blend", g.BLEND_TF32X3)):
        C = g.Cascade(descs)
        C.set_tuning(*tuning)
        out[name] = timed([C], prec, True)
    C = g.Cascade(descs)
    C.set_tuning(*tuning)
    out["fp32_eager"] = timed([C], g.BLEND_FP32, False)
    singles = []
    for d in descs:
        C1 = g.Cascade([d])
        C1.set_tuning(*tuning)
        singles.append(C1)
    out["fp32_unbatched"] = timed(singles, g.BLEND_FP32, True)
    return out


def run_paper_resolution(args, g, torch, stream, scene, L, pos, nrm, camera, flush):
    """The same city step with the paper's tile resolution: 8x8 irradiance and
    16x16 visibility interiors (Sec. 7.1), FP32 blend."""
    desc = synth.city_volume(irr_n=8, dist_n=16)
    vol = g.Volume(desc)
    out = torch.empty_like(pos)
    frame = 0
    for _ in range(args.warmup):
        vol.update(scene, L, frame, stream=stream)
        vol.query(pos, nrm, camera, out, stream=stream)
        frame += 1
    torch.cuda.synchronize()
    n_active = int((vol.states() == g.STATE_VIGILANT).sum().item())
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    vol.read_timings()
    vol.enable_timing(True)
    for k in range(args.steps):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        vol.update(scene, L, frame, stream=stream)
        vol.query(pos, nrm, camera, out, stream=stream)
        evs[k][1].record(stream)
        frame += 1
    torch.cuda.synchronize()
    tm = vol.read_timings()
    vol.enable_timing(False)
    vol.poll_status()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    return {"workload": "city, 8x8 irradiance / 16x16 visibility interiors, FP32 blend",
            "ms_per_step": ms, "grays_per_s": n_active * desc.rays_per_probe / (ms * 1e-3) / 1e9,
            "blend_ms": tm["blend"][0] / max(tm["blend"][1], 1), "active_probes": n_active}


def run_optimizer(args, g, torch, stream, scene, L):
    """Probe position optimizer (Sec. 5) on the city volume: the first frame
    (every probe new: 5 optimizer iterations, then classification) with and
    without it, and the probe states it leads to."""
    out = {}
    for iters in (0, 5):
        times = []
        for rep in range(3):
            vol = g.Volume(synth.city_volume(optimizer_iters=iters))
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            vol.update(scene, L, 0, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        st = vol.states().cpu().numpy()
        out[f"iters_{iters}"] = {"first_frame_ms": float(np.median(times)),
                                 "vigilant": int((st == g.STATE_VIGILANT).sum()),
                                 "off": int((st == g.STATE_OFF).sum()),
                                 "moved": int((vol.offsets().abs().sum(1) > 0).sum().item())}
    return out


def run_dynamic(args, g, torch, stream, scene, L, pos, nrm, camera, flush, converge=0):
    """Dynamic objects (Sec. 6.3) in the city: 32 vehicle-sized boxes (4 x 1.5 x
    2 m) flying straight lines over the streets at 5-30 m, where the sleeping
    probes are, waking those near them; the same step as the headline (update
    + 1080p query) with the boxes updated every frame.  converge: batches of
    the optional converge pass for the probes woken each frame."""
    desc = synth.city_volume(converge_batches=converge)
    vol = g.Volume(desc)
    out = torch.empty_like(pos)
    rng = np.random.default_rng(4004)
    lane = rng.integers(-7, 8, 32) * 4.0                 # street lines between the 4 m lots
    start = rng.uniform(-30.0, 30.0, 32)
    along_x = rng.integers(0, 2, 32).astype(bool)
    height = rng.uniform(5.0, 30.0, 32)

    def boxes(f):
        s = (start + 0.5 * f + 30.0) % 60.0 - 30.0
        c = np.stack([np.where(along_x, s, lane), height, np.where(along_x, lane, s)], 1)
        h = np.where(along_x[:, None], [2.0, 0.75, 1.0], [1.0, 0.75, 2.0])
        return np.concatenate([c - h, c + h], 1)

    frame = 0
    for _ in range(args.warmup):
        vol.set_dynamic_boxes(boxes(frame))
        vol.update(scene, L, frame, stream=stream)
        vol.query(pos, nrm, camera, out, stream=stream)
        frame += 1
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    awake = []
    for k in range(args.steps):
        vol.set_dynamic_boxes(boxes(frame))
        flush.fill_(float(k))
        evs[k][0].record(stream)
        vol.update(scene, L, frame, stream=stream)
        vol.query(pos, nrm, camera, out, stream=stream)
        evs[k][1].record(stream)
        frame += 1
    torch.cuda.synchronize()
    st = vol.states()
    n_awake = int((st == g.STATE_AWAKE).sum().item())
    n_active = int(((st == g.STATE_VIGILANT) | (st == g.STATE_AWAKE)).sum().item())
    vol.poll_status()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    return {"workload": "city + 32 vehicle-sized boxes flying at 5-30 m, waking sleeping probes", "ms_per_step": ms,
            "grays_per_s": n_active * desc.rays_per_probe / (ms * 1e-3) / 1e9, "awake_probes": n_awake,
            "active_probes": n_active, "converge_batches": converge}


def run_diff(args, g, torch, stream):
    """Differentiation: 16x8x16 probes (2,048, 128 rays) in a 192k-triangle
    interior with 64 emissive quads and 257 objects; two frames from a zero
    atlas (direct + one bounce, gamma 1) queried at 1M surface points; Adam
    (lr 0.02) on emitter radiance and albedo toward hidden seeded targets."""
    sc, truth_alb, truth_em = synth.interior_scene()
    L = synth.Lights()
    desc = synth.interior_volume()
    scene = g.Scene.from_arrays(sc)
    vol = g.Volume(desc)
    pts, nrm = synth.surface_points(sc, 1_000_000, seed=3005)
    P = torch.tensor(pts, dtype=torch.float32, device="cuda")
    N_ = torch.tensor(nrm, dtype=torch.float32, device="cuda")
    cam = np.array([0.0, 10.0, 0.0])
    ta = torch.tensor(truth_alb, dtype=torch.float32, device="cuda")
    te = torch.tensor(truth_em, dtype=torch.float32, device="cuda")
    with torch.no_grad():
        target = g.IrradianceField.apply(ta, te, vol, scene, L, P, N_, cam, 0, 2).clone()
    rng = synth.Rng(4005)
    emit0 = np.repeat(rng.uniform(len(truth_em), 0.1, 2.0)[:, None], 3, axis=1)
    # untimed warm-up steps on throwaway copies (first-use costs of the
    # autograd, optimizer and adjoint launches stay out of the timed loop)
    wa = torch.full_like(ta, 0.5).requires_grad_(True)
    we = torch.tensor(emit0, dtype=torch.float32, device="cuda").requires_grad_(True)
    wopt = torch.optim.Adam([wa, we], lr=0.02)
    for _ in range(args.warmup):
        wopt.zero_grad()
        ((g.IrradianceField.apply(wa, we, vol, scene, L, P, N_, cam, 0, 2) - target) ** 2).mean().backward()
        wopt.step()
    torch.cuda.synchronize()
    albedo = torch.full_like(ta, 0.5).requires_grad_(True)
    emit = torch.tensor(emit0, dtype=torch.float32, device="cuda").requires_grad_(True)
    opt = torch.optim.Adam([albedo, emit], lr=0.02)
    losses = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    steps = 200
    e0.record(stream)
    for _ in range(steps):
        opt.zero_grad()
        E = g.IrradianceField.apply(albedo, emit, vol, scene, L, P, N_, cam, 0, 2)
        loss = ((E - target) ** 2).mean()
        loss.backward()
        opt.step()
        losses.append(loss.detach())
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    losses = [float(x) for x in losses]
    return {"workload": "interior 192,140 tris, 257 objects, 64 emitters; 2,048 probes x 128 rays; 2 frames; "
                        "1M query points; Adam lr 0.02",
            "adam_steps": steps, "ms_per_step": ms, "loss_first": losses[0], "loss_last": losses[-1],
            "emitter_max_abs_err": float((emit.detach() - te).abs().max()),
            "emitter_mean_abs_err": float((emit.detach() - te).abs().mean())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--replicas", action="store_true",
                    help="several GPUs: independent replicas instead of the sharded update")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the tensor-core blend timings and the precision configurations")
    ap.add_argument("--no-cascade", action="store_true", help="skip the batched cascade workload")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiation workload")
    ap.add_argument("--no-paper-res", action="store_true",
                    help="skip the next-row lines (paper tile resolution, position optimizer, dynamic objects)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        # several GPUs: the headline step only (the other workloads are single-GPU measurements)
        args.no_mixed = args.no_cascade = args.no_diff = args.no_paper_res = True
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
