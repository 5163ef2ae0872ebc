"""Benchmark of the visual-sphere rasterizer on one GB300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl vsr|reference]

Workload: the single-view frame -- a 1920x1080 Universal-perspective map
(k=0.32, l=0.62, s=0.86, Omega=270 deg, horizontal AOV) of a level-5
icosphere of radius 50 around the eye (20,480 triangles) plus 200,000 seeded
random triangles (radius U[1, 40], edge ~0.02 rad); synthetic, seeded.

One step is the whole hot path over that frame: perspective map + tile cones
(a1), triangle set-up (a2), tile binning (a3), tile coverage / depth /
visibility and the front-to-back merge (a4 + a5), all inputs resident in
HBM.  a1 and a2 share no data: a1 runs on a second stream, concurrently with
a2, and a3 waits for both.  The metric is pixel x triangle tests/s: algorithmic tests (pixel
inside a triangle's enlarged miter cap, counted by the raster kernel) per
second of step time.  L2 is flushed (a 256 MB write) before every timed
step, outside its CUDA events.

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs its
own replica of the frame ("replicas only": the path has no exchange step)
and the value is the total over ranks divided by the slowest rank's time.
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
sys.path.insert(0, ROOT)

METRIC = "pixel x triangle tests/s"
WORKLOAD = "single-view 1920x1080, k=0.32 l=0.62 s=0.86 Omega=270, icosphere L5 + 200k triangles"
UNIT = "tests/s"
OPS_PER_TEST = 20  # FP32 ops of one algorithmic test: 4 three-term dots (12 FMA), 3 min, ramp FMA, 4 compares
LANES_PER_SM = 128  # FP32 lanes per Blackwell SM
# kernels of libvsr.so per step: map (the map stream), set-up, triangle
# filing, tile bins, work items, raster (the memsets between them are not
# kernels of the library)
LAUNCHES_PER_STEP = 6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="vsr", choices=["vsr", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=200000, help="pixels of the CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-frames", type=int, default=4, help="e2e: frames in flight ((map, scene) pairs used in turn)")
    ap.add_argument("--workload", default="single", choices=["single", "batched", "serving", "grad"],
                    help="single: the 1080p single-view frame (default); batched: 64 mixed views of a "
                         "1M-triangle scene, batched launch vs per-view plain launches")
    ap.add_argument("--views", type=int, default=64)
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: seconds of arrivals per lens stream")
    ap.add_argument("--slots", type=int, default=8, help="serving: requests in flight")
    ap.add_argument("--no-legs", action="store_true",
                    help="single workload: skip the dense, batched and serving legs of the JSON line")
    ap.add_argument("--leg-frames", type=int, default=50, help="batched leg: timed frames per arm")
    ap.add_argument("--leg-seconds", type=float, default=10.0, help="serving leg: seconds of arrivals")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload():
    from paper_2003_10558_gb300 import scenes
    lens, tris, cam = scenes.single_view_scene()
    return lens, tris, cam


RASTER_SOURCES = ("paper_2003_10558_gb300/csrc/raster.cu", "paper_2003_10558_gb300/csrc/stage.cuh",
                  "paper_2003_10558_gb300/csrc/df.cuh", "paper_2003_10558_gb300/csrc/vsr_internal.cuh")
RASTER_PROFILE = "raster_items_kernel_1080p_single_view.md"


def raster_traffic():
    """DRAM bytes per raster launch from the committed ncu summary, or None
    when the kernel's sources changed since that capture."""
    import hashlib
    import re
    try:
        with open(os.path.join(ROOT, "profiles", RASTER_PROFILE)) as f:
            txt = f.read()
        h = hashlib.sha256()
        for p in RASTER_SOURCES:
            with open(os.path.join(ROOT, p), "rb") as f:
                h.update(f.read())
        want = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", txt).group(1)
        if h.hexdigest()[:16] != want:
            return None
        return int(re.search(r"traffic_bytes_per_launch:\s*(\d+)", txt).group(1))
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.path = os.path.join(tempfile.gettempdir(), f"vsr_clocks_{os.getpid()}.csv")
        self.proc = None
        self.index = index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def load(self, step, seconds=0.5):
        """Keep the GPU under the workload's own load (untimed steps) long
        enough for several samples before the timed region starts."""
        import torch
        t_end = time.time() + seconds
        while time.time() < t_end:
            step()
            torch.cuda.synchronize()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as f:
                for line in f:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) < 9:
                        continue
                    try:
                        sm.append(float(p[1]))
                        smax.append(float(p[2]))
                    except ValueError:
                        continue
                    for n, v in zip(names, p[5:9]):
                        if v.lower() in ("active", "0x1", "1"):
                            reasons.add(n)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_frame(lens, tris, cam):
    """The oracle's map and set-up records of the frame (untimed)."""
    import oracle
    m64, _ = oracle.make_map(lens["W"], lens["H"], lens["k"], lens["l"], lens["s"], lens["omega"])
    return m64, oracle.setup(tris, cam)


def cpu_baseline(lens, tris, cam, n_pix, seed=123, frame=None):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    its raster stage (brute force over every triangle) on n_pix seeded pixels
    of the oracle's own map (frame: the map and records, made here if None).
    Returns (tests/s, seconds, n_alg, threads)."""
    import oracle
    m64, rec = frame if frame is not None else oracle_frame(lens, tris, cam)
    rng = np.random.default_rng(seed)
    pix = rng.integers(0, lens["W"] * lens["H"], n_pix)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    out = oracle.raster(m64, rec, pixels=pix, nthreads=threads)
    dt = time.perf_counter() - t0
    # extrapolate nothing: tests/s of the sampled pixels
    return out["n_alg"] / dt, dt, out["n_alg"], threads


def run_reference(args, rank, world):
    if rank != 0:
        return
    lens, tris, cam = workload()
    # each step: a bounded sample of the frame -- the samples of all K steps
    # together cpu_sample pixels, but at least 8192 a step, since each call
    # of the oracle's raster carries a fixed ~0.2 s -- so K + W steps end in
    # a few minutes
    n_pix = max(8192, args.cpu_sample // max(1, args.steps))
    frame = oracle_frame(lens, tris, cam)
    for _ in range(args.warmup):
        cpu_baseline(lens, tris, cam, 64, frame=frame)
    vals, tot_alg, tot_t = [], 0, 0.0
    threads = os.cpu_count() or 1
    for k in range(args.steps):
        v, dt, n_alg, threads = cpu_baseline(lens, tris, cam, n_pix, seed=1000 + k, frame=frame)
        vals.append(v)
        tot_alg += n_alg
        tot_t += dt
    value = tot_alg / tot_t
    sample = (f"{n_pix} seeded pixels per step of the 1920x1080 single-view frame; oracle raster stage, "
              f"brute force over all {len(tris)} triangles per pixel")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "W": lens["W"], "H": lens["H"],
                                            "T": int(len(tris))},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def run_vsr(args, rank, world, local):
    import torch
    import torch.distributed as dist
    from paper_2003_10558_gb300 import vsr as V
    from paper_2003_10558_gb300 import build as B
    from paper_2003_10558_gb300 import replicas

    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    B.build()
    V.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    lens, tris_np, cam = workload()
    W, H = lens["W"], lens["H"]
    T = int(len(tris_np))
    tris = torch.from_numpy(tris_np).to(dev)
    m = V.Map(W, H, lens["k"], lens["l"], lens["s"], lens["omega"])
    sc = V.Scene(tris, cam)
    out = {"id": torch.empty((H, W), dtype=torch.int32, device=dev),
           "depth": torch.empty((H, W), dtype=torch.float32, device=dev),
           "cov": torch.empty((H, W), dtype=torch.float32, device=dev)}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # the map kernel's stream gets the higher priority: the set-up fills the
    # SMs the map leaves idle
    side = torch.cuda.Stream(device=dev, priority=-1)
    ev_fork, ev_map = torch.cuda.Event(), torch.cuda.Event()

    def step(evs=None):
        # a1 on a second stream, concurrent with a2 (they share no data);
        # the fork also orders the map's rewrite after the previous raster
        ev_fork.record(stream)
        side.wait_event(ev_fork)
        m.update(W, H, lens["k"], lens["l"], lens["s"], lens["omega"], stream=side)  # a1
        ev_map.record(side)
        sc.update(tris, cam)  # a2
        stream.wait_event(ev_map)
        if evs:
            evs[0].record(stream)
        V.bin(m, sc)  # a3
        if evs:
            evs[1].record(stream)
        V.raster(m, sc, out=out, binned=True)  # a4 + a5
        if evs:
            evs[2].record(stream)

    # algorithmic units of one step (counted once, untimed)
    V.bin(m, sc)
    n_alg = V.raster(m, sc, stats=True)["n_alg"]  # counted with the cap test alone
    n_exec = V.raster(m, sc, stats="exec")["n_exec"]  # pixel x triangle pairs the timed kernel evaluates
    pairs = sc.bin_pairs()
    assert V.last_device_status() == 0

    for _ in range(max(3, args.warmup)):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    K = args.steps

    def evt():
        return torch.cuda.Event(enable_timing=True)

    ev0 = [evt() for _ in range(K)]
    stage = [[evt() for _ in range(3)] for _ in range(K)]
    with ClockSampler(local) as clk:
        clk.load(lambda: (flush.fill_(1.0), step()))
        torch.cuda.synchronize()
        for k in range(K):
            flush.fill_(float(k))
            ev0[k].record(stream)
            step(stage[k])
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    assert V.last_device_status() == 0
    step_ms = [a.elapsed_time(st_[2]) for a, st_ in zip(ev0, stage)]
    rast_ms = [st_[1].elapsed_time(st_[2]) for st_ in stage]
    stage_ms = {"map||setup": statistics.mean(a.elapsed_time(s[0]) for a, s in zip(ev0, stage)),
                "bin": statistics.mean(s[0].elapsed_time(s[1]) for s in stage),
                "raster": statistics.mean(rast_ms)}
    # the two overlapped stages alone (untimed diagnostics)
    for name, fn in (("map", lambda: m.update(W, H, lens["k"], lens["l"], lens["s"], lens["omega"])),
                     ("setup", lambda: sc.update(tris, cam))):
        a, b = evt(), evt()
        flush.fill_(0.0)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        stage_ms[name + " alone"] = a.elapsed_time(b)
    # the same frame with the map cached (a lens that does not change): set-up,
    # binning and raster only, L2 flushed before each step as above
    c0 = [evt() for _ in range(K)]
    c1 = [evt() for _ in range(K)]
    for k in range(K):
        flush.fill_(float(k))
        c0[k].record(stream)
        sc.update(tris, cam)
        V.bin(m, sc)
        V.raster(m, sc, out=out, binned=True)
        c1[k].record(stream)
    torch.cuda.synchronize()
    assert V.last_device_status() == 0
    cached_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(c0, c1))
    # the per-fragment pixel step on the same frame (binning for its wider
    # caps + raster), a quality variant: mean of K calls
    pm = V.Map.from_spec(V.MAP_UNIVERSAL, W, H, (lens["k"], lens["l"], lens["s"], lens["omega"]), derivatives=True)
    ps_sc = V.Scene(tris, cam)
    V.raster_pstep(pm, ps_sc, out=out)
    torch.cuda.synchronize()
    a, b = evt(), evt()
    a.record(stream)
    for _ in range(K):
        V.raster_pstep(pm, ps_sc, out=out)
    b.record(stream)
    torch.cuda.synchronize()
    assert V.last_device_status() == 0
    pstep_ms = a.elapsed_time(b) / K
    del pm, ps_sc
    # the same frame with the diagonal angle of view (Omega spans the image
    # diagonal): the whole step, L2 flushed before each, with its own N_alg
    dm = V.Map(W, H, lens["k"], lens["l"], lens["s"], lens["omega"], aov=V.AOV_DIAGONAL)
    dsc = V.Scene(tris, cam)  # bins sized for this map at its first binning
    V.bin(dm, dsc)
    n_alg_diag = V.raster(dm, dsc, stats=True)["n_alg"]
    diag_ms = []
    for k in range(K):
        flush.fill_(float(k))
        a, b = evt(), evt()
        a.record(stream)
        dm.update(W, H, lens["k"], lens["l"], lens["s"], lens["omega"], aov=V.AOV_DIAGONAL)
        dsc.update(tris, cam)
        V.bin(dm, dsc)
        V.raster(dm, dsc, out=out, binned=True)
        b.record(stream)
        diag_ms.append((a, b))
    torch.cuda.synchronize()
    assert V.last_device_status() == 0
    diag_ms = statistics.mean(a.elapsed_time(b) for a, b in diag_ms)
    del dm, dsc
    # the dense reference (no binning: every pixel against every triangle) on
    # the same frame, its outputs against the binned path's
    dense = None
    if not args.no_legs:
        V.bin(m, sc)
        ref = {k: v.clone() for k, v in V.raster(m, sc, binned=True).items()}
        dout = V.raster_dense(m, sc)
        torch.cuda.synchronize()
        same = all(torch.equal(ref[k], dout[k]) for k in ("id", "depth", "cov"))
        KD = 2
        a, b = evt(), evt()
        a.record(stream)
        for _ in range(KD):
            V.raster_dense(m, sc, out=dout)
        b.record(stream)
        torch.cuda.synchronize()
        assert V.last_device_status() == 0
        dense_ms = a.elapsed_time(b) / KD
        dense = {"kernel": "raster_dense_kernel", "ms": dense_ms, "launches": KD,
                 "pair_tests_per_frame": W * H * T,
                 "binned_bin_plus_raster_ms": stage_ms["bin"] + stage_ms["raster"],
                 "speedup_binned_vs_dense": dense_ms / (stage_ms["bin"] + stage_ms["raster"]),
                 "outputs_identical": bool(same)}
        del ref, dout
    # replicas: tests summed over ranks, time of the slowest rank
    total_units, tot_s = replicas.combine(n_alg * K, sum(step_ms) / 1000.0)
    ms_per_step = 1000.0 * tot_s / K
    value = total_units / tot_s

    # end to end through the C ABI with host buffers (pinned): every step
    # regenerates the map for the lens and renders from the host triangles
    # into host outputs; the transfers are inside the timed region
    e2e = None
    if not args.no_e2e:
        tris_pin = torch.from_numpy(tris_np).pin_memory()
        tris_host = tris_pin.numpy()

        def host_outputs():
            o = {"id": torch.empty((H, W), dtype=torch.int32).pin_memory().numpy().view(np.uint32),
                 "depth": torch.empty((H, W), dtype=torch.float32).pin_memory().numpy(),
                 "cov": torch.empty((H, W), dtype=torch.float32).pin_memory().numpy()}
            return o

        def timed_wall(step, n):
            for _ in range(max(3, args.warmup)):
                step()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(n):
                step()
            torch.cuda.synchronize()
            return time.perf_counter() - t0

        # one frame at a time: vsr_map_update + vsr_render_host (which waits)
        work, host_out = V.Scene(), host_outputs()

        def sync_step():
            m.update(W, H, lens["k"], lens["l"], lens["s"], lens["omega"])
            V.render_host(m, work, tris_host, cam, out=host_out)

        sync_units, sync_s = replicas.combine(n_alg * K, timed_wall(sync_step, K))
        # a stream of frames: F (map, scene, outputs) sets in turn, each on
        # a stream of its own, vsr_render_host_async + vsr_render_host_wait,
        # so one frame's raster and host transfers overlap the next one's map,
        # set-up and binning
        F = max(1, args.e2e_frames)
        pm = [m] + [V.Map(W, H, lens["k"], lens["l"], lens["s"], lens["omega"]) for _ in range(F - 1)]
        pw, po = [work] + [V.Scene() for _ in range(F - 1)], [host_out] + [host_outputs() for _ in range(F - 1)]
        ps = [torch.cuda.Stream(device=dev) for _ in range(F)]
        pend = [False] * F
        frame = [0]

        def wait_frame(i):
            if pend[i]:
                pend[i] = False
                if V.render_host_wait(pw[i]) != 0:  # outgrew its bins: render it again
                    V.render_host(pm[i], pw[i], tris_host, cam, out=po[i], stream=ps[i])

        def pipe_step():
            i = frame[0] % F
            frame[0] += 1
            wait_frame(i)
            pm[i].update(W, H, lens["k"], lens["l"], lens["s"], lens["omega"], stream=ps[i])
            V.render_host_async(pm[i], pw[i], tris_host, cam, out=po[i], stream=ps[i])
            pend[i] = True

        def pipe_run(n):
            for _ in range(n):
                pipe_step()
            for i in range(F):
                wait_frame(i)

        pipe_run(max(3, args.warmup))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pipe_run(K)
        torch.cuda.synchronize()
        e2e_units, e2e_s = replicas.combine(n_alg * K, time.perf_counter() - t0)
        same = all(np.array_equal(po[0][k].view(np.uint32), o[k].view(np.uint32)) for o in po[1:] for k in po[0])
        e2e = {"value": e2e_units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": T * 36,
               "d2h_bytes_per_step": W * H * 12, "ms_per_step": 1000.0 * e2e_s / K, "frames_in_flight": F,
               "api": "vsr_map_update + vsr_render_host_async / vsr_render_host_wait, pinned host buffers",
               "outputs_identical_across_pairs": bool(same),
               "one_frame_at_a_time": {"value": sync_units / sync_s, "ms_per_step": 1000.0 * sync_s / K,
                                       "api": "vsr_map_update + vsr_render_host"}}

    # the batched and serving workloads, short (single GPU only)
    batched = serving = None
    if not args.no_legs and world == 1:
        del flush
        torch.cuda.empty_cache()
        vb, tb, vp, tp, same_b, cfg, all_views = batched_leg(args, rank, world, dev, args.leg_frames)
        batched = {"value": vb / tb, "unit": "views/s", "plain_value": vp / tp,
                   "speedup_vs_plain": (vb / tb) / (vp / tp), "frames": args.leg_frames,
                   "ms_per_frame": 1000 * tb / args.leg_frames, "plain_ms_per_frame": 1000 * tp / args.leg_frames,
                   "outputs_identical": bool(same_b), "batch": cfg,
                   "workload": f"{len(all_views)} mixed views (512^2..2048x1024) of one 1M-triangle scene, "
                               "maps cached, CUDA-event timed"}
        res, server = serving_leg(args, dev, args.leg_seconds, streams=("pooled",))
        serving = dict(res["pooled"], server=server,
                       workload="Poisson arrivals at %g/s for %g s, lenses from a pool of 256, 4 resident scenes "
                                "(100k-1M triangles), views of the batched distribution, host clock"
                                % (args.rate, args.leg_seconds))
    if rank != 0:
        return
    pk, pk_kind = peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak_ops = props.multi_processor_count * LANES_PER_SM * sm_mhz * 1e6
    rast_mean_s = statistics.mean(rast_ms) / 1000.0
    achieved = n_alg * OPS_PER_TEST / rast_mean_s
    traffic = raster_traffic()
    # achieved HBM bandwidth of the memory-bound stages (algorithmic bytes /
    # their live CUDA-event times): the map with its tile cones and geometry
    # (16 B per pixel + 48 B per tile), the
    # set-up (36 B read + 160 B written per triangle) and the raster's own
    # streams (16 B map read + 12 B outputs written per pixel)
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    ntiles = ((W + 15) // 16) * ((H + 15) // 16)

    def bw(nbytes, ms):
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"bytes": int(nbytes), "ms": ms, "GB_per_s": gbs, "frac": gbs / hbm_peak}

    hbm = {"peak_GB_per_s": hbm_peak, "peak_source": f"{pk_kind} hbm_gbs",
           "map": bw(16 * W * H + 48 * ntiles, stage_ms["map alone"]),
           "setup": bw(196 * T, stage_ms["setup alone"]),
           "raster_map_read_and_outputs": bw(28 * W * H, statistics.mean(rast_ms))}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded scene generator)",
        "config": {"workload": WORKLOAD,
                   "W": W, "H": H, "T": T, "l2": "flushed before every step (256 MB write, outside the events)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "frames_per_s": world * K / tot_s,
        "step_ms_distribution": {"median": statistics.median(step_ms), "p10": float(np.percentile(step_ms, 10)),
                                 "p90": float(np.percentile(step_ms, 90)), "steps": len(step_ms)},
        "raster_kernel_ms": statistics.mean(rast_ms),
        "stage_ms": stage_ms,
        "n_alg_per_step": n_alg, "n_exec_per_step": n_exec, "bin_pairs_per_step": pairs,
        "map_cached": {"ms_per_step": cached_ms, "value": n_alg / (cached_ms / 1000.0), "unit": UNIT,
                       "frames_per_s": 1000.0 / cached_ms},
        "variants": {"pstep_bin_and_raster_ms": pstep_ms,
                     "diagonal_aov": {"ms_per_step": diag_ms, "value": n_alg_diag / (diag_ms / 1000.0), "unit": UNIT,
                                      "n_alg_per_step": n_alg_diag,
                                      "step": "map, set-up, binning, raster in sequence on one stream"}},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s (FP32)",
                     "frac": achieved / peak_ops, "traffic": traffic,
                     "kernel": "raster_items_kernel", "peak_source": f"{props.multi_processor_count} SMs x "
                     f"{LANES_PER_SM} FP32 lanes x {sm_mhz:.0f} MHz ({pk_kind} sm_max_mhz)"},
        "clocks": clk.summary(),
        "gpu_launches": LAUNCHES_PER_STEP * K,
        "hbm": hbm,
    }
    if dense is not None:
        line["dense"] = dense
    if batched is not None:
        line["batched"] = batched
    if serving is not None:
        line["serving"] = serving
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and world == 1:
        v, dt, na, thr = cpu_baseline(lens, tris_np, cam, args.cpu_sample)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
                                "sample": f"{args.cpu_sample} seeded pixels of the frame, oracle raster stage "
                                          f"(brute force over all {T} triangles), {dt:.1f} s"}
    print(json.dumps(line), flush=True)


def batched_leg(args, rank, world, dev, K):
    """The batched workload: 64 views of one 1M-triangle scene (sizes from
    {512^2, 1024^2, 2048x1024, 1920x1080}, k ~ U[-1,1], l, s ~ U[0.5,1],
    Omega ~ U[90,360], eye uniform in a radius-5 ball), maps cached.  Views/s
    of the batched path (one CUDA graph of per-view chains per frame) against
    per-view plain launches (set-up, binning, raster per view), each over K
    timed frames (CUDA events), with the outputs of the last frame compared
    bit for bit.  Returns (views_batched, s_batched, views_plain, s_plain,
    same, batch config, all views)."""
    import torch
    from paper_2003_10558_gb300 import vsr as V
    from paper_2003_10558_gb300 import scenes, replicas
    all_views = scenes.batched_views(args.views)
    # replicas: each rank renders its share of the views (pixel-balanced)
    views = [all_views[i] for i in replicas.shard_views([v["W"] * v["H"] for v in all_views], rank, world)]
    tris = torch.from_numpy(scenes.batched_scene()).to(dev)
    maps = [V.Map(v["W"], v["H"], v["k"], v["l"], v["s"], v["omega"]) for v in views]
    cams = np.stack([v["cam"] for v in views])

    def outs():
        return [{"id": torch.empty((v["H"], v["W"]), dtype=torch.int32, device=dev),
                 "depth": torch.empty((v["H"], v["W"]), dtype=torch.float32, device=dev),
                 "cov": torch.empty((v["H"], v["W"]), dtype=torch.float32, device=dev)} for v in views]

    ob, op = outs(), outs()
    batch = V.Batch()
    plain_scenes = [V.Scene() for _ in views]
    stream = torch.cuda.current_stream()

    def batched():
        batch.render(maps, tris, cams, ob)

    def plain():
        for v, m, sc, o in zip(views, maps, plain_scenes, op):
            sc.update(tris, v["cam"])
            V.raster(m, sc, out=o)

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0

    vb, tb = replicas.combine(len(views) * K, timed(batched))
    vp, tp = replicas.combine(len(views) * K, timed(plain))
    assert V.last_device_status() == 0
    same = all(torch.equal(a[k], b[k]) for a, b in zip(ob, op) for k in ("id", "depth", "cov"))
    cfg = batch.config()
    del ob, op, batch, plain_scenes, maps, tris
    torch.cuda.empty_cache()
    return vb, tb, vp, tp, same, cfg, all_views


def run_batched(args, rank, world, local):
    """64 views of one 1M-triangle scene, batched graph against per-view
    plain launches (see batched_leg); max(10, steps // 2) frames per arm."""
    import torch
    import torch.distributed as dist
    from paper_2003_10558_gb300 import vsr as V
    from paper_2003_10558_gb300 import build as B
    from paper_2003_10558_gb300 import scenes

    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    B.build()
    V.load()
    dev = torch.device("cuda", local)
    K = max(10, args.steps // 2)  # frames of ~0.1 s: about a second per arm
    vb, tb, vp, tp, same, cfg, all_views = batched_leg(args, rank, world, dev, K)
    if rank != 0:
        return
    npx = sum(v["W"] * v["H"] for v in all_views)
    line = {"metric": "views/s (batched multi-view frame)", "value": vb / tb, "unit": "views/s",
            "plain_value": vp / tp, "speedup_vs_plain": (vb / tb) / (vp / tp), "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_frame": 1000 * tb / K, "plain_ms_per_frame": 1000 * tp / K,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic (seeded scene generator)",
            "outputs_identical": bool(same), "batch": cfg,
            "scaling": "strong",
            "config": {"workload": f"{len(all_views)} mixed views (512^2..2048x1024), one 1M-triangle scene",
                       "views": len(all_views), "pixels": npx, "T": 1_000_000, "maps": "cached",
                       "parallelism": f"views sharded over {world} replicas" if world > 1 else "single GPU"}}
    print(json.dumps(line), flush=True)


def serving_leg(args, dev, duration, streams=("fresh", "pooled"), seed=3):
    """Poisson arrivals at args.rate over 4 resident scenes of {100k, 300k,
    600k, 1M} triangles (the batched workload's generator, seeds 30-33),
    views drawn from the batched workload's distribution, 40 GB budget.  Two
    lens streams: every request a fresh lens draw (map cache ~always misses),
    and lenses drawn from a pool of 256 (the cache hits).  Latency = result
    ready minus arrival (host clock); the client owns 96 output buffer sets
    and waits for a set's previous request before reusing it (that wait
    counts in the latency).  Returns {stream: stats} and the server's
    counters."""
    import torch
    from paper_2003_10558_gb300 import vsr as V
    from paper_2003_10558_gb300 import scenes
    sizes = [100_000, 300_000, 600_000, 1_000_000]
    srv = V.Server(budget_bytes=40 << 30, slots=args.slots)
    scene_t = [torch.from_numpy(scenes.random_triangles(n, 1.0, 60.0, 0.0096, 30 + i)).to(dev)
               for i, n in enumerate(sizes)]
    sids = [srv.add_scene(t) for t in scene_t]
    Wm, Hm = 2048, 1080
    nbuf = 96
    bufs = [{"id": torch.empty(Wm * Hm, dtype=torch.int32, device=dev),
             "depth": torch.empty(Wm * Hm, dtype=torch.float32, device=dev),
             "cov": torch.empty(Wm * Hm, dtype=torch.float32, device=dev)} for _ in range(nbuf)]
    rng = np.random.default_rng(seed)

    def draw_lens(r):
        W, H = scenes.VIEW_SIZES[r.integers(len(scenes.VIEW_SIZES))]
        return dict(W=int(W), H=int(H), k=float(r.uniform(-1, 1)), l=float(r.uniform(0.5, 1)),
                    s=float(r.uniform(0.5, 1)), omega=float(r.uniform(90, 360)))

    pool = [draw_lens(rng) for _ in range(256)]

    def run_stream(pooled):
        n = int(args.rate * duration)
        arrivals = np.cumsum(rng.exponential(1.0 / args.rate, n))
        pending = [None] * nbuf
        done = []
        t0 = V.Server.now() + 0.05
        for i in range(n):
            lens = pool[rng.integers(len(pool))] if pooled else draw_lens(rng)
            d = rng.normal(size=3)
            cam = scenes.camera(5.0 * rng.uniform() ** (1 / 3) * d / np.linalg.norm(d))
            b = i % nbuf
            if pending[b] is not None:
                done.append((pending[b][1], srv.wait(pending[b][0])))
            arr = t0 + arrivals[i]
            while V.Server.now() < arr:
                pass
            npx = lens["W"] * lens["H"]
            out = {k: bufs[b][k][:npx] for k in ("id", "depth", "cov")}
            pending[b] = (srv.submit(sids[int(rng.integers(4))], lens, cam, out), arr)
        for p in pending:
            if p is not None:
                done.append((p[1], srv.wait(p[0])))
        lat = np.array([r["t_done"] - arr for arr, r in done])
        ok = all(r["status"] == 0 for _, r in done)
        span = max(r["t_done"] for _, r in done) - t0
        hits = np.mean([r["map_cache_hit"] for _, r in done])
        # latency over the first and the last tenth of the arrivals: a queue
        # that grows without bound shows as a rising p50
        tenth = max(1, len(lat) // 10)
        return {"requests": n, "all_ok": ok, "frames_per_s": n / span, "p50_ms": 1000 * float(np.percentile(lat, 50)),
                "p99_ms": 1000 * float(np.percentile(lat, 99)),
                "p50_first_tenth_ms": 1000 * float(np.percentile(lat[:tenth], 50)),
                "p50_last_tenth_ms": 1000 * float(np.percentile(lat[-tenth:], 50)),
                "map_hit_rate": float(hits), "offered_rate": args.rate, "seconds": span}

    out = {}
    for name in streams:
        out[name] = run_stream(name == "pooled")
    st = srv.stats()
    srv.close()
    del bufs, scene_t
    torch.cuda.empty_cache()
    return out, {"slots": args.slots, "budget_bytes": 40 << 30, "reruns": st["reruns"],
                 "map_evictions": st["map_evictions"], "bytes_in_use": st["bytes_in_use"]}


def run_serving(args, rank, world, local):
    """The serving workload (see serving_leg): both lens streams, each
    args.duration seconds of arrivals."""
    import torch
    from paper_2003_10558_gb300 import vsr as V
    from paper_2003_10558_gb300 import build as B

    torch.cuda.set_device(local)
    B.build()
    V.load()
    dev = torch.device("cuda", local)
    res, server = serving_leg(args, dev, args.duration, seed=3 + 17 * rank)
    if rank != 0:
        return
    line = {"metric": "serving frames/s and p50/p99 latency", "value": res["pooled"]["frames_per_s"],
            "unit": "frames/s", "higher_is_better": True, "n_gpus": world, "dtype": "f32",
            "data": "synthetic (seeded scene generator)", "pooled_lenses": res["pooled"],
            "fresh_lenses": res["fresh"], "server": server,
            "config": {"workload": "Poisson arrivals, 4 resident scenes (100k-1M triangles), mixed views",
                       "rate": args.rate, "duration_s": args.duration, "scenes": [100_000, 300_000, 600_000,
                                                                                  1_000_000]}}
    print(json.dumps(line), flush=True)


def run_grad(args, rank, world, local):
    """The differentiation workload: 1024x1024 map at the fit's start lens
    (k=0.6, l=1, s=1, Omega=180), 10,000 seeded triangles with vertex noise,
    per-triangle colours.  One step is one forward and backward of the shaded
    image: map (a1) and set-up (a2) for the current lens and vertices, binning
    (a3), fragment lists with the sorted front-to-back merge (a4 + a5), then
    the adjoint to vertices, colours and (k, l, s, Omega) with a fixed
    upstream dL/dI.  Reports differentiable frames/s and the stage times."""
    import torch
    import torch.distributed as dist
    from paper_2003_10558_gb300 import vsr as V
    from paper_2003_10558_gb300 import build as B
    from paper_2003_10558_gb300 import scenes, replicas

    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    B.build()
    V.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    target, start, tris_t, noisy, colors, W, H = scenes.grad_scene()
    tris = torch.from_numpy(noisy).to(dev)
    col = torch.from_numpy(colors).to(dev)
    r = V.ShadedRenderer(W, H)
    up = torch.from_numpy(np.random.default_rng(5).normal(size=(H, W)).astype(np.float32)).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    T = tris.shape[0]

    def step(evs=None):
        r.set_lens(start["k"], start["l"], start["s"], start["omega"])
        r.scene.update(tris, r.cam)
        if evs:
            evs[0].record(stream)
        out = V.raster_shaded(r.map, r.scene, r.frags, col)
        if evs:
            evs[1].record(stream)
        V.raster_backward(r.map, r.scene, r.frags, tris, col, out["id"], dimage=up)
        if evs:
            evs[2].record(stream)

    for _ in range(max(3, args.warmup)):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    assert V.last_device_status() == 0
    K = args.steps
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    stage = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    with ClockSampler(local) as clk:
        clk.load(lambda: (flush.fill_(1.0), step()))
        torch.cuda.synchronize()
        for k in range(K):
            flush.fill_(float(k))
            ev0[k].record(stream)
            step(stage[k])
        torch.cuda.synchronize()
    assert V.last_device_status() == 0
    step_ms = [a.elapsed_time(s_[2]) for a, s_ in zip(ev0, stage)]
    frames, tot_s = replicas.combine(K, sum(step_ms) / 1000.0)
    if rank != 0:
        return
    line = {"metric": "differentiable frames/s (forward + backward)", "value": frames / tot_s, "unit": "frames/s",
            "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": 1000.0 * tot_s / K * world,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded scene generator)",
            "stage_ms": {"map+setup": statistics.mean(a.elapsed_time(s_[0]) for a, s_ in zip(ev0, stage)),
                         "forward": statistics.mean(s_[0].elapsed_time(s_[1]) for s_ in stage),
                         "backward": statistics.mean(s_[1].elapsed_time(s_[2]) for s_ in stage)},
            "config": {"workload": "differentiation 1024x1024, k=0.6 l=1 s=1 Omega=180, 10k triangles",
                       "W": W, "H": H, "T": int(T), "l2": "flushed before every step (256 MB write, outside the events)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.workload == "serving":
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the serving workload has no CPU arm; "
                                  "the oracle is timed on the single-view workload"}))
            return
        run_serving(args, rank, world, local)
        return
    if args.workload == "grad":
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the differentiation workload has no CPU arm; "
                                  "the oracle is timed on the single-view workload"}))
            return
        run_grad(args, rank, world, local)
        return
    if args.workload == "batched":
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no CPU arm; "
                                  "the oracle is timed on the single-view workload"}))
            return
        run_batched(args, rank, world, local)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_vsr(args, rank, world, local)


if __name__ == "__main__":
    main()
