"""Benchmark of the SNeRG deferred volume render on one node.

Default (no flags): N=1. Workload of the headline number: the 1024^3 grid (32^3
macroblocks, ~5% occupied, thin shells on seeded closed surfaces) rendered as one
800x800 view at 39 degrees FOV (the paper's Synthetic 360 set-up, App. B). A step is one
forward render of that view (ray generation, block-skipping march, density probe,
trilinear fetch, compositing, early exit, per-pixel MLP, store). The same JSON line also
carries the batched multi-camera render (64 cameras of mixed resolutions in one
persistent graph launch, vs one launch per camera) and the forward+backward of 65,536
rays on the 512^3 grid, each timed the same way.

Timing: CUDA events on the launching stream around each step, L2 flushed (256 MiB
write) before every timed step, W untimed warm-up steps, barrier + synchronize around
the timed region, max over ranks. Under torchrun (N>1) each rank renders its own seeded
view of the same grid (weak scaling, no data-path collective).

--impl reference: the FP64 CPU oracle timed on this machine's host cores on the same
workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s & 800² frames/s, batched vs plain; fwd+bwd Mrays/s; % HBM roofline"
CSRC = os.path.join(ROOT, "paper_2103_14645_gb300", "csrc")

# the sources each profiled kernel is compiled from (march core + its launcher)
FWD_SOURCES = ("snerg_internal.cuh", "snerg_fwd.cu")
BWD_SOURCES = ("snerg_internal.cuh", "snerg_bwd.cu")


def kernel_source_digest(sources=FWD_SOURCES) -> str:
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(profile: str, sources=FWD_SOURCES):
    """DRAM bytes per launch from the committed ncu summary profiles/<profile>.md, if it
    was taken on the current kernel sources (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", profile + ".md")) as f:
            txt = f.read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_digest") != kernel_source_digest(sources):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def march_bytes(cnt, rays):
    """Algorithmic bytes of a forward march (per launch): 4 B per indirection entry read,
    1 B per lattice sample in an occupied block (the density probe), 64 B per composited
    sample (8 corners x 8 channels), 12 B of output colour per ray. cnt = column sums of
    the debug counts (steps, composited, indirection reads)."""
    return 4.0 * cnt[2] + 1.0 * cnt[0] + 64.0 * cnt[1] + 12.0 * rays


# adjoint per composited sample: the stencil again (64 B) and two 16-byte vector atomics
# per corner into the gradient atlas, each a read and a write at the L2 (8 x 2 x 32 B)
ADJ_BYTES_PER_SAMPLE = 64 + 8 * 2 * 32
MLP_GRAD_BYTES_PER_CTA = 883 * 4 * 2      # one atomic per parameter per CTA (read + write)


def roofline(alg_bytes, ms, kernel, profile=None, sources=FWD_SOURCES, launches=1):
    """The roofline object of one timed launch (or `launches` launches per step): counted
    algorithmic bytes over the mean CUDA-event time, against the measured HBM copy peak.
    profile: the ncu summary (or a list of (summary, sources), one per launch of the step)
    whose DRAM bytes give `traffic`."""
    peaks, src = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    traffic = None
    if isinstance(profile, list):
        parts = [profiled_traffic(p, s) for p, s in profile]
        traffic = None if any(t is None for t in parts) else sum(parts)
    elif profile:
        traffic = profiled_traffic(profile, sources)
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "peak_source": f"{src} hbm_gbs", "kernel": kernel, "launches_per_step": launches,
            ("algorithmic_bytes_per_launch" if launches == 1 else "algorithmic_bytes_per_step"): int(alg_bytes)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_cameras(sc, rank: int):
    """Weak scaling: rank 0 renders the workload's own view, every other rank its own
    seeded 800x800 view of the same grid (rays are independent; no data is exchanged)."""
    from paper_2103_14645_gb300 import synth
    if rank == 0:
        return sc.cameras
    return synth.orbit_cameras(np.random.default_rng(9000 + rank), [(800, 800)], synth.CAM_RADIUS)


def reduce_max(value: float, device) -> float:
    """Max over ranks of a per-rank time (identity without a process group)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mrays(world_size: int, rays_per_rank: int, t_max_ms: float) -> float:
    """Aggregate throughput: all ranks' rays over the slowest rank's step time."""
    return world_size * rays_per_rank / (t_max_ms * 1e-3) / 1e6


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# -------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# -------------------------------------------------------------------------------------
def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    from paper_2103_14645_gb300 import synth
    # rank 0 runs alone (the other ranks have returned): every host core this process may
    # use, whatever thread count a launcher set for per-rank work
    oracle.set_threads(len(os.sched_getaffinity(0)))
    sc = synth.make_scene("shell1024")
    pix_all = synth.all_pixels(sc.cameras)
    # a bounded sample per step: a seeded quarter of the view's rays
    rng = np.random.default_rng(0)
    n = pix_all.shape[0] // 4
    samples = [pix_all[rng.choice(pix_all.shape[0], n, replace=False)] for _ in range(4)]
    oracle.render_rays(sc, samples[0][:1000])
    for i in range(args.warmup):
        oracle.render_rays(sc, samples[i % 4])
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.render_rays(sc, samples[i % 4])
    dt = time.perf_counter() - t0
    v = n * args.steps / dt / 1e6
    cores = oracle.threads()
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "Mrays/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "shell1024: 1024^3 grid, 32^3 blocks, one 800x800 view (seeded quarter of its "
                                   "rays per step)", "impl": "FP64 C oracle, OpenMP", "scene_checksum": sc.checksum()},
            "cpu_baseline": {"value": round(v, 4), "unit": "Mrays/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} seeded rays of the 800x800 view per step"},
            "e2e": {"value": round(v, 4), "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------------------------
# our arm
# -------------------------------------------------------------------------------------
def time_steps(fn, steps, warmup, stream, flush, counter=None):
    """Per-step CUDA-event times (ms) of `fn` after `warmup` untimed calls, with the L2
    flushed before each timed step; with `counter`, also the kernel launches counted
    during the timed steps."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    c0 = counter() if counter else 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        flush()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    if counter:
        return ms, counter() - c0
    return ms


def run_ours(args, ws, rank, local):
    import torch
    from paper_2103_14645_gb300 import renderer, synth
    dist = ws > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def flush():
        flush_buf.fill_(1)

    def barrier():
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()

    sc = synth.make_scene("shell1024")
    cams = rank_cameras(sc, rank)
    r = renderer.Renderer.from_scene(sc, dev)
    # serving: the view-dependence weights are fixed, stored once in the handle and passed
    # to the kernels as parameters (mlp=None below)
    r.set_mlp(sc.mlp)
    mlp = None
    out = torch.empty((800 * 800, 3), dtype=torch.float32, device=dev)
    n_rays = 800 * 800

    # counted algorithmic bytes of one launch (untimed debug render)
    dbg = r.render(cams, mlp, counts=True)
    r.check_status()
    cnt = dbg["counts"].double().sum(0).cpu().numpy()
    alg_bytes = march_bytes(cnt, n_rays)
    del dbg

    sampler = ClockSampler(local)
    sampler.start()
    # the view is rendered both ways -- one plain launch, and the persistent kernel in its
    # captured graph (autotuned during the warm-up) -- and the faster one is the headline
    modes = {}
    for mode in ("plain", "persistent"):
        pers = mode == "persistent"
        barrier()
        ms_m, n_launch = time_steps(lambda: r.render(cams, mlp, out=out, persistent=pers), args.steps, args.warmup,
                                    stream, flush, counter=lambda: r.launches)
        barrier()
        modes[mode] = (float(np.mean(ms_m)), n_launch)
    best = min(modes, key=lambda m: reduce_max(modes[m][0], dev))
    t_step, launches = modes[best]
    t_max = reduce_max(t_step, dev)
    value = whole_job_mrays(ws, n_rays, t_max)

    # side figure (not the headline): the viewer's tile schedule on this view -- each step's
    # tiles ordered by the costs recorded on the step before, which renders the same view
    r.render(cams, mlp, out=out, schedule=True)
    ms_sched = time_steps(lambda: r.render(cams, mlp, out=out, schedule=True), args.steps, args.warmup, stream, flush)

    # end to end through the public API with host buffers: camera record in, image out
    host_out = torch.empty((n_rays, 3), dtype=torch.float32, pin_memory=True)

    def e2e_step():
        # the kernels store the pixels straight into the pinned host buffer through the
        # device's mapping of it (NVLink-C2C); the step ends when they are all there
        r.render_to_host(cams, host_out, mlp)

    barrier()
    ms_e2e = time_steps(e2e_step, args.steps, args.warmup, stream, flush)
    barrier()
    e2e = whole_job_mrays(ws, n_rays, reduce_max(float(np.mean(ms_e2e)), dev))

    extra = {}
    if not args.no_extra:
        extra = extra_sections(args, r, sc, dev, stream, flush, barrier)
        # the non-deferred comparison model on the same view (the paper's per-sample
        # ablation): the view-dependence MLP at every composited sample
        from paper_2103_14645_gb300 import synth as _synth
        ps_scene = _synth.custom_scene(sc.N, sc.B, sc.ind, sc.atlas, sc.sigma_max, sc.mlp, sc.cameras,
                                       flags=renderer.FLAG_PER_SAMPLE_MLP)
        rps = renderer.Renderer.from_scene(ps_scene, dev)
        rps.set_mlp(sc.mlp)
        ms_ps = time_steps(lambda: rps.render(cams, None, out=out), max(3, min(args.steps, 10)), 2, stream, flush)
        extra["per_sample_mlp"] = {"ms_per_frame": round(float(np.mean(ms_ps)), 4),
                                   "mrays_s": round(n_rays / (np.mean(ms_ps) * 1e-3) / 1e6, 3),
                                   "slowdown_vs_deferred": round(float(np.mean(ms_ps)) / t_step, 3)}
        del rps
        # and without the view-dependence network (the paper's other performance ablation)
        nm_scene = _synth.custom_scene(sc.N, sc.B, sc.ind, sc.atlas, sc.sigma_max, sc.mlp, sc.cameras,
                                       flags=renderer.FLAG_NO_MLP)
        rnm = renderer.Renderer.from_scene(nm_scene, dev)
        rnm.set_mlp(sc.mlp)
        ms_nm = time_steps(lambda: rnm.render(cams, None, out=out), max(3, min(args.steps, 10)), 2, stream, flush)
        extra["no_mlp"] = {"ms_per_frame": round(float(np.mean(ms_nm)), 4),
                           "mrays_s": round(n_rays / (np.mean(ms_nm) * 1e-3) / 1e6, 3),
                           "deferred_over_no_mlp": round(t_step / float(np.mean(ms_nm)), 3)}
        del rnm
    clocks = sampler.stop()

    if rank != 0:
        if dist:
            tdist.destroy_process_group()
        return
    kname = "render_persistent_kernel" if best == "persistent" else "render_image_kernel"
    rl = roofline(alg_bytes, t_step, kname,
                  profile="render_persistent_shell1024" if best == "persistent" else "render_image_shell1024")
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Mrays/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"shell1024: {sc.N}^3 grid, {sc.B}^3 blocks, {sc.occupancy * 100:.1f}% occupied "
                               f"({sc.nb} blocks), one 800x800 view, 39 deg FOV",
                   "scene_checksum": sc.checksum(),
                   "l2": "flushed before every timed step (256 MiB write)",
                   "launch": "persistent kernel, CUDA-graph replay" if best == "persistent" else "plain (one launch per view)"},
        "launch_modes_ms": {m: round(v[0], 4) for m, v in modes.items()},
        "viewer_schedule": {"ms_per_frame": round(float(np.mean(ms_sched)), 4),
                            "mrays_s": round(n_rays / (float(np.mean(ms_sched)) * 1e-3) / 1e6, 3),
                            "note": "tiles ordered by the costs of the previous render, which is the same view; "
                                    "not the headline (see orbit.scheduled_* for consecutive different views)"},
        "frames_per_s": round(1e3 / t_max, 2),
        "roofline": rl,
        "e2e": {"value": round(e2e, 3), "unit": "Mrays/s", "h2d_bytes_per_step": 80 * len(cams),
                "d2h_bytes_per_step": n_rays * 12},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    line.update(extra)
    if ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(sc)
    print(json.dumps(line), flush=True)
    if dist:
        tdist.destroy_process_group()


def extra_sections(args, r, sc, dev, stream, flush, barrier):
    import torch
    from paper_2103_14645_gb300 import renderer, synth
    out = {}
    # batched: 64 cameras of mixed resolutions on the same grid
    bsc = synth.make_scene("batch1024")
    cams = bsc.cameras
    n_pix = bsc.n_pixels
    r.set_mlp(bsc.mlp)
    mlp = None
    reps = max(3, min(args.steps, 10))
    # counted algorithmic bytes of the batch (untimed debug render of the 64 cameras)
    dbg = r.render(cams, mlp, counts=True)
    cnt_b = dbg["counts"].double().sum(0).cpu().numpy()
    del dbg
    buf = torch.empty((n_pix, 3), dtype=torch.float32, device=dev)
    barrier()
    ms_b = time_steps(lambda: r.render(cams, mlp, out=buf, persistent=True), reps, 2, stream, flush)
    ms_p = time_steps(lambda: r.render(cams, mlp, out=buf), reps, 2, stream, flush)
    barrier()
    tw, th, c = r.persistent_config()
    # end to end: the same persistent launch storing the 64 images straight into pinned
    # host memory (487 MB per batch through the device's mapping)
    host = torch.empty((n_pix, 3), dtype=torch.float32, pin_memory=True)
    ms_h = time_steps(lambda: r.render(cams, mlp, out=host, persistent=True), reps, 2, stream, flush)
    del host
    out["batched"] = {"cameras": int(len(cams)), "rays": n_pix, "scene_checksum": bsc.checksum(),
                      "persistent_to_host_mrays_s": round(n_pix / (np.mean(ms_h) * 1e-3) / 1e6, 3),
                      "persistent_mrays_s": round(n_pix / (np.mean(ms_b) * 1e-3) / 1e6, 3),
                      "plain_mrays_s": round(n_pix / (np.mean(ms_p) * 1e-3) / 1e6, 3),
                      "ratio": round(float(np.mean(ms_p) / np.mean(ms_b)), 4),
                      "tile": [tw, th], "ctas_per_sm": c,
                      "ms_persistent": round(float(np.mean(ms_b)), 3), "ms_plain": round(float(np.mean(ms_p)), 3),
                      "roofline": roofline(march_bytes(cnt_b, n_pix), float(np.mean(ms_b)), "render_persistent_kernel",
                                           profile="render_persistent_batch1024"),
                      "roofline_plain": roofline(march_bytes(cnt_b, n_pix), float(np.mean(ms_p)), "render_image_kernel",
                                                 launches=int(len(cams)))}
    del buf
    # forward + backward of 65,536 rays on the 512^3 grid
    wsc = synth.make_scene("bwd512")
    rb = renderer.Renderer.from_scene(wsc, dev)
    pix = torch.from_numpy(wsc.extra["pix"]).to(dev)
    tgt = torch.from_numpy(wsc.extra["target"]).to(dev)
    wm = torch.from_numpy(wsc.mlp).to(dev)
    ga = torch.zeros(wsc.atlas.shape, dtype=torch.float32, device=dev)
    gm = torch.zeros(883, dtype=torch.float32, device=dev)
    c = torch.empty((pix.shape[0], 3), dtype=torch.float32, device=dev)

    def fwd():
        rb.render_rays(wsc.cameras, pix, wm, out=c)

    def fwd_bwd():
        # a training step: the forward keeps its per-ray state for the backward's single march
        f = rb.render_rays(wsc.cameras, pix, wm, out=c, aux=True, counts=True)
        rb.backward(wsc.cameras, pix, wm, c - tgt, ga, gm, fwd_aux=f["aux"], fwd_counts=f["counts"])

    loss = torch.zeros(1, dtype=torch.float32, device=dev)

    def fused():
        # render, L2 loss and adjoint of every ray in one launch (snerg_train_rays)
        rb.train_rays(wsc.cameras, pix, wm, tgt, ga, gm, loss=loss, out=c)

    ms_f = time_steps(fwd, reps, 2, stream, flush)
    ms_fb = time_steps(fwd_bwd, reps, 2, stream, flush)
    ms_tr = time_steps(fused, reps, 2, stream, flush)
    n = pix.shape[0]
    cnt = rb.render_rays(wsc.cameras, pix, wm, counts=True)["counts"].double().sum(0).cpu().numpy()
    rl_fb, rl_tr = training_rooflines(cnt, n, float(np.mean(ms_fb)), float(np.mean(ms_tr)), "bwd512")
    out["fwd_bwd"] = {"workload": f"bwd512: {wsc.N}^3 grid, {wsc.occupancy * 100:.1f}% occupied, {n} rays over 8 views",
                      "scene_checksum": wsc.checksum(),
                      "fwd_mrays_s": round(n / (np.mean(ms_f) * 1e-3) / 1e6, 3),
                      "fwd_bwd_mrays_s": round(n / (np.mean(ms_fb) * 1e-3) / 1e6, 3),
                      "fused_train_mrays_s": round(n / (np.mean(ms_tr) * 1e-3) / 1e6, 3),
                      "ms_fwd": round(float(np.mean(ms_f)), 4), "ms_fwd_bwd": round(float(np.mean(ms_fb)), 4),
                      "ms_fused_train": round(float(np.mean(ms_tr)), 4),
                      "roofline_fwd": roofline(march_bytes(cnt, n) + 12 * n, float(np.mean(ms_f)), "render_rays_kernel",
                                               profile="render_rays_bwd512"),
                      "roofline": rl_fb, "roofline_fused_train": rl_tr}
    # fine-tuning steps (Sec. 5.5): render -> L2 loss -> adjoint -> Adam, all in the library
    ft = renderer.FineTuner(rb, wsc.mlp)
    ms_ft = time_steps(lambda: ft.step(wsc.cameras, pix, tgt), reps, 2, stream, flush)
    out["finetune"] = {"ms_per_step": round(float(np.mean(ms_ft)), 4),
                       "mrays_s": round(n / (np.mean(ms_ft) * 1e-3) / 1e6, 3),
                       "steps_per_s": round(1e3 / float(np.mean(ms_ft)), 1)}
    # the same steps also fine-tuning the baked colours/features through an FP32 shadow
    # atlas, requantised into the scene's codes after every step
    rs = renderer.Renderer.from_scene(wsc, dev)
    fta = renderer.FineTuner(rs, wsc.mlp, atlas=wsc.atlas, atlas_lr=1.0 / 255.0)
    ms_fa = time_steps(lambda: fta.step(wsc.cameras, pix, tgt), reps, 2, stream, flush)
    out["finetune"]["shadow_atlas_ms_per_step"] = round(float(np.mean(ms_fa)), 4)
    out["finetune"]["shadow_atlas_values"] = int(fta.shadow.numel())
    del rs, fta
    del rb, ga, gm
    out["create"] = create_section(sc, dev)
    out["bake"] = bake_section(args, dev, stream, flush)
    out["orbit"] = orbit_section(args, r, sc, dev, stream, flush)
    if not args.no_large:
        out["large"] = large_section(args, dev, stream, flush)
    return out


def training_rooflines(cnt, n, ms_fb, ms_tr, tag):
    """Rooflines of a training step over n listed rays (cnt: column sums of the forward's
    debug counts). Two-launch form: the ray-list forward (march, 12 B pixel record in, 12 B
    colour and 48 B per-ray state out) and the adjoint (pixel, dL/dC and the state in; per
    composited sample the stencil again and the vector atomics into the gradient atlas; one
    atomic per MLP parameter per CTA). One-launch form (snerg_train_rays): the march, pixel
    and target in, colour out, and the same adjoint traffic. The adjoint's own march through
    block entries and density probes is not counted (a lower bound)."""
    ctas = -(-n // 128)
    adj = ADJ_BYTES_PER_SAMPLE * cnt[1] + MLP_GRAD_BYTES_PER_CTA * ctas
    two = (march_bytes(cnt, n) + 12 * n + 48 * n) + (72 * n + adj)
    one = march_bytes(cnt, n) + 24 * n + adj
    return (roofline(two, ms_fb, "render_rays_kernel + backward_rays_kernel<0, 1>",
                     profile=[(f"render_rays_{tag}", FWD_SOURCES), (f"backward_rays_{tag}", BWD_SOURCES)],
                     launches=2),
            roofline(one, ms_tr, "backward_rays_kernel<1, 0> (snerg_train_rays)", profile=f"train_rays_{tag}",
                     sources=BWD_SOURCES))


def orbit_section(args, r, sc, dev, stream, flush):
    """The paper's timing protocol (App. B): the average frame time of a 150-frame camera
    animation orbiting the scene, 800x800 at 39 deg FOV, here on the 1024^3 grid (one
    plain launch per frame, L2 flushed before every frame); also with the viewer's tile
    schedule (each frame's tiles launched in the order of the previous frame's tile costs),
    and the whole animation as one persistent launch."""
    import math
    import torch
    from paper_2103_14645_gb300 import synth
    r.set_mlp(sc.mlp)
    out = torch.empty((800 * 800, 3), dtype=torch.float32, device=dev)
    el = math.radians(20.0)
    cams = []
    for i in range(150):
        az = 2.0 * math.pi * i / 150
        pos = synth.CAM_RADIUS * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        cams.append(synth.look_at_camera(pos, (0.0, 0.0, 0.0), 800, 800, 39.0))
    for c in cams[:3]:
        r.render(np.asarray([c]), None, out=out)
    torch.cuda.synchronize()
    ms = []
    for c in cams:
        one = np.asarray([c])
        flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r.render(one, None, out=out)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    ms = np.asarray(ms)
    # a viewer playing the animation: each frame's tiles launched in the order of the tile
    # costs recorded on the previous frame (snerg_render_opts.schedule); the first frame
    # of the run (the one before the timed frames) in raster order
    r.render(np.asarray([cams[-1]]), None, out=out, schedule=True)
    ms_s = []
    for c in cams:
        one = np.asarray([c])
        flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r.render(one, None, out=out, schedule=True)
        b.record(stream)
        torch.cuda.synchronize()
        ms_s.append(a.elapsed_time(b))
    ms_s = np.asarray(ms_s)
    # the whole animation as one persistent batched launch (throughput, e.g. a video export),
    # delivered straight into pinned host memory
    seq = np.stack(cams).copy()
    seq["out_offset"] = np.arange(150, dtype=np.int64) * 800 * 800
    host = torch.empty((150 * 800 * 800, 3), dtype=torch.float32, pin_memory=True)
    ms_b = time_steps(lambda: r.render(seq, None, out=host, persistent=True), 3, 2, stream, flush)
    del host
    t_b = float(np.mean(ms_b))
    return {"frames": 150, "batched_ms_per_frame": round(t_b / 150, 4),
            "batched_frames_per_s": round(150 * 1e3 / t_b, 1),
            "ms_per_frame_mean": round(float(ms.mean()), 4),
            "ms_per_frame_min": round(float(ms.min()), 4), "ms_per_frame_max": round(float(ms.max()), 4),
            "frames_per_s": round(1e3 / float(ms.mean()), 1),
            "mrays_s": round(800 * 800 / (float(ms.mean()) * 1e-3) / 1e6, 3),
            "scheduled_ms_per_frame_mean": round(float(ms_s.mean()), 4),
            "scheduled_frames_per_s": round(1e3 / float(ms_s.mean()), 1),
            "scheduled_mrays_s": round(800 * 800 / (float(ms_s.mean()) * 1e-3) / 1e6, 3),
            "paper_webgl_ms_per_frame": 11.9}


def create_section(sc, dev):
    """snerg_create on device-resident inputs: validation, the per-octant distance maps and
    the padded atlas (the set-up between a bake and the first frame)."""
    import torch
    from paper_2103_14645_gb300 import renderer
    ind = torch.from_numpy(np.ascontiguousarray(sc.ind, np.int32)).to(dev)
    atl = torch.from_numpy(np.ascontiguousarray(sc.atlas, np.uint8)).to(dev)
    ms = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rr = renderer.Renderer(sc.N, sc.B, sc.bmin, sc.extent, sc.sigma_max, sc.bg, ind, atl)
        torch.cuda.synchronize()
        ms.append((time.perf_counter() - t0) * 1e3)
        rr.close()
        del rr
    return {"workload": f"{sc.name}: {sc.N}^3 grid, {sc.nb} blocks of {sc.B}^3", "ms": round(min(ms), 3)}


def bake_section(args, dev, stream, flush):
    """GPU bake (Sec. 5.3-5.4) of a 64-blob analytic field on the 1024^3 grid of 32^3
    blocks: alpha at every voxel centre, tau_alpha culling, packing, 16-sample anti-aliased
    8-bit content of every kept voxel. One call = the whole bake (it synchronises)."""
    import torch
    from paper_2103_14645_gb300 import renderer, synth
    N, B = 1024, 32
    f = synth.analytic_field(1)
    field = renderer.bake_field(f["blobs"], f["colors"], f["jitter"])
    ind, atl = renderer.bake(N, B, synth.WORLD_BMIN, synth.WORLD_EXTENT, 200.0, field, dev)
    nb = int(atl.shape[0])
    reps = max(3, min(args.steps, 5))
    ms = time_steps(lambda: renderer.bake(N, B, synth.WORLD_BMIN, synth.WORLD_EXTENT, 200.0, field, dev,
                                          max_blocks=nb), reps, 2, stream, flush)
    t = float(np.mean(ms))
    kept_vox = nb * B ** 3
    del ind, atl
    return {"workload": f"1024^3 grid, 32^3 blocks, 64 Gaussian blobs on a sphere; {nb} blocks kept "
                        f"({nb / (N // B) ** 3 * 100:.1f}%)",
            "ms": round(t, 3), "dense_gvox_s": round(N ** 3 / (t * 1e-3) / 1e9, 2),
            "kept_gsamples_s": round(16 * kept_vox / (t * 1e-3) / 1e9, 2),
            "atlas_gb_s": round(kept_vox * 8 / (t * 1e-3) / 1e9, 1)}


def large_section(args, dev, stream, flush):
    """2048^3 grid: 8 views at 1920x1080 in one persistent launch, then forward and
    forward+backward over 262,144 seeded rays."""
    import torch
    from paper_2103_14645_gb300 import renderer, synth
    sc = synth.make_scene("shell2048")
    r = renderer.Renderer.from_scene(sc, dev)
    r.set_mlp(sc.mlp)
    mlp = torch.from_numpy(sc.mlp).to(dev)
    n_pix = sc.n_pixels
    buf = torch.empty((n_pix, 3), dtype=torch.float32, device=dev)
    reps = max(3, min(args.steps, 10))
    dbg = r.render(sc.cameras, None, counts=True)
    alg = march_bytes(dbg["counts"].double().sum(0).cpu().numpy(), n_pix)
    del dbg
    ms_b = time_steps(lambda: r.render(sc.cameras, None, out=buf, persistent=True), reps, 2, stream, flush)
    del buf
    pix = torch.from_numpy(sc.extra["pix"]).to(dev)
    tgt = torch.from_numpy(sc.extra["target"]).to(dev)
    n = pix.shape[0]
    ga = torch.zeros(sc.atlas.shape, dtype=torch.float32, device=dev)
    gm = torch.zeros(883, dtype=torch.float32, device=dev)
    c = torch.empty((n, 3), dtype=torch.float32, device=dev)

    def fwd():
        r.render_rays(sc.cameras, pix, mlp, out=c)

    def fwd_bwd():
        f = r.render_rays(sc.cameras, pix, mlp, out=c, aux=True, counts=True)
        r.backward(sc.cameras, pix, mlp, c - tgt, ga, gm, fwd_aux=f["aux"], fwd_counts=f["counts"])

    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    ms_f = time_steps(fwd, reps, 2, stream, flush)
    ms_fb = time_steps(fwd_bwd, reps, 2, stream, flush)
    ms_tr = time_steps(lambda: r.train_rays(sc.cameras, pix, mlp, tgt, ga, gm, loss=loss, out=c), reps, 2, stream,
                       flush)
    r.check_status()
    cnt_r = r.render_rays(sc.cameras, pix, mlp, counts=True)["counts"].double().sum(0).cpu().numpy()
    rl_fb, rl_tr = training_rooflines(cnt_r, n, float(np.mean(ms_fb)), float(np.mean(ms_tr)), "shell2048")
    t_b = float(np.mean(ms_b))
    return {"workload": f"shell2048: {sc.N}^3 grid, {sc.B}^3 blocks, {sc.occupancy * 100:.1f}% occupied "
                        f"({sc.nb} blocks), 8 views at 1920x1080 + {n} backward rays",
            "scene_checksum": sc.checksum(),
            "batched_fwd_mrays_s": round(n_pix / (t_b * 1e-3) / 1e6, 3),
            "batched_fwd_ms": round(t_b, 3),
            "batched_fwd_roofline": roofline(alg, t_b, "render_persistent_kernel", profile="render_persistent_shell2048"),
            "rays_fwd_mrays_s": round(n / (np.mean(ms_f) * 1e-3) / 1e6, 3),
            "rays_fwd_bwd_mrays_s": round(n / (np.mean(ms_fb) * 1e-3) / 1e6, 3),
            "rays_fused_train_mrays_s": round(n / (np.mean(ms_tr) * 1e-3) / 1e6, 3),
            "rays_fwd_roofline": roofline(march_bytes(cnt_r, n) + 12 * n, float(np.mean(ms_f)), "render_rays_kernel",
                                          profile="render_rays_shell2048"),
            "rays_fwd_bwd_roofline": rl_fb, "rays_fused_train_roofline": rl_tr}


def cpu_baseline(sc):
    import oracle
    from paper_2103_14645_gb300 import synth
    pix = synth.all_pixels(sc.cameras)
    oracle.render_rays(sc, pix[:1000])
    threads = oracle.threads()
    t0 = time.perf_counter()
    oracle.render_rays(sc, pix)
    dt = time.perf_counter() - t0
    # one thread on every 16th ray of the view
    oracle.set_threads(1)
    sub = pix[::16]
    t1 = time.perf_counter()
    oracle.render_rays(sc, sub)
    dt1 = time.perf_counter() - t1
    oracle.set_threads(threads)
    return {"value": round(pix.shape[0] / dt / 1e6, 4), "unit": "Mrays/s", "cores": threads,
            "kind": "oracle", "sample": "the full 800x800 view once (640,000 rays), FP64 C oracle with OpenMP",
            "single_core_value": round(sub.shape[0] / dt1 / 1e6, 4),
            "single_core_sample": f"every 16th ray of the view ({sub.shape[0]} rays), one thread"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true", help="headline workload only")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-large", action="store_true", help="skip the 2048^3 section")
    ap.add_argument("--only", choices=["large"], default=None,
                    help="run one extra section alone and print its JSON (for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    ws, rank, local = dist_setup()
    if args.only == "large":
        import torch
        dev = torch.device("cuda", local)
        torch.cuda.set_device(dev)
        stream = torch.cuda.current_stream(dev)
        flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        print(json.dumps({"large": large_section(args, dev, stream, lambda: flush_buf.fill_(1))}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
