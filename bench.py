"""Benchmark: compressed-VDB path tracing on one GB300 (or N replicas).

Workload (the headline): the full-scale cloud, a seeded 1987 x 1351 x 2449
float32 volume (26.3 GB; Worley-modulated 8-octave fBm with an anvil height
profile, ~73 % exactly 0; it stands in for the paper's WDAS cloud, whose
dimensions it has), encoded at 1:10 into the VDB grid, path traced at
1920 x 1080 x 64 spp with delta tracking, albedo 0.95, Henyey-Greenstein
g = 0.8, up to 32 bounces, one directional light plus a constant environment;
the same renderer on the dense volume in a 3D CUDA texture is the comparator.

A step is one pass of the whole hot path over the input already in HBM:
encode (histogram/background, brick ranges, scores, selection, tree build,
prune, macrocell ranges) + render (majorants, DDA, Woodcock tracking,
ratio-tracked light, scattering, accumulation).  `value` is Mpaths/s of those
steps, timed with CUDA events on the launching stream (the 26.3 GB input is
far larger than L2 and every step re-reads it).  `e2e` runs the same step
through the C ABI with host buffers: the volume is copied from pinned host
memory inside vdbc_encode and the image is read back to the host inside
vdbc_render.  Errors are stated for every image: PSNR against the lossless
render and against the dense texture (FP64 reductions on the device,
vdbc_compare), and the mean / largest absolute difference from the FP64 CPU
oracle's render of the same pixels with the same random numbers
(`cpu_baseline.error_vs_oracle`).  The 512^3 turbulent medium at 1:10
(1024^2 x 16 spp) is reported beside it (`turbulence512`).

--impl reference times the FP64 CPU oracle (the test oracle, as it stands)
on the host cores over a bounded pixel sample of the same frame.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpaths/s and density lookups/s vs dense-texture render at stated PSNR; HBM GB/s"
WORKLOAD = "cloud1987x1351x2449_r10_pt1920x1080_64spp"
PROFILE = "k_pt_vdb_cloud1987_r10"          # the committed ncu summary of the headline's tracker launch
PROFILE_512 = "k_pt_vdb_turbulence512"
SEED = 2024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vdbc", choices=["vdbc", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 32-volume batched section")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-decoder section")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 512^3 medium section")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--study", choices=["worstcase", "metrics", "hdda", "fullscale"],
                    help="one of the studies beside the benchmark (one JSON line each): lossless dense-noise "
                         "sizes 32^3..2048^3 vs the texture; f1/f2/f3 x rate volume PSNR; hierarchical vs "
                         "uniform DDA; the 1987x1351x2449 cloud at five rates")
    ap.add_argument("--profile-learned", action="store_true",
                    help="ncu capture case of the learned codec: 50 training steps and two 512^2 x 16 spp "
                         "renders of a learned 512^3 medium")
    ap.add_argument("--profile-encode", action="store_true",
                    help="the encoder's capture case: the 994x676x1225 cloud encoded twice at 1:10")
    ap.add_argument("--profile-case-full", action="store_true",
                    help="the same grid rendered twice at the 512^3 block's 1024x1024 x 16 spp")
    ap.add_argument("--profile-case", action="store_true",
                    help="the ncu capture case: the 512^3 medium's grid at a 512x512 image, two renders")
    ap.add_argument("--save-cloud-grid", metavar="PATH",
                    help="encode the full-scale cloud at 1:10 and save the grid to PATH (for --profile-grid)")
    ap.add_argument("--profile-grid", metavar="PATH",
                    help="the headline's ncu capture case: the grid file PATH loaded alone on the device "
                         "(no dense volume or texture) and rendered twice at the headline's frame")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(world=1):
    """The benchmark's `config` (both arms): the 1987x1351x2449 cloud at 1:10, 1920x1080 x 64 spp."""
    from volgen import scenes

    w = scenes.CLOUD_1987
    return {"workload": WORKLOAD, "volume": "1987x1351x2449 f32 cloud (Worley-modulated 8-octave fBm, anvil "
                                            "profile, ~73% zero; the WDAS cloud's dimensions)",
            "ratio": "1:10", "payload": "fp32", "macrocell": w["macrocell"],
            "texture_macrocell": w["texture_macrocell"], "image": "%dx%d" % (w["width"], w["height"]),
            "spp": w["spp"], "max_bounces": w["medium"]["max_bounces"], "albedo": w["medium"]["albedo"],
            "g": w["medium"]["g"], "parallelism": "replicas" if world > 1 else "single",
            "l2": "input 26.3 GB > L2, re-read every step"}


def replica_throughput(total_ms, paths_per_step, steps, world, device=None):
    """Whole-job throughput of N independent replicas: the timed region is the
    max over ranks (one all-reduce of the timing, no data-path collective) and
    the value counts every rank's paths.  Returns (max_ms, Mpaths/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * paths_per_step * steps / (total_ms * 1e-3) / 1e6


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once samples flow (nvidia-smi takes a while to start)
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.skip = len(self.lines)
        except Exception:
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
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        during = self.lines[getattr(self, "skip", 0):]
        if not during:          # a region shorter than the sampling period: the sample just before it
            during = self.lines[-1:]
        for l in during:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash():
    """sha256 (first 16 hex digits) of the tracker's sources with comments and
    blank lines removed: the code the ncu counters were taken on."""
    import re

    h = hashlib.sha256()
    for f in ("render.cu", "vdbc_device.cuh"):
        with open(os.path.join(ROOT, "paper_2504_04564_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        lines = [ln.rstrip() for ln in src.splitlines() if ln.strip()]
        h.update("\n".join(lines).encode())
    return h.hexdigest()[:16]


def profiled_fields(name=PROFILE_512):
    """The `key: value` figures of the committed ncu summary profiles/<name>.md,
    if it was taken on the current tracker source; else None."""
    path = os.path.join(ROOT, "profiles", name + ".md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    fields = {}
    for line in txt.splitlines():
        if ":" in line and not line.startswith(("#", "|", " ", "-")):
            k, val = line.split(":", 1)
            fields[k.strip()] = val.strip()
    if fields.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return fields


def profiled_traffic(name=PROFILE_512):
    """DRAM bytes per launch of the path-tracing kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    f = profiled_fields(name)
    try:
        return float(f["dram_bytes_per_launch_full_size"]) if f else None
    except (KeyError, ValueError):
        return None


def scene(w):
    from volgen import scenes
    cam = scenes.pinhole_orbit(w["dims"], w["width"], w["height"])
    return cam, w["medium"]


def _env(local=0):
    import torch

    import __graft_entry__ as ge
    ge.build()
    import paper_2504_04564_gb300 as v
    import volgen
    from volgen import scenes
    return torch, v, volgen, scenes


def timed_steps(torch, v, vol, w, cam, med, img, stream, steps, warmup, barrier):
    """W untimed and K timed encode + render steps; per-step event times and
    the last step's grid (still open)."""
    for _ in range(max(warmup, 3)):
        g = v.vdbc_encode(vol, w["ratio"], macrocell=w["macrocell"], stream=stream)
        v.vdbc_render(g, cam, med, w["spp"], SEED, img, stream=stream)
        g.close()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    g = None
    for i in range(steps):
        a, b, c = ev[i]
        a.record(stream)
        if g is not None:
            g.close()          # the previous step's grid, freed in stream order as a user's loop frees it
        g = v.vdbc_encode(vol, w["ratio"], macrocell=w["macrocell"], stream=stream)
        b.record(stream)
        v.vdbc_render(g, cam, med, w["spp"], SEED, img, stream=stream)
        c.record(stream)
    t_end.record(stream)
    barrier()
    total_ms = t_start.elapsed_time(t_end)
    enc_ms = [ev[i][0].elapsed_time(ev[i][1]) for i in range(steps)]
    ren_ms = [ev[i][1].elapsed_time(ev[i][2]) for i in range(steps)]
    return total_ms, enc_ms, ren_ms, g


def tracker_roofline(v, g, cam, med, w, img, stream, first_kernel_ms, lookups, profile_name):
    """Roofline of the dominant kernel (the path tracer): algorithmic bytes per
    density lookup = 8 FP32 voxel values = 32 B, over the tracker kernel's own
    duration (CUDA events the library records around its launch on the
    render's stream): the last timed step and four more launches."""
    kms = [float(first_kernel_ms)]
    for _ in range(4):
        v.vdbc_render(g, cam, med, w["spp"], SEED, img, stream=stream)
        kms.append(float(v.vdbc_render_stats_get(g, stream=stream).kernel_ms))
    kms = [k for k in kms if k > 0]
    kernel_ms = sum(kms) / len(kms)
    peak, peak_kind = measured_peaks()
    achieved = lookups * 32.0 / (kernel_ms * 1e-3) / 1e9
    prof = profiled_fields(profile_name)

    def num(k):
        try:
            return float(prof[k]) if prof and k in prof else None
        except ValueError:
            return None
    return {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 5), "traffic": num("dram_bytes_per_launch_full_size"),
            "kernel": "k_pt<VdbSamplerT<0>>", "kernel_ms": round(kernel_ms, 3), "kernel_launches_timed": len(kms),
            "peak_source": peak_kind, "algorithmic_bytes_per_lookup": 32,
            "l2_hit_rate_pct": num("lts_sector_hit_rate_pct"), "sectors_per_request": num("l1tex_sectors_per_request"),
            "dram_gbs_profiled": num("dram_gbs_profiled"), "profile": "profiles/%s.md" % profile_name if prof else None}


def compare(v, a, b, stream=None):
    """FP64 error of image b against image a on the device (RGB)."""
    st = v.vdbc_compare(a, b, stride=4, channels=3, stream=stream)
    return {"psnr_db": (round(st.psnr, 3) if math.isfinite(st.psnr) else "inf"), "rmse": st.rmse,
            "mean_abs": st.mean_abs, "max_abs": st.max_abs}


def run_vdbc(args):
    import numpy as np

    torch, v, volgen, scenes = _env()
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    w = scenes.CLOUD_1987
    cam_args, med_args = scene(w)
    cam = v.make_camera(*cam_args)
    med = v.make_medium(v.MODE_PT, **med_args)
    vol = volgen.generate_torch(volgen.make_params(w["kind"], w["dims"], w["seed"]), dev)
    stream = torch.cuda.current_stream(dev)
    H, W = w["height"], w["width"]
    img = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    paths_per_step = H * W * w["spp"]

    # --- timed region: K whole steps (encode + render) with clocks sampled
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = v.vdbc_kernel_launches()
    total_ms, enc_ms, ren_ms, g = timed_steps(torch, v, vol, w, cam, med, img, stream, args.steps, args.warmup,
                                              barrier)
    launches = v.vdbc_kernel_launches() - launches0
    clk = clocks.stop()
    stats = v.vdbc_render_stats_get(g, stream=stream)
    info = g.info
    total_ms, value = replica_throughput(total_ms, paths_per_step, args.steps, world, dev)
    ms_per_step = total_ms / args.steps
    render_ms = sum(ren_ms) / len(ren_ms)
    lookups = int(stats.lookups)
    vdb_img = img.clone()
    roof = tracker_roofline(v, g, cam, med, w, img, stream, stats.kernel_ms, lookups, PROFILE)
    g.close()

    # --- comparator: the same renderer on the dense 3D texture; the lossless
    # (1:1) render; image errors in FP64 on the device
    tex = v.vdbc_volume_create(vol, v.FILTER_TEXTURE, macrocell=w["texture_macrocell"], stream=stream)
    dimg = torch.empty_like(img)
    for _ in range(2):
        v.vdbc_render_dense(tex, cam, med, w["spp"], SEED, dimg, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, min(args.steps, 3))
    e0.record(stream)
    for _ in range(reps):
        v.vdbc_render_dense(tex, cam, med, w["spp"], SEED, dimg, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    dense_ms = e0.elapsed_time(e1) / reps
    dstats = v.vdbc_volume_render_stats_get(tex, stream=stream)
    tex.close()
    torch.cuda.empty_cache()
    g1 = v.vdbc_encode(vol, 1.0, macrocell=w["macrocell"], stream=stream)   # the uncompressed (lossless) render
    ref_img = torch.empty_like(img)
    v.vdbc_render(g1, cam, med, w["spp"], SEED, ref_img, stream=stream)
    torch.cuda.synchronize()
    lossless_bytes = int(g1.info.total_bytes)
    g1.close()
    errors = {"vdb_r10_vs_lossless_r1": compare(v, ref_img, vdb_img), "vdb_r10_vs_dense_texture": compare(v, dimg, vdb_img),
              "lossless_r1_vs_dense_texture": compare(v, dimg, ref_img),
              "reduction": "FP64 on the device (vdbc_compare), RGB of every pixel, peak 1"}
    host_vol = None
    if rank == 0 and not args.no_cpu_baseline:
        host_vol = vol.cpu().numpy()           # the oracle's input: the same generator output
    del vol
    torch.cuda.empty_cache()

    # --- end to end through the C ABI with host buffers: every step uploads
    # the volume from pinned host memory (vdbc_encode on a host pointer) and
    # reads the image back (vdbc_render into host memory).  Two host threads,
    # one stream each, take alternate steps, so one step's upload overlaps the
    # other's tracker; calls on different handles may run concurrently.
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(torch, v, volgen, w, cam, med, dev, args, barrier, world, paths_per_step)

    secondary = None if args.no_secondary else run_turbulence_section(torch, v, volgen, scenes, dev, stream, args)
    batch = None if args.no_batch else run_batch_section(v, volgen, scenes, dev, stream, args)
    learned = None if args.no_learned else run_learned_section(v, volgen, scenes, dev, stream)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Mpaths/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(world),
        "render_ms": round(render_ms, 3), "encode_ms": round(sum(enc_ms) / len(enc_ms), 3),
        "lookups_per_step": lookups, "glookups_per_s": round(lookups / (render_ms * 1e-3) / 1e9, 3),
        "dense_texture": {"ms_render": round(dense_ms, 3),
                          "mpaths_per_s": round(paths_per_step / (dense_ms * 1e-3) / 1e6, 3),
                          "vdb_over_dense_render_only": round(dense_ms / render_ms, 4),
                          "vdb_over_dense_step": round(dense_ms / ms_per_step, 4),
                          "lookups": int(dstats.lookups)},
        "errors": errors,
        "psnr_db": {"vdb_r10_vs_uncompressed_r1": errors["vdb_r10_vs_lossless_r1"]["psnr_db"],
                    "vdb_r10_vs_dense_texture": errors["vdb_r10_vs_dense_texture"]["psnr_db"]},
        "grid": {"total_bytes": int(info.total_bytes), "payload_bytes": int(info.payload_bytes),
                 "n_active_bricks": int(info.n_active), "n_bricks": int(info.n_bricks),
                 "n_leaves": int(info.n_leaves), "lossless_total_bytes": lossless_bytes,
                 "dense_bytes": int(np.prod(w["dims"])) * 4},
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": e2e,
        "turbulence512": secondary,
        "batch": batch,
        "learned": learned,
    }
    if rank == 0 and not args.no_cpu_baseline:
        oc = CpuOracle(host=host_vol)
        del host_vol
        line["cpu_baseline"] = oc.measure(args.cpu_seconds)
        line["cpu_baseline"]["error_vs_oracle"] = oc.error_against(vdb_img.cpu().numpy())
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_e2e(torch, v, volgen, w, cam, med, dev, args, barrier, world, paths_per_step):
    import numpy as np

    H, W = w["height"], w["width"]
    host_vol = volgen.generate_torch(volgen.make_params(w["kind"], w["dims"], w["seed"]), dev).cpu().pin_memory()
    torch.cuda.empty_cache()
    nlanes = int(os.environ.get("VDBC_E2E_LANES", "2"))
    lanes = [dict(stream=torch.cuda.Stream(device=dev), img=np.empty((H, W, 4), dtype=np.float32))
             for _ in range(nlanes)]

    def e2e_steps(lane, n):
        torch.cuda.set_device(dev)
        st = lane["stream"].cuda_stream
        for _ in range(n):
            g = v.vdbc_encode(host_vol, w["ratio"], macrocell=w["macrocell"], stream=st)
            v.vdbc_render(g, cam, med, w["spp"], SEED, lane["img"], stream=st)
            g.close()

    def run_pair(counts):
        errs = []

        def body(lane, n):
            try:
                e2e_steps(lane, n)
            except Exception as ex:       # surfaced below, on the calling thread
                errs.append(ex)
        ts = [threading.Thread(target=body, args=(lanes[i], counts[i])) for i in range(len(lanes))]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        if errs:
            raise errs[0]

    torch.cuda.synchronize()
    run_pair([1] * len(lanes))
    barrier()
    t0 = time.perf_counter()
    run_pair([args.steps // len(lanes) + (1 if i < args.steps % len(lanes) else 0) for i in range(len(lanes))])
    barrier()
    e2e_s = time.perf_counter() - t0
    out = {"value": round(world * paths_per_step * args.steps / e2e_s / 1e6, 3), "unit": "Mpaths/s",
           "h2d_bytes_per_step": int(host_vol.numel() * 4), "d2h_bytes_per_step": int(H * W * 16),
           "pipeline": "%d host threads, a stream each; one step's upload overlaps the others' work" % len(lanes)}
    del host_vol
    torch.cuda.empty_cache()
    return out


def run_turbulence_section(torch, v, volgen, scenes, dev, stream, args):
    """The 512^3 turbulent medium at 1:10 (1024^2 x 16 spp): the same step
    (encode + render) timed the same way, its roofline, the dense texture and
    PSNR.  Its 54 MB grid stays in L2, so this block shows the tracker with
    the grid on chip, beside the headline's HBM-resident cloud grid."""
    w = scenes.TURBULENCE_512
    cam_args, med_args = scene(w)
    cam = v.make_camera(*cam_args)
    med = v.make_medium(v.MODE_PT, **med_args)
    vol = volgen.generate_torch(volgen.make_params(w["kind"], w["dims"], w["seed"]), dev)
    H, W = w["height"], w["width"]
    img = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    paths = H * W * w["spp"]
    steps = max(3, min(args.steps, 10))
    total_ms, enc_ms, ren_ms, g = timed_steps(torch, v, vol, w, cam, med, img, stream, steps, 3,
                                              torch.cuda.synchronize)
    stats = v.vdbc_render_stats_get(g, stream=stream)
    render_ms = sum(ren_ms) / len(ren_ms)
    vdb_img = img.clone()
    roof = tracker_roofline(v, g, cam, med, w, img, stream, stats.kernel_ms, int(stats.lookups), PROFILE_512)
    g.close()
    tex = v.vdbc_volume_create(vol, v.FILTER_TEXTURE, macrocell=w["texture_macrocell"], stream=stream)
    dimg = torch.empty_like(img)
    v.vdbc_render_dense(tex, cam, med, w["spp"], SEED, dimg, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        v.vdbc_render_dense(tex, cam, med, w["spp"], SEED, dimg, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    dense_ms = e0.elapsed_time(e1) / 3
    tex.close()
    g1 = v.vdbc_encode(vol, 1.0, macrocell=w["macrocell"], stream=stream)
    ref_img = torch.empty_like(img)
    v.vdbc_render(g1, cam, med, w["spp"], SEED, ref_img, stream=stream)
    torch.cuda.synchronize()
    g1.close()
    del vol
    torch.cuda.empty_cache()
    ms_per_step = total_ms / steps
    return {"workload": "turbulence512_r10_pt1024sq_16spp", "steps": steps,
            "mpaths_per_s": round(paths / (ms_per_step * 1e-3) / 1e6, 3), "ms_per_step": round(ms_per_step, 3),
            "render_ms": round(render_ms, 3), "encode_ms": round(sum(enc_ms) / len(enc_ms), 3),
            "lookups_per_frame": int(stats.lookups), "roofline": roof,
            "dense_texture": {"ms_render": round(dense_ms, 3),
                              "mpaths_per_s": round(paths / (dense_ms * 1e-3) / 1e6, 3),
                              "vdb_over_dense_render_only": round(dense_ms / render_ms, 4)},
            "errors": {"vdb_r10_vs_lossless_r1": compare(v, ref_img, vdb_img),
                       "vdb_r10_vs_dense_texture": compare(v, dimg, vdb_img)}}


def batch_oracle_errors(specs, hosts, images, spp_total, pixels_per_job=32):
    """Per volume of the batch: the FP64 oracle encodes and decodes the volume
    itself and renders `pixels_per_job` random pixels with the samples the
    batch images hold (spp_total per pixel, the same random numbers); the
    mean absolute error per channel (largest of R, G, B) and the largest
    absolute error of the GPU image there.  Volumes are done on host threads."""
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    from volgen import scenes

    def one(i):
        sp, host = specs[i], hosts[i]
        e = oracle.encode(host, sp["ratio"], payload=sp["payload"])
        D = oracle.decode_dense(host, e["active"], e["background_bits"], sp["payload"])
        mx = oracle.macrocell_minmax(D, sp["macrocell"])[1]
        pix = np.sort(np.random.default_rng(100 + i).choice(sp["width"] * sp["height"], pixels_per_job, replace=False))
        cam = oracle.make_camera(*scenes.pinhole_orbit(sp["dims"], sp["width"], sp["height"], direction=sp["direction"]))
        ref = oracle.render_pixels(D, mx, cam, oracle.make_medium(1, macrocell=sp["macrocell"], **sp["medium"]),
                                   sp["spp"] * spp_total, sp["seed"], pix)
        d = np.abs(images[i].reshape(-1, 4).astype(np.float64)[pix, :3] - ref[:, :3])
        return float(d.mean(axis=0).max()), float(d.max())

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        res = list(ex.map(one, range(len(specs))))
    return {"mean_abs_per_volume": [r[0] for r in res], "max_abs_per_volume": [r[1] for r in res],
            "worst_mean_abs": max(r[0] for r in res), "tolerance_mean_abs": 1e-4,
            "within_tolerance": bool(max(r[0] for r in res) <= 1e-4), "pixels_per_volume": pixels_per_job,
            "samples_per_pixel": "each job's spp x %d frames" % spp_total, "oracle_s": round(time.perf_counter() - t0, 2)}


def run_batch_section(v, volgen, scenes, dev, stream, args):
    """The batched form: 32 volumes of uneven size (FP16/FP8 leaves, rates 1:4..1:20,
    images 256^2..1024^2, 4..32 spp) in one persistent launch per payload group
    per frame from a captured CUDA graph, against rendering the same jobs one
    by one; every volume's image checked against the FP64 oracle."""
    import torch

    specs = scenes.batch_jobs()
    grids, imgs, jobs, hosts = [], [], [], []
    payload_bytes = 0
    for sp in specs:
        vol = volgen.generate_torch(volgen.make_params(sp["kind"], sp["dims"], sp["seed"]), dev)
        g = v.vdbc_encode(vol, sp["ratio"], payload=sp["payload"], macrocell=sp["macrocell"], stream=stream)
        if not args.no_cpu_baseline:
            hosts.append(vol.cpu().numpy())
        del vol
        payload_bytes += int(g.info.payload_bytes)
        cam = v.make_camera(*scenes.pinhole_orbit(sp["dims"], sp["width"], sp["height"], direction=sp["direction"]))
        med = v.make_medium(v.MODE_PT, **sp["medium"])
        img = torch.empty((sp["height"], sp["width"], 4), dtype=torch.float32, device=dev)
        grids.append(g)
        imgs.append(img)
        jobs.append((v.make_job(g, cam, med, sp["spp"], sp["seed"], img), cam, med))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = v.vdbc_batch_create([j[0] for j in jobs], autotune=True, stream=stream, keep=(grids, imgs))
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    tuning = v.vdbc_batch_get_tuning(b)
    paths = sum(sp["width"] * sp["height"] * sp["spp"] for sp in specs)
    frames = max(2, min(args.steps, 3))
    v.vdbc_batch_render_frames(b, 1, stream=stream)        # warm-up frame
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    v.vdbc_batch_render_frames(b, frames, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1) / frames
    st = v.vdbc_batch_stats_get(b, stream=stream)
    batch_imgs = [im.cpu().numpy() for im in imgs]          # the running mean of 1 + frames frames
    # the plain form: one vdbc_render per job, same samples, with the coarse
    # DDA level the tuner chose for the batch
    os.environ["VDBC_PT_COARSE"] = str(int(tuning.coarse))
    for (job, cam, med), sp, img in zip(jobs[:1], specs[:1], imgs[:1]):
        v.vdbc_render(grids[0], cam, med, sp["spp"], sp["seed"], img, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for (job, cam, med), sp, img, g in zip(jobs, specs, imgs, grids):
        v.vdbc_render(g, cam, med, sp["spp"], sp["seed"], img, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    os.environ.pop("VDBC_PT_COARSE", None)
    b.close()
    for g in grids:
        g.close()
    errors = batch_oracle_errors(specs, hosts, batch_imgs, 1 + frames) if hosts else None
    return {"jobs": len(specs), "paths_per_frame": paths, "frame_ms": round(batch_ms, 3), "error_vs_oracle": errors,
            "mpaths_per_s": round(paths / (batch_ms * 1e-3) / 1e6, 3),
            "one_by_one_ms": round(plain_ms, 3),
            "one_by_one_mpaths_per_s": round(paths / (plain_ms * 1e-3) / 1e6, 3),
            "speedup_vs_one_by_one": round(plain_ms / batch_ms, 4),
            "payload_bytes": payload_bytes, "lookups_per_frame": int(st.lookups),
            "tuning": {"threads": tuning.threads, "chunk": tuning.chunk, "paths_per_lane_per_refill": tuning.chunk // 32,
                       "coarse": tuning.coarse, "accessor_depth": tuning.depth},
            "create_s_incl_autotune": round(create_s, 3),
            "workload": "32 blob+fBm volumes, edges 64..384, rates 1:4..1:20, FP16/FP8, 256^2..1024^2, 4..32 spp, "
                        "%d^3 cells" % specs[0]["macrocell"]}


def run_learned_section(v, volgen, scenes, dev, stream):
    """The learned leaf decoder on the 994 x 676 x 1225 cloud: a learned grid
    built from every non-empty brick and held to the bytes of VDB FP32 at 1:10,
    against VDB FP32 and FP16 at 1:10 (equal bytes by the rate's definition);
    volume PSNR against the input, and each at 1920 x 1080 x 32 spp against
    the dense-texture render (image PSNR, Mpaths/s)."""
    import math

    import torch

    w = scenes.CLOUD_994
    vol = volgen.generate_torch(volgen.make_params(w["kind"], w["dims"], w["seed"]), dev)
    torch.cuda.synchronize()

    def vpsnr(g):
        # volume PSNR (peak 1, the paper's convention) from the FP64 device reduction
        out = torch.empty_like(vol)
        v.vdbc_grid_decode(g, out, stream=stream)
        st = v.vdbc_compare(vol, out, stream=stream)
        return round(st.psnr, 3) if math.isfinite(st.psnr) else "inf"

    full = v.vdbc_encode(vol, 1.0, macrocell=w["macrocell"], stream=stream)
    vdb32 = v.vdbc_encode(vol, w["ratio"], macrocell=w["macrocell"], stream=stream)
    vdb16 = v.vdbc_encode(vol, w["ratio"], payload=v.FP16, macrocell=w["macrocell"], stream=stream)
    budget = int(vdb32.info.total_bytes)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    learned, losses = v.vdbc_learn(full, max_bytes=budget, stream=stream, **w["learn"])
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    cam = v.make_camera(*scenes.pinhole_orbit(w["dims"], w["width"], w["height"]))
    med = v.make_medium(v.MODE_PT, **w["medium"])
    dense = v.vdbc_volume_create(vol, v.FILTER_TEXTURE, w.get("texture_macrocell", w["macrocell"]), stream=stream)
    img = torch.empty((w["height"], w["width"], 4), dtype=torch.float32, device=dev)
    paths = w["width"] * w["height"] * w["spp"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_render(target, is_dense=False):
        fn = v.vdbc_render_dense if is_dense else v.vdbc_render
        fn(target, cam, med, w["spp"], 1, img, stream=stream)      # warm-up
        e0.record(stream)
        fn(target, cam, med, w["spp"], 1, img, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        st = (v.vdbc_volume_render_stats_get if is_dense else v.vdbc_render_stats_get)(target, stream=stream)
        return e0.elapsed_time(e1), img.clone(), int(st.lookups)

    ref_ms, ref, ref_lk = timed_render(dense, True)

    def entry(g, name):
        ms, im, lk = timed_render(g)
        err = compare(v, ref, im, stream)
        info = g.info
        return {"total_bytes": int(info.total_bytes), "volume_psnr_db": vpsnr(g),
                "image_psnr_vs_dense_db": err["psnr_db"], "image_rmse_vs_dense": err["rmse"],
                "render_ms": round(ms, 3), "mpaths_per_s": round(paths / (ms * 1e-3) / 1e6, 3),
                "lookups": lk}

    res = {"workload": "cloud994x676x1225_learned_vs_vdb_r10_pt1920x1080_32spp",
           "zero_fraction": round(float((vol == 0).float().mean()), 4),
           "byte_budget": budget,
           "dense_texture": {"render_ms": round(ref_ms, 3), "mpaths_per_s": round(paths / (ref_ms * 1e-3) / 1e6, 3),
                             "lookups": ref_lk},
           "vdb_fp32_r10": entry(vdb32, "vdb32"), "vdb_fp16_r10": entry(vdb16, "vdb16")}
    le = entry(learned, "learned")
    le.update({"n_neural": int(learned.info.n_neural), "n_raw": int(learned.info.n_leaves),
               "train_s": round(train_s, 3), "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
               "training": dict(w["learn"]), "source_leaves": int(full.info.n_leaves)})
    res["learned"] = le
    for g in (full, vdb32, vdb16, learned):
        g.close()
    dense.close()
    del vol
    torch.cuda.empty_cache()
    return res


def input_volume(w):
    """The workload's input on the host: the seeded generator's output, made
    on the device when one is present (its device and host builds give the
    same bits; the host build alone takes minutes at 6.57 G voxels)."""
    import volgen

    p = volgen.make_params(w["kind"], w["dims"], w["seed"])
    try:
        import torch
        if torch.cuda.is_available():
            out = volgen.generate_torch(p).cpu().numpy()
            torch.cuda.empty_cache()
            return out
    except ImportError:
        pass
    return volgen.generate_host(p, threads=os.cpu_count() or 1)


class CpuOracle:
    """The FP64 oracle (unchanged) on the host cores.  The workload's volume is
    encoded once by the oracle (B, brick ranges, scores, selection) and decoded
    to the dense grid D that its renderer samples.  A measurement traces a
    random pixel sample of the frame (every spp of each pixel) sized to about
    budget_s seconds; error_against() traces every 16th row and column of the
    frame and compares the GPU image there."""

    def __init__(self, host=None, w=None):
        import numpy as np

        import oracle
        from volgen import scenes

        self.np, self.oracle = np, oracle
        self.w = w = w or scenes.CLOUD_1987
        self.cores = os.cpu_count() or 1
        if host is None:
            host = input_volume(w)
        t0 = time.perf_counter()
        e = oracle.encode(host, w["ratio"])
        self.n_active = int(e["n_active"])
        self.D = oracle.decode_dense(host, e["active"], e["background_bits"])
        del host, e
        self.mx = oracle.macrocell_minmax(self.D, w["macrocell"])[1]
        self.enc_s = time.perf_counter() - t0
        cam_args, med_args = scene(w)
        self.cam = oracle.make_camera(*cam_args)
        self.med = oracle.make_medium(1, macrocell=w["macrocell"], **med_args)
        W, H = w["width"], w["height"]
        pix = np.arange(W * H, dtype=np.int64)
        np.random.default_rng(0).shuffle(pix)     # an unbiased subset of the frame at any size
        self.pix = pix
        self.n = min(4096, pix.size)

    def _render(self, pixels):
        w = self.w
        return self.oracle.render_pixels(self.D, self.mx, self.cam, self.med, w["spp"], SEED, pixels,
                                         threads=self.cores)

    def measure(self, budget_s):
        w = self.w
        t0 = time.perf_counter()
        self._render(self.pix[:self.n])
        dt = time.perf_counter() - t0
        # size the next sample to about budget_s
        self.n = int(min(self.pix.size, max(16, self.n * budget_s / max(dt, 1e-3))))
        paths = self.n * w["spp"]
        t0 = time.perf_counter()
        self._render(self.pix[:self.n])
        dt = time.perf_counter() - t0
        return {"value": round(paths / dt / 1e6, 6), "unit": "Mpaths/s", "cores": self.cores, "kind": "oracle",
                "sample": "%d random pixels of the %dx%d frame x %d spp = %d paths in %.2f s; the oracle's "
                          "encode + decode + macrocells of the full %dx%dx%d volume took %.1f s (not in the rate)"
                          % (self.n, w["width"], w["height"], w["spp"], paths, dt, *w["dims"], self.enc_s)}

    def error_against(self, gpu_rgba):
        """Mean and largest absolute difference per channel between the GPU
        image and the oracle's FP64 render at every 16th row and column (the
        same pixels, samples and random numbers)."""
        np, w = self.np, self.w
        W, H = w["width"], w["height"]
        ys, xs = np.meshgrid(np.arange(8, H, 16), np.arange(8, W, 16), indexing="ij")
        pix = (ys * W + xs).ravel().astype(np.int64)
        t0 = time.perf_counter()
        ref = self._render(pix)
        dt = time.perf_counter() - t0
        got = np.asarray(gpu_rgba, dtype=np.float64).reshape(-1, 4)[pix]
        d = np.abs(got[:, :3] - ref[:, :3])
        mean_abs = [float(x) for x in d.mean(axis=0)]
        return {"pixels": int(pix.size), "spp": w["spp"], "paths": int(pix.size) * w["spp"],
                "sample": "every 16th row and column of the frame", "mean_abs_rgb": mean_abs,
                "max_abs": float(d.max()), "tolerance_mean_abs": 1e-4,
                "within_tolerance": bool(max(mean_abs) <= 1e-4), "oracle_s": round(dt, 2),
                "oracle_active_bricks": self.n_active}


def cpu_baseline(budget_s):
    return CpuOracle().measure(budget_s)


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    steps = max(1, args.steps)
    co = CpuOracle()
    per = max(1.0, min(20.0, 100.0 / (steps + max(args.warmup, 0))))
    for _ in range(max(args.warmup, 0)):
        co.measure(per)
    vals, cb = [], None
    t0 = time.perf_counter()
    for _ in range(steps):
        cb = co.measure(per)
        vals.append(cb["value"])
    total = time.perf_counter() - t0
    value = sum(vals) / len(vals)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Mpaths/s",
            "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": round(total * 1e3 / steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(world),
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"], "value": round(value, 6),
                             "unit": "Mpaths/s"},
            "e2e": {"value": round(value, 6), "unit": "Mpaths/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile_case(full=False):
    """The capture case for `ncu --set full`: the 512^3 medium at 1:10 (same
    grid as the benchmark's 512^3 block), rendered twice at 512x512 x 16 spp so
    that a full-section capture of the second launch stays small; with `full`,
    at the block's own 1024x1024 x 16 spp (for one-pass DRAM counters)."""
    torch, v, volgen, scenes = _env()
    w = scenes.TURBULENCE_512
    n = w["width"] if full else 512
    cam = v.make_camera(*scenes.pinhole_orbit(w["dims"], n, n))
    med = v.make_medium(v.MODE_PT, **w["medium"])
    vol = volgen.generate_torch(volgen.make_params(w["kind"], w["dims"], w["seed"]))
    g = v.vdbc_encode(vol, w["ratio"], macrocell=w["macrocell"])
    img = torch.empty((n, n, 4), dtype=torch.float32, device="cuda")
    for _ in range(2):
        v.vdbc_render(g, cam, med, w["spp"], SEED, img)
    torch.cuda.synchronize()
    st = v.vdbc_render_stats_get(g)
    print(json.dumps({"profile_case": "turbulence512_r10_pt%dsq_16spp" % n, "lookups": int(st.lookups),
                      "paths": int(st.paths), "kernel_ms": float(st.kernel_ms)}))


def run_profile_encode():
    """The encoder's capture case: the 994 x 676 x 1225 cloud (3.3 GB, the
    full-scale cloud's generator at half the edge) encoded twice at 1:10."""
    torch, v, volgen, scenes = _env()
    w = scenes.CLOUD_994
    vol = volgen.generate_torch(volgen.make_params(w["kind"], w["dims"], w["seed"]))
    for _ in range(2):
        g = v.vdbc_encode(vol, w["ratio"], macrocell=w["macrocell"])
        torch.cuda.synchronize()
        n_active = int(g.info.n_active)
        g.close()
    print(json.dumps({"profile_case": "cloud994x676x1225_encode_r10", "n_active": n_active}))


def run_save_cloud_grid(path):
    """Encodes the headline's volume at its rate and saves the grid (the input
    of --profile-grid, which then holds nothing else on the device)."""
    torch, v, volgen, scenes = _env()
    w = scenes.CLOUD_1987
    vol = volgen.generate_torch(volgen.make_params(w["kind"], w["dims"], w["seed"]))
    g = v.vdbc_encode(vol, w["ratio"], macrocell=w["macrocell"])
    v.vdbc_grid_save(g, path)
    print(json.dumps({"saved": path, "total_bytes": int(g.info.total_bytes), "n_active": int(g.info.n_active)}))


def run_profile_grid(path):
    """The headline's capture case: the saved grid loaded alone on the device
    (about 2.6 GB) and rendered twice at the headline's frame (1920x1080 x
    64 spp, albedo 0.95, g 0.8, 32 bounces)."""
    torch, v, volgen, scenes = _env()
    w = scenes.CLOUD_1987
    g = v.vdbc_grid_load(path)
    cam = v.make_camera(*scenes.pinhole_orbit(w["dims"], w["width"], w["height"]))
    med = v.make_medium(v.MODE_PT, **w["medium"])
    img = torch.empty((w["height"], w["width"], 4), dtype=torch.float32, device="cuda")
    for _ in range(2):
        v.vdbc_render(g, cam, med, w["spp"], SEED, img)
    torch.cuda.synchronize()
    st = v.vdbc_render_stats_get(g)
    print(json.dumps({"profile_case": WORKLOAD, "grid_bytes": int(g.info.total_bytes), "lookups": int(st.lookups),
                      "paths": int(st.paths), "kernel_ms": float(st.kernel_ms)}))


def run_profile_learned():
    """The capture case of the learned codec: the 512^3 medium's every
    non-empty brick turned into a learned grid held to the bytes of VDB 1:10
    (50 training steps, 64 samples per leaf), rendered twice at 512x512 x 16 spp."""
    import torch

    import __graft_entry__ as ge
    ge.build()
    import paper_2504_04564_gb300 as v
    import volgen
    from volgen import scenes

    w = scenes.TURBULENCE_512
    cam = v.make_camera(*scenes.pinhole_orbit(w["dims"], 512, 512))
    med = v.make_medium(v.MODE_PT, **w["medium"])
    vol = volgen.generate_torch(volgen.make_params(w["kind"], w["dims"], w["seed"]))
    full = v.vdbc_encode(vol, 1.0, macrocell=w["macrocell"])
    budget = int(v.vdbc_encode(vol, w["ratio"], macrocell=w["macrocell"]).info.total_bytes)
    g, losses = v.vdbc_learn(full, steps=50, samples_per_leaf=64, lr=2e-3, lr_latent=2e-2, max_bytes=budget, seed=1)
    img = torch.empty((512, 512, 4), dtype=torch.float32, device="cuda")
    for _ in range(2):
        v.vdbc_render(g, cam, med, w["spp"], SEED, img)
    torch.cuda.synchronize()
    st = v.vdbc_render_stats_get(g)
    print(json.dumps({"profile_case": "turbulence512_learned_pt512sq_16spp", "lookups": int(st.lookups),
                      "paths": int(st.paths), "n_neural": int(g.info.n_neural), "n_raw": int(g.info.n_leaves),
                      "loss_last": float(losses[-1])}))


def _study_env():
    import torch

    import __graft_entry__ as ge
    ge.build()
    import paper_2504_04564_gb300 as v
    import volgen
    from volgen import scenes
    return torch, v, volgen, scenes


def _timed_render(torch, v, target, cam, med, spp, img, dense=False, reps=1):
    fn = v.vdbc_render_dense if dense else v.vdbc_render
    fn(target, cam, med, spp, 1, img)                      # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn(target, cam, med, spp, 1, img)
    e1.record()
    torch.cuda.synchronize()
    st = (v.vdbc_volume_render_stats_get if dense else v.vdbc_render_stats_get)(target)
    return e0.elapsed_time(e1) / reps, int(st.lookups)


def study_worstcase():
    """The paper's worst case (tab:worstcase): dense noise in (0, 1] that leaves
    no brick empty, encoded losslessly (1:1) at 32^3..2048^3; grid bytes
    against the dense bytes, and path-tracing throughput of the grid against
    the dense texture (1024^2 x 4 spp, the benchmark's medium and macrocells)."""
    torch, v, volgen, scenes = _study_env()
    rows = []
    for n in (32, 64, 128, 256, 512, 1024, 2048):
        dims = (n, n, n)
        vol = volgen.generate_torch(volgen.make_params("noise", dims, 7))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = v.vdbc_encode(vol, 1.0, macrocell=scenes.TURBULENCE_512["macrocell"])
        torch.cuda.synchronize()
        enc_ms = (time.perf_counter() - t0) * 1e3
        dense = v.vdbc_volume_create(vol, v.FILTER_TEXTURE, scenes.TURBULENCE_512["texture_macrocell"])
        cam = v.make_camera(*scenes.pinhole_orbit(dims, 1024, 1024))
        med = v.make_medium(v.MODE_PT, **scenes.pt_medium_args())
        img = torch.empty((1024, 1024, 4), dtype=torch.float32, device="cuda")
        paths = 1024 * 1024 * 4
        ms_g, lk_g = _timed_render(torch, v, g, cam, med, 4, img)
        ms_d, lk_d = _timed_render(torch, v, dense, cam, med, 4, img, dense=True)
        info = g.info
        dense_bytes = n * n * n * 4
        rows.append({"n": n, "dense_bytes": dense_bytes, "grid_bytes": int(info.total_bytes),
                     "overhead_pct": round(100.0 * (int(info.total_bytes) / dense_bytes - 1.0), 2),
                     "n_leaves": int(info.n_leaves), "n_tiles": int(info.n_tiles), "encode_ms": round(enc_ms, 2),
                     "grid_mpaths_per_s": round(paths / (ms_g * 1e-3) / 1e6, 2),
                     "texture_mpaths_per_s": round(paths / (ms_d * 1e-3) / 1e6, 2),
                     "grid_over_texture": round(ms_d / ms_g, 4), "lookups_grid": lk_g, "lookups_texture": lk_d})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        g.close()
        dense.close()
        del vol
        torch.cuda.empty_cache()
    return {"study": "worstcase_dense_noise_lossless",
            "render": "pt 1024x1024x4spp, density 20/unit, %d^3 cells (grid), %d^3 (texture)"
                      % (scenes.TURBULENCE_512["macrocell"], scenes.TURBULENCE_512["texture_macrocell"]),
            "rows": rows}


def study_metrics():
    """f1/f2/f3 x rate (Fig. fig:distance): volume PSNR (peak 1) of the decoded
    grid against the input, on the 512^3 medium and the 994x676x1225 cloud."""
    torch, v, volgen, scenes = _study_env()
    out = {"study": "metric_rate_psnr", "rates": [1.0, 1.33, 2.0, 4.0, 6.0, 10.0, 20.0, 50.0], "volumes": {}}
    for name, kind, dims in (("turbulence512", "turbulence", (512, 512, 512)), ("cloud994", "cloud", (994, 676, 1225))):
        vol = volgen.generate_torch(volgen.make_params(kind, dims, 0))
        dec = torch.empty_like(vol)
        res = {}
        for metric in (v.F1, v.F2, v.F3):
            curve = []
            for r in out["rates"]:
                g = v.vdbc_encode(vol, r, metric=metric)
                v.vdbc_grid_decode(g, dec)
                mse = float(((dec.double() - vol.double()) ** 2).mean())
                curve.append(round(10 * math.log10(1.0 / mse), 3) if mse > 0 else None)
                g.close()
            res["f%d" % metric] = curve
        out["volumes"][name] = res
        del vol, dec
        torch.cuda.empty_cache()
    return out


def study_hdda():
    """Hierarchical against uniform DDA (Section 4 found diminishing returns):
    the benchmark's frame with the coarse level (8^3 blocks of macrocells; at
    16^3 cells a block is a lower node's 128^3 voxels) on and off, per
    macrocell size.  (The renderer turns the level on for cells of at most 8
    voxels; the study forces both settings.)"""
    torch, v, volgen, scenes = _study_env()
    w = scenes.TURBULENCE_512
    vol = volgen.generate_torch(volgen.make_params(w["kind"], w["dims"], w["seed"]))
    cam = v.make_camera(*scenes.pinhole_orbit(w["dims"], w["width"], w["height"]))
    med = v.make_medium(v.MODE_PT, **w["medium"])
    img = torch.empty((w["height"], w["width"], 4), dtype=torch.float32, device="cuda")
    paths = w["width"] * w["height"] * w["spp"]
    rows = []
    for mc in (8, 16, 32, 48, 64):
        g = v.vdbc_encode(vol, w["ratio"], macrocell=mc)
        for coarse in ("1", "0"):
            os.environ["VDBC_PT_COARSE"] = coarse
            ms, lk = _timed_render(torch, v, g, cam, med, w["spp"], img, reps=3)
            rows.append({"macrocell": mc, "hierarchical": coarse == "1", "render_ms": round(ms, 3),
                         "mpaths_per_s": round(paths / (ms * 1e-3) / 1e6, 2), "lookups": lk})
        g.close()
    os.environ.pop("VDBC_PT_COARSE", None)
    return {"study": "hierarchical_vs_uniform_dda", "workload": "turbulence512_r10_pt1024sq_16spp", "rows": rows}


def study_fullscale():
    """The 1987 x 1351 x 2449 cloud (26.3 GB) at 1:20, 1:10, 1:6, 1:5 and 1:4,
    1920x1080 x 64 spp, up to 32 bounces, against the dense texture: Mpaths/s,
    lookups/s, algorithmic lookup GB/s as a fraction of the measured HBM
    bandwidth, volume PSNR and image PSNR against the texture render."""
    torch, v, volgen, scenes = _study_env()
    dims = (1987, 1351, 2449)
    vol = volgen.generate_torch(volgen.make_params("cloud", dims, 0))
    torch.cuda.synchronize()
    W, H, spp = 1920, 1080, 64
    cam = v.make_camera(*scenes.pinhole_orbit(dims, W, H))
    med = v.make_medium(v.MODE_PT, **scenes.pt_medium_args(albedo=0.95, g=0.8, max_bounces=32))
    img = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    paths = W * H * spp
    peak, _ = measured_peaks()
    mc = scenes.CLOUD_1987["macrocell"]
    dense = v.vdbc_volume_create(vol, v.FILTER_TEXTURE, scenes.CLOUD_1987["texture_macrocell"])
    ms_d, lk_d = _timed_render(torch, v, dense, cam, med, spp, img, dense=True)
    ref = img.clone()
    dense.close()
    rows = []
    dec = None
    for r in (20.0, 10.0, 6.0, 5.0, 4.0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = v.vdbc_encode(vol, r, macrocell=mc)
        torch.cuda.synchronize()
        enc_ms = (time.perf_counter() - t0) * 1e3
        ms, lk = _timed_render(torch, v, g, cam, med, spp, img)
        mse_i = float(((img[..., :3].double() - ref[..., :3].double()) ** 2).mean())
        if dec is None:
            dec = torch.empty_like(vol)
        v.vdbc_grid_decode(g, dec)
        mse_v = float(((dec.double() - vol.double()) ** 2).mean())
        gbs = lk * 32 / (ms * 1e-3) / 1e9
        info = g.info
        rows.append({"rate": r, "payload_bytes": int(info.payload_bytes), "total_bytes": int(info.total_bytes),
                     "encode_ms": round(enc_ms, 1), "render_ms": round(ms, 2),
                     "mpaths_per_s": round(paths / (ms * 1e-3) / 1e6, 2), "glookups_per_s": round(lk / ms / 1e6, 3),
                     "lookup_gbs": round(gbs, 1), "lookup_gbs_frac_of_measured_hbm": round(gbs / peak, 4),
                     "volume_psnr_db": round(10 * math.log10(1.0 / max(mse_v, 1e-30)), 3),
                     "image_psnr_vs_texture_db": round(10 * math.log10(1.0 / max(mse_i, 1e-30)), 3)})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        g.close()
    return {"study": "fullscale_cloud1987x1351x2449", "render": "pt 1920x1080x64spp, albedo 0.95, g 0.8, 32 bounces",
            "texture": {"render_ms": round(ms_d, 2), "mpaths_per_s": round(paths / (ms_d * 1e-3) / 1e6, 2),
                        "lookups": lk_d},
            "zero_fraction": round(float((vol == 0).float().mean()), 4), "rows": rows}


if __name__ == "__main__":
    a = parse()
    if a.study:
        import math
        res = {"worstcase": study_worstcase, "metrics": study_metrics, "hdda": study_hdda,
               "fullscale": study_fullscale}[a.study]()
        print(json.dumps(res), flush=True)
    elif a.profile_learned:
        run_profile_learned()
    elif a.save_cloud_grid:
        run_save_cloud_grid(a.save_cloud_grid)
    elif a.profile_grid:
        run_profile_grid(a.profile_grid)
    elif a.profile_case:
        run_profile_case()
    elif a.profile_case_full:
        run_profile_case(full=True)
    elif a.profile_encode:
        run_profile_encode()
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_vdbc(a)
