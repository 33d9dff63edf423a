"""Child process of tests/test_gpu_checked.py.

The package binds one library per process, chosen at import by VDBC_CHECKED,
so the bounds-checked build runs here, in its own interpreter:

    VDBC_CHECKED=1 python tests/checked_child.py workload OUT.npz
    VDBC_CHECKED=1 VDBC_FAULT=bounds python tests/checked_child.py bad GRID OUT.npz X Y

`workload` writes the outputs of run_workload() (which the parent also runs
in-process on the plain build); `bad` loads a grid file with one leaf entry
past the last leaf, decodes it and marches one ray through that leaf, and
records what each call returned.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DIMS = (40, 36, 44)


def ramp_tf():
    r = np.arange(256, dtype=np.float32) / 255.0
    return np.stack([r, r, r, r], axis=1)


def run_workload(v, torch, vg, sc):
    """Encodes, decodes and renders (PT, EA, ISO) FP32/FP16/FP8 grids, a
    learned grid and a two-job batch; returns every output and error word."""
    dev = torch.device("cuda:0")
    out = {}
    host = vg.generate_host(vg.make_params("blobs", DIMS, 3))
    vol = torch.from_numpy(host).to(dev)
    cam = v.make_camera(*sc.pinhole_orbit(DIMS, 24, 20))
    pt = v.make_medium(v.MODE_PT, **sc.pt_medium_args(density_scale=30.0, g=0.5, max_bounces=4))
    ea = v.make_medium(v.MODE_EA, tf=ramp_tf(), step=0.5)
    iso = v.make_medium(v.MODE_ISO, step=0.5, iso=0.3)
    grids = {}
    for payload in (v.FP32, v.FP16, v.FP8):
        g = v.vdbc_encode(vol, 4.0, payload=payload)
        grids[payload] = g
        dec = torch.empty_like(vol)
        v.vdbc_grid_decode(g, dec)
        out["decode_%d" % payload] = dec.cpu().numpy()
        for name, med, spp in (("pt", pt, 2), ("ea", ea, 1), ("iso", iso, 1)):
            img = torch.zeros((20, 24, 4), dtype=torch.float32, device=dev)
            v.vdbc_render(g, cam, med, spp, 7, img)
            torch.cuda.synchronize()
            out["%s_%d" % (name, payload)] = img.cpu().numpy()
            st = v.vdbc_render_stats_get(g)
            out["flags_%s_%d" % (name, payload)] = np.uint64(st.error_flags)
            if name == "pt":       # the tracker's event counters (zero unless built with them)
                out["events_pt_%d" % payload] = np.array(list(st.events) + [st.lookups, st.paths], dtype=np.uint64)
    npos = ((DIMS[0] + 7) // 8) * ((DIMS[1] + 7) // 8) * ((DIMS[2] + 7) // 8)
    half = torch.arange(npos, device=dev) % 2 + 1          # neural and raw leaves, alternating by position
    learned, _ = v.vdbc_learn(grids[v.FP16], steps=3, samples_per_leaf=16, seed=5, force=half.to(torch.uint8))
    out["n_neural"] = np.int64(learned.info.n_neural)
    dec = torch.empty_like(vol)
    v.vdbc_grid_decode(learned, dec)
    out["decode_learned"] = dec.cpu().numpy()
    for name, med, spp in (("pt", pt, 2), ("iso", iso, 1)):
        img = torch.zeros((20, 24, 4), dtype=torch.float32, device=dev)
        v.vdbc_render(learned, cam, med, spp, 7, img)
        torch.cuda.synchronize()
        out["%s_learned" % name] = img.cpu().numpy()
        out["flags_%s_learned" % name] = np.uint64(v.vdbc_render_stats_get(learned).error_flags)
    imgs = [torch.zeros((20, 24, 4), dtype=torch.float32, device=dev) for _ in range(2)]
    jobs = [v.make_job(grids[p], cam, pt, 2, 11 + i, imgs[i]) for i, p in enumerate((v.FP16, v.FP8))]
    b = v.vdbc_batch_create(jobs, autotune=False, keep=(imgs, grids))
    v.vdbc_batch_render_frames(b, 2)
    torch.cuda.synchronize()
    for i in range(2):
        out["batch_%d" % i] = imgs[i].cpu().numpy()
    out["flags_batch"] = np.uint64(v.vdbc_batch_stats_get(b).error_flags)
    return out


def run_bad(v, torch, path, x, y):
    """Loads the corrupted grid, decodes it and marches one ray through (x, y)."""
    res = {}
    g = v.vdbc_grid_load(path)
    info = g.info
    res["background_bits"] = np.uint32(info.background_bits)
    dec = torch.full(tuple(info.dims[::-1]), float("nan"), dtype=torch.float32, device="cuda:0")
    try:
        v.vdbc_grid_decode(g, dec)
        res["decode_status"] = np.int32(0)
    except v.VdbcError as e:
        res["decode_status"] = np.int32(e.status)
    torch.cuda.synchronize()
    res["decode"] = dec.cpu().numpy()
    M = float(max(info.dims))
    cam = v.make_camera(v.CAM_ORTHO, 1, 1, ((x + 0.5) / M, (y + 0.5) / M, -1.0), ((x + 0.5) / M, (y + 0.5) / M, 0.0),
                        (0, 1, 0), 0.01)
    med = v.make_medium(v.MODE_EA, tf=ramp_tf(), step=0.5)
    img = np.zeros((1, 1, 4), dtype=np.float32)
    try:
        v.vdbc_render(g, cam, med, 1, 0, img)
        res["render_status"] = np.int32(0)
    except v.VdbcError as e:
        res["render_status"] = np.int32(e.status)
    # the context is still usable: the same ray through an intact grid
    ok = v.vdbc_encode(dec.nan_to_num(0.0).contiguous(), 1.0)
    v.vdbc_render(ok, cam, med, 1, 0, img)
    res["after"] = img
    return res


def main():
    import torch
    import paper_2504_04564_gb300 as v
    import volgen as vg
    from volgen import scenes as sc

    if not v.vdbc_version().endswith("checked"):
        raise SystemExit("not the checked build: " + v.vdbc_version())
    torch.cuda.set_device(0)
    if sys.argv[1] == "workload":
        np.savez(sys.argv[2], **run_workload(v, torch, vg, sc))
    elif sys.argv[1] == "bad":
        np.savez(sys.argv[3], **run_bad(v, torch, sys.argv[2], int(sys.argv[4]), int(sys.argv[5])))
    else:
        raise SystemExit("unknown mode " + sys.argv[1])


if __name__ == "__main__":
    main()
