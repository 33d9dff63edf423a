"""The batched path tracer: many grids of uneven size and payload, each with
its own camera, medium, spp and seed, in one persistent launch per frame,
replayed from a captured CUDA graph.  Every job's image must equal what the
single-job renderer gives for the same samples (F frames of spp samples are
sample ids 0 .. F*spp-1), and the FP64 oracle within the path-tracing
tolerance."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
PT_MEAN_ABS = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__ as g
    g.build()
    import oracle
    import paper_2504_04564_gb300 as v
    import volgen
    from volgen import scenes
    return dict(torch=torch, v=v, orc=oracle, vg=volgen, sc=scenes, dev=torch.device("cuda:0"))


JOBS = [  # kind, dims, ratio, payload, image (w, h), spp, seed, g, macrocell
    ("blobs", (72, 64, 90), 4.0, 1, (40, 33), 3, 11, 0.6, 8),
    ("turbulence", (96, 80, 64), 10.0, 2, (24, 24), 2, 12, 0.3, 16),
    ("blobs", (64, 110, 70), 6.0, 0, (17, 29), 4, 13, 0.8, 8),
    ("turbulence", (80, 80, 80), 20.0, 1, (32, 20), 1, 14, 0.0, 4),
    ("blobs", (130, 64, 64), 4.0, 2, (9, 7), 5, 15, -0.3, 8),
]


def build_jobs(env):
    torch, v, vg, sc = env["torch"], env["v"], env["vg"], env["sc"]
    out = []
    for i, (kind, dims, ratio, payload, (w, h), spp, seed, g, mc) in enumerate(JOBS):
        host = vg.generate_host(vg.make_params(kind, dims, seed))
        grid = v.vdbc_encode(torch.from_numpy(host).to(env["dev"]), ratio, payload=payload, macrocell=mc)
        cam = v.make_camera(*sc.pinhole_orbit(dims, w, h, direction=(0.6 - 0.2 * i, 0.4, 0.7)))
        med_args = sc.pt_medium_args(density_scale=25.0 + 5 * i, g=g, max_bounces=4 + 3 * i)
        med = v.make_medium(v.MODE_PT, **med_args)
        img = torch.full((h, w, 4), -1.0, dtype=torch.float32, device=env["dev"])
        out.append(dict(host=host, grid=grid, cam=cam, med=med, med_args=med_args, img=img, spp=spp, seed=seed,
                        ratio=ratio, payload=payload, dims=dims, wh=(w, h), mc=mc, i=i))
    return out


def test_batch_frames_equal_single_renders(env):
    torch, v = env["torch"], env["v"]
    jobs = build_jobs(env)
    structs = [v.make_job(j["grid"], j["cam"], j["med"], j["spp"], j["seed"], j["img"]) for j in jobs]
    b = v.vdbc_batch_create(structs, autotune=False, keep=jobs)
    frames = 3
    v.vdbc_batch_render_frames(b, frames)
    torch.cuda.synchronize()
    st = v.vdbc_batch_stats_get(b)
    assert st.error_flags == 0 and st.paths == sum(j["spp"] * j["wh"][0] * j["wh"][1] for j in jobs)
    for j in jobs:
        single = torch.empty_like(j["img"])
        v.vdbc_render(j["grid"], j["cam"], j["med"], frames * j["spp"], j["seed"], single)
        torch.cuda.synchronize()
        a, s_ = j["img"].cpu().numpy(), single.cpu().numpy()
        # same samples; only the order of the per-pixel sums differs
        assert np.abs(a - s_).max() <= 2e-6 * max(1.0, np.abs(s_).max()), j["i"]
    # reset restarts the accumulation: one frame again equals a single render with spp samples
    v.vdbc_batch_reset(b)
    v.vdbc_batch_render_frames(b, 1)
    torch.cuda.synchronize()
    j = jobs[0]
    single = torch.empty_like(j["img"])
    v.vdbc_render(j["grid"], j["cam"], j["med"], j["spp"], j["seed"], single)
    torch.cuda.synchronize()
    assert np.abs(j["img"].cpu().numpy() - single.cpu().numpy()).max() <= 2e-6
    b.close()


def test_batch_matches_oracle_per_volume(env):
    torch, v, orc = env["torch"], env["v"], env["orc"]
    jobs = build_jobs(env)
    structs = [v.make_job(j["grid"], j["cam"], j["med"], j["spp"], j["seed"], j["img"]) for j in jobs]
    b = v.vdbc_batch_create(structs, autotune=True, keep=jobs)
    t = v.vdbc_batch_get_tuning(b)
    assert t.threads in (128, 256) and t.chunk >= 32 and t.coarse in (0, 1) and t.frame_ms > 0
    assert t.depth in (1, 2) and (t.depth == 1 or t.threads == 256)
    v.vdbc_batch_render_frames(b, 2)
    torch.cuda.synchronize()
    for j in jobs:
        e = orc.encode(j["host"], j["ratio"], payload=j["payload"])
        D = orc.decode_dense(j["host"], e["active"], e["background_bits"], j["payload"])
        mx = orc.macrocell_minmax(D, j["mc"])[1]
        w, h = j["wh"]
        cam_args = env["sc"].pinhole_orbit(j["dims"], w, h, direction=(0.6 - 0.2 * j["i"], 0.4, 0.7))
        ref = orc.render_image(D, mx, orc.make_camera(*cam_args), orc.make_medium(1, macrocell=j["mc"],
                               **j["med_args"]), 2 * j["spp"], j["seed"], threads=8)
        err = np.abs(j["img"].cpu().numpy()[..., :3] - ref[..., :3]).mean(axis=(0, 1))
        assert np.all(err <= PT_MEAN_ABS), (j["i"], err)
    b.close()


def test_batch_rejects_bad_jobs(env):
    torch, v = env["torch"], env["v"]
    jobs = build_jobs(env)[:1]
    j = jobs[0]
    ea = v.make_medium(v.MODE_EA, tf=env["sc"].linear_ramp_tf(), step=0.5)
    with pytest.raises(v.VdbcError) as ex:
        v.vdbc_batch_create([v.make_job(j["grid"], j["cam"], ea, 1, 0, j["img"])], autotune=False, keep=jobs)
    assert ex.value.status == v.ERR_INVALID_ARG
    with pytest.raises(v.VdbcError):
        v.vdbc_batch_create([], autotune=False)


def test_batch_accumulation_state_checkpoint(env):
    """The progressive state (frame counter and per-pixel sums) taken after
    two frames and restored into a fresh batch of the same jobs: three more
    frames there give every job the image of five frames in one batch."""
    torch, v = env["torch"], env["v"]
    jobs = build_jobs(env)
    structs = [v.make_job(j["grid"], j["cam"], j["med"], j["spp"], j["seed"], j["img"]) for j in jobs]
    b = v.vdbc_batch_create(structs, autotune=False, keep=jobs)
    v.vdbc_batch_render_frames(b, 2)
    frame, sums = v.vdbc_batch_get_state(b)
    assert frame == 2 and sums.size == 4 * sum(w * h for (w, h) in (j["wh"] for j in jobs))
    v.vdbc_batch_render_frames(b, 3)
    torch.cuda.synchronize()
    want = [j["img"].cpu().numpy() for j in jobs]
    imgs = [torch.full_like(j["img"], -1.0) for j in jobs]
    structs2 = [v.make_job(j["grid"], j["cam"], j["med"], j["spp"], j["seed"], im) for j, im in zip(jobs, imgs)]
    b2 = v.vdbc_batch_create(structs2, autotune=False, keep=(jobs, imgs))
    v.vdbc_batch_set_state(b2, frame, sums)
    v.vdbc_batch_render_frames(b2, 3)
    torch.cuda.synchronize()
    for w, im in zip(want, imgs):
        assert np.array_equal(w.view(np.uint32), im.cpu().numpy().view(np.uint32))
    assert v.vdbc_batch_get_state(b2)[0] == 5
    with pytest.raises(ValueError):
        v.vdbc_batch_set_state(b2, 0, sums[:-4])
    with pytest.raises(v.VdbcError):
        v.vdbc_batch_set_state(b2, -1, sums)


def test_full_size_batch_frame_equals_single_renders(env, monkeypatch):
    """The batch workload at full size, in the launch configuration the
    benchmark times (32 blob+fBm volumes of edges 64..384, FP16/FP8 leaves at
    1:4..1:20, 256^2..1024^2 images, 4..32 spp; autotuned, graph-replayed): one
    frame gives every job the image of its own single render with the tuner's
    DDA setting, bit for bit, with clean error flags."""
    torch, v, vg, sc = env["torch"], env["v"], env["vg"], env["sc"]
    specs = sc.batch_jobs()
    grids, imgs, structs, views = [], [], [], []
    for sp in specs:
        vol = vg.generate_torch(vg.make_params(sp["kind"], sp["dims"], sp["seed"]))
        g = v.vdbc_encode(vol, sp["ratio"], payload=sp["payload"], macrocell=sp["macrocell"])
        del vol
        cam = v.make_camera(*sc.pinhole_orbit(sp["dims"], sp["width"], sp["height"], direction=sp["direction"]))
        med = v.make_medium(v.MODE_PT, **sp["medium"])
        img = torch.full((sp["height"], sp["width"], 4), -1.0, dtype=torch.float32, device=env["dev"])
        grids.append(g)
        imgs.append(img)
        views.append((cam, med))
        structs.append(v.make_job(g, cam, med, sp["spp"], sp["seed"], img))
    b = v.vdbc_batch_create(structs, autotune=True, keep=(grids, imgs))
    coarse = v.vdbc_batch_get_tuning(b).coarse
    v.vdbc_batch_render_frames(b, 1)
    torch.cuda.synchronize()
    st = v.vdbc_batch_stats_get(b)
    assert st.error_flags == 0 and st.paths == sum(sp["width"] * sp["height"] * sp["spp"] for sp in specs)
    monkeypatch.setenv("VDBC_PT_COARSE", str(int(coarse)))
    one = torch.empty_like(imgs[0])
    for sp, g, img, (cam, med) in zip(specs, grids, imgs, views):
        one = torch.empty_like(img)
        v.vdbc_render(g, cam, med, sp["spp"], sp["seed"], one)
        torch.cuda.synchronize()
        assert np.array_equal(img.cpu().numpy().view(np.uint32), one.cpu().numpy().view(np.uint32)), sp
    b.close()


def test_full_size_batch_per_volume_error_against_oracle(env):
    """The batch workload at full size (the benchmark's 32 volumes, payloads,
    rates, cameras, spp and cells): per volume, 16 sampled pixels of the batch
    frame against the FP64 oracle rendering the same samples on its own
    encode and decode of that volume; mean abs error <= 1e-4 per channel for
    every volume (the per-volume errors are in the assertion message)."""
    torch, v, orc, vg, sc = env["torch"], env["v"], env["orc"], env["vg"], env["sc"]
    specs = sc.batch_jobs()
    hosts, grids, imgs, structs, cams = [], [], [], [], []
    for sp in specs:
        host = vg.generate_host(vg.make_params(sp["kind"], sp["dims"], sp["seed"]))
        g = v.vdbc_encode(torch.from_numpy(host).to(env["dev"]), sp["ratio"], payload=sp["payload"],
                          macrocell=sp["macrocell"])
        cam_args = sc.pinhole_orbit(sp["dims"], sp["width"], sp["height"], direction=sp["direction"])
        img = torch.zeros((sp["height"], sp["width"], 4), dtype=torch.float32, device=env["dev"])
        hosts.append(host)
        grids.append(g)
        imgs.append(img)
        cams.append(cam_args)
        structs.append(v.make_job(g, v.make_camera(*cam_args), v.make_medium(v.MODE_PT, **sp["medium"]),
                                  sp["spp"], sp["seed"], img))
    b = v.vdbc_batch_create(structs, autotune=False, keep=(grids, imgs))
    v.vdbc_batch_render_frames(b, 1)
    torch.cuda.synchronize()
    rng = np.random.default_rng(23)
    errs = []
    for sp, host, img, cam_args in zip(specs, hosts, imgs, cams):
        e = orc.encode(host, sp["ratio"], payload=sp["payload"])
        D = orc.decode_dense(host, e["active"], e["background_bits"], sp["payload"])
        mx = orc.macrocell_minmax(D, sp["macrocell"])[1]
        pix = np.sort(rng.choice(sp["width"] * sp["height"], 16, replace=False))
        ref = orc.render_pixels(D, mx, orc.make_camera(*cam_args),
                                orc.make_medium(1, macrocell=sp["macrocell"], **sp["medium"]),
                                sp["spp"], sp["seed"], pix, threads=8)
        got = img.cpu().numpy().reshape(-1, 4).astype(np.float64)[pix, :3]
        errs.append(float(np.abs(got - ref[:, :3]).mean(axis=0).max()))
    report = ", ".join("%d:%.1e" % (i, x) for i, x in enumerate(errs))
    assert max(errs) <= PT_MEAN_ABS, report
    b.close()
