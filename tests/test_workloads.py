"""The synthetic workload recipes the benchmark and the full-size tests use:
shapes, rates, payloads, image sizes and samples as stated, and the batch
drawn deterministically from its seed."""
from volgen import scenes


def test_benchmark_scenes():
    t = scenes.TURBULENCE_512
    assert t["dims"] == (512, 512, 512) and t["ratio"] == 10.0 and (t["width"], t["height"], t["spp"]) == (1024, 1024, 16)
    assert t["medium"]["albedo"] == 0.9 and t["medium"]["g"] == 0.6 and t["medium"]["max_bounces"] == 16
    assert t["medium"]["density_scale"] == 20.0 and (t["macrocell"], t["texture_macrocell"]) == (56, 64)
    c = scenes.CLOUD_994
    assert c["dims"] == (994, 676, 1225) and c["ratio"] == 10.0 and (c["width"], c["height"], c["spp"]) == (1920, 1080, 32)
    assert c["medium"]["albedo"] == 0.95 and c["medium"]["g"] == 0.8
    f = scenes.CLOUD_1987
    assert f["dims"] == (1987, 1351, 2449) and f["ratio"] == 10.0 and (f["width"], f["height"], f["spp"]) == (1920, 1080, 64)
    assert f["medium"]["albedo"] == 0.95 and f["medium"]["g"] == 0.8 and f["medium"]["max_bounces"] == 32
    assert f["kind"] == c["kind"] and (f["macrocell"], f["texture_macrocell"]) == (128, 128)
    e = scenes.BLOBS_64_EA
    assert e["dims"] == (64, 64, 64) and e["ratio"] == 4.0 and (e["width"], e["height"]) == (128, 128) and e["step"] == 0.5


def test_batch_recipe_and_determinism():
    jobs = scenes.batch_jobs()
    assert len(jobs) == 32 and jobs == scenes.batch_jobs()
    assert scenes.batch_jobs(seed=1) != jobs
    for j in jobs:
        assert all(64 <= d <= 384 for d in j["dims"])
        assert j["ratio"] in (4.0, 6.0, 10.0, 20.0) and j["payload"] in (1, 2)
        assert j["width"] == j["height"] and 256 <= j["width"] <= 1024 and 4 <= j["spp"] <= 32
        assert j["macrocell"] == scenes.BATCH_MACROCELL
    assert {j["payload"] for j in jobs} == {1, 2}                 # both payload groups present
    assert len({j["seed"] for j in jobs}) == 32
