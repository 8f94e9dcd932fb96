"""Host logic of the RANSAC launch-shape autotuner: it picks the fastest
candidate, caches the choice per (device, workload bucket, plan kind) and
does not time again on a cache hit.  GPU timing and the device key are
replaced by fakes, so this runs on the CPU."""
import json

from paper_2402_18008_gb300 import autotune


def _fake(monkeypatch, tmp_path, cost):
    monkeypatch.setenv("ACA_AUTOTUNE_CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(autotune, "_key", lambda device, P, n, k, tag="":
                        f"FakeGPU|152|{autotune._bucket(P, n, k)}" + (f"|{tag}" if tag else ""))
    timed = []

    def time_plan(plan, reps=10):
        timed.append(plan)
        return cost[plan]

    monkeypatch.setattr(autotune, "time_plan", time_plan)
    return timed


CANDS = [dict(block_warps=w, hyps_per_thread=h, tile_points=t) for w, h, t in
         [(4, 1, 256), (4, 4, 2048), (8, 2, 1024), (16, 2, 1024)]]


def _name(c):
    return json.dumps(c, sort_keys=True)


def test_picks_the_fastest_and_caches(monkeypatch, tmp_path):
    cost = {_name(c): ms for c, ms in zip(CANDS, [3.0, 0.7, 1.1, 0.9])}
    timed = _fake(monkeypatch, tmp_path, cost)
    make = lambda **kw: _name(kw)
    best, timings = autotune.tune(make, 512, 1_000_000, 750_000, device=0, candidates=CANDS)
    assert best == CANDS[1]
    assert len(timed) == len(CANDS) and timings[_name(CANDS[1])] == 0.7
    # a second plan of the same bucket reads the cache, times nothing
    best2, _ = autotune.tune(make, 512, 1_000_000, 750_000, device=0, candidates=CANDS)
    assert best2 == best and len(timed) == len(CANDS)
    stored = json.load(open(tmp_path / "autotune.json"))
    assert len(stored) == 1 and list(stored.values())[0]["params"] == CANDS[1]


def test_tags_and_buckets_keep_separate_entries(monkeypatch, tmp_path):
    cost = {_name(c): ms for c, ms in zip(CANDS, [0.5, 0.7, 1.1, 0.9])}
    timed = _fake(monkeypatch, tmp_path, cost)
    make = lambda **kw: _name(kw)
    autotune.tune(make, 512, 1_000_000, 750_000, device=0, candidates=CANDS)
    autotune.tune(make, 512, 1_000_000, 750_000, device=0, candidates=CANDS, tag="adaptive")
    autotune.tune(make, 1, 2000, 4096, device=0, candidates=CANDS)
    assert len(timed) == 3 * len(CANDS)
    keys = sorted(json.load(open(tmp_path / "autotune.json")))
    assert len(keys) == 3 and sum(k.endswith("|adaptive") for k in keys) == 1
    # use_cache=False always times
    autotune.tune(make, 1, 2000, 4096, device=0, candidates=CANDS, use_cache=False)
    assert len(timed) == 4 * len(CANDS)


def test_bucket_rounds_to_powers_of_two():
    assert autotune._bucket(512, 512 * 2000, 512 * 1400) == "P9-N11-K10"
    assert autotune._bucket(500, 500 * 2100, 500 * 1500) == "P9-N11-K11"
    assert autotune._bucket(0, 0, 0) == "P0-N0-K0"
    # the default candidates respect the launch limits the library checks
    for c in autotune.CANDIDATES:
        assert c["hyps_per_thread"] <= c["block_warps"] <= 16 and c["tile_points"] % 32 == 0
