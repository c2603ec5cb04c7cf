"""Host logic of the serving loop and of bench.py that needs no GPU: request streams, bucket keys,
level counts, admission by the device-memory budget (with a stand-in bucket), and the counting
behind the bench's rooflines."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_levels_and_bins():
    from paper_1308_6634_gb300 import serving
    assert serving.levels_for(1024) == 7 and serving.levels_for(128) == 4 and serving.levels_for(16) == 1
    for n in (128, 256, 512, 1024):
        L = serving.levels_for(n)
        assert n % (1 << (L - 1)) == 0 and n >> (L - 1) == 16  # coarsened down to 16 cells per axis
        b = serving.n_bins_for(n)
        assert b % 2 == 1 and b >= n * math.sqrt(2.0) and b - n * math.sqrt(2.0) < 2


def test_radius_classes_and_bucket_keys():
    from paper_1308_6634_gb300 import serving
    assert serving.r_class(1.5) == 6 and serving.r_class(2.0) == 6 and serving.r_class(2.1) == 9
    assert serving.r_class(5.0) == 15
    with pytest.raises(ValueError):
        serving.r_class(5.1)
    r = serving.Request(rid=0, kind="blur", n=256, reg="tv", T=1e-2, tau=1e-3, n_outer=2, n_inner=3, seed=1,
                        sigma=3.2)
    assert serving.bucket_key(r) == ("blur", 256, 12)
    r2 = serving.Request(rid=1, kind="joseph", n=128, reg="tv", T=1e-2, tau=1e-3, n_outer=2, n_inner=3, seed=1,
                         n_angles=240)
    assert serving.bucket_key(r2) == ("joseph", 128, 240)


def test_stream_is_seeded_poisson_with_the_configured_mix():
    from paper_1308_6634_gb300 import serving
    a = serving.make_stream(2000, rate=200.0, seed=0)
    b = serving.make_stream(2000, rate=200.0, seed=0)
    assert [(r.kind, r.n, r.seed, r.t_arrival) for r in a] == [(r.kind, r.n, r.seed, r.t_arrival) for r in b]
    t = np.array([r.t_arrival for r in a])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0  # mean inter-arrival within 10 %
    kinds = np.array([r.kind == "blur" for r in a])
    assert abs(kinds.mean() - 0.5) < 0.05
    sizes = np.array([r.n for r in a])
    for n, p in zip(serving.SIZES, serving.SIZE_P):
        assert abs(np.mean(sizes == n) - p) < 0.04
    for r in a:
        if r.kind == "blur":
            assert 1.5 <= r.sigma <= 5.0 and r.n_angles == 0
        else:
            assert r.n_angles in serving.ANGLES


def test_bucket_bytes_grow_with_slots():
    from paper_1308_6634_gb300 import serving
    for key in [("blur", 256, 12), ("joseph", 128, 180)]:
        one, four = serving.bucket_bytes(key, 1), serving.bucket_bytes(key, 4)
        assert 0 < one < four


def test_admission_by_budget_releases_idle_buckets(monkeypatch):
    """Buckets are created while the budget allows; when it is full the least recently used idle
    bucket is released, and with no idle bucket the request waits (a refusal is counted)."""
    from paper_1308_6634_gb300 import serving

    class FakeBucket:
        def __init__(self, key, slots, torch):
            self.key, self.slots, self.busy = key, slots, False
            self.last_used = 0.0

        def idle(self):
            return not self.busy

    monkeypatch.setattr(serving, "Bucket", FakeBucket)
    monkeypatch.setattr(serving, "bucket_bytes", lambda key, slots: 100)
    eng = serving.Engine(hbm_budget_bytes=250)
    b1 = eng.bucket(("blur", 128, 6))
    b1.busy = True
    b1.last_used = 1.0
    b2 = eng.bucket(("blur", 128, 9))
    b2.last_used = 2.0
    assert eng.bytes_used == 200 and len(eng.buckets) == 2
    b3 = eng.bucket(("blur", 128, 12))  # full: the idle b2 is released, not the busy b1
    assert b3 is not None and ("blur", 128, 9) not in eng.buckets and ("blur", 128, 6) in eng.buckets
    b3.busy = True
    assert eng.bucket(("joseph", 128, 180)) is None and eng.refused == 1
    assert eng.bucket(("blur", 128, 6)) is b1  # an existing bucket is found, not created


def test_joseph_sample_count_matches_brute_force():
    import bench
    n, na, nb = 12, 6, 19
    c = (n - 1) / 2.0
    brute = 0
    for a in range(na):
        th = a * math.pi / na
        for k in range(nb):
            s = k - (nb - 1) / 2.0
            for q in range(n):
                y = q - c
                if 4 * a < na or 4 * a > 3 * na:
                    u = (s - y * math.sin(th)) / math.cos(th)
                else:
                    u = (s - y * math.cos(th)) / math.sin(th)
                brute += abs(u) <= c
    assert bench.joseph_samples(n, na, nb) == brute


def test_algorithmic_units():
    import bench
    from paper_1308_6634_gb300 import synth
    W = synth.WORKLOADS["deblur1024_fp32"]
    u = bench.alg_units(W)
    # finest V-cycle level, mean of pre (b, kappa in; x, restricted residual out) and post (x_in, b,
    # kappa, coarse correction in; x out): (3.25 + 4.25) / 2 vector words; the reciprocal diagonal
    # the kernels also read is reported beside it, not counted
    assert u["gs_fine"] == pytest.approx(3.75) and u["adj"] == 3.0
    assert bench.beyond_alg_units(W)["gs_fine"] == 1.0
    assert u["fwd"] == pytest.approx((3.0 + 7.0 * 49) / 50)  # the update fused into 49 of 50 forward maps
    assert bench.alg_units(W, kappa_bf16=True)["gs_fine"] == pytest.approx(3.25)
