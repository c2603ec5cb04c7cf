"""Slots and the continuous-batching serving loop.

A slot of a serving handle runs Algorithm 3 one lagged-diffusivity step at a time; its
arithmetic is that of a one-instance solve (instances of a launch never mix), so a request must
give the same result alone and in any mix of other requests, buckets and arrival times.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_6634_gb300 import build
    build.build()


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64).ravel(), np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _deblur_data(n, sigma, R, seed):
    from paper_1308_6634_gb300 import plsqr, synth
    f = synth.phantom_rects_disks(n, 6, 4, seed)
    x = torch.as_tensor(f, dtype=torch.float32, device="cuda")
    Af = plsqr.plsqr_blur_noalloc(x, (sigma, sigma), (R, R))
    z = torch.as_tensor(synth.standard_noise((n, n), seed + 1), device="cuda")
    return (Af.double() + 0.01 * float(Af.double().norm()) / n * z).float().contiguous()


@pytest.mark.parametrize("per_slot_sigma", [False, True])
def test_slot_steps_equal_one_instance_solve(per_slot_sigma):
    """n_outer plsqr_step calls on one slot (the other slots empty) reproduce plsqr_solve on a
    one-instance handle bit for bit; with a per-slot sigma equal to the operator's (ceil(3 sigma)
    = radius) the per-slot taps equal the operator's taps."""
    from paper_1308_6634_gb300 import plsqr
    n, sigma, R, n_outer, n_inner = 96, 4.0, 12, 3, 8
    g = _deblur_data(n, sigma, R, 3)
    S1 = plsqr.Solver((n, n), "fp32", levels=3, max_batch=1)
    S1.set_operator("blur", sigma=(sigma, sigma), radius=(R, R))
    f1, info1 = S1.solve(g, "pm_log", 5e-2, 1e-3, n_outer, n_inner)
    S = plsqr.Solver((n, n), "fp32", levels=3, max_batch=4)
    S.set_operator("blur", sigma=(sigma, sigma), radius=(R, R))
    S.slot_start(2, g, "pm_log", 5e-2, 1e-3, n_outer, n_inner, sigma=(sigma, sigma) if per_slot_sigma else None)
    for _ in range(n_outer):
        S.step()
    f2, info2 = S.slot_finish(2, n_outer, n_inner)
    torch.cuda.synchronize()
    assert info2["status"] == 0
    assert torch.equal(f1, f2)
    assert np.array_equal(info1["rbar_hist"], info2["rbar_hist"])
    assert np.array_equal(info1["resid_hist"], info2["resid_hist"])
    assert np.allclose(info1["R_hist"], info2["R_hist"], rtol=0, atol=0, equal_nan=True)


def test_slot_with_own_sigma_matches_oracle():
    """A slot with sigma 2.3 (support ceil(6.9) = 7, zero-padded to the handle's radius 9) against
    the oracle's blur of radius 7: the first residual estimates before rounding chaos."""
    import oracle as O
    from paper_1308_6634_gb300 import plsqr, synth
    n, sigma = 64, 2.3
    f = synth.phantom_rects_disks(n, 6, 4, 5)
    op = O.Operator("blur", (n, n), sigma=(sigma, sigma), radius=(7, 7))
    g = synth.add_noise(op.A(f), 0.01, synth.standard_noise((n, n), 6))
    ref = O.solve(op, g, "tv", 1e-2, 1e-3, 1, 5, 3, 2, 1)
    S = plsqr.Solver((n, n), "fp32", levels=3, max_batch=2)
    S.set_operator("blur", sigma=(3.0, 3.0), radius=(9, 9))
    S.slot_start(1, torch.as_tensor(g, dtype=torch.float32, device="cuda"), "tv", 1e-2, 1e-3, 1, 5,
                 sigma=(sigma, sigma))
    S.step()
    fs, info = S.slot_finish(1, 1, 5)
    assert _rel(info["rbar_hist"][0], ref["rbar_hist"][0]) < 1e-4
    assert _rel(fs.double().cpu().numpy(), ref["f"]) < 1e-3


def test_slot_api_errors():
    from paper_1308_6634_gb300 import plsqr
    n = 64
    S = plsqr.Solver((n, n), "fp32", levels=3, max_batch=2)
    S.set_operator("blur", sigma=(2.0, 2.0), radius=(6, 6))
    g = torch.zeros((n, n), dtype=torch.float32, device="cuda") + 1.0
    with pytest.raises(plsqr.PlsqrError) as e:
        S.slot_start(2, g, "tv", 1e-2, 0.0, 2, 4)            # no such slot
    assert e.value.code == plsqr.E_INVALID
    with pytest.raises(plsqr.PlsqrError) as e:
        S.slot_start(0, g, "tv", 1e-2, 0.0, 2, 4, sigma=(2.5, 2.5))   # ceil(7.5) = 8 > radius 6
    assert e.value.code == plsqr.E_INVALID
    S.slot_start(0, g, "tv", 1e-2, 0.0, 2, 4)
    with pytest.raises(plsqr.PlsqrError) as e:
        S.slot_start(0, g, "tv", 1e-2, 0.0, 2, 4)             # busy
    assert e.value.code == plsqr.E_STATE
    with pytest.raises(plsqr.PlsqrError) as e:
        S.slot_start(1, g, "tv", 1e-2, 0.0, 2, 5)             # different n_inner
    assert e.value.code == plsqr.E_INVALID
    with pytest.raises(plsqr.PlsqrError) as e:
        S.solve(g, "tv", 1e-2, 0.0, 2, 4)                     # slot mode
    assert e.value.code == plsqr.E_STATE
    # the single-operation entry points would use the slots' state and scratch vectors
    for call in (lambda: S.apply_A(g), lambda: S.apply_At(g), lambda: S.diffusivity(g, "tv", 1e-2),
                 lambda: S.prec_setup(g), lambda: S.prec_apply(g), lambda: S.apply_M(g),
                 lambda: S.mlsqr(g, 0.0, 3)):
        with pytest.raises(plsqr.PlsqrError) as e:
            call()
        assert e.value.code == plsqr.E_STATE
    S.step()
    S.step()
    S.step()  # the slot has reached its target: nothing left to run
    f, info = S.slot_finish(0, 2, 4)
    assert info["status"] == 0 and torch.isfinite(f).all()
    with pytest.raises(plsqr.PlsqrError) as e:
        S.slot_finish(0, 2, 4)                                # not running
    assert e.value.code == plsqr.E_STATE


def test_each_result_is_the_same_alone_and_in_the_mix():
    """A stream of deblurring and tomography requests of two sizes, different blur widths,
    regularisers and angle counts, arriving while others run (continuous batching over several
    buckets whose steps overlap on the device), against each request served alone."""
    from paper_1308_6634_gb300 import serving
    reqs = serving.make_stream(14, rate=400.0, seed=3, n_outer=3, n_inner=6, sizes=(64, 128), size_p=(0.5, 0.5),
                               angles=(60, 90))
    data = {r.rid: serving.make_data(r, torch, torch.device("cuda"))[0] for r in reqs}
    eng = serving.Engine(keep_results=True, slots_for_size={64: 4, 128: 2})
    eng.run(reqs, data)
    mixed = eng.results()
    summary = serving.summarize(reqs)
    assert summary["requests"] == 14 and summary["breakdowns"] == 0
    assert len({r.bucket for r in reqs}) >= 3
    assert max(b.steps for b in eng.buckets.values()) > 3  # some bucket admitted requests mid-run
    for r in reqs:
        alone = serving.Engine(keep_results=True, slots_for_size={64: 4, 128: 2})
        r2 = serving.Request(**{k: getattr(r, k) for k in ("rid", "kind", "n", "reg", "T", "tau", "n_outer",
                                                            "n_inner", "seed", "sigma", "n_angles")})
        alone.run([r2], data, realtime=False)
        f_alone, info_alone = alone.results()[r.rid]
        f_mix, info_mix = mixed[r.rid]
        assert torch.equal(f_alone, f_mix), r
        assert np.array_equal(info_alone["rbar_hist"], info_mix["rbar_hist"]), r


def test_admission_waits_for_memory():
    """With a budget that holds one bucket, requests of a second bucket wait until the first is
    idle and released, and all complete."""
    from paper_1308_6634_gb300 import serving
    reqs = serving.make_stream(6, rate=1000.0, seed=4, n_outer=2, n_inner=4, sizes=(64,), size_p=(1.0,),
                               angles=(60,))
    data = {r.rid: serving.make_data(r, torch, torch.device("cuda"))[0] for r in reqs}
    keys = {serving.bucket_key(r) for r in reqs}
    one = max(serving.bucket_bytes(k, 4) for k in keys)
    eng = serving.Engine(hbm_budget_bytes=one, slots_for_size={64: 4})
    eng.run(reqs, data)
    assert all(np.isfinite(r.t_done) for r in reqs)
    assert len(eng.buckets) == 1


def test_outer_stop_frees_the_slot_early_with_the_solo_result():
    """A request carrying the outer stopping rule (Algorithm 3 step 5: R fell by less than r_rel)
    is reported stopped (state 2) once the step that stopped it is done, leaves its slot before its
    n_outer steps, and its f and histories are those of plsqr_solve alone with the same rule."""
    from paper_1308_6634_gb300 import plsqr, serving
    n, sigma, R, n_outer, n_inner, r_rel = 96, 4.0, 12, 12, 8, 0.05
    g = _deblur_data(n, sigma, R, 5)
    S1 = plsqr.Solver((n, n), "fp32", levels=3, max_batch=1)
    S1.set_operator("blur", sigma=(sigma, sigma), radius=(R, R))
    S1.set_stopping(r_rel=r_rel)
    f1, info1 = S1.solve(g, "pm_log", 5e-2, 1e-3, n_outer, n_inner)
    rows = int(np.sum(np.isfinite(info1["rbar_hist"][:, 0])))
    assert 2 <= rows < n_outer  # the rule stopped the solve early
    # the slot API: the slot reports the stop and its result is the solo one
    S = plsqr.Solver((n, n), "fp32", levels=3, max_batch=4)
    S.set_operator("blur", sigma=(sigma, sigma), radius=(R, R))
    S.set_stopping(r_rel=r_rel, index=1)
    S.slot_start(1, g, "pm_log", 5e-2, 1e-3, n_outer, n_inner)
    steps = 0
    while True:
        S.step()
        steps += 1
        torch.cuda.synchronize()
        k, state = S.slot_progress(1)
        if state == 2 or k >= n_outer:
            break
    assert state == 2 and steps < n_outer
    f2, info2 = S.slot_finish(1, n_outer, n_inner)
    torch.cuda.synchronize()
    assert torch.equal(f1, f2)
    assert np.array_equal(info1["rbar_hist"][:rows], info2["rbar_hist"][:rows])
    # the engine frees the slot early and keeps the result
    req = serving.Request(rid=0, kind="blur", n=n, reg="pm_log", T=5e-2, tau=1e-3, n_outer=n_outer,
                          n_inner=n_inner, seed=5, sigma=sigma, r_rel=r_rel)
    eng = serving.Engine(keep_results=True, slots_for_size={n: 4})
    eng.run([req], {0: g}, realtime=False)
    f3, _ = eng.results()[0]
    b = next(iter(eng.buckets.values()))
    assert b.steps < n_outer
    assert torch.equal(f1, f3)


def test_slot_history_regrowth_keeps_per_slot_taps():
    """A slot started on an idle handle with a longer history than before regrows the shared
    history storage; the per-slot blur taps (pinned host staging) stay valid through it, and the
    second request still equals its one-instance solve."""
    from paper_1308_6634_gb300 import plsqr
    n, sigma, R = 96, 4.0, 12
    g = _deblur_data(n, sigma, R, 5)
    S = plsqr.Solver((n, n), "fp32", levels=3, max_batch=2)
    S.set_operator("blur", sigma=(sigma, sigma), radius=(R, R))
    S.slot_start(0, g, "tv", 1e-2, 1e-3, 1, 4, sigma=(sigma, sigma))
    S.step()
    S.slot_finish(0, 1, 4)
    S.slot_start(1, g, "pm_log", 5e-2, 1e-3, 3, 8, sigma=(sigma, sigma))   # longer history: regrown
    for _ in range(3):
        S.step()
    f2, info2 = S.slot_finish(1, 3, 8)
    S1 = plsqr.Solver((n, n), "fp32", levels=3, max_batch=1)
    S1.set_operator("blur", sigma=(sigma, sigma), radius=(R, R))
    f1, info1 = S1.solve(g, "pm_log", 5e-2, 1e-3, 3, 8)
    torch.cuda.synchronize()
    assert info2["status"] == 0
    assert torch.equal(f1, f2)
    assert np.array_equal(info1["rbar_hist"], info2["rbar_hist"])
    S.close()


@pytest.mark.parametrize("per_slot_sigma,stop", [(False, False), (True, False), (False, True)])
def test_checkpoint_resume_equals_uninterrupted_solve(per_slot_sigma, stop):
    """A request saved after k outer steps (plsqr_slot_save) and restored into another slot of
    another handle (plsqr_slot_restore: other max_batch, other slot index, a running neighbour)
    finishes with f and histories bit for bit those of the uninterrupted run: between outer steps
    of Algorithm 3 the state is f^k with its scalars and histories.  With the outer stopping rule
    on, the rule compares R(f^k) with the saved R(f^{k-1})."""
    from paper_1308_6634_gb300 import plsqr
    n, sigma, R, n_outer, n_inner, k = 96, 4.0, 12, 4, 6, 2
    g = _deblur_data(n, sigma, R, 7)
    sg = (3.5, 3.5) if per_slot_sigma else None

    def handle(B):
        S = plsqr.Solver((n, n), "fp32", levels=3, max_batch=B)
        S.set_operator("blur", sigma=(sigma, sigma), radius=(R, R))
        if stop:
            S.set_stopping(0.0, 0.0, 0.05)
        return S

    S1 = handle(2)
    S1.slot_start(0, g, "pm_log", 5e-2, 1e-3, n_outer, n_inner, sigma=sg)
    for _ in range(n_outer):
        S1.step()
    f1, info1 = S1.slot_finish(0, n_outer, n_inner)
    S2 = handle(2)
    S2.slot_start(1, g, "pm_log", 5e-2, 1e-3, n_outer, n_inner, sigma=sg)
    for _ in range(k):
        S2.step()
    ck = S2.slot_save(1)
    assert len(ck) == plsqr.lib().plsqr_slot_state_bytes(S2.h)
    S3 = handle(3)
    other = _deblur_data(n, sigma, R, 9)
    S3.slot_start(0, other, "tv", 1e-2, 1e-3, n_outer, n_inner)
    S3.step()
    S3.slot_restore(2, ck, n_outer, n_inner)
    assert S3.slot_progress(2)[0] == k
    for _ in range(n_outer - k):
        S3.step()
    f3, info3 = S3.slot_finish(2, n_outer, n_inner)
    S3.slot_finish(0, n_outer, n_inner)
    torch.cuda.synchronize()
    assert info3["status"] == info1["status"]
    assert torch.equal(f1, f3)
    for key in ("rbar_hist", "R_hist", "resid_hist"):
        assert np.array_equal(info1[key], info3[key], equal_nan=True), key


def test_checkpoint_restore_refusals():
    """plsqr_slot_restore refuses a buffer that is not a checkpoint, one that is truncated, one of
    another grid, and a busy slot, and leaves the handle usable."""
    from paper_1308_6634_gb300 import plsqr
    n, sigma, R = 64, 3.0, 9
    g = _deblur_data(n, sigma, R, 11)
    S = plsqr.Solver((n, n), "fp32", levels=3, max_batch=2)
    S.set_operator("blur", sigma=(sigma, sigma), radius=(R, R))
    S.slot_start(0, g, "tv", 1e-2, 1e-3, 2, 4)
    S.step()
    ck = S.slot_save(0)
    with pytest.raises(plsqr.PlsqrError) as e:
        S.slot_restore(1, b"\0" * len(ck), 2, 4)
    assert e.value.code == plsqr.E_INVALID
    with pytest.raises(plsqr.PlsqrError) as e:
        S.slot_restore(1, ck[: len(ck) // 2], 2, 4)
    assert e.value.code == plsqr.E_INVALID
    with pytest.raises(plsqr.PlsqrError):
        S.slot_restore(0, ck, 2, 4)  # busy
    T = plsqr.Solver((2 * n, n), "fp32", levels=3, max_batch=1)
    T.set_operator("blur", sigma=(sigma, sigma), radius=(R, R))
    with pytest.raises(plsqr.PlsqrError) as e:
        T.slot_restore(0, ck, 2, 4)
    assert e.value.code == plsqr.E_INVALID
    S.slot_restore(1, ck, 2, 4)
    S.step()
    fa, ia = S.slot_finish(0, 2, 4)
    fb, ib = S.slot_finish(1, 2, 4)
    torch.cuda.synchronize()
    assert torch.equal(fa, fb)
