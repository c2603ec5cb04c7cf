"""The whole 2D V-cycle in one cooperative launch against the per-level launches: the tiles run
the same device functions with the same arithmetic per cell, the coarse rows the same dot
products and alpha the same per-tile partial sums in the same order, so the priorconditioner, the
MLSQR iterates and whole solves must agree bit for bit (Sec. 4.2: one fixed symmetric operator,
whatever the schedule)."""
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


def _P():
    from paper_1308_6634_gb300 import plsqr
    return plsqr


def dev(x, prec):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32 if prec == "fp32" else torch.float64,
                           device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _kappa_field(shape, seed=5):
    import oracle as O
    from paper_1308_6634_gb300 import synth
    rng = np.random.default_rng(seed)
    f = synth.phantom_rects_disks(max(shape), 8, 5, seed)[: shape[0], : shape[1]] + 0.01 * rng.standard_normal(shape)
    return O.diffusivity(f, "pm_log", 0.05)[0]


def _tma_rows(shape, levels, prec):
    """Every smoothed level's rows are whole 16-byte units (the cooperative launch stages by TMA)."""
    esz = 8 if prec == "fp64" else 4
    return all(((shape[1] >> l) * esz) % 16 == 0 for l in range(levels))


def _solver(monkeypatch, coop, shape, prec, first_level=0, **kw):
    monkeypatch.setenv("PLSQR_MG_COOP", "1" if coop else "0")
    monkeypatch.setenv("PLSQR_MG_COOP_LEVEL", str(first_level))
    S = _P().Solver(shape, prec, **kw)
    ok = coop and _tma_rows(shape, kw.get("levels", 1), prec)
    assert S.mg_schedule(detail=True) == ((1, first_level, 0) if ok else (0, -1, 0))
    return S


@pytest.mark.parametrize("shape,levels,prec", [((1024, 1024), 6, "fp32"), ((136, 208), 4, "fp32"),
                                               ((136, 208), 4, "fp64"), ((64, 64), 3, "fp64"),
                                               ((32, 48), 2, "fp32"), ((136, 200), 4, "fp32")])
def test_cooperative_vcycle_equals_per_level_launches(monkeypatch, shape, levels, prec):
    """From every first level (the levels above it keep their per-level launches).  136 x 200 has a
    level whose rows are not whole 16-byte units: the cooperative launch is refused there."""
    kappa = _kappa_field(shape)
    b = np.random.default_rng(21).standard_normal(shape)
    S = _solver(monkeypatch, False, shape, prec, levels=levels)
    S.prec_setup(dev(kappa, prec))
    ref = host(S.prec_apply(dev(b, prec)))
    assert np.all(np.isfinite(ref))
    for lc in range(levels - 1):
        S = _solver(monkeypatch, True, shape, prec, first_level=lc, levels=levels)
        S.prec_setup(dev(kappa, prec))
        assert np.array_equal(host(S.prec_apply(dev(b, prec))), ref), lc


@pytest.mark.parametrize("prec,cycles", [("fp32", 1), ("fp64", 2)])
def test_cooperative_solve_batch_equals_per_level_launches(monkeypatch, prec, cycles):
    """Three instances with different regularisers in one batch (tiles of every instance share
    the cooperative grid): f and every history bit for bit.  alpha sums per-tile partials, so both
    handles use the cooperative launch's tile shapes (32 x 32 finest, 16 x 16 coarser)."""
    import oracle as O
    from paper_1308_6634_gb300 import synth
    n = 128
    gs = []
    for seed in range(3):
        f = synth.phantom_rects_disks(n, 8, 5, seed)
        op = O.Operator("blur", (n, n), sigma=(2.0, 2.0), radius=(6, 6))
        gs.append(op.A(f) + 0.01 * np.random.default_rng(seed + 40).standard_normal((n, n)))
    regs, Ts, taus = ["tv", "pm_log", "pm_exp"], [1e-2, 5e-2, 2e-2], [1e-3, 0.0, 5e-3]
    res = []
    for coop, lc in ((False, 0), (True, 0), (True, 1)):
        S = _solver(monkeypatch, coop, (n, n), prec, first_level=lc, levels=4, cycles=cycles, max_batch=3)
        S.set_operator("blur", sigma=(2.0, 2.0), radius=(6, 6))
        S.set_tile_shape(0, 1)
        for l in (1, 2):
            S.set_tile_shape(l, 3)
        fs, infos = S.solve_batch([dev(g, prec) for g in gs], regs, Ts, taus, 3, 12)
        res.append(([host(f) for f in fs], infos))
    for r in res[1:]:
        for k in range(3):
            assert np.array_equal(res[0][0][k], r[0][k])
            for key in ("rbar_hist", "R_hist", "resid_hist"):
                assert np.array_equal(res[0][1][k][key], r[1][k][key], equal_nan=True), key
            assert r[1][k]["status"] == 0


def test_schedule_is_chosen_by_timing_and_unsupported_grids_keep_per_level(monkeypatch):
    monkeypatch.delenv("PLSQR_MG_COOP", raising=False)
    from paper_1308_6634_gb300 import synth
    n = 256
    S = _P().Solver((n, n), "fp32", levels=4)
    S.set_operator("blur", sigma=(2.0, 2.0), radius=(6, 6))
    assert S.mg_schedule() == -1  # not decided before the first solve
    S.solve(dev(synth.phantom_rects_disks(n, 6, 4, 1), "fp32"), "tv", 1e-2, 1e-3, 1, 3)
    coop, lc, cap = S.mg_schedule(detail=True)
    assert coop in (0, 1) and (coop == 0 and lc == -1 or 0 <= lc <= 2) and cap >= 0
    S3 = _P().Solver((16, 16, 16), "fp32", levels=2)
    assert S3.mg_schedule() == 0  # 3D: per-level launches
    monkeypatch.setenv("PLSQR_MG_COOP", "0")
    assert _P().Solver((n, n), "fp32", levels=4).mg_schedule() == 0
