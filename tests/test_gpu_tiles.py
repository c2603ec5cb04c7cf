"""Tile shapes of the 2D V-cycle and their autotuner: every compiled shape must give the same
priorconditioner bit for bit (the same arithmetic per cell in the same order; only the schedule
differs), so a tuned handle solves exactly like an untuned one."""
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

N_COARSE = 6  # shapes 0..5 of the coarser levels
N_FINE = 6    # shapes 0..5 of the finest level


@pytest.mark.parametrize("shape,levels,prec", [((1024, 1024), 6, "fp32"), ((136, 200), 4, "fp32"),
                                               ((136, 200), 4, "fp64"), ((64, 64), 3, "fp64"),
                                               ((32, 48), 2, "fp32")])
def test_every_tile_shape_gives_the_same_vcycle(shape, levels, prec):
    kappa = _kappa_field(shape)
    b = np.random.default_rng(21).standard_normal(shape)
    S = _P().Solver(shape, prec, levels=levels)
    S.prec_setup(dev(kappa, prec))
    ref = host(S.prec_apply(dev(b, prec)))
    assert np.all(np.isfinite(ref))
    for fine in range(N_FINE):
        for coarse in range(N_COARSE):
            S.set_tile_shape(0, fine)
            for l in range(1, levels - 1):
                S.set_tile_shape(l, coarse)
            got = host(S.prec_apply(dev(b, prec)))
            assert np.array_equal(got, ref), (fine, coarse)


def test_tile_shape_queries_and_invalid_shapes():
    S = _P().Solver((256, 256), "fp32", levels=4)
    assert S.tile_shape(0)[1:] == (64, 32, 256)   # the defaults before any tuning
    assert S.tile_shape(1)[1:] == (64, 32, 1024)
    assert S.tile_shape(3)[0] == -1               # the coarsest level is the exact solve
    S.set_tile_shape(1, 3)
    assert S.tile_shape(1) == (3, 16, 16, 256)
    for lv, sh in [(0, N_FINE), (1, N_COARSE), (3, 0), (-1, 0)]:
        with pytest.raises(RuntimeError):
            S.set_tile_shape(lv, sh)
    S3 = _P().Solver((16, 16, 16), "fp32", levels=2)
    assert S3.tile_shape(0) == (1, 1, 1, 256)      # 3D: one plane per thread before any tuning
    S3.set_tile_shape(0, 4)
    assert S3.tile_shape(0) == (4, 1, 4, 256)
    for sh in (0, 3, 8):
        with pytest.raises(RuntimeError):
            S3.set_tile_shape(0, sh)
    assert S3.tile_shape(1)[0] == -1               # the coarsest level is the exact solve


@pytest.mark.parametrize("shape,levels,prec", [((40, 24, 56), 3, "fp32"), ((24, 24, 24), 4, "fp64"),
                                               ((12, 20, 8), 2, "fp32")])
def test_every_plane_count_gives_the_same_3d_vcycle(shape, levels, prec):
    """The 3D half sweeps with 1, 2 or 4 planes per thread on every level (ragged last chunk of
    planes included): the V-cycle is bit for bit the same."""
    import oracle as O
    from paper_1308_6634_gb300 import synth
    rng = np.random.default_rng(23)
    f = synth.phantom_ellipsoids(shape, 6, 5) + 0.01 * rng.standard_normal(shape)
    kappa = O.diffusivity(f, "tv", 1e-2)[0]
    b = rng.standard_normal(shape)
    S = _P().Solver(shape, prec, levels=levels, cycles=2)
    S.prec_setup(dev(kappa, prec))
    for l in range(levels - 1):
        S.set_tile_shape(l, 1)
    ref = host(S.prec_apply(dev(b, prec)))
    assert np.all(np.isfinite(ref))
    for zc in (2, 4):
        for l in range(levels - 1):
            S.set_tile_shape(l, zc)
        assert np.array_equal(host(S.prec_apply(dev(b, prec))), ref), zc


def test_autotuned_solve_equals_default_shapes(monkeypatch):
    """The first solve tunes the shapes; the solve is bit for bit the one with the default shapes."""
    import oracle as O
    from paper_1308_6634_gb300 import synth
    n = 256
    f = synth.phantom_rects_disks(n, 10, 6, 3)
    op = O.Operator("blur", (n, n), sigma=(3.0, 3.0), radius=(9, 9))
    g = op.A(f) + 0.01 * np.random.default_rng(4).standard_normal((n, n))
    outs, shapes = [], []
    for tune in ("1", "0"):
        monkeypatch.setenv("PLSQR_AUTOTUNE", tune)
        S = _P().Solver((n, n), "fp32", levels=4)
        S.set_operator("blur", sigma=(3.0, 3.0), radius=(9, 9))
        r = S.solve(dev(g, "fp32"), "tv", 1e-2, 1e-3, 3, 10)
        outs.append(host(r[0] if isinstance(r, tuple) else r))
        shapes.append([S.tile_shape(l) for l in range(3)])
    assert np.array_equal(outs[0], outs[1])
    assert all(s[0] == 0 for s in shapes[1])
    for l, (sid, tx, ty, nth) in enumerate(shapes[0]):
        assert 0 <= sid < (N_FINE if l == 0 else N_COARSE) and tx > 0 and ty > 0 and nth > 0


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_explicit_autotune_keeps_the_hierarchy(prec):
    """plsqr_autotune between plsqr_prec_setup and plsqr_prec_apply times the kernels on the
    handle's buffers; the hierarchy it reads must come out unchanged."""
    shape, levels = (256, 256), 4
    kappa = _kappa_field(shape)
    b = np.random.default_rng(22).standard_normal(shape)
    S = _P().Solver(shape, prec, levels=levels)
    S.prec_setup(dev(kappa, prec))
    ref = host(S.prec_apply(dev(b, prec)))
    S.autotune(fresh=True)
    got = host(S.prec_apply(dev(b, prec)))
    assert np.array_equal(got, ref)


def test_explicit_shapes_survive_a_kappa_storage_change():
    """Shapes set by plsqr_set_tile_shape are kept when the kappa storage changes; the solve
    with bfloat16 kappa then runs with them instead of tuning again."""
    from paper_1308_6634_gb300 import synth
    n = 128
    g = synth.phantom_rects_disks(n, 6, 4, 2)
    S = _P().Solver((n, n), "fp32", levels=3)
    S.set_operator("blur", sigma=(2.0, 2.0), radius=(6, 6))
    S.set_tile_shape(0, 2)
    S.set_tile_shape(1, 5)
    S.set_kappa_bf16(True)
    S.solve(dev(g, "fp32"), "tv", 1e-2, 1e-3, 2, 4)
    assert S.tile_shape(0)[0] == 2 and S.tile_shape(1)[0] == 5
