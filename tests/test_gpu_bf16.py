"""The bfloat16-kappa variant: kappa kept in bfloat16, widened to float by the finest V-cycle
level and the first coarsening.  Its results are compared twice, as the variant is a different
priorconditioner and not only different arithmetic: with the oracle fed the same rounded kappa
(tight), and with the plain oracle (the size of the change)."""
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


def _kappa(shape, seed=5):
    import oracle as O
    from paper_1308_6634_gb300 import synth
    rng = np.random.default_rng(seed)
    f = synth.phantom_rects_disks(max(shape), 8, 5, seed)[: shape[0], : shape[1]] + 0.01 * rng.standard_normal(shape)
    return O.diffusivity(f, "pm_log", 0.05)[0]


@pytest.mark.parametrize("shape,levels", [((256, 256), 4), ((136, 200), 4), ((64, 64), 3)])
def test_priorconditioner_with_bf16_kappa(shape, levels):
    import oracle as O
    from paper_1308_6634_gb300 import plsqr
    kappa = _kappa(shape)
    kr = np.vectorize(O.round_bf16)(kappa)
    b = np.random.default_rng(6).standard_normal(shape)
    S = plsqr.Solver(shape, "fp32", levels=levels)
    S.set_kappa_bf16(True)
    S.prec_setup(torch.as_tensor(kappa, dtype=torch.float32, device="cuda"))
    got = S.prec_apply(torch.as_tensor(b, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    same = O.Multigrid(kr, levels, 2, 1).apply(b)
    plain = O.Multigrid(kappa, levels, 2, 1).apply(b)
    print(shape, "vs rounded-kappa oracle", _rel(got, same), "vs plain oracle", _rel(got, plain))
    assert _rel(got, same) < 1e-4
    assert _rel(got, plain) < 2e-2


def test_mlsqr_with_bf16_kappa():
    """Four MLSQR iterations (before rounding chaos: on this problem the float32 model of the
    iteration already departs from double by 2e-6 at the sixth) with the V-cycle of a structured
    kappa: against the oracle's MLSQR with the V-cycle of the same rounded kappa."""
    import oracle as O
    from paper_1308_6634_gb300 import plsqr, synth
    n = 128
    f = synth.phantom_rects_disks(n, 10, 6, 1)
    op = O.Operator("blur", (n, n), sigma=(3.0, 3.0), radius=(9, 9))
    g = synth.add_noise(op.A(f), 0.01, synth.standard_noise((n, n), 2))
    kappa = _kappa((n, n), 7)
    kr = np.vectorize(O.round_bf16)(kappa)
    f_same, h_same, _ = O.mlsqr(op, g, 1e-3, 4, prec=O.Multigrid(kr, 4, 2, 1))
    f_plain, h_plain, _ = O.mlsqr(op, g, 1e-3, 4, prec=O.Multigrid(kappa, 4, 2, 1))
    S = plsqr.Solver((n, n), "fp32", levels=4)
    S.set_operator("blur", sigma=(3.0, 3.0), radius=(9, 9))
    S.set_kappa_bf16(True)
    S.prec_setup(torch.as_tensor(kappa, dtype=torch.float32, device="cuda"))
    fg, hg, rc = S.mlsqr(torch.as_tensor(g, dtype=torch.float32, device="cuda"), 1e-3, 4)
    fg = fg.double().cpu().numpy()
    print("f vs rounded-kappa oracle", _rel(fg, f_same), "vs plain oracle", _rel(fg, f_plain))
    assert rc == 0
    assert _rel(hg, h_same) < 1e-5
    assert _rel(fg, f_same) < 1e-4


def test_first_outer_step_equals_float_kappa():
    """kappa(0) = 1 for the first outer step is exact in bfloat16, so that step is bit for bit the
    float-kappa one; the later steps differ by the rounding of kappa only."""
    from paper_1308_6634_gb300 import plsqr, synth
    n = 128
    f = synth.phantom_rects_disks(n, 10, 6, 1)
    g = torch.as_tensor(f, dtype=torch.float32, device="cuda")
    outs = []
    for kb in (False, True):
        S = plsqr.Solver((n, n), "fp32", levels=4)
        S.set_operator("blur", sigma=(3.0, 3.0), radius=(9, 9))
        S.set_kappa_bf16(kb)
        outs.append(S.solve(S.apply_A(g), "pm_log", 5e-2, 1e-3, 3, 8))
    (f0, i0), (f1, i1) = outs
    assert i1["status"] == 0 and torch.isfinite(f1).all()
    assert np.array_equal(i0["rbar_hist"][0], i1["rbar_hist"][0])
    assert not np.array_equal(i0["rbar_hist"][1], i1["rbar_hist"][1])


def test_bf16_kappa_rejected_where_not_built():
    from paper_1308_6634_gb300 import plsqr
    for shape, prec, levels, cycles in [((16, 16, 16), "fp32", 2, 1), ((64, 64), "fp64", 3, 1),
                                        ((64, 64), "fp32", 1, 1), ((64, 64), "fp32", 3, 2)]:
        S = plsqr.Solver(shape, prec, levels=levels, cycles=cycles)
        with pytest.raises(plsqr.PlsqrError) as e:
            S.set_kappa_bf16(True)
        assert e.value.code == plsqr.E_INVALID
