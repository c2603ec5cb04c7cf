"""Failures made on the host, none of which faults, traps or hangs the GPU: data with a NaN, a
workspace that cannot be allocated, and a bounded device wait that runs out (a barrier whose bytes
never arrive).  Each must come back as a status, and the device must stay usable afterwards."""
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


def _still_usable():
    from paper_1308_6634_gb300 import plsqr
    S = plsqr.Solver((32, 32), "fp32", levels=2)
    S.set_operator("blur", sigma=(1.0, 1.0), radius=(3, 3))
    x = torch.ones((32, 32), dtype=torch.float32, device="cuda")
    y = S.apply_A(x)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all() and abs(float(y[16, 16]) - 1.0) < 1e-5


def test_bounded_wait_runs_out_with_a_timeout_status():
    from paper_1308_6634_gb300 import plsqr
    assert plsqr.selftest_wait(True) == 0
    assert plsqr.selftest_wait(False) == plsqr.E_TIMEOUT
    _still_usable()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nan_in_the_data_is_a_breakdown(prec):
    from paper_1308_6634_gb300 import plsqr
    g = np.random.default_rng(2).standard_normal((64, 64))
    g[10, 20] = np.nan
    S = plsqr.Solver((64, 64), prec, levels=3)
    S.set_operator("blur", sigma=(2.0, 2.0), radius=(6, 6))
    f, info = S.solve(torch.as_tensor(g, dtype=torch.float32 if prec == "fp32" else torch.float64, device="cuda"),
                      "tv", 1e-2, 5e-3, 2, 5)
    torch.cuda.synchronize()
    assert info["status"] == plsqr.E_BREAKDOWN
    assert torch.isfinite(f).all()  # the last complete iterate: f = 0
    _still_usable()


def test_workspace_that_does_not_fit_is_reported():
    from paper_1308_6634_gb300 import plsqr
    with pytest.raises(plsqr.PlsqrError) as e:
        plsqr.Solver((16384, 16384), "fp64", levels=8, max_batch=4096)
    assert e.value.code == plsqr.E_NOMEM
    _still_usable()
