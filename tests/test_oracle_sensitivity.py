"""Rounding sensitivity of the method itself (evidence behind the long-horizon parity
tolerances) and a check that the test-side FP32 rounding model runs the oracle's algorithm.

Sec. 2.1 notes that priorconditioning does not cluster eigenvalues and can raise the
condition number; in finite precision this makes the MLSQR iterates after a few tens of
iterations sensitive to rounding (loss of orthogonality), while plain LSQR on the same
blur stays stable much longer."""
import numpy as np

import oracle as O
from envelope import fp32_model_mlsqr, problem, rel
from paper_1308_6634_gb300 import synth


def test_priorconditioned_iterates_are_rounding_sensitive():
    W = synth.WORKLOADS["deblur64_fp64"]
    op, g, _ = problem(W)
    ref = O.solve(op, g, W.reg, W.T, W.tau, W.n_outer, W.n_inner, W.levels, W.nu, W.cycles)
    gp = g * (1 + 1e-16 * np.random.default_rng(1).standard_normal(g.shape))
    pert = O.solve(op, gp, W.reg, W.T, W.tau, W.n_outer, W.n_inner, W.levels, W.nu, W.cycles)
    # a perturbation at the unit roundoff of double moves the 10 x 30 result by > 1e-5
    assert rel(pert["f"], ref["f"]) > 1e-5
    assert rel(pert["rbar_hist"], ref["rbar_hist"]) > 1e-5
    # ... but not the first iterations of the first outer step
    assert rel(pert["rbar_hist"][0][:5], ref["rbar_hist"][0][:5]) < 1e-13


def test_fp32_model_without_rounding_is_the_oracle():
    W = synth.WORKLOADS["deblur64_fp64"]
    op, g, _ = problem(W)
    kappa = O.diffusivity(W.phantom_image(0), W.reg, W.T)[0]
    mg = O.Multigrid(kappa, W.levels, W.nu, W.cycles)
    for tau in (0.0, W.tau):
        f_ref, h_ref, _ = O.mlsqr(op, g, tau, 6, prec=mg)
        f, h = fp32_model_mlsqr(op, mg, g, tau, 6, _r32=lambda x: x)
        assert rel(f, f_ref) < 1e-10 and rel(h, h_ref) < 1e-12
        f32, h32 = fp32_model_mlsqr(op, mg, g, tau, 6)
        assert 1e-9 < rel(h32, h_ref) < 1e-4
