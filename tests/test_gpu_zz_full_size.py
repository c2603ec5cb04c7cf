"""Parity at the full sizes of the 192^3 inpainting and 512^2 tomography workloads, in the launch
configuration the benchmark times (one instance, the workload's levels, sweeps and cycles).

The oracle computes these outputs whole in seconds: the forward and adjoint maps on the
workload's own data, the diffusivity, the V-cycle and M_f from a structured kappa, and the first
MLSQR iterations with that V-cycle (before rounding chaos, §2.1).  The 1024^2 deblurring workload
has its own full-size test beside the other parity tests.  This file is collected after them
because it is the slowest (the 192^3 phantom and oracle iterations take tens of seconds).

Tolerances are those of the smaller parity cases: FP32 operators to 1e-5 (2e-5 for Joseph), the
diffusivity to 2e-6, the V-cycle to 1e-4, four MLSQR iterations to 1e-3 on f and 1e-4 on the
residual estimates.  A float32 model of the four iterations (every vector rounded to float32)
stays within 1e-6 of the oracle on f and 1e-9 on the estimates at both sizes.
"""
import numpy as np
import pytest

import oracle as O
from envelope import rel
from paper_1308_6634_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = ["inpaint192_fp32", "tomo512_fp32"]
N_ITER = 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_6634_gb300 import build
    build.build()


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32).cuda()


def host(t):
    return t.detach().double().cpu().numpy()


_PROBLEMS = {}


def _problem(name):
    """(workload, true image, oracle operator, noisy data, mask) for seed 0, built once."""
    if name not in _PROBLEMS:
        W = synth.WORKLOADS[name]
        f, mask, z = W.inputs(0)
        op = O.Operator(W.kind, W.shape, sigma=W.sigma, radius=W.radius, mask=mask, n_angles=W.n_angles,
                        n_bins=W.n_bins)
        g = synth.add_noise(op.A(f), W.noise, z)
        _PROBLEMS[name] = (W, f, op, g, mask)
    return _PROBLEMS[name]


def _solver(W, mask):
    from paper_1308_6634_gb300 import plsqr
    S = plsqr.Solver(W.shape, W.precision, levels=W.levels, sweeps=W.nu, cycles=W.cycles)
    S.set_operator(W.kind, sigma=W.sigma, radius=W.radius, mask=mask, n_angles=W.n_angles, n_bins=W.n_bins)
    return S


def _kappa(W, f):
    """A structured diffusivity: the workload's regulariser on its true image plus 1% noise."""
    fn = f + 0.01 * np.random.default_rng(5).standard_normal(W.shape)
    return O.diffusivity(fn, W.reg, W.T)[0]


@pytest.mark.parametrize("name", CASES)
def test_operators_full_size(name):
    W, f, op, g, mask = _problem(name)
    S = _solver(W, mask)
    tol = 2e-5 if W.kind == "joseph" else 1e-5
    Af = host(S.apply_A(dev(f)))
    assert rel(Af, op.A(f)) < tol
    Atg = host(S.apply_At(dev(g)))
    assert rel(Atg, op.At(g)) < tol
    # Adjoint identity of the float32 pair on the workload's data.  The forward and adjoint
    # kernels each round differently from the oracle (the Joseph pair forms its interpolation
    # weights from different float32 expressions, ray march versus gather), and with g close to
    # A f the inner products carry no cancellation, so that rounding shows in full.  The bar is
    # therefore what each map's own measured deviation from the (exact-transpose, FP64) oracle
    # explains, plus a double-rounding term:
    #   |<Af,g> - <f,A^T g>| <= |<Af - A_ref f, g>| + |<f, A^T g - A_ref^T g>| + 1e-12 ||Af|| ||g||.
    # A transposition slip (a wrong bin, weight or angle in one of the two maps) breaks the
    # entrywise checks above and this identity together.
    Af_ref, Atg_ref = op.A(f), op.At(g)
    lhs, rhs = float((Af * g).sum()), float((f * Atg).sum())
    explained = abs(float(((Af - Af_ref) * g).sum())) + abs(float((f * (Atg - Atg_ref)).sum()))
    scale = np.linalg.norm(Af) * np.linalg.norm(g)
    print(f"{name} float32 adjoint identity: {abs(lhs - rhs) / scale:.2e} of ||Af|| ||g||, "
          f"explained by the maps' own rounding: {explained / scale:.2e}")
    assert abs(lhs - rhs) <= explained + 1e-12 * scale


@pytest.mark.parametrize("name", CASES)
def test_adjoint_identity_fp64_full_size(name):
    """The double-precision pair at the full workload size is a transpose to 1e-12, on random
    signed vectors and on the workload's own data (the gather adjoint must be the exact
    transpose of the forward map; in double the two weight formulas agree to ~1e-15)."""
    W, f, op, g, mask = _problem(name)
    from paper_1308_6634_gb300 import plsqr
    S = plsqr.Solver(W.shape, "fp64", levels=W.levels, sweeps=W.nu, cycles=W.cycles)
    S.set_operator(W.kind, sigma=W.sigma, radius=W.radius, mask=mask, n_angles=W.n_angles, n_bins=W.n_bins)
    rng = np.random.default_rng(9)
    d64 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).cuda()
    for x, y in ((rng.standard_normal(W.shape), rng.standard_normal(g.shape)), (f, g)):
        Ax = host(S.apply_A(d64(x)))
        Aty = host(S.apply_At(d64(y)))
        assert rel(Ax, op.A(x)) < 1e-11 and rel(Aty, op.At(y)) < 1e-11
        err = abs(float((Ax * y).sum()) - float((x * Aty).sum())) / (np.linalg.norm(Ax) * np.linalg.norm(y))
        print(f"{name} float64 adjoint identity: {err:.2e}")
        assert err < 1e-12


@pytest.mark.parametrize("name", CASES)
def test_diffusivity_and_priorconditioner_full_size(name):
    W, f, op, g, mask = _problem(name)
    S = _solver(W, mask)
    kappa, R = S.diffusivity(dev(f), W.reg, W.T)
    k_ref, R_ref = O.diffusivity(f, W.reg, W.T, kfloor=1e-4)
    assert rel(host(kappa), k_ref) < 2e-6
    assert R == pytest.approx(R_ref, rel=2e-6)
    k = _kappa(W, f)
    b = np.random.default_rng(6).standard_normal(W.shape)
    S.prec_setup(dev(k))
    mg = O.Multigrid(k, W.levels, W.nu, W.cycles)
    assert rel(host(S.prec_apply(dev(b))), mg.apply(b)) < 1e-4
    assert rel(host(S.apply_M(dev(b))), O.apply_M(k, b)) < 1e-6


@pytest.mark.parametrize("name", CASES)
def test_first_mlsqr_iterations_full_size(name):
    W, f, op, g, mask = _problem(name)
    k = _kappa(W, f)
    f_ref, h_ref, st = O.mlsqr(op, g, W.tau, N_ITER, prec=O.Multigrid(k, W.levels, W.nu, W.cycles))
    S = _solver(W, mask)
    S.prec_setup(dev(k))
    fg, hist, rc = S.mlsqr(dev(g), W.tau, N_ITER)
    assert rc == 0 and st == 0 and len(hist) == N_ITER
    ef, eh = rel(host(fg), f_ref), rel(hist, h_ref)
    print(f"{name} {N_ITER} MLSQR iterations: f {ef:.2e}, rbar {eh:.2e}")
    assert ef < 1e-3 and eh < 1e-4
