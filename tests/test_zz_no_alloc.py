"""plsqr_blur_noalloc: the separable blur for callers that cannot allocate device memory.

Serving processes that give all device memory to their own pool, code running during CUDA
stream capture and latency-critical loops cannot afford cudaMalloc; this entry point keeps its
scratch (the taps and the intermediate volume of the 3D blur) in a fixed file-scope device array
instead.  Its result must equal the handle-based plsqr_apply_A with the same blur, and two calls
in a row must not interfere through the shared array.  This file is collected last on purpose.
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
    a, b = a.double().cpu().numpy().ravel(), b.double().cpu().numpy().ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [((40, 48, 56), (3.0, 3.0, 5.0), (9, 9, 15)),   # 3D: the intermediate volume is the scratch
         ((96, 160), (4.0, 4.0), (12, 12)),             # 2D, register-blocked radius
         ((67, 45), (1.5, 4.0), (4, 12))]               # 2D, unequal radii, ragged tiles


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("shape,sigma,radius", CASES)
def test_noalloc_blur_matches_apply_A_on_two_calls(prec, shape, sigma, radius):
    from paper_1308_6634_gb300 import plsqr
    dt = torch.float64 if prec == "fp64" else torch.float32
    # the handle is only the reference's carrier; enough levels keep its coarsest band narrow
    levels = 1 if any(n % 2 for n in shape) else (4 if len(shape) == 3 else 2)
    S = plsqr.Solver(shape, prec, levels=levels)
    S.set_operator("blur", sigma=sigma, radius=radius)
    gen = torch.Generator(device="cpu").manual_seed(7)
    for call in range(2):
        x = torch.randn(shape, generator=gen, dtype=torch.float64).to(dt).cuda()
        ref = S.apply_A(x)
        got = plsqr.plsqr_blur_noalloc(x, sigma, radius)
        torch.cuda.synchronize()
        assert _rel(got, ref) < (1e-12 if prec == "fp64" else 1e-6), call


def test_noalloc_blur_rejects_grids_beyond_the_scratch():
    from paper_1308_6634_gb300 import plsqr
    x = torch.zeros((130, 130, 130), dtype=torch.float32, device="cuda")  # 2,197,000 floats > 2,096,640
    with pytest.raises(plsqr.PlsqrError) as e:
        plsqr.plsqr_blur_noalloc(x, (2.0, 2.0, 2.0), (6, 6, 6))
    assert e.value.code == plsqr.E_INVALID


def test_noalloc_blur_rejects_launch_limits_and_overlapping_buffers():
    """Sizes whose launch would be invalid, and x overlapping y, are refused before anything is
    enqueued (the call returns PLSQR_E_INVALID and the stream stays usable)."""
    from paper_1308_6634_gb300 import plsqr
    x = torch.zeros((1, 1 << 20, 1), dtype=torch.float32, device="cuda")  # ny = 2^20: z-pass grid.y > 65535
    with pytest.raises(plsqr.PlsqrError) as e:
        plsqr.plsqr_blur_noalloc(x, (2.0, 2.0, 2.0), (6, 6, 6))
    assert e.value.code == plsqr.E_INVALID
    buf = torch.zeros(2 * 64 * 64, dtype=torch.float32, device="cuda")
    a, b = buf[: 64 * 64].view(64, 64), buf[64 * 32: 64 * 96].view(64, 64)
    for y in (a, b):
        with pytest.raises(plsqr.PlsqrError) as e:
            plsqr.plsqr_blur_noalloc(a, (2.0, 2.0), (6, 6), y=y)
        assert e.value.code == plsqr.E_INVALID
    torch.cuda.synchronize()
