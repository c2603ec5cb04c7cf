"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/plsqr.h.

No compute call is made here (no GPU in this process is assumed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "plsqr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(plsqr_[A-Za-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["plsqr_create", "plsqr_set_operator", "plsqr_solve", "plsqr_destroy"]:
        assert n in names


def test_library_builds_loads_and_exports_all_symbols():
    from paper_1308_6634_gb300 import build, plsqr
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (plsqr_\w+)", out))
    for n in _declared():
        assert n in exported, n
    L = plsqr.lib()
    for n in _declared():
        assert hasattr(L, n)
    assert sorted(plsqr.EXPORTED) == _declared()


def test_workspace_bytes_and_invalid_configs_without_gpu():
    from paper_1308_6634_gb300 import plsqr
    c = plsqr.make_config((1024, 1024), "fp32", levels=6)
    nb = plsqr.plsqr_workspace_bytes(c)
    assert nb > 10 * 1024 * 1024 * 4
    bad = plsqr.make_config((100, 100), "fp32", levels=4)  # 100 not divisible by 8
    assert plsqr.plsqr_workspace_bytes(bad) == -1
    too_coarse = plsqr.make_config((512, 512), "fp32", levels=1)
    assert plsqr.plsqr_workspace_bytes(too_coarse) == -1


@pytest.mark.parametrize("prec,esz", [("fp32", 4), ("fp64", 8)])
def test_workspace_counts_the_joseph_forward_parts(prec, esz):
    """A Joseph operator whose launches can split each angle over two blocks (n_angles x instances
    below 3 x 152) adds the scratch of the two row parts (2 x data length per instance) and an
    arrival counter per angle and instance; at 456 angles no instance qualifies.  The two operators
    compared have the same data length, so the workspaces differ by exactly that scratch: 455
    angles, one instance at max_batch 1 and still one at 4; 60 angles at max_batch 8, seven."""
    from paper_1308_6634_gb300 import plsqr

    def extra(max_batch, na_split, nb_split, na_whole, nb_whole):
        assert na_split * nb_split == na_whole * nb_whole
        c = plsqr.make_config((256, 256), prec, levels=4, max_batch=max_batch)
        split = plsqr.plsqr_workspace_bytes(c, plsqr.make_operator("joseph", n_angles=na_split, n_bins=nb_split))
        whole = plsqr.plsqr_workspace_bytes(c, plsqr.make_operator("joseph", n_angles=na_whole, n_bins=nb_whole))
        assert split > 0 and whole > 0
        return split - whole

    assert extra(1, 455, 456, 456, 455) == 1 * (2 * esz * 455 * 456 + 4 * 455)
    assert extra(4, 455, 456, 456, 455) == 1 * (2 * esz * 455 * 456 + 4 * 455)
    assert extra(8, 60, 2280, 600, 228) == 7 * (2 * esz * 60 * 2280 + 4 * 60)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library every entry of the binding raises; nothing falls back to the
    oracle or to any other CPU path."""
    from paper_1308_6634_gb300 import plsqr
    monkeypatch.setattr(plsqr, "_lib", None)
    monkeypatch.setattr(plsqr, "LIB_PATH", str(tmp_path / "libplsqr.so"))
    with pytest.raises(ImportError):
        plsqr.lib()
    with pytest.raises(ImportError):
        plsqr.plsqr_workspace_bytes(plsqr.make_config((64, 64), "fp32", levels=3))
    with pytest.raises(ImportError):
        plsqr.projected_solve([1.0, 0.5, 0.2], [1.0, 0.3, 0.1], 0.0)


def test_boundary_from_plain_c():
    """tests/c/abi_from_c.c includes the header as C99 (-pedantic -Werror), links the library and
    runs its host-only entry points: the workspace size and the projected solve of (3.6) with
    k = 1 against its closed form."""
    from paper_1308_6634_gb300 import build
    lib = build.build()
    libdir = os.path.dirname(lib)
    out_dir = os.path.join(ROOT, "tests", "c", "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "abi_from_c")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_from_c.c"), "-L", libdir, "-lplsqr", f"-Wl,-rpath,{libdir}", "-lm",
           "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    p = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert p.returncode == 0 and p.stdout.strip().endswith("ok"), p.stdout + p.stderr


def test_noalloc_binding_refuses_other_dtypes_before_the_library():
    """plsqr_blur_noalloc takes float32 or float64 arrays only: a half-precision tensor (2-byte
    elements, where the kernels would read and write 4 or 8 bytes per value) and a y of another
    dtype than x are refused by the binding before any library call."""
    torch = pytest.importorskip("torch")
    from paper_1308_6634_gb300 import plsqr
    for dt in (torch.float16, torch.bfloat16, torch.int32):
        with pytest.raises(TypeError):
            plsqr.plsqr_blur_noalloc(torch.zeros((8, 8), dtype=dt), (1.0, 1.0), (2, 2))
    with pytest.raises(TypeError):
        plsqr.plsqr_blur_noalloc(torch.zeros((8, 8), dtype=torch.float32), (1.0, 1.0), (2, 2),
                                 y=torch.zeros((8, 8), dtype=torch.float16))


def test_checkpoint_entry_points_refuse_a_null_handle_without_gpu():
    """The checkpoint entry points check their handle before touching the device."""
    from paper_1308_6634_gb300 import plsqr
    L = plsqr.lib()
    assert L.plsqr_slot_state_bytes(None) == -1
    buf = (plsqr.C.c_char * 64)()
    assert L.plsqr_slot_save(None, 0, buf, 64) == plsqr.E_INVALID
    assert L.plsqr_slot_restore(None, 0, buf, 64) == plsqr.E_INVALID
