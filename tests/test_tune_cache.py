"""The autotuner's tile-shape cache moved between processes as text or JSON (no GPU needed):
entries round-trip, a later entry for the same level replaces the earlier one, and a malformed
line or an unknown shape is refused with nothing merged."""
import json

import pytest


def _P():
    from paper_1308_6634_gb300 import build, plsqr
    build.build()
    return plsqr


def _entries(plsqr):
    return {tuple(int(v) for v in ln.split()) for ln in plsqr.tune_cache_export().splitlines() if ln.strip()}


def test_text_round_trip_and_replacement():
    P = _P()
    text = "777 512 1 4 2 1 0 2\n\n777 512 1 4 2 0 0 5\n"
    assert P.tune_cache_import(text) == 2
    got = _entries(P)
    assert (777, 512, 1, 4, 2, 1, 0, 2) in got and (777, 512, 1, 4, 2, 0, 0, 5) in got
    assert P.tune_cache_import("777 512 1 4 2 1 0 1") == 1   # the same level class again
    got = _entries(P)
    assert (777, 512, 1, 4, 2, 1, 0, 1) in got and (777, 512, 1, 4, 2, 1, 0, 2) not in got


def test_json_round_trip():
    P = _P()
    P.tune_cache_import("778 64 8 8 3 0 1 3\n")
    d = json.loads(P.tune_cache_json())
    assert d["format"] == 1
    e = [x for x in d["entries"] if x["nx"] == 778]
    assert e == [dict(nx=778, ny=64, batch=8, element_size=8, sweeps=3, finest=0, kappa_bf16=1, shape=3)]
    before = _entries(P)
    assert P.tune_cache_load_json(P.tune_cache_json()) == len(before)
    assert _entries(P) == before


@pytest.mark.parametrize("bad", ["779 64 1 4 2 1 0 6",       # level 0 has shapes 0..5
                                 "779 64 1 4 2 0 0 6",       # coarser levels 0..5
                                 "779 64 1 2 2 0 0 1",       # element size 4 or 8
                                 "779 64 1 4 4 0 0 1",       # 1..3 sweeps
                                 "779 64 1 4 2 0 0",         # seven fields
                                 "779 64 1 4 2 0 0 1 9",     # nine fields
                                 "779 64 0 4 2 0 0 1",       # batch >= 1
                                 "779 x 1 4 2 0 0 1"])
def test_malformed_text_is_refused_whole(bad):
    P = _P()
    before = _entries(P)
    with pytest.raises(P.PlsqrError):
        P.tune_cache_import("780 64 1 4 2 0 0 1\n" + bad + "\n")
    assert _entries(P) == before


def test_serving_engine_loads_and_saves_the_cache():
    """The engine loads a cache file at start and writes the process's choices back (the file
    lives in a git-ignored folder of the test tree)."""
    import os
    P = _P()
    from paper_1308_6634_gb300 import serving
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build")
    os.makedirs(d, exist_ok=True)
    path = os.path.join(d, "tune_cache.json")
    with open(path, "w") as fh:
        fh.write(json.dumps({"format": 1, "entries": [dict(nx=781, ny=128, batch=16, element_size=4, sweeps=2,
                                                             finest=1, kappa_bf16=0, shape=1)]}))
    eng = serving.Engine(tune_cache=path)
    assert (781, 128, 16, 4, 2, 1, 0, 1) in _entries(P)
    os.remove(path)
    eng.save_tune_cache()
    saved = json.load(open(path))
    assert dict(nx=781, ny=128, batch=16, element_size=4, sweeps=2, finest=1, kappa_bf16=0, shape=1) in saved["entries"]
    os.remove(path)
