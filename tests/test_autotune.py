"""Autotuner: candidate enumeration and the JSON cache (CPU), and on a GPU that
the chosen shapes preserve results bit for bit and are cached."""
import json

import numpy as np
import pytest

from paper_2011_04747_gb300 import autotune
from parity_util import ensure_lib, gpu_available


def test_candidate_grid():
    c = autotune.candidates()
    assert len(c) == 192
    assert len({json.dumps(x, sort_keys=True) for x in c}) == 192
    assert autotune.candidates({"react_block": (32,), "bucket_k": (0, 1)}) == [
        {"bucket_k": 0, "react_block": 32}, {"bucket_k": 1, "react_block": 32}]


def test_cache_roundtrip(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    assert autotune.load_cache(p) == {}
    autotune.store_cache(p, "a", {"tuning": {"react_block": 64}, "ms_per_sim_ms": 1.0})
    autotune.store_cache(p, "b", {"tuning": {"react_block": 128}, "ms_per_sim_ms": 2.0})
    d = autotune.load_cache(p)
    assert d["a"]["tuning"]["react_block"] == 64 and d["b"]["ms_per_sim_ms"] == 2.0
    (tmp_path / "bad.json").write_text("{not json")
    assert autotune.load_cache(str(tmp_path / "bad.json")) == {}


@pytest.mark.gpu
@pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")
def test_autotune_preserves_results_and_caches(tmp_path):
    import inputs as I

    binding = ensure_lib()
    wl = I.tp06_slab_3d(31, 29, 9)
    s = binding.solver_from_workload(wl)
    space = {"react_block": (64, 128), "fuse_diffusion": (1, 0), "bucket_k": (1, 0), "pdl": (1, 0)}
    rep = autotune.autotune(s, sim_ms=5.0, space=space, cache_path=str(tmp_path / "t.json"))
    assert not rep["cached"] and rep["rejected"] == 0 and rep["candidates"] == 16
    s.daeti_advance(10.0)
    v = s.daeti_read_v()
    s.close()
    ref = binding.solver_from_workload(wl)
    ref.daeti_advance(10.0)
    assert np.array_equal(ref.daeti_read_v(), v)
    rep2 = autotune.autotune(ref, sim_ms=5.0, space=space, cache_path=str(tmp_path / "t.json"))
    assert rep2["cached"] and rep2["tuning"] == rep["tuning"]
    ref.close()
