"""The autotuner (paper_1412_0464_gb300/autotune.py): cache keys, candidate
sets and the cache round trip on the CPU; on the GPU, a tuning run on a 2-D and
a 3-D workload whose chosen parameters leave the preconditioner unchanged up
to complex64 rounding, and a second call served from the cache."""

import json

import numpy as np
import pytest

import synth
from paper_1412_0464_gb300 import autotune


def test_keys_separate_what_changes_the_work():
    a = synth.scaled_workload(2, 120, w_out=8, J=6)
    k = autotune.workload_key(a, "dev")
    assert k == autotune.workload_key(a, "dev")
    assert k != autotune.workload_key(a, "other")
    assert k != autotune.workload_key(a, "dev", {"precision": "fp64"})
    assert k != autotune.workload_key(a, "dev", {"sweep": "UD"})
    assert k != autotune.workload_key(synth.scaled_workload(2, 122, w_out=8, J=6), "dev")
    assert k != autotune.workload_key(a, "dev", {"max_rhs": 8})


def test_candidates():
    c2 = synth.scaled_workload(2, 1000)
    cand = autotune.candidates(c2, sms=152)
    assert {"segments": 0} in cand and len(cand) >= 3
    assert all(c["segments"] == 0 or 2 <= c["segments"] <= 2 * 152 for c in cand)
    c4 = synth.scaled_workload(4, 32)
    assert autotune.candidates(c4) == [{"block_3d": 64}, {"block_3d": 128}, {"block_3d": 256}]


def test_choose_and_cache_round_trip(tmp_path):
    times = {json.dumps({"segments": 0}): 2.0, json.dumps({"segments": 40}): 1.5,
             json.dumps({"segments": 80}): 1.5}
    assert json.loads(autotune.choose(times)) == {"segments": 40}
    p = str(tmp_path / "t.json")
    assert autotune.load_cache(p) == {}
    autotune.store("k1", {"params": {"segments": 40}}, p)
    autotune.store("k2", {"params": {"block_3d": 64}}, p)
    d = autotune.load_cache(p)
    assert d["k1"]["params"] == {"segments": 40} and d["k2"]["params"] == {"block_3d": 64}


@pytest.mark.gpu
@pytest.mark.parametrize("idx,n,w_out,J", [(2, 160, 8, 6), (4, 24, 4, 2)])
def test_tuning_run_and_cache(idx, n, w_out, J, tmp_path):
    torch = pytest.importorskip("torch")
    import paper_1412_0464_gb300 as hz
    hz.build()
    cfg = synth.scaled_workload(idx, n, w_out=w_out, J=J, n_src=1)
    p = str(tmp_path / "cache.json")
    e = autotune.tune(cfg, path=p, reps=2)
    assert len(e["ms"]) == len(autotune.candidates(
        cfg, torch.cuda.get_device_properties(0).multi_processor_count))
    assert all(v > 0 for v in e["ms"].values())
    assert autotune.tune(cfg, path=p)["when"] == e["when"]       # served from the cache
    f = torch.from_numpy(synth.sources(cfg)[:1]).cuda()
    ref = hz.Solver.from_workload(cfg)
    ref.factor()
    z0 = ref.precond(f).cpu().numpy()
    s = autotune.tuned_solver(cfg, path=p)
    s.factor()
    z1 = s.precond(f).cpu().numpy()
    assert np.linalg.norm(z1 - z0) <= 3e-4 * np.linalg.norm(z0)
