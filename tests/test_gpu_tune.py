"""Launch-shape autotuner: every candidate shape of the step kernels computes bit-identical
fields (so the tuner's choice can never change a result), the tuned handle still matches
the oracle, choices are cached per kind of group, and invalid shapes are refused."""
import numpy as np
import pytest

import oracle
from paper_1911_03225_gb300 import FDM, Batch, FDMError, Params, inputs
from paper_1911_03225_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def coupled(n1, n2, precision, autotune=0):
    return Params(n1=n1, n2=n2, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRAIN_RAMP,
                  eps_bar13_rate=1e-4, cfl=0.4, theta=1.0, precision=precision, autotune=autotune)


def run(p, up0, steps, cfg=None):
    with FDM(p) as sim:
        if cfg is not None:
            sim.set_launch_config(cfg)
            got = sim.launch_config()
            for k in ("rows_per_block", "cols_per_block", "stencil_block_rows", "stencil_nodes",
                      "stencil_min_blocks"):
                assert got[k] == cfg[k]
        sim.set_plastic_distortion(up0)
        info = sim.step(steps)
        return sim.read_fields("up13", "tau13"), info


@pytest.mark.parametrize("precision", [B.FP64, B.MIXED, B.DF64])
@pytest.mark.parametrize("n1,n2", [(128, 128), (64, 256)])
def test_every_candidate_shape_gives_identical_fields(precision, n1, n2):
    p = coupled(n1, n2, precision)
    up0 = inputs.random_up(max(n1, n2), seed=3, ell=8.0)[:n2, :n1].copy()
    up0 -= up0.mean()
    ref, info = run(p, up0, 6)
    cands = B.launch_candidates(p)
    assert len(cands) >= 4
    for cfg in cands:
        got, gi = run(p, up0, 6, cfg)
        np.testing.assert_array_equal(got["up13"], ref["up13"])
        np.testing.assert_array_equal(got["tau13"], ref["tau13"])
        assert gi.t == info.t and gi.mean_up13 == info.mean_up13


def test_tuned_handle_matches_oracle_and_reports_times():
    n, steps = 256, 10
    p = coupled(n, n, B.FP64, autotune=1)
    up0 = inputs.random_up(n, seed=21, ell=8.0)
    with FDM(p) as sim:
        cfg = sim.launch_config()
        sim.set_plastic_distortion(up0)
        sim.step(steps)
        got = sim.read_fields("up13")["up13"]
    assert cfg["tuned"] == 1 and all(t > 0 for t in cfg["kernel_us"])
    cands = B.launch_candidates(p)
    assert cfg["rows_per_block"] in {c["rows_per_block"] for c in cands}
    assert cfg["cols_per_block"] in {c["cols_per_block"] for c in cands}
    stencil = lambda c: (c["stencil_block_rows"], c["stencil_nodes"], c["stencil_min_blocks"])  # noqa: E731
    assert stencil(cfg) in {stencil(c) for c in cands}
    op = oracle.Params(n1=n, n2=n, velocity_mode=1, loading_mode=1, eps_bar13_rate=1e-4, cfl=0.4, theta=1.0)
    ref, rc = oracle.run(op, up0, steps)
    assert np.linalg.norm(got - ref.up13) / np.linalg.norm(ref.up13) < 1e-11
    # the choice is cached: a second handle of the same kind gets it without timing again
    with FDM(p) as sim2:
        assert sim2.launch_config() == cfg


def test_batch_groups_are_tuned():
    params = [coupled(64, 64, B.MIXED, autotune=1), coupled(128, 128, B.FP64, autotune=1),
              coupled(64, 64, B.MIXED, autotune=1)]
    with Batch(params) as b:
        cfgs = [b.launch_config(i) for i in range(3)]
    assert all(c["tuned"] == 1 for c in cfgs)
    assert cfgs[0] == cfgs[2]


def test_invalid_launch_shapes_refused():
    p = coupled(64, 64, B.FP64)
    with FDM(p) as sim:
        good = sim.launch_config()
        assert good["tuned"] == 0
        for bad in ({**good, "rows_per_block": 3}, {**good, "cols_per_block": 64},
                    {**good, "stencil_block_rows": 5}, {**good, "stencil_min_blocks": 9}):
            with pytest.raises(FDMError) as e:
                sim.set_launch_config(bad)
            assert e.value.status == B.FDM_ERR_INVALID_ARG
        assert sim.launch_config() == good


def test_tuning_persists_across_processes(tmp_path):
    """With FDM_TUNE_CACHE set, the first process times the shapes and appends one JSON line;
    a second process reads the choice back instead of timing again."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = tmp_path / "tune.jsonl"
    code = ("import json, sys; sys.path.insert(0, %r)\n"
            "from paper_1911_03225_gb300 import FDM, Params\n"
            "from paper_1911_03225_gb300 import binding as B\n"
            "p = Params(n1=256, n2=128, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRAIN_RAMP, "
            "eps_bar13_rate=1e-4, cfl=0.4, precision=B.MIXED, autotune=1)\n"
            "with FDM(p) as s: print(json.dumps(s.launch_config()))\n" % root)
    env = dict(os.environ, FDM_TUNE_CACHE=str(path))
    runs = [subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
            for _ in range(2)]
    for r in runs:
        assert r.returncode == 0, r.stderr[-2000:]
    first, second = (json.loads(r.stdout.strip().splitlines()[-1]) for r in runs)
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(lines) == 1 and lines[0]["n1"] == 256 and lines[0]["n2"] == 128
    assert first["tuned"] == 1 and second["tuned"] == 1
    for k in ("rows_per_block", "cols_per_block", "stencil_block_rows", "stencil_nodes", "stencil_min_blocks"):
        assert first[k] == second[k]
    assert second["kernel_us"] == pytest.approx(lines[0]["kernel_us"], abs=1e-9)
    assert first["kernel_us"] == pytest.approx(second["kernel_us"], abs=1e-3)
