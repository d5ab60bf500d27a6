"""Batched instances and the continuous-batching server: every instance's result must be the
same as when it runs alone (the kernels are deterministic, so equality is exact), and the
batched FP64 result must match the oracle."""
import numpy as np
import pytest

import oracle
from paper_1911_03225_gb300 import FDM, Batch, Params, inputs
from paper_1911_03225_gb300 import binding as B
from paper_1911_03225_gb300.serve import Request, Server, poisson_arrivals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def coupled(n, precision=B.FP64):
    return Params(n1=n, n2=n, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRAIN_RAMP, eps_bar13_rate=1e-4,
                  cfl=0.4, theta=1.0, precision=precision)


def alone(p, up0, steps):
    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        info = sim.step(steps)
        return sim.read_fields("up13", "tau13"), info


def test_batch_equals_single_runs_with_uneven_sizes_and_budgets():
    specs = [(64, B.FP64, 0, 30), (128, B.MIXED, 1, 17), (64, B.FP64, 2, 9), (32, B.MIXED, 3, 30),
             (128, B.FP64, 4, 25), (64, B.MIXED, 5, 0)]
    params = [coupled(n, prec) for n, prec, _, _ in specs]
    ups = [inputs.random_up(n, seed=s, ell=8.0) for n, _, s, _ in specs]
    with Batch(params) as b:
        assert b.launches_per_step() == 4 * 5   # (64,FP64) x2 share a group
        for i, (n, prec, s, steps) in enumerate(specs):
            b.set_plastic_distortion(i, ups[i])
            b.set_budget(i, steps)
        b.enqueue_steps(12)
        left = b.sync()
        assert list(left) == [max(st - 12, 0) for *_, st in specs]
        b.enqueue_steps(20)
        assert (b.sync() == 0).all()
        got = [b.read_fields(i, "up13", "tau13") for i in range(len(specs))]
        infos = [b.info(i) for i in range(len(specs))]
    for i, (n, prec, s, steps) in enumerate(specs):
        assert infos[i].step == steps
        if steps == 0:
            np.testing.assert_allclose(got[i]["up13"], ups[i], atol=1e-6 if prec == B.MIXED else 0)
            continue
        ref, info = alone(params[i], ups[i], steps)
        np.testing.assert_array_equal(got[i]["up13"], ref["up13"])
        np.testing.assert_array_equal(got[i]["tau13"], ref["tau13"])
        assert infos[i].t == info.t


def test_batched_fp64_matches_oracle():
    n, steps = 64, 40
    params = [coupled(n), coupled(n)]
    ups = [inputs.random_up(n, seed=11, ell=6.0), inputs.random_up(n, seed=12, ell=6.0)]
    with Batch(params) as b:
        for i in range(2):
            b.set_plastic_distortion(i, ups[i])
            b.set_budget(i, steps)
        b.enqueue_steps(steps)
        b.sync()
        got = [b.read_fields(i, "up13")["up13"] for i in range(2)]
    op = oracle.Params(n1=n, n2=n, velocity_mode=1, loading_mode=1, eps_bar13_rate=1e-4, cfl=0.4, theta=1.0)
    for i in range(2):
        ref, rc = oracle.run(op, ups[i], steps)
        assert np.linalg.norm(got[i] - ref.up13) / np.linalg.norm(ref.up13) < 1e-11


def test_served_results_equal_alone_runs():
    """Requests of different sizes, lengths and precisions arrive over time; the server
    admits them into free slots while others run.  Each result equals its solo run."""
    rng = np.random.default_rng(5)
    sizes = [32, 64, 128]
    reqs = []
    arr = poisson_arrivals(200.0, 14, seed=9)
    for k in range(14):
        n = int(rng.choice(sizes))
        prec = B.FP64 if k % 2 == 0 else B.MIXED
        reqs.append(Request(rid=k, n=n, steps=int(rng.integers(5, 60)), precision=prec, arrival=float(arr[k]),
                            up13=inputs.random_up(n, seed=100 + k, ell=6.0)))
    base = coupled(32)
    classes = {(n, p): 2 for n in sizes for p in (B.FP64, B.MIXED)}
    srv = Server(base, classes, hbm_budget=40e6, tick_steps=4)
    try:
        results, stats = srv.run(reqs)
    finally:
        srv.close()
    assert stats["completed"] == len(reqs)
    assert stats["p99_latency_s"] >= stats["p50_latency_s"] > 0
    by_id = {r.rid: r for r in results}
    for k in (0, 1, 2, 5, 8):
        r = reqs[k]
        ref, info = alone(Params(**{**base.__dict__, "n1": r.n, "n2": r.n, "precision": r.precision}), r.up13, r.steps)
        np.testing.assert_array_equal(by_id[k].up13, ref["up13"])
        assert by_id[k].t == info.t


def test_server_retires_failed_requests_and_keeps_the_others():
    """A request with a non-finite input is refused at admission; one whose simulation
    leaves the finite range (U13 of 1e308 drives an infinite stress) is retired with
    FDM_ERR_NONFINITE and its slot freed; every other request completes and equals its solo
    run, including one admitted into the freed slot afterwards."""
    n = 32
    base = coupled(n)
    good = [inputs.random_up(n, seed=200 + k, ell=6.0) for k in range(3)]
    nan_in = good[0].copy()
    nan_in[4, 5] = np.nan
    blow = np.zeros((n, n))
    blow[3, 4] = 1e308
    reqs = [Request(rid=0, n=n, steps=20, precision=B.FP64, arrival=0.0, up13=good[0]),
            Request(rid=1, n=n, steps=20, precision=B.FP64, arrival=0.0, up13=nan_in),
            Request(rid=2, n=n, steps=40, precision=B.FP64, arrival=0.0, up13=blow),
            Request(rid=3, n=n, steps=30, precision=B.FP64, arrival=0.0, up13=good[1]),
            Request(rid=4, n=n, steps=12, precision=B.FP64, arrival=0.0, up13=good[2])]
    srv = Server(base, {(n, B.FP64): 2}, hbm_budget=1e9, tick_steps=4)
    try:
        results, stats = srv.run(reqs)
        failed = {r.rid: r.status for r in srv.failed}
    finally:
        srv.close()
    assert failed == {1: B.FDM_ERR_INVALID_ARG, 2: B.FDM_ERR_NONFINITE}
    assert stats["completed"] == 3 and stats["failed"] == 2
    by_id = {r.rid: r for r in results}
    for k, up in ((0, good[0]), (3, good[1]), (4, good[2])):
        ref, info = alone(base, up, reqs[k].steps)
        np.testing.assert_array_equal(by_id[k].up13, ref["up13"])
        assert by_id[k].t == info.t


def test_hbm_budget_bounds_admission_while_slots_are_free():
    """The budget is a ledger of device memory actually held: with room for one group of the
    class, a second request waits although the class allows four resident simulations, and
    runs once the first has finished (its idle group then serves it).  After every tick the
    ledger equals the device bytes of the allocated groups and the device's used memory
    follows it; closing the server returns the memory.  A request of a class the server does
    not offer, and one whose group alone is over the budget, are retired at arrival."""
    import torch
    n = 64
    base = coupled(n)
    ups = [inputs.random_up(n, seed=300 + k, ell=6.0) for k in range(3)]
    probe = Server(base, {(n, B.FP64): 4, (256, B.FP64): 1}, hbm_budget=1e12, tick_steps=4, group_size=1)
    one = probe.group_bytes((n, B.FP64))
    big = probe.group_bytes((256, B.FP64))
    assert big > 2 * one
    reqs = [Request(rid=k, n=n, steps=12 + 4 * k, precision=B.FP64, arrival=0.0, up13=ups[k]) for k in range(3)]
    reqs.append(Request(rid=3, n=128, steps=8, precision=B.FP64, arrival=0.0, up13=inputs.random_up(128, seed=1)))
    reqs.append(Request(rid=4, n=256, steps=8, precision=B.FP64, arrival=0.0, up13=inputs.random_up(256, seed=2)))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    seen = []

    def monitor(srv):
        torch.cuda.synchronize()
        assert srv.bytes_in_use == sum(g.nbytes for g in srv.groups) <= srv.hbm_budget
        assert srv.resident <= 1
        seen.append((srv.bytes_in_use, free0 - torch.cuda.mem_get_info()[0]))

    srv = Server(base, {(n, B.FP64): 4, (256, B.FP64): 1}, hbm_budget=1.5 * one, tick_steps=4, group_size=1)
    try:
        results, stats = srv.run(reqs, monitor=monitor)
    finally:
        srv.close()
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (8 << 20)
    assert stats["completed"] == 3 and stats["max_resident"] == 1 and stats["peak_bytes"] == one
    assert {r.rid: r.status for r in srv.failed} == {3: B.FDM_ERR_INVALID_ARG, 4: B.FDM_ERR_OOM}
    assert stats["groups_allocated"] == 1    # the idle group of the finished request is reused
    # small buffers share the driver's pages, so the device's used memory can sit a little
    # below or above the ledger; it never holds more than the one group
    for ledger, used in seen:
        assert ledger == one and used < one + (64 << 20)
    by_id = {r.rid: r for r in results}
    fin = sorted(results, key=lambda r: r.finished)
    assert [r.rid for r in fin] == [0, 1, 2]
    assert by_id[1].admitted >= by_id[0].finished and by_id[2].admitted >= by_id[1].finished
    for k in range(3):
        ref, info = alone(base, ups[k], reqs[k].steps)
        np.testing.assert_array_equal(by_id[k].up13, ref["up13"])


def test_allocation_failures_release_everything():
    """Host-side fault injection: each allocation of a handle or a batch in turn fails; the
    call returns FDM_ERR_OOM with no handle and no device memory left behind."""
    import torch
    p = coupled(64)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for make in (lambda: FDM(p), lambda: Batch([p, coupled(32, B.MIXED), p])):
            k, done = 0, False
            while not done:
                B.debug_fail_allocation(k)
                try:
                    obj = make()
                except B.FDMError as e:
                    assert e.status == B.FDM_ERR_OOM
                    k += 1
                    continue
                B.debug_fail_allocation(-1)
                obj.close()
                done = True
            assert k >= 10
    finally:
        B.debug_fail_allocation(-1)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (8 << 20)


def test_persistent_launch_equals_graph_steps():
    """The batched steps as one persistent cooperative launch (every phase of every size class,
    grid barriers between phases) give the same results bit for bit as the graph-replayed
    per-kernel launches, with uneven sizes and step budgets."""
    specs = [(64, 0, 30), (128, 1, 17), (64, 2, 9), (256, 3, 30), (128, 4, 0), (32, 5, 22)]
    params = [coupled(n, B.MIXED) for n, _, _ in specs]
    ups = [inputs.random_up(n, seed=40 + s, ell=8.0) for n, s, _ in specs]
    out = {}
    for mode in ("graph", "persistent"):
        with Batch(params) as b:
            for i, (n, s, steps) in enumerate(specs):
                b.set_plastic_distortion(i, ups[i])
                b.set_budget(i, steps)
            if mode == "graph":
                b.enqueue_steps(12)
                b.enqueue_steps(20)
            else:
                b.enqueue_steps_persistent(12)
                b.enqueue_steps_persistent(20)
            assert (b.sync() == 0).all()
            out[mode] = [(b.read_fields(i, "up13", "tau13"), b.info(i)) for i in range(len(specs))]
    for i, (n, s, steps) in enumerate(specs):
        (fg, ig), (fp, ip) = out["graph"][i], out["persistent"][i]
        assert ip.step == ig.step == steps and ip.t == ig.t
        np.testing.assert_array_equal(fp["up13"], fg["up13"])
        np.testing.assert_array_equal(fp["tau13"], fg["tau13"])


def test_persistent_launch_barrier_wait_is_bounded():
    """A barrier that can never complete (the test hook makes it wait for one block more than
    the grid holds) gives up after its limit: the launch ends, the batch reports
    FDM_ERR_TIMEOUT, and the device stays usable (a new batch steps normally)."""
    import time
    n = 64
    params = [coupled(n, B.MIXED), coupled(128, B.MIXED)]
    ups = [inputs.random_up(n, seed=50, ell=6.0), inputs.random_up(128, seed=51, ell=6.0)]
    try:
        B.debug_barrier(1, 0.05)
        with Batch(params) as b:
            for i in range(2):
                b.set_plastic_distortion(i, ups[i])
                b.set_budget(i, 5)
            t0 = time.perf_counter()
            b.enqueue_steps_persistent(3)
            with pytest.raises(B.FDMError) as e:
                b.sync()
            assert e.value.status == B.FDM_ERR_TIMEOUT
            assert time.perf_counter() - t0 < 5.0
    finally:
        B.debug_barrier(0, 0.0)
    with Batch(params) as b:
        for i in range(2):
            b.set_plastic_distortion(i, ups[i])
            b.set_budget(i, 5)
        b.enqueue_steps_persistent(5)
        assert (b.sync() == 0).all()
        got = b.read_fields(0, "up13")["up13"]
    with Batch(params) as b:
        for i in range(2):
            b.set_plastic_distortion(i, ups[i])
            b.set_budget(i, 5)
        b.enqueue_steps(5)
        b.sync()
        np.testing.assert_array_equal(got, b.read_fields(0, "up13")["up13"])


def test_persistent_launch_refuses_other_precisions_and_narrow_grids():
    """The persistent trial runs mixed-precision groups of at least 32 columns; anything else
    is refused before any launch, and the batch still steps through the graphs."""
    up = inputs.random_up(64, seed=60, ell=6.0)
    for params in ([coupled(64, B.FP64)], [coupled(64, B.MIXED), coupled(64, B.DF64)]):
        with Batch(params) as b:
            for i in range(len(params)):
                b.set_plastic_distortion(i, up)
                b.set_budget(i, 3)
            with pytest.raises(B.FDMError) as e:
                b.enqueue_steps_persistent(3)
            assert e.value.status == B.FDM_ERR_INVALID_ARG
            b.enqueue_steps(3)
            assert (b.sync() == 0).all()
    narrow = Params(**{**coupled(16, B.MIXED).__dict__, "n1": 16, "n2": 64})
    with Batch([narrow]) as b:
        b.set_plastic_distortion(0, inputs.random_up(64, seed=61, ell=6.0)[:, :16].copy())
        b.set_budget(0, 2)
        with pytest.raises(B.FDMError) as e:
            b.enqueue_steps_persistent(2)
        assert e.value.status == B.FDM_ERR_INVALID_ARG
