"""pb_batch_cancel on the GPU: a request cancelled while queued, one stopped
while its solve runs on the device, one whose result was already complete,
and an unknown ticket; the server's later results against the oracle."""
import time

import numpy as np
import pytest

import oracle
from paper_1704_02745_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pbm():
    from paper_1704_02745_gb300 import build, pb
    build.build()
    pb.load()
    return pb


@pytest.fixture(scope="module")
def ctx(pbm):
    c = pbm.Context(0)
    yield c
    c.close()


def wait_until(pred, seconds=60.0):
    t0 = time.perf_counter()
    while not pred():
        if time.perf_counter() - t0 > seconds:
            raise AssertionError("condition not reached")
        time.sleep(0.0005)


def test_cancel_queued_running_finished_and_unknown(pbm, ctx):
    big = inputs.globule_257()  # a plain FP64 solve of it runs for a good part of a second
    spec_big = big.grid.replace(dh="f32")
    small = inputs.small_33()
    other = inputs.random_small(21, 45, 41, 39, n_atoms=25)
    # room for the big grid and one small one: `other` (a third grid) waits in the queue
    budget = pbm.pb_grid_bytes(pbm.grid_desc(spec_big), "f64") + \
        pbm.pb_grid_bytes(pbm.grid_desc(small.grid), "f64") + (1 << 20)
    with pbm.Server(ctx, budget, precision="f64", tol=1e-9, warm_start=True) as srv:
        t_small = srv.submit(2, small.grid, small.atoms)
        r, _ = srv.poll(t_small, 60000)
        assert r.status == 0
        # finished but not yet polled: cancel is too late, the result stands
        t_done = srv.submit(2, small.grid, small.atoms)
        wait_until(lambda: srv.stats()["completed"] >= 2)
        assert srv.cancel(t_done) is False
        r_done, _ = srv.poll(t_done, 60000)
        assert r_done.status == 0
        # running: stopped on the device at the worker's next round
        t_big = srv.submit(1, spec_big, big.atoms)
        wait_until(lambda: srv.stats()["active"] >= 1)
        t_q = srv.submit(3, other.grid, other.atoms)  # needs a grid the budget has no room for
        assert srv.cancel(t_q) is True               # cancelled in the queue
        assert srv.cancel(t_big) is True
        r_q, _ = srv.poll(t_q, 60000)
        assert r_q.status == pbm.PB_ERR_CANCELLED
        r_big, _ = srv.poll(t_big, 60000)
        assert r_big.status == pbm.PB_ERR_CANCELLED and r_big.energy == 0.0
        with pytest.raises(pbm.PbError) as ei:
            srv.cancel(t_big)  # already returned
        assert ei.value.status == pbm.PB_ERR_NOT_FOUND
        with pytest.raises(pbm.PbError):
            srv.cancel(123456789)
        # the server goes on: the cancelled trajectory's grid starts cold
        r_next, _ = srv.poll(srv.submit(3, other.grid, other.atoms), 60000)
        r_small, _ = srv.poll(srv.submit(2, small.grid, small.atoms), 60000)
        r_big2, _ = srv.poll(srv.submit(1, spec_big, big.atoms), 600000)
    for r, p in ((r_next, other), (r_small, small)):
        s = oracle.setup(p.grid, p.atoms)
        e_ref = oracle.energy(s, oracle.pcg(s, tol=1e-11).phi)
        assert r.status == 0 and abs(r.energy - e_ref) <= 1e-8 * abs(e_ref)
    assert r_big2.status == 0 and r_big2.warm_started == 0 and r_big2.info.relres_true < 1e-9
