"""Continuous-batching server on the GPU: every request's result is the same
alone and in the mix (bitwise), with admission limited by a memory budget."""
import numpy as np
import pytest

from paper_2205_12721_b300 import capi, meshgen
from paper_2205_12721_b300.serve import Server, summarize

pytestmark = pytest.mark.gpu


def _jobs(n=10):
    return meshgen.serving_workload(n, rate=2000.0, seed=7, n2=(4, 10), n3=(2, 4), orders=(1, 2, 3))


@pytest.mark.parametrize("budget", [8 << 30, 6 << 20])
def test_served_equals_alone(budget):
    jobs = _jobs()
    srv = Server(budget, newton_rtol=1e-6, newton_max_it=40, minres_max_it=60)
    done = {r["job"]["id"]: r for r in srv.run(jobs, keep_positions=True)}
    srv.close()
    assert len(done) == len(jobs)
    for j in jobs:
        a = Server(8 << 30, newton_rtol=1e-6, newton_max_it=40, minres_max_it=60)
        (ra,) = a.run([dict(j, arrival=0.0)], keep_positions=True)
        a.close()
        rm = done[j["id"]]
        assert rm["status"] == capi.OK and ra["status"] == capi.OK
        assert rm["grad_norm"] <= 1e-6 * rm["grad_norm0"] or rm["newton_its"] == 40
        assert rm["newton_its"] == ra["newton_its"]
        assert np.array_equal(rm["x"], ra["x"])
    s = summarize(list(done.values()))
    assert s["ok"] == len(jobs) and s["p99_s"] >= s["p50_s"] > 0
