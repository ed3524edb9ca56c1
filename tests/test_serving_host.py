"""Host logic of the continuous-batching server (FIFO admission under a
memory budget, per-tick stepping of active groups, retirement and latency
accounting), exercised on the CPU with a stand-in for the GPU batch."""
import itertools

from paper_2205_12721_b300 import meshgen, serve


class FakeBatch:
    """Converges each mesh after a number of steps equal to its order."""

    def __init__(self, order):
        self.order = order
        self.slots = {}
        self.ids = itertools.count()
        self.steps = 0

    def mesh_bytes(self, E, Nx):
        return 1000 * E

    def add_structured(self, m, h0=1.0):
        s = next(self.ids)
        self.slots[s] = {"left": self.order, "its": 0}
        return s

    def step(self):
        self.steps += 1
        for v in self.slots.values():
            if v["left"] > 0:
                v["left"] -= 1
                v["its"] += 1
        return sum(1 for v in self.slots.values() if v["left"] > 0)

    def state(self, s):
        v = self.slots[s]
        return {"done": int(v["left"] == 0), "status": 0, "newton_its": v["its"], "minres_its": 0,
                "energy0": 1.0, "energy": 0.0, "grad_norm0": 1.0, "grad_norm": 0.0,
                "min_det": 1.0, "alpha": 1.0}

    def remove(self, s):
        del self.slots[s]

    def close(self):
        pass


def test_admission_retirement_and_latency(monkeypatch):
    jobs = meshgen.serving_workload(12, rate=1e6, seed=3, n2=(2, 3), n3=(1, 2), orders=(1, 2, 3))
    srv = serve.Server(mem_budget_bytes=10 ** 12)
    fakes = {}

    def group(dim, order, metric):
        return fakes.setdefault((dim, order, metric), FakeBatch(order))

    monkeypatch.setattr(srv, "group", group)
    srv.groups = fakes
    done = srv.run(jobs, build=lambda j: meshgen.structured(j["dim"], 1, j["n"]))
    assert sorted(r["job"]["id"] for r in done) == list(range(12))
    for r in done:
        assert r["newton_its"] == r["job"]["order"]
        assert r["latency"] >= 0 and r["done_at"] >= r["admitted"]
    assert srv.used == 0
    # a budget that admits one mesh at a time still serves everything, FIFO
    srv2 = serve.Server(mem_budget_bytes=1)
    fakes.clear()
    monkeypatch.setattr(srv2, "group", group)
    srv2.groups = fakes
    done2 = srv2.run(jobs, build=lambda j: meshgen.structured(j["dim"], 1, j["n"]))
    order = [r["job"]["id"] for r in sorted(done2, key=lambda r: r["admitted"])]
    assert order == sorted(order)
    assert srv2.used == 0 and len(done2) == 12
