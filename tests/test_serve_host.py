"""Scheduling logic of the serving loop, on the host with a stand-in batch:
admission by capacity in arrival order, no request advanced past its step
count, every request retired exactly once with its own final state."""
import numpy as np

from paper_2505_20418_gb300 import maze as M
from paper_2505_20418_gb300 import serve


class FakeBatch:
    """Slots and an arena budget; a simulation's state is its step counter."""

    def __init__(self, slots, budget):
        self.slots, self.budget = slots, budget
        self.sims = {}
        self.order = set()
        self.used = 0
        self.log = []

    def try_add(self, pos, vel, types, L, N, tf, **kw):
        need = N ** 3
        free = [i for i in range(self.slots) if i not in self.sims]
        if not free or self.used + need > self.budget:
            return None
        i = free[0]
        self.sims[i] = {"need": need, "steps": 0, "n": len(pos)}
        self.used += need
        self.log.append(("add", i))
        return i

    def refresh(self):
        """Newcomers join the work order (every admission finishes at once here)."""
        joined = [i for i in self.sims if i not in self.order]
        self.order.update(joined)
        return joined

    def step_ready_async(self, k):
        for i in self.order:
            self.sims[i]["steps"] += k
        self.log.append(("step", k, len(self.order)))

    def sync_status(self):
        return M.MAZE_OK

    def all_stats(self):
        return [{"status": 0, "step": self.sims[i]["steps"] if i in self.sims else -1} for i in range(self.slots)]

    def get(self, i, what):
        return np.full((self.sims[i]["n"], 3), float(self.sims[i]["steps"]))

    def remove(self, i):
        self.order.discard(i)
        self.used -= self.sims.pop(i)["need"]
        self.log.append(("remove", i))

    def close(self):
        pass


def test_admission_order_capacity_and_exact_step_counts():
    reqs = serve.poisson_requests(12, rate=1000.0, sizes=(64, 216, 512), steps=(3, 17), seed=77)
    fb = FakeBatch(slots=3, budget=2 * 24 ** 3 + 16 ** 3)
    srv = serve.Server(0, 0, batch=fb, chunk=4)
    out = srv.run(reqs, realtime=False)
    assert out["served"] == 12
    for q in reqs:
        # the final state shows exactly the requested number of steps
        assert np.all(q.final_pos == q.steps)
        assert q.admitted is not None and q.finished >= q.admitted
    # admitted in arrival order
    order = [q.rid for q in sorted(reqs, key=lambda q: q.admitted)]
    assert order == sorted(order)
    # never more simulations than slots, never over the memory budget
    assert max(e[2] for e in fb.log if e[0] == "step") <= 3
    assert out["box_steps"] == sum(q.steps for q in reqs)


def test_poisson_requests_are_seeded_and_in_range():
    a = serve.poisson_requests(50, rate=200.0, seed=3)
    b = serve.poisson_requests(50, rate=200.0, seed=3)
    assert [(q.arrival, q.work.n_ions, q.steps) for q in a] == [(q.arrival, q.work.n_ions, q.steps) for q in b]
    t = np.array([q.arrival for q in a])
    assert np.all(np.diff(t) > 0)
    assert 50 <= min(q.steps for q in a) and max(q.steps for q in a) <= 2000
    # mean inter-arrival near 1/rate (50 samples: loose)
    assert 0.5 / 200 < np.diff(np.r_[0.0, t]).mean() < 2.0 / 200
