"""Scheduling logic of the request loop (serve.Server) with a fake batch engine and a
simulated clock: arrivals, FIFO admission under the HBM budget and the slot limit,
continuous admission as slots free up, retirement on the residual or the step cap."""
import numpy as np
import pytest

from paper_1810_08137_gb300 import inputs as I
from paper_1810_08137_gb300 import serve


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakeInstance:
    def __init__(self, batch, slot):
        self.b, self.slot = batch, slot

    def init_maxwellian(self, *prim):
        self.b.steps[self.slot] = 0

    def residual(self):
        # decays geometrically with the instance's own step count (rate from its config)
        return np.full(4, self.b.rate[self.slot] ** self.b.steps[self.slot])

    def get_state(self):
        return self.b.steps[self.slot]


class FakeBatch:
    def __init__(self, clock, step_time=1e-3):
        self.clock, self.step_time = clock, step_time
        self.steps, self.rate, self.log = {}, {}, []
        self.next = 0

    def admit(self, cfg):
        s = self.next
        self.next += 1
        self.rate[s] = cfg.kn  # test hook: kn doubles as the residual decay rate
        self.steps[s] = 0
        self.log.append(("admit", cfg.name, self.clock()))
        return s

    def retire(self, slot):
        self.log.append(("retire", slot, self.clock()))
        del self.steps[slot]

    def instance(self, slot):
        return FakeInstance(self, slot)

    def step(self, n):
        for s in self.steps:
            self.steps[s] += n
        self.clock.t += n * self.step_time

    def sync(self):
        pass


def req(k, arrival, rate, nx=10):
    cfg = I.channel_config(nx=nx, ny=nx // 2, n_vel=8, kn=rate, name=f"r{k}")
    return serve.Request(rid=k, arrival=arrival, cfg=cfg, prim=())


def test_all_finish_fifo_and_limits():
    clk = Clock()
    fb = FakeBatch(clk)
    rs = [req(k, 0.01 * k, 0.5 + 0.01 * k) for k in range(10)]
    srv = serve.Server(fb, lambda c: 100, hbm_budget=300, max_slots=5, tol=1e-6,
                       max_steps=5000, check_every=7, clock=clk, sleep=clk.sleep)
    st = srv.run(rs)
    s = st.summary()
    assert s["finished"] == 10 and s["converged"] == 10
    assert st.peak_bytes <= 300 and st.peak_active <= 3  # budget binds before the slot limit
    admits = [e[1] for e in fb.log if e[0] == "admit"]
    assert admits == [f"r{k}" for k in range(10)]        # arrival order, no overtaking
    for r in rs:
        assert r.admitted >= r.arrival and r.finished > r.admitted
        assert r.residual < 1e-6 and r.steps % 7 == 0 or r.steps == 5000
    assert s["p50_s"] <= s["p99_s"]


def test_step_cap_marks_not_converged():
    clk = Clock()
    fb = FakeBatch(clk)
    rs = [req(0, 0.0, 0.999), req(1, 0.0, 0.5)]
    srv = serve.Server(fb, lambda c: 1, hbm_budget=0, max_slots=4, tol=1e-6, max_steps=300,
                       check_every=50, clock=clk, sleep=clk.sleep)
    st = srv.run(rs)
    assert rs[0].steps == 300 and not rs[0].converged
    assert rs[1].converged and rs[1].steps < 300
    assert st.summary()["converged"] == 1


def test_late_arrival_waits_and_idle_server_sleeps():
    clk = Clock()
    fb = FakeBatch(clk)
    rs = [req(0, 0.0, 0.5), req(1, 10.0, 0.5)]
    srv = serve.Server(fb, lambda c: 1, hbm_budget=0, max_slots=4, tol=1e-3, max_steps=1000,
                       check_every=5, clock=clk, sleep=clk.sleep)
    srv.run(rs)
    assert rs[1].admitted >= 10.0
    assert rs[0].finished < 10.0


def test_request_over_budget_is_refused():
    clk = Clock()
    fb = FakeBatch(clk)
    srv = serve.Server(fb, lambda c: 1000, hbm_budget=10, max_slots=4, clock=clk, sleep=clk.sleep)
    with pytest.raises(RuntimeError):
        srv.run([req(0, 0.0, 0.5)])


def test_poisson_arrivals_are_seeded_and_increasing():
    a = I.poisson_arrivals(20.0, 64, I.seed_for(5))
    b = I.poisson_arrivals(20.0, 64, I.seed_for(5))
    assert np.array_equal(a, b) and np.all(np.diff(a) > 0)
    assert 1.5 < a[-1] < 6.0  # 64 arrivals at 20/s


def test_mode_switching_follows_work_in_flight():
    """The served batch runs one persistent launch per step when the admitted work is large
    and phase launches when it is small (no GPU: a fake engine records the mode per step)."""
    from paper_1810_08137_gb300 import serve

    class Fake:
        def __init__(self):
            self.persistent, self.modes, self.n = True, [], 0

        def set_persistent(self, on):
            self.persistent = bool(on)

        def admit(self, cfg):
            self.n += 1
            return self.n

        def retire(self, slot):
            pass

        def step(self, n=1):
            self.modes.append(self.persistent)

    small = I.channel_config(nx=10, ny=5, n_vel=8)        # 3200 vc
    big = I.channel_config(nx=100, ny=50, n_vel=40)       # 8e6 vc
    eng = serve.ModeSwitchingBatch(Fake(), persistent_min_vc=1_000_000)
    a = eng.admit(small)
    eng.step()
    b = eng.admit(big)
    eng.step()
    eng.retire(b)
    eng.step()
    eng.retire(a)
    assert eng._b.modes == [False, True, False]
