"""Host logic of Mesh.advance (the Newton-count time step control of Sec. 4 and the SDIRK
scheme routing), driven on the CPU by a stand-in mesh whose steps report scripted Newton
iteration counts.  No GPU and no library compute call."""
import pytest
import torch

from oracle import solver


class FakeMesh:
    """dt_estimate / newton_step / sdirk_step with the Mesh signatures; a step adds h to
    every entry of u and reports the next scripted count (None: the solve fails)."""

    def __init__(self, counts, dt_est=0.01):
        import paper_2609_16424_b300 as lh
        self.lh = lh
        self.counts = list(counts)
        self.dt_est = dt_est
        self.calls = []

    def dt_estimate(self, u):
        return self.dt_est

    def _step(self, kind, u, k, h, **kw):
        self.calls.append((kind, kw.get("scheme"), h))
        its = self.counts.pop(0) if self.counts else 2
        if its is None:
            raise self.lh.LHError(5, "scripted failure")
        u += h
        return {"newton_its": 3 * its, "newton_its_max": its}

    def newton_step(self, u, k, h, **kw):
        return self._step("newton", u, k, h, **kw)

    def sdirk_step(self, u, k, h, scheme=3, **kw):
        return self._step("sdirk", u, k, h, scheme=scheme, **kw)


def _advance(fake, t_end, **kw):
    import paper_2609_16424_b300 as lh
    u = torch.zeros(4, dtype=torch.float64)
    out = lh.Mesh.advance(fake, u, t_end, **kw)
    return u, out


@pytest.mark.parametrize("scheme", [2, 3, 4])
def test_controller_follows_the_rule_and_routes_the_scheme(scheme):
    counts = [1, 1, 2, 5, None, 3, 0, 1, 4, 2] + [2] * 40
    fake = FakeMesh(counts)
    u, (steps, rejected, hist) = _advance(fake, 0.2, fs_cfl=2.0, scheme=scheme)
    dt = 2.0 * fake.dt_est
    for (c_dt, h, its, accepted) in hist:
        assert c_dt == pytest.approx(dt, rel=1e-14)
        dt, ok = solver.dt_control(dt, 4 if its is None else its)
        assert ok == accepted
    assert steps == sum(1 for a in hist if a[3]) and rejected == len(hist) - steps == 3
    # u moved by the accepted steps only, and the last step ends at t_end exactly
    assert float(u[0]) == pytest.approx(0.2, rel=1e-12)
    assert sum(h for _, h, _, a in hist if a) == pytest.approx(0.2, rel=1e-12)
    kinds = {c[0] for c in fake.calls}
    assert kinds == ({"newton"} if scheme == 2 else {"sdirk"})
    if scheme != 2:
        assert {c[1] for c in fake.calls} == {scheme}


def test_controller_reads_the_largest_stage_count():
    """newton_its sums the stages (here 3x), the rule reads newton_its_max."""
    fake = FakeMesh([1] * 10)
    _, (steps, rejected, hist) = _advance(fake, 0.05, fs_cfl=1.0, scheme=3)
    assert rejected == 0 and all(a[2] == 1 for a in hist)
    assert hist[1][0] == pytest.approx(1.05 * hist[0][0], rel=1e-14)


def test_fixed_dt_and_attempt_limit():
    fake = FakeMesh([0, 1, 5, 1, 1] + [1] * 40)
    _, (steps, rejected, hist) = _advance(fake, 1.0, fs_cfl=1.0, grow=False)
    dts = [a[0] for a in hist]
    assert all(b <= a * (1 + 1e-15) for a, b in zip(dts, dts[1:]))   # never enlarged
    assert rejected == 1 and dts[3] == pytest.approx(0.85 * dts[0], rel=1e-14)
    fake = FakeMesh([5] * 100)
    u, (steps, rejected, hist) = _advance(fake, 1.0, fs_cfl=1.0, max_attempts=7)
    assert len(hist) == 7 and steps == 0 and rejected == 7 and float(u[0]) == 0.0
