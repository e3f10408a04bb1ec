"""Host logic of the time loop (lh_advance: the Newton-count time step control of Sec. 4),
driven on the CPU through lh_advance_replay, the same C loop fed with scripted Newton
iteration counts instead of solves.  No GPU and no library compute call.  Each attempt is
checked against the oracle's statement of the rule (oracle.solver.dt_control)."""
import pytest

from oracle import solver


def _replay(counts, t_end, dt_est=0.01, **kw):
    import paper_2609_16424_b300 as lh
    return lh.advance_replay(counts, dt_est, t_end, **kw)


def _check_rule(hist, dt0):
    dt = dt0
    for (c_dt, h, its, accepted) in hist:
        assert c_dt == pytest.approx(dt, rel=1e-14)
        dt, ok = solver.dt_control(dt, 4 if its is None else its)
        assert ok == accepted


@pytest.mark.parametrize("scheme", [2, 3, 4])
def test_controller_follows_the_rule(scheme):
    counts = [1, 1, 2, 5, None, 3, 0, 1, 4, 2] + [2] * 40
    steps, rejected, hist, t = _replay(counts, 0.2, fs_cfl=2.0, scheme=scheme)
    _check_rule(hist, 2.0 * 0.01)
    assert steps == sum(1 for a in hist if a[3]) and rejected == len(hist) - steps == 3
    # the accepted steps reach t_end exactly; the last one is clipped
    assert t == pytest.approx(0.2, rel=1e-12)
    assert sum(h for _, h, _, a in hist if a) == pytest.approx(0.2, rel=1e-12)
    assert hist[-1][1] <= hist[-1][0]


def test_controller_grows_after_one_iteration():
    steps, rejected, hist, _ = _replay([1] * 10, 0.05, fs_cfl=1.0, scheme=3)
    assert rejected == 0 and all(a[2] == 1 for a in hist)
    assert hist[1][0] == pytest.approx(1.05 * hist[0][0], rel=1e-14)


def test_fixed_dt_and_attempt_limit():
    steps, rejected, hist, _ = _replay([0, 1, 5, 1, 1] + [1] * 40, 1.0, fs_cfl=1.0, enlarge=0)
    dts = [a[0] for a in hist]
    assert all(b <= a * (1 + 1e-15) for a, b in zip(dts, dts[1:]))   # never enlarged
    assert rejected == 1 and dts[3] == pytest.approx(0.85 * dts[0], rel=1e-14)
    steps, rejected, hist, t = _replay([5] * 100, 1.0, fs_cfl=1.0, max_attempts=7)
    assert len(hist) == 7 and steps == 0 and rejected == 7 and t == 0.0


def test_dt_floor_and_option_checks():
    import paper_2609_16424_b300 as lh
    with pytest.raises(lh.LHError) as ei:
        _replay([None] * 200, 1.0, fs_cfl=1.0, dt_min=1e-3)
    assert ei.value.status == 5          # LH_ENOCONV once dt < dt_min
    for bad in ({"scheme": 5}, {"shrink": 1.2}, {"grow_its": 4, "reject_its": 4}, {"max_steps": 0}):
        with pytest.raises(lh.LHError) as ei:
            _replay([2], 1.0, **bad)
        assert ei.value.status == 1


def test_first_dt_from_dt0():
    steps, rejected, hist, _ = _replay([2] * 10, 0.05, dt0=0.02)
    assert hist[0][0] == 0.02 and steps == 3 and rejected == 0
