"""Host logic of the load-stepping drivers (no GPU): the schedule candidates of the autotuner, the
adaptive displacement path of the strip footing (on a stand-in context), the external work."""
import numpy as np
import pytest

from paper_1805_04155_gb300 import drivers as D
from paper_1805_04155_gb300 import ep


def test_schedule_candidates_cover_precisions_methods_and_preconditioners():
    sym = D.schedule_candidates(True, {"newton_rtol": 1e-10})
    non = D.schedule_candidates(False)
    assert len(sym) == len(non) == 8
    assert {c["krylov"] for c in sym} == {1, 3} and {c["krylov"] for c in non} == {2, 3}   # CG only if symmetric
    for cs in (sym, non):
        assert {c["precision"] for c in cs} == {ep.EP_FP64, ep.EP_MIXED}
        assert {c["precond"] for c in cs} == {1, 2}
        assert len({tuple(sorted(c.items())) for c in cs}) == len(cs)
    assert all(c["newton_rtol"] == 1e-10 for c in sym)


class _FakeFooting:
    """A context stand-in whose footing pressure follows p(u) = min(k u, p_lim) (rigid-plastic limit),
    and whose solve fails for increments above `du_fail` (a Newton failure on a too-large step)."""

    def __init__(self, k=100.0, p_lim=5.0, du_fail=0.05, n_nodes=4, dim=2):
        self.k, self.p_lim, self.du_fail = k, p_lim, du_fail
        self.u = 0.0
        self.dim = dim
        self.n_nodes = n_nodes
        self.calls = []
        self.h = None

    def solve_load_path(self, zeta, opts, raise_on_error=True):
        z = float(zeta[-1])
        self.calls.append(z - self.u)
        if z - self.u > self.du_fail:
            return ep.EP_ERR_NEWTON_NO_CONVERGENCE, []
        self.u = z
        return ep.EP_OK, [object()]

    def get(self, field):
        assert field == ep.EP_F_INT
        F = np.zeros((self.n_nodes, self.dim))
        p = min(self.k * self.u, self.p_lim)
        F[:2, self.dim - 1] = -p * 1.0 / 2      # two footing nodes share the load of a unit-width footing
        return F.ravel()


class _Problem:
    extra = {"footing_nodes": np.array([0, 1]), "footing": 1.0}


def test_strip_footing_path_doubles_on_the_plateau_and_halves_on_failure(monkeypatch):
    import numpy as np_
    ctx = _FakeFooting()
    monkeypatch.setattr(ep, "default_opts", lambda **kw: None)
    us, ps, _ = D.strip_footing_path(ctx, _Problem(), u_max=0.3, du0=0.01, soft=0.1)
    steps = np_.diff(np_.concatenate([[0.0], us]))
    assert abs(us[-1] - 0.3) < 1e-12
    assert np_.all(np_.diff(ps) >= -1e-12) and abs(ps[-1] - 5.0) < 1e-12
    assert steps[0] == 0.01
    # elastic (slope k) until p_lim at u = 0.05: the increment stays 0.01; on the plateau it doubles
    assert np_.allclose(steps[:5], 0.01)
    assert steps.max() <= ctx.du_fail + 1e-12      # larger increments failed and were halved
    assert any(c > ctx.du_fail for c in ctx.calls)  # a failure happened and was recovered
    assert len(us) < 0.3 / 0.01                     # fewer steps than a uniform path


def test_external_work_is_the_load_times_displacement():
    class P:
        f_unit = np.array([1.0, -2.0, 0.5])

    class Ctx:
        def get(self, field):
            assert field == ep.EP_U
            return np.array([2.0, 1.0, 4.0])
    assert D.external_work(Ctx(), P()) == 2.0


class _FakeTuneCtx:
    """Stand-in context for the autotuner: each schedule takes a set time per step (or fails), and the
    state fields are plain arrays that a solve overwrites."""

    class _Mat:
        model, phi, psi, Hc = ep.EP_VM_ISO, 0.0, 0.0, 0.0

    def __init__(self, times):
        self.times = times                  # (precision, krylov, precond) -> ms per step, or None (fails)
        self.material = self._Mat()
        self.state = {f: np.zeros(3) for f in D.STATE_FIELDS}
        self.trials = []

    def get(self, field):
        return self.state[field]

    def set(self, field, value):
        self.state[field] = np.array(value, copy=True)

    def solve_load_path(self, zeta, opts, raise_on_error=True):
        key = (opts.precision, opts.krylov, opts.precond)
        if (opts.asm_tile, opts.krylov_graphs) != (1, 1):
            key = key + (opts.asm_tile, opts.krylov_graphs)
        # every trial must start from the saved (zero) state
        self.trials.append((key, all(np.all(v == 0.0) for v in self.state.values())))
        for f in self.state:
            self.state[f] = self.state[f] + 1.0
        t = self.times.get(key)
        if t is None:
            return ep.EP_ERR_KRYLOV, []

        class R:
            t_step_ms = t
        return ep.EP_OK, [R() for _ in zeta]


@pytest.fixture(scope="module")
def built():
    """ep.default_opts and the error messages come from the library (host calls only)."""
    from paper_1805_04155_gb300 import build as b
    b.build()


def test_autotune_picks_the_fastest_schedule_and_restores_the_state(built):
    times = {(ep.EP_FP64, 1, 2): 3.0, (ep.EP_FP64, 1, 1): 5.0, (ep.EP_FP64, 3, 2): 2.5, (ep.EP_FP64, 3, 1): None,
             (ep.EP_MIXED, 1, 2): 2.0, (ep.EP_MIXED, 1, 1): None, (ep.EP_MIXED, 3, 2): 4.0, (ep.EP_MIXED, 3, 1): 9.0}
    ctx = _FakeTuneCtx(times)
    best, table = D.autotune(ctx, [0.1, 0.2, 0.3, 0.4], trial_steps=3, kernel_schedules=False)
    assert (best.precision, best.krylov, best.precond) == (ep.EP_MIXED, 1, 2)
    assert len(table) == 8 and sum(t is None for _, t in table) == 2
    assert all(fresh for _, fresh in ctx.trials)                 # each trial started from the saved state
    assert all(np.all(v == 0.0) for v in ctx.state.values())     # and the state is restored at the end
    assert dict(((c["precision"], c["krylov"], c["precond"]), t) for c, t in table)[(ep.EP_FP64, 3, 2)] == \
        3 * 2.5 / 1e3


def test_autotune_second_stage_picks_the_fastest_kernel_schedule(built):
    """Stage 2 varies the assembly tile and the Krylov launch form on the best solver schedule only,
    and keeps the stage-1 schedule when no kernel schedule beats it."""
    times = {(ep.EP_FP64, 1, 2): 3.0, (ep.EP_MIXED, 1, 2): 2.0,
             (ep.EP_MIXED, 1, 2, 2, 1): 1.5, (ep.EP_MIXED, 1, 2, 1, 0): 2.5, (ep.EP_MIXED, 1, 2, 2, 0): None}
    ctx = _FakeTuneCtx(times)
    best, table = D.autotune(ctx, [0.1, 0.2, 0.3], trial_steps=3)
    assert (best.precision, best.krylov, best.precond, best.asm_tile, best.krylov_graphs) == (ep.EP_MIXED, 1, 2, 2, 1)
    stage2 = table[8:]
    assert len(stage2) == 4 and all(c["precision"] == ep.EP_MIXED and c["krylov"] == 1 for c, _ in stage2)
    assert all(fresh for _, fresh in ctx.trials)
    ctx2 = _FakeTuneCtx({(ep.EP_FP64, 1, 2): 3.0, (ep.EP_FP64, 1, 2, 2, 1): 4.0})
    best2, _ = D.autotune(ctx2, [0.1], trial_steps=1)
    assert (best2.precision, best2.asm_tile, best2.krylov_graphs) == (ep.EP_FP64, 1, 1)


def test_autotune_reports_when_every_schedule_fails(built):
    ctx = _FakeTuneCtx({})
    with pytest.raises(ep.EPError):
        D.autotune(ctx, [0.1], trial_steps=1)
