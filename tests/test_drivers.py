"""Host logic of the load-stepping drivers (no GPU): the schedule candidates of the autotuner."""
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
