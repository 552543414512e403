"""Host logic of the autotuner: which candidates a round proposes around a
winner (no GPU involved)."""
from paper_2408_09662_gb300.tune import _refinements


def test_one_thread_refinements_follow_the_live_set():
    # 100 live FP32 values: 2 and 4 instances per thread fit, a cap of 128 would not bind
    c = _refinements({"ways": 0}, "f32", 1407, 100)
    assert {"ways": 0, "inst_per_thread": 4} in c and {"ways": 0, "maxrregcount": 128} not in c
    assert {"ways": 0, "maxrregcount": 96} in c and {"ways": 0, "maxrregcount": 64} in c
    # FP64 values take two registers each
    c = _refinements({"ways": 0}, "f64", 1407, 100)
    assert {"ways": 0, "inst_per_thread": 4} not in c and {"ways": 0, "maxrregcount": 128} in c
    # the MPC's 906 live values: no extra instances per thread at all
    c = _refinements({"ways": 0}, "f64", 45171, 906)
    assert all("inst_per_thread" not in x for x in c) and len(c) == 3


def test_reverse_sweep_refinements_assume_a_larger_live_set():
    fwd = _refinements({"ways": 0}, "f32", 1407, 100)
    adj = _refinements({"ways": 0}, "f32", 1407, 100, adjoint=True)
    assert {"ways": 0, "maxrregcount": 128} in adj and {"ways": 0, "maxrregcount": 128} not in fwd
    assert {"ways": 0, "inst_per_thread": 4} in fwd and {"ways": 0, "inst_per_thread": 4} not in adj


def test_cooperative_refinements_are_groups_per_cta():
    c = _refinements({"ways": 4}, "f64", 20000, 300)
    assert c == [{"ways": 4, "coop_groups": 2}, {"ways": 4, "coop_groups": 4}]
    assert _refinements({"ways": 8, "fmad": 0}, "f32", 20000, 300, adjoint=True)[0] == \
        {"ways": 8, "fmad": 0, "coop_groups": 2}
