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


def test_cache_key_separates_what_changes_the_choice(monkeypatch):
    import types
    import torch
    from paper_2408_09662_gb300 import tune
    props = types.SimpleNamespace(name="GB300", major=10, minor=3)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda device: props)
    ir, other = b"program-a", b"program-b"
    k = tune._key(ir, "f32", 65536, {"fmad": 0}, "cuda:0")
    assert k.startswith(__import__("hashlib").sha256(ir).hexdigest()[:20] + "|GB300|sm_103|f32|N<=65536|fmad=0")
    # same bucket (next power of two), different buckets, dtypes, programs, fixed options
    assert tune._key(ir, "f32", 40000, {"fmad": 0}, "cuda:0") == k
    assert tune._key(ir, "f32", 65537, {"fmad": 0}, "cuda:0") != k
    assert tune._key(ir, "f64", 65536, {"fmad": 0}, "cuda:0") != k
    assert tune._key(other, "f32", 65536, {"fmad": 0}, "cuda:0") != k
    assert tune._key(ir, "f32", 65536, {}, "cuda:0") != k
    # fixed options in any order give one key
    assert tune._key(ir, "f32", 1, {"a": 1, "b": 2}, "cuda:0") == tune._key(ir, "f32", 1, {"b": 2, "a": 1}, "cuda:0")
    # the reverse sweep's choice is kept apart from the forward one
    ka = tune._key(ir, "f32", 65536, {"fmad": 0}, "cuda:0", "adjoint(reduce_broadcast=True)")
    assert ka != k and ka.startswith(k)


def test_cache_file_round_trip(tmp_path):
    from paper_2408_09662_gb300 import tune
    path = str(tmp_path / "sub" / "tuning.json")
    assert tune._load_cache(path) == {}
    tune._store_cache(path, "k1", {"options": {"ways": 4}, "ms": 1.0})
    tune._store_cache(path, "k2", {"options": {"ways": 0}, "ms": 2.0})
    d = tune._load_cache(path)
    assert d["k1"]["options"] == {"ways": 4} and d["k2"]["ms"] == 2.0
    open(path, "w").write("{not json")
    assert tune._load_cache(path) == {}          # a damaged file is ignored, not fatal
