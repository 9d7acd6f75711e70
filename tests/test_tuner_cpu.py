"""Host logic of the batched tuner (no GPU): size classes, the candidate plans it times, and the
committed GB300 table -- every plan it can hand to the library passes the library's own plan
validation, and arrays outside the table fall back to their default plan."""
import paper_2302_03317_gb300 as rip
from paper_2302_03317_gb300 import tuner


def _valid(plan, n, w):
    return rip.rip_shuffle_workspace_size(n, w, plan) > 0


def test_size_class_is_floor_log2():
    assert tuner.size_class(1) == 0
    assert tuner.size_class(255) == 7
    assert tuner.size_class(256) == 8
    assert tuner.size_class((1 << 20) - 1) == 19
    assert tuner.size_class(1 << 20) == 20


def test_every_candidate_is_a_valid_plan():
    for c in range(tuner.CLASS_LO, tuner.CLASS_HI + 1):
        for w in (4, 8):
            cands = tuner.candidate_plans(c, w)
            assert cands, c
            keys = {(tuple(p.ks), tuple(p.Ts), tuple(p.Bs)) for p in cands}
            assert len(keys) == len(cands)  # no duplicates
            for p in cands:
                assert p.base == tuner.BASE
                assert all(t % b == 0 for t, b in zip(p.Ts, p.Bs))
                assert _valid(p, 1 << c, w) and _valid(p, (2 << c) - 1, w)


def test_committed_table_covers_the_classes_with_valid_plans():
    table = tuner.load_table(tuner.default_table_path(4))
    assert table["elem_bytes"] == 4
    classes = sorted(int(c) for c in table["classes"])
    assert classes == list(range(tuner.CLASS_LO, tuner.CLASS_HI + 1))
    for c in classes:
        (p,) = tuner.plans_for([1 << c], table)
        assert _valid(p, 1 << c, 4) and _valid(p, (2 << c) - 1, 4)


def test_plans_for_uses_the_class_entry_or_the_default_plan():
    table = tuner.load_table(tuner.default_table_path(4))
    e = table["classes"]["12"]
    inside, below, above = tuner.plans_for([5000, 100, 1 << 22], table)
    assert list(inside.ks) == e["ks"] and list(inside.Ts) == e["Ts"] and list(inside.Bs) == e["Bs"]
    for n, p in ((100, below), (1 << 22, above)):
        d = rip.rip_default_plan(n, 4)
        assert (list(p.ks), list(p.Ts), list(p.Bs), p.base) == (list(d.ks), list(d.Ts), list(d.Bs), d.base)
