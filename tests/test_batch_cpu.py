"""Host logic of batched uneven populations: the partition into classes, the
price grids and the autotuner's candidate names (no GPU)."""
import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2410_22165_gb300.batch import autotune, plan_classes, price_grid  # noqa: E402

rng = np.random.default_rng(0)
POPS = rng.choice([10, 50, 100, 250, 500], 300).tolist() + [1, 31, 32, 33, 64, 65, 256, 257]
LEVELS = rng.choice([5, 10, 20], len(POPS)).tolist()


@pytest.mark.parametrize("granularity", ["exact", "pow2", "coarse", "by_actions"])
def test_every_environment_in_exactly_one_class(granularity):
    classes = plan_classes(POPS, LEVELS, granularity)
    seen = sorted(e for _, _, idx in classes for e in idx)
    assert seen == list(range(len(POPS)))
    for P, A_max, idx in classes:
        assert all(LEVELS[e] == P for e in idx)                 # a class shares its action space
        assert A_max == max(POPS[e] for e in idx)               # CTA size of its largest population
    keys = [(P, A_max) for P, A_max, _ in classes]
    if granularity == "exact":
        assert len(classes) == len(set(zip(POPS, LEVELS)))
        assert all(len({POPS[e] for e in idx}) == 1 for _, _, idx in classes)
    elif granularity == "pow2":
        def pow2(a):
            n = 32
            while n < a:
                n *= 2
            return n
        assert all(len({pow2(POPS[e]) for e in idx}) == 1 for _, _, idx in classes)
    elif granularity == "coarse":
        bucket = lambda a: 64 if a <= 64 else 256 if a <= 256 else 1024
        assert all(len({bucket(POPS[e]) for e in idx}) == 1 for _, _, idx in classes)
    else:
        assert len(classes) == len(set(LEVELS))
    assert len(set(keys)) == len(keys) or granularity != "by_actions"


def test_unknown_granularity_is_refused():
    with pytest.raises(ValueError):
        plan_classes(POPS, LEVELS, "fine")


def test_price_grids():
    for P in (3, 5, 10, 20):
        g = price_grid(P)
        assert g["P"] == P and g["price_ticks"] == list(range(1, P + 1))
        prices = [g["price_tick"] * k for k in g["price_ticks"]]
        assert np.allclose(prices, [(k + 1) * 10.0 / P for k in range(P)])


def test_autotune_refuses_unknown_candidates_before_any_work():
    with pytest.raises(ValueError):
        autotune(POPS, LEVELS, {}, candidates=("exact+fast",), device="cpu")


def test_candidate_names():
    from paper_2410_22165_gb300.batch import parse_candidate
    assert parse_candidate("exact") == ("exact", False, None)
    assert parse_candidate("coarse+merge") == ("coarse", True, None)
    assert parse_candidate("pow2+chains3") == ("pow2", False, 3)
    assert parse_candidate("exact+merge+chains2") == ("exact", True, 2)
    for bad in ("exact+chains5", "exact+chains0", "tiny", "exact+fast"):
        with pytest.raises(ValueError):
            parse_candidate(bad)
    with pytest.raises(ValueError):              # a bad name later in the list: refused before any work
        autotune(POPS, LEVELS, {}, candidates=("exact", "pow2+chains9"), device="cpu")
