"""Host logic of the ablation tables: the quality/cost choice and the Pareto
front, on hand-made rows."""
from paper_2512_04556_gb300 import ablation

ROWS = [
    dict(L=1, T=8, taps=8, median_rel_mse=0.30, filter_4k_ms=0.4),
    dict(L=2, T=8, taps=16, median_rel_mse=0.12, filter_4k_ms=0.6),
    dict(L=4, T=4, taps=16, median_rel_mse=0.15, filter_4k_ms=0.7),
    dict(L=4, T=8, taps=32, median_rel_mse=0.05, filter_4k_ms=1.0),
    dict(L=2, T=16, taps=32, median_rel_mse=0.04, filter_4k_ms=1.1),
    dict(L=4, T=16, taps=64, median_rel_mse=0.01, filter_4k_ms=1.9),
    dict(L=8, T=4, taps=32, median_rel_mse=0.09, filter_4k_ms=1.5),
]


def test_choose_cheapest_meeting_target():
    c = ablation.choose(ROWS, 0.2, "taps")
    assert (c["L"], c["T"]) == (2, 8)          # 16 taps; (4, 4) ties on taps but is worse
    c = ablation.choose(ROWS, 0.045, "filter_4k_ms")
    assert (c["L"], c["T"]) == (2, 16)
    c = ablation.choose(ROWS, 0.05, "filter_4k_ms")
    assert (c["L"], c["T"]) == (4, 8)
    assert ablation.choose(ROWS, 0.001) is None


def test_pareto_front():
    front = [(r["L"], r["T"]) for r in ablation.pareto(ROWS)]
    assert front == [(1, 8), (2, 8), (4, 8), (2, 16), (4, 16)]
    # every dropped row is dominated by a front row
    for r in ROWS:
        if (r["L"], r["T"]) in front:
            continue
        assert any(f["filter_4k_ms"] <= r["filter_4k_ms"] and f["median_rel_mse"] <= r["median_rel_mse"]
                   for f in ablation.pareto(ROWS))
