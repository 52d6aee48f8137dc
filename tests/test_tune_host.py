"""The autotuner's choice rule (host logic, no GPU): the fastest candidate whose compression
ratio is within ratio_slack of the best ratio, over the product of the candidate lists."""
from paper_2511_04140_gb300 import tune


def test_choice_rule(monkeypatch):
    table = {  # (block, c_ctas, d_ctas) -> (gbs, ratio)
        (512, 0, 0): (500.0, 0.80), (512, 3, 0): (520.0, 0.80),
        (1024, 0, 0): (600.0, 0.70), (1024, 3, 0): (650.0, 0.70),
        (1025, 0, 0): (700.0, 0.72), (1025, 3, 0): (720.0, 0.75),
    }
    seen = []

    def fake(sample, block, c, d, reps=3):
        seen.append((block, c, d))
        g, r = table[(block, c, d)]
        return {"block": block, "compress_ctas_per_sm": c, "decompress_ctas_per_sm": d, "gbs": g, "ratio": r}

    monkeypatch.setattr(tune, "measure", fake)
    out = tune.autotune([], blocks=(512, 1024, 1025), compress_ctas=(0, 3), decompress_ctas=(0,), ratio_slack=0.05)
    assert sorted(seen) == sorted(table)
    # within 5 % of the best ratio 0.70: ratios <= 0.735 -> (1024, *) and (1025, 0, 0); fastest is 700
    assert (out["choice"]["block"], out["choice"]["compress_ctas_per_sm"]) == (1025, 0)
    out = tune.autotune([], blocks=(512, 1024, 1025), compress_ctas=(0, 3), decompress_ctas=(0,), ratio_slack=0.0)
    assert (out["choice"]["block"], out["choice"]["compress_ctas_per_sm"]) == (1024, 3)
    assert len(out["table"]) == 6
