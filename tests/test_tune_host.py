"""The autotuner's search and choice rule (host logic, no GPU): every block size and CTA shape
at the occupancy limit, then the resident-CTA caps at the best of those; the fastest
candidate whose compression ratio is within ratio_slack of the best ratio wins."""
from paper_2511_04140_gb300 import tune


def test_choice_rule(monkeypatch):
    # (block, c_ctas, d_ctas, c_warps, d_warps) -> (gbs, ratio)
    def perf(block, c, d, cw, dw):
        base = {512: (500.0, 0.80), 1024: (600.0, 0.70), 1025: (700.0, 0.72)}[block]
        return base[0] + 10 * (cw == 8) + 5 * (dw == 2) + 20 * (c == 3), base[1]

    seen = []

    def fake(sample, block, c, d, reps=3, cw=4, dw=4):
        seen.append((block, c, d, cw, dw))
        g, r = perf(block, c, d, cw, dw)
        return {"block": block, "compress_ctas_per_sm": c, "decompress_ctas_per_sm": d,
                "compress_warps_per_cta": cw, "decompress_warps_per_cta": dw, "gbs": g, "ratio": r}

    monkeypatch.setattr(tune, "measure", fake)
    out = tune.autotune([], blocks=(512, 1024, 1025), compress_ctas=(0, 3), decompress_ctas=(0,),
                        compress_warps=(4, 8), decompress_warps=(2, 4), ratio_slack=0.05)
    # first pass: 3 blocks x 2 x 2 shapes at (0, 0); second pass: the caps at the best shape
    assert len(seen) == 12 + 1
    assert seen[-1] == (1025, 3, 0, 8, 2)
    c = out["choice"]
    assert (c["block"], c["compress_ctas_per_sm"], c["compress_warps_per_cta"], c["decompress_warps_per_cta"]) == \
        (1025, 3, 8, 2)
    # no slack: only block 1024 (best ratio) qualifies
    seen.clear()
    out = tune.autotune([], blocks=(512, 1024, 1025), compress_ctas=(0, 3), decompress_ctas=(0,),
                        compress_warps=(4, 8), decompress_warps=(2, 4), ratio_slack=0.0)
    assert out["choice"]["block"] == 1024 and out["choice"]["compress_ctas_per_sm"] == 3
