"""Host logic of the autotuner with a fake timer (no GPU)."""
import json

from paper_2510_02894_gb300 import autotune


def test_staged_search_picks_fastest(tmp_path):
    state = {"tile": 128, "threads": 128, "ctas_per_sm": 8, "cell_shift": 4}

    def set_tuning(**kw):
        state.update(kw)

    def get_tuning():
        return dict(state)

    # a cost with its minimum at cell_shift 3, tile 256 / 128 threads, 16 CTAs per SM
    def cost():
        return (abs(state["cell_shift"] - 3) * 5 + (0 if (state["tile"], state["threads"]) == (256, 128) else 3) +
                abs(state["ctas_per_sm"] - 16) * 0.1 + 1.0)

    calls = []

    def time_ms(run, reps):
        run()
        calls.append(dict(state))
        return cost()

    cache = tmp_path / "t.json"
    best, table = autotune.tune(lambda: None, "lbl", time_ms=time_ms, set_tuning=set_tuning, get_tuning=get_tuning,
                                cache_path=str(cache))
    assert best == {"tile": 256, "threads": 128, "ctas_per_sm": 16, "cell_shift": 3}
    assert state == best  # left applied
    assert len(table) == 1 + 2 + 6 + 3
    assert len(calls) == len(table) + 2  # the winner confirmed against the start
    data = json.load(open(cache))
    assert data["lbl"]["config"] == best
    state.update(tile=64, threads=64)
    assert autotune.apply("lbl", str(cache), set_tuning=set_tuning) == best and state == best
    assert autotune.apply("missing", str(cache), set_tuning=set_tuning) is None


def test_gain_within_margin_keeps_start(tmp_path):
    """A configuration only 0.5 % faster (timing noise) does not replace the start."""
    state = {"tile": 128, "threads": 128, "ctas_per_sm": 8, "cell_shift": 4}

    def set_tuning(**kw):
        state.update(kw)

    def time_ms(run, reps):
        return 1.0 - (0.005 if state["cell_shift"] == 5 else 0.0)

    best, _ = autotune.tune(lambda: None, "n", time_ms=time_ms, set_tuning=set_tuning,
                            get_tuning=lambda: dict(state), cache_path=str(tmp_path / "n.json"))
    assert best["cell_shift"] == 4 and state == best


def test_bucket_labels():
    assert autotune.bucket(1, 468476) == "rois2^0_verts2^19"
    assert autotune.bucket(256, 3_000_000) == "rois2^8_verts2^22"
