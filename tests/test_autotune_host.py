"""Host logic of the autotuner: the confirmation stage re-rates the fastest distinct tunings of the descent
on a longer run and lets that run decide (no GPU: the rate function is a stand-in)."""
from paper_1401_7494_gb300 import autotune


def _t(k, z):
    return {"views_per_pass": k, "zrun": z, "xvec": 1, "block_x": 8, "block_y": 16, "gather": 5, "tex_zrun": 0}


def test_confirm_best_re_rates_the_top_distinct_tunings():
    trials = [{"tuning": _t(16, 8), "gups": 1300.0},
              {"tuning": _t(32, 16), "gups": 1320.0},
              {"tuning": _t(32, 16), "gups": 1320.0},          # the same tuning seen twice
              {"tuning": _t(24, 8), "gups": 1290.0},
              {"tuning": _t(8, 8), "gups": 1100.0}]
    long_run = {(16, 8): 1250.0, (32, 16): 1200.0, (24, 8): 1265.0, (8, 8): 2000.0}
    calls = []

    def rate(t):
        calls.append((t["views_per_pass"], t["zrun"]))
        return long_run[(t["views_per_pass"], t["zrun"])]

    best, gups, rows = autotune.confirm_best(trials, rate, top=3)
    assert calls == [(32, 16), (16, 8), (24, 8)]            # fastest first, duplicates once, fourth not run
    assert best == _t(24, 8) and gups == 1265.0              # the long run decides
    assert [(r[1], r[2]) for r in rows] == [(1320.0, 1200.0), (1300.0, 1250.0), (1290.0, 1265.0)]


def test_confirm_best_with_fewer_trials_than_top():
    best, gups, rows = autotune.confirm_best([{"tuning": _t(16, 8), "gups": 5.0}], lambda t: 7.0, top=3)
    assert best == _t(16, 8) and gups == 7.0 and len(rows) == 1


def test_tuning_cache_round_trip_and_fallbacks(tmp_path):
    from paper_1401_7494_gb300 import tuning
    path = tmp_path / "cache.json"
    gpu = "Test GPU"
    assert tuning.lookup(512, "f32", "soft", gpu=gpu, path=path) == tuning.DEFAULT        # empty cache
    tuning.store(512, "f32", "soft", _t(24, 8), 1268.0, gpu=gpu, path=path)
    assert tuning.lookup(512, "f32", "soft", gpu=gpu, path=path) == _t(24, 8)
    # a block-frame key without its own entry falls back to the global-frame entry ...
    assert tuning.lookup(512, "f32", "soft", gpu=gpu, path=path, frame="block") == _t(24, 8)
    # ... and uses its own once stored, without touching the global one
    tuning.store(512, "f32", "soft", _t(32, 16), 1228.0, gpu=gpu, path=path, frame="block")
    assert tuning.lookup(512, "f32", "soft", gpu=gpu, path=path, frame="block") == _t(32, 16)
    assert tuning.lookup(512, "f32", "soft", gpu=gpu, path=path) == _t(24, 8)
    # other keys and other GPUs get the default
    assert tuning.lookup(1024, "f32", "soft", gpu=gpu, path=path) == tuning.DEFAULT
    assert tuning.lookup(512, "f16", "soft", gpu=gpu, path=path) == tuning.DEFAULT
    assert tuning.lookup(512, "f32", "soft", gpu="Other GPU", path=path) == tuning.DEFAULT
    # the default drops the x-vector for a volume it does not divide
    assert tuning.lookup(37, "f32", "soft", gpu=gpu, path=path)["xvec"] == 1


def test_search_leaves_out_what_the_library_rejects():
    """The view split is searched only with software interpolation in the global frame (the library returns
    RCT_ENOTSUP for it with block frames or texture filtering, which once ended a block-frame search)."""
    assert "view_split" in autotune.search_params("soft", "global")
    assert "view_split" not in autotune.search_params("soft", "block")
    assert "view_split" not in autotune.search_params("tex", "global")
    assert "gather" not in autotune.search_params("tex", "global")
    assert autotune.search_params("soft", "block") == ["gather", "views_per_pass", "zrun", "xvec", "block"]
