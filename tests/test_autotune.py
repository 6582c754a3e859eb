"""Host logic of the schedule autotuner (no GPU): the coordinate search, the
validity rules it shares with the library, and the keyword split."""
from paper_2110_12511_gb300 import autotune as at


def test_coordinate_search_finds_separable_optimum():
    # a separable cost: each knob has one best value; the search must find all of them
    best_vals = {"graph_rounds": True, "warp_max_w": 256, "group_max_w": 1024, "item_w": 131072, "bucket_shift": 16,
                 "count_scratch": 1, "fd_cluster_min": 8192}

    def measure(cfg):
        return 1.0 + sum(0.1 for k, v in best_vals.items() if cfg.get(k) != v)

    cfg, t, table = at.coordinate_search(measure)
    assert cfg == best_vals
    assert abs(t - 1.0) < 1e-12
    assert len(table) <= 1 + sum(len(v) for v in at.SPACE.values())


def test_coordinate_search_skips_invalid_and_keeps_default_on_ties():
    seen = []

    def measure(cfg):
        seen.append(dict(cfg))
        return 1.0

    cfg, _, _ = at.coordinate_search(measure, space={"warp_max_w": [0, 1024], "group_max_w": [0, 128]})
    assert cfg == at.DEFAULT  # ties keep the incumbent
    assert all(at.valid(c) for c in seen)
    assert not any(c.get("warp_max_w") == 1024 for c in seen)  # above the warp class limit
    assert not any(c.get("group_max_w") == 128 for c in seen)  # below the default warp limit


def test_valid_and_split():
    assert at.valid(at.DEFAULT)
    assert not at.valid({"warp_max_w": 600})
    assert not at.valid({"warp_max_w": 256, "group_max_w": 128})
    assert not at.valid({"item_w": 1000})
    assert not at.valid({"bucket_shift": 12})
    assert not at.valid({"count_scratch": 4})
    kw = at.split({"graph_rounds": True, "warp_max_w": 128, "item_w": 8192, "bucket_shift": 16, "count_scratch": 2,
                   "fd_cluster_min": 8192})
    assert kw == {"graph_rounds": True, "bucket_shift": 16,
                  "schedule": {"warp_max_w": 128, "group_max_w": 0, "item_w": 8192, "count_scratch": 2,
                               "fd_cluster_min": 8192}}
