"""Host-side arithmetic of bench.py: the algorithmic bytes behind the roofline
objects, the voiding of stored ncu traffic when the kernel sources change,
time-to-residual lookup and the whole-job aggregation of one rank.  No GPU."""
import bench


class _FakeProblem:
    """Stands in for stc.Problem: fixed event totals and the face count."""

    def __init__(self, F, ms, cnt):
        self.F, self.ms, self.cnt = F, ms, cnt

    def kernel_timing(self, kind):
        return self.ms, self.cnt

    def field_shape(self, name):
        assert name == "V"
        return (0, self.F)


def _faces(n, nz):
    return 3 * n * n * (n + 1) if nz else 2 * n * (n + 1)


def test_algorithmic_bytes_follow_the_per_cell_rules():
    # 3D 64^3 x 60: SCGS 108 B per cell per sweep over an eighth of the cells;
    # colour residual (3.25 F + 2.5 C) floats per timestep over N + 1 timesteps
    G = _FakeProblem(_faces(64, 64), ms=1.0, cnt=1)
    r, _ = bench.kernel_roofline(G, 0, 3, 64, 64, 60, 6800.0, "measured")
    assert r["algorithmic_bytes_per_launch"] == 108 * 64 ** 3 * 60 / 8 == 212336640
    r, _ = bench.kernel_roofline(G, 1, 3, 64, 64, 60, 6800.0, "measured")
    F, C = _faces(64, 64), 64 ** 3
    assert r["algorithmic_bytes_per_launch"] == 4 * (3.25 * F + 2.5 * C) * 61 == 793292800
    # 2D 128^2 x 40: 80 B per cell per sweep over a quarter of the cells;
    # (4.5 F + 3 C) floats per timestep
    G = _FakeProblem(_faces(128, 0), ms=1.0, cnt=1)
    r, _ = bench.kernel_roofline(G, 0, 2, 128, 0, 40, 6800.0, "measured")
    assert r["algorithmic_bytes_per_launch"] == 80 * 128 ** 2 * 40 / 4 == 13107200
    r, _ = bench.kernel_roofline(G, 1, 2, 128, 0, 40, 6800.0, "measured")
    assert r["algorithmic_bytes_per_launch"] == 4 * (4.5 * _faces(128, 0) + 3 * 128 ** 2) * 41 == 32432640


def test_achieved_and_fraction_are_bytes_over_the_event_average():
    G = _FakeProblem(_faces(64, 64), ms=8.0, cnt=16)      # 0.5 ms per launch
    r, total = bench.kernel_roofline(G, 0, 3, 64, 64, 60, 6800.0, "measured")
    assert total == 8.0 and r["launches_timed"] == 16
    assert abs(r["avg_launch_us"] - 500.0) < 1e-9
    assert abs(r["achieved"] - 212336640 / 0.5e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 6800.0) < 1e-15
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6800.0
    # nothing timed: no roofline object
    assert bench.kernel_roofline(_FakeProblem(10, 0.0, 0), 0, 3, 64, 64, 60, 6800.0, "measured")[0] is None


def test_stored_traffic_is_reported_only_for_the_sources_it_was_measured_on(monkeypatch):
    G = _FakeProblem(_faces(64, 64), ms=1.0, cnt=1)
    stored, digest = bench.MEASURED_TRAFFIC[("scgs", 3)]
    monkeypatch.setattr(bench, "source_digest", lambda kind, dim: digest)
    assert bench.kernel_roofline(G, 0, 3, 64, 64, 60, 6800.0, "measured")[0]["traffic"] == stored
    monkeypatch.setattr(bench, "source_digest", lambda kind, dim: "0" * 16)
    assert bench.kernel_roofline(G, 0, 3, 64, 64, 60, 6800.0, "measured")[0]["traffic"] is None


def test_source_digest_covers_the_listed_kernel_files():
    d = bench.source_digest("scgs", 3)
    assert len(d) == 16 and d == bench.source_digest("cres", 3)   # same files for both 3D kinds
    assert d != bench.source_digest("scgs", 2)


def test_seconds_to_a_residual_is_the_first_crossing():
    hist = [(1.0, 0.1, 1.0), (0.5, 0.2, 1.0), (0.009, 0.3, 0.5), (0.02, 0.4, 0.5), (0.0009, 0.5, 0.5)]
    assert bench.seconds_to(hist, 1e-2) == 0.3
    assert bench.seconds_to(hist, 1e-3) == 0.5
    assert bench.seconds_to(hist, 1e-4) is None
    assert bench.seconds_to([], 1.0) is None


def test_one_rank_aggregate_is_cells_over_the_step_time():
    ms, value = bench.aggregate(500.0, 64 ** 3 * 60 * 4, 1, None)
    assert ms == 500.0 and abs(value - 64 ** 3 * 60 * 4 / 0.5) < 1e-6
