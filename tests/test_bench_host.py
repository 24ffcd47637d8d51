"""CPU checks of the benchmark's host-side bookkeeping: the reference arm runs
the oracle with the library's own defaults, the algorithmic-byte formulas
behind the roofline fractions, and the rule that a committed DRAM-traffic
figure is reported only while its kernel source is unchanged."""
import hashlib
import importlib.util
import os

import pytest

from tests.conftest import ROOT


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test",
                                                  os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_reference_arm_uses_the_library_defaults(bench):
    import paper_2112_10591_gb300 as eb
    p = eb.ebof_default_params(1280, 720)
    ref = bench._reference_params()
    for k, v in ref.items():
        assert getattr(p, k) == pytest.approx(v), k


def test_algorithmic_bytes_per_launch(bench):
    import paper_2112_10591_gb300 as eb
    p = eb.ebof_default_params(1280, 720)
    geo = bench.geo_levels(p)
    assert [g[:2] for g in geo] == [(1280, 720), (640, 360), (320, 180), (160, 90), (80, 45)]
    # 12x12 patches at stride 4, the last one flush with the border
    assert geo[0][2:] == (318, 178)
    P = 1280 * 720
    ab = lambda s, l=0, n=0: bench.algorithmic_bytes_per_launch(s, l, geo, n, P)
    assert ab("var_sor") == 44 * P          # 7 coefficient planes and U in, U out
    assert ab("var_coeff", 1) == 52 * 640 * 360
    assert ab("scatter", -1, 275_000) == 13 * 275_000
    assert ab("patch_search", 4) == 16 * 80 * 45 + 8 * geo[4][2] * geo[4][3]  # no coarser level
    assert ab("unknown") == 0.0


def test_stage_fractions_per_frame(bench):
    # about 250 B per pixel per 1280x720 frame in all (230 MB)
    P = 1280 * 720
    ms = {k: 1.0 for k in ("scatter", "denoise_fill", "edt_cols", "edt_rows_surface", "pyramid",
                           "patch_search", "densify", "var_coeff", "var_sor")}
    out = bench.stage_hbm_fractions(ms, P, 275_000, 5, 5, 6799.3)
    total = out["all stages"]["bytes_per_frame"]
    assert 220e6 < total < 240e6
    a8 = out["A8 variational"]
    assert a8["bytes_per_frame"] == pytest.approx(5 * 24.0 * P * sum(4.0 ** -l for l in range(5)))
    # 2 ms of stage time for those bytes (the fraction is reported to 4 decimals)
    assert a8["frac"] == pytest.approx(a8["bytes_per_frame"] / 2e-3 / 1e9 / 6799.3, abs=1e-4)


def test_traffic_figures_follow_their_sources(bench, tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("// kernel\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic.txt").write_text(
        "# kernel stage level bytes source sha256\n"
        "k var_sor 0 123 k.cu %s\n" % sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.dram_traffic("var_sor", 0) == 123
    assert bench.dram_traffic("var_sor", 1) is None
    src.write_text("// kernel, changed\n")
    assert bench.dram_traffic("var_sor", 0) is None


def test_a8_roofline_reproduces_by_hand(bench):
    # 24 B per level-0 pixel per outer iteration over that iteration's
    # coefficient and SOR time; the figures of a level-0 profile of 0.0972 +
    # 0.1124 ms per frame over 5 iterations give 528 GB/s
    P = 1280 * 720
    r = bench.a8_outer_iteration_roofline({"var_coeff": 0.0972, "var_sor": 0.1124}, P, 5, 400,
                                          6799.3, 22161408, 33199104)
    assert r["bytes_per_unit"] == 24 * P
    assert r["us_per_unit"] == pytest.approx((0.0972 + 0.1124) * 1000 / 5)
    assert r["achieved"] == pytest.approx(24 * P / ((0.0972 + 0.1124) / 5 / 1000) / 1e9)
    assert r["achieved"] == pytest.approx(528, abs=1)
    assert r["frac"] == pytest.approx(r["achieved"] / 6799.3)
    assert r["traffic"] == 22161408 + 33199104
    assert bench.a8_outer_iteration_roofline({}, P, 5, 1, 6799.3, None, None) is None


def test_a6_flop_roof(bench):
    import paper_2112_10591_gb300 as eb
    p = eb.ebof_default_params(1280, 720)
    geo = bench.geo_levels(p)
    by = {"all": {}, "0": {"patch_search": 0.08}, "1": {"patch_search": 0.02}}
    r = bench.a6_flop_roof(by, geo, 12, 12, 2070.0)
    f0 = 25 * 144 * 12 * 318 * 178
    assert r["level0"]["flop"] == f0 and f0 == pytest.approx(2.445e9, rel=1e-3)
    assert r["flop_per_frame"] > f0
    assert r["ms_per_frame"] == pytest.approx(0.1)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_both_arms_report_the_same_config(bench):
    import paper_2112_10591_gb300 as eb
    p = eb.ebof_default_params(1280, 720)
    ours = bench.bench_config(bench._params_dict(p), 201, 1)
    ref = bench.bench_config(bench._reference_params(), 201, 1)
    assert ours == ref
