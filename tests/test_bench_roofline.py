"""The benchmark's roofline arithmetic on hand-made profiles (no GPU): each
kind of work is weighed at its own rate, a class is bound by the longer of
its integer-pipe and HBM times, and a multi-kernel operation's roof is the sum
of its kernels' own roof times."""
import pytest

import bench

RATES = {"per_second": 1.0e12, "mac_per_second": 2.0e12, "mac3_per_second": 4.0e12,
         "butterfly_per_second": 0.5e12}


@pytest.fixture(autouse=True)
def fixed_rates(monkeypatch):
    for k, v in RATES.items():
        monkeypatch.setitem(bench.ALU_PEAK, k, v)


def prof(ms, bfly=0.0, shoup=0.0, mac=0.0, mac3=0.0, by=0.0, launches=1):
    return {"ms": ms, "work": bfly + shoup + mac + mac3, "bfly": bfly, "mac": mac, "mac3": mac3, "bytes": by,
            "launches": launches}


def test_each_kind_at_its_own_rate():
    # 1e9 of each kind: 2 ms + 1 ms + 0.5 ms + 0.25 ms = 3.75 ms at the roof
    p = prof(7.5, bfly=1e9, shoup=1e9, mac=1e9, mac3=1e9)
    r = bench.class_roof(p, hbm_peak=1000.0, peak_kind="test", name="ks_ntt_rot_products")
    assert r["bound"] == "alu"
    assert r["frac"] == pytest.approx(3.75 / 7.5)
    assert r["peak"] == pytest.approx(4e9 / 3.75e-3 / 1e9)
    assert r["achieved"] == pytest.approx(4e9 / 7.5e-3 / 1e9)
    assert r["work_mix"] == {"butterflies": 1e9, "shoup_products": 1e9, "macs": 1e9, "split_macs": 1e9}
    assert r["frac_shoup_only"] == pytest.approx(4e9 / 7.5e-3 / RATES["per_second"])
    assert bench.roof_time(p, 1000.0) == pytest.approx(3.75e-3)


def test_hbm_bound_class():
    # 1e8 products (0.1 ms) but 10 GB at 1000 GB/s (10 ms): bound by HBM
    p = prof(20.0, shoup=1e8, by=10e9)
    r = bench.class_roof(p, hbm_peak=1000.0, peak_kind="test", name="ntt")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx(10.0 / 20.0)
    assert bench.roof_time(p, 1000.0) == pytest.approx(10e-3)


def test_butterfly_chain_fraction_counts_butterflies_only():
    # an inverse transform: 1e9 butterflies (2 ms) plus 1e8 scaling products (0.1 ms) in 4.2 ms
    p = prof(4.2, bfly=1e9, shoup=1e8)
    r = bench.class_roof(p, hbm_peak=1e6, peak_kind="test", name="intt")
    assert r["frac"] == pytest.approx(2.1 / 4.2)
    assert r["butterfly_chain_frac"] == pytest.approx((1e9 / 4.2e-3) / RATES["butterfly_per_second"])


def test_composite_roof_takes_each_kernels_own_bound():
    # an integer-bound kernel (roof 2 ms of 4 ms) and an HBM-bound one (roof 5 ms of 6 ms): 7/10;
    # the two summed into one class are bound by the larger of the summed times, max(2.1, 5) / 10
    a = prof(4.0, bfly=1e9)
    b = prof(6.0, shoup=1e8, by=5e9)
    t_roof = bench.roof_time(a, 1000.0) + bench.roof_time(b, 1000.0)
    assert t_roof / 10e-3 == pytest.approx(0.7)
    summed = {k: a[k] + b[k] for k in a}
    r = bench.class_roof(summed, hbm_peak=1000.0, peak_kind="test", name="op", integer=True)
    assert r["frac"] == pytest.approx(0.5)
    assert t_roof / 10e-3 >= r["frac"]  # a sum of maxima is never below the maximum of the sums


def test_traffic_ratio_from_its_capture():
    assert 0.5 < bench.KS_ROT_TRAFFIC_PER_ALG_BYTE < 1.5
