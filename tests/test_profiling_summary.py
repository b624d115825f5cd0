"""The launch-list summarizer behind the committed ncu summaries (paper_2308_16395_gb300/profiling.py)
on a small synthetic ncu CSV: launch order kept, kernel names shortened, units converted, totals,
shares, per-unit times and DRAM bytes per launch as defined."""

import pytest

from paper_2308_16395_gb300 import profiling

HEAD = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
        '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n')


def _row(i, kernel, metric, unit, value):
    return (f'"{i}","1","python3","h","{kernel}","1","7","(512, 1, 1)","(152, 1, 1)","0","10.3",'
            f'"Command line profiler metrics","{metric}","{unit}","{value}"\n')


def test_summary_of_a_launch_list(tmp_path):
    p = tmp_path / "launches.csv"
    rows = [
        "==PROF== a line ncu prints that is not CSV\n", HEAD,
        _row(0, "void k_init(Ctl *, int)", "gpu__time_duration.sum", "usecond", "5"),
        _row(1, "void k_tc_pass16<1, 0>(Ctl *, int, CUtensorMap_st)", "gpu__time_duration.sum", "nsecond", "180,000"),
        _row(1, "void k_tc_pass16<1, 0>(Ctl *, int, CUtensorMap_st)", "dram__bytes_read.sum", "Mbyte", "600"),
        _row(1, "void k_tc_pass16<1, 0>(Ctl *, int, CUtensorMap_st)", "dram__bytes_write.sum", "Kbyte", "500"),
        _row(2, "void k_decide(Ctl *, int)", "gpu__time_duration.sum", "usecond", "10"),
        _row(3, "void k_tc_pass16<1, 0>(Ctl *, int, CUtensorMap_st)", "gpu__time_duration.sum", "msecond", "0.2"),
        _row(3, "void k_tc_pass16<1, 0>(Ctl *, int, CUtensorMap_st)", "dram__bytes_read.sum", "byte", "400000000"),
        _row(3, "void k_tc_pass16<1, 0>(Ctl *, int, CUtensorMap_st)", "dram__bytes_write.sum", "byte", "1500000"),
    ]
    p.write_text("".join(rows))
    launches = profiling.read(str(p))
    assert [L["id"] for L in launches] == [0, 1, 2, 3]
    assert [L["kernel"] for L in launches] == ["k_init", "k_tc_pass16<1, 0>", "k_decide", "k_tc_pass16<1, 0>"]
    assert launches[1]["metrics"]["gpu__time_duration.sum"] == 180000.0
    assert launches[1]["metrics"]["dram__bytes_read.sum"] == 600e6
    assert launches[3]["metrics"]["gpu__time_duration.sum"] == 200000.0
    out, total_us = profiling.summarize(launches[1:], per=2.0)       # the first launch skipped
    assert total_us == pytest.approx(390.0)
    top = out[0]
    assert top["kernel"] == "k_tc_pass16<1, 0>" and top["launches"] == 2
    assert top["total_us"] == pytest.approx(380.0) and top["avg_us"] == pytest.approx(190.0)
    assert top["share"] == pytest.approx(380.0 / 390.0)
    assert top["per_unit_us"] == pytest.approx(190.0)
    assert top["dram_mb_per_launch"] == pytest.approx((600e6 + 0.5e6 + 400e6 + 1.5e6) / 2 / 1e6)
    assert out[1]["kernel"] == "k_decide" and out[1]["dram_mb_per_launch"] == 0.0
    assert sum(r["share"] for r in out) == pytest.approx(1.0)
