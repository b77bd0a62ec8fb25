"""bench.py's roofline line on CPU, from fabricated per-class profile figures:
achieved = the class's algorithmic work / its summed CUDA-event time,
frac = achieved / peak, and the DRAM traffic only where a capture of the
current kernel is recorded."""
import pytest

import bench


def _r(dom, ms, launches, nbytes, flops, key=("cube48_x16", "mixed_tf32", "spectral", "ir")):
    return {"peaks": {"hbm_gbs": 6780.0, "sm_max_mhz": 2070.0}, "peak_src": "measured",
            "dominant": dom, "traffic_key": key,
            "prof": {dom: {"ms": ms, "launches": launches, "bytes": nbytes, "flops": flops}}}


def test_double_float_residual_is_an_fp32_pipe_roofline():
    # 2 launches of the 16-right-hand-side 48^3 residual: 109 flops per dof
    dofs = 905969664
    e = bench.roofline_entry(_r("stencil_df", 74.8738, 2, 2 * 24 * dofs, 2 * 109 * dofs))
    peak = 152 * 128 * 2070e6 * 2 / 12 / 1e12
    assert e["bound"] == "alu" and e["unit"] == "TFLOP/s"
    assert e["peak"] == pytest.approx(peak)
    assert e["achieved"] == pytest.approx(2 * 109 * dofs / 74.8738e-3 / 1e12)
    assert e["frac"] == pytest.approx(e["achieved"] / peak)
    assert 0.3 < e["frac"] < 0.5
    assert e["per_launch_ms"] == pytest.approx(37.4369)
    # the kernel changed after its DRAM counters were taken: no traffic figure
    assert e["traffic"] is None and "traffic_source" not in e


def test_bandwidth_class_uses_the_measured_copy_rate():
    e = bench.roofline_entry(_r("spec", 50.0, 10, 300e9, 1e9))
    assert e["bound"] == "hbm" and e["unit"] == "GB/s"
    assert e["achieved"] == pytest.approx(300e9 / 50e-3 / 1e9)
    assert e["frac"] == pytest.approx(e["achieved"] / 6780.0)
    assert e["algorithmic_bytes_per_launch"] == pytest.approx(30e9)
