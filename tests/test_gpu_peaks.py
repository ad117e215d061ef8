"""The ALU microbenchmarks run and return plausible figures."""
import pytest

pytestmark = pytest.mark.gpu


def test_alu_peaks():
    from paper_1911_10487_gb300 import build
    build.build()
    from paper_1911_10487_gb300._abi import fs_measure_alu_peaks
    r = fs_measure_alu_peaks(0)
    print(r)
    assert r["sms"] > 0 and r["clock_mhz"] > 0
    assert r["fp32_tflops"] > r["fp64_tflops"] > 0
    assert r["fp64_fma_cycles_1lane"] > 0 and r["fp64_div_cycles_1lane"] > r["fp64_fma_cycles_1lane"]
