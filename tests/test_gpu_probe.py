"""The FMA-throughput probe behind the arithmetic rooflines (gsm_probe_fma).

Checked against what the B300 datasheet fixes, not against itself: 148 SMs
x 128 FP32 lanes x 2 flops at up to 2.032 GHz bound the FP32 rate from
above (~77 TFLOP/s), the FP64 rate is a small fraction of it, and a packed
pair instruction does two lanes' work in one issue slot, so its flop rate
cannot be below the scalar one by more than scheduling noise."""
import math

import pytest

from gpu_common import gsm

pytestmark = pytest.mark.gpu


def test_probe_rates_are_physical():
    g = gsm()
    fp64, fp32, fp32x2 = (g.probe_fma(k) for k in (0, 1, 2))
    for r in (fp64, fp32, fp32x2):
        assert math.isfinite(r) and r > 0
    # FP32 FMA: at least half the nominal lane rate, never above the
    # maximum-clock bound (148 x 128 x 2 x 2.032 GHz = 77.0 TFLOP/s)
    assert 35.0 < fp32 < 77.1, fp32
    assert 0.9 * fp32 < fp32x2 < 77.1 * 1.02, (fp32, fp32x2)
    # FP64 is far below FP32 on this part (the reason for the double-float
    # residual): below a tenth of it, and above zero by a margin
    assert 0.1 < fp64 < 0.1 * fp32, (fp64, fp32)


def test_probe_rejects_unknown_kind():
    g = gsm()
    for kind in (-1, 3):
        with pytest.raises(g.GsmError) as ei:
            g.probe_fma(kind)
        assert ei.value.status == g.GSM_ERR_ARG
