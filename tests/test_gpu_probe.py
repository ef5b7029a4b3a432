"""The reduction-throughput probe (rw_probe_red) the bench reads the map
scatter's roofline against: every add lands, bad arguments are refused."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_probe_red_adds_every_value_and_checks_arguments():
    from paper_2605_15418_gb300 import raywave as RW
    ctx = RW.Context()
    m = torch.zeros(256, 320, dtype=torch.float32, device="cuda")
    win, nwin = 32, 1000
    ctx.probe_red(m, win, nwin)
    torch.cuda.synchronize()
    total = float(m.double().sum())
    assert abs(total - 1e-3 * win * win * nwin) <= 1e-4 * 1e-3 * win * win * nwin
    # windows stay inside the map, and a window's pixels each get one add
    assert int((m > 0).sum()) <= 256 * 320
    for bad in ((0, 1), (257, 1), (8, -1)):
        with pytest.raises(RW.RayWaveError):
            ctx.probe_red(m, *bad)
