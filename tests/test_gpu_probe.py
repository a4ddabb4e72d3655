"""The roof probes: measured L2 load bandwidth and scattered float4 atomic
throughput, the denominators of the load and atomic rooflines."""
import pytest

from paper_2503_12174_gb300 import dpcs
from gpu_util import ctx, need_cuda

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    need_cuda()
    c = ctx()
    gbs = c.probe_l2_load(32 << 20, 16)
    # 512 MiB of loads; any rate below 1 TB/s or above 1 PB/s means the loads were not done
    assert 1e3 < gbs < 1e6
    ga = c.probe_atomic4(512 * 512, 1 << 24)
    assert 0.1 < ga < 1e4
    assert c.launch_count >= 8


def test_probe_bad_arguments_refused():
    need_cuda()
    c = ctx()
    for nbytes, passes in ((15, 1), (0, 1), ((64 << 20) + 16, 1), (1 << 20, 0)):
        with pytest.raises(dpcs.DPCSError) as e:
            c.probe_l2_load(nbytes, passes)
        assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
    for texels, n in ((0, 1), ((1 << 24) + 1, 1), (16, 0)):
        with pytest.raises(dpcs.DPCSError) as e:
            c.probe_atomic4(texels, n)
        assert e.value.status == dpcs.DPCS_ERR_INVALID_ARG
    assert c.probe_l2_load(1 << 20, 1) > 0  # the context still works
