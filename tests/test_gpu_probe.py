"""The roof probes of the measurement library (libdpcs_probe.so): measured L2
load bandwidth and scattered float4 atomic throughput, the denominators of
the load and atomic rooflines."""
import pytest

from paper_2503_12174_gb300 import probe
from gpu_util import need_cuda

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    need_cuda()
    gbs = probe.dpcs_probe_l2_load(0, 32 << 20, 16)
    # 512 MiB of loads; any rate below 1 TB/s or above 1 PB/s means the loads were not done
    assert 1e3 < gbs < 1e6
    ga = probe.dpcs_probe_atomic4(0, 512 * 512, 1 << 24)
    assert 0.1 < ga < 1e4


def test_probe_bad_arguments_refused():
    need_cuda()
    for nbytes, passes in ((15, 1), (0, 1), ((64 << 20) + 16, 1), (1 << 20, 0)):
        with pytest.raises(probe.ProbeError) as e:
            probe.dpcs_probe_l2_load(0, nbytes, passes)
        assert e.value.status == -1
    for texels, n in ((0, 1), ((1 << 24) + 1, 1), (16, 0)):
        with pytest.raises(probe.ProbeError) as e:
            probe.dpcs_probe_atomic4(0, texels, n)
        assert e.value.status == -1
    assert probe.dpcs_probe_l2_load(0, 1 << 20, 1) > 0  # still works after refusals
