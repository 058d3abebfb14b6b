"""The tensor-core kernels' bounded waits, made to run out on purpose.

tpcf_set_wait_limit(polls, unmet_wait=1) makes every tensor-core kernel, once
its own MMAs have completed, wait once more on an mbarrier phase that nothing
completes (a flag that nothing sets), for 1000 polls: the kernels must then
latch the device error (TPCF_ERR_TIMEOUT at the next tpcf_stream_status),
release their tensor memory and return, leaving the context usable.  No fault
is involved: the wait ends by its poll count.  With the default restored the
same calls succeed and give the same results as before.
"""
import numpy as np
import pytest

from paper_2408_03036_gb300 import synth
from paper_2408_03036_gb300 import tpcf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03036_gb300 import build as B
    B.build()
    tpcf.lib()
    yield torch
    tpcf.lib().tpcf_set_wait_limit(0, 0)


def test_emulator_products_time_out_and_recover(gpu):
    torch = gpu
    widths = [6, 128, 128, 300]
    emu = tpcf.Emulator(widths, seed=3)
    x = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, (3000, 6)).astype(np.float32)).cuda()
    ref = emu.predict(x).clone()
    tpcf.stream_status()
    assert tpcf.lib().tpcf_set_wait_limit(1000, 1) == 0
    emu.predict(x)
    with pytest.raises(tpcf.TpcfError) as ei:
        tpcf.stream_status()
    assert ei.value.code == -4
    assert tpcf.lib().tpcf_set_wait_limit(0, 0) == 0
    again = emu.predict(x)
    tpcf.stream_status()
    assert torch.equal(again, ref)
    emu.close()


def test_split_precision_coupling_times_out_and_recovers(gpu):
    cfg = tpcf.Config(r_min=10.0, r_max=60.0, n_bins=6, l_max=4, Ls=(0, 2, 4), box=300.0, precision="bf16x3")
    xyz, w = synth.poisson(6000, 4)
    ref = tpcf.estimate_3pcf(cfg, xyz, w)
    tpcf.stream_status()
    assert tpcf.lib().tpcf_set_wait_limit(1000, 1) == 0
    tpcf.estimate_3pcf(cfg, xyz, w)
    with pytest.raises(tpcf.TpcfError) as ei:
        tpcf.stream_status()
    assert ei.value.code == -4
    assert tpcf.lib().tpcf_set_wait_limit(0, 0) == 0
    again = tpcf.estimate_3pcf(cfg, xyz, w)
    tpcf.stream_status()
    zr, za = ref.zeta.cpu().numpy(), again.zeta.cpu().numpy()
    # same inputs and kernels: only the order of floating-point atomics differs
    assert np.abs(za - zr).max() <= 1e-6 * np.abs(zr).max()
