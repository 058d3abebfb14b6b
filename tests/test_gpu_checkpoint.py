"""Checkpoint / resume on the GPU: a batch of mocks interrupted after its first
group resumes from the stored results and gives what one uninterrupted batched
call gives; an emulator restored from a checkpoint (weights, Adam state, input box
and output scaling) continues training as the original does."""
import numpy as np
import pytest

from paper_2408_03036_gb300 import checkpoint as ck
from paper_2408_03036_gb300 import synth, tpcf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03036_gb300 import build as B
    B.build()
    tpcf.lib()
    return torch


class Interrupt(Exception):
    pass


def test_interrupted_batch_resumes(gpu, tmp_path):
    sizes = [3000, 1200, 2500, 800, 2100, 1600]
    xs, ws = [], []
    for k, n in enumerate(sizes):
        x, w = synth.poisson(n, 40 + k)
        xs.append(x)
        ws.append(w)
    xyz, w = np.concatenate(xs), np.concatenate(ws)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    cfg = tpcf.Config(r_min=20.0, r_max=120.0, n_bins=8, l_max=4, Ls=(0, 2, 4), periodic=True, box=500.0)
    ref, _ = tpcf.estimate_3pcf_batched(cfg, xyz, w, off)
    ref = ref.cpu().numpy()

    calls = []

    def stop_after_first(ids):
        calls.append(list(ids))
        raise Interrupt()

    with pytest.raises(Interrupt):
        ck.estimate_mocks_resumable(cfg, xyz, w, off, tmp_path, seed=40, group=2, on_group=stop_after_first)
    assert ck.MockResults(tmp_path, cfg, 40, len(sizes)).done() == {0, 1}
    first = [ck.MockResults(tmp_path, cfg, 40, len(sizes)).load(k)[0] for k in (0, 1)]

    calls.clear()
    z, status = ck.estimate_mocks_resumable(cfg, xyz, w, off, tmp_path, seed=40, group=2,
                                            on_group=lambda ids: calls.append(list(ids)))
    assert calls == [[2, 3], [4, 5]]                       # only the mocks still to do
    assert list(status) == [0] * len(sizes)
    for k in (0, 1):
        assert np.array_equal(z[k], first[k])              # stored results are kept as they were
    # the pair stage's queue order is set by atomics, so two runs agree to FP32
    # rounding: the FP32 bar per multipole
    for k in range(len(sizes)):
        for q in range(ref.shape[1]):
            den = np.abs(ref[k, q]).max()
            assert np.abs(z[k, q] - ref[k, q]).max() <= 1e-5 * den, (k, q)
    with pytest.raises(ValueError):                       # another seed is not mixed in
        ck.estimate_mocks_resumable(cfg, xyz, w, off, tmp_path, seed=41)


def test_emulator_checkpoint_resumes_training(gpu, tmp_path):
    torch = gpu
    widths = [6, 64, 64, 40]
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.uniform(-1, 1, (4, 512, 6)).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.normal(size=(4, 512, 40)).astype(np.float32)).cuda()
    a = tpcf.Emulator(widths, seed=5)
    a.set_input_box(np.full(6, -1.5, np.float32), np.full(6, 1.5, np.float32))
    a.fit_output_scaling(y[0])
    for k in range(2):
        a.train_step(x[k], y[k], 1e-3)
    path = tmp_path / "emu.npz"
    a.save(path)
    b = tpcf.Emulator.load(path)
    assert torch.equal(a.get_params(), b.get_params())
    ma, va, sa = a.optimizer_state()
    mb, vb, sb = b.optimizer_state()
    assert sa == sb == 2 and torch.equal(ma, mb) and torch.equal(va, vb)
    for e in (a, b):
        for k in range(2, 4):
            e.train_step(x[k], y[k], 1e-3)
    pa, pb = a.get_params(), b.get_params()
    # the bias gradients are summed with atomics: equal up to FP32 summation order
    assert torch.allclose(pa, pb, rtol=1e-5, atol=1e-6)
    assert torch.allclose(a.predict(x[0]), b.predict(x[0]), rtol=1e-4, atol=1e-4)
    tpcf.stream_status()
    a.close()
    b.close()
