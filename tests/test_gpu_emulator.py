"""The MLP emulator through the C ABI: gradients and predictions against the FP64
network reference, and a trained emulator against the plain tree-level model
(the reference it stands in for), with what it gains in evaluation speed."""
import multiprocessing as mp
import time

import numpy as np
import pytest

from paper_2408_03036_gb300 import tpcf

pytestmark = pytest.mark.gpu

BOX_LO = np.array([0.5, 1.0, -1.0, 0.6, 0.95, -0.05], dtype=np.float32)
BOX_HI = np.array([1.0, 3.0, 2.0, 1.0, 1.05, 0.05], dtype=np.float32)


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03036_gb300 import build as B
    B.build()
    tpcf.lib()
    return torch


_MODEL = None


def _set_model(m):
    global _MODEL
    _MODEL = m


def _evaluate(th):
    return _MODEL(th)


@pytest.fixture(scope="module")
def plain_model():
    """The plain model's templates on the (alpha, eps) grid, built in a process
    pool started with spawn (no CUDA state is inherited)."""
    from oracle import treelevel as T
    setup = T.ModelSetup()
    al = np.linspace(0.935, 1.065, 7)
    ep = np.linspace(-0.065, 0.065, 7)
    with mp.get_context("spawn").Pool(min(16, mp.cpu_count())) as pool:
        return T.TemplateModel.build(setup, al, ep, pool=pool)


def evaluate_parallel(model, th):
    """The plain model at every row of th, in a spawn process pool (host cores)."""
    n = min(16, mp.cpu_count())
    chunks = np.array_split(th, n)
    with mp.get_context("spawn").Pool(n, initializer=_set_model, initargs=(model,)) as pool:
        return np.concatenate(pool.map(_evaluate, chunks))


def rand_net(torch, widths, seed):
    rng = np.random.default_rng(seed)
    emu = tpcf.Emulator(widths, seed=seed)
    p = rng.normal(0, 0.3, emu.n_params).astype(np.float32)
    emu.set_params(torch.from_numpy(p).cuda())
    return emu, p


@pytest.mark.parametrize("widths,batch", [([6, 32, 32, 20], 37), ([6, 64, 64, 64, 64, 150], 5000)])
def test_gradients_match_fp64_reference(gpu, widths, batch):
    """Loss and every parameter gradient (several internal chunks for batch 5000)."""
    from oracle import mlp_oracle as MO
    torch = gpu
    emu, p = rand_net(torch, widths, 7)
    emu.set_input_box(BOX_LO, BOX_HI)
    rng = np.random.default_rng(8)
    x = (BOX_LO + rng.random((batch, 6)) * (BOX_HI - BOX_LO)).astype(np.float32)
    y = rng.normal(1.0, 2.0, (batch, widths[-1])).astype(np.float32)
    yd = torch.from_numpy(y).cuda()
    emu.fit_output_scaling(yd)
    mu, sd = emu.output_scaling()
    g, loss = emu.gradients(torch.from_numpy(x).cuda(), yd)
    lref, gref = MO.loss_and_grad(p, widths, x, y, BOX_LO.astype(np.float64), BOX_HI.astype(np.float64),
                                  mu.astype(np.float64), sd.astype(np.float64))
    tpcf.stream_status()
    assert abs(loss.item() - lref) <= 1e-5 * lref
    gg = g.cpu().numpy().astype(np.float64)
    off = 0
    for l in range(len(widths) - 1):
        for n in (widths[l] * widths[l + 1], widths[l + 1]):
            blk, ref = gg[off:off + n], gref[off:off + n]
            assert np.abs(blk - ref).max() <= 2e-4 * np.abs(ref).max(), (l, n)
            off += n
    emu.close()


def test_predictions_match_fp64_reference(gpu):
    from oracle import mlp_oracle as MO
    torch = gpu
    widths = [6, 48, 48, 30]
    emu, p = rand_net(torch, widths, 3)
    emu.set_input_box(BOX_LO, BOX_HI)
    rng = np.random.default_rng(9)
    x = (BOX_LO + rng.random((9000, 6)) * (BOX_HI - BOX_LO)).astype(np.float32)
    y = rng.normal(0.5, 3.0, (100, 30)).astype(np.float32)
    emu.fit_output_scaling(torch.from_numpy(y).cuda())
    mu, sd = emu.output_scaling()
    out = emu.predict(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = MO.predict(p, widths, x, BOX_LO.astype(np.float64), BOX_HI.astype(np.float64), mu.astype(np.float64),
                     sd.astype(np.float64))
    tpcf.stream_status()
    # the products take bf16 operands on both sides; an FP32 activation within an
    # ulp of a bf16 rounding boundary can round the other way on the device (its
    # SiLU is FP32) than in the FP64 reference: one bf16 ulp (2^-8) on that
    # element, which moves the outputs by a few 1e-4 of their largest value
    assert np.abs(out - ref).max() <= 5e-4 * np.abs(ref).max()
    emu.close()


def per_multipole_error(pred, ref, n_mult):
    """max over bins |pred - ref| / max over bins |ref|, per sample and multipole."""
    p = pred.reshape(pred.shape[0], n_mult, -1)
    r = ref.reshape(ref.shape[0], n_mult, -1)
    return np.abs(p - r).max(-1) / np.abs(r).max(-1)


def test_trained_emulator_reproduces_the_plain_model(gpu, plain_model):
    """Trained on Latin-hypercube samples of the plain model with the project's
    own tensor-core kernels; on held-out parameters the per-sample, per-multipole
    error max|zeta_emu - zeta_model| / max|zeta_model| has its median and its
    95th percentile within 1 %, and the network evaluates far faster than the
    plain model."""
    from oracle import treelevel as T
    torch = gpu
    n_train, n_test = 200000, 2000    # the emulator configuration's 200k Latin-hypercube samples
    th = T.latin_hypercube(n_train + n_test, 7).astype(np.float32)
    z = evaluate_parallel(plain_model, th).astype(np.float32)
    xtr, ytr = torch.from_numpy(th[:n_train]).cuda(), torch.from_numpy(z[:n_train]).cuda()
    widths = [6, 256, 256, 256, 256, z.shape[1]]
    emu = tpcf.Emulator(widths, seed=11)
    emu.set_input_box(BOX_LO, BOX_HI)
    emu.fit_output_scaling(ytr)
    g = torch.Generator(device="cuda").manual_seed(5)
    steps, bs = 20000, 512
    for s in range(steps):
        idx = torch.randint(0, n_train, (bs,), device="cuda", generator=g)
        lr = 2e-3 * 0.5 * (1 + np.cos(np.pi * s / steps)) + 1e-5
        emu.train_step(xtr[idx].contiguous(), ytr[idx].contiguous(), lr)
    pred = emu.predict(torch.from_numpy(th[n_train:]).cuda()).cpu().numpy()
    tpcf.stream_status()
    err = per_multipole_error(pred, z[n_train:], len(T.MULTIPOLES))
    print("emulator error: median %.3g %%, 95th percentile %.3g %%, max %.3g %%"
          % (100 * np.median(err), 100 * np.percentile(err, 95), 100 * err.max()))
    assert np.median(err) <= 0.01, np.median(err)
    assert np.percentile(err, 95) <= 0.01, np.percentile(err, 95)
    # what the network gains: evaluations per second against the plain model
    setup = plain_model.setup
    t0 = time.perf_counter()
    T.model_direct(setup, tuple(float(v) for v in th[n_train]))
    t_plain = time.perf_counter() - t0
    xs = torch.from_numpy(th[n_train:]).cuda()
    emu.predict(xs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(10):
        emu.predict(xs)
    torch.cuda.synchronize()
    t_emu = (time.perf_counter() - t0) / (10 * n_test)
    assert t_plain / t_emu > 1e4
    emu.close()
