#!/usr/bin/env python3
"""Throughput of the GB300 anisotropic 3PCF estimator (primaries per second).

Workload (the clustered-halo configuration): a seeded lognormal catalogue of
N_D = 400,000 points (Gaussian field on a 512^3 mesh, P_G(k) ~ k^-1.5
exp(-(k/0.5)^2), sigma_G = 1, Kaiser-like LOS shift f = 0.8) in an open cube of
side 1000 Mpc/h, with N_R = 1,200,000 uniform randoms for the data-minus-random
edge correction; 20 linear bins 10-150 Mpc/h, l_max = 4, L in {0, 2, 4}.
A step is one full tpcf_estimate_3pcf: grids, the pair stage on the D-R field,
the random-only RRR pass, the coupling and the TripoSH projection.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3PCF primaries/s & mocks/hour at l_max=4 (mixed vs plain FP32 GPU, err≤1e-4)"
UNIT = "primaries/s"
ND, NR, BOX, MESH = 400_000, 1_200_000, 1000.0, 512
SEED_D, SEED_R = 2, 3
WORKLOAD = ("clustered lognormal halos N_D=400000 (512^3 mesh, P~k^-1.5 exp(-(k/0.5)^2), sigma_G=1, "
            "LOS shift f=0.8) + N_R=1200000 randoms, open cube L=1000 Mpc/h, 20 bins 10-150 Mpc/h, "
            "l_max=4, L={0,2,4}")
FLOP_PER_PAIR = 4 * 25 + 15   # algorithmic FP32 work per accepted pair at l_max = 4
# DRAM bytes (read + write) per primary of the harmonic pair kernel, from one ncu
# capture of the current kernel at this workload's density (400,000 primaries in
# a 630 Mpc/h cube: 19.7 MB read + 778.2 MB written, the a_lm output); the
# traffic grows with the primaries, so a launch moves this times its primaries
PAIR_DRAM_BYTES_PER_PRIMARY = 1995.0
# covariance batch: lognormal mocks (same field recipe, 256^3 mesh) in a periodic
# cube of side 1000 Mpc/h, sizes uniform in [100k, 400k], analytic randoms
N_MOCKS, MOCK_LO, MOCK_HI, MOCK_MESH, SEED_MOCKS = 256, 100_000, 400_000, 256, 77
# many small mocks of the same recipe (10k-20k points, 128^3 mesh), where a call
# per mock pays its fixed cost (host set-up, synchronisations, launches) against
# about 0.1 ms of pair work
N_SMALL, SMALL_LO, SMALL_HI, SMALL_MESH = 1024, 10_000, 20_000, 128


def config(precision="fp32"):
    from paper_2408_03036_gb300 import tpcf
    return tpcf.Config(r_min=10.0, r_max=150.0, n_bins=20, l_max=4, Ls=(0, 2, 4), periodic=False,
                       box=BOX, precision=precision)


def mock_config(precision="fp32", **kw):
    from paper_2408_03036_gb300 import tpcf
    return tpcf.Config(r_min=10.0, r_max=150.0, n_bins=20, l_max=4, Ls=(0, 2, 4), periodic=True,
                       box=BOX, precision=precision, **kw)


def make_inputs(rank=0):
    from paper_2408_03036_gb300 import synth
    d, dw = synth.lognormal(ND, BOX, SEED_D + 1000 * rank, mesh=MESH)
    r, rw = synth.randoms(NR, SEED_R + 1000 * rank)
    return d, dw, r, rw


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(target_s=12.0, max_prim=20000):
    """The FP64 oracle as it stands, on a bounded random sample of primaries of
    the same workload (numerator pass over the D-R field plus the proportional
    random-only RRR pass), on all host cores."""
    import numpy as np
    from oracle import oracle as ora
    d, dw, r, rw = make_inputs()
    o = ora.Config(10.0, 150.0, 20, 4, (0, 2, 4), False, BOX)
    alpha = float(dw.astype(np.float64).sum() / rw.astype(np.float64).sum())
    fx = np.concatenate([d, r])
    fw = np.concatenate([dw.astype(np.float64), -alpha * rw.astype(np.float64)])
    rng = np.random.default_rng(11)
    ntot = ND + NR

    def timed(nprim):
        pf = np.sort(rng.choice(ntot, size=nprim, replace=False))
        pr = np.sort(rng.choice(NR, size=max(1, int(round(nprim * NR / ntot))), replace=False))
        t = time.perf_counter()
        ora.run(o, fx, fw, prim=pf)
        ora.run(o, r, alpha * rw.astype(np.float64), prim=pr, l_max=0)
        return time.perf_counter() - t

    n = 64
    t = timed(n)
    n2 = int(min(max_prim, max(n, n * target_s / max(t, 1e-3))))
    t2 = timed(n2)
    return {"value": n2 / t2, "unit": UNIT, "cores": ora.max_threads(), "kind": "oracle",
            "sample": "%d random primaries of the D-R field (+%d of the random-only RRR pass) against all "
                      "%d points, %.1f s" % (n2, int(round(n2 * NR / ntot)), ntot, t2)}


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import numpy as np
    from oracle import oracle as ora
    d, dw, r, rw = make_inputs()
    o = ora.Config(10.0, 150.0, 20, 4, (0, 2, 4), False, BOX)
    alpha = float(dw.astype(np.float64).sum() / rw.astype(np.float64).sum())
    fx = np.concatenate([d, r])
    fw = np.concatenate([dw.astype(np.float64), -alpha * rw.astype(np.float64)])
    ntot = ND + NR
    rng = np.random.default_rng(12)
    per_step_s = max(2.0, min(15.0, 150.0 / max(1, args.steps + args.warmup)))

    def step(nprim):
        pf = np.sort(rng.choice(ntot, size=nprim, replace=False))
        pr = np.sort(rng.choice(NR, size=max(1, int(round(nprim * NR / ntot))), replace=False))
        t = time.perf_counter()
        ora.run(o, fx, fw, prim=pf)
        ora.run(o, r, alpha * rw.astype(np.float64), prim=pr, l_max=0)
        return time.perf_counter() - t

    t = step(32)
    nprim = int(max(32, min(50000, 32 * per_step_s / max(t, 1e-3))))
    for _ in range(args.warmup):
        step(max(8, nprim // 16))
    times = [step(nprim) for _ in range(args.steps)]
    total = sum(times)
    value = nprim * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_primaries_per_step": nprim},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ora.max_threads(), "kind": "oracle",
                             "sample": "%d random primaries per step (+%d random-only RRR primaries) of the "
                                       "%d-point D-R field" % (nprim, int(round(nprim * NR / ntot)), ntot)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    from paper_2408_03036_gb300 import build as B
    from paper_2408_03036_gb300 import tpcf

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    from paper_2408_03036_gb300 import shard
    dev = torch.device("cuda", local)
    cfg = config(args.precision)
    # one catalogue; with several ranks each takes the primaries of its z slab
    # (secondaries within r_max of it) and the partials are summed over the group
    d, dw, r, rw = make_inputs()
    dx = torch.from_numpy(d.view(np.int32)).to(dev)
    dwt = torch.from_numpy(dw).to(dev)
    rx = torch.from_numpy(r.view(np.int32)).to(dev)
    rwt = torch.from_numpy(rw).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2
    share = shard.ShardInputs(cfg, d, dw, r, rw, rank, ws, dev) if ws > 1 else None

    def step():
        if share is not None:
            return shard.estimate_prepared(cfg, share, stream=stream)
        return tpcf.estimate_3pcf(cfg, dx, dwt, rx, rwt, stream=stream, device=dev)

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize(dev)
    tpcf.stream_status(stream)
    pairs_per_step = int(res.pair_counts.sum().item())

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = tpcf.kernel_launches()
    with ClockSampler(dev.index) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
    launches = tpcf.kernel_launches() - launches0
    tpcf.stream_status(stream)
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    prim_per_step = ND + NR   # the whole catalogue, shared out over the ranks
    value = prim_per_step * args.steps / (ms_max / 1000.0)

    # the plain FP32 form of the same step (FP32 Gram coupling), timed the same way
    plain = None
    if args.precision != "fp32":
        pcfg = config("fp32")
        def pstep():
            if share is not None:
                return shard.estimate_prepared(pcfg, share, stream=stream)
            return tpcf.estimate_3pcf(pcfg, dx, dwt, rx, rwt, stream=stream, device=dev)

        for _ in range(max(1, args.warmup // 2)):
            pres = pstep()
        torch.cuda.synchronize(dev)
        # the mixed step's multipoles against the plain step's, per multipole
        zm, zp = res.zeta.cpu().numpy(), pres.zeta.cpu().numpy()
        den = np.abs(zp).max(axis=(1, 2))
        mixed_err = float((np.abs(zm - zp).max(axis=(1, 2)) / np.where(den > 0, den, 1.0)).max())
        pms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            pstep()
            e0.record(stream)
            torch.cuda.synchronize(dev)
            pms += s0.elapsed_time(e0)
        tpcf.stream_status(stream)
        if dist:
            tp = torch.tensor([pms], dtype=torch.float64, device=dev)
            dist.all_reduce(tp, op=dist.ReduceOp.MAX)
            pms = float(tp.item())
        pvalue = prim_per_step * args.steps / (pms / 1000.0)
        plain = {"value": pvalue, "unit": UNIT, "ms_per_step": pms / args.steps, "mixed_over_plain": value / pvalue,
                 "mixed_vs_plain_max_rel_err": mixed_err}

    # dominant kernel: the pair stage on the D-R field, timed alone with events
    roof = roofline(cfg, d, dw, r, rw, dev, stream, tpcf)

    # the other estimator forms on the same workload (one call each per step)
    variants = None if args.no_variants else variants_report(cfg, dx, dwt, rx, rwt, dev, stream, tpcf, flush,
                                                             ms_max / args.steps)

    stages = None if (args.no_variants or rank != 0) else stages_report(cfg, dx, dwt, rx, rwt, dev, stream, tpcf)

    # end to end through the host-buffer entry point (copies inside the timed region)
    e2e = end_to_end(cfg, d, dw, r, rw, args, stream, tpcf, ws, rank)

    del dx, dwt, rx, rwt
    torch.cuda.empty_cache()   # the batch sizes its groups from the free device memory
    mocks = batch_mocks(args, dev, stream, tpcf, flush, rank) if args.mocks > 0 else None

    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f32/" + args.precision, "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": args.precision,
                       "parallelism": "z-slab shards, FP64 partials summed (NCCL)" if ws > 1 else "one GPU",
                       "primaries_per_step": prim_per_step, "pairs_per_step": pairs_per_step,
                       "l2": "flushed between timed steps (256 MB write, outside the events)"},
            "clocks": clk.summary(), "gpu_launches": int(launches), "roofline": roof, "e2e": e2e,
            "pairs_per_s": pairs_per_step * args.steps / (ms_max / 1000.0)}
    if plain is not None:
        line["plain_fp32"] = plain
    if variants is not None:
        line["variants"] = variants
    if stages is not None:
        line["stages"] = stages
    if mocks is not None:
        line["mocks_per_hour"] = mocks
    if not args.no_precision:
        line["precision_vs_oracle"] = precision_report(dev, stream, tpcf)
    if not args.no_emulator:
        line["emulator"] = emulator_report(dev, stream, tpcf, with_cpu=not args.no_cpu_baseline)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def _event_ms(fn, stream, dev, reps=3, warm=1):
    """Median CUDA-event time of fn() on the stream (after `warm` untimed calls)."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize(dev)
    ms = []
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        fn()
        e.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(s.elapsed_time(e))
    return statistics.median(ms)


def stages_report(cfg, dx, dwt, rx, rwt, dev, stream, tpcf):
    """The steps of the path reported on their own:
      * grid build of the headline D - R field (1.6 M records): bandwidth with 32
        algorithmic bytes per point (coordinates and weight read, record written);
      * the random-only count pass (tpcf_pair_counts on the 1.2 M randoms), the
        RRR normaliser's pass when the data weights can be negative;
      * the small configuration: Poisson N = 20,000 in a periodic cube L = 500,
        10 bins 20-120, l_max 4, the whole estimate per call."""
    import numpy as np
    import torch
    from paper_2408_03036_gb300 import synth
    out = {}
    alpha = float(dwt.double().sum().item() / rwt.double().sum().item())
    fx = torch.cat([dx, rx])
    fw = torch.cat([dwt, (-alpha * rwt.double()).float()])
    n = fx.shape[0]
    grids = []

    def build():
        grids.append(tpcf.Grid(cfg, fx, fw, stream=stream, device=dev))

    ms = _event_ms(build, stream, dev)
    for g in grids:
        g.close()
    out["grid_build"] = {"points": n, "ms": ms, "points_per_s": n / (ms / 1000.0),
                         "hbm_gbs": 32.0 * n / (ms / 1000.0) / 1e9, "bytes_per_point": 32}
    rg = tpcf.Grid(cfg, rx, rwt, stream=stream, device=dev)
    res = []
    ms = _event_ms(lambda: res.append(tpcf.pair_counts(rg, cfg, stream=stream)), stream, dev)
    pairs = int(res[-1][1].sum().item())
    rg.close()
    nr = rx.shape[0]
    out["random_count_pass"] = {"primaries": nr, "pairs": pairs, "ms": ms, "primaries_per_s": nr / (ms / 1000.0),
                                "pairs_per_s": pairs / (ms / 1000.0)}
    x, w = synth.poisson(20_000, 1)
    xd = torch.from_numpy(x.view(np.int32)).to(dev)
    wd = torch.from_numpy(w).to(dev)
    small = {"workload": "Poisson N=20000, periodic L=500, 10 bins 20-120, l_max=4, L={0,2,4}"}
    for prec in ("fp32", "bf16x3"):
        c = tpcf.Config(r_min=20.0, r_max=120.0, n_bins=10, l_max=4, Ls=(0, 2, 4), periodic=True, box=500.0,
                        precision=prec)
        ms = _event_ms(lambda: tpcf.estimate_3pcf(c, xd, wd, stream=stream, device=dev), stream, dev, reps=5)
        small[prec] = {"ms": ms, "primaries_per_s": 20_000 / (ms / 1000.0)}
    tpcf.stream_status(stream)
    # the oracle on the same small case, on the host cores
    from oracle import oracle as ora
    o = ora.Config(20.0, 120.0, 10, 4, (0, 2, 4), True, 500.0)
    t0 = time.perf_counter()
    ora.estimate(o, x, w)
    small["oracle"] = {"s": time.perf_counter() - t0, "cores": ora.max_threads(), "cpu": cpu_model()}
    out["small_case"] = small
    return out


def cpu_model():
    """The host CPU's model string (or the architecture if the system gives none)."""
    import platform
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def variants_report(cfg, dx, dwt, rx, rwt, dev, stream, tpcf, flush, plain_ms, reps=2):
    """Primaries per second of the estimator's other forms on the headline
    workload: with the even 2PCF multipoles, with the full anisotropic edge
    correction (every RRR^m_{l1 l2} and the per-bin-pair solve), and with a
    varying line of sight from an observer outside the cube."""
    import dataclasses
    import torch
    n = dx.shape[0] + rx.shape[0]
    vlos = dataclasses.replace(cfg, los="observer", observer=(-0.5 * BOX, -0.5 * BOX, -0.5 * BOX))
    calls = {
        "with_2pcf": lambda: tpcf.estimate_3pcf(cfg, dx, dwt, rx, rwt, stream=stream, device=dev, want_xi=True),
        "full_edge_correction": lambda: tpcf.estimate_3pcf_full_edge(cfg, dx, dwt, rx, rwt, stream=stream,
                                                                     device=dev),
        "varying_los": lambda: tpcf.estimate_3pcf(vlos, dx, dwt, rx, rwt, stream=stream, device=dev),
    }
    out = {"plain_ms": plain_ms}
    for name, call in calls.items():
        call()
        torch.cuda.synchronize(dev)
        tpcf.stream_status(stream)
        ms = 0.0
        for _ in range(reps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            call()
            e.record(stream)
            torch.cuda.synchronize(dev)
            ms += s.elapsed_time(e)
        tpcf.stream_status(stream)
        ms /= reps
        out[name] = {"ms_per_step": ms, "primaries_per_s": n / (ms / 1000.0), "over_plain": ms / plain_ms}
    return out


def batch_mocks(args, dev, stream, tpcf, flush, rank=0):
    """Mocks per hour for the covariance batch: one graph-captured batch run per
    step (all mocks' pair stages in one persistent launch per group), plain FP32
    coupling against the bf16x3 tensor-core coupling, plus one-catalogue calls
    on a sample of the same mocks as the unbatched comparison."""
    import numpy as np
    import torch
    from paper_2408_03036_gb300 import synth
    n_mocks = args.mocks
    sizes = synth.mock_sizes(n_mocks, MOCK_LO, MOCK_HI, SEED_MOCKS + 1000 * rank)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    xyz = torch.empty((int(off[-1]), 3), dtype=torch.int32, device=dev)
    for k, n in enumerate(sizes):
        x, _ = synth.lognormal_device(int(n), BOX, SEED_MOCKS + 1000 * rank + 1 + k, mesh=MOCK_MESH, device=dev)
        xyz[off[k]:off[k + 1]] = x
        del x
    w = torch.ones(int(off[-1]), dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)
    # tile shapes for this density from the autotuner (a batch's tiles hold
    # primaries of one mock only)
    tuned = tpcf.autotune(mock_config("fp32"), xyz[:int(off[1])], w[:int(off[1])], stream=stream, device=dev)
    out = {"mocks": n_mocks, "points": int(off[-1]), "sizes": [int(sizes.min()), int(sizes.max())],
           "tuned": {"cell_div": tuned.cell_div, "chunk": tuned.chunk, "tile_primaries": tuned.tile_primaries}}
    zs = {}
    for prec in ("fp32", "bf16x3"):
        cfg = mock_config(prec, cell_div=tuned.cell_div, chunk=tuned.chunk, tile_primaries=tuned.tile_primaries)
        b = tpcf.Batch(cfg, off)
        z = b.zeta_buffer(dev)
        b.run_graph(xyz, w, z, stream=stream)          # eager run + capture (warm-up)
        b.run_graph(xyz, w, z, stream=stream)          # first graph launch (warm-up)
        torch.cuda.synchronize(dev)
        tpcf.stream_status(stream)
        ms = 0.0
        for _ in range(args.batch_steps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            b.run_graph(xyz, w, z, stream=stream)
            e.record(stream)
            torch.cuda.synchronize(dev)
            ms += s.elapsed_time(e)
        tpcf.stream_status(stream)
        groups, nc = b.info()
        out[prec] = {"mocks_per_hour": n_mocks * args.batch_steps / (ms / 1000.0) * 3600.0,
                     "s_per_batch": ms / 1000.0 / args.batch_steps, "groups": groups, "cells_per_axis": nc}
        zs[prec] = z.cpu().numpy()
        if prec == "fp32":
            out["covariance"] = covariance_report(cfg, z, stream, tpcf, dev)
        b.close()
        del z
    # mixed against plain: worst over mocks and multipoles of max|diff| / max|plain|
    zf, zb = zs["fp32"], zs["bf16x3"]
    den = np.abs(zf).max(axis=(2, 3))
    num = np.abs(zb - zf).max(axis=(2, 3))
    out["bf16x3_vs_fp32_max_rel_err"] = float((num / np.where(den > 0, den, 1.0)).max())
    out["mixed_over_plain"] = out["bf16x3"]["mocks_per_hour"] / out["fp32"]["mocks_per_hour"]
    # unbatched: one tpcf_estimate_3pcf per mock over every mock of the batch (the
    # same tuned cells and queues), timed the same way
    out["sequential"] = {"note": "one tpcf_estimate_3pcf call per mock, all mocks, same tuned cells, queue and tiles"}
    for prec in ("fp32", "bf16x3"):
        cfg = mock_config(prec, cell_div=tuned.cell_div, chunk=tuned.chunk, tile_primaries=tuned.tile_primaries)
        for k in range(2):
            tpcf.estimate_3pcf(cfg, xyz[off[k]:off[k + 1]], w[off[k]:off[k + 1]], stream=stream, device=dev,
                               want_all=False)
        torch.cuda.synchronize(dev)
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for k in range(n_mocks):
            tpcf.estimate_3pcf(cfg, xyz[off[k]:off[k + 1]], w[off[k]:off[k + 1]], stream=stream, device=dev,
                               want_all=False)
        e.record(stream)
        torch.cuda.synchronize(dev)
        tpcf.stream_status(stream)
        t = s.elapsed_time(e) / 1000.0
        out["sequential"][prec] = {"mocks_per_hour": n_mocks / t * 3600.0, "s_per_batch": t}
        out["batched_over_sequential_" + prec] = out[prec]["mocks_per_hour"] / (n_mocks / t * 3600.0)
    del xyz, w
    out["small_mocks"] = small_mock_batch(dev, stream, tpcf, flush, rank)
    return out


def small_mock_batch(dev, stream, tpcf, flush, rank=0):
    """The batch against one tpcf_estimate_3pcf call per mock on many small mocks
    (N_SMALL lognormal mocks of SMALL_LO..SMALL_HI points in the same periodic box),
    where a call's fixed cost is comparable with its pair work: one graph launch of
    the whole batch against the loop of calls, each with its default tiles, both
    couplings."""
    import numpy as np
    import torch
    from paper_2408_03036_gb300 import synth
    seed0 = SEED_MOCKS + 500 + 1000 * rank
    sizes = synth.mock_sizes(N_SMALL, SMALL_LO, SMALL_HI, seed0)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    xyz = torch.empty((int(off[-1]), 3), dtype=torch.int32, device=dev)
    for k, n in enumerate(sizes):
        x, _ = synth.lognormal_device(int(n), BOX, seed0 + 1 + k, mesh=SMALL_MESH, device=dev)
        xyz[off[k]:off[k + 1]] = x
        del x
    w = torch.ones(int(off[-1]), dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)
    out = {"mocks": N_SMALL, "points": int(off[-1]), "sizes": [int(sizes.min()), int(sizes.max())],
           "note": "one graph launch of the batch vs one tpcf_estimate_3pcf call per mock; default tiles"}
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for prec in ("fp32", "bf16x3"):
        cfg = mock_config(prec)
        b = tpcf.Batch(cfg, off)
        z = b.zeta_buffer(dev)
        b.run_graph(xyz, w, z, stream=stream)          # eager run + capture (warm-up)
        b.run_graph(xyz, w, z, stream=stream)          # first graph launch (warm-up)
        torch.cuda.synchronize(dev)
        tpcf.stream_status(stream)
        flush.zero_()
        s.record(stream)
        b.run_graph(xyz, w, z, stream=stream)
        e.record(stream)
        torch.cuda.synchronize(dev)
        tpcf.stream_status(stream)
        tb = s.elapsed_time(e) / 1000.0
        b.close()
        del z
        cfg1 = mock_config(prec)
        for k in range(2):
            tpcf.estimate_3pcf(cfg1, xyz[off[k]:off[k + 1]], w[off[k]:off[k + 1]], stream=stream, device=dev,
                               want_all=False)
        torch.cuda.synchronize(dev)
        flush.zero_()
        s.record(stream)
        for k in range(N_SMALL):
            tpcf.estimate_3pcf(cfg1, xyz[off[k]:off[k + 1]], w[off[k]:off[k + 1]], stream=stream, device=dev,
                               want_all=False)
        e.record(stream)
        torch.cuda.synchronize(dev)
        tpcf.stream_status(stream)
        ts = s.elapsed_time(e) / 1000.0
        out[prec] = {"batched_mocks_per_hour": N_SMALL / tb * 3600.0, "sequential_mocks_per_hour": N_SMALL / ts * 3600.0,
                     "batched_over_sequential": ts / tb}
    return out


def covariance_report(cfg, z, stream, tpcf, dev, reps=3):
    """Eq. covariance over the batch's mocks, on its zeta array in place: the
    paper's six multipoles with eta = 3, and every entry of every multipole.
    FLOP: 2 per multiply-add over the computed upper-triangle tiles."""
    import torch
    sel = [(0, 0, 0), (1, 1, 0), (2, 2, 0), (2, 0, 2), (1, 1, 2), (3, 1, 2)]
    cases = {"six_multipoles_eta3": tpcf.data_vector_index(cfg, sel, 3), "all_entries": None}
    out = {"mocks": int(z.shape[0])}
    for name, idx in cases.items():
        di = None if idx is None else torch.as_tensor(idx).to(dev)
        nd = z[0].numel() if idx is None else int(idx.size)
        tpcf.covariance(z, idx=di, n_dv=nd, stream=stream)
        torch.cuda.synchronize(dev)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for _ in range(reps):
            tpcf.covariance(z, idx=di, n_dv=nd, stream=stream)
        e.record(stream)
        torch.cuda.synchronize(dev)
        tpcf.stream_status(stream)
        t = s.elapsed_time(e) / 1000.0 / reps
        nt = (nd + 63) // 64
        flop = 2.0 * (nt * (nt + 1) // 2) * 64 * 64 * int(z.shape[0])
        r = {"n_dv": nd, "ms": t * 1000.0, "fp64_gflops": flop / t / 1e9}
        if int(z.shape[0]) > nd + 4:
            h, m1 = tpcf.covariance_factors(int(z.shape[0]), nd, 7)
            r.update({"hartlap": h, "percival_m1_7_params": m1})
        out[name] = r
    return out


def gram_flop_per_primary(nb, lmax):
    """Algorithmic FLOP of the Gram coupling per primary: for every m, the
    symmetric block of n_m = n_b (l_max - m + 1) rows (real part only at m = 0,
    real and imaginary above), 2 FLOP per multiply-add over the upper triangle."""
    return sum((1 if m == 0 else 2) * (nb * (lmax - m + 1)) ** 2 for m in range(lmax + 1))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "of measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "of fallback"


def coupling_report(cfg, alm, wprim, counts, diag, wsp, dev, stream, tpcf, reps=3):
    """The coupling step alone on the workload's per-primary a_lm: plain FP32 Gram
    against the bf16x3 and tf32x3 tensor-core Grams (three MMAs per useful MAC)."""
    import dataclasses
    import torch
    peaks, which = measured_peaks()
    K = alm.shape[0]
    flop = gram_flop_per_primary(cfg.n_bins, cfg.l_max) * K
    out = {"primaries": K, "algorithmic_flop": flop}
    for prec in ("fp32", "bf16x3", "tf32x3"):
        c = dataclasses.replace(cfg, precision=prec)
        tpcf.couple_multipoles(c, alm, wprim, counts, diag, wsp, stream=stream)
        torch.cuda.synchronize(dev)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(reps):
            s.record(stream)
            tpcf.couple_multipoles(c, alm, wprim, counts, diag, wsp, stream=stream)
            e.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(s.elapsed_time(e))
        t = statistics.median(ms) / 1000.0
        # the Gram reads every primary's a_lm row (and weight) once: an HBM-bound step
        nbytes = alm.numel() * 4 + wprim.numel() * 4
        r = {"ms": t * 1000.0, "algorithmic_tflops": flop / t / 1e12, "hbm_gbs": nbytes / t / 1e9,
             "hbm_frac": nbytes / t / 1e9 / peaks["hbm_gbs"], "hbm_note": which + " copy bandwidth"}
        if prec != "fp32":
            # tensor-pipe work: three MMAs over the full square blocks (twice the
            # upper-triangle count); tf32 runs at half the bf16 rate
            peak = peaks["bf16_tflops"] * (1.0 if prec == "bf16x3" else 0.5)
            r["tensor_tflops"] = 6 * flop / t / 1e12
            r["tensor_peak_tflops"] = peak
            r["tensor_frac"] = r["tensor_tflops"] / peak
            r["peak_note"] = which + (" bf16" if prec == "bf16x3" else " bf16 x 0.5 (nominal tf32/bf16 ratio)")
        out[prec] = r
    return out


def precision_report(dev, stream, tpcf):
    """Per-multipole error against the FP64 oracle on the precision workload:
    Poisson N=20,000 in a periodic cube L=500, l_max 6, 30 bins 5-155, L in
    {0,2,4,6}, for the plain FP32 coupling and the two tensor-core splits."""
    import numpy as np
    import torch
    from oracle import oracle as ora
    from paper_2408_03036_gb300 import synth
    x, w = synth.poisson(20_000, 5)
    o = ora.Config(5.0, 155.0, 30, 6, (0, 2, 4, 6), True, 500.0)
    t = time.perf_counter()
    est = ora.estimate(o, x, w)
    out = {"workload": "Poisson N=20000, periodic L=500, 30 bins 5-155, l_max=6, L={0,2,4,6}",
           "oracle_s": time.perf_counter() - t, "n_mult": len(est.mults)}
    for prec in ("fp32", "bf16x3", "tf32x3"):
        cfg = tpcf.Config(r_min=5.0, r_max=155.0, n_bins=30, l_max=6, Ls=(0, 2, 4, 6), periodic=True, box=500.0,
                          precision=prec)
        res = tpcf.estimate_3pcf(cfg, x, w, stream=stream, device=dev)
        tpcf.stream_status(stream)
        xd = torch.from_numpy(x.view(np.int32)).to(dev)
        wd = torch.from_numpy(w).to(dev)
        gms = _event_ms(lambda: tpcf.estimate_3pcf(cfg, xd, wd, stream=stream, device=dev), stream, dev)
        zg = res.zeta.cpu().numpy()
        err = []
        for k in range(len(est.mults)):
            den = np.abs(est.zeta[k]).max()
            err.append(float(np.abs(zg[k] - est.zeta[k]).max() / den) if den > 0 else 0.0)
        err = np.array(err)
        out[prec] = {"max_rel_err": float(err.max()), "median_rel_err": float(np.median(err)),
                     "worst": "%d%d%d" % tuple(est.mults[int(err.argmax())]),
                     "counts_exact": bool(np.array_equal(res.triplet_counts.cpu().numpy(), est.trip_counts)),
                     "gpu_ms": gms, "gpu_primaries_per_s": 20_000 / (gms / 1000.0)}
    return out


EMU_WIDTHS = [6, 256, 256, 256, 256, 3150]   # theta -> 15 multipoles x 210 (r1 <= r2) of 20 bins


_EMU_MODEL = None


def _emu_set_model(m):
    global _EMU_MODEL
    _EMU_MODEL = m


def _emu_evaluate(th):
    return _EMU_MODEL(th)


def emulator_report(dev, stream, tpcf, with_cpu=True, steps=2000):
    """The MLP emulator of the tree-level multipoles (the emulator configuration:
    200k Latin-hypercube samples of the plain model):
      * throughput of the project's tensor-core kernels, training at batches of 512,
        4096 and 32768 and inference over 200k parameter vectors, against the measured
        bf16 peak (random parameters and targets: timing only);
      * accuracy: trained on the 200k samples of the plain model (evaluated on the
        host cores in a spawn process pool) for 20,000 steps of 512, judged on 2000
        held-out samples by max|zeta_emu - zeta_model| / max|zeta_model| per sample
        and multipole;
      * the plain model's time per parameter vector on one host core (CPU baseline)."""
    import multiprocessing as mp
    import numpy as np
    import torch
    lo = np.array([0.5, 1.0, -1.0, 0.6, 0.95, -0.05], np.float32)
    hi = np.array([1.0, 3.0, 2.0, 1.0, 1.05, 0.05], np.float32)
    peaks, which = measured_peaks()
    per_sample_flop = 2 * sum(a * b for a, b in zip(EMU_WIDTHS[:-1], EMU_WIDTHS[1:]))
    n = 200_000
    g = torch.Generator(device=dev).manual_seed(3)
    x = torch.from_numpy(lo).to(dev) + torch.rand((n, 6), device=dev, generator=g) * torch.from_numpy(hi - lo).to(dev)
    y = torch.randn((n, EMU_WIDTHS[-1]), device=dev, generator=g)
    emu = tpcf.Emulator(EMU_WIDTHS, seed=1, device=dev)
    emu.set_input_box(lo, hi)
    emu.fit_output_scaling(y, stream=stream)
    rep = {"widths": EMU_WIDTHS, "peak_tflops": peaks["bf16_tflops"], "peak_note": which + " bf16 (burst)",
           "note": "bf16 operands, FP32 accumulation in tensor memory (tcgen05 GEMM kernels)"}
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for batch in (512, 4096, 32768):
        idx = [torch.randint(0, n, (batch,), device=dev, generator=g) for _ in range(8)]
        xb, yb = [x[i].contiguous() for i in idx], [y[i].contiguous() for i in idx]
        for k in range(10):
            emu.train_step(xb[k % 8], yb[k % 8], 1e-3, stream=stream)
        torch.cuda.synchronize(dev)
        st = steps if batch == 512 else max(50, steps * 512 // (8 * batch))
        s.record(stream)
        for k in range(st):
            emu.train_step(xb[k % 8], yb[k % 8], 1e-3, stream=stream)
        e.record(stream)
        torch.cuda.synchronize(dev)
        t = s.elapsed_time(e) / 1000.0
        tf = 3 * per_sample_flop * st * batch / t / 1e12
        rep["train_batch_%d" % batch] = {"samples_per_s": st * batch / t, "tflops": tf,
                                         "frac": tf / peaks["bf16_tflops"]}
    out = torch.empty((n, EMU_WIDTHS[-1]), device=dev)
    emu.predict(x, out=out, stream=stream)
    torch.cuda.synchronize(dev)
    s.record(stream)
    emu.predict(x, out=out, stream=stream)
    e.record(stream)
    torch.cuda.synchronize(dev)
    t_inf = s.elapsed_time(e) / 1000.0
    tpcf.stream_status(stream)
    emu.close()
    del x, y, out
    tf = per_sample_flop * n / t_inf / 1e12
    rep["infer"] = {"theta_per_s": n / t_inf, "tflops": tf, "frac": tf / peaks["bf16_tflops"]}
    # accuracy against the plain model on the emulator configuration
    from oracle import treelevel as T
    t0 = time.perf_counter()
    ncpu = min(16, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(ncpu) as pool:
        model = T.TemplateModel.build(T.ModelSetup(), np.linspace(0.935, 1.065, 7), np.linspace(-0.065, 0.065, 7),
                                      pool=pool)
    n_train, n_test = 200_000, 2000
    th = T.latin_hypercube(n_train + n_test, 7).astype(np.float32)
    with mp.get_context("spawn").Pool(ncpu, initializer=_emu_set_model, initargs=(model,)) as pool:
        z = np.concatenate(pool.map(_emu_evaluate, np.array_split(th, ncpu))).astype(np.float32)
    t_model = time.perf_counter() - t0
    xtr, ytr = torch.from_numpy(th[:n_train]).to(dev), torch.from_numpy(z[:n_train]).to(dev)
    emu = tpcf.Emulator(EMU_WIDTHS, seed=11, device=dev)
    emu.set_input_box(lo, hi)
    emu.fit_output_scaling(ytr, stream=stream)
    gt = torch.Generator(device=dev).manual_seed(5)
    n_steps, bs = 20000, 512
    t0 = time.perf_counter()
    for k in range(n_steps):
        i = torch.randint(0, n_train, (bs,), device=dev, generator=gt)
        lr = 2e-3 * 0.5 * (1 + math.cos(math.pi * k / n_steps)) + 1e-5
        emu.train_step(xtr[i].contiguous(), ytr[i].contiguous(), lr, stream=stream)
    torch.cuda.synchronize(dev)
    t_fit = time.perf_counter() - t0
    pred = emu.predict(torch.from_numpy(th[n_train:]).to(dev), stream=stream).cpu().numpy()
    tpcf.stream_status(stream)
    emu.close()
    nm = len(T.MULTIPOLES)
    p, r = pred.reshape(n_test, nm, -1), z[n_train:].reshape(n_test, nm, -1)
    err = np.abs(p - r).max(-1) / np.abs(r).max(-1)
    rep["accuracy"] = {"train_samples": n_train, "test_samples": n_test, "steps": n_steps, "batch": bs,
                       "median_rel_err": float(np.median(err)), "p95_rel_err": float(np.percentile(err, 95)),
                       "max_rel_err": float(err.max()), "train_s": t_fit, "model_samples_s": t_model,
                       "metric": "per sample and multipole: max over bins |emu - model| / max over bins |model|"}
    if with_cpu:
        setup = T.ModelSetup()
        t0 = time.perf_counter()
        T.model_direct(setup, (0.86, 2.7, 0.8, 0.828, 1.0, 0.0))
        rep["cpu_baseline"] = {"kind": "plain tree-level model (oracle)", "s_per_theta": time.perf_counter() - t0,
                               "cores": 1}
    return rep


def fp32_peak_tflops(dev):
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return 2.0 * 128 * sms * 2070e6 / 1e12


def roofline(cfg, d, dw, r, rw, dev, stream, tpcf, reps=3):
    """Pair stage alone: algorithmic FP32 FLOP / kernel time, against the FP32 FMA peak."""
    import numpy as np
    import torch
    alpha = float(dw.astype(np.float64).sum() / rw.astype(np.float64).sum())
    fx = np.concatenate([d, r])
    fw = np.concatenate([dw, (-alpha * rw.astype(np.float64)).astype(np.float32)])
    grid = tpcf.Grid(cfg, fx, fw, stream=stream, device=dev)
    out = None
    for _ in range(2):
        out = tpcf.accumulate_alm(grid, cfg, stream=stream)
    torch.cuda.synchronize(dev)
    pairs = int(out[4].sum().item())
    n_grid = grid.info()[0]
    _, gw, _ = grid.points(stream=stream)   # primary weights in grid order
    coupling = coupling_report(cfg, out[0], gw, out[1], out[2], out[3], dev, stream, tpcf)
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(reps):
        s.record(stream)
        tpcf.accumulate_alm(grid, cfg, stream=stream)
        e.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(s.elapsed_time(e))
    grid.close()
    t = statistics.median(ms) / 1000.0
    achieved = FLOP_PER_PAIR * pairs / t / 1e12
    peak = fp32_peak_tflops(dev)
    scalar_tf, paired_tf = tpcf.measure_fp32_peak(stream=stream)
    return {"bound": "alu", "kernel": "k_pairs_q (harmonic pair stage, D-R field)", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": PAIR_DRAM_BYTES_PER_PRIMARY * n_grid,
            "traffic_note": "bytes per launch, scaled by primaries from a capture of 400,000 primaries",
            "per_launch": {"pairs": pairs, "flop_per_pair": FLOP_PER_PAIR, "ms": t * 1000.0,
                           "primaries": n_grid},
            "peak_note": "FP32 FMA pipe: 2 x 128 lanes x SMs x 2070 MHz (recipe unit counts and max clock)",
            "measured_fp32": {"scalar_fma_tflops": scalar_tf, "ffma2_tflops": paired_tf,
                              "frac_of_scalar_fma": achieved / scalar_tf,
                              "note": "FMA-chain microbenchmark in this run (tpcf_measure_fp32_peak)"},
            "coupling": coupling}


def end_to_end(cfg, d, dw, r, rw, args, stream, tpcf, ws=1, rank=0):
    """The same metric through the public entry point from host buffers: the
    host-buffer estimate on one GPU; with several ranks the sharded estimate
    (partition, copies of the rank's share, partials, the sum over the group and
    the finished multipoles back on the host), timed as the slowest rank."""
    import numpy as np
    import torch
    from paper_2408_03036_gb300 import shard
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    hd, hdw, hr, hrw = pin(d), pin(dw), pin(r), pin(rw)
    steps = max(1, min(args.steps, 3))
    dev = torch.device("cuda", torch.cuda.current_device())

    def call():
        if ws > 1:
            res = shard.estimate_3pcf_sharded(cfg, hd, hdw, hr, hrw, rank, ws, device=dev, stream=stream)
            out = [res.zeta.cpu(), res.nnn.cpu(), res.rrr.cpu(), res.pair_counts.cpu(), res.triplet_counts.cpu()]
            return out, sum(t.numel() * t.element_size() for t in out)
        res = tpcf.estimate_3pcf_host(cfg, hd, hdw, hr, hrw, stream=stream)
        return res, res.zeta.nbytes + res.nnn.nbytes + res.rrr.nbytes + res.pair_counts.nbytes + \
            res.triplet_counts.nbytes

    call()   # warm
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    tot = 0.0
    for _ in range(steps):
        s.record(stream)
        _, bo = call()
        e.record(stream)
        torch.cuda.synchronize()
        tot += s.elapsed_time(e)
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([tot], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot = float(t.item())
    bi = hd.nbytes + hdw.nbytes + hr.nbytes + hrw.nbytes
    return {"value": (ND + NR) * steps / (tot / 1000.0), "unit": UNIT, "h2d_bytes_per_step": int(bi),
            "d2h_bytes_per_step": int(bo), "steps": steps}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "bf16x3", "tf32x3"], default="bf16x3",
                    help="coupling arithmetic of the headline step (the plain FP32 step is timed beside it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mocks", type=int, default=N_MOCKS, help="mocks in the covariance batch (0: skip)")
    ap.add_argument("--no-precision", action="store_true", help="skip the per-multipole precision report")
    ap.add_argument("--no-variants", action="store_true", help="skip the 2PCF / full-edge / varying-LOS timings")
    ap.add_argument("--no-emulator", action="store_true", help="skip the emulator throughput report")
    ap.add_argument("--batch-steps", type=int, default=1, help="timed graph launches of the batch")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)   # at least three untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
