"""Multi-rank logic of bench.py on CPU ranks (gloo, world size 2).

Each rank contributes its own timing; rank 0 must see the maximum, and the
whole-job value counts the units of every rank over that maximum (replicas,
weak scaling).
"""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _worker(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    b = _bench()
    elapsed = [1.5, 2.5][rank]
    m = b.max_over_ranks(elapsed, dist, "cpu")
    v = b.aggregate_rate(world, 1000.0, m)
    q.put((rank, m, v))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, m, v in res:
        assert m == 2.5
        assert v == pytest.approx(2 * 1000.0 / 2.5)


def test_single_rank_is_identity():
    b = _bench()
    assert b.max_over_ranks(3.0) == 3.0
    assert b.aggregate_rate(1, 10.0, 2.0) == 5.0


def test_denoiser_flops_against_the_oracle_layer_list():
    """The FLOP count behind the denoiser line, recounted from the oracle's
    layer list: each layer's level from its name (encoder 'enc{l}', decoder
    'dec{l}'), 2 k^2 Cin Cout multiply-adds per pixel of that level."""
    from oracle import unet
    b = _bench()
    for levels, base, n in [(5, 32, 512), (3, 64, 128), (1, 32, 64)]:
        ref = 0.0
        for name, co, ci, k in unet.layer_specs(levels, base):
            lv = int(name[3:].split(".")[0]) if name != "head" else 0
            ref += 2.0 * k * k * ci * co * (n >> lv) ** 2
        assert b.denoiser_flops(levels, base, n) == ref


def test_onchip_roofline_arithmetic(monkeypatch):
    """roofline.onchip = committed wavefronts per launch / launch time against
    one 128-byte wavefront per SM per clock; None without a committed count,
    a launch time or a clock."""
    b = _bench()
    monkeypatch.setattr(b, "profile_value", lambda k, w, key: 1.0e7 if key == "smem_wavefronts_per_launch" else None)
    r = b.onchip_roofline("k", "w", 50e-6, 2000.0, sms=100)
    assert r["achieved"] == 1.0e7 / 50e-6
    assert r["peak"] == 100 * 2000.0 * 1e6
    assert abs(r["frac"] - (1.0e7 / 50e-6) / (100 * 2.0e9)) < 1e-12
    assert b.onchip_roofline("k", "w", 0.0, 2000.0) is None
    assert b.onchip_roofline("k", "w", 50e-6, None) is None
    monkeypatch.setattr(b, "profile_value", lambda k, w, key: None)
    assert b.onchip_roofline("k", "w", 50e-6, 2000.0) is None
