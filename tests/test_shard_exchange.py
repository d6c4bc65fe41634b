"""The data plane of the slab-distributed solve (paradiag_gb300.shard) on CPU:
the halo exchange of grid lines, the all-to-all from line slabs to frequency
slabs and back, and the all-reduce of the residual norm, over a gloo process
group of world size 2 and 3 (one process per rank) and with the in-process
exchange.  The frequency slabs must equal the rows of the whole spectrum bit
for bit (the single-rank transpose), the round trip must give back every
rank's owned lines, and the halos must hold the neighbours' boundary lines.

The spectrum of a rank lives in its slab plan on a GPU; here a CPU tensor
stands in for it (the pack / unpack copies are the only plan calls of the
exchange), so the test runs without a GPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NT, NH, LINES, PTS, PITCH = 6, 5, 11, 3, 4


def _global_spectrum(torch):
    """The whole step-(b) spectrum [nh][lines][2 pitch] (float32 pairs), seeded."""
    import workloads as W
    v = W.uniform(W.SEED_BASE + 80, NH * LINES * 2 * PITCH, -1.0, 1.0)
    return torch.tensor(v, dtype=torch.float32).view(NH, LINES, 2 * PITCH)


def _global_field(torch):
    import workloads as W
    v = W.uniform(W.SEED_BASE + 81, NT * LINES * PTS, -1.0, 1.0)
    return torch.tensor(v, dtype=torch.float64).view(NT, LINES, PTS)


def _fake_rank(torch, layout, r):
    """A RankState whose spectrum is a CPU tensor [nh][ys + 2][2 pitch]."""
    from paradiag_gb300 import shard

    class FakeRank(shard.RankState):
        def __init__(self):
            self.torch, self.layout, self.r = torch, layout, r
            self.l0, self.l1 = layout.line_ranges[r]
            self.ys = self.l1 - self.l0
            self.nt, self.pitch = NT, PITCH
            self.ex = shard._SpectrumSlabs(torch, layout, r, PITCH, torch.float32, "cpu")
            self.spec = torch.full((NH, self.ys + 2, 2 * PITCH), float("nan"))
            self.u = torch.zeros((NT, (self.ys + 2) * PTS), dtype=torch.float64)

        def pack(self):
            offs = shard._offsets(self.ex.send_counts)
            for d in range(layout.world):
                k0, k1 = layout.k_ranges[d]
                n = self.ex.send_counts[d]
                self.ex.send[offs[d]:offs[d] + n].copy_(self.spec[k0:k1, 1:self.ys + 1, :].reshape(-1))

        def unpack(self):
            offs = shard._offsets(self.ex.send_counts)
            self.spec[:, 0, :] = 0.0
            self.spec[:, self.ys + 1, :] = 0.0
            for s in range(layout.world):
                k0, k1 = layout.k_ranges[s]
                n = self.ex.send_counts[s]
                self.spec[k0:k1, 1:self.ys + 1, :].copy_(
                    self.ex.recv2[offs[s]:offs[s] + n].view(k1 - k0, self.ys, 2 * PITCH))

    rk = FakeRank()
    g, f = _global_spectrum(torch), _global_field(torch)
    rk.spec[:, 1:rk.ys + 1, :].copy_(g[:, rk.l0:rk.l1, :])
    rk.view(rk.u)[:, 1:rk.ys + 1, :].copy_(f[:, rk.l0:rk.l1, :])
    return rk


def _verify(torch, layout, ranks, g, f):
    for rk in ranks:
        k0, k1 = layout.k_ranges[rk.r]
        assert torch.equal(rk.ex.kslab, g[k0:k1])                      # the transpose, bit for bit
        v = rk.view(rk.u)
        lo = f[:, rk.l0 - 1, :] if rk.l0 > 0 else torch.zeros_like(f[:, 0, :])
        hi = f[:, rk.l1, :] if rk.l1 < LINES else torch.zeros_like(f[:, 0, :])
        assert torch.equal(v[:, 0, :], lo) and torch.equal(v[:, rk.ys + 1, :], hi)
        assert torch.equal(v[:, 1:rk.ys + 1, :], f[:, rk.l0:rk.l1, :])


@pytest.mark.parametrize("world", [1, 2, 3])
def test_local_exchange_transpose_and_halo(world):
    import torch
    from paradiag_gb300 import shard
    layout = shard.SlabLayout(LINES, PTS, NH, world)
    ranks = [_fake_rank(torch, layout, r) for r in range(world)]
    ex = shard.LocalExchange(torch)
    ex.halo(ranks, "u")
    ex.to_kslab(ranks)
    g, f = _global_spectrum(torch), _global_field(torch)
    _verify(torch, layout, ranks, g, f)
    ex.from_kslab(ranks)
    for rk in ranks:
        assert torch.equal(rk.spec[:, 1:rk.ys + 1, :], g[:, rk.l0:rk.l1, :])
        assert float(rk.spec[:, 0, :].abs().sum()) == 0.0
    assert ex.allreduce_sum([1.5] * world) == 1.5 * world


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paradiag_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        layout = shard.SlabLayout(LINES, PTS, NH, world)
        rk = _fake_rank(torch, layout, rank)
        ex = shard.DistExchange(torch)
        ex.halo([rk], "u")
        ex.to_kslab([rk])
        g, f = _global_spectrum(torch), _global_field(torch)
        _verify(torch, layout, [rk], g, f)
        ex.from_kslab([rk])
        assert torch.equal(rk.spec[:, 1:rk.ys + 1, :], g[:, rk.l0:rk.l1, :])
        s = ex.allreduce_sum([float(rank + 1)])
        assert s == world * (world + 1) / 2
        q.put((rank, "ok"))
    except Exception as e:        # reported to the parent, which fails the test
        q.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_exchange_matches_single_rank_transpose(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    assert out == [(r, "ok") for r in range(world)], out


def test_slab_layout_and_space():
    from paradiag_gb300 import shard
    lay = shard.SlabLayout(255, 255, 129, 4)
    assert lay.line_ranges[0] == (0, 64) and lay.line_ranges[-1] == (192, 255)
    assert sum(b - a for a, b in lay.k_ranges) == 129
    sp = dict(dim=2, nx=255, ny=255, ly=1.0)
    s = shard.slab_space(sp, 255, 64, 128)
    # the slab keeps the whole grid's spacing h_y = 1/256
    assert s["ny"] == 66 and abs(s["ly"] / (s["ny"] + 1) - 1.0 / 256) < 1e-15
    s1 = shard.slab_space(dict(dim=1, nx=127, lx=1.0), 127, 10, 20)
    assert s1["nx"] == 12 and abs(s1["lx"] / 13 - 1.0 / 128) < 1e-15
