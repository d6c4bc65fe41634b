"""A ParaDiag-II solve spread over several GPUs: slabs of grid lines for the
residual and the time transforms, slabs of time frequencies for step (b).

Steps (a) and (c) of eq. 1.3 act on every spatial point independently and
step (b) on every time frequency independently (the paper's discussion after
Lemma 1), so rank r of G owns

* the grid lines [l0_r, l1_r) of the slab direction (y in 2D, x for a 1D
  Dirichlet problem) for the residual r = b - A u (eq. 5.1), the Gamma scaling
  and FFT along t, the x-eigentransforms (2D) and the update;
* the frequencies [k0_r, k1_r) of the half spectrum for the shifted solves.

One iteration of the stationary method eq. 5.1 then reads
  halo exchange of u (one grid line to each neighbour, every time level)
  r = b - A u on the rank's slab plan (its lines plus one halo line each side)
  ||r||^2 over the owned lines, summed over the ranks (an all-reduce)
  step (a) (+ forward x-transform)            pd_precond_forward
  all-to-all: line slabs -> frequency slabs   (the exchange below)
  step (b) on the frequency slab              pd_precond_solve_rows (whole-grid plan)
  all-to-all back: frequency slabs -> line slabs
  (inverse x-transform +) step (c)            pd_precond_backward
  u += z on the owned lines                   pd_shard_update
Every arithmetic step runs in the library's kernels; this module only moves
data (slab copies, halo exchange, all-to-all, the all-reduce of one FP64
scalar).  The exchange volume per iteration is the spectrum twice (4 bytes
per real unknown each way on mixed plans) plus two grid lines per rank.

Two exchange backends share the algorithm: DistExchange (one rank per
process, torch.distributed: NCCL on GPUs, gloo on CPU tensors) and
LocalExchange (every rank in one process, on one device: the exchange is a
set of local copies), which checks the slab logic on a single GPU.
"""
from __future__ import annotations

import math


def split_range(n: int, parts: int, i: int):
    """[start, stop) of part i of n items split into `parts` near-equal parts."""
    base, extra = divmod(n, parts)
    start = i * base + min(i, extra)
    return start, start + base + (1 if i < extra else 0)


class SlabLayout:
    """Line slabs and frequency slabs of a world of G ranks.

    lines: grid lines of the slab direction (ny in 2D, nx in 1D); pts: points
    per line (nx in 2D, 1 in 1D); nh: frequencies of the half spectrum."""

    def __init__(self, lines: int, pts: int, nh: int, world: int):
        if world < 1 or world > lines or world > nh:
            raise ValueError("need 1 <= world <= min(lines, frequencies)")
        self.lines, self.pts, self.nh, self.world = lines, pts, nh, world
        self.line_ranges = [split_range(lines, world, r) for r in range(world)]
        self.k_ranges = [split_range(nh, world, r) for r in range(world)]

    def owned(self, r):
        l0, l1 = self.line_ranges[r]
        return l1 - l0


def slab_space(space: dict, lines: int, l0: int, l1: int) -> dict:
    """Space of the slab plan of lines [l0, l1): those lines plus one halo line
    on each side, the grid spacing of the whole problem kept (a Dirichlet
    direction with n interior points has h = L/(n+1), so the slab with n + 2
    lines has length h (n + 3))."""
    s = dict(space)
    ext = l1 - l0 + 2
    if space.get("dim", 1) == 2:
        h = space.get("ly", 1.0) / (lines + 1)
        s["ny"], s["ly"] = ext, h * (ext + 1)
    else:
        h = space.get("lx", 1.0) / (lines + 1)
        s["nx"], s["lx"] = ext, h * (ext + 1)
    return s


class _SpectrumSlabs:
    """Device buffers of one rank's exchange: the outgoing blocks, the
    incoming blocks and the frequency slab [ks][lines][pitch] (pitch complex
    values, as float32 / float64 pairs)."""

    def __init__(self, torch, layout: SlabLayout, r: int, pitch: int, dtype, device):
        self.layout, self.r, self.pitch = layout, r, pitch
        k0, k1 = layout.k_ranges[r]
        ks, ys = k1 - k0, layout.owned(r)
        self.kslab = torch.zeros((ks, layout.lines, 2 * pitch), dtype=dtype, device=device)
        # to rank d: frequencies of d x my lines; from rank s: my frequencies x lines of s
        self.send_counts = [(layout.k_ranges[d][1] - layout.k_ranges[d][0]) * ys * 2 * pitch
                            for d in range(layout.world)]
        self.recv_counts = [ks * layout.owned(s) * 2 * pitch for s in range(layout.world)]
        self.send = torch.zeros(sum(self.send_counts), dtype=dtype, device=device)
        self.recv = torch.zeros(sum(self.recv_counts), dtype=dtype, device=device)
        # the reverse exchange swaps the roles
        self.send2 = torch.zeros(sum(self.recv_counts), dtype=dtype, device=device)
        self.recv2 = torch.zeros(sum(self.send_counts), dtype=dtype, device=device)


def _offsets(counts):
    out, acc = [], 0
    for c in counts:
        out.append(acc)
        acc += c
    return out


class RankState:
    """One rank's plans and arrays: the slab plan, the whole-grid plan for
    step (b), the slab's b, u (with halo lines) and work arrays."""

    def __init__(self, pd, torch, space: dict, nt, dt, alpha, scheme, theta, precision,
                 layout: SlabLayout, r: int, device):
        self.pd, self.torch, self.layout, self.r = pd, torch, layout, r
        l0, l1 = layout.line_ranges[r]
        self.l0, self.l1 = l0, l1
        self.ys = l1 - l0
        self.local = pd.Plan(slab_space(space, layout.lines, l0, l1), nt, dt, alpha, scheme, theta,
                             precision)
        self.whole = pd.Plan(space, nt, dt, alpha, scheme, theta, precision)
        st, _, nh, lines, pitch, eb = pd.pd_plan_spectrum(self.local.handle)
        if st != pd.PD_OK:
            raise pd.PDError(st, "pd_plan_spectrum")
        self.pitch = pitch
        dtype = torch.float32 if eb == 8 else torch.float64
        self.ex = _SpectrumSlabs(torch, layout, r, pitch, dtype, device)
        self.S_ext = (self.ys + 2) * layout.pts
        self.nt = nt
        z = lambda: torch.zeros((nt, self.S_ext), dtype=torch.float64, device=device)
        self.b, self.u, self.r_, self.z = z(), z(), z(), z()

    def close(self):
        self.local.close()
        self.whole.close()

    # the lines of the slab plan are 0 (halo), 1 .. ys (owned), ys + 1 (halo)
    def view(self, x):
        return x.view(self.nt, self.ys + 2, self.layout.pts)

    def check(self, st, what):
        if st != self.pd.PD_OK:
            raise self.pd.PDError(st, what)

    def pack(self):
        """Owned lines of the step-(b) spectrum into the send buffer, one
        block per destination's frequency range."""
        ex, L = self.ex, self.layout
        offs = _offsets(ex.send_counts)
        for d in range(L.world):
            k0, k1 = L.k_ranges[d]
            if k1 > k0 and self.ys > 0:
                self.check(self.pd.pd_spectrum_get(self.local.handle, k0, k1, 1, self.ys + 1,
                                                   ex.send[offs[d]:].data_ptr()), "pd_spectrum_get")

    def unpack_kslab(self):
        """Incoming blocks (my frequencies x the lines of each source) into the
        frequency slab."""
        ex, L = self.ex, self.layout
        offs = _offsets(ex.recv_counts)
        ks = L.k_ranges[self.r][1] - L.k_ranges[self.r][0]
        for s in range(L.world):
            a0, a1 = L.line_ranges[s]
            blk = ex.recv[offs[s]:offs[s] + ex.recv_counts[s]].view(ks, a1 - a0, 2 * self.pitch)
            ex.kslab[:, a0:a1, :].copy_(blk)

    def pack_kslab(self):
        """The frequency slab, split by the destinations' lines, into the
        reverse send buffer."""
        ex, L = self.ex, self.layout
        offs = _offsets(ex.recv_counts)
        ks = L.k_ranges[self.r][1] - L.k_ranges[self.r][0]
        for d in range(L.world):
            a0, a1 = L.line_ranges[d]
            ex.send2[offs[d]:offs[d] + ex.recv_counts[d]].view(ks, a1 - a0, 2 * self.pitch).copy_(
                ex.kslab[:, a0:a1, :])

    def unpack(self):
        """Incoming blocks (each source's frequencies x my lines) back into the
        slab plan's spectrum; the halo lines' spectrum is zeroed."""
        ex, L = self.ex, self.layout
        offs = _offsets(ex.send_counts)
        pd, h = self.pd, self.local.handle
        nh = L.nh
        self.check(pd.pd_spectrum_put(h, 0, nh, 0, 1, None), "pd_spectrum_put")
        self.check(pd.pd_spectrum_put(h, 0, nh, self.ys + 1, self.ys + 2, None), "pd_spectrum_put")
        for s in range(L.world):
            k0, k1 = L.k_ranges[s]
            if k1 > k0 and self.ys > 0:
                self.check(pd.pd_spectrum_put(h, k0, k1, 1, self.ys + 1,
                                              ex.recv2[offs[s]:].data_ptr()), "pd_spectrum_put")


class LocalExchange:
    """Every rank in this process: the collectives are local copies."""

    def __init__(self, torch):
        self.torch = torch

    def halo(self, ranks, field):
        """Line 1 of rank r goes to the top halo of rank r-1, line ys of rank r
        to the bottom halo of rank r+1 (every time level); the outer halos of
        the first and last rank stay zero (Dirichlet)."""
        G = len(ranks)
        for r in range(G):
            v = ranks[r].view(getattr(ranks[r], field))
            if r > 0:
                w = ranks[r - 1].view(getattr(ranks[r - 1], field))
                v[:, 0, :].copy_(w[:, ranks[r - 1].ys, :])
            if r < G - 1:
                w = ranks[r + 1].view(getattr(ranks[r + 1], field))
                v[:, ranks[r].ys + 1, :].copy_(w[:, 1, :])

    def to_kslab(self, ranks):
        for rk in ranks:
            rk.pack()
        G = len(ranks)
        for r in range(G):
            so = _offsets(ranks[r].ex.send_counts)
            for d in range(G):
                ro = _offsets(ranks[d].ex.recv_counts)
                n = ranks[r].ex.send_counts[d]
                ranks[d].ex.recv[ro[r]:ro[r] + n].copy_(ranks[r].ex.send[so[d]:so[d] + n])
        for rk in ranks:
            rk.unpack_kslab()

    def from_kslab(self, ranks):
        for rk in ranks:
            rk.pack_kslab()
        G = len(ranks)
        for r in range(G):
            so = _offsets(ranks[r].ex.recv_counts)
            for d in range(G):
                ro = _offsets(ranks[d].ex.send_counts)
                n = ranks[r].ex.recv_counts[d]
                ranks[d].ex.recv2[ro[r]:ro[r] + n].copy_(ranks[r].ex.send2[so[d]:so[d] + n])
        for rk in ranks:
            rk.unpack()

    def allreduce_sum(self, values):
        return sum(values)


class DistExchange:
    """One rank per process over a torch.distributed process group."""

    def __init__(self, torch, group=None):
        import torch.distributed as dist
        self.torch, self.dist, self.group = torch, dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def halo(self, ranks, field):
        (rk,) = ranks
        torch, dist = self.torch, self.dist
        v = rk.view(getattr(rk, field))
        ops, bufs = [], []
        r, G = self.rank, self.world
        if r > 0:       # my first line to r-1; its last line into my bottom halo
            sb = v[:, 1, :].contiguous()
            rb = torch.empty_like(sb)
            ops += [dist.P2POp(dist.isend, sb, r - 1, self.group),
                    dist.P2POp(dist.irecv, rb, r - 1, self.group)]
            bufs.append((rb, 0))
        if r < G - 1:   # my last line to r+1; its first line into my top halo
            sb = v[:, rk.ys, :].contiguous()
            rb = torch.empty_like(sb)
            ops += [dist.P2POp(dist.isend, sb, r + 1, self.group),
                    dist.P2POp(dist.irecv, rb, r + 1, self.group)]
            bufs.append((rb, rk.ys + 1))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for rb, line in bufs:
            v[:, line, :].copy_(rb)

    def _a2a(self, out, inp, out_counts, in_counts):
        self.dist.all_to_all_single(out, inp, output_split_sizes=out_counts,
                                    input_split_sizes=in_counts, group=self.group)

    def to_kslab(self, ranks):
        (rk,) = ranks
        rk.pack()
        self._a2a(rk.ex.recv, rk.ex.send, rk.ex.recv_counts, rk.ex.send_counts)
        rk.unpack_kslab()

    def from_kslab(self, ranks):
        (rk,) = ranks
        rk.pack_kslab()
        self._a2a(rk.ex.recv2, rk.ex.send2, rk.ex.send_counts, rk.ex.recv_counts)
        rk.unpack()

    def allreduce_sum(self, values):
        (v,) = values
        t = self.torch.tensor([v], dtype=self.torch.float64,
                              device="cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu")
        self.dist.all_reduce(t, group=self.group)
        return float(t.item())


class ShardedSolver:
    """The stationary iteration eq. 5.1 over G ranks.  `ranks` holds the
    RankState of every rank this process runs (all of them for LocalExchange,
    its own for DistExchange)."""

    def __init__(self, pd, torch, ranks, exchange):
        self.pd, self.torch, self.ranks, self.ex = pd, torch, ranks, exchange

    def set_rhs(self, b_lines):
        """b_lines[i]: the rank's owned part of b, [Nt][ys * pts]."""
        for rk, bl in zip(self.ranks, b_lines):
            rk.view(rk.b)[:, 1:rk.ys + 1, :].copy_(bl.view(rk.nt, rk.ys, -1))

    def solve(self, tol=1e-10, maxit=50):
        pd = self.pd
        for rk in self.ranks:
            rk.u.zero_()
        nb2 = self.ex.allreduce_sum([self._norm2(rk, rk.b) for rk in self.ranks])
        nb = math.sqrt(nb2)
        it, rel = 0, float("inf")
        while True:
            self.ex.halo(self.ranks, "u")
            for rk in self.ranks:
                rk.check(pd.pd_residual(rk.local.handle, rk.b.data_ptr(), rk.u.data_ptr(),
                                        rk.r_.data_ptr()), "pd_residual")
                # the halo lines' residual is not this rank's (its outer
                # neighbours are missing): zero it before the transforms, whose
                # FP16 scaling follows the largest value of the slab
                v = rk.view(rk.r_)
                v[:, 0, :].zero_()
                v[:, rk.ys + 1, :].zero_()
            nr2 = self.ex.allreduce_sum([self._norm2(rk, rk.r_) for rk in self.ranks])
            rel = math.sqrt(nr2) / nb if nb > 0 else math.sqrt(nr2)
            if not math.isfinite(rel):
                raise pd.PDError(pd.PD_ERR_NONFINITE, "sharded solve")
            if rel <= tol or it >= maxit:
                break
            for rk in self.ranks:
                rk.check(pd.pd_precond_forward(rk.local.handle, rk.r_.data_ptr()),
                         "pd_precond_forward")
            self.ex.to_kslab(self.ranks)
            for rk in self.ranks:
                k0, k1 = rk.layout.k_ranges[rk.r]
                rk.check(pd.pd_precond_solve_rows(rk.whole.handle, k0, k1,
                                                  rk.ex.kslab.data_ptr()), "pd_precond_solve_rows")
            self.ex.from_kslab(self.ranks)
            for rk in self.ranks:
                rk.check(pd.pd_precond_backward(rk.local.handle, rk.z.data_ptr()),
                         "pd_precond_backward")
                rk.check(pd.pd_shard_update(rk.local.handle, rk.z.data_ptr(), rk.u.data_ptr(), 1,
                                            rk.ys), "pd_shard_update")
            it += 1
        if rel > tol:
            raise pd.PDError(pd.PD_ERR_NOT_CONVERGED, "sharded solve reached maxit")
        return it, rel

    def _norm2(self, rk, x):
        st, v = self.pd.pd_shard_norm2(rk.local.handle, x.data_ptr(), 1, rk.ys)
        rk.check(st, "pd_shard_norm2")
        return v

    def owned(self, rk, x):
        """The rank's owned lines of a slab array, [Nt][ys * pts]."""
        return rk.view(x)[:, 1:rk.ys + 1, :].reshape(rk.nt, -1)
