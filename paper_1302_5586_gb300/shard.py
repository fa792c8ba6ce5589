"""Row-band decompositions over several ranks: one large image's conv2d
(read-only halo rows, no exchange) and the Jacobi iteration (halo exchange).

Convolution of one image (`BandConv2d`): rank q computes the output rows
[r0, r1) of an even split of the image's rows.  It reads input rows
[r0 - kh//2, r1 + kh - 1 - kh//2), clipped to the image: inside that
sub-image every window of an owned output row reads the same rows as in the
whole image (at the image's top and bottom edge the sub-image's edge row is
the image's, so clamp-to-edge clamps to the same row), so the owned rows are
the same bits as one undivided call.  Nothing is exchanged; gathering the
bands (if wanted) is one all-gather.

Jacobi:

The grid's rows are split into contiguous bands, one per rank (rank 0 also
owns the top boundary row, the last rank the bottom one).  A rank holds its
band plus `halo` rows above and below.  Every `halo` sweeps the ranks swap
their outermost owned rows with their neighbours (one point-to-point message
per neighbour and direction), then each runs `halo` sweeps on its local array
treating the array's first and last rows as fixed: stale data in the halo
rows moves inward one row per sweep and never reaches the owned rows, so the
owned rows are the same bits as on one undivided grid.  The residual of an
iterate is the FP64 sum over each band's owned interior rows, summed across
ranks with one all-reduce of a single double, then square-rooted.

The sweep and the residual are passed in (`sweep(local, n)` and
`resid(sub)`), so the same code drives the library's CUDA kernels on device
tensors (NCCL) or any host implementation on CPU tensors (gloo).
"""
from __future__ import annotations

import math


def conv_band_bounds(h: int, rank: int, world: int):
    """Output rows [r0, r1) of `rank` in an even split of h rows."""
    q, rem = divmod(h, world)
    r0 = rank * q + min(rank, rem)
    return r0, r0 + q + (1 if rank < rem else 0)


class BandConv2d:
    """One rank's share of a clamp-to-edge conv2d of one h-row image with a
    kh-row filter: the input rows it reads and the output rows it owns."""

    def __init__(self, h: int, kh: int, rank: int, world: int):
        if kh < 1 or h < 1 or world < 1 or not 0 <= rank < world:
            raise ValueError("need h >= 1, kh >= 1 and 0 <= rank < world")
        self.h, self.kh, self.rank, self.world = h, kh, rank, world
        self.r0, self.r1 = conv_band_bounds(h, rank, world)
        ah = kh // 2
        self.lo = max(0, self.r0 - ah) if self.r1 > self.r0 else self.r0
        self.hi = min(h, self.r1 + kh - 1 - ah) if self.r1 > self.r0 else self.r0

    def input_rows(self):
        """Global input rows [lo, hi) the rank reads (its band plus halo rows)."""
        return self.lo, self.hi

    def owned(self, sub_out):
        """The owned output rows inside the sub-image's output (rows of the
        last axis but one)."""
        return sub_out[..., self.r0 - self.lo:self.r1 - self.lo, :]

    def run(self, img, conv):
        """conv(sub_image) -> output of the same shape; returns the owned rows.
        `img` holds all rows (e.g. a read-only mapping); only [lo, hi) are read."""
        sub = img[..., self.lo:self.hi, :]
        if self.r1 == self.r0:  # more ranks than rows: nothing to compute
            return sub
        return self.owned(conv(sub))


def band_bounds(h: int, rank: int, world: int):
    """Rows [r0, r1) owned by `rank`: the interior rows 1..h-2 split as evenly
    as possible, the boundary rows attached to the first and last bands."""
    inner = max(h - 2, 0)
    q, rem = divmod(inner, world)
    r0 = 1 + rank * q + min(rank, rem)
    r1 = r0 + q + (1 if rank < rem else 0)
    if rank == 0:
        r0 = 0
    if rank == world - 1:
        r1 = h
    return r0, r1


class BandJacobi:
    """One rank's share of an h x w Jacobi iteration."""

    def __init__(self, h: int, w: int, rank: int, world: int, halo: int, dist, group=None):
        self.h, self.w, self.rank, self.world, self.halo = h, w, rank, world, max(1, halo)
        self.dist, self.group = dist, group
        self.r0, self.r1 = band_bounds(h, rank, world)
        for q in range(world):  # every band must hold at least `halo` rows
            a, z = band_bounds(h, q, world)
            if z - a < self.halo:
                raise ValueError(f"band of rank {q} has {z - a} rows, fewer than the halo ({self.halo})")
        self.lo = max(0, self.r0 - self.halo)
        self.hi = min(h, self.r1 + self.halo)

    def local_slice(self):
        """Global rows held locally: [lo, hi)."""
        return self.lo, self.hi

    def owned(self, local):
        """View of the owned rows inside the local array."""
        return local[self.r0 - self.lo:self.r1 - self.lo]

    def exchange(self, local):
        """Send the outermost `halo` owned rows to each neighbour and receive
        its rows into the matching halo rows."""
        d, reqs, k = self.dist, [], self.halo
        top, bot = self.r0 - self.lo, self.hi - self.r1  # halo rows present above / below
        if self.rank > 0 and top > 0:
            send = local[top:top + min(k, top)].contiguous()
            recv = local[0:top]
            buf = recv.contiguous().clone()
            reqs.append((d.isend(send, self.rank - 1, group=self.group), None, None))
            reqs.append((d.irecv(buf, self.rank - 1, group=self.group), recv, buf))
        if self.rank < self.world - 1 and bot > 0:
            n = local.shape[0]
            send = local[n - bot - min(k, bot):n - bot].contiguous()
            recv = local[n - bot:n]
            buf = recv.contiguous().clone()
            reqs.append((d.isend(send, self.rank + 1, group=self.group), None, None))
            reqs.append((d.irecv(buf, self.rank + 1, group=self.group), recv, buf))
        for req, dst, buf in reqs:
            req.wait()
            if dst is not None:
                dst.copy_(buf)

    def residual(self, local, resid):
        """sqrt of the all-reduced sum over owned interior rows of r^2."""
        a = max(self.r0 - 1, 0) - self.lo
        b = min(self.r1 + 1, self.h) - self.lo
        part = resid(local[a:b]) ** 2
        t = self._tensor_like(local, part)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return math.sqrt(float(t.item()))

    @staticmethod
    def _tensor_like(local, value):
        import torch
        return torch.tensor([value], dtype=torch.float64, device=local.device)

    def run(self, local, iters: int, check_every: int, sweep, resid):
        """iters sweeps on the local array; residuals of the iterates after
        sweeps m*check_every (returned as a list, identical on every rank)."""
        res = []
        done = 0
        while done < iters:
            self.exchange(local)
            # never step past a checkpoint: the residual needs fresh halo rows
            n = min(self.halo, iters - done)
            if check_every > 0:
                n = min(n, check_every - done % check_every)
            sweep(local, n)
            done += n
            if check_every > 0 and done % check_every == 0:
                self.exchange(local)
                res.append(self.residual(local, resid))
        return res
