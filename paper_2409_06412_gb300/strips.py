"""Row-strip decomposition of ONE lattice over ranks (one GPU per rank), with
a halo of K_t rows exchanged every K_t BBK steps.

The configurations of a batch shard with no exchange at all (``sharding``);
this module is for a single lattice too large for one GPU.  The lattice
(site s = y Lx + x, rows contiguous) is cut along y into strips of whole rows.
Rank r owns global rows [y0, y0 + rows) and holds them in a buffer of
rows + 2 K_t rows: K_t ghost rows above (global y0 - K_t .. y0 - 1, owned by
the rank ``up``) and K_t below (owned by ``down``), periodic in y.

One BBK step reads the angles of the four nearest neighbours (Eq.
XY-Hamilton-Field), so in the leapfrog storage (theta_k, v_k) each step makes
one more row at either end of the buffer stale: after j steps of a window the
state is exact on local rows [j, R - j), and after K_t steps exactly on the
owned rows.  Then each rank sends its first K_t owned rows to ``up`` (they
become up's lower ghost rows) and its last K_t owned rows to ``down`` (down's
upper ghost rows), and the next window starts.  A window of K_t steps updates
rows + 2 (K_t - j) rows at step j, so it recomputes K_t (K_t - 1) rows over
rows x K_t owned row-steps: the price of exchanging once per K_t steps instead
of every step.

Every halo block is K_t x Lx contiguous sites of each state array of a
lattice, so on GPUs one exchange is two peer copies per array and lattice
(``cudaMemcpyPeerAsync`` into the neighbour's ghost rows, on a copy stream);
no TMA multicast: each block has exactly one reader.  Noise stays keyed by
the global site index, so the split run reproduces the whole-lattice run bit
for bit, and the FP64 moment partial sums over owned rows add up across ranks
(``sharding.reduce_moments``).

This module plans and performs the exchange on the host: ``plan_strips``,
``halo_copies`` (the copy list, in local rows), ``apply_copies`` (all ranks'
buffers in one process) and ``exchange`` (one rank's buffers over
torch.distributed point-to-point messages: gloo on the CPU, NCCL on GPUs).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Strip:
    """Rows of one rank.  Local row i of its buffer is global row
    (y0 - halo + i) mod Ly, i = 0 .. rows + 2 halo - 1."""
    rank: int
    y0: int
    rows: int
    halo: int
    Lx: int
    Ly: int
    up: int
    down: int

    @property
    def buffer_rows(self) -> int:
        return self.rows + 2 * self.halo

    @property
    def buffer_y0(self) -> int:
        """Global row of local row 0."""
        return (self.y0 - self.halo) % self.Ly

    @property
    def owned(self) -> slice:
        """Local rows of the owned rows."""
        return slice(self.halo, self.halo + self.rows)

    def global_rows(self) -> np.ndarray:
        return (self.buffer_y0 + np.arange(self.buffer_rows)) % self.Ly

    def exact_rows(self, j: int) -> tuple[int, int]:
        """Local rows [lo, hi) still exact after j steps of a window (the
        leapfrog state; the rows a stepper has to update at step j)."""
        if not 0 <= j <= self.halo:
            raise ValueError(f"a window has at most {self.halo} steps, got step {j}")
        return j, self.buffer_rows - j

    def fill(self, whole: np.ndarray) -> np.ndarray:
        """The buffer cut from a whole-lattice array (..., Ly, Lx)."""
        return np.ascontiguousarray(whole[..., self.global_rows(), :])

    def recompute_fraction(self) -> float:
        """Row-steps computed beyond the owned ones, per owned row-step."""
        return (self.halo - 1) / self.rows


@dataclass(frozen=True)
class HaloCopy:
    """Rows [src_row, src_row + n_rows) of rank src's buffer go to rows
    [dst_row, dst_row + n_rows) of rank dst's buffer.  ``upward`` marks the
    copy of the sender's first owned rows to its ``up`` neighbour."""
    src: int
    src_row: int
    dst: int
    dst_row: int
    n_rows: int
    upward: bool


def split_rows(Ly: int, world: int, align: int = 1) -> list[int]:
    """Rows per rank: Ly cut into ``world`` parts as even as possible, each a
    multiple of ``align`` (the band height of the stepping kernel)."""
    if world < 1 or align < 1 or Ly % align:
        raise ValueError(f"cannot split {Ly} rows over {world} ranks in units of {align}")
    units = Ly // align
    if units < world:
        raise ValueError(f"{Ly} rows give fewer than {world} units of {align}")
    base, extra = divmod(units, world)
    return [(base + (1 if r < extra else 0)) * align for r in range(world)]


def plan_strips(Lx: int, Ly: int, world: int, k_t: int, align: int = 1) -> list[Strip]:
    """One strip per rank, rank r below rank r - 1 (periodic).  Every strip
    must own at least k_t rows, so that each ghost block comes from one
    neighbour."""
    if k_t < 1:
        raise ValueError("k_t must be at least 1")
    rows = split_rows(Ly, world, align)
    if min(rows) < k_t:
        raise ValueError(f"a strip of {min(rows)} rows cannot feed a halo of {k_t} rows")
    out, y0 = [], 0
    for r, n in enumerate(rows):
        out.append(Strip(rank=r, y0=y0, rows=n, halo=k_t, Lx=Lx, Ly=Ly,
                         up=(r - 1) % world, down=(r + 1) % world))
        y0 += n
    return out


def halo_copies(strips: list[Strip]) -> list[HaloCopy]:
    """The copies of one exchange: two per rank (per state array)."""
    out = []
    for s in strips:
        u, d = strips[s.up], strips[s.down]
        # first owned rows -> the lower ghost rows of the rank above
        out.append(HaloCopy(s.rank, s.halo, u.rank, u.halo + u.rows, s.halo, True))
        # last owned rows -> the upper ghost rows of the rank below
        out.append(HaloCopy(s.rank, s.rows, d.rank, 0, s.halo, False))
    return out


def bytes_per_exchange(strips: list[Strip], bytes_per_site: int = 8) -> int:
    """Bytes moved by one exchange over all ranks (FP32 theta and v: 8)."""
    return sum(c.n_rows * strips[c.src].Lx * bytes_per_site for c in halo_copies(strips))


def window_lengths(n: int, k_t: int) -> list[int]:
    """Steps between exchanges: k_t, ..., k_t and the remainder."""
    return [k_t] * (n // k_t) + ([n % k_t] if n % k_t else [])


def apply_copies(buffers: list[list[np.ndarray]], copies: list[HaloCopy]) -> None:
    """Perform an exchange on all ranks' buffers held in one process:
    buffers[rank][a] is state array a of that rank, (rows, Lx).  Reads only
    owned rows and writes only ghost rows, so the order does not matter."""
    for c in copies:
        for a in range(len(buffers[c.src])):
            buffers[c.dst][a][c.dst_row:c.dst_row + c.n_rows] = buffers[c.src][a][c.src_row:c.src_row + c.n_rows]


def exchange(strip: Strip, arrays: list, strips: list[Strip], group=None) -> None:
    """One rank's side of an exchange over torch.distributed: ``arrays`` are
    its state buffers (torch tensors, or numpy arrays on the CPU, shape
    (rows, Lx)); their ghost rows are overwritten in place.  Messages carry the
    tag 2 a + (0 upward, 1 downward), so the two blocks a rank gets from a
    single neighbour (two ranks, periodic) stay apart.  A world of one copies
    its own rows."""
    import torch
    import torch.distributed as dist

    tens = [torch.from_numpy(a) if isinstance(a, np.ndarray) else a for a in arrays]
    copies = [c for c in halo_copies(strips) if c.src == strip.rank or c.dst == strip.rank]
    world = len(strips)
    if world == 1:
        for c in copies:
            for t in tens:
                t[c.dst_row:c.dst_row + c.n_rows] = t[c.src_row:c.src_row + c.n_rows].clone()
        return
    reqs, recv = [], []
    for a, t in enumerate(tens):
        for c in copies:
            tag = 2 * a + (0 if c.upward else 1)
            if c.src == strip.rank:
                blk = t[c.src_row:c.src_row + c.n_rows].contiguous()
                reqs.append(dist.isend(blk, dst=c.dst, group=group, tag=tag))
            if c.dst == strip.rank:
                blk = torch.empty_like(t[c.dst_row:c.dst_row + c.n_rows]).contiguous()
                reqs.append(dist.irecv(blk, src=c.src, group=group, tag=tag))
                recv.append((t, c, blk))
    for q in reqs:
        q.wait()
    for t, c, blk in recv:
        t[c.dst_row:c.dst_row + c.n_rows] = blk
