"""One inversion's swarm split across processes, one GPU each (the
synchronous swarm of Sec. 3.4 / Eq. 8: every generation evaluates all
particles, then the global best is the lowest personal best of the whole
swarm).

Each process holds a contiguous slice of the particles and evaluates them on
its own GPU; one exchange per generation joins the slices: an all-reduce
MIN of the 64-bit global-best keys ((float bits of the misfit) << 32 |
swarm-wide particle index: lowest misfit, lowest index on ties) and the
owner's personal-best position, broadcast as an all-reduce SUM to which
every other process adds zeros (exact).  The arithmetic of the swarm stays
in the library (afm_pso_init_slice / afm_pso_best_slice /
afm_pso_move_slice, afm_forward_batch); this module only moves the key and
the D coordinates between processes, so the split swarm is afm_invert's
swarm bit for bit.
"""
from __future__ import annotations

from . import afminv as A


def slice_of(P: int, rank: int, world: int):
    """Contiguous share [lo, hi) of P particles for a rank; the shares
    partition range(P) and differ in size by at most one."""
    q, r = divmod(P, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def key_index(key: int) -> int:
    return key & 0xFFFFFFFF


def exchange_dist(key: int, owner, D: int, device, group=None):
    """The swarm's global best from this process's slice: (minimum key over
    all processes, the owner's personal-best position of that particle).
    key: this slice's best key (non-negative, below 2**63); owner(kmin) ->
    (owns, pos): whether this process holds particle key_index(kmin) and, if
    so, its position, a float32 [D] tensor on `device` (CUDA for NCCL, CPU
    for gloo)."""
    import torch
    import torch.distributed as dist
    k = torch.tensor([key], dtype=torch.int64, device=device)
    dist.all_reduce(k, op=dist.ReduceOp.MIN, group=group)
    kmin = int(k.item())
    owns, p = owner(kmin)
    buf = p.clone() if owns else torch.zeros(D, dtype=torch.float32, device=device)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return kmin, buf


class Slice:
    """Particles lo .. hi - 1 of the swarm of cfg.P on this process's GPU."""

    def __init__(self, prob, U, cfg, lo: int, hi: int, device=None):
        self.prob, self.U, self.cfg, self.lo, self.hi = prob, U, cfg, lo, hi
        self.D = int(prob.n_free)
        self.sw = A.pso_init_slice(cfg, lo, hi - lo, self.D, device=device)

    def evaluate(self, it: int) -> int:
        """Misfits of the slice's current positions, its personal bests, and
        its best key."""
        _, S = A.forward_batch(self.prob, self.sw.x, self.U, want_defl=False)
        A.pso_best_slice(self.cfg, self.lo, self.sw, S, it)
        return int(self.sw.gbest.item())

    def owns(self, g: int) -> bool:
        return self.lo <= g < self.hi

    def position(self, g: int):
        """Personal-best position [D] of swarm particle g (in this slice)."""
        return self.sw.pbest_x[:, g - self.lo].contiguous()

    def move(self, pos, it: int) -> None:
        A.pso_move_slice(self.cfg, self.lo, self.sw, pos, it)


def invert_split(prob, U, cfg, rank: int, world: int, group=None) -> dict:
    """The inversion of afm_invert with the swarm split over `world`
    processes (torch.distributed initialised; NCCL with one GPU per rank,
    or gloo with CPU staging of the exchange).  Every rank returns the same
    winner: normalised x [D] (float32), FP32 misfit S, swarm index, the
    global-best key after each generation, and its FP64 re-evaluation."""
    import struct

    import torch
    import torch.distributed as dist
    lo, hi = slice_of(cfg.P, rank, world)
    sl = Slice(prob, U, cfg, lo, hi, device=U.device.index)
    xdev = torch.device("cpu") if dist.get_backend(group) == "gloo" else U.device

    def owner(kmin):
        g = key_index(kmin)
        return (True, sl.position(g).to(xdev)) if sl.owns(g) else (False, None)
    keys = []
    pos = None
    for it in range(cfg.iters + 1):
        key = sl.evaluate(it)
        kmin, pos = exchange_dist(key, owner, sl.D, xdev, group)
        pos = pos.to(U.device)
        keys.append(kmin)
        if it < cfg.iters:
            sl.move(pos, it)
    S32 = struct.unpack("<f", struct.pack("<I", keys[-1] >> 32))[0]
    _, S64 = A.forward_batch_f64(prob, pos.double().reshape(-1, 1), U.double(), want_defl=False)
    return {"x": pos.cpu().numpy(), "S": S32, "winner": key_index(keys[-1]), "keys": keys,
            "S_f64": float(S64.item()), "slice": (lo, hi)}
