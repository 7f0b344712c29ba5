"""Slice-range ledger: distribution, checkpoint/resume and recovery of lost
slices for one amplitude.

The paper's scheme (Sec. III.A) runs the 2^k subnetworks on independent
workers that each return one scalar per subgraph to a master; Sec. V notes
that when workers are lost only their missing subgraphs need recomputing.
Here the 2^k slices are split into fixed contiguous ranges; every range's
compensated partial sum (sum, compensation) is recorded once computed, can
be written to and reloaded from a JSON checkpoint, and the final amplitude
is the fixed-order (ascending range) compensated sum of the recorded
partials -- independent of which worker computed what, or when.

`sharded_amplitude` is the data path of one amplitude over several ranks
(Sec. III.A, Sec. IV.B: only one scalar per subgraph goes back): rank g
contracts the contiguous slice range [g S / G, (g+1) S / G) and the ranks'
(sum, compensation) pairs meet in one all-gather (gloo on the CPU, NCCL on
GPUs), summed in ascending g order on every rank.

`run_ranks` distributes ranges round-robin over the ranks of a
torch.distributed process group.  Workers publish each finished range in the
group's key-value store; rank 0 waits for them with a deadline and then
recomputes, itself, every range that no worker delivered (a worker that
raised, exited or never joined).  No GPU is involved in detecting a failure.
"""
from __future__ import annotations

import json
import os
import time
from typing import Callable, Dict, List, Optional, Tuple

Range = Tuple[int, int]
# compute(lo, hi) -> (sum, compensation) as complex numbers, unscaled
ComputeFn = Callable[[int, int], Tuple[complex, complex]]


def _kahan(sum_re, comp_re, v):
    y = v - comp_re
    t = sum_re + y
    return t, (t - sum_re) - y


class SliceLedger:
    def __init__(self, n_slices: int, chunk: int, path: Optional[str] = None):
        if n_slices < 0 or chunk <= 0:
            raise ValueError("n_slices >= 0 and chunk > 0 required")
        self.n_slices = int(n_slices)
        self.chunk = int(chunk)
        self.path = path
        self.ranges: List[Range] = [(lo, min(lo + chunk, n_slices)) for lo in range(0, n_slices, chunk)]
        self.done: Dict[Range, Tuple[complex, complex]] = {}
        if path and os.path.exists(path):
            self.load()

    def pending(self) -> List[Range]:
        return [r for r in self.ranges if r not in self.done]

    def record(self, r: Range, total: complex, comp: complex, save: bool = True):
        r = (int(r[0]), int(r[1]))
        if r not in self.ranges:
            raise ValueError(f"{r} is not a range of this ledger")
        self.done[r] = (complex(total), complex(comp))
        if save and self.path:
            self.save()

    def complete(self) -> bool:
        return len(self.done) == len(self.ranges)

    def total(self) -> complex:
        """Compensated sum of every range's partial, in ascending range order."""
        if not self.complete():
            raise RuntimeError(f"{len(self.pending())} ranges are missing")
        sr = cr = si = ci = 0.0
        for r in self.ranges:
            s, c = self.done[r]
            for v_re, v_im in ((s.real, s.imag), (-c.real, -c.imag)):
                sr, cr = _kahan(sr, cr, v_re)
                si, ci = _kahan(si, ci, v_im)
        return complex(sr - cr, si - ci)

    def to_json(self) -> dict:
        return {"n_slices": self.n_slices, "chunk": self.chunk,
                "done": [[lo, hi, s.real, s.imag, c.real, c.imag] for (lo, hi), (s, c) in sorted(self.done.items())]}

    def save(self):
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.to_json(), f)
        os.replace(tmp, self.path)

    def load(self):
        with open(self.path) as f:
            d = json.load(f)
        if d["n_slices"] != self.n_slices or d["chunk"] != self.chunk:
            raise ValueError("checkpoint belongs to a different slicing")
        for lo, hi, sr, si, cr, ci in d["done"]:
            self.done[(lo, hi)] = (complex(sr, si), complex(cr, ci))


def run_local(ledger: SliceLedger, compute: ComputeFn) -> complex:
    """Computes every pending range (resuming a checkpoint) and sums."""
    for r in ledger.pending():
        s, c = compute(*r)
        ledger.record(r, s, c)
    return ledger.total()


def _key(r: Range) -> str:
    return f"qtn_range_{r[0]}_{r[1]}"


def run_ranks(ledger: SliceLedger, compute: ComputeFn, rank: int, world: int, store,
              deadline_s: float = 30.0, poll_s: float = 0.05) -> Optional[complex]:
    """Round-robin ranges over `world` ranks; rank 0 gathers from `store`
    (a torch.distributed Store), recomputes what is missing after
    `deadline_s`, and returns the amplitude sum (other ranks return None).
    Returns also on rank 0 the list of ranges it had to recompute, in
    `ledger.recomputed`."""
    mine = [r for i, r in enumerate(ledger.ranges) if i % world == rank]
    for r in mine:
        if r in ledger.done:
            s, c = ledger.done[r]
        else:
            s, c = compute(*r)
        store.set(_key(r), json.dumps([s.real, s.imag, c.real, c.imag]))
        if rank == 0:
            ledger.record(r, s, c, save=False)
    if rank != 0:
        return None
    t_end = time.monotonic() + deadline_s
    waiting = set(ledger.pending())
    while waiting and time.monotonic() < t_end:
        for r in list(waiting):
            if store.check([_key(r)]):
                sr, si, cr, ci = json.loads(store.get(_key(r)))
                ledger.record(r, complex(sr, si), complex(cr, ci), save=False)
                waiting.discard(r)
        if waiting:
            time.sleep(poll_s)
    ledger.recomputed = sorted(waiting)
    for r in ledger.recomputed:  # Sec. V: recompute only the lost subgraphs
        s, c = compute(*r)
        ledger.record(r, s, c, save=False)
    if ledger.path:
        ledger.save()
    return ledger.total()


def shard_range(n_slices: int, rank: int, world: int) -> Range:
    """Contiguous slice range of rank `rank` of `world`: [g S / G, (g+1) S / G)."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("0 <= rank < world required")
    return (n_slices * rank // world, n_slices * (rank + 1) // world)


class ShardsLost(RuntimeError):
    pass


def sharded_amplitude(compute: ComputeFn, n_slices: int, rank: int, world: int, dist, device="cpu",
                      recover: bool = True):
    """One amplitude contracted by `world` ranks: this rank computes its
    contiguous range (compute(lo, hi) -> (sum, comp)), one all_gather of the
    four doubles (sum.re, sum.im, comp.re, comp.im) per rank, and every rank
    adds the pairs in ascending rank order (compensated, so the result does
    not depend on the schedule).  Returns (total, recomputed ranges).

    If the collective fails (a rank died or never joined; the process
    group's timeout bounds the wait), the surviving rank recomputes every
    other rank's range itself when `recover` is set (Sec. V: only the lost
    subgraphs), else raises ShardsLost."""
    import torch

    mine = shard_range(n_slices, rank, world)
    s, c = compute(*mine)
    local = torch.tensor([s.real, s.imag, c.real, c.imag], dtype=torch.float64, device=device)
    parts = [torch.zeros(4, dtype=torch.float64, device=device) for _ in range(world)]
    recomputed: List[Range] = []
    try:
        dist.all_gather(parts, local)
        got = [p.cpu().tolist() for p in parts]
    except Exception as e:  # a lost rank: the collective ended with an error
        if not recover:
            raise ShardsLost(str(e)) from e
        got = []
        for g in range(world):
            if g == rank:
                got.append([s.real, s.imag, c.real, c.imag])
            else:
                r = shard_range(n_slices, g, world)
                recomputed.append(r)
                sg, cg = compute(*r)
                got.append([sg.real, sg.imag, cg.real, cg.imag])
    led = SliceLedger(n_slices, max(1, n_slices))
    led.ranges = [shard_range(n_slices, g, world) for g in range(world)]
    for g, (sr, si, cr, ci) in enumerate(got):
        led.record(led.ranges[g], complex(sr, si), complex(cr, ci), save=False)
    return led.total(), recomputed
