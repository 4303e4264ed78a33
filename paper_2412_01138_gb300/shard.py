"""Mode-sharded Parareal solve: one libpe context per rank, each owning a block of modes.

After the diagonalisation of Sec. 2.3 every mode obeys its own scalar ODE, and in
Algorithm 1 only the stopping rule couples the modes: the relative residual
r = sqrt(sum_n ||U^n_new - U^n_old||_0^2) / sqrt(sum_n ||U^n_new||_0^2) sums over all of
them.  So a solve splits across ranks as contiguous blocks of the slowest axis' mode
index (``pe_options.mode_begin`` / ``mode_end``); each rank runs the tables, the coarse
sweep, the fine sweeps and the corrections of its own modes, and per iteration the ranks
exchange two float64 numbers (an all-reduce of the two residual sums).  The nodal output
is the sum over ranks of each rank's nodal field of its own modes (an all-reduce of the
whole grid's values), since the inverse transform is linear.

This module holds the host side of that scheme: the partition, the combination of the
sums and of the nodal fields (through ``torch.distributed`` when a process group is
given, as plain sums otherwise), and a driver of one rank's solve through the C-ABI.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np


def shard_ranges(n0: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous blocks [begin, end) of the axis-0 mode indices 0..n0-1, one per rank, sizes
    differing by at most one (the first n0 % world ranks take one more)."""
    if world < 1 or n0 < world:
        raise ValueError(f"cannot split {n0} axis-0 modes over {world} ranks")
    base, extra = divmod(n0, world)
    out, b = [], 0
    for r in range(world):
        e = b + base + (1 if r < extra else 0)
        out.append((b, e))
        b = e
    return out


def allreduce_sum(values, dist=None, device="cpu") -> np.ndarray:
    """Element-wise sum of `values` over the ranks of the default process group (the values
    themselves without one).  Float64 throughout."""
    arr = np.asarray(values, dtype=np.float64)
    if dist is None:
        return arr.copy()
    import torch

    t = torch.as_tensor(arr, dtype=torch.float64, device=device).contiguous()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()


def relative_residual(total_sums: Sequence[float]) -> float:
    """The stopping rule's r from the totals (sum mu dU^2, sum mu U^2), as the library computes it."""
    num, den = float(total_sums[0]), float(total_sums[1])
    return float(np.sqrt(num) / np.sqrt(den)) if den > 0.0 else float(np.sqrt(num))


class ShardedSolver:
    """One rank's part of a mode-sharded solve (rank r of world owns shard_ranges(n0, world)[r]).

    ``solve`` runs Algorithm 1 on the rank's modes, combining the residual sums of every rank
    after each iteration, and stops when the combined residual reaches tol (or k = N, or
    max_iter); ``solution`` returns the whole grid's nodal solution (combined over ranks).
    """

    def __init__(self, prob, rank: int, world: int, dist=None, device="cpu", **solver_kw):
        from . import pe

        self.prob, self.rank, self.world, self.dist, self.device = prob, rank, world, dist, device
        self.range = shard_ranges(prob.n[0], world)[rank]
        self.solver = pe.Solver(prob, mode_range=self.range, **solver_kw)
        self.k = 0

    def close(self):
        self.solver.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, tol: float, nodal_u0=None, max_iter: Optional[int] = None) -> dict:
        from . import pe

        if nodal_u0 is None:
            self.solver.set_problem()
        else:
            self.solver.set_problem(pe.PE_FIELD_NODAL, nodal=nodal_u0)
        cap = self.prob.N if max_iter is None else min(max_iter, self.prob.N)
        history = []
        r = float("inf")
        self.k = 0
        while self.k < cap:
            sums = self.solver.iterate_sums()
            r = relative_residual(allreduce_sum(sums, self.dist, self.device))
            self.k += 1
            history.append(r)
            if r <= tol:
                break
        return {"k": self.k, "residual": r, "history": history}

    def modal(self, slice_: int):
        """This rank's modes of U^slice (a contiguous block of the C-ordered modal array)."""
        return self.solver.modal(slice_)

    def solution(self, slice_: Optional[int] = None):
        """Whole-grid nodal values at T_slice (default: the final time), combined over ranks."""
        part = self.solver.solution(self.prob.N if slice_ is None else slice_)
        return allreduce_sum(part, self.dist, self.device)
