"""One design problem sharded over the ranks of a process group, by wavelength and source.

Sec. II: the symbolic factorisation depends only on the grid and the design box, so every
wavelength (and every source of a wavelength) shares it, while each wavelength's matrix is
factorised and solved on its own.  The objective F and the design gradient dF/deps are sums
over (wavelength, source) pairs.  So the pairs split into independent shards: each rank
builds its own solver context(s) for its pairs (the symbolic plan, a function of the grid
and design box only, comes out the same on every rank), runs the whole design iteration on
them, and one all-reduce (sum) of [dF/deps, F] completes the iteration on every rank.  That
all-reduce is the path's only exchange.

Pairs are numbered wavelength-major (u = w * n_src + s) and cut into contiguous, balanced
blocks, one per rank; a rank whose block is empty contributes zeros.  A rank's pairs are
grouped into contexts: consecutive wavelengths with the same sources share one context, so
that a block of whole wavelengths is one batched multi-wavelength context.
"""
from __future__ import annotations

from typing import Callable, Sequence

import torch


def shard_pairs(n_omega: int, n_src: int, world: int, rank: int) -> list[tuple[int, list[int]]]:
    """The (wavelength, [sources]) pairs of one rank, in wavelength order."""
    if not (0 <= rank < world) or n_omega < 1 or n_src < 1:
        raise ValueError("need 0 <= rank < world, n_omega >= 1, n_src >= 1")
    total = n_omega * n_src
    lo, hi = rank * total // world, (rank + 1) * total // world
    out: list[tuple[int, list[int]]] = []
    for u in range(lo, hi):
        w, s = divmod(u, n_src)
        if out and out[-1][0] == w:
            out[-1][1].append(s)
        else:
            out.append((w, [s]))
    return out


def context_groups(pairs: Sequence[tuple[int, list[int]]]) -> list[tuple[list[int], list[int]]]:
    """Consecutive wavelengths with identical source lists merged: [(wavelengths, sources)]."""
    groups: list[tuple[list[int], list[int]]] = []
    for w, srcs in pairs:
        if groups and groups[-1][1] == srcs and groups[-1][0][-1] == w - 1:
            groups[-1][0].append(w)
        else:
            groups.append(([w], list(srcs)))
    return groups


class ShardedProblem:
    """The rank's share of a design problem plus the all-reduce that completes each iteration.

    make_problem(wavelengths, sources) must return an object with iteration(eps_design) ->
    (F, dF/deps [w*h]) over exactly those wavelengths and sources (an autograd.DesignProblem on
    a solver built for them).  group: a torch.distributed process group, or None for a single
    process (no all-reduce)."""

    def __init__(self, make_problem: Callable, n_omega: int, n_src: int, n_design: int,
                 device, group=None):
        import torch.distributed as dist
        self.group = group
        self.dist = dist if (group is not None or (dist.is_available() and dist.is_initialized())) else None
        world = self.dist.get_world_size(group) if self.dist else 1
        rank = self.dist.get_rank(group) if self.dist else 0
        self.pairs = shard_pairs(n_omega, n_src, world, rank)
        self.groups = context_groups(self.pairs)
        self.problems = [make_problem(ws, ss) for ws, ss in self.groups]
        self.n_design = n_design
        self.acc = torch.zeros(n_design + 1, dtype=torch.float64, device=device)

    @property
    def n_pairs(self) -> int:
        return sum(len(s) for _, s in self.pairs)

    def iteration(self, eps_design: torch.Tensor, grad_out: torch.Tensor | None = None):
        """One design iteration of the whole problem: (F, dF/deps), the same on every rank."""
        reduce = self.dist is not None and self.dist.get_world_size(self.group) > 1
        if len(self.problems) == 1 and not reduce:
            # a single context and no exchange: its gradient kernel writes the result in place
            return self.problems[0].iteration(eps_design, grad_out=grad_out)
        g = self.acc[:self.n_design]
        if not self.problems:
            self.acc.zero_()
        for k, p in enumerate(self.problems):
            # the gradient kernel sums the contexts' shares into the reduction buffer itself
            F, _ = p.iteration(eps_design, grad_out=g, accumulate=k > 0)
            if k == 0:
                self.acc[self.n_design:].copy_(F.reshape(1))
            else:
                self.acc[self.n_design] += F.reshape(())
        if reduce:
            self.dist.all_reduce(self.acc, op=self.dist.ReduceOp.SUM, group=self.group)
        if grad_out is not None:
            grad_out.copy_(g)
            g = grad_out
        return self.acc[self.n_design], g
