"""Multi-GPU sharding.  Packages are independent (paper Sect. 1 and 4.2), so
each rank traces its own range of package ids of every item, and one
all-reduce (integer sum) of the int64 counters gives every rank the counters
of all packages -- bit-identical to one device tracing them all, because
fixed-point sums do not depend on their order.  The absorbed-power integral
and the temperature update then run redundantly on every rank, with no
broadcast.

Two uses:

* ``shard_items``: a batch of items, n packages per rank per item (weak
  scaling; the bench's tracer pass).
* ``iterate_sharded``: the whole iteration (iteration 0 with the constant
  sources, then frozen-seed dust iterations to max |dT| < tol) with each
  item's package ids split across the ranks and one counter all-reduce per
  tracer launch.  It drives a backend with five operations (trace, package
  energy, absorbed power, temperature update, dust emission weights);
  ``LibraryBackend`` is the library itself.
"""
from __future__ import annotations


def package_range(rank: int, world: int, n_per_rank: int):
    """(pid_offset, n_packages) of a rank when every rank traces n_per_rank."""
    if not (0 <= rank < world) or n_per_rank < 0:
        raise ValueError("bad rank / world / count")
    if (rank + 1) * n_per_rank > 2 ** 32:
        raise ValueError("package ids exceed 2^32")
    return rank * n_per_rank, n_per_rank


def split_range(n_total: int, rank: int, world: int):
    """(pid_offset, n_packages) of a rank's share of n_total package ids:
    [floor(r n / W), floor((r + 1) n / W)), so the ranks cover every id once."""
    if not (0 <= rank < world) or n_total < 0:
        raise ValueError("bad rank / world / count")
    if n_total > 2 ** 32:
        raise ValueError("package ids exceed 2^32")
    lo = rank * n_total // world
    hi = (rank + 1) * n_total // world
    return lo, hi - lo


def shard_items(specs, rank: int, world: int):
    """Rank's share of batch items given for one device (n_packages per rank)."""
    out = []
    for s in specs:
        off, n = package_range(rank, world, s["n_packages"])
        t = dict(s)
        t["pid_offset"] = s.get("pid_offset", 0) + off
        t["n_packages"] = n
        out.append(t)
    return out


def allreduce_counters(tally, group=None):
    """Integer-sum all-reduce of an int64 counter tensor (in place)."""
    import torch
    import torch.distributed as dist
    if tally.dtype != torch.int64:
        raise TypeError("counters must be int64")
    dist.all_reduce(tally, op=dist.ReduceOp.SUM, group=group)
    return tally


class LibraryBackend:
    """The library (one context, one cloud) as the backend of
    iterate_sharded: counters, A and T are device tensors."""

    def __init__(self, ctx, cloud_id: int, n_cells: int, n_leaf: int, n_freq: int):
        import torch
        self.ctx, self.cid = ctx, cloud_id
        self.n_cells, self.n_leaf, self.n_freq = n_cells, n_leaf, n_freq
        self.torch = torch
        self.dT = torch.zeros(1, dtype=torch.float64, device="cuda")

    def zeros(self, n, dtype):
        t = self.torch
        return t.zeros(n, dtype={"i8": t.int64, "f8": t.float64, "f4": t.float32}[dtype], device="cuda")

    def trace(self, specs, tally):
        """Adds the items' deposits to tally; returns their photon-cell steps."""
        stats = self.torch.zeros((len(specs), 4), dtype=self.torch.int64, device="cuda")
        self.ctx.simulate(self.ctx.items([dict(s, cloud=self.cid) for s in specs]), tally, stats)
        return int(stats[:, 2].sum().item())

    def package_energy(self, source, n_total):
        return self.torch.from_numpy(self.ctx.package_energy(self.cid, source, n_total)).cuda()

    def absorbed_power(self, tally, e_unit, A_in, A_out):
        self.ctx.absorbed_power(self.cid, tally, self.n_cells, e_unit, A_out, A_in=A_in)

    def temperature(self, A, T):
        """T <- T(A) in place; returns max |T - T_prev| over leaves."""
        self.ctx.update_temperature(self.cid, A, T, self.dT)
        return float(self.dT.item())

    def dust_emission(self, T, n_per_cell):
        """(weights [n_freq][n_leaf], energy of one unit per frequency)."""
        w = self.torch.empty((self.n_freq, self.n_leaf), dtype=self.torch.int64, device="cuda")
        e = self.torch.empty(self.n_freq, dtype=self.torch.float64, device="cuda")
        self.ctx.dust_emission(self.cid, T, w, e, n_per_cell=n_per_cell)
        return w, e

    def copy(self, dst, src):
        dst.copy_(src)


def iterate_sharded(backend, T, *, rank=0, world=1, n_background=0, n_point=0, n_per_cell=1, max_iter=0,
                    dT_tol=0.1, T_seed=None, allreduce=None):
    """The iteration of soc_iterate (paper Sect. 2.1.2 / 3.3), sharded: every
    item's package ids are split across the `world` ranks (split_range), the
    counters of each tracer launch are summed over the ranks (`allreduce`,
    default allreduce_counters; not called when world == 1), and every rank
    then computes A and T itself.  T (the backend's temperature array) is
    updated in place.  With the same total package counts the result equals
    one rank tracing everything, bit for bit.  Returns iterations, converged,
    the max |dT| history and the steps of this rank's packages."""
    reduce = (lambda t: t) if world == 1 else (allreduce or allreduce_counters)
    nf, n = backend.n_freq, backend.n_cells
    steps = 0
    A_const = backend.zeros(n, "f8")
    for source, n_total in ((0, n_background), (1, n_point)):
        if not n_total:
            continue
        off, cnt = split_range(n_total, rank, world)
        tally = backend.zeros(nf * n, "i8")
        specs = [dict(source=source, freq=f, pid_offset=off, n_packages=cnt, tally_offset=f * n) for f in range(nf)]
        if cnt:
            steps += backend.trace(specs, tally)
        reduce(tally)
        backend.absorbed_power(tally, backend.package_energy(source, n_total), A_const, A_const)
    if T_seed is not None:
        backend.copy(T, T_seed)
    else:
        backend.temperature(A_const, T)
    A = backend.zeros(n, "f8")
    hist, conv = [], False
    n_dust = backend.n_leaf * n_per_cell
    for _ in range(max_iter):
        w, e = backend.dust_emission(T, n_per_cell)
        off, cnt = split_range(n_dust, rank, world)
        tally = backend.zeros(nf * n, "i8")
        # frozen dust random numbers: iteration key 1 in every dust iteration
        specs = [dict(source=2, freq=f, iteration=1, pid_offset=off, n_packages=cnt, tally_offset=f * n,
                      dust_w=w[f], n_per_cell=n_per_cell) for f in range(nf)]
        if cnt:
            steps += backend.trace(specs, tally)
        reduce(tally)
        backend.absorbed_power(tally, e, A_const, A)
        hist.append(backend.temperature(A, T))
        if hist[-1] < dT_tol:
            conv = True
            break
    return dict(iterations=len(hist), converged=conv, history=hist, steps=steps)
