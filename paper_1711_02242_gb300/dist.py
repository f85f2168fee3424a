"""One phaseless-AFQMC population sharded over the ranks of a process group.

Walkers are independent between population controls (Sec. 3.5), so rank r
steps its own n walkers, the global walkers [r n, (r + 1) n) (their fields
keyed by the global index, params.walker0 = r n, one seed for all ranks).
Two steps need the whole population:

* the mixed estimator (Eq. localenergy): each rank's sums (sum W Re E_loc,
  sum W) are added over the ranks (all_reduce, 32 bytes);
* the comb (Sec. 3.4.4): every rank gathers all n_all weights (all_gather,
  8 bytes per walker), computes the same parents for the n_all new slots on
  its GPU (afqmc_comb_plan: the single-state comb's arithmetic over the global
  walker order), and the parents' rows (orbitals, Theta, log overlap) move
  point to point to the ranks owning the new slots.

The module only moves data and bookkeeps indices; the comb, packing and
unpacking run in the library's kernels through a `shard` object with the
methods of ``StateShard`` (the tests drive the same code with another shard
type on the CPU).  All shards hold the same number of walkers.
"""
from __future__ import annotations

import ctypes

import numpy as np


def transfer_plan(parent_all, n, rank, world):
    """Where the rows of the comb's parents go.

    parent_all[k] is the global parent of global slot k (slots of rank q are
    [q n, (q + 1) n)).  Returns (send, recv), dicts keyed by rank q:
      send[q]  indices of this rank's walkers whose rows rank q receives, in
               the order of q's slots;
      recv[q]  this rank's slots filled by those rows from rank q, in the
               same order.
    send[rank] / recv[rank] are the copies that stay on this rank."""
    parent_all = np.asarray(parent_all, np.int64)
    lo = rank * n
    send, recv = {}, {}
    for q in range(world):
        slots_q = parent_all[q * n:(q + 1) * n]
        mine = (slots_q >= lo) & (slots_q < lo + n)
        send[q] = (slots_q[mine] - lo).astype(np.int32)
    mine_slots = parent_all[lo:lo + n]
    src_rank = mine_slots // n
    for q in range(world):
        recv[q] = np.nonzero(src_rank == q)[0].astype(np.int32)
    return send, recv


class ShardedPopulation:
    """Steps a sharded population: every `pc_period` steps the global comb,
    every `energy_period` steps the global mixed estimator (after the comb,
    as a single state orders them)."""

    def __init__(self, shard, pc_period=0, energy_period=0, group=None):
        import torch.distributed as dist

        self.shard = shard
        self.pc_period = int(pc_period)
        self.energy_period = int(energy_period)
        self.group = group
        self.dist = dist
        if dist.is_available() and dist.is_initialized():
            self.world = dist.get_world_size(group)
            self.rank = dist.get_rank(group)
        else:
            self.world, self.rank = 1, 0
        self.step = 0
        self.records = []  # (step, E, sum W) of the whole population
        self.parents = []  # (step, global parents) of every comb

    def _next_stop(self):
        nxt = []
        for per in (self.pc_period, self.energy_period):
            if per > 0:
                nxt.append((self.step // per + 1) * per)
        return min(nxt) if nxt else None

    def run(self, nsteps):
        end = self.step + int(nsteps)
        while self.step < end:
            stop = self._next_stop()
            k = end - self.step if stop is None else min(stop, end) - self.step
            self.shard.propagate(k)
            self.step += k
            if self.pc_period and self.step % self.pc_period == 0:
                self.comb()
            if self.energy_period and self.step % self.energy_period == 0:
                self.records.append((self.step,) + self.energy())
        return self

    def _all_gather(self, t):
        if self.world == 1:
            return t
        parts = [t.new_empty(t.shape) for _ in range(self.world)]
        self.dist.all_gather(parts, t, group=self.group)
        return __import__("torch").cat(parts)

    def comb(self):
        """The comb over the whole population (Sec. 3.4.4)."""
        import torch

        sh = self.shard
        w_all = self._all_gather(sh.weights())
        parent_all = sh.comb_parents(w_all)  # host int array, global indices
        self.parents.append((self.step, parent_all))
        if parent_all.size == 0 or parent_all[0] < 0:
            return  # no weight left anywhere: nothing moves
        send, recv = transfer_plan(parent_all, sh.n, self.rank, self.world)
        # every outgoing row (the ones that stay here too) is packed before any
        # slot is overwritten
        out = {q: sh.pack(send[q]) for q in range(self.world) if send[q].size}
        inc = {}
        reqs = []
        for q in range(self.world):
            if q == self.rank:
                continue
            if send[q].size:
                reqs.append(self.dist.isend(out[q], q, group=self.group))
            if recv[q].size:
                inc[q] = sh.empty_rows(recv[q].size)
                reqs.append(self.dist.irecv(inc[q], q, group=self.group))
        for r in reqs:
            r.wait()
        if send[self.rank].size:
            inc[self.rank] = out[self.rank]
        slots = np.concatenate([recv[q] for q in sorted(inc)])
        rows = torch.cat([inc[q] for q in sorted(inc)])
        assert slots.size == sh.n
        sh.unpack(slots, rows)

    def energy(self):
        """(E, sum W) of the whole population: the ranks' estimator sums added."""
        s = self.shard.energy_sums()
        if self.world > 1:
            self.dist.all_reduce(s, group=self.group)
        s = s.cpu().numpy()
        return float(s[0] / s[1]) if s[1] != 0 else float("nan"), float(s[1])


class StateShard:
    """A library state as one shard (its own GPU and stream): the comb's plan,
    packing and unpacking and the estimator run in the library's kernels; the
    tensors this class hands to torch.distributed live on the state's device."""

    def __init__(self, run):
        import torch

        import paper_1711_02242_gb300 as pkg

        self.pkg, self.run = pkg, run
        self.lib = pkg.lib()
        self.n = run.p.nwalkers
        self.dev = run.device
        nb = ctypes.c_size_t(0)
        pkg._check(self.lib.afqmc_walker_row_bytes(run.s, ctypes.byref(nb)))
        self.row = nb.value // 8
        self.torch = torch

    def _sync(self):
        self.run.stream.synchronize()

    def propagate(self, k):
        self.run.propagate(k)

    def weights(self):
        w = self.torch.empty(self.n, dtype=self.torch.float64, device=self.dev)
        self.pkg._check(self.lib.afqmc_export_weights(self.run.s, ctypes.c_void_p(w.data_ptr())))
        self._sync()
        return w

    def comb_parents(self, w_all):
        t = self.torch
        n_all = w_all.numel()
        w_all = w_all.to(self.dev).contiguous()
        cum = t.empty(n_all, dtype=t.float64, device=self.dev)
        par = t.empty(n_all, dtype=t.int32, device=self.dev)
        self.pkg._check(self.lib.afqmc_comb_plan(self.run.s, ctypes.c_void_p(w_all.data_ptr()),
                                                 n_all, ctypes.c_void_p(cum.data_ptr()),
                                                 ctypes.c_void_p(par.data_ptr())))
        self._sync()
        self._keep = (w_all, cum, par)
        return par.cpu().numpy()

    def empty_rows(self, k):
        return self.torch.empty((k, self.row), dtype=self.torch.float64, device=self.dev)

    def pack(self, idx):
        t = self.torch
        d_idx = t.as_tensor(np.ascontiguousarray(idx, np.int32), device=self.dev)
        rows = self.empty_rows(idx.size)
        self.pkg._check(self.lib.afqmc_pack_walkers(self.run.s, ctypes.c_void_p(d_idx.data_ptr()),
                                                    int(idx.size),
                                                    ctypes.c_void_p(rows.data_ptr())))
        self._sync()
        return rows

    def unpack(self, slots, rows):
        t = self.torch
        d_slots = t.as_tensor(np.ascontiguousarray(slots, np.int32), device=self.dev)
        rows = rows.to(self.dev).contiguous()
        self.pkg._check(self.lib.afqmc_unpack_walkers(self.run.s,
                                                      ctypes.c_void_p(d_slots.data_ptr()),
                                                      int(slots.size),
                                                      ctypes.c_void_p(rows.data_ptr())))
        self._sync()

    def energy_sums(self):
        t = self.torch
        self.run.energy()  # evaluates the local energies and the state's sums
        s = t.empty(4, dtype=t.float64, device=self.dev)
        self.pkg._check(self.lib.afqmc_energy_sums(self.run.s, ctypes.c_void_p(s.data_ptr())))
        self._sync()
        return s
