"""One population sharded over ranks (paper_1711_02242_gb300.dist) on the
CPU: gloo, world size 2, each rank's shard stepped by the oracle.  The
sharded comb (weights gathered, the same parents on every rank, rows moved
point to point) must give exactly what one comb over the concatenated
population gives: the same parents, walkers, overlaps, weights and energies
bit for bit (Sec. 3.4.4 with the walkers independent between combs,
Sec. 3.5)."""
import dataclasses
import os
import socket

import numpy as np
import pytest

import workloads
from oracle import afqmc, philox, scf

N_LOCAL, WORLD, STEPS = 8, 2, 30
PARAMS = dict(dt=0.005, seed=7, qr_period=5, pc_period=5, energy_period=2)


def _system():
    w = workloads.config("c0")
    h1, L, _ = w.hamiltonian()
    C, _, _, _ = scf.rhf(h1, L, w.N)
    return h1, L, C


class OracleShard:
    """A shard of the population stepped by the oracle (test double of
    dist.StateShard)."""

    def __init__(self, h1, L, C, n, rank):
        import torch

        self.torch = torch
        p = afqmc.Params(**dict(PARAMS, pc_period=0, energy_period=0, walker0=rank * n))
        self.o = afqmc.Oracle(h1, L, C, n, p)
        self.n = n
        self.nm = self.o.phi[0].size
        self.row = 4 * self.nm + 2

    def propagate(self, k):
        self.o.run(k)

    def weights(self):
        return self.torch.tensor(np.array(self.o.weight, np.float64))

    def comb_parents(self, w_all):
        u = philox.comb_uniform(self.o.p.seed, self.o.step_count - 1)
        parent, self.wnew = afqmc.comb(w_all.numpy(), u)
        return np.full(w_all.numel(), -1) if parent is None else parent

    def empty_rows(self, k):
        return self.torch.empty((k, self.row), dtype=self.torch.float64)

    def pack(self, idx):
        o = self.o
        rows = np.concatenate([o.phi[idx].reshape(len(idx), -1).view(np.float64),
                               o.theta[idx].reshape(len(idx), -1).view(np.float64),
                               np.stack([o.logdet[idx].real, o.logdet[idx].imag], 1)], 1)
        return self.torch.tensor(rows)

    def unpack(self, slots, rows):
        o, nm = self.o, self.nm
        r = rows.numpy()
        o.phi[slots] = r[:, :2 * nm].copy().view(np.complex128).reshape(o.phi[slots].shape)
        o.theta[slots] = r[:, 2 * nm:4 * nm].copy().view(np.complex128).reshape(o.theta[slots].shape)
        o.logdet[slots] = r[:, 4 * nm] + 1j * r[:, 4 * nm + 1]
        o.weight[slots] = self.wnew

    def energy_sums(self):
        num, den = self.o.energy_sums()
        return self.torch.tensor([num, den, 0.0, 0.0], dtype=self.torch.float64)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, port, out):
    import torch.distributed as dist

    from paper_1711_02242_gb300.dist import ShardedPopulation

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    h1, L, C = _system()
    pop = ShardedPopulation(OracleShard(h1, L, C, N_LOCAL, rank), pc_period=PARAMS["pc_period"],
                            energy_period=PARAMS["energy_period"]).run(STEPS)
    o = pop.shard.o
    out.put((rank, o.phi, o.theta, o.logdet, o.weight, pop.records,
             [(s, np.asarray(p)) for s, p in pop.parents]))
    dist.barrier()
    dist.destroy_process_group()


def _central():
    """The same population combed centrally: both shards stepped in one
    process, the comb over the concatenated weights and walkers."""
    h1, L, C = _system()
    shards = [OracleShard(h1, L, C, N_LOCAL, r).o for r in range(WORLD)]
    records, parents = [], []
    for n in range(1, STEPS + 1):
        for o in shards:
            o.step()
        if n % PARAMS["pc_period"] == 0:
            w = np.concatenate([o.weight for o in shards])
            parent, wnew = afqmc.comb(w, philox.comb_uniform(PARAMS["seed"], n - 1))
            parents.append((n, parent))
            cat = {k: np.concatenate([getattr(o, k) for o in shards])[parent]
                   for k in ("phi", "theta", "logdet")}
            for r, o in enumerate(shards):
                sl = slice(r * N_LOCAL, (r + 1) * N_LOCAL)
                for k, v in cat.items():
                    setattr(o, k, v[sl].copy())
                o.weight = np.full(N_LOCAL, wnew)
        if n % PARAMS["energy_period"] == 0:
            s = [o.energy_sums() for o in shards]
            num, den = s[0][0] + s[1][0], s[0][1] + s[1][1]
            records.append((n, num / den, den))
    return shards, records, parents


def test_transfer_plan_routes_every_slot():
    from paper_1711_02242_gb300.dist import transfer_plan

    n, world = 4, 3
    parent = np.array([0, 0, 5, 5, 5, 6, 9, 11, 11, 11, 2, 3])
    for rank in range(world):
        send, recv = transfer_plan(parent, n, rank, world)
        assert sum(v.size for v in recv.values()) == n
        for q in range(world):
            slots_q = parent[q * n:(q + 1) * n]
            expect_send = [p - rank * n for p in slots_q if rank * n <= p < (rank + 1) * n]
            assert list(send[q]) == expect_send
            assert list(recv[q]) == [k for k in range(n) if parent[rank * n + k] // n == q]
    # rank 1's slots hold parents 5, 6 (its own walkers 1, 2), 9 and 11 (rank
    # 2's walkers 1 and 3); rank 0's slots 2 and 3 take rank 1's walker 1
    send, recv = transfer_plan(parent, n, 1, world)
    assert list(send[1]) == [1, 2] and list(recv[1]) == [0, 1] and list(recv[2]) == [2, 3]
    assert list(send[0]) == [1, 1] and send[2].size == 0


def test_sharded_comb_equals_one_comb_over_the_whole_population():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(WORLD)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards, records, parents = _central()
    assert len(parents) == STEPS // PARAMS["pc_period"]
    for r, (rank, phi, theta, logdet, weight, recs, pars) in enumerate(res):
        o = shards[r]
        assert np.array_equal(phi, o.phi) and np.array_equal(theta, o.theta)
        assert np.array_equal(logdet, o.logdet) and np.array_equal(weight, o.weight)
        assert recs == records
        assert len(pars) == len(parents)
        for (s1, p1), (s2, p2) in zip(pars, parents):
            assert s1 == s2 and np.array_equal(p1, p2)
    # the combs moved walkers between the shards
    assert any(np.any(p[:N_LOCAL] >= N_LOCAL) or np.any(p[N_LOCAL:] < N_LOCAL)
               for _, p in parents)


def test_shards_draw_the_fields_of_their_global_walkers():
    """Without combs, the two shards' walks are the walkers [0, n) and
    [n, 2n) of one 2n-walker run (fields keyed by global walker index)."""
    h1, L, C = _system()
    p = afqmc.Params(**dict(PARAMS, pc_period=0, energy_period=0))
    whole = afqmc.Oracle(h1, L, C, WORLD * N_LOCAL, p).run(6)
    for r in range(WORLD):
        part = afqmc.Oracle(h1, L, C, N_LOCAL, dataclasses.replace(p, walker0=r * N_LOCAL)).run(6)
        sl = slice(r * N_LOCAL, (r + 1) * N_LOCAL)
        assert np.max(np.abs(part.phi - whole.phi[sl])) < 1e-12
        assert np.max(np.abs(part.weight - whole.weight[sl]) / np.abs(whole.weight[sl])) < 1e-12
