"""Sharded states with qubit-swap exchange, on the host (no GPU).

The library plans the exchange schedule (shard_plan); these tests replay it: every
non-diagonal gate must find its qubits local, segments must cover the circuit in order,
and two gloo ranks that each hold one shard (one global qubit), exchanging half a shard
by point-to-point messages exactly as the schedule's swaps prescribe (shard with global
bit 0 gives its amplitudes with local bit l = 1, its partner those with l = 0, at equal
other bits), must reproduce the oracle's state.  Local gates are applied with the
oracle's dense gather/scatter on each rank's shard; diagonal gates on the global qubit
become the rank's phase or a diagonal on the local partner.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import paper_2406_19212_gb300 as gb
from oracle import oracle as O
from paper_2406_19212_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def is_diagonal(op):
    if op.name == "RZ":
        return True
    if op.param >= 0:
        return False
    M = O.gate_matrix(op)
    return np.count_nonzero(M - np.diag(np.diag(M))) == 0


def replay(steps, ops, n, g):
    """Positions after the schedule; asserts locality of every non-diagonal gate and
    that the segments cover the ops in order."""
    L = n - g
    pos = list(range(n))
    covered = 0
    for kind, a, b in steps:
        if kind == "swap":
            assert 0 <= a < g and 0 <= b < L
            x = pos.index(L + a)
            y = pos.index(b)
            pos[x], pos[y] = pos[y], pos[x]
            continue
        assert a == covered and b > a
        for op in ops[a:b]:
            if not is_diagonal(op):
                assert all(pos[q] < L for q in op.qubits), (op, pos)
        covered = b
    assert covered == len(ops)
    return pos


@pytest.mark.parametrize("n,g,seed", [(6, 1, 0), (8, 2, 1), (9, 3, 2), (12, 4, 3)])
def test_schedule_is_valid(n, g, seed):
    gb.load()
    w = I.random_circuit(n, 150, seed)
    c = gb.circuit_create(w.circuit)
    steps = gb.shard_plan(c, g)
    replay(steps, w.circuit.ops, n, g)
    needing = sum(1 for op in w.circuit.ops
                  if not is_diagonal(op) and any(q >= n - g for q in op.qubits))
    assert sum(1 for s in steps if s[0] == "swap") >= (1 if needing else 0)


def test_local_and_diagonal_global_gates_need_no_exchange():
    gb.load()
    n = 8
    ops = [I.Op("H", (q,)) for q in range(6)] + [I.Op("RZ", (7,), param=0), I.Op("CZ", (3, 7)),
                                                   I.Op("CZ", (6, 7)), I.Op("CNOT", (0, 5))]
    c = gb.circuit_create(I.Circuit(n, ops, 1))
    assert gb.shard_plan(c, 2) == [("ops", 0, len(ops))]


def test_furthest_next_use_victim():
    """With one global qubit (7) needed by a gate, the local qubit given up is the one
    whose next non-diagonal use is farthest away (never used again: qubit 6)."""
    gb.load()
    n = 8
    ops = [I.Op("H", (q,)) for q in range(7)] + [I.Op("H", (7,))] + [I.Op("H", (q,)) for q in range(6)]
    c = gb.circuit_create(I.Circuit(n, ops, 0))
    steps = gb.shard_plan(c, 1)
    assert ("swap", 0, 6) in steps and sum(1 for s in steps if s[0] == "swap") == 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _half_indices(L, l, bit):
    i = np.arange(1 << (L - 1), dtype=np.int64)
    low = (1 << l) - 1
    x0 = ((i & ~low) << 1) | (i & low)
    return x0 | (bit << l)


def _rank_main(rank, port, n, seed, out):
    import torch
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        g, L = 1, n - 1
        w = I.random_circuit(n, 120, seed)
        c = gb.circuit_create(w.circuit)
        steps = gb.shard_plan(c, g)
        psi = np.zeros(1 << L, complex)
        if rank == 0:
            psi[0] = 1.0
        pos = list(range(n))
        for kind, a, b in steps:
            if kind == "swap":
                l = b
                send = psi[_half_indices(L, l, 1 - rank)].copy()   # rank 0: bit l = 1; rank 1: bit l = 0
                recv = np.empty_like(send)
                st, rt = torch.from_numpy(send.view(np.float64)), torch.from_numpy(recv.view(np.float64))
                if rank == 0:
                    dist.send(st, 1)
                    dist.recv(rt, 1)
                else:
                    dist.recv(rt, 0)
                    dist.send(st, 0)
                psi[_half_indices(L, l, 1 - rank)] = recv
                x, y = pos.index(L + a), pos.index(l)
                pos[x], pos[y] = pos[y], pos[x]
                continue
            for op in w.circuit.ops[a:b]:
                M = O.gate_matrix(op, w.theta)
                q = [pos[x] for x in op.qubits]
                if all(p < L for p in q):
                    psi = O.apply_matrix(psi, L, q, M)
                    continue
                d = np.diag(M)   # a diagonal gate touching the global qubit (this rank's bit)
                if len(q) == 1:
                    psi = psi * d[rank]
                elif q[0] >= L and q[1] >= L:
                    psi = psi * d[rank + 2 * rank]
                elif q[0] >= L:
                    psi = O.apply_matrix(psi, L, [q[1]], np.diag([d[rank], d[rank + 2]]))
                else:
                    psi = O.apply_matrix(psi, L, [q[0]], np.diag([d[2 * rank], d[1 + 2 * rank]]))
        # gather both shards on rank 0 and read them through the final positions
        buf = torch.from_numpy(psi.view(np.float64).copy())
        if rank == 1:
            dist.send(buf, 0)
            out.put((rank, None))
        else:
            other = torch.empty_like(buf)
            dist.recv(other, 1)
            full = np.concatenate([psi, other.numpy().view(complex)])
            dim = 1 << n
            logical = np.empty(dim, complex)
            for x in range(dim):
                phys = sum(1 << pos[qq] for qq in range(n) if (x >> qq) & 1)
                logical[x] = full[phys]
            ref = O.apply_circuit(w.circuit, w.theta)
            out.put((rank, float(np.abs(logical - ref).max())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n,seed", [(7, 5), (9, 6)])
def test_two_gloo_ranks_execute_the_schedule(n, seed):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, n, seed, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] is not None and res[0] < 1e-12
