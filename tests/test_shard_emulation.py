"""Host emulation, on gloo ranks, of the sharded execution a multi-GPU build
would use for one state: the state is split by its top g address bits over
2^g ranks, and

- a step whose target is a local bit runs on each rank's shard, its controls
  on global bits becoming a per-rank predicate (all-or-nothing per shard);
- a step whose target is a global bit pairs rank r with r ^ (1 << bit): the
  two ranks select the same local rows (local controls and polarity) and
  swap them, if the global controls hold for r (they hold for the partner
  too, since the ranks differ only in the target bit).

The shards, gathered, must equal the oracle's state bit for bit.  No GPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _sharded_apply(rank, world, M, shard, steps):
    """Apply steps to this rank's shard; returns (shard, rows sent)."""
    g = world.bit_length() - 1
    ml = M - g  # local address bits
    lmask = (1 << ml) - 1
    idx = np.arange(1 << ml, dtype=np.uint64)
    sent = 0
    for s in steps:
        t, cm, cp = int(s["target"]), int(s["ctrl_mask"]), int(s["ctrl_pol"])
        cg, pg = cm >> ml, cp >> ml  # controls on global bits
        if (rank & cg) != pg:
            continue  # the step does not fire anywhere in this shard
        cl, pl = cm & lmask, cp & lmask
        sel = (idx & np.uint64(cl)) == np.uint64(pl)
        if t < ml:  # local target: swap pairs inside the shard
            lo = sel & ((idx >> np.uint64(t)) & np.uint64(1) == 0)
            a = idx[lo]
            b = a | np.uint64(1 << t)
            tmp = shard[a].copy()
            shard[a] = shard[b]
            shard[b] = tmp
        else:  # global target: swap the selected rows with the partner rank
            partner = rank ^ (1 << (t - ml))
            rows = idx[sel]
            out = torch.from_numpy(shard[rows].view(np.float64).copy())
            inc = torch.empty_like(out)
            if rank < partner:
                dist.send(out, partner)
                dist.recv(inc, partner)
            else:
                dist.recv(inc, partner)
                dist.send(out, partner)
            shard[rows] = inc.numpy().view(np.complex128)
            sent += len(rows)
    return shard, sent


def _rank_main(rank, world, port, M, seed, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_quant_ph_0308158_gb300 import workloads as W
        k1 = W.random_state(M, np.complex128, seed)
        steps = W.random_circuit(M, 300, seed, max_controls=3)
        n_l = (1 << M) // world
        shard = k1[rank * n_l:(rank + 1) * n_l].copy()
        shard, sent = _sharded_apply(rank, world, M, shard, steps)
        out[rank] = (shard.view(np.float64).tolist(), sent)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_schedule_equals_the_oracle(world):
    import oracle
    from paper_quant_ph_0308158_gb300 import workloads as W
    M, seed = 10, 17 + world
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, M, seed, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    got = np.concatenate([np.array(out[r][0]).view(np.complex128) for r in range(world)])
    want = oracle.apply_circuit(M, W.random_state(M, np.complex128, seed),
                                W.random_circuit(M, 300, seed, max_controls=3))
    np.testing.assert_array_equal(got, want)
    assert all(out[r][1] > 0 for r in range(world))  # global targets exchanged rows
