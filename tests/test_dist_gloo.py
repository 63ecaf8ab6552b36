"""Multi-rank best-of over CPU ranks (gloo, world size 2; no GPU).

The sharded multi-start must give exactly the single-process best-of: each
rank runs its share of starts (here with the CPU oracle as the local solver),
one all-reduce MIN of the packed (cost, start) key picks the winner, and the
owner broadcasts the winning solution.  A rank that fails before the
collective makes the other rank's collective end with an error after the
process-group timeout instead of hanging.
"""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1704_05132_gb300 import dist as D


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_pack_shard_helpers():
    assert D.unpack_key(D.pack_key(12345, 7)) == (12345, 7)
    assert D.pack_key(5, 9) < D.pack_key(5, 10) < D.pack_key(6, 0)
    assert D.unpack_key(D.pack_key(1 << 62, 3))[0] == (1 << 63) - 1
    # every key, the empty-rank sentinel and the largest finite cost
    # included, fits int64 and keeps its order there
    lo, hi = -(1 << 63), (1 << 63) - 1
    sentinel = D.pack_key(D.INF_COST, (1 << D.KEY_INDEX_BITS) - 1)
    big = D.pack_key(D.INF_COST - 1, 0)
    assert lo <= D.pack_key(0, 0) < big < sentinel <= hi
    assert D.unpack_key(big) == (D.INF_COST - 1, 0)
    for n, w in [(10, 3), (4096, 8), (3, 4), (1, 2)]:
        parts = [D.shard(n, r, w) for r in range(w)]
        assert parts[0][0] == 0 and parts[-1][1] == n
        assert all(parts[i][1] == parts[i + 1][0] for i in range(w - 1))
        assert max(h - l for l, h in parts) - min(h - l for l, h in parts) <= 1


def test_start_count_checked_before_any_collective():
    """No starts (or more than the 24-bit start index holds) is refused on
    the host, before a process group is even needed."""
    from paper_1704_05132_gb300 import gen
    inst = gen.plain_small()
    for n in (0, -1, 1 << 24):
        with pytest.raises(ValueError, match="nstarts"):
            D.multistart(inst, 0, n, 10)


def _oracle_solve(inst, seed0, count, iters, kmax, mode):
    import oracle
    best, res = oracle.multistart(oracle.Instance.from_arrays(inst),
                                  [seed0 + i for i in range(count)], iters, kmax, mode)
    return res[best].best_cost, best, res[best].gM, res[best].gR


def _worker(rank, world, port, nstarts, out_q, fail_rank):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=4))
    from paper_1704_05132_gb300 import gen
    inst = gen.make_instance(4, 2, K=3, T=8)
    try:
        if rank == fail_rank:
            raise RuntimeError("injected failure before the collective")
        res = D.multistart(inst, 100, nstarts, 6, 3, 0, solve=_oracle_solve)
        out_q.put((rank, "ok", res[0], res[1], res[2].tolist(), res[3].tolist()))
    except Exception as e:  # the surviving rank reports the collective error
        out_q.put((rank, "error", type(e).__name__, str(e)[:200], None, None))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, nstarts, fail_rank=-1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, nstarts, q, fail_rank))
             for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    return sorted(out)


@pytest.mark.parametrize("world,nstarts", [(2, 7), (3, 2)])
def test_sharded_bestof_equals_single_process(world, nstarts):
    """Also with fewer starts than ranks: a rank without starts contributes
    only the sentinel key and still receives the winner's solution."""
    import oracle
    from paper_1704_05132_gb300 import gen
    inst = gen.make_instance(4, 2, K=3, T=8)
    best, res = oracle.multistart(oracle.Instance.from_arrays(inst),
                                  [100 + i for i in range(nstarts)], 6, 3, 0)
    out = _run(world, nstarts)
    assert len(out) == world
    for rank, status, cost, start, gm, gr in out:
        assert status == "ok"
        assert (cost, start) == (res[best].best_cost, best)
        assert np.array_equal(np.array(gm), res[best].gM)
        assert np.array_equal(np.array(gr), res[best].gR)


def test_failed_rank_does_not_hang_the_other():
    out = _run(2, 4, fail_rank=1)
    assert out[1][1] == "error" and "injected" in out[1][3]
    assert out[0][1] == "error"  # the collective failed instead of waiting forever
