"""The multi-rank path of bench.py on CPU with the gloo backend, world size 2:
each rank renders its own cameras (interleaved views of one orbit, no data
exchanged), and the only collectives are the host-side timing and count
reductions."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _key(cam):
    return tuple(round(float(v), 9) for row in cam["viewmat"] for v in row)


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    from paper_2603_18707_b300 import synth

    class A:
        impl = "ours"

    w, r, _ = bench.dist_setup(A)
    assert (w, r) == (world, rank) and dist.get_backend() == "gloo"
    cams = synth.shard_orbit(4, r, w, 64, 48)
    gathered = [None] * w
    dist.all_gather_object(gathered, [_key(c) for c in cams])
    bench.barrier(w)
    mx = bench.max_over_ranks(float(r + 1), w)
    sm = bench.sum_over_ranks(float(10 * (r + 1)), w)
    out.put((r, gathered, mx, sm))
    dist.destroy_process_group()


def test_two_ranks_shard_cameras_and_reduce_timings():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, gathered, mx, sm in res:
        assert mx == 2.0 and sm == 30.0
        flat = [p for g in gathered for p in g]
        assert len(set(flat)) == len(flat) == 8  # disjoint views
        # together: the 8 views of one orbit, rank r holding views 2k + r
        from paper_2603_18707_b300 import synth
        ref = synth.orbit_cameras(8, 64, 48)
        for k in range(8):
            assert _key(ref[k]) == gathered[k % 2][k // 2]


if __name__ == "__main__":
    pytest.main([__file__, "-q"])
