"""The N > 1 path on CPU: two `gloo` ranks run as independent replicas, each localizing its
own frames (the oracle stands in for the GPU step), timed inside a barrier-bracketed region
and reduced by max over ranks, as the benchmark does on N GPUs."""
import multiprocessing as mp
import os
import socket
import time

import pytest

from paper_2410_02314_gb300 import replicas, synth

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica_frames(rank):
    return synth.workload_small(T=1, H=32, W=32, frame_seed=replicas.frame_seed(11, rank))


def _rank_main(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(WORLD),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import oracle

    ri = replicas.rank_info()
    dist.init_process_group("gloo", init_method="env://", rank=ri.rank, world_size=ri.world)
    try:
        w = _replica_frames(ri.rank)
        net = oracle.Net(w.spec.to_json(), w.blob)
        delay = 0.05 + 0.25 * ri.rank  # rank 1 is the slow one

        def run():
            t0 = time.perf_counter()
            recs, _, _ = oracle.localize(net, w.frames, 0.5)
            time.sleep(delay)
            return recs, time.perf_counter() - t0

        recs, own = replicas.timed_region(run, dist)
        worst = replicas.max_over_ranks(own, dist)
        q.put((ri.rank, own, worst, recs.tobytes(), w.frames.tobytes()))
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def replica_results():
    import oracle

    oracle.build()  # compile once before the ranks load it
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(WORLD):
        r = q.get(timeout=120)
        out[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def test_max_over_ranks_is_the_slowest_rank(replica_results):
    owns = [replica_results[r][1] for r in range(WORLD)]
    worsts = [replica_results[r][2] for r in range(WORLD)]
    assert worsts[0] == worsts[1] == max(owns)
    assert max(owns) >= 0.3  # rank 1 slept 0.3 s inside the region
    rate = replicas.whole_job_rate(1, worsts[0], WORLD)
    assert rate == pytest.approx(WORLD / max(owns))


def test_replicas_localize_their_own_frames_independently(replica_results):
    import oracle

    assert replica_results[0][4] != replica_results[1][4]  # different frames per rank
    for r in range(WORLD):
        w = _replica_frames(r)
        net = oracle.Net(w.spec.to_json(), w.blob)
        alone, _, _ = oracle.localize(net, w.frames, 0.5)
        assert replica_results[r][3] == alone.tobytes()  # no data crossed between ranks


def test_rank_info_defaults_and_env():
    assert replicas.rank_info({}) == replicas.RankInfo(0, 1, 0)
    assert replicas.rank_info({"RANK": "3", "WORLD_SIZE": "4", "LOCAL_RANK": "1"}) == replicas.RankInfo(3, 4, 1)
    assert replicas.max_over_ranks(2.5) == 2.5
    assert replicas.frame_seed(3, 0) != replicas.frame_seed(3, 1)
