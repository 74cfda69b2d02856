"""The one-process-per-GPU host logic on CPU, as two gloo ranks on 127.0.0.1.

* Strong sharding: the ranks' contiguous shards partition the table, and the
  decisions each rank computes for its shard (float64 oracle, tiny decoder)
  gathered on rank 0 equal a single process's decisions over the whole table
  -- tuples are independent, nothing on the data path crosses ranks.
* Weak sharding: rank seeds give different tables of the same size.
* Timing: the job time is the maximum over ranks and the job rate counts all
  ranks' tuples.
* Failure detection on the host: a rank that raises before the timing
  collective is noticed by the other rank as an error of that collective
  within the process group's timeout (no GPU involved)."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _tiny():
    from paper_2602_04430_b300 import synth
    cfg = synth.ModelConfig(layers=2, d=32, hq=4, hkv=2, hd=8, ffn=48, vocab=64, dtype="f32", name="t")
    w = synth.make_weights(cfg, seed=41, std=0.3)
    table = synth.make_table_from_lengths([3, 9, 17, 5, 12, 7, 20], cfg.vocab, seed=42)
    op = synth.make_prompt(5, cfg.vocab, seed=43, label_ids=(1, 0), r=0.5)
    return cfg, w, table, op


def _decisions(cfg, w, table, op, tuples):
    from oracle import operator as O
    _, labels, _ = O.run_table(cfg, w, table, op, tuples=list(tuples))
    return [int(x) for x in labels]


def _worker(rank, world, port, mode, out_dir):
    import torch
    import torch.distributed as dist
    from paper_2602_04430_b300 import multigpu, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    result = {}
    try:
        if mode == "shards":
            cfg, w, table, op = _tiny()
            T = len(table["offsets"]) - 1
            b, e = multigpu.shard_range(T, world, rank)
            mine = _decisions(cfg, w, table, op, range(b, e))
            gathered = [None] * world
            dist.all_gather_object(gathered, (b, e, mine))
            result["gathered"] = gathered
            result["ms_max"] = multigpu.reduce_max(10.0 + 5 * rank, dist)
            result["seed_tables_differ"] = None
            tw = synth.make_table(synth.TABLES["tiny"], cfg.vocab, seed=multigpu.rank_seed(1000, rank), n_tuples=4)
            all_tok = [None] * world
            dist.all_gather_object(all_tok, (len(tw["offsets"]) - 1, tw["tokens"][:64].tolist()))
            result["weak"] = all_tok
        elif mode == "failure":
            if rank == 1:
                raise RuntimeError("rank 1 fails before its timing collective")
            try:
                multigpu.reduce_max(1.0, dist)
                result["noticed"] = False
            except Exception as exc:   # gloo: peer closed / timeout
                result["noticed"] = True
                result["error"] = type(exc).__name__
    except RuntimeError as exc:
        result["raised"] = str(exc)
    finally:
        torch.save(result, os.path.join(out_dir, f"rank{rank}.pt"))
        if mode != "failure":
            dist.destroy_process_group()


def _run(mode, tmp_path, world=2):
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, port, mode, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
            p.join()
            pytest.fail("a rank did not finish")
    import torch
    return [torch.load(os.path.join(tmp_path, f"rank{r}.pt")) for r in range(world)]


def test_shards_equal_single_process(tmp_path):
    from paper_2602_04430_b300 import multigpu
    res = _run("shards", tmp_path)
    cfg, w, table, op = _tiny()
    T = len(table["offsets"]) - 1
    g = res[0]["gathered"]
    # contiguous, disjoint, covering
    assert [x[0] for x in g] == [0, g[0][1]] and g[-1][1] == T and g[0][1] == g[1][0]
    assert abs((g[0][1] - g[0][0]) - (g[1][1] - g[1][0])) <= 1
    merged = [d for (_, _, ds) in g for d in ds]
    assert merged == _decisions(cfg, w, table, op, range(T))
    # the job time is the slowest rank's; the job rate counts every rank's tuples
    assert res[0]["ms_max"] == res[1]["ms_max"] == 15.0
    assert multigpu.job_rate([4, 3], 15.0) == pytest.approx(7 / 0.015)
    # weak sharding: same size, different tables per rank
    (n0, t0), (n1, t1) = res[0]["weak"]
    assert n0 == n1 == 4 and t0 != t1


def test_failed_rank_is_noticed(tmp_path):
    res = _run("failure", tmp_path)
    assert "raised" in res[1]
    assert res[0]["noticed"] is True


@pytest.mark.parametrize("n,world", [(0, 1), (7, 2), (10, 3), (2, 4)])
def test_shard_range_partitions(n, world):
    from paper_2602_04430_b300 import multigpu
    spans = [multigpu.shard_range(n, world, r) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
    sizes = [e - b for b, e in spans]
    assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        multigpu.shard_range(n, world, world)
