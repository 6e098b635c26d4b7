"""The replica driver (independent updates per rank, Sec. 4.4) on CPU:
task sharding, the gather of results in task order, distributed central
differences and line searches against serial evaluation, and failure
detection.  The failure tests make a task raise on one rank, and make one
rank exit before the gather; the other rank must end with an error, not
hang.  Ranks are world-size-2 gloo process groups on 127.0.0.1."""
import json
import os
import socket
import sys

import numpy as np
import pytest

from paper_2001_11619_gb300 import replicas as R

HERE = os.path.dirname(os.path.abspath(__file__))


def test_shard_covers_every_task_once():
    for size in range(1, 6):
        for n in range(0, 14):
            seen = sorted(i for r in range(size) for i in R.shard(n, r, size))
            assert seen == list(range(n))
            counts = [len(R.shard(n, r, size)) for r in range(size)]
            assert max(counts) - min(counts) <= 1
    with pytest.raises(ValueError):
        R.shard(3, 2, 2)


def _poly(t):
    # degree 4: fourth-order central differences are exact up to rounding
    t = np.asarray(t)
    return float(np.sum(t ** 4) + 3.0 * t[0] * t[1] ** 2 - 2.0 * t[-1])


def _poly_grad(t):
    g = 4.0 * t ** 3
    g[0] += 3.0 * t[1] ** 2
    g[1] += 6.0 * t[0] * t[1]
    g[-1] -= 2.0
    return g


THETA = np.array([0.3, -1.1, 0.7, 2.0])


def test_single_process_matches_definitions():
    g4 = R.fd_gradient(_poly, THETA, 1e-3, order=4)
    assert np.allclose(g4, _poly_grad(THETA), rtol=1e-9, atol=1e-9)
    g2 = R.fd_gradient(_poly, THETA, 1e-4, order=2)
    assert np.allclose(g2, _poly_grad(THETA), rtol=1e-6, atol=1e-6)
    a, vals = R.line_search(lambda t: float(np.sum((t - 1.0) ** 2)), THETA,
                            np.ones(4), [-0.5, 0.0, 0.5, 1.0])
    assert vals == [float(np.sum((THETA + s - 1.0) ** 2))
                    for s in (-0.5, 0.0, 0.5, 1.0)]
    assert a == [-0.5, 0.0, 0.5, 1.0][int(np.argmin(vals))]
    assert R.max_over_ranks(2.5) == 2.5
    with pytest.raises(R.ReplicaError, match="rank 0"):
        R.run_batch([1, 2], lambda t: 1 / (t - 2))


# ---------------------------------------------------------------------------
# two gloo ranks


def _worker(rank, size, port, mode, outdir):
    import datetime

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=size,
                            timeout=datetime.timedelta(seconds=30))
    out = {"rank": rank}
    try:
        if mode == "batch":
            done = []

            def ev(t):
                done.append(t)
                return t * t + 0.5

            out["results"] = R.run_batch(list(range(7)), ev)
            out["evaluated"] = done
            out["grad"] = R.fd_gradient(_poly, THETA, 1e-3).tolist()
            a, vals = R.line_search(lambda t: float(np.sum((t - 1.0) ** 2)),
                                    THETA, np.ones(4), [-0.5, 0.0, 0.5, 1.0])
            out["alpha"], out["vals"] = a, vals
            out["tmax"] = R.max_over_ranks(10.0 + rank)
        elif mode == "raise":
            def ev(t):
                if rank == 1 and t == 3:
                    raise FloatingPointError("singular trial")
                return float(t)
            try:
                R.run_batch(list(range(6)), ev)
                out["error"] = None
            except R.ReplicaError as e:
                out["error"] = str(e)
        elif mode == "exit":
            if rank == 1:
                # leaves between steps, before the gather
                os._exit(0)
            try:
                R.run_batch(list(range(4)), float)
                out["error"] = None
            except Exception as e:  # the collective with a dead peer
                out["error"] = type(e).__name__
    finally:
        with open(os.path.join(outdir, f"r{rank}.json"), "w") as fh:
            json.dump(out, fh)
    if mode != "exit":
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spawn(mode, tmp_path, size=2):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker,
                         args=(r, size, port, mode, str(tmp_path)))
             for r in range(size)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
            pytest.fail(f"rank process hung in mode {mode}")
    res = {}
    for r in range(size):
        f = tmp_path / f"r{r}.json"
        if f.exists():
            res[r] = json.loads(f.read_text())
    return res


def test_two_ranks_match_serial(tmp_path):
    res = _spawn("batch", tmp_path)
    want = [t * t + 0.5 for t in range(7)]
    for r in (0, 1):
        assert res[r]["results"] == want
        assert res[r]["evaluated"] == R.shard(7, r, 2)
        # bitwise equal to the single-process gradient and line search
        assert res[r]["grad"] == R.fd_gradient(_poly, THETA, 1e-3).tolist()
        a, vals = R.line_search(lambda t: float(np.sum((t - 1.0) ** 2)),
                                THETA, np.ones(4), [-0.5, 0.0, 0.5, 1.0])
        assert res[r]["alpha"] == a and res[r]["vals"] == vals
        assert res[r]["tmax"] == 11.0


def test_task_failure_reaches_every_rank(tmp_path):
    res = _spawn("raise", tmp_path)
    for r in (0, 1):
        assert res[r]["error"] is not None
        assert "rank 1" in res[r]["error"] and "singular trial" in res[r]["error"]
        assert "rank 0" not in res[r]["error"]


def test_dead_rank_ends_the_batch_with_an_error(tmp_path):
    res = _spawn("exit", tmp_path)
    assert 1 not in res  # rank 1 left without writing
    assert res[0]["error"] is not None


if __name__ == "__main__":
    sys.exit(pytest.main([__file__, "-q"]))
