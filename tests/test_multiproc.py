"""The N > 1 path of bench.py on CPU: two gloo ranks, each advancing its own
replica ensemble (members are independent, so nothing but a barrier and the
max of the timed durations crosses ranks), and each building the library's
handle for its replica on the host (the same operators and workspace on every
rank, so replicas need no exchange of either)."""
import hashlib
import os
import queue
import socket
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

G = dict(flow="couette", mx=16, my=17, mz=16, lx=1.75 * np.pi, lz=1.2 * np.pi, re=400.0, dt=0.01, members=2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank):
    import bench
    import oracle
    st = bench.initial_state(G, rank)
    ch = oracle.Channel(G["mx"], G["my"], G["mz"], G["lx"], G["lz"], G["re"], G["dt"], G["flow"])
    x = ch.step(tuple(st[k] for k in ("v", "eta", "U", "W")), 2)
    return ch.stats(x)["e_total"]


def _library_replica():
    """The host side of a replica's handle: workspace bytes and a digest of the
    operators of one wavenumber pair (no GPU: dns_create builds them on the host)."""
    import paper_2306_12739_gb300 as dns
    h = dns.dns_create(dns.make_config([G], precision="mixed"), 0)
    try:
        nbytes = dns.dns_workspace_size(h)
        ops = dns.dns_export_operators(h, 0, 1, 1, G["my"] - 2)
        digest = hashlib.sha256(b"".join(np.ascontiguousarray(a).tobytes() for a in ops)).hexdigest()
    finally:
        dns.dns_destroy(h)
    return int(nbytes), digest


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    try:
        import bench
        r, w, dist = bench.dist_setup()
        assert (r, w) == (rank, world) and dist is not None
        t0 = time.perf_counter()
        energy = _replica(rank)
        dt = time.perf_counter() - t0 + 0.05 * rank      # ranks finish at different times
        lib = _library_replica()
        tmax = bench.reduce_max(dt, dist)
        value = bench.aggregate(G["members"] * 2, tmax, w)
        gathered = [None] * w
        dist.all_gather_object(gathered, energy.tolist())
        libs = [None] * w
        dist.all_gather_object(libs, lib)
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, dt, tmax, value, gathered, libs))
    except Exception as exc:  # pragma: no cover - reported to the parent
        q.put((rank, "error", repr(exc)))


def test_two_gloo_ranks_run_replicas_and_report_whole_job_throughput():
    import __graft_entry__
    __graft_entry__.build()          # the ranks load the library built here
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = {}
    try:
        for _ in range(2):
            item = q.get(timeout=240)
            assert item[1] != "error", item
            results[item[0]] = item
    except queue.Empty:  # pragma: no cover
        pytest.fail("a rank did not report")
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    dts = [results[r][1] for r in range(2)]
    for r in range(2):
        _, dt, tmax, value, gathered, libs = results[r]
        assert tmax == pytest.approx(max(dts))                      # max over ranks
        assert value == pytest.approx(G["members"] * 2 * 2 / max(dts))   # all ranks' member-steps / slowest
        # each rank advanced a distinct replica, identical to running it alone
        assert not np.allclose(gathered[0], gathered[1])
        # and built the same handle: workspace size and operators
        assert libs[0] == libs[1] and libs[0][0] > 0
    alone = [_replica(r) for r in range(2)]
    for r in range(2):
        assert np.allclose(results[0][4][r], alone[r], rtol=1e-13, atol=0)


E4 = dict(G, members=4)


def _shard_stats(lo, hi):
    """Oracle statistics of members lo..hi-1 of one seeded 4-member ensemble
    after two steps (members are independent: a shard is the same computation)."""
    import dns_synth
    import oracle
    st = dns_synth.make_state(E4["mx"], E4["my"], E4["mz"], E4["lx"], E4["lz"], E4["flow"], E4["members"], 500, 5e-2)
    ch = oracle.Channel(E4["mx"], E4["my"], E4["mz"], E4["lx"], E4["lz"], E4["re"], E4["dt"], E4["flow"])
    x = ch.step(tuple(st[k][lo:hi] for k in ("v", "eta", "U", "W")), 2)
    return ch.stats(x)


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    try:
        import bench
        r, w, dist = bench.dist_setup()
        per = E4["members"] // w
        s = _shard_stats(r * per, (r + 1) * per)
        # host-side sums over the ranks' member ranges: the ensemble means
        sums = torch.tensor([s["e_total"].sum(), s["e_pert"].sum(), s["tau_bottom"].sum()] + list(s["uu"].sum(0)),
                            dtype=torch.float64)
        dist.all_reduce(sums)
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, "ok", (sums / E4["members"]).numpy(), s["e_total"]))
    except Exception as exc:  # pragma: no cover - reported to the parent
        q.put((rank, "error", repr(exc)))


def test_member_range_sharding_with_host_summed_statistics_equals_one_ensemble():
    """One ensemble split by member range over two gloo ranks, each advancing
    its own members, statistics summed on the host: the ensemble means and
    every member's values equal those of the whole ensemble in one process."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = {}
    try:
        for _ in range(2):
            item = q.get(timeout=240)
            assert item[1] != "error", item
            results[item[0]] = item
    except queue.Empty:  # pragma: no cover
        pytest.fail("a rank did not report")
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    whole = _shard_stats(0, E4["members"])
    want = np.array([whole["e_total"].mean(), whole["e_pert"].mean(), whole["tau_bottom"].mean()]
                    + list(whole["uu"].mean(0)))
    for r in range(2):
        assert np.allclose(results[r][2], want, rtol=1e-12, atol=1e-18)
    per_member = np.concatenate([results[0][3], results[1][3]])
    assert np.allclose(per_member, whole["e_total"], rtol=1e-13, atol=0)
