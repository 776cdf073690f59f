"""Served form (rewl_server_*): requests of different models and sizes are
admitted by slots and device memory and run together; every result must be
bit-identical to the same request solved alone with rewl_create/rewl_step."""
import numpy as np
import pytest

from paper_1305_5615_gb300 import rewl

pytestmark = pytest.mark.gpu

REQS = [dict(model="ising", L=8, windows=4, walkers_per_window=2, lnf_final=1e-4, seed=11, q=2),
        dict(model="potts", L=6, windows=3, walkers_per_window=2, lnf_final=1e-3, seed=12, q=3),
        dict(model="ea", L=8, windows=4, walkers_per_window=2, lnf_final=1e-3, seed=13, q=2)]


def _alone(r):
    D = rewl.REWL(r["model"], r["L"], r["windows"], 0.75, r["walkers_per_window"], 0.8, r["lnf_final"], r["seed"],
                  q=r["q"])
    assert D.step(0)   # runs to completion
    return D.lng(), D.info["sweep_clock"]


def _submit(S, r):
    return S.submit(r["model"], r["L"], r["windows"], 0.75, r["walkers_per_window"], 0.8, r["lnf_final"], r["seed"],
                    q=r["q"])


def test_results_in_the_mix_equal_results_alone():
    alone = [_alone(r) for r in REQS]
    S = rewl.RewlServer(device_bytes=1 << 30, max_running=2)   # two slots: the third request waits
    ids = [_submit(S, r) for r in REQS]
    assert S.poll(ids[2])["state"] == rewl.REQ_QUEUED
    for _ in range(100000):
        st = S.run(50)
        if st["finished"] + st["failed"] == len(REQS):
            break
    assert st["finished"] == len(REQS) and st["failed"] == 0
    for rid, ((g, e0, de), sweeps) in zip(ids, alone):
        info = S.poll(rid)
        assert info["state"] == rewl.REQ_DONE and info["sweeps"] == sweeps
        gm, e0m, dem = S.result(rid)
        assert (e0m, dem) == (e0, de)
        assert np.array_equal(gm.view(np.uint64), g.view(np.uint64))   # bit-identical
        assert info["latency_ms"] >= info["run_ms"] >= 0 and info["queued_ms"] >= 0


def test_admission_by_device_memory():
    probe = rewl.RewlServer(device_bytes=1 << 30, max_running=8)
    rid = _submit(probe, REQS[0])
    need = probe.poll(rid)["device_bytes"]
    probe.close()
    S = rewl.RewlServer(device_bytes=need + need // 2, max_running=8)   # memory for one request at a time
    ids = [_submit(S, REQS[0]) for _ in range(3)]
    st = S.run(1)
    assert st["running"] == 1 and st["queued"] == 2 and st["device_bytes_in_use"] == need
    for _ in range(100000):
        st = S.run(50)
        if st["finished"] == 3:
            break
    assert st["finished"] == 3 and st["device_bytes_in_use"] == 0
    res = [S.result(i)[0] for i in ids]
    assert all(np.array_equal(res[0].view(np.uint64), r.view(np.uint64)) for r in res)   # same seed, same result
    with pytest.raises(rewl.RewlError) as e:
        rewl.RewlServer(device_bytes=need // 2, max_running=8).submit("ising", 8, 4, 0.75, 2, 0.8, 1e-4, 1)
    assert e.value.status == 2


def test_cancel_leaves_others_unchanged():
    (g0, _, _), _ = _alone(REQS[0])
    S = rewl.RewlServer(device_bytes=1 << 30, max_running=4)
    a = _submit(S, REQS[0])
    b = _submit(S, REQS[1])
    c = _submit(S, REQS[2])
    S.run(3)
    S.cancel(b)
    S.cancel(c)
    assert S.poll(b)["state"] == rewl.REQ_CANCELLED and S.poll(c)["state"] == rewl.REQ_CANCELLED
    for _ in range(100000):
        st = S.run(50)
        if st["running"] == 0 and st["queued"] == 0:
            break
    assert S.poll(a)["state"] == rewl.REQ_DONE
    assert np.array_equal(S.result(a)[0].view(np.uint64), g0.view(np.uint64))
    with pytest.raises(rewl.RewlError) as e:
        S.result(b)
    assert e.value.status == 7


def test_bad_requests():
    S = rewl.RewlServer(device_bytes=1 << 30, max_running=2)
    with pytest.raises(rewl.RewlError):
        S.submit("ising", 8, 4, 1.5, 2, 0.8, 1e-4, 1)
    with pytest.raises(rewl.RewlError):
        S.submit("ising", 300, 4, 0.75, 2, 0.8, 1e-4, 1)
    for flatness, lnf_final in ((0.0, 1e-4), (1.5, 1e-4), (0.8, 0.0), (0.8, 1e-13)):  # malformed: refused at once
        with pytest.raises(rewl.RewlError) as e:
            S.submit("ising", 8, 4, 0.75, 2, flatness, lnf_final, 1)
        assert e.value.status == 1
    # fails at admission (windows narrower than 3 bins), reported as a failed request
    rid = S.submit("ising", 8, 200, 0.75, 1, 0.8, 1e-4, 1)
    S.run(1)
    assert S.poll(rid)["state"] == rewl.REQ_FAILED and S.poll(rid)["error"] == 1
    with pytest.raises(rewl.RewlError) as e:
        S.poll(999999)
    assert e.value.status == 8


def test_one_shape_group_grows_and_shapes_run_side_by_side():
    """Twelve +-J disorder realisations of one shape (more than a group's first
    table of eight slots) beside two Ising requests of another shape, with
    requests arriving while others run: every result equals its result alone,
    and the sweep and trial counters equal those of the solve alone."""
    glass = [dict(model="ea", L=6, windows=3, walkers_per_window=2, lnf_final=1e-2, seed=100 + i, q=2)
             for i in range(12)]
    ising = [dict(model="ising", L=8, windows=4, walkers_per_window=2, lnf_final=1e-3, seed=200 + i, q=2)
             for i in range(2)]
    alone = {}
    for r in glass + ising:
        D = rewl.REWL(r["model"], r["L"], r["windows"], 0.75, r["walkers_per_window"], 0.8, r["lnf_final"],
                      r["seed"], q=r["q"])
        assert D.step(0)
        alone[r["seed"]] = (D.lng()[0], D.info["sweep_clock"], D.info["attempts"])
        D.close()
    S = rewl.RewlServer(device_bytes=1 << 30, max_running=16)
    ids = {}
    for r in ising + glass[:6]:
        ids[r["seed"]] = _submit(S, r)
    S.run(5)                                  # the rest arrive while these run
    for r in glass[6:]:
        ids[r["seed"]] = _submit(S, r)
    for _ in range(100000):
        st = S.run(50)
        if st["running"] == 0 and st["queued"] == 0:
            break
    assert st["finished"] == len(ids) and st["failed"] == 0
    for seed, rid in ids.items():
        g, sweeps, attempts = alone[seed]
        info = S.poll(rid)
        assert info["sweeps"] == sweeps and info["attempts"] == attempts, seed
        assert np.array_equal(S.result(rid)[0].view(np.uint64), g.view(np.uint64)), seed
    assert st["attempts"] == sum(alone[s][2] for s in ids)


def test_many_walkers_take_the_plain_chain_form_and_match_alone():
    """Forty requests of 32 walkers (1280 > 8 per SM on 152 SMs) run the
    batched sweep without producer warps; with the first three alone they run
    it with them.  Either way the results equal the solves alone."""
    reqs = [dict(model="ising", L=6, windows=4, walkers_per_window=8, lnf_final=1e-2, seed=300 + i, q=2)
            for i in range(40)]
    alone = {}
    for r in reqs[:3] + reqs[-2:]:
        D = rewl.REWL(r["model"], r["L"], r["windows"], 0.75, r["walkers_per_window"], 0.8, r["lnf_final"],
                      r["seed"], q=r["q"])
        assert D.step(0)
        alone[r["seed"]] = D.lng()[0]
        D.close()
    for batch in (reqs[:3], reqs):
        S = rewl.RewlServer(device_bytes=4 << 30, max_running=64)
        ids = {r["seed"]: _submit(S, r) for r in batch}
        for _ in range(100000):
            st = S.run(20)
            if st["running"] == 0 and st["queued"] == 0:
                break
        assert st["finished"] == len(batch)
        for seed, g in alone.items():
            if seed in ids:
                assert np.array_equal(S.result(ids[seed])[0].view(np.uint64), g.view(np.uint64)), seed
        S.close()


def test_admission_by_active_walkers():
    """With a target of 16 active walkers, a request of 8 windows x 2 walkers
    fills it: the next request waits although a slot and memory are free, and
    is admitted once windows of the first have finished.  Results stay
    bit-identical to solves alone."""
    r = dict(model="ising", L=8, windows=8, walkers_per_window=2, lnf_final=1e-3, seed=21, q=2)
    r2 = dict(r, seed=22)
    alone = [_alone(x) for x in (r, r2)]
    S = rewl.RewlServer(device_bytes=1 << 30, max_running=8, walker_target=16)
    ids = [_submit(S, r), _submit(S, r2)]
    st = S.run(1)
    assert st["running"] == 1 and st["queued"] == 1
    for _ in range(100000):
        st = S.run(20)
        if st["finished"] == 2:
            break
    assert st["finished"] == 2
    assert S.poll(ids[1])["queued_ms"] > 0
    for rid, ((g, _, _), sweeps) in zip(ids, alone):
        assert S.poll(rid)["sweeps"] == sweeps
        assert np.array_equal(S.result(rid)[0].view(np.uint64), g.view(np.uint64))


def test_submit_and_poll_do_not_wait_for_a_running_round():
    """rewl_server_run releases the server's lock while it waits on the GPU:
    submissions and polls from another thread return at once while a long
    replay of rounds is in flight, and the new request is then served."""
    import threading
    import time

    big = dict(model="ising", L=128, windows=8, walkers_per_window=4, lnf_final=1e-6, seed=5, q=2)  # ~0.1 s rounds
    S = rewl.RewlServer(device_bytes=1 << 30, max_running=8)
    first = _submit(S, big)
    S.run(2)                      # the group's replay length adapts after its first replay
    stop = threading.Event()

    def drive():
        while not stop.is_set():
            S.run(1)

    th = threading.Thread(target=drive)
    th.start()
    try:
        time.sleep(0.2)
        worst = 0.0
        for _ in range(20):
            t0 = time.perf_counter()
            S.poll(first)
            worst = max(worst, time.perf_counter() - t0)
        t0 = time.perf_counter()
        rid = _submit(S, REQS[0])
        worst = max(worst, time.perf_counter() - t0)
        assert worst < 0.05, worst   # one round of the big request lasts about 0.1 s; the calls do not wait for it
        for _ in range(100000):
            if S.poll(rid)["state"] == rewl.REQ_DONE:
                break
            time.sleep(0.01)
    finally:
        stop.set()
        th.join()
    (g, _, _), sweeps = _alone(REQS[0])
    assert S.poll(rid)["sweeps"] == sweeps
    assert np.array_equal(S.result(rid)[0].view(np.uint64), g.view(np.uint64))
    S.cancel(first)


def test_private_groups_for_long_rounds_equal_results_alone():
    """Requests whose round lasts milliseconds (Ising 24 x 24 and Potts 24 x 24: 57 600 trials per
    walker per round) get a group of their own; beside them small requests share one.  Every
    result stays bit-identical to the request solved alone."""
    reqs = [dict(model="ising", L=24, windows=4, walkers_per_window=2, lnf_final=1e-3, seed=31, q=2),
            dict(model="ising", L=24, windows=4, walkers_per_window=2, lnf_final=1e-3, seed=32, q=2),
            dict(model="potts", L=24, windows=4, walkers_per_window=2, lnf_final=1e-2, seed=33, q=3),
            dict(model="ising", L=8, windows=4, walkers_per_window=2, lnf_final=1e-4, seed=34, q=2)]
    alone = [_alone(r) for r in reqs]
    S = rewl.RewlServer(device_bytes=1 << 30, max_running=8)
    ids = [_submit(S, r) for r in reqs]
    for _ in range(100000):
        st = S.run(20)
        if st["finished"] + st["failed"] == len(reqs):
            break
    assert st["finished"] == len(reqs) and st["failed"] == 0
    for rid, ((g, e0, de), sweeps) in zip(ids, alone):
        assert S.poll(rid)["sweeps"] == sweeps
        assert np.array_equal(S.result(rid)[0].view(np.uint64), g.view(np.uint64))
