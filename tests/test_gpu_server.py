"""The continuous-batching server (kf_server_*) through the C ABI.

Each event's result must be the same alone and in the mix: events run
alone through kf_kalman_chain give the reference, then all events go
through the server concurrently (batched with whatever else is in flight);
the results must match bit for bit (one thread per track, same arithmetic).
Events are either copied through the arena or, where the GPU reaches their
host arrays in place, read and written there by the batch kernel (the
direct path); both, and batches that mix them, are covered.  Failure paths
are exercised on the host: a paused server makes a bounded wait time out,
and an event larger than the arena is refused."""
import threading
import time

import numpy as np
import pytest
import torch

import oracle
import parity_log
from oracle import compare
from paper_2401_14221_gb300 import build as kbuild
from paper_2401_14221_gb300 import kf
from paper_2401_14221_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def events():
    rng = np.random.default_rng(5)
    sizes = W.lognormal_event_sizes(rng, 40, median=800.0, lo=50, hi=6000)
    return W.make_chain(events=len(sizes), seed=51, sizes=sizes, pool=20000)


@pytest.fixture(params=[kf.KF_HOST_COPY, kf.KF_HOST_DIRECT], ids=["copy", "direct"])
def host_path(request, dev):
    """Events copied through the arena, or worked on in place by the kernel."""
    kf.kf_set_host_path(request.param)
    yield request.param
    kf.kf_set_host_path(kf.KF_HOST_AUTO)


def event_arrays(cw, e, pinned=True):
    lo = int(cw.event_sizes[:e].sum())
    hi = lo + int(cw.event_sizes[e])
    pin = lambda t: t.pin_memory() if pinned else t
    host = lambda a: pin(torch.from_numpy(np.ascontiguousarray(a)))
    ins = (host(cw.state[:, lo:hi]), host(cw.cov[:, lo:hi]), host(cw.charge[lo:hi]),
           host(cw.hit[:, :, lo:hi]), host(cw.hitcov[:, :, lo:hi]))
    n = hi - lo
    outs = (pin(torch.empty((6, n), dtype=torch.float32)),
            pin(torch.empty((21, n), dtype=torch.float32)),
            pin(torch.empty(n, dtype=torch.uint8)))
    return lo, hi, ins, outs


def alone(cw, e, dev):
    lo, hi = int(cw.event_sizes[:e].sum()), int(cw.event_sizes[:e + 1].sum())
    sub = W.ChainWorkload(n=hi - lo, bz=cw.bz, kinds=cw.kinds, pos=cw.pos,
                          event_sizes=np.array([hi - lo]), state=cw.state[:, lo:hi],
                          cov=cw.cov[:, lo:hi], charge=cw.charge[lo:hi], hit=cw.hit[:, :, lo:hi],
                          hitcov=cw.hitcov[:, :, lo:hi], truth_pool_layers=cw.truth_pool_layers,
                          truth_index=cw.truth_index[lo:hi])
    dc = kf.chain_upload(sub, kf.KF_SOA, 0, dev)
    dc.run()
    return dc.download()


def make_server(cw, dev, arena_bytes, slots=64, precision=kf.KF_FP32):
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device=dev)
    return kf.Server(cw.bz, cw.kinds, cw.pos, arena, max_events_in_flight=slots,
                     precision=precision)


@pytest.mark.parametrize("mode", ["copy", "direct", "mixed"])
def test_results_alone_equal_results_in_the_mix(dev, events, mode):
    # mixed: every other event is copied through the arena, the rest are
    # direct, so batches hold both kinds
    cw = events
    refs = [alone(cw, e, dev) for e in range(len(cw.event_sizes))]
    srv = make_server(cw, dev, 512 << 20)
    lock = threading.Lock()
    path = {"copy": lambda e: kf.KF_HOST_COPY, "direct": lambda e: kf.KF_HOST_DIRECT,
            "mixed": lambda e: kf.KF_HOST_COPY if e % 2 else kf.KF_HOST_DIRECT}[mode]
    try:
        arrays = [event_arrays(cw, e) for e in range(len(cw.event_sizes))]
        tickets = [None] * len(arrays)

        def submit(idx, gap):
            for e in idx:
                _, _, ins, outs = arrays[e]
                with lock:  # the host-path mode is process-wide
                    kf.kf_set_host_path(path(e))
                    tickets[e] = srv.submit(*ins, *outs)
                time.sleep(gap * (e % 3))
        # first half: two threads submit while the server is paused, so the
        # events share batches; second half: submitted while batches run
        half = len(arrays) // 2
        srv.pause(True)
        th = [threading.Thread(target=submit, args=(range(k, half, 2), 0.0)) for k in (0, 1)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        srv.pause(False)
        th = [threading.Thread(target=submit, args=(range(half + k, len(arrays), 2), 2e-4))
              for k in (0, 1)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for e, t in enumerate(tickets):
            srv.wait(t, 60.0)
        st = srv.stats()
        assert st["events_done"] == len(arrays)
        assert st["max_batch_events"] > 1  # requests were batched together
        for e, (_, _, _, outs) in enumerate(arrays):
            ref = refs[e]
            assert np.array_equal(outs[0].numpy(), ref[0])
            assert np.array_equal(outs[1].numpy(), ref[1])
            assert np.array_equal(outs[2].numpy(), ref[2])
    finally:
        kf.kf_set_host_path(kf.KF_HOST_AUTO)
        srv.close()


def test_direct_events_in_pageable_memory(dev, events):
    # on a device that walks the host page tables, events in ordinary
    # (pageable) host memory take the direct path too
    cw = events
    srv = make_server(cw, dev, 64 << 20)
    kf.kf_set_host_path(kf.KF_HOST_DIRECT)
    try:
        for e in range(0, len(cw.event_sizes), 7):
            _, _, ins, outs = event_arrays(cw, e, pinned=False)
            try:
                t = srv.submit(*ins, *outs)
            except kf.KfError as err:
                if "not reachable" in str(err):
                    pytest.skip("this device does not reach pageable host memory")
                raise
            srv.wait(t, 60.0)
            ref = alone(cw, e, dev)
            for a, b in zip(outs, ref):
                assert np.array_equal(a.numpy(), b)
        st = srv.stats()
        assert st["copyin_p99_ms"] == 0.0 and st["out_p99_ms"] < 1.0
        # direct events copy nothing: no device copy time either
        assert st["gpu_copyin_p99_ms"] == 0.0 and st["gpu_out_p99_ms"] == 0.0
        assert st["gpu_compute_p50_ms"] > 0.0
    finally:
        kf.kf_set_host_path(kf.KF_HOST_AUTO)
        srv.close()


def test_direct_adaptive_events_without_status(dev, events):
    # a direct event given no status array keeps KF_ADAPTIVE's redo marks in
    # the arena; its results equal those of the same event given one
    cw = events
    srv = make_server(cw, dev, 64 << 20, precision=kf.KF_ADAPTIVE)
    kf.kf_set_host_path(kf.KF_HOST_DIRECT)
    try:
        for e in range(0, len(cw.event_sizes), 5):
            _, _, ins, outs = event_arrays(cw, e)
            _, _, _, outs2 = event_arrays(cw, e)
            t1 = srv.submit(*ins, *outs)
            t2 = srv.submit(*ins, outs2[0], outs2[1], None)
            srv.wait(t1, 60.0)
            srv.wait(t2, 60.0)
            assert torch.equal(outs[0], outs2[0]) and torch.equal(outs[1], outs2[1])
    finally:
        kf.kf_set_host_path(kf.KF_HOST_AUTO)
        srv.close()


@pytest.mark.parametrize("precision", [kf.KF_ADAPTIVE, kf.KF_FP64])
def test_server_results_match_the_oracle(dev, events, precision, host_path):
    # adaptive: tracks with an ill-conditioned layer (grazing crossings) run
    # the whole chain again in double; FP64: every track in double.  Both
    # keep every track within the bounds.
    cw = events
    srv = make_server(cw, dev, 256 << 20, precision=precision)
    try:
        for e in range(0, len(cw.event_sizes), 9):
            lo, hi, ins, outs = event_arrays(cw, e)
            srv.wait(srv.submit(*ins, *outs))
            hit = np.ascontiguousarray(cw.hit[:, :, lo:hi].transpose(0, 2, 1), dtype=np.float64)
            hc = np.ascontiguousarray(cw.hitcov[:, :, lo:hi].transpose(0, 2, 1), dtype=np.float64)
            o_st, o_cv, o_stat = oracle.chain_batch(cw.kinds, cw.pos, cw.state.T[lo:hi],
                                                    cw.cov.T[lo:hi], cw.charge[lo:hi], hit, hc,
                                                    cw.bz)
            r = np.hypot(o_st[:, 0], o_st[:, 1])
            on_plane = np.isin(o_st[:, 2], cw.pos[cw.kinds == W.P2Z].astype(np.float64))
            on_cyl = np.zeros(hi - lo, dtype=bool)
            for R in cw.pos[cw.kinds == W.P2R].astype(np.float64):
                on_cyl |= np.abs(r - R) <= 1e-5 * R
            rep = compare.compare(outs[0].numpy().T, outs[1].numpy().T, outs[2].numpy(), o_st,
                                  o_cv, o_stat, on_cylinder=on_cyl & ~on_plane)
            parity_log.expect_ok("server", rep)
    finally:
        srv.close()


def test_admission_waits_for_arena_space(dev, events):
    # an arena that holds about two of the largest copied events: the rest
    # wait
    cw = events
    kf.kf_set_host_path(kf.KF_HOST_COPY)
    sizes = cw.event_sizes[:12]
    arena_bytes = 2 * kf.kf_server_event_bytes(int(sizes.max()), cw.L) + 4096
    fits = arena_bytes // kf.kf_server_event_bytes(int(sizes.min()), cw.L)
    srv = make_server(cw, dev, arena_bytes)
    try:
        arrays = [event_arrays(cw, e) for e in range(12)]
        tickets = [srv.submit(*a[2], *a[3]) for a in arrays]
        for t in tickets:
            srv.wait(t, 60.0)
        st = srv.stats()
        assert st["events_done"] == 12 and st["max_batch_events"] <= min(fits, 11)
        for e, (_, _, _, outs) in enumerate(arrays):
            ref = alone(cw, e, dev)
            assert np.array_equal(outs[0].numpy(), ref[0])
    finally:
        kf.kf_set_host_path(kf.KF_HOST_AUTO)
        srv.close()


def test_paused_server_wait_times_out_then_completes(dev, events, host_path):
    cw = events
    srv = make_server(cw, dev, 64 << 20)
    try:
        srv.pause(True)
        _, _, ins, outs = event_arrays(cw, 0)
        t = srv.submit(*ins, *outs)
        with pytest.raises(kf.KfError) as e:
            srv.wait(t, 0.05)
        assert e.value.code == kf.KF_ERR_TIMEOUT
        assert not srv.poll(t)
        srv.pause(False)
        srv.wait(t, 60.0)
        # the latency split: the event sat in the queue for the whole pause
        st = srv.stats()
        assert st["events_done"] == 1 and st["queue_p50_ms"] >= 50.0
        for ph in ("queue", "ready", "copyin", "compute", "out"):
            assert 0.0 <= st[f"{ph}_p50_ms"] <= st[f"{ph}_p99_ms"]
        assert st["copyin_p50_ms"] <= st["ready_p50_ms"]  # copy-in is part of ready
        assert st["queue_p50_ms"] + st["ready_p50_ms"] + st["compute_p50_ms"] + \
            st["out_p50_ms"] <= st["max_ms"] + 1e-6
        # the device's own durations (timing events in the streams) fit
        # inside what the scheduler observed for the phase; a direct event
        # copies nothing
        copied = host_path == kf.KF_HOST_COPY
        for ph in ("copyin", "compute", "out"):
            assert 0.0 <= st[f"gpu_{ph}_p50_ms"] <= st[f"{ph}_p50_ms"] + 0.05
            assert st[f"gpu_{ph}_p50_ms"] > 0.0 or (ph != "compute" and not copied)
        assert st["copyin_issue_p50_ms"] <= st["copyin_p50_ms"]
    finally:
        srv.close()


def test_event_larger_than_arena_is_refused(dev, events):
    # a copied event needs its whole arrays in the arena, a direct one only
    # its status marks (n bytes rounded up to 256)
    cw = events
    big = int(np.argmax(cw.event_sizes))
    n = int(cw.event_sizes[big])
    for path, arena_bytes in ((kf.KF_HOST_COPY, 1 << 20), (kf.KF_HOST_DIRECT, n - 256)):
        srv = make_server(cw, dev, arena_bytes)
        kf.kf_set_host_path(path)
        try:
            _, _, ins, outs = event_arrays(cw, big)
            with pytest.raises(kf.KfError) as e:
                srv.submit(*ins, *outs)
            assert e.value.code == kf.KF_ERR_ARG
        finally:
            kf.kf_set_host_path(kf.KF_HOST_AUTO)
            srv.close()
