"""The continuous-batching server (ism_server_*) on the GPU.

Each request is one room with 1 source and 1-16 receivers drawn like the
serving stream (sides 3-10 m, T60 0.2-1.0 s, 16 kHz, Tdiff = min(0.25 s,
T60), Tmax = T60).  A request's RIRs must be bit-identical whether it is
computed alone through ism_simulate_host or inside any mix of the server's
batches, and its image-source part must match the FP64 oracle to 1e-5 of
its peak.
"""
import threading

import numpy as np
import pytest

import oracle
from paper_1810_11359_gb300 import ism, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def feasible(L, rt):
    try:
        ism.ism_beta_sabine(L, rt)
        return True
    except ism.IsmError:
        return False


def request_args(room):
    """Arguments of one request of the serving stream."""
    beta = ism.ism_beta_sabine(room.L, room.rt60)
    Tdiff = min(0.25, room.rt60)
    Tw = room.window()
    N = ism.ism_nb_img_from_t(Tdiff, room.L, room.c, Tw)
    return dict(L=room.L, beta=beta, pos_src=room.pos_src, pos_rcv=room.pos_rcv, nb_img=N, Tmax=room.Tmax,
                fs=room.fs, Tdiff=Tdiff, Tw=Tw, seed=room.seed)


def alone(a):
    return ism.ism_simulate_host(a["L"], a["beta"], a["pos_src"], a["pos_rcv"], a["nb_img"], a["Tmax"], a["fs"],
                                 Tdiff=a["Tdiff"], Tw=a["Tw"], seed=a["seed"])


def submit(server, a):
    return server.submit(a["L"], a["beta"], a["pos_src"], a["pos_rcv"], a["nb_img"], a["Tmax"], a["fs"],
                         Tdiff=a["Tdiff"], Tw=a["Tw"], seed=a["seed"])


def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = [request_args(r.room) for r in workloads.serving_requests(80, seed=4, feasible=feasible)]
    ref = [alone(a) for a in reqs]
    with ism.Server(hbm_budget=2 << 30, max_inflight=3, max_batch=16) as srv:
        # request 0 alone on an idle server, then everything at once from two threads
        t0, out0 = submit(srv, reqs[0])
        srv.wait(t0)
        assert np.array_equal(out0.view(np.uint32), ref[0].view(np.uint32))
        tickets = [None] * len(reqs)

        def submitter(idx):
            for i in idx:
                tickets[i] = submit(srv, reqs[i])

        th = [threading.Thread(target=submitter, args=(range(k, len(reqs), 2),)) for k in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for i, (t, out) in enumerate(tickets):
            lat = srv.wait(t)
            assert lat > 0
            assert np.array_equal(out.view(np.uint32), ref[i].view(np.uint32)), i
        st = srv.stats()
        assert st["completed"] == len(reqs) + 1 and st["failed"] == 0
        assert st["batches"] >= 2 and st["inflight_peak"] >= 2      # batches overlapped on the GPU
        assert st["dev_in_use"] == 0 and st["host_in_use"] == 0     # everything returned to the pools
    # the image-source part of a few requests against the oracle
    for i in [0, 17, 55]:
        a = reqs[i]
        b32 = np.asarray(a["beta"], np.float32).astype(np.float64)
        n_ism = oracle.n_samples(np.float32(a["Tdiff"]), a["fs"])
        ps = np.repeat(a["pos_src"], a["pos_rcv"].shape[0], axis=0).astype(np.float64)
        pr = a["pos_rcv"].astype(np.float64)
        h = oracle.rir_list(a["L"], b32, float(np.float32(343.0)), float(np.float32(a["fs"])),
                            float(np.float32(a["Tw"])), ps, pr, a["nb_img"], n_ism)
        got = ref[i].reshape(-1, ref[i].shape[-1])[:, :n_ism].astype(np.float64)
        assert np.max(np.abs(got - h)) <= TOL_FP32 * np.max(np.abs(h)), i
        assert np.all(np.isfinite(ref[i]))


def test_admission_under_a_small_budget():
    """A 64 MiB pool holds only a few requests with their workspace at a time:
    every request still completes, in arrival order of admission, and the
    pool never holds more than its budget."""
    reqs = [request_args(r.room) for r in workloads.serving_requests(40, seed=8, feasible=feasible)]
    budget = 64 << 20
    with ism.Server(hbm_budget=budget, host_budget=16 << 20, max_inflight=2, max_batch=8) as srv:
        tk = []
        for a in reqs:
            try:
                tk.append((submit(srv, a), a))
            except ism.IsmError as e:
                assert e.status == ism.STATUS_CODES["ISM_ERR_OOM"]     # can never fit 64 MiB
        assert len(tk) >= 10
        for (t, out), a in tk:
            srv.wait(t)
            assert np.array_equal(out.view(np.uint32), alone(a).view(np.uint32))
        st = srv.stats()
        assert st["dev_peak"] <= budget and st["failed"] == 0


def test_request_larger_than_the_budget_is_rejected_at_submit():
    room = workloads.trajectory_array()      # 512 RIRs x 57,600 samples: 118 MB of output alone
    beta = ism.ism_beta_sabine(room.L, room.rt60)
    N = ism.ism_nb_img_from_t(room.Tdiff, room.L, room.c, room.window())
    with ism.Server(hbm_budget=32 << 20) as srv:
        with pytest.raises(ism.IsmError) as ei:
            srv.submit(room.L, beta, room.pos_src, room.pos_rcv, N, room.Tmax, room.fs, Tdiff=room.Tdiff,
                       Tw=room.window())
        assert ei.value.status == ism.STATUS_CODES["ISM_ERR_OOM"]
        assert srv.stats()["submitted"] == 0


def test_invalid_requests_fail_on_the_host_at_submit():
    L = np.array([4.0, 5.0, 3.0])
    beta = ism.ism_beta_sabine(L, 0.5)
    N = ism.ism_nb_img_from_t(0.2, L, 343.0, 32 / 16000)
    with ism.Server(hbm_budget=64 << 20) as srv:
        for ps, pr in [([[4.5, 1.0, 1.0]], [[1.0, 1.0, 1.0]]), ([[1.0, 1.0, 1.0]], [[1.0, -0.1, 1.0]])]:
            with pytest.raises(ism.IsmError) as ei:
                srv.submit(L, beta, ps, pr, N, 0.2, 16000.0, Tw=32 / 16000)
            assert ei.value.status == ism.STATUS_CODES["ISM_ERR_INVALID_ARG"]
        with pytest.raises(ism.IsmError):
            srv.submit(L, beta, [[1.0, 1.0, 1.0]], [[2.0, 2.0, 2.0]], [0, 3, 3], 0.2, 16000.0)
        # the server still serves after rejecting them
        t, out = srv.submit(L, beta, [[1.0, 1.0, 1.0]], [[2.0, 2.0, 2.0]], N, 0.2, 16000.0, Tw=32 / 16000)
        srv.wait(t)
        assert np.all(np.isfinite(out))


def test_wait_timeout_poll_and_ticket_release():
    room = workloads.trajectory_array()
    beta = ism.ism_beta_sabine(room.L, room.rt60)
    N = ism.ism_nb_img_from_t(room.Tdiff, room.L, room.c, room.window())
    with ism.Server(hbm_budget=2 << 30) as srv:
        t, out = srv.submit(room.L, beta, room.pos_src[:16], room.pos_rcv, N, room.Tmax, room.fs,
                            Tdiff=room.Tdiff, Tw=room.window(), seed=3)
        try:
            srv.wait(t, timeout_s=0.0)
            timed_out = False
        except ism.IsmError as e:
            assert e.status == ism.STATUS_CODES["ISM_ERR_TIMEOUT"]
            timed_out = True
        if timed_out:
            srv.wait(t)                      # the ticket stayed valid
        with pytest.raises(ism.IsmError):    # and is released once waited for
            srv.poll(t)
        assert np.all(np.isfinite(out))


def test_destroy_with_queued_requests_returns():
    reqs = [request_args(r.room) for r in workloads.serving_requests(200, seed=9, feasible=feasible)]
    srv = ism.Server(hbm_budget=256 << 20, max_inflight=1, max_batch=4)
    for a in reqs:
        submit(srv, a)
    srv.close()        # finishes what is on the GPU, cancels the rest, joins its threads


def test_batch_submit_matches_alone_and_is_all_or_nothing():
    """ism_server_submit_batch: 60 requests in one call give, bitwise, each
    request's RIRs computed alone; a call with one bad job (a receiver outside
    its room) queues none of its jobs and names the bad one."""
    reqs = [request_args(r.room) for r in workloads.serving_requests(60, seed=12, feasible=feasible)]
    ref = [alone(a) for a in reqs]
    with ism.Server(hbm_budget=2 << 30, max_inflight=3, max_batch=16) as srv:
        got = srv.submit_many(reqs)
        for (t, out), r in zip(got, ref):
            assert srv.wait(t) > 0
            assert np.array_equal(out.view(np.uint32), r.view(np.uint32))
        # page-locked result buffers: the kernels write the RIRs into them directly
        pinned = [torch.full(r.shape, float("nan")).pin_memory() for r in ref]
        got = srv.submit_many(reqs, outs=[o.numpy() for o in pinned])
        for (t, out), r in zip(got, ref):
            srv.wait(t)
            assert np.array_equal(out.view(np.uint32), r.view(np.uint32))
        before = srv.stats()["submitted"]
        bad = [dict(a) for a in reqs[:5]]
        bad[3]["pos_rcv"] = np.array([[-1.0, 1.0, 1.0]], np.float32)
        with pytest.raises(ism.IsmError, match="job 3"):
            srv.submit_many(bad)
        assert srv.stats()["submitted"] == before
