"""Serving loop with continuous batching: every request's outputs are the same
in a busy mix as alone (lbl_session_run) and as the oracle's; admission waits
for memory; requests that can never fit are refused."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_02612_gb300 as L  # noqa: E402


@pytest.fixture(scope="module")
def resident():
    rng = np.random.default_rng(12)
    wls = [synth.make("plain", seed=21), synth.make("driving", seed=22, edges=15_000),
           synth.make("paper", seed=23, edges=20_000)]
    mons = [synth.random_monitor(rng, 5, 3, wls[0].P), None, None]
    flags = [L.LBL_UPLOAD_QUAD, 0, L.LBL_UPLOAD_QUAD]  # quadtree and CSR residents in one server
    rms = [L.lbl_roadmap_upload(w.agent, w.rowptr, w.colidx, flags=f) for w, f in zip(wls, flags)]
    mhs = [L.lbl_monitor_create(m.n_states, m.m, m.relbits, m.delta, m.reject) if m else None for m in mons]
    yield wls, mons, rms, mhs
    for m in mhs:
        if m:
            L.lbl_monitor_free(m)
    for r in rms:
        L.lbl_roadmap_free(r)


def _alone(wl, rm, mh, planes, pose):
    ss = L.lbl_session_create(rm, wl.world, wl.P, mh)
    try:
        out = torch.empty(wl.n_edges, dtype=torch.uint64).pin_memory()
        nxt = torch.empty(wl.n_edges, dtype=torch.uint64).pin_memory() if mh else None
        viol = torch.empty(wl.n_edges, dtype=torch.uint16).pin_memory() if mh else None
        L.lbl_session_run(ss, planes, pose, out, nxt, viol)
        torch.cuda.synchronize()
        return out.numpy().copy(), (nxt.numpy().copy() if mh else None), (viol.numpy().copy() if mh else None)
    finally:
        L.lbl_session_free(ss)


def test_results_in_the_mix_equal_results_alone(resident):
    """60 requests submitted back to back (every buffer made beforehand), so
    that most arrive while earlier batches are on the device: the server must
    put several requests into one batch (max_batch >= 2, fewer batches than
    requests), and every request's labels and monitor outputs equal the same
    request run alone and the oracle's."""
    wls, mons, rms, mhs = resident
    rng = np.random.default_rng(3)
    prepared = []
    for i in range(60):
        k = int(rng.integers(0, 3))
        wl = wls[k]
        planes = torch.from_numpy(wl.planes).pin_memory()
        pose = synth.random_pose(rng, wl.world)
        out = torch.zeros(wl.n_edges, dtype=torch.uint64).pin_memory()
        nxt = torch.zeros(wl.n_edges, dtype=torch.uint64).pin_memory() if mhs[k] else None
        viol = torch.zeros(wl.n_edges, dtype=torch.uint16).pin_memory() if mhs[k] else None
        prepared.append((k, planes, pose, out, nxt, viol))
    srv = L.lbl_server_create(rms, [w.P for w in wls], mhs, lanes=2, mem_budget=512 << 20)
    reqs = []
    try:
        for k, planes, pose, out, nxt, viol in prepared:
            reqs.append((L.lbl_server_submit(srv, k, wls[k].world, planes, pose, out, nxt, viol),) + (k, planes, pose,
                                                                                                      out, nxt, viol))
        lats = [L.lbl_server_wait(srv, r[0], 20000) for r in reqs]
        assert all(x > 0 for x in lats)
        st = L.lbl_server_stats(srv)
        assert st["completed"] == 60 and st["arena_used"] == 0
        assert st["max_batch"] >= 2 and st["batches"] < st["completed"], st  # requests were batched together
        for j, (t, k, planes, pose, out, nxt, viol) in enumerate(reqs):
            wl, rm, mh, m = wls[k], rms[k], mhs[k], mons[k]
            aL, aN, aV = _alone(wl, rm, mh, planes, pose)
            assert np.array_equal(out.numpy(), aL), j
            if mh:
                assert np.array_equal(nxt.numpy(), aN) and np.array_equal(viol.numpy(), aV), j
            O = oracle.frame_transform(wl.world, wl.planes, pose, wl.agent)
            want = oracle.label(wl.rowptr, wl.colidx, O, wl.P, threads=8)
            assert np.array_equal(out.numpy(), want), j
            if mh:
                wn, wv = oracle.monitor(m.n_states, m.m, m.relbits, m.delta, m.reject, want)
                assert np.array_equal(nxt.numpy(), wn) and np.array_equal(viol.numpy(), wv), j
    finally:
        L.lbl_server_free(srv)


def test_admission_waits_for_memory_and_refuses_oversize(resident):
    wls, mons, rms, mhs = resident
    wl = wls[1]  # driving: 32 x 256^2 planes + 256^2 words + labels ~ 2.7 MB per request
    srv = L.lbl_server_create([rms[1]], [wl.P], None, lanes=2, mem_budget=6 << 20)  # room for two
    try:
        rng = np.random.default_rng(9)
        planes = torch.from_numpy(wl.planes).pin_memory()
        outs, ts = [], []
        for i in range(12):
            out = torch.zeros(wl.n_edges, dtype=torch.uint64).pin_memory()
            ts.append(L.lbl_server_submit(srv, 0, wl.world, planes, synth.random_pose(rng, wl.world), out))
            outs.append(out)
        for t in ts:
            L.lbl_server_wait(srv, t, 20000)
        st = L.lbl_server_stats(srv)
        assert st["completed"] == 12 and st["max_batch"] <= 2 and st["arena_used"] == 0
        big = synth.world_grid(4096, 4096, 0.25)  # 32 x 16M planes: more than the budget
        with pytest.raises(L.LblError) as ei:
            L.lbl_server_submit(srv, 0, big, planes, wl.pose, outs[0])
        assert ei.value.code == L.LBL_ENOMEM
        with pytest.raises(L.LblError):
            L.lbl_server_wait(srv, 10**9, 10)
    finally:
        L.lbl_server_free(srv)


def test_wait_is_bounded_and_reports_timeout(resident):
    """A wait that runs out returns LBL_ETIMEOUT and leaves the ticket valid: a
    later wait on it succeeds.  The arena holds one request at a time, so the
    last of eight requests is still queued behind seven when it is first waited
    on with a zero limit."""
    wls, mons, rms, mhs = resident
    wl = wls[1]
    srv = L.lbl_server_create([rms[1]], [wl.P], None, lanes=1, mem_budget=3 << 20)
    try:
        rng = np.random.default_rng(4)
        planes = torch.from_numpy(wl.planes).pin_memory()
        outs, ts = [], []
        for i in range(8):
            out = torch.zeros(wl.n_edges, dtype=torch.uint64).pin_memory()
            ts.append(L.lbl_server_submit(srv, 0, wl.world, planes, synth.random_pose(rng, wl.world), out))
            outs.append(out)
        with pytest.raises(L.LblError) as ei:
            L.lbl_server_wait(srv, ts[-1], 0)
        assert ei.value.code == L.LBL_ETIMEOUT
        for t in ts:
            assert L.lbl_server_wait(srv, t, 20000) > 0
        assert L.lbl_server_stats(srv)["completed"] == 8
    finally:
        L.lbl_server_free(srv)
