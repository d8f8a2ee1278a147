"""Time-augmented (x, y, tau) workspace on the GPU: the 3-D frame transform and
every labeling form equal the oracle bit for bit; a 2-D world under a 3-D agent
grid is a static world; batches mix 2-D and 3-D frames."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_02612_gb300 as L  # noqa: E402


@pytest.fixture(scope="module")
def p3():
    return synth.make_paper3d(seed=2, edges=30_000)


def _O(world, vols, pose, agent):
    O = torch.empty(agent.cells, dtype=torch.uint64, device="cuda")
    L.lbl_frame_transform(world, torch.from_numpy(np.ascontiguousarray(vols)).cuda(), vols.shape[0], pose, agent, O)
    torch.cuda.synchronize()
    return O


@pytest.mark.parametrize("order", [synth.MORTON, synth.ROWMAJOR])
def test_frame_transform3_matches_oracle(p3, order):
    wl = p3
    agent = synth.agent_grid3(wl.agent.w, wl.agent.res, wl.agent.d, wl.agent.tres, order)
    rng = np.random.default_rng(4)
    for T in (0.0, 0.05 * 7, -0.35, 0.123, 100.0):
        pose = synth.random_pose(rng, wl.world) + (T,)
        got = _O(wl.world, wl.planes, pose, agent).cpu().numpy()
        assert np.array_equal(got, oracle.frame_transform3(wl.world, wl.planes, pose, agent)), T


def test_frame_transform3_odd_world_and_static_world():
    rng = np.random.default_rng(6)
    world = synth.Grid(40, 33, 0.3, -1.0, 2.0, synth.ROWMAJOR, 19, 0.07, -0.2)
    vols = (rng.random((5, 19, 33, 40)) < 0.3).astype(np.uint8)
    agent = synth.agent_grid3(16, 0.25, 16, 0.05, synth.MORTON)
    pose = (5.0, 7.0, 1.1, 0.31)
    assert np.array_equal(_O(world, vols, pose, agent).cpu().numpy(),
                          oracle.frame_transform3(world, vols, pose, agent))
    # a 2-D world under the 3-D agent grid: every slab reads the same plane
    world2 = synth.world_grid(40, 33, 0.3)
    planes = (rng.random((5, 33, 40)) < 0.3).astype(np.uint8)
    world2r = synth.Grid(40, 33, 0.3, 0.0, 0.0, synth.ROWMAJOR, 1, 1.0, 0.0)
    static = synth.Grid(40, 33, 0.3, 0.0, 0.0, synth.ROWMAJOR, agent.d, agent.tres, 0.0)
    want = oracle.frame_transform3(static, np.repeat(planes[:, None], agent.d, axis=1), (5.0, 7.0, 1.1, 0.0), agent)
    assert np.array_equal(_O(world2r, planes, pose, agent).cpu().numpy(), want)
    # a time-augmented world needs a time-augmented agent grid
    with pytest.raises(L.LblError):
        _O(world, vols, pose, synth.agent_grid(16, 0.25, synth.MORTON))
    assert world2.d == 1


def test_labels3_all_forms_match_oracle(p3):
    wl = p3
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx,
                              flags=L.LBL_UPLOAD_BITTILE | L.LBL_UPLOAD_SECTOR | L.LBL_UPLOAD_QUAD | L.LBL_UPLOAD_MMA)
    try:
        O = _O(wl.world, wl.planes, wl.pose, wl.agent)
        want = oracle.label(wl.rowptr, wl.colidx, O.cpu().numpy(), wl.P, threads=8)
        assert (want != 0).any()
        for cfg in (dict(algo=L.LBL_ALGO_CSR), dict(algo=L.LBL_ALGO_CSR, lanes_per_edge=16),
                    dict(algo=L.LBL_ALGO_BITTILE), dict(algo=L.LBL_ALGO_SECTOR), dict(algo=L.LBL_ALGO_QUAD),
                    dict(algo=L.LBL_ALGO_CSR, pipeline=L.LBL_PIPE_BULK), dict(algo=L.LBL_ALGO_MMA)):
            out = torch.empty(wl.n_edges, dtype=torch.uint64, device="cuda")
            L.lbl_label(rm, O, wl.P, out, cfg=cfg)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), want), cfg
    finally:
        L.lbl_roadmap_free(rm)


def test_batch_mixes_2d_and_3d_frames(p3):
    w2 = synth.make("driving", seed=9, edges=4000)
    items = [(p3, p3.pose), (w2, w2.pose), (p3, p3.pose[:3] + (0.4,))]
    rms = [L.lbl_roadmap_upload(w.agent, w.rowptr, w.colidx) for w, _ in items]
    b = L.lbl_batch_create(rms, [w.P for w, _ in items])
    try:
        frames = []
        for w, pose in items:
            frames.append(dict(world=w.world, d_planes=torch.from_numpy(w.planes).cuda(), pose=pose,
                               d_O=torch.zeros(w.agent.cells, dtype=torch.uint64, device="cuda"),
                               d_L=torch.zeros(w.n_edges, dtype=torch.uint64, device="cuda")))
        L.lbl_batch_set_frames(b, frames)
        L.lbl_batch_launch(b)
        torch.cuda.synchronize()
        for (w, pose), f in zip(items, frames):
            O = (oracle.frame_transform3(w.world, w.planes, pose, w.agent) if w.agent.d > 1
                 else oracle.frame_transform(w.world, w.planes, pose, w.agent))
            assert np.array_equal(f["d_O"].cpu().numpy(), O)
            assert np.array_equal(f["d_L"].cpu().numpy(), oracle.label(w.rowptr, w.colidx, O, w.P, threads=8))
    finally:
        L.lbl_batch_free(b)
        for r in rms:
            L.lbl_roadmap_free(r)
    assert math.isfinite(p3.pose[0])
