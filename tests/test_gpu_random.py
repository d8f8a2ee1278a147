"""Seeded randomized parity: random grids (z-order squares, odd row-major
rectangles, time-augmented volumes), random rows (empty, runs, scattered sets),
every proposition count at a word boundary, optional random monitors; every
labeling form and depth, and both frame transforms (byte gathers, packed
words), against the oracle bit for bit.  Time-augmented frames use worlds of
two or more slabs; a 2-D world under a time-augmented agent grid is the
static-world case of test_gpu_3d."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_02612_gb300 as L  # noqa: E402

FLAGS = L.LBL_UPLOAD_BITTILE | L.LBL_UPLOAD_SECTOR | L.LBL_UPLOAD_QUAD | L.LBL_UPLOAD_MMA
FORMS = [dict(algo=L.LBL_ALGO_CSR), dict(algo=L.LBL_ALGO_CSR, lanes_per_edge=8, early_exit=1),
         dict(algo=L.LBL_ALGO_CSR, pipeline=L.LBL_PIPE_BULK), dict(algo=L.LBL_ALGO_CSR, pipeline=L.LBL_PIPE_ASYNC),
         dict(algo=L.LBL_ALGO_BITTILE), dict(algo=L.LBL_ALGO_SECTOR), dict(algo=L.LBL_ALGO_QUAD),
         dict(algo=L.LBL_ALGO_QUAD, depth=8), dict(algo=L.LBL_ALGO_QUAD, depth=16),
         dict(algo=L.LBL_ALGO_QUAD, pipeline=L.LBL_PIPE_FRONT), dict(algo=L.LBL_ALGO_MMA),
         dict(algo=L.LBL_ALGO_AUTO)]
PROPS = [0, 1, 2, 5, 8, 9, 16, 17, 31, 32, 33, 63, 64]


def _case(rng):
    kind = int(rng.integers(0, 3))
    if kind == 0:
        agent = synth.agent_grid(int(2 ** rng.integers(2, 10)), 0.25, synth.MORTON)
    elif kind == 1:
        agent = synth.Grid(int(rng.integers(1, 700)), int(rng.integers(1, 300)), 0.3, 0.0, 0.0, synth.ROWMAJOR)
    else:
        n = int(2 ** rng.integers(2, 6))
        agent = synth.agent_grid3(n, 0.4, n, 0.05, int(rng.integers(0, 2)))
    cells = agent.cells
    rows = []
    for _ in range(int(rng.integers(0, 3000))):
        r = rng.random()
        if r < 0.1:
            rows.append(np.zeros(0, np.int64))
        elif r < 0.5:
            a = int(rng.integers(0, cells))
            rows.append(np.arange(a, a + int(rng.integers(1, min(cells - a, 600) + 1))))
        else:
            rows.append(np.sort(rng.choice(cells, size=int(rng.integers(1, min(cells, 400) + 1)), replace=False)))
    E = len(rows)
    rowptr = np.zeros(E + 1, np.int64)
    if E:
        rowptr[1:] = np.cumsum([len(r) for r in rows])
    colidx = np.concatenate(rows).astype(np.int32) if E and rowptr[-1] else np.zeros(0, np.int32)
    P = int(rng.choice(PROPS))
    O = rng.integers(0, 2**63, size=cells, dtype=np.uint64)
    O[rng.random(cells) < 0.7] = 0
    return agent, rowptr, colidx, P, O


@pytest.mark.parametrize("seed", range(4))
def test_random_roadmaps_every_form(seed):
    rng = np.random.default_rng(900 + seed)
    for _ in range(12):
        agent, rowptr, colidx, P, O_h = _case(rng)
        E = rowptr.shape[0] - 1
        mon = (synth.random_monitor(rng, int(rng.integers(2, 17)), int(rng.integers(0, min(8, max(P, 1)) + 1)),
                                    max(P, 1)) if rng.random() < 0.5 else None)
        rm = L.lbl_roadmap_upload(agent, rowptr, colidx, flags=FLAGS)
        mh = L.lbl_monitor_create(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject) if mon else None
        try:
            O = torch.from_numpy(O_h).cuda()
            want = oracle.label(rowptr, colidx, O_h, P)
            if mon:
                wn, wv = oracle.monitor(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject, want)
            for cfg in FORMS:
                out = torch.full((max(E, 1),), 0x77, dtype=torch.int64, device="cuda").view(torch.uint64)[:E]
                nx = torch.empty(max(E, 1), dtype=torch.uint64, device="cuda")[:E] if mon else None
                vi = torch.empty(max(E, 1), dtype=torch.uint16, device="cuda")[:E] if mon else None
                L.lbl_label(rm, O, P, out, mh, nx, vi, cfg)
                torch.cuda.synchronize()
                assert np.array_equal(out.cpu().numpy(), want), (agent, E, P, cfg)
                if mon:
                    assert np.array_equal(nx.cpu().numpy(), wn), (agent, E, P, cfg)
                    assert np.array_equal(vi.cpu().numpy(), wv), (agent, E, P, cfg)
            L.lbl_roadmap_status(rm)
        finally:
            if mh:
                L.lbl_monitor_free(mh)
            L.lbl_roadmap_free(rm)


@pytest.mark.parametrize("seed", range(3))
def test_random_frames_both_transforms(seed):
    rng = np.random.default_rng(950 + seed)
    for _ in range(10):
        if rng.random() < 0.3:
            n = int(2 ** rng.integers(2, 5))
            world = synth.Grid(int(rng.integers(1, 40)), int(rng.integers(1, 40)), float(rng.uniform(0.1, 0.5)),
                               float(rng.uniform(-3, 3)), float(rng.uniform(-3, 3)), synth.ROWMAJOR,
                               int(rng.integers(2, 9)), float(rng.uniform(0.02, 0.2)), float(rng.uniform(-0.2, 0.2)))
            agent = synth.agent_grid3(n, float(rng.uniform(0.1, 0.6)), n, float(rng.uniform(0.02, 0.2)),
                                      int(rng.integers(0, 2)))
            pose = (float(rng.uniform(-2, 8)), float(rng.uniform(-2, 8)), float(rng.uniform(-7, 7)),
                    float(rng.uniform(-0.3, 0.5)))
            shape = (world.d, world.h, world.w)
        else:
            world = synth.Grid(int(rng.integers(1, 300)), int(rng.integers(1, 300)), float(rng.uniform(0.1, 0.5)),
                               float(rng.uniform(-5, 5)), float(rng.uniform(-5, 5)), synth.ROWMAJOR)
            agent = (synth.agent_grid(int(2 ** rng.integers(2, 8)), float(rng.uniform(0.1, 0.6)), synth.MORTON)
                     if rng.random() < 0.5 else
                     synth.Grid(int(rng.integers(1, 200)), int(rng.integers(1, 200)), float(rng.uniform(0.1, 0.6)),
                                float(rng.uniform(-20, 0)), float(rng.uniform(-20, 0)), synth.ROWMAJOR))
            pose = (float(rng.uniform(-5, 60)), float(rng.uniform(-5, 60)), float(rng.uniform(-7, 7)))
            shape = (world.h, world.w)
        P = int(rng.choice(PROPS))
        planes = ((rng.random((P,) + shape) < rng.uniform(0.02, 0.9)).astype(np.uint8)
                  * rng.integers(1, 256, size=(P,) + shape).astype(np.uint8))
        want = (oracle.frame_transform3(world, planes, pose, agent) if len(shape) == 3
                else oracle.frame_transform(world, planes, pose, agent))
        d_planes = torch.from_numpy(planes.reshape(-1)).cuda() if P else torch.empty(1, dtype=torch.uint8,
                                                                                        device="cuda")
        O = torch.empty(agent.cells, dtype=torch.uint64, device="cuda")
        L.lbl_frame_transform(world, d_planes, P, pose, agent, O)
        torch.cuda.synchronize()
        assert np.array_equal(O.cpu().numpy(), want), (world, agent, P, pose)
        words = torch.empty(world.cells, dtype=getattr(torch, L.packed_word_dtype(P)), device="cuda")
        O2 = torch.empty(agent.cells, dtype=torch.uint64, device="cuda")
        L.lbl_pack_planes(world, d_planes, P, words)
        L.lbl_frame_transform_words(world, words, P, pose, agent, O2)
        torch.cuda.synchronize()
        assert np.array_equal(O2.cpu().numpy(), want), (world, agent, P, pose)


def test_grids_past_32768_a_side_are_rejected():
    """Grids have at most 32768 cells a side (and slabs) and fewer than 2^31
    cells, which keeps every transform index 32-bit; larger grids are refused
    before any device work."""
    buf = torch.zeros(64, dtype=torch.uint64, device="cuda")
    small = synth.world_grid(4, 4, 0.3)
    for agent in (synth.Grid(3, 40_000, 0.01, 0.0, 0.0, synth.ROWMAJOR),
                  synth.Grid(2, 3, 0.4, -0.4, -0.6, synth.ROWMAJOR, 40_000, 0.001, 0.0)):
        with pytest.raises(L.LblError):
            L.lbl_frame_transform(small, buf.view(torch.uint8), 1, (0.0, 0.0, 0.0, 0.0), agent, buf)
    with pytest.raises(L.LblError):
        L.lbl_pack_planes(synth.world_grid(40_000, 2, 0.3), buf.view(torch.uint8), 1, buf.view(torch.uint8))
