"""GPU parity: every CUDA result equals the oracle bit for bit (integer and
bitwise work, so the tolerance is zero).  Inputs are seeded synthetic
workloads; every call goes through the C ABI."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_02612_gb300 as L  # noqa: E402
from paper_1810_02612_gb300.lbl import lbl_grid  # noqa: E402


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def empty_u64(n):
    return torch.empty(max(n, 1), dtype=torch.uint64, device="cuda")[:n]


def empty_u16(n):
    return torch.empty(max(n, 1), dtype=torch.uint16, device="cuda")[:n]


class Roadmap:
    def __init__(self, agent, rowptr, colidx, bittile=False):
        self.E = rowptr.shape[0] - 1
        every_form = L.LBL_UPLOAD_BITTILE | L.LBL_UPLOAD_SECTOR | L.LBL_UPLOAD_QUAD | L.LBL_UPLOAD_MMA
        self.h = L.lbl_roadmap_upload(agent, rowptr, colidx, flags=every_form if bittile else 0)

    def __del__(self):
        if getattr(self, "h", None):
            L.lbl_roadmap_free(self.h)


def gpu_O(wl, pose=None, planes=None):
    planes = wl.planes if planes is None else planes
    O = empty_u64(wl.agent.cells)
    L.lbl_frame_transform(wl.world, cuda(planes), planes.shape[0], wl.pose if pose is None else pose, wl.agent, O)
    return O


def gpu_label(rm, O, P, cfg=None, mon=None):
    out = empty_u64(rm.E)
    nxt = empty_u64(rm.E) if mon else None
    viol = empty_u16(rm.E) if mon else None
    L.lbl_label(rm.h, O, P, out, mon, nxt, viol, cfg)
    if mon:
        return host(out), host(nxt), host(viol)
    return host(out)


CFGS = [
    dict(algo=L.LBL_ALGO_CSR),                   # streaming form, default partition
    dict(algo=L.LBL_ALGO_CSR, ctas_per_sm=1),    # streaming form, re-partitioned
    dict(algo=L.LBL_ALGO_CSR, ctas_per_sm=2, pipeline=L.LBL_PIPE_BULK),
    dict(algo=L.LBL_ALGO_CSR, pipeline=L.LBL_PIPE_BULK),
    dict(algo=L.LBL_ALGO_CSR, pipeline=L.LBL_PIPE_ASYNC),
    dict(algo=L.LBL_ALGO_CSR, ctas_per_sm=3, pipeline=L.LBL_PIPE_ASYNC),
    dict(algo=L.LBL_ALGO_CSR, lanes_per_edge=4, early_exit=0),
    dict(algo=L.LBL_ALGO_CSR, lanes_per_edge=8, early_exit=0),
    dict(algo=L.LBL_ALGO_CSR, lanes_per_edge=16, early_exit=1),
    dict(algo=L.LBL_ALGO_CSR, lanes_per_edge=32, early_exit=0),
    dict(algo=L.LBL_ALGO_CSR, lanes_per_edge=32, early_exit=1),
    dict(algo=L.LBL_ALGO_BITTILE, early_exit=0),
    dict(algo=L.LBL_ALGO_SECTOR),
    dict(algo=L.LBL_ALGO_SECTOR, depth=8),
    dict(algo=L.LBL_ALGO_CSR, depth=12),
    dict(algo=L.LBL_ALGO_CSR, depth=16),
    dict(algo=L.LBL_ALGO_BITTILE, early_exit=1),
    dict(algo=L.LBL_ALGO_QUAD),
    dict(algo=L.LBL_ALGO_QUAD, depth=12),
    dict(algo=L.LBL_ALGO_QUAD, depth=16),
    dict(algo=L.LBL_ALGO_QUAD, ctas_per_sm=1),
    dict(algo=L.LBL_ALGO_QUAD, pipeline=L.LBL_PIPE_FRONT),      # moving front, whatever the size
    dict(algo=L.LBL_ALGO_QUAD, pipeline=L.LBL_PIPE_REGISTERS),  # fixed per-warp ranges
    dict(algo=L.LBL_ALGO_MMA),                                  # tensor cores
    dict(algo=L.LBL_ALGO_AUTO),
]


@pytest.fixture(scope="module")
def plain():
    return synth.make("plain", seed=3)


@pytest.fixture(scope="module")
def driving_small():
    return synth.make("driving", seed=4, edges=20_000)


@pytest.fixture(scope="module")
def large_small():
    return synth.make("large", seed=5, edges=30_000)


@pytest.fixture(scope="module")
def paper_small():
    return synth.make("paper", seed=6, edges=40_000)


# ------------------------------------------------------------ frame transform

@pytest.mark.parametrize("name", ["plain", "driving_small", "large_small", "paper_small"])
def test_frame_transform_matches_oracle(name, request):
    wl = request.getfixturevalue(name)
    rng = np.random.default_rng(1)
    poses = [wl.pose, synth.random_pose(rng, wl.world), (wl.pose[0], wl.pose[1], math.pi / 2),
             (wl.pose[0] + 3.3, wl.pose[1] - 7.1, -2.5), (-50.0, 10.0, 0.7)]  # last: mostly off the world
    for pose in poses:
        got = host(gpu_O(wl, pose=pose))
        want = oracle.frame_transform(wl.world, wl.planes, pose, wl.agent)
        assert np.array_equal(got, want), pose


@pytest.mark.parametrize("P", [0, 1, 7, 8, 9, 63, 64])
def test_frame_transform_prop_counts_and_odd_grids(P):
    rng = np.random.default_rng(P)
    world = synth.world_grid(53, 41, 0.37)
    planes = (rng.random((P, 41, 53)) < 0.3).astype(np.uint8) * rng.integers(1, 255, size=(P, 41, 53)).astype(np.uint8)
    for agent in (synth.agent_grid(32, 0.25, synth.MORTON), synth.Grid(37, 29, 0.3, -5.0, -4.0, synth.ROWMAJOR)):
        pose = (9.0 + rng.random(), 7.5 + rng.random(), rng.random() * 6.3)
        O = empty_u64(agent.cells)
        L.lbl_frame_transform(world, cuda(planes) if P else torch.empty(1, dtype=torch.uint8, device="cuda"), P,
                              pose, agent, O)
        assert np.array_equal(host(O), oracle.frame_transform(world, planes, pose, agent))


def _packed(planes):
    P = planes.shape[0]
    flat = planes.reshape(P, int(np.prod(planes.shape[1:])))
    w = np.zeros(flat.shape[1], np.uint64)
    for p in range(P):
        w |= (flat[p] != 0).astype(np.uint64) << np.uint64(p)
    return w


def _words_buf(cells, P, fill=0x55):
    """a packed-word buffer of the width lbl_pack_planes writes, every byte `fill`"""
    dt = getattr(torch, L.packed_word_dtype(P))
    return torch.full((cells * L.packed_word_bytes(P),), fill, dtype=torch.uint8, device="cuda").view(dt)


def _words_host(words):
    w = words.cpu().numpy()
    return w.view({1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}[w.itemsize]).astype(np.uint64)


@pytest.mark.parametrize("P", [0, 1, 2, 7, 8, 9, 16, 17, 31, 32, 33, 63, 64])
def test_pack_planes_and_packed_transform(P):
    """Packed words (as narrow as P allows) equal the plain definition for
    4-byte aligned and unaligned planes, cell counts divisible by 4 or not, and
    words at and off their vector alignment; the packed transform equals the
    oracle's."""
    rng = np.random.default_rng(70 + P)
    wb = L.packed_word_bytes(P)
    for world, misalign, woff in ((synth.world_grid(53, 41, 0.37), 0, 0), (synth.world_grid(64, 48, 0.37), 0, 0),
                                  (synth.world_grid(64, 48, 0.37), 1, 0), (synth.world_grid(64, 48, 0.37), 0, 1),
                                  (synth.world_grid(3, 1, 0.37), 0, 0), (synth.world_grid(1, 1, 0.37), 0, 0)):
        cells = world.cells
        planes = (rng.random((P, world.h, world.w)) < 0.3).astype(np.uint8) * rng.integers(
            1, 255, size=(P, world.h, world.w)).astype(np.uint8)
        buf = torch.zeros(P * cells + 8, dtype=torch.uint8, device="cuda")
        d_planes = buf[misalign:misalign + P * cells]
        d_planes.copy_(torch.from_numpy(planes.reshape(-1)).cuda())
        words = _words_buf(cells + 1, P)[woff:woff + cells]  # woff = 1: one word past a 16-byte boundary
        L.lbl_pack_planes(world, d_planes, P, words)
        torch.cuda.synchronize()
        assert np.array_equal(_words_host(words), _packed(planes)), (world.w, misalign, woff)
        for agent in (synth.agent_grid(32, 0.25, synth.MORTON), synth.Grid(37, 29, 0.3, -5.0, -4.0, synth.ROWMAJOR)):
            pose = (9.0 + rng.random(), 7.5 + rng.random(), rng.random() * 6.3)
            O = empty_u64(agent.cells)
            L.lbl_frame_transform_words(world, words, P, pose, agent, O)
            assert np.array_equal(host(O), oracle.frame_transform(world, planes, pose, agent))
    assert wb == (1 if P <= 8 else 2 if P <= 16 else 4 if P <= 32 else 8)


def test_pack_planes_all_byte_values():
    """every byte value 0..255 in every plane position packs to (value != 0)"""
    world = synth.world_grid(256, 4, 1.0)
    for P in (8, 64):
        planes = np.zeros((P, 4, 256), np.uint8)
        for p in range(P):
            planes[p] = np.roll(np.arange(256, dtype=np.uint8), 7 * p)[None, :]
        words = _words_buf(world.cells, P)
        L.lbl_pack_planes(world, cuda(planes), P, words)
        torch.cuda.synchronize()
        assert np.array_equal(_words_host(words), _packed(planes))


def test_packed_words_must_match_width():
    world = synth.world_grid(8, 8, 1.0)
    planes = torch.zeros(9 * 64, dtype=torch.uint8, device="cuda")
    with pytest.raises(TypeError):
        L.lbl_pack_planes(world, planes, 9, empty_u64(64))  # 9 propositions pack into 16-bit words
    words = torch.zeros(2 * 64 + 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LblError):  # a raw pointer one byte past a 16-bit boundary
        L.lbl_pack_planes(world, planes, 9, words.data_ptr() + 1)
    with pytest.raises(L.LblError):
        L.lbl_frame_transform_words(world, words.data_ptr() + 1, 9, (1.0, 1.0, 0.0), world, empty_u64(64))


def test_packed_transform_time_augmented():
    rng = np.random.default_rng(77)
    world = synth.Grid(20, 17, 0.3, 0.0, 0.0, synth.ROWMAJOR, 12, 0.07, -0.1)
    agent = synth.agent_grid3(8, 0.25, 8, 0.05, synth.MORTON)
    for P in (5, 40):
        vols = (rng.random((P, 12, 17, 20)) < 0.5).astype(np.uint8)
        words = _words_buf(world.cells, P)
        L.lbl_pack_planes(world, cuda(vols), P, words)
        torch.cuda.synchronize()
        assert np.array_equal(_words_host(words), _packed(vols))
        for _ in range(3):
            pose = (2 + 2 * rng.random(), 2 + 2 * rng.random(), 6.3 * rng.random(), 0.3 * rng.random() - 0.1)
            O = empty_u64(agent.cells)
            L.lbl_frame_transform_words(world, words, P, pose, agent, O)
            assert np.array_equal(host(O), oracle.frame_transform3(world, vols, pose, agent))


def test_frame_transform_rejects_out_of_range_pose():
    world = synth.world_grid(8, 8, 1.0)
    agent = synth.agent_grid(8, 1.0, synth.MORTON)
    O = empty_u64(64)
    with pytest.raises(L.LblError) as ei:
        L.lbl_frame_transform(world, cuda(np.zeros((1, 8, 8), np.uint8)), 1, (1e12, 0.0, 0.0), agent, O)
    assert ei.value.code == L.LBL_EINVAL
    with pytest.raises(L.LblError):
        L.lbl_frame_transform(world, cuda(np.zeros((1, 8, 8), np.uint8)), 65, (0.0, 0.0, 0.0), agent, O)


# ---------------------------------------------------------------- labeling

@pytest.mark.parametrize("name", ["plain", "driving_small", "large_small", "paper_small"])
def test_label_all_algorithms_match_oracle(name, request):
    wl = request.getfixturevalue(name)
    rm = Roadmap(wl.agent, wl.rowptr, wl.colidx, bittile=True)
    O = gpu_O(wl)
    O_h = host(O)
    want = oracle.label(wl.rowptr, wl.colidx, O_h, wl.P, threads=8)
    for cfg in CFGS:
        assert np.array_equal(gpu_label(rm, O, wl.P, cfg), want), cfg
    assert np.array_equal(gpu_label(rm, O, wl.P, None), want)
    L.lbl_roadmap_status(rm.h)  # no kernel gave up a bounded wait


def test_label_with_fused_monitor_matches_oracle(large_small):
    wl = large_small
    rm = Roadmap(wl.agent, wl.rowptr, wl.colidx, bittile=True)
    mon = wl.monitor
    h = L.lbl_monitor_create(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject)
    try:
        O = gpu_O(wl)
        want_L = oracle.label(wl.rowptr, wl.colidx, host(O), wl.P, threads=8)
        want_n, want_v = oracle.monitor(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject, want_L)
        # the reject sink always rejects (bit 15); the other states must vary
        assert len(np.unique(want_v)) > 4
        for cfg in CFGS:
            got_L, got_n, got_v = gpu_label(rm, O, wl.P, cfg, mon=h)
            assert np.array_equal(got_L, want_L), cfg
            assert np.array_equal(got_n, want_n), cfg
            assert np.array_equal(got_v, want_v), cfg
    finally:
        L.lbl_monitor_free(h)


def _hand_csr(rng, lengths, n_cells):
    rowptr = np.zeros(len(lengths) + 1, np.int64)
    cols = []
    for i, k in enumerate(lengths):
        c = np.sort(rng.choice(n_cells, size=k, replace=False)).astype(np.int32)
        cols.append(c)
        rowptr[i + 1] = rowptr[i] + k
    colidx = np.concatenate(cols) if cols else np.zeros(0, np.int32)
    return rowptr, colidx


@pytest.mark.parametrize("P", [1, 2, 5, 33, 64])
def test_label_ragged_rows_and_alignments(P):
    """Rows of length 0..4097 starting at every offset modulo 4, including
    the first and last cell of the grid."""
    rng = np.random.default_rng(40 + P)
    agent = synth.Grid(101, 83, 0.5, 0.0, 0.0, synth.ROWMAJOR)  # cells not a multiple of 64
    lengths = [0, 1, 2, 3, 4, 5, 0, 0, 7, 31, 32, 33, 127, 128, 129, 1, 255, 256, 257, 511, 512, 513, 1023,
               1024, 1025, 4095, 4096, 4097, 3, 0]
    lengths += list(rng.integers(0, 300, size=300))
    rowptr, colidx = _hand_csr(rng, lengths, agent.cells)
    colidx[rowptr[1]] = 0 if lengths[1] else colidx[rowptr[1]]
    colidx[rowptr[26]:rowptr[27]][-1] = agent.cells - 1
    colidx[rowptr[26]:rowptr[27]].sort()
    O_h = np.zeros(agent.cells, np.uint64)
    sparse = rng.random(agent.cells) < 0.002
    O_h[sparse] = rng.integers(0, 2**63, size=sparse.sum(), dtype=np.uint64) | np.uint64(1 << 63)
    O_h[0] = np.uint64(1)
    O_h[agent.cells - 1] = np.uint64(1 << (P - 1))
    rm = Roadmap(agent, rowptr, colidx, bittile=True)
    want = oracle.label(rowptr, colidx, O_h, P)
    O = cuda(O_h)
    for cfg in CFGS:
        assert np.array_equal(gpu_label(rm, O, P, cfg), want), cfg


def test_label_mostly_empty_rows():
    """Long runs of empty rows between short ones, and a roadmap whose rows
    are all empty: every edge still gets its (possibly zero) label."""
    rng = np.random.default_rng(77)
    agent = synth.agent_grid(64, 0.5, synth.MORTON)
    lengths = np.where(rng.random(20_000) < 0.03, rng.integers(1, 200, size=20_000), 0)
    lengths[-500:] = 0
    rowptr, colidx = _hand_csr(rng, list(lengths), agent.cells)
    O_h = rng.integers(0, 2**63, size=agent.cells, dtype=np.uint64)
    rm = Roadmap(agent, rowptr, colidx, bittile=True)
    want = oracle.label(rowptr, colidx, O_h, 64)
    for cfg in CFGS:
        assert np.array_equal(gpu_label(rm, cuda(O_h), 64, cfg), want), cfg
    rm0 = Roadmap(agent, np.zeros(1001, np.int64), np.zeros(0, np.int32), bittile=True)
    for cfg in CFGS:
        assert (gpu_label(rm0, cuda(O_h), 64, cfg) == 0).all(), cfg


def test_label_full_and_empty_occupancy(plain):
    wl = plain
    rm = Roadmap(wl.agent, wl.rowptr, wl.colidx, bittile=True)
    nonempty = np.diff(wl.rowptr) > 0
    for P in (1, 4, 64):
        full = cuda(np.full(wl.agent.cells, np.uint64(2**64 - 1), np.uint64))
        zero = cuda(np.zeros(wl.agent.cells, np.uint64))
        m = np.uint64(2**P - 1) if P < 64 else np.uint64(2**64 - 1)
        for cfg in CFGS:
            got = gpu_label(rm, full, P, cfg)
            assert np.array_equal(got[nonempty], np.full(nonempty.sum(), m)) and (got[~nonempty] == 0).all()
            assert (gpu_label(rm, zero, P, cfg) == 0).all()


def test_label_zero_edges_and_zero_props():
    agent = synth.agent_grid(8, 1.0, synth.MORTON)
    rm = Roadmap(agent, np.zeros(1, np.int64), np.zeros(0, np.int32), bittile=True)
    L.lbl_label(rm.h, None, 3, None)  # nothing to do
    rm2 = Roadmap(agent, np.array([0, 2, 3], np.int64), np.array([1, 5, 9], np.int32), bittile=True)
    O = cuda(np.full(64, np.uint64(2**64 - 1), np.uint64))
    for cfg in CFGS:
        assert (gpu_label(rm2, O, 0, cfg) == 0).all()


@pytest.mark.parametrize("bad", ["range", "negative", "unsorted", "duplicate", "rowptr_desc", "rowptr_end"])
def test_upload_rejects_malformed_csr(bad):
    agent = synth.agent_grid(8, 1.0, synth.MORTON)
    rowptr = np.array([0, 3, 5, 8], np.int64)
    colidx = np.array([1, 2, 3, 10, 11, 4, 5, 6], np.int32)
    if bad == "range":
        colidx[4] = 64
    elif bad == "negative":
        colidx[0] = -1
    elif bad == "unsorted":
        colidx[1], colidx[2] = 3, 2
    elif bad == "duplicate":
        colidx[2] = 2
    elif bad == "rowptr_desc":
        rowptr = np.array([0, 6, 5, 8], np.int64)
    elif bad == "rowptr_end":
        rowptr = np.array([0, 3, 5, 7], np.int64)
    with pytest.raises(L.LblError) as ei:
        L.lbl_roadmap_upload(agent, rowptr, colidx)
    assert ei.value.code == L.LBL_EINVAL


def test_upload_from_device_pointers_and_info(plain):
    wl = plain
    h = L.lbl_roadmap_upload(wl.agent, cuda(wl.rowptr), cuda(wl.colidx))
    try:
        E, nnz, nbt, nsec, ndy, b = L.lbl_roadmap_info(h)
        assert nbt == 0 and nsec == 0 and ndy == 0
        assert (E, nnz) == (wl.n_edges, wl.nnz) and b >= 8 * (E + 1) + 4 * nnz
        O = gpu_O(wl)
        out = empty_u64(E)
        L.lbl_label(h, O, wl.P, out)
        assert np.array_equal(host(out), oracle.label(wl.rowptr, wl.colidx, host(O), wl.P))
    finally:
        L.lbl_roadmap_free(h)


def _quad_count(rowptr, colidx, levels=4):
    """Maximal blocks of 4^j cells per row, counted by a plain scan (test helper)."""
    counts = []
    for e in range(rowptr.shape[0] - 1):
        row = colidx[rowptr[e]:rowptr[e + 1]].astype(np.int64)
        k, n = 0, 0
        while k < row.shape[0]:
            j = 0
            while j < levels:
                size = 4 << (2 * j)
                if row[k] % size or k + size > row.shape[0] or row[k + size - 1] != row[k] + size - 1:
                    break
                j += 1
            k += 1 << (2 * j)
            n += 1
        counts.append(n)
    return np.array(counts, np.int64)


def _tiled_rows(rowptr, colidx, w):
    """Each row's cells of a row-major grid w wide as sorted indices of the
    tiled order (16 x 16 tiles in row-major order, z-order inside a tile: x in
    the odd bits, y in the even bits), test helper."""
    c = colidx.astype(np.int64)
    x, y = c % w, c // w
    lx, ly = x % 16, y % 16
    z = np.zeros_like(c)
    for i in range(4):
        z |= ((lx >> i) & 1) << (2 * i + 1)
        z |= ((ly >> i) & 1) << (2 * i)
    t = ((y // 16) * (w // 16) + x // 16) * 256 + z
    out = np.empty_like(t)
    for e in range(rowptr.shape[0] - 1):
        out[rowptr[e]:rowptr[e + 1]] = np.sort(t[rowptr[e]:rowptr[e + 1]])
    return out


@pytest.mark.parametrize("order", [synth.MORTON, synth.ROWMAJOR, "tiled"])
def test_quad_runs_at_every_alignment(order):
    """Rows made of runs of 1..700 consecutive cells at every offset modulo 256,
    rows covering the whole grid, rows ending at its last cell and single
    cells: quadtree-form labels equal the oracle's for every proposition
    count (8-, 16-, 32- and 64-bit pyramid words; O words carry bits above P,
    which the labels must drop), and the form holds exactly one entry per
    maximal block of the grid's quadtree order (z-order; runs of a grid row on
    a row-major grid of partial tiles; squares of the tiled order on a
    row-major grid of whole 16 x 16 tiles)."""
    rng = np.random.default_rng(91 + (order if order != "tiled" else 7))
    if order == synth.MORTON:
        agent = synth.agent_grid(64, 0.5, order)
    elif order == synth.ROWMAJOR:
        agent = synth.Grid(77, 53, 0.5, 0.0, 0.0, order)
    else:
        agent = synth.Grid(80, 48, 0.5, 0.0, 0.0, synth.ROWMAJOR)
    cells = agent.cells
    rows = [np.arange(cells), np.arange(cells - 300, cells), np.array([cells - 1]), np.array([0]), np.arange(0, 256),
            np.arange(1, 257), np.arange(255, 512)]
    for start in range(0, 256, 7):
        for length in (1, 2, 3, 255, 256, 257, 700):
            if start + length <= cells:
                rows.append(np.arange(start, start + length))
    for _ in range(200):  # a few random runs per row
        parts = []
        for _ in range(int(rng.integers(1, 5))):
            a = int(rng.integers(0, cells - 1))
            parts.append(np.arange(a, min(cells, a + int(rng.integers(1, 400)))))
        rows.append(np.unique(np.concatenate(parts)))
    rows.append(np.array([], np.int64))
    rowptr = np.zeros(len(rows) + 1, np.int64)
    rowptr[1:] = np.cumsum([r.shape[0] for r in rows])
    colidx = np.concatenate(rows).astype(np.int32)
    rm = Roadmap(agent, rowptr, colidx, bittile=True)
    if order == "tiled":  # one-row runs are single cells there: no bound on the ratio
        want_entries = int(_quad_count(rowptr, _tiled_rows(rowptr, colidx, agent.w)).sum())
    else:
        want_entries = int(_quad_count(rowptr, colidx).sum())
        assert want_entries < 0.3 * colidx.shape[0]
    assert L.lbl_roadmap_info(rm.h)[4] == want_entries
    for P in (1, 2, 8, 9, 16, 17, 31, 32, 33, 64):  # every pyramid word width and its edges
        O_h = np.zeros(cells, np.uint64)
        hit = rng.random(cells) < 0.01
        O_h[hit] = rng.integers(1, 2**63, size=hit.sum(), dtype=np.uint64)
        O_h[cells - 1] = np.uint64(1 << (P - 1))
        want = oracle.label(rowptr, colidx, O_h, P)
        for depth in (8, 12, 16):
            assert np.array_equal(gpu_label(rm, cuda(O_h), P, dict(algo=L.LBL_ALGO_QUAD, depth=depth)), want), P
        front = dict(algo=L.LBL_ALGO_QUAD, pipeline=L.LBL_PIPE_FRONT)
        assert np.array_equal(gpu_label(rm, cuda(O_h), P, front), want), P


def test_quad_rejects_csr_pipelines(plain):
    rm = Roadmap(plain.agent, plain.rowptr, plain.colidx, bittile=True)
    for pipe in (L.LBL_PIPE_BULK, L.LBL_PIPE_ASYNC, 7):
        with pytest.raises(L.LblError) as ei:
            gpu_label(rm, gpu_O(plain), plain.P, dict(algo=L.LBL_ALGO_QUAD, pipeline=pipe))
        assert ei.value.code == L.LBL_EINVAL


def test_mma_needs_its_upload_flag_and_a_grid_of_at_most_2pow22_cells(plain):
    rm = Roadmap(plain.agent, plain.rowptr, plain.colidx, bittile=False)
    with pytest.raises(L.LblError) as ei:
        gpu_label(rm, gpu_O(plain), plain.P, dict(algo=L.LBL_ALGO_MMA))
    assert ei.value.code == L.LBL_EUNSUPPORTED
    big = synth.Grid(4096, 2048, 0.1, 0.0, 0.0, synth.ROWMAJOR)  # 2^23 cells
    with pytest.raises(L.LblError) as ei:
        L.lbl_roadmap_upload(big, np.array([0, 1], np.int64), np.array([5], np.int32), flags=L.LBL_UPLOAD_MMA)
    assert ei.value.code == L.LBL_EINVAL


def test_quad_needs_its_upload_flag(plain):
    rm = Roadmap(plain.agent, plain.rowptr, plain.colidx, bittile=False)
    with pytest.raises(L.LblError) as ei:
        gpu_label(rm, gpu_O(plain), plain.P, dict(algo=L.LBL_ALGO_QUAD))
    assert ei.value.code == L.LBL_EUNSUPPORTED


def test_bittile_needs_its_upload_flag(plain):
    rm = Roadmap(plain.agent, plain.rowptr, plain.colidx, bittile=False)
    with pytest.raises(L.LblError) as ei:
        gpu_label(rm, gpu_O(plain), plain.P, dict(algo=L.LBL_ALGO_BITTILE))
    assert ei.value.code == L.LBL_EUNSUPPORTED


# ----------------------------------------------------------------- monitor

@pytest.mark.parametrize("n_states,m,reject", [(1, 0, -1), (3, 1, 2), (5, 3, -1), (16, 8, 15), (9, 6, 0)])
def test_monitor_step_matches_oracle(n_states, m, reject):
    rng = np.random.default_rng(n_states * 10 + m)
    relbits = rng.choice(64, size=m, replace=False).astype(np.uint8)
    delta = rng.integers(0, n_states, size=(n_states, 1 << m)).astype(np.uint8)
    Lw = rng.integers(0, 2**64 - 1, size=70_001, dtype=np.uint64)
    h = L.lbl_monitor_create(n_states, m, relbits, delta, reject)
    try:
        nxt, viol = empty_u64(Lw.shape[0]), empty_u16(Lw.shape[0])
        L.lbl_monitor_step(h, cuda(Lw), Lw.shape[0], nxt, viol)
        wn, wv = oracle.monitor(n_states, m, relbits, delta, reject, Lw)
        assert np.array_equal(host(nxt), wn) and np.array_equal(host(viol), wv)
    finally:
        L.lbl_monitor_free(h)


# ----------------------------------------------------------------- session

def test_session_run_from_host_memory(large_small):
    wl = large_small
    rm = Roadmap(wl.agent, wl.rowptr, wl.colidx)
    mon = wl.monitor
    hm = L.lbl_monitor_create(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject)
    ss = L.lbl_session_create(rm.h, wl.world, wl.P, hm)
    try:
        planes = torch.from_numpy(wl.planes).pin_memory()
        outL = torch.empty(wl.n_edges, dtype=torch.uint64).pin_memory()
        outN = torch.empty(wl.n_edges, dtype=torch.uint64).pin_memory()
        outV = torch.empty(wl.n_edges, dtype=torch.uint16).pin_memory()
        rng = np.random.default_rng(8)
        for _ in range(3):
            pose = synth.random_pose(rng, wl.world)
            L.lbl_session_run(ss, planes, pose, outL, outN, outV)
            torch.cuda.synchronize()
            O = oracle.frame_transform(wl.world, wl.planes, pose, wl.agent)
            want = oracle.label(wl.rowptr, wl.colidx, O, wl.P, threads=8)
            wn, wv = oracle.monitor(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject, want)
            assert np.array_equal(outL.numpy(), want)
            assert np.array_equal(outN.numpy(), wn) and np.array_equal(outV.numpy(), wv)
    finally:
        L.lbl_session_free(ss)
        L.lbl_monitor_free(hm)


@pytest.mark.parametrize("flags", [0, "quad", "front"])
def test_session_chunked_copies_match_oracle(flags):
    """Roadmaps of 2^16 edges or more: the session labels them on its own
    stream with its own pyramid and partition, then copies the results to the
    host; by the per-warp stream (the size rule at 90k edges) or the moving
    front (forced here; chosen by size on large roadmaps)."""
    wl = synth.make("large", seed=14, edges=90_000)
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD if flags else 0)
    mon = wl.monitor
    hm = L.lbl_monitor_create(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject)
    cfg = dict(algo=L.LBL_ALGO_QUAD, pipeline=L.LBL_PIPE_FRONT) if flags == "front" else None
    ss = L.lbl_session_create(rm, wl.world, wl.P, hm, cfg)
    try:
        planes = torch.from_numpy(wl.planes).pin_memory()
        outL = torch.full((wl.n_edges,), 7, dtype=torch.int64).view(torch.uint64).pin_memory()
        outN = torch.empty(wl.n_edges, dtype=torch.uint64).pin_memory()
        outV = torch.empty(wl.n_edges, dtype=torch.uint16).pin_memory()
        rng = np.random.default_rng(15)
        s = torch.cuda.Stream()
        for _ in range(2):
            pose = synth.random_pose(rng, wl.world)
            L.lbl_session_run(ss, planes, pose, outL, outN, outV, stream=s)
            s.synchronize()  # the caller's stream covers the copies made on the session's own stream
            O = oracle.frame_transform(wl.world, wl.planes, pose, wl.agent)
            want = oracle.label(wl.rowptr, wl.colidx, O, wl.P, threads=8)
            wn, wv = oracle.monitor(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject, want)
            assert np.array_equal(outL.numpy(), want)
            assert np.array_equal(outN.numpy(), wn) and np.array_equal(outV.numpy(), wv)
    finally:
        L.lbl_session_free(ss)
        L.lbl_monitor_free(hm)
        L.lbl_roadmap_free(rm)


def test_session_frames_back_to_back():
    """Frames enqueued without waiting: the plane copies of frame i+1 overlap
    frame i (two device slots, reused every other frame) and every frame's
    outputs still equal the oracle's."""
    wl = synth.make("large", seed=16, edges=80_000)
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=L.LBL_UPLOAD_QUAD)
    mon = wl.monitor
    hm = L.lbl_monitor_create(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject)
    ss = L.lbl_session_create(rm, wl.world, wl.P, hm)
    try:
        rng = np.random.default_rng(17)
        plane_sets = [np.ascontiguousarray(wl.planes), np.ascontiguousarray(wl.planes[::-1]),
                      np.ascontiguousarray(np.roll(wl.planes, 5, axis=0))]
        frames = []
        for i in range(6):
            planes = plane_sets[i % 3]
            frames.append(dict(planes=planes, h_planes=torch.from_numpy(planes).pin_memory(),
                               pose=synth.random_pose(rng, wl.world),
                               L=torch.empty(wl.n_edges, dtype=torch.uint64).pin_memory(),
                               N=torch.empty(wl.n_edges, dtype=torch.uint64).pin_memory(),
                               V=torch.empty(wl.n_edges, dtype=torch.uint16).pin_memory()))
        s = torch.cuda.Stream()
        for f in frames:
            L.lbl_session_run(ss, f["h_planes"], f["pose"], f["L"], f["N"], f["V"], stream=s)
        s.synchronize()
        for i, f in enumerate(frames):
            O = oracle.frame_transform(wl.world, f["planes"], f["pose"], wl.agent)
            want = oracle.label(wl.rowptr, wl.colidx, O, wl.P, threads=8)
            wn, wv = oracle.monitor(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject, want)
            assert np.array_equal(f["L"].numpy(), want), i
            assert np.array_equal(f["N"].numpy(), wn) and np.array_equal(f["V"].numpy(), wv), i
    finally:
        L.lbl_session_free(ss)
        L.lbl_monitor_free(hm)
        L.lbl_roadmap_free(rm)


def test_autotune_choice_is_exact_and_sticks(driving_small):
    wl = driving_small
    rm = Roadmap(wl.agent, wl.rowptr, wl.colidx, bittile=True)
    O = gpu_O(wl)
    want = oracle.label(wl.rowptr, wl.colidx, host(O), wl.P, threads=8)
    out = empty_u64(rm.E)
    chosen = L.lbl_roadmap_autotune(rm.h, O, wl.P, out, reps=2)
    assert chosen["algo"] in (L.LBL_ALGO_CSR, L.LBL_ALGO_BITTILE, L.LBL_ALGO_SECTOR, L.LBL_ALGO_QUAD, L.LBL_ALGO_MMA)
    assert np.array_equal(host(out), want)
    assert np.array_equal(gpu_label(rm, O, wl.P, dict(algo=L.LBL_ALGO_AUTO)), want)
    assert np.array_equal(gpu_label(rm, O, wl.P, None), want)
    L.lbl_roadmap_status(rm.h)


def test_autotune_on_a_roadmap_without_derived_forms(driving_small):
    """A CSR-only roadmap: the tuner tries only the forms the roadmap has."""
    wl = driving_small
    rm = Roadmap(wl.agent, wl.rowptr, wl.colidx, bittile=False)
    O = gpu_O(wl)
    out = empty_u64(rm.E)
    chosen = L.lbl_roadmap_autotune(rm.h, O, wl.P, out, reps=1)
    assert chosen["algo"] == L.LBL_ALGO_CSR
    assert np.array_equal(host(out), oracle.label(wl.rowptr, wl.colidx, host(O), wl.P, threads=8))


@pytest.mark.parametrize("order", [synth.MORTON, synth.ROWMAJOR])
def test_quad_rows_in_locality_order_or_the_callers(order):
    """The quadtree rows of a 2-D roadmap are stored sorted for locality (labels
    and monitor outputs written back to the caller's edges) unless
    LBL_UPLOAD_KEEP_ORDER keeps the caller's order; both equal the oracle."""
    wl = synth.make("large", seed=21, edges=40_000, order=order)
    mon = wl.monitor
    hm = L.lbl_monitor_create(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject)
    O_h = oracle.frame_transform(wl.world, wl.planes, wl.pose, wl.agent)
    want = oracle.label(wl.rowptr, wl.colidx, O_h, wl.P, threads=8)
    wn, wv = oracle.monitor(mon.n_states, mon.m, mon.relbits, mon.delta, mon.reject, want)
    try:
        for flags in (L.LBL_UPLOAD_QUAD, L.LBL_UPLOAD_QUAD | L.LBL_UPLOAD_KEEP_ORDER):
            rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=flags)
            try:
                out, nx, vi = empty_u64(wl.n_edges), empty_u64(wl.n_edges), empty_u16(wl.n_edges)
                L.lbl_label(rm, cuda(O_h), wl.P, out, hm, nx, vi, dict(algo=L.LBL_ALGO_QUAD))
                assert np.array_equal(host(out), want), flags
                assert np.array_equal(host(nx), wn) and np.array_equal(host(vi), wv), flags
            finally:
                L.lbl_roadmap_free(rm)
    finally:
        L.lbl_monitor_free(hm)
