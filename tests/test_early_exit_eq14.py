"""Early termination (Sec. 5, eq. 14) on Bernoulli inputs.

With every voxel occupied by the motion with probability p_mot and by the
predicate with probability p_pred, independently, the voxel index T (1-based)
of the first voxel that both occupy is geometric with success probability
p = p_pred * p_mot, so E[T] = 1 / (p_pred * p_mot) (eq. 14): that is where an
early-terminating scan of the voxels in order stops.

Each trial t draws N voxels (cells t*N .. t*N+N-1 of a row-major grid of N
columns); its rows are the motion voxels of every prefix of length n = 1..N.
Proposition 0 labels row (t, n) iff the first common voxel lies within the
first n voxels, so the labels of the prefixes give T exactly: T = 1 + the
number of prefixes left unlabelled.  The CPU test reads T from the oracle's
labels; the GPU test from the labeling kernels with early exit on (which must
equal the oracle), and both check the mean of T against eq. 14 within 4.5
standard errors, and the ratio of two predicate occupancies against the
ratio eq. 14 predicts."""
import math

import numpy as np
import pytest

import oracle
import synth


def _trials(seed, n_trials, N, p_pred, p_mot):
    rng = np.random.default_rng(seed)
    mot = rng.random((n_trials, N)) < p_mot
    pred = rng.random((n_trials, N)) < p_pred
    O = np.zeros(n_trials * N, np.uint64)
    O[pred.ravel()] = 1
    # rows: for trial t and prefix length n, the motion voxels among its first n
    counts = np.cumsum(mot, axis=1)  # motion voxels in each prefix
    rowlen = counts.ravel()          # row (t, n-1) has counts[t, n-1] entries
    rowptr = np.zeros(n_trials * N + 1, np.int64)
    rowptr[1:] = np.cumsum(rowlen)
    cols = []
    for t in range(n_trials):
        idx = (t * N + np.flatnonzero(mot[t])).astype(np.int32)
        c = counts[t]
        cols.extend(idx[: c[n]] for n in range(N))
    colidx = np.concatenate(cols) if rowptr[-1] else np.zeros(0, np.int32)
    grid = synth.Grid(N, n_trials, 0.1, 0.0, 0.0, synth.ROWMAJOR)
    return grid, rowptr, colidx.astype(np.int32), O


def _first_hits(labels, n_trials, N):
    lab = (labels.reshape(n_trials, N) & np.uint64(1)).astype(bool)
    assert (np.diff(lab.astype(np.int8), axis=1) >= 0).all()  # a longer prefix keeps the label
    T = 1 + (~lab).sum(axis=1)
    return T[lab[:, -1]], lab[:, -1].mean()  # trials with a hit within N voxels


def _check_mean(T, frac_hit, p, N):
    mean, sd = 1.0 / p, math.sqrt(1.0 - p) / p
    assert frac_hit > 1 - 1e-3 and (1 - p) ** N < 1e-4  # truncation at N is negligible
    assert abs(T.mean() - mean) < 4.5 * sd / math.sqrt(T.shape[0]), (T.mean(), mean)


CASES = [(0.9, 0.05, 2000, 250), (0.1, 0.05, 400, 2400)]  # (p_pred, p_mot, trials, voxels per trial)


@pytest.mark.parametrize("p_pred,p_mot,n_trials,N", CASES)
def test_eq14_mean_voxels_to_first_hit_from_the_oracle(p_pred, p_mot, n_trials, N):
    grid, rowptr, colidx, O = _trials(14, n_trials, N, p_pred, p_mot)
    labels = oracle.label(rowptr, colidx, O, 1, threads=4)
    T, frac = _first_hits(labels, n_trials, N)
    _check_mean(T, frac, p_pred * p_mot, N)


def test_eq14_ratio_of_two_occupancies_from_the_oracle():
    """eq. 14 predicts that a predicate occupying 9x more voxels stops 9x
    sooner on Bernoulli inputs (the paper's 90 for 90 % vs 1 %)."""
    means = []
    for p_pred, p_mot, n_trials, N in CASES:
        grid, rowptr, colidx, O = _trials(15, n_trials, N, p_pred, p_mot)
        T, _ = _first_hits(oracle.label(rowptr, colidx, O, 1, threads=4), n_trials, N)
        means.append(T.mean())
    assert 7.5 < means[1] / means[0] < 10.8, means


@pytest.mark.gpu
@pytest.mark.parametrize("p_pred,p_mot,n_trials,N", CASES)
def test_eq14_with_early_exit_kernels(p_pred, p_mot, n_trials, N):
    torch = pytest.importorskip("torch")
    import paper_1810_02612_gb300 as L
    grid, rowptr, colidx, O_h = _trials(16, n_trials, N, p_pred, p_mot)
    want = oracle.label(rowptr, colidx, O_h, 1, threads=4)
    rm = L.lbl_roadmap_upload(grid, rowptr, colidx, flags=L.LBL_UPLOAD_BITTILE)
    try:
        O = torch.from_numpy(O_h).cuda()
        E = rowptr.shape[0] - 1
        for cfg in (dict(algo=L.LBL_ALGO_CSR, lanes_per_edge=8, early_exit=1),
                    dict(algo=L.LBL_ALGO_CSR, lanes_per_edge=32, early_exit=1),
                    dict(algo=L.LBL_ALGO_BITTILE, early_exit=1)):
            out = torch.empty(E, dtype=torch.uint64, device="cuda")
            L.lbl_label(rm, O, 1, out, cfg=cfg)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.array_equal(got, want), cfg
            T, frac = _first_hits(got, n_trials, N)
            _check_mean(T, frac, p_pred * p_mot, N)
    finally:
        L.lbl_roadmap_free(rm)
