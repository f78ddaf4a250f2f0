"""Block layout of the folded CUDA-core contraction (pat_fold_blocks, host
only): every D4 representative {|kx|, |ky|} sits in exactly one block slot,
the blocks of a chunk hold representatives of one radius kx^2 + ky^2 at each
lane, and the chunk counts follow from counting radii by their number of
representatives."""
import numpy as np
import pytest

from paper_2603_28150_gb300 import pat


def _reps(P):
    h = P // 2
    return [(a, b) for a in range(h + 1) for b in range(a, h + 1)]


def _chunks_by_counting(P):
    """Independent count: radii grouped by how many representatives share them,
    32 radii per chunk; never more chunks than one row per representative."""
    per = {}
    for a, b in _reps(P):
        per[a * a + b * b] = per.get(a * a + b * b, 0) + 1
    sizes = {}
    for m in per.values():
        sizes[m] = sizes.get(m, 0) + 1
    shared = sum((n + 31) // 32 for n in sizes.values())
    return min(shared, (len(_reps(P)) + 31) // 32)


@pytest.mark.parametrize("P", [16, 24, 48, 64, 96, 128, 256, 512])
@pytest.mark.parametrize("radial", [False, True])
def test_every_representative_once_and_radii_shared(P, radial):
    f = pat.fold_blocks(P, radial)
    reps = _reps(P)
    U = len(reps)
    key = np.array([a * a + b * b for a, b in reps])
    rr = f["rb_rep"]
    used = rr[rr >= 0]
    assert np.array_equal(np.sort(used), np.arange(U))
    assert f["rb_chunk"].min() >= 0 and f["rb_chunk"].max() < f["nch"]
    # every chunk is read by at least one block, and the blocks of a chunk are consecutive
    chunks = f["rb_chunk"]
    assert set(chunks.tolist()) == set(range(f["nch"]))
    assert np.all(np.diff(chunks) >= 0)
    for j in range(f["nrb"]):
        c = chunks[j]
        for lane in range(32):
            u = rr[j, lane]
            src = f["row_rep"][c, lane]
            if u < 0:
                continue
            assert f["rep_row"][u] == 32 * c + lane
            assert src >= 0 and key[src] == key[u]       # the stored row holds u's radius
    # a stored row with no representative is read by no block slot
    for c in range(f["nch"]):
        for lane in range(32):
            if f["row_rep"][c, lane] < 0:
                assert np.all(rr[chunks == c, lane] < 0)
    if not radial:
        assert f["nrb"] == f["nch"] == (U + 31) // 32
        assert np.array_equal(f["rep_row"], np.arange(U))


@pytest.mark.parametrize("P", [16, 24, 32, 48, 64, 128, 256, 512, 768])
def test_chunk_counts(P):
    f = pat.fold_blocks(P, True)
    assert f["nch"] == _chunks_by_counting(P)
    ident = (len(_reps(P)) + 31) // 32
    if f["nch"] == ident:      # sharing would store no fewer chunks: the identity layout
        assert f["nrb"] == ident and np.array_equal(f["rep_row"], np.arange(len(_reps(P))))


def test_benchmark_grid_counts():
    """256 x 256: 8385 representatives on 5924 radii; 189 chunks read by 277
    blocks instead of 263 chunks (0.72 of the table)."""
    f = pat.fold_blocks(256, True)
    assert (f["nch"], f["nrb"]) == (189, 277)
    assert len({a * a + b * b for a, b in _reps(256)}) == 5924
    assert pat.fold_blocks(256, False)["nch"] == 263


def test_rejects_bad_lengths():
    for P in (0, 1, 7, -4):
        with pytest.raises(pat.PatError):
            pat.fold_blocks(P, True)


def test_plan_estimate_representations():
    """pat_plan_estimate's table bytes for the complex, per-bin real, D4-folded
    and radially shared representations (4 depths per 16-byte group, chunks of
    32 rows), and the per-representative tensor tiles of a folded plan."""
    n, nz, nt, P = 128, 64, 256, 256
    K = (P // 2 + 1) * P
    row = nt * nz * 4
    chunks = lambda rows: (rows + 31) // 32 * 32  # noqa: E731
    U = len(_reps(P))
    tbc, _ = pat.plan_estimate(n, n, nz, nt, P, P, real_table=False)
    tbr, _ = pat.plan_estimate(n, n, nz, nt, P, P)
    tbf, _ = pat.plan_estimate(n, n, nz, nt, P, P, fold=True)
    tbx, ws = pat.plan_estimate(n, n, nz, nt, P, P, fold=True, radial=True)
    assert tbr == chunks(K) * row and tbc == 2 * tbr
    assert tbf == chunks(U) * row
    assert tbx == 32 * pat.fold_blocks(P, True)["nch"] * row == 396361728
    assert ws == pat.workspace_size(n, n, nz, nt, P, P)
    # tensor tiles: hi + lo BF16 per (representative, t, z), both directions
    t128, _ = pat.plan_estimate(n, n, 128, 512, P, P, max_batch=16, bf16_split=True, fold=True,
                                radial=True)
    assert t128 == 32 * pat.fold_blocks(P, True)["nch"] * 512 * 128 * 4 + 2 * U * 512 * 128 * 4
    # a rectangular grid cannot fold: the per-bin count
    assert pat.plan_estimate(n, 64, nz, nt, P, 128, fold=True)[0] == \
        pat.plan_estimate(n, 64, nz, nt, P, 128)[0]
