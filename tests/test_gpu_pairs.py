"""Whole-series DTW without an external upper bound: the pairwise matrix
(each pair pruned under its own diagonal cost) and k-NN / 1-NN classification
(each pair pruned under the test's current k-th best), against the oracle."""
import numpy as np
import pytest

import oracle as O
from gpu_util import dist_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2010_05371_gb300 import api, synth  # noqa: E402


def series_set(count, length, seed, ecg=False):
    out = []
    for s in range(count):
        x = synth.ecg_query(length, seed + s) if ecg else synth.random_walk(length, seed + s)
        out.append(np.asarray(x, dtype=np.float64))
    return np.stack(out)


@pytest.mark.parametrize("length,w,ecg", [(64, 6, False), (200, 200, False), (300, 30, True), (700, 700, False),
                                          (1300, 260, False)])
def test_pairwise_matrix(length, w, ecg):
    A = series_set(5, length, 100, ecg)
    B = series_set(7, length, 200, ecg)
    got = api.pairwise(torch.tensor(A, dtype=torch.float32, device="cuda"),
                       torch.tensor(B, dtype=torch.float32, device="cuda"), w).cpu().numpy()
    Af, Bf = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
    for i in range(len(A)):
        for j in range(len(B)):
            ref = O.dtw(O.znorm(Af[i]), O.znorm(Bf[j]), w)
            assert dist_close(float(got[i, j]), ref, length), (i, j, got[i, j], ref)


def test_pairwise_raw_and_identity():
    A = series_set(4, 150, 7)
    T = torch.tensor(A, dtype=torch.float32, device="cuda")
    got = api.pairwise(T, T, 15, znorm=False).cpu().numpy()
    assert np.all(np.diag(got) == 0.0)
    np.testing.assert_array_equal(got, got.T)   # DTW is symmetric, exactly
    Af = A.astype(np.float32).astype(np.float64)
    assert dist_close(float(got[0, 1]), O.dtw(Af[0], Af[1], 15), 150)


@pytest.mark.parametrize("length,w,k", [(128, 13, 1), (256, 60, 3), (900, 900, 1), (1500, 300, 2)])
def test_nearest_series(length, w, k):
    train = series_set(40, length, 300)
    test = series_set(6, length, 400)
    idx, dist = api.nearest_series(torch.tensor(train, dtype=torch.float32, device="cuda"),
                                   torch.tensor(test, dtype=torch.float32, device="cuda"), w, k)
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    tr, te = train.astype(np.float32).astype(np.float64), test.astype(np.float32).astype(np.float64)
    for t in range(len(test)):
        d = np.array([O.dtw(O.znorm(tr[j]), O.znorm(te[t]), w) for j in range(len(train))])
        order = np.lexsort((np.arange(len(d)), d))[:k]
        for r in range(k):
            assert dist_close(float(dist[t, r]), float(d[order[r]]), length)
            if idx[t, r] != order[r]:
                assert dist_close(float(d[idx[t, r]]), float(d[order[r]]), length)


def test_fewer_training_series_than_k():
    train = torch.tensor(series_set(2, 64, 1), dtype=torch.float32, device="cuda")
    test = torch.tensor(series_set(3, 64, 9), dtype=torch.float32, device="cuda")
    idx, dist = api.nearest_series(train, test, 8, 4)
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    assert np.all(idx[:, 2:] == -1) and np.all(np.isinf(dist[:, 2:]))
    assert np.all(idx[:, :2] >= 0)
