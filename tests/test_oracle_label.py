"""Pins of the oracle's cluster identification (breadth-first search, Sec. II.B.1).

* Independent library: scipy's ``csgraph.connected_components`` on the bond
  graph (periodic and open), relabelled to the minimum site index, must equal
  the oracle's labels element by element; for images, ``scipy.ndimage.label``
  of each grey level with 4-connectivity.
* Brute force: the Fortuin-Kasteleyn identity (Sec. II, Eqs. 2-5) on the
  3 x 3 torus -- the random-cluster sum over all 2^18 bond sets, with the
  oracle counting clusters, equals the Potts partition function enumerated
  over all q^9 spin states.  A missing wrap bond or a miscounted cluster
  breaks the identity.
* Invariants of a canonical labeling.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import oracle
import oracle.exact as ex


def _scipy_labels(mask, H, W, periodic):
    N = H * W
    east, north = oracle.unpack_mask(mask, N)
    i = np.arange(N)
    y, x = i // W, i % W
    rows, cols = [], []
    ok_e = east.astype(bool) & (periodic | (x + 1 < W))
    rows.append(i[ok_e]); cols.append((y * W + (x + 1) % W)[ok_e])
    ok_n = north.astype(bool) & (periodic | (y + 1 < H))
    rows.append(i[ok_n]); cols.append((((y + 1) % H) * W + x)[ok_n])
    r = np.concatenate(rows); c = np.concatenate(cols)
    A = coo_matrix((np.ones(r.size), (r, c)), shape=(N, N))
    n, comp = connected_components(A, directed=False)
    first = np.full(n, N, dtype=np.int64)
    np.minimum.at(first, comp, i)
    return first[comp].astype(np.int32), n


def _random_mask(H, W, p, seed):
    rng = np.random.default_rng(seed)
    N = H * W
    return oracle.pack_mask(rng.random(N) < p, rng.random(N) < p)


SHAPES = [(1, 1), (1, 7), (7, 1), (2, 2), (3, 5), (5, 3), (4, 4), (17, 33), (64, 64), (100, 36), (129, 257)]


@pytest.mark.parametrize("H,W", SHAPES)
@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("p", [0.3, 0.5, 0.7, 1.0])
def test_label_matches_scipy(H, W, periodic, p):
    mask = _random_mask(H, W, p, seed=H * 1000 + W + int(p * 10))
    lab, n = oracle.label(mask, H, W, periodic)
    ref, nref = _scipy_labels(mask, H, W, periodic)
    assert n == nref
    assert np.array_equal(lab, ref)


def test_label_perc_masks_match_scipy():
    for k in range(3):
        mask = oracle.perc_mask(256, 256, k)
        lab, n = oracle.label(mask, 256, 256, True)
        ref, nref = _scipy_labels(mask, 256, 256, True)
        assert n == nref and np.array_equal(lab, ref)


def test_label_invariants():
    H, W = 96, 160
    mask = oracle.perc_mask(H, W, 11)
    lab, n = oracle.label(mask, H, W, True)
    i = np.arange(H * W)
    assert np.all(lab <= i)                       # label is the cluster minimum
    assert np.array_equal(lab[lab], lab)          # roots label themselves
    assert np.unique(lab).size == n
    east, north = oracle.unpack_mask(mask, H * W)
    y, x = i // W, i % W
    e = east.astype(bool); nb = north.astype(bool)
    assert np.all(lab[e] == lab[(y * W + (x + 1) % W)[e]])
    assert np.all(lab[nb] == lab[(((y + 1) % H) * W + x)[nb]])


@pytest.mark.parametrize("periodic", [True, False])
def test_image_labels_match_ndimage(periodic):
    rng = np.random.default_rng(3)
    px = rng.integers(0, 3, size=(37, 53)).astype(np.uint8)
    mask = oracle.bonds_from_pixels(px, periodic)
    lab, n = oracle.label(mask, 37, 53, periodic)
    if periodic:
        ref, nref = _scipy_labels(mask, 37, 53, True)
        assert n == nref and np.array_equal(lab, ref)
        return
    # open boundaries: ndimage.label per level, 4-connectivity, then min-index relabel
    ref = np.full(px.size, -1, dtype=np.int64)
    total = 0
    for lev in np.unique(px):
        comp, nc = ndi.label(px == lev)
        total += nc
        comp = comp.reshape(-1)
        sel = comp > 0
        first = np.full(nc + 1, px.size, dtype=np.int64)
        np.minimum.at(first, comp[sel], np.nonzero(sel)[0])
        ref[sel] = first[comp[sel]]
    assert n == total
    assert np.array_equal(lab, ref.astype(np.int32))


@pytest.mark.parametrize("q,K", [(2, 0.7), (3, 1.0050525)])
def test_fk_identity_3x3_torus(q, K):
    """Eq. 5 (random-cluster form) == Eq. 2 (spin form) on the 3 x 3 torus."""
    fk = ex.fk_sum(3, 3, q, K, lambda m: oracle.label(m, 3, 3, True)[1])
    Z = ex.potts_Z_bruteforce(3, 3, q, K)
    assert abs(fk / Z - 1.0) < 1e-11
