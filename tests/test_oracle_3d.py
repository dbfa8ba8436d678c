"""Pins of the oracle's simple-cubic (3D) Swendsen-Wang sweep.

The paper presents the method on the square lattice and states that the
generalisation to three dimensions is direct (Secs. II and II.B); the oracle
runs the same three steps on a periodic X x Y x Z box with six neighbours.

* labeling: scipy ``connected_components`` on the periodic 3D bond graph
  (random masks, boxes with sides 1 to 9, densities 0.1 to 1), relabelled
  to the minimum site index; canonical-label invariants; a box of depth 1
  with no +z bond labels like the 2D oracle on the same square mask;
* activation (Eq. 7): bonds between unequal spins never open; an equal-spin
  bond opens iff word d of the site's BOND3 Philox draw is below T
  (closed form from the separately pinned Philox), binomial in T / 2^32;
* observables: numpy rolls over the three axes;
* whole chain: the Potts Boltzmann distribution on 2 x 2 x 2 and
  2 x 2 x 4 tori (q = 2) and 2 x 2 x 2 (q = 3) from exact enumeration of all
  spin states, within binned error bars.
"""
import math

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import oracle
import oracle.exact as ex

KC3_ISING = 0.2216546   # simple-cubic Ising critical coupling (literature, ~1e-7); only sets a test point


def _neighbours(X, Y, Z):
    i = np.arange(X * Y * Z)
    x, y, z = i % X, (i // X) % Y, i // (X * Y)
    return [(z * Y + y) * X + (x + 1) % X, (z * Y + (y + 1) % Y) * X + x, (((z + 1) % Z) * Y + y) * X + x]


def _scipy_labels(mask, X, Y, Z):
    N = X * Y * Z
    i = np.arange(N)
    nb = _neighbours(X, Y, Z)
    src, dst = [], []
    for d in range(3):
        sel = ((mask >> d) & 1) == 1
        src.append(i[sel])
        dst.append(nb[d][sel])
    src, dst = np.concatenate(src), np.concatenate(dst)
    g = coo_matrix((np.ones(src.size), (src, dst)), shape=(N, N))
    _, comp = connected_components(g, directed=False)
    first = np.full(comp.max() + 1, N, dtype=np.int64)
    np.minimum.at(first, comp, i)
    return first[comp].astype(np.int32), comp.max() + 1


@pytest.mark.parametrize("X,Y,Z", [(2, 2, 2), (4, 4, 4), (3, 5, 7), (9, 1, 4), (1, 6, 6), (8, 8, 3), (5, 5, 5)])
@pytest.mark.parametrize("density", [0.1, 0.25, 0.5, 1.0])
def test_labels_match_scipy(X, Y, Z, density):
    rng = np.random.default_rng(X * 100 + Y * 10 + Z)
    bits = rng.random((X * Y * Z, 3)) < density
    mask = (bits[:, 0] | (bits[:, 1] << 1) | (bits[:, 2] << 2)).astype(np.uint8)
    lab, n = oracle.label3(mask, X, Y, Z)
    ref, nref = _scipy_labels(mask, X, Y, Z)
    assert n == nref and np.array_equal(lab, ref)
    i = np.arange(X * Y * Z)
    assert np.all(lab <= i) and np.array_equal(lab[lab], lab)
    for d, nb in enumerate(_neighbours(X, Y, Z)):
        sel = ((mask >> d) & 1) == 1
        assert np.array_equal(lab[i[sel]], lab[nb[sel]])


def test_depth_one_box_labels_like_the_square_lattice():
    X, Y = 37, 23
    rng = np.random.default_rng(4)
    e = (rng.random(X * Y) < 0.5).astype(np.uint8)
    n = (rng.random(X * Y) < 0.5).astype(np.uint8)
    lab2, n2 = oracle.label(oracle.pack_mask(e, n), Y, X, True)
    lab3, n3 = oracle.label3(e | (n << 1), X, Y, 1)
    assert n2 == n3 and np.array_equal(lab2, lab3)


def test_activation_closed_form():
    X, Y, Z, q, seed, sweep = 6, 4, 5, 3, 99, 12
    s = oracle.init_spins3(X, Y, Z, q, seed, True)
    T = oracle.threshold(0.8)
    m = oracle.activate3(X, Y, Z, s, seed, sweep, T)
    nb = _neighbours(X, Y, Z)
    for i in range(X * Y * Z):
        w = oracle.philox4x32_10((i, sweep, 0, oracle.TAG_BOND3), (seed, 0))
        for d in range(3):
            want = int(s[i] == s[nb[d][i]] and w[d] < T)
            assert ((m[i] >> d) & 1) == want, (i, d)


def test_activation_binomial():
    X = Y = Z = 32
    s = np.zeros(X * Y * Z, dtype=np.int8)            # every bond joins equal spins
    T = oracle.threshold(0.5)
    m = oracle.activate3(X, Y, Z, s, 5, 0, T)
    n_open = sum(int(((m >> d) & 1).sum()) for d in range(3))
    n = 3 * X * Y * Z
    p = T / 2.0 ** 32
    assert abs(n_open - n * p) < 5 * math.sqrt(n * p * (1 - p))
    rng = np.random.default_rng(2)
    s = rng.integers(0, 2, X * Y * Z).astype(np.int8)
    m = oracle.activate3(X, Y, Z, s, 5, 1, 1 << 32)
    for d, nb in enumerate(_neighbours(X, Y, Z)):
        assert np.array_equal((m >> d) & 1, (s == s[nb]).astype(np.uint8))


def test_observables_numpy():
    X, Y, Z, q = 7, 6, 5, 4
    rng = np.random.default_rng(1)
    s = rng.integers(0, q, X * Y * Z).astype(np.int8)
    a = s.reshape(Z, Y, X)
    n_eq = sum(int((a == np.roll(a, -1, axis=ax)).sum()) for ax in (0, 1, 2))
    want = [n_eq] + [int((s == k).sum()) for k in range(q)]
    assert list(oracle.observables3(X, Y, Z, q, s)) == want


def test_init_matches_square_lattice_draws():
    s3 = oracle.init_spins3(8, 8, 1, 5, 17, True)
    assert np.array_equal(s3, oracle.init_spins(8, 5, 17, True))
    assert not oracle.init_spins3(4, 4, 4, 5, 17, False).any()


def _binned(x, nbins=50):
    x = np.asarray(x, dtype=np.float64)
    b = x[: len(x) // nbins * nbins].reshape(nbins, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nbins)


@pytest.mark.parametrize("dims,q,K", [((2, 2, 2), 2, 2 * KC3_ISING), ((2, 2, 4), 2, 2 * KC3_ISING),
                                      ((2, 2, 2), 3, math.log(1 + math.sqrt(3)) * 0.6),
                                      ((2, 2, 4), 2, 2 * 0.35)])
def test_chain_against_enumeration(dims, q, K):
    X, Y, Z = dims
    T = oracle.threshold(K)
    s0 = oracle.init_spins3(X, Y, Z, q, 11, True)
    _, obs = oracle.chain3(X, Y, Z, q, T, 11, 0, 200_000, s0)
    obs = obs[500:]
    n_eq, counts = ex.enumerate_potts_3d(X, Y, Z, q)
    exact = ex.moments_from_states(n_eq, counts, K, q)
    n = obs[:, 0].astype(np.float64)
    series = [(n, "n_eq"), (n * n, "n_eq2")]
    if q == 2:
        series.append((np.abs(obs[:, 1] - obs[:, 2]), "absM"))
    for x, key in series:
        m, e = _binned(x)
        assert abs(m - exact[key]) < 4.5 * e, (key, m, exact[key], e)
