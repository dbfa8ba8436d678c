"""Exact results for small and finite Potts / Ising tori.

TEST INFRASTRUCTURE ONLY (see the package docstring).  These functions know
nothing about Swendsen-Wang dynamics; they give the equilibrium quantities the
SW Markov chain must reproduce, and pin the oracle from outside itself.

* :func:`enumerate_potts` -- brute force over all q^N spin states of an
  Lx x Ly periodic torus: the joint histogram of (n_eq, n_0..n_{q-1}).
* :func:`potts_dos` -- exact density of states g(n_eq) of the q-state Potts
  model on an Lx x Ly torus by a row transfer matrix with an energy index.
* :func:`ising_torus_logZ` -- the exact finite-torus partition function of
  the 2D Ising model (Kaufman 1949; Ferdinand & Fisher 1969, the exact result
  the paper compares its q = 2 runs with in Sec. II.A).
* :func:`fk_sum` -- the random-cluster (Fortuin-Kasteleyn) sum of Sec. II,
  Eq. 5, over every bond set of a tiny torus, with the number of clusters of
  each bond set counted by a caller-supplied labeling function.

Notation: Potts energy H = -J sum delta(s_i, s_j) (Eq. 1), n_eq = number of
lattice bonds joining equal spins, so H = -J n_eq and the Boltzmann weight is
exp(K n_eq) with K = beta J.  For q = 2 in the +-1 Ising convention
H = -J sum sigma_i sigma_j = -J (2 n_eq - E) with E = 2N bonds, i.e.
K_potts = 2 K_ising.
"""
import itertools
import math

import numpy as np


# ---------------------------------------------------------------------------
# Brute-force enumeration
# ---------------------------------------------------------------------------
def _torus_bonds(Lx, Ly):
    """List of (i, j) for the 2N nearest-neighbour bonds of a periodic torus."""
    bonds = []
    for y in range(Ly):
        for x in range(Lx):
            i = y * Lx + x
            bonds.append((i, y * Lx + (x + 1) % Lx))
            bonds.append((i, ((y + 1) % Ly) * Lx + x))
    return bonds


def enumerate_potts(Lx, Ly, q):
    """All q^N states of the periodic Lx x Ly torus.

    Returns (n_eq int64[q^N], counts int64[q^N, q]) with counts[:, k] the number
    of sites in state k.  Memory is q^N * N bytes: keep q^N <= ~2^20."""
    N = Lx * Ly
    n_states = q ** N
    if n_states > (1 << 22):
        raise ValueError("too many states for brute force")
    idx = np.arange(n_states, dtype=np.int64)
    spins = np.empty((n_states, N), dtype=np.int8)
    for site in range(N):
        spins[:, site] = idx % q
        idx //= q
    n_eq = np.zeros(n_states, dtype=np.int64)
    for i, j in _torus_bonds(Lx, Ly):
        n_eq += spins[:, i] == spins[:, j]
    counts = np.stack([(spins == k).sum(axis=1) for k in range(q)], axis=1).astype(np.int64)
    return n_eq, counts


def _cubic_bonds(X, Y, Z):
    """List of (i, j) for the 3N bonds of a periodic X x Y x Z box, site
    i = (z Y + y) X + x, each site bonded to its +x, +y, +z neighbour (for a
    side of 2 the two bonds between a pair are distinct bonds)."""
    bonds = []
    for z in range(Z):
        for y in range(Y):
            for x in range(X):
                i = (z * Y + y) * X + x
                bonds.append((i, (z * Y + y) * X + (x + 1) % X))
                bonds.append((i, (z * Y + (y + 1) % Y) * X + x))
                bonds.append((i, (((z + 1) % Z) * Y + y) * X + x))
    return bonds


def enumerate_potts_3d(X, Y, Z, q):
    """All q^N states of the periodic X x Y x Z simple-cubic box; same
    returns as enumerate_potts."""
    N = X * Y * Z
    n_states = q ** N
    if n_states > (1 << 22):
        raise ValueError("too many states for brute force")
    idx = np.arange(n_states, dtype=np.int64)
    spins = np.empty((n_states, N), dtype=np.int8)
    for site in range(N):
        spins[:, site] = idx % q
        idx //= q
    n_eq = np.zeros(n_states, dtype=np.int64)
    for i, j in _cubic_bonds(X, Y, Z):
        n_eq += spins[:, i] == spins[:, j]
    counts = np.stack([(spins == k).sum(axis=1) for k in range(q)], axis=1).astype(np.int64)
    return n_eq, counts


def moments_from_states(n_eq, counts, K, q):
    """Exact Boltzmann averages at coupling K (Potts delta convention):
    <n_eq>, <n_eq^2>, and for q = 2 <|M|>, <M^2> with M = n_0 - n_1."""
    n = n_eq.astype(np.float64)
    logw = K * n
    w = np.exp(logw - logw.max())
    Z = w.sum()
    out = {"n_eq": float((w * n).sum() / Z), "n_eq2": float((w * n * n).sum() / Z)}
    if q == 2:
        M = (counts[:, 0] - counts[:, 1]).astype(np.float64)
        out["absM"] = float((w * np.abs(M)).sum() / Z)
        out["M2"] = float((w * M * M).sum() / Z)
    return out


# ---------------------------------------------------------------------------
# Transfer matrix density of states
# ---------------------------------------------------------------------------
def potts_dos(Lx, Ly, q):
    """Exact g(n) = number of spin states with n_eq = n on the Lx x Ly torus.

    Row transfer matrix over the q^Lx row configurations, with the running
    count of equal bonds as an extra index.  Counts stay exact in float64
    while q^(Lx*Ly) < 2^53."""
    R = q ** Lx
    if q ** (Lx * Ly) >= 2 ** 53:
        raise ValueError("state count exceeds exact float64 range")
    rows = np.array(list(itertools.product(range(q), repeat=Lx)), dtype=np.int64)[:, ::-1]
    # equal horizontal bonds inside a row (periodic in x)
    h = np.zeros(R, dtype=np.int64)
    for x in range(Lx):
        h += rows[:, x] == rows[:, (x + 1) % Lx]
    # equal vertical bonds between row a (below) and row b (above)
    v = np.zeros((R, R), dtype=np.int64)
    for x in range(Lx):
        v += rows[:, None, x] == rows[None, :, x]
    Emax = 2 * Lx * Ly
    # S[a0, E, b]: weight of partial configurations with first row a0, current row b
    S = np.zeros((R, Emax + 1, R), dtype=np.float64)
    S[np.arange(R), h, np.arange(R)] = 1.0
    step = v + h[None, :]                    # adding row c above row b adds v(b,c) + h(c)
    for _ in range(Ly - 1):
        new = np.zeros_like(S)
        for e in range(0, 2 * Lx + 1):
            Me = (step == e).astype(np.float64)
            if not Me.any():
                continue
            prod = S.reshape(R * (Emax + 1), R) @ Me
            prod = prod.reshape(R, Emax + 1, R)
            new[:, e:, :] += prod[:, : Emax + 1 - e, :]
        S = new
    # close the torus: vertical bonds between the last row b and the first row a0
    g = np.zeros(Emax + 1, dtype=np.float64)
    for a0 in range(R):
        for e in range(0, Lx + 1):
            sel = v[:, a0] == e
            if not sel.any():
                continue
            part = S[a0][:, sel].sum(axis=1)
            g[e:] += part[: Emax + 1 - e]
    return np.rint(g).astype(np.int64)


def dos_moments(g, K):
    """<n>, <n^2> and the normalised distribution P(n) from a density of states."""
    n = np.arange(g.size, dtype=np.float64)
    with np.errstate(divide="ignore"):
        logw = np.where(g > 0, np.log(np.maximum(g, 1)) + K * n, -np.inf)
    w = np.exp(logw - logw[np.isfinite(logw)].max())
    Z = w.sum()
    P = w / Z
    return {"n_eq": float((P * n).sum()), "n_eq2": float((P * n * n).sum()), "P": P}


# ---------------------------------------------------------------------------
# Exact finite-torus Ising partition function (Kaufman 1949)
# ---------------------------------------------------------------------------
def ising_torus_logZ(m, n, K, mp=None):
    """ln Z of the Ising model H = -J sum sigma_i sigma_j on an m x n torus at
    K = beta J, in mpmath arithmetic.

    Kaufman's result: Z = 1/2 (2 sinh 2K)^(mn/2) (Z1 + Z2 + Z3 + Z4) with
      Z1 = prod_{r=0}^{n-1} 2 cosh(m g_{2r+1} / 2)
      Z2 = prod_{r=0}^{n-1} 2 sinh(m g_{2r+1} / 2)
      Z3 = prod_{r=0}^{n-1} 2 cosh(m g_{2r} / 2)
      Z4 = prod_{r=0}^{n-1} 2 sinh(m g_{2r} / 2)
    where cosh g_l = cosh 2K coth 2K - cos(pi l / n) for l >= 1 and
    g_0 = 2K + ln tanh K (which changes sign at the critical point)."""
    if mp is None:
        import mpmath as mp
    K = mp.mpf(K)
    c = mp.cosh(2 * K) * mp.coth(2 * K)

    def gam(l):
        if l % (2 * n) == 0:
            return 2 * K + mp.log(mp.tanh(K))
        return mp.acosh(c - mp.cos(mp.pi * l / n))

    Z1 = Z2 = Z3 = Z4 = mp.mpf(1)
    for r in range(n):
        go = gam(2 * r + 1)
        ge = gam(2 * r)
        Z1 *= 2 * mp.cosh(m * go / 2)
        Z2 *= 2 * mp.sinh(m * go / 2)
        Z3 *= 2 * mp.cosh(m * ge / 2)
        Z4 *= 2 * mp.sinh(m * ge / 2)
    return (mp.log(mp.mpf(1) / 2) + (m * n / mp.mpf(2)) * mp.log(2 * mp.sinh(2 * K))
            + mp.log(Z1 + Z2 + Z3 + Z4))


def ising_torus_energy_moments(L, K, dps=60):
    """Exact <S>, Var(S) of S = sum sigma_i sigma_j on the L x L torus at K,
    from derivatives of ln Z (high-precision numerical differentiation)."""
    import mpmath as mp
    with mp.workdps(dps):
        f = lambda k: ising_torus_logZ(L, L, k, mp)
        d1 = mp.diff(f, mp.mpf(K), 1)
        d2 = mp.diff(f, mp.mpf(K), 2)
        return float(d1), float(d2)


# ---------------------------------------------------------------------------
# Fortuin-Kasteleyn / random-cluster sum (Sec. II, Eq. 5)
# ---------------------------------------------------------------------------
def fk_sum(Lx, Ly, q, K, n_clusters_of):
    """exp(K E) * sum_b p^|b| (1-p)^(E-|b|) q^C(b) over all 2^E bond sets b of
    the periodic Lx x Ly torus (E = 2 Lx Ly), with p = 1 - exp(-K).

    Bond set b is an integer whose bit 2i is the east bond of site i and bit
    2i+1 its north bond, i.e. exactly the packed mask layout read little-endian;
    ``n_clusters_of(mask)`` gets that packed mask (uint8 array) and returns the
    number of connected components.  The prefactor is exp(K) per lattice bond
    (the product over bonds in Eq. 3 gives one factor e^{beta J} per bond)."""
    N = Lx * Ly
    E = 2 * N
    n_bytes = (N + 3) // 4
    p = -math.expm1(-K)
    total = 0.0
    for b in range(1 << E):
        mask = np.frombuffer(b.to_bytes(n_bytes, "little"), dtype=np.uint8)
        nb = bin(b).count("1")
        C = n_clusters_of(mask)
        total += p ** nb * (1 - p) ** (E - nb) * float(q) ** C
    return math.exp(K * E) * total


def potts_Z_bruteforce(Lx, Ly, q, K):
    n_eq, _ = enumerate_potts(Lx, Ly, q)
    return float(np.exp(K * n_eq.astype(np.float64)).sum())


# ---------------------------------------------------------------------------
# Closed forms quoted by the tests
# ---------------------------------------------------------------------------
def critical_p(q):
    """Self-dual FK bond probability p_c = sqrt(q) / (1 + sqrt(q))."""
    return math.sqrt(q) / (1.0 + math.sqrt(q))


PERC_CLUSTER_DENSITY = (3.0 * math.sqrt(3.0) - 5.0) / 2.0
"""Clusters per site of critical bond percolation on the square lattice
(Ziff, Finch & Adamchik, PRL 79, 3447 (1997))."""
