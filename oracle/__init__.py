"""Serial CPU oracle for the Swendsen-Wang sweep and bond-graph labeling.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA library (``paper_1105_5804_gb300``) and imports
nothing from it.

The arithmetic lives in ``swccl_oracle.c`` (plain serial C, one function per
step of the method, each citing the passage of Weigel, arXiv:1105.5804 it
follows).  This module only marshals numpy arrays into it.  Exact reference
results used to pin the oracle (enumeration, transfer matrix, the finite
torus Ising partition function) live in :mod:`oracle.exact`.

Conventions (paper silent; fixed here and restated in the design notes):
site i = y*W + x, east = (x+1, y), north = (x, y+1); packed mask with site i
in bits 2*(i&3) (east) and 2*(i&3)+1 (north) of byte i>>2.
"""
import ctypes
import numpy as np

from . import build as _build

TAG_BOND, TAG_FLIP, TAG_INIT, TAG_PERC, TAG_SEED, TAG_BOND3 = 0, 1, 2, 3, 4, 5
CONV_AUTO, CONV_POTTS, CONV_ISING = 0, 1, 2

_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_philox4x32_10.restype = None
        L.or_coupling_K.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.or_coupling_K.restype = ctypes.c_double
        L.or_threshold.argtypes = [ctypes.c_double]
        L.or_threshold.restype = ctypes.c_uint64
        L.or_flip_state.argtypes = [ctypes.c_uint32, ctypes.c_int]
        L.or_flip_state.restype = ctypes.c_int
        L.or_init_spins.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
        L.or_init_spins.restype = None
        L.or_activate.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                  ctypes.c_uint64, ctypes.c_void_p]
        L.or_activate.restype = None
        L.or_perc_mask.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p]
        L.or_perc_mask.restype = None
        L.or_bonds_from_pixels.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p]
        L.or_bonds_from_pixels.restype = None
        L.or_label.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.or_label.restype = ctypes.c_int64
        L.or_flip.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                              ctypes.c_void_p, ctypes.c_void_p]
        L.or_flip.restype = None
        L.or_observables.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.or_observables.restype = None
        L.or_sweep.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.or_sweep.restype = ctypes.c_int
        L.or_chain.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                               ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        L.or_chain.restype = ctypes.c_int
        L.or_few_seed.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64]
        L.or_few_seed.restype = ctypes.c_int64
        L.or_few_sweep.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                   ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p]
        L.or_few_sweep.restype = ctypes.c_int
        L.or_few_chain.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                   ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_void_p]
        L.or_few_chain.restype = ctypes.c_int
        i3 = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.or3_init_spins.argtypes = i3 + [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
        L.or3_init_spins.restype = None
        L.or3_activate.argtypes = i3 + [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_void_p]
        L.or3_activate.restype = None
        L.or3_label.argtypes = i3 + [ctypes.c_void_p, ctypes.c_void_p]
        L.or3_label.restype = ctypes.c_int64
        L.or3_observables.argtypes = i3 + [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.or3_observables.restype = None
        L.or3_sweep.argtypes = i3 + [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.or3_sweep.restype = ctypes.c_int
        L.or3_chain.argtypes = i3 + [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        L.or3_chain.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def mask_bytes(n_sites: int) -> int:
    return (n_sites + 3) // 4


# --------------------------------------------------------------------------
# Generator, coupling, threshold
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 block function: 4 counter words, 2 key words -> 4 words."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def coupling_K(q: int, beta: float, J: float = 1.0, convention: int = CONV_AUTO) -> float:
    return lib().or_coupling_K(q, beta, J, convention)


def threshold(K: float) -> int:
    """T = min(2^32, floor(p 2^32)) with p = 1 - exp(-K)."""
    return int(lib().or_threshold(K))


def flip_state(w: int, q: int) -> int:
    return lib().or_flip_state(int(w) & 0xFFFFFFFF, q)


# --------------------------------------------------------------------------
# Steps of the sweep
# --------------------------------------------------------------------------
def init_spins(L: int, q: int, seed: int, hot: bool) -> np.ndarray:
    s = np.zeros(L * L, dtype=np.int8)
    lib().or_init_spins(L, q, seed, 1 if hot else 0, _ptr(s))
    return s


def activate(L: int, spins, seed: int, sweep: int, T: int) -> np.ndarray:
    spins = _c(spins, np.int8).reshape(-1)
    assert spins.size == L * L
    m = np.zeros(mask_bytes(L * L), dtype=np.uint8)
    lib().or_activate(L, _ptr(spins), seed, sweep, T, _ptr(m))
    return m


def perc_mask(H: int, W: int, k: int) -> np.ndarray:
    m = np.zeros(mask_bytes(H * W), dtype=np.uint8)
    lib().or_perc_mask(H, W, k, _ptr(m))
    return m


def bonds_from_pixels(px, periodic: bool) -> np.ndarray:
    px = _c(px, np.uint8)
    H, W = px.shape
    m = np.zeros(mask_bytes(H * W), dtype=np.uint8)
    lib().or_bonds_from_pixels(H, W, 1 if periodic else 0, _ptr(px), _ptr(m))
    return m


def label(mask, H: int, W: int, periodic: bool):
    """Canonical (minimum site index) labels by breadth-first search.

    Returns (labels int32[H*W], number of clusters)."""
    mask = _c(mask, np.uint8).reshape(-1)
    assert mask.size >= mask_bytes(H * W)
    lab = np.empty(H * W, dtype=np.int32)
    n = lib().or_label(H, W, 1 if periodic else 0, _ptr(mask), _ptr(lab))
    if n < 0:
        raise MemoryError("oracle labeling: allocation failed")
    return lab, int(n)


def flip(labels, q: int, seed: int, sweep: int) -> np.ndarray:
    labels = _c(labels, np.int32).reshape(-1)
    s = np.empty(labels.size, dtype=np.int8)
    lib().or_flip(labels.size, q, seed, sweep, _ptr(labels), _ptr(s))
    return s


def observables(L: int, q: int, spins) -> np.ndarray:
    spins = _c(spins, np.int8).reshape(-1)
    out = np.zeros(1 + q, dtype=np.int64)
    lib().or_observables(L, q, _ptr(spins), _ptr(out))
    return out


def sweep(L: int, q: int, T: int, seed: int, sweep_index: int, spins):
    """One sweep.  Returns (new spins, mask, canonical labels, observables)."""
    s = _c(spins, np.int8).reshape(-1).copy()
    m = np.zeros(mask_bytes(L * L), dtype=np.uint8)
    lab = np.empty(L * L, dtype=np.int32)
    obs = np.zeros(1 + q, dtype=np.int64)
    rc = lib().or_sweep(L, q, T, seed, sweep_index, _ptr(s), _ptr(m), _ptr(lab), _ptr(obs))
    if rc != 0:
        raise MemoryError("oracle sweep failed")
    return s, m, lab, obs


def chain(L: int, q: int, T: int, seed: int, sweep0: int, n_sweeps: int, spins):
    """n_sweeps sweeps from sweep0.  Returns (final spins, obs int64[n_sweeps, 1+q])."""
    s = _c(spins, np.int8).reshape(-1).copy()
    obs = np.zeros((n_sweeps, 1 + q), dtype=np.int64)
    rc = lib().or_chain(L, q, T, seed, sweep0, n_sweeps, _ptr(s), _ptr(obs))
    if rc != 0:
        raise MemoryError("oracle chain failed")
    return s, obs


# --------------------------------------------------------------------------
# Few-cluster update (Sec. III, variant (c) of the single-cluster algorithm)
# --------------------------------------------------------------------------
def few_seed(L: int, ell: int, seed: int, sweep_index: int, b: int) -> int:
    """Seed site of block b of the ell x ell block grid at this sweep."""
    return int(lib().or_few_seed(L, ell, seed, sweep_index, b))


def few_sweep(L: int, q: int, T: int, P: int, ell: int, seed: int, sweep_index: int, spins):
    """One few-cluster sweep (flip threshold P).  Returns (new spins, mask,
    canonical labels, observables)."""
    s = _c(spins, np.int8).reshape(-1).copy()
    m = np.zeros(mask_bytes(L * L), dtype=np.uint8)
    lab = np.empty(L * L, dtype=np.int32)
    obs = np.zeros(1 + q, dtype=np.int64)
    rc = lib().or_few_sweep(L, q, T, P, ell, seed, sweep_index, _ptr(s), _ptr(m), _ptr(lab), _ptr(obs))
    if rc != 0:
        raise ValueError("oracle few-cluster sweep failed (ell must divide L)")
    return s, m, lab, obs


def few_chain(L: int, q: int, T: int, P: int, ell: int, seed: int, sweep0: int, n_sweeps: int, spins):
    """n_sweeps few-cluster sweeps from sweep0.  Returns (final spins, obs)."""
    s = _c(spins, np.int8).reshape(-1).copy()
    obs = np.zeros((n_sweeps, 1 + q), dtype=np.int64)
    rc = lib().or_few_chain(L, q, T, P, ell, seed, sweep0, n_sweeps, _ptr(s), _ptr(obs))
    if rc != 0:
        raise ValueError("oracle few-cluster chain failed (ell must divide L)")
    return s, obs


# --------------------------------------------------------------------------
# Simple-cubic lattice X x Y x Z (periodic), site i = (z*Y + y)*X + x; bond
# mask one byte per site, bit d = bond to the +x / +y / +z neighbour
# --------------------------------------------------------------------------
def init_spins3(X: int, Y: int, Z: int, q: int, seed: int, hot: bool) -> np.ndarray:
    s = np.empty(X * Y * Z, dtype=np.int8)
    lib().or3_init_spins(X, Y, Z, q, seed, int(bool(hot)), _ptr(s))
    return s


def activate3(X: int, Y: int, Z: int, spins, seed: int, sweep_index: int, T: int) -> np.ndarray:
    spins = _c(spins, np.int8).reshape(-1)
    m = np.zeros(X * Y * Z, dtype=np.uint8)
    lib().or3_activate(X, Y, Z, _ptr(spins), seed, sweep_index, T, _ptr(m))
    return m


def label3(mask, X: int, Y: int, Z: int):
    """Canonical labels of a 3D bond mask.  Returns (labels, number of clusters)."""
    mask = _c(mask, np.uint8).reshape(-1)
    lab = np.empty(X * Y * Z, dtype=np.int32)
    n = lib().or3_label(X, Y, Z, _ptr(mask), _ptr(lab))
    if n < 0:
        raise MemoryError("oracle 3D labeling failed")
    return lab, int(n)


def observables3(X: int, Y: int, Z: int, q: int, spins) -> np.ndarray:
    spins = _c(spins, np.int8).reshape(-1)
    out = np.zeros(1 + q, dtype=np.int64)
    lib().or3_observables(X, Y, Z, q, _ptr(spins), _ptr(out))
    return out


def sweep3(X: int, Y: int, Z: int, q: int, T: int, seed: int, sweep_index: int, spins):
    """One 3D sweep.  Returns (new spins, mask, canonical labels, observables)."""
    s = _c(spins, np.int8).reshape(-1).copy()
    m = np.zeros(X * Y * Z, dtype=np.uint8)
    lab = np.empty(X * Y * Z, dtype=np.int32)
    obs = np.zeros(1 + q, dtype=np.int64)
    if lib().or3_sweep(X, Y, Z, q, T, seed, sweep_index, _ptr(s), _ptr(m), _ptr(lab), _ptr(obs)) != 0:
        raise MemoryError("oracle 3D sweep failed")
    return s, m, lab, obs


def chain3(X: int, Y: int, Z: int, q: int, T: int, seed: int, sweep0: int, n_sweeps: int, spins):
    """n_sweeps 3D sweeps from sweep0.  Returns (final spins, obs)."""
    s = _c(spins, np.int8).reshape(-1).copy()
    obs = np.zeros((n_sweeps, 1 + q), dtype=np.int64)
    if lib().or3_chain(X, Y, Z, q, T, seed, sweep0, n_sweeps, _ptr(s), _ptr(obs)) != 0:
        raise MemoryError("oracle 3D chain failed")
    return s, obs


# --------------------------------------------------------------------------
# Mask conveniences for tests (unpacking only; no method arithmetic)
# --------------------------------------------------------------------------
def unpack_mask(mask, n_sites: int):
    """Return (east, north) uint8 arrays of length n_sites from a packed mask."""
    mask = np.asarray(mask, dtype=np.uint8).reshape(-1)
    i = np.arange(n_sites)
    b = mask[i >> 2] >> (2 * (i & 3)).astype(np.uint8)
    return (b & 1).astype(np.uint8), ((b >> 1) & 1).astype(np.uint8)


def pack_mask(east, north) -> np.ndarray:
    east = np.asarray(east, dtype=np.uint8).reshape(-1)
    north = np.asarray(north, dtype=np.uint8).reshape(-1)
    n = east.size
    m = np.zeros(mask_bytes(n), dtype=np.uint8)
    i = np.arange(n)
    bits = ((east & 1) | ((north & 1) << 1)).astype(np.uint8) << (2 * (i & 3)).astype(np.uint8)
    np.bitwise_or.at(m, i >> 2, bits)
    return m
