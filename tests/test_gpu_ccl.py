"""GPU parity of the stand-alone labeling path against the oracle, through the C ABI.

Masks: critical percolation (generated on the GPU by ccl_perc_mask and
compared bit for bit with the oracle's), numpy random masks at several
densities, image bonds.  Shapes span one tile, several tiles, ragged tails
in both directions, single rows and columns, periodic and open boundaries.
Labels must equal the oracle's breadth-first-search labels element by
element (integer work: bit-exact).  At the 4096^2 size of the labeling
workload all 100 seeds are compared in full and checked for the properties
every canonical labeling has.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1105_5804_gb300 as sw
from paper_1105_5804_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (1, 7), (7, 1), (2, 2), (3, 5), (64, 128), (65, 129), (63, 127), (128, 256),
          (200, 300), (1, 1000), (1000, 1), (130, 4), (4, 130), (257, 129), (513, 385)]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu_label(mask_np, H, W, periodic, tile_w=None):
    """Labels through the binding (tile_w None: the build it routes labeling
    to) or through the C ABI of the build with tile_w-wide tiles."""
    m = _dev(mask_np)
    lab = torch.full((H * W,), -7, dtype=torch.int32, device="cuda")
    if tile_w is None:
        sw.ccl_label(m, lab, H, W, periodic)
    else:
        L = sw.lib(tile_w)
        rc = L.ccl_label(ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(lab.data_ptr()), H, W,
                         1 if periodic else 0, None)
        assert rc == 0, L.sw_last_error()
        torch.cuda.synchronize()
    sw.ccl_status()
    return lab.cpu().numpy()


@pytest.mark.parametrize("H,W", SHAPES)
def test_perc_mask_bit_exact(H, W):
    m = torch.zeros(sw.mask_bytes(H * W), dtype=torch.uint8, device="cuda")
    for k in (0, 3, 2 ** 40 + 5):
        sw.ccl_perc_mask(k, m, H, W)
        assert np.array_equal(m.cpu().numpy(), oracle.perc_mask(H, W, k))


@pytest.mark.parametrize("H,W", SHAPES)
@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("p", [0.25, 0.5, 0.62, 0.9, 1.0])
def test_labels_random_masks(H, W, periodic, p):
    mask = inputs.random_mask(H, W, p, seed=H * 7919 + W * 31 + int(100 * p))
    ref, _ = oracle.label(mask, H, W, periodic)
    assert np.array_equal(_gpu_label(mask, H, W, periodic), ref)


# every build's labeling (the binding routes stand-alone labeling to one of
# them), on shapes that are ragged for each tile width
@pytest.mark.parametrize("tile_w", sw.TILE_WIDTHS)
@pytest.mark.parametrize("H,W", [(1, 1), (7, 1), (63, 127), (65, 129), (257, 129), (513, 385), (1000, 999)])
@pytest.mark.parametrize("periodic", [True, False])
def test_labels_every_tile_width(tile_w, H, W, periodic):
    for p in (0.5, 0.62):
        mask = inputs.random_mask(H, W, p, seed=H * 131 + W + int(100 * p))
        ref, _ = oracle.label(mask, H, W, periodic)
        assert np.array_equal(_gpu_label(mask, H, W, periodic, tile_w), ref), (tile_w, p)


def test_labels_empty_and_full_masks():
    for H, W in [(64, 128), (100, 300), (5, 5)]:
        for periodic in (True, False):
            for fill in (0x00, 0xFF):
                mask = np.full(sw.mask_bytes(H * W), fill, dtype=np.uint8)
                ref, _ = oracle.label(mask, H, W, periodic)
                assert np.array_equal(_gpu_label(mask, H, W, periodic), ref)


def _snake(H, W, vertical):
    east = np.zeros((H, W), dtype=np.uint8)
    north = np.zeros((H, W), dtype=np.uint8)
    if not vertical:
        east[:, :-1] = 1
        for y in range(H - 1):
            north[y, W - 1 if y % 2 == 0 else 0] = 1
    else:
        north[:-1, :] = 1
        for x in range(W - 1):
            east[H - 1 if x % 2 == 0 else 0, x] = 1
    return oracle.pack_mask(east.reshape(-1), north.reshape(-1))


def _comb(H, W):
    east = np.zeros((H, W), dtype=np.uint8)
    north = np.zeros((H, W), dtype=np.uint8)
    east[H // 2, :-1] = 1           # spine along one row
    north[:-1, :] = 1               # teeth along every column
    north[H // 2 - 1, 1::2] = 0     # cut odd teeth below the spine
    return oracle.pack_mask(east.reshape(-1), north.reshape(-1))


@pytest.mark.parametrize("H,W", [(300, 260), (260, 300), (1000, 130), (129, 1025)])
@pytest.mark.parametrize("kind", ["snake_h", "snake_v", "comb"])
def test_labels_adversarial_long_paths(H, W, kind):
    """One path that winds through every row (or column) of a multi-tile
    grid -- the worst case for seam merging: one cluster, a chain of hooks
    through every tile -- and a comb whose teeth hang off one spine."""
    mask = _comb(H, W) if kind == "comb" else _snake(H, W, kind == "snake_v")
    for periodic in (True, False):
        ref, n = oracle.label(mask, H, W, periodic)
        if kind != "comb":
            assert n == 1
        for _ in range(3):          # the merge is racy by design: repeat
            assert np.array_equal(_gpu_label(mask, H, W, periodic), ref)


@pytest.mark.parametrize("H,W", [(64, 128), (200, 300), (513, 385), (1000, 999)])
@pytest.mark.parametrize("periodic", [True, False])
def test_labels_perc_and_image_masks(H, W, periodic):
    for k in (1, 2):
        mask = oracle.perc_mask(H, W, k)
        ref, _ = oracle.label(mask, H, W, periodic)
        assert np.array_equal(_gpu_label(mask, H, W, periodic), ref)
    px = inputs.blurred_noise_image(H, W, seed=H + W)
    m = torch.zeros(sw.mask_bytes(H * W), dtype=torch.uint8, device="cuda")
    sw.ccl_bonds_from_pixels(_dev(px.reshape(-1)), m, H, W, periodic)
    om = oracle.bonds_from_pixels(px, periodic)
    assert np.array_equal(m.cpu().numpy(), om)
    ref, _ = oracle.label(om, H, W, periodic)
    assert np.array_equal(_gpu_label(om, H, W, periodic), ref)


def test_label_ws_matches_label_and_reuses_workspace():
    H, W = 777, 555
    ws = torch.empty(sw.ccl_workspace_bytes(H, W), dtype=torch.uint8, device="cuda")
    for k in range(3):
        mask = oracle.perc_mask(H, W, 10 + k)
        ref, _ = oracle.label(mask, H, W, True)
        lab = torch.empty(H * W, dtype=torch.int32, device="cuda")
        sw.ccl_label_ws(_dev(mask), lab, H, W, True, ws)
        sw.ccl_status()
        assert np.array_equal(lab.cpu().numpy(), ref)


def _invariants(lab, mask, H, W):
    """Properties of a canonical labeling that hold at any size (torch on GPU)."""
    N = H * W
    i = torch.arange(N, device="cuda", dtype=torch.int64)
    l64 = lab.long()
    assert bool((l64 <= i).all())
    assert bool((l64 >= 0).all())
    assert torch.equal(lab[l64], lab)
    m = mask.long()
    bits = (m[i >> 2] >> (2 * (i & 3))) & 3
    y, x = i // W, i % W
    e = (bits & 1).bool()
    n = (bits & 2).bool()
    east = y * W + (x + 1) % W
    north = ((y + 1) % H) * W + x
    assert torch.equal(lab[e], lab[east[e]])
    assert torch.equal(lab[n], lab[north[n]])
    return int((l64 == i).sum())


def _oracle_perc_labels(k, H, W):
    """The oracle's mask of seed k and its canonical labels (runs in a worker
    thread: the oracle's C calls release the interpreter lock)."""
    om = oracle.perc_mask(H, W, k)
    ref, n = oracle.label(om, H, W, True)
    return om, ref, n


def test_labeling_workload_4096_seeds():
    """Critical percolation on the periodic 4096 x 4096 lattice, seeds 0..99,
    every seed element by element against the oracle (mask and labels), and
    every seed for the invariants of a canonical labeling, with the number of
    roots equal to the oracle's cluster count (a wrong join of two clusters
    keeps every other invariant); the mean cluster density is near
    (3 sqrt3 - 5)/2."""
    import concurrent.futures as cf
    import os
    H = W = 4096
    seeds = list(range(100))
    mask = torch.empty(sw.mask_bytes(H * W), dtype=torch.uint8, device="cuda")
    lab = torch.empty(H * W, dtype=torch.int32, device="cuda")
    dens = []
    workers = max(2, min(16, (os.cpu_count() or 2)))
    with cf.ThreadPoolExecutor(workers) as pool:
        futs = {k: pool.submit(_oracle_perc_labels, k, H, W) for k in seeds[:workers]}
        for k in seeds:
            sw.ccl_perc_mask(k, mask, H, W)
            sw.ccl_label(mask, lab, H, W, True)
            sw.ccl_status()
            om, ref, n = futs.pop(k).result()
            nxt = k + workers
            if nxt < len(seeds):
                futs[nxt] = pool.submit(_oracle_perc_labels, nxt, H, W)
            assert np.array_equal(mask.cpu().numpy(), om), k
            assert np.array_equal(lab.cpu().numpy(), ref), k
            n_roots = _invariants(lab, mask, H, W)
            assert n_roots == n, k
            dens.append(n_roots / (H * W))
    import oracle.exact as exact
    assert abs(np.mean(dens) - exact.PERC_CLUSTER_DENSITY) < 2e-4


def test_label_batch_mixed_grids_equal_oracle_and_single_calls():
    """ccl_label_batch over grids of different sizes, densities and boundary
    conditions (one launch per step for all): every grid's labels equal the
    oracle's and those of ccl_label alone."""
    rng = np.random.default_rng(17)
    shapes = [(1, 1), (3, 5), (64, 256), (65, 257), (200, 300), (1000, 7), (7, 1000), (333, 444), (2048, 300)]
    masks, labs, H, W, P, refs = [], [], [], [], [], []
    for j, (h, w) in enumerate(shapes):
        periodic = bool(j % 2)
        p = float(rng.choice([0.3, 0.5, 0.62, 0.9]))
        m = inputs.random_mask(h, w, p, seed=50 + j)
        masks.append(_dev(m))
        labs.append(torch.full((h * w,), -1, dtype=torch.int32, device="cuda"))
        H.append(h); W.append(w); P.append(periodic)
        refs.append(oracle.label(m, h, w, periodic)[0])
    ws = torch.empty(sw.ccl_batch_workspace_bytes(H, W), dtype=torch.uint8, device="cuda")
    for _ in range(2):            # the second call reuses the workspace
        for lab in labs:
            lab.fill_(-1)
        sw.ccl_label_batch(masks, labs, H, W, P, ws)
        sw.ccl_status()
        for j in range(len(shapes)):
            got = labs[j].cpu().numpy()
            assert np.array_equal(got, refs[j]), shapes[j]
            assert np.array_equal(got, _gpu_label(masks[j].cpu().numpy(), H[j], W[j], P[j]))


def test_label_batch_rejects_small_workspace():
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    m = torch.zeros(sw.mask_bytes(64 * 64), dtype=torch.uint8, device="cuda")
    lab = torch.zeros(64 * 64, dtype=torch.int32, device="cuda")
    with pytest.raises(sw.SwcclError):
        sw.ccl_label_batch([m], [lab], [64], [64], [True], ws)


def test_copy_pixels_2d_windows_and_errors():
    """The upload step of a labeling request: windows of a larger host image
    (pageable and pinned) or device image land packed on the device, and the
    labels of the uploaded window equal those of the packed copy."""
    rng = np.random.default_rng(8)
    big = rng.integers(0, 8, (300, 517)).astype(np.uint8)
    pinned_t = torch.empty((300, 517), dtype=torch.uint8, pin_memory=True)
    pinned = pinned_t.numpy()
    pinned[:] = big
    dev_big = torch.from_numpy(big).cuda()
    for (y, x, H, W) in [(0, 0, 300, 517), (17, 33, 101, 203), (299, 516, 1, 1), (5, 0, 64, 517)]:
        want = np.ascontiguousarray(big[y:y + H, x:x + W]).reshape(-1)
        for src in (big[y:y + H, x:x + W], pinned[y:y + H, x:x + W], dev_big[y:y + H, x:x + W]):
            dst = torch.zeros(H * W, dtype=torch.uint8, device="cuda")
            sw.ccl_copy_pixels_2d(src, dst)
            torch.cuda.synchronize()
            assert np.array_equal(dst.cpu().numpy(), want), (y, x, H, W)
        m = torch.empty(sw.mask_bytes(H * W), dtype=torch.uint8, device="cuda")
        sw.ccl_bonds_from_pixels(dst, m, H, W, False)
        lab = torch.empty(H * W, dtype=torch.int32, device="cuda")
        sw.ccl_label(m, lab, H, W, False)
        ref, _ = oracle.label(oracle.bonds_from_pixels(want.reshape(H, W), False), H, W, False)
        assert np.array_equal(lab.cpu().numpy(), ref)
    dst = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        sw.ccl_copy_pixels_2d(big[:4, :4].T, dst)                     # columns not contiguous
    with pytest.raises(ValueError):
        sw.ccl_copy_pixels_2d(big[:4, :8], dst)                       # dst too small
    L = sw.lib()
    assert L.ccl_copy_pixels_2d(None, 4, ctypes.c_void_p(dst.data_ptr()), 4, 4, 0, None) == sw.SW_ERR_ARG
    assert L.ccl_copy_pixels_2d(ctypes.c_void_p(big.ctypes.data), 3, ctypes.c_void_p(dst.data_ptr()), 4, 4, 0,
                                None) == sw.SW_ERR_ARG                # pitch < W
