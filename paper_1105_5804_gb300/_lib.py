"""ctypes binding of libswccl.so (C ABI in include/swccl.h).

Argument marshalling only: every step of the method runs in the CUDA
kernels of the library.  Device buffers are passed as torch CUDA tensors
(their ``data_ptr()``), streams as ``torch.cuda.Stream`` / raw handles.
There is no fallback: if the library is not built, every call raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libswccl.so")

SW_OK, SW_ERR_ARG, SW_ERR_OOM, SW_ERR_CUDA, SW_ERR_TIMEOUT, SW_ERR_STATE = 0, 1, 2, 3, 4, 5
SW_CONV_AUTO, SW_CONV_POTTS, SW_CONV_ISING = 0, 1, 2
SW_N_PHASES = 5
SW_MODE_STAGED, SW_MODE_FUSED = 0, 1
SW_BATCH_PHASES, SW_BATCH_PERSISTENT = 0, 1
SW_UPDATE_SW, SW_UPDATE_FEW = 0, 1
PHASE_NAMES = ("activate", "local", "merge", "roots", "flip")
SW3_N_PHASES = 4
PHASE_NAMES3 = ("local", "merge", "flip", "advance")


class SwcclError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("swccl error %d: %s" % (code, msg))
        self.code = code


_libs = {}
TILE_WIDTHS = (256, 128, 64)


def _lib_path(tile_w):
    return LIB_PATH if tile_w == 256 else os.path.join(HERE, "_build", "libswccl_w%d.so" % tile_w)


def lib(tile_w=256):
    """The loaded library (the build with labeling tiles tile_w wide: 256,
    or 128 / 64 for batches).  Raises if it has not been built."""
    if tile_w in _libs:
        return _libs[tile_w]
    if tile_w not in TILE_WIDTHS:
        raise ValueError("tile width must be one of %s" % (TILE_WIDTHS,))
    path = _lib_path(tile_w)
    if not os.path.exists(path):
        raise RuntimeError("%s is not built; run __graft_entry__.build() "
                           "or python -m paper_1105_5804_gb300.build" % path)
    L = ctypes.CDLL(path)
    vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        "sw_last_error": ([], ctypes.c_char_p),
        "sw_threshold_for": ([i32, dbl, dbl, i32], u64),
        "sw_create": ([i32, i32, dbl, u64], vp),
        "sw_create_ex": ([i32, i32, dbl, dbl, i32, u64, i32, vp], vp),
        "sw_create_threshold": ([i32, i32, u64, u64, i32, vp], vp),
        "sw_destroy": ([vp], i32),
        "sw_sweep": ([vp, i32], i32),
        "sw_sync": ([vp], i32),
        "sw_observables": ([vp, vp, i32, ctypes.POINTER(i32)], i32),
        "sw_get_spins": ([vp, vp, i32], i32),
        "sw_set_spins": ([vp, vp, i32], i32),
        "sw_sweep_io": ([vp, vp, i32, vp, vp], i32),
        "sw_debug_dump": ([vp, vp, vp, i32], i32),
        "sw_get_info": ([vp, vp], i32),
        "sw_stream": ([vp], vp),
        "sw_set_timing": ([vp, i32], i32),
        "sw_set_mode": ([vp, i32], i32),
        "sw_set_update": ([vp, i32, i32, u64], i32),
        "sw_prob_threshold": ([dbl], u64),
        "sw_phase_times": ([vp, vp, ctypes.POINTER(i64)], i32),
        "ccl_label": ([vp, vp, i32, i32, i32, vp], i32),
        "ccl_workspace_bytes": ([i32, i32], i64),
        "ccl_label_ws": ([vp, vp, i32, i32, i32, vp, i64, vp], i32),
        "ccl_bonds_from_pixels": ([vp, vp, i32, i32, i32, vp], i32),
        "ccl_perc_mask": ([u64, vp, i32, i32, vp], i32),
        "ccl_copy_pixels_2d": ([vp, i64, vp, i32, i32, i32, vp], i32),
        "ccl_label_noalloc": ([vp, vp, i32, i32, i32, vp], i32),
        "ccl_status": ([], i32),
        "sw_probe_philox": ([i64, i32, vp, vp], i32),
        "ccl_batch_workspace_bytes": ([i32, vp, vp], i64),
        "ccl_label_batch": ([i32, vp, vp, vp, vp, vp, vp, i64, vp], i32),
        "sw_batch_create": ([i32, vp, vp, vp, vp, i32, i32, vp], vp),
        "sw_batch_destroy": ([vp], i32),
        "sw_batch_device_bytes": ([i32, vp, vp], i64),
        "sw_batch_create_ws": ([i32, vp, vp, vp, vp, i32, i32, vp, i64, vp], vp),
        "sw_batch_set_graph": ([vp, i32], i32),
        "sw_batch_set_schedule": ([vp, i32, i32], i32),
        "sw_batch_sweep": ([vp, i32], i32),
        "sw_batch_set_barrier_limit": ([vp, ctypes.c_longlong], i32),
        "sw_batch_sync": ([vp], i32),
        "sw_batch_observables": ([vp, i32, vp, i32, ctypes.POINTER(i32)], i32),
        "sw_batch_observables_async": ([vp, i32, vp, i32, ctypes.POINTER(i32)], i32),
        "sw_batch_get_spins": ([vp, i32, vp, i32], i32),
        "sw_batch_info": ([vp, vp], i32),
        "sw_batch_stream": ([vp], vp),
        "sw3_create": ([i32, i32, i32, i32, u64, u64, i32, vp], vp),
        "sw3_create_ex": ([i32, i32, i32, i32, dbl, dbl, i32, u64, i32, vp], vp),
        "sw3_destroy": ([vp], i32),
        "sw3_sweep": ([vp, i32], i32),
        "sw3_sync": ([vp], i32),
        "sw3_observables": ([vp, vp, i32, ctypes.POINTER(i32)], i32),
        "sw3_get_spins": ([vp, vp, i32], i32),
        "sw3_set_spins": ([vp, vp, i32], i32),
        "sw3_labels": ([vp, vp, i32], i32),
        "sw3_stream": ([vp], vp),
        "sw3_get_info": ([vp, vp], i32),
        "sw3_set_timing": ([vp, i32], i32),
        "sw3_phase_times": ([vp, vp, ctypes.POINTER(i64)], i32),
    }
    for name, (args, res) in sig.items():
        if tile_w != 256 and name.startswith("sw3_"):
            continue            # the narrow-tile builds have no simple-cubic kernels
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _libs[tile_w] = L
    return L


def sw_last_error():
    return lib().sw_last_error().decode()


def _check(rc):
    if rc != SW_OK:
        raise SwcclError(rc, sw_last_error())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype, numel=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must have dtype %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if numel is not None and t.numel() < numel:
        raise ValueError("%s needs at least %d elements" % (name, numel))
    return ctypes.c_void_p(t.data_ptr())


def mask_bytes(n_sites):
    return (n_sites + 3) // 4


# ---------------------------------------------------------------------------
# Swendsen-Wang chain
# ---------------------------------------------------------------------------
def sw_threshold_for(q, beta, J=1.0, convention=SW_CONV_AUTO):
    return int(lib().sw_threshold_for(q, beta, J, convention))


def _handle(h):
    if not h:
        raise SwcclError(SW_ERR_ARG, sw_last_error())
    return h


def sw_create(L, q, beta, seed):
    return _handle(lib().sw_create(L, q, beta, seed))


def sw_create_ex(L, q, beta, J, convention, seed, hot_start, stream=0):
    return _handle(lib().sw_create_ex(L, q, beta, J, convention, seed, 1 if hot_start else 0,
                                      _stream(stream) if stream else None))


def sw_create_threshold(L, q, T, seed, hot_start, stream=0):
    return _handle(lib().sw_create_threshold(L, q, T, seed, 1 if hot_start else 0,
                                             _stream(stream) if stream else None))


def sw_destroy(h):
    _shape.pop(h, None)
    _check(lib().sw_destroy(h))


def sw_sweep(h, n):
    _check(lib().sw_sweep(h, n))


def sw_sync(h):
    _check(lib().sw_sync(h))


def sw_get_info(h):
    info = np.zeros(8, dtype=np.int64)
    _check(lib().sw_get_info(h, info.ctypes.data))
    keys = ("L", "q", "T", "seed", "sweeps", "obs_capacity", "tile_h", "tile_w")
    return {k: int(v) for k, v in zip(keys, info)}


_shape = {}   # handle -> (L, q): fixed for a handle's life, dropped by sw_destroy


def _Lq(h):
    v = _shape.get(h)
    if v is None:
        i = sw_get_info(h)
        v = _shape[h] = (i["L"], i["q"])
    return v


def sw_observables(h, max_sweeps=4096):
    q = _Lq(h)[1]
    out = np.zeros((max_sweeps, 1 + q), dtype=np.int64)
    n = ctypes.c_int(0)
    _check(lib().sw_observables(h, out.ctypes.data, max_sweeps, ctypes.byref(n)))
    return out[: n.value]


def sw_get_spins(h, out=None):
    """Current spins: into ``out`` (a host numpy int8 array or a CUDA int8
    tensor) or into a new numpy array."""
    N = _Lq(h)[0] ** 2
    if out is None or isinstance(out, np.ndarray):
        a = np.empty(N, dtype=np.int8) if out is None else out
        if a.dtype != np.int8 or a.size < N or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a contiguous int8 array of %d elements" % N)
        _check(lib().sw_get_spins(h, a.ctypes.data, 0))
        return a
    import torch
    _check(lib().sw_get_spins(h, _dev(out, torch.int8, N, "out"), 1))
    return out


def sw_set_spins(h, src):
    import torch
    N = _Lq(h)[0] ** 2
    if isinstance(src, torch.Tensor) and src.is_cuda:
        _check(lib().sw_set_spins(h, _dev(src, torch.int8, N, "src"), 1))
    else:
        a = np.ascontiguousarray(src, dtype=np.int8).reshape(-1)
        if a.size != N:
            raise ValueError("need %d spins" % N)
        _check(lib().sw_set_spins(h, a.ctypes.data, 0))


def sw_sweep_io(h, n, inp=None, obs_out=None, out=None):
    """One asynchronous pipeline step (see include/swccl.h): inp (CUDA int8
    tensor of L*L spins or None) replaces the spins if valid, n sweeps run,
    their observables go to obs_out (int64 tensor of n x (1+q), pinned host
    or CUDA, or None) and the spins to out (CUDA int8 tensor or None).
    Nothing waits for the device."""
    import torch
    L, q = _Lq(h)
    N = L * L
    ip = _dev(inp, torch.int8, N, "inp") if inp is not None else None
    op = _dev(out, torch.int8, N, "out") if out is not None else None
    if obs_out is not None:
        if obs_out.dtype != torch.int64 or not obs_out.is_contiguous() or obs_out.numel() < n * (q + 1):
            raise ValueError("obs_out must be a contiguous int64 tensor of at least n x (1 + q) elements")
        if not obs_out.is_cuda and not obs_out.is_pinned():
            raise ValueError("obs_out must be pinned host memory or a CUDA tensor")
        obs_ptr = ctypes.c_void_p(obs_out.data_ptr())
    else:
        obs_ptr = None
    _check(lib().sw_sweep_io(_handle(h), ip, n, obs_ptr, op))


def sw_debug_dump(h, mask_out=None, labels_out=None):
    """(mask, labels) of the last sweep, as numpy arrays, or into CUDA tensors."""
    import torch
    N = _Lq(h)[0] ** 2
    if mask_out is None and labels_out is None:
        m = np.empty(mask_bytes(N), dtype=np.uint8)
        lab = np.empty(N, dtype=np.int32)
        _check(lib().sw_debug_dump(h, m.ctypes.data, lab.ctypes.data, 0))
        return m, lab
    mp = _dev(mask_out, torch.uint8, mask_bytes(N), "mask_out") if mask_out is not None else None
    lp = _dev(labels_out, torch.int32, N, "labels_out") if labels_out is not None else None
    _check(lib().sw_debug_dump(h, mp, lp, 1))
    return mask_out, labels_out


def sw_stream(h):
    return int(lib().sw_stream(h) or 0)


def sw_set_mode(h, mode):
    _check(lib().sw_set_mode(h, mode))


def sw_set_update(h, update, ell=0, P=0):
    _check(lib().sw_set_update(h, update, ell, P))


def sw_prob_threshold(p):
    return int(lib().sw_prob_threshold(p))


def sw_set_timing(h, enable):
    _check(lib().sw_set_timing(h, 1 if enable else 0))


def sw_phase_times(h):
    ms = np.zeros(SW_N_PHASES, dtype=np.float64)
    n = ctypes.c_int64(0)
    _check(lib().sw_phase_times(h, ms.ctypes.data, ctypes.byref(n)))
    return dict(zip(PHASE_NAMES, ms.tolist())), int(n.value)


# ---------------------------------------------------------------------------
# Simple-cubic chains
# ---------------------------------------------------------------------------
def sw3_create(X, Y, Z, q, T, seed, hot_start=False, stream=0):
    return _handle(lib().sw3_create(X, Y, Z, q, T, seed, 1 if hot_start else 0,
                                    _stream(stream) if stream else None))


def sw3_create_ex(X, Y, Z, q, beta, J=1.0, convention=SW_CONV_AUTO, seed=0, hot_start=False, stream=0):
    return _handle(lib().sw3_create_ex(X, Y, Z, q, beta, J, convention, seed, 1 if hot_start else 0,
                                       _stream(stream) if stream else None))


def sw3_destroy(h):
    _check(lib().sw3_destroy(h))


def sw3_sweep(h, n):
    _check(lib().sw3_sweep(h, n))


def sw3_sync(h):
    _check(lib().sw3_sync(h))


def sw3_get_info(h):
    info = np.zeros(8, dtype=np.int64)
    _check(lib().sw3_get_info(h, info.ctypes.data))
    keys = ("X", "Y", "Z", "q", "T", "seed", "sweeps", "obs_cap")
    return {k: int(v) for k, v in zip(keys, info)}


def _n3(h):
    i = sw3_get_info(h)
    return i["X"] * i["Y"] * i["Z"]


def sw3_observables(h, max_sweeps=4096):
    q = sw3_get_info(h)["q"]
    out = np.zeros((max_sweeps, 1 + q), dtype=np.int64)
    n = ctypes.c_int(0)
    _check(lib().sw3_observables(h, out.ctypes.data, max_sweeps, ctypes.byref(n)))
    return out[: n.value]


def sw3_get_spins(h, out=None):
    """Current spins into ``out`` (host int8 array or CUDA int8 tensor) or a new array."""
    N = _n3(h)
    if out is None or isinstance(out, np.ndarray):
        a = np.empty(N, dtype=np.int8) if out is None else out
        if a.dtype != np.int8 or a.size < N or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a contiguous int8 array of %d elements" % N)
        _check(lib().sw3_get_spins(h, a.ctypes.data, 0))
        return a
    import torch
    _check(lib().sw3_get_spins(h, _dev(out, torch.int8, N, "out"), 1))
    return out


def sw3_set_spins(h, src):
    import torch
    N = _n3(h)
    if isinstance(src, torch.Tensor) and src.is_cuda:
        _check(lib().sw3_set_spins(h, _dev(src, torch.int8, N, "src"), 1))
    else:
        a = np.ascontiguousarray(src, dtype=np.int8).reshape(-1)
        if a.size != N:
            raise ValueError("need %d spins" % N)
        _check(lib().sw3_set_spins(h, a.ctypes.data, 0))


def sw3_labels(h, out=None):
    """Canonical labels of the last sweep's clusters (numpy, or into a CUDA int32 tensor)."""
    N = _n3(h)
    if out is None:
        a = np.empty(N, dtype=np.int32)
        _check(lib().sw3_labels(h, a.ctypes.data, 0))
        return a
    import torch
    _check(lib().sw3_labels(h, _dev(out, torch.int32, N, "out"), 1))
    return out


def sw3_stream(h):
    return lib().sw3_stream(h)


def sw3_set_timing(h, enable):
    _check(lib().sw3_set_timing(h, 1 if enable else 0))


def sw3_phase_times(h):
    ms = np.zeros(SW3_N_PHASES, dtype=np.float64)
    n = ctypes.c_int64(0)
    _check(lib().sw3_phase_times(h, ms.ctypes.data, ctypes.byref(n)))
    return dict(zip(PHASE_NAMES3, ms.tolist())), int(n.value)


# ---------------------------------------------------------------------------
# Stand-alone labeling
# ---------------------------------------------------------------------------
# The labeling calls below (ccl_label, ccl_label_ws, ccl_label_noalloc,
# ccl_label_batch and their workspace sizes) go to the build with 128-wide
# tiles: it labels 2048^2 to 8192^2 grids 2-6 % faster than the 256-wide
# build the sweep uses (twice the tiles fill the last wave of CTAs better).
# Both builds export the same C ABI and give the same labels.
CCL_TILE_W = 128


def _ccl():
    return lib(CCL_TILE_W)


def ccl_label(bond_mask, labels, H, W, periodic, stream=None):
    import torch
    N = H * W
    L = _ccl()
    _bcheck(L, L.ccl_label(_dev(bond_mask, torch.uint8, mask_bytes(N), "bond_mask"),
                           _dev(labels, torch.int32, N, "labels"), H, W, 1 if periodic else 0,
                           _stream(stream)))
    return labels


def ccl_workspace_bytes(H, W):
    return int(_ccl().ccl_workspace_bytes(H, W))


def ccl_label_ws(bond_mask, labels, H, W, periodic, workspace, stream=None):
    import torch
    N = H * W
    L = _ccl()
    _bcheck(L, L.ccl_label_ws(_dev(bond_mask, torch.uint8, mask_bytes(N), "bond_mask"),
                              _dev(labels, torch.int32, N, "labels"), H, W, 1 if periodic else 0,
                              _dev(workspace, torch.uint8, None, "workspace"), workspace.numel(),
                              _stream(stream)))
    return labels


def ccl_bonds_from_pixels(px, mask, H, W, periodic, stream=None):
    import torch
    N = H * W
    _check(lib().ccl_bonds_from_pixels(_dev(px, torch.uint8, N, "px"),
                                       _dev(mask, torch.uint8, mask_bytes(N), "mask"), H, W,
                                       1 if periodic else 0, _stream(stream)))
    return mask


def ccl_copy_pixels_2d(src, dst, stream=None):
    """Upload an image window into the CUDA uint8 tensor ``dst`` (H*W
    elements): ``src`` is a 2-D numpy uint8 array (a view of a larger image,
    rows contiguous) or a 2-D CUDA tensor with unit column stride.  The copy
    is asynchronous on ``stream``; keep ``src`` alive until it has run."""
    import torch
    if isinstance(src, torch.Tensor) and src.is_cuda:
        if src.dim() != 2 or src.dtype != torch.uint8 or src.stride(1) != 1:
            raise ValueError("src must be a 2-D uint8 CUDA tensor with unit column stride")
        H, W = src.shape
        ptr, pitch, dev = src.data_ptr(), src.stride(0), 1
    else:
        if not isinstance(src, np.ndarray) or src.ndim != 2 or src.dtype != np.uint8 or src.strides[1] != 1:
            raise ValueError("src must be a 2-D uint8 numpy array with contiguous rows")
        H, W = src.shape
        ptr, pitch, dev = src.ctypes.data, src.strides[0], 0
    _check(lib().ccl_copy_pixels_2d(ctypes.c_void_p(ptr), pitch, _dev(dst, torch.uint8, H * W, "dst"), H, W, dev,
                                    _stream(stream)))


def ccl_perc_mask(k, mask, H, W, stream=None):
    import torch
    _check(lib().ccl_perc_mask(k, _dev(mask, torch.uint8, mask_bytes(H * W), "mask"), H, W,
                               _stream(stream)))
    return mask


CCL_NOALLOC_SCRATCH_BYTES = 64 << 20


def ccl_label_noalloc(bond_mask, labels, H, W, periodic, stream=None):
    """ccl_label without any allocation (fixed device scratch array); see
    include/swccl.h for who needs it and its size limit."""
    import torch
    N = H * W
    L = _ccl()
    _bcheck(L, L.ccl_label_noalloc(_dev(bond_mask, torch.uint8, mask_bytes(N), "bond_mask"),
                                   _dev(labels, torch.int32, N, "labels"), H, W, 1 if periodic else 0,
                                   _stream(stream)))
    return labels


def sw_probe_philox(calls_per_thread, blocks, sink, stream=None):
    """Enqueue the Philox-only throughput kernel (measurement helper)."""
    import torch
    _check(lib().sw_probe_philox(calls_per_thread, blocks, _dev(sink, torch.int32, blocks * 256, "sink"),
                                 _stream(stream)))


def ccl_status():
    """Device-side failures of labeling calls, in every loaded build."""
    for L in list(_libs.values()):
        _bcheck(L, L.ccl_status())


# ---------------------------------------------------------------------------
# Batches of chains
# ---------------------------------------------------------------------------
_batch_lib = {}     # batch handle -> tile width of the library that made it


def _blib(b):
    return lib(_batch_lib.get(b, 256))


def sw_batch_create(L, q, beta, seed, convention=SW_CONV_AUTO, hot_start=False, stream=0, tile_w=256):
    """L, q, beta, seed: sequences of equal length (one entry per chain).
    tile_w: width of the labeling tiles (256, 128 or 64; the library built
    for it runs the batch)."""
    n = len(L)
    La = np.ascontiguousarray(L, dtype=np.int32)
    qa = np.ascontiguousarray(q, dtype=np.int32)
    ba = np.ascontiguousarray(beta, dtype=np.float64)
    sa = np.ascontiguousarray(seed, dtype=np.uint64)
    if not (qa.size == ba.size == sa.size == n):
        raise ValueError("L, q, beta, seed must have equal lengths")
    h = lib(tile_w).sw_batch_create(n, La.ctypes.data, qa.ctypes.data, ba.ctypes.data, sa.ctypes.data,
                                    convention, 1 if hot_start else 0, _stream(stream) if stream else None)
    if not h:
        raise SwcclError(SW_ERR_ARG, lib(tile_w).sw_last_error().decode())
    _batch_lib[h] = tile_w
    return h


def sw_batch_device_bytes(L, q, tile_w=256):
    La = np.ascontiguousarray(L, dtype=np.int32)
    qa = np.ascontiguousarray(q, dtype=np.int32)
    if La.size != qa.size:
        raise ValueError("L and q need one entry per chain")
    n = int(lib(tile_w).sw_batch_device_bytes(La.size, La.ctypes.data, qa.ctypes.data))
    if n < 0:
        raise SwcclError(SW_ERR_ARG, lib(tile_w).sw_last_error().decode())
    return n


def sw_batch_create_ws(L, q, beta, seed, workspace, convention=SW_CONV_AUTO, hot_start=False, stream=0,
                       tile_w=256):
    """As sw_batch_create with the batch's device memory taken from
    `workspace` (a CUDA uint8 tensor of at least sw_batch_device_bytes(L, q)
    bytes, 256-byte aligned), which must outlive the batch."""
    import torch
    n = len(L)
    La = np.ascontiguousarray(L, dtype=np.int32)
    qa = np.ascontiguousarray(q, dtype=np.int32)
    ba = np.ascontiguousarray(beta, dtype=np.float64)
    sa = np.ascontiguousarray(seed, dtype=np.uint64)
    if not (La.size == qa.size == ba.size == sa.size == n):
        raise ValueError("L, q, beta, seed need one entry per chain")
    ws = _dev(workspace, torch.uint8, None, "workspace")
    h = lib(tile_w).sw_batch_create_ws(n, La.ctypes.data, qa.ctypes.data, ba.ctypes.data, sa.ctypes.data,
                                       convention, 1 if hot_start else 0, ws, workspace.numel(), _stream(stream))
    if not h:
        raise SwcclError(SW_ERR_ARG, lib(tile_w).sw_last_error().decode())
    _batch_lib[h] = tile_w
    return h


def sw_batch_set_graph(b, enable):
    _bcheck(_blib(b), _blib(b).sw_batch_set_graph(b, 1 if enable else 0))


def sw_batch_destroy(b):
    L = _blib(b)
    _batch_lib.pop(b, None)
    _bcheck(L, L.sw_batch_destroy(b))


def _bcheck(L, rc):
    if rc != SW_OK:
        raise SwcclError(rc, L.sw_last_error().decode())


def sw_batch_set_schedule(b, schedule, blocks_per_sm=0):
    _bcheck(_blib(b), _blib(b).sw_batch_set_schedule(b, schedule, blocks_per_sm))


def sw_batch_set_barrier_limit(b, cycles):
    _bcheck(_blib(b), _blib(b).sw_batch_set_barrier_limit(b, int(cycles)))


def sw_batch_sweep(b, n):
    _bcheck(_blib(b), _blib(b).sw_batch_sweep(b, n))


def sw_batch_sync(b):
    _bcheck(_blib(b), _blib(b).sw_batch_sync(b))


def sw_batch_info(b):
    info = np.zeros(8, dtype=np.int64)
    _bcheck(_blib(b), _blib(b).sw_batch_info(b, info.ctypes.data))
    keys = ("chains", "sites", "tiles", "sweeps", "schedule", "persistent_blocks", "graph", "obs_capacity")
    out = {k: int(v) for k, v in zip(keys, info)}
    out["tile_w"] = _batch_lib.get(b, 256)
    return out


def sw_batch_observables(b, replica, q, max_sweeps=4096):
    out = np.zeros((max_sweeps, 1 + q), dtype=np.int64)
    n = ctypes.c_int(0)
    _bcheck(_blib(b), _blib(b).sw_batch_observables(b, replica, out.ctypes.data, max_sweeps, ctypes.byref(n)))
    return out[: n.value]


def sw_batch_observables_async(b, replica, q, out):
    """Enqueue the unread observable rows of chain `replica` into `out` (a
    pinned host or CUDA int64 tensor of shape (rows, 1 + q)); returns the
    number of rows that will arrive when the batch's stream gets there."""
    import torch
    if not isinstance(out, torch.Tensor) or out.dtype != torch.int64 or not out.is_contiguous() or \
            out.dim() != 2 or out.shape[1] != 1 + q or not (out.is_cuda or out.is_pinned()):
        raise ValueError("out must be a contiguous int64 (rows, 1 + q) tensor in pinned host or device memory")
    n = ctypes.c_int(0)
    _bcheck(_blib(b), _blib(b).sw_batch_observables_async(b, replica, ctypes.c_void_p(out.data_ptr()), out.shape[0],
                                            ctypes.byref(n)))
    return n.value


def sw_batch_get_spins(b, replica, L, out=None):
    if out is None or isinstance(out, np.ndarray):
        a = np.empty(L * L, dtype=np.int8) if out is None else out
        _bcheck(_blib(b), _blib(b).sw_batch_get_spins(b, replica, a.ctypes.data, 0))
        return a
    import torch
    _bcheck(_blib(b), _blib(b).sw_batch_get_spins(b, replica, _dev(out, torch.int8, L * L, "out"), 1))
    return out


def sw_batch_stream(b):
    return int(_blib(b).sw_batch_stream(b) or 0)


# ---------------------------------------------------------------------------
# Batched labeling
# ---------------------------------------------------------------------------
def ccl_batch_workspace_bytes(H, W):
    Ha = np.ascontiguousarray(H, dtype=np.int32)
    Wa = np.ascontiguousarray(W, dtype=np.int32)
    return int(_ccl().ccl_batch_workspace_bytes(len(Ha), Ha.ctypes.data, Wa.ctypes.data))


def ccl_label_batch(masks, labels, H, W, periodic, workspace, stream=None):
    """masks / labels: sequences of CUDA tensors (uint8 packed masks, int32
    labels); H, W, periodic: sequences of ints."""
    import torch
    n = len(masks)
    Ha = np.ascontiguousarray(H, dtype=np.int32)
    Wa = np.ascontiguousarray(W, dtype=np.int32)
    Pa = np.ascontiguousarray([1 if p else 0 for p in periodic], dtype=np.int32)
    if not (len(labels) == Ha.size == Wa.size == Pa.size == n):
        raise ValueError("masks, labels, H, W, periodic must have equal lengths")
    mp = (ctypes.c_void_p * max(n, 1))()
    lp = (ctypes.c_void_p * max(n, 1))()
    for j in range(n):
        N = int(Ha[j]) * int(Wa[j])
        mp[j] = _dev(masks[j], torch.uint8, mask_bytes(N), "masks[%d]" % j).value
        lp[j] = _dev(labels[j], torch.int32, N, "labels[%d]" % j).value
    L = _ccl()
    _bcheck(L, L.ccl_label_batch(n, mp, lp, Ha.ctypes.data, Wa.ctypes.data, Pa.ctypes.data,
                                 _dev(workspace, torch.uint8, None, "workspace"), workspace.numel(),
                                 _stream(stream)))
    return labels
