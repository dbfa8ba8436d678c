"""GB300-native Swendsen-Wang cluster updates and bond-graph labeling.

Python binding of libswccl.so: the C ABI declared in ``include/swccl.h``
(Weigel, arXiv:1105.5804: bond activation, cluster identification, cluster
flip).  All computation runs in the library's sm_103a kernels; PyTorch only
supplies device memory and streams.  Importing this package does not load the
library; the first call does, and raises if it was not built.
"""
from ._lib import (  # noqa: F401
    SW_OK, SW_ERR_ARG, SW_ERR_OOM, SW_ERR_CUDA, SW_ERR_TIMEOUT, SW_ERR_STATE,
    SW_CONV_AUTO, SW_CONV_POTTS, SW_CONV_ISING, SW_N_PHASES, PHASE_NAMES, SW_MODE_STAGED, SW_MODE_FUSED,
    SwcclError, lib, mask_bytes,
    sw_last_error, sw_threshold_for, sw_create, sw_create_ex, sw_create_threshold, sw_destroy,
    sw_sweep, sw_sync, sw_observables, sw_get_spins, sw_set_spins, sw_sweep_io, sw_debug_dump, sw_get_info,
    sw_stream, sw_set_timing, sw_phase_times, sw_set_mode, SW_UPDATE_SW, SW_UPDATE_FEW, sw_set_update,
    sw_prob_threshold,
    ccl_label, ccl_workspace_bytes, ccl_label_ws, ccl_bonds_from_pixels, ccl_perc_mask, ccl_status,
    ccl_copy_pixels_2d,
    ccl_label_noalloc, CCL_NOALLOC_SCRATCH_BYTES, sw_probe_philox,
    SW_BATCH_PHASES, SW_BATCH_PERSISTENT, TILE_WIDTHS, sw_batch_create, sw_batch_destroy, sw_batch_set_schedule,
    sw_batch_set_barrier_limit, sw_batch_device_bytes, sw_batch_create_ws, sw_batch_set_graph, sw_batch_sweep,
    sw_batch_sync, sw_batch_info, sw_batch_observables, sw_batch_observables_async, sw_batch_get_spins,
    sw_batch_stream,
    ccl_batch_workspace_bytes, ccl_label_batch,
    SW3_N_PHASES, PHASE_NAMES3, sw3_create, sw3_create_ex, sw3_destroy, sw3_sweep, sw3_sync, sw3_get_info,
    sw3_observables, sw3_get_spins, sw3_set_spins, sw3_labels, sw3_stream, sw3_set_timing, sw3_phase_times,
)


class SwendsenWang:
    """Owning wrapper of one chain handle (``sw_create_ex``)."""

    def __init__(self, L, q, beta, seed, J=1.0, convention=SW_CONV_AUTO, hot_start=False,
                 threshold=None, stream=0):
        if threshold is None:
            self.h = sw_create_ex(L, q, beta, J, convention, seed, hot_start, stream)
        else:
            self.h = sw_create_threshold(L, q, threshold, seed, hot_start, stream)
        self.L, self.q = L, q

    def sweep(self, n=1):
        sw_sweep(self.h, n)

    def set_mode(self, mode):
        sw_set_mode(self.h, mode)

    def observables(self, max_sweeps=4096):
        return sw_observables(self.h, max_sweeps)

    def spins(self, out=None):
        return sw_get_spins(self.h, out)

    def set_spins(self, src):
        sw_set_spins(self.h, src)

    def debug_dump(self):
        return sw_debug_dump(self.h)

    def info(self):
        return sw_get_info(self.h)

    @property
    def stream(self):
        return sw_stream(self.h)

    def close(self):
        if self.h:
            sw_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
