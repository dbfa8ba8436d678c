"""ccl_label_noalloc: labeling for callers that cannot allocate device memory.

Some callers of this library cannot call cudaMalloc when they label:
serving loops that must not stall the device with cudaFree, and programs
whose device memory belongs to another framework's allocator.
ccl_label_noalloc takes its scratch from one fixed device array instead.
This test calls it through the C ABI and checks its labels against the
allocating entry point ccl_label, element by element (integer labels:
bit-exact), on two calls in a row with different grids, so the second call
runs on the scratch the first one left behind; that the calls, once the
first call on the device has set up the array, leave the device's free
memory as it was; and that a grid too large for the fixed array is refused
before anything runs.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

import paper_1105_5804_gb300 as sw

pytestmark = pytest.mark.gpu


def _labels(fn, mask, H, W, periodic):
    lab = torch.full((H * W,), -3, dtype=torch.int32, device="cuda")
    fn(mask, lab, H, W, periodic)
    sw.ccl_status()
    return lab.cpu().numpy()


def test_noalloc_matches_ccl_label_on_two_calls_in_a_row():
    # the first call on a device resolves the scratch array's address; with
    # lazy module loading the driver places the array in device memory then
    tiny = torch.zeros(1, dtype=torch.uint8, device="cuda")
    _labels(sw.ccl_label_noalloc, tiny, 1, 1, True)
    cases = [(2048, 1536, 17, True), (999, 1001, 4, False)]
    for H, W, k, periodic in cases:
        mask = torch.empty(sw.mask_bytes(H * W), dtype=torch.uint8, device="cuda")
        sw.ccl_perc_mask(k, mask, H, W)
        ref = _labels(sw.ccl_label, mask, H, W, periodic)
        lab = torch.full((H * W,), -3, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        used0 = torch.cuda.memory_allocated()
        sw.ccl_label_noalloc(mask, lab, H, W, periodic)
        sw.ccl_status()
        free1, _ = torch.cuda.mem_get_info()
        assert torch.cuda.memory_allocated() == used0
        assert free1 >= free0          # the call took no device memory
        assert np.array_equal(lab.cpu().numpy(), ref)


def test_noalloc_refuses_grids_beyond_its_fixed_scratch():
    H = W = 4096
    assert sw.ccl_workspace_bytes(H, W) > sw.CCL_NOALLOC_SCRATCH_BYTES
    mask = torch.zeros(sw.mask_bytes(H * W), dtype=torch.uint8, device="cuda")
    lab = torch.zeros(H * W, dtype=torch.int32, device="cuda")
    with pytest.raises(sw.SwcclError) as ei:
        sw.ccl_label_noalloc(mask, lab, H, W, True)
    assert ei.value.code == sw.SW_ERR_ARG
    assert "scratch" in str(ei.value)
    assert int(lab.abs().sum()) == 0          # nothing ran
