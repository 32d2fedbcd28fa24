"""Failure detection without a GPU fault.

Device waits are bounded: a wait that runs out records APPD_ERR_TIMEOUT in
the device status word and the kernel returns, so the context stays usable.
The probe below makes one CTA of a cooperative launch skip the barrier (a
flag that nothing sets); nothing faults or hangs."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2407_07058_gb300 import appd


@pytest.mark.gpu
def test_bounded_wait_reports_timeout_and_context_survives():
    assert appd.last_device_status() == 0
    appd.probe_bounded_wait(200)
    torch.cuda.synchronize()
    assert appd.last_device_status() == 6          # APPD_ERR_TIMEOUT, then cleared
    assert appd.last_device_status() == 0
    W = synth.hash_u32(777, seed=3)
    M = appd.solve(torch.from_numpy(W.view(np.int32)).cuda())
    torch.cuda.synchronize()
    assert appd.last_device_status() == 0
    assert np.array_equal(M.cpu().numpy().view(np.uint32), oracle.appd(W))


@pytest.mark.gpu
def test_solve_after_timeout_without_reading_status_is_still_correct():
    # the abort word is per launch: a timeout of an earlier launch does not
    # poison later solves even before the status is read
    appd.probe_bounded_wait(100)
    W = synth.uniform01(513, seed=4)
    M = appd.solve(torch.from_numpy(W).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(M.cpu().numpy().view(np.uint32), oracle.appd(W).view(np.uint32))
    assert appd.last_device_status() == 6
    assert appd.last_device_status() == 0


def test_host_side_rejections_need_no_gpu():
    with pytest.raises(ValueError):
        appd.solve(torch.zeros((4, 4)))              # CPU tensor: no CPU path
    with pytest.raises(ValueError):
        appd.solve(torch.zeros((4, 5)))
    lib = appd.load()
    assert lib.appd_probe_bounded_wait(0, None) == 1
    assert lib.appd_probe_bounded_wait(20000, None) == 1
    assert lib.appd_batched_tuning(3, 256, 2048) == 1
    assert lib.appd_batched_tuning(1, 100, 2048) == 1
