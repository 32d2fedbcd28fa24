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


@pytest.mark.gpu
def test_stale_failure_flags_do_not_poison_later_solves():
    """A failure flag left set in a cached control block (as a solve whose
    bounded wait ran out leaves it) must not stop the next solve on that
    block: the single-solve workspace, the batched workspace slices and the
    no-allocation array each start their next solve clean and give the
    oracle's result, with no device error reported."""
    lib = appd.load()
    stream = torch.cuda.current_stream().cuda_stream
    W1 = synth.uniform01(1500, seed=41)                 # single solve (grid kernels)
    sizes = [40, 300, 1000, 77, 1024]                   # batched, one graph per CTA
    Wb = [synth.hash_u32(n, seed=50 + k) for k, n in enumerate(sizes)]
    W3 = synth.hash_u32(900, seed=60)                   # no-allocation entry point
    offs = np.cumsum([0] + [n * n for n in sizes])[:-1].astype(np.int64)
    flat = np.concatenate([w.reshape(-1) for w in Wb]).view(np.int32)

    def run_all():
        M1 = appd.solve(torch.from_numpy(W1).cuda())
        Tb = torch.from_numpy(flat).cuda()
        Mb = appd.solve_batched(Tb, offs, sizes, dts=[appd.U32] * len(sizes))
        T3 = torch.from_numpy(W3.view(np.int32)).cuda()
        M3 = torch.full_like(T3, -1)
        assert lib.appd_solve_noalloc(T3.data_ptr(), 900, appd.U32, M3.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        return M1, Mb, M3

    run_all()                                            # create every workspace
    assert appd.last_device_status() == 0
    appd.debug_mark_failed()
    M1, Mb, M3 = run_all()
    assert appd.last_device_status() == 0
    assert np.array_equal(M1.cpu().numpy().view(np.uint32), oracle.appd(W1).view(np.uint32))
    got = Mb.cpu().numpy().view(np.uint32)
    for k, n in enumerate(sizes):
        o = int(offs[k])
        assert np.array_equal(got[o: o + n * n].reshape(n, n), oracle.appd(Wb[k])), f"graph {k}"
    assert np.array_equal(M3.cpu().numpy().view(np.uint32), oracle.appd(W3))
