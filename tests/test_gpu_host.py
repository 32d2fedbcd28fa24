"""The host-memory entry points: appd_solve_host (synchronous) and
appd_solve_host_async (pipelined), bit-exact against the oracle, with
several asynchronous calls in flight on pinned buffers."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2407_07058_gb300 import appd
from tests.test_gpu_parity import assert_bits

pytestmark = pytest.mark.gpu


def test_host_async_pipelined_calls():
    sizes = [700, 700, 1000, 333, 700]
    Ws = [synth.uniform01(n, seed=40 + k) if k % 2 == 0 else synth.hash_u32(n, seed=40 + k)
          for k, n in enumerate(sizes)]
    Wh = [torch.from_numpy(W.view(np.int32)).pin_memory() for W in Ws]
    Mh = [torch.empty_like(w).pin_memory() for w in Wh]
    st = torch.cuda.current_stream()
    for k, (w, m) in enumerate(zip(Wh, Mh)):
        dt = appd.F32 if Ws[k].dtype == np.float32 else appd.U32
        appd.solve_host_async_ptr(w.data_ptr(), sizes[k], dt, m.data_ptr(), st)
    appd.solve_host_wait(st)
    st.synchronize()
    assert appd.last_device_status() == 0
    for k, W in enumerate(Ws):
        got = Mh[k].numpy().view(W.dtype)
        assert_bits(got, oracle.appd(W), f"async call {k} n={sizes[k]}")


def test_host_async_then_device_solve_on_the_same_stream():
    W1 = synth.uniform01(900, seed=51)
    W2 = synth.uniform01(900, seed=52)
    w1 = torch.from_numpy(W1).pin_memory()
    m1 = torch.empty_like(w1).pin_memory()
    appd.solve_host_async_ptr(w1.data_ptr(), 900, appd.F32, m1.data_ptr())
    M2 = appd.solve(torch.from_numpy(W2).cuda())          # shares the workspace
    appd.solve_host_wait()
    torch.cuda.current_stream().synchronize()
    assert_bits(m1.numpy(), oracle.appd(W1), "async")
    assert_bits(M2.cpu().numpy(), oracle.appd(W2), "device after async")
    assert_bits(appd.solve_host(W2), oracle.appd(W2), "synchronous host entry")


def test_host_async_steady_state_reuses_buffer_pairs():
    # eight same-size calls: every buffer pair is reused while earlier copies
    # and solves are still in flight (the copy in of call k + 2 follows only
    # the solve of call k, not its copy out)
    n = 2048
    Ws = [synth.uniform01(n, seed=70 + k) if k % 3 else synth.hash_u32(n, seed=70 + k) for k in range(8)]
    Wh = [torch.from_numpy(W.view(np.int32)).pin_memory() for W in Ws]
    Mh = [torch.empty_like(w).pin_memory() for w in Wh]
    st = torch.cuda.current_stream()
    for k, (w, m) in enumerate(zip(Wh, Mh)):
        dt = appd.F32 if Ws[k].dtype == np.float32 else appd.U32
        appd.solve_host_async_ptr(w.data_ptr(), n, dt, m.data_ptr(), st)
    appd.solve_host_wait(st)
    st.synchronize()
    assert appd.last_device_status() == 0
    for k, W in enumerate(Ws):
        assert_bits(Mh[k].numpy().view(W.dtype), oracle.appd(W), f"steady-state call {k}")
