"""The batched path's autotuner: it searches the documented candidate grid,
installs the winner, caches it per GPU, reuses the cache without a new search,
and the tuned path stays bit-exact against the oracle."""
import json

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2407_07058_gb300 import appd
from tests.test_gpu_parity import _batch, assert_bits

pytestmark = pytest.mark.gpu


def test_autotune_installs_caches_and_stays_exact(tmp_path):
    cache = tmp_path / "tuning.jsonl"
    try:
        t = appd.batched_autotune(str(cache))
        assert t["ctas_per_sm"] == 1
        assert t["fill_rows"] in (256, 512, 1024, 2048)
        assert t["n_split"] in (512, 1024, 2048, 4096)
        assert t["prim_max"] in (0, 64, 128, 256, 512)
        lines = cache.read_text().splitlines()
        assert len(lines) == 1
        rec = json.loads(lines[0])
        assert (rec["fill_rows"], rec["n_split"], rec["prim_max"]) == (t["fill_rows"], t["n_split"],
                                                                       t["prim_max"])
        assert rec["key"].startswith(torch.cuda.get_device_name(0).replace('"', "_"))
        assert rec["ms"] > 0
        # a second call reads the cache: same answer, no new line
        appd.batched_tuning()
        appd.batched_prim_max()
        assert appd.batched_autotune(str(cache)) == t
        assert len(cache.read_text().splitlines()) == 1
        # the tuned batched path is still exact
        sizes = [int(x) for x in synth.cfg4_sizes(40)] + [t["n_split"] + 3]
        Ws, offs, flat = _batch(sizes, [0] * len(sizes), seed0=4321)
        T = torch.from_numpy(flat.view(np.int32)).cuda()
        M = appd.solve_batched(T, offs, sizes)
        torch.cuda.synchronize()
        assert appd.last_device_status() == 0
        Mh = M.cpu().numpy().view(np.uint32)
        for g in list(range(12)) + [len(sizes) - 1]:
            n = sizes[g]
            got = Mh[offs[g]: offs[g] + n * n].reshape(n, n).view(np.float32)
            assert_bits(got, oracle.appd(Ws[g]), f"graph {g} n={n} tuned {t}")
    finally:
        appd.batched_tuning()
        appd.batched_prim_max()


@pytest.mark.parametrize("prim_max", [0, 64, 512])
def test_batched_warp_prim_limits_stay_exact(prim_max):
    """Every warp-Prim limit gives the oracle's matrices (graphs on both sides
    of each limit, both dtypes, ties)."""
    sizes = [2, 3, 31, 32, 33, 63, 64, 65, 100, 255, 256, 257, 511, 512, 513, 700, 1, 5]
    dts = [g % 2 for g in range(len(sizes))]
    Ws, offs, flat = _batch(sizes, dts, seed0=777)
    try:
        appd.batched_prim_max(prim_max)
        T = torch.from_numpy(flat.view(np.int32)).cuda()
        M = appd.solve_batched(T, offs, sizes, dts=dts)
        torch.cuda.synchronize()
        assert appd.last_device_status() == 0
        Mh = M.cpu().numpy().view(np.uint32)
        for g, n in enumerate(sizes):
            got = Mh[offs[g]: offs[g] + n * n].reshape(n, n).view(Ws[g].dtype)
            assert_bits(got, oracle.appd(Ws[g]), f"graph {g} n={n} prim_max={prim_max}")
    finally:
        appd.batched_prim_max()
