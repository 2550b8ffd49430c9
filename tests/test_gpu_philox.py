"""The device Philox-4x32-10 against the CPU oracle's and cuRAND's."""

import ctypes
import os
import subprocess

import numpy as np
import pytest
import torch

from gpu_common import built, need_gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _curand_lib():
    out = os.path.join(HERE, "_build", "libcurand_ref.so")
    src = os.path.join(HERE, "curand_ref.cu")
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(out), exist_ok=True)
        subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                               "-Xcompiler", "-fPIC", "-o", out, src])
    L = ctypes.CDLL(out)
    L.curand_ref_philox.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong]
    return L


@pytest.mark.gpu
def test_device_philox_matches_oracle_and_curand(orc):
    need_gpu()
    built()
    from paper_2404_08364_gb300 import _fw
    rng = np.random.default_rng(5)
    n = 1 << 20
    inp = rng.integers(0, 2**32, size=(n, 6), dtype=np.uint64).astype(np.uint32)
    inp[:1000, 0] = np.arange(1000)          # walk-style counters: small t,
    inp[:1000, 1:4] = 0                      # small query ids
    d_in = torch.from_numpy(inp.view(np.int32)).cuda()
    d_out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    _fw.check(_fw.lib().fw_philox(ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr()), n,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    ours = d_out.cpu().numpy().view(np.uint32)
    ref = torch.empty_like(d_out)
    assert _curand_lib().curand_ref_philox(d_in.data_ptr(), ref.data_ptr(), n) == 0
    assert np.array_equal(ours, ref.cpu().numpy().view(np.uint32))
    for i in list(range(0, 1000, 37)) + list(range(1000, n, n // 50)):
        assert orc.philox4x32_10(inp[i, :4], inp[i, 4:]) == [int(x) for x in ours[i]]
