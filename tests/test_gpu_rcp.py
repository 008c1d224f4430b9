"""The FP64 reciprocal of the WENO5 interface (rcp_newton): the hardware
estimate refined by two Newton-Raphson steps r <- r + r (1 - x r). Each step
squares the relative error of the estimate, and the last one rounds once, so
the result is within one unit in the last place of 1/x for every positive
normal x whose reciprocal is normal (the range the interface calls it on,
1e-290 .. 1e290). Checked against numpy's correctly rounded 1/x."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("rcp") / "librcp_probe.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                           "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "paper_2507_11542_gb300", "csrc"),
                           "-I" + os.path.join(ROOT, "include"), "-o", out,
                           os.path.join(HERE, "probes", "rcp_probe.cu")])
    lib = ctypes.CDLL(out)
    lib.rcp_probe.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong]
    return lib


def test_rcp_newton_is_within_one_ulp(probe):
    import torch
    rng = np.random.default_rng(5)
    n = 1 << 20
    mant = rng.uniform(1.0, 2.0, size=n)
    expo = rng.integers(-960, 961, size=n)
    x = np.ldexp(mant, expo)
    x[:8] = [1.0, 2.0, 1.5, 1e-290, 1e290, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0), 3.0]
    xd = torch.from_numpy(x).cuda()
    rd = torch.empty_like(xd)
    assert probe.rcp_probe(xd.data_ptr(), rd.data_ptr(), n) == 0
    r = rd.cpu().numpy()
    exact = 1.0 / x
    ulps = np.abs(r - exact) / np.spacing(exact)
    print("rcp_newton: max error %.3g ulp, %.4f%% of results not correctly rounded"
          % (ulps.max(), 100.0 * np.mean(r != exact)))
    assert ulps.max() <= 1.0
    assert r[0] == 1.0 and r[1] == 0.5
