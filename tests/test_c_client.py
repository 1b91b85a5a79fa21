"""The C ABI used from plain C (tests/c/abi_client.c, built with gcc against
include/td.h and libtd.so): it builds without a GPU; on the GPU its results
match the CPU FP64 oracle."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build(tmp_path):
    from paper_2603_06010_b300 import build
    lib = build.build()
    exe = str(tmp_path / "abi_client")
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", "c", "abi_client.c"), "-o", exe,
           "-L", libdir, "-ltd", f"-Wl,-rpath,{libdir}", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_client_builds(tmp_path):
    assert os.path.exists(_build(tmp_path))


@pytest.mark.gpu
def test_c_client_matches_oracle(tmp_path):
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2603_06010_b300 import inputs
    exe = _build(tmp_path)
    n, K = 1500, 37
    mask = np.ones(n, np.uint8)
    mask[400:620] = 0
    acf = inputs.acf_from_psd(n, 2048.0)
    R = inputs.noise_residuals(n, 2048.0, K, 4711, mask=mask)
    inp, outp = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        np.array([n, K, 1], np.int64).tofile(f)
        acf.astype(np.float64).tofile(f)
        mask.tofile(f)
        np.ascontiguousarray(R, np.float32).tofile(f)
    r = subprocess.run([exe, str(inp), str(outp)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    out = np.fromfile(outp, np.float64)
    logL, chi2, logdet, same = out[:K], out[K:2 * K], out[2 * K], out[2 * K + 1]
    assert same == 1.0, "segment saved and loaded through the C ABI gave different bits"
    o = oracle.OracleSegment(acf, mask)
    exp_chi = o.chi2(R)
    assert abs(logdet - o.logdet) <= 1e-9 * abs(o.logdet)
    assert np.max(np.abs(chi2 - exp_chi) / exp_chi) <= 1e-7
    assert np.max(np.abs(logL - oracle.loglike_from_chi2(exp_chi, o.logdet, o.n_kept))) <= 1e-3
